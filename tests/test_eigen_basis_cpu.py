"""The facts the mixed set-up's eigen estimate rests on, checked on the CPU.

Sec. 3.2 takes the Chebyshev bounds from the Ritz values of an Arnoldi run on
B^{-1} A_l.  The FP32 set-up forms the same Ritz values from another basis of
the same Krylov space: the Chebyshev polynomials of 2M - I (M = B^{-1} A_l)
applied to the start vector, projected through its Gram matrix.  Two facts
make that exact and well conditioned:

* Rayleigh-Ritz does not depend on the basis: with K = Q R (Q Arnoldi's
  orthonormal basis), (K^T K)^{-1} K^T M K = R^{-1} (Q^T M Q) R, a similarity
  of Arnoldi's Hessenberg matrix;
* for symmetric Gauss-Seidel B - A = L D^{-1} L^T is positive semi-definite,
  so the spectrum of M lies in (0, 1], where the Chebyshev polynomials of
  2x - 1 stay bounded by 1.

The Chebyshev-basis computation below is a restatement written for this test;
it shares nothing with the CUDA code.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import gmg_oracle as O
from streamer_inputs import make_inputs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _chebyshev_basis_ritz(matvec, v0, steps):
    """Largest Ritz value of K_steps(M, v0) from the basis v_1 = (2M - I) v_0,
    v_{j+1} = 2 (2M - I) v_j - v_{j-1}, with every vector rounded to FP32,
    as the GPU keeps them."""
    v = [(v0 / np.linalg.norm(v0)).astype(np.float32)]
    v.append((2.0 * matvec(v[0]) - v[0]).astype(np.float32))
    for j in range(1, steps):
        v.append((4.0 * matvec(v[j]) - 2.0 * v[j] - v[j - 1]).astype(np.float32))
    K = np.stack([x.astype(np.float64) for x in v])
    G = K @ K.T
    # M v_0 = (v_1 + v_0)/2, M v_j = (v_{j+1} + 2 v_j + v_{j-1})/4
    Mm = np.zeros((steps + 1, steps))
    Mm[0, 0] = Mm[1, 0] = 0.5
    for j in range(1, steps):
        Mm[j - 1, j], Mm[j, j], Mm[j + 1, j] = 0.25, 0.5, 0.25
    R = np.linalg.cholesky(G[:steps, :steps]).T
    Ri = np.linalg.inv(R)
    H = Ri.T @ (G[:steps, :] @ Mm) @ Ri
    return float(np.max(np.linalg.eigvals(H).real)), H, G


@pytest.mark.parametrize("n,workload", [(16, "twochannel512"), (32, "twochannel512"), (16, "channel256")])
def test_chebyshev_basis_gives_arnoldis_ritz_value(n, workload):
    inp = make_inputs(workload, n=n)
    p = O.OracleParams()
    grid = O.Grid(n, n, n)
    levels = [(grid, np.asarray(inp["a"], np.float64))]
    while levels[-1][0].nx > 8:
        g, a = levels[-1]
        levels.append((g.coarser(), O.coarsen_level(a, p)))
    for g, a in levels:
        def matvec(x, g=g, a=a):
            y = O.apply_operator(g, a, x.reshape(g.shape).astype(np.float64))
            return O.smoother_preconditioner(g, a, y, "sgs").ravel()
        _, _, lam_arnoldi = O.estimate_eig_bounds(g, a, p)
        lam, H, G = _chebyshev_basis_ritz(matvec, O.hash_start_vector(g.size), p.eig_steps)
        assert lam == pytest.approx(lam_arnoldi, rel=1e-8)
        # the projected matrix is Arnoldi's Hessenberg matrix up to rounding
        assert np.abs(np.tril(H, -2)).max() < 1e-12 * np.abs(H).max()
        # every new vector keeps a resolvable part outside the previous ones
        R = np.linalg.cholesky(G[:-1, :-1]).T
        assert (np.diag(R) ** 2 / np.diag(G[:-1, :-1])).min() > 1e-2


def test_chebyshev_basis_reproduces_a_planted_spectrum():
    """On a diagonal M with known eigenvalues in (0, 1] the 10-dimensional
    projection finds the largest one (the basis spans the space when there
    are only 10 distinct eigenvalues)."""
    lam = np.array([0.03, 0.11, 0.2, 0.35, 0.5, 0.62, 0.71, 0.83, 0.9, 0.97])
    d = np.repeat(lam, 40)
    v0 = np.random.default_rng(5).standard_normal(d.size)
    got, _, _ = _chebyshev_basis_ritz(lambda x: d * x.astype(np.float64), v0, 9)
    assert got <= 0.97 + 1e-6
    got10, _, _ = _chebyshev_basis_ritz(lambda x: d * x.astype(np.float64), v0, 10)
    assert got10 == pytest.approx(0.97, rel=1e-5)


@pytest.mark.parametrize("seed,contrast", [(1, 1.0), (2, 1e3), (3, 1e5)])
def test_symmetric_gauss_seidel_spectrum_lies_in_zero_one(seed, contrast):
    """Dense B^{-1} A of the red-black SSOR sweep on a small grid with a
    random coefficient: real eigenvalues, all in (0, 1]."""
    shape = (4, 5, 6)
    rng = np.random.default_rng(seed)
    a = np.exp(rng.uniform(0, np.log(contrast), size=shape)) if contrast > 1 else np.ones(shape)
    g = O.Grid(shape[2], shape[1], shape[0])
    n = g.size
    M = np.zeros((n, n))
    A = O.dense_operator(g, a)
    for c in range(n):
        M[:, c] = O.sgs_redblack(g, a, A[:, c].reshape(shape)).ravel()
    ev = np.linalg.eigvals(M)
    assert np.abs(ev.imag).max() < 1e-10
    assert ev.real.min() > 0.0
    assert ev.real.max() <= 1.0 + 1e-12

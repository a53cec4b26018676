"""Pins of the FP64 oracle against things other than itself.

Each test fixes one part of the oracle by something the paper or the
mathematics determines independently: a hand-derived operator (golden file),
closed-form spectra (DCT-II / DST-II), a manufactured solution, a 1-D
tridiagonal reduction, dense linear algebra at 8^3, the recursion for the
V-cycle matrix M_l of Appendix A, the Chebyshev polynomial of eq. (qntn),
and finite differences for the adjoint.
"""
import os

import numpy as np
import pytest
import scipy.fft
import scipy.linalg

from oracle import gmg_oracle as O
from streamer_inputs import random_coefficient, random_field, make_inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid(shape, l=(1.0, 1.0, 1.0)):
    nz, ny, nx = shape
    return O.Grid(nx, ny, nz, *l)


# ---------------------------------------------------------------------------
# Operator eq. (e18) + boundary conditions
# ---------------------------------------------------------------------------


def _read_golden(name):
    rows = {}
    A = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            vals = [float(v) for v in vals]
            if key == "A":
                A.append(vals)
            else:
                rows[key] = vals
    rows["A"] = np.array(A)
    return rows


def test_operator_matches_hand_derived_golden():
    g = _read_golden("operator_2x1x2.txt")
    nx, ny, nz = (int(v) for v in g["shape"])
    grid = O.Grid(nx, ny, nz)
    a = np.array(g["a"]).reshape(grid.shape)
    np.testing.assert_allclose(O.dense_operator(grid, a), g["A"], rtol=0, atol=1e-12)
    gb, gt = g["g"]
    b = O.assemble_rhs(grid, a, np.zeros(grid.shape), gb, gt)
    np.testing.assert_allclose(b.ravel(), g["b"], rtol=0, atol=1e-12)
    phi = np.array(g["phi"]).reshape(grid.shape)
    ex, ey, ez = O.field_from_potential(grid, phi, gb, gt)
    np.testing.assert_allclose(ex.ravel(), g["Ex"], atol=1e-12)
    np.testing.assert_allclose(ey.ravel(), g["Ey"], atol=1e-12)
    np.testing.assert_allclose(ez.ravel(), g["Ez"], atol=1e-12)


def test_pointwise_operator_matches_golden_and_whole_array():
    """apply_operator_at (the cell-by-cell form used at full size): on the
    hand-derived 2x1x2 golden grid its columns on unit vectors are the golden
    matrix; on a ragged anisotropic grid it equals the whole-array operator at
    every cell, walls, plates and corners included."""
    g = _read_golden("operator_2x1x2.txt")
    nx, ny, nz = (int(v) for v in g["shape"])
    grid = O.Grid(nx, ny, nz)
    a = np.array(g["a"]).reshape(grid.shape)
    cells = [(k, j, i) for k in range(nz) for j in range(ny) for i in range(nx)]
    cols = []
    for n in range(grid.size):
        e = np.zeros(grid.size)
        e[n] = 1.0
        cols.append(O.apply_operator_at(grid, a, e.reshape(grid.shape), cells))
    np.testing.assert_allclose(np.array(cols).T, g["A"], rtol=0, atol=1e-12)
    shape = (5, 3, 7)
    grid = _grid(shape, (0.7, 1.3, 0.4))
    a = random_coefficient(3, shape, contrast=1e3)
    x = random_field(4, shape)
    cells = [(k, j, i) for k in range(shape[0]) for j in range(shape[1]) for i in range(shape[2])]
    np.testing.assert_allclose(O.apply_operator_at(grid, a, x, cells), O.apply_operator(grid, a, x).ravel(),
                               rtol=1e-13, atol=1e-13 * np.abs(O.apply_operator(grid, a, x)).max())


def test_pointwise_field_matches_golden_and_whole_array():
    """field_at against the golden field of the 2x1x2 grid and against
    field_from_potential on a ragged anisotropic grid, every cell."""
    g = _read_golden("operator_2x1x2.txt")
    nx, ny, nz = (int(v) for v in g["shape"])
    grid = O.Grid(nx, ny, nz)
    phi = np.array(g["phi"]).reshape(grid.shape)
    gb, gt = g["g"]
    cells = [(k, j, i) for k in range(nz) for j in range(ny) for i in range(nx)]
    e = O.field_at(grid, phi, gb, gt, cells)
    np.testing.assert_allclose(e[:, 0], g["Ex"], atol=1e-12)
    np.testing.assert_allclose(e[:, 1], g["Ey"], atol=1e-12)
    np.testing.assert_allclose(e[:, 2], g["Ez"], atol=1e-12)
    shape = (4, 5, 6)
    grid = _grid(shape, (0.9, 1.1, 0.3))
    phi = random_field(5, shape)
    cells = [(k, j, i) for k in range(shape[0]) for j in range(shape[1]) for i in range(shape[2])]
    ref = np.stack([c.ravel() for c in O.field_from_potential(grid, phi, 0.3, 2.0)], axis=1)
    np.testing.assert_allclose(O.field_at(grid, phi, 0.3, 2.0, cells), ref, rtol=1e-14, atol=1e-12)


def test_operator_symmetric_positive_definite():
    shape = (5, 6, 4)
    grid = _grid(shape, (0.7, 1.3, 1.0))
    a = random_coefficient(1, shape, contrast=1e3)
    A = O.dense_operator(grid, a)
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-12 * np.abs(A).max())
    lam = np.linalg.eigvalsh(A)
    assert lam.min() > 0.0
    np.linalg.cholesky(A)
    # D - N splitting and diagonal agree with the dense matrix
    np.testing.assert_allclose(np.diag(A), O.diagonal(grid, a).ravel(), rtol=1e-14)
    x = random_field(2, shape)
    np.testing.assert_allclose(O.apply_operator(grid, a, x),
                               O.diagonal(grid, a) * x - O.neighbour_sum(grid, a, x), rtol=1e-12, atol=1e-10)


def _spectral_symbols(grid):
    """Eigenvalues of the constant-coefficient operator: DCT-II modes (Neumann)
    in x, y and DST-II modes (Dirichlet through the ghost -phi) in z, each
    (4/h^2) sin^2(pi m / (2n)); m = 0..n-1 for cosines, 1..n for sines."""
    lx = 4.0 / grid.hx**2 * np.sin(np.pi * np.arange(grid.nx) / (2 * grid.nx)) ** 2
    ly = 4.0 / grid.hy**2 * np.sin(np.pi * np.arange(grid.ny) / (2 * grid.ny)) ** 2
    lz = 4.0 / grid.hz**2 * np.sin(np.pi * np.arange(1, grid.nz + 1) / (2 * grid.nz)) ** 2
    return lz[:, None, None] + ly[None, :, None] + lx[None, None, :]


def _spectral_apply(grid, x, inverse=False):
    lam = _spectral_symbols(grid)
    c = scipy.fft.dctn(x, type=2, axes=(1, 2), norm="ortho")
    c = scipy.fft.dst(c, type=2, axis=0, norm="ortho")
    c = c / lam if inverse else c * lam
    c = scipy.fft.idst(c, type=2, axis=0, norm="ortho")
    return scipy.fft.idctn(c, type=2, axes=(1, 2), norm="ortho")


def test_constant_coefficient_operator_is_diagonal_in_dct_dst_basis():
    shape = (6, 10, 8)
    grid = _grid(shape, (1.0, 2.0, 0.5))
    a = np.ones(shape)
    x = random_field(3, shape)
    np.testing.assert_allclose(O.apply_operator(grid, a, x), _spectral_apply(grid, x), rtol=1e-11, atol=1e-9)


def test_fgmres_const32_matches_spectral_exact_solution():
    """Workload const32 (a = 1): the solve agrees with the exact discrete
    solution from the DCT/DST diagonalisation within cond(A) * rtol."""
    inp = make_inputs("const32")
    a, f = inp["a"], inp["f"]
    grid = _grid(a.shape)
    params = O.OracleParams()
    phi, info, _ = O.solve(params, a, f)
    assert info.converged and info.true_rel_residual < 1e-8
    b = O.assemble_rhs(grid, a, f, params.phi_bottom, params.phi_top)
    exact = _spectral_apply(grid, b, inverse=True)
    lam = _spectral_symbols(grid)
    cond = lam.max() / lam.min()
    assert np.linalg.norm(phi - exact) / np.linalg.norm(exact) < cond * 1e-8
    assert np.linalg.norm(phi - exact) / np.linalg.norm(exact) < 1e-7


def test_one_dimensional_reduction_matches_tridiagonal_solve():
    """a = a(z), f = f(z): phi is independent of x, y and equals the solution
    of the 1-D finite-volume problem (Thomas / banded solve)."""
    nz, ny, nx = 32, 8, 8
    grid = O.Grid(nx, ny, nz)
    z = (np.arange(nz) + 0.5) / nz
    az = 1.0 + 50.0 * np.exp(-((z - 0.5) / 0.1) ** 2)
    fz = 100.0 * np.sin(3 * z)
    a = np.broadcast_to(az[:, None, None], grid.shape).copy()
    f = np.broadcast_to(fz[:, None, None], grid.shape).copy()
    params = O.OracleParams(rtol=1e-13, phi_bottom=0.3, phi_top=-1.0, coarse_min=2)
    phi, info, _ = O.solve(params, a, f)
    assert info.converged
    # 1-D system: -(a_{k+1/2}(u_{k+1}-u_k) - a_{k-1/2}(u_k-u_{k-1}))/h^2 = f_k
    h2 = grid.hz**2
    af = 0.5 * (az[1:] + az[:-1])
    upper = np.zeros(nz)
    diag = np.zeros(nz)
    lower = np.zeros(nz)
    rhs = fz.copy()
    diag[:-1] += af / h2
    diag[1:] += af / h2
    upper[1:] = -af / h2
    lower[:-1] = -af / h2
    diag[0] += 2 * az[0] / h2
    diag[-1] += 2 * az[-1] / h2
    rhs[0] += 2 * az[0] * params.phi_bottom / h2
    rhs[-1] += 2 * az[-1] * params.phi_top / h2
    u = scipy.linalg.solve_banded((1, 1), np.vstack([upper, diag, lower]), rhs)
    np.testing.assert_allclose(phi, np.broadcast_to(u[:, None, None], grid.shape), rtol=1e-9, atol=1e-10)


def _mms(variable):
    sympy = pytest.importorskip("sympy")
    x, y, z = sympy.symbols("x y z")
    phi = sympy.cos(sympy.pi * x) * sympy.cos(sympy.pi * y) * sympy.sin(sympy.pi * z) + z
    if variable:
        a = 2 + sympy.cos(sympy.pi * x) * sympy.cos(sympy.pi * y) * sympy.cos(sympy.pi * z)
    else:
        a = sympy.Integer(1)
    f = -sum(sympy.diff(a * sympy.diff(phi, v), v) for v in (x, y, z))
    grads = [-sympy.diff(phi, v) for v in (x, y, z)]
    mk = lambda e: sympy.lambdify((x, y, z), e, "numpy")   # noqa: E731
    return mk(phi), mk(a), mk(f), [mk(g) for g in grads]


@pytest.mark.parametrize("variable", [False, True])
def test_manufactured_solution_second_order(variable):
    """phi = cos(pi x) cos(pi y) sin(pi z) + z satisfies the plate data 0 / 1
    and zero flux on the side walls; the discrete solution and E converge at
    second order (Sec. 2.2 expects second-order accuracy)."""
    phi_fn, a_fn, f_fn, grad_fns = _mms(variable)
    errs, eerrs = [], []
    for n in (16, 32, 64):
        grid = O.Grid(n, n, n)
        c = (np.arange(n) + 0.5) / n
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        a = np.broadcast_to(a_fn(X, Y, Z), grid.shape).astype(np.float64).copy()
        f = np.broadcast_to(f_fn(X, Y, Z), grid.shape).astype(np.float64).copy()
        params = O.OracleParams(rtol=1e-12, phi_bottom=0.0, phi_top=1.0)
        phi, info, _ = O.solve(params, a, f)
        assert info.converged
        errs.append(np.abs(phi - phi_fn(X, Y, Z)).max())
        ex, ey, ez = O.field_from_potential(grid, phi, 0.0, 1.0)
        # a fixed physical interior region, [0.25, 0.75]^3 (the cells next to
        # the plates converge pre-asymptotically)
        m = (c > 0.25) & (c < 0.75)
        s = np.ix_(m, m, m)
        e = max(np.abs(ex - grad_fns[0](X, Y, Z))[s].max(),
                np.abs(ey - grad_fns[1](X, Y, Z))[s].max(),
                np.abs(ez - grad_fns[2](X, Y, Z))[s].max())
        eerrs.append(e)
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    eorders = np.log2(np.array(eerrs[:-1]) / np.array(eerrs[1:]))
    assert np.all(orders > 1.8), (errs, orders)
    assert np.all(eorders > 1.75), (eerrs, eorders)


def test_linear_potential_gives_uniform_field():
    """phi = z at the cell centres with plate data 0 and lz satisfies the ghost
    rule exactly, so E = (0, 0, -1) in every cell, boundary cells included."""
    shape = (7, 5, 6)
    grid = _grid(shape, (1.0, 1.0, 2.0))
    z = (np.arange(shape[0]) + 0.5) * grid.hz
    phi = np.broadcast_to(z[:, None, None], shape).copy()
    ex, ey, ez = O.field_from_potential(grid, phi, 0.0, 2.0)
    np.testing.assert_allclose(ex, 0.0, atol=1e-14)
    np.testing.assert_allclose(ey, 0.0, atol=1e-14)
    np.testing.assert_allclose(ez, -1.0, rtol=1e-13)
    # and A phi - bc = 0 for a = 1 (a linear potential is harmonic)
    a = np.ones(shape)
    r = O.apply_operator(grid, a, phi) - O.assemble_rhs(grid, a, np.zeros(shape), 0.0, 2.0)
    np.testing.assert_allclose(r, 0.0, atol=1e-10)


# ---------------------------------------------------------------------------
# Smoother: eq. (qntn), SSOR in red-black order
# ---------------------------------------------------------------------------


def _cheb_T(s, t):
    return np.polynomial.chebyshev.chebval(t, [0] * s + [1])


@pytest.mark.parametrize("steps", [1, 2, 3, 4])
def test_chebyshev_smoother_closed_form_on_eigenmode(steps):
    """With B = I and constant a, an eigenmode u with eigenvalue lam is mapped
    (b = 0) to q(lam) u, q = T_s((lmax+lmin-2 lam)/(lmax-lmin)) / T_s((lmax+lmin)/(lmax-lmin)),
    eq. (qntn) with s = n+1 steps."""
    shape = (8, 8, 8)
    grid = _grid(shape)
    a = np.ones(shape)
    lam_all = _spectral_symbols(grid)
    lmax, lmin = 1.1 * lam_all.max(), 0.1 * lam_all.max()
    for (mz, my, mx) in [(0, 0, 0), (2, 3, 1), (7, 7, 7), (4, 0, 6)]:
        c = np.zeros(shape)
        c[mz, my, mx] = 1.0
        u = scipy.fft.idst(scipy.fft.idctn(c, type=2, axes=(1, 2), norm="ortho"), type=2, axis=0, norm="ortho")
        lam = lam_all[mz, my, mx]
        out = O.chebyshev_smooth(grid, a, np.zeros(shape), u, lmax, lmin, steps, pc="identity")
        q = _cheb_T(steps, (lmax + lmin - 2 * lam) / (lmax - lmin)) / _cheb_T(steps, (lmax + lmin) / (lmax - lmin))
        np.testing.assert_allclose(out, q * u, atol=1e-13 * np.abs(u).max() + 1e-15)


def _rb_split(grid, a):
    A = O.dense_operator(grid, a)
    red = O.red_mask(grid).ravel()
    perm = np.concatenate([np.flatnonzero(red), np.flatnonzero(~red)])
    Ap = A[np.ix_(perm, perm)]
    D = np.diag(np.diag(Ap))
    L = np.tril(Ap, -1)
    U = np.triu(Ap, 1)
    return A, perm, D, L, U


def test_sgs_is_ssor_in_red_black_order():
    """z = B^{-1} r with B = (D+L) D^{-1} (D+U) in red-black ordering (SSOR, omega = 1)."""
    shape = (4, 6, 5)
    grid = _grid(shape)
    a = random_coefficient(4, shape, contrast=100.0)
    _, perm, D, L, U = _rb_split(grid, a)
    B = (D + L) @ np.linalg.inv(D) @ (D + U)
    r = random_field(5, shape).ravel()
    zp = np.linalg.solve(B, r[perm])
    z = np.empty_like(zp)
    z[perm] = zp
    np.testing.assert_allclose(O.sgs_redblack(grid, a, r.reshape(shape)).ravel(), z, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("steps", [2, 3])
def test_preconditioned_chebyshev_matches_matrix_polynomial(steps):
    """x -> S(x, b=0) equals q_s(B^{-1}A) x, q_s from eq. (qntn), evaluated by
    the Chebyshev three-term recurrence on the dense matrix B^{-1}A."""
    shape = (4, 4, 6)
    grid = _grid(shape)
    a = random_coefficient(6, shape, contrast=30.0)
    A, perm, D, L, U = _rb_split(grid, a)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    B = ((D + L) @ np.linalg.inv(D) @ (D + U))[np.ix_(inv, inv)]
    C = np.linalg.solve(B, A)
    lmax, lmin = 1.05, 0.2
    n = C.shape[0]
    Y = ((lmax + lmin) * np.eye(n) - 2 * C) / (lmax - lmin)
    T0, T1 = np.eye(n), Y
    for _ in range(steps - 1):
        T0, T1 = T1, 2 * Y @ T1 - T0
    q = T1 / _cheb_T(steps, (lmax + lmin) / (lmax - lmin))
    x = random_field(7, shape)
    out = O.chebyshev_smooth(grid, a, np.zeros(shape), x, lmax, lmin, steps, pc="sgs")
    np.testing.assert_allclose(out.ravel(), q @ x.ravel(), rtol=1e-11, atol=1e-12)


def test_eigen_estimate_bounds_the_sgs_spectrum():
    """lam_hat (Sec. 3.2) is a Ritz value of B^{-1}A: below its largest
    eigenvalue, within a few percent of it, and B^{-1}A has spectrum in (0, 1]."""
    shape = (8, 8, 8)
    grid = _grid(shape)
    a = random_coefficient(8, shape, contrast=1e3)
    A, perm, D, L, U = _rb_split(grid, a)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    B = ((D + L) @ np.linalg.inv(D) @ (D + U))[np.ix_(inv, inv)]
    ev = np.linalg.eigvals(np.linalg.solve(B, A)).real
    assert ev.min() > 0 and ev.max() <= 1.0 + 1e-12
    lmax, lmin, lam_hat = O.estimate_eig_bounds(grid, a, O.OracleParams())
    assert lam_hat <= ev.max() * (1 + 1e-12)
    assert lam_hat > 0.9 * ev.max()
    assert lmax == pytest.approx(1.1 * lam_hat) and lmin == pytest.approx(0.1 * lam_hat)


def test_splitmix64_reference_values():
    """splitmix64 from the published generator: the first outputs for seed 0
    (state advanced by the golden gamma before mixing)."""
    out = O.splitmix64(np.arange(3, dtype=np.uint64))
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


# ---------------------------------------------------------------------------
# Transfers, V-cycle (Appendix A), coarse solve
# ---------------------------------------------------------------------------


def test_transfers_reproduce_constants_and_linears():
    c = random_field(9, (4, 4, 4))
    assert O.restrict(np.full((8, 8, 8), 3.5)) == pytest.approx(np.full((4, 4, 4), 3.5))
    # piecewise-constant prolongation is 8 x the adjoint of restriction
    f = random_field(10, (8, 8, 8))
    assert np.dot(O.prolong(c, "constant").ravel(), f.ravel()) == pytest.approx(8 * np.dot(c.ravel(), O.restrict(f).ravel()))
    # trilinear reproduces a linear function away from the walls
    n = 8
    cc = (np.arange(n) + 0.5) / n
    cf = (np.arange(2 * n) + 0.5) / (2 * n)
    Zc, Yc, Xc = np.meshgrid(cc, cc, cc, indexing="ij")
    Zf, Yf, Xf = np.meshgrid(cf, cf, cf, indexing="ij")
    lin = lambda X, Y, Z: 1 + 2 * X - 3 * Y + 0.5 * Z   # noqa: E731
    p = O.prolong(lin(Xc, Yc, Zc))
    np.testing.assert_allclose(p[1:-1, 1:-1, 1:-1], lin(Xf, Yf, Zf)[1:-1, 1:-1, 1:-1], atol=1e-13)
    # Neumann walls: constants are reproduced up to the wall in x and y
    pc = O.prolong(np.ones((4, 4, 4)))
    np.testing.assert_allclose(pc[1:-1], 1.0, atol=1e-15)
    # Dirichlet plates: odd ghost halves the boundary child in z
    np.testing.assert_allclose(pc[0], 0.5, atol=1e-15)


def test_series_coarsening_of_a_constant_is_rediscretisation():
    """With a constant coefficient every coarse face, plates included, carries
    that constant (R3 reduces to eq. (e18) on the coarse grid): the coarse
    operator equals the re-discretised one on every level."""
    shape = (16, 8, 12)
    grid = _grid(shape, (1.2, 0.7, 2.0))
    a = np.full(shape, 3.25)
    f = O.faces_of_cells(a)
    g = grid
    for _ in range(2):
        f = O.coarsen_faces(f)
        g = g.coarser()
        x = random_field(90, g.shape)
        np.testing.assert_allclose(O.apply_operator(g, f, x), O.apply_operator(g, np.full(g.shape, 3.25), x),
                                   rtol=1e-13, atol=1e-12)


def _layered(n, seed, contrast=1e4):
    return random_coefficient(seed, (n,), contrast=contrast)


def test_series_coarsening_keeps_the_plate_to_plate_resistance():
    """A medium layered in z (a = a(z)) is a chain of resistors between the
    plates.  On the fine grid of eq. (e18) its resistance per unit area is
    sum_links hz / a_link + (hz/2)/a_0 + (hz/2)/a_{n-1} (the face means of
    Sec. 2.2, the plate faces of R1 over half a cell).  Series coarsening must
    keep that total on every level, H/A per coarse link and (H/2)/P per plate;
    a wrong half factor, a swapped link or an arithmetic mean along the
    normal changes it."""
    nz = 32
    az = _layered(nz, 91)
    shape = (nz, 8, 8)
    a = np.broadcast_to(az[:, None, None], shape).copy()
    h = 1.0 / nz
    fine = np.sum(h / (0.5 * (az[1:] + az[:-1]))) + 0.5 * h / az[0] + 0.5 * h / az[-1]
    f = O.faces_of_cells(a)
    H = h
    for _ in range(3):
        f = O.coarsen_faces(f)
        H *= 2
        col = f.az[:, 0, 0]
        total = np.sum(H / col) + 0.5 * H / f.bottom[0, 0] + 0.5 * H / f.top[0, 0]
        assert total == pytest.approx(fine, rel=1e-13)
        for v in (f.az, f.bottom, f.top):        # no variation across the layers' planes
            assert np.ptp(v, axis=(-2, -1)).max() <= 1e-12 * v.max()


def test_series_coarsening_keeps_the_parallel_conductance():
    """A medium layered in x, a = a(x), conducts in z through parallel columns:
    the total conductance of a z-face, sum over its columns of a / h^2 times
    the column's area, is kept on every level (the arithmetic mean across)."""
    nx = 16
    ax_ = _layered(nx, 92, contrast=1e3)
    shape = (8, 4, nx)
    a = np.broadcast_to(ax_[None, None, :], shape).copy()
    f = O.faces_of_cells(a)
    total = ax_.sum()           # per unit height: sum of the columns' a times width h = 1/nx, times nx
    for lev in range(2):
        f = O.coarsen_faces(f)
        m = f.az.shape[2]
        assert f.az[0, 0].sum() * (nx / m) == pytest.approx(total, rel=1e-13)
        assert f.bottom[0].sum() * (nx / m) == pytest.approx(total, rel=1e-13)


@pytest.mark.parametrize("axis", [2, 1])
def test_series_coarsening_along_x_and_y_matches_the_fine_chain(axis):
    """The same series rule along x and y: for a medium layered along that
    axis, the first coarse level's links from the first coarse cell's centre to
    the last one's (the midpoints of their inner fine links) add up to the fine
    chain in between: half of each end's inner link and every link between."""
    n = 32
    av = _layered(n, 93 + axis)
    shape = [8, 8, 8]
    shape[axis] = n
    idx = [None, None, None]
    idx[axis] = slice(None)
    a = np.broadcast_to(av[tuple(idx)], shape).copy()
    h = 1.0 / n
    links = 0.5 * (av[1:] + av[:-1])
    f = O.coarsen_faces(a)
    coarse = f.ax[0, 0] if axis == 2 else f.ay[0, :, 0]
    fine = np.sum(h / links[1:n - 2]) + 0.5 * h / links[0] + 0.5 * h / links[n - 2]
    assert np.sum(2 * h / coarse) == pytest.approx(fine, rel=1e-13)
    other = f.ax if axis == 2 else f.ay
    assert np.ptp(np.moveaxis(other, axis, -1), axis=(0, 1)).max() <= 1e-12 * other.max()


def _constant_flux_profile(links, h, start=0.0):
    """Potential at the cell centres of a 1-D chain with unit flux through every
    link: phi_{m+1} = phi_m - h / A_m."""
    phi = np.empty(links.size + 1)
    phi[0] = start
    for m in range(links.size):
        phi[m + 1] = phi[m] - h / links[m]
    return phi


def test_opdep_prolongation_is_exact_for_a_constant_flux_in_z():
    """In a medium layered in z, a potential that carries one flux through every
    fine link (and through the bottom plate, where it is 0) is linear in the
    resistance along the path.  Its values at the coarse centres (the
    midpoints of the inner fine links) interpolated by the operator-dependent
    prolongation give the fine values back, the boundary child at the bottom
    plate included (R4, "opdep").  Trilinear weights do not."""
    nz = 16
    az = _layered(nz, 94)
    shape = (nz, 2, 4)
    a = np.broadcast_to(az[:, None, None], shape).copy()
    h = 1.0 / nz
    links = 0.5 * (az[1:] + az[:-1])
    # unit flux downwards into the bottom plate (value 0 there): phi_0 = (h/2)/a_0
    phi = _constant_flux_profile(-links, h, start=0.5 * h / az[0])
    coarse = 0.5 * (phi[0::2] + phi[1::2])      # midpoint of each coarse cell's inner link
    c3 = np.broadcast_to(coarse[:, None, None], (nz // 2, 1, 2)).copy()
    got = O.prolong(c3, "opdep", a)
    want = np.broadcast_to(phi[:, None, None], shape)
    np.testing.assert_allclose(got[:-1], want[:-1], rtol=1e-12)   # the top child meets the top plate's 0
    tri = O.prolong(c3, "trilinear")
    assert np.abs(tri[:-1] - want[:-1]).max() > 1e-3 * np.abs(want).max()


def test_opdep_prolongation_is_exact_for_a_constant_flux_in_x():
    """The same along x, away from the two wall children (which copy their
    parent, the Neumann mirror)."""
    nx = 16
    axv = _layered(nx, 95)
    shape = (2, 2, nx)
    a = np.broadcast_to(axv[None, None, :], shape).copy()
    h = 1.0 / nx
    links = 0.5 * (axv[1:] + axv[:-1])
    phi = _constant_flux_profile(links, h, start=1.0)
    coarse = 0.5 * (phi[0::2] + phi[1::2])
    c3 = np.broadcast_to(coarse[None, None, :], (1, 1, nx // 2)).copy()
    # z: one coarse plane between the plates; its z weights multiply every x value alike
    got = O.prolong(c3, "opdep", a)
    wz = O.prolong_weights(a)[2]
    np.testing.assert_allclose(got[:, :, 1:-1] / wz[:, :, 1:-1], np.broadcast_to(phi[1:-1], (2, 2, nx - 2)),
                               rtol=1e-12)
    np.testing.assert_allclose(got[:, :, 0] / wz[:, :, 0], coarse[0], rtol=1e-14)
    np.testing.assert_allclose(got[:, :, -1] / wz[:, :, -1], coarse[-1], rtol=1e-14)


def test_opdep_prolongation_of_a_constant_coefficient_is_trilinear():
    rng = np.random.default_rng(96)
    for shape in ((8, 6, 10), (4, 4, 4), (16, 8, 12)):
        a = np.full(shape, 7.0)
        e = rng.standard_normal(tuple(s // 2 for s in shape))
        np.testing.assert_allclose(O.prolong(e, "opdep", a), O.prolong(e, "trilinear"), rtol=0, atol=1e-14)
        np.testing.assert_allclose(O.prolong(e, "opdep", O.faces_of_cells(a)), O.prolong(e, "trilinear"),
                                   rtol=0, atol=1e-14)


def test_series_coarse_operators_are_symmetric_positive_definite():
    shape = (8, 8, 8)
    a = random_coefficient(97, shape, contrast=1e4)
    f = O.coarsen_faces(a)
    g = _grid(shape).coarser()
    A = O.dense_operator(g, f)
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-12 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).min() > 0


def _dense_from_map(fn, n, shape):
    m = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        m[:, i] = fn(e.reshape(shape)).ravel()
    return m


TRANSFER_CASES = [(4, "opdep", "series"), (2, "opdep", "series"), (2, "trilinear", "series"),
                  (4, "trilinear", "mean"), (2, "trilinear", "mean"), (2, "constant", "mean")]


@pytest.mark.parametrize("coarse_min,prolongation,coarsening", TRANSFER_CASES)
def test_vcycle_equals_appendix_a_recursion(coarse_min, prolongation, coarsening):
    """vcycle(v) = M_L v with M_1 = A_1^{-1}, M_l = Q_l P_l + P_l +
    Q_l P_{l-1,l} M_{l-1} R_{l,l-1} (I - A_l P_l) (Appendix A), where the
    smoother x -> Q_l x + P_l b (eq. (e19)) is read off as dense matrices."""
    shape = (8, 8, 8)
    grid = _grid(shape)
    a = random_coefficient(11, shape, contrast=50.0)
    params = O.OracleParams(coarse_min=coarse_min, prolongation=prolongation, cheb_steps=3, coarsening=coarsening)
    hier = O.build_hierarchy(grid, a, params)
    M = None
    for li, lev in enumerate(hier.levels):
        n = lev.grid.size
        A = O.dense_operator(lev.grid, lev.a)
        if li == 0:
            M = np.linalg.inv(A)
            continue
        sm = lambda x, b: O.chebyshev_smooth(lev.grid, lev.a, b, x, lev.lam_max, lev.lam_min,   # noqa: E731
                                             params.cheb_steps, params.smoother_pc)
        P = _dense_from_map(lambda e: sm(None, e), n, lev.grid.shape)
        Q = _dense_from_map(lambda e: sm(e, np.zeros(lev.grid.shape)), n, lev.grid.shape)
        # the smoother is a consistent iteration: Q = I - P A  (eq. (e19))
        np.testing.assert_allclose(Q, np.eye(n) - P @ A, atol=1e-11)
        cshape = hier.levels[li - 1].grid.shape
        nc = hier.levels[li - 1].grid.size
        R = np.array([O.restrict(e.reshape(lev.grid.shape)).ravel() for e in np.eye(n)]).T
        Pr = np.array([O.prolong(e.reshape(cshape), prolongation, lev.a).ravel() for e in np.eye(nc)]).T
        M = Q @ P + P + Q @ Pr @ M @ R @ (np.eye(n) - A @ P)
    v = random_field(12, shape)
    np.testing.assert_allclose(O.vcycle(hier, v).ravel(), M @ v.ravel(), rtol=1e-10, atol=1e-12)


def test_coarse_direct_solve_residual():
    shape = (4, 4, 4)
    grid = _grid(shape)
    a = random_coefficient(13, shape, contrast=1e3)
    hier = O.build_hierarchy(grid, a, O.OracleParams(coarse_min=4))
    assert len(hier.levels) == 1
    b = random_field(14, shape)
    x = O.coarse_solve(hier, b)
    A = O.dense_operator(grid, a)
    assert np.linalg.norm(A @ x.ravel() - b.ravel()) <= 1e-14 * np.linalg.norm(A) * np.linalg.norm(x)


def test_level_count_rules():
    assert O.level_count(32, 32, 32, 4) == 4
    assert O.level_count(512, 512, 512, 4) == 8
    assert O.level_count(256, 256, 320, 4) == 7          # 4 x 4 x 5 coarsest
    with pytest.raises(ValueError):
        O.level_count(12, 12, 10, 4)


# ---------------------------------------------------------------------------
# FGMRES, Algorithm 1
# ---------------------------------------------------------------------------


def test_fgmres_matches_dense_direct_solve_8cube():
    shape = (8, 8, 8)
    grid = _grid(shape)
    a = random_coefficient(15, shape, contrast=1e3)
    f = random_field(16, shape) * 100
    for coarse_min in (4, 2):
        params = O.OracleParams(coarse_min=coarse_min)
        phi, info, _ = O.solve(params, a, f)
        assert info.converged and info.true_rel_residual < 1e-8
        A = O.dense_operator(grid, a)
        b = O.assemble_rhs(grid, a, f, params.phi_bottom, params.phi_top)
        exact = np.linalg.solve(A, b.ravel())
        cond = np.linalg.cond(A)
        assert np.linalg.norm(phi.ravel() - exact) / np.linalg.norm(exact) <= cond * 1e-8


def test_fgmres_exact_preconditioner_converges_in_one_step():
    shape = (6, 4, 4)
    grid = _grid(shape)
    a = random_coefficient(17, shape, contrast=10.0)
    A = O.dense_operator(grid, a)
    Ainv = np.linalg.inv(A)
    b = random_field(18, shape)
    x, info = O.fgmres(grid, a, b, None, lambda v: (Ainv @ v.ravel()).reshape(shape), O.OracleParams(rtol=1e-12))
    assert info.iterations == 1 and info.converged
    np.testing.assert_allclose(x.ravel(), Ainv @ b.ravel(), rtol=1e-10)


def test_fgmres_identity_preconditioner_is_gmres():
    """With M = I, FGMRES is GMRES: least-squares residuals never increase and
    equal the minimal residual over the Krylov space K_j(A, b)."""
    shape = (4, 4, 4)
    grid = _grid(shape)
    a = random_coefficient(19, shape, contrast=10.0)
    A = O.dense_operator(grid, a)
    b = random_field(20, shape)
    params = O.OracleParams(rtol=1e-10, restart=30, max_iters=12)
    _, info = O.fgmres(grid, a, b, None, lambda v: np.array(v, copy=True), params)
    h = np.array(info.history)
    assert np.all(np.diff(h) <= 1e-12)
    K = [b.ravel() / np.linalg.norm(b)]
    for j in range(6):
        K.append(A @ K[-1])
        K[-1] /= np.linalg.norm(K[-1])
        Qk, _ = np.linalg.qr(np.array(K[:-1]).T)
        AQ = A @ Qk
        y = np.linalg.lstsq(AQ, b.ravel(), rcond=None)[0]
        mr = np.linalg.norm(b.ravel() - AQ @ y) / np.linalg.norm(b)
        assert h[j] == pytest.approx(mr, rel=1e-6, abs=1e-13)


def test_restart_and_true_residual_rule():
    """Restart m = 2 forces several cycles; the returned x has true residual
    below rtol and the iteration cap reports non-convergence."""
    inp = make_inputs("channel128", n=16)
    params = O.OracleParams(restart=2, coarse_min=4)
    phi, info, _ = O.solve(params, inp["a"], inp["f"])
    assert info.converged and info.restarts > 2 and info.true_rel_residual < 1e-8
    params = O.OracleParams(max_iters=2)
    phi, info, _ = O.solve(params, inp["a"], inp["f"])
    assert not info.converged and info.iterations == 2


def test_scaling_invariance():
    """(a, f) -> (c a, c f) leaves phi unchanged: A and b both scale by c."""
    inp = make_inputs("channel128", n=16)
    params = O.OracleParams(rtol=1e-12)
    p1, _, _ = O.solve(params, inp["a"], inp["f"])
    p2, _, _ = O.solve(params, 7.0 * inp["a"], 7.0 * inp["f"])
    np.testing.assert_allclose(p1, p2, rtol=1e-9, atol=1e-11)


# ---------------------------------------------------------------------------
# Adjoint (not in the paper: derivative of the discrete solve)
# ---------------------------------------------------------------------------


def test_adjoint_matches_finite_differences_dense():
    """L = w . phi(a, f) with phi from a dense direct solve; central differences
    in a_p and f_p agree with dL/da from the adjoint face formula and with
    dL/df = lambda = A^{-1} w."""
    shape = (4, 3, 5)
    grid = _grid(shape, (1.0, 0.8, 1.2))
    a = random_coefficient(21, shape, contrast=20.0)
    f = random_field(22, shape) * 10
    w = random_field(23, shape)
    gb, gt = 0.4, 1.3

    def loss(aa, ff):
        A = O.dense_operator(grid, aa)
        b = O.assemble_rhs(grid, aa, ff, gb, gt)
        return float(np.dot(w.ravel(), np.linalg.solve(A, b.ravel())))

    A = O.dense_operator(grid, a)
    phi = np.linalg.solve(A, O.assemble_rhs(grid, a, f, gb, gt).ravel()).reshape(shape)
    lam = np.linalg.solve(A, w.ravel()).reshape(shape)
    ga = O.adjoint_coefficient_grad(grid, phi, lam, gb, gt)
    rng = np.random.default_rng(24)
    for p in rng.choice(a.size, size=12, replace=False):
        da = np.zeros(a.size)
        h = 1e-4 * a.ravel()[p]     # truncation ~1e-8, round-off noise ~1e-9 (relative)
        da[p] = h
        da = da.reshape(shape)
        fd = (loss(a + da, f) - loss(a - da, f)) / (2 * h)
        assert ga.ravel()[p] == pytest.approx(fd, rel=1e-6, abs=1e-9)
        df = np.zeros(a.size)
        df[p] = 1e-3
        df = df.reshape(shape)
        fdf = (loss(a, f + df) - loss(a, f - df)) / 2e-3
        assert lam.ravel()[p] == pytest.approx(fdf, rel=1e-8, abs=1e-12)


def test_adjoint_dot_product_identity():
    """w . A^{-1} f = f . A^{-1} w for the solver's (symmetric) operator."""
    inp = make_inputs("adjoint", n=16)
    params = O.OracleParams(rtol=1e-12)
    phi, _, hier = O.solve(params, inp["a"], inp["f"], homogeneous=True)
    lam, _, _ = O.solve(params, inp["a"], inp["w"], homogeneous=True, hierarchy=hier)
    lhs = np.dot(inp["w"].ravel(), phi.ravel())
    rhs = np.dot(inp["f"].ravel(), lam.ravel())
    assert lhs == pytest.approx(rhs, rel=1e-9)


# ---------------------------------------------------------------------------
# Full multigrid (the first time step's preconditioner, Sec. 3.2)
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("coarse_min,prolongation,coarsening", TRANSFER_CASES)
def test_fmg_equals_dense_recursion(coarse_min, prolongation, coarsening):
    """A V-cycle from a guess x0 is the consistent iteration x0 + M_l (b - A_l x0),
    so full multigrid is the matrix F_l = P F_{l-1} R + M_l (I - A_l P F_{l-1} R)
    with F_1 = A_1^{-1}; M_l is read off the zero-guess V-cycle as a dense matrix."""
    shape = (8, 8, 8)
    grid = _grid(shape)
    a = random_coefficient(41, shape, contrast=30.0)
    params = O.OracleParams(coarse_min=coarse_min, prolongation=prolongation, coarsening=coarsening)
    hier = O.build_hierarchy(grid, a, params)
    F = None
    for li, lev in enumerate(hier.levels):
        n = lev.grid.size
        A = O.dense_operator(lev.grid, lev.a)
        if li == 0:
            F = np.linalg.inv(A)
            continue
        M = _dense_from_map(lambda e: O.vcycle(hier, e, li), n, lev.grid.shape)
        cshape = hier.levels[li - 1].grid.shape
        nc = hier.levels[li - 1].grid.size
        R = np.array([O.restrict(e.reshape(lev.grid.shape)).ravel() for e in np.eye(n)]).T
        Pr = np.array([O.prolong(e.reshape(cshape), prolongation, lev.a).ravel() for e in np.eye(nc)]).T
        X0 = Pr @ F @ R
        F = X0 + M @ (np.eye(n) - A @ X0)
    v = random_field(42, shape)
    np.testing.assert_allclose(O.fmg(hier, v).ravel(), F @ v.ravel(), rtol=1e-10, atol=1e-12)


def test_vcycle_from_a_zero_guess_is_the_vcycle():
    shape = (16, 16, 16)
    grid = _grid(shape)
    a = random_coefficient(43, shape, contrast=100.0)
    hier = O.build_hierarchy(grid, a, O.OracleParams(coarse_min=4))
    b = random_field(44, shape)
    np.testing.assert_allclose(O.vcycle_from(hier, b, np.zeros(shape)), O.vcycle(hier, b), rtol=0, atol=1e-14)
    # from the exact solution nothing changes (the cycle is a consistent iteration)
    x = random_field(45, shape)
    xb = O.apply_operator(grid, a, x)
    np.testing.assert_allclose(O.vcycle_from(hier, xb, x), x, rtol=1e-11, atol=1e-11)


def test_fmg_preconditioned_fgmres_converges_no_slower():
    shape = (32, 32, 32)
    inp = make_inputs("channel128", shape=shape)
    pv = O.OracleParams(coarse_min=4, cycle="v")
    pf = O.OracleParams(coarse_min=4, cycle="fmg")
    pa = O.OracleParams(coarse_min=4, cycle="auto")
    _, iv, _ = O.solve(pv, inp["a"], inp["f"])
    _, i_f, _ = O.solve(pf, inp["a"], inp["f"])
    _, ia, _ = O.solve(pa, inp["a"], inp["f"])       # zero guess: FMG
    assert iv.converged and i_f.converged and ia.converged
    assert i_f.iterations <= iv.iterations
    assert ia.iterations == i_f.iterations
    assert i_f.true_rel_residual < 1e-8


# ---------------------------------------------------------------------------
# Coefficient and right-hand side from the densities, eq. (semi2) / (e18)
# ---------------------------------------------------------------------------

E_OVER_EPS0 = O.ELEMENTARY_CHARGE / O.VACUUM_PERMITTIVITY_CM


def test_assembly_constant_densities_closed_form():
    shape = (6, 5, 4)
    grid = _grid(shape, (2.0, 1.0, 0.5))
    ne = np.full(shape, 3.0e13)
    npos = np.full(shape, 5.0e13)
    a, f = O.assemble_coefficient_rhs(grid, ne, npos, 2e-12, -381.6, 3.42, (2190.0, 2190.0, 1800.0), E_OVER_EPS0)
    np.testing.assert_allclose(a, 1.0 + E_OVER_EPS0 * 1e-12 * (3.42 * 5.0e13 + 381.6 * 3.0e13), rtol=1e-15)
    # no diffusion term for uniform densities
    np.testing.assert_allclose(f, E_OVER_EPS0 * 2.0e13, rtol=1e-14)


def test_assembly_vacuum_coefficient_matches_the_papers_magnitude():
    """At n_e = n_p = 1e14 cm^-3, tau = 2 ps and the mobilities of Sec. 5.2
    (|mu_e| = 2.9e5/760, mu_p = 2.6e3/760 cm^2/(V s)) the coefficient is about
    1.07: the mild contrast of the paper's own runs."""
    shape = (4, 4, 4)
    grid = _grid(shape)
    n = np.full(shape, 1e14)
    a, _ = O.assemble_coefficient_rhs(grid, n, n, 2e-12, -2.9e5 / 760, 2.6e3 / 760, (2190.0, 2190.0, 1800.0),
                                      E_OVER_EPS0)
    assert a[0, 0, 0] == pytest.approx(1.0697, abs=5e-4)


def test_assembly_diffusion_term_on_a_quadratic_profile():
    """n_e = i^2 along x: delta^2 = 2 inside; the Neumann ghosts give
    n_1 - n_0 = 1 at the first cell and n_{m-2} - n_{m-1} = -(2m - 3) at the last."""
    m = 7
    shape = (3, 4, m)
    grid = _grid(shape, (float(m), 1.0, 1.0))          # hx = 1
    i = np.arange(m, dtype=np.float64)
    ne = np.broadcast_to(i ** 2, shape).copy()
    zero = np.zeros(shape)
    tau, dx = 1.0, 1.0
    a, f = O.assemble_coefficient_rhs(grid, ne, zero, tau, 0.0, 0.0, (dx, 5.0, 7.0), 1.0)
    d2 = np.full(m, 2.0)
    d2[0] = 1.0
    d2[-1] = -(2 * m - 3)
    np.testing.assert_allclose(f, np.broadcast_to(-ne[0, 0] - 0.5 * tau * dx * d2, shape), rtol=0, atol=1e-12)
    np.testing.assert_allclose(a, 1.0, rtol=0, atol=0)


def test_assembly_diffusion_term_conserves_charge():
    """With zero-flux ghosts the second differences telescope: the diffusion
    term sums to zero, so sum(f) = (e/eps0) sum(n_p - n_e) for any densities."""
    shape = (8, 6, 10)
    grid = _grid(shape, (1.0, 0.7, 1.3))
    ne = 1e12 * (1.0 + random_field(46, shape) ** 2)
    npos = 1e12 * (1.0 + random_field(47, shape) ** 2)
    _, f = O.assemble_coefficient_rhs(grid, ne, npos, 3e-12, 381.6, 3.42, (2190.0, 2190.0, 1800.0), E_OVER_EPS0)
    assert f.sum() == pytest.approx(E_OVER_EPS0 * (npos - ne).sum(), rel=1e-9)


# ---------------------------------------------------------------------------
# The other Krylov methods of the paper's comparison (Tables t1, t2)
# ---------------------------------------------------------------------------


def _dense_problem(seed=50, contrast=20.0):
    shape = (8, 8, 8)
    grid = _grid(shape)
    a = random_coefficient(seed, shape, contrast=contrast)
    A = O.dense_operator(grid, a)
    b = random_field(seed + 1, shape)
    return grid, a, A, b


@pytest.mark.parametrize("method", O.KRYLOV_METHODS)
def test_krylov_with_the_exact_preconditioner_takes_one_iteration(method):
    grid, a, A, b = _dense_problem()
    Ainv = np.linalg.inv(A)
    x, info = O.krylov(method, grid, a, b, None, lambda v: (Ainv @ v.ravel()).reshape(grid.shape),
                       O.OracleParams(rtol=1e-10))
    assert info.converged and info.iterations == 1
    np.testing.assert_allclose(A @ x.ravel(), b.ravel(), rtol=0, atol=1e-10 * np.linalg.norm(b))


def test_gmres_equals_fgmres_for_a_fixed_preconditioner():
    grid, a, A, b = _dense_problem(52)
    hier = O.build_hierarchy(grid, a, O.OracleParams(coarse_min=2))
    pc = lambda v: O.vcycle(hier, v)   # noqa: E731  (a fixed linear map)
    params = O.OracleParams(rtol=1e-11, restart=5)
    x1, i1 = O.krylov("fgmres", grid, a, b, None, pc, params)
    x2, i2 = O.krylov("gmres", grid, a, b, None, pc, params)
    assert i1.iterations == i2.iterations and i1.restarts == i2.restarts
    np.testing.assert_allclose(x2, x1, rtol=1e-9, atol=1e-12)


def test_fcg_equals_pcg_for_a_symmetric_preconditioner():
    grid, a, A, b = _dense_problem(54)
    dinv = 1.0 / np.diag(A)
    pc = lambda v: (dinv * v.ravel()).reshape(grid.shape)   # noqa: E731  (Jacobi: SPD)
    params = O.OracleParams(rtol=1e-10, max_iters=500)
    x1, i1 = O.krylov("cg", grid, a, b, None, pc, params)
    x2, i2 = O.krylov("fcg", grid, a, b, None, pc, params)
    assert i1.iterations == i2.iterations
    np.testing.assert_allclose(x2, x1, rtol=1e-8, atol=1e-12)


@pytest.mark.parametrize("method", ["cg", "cgs", "bicgstab"])
def test_short_recurrences_match_scipy(method):
    """The same textbook algorithms in SciPy (Jacobi-preconditioned, relative
    tolerance on ||r||/||b||): the same iteration count within one step and
    the same solution."""
    import scipy.sparse.linalg as sla
    grid, a, A, b = _dense_problem(56)
    dinv = 1.0 / np.diag(A)
    M = sla.LinearOperator(A.shape, matvec=lambda v: dinv * v)
    count = [0]

    def cb(_):
        count[0] += 1
    fn = {"cg": sla.cg, "cgs": sla.cgs, "bicgstab": sla.bicgstab}[method]
    xs, flag = fn(A, b.ravel(), rtol=1e-9, atol=0.0, maxiter=1000, M=M, callback=cb)
    assert flag == 0
    x, info = O.krylov(method, grid, a, b, None, lambda v: (dinv * v.ravel()).reshape(grid.shape),
                       O.OracleParams(rtol=1e-9, max_iters=1000))
    assert abs(info.iterations - count[0]) <= 1, (info.iterations, count[0])
    np.testing.assert_allclose(x.ravel(), xs, rtol=1e-6, atol=1e-9 * np.abs(xs).max())


@pytest.mark.parametrize("method", O.KRYLOV_METHODS)
def test_krylov_methods_reach_the_true_residual_with_multigrid(method):
    inp = make_inputs("channel128", shape=(16, 16, 16))
    phi, info, _ = O.solve(O.OracleParams(coarse_min=4), inp["a"], inp["f"], method=method)
    assert info.converged and info.true_rel_residual < 1e-8


# ---------------------------------------------------------------------------
# Transport and the semi-implicit time step, eqs. (e1)-(e2) (Sec. 2.1, 2.2)
# ---------------------------------------------------------------------------


def test_koren_limiter_closed_form():
    r = np.array([-3.0, -0.1, 0.0, 0.1, 0.25, 0.5, 1.0, 2.0, 2.5, 4.0, 100.0])
    phi = np.maximum(0.0, np.minimum(np.minimum(2 * r, (1 + 2 * r) / 3), 2.0))
    # phi(r) b with b = 1 and b = -2 (a = r b)
    np.testing.assert_allclose(O.koren_slope(r * 1.0, np.ones_like(r)), phi, rtol=0, atol=1e-15)
    np.testing.assert_allclose(O.koren_slope(r * -2.0, np.full_like(r, -2.0)), -2.0 * phi, rtol=0, atol=1e-15)
    assert O.koren_slope(np.array([1.0]), np.array([0.0]))[0] == 0.0      # flat upwind side


def test_ionization_coefficient_values():
    e = np.array([0.0, 1e4, 2.08e5])
    a = O.ionization_coefficient(e)
    assert a[0] == 0.0
    assert a[1] == pytest.approx(5.7 * 760 * np.exp(-260 * 760 / 1e4), rel=1e-14)
    assert a[2] == pytest.approx(5.7 * 760 * np.exp(-260 * 760 / 2.08e5), rel=1e-14)


def _uniform_field_case(m=12, e0=1.5e5):
    """phi = -e0 x on a unit cube of m^3 cells with both plates at 0 V:
    interior x-faces carry E_x = e0, y- and z-faces carry no field inside."""
    shape = (m, m, m)
    grid = _grid(shape)
    x = (np.arange(m) + 0.5) / m
    phi = np.broadcast_to(-e0 * x, shape).copy()
    return grid, phi, e0


def test_transport_rhs_linear_density_in_a_uniform_field():
    grid, phi, e0 = _uniform_field_case()
    m = grid.nx
    idx = np.arange(m, dtype=np.float64)
    ne = np.broadcast_to(1e12 + 1e10 * idx, grid.shape).copy()       # linear in x: the slopes are exact
    npos = np.broadcast_to(2e12 - 3e9 * idx, grid.shape).copy()
    mu_e, mu_p = 380.0, 3.4
    re, rp = O.transport_rhs(grid, ne, npos, phi, 0.0, 0.0, mu_e, mu_p, (1.0e3, 2.0e3, 3.0e3))
    g_e, g_p = 1e10 / grid.hx, -3e9 / grid.hx
    lam = O.ionization_coefficient(np.array([e0]))[0] * mu_e * e0
    inner = (slice(3, m - 3),) * 3
    # electrons drift at -mu_e E: -div(v n) = mu_e e0 dn/dx; no diffusion of a linear profile
    np.testing.assert_allclose(re[inner], mu_e * e0 * g_e + lam * ne[inner], rtol=1e-11)
    np.testing.assert_allclose(rp[inner], -mu_p * e0 * g_p + lam * ne[inner], rtol=1e-11)


def test_two_stage_step_is_the_explicit_midpoint_rule():
    """Uniform densities in a uniform field grow by the ionization source only:
    the predictor-corrector of eqs. (e1)-(e2) gives n (1 + tau l + (tau l)^2 / 2)."""
    grid, phi, e0 = _uniform_field_case(m=14)
    ne = np.full(grid.shape, 1e12)
    npos = np.full(grid.shape, 1.2e12)
    mu_e, mu_p, tau = 380.0, 3.4, 2e-12
    lam = O.ionization_coefficient(np.array([e0]))[0] * mu_e * e0
    args = (phi, 0.0, 0.0, mu_e, mu_p, (0.0, 0.0, 0.0))
    he, hp = O.transport_stage(grid, ne, npos, ne, npos, *args, 0.5 * tau)
    e1, p1 = O.transport_stage(grid, ne, npos, he, hp, *args, tau)
    inner = (slice(5, 9),) * 3
    np.testing.assert_allclose(e1[inner], 1e12 * (1 + tau * lam + 0.5 * (tau * lam) ** 2), rtol=1e-13)
    np.testing.assert_allclose(p1[inner], 1.2e12 + tau * lam * 1e12 * (1 + 0.5 * tau * lam), rtol=1e-13)


def test_drift_divergence_second_order_on_a_smooth_monotone_profile():
    errs = []
    for m in (32, 64):
        grid, phi, e0 = _uniform_field_case(m=m, e0=1e5)
        x = (np.arange(m) + 0.5) / m
        prof = np.exp(-((x - 0.3) / 0.25) ** 2)                     # decreasing for x > 0.3
        ne = np.broadcast_to(1e12 * prof, grid.shape).copy()
        re, _ = O.transport_rhs(grid, ne, ne, phi, 0.0, 0.0, 380.0, 0.0, (0.0, 0.0, 0.0))
        lam = O.ionization_coefficient(np.array([e0]))[0] * 380.0 * e0
        exact = 380.0 * e0 * 1e12 * prof * (-2 * (x - 0.3) / 0.25 ** 2)   # mu_e E dn/dx
        sel = (x > 0.45) & (x < 0.85)
        k = m // 2
        errs.append(np.abs(re[k, k, sel] - lam * ne[k, k, sel] - exact[sel]).max() / np.abs(exact[sel]).max())
    assert np.log2(errs[0] / errs[1]) > 1.8, errs


def test_stable_step_keeps_densities_non_negative():
    shape = (10, 12, 14)
    grid = _grid(shape)
    rng = np.random.default_rng(7)
    ne = np.where(rng.uniform(size=shape) > 0.7, 1e13, 0.0)         # sharp, non-negative
    npos = ne[::-1].copy()
    phi = 2e4 * random_field(60, shape)
    mu_e, mu_p, dd = 380.0, 3.4, (2190.0, 2190.0, 1800.0)
    ef = O.face_fields(grid, phi, 0.0, 2e4)
    rate = sum(mu_e * np.abs(e).max() / h + 2 * d / h ** 2 for e, h, d in zip(ef, (grid.hx, grid.hy, grid.hz), dd))
    tau = 0.4 / rate
    args = (phi, 0.0, 2e4, mu_e, mu_p, dd)
    he, hp = O.transport_stage(grid, ne, npos, ne, npos, *args, 0.5 * tau)
    e1, p1 = O.transport_stage(grid, ne, npos, he, hp, *args, tau)
    assert e1.min() >= -1e-6 * ne.max() and p1.min() >= -1e-6 * npos.max()


def _linear_between_plates(shape, g_b, g_t, lz=1.0):
    """phi_k = g_b + (g_t - g_b) z_k / lz at the cell centres z_k = (k + 1/2) hz:
    the exact discrete potential for constant a, f = 0 and plate data g_b, g_t."""
    grid = _grid(shape, (1.0, 1.0, lz))
    z = (np.arange(shape[0]) + 0.5) * grid.hz
    phi = np.broadcast_to((g_b + (g_t - g_b) * z / lz)[:, None, None], shape).copy()
    return grid, phi


def test_face_fields_at_the_plates_and_side_walls():
    """Plate faces use the Dirichlet ghost 2g - phi_p (Sec. 2.2 ghost cells; the
    potential's plate condition of Sec. 2), side-wall faces the mirror ghost of
    the homogeneous Neumann condition.  With phi linear between the plates, every
    z face, both plate faces included, carries -(g_t - g_b)/lz; a ghost g - phi
    would give -(g_b + s)/hz and (g_t - s)/hz on the plates (s the potential
    step of one cell), so both plate data are non-zero here.  A side-wall face
    carries no field whatever phi is."""
    g_b, g_t, lz = 3.0, -5.0, 2.0
    shape = (9, 4, 5)
    grid, phi = _linear_between_plates(shape, g_b, g_t, lz)
    fx, fy, fz = O.face_fields(grid, phi, g_b, g_t)
    assert fz.shape == (10, 4, 5)
    np.testing.assert_allclose(fz, -(g_t - g_b) / lz, rtol=1e-13)
    np.testing.assert_array_equal(fx, 0.0)
    np.testing.assert_array_equal(fy, 0.0)
    # side walls under a potential that varies along every axis
    rng = np.random.default_rng(11)
    phi = rng.standard_normal(shape)
    fx, fy, fz = O.face_fields(grid, phi, g_b, g_t)
    assert fx.shape == (9, 4, 6) and fy.shape == (9, 5, 5)
    for wall in (fx[:, :, 0], fx[:, :, -1], fy[:, 0, :], fy[:, -1, :]):
        np.testing.assert_array_equal(wall, 0.0)
    # a plate face by hand: bottom ghost 2 g_b - phi_0, top ghost 2 g_t - phi_{m-1}
    np.testing.assert_allclose(fz[0], -(phi[0] - (2 * g_b - phi[0])) / grid.hz, rtol=1e-14)
    np.testing.assert_allclose(fz[-1], -((2 * g_t - phi[-1]) - phi[-1]) / grid.hz, rtol=1e-14)


def _drift_only(grid, ne, npos, phi, g_b, g_t, mu_e, mu_p):
    """transport_rhs with the diffusion off, in a field weak enough (|E| <= 2 kV/cm)
    that the ionization source alpha(|E|) mu_e |E| n_e is below 1e-40 of the
    density per second (alpha = 5.7 P exp(-260 P/|E|), Sec. 5.2): what is left
    is the drift -div(v n) alone."""
    ex, ey, ez = O.field_from_potential(grid, phi, g_b, g_t)
    eabs = np.sqrt(ex * ex + ey * ey + ez * ez).max()
    assert eabs <= 2.0e3
    assert 5.7 * 760.0 * np.exp(-260.0 * 760.0 / eabs) * mu_e * eabs < 1e-40
    return O.transport_rhs(grid, ne, npos, phi, g_b, g_t, mu_e, mu_p, (0.0, 0.0, 0.0))


def test_drift_through_the_plates_with_neumann_density_ghosts():
    """Drift across the plates.  The densities take homogeneous Neumann ghosts
    at every boundary (the model's conditions, Sec. 2: all boundaries for n_e,
    the inflow boundaries for n_p), so a face on a plate carries the upwind
    ghost's density, and the MUSCL slope of a boundary cell is zero (one of its
    two differences vanishes).  With phi linear between the plates the field is
    E_z = -(g_t - g_b)/lz on every z face, plates included.  Electrons drift
    at v_e = -mu_e E_z (up for g_t > g_b), ions at v_p = mu_p E_z (down).

    For n_k = n0 + c k (k = 0..m-1) the fluxes are worked out by hand:
    electrons (upwind below): F_0 = F_1 = v n_0, F_k = v (n_{k-1} + c/2) for
    2 <= k <= m-1, F_m = v n_{m-1}; ions (upwind above): F_0 = v n_0,
    F_k = v (n_k - c/2) for 1 <= k <= m-2, F_{m-1} = F_m = v n_{m-1}.  So
    -div(v n) per cell is, bottom to top, electrons: 0, -3vc/2h, -vc/h ...,
    -vc/2h; ions: -vc/2h, -vc/h ..., -3vc/2h, 0.  A plate that lets no flux
    through, or a plate ghost g - phi in the field, fails the end cells."""
    m = 10
    shape = (m, 3, 4)
    g_b, g_t = 200.0, 1200.0
    grid, phi = _linear_between_plates(shape, g_b, g_t)
    h = grid.hz
    mu_e, mu_p = 380.0, 3.4
    ez = -(g_t - g_b)
    c, n0 = 4.0e10, 1.0e12
    k = np.arange(m, dtype=np.float64)
    nk = np.broadcast_to((n0 + c * k)[:, None, None], shape).copy()
    de, dp = _drift_only(grid, nk, nk, phi, g_b, g_t, mu_e, mu_p)
    ve, vp = -mu_e * ez, mu_p * ez
    assert ve > 0 > vp
    want_e = np.full(m, -ve * c / h)
    want_e[0], want_e[1], want_e[-1] = 0.0, -1.5 * ve * c / h, -0.5 * ve * c / h
    want_p = np.full(m, -vp * c / h)
    want_p[0], want_p[-2], want_p[-1] = -0.5 * vp * c / h, -1.5 * vp * c / h, 0.0
    scale = abs(ve) * c / h
    np.testing.assert_allclose(de, np.broadcast_to(want_e[:, None, None], shape), rtol=0,
                               atol=1e-12 * scale)
    np.testing.assert_allclose(dp, np.broadcast_to(want_p[:, None, None], shape), rtol=0,
                               atol=1e-12 * abs(vp) * c / h)
    # a uniform density: the plate inflow carries the ghost's density, so no cell changes
    flat = np.full(shape, n0)
    de, dp = _drift_only(grid, flat, flat, phi, g_b, g_t, mu_e, mu_p)
    np.testing.assert_allclose(de, 0.0, atol=1e-13 * ve * n0 / h)
    np.testing.assert_allclose(dp, 0.0, atol=1e-13 * abs(vp) * n0 / h)


def test_drift_against_the_side_walls():
    """Drift towards a side wall.  phi = -e0 x gives E_x = e0 on the interior
    x faces and none on the walls (mirror ghost of the Neumann condition), so
    nothing crosses a wall.  Electrons move at v = -mu_e e0 (towards x = 0),
    ions at mu_p e0 (away from it).  For n_i = n0 + c i and electrons (upwind
    on the right): F_i = v (n_i - c/2) for 1 <= i <= m-2, F_{m-1} = v n_{m-1},
    walls 0; so -div(v n) is -v (n_0 + c/2)/h in the first cell (inflow piles
    up at the wall), -v c/h inside, -3vc/2h in cell m-2 and v n_{m-1}/h in the
    last cell (outflow, no inflow).  Ions (upwind on the left): F_1 = v n_0,
    F_i = v (n_{i-1} + c/2) for 2 <= i <= m-1; -div: -v n_0/h, -3vc/2h, -vc/h
    ..., and v (n_{m-2} + c/2)/h in the last cell.  The plates (phi = 0 there,
    so their faces carry a field) are kept out: layers 1..m-2 only."""
    m = 11
    grid, phi, e0 = _uniform_field_case(m=m, e0=50.0)
    h = grid.hx
    mu_e, mu_p = 380.0, 3.4
    c, n0 = 3.0e10, 1.0e12
    n = n0 + c * np.arange(m, dtype=np.float64)
    dens = np.broadcast_to(n, grid.shape).copy()
    de, dp = _drift_only(grid, dens, dens, phi, 0.0, 0.0, mu_e, mu_p)
    de, dp = de[1:-1], dp[1:-1]
    v = -mu_e * e0
    want_e = np.full(m, -v * c / h)
    want_e[0] = -v * (n[0] + 0.5 * c) / h
    want_e[-2] = -1.5 * v * c / h
    want_e[-1] = v * n[-1] / h
    u = mu_p * e0
    want_p = np.full(m, -u * c / h)
    want_p[0] = -u * n[0] / h
    want_p[1] = -1.5 * u * c / h
    want_p[-1] = u * (n[-2] + 0.5 * c) / h
    np.testing.assert_allclose(de, np.broadcast_to(want_e, de.shape), rtol=1e-12, atol=1e-12 * abs(v) * c / h)
    np.testing.assert_allclose(dp, np.broadcast_to(want_p, dp.shape), rtol=1e-12, atol=1e-12 * u * c / h)


def test_semi_implicit_step_on_a_neutral_uniform_plasma():
    """The whole step of eqs. (e1)-(e2) in closed form.  Uniform n_e = n_p = n0:
    eq. (semi2) gives f = 0 and a constant coefficient, so the discrete
    potential is linear between the plates (exact for e18 with the 2g - phi
    ghost); E_z = -phi_0 on every face and cell; the drift of a uniform
    density cancels in every cell (Neumann ghosts at the plates), diffusion
    vanishes, and only the ionization source lam n_e = alpha(|E|) mu_e |E| n_e
    acts, so the predictor-corrector gives n_e (1 + tau lam + (tau lam)^2/2) and
    n_p + tau lam n_e (1 + tau lam/2) in every cell, boundary cells included."""
    from streamer_inputs import MU_E, MU_P, DIFFUSION, PHI0
    shape = (16, 8, 8)
    n0 = 5.0e13
    ne = np.full(shape, n0)
    npos = np.full(shape, n0)
    tau = 2e-12
    params = O.OracleParams(coarse_min=4, phi_top=PHI0, rtol=1e-13)
    e_over = O.ELEMENTARY_CHARGE / O.VACUUM_PERMITTIVITY_CM
    ne1, np1, phi, info = O.semi_implicit_step(params, ne, npos, tau, MU_E, MU_P, DIFFUSION, e_over)
    assert info.converged
    _, lin = _linear_between_plates(shape, 0.0, PHI0)
    np.testing.assert_allclose(phi, lin, rtol=0, atol=1e-10 * PHI0)
    lam = IONIZATION_RATE(PHI0, abs(MU_E))
    tl = tau * lam
    assert 1e-4 < tl < 1e-1
    np.testing.assert_allclose(ne1, n0 * (1 + tl + 0.5 * tl * tl), rtol=1e-12)
    np.testing.assert_allclose(np1, n0 + tl * n0 * (1 + 0.5 * tl), rtol=1e-12)


def IONIZATION_RATE(e_abs, mu_e):
    """alpha(|E|) mu_e |E| with alpha = 5.7 P exp(-260 P/|E|) cm^-1, P = 760 Torr
    (Sec. 5.2), written out for the closed-form step."""
    return 5.7 * 760.0 * np.exp(-260.0 * 760.0 / e_abs) * mu_e * e_abs

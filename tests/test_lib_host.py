"""Host-side checks of libgmg that need no GPU: the library loads, exports
every entry point declared in include/gmg.h, validates parameters before any
device work, and computes the Chebyshev eigen estimate's lam_hat (Sec. 3.2)
from a small Hessenberg matrix like numpy does."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1812_08606_gb300 import build, gmg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return gmg.load()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "gmg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?[\s\*])([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "return")))


def test_header_symbols_exported(lib):
    names = _declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    # the Python binding uses the same names
    for name in names:
        assert hasattr(gmg, name), name


def test_default_params_follow_the_paper(lib):
    p = gmg.gmg_default_params(64, 64, 80)
    assert (p.nx, p.ny, p.nz) == (64, 64, 80)
    assert p.rtol == 1e-8 and p.eig_steps == 10 and p.eig_hi == 1.1 and p.eig_lo == 0.1
    assert p.cheb_steps == 3 and p.coarse_min == 4 and p.restart == 20
    assert p.precision == gmg.GMG_PREC_MIXED and p.smoother_pc == gmg.GMG_PC_SGS


@pytest.mark.parametrize("change", [
    dict(nx=12, ny=12, nz=10),           # does not halve down to coarse_min
    dict(nx=0),
    dict(lx=0.0),
    dict(cheb_steps=0),
    dict(restart=64),
    dict(rtol=0.0),
    dict(eig_hi=0.05),
    dict(precision=7),
    dict(smoother_pc=3),
    dict(nx=256, ny=256, nz=256, coarse_min=32),   # dense coarsest grid too large
])
def test_invalid_params_rejected_before_device_work(lib, change):
    p = gmg.gmg_default_params(32, 32, 32)
    for k, v in change.items():
        setattr(p, k, v)
    out = ctypes.c_void_p()
    # a_dev is never dereferenced when validation fails
    st = lib.gmg_setup(ctypes.byref(p), ctypes.c_void_p(16), None, ctypes.byref(out))
    assert st == gmg.GMG_ERR_ARG and not out.value


def test_status_strings(lib):
    for s in range(7):
        assert gmg.status_string(s)
    assert "converged" in gmg.status_string(gmg.GMG_ERR_NOT_CONVERGED)


def test_hessenberg_max_eig_matches_numpy(lib):
    rng = np.random.default_rng(5)
    for m in (1, 2, 3, 5, 10, 17, 32):
        for trial in range(20):
            H = np.triu(rng.standard_normal((m, m)), -1)
            if trial % 3 == 0:                       # nearly symmetric, like Arnoldi on B^{-1}A
                H = np.triu(H + H.T, -1) + np.diag(rng.uniform(0, 2, m))
                H = np.triu(H, -1)
            ref = np.linalg.eigvals(H).real.max()
            got = gmg.gmg_hessenberg_max_real_eig(H)
            assert got == pytest.approx(ref, rel=1e-10, abs=1e-12 * np.abs(H).max()), (m, trial)


def test_hessenberg_from_arnoldi_of_sgs_operator(lib):
    """The matrix the set-up sees: 10-step Arnoldi of B^{-1} A from the oracle."""
    from oracle import gmg_oracle as O
    from streamer_inputs import random_coefficient
    grid = O.Grid(8, 8, 8)
    a = random_coefficient(3, grid.shape, 1e3)
    params = O.OracleParams()

    def mv(v):
        return O.sgs_redblack(grid, a, O.apply_operator(grid, a, v.reshape(grid.shape)))

    H = O.arnoldi_hessenberg(mv, O.hash_start_vector(grid.size), 10)
    assert gmg.gmg_hessenberg_max_real_eig(H) == pytest.approx(np.linalg.eigvals(H).real.max(), rel=1e-13)
    del params

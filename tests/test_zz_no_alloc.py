"""The allocation-free coarsest-grid solve against the context-based one.

gmg_coarse_solve_noalloc serves callers that cannot allocate device memory;
its scratch is a fixed array inside the library.  Here it must reproduce
gmg_coarse_solve (the direct solve that gmg_setup prepares with allocated
scratch) on two calls in a row, so a second call is not disturbed by what the
first left in the shared array.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1812_08606_gb300 import build, gmg  # noqa: E402
from streamer_inputs import random_coefficient, random_field  # noqa: E402

DEV = torch.device("cuda:0")
TOL = 1e-12   # FP64 kernels: the same dense factorisation, different scratch


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    gmg.load()


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV, torch.float64)


def _coarse_case(shape, coarse_min, seed, lengths=(1.0, 1.0, 1.0)):
    nz, ny, nx = shape
    # the allocation-free solve takes a cell coefficient (eq. (e18)), so the
    # context keeps cell coefficients on its coarse levels (8-child means)
    p = gmg.gmg_default_params(nx, ny, nz, coarse_min=coarse_min, precision=gmg.GMG_PREC_FP64,
                               lx=lengths[0], ly=lengths[1], lz=lengths[2], coarsening=gmg.GMG_COARSEN_MEAN)
    ctx = gmg.gmg_setup(p, _t(random_coefficient(seed, shape, contrast=1e3)))
    info = gmg.gmg_level_info(ctx, 0)
    cshape = info["shape"]
    a0 = torch.empty(cshape, dtype=torch.float64, device=DEV)
    gmg.gmg_level_coefficient(ctx, 0, a0)
    cp = gmg.gmg_default_params(cshape[2], cshape[1], cshape[0], lx=lengths[0], ly=lengths[1], lz=lengths[2])
    return ctx, a0, cp, cshape


@pytest.mark.parametrize("shape,coarse_min,lengths", [((32, 32, 32), 8, (1.0, 1.0, 1.0)),
                                                      ((16, 24, 40), 2, (1.0, 0.7, 1.3))])
def test_noalloc_coarse_solve_matches_context_solve_twice(shape, coarse_min, lengths):
    ctx, a0, cp, cshape = _coarse_case(shape, coarse_min, 500, lengths)
    ctx2, a02, cp2, cshape2 = _coarse_case(shape, coarse_min, 501, lengths)
    for call, (c, a, p, s) in enumerate(((ctx, a0, cp, cshape), (ctx2, a02, cp2, cshape2))):
        b = _t(random_field(510 + call, s) * 100)
        x_ref = torch.empty(s, dtype=torch.float64, device=DEV)
        gmg.gmg_coarse_solve(c, b, x_ref)
        x = torch.full(s, float("nan"), dtype=torch.float64, device=DEV)
        gmg.gmg_coarse_solve_noalloc(p, a, b, x)
        torch.cuda.synchronize()
        err = float((x - x_ref).norm() / x_ref.norm())
        assert err < TOL, (call, err)


def test_noalloc_rejects_sizes_beyond_the_scratch():
    lib = gmg.load()
    p = gmg.gmg_default_params(16, 8, 8)   # 1024 unknowns > 512
    assert p.nx * p.ny * p.nz > gmg.GMG_NOALLOC_MAX_UNKNOWNS
    buf = torch.zeros(p.nx * p.ny * p.nz, dtype=torch.float64, device=DEV)
    st = lib.gmg_coarse_solve_noalloc(ctypes.byref(p), buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), None)
    assert st == gmg.GMG_ERR_ARG


@pytest.mark.parametrize("field,value", [("lx", float("inf")), ("lz", float("nan")), ("ly", 0.0)])
def test_noalloc_rejects_lengths_that_are_not_positive_and_finite(field, value):
    """An infinite length would make the face coefficients vanish silently;
    the call refuses it, as gmg_setup does."""
    lib = gmg.load()
    p = gmg.gmg_default_params(4, 4, 4)
    setattr(p, field, value)
    buf = torch.ones(64, dtype=torch.float64, device=DEV)
    st = lib.gmg_coarse_solve_noalloc(ctypes.byref(p), buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), None)
    assert st == gmg.GMG_ERR_ARG

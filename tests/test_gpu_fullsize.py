"""Full-size checks in the benchmark's own configuration (512^3 two-channel
streamer, contrast 1e4, mixed precision, default parameters).

The oracle cannot run the 512^3 solve in test time, so the checks are
properties that hold at any size, computed by the oracle on the CPU from the
GPU's output: the true FP64 relative residual of phi (eq. (criterion)) is
below 1e-8, and the FP32 field equals the oracle's central differences of the
same phi to FP32 accuracy.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import gmg_oracle as O  # noqa: E402
from streamer_inputs import make_inputs  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1812_08606_gb300 import build, gmg  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    gmg.load()


def test_twochannel512_solve_and_field_properties():
    inp = make_inputs("twochannel512")
    a, f = inp["a"], inp["f"]
    n = a.shape[0]
    p = gmg.gmg_default_params(n, n, n)
    ctx = gmg.gmg_setup(p, torch.from_numpy(a).to(DEV))
    phi = torch.zeros(a.shape, dtype=torch.float64, device=DEV)
    info = gmg.fgmres_solve(ctx, torch.from_numpy(f).to(DEV), phi)
    e = [torch.empty(a.shape, dtype=torch.float32, device=DEV) for _ in range(3)]
    gmg.field_from_potential(ctx, phi, *e)
    torch.cuda.synchronize()
    assert info.converged and info.true_rel_residual < 1e-8
    phi_h = phi.cpu().numpy()
    grid = O.Grid(n, n, n)
    b = O.assemble_rhs(grid, a, f, p.phi_bottom, p.phi_top)
    rel = np.linalg.norm(b - O.apply_operator(grid, a, phi_h)) / np.linalg.norm(b)
    print(f"512^3: {info.iterations} iterations, library true residual {info.true_rel_residual:.3e}, "
          f"oracle true residual {rel:.3e}")
    assert rel < 1e-8
    assert rel == pytest.approx(info.true_rel_residual, rel=1e-3)
    del b
    ref = O.field_from_potential(grid, phi_h, p.phi_bottom, p.phi_top)
    for got, r in zip(e, ref):
        g = got.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(g - r) / np.linalg.norm(r) < 1e-6
        assert np.abs(g - r).max() < 1e-5 * np.abs(r).max()


# The fused smoother hands out whole tile columns (one resident block per SM)
# before it splits the leftover columns into z-segments.  The grids of the
# kernel-level parity tests have fewer tiles than blocks, so only the split
# runs there.  On this grid the finest level runs on the copy-fed kernel (56 x
# 20 tiles): 19 x 26 = 494 tiles, so on 152 SMs every block takes 3 whole
# columns first and the 38 left over are split.
SPLIT_SHAPE = (64, 512, 1024)          # (nz, ny, nx); coarsest 2 x 16 x 32 with coarse_min 2
LAM_MAX, LAM_MIN = 1.0989, 0.0999       # one interval, given to both sides


def _tiles(shape):
    nz, ny, nx = shape
    return -(-nx // 56) * -(-ny // 20)


def _maxrel(x, ref):
    return float(np.abs(x - ref).max() / np.abs(ref).max())


@pytest.fixture(scope="module")
def split_case():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tiles = _tiles(SPLIT_SHAPE)
    assert tiles // sms >= 1 and tiles % sms != 0, (tiles, sms)
    a = make_inputs("twochannel512", shape=SPLIT_SHAPE)["a"]
    nz, ny, nx = SPLIT_SHAPE
    p = gmg.gmg_default_params(nx, ny, nz, coarse_min=2, precision=gmg.GMG_PREC_MIXED)
    ctx = gmg.gmg_setup(p, torch.from_numpy(a).to(DEV))
    for lev in range(1, gmg.gmg_num_levels(ctx)):
        gmg.gmg_level_set_bounds(ctx, lev, LAM_MAX, LAM_MIN)
    return ctx, a, p


def test_fused_smoother_whole_column_split_elementwise(split_case):
    """Three Chebyshev + red-black SSOR steps on the finest level of the split
    grid, from zero and from a given x, against the oracle on the same
    FP32-rounded inputs, cell by cell."""
    ctx, a, p = split_case
    lev = gmg.gmg_num_levels(ctx) - 1
    rng = np.random.default_rng(4242)
    q = lambda v: v.astype(np.float32).astype(np.float64)   # noqa: E731
    b = q(rng.uniform(-1, 1, SPLIT_SHAPE))
    x0 = q(rng.uniform(-1, 1, SPLIT_SHAPE))
    nz, ny, nx = SPLIT_SHAPE
    grid = O.Grid(nx, ny, nz)
    for x_is_zero in (True, False):
        x = torch.from_numpy(x0).to(DEV, torch.float32)
        gmg.gmg_level_smooth(ctx, lev, torch.from_numpy(b).to(DEV, torch.float32), x, x_is_zero)
        got = x.cpu().numpy().astype(np.float64)
        ref = O.chebyshev_smooth(grid, q(a), b, None if x_is_zero else x0, LAM_MAX, LAM_MIN, p.cheb_steps, "sgs")
        err = _maxrel(got, ref)
        print(f"split smoother x_is_zero={x_is_zero}: max element error {err:.2e} of max |ref|")
        assert err < 2e-5, (x_is_zero, err)


def test_vcycle_whole_column_split_elementwise(split_case):
    """One mixed-precision V-cycle on the split grid against the oracle's
    V-cycle with the same Chebyshev intervals, cell by cell."""
    ctx, a, p = split_case
    L = gmg.gmg_num_levels(ctx)
    nz, ny, nx = SPLIT_SHAPE
    params = O.OracleParams(coarse_min=2)
    levels = [O.Level(O.Grid(nx, ny, nz), a)]
    for _ in range(L - 1):
        prev = levels[-1]
        levels.append(O.Level(prev.grid.coarser(), O.coarsen_level(prev.a, params)))
    hier = O.Hierarchy(params, list(reversed(levels)))
    for lev in hier.levels[1:]:
        lev.lam_max, lev.lam_min = LAM_MAX, LAM_MIN
    c = hier.levels[0]
    import scipy.linalg
    hier.coarse_chol = scipy.linalg.cho_factor(O.dense_operator(c.grid, c.a), lower=True)
    v = np.random.default_rng(4343).uniform(-1, 1, SPLIT_SHAPE)
    z = torch.empty(SPLIT_SHAPE, dtype=torch.float64, device=DEV)
    gmg.gmg_apply_preconditioner(ctx, torch.from_numpy(v).to(DEV), z)
    got = z.cpu().numpy()
    ref = O.vcycle(hier, v.astype(np.float32).astype(np.float64))
    err = _maxrel(got, ref)
    l2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"split V-cycle: max element error {err:.2e} of max |ref|, l2 {l2:.2e}")
    assert l2 < 1e-4 and err < 1e-3

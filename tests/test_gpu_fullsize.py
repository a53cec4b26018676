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

"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Element-by-element comparisons on seeded inputs, kernel by kernel (operator,
smoother preconditioner, Chebyshev smoothing, fused residual + restriction,
prolongation, coarse solve), then the V-cycle, then whole solves.

Tolerances: FP64 kernels agree with the oracle to ~1e-13 relative (different
summation order only).  FP32 kernels are compared with the oracle evaluated
on the same FP32-rounded inputs, to a few FP32 ulps scaled by the stencil's
cancellation (5e-5 relative to the operator norm).  FP64 solves must match the
oracle's phi within 1e-10 relative with the same iteration count; every solve
must reach a true FP64 residual below 1e-8.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import gmg_oracle as O  # noqa: E402
from streamer_inputs import (make_inputs, random_coefficient, random_field, streamer_densities,  # noqa: E402
                             MU_E, MU_P, DIFFUSION, PHI0)

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1812_08606_gb300 import gmg  # noqa: E402

DEV = torch.device("cuda:0")
RAGGED = (16, 24, 40)     # (nz, ny, nx): x not a multiple of the 32-wide tile; coarsest 2 x 3 x 5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1812_08606_gb300 import build
    build.build()
    gmg.load()


def _t(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV, dtype)


def _np(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def _params(shape, **kw):
    nz, ny, nx = shape
    return gmg.gmg_default_params(nx, ny, nz, **kw)


def _ogrid(shape, p=None):
    nz, ny, nx = shape
    if p is None:
        return O.Grid(nx, ny, nz)
    return O.Grid(nx, ny, nz, p.lx, p.ly, p.lz)


def _rel(x, ref):
    return np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300)


def _maxrel(x, ref):
    """Largest element-wise difference, relative to the largest |ref|."""
    return float(np.abs(np.asarray(x) - np.asarray(ref)).max() / max(np.abs(ref).max(), 1e-300))


# An element-wise bound beside every relative-norm bound: a norm can hide a few
# wrong cells (a plate row, a tile seam) in a large grid, a maximum cannot.
ELEMENT_FACTOR = 10.0


def _close(x, ref, tol, what=""):
    """Relative L2 error below tol and every element within ELEMENT_FACTOR * tol
    of the largest |ref|; returns (l2, max) for printing."""
    l2, mx = _rel(x, ref), _maxrel(x, ref)
    assert l2 < tol, (what, "l2", l2, tol)
    assert mx < ELEMENT_FACTOR * tol, (what, "max", mx, ELEMENT_FACTOR * tol)
    return l2, mx


def _oracle_hierarchy(a, p):
    op = O.OracleParams(lx=p.lx, ly=p.ly, lz=p.lz, phi_bottom=p.phi_bottom, phi_top=p.phi_top,
                        coarse_min=p.coarse_min, cheb_steps=p.cheb_steps, restart=p.restart,
                        max_iters=p.max_iters, rtol=p.rtol, eig_steps=p.eig_steps, eig_hi=p.eig_hi,
                        eig_lo=p.eig_lo, prolongation=["trilinear", "constant", "opdep"][p.prolongation],
                        smoother_pc=["sgs", "jacobi", "identity"][p.smoother_pc],
                        cycle=["v", "fmg", "auto"][p.cycle], coarsening=["mean", "series"][p.coarsening])
    return op


def _olevels(a, p):
    """The oracle's operator of every level (index 0 = coarsest, as the
    library numbers them): the cell coefficient on the finest level and, below,
    what the context's coarsening makes of it (FaceCoefficients or 8-child
    means)."""
    op = _oracle_hierarchy(a, p)
    ops = [a]
    for _ in range(O.level_count(p.nx, p.ny, p.nz, p.coarse_min) - 1):
        ops.append(O.coarsen_level(ops[-1], op))
    return ops[::-1]


def _q32(op):
    """The FP32 rounding of an operator (cell coefficient or faces), in FP64."""
    r = lambda v: v.astype(np.float32).astype(np.float64)   # noqa: E731
    if isinstance(op, O.FaceCoefficients):
        return O.FaceCoefficients(r(op.ax), r(op.ay), r(op.az), r(op.bottom), r(op.top))
    return r(op)


def _face_entries(grid, op):
    """(kx, ky, kz, ktop) of an oracle operator in the library's face layout:
    matrix entries of each cell's low faces, the bottom plate at k = 0."""
    cx, cy, cz = O.face_coefficients(grid, op)
    pb, pt = O.plate_coefficients(grid, op)
    kx = np.zeros(grid.shape)
    kx[:, :, 1:] = cx
    ky = np.zeros(grid.shape)
    ky[:, 1:, :] = cy
    kz = np.empty(grid.shape)
    kz[1:] = cz
    kz[0] = pb
    return kx, ky, kz, pt


# ---------------------------------------------------------------------------
# Operator and right-hand side
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("shape,lengths", [(RAGGED, (1.0, 1.0, 1.0)), ((32, 32, 32), (0.5, 1.5, 1.0)),
                                           ((8, 8, 10), (1.0, 1.0, 1.25))])
def test_apply_operator_and_rhs_fp64(shape, lengths):
    a = random_coefficient(101, shape, contrast=1e3)
    x = random_field(102, shape)
    f = random_field(103, shape)
    cm = 2 if shape == RAGGED else 4
    p = _params(shape, coarse_min=cm, lx=lengths[0], ly=lengths[1], lz=lengths[2], phi_bottom=0.3, phi_top=-2.0)
    ctx = gmg.gmg_setup(p, _t(a))
    y = torch.empty(shape, dtype=torch.float64, device=DEV)
    gmg.apply_operator(ctx, _t(x), y)
    grid = _ogrid(shape, p)
    ref = O.apply_operator(grid, a, x)
    _close(_np(y), ref, 1e-14)
    b = torch.empty_like(y)
    gmg.assemble_rhs(ctx, _t(f), b)
    np.testing.assert_allclose(_np(b), O.assemble_rhs(grid, a, f, 0.3, -2.0), rtol=1e-14, atol=1e-12)


@pytest.mark.parametrize("arith,tol", [(gmg.GMG_OUTER_DOUBLE_FLOAT, 2e-14), (gmg.GMG_OUTER_FP64, 1e-15)])
@pytest.mark.parametrize("shape", [RAGGED, (64, 64, 64), (10, 8, 8), (8, 24, 144)])
def test_outer_arnoldi_product(arith, tol, shape):
    """w = A z_j for an FP32 z_j (the mixed-precision Arnoldi product) against
    the FP64 oracle operator on the same z; double-float arithmetic keeps a
    48-bit significand, so it agrees to ~1e-14."""
    a = make_inputs("twochannel512", shape=shape)["a"] if shape[0] >= 16 else random_coefficient(240, shape, 1e4)
    z = random_field(241, shape).astype(np.float32)
    cm = 2 if shape in (RAGGED, (8, 24, 144)) else 4
    p = _params(shape, coarse_min=cm, precision=gmg.GMG_PREC_MIXED, outer_arith=arith)
    ctx = gmg.gmg_setup(p, _t(a))
    w = torch.empty(shape, dtype=torch.float64, device=DEV)
    gmg.gmg_apply_outer(ctx, _t(z, torch.float32), w)
    ref = O.apply_operator(_ogrid(shape), a, z.astype(np.float64))
    err = np.abs(_np(w) - ref).max() / np.abs(ref).max()
    assert err < tol, err


def test_outer_product_pair_and_cell_kernels_agree_bitwise():
    """The double-float product has a cell-pair kernel (even rows, 16-byte
    aligned output) and a one-cell kernel (any other layout) doing the same
    operations per cell; an output offset by one double takes the latter."""
    shape = (8, 24, 144)
    a = random_coefficient(243, shape, 1e4)
    z = random_field(244, shape).astype(np.float32)
    p = _params(shape, coarse_min=2, precision=gmg.GMG_PREC_MIXED, outer_arith=gmg.GMG_OUTER_DOUBLE_FLOAT)
    ctx = gmg.gmg_setup(p, _t(a))
    n = int(np.prod(shape))
    w_pair = torch.empty(shape, dtype=torch.float64, device=DEV)
    gmg.gmg_apply_outer(ctx, _t(z, torch.float32), w_pair)
    buf = torch.empty(n + 1, dtype=torch.float64, device=DEV)
    w_cell = buf[1:].view(shape)
    assert w_cell.data_ptr() % 16 == 8
    gmg.gmg_apply_outer(ctx, _t(z, torch.float32), w_cell)
    assert torch.equal(w_pair, w_cell)


# RAGGED: the fused smoother on the finest (cell-form) level only; (16, 48, 80):
# also on the face-form level below.  eig_steps 10 takes the Chebyshev basis
# and its Gram matrix (11 vectors); 12 is past the Gram kernel's 12 vectors and
# takes FP32 Gram-Schmidt with the fused product.
@pytest.mark.parametrize("shape", [RAGGED, (16, 48, 80)])
@pytest.mark.parametrize("eig_steps", [10, 12])
def test_mixed_eigen_bounds_close_to_fp64(shape, eig_steps):
    """The mixed set-up runs its eigen estimate in FP32 (the bounds only steer
    the FP32 smoother); they agree with the FP64 oracle's Arnoldi to 1e-5."""
    a = random_coefficient(242, shape, contrast=1e3)
    p = _params(shape, coarse_min=2, precision=gmg.GMG_PREC_MIXED, eig_steps=eig_steps)
    ctx = gmg.gmg_setup(p, _t(a))
    hier = O.build_hierarchy(_ogrid(shape), a, _oracle_hierarchy(a, p))
    for lev in range(1, gmg.gmg_num_levels(ctx)):
        info = gmg.gmg_level_info(ctx, lev)
        assert info["lam_max"] == pytest.approx(hier.levels[lev].lam_max, rel=1e-5)
        assert info["lam_min"] == pytest.approx(hier.levels[lev].lam_min, rel=1e-5)


@pytest.mark.parametrize("coarsening", [gmg.GMG_COARSEN_SERIES, gmg.GMG_COARSEN_MEAN])
@pytest.mark.parametrize("prec", [gmg.GMG_PREC_FP64, gmg.GMG_PREC_MIXED])
def test_level_coefficients_and_operators(prec, coarsening):
    """Every level's operator against the oracle's: the 8-child means or the
    series-parallel faces element by element (the face entries of the
    finest, cell-coefficient level too), and y = A_l x."""
    shape = RAGGED
    a = random_coefficient(104, shape, contrast=1e3)
    p = _params(shape, coarse_min=2, precision=prec, coarsening=coarsening)
    ctx = gmg.gmg_setup(p, _t(a))
    L = gmg.gmg_num_levels(ctx)
    assert L == 4
    ops = _olevels(a, p)
    dt = ctx.level_dtype
    fp32 = dt == torch.float32
    for lev in range(L - 1, -1, -1):
        info = gmg.gmg_level_info(ctx, lev)
        s = info["shape"]
        g = _ogrid(s)
        op = ops[lev]
        if not isinstance(op, O.FaceCoefficients):
            assert s == op.shape
            ac = torch.empty(s, dtype=torch.float64, device=DEV)
            gmg.gmg_level_coefficient(ctx, lev, ac)
            np.testing.assert_allclose(_np(ac), op, rtol=1e-15)
        else:
            with pytest.raises(gmg.GMGError):
                gmg.gmg_level_coefficient(ctx, lev, torch.empty(s, dtype=torch.float64, device=DEV))
        ftol = 5e-6 if (fp32 and isinstance(op, O.FaceCoefficients)) else 1e-14
        for got, want, name in zip(gmg.gmg_level_faces(ctx, lev), _face_entries(g, op), "xyzt"):
            got = _np(got)
            assert np.all(np.abs(got - want) <= ftol * np.abs(want) + 1e-300), (lev, name)
        x = random_field(105 + lev, s)
        xin = x.astype(np.float32).astype(np.float64) if fp32 else x
        y = torch.empty(s, dtype=dt, device=DEV)
        gmg.gmg_level_apply(ctx, lev, _t(xin, dt), y)
        ref = O.apply_operator(g, _q32(op) if fp32 else op, xin)
        tol = 1e-14 if dt == torch.float64 else 5e-6
        _close(_np(y), ref, tol, lev)


# ---------------------------------------------------------------------------
# Smoother
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("prec", [gmg.GMG_PREC_FP64, gmg.GMG_PREC_MIXED])
@pytest.mark.parametrize("pc", [gmg.GMG_PC_SGS, gmg.GMG_PC_JACOBI, gmg.GMG_PC_IDENTITY])
def test_smoother_preconditioner_and_chebyshev(prec, pc):
    shape = RAGGED
    a = random_coefficient(110, shape, contrast=1e2)
    p = _params(shape, coarse_min=2, precision=prec, smoother_pc=pc)
    op = _oracle_hierarchy(a, p)
    ctx = gmg.gmg_setup(p, _t(a))
    dt = ctx.level_dtype
    fp32 = dt == torch.float32
    q = _q32 if fp32 else (lambda v: v)
    tol = 2e-5 if fp32 else 1e-13
    # the oracle's own bounds drive both sides' Chebyshev steps
    hier = O.build_hierarchy(_ogrid(shape), a, op)
    for lev in range(gmg.gmg_num_levels(ctx) - 1, 0, -1):
        oa = hier.levels[lev].a
        gmg.gmg_level_set_bounds(ctx, lev, hier.levels[lev].lam_max, hier.levels[lev].lam_min)
        info = gmg.gmg_level_info(ctx, lev)
        s = info["shape"]
        g = _ogrid(s)
        r = q(random_field(111 + lev, s))
        z = torch.empty(s, dtype=dt, device=DEV)
        gmg.gmg_level_smoother_pc(ctx, lev, _t(r, dt), z)
        ref = O.smoother_preconditioner(g, q(oa), r, op.smoother_pc)
        _close(_np(z), ref, tol, ("pc", lev))
        # Chebyshev from zero and from a given x, with the oracle's bounds
        b = q(random_field(121 + lev, s))
        x0 = q(random_field(131 + lev, s))
        for x_is_zero in (True, False):
            x = _t(x0, dt)
            gmg.gmg_level_smooth(ctx, lev, _t(b, dt), x, x_is_zero)
            lv = hier.levels[lev]
            ref = O.chebyshev_smooth(g, q(oa), b, None if x_is_zero else x0, lv.lam_max, lv.lam_min,
                                     p.cheb_steps, op.smoother_pc)
            _close(_np(x), ref, 5 * tol, ("cheb", lev, x_is_zero))


# A Chebyshev interval for smoother-only checks: the SSOR-preconditioned
# spectrum lies in (0, 1], and 1.1 x / 0.1 x of a Ritz value near 1 is what
# the set-up finds (Sec. 3.2).
FIXED_LAM_MAX, FIXED_LAM_MIN = 1.0989, 0.0999


@pytest.mark.parametrize("shape,cm", [((48, 40, 72), 5), ((64, 64, 64), 4), (RAGGED, 2), ((8, 28, 64), 2)])
def test_fused_smoother_matches_separate_kernels_and_oracle(shape, cm):
    """The fused one-pass Chebyshev + red-black SSOR step against the
    separate residual / half-sweep kernels and the oracle, on grids with
    partial tiles and several z-chunks.  smoother_kernel 0 runs the finest
    level of the 48 x 40 x 72, 64^3 and 8 x 28 x 64 grids on the kernel fed by
    bulk-tensor copies (56 x 20 tiles; 8 x 28 x 64 is near the smallest grid it
    takes: 4 tiles, 8 blocks with 4 planes each) and 2 the same step without
    them (56 x 18 tiles): the same arithmetic in the same order, so the two
    agree bit for bit."""
    a = make_inputs("twochannel512", shape=shape)["a"]
    ctxs = [gmg.gmg_setup(_params(shape, coarse_min=cm, smoother_kernel=k), _t(a)) for k in (0, 1, 2)]
    ops = _olevels(a, ctxs[0].params)
    for lev in range(gmg.gmg_num_levels(ctxs[0]) - 1, 0, -1):
        oa = _q32(ops[lev])
        for ctx in ctxs:   # one interval, given from outside, for every side
            gmg.gmg_level_set_bounds(ctx, lev, FIXED_LAM_MAX, FIXED_LAM_MIN)
        info = gmg.gmg_level_info(ctxs[0], lev)
        s = info["shape"]
        b = random_field(300 + lev, s).astype(np.float32)
        x0 = random_field(310 + lev, s).astype(np.float32)
        for x_is_zero in (True, False):
            outs = []
            for ctx in ctxs:
                x = _t(x0, torch.float32)
                gmg.gmg_level_smooth(ctx, lev, _t(b, torch.float32), x, x_is_zero)
                outs.append(_np(x))
            ref = O.chebyshev_smooth(_ogrid(s), oa, b.astype(np.float64),
                                     None if x_is_zero else x0.astype(np.float64), FIXED_LAM_MAX,
                                     FIXED_LAM_MIN, 3, "sgs")
            _close(outs[0], outs[1], 1e-5, (lev, x_is_zero))
            _close(outs[0], ref, 1e-4, (lev, x_is_zero))
            assert np.array_equal(outs[0], outs[2]), (lev, x_is_zero, _maxrel(outs[0], outs[2]))
    v = random_field(320, shape)
    zs = []
    for ctx in ctxs:
        z = torch.empty(shape, dtype=torch.float64, device=DEV)
        gmg.gmg_apply_preconditioner(ctx, _t(v), z)
        zs.append(_np(z))
    _close(zs[0], zs[1], 1e-5)
    assert np.array_equal(zs[0], zs[2])
    f = make_inputs("twochannel512", shape=shape)["f"]
    its = []
    for ctx in ctxs:
        phi = torch.zeros(shape, dtype=torch.float64, device=DEV)
        info = gmg.fgmres_solve(ctx, _t(f), phi)
        assert info.converged and _true_residual(shape, ctx.params, a, f, _np(phi)) < 1e-8
        its.append(info.iterations)
    assert abs(its[0] - its[1]) <= 1 and its[0] == its[2]


def test_eigen_bounds_match_oracle():
    shape = RAGGED
    a = random_coefficient(140, shape, contrast=1e3)
    p = _params(shape, coarse_min=2, precision=gmg.GMG_PREC_FP64, orthogonalization=gmg.GMG_ORTH_MGS)
    ctx = gmg.gmg_setup(p, _t(a))
    hier = O.build_hierarchy(_ogrid(shape), a, _oracle_hierarchy(a, p))
    for lev in range(1, gmg.gmg_num_levels(ctx)):
        info = gmg.gmg_level_info(ctx, lev)
        assert info["lam_max"] == pytest.approx(hier.levels[lev].lam_max, rel=1e-11)
        assert info["lam_min"] == pytest.approx(hier.levels[lev].lam_min, rel=1e-11)


# (8, 24, 144): 72 and 36 cell pairs per row on the two finest levels, so a row
# spans 3 and 2 warps and the x-neighbours cross warp and block boundaries.
@pytest.mark.parametrize("shape", [RAGGED, (8, 24, 144)])
@pytest.mark.parametrize("prec", [gmg.GMG_PREC_FP64, gmg.GMG_PREC_MIXED])
@pytest.mark.parametrize("mode,coarsening", [(gmg.GMG_PROLONG_OPDEP, gmg.GMG_COARSEN_SERIES),
                                             (gmg.GMG_PROLONG_OPDEP, gmg.GMG_COARSEN_MEAN),
                                             (gmg.GMG_PROLONG_TRILINEAR, gmg.GMG_COARSEN_SERIES),
                                             (gmg.GMG_PROLONG_TRILINEAR, gmg.GMG_COARSEN_MEAN),
                                             (gmg.GMG_PROLONG_CONSTANT, gmg.GMG_COARSEN_MEAN)])
def test_transfers_and_coarse_solve(prec, mode, coarsening, shape):
    a = random_coefficient(150, shape, contrast=1e2)
    p = _params(shape, coarse_min=2, precision=prec, prolongation=mode, coarsening=coarsening)
    ctx = gmg.gmg_setup(p, _t(a))
    dt = ctx.level_dtype
    fp32 = dt == torch.float32
    q = _q32 if fp32 else (lambda v: v)
    tol = 2e-6 if fp32 else 1e-14
    ops = _olevels(a, p)
    kind = ["trilinear", "constant", "opdep"][mode]
    L = gmg.gmg_num_levels(ctx)
    for lev in range(L - 1, 0, -1):
        s = gmg.gmg_level_info(ctx, lev)["shape"]
        sc = gmg.gmg_level_info(ctx, lev - 1)["shape"]
        b, x = q(random_field(151 + lev, s)), q(random_field(161 + lev, s))
        coarse = torch.empty(sc, dtype=dt, device=DEV)
        gmg.gmg_level_residual_restrict(ctx, lev, _t(b, dt), _t(x, dt), coarse)
        ref = O.restrict(b - O.apply_operator(_ogrid(s), q(ops[lev]), x))
        _close(_np(coarse), ref, (5e-5 if fp32 else 1e-13), ("restrict", lev))
        e = q(random_field(171 + lev, sc))
        xt = _t(x, dt)
        gmg.gmg_level_prolong_add(ctx, lev, _t(e, dt), xt)
        ref = x + O.prolong(e, kind, q(ops[lev]))
        _close(_np(xt), ref, tol, ("prolong", lev))
    # coarsest direct solve
    sc = gmg.gmg_level_info(ctx, 0)["shape"]
    b = q(random_field(180, sc))
    x = torch.empty(sc, dtype=dt, device=DEV)
    gmg.gmg_coarse_solve(ctx, _t(b, dt), x)
    A = O.dense_operator(_ogrid(sc), ops[0])
    ref = np.linalg.solve(A, b.ravel()).reshape(sc)
    _close(_np(x), ref, (1e-5 if fp32 else 1e-12))


def _offset_view(arr, dtype):
    """A contiguous device copy of arr whose storage starts 4 bytes past an
    8-byte boundary (as a sub-view of a larger allocation can)."""
    n = arr.size
    buf = torch.empty(n + 1, dtype=dtype, device=DEV)
    v = buf[1:].view(arr.shape)
    v.copy_(torch.from_numpy(np.ascontiguousarray(arr)).to(DEV))
    assert v.data_ptr() % 8 == 4
    return v


def test_solve_with_unaligned_right_hand_side():
    """An f that starts 8 bytes off a 16-byte boundary takes the scalar
    right-hand-side kernel; the solve agrees with the aligned one (the plate
    terms are associated differently, so to rounding)."""
    inp = make_inputs("channel128", n=32)
    shape = inp["a"].shape
    p = _params(shape, precision=gmg.GMG_PREC_MIXED)
    ctx = gmg.gmg_setup(p, _t(inp["a"]))
    n = int(np.prod(shape))
    f_al = _t(inp["f"])
    buf = torch.empty(n + 1, dtype=torch.float64, device=DEV)
    f_off = buf[1:].view(shape)
    f_off.copy_(f_al)
    assert f_off.data_ptr() % 16 == 8
    b1, b2 = torch.empty_like(f_al), torch.empty_like(f_al)
    gmg.assemble_rhs(ctx, f_al, b1)
    gmg.assemble_rhs(ctx, f_off, b2)
    _close(_np(b2), _np(b1), 1e-15)
    x1, x2 = torch.zeros_like(f_al), torch.zeros_like(f_al)
    i1, i2 = gmg.fgmres_solve(ctx, f_al, x1), gmg.fgmres_solve(ctx, f_off, x2)
    assert i1.converged and i2.converged and i1.iterations == i2.iterations
    _close(_np(x2), _np(x1), 1e-12)


def test_level_ops_accept_arrays_off_the_pair_alignment():
    """The FP32 level kernels that move cell pairs as float2 need 8-byte
    aligned arrays; arrays that are not take the one-cell kernels and give the
    same results to FP32 rounding."""
    shape = (8, 24, 144)
    a = random_coefficient(320, shape, 1e3)
    ctx = gmg.gmg_setup(_params(shape, coarse_min=2, precision=gmg.GMG_PREC_MIXED), _t(a))
    lev = gmg.gmg_num_levels(ctx) - 1
    s = gmg.gmg_level_info(ctx, lev)["shape"]
    sc = gmg.gmg_level_info(ctx, lev - 1)["shape"]
    b = random_field(321, s).astype(np.float32)
    x0 = random_field(322, s).astype(np.float32)
    e = random_field(323, sc).astype(np.float32)
    # restriction
    c1 = torch.empty(sc, dtype=torch.float32, device=DEV)
    c2 = torch.empty(sc, dtype=torch.float32, device=DEV)
    gmg.gmg_level_residual_restrict(ctx, lev, _t(b, torch.float32), _t(x0, torch.float32), c1)
    gmg.gmg_level_residual_restrict(ctx, lev, _offset_view(b, torch.float32), _offset_view(x0, torch.float32), c2)
    _close(_np(c2), _np(c1), 1e-5)
    # prolongation
    x1 = _t(x0, torch.float32)
    x2 = _offset_view(x0, torch.float32)
    gmg.gmg_level_prolong_add(ctx, lev, _t(e, torch.float32), x1)
    gmg.gmg_level_prolong_add(ctx, lev, _t(e, torch.float32), x2)
    _close(_np(x2), _np(x1), 1e-6)
    # smoothing (fused kernel for aligned arrays, separate kernels otherwise)
    for x_is_zero in (True, False):
        x1 = _t(x0, torch.float32)
        x2 = _offset_view(x0, torch.float32)
        gmg.gmg_level_smooth(ctx, lev, _t(b, torch.float32), x1, x_is_zero)
        gmg.gmg_level_smooth(ctx, lev, _offset_view(b, torch.float32), x2, x_is_zero)
        _close(_np(x2), _np(x1), 1e-5, x_is_zero)


@pytest.mark.parametrize("shape,cm", [(RAGGED, 2), ((32, 32, 32), 4), ((20, 16, 16), 4)])
def test_vcycle_fp64_matches_oracle(shape, cm):
    a = make_inputs("channel128", shape=shape)["a"]
    p = _params(shape, coarse_min=cm, precision=gmg.GMG_PREC_FP64, orthogonalization=gmg.GMG_ORTH_MGS)
    ctx = gmg.gmg_setup(p, _t(a))
    hier = O.build_hierarchy(_ogrid(shape), a, _oracle_hierarchy(a, p))
    v = random_field(190, shape)
    z = torch.empty(shape, dtype=torch.float64, device=DEV)
    gmg.gmg_apply_preconditioner(ctx, _t(v), z)
    _close(_np(z), O.vcycle(hier, v), 1e-12)


def test_vcycle_mixed_close_to_oracle():
    shape = (32, 32, 32)
    a = make_inputs("channel128", n=32)["a"]
    p = _params(shape, precision=gmg.GMG_PREC_MIXED)
    ctx = gmg.gmg_setup(p, _t(a))
    hier = O.build_hierarchy(_ogrid(shape), a, _oracle_hierarchy(a, p))
    v = random_field(191, shape)
    z = torch.empty(shape, dtype=torch.float64, device=DEV)
    gmg.gmg_apply_preconditioner(ctx, _t(v), z)
    _close(_np(z), O.vcycle(hier, v), 1e-4)


# ---------------------------------------------------------------------------
# Whole solves
# ---------------------------------------------------------------------------


def _true_residual(shape, p, a, f, phi, homogeneous=False):
    g = _ogrid(shape, p)
    b = f if homogeneous else O.assemble_rhs(g, a, f, p.phi_bottom, p.phi_top)
    return np.linalg.norm(b - O.apply_operator(g, a, phi)) / np.linalg.norm(b)


@pytest.mark.parametrize("workload,n,orth", [("const32", 32, gmg.GMG_ORTH_MGS), ("channel128", 32, gmg.GMG_ORTH_CGS2),
                                             ("channel128", 64, gmg.GMG_ORTH_MGS),
                                             ("twochannel512", 32, gmg.GMG_ORTH_CGS2)])
def test_fp64_solve_matches_oracle(workload, n, orth):
    inp = make_inputs(workload, n=n)
    shape = inp["a"].shape
    p = _params(shape, precision=gmg.GMG_PREC_FP64, orthogonalization=orth)
    ref, rinfo, _ = O.solve(_oracle_hierarchy(inp["a"], p), inp["a"], inp["f"])
    ctx = gmg.gmg_setup(p, _t(inp["a"]))
    phi = torch.zeros(shape, dtype=torch.float64, device=DEV)
    info = gmg.fgmres_solve(ctx, _t(inp["f"]), phi)
    out = _np(phi)
    assert info.converged and info.iterations == rinfo.iterations
    assert _true_residual(shape, p, inp["a"], inp["f"], out) < 1e-8
    assert info.true_rel_residual == pytest.approx(rinfo.true_rel_residual, rel=1e-4)
    np.testing.assert_allclose(info.history, rinfo.history, rtol=1e-5)
    _close(out, ref, 1e-10)


@pytest.mark.parametrize("workload,n,kappa,arith", [("const32", 32, None, 1), ("channel128", 64, None, 1),
                                                    ("channel256", 64, 1e1, 1), ("channel256", 64, 1e3, 1),
                                                    ("channel256", 64, 1e4, 1), ("twochannel512", 64, None, 1),
                                                    ("twochannel512", 64, None, 0)])
def test_mixed_solve_residual_and_error(workload, n, kappa, arith):
    inp = make_inputs(workload, n=n, kappa=kappa)
    shape = inp["a"].shape
    p = _params(shape, precision=gmg.GMG_PREC_MIXED, outer_arith=arith)
    ref, rinfo, _ = O.solve(_oracle_hierarchy(inp["a"], p), inp["a"], inp["f"])
    ctx = gmg.gmg_setup(p, _t(inp["a"]))
    phi = torch.zeros(shape, dtype=torch.float64, device=DEV)
    info = gmg.fgmres_solve(ctx, _t(inp["f"]), phi)
    out = _np(phi)
    tr = _true_residual(shape, p, inp["a"], inp["f"], out)
    print(f"{workload} n={n} mixed iters {info.iterations} (oracle {rinfo.iterations}) true {tr:.2e} "
          f"phi rel err {_rel(out, ref):.2e}")
    assert info.converged and tr < 1e-8
    assert abs(info.iterations - rinfo.iterations) <= 2
    _close(out, ref, 1e-6)


def test_warm_start_and_restart():
    inp = make_inputs("channel128", n=32)
    shape = inp["a"].shape
    p = _params(shape, precision=gmg.GMG_PREC_MIXED, restart=3)
    ctx = gmg.gmg_setup(p, _t(inp["a"]))
    phi = torch.zeros(shape, dtype=torch.float64, device=DEV)
    info = gmg.fgmres_solve(ctx, _t(inp["f"]), phi)
    assert info.converged and info.restarts >= 2
    # warm start from the converged phi: converges at once (0 iterations)
    info2 = gmg.fgmres_solve(ctx, _t(inp["f"]), phi)
    assert info2.converged and info2.iterations == 0


def test_edge_cases():
    shape = (8, 8, 8)
    a = random_coefficient(200, shape, contrast=10.0)
    # zero right-hand side and zero plate data -> phi = 0
    p = _params(shape, phi_top=0.0)
    ctx = gmg.gmg_setup(p, _t(a))
    phi = torch.ones(shape, dtype=torch.float64, device=DEV)
    info = gmg.fgmres_solve(ctx, torch.zeros(shape, dtype=torch.float64, device=DEV), phi)
    assert info.converged and float(phi.abs().max()) == 0.0
    # iteration cap
    p = _params(shape, max_iters=1)
    ctx = gmg.gmg_setup(p, _t(a))
    phi = torch.zeros(shape, dtype=torch.float64, device=DEV)
    info = gmg.fgmres_solve(ctx, _t(random_field(201, shape)), phi)
    assert not info.converged and info.iterations == 1
    # non-finite input
    f = random_field(202, shape)
    f[3, 3, 3] = np.nan
    with pytest.raises(gmg.GMGError) as e:
        gmg.fgmres_solve(ctx, _t(f), torch.zeros(shape, dtype=torch.float64, device=DEV))
    assert e.value.status == gmg.GMG_ERR_NONFINITE
    # bad coefficient
    bad = a.copy()
    bad[0, 0, 0] = -1.0
    with pytest.raises(gmg.GMGError) as e:
        gmg.gmg_setup(_params(shape), _t(bad))
    assert e.value.status == gmg.GMG_ERR_ARG
    # shape that does not halve to coarse_min
    with pytest.raises(gmg.GMGError):
        gmg.gmg_setup(gmg.gmg_default_params(12, 12, 10), _t(np.ones((10, 12, 12))))
    # only the coarsest grid: the direct solve answers in one iteration
    p = _params((4, 4, 4), precision=gmg.GMG_PREC_FP64)
    a4 = random_coefficient(203, (4, 4, 4), 10.0)
    ctx = gmg.gmg_setup(p, _t(a4))
    phi = torch.zeros((4, 4, 4), dtype=torch.float64, device=DEV)
    info = gmg.fgmres_solve(ctx, _t(random_field(204, (4, 4, 4))), phi)
    assert info.converged and info.iterations == 1


def test_allocation_failure_is_reported_and_recoverable():
    shape = (16, 16, 16)
    a = _t(random_coefficient(210, shape, 10.0))
    for k in (1, 3, 7):
        gmg.gmg_test_fail_allocation_after(k)
        with pytest.raises(gmg.GMGError) as e:
            gmg.gmg_setup(_params(shape), a)
        assert e.value.status == gmg.GMG_ERR_ALLOC
    gmg.gmg_test_fail_allocation_after(0)
    ctx = gmg.gmg_setup(_params(shape), a)
    phi = torch.zeros(shape, dtype=torch.float64, device=DEV)
    assert gmg.fgmres_solve(ctx, _t(random_field(211, shape)), phi).converged


def test_host_buffer_solve_matches_device_solve():
    inp = make_inputs("channel128", n=32)
    shape = inp["a"].shape
    p = _params(shape)
    ctx = gmg.gmg_setup(p, _t(inp["a"]))
    phi_d = torch.zeros(shape, dtype=torch.float64, device=DEV)
    gmg.fgmres_solve(ctx, _t(inp["f"]), phi_d)
    ctx2 = gmg.gmg_setup(p, _t(np.ones(shape)))
    a_h = torch.from_numpy(inp["a"]).pin_memory()
    f_h = torch.from_numpy(inp["f"]).pin_memory()
    phi_h = torch.zeros(shape, dtype=torch.float64).pin_memory()
    e = [torch.empty(shape, dtype=torch.float32).pin_memory() for _ in range(3)]
    info = gmg.gmg_solve_host(ctx2, a_h, f_h, phi_h, None, *e)
    assert info.converged
    np.testing.assert_array_equal(phi_h.numpy(), _np(phi_d))
    ex, ey, ez = O.field_from_potential(_ogrid(shape), phi_h.numpy(), 0.0, 1.0)
    for got, ref in zip(e, (ex, ey, ez)):
        _close(got.numpy().astype(np.float64), ref, 1e-6)


def test_pipelined_host_solves_match_synchronous_ones():
    """Three back-to-back gmg_solve_host_async calls on different inputs and
    into different host arrays, then gmg_host_wait: each result equals the
    synchronous gmg_solve_host's bit for bit (the copy-out of one call overlaps
    the next call's uploads and set-up without a race on the staging arrays)."""
    shape = (16, 24, 32)
    p = _params(shape)
    cases = []
    for seed in (520, 521, 522):
        a = 1.0 + 0.5 * (random_field(seed, shape) + 1.0)
        f = random_field(seed + 10, shape)
        cases.append((torch.from_numpy(a).pin_memory(), torch.from_numpy(f).pin_memory()))
    ctx_s = gmg.gmg_setup(p, _t(np.ones(shape)))
    want = []
    for a_h, f_h in cases:
        phi = torch.zeros(shape, dtype=torch.float64).pin_memory()
        e = [torch.empty(shape, dtype=torch.float32).pin_memory() for _ in range(3)]
        gmg.gmg_solve_host(ctx_s, a_h, f_h, phi, None, *e)
        want.append((phi, e))
    ctx_a = gmg.gmg_setup(p, _t(np.ones(shape)))
    got = []
    for a_h, f_h in cases:
        phi = torch.full(shape, np.nan, dtype=torch.float64).pin_memory()
        e = [torch.full(shape, np.nan, dtype=torch.float32).pin_memory() for _ in range(3)]
        info = gmg.gmg_solve_host_async(ctx_a, a_h, f_h, phi, None, *e)
        assert info.converged
        got.append((phi, e))
    gmg.gmg_host_wait(ctx_a)
    for (pw, ew), (pg, eg) in zip(want, got):
        assert torch.equal(pw, pg)
        for a_, b_ in zip(ew, eg):
            assert torch.equal(a_, b_)
    gmg.gmg_host_wait(ctx_s)
    ctx_a.close()
    ctx_s.close()


def test_pipelined_host_copy_out_completes_on_the_next_call_or_the_wait():
    """The pipelined call holds its copy-out back for the next call (after that
    call's upload of a) or for gmg_host_wait.  An async call followed by a
    synchronous one: both results are complete when the synchronous call
    returns.  An async call that reuses the coefficient (a_host NULL), then
    gmg_host_wait: complete too.  All equal the synchronous results bit for bit."""
    shape = (16, 24, 32)
    p = _params(shape)
    cases = []
    for seed in (530, 531):
        a = 1.0 + 0.5 * (random_field(seed, shape) + 1.0)
        f = random_field(seed + 10, shape)
        cases.append((torch.from_numpy(a).pin_memory(), torch.from_numpy(f).pin_memory()))

    def bufs(fill):
        phi = torch.full(shape, fill, dtype=torch.float64).pin_memory()
        return phi, [torch.full(shape, fill, dtype=torch.float32).pin_memory() for _ in range(3)]

    ctx_s = gmg.gmg_setup(p, _t(np.ones(shape)))
    want = []
    for a_h, f_h in cases:
        phi, e = bufs(0.0)
        gmg.gmg_solve_host(ctx_s, a_h, f_h, phi, None, *e)
        want.append((phi, e))
    f_only = torch.from_numpy(random_field(545, shape)).pin_memory()
    phi3, e3 = bufs(0.0)
    gmg.gmg_solve_host(ctx_s, None, f_only, phi3, None, *e3)

    ctx_a = gmg.gmg_setup(p, _t(np.ones(shape)))
    got0, got1, got3 = bufs(np.nan), bufs(np.nan), bufs(np.nan)
    assert gmg.gmg_solve_host_async(ctx_a, cases[0][0], cases[0][1], got0[0], None, *got0[1]).converged
    assert gmg.gmg_solve_host(ctx_a, cases[1][0], cases[1][1], got1[0], None, *got1[1]).converged
    for (pw, ew), (pg, eg) in zip(want, (got0, got1)):
        assert torch.equal(pw, pg)
        for a_, b_ in zip(ew, eg):
            assert torch.equal(a_, b_)
    assert gmg.gmg_solve_host_async(ctx_a, None, f_only, got3[0], None, *got3[1]).converged
    gmg.gmg_host_wait(ctx_a)
    assert torch.equal(phi3, got3[0])
    for a_, b_ in zip(e3, got3[1]):
        assert torch.equal(a_, b_)
    ctx_a.close()
    ctx_s.close()


def test_full_size_solve_step_sampled_parity():
    """The benchmarked solve step at full size (512^3 two-channel workload, mixed
    precision, the bench's parameters): converged, with the true FP64 residual
    below 1e-8 both as reported and as recomputed with the FP64 operator-apply
    kernel; that operator and the FP32 field agree with the oracle at sampled
    cells (plates, walls and corners included), computed one by one."""
    n = 512
    inp = make_inputs("twochannel512", n=n)
    shape = inp["a"].shape
    p = gmg.gmg_default_params(n, n, n, precision=gmg.GMG_PREC_MIXED)
    a, f = _t(inp["a"]), _t(inp["f"])
    ctx = gmg.gmg_setup(p, a)
    phi = torch.zeros(shape, dtype=torch.float64, device=DEV)
    info = gmg.fgmres_solve(ctx, f, phi)
    assert info.converged and info.true_rel_residual < 1e-8
    b, y = torch.empty_like(phi), torch.empty_like(phi)
    gmg.assemble_rhs(ctx, f, b)
    gmg.apply_operator(ctx, phi, y)
    rel = (torch.linalg.vector_norm(b - y) / torch.linalg.vector_norm(b)).item()
    assert rel < 1e-8 and rel == pytest.approx(info.true_rel_residual, rel=1e-3)
    e = [torch.empty(shape, dtype=torch.float32, device=DEV) for _ in range(3)]
    gmg.field_from_potential(ctx, phi, *e)
    rng = np.random.default_rng(512)
    cells = [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(2048)]
    cells += [(k, j, i) for k in (0, n - 1) for j in (0, 7, n - 1) for i in (0, 5, n - 1)]
    idx = torch.tensor([(k * n + j) * n + i for k, j, i in cells], device=DEV)
    phi_h = _np(phi)
    grid = _ogrid(shape, p)
    ref_y = O.apply_operator_at(grid, inp["a"], phi_h, cells)
    got_y = _np(y.reshape(-1)[idx])
    assert np.abs(got_y - ref_y).max() <= 1e-12 * np.abs(ref_y).max()
    ref_e = O.field_at(grid, phi_h, p.phi_bottom, p.phi_top, cells)
    for d in range(3):
        got = _np(e[d].reshape(-1)[idx])
        np.testing.assert_allclose(got, ref_e[:, d], rtol=1e-6, atol=1e-6 * np.abs(ref_e[:, d]).max())
    ctx.close()


# ---------------------------------------------------------------------------
# Field and adjoint
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_field_matches_oracle(dtype):
    shape = RAGGED
    p = _params(shape, coarse_min=2, phi_bottom=0.2, phi_top=3.0, lx=2.0, lz=0.5)
    ctx = gmg.gmg_setup(p, _t(np.ones(shape)))
    phi = random_field(220, shape)
    e = [torch.empty(shape, dtype=dtype, device=DEV) for _ in range(3)]
    gmg.field_from_potential(ctx, _t(phi), *e)
    ref = O.field_from_potential(_ogrid(shape, p), phi, 0.2, 3.0)
    for got, r in zip(e, ref):
        np.testing.assert_allclose(_np(got), r, rtol=1e-13 if dtype == torch.float64 else 1e-6,
                                   atol=1e-12 if dtype == torch.float64 else 1e-5 * np.abs(r).max())


def test_adjoint_grad_kernel_matches_oracle():
    shape = RAGGED
    p = _params(shape, coarse_min=2, phi_bottom=0.4, phi_top=1.3, ly=0.8)
    ctx = gmg.gmg_setup(p, _t(np.ones(shape)))
    phi, lam = random_field(230, shape), random_field(231, shape)
    out = torch.empty(shape, dtype=torch.float64, device=DEV)
    gmg.adjoint_coefficient_grad(ctx, _t(phi), _t(lam), out)
    ref = O.adjoint_coefficient_grad(_ogrid(shape, p), phi, lam, 0.4, 1.3)
    _close(_np(out), ref, 1e-14)


def test_autograd_finite_differences_and_cpu_adjoint():
    """Central differences on 64 seeded entries of a 32^3 instance.

    L is linear in f, so a large step (1 or |f_q|) is exact up to the solve
    error (measured 6e-9 at worst; held to 1e-6).  For a, two steps: the
    configured 1e-6 relative step and a 1e-3 step, whose truncation error is
    ~1e-6 (measured 4.5e-7 at worst; held to 1e-5).  At 1e-6 the truncation
    error is near 1e-12 and the solve error of L divided by the step
    dominates: with the forward solves at rtol = 1e-13 the worst of the 64
    entries is 1.1e-3 off.  That error is known to first order: a solve that
    returns x~ with residual r~ = b - A x~ has w . x~ = w . x - lambda . r~
    (A^T lambda = w), so adding lambda . r~ of each solve (r~ from the
    oracle's operator in FP64, lambda from the oracle's adjoint solve) removes
    it.  What stays is the FP64 rounding of L and of r~ divided by the step
    (about eps |lambda| |A| |x~| / 2h): measured 3.7e-6 median and 7.9e-5 at
    worst, held to 3e-4."""
    from paper_1812_08606_gb300 import PoissonSolver
    inp = make_inputs("adjoint", n=32)
    shape = inp["a"].shape
    solver = PoissonSolver(shape, rtol=1e-13, precision=gmg.GMG_PREC_MIXED, max_iters=60)
    a = _t(inp["a"]).requires_grad_(True)
    f = _t(inp["f"]).requires_grad_(True)
    w = _t(inp["w"])
    loss = (w * solver.solve(a, f)).sum()
    loss.backward()
    ga, gf = _np(a.grad), _np(f.grad)
    prm = solver.params
    grid = _ogrid(shape, prm)
    gb, gt = prm.phi_bottom, prm.phi_top
    op = O.OracleParams(lx=prm.lx, ly=prm.ly, lz=prm.lz, phi_bottom=gb, phi_top=gt, rtol=1e-13, max_iters=60)
    lam_o, _, _ = O.solve(op, inp["a"], inp["w"], homogeneous=True)
    rng = np.random.default_rng(20181225)
    idx = rng.choice(a.numel(), size=64, replace=False)

    def L(av, fv):
        """w . x~ and the first-order error of the solve, lambda . r~."""
        with torch.no_grad():
            phi = solver.solve(av, fv)
            val = float((w * phi).sum())
        an, fn, ph = _np(av), _np(fv), _np(phi)
        r = O.assemble_rhs(grid, an, fn, gb, gt) - O.apply_operator(grid, an, ph)
        return val, float(np.sum(lam_o * r))

    base_a, base_f = a.detach().clone(), f.detach().clone()
    errs = {("a", 1e-6): [], ("a", 1e-3): [], ("f", None): [], ("a corrected", 1e-6): []}
    tols = {("a", 1e-3): 1e-5, ("f", None): 1e-6, ("a corrected", 1e-6): 3e-4}
    for q in idx:
        for which, step in (("a", 1e-6), ("a", 1e-3), ("f", None)):
            grad, base = (ga, base_a) if which == "a" else (gf, base_f)
            v = abs(float(base.view(-1)[q]))
            h = step * v if which == "a" else max(v, 1.0)
            plus, minus = base.clone(), base.clone()
            plus.view(-1)[q] += h
            minus.view(-1)[q] -= h
            if which == "a":
                (lp, ep), (lm, em) = L(plus, base_f), L(minus, base_f)
            else:
                (lp, ep), (lm, em) = L(base_a, plus), L(base_a, minus)
            fd = (lp - lm) / (2 * h)
            g = grad.ravel()[q]
            scale = lambda x: max(abs(x), 1e-4 * np.abs(grad).max())
            errs[(which, step)].append(abs(g - fd) / scale(fd))
            if which == "a" and step == 1e-6:
                fdc = ((lp + ep) - (lm + em)) / (2 * h)
                errs[("a corrected", step)].append(abs(g - fdc) / scale(fdc))
    for key, e in errs.items():
        print(f"FD {key}: median {np.median(e):.2e}, max {np.max(e):.2e}")
    for key, tol in tols.items():
        worst = int(np.argmax(errs[key]))
        assert errs[key][worst] < tol, (key, int(idx[worst]), errs[key][worst])
    # the uncorrected 1e-6 differences are off by no more than the solve error explains
    assert max(errs[("a", 1e-6)]) < 1e-2
    # dot test: w . A^{-1} f = f . A^{-1} w on the homogeneous problem
    ctx = solver.ctx
    solver.set_coefficient(base_a)
    x1 = torch.zeros(shape, dtype=torch.float64, device=DEV)
    x2 = torch.zeros_like(x1)
    gmg.fgmres_solve(ctx, base_f, x1, homogeneous_bc=True)
    gmg.fgmres_solve(ctx, w, x2, homogeneous_bc=True)
    assert float((w * x1).sum()) == pytest.approx(float((base_f * x2).sum()), rel=1e-10)


def test_autograd_raises_when_a_solve_does_not_converge():
    """A forward or adjoint solve stopped by max_iters must not hand back phi
    or a gradient as if it were converged."""
    from paper_1812_08606_gb300 import PoissonSolver
    inp = make_inputs("adjoint", n=16)
    shape = inp["a"].shape
    solver = PoissonSolver(shape, rtol=1e-12, max_iters=1, coarse_min=2)
    a = _t(inp["a"]).requires_grad_(True)
    f = _t(inp["f"]).requires_grad_(True)
    with pytest.raises(gmg.GMGError) as e:
        solver.solve(a, f)
    assert e.value.status == gmg.GMG_ERR_NOT_CONVERGED
    # the adjoint solve alone: a forward solve that converges, an adjoint capped at one step
    solver2 = PoissonSolver(shape, rtol=1e-12, max_iters=40, coarse_min=2)
    phi = solver2.solve(a, f)
    assert solver2.last_info.converged
    solver2.params.max_iters = 1
    solver2.close()
    solver2.ctx = None
    solver2.set_coefficient(a)   # a new context with the one-step cap
    with pytest.raises(gmg.GMGError):
        torch.autograd.grad((_t(inp["w"]) * phi).sum(), (a, f))
    # non-strict: the unconverged result comes back with its info
    loose = PoissonSolver(shape, rtol=1e-12, max_iters=1, coarse_min=2, strict=False)
    loose.solve(a.detach(), f.detach())
    assert not loose.last_info.converged


def test_autograd_follows_the_current_torch_stream():
    """With stream=None the library runs on whatever stream is current at the
    call, so the solve sees f written on a side stream just before it."""
    from paper_1812_08606_gb300 import PoissonSolver
    inp = make_inputs("adjoint", n=16)
    shape = inp["a"].shape
    solver = PoissonSolver(shape, rtol=1e-10, coarse_min=2)
    a = _t(inp["a"])
    ref = solver.solve(a, _t(inp["f"])).clone()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        f = torch.empty(shape, dtype=torch.float64, device=DEV)
        torch.cuda._sleep(2_000_000)    # keep the side stream busy before f is written
        f.copy_(_t(inp["f"]))
        phi = solver.solve(a, f)
    side.synchronize()
    _close(_np(phi), _np(ref), 1e-12)


def test_autograd_matches_cpu_adjoint_64():
    from paper_1812_08606_gb300 import PoissonSolver
    inp = make_inputs("adjoint", n=64)
    shape = inp["a"].shape
    solver = PoissonSolver(shape, rtol=1e-12)
    a = _t(inp["a"]).requires_grad_(True)
    f = _t(inp["f"]).requires_grad_(True)
    (_t(inp["w"]) * solver.solve(a, f)).sum().backward()
    op = O.OracleParams(rtol=1e-12)
    phi, _, hier = O.solve(op, inp["a"], inp["f"])
    lam, _, _ = O.solve(op, inp["a"], inp["w"], homogeneous=True, hierarchy=hier)
    ga = O.adjoint_coefficient_grad(_ogrid(shape), phi, lam, 0.0, 1.0)
    ef = _close(_np(f.grad), lam, 1e-7, "dL/df")
    ea = _close(_np(a.grad), ga, 1e-6, "dL/da")
    print(f"adjoint vs CPU at 64^3 (l2, max): dL/df {ef}, dL/da {ea}")


# ---------------------------------------------------------------------------
# Full multigrid (first time step) and the assembly from the densities
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("shape,cm", [(RAGGED, 2), ((32, 32, 32), 4), ((8, 24, 144), 2)])
def test_fmg_preconditioner_fp64_matches_oracle(shape, cm):
    a = make_inputs("channel128", shape=shape)["a"] if shape[0] >= 16 else random_coefficient(330, shape, 1e3)
    p = _params(shape, coarse_min=cm, precision=gmg.GMG_PREC_FP64, cycle=gmg.GMG_CYCLE_FMG)
    ctx = gmg.gmg_setup(p, _t(a))
    hier = O.build_hierarchy(_ogrid(shape), a, _oracle_hierarchy(a, p))
    v = random_field(331, shape)
    z = torch.empty(shape, dtype=torch.float64, device=DEV)
    gmg.gmg_apply_preconditioner(ctx, _t(v), z)
    _close(_np(z), O.fmg(hier, v), 1e-12)


def test_fmg_preconditioner_mixed_close_to_oracle():
    shape = (32, 32, 32)
    a = make_inputs("twochannel512", shape=shape)["a"]
    p = _params(shape, precision=gmg.GMG_PREC_MIXED, cycle=gmg.GMG_CYCLE_FMG)
    ctx = gmg.gmg_setup(p, _t(a))
    hier = O.build_hierarchy(_ogrid(shape), a, _oracle_hierarchy(a, p))
    v = random_field(332, shape)
    z = torch.empty(shape, dtype=torch.float64, device=DEV)
    gmg.gmg_apply_preconditioner(ctx, _t(v), z)
    _close(_np(z), O.fmg(hier, v), 1e-4)


@pytest.mark.parametrize("workload,n", [("channel128", 32), ("twochannel512", 32)])
def test_fmg_solve_fp64_matches_oracle(workload, n):
    inp = make_inputs(workload, n=n)
    shape = inp["a"].shape
    p = _params(shape, precision=gmg.GMG_PREC_FP64, orthogonalization=gmg.GMG_ORTH_MGS, cycle=gmg.GMG_CYCLE_FMG)
    ref, rinfo, _ = O.solve(_oracle_hierarchy(inp["a"], p), inp["a"], inp["f"])
    ctx = gmg.gmg_setup(p, _t(inp["a"]))
    phi = torch.zeros(shape, dtype=torch.float64, device=DEV)
    info = gmg.fgmres_solve(ctx, _t(inp["f"]), phi)
    assert info.fmg == 1
    assert info.iterations == rinfo.iterations
    _close(_np(phi), ref, 1e-10)
    assert info.true_rel_residual < 1e-8


def test_auto_cycle_takes_fmg_only_from_a_zero_guess():
    """Sec. 3.2: full multigrid for the first step (no previous potential),
    V-cycles once a previous potential is the initial guess."""
    inp = make_inputs("twochannel512", n=64)
    shape = inp["a"].shape
    res = {}
    for cyc in (gmg.GMG_CYCLE_V, gmg.GMG_CYCLE_AUTO):
        p = _params(shape, precision=gmg.GMG_PREC_MIXED, cycle=cyc)
        ctx = gmg.gmg_setup(p, _t(inp["a"]))
        phi = torch.zeros(shape, dtype=torch.float64, device=DEV)
        first = gmg.fgmres_solve(ctx, _t(inp["f"]), phi)
        assert first.true_rel_residual < 1e-8
        # the next "time step": slightly changed coefficient, warm start from phi
        gmg.gmg_update_coefficient(ctx, _t(inp["a"] * 1.001))
        second = gmg.fgmres_solve(ctx, _t(inp["f"]), phi)
        assert second.true_rel_residual < 1e-8
        res[cyc] = (first, second)
    v1, v2 = res[gmg.GMG_CYCLE_V]
    a1, a2 = res[gmg.GMG_CYCLE_AUTO]
    assert (v1.fmg, v2.fmg, a1.fmg, a2.fmg) == (0, 0, 1, 0)
    assert a1.iterations <= v1.iterations
    assert a2.iterations == v2.iterations
    assert v2.iterations < v1.iterations          # the warm start pays


def _densities(shape, seed):
    """Smooth positive densities of streamer magnitude (cm^-3): a channel
    profile plus seeded smooth noise, electrons and ions different."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) / nz, (np.arange(ny) + 0.5) / ny, (np.arange(nx) + 0.5) / nx,
                          indexing="ij")
    prof = np.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2) / 0.05 ** 2 - (z - 0.5) ** 2 / 0.1 ** 2)
    ne = 1e8 + 1e14 * prof * (1.0 + 0.1 * random_field(seed, shape))
    npos = 1e8 + 1e14 * prof * (1.0 + 0.1 * random_field(seed + 1, shape))
    return ne, npos


@pytest.mark.parametrize("shape,lengths", [(RAGGED, (1.0, 1.0, 1.0)), ((8, 24, 144), (2.0, 1.0, 0.5))])
def test_assembly_matches_oracle(shape, lengths):
    ne, npos = _densities(shape, 340)
    p = _params(shape, lx=lengths[0], ly=lengths[1], lz=lengths[2])
    nz, ny, nx = shape
    grid = O.Grid(nx, ny, nz, *lengths)
    kw = dict(tau=2e-12, mu_e=-2.9e5 / 760, mu_p=2.6e3 / 760, diffusion=(2190.0, 2190.0, 1800.0))
    a_ref, f_ref = O.assemble_coefficient_rhs(grid, ne, npos, kw["tau"], kw["mu_e"], kw["mu_p"], kw["diffusion"],
                                              gmg.E_OVER_EPS0_CM)
    a = torch.empty(shape, dtype=torch.float64, device=DEV)
    f = torch.empty(shape, dtype=torch.float64, device=DEV)
    gmg.assemble_coefficient_rhs(p, _t(ne), _t(npos), a, f, **kw)
    np.testing.assert_allclose(_np(a), a_ref, rtol=1e-14, atol=0)
    assert np.abs(_np(f) - f_ref).max() <= 1e-13 * np.abs(f_ref).max()


def test_assembly_rejects_bad_arguments():
    shape = (8, 8, 8)
    p = _params(shape)
    ne = torch.ones(shape, dtype=torch.float64, device=DEV)
    a = torch.empty_like(ne)
    f = torch.empty_like(ne)
    with pytest.raises(gmg.GMGError) as e:
        gmg.assemble_coefficient_rhs(p, ne, ne, a, f, tau=-1.0, mu_e=1.0, mu_p=1.0)
    assert e.value.status == gmg.GMG_ERR_ARG
    with pytest.raises(gmg.GMGError):
        gmg.assemble_coefficient_rhs(p, ne, ne, ne, f, tau=1.0, mu_e=1.0, mu_p=1.0)      # a aliases n_e
    with pytest.raises(gmg.GMGError):
        gmg.assemble_coefficient_rhs(p, ne, ne, a, f, tau=1.0, mu_e=float("nan"), mu_p=1.0)


def test_time_steps_from_assembled_densities_converge_with_few_iterations():
    """The f-1 loop on a 64^3 streamer (eq. (51) densities, Sec. 5.2 mobilities,
    52 kV): assemble a and f, renew the set-up, solve warm-started from the
    previous potential; the first step uses FMG (cycle = auto).  The oracle
    takes 3-4 iterations on the warm steps of this sequence."""
    shape = (64, 64, 64)
    p = _params(shape, precision=gmg.GMG_PREC_MIXED, cycle=gmg.GMG_CYCLE_AUTO, phi_top=PHI0)
    ctx = None
    phi = torch.zeros(shape, dtype=torch.float64, device=DEV)
    a = torch.empty(shape, dtype=torch.float64, device=DEV)
    f = torch.empty(shape, dtype=torch.float64, device=DEV)
    iters = []
    for step in range(4):
        ne, npos = streamer_densities(shape, step, xp=torch, device=DEV)
        gmg.assemble_coefficient_rhs(p, ne, npos, a, f, tau=2e-12, mu_e=MU_E, mu_p=MU_P, diffusion=DIFFUSION)
        if ctx is None:
            ctx = gmg.gmg_setup(p, a)
        else:
            gmg.gmg_update_coefficient(ctx, a)
        info = gmg.fgmres_solve(ctx, f, phi)
        assert info.true_rel_residual < 1e-8
        assert info.fmg == (1 if step == 0 else 0)
        iters.append(info.iterations)
    assert max(iters[1:]) <= 4, iters


# ---------------------------------------------------------------------------
# The paper's anisotropic meshes (nz = 1.25 nx on the unit cube, coarsest 4 x 4 x 5)
# ---------------------------------------------------------------------------


def _streamer_problem(shape):
    nz, ny, nx = shape
    ne, npos = streamer_densities(shape, 0)
    a, f = O.assemble_coefficient_rhs(O.Grid(nx, ny, nz), ne, npos, 2e-12, MU_E, MU_P, DIFFUSION,
                                      gmg.E_OVER_EPS0_CM)
    return a, f


@pytest.mark.parametrize("cycle", [gmg.GMG_CYCLE_V, gmg.GMG_CYCLE_FMG])
def test_anisotropic_fp64_solve_matches_oracle(cycle):
    shape = (20, 16, 16)                      # 16 x 16 x 20 -> 8 x 8 x 10 -> 4 x 4 x 5
    a, f = _streamer_problem(shape)
    p = _params(shape, precision=gmg.GMG_PREC_FP64, orthogonalization=gmg.GMG_ORTH_MGS, cycle=cycle, phi_top=PHI0)
    ref, rinfo, _ = O.solve(_oracle_hierarchy(a, p), a, f)
    ctx = gmg.gmg_setup(p, _t(a))
    assert gmg.gmg_level_info(ctx, 0)["shape"] == (5, 4, 4)
    phi = torch.zeros(shape, dtype=torch.float64, device=DEV)
    info = gmg.fgmres_solve(ctx, _t(f), phi)
    assert info.iterations == rinfo.iterations
    _close(_np(phi), ref, 1e-10)


@pytest.mark.parametrize("shape", [(40, 32, 32), (80, 64, 64)])
def test_anisotropic_mixed_solve_meets_tolerance(shape):
    a, f = _streamer_problem(shape)
    p = _params(shape, precision=gmg.GMG_PREC_MIXED, cycle=gmg.GMG_CYCLE_AUTO, phi_top=PHI0)
    ctx = gmg.gmg_setup(p, _t(a))
    phi = torch.zeros(shape, dtype=torch.float64, device=DEV)
    info = gmg.fgmres_solve(ctx, _t(f), phi)
    assert info.fmg == 1 and info.true_rel_residual < 1e-8
    assert _true_residual(shape, _oracle_hierarchy(a, p), a, f, _np(phi)) < 1e-8
    ref, _, _ = O.solve(O.OracleParams(coarse_min=4, phi_top=PHI0, rtol=1e-11), a, f)
    _close(_np(phi), ref, 1e-6)


# ---------------------------------------------------------------------------
# The other Krylov methods of the paper's comparison (Tables t1, t2)
# ---------------------------------------------------------------------------

KRYLOV = ["fgmres", "gmres", "cg", "fcg", "cgs", "bicgstab"]


@pytest.mark.parametrize("method", KRYLOV)
def test_krylov_fp64_matches_oracle(method):
    inp = make_inputs("channel128", n=32)
    shape = inp["a"].shape
    p = _params(shape, precision=gmg.GMG_PREC_FP64, orthogonalization=gmg.GMG_ORTH_MGS)
    ref, rinfo, _ = O.solve(_oracle_hierarchy(inp["a"], p), inp["a"], inp["f"], method=method)
    ctx = gmg.gmg_setup(p, _t(inp["a"]))
    phi = torch.zeros(shape, dtype=torch.float64, device=DEV)
    info = gmg.gmg_krylov_solve(ctx, method, _t(inp["f"]), phi)
    assert info.converged and info.true_rel_residual < 1e-8
    assert info.iterations == rinfo.iterations, (info.iterations, rinfo.iterations)
    _close(_np(phi), ref, 1e-9)


@pytest.mark.parametrize("method", KRYLOV)
def test_krylov_mixed_meets_the_true_residual(method):
    inp = make_inputs("twochannel512", n=64)
    shape = inp["a"].shape
    p = _params(shape, precision=gmg.GMG_PREC_MIXED)
    ctx = gmg.gmg_setup(p, _t(inp["a"]))
    phi = torch.zeros(shape, dtype=torch.float64, device=DEV)
    info = gmg.gmg_krylov_solve(ctx, method, _t(inp["f"]), phi)
    assert info.converged and info.true_rel_residual < 1e-8
    assert _true_residual(shape, _oracle_hierarchy(inp["a"], p), inp["a"], inp["f"], _np(phi)) < 1e-8
    per_iter = 2 if method in ("cgs", "bicgstab") else 1
    extra = info.restarts if method == "gmres" else 0      # GMRES: one more M per cycle for x
    assert info.precond_calls == per_iter * info.iterations + extra


def test_krylov_rejects_unknown_method_and_short_restart():
    shape = (16, 16, 16)
    inp = make_inputs("channel128", shape=shape)
    ctx = gmg.gmg_setup(_params(shape, restart=5), _t(inp["a"]))
    phi = torch.zeros(shape, dtype=torch.float64, device=DEV)
    with pytest.raises(gmg.GMGError) as e:
        gmg.gmg_krylov_solve(ctx, 17, _t(inp["f"]), phi)
    assert e.value.status == gmg.GMG_ERR_ARG
    with pytest.raises(gmg.GMGError):
        gmg.gmg_krylov_solve(ctx, "bicgstab", _t(inp["f"]), phi)     # needs restart >= 7
    info = gmg.gmg_krylov_solve(ctx, "gmres", _t(inp["f"]), phi)     # GMRES works with any restart
    assert info.true_rel_residual < 1e-8


# ---------------------------------------------------------------------------
# The semi-implicit time step: MUSCL/Koren transport stages, eqs. (e1)-(e2)
# ---------------------------------------------------------------------------

from paper_1812_08606_gb300.streamer import SemiImplicitStepper  # noqa: E402


@pytest.mark.parametrize("shape,lengths", [(RAGGED, (1.0, 1.0, 1.0)), ((8, 24, 144), (2.0, 1.0, 0.5)),
                                           ((4, 2, 34), (1.0, 1.0, 1.0)), ((64, 75, 100), (1.0, 0.7, 0.6))])
def test_transport_stage_matches_oracle(shape, lengths):
    nz, ny, nx = shape
    grid = O.Grid(nx, ny, nz, *lengths)
    ne, npos = _densities(shape, 350)
    he, hp = ne * (1 + 0.1 * random_field(352, shape)), npos * (1 + 0.1 * random_field(353, shape))
    phi = 3e4 * random_field(351, shape) + 1e4
    p = _params(shape, lx=lengths[0], ly=lengths[1], lz=lengths[2], phi_bottom=-2e3, phi_top=5e4)
    kw = dict(mu_e=MU_E, mu_p=MU_P, diffusion=DIFFUSION)
    ref_e, ref_p = O.transport_stage(grid, ne, npos, he, hp, phi, -2e3, 5e4, MU_E, MU_P, DIFFUSION, 3e-12)
    oe = torch.empty(shape, dtype=torch.float64, device=DEV)
    op = torch.empty_like(oe)
    gmg.transport_stage(p, _t(ne), _t(npos), _t(he), _t(hp), _t(phi), 3e-12, oe, op, **kw)
    assert np.abs(_np(oe) - ref_e).max() <= 1e-12 * np.abs(ref_e).max()
    assert np.abs(_np(op) - ref_p).max() <= 1e-12 * np.abs(ref_p).max()
    # in place on the base arrays gives the same
    be, bp = _t(ne), _t(npos)
    gmg.transport_stage(p, be, bp, _t(he), _t(hp), _t(phi), 3e-12, be, bp, **kw)
    assert torch.equal(be, oe) and torch.equal(bp, op)


def test_transport_stage_without_electron_mobility():
    """mu_e = 0 takes the kernel variant with the electron diffusion as second
    differences (with mu_e > 0 it rides on the face values); both against the
    oracle, and both with diffusion."""
    shape = (12, 20, 40)
    grid = O.Grid(40, 20, 12, 1.0, 0.8, 0.6)
    ne, npos = _densities(shape, 360)
    phi = 2e4 * random_field(361, shape)
    p = _params(shape, lx=1.0, ly=0.8, lz=0.6, phi_bottom=0.0, phi_top=2e4)
    for mu_e in (0.0, MU_E):
        ref_e, ref_p = O.transport_stage(grid, ne, npos, ne, npos, phi, 0.0, 2e4, mu_e, MU_P, DIFFUSION, 3e-12)
        oe = torch.empty(shape, dtype=torch.float64, device=DEV)
        op = torch.empty_like(oe)
        gmg.transport_stage(p, _t(ne), _t(npos), _t(ne), _t(npos), _t(phi), 3e-12, oe, op, mu_e=mu_e, mu_p=MU_P,
                            diffusion=DIFFUSION)
        assert np.abs(_np(oe) - ref_e).max() <= 1e-12 * np.abs(ref_e).max()
        assert np.abs(_np(op) - ref_p).max() <= 1e-12 * np.abs(ref_p).max()


def test_transport_stage_rejects_aliasing():
    shape = (8, 8, 8)
    p = _params(shape)
    x = [torch.ones(shape, dtype=torch.float64, device=DEV) for _ in range(4)]
    phi = torch.zeros(shape, dtype=torch.float64, device=DEV)
    with pytest.raises(gmg.GMGError):
        gmg.transport_stage(p, x[0], x[1], x[2], x[3], phi, 1.0, x[2], x[1], mu_e=1.0, mu_p=1.0)   # out = eval
    with pytest.raises(gmg.GMGError):
        gmg.transport_stage(p, x[0], x[1], x[2], x[3], phi, 1.0, x[0], x[0], mu_e=1.0, mu_p=1.0)   # out_e = out_p


@pytest.mark.parametrize("shape,lengths,mu_e", [(RAGGED, (1.0, 1.0, 1.0), MU_E), ((48, 20, 72), (1.0, 0.5, 1.5), MU_E),
                                                 ((48, 20, 72), (1.0, 0.5, 1.5), 0.0)])
def test_transport_step_matches_two_stages_and_oracle(shape, lengths, mu_e):
    """Predictor + corrector with the shared ionization rate: bit-identical to
    the two transport_stage calls, and to the oracle's stages within 1e-12
    (mu_e = 0 takes the kernel variant without the diffusion on the faces)."""
    nz, ny, nx = shape
    grid = O.Grid(nx, ny, nz, *lengths)
    ne, npos = _densities(shape, 380)
    phi = 3e4 * random_field(381, shape) + 1e4
    p = _params(shape, lx=lengths[0], ly=lengths[1], lz=lengths[2], phi_bottom=-1e3, phi_top=4e4)
    kw = dict(mu_e=mu_e, mu_p=MU_P, diffusion=DIFFUSION)
    tau = 2e-12
    args = (phi, -1e3, 4e4, mu_e, MU_P, DIFFUSION)
    he_ref, hp_ref = O.transport_stage(grid, ne, npos, ne, npos, *args, 0.5 * tau)
    ref_e, ref_p = O.transport_stage(grid, ne, npos, he_ref, hp_ref, *args, tau)
    z = lambda: torch.empty(shape, dtype=torch.float64, device=DEV)   # noqa: E731
    he, hp, oe, op, rate = z(), z(), z(), z(), z()
    gmg.transport_step(p, _t(ne), _t(npos), _t(phi), tau, he, hp, oe, op, rate, **kw)
    assert np.abs(_np(oe) - ref_e).max() <= 1e-12 * np.abs(ref_e).max()
    assert np.abs(_np(op) - ref_p).max() <= 1e-12 * np.abs(ref_p).max()
    assert np.abs(_np(he) - he_ref).max() <= 1e-12 * np.abs(he_ref).max()
    # the same two stages through transport_stage (the rate computed in place)
    se, sp, te, tp = z(), z(), z(), z()
    gmg.transport_stage(p, _t(ne), _t(npos), _t(ne), _t(npos), _t(phi), 0.5 * tau, se, sp, **kw)
    gmg.transport_stage(p, _t(ne), _t(npos), se, sp, _t(phi), tau, te, tp, **kw)
    assert torch.equal(se, he) and torch.equal(sp, hp) and torch.equal(te, oe) and torch.equal(tp, op)
    # the rate is alpha(|E|) mu_e |E| of the central-difference field
    ex, ey, ez = O.field_from_potential(grid, phi, -1e3, 4e4)
    eabs = np.sqrt(ex * ex + ey * ey + ez * ez)
    np.testing.assert_allclose(_np(rate), O.ionization_coefficient(eabs) * mu_e * eabs, rtol=1e-12, atol=0)
    # in place on n
    be, bp = _t(ne), _t(npos)
    gmg.transport_step(p, be, bp, _t(phi), tau, he, hp, be, bp, rate, **kw)
    assert torch.equal(be, oe) and torch.equal(bp, op)


def test_transport_step_rejects_aliasing():
    shape = (8, 8, 8)
    p = _params(shape)
    x = [torch.ones(shape, dtype=torch.float64, device=DEV) for _ in range(7)]
    ne, np_, phi, he, hp, rate, oe = x
    kw = dict(mu_e=1.0, mu_p=1.0)
    for args in [(ne, np_, phi, 1.0, ne, hp, oe, oe.clone(), rate),      # half = n
                 (ne, np_, phi, 1.0, he, hp, oe, oe.clone(), oe),        # rate = out
                 (ne, np_, phi, 1.0, he, he, oe, oe.clone(), rate),      # half_e = half_p
                 (ne, np_, phi, 1.0, he, hp, phi, oe, rate),              # out = phi
                 (ne, np_, phi, 1.0, he, hp, np_, ne, rate),              # out swapped with n
                 (ne, np_, phi, float("nan"), he, hp, oe, oe.clone(), rate)]:
        with pytest.raises(gmg.GMGError):
            gmg.transport_step(p, *args, **kw)


def test_round_to_f32_matches_the_conversion_instruction():
    """The integer-pipe FP64 -> FP32 rounding equals the hardware conversion
    bit for bit: random bit patterns over the whole FP64 range, values near
    the FP32 limits and subnormals, exact ties (both parities), overflow,
    zeros, infinities; NaN stays NaN."""
    rng = np.random.default_rng(390)
    bits = rng.integers(0, 2 ** 63, size=1 << 20, dtype=np.int64).astype(np.uint64)
    bits[::2] |= np.uint64(1) << np.uint64(63)
    rnd = bits.view(np.float64)
    # values around the FP32 grid: FP32 values plus offsets of about half an FP32 ulp
    f = rng.standard_normal(1 << 18).astype(np.float32)
    g = f.astype(np.float64)
    ulp = np.spacing(np.abs(f)).astype(np.float64)
    ties = np.concatenate([g + 0.5 * ulp, g - 0.5 * ulp, g + 0.5 * ulp * (1 + 2.0 ** -30), g + 0.5 * ulp * (1 - 2.0 ** -30)])
    fmax, tiny = float(np.finfo(np.float32).max), float(np.finfo(np.float32).smallest_subnormal)
    edge = np.array([0.0, -0.0, np.inf, -np.inf, fmax, -fmax, fmax * (1 + 2.0 ** -25), fmax * (1 + 2.0 ** -24),
                     fmax * 2, 1e300, -1e300, tiny, tiny / 2, tiny * 0.5000001, tiny * 1.5, tiny * 2.5, tiny / 3,
                     float(np.finfo(np.float32).tiny), float(np.finfo(np.float32).tiny) * (1 - 2.0 ** -25),
                     5e-324, -5e-324, 1e-310, 2.0 ** -149, 2.0 ** -150, 2.0 ** -150 * (1 + 2.0 ** -40),
                     2.0 ** -126 - 2.0 ** -150, 1.0, -1.0, 1 + 2.0 ** -24, 1 + 3 * 2.0 ** -24, 3.0 ** 40])
    sub = rng.uniform(-1, 1, 1 << 16) * 2.0 ** rng.uniform(-160, -120, 1 << 16)
    x = np.concatenate([rnd, ties, edge, sub])
    src = torch.from_numpy(x).to(DEV)
    dst = torch.empty(x.size, dtype=torch.float32, device=DEV)
    gmg.gmg_round_to_f32(src, dst)
    ref = src.float()   # the hardware conversion, round to nearest even
    torch.cuda.synchronize()
    nan = torch.isnan(src)
    assert torch.isnan(dst[nan]).all()
    got, want = dst[~nan].view(torch.int32), ref[~nan].view(torch.int32)
    bad = (got != want).nonzero()
    assert bad.numel() == 0, (x[~nan.cpu().numpy()][bad[:5].cpu().numpy().ravel()], got[bad[:5]].cpu(), want[bad[:5]].cpu())


def test_semi_implicit_step_fp64_matches_oracle():
    shape = (16, 16, 16)
    ne, npos = streamer_densities(shape, 0)
    p = _params(shape, precision=gmg.GMG_PREC_FP64, orthogonalization=gmg.GMG_ORTH_MGS, cycle=gmg.GMG_CYCLE_AUTO,
                phi_top=PHI0)
    ref_e, ref_p, ref_phi, rinfo = O.semi_implicit_step(_oracle_hierarchy(ne, p), ne, npos, 2e-12, MU_E, MU_P,
                                                        DIFFUSION, gmg.E_OVER_EPS0_CM)
    st = SemiImplicitStepper(p, 2e-12, MU_E, MU_P, DIFFUSION)
    oe = torch.empty(shape, dtype=torch.float64, device=DEV)
    op = torch.empty_like(oe)
    info = st.step(_t(ne), _t(npos), oe, op)
    assert info.iterations == rinfo.iterations and info.fmg == 1
    _close(_np(st.phi), ref_phi, 1e-10)
    assert np.abs(_np(oe) - ref_e).max() <= 1e-9 * np.abs(ref_e).max()
    assert np.abs(_np(op) - ref_p).max() <= 1e-9 * np.abs(ref_p).max()
    st.close()


def test_semi_implicit_steps_mixed_stay_positive_and_warm():
    """Five 2 ps steps of the eq. (51) streamer at 64^3 in 52 kV: the densities
    stay finite and non-negative, the first step takes FMG and later steps
    need few iterations from the previous potential."""
    shape = (64, 64, 64)
    ne0, np0 = streamer_densities(shape, 0, xp=torch, device=DEV)
    p = _params(shape, precision=gmg.GMG_PREC_MIXED, cycle=gmg.GMG_CYCLE_AUTO, phi_top=PHI0)
    st = SemiImplicitStepper(p, 2e-12, MU_E, MU_P, DIFFUSION)
    ne, npos = ne0.clone(), np0.clone()
    iters = []
    for _ in range(5):
        info = st.step(ne, npos, ne, npos)
        assert info.true_rel_residual < 1e-8
        iters.append(info.iterations)
    assert torch.isfinite(ne).all() and torch.isfinite(npos).all()
    assert ne.min().item() >= -1e-6 * ne0.max().item() and npos.min().item() >= -1e-6 * np0.max().item()
    assert not torch.equal(ne, ne0)
    assert max(iters[1:]) <= 5, iters
    st.close()


# ---------------------------------------------------------------------------
# Edge cases of the first-step, Krylov and transport entry points
# ---------------------------------------------------------------------------


def test_fmg_on_a_single_level_is_the_direct_solve():
    shape = (4, 4, 6)                      # coarse_min 4: one level, the dense Cholesky
    a = random_coefficient(360, shape, 1e2)
    f = random_field(361, shape)
    p = _params(shape, coarse_min=4, precision=gmg.GMG_PREC_FP64, cycle=gmg.GMG_CYCLE_FMG)
    ctx = gmg.gmg_setup(p, _t(a))
    assert gmg.gmg_num_levels(ctx) == 1
    phi = torch.zeros(shape, dtype=torch.float64, device=DEV)
    info = gmg.fgmres_solve(ctx, _t(f), phi)
    assert info.iterations == 1 and info.true_rel_residual < 1e-12


@pytest.mark.parametrize("method", ["cg", "bicgstab", "gmres"])
def test_krylov_iteration_cap_reports_not_converged(method):
    inp = make_inputs("twochannel512", n=32)
    shape = inp["a"].shape
    ctx = gmg.gmg_setup(_params(shape, max_iters=2), _t(inp["a"]))
    phi = torch.zeros(shape, dtype=torch.float64, device=DEV)
    info = gmg.gmg_krylov_solve(ctx, method, _t(inp["f"]), phi)
    assert info.converged == 0 and info.iterations == 2
    assert np.isfinite(_np(phi)).all()


@pytest.mark.parametrize("shape", [(1, 5, 6), (3, 1, 8), (5, 6, 2)])
def test_transport_and_assembly_on_thin_grids(shape):
    nz, ny, nx = shape
    grid = O.Grid(nx, ny, nz)
    ne, npos = _densities(shape, 370)
    phi = 1e4 * random_field(371, shape)
    p = _params(shape, phi_top=3e3)
    ref_e, ref_p = O.transport_stage(grid, ne, npos, ne, npos, phi, 0.0, 3e3, MU_E, MU_P, DIFFUSION, 2e-12)
    oe = torch.empty(shape, dtype=torch.float64, device=DEV)
    op = torch.empty_like(oe)
    gmg.transport_stage(p, _t(ne), _t(npos), _t(ne), _t(npos), _t(phi), 2e-12, oe, op, mu_e=MU_E, mu_p=MU_P,
                        diffusion=DIFFUSION)
    assert np.abs(_np(oe) - ref_e).max() <= 1e-12 * np.abs(ref_e).max()
    assert np.abs(_np(op) - ref_p).max() <= 1e-12 * np.abs(ref_p).max()
    a_ref, f_ref = O.assemble_coefficient_rhs(grid, ne, npos, 2e-12, MU_E, MU_P, DIFFUSION, gmg.E_OVER_EPS0_CM)
    a = torch.empty_like(oe)
    f = torch.empty_like(oe)
    gmg.assemble_coefficient_rhs(p, _t(ne), _t(npos), a, f, tau=2e-12, mu_e=MU_E, mu_p=MU_P, diffusion=DIFFUSION)
    np.testing.assert_allclose(_np(a), a_ref, rtol=1e-14)
    assert np.abs(_np(f) - f_ref).max() <= 1e-13 * np.abs(f_ref).max()

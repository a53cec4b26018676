"""Plain FP64 CPU oracle for the GMG-preconditioned FGMRES Poisson-type solve.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
baseline leg of the benchmark may import this module.  It shares no code with
the CUDA library; both sides only read the seeded inputs of
``streamer_inputs``.

It computes, slowly and literally, what the paper's elliptic solver computes
(Lin, Zhuang, Cai, Zeng, Bao, "An efficient and accurate MPI-based parallel
simulator for streamer discharges in three dimensions"):

* the cell-centred 7-point finite-volume operator of eq. (e18), Sec. 2.2, with
  face coefficients equal to the mean of the two adjacent cells;
* the Dirichlet plates / Neumann side-walls of the model eq. (eM), Sec. 1,
  imposed through ghost cells (Sec. 2.2 and Sec. 4);
* FGMRES with right preconditioning, Algorithm 1 (Sec. 3.1), with
  modified Gram-Schmidt, restarts and the stopping rule eq. (criterion) of
  Sec. 5.2;
* one geometric-multigrid V-cycle from a zero guess as the preconditioner
  (Sec. 3.2, eq. (eRichard), Appendix A), or full multigrid for a solve
  without a previous potential (the first time step, Sec. 3.2);
* the Chebyshev smoother eq. (smootheq)-(qntn)-(e19) with a one-step SSOR
  preconditioner and eigen bounds 1.1 / 0.1 times the largest Ritz value of a
  10-step Arnoldi run (Sec. 3.2);
* a direct (Cholesky) solve on the coarsest grid (Sec. 3.2);
* E = -grad(phi) by central differences (Sec. 2.2);
* the coefficient and right-hand side of eq. (semi2) / (e18) from the
  electron and ion densities (Sec. 2.1, 2.2);
* the second-order semi-implicit step eqs. (e1)-(e2) with the MUSCL / Koren
  finite-volume transport of Sec. 2.2;
* the discrete adjoint of the solve (not in the paper; derived from e18).

Readings of points the paper leaves open (each is listed with its reason in
the design notes of the repository):

R1 boundary-face coefficient on the plates equals the cell's own coefficient;
R2 Dirichlet ghost phi_g = 2 g - phi_p (linear extrapolation to the plate);
R3 coarse operators (default, "series") carry one coefficient per face,
   homogenised from the finer level's faces: along the face normal the three
   fine links between the two coarse cell centres act in series, across it
   the four fine columns act in parallel; the plates' faces likewise.  The
   alternative "mean" re-discretises eq. (e18) from the 8-child mean of a;
R4 restriction = mean of 8 children; prolongation (default "opdep") =
   per axis a 1-D interpolation between the parent and the neighbour on the
   child's side weighted by the series conductances of the fine links in
   between (harmonic), combined as a tensor product over x, y, z; with a
   constant coefficient it is the cell-centred trilinear one, which stays an
   option, as does piecewise constant;
R5 "one-step local SSOR" = one symmetric Gauss-Seidel sweep (omega = 1) in
   red-black order (red = (i+j+k) even): red, black, red half-sweeps;
R6 "quadratic-polynomial" Chebyshev: the smoother is defined by p_n in
   eq. (smootheq) with q_{n+1}(x) = 1 - x p_n(x); a quadratic p_2 gives
   q_3 = T_3 (scaled), i.e. 3 Chebyshev steps per smoothing;
R7 the 10-step Arnoldi for the eigen bounds runs on the smoother's operator
   B^{-1} A_l from a splitmix64-hash start vector;
R8 after FGMRES's own stopping test, the true residual ||b - A x|| / ||b|| is
   also required to be below the tolerance, else the method restarts;
R14 full multigrid carries the right-hand side down by the same 8-child mean
   as the residuals, prolongs each level's result with the V-cycle's
   prolongation and takes one V-cycle per level;
R15 the densities take homogeneous Neumann ghosts in the diffusion term of
   eq. (e18), and the mobilities enter with their magnitudes;
R19 transport: face values by MUSCL with the Koren limiter
   phi(r) = max(0, min(2r, (1+2r)/3, 2)), densities with two layers of
   Neumann ghosts, face fields from phi with the solve's ghosts (mirror on the
   side walls, 2 g - phi on the plates), |E| of the source from the
   cell-centred central differences.

Array layout: ``(nz, ny, nx)`` float64, x fastest.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

# ---------------------------------------------------------------------------
# Grid and parameters
# ---------------------------------------------------------------------------


@dataclass
class OracleParams:
    """Solver parameters; defaults are the paper's values unless noted."""

    lx: float = 1.0
    ly: float = 1.0
    lz: float = 1.0
    phi_bottom: float = 0.0      # Dirichlet data at z = 0   (eq. (eM) plates)
    phi_top: float = 1.0         # Dirichlet data at z = lz
    coarse_min: int = 4          # coarsest grid: smallest side reaches this
    cheb_steps: int = 3          # R6
    restart: int = 20            # FGMRES m; the paper uses 30 (Sec. 3.1)
    max_iters: int = 200
    rtol: float = 1e-8           # eq. (criterion), Sec. 5.2
    eig_steps: int = 10          # Sec. 3.2
    eig_hi: float = 1.1          # Sec. 3.2
    eig_lo: float = 0.1          # Sec. 3.2
    prolongation: str = "opdep"       # R4; or "trilinear", "constant"
    coarsening: str = "series"        # R3; or "mean"
    smoother_pc: str = "sgs"          # R5; or "jacobi", "identity"
    cycle: str = "v"             # preconditioner: "v", "fmg", or "auto" (FMG for a zero guess, Sec. 3.2)


@dataclass
class Grid:
    """Uniform cell-centred grid (Sec. 2.2): cells I_{i,j,k} of size hx*hy*hz."""

    nx: int
    ny: int
    nz: int
    lx: float = 1.0
    ly: float = 1.0
    lz: float = 1.0

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def hx(self):
        return self.lx / self.nx

    @property
    def hy(self):
        return self.ly / self.ny

    @property
    def hz(self):
        return self.lz / self.nz

    @property
    def size(self):
        return self.nx * self.ny * self.nz

    def coarser(self) -> "Grid":
        return Grid(self.nx // 2, self.ny // 2, self.nz // 2, self.lx, self.ly, self.lz)


# ---------------------------------------------------------------------------
# Operator, eq. (e18)
# ---------------------------------------------------------------------------


@dataclass
class FaceCoefficients:
    """A 7-point operator of the form of eq. (e18) given by one coefficient per
    face instead of the face means of a cell coefficient (the coarse levels of
    reading R3).  a-values, before the division by h^2:
      ax (nz, ny, nx-1): face between cells i and i+1 along x; ay, az likewise;
      bottom, top (ny, nx): the plate faces (a coefficient over the half cell
      between the cell centre and the plate, as a_p is in R1).
    The side walls carry no flux."""

    ax: np.ndarray
    ay: np.ndarray
    az: np.ndarray
    bottom: np.ndarray
    top: np.ndarray

    @property
    def shape(self):
        return (self.az.shape[0] + 1,) + self.bottom.shape


def faces_of_cells(a: np.ndarray) -> FaceCoefficients:
    """The face form of eq. (e18): interior faces the mean of the two cells
    (Sec. 2.2), plate faces the cell's own coefficient (R1)."""
    return FaceCoefficients(0.5 * (a[:, :, 1:] + a[:, :, :-1]), 0.5 * (a[:, 1:, :] + a[:, :-1, :]),
                            0.5 * (a[1:] + a[:-1]), np.array(a[0], copy=True), np.array(a[-1], copy=True))


def face_coefficients(grid: Grid, a):
    """Interior face coefficients divided by h^2 (eq. (e18) and the face means
    P_{i+1/2,j,k} = (P_{i+1,j,k} + P_{i,j,k}) / 2 of Sec. 2.2), or the stored
    face values of a FaceCoefficients operator.

    Returns (cx, cy, cz) with cx[k,j,i] the coefficient of the face between
    cells i and i+1 (shape (nz,ny,nx-1)), and likewise for y and z.
    """
    if isinstance(a, FaceCoefficients):
        return a.ax / grid.hx**2, a.ay / grid.hy**2, a.az / grid.hz**2
    cx = 0.5 * (a[:, :, 1:] + a[:, :, :-1]) / grid.hx**2
    cy = 0.5 * (a[:, 1:, :] + a[:, :-1, :]) / grid.hy**2
    cz = 0.5 * (a[1:, :, :] + a[:-1, :, :]) / grid.hz**2
    return cx, cy, cz


def plate_coefficients(grid: Grid, a: np.ndarray):
    """Coefficients 2 a_p / hz^2 of the two Dirichlet plate faces (R1, R2).

    A plate face carries a_f = a_p (R1) and the ghost value 2g - phi_p (R2), so
    its flux a_p (phi_p - phi_g) / hz^2 = 2 a_p (phi_p - g) / hz^2.
    A FaceCoefficients operator gives its plate a-values the same way.
    """
    if isinstance(a, FaceCoefficients):
        return 2.0 * a.bottom / grid.hz**2, 2.0 * a.top / grid.hz**2
    return 2.0 * a[0] / grid.hz**2, 2.0 * a[-1] / grid.hz**2


def apply_operator(grid: Grid, a: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y = A x: the left-hand side of eq. (e18) with zero Dirichlet data.

    (A x)_p = sum over interior faces f=(p,q) of a_f (x_p - x_q) / h_f^2
            + sum over plate faces of p of 2 a_p x_p / hz^2.
    Side faces in x and y carry no flux (homogeneous Neumann, eq. (eM)).
    """
    cx, cy, cz = face_coefficients(grid, a)
    y = np.zeros_like(x, dtype=np.float64)
    flux = cx * (x[:, :, :-1] - x[:, :, 1:])
    y[:, :, :-1] += flux
    y[:, :, 1:] -= flux
    flux = cy * (x[:, :-1, :] - x[:, 1:, :])
    y[:, :-1, :] += flux
    y[:, 1:, :] -= flux
    flux = cz * (x[:-1, :, :] - x[1:, :, :])
    y[:-1, :, :] += flux
    y[1:, :, :] -= flux
    pb, pt = plate_coefficients(grid, a)
    y[0] += pb * x[0]
    y[-1] += pt * x[-1]
    return y


def diagonal(grid: Grid, a: np.ndarray) -> np.ndarray:
    """Diagonal of A: the sum of the face coefficients of each cell."""
    cx, cy, cz = face_coefficients(grid, a)
    d = np.zeros(grid.shape)
    d[:, :, :-1] += cx
    d[:, :, 1:] += cx
    d[:, :-1, :] += cy
    d[:, 1:, :] += cy
    d[:-1, :, :] += cz
    d[1:, :, :] += cz
    pb, pt = plate_coefficients(grid, a)
    d[0] += pb
    d[-1] += pt
    return d


def neighbour_sum(grid: Grid, a: np.ndarray, x: np.ndarray) -> np.ndarray:
    """N x = sum over interior faces f=(p,q) of a_f x_q / h_f^2, so A = D - N."""
    cx, cy, cz = face_coefficients(grid, a)
    s = np.zeros(grid.shape)
    s[:, :, :-1] += cx * x[:, :, 1:]
    s[:, :, 1:] += cx * x[:, :, :-1]
    s[:, :-1, :] += cy * x[:, 1:, :]
    s[:, 1:, :] += cy * x[:, :-1, :]
    s[:-1, :, :] += cz * x[1:, :, :]
    s[1:, :, :] += cz * x[:-1, :, :]
    return s


def apply_operator_at(grid: Grid, a: np.ndarray, x: np.ndarray, cells) -> np.ndarray:
    """(A x)_p of apply_operator at the listed cells (k, j, i) only, one cell at a
    time from its 7-point neighbourhood: each interior face adds the face mean
    (a_p + a_q)/2 times (x_p - x_q) / h^2 (eq. (e18), Sec. 2.2), a plate face adds
    2 a_p x_p / hz^2 (R1, R2), a side wall adds nothing.  For checks on grids too
    large for the whole-array form."""
    nz, ny, nx = x.shape
    steps = ((0, 0, -1, grid.hx), (0, 0, 1, grid.hx), (0, -1, 0, grid.hy), (0, 1, 0, grid.hy),
             (-1, 0, 0, grid.hz), (1, 0, 0, grid.hz))
    out = np.empty(len(cells))
    for n, (k, j, i) in enumerate(cells):
        xp, ap = float(x[k, j, i]), float(a[k, j, i])
        s = 0.0
        for dk, dj, di, h in steps:
            kk, jj, ii = k + dk, j + dj, i + di
            if 0 <= kk < nz and 0 <= jj < ny and 0 <= ii < nx:
                s += 0.5 * (ap + float(a[kk, jj, ii])) / h**2 * (xp - float(x[kk, jj, ii]))
            elif dk != 0:
                s += 2.0 * ap / grid.hz**2 * xp
        out[n] = s
    return out


def assemble_rhs(grid: Grid, a: np.ndarray, f: np.ndarray, g_bottom: float, g_top: float) -> np.ndarray:
    """b = f + the plate terms 2 a_p g / hz^2 (eq. (e18) with ghosts, R1/R2)."""
    b = np.array(f, dtype=np.float64, copy=True)
    pb, pt = plate_coefficients(grid, a)
    b[0] += pb * g_bottom
    b[-1] += pt * g_top
    return b


def dense_operator(grid: Grid, a: np.ndarray) -> np.ndarray:
    """A as a dense matrix (columns A e_i); small grids only."""
    n = grid.size
    m = np.zeros((n, n))
    e = np.zeros(n)
    for i in range(n):
        e[:] = 0.0
        e[i] = 1.0
        m[:, i] = apply_operator(grid, a, e.reshape(grid.shape)).ravel()
    return m


# ---------------------------------------------------------------------------
# Smoother: preconditioned Chebyshev, eqs. (smootheq), (qntn), (e19); SSOR (R5)
# ---------------------------------------------------------------------------


def red_mask(grid: Grid) -> np.ndarray:
    k, j, i = np.indices(grid.shape)
    return (i + j + k) % 2 == 0


def sgs_redblack(grid: Grid, a: np.ndarray, r: np.ndarray) -> np.ndarray:
    """z = B^{-1} r for one symmetric Gauss-Seidel sweep (SSOR, omega = 1) from
    z = 0 in red-black ordering (R5).

    Forward sweep: red cells, then black cells.  Backward sweep: black cells,
    then red cells.  In a 7-point stencil a black cell sees only red
    neighbours, so the backward black update repeats the forward one and the
    sweep is red, black, red.
    """
    dg = diagonal(grid, a)
    red = red_mask(grid)
    black = ~red
    z = np.zeros(grid.shape)
    z[red] = r[red] / dg[red]
    nb = neighbour_sum(grid, a, z)
    z[black] = (r[black] + nb[black]) / dg[black]
    nb = neighbour_sum(grid, a, z)
    z[red] = (r[red] + nb[red]) / dg[red]
    return z


def smoother_preconditioner(grid: Grid, a: np.ndarray, r: np.ndarray, kind: str) -> np.ndarray:
    if kind == "sgs":
        return sgs_redblack(grid, a, r)
    if kind == "jacobi":
        return r / diagonal(grid, a)
    if kind == "identity":
        return np.array(r, copy=True)
    raise ValueError(kind)


def chebyshev_smooth(grid: Grid, a: np.ndarray, b: np.ndarray, x: np.ndarray | None,
                     lam_max: float, lam_min: float, steps: int, pc: str = "sgs") -> np.ndarray:
    """``steps`` preconditioned Chebyshev iterations for A x = b (Sec. 3.2).

    The error is multiplied by q_s(B^{-1}A), q_s the scaled Chebyshev
    polynomial of eq. (qntn) on [lam_min, lam_max].  Three-term recurrence of
    the preconditioned Chebyshev iteration (Saad, Iterative Methods for Sparse
    Linear Systems, 2nd ed., Sec. 12.3):
        theta = (lmax + lmin)/2, delta = (lmax - lmin)/2, sigma = theta/delta,
        rho_0 = 1/sigma;  d_0 = B^{-1} r_0 / theta;  x_1 = x_0 + d_0;
        rho_k = 1/(2 sigma - rho_{k-1}),
        d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / delta) B^{-1} r_k,
        x_{k+1} = x_k + d_k,  with r_k = b - A x_k.
    ``x is None`` means a zero initial guess (then r_0 = b).
    """
    theta = 0.5 * (lam_max + lam_min)
    delta = 0.5 * (lam_max - lam_min)
    sigma = theta / delta
    rho = 1.0 / sigma
    if x is None:
        x = np.zeros(grid.shape)
        r = np.array(b, copy=True)
    else:
        x = np.array(x, dtype=np.float64, copy=True)
        r = b - apply_operator(grid, a, x)
    d = smoother_preconditioner(grid, a, r, pc) / theta
    x = x + d
    for _ in range(1, steps):
        rho_new = 1.0 / (2.0 * sigma - rho)
        r = b - apply_operator(grid, a, x)
        z = smoother_preconditioner(grid, a, r, pc)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * z
        x = x + d
        rho = rho_new
    return x


# ---------------------------------------------------------------------------
# Eigen bounds (Sec. 3.2, R7)
# ---------------------------------------------------------------------------

_MASK64 = (1 << 64) - 1


def splitmix64(index: np.ndarray) -> np.ndarray:
    """splitmix64 output for counter ``index`` (Steele, Lea, Flood, "Fast
    splittable pseudorandom number generators", OOPSLA 2014): state =
    (index + 1) * 0x9E3779B97F4A7C15, then the mix function of the
    published generator."""
    with np.errstate(over="ignore"):
        z = (index.astype(np.uint64) + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def hash_start_vector(n: int) -> np.ndarray:
    """u_i in [-1, 1): top 53 bits of splitmix64(i) scaled to [0,1), times 2, minus 1."""
    bits = splitmix64(np.arange(n, dtype=np.uint64)) >> np.uint64(11)
    return bits.astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


def arnoldi_hessenberg(matvec, v0: np.ndarray, steps: int) -> np.ndarray:
    """The Arnoldi process of Algorithm 1 with modified Gram-Schmidt and no
    preconditioning: returns the square upper Hessenberg H_m (m <= steps)."""
    n = v0.size
    V = [v0 / np.linalg.norm(v0)]
    H = np.zeros((steps + 1, steps))
    m = steps
    for j in range(steps):
        w = matvec(V[j]).ravel().astype(np.float64)
        for i in range(j + 1):
            H[i, j] = np.dot(w, V[i])
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] == 0.0:
            m = j + 1
            break
        V.append(w / H[j + 1, j])
    del n
    return H[:m, :m]


def estimate_eig_bounds(grid: Grid, a: np.ndarray, params: OracleParams):
    """lambda_max = eig_hi * lam_hat, lambda* = eig_lo * lam_hat with lam_hat the
    largest eigenvalue of the Arnoldi H_m of B^{-1} A_l (Sec. 3.2, R7)."""
    def matvec(v):
        return smoother_preconditioner(grid, a, apply_operator(grid, a, v.reshape(grid.shape)),
                                       params.smoother_pc)

    H = arnoldi_hessenberg(matvec, hash_start_vector(grid.size), params.eig_steps)
    lam_hat = float(np.max(np.linalg.eigvals(H).real))
    return params.eig_hi * lam_hat, params.eig_lo * lam_hat, lam_hat


# ---------------------------------------------------------------------------
# Grid transfers and hierarchy (Sec. 3.2, R3, R4)
# ---------------------------------------------------------------------------


def restrict(fine: np.ndarray) -> np.ndarray:
    """Mean of the 8 fine children of each coarse cell (R4)."""
    nz, ny, nx = fine.shape
    return fine.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).mean(axis=(1, 3, 5))


def coarsen_coefficient(a: np.ndarray) -> np.ndarray:
    """Coarse coefficient = mean of the 8 children (R3, "mean")."""
    return restrict(a)


def _pair_mean(u: np.ndarray, axis: int) -> np.ndarray:
    """Mean of neighbouring pairs (2m, 2m+1) along axis."""
    u = np.moveaxis(u, axis, 0)
    return np.moveaxis(0.5 * (u[0::2] + u[1::2]), 0, axis)


def coarsen_faces(a) -> FaceCoefficients:
    """The coarse operator of R3 ("series") from the finer level's operator
    (a cell coefficient of eq. (e18) or a FaceCoefficients).

    Take the coarse face between coarse cells I-1 and I along an axis.  Along
    the path between their centres lie, in series, half of the inner fine link
    of cell I-1 (between its two children), the whole fine link shared by the
    two coarse cells, and half of the inner fine link of cell I.  With fine
    link a-values A1, A2, A3 over the fine spacing h, the path of length 2h has
    the a-value 2 / (1/(2 A1) + 1/A2 + 1/(2 A3)).  The four fine columns that
    cross the coarse face act in parallel: the coarse face takes their mean.
    A coarse plate face: half the inner link of the boundary coarse cell in
    series with the fine plate face (a-value over h/2), 2 / (1/A + 1/P), and
    the mean over the four fine columns.  With a constant coefficient every
    coarse face gets that constant, which is eq. (e18) re-discretised."""
    f = a if isinstance(a, FaceCoefficients) else faces_of_cells(a)

    def along(links, axis):
        # links: interior fine faces along axis (n-1 of them); coarse interior faces m = 0..n/2-2
        u = np.moveaxis(links, axis, 0)
        s = 2.0 / (0.5 / u[0:-2:2] + 1.0 / u[1:-1:2] + 0.5 / u[2::2])
        return np.moveaxis(s, 0, axis)

    ax = along(f.ax, 2)
    ax = _pair_mean(_pair_mean(ax, 1), 0)
    ay = along(f.ay, 1)
    ay = _pair_mean(_pair_mean(ay, 2), 0)
    az = along(f.az, 0)
    az = _pair_mean(_pair_mean(az, 2), 1)
    bottom = _pair_mean(_pair_mean(2.0 / (1.0 / f.az[0] + 1.0 / f.bottom), 1), 0)
    top = _pair_mean(_pair_mean(2.0 / (1.0 / f.az[-1] + 1.0 / f.top), 1), 0)
    return FaceCoefficients(ax, ay, az, bottom, top)


def coarsen_level(a, params) -> object:
    """The next coarser level's operator (R3): FaceCoefficients ("series") or
    the 8-child mean of the cell coefficient ("mean")."""
    if params.coarsening == "series":
        return coarsen_faces(a)
    if params.coarsening == "mean":
        return coarsen_coefficient(a)
    raise ValueError(params.coarsening)


def _prolong_axis(e: np.ndarray, axis: int, dirichlet: bool) -> np.ndarray:
    """1-D cell-centred linear interpolation along ``axis``: a fine child sits a
    quarter coarse cell from its parent's centre, so it takes 3/4 of the
    parent and 1/4 of the neighbour on its side.  Beyond the domain the
    neighbour is a ghost: equal to the parent at a Neumann wall, minus the
    parent at a (homogeneous) Dirichlet plate."""
    e = np.moveaxis(e, axis, 0)
    n = e.shape[0]
    ghost_lo = -e[:1] if dirichlet else e[:1]
    ghost_hi = -e[-1:] if dirichlet else e[-1:]
    left = np.concatenate([ghost_lo, e[:-1]], axis=0)    # neighbour below each parent
    right = np.concatenate([e[1:], ghost_hi], axis=0)    # neighbour above each parent
    out = np.empty((2 * n,) + e.shape[1:])
    out[0::2] = 0.75 * e + 0.25 * left
    out[1::2] = 0.75 * e + 0.25 * right
    return np.moveaxis(out, 0, axis)


def _opdep_parent_weight(links: np.ndarray, n: int, plate_lo, plate_hi) -> np.ndarray:
    """Weight of the parent for each fine cell along one axis (axis 0 of the
    arrays), from the series resistances of the fine links (R4, "opdep").

    links[m] (m = 0..n-2): a-value of the fine link between cells m and m+1.
    A child sits half a fine cell from its parent's centre (which lies on the
    parent's inner link); towards the neighbour on its side lie the fine link
    it shares with that coarse cell and half of the neighbour's inner link.  In
    units of h: R_parent = 1/(2 A_inner), R_neighbour = 1/A_shared +
    1/(2 A_neighbour_inner); the child takes the conductance-weighted mean
    (1/R_p e_p + 1/R_n e_n) / (1/R_p + 1/R_n).  At a side wall there is no
    neighbour (weight 1 on the parent, the Neumann mirror); at a plate the
    neighbour is the plate itself, value 0, over the half cell with the plate
    face's a-value P: R_n = 1/(2 P) (plate_lo / plate_hi; None for a wall)."""
    m = n // 2
    w = np.ones((n,) + links.shape[1:])
    for I in range(m):
        c = 2 * I                      # child nearer the lower neighbour I-1
        rp = 0.5 / links[c]
        if I > 0:
            rn = 1.0 / links[c - 1] + 0.5 / links[c - 2]
            w[c] = (1.0 / rp) / (1.0 / rp + 1.0 / rn)
        elif plate_lo is not None:
            rn = 0.5 / plate_lo
            w[c] = (1.0 / rp) / (1.0 / rp + 1.0 / rn)
        c = 2 * I + 1                  # child nearer the upper neighbour I+1
        rp = 0.5 / links[c - 1]
        if I < m - 1:
            rn = 1.0 / links[c] + 0.5 / links[c + 1]
            w[c] = (1.0 / rp) / (1.0 / rp + 1.0 / rn)
        elif plate_hi is not None:
            rn = 0.5 / plate_hi
            w[c] = (1.0 / rp) / (1.0 / rp + 1.0 / rn)
    return w


def prolong_weights(fine_coef):
    """Per fine cell, the parent weights (wx, wy, wz) of the operator-dependent
    prolongation into the level whose operator is fine_coef (R4, "opdep")."""
    f = fine_coef if isinstance(fine_coef, FaceCoefficients) else faces_of_cells(fine_coef)
    nz, ny, nx = f.az.shape[0] + 1, f.ay.shape[1] + 1, f.ax.shape[2] + 1
    wx = np.moveaxis(_opdep_parent_weight(np.moveaxis(f.ax, 2, 0), nx, None, None), 0, 2)
    wy = np.moveaxis(_opdep_parent_weight(np.moveaxis(f.ay, 1, 0), ny, None, None), 0, 1)
    wz = _opdep_parent_weight(f.az, nz, f.bottom, f.top)
    return wx, wy, wz


def _prolong_opdep(coarse: np.ndarray, fine_coef) -> np.ndarray:
    """e_child = sum over the 8 combinations of (parent or neighbour) per axis
    of the product of the per-axis weights times that coarse value; the
    neighbour beyond a plate is 0, beyond a side wall it has weight 0."""
    wx, wy, wz = prolong_weights(fine_coef)
    nzc, nyc, nxc = coarse.shape
    nz, ny, nx = 2 * nzc, 2 * nyc, 2 * nxc
    k, j, i = np.arange(nz), np.arange(ny), np.arange(nx)
    own = (k // 2, j // 2, i // 2)
    nbr = (np.where(k % 2 == 0, k // 2 - 1, k // 2 + 1), np.where(j % 2 == 0, j // 2 - 1, j // 2 + 1),
           np.where(i % 2 == 0, i // 2 - 1, i // 2 + 1))
    inside = [(nbr[0] >= 0) & (nbr[0] < nzc), (nbr[1] >= 0) & (nbr[1] < nyc), (nbr[2] >= 0) & (nbr[2] < nxc)]
    out = np.zeros((nz, ny, nx))
    for sz in (0, 1):
        for sy in (0, 1):
            for sx in (0, 1):
                kk = np.clip(nbr[0], 0, nzc - 1) if sz else own[0]
                jj = np.clip(nbr[1], 0, nyc - 1) if sy else own[1]
                ii = np.clip(nbr[2], 0, nxc - 1) if sx else own[2]
                val = coarse[kk[:, None, None], jj[None, :, None], ii[None, None, :]]
                if sz:   # beyond a plate the neighbour value is the homogeneous Dirichlet 0
                    val = val * inside[0][:, None, None]
                w = (1.0 - wz if sz else wz) * (1.0 - wy if sy else wy) * (1.0 - wx if sx else wx)
                out += w * val
    return out


def prolong(coarse: np.ndarray, kind: str = "trilinear", fine_coef=None) -> np.ndarray:
    """Coarse-to-fine interpolation P_{l-1,l} (R4); "opdep" needs the fine
    level's operator (cell coefficient or FaceCoefficients)."""
    if kind == "constant":
        return coarse.repeat(2, axis=0).repeat(2, axis=1).repeat(2, axis=2)
    if kind == "opdep":
        return _prolong_opdep(coarse, fine_coef)
    if kind != "trilinear":
        raise ValueError(kind)
    e = _prolong_axis(coarse, 2, dirichlet=False)   # x: Neumann walls
    e = _prolong_axis(e, 1, dirichlet=False)        # y: Neumann walls
    e = _prolong_axis(e, 0, dirichlet=True)         # z: Dirichlet plates
    return e


@dataclass
class Level:
    grid: Grid
    a: object          # cell coefficient (finest level, or R3 "mean") or FaceCoefficients
    lam_max: float = 0.0
    lam_min: float = 0.0
    lam_hat: float = 0.0


@dataclass
class Hierarchy:
    params: OracleParams
    levels: list = field(default_factory=list)   # levels[0] coarsest ... levels[-1] finest
    coarse_chol: object = None


def level_count(nx: int, ny: int, nz: int, coarse_min: int) -> int:
    """Number of grids: halve every side until the smallest reaches coarse_min."""
    count = 1
    while min(nx, ny, nz) > coarse_min:
        if nx % 2 or ny % 2 or nz % 2:
            raise ValueError("grid sides must halve down to the coarsest grid")
        nx, ny, nz = nx // 2, ny // 2, nz // 2
        count += 1
    if min(nx, ny, nz) != coarse_min:
        raise ValueError("smallest side must reach coarse_min by halving")
    return count


def build_hierarchy(grid: Grid, a: np.ndarray, params: OracleParams) -> Hierarchy:
    """Coefficients per level, eigen bounds per smoothed level, and the Cholesky
    factor of the coarsest operator (the set-up renewed each time step, Sec. 3)."""
    nlev = level_count(grid.nx, grid.ny, grid.nz, params.coarse_min)
    fine_to_coarse = [Level(grid, np.asarray(a, dtype=np.float64))]
    for _ in range(nlev - 1):
        prev = fine_to_coarse[-1]
        fine_to_coarse.append(Level(prev.grid.coarser(), coarsen_level(prev.a, params)))
    hier = Hierarchy(params, list(reversed(fine_to_coarse)))
    for lev in hier.levels[1:]:
        lev.lam_max, lev.lam_min, lev.lam_hat = estimate_eig_bounds(lev.grid, lev.a, params)
    coarse = hier.levels[0]
    hier.coarse_chol = scipy.linalg.cho_factor(dense_operator(coarse.grid, coarse.a), lower=True)
    return hier


def coarse_solve(hier: Hierarchy, b: np.ndarray) -> np.ndarray:
    """Direct solve A_1 x = b on the coarsest grid (Sec. 3.2): Cholesky."""
    g = hier.levels[0].grid
    return scipy.linalg.cho_solve(hier.coarse_chol, b.ravel()).reshape(g.shape)


# ---------------------------------------------------------------------------
# V-cycle preconditioner: eq. (eRichard), Appendix A
# ---------------------------------------------------------------------------


def vcycle(hier: Hierarchy, b: np.ndarray, level: int | None = None) -> np.ndarray:
    """One V-cycle from a zero guess for A_l x = b (Sec. 3.2, Appendix A):
    pre-smooth from 0, restrict the residual, recurse, prolong and add the
    correction, post-smooth with the same polynomial; the coarsest grid is
    solved directly.  The map b -> x is the matrix M_l of Appendix A."""
    p = hier.params
    if level is None:
        level = len(hier.levels) - 1
    if level == 0:
        return coarse_solve(hier, b)
    lev = hier.levels[level]
    x = chebyshev_smooth(lev.grid, lev.a, b, None, lev.lam_max, lev.lam_min, p.cheb_steps, p.smoother_pc)
    r = b - apply_operator(lev.grid, lev.a, x)
    e = vcycle(hier, restrict(r), level - 1)
    x = x + prolong(e, p.prolongation, lev.a)
    x = chebyshev_smooth(lev.grid, lev.a, b, x, lev.lam_max, lev.lam_min, p.cheb_steps, p.smoother_pc)
    return x


def vcycle_from(hier: Hierarchy, b: np.ndarray, x: np.ndarray, level: int | None = None) -> np.ndarray:
    """One V-cycle for A_l x = b starting from the guess x: pre-smoothing
    starts from x, the coarse-grid correction and post-smoothing are those of
    ``vcycle``.  The result is x + M_l (b - A_l x)."""
    p = hier.params
    if level is None:
        level = len(hier.levels) - 1
    if level == 0:
        return coarse_solve(hier, b)
    lev = hier.levels[level]
    x = chebyshev_smooth(lev.grid, lev.a, b, x, lev.lam_max, lev.lam_min, p.cheb_steps, p.smoother_pc)
    r = b - apply_operator(lev.grid, lev.a, x)
    e = vcycle(hier, restrict(r), level - 1)
    x = x + prolong(e, p.prolongation, lev.a)
    x = chebyshev_smooth(lev.grid, lev.a, b, x, lev.lam_max, lev.lam_min, p.cheb_steps, p.smoother_pc)
    return x


def fmg(hier: Hierarchy, b: np.ndarray) -> np.ndarray:
    """Full multigrid, the preconditioner of the first time step (Sec. 3.2):
    the right-hand side is carried down to every level by the same 8-child
    mean as the residuals; the coarsest equation is solved directly; going
    up, each level starts from the prolonged solution of the level below and
    takes one V-cycle."""
    p = hier.params
    top = len(hier.levels) - 1
    rhs = [None] * (top + 1)
    rhs[top] = b
    for level in range(top, 0, -1):
        rhs[level - 1] = restrict(rhs[level])
    x = coarse_solve(hier, rhs[0])
    for level in range(1, top + 1):
        x = vcycle_from(hier, rhs[level], prolong(x, p.prolongation, hier.levels[level].a), level)
    return x


# ---------------------------------------------------------------------------
# FGMRES, Algorithm 1 (Sec. 3.1) with the stopping rule eq. (criterion)
# ---------------------------------------------------------------------------


@dataclass
class SolveInfo:
    iterations: int = 0
    restarts: int = 0
    converged: bool = False
    true_rel_residual: float = float("nan")
    history: list = field(default_factory=list)   # Arnoldi residual estimates / ||b||


def _least_squares_residual(Hbar: np.ndarray, beta: float):
    """min_y || beta e_1 - Hbar y || (the least-squares step of Algorithm 1)
    by a library least-squares solve; returns (y, residual norm)."""
    rhs = np.zeros(Hbar.shape[0])
    rhs[0] = beta
    y = np.linalg.lstsq(Hbar, rhs, rcond=None)[0]
    return y, float(np.linalg.norm(rhs - Hbar @ y))


def fgmres(grid: Grid, a: np.ndarray, b: np.ndarray, x0: np.ndarray | None, precond,
           params: OracleParams) -> tuple[np.ndarray, SolveInfo]:
    """Restarted FGMRES with right preconditioning (Algorithm 1, Sec. 3.1).

    Arnoldi uses modified Gram-Schmidt; the stopping test compares the
    least-squares residual with rtol * ||b|| (eq. (criterion)); after forming
    x_k = x_0 + Z_k y_k the true residual is checked (R8) and the method
    restarts from x_k if it is not below the tolerance.
    """
    info = SolveInfo()
    m = params.restart
    x = np.zeros(grid.shape) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        info.converged = True
        info.true_rel_residual = 0.0
        return np.zeros(grid.shape), info
    while True:
        r = b - apply_operator(grid, a, x)
        beta = float(np.linalg.norm(r))
        info.true_rel_residual = beta / bnorm
        if info.true_rel_residual < params.rtol:
            info.converged = True
            return x, info
        if info.iterations >= params.max_iters or beta == 0.0:
            return x, info
        V = [r.ravel() / beta]
        Z = []
        H = np.zeros((m + 1, m))
        k = 0
        y = np.zeros(0)
        for j in range(m):
            z = precond(V[j].reshape(grid.shape)).ravel()
            Z.append(z)
            w = apply_operator(grid, a, z.reshape(grid.shape)).ravel()
            for i in range(j + 1):
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            k = j + 1
            info.iterations += 1
            y, res = _least_squares_residual(H[: j + 2, : j + 1], beta)
            info.history.append(res / bnorm)
            if H[j + 1, j] == 0.0:
                break                                   # lucky breakdown: exact in K_j
            V.append(w / H[j + 1, j])
            if res / bnorm < params.rtol or info.iterations >= params.max_iters:
                break
        for i in range(k):
            x = x + y[i] * Z[i].reshape(grid.shape)
        info.restarts += 1


# ---------------------------------------------------------------------------
# The other preconditioned Krylov methods of the paper's comparison (Sec. 5.4,
# Tables t1 and t2): GMRES, CG, FCG, CGS and BiCGSTAB with the same multigrid
# preconditioner, all right-preconditioned.  Each stops when its recurrence
# residual falls below rtol ||b||, then checks the true residual and, if that
# is not below the tolerance, starts again from the current iterate (R8).
# ---------------------------------------------------------------------------

KRYLOV_METHODS = ("fgmres", "gmres", "cg", "fcg", "cgs", "bicgstab")


def gmres(grid: Grid, a: np.ndarray, b: np.ndarray, x0: np.ndarray | None, precond,
          params: OracleParams) -> tuple[np.ndarray, SolveInfo]:
    """Restarted right-preconditioned GMRES: Arnoldi (modified Gram-Schmidt)
    on A M stores only V; after k steps x = x_0 + M (V_k y_k)."""
    info = SolveInfo()
    m = params.restart
    x = np.zeros(grid.shape) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        info.converged, info.true_rel_residual = True, 0.0
        return np.zeros(grid.shape), info
    while True:
        r = b - apply_operator(grid, a, x)
        beta = float(np.linalg.norm(r))
        info.true_rel_residual = beta / bnorm
        if info.true_rel_residual < params.rtol:
            info.converged = True
            return x, info
        if info.iterations >= params.max_iters or beta == 0.0:
            return x, info
        V = [r.ravel() / beta]
        H = np.zeros((m + 1, m))
        k = 0
        y = np.zeros(0)
        for j in range(m):
            w = apply_operator(grid, a, precond(V[j].reshape(grid.shape))).ravel()
            for i in range(j + 1):
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            k = j + 1
            info.iterations += 1
            y, res = _least_squares_residual(H[: j + 2, : j + 1], beta)
            info.history.append(res / bnorm)
            if H[j + 1, j] == 0.0:
                break
            V.append(w / H[j + 1, j])
            if res / bnorm < params.rtol or info.iterations >= params.max_iters:
                break
        u = sum(y[i] * V[i] for i in range(k))
        x = x + precond(u.reshape(grid.shape))
        info.restarts += 1


def _restarting(method_step):
    """Wrap a short-recurrence method: run it from the current x until its
    recurrence residual meets rtol ||b|| (or the iteration cap), then check the
    true residual and start it again from x if needed (R8)."""
    def run(grid, a, b, x0, precond, params):
        info = SolveInfo()
        x = np.zeros(grid.shape) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
        bnorm = float(np.linalg.norm(b))
        if bnorm == 0.0:
            info.converged, info.true_rel_residual = True, 0.0
            return np.zeros(grid.shape), info
        while True:
            r = b - apply_operator(grid, a, x)
            info.true_rel_residual = float(np.linalg.norm(r)) / bnorm
            if info.true_rel_residual < params.rtol:
                info.converged = True
                return x, info
            if info.iterations >= params.max_iters:
                return x, info
            x = method_step(grid, a, x, r, precond, params, bnorm, info)
            info.restarts += 1
    return run


def _stop(info, params, rnorm, bnorm):
    info.iterations += 1
    info.history.append(rnorm / bnorm)
    return rnorm / bnorm < params.rtol or info.iterations >= params.max_iters


@_restarting
def cg(grid, a, x, r, precond, params, bnorm, info):
    """Preconditioned conjugate gradients (Saad, Algorithm 9.1)."""
    z = precond(r)
    p = z.copy()
    rho = float(np.vdot(r, z))
    while True:
        q = apply_operator(grid, a, p)
        alpha = rho / float(np.vdot(p, q))
        x = x + alpha * p
        r = r - alpha * q
        if _stop(info, params, float(np.linalg.norm(r)), bnorm):
            return x
        z = precond(r)
        rho_new = float(np.vdot(r, z))
        p = z + (rho_new / rho) * p
        rho = rho_new


@_restarting
def fcg(grid, a, x, r, precond, params, bnorm, info):
    """Flexible conjugate gradients with one stored direction (Notay's FCG(1)):
    p_k = z_k - ((z_k, q_{k-1}) / (p_{k-1}, q_{k-1})) p_{k-1}, q = A p,
    alpha_k = (p_k, r_k) / (p_k, q_k)."""
    p_prev = q_prev = None
    pq_prev = 0.0
    while True:
        z = precond(r)
        p = z if p_prev is None else z - (float(np.vdot(z, q_prev)) / pq_prev) * p_prev
        q = apply_operator(grid, a, p)
        pq = float(np.vdot(p, q))
        alpha = float(np.vdot(p, r)) / pq
        x = x + alpha * p
        r = r - alpha * q
        if _stop(info, params, float(np.linalg.norm(r)), bnorm):
            return x
        p_prev, q_prev, pq_prev = p, q, pq


@_restarting
def cgs(grid, a, x, r, precond, params, bnorm, info):
    """Conjugate gradient squared (Saad, Algorithm 7.6), right-preconditioned:
    the search directions p and u + q are preconditioned before A acts."""
    rt = r.copy()
    rho_old = 1.0
    u = q = p = np.zeros(grid.shape)
    first = True
    while True:
        rho = float(np.vdot(rt, r))
        beta = 0.0 if first else rho / rho_old
        u = r + beta * q
        p = u + beta * (q + beta * p)
        first = False
        ph = precond(p)
        vh = apply_operator(grid, a, ph)
        alpha = rho / float(np.vdot(rt, vh))
        q = u - alpha * vh
        uh = precond(u + q)
        x = x + alpha * uh
        r = r - alpha * apply_operator(grid, a, uh)
        rho_old = rho
        if _stop(info, params, float(np.linalg.norm(r)), bnorm):
            return x


@_restarting
def bicgstab(grid, a, x, r, precond, params, bnorm, info):
    """BiCGSTAB (Saad, Algorithm 7.7), right-preconditioned."""
    rt = r.copy()
    p = r.copy()
    rho = float(np.vdot(rt, r))
    while True:
        ph = precond(p)
        v = apply_operator(grid, a, ph)
        alpha = rho / float(np.vdot(rt, v))
        s = r - alpha * v
        sh = precond(s)
        t = apply_operator(grid, a, sh)
        tt = float(np.vdot(t, t))
        omega = float(np.vdot(t, s)) / tt if tt > 0.0 else 0.0
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        if _stop(info, params, float(np.linalg.norm(r)), bnorm):
            return x
        rho_new = float(np.vdot(rt, r))
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        rho = rho_new


def krylov(method: str, grid: Grid, a: np.ndarray, b: np.ndarray, x0, precond, params: OracleParams):
    """Dispatch to one of the methods of the paper's comparison."""
    fn = {"fgmres": fgmres, "gmres": gmres, "cg": cg, "fcg": fcg, "cgs": cgs, "bicgstab": bicgstab}[method]
    return fn(grid, a, b, x0, precond, params)


def solve(params: OracleParams, a: np.ndarray, f: np.ndarray, phi0: np.ndarray | None = None,
          homogeneous: bool = False, hierarchy: Hierarchy | None = None, method: str = "fgmres"):
    """phi solving -div(a grad phi) = f with the plate data of ``params``
    (or zero plate data if ``homogeneous``), by GMG-preconditioned FGMRES."""
    nz, ny, nx = a.shape
    grid = Grid(nx, ny, nz, params.lx, params.ly, params.lz)
    hier = hierarchy if hierarchy is not None else build_hierarchy(grid, a, params)
    if homogeneous:
        b = np.array(f, dtype=np.float64, copy=True)
    else:
        b = assemble_rhs(grid, a, f, params.phi_bottom, params.phi_top)
    cycle = params.cycle
    if cycle == "auto":   # Sec. 3.2: FMG when there is no previous potential, V-cycles after
        cycle = "fmg" if phi0 is None or not np.any(phi0) else "v"
    precond = (lambda v: fmg(hier, v)) if cycle == "fmg" else (lambda v: vcycle(hier, v))
    phi, info = krylov(method, grid, a, b, phi0, precond, params)
    return phi, info, hier


# ---------------------------------------------------------------------------
# Coefficient and right-hand side of the elliptic step from the densities
# ---------------------------------------------------------------------------

ELEMENTARY_CHARGE = 1.602176634e-19          # C (exact in the SI)
VACUUM_PERMITTIVITY_CM = 8.8541878128e-14   # F/cm (CODATA 2018)


def neumann_second_difference(u: np.ndarray, axis: int) -> np.ndarray:
    """delta^2 u = u_{i+1} - 2 u_i + u_{i-1} along ``axis`` with the
    homogeneous Neumann condition of the densities (ghost = interior cell),
    Sec. 2.2."""
    u = np.moveaxis(u, axis, 0)
    ext = np.concatenate([u[:1], u, u[-1:]], axis=0)
    return np.moveaxis(ext[2:] - 2.0 * u + ext[:-2], 0, axis)


def assemble_coefficient_rhs(grid: Grid, n_e: np.ndarray, n_p: np.ndarray, tau: float, mu_e: float,
                             mu_p: float, diffusion: tuple, e_over_eps0: float):
    """a and f of the elliptic equation eq. (semi2) in its discrete form
    eq. (e18), divided through by eps0/e so that a = 1 in vacuum:

        P = eps0/e + (tau/2)(mu_p n_p + mu_e n_e),   a = (e/eps0) P,
        f = (e/eps0) [n_p - n_e - (tau/2) sum_alpha D_alpha delta_alpha^2 n_e / h_alpha^2].

    The mobility enters with its magnitude (R11: the sign of mu_e differs
    between Sec. 2 and Sec. 5.2)."""
    a = 1.0 + e_over_eps0 * 0.5 * tau * (abs(mu_p) * n_p + abs(mu_e) * n_e)
    dx, dy, dz = diffusion
    lap = (dx / grid.hx ** 2 * neumann_second_difference(n_e, 2)
           + dy / grid.hy ** 2 * neumann_second_difference(n_e, 1)
           + dz / grid.hz ** 2 * neumann_second_difference(n_e, 0))
    f = e_over_eps0 * (n_p - n_e - 0.5 * tau * lap)
    return a, f


# ---------------------------------------------------------------------------
# The semi-implicit time step around the solve (eqs. (e1)-(e2), Sec. 2.1) with
# the finite-volume transport of Sec. 2.2 (MUSCL with the Koren limiter)
# ---------------------------------------------------------------------------

PRESSURE_TORR = 760.0
IONIZATION_A = 5.7      # alpha(|E|) = A P exp(-B P / |E|) cm^-1, Sec. 5.2
IONIZATION_B = 260.0


def ionization_coefficient(e_abs: np.ndarray, pressure: float = PRESSURE_TORR) -> np.ndarray:
    """alpha(|E|) = 5.7 P exp(-260 P / |E|) cm^-1 (|E| in V/cm, P in Torr), Sec. 5.2; 0 where |E| = 0."""
    e_abs = np.asarray(e_abs, dtype=np.float64)
    out = np.zeros_like(e_abs)
    nz = e_abs > 0
    out[nz] = IONIZATION_A * pressure * np.exp(-IONIZATION_B * pressure / e_abs[nz])
    return out


def koren_slope(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Limited slope phi(r) b of the Koren limiter phi(r) = max(0, min(2r, (1+2r)/3, 2)),
    r = a / b (a: the downwind difference, b: the upwind one), written without
    the division: 0 if a b <= 0, else sign(b) min(2|a|, (|b| + 2|a|)/3, 2|b|)."""
    aa, ab = np.abs(a), np.abs(b)
    s = np.sign(b) * np.minimum(np.minimum(2.0 * aa, (ab + 2.0 * aa) / 3.0), 2.0 * ab)
    return np.where(a * b > 0.0, s, 0.0)


def face_fields(grid: Grid, phi: np.ndarray, g_bottom: float, g_top: float):
    """Face-normal fields E_f = -(phi_q - phi_p)/h on every face of every axis,
    boundary faces included (arrays one longer than the grid along the axis):
    zero on the side walls (mirror ghosts), -2 (phi_0 - g)/hz-type values on
    the plates (ghost 2 g - phi)."""
    out = []
    for axis, h in ((2, grid.hx), (1, grid.hy), (0, grid.hz)):
        u = np.moveaxis(phi, axis, 0)
        if axis == 0:
            lo, hi = 2.0 * g_bottom - u[:1], 2.0 * g_top - u[-1:]
        else:
            lo, hi = u[:1], u[-1:]
        ext = np.concatenate([lo, u, hi], axis=0)
        out.append(np.moveaxis(-(ext[1:] - ext[:-1]) / h, 0, axis))
    return out   # (E_x faces, E_y faces, E_z faces)


def _drift_divergence(n: np.ndarray, velocity_faces, grid: Grid) -> np.ndarray:
    """div(v n) by the finite-volume MUSCL scheme: on each face the upwind
    cell's value extrapolated with the Koren-limited slope, times the face
    velocity; densities take homogeneous Neumann ghosts (two layers)."""
    div = np.zeros_like(n)
    for (axis, h), v in zip(((2, grid.hx), (1, grid.hy), (0, grid.hz)), velocity_faces):
        u = np.moveaxis(n, axis, 0)
        vv = np.moveaxis(v, axis, 0)
        m = u.shape[0]
        ext = np.concatenate([u[1:2] if m > 1 else u[:1], u[:1], u, u[-1:], u[-2:-1] if m > 1 else u[-1:]], axis=0)
        # face k between cells k-1 and k (k = 0..m), padded index of cell i is i + 2
        left = ext[1:m + 2] + 0.5 * koren_slope(ext[2:m + 3] - ext[1:m + 2], ext[1:m + 2] - ext[0:m + 1])
        right = ext[2:m + 3] + 0.5 * koren_slope(ext[1:m + 2] - ext[2:m + 3], ext[2:m + 3] - ext[3:m + 4])
        flux = np.where(vv > 0.0, vv * left, vv * right)
        div += np.moveaxis((flux[1:] - flux[:-1]) / h, 0, axis)
    return div


def transport_rhs(grid: Grid, n_e: np.ndarray, n_p: np.ndarray, phi: np.ndarray, g_bottom: float, g_top: float,
                  mu_e: float, mu_p: float, diffusion: tuple):
    """Right-hand sides of the transport equations of eq. (eM) for the field
    E = -grad(phi):  dn_e/dt = div(mu_e E n_e) + div(D_e grad n_e) + S,
    dn_p/dt = -div(mu_p E n_p) + S,  S = alpha(|E|) mu_e |E| n_e, with |E| at
    the cell centres from the central differences of Sec. 2.2 (R19)."""
    ef = face_fields(grid, phi, g_bottom, g_top)
    ve = [-abs(mu_e) * e for e in ef]              # electrons drift against E
    vp = [abs(mu_p) * e for e in ef]
    ex, ey, ez = field_from_potential(grid, phi, g_bottom, g_top)
    eabs = np.sqrt(ex * ex + ey * ey + ez * ez)
    src = ionization_coefficient(eabs) * abs(mu_e) * eabs * n_e
    dx, dy, dz = diffusion
    diff = (dx / grid.hx ** 2 * neumann_second_difference(n_e, 2)
            + dy / grid.hy ** 2 * neumann_second_difference(n_e, 1)
            + dz / grid.hz ** 2 * neumann_second_difference(n_e, 0))
    return -_drift_divergence(n_e, ve, grid) + diff + src, -_drift_divergence(n_p, vp, grid) + src


def transport_stage(grid, base_e, base_p, eval_e, eval_p, phi, g_bottom, g_top, mu_e, mu_p, diffusion, c):
    """One explicit stage: base + c * (transport right-hand side at eval)."""
    re, rp = transport_rhs(grid, eval_e, eval_p, phi, g_bottom, g_top, mu_e, mu_p, diffusion)
    return base_e + c * re, base_p + c * rp


def semi_implicit_step(params: OracleParams, n_e: np.ndarray, n_p: np.ndarray, tau: float, mu_e: float,
                       mu_p: float, diffusion: tuple, e_over_eps0: float, phi_prev: np.ndarray | None = None):
    """The second-order semi-implicit step, eqs. (e1)-(e2): the elliptic
    equation eq. (semi2) gives phi^{n+1/2} (assembled from n^n); the predictor
    n^{n+1/2} = n^n + (tau/2) R(n^n) and the corrector n^{n+1} = n^n +
    tau R(n^{n+1/2}) both use E^{n+1/2}."""
    nz, ny, nx = n_e.shape
    grid = Grid(nx, ny, nz, params.lx, params.ly, params.lz)
    a, f = assemble_coefficient_rhs(grid, n_e, n_p, tau, mu_e, mu_p, diffusion, e_over_eps0)
    phi, info, _ = solve(params, a, f, phi0=phi_prev)
    args = (phi, params.phi_bottom, params.phi_top, mu_e, mu_p, diffusion)
    he, hp = transport_stage(grid, n_e, n_p, n_e, n_p, *args, 0.5 * tau)
    ne1, np1 = transport_stage(grid, n_e, n_p, he, hp, *args, tau)
    return ne1, np1, phi, info


# ---------------------------------------------------------------------------
# Field and adjoint
# ---------------------------------------------------------------------------


def field_from_potential(grid: Grid, phi: np.ndarray, g_bottom: float, g_top: float):
    """E = -grad(phi) by cell-centred central differences (Sec. 2.2), with the
    ghost values of the boundary conditions: mirror (Neumann) on x/y walls and
    2g - phi (R2) on the plates."""
    def central(u, axis, h, ghost_lo, ghost_hi):
        u = np.moveaxis(u, axis, 0)
        ext = np.concatenate([ghost_lo(u[:1]), u, ghost_hi(u[-1:])], axis=0)
        return np.moveaxis(-(ext[2:] - ext[:-2]) / (2.0 * h), 0, axis)

    mirror = lambda edge: edge                       # noqa: E731
    ex = central(phi, 2, grid.hx, mirror, mirror)
    ey = central(phi, 1, grid.hy, mirror, mirror)
    ez = central(phi, 0, grid.hz, lambda e: 2.0 * g_bottom - e, lambda e: 2.0 * g_top - e)
    return ex, ey, ez


def field_at(grid: Grid, phi: np.ndarray, g_bottom: float, g_top: float, cells) -> np.ndarray:
    """(Ex, Ey, Ez) of field_from_potential at the listed cells (k, j, i) only,
    one cell at a time: central differences with a mirror ghost beyond a side
    wall and 2g - phi beyond a plate (Sec. 2.2, R2).  Returns shape (len, 3)."""
    nz, ny, nx = phi.shape
    out = np.empty((len(cells), 3))
    for n, (k, j, i) in enumerate(cells):
        c = float(phi[k, j, i])
        xm = float(phi[k, j, i - 1]) if i > 0 else c
        xp = float(phi[k, j, i + 1]) if i < nx - 1 else c
        ym = float(phi[k, j - 1, i]) if j > 0 else c
        yp = float(phi[k, j + 1, i]) if j < ny - 1 else c
        zm = float(phi[k - 1, j, i]) if k > 0 else 2.0 * g_bottom - c
        zp = float(phi[k + 1, j, i]) if k < nz - 1 else 2.0 * g_top - c
        out[n] = (-(xp - xm) / (2.0 * grid.hx), -(yp - ym) / (2.0 * grid.hy), -(zp - zm) / (2.0 * grid.hz))
    return out


def adjoint_coefficient_grad(grid: Grid, phi: np.ndarray, lam: np.ndarray,
                             g_bottom: float, g_top: float) -> np.ndarray:
    """dL/da for L(phi), phi = A(a)^{-1} b(a, f), given lambda = A^{-1} dL/dphi.

    dL/da_p = lambda^T (d b/d a_p - (d A/d a_p) phi).  With a_f = (a_p+a_q)/2
    on interior faces and a_f = a_p on plate faces (eq. (e18), R1, R2):
      dL/da_p = -1/2 sum_{interior f=(p,q)} (lam_p - lam_q)(phi_p - phi_q)/h_f^2
                - sum_{plate faces of p} 2 lam_p (phi_p - g)/hz^2.
    Not in the paper: the derivative of its discrete operator.
    """
    g = np.zeros(grid.shape)
    for axis, h in ((2, grid.hx), (1, grid.hy), (0, grid.hz)):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[axis] = slice(0, -1)
        hi[axis] = slice(1, None)
        lo, hi = tuple(lo), tuple(hi)
        t = 0.5 * (lam[lo] - lam[hi]) * (phi[lo] - phi[hi]) / h**2
        g[lo] -= t
        g[hi] -= t
    g[0] -= 2.0 * lam[0] * (phi[0] - g_bottom) / grid.hz**2
    g[-1] -= 2.0 * lam[-1] * (phi[-1] - g_top) / grid.hz**2
    return g

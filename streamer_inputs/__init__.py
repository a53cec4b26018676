"""Seeded synthetic inputs shaped like the paper's streamer workloads.

This module only *generates inputs* (coefficient ``a``, source ``f``, loss
weights ``w``); it holds none of the solver's arithmetic, so both the CPU oracle
and the CUDA path may import it without sharing any part of the method.

Shapes follow the paper's streamer geometry: a unit-cube domain with the plates
at z = 0 and z = 1 (Sec. 5.2), a Gaussian streamer channel (the initial density
of eq. (51), Sec. 5.2) and two interacting channels (Sec. 6.2).  In the
semi-implicit scheme the elliptic coefficient grows with the electron density
(the coefficient ``P`` of Sec. 2.2, eq. (e18)), so ``a = 1 + kappa * n`` with
``n`` a normalised channel profile; ``kappa`` sets the coefficient contrast.

All arrays are float64, C-contiguous, shaped ``(nz, ny, nx)`` with x fastest,
and sampled at the cell centres ``((i+1/2)hx, (j+1/2)hy, (k+1/2)hz)``.

Workloads (seed = 20181220 + workload index):

* ``const32``      : 32^3, a = 1, two opposite Gaussian heads + U(-1,1) noise.
* ``channel128``   : 128^3, one channel, kappa = 1e3, same source.
* ``channel256``   : 256^3, one channel, kappa in {1e1, 1e3, 1e4}.
* ``twochannel512``: 512^3, two channels at x = 0.4, 0.6, sigma_r = 0.03,
                     kappa = 1e4, four seeded-sign heads + noise.
* ``adjoint``      : the ``channel128`` problem plus a smoothed N(0,1) loss
                     weight field ``w`` (3-cell box filter, replicated edges).

Every generator accepts an explicit ``n`` so tests can build the same shapes at
small sizes.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20181220

# Workload index -> default grid size (cells per side).
WORKLOADS = {
    "const32": (1, 32),
    "channel128": (2, 128),
    "channel256": (3, 256),
    "twochannel512": (4, 512),
    "adjoint": (5, 128),
}

HEAD_WIDTH = 0.05        # Gaussian charge-head width
HEAD_AMPLITUDE = 1.0e3   # Gaussian charge-head amplitude
CHANNEL_SIGMA = 0.03     # channel radius (two-streamer case of Sec. 6.2 uses 0.03)
WINDOW_LO, WINDOW_HI, WINDOW_EDGE = 0.3, 0.7, 0.02


def cell_centres(n: int, length: float = 1.0) -> np.ndarray:
    """Cell-centre coordinates of ``n`` uniform cells on ``[0, length]``."""
    h = length / n
    return (np.arange(n, dtype=np.float64) + 0.5) * h


def _grid(shape):
    nz, ny, nx = shape
    return cell_centres(nx), cell_centres(ny), cell_centres(nz)


def z_window(z: np.ndarray) -> np.ndarray:
    """Smooth window equal to 1 on 0.3 < z < 0.7 with tanh edges of width 0.02."""
    return 0.5 * (np.tanh((z - WINDOW_LO) / WINDOW_EDGE) - np.tanh((z - WINDOW_HI) / WINDOW_EDGE))


def channel_profile(shape, axes=((0.5, 0.5),), sigma=CHANNEL_SIGMA) -> np.ndarray:
    """Sum of Gaussian channel profiles exp(-r^2/sigma^2) times the z window."""
    x, y, z = _grid(shape)
    xy = np.zeros((shape[1], shape[2]))
    for (cx, cy) in axes:
        xy += np.exp(-((y[:, None] - cy) ** 2) / sigma**2) * np.exp(-((x[None, :] - cx) ** 2) / sigma**2)
    return z_window(z)[:, None, None] * xy[None, :, :]


def gaussian_head(shape, centre, width=HEAD_WIDTH) -> np.ndarray:
    """exp(-|x - centre|^2 / width^2) on the cell centres (separable product)."""
    x, y, z = _grid(shape)
    cx, cy, cz = centre
    gx = np.exp(-((x - cx) ** 2) / width**2)
    gy = np.exp(-((y - cy) ** 2) / width**2)
    gz = np.exp(-((z - cz) ** 2) / width**2)
    return gz[:, None, None] * gy[None, :, None] * gx[None, None, :]


# Double-headed streamer of the paper's tests (eq. (51), Sec. 5.2): densities in
# cm^-3 on a cm domain, the channel axis at x = y = 1 (on the unit cube: the
# corner, a symmetric quarter of the streamer between zero-flux walls).
STREAMER_SIGMA_Z = 0.027
STREAMER_SIGMA_R = 0.021
STREAMER_BACKGROUND = 1.0e8
STREAMER_PEAK = 1.0e14
# Sec. 5.2 constants at 760 Torr (cm^2/(V s), cm^2/s, V)
MU_E = 2.9e5 / 760.0
MU_P = 2.6e3 / 760.0
DIFFUSION = (2190.0, 2190.0, 1800.0)
PHI0 = 52.0e3


def streamer_densities(shape, step: int = 0, drift: float = 0.01, ion_growth: float = 0.05, xp=np, device=None):
    """(n_e, n_p) for step ``step`` of a synthetic time-step sequence: the
    eq. (51) profile with its centre at z = 0.5 + drift * step, and the ion
    density scaled by (1 + ion_growth * step) (a stand-in for the charge
    separation the transport would produce).  ``xp`` is numpy (default) or
    torch (then the arrays are built on ``device``); both evaluate the same
    separable product."""
    x, y, z = _grid(shape)
    gz = np.exp(-(((z - (0.5 + drift * step)) / STREAMER_SIGMA_Z) ** 2))
    gy = np.exp(-((y - 1.0) ** 2) / STREAMER_SIGMA_R ** 2)
    gx = np.exp(-((x - 1.0) ** 2) / STREAMER_SIGMA_R ** 2)
    if xp is np:
        prof = gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    else:
        t = lambda v: xp.from_numpy(v).to(device)   # noqa: E731
        prof = t(gz)[:, None, None] * t(gy)[None, :, None] * t(gx)[None, None, :]
    ne = STREAMER_BACKGROUND + STREAMER_PEAK * prof
    return ne, ne * (1.0 + ion_growth * step)


def _noise(rng, shape):
    return rng.uniform(-1.0, 1.0, size=shape)


def make_inputs(workload: str, n: int | None = None, kappa: float | None = None,
                shape: tuple | None = None) -> dict:
    """Build one seeded workload.

    Returns a dict with ``a``, ``f`` (float64 ``(nz,ny,nx)``), ``phi_bottom``,
    ``phi_top``, ``kappa``, ``seed`` and, for ``adjoint``, the loss weights ``w``.
    ``shape`` overrides ``n`` for anisotropic tests.
    """
    index, n_default = WORKLOADS[workload]
    if shape is None:
        n = n_default if n is None else int(n)
        shape = (n, n, n)
    shape = tuple(int(s) for s in shape)
    seed = BASE_SEED + index
    rng = np.random.default_rng(seed)
    out = {"workload": workload, "shape": shape, "seed": seed, "phi_bottom": 0.0, "phi_top": 1.0}

    if workload == "twochannel512":
        kappa = 1.0e4 if kappa is None else float(kappa)
        axes = ((0.4, 0.5), (0.6, 0.5))
        n_e = channel_profile(shape, axes=axes)
        signs = rng.choice(np.array([-1.0, 1.0]), size=4)
        f = np.zeros(shape)
        s = 0
        for (cx, cy) in axes:
            for cz in (0.3, 0.7):
                f += signs[s] * HEAD_AMPLITUDE * gaussian_head(shape, (cx, cy, cz))
                s += 1
        f += _noise(rng, shape)
        out["head_signs"] = signs
    else:
        if workload == "const32":
            kappa = 0.0
            n_e = np.zeros(shape)
        else:
            kappa = 1.0e3 if kappa is None else float(kappa)
            n_e = channel_profile(shape)
        f = HEAD_AMPLITUDE * (gaussian_head(shape, (0.5, 0.5, 0.4)) - gaussian_head(shape, (0.5, 0.5, 0.6)))
        f += _noise(rng, shape)

    a = 1.0 + kappa * n_e
    out["a"] = np.ascontiguousarray(a, dtype=np.float64)
    out["f"] = np.ascontiguousarray(f, dtype=np.float64)
    out["kappa"] = kappa
    if workload == "adjoint":
        out["w"] = smoothed_normal(rng, shape)
    return out


def smoothed_normal(rng, shape) -> np.ndarray:
    """Standard-normal field smoothed by a 3-cell box filter per axis (edges replicated)."""
    g = rng.standard_normal(size=shape)
    for axis in range(3):
        p = np.pad(g, [(1, 1) if ax == axis else (0, 0) for ax in range(3)], mode="edge")
        sl = [slice(None)] * 3
        acc = np.zeros(shape)
        for off in range(3):
            sl[axis] = slice(off, off + shape[axis])
            acc += p[tuple(sl)]
        g = acc / 3.0
    return np.ascontiguousarray(g)


def random_field(seed: int, shape, lo=-1.0, hi=1.0) -> np.ndarray:
    """Plain seeded uniform field, used for operator-level parity inputs."""
    return np.random.default_rng(seed).uniform(lo, hi, size=tuple(shape))


def random_coefficient(seed: int, shape, contrast=10.0) -> np.ndarray:
    """Seeded positive coefficient with values in [1, 1 + contrast] (log-uniform)."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(0.0, np.log1p(contrast), size=tuple(shape)))

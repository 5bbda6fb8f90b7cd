"""Seeded synthetic inputs shaped like the paper's experiments (Section 5).

This module holds only the random-number generator and the painting of the
coefficient, source and initial fields.  It contains none of the method's
arithmetic, so both the CUDA path and the FP64 oracle may take their inputs
from it.

The paper's fields exist only as figure images (Section 5, Figs. 2-13), so the
generators below stand in for them: a unit square, background kappa = 1 with
straight high-conductivity channels and square inclusions (high contrast),
smooth Gaussian sources, and Gaussian-bump initial data.

Random stream: splitmix64 (Steele, Lea, Flood 2014), uniforms from the top
53 bits.  Seed = 241109244 + 1000 * config_index + instance.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

_MASK = (1 << 64) - 1
SEED_BASE = 241109244


class SplitMix64:
    """splitmix64 stream; uniform() returns k * 2**-53, k the top 53 bits."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] inclusive."""
        return lo + min(int(self.uniform() * (hi - lo + 1)), hi - lo)


@dataclass
class Problem:
    """One instance: grid, multiscale-space parameters, time grid and fields.

    n_f   fine cells per side (h = 1/n_f); nodes (n_f+1)^2, x fastest
    nc    coarse blocks per side (H = 1/nc); n_f % nc == 0
    J     auxiliary modes per block taken for V_H1 (J+1 smallest eigenpairs)
    ell   oversampling layers of the CEM windows K_i^+
    N, P  coarse intervals and fine steps per interval
    T     final time (None: choose a stable T from the spaces)
    alpha WR periodic-like parameter
    kappa cell coefficient [n_f, n_f] (row = y, col = x)
    f     nodal source shape [(n_f+1)^2]; amp[n] multiplies it on interval n
    u0    nodal initial condition [(n_f+1)^2] (zero on the boundary)
    """
    name: str
    n_f: int
    nc: int
    J: int
    ell: int
    N: int
    P: int
    alpha: float
    eps: float
    T: float | None
    kappa: np.ndarray = field(repr=False)
    f: np.ndarray = field(repr=False)
    u0: np.ndarray = field(repr=False)
    amp: np.ndarray = field(repr=False)
    meta: dict = field(default_factory=dict)

    def describe(self) -> dict:
        d = {k: v for k, v in asdict(self).items() if k not in ("kappa", "f", "u0", "amp")}
        return d


def _node_xy(n_f: int):
    x = np.arange(n_f + 1) / n_f
    X, Y = np.meshgrid(x, x)          # Y[j, i] = y_j, X[j, i] = x_i
    return X.ravel(), Y.ravel()


def paint_kappa(rng: SplitMix64, n_f: int, n_channels: int, ch_value: float, ch_width: int,
                n_incl: int = 0, incl_value: float = 0.0, incl_side=(2, 4),
                margin: int | None = None) -> np.ndarray:
    """Background 1; axis-aligned channels (orientation a fair coin, length
    U[0.5,1]*(n_f - 2 margin) cells, width ch_width cells, placed uniformly on
    the cell lattice) and square inclusions (side uniform in incl_side cells).
    Overlaps take the maximum.  Every feature keeps `margin` cells (default
    max(1, n_f // 32)) away from the boundary: a high-conductivity feature
    touching the Dirichlet boundary forces the fracture-average basis to drop
    to zero inside it, and the energy of V_H2 then grows with the contrast."""
    m = max(1, n_f // 32) if margin is None else margin
    span = n_f - 2 * m
    k = np.ones((n_f, n_f))
    for _ in range(n_channels):
        horizontal = rng.uniform() < 0.5
        length = max(1, int(math.floor(rng.uniform(0.5, 1.0) * span)))
        a0 = m + rng.randint(0, span - length)
        b0 = m + rng.randint(0, span - ch_width)
        if horizontal:
            sl = (slice(b0, b0 + ch_width), slice(a0, a0 + length))
        else:
            sl = (slice(a0, a0 + length), slice(b0, b0 + ch_width))
        k[sl] = np.maximum(k[sl], ch_value)
    for _ in range(n_incl):
        s = rng.randint(incl_side[0], incl_side[1])
        x0 = m + rng.randint(0, span - s)
        y0 = m + rng.randint(0, span - s)
        k[y0:y0 + s, x0:x0 + s] = np.maximum(k[y0:y0 + s, x0:x0 + s], incl_value)
    return close_gaps(k)


def close_gaps(k: np.ndarray) -> np.ndarray:
    """Fill background cells lying between two high-conductivity cells (left
    and right, or below and above) with the larger neighbour, until none is
    left.  A background strip one cell wide between two channels has every
    Q1 node on a channel, so the fine grid cannot represent a background
    function that vanishes on the channels beside it."""
    k = k.copy()
    bg = k.min()
    while True:
        hi = k > bg
        lr = np.zeros_like(hi)
        ud = np.zeros_like(hi)
        lr[:, 1:-1] = hi[:, :-2] & hi[:, 2:]
        ud[1:-1, :] = hi[:-2, :] & hi[2:, :]
        fill = (~hi) & (lr | ud)
        if not fill.any():
            return k
        nb = np.zeros_like(k)
        nb[:, 1:-1] = np.maximum(nb[:, 1:-1], np.where(lr[:, 1:-1], np.maximum(k[:, :-2], k[:, 2:]), 0))
        nb[1:-1, :] = np.maximum(nb[1:-1, :], np.where(ud[1:-1, :], np.maximum(k[:-2, :], k[2:, :]), 0))
        k[fill] = nb[fill]


def gaussian_sum(rng: SplitMix64, n_f: int, count: int, centre=(0.1, 0.9), sigma=(0.03, 0.1),
                 amp=(0.5, 1.0)) -> np.ndarray:
    X, Y = _node_xy(n_f)
    g = np.zeros_like(X)
    for _ in range(count):
        cx, cy = rng.uniform(*centre), rng.uniform(*centre)
        s = rng.uniform(*sigma)
        a = rng.uniform(*amp)
        g += a * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * s * s))
    return g


def zero_boundary(v: np.ndarray, n_f: int) -> np.ndarray:
    g = v.reshape(n_f + 1, n_f + 1).copy()
    g[0, :] = g[-1, :] = 0.0
    g[:, 0] = g[:, -1] = 0.0
    return g.ravel()


def config_c1(instance: int = 0) -> Problem:
    """64x64 fine, 8x8 coarse, J = 2, two oversampling layers; 8 channels of
    width 2 cells, value 1e4; f = 1, u0 = 0; N = 8 intervals x 16 fine steps."""
    rng = SplitMix64(SEED_BASE + 0 * 1000 + instance)
    n_f = 64
    kappa = paint_kappa(rng, n_f, 8, 1e4, 2)
    nn = (n_f + 1) ** 2
    return Problem("channels_64x64", n_f, 8, 2, 2, 8, 16, 0.1, 1e-10, None, kappa,
                   np.ones(nn), np.zeros(nn), np.ones(8), {"contrast": 1e4})


def config_c2(instance: int = 0) -> Problem:
    """256x256 fine, 16x16 coarse, J = 4, four layers; 40 channels and 60
    square inclusions of value 1e6; f = sum of 10 Gaussians; u0 = 0;
    N = 64 intervals x 64 fine steps."""
    rng = SplitMix64(SEED_BASE + 1 * 1000 + instance)
    n_f = 256
    kappa = paint_kappa(rng, n_f, 40, 1e6, 2, n_incl=60, incl_value=1e6)
    f = gaussian_sum(rng, n_f, 10)
    nn = (n_f + 1) ** 2
    return Problem("channels_inclusions_256x256", n_f, 16, 4, 4, 64, 64, 0.1, 1e-10, None, kappa,
                   f, np.zeros(nn), np.ones(64), {"contrast": 1e6})


def config_c3(instance: int = 0) -> Problem:
    """128x128 fine, 16x16 coarse, J = 3, two layers; 30 channels of value
    1e5; u0 = 20 Gaussian bumps (amplitude U[-1,1]); source = one Gaussian
    at the centre times 16 amplitudes U[0.5,1.5], each held over two of the
    N = 32 intervals; P = 32."""
    rng = SplitMix64(SEED_BASE + 2 * 1000 + instance)
    n_f = 128
    kappa = paint_kappa(rng, n_f, 30, 1e5, 2)
    u0 = zero_boundary(gaussian_sum(rng, n_f, 20, centre=(0.1, 0.9), sigma=(0.02, 0.08),
                                    amp=(-1.0, 1.0)), n_f)
    X, Y = _node_xy(n_f)
    f = np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / (2 * 0.1 ** 2))
    a16 = np.array([rng.uniform(0.5, 1.5) for _ in range(16)])
    amp = np.repeat(a16, 2)
    return Problem("observed_128x128", n_f, 16, 3, 2, 32, 32, 0.1, 1e-10, None, kappa,
                   f, u0, amp, {"contrast": 1e5, "amp16": a16})


def config_c4(instance: int = 0, sizes=(64, 96, 128, 192, 256)) -> Problem:
    """One instance of the many-instance workload: fine grid drawn uniformly
    from `sizes`, coarse blocks of 8 fine cells, J in {2, 3, 4}, contrast
    10^U(3, 6), channel and inclusion counts in {5..50}, N in {16, 32, 64},
    P = 32, two oversampling layers; f = sum of 10 Gaussians, u0 = 0.
    The jump tolerance is relative (eps = -1e-10: 1e-10 of the largest
    G-sweep state): the stable final times of these instances span 1e-7 to
    1e-2, and so do their solutions' magnitudes."""
    rng = SplitMix64(SEED_BASE + 3 * 1000 + instance)
    n_f = sizes[rng.randint(0, len(sizes) - 1)]
    J = rng.randint(2, 4)
    contrast = 10.0 ** rng.uniform(3.0, 6.0)
    n_ch = rng.randint(5, 50)
    n_in = rng.randint(5, 50)
    N = (16, 32, 64)[rng.randint(0, 2)]
    kappa = paint_kappa(rng, n_f, n_ch, contrast, 2, n_incl=n_in, incl_value=contrast)
    f = gaussian_sum(rng, n_f, 10)
    nn = (n_f + 1) ** 2
    return Problem(f"batch_{instance}_{n_f}x{n_f}", n_f, n_f // 8, J, 2, N, 32, 0.1, -1e-10, None, kappa, f,
                   np.zeros(nn), np.ones(N), {"contrast": contrast, "channels": n_ch, "inclusions": n_in})


def config_c5(instance: int = 0) -> Problem:
    """1024x1024 fine, 32x32 coarse, J = 4, four layers; 200 channels and
    400 inclusions of value 1e6; f as in the 256x256 case; N = 256 x P = 32."""
    rng = SplitMix64(SEED_BASE + 4 * 1000 + instance)
    n_f = 1024
    kappa = paint_kappa(rng, n_f, 200, 1e6, 2, n_incl=400, incl_value=1e6)
    f = gaussian_sum(rng, n_f, 10)
    nn = (n_f + 1) ** 2
    return Problem("channels_inclusions_1024x1024", n_f, 32, 4, 4, 256, 32, 0.1, 1e-10, None, kappa,
                   f, np.zeros(nn), np.ones(256), {"contrast": 1e6})


def config_paper_grid(N: int = 20, P: int = 30, instance: int = 0) -> Problem:
    """The grid of the paper's experiments (Section 5): h = 1/100, H = 1/10
    (100x100 fine cells, 10x10 coarse blocks), J = 2, two oversampling
    layers; 20 channels of width 2 cells and value 1e4 (the first
    experiment's contrast); f = 1, u0 = 0; N intervals x P fine steps
    (the first experiment: N = 20, P = 30, N P = 600)."""
    rng = SplitMix64(SEED_BASE + 6 * 1000 + instance)
    n_f = 100
    kappa = paint_kappa(rng, n_f, 20, 1e4, 2)
    nn = (n_f + 1) ** 2
    return Problem("channels_100x100", n_f, 10, 2, 2, N, P, 0.1, 1e-10, None, kappa, np.ones(nn),
                   np.zeros(nn), np.ones(N), {"contrast": 1e4})


def config_small(n_f=16, nc=4, J=2, ell=1, N=4, P=8, seed=7, contrast=1e3, channels=2,
                 u0_kind="bumps", f_kind="ones", alpha=0.1) -> Problem:
    """Small instance for fast tests (several tiles, ragged sizes)."""
    rng = SplitMix64(SEED_BASE + 9000 + seed)
    kappa = paint_kappa(rng, n_f, channels, contrast, max(1, n_f // 32))
    nn = (n_f + 1) ** 2
    if u0_kind == "bumps":
        u0 = zero_boundary(gaussian_sum(rng, n_f, 3, sigma=(0.1, 0.2), amp=(-1, 1)), n_f)
    elif u0_kind == "sin":
        X, Y = _node_xy(n_f)
        u0 = zero_boundary(np.sin(np.pi * X) * np.sin(np.pi * Y), n_f)
    else:
        u0 = np.zeros(nn)
    if f_kind == "ones":
        f = np.ones(nn)
    elif f_kind == "gauss":
        f = gaussian_sum(rng, n_f, 3)
    else:
        f = np.zeros(nn)
    amp = np.array([rng.uniform(0.5, 1.5) for _ in range(N)])
    return Problem(f"small_{n_f}", n_f, nc, J, ell, N, P, alpha, 1e-10, None, kappa, f, u0, amp,
                   {"contrast": contrast})


def observation_nodes(n_f: int, count: int, seed: int) -> np.ndarray:
    """Distinct interior node indices (x fastest) drawn with splitmix64."""
    rng = SplitMix64(SEED_BASE + 5000 + seed)
    chosen = []
    seen = set()
    while len(chosen) < count:
        i = rng.randint(1, n_f - 1)
        j = rng.randint(1, n_f - 1)
        k = j * (n_f + 1) + i
        if k not in seen:
            seen.add(k)
            chosen.append(k)
    return np.array(chosen, dtype=np.int64)


CONFIGS = {"c1": config_c1, "c2": config_c2, "c3": config_c3, "c4": config_c4, "c5": config_c5}

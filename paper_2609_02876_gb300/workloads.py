"""Seeded synthetic ensembles shaped like the paper's workloads.

This module holds only input generation (no solver arithmetic). Both the
oracle tests and the GPU path draw their inputs from it, so the two sides see
bit-identical inputs.

Random numbers come from splitmix64 (Steele, Lea & Flood, OOPSLA 2014), used
as a counter-based generator: draw i of stream s is mix64(seed_s + (i + 1) *
0x9E3779B97F4A7C15), and a uniform double is its top 53 bits times 2^-53.
Normals use the Box-Muller transform. Every ensemble is a pure function of
(config name, n, stream seed).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

PROBLEM_IDS = {"lorenz": 0, "vdp": 1, "robertson": 2, "hires": 3, "linear": 4, "lv_ude": 5, "nrob": 6}


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Draws start..start+count-1 of the splitmix64 stream with the given seed."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, lo=0.0, hi=1.0) -> np.ndarray:
    u = (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def normal(seed: int, count: int) -> np.ndarray:
    m = (count + 1) // 2
    u = (splitmix64(seed, 2 * m) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    u1 = 1.0 - u[:m]  # in (0, 1]
    u2 = u[m:]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    return z[:count]


def _stream(config_index: int, field: int, seed: int = 0) -> int:
    return (seed << 40) ^ (config_index << 32) ^ field


def uniform_saves(t0: float, t1: float, n_save: int) -> np.ndarray:
    """n_save uniform save times in (t0, t1]: t0 + (t1 - t0) j / n_save, j = 1..n_save."""
    j = np.arange(1, n_save + 1, dtype=np.float64)
    s = t0 + (t1 - t0) * j / n_save
    s[-1] = t1
    return s


def log_saves(t0: float, t1: float, n_save: int) -> np.ndarray:
    """n_save log-spaced save times in (t0, t1]."""
    a, b = np.log10(t0), np.log10(t1)
    s = 10.0 ** (a + (b - a) * np.arange(1, n_save + 1) / n_save)
    s[-1] = t1
    return s


HIRES_RATES = np.array([1.71, 0.43, 8.32, 0.0007, 8.75, 10.03, 0.035, 1.12, 1.745, 280.0, 0.69, 1.81])
HIRES_Y0 = np.array([1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0057])
ROBERTSON_RATES = np.array([0.04, 3e7, 1e4])
UDE_HIDDEN = 16
UDE_NW = UDE_HIDDEN * 2 + UDE_HIDDEN + UDE_HIDDEN * UDE_HIDDEN + UDE_HIDDEN + 2 * UDE_HIDDEN + 2


# Output bias of the untrained Robertson neural term: softplus(-9) = 1.2e-4, so the
# term starts at the size of the rate it replaces (k2 y2^2 with y2 ~ 1e-5 .. 3e-5
# and k2 = 3e7 is 1e-3 .. 3e-2 early, falling later), not at softplus(0) = 0.69.
NROB_B3 = -9.0


def glorot_mlp(seed: int = 0) -> np.ndarray:
    """Glorot-uniform 2-16-16-2 weights, zero biases, flat layout
    W1[16][2], b1[16], W2[16][16], b2[16], W3[2][16], b3[2]."""
    H = UDE_HIDDEN
    parts = []
    for li, (fi, fo) in enumerate([(2, H), (H, H), (H, 2)]):
        a = np.sqrt(6.0 / (fi + fo))
        parts.append(uniform(_stream(99, li, seed), fi * fo, -a, a))
        parts.append(np.zeros(fo))
    w = np.concatenate(parts)
    assert w.size == UDE_NW
    return w


NROB_NW = 16 * 3 + 16 + 16 * 16 + 16 + 16 + 1  # 353


def glorot_nrob(seed: int = 0, b3: float = NROB_B3) -> np.ndarray:
    """Glorot-uniform 3-16-16-1 weights of the Robertson neural term, zero hidden
    biases, output bias b3; flat layout W1[16][3], b1[16], W2[16][16], b2[16], W3[16], b3."""
    H = UDE_HIDDEN
    parts = []
    for li, (fi, fo) in enumerate([(3, H), (H, H), (H, 1)]):
        a = np.sqrt(6.0 / (fi + fo))
        parts.append(uniform(_stream(98, li, seed), fi * fo, -a, a))
        parts.append(np.zeros(fo))
    w = np.concatenate(parts)
    w[-1] = b3
    assert w.size == NROB_NW
    return w


def _logu(seed, n, lo=0.9, hi=1.1):
    return np.exp(uniform(seed, n, np.log(lo), np.log(hi)))


def make(name: str, n: int, rtol: float | None = None, seed: int = 0) -> dict:
    """A seeded ensemble. Arrays are per trajectory: params (n, P), y0 (n, d).

    lorenz:      sigma~U[8,12], rho~U[20,30], beta~U[2,3]; y0~N((1,1,1), 0.1^2 I);
                 t in [0, 1]; 10 uniform saves; rtol 1e-6, atol = 1e-2 rtol.
    vdp:         mu~U[0.5,2]; y0~U[-2,2]^2; t in [0, 10]; 50 uniform saves.
    robertson:   k = (0.04, 3e7, 1e4) * logU[0.9,1.1]; y0 = (1,0,0); t in [1e-5, 1e5];
                 20 log-spaced saves; rtol 1e-6, atol 1e-10.
    hires:       12 literal rates * logU[0.9,1.1]; the standard y0; t in [0, 321.8122];
                 10 uniform saves; rtol 1e-6, atol 1e-10.
    lv_ude:      a~U[1,1.5], d~U[2,3]; y0~U[0.5,2]^2; t in [0, 5]; 10 uniform saves;
                 shared Glorot MLP (seed 0); rtol 1e-6, atol 1e-8.
    nrob:        Robertson with the k2 y2^2 term replaced by a shared MLP 3-16-16-1 (tanh,
                 softplus output; Glorot seed 0, output bias NROB_B3); k1~U[0.04,0.06], k3 = 1e4;
                 y0 = (1,0,0); t in [1e-5, 1e5]; 20 log-spaced saves; rtol 1e-6, atol 1e-10.
    lorenz_paper: the paper's timing ensemble (rho evenly over [0, 21], sigma = 10,
                 beta = 8/3, y0 = (1, 0, 0), t in [0, 1], rtol 1e-6, atol 1e-9).
    """
    if name == "lorenz":
        ci = 0
        rtol = 1e-6 if rtol is None else rtol
        p = np.stack([uniform(_stream(ci, 0, seed), n, 8, 12), uniform(_stream(ci, 1, seed), n, 20, 30),
                      uniform(_stream(ci, 2, seed), n, 2, 3)], 1)
        y0 = 1.0 + 0.1 * normal(_stream(ci, 3, seed), 3 * n).reshape(n, 3)
        return dict(problem="lorenz", params=p, y0=y0, t0=0.0, t1=1.0, save_t=uniform_saves(0.0, 1.0, 10),
                    rtol=rtol, atol=1e-2 * rtol, w=None)
    if name == "vdp":
        ci = 1
        rtol = 1e-6 if rtol is None else rtol
        p = uniform(_stream(ci, 0, seed), n, 0.5, 2.0).reshape(n, 1)
        y0 = uniform(_stream(ci, 1, seed), 2 * n, -2.0, 2.0).reshape(n, 2)
        return dict(problem="vdp", params=p, y0=y0, t0=0.0, t1=10.0, save_t=uniform_saves(0.0, 10.0, 50),
                    rtol=rtol, atol=1e-2 * rtol, w=None)
    if name == "robertson":
        ci = 2
        rtol = 1e-6 if rtol is None else rtol
        p = ROBERTSON_RATES[None, :] * _logu(_stream(ci, 0, seed), 3 * n).reshape(n, 3)
        y0 = np.tile(np.array([1.0, 0.0, 0.0]), (n, 1))
        return dict(problem="robertson", params=p, y0=y0, t0=1e-5, t1=1e5, save_t=log_saves(1e-5, 1e5, 20),
                    rtol=rtol, atol=1e-10, w=None)
    if name == "hires":
        ci = 3
        rtol = 1e-6 if rtol is None else rtol
        p = HIRES_RATES[None, :] * _logu(_stream(ci, 0, seed), 12 * n).reshape(n, 12)
        y0 = np.tile(HIRES_Y0, (n, 1))
        return dict(problem="hires", params=p, y0=y0, t0=0.0, t1=321.8122,
                    save_t=uniform_saves(0.0, 321.8122, 10), rtol=rtol, atol=1e-10, w=None)
    if name == "lv_ude":
        ci = 4
        rtol = 1e-6 if rtol is None else rtol
        p = np.stack([uniform(_stream(ci, 0, seed), n, 1.0, 1.5), uniform(_stream(ci, 1, seed), n, 2.0, 3.0)], 1)
        y0 = uniform(_stream(ci, 2, seed), 2 * n, 0.5, 2.0).reshape(n, 2)
        return dict(problem="lv_ude", params=p, y0=y0, t0=0.0, t1=5.0, save_t=uniform_saves(0.0, 5.0, 10),
                    rtol=rtol, atol=1e-2 * rtol, w=glorot_mlp(0))
    if name == "nrob":
        ci = 6
        rtol = 1e-6 if rtol is None else rtol
        p = np.stack([uniform(_stream(ci, 0, seed), n, 0.04, 0.06), np.full(n, 1e4)], 1)
        y0 = np.tile(np.array([1.0, 0.0, 0.0]), (n, 1))
        return dict(problem="nrob", params=p, y0=y0, t0=1e-5, t1=1e5, save_t=log_saves(1e-5, 1e5, 20),
                    rtol=rtol, atol=1e-10, w=glorot_nrob(0))
    if name == "lorenz_paper":
        rtol = 1e-6 if rtol is None else rtol
        rho = np.linspace(0.0, 21.0, n)
        p = np.stack([np.full(n, 10.0), rho, np.full(n, 8.0 / 3.0)], 1)
        y0 = np.tile(np.array([1.0, 0.0, 0.0]), (n, 1))
        return dict(problem="lorenz", params=p, y0=y0, t0=0.0, t1=1.0, save_t=np.array([1.0]),
                    rtol=rtol, atol=1e-9, w=None)
    raise KeyError(name)

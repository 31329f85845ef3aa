"""Seeded synthetic inputs for tensor-product spline smoothing.

This module holds only random-number generation and the recipes of the
synthetic workloads (point clouds and noisy responses).  It contains none of
the smoothing method's arithmetic, so both the CUDA path's harness and the
CPU oracle can draw identical inputs from it without sharing any code of the
method.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used in counter mode, so the i-th draw of a
stream is mix(key + (i+1) * GAMMA).  Uniform doubles take the top 53 bits;
normals use the Box-Muller transform.

Bit-identical on x86_64 and aarch64: besides numpy uint64 arithmetic, the
recipes use only IEEE-754 basic operations (+, -, *, /, sqrt, frexp/ldexp,
rint), each correctly rounded, in a fixed order.  numpy's own log/exp/sin/cos
are vectorised differently per CPU and may differ in the last bit, so the
logarithm, exponential, sine and cosine below are evaluated from their power
series after an exact argument reduction (accurate to a few units in the last
place; what matters here is that both machines draw the same numbers), and
sums over coordinates are written out instead of reduced by numpy.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from decimal import Decimal

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


# ---------------------------------------------------------------- portable elementary functions

_LN2_DEC = "0.69314718055994530941723212145817656807550013436"   # ln 2 to 47 digits
_LN2 = float(_LN2_DEC)                    # the double nearest ln 2
_LN2_HI = 2977044472.0 / 4294967296.0     # ln 2 to 32 bits: k * _LN2_HI is exact for |k| < 2^21
_LN2_LO = float(Decimal(_LN2_DEC) - Decimal(2977044472) / Decimal(4294967296))   # the rest, rounded once
_SQRT_HALF = 0.7071067811865476
_TWO_PI = 6.283185307179586


def _horner(c: list, z: np.ndarray) -> np.ndarray:
    acc = np.full_like(z, c[-1])
    for a in reversed(c[:-1]):
        acc = acc * z + a
    return acc


def plog(u: np.ndarray) -> np.ndarray:
    """Natural logarithm of u > 0: u = m 2^e with m in [sqrt(1/2), sqrt(2)),
    log m = 2 atanh(s), s = (m - 1)/(m + 1), |s| < 0.172, by 14 terms of the
    atanh series."""
    u = np.asarray(u, dtype=np.float64)
    m, e = np.frexp(u)
    low = m < _SQRT_HALF
    m = np.where(low, m * 2.0, m)
    e = np.where(low, e - 1, e).astype(np.float64)
    s = (m - 1.0) / (m + 1.0)
    poly = _horner([1.0 / (2 * k + 1) for k in range(14)], s * s)
    return e * _LN2 + 2.0 * s * poly


def pexp(x: np.ndarray) -> np.ndarray:
    """e^x: x = k ln 2 + r with |r| <= ln2 / 2 (two-part ln 2), e^r by 18 terms
    of its series, scaled by 2^k."""
    x = np.asarray(x, dtype=np.float64)
    k = np.rint(x / _LN2)
    k = np.clip(k, -1100.0, 1100.0)
    r = (x - k * _LN2_HI) - k * _LN2_LO
    p = _horner([1.0 / math.factorial(j) for j in range(18)], r)
    return np.ldexp(p, k.astype(np.int64))


def _sincos_reduced(t: np.ndarray):
    """t in turns: t = q/4 + r, |r| <= 1/8 (exact for |t| <= 2^50); returns
    (sin 2 pi r, cos 2 pi r, q mod 4) by 12-term series."""
    t = np.asarray(t, dtype=np.float64)
    k = np.rint(4.0 * t)
    r = t - k * 0.25
    x = r * _TWO_PI
    z = x * x
    c = _horner([(-1.0) ** j / math.factorial(2 * j) for j in range(12)], z)
    sn = x * _horner([(-1.0) ** j / math.factorial(2 * j + 1) for j in range(12)], z)
    return sn, c, np.mod(k, 4.0)


def psin_turns(t: np.ndarray) -> np.ndarray:
    """sin(2 pi t)."""
    sn, c, q = _sincos_reduced(t)
    return np.select([q == 0, q == 1, q == 2], [sn, c, -sn], -c)


def pcos_turns(t: np.ndarray) -> np.ndarray:
    """cos(2 pi t)."""
    sn, c, q = _sincos_reduced(t)
    return np.select([q == 0, q == 1, q == 2], [c, -sn, -c], sn)


def _sq_dist(x: np.ndarray, c) -> np.ndarray:
    """|x_i - c|^2, summed over the coordinates in order."""
    d = x[:, 0] - c[0]
    r2 = d * d
    for p in range(1, x.shape[1]):
        d = x[:, p] - c[p]
        r2 = r2 + d * d
    return r2


def _log_uniform(lo: float, hi: float, u: float) -> float:
    """exp(log lo + u (log hi - log lo)) with the portable functions."""
    a, b = plog(np.array([lo, hi]))
    return float(pexp(np.array([a + u * (b - a)]))[0])


def _stream_key(seed: int, stream: int) -> np.uint64:
    base = np.array([(seed * 0x2545F4914F6CDD1D + stream * 0x632BE59BD9B4E019) & 0xFFFFFFFFFFFFFFFF],
                    dtype=np.uint64)
    return _mix(base)[0]


def splitmix_u64(seed: int, stream: int, count: int) -> np.ndarray:
    """count raw 64-bit draws of stream `stream` under `seed`."""
    key = _stream_key(seed, stream)
    with np.errstate(over="ignore"):
        ctr = np.arange(1, count + 1, dtype=np.uint64) * GAMMA + key
    return _mix(ctr)


def uniform(seed: int, stream: int, count: int) -> np.ndarray:
    """count doubles in [0, 1)."""
    return (splitmix_u64(seed, stream, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """count standard normal doubles (Box-Muller, cosine branch)."""
    u = uniform(seed, stream, 2 * count)
    u1 = 1.0 - u[:count]          # (0, 1]
    u2 = u[count:]
    return np.sqrt(-2.0 * plog(u1)) * pcos_turns(u2)


@dataclass
class Problem:
    """One smoothing problem: points x (n x P, row-major), responses y, grid and penalty."""
    name: str
    P: int
    q: int
    intervals: list          # N_p, knot intervals per dimension on the finest grid
    levels: int              # number of grid levels G
    lam: float
    tol: float
    x: np.ndarray
    y: np.ndarray
    lo: list = field(default_factory=list)
    hi: list = field(default_factory=list)
    precision: str = "fp64"  # "fp64" or "mixed"

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def K(self) -> int:
        k = 1
        for N in self.intervals:
            k *= N + self.q
        return k


def uniform_points(seed: int, stream: int, n: int, P: int) -> np.ndarray:
    return uniform(seed, stream, n * P).reshape(n, P)


def pr1(seed: int = 0, n: int = 2000) -> Problem:
    """P=2, 16 intervals, n=2000 uniform, y = sin(2 pi x1) cos(2 pi x2) + N(0, 0.1^2)."""
    x = uniform_points(seed, 1, n, 2)
    y = psin_turns(x[:, 0]) * pcos_turns(x[:, 1]) + 0.1 * normal(seed, 2, n)
    return Problem("pr1", 2, 3, [16, 16], 3, 1e-3, 1e-10, x, y, [0.0] * 2, [1.0] * 2)


def gaussian_mixture_points(seed: int, n: int, P: int, comps: int = 3) -> np.ndarray:
    """Equal-weight isotropic Gaussian mixture clipped to [0,1]^P.

    Means are U[0.2,0.8]^P and standard deviations U[0.05,0.15], one per
    component.  Clipping leaves points exactly on the boundary faces.
    """
    means = 0.2 + 0.6 * uniform(seed, 10, comps * P).reshape(comps, P)
    sig = 0.05 + 0.10 * uniform(seed, 11, comps)
    comp = np.minimum((uniform(seed, 12, n) * comps).astype(np.int64), comps - 1)
    z = normal(seed, 13, n * P).reshape(n, P)
    x = means[comp] + sig[comp, None] * z
    return np.clip(x, 0.0, 1.0)


def scale(seed: int = 1, n: int = 1_000_000) -> Problem:
    """P=3, 64 intervals, clustered mixture, y = exp(-|x-0.5|^2/0.05) + N(0, 0.05^2)."""
    x = gaussian_mixture_points(seed, n, 3)
    r2 = _sq_dist(x, [0.5] * 3)
    y = pexp(-r2 / 0.05) + 0.05 * normal(seed, 14, n)
    return Problem("scale", 3, 3, [64, 64, 64], 6, 1e-4, 1e-8, x, y, [0.0] * 3, [1.0] * 3)


def mixed(seed: int = 2, n: int = 4_000_000) -> Problem:
    """P=4, 32 intervals, n uniform stored as FP32, y = prod sin(pi x_d) + N(0, 0.1^2)."""
    x = uniform_points(seed, 1, n, 4).astype(np.float32)
    xd = x.astype(np.float64)
    f = psin_turns(0.5 * xd[:, 0])
    for p in range(1, 4):
        f = f * psin_turns(0.5 * xd[:, p])
    y = (f + 0.1 * normal(seed, 2, n)).astype(np.float32)
    return Problem("mixed", 4, 3, [32] * 4, 5, 1e-3, 1e-10, x, y, [0.0] * 4, [1.0] * 4,
                   precision="mixed")


def bumps_response(seed: int, stream: int, x: np.ndarray, noise: float = 0.05) -> np.ndarray:
    """Sum of 3 Gaussian bumps (amplitude U[-1,1], width U[0.05,0.3], centre U[0,1]^P) + noise."""
    n, P = x.shape
    amp = -1.0 + 2.0 * uniform(seed, stream, 3)
    wid = 0.05 + 0.25 * uniform(seed, stream + 1, 3)
    cen = uniform(seed, stream + 2, 3 * P).reshape(3, P)
    y = np.zeros(n)
    for b in range(3):
        r2 = _sq_dist(x, cen[b])
        y += amp[b] * pexp(-r2 / (2.0 * (wid[b] * wid[b])))
    return y + noise * normal(seed, stream + 3, n)


def levels_for(N: int, coarsest: int = 2) -> int:
    """Levels from N intervals down to `coarsest` intervals by halving."""
    g = 1
    while (N >> (g - 1)) > coarsest:
        g += 1
    return g


BATCH_GRIDS = {1: [8, 16, 32, 64], 2: [8, 16, 32, 64], 3: [8, 16]}


def batched(seed: int = 3, count: int = 512, n_lo: float = 1e3, n_hi: float = 1e5,
            max_coef: int = 40_000) -> list:
    """Independent problems: P in {1,2,3}, N in {8,16,32,64} with K <= max_coef,
    n log-uniform in [n_lo, n_hi], lambda log-uniform in [1e-5, 1e-1]."""
    probs = []
    r = uniform(seed, 100, 4 * count).reshape(count, 4)
    for k in range(count):
        P = 1 + min(int(r[k, 0] * 3), 2)
        grids = [N for N in BATCH_GRIDS[P] if (N + 3) ** P <= max_coef]
        N = grids[min(int(r[k, 1] * len(grids)), len(grids) - 1)]
        n = int(round(_log_uniform(n_lo, n_hi, r[k, 2])))
        lam = _log_uniform(1e-5, 1e-1, r[k, 3])
        x = uniform_points(seed, 1000 + 8 * k, n, P)
        y = bumps_response(seed, 1001 + 8 * k, x)
        probs.append(Problem(f"batch{k}", P, 3, [N] * P, levels_for(N), lam, 1e-8, x, y,
                             [0.0] * P, [1.0] * P, precision="mixed"))
    return probs


SERVE_GRIDS = {2: [32, 64, 128], 3: [16, 32, 64], 4: [16, 32], 5: [16]}


@dataclass
class Request:
    t_arrival: float
    problem: Problem


def serving_trace(seed: int = 4, count: int = 2000, rate: float = 200.0, n_lo: float = 1e4,
                  n_hi: float = 2e6, P_choices=(2, 3, 4, 5), materialize: bool = True) -> list:
    """Poisson arrivals (exponential gaps, mean 1/rate s) of smoothing requests.

    P uniform over P_choices, N from SERVE_GRIDS[P], n log-uniform in
    [n_lo, n_hi], lambda log-uniform in [1e-5, 1e-2], uniform points and a
    3-bump response.  With materialize=False the points are not drawn
    (x, y are None) so a trace can be inspected cheaply.
    """
    r = uniform(seed, 200, 5 * count).reshape(count, 5)
    t = np.cumsum(-plog(1.0 - r[:, 0]) / rate)
    out = []
    for k in range(count):
        P = P_choices[min(int(r[k, 1] * len(P_choices)), len(P_choices) - 1)]
        grids = SERVE_GRIDS[P]
        N = grids[min(int(r[k, 2] * len(grids)), len(grids) - 1)]
        n = int(round(_log_uniform(n_lo, n_hi, r[k, 3])))
        lam = _log_uniform(1e-5, 1e-2, r[k, 4])
        if materialize:
            x = uniform_points(seed, 5000 + 8 * k, n, P)
            y = bumps_response(seed, 5001 + 8 * k, x)
        else:
            x = np.zeros((n, P)); y = None
        out.append(Request(float(t[k]), Problem(f"req{k}", P, 3, [N] * P, levels_for(N), lam, 1e-8,
                                                x, y, [0.0] * P, [1.0] * P, precision="mixed")))
    return out


def paper_sigmoid(seed: int, n: int, P: int) -> tuple:
    """Section 4 test data: uniform x in [0,1]^P, y = f_P(x) + N(0, 0.1^2) with
    f_P(x) = 1 / (1 + exp(-16 (|x|^2 / P - 0.5))) (the bounded reading of the
    sigmoid; the printed denominator 1 - exp(...) has a pole)."""
    x = uniform_points(seed, 1, n, P)
    f = 1.0 / (1.0 + pexp(-16.0 * (_sq_dist(x, [0.0] * P) / P - 0.5)))
    return x, f + 0.1 * normal(seed, 2, n)

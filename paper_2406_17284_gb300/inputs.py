"""Seeded synthetic inputs shared by the CUDA tests, the benchmark and the oracle.

This module holds no arithmetic of the method itself: it only draws initial
grids, places textbook Game-of-Life patterns and lists workload parameters.

Random cells come from a counter-based generator so that any window of a huge
grid can be regenerated on its own: cell (y, x) of a grid of width W drawn with
``seed`` uses the 64-bit SplitMix64 output (Steele, Lea & Flood, OOPSLA 2014;
the finaliser of Java's SplittableRandom) for counter i = y*W + x:

    z = seed + (i + 1) * 0x9E3779B97F4A7C15          (mod 2^64)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    z =  z ^ (z >> 31)

Bernoulli(p) cells are alive when z < floor(p * 2^64); uniform states over
{0..C-1} are ((z >> 32) * C) >> 32.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counters: np.ndarray, seed: int) -> np.ndarray:
    """SplitMix64 outputs for an array of uint64 counters (vectorised)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (counters.astype(np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _window_counters(W: int, y0: int, x0: int, h: int, w: int) -> np.ndarray:
    ys = np.arange(y0, y0 + h, dtype=np.uint64)[:, None]
    xs = np.arange(x0, x0 + w, dtype=np.uint64)[None, :]
    return ys * np.uint64(W) + xs


def _threshold(p: float) -> np.uint64:
    if not (0.0 <= p <= 1.0):
        raise ValueError("p must be in [0, 1]")
    t = int(math.floor(p * 2.0 ** 64))
    return np.uint64(min(t, 2 ** 64 - 1))


def _rows_parallel(H: int, fn, out: np.ndarray, chunk: int = 512):
    if H * out.shape[1] < (1 << 22):
        fn(0, H, out)
        return out
    workers = min(32, os.cpu_count() or 1)
    with ThreadPoolExecutor(workers) as ex:
        list(ex.map(lambda y: fn(y, min(H, y + chunk), out), range(0, H, chunk)))
    return out


def bernoulli_window(H: int, W: int, p: float, seed: int, y0: int = 0, x0: int = 0,
                     h: int | None = None, w: int | None = None) -> np.ndarray:
    """Window [y0, y0+h) x [x0, x0+w) of the Bernoulli(p) grid (H, W, seed) as uint8.

    Coordinates outside the grid are returned as 0 (dead ghost cells).
    """
    h = H - y0 if h is None else h
    w = W - x0 if w is None else w
    thr = _threshold(p)
    out = np.zeros((h, w), dtype=np.uint8)
    ya, yb = max(y0, 0), min(y0 + h, H)
    xa, xb = max(x0, 0), min(x0 + w, W)
    if ya >= yb or xa >= xb:
        return out
    inner = out[ya - y0:yb - y0, xa - x0:xb - x0]

    def fill(r0, r1, dst):
        z = splitmix64(_window_counters(W, ya + r0, xa, r1 - r0, xb - xa), seed)
        dst[r0:r1] = (z < thr).astype(np.uint8)

    _rows_parallel(yb - ya, fill, inner)
    return out


def bernoulli(H: int, W: int, p: float, seed: int) -> np.ndarray:
    """Whole H x W grid of alive(1)/dead(0) cells drawn Bernoulli(p)."""
    return bernoulli_window(H, W, p, seed)


def uniform_states_window(H: int, W: int, C: int, seed: int, y0: int = 0, x0: int = 0,
                          h: int | None = None, w: int | None = None) -> np.ndarray:
    """Window of the grid whose cells are uniform over {0..C-1}; outside cells are 0."""
    if not (2 <= C <= 256):
        raise ValueError("C must be in [2, 256]")
    h = H - y0 if h is None else h
    w = W - x0 if w is None else w
    out = np.zeros((h, w), dtype=np.uint8)
    ya, yb = max(y0, 0), min(y0 + h, H)
    xa, xb = max(x0, 0), min(x0 + w, W)
    if ya >= yb or xa >= xb:
        return out
    inner = out[ya - y0:yb - y0, xa - x0:xb - x0]

    def fill(r0, r1, dst):
        z = splitmix64(_window_counters(W, ya + r0, xa, r1 - r0, xb - xa), seed)
        dst[r0:r1] = (((z >> np.uint64(32)) * np.uint64(C)) >> np.uint64(32)).astype(np.uint8)

    _rows_parallel(yb - ya, fill, inner)
    return out


def uniform_states(H: int, W: int, C: int, seed: int) -> np.ndarray:
    return uniform_states_window(H, W, C, seed)


# --------------------------------------------------------------------------
# Textbook Game-of-Life patterns (Gardner, Sci. Am. 223, 1970), as (dy, dx)
# offsets of the live cells.
# --------------------------------------------------------------------------
PATTERNS = {
    "block": [(0, 0), (0, 1), (1, 0), (1, 1)],
    "beehive": [(0, 1), (0, 2), (1, 0), (1, 3), (2, 1), (2, 2)],
    "loaf": [(0, 1), (0, 2), (1, 0), (1, 3), (2, 1), (2, 3), (3, 2)],
    "blinker": [(0, 0), (0, 1), (0, 2)],
    "toad": [(0, 1), (0, 2), (0, 3), (1, 0), (1, 1), (1, 2)],
    "beacon": [(0, 0), (0, 1), (1, 0), (2, 3), (3, 2), (3, 3)],
    # glider heading towards +y, +x (down-right)
    "glider": [(0, 1), (1, 2), (2, 0), (2, 1), (2, 2)],
}


def place(grid: np.ndarray, name: str, y: int, x: int, state: int = 1) -> np.ndarray:
    for dy, dx in PATTERNS[name]:
        grid[y + dy, x + dx] = state
    return grid


# --------------------------------------------------------------------------
# Workload parameters
# --------------------------------------------------------------------------
def scaled_rule_ranges(r: int) -> tuple[int, int, int, int]:
    """(s1, s2, b1, b2) of the radius-scaled rule used by the radius sweeps.

    With n = (2r+1)^2: S round(0.34n)..round(0.58n), B round(0.34n)..round(0.45n),
    rounding half up in exact integer arithmetic, (p*n + 50) // 100.
    """
    n = (2 * r + 1) ** 2
    rnd = lambda pct: (pct * n + 50) // 100  # noqa: E731
    return rnd(34), rnd(58), rnd(34), rnd(45)


def scaled_rule(r: int, M: int = 1, C: int = 2) -> dict:
    s1, s2, b1, b2 = scaled_rule_ranges(r)
    return dict(r=r, C=C, M=M, s1=s1, s2=s2, b1=b1, b2=b2)


def vn_scaled_rule_ranges(r: int) -> tuple[int, int, int, int]:
    """The same percentages for the simplified von Neumann cross (vertical plus
    horizontal segment of half-length r): n = 4r + 1 cells, the centre once."""
    n = 4 * r + 1
    rnd = lambda pct: (pct * n + 50) // 100  # noqa: E731
    return rnd(34), rnd(58), rnd(34), rnd(45)


def vn_scaled_rule(r: int, M: int = 1, C: int = 2) -> dict:
    s1, s2, b1, b2 = vn_scaled_rule_ranges(r)
    return dict(r=r, C=C, M=M, s1=s1, s2=s2, b1=b1, b2=b2, nbhd="N")


CONWAY = dict(r=1, C=2, M=0, s1=2, s2=3, b1=3, b2=3)
MULTISTATE_R10_C16 = dict(r=10, C=16, M=1, s1=150, s2=260, b1=150, b2=200)


def batch_instances(count: int, seed: int, side_lo: int = 64, side_hi: int = 2048) -> list[dict]:
    """Heterogeneous batch: sides log-uniform in [side_lo, side_hi] (independent H, W),
    r uniform in 1..16, M uniform in {0,1}, p uniform in [0.2, 0.6], the scaled rule, C = 2.
    Each instance carries its own grid seed.
    """
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    lo, hi = math.log(side_lo), math.log(side_hi)
    for i in range(count):
        H = int(round(math.exp(rng.uniform(lo, hi))))
        W = int(round(math.exp(rng.uniform(lo, hi))))
        r = int(rng.integers(1, 17))
        M = int(rng.integers(0, 2))
        p = float(rng.uniform(0.2, 0.6))
        out.append(dict(H=H, W=W, p=p, seed=int(seed * 100003 + i), rule=scaled_rule(r, M)))
    return out

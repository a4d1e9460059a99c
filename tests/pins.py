"""Pins for the CPU oracle: facts fixed by the CAT paper and by mathematics.

Each ``pin_*`` function takes an oracle library handle (``oracle.load()`` or a
deliberately mutated build) and raises ``AssertionError`` when the oracle
disagrees with the fact.  ``tests/test_oracle_pins.py`` runs them against the
real oracle and against mutated builds (each mutated build must fail at least
one pin).

None of these re-types the oracle's loop: the box count is checked against the
paper's own band-matrix product (Sec. IV, Eqs. 1-2, evaluated with numpy's
integer matmul), a summed-area table, closed forms and textbook Game-of-Life
behaviour; the simplified von Neumann count against Eq. 3's products, its
impulse response and closed forms; the transition against a table built from
the rule's ranges.
"""
from __future__ import annotations

import os

import numpy as np

from oracle import oracle
from paper_2406_17284_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ---------------------------------------------------------------- references
def band(n: int, r: int, periodic: bool) -> np.ndarray:
    """The band matrix Pi of Sec. IV: ones where |i - j| <= r (circulant if periodic).

    For a torus narrower than the box, offsets that land on the same cell are
    counted once per offset, as with a halo of ghost copies.
    """
    P = np.zeros((n, n), dtype=np.int64)
    for i in range(n):
        for d in range(-r, r + 1):
            j = i + d
            if periodic:
                P[i, j % n] += 1
            elif 0 <= j < n:
                P[i, j] += 1
    return P


def band_product_sums(grid: np.ndarray, r: int, periodic: bool) -> np.ndarray:
    """R = Pi_H * Lambda * Pi_W (Eqs. 1-2): horizontal then vertical reduction."""
    lam = (grid == 1).astype(np.int64)
    H, W = lam.shape
    Hm = lam @ band(W, r, periodic)          # Eq. 1: H = Lambda x Pi
    return band(H, r, periodic) @ Hm         # Eq. 2: R = Pi x H


def cross_product_sums(grid: np.ndarray, r: int, periodic: bool) -> np.ndarray:
    """Eq. 3: R = Pi * Lambda + H with H = Lambda * Pi (vertical plus horizontal reduction)."""
    lam = (grid == 1).astype(np.int64)
    H, W = lam.shape
    return band(H, r, periodic) @ lam + lam @ band(W, r, periodic)


def sat_sums(grid: np.ndarray, r: int) -> np.ndarray:
    """Box sums with a zero boundary from a summed-area table."""
    lam = (grid == 1).astype(np.int64)
    H, W = lam.shape
    T = np.zeros((H + 1, W + 1), dtype=np.int64)
    T[1:, 1:] = lam.cumsum(0).cumsum(1)
    y = np.arange(H)[:, None]
    x = np.arange(W)[None, :]
    y0, y1 = np.clip(y - r, 0, H), np.clip(y + r + 1, 0, H)
    x0, x1 = np.clip(x - r, 0, W), np.clip(x + r + 1, 0, W)
    return T[y1, x1] - T[y0, x1] - T[y1, x0] + T[y0, x0]


def table_transition(grid: np.ndarray, S: np.ndarray, rule: oracle.Rule) -> np.ndarray:
    """Next states from box sums through lookup tables built from the rule's ranges.

    A live cell's own state is in S once (Moore) or twice (Eq. 3); the rule's
    count k keeps it once when M = 1 and drops it when M = 0.
    """
    C, M = rule.C, rule.M
    twice = 2 if rule.nbhd == "N" else 1
    n_max = int(S.max(initial=0)) + 2
    born = np.zeros(n_max + 1, dtype=np.uint8)
    born[max(rule.b1, 0):max(min(rule.b2, n_max) + 1, 0)] = 1
    keep = np.zeros(n_max + 1, dtype=np.uint8)
    keep[max(rule.s1, 0):max(min(rule.s2, n_max) + 1, 0)] = 1
    out = np.zeros_like(grid)
    dead = grid == 0
    alive = grid == 1
    k_alive = S - (twice - M)
    out[dead] = born[np.clip(S[dead], 0, n_max)]
    surv = keep[np.clip(k_alive[alive], 0, n_max)]
    out[alive] = np.where(surv == 1, 1, 2 if C > 2 else 0)
    dying = grid >= 2
    nxt = grid[dying].astype(np.int64) + 1
    out[dying] = np.where(nxt == C, 0, nxt).astype(np.uint8)
    return out


def read_table_iv():
    rows = []
    with open(os.path.join(GOLDEN, "ltl_table_iv.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            r, C, M, s1, s2, b1, b2, N, dens, name = line.split()
            rows.append(dict(rule=oracle.Rule(int(r), int(C), int(M), int(s1), int(s2), int(b1), int(b2)),
                             N=N, density=float(dens), name=name))
    return rows


def read_conway_patterns():
    rows = []
    with open(os.path.join(GOLDEN, "conway_patterns.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, period, dy, dx = line.split()
            rows.append((name, int(period), int(dy), int(dx)))
    return rows


CONWAY = oracle.Rule(**inputs.CONWAY)


# --------------------------------------------------------------------- pins
def pin_band_product(lib):
    """Oracle box sums == the paper's two band products, both boundaries."""
    rng = np.random.default_rng(11)
    for (H, W) in [(1, 1), (3, 5), (7, 4), (12, 12), (17, 9), (20, 33)]:
        for r in (0, 1, 2, 3, 5, 8, 16, 24, 32):
            for C in (2, 4):
                g = rng.integers(0, C, size=(H, W), dtype=np.uint8)
                for periodic in (False, True):
                    got = oracle.box_sums(g, r, oracle.PERIODIC if periodic else oracle.ZERO, lib=lib)
                    want = band_product_sums(g, r, periodic)
                    assert np.array_equal(got, want), (H, W, r, C, periodic)


def pin_sat(lib):
    """Oracle box sums == summed-area-table recount (zero boundary), up to 512^2."""
    for (H, W, p, seed) in [(256, 256, 0.5, 1), (512, 384, 0.35, 2), (131, 517, 0.8, 3)]:
        g = inputs.bernoulli(H, W, p, seed)
        for r in (1, 4, 7, 11, 16):
            assert np.array_equal(oracle.box_sums(g, r, lib=lib), sat_sums(g, r)), (H, W, r)


def pin_all_ones(lib):
    """All-ones grid, zero halo: S(y,x) = clipped box area (max (2r+1)^2 = 1089)."""
    for (H, W) in [(40, 40), (70, 45), (3, 100)]:
        g = np.ones((H, W), np.uint8)
        for r in (1, 2, 9, 16, 32):
            y = np.arange(H)[:, None]
            x = np.arange(W)[None, :]
            area = (np.minimum(y + r, H - 1) - np.maximum(y - r, 0) + 1) * \
                   (np.minimum(x + r, W - 1) - np.maximum(x - r, 0) + 1)
            assert np.array_equal(oracle.box_sums(g, r, lib=lib), area), (H, W, r)
    g = np.ones((80, 80), np.uint8)
    assert oracle.box_sums(g, 16, lib=lib)[40, 40] == 33 * 33
    assert oracle.box_sums(g, 32, lib=lib)[40, 40] == 65 * 65


def pin_impulse(lib):
    """A single live cell gives S = the (2r+1)^2 box of ones around it (band impulse response)."""
    for r in (1, 3, 8, 16, 25):
        n = 2 * r + 9
        g = np.zeros((n, n + 3), np.uint8)
        cy, cx = n // 2, n // 2 + 1
        g[cy, cx] = 1
        want = np.zeros_like(g, dtype=np.int32)
        want[cy - r:cy + r + 1, cx - r:cx + r + 1] = 1
        assert np.array_equal(oracle.box_sums(g, r, lib=lib), want), r


def pin_transition_table(lib):
    """Oracle steps == table-driven transition on band-product sums, random rules incl. C > 2."""
    rng = np.random.default_rng(5)
    for trial in range(60):
        H, W = int(rng.integers(1, 14)), int(rng.integers(1, 14))
        r = int(rng.integers(1, 6))
        C = int(rng.choice([2, 3, 5, 16]))
        M = int(rng.integers(0, 2))
        n = (2 * r + 1) ** 2
        s1, s2 = sorted(int(v) for v in rng.integers(0, n + 1, 2))
        b1, b2 = sorted(int(v) for v in rng.integers(1, n + 1, 2))
        rule = oracle.Rule(r, C, M, s1, s2, b1, b2)
        g = rng.integers(0, C, size=(H, W), dtype=np.uint8)
        periodic = bool(rng.integers(0, 2))
        got = oracle.step(g, rule, oracle.PERIODIC if periodic else oracle.ZERO, lib=lib)
        want = table_transition(g, band_product_sums(g, r, periodic), rule)
        assert np.array_equal(got, want), (trial, rule, periodic)


def pin_conway(lib):
    """Textbook Game of Life: still lifes, period-2 oscillators, glider shift (1,1) per 4 steps."""
    for name, period, dy, dx in read_conway_patterns():
        g = np.zeros((24, 24), np.uint8)
        inputs.place(g, name, 8, 8)
        one = oracle.step(g, CONWAY, lib=lib)
        after = oracle.step(g, CONWAY, n_steps=period, lib=lib)
        shifted = np.roll(g, (dy, dx), (0, 1))
        assert np.array_equal(after, shifted), name
        if period > 1:
            assert not np.array_equal(one, g), name
    # a glider keeps moving: 20 steps -> shifted by (5, 5)
    g = np.zeros((32, 32), np.uint8)
    inputs.place(g, "glider", 2, 2)
    want = np.zeros_like(g)
    inputs.place(want, "glider", 7, 7)
    assert np.array_equal(oracle.step(g, CONWAY, n_steps=20, lib=lib), want)


def pin_all_zero(lib):
    """An all-dead grid stays dead under every rule with b1 >= 1."""
    for row in read_table_iv():
        rule = row["rule"]
        assert rule.b1 >= 1
        g = np.zeros((40, 37), np.uint8)
        assert not oracle.step(g, rule, n_steps=3, lib=lib).any(), rule


def pin_decay_chain(lib):
    """An isolated cell in state c >= 2 reaches 0 after exactly C - c steps; a lone live
    cell under M0 with s1 >= 1 dies into state 2 and is gone after C - 1 steps."""
    for C in (3, 5, 16):
        rule = oracle.Rule(2, C, 0, 1, 5, 3, 6)
        for c in range(2, C):
            g = np.zeros((9, 9), np.uint8)
            g[4, 4] = c
            for t in range(1, C - c + 1):
                g = oracle.step(g, rule, lib=lib)
                want = 0 if t == C - c else c + t
                assert g[4, 4] == want and g.sum() == want, (C, c, t)
        g = np.zeros((9, 9), np.uint8)
        g[4, 4] = 1
        g1 = oracle.step(g, rule, lib=lib)
        assert g1[4, 4] == 2 and g1.sum() == 2
        assert not oracle.step(g, rule, n_steps=C - 1, lib=lib).any()


def pin_periodic_translation(lib):
    """Periodic boundary: stepping commutes with cyclic shifts."""
    rng = np.random.default_rng(3)
    g = rng.integers(0, 3, size=(23, 31), dtype=np.uint8)
    rule = oracle.Rule(3, 3, 1, 10, 25, 9, 14)
    base = oracle.step(g, rule, oracle.PERIODIC, lib=lib)
    for sy, sx in [(1, 0), (0, 1), (5, 17), (22, 30)]:
        moved = oracle.step(np.roll(g, (sy, sx), (0, 1)), rule, oracle.PERIODIC, lib=lib)
        assert np.array_equal(moved, np.roll(base, (sy, sx), (0, 1))), (sy, sx)


def pin_transpose(lib):
    """The Moore box is symmetric: step(G^T) == step(G)^T on a rectangular grid."""
    g = inputs.bernoulli(37, 53, 0.45, 9)
    for row in read_table_iv()[:6]:
        rule = row["rule"]
        for b in (oracle.ZERO, oracle.PERIODIC):
            assert np.array_equal(oracle.step(g.T.copy(), rule, b, lib=lib),
                                  oracle.step(g, rule, b, lib=lib).T), (rule, b)


def pin_middle_flag(lib):
    """M0 with survival s1..s2 == M1 with survival s1+1..s2+1 (centre of a live cell is 1)."""
    g = inputs.bernoulli(48, 48, 0.4, 4)
    for r in (1, 4, 9):
        s1, s2, b1, b2 = inputs.scaled_rule_ranges(r)
        m0 = oracle.Rule(r, 2, 0, s1, s2, b1, b2)
        m1 = oracle.Rule(r, 2, 1, s1 + 1, s2 + 1, b1, b2)
        assert np.array_equal(oracle.step(g, m0, lib=lib), oracle.step(g, m1, lib=lib)), r


# ------------------------------------------- simplified von Neumann (Eq. 3)
def pin_vn_band_product(lib):
    """Oracle cross sums == Pi x Lambda + Lambda x Pi (Eq. 3), both boundaries."""
    rng = np.random.default_rng(12)
    for (H, W) in [(1, 1), (3, 5), (7, 4), (12, 12), (17, 9), (20, 33)]:
        for r in (0, 1, 2, 5, 8, 16):
            g = rng.integers(0, 3, size=(H, W), dtype=np.uint8)
            for periodic in (False, True):
                got = oracle.box_sums(g, r, oracle.PERIODIC if periodic else oracle.ZERO, lib=lib, nbhd="N")
                assert np.array_equal(got, cross_product_sums(g, r, periodic)), (H, W, r, periodic)


def pin_vn_impulse(lib):
    """A single live cell gives a cross of arm length r, 2 at its centre (on both segments)."""
    for r in (1, 4, 16):
        n = 2 * r + 7
        g = np.zeros((n, n + 2), np.uint8)
        cy, cx = n // 2, n // 2 + 1
        g[cy, cx] = 1
        want = np.zeros(g.shape, np.int32)
        want[cy - r:cy + r + 1, cx] += 1
        want[cy, cx - r:cx + r + 1] += 1
        assert want[cy, cx] == 2
        assert np.array_equal(oracle.box_sums(g, r, lib=lib, nbhd="N"), want), r


def pin_vn_all_ones(lib):
    """All-ones grid, zero halo: the clipped vertical plus the clipped horizontal segment length."""
    for (H, W) in [(40, 40), (70, 45), (3, 100)]:
        g = np.ones((H, W), np.uint8)
        for r in (1, 9, 16):
            y = np.arange(H)[:, None]
            x = np.arange(W)[None, :]
            want = (np.minimum(y + r, H - 1) - np.maximum(y - r, 0) + 1) + \
                   (np.minimum(x + r, W - 1) - np.maximum(x - r, 0) + 1)
            assert np.array_equal(oracle.box_sums(g, r, lib=lib, nbhd="N"), want), (H, W, r)
    assert oracle.box_sums(np.ones((80, 80), np.uint8), 16, lib=lib, nbhd="N")[40, 40] == 66


def pin_vn_transition_table(lib):
    """Oracle steps (nbhd N) == table-driven transition on Eq. 3 sums, random rules incl. C > 2."""
    rng = np.random.default_rng(6)
    for trial in range(60):
        H, W = int(rng.integers(1, 14)), int(rng.integers(1, 14))
        r = int(rng.integers(1, 6))
        C = int(rng.choice([2, 3, 16]))
        M = int(rng.integers(0, 2))
        n = 4 * r + 1
        s1, s2 = sorted(int(v) for v in rng.integers(0, n + 1, 2))
        b1, b2 = sorted(int(v) for v in rng.integers(1, n + 1, 2))
        rule = oracle.Rule(r, C, M, s1, s2, b1, b2, "N")
        g = rng.integers(0, C, size=(H, W), dtype=np.uint8)
        periodic = bool(rng.integers(0, 2))
        got = oracle.step(g, rule, oracle.PERIODIC if periodic else oracle.ZERO, lib=lib)
        want = table_transition(g, cross_product_sums(g, r, periodic), rule)
        assert np.array_equal(got, want), (trial, rule, periodic)


def pin_vn_neighbour_count(lib):
    """Counts from first principles: a lone live cell has 0 live neighbours (survives
    S0..0 under M0, S1..1 under M1, dies under M0 S1..1); a dead cell with one live
    cell on its cross (distance r along an axis) is born under B1..1, with one just
    off the cross (diagonal) it is not."""
    for r in (1, 3, 7):
        n = 2 * r + 5
        g = np.zeros((n, n), np.uint8)
        c = n // 2
        g[c, c] = 1
        assert oracle.step(g, oracle.Rule(r, 2, 0, 0, 0, 9, 9, "N"), lib=lib)[c, c] == 1
        assert oracle.step(g, oracle.Rule(r, 2, 1, 1, 1, 9, 9, "N"), lib=lib)[c, c] == 1
        assert oracle.step(g, oracle.Rule(r, 2, 0, 1, 1, 9, 9, "N"), lib=lib)[c, c] == 0
        for (dy, dx), born in [((0, r), 1), ((-r, 0), 1), ((1, 1), 0)]:
            h = np.zeros((n, n), np.uint8)
            h[c + dy, c + dx] = 1
            assert oracle.step(h, oracle.Rule(r, 2, 0, 5, 5, 1, 1, "N"), lib=lib)[c, c] == born, (r, dy, dx)


def pin_vn_symmetry(lib):
    """The cross is symmetric (step(G^T) == step(G)^T) and the periodic step commutes
    with cyclic shifts."""
    g = inputs.bernoulli(37, 53, 0.45, 10)
    rule = oracle.Rule(4, 2, 1, 5, 11, 5, 8, "N")
    for b in (oracle.ZERO, oracle.PERIODIC):
        assert np.array_equal(oracle.step(g.T.copy(), rule, b, lib=lib), oracle.step(g, rule, b, lib=lib).T), b
    base = oracle.step(g, rule, oracle.PERIODIC, lib=lib)
    for sy, sx in [(1, 0), (0, 1), (5, 17)]:
        moved = oracle.step(np.roll(g, (sy, sx), (0, 1)), rule, oracle.PERIODIC, lib=lib)
        assert np.array_equal(moved, np.roll(base, (sy, sx), (0, 1))), (sy, sx)


ALL_PINS = [pin_band_product, pin_sat, pin_all_ones, pin_impulse, pin_transition_table,
            pin_conway, pin_all_zero, pin_decay_chain, pin_periodic_translation,
            pin_transpose, pin_middle_flag, pin_vn_band_product, pin_vn_impulse,
            pin_vn_all_ones, pin_vn_transition_table, pin_vn_neighbour_count, pin_vn_symmetry]

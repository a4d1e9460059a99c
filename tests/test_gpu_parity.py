"""CUDA path vs the CPU oracle, element by element (bit-exact: integer work).

Every kernel/dtype the library serves is run on the same seeded inputs as the
oracle: box counts (the two band products) and whole steps, at sizes that span
several 128 x 128 tiles with ragged tails, the degenerate shapes, the rules of
the paper's Table IV, multi-state decay, and the full 16384^2 launch checked
on sampled windows.
"""
import functools

import numpy as np
import pytest

from oracle import oracle
from paper_2406_17284_gb300 import inputs
from tests import pins

pytestmark = pytest.mark.gpu

KERNELS = [("tcgen05", "fp8"), ("tcgen05", "fp16"), ("mma_sync", "fp16"), ("mma_sync", "int8"),
           ("stencil", "auto"), ("runsum", "auto")]
KIDS = [f"{k}-{d}" for k, d in KERNELS]


@pytest.fixture(scope="module")
def cat():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2406_17284_gb300 import build
    build.build()
    from paper_2406_17284_gb300 import cat as catmod
    catmod.load()
    return catmod


def rule_dict(r, C=2, M=1, s=None, b=None):
    s1, s2, b1, b2 = inputs.scaled_rule_ranges(r)
    if s is not None:
        s1, s2 = s
    if b is not None:
        b1, b2 = b
    return dict(r=r, C=C, M=M, s1=s1, s2=s2, b1=b1, b2=b2)


def orule(d):
    return oracle.Rule(d["r"], d["C"], d["M"], d["s1"], d["s2"], d["b1"], d["b2"])


@functools.lru_cache(maxsize=None)
def _grid(H, W, p, seed):
    return inputs.bernoulli(H, W, p, seed)


@functools.lru_cache(maxsize=None)
def _oracle_run(H, W, p, seed, rule_items, steps):
    return oracle.step(_grid(H, W, p, seed), orule(dict(rule_items)), n_steps=steps)


def run_gpu(cat, kernel, dtype, grid, rule, steps):
    g = cat.Grid(grid.shape[0], grid.shape[1], rule, kernel=kernel, dtype=dtype)
    try:
        g.set_state(grid)
        g.step(steps)
        out = g.get_state()
        assert g.status() == cat.CAT_OK
        return out
    finally:
        g.close()


def assert_same(got, want, what):
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        y, x = bad[0]
        raise AssertionError(f"{what}: {len(bad)} cells differ, first at ({y},{x}): got {got[y, x]} want {want[y, x]}")


# ------------------------------------------------------------- box counts
@pytest.mark.parametrize("kernel,dtype", KERNELS, ids=KIDS)
def test_box_sums_exact_every_radius(cat, kernel, dtype):
    grid = _grid(300, 437, 0.5, 7)
    for r in range(1, 17):
        g = cat.Grid(300, 437, rule_dict(r), kernel=kernel, dtype=dtype)
        try:
            g.set_state(grid)
            assert_same(g.box_sums(), oracle.box_sums(grid, r), f"S r={r}")
        finally:
            g.close()


@pytest.mark.parametrize("kernel,dtype", KERNELS, ids=KIDS)
def test_box_sums_all_ones_and_impulse(cat, kernel, dtype):
    ones = np.ones((260, 270), np.uint8)
    imp = np.zeros((200, 333), np.uint8)
    imp[100, 129] = 1
    imp[0, 0] = 1
    imp[199, 332] = 1
    for r in (1, 7, 8, 15, 16):
        for grid in (ones, imp):
            g = cat.Grid(*grid.shape, rule_dict(r), kernel=kernel, dtype=dtype)
            try:
                g.set_state(grid)
                assert_same(g.box_sums(), oracle.box_sums(grid, r), f"S r={r}")
            finally:
                g.close()
    assert oracle.box_sums(ones, 16).max() == 1089


# ------------------------------------------------------------------ steps
@pytest.mark.parametrize("kernel,dtype", KERNELS, ids=KIDS)
def test_conway_256_100_steps(cat, kernel, dtype):
    """256 x 256, Bernoulli(0.5), R1 C2 M0 S2..3 B3..3, zero halo, 100 steps."""
    grid = _grid(256, 256, 0.5, 1)
    want = _oracle_run(256, 256, 0.5, 1, tuple(inputs.CONWAY.items()), 100)
    assert_same(run_gpu(cat, kernel, dtype, grid, inputs.CONWAY, 100), want, "conway")


@pytest.mark.parametrize("kernel,dtype", KERNELS, ids=KIDS)
def test_conway_patterns(cat, kernel, dtype):
    for name, period, dy, dx in pins.read_conway_patterns():
        g = np.zeros((40, 300), np.uint8)
        inputs.place(g, name, 10, 126)  # straddles a tile boundary
        got = run_gpu(cat, kernel, dtype, g, inputs.CONWAY, period)
        assert_same(got, np.roll(g, (dy, dx), (0, 1)), name)


@pytest.mark.parametrize("kernel,dtype", KERNELS, ids=KIDS)
def test_scaled_rules_every_radius(cat, kernel, dtype):
    """The radius-scaled rule (S 0.34n..0.58n, B 0.34n..0.45n), M0 and M1, 3 steps."""
    for r in range(1, 17):
        M = r % 2
        rule = rule_dict(r, M=M)
        want = _oracle_run(384, 520, 0.5, 100 + r, tuple(rule.items()), 3)
        got = run_gpu(cat, kernel, dtype, _grid(384, 520, 0.5, 100 + r), rule, 3)
        assert_same(got, want, f"r={r} M={M}")


@pytest.mark.parametrize("kernel,dtype", KERNELS, ids=KIDS)
def test_paper_table_iv_rules(cat, kernel, dtype):
    for row in pins.read_table_iv():
        rr = row["rule"]
        rule = dict(r=rr.r, C=rr.C, M=rr.M, s1=rr.s1, s2=rr.s2, b1=rr.b1, b2=rr.b2)
        grid = _grid(300, 260, row["density"], 500 + rr.r)
        want = _oracle_run(300, 260, row["density"], 500 + rr.r, tuple(rule.items()), 4)
        assert_same(run_gpu(cat, kernel, dtype, grid, rule, 4), want, row["name"])


@pytest.mark.parametrize("kernel,dtype", KERNELS, ids=KIDS)
def test_multistate_decay(cat, kernel, dtype):
    """Only state 1 is counted; states 2..C-1 decay (R10 C16, small C, and C =
    128, 200, 255 around the tcgen05 epilogue's two formulations, C <= 128 and
    C > 128)."""
    cases = [(inputs.MULTISTATE_R10_C16, 16), (dict(r=3, C=3, M=0, s1=10, s2=25, b1=9, b2=14), 3),
             (dict(r=16, C=5, M=1, s1=300, s2=700, b1=320, b2=500), 5),
             (dict(r=5, C=128, M=1, s1=3, s2=40, b1=2, b2=30), 128),
             (dict(r=9, C=200, M=0, s1=2, s2=90, b1=1, b2=60), 200),
             (dict(r=2, C=255, M=1, s1=1, s2=9, b1=1, b2=6), 255)]
    for rule, C in cases:
        grid = inputs.uniform_states(290, 310, C, 17 + C)
        want = oracle.step(grid, orule(rule), n_steps=5)
        assert_same(run_gpu(cat, kernel, dtype, grid, rule, 5), want, f"C={C}")


@pytest.mark.parametrize("kernel,dtype", KERNELS, ids=KIDS)
def test_degenerate_shapes(cat, kernel, dtype):
    shapes = [(1, 1), (1, 200), (200, 1), (2, 3), (127, 129), (128, 128), (129, 255), (17, 300), (300, 17)]
    for i, (H, W) in enumerate(shapes):
        for r in (1, 5, 16):
            rule = rule_dict(r, M=0, b=(1, 3 * r))
            grid = inputs.bernoulli(H, W, 0.45, 900 + i)
            want = oracle.step(grid, orule(rule), n_steps=2)
            assert_same(run_gpu(cat, kernel, dtype, grid, rule, 2), want, f"{H}x{W} r={r}")


@pytest.mark.parametrize("kernel,dtype", KERNELS, ids=KIDS)
def test_empty_ranges_and_zero_steps(cat, kernel, dtype):
    grid = _grid(150, 150, 0.5, 3)
    rule = dict(r=2, C=2, M=1, s1=5, s2=4, b1=9, b2=2)  # nothing survives, nothing is born
    assert not run_gpu(cat, kernel, dtype, grid, rule, 1).any()
    assert_same(run_gpu(cat, kernel, dtype, grid, rule, 0), grid, "zero steps")


# --------------------------------------------------- full-size, sampled check
@pytest.mark.parametrize("dtype", ["fp8", "fp16"])
def test_full_16384_one_step_sampled_windows(cat, dtype):
    """16384^2 Bernoulli(0.5), the bench's launch; one step checked on 24 windows
    (interior, edges and corners) recomputed by the oracle from the step's input."""
    import torch
    N = 16384
    grid_host = inputs.bernoulli(N, N, 0.5, 2024)
    rng = np.random.default_rng(0)
    for r in (1, 8, 16):
        rule = rule_dict(r)
        g = cat.Grid(N, N, rule, kernel="tcgen05", dtype=dtype)
        try:
            g.set_state(grid_host)
            g.step(1)
            torch.cuda.synchronize()
            assert g.status() == cat.CAT_OK
            out = g.state_tensor()
            corners = [(0, 0), (0, N - 256), (N - 256, 0), (N - 256, N - 256)]
            spots = corners + [tuple(int(v) for v in rng.integers(0, N - 256, 2)) for _ in range(20)]
            for (y0, x0) in spots:
                ya, xa = max(0, y0 - r), max(0, x0 - r)
                yb, xb = min(N, y0 + 256 + r), min(N, x0 + 256 + r)
                win = grid_host[ya:yb, xa:xb]
                want = oracle.step(win, orule(rule))[y0 - ya:y0 - ya + 256, x0 - xa:x0 - xa + 256]
                got = out[y0:y0 + 256, x0:x0 + 256].cpu().numpy()
                assert_same(got, want, f"r={r} window ({y0},{x0})")
        finally:
            g.close()


# ------------------------------------------------------ failure detection
def test_bounded_wait_reports_timeout_and_context_survives(cat):
    grid = _grid(256, 256, 0.5, 1)
    g = cat.Grid(256, 256, inputs.CONWAY, kernel="tcgen05", dtype="fp8")
    try:
        g.set_state(grid)
        cat.cat_debug_control(g.handle, 2, 20)   # 20 ms limit
        cat.cat_debug_control(g.handle, 1, 1)    # wait on a barrier nothing arrives at
        g.step(1)
        assert g.status() == cat.CAT_ERR_TIMEOUT
        cat.cat_debug_control(g.handle, 1, 0)
        cat.cat_debug_control(g.handle, 2, 2000)
        g.set_state(grid)
        g.step(3)
        assert g.status() == cat.CAT_OK
        want = _oracle_run(256, 256, 0.5, 1, tuple(inputs.CONWAY.items()), 3)
        assert_same(g.get_state(), want, "after timeout")
    finally:
        g.close()


# ------------------------------------------------- workload-scale parity cases
@pytest.mark.parametrize("dtype", ["fp8", "fp16"])
def test_radius_sweep_4096_every_radius(cat, dtype):
    """4096^2 Bernoulli(0.5), the radius-scaled rule (C2 M1) for r = 1..16, 2 steps, full equality."""
    grid = inputs.bernoulli(4096, 4096, 0.5, 4096)
    for r in range(1, 17):
        rule = rule_dict(r, M=1)
        want = _oracle_run(4096, 4096, 0.5, 4096, tuple(rule.items()), 2)
        assert_same(run_gpu(cat, "tcgen05", dtype, grid, rule, 2), want, f"4096^2 r={r}")


def test_cross_dtype_equality_after_many_steps(cat):
    """Every kernel/dtype reaches the same state after 20 steps on 2048^2 (p = 0.35)."""
    grid = inputs.bernoulli(2048, 2048, 0.35, 35)
    for r in (1, 5, 10, 16):
        rule = rule_dict(r, M=1)
        outs = {f"{k}/{d}": run_gpu(cat, k, d, grid, rule, 20) for k, d in KERNELS}
        ref = outs["tcgen05/fp16"]
        for name, o in outs.items():
            assert_same(o, ref, f"r={r} {name} vs tcgen05/fp16")
        # and the oracle agrees after the same 20 steps
        want = oracle.step(grid, orule(rule), n_steps=20)
        assert_same(ref, want, f"r={r} oracle")


def test_multistate_r10_c16_49152_thousand_steps(cat):
    """The multi-state workload at full size: 49152^2, states uniform over
    {0..15}, R10 C16 M1 S150..260 B150..200, FP8 operands (re-encoded window).
    One step is checked against the oracle on 6 windows after steps 1, 2 and 7;
    with ~1/16 of the cells alive (counts ~28 << 150) nothing is born and every
    live cell decays, so the grid is all dead by step 16 and stays dead through
    step 1000."""
    N, C = 49152, 16
    rule = inputs.MULTISTATE_R10_C16
    g = cat.Grid(N, N, rule, kernel="tcgen05", dtype="fp8")
    rng = np.random.default_rng(49152)
    try:
        g.set_state(inputs.uniform_states(N, N, C, 4915))
        done = 0
        for check_at in (1, 2, 7):
            g.step(check_at - 1 - done)
            pos = [tuple(int(v) for v in rng.integers(0, N - 128, 2)) for _ in range(6)]
            pos[0] = (0, N - 128)                       # a corner tile with zero halo on two sides
            st = g.state_tensor()
            befores = []
            for y0, x0 in pos:
                ya, xa = max(0, y0 - 10), max(0, x0 - 10)
                befores.append((ya, xa, st[ya:min(N, y0 + 138), xa:min(N, x0 + 138)].cpu().numpy()))
            g.step(1)
            done = check_at
            assert g.status() == cat.CAT_OK
            st = g.state_tensor()
            for (y0, x0), (ya, xa, win) in zip(pos, befores):
                want = oracle.step(win, orule(rule))[y0 - ya:y0 - ya + 128, x0 - xa:x0 - xa + 128]
                assert_same(st[y0:y0 + 128, x0:x0 + 128].cpu().numpy(), want, f"step {check_at} window ({y0},{x0})")
        g.step(16 - done)
        assert not bool(g.state_tensor().any().item())
        g.step(1000 - 16)
        assert g.status() == cat.CAT_OK
        assert not bool(g.state_tensor().any().item())
    finally:
        g.close()


def test_multistate_r10_c16_windows(cat):
    """R10 C16 M1 S150..260 B150..200 from states uniform over {0..15}, 4096^2.
    One step is checked on 8 windows against the oracle at steps 1, 2, 7 and 14.
    Only ~1/16 of the cells start alive (counts ~28 << 150), so nothing is born,
    every live cell dies and decays: the grid must be all dead after 16 steps."""
    N, C = 4096, 16
    rule = inputs.MULTISTATE_R10_C16
    g = cat.Grid(N, N, rule, kernel="tcgen05", dtype="fp8")
    rng = np.random.default_rng(16)
    try:
        g.set_state(inputs.uniform_states(N, N, C, 1616))
        done = 0
        for check_at in (1, 2, 7, 14):
            g.step(check_at - 1 - done)
            before = g.state_tensor().cpu().numpy().copy()
            g.step(1)
            done = check_at
            after = g.state_tensor().cpu().numpy()
            assert g.status() == cat.CAT_OK
            for _ in range(8):
                y0, x0 = (int(v) for v in rng.integers(0, N - 128, 2))
                ya, xa = max(0, y0 - 10), max(0, x0 - 10)
                win = before[ya:min(N, y0 + 138), xa:min(N, x0 + 138)]
                want = oracle.step(win, orule(rule))[y0 - ya:y0 - ya + 128, x0 - xa:x0 - xa + 128]
                assert_same(after[y0:y0 + 128, x0:x0 + 128], want, f"step {check_at} window ({y0},{x0})")
            if check_at == 1:
                assert int((after >= 2).sum()) > 0 and int((after == 1).sum()) == 0
        g.step(16 - done)
        assert not g.state_tensor().cpu().numpy().any()
    finally:
        g.close()

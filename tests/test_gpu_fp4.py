"""FP4 (e2m1) operands on the tcgen05 kernel vs the CPU oracle, element by element.

The window is re-encoded in shared memory as e2m1 (a state-1 cell is code 1 =
0.5; kind::f8f6f4 reads e2m1 from shared memory as 16 elements packed into the
first 8 bytes of every 16-byte unit) and multiplied by an e2m1 band of ones
held in tensor memory (one element per byte, code in bits 2..5), so pass 1
gives H / 2 exactly.  H <= 33 is not an e2m1 number (the largest is 6), so
pass 2 is the FP8 kernel's: H as e4m3 against the e4m3 band of ones when
2r+1 <= 15 (the e2m1 / e4m3 mix of kind::f8f6f4), else the f16 values H / 2
against an f16 band of 2^-8 (Sec. VI names lower precisions; Sec. V-A argues
exactness for FP16, which both operand sets keep).  Every storage the FP4 kernel
serves (uint8, one bit, four bits per cell) is checked: box counts at every
radius, all-ones and impulse grids (H = 33 and S = 1089 at r = 16), whole
steps of the scaled rules and of the paper's Table IV, multi-state decay,
ragged and degenerate shapes, and the 16384^2 launch on sampled windows.
"""
import numpy as np
import pytest

from oracle import oracle
from paper_2406_17284_gb300 import inputs
from tests import pins

pytestmark = pytest.mark.gpu


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


def orule(d):
    return oracle.Rule(d["r"], d["C"], d["M"], d["s1"], d["s2"], d["b1"], d["b2"])


def assert_same(got, want, what):
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        y, x = bad[0]
        raise AssertionError(f"{what}: {len(bad)} cells differ, first at ({y},{x}): got {got[y, x]} want {want[y, x]}")


STORAGES = ["u8", "bit1", "nib4"]


def store(cat, name):
    return {"u8": cat.STORE_U8, "bit1": cat.STORE_BIT1, "nib4": cat.STORE_NIB4}[name]


def fp4_grid(cat, H, W, rule, storage="u8", **kw):
    return cat.Grid(H, W, rule, kernel="tcgen05", dtype="fp4", storage=store(cat, storage), **kw)


def run(cat, grid, rule, steps, storage="u8", **kw):
    g = fp4_grid(cat, grid.shape[0], grid.shape[1], rule, storage, **kw)
    try:
        g.set_state(grid)
        g.step(steps)
        out = g.get_state()
        assert g.status() == cat.CAT_OK
        return out
    finally:
        g.close()


def table_iv():
    rows = []
    with open(__file__.rsplit("/", 1)[0] + "/golden/ltl_table_iv.txt") as f:
        for ln in f:
            if ln.startswith("#") or not ln.strip():
                continue
            r, C, M, s1, s2, b1, b2 = (int(v) for v in ln.split()[:7])
            rows.append(dict(r=r, C=C, M=M, s1=s1, s2=s2, b1=b1, b2=b2))
    return rows


# ------------------------------------------------------------- box counts
@pytest.mark.parametrize("storage", STORAGES)
def test_box_sums_every_radius(cat, storage):
    grid = inputs.bernoulli(300, 437, 0.5, 41)
    for r in range(1, 17):
        g = fp4_grid(cat, 300, 437, inputs.scaled_rule(r), storage)
        try:
            g.set_state(grid)
            assert_same(g.box_sums(), oracle.box_sums(grid, r), f"{storage} S r={r}")
        finally:
            g.close()


@pytest.mark.parametrize("storage", STORAGES)
def test_box_sums_all_ones_and_impulse(cat, storage):
    """All ones: H = 2r + 1 (33 at r = 16, both e4m3 digits non-zero) and S up
    to 1089; an impulse: a (2r+1)^2 box of ones around each live cell."""
    ones = np.ones((260, 270), np.uint8)
    imp = np.zeros((200, 333), np.uint8)
    imp[100, 129] = imp[0, 0] = imp[199, 332] = 1
    for r in (1, 2, 7, 8, 15, 16):
        for grid in (ones, imp):
            g = fp4_grid(cat, *grid.shape, inputs.scaled_rule(r), storage)
            try:
                g.set_state(grid)
                assert_same(g.box_sums(), oracle.box_sums(grid, r), f"{storage} S r={r}")
            finally:
                g.close()
    assert oracle.box_sums(ones, 16).max() == 1089


def test_multistate_counts_state_one_only(cat):
    """States 0..15: only state 1 is an e2m1 0.5 in the window operand."""
    grid = inputs.uniform_states(260, 301, 16, 5)
    for storage in ("u8", "nib4"):
        for r in (1, 8, 16):
            g = fp4_grid(cat, 260, 301, dict(inputs.MULTISTATE_R10_C16, r=r), storage)
            try:
                g.set_state(grid)
                assert_same(g.box_sums(), oracle.box_sums(grid, r), f"{storage} multi-state S r={r}")
            finally:
                g.close()


# ------------------------------------------------------------------ steps
@pytest.mark.parametrize("storage", STORAGES)
def test_conway_256_100_steps_and_patterns(cat, storage):
    grid = inputs.bernoulli(256, 256, 0.5, 1)
    want = oracle.step(grid, orule(inputs.CONWAY), n_steps=100)
    assert_same(run(cat, grid, inputs.CONWAY, 100, storage), want, f"{storage} conway")
    for name, period, dy, dx in pins.read_conway_patterns():
        g = np.zeros((40, 300), np.uint8)
        inputs.place(g, name, 10, 126)  # straddles a tile boundary
        assert_same(run(cat, g, inputs.CONWAY, period, storage), np.roll(g, (dy, dx), (0, 1)), f"{storage} {name}")


@pytest.mark.parametrize("storage", STORAGES)
def test_scaled_rules_every_radius(cat, storage):
    """The radius-scaled rule, M0 and M1, 3 steps, on a ragged 300 x 437 grid."""
    grid = inputs.bernoulli(300, 437, 0.5, 77)
    for r in range(1, 17):
        for M in (0, 1):
            rule = inputs.scaled_rule(r, M=M)
            want = oracle.step(grid, orule(rule), n_steps=3)
            assert_same(run(cat, grid, rule, 3, storage), want, f"{storage} r={r} M={M}")


@pytest.mark.parametrize("rule", table_iv(), ids=lambda d: f"r{d['r']}")
def test_paper_table_iv_rules(cat, rule):
    for i, (H, W) in enumerate([(200, 300), (65, 1000)]):
        grid = inputs.bernoulli(H, W, 0.3 + 0.2 * i, 500 + i + rule["r"])
        want = oracle.step(grid, orule(rule), n_steps=5)
        for storage in STORAGES:
            assert_same(run(cat, grid, rule, 5, storage), want, f"{storage} {H}x{W}")


@pytest.mark.parametrize("storage", ["u8", "nib4"])
def test_multistate_decay(cat, storage):
    for rule in (dict(r=3, C=5, M=0, s1=10, s2=30, b1=12, b2=25), dict(r=7, C=3, M=1, s1=70, s2=130, b1=75, b2=110),
                 dict(r=16, C=16, M=1, s1=370, s2=630, b1=370, b2=490), dict(inputs.MULTISTATE_R10_C16)):
        g = inputs.bernoulli(300, 437, 0.5, 9)
        u = inputs.uniform_states(300, 437, 16, 10)
        grid = (np.where(u >= 12, u, g) % rule["C"]).astype(np.uint8)
        want = oracle.step(grid, orule(rule), n_steps=4)
        assert_same(run(cat, grid, rule, 4, storage), want, f"{storage} C={rule['C']} r={rule['r']}")


@pytest.mark.parametrize("storage", STORAGES)
def test_degenerate_shapes_and_empty_ranges(cat, storage):
    for i, (H, W) in enumerate([(1, 1), (1, 257), (200, 1), (129, 131), (3, 7), (128, 128), (129, 4100)]):
        for r in (1, 9, 16):
            rule = inputs.scaled_rule(r, M=i % 2)
            grid = inputs.bernoulli(H, W, 0.5, 60 + i + r)
            want = oracle.step(grid, orule(rule), n_steps=2)
            assert_same(run(cat, grid, rule, 2, storage), want, f"{storage} {H}x{W} r={r}")
    grid = inputs.bernoulli(181, 517, 0.5, 3)
    empty = dict(inputs.scaled_rule(12), s1=5, s2=4, b1=0, b2=10 ** 6)   # nothing survives; every dead cell is born
    assert_same(run(cat, grid, empty, 1, storage), oracle.step(grid, orule(empty)), f"{storage} empty ranges")


def test_full_16384_equals_fp8_and_oracle_windows(cat):
    """16384^2, r = 5 and 16: one FP4 step on uint8, one-bit and four-bit
    storage equals the FP8 step cell for cell, and the oracle on sampled
    windows (corners included)."""
    import torch
    N = 16384
    host = inputs.bernoulli(N, N, 0.5, 2024)
    rng = np.random.default_rng(11)
    for r in (5, 16):
        rule = inputs.scaled_rule(r, M=1)
        ref = cat.Grid(N, N, rule, kernel="tcgen05", dtype="fp8")
        try:
            ref.set_state(host)
            ref.step(1)
            want_all = ref.get_state()
        finally:
            ref.close()
        for storage in STORAGES:
            g = fp4_grid(cat, N, N, rule, storage)
            try:
                g.set_state(host)
                g.step(1)
                torch.cuda.synchronize()
                assert g.status() == cat.CAT_OK
                assert_same(g.get_state(), want_all, f"{storage} r={r} vs FP8")
            finally:
                g.close()
        for y0, x0 in [(0, 0), (N - 256, N - 256)] + [tuple(int(v) for v in rng.integers(0, N - 256, 2)) for _ in range(6)]:
            ya, xa = max(0, y0 - r), max(0, x0 - r)
            win = host[ya:min(N, y0 + 256 + r), xa:min(N, x0 + 256 + r)]
            want = oracle.step(win, orule(rule))[y0 - ya:y0 - ya + 256, x0 - xa:x0 - xa + 256]
            assert_same(want_all[y0:y0 + 256, x0:x0 + 256], want, f"r={r} window ({y0},{x0})")


def test_storage_and_dtype_switches_keep_the_state(cat):
    rule = inputs.scaled_rule(9, M=1)
    grid = inputs.bernoulli(333, 270, 0.5, 19)
    g = cat.Grid(333, 270, rule, kernel="tcgen05", dtype="fp8")
    try:
        g.set_state(grid)
        for storage, dtype in ((cat.STORE_U8, cat.DTYPE_FP4_E2M1), (cat.STORE_BIT1, cat.DTYPE_FP4_E2M1),
                               (cat.STORE_NIB4, cat.DTYPE_FP4_E2M1), (cat.STORE_U8, cat.DTYPE_FP8_E4M3)):
            cat.cat_set_options(g.handle, cat.KERNEL_TCGEN05, dtype, storage, 1)
            g.storage = storage
            g.step(1)
        assert_same(g.get_state(), oracle.step(grid, orule(rule), n_steps=4), "four steps across switches")
    finally:
        g.close()


def test_unsupported(cat):
    for rule, kw in ((inputs.vn_scaled_rule(4), {}),                       # the von Neumann cross
                     (inputs.scaled_rule(17), {}),                         # r > 16 (96 x 96 tile)
                     (inputs.scaled_rule(4), dict(steps_per_launch=2)),    # several steps per launch
                     (inputs.scaled_rule(4), dict(tile=96))):
        with pytest.raises(cat.CatError) as e:
            cat.Grid(64, 64, rule, kernel="tcgen05", dtype="fp4", **kw)
        assert e.value.code == cat.CAT_ERR_UNSUPPORTED, (rule, kw)
    with pytest.raises(cat.CatError) as e:
        cat.Grid(64, 64, inputs.scaled_rule(4), kernel="mma_sync", dtype="fp4")
    assert e.value.code == cat.CAT_ERR_UNSUPPORTED


def test_batch_step_steps_fp4_instances_one_by_one(cat):
    rules = [inputs.scaled_rule(r, M=r % 2) for r in (1, 6, 12, 16)]
    grids = [inputs.bernoulli(100 + 37 * i, 300 - 41 * i, 0.45, 70 + i) for i in range(4)]
    gs = [fp4_grid(cat, *g.shape, rl, ("u8", "bit1", "nib4", "u8")[i]) for i, (g, rl) in enumerate(zip(grids, rules))]
    try:
        for g, host in zip(gs, grids):
            g.set_state(host)
        cat.cat_batch_step([g.handle for g in gs], 3)
        for g, host, rl in zip(gs, grids, rules):
            assert g.status() == cat.CAT_OK
            assert_same(g.get_state(), oracle.step(host, orule(rl), n_steps=3), f"batched r={rl['r']}")
    finally:
        for g in gs:
            g.close()


def test_auto_dtype_takes_fp4_on_four_bit_storage(cat):
    """CAT_DTYPE_AUTO: FP4 operands on four-bit storage (two-state and
    multi-state rules), FP8 on uint8 and one-bit storage; the chosen operands
    step like the oracle."""
    cases = [(inputs.scaled_rule(12, M=1), cat.STORE_NIB4, cat.DTYPE_FP4_E2M1),
             (dict(inputs.MULTISTATE_R10_C16), cat.STORE_NIB4, cat.DTYPE_FP4_E2M1),
             (dict(r=3, C=5, M=0, s1=10, s2=30, b1=12, b2=25), cat.STORE_NIB4, cat.DTYPE_FP4_E2M1),
             (inputs.scaled_rule(12, M=1), cat.STORE_U8, cat.DTYPE_FP8_E4M3),
             (dict(inputs.MULTISTATE_R10_C16), cat.STORE_U8, cat.DTYPE_FP8_E4M3),
             (inputs.scaled_rule(12, M=1), cat.STORE_BIT1, cat.DTYPE_FP8_E4M3)]
    for i, (rule, storage, want_dtype) in enumerate(cases):
        H, W = 210 + 13 * i, 333 - 17 * i
        if rule["C"] > 2:
            host = (inputs.uniform_states(H, W, rule["C"], 90 + i) * (inputs.bernoulli(H, W, 0.3, 95 + i) == 0)
                    + inputs.bernoulli(H, W, 0.3, 95 + i)).astype(np.uint8) % rule["C"]
        else:
            host = inputs.bernoulli(H, W, 0.5, 90 + i)
        g = cat.Grid(H, W, rule, kernel="tcgen05", dtype="auto", storage=storage)
        try:
            assert cat.cat_get_options(g.handle)["dtype"] == want_dtype, (rule, storage)
            g.set_state(host)
            g.step(3)
            assert g.status() == cat.CAT_OK
            assert_same(g.get_state(), oracle.step(host, orule(rule), n_steps=3), f"auto dtype case {i}")
        finally:
            g.close()

"""Four-bit storage (CAT_STORE_NIB4) vs the CPU oracle, element by element.

The grid lives in HBM as two cells per byte (the even x in the low nibble);
the step kernel unpacks its windows into state-1 flags (the FP8 operand) in
shared memory and applies the multi-state rule to the unpacked centre states
in its epilogue, packing the next states again.  Multi-state rules follow
the decay reading of Sec. V-A's notation (state 1 fails survival -> 2, then
+1 per step to 0 after C - 1).  The packed bytes are also compared with the
nibble packing written out in numpy, and the nibble past an odd W must stay 0.
"""
import numpy as np
import pytest

from oracle import oracle
from paper_2406_17284_gb300 import inputs

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


def nib_packed(grid):
    H, W = grid.shape
    g = np.zeros((H, W + (W & 1)), np.uint8)
    g[:, :W] = grid
    return (g[:, 0::2] | (g[:, 1::2] << 4)).astype(np.uint8)


def nib_grid(cat, H, W, rule):
    return cat.Grid(H, W, rule, kernel="tcgen05", dtype="fp8", storage=cat.STORE_NIB4)


def live_c16(H, W, seed):
    """States 0/1 Bernoulli(0.5) plus a sprinkle of decaying states 2..15."""
    g = inputs.bernoulli(H, W, 0.5, seed)
    u = inputs.uniform_states(H, W, 16, seed + 1)
    return np.where(u >= 12, u, g).astype(np.uint8)


def test_round_trip_and_packed_layout(cat):
    for H, W in ((1, 1), (3, 7), (129, 255), (300, 437), (256, 1024)):
        grid = inputs.uniform_states(H, W, 16, H + W)
        g = nib_grid(cat, H, W, dict(inputs.MULTISTATE_R10_C16))
        try:
            g.set_state(grid)
            assert_same(g.get_state(), grid, f"round trip {H}x{W}")
            assert_same(g.state_tensor().cpu().numpy(), nib_packed(grid), f"packing {H}x{W}")
        finally:
            g.close()


RULES = [
    dict(inputs.MULTISTATE_R10_C16),
    dict(r=3, C=5, M=0, s1=10, s2=30, b1=12, b2=25),
    dict(r=7, C=3, M=1, s1=70, s2=130, b1=75, b2=110),
    dict(r=16, C=16, M=1, s1=370, s2=630, b1=370, b2=490),
    inputs.scaled_rule(9, M=0),   # C = 2 on four-bit storage
    dict(inputs.CONWAY),
]


@pytest.mark.parametrize("rule", RULES, ids=lambda d: f"r{d['r']}C{d['C']}")
def test_steps_vs_oracle_on_ragged_shapes(cat, rule):
    for i, (H, W) in enumerate([(300, 437), (129, 131), (1, 257), (200, 1)]):
        C = rule["C"]
        grid = live_c16(H, W, 70 + i) % C if C > 2 else inputs.bernoulli(H, W, 0.4, 70 + i)
        grid = grid.astype(np.uint8)
        g = nib_grid(cat, H, W, rule)
        try:
            g.set_state(grid)
            g.step(4)
            assert g.status() == cat.CAT_OK
            assert_same(g.get_state(), oracle.step(grid, orule(rule), n_steps=4), f"{H}x{W}")
            # nothing written past W (an odd W leaves the last byte's high nibble 0)
            if W & 1:
                assert int((g.state_tensor()[:, -1] >> 4).max().item()) == 0
        finally:
            g.close()


def test_box_sums_count_state_one_only(cat):
    grid = inputs.uniform_states(260, 301, 16, 5)
    for r in (1, 8, 16):
        g = nib_grid(cat, 260, 301, dict(inputs.MULTISTATE_R10_C16, r=r))
        try:
            g.set_state(grid)
            assert_same(g.box_sums(), oracle.box_sums(grid, r), f"S r={r}")
        finally:
            g.close()


def test_storage_switches_keep_the_state(cat):
    rule = dict(inputs.MULTISTATE_R10_C16)
    grid = live_c16(333, 270, 9)
    g = cat.Grid(333, 270, rule, kernel="tcgen05", dtype="fp8")
    try:
        g.set_state(grid)
        cat.cat_set_options(g.handle, cat.KERNEL_TCGEN05, cat.DTYPE_FP8_E4M3, cat.STORE_NIB4, 1)
        g.storage = cat.STORE_NIB4
        assert_same(g.get_state(), grid, "U8 -> NIB4")
        g.step(3)
        want = oracle.step(grid, orule(rule), n_steps=3)
        cat.cat_set_options(g.handle, cat.KERNEL_TCGEN05, cat.DTYPE_FP8_E4M3, cat.STORE_U8, 1)
        g.storage = cat.STORE_U8
        assert_same(g.get_state(), want, "NIB4 -> U8")
        g.step(2)
        assert_same(g.get_state(), oracle.step(grid, orule(rule), n_steps=5), "steps after the switch")
    finally:
        g.close()
    two = inputs.bernoulli(200, 300, 0.5, 3)
    conway = dict(inputs.CONWAY)
    h = cat.Grid(200, 300, conway, kernel="tcgen05", dtype="fp8", storage=cat.STORE_NIB4)
    try:
        h.set_state(two)
        cat.cat_set_options(h.handle, cat.KERNEL_TCGEN05, cat.DTYPE_FP8_E4M3, cat.STORE_BIT1, 1)   # NIB4 -> BIT1
        h.storage = cat.STORE_BIT1
        h.step(2)
        cat.cat_set_options(h.handle, cat.KERNEL_TCGEN05, cat.DTYPE_FP8_E4M3, cat.STORE_NIB4, 1)   # BIT1 -> NIB4
        h.storage = cat.STORE_NIB4
        h.step(2)
        assert_same(h.get_state(), oracle.step(two, orule(conway), n_steps=4), "BIT1 <-> NIB4")
    finally:
        h.close()


def test_full_16384_multistate_windows(cat):
    """16384^2, R10 C16 from a live start, 3 steps; one step checked on 12
    windows (corners included) recomputed from the state before it."""
    N = 16384
    rule = dict(inputs.MULTISTATE_R10_C16)
    host = live_c16(N, N, 16384)
    g = nib_grid(cat, N, N, rule)
    rng = np.random.default_rng(4)
    try:
        g.set_state(host)
        g.step(2)
        before = g.get_state()
        g.step(1)
        assert g.status() == cat.CAT_OK
        after = g.get_state()
        counts = np.bincount(after[::64, ::64].ravel(), minlength=16)
        assert counts[1] > 0 and counts[2:].sum() > 0
        for y0, x0 in [(0, 0), (0, N - 192), (N - 192, 0), (N - 192, N - 192)] + \
                [tuple(int(v) for v in rng.integers(0, N - 192, 2)) for _ in range(8)]:
            ya, xa = max(0, y0 - 10), max(0, x0 - 10)
            win = before[ya:min(N, y0 + 202), xa:min(N, x0 + 202)]
            want = oracle.step(win, orule(rule))[y0 - ya:y0 - ya + 192, x0 - xa:x0 - xa + 192]
            assert_same(after[y0:y0 + 192, x0:x0 + 192], want, f"window ({y0},{x0})")
    finally:
        g.close()


def test_unsupported(cat):
    for rule, kw in ((dict(inputs.MULTISTATE_R10_C16, C=17), {}),
                     (dict(inputs.MULTISTATE_R10_C16, r=20), {}),
                     (dict(inputs.MULTISTATE_R10_C16), dict(boundary=cat.BOUNDARY_PERIODIC)),
                     (dict(inputs.MULTISTATE_R10_C16), dict(kernel="tcgen05", dtype="fp16")),
                     (dict(inputs.MULTISTATE_R10_C16), dict(kernel="tcgen05", dtype="fp8", steps_per_launch=2))):
        with pytest.raises(cat.CatError) as e:
            cat.Grid(64, 64, rule, storage=cat.STORE_NIB4, **kw)
        assert e.value.code == cat.CAT_ERR_UNSUPPORTED, (rule, kw)

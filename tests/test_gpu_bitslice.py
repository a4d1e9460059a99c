"""The bit-sliced CUDA-core kernel (CAT_KERNEL_BITSLICE, one-bit storage,
r <= 5) vs the CPU oracle, element by element.

The kernel adds the counts of 32 cells per word as bit planes; every case
below checks the funnel-shifted neighbours across word and warp boundaries,
the grid edges (zero halo, ragged W), the bit-sliced adders (counts compared
directly), the bit-serial range tests and the M flag.  Paper: Sec. V-B (the
packed-cell regime at r <= 2), Sec. V-A (Table IV rules, notation).
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


def table_iv(max_r):
    rows = []
    with open(__file__.rsplit("/", 1)[0] + "/golden/ltl_table_iv.txt") as f:
        for ln in f:
            if ln.startswith("#") or not ln.strip():
                continue
            r, C, M, s1, s2, b1, b2 = (int(v) for v in ln.split()[:7])
            if r <= max_r:
                rows.append(dict(r=r, C=C, M=M, s1=s1, s2=s2, b1=b1, b2=b2))
    return rows


def grid_of(cat, H, W, rule):
    return cat.Grid(H, W, rule, kernel="bitslice", storage=cat.STORE_BIT1)


def run(cat, grid, rule, steps):
    g = grid_of(cat, grid.shape[0], grid.shape[1], rule)
    try:
        g.set_state(grid)
        g.step(steps)
        out = g.get_state()
        assert g.status() == cat.CAT_OK
        return out
    finally:
        g.close()


SHAPES = [(1, 1), (1, 33), (3, 31), (5, 32), (77, 100), (40, 1025), (130, 8200), (33, 64)]


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5])
def test_counts(cat, r):
    for i, (H, W) in enumerate(SHAPES):
        grid = inputs.bernoulli(H, W, 0.5, 50 + 7 * i + r)
        g = grid_of(cat, H, W, inputs.scaled_rule(r))
        try:
            g.set_state(grid)
            assert_same(g.box_sums(), oracle.box_sums(grid, r), f"S r={r} {H}x{W}")
            ones = np.ones((H, W), np.uint8)
            g.set_state(ones)
            assert_same(g.box_sums(), oracle.box_sums(ones, r), f"all-ones r={r} {H}x{W}")
        finally:
            g.close()


def test_conway_patterns_and_100_steps(cat):
    grid = inputs.bernoulli(256, 256, 0.5, 2024)
    assert_same(run(cat, grid, inputs.CONWAY, 100), oracle.step(grid, orule(inputs.CONWAY), n_steps=100), "Conway 100")
    pat = np.zeros((64, 96), np.uint8)
    inputs.place(pat, "block", 2, 2)
    inputs.place(pat, "blinker", 10, 30)
    inputs.place(pat, "glider", 20, 28)      # crosses the word boundary at x = 32
    after4 = run(cat, pat, inputs.CONWAY, 4)
    assert_same(after4, oracle.step(pat, orule(inputs.CONWAY), n_steps=4), "patterns")
    # the glider moved by (1, 1), the block stayed, the blinker is back
    assert after4[2:4, 2:4].all() and after4[10, 30:33].all()
    assert after4[21, 30] == 1 and after4[23, 29:32].all()


@pytest.mark.parametrize("rule", table_iv(5), ids=lambda d: f"r{d['r']}")
def test_table_iv_rules(cat, rule):
    for i, (H, W) in enumerate([(200, 300), (65, 1000), (1, 70)]):
        grid = inputs.bernoulli(H, W, 0.3 + 0.1 * i, 300 + i + rule["r"])
        assert_same(run(cat, grid, rule, 5), oracle.step(grid, orule(rule), n_steps=5), f"{H}x{W}")


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("M", [0, 1])
def test_scaled_rules_and_empty_ranges(cat, r, M):
    grid = inputs.bernoulli(181, 517, 0.5, 10 * r + M)
    rule = inputs.scaled_rule(r, M)
    assert_same(run(cat, grid, rule, 6), oracle.step(grid, orule(rule), n_steps=6), f"scaled r={r} M={M}")
    empty = dict(rule, s1=5, s2=4, b1=0, b2=10 ** 6)      # nothing survives; every dead cell is born
    assert_same(run(cat, grid, empty, 1), oracle.step(grid, orule(empty), n_steps=1), "empty survival range")


def test_full_16384_equals_tcgen05_bits_and_oracle_windows(cat):
    import torch
    N = 16384
    host = inputs.bernoulli(N, N, 0.5, 2024)
    rng = np.random.default_rng(5)
    for r in (1, 2):
        rule = inputs.scaled_rule(r, M=1)
        a = grid_of(cat, N, N, rule)
        b = cat.Grid(N, N, rule, kernel="tcgen05", dtype="fp8", storage=cat.STORE_BIT1)
        try:
            a.set_state(host)
            b.set_state(host)
            a.step(2)
            b.step(2)
            torch.cuda.synchronize()
            assert a.status() == cat.CAT_OK and b.status() == cat.CAT_OK
            assert torch.equal(a.state_tensor(), b.state_tensor()), f"r={r}: bit-sliced and tcgen05 packed rows differ"
            out = a.get_state()
            for y0, x0 in [(0, 0), (N - 128, N - 128)] + [tuple(int(v) for v in rng.integers(0, N - 128, 2))
                                                          for _ in range(6)]:
                ya, xa = max(0, y0 - 2 * r), max(0, x0 - 2 * r)
                win = host[ya:min(N, y0 + 128 + 2 * r), xa:min(N, x0 + 128 + 2 * r)]
                want = oracle.step(win, orule(rule), n_steps=2)[y0 - ya:y0 - ya + 128, x0 - xa:x0 - xa + 128]
                assert_same(out[y0:y0 + 128, x0:x0 + 128], want, f"r={r} window ({y0},{x0})")
        finally:
            a.close()
            b.close()


def test_unsupported(cat):
    for rule, kw in ((inputs.scaled_rule(6), dict(storage=cat.STORE_BIT1)),
                     (inputs.scaled_rule(2), dict(storage=cat.STORE_U8)),
                     (inputs.vn_scaled_rule(2), dict(storage=cat.STORE_U8))):
        with pytest.raises(cat.CatError) as e:
            cat.Grid(64, 64, rule, kernel="bitslice", **kw)
        assert e.value.code == cat.CAT_ERR_UNSUPPORTED, (rule, kw)


@pytest.mark.parametrize("r,k", [(1, 2), (1, 3), (1, 8), (2, 4), (4, 2), (5, 1)])
def test_temporal_blocking_vs_oracle(cat, r, k):
    """k steps per launch on tiles kept in shared memory (a k r-cell stale
    halo): shapes that cross block tiles (126 words = 4032 cells wide, 32 rows
    high) and grid edges, step counts that do and do not divide by k."""
    rule = inputs.scaled_rule(r, M=r % 2)
    for i, (H, W) in enumerate([(200, 4100), (33, 8100), (70, 31), (1, 300), (129, 4032)]):
        grid = inputs.bernoulli(H, W, 0.5, 900 + 10 * r + i)
        g = cat.Grid(H, W, rule, kernel="bitslice", storage=cat.STORE_BIT1, steps_per_launch=k)
        try:
            g.set_state(grid)
            g.step(2 * k + 1)
            assert g.status() == cat.CAT_OK
            assert_same(g.get_state(), oracle.step(grid, orule(rule), n_steps=2 * k + 1), f"{H}x{W} r={r} k={k}")
            assert not np.unpackbits(g.state_tensor().cpu().numpy(), axis=1, bitorder="little")[:, W:].any()
        finally:
            g.close()


def test_temporal_blocking_conway_and_limits(cat):
    grid = inputs.bernoulli(1024, 1024, 0.5, 77)
    g = cat.Grid(1024, 1024, inputs.CONWAY, kernel="bitslice", storage=cat.STORE_BIT1, steps_per_launch=8)
    try:
        g.set_state(grid)
        g.step(100)
        assert_same(g.get_state(), oracle.step(grid, orule(inputs.CONWAY), n_steps=100), "Conway 100, k = 8")
    finally:
        g.close()
    with pytest.raises(cat.CatError) as e:
        cat.Grid(64, 64, inputs.scaled_rule(3), kernel="bitslice", storage=cat.STORE_BIT1, steps_per_launch=3)
    assert e.value.code == cat.CAT_ERR_UNSUPPORTED      # k r = 9 > 8

"""Radii 17..32 vs the CPU oracle, cell by cell.

Beyond the fragment size the paper extends its scheme with a second halo
fragment and five band fragments per reduction (Sec. VII); the FP16 fragment
kernel does that, with FP32 accumulation in step 2 since the counts reach
65^2 = 4225.  The tcgen05 kernel serves these radii on 128 x 128 output
tiles inside a 192 x 192 window (a 32-cell halo; e4m3 operands, the
horizontal sums split into H & 15 and H >> 4 against a band of ones and a
band of 16s, f32 accumulation in pass 2), which CAT_KERNEL_AUTO picks for
two-state rules, or on 96 x 96 tiles inside the 160 x 160 window
(cat_set_tile(96, 96)).  The CUDA-core stencil serves these radii too (and
the simplified von Neumann cross).  cat_set_tile also puts radii up to 16 on
the 96 x 96 tile or the 192-row window, and short-window radii on the full
window.
"""
import numpy as np
import pytest

from oracle import oracle
from paper_2406_17284_gb300 import inputs

pytestmark = pytest.mark.gpu

KERNELS = [("tcgen05", "fp8"), ("tcgen05-96", "fp8"), ("mma_sync", "fp16"), ("stencil", "auto"), ("runsum", "auto"),
           ("auto", "auto")]
KIDS = ["tcgen05-fp8", "tcgen05-fp8-tile96", "mma_sync-fp16", "stencil", "runsum", "auto"]


def grid_of(cat, H, W, rule, kernel, dtype):
    """A Grid; "tcgen05-96" is the tcgen05 kernel on the 96 x 96 tile."""
    if kernel == "tcgen05-96":
        return cat.Grid(H, W, rule, kernel="tcgen05", dtype=dtype, tile=96)
    return cat.Grid(H, W, rule, kernel=kernel, dtype=dtype)
RADII = (17, 20, 24, 31, 32)


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
    return oracle.Rule(d["r"], d["C"], d["M"], d["s1"], d["s2"], d["b1"], d["b2"], d.get("nbhd", "M"))


def assert_same(got, want, what):
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        y, x = bad[0]
        raise AssertionError(f"{what}: {len(bad)} cells differ, first at ({y},{x}): got {got[y, x]} want {want[y, x]}")


def run(cat, kernel, dtype, grid, rule, steps):
    g = grid_of(cat, grid.shape[0], grid.shape[1], rule, kernel, dtype)
    try:
        g.set_state(grid)
        g.step(steps)
        out = g.get_state()
        assert g.status() == cat.CAT_OK
        return out
    finally:
        g.close()


@pytest.mark.parametrize("kernel,dtype", KERNELS, ids=KIDS)
def test_counts(cat, kernel, dtype):
    grid = inputs.bernoulli(300, 437, 0.5, 17)
    ones = np.ones((200, 230), np.uint8)
    for r in RADII:
        for g_ in (grid, ones):
            g = grid_of(cat, *g_.shape, inputs.scaled_rule(r), kernel, dtype)
            try:
                g.set_state(g_)
                assert_same(g.box_sums(), oracle.box_sums(g_, r), f"S r={r}")
            finally:
                g.close()
    assert oracle.box_sums(ones, 32)[100, 100] == 65 * 65


@pytest.mark.parametrize("kernel,dtype", KERNELS, ids=KIDS)
def test_steps(cat, kernel, dtype):
    """The radius-scaled rule, M0 and M1, 3 steps on ragged shapes."""
    for i, (H, W) in enumerate([(384, 523), (130, 70), (1, 300), (257, 1)]):
        for r in RADII:
            rule = inputs.scaled_rule(r, M=(r + i) % 2)
            grid = inputs.bernoulli(H, W, 0.5, 1000 + 37 * i + r)
            want = oracle.step(grid, orule(rule), n_steps=3)
            assert_same(run(cat, kernel, dtype, grid, rule, 3), want, f"{H}x{W} r={r}")


def test_multistate_and_cross(cat):
    """C > 2 on the fragment kernel and the stencil; the simplified von Neumann
    cross with r > 16 on the stencil (AUTO picks it)."""
    rule = dict(r=20, C=6, M=1, s1=300, s2=900, b1=350, b2=700)
    grid = inputs.uniform_states(260, 300, 6, 77)
    want = oracle.step(grid, orule(rule), n_steps=4)
    assert_same(run(cat, "mma_sync", "fp16", grid, rule, 4), want, "C=6 fragment")
    assert_same(run(cat, "stencil", "auto", grid, rule, 4), want, "C=6 stencil")
    assert_same(run(cat, "runsum", "auto", grid, rule, 4), want, "C=6 running sums")
    cross = inputs.vn_scaled_rule(28)
    g2 = inputs.bernoulli(300, 280, 0.5, 78)
    want = oracle.step(g2, orule(cross), n_steps=3)
    assert_same(run(cat, "auto", "auto", g2, cross, 3), want, "cross r=28")


def test_unsupported(cat):
    rule = inputs.scaled_rule(20)
    for kernel, dtype in (("tcgen05", "fp16"), ("mma_sync", "int8")):
        with pytest.raises(cat.CatError) as e:
            cat.Grid(64, 64, rule, kernel=kernel, dtype=dtype)
        assert e.value.code == cat.CAT_ERR_UNSUPPORTED, (kernel, dtype)
    for bad in (dict(rule=inputs.scaled_rule(20, C=3)), dict(rule=rule, steps_per_launch=2)):
        with pytest.raises(cat.CatError) as e:
            cat.Grid(64, 64, bad["rule"], kernel="tcgen05", dtype="fp8",
                     steps_per_launch=bad.get("steps_per_launch", 1))
        assert e.value.code == cat.CAT_ERR_UNSUPPORTED, bad
    g = cat.Grid(64, 64, rule, kernel="tcgen05", dtype="fp8")
    try:
        for args, code in (((128, 128, 160), cat.CAT_ERR_UNSUPPORTED), ((0, 0, 160), cat.CAT_ERR_UNSUPPORTED),
                           ((64, 64, 0), cat.CAT_ERR_INVALID_ARG), ((96, 96, 150), cat.CAT_ERR_INVALID_ARG),
                           ((96, 96, 144), cat.CAT_ERR_UNSUPPORTED), ((96, 96, 192), cat.CAT_ERR_UNSUPPORTED),
                           ((128, 128, 200), cat.CAT_ERR_INVALID_ARG)):
            with pytest.raises(cat.CatError) as e:
                cat.cat_set_tile(g.handle, *args)
            assert e.value.code == code, args
    finally:
        g.close()
    with pytest.raises(cat.CatError) as e:
        cat.Grid(64, 64, inputs.vn_scaled_rule(20), kernel="mma_sync", dtype="fp16")
    assert e.value.code == cat.CAT_ERR_UNSUPPORTED
    for kw in (dict(boundary=cat.BOUNDARY_PERIODIC), dict(storage=cat.STORE_BIT1)):
        with pytest.raises(cat.CatError) as e:
            cat.Grid(64, 64, rule, **kw)
        assert e.value.code == cat.CAT_ERR_UNSUPPORTED, kw


def test_full_4096_sampled_windows(cat):
    """4096^2 Bernoulli(0.5), r = 20 (f16 pass 2), 24 and 32, two steps of the
    tcgen05 192-row window (several tiles per CTA) checked on 12 windows
    (corners included) and equal to the stencil, the fragment kernel and the
    96 x 96 tile everywhere."""
    import torch
    N = 4096
    host = inputs.bernoulli(N, N, 0.5, 4242)
    d = torch.from_numpy(host).cuda()
    rng = np.random.default_rng(3)
    for r in (20, 24, 32):
        rule = inputs.scaled_rule(r)
        a = cat.Grid(N, N, rule, kernel="tcgen05", dtype="fp8")
        b = cat.Grid(N, N, rule, kernel="stencil", dtype="auto")
        c = cat.Grid(N, N, rule, kernel="mma_sync", dtype="fp16")
        a96 = cat.Grid(N, N, rule, kernel="tcgen05", dtype="fp8", tile=96)
        try:
            for g in (a, b, c, a96):
                g.set_state(d)
                g.step(2)
            torch.cuda.synchronize()
            assert all(g.status() == cat.CAT_OK for g in (a, b, c, a96))
            out = a.state_tensor()
            assert int((out != b.state_tensor()).sum()) == 0, f"r={r}: tcgen05 192-row window and stencil differ"
            assert int((out != c.state_tensor()).sum()) == 0, f"r={r}: tcgen05 192-row window and fragment kernel differ"
            assert int((out != a96.state_tensor()).sum()) == 0, f"r={r}: 192-row window and 96 x 96 tile differ"
            spots = [(0, 0), (0, N - 200), (N - 200, 0), (N - 200, N - 200)] + \
                [tuple(int(v) for v in rng.integers(0, N - 200, 2)) for _ in range(8)]
            for (y0, x0) in spots:
                ya, xa = max(0, y0 - 2 * r), max(0, x0 - 2 * r)
                yb, xb = min(N, y0 + 200 + 2 * r), min(N, x0 + 200 + 2 * r)
                want = oracle.step(host[ya:yb, xa:xb], orule(rule), n_steps=2)[y0 - ya:y0 - ya + 200, x0 - xa:x0 - xa + 200]
                assert_same(out[y0:y0 + 200, x0:x0 + 200].cpu().numpy(), want, f"r={r} window ({y0},{x0})")
        finally:
            a.close()
            b.close()
            c.close()
            a96.close()


@pytest.mark.parametrize("r", [1, 5, 8, 13, 16])
def test_wide_tile_for_small_radii(cat, r):
    """cat_set_tile(96, 96) on radii up to 16: counts and 3 steps vs the oracle."""
    grid = inputs.bernoulli(301, 389, 0.45, 900 + r)
    rule = inputs.scaled_rule(r, M=r % 2)
    g = cat.Grid(301, 389, rule, kernel="tcgen05", dtype="fp8", tile=96)
    try:
        g.set_state(grid)
        assert_same(g.box_sums(), oracle.box_sums(grid, r), f"S r={r}")
        g.step(3)
        assert g.status() == cat.CAT_OK
        assert_same(g.get_state(), oracle.step(grid, orule(rule), n_steps=3), f"steps r={r}")
    finally:
        g.close()


@pytest.mark.parametrize("r", [1, 4, 7])
def test_full_window_for_short_window_radii(cat, r):
    """cat_set_tile(0, 0, 160): radii up to 7 on the 160-row window (the
    standard kernel with its separate D1 and D2 regions) vs the oracle."""
    grid = inputs.bernoulli(333, 270, 0.5, 700 + r)
    rule = inputs.scaled_rule(r, M=(r + 1) % 2)
    g = cat.Grid(333, 270, rule, kernel="tcgen05", dtype="fp8", window=160)
    try:
        g.set_state(grid)
        g.step(3)
        assert g.status() == cat.CAT_OK
        assert_same(g.get_state(), oracle.step(grid, orule(rule), n_steps=3), f"r={r}")
    finally:
        g.close()


@pytest.mark.parametrize("r", [1, 5, 8, 13, 16])
def test_big_window_for_small_radii(cat, r):
    """cat_set_tile(0, 0, 192) on radii up to 16: the 128 x 128 tile in the
    192 x 192 window, counts and 3 steps vs the oracle on a ragged shape."""
    grid = inputs.bernoulli(301, 389, 0.45, 950 + r)
    rule = inputs.scaled_rule(r, M=(r + 1) % 2)
    g = cat.Grid(301, 389, rule, kernel="tcgen05", dtype="fp8", window=192)
    try:
        opts = cat.cat_get_options(g.handle)
        assert (opts["tile"], opts["window"]) == (128, 192)
        g.set_state(grid)
        assert_same(g.box_sums(), oracle.box_sums(grid, r), f"S r={r}")
        g.step(3)
        assert g.status() == cat.CAT_OK
        assert_same(g.get_state(), oracle.step(grid, orule(rule), n_steps=3), f"steps r={r}")
    finally:
        g.close()


def test_r_above_16_options_and_edges(cat):
    """Radii above 16 take the 192-row window by default (tile 128) and the
    96 x 96 tile on request; both agree with the oracle on tiny, one-row,
    one-column and tile-boundary shapes, all-ones grids (S = 2025 at r = 22,
    the largest count the f16 pass 2 holds, 2209 at r = 23, 4225 at r = 32)
    and an impulse."""
    rule = inputs.scaled_rule(32, M=1)
    g = cat.Grid(64, 64, rule, kernel="tcgen05", dtype="fp8")
    try:
        opts = cat.cat_get_options(g.handle)
        assert (opts["tile"], opts["window"]) == (128, 192)
        cat.cat_set_tile(g.handle, 96, 96, 0)
        opts = cat.cat_get_options(g.handle)
        assert (opts["tile"], opts["window"]) == (96, 0)
    finally:
        g.close()
    imp = np.zeros((260, 300), np.uint8)
    imp[130, 150] = 1
    shapes = [inputs.bernoulli(5, 7, 0.5, 1), inputs.bernoulli(1, 513, 0.5, 2), inputs.bernoulli(513, 1, 0.5, 3),
              inputs.bernoulli(128, 256, 0.5, 4), inputs.bernoulli(129, 257, 0.5, 5), np.ones((200, 230), np.uint8), imp]
    for tile in (0, 96):
        for i, grid in enumerate(shapes):
            for r in (17, 22, 23, 32):   # 22 / 23: the last f16 and first f32 pass 2 of the 192-row window
                rl = inputs.scaled_rule(r, M=i % 2)
                g = cat.Grid(*grid.shape, rl, kernel="tcgen05", dtype="fp8", tile=tile)
                try:
                    g.set_state(grid)
                    assert_same(g.box_sums(), oracle.box_sums(grid, r), f"S tile={tile} {grid.shape} r={r}")
                    g.step(2)
                    assert g.status() == cat.CAT_OK
                    assert_same(g.get_state(), oracle.step(grid, orule(rl), n_steps=2), f"tile={tile} {grid.shape} r={r}")
                finally:
                    g.close()

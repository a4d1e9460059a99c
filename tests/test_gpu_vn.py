"""Simplified von Neumann neighbourhood (Eq. 3) vs the CPU oracle, cell by cell.

The count of a cell is the sum over the vertical and the horizontal segment of
half-length r through it, the centre counted on both (R = Pi x Lambda + H).
The tcgen05 kernel accumulates both band products in one tensor-memory
region (FP8 operands, two-state rules); the paper-style fragment kernel (FP16
wmma) starts its second step from F^H as the MMA's C operand; the CUDA-core
stencil serves every C.
Both are compared with the oracle on counts and on whole steps, at sizes that
span several tiles with ragged tails, on the degenerate shapes, with the
periodic boundary, and on the full 16384^2 launch through sampled windows.
"""
import functools

import numpy as np
import pytest

from oracle import oracle
from paper_2406_17284_gb300 import inputs

pytestmark = pytest.mark.gpu

KERNELS = [("tcgen05", "fp8"), ("mma_sync", "fp16"), ("stencil", "auto")]
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


def orule(d):
    return oracle.Rule(d["r"], d["C"], d["M"], d["s1"], d["s2"], d["b1"], d["b2"], d.get("nbhd", "M"))


@functools.lru_cache(maxsize=None)
def _grid(H, W, p, seed):
    return inputs.bernoulli(H, W, p, seed)


def assert_same(got, want, what):
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        y, x = bad[0]
        raise AssertionError(f"{what}: {len(bad)} cells differ, first at ({y},{x}): got {got[y, x]} want {want[y, x]}")


def run(cat, kernel, dtype, grid, rule, steps, boundary=0):
    g = cat.Grid(grid.shape[0], grid.shape[1], rule, kernel=kernel, dtype=dtype, boundary=boundary)
    try:
        g.set_state(grid)
        g.step(steps)
        out = g.get_state()
        assert g.status() == cat.CAT_OK
        return out
    finally:
        g.close()


def sums(cat, kernel, dtype, grid, rule, boundary=0):
    g = cat.Grid(grid.shape[0], grid.shape[1], rule, kernel=kernel, dtype=dtype, boundary=boundary)
    try:
        g.set_state(grid)
        return g.box_sums()
    finally:
        g.close()


@pytest.mark.parametrize("kernel,dtype", KERNELS, ids=KIDS)
def test_counts_every_radius(cat, kernel, dtype):
    grid = _grid(300, 437, 0.5, 7)
    for r in range(1, 17):
        got = sums(cat, kernel, dtype, grid, inputs.vn_scaled_rule(r))
        assert_same(got, oracle.box_sums(grid, r, nbhd="N"), f"R r={r}")


@pytest.mark.parametrize("kernel,dtype", KERNELS, ids=KIDS)
def test_counts_impulse_and_all_ones(cat, kernel, dtype):
    ones = np.ones((260, 270), np.uint8)
    imp = np.zeros((200, 333), np.uint8)
    imp[100, 129] = 1
    imp[0, 0] = 1
    imp[199, 332] = 1
    for r in (1, 7, 8, 16):
        for grid in (ones, imp):
            got = sums(cat, kernel, dtype, grid, inputs.vn_scaled_rule(r))
            assert_same(got, oracle.box_sums(grid, r, nbhd="N"), f"R r={r}")
    assert oracle.box_sums(ones, 16, nbhd="N")[130, 135] == 66


@pytest.mark.parametrize("kernel,dtype", KERNELS, ids=KIDS)
def test_scaled_rules_every_radius(cat, kernel, dtype):
    """The cross-scaled rule (n = 4r + 1), M0 and M1, 3 steps on 384 x 523."""
    for r in range(1, 17):
        rule = inputs.vn_scaled_rule(r, M=r % 2)
        grid = _grid(384, 523, 0.5, 200 + r)
        want = oracle.step(grid, orule(rule), n_steps=3)
        assert_same(run(cat, kernel, dtype, grid, rule, 3), want, f"r={r}")


@pytest.mark.parametrize("kernel,dtype", KERNELS, ids=KIDS)
def test_degenerate_shapes(cat, kernel, dtype):
    shapes = [(1, 1), (1, 200), (200, 1), (2, 3), (127, 129), (128, 128), (129, 255), (17, 300), (300, 17)]
    for i, (H, W) in enumerate(shapes):
        for r in (1, 5, 16):
            rule = dict(inputs.vn_scaled_rule(r, M=0), b1=1, b2=2 * r)
            grid = inputs.bernoulli(H, W, 0.45, 950 + i)
            want = oracle.step(grid, orule(rule), n_steps=2)
            assert_same(run(cat, kernel, dtype, grid, rule, 2), want, f"{H}x{W} r={r}")


def test_periodic_boundary(cat):
    """The cross wraps around the torus (tcgen05 with the ghost frame)."""
    for (H, W) in ((130, 300), (256, 256), (40, 20)):
        for r in (1, 6, 16):
            rule = inputs.vn_scaled_rule(r)
            grid = _grid(H, W, 0.5, 300 + r)
            got = sums(cat, "tcgen05", "fp8", grid, rule, boundary=cat.BOUNDARY_PERIODIC)
            assert_same(got, oracle.box_sums(grid, r, oracle.PERIODIC, nbhd="N"), f"R {H}x{W} r={r}")
            want = oracle.step(grid, orule(rule), oracle.PERIODIC, n_steps=3)
            assert_same(run(cat, "tcgen05", "fp8", grid, rule, 3, cat.BOUNDARY_PERIODIC), want, f"{H}x{W} r={r}")


def test_multistate_on_the_stencil(cat):
    """C > 2 with the cross: the default kernel is the stencil; the tcgen05 kernel refuses."""
    for C, rule in ((3, dict(r=3, C=3, M=0, s1=2, s2=6, b1=3, b2=5, nbhd="N")),
                    (16, dict(r=10, C=16, M=1, s1=8, s2=20, b1=7, b2=12, nbhd="N"))):
        grid = inputs.uniform_states(290, 310, C, 40 + C)
        want = oracle.step(grid, orule(rule), n_steps=5)
        assert_same(run(cat, "auto", "auto", grid, rule, 5), want, f"C={C} auto")
        assert_same(run(cat, "stencil", "auto", grid, rule, 5), want, f"C={C} stencil")
        assert_same(run(cat, "mma_sync", "fp16", grid, rule, 5), want, f"C={C} mma_sync")
        with pytest.raises(cat.CatError) as e:
            cat.Grid(64, 64, rule, kernel="tcgen05", dtype="fp8")
        assert e.value.code == cat.CAT_ERR_UNSUPPORTED


def test_unsupported_combinations(cat):
    rule = inputs.vn_scaled_rule(4)
    for kernel, dtype in (("mma_sync", "int8"), ("tcgen05", "fp16")):
        with pytest.raises(cat.CatError) as e:
            cat.Grid(64, 64, rule, kernel=kernel, dtype=dtype)
        assert e.value.code == cat.CAT_ERR_UNSUPPORTED, (kernel, dtype)
    with pytest.raises(cat.CatError) as e:
        cat.Grid(64, 64, rule, storage=cat.STORE_BIT1)
    assert e.value.code == cat.CAT_ERR_UNSUPPORTED


def test_batch_mixes_neighbourhoods(cat):
    """A batch of cross and Moore instances steps each one; results match the oracle."""
    specs = [(200, 301, inputs.vn_scaled_rule(3)), (150, 129, inputs.scaled_rule(9)),
             (257, 64, inputs.vn_scaled_rule(16, M=0))]
    grids, wants = [], []
    try:
        for i, (H, W, rule) in enumerate(specs):
            grid = _grid(H, W, 0.5, 80 + i)
            g = cat.Grid(H, W, rule, kernel="tcgen05", dtype="fp8")
            g.set_state(grid)
            grids.append(g)
            wants.append(oracle.step(grid, orule(rule), n_steps=4))
        cat.cat_batch_step([g.handle for g in grids], 4)
        for g, w, s in zip(grids, wants, specs):
            assert g.status() == cat.CAT_OK
            assert_same(g.get_state(), w, f"instance {s[:2]}")
    finally:
        for g in grids:
            g.close()


def test_bounded_wait_reports_timeout(cat):
    grid = _grid(256, 256, 0.5, 1)
    rule = inputs.vn_scaled_rule(2)
    g = cat.Grid(256, 256, rule, kernel="tcgen05", dtype="fp8")
    try:
        g.set_state(grid)
        cat.cat_debug_control(g.handle, 2, 20)
        cat.cat_debug_control(g.handle, 1, 1)
        g.step(1)
        assert g.status() == cat.CAT_ERR_TIMEOUT
        cat.cat_debug_control(g.handle, 1, 0)
        cat.cat_debug_control(g.handle, 2, 2000)
        g.set_state(grid)
        g.step(3)
        assert g.status() == cat.CAT_OK
        assert_same(g.get_state(), oracle.step(grid, orule(rule), n_steps=3), "after timeout")
    finally:
        g.close()


# ---------------------------------------------------- workload-scale checks
def test_radius_sweep_4096_every_radius(cat):
    """4096^2 Bernoulli(0.5), the cross-scaled rule (C2 M1), r = 1..16, 2 steps, full equality."""
    grid = inputs.bernoulli(4096, 4096, 0.5, 4097)
    for r in range(1, 17):
        rule = inputs.vn_scaled_rule(r)
        want = oracle.step(grid, orule(rule), n_steps=2)
        assert_same(run(cat, "tcgen05", "fp8", grid, rule, 2), want, f"4096^2 r={r}")


def test_full_16384_sampled_windows(cat):
    """16384^2 Bernoulli(0.5): one tcgen05 step checked against the oracle on 24
    windows (corners included), then 5 steps equal to the stencil on every cell."""
    import torch
    N = 16384
    grid_host = inputs.bernoulli(N, N, 0.5, 2025)
    d_grid = torch.from_numpy(grid_host).cuda()
    rng = np.random.default_rng(2)
    for r in (1, 8, 16):
        rule = inputs.vn_scaled_rule(r)
        g = cat.Grid(N, N, rule, kernel="tcgen05", dtype="fp8")
        st = cat.Grid(N, N, rule, kernel="stencil", dtype="auto")
        try:
            g.set_state(d_grid)
            st.set_state(d_grid)
            g.step(1)
            torch.cuda.synchronize()
            assert g.status() == cat.CAT_OK
            out = g.state_tensor()
            corners = [(0, 0), (0, N - 256), (N - 256, 0), (N - 256, N - 256)]
            spots = corners + [tuple(int(v) for v in rng.integers(0, N - 256, 2)) for _ in range(20)]
            for (y0, x0) in spots:
                ya, xa = max(0, y0 - r), max(0, x0 - r)
                yb, xb = min(N, y0 + 256 + r), min(N, x0 + 256 + r)
                want = oracle.step(grid_host[ya:yb, xa:xb], orule(rule))[y0 - ya:y0 - ya + 256, x0 - xa:x0 - xa + 256]
                assert_same(out[y0:y0 + 256, x0:x0 + 256].cpu().numpy(), want, f"r={r} window ({y0},{x0})")
            g.step(4)
            st.step(5)
            torch.cuda.synchronize()
            assert g.status() == cat.CAT_OK
            diff = int((g.state_tensor() != st.state_tensor()).sum())
            assert diff == 0, f"r={r}: {diff} cells differ between tcgen05 and the stencil after 5 steps"
        finally:
            g.close()
            st.close()

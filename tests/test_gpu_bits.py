"""One-bit storage (CAT_STORE_BIT1) vs the CPU oracle, element by element.

The grid lives in HBM as 8 cells per byte; the step kernel unpacks its
windows into the FP8 operand in shared memory and packs the next state in its
epilogue.  The oracle sees the same grids one byte per cell, so every case
checks the packing, the band products and the rule together.  The packed
bytes are also compared with numpy's little-endian bit packing, and the bits
past W in a row's last byte must stay 0 (the kernel reads them as neighbours
of the next step).
"""
import functools

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


def rule_dict(r, M=1, b=None):
    s1, s2, b1, b2 = inputs.scaled_rule_ranges(r)
    if b is not None:
        b1, b2 = b
    return dict(r=r, C=2, M=M, s1=s1, s2=s2, b1=b1, b2=b2)


def orule(d):
    return oracle.Rule(d["r"], d["C"], d["M"], d["s1"], d["s2"], d["b1"], d["b2"])


@functools.lru_cache(maxsize=None)
def _grid(H, W, p, seed):
    return inputs.bernoulli(H, W, p, seed)


def assert_same(got, want, what):
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        y, x = bad[0]
        raise AssertionError(f"{what}: {len(bad)} cells differ, first at ({y},{x}): got {got[y, x]} want {want[y, x]}")


def bits_grid(cat, H, W, rule):
    return cat.Grid(H, W, rule, kernel="tcgen05", dtype="fp8", storage=cat.STORE_BIT1)


def run_bits(cat, grid, rule, steps):
    g = bits_grid(cat, grid.shape[0], grid.shape[1], rule)
    try:
        g.set_state(grid)
        g.step(steps)
        out = g.get_state()
        assert g.status() == cat.CAT_OK
        return out
    finally:
        g.close()


def packed(grid):
    return np.packbits(grid.astype(bool), axis=1, bitorder="little")


def test_set_get_round_trip_and_packed_layout(cat):
    """set_state/get_state are exact; state_tensor holds the little-endian packing."""
    for H, W in ((1, 1), (3, 7), (129, 255), (300, 437), (256, 1024)):
        grid = _grid(H, W, 0.5, H + W)
        g = bits_grid(cat, H, W, inputs.CONWAY)
        try:
            g.set_state(grid)
            assert_same(g.get_state(), grid, f"{H}x{W} round trip")
            assert_same(g.state_tensor().cpu().numpy(), packed(grid), f"{H}x{W} packed bytes")
        finally:
            g.close()


def test_box_sums_every_radius(cat):
    grid = _grid(300, 437, 0.5, 7)
    for r in range(1, 17):
        g = bits_grid(cat, 300, 437, rule_dict(r))
        try:
            g.set_state(grid)
            assert_same(g.box_sums(), oracle.box_sums(grid, r), f"S r={r}")
        finally:
            g.close()


def test_box_sums_all_ones(cat):
    """Every cell alive, W not a multiple of 8: the dead cells past W stay out of the counts."""
    ones = np.ones((260, 270), np.uint8)
    for r in (1, 7, 8, 16):
        g = bits_grid(cat, 260, 270, rule_dict(r))
        try:
            g.set_state(ones)
            assert_same(g.box_sums(), oracle.box_sums(ones, r), f"S r={r}")
        finally:
            g.close()


def test_conway_256_100_steps(cat):
    grid = _grid(256, 256, 0.5, 1)
    want = oracle.step(grid, orule(inputs.CONWAY), n_steps=100)
    assert_same(run_bits(cat, grid, inputs.CONWAY, 100), want, "conway")


def test_scaled_rules_every_radius(cat):
    """The radius-scaled rule, M0 and M1, 3 steps, on 384 x 523 (ragged in x and y)."""
    for r in range(1, 17):
        rule = rule_dict(r, M=r % 2)
        grid = _grid(384, 523, 0.5, 100 + r)
        want = oracle.step(grid, orule(rule), n_steps=3)
        assert_same(run_bits(cat, grid, rule, 3), want, f"r={r}")


def test_degenerate_shapes_and_births_at_the_edge(cat):
    """Births spread into the cells next to x = W - 1; the packed bits past W stay 0."""
    shapes = [(1, 1), (1, 200), (200, 1), (2, 3), (127, 129), (128, 128), (129, 255), (17, 300), (300, 17),
              (130, 1023), (64, 2049)]
    for i, (H, W) in enumerate(shapes):
        for r in (1, 5, 8, 16):
            rule = rule_dict(r, M=0, b=(1, 3 * r))
            grid = inputs.bernoulli(H, W, 0.45, 900 + i)
            g = bits_grid(cat, H, W, rule)
            try:
                g.set_state(grid)
                g.step(2)
                got = g.get_state()
                want = oracle.step(grid, orule(rule), n_steps=2)
                assert_same(got, want, f"{H}x{W} r={r}")
                assert_same(g.state_tensor().cpu().numpy(), packed(want), f"{H}x{W} r={r} packed bytes")
            finally:
                g.close()


def test_storage_switch_keeps_the_state(cat):
    """U8 -> BIT1 -> U8 with steps in between equals 9 uninterrupted oracle steps."""
    rule = rule_dict(6)
    grid = _grid(333, 517, 0.5, 61)
    want = oracle.step(grid, orule(rule), n_steps=9)
    g = cat.Grid(333, 517, rule, kernel="tcgen05", dtype="fp8")
    try:
        g.set_state(grid)
        g.step(3)
        cat.cat_set_options(g.handle, cat.KERNEL_TCGEN05, cat.DTYPE_FP8_E4M3, cat.STORE_BIT1)
        g.storage = cat.STORE_BIT1
        g.step(3)
        mid = oracle.step(grid, orule(rule), n_steps=6)
        assert_same(g.get_state(), mid, "after the switch to BIT1")
        cat.cat_set_options(g.handle, cat.KERNEL_MMA_SYNC, cat.DTYPE_FP16, cat.STORE_U8)
        g.storage = cat.STORE_U8
        g.step(3)
        assert g.status() == cat.CAT_OK
        assert_same(g.get_state(), want, "after the switch back to U8 (mma.sync)")
    finally:
        g.close()


def test_unsupported_combinations(cat):
    conway = cat.make_rule(**inputs.CONWAY)
    with pytest.raises(cat.CatError) as e:
        cat.cat_create_ex(64, 64, cat.make_rule(3, 3, 0, 10, 25, 9, 14), cat.BOUNDARY_ZERO, cat.STORE_BIT1)
    assert e.value.code == cat.CAT_ERR_UNSUPPORTED
    with pytest.raises(cat.CatError) as e:
        cat.cat_create_ex(64, 64, conway, cat.BOUNDARY_PERIODIC, cat.STORE_BIT1)
    assert e.value.code == cat.CAT_ERR_UNSUPPORTED
    with pytest.raises(cat.CatError) as e:
        cat.cat_create_ex(64, 64, conway, cat.BOUNDARY_ZERO, 7)
    assert e.value.code == cat.CAT_ERR_INVALID_ARG
    h = cat.cat_create_ex(64, 64, conway, cat.BOUNDARY_ZERO, cat.STORE_BIT1)
    try:
        for kernel, dtype in ((cat.KERNEL_TCGEN05, cat.DTYPE_FP16), (cat.KERNEL_MMA_SYNC, cat.DTYPE_FP16),
                              (cat.KERNEL_STENCIL, cat.DTYPE_AUTO)):
            with pytest.raises(cat.CatError) as e:
                cat.cat_set_options(h, kernel, dtype, cat.STORE_BIT1)
            assert e.value.code == cat.CAT_ERR_UNSUPPORTED
    finally:
        cat.cat_destroy(h)


def test_batch_step_mixes_storages(cat):
    """A batch holding BIT1 and U8 instances steps each one; results match the oracle."""
    specs = [(200, 301, 3, cat.STORE_BIT1), (150, 129, 9, cat.STORE_U8), (257, 64, 16, cat.STORE_BIT1)]
    grids, wants = [], []
    try:
        for i, (H, W, r, st) in enumerate(specs):
            rule = rule_dict(r)
            grid = _grid(H, W, 0.5, 70 + i)
            g = cat.Grid(H, W, rule, kernel="tcgen05", dtype="fp8", storage=st)
            g.set_state(grid)
            grids.append(g)
            wants.append(oracle.step(grid, orule(rule), n_steps=4))
        cat.cat_batch_step([g.handle for g in grids], 4)
        for g, w, s in zip(grids, wants, specs):
            assert g.status() == cat.CAT_OK
            assert_same(g.get_state(), w, f"instance {s}")
    finally:
        for g in grids:
            g.close()


def test_bounded_wait_reports_timeout(cat):
    grid = _grid(256, 256, 0.5, 1)
    g = bits_grid(cat, 256, 256, inputs.CONWAY)
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
        assert_same(g.get_state(), oracle.step(grid, orule(inputs.CONWAY), n_steps=3), "after timeout")
    finally:
        g.close()


# ---------------------------------------------------- full-size launch checks
def test_full_16384_sampled_windows_and_u8_equality(cat):
    """16384^2 Bernoulli(0.5), the headline grid: one BIT1 step checked against
    the oracle on 24 windows, and 5 steps equal to the uint8 path on every cell."""
    import torch
    N = 16384
    grid_host = inputs.bernoulli(N, N, 0.5, 2024)
    d_grid = torch.from_numpy(grid_host).cuda()
    rng = np.random.default_rng(1)
    for r in (1, 7, 8, 16):
        rule = rule_dict(r)
        g = bits_grid(cat, N, N, rule)
        u = cat.Grid(N, N, rule, kernel="tcgen05", dtype="fp8")
        try:
            g.set_state(d_grid)
            u.set_state(d_grid)
            g.step(1)
            out = torch.empty((N, N), dtype=torch.uint8, device="cuda")
            cat.cat_get_state(g.handle, out.data_ptr(), N, True)
            torch.cuda.synchronize()
            assert g.status() == cat.CAT_OK
            corners = [(0, 0), (0, N - 256), (N - 256, 0), (N - 256, N - 256)]
            spots = corners + [tuple(int(v) for v in rng.integers(0, N - 256, 2)) for _ in range(20)]
            for (y0, x0) in spots:
                ya, xa = max(0, y0 - r), max(0, x0 - r)
                yb, xb = min(N, y0 + 256 + r), min(N, x0 + 256 + r)
                want = oracle.step(grid_host[ya:yb, xa:xb], orule(rule))[y0 - ya:y0 - ya + 256, x0 - xa:x0 - xa + 256]
                assert_same(out[y0:y0 + 256, x0:x0 + 256].cpu().numpy(), want, f"r={r} window ({y0},{x0})")
            g.step(4)
            u.step(5)
            cat.cat_get_state(g.handle, out.data_ptr(), N, True)
            torch.cuda.synchronize()
            assert g.status() == cat.CAT_OK and u.status() == cat.CAT_OK
            diff = int((out != u.state_tensor()).sum())
            assert diff == 0, f"r={r}: {diff} cells differ between BIT1 and U8 after 5 steps"
        finally:
            g.close()
            u.close()


def test_ragged_6600x1001_two_steps(cat):
    """A tall grid whose width is not a multiple of 8 or 128, full equality."""
    H, W = 6600, 1001
    rule = rule_dict(12, M=0)
    grid = _grid(H, W, 0.4, 66)
    want = oracle.step(grid, orule(rule), n_steps=2)
    assert_same(run_bits(cat, grid, rule, 2), want, "6600x1001")

"""Periodic boundary (the grid wraps around in both directions, the paper's own
setting, Sec. V) on the tcgen05 kernel, against the oracle's periodic mode.

The GPU keeps a periodic grid inside a 16-cell ghost frame that a small kernel
refreshes before every step; the cases cover grids smaller than the frame (the
box then wraps onto itself several times), grids that are not a multiple of
the 128-cell tile, every kind of edge and corner tile, and radii 1..16.
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
    return oracle.Rule(**{k: d[k] for k in ("r", "C", "M", "s1", "s2", "b1", "b2")})


def assert_same(got, want, what):
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        y, x = bad[0]
        raise AssertionError(f"{what}: {len(bad)} cells differ, first at ({y},{x}): got {got[y, x]} want {want[y, x]}")


CASES = [  # H, W, r, steps
    (300, 437, 9, 4), (128, 256, 16, 2), (7, 13, 3, 5), (1, 1, 1, 2), (200, 5, 4, 3),
    (515, 129, 12, 2), (64, 64, 1, 10), (17, 300, 16, 2), (256, 1000, 6, 3),
]


@pytest.mark.parametrize("dtype", ["fp8", "fp16", "fp4"])
def test_periodic_steps_match_oracle(cat, dtype):
    for H, W, r, steps in CASES:
        rule = inputs.scaled_rule(r, M=1)
        grid = inputs.bernoulli(H, W, 0.4, 100 + H + W + r)
        g = cat.Grid(H, W, rule, kernel="tcgen05", dtype=dtype, boundary=cat.BOUNDARY_PERIODIC)
        try:
            g.set_state(grid)
            g.step(steps)
            assert g.status() == cat.CAT_OK
            want = oracle.step(grid, orule(rule), oracle.PERIODIC, n_steps=steps)
            assert_same(g.get_state(), want, f"periodic {dtype} {H}x{W} r={r} after {steps} steps")
        finally:
            g.close()


def test_periodic_box_sums_match_oracle(cat):
    for H, W, r, _ in CASES:
        rule = inputs.scaled_rule(r, M=1)
        grid = inputs.bernoulli(H, W, 0.5, 7 + H * W + r)
        g = cat.Grid(H, W, rule, kernel="tcgen05", dtype="fp8", boundary=cat.BOUNDARY_PERIODIC)
        try:
            g.set_state(grid)
            got = g.box_sums()
            want = oracle.box_sums(grid, r, oracle.PERIODIC)
            assert_same(got, want, f"periodic box sums {H}x{W} r={r}")
        finally:
            g.close()


def test_periodic_step_commutes_with_cyclic_shift(cat):
    """Stepping a shifted grid equals shifting the stepped grid (periodic boundary
    only); checked on the GPU alone, across tile and grid edges."""
    H, W, r = 300, 437, 7
    rule = inputs.scaled_rule(r, M=1)
    grid = inputs.bernoulli(H, W, 0.45, 31)
    outs = []
    for shift in ((0, 0), (131, 250)):
        g = cat.Grid(H, W, rule, kernel="tcgen05", dtype="fp8", boundary=cat.BOUNDARY_PERIODIC)
        try:
            g.set_state(np.ascontiguousarray(np.roll(grid, shift, (0, 1))))
            g.step(3)
            outs.append(np.roll(g.get_state(), (-shift[0], -shift[1]), (0, 1)))
        finally:
            g.close()
    assert_same(outs[1], outs[0], "shifted run")


def test_periodic_glider_comes_home(cat):
    """A Conway glider moves one cell diagonally every 4 steps, so on a 32 x 32
    torus it is back where it started after 128 steps, having crossed every edge."""
    N = 32
    grid = np.zeros((N, N), dtype=np.uint8)
    inputs.place(grid, "glider", 29, 29)   # next to the corner, heading across it
    g = cat.Grid(N, N, inputs.CONWAY, kernel="tcgen05", dtype="fp8", boundary=cat.BOUNDARY_PERIODIC)
    try:
        g.set_state(grid)
        g.step(4 * N)
        assert_same(g.get_state(), grid, "glider after 128 steps")
        g.step(2)
        assert_same(g.get_state(), oracle.step(grid, orule(inputs.CONWAY), oracle.PERIODIC, n_steps=2), "glider + 2")
    finally:
        g.close()


def test_periodic_rejected_by_comparator_kernels(cat):
    g = cat.Grid(64, 64, inputs.CONWAY, kernel="tcgen05", dtype="fp8", boundary=cat.BOUNDARY_PERIODIC)
    try:
        with pytest.raises(cat.CatError):
            cat.cat_set_options(g.handle, cat.KERNEL_MMA_SYNC, cat.DTYPE_FP16)
    finally:
        g.close()

"""Several steps per launch (steps_per_launch > 1) vs the CPU oracle.

cat_step then runs k steps in one cooperative launch of the tcgen05 kernel:
odd steps swap the buffers, and the CTAs meet on a grid-wide barrier between
steps (Sec. IV-C's ping-pong, without a launch per step).  Every operand and
storage variant goes through it: FP8 (short window for r <= 7, standard
window above), FP16, the re-encoded multi-state window and one-bit storage.
Grids from one tile to more tiles than CTAs (uneven tiles per CTA) are
stepped with step counts that do and do not divide by k.
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
    return oracle.Rule(d["r"], d["C"], d["M"], d["s1"], d["s2"], d["b1"], d["b2"], d.get("nbhd", "M"))


def assert_same(got, want, what):
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        y, x = bad[0]
        raise AssertionError(f"{what}: {len(bad)} cells differ, first at ({y},{x}): got {got[y, x]} want {want[y, x]}")


def run(cat, grid, rule, steps, k, dtype="fp8", storage=0, calls=1):
    g = cat.Grid(grid.shape[0], grid.shape[1], rule, kernel="tcgen05", dtype=dtype, storage=storage,
                 steps_per_launch=k)
    try:
        g.set_state(grid)
        for _ in range(calls):
            g.step(steps)
        out = g.get_state()
        assert g.status() == cat.CAT_OK
        return out
    finally:
        g.close()


VARIANTS = [("fp8", 0, False), ("fp16", 0, False), ("fp8", 0, True), ("fp8", 1, False)]
VIDS = ["fp8", "fp16", "fp8-multistate", "fp8-bits"]


@pytest.mark.parametrize("dtype,storage,multi", VARIANTS, ids=VIDS)
def test_matches_oracle(cat, dtype, storage, multi):
    shapes = [(100, 90), (300, 437), (2048, 2048), (2600, 1100)]   # 1 tile .. more tiles than CTAs
    for i, (H, W) in enumerate(shapes):
        for r, k, steps in ((3, 2, 5), (10, 4, 8), (16, 8, 7)):
            if multi:
                rule = dict(r=r, C=5, M=1, s1=r, s2=3 * r * r, b1=r, b2=2 * r * r)
                grid = inputs.uniform_states(H, W, 5, 60 + i)
            else:
                rule = inputs.scaled_rule(r, M=i % 2)
                grid = inputs.bernoulli(H, W, 0.5, 70 + i)
            want = oracle.step(grid, orule(rule), n_steps=steps)
            got = run(cat, grid, rule, steps, k, dtype, storage)
            assert_same(got, want, f"{H}x{W} r={r} k={k} steps={steps}")


def test_conway_100_steps_one_launch(cat):
    grid = inputs.bernoulli(256, 256, 0.5, 1)
    want = oracle.step(grid, orule(inputs.CONWAY), n_steps=100)
    assert_same(run(cat, grid, inputs.CONWAY, 100, 100), want, "conway, 100 steps per launch")


def test_repeated_calls_keep_the_barrier_count(cat):
    """Many multi-step launches on one instance (the barrier counter keeps growing)."""
    grid = inputs.bernoulli(1024, 1024, 0.45, 5)
    rule = inputs.scaled_rule(6)
    want = oracle.step(grid, orule(rule), n_steps=60)
    assert_same(run(cat, grid, rule, 3, 3, calls=20), want, "20 calls of 3 steps")


def test_equals_one_step_per_launch_16384(cat):
    import torch
    N = 16384
    d = torch.from_numpy(inputs.bernoulli(N, N, 0.5, 2026)).cuda()
    for r in (2, 12):
        rule = inputs.scaled_rule(r)
        a = cat.Grid(N, N, rule, kernel="tcgen05", dtype="fp8", steps_per_launch=4)
        b = cat.Grid(N, N, rule, kernel="tcgen05", dtype="fp8")
        try:
            a.set_state(d)
            b.set_state(d)
            a.step(9)
            b.step(9)
            torch.cuda.synchronize()
            assert a.status() == cat.CAT_OK and b.status() == cat.CAT_OK
            diff = int((a.state_tensor() != b.state_tensor()).sum())
            assert diff == 0, f"r={r}: {diff} cells differ"
        finally:
            a.close()
            b.close()


def test_unsupported_combinations(cat):
    for kw in (dict(kernel="mma_sync", dtype="fp16"), dict(kernel="stencil", dtype="auto"),
               dict(boundary=cat.BOUNDARY_PERIODIC)):
        with pytest.raises(cat.CatError) as e:
            cat.Grid(64, 64, inputs.scaled_rule(3), steps_per_launch=4, **kw)
        assert e.value.code == cat.CAT_ERR_UNSUPPORTED, kw
    with pytest.raises(cat.CatError) as e:
        cat.Grid(64, 64, inputs.vn_scaled_rule(3), steps_per_launch=4)
    assert e.value.code == cat.CAT_ERR_UNSUPPORTED


def test_bounded_wait_reports_timeout_and_recovers(cat):
    """A launch that gives up (here: the pass-1 issuer waits on a barrier nothing
    arrives at) reports CAT_ERR_TIMEOUT; after cat_status the barrier counter is
    reset and multi-step launches run correctly again."""
    grid = inputs.bernoulli(600, 700, 0.5, 3)
    rule = inputs.scaled_rule(4)
    g = cat.Grid(600, 700, rule, kernel="tcgen05", dtype="fp8", steps_per_launch=4)
    try:
        g.set_state(grid)
        cat.cat_debug_control(g.handle, 2, 20)
        cat.cat_debug_control(g.handle, 1, 1)
        g.step(8)
        assert g.status() == cat.CAT_ERR_TIMEOUT
        cat.cat_debug_control(g.handle, 1, 0)
        cat.cat_debug_control(g.handle, 2, 2000)
        g.set_state(grid)
        g.step(8)
        assert g.status() == cat.CAT_OK
        assert_same(g.get_state(), oracle.step(grid, orule(rule), n_steps=8), "after timeout")
    finally:
        g.close()

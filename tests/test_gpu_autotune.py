"""The autotuner (cat_autotune, cat_autotune_batch) picks a configuration by
timing, keeps the state it was called on, writes its JSON-lines cache, and
what it picks stays bit-exact against the oracle.  With CAT_AUTOTUNE_CACHE
set, CAT_KERNEL_AUTO takes the cached choice."""
import json
import os
import statistics

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


def rate_of(cat, g, n, steps=8, reps=3):
    """cell-updates/s of the instance's current options (state restored after)."""
    import torch
    before = g.get_state()
    g.step(steps)
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.step(steps)
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    g.set_state(before)
    return n * steps / (statistics.median(times) / 1000.0)


CASES = [(2048, 2048, 4, 1), (4096, 4096, 12, 0), (1000, 3000, 20, 1)]


@pytest.mark.parametrize("H,W,r,M", CASES, ids=[f"{c[0]}x{c[1]}-r{c[2]}" for c in CASES])
def test_autotune_picks_a_fastest_configuration_and_stays_exact(cat, tmp_path, H, W, r, M):
    rule = inputs.scaled_rule(r, M)
    grid = inputs.bernoulli(H, W, 0.5, H + r)
    cache = str(tmp_path / "tune.jsonl")
    g = cat.Grid(H, W, rule)
    try:
        g.set_state(grid)
        cat.cat_autotune(g.handle, 8, cache)
        assert np.array_equal(g.get_state(), grid), "the autotuner changed the state"
        chosen = cat.cat_get_options(g.handle)
        lines = [json.loads(ln) for ln in open(cache)]
        assert len(lines) == 1 and lines[0]["kernel"] == chosen["kernel"]
        assert lines[0]["steps_per_launch"] == chosen["steps_per_launch"]
        assert f"H={H} W={W} r={r}" in lines[0]["key"]
        best = rate_of(cat, g, H * W, steps=8 * chosen["steps_per_launch"])
        # the chosen configuration is at least as fast (within timing noise) as
        # the fixed rule and the other tcgen05 dtype
        for kernel, dtype in (("tcgen05", "fp8"), ("tcgen05", "fp16"), ("mma_sync", "fp16")):
            try:
                other = cat.Grid(H, W, rule, kernel=kernel, dtype=dtype)
            except cat.CatError:
                continue
            try:
                other.set_state(grid)
                assert best >= 0.85 * rate_of(cat, other, H * W), (kernel, dtype, chosen)
            finally:
                other.close()
        # bit-exact with what was chosen
        g.set_state(grid)
        g.step(3)
        assert g.status() == cat.CAT_OK
        assert np.array_equal(g.get_state(), oracle.step(grid, orule(rule), n_steps=3))
        # a second call reads the cache instead of timing, and a fresh AUTO
        # instance takes the cached choice when CAT_AUTOTUNE_CACHE names the file
        cat.cat_autotune(g.handle, 8, cache)
        assert len(open(cache).readlines()) == 1
        os.environ["CAT_AUTOTUNE_CACHE"] = cache
        try:
            fresh = cat.Grid(H, W, rule, kernel="auto", dtype="auto")
            try:
                assert cat.cat_get_options(fresh.handle) == chosen
                fresh.set_state(grid)
                fresh.step(2)
                assert np.array_equal(fresh.get_state(), oracle.step(grid, orule(rule), n_steps=2))
            finally:
                fresh.close()
        finally:
            del os.environ["CAT_AUTOTUNE_CACHE"]
    finally:
        g.close()


def test_autotune_one_bit_storage_small_radius(cat, tmp_path):
    """One-bit storage at r = 1: the candidates include the bit-sliced kernel."""
    H, W = 4096, 4096
    rule = inputs.scaled_rule(1, 1)
    grid = inputs.bernoulli(H, W, 0.5, 11)
    g = cat.Grid(H, W, rule, storage=cat.STORE_BIT1)
    try:
        g.set_state(grid)
        cat.cat_autotune(g.handle, 8, str(tmp_path / "t.jsonl"))
        assert np.array_equal(g.get_state(), grid)
        g.step(4)
        assert np.array_equal(g.get_state(), oracle.step(grid, orule(rule), n_steps=4))
    finally:
        g.close()


def test_autotune_batch(cat):
    rng = np.random.default_rng(9)
    specs = []
    for i in range(24):
        H, W = (int(v) for v in rng.integers(40, 700, 2))
        specs.append((inputs.bernoulli(H, W, 0.4, 70 + i), inputs.scaled_rule(int(rng.integers(1, 17)), i % 2)))
    grids = [cat.Grid(g.shape[0], g.shape[1], rule) for g, rule in specs]
    try:
        for G, (g, _) in zip(grids, specs):
            G.set_state(g)
        dt = cat.cat_autotune_batch([G.handle for G in grids], 4)
        assert dt in (cat.DTYPE_FP8_E4M3, cat.DTYPE_FP16)
        for G, (g, _) in zip(grids, specs):
            assert np.array_equal(G.get_state(), g)
            assert cat.cat_get_options(G.handle)["dtype"] == dt
        cat.cat_batch_step([G.handle for G in grids], 3)
        for G, (g, rule) in zip(grids, specs):
            assert np.array_equal(G.get_state(), oracle.step(g, orule(rule), n_steps=3))
    finally:
        for G in grids:
            G.close()

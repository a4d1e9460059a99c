"""Batched persistent launch (cat_batch_step) vs the oracle, per instance, bit-exact."""
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


def make_batch(seed, count, lo, hi, multistate=False, r_max=16):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        H = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        W = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        r = int(rng.integers(1, r_max + 1))
        M = int(rng.integers(0, 2))
        if multistate and i % 2 == 0:
            C = int(rng.choice([3, 5, 16]))
            rule = inputs.scaled_rule(r, M, C)
            grid = inputs.uniform_states(H, W, C, seed * 1000 + i)
        else:
            rule = inputs.scaled_rule(r, M)
            grid = inputs.bernoulli(H, W, float(rng.uniform(0.2, 0.6)), seed * 1000 + i)
        out.append((grid, rule))
    out.append((inputs.bernoulli(1, 1, 1.0, 1), inputs.scaled_rule(3, 0)))   # degenerate shapes
    out.append((inputs.bernoulli(1, 300, 0.5, 2), inputs.scaled_rule(min(16, r_max), 1)))
    out.append((inputs.bernoulli(129, 1, 0.5, 3), inputs.scaled_rule(2, 1)))
    return out


def check_batch(cat, batch, steps_list, kernel="tcgen05", dtype="fp8", individual=None):
    grids = [cat.Grid(g.shape[0], g.shape[1], rule, kernel=kernel, dtype=dtype) for g, rule in batch]
    try:
        for G, (g, _) in zip(grids, batch):
            G.set_state(g)
        total = 0
        for n in steps_list:
            cat.cat_batch_step([G.handle for G in grids], n)
            total += n
            if individual is not None:  # step one instance on its own: its buffer parity drifts
                grids[individual].step(1)
        for i, (G, (g, rule)) in enumerate(zip(grids, batch)):
            assert G.status() == cat.CAT_OK
            extra = 1 if i == individual else 0
            want = oracle.step(g, orule(rule), n_steps=total + extra * len(steps_list))
            got = G.get_state()
            assert np.array_equal(got, want), f"instance {i} {g.shape} {rule}: {(got != want).sum()} cells differ"
    finally:
        for G in grids:
            G.close()


@pytest.mark.parametrize("dtype", ["fp8", "fp16"])
def test_batch_mixed_sizes_radii_rules(cat, dtype):
    check_batch(cat, make_batch(1, 40, 8, 700), [5], dtype=dtype)


def test_batch_small_radii_short_window(cat):
    # every grid has r <= 7 and C = 2: the FP8 batch runs the short-window kernel
    # (three tiles in flight, both e4m3 bands rebuilt whenever the radius changes)
    check_batch(cat, make_batch(6, 40, 8, 700, r_max=7), [3, 2])


def test_batch_graph_replay_odd_steps(cat):
    # 3 + 3 + 2 steps: the cached graph is reused with both start parities
    check_batch(cat, make_batch(2, 24, 16, 400), [3, 3, 2, 3])


def test_batch_parity_drift_reupload(cat):
    check_batch(cat, make_batch(3, 12, 16, 300), [2, 1, 2], individual=4)


def test_batch_multistate_encode_path(cat):
    check_batch(cat, make_batch(4, 20, 16, 400, multistate=True), [4])


@pytest.mark.parametrize("kernel,dtype", [("mma_sync", "int8"), ("stencil", "auto"), ("mma_sync", "fp16"),
                                          ("runsum", "auto")])
def test_batch_comparator_kernels(cat, kernel, dtype):
    check_batch(cat, make_batch(5, 10, 16, 300), [3], kernel=kernel, dtype=dtype)


def test_batch_under_caller_graph_capture(cat):
    import torch
    batch = make_batch(6, 10, 32, 300)
    grids = [cat.Grid(g.shape[0], g.shape[1], rule) for g, rule in batch]
    try:
        for G, (g, _) in zip(grids, batch):
            G.set_state(g)
        hs = [G.handle for G in grids]
        cat.cat_batch_step(hs, 2)  # warm-up (plan built, kernels configured) outside capture
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            cat.cat_batch_step(hs, 2)   # even: the handles' buffer parity is unchanged
        for _ in range(3):
            graph.replay()
        torch.cuda.synchronize()
        for G, (g, rule) in zip(grids, batch):
            want = oracle.step(g, orule(rule), n_steps=2 + 2 * 3)
            assert np.array_equal(G.get_state(), want)
    finally:
        for G in grids:
            G.close()


def test_batch_rejects_bad_lists(cat):
    g = cat.Grid(64, 64, inputs.CONWAY)
    h = cat.Grid(64, 64, inputs.CONWAY, dtype="fp16")
    try:
        with pytest.raises(cat.CatError):
            cat.cat_batch_step([g.handle, g.handle], 1)
        with pytest.raises(cat.CatError):
            cat.cat_batch_step([g.handle, h.handle], 1)
        cat.cat_batch_step([], 1)
        cat.cat_batch_step([g.handle], 0)
    finally:
        g.close()
        h.close()

"""Full-size workloads checked per instance against the oracle.

* The batched workload at its real size: 4096 grids (sides log-uniform in
  [64, 2048], independent H and W; r uniform in 1..16; M uniform in {0, 1};
  p uniform in [0.2, 0.6]; the radius-scaled rule, C = 2), the draw the
  benchmark times, advanced by cat_batch_step (one persistent launch over the
  tile work-list of all 4096 grids per step, replayed from a CUDA graph).
  At least 64 grids are compared with the oracle cell by cell after 4 steps:
  the 16 largest, one grid for every (r, M) pair, and a seeded random rest.
* The multi-state rule R10 C16 M1 S150..260 B150..200 from a live start
  (states 0/1 drawn Bernoulli(0.5), so counts sit inside the survival range):
  cells keep being born, surviving and decaying through step 100, where one
  step is checked on windows against the oracle (Sec. V-A notation; the
  decay reading of multi-state rules: state 1 fails survival -> 2, then +1
  per step to 0 after C - 1).
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from oracle import oracle
from paper_2406_17284_gb300 import inputs

pytestmark = pytest.mark.gpu

SEED = 2024   # the benchmark's draw of the batched workload


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


def checked_subset(specs, n_min=64, seed=7):
    """The 16 largest grids, the smallest grid of every (r, M) pair, then seeded
    random grids until n_min are chosen."""
    size = lambda i: specs[i]["H"] * specs[i]["W"]   # noqa: E731
    order = sorted(range(len(specs)), key=size)
    chosen = set(order[-16:])
    for r in range(1, 17):
        for M in (0, 1):
            cands = [i for i in order if specs[i]["rule"]["r"] == r and specs[i]["rule"]["M"] == M]
            assert cands, f"no grid with r={r} M={M} in the draw"
            chosen.add(cands[0])
    rng = np.random.default_rng(seed)
    while len(chosen) < n_min:
        chosen.add(int(rng.integers(0, len(specs))))
    return sorted(chosen)


def test_batch_4096_grids_per_instance_vs_oracle(cat):
    specs = inputs.batch_instances(4096, seed=SEED)
    with ThreadPoolExecutor(16) as ex:
        hosts = list(ex.map(lambda d: inputs.bernoulli(d["H"], d["W"], d["p"], d["seed"]), specs))
    check = checked_subset(specs)
    assert len(check) >= 64
    rs = {specs[i]["rule"]["r"] for i in check}
    Ms = {specs[i]["rule"]["M"] for i in check}
    assert rs == set(range(1, 17)) and Ms == {0, 1}
    grids = []
    try:
        for d, h in zip(specs, hosts):
            g = cat.Grid(d["H"], d["W"], d["rule"], kernel="tcgen05", dtype="fp8")
            grids.append(g)
            g.set_state(h)
        handles = [g.handle for g in grids]
        cat.cat_batch_step(handles, 3)      # one graph of 3 persistent launches
        cat.cat_batch_step(handles, 1)      # and a graph of one (the other buffer parity)
        for i in check:
            assert grids[i].status() == cat.CAT_OK
        bad = []
        for i in check:
            want = oracle.step(hosts[i], orule(specs[i]["rule"]), n_steps=4)
            got = grids[i].get_state()
            if not np.array_equal(got, want):
                bad.append((i, specs[i]["H"], specs[i]["W"], specs[i]["rule"]["r"], int((got != want).sum())))
        assert not bad, f"grids differing from the oracle (index, H, W, r, cells): {bad}"
        # the largest grids reach the 16 x 16-tile end of the work-list range
        big = max(check, key=lambda i: specs[i]["H"] * specs[i]["W"])
        assert specs[big]["H"] * specs[big]["W"] > 1800 * 1800
    finally:
        for g in grids:
            g.close()


def test_multistate_r10_c16_live_dynamics_at_step_100(cat):
    N = 4096
    rule = inputs.MULTISTATE_R10_C16
    g = cat.Grid(N, N, rule, kernel="tcgen05", dtype="fp8")
    rng = np.random.default_rng(100)
    try:
        g.set_state(inputs.bernoulli(N, N, 0.5, 1016))
        g.step(99)
        before = g.state_tensor().cpu().numpy().copy()
        g.step(1)
        assert g.status() == cat.CAT_OK
        after = g.state_tensor().cpu().numpy()
        counts = np.bincount(after.ravel(), minlength=16)
        # alive, and decaying cells in several states: the dynamics are not empty
        assert counts[1] > N * N // 50 and counts[2:].sum() > N * N // 50
        assert (counts[2:] > 0).sum() >= 10
        spots = [(0, 0), (0, N - 192), (N - 192, 0), (N - 192, N - 192)]
        spots += [tuple(int(v) for v in rng.integers(0, N - 192, 2)) for _ in range(8)]
        for y0, x0 in spots:
            ya, xa = max(0, y0 - 10), max(0, x0 - 10)
            win = before[ya:min(N, y0 + 202), xa:min(N, x0 + 202)]
            want = oracle.step(win, orule(rule))[y0 - ya:y0 - ya + 192, x0 - xa:x0 - xa + 192]
            got = after[y0:y0 + 192, x0:x0 + 192]
            assert np.array_equal(got, want), f"step 100 window ({y0},{x0}): {int((got != want).sum())} cells differ"
    finally:
        g.close()

"""Ordering of the one-step tcgen05 launches, which are programmatically
dependent on the previous kernel in the stream (a launch's set-up may overlap
the previous kernel's drain; it touches global memory only after
griddepcontrol.wait).

Checked against the CPU oracle, element by element:
* a torch kernel that rewrites a bound state buffer between two steps (a
  kernel without the trigger: the next step must see all of its writes), and
  a torch kernel reading the state right after a step;
* steps of different instances and kernel variants interleaved on one stream
  (FP8 standard and short window, FP4, von Neumann, four bits per cell), each
  grid stepped several times;
* the same sequence captured into a CUDA graph and replayed.
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


def test_foreign_kernels_between_steps(cat):
    import torch
    H, W, pitch = 1000, 1200, 1216
    rule = inputs.scaled_rule(9)
    grid = inputs.bernoulli(H, W, 0.5, 31)
    a = torch.zeros((H, pitch), dtype=torch.uint8, device="cuda")
    b = torch.zeros((H, pitch), dtype=torch.uint8, device="cuda")
    a[:, :W] = torch.from_numpy(grid).cuda()
    g = cat.Grid(H, W, rule, kernel="tcgen05", dtype="fp8")
    try:
        cat.cat_bind(g.handle, a.data_ptr(), b.data_ptr(), pitch)
        want = grid
        for k in range(6):
            g.step(1)                       # reads the buffer the torch kernel below wrote
            cur = b if k % 2 == 0 else a
            snap = cur[:, :W].clone()       # a torch kernel reading the state right after the step
            want = oracle.step(want, orule(rule))
            # rewrite a band of rows and a column stripe of the current state in place
            cur[100 + 50 * k:160 + 50 * k, :W] ^= 1
            cur[:, 7 * k:7 * k + 40] = 0
            torch.cuda.synchronize()
            assert np.array_equal(snap.cpu().numpy(), want), f"state after step {k + 1}"
            want = want.copy()
            want[100 + 50 * k:160 + 50 * k, :] ^= 1
            want[:, 7 * k:7 * k + 40] = 0
        g.step(1)
        torch.cuda.synchronize()
        assert g.status() == cat.CAT_OK
        assert np.array_equal(g.get_state(), oracle.step(want, orule(rule)))
    finally:
        g.close()


def _instances(cat):
    specs = [("fp8 r12", inputs.scaled_rule(12), dict(dtype="fp8"), 700, 900),
             ("fp8 short window r4", inputs.scaled_rule(4), dict(dtype="fp8"), 300, 1100),
             ("fp4 r16", inputs.scaled_rule(16), dict(dtype="fp4"), 520, 390),
             ("von Neumann r6", inputs.vn_scaled_rule(6), dict(dtype="fp8"), 400, 640),
             ("four bits C5", dict(r=3, C=5, M=0, s1=10, s2=30, b1=12, b2=25), dict(dtype="fp8", storage=cat.STORE_NIB4),
              260, 777)]
    out = []
    for i, (name, rule, opts, H, W) in enumerate(specs):
        if rule["C"] > 2:
            host = (inputs.uniform_states(H, W, rule["C"], 40 + i) * (inputs.bernoulli(H, W, 0.3, 50 + i) == 0)
                    + inputs.bernoulli(H, W, 0.3, 50 + i)).astype(np.uint8) % rule["C"]
        else:
            host = inputs.bernoulli(H, W, 0.5, 40 + i)
        out.append((name, rule, opts, host))
    return out


def test_interleaved_instances(cat):
    import torch
    inst = _instances(cat)
    grids = [cat.Grid(h.shape[0], h.shape[1], rule, kernel="tcgen05", **opts) for _, rule, opts, h in inst]
    try:
        for g, (_, _, _, h) in zip(grids, inst):
            g.set_state(h)
        for _ in range(4):
            for g in grids:
                g.step(1)
        grids[0].step(3)                    # one grid stepped back to back
        torch.cuda.synchronize()
        for g, (name, rule, _, h), n in zip(grids, inst, [7, 4, 4, 4, 4]):
            assert g.status() == cat.CAT_OK
            assert np.array_equal(g.get_state(), oracle.step(h, orule(rule), n_steps=n)), name
    finally:
        for g in grids:
            g.close()


def test_steps_under_graph_capture(cat):
    import torch
    inst = _instances(cat)
    grids = [cat.Grid(h.shape[0], h.shape[1], rule, kernel="tcgen05", **opts) for _, rule, opts, h in inst]
    try:
        for g, (_, _, _, h) in zip(grids, inst):
            g.set_state(h)
        s = torch.cuda.Stream()
        for g in grids:                     # kernels configured before capture
            g.step(2, s)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            for _ in range(2):              # even: each handle's buffer parity is unchanged
                for g in grids:
                    g.step(1, s)
        for _ in range(3):
            graph.replay()
        torch.cuda.synchronize()
        for g, (name, rule, _, h) in zip(grids, inst):
            assert g.status() == cat.CAT_OK
            assert np.array_equal(g.get_state(), oracle.step(h, orule(rule), n_steps=2 + 2 * 3)), name
    finally:
        for g in grids:
            g.close()

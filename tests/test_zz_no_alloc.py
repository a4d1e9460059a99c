"""The allocation-free batched step agrees with the allocating entry points.

cat_batch_step_static serves callers that cannot allocate device memory
themselves -- their own allocator already owns the memory budget, their
footprint is fixed up front, or a cudaMalloc/cudaFree (which can synchronise
the device) is not acceptable where they run.  It keeps its tile work-list in
a fixed array inside the library and writes into buffers the caller owns.

Here the caller's buffers come from torch.  Each batch is advanced by two
calls in a row (in -> out, then out -> in) through the C ABI, and after each
call every grid must equal, bit for bit, the state that cat_step reaches on an
ordinary instance; after the first call it must also equal the CPU oracle's
step.  A batch of exactly CAT_STATIC_MAX_GRIDS small grids is checked against
the oracle too, and the rejections (no status word, overlapping buffers, a
capturing stream, oversized batches) are checked to launch nothing.  The file
is named so that pytest collects it last.
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


def batch_cases(multistate):
    rng = np.random.default_rng(77 if multistate else 76)
    shapes = [(1, 1), (1, 300), (129, 257), (300, 200), (64, 64), (250, 131), (517, 90), (128, 128)]
    out = []
    for i, (H, W) in enumerate(shapes):
        r = [1, 3, 7, 8, 12, 16, 5, 10][i]
        M = int(rng.integers(0, 2))
        if multistate and i % 3 == 0:
            C = 16
            rule = inputs.scaled_rule(r, M, C)
            grid = inputs.uniform_states(H, W, C, 300 + i)
        else:
            rule = inputs.scaled_rule(r, M)
            grid = inputs.bernoulli(H, W, float(rng.uniform(0.25, 0.55)), 200 + i)
        out.append((grid, rule))
    return out


def orule(d):
    return oracle.Rule(d["r"], d["C"], d["M"], d["s1"], d["s2"], d["b1"], d["b2"])


def make_descs(cat, cases):
    """Caller-owned torch buffers (input filled, output zero) and their descriptors."""
    import torch
    bufs, descs = [], []
    for grid, rule in cases:
        H, W = grid.shape
        pitch = (W + 15) // 16 * 16
        a = torch.zeros((H, pitch), dtype=torch.uint8, device="cuda")
        b = torch.zeros((H, pitch), dtype=torch.uint8, device="cuda")
        a[:, :W] = torch.from_numpy(grid).cuda()
        bufs.append((a, b))
        d = cat.cat_grid_desc_t()
        d.H, d.W, d.pitch = H, W, pitch
        d.rule = cat.make_rule(**{k: rule[k] for k in ("r", "C", "M", "s1", "s2", "b1", "b2")})
        d.in_, d.out = a.data_ptr(), b.data_ptr()
        descs.append(d)
    return bufs, descs


def reference_states(cat, grid, rule, dtype, steps):
    g = cat.Grid(grid.shape[0], grid.shape[1], rule, kernel="tcgen05", dtype=dtype)
    try:
        g.set_state(grid)
        states = []
        for _ in range(steps):
            g.step(1)
            states.append(g.get_state())
        return states
    finally:
        g.close()


@pytest.mark.parametrize("dtype", ["fp8", "fp16"])
@pytest.mark.parametrize("multistate", [False, True], ids=["C2", "mixedC"])
def test_static_batch_matches_cat_step_on_two_calls(cat, dtype, multistate):
    import torch
    cases = batch_cases(multistate)
    bufs, descs = make_descs(cat, cases)
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    want = [reference_states(cat, g, rule, dtype, 2) for g, rule in cases]
    torch.cuda.synchronize()
    for call in range(2):
        for d, (a, b) in zip(descs, bufs):
            src, dst = (a, b) if call == 0 else (b, a)
            d.in_, d.out = src.data_ptr(), dst.data_ptr()
        rc = cat.cat_batch_step_static(descs, cat.DTYPES[dtype], status.data_ptr())
        assert rc == cat.CAT_OK, cat.load().cat_last_error()
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        for i, ((grid, rule), (a, b)) in enumerate(zip(cases, bufs)):
            dst = b if call == 0 else a
            got = dst[:, : grid.shape[1]].cpu().numpy()
            assert np.array_equal(got, want[i][call]), f"call {call}, grid {i} {grid.shape} {rule}"
            if call == 0:
                assert np.array_equal(got, oracle.step(grid, orule(rule))), f"oracle, grid {i} {grid.shape} {rule}"


def test_static_batch_at_the_grid_limit_vs_oracle(cat):
    """Exactly CAT_STATIC_MAX_GRIDS small grids (every radius, both M, ragged
    shapes) in one call, each compared with the oracle."""
    import torch
    rng = np.random.default_rng(256)
    cases = []
    for i in range(cat.CAT_STATIC_MAX_GRIDS):
        H, W = (int(v) for v in rng.integers(1, 72, 2))
        rule = inputs.scaled_rule(1 + i % 16, (i // 16) % 2)
        cases.append((inputs.bernoulli(H, W, float(rng.uniform(0.2, 0.6)), 4000 + i), rule))
    bufs, descs = make_descs(cat, cases)
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    assert cat.cat_batch_step_static(descs, cat.DTYPE_FP8_E4M3, status.data_ptr()) == cat.CAT_OK
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    for i, ((grid, rule), (_, b)) in enumerate(zip(cases, bufs)):
        got = b[:, : grid.shape[1]].cpu().numpy()
        assert np.array_equal(got, oracle.step(grid, orule(rule))), f"grid {i} {grid.shape} {rule}"


def test_static_batch_rejections_launch_nothing(cat):
    import torch
    cases = batch_cases(False)[:3]
    bufs, descs = make_descs(cat, cases)
    status = torch.zeros((1,), dtype=torch.int32, device="cuda")
    outs_before = [b.clone() for _, b in bufs]
    # no status word: a timeout could not be reported
    assert cat.cat_batch_step_static(descs, cat.DTYPE_FP8_E4M3, None) == cat.CAT_ERR_INVALID_ARG
    assert b"d_status" in cat.load().cat_last_error()
    # grid 1 writes into grid 2's input
    d1_out = descs[1].out
    descs[1].out = descs[2].in_ + 16
    assert cat.cat_batch_step_static(descs, cat.DTYPE_FP8_E4M3, status.data_ptr()) == cat.CAT_ERR_INVALID_ARG
    assert b"also uses" in cat.load().cat_last_error()
    # two grids write the same output
    descs[1].out = descs[2].out
    assert cat.cat_batch_step_static(descs, cat.DTYPE_FP8_E4M3, status.data_ptr()) == cat.CAT_ERR_INVALID_ARG
    descs[1].out = d1_out
    # a capturing stream
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        rc = cat.cat_batch_step_static(descs, cat.DTYPE_FP8_E4M3, status.data_ptr(), stream=side)
    assert rc == cat.CAT_ERR_INVALID_ARG
    assert b"captured" in cat.load().cat_last_error()
    torch.cuda.synchronize()
    for (_, b), before in zip(bufs, outs_before):
        assert torch.equal(b, before)


def test_static_batch_rejects_oversized_batches(cat):
    d = cat.cat_grid_desc_t()
    d.in_, d.out, d.H, d.W, d.pitch = 256, 512, 8, 8, 16
    d.rule = cat.make_rule(**inputs.CONWAY)
    too_many = [d] * (cat.CAT_STATIC_MAX_GRIDS + 1)
    assert cat.cat_batch_step_static(too_many, status_ptr=1024) == cat.CAT_ERR_INVALID_ARG
    assert b"static limit" in cat.load().cat_last_error()
    big = cat.cat_grid_desc_t()
    big.in_, big.out, big.H, big.W, big.pitch = 256, 512, 33000, 33000, 33008
    big.rule = cat.make_rule(**inputs.CONWAY)
    assert cat.cat_batch_step_static([big], status_ptr=1024) == cat.CAT_ERR_INVALID_ARG
    assert b"tiles" in cat.load().cat_last_error()

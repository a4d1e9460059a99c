"""The allocation-free batched step agrees with the allocating entry points.

cat_batch_step_static serves callers that cannot allocate device memory
themselves -- their own allocator already owns the memory budget, their
footprint is fixed up front, or a cudaMalloc/cudaFree (which can synchronise
the device) is not acceptable where they run.  It keeps its tile work-list in
a fixed array inside the library and writes into buffers the caller owns.

Here the caller's buffers come from torch.  Each batch is advanced by two
calls in a row (in -> out, then out -> in) through the C ABI, and after each
call every grid must equal, bit for bit, the state that cat_step reaches on an
ordinary instance.  The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

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
        descs.append(d)
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


def test_static_batch_rejects_oversized_batches(cat):
    d = cat.cat_grid_desc_t()
    d.in_, d.out, d.H, d.W, d.pitch = 256, 512, 8, 8, 16
    d.rule = cat.make_rule(**inputs.CONWAY)
    too_many = [d] * (cat.CAT_STATIC_MAX_GRIDS + 1)
    assert cat.cat_batch_step_static(too_many) == cat.CAT_ERR_INVALID_ARG
    assert b"static limit" in cat.load().cat_last_error()
    big = cat.cat_grid_desc_t()
    big.in_, big.out, big.H, big.W, big.pitch = 256, 512, 33000, 33000, 33008
    big.rule = cat.make_rule(**inputs.CONWAY)
    assert cat.cat_batch_step_static([big]) == cat.CAT_ERR_INVALID_ARG
    assert b"tiles" in cat.load().cat_last_error()

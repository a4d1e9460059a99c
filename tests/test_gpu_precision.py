"""Operand precisions on the 32768^2 workload: p = 0.35, the scaled rule (C2 M1),
r in {1, 5, 10, 16}, 50 steps from the same seeded state with the tcgen05 FP8
kernel (e4m3 operands) and the tcgen05 FP4 kernel (e2m1 pass-1 operands, e4m3
digits in pass 2), each on uint8 and on one-bit storage, the tcgen05 FP16
kernel and the INT8 fragment kernel (mma.sync m16n8k32; sm_103a has no tcgen05
kind::i8).  All six must hold the same grid, bit for bit (the one-bit grids
compared as packed rows), after 49 and after 50 steps, and step 50 is checked
against the oracle on 64 random 256 x 256 windows (Sec. V-A: the method is
exact, so every precision reaches the one correct result).
"""
import numpy as np
import pytest

from oracle import oracle
from paper_2406_17284_gb300 import inputs

pytestmark = pytest.mark.gpu

N, STEPS, WINDOWS, WIN = 32768, 50, 64, 256
KERNELS = [("tcgen05", "fp8"), ("tcgen05", "fp16"), ("mma_sync", "int8"), ("tcgen05", "fp4")]


def pack_rows(t):
    """uint8 0/1 cells (H x W, W % 8 == 0) -> one bit per cell, lowest x in the lowest bit."""
    import torch
    w = torch.tensor([1, 2, 4, 8, 16, 32, 64, 128], dtype=torch.int32, device=t.device)
    return (t.reshape(t.shape[0], -1, 8).to(torch.int32) * w).sum(-1).to(torch.uint8)


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


@pytest.mark.parametrize("r", [1, 5, 10, 16])
def test_precisions_agree_and_match_oracle_32768(cat, r):
    import torch
    rule = inputs.scaled_rule(r, M=1)
    orl = oracle.Rule(**{k: rule[k] for k in ("r", "C", "M", "s1", "s2", "b1", "b2")})
    init = inputs.bernoulli(N, N, 0.35, 3200 + r)
    grids = [cat.Grid(N, N, rule, kernel=k, dtype=d) for k, d in KERNELS]
    bits = [cat.Grid(N, N, rule, kernel="tcgen05", dtype=d, storage=cat.STORE_BIT1) for d in ("fp8", "fp4")]
    grids += bits
    try:
        for g in grids:
            g.set_state(init)
        del init
        for g in grids:
            g.step(STEPS - 1)
        ref = grids[0].state_tensor()
        for g, (k, d) in zip(grids[1:], KERNELS[1:]):
            assert torch.equal(g.state_tensor(), ref), f"{k}/{d} differs from tcgen05/fp8 after {STEPS - 1} steps"
        for b, d in zip(bits, ("fp8", "fp4")):
            assert torch.equal(b.state_tensor(), pack_rows(ref)), f"one-bit storage ({d}) differs after {STEPS - 1} steps"
        rng = np.random.default_rng(r)
        pos = [tuple(int(v) for v in rng.integers(0, N - WIN, 2)) for _ in range(WINDOWS)]
        pos[:4] = [(0, 0), (0, N - WIN), (N - WIN, 0), (N - WIN, N - WIN)]   # the four corners
        befores = []
        for y0, x0 in pos:
            ya, xa = max(0, y0 - r), max(0, x0 - r)
            befores.append((ya, xa, ref[ya:min(N, y0 + WIN + r), xa:min(N, x0 + WIN + r)].cpu().numpy()))
        for g in grids:
            g.step(1)
            assert g.status() == cat.CAT_OK
        ref = grids[0].state_tensor()
        for g, (k, d) in zip(grids[1:], KERNELS[1:]):
            assert torch.equal(g.state_tensor(), ref), f"{k}/{d} differs from tcgen05/fp8 after {STEPS} steps"
        for b, d in zip(bits, ("fp8", "fp4")):
            assert torch.equal(b.state_tensor(), pack_rows(ref)), f"one-bit storage ({d}) differs after {STEPS} steps"
        for (y0, x0), (ya, xa, win) in zip(pos, befores):
            want = oracle.step(win, orl)[y0 - ya:y0 - ya + WIN, x0 - xa:x0 - xa + WIN]
            got = ref[y0:y0 + WIN, x0:x0 + WIN].cpu().numpy()
            if not np.array_equal(got, want):
                bad = np.argwhere(got != want)
                raise AssertionError(f"r={r} window ({y0},{x0}): {len(bad)} cells differ from the oracle")
        assert int(ref.sum()) > 0, "the grid died out; the check would be vacuous"
    finally:
        for g in grids:
            g.close()

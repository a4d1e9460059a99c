"""cat_bind: an instance stepping two caller-owned device buffers (torch tensors).

The state is read from the first buffer as it is, steps alternate between the
two (as cat_state_ptr reports), results match the CPU oracle, and the buffers
stay the caller's after cat_destroy.
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


@pytest.mark.parametrize("kernel,dtype,k", [("tcgen05", "fp8", 1), ("tcgen05", "fp8", 3), ("tcgen05", "fp16", 1),
                                            ("mma_sync", "fp16", 1), ("stencil", "auto", 1),
                                            ("runsum", "auto", 1)])
def test_steps_on_torch_buffers(cat, kernel, dtype, k):
    import torch
    H, W, pitch = 333, 517, 544            # pitch above the minimum, a multiple of 16
    rule = inputs.scaled_rule(7)
    grid = inputs.bernoulli(H, W, 0.5, 90)
    a = torch.zeros((H, pitch), dtype=torch.uint8, device="cuda")
    b = torch.full((H, pitch), 7, dtype=torch.uint8, device="cuda")   # garbage the step must overwrite
    a[:, :W] = torch.from_numpy(grid).cuda()
    g = cat.Grid(H, W, rule, kernel=kernel, dtype=dtype, steps_per_launch=k)
    try:
        cat.cat_bind(g.handle, a.data_ptr(), b.data_ptr(), pitch)
        assert cat.cat_state_ptr(g.handle) == (a.data_ptr(), pitch)
        g.step(1)
        torch.cuda.synchronize()
        assert g.status() == cat.CAT_OK
        assert cat.cat_state_ptr(g.handle)[0] == b.data_ptr()
        assert np.array_equal(b[:, :W].cpu().numpy(), oracle.step(grid, orule(rule)))
        g.step(4)
        torch.cuda.synchronize()
        assert g.status() == cat.CAT_OK
        assert cat.cat_state_ptr(g.handle)[0] == b.data_ptr()
        want = oracle.step(grid, orule(rule), n_steps=5)
        assert np.array_equal(b[:, :W].cpu().numpy(), want)
        assert np.array_equal(g.get_state(), want)
    finally:
        g.close()
    a.fill_(3)                              # still the caller's memory
    torch.cuda.synchronize()
    assert int(a[0, 0]) == 3


def test_rejections(cat):
    import torch
    rule = inputs.scaled_rule(3)
    a = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    b = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    g = cat.Grid(64, 64, rule, boundary=cat.BOUNDARY_PERIODIC)
    try:
        with pytest.raises(cat.CatError) as e:
            cat.cat_bind(g.handle, a.data_ptr(), b.data_ptr(), 64)
        assert e.value.code == cat.CAT_ERR_UNSUPPORTED
    finally:
        g.close()
    g = cat.Grid(64, 60, rule)
    try:
        for args in ((a.data_ptr(), b.data_ptr(), 40), (a.data_ptr(), a.data_ptr(), 64),
                     (a.data_ptr(), b.data_ptr(), 56)):
            with pytest.raises(cat.CatError) as e:
                cat.cat_bind(g.handle, *args)
            assert e.value.code == cat.CAT_ERR_INVALID_ARG, args
        host = np.zeros((64, 64), np.uint8)
        with pytest.raises(cat.CatError) as e:
            cat.cat_bind(g.handle, host.ctypes.data, b.data_ptr(), 64)
        assert e.value.code == cat.CAT_ERR_INVALID_ARG
        cat.cat_bind(g.handle, a.data_ptr(), b.data_ptr(), 64)
        with pytest.raises(cat.CatError) as e:
            cat.cat_set_options(g.handle, cat.KERNEL_TCGEN05, cat.DTYPE_FP8_E4M3, cat.STORE_BIT1)
        assert e.value.code == cat.CAT_ERR_UNSUPPORTED
    finally:
        g.close()

"""Single-kernel workloads for profiling: one grid, a few launches of one kernel.

    python -m paper_2406_17284_gb300.profile_cases <case> [--size N] [--steps K]

Each case builds one seeded synthetic grid (16384 x 16384 by default, the
radius sweep's size), sets it and steps it K times (default 3) through the C
ABI, so that a profiler can skip the first launches and capture one, e.g.
``ncu --set full --clock-control none -k regex:ltl_wide -s 2 -c 1 python -m
paper_2406_17284_gb300.profile_cases wide_r24``.  The grid is Bernoulli(0.5)
(two-state rules) or, for the multi-state case, states 0/1 with a quarter of
the cells in the decaying states 12..15.
"""
from __future__ import annotations

import argparse
import sys

import numpy as np

from . import build, cat, inputs

CASES = {
    # name: (rule, Grid options, kernel name a profiler filters on)
    "fp8_r16": (inputs.scaled_rule(16), dict(kernel="tcgen05", dtype="fp8"), "ltl_tc_kernel"),
    "fp8_r4": (inputs.scaled_rule(4), dict(kernel="tcgen05", dtype="fp8"), "ltl_tc_kernel"),
    "fp16_r16": (inputs.scaled_rule(16), dict(kernel="tcgen05", dtype="fp16"), "ltl_tc_kernel"),
    "vn_r16": (inputs.vn_scaled_rule(16), dict(kernel="tcgen05", dtype="fp8"), "ltl_vn_kernel"),
    "bits_r16": (inputs.scaled_rule(16), dict(kernel="tcgen05", dtype="fp8", storage=cat.STORE_BIT1), "ltl_bits_kernel"),
    "wide_r24": (inputs.scaled_rule(24), dict(kernel="tcgen05", dtype="fp8", tile=96), "ltl_wide_kernel"),
    "big_r24": (inputs.scaled_rule(24), dict(kernel="tcgen05", dtype="fp8"), "ltl_big_kernel"),
    "big_r20": (inputs.scaled_rule(20), dict(kernel="tcgen05", dtype="fp8"), "ltl_big16_kernel"),
    "nib_c16": (inputs.MULTISTATE_R10_C16, dict(kernel="tcgen05", dtype="fp8", storage=cat.STORE_NIB4), "ltl_nib_kernel"),
    "fp4_r16": (inputs.scaled_rule(16), dict(kernel="tcgen05", dtype="fp4"), "ltl_fp4_kernel"),
    "bitslice_r1": (inputs.scaled_rule(1), dict(kernel="bitslice", storage=cat.STORE_BIT1), "ltl_swar_kernel"),
    "bitslice_r2": (inputs.scaled_rule(2), dict(kernel="bitslice", storage=cat.STORE_BIT1), "ltl_swar_kernel"),
    "runsum_r8": (inputs.scaled_rule(8), dict(kernel="runsum", dtype="auto"), "runsum_kernel"),
    "stencil_r1": (inputs.scaled_rule(1), dict(kernel="stencil", dtype="auto"), "smem_stencil_kernel"),
}


def initial(rule: dict, n: int) -> np.ndarray:
    if rule["C"] > 2:
        g = inputs.bernoulli(n, n, 0.5, 77)
        u = inputs.uniform_states(n, n, 16, 78)
        return np.where(u >= 12, u, g).astype(np.uint8) % rule["C"]
    return inputs.bernoulli(n, n, 0.5, 2024)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=sorted(CASES))
    ap.add_argument("--size", type=int, default=16384)
    ap.add_argument("--steps", type=int, default=3)
    a = ap.parse_args(argv)
    import torch
    build.build()
    cat.load()
    rule, opts, _ = CASES[a.case]
    g = cat.Grid(a.size, a.size, rule, **opts)
    try:
        g.set_state(initial(rule, a.size))
        for _ in range(a.steps):
            g.step(1)
        torch.cuda.synchronize()
        rc = g.status()
    finally:
        g.close()
    print(f"{a.case}: {a.size}x{a.size}, {a.steps} launches, status {rc}")
    return 0 if rc == cat.CAT_OK else 1


if __name__ == "__main__":
    sys.exit(main())

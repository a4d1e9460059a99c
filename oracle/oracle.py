"""CPU oracle for the Larger-than-Life step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this module.  It never imports the CUDA package and the CUDA package
never imports it; the two sides share only the seeded input generators.

The arithmetic lives in ``ltl_oracle.c`` (a plain per-cell (2r+1)^2 loop, see its
header for the passages of the CAT paper it follows: Sec. IV Eqs. 1-2 for the
box count, Eq. 3 for the simplified von Neumann count, Sec. V-A for the
R C M S B N rule).  This file compiles it with gcc
and marshals numpy arrays into it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ltl_oracle.c")
_LIB_NAME = "liboracle.so"

ZERO = 0
PERIODIC = 1


@dataclass(frozen=True)
class Rule:
    """LTL rule R_r C_c M_m S_{s1..s2} B_{b1..b2} N_n (Sec. V-A notation); nbhd "M" is
    the Moore box, "N" the simplified von Neumann cross of Eq. 3."""

    r: int
    C: int
    M: int
    s1: int
    s2: int
    b1: int
    b2: int
    nbhd: str = "M"


class _CRule(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("r", "C", "M", "s1", "s2", "b1", "b2", "nbhd")]


def _crule(rule: Rule) -> _CRule:
    if rule.nbhd not in ("M", "N"):
        raise ValueError(f"unknown neighbourhood {rule.nbhd!r}")
    return _CRule(rule.r, rule.C, rule.M, rule.s1, rule.s2, rule.b1, rule.b2, 1 if rule.nbhd == "N" else 0)


def compile_oracle(out_dir: str | None = None, mutation: int = 0) -> str:
    """Compile ``ltl_oracle.c`` into a shared library and return its path.

    ``mutation`` > 0 plants one of the known mistakes of the C source (used only
    by the tests that show the pins catch such mistakes).
    """
    out_dir = out_dir or _HERE
    name = _LIB_NAME if mutation == 0 else f"liboracle_mut{mutation}.so"
    path = os.path.join(out_dir, name)
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           f"-DORACLE_MUTATION={int(mutation)}", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


_lib = None
_lock = threading.Lock()


def _bind(lib):
    i64, i32, p = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
    lib.oracle_box_sums.argtypes = [p, i64, i64, i64, i32, i32, p, i64]
    lib.oracle_cross_sums.argtypes = [p, i64, i64, i64, i32, i32, p, i64]
    lib.oracle_step.argtypes = [p, p, i64, i64, i64, ctypes.POINTER(_CRule), i32]
    lib.oracle_run.argtypes = [p, i64, i64, i64, ctypes.POINTER(_CRule), i32, i64]
    for f in (lib.oracle_box_sums, lib.oracle_cross_sums, lib.oracle_step, lib.oracle_run,
              lib.oracle_num_threads):
        f.restype = ctypes.c_int
    return lib


def load(path: str | None = None):
    """Load (building if needed) the oracle library; ``path`` selects a variant."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            so = os.path.join(_HERE, _LIB_NAME)
            if (not os.path.exists(so)) or os.path.getmtime(so) < os.path.getmtime(_SRC):
                compile_oracle()
            _lib = _bind(ctypes.CDLL(so))
    return _lib


def _grid(g: np.ndarray) -> np.ndarray:
    g = np.ascontiguousarray(g, dtype=np.uint8)
    if g.ndim != 2:
        raise ValueError("grid must be 2-D")
    return g


def box_sums(grid: np.ndarray, r: int, boundary: int = ZERO, lib=None, nbhd: str = "M") -> np.ndarray:
    """L(y,x): state-1 cells in the (2r+1)^2 Moore box (centre included), or with
    nbhd "N" on the vertical plus the horizontal segment (Eq. 3, centre twice)."""
    lib = lib or load()
    g = _grid(grid)
    H, W = g.shape
    S = np.empty((H, W), dtype=np.int32)
    fn = lib.oracle_cross_sums if nbhd == "N" else lib.oracle_box_sums
    rc = fn(g.ctypes.data, H, W, W, int(r), int(boundary), S.ctypes.data, W)
    if rc != 0:
        raise ValueError(f"oracle_box_sums failed ({rc})")
    return S


def step(grid: np.ndarray, rule: Rule, boundary: int = ZERO, n_steps: int = 1, lib=None) -> np.ndarray:
    """Grid after ``n_steps`` synchronous LTL steps (returns a new array)."""
    lib = lib or load()
    g = _grid(grid).copy()
    H, W = g.shape
    cr = _crule(rule)
    rc = lib.oracle_run(g.ctypes.data, H, W, W, ctypes.byref(cr), int(boundary), int(n_steps))
    if rc != 0:
        raise ValueError(f"oracle_run failed ({rc})")
    return g


def num_threads(lib=None) -> int:
    return int((lib or load()).oracle_num_threads())

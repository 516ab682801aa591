"""Driver for the C bucket elimination of ve.c (test infrastructure only).

ve_amplitude(circ, x, order, slices) evaluates <x|C|0> as Section 3.B describes: build
the graphical model (graph.build), substitute the inputs and outputs, split the sum over
the 2^k values of the sliced variables (Section 3.B.2), eliminate the remaining variables
in the given order (Section 3.B.1) and add the slice terms.
"""
import ctypes
import math
import os
import subprocess

import numpy as np

from . import graph as GR

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "_oracle_ve.so")
_lib = None


def build_library(force: bool = False) -> str:
    """Compile ve.c into oracle/_oracle_ve.so with gcc and OpenMP."""
    src = os.path.join(_HERE, "ve.c")
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(src):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               src, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_library())
        f = _lib.oracle_ve
        P = ctypes.c_void_p
        f.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P, P, ctypes.c_int, P,
                      ctypes.c_int, P, ctypes.c_long, P, P, ctypes.c_int, ctypes.c_int]
        f.restype = ctypes.c_int
    return _lib


def _flat(data: np.ndarray) -> np.ndarray:
    """Entries with bit j of the flat index = axis j (axis 0 least significant)."""
    r = data.ndim
    return np.ascontiguousarray(data.transpose(tuple(range(r - 1, -1, -1)))).reshape(-1)


def slice_terms(circ, x: int, order, slices, slice_ids=None, max_rank: int = 30,
                threads: int = 0, model=None):
    """Per-slice terms beta_s (complex128 array) for the requested slice numbers."""
    model = model if model is not None else GR.build(circ)
    tens, scalar = GR.restricted_tensors(model, x)
    n_vars = len(model.variables)
    slices = [int(v) for v in slices]
    order = [int(v) for v in order]
    if slice_ids is None:
        slice_ids = np.arange(1 << len(slices), dtype=np.int64)
    slice_ids = np.ascontiguousarray(slice_ids, dtype=np.int64)
    rank = np.array([len(ids) for ids, _ in tens], dtype=np.int32)
    var_off = np.zeros(len(tens), dtype=np.int32)
    var_off[1:] = np.cumsum(rank)[:-1]
    vars_ = np.array([v for ids, _ in tens for v in ids], dtype=np.int32)
    flats = [_flat(d) for _, d in tens]
    sizes = np.array([f.size for f in flats], dtype=np.int64)
    data_off = np.zeros(len(tens), dtype=np.int64)
    data_off[1:] = np.cumsum(sizes)[:-1]
    data = np.ascontiguousarray(np.concatenate(flats) if flats else np.zeros(1, np.complex128))
    o = np.array(order, dtype=np.int32) if order else np.zeros(1, np.int32)
    s = np.array(slices, dtype=np.int32) if slices else np.zeros(1, np.int32)
    out = np.zeros(2 * len(slice_ids), dtype=np.float64)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    st = _load().oracle_ve(n_vars, len(tens), vp(rank), vp(var_off),
                           vp(vars_ if vars_.size else np.zeros(1, np.int32)), vp(data_off),
                           vp(data), len(order), vp(o), len(slices), vp(s), len(slice_ids),
                           vp(slice_ids), vp(out), max_rank, threads)
    if st != 0:
        raise RuntimeError({1: "out of memory", 2: "tensor rank above the cap",
                            3: "order and slices must cover every variable exactly once",
                            4: "a variable was left uneliminated"}.get(st, f"status {st}"))
    return scalar * (out[0::2] + 1j * out[1::2])


def exact_sum(terms) -> complex:
    """Correctly rounded sum of complex terms (math.fsum on each part)."""
    terms = np.asarray(terms)
    return complex(math.fsum(terms.real.tolist()), math.fsum(terms.imag.tolist()))


def ve_amplitude(circ, x: int, order=None, slices=(), threads: int = 0, max_rank: int = 30,
                 model=None) -> complex:
    """<x|C|0> by variable elimination; order defaults to the canonical numbering."""
    model = model if model is not None else GR.build(circ)
    slices = list(slices)
    if order is None:
        ss = set(slices)
        order = [v for v in range(len(model.variables)) if v not in ss]
    return exact_sum(slice_terms(circ, x, order, slices, None, max_rank, threads, model))

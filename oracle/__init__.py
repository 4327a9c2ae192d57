"""Oracle for flooding Min-Sum decoding (arXiv 2507.10424) -- TEST INFRASTRUCTURE ONLY.

A plain, slow CPU implementation written from the paper (Algorithm 1 in graph form with
the check update of eq. (eta_update) taken literally or through Observations 1-2, and
Algorithm 2 in dense masked form). It shares no code with the CUDA path. Only the test
suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may use it; the
product path never does.

Parity status of each function (what pins it, see tests/test_oracle_pins.py):
* ``syndrome``              -- pinned: Tanner example of Section II-A (all 1024 vectors),
                               Fig. 1 single parity check, GF(2) brute force.
* ``check_row``             -- pinned: literal eq. (eta_update) vs Observations 1-2,
                               degree-2 and degree-3 closed forms.
* ``decode_f32/f64/fixed``  -- pinned: exact max-marginals on cycle-free graphs, codeword
                               invariants, power-of-two scaling, channel symmetry, binary64
                               error bound, fixed/float cross-mode identity.
* ``decode_dense_f32``      -- pinned: identical to the graph form (Algorithms 1 and 2).
* ``quantize``              -- pinned: closed-form table of the rounding/clamping rule.
* ``decode_weighted_f32/f64`` (normalised/offset Min-Sum with learned weights, an
  extension of eq. eta_update) -- pinned: unit weights equal plain Min-Sum bit for bit,
  single-check closed form, a silencing offset, reuse of the last table row, agreement
  of the binary64 C and PyTorch implementations (tests/test_learned_oracle.py).
* ``learned_ref`` (PyTorch, autograd) -- pinned: its forward against the C oracle in
  binary64, its gradient against central finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "minsum_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

CHECK_TWOMIN = 0
CHECK_BRUTE = 1
PAPER_SLICER = 1
SAT = 32767


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, binary32 without contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.orc_graph_create.argtypes = [i32, i32, i64, P, P, ctypes.POINTER(P)]
        L.orc_graph_from_dense.argtypes = [i32, i32, P, ctypes.POINTER(P)]
        L.orc_graph_free.argtypes = [P]
        L.orc_graph_edges.argtypes = [P]
        L.orc_graph_edges.restype = i64
        L.orc_syndrome.argtypes = [P, P, P]
        L.orc_syndrome.restype = i64
        for name in ("orc_check_row_f32", "orc_check_row_f64", "orc_check_row_i32"):
            getattr(L, name).argtypes = [ctypes.c_int, i64, P, P]
        L.orc_quantize.argtypes = [P, i64, P]
        for name in ("orc_decode_f32", "orc_decode_f64", "orc_decode_fixed"):
            getattr(L, name).argtypes = [P, P, i64, i32, i32, i32, i32, i32, i32, P, P, P, P]
        for name in ("orc_trace_f32", "orc_trace_fixed"):
            getattr(L, name).argtypes = [P, P, i32, i32, i32, i32, i32, P, P, P, P, P]
        L.orc_decode_dense_f32.argtypes = [i32, i32, P, P, i32, i32, i32, P, P, P, P]
        L.orc_decode_weighted_f32.argtypes = [P, P, i64, i32, i32, i32, i32, P, i32, i32, P, P,
                                              P, P, P, P]
        L.orc_decode_weighted_f64.argtypes = [P, P, i64, i32, P, i32, i32, P, P, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


class Graph:
    """Check sets N_i and bit sets M_j of H (Section II-B), built by the oracle itself."""

    def __init__(self, M: int, N: int, rows=None, cols=None, dense=None):
        L = lib()
        h = ctypes.c_void_p()
        if dense is not None:
            H = np.ascontiguousarray(dense, dtype=np.uint8)
            rc = L.orc_graph_from_dense(M, N, _p(H), ctypes.byref(h))
        else:
            r = np.ascontiguousarray(rows, dtype=np.int32)
            c = np.ascontiguousarray(cols, dtype=np.int32)
            rc = L.orc_graph_create(M, N, r.shape[0], _p(r), _p(c), ctypes.byref(h))
        if rc != 0:
            raise ValueError(f"oracle rejected H (code {rc})")
        self.M, self.N, self.h = M, N, h
        self.E = int(L.orc_graph_edges(h))

    @classmethod
    def from_code(cls, code):
        return cls(code.M, code.N, rows=code.rows, cols=code.cols)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_graph_free(self.h)
            self.h = None


def syndrome(g: Graph, bits: np.ndarray):
    """Returns (number of unsatisfied checks, z uint8 [M])."""
    b = np.ascontiguousarray(bits, dtype=np.uint8)
    z = np.zeros(g.M, dtype=np.uint8)
    n = lib().orc_syndrome(g.h, _p(b), _p(z))
    return int(n), z


def check_row(lam: np.ndarray, variant: int = CHECK_TWOMIN) -> np.ndarray:
    """One check node's outgoing messages from its incoming lambda values."""
    lam = np.ascontiguousarray(lam)
    out = np.empty_like(lam)
    fn = {np.dtype(np.float32): lib().orc_check_row_f32, np.dtype(np.float64): lib().orc_check_row_f64,
          np.dtype(np.int32): lib().orc_check_row_i32}[lam.dtype]
    fn(variant, lam.shape[0], _p(lam), _p(out))
    return out


def quantize(llr: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(llr, dtype=np.float32)
    q = np.empty(x.shape, dtype=np.int8)
    lib().orc_quantize(_p(x), x.size, _p(q))
    return q


def _decode(fn, g, inp, soft_dtype, L, early_stop, check_every, variant, flags, threads, want_soft):
    inp = np.ascontiguousarray(inp)
    if inp.ndim == 1:
        inp = inp[None, :]
    F = inp.shape[0]
    assert inp.shape[1] == g.N
    bits = np.zeros((F, g.N), dtype=np.uint8)
    iters = np.zeros(F, dtype=np.int32)
    ok = np.zeros(F, dtype=np.uint8)
    soft = np.zeros((F, g.N), dtype=soft_dtype) if want_soft else None
    if threads is None:
        threads = os.cpu_count() or 1
    rc = fn(g.h, _p(inp), F, L, int(early_stop), check_every, variant, flags, threads,
            _p(bits), _p(iters), _p(ok), _p(soft))
    if rc != 0:
        raise RuntimeError(f"oracle decode failed ({rc})")
    return bits, iters, ok, soft


def decode_f32(g, llr, L, early_stop=True, check_every=1, variant=CHECK_TWOMIN, flags=0,
               threads=None, soft=True):
    """Algorithm 1 in binary32. Returns (bits [F][N], iters [F], ok [F], s [F][N])."""
    return _decode(lib().orc_decode_f32, g, np.asarray(llr, np.float32), np.float32, L, early_stop,
                   check_every, variant, flags, threads, soft)


def decode_f64(g, llr, L, early_stop=True, check_every=1, variant=CHECK_TWOMIN, flags=0,
               threads=None, soft=True):
    """Algorithm 1 in binary64."""
    return _decode(lib().orc_decode_f64, g, np.asarray(llr, np.float64), np.float64, L, early_stop,
                   check_every, variant, flags, threads, soft)


def decode_fixed(g, q, L, early_stop=True, check_every=1, variant=CHECK_TWOMIN, flags=0,
                 threads=None, soft=True):
    """Algorithm 1 in saturating fixed point from int8 LLRs (step 0.25). s is int16."""
    return _decode(lib().orc_decode_fixed, g, np.asarray(q, np.int8), np.int16, L, early_stop,
                   check_every, variant, flags, threads, soft)


def trace_f32(g, llr, L, early_stop=False, check_every=1, variant=CHECK_TWOMIN, flags=0):
    """One frame; returns (bits, iters, ok, eta [L][E], s [L][N]); edges in row-major order."""
    r = np.ascontiguousarray(llr, dtype=np.float32)
    bits = np.zeros(g.N, np.uint8)
    it, ok = ctypes.c_int32(), ctypes.c_uint8()
    eta = np.zeros((max(L, 1), g.E), np.float32)
    s = np.zeros((max(L, 1), g.N), np.float32)
    rc = lib().orc_trace_f32(g.h, _p(r), L, int(early_stop), check_every, variant, flags, _p(bits),
                             ctypes.byref(it), ctypes.byref(ok), _p(eta), _p(s))
    assert rc == 0
    return bits, it.value, ok.value, eta, s


def trace_fixed(g, q, L, early_stop=False, check_every=1, variant=CHECK_TWOMIN, flags=0):
    qq = np.ascontiguousarray(q, dtype=np.int8)
    bits = np.zeros(g.N, np.uint8)
    it, ok = ctypes.c_int32(), ctypes.c_uint8()
    eta = np.zeros((max(L, 1), g.E), np.int16)
    s = np.zeros((max(L, 1), g.N), np.int16)
    rc = lib().orc_trace_fixed(g.h, _p(qq), L, int(early_stop), check_every, variant, flags,
                               _p(bits), ctypes.byref(it), ctypes.byref(ok), _p(eta), _p(s))
    assert rc == 0
    return bits, it.value, ok.value, eta, s


def column_classes(code):
    """Class of each bit for learned weights: index of its column weight among the sorted
    distinct column weights (a single class for a regular code)."""
    w = code.col_weights()
    degrees = np.unique(w)
    return np.searchsorted(degrees, w).astype(np.int32), degrees


def decode_weighted_f32(g, llr, L, col_class, alpha, beta, early_stop=True, check_every=1,
                        flags=0):
    """Normalised/offset Min-Sum: magnitudes max(fma(alpha, m, -beta), 0); tables [n_w][C]."""
    r = np.ascontiguousarray(np.atleast_2d(llr), dtype=np.float32)
    F = r.shape[0]
    cc = np.ascontiguousarray(col_class, dtype=np.int32)
    a = np.ascontiguousarray(alpha, dtype=np.float32)
    b = np.ascontiguousarray(beta, dtype=np.float32)
    n_w, C = (a.shape if a.ndim == 2 else (0, int(cc.max()) + 1))
    bits = np.zeros((F, g.N), np.uint8)
    iters = np.zeros(F, np.int32)
    ok = np.zeros(F, np.uint8)
    soft = np.zeros((F, g.N), np.float32)
    rc = lib().orc_decode_weighted_f32(g.h, _p(r), F, L, int(early_stop), check_every, flags,
                                       _p(cc), C, n_w, _p(a), _p(b), _p(bits), _p(iters), _p(ok),
                                       _p(soft))
    assert rc == 0
    return bits, iters, ok, soft


def decode_weighted_f64(g, llr, L, col_class, alpha, beta):
    """Binary64, exactly L iterations; returns the posteriors [F][N]."""
    r = np.ascontiguousarray(np.atleast_2d(llr), dtype=np.float64)
    F = r.shape[0]
    cc = np.ascontiguousarray(col_class, dtype=np.int32)
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    soft = np.zeros((F, g.N), np.float64)
    rc = lib().orc_decode_weighted_f64(g.h, _p(r), F, L, _p(cc), a.shape[1], a.shape[0], _p(a),
                                       _p(b), _p(soft))
    assert rc == 0
    return soft


def decode_dense_f32(H: np.ndarray, llr: np.ndarray, L: int, early_stop=True, flags=0):
    """Algorithm 2 (dense masked map-reduce form), one frame."""
    H = np.ascontiguousarray(H, dtype=np.uint8)
    r = np.ascontiguousarray(llr, dtype=np.float32)
    m, n = H.shape
    b = np.zeros(n, np.uint8)
    it, ok = ctypes.c_int32(), ctypes.c_uint8()
    soft = np.zeros(n, np.float32)
    rc = lib().orc_decode_dense_f32(m, n, _p(H), _p(r), L, int(early_stop), flags, _p(b),
                                    ctypes.byref(it), ctypes.byref(ok), _p(soft))
    assert rc == 0
    return b, it.value, ok.value, soft

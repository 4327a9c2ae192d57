"""Python binding of ``libldpc.so`` (argument marshalling only).

Every decoding step runs in the library's CUDA kernels; this module passes pointers,
sizes and the current torch stream through ctypes. The functions carry the C names of
``include/ldpc.h``; :class:`Decoder` wraps them for torch tensors. Loading fails loudly
when the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libldpc.so")

LDPC_OK = 0
LDPC_ERR_INVALID_ARG = -1
LDPC_ERR_INVALID_H = -2
LDPC_ERR_BAD_POINTER = -3
LDPC_ERR_OOM = -4
LDPC_ERR_CUDA = -5
LDPC_ERR_TIMEOUT = -6
LDPC_ERR_DEVICE_CHECK = -7
LDPC_ERR_UNSUPPORTED = -8
LDPC_MODE_FP32 = 0
LDPC_MODE_FIXED = 1
LDPC_H_DENSE_U8 = 0
LDPC_H_PACKED_U32 = 1
LDPC_H_CSR = 2
LDPC_LLR_F32 = 0
LDPC_LLR_I8 = 1
LDPC_FLAG_PAPER_SLICER = 1
LDPC_FLAG_DEBUG = 2
LDPC_VARIANT_AUTO = 0
LDPC_VARIANT_STREAM = 1
LDPC_VARIANT_RESIDENT = 2
LDPC_VARIANT_DENSE = 3
LDPC_VARIANT_CLUSTER = 4
LDPC_NOALLOC_SCRATCH_BYTES = 32 << 20

# name -> (restype, argtypes), exactly the declarations of include/ldpc.h
P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
PI32, PI64 = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
SIGNATURES = {
    "ldpc_create": (P, [I32, I32, P]),
    "ldpc_create_ex": (P, [I32, I32, I32, P, P, I32, I32]),
    "ldpc_decode": (ctypes.c_int, [P, P, I32, I32, P, P]),
    "ldpc_decode_i8": (ctypes.c_int, [P, P, I32, I32, P, P]),
    "ldpc_decode_ex": (ctypes.c_int, [P, P, I32, I32, I32, I32, I32, P, P, P, P]),
    "ldpc_decode_host": (ctypes.c_int, [P, P, I32, I32, I32, I32, I32, P, P, P, P]),
    "ldpc_decode_noalloc": (ctypes.c_int, [P, P, I32, I32, I32, I32, I32, P, P, P, P]),
    "ldpc_batch_create": (P, [I32, P]),
    "ldpc_batch_set_stream": (ctypes.c_int, [P, P]),
    "ldpc_batch_set_io": (ctypes.c_int, [P, I32, P, I32, P, P, P, P]),
    "ldpc_batch_prepare": (ctypes.c_int, [P, I32, I32]),
    "ldpc_batch_launch": (ctypes.c_int, [P]),
    "ldpc_batch_decode": (ctypes.c_int, [P, I32, I32]),
    "ldpc_batch_capture": (ctypes.c_int, [P]),
    "ldpc_batch_replay": (ctypes.c_int, [P]),
    "ldpc_batch_set_threads": (ctypes.c_int, [P, I32]),
    "ldpc_batch_set_tile_frames": (ctypes.c_int, [P, I32]),
    "ldpc_batch_get_tile_frames": (ctypes.c_int, [P, PI32]),
    "ldpc_batch_autotune": (ctypes.c_int, [P, I32, I32, PI32, ctypes.POINTER(ctypes.c_float)]),
    "ldpc_batch_info": (ctypes.c_int, [P, PI32, PI32, PI32, PI32]),
    "ldpc_batch_set_large_codes": (ctypes.c_int, [P, I32]),
    "ldpc_batch_set_sm_split": (ctypes.c_int, [P, I32]),
    "ldpc_batch_get_sm_split": (ctypes.c_int, [P, PI32]),
    "ldpc_batch_destroy": (None, [P]),
    "ldpc_set_stream": (ctypes.c_int, [P, P]),
    "ldpc_set_mode": (ctypes.c_int, [P, I32]),
    "ldpc_set_variant": (ctypes.c_int, [P, I32]),
    "ldpc_set_stream_group": (ctypes.c_int, [P, I32]),
    "ldpc_set_stream_staging": (ctypes.c_int, [P, I32, I32, I32]),
    "ldpc_get_stream_staging": (ctypes.c_int, [P, PI32, PI32, PI32]),
    "ldpc_set_stream_messages": (ctypes.c_int, [P, I32]),
    "ldpc_get_stream_messages": (ctypes.c_int, [P, PI32]),
    "ldpc_read_messages": (ctypes.c_int, [P, I32, P]),
    "ldpc_check_device": (ctypes.c_int, [P]),
    "ldpc_set_wait_limit": (ctypes.c_int, [P, I32]),
    "ldpc_set_debug": (ctypes.c_int, [P, I32]),
    "ldpc_debug_report": (ctypes.c_int, [P, PI32, PI64]),
    "ldpc_set_cluster_shape": (ctypes.c_int, [P, I32, I32, I32]),
    "ldpc_get_cluster_shape": (ctypes.c_int, [P, PI32, PI32, PI32, PI32]),
    "ldpc_set_tuning": (ctypes.c_int, [P, I32, I32, I32]),
    "ldpc_get_tuning": (ctypes.c_int, [P, PI32, PI32, PI32]),
    "ldpc_autotune": (ctypes.c_int, [P, I32, I32, ctypes.POINTER(ctypes.c_float)]),
    "ldpc_autotune_data": (ctypes.c_int, [P, P, I32, I32, I32, I32, ctypes.POINTER(ctypes.c_float)]),
    "ldpc_classes": (ctypes.c_int, [P, PI32, PI32]),
    "ldpc_set_weights": (ctypes.c_int, [P, I32, P, P]),
    "ldpc_train_workspace_size": (ctypes.c_int, [P, I32, I32, ctypes.POINTER(ctypes.c_uint64)]),
    "ldpc_train_forward": (ctypes.c_int, [P, P, I32, I32, P, P, P, I32, P, ctypes.c_uint64]),
    "ldpc_train_backward": (ctypes.c_int, [P, I32, I32, P, P, P, I32, P, P, P, ctypes.c_uint64]),
    "ldpc_get_variant": (ctypes.c_int, [P, PI32]),
    "ldpc_reserve": (ctypes.c_int, [P, I32]),
    "ldpc_info": (ctypes.c_int, [P, PI32, PI32, PI64, PI32, PI32]),
    "ldpc_last_kernel_count": (ctypes.c_int, [P, PI32]),
    "ldpc_last_error": (ctypes.c_int, []),
    "ldpc_last_cuda_error": (ctypes.c_int, []),
    "ldpc_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "ldpc_destroy": (None, [P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the library (raises if it is missing: build it with ``build.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing; build it with paper_2507_10424_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class LdpcError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        msg = load().ldpc_strerror(status).decode()
        super().__init__(f"{what}: {msg} ({status})" if what else f"{msg} ({status})")
        self.status = status


def _check(status: int, what: str):
    if status != LDPC_OK:
        raise LdpcError(status, what)


def _host(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


# ----------------------------------------------------------- thin C-name wrappers

def ldpc_create(M: int, N: int, H: np.ndarray):
    return load().ldpc_create(M, N, _host(np.ascontiguousarray(H, dtype=np.uint8)))


def ldpc_create_ex(M, N, h_format, h_a, h_b, mode, flags):
    return load().ldpc_create_ex(M, N, h_format, h_a, h_b, mode, flags)


def ldpc_decode(h, llr_ptr, frames, max_iter, bits_ptr, iters_ptr):
    return load().ldpc_decode(h, llr_ptr, frames, max_iter, bits_ptr, iters_ptr)


def ldpc_decode_i8(h, llr_ptr, frames, max_iter, bits_ptr, iters_ptr):
    return load().ldpc_decode_i8(h, llr_ptr, frames, max_iter, bits_ptr, iters_ptr)


def ldpc_decode_ex(h, llr_ptr, llr_dtype, frames, max_iter, early_stop, check_every, bits_ptr,
                   iters_ptr, ok_ptr, soft_ptr):
    return load().ldpc_decode_ex(h, llr_ptr, llr_dtype, frames, max_iter, early_stop, check_every,
                                 bits_ptr, iters_ptr, ok_ptr, soft_ptr)


def ldpc_decode_host(h, llr_ptr, llr_dtype, frames, max_iter, early_stop, check_every, bits_ptr,
                     iters_ptr, ok_ptr, soft_ptr):
    return load().ldpc_decode_host(h, llr_ptr, llr_dtype, frames, max_iter, early_stop, check_every,
                                   bits_ptr, iters_ptr, ok_ptr, soft_ptr)


def ldpc_decode_noalloc(h, llr_ptr, llr_dtype, frames, max_iter, early_stop, check_every, bits_ptr,
                        iters_ptr, ok_ptr, soft_ptr):
    """Decode with scratch from the library's static device array (no allocation)."""
    return load().ldpc_decode_noalloc(h, llr_ptr, llr_dtype, frames, max_iter, early_stop,
                                      check_every, bits_ptr, iters_ptr, ok_ptr, soft_ptr)


def ldpc_set_stream(h, stream_ptr):
    return load().ldpc_set_stream(h, stream_ptr)


def ldpc_set_mode(h, mode):
    return load().ldpc_set_mode(h, mode)


def ldpc_set_stream_group(h, frames_per_group):
    return load().ldpc_set_stream_group(h, frames_per_group)


def ldpc_set_stream_staging(h, warps_per_cta, stages, frames_per_lane=0):
    return load().ldpc_set_stream_staging(h, warps_per_cta, stages, frames_per_lane)


def ldpc_get_stream_staging(h):
    w, s, v = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().ldpc_get_stream_staging(h, ctypes.byref(w), ctypes.byref(s), ctypes.byref(v)),
           "ldpc_get_stream_staging")
    return w.value, s.value, v.value


def ldpc_read_messages(h, frames, out_ptr):
    return load().ldpc_read_messages(h, frames, out_ptr)


def ldpc_set_stream_messages(h, compressed):
    return load().ldpc_set_stream_messages(h, compressed)


def ldpc_get_stream_messages(h):
    c = ctypes.c_int32()
    _check(load().ldpc_get_stream_messages(h, ctypes.byref(c)), "ldpc_get_stream_messages")
    return c.value


def ldpc_check_device(h):
    return load().ldpc_check_device(h)


def ldpc_set_wait_limit(h, tries):
    return load().ldpc_set_wait_limit(h, tries)


def ldpc_set_cluster_shape(h, cluster_size, frames_per_tile, threads):
    return load().ldpc_set_cluster_shape(h, cluster_size, frames_per_tile, threads)


def ldpc_get_cluster_shape(h):
    """(cluster_size, frames_per_tile, threads, clusters) of the cluster variant."""
    v = [ctypes.c_int32() for _ in range(4)]
    _check(load().ldpc_get_cluster_shape(h, *[ctypes.byref(x) for x in v]), "ldpc_get_cluster_shape")
    return tuple(x.value for x in v)


def ldpc_set_variant(h, variant):
    return load().ldpc_set_variant(h, variant)


def ldpc_set_tuning(h, frames_per_tile, threads, index_placement=0):
    return load().ldpc_set_tuning(h, frames_per_tile, threads, index_placement)


def ldpc_get_tuning(h):
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().ldpc_get_tuning(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "ldpc_get_tuning")
    return a.value, b.value, c.value


def ldpc_autotune(h, frames, max_iter):
    ms = ctypes.c_float()
    _check(load().ldpc_autotune(h, frames, max_iter, ctypes.byref(ms)), "ldpc_autotune")
    return ms.value


def ldpc_autotune_data(h, llr_ptr, frames, max_iter, early_stop, check_every):
    ms = ctypes.c_float()
    _check(load().ldpc_autotune_data(h, ctypes.c_void_p(llr_ptr), frames, max_iter, early_stop,
                                     check_every, ctypes.byref(ms)), "ldpc_autotune_data")
    return ms.value


def ldpc_classes(h):
    n = ctypes.c_int32()
    _check(load().ldpc_classes(h, ctypes.byref(n), None), "ldpc_classes")
    deg = (ctypes.c_int32 * max(n.value, 1))()
    _check(load().ldpc_classes(h, ctypes.byref(n), deg), "ldpc_classes")
    return [deg[i] for i in range(n.value)]


def ldpc_set_weights(h, n_rows, alpha_ptr, beta_ptr):
    return load().ldpc_set_weights(h, n_rows, alpha_ptr, beta_ptr)


def ldpc_train_workspace_size(h, frames, iters):
    b = ctypes.c_uint64()
    _check(load().ldpc_train_workspace_size(h, frames, iters, ctypes.byref(b)),
           "ldpc_train_workspace_size")
    return b.value


def ldpc_train_forward(h, llr_ptr, frames, iters, alpha_ptr, beta_ptr, soft_ptr, soft_every,
                       work_ptr, work_bytes):
    return load().ldpc_train_forward(h, llr_ptr, frames, iters, alpha_ptr, beta_ptr, soft_ptr,
                                     soft_every, work_ptr, work_bytes)


def ldpc_train_backward(h, frames, iters, alpha_ptr, beta_ptr, grad_soft_ptr, soft_every,
                        grad_alpha_ptr, grad_beta_ptr, work_ptr, work_bytes):
    return load().ldpc_train_backward(h, frames, iters, alpha_ptr, beta_ptr, grad_soft_ptr,
                                      soft_every, grad_alpha_ptr, grad_beta_ptr, work_ptr,
                                      work_bytes)


def ldpc_get_variant(h):
    v = ctypes.c_int32()
    _check(load().ldpc_get_variant(h, ctypes.byref(v)), "ldpc_get_variant")
    return v.value


def ldpc_reserve(h, max_frames):
    return load().ldpc_reserve(h, max_frames)


def ldpc_info(h):
    M, N, dc, dv = (ctypes.c_int32() for _ in range(4))
    E = ctypes.c_int64()
    _check(load().ldpc_info(h, ctypes.byref(M), ctypes.byref(N), ctypes.byref(E), ctypes.byref(dc),
                            ctypes.byref(dv)), "ldpc_info")
    return dict(M=M.value, N=N.value, E=E.value, max_dc=dc.value, max_dv=dv.value)


def ldpc_last_kernel_count(h):
    c = ctypes.c_int32()
    _check(load().ldpc_last_kernel_count(h, ctypes.byref(c)), "ldpc_last_kernel_count")
    return c.value


def ldpc_last_error():
    return load().ldpc_last_error()


def ldpc_last_cuda_error():
    return load().ldpc_last_cuda_error()


def ldpc_strerror(status):
    return load().ldpc_strerror(status).decode()


def ldpc_destroy(h):
    load().ldpc_destroy(h)


# ----------------------------------------------------------- torch-facing wrapper

class Decoder:
    """A decoder handle for one parity matrix.

    ``H`` may be a dense 0/1 matrix (numpy, [M][N]), or give ``csr=(row_ptr, col_idx)`` or
    ``packed=uint32 [M][ceil(N/32)]`` with ``M`` and ``N``. ``mode`` is "fp32" or "fixed".
    """

    def __init__(self, H=None, *, M=None, N=None, csr=None, packed=None, mode="fp32",
                 paper_slicer=False, debug=False):
        lib = load()
        m = {"fp32": LDPC_MODE_FP32, "fixed": LDPC_MODE_FIXED}[mode]
        flags = (LDPC_FLAG_PAPER_SLICER if paper_slicer else 0) | (LDPC_FLAG_DEBUG if debug else 0)
        keep = []
        if H is not None:
            Hn = np.ascontiguousarray(H, dtype=np.uint8)
            M, N = Hn.shape
            keep.append(Hn)
            args = (LDPC_H_DENSE_U8, _host(Hn), None)
        elif csr is not None:
            rp = np.ascontiguousarray(csr[0], dtype=np.int64)
            ci = np.ascontiguousarray(csr[1], dtype=np.int32)
            keep += [rp, ci]
            args = (LDPC_H_CSR, _host(rp), _host(ci))
        elif packed is not None:
            pk = np.ascontiguousarray(packed, dtype=np.uint32)
            keep.append(pk)
            args = (LDPC_H_PACKED_U32, _host(pk), None)
        else:
            raise ValueError("give H, csr or packed")
        self.h = lib.ldpc_create_ex(int(M), int(N), args[0], args[1], args[2], m, flags)
        if not self.h:
            raise LdpcError(lib.ldpc_last_error(), "ldpc_create_ex")
        self.M, self.N, self.mode = int(M), int(N), mode

    @classmethod
    def from_code(cls, code, **kw):
        rp, ci = code.csr()
        return cls(M=code.M, N=code.N, csr=(rp, ci), **kw)

    def close(self):
        if getattr(self, "h", None):
            load().ldpc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return ldpc_info(self.h)

    def set_variant(self, variant: str):
        v = {"auto": LDPC_VARIANT_AUTO, "stream": LDPC_VARIANT_STREAM,
             "resident": LDPC_VARIANT_RESIDENT, "dense": LDPC_VARIANT_DENSE,
             "cluster": LDPC_VARIANT_CLUSTER}[variant]
        _check(load().ldpc_set_variant(self.h, v), "ldpc_set_variant")

    def set_cluster_shape(self, cluster_size=0, frames_per_tile=0, threads=0):
        """Cluster variant: CTAs per cluster, frames per tile, CTA size (0 = automatic)."""
        _check(load().ldpc_set_cluster_shape(self.h, cluster_size, frames_per_tile, threads),
               "ldpc_set_cluster_shape")

    def cluster_shape(self):
        """(cluster_size, frames_per_tile, threads, clusters resident at once)."""
        return ldpc_get_cluster_shape(self.h)

    def set_stream_group(self, frames_per_group: int):
        """Streaming variant: 0 automatic L2-sized frame groups, -1 none, > 0 group size."""
        _check(load().ldpc_set_stream_group(self.h, frames_per_group), "ldpc_set_stream_group")

    def set_stream_staging(self, warps_per_cta=0, stages=0, frames_per_lane=0):
        """Streaming check pass: warps per CTA, shared-memory stages per warp and frames per
        lane of the staged (bulk-copy) kernel; 0 = automatic, stages -1 = unstaged kernel."""
        _check(load().ldpc_set_stream_staging(self.h, warps_per_cta, stages, frames_per_lane),
               "ldpc_set_stream_staging")

    def set_stream_messages(self, compressed: bool):
        """Streaming variant, FP32, rows of at most 16 edges: keep each row's messages
        compressed (two minima, location, signs) or one message per edge slot."""
        _check(load().ldpc_set_stream_messages(self.h, int(bool(compressed))),
               "ldpc_set_stream_messages")

    def stream_messages_compressed(self) -> bool:
        return bool(ldpc_get_stream_messages(self.h))

    def stream_staging(self):
        """(warps per CTA, stages, frames per lane) in force; stages 0 when the staged kernel
        is off, frames per lane 0 when automatic."""
        return ldpc_get_stream_staging(self.h)

    def read_messages(self, frames: int):
        """Messages eta after the last iteration of the last decode (streaming variant, no
        early stop): a CUDA float32 tensor [frames][E], edges in CSR order, LLR units."""
        import torch
        E = self.info()["E"]
        out = torch.empty((frames, E), dtype=torch.float32, device="cuda")
        _check(load().ldpc_read_messages(self.h, frames, ctypes.c_void_p(out.data_ptr())),
               "ldpc_read_messages")
        return out

    def check_device(self):
        """Wait for the handle's stream and raise LdpcError(LDPC_ERR_TIMEOUT) if a bounded
        wait inside a kernel ran out since the last check."""
        _check(load().ldpc_check_device(self.h), "ldpc_check_device")

    def set_debug(self, on: bool):
        """Device-side debug checks before every decode (index arrays in range, no NaN LLR);
        a decode they refuse raises LdpcError(LDPC_ERR_DEVICE_CHECK)."""
        _check(load().ldpc_set_debug(self.h, int(bool(on))), "ldpc_set_debug")

    def debug_report(self):
        """(what, where) of the last refused decode's first violation, then cleared: what 0
        none, 1 a NaN LLR (where = frame * N + bit), 2 an index array (where = id << 40 |
        entry)."""
        what, where = ctypes.c_int32(), ctypes.c_int64()
        _check(load().ldpc_debug_report(self.h, ctypes.byref(what), ctypes.byref(where)),
               "ldpc_debug_report")
        return what.value, where.value

    def set_wait_limit(self, tries: int):
        """Tries of each bounded wait in the staged kernels (0: give up at once)."""
        _check(load().ldpc_set_wait_limit(self.h, tries), "ldpc_set_wait_limit")

    def set_tuning(self, frames_per_tile=0, threads=0, index_placement=0):
        _check(load().ldpc_set_tuning(self.h, frames_per_tile, threads, index_placement),
               "ldpc_set_tuning")

    def tuning(self):
        return ldpc_get_tuning(self.h)

    def classes(self):
        """Column weight of each learned-weight class (distinct column weights, ascending)."""
        return ldpc_classes(self.h)

    def set_weights(self, alpha=None, beta=None):
        """Learned weights [rows][classes] (numpy or CPU tensors); None clears them."""
        if alpha is None:
            _check(load().ldpc_set_weights(self.h, 0, None, None), "ldpc_set_weights")
            return
        a = np.ascontiguousarray(np.asarray(alpha, dtype=np.float32))
        b = np.ascontiguousarray(np.asarray(beta, dtype=np.float32))
        if a.shape != b.shape or a.ndim != 2 or a.shape[1] != len(self.classes()):
            raise ValueError("alpha and beta must be [rows][n_classes]")
        _check(load().ldpc_set_weights(self.h, a.shape[0], _host(a), _host(b)), "ldpc_set_weights")

    def autotune(self, frames: int, max_iter: int, llr=None, early_stop: bool = True,
                 check_every: int = 1) -> float:
        """Pick the fastest launch shape on this device for the variant the next decode runs
        (resident: tile shape; streaming: check-pass staging); returns its time (ms).
        Without llr the shapes are timed without early stop (the work then does not depend
        on the values); with llr (a contiguous CUDA FP32 tensor [F][N]) they decode those
        frames with the given early-stop settings."""
        import torch
        _check(load().ldpc_set_stream(self.h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
               "ldpc_set_stream")
        if llr is None:
            return ldpc_autotune(self.h, frames, max_iter)
        if (not llr.is_cuda or not llr.is_contiguous() or llr.dtype != torch.float32
                or llr.dim() != 2 or llr.shape[1] != self.N):
            raise ValueError("llr must be a contiguous CUDA float32 tensor [F][N]")
        return ldpc_autotune_data(self.h, llr.data_ptr(), min(frames, llr.shape[0]), max_iter,
                                  int(bool(early_stop)), check_every)

    def variant(self) -> str:
        return {LDPC_VARIANT_STREAM: "stream", LDPC_VARIANT_RESIDENT: "resident",
                LDPC_VARIANT_DENSE: "dense", LDPC_VARIANT_CLUSTER: "cluster"}[ldpc_get_variant(self.h)]

    def set_mode(self, mode: str):
        _check(load().ldpc_set_mode(self.h, {"fp32": LDPC_MODE_FP32, "fixed": LDPC_MODE_FIXED}[mode]),
               "ldpc_set_mode")
        self.mode = mode

    def reserve(self, frames: int):
        _check(load().ldpc_reserve(self.h, frames), "ldpc_reserve")

    def last_kernel_count(self) -> int:
        return ldpc_last_kernel_count(self.h)

    def decode(self, llr, max_iter: int, early_stop: bool = True, check_every: int = 1,
               want_ok: bool = False, want_soft: bool = False, out=None):
        """Decode a CUDA tensor of LLRs [F][N] (float32, or int8 in fixed mode).

        Returns (bits uint8 [F][N], iters int32 [F], ok uint8 [F] or None, soft float32
        [F][N] or None), allocated on the tensor's device unless ``out`` gives them.
        """
        import torch

        if not llr.is_cuda or not llr.is_contiguous() or llr.dim() != 2 or llr.shape[1] != self.N:
            raise ValueError("llr must be a contiguous CUDA tensor [F][N]")
        dt = {torch.float32: LDPC_LLR_F32, torch.int8: LDPC_LLR_I8}[llr.dtype]
        F = llr.shape[0]
        dev = llr.device
        if out is None:
            bits = torch.empty((F, self.N), dtype=torch.uint8, device=dev)
            iters = torch.empty(F, dtype=torch.int32, device=dev)
            ok = torch.empty(F, dtype=torch.uint8, device=dev) if want_ok else None
            soft = torch.empty((F, self.N), dtype=torch.float32, device=dev) if want_soft else None
        else:
            bits, iters, ok, soft = out
        lib = load()
        _check(lib.ldpc_set_stream(self.h, ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)),
               "ldpc_set_stream")
        st = lib.ldpc_decode_ex(self.h, ctypes.c_void_p(llr.data_ptr()), dt, F, max_iter,
                                int(bool(early_stop)), check_every, ctypes.c_void_p(bits.data_ptr()),
                                ctypes.c_void_p(iters.data_ptr()),
                                ctypes.c_void_p(ok.data_ptr()) if ok is not None else None,
                                ctypes.c_void_p(soft.data_ptr()) if soft is not None else None)
        _check(st, "ldpc_decode_ex")
        return bits, iters, ok, soft

    def decode_host(self, llr, max_iter: int, early_stop: bool = True, check_every: int = 1,
                    out=None, want_ok=False, want_soft=False):
        """Decode host (CPU, preferably pinned) torch tensors; synchronous."""
        import torch

        if llr.is_cuda or not llr.is_contiguous() or llr.shape[1] != self.N:
            raise ValueError("llr must be a contiguous CPU tensor [F][N]")
        dt = {torch.float32: LDPC_LLR_F32, torch.int8: LDPC_LLR_I8}[llr.dtype]
        F = llr.shape[0]
        if out is None:
            pin = llr.is_pinned()
            bits = torch.empty((F, self.N), dtype=torch.uint8, pin_memory=pin)
            iters = torch.empty(F, dtype=torch.int32, pin_memory=pin)
            ok = torch.empty(F, dtype=torch.uint8, pin_memory=pin) if want_ok else None
            soft = torch.empty((F, self.N), dtype=torch.float32, pin_memory=pin) if want_soft else None
        else:
            bits, iters, ok, soft = out
        lib = load()
        _check(lib.ldpc_set_stream(self.h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
               "ldpc_set_stream")
        st = lib.ldpc_decode_host(self.h, ctypes.c_void_p(llr.data_ptr()), dt, F, max_iter,
                                  int(bool(early_stop)), check_every, ctypes.c_void_p(bits.data_ptr()),
                                  ctypes.c_void_p(iters.data_ptr()),
                                  ctypes.c_void_p(ok.data_ptr()) if ok is not None else None,
                                  ctypes.c_void_p(soft.data_ptr()) if soft is not None else None)
        _check(st, "ldpc_decode_host")
        return bits, iters, ok, soft


class Batch:
    """Several codes decoded in one persistent launch (and, once captured, one CUDA graph).

    ``decoders``: :class:`Decoder` objects (kept alive by the batch). Buffers are torch CUDA
    tensors given per code with :meth:`set_io`.
    """

    def __init__(self, decoders):
        import torch
        self.decoders = list(decoders)
        arr = (ctypes.c_void_p * len(self.decoders))(*[d.h for d in self.decoders])
        self._arr = arr
        self.b = load().ldpc_batch_create(len(self.decoders), ctypes.cast(arr, ctypes.c_void_p))
        if not self.b:
            raise LdpcError(LDPC_ERR_INVALID_ARG, "ldpc_batch_create")
        self.stream = torch.cuda.Stream()
        _check(load().ldpc_batch_set_stream(self.b, ctypes.c_void_p(self.stream.cuda_stream)),
               "ldpc_batch_set_stream")
        self._keep = {}

    def set_io(self, code, llr, want_ok=False, want_soft=False):
        """Allocate the outputs of code `code` for the CUDA tensor `llr` [F][N]; returns them."""
        import torch
        F, N = llr.shape
        bits = torch.empty((F, N), dtype=torch.uint8, device=llr.device)
        iters = torch.empty(F, dtype=torch.int32, device=llr.device)
        ok = torch.empty(F, dtype=torch.uint8, device=llr.device) if want_ok else None
        soft = torch.empty((F, N), dtype=torch.float32, device=llr.device) if want_soft else None
        P_ = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        _check(load().ldpc_batch_set_io(self.b, code, P_(llr), F, P_(bits), P_(iters), P_(ok), P_(soft)),
               "ldpc_batch_set_io")
        self._keep[code] = (llr, bits, iters, ok, soft)
        return bits, iters, ok, soft

    def prepare(self, max_iter, early_stop=True):
        _check(load().ldpc_batch_prepare(self.b, max_iter, int(early_stop)), "ldpc_batch_prepare")

    def launch(self):
        _check(load().ldpc_batch_launch(self.b), "ldpc_batch_launch")

    def decode(self, max_iter, early_stop=True):
        _check(load().ldpc_batch_decode(self.b, max_iter, int(early_stop)), "ldpc_batch_decode")

    def set_large_codes(self, streaming: bool):
        """Codes too large for shared memory: streaming kernels (True) or the persistent
        launch from global scratch (False); takes effect at the next prepare."""
        _check(load().ldpc_batch_set_large_codes(self.b, int(streaming)), "ldpc_batch_set_large_codes")

    def set_sm_split(self, sms: int):
        """Run the persistent kernel on at most `sms` SMs and the streamed large codes on the
        others (0: no split); takes effect at the next prepare."""
        _check(load().ldpc_batch_set_sm_split(self.b, sms), "ldpc_batch_set_sm_split")

    def sm_split(self) -> int:
        v = ctypes.c_int32()
        _check(load().ldpc_batch_get_sm_split(self.b, ctypes.byref(v)), "ldpc_batch_get_sm_split")
        return v.value

    def capture(self):
        _check(load().ldpc_batch_capture(self.b), "ldpc_batch_capture")

    def replay(self):
        _check(load().ldpc_batch_replay(self.b), "ldpc_batch_replay")

    def set_tile_frames(self, max_frames_per_tile: int):
        """At most 1, 2 or 4 frames per tile for the codes in shared memory; takes effect
        at the next prepare."""
        _check(load().ldpc_batch_set_tile_frames(self.b, max_frames_per_tile),
               "ldpc_batch_set_tile_frames")

    def tile_frames(self) -> int:
        v = ctypes.c_int32()
        _check(load().ldpc_batch_get_tile_frames(self.b, ctypes.byref(v)), "ldpc_batch_get_tile_frames")
        return v.value

    def autotune(self, max_iter, early_stop=True):
        """Time every cap on the frames per tile x CTA size on the prepared buffers, keep the
        fastest and leave the batch prepared with it; returns (threads, ms)."""
        t, ms = ctypes.c_int32(), ctypes.c_float()
        _check(load().ldpc_batch_autotune(self.b, max_iter, int(early_stop), ctypes.byref(t),
                                          ctypes.byref(ms)), "ldpc_batch_autotune")
        return t.value, ms.value

    def info(self):
        v = [ctypes.c_int32() for _ in range(4)]
        _check(load().ldpc_batch_info(self.b, *[ctypes.byref(x) for x in v]), "ldpc_batch_info")
        return dict(zip(("n_codes", "n_tiles", "threads", "codes_in_shared_memory"), [x.value for x in v]))

    def close(self):
        if getattr(self, "b", None):
            load().ldpc_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""H ingestion on the GPU (Section II-B: H given by its rows, the sets N_i and M_j derived).

The same parity matrix is handed to the library in each of its three formats:
* dense uint8 [M][N] through ``ldpc_create`` (the plain create call) and through
  ``ldpc_create_ex(LDPC_H_DENSE_U8)``;
* bit-packed rows (``LDPC_H_PACKED_U32``: bit j % 32 of word j / 32 is H(i, j)), packed here
  with numpy's little-endian bit order, independently of the input generators;
* CSR with the columns of every row shuffled (the format accepts any order in a row).

Every handle must report the same dimensions and degrees, and decode the same frames
exactly as the oracle does (which builds its own graph from the dense matrix): FP32 through
``ldpc_decode``, fixed point through ``ldpc_decode_i8`` on int8 LLRs, on the resident and
the streaming variants. The codes cover the Tanner example of Section II-A, the quasi-cyclic
N = 2304 code, and an irregular code whose N is not a multiple of 32, with a row of weight 0
and columns of weight 0.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2507_10424_gb300 import inputs

pytestmark = pytest.mark.gpu


def pack_rows_little_endian(H):
    """uint32 [M][ceil(N/32)] with bit (j % 32) of word (j // 32) equal to H[i, j]."""
    M, N = H.shape
    W = (N + 31) // 32
    padded = np.zeros((M, W * 32), np.uint8)
    padded[:, :N] = H
    by = np.packbits(padded, axis=1, bitorder="little")  # bit k of byte b is column 8 b + k
    return np.ascontiguousarray(by).view("<u4").astype(np.uint32).reshape(M, W)


def tanner_code():
    from conftest import read_golden
    sets = [r[1] for r in read_golden("tanner_10x5.txt")]
    return inputs.code_from_index_sets(sets, 10)


def ragged_irregular_code():
    """N = 1001 (N % 32 = 9): an irregular code on the first 990 bits, 11 bits of weight 0,
    and a check of weight 0 between the others."""
    base = inputs.irregular_code(990, 396, [2, 3, 8], [0.5, 0.375, 0.125], 13)
    sets = [list(base.cols[base.rows == i] + 1) for i in range(base.M)]
    sets.insert(57, [])
    return inputs.code_from_index_sets(sets, 1001)


CODES = {"tanner": tanner_code, "qc2304": inputs.cfg_qc_2304, "irregular1001": ragged_irregular_code}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2507_10424_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return torch


def make_handles(code, mode):
    """(label, handle) for every ingestion route of one mode."""
    from paper_2507_10424_gb300 import ldpc
    H = code.dense()
    M, N = H.shape
    m = ldpc.LDPC_MODE_FP32 if mode == "fp32" else ldpc.LDPC_MODE_FIXED
    rng = np.random.default_rng(M * 7 + N)
    rp, ci = code.csr()
    ci = ci.copy()
    for i in range(M):  # any column order within a row
        seg = ci[rp[i]:rp[i + 1]]
        ci[rp[i]:rp[i + 1]] = seg[rng.permutation(seg.size)]
    packed = pack_rows_little_endian(H)
    P = ldpc._host
    out = []
    if mode == "fp32":
        out.append(("ldpc_create (dense)", ldpc.ldpc_create(M, N, H)))
    out.append(("dense", ldpc.ldpc_create_ex(M, N, ldpc.LDPC_H_DENSE_U8, P(H), None, m, 0)))
    out.append(("packed", ldpc.ldpc_create_ex(M, N, ldpc.LDPC_H_PACKED_U32, P(packed), None, m, 0)))
    out.append(("csr", ldpc.ldpc_create_ex(M, N, ldpc.LDPC_H_CSR, P(rp), P(ci), m, 0)))
    for label, h in out:
        assert h, f"{label}: create failed ({ldpc.ldpc_last_error()})"
    return out


@pytest.mark.parametrize("name", sorted(CODES))
def test_every_format_gives_the_same_graph(torch_cuda, name):
    from paper_2507_10424_gb300 import ldpc
    code = CODES[name]()
    rw, cw = code.row_weights(), code.col_weights()
    want = dict(M=code.M, N=code.N, E=code.E, max_dc=int(rw.max()), max_dv=int(cw.max()))
    for mode in ("fp32", "fixed"):
        for label, h in make_handles(code, mode):
            assert ldpc.ldpc_info(h) == want, (mode, label)
            assert ldpc.ldpc_classes(h) == sorted(set(cw.tolist())), (mode, label)
            ldpc.ldpc_destroy(h)


@pytest.mark.parametrize("mode", ["fp32", "fixed"])
@pytest.mark.parametrize("name", sorted(CODES))
def test_every_format_decodes_like_the_oracle(torch_cuda, name, mode):
    torch = torch_cuda
    from paper_2507_10424_gb300 import ldpc
    code = CODES[name]()
    F, L = (300, 12) if code.N < 2000 else (200, 10)
    if name == "qc2304":
        cw = inputs.Encoder(code).random_codewords(F, 17)
        llr = np.concatenate([inputs.bpsk_awgn_llr(cw[k * 40:(k + 1) * 40], e, code.design_rate, 60 + k)
                              for k, e in enumerate([1.0, 1.5, 2.0, 2.5, 3.0])])
    elif name == "tanner":
        llr = (np.random.default_rng(4).standard_normal((F, code.N)) * 1.5 + 0.6).astype(np.float32)
    else:
        llr = inputs.all_zero_awgn_llr(F, code.N, 2.2, code.design_rate, 18)
    g = oracle.Graph(code.M, code.N, dense=code.dense())
    q = oracle.quantize(llr)
    if mode == "fp32":
        want_bits, want_iters = oracle.decode_f32(g, llr, L)[:2]
        x = torch.from_numpy(llr).cuda()
        call = ldpc.ldpc_decode
    else:
        want_bits, want_iters = oracle.decode_fixed(g, q, L)[:2]
        x = torch.from_numpy(q).cuda()
        call = ldpc.ldpc_decode_i8
    assert want_iters.max() > 1
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for label, h in make_handles(code, mode):
        for variant in (ldpc.LDPC_VARIANT_RESIDENT, ldpc.LDPC_VARIANT_STREAM):
            assert ldpc.ldpc_set_variant(h, variant) == ldpc.LDPC_OK
            assert ldpc.ldpc_set_stream(h, stream) == ldpc.LDPC_OK
            bits = torch.full((F, code.N), 5, dtype=torch.uint8, device="cuda")
            iters = torch.full((F,), -1, dtype=torch.int32, device="cuda")
            st = call(h, ctypes.c_void_p(x.data_ptr()), F, L, ctypes.c_void_p(bits.data_ptr()),
                      ctypes.c_void_p(iters.data_ptr()))
            assert st == ldpc.LDPC_OK, (label, variant, st)
            torch.cuda.synchronize()
            tag = f"{name} {mode} {label} variant={variant}"
            assert (iters.cpu().numpy() == want_iters).all(), tag
            assert (bits.cpu().numpy() == want_bits).all(), tag
        ldpc.ldpc_destroy(h)

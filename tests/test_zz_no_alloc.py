"""ldpc_decode_noalloc: decoding for callers that cannot allocate device memory.

Serving loops that must not stall on the allocator, processes whose device memory is
already held by another allocator, and embeddings that forbid allocation after start-up
cannot let a decode call cudaMalloc. This entry point takes its scratch from a static
device array inside the library instead. The test calls it through the C ABI twice in a
row, on two different batches, and checks each result against ldpc_decode_ex (the
regular entry point) on the same batch: bits, iteration counts and status identical,
posteriors within 1e-5 relative (exact in fixed point); the first test also compares
with the oracle directly. The same comparison covers learned
weights set on the handle and an irregular code on the padded row layout (more message
slots than edges). Requests are accepted up to the size the header's formula gives and
refused beyond it. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2507_10424_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL = 1e-5


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _run(fn, torch, dec, x, L, early_stop):
    F, N = x.shape
    bits = torch.full((F, N), 7, dtype=torch.uint8, device="cuda")
    iters = torch.full((F,), -5, dtype=torch.int32, device="cuda")
    ok = torch.full((F,), 9, dtype=torch.uint8, device="cuda")
    soft = torch.full((F, N), float("nan"), dtype=torch.float32, device="cuda")
    dtype = 0 if x.dtype == torch.float32 else 1
    st = fn(dec.h, _ptr(x), dtype, F, L, int(early_stop), 1, _ptr(bits), _ptr(iters), _ptr(ok),
            _ptr(soft))
    torch.cuda.synchronize()
    return st, bits.cpu().numpy(), iters.cpu().numpy(), ok.cpu().numpy(), soft.cpu().numpy()


@pytest.mark.parametrize("mode", ["fp32", "fixed"])
def test_noalloc_matches_regular_entry_point_twice(mode):
    import torch
    from paper_2507_10424_gb300 import build, ldpc
    build.build()
    code = inputs.cfg_regular_576()
    dec = ldpc.Decoder.from_code(code, mode=mode)
    ldpc.ldpc_set_stream(dec.h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    batches = [inputs.all_zero_awgn_llr(1000, code.N, 2.0, code.design_rate, 71),
               inputs.all_zero_awgn_llr(777, code.N, 2.5, code.design_rate, 72)]
    for k, llr in enumerate(batches):
        x = torch.from_numpy(llr).cuda()
        es = k == 0
        st_a, *got = _run(ldpc.ldpc_decode_noalloc, torch, dec, x, 20, es)
        st_b, *want = _run(ldpc.ldpc_decode_ex, torch, dec, x, 20, es)
        assert st_a == ldpc.LDPC_OK and st_b == ldpc.LDPC_OK
        assert (got[0] == want[0]).all() and (got[1] == want[1]).all() and (got[2] == want[2]).all()
        if mode == "fixed":
            assert (got[3] == want[3]).all()
        else:
            np.testing.assert_allclose(got[3], want[3], rtol=RTOL, atol=0)
        assert want[1].max() > 1
        g = oracle.Graph.from_code(code)  # and the oracle itself, directly
        if mode == "fixed":
            ob, oi, ook, os_ = oracle.decode_fixed(g, oracle.quantize(llr), 20, es)
            os_ = os_.astype(np.float32) * 0.25
        else:
            ob, oi, ook, os_ = oracle.decode_f32(g, llr, 20, es)
        assert (got[0] == ob).all() and (got[1] == oi).all() and (got[2] == ook).all()
        assert (got[3] == os_).all()
    dec.close()


def test_noalloc_rejects_requests_larger_than_its_array():
    import torch
    from paper_2507_10424_gb300 import build, ldpc
    build.build()
    code = inputs.cfg_qc_2304()
    dec = ldpc.Decoder.from_code(code)
    F = 2048  # about 160 MB of scratch for this code, more than the static array
    x = torch.zeros((F, code.N), dtype=torch.float32, device="cuda")
    st, *_ = _run(ldpc.ldpc_decode_noalloc, torch, dec, x, 10, True)
    assert st == ldpc.LDPC_ERR_INVALID_ARG
    dec.close()


def _compare(torch, fn_a, fn_b, dec, llr, L, mode, early_stop):
    from paper_2507_10424_gb300 import ldpc
    x = torch.from_numpy(llr).cuda()
    st_a, *got = _run(fn_a, torch, dec, x, L, early_stop)
    st_b, *want = _run(fn_b, torch, dec, x, L, early_stop)
    assert st_a == ldpc.LDPC_OK and st_b == ldpc.LDPC_OK
    assert (got[0] == want[0]).all() and (got[1] == want[1]).all() and (got[2] == want[2]).all()
    if mode == "fixed":
        assert (got[3] == want[3]).all()
    else:
        np.testing.assert_allclose(got[3], want[3], rtol=RTOL, atol=0)
    return want


def test_noalloc_with_learned_weights():
    """Weights set with ldpc_set_weights reach the allocation-free path too."""
    import torch
    from paper_2507_10424_gb300 import build, ldpc
    build.build()
    code = inputs.cfg_regular_576()
    dec = ldpc.Decoder.from_code(code)
    ldpc.ldpc_set_stream(dec.h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    rows = 6
    alpha = np.linspace(0.7, 0.9, rows, dtype=np.float32)[:, None]
    beta = np.linspace(0.25, 0.1, rows, dtype=np.float32)[:, None]
    dec.set_weights(alpha, beta)
    llr = inputs.all_zero_awgn_llr(600, code.N, 2.0, code.design_rate, 73)
    for es in (True, False):
        want = _compare(torch, ldpc.ldpc_decode_noalloc, ldpc.ldpc_decode_ex, dec, llr, 12, "fp32", es)
    plain = ldpc.Decoder.from_code(code)
    ldpc.ldpc_set_stream(plain.h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    st, *p = _run(ldpc.ldpc_decode_ex, torch, plain, torch.from_numpy(llr).cuda(), 12, False)
    assert st == ldpc.LDPC_OK and not np.array_equal(p[3], want[3])  # the weights did act
    dec.close()
    plain.close()


@pytest.mark.parametrize("mode", ["fp32", "fixed"])
def test_noalloc_on_a_padded_irregular_code(mode):
    """Rows of 6 and 7 edges own 8 message slots each: the scratch layout uses the slot
    count, not the edge count."""
    import torch
    from paper_2507_10424_gb300 import build, ldpc
    build.build()
    code = inputs.irregular_code(3000, 1500, [2, 3, 8], [0.5, 0.375, 0.125], 21)
    assert code.row_weights().max() <= 8 and 8 * code.M > code.E
    dec = ldpc.Decoder.from_code(code, mode=mode)
    ldpc.ldpc_set_stream(dec.h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    llr = inputs.all_zero_awgn_llr(200, code.N, 1.8, code.design_rate, 74)  # 18.4 MB of scratch in FP32
    for es in (True, False):
        want = _compare(torch, ldpc.ldpc_decode_noalloc, ldpc.ldpc_decode_ex, dec, llr, 25, mode, es)
    assert want[1].max() > 1
    dec.close()


def test_noalloc_accepts_up_to_the_documented_size():
    """Scratch = Fp (S m + N (m + r) + max_iter + 15) + 256 bytes, Fp = frames rounded up
    to 256, S = 8 M for rows of at most 8 edges; FP32: m = r = 4."""
    import torch
    from paper_2507_10424_gb300 import build, ldpc
    build.build()
    code = inputs.cfg_regular_576()
    L = 5
    need = lambda Fp: Fp * (8 * code.M * 4 + code.N * 8 + L + 15) + 256
    Fp = 256
    while need(Fp + 256) <= ldpc.LDPC_NOALLOC_SCRATCH_BYTES:
        Fp += 256
    dec = ldpc.Decoder.from_code(code)
    ldpc.ldpc_set_stream(dec.h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    for F, status in ((Fp, ldpc.LDPC_OK), (Fp + 1, ldpc.LDPC_ERR_INVALID_ARG)):
        x = torch.zeros((F, code.N), dtype=torch.float32, device="cuda")
        st, *out = _run(ldpc.ldpc_decode_noalloc, torch, dec, x, L, False)
        assert st == status, (F, st)
        if status == ldpc.LDPC_OK:
            assert (out[1] == L).all() and (out[0] == 0).all()
    dec.close()

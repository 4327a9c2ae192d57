"""ldpc_decode_noalloc: decoding for callers that cannot allocate device memory.

Serving loops that must not stall on the allocator, processes whose device memory is
already held by another allocator, and embeddings that forbid allocation after start-up
cannot let a decode call cudaMalloc. This entry point takes its scratch from a static
device array inside the library instead. The test calls it through the C ABI twice in a
row, on two different batches, and checks each result against ldpc_decode_ex (the
regular entry point) on the same batch: bits, iteration counts and status identical,
posteriors within 1e-5 relative (exact in fixed point). It also checks that a request
larger than the static array is refused. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

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

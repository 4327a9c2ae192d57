"""Batched decoding of several codes in one persistent launch, and its CUDA-graph replay,
against the oracle (bits, iteration counts and status identical, posteriors within 1e-5
relative) and against the per-code decode path."""
import numpy as np
import pytest

import oracle
from paper_2507_10424_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2507_10424_gb300 import build
    build.build()
    return torch


def mixed_small():
    codes = [inputs.cfg_regular_576(), inputs.irregular_code(240, 120, [2, 3, 6], [0.4, 0.4, 0.2], 11),
             inputs.qc_code(4, 8, 32, 0.7, 3),
             inputs.irregular_code(16200, 2700, [2, 3, 4, 8], [0.3, 0.4, 0.2, 0.1], 7)]
    frames = [131, 70, 0, 5]  # ragged, one code without frames, one code too large for smem
    return codes, frames


def check_code(code, llr, out, L, label, early_stop=True):
    bits, iters, ok, soft = [t.cpu().numpy() for t in out]
    g = oracle.Graph.from_code(code)
    wb, wi, wok, ws = oracle.decode_f32(g, llr, L, early_stop)
    assert (iters == wi).all(), label
    assert (ok == wok).all(), label
    assert (bits == wb).all(), label
    np.testing.assert_allclose(soft, ws, rtol=1e-5, atol=0, err_msg=label)


@pytest.mark.parametrize("large_streaming", [True, False])
def test_batch_matches_oracle_and_graph_replay(torch_cuda, large_streaming):
    """The code too large for shared memory goes through the streaming kernels on the
    side stream (True) or the persistent launch's global scratch (False)."""
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Batch, Decoder
    codes, frames = mixed_small()
    decs = [Decoder.from_code(c) for c in codes]
    batch = Batch(decs)
    batch.set_large_codes(large_streaming)
    L = 25
    ins, outs = [], []
    for k, (c, F) in enumerate(zip(codes, frames)):
        llr = inputs.all_zero_awgn_llr(max(F, 1), c.N, 2.0, c.design_rate, 50 + k)[:F]
        x = torch.from_numpy(np.ascontiguousarray(llr)).cuda()
        ins.append((llr, x))
        outs.append(batch.set_io(k, x, want_ok=True, want_soft=True))
    batch.decode(L)
    batch.stream.synchronize()
    info = batch.info()
    assert info["codes_in_shared_memory"] == 3
    assert info["n_tiles"] >= (sum(frames[:3]) // 4 if large_streaming else sum(frames) // 4)
    for k, c in enumerate(codes):
        if frames[k]:
            check_code(c, ins[k][0], outs[k], L, f"code {k}")
    # the same launch recorded in a CUDA graph, replayed on new LLRs in the same buffers
    batch.capture()
    for rep in range(2):
        for k, (c, F) in enumerate(zip(codes, frames)):
            if F:
                llr = inputs.all_zero_awgn_llr(F, c.N, 2.0, c.design_rate, 90 + 10 * rep + k)
                ins[k][1].copy_(torch.from_numpy(llr))
                ins[k] = (llr, ins[k][1])
        torch.cuda.synchronize()
        batch.replay()
        batch.stream.synchronize()
        for k, c in enumerate(codes):
            if frames[k]:
                check_code(c, ins[k][0], outs[k], L, f"replay {rep} code {k}")
    batch.close()


def test_batch_autotune_and_per_code_path_agree(torch_cuda):
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Batch, Decoder
    codes = [inputs.cfg_regular_576(), inputs.cfg_qc_2304()]
    frames = [300, 200]
    decs = [Decoder.from_code(c) for c in codes]
    batch = Batch(decs)
    xs, outs = [], []
    for k, (c, F) in enumerate(zip(codes, frames)):
        x = torch.from_numpy(inputs.all_zero_awgn_llr(F, c.N, 2.5, c.design_rate, 60 + k)).cuda()
        xs.append(x)
        outs.append(batch.set_io(k, x, want_soft=True))
    threads, ms = batch.autotune(20)
    assert threads % 32 == 0 and ms > 0
    batch.decode(20)
    batch.stream.synchronize()
    for k in range(2):
        b, it, _, sf = decs[k].decode(xs[k], 20, want_soft=True)
        torch.cuda.synchronize()
        assert (b == outs[k][0]).all() and (it == outs[k][1]).all() and (sf == outs[k][3]).all()
    batch.close()


@pytest.mark.parametrize("cap", [1, 2, 4])
def test_batch_frames_per_tile_caps_and_both_kernel_forms(torch_cuda, cap):
    """Every cap on the frames per tile, with early stop (the kernel form that tests the
    syndrome in the row pass) and without, gives the oracle's results; invalid caps are
    refused and leave the cap as it was."""
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Batch, Decoder, LdpcError
    codes, frames = mixed_small()
    decs = [Decoder.from_code(c) for c in codes]
    batch = Batch(decs)
    L = 25
    ins, outs = [], []
    for k, (c, F) in enumerate(zip(codes, frames)):
        llr = inputs.all_zero_awgn_llr(max(F, 1), c.N, 2.0, c.design_rate, 70 + k)[:F]
        x = torch.from_numpy(np.ascontiguousarray(llr)).cuda()
        ins.append(llr)
        outs.append(batch.set_io(k, x, want_ok=True, want_soft=True))
    assert batch.tile_frames() == 4
    batch.set_tile_frames(cap)
    assert batch.tile_frames() == cap
    for bad in (0, 3, 8):
        with pytest.raises(LdpcError):
            batch.set_tile_frames(bad)
    assert batch.tile_frames() == cap
    for es in (True, False, True):
        batch.decode(L, early_stop=es)
        batch.stream.synchronize()
        assert batch.info()["n_tiles"] >= sum(frames[:3]) // cap
        for k, c in enumerate(codes):
            if frames[k]:
                check_code(c, ins[k], outs[k], L, f"cap {cap} early_stop={es} code {k}", es)
    batch.close()


@pytest.mark.parametrize("sms", [19, 76])
def test_batch_sm_split_keeps_results(torch_cuda, sms):
    """The persistent kernel on a subset of the SMs and the streamed large code's passes on
    the others, launched directly and from a graph: the same results as the oracle."""
    torch = torch_cuda
    from paper_2507_10424_gb300 import ldpc
    from paper_2507_10424_gb300.ldpc import Batch, Decoder, LdpcError
    codes, frames = mixed_small()
    frames = [131, 70, 40, 37]
    decs = [Decoder.from_code(c) for c in codes]
    batch = Batch(decs)
    with pytest.raises(LdpcError):
        batch.set_sm_split(-1)
    batch.set_sm_split(sms)
    assert batch.sm_split() == sms
    L = 20
    ins, outs = [], []
    for k, (c, F) in enumerate(zip(codes, frames)):
        llr = inputs.all_zero_awgn_llr(F, c.N, 2.2, c.design_rate, 150 + k)
        x = torch.from_numpy(llr).cuda()
        ins.append(llr)
        outs.append(batch.set_io(k, x, want_ok=True, want_soft=True))
    batch.decode(L)
    batch.stream.synchronize()
    for k, c in enumerate(codes):
        check_code(c, ins[k], outs[k], L, f"split {sms} code {k}")
    batch.capture()
    batch.replay()
    batch.stream.synchronize()
    for k, c in enumerate(codes):
        check_code(c, ins[k], outs[k], L, f"split {sms} replay code {k}")
    threads, ms = batch.autotune(L)
    assert ms > 0 and 0 <= batch.sm_split() < 152
    batch.close()

"""The streaming variant's check pass on the padded row layout: the staged kernel (bulk
asynchronous copies into shared-memory stages, one pipeline per warp) in several shapes,
and the unstaged kernel, each against the CPU oracle (fixed point bit-exact; FP32 bits,
iterations and status identical, posteriors within 1e-5 relative). Also the bounded waits:
a wait limit of 0 makes every staged wait give up at once, which must surface as
LDPC_ERR_TIMEOUT from ldpc_check_device without a fault, and the next decode must be
correct again.
"""
import numpy as np
import pytest

from paper_2507_10424_gb300 import inputs
from test_gpu_parity import assert_parity, oracle_decode, torch_cuda  # noqa: F401

pytestmark = pytest.mark.gpu

# (warps per CTA, stages, frames per lane): unstaged, then staged shapes including the
# smallest ones and narrower lanes than the mode's vector
SHAPES = [(0, -1, 0), (1, 2, 0), (4, 3, 0), (8, 3, 0), (2, 8, 0), (12, 2, 2), (12, 2, 1)]


def staged_decode(torch, code, llr, L, mode, shape, early_stop=True, paper_slicer=False):
    from paper_2507_10424_gb300.ldpc import Decoder
    dec = Decoder.from_code(code, mode=mode, paper_slicer=paper_slicer)
    dec.set_variant("stream")
    dec.set_stream_staging(*shape)
    x = torch.from_numpy(np.ascontiguousarray(llr)).cuda()
    bits, iters, ok, soft = dec.decode(x, L, early_stop=early_stop, want_ok=True, want_soft=True)
    dec.check_device()
    got = (bits.cpu().numpy(), iters.cpu().numpy(), ok.cpu().numpy(), soft.cpu().numpy())
    dec.close()
    return got


def codes():
    # rows of 6-7 edges (8 slots), of 10-16 edges (16 slots), and an irregular code with
    # mixed row weights 3..8
    return {
        "regular576": inputs.cfg_regular_576(),
        "qc2304": inputs.cfg_qc_2304(),
        "irregular1200": inputs.irregular_code(1200, 500, [2, 3, 8], [0.5, 0.375, 0.125], 9),
    }


@pytest.mark.parametrize("mode", ["fp32", "fixed"])
@pytest.mark.parametrize("name", ["regular576", "qc2304", "irregular1200"])
def test_staged_shapes_match_oracle(torch_cuda, mode, name):
    code = codes()[name]
    F = 300  # not a multiple of a frame block: the last block is ragged
    llr = inputs.all_zero_awgn_llr(F, code.N, 2.0, code.design_rate, 41)
    for early_stop in (True, False):
        want = oracle_decode(code, llr, 12, mode, early_stop=early_stop)
        for shape in SHAPES:
            got = staged_decode(torch_cuda, code, llr, 12, mode, shape, early_stop)
            assert_parity(got, want, mode, f"{name} {mode} {shape} early_stop={early_stop}")


@pytest.mark.parametrize("mode", ["fp32", "fixed"])
def test_staged_paper_slicer_and_random_codewords(torch_cuda, mode):
    code = inputs.cfg_regular_576()
    cw = inputs.Encoder(code).random_codewords(200, 5)
    llr = inputs.bpsk_awgn_llr(cw, 2.5, code.design_rate, 6)
    want = oracle_decode(code, llr, 15, mode, paper_slicer=True)
    got = staged_decode(torch_cuda, code, llr, 15, mode, (4, 3, 0), paper_slicer=True)
    assert_parity(got, want, mode, "paper slicer")


def test_staging_settings_round_trip(torch_cuda):
    from paper_2507_10424_gb300.ldpc import Decoder, LdpcError
    dec = Decoder.from_code(inputs.cfg_regular_576())
    assert dec.stream_staging() == (12, 2, 0)
    dec.set_stream_staging(2, 5, 2)
    assert dec.stream_staging() == (2, 5, 2)
    dec.set_stream_staging(0, -1)
    assert dec.stream_staging()[1] == 0
    for bad in ((13, 3, 0), (-1, 3, 0), (4, 1, 0), (4, 9, 0), (4, -2, 0), (4, 3, 3), (4, 3, 16)):
        with pytest.raises(LdpcError):
            dec.set_stream_staging(*bad)
    dec.close()
    # rows of 16 slots: compressed FP32 stages do not fit 12 warps' shared memory, so the
    # automatic shape takes 8 warps and keeps the messages compressed; fixed point keeps 12
    qc = Decoder.from_code(inputs.cfg_qc_2304())
    assert qc.stream_staging() == (8, 2, 0) and qc.stream_messages_compressed()
    qc.set_mode("fixed")
    assert qc.stream_staging() == (12, 2, 0) and not qc.stream_messages_compressed()
    qc.close()


@pytest.mark.parametrize("mode", ["fp32", "fixed"])
def test_wait_that_runs_out_is_reported_and_the_next_decode_is_correct(torch_cuda, mode):
    from paper_2507_10424_gb300.ldpc import Decoder, LdpcError, LDPC_ERR_TIMEOUT
    torch = torch_cuda
    code = inputs.cfg_regular_576()
    llr = inputs.all_zero_awgn_llr(256, code.N, 2.0, code.design_rate, 43)
    x = torch.from_numpy(llr).cuda()
    dec = Decoder.from_code(code, mode=mode)
    dec.set_variant("stream")
    dec.set_stream_staging(4, 3, 0)
    dec.set_wait_limit(0)  # every staged wait gives up at its first look
    dec.decode(x, 10)
    with pytest.raises(LdpcError) as e:
        dec.check_device()
    assert e.value.status == LDPC_ERR_TIMEOUT
    dec.check_device()  # the word was cleared by the read
    dec.set_wait_limit(1 << 16)
    bits, iters, ok, soft = dec.decode(x, 10, want_ok=True, want_soft=True)
    dec.check_device()
    got = (bits.cpu().numpy(), iters.cpu().numpy(), ok.cpu().numpy(), soft.cpu().numpy())
    assert_parity(got, oracle_decode(code, llr, 10, mode), mode, "after a timeout")
    dec.close()


@pytest.mark.parametrize("mode", ["fp32", "fixed"])
@pytest.mark.parametrize("on_data", [False, True])
def test_autotune_picks_a_staging_and_keeps_results(torch_cuda, mode, on_data):
    from paper_2507_10424_gb300.ldpc import Decoder
    torch = torch_cuda
    code = codes()["irregular1200"]
    llr = inputs.all_zero_awgn_llr(700, code.N, 2.0, code.design_rate, 44)
    dec = Decoder.from_code(code, mode=mode)
    dec.set_variant("stream")
    ms = dec.autotune(700, 12, llr=torch.from_numpy(llr).cuda() if on_data else None)
    assert ms > 0
    w, s, v = dec.stream_staging()
    assert (s == 0) or (1 <= w <= 12 and 2 <= s <= 8)
    bits, iters, ok, soft = dec.decode(torch.from_numpy(llr).cuda(), 12, want_ok=True, want_soft=True)
    dec.check_device()
    got = (bits.cpu().numpy(), iters.cpu().numpy(), ok.cpu().numpy(), soft.cpu().numpy())
    assert_parity(got, oracle_decode(code, llr, 12, mode), mode, f"autotuned {(w, s, v)}")
    dec.close()


@pytest.mark.parametrize("mode", ["fp32", "fixed"])
@pytest.mark.parametrize("shape", [(0, -1, 0), (12, 2, 0)])
def test_frame_compaction_keeps_every_output(torch_cuda, mode, shape):
    """Early stop with frames that stop at many different iterations (Eb/N0 spread over
    1.5-5 dB, frames shuffled): the streaming decode compacts the running frames to the
    front several times. Every frame's bits, iterations, status and posteriors must still
    equal the oracle's, including frames written out early by a compaction."""
    code = inputs.cfg_regular_576()
    F = 1500
    rng = np.random.default_rng(12)
    cw = inputs.Encoder(code).random_codewords(F, 13)
    snr = rng.permutation(np.linspace(1.5, 5.0, F))
    llr = np.concatenate([inputs.bpsk_awgn_llr(cw[k:k + 1], float(snr[k]), code.design_rate, 500 + k)
                          for k in range(F)])
    want = oracle_decode(code, llr, 30, mode)
    assert len(np.unique(want[1])) > 8  # stops spread over many iterations
    got = staged_decode(torch_cuda, code, llr, 30, mode, shape)
    assert_parity(got, want, mode, f"compaction {shape}")


@pytest.mark.parametrize("mode", ["fp32", "fixed"])
@pytest.mark.parametrize("shape", [(0, -1, 0), (8, 2, 0), (12, 2, 1)])
def test_passes_bounded_by_positions_in_use(torch_cuda, mode, shape):
    """Most frames stop at the pre-check and the rest never stop: after the first compaction
    the running frames fill only the first frame blocks, and the check and bit passes skip
    every block behind them. A frame count that is not a multiple of the block size, the
    stopped frames scattered (not a prefix); outputs of every frame equal the oracle's,
    with early stop and, for the same frames, without (no compaction)."""
    code = inputs.cfg_regular_576()
    F = 2077
    rng = np.random.default_rng(31)
    llr = inputs.all_zero_awgn_llr(F, code.N, 0.5, code.design_rate, 32)
    stop = rng.permutation(F)[: F - 300]  # 1777 frames are codewords at the pre-check
    llr[stop] = np.abs(llr[stop]) + 1.0
    for es in (True, False):
        want = oracle_decode(code, llr, 17, mode, early_stop=es)
        if es:
            assert (want[1][stop] == 0).all() and (want[1] > 12).sum() > 200
        got = staged_decode(torch_cuda, code, llr, 17, mode, shape, early_stop=es)
        assert_parity(got, want, mode, f"bounded passes {shape} early_stop={es}")


@pytest.mark.parametrize("mode", ["fp32", "fixed"])
def test_bits_only_outputs_match_oracle(torch_cuda, mode):
    """Decodes that ask for no posteriors take their final syndrome, and (without early
    stop) their output bits, from the decisions the last bit pass packs one byte per lane.
    Checked against the oracle on codes with 8- and 16-slot padded rows, rows longer than
    16 edges (CSR), a length that is not a multiple of 16, ragged frame counts, both
    slicers, lanes of every width, and an output buffer that starts at an odd address."""
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Decoder
    cs = dict(codes())
    cs["irregular1000"] = inputs.irregular_code(1000, 500, [2, 3, 8], [0.5, 0.375, 0.125], 12)
    cs["paper_shaped"] = inputs.cfg_paper_shaped()
    for name, code in cs.items():
        F = 300 if code.N < 4000 else 40
        llr = inputs.all_zero_awgn_llr(F, code.N, 2.0, code.design_rate, 43)
        x = torch.from_numpy(llr).cuda()
        for paper in (False, True):
            for early_stop in (False, True):
                want = oracle_decode(code, llr, 9, mode, early_stop=early_stop, paper_slicer=paper)
                for shape in [(0, 0, 0), (0, -1, 0), (12, 2, 4), (12, 2, 2)]:
                    dec = Decoder.from_code(code, mode=mode, paper_slicer=paper)
                    dec.set_variant("stream")
                    dec.set_stream_staging(*shape)
                    raw = torch.full((F * code.N + 1,), 7, dtype=torch.uint8, device="cuda")
                    bits = raw[1:].view(F, code.N)  # odd address: no 16-byte stores
                    iters = torch.empty(F, dtype=torch.int32, device="cuda")
                    ok = torch.empty(F, dtype=torch.uint8, device="cuda")
                    dec.decode(x, 9, early_stop=early_stop, out=(bits, iters, ok, None))
                    dec.check_device()
                    what = f"{name} {mode} paper={paper} early_stop={early_stop} {shape}"
                    assert raw[0].item() == 7, what
                    np.testing.assert_array_equal(bits.cpu().numpy(), want[0], err_msg=what)
                    np.testing.assert_array_equal(iters.cpu().numpy(), want[1], err_msg=what)
                    np.testing.assert_array_equal(ok.cpu().numpy(), want[2], err_msg=what)
                    # the same decode into an aligned buffer
                    b2, it2, ok2, _ = dec.decode(x, 9, early_stop=early_stop, want_ok=True)
                    np.testing.assert_array_equal(b2.cpu().numpy(), want[0], err_msg=what)
                    np.testing.assert_array_equal(ok2.cpu().numpy(), want[2], err_msg=what)
                    dec.close()

"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by element.

Tolerances (from the specification of the two modes):
* fixed point (int8 LLR, saturating int16 messages): bit-exact -- bits, iterations,
  status and every posterior;
* FP32: decoded bits, iteration counts and status identical; posteriors within 1e-5
  relative (the contract), and, since every kernel adds in the oracle's order (r_j first,
  then the column's messages by ascending check) with one binary32 rounding per operation,
  also bit-identical: ``assert_parity`` checks both, so a change of summation order shows
  up as a failure even while it stays within the tolerance.
"""
import numpy as np
import pytest

import oracle
from paper_2507_10424_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2507_10424_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return torch


def gpu_decode(torch, code, llr, L, mode="fp32", variant="auto", early_stop=True, check_every=1,
               paper_slicer=False, i8=False):
    from paper_2507_10424_gb300.ldpc import Decoder
    dec = Decoder.from_code(code, mode=mode, paper_slicer=paper_slicer)
    dec.set_variant(variant)
    x = torch.from_numpy(np.ascontiguousarray(llr)).cuda()
    bits, iters, ok, soft = dec.decode(x, L, early_stop=early_stop, check_every=check_every,
                                       want_ok=True, want_soft=True)
    torch.cuda.synchronize()
    used = dec.variant()
    n = dec.last_kernel_count()
    dec.close()
    return bits.cpu().numpy(), iters.cpu().numpy(), ok.cpu().numpy(), soft.cpu().numpy(), used, n


def oracle_decode(code, llr, L, mode="fp32", early_stop=True, check_every=1, paper_slicer=False,
                  i8=False):
    g = oracle.Graph.from_code(code)
    flags = oracle.PAPER_SLICER if paper_slicer else 0
    if mode == "fp32":
        return oracle.decode_f32(g, llr, L, early_stop, check_every, flags=flags)
    q = llr if i8 else oracle.quantize(llr)
    b, it, ok, s = oracle.decode_fixed(g, q, L, early_stop, check_every, flags=flags)
    return b, it, ok, s.astype(np.float32) * 0.25


def assert_parity(got, want, mode, label=""):
    gb, gi, gok, gs = got[:4]
    wb, wi, wok, ws = want
    assert (gi == wi).all(), f"{label}: iterations differ in {(gi != wi).sum()} frames"
    assert (gok == wok).all(), f"{label}: status differs in {(gok != wok).sum()} frames"
    assert (gb == wb).all(), f"{label}: bits differ in {(gb != wb).sum()} positions"
    if mode == "fixed":
        assert (gs == ws).all(), f"{label}: fixed-point posteriors differ"
    else:
        np.testing.assert_allclose(gs, ws, rtol=RTOL, atol=0, err_msg=label)
        inexact = int((gs != ws).sum())
        assert inexact == 0, f"{label}: {inexact} FP32 posteriors within tolerance but not identical"


def tanner_code():
    from conftest import read_golden
    sets = [r[1] for r in read_golden("tanner_10x5.txt")]
    return inputs.code_from_index_sets(sets, 10)


MODES = ["fp32", "fixed"]
VARIANTS = ["stream", "resident", "cluster"]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("variant", VARIANTS)
def test_tanner_example(torch_cuda, mode, variant):
    code = tanner_code()
    rng = np.random.default_rng(1)
    llr = (rng.standard_normal((300, 10)) * 1.5 + 0.5).astype(np.float32)
    got = gpu_decode(torch_cuda, code, llr, 12, mode, variant)
    assert got[4] == variant
    assert_parity(got, oracle_decode(code, llr, 12, mode), mode, "tanner")


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("variant", VARIANTS)
def test_regular_576_all_zero_2p5dB(torch_cuda, mode, variant):
    """(3,6)-regular N=576, 1024 frames of the all-zero codeword at Eb/N0 = 2.5 dB, 20 iterations."""
    code = inputs.cfg_regular_576()
    llr = inputs.all_zero_awgn_llr(1024, code.N, 2.5, code.design_rate, 11)
    got = gpu_decode(torch_cuda, code, llr, 20, mode, variant)
    want = oracle_decode(code, llr, 20, mode)
    assert_parity(got, want, mode, "regular576")
    assert want[1].max() > 1  # the case exercises several iterations


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("early_stop", [False, True])
def test_qc_2304_random_codewords(torch_cuda, mode, variant, early_stop):
    """QC 12x24, Z=96: random codewords over an SNR sweep, 10 iterations."""
    code = inputs.cfg_qc_2304()
    enc = inputs.Encoder(code)
    F = 300  # ragged: not a multiple of any tile or vector width
    cw = enc.random_codewords(F, 21)
    ebn0 = np.repeat([1.0, 1.5, 2.0, 2.5, 3.0], F // 5)
    llr = np.concatenate([inputs.bpsk_awgn_llr(cw[k * 60:(k + 1) * 60], e, code.design_rate, 30 + k)
                          for k, e in enumerate([1.0, 1.5, 2.0, 2.5, 3.0])])
    got = gpu_decode(torch_cuda, code, llr, 10, mode, variant, early_stop=early_stop)
    want = oracle_decode(code, llr, 10, mode, early_stop=early_stop)
    assert_parity(got, want, mode, "qc2304")
    del ebn0


@pytest.mark.parametrize("mode", MODES)
def test_irregular_64800_streaming(torch_cuda, mode):
    """Irregular N=64800 (weights 2/3/8), all-zero codeword at 1.0 dB, 50 iterations, early stop."""
    code = inputs.cfg_irregular_64800()
    llr = inputs.all_zero_awgn_llr(24, code.N, 1.0, code.design_rate, 41)
    got = gpu_decode(torch_cuda, code, llr, 50, mode, "stream")
    assert got[4] == "stream"
    assert_parity(got, oracle_decode(code, llr, 50, mode), mode, "irregular64800")


@pytest.mark.parametrize("mode", MODES)
def test_irregular_64800_cluster(torch_cuda, mode):
    """The same code with a tile held across a thread-block cluster (one FP32 frame is
    about 1.3 MB: more than one SM's shared memory, less than eight SMs')."""
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Decoder
    code = inputs.cfg_irregular_64800()
    llr = inputs.all_zero_awgn_llr(24, code.N, 1.3, code.design_rate, 43)
    got = gpu_decode(torch, code, llr, 50, mode, "cluster")
    assert got[4] == "cluster"
    assert_parity(got, oracle_decode(code, llr, 50, mode), mode, "irregular64800 cluster")
    dec = Decoder.from_code(code, mode=mode)
    C, FT, threads, clusters = dec.cluster_shape()
    assert C in (4, 8, 16) and clusters * C <= 152 and clusters >= 1
    dec.close()


@pytest.mark.parametrize("mode", MODES)
def test_every_cluster_shape(torch_cuda, mode):
    """Results must not depend on the cluster size, frames per tile or CTA size."""
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Decoder, LdpcError
    code = inputs.irregular_code(2000, 1000, [2, 3, 8], [0.5, 0.375, 0.125], 9)
    llr = inputs.all_zero_awgn_llr(45, code.N, 1.6, code.design_rate, 12)
    x = torch.from_numpy(llr).cuda()
    tried = set()
    for es in (True, False):
        want = oracle_decode(code, llr, 18, mode, early_stop=es)
        for C in (1, 2, 4, 8, 16):
            for ft in (0, 1, 2, 4):
                for th in (0, 256, 608):
                    dec = Decoder.from_code(code, mode=mode)
                    dec.set_cluster_shape(C, ft, th)
                    try:
                        dec.set_variant("cluster")
                    except LdpcError:
                        dec.close()
                        continue
                    shape = dec.cluster_shape()
                    assert shape[0] == C and (ft == 0 or shape[1] == ft)
                    b, it, ok, sf = dec.decode(x, 18, early_stop=es, want_ok=True, want_soft=True)
                    torch.cuda.synchronize()
                    got = (b.cpu().numpy(), it.cpu().numpy(), ok.cpu().numpy(), sf.cpu().numpy())
                    assert_parity(got, want, mode, f"C={C} FT={ft} threads={th} early_stop={es}")
                    tried.add((C, shape[1]))
                    dec.close()
    assert {(1, 1), (2, 1), (4, 1), (8, 1)} <= tried


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("group", [32, 64])
def test_streaming_in_l2_sized_frame_groups(torch_cuda, mode, group):
    """The streaming variant decoding a batch in frame groups (one frame per lane), with a
    ragged last group, against the oracle; early stop on and off."""
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Decoder
    code = inputs.irregular_code(2000, 1000, [2, 3, 8], [0.5, 0.375, 0.125], 9)
    llr = inputs.all_zero_awgn_llr(150, code.N, 1.8, code.design_rate, 19)
    for es in (True, False):
        dec = Decoder.from_code(code, mode=mode)
        dec.set_variant("stream")
        dec.set_stream_group(group)
        b, it, ok, sf = dec.decode(torch.from_numpy(llr).cuda(), 30, early_stop=es, want_ok=True,
                                   want_soft=True)
        torch.cuda.synchronize()
        got = (b.cpu().numpy(), it.cpu().numpy(), ok.cpu().numpy(), sf.cpu().numpy())
        assert_parity(got, oracle_decode(code, llr, 30, mode, early_stop=es), mode, f"group={group}")
        dec.close()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("variant", VARIANTS)
def test_check_every_and_paper_slicer(torch_cuda, mode, variant):
    code = inputs.qc_code(4, 8, 32, 0.7, 3)
    rng = np.random.default_rng(8)
    llr = (rng.standard_normal((257, code.N)) * 1.4 + 1.1).astype(np.float32)
    for ce in (1, 3, 6):
        got = gpu_decode(torch_cuda, code, llr, 25, mode, variant, check_every=ce)
        assert_parity(got, oracle_decode(code, llr, 25, mode, check_every=ce), mode, f"ce={ce}")
    tc = tanner_code()
    l2 = (rng.standard_normal((129, 10)) * 1.5 + 0.4).astype(np.float32)
    got = gpu_decode(torch_cuda, tc, l2, 9, mode, variant, paper_slicer=True)
    assert_parity(got, oracle_decode(tc, l2, 9, mode, paper_slicer=True), mode, "paper slicer")


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("variant", VARIANTS)
def test_long_rows_and_empty_rows_columns(torch_cuda, mode, variant):
    """Rows longer than 32 (in-place lambda path), weight-0 rows and weight-0 columns."""
    rng = np.random.default_rng(5)
    N = 180
    sets = [sorted(rng.choice(N - 5, size=d, replace=False) + 1) for d in (40, 70, 33, 3, 2, 12)]
    sets.insert(2, [])  # a row of weight 0
    code = inputs.code_from_index_sets(sets, N)  # the last 5 columns have weight 0
    llr = (rng.standard_normal((131, N)) * 2 + 0.3).astype(np.float32)
    got = gpu_decode(torch_cuda, code, llr, 15, mode, variant)
    assert_parity(got, oracle_decode(code, llr, 15, mode), mode, "long rows")


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("variant", VARIANTS)
def test_ties_and_signed_zeros(torch_cuda, mode, variant):
    """LLRs drawn from {-2, -1, -0.0, +0.0, 1, 2}: ties in every row, zero messages of both
    signs, zero posteriors; decisions, iteration counts and values must still agree."""
    code = inputs.qc_code(4, 8, 32, 0.7, 4)
    rng = np.random.default_rng(17)
    llr = rng.choice(np.array([-2.0, -1.0, -0.0, 0.0, 1.0, 2.0], np.float32), size=(199, code.N))
    for es in (True, False):
        got = gpu_decode(torch_cuda, code, llr, 12, mode, variant, early_stop=es)
        assert_parity(got, oracle_decode(code, llr, 12, mode, early_stop=es), mode, "ties/zeros")


@pytest.mark.parametrize("variant", VARIANTS)
def test_int8_input_and_saturation(torch_cuda, variant):
    rng = np.random.default_rng(2)
    n_bits = 40
    sets = [sorted(rng.choice(n_bits, size=int(rng.integers(2, 5)), replace=False) + 1)
            for _ in range(120)]
    code = inputs.code_from_index_sets(sets, n_bits)
    q = rng.choice([-127, 127, -3, 5], size=(67, n_bits)).astype(np.int8)
    got = gpu_decode(torch_cuda, code, q, 12, "fixed", variant, early_stop=False)
    want = oracle_decode(code, q, 12, "fixed", early_stop=False, i8=True)
    assert_parity(got, want, "fixed", "int8 saturation")
    assert np.abs(want[3]).max() == 32767 * 0.25  # saturation reached


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("variant", VARIANTS)
def test_edge_cases(torch_cuda, mode, variant):
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Decoder
    code = inputs.qc_code(3, 6, 32, 0.8, 9)
    enc = inputs.Encoder(code)
    cw = enc.random_codewords(33, 2)
    llr = ((1 - 2 * cw.astype(np.float32)) * 2.75).astype(np.float32)
    got = gpu_decode(torch, code, llr, 10, mode, variant)
    assert (got[1] == 0).all() and (got[2] == 1).all() and (got[0] == cw).all()
    for F in (1, 2, 7):
        rng = np.random.default_rng(F)
        l2 = (rng.standard_normal((F, code.N)) + 0.5).astype(np.float32)
        for L in (0, 1, 4):
            got = gpu_decode(torch, code, l2, L, mode, variant)
            assert_parity(got, oracle_decode(code, l2, L, mode), mode, f"F={F} L={L}")
    dec = Decoder.from_code(code, mode=mode)
    dec.set_variant(variant)
    empty = torch.zeros((0, code.N), dtype=torch.float32, device="cuda")
    b, it, _, _ = dec.decode(empty, 5)
    assert b.shape == (0, code.N) and it.shape == (0,)


@pytest.mark.parametrize("mode", MODES)
def test_every_resident_launch_shape(torch_cuda, mode):
    """Results must not depend on the launch shape: frames per tile and CTA size, each with
    early stop (the kernels that test the syndrome inside the row pass; frames of one tile
    stop at different iterations) and without (the syndrome after the last iteration)."""
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Decoder, LdpcError
    code = inputs.cfg_qc_2304()
    F = 67
    cw = inputs.Encoder(code).random_codewords(F, 5)
    snr = np.random.default_rng(7).permutation(np.linspace(2.5, 8.0, F))
    llr = np.concatenate([inputs.bpsk_awgn_llr(cw[k:k + 1], float(snr[k]), code.design_rate, 600 + k)
                          for k in range(F)])
    llr[[3, 40]] = (1 - 2 * cw[[3, 40]].astype(np.float32)) * 4.0  # codewords at the input
    want = {es: oracle_decode(code, llr, 8, mode, early_stop=es) for es in (True, False)}
    assert len(np.unique(want[True][1])) >= 7  # tiles mix frames that stop at k = 0 .. 8
    x = torch.from_numpy(llr).cuda()
    tried = 0
    for ft in (1, 2, 4):
        for th in (0, 96, 256, 640, 768, 1024):
            for ip in (1, 2):
                dec = Decoder.from_code(code, mode=mode)
                dec.set_variant("resident")
                try:
                    dec.set_tuning(ft, th, ip)
                except LdpcError:
                    continue
                assert dec.tuning()[2] == ip
                for es in (True, False):
                    b, it, ok, sf = dec.decode(x, 8, early_stop=es, want_ok=True, want_soft=True)
                    torch.cuda.synchronize()
                    got = (b.cpu().numpy(), it.cpu().numpy(), ok.cpu().numpy(), sf.cpu().numpy())
                    assert_parity(got, want[es], mode, f"FT={ft} threads={th} index={ip} es={es}")
                tried += 1
                dec.close()
    assert tried >= 12


@pytest.mark.parametrize("mode", MODES)
def test_every_resident_launch_shape_small_code(torch_cuda, mode):
    """The same on the (3,6)-regular N=576 code, whose tiles of 4 FP32 frames fit shared
    memory: the early-stop kernels that read per-slot decision bytes (fixed point, and FP32
    tiles of 4 frames) in every frames-per-tile and CTA size, with the syndrome tested every
    iteration and every third (the column pass writes the bytes only before a tested
    iteration)."""
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Decoder, LdpcError
    code = inputs.cfg_regular_576()
    F = 203
    snr = np.random.default_rng(8).permutation(np.linspace(1.5, 6.0, F))
    llr = np.concatenate([inputs.all_zero_awgn_llr(1, code.N, float(snr[k]), code.design_rate, 700 + k)
                          for k in range(F)])
    llr[[5, 150]] = 3.0  # codewords at the input
    x = torch.from_numpy(llr).cuda()
    tried = 0
    for ce in (1, 3):
        want = oracle_decode(code, llr, 14, mode, early_stop=True, check_every=ce)
        assert len(np.unique(want[1])) >= 5
        for ft in (1, 2, 4):
            for th in (0, 96, 288, 512):
                for ip in (1, 2):
                    dec = Decoder.from_code(code, mode=mode)
                    dec.set_variant("resident")
                    try:
                        dec.set_tuning(ft, th, ip)
                    except LdpcError:
                        continue
                    b, it, ok, sf = dec.decode(x, 14, early_stop=True, check_every=ce, want_ok=True,
                                               want_soft=True)
                    torch.cuda.synchronize()
                    got = (b.cpu().numpy(), it.cpu().numpy(), ok.cpu().numpy(), sf.cpu().numpy())
                    assert_parity(got, want, mode, f"FT={ft} threads={th} index={ip} check_every={ce}")
                    tried += 1
                    dec.close()
    assert tried >= 30


@pytest.mark.parametrize("mode", MODES)
def test_autotune_keeps_results(torch_cuda, mode):
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Decoder
    code = inputs.cfg_regular_576()
    llr = inputs.all_zero_awgn_llr(500, code.N, 2.0, code.design_rate, 91)
    dec = Decoder.from_code(code, mode=mode)
    ms = dec.autotune(4096, 10)
    ft, th, ip = dec.tuning()
    assert ms > 0 and ft in (1, 2, 4) and th % 32 == 0 and 64 <= th <= 1024 and ip in (1, 2)
    b, it, ok, sf = dec.decode(torch.from_numpy(llr).cuda(), 20, want_ok=True, want_soft=True)
    torch.cuda.synchronize()
    got = (b.cpu().numpy(), it.cpu().numpy(), ok.cpu().numpy(), sf.cpu().numpy())
    assert_parity(got, oracle_decode(code, llr, 20, mode), mode, "after autotune")


@pytest.mark.parametrize("mode", MODES)
def test_paper_shaped_code_with_check_every_6(torch_cuda, mode):
    """The stand-in with the paper's code dimensions (rows of 32 edges, columns of 4), at
    most 60 iterations and the syndrome tested every 6 as in the paper's runs; Eb/N0 from
    the paper's 3.0 dB up to 6.5 dB so that frames stop at 6, 12 and 60 iterations."""
    code = inputs.cfg_paper_shaped()
    cw = inputs.Encoder(code).random_codewords(24, 31)
    snr = np.linspace(3.0, 6.5, 24)
    llr = np.concatenate([inputs.bpsk_awgn_llr(cw[k:k + 1], float(snr[k]), code.design_rate, 50 + k)
                          for k in range(24)])
    want = oracle_decode(code, llr, 60, mode, check_every=6)
    assert len(np.unique(want[1])) >= 3
    got = gpu_decode(torch_cuda, code, llr, 60, mode, check_every=6)
    assert_parity(got, want, mode, "paper-shaped")


@pytest.mark.parametrize("mode", MODES)
def test_autotune_on_the_callers_frames(torch_cuda, mode):
    """ldpc_autotune_data times the shapes on the caller's frames with early stop; the
    decode after it must still equal the oracle, the frames must be left as they were,
    and invalid arguments must be refused before any work."""
    torch = torch_cuda
    from paper_2507_10424_gb300 import ldpc
    from paper_2507_10424_gb300.ldpc import Decoder, LdpcError
    code = inputs.cfg_regular_576()
    llr = inputs.all_zero_awgn_llr(700, code.N, 2.0, code.design_rate, 92)
    x = torch.from_numpy(llr).cuda()
    dec = Decoder.from_code(code, mode=mode)
    ms = dec.autotune(700, 20, llr=x, early_stop=True)
    ft, th, ip = dec.tuning()
    assert ms > 0 and ft in (1, 2, 4) and th % 32 == 0 and 64 <= th <= 1024 and ip in (1, 2)
    assert np.array_equal(x.cpu().numpy(), llr)
    b, it, ok, sf = dec.decode(x, 20, want_ok=True, want_soft=True)
    torch.cuda.synchronize()
    got = (b.cpu().numpy(), it.cpu().numpy(), ok.cpu().numpy(), sf.cpu().numpy())
    assert_parity(got, oracle_decode(code, llr, 20, mode), mode, "after autotune on data")
    for args, status in (((x.data_ptr(), 700, 20, 2, 1), ldpc.LDPC_ERR_INVALID_ARG),
                         ((x.data_ptr(), 700, 20, 1, 0), ldpc.LDPC_ERR_INVALID_ARG),
                         ((x.data_ptr(), 0, 20, 1, 1), ldpc.LDPC_ERR_INVALID_ARG),
                         ((x.data_ptr(), 700, -1, 1, 1), ldpc.LDPC_ERR_INVALID_ARG),
                         ((llr.ctypes.data, 700, 20, 1, 1), ldpc.LDPC_ERR_BAD_POINTER)):
        with pytest.raises(LdpcError) as e:
            ldpc.ldpc_autotune_data(dec.h, *args)
        assert e.value.status == status
    assert dec.tuning() == (ft, th, ip)
    with pytest.raises(ValueError):
        dec.autotune(700, 20, llr=x.double())
    dec.close()


def test_errors_on_device_arguments(torch_cuda):
    torch = torch_cuda
    import ctypes
    from paper_2507_10424_gb300 import ldpc
    code = inputs.qc_code(3, 6, 32, 0.8, 9)
    dec = ldpc.Decoder.from_code(code)
    x = torch.zeros((4, code.N), device="cuda")
    bits = torch.zeros((4, code.N), dtype=torch.uint8, device="cuda")
    it = torch.zeros(4, dtype=torch.int32, device="cuda")
    host = np.zeros((4, code.N), np.float32)
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    assert ldpc.ldpc_decode(dec.h, ctypes.c_void_p(host.ctypes.data), 4, 5, P(bits), P(it)) == \
        ldpc.LDPC_ERR_BAD_POINTER
    assert ldpc.ldpc_decode(dec.h, P(x), -1, 5, P(bits), P(it)) == ldpc.LDPC_ERR_INVALID_ARG
    assert ldpc.ldpc_decode(dec.h, P(x), 4, -2, P(bits), P(it)) == ldpc.LDPC_ERR_INVALID_ARG
    assert ldpc.ldpc_decode_i8(dec.h, P(x), 4, 5, P(bits), P(it)) == ldpc.LDPC_ERR_INVALID_ARG
    assert ldpc.ldpc_decode_ex(dec.h, P(x), 0, 4, 5, 1, 0, P(bits), P(it), None, None) == \
        ldpc.LDPC_ERR_INVALID_ARG
    assert ldpc.ldpc_decode(dec.h, P(x), 0, 5, P(bits), P(it)) == ldpc.LDPC_OK
    big = inputs.cfg_irregular_64800()
    d2 = ldpc.Decoder.from_code(big)
    with pytest.raises(ldpc.LdpcError):
        d2.set_variant("resident")


@pytest.mark.parametrize("early_stop", [True, False])
def test_dense_map_reduce_variant(torch_cuda, early_stop):
    """The paper's dense m x n form (Algorithm 2) on the GPU: bit-exact with the oracle."""
    for code, F, L in ((tanner_code(), 77, 9), (inputs.cfg_regular_576(), 64, 20),
                       (inputs.qc_code(4, 8, 32, 0.7, 3), 33, 12)):
        llr = inputs.all_zero_awgn_llr(F, code.N, 2.0, code.design_rate, 7) if code.N > 10 else \
            (np.random.default_rng(3).standard_normal((F, 10)) * 1.5 + 0.5).astype(np.float32)
        for ce in (1, 3):
            got = gpu_decode(torch_cuda, code, llr, L, "fp32", "dense", early_stop=early_stop,
                             check_every=ce)
            assert got[4] == "dense"
            assert_parity(got, oracle_decode(code, llr, L, "fp32", early_stop=early_stop,
                                             check_every=ce), "fp32", f"dense N={code.N}")


def test_workspace_too_large_is_an_error_not_a_crash(torch_cuda):
    """Reserving a streaming workspace larger than the device returns LDPC_ERR_OOM (nothing
    is launched and no frame buffer is involved), and the handle stays usable. Every
    buffer passed to a decode here holds the frames it is told about."""
    torch = torch_cuda
    import ctypes
    from paper_2507_10424_gb300 import ldpc
    code = inputs.cfg_irregular_64800()
    dec = ldpc.Decoder.from_code(code)
    dec.set_variant("stream")
    x = torch.zeros((8, code.N), device="cuda")
    bits = torch.zeros((8, code.N), dtype=torch.uint8, device="cuda")
    it = torch.zeros(8, dtype=torch.int32, device="cuda")
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    huge = 2_000_000  # frames: about 1.6 TB of edge messages, more than the device holds
    assert ldpc.ldpc_reserve(dec.h, huge) == ldpc.LDPC_ERR_OOM
    assert ldpc.ldpc_decode(dec.h, P(x), 8, 5, P(bits), P(it)) == ldpc.LDPC_OK
    torch.cuda.synchronize()
    assert (it.cpu().numpy() >= 0).all()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("F", [2500, 9000])
def test_host_buffer_pipeline_matches_device_path(torch_cuda, mode, F):
    """2500 frames: even chunks with a ragged last one; 9000 frames: chunk sizes that ramp
    up from and back down to 1024 frames, with a short chunk between."""
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Decoder
    code = inputs.cfg_qc_2304()
    llr = inputs.all_zero_awgn_llr(F, code.N, 1.5, code.design_rate, 77)
    dec = Decoder.from_code(code, mode=mode)
    xh = torch.from_numpy(llr).pin_memory()
    bh, ih, okh, sh = dec.decode_host(xh, 10, want_ok=True, want_soft=True)
    bd, idv, okd, sd = dec.decode(xh.cuda(), 10, want_ok=True, want_soft=True)
    torch.cuda.synchronize()
    assert (bh.numpy() == bd.cpu().numpy()).all() and (ih.numpy() == idv.cpu().numpy()).all()
    assert (okh.numpy() == okd.cpu().numpy()).all() and (sh.numpy() == sd.cpu().numpy()).all()
    sel = np.arange(0, F, 97)
    want = oracle_decode(code, llr[sel], 10, mode)
    assert_parity((bh.numpy()[sel], ih.numpy()[sel], okh.numpy()[sel], sh.numpy()[sel]), want, mode,
                  "host pipeline")


@pytest.mark.slow
@pytest.mark.parametrize("mode", MODES)
def test_full_size_qc_2304_65536_frames_sampled(torch_cuda, mode):
    """The benchmark's workload at full size (65536 random codewords, 10 iterations without
    early stop) in the launch configuration the benchmark times: ``autotune(65536, 10)``
    picks the resident launch shape as the benchmark does, and the decode writes the
    decisions and iteration counts only (no status, no posteriors), as the timed step
    does. A second decode with status and posteriors must give the same decisions; sampled
    frames are compared with the oracle, the status flag with the syndrome on more frames."""
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Decoder
    code = inputs.cfg_qc_2304()
    F = 65536
    cw = inputs.Encoder(code).random_codewords(F, 123)
    llr = inputs.bpsk_awgn_llr(cw, 2.0, code.design_rate, 124)
    dec = Decoder.from_code(code, mode=mode)
    dec.autotune(F, 10)
    shape = dec.tuning()
    assert dec.variant() == "resident"
    x = torch.from_numpy(llr).cuda()
    timed_bits, timed_iters, _, _ = dec.decode(x, 10, early_stop=False)
    bits, iters, ok, soft = dec.decode(x, 10, early_stop=False, want_ok=True, want_soft=True)
    torch.cuda.synchronize()
    assert torch.equal(timed_bits, bits) and torch.equal(timed_iters, iters)
    rng = np.random.default_rng(5)
    sel = np.sort(np.concatenate([rng.choice(F, 60, replace=False), [0, 1, F - 2, F - 1]]))
    want = oracle_decode(code, llr[sel], 10, mode, early_stop=False)
    got = (bits[sel].cpu().numpy(), iters[sel].cpu().numpy(), ok[sel].cpu().numpy(),
           soft[sel].cpu().numpy())
    assert_parity(got, want, mode, f"full-size sample, tuning {shape}")
    assert (iters == 10).all()
    # decoded bits are codewords of H for every frame flagged ok (syndrome property at any size)
    g = oracle.Graph.from_code(code)
    okn = ok.cpu().numpy()
    bn = bits.cpu().numpy()
    for f in rng.choice(F, 200, replace=False):
        assert okn[f] == (oracle.syndrome(g, bn[f])[0] == 0)
    dec.close()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("shape", ["resident 2,768,1", "resident 4,768,1", "resident 1,1024,2",
                                   "stream", "cluster"])
def test_posteriors_after_every_iteration(torch_cuda, mode, shape):
    """Decodes stopped after k = 1 .. 10 iterations (no early stop) return the posteriors
    s of iteration k; each must equal the oracle's (bit for bit in both modes), so every
    iteration's messages enter the comparison, not only the last one's. The resident shapes
    include the benchmark's (2 frames per tile, 768 threads, index arrays in shared memory)."""
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Decoder, LdpcError
    code = inputs.cfg_qc_2304()
    F = 45
    cw = inputs.Encoder(code).random_codewords(F, 77)
    llr = np.concatenate([inputs.bpsk_awgn_llr(cw[k * 9:(k + 1) * 9], e, code.design_rate, 90 + k)
                          for k, e in enumerate([1.0, 1.5, 2.0, 2.5, 3.0])])
    dec = Decoder.from_code(code, mode=mode)
    if shape.startswith("resident"):
        dec.set_variant("resident")
        ft, th, ip = (int(v) for v in shape.split()[1].split(","))
        try:
            dec.set_tuning(ft, th, ip)
        except LdpcError:
            pytest.skip(f"{shape} does not fit this code in {mode}")
    else:
        dec.set_variant(shape)
    x = torch.from_numpy(llr).cuda()
    for k in range(1, 11):
        b, it, ok, sf = dec.decode(x, k, early_stop=False, want_ok=True, want_soft=True)
        torch.cuda.synchronize()
        got = (b.cpu().numpy(), it.cpu().numpy(), ok.cpu().numpy(), sf.cpu().numpy())
        assert_parity(got, oracle_decode(code, llr, k, mode, early_stop=False), mode,
                      f"{shape} after iteration {k}")
    dec.close()


@pytest.mark.parametrize("mode", MODES)
def test_full_size_irregular_64800_4096_frames_sampled(torch_cuda, mode):
    """The large irregular code at the size `bench.py --workload irregular64800` times (4096
    all-zero frames at 1.0 dB, 50 iterations without early stop, autotuned check-pass
    staging), checked on sampled frames against the oracle, and the status flag against the
    syndrome of the decided bits on more frames."""
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Decoder
    code = inputs.cfg_irregular_64800()
    F = 4096
    llr = inputs.all_zero_awgn_llr(F, code.N, 1.0, code.design_rate, 1000)
    dec = Decoder.from_code(code, mode=mode)
    dec.autotune(F, 50)
    x = torch.from_numpy(llr).cuda()
    bits, iters, ok, soft = dec.decode(x, 50, early_stop=False, want_ok=True, want_soft=True)
    dec.check_device()
    rng = np.random.default_rng(6)
    sel = np.sort(np.concatenate([rng.choice(F, 6, replace=False), [0, F - 1]]))
    want = oracle_decode(code, llr[sel], 50, mode, early_stop=False)
    got = (bits[sel].cpu().numpy(), iters[sel].cpu().numpy(), ok[sel].cpu().numpy(),
           soft[sel].cpu().numpy())
    assert_parity(got, want, mode, f"full-size sample, staging {dec.stream_staging()}")
    assert (iters == 50).all()
    g = oracle.Graph.from_code(code)
    okn = ok.cpu().numpy()
    bn = bits.cpu().numpy()
    for f in rng.choice(F, 64, replace=False):
        assert okn[f] == (oracle.syndrome(g, bn[f])[0] == 0)
    dec.close()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("which", ["qc2304 (padded rows)", "qc2304 (padded rows, per-edge messages)",
                                   "paper-shaped (rows of 32: CSR slots)"])
def test_messages_after_the_last_iteration(torch_cuda, mode, which):
    """The check-to-bit messages eta themselves (eq. eta_update), read back from the
    streaming workspace after k iterations without early stop, against the oracle's trace
    of the same frames: bit-exact in fixed point; in FP32 within 1e-5 relative, and
    identical (the check update only compares and selects). FP32 codes with short rows keep
    compressed messages by default (rebuilt for the read-back), or per-edge ones."""
    torch = torch_cuda
    from paper_2507_10424_gb300 import ldpc
    from paper_2507_10424_gb300.ldpc import Decoder, LdpcError
    code = inputs.cfg_qc_2304() if which.startswith("qc") else inputs.cfg_paper_shaped()
    F = 21
    cw = inputs.Encoder(code).random_codewords(F, 44)
    llr = inputs.bpsk_awgn_llr(cw, 2.0 if which.startswith("qc") else 3.2, code.design_rate, 45)
    g = oracle.Graph.from_code(code)
    dec = Decoder.from_code(code, mode=mode)
    dec.set_variant("stream")
    dec.set_stream_staging(8, 2)  # fits rows of 16 edges with compressed messages
    dec.set_stream_messages("per-edge" not in which)
    assert dec.stream_messages_compressed() == (mode == "fp32" and which == "qc2304 (padded rows)")
    x = torch.from_numpy(llr).cuda()
    for k in (1, 3, 7):
        dec.decode(x, k, early_stop=False)
        eta = dec.read_messages(F).cpu().numpy()
        for f in range(F):
            if mode == "fp32":
                want = oracle.trace_f32(g, llr[f], k)[3][k - 1]
                np.testing.assert_allclose(eta[f], want, rtol=RTOL, atol=0, err_msg=f"k={k} f={f}")
                assert (eta[f] == want).all(), f"k={k} frame {f}: messages not identical"
            else:
                want = oracle.trace_fixed(g, oracle.quantize(llr[f]), k)[3][k - 1]
                assert (eta[f] * 4 == want).all(), f"k={k} frame {f}"
    # no messages after an early-stop decode, nor after a resident one
    dec.decode(x, 3, early_stop=True)
    with pytest.raises(LdpcError) as e:
        dec.read_messages(1)
    assert e.value.status == ldpc.LDPC_ERR_UNSUPPORTED
    dec.close()


@pytest.mark.parametrize("compressed", [True, False])
@pytest.mark.parametrize("which", ["qc2304", "irregular2000", "learned576"])
def test_streaming_message_formats(torch_cuda, compressed, which):
    """FP32 streaming decodes with the rows' messages compressed (two minima, location,
    signs) or stored per edge slot, with early stop (syndrome every 1 and every 3
    iterations, frame compaction) and without: identical to the oracle either way; the
    learned case rebuilds each message with the weights of the iteration that sent it."""
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Decoder
    if which == "qc2304":
        code = inputs.cfg_qc_2304()
        cw = inputs.Encoder(code).random_codewords(300, 61)
        llr = inputs.bpsk_awgn_llr(cw, 3.8, code.design_rate, 62)  # frames stop at many iterations
        L = 20
    elif which == "irregular2000":
        code = inputs.irregular_code(2000, 1000, [2, 3, 8], [0.5, 0.375, 0.125], 9)
        llr = inputs.all_zero_awgn_llr(700, code.N, 1.9, code.design_rate, 63)
        L = 30
    else:
        code = inputs.cfg_regular_576()
        llr = inputs.all_zero_awgn_llr(500, code.N, 2.0, code.design_rate, 64)
        L = 15
    dec = Decoder.from_code(code)
    dec.set_variant("stream")
    if which == "qc2304":  # rows of up to 16 edges: 8 warps x 2 stages fit in shared memory
        dec.set_stream_staging(8, 2)
    dec.set_stream_messages(compressed)
    assert dec.stream_messages_compressed() == compressed
    alpha = beta = None
    if which == "learned576":
        alpha = np.linspace(0.7, 0.95, 6, dtype=np.float32)[:, None]
        beta = np.linspace(0.3, 0.05, 6, dtype=np.float32)[:, None]
        dec.set_weights(alpha, beta)
    x = torch.from_numpy(llr).cuda()
    g = oracle.Graph.from_code(code)
    for es, ce in ((True, 1), (True, 3), (False, 1)):
        b, it, ok, sf = dec.decode(x, L, early_stop=es, check_every=ce, want_ok=True, want_soft=True)
        torch.cuda.synchronize()
        got = (b.cpu().numpy(), it.cpu().numpy(), ok.cpu().numpy(), sf.cpu().numpy())
        if alpha is None:
            want = oracle.decode_f32(g, llr, L, es, ce)
        else:
            cc, _ = oracle.column_classes(code)
            want = oracle.decode_weighted_f32(g, llr, L, cc, alpha, beta, early_stop=es, check_every=ce)
        assert_parity(got, want, "fp32", f"{which} compressed={compressed} es={es} ce={ce}")
        if es:
            assert len(np.unique(want[1])) >= 3
    dec.close()

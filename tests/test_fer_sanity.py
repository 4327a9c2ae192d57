"""Error-rate sanity of the decoder against the channel (Section VI: BPSK over AWGN, the
all-zero codeword or random codewords at a stated SNR).

The paper's error-rate curves exist only as figures, so no value can be compared; what the
mathematics fixes is checked instead:
* the channel: hard decisions of the LLRs err with the uncoded BPSK probability
  Q(sqrt(2 R Eb/N0)) (R the design rate), a closed form independent of the decoder;
* the decoder: at the (3,6) N=576 code's SNRs the decoded bit error rate lies below that
  uncoded rate, and the frame error rate does not increase with the SNR (within the
  Monte-Carlo error of the counts);
* the quasi-cyclic N=2304 code of the throughput workload (a dense code for LDPC: column
  weights 3-9): its frame error rate is near 1 at 1-3 dB, where the decodes that fail end
  with more bit errors than the channel made (decoded BER above the uncoded rate), and
  falls steeply between 3.5 and 4.5 dB, above which the decoded BER is far below the
  uncoded one. So FER ~ 1 at the benchmark's SNRs is a property of the code's threshold,
  not of the channel or the LLR scaling.
The oracle is checked on the CPU; the library on the GPU with more frames.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2507_10424_gb300 import inputs


def uncoded_ber(ebn0_db, rate):
    """Q(sqrt(2 R Eb/N0)) = erfc(sqrt(R Eb/N0)) / 2."""
    return 0.5 * math.erfc(math.sqrt(rate * 10.0 ** (ebn0_db / 10.0)))


def mc_sigma(p, n):
    return math.sqrt(max(p * (1 - p), 1.0 / n) / n)


def test_channel_hard_decisions_err_at_the_bpsk_rate():
    for ebn0, rate, seed in ((2.5, 0.5, 3), (1.0, 0.5, 4), (3.0, 0.75, 5)):
        llr = inputs.all_zero_awgn_llr(2000, 576, ebn0, rate, seed)
        p = float((llr < 0).mean())
        want = uncoded_ber(ebn0, rate)
        assert abs(p - want) < 5 * mc_sigma(want, llr.size), (ebn0, rate, p, want)


def error_rates(bits, sent):
    wrong = bits != sent
    return float(wrong.any(axis=1).mean()), float(wrong.mean())


def assert_sane(rates, rate, F, label, ber_from=None):
    """rates: {Eb/N0: (FER, BER)} in ascending SNR."""
    snrs = sorted(rates)
    for a, b in zip(snrs, snrs[1:]):
        fa, fb = rates[a][0], rates[b][0]
        tol = 3 * math.hypot(mc_sigma(fa, F), mc_sigma(fb, F))
        assert fb <= fa + tol, f"{label}: FER rises from {a} dB ({fa}) to {b} dB ({fb})"
    for e in snrs:
        if ber_from is None or e >= ber_from:
            assert rates[e][1] < uncoded_ber(e, rate), f"{label}: BER at {e} dB not below uncoded"


def test_oracle_regular_576_ber_below_uncoded_fer_non_increasing():
    code = inputs.cfg_regular_576()
    g = oracle.Graph.from_code(code)
    F = 3000
    rates = {}
    for k, e in enumerate((1.5, 2.0, 2.5, 3.0)):
        llr = inputs.all_zero_awgn_llr(F, code.N, e, code.design_rate, 500 + k)
        bits = oracle.decode_f32(g, llr, 20, soft=False)[0]
        rates[e] = error_rates(bits, 0)
    assert_sane(rates, code.design_rate, F, "oracle (3,6) N=576")
    assert rates[3.0][0] < rates[1.5][0]  # a waterfall, not a flat line
    assert rates[2.5][1] < 0.1 * uncoded_ber(2.5, code.design_rate)


def test_oracle_qc_2304_waterfall_near_4dB():
    """Random codewords, 10 iterations without early stop (the benchmark's decode)."""
    code = inputs.cfg_qc_2304()
    g = oracle.Graph.from_code(code)
    enc = inputs.Encoder(code)
    F = 200
    rates = {}
    for k, e in enumerate((1.0, 2.0, 2.5, 3.0, 3.5, 4.0, 4.5)):
        cw = enc.random_codewords(F, 700 + k)
        llr = inputs.bpsk_awgn_llr(cw, e, code.design_rate, 800 + k)
        bits = oracle.decode_f32(g, llr, 10, early_stop=False, soft=False)[0]
        rates[e] = error_rates(bits, cw)
    assert_sane(rates, code.design_rate, F, "oracle QC N=2304", ber_from=4.0)
    assert rates[1.0][0] > 0.95 and rates[3.0][0] > 0.9  # FER near 1 where the benchmark runs
    assert rates[3.0][1] > uncoded_ber(3.0, code.design_rate)  # failed decodes spread errors
    assert rates[4.0][0] < 0.2 and rates[4.5][0] < 0.05
    assert rates[4.0][1] < 0.2 * uncoded_ber(4.0, code.design_rate)


@pytest.mark.gpu
@pytest.mark.parametrize("mode", ["fp32", "fixed"])
def test_library_regular_576_ber_below_uncoded_fer_non_increasing(mode):
    import torch
    from paper_2507_10424_gb300 import build
    from paper_2507_10424_gb300.ldpc import Decoder
    build.build()
    code = inputs.cfg_regular_576()
    dec = Decoder.from_code(code, mode=mode)
    F = 20000
    rates = {}
    for k, e in enumerate((1.5, 2.0, 2.5, 3.0, 3.5)):
        llr = inputs.all_zero_awgn_llr(F, code.N, e, code.design_rate, 900 + k)
        bits = dec.decode(torch.from_numpy(llr).cuda(), 20)[0]
        rates[e] = error_rates(bits.cpu().numpy(), 0)
    dec.close()
    assert_sane(rates, code.design_rate, F, f"library (3,6) N=576 {mode}")
    assert rates[3.5][0] < 0.2 * rates[2.0][0]


@pytest.mark.gpu
def test_library_qc_2304_waterfall_near_4dB():
    """The throughput workload's code and decode (random codewords, 10 iterations without
    early stop) on the library, beyond the benchmark's 1-3 dB."""
    import torch
    from paper_2507_10424_gb300 import build
    from paper_2507_10424_gb300.ldpc import Decoder
    build.build()
    code = inputs.cfg_qc_2304()
    enc = inputs.Encoder(code)
    dec = Decoder.from_code(code)
    F = 4000
    rates = {}
    for k, e in enumerate((1.0, 2.0, 3.0, 3.5, 4.0, 4.5)):
        cw = enc.random_codewords(F, 1700 + k)
        llr = inputs.bpsk_awgn_llr(cw, e, code.design_rate, 1800 + k)
        bits = dec.decode(torch.from_numpy(llr).cuda(), 10, early_stop=False)[0]
        rates[e] = error_rates(bits.cpu().numpy(), cw)
    dec.close()
    assert_sane(rates, code.design_rate, F, "library QC N=2304", ber_from=4.0)
    assert rates[3.0][0] > 0.9 and rates[4.0][0] < 0.2 and rates[4.5][0] < 0.02

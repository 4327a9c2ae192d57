"""Device-side debug checks (ldpc_set_debug / LDPC_FLAG_DEBUG / LDPC_DEBUG=1): on valid
handles they pass and change no result, on every layout the codes here build (sliced
resident layout, padded streaming rows, CSR/CSC, weight classes); a NaN LLR makes the
decode refuse with LDPC_ERR_DEVICE_CHECK before any decode kernel runs (outputs left as
they were) and reports the first NaN's frame and bit. A corrupted index array cannot be
produced through the API, so the index checks are tested here for the absence of false
alarms only."""
import numpy as np
import pytest

from paper_2507_10424_gb300 import inputs
from test_gpu_parity import torch_cuda  # noqa: F401

pytestmark = pytest.mark.gpu


def codes():
    mixed, _ = inputs.cfg_mixed_codes()
    return {"regular576": inputs.cfg_regular_576(), "qc2304": inputs.cfg_qc_2304(),
            "irregular1200": inputs.irregular_code(1200, 500, [2, 3, 8], [0.5, 0.375, 0.125], 9),
            "paper_shaped": inputs.cfg_paper_shaped(), "irregular16200": mixed[-1]}


def run(torch, dec, x, L, variant):
    dec.set_variant(variant)
    out = (torch.full((x.shape[0], dec.N), 0xAB, dtype=torch.uint8, device="cuda"),
           torch.full((x.shape[0],), -7, dtype=torch.int32, device="cuda"), None, None)
    dec.decode(x, L, out=out)
    torch.cuda.synchronize()
    return out[0].cpu().numpy(), out[1].cpu().numpy()


@pytest.mark.parametrize("mode", ["fp32", "fixed"])
@pytest.mark.parametrize("name", list(codes()))
def test_checks_pass_on_valid_handles_and_change_nothing(torch_cuda, mode, name):
    from paper_2507_10424_gb300.ldpc import Decoder
    torch = torch_cuda
    code = codes()[name]
    llr = inputs.all_zero_awgn_llr(64, code.N, 2.0, code.design_rate, 5)
    x = torch.from_numpy(llr).cuda()
    plain = Decoder.from_code(code, mode=mode)
    checked = Decoder.from_code(code, mode=mode, debug=True)
    for variant in ("auto", "stream"):
        want = run(torch, plain, x, 12, variant)
        got = run(torch, checked, x, 12, variant)
        assert (got[0] == want[0]).all() and (got[1] == want[1]).all(), (name, variant)
        assert checked.debug_report() == (0, 0)
    plain.close()
    checked.close()


@pytest.mark.parametrize("variant", ["resident", "stream"])
def test_nan_llr_is_refused_before_any_decode(torch_cuda, variant):
    from paper_2507_10424_gb300.ldpc import Decoder, LdpcError, LDPC_ERR_DEVICE_CHECK
    torch = torch_cuda
    code = inputs.cfg_regular_576()
    llr = inputs.all_zero_awgn_llr(40, code.N, 2.0, code.design_rate, 6)
    bad = llr.copy()
    bad[5, 2] = np.nan
    bad[3, 17] = np.nan  # the first in frame-major order
    dec = Decoder.from_code(code, debug=True)
    with pytest.raises(LdpcError) as e:
        run(torch, dec, torch.from_numpy(bad).cuda(), 10, variant)
    assert e.value.status == LDPC_ERR_DEVICE_CHECK
    # the outputs were left as they were: no decode kernel ran
    dec.set_variant(variant)
    out = (torch.full((40, code.N), 0xAB, dtype=torch.uint8, device="cuda"),
           torch.full((40,), -7, dtype=torch.int32, device="cuda"), None, None)
    with pytest.raises(LdpcError):
        dec.decode(torch.from_numpy(bad).cuda(), 10, out=out)
    torch.cuda.synchronize()
    assert (out[0].cpu().numpy() == 0xAB).all() and (out[1].cpu().numpy() == -7).all()
    assert dec.debug_report() == (1, 3 * code.N + 17)
    assert dec.debug_report() == (0, 0)  # cleared by the read
    # a clean batch decodes, and equals the unchecked decoder's result
    good = run(torch, dec, torch.from_numpy(llr).cuda(), 10, variant)
    ref = Decoder.from_code(code)
    assert all((a == b).all() for a, b in zip(good, run(torch, ref, torch.from_numpy(llr).cuda(), 10, variant)))
    # with the checks off the same NaN batch is not refused
    dec.set_debug(False)
    run(torch, dec, torch.from_numpy(bad).cuda(), 10, variant)
    ref.close()
    dec.close()


def test_debug_from_the_environment_and_int8_input(torch_cuda, monkeypatch):
    from paper_2507_10424_gb300.ldpc import Decoder, LdpcError, LDPC_ERR_DEVICE_CHECK
    torch = torch_cuda
    code = inputs.cfg_regular_576()
    bad = inputs.all_zero_awgn_llr(8, code.N, 2.0, code.design_rate, 7)
    bad[0, 0] = np.nan
    x = torch.from_numpy(bad).cuda()
    monkeypatch.setenv("LDPC_DEBUG", "1")
    dec = Decoder.from_code(code)
    with pytest.raises(LdpcError) as e:
        run(torch, dec, x, 5, "auto")
    assert e.value.status == LDPC_ERR_DEVICE_CHECK and dec.debug_report() == (1, 0)
    dec.close()
    monkeypatch.setenv("LDPC_DEBUG", "0")
    dec = Decoder.from_code(code)
    run(torch, dec, x, 5, "auto")  # not refused
    dec.close()
    # int8 input (fixed point) has no NaN: the index checks alone run and pass
    monkeypatch.setenv("LDPC_DEBUG", "1")
    dec = Decoder.from_code(code, mode="fixed")
    q = torch.from_numpy(np.clip(np.rint(4 * np.nan_to_num(bad)), -127, 127).astype(np.int8)).cuda()
    run(torch, dec, q, 5, "auto")
    assert dec.debug_report() == (0, 0)
    dec.close()

"""GPU tests of the learned (normalised / offset) Min-Sum decoder: weighted inference
against the oracle (bit-exact decisions and iteration counts, posteriors within 1e-5
relative), the training forward against the decode path, and the hand-written adjoint
against an autograd reference (tiny codes) and against central finite differences of the
binary64 oracle (eps = 1e-3, relative tolerance 1e-3)."""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import learned_ref
from paper_2507_10424_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2507_10424_gb300 import build
    build.build()
    return torch


def irregular_code():
    return inputs.irregular_code(240, 120, [2, 3, 6], [0.4, 0.4, 0.2], 11)


def random_weights(T, C, seed):
    rng = np.random.default_rng(seed)
    return (rng.uniform(0.6, 1.0, (T, C)).astype(np.float32),
            rng.uniform(0.0, 0.4, (T, C)).astype(np.float32))


@pytest.mark.parametrize("variant", ["stream", "resident", "cluster"])
@pytest.mark.parametrize("early_stop", [True, False])
def test_weighted_decode_matches_oracle(torch_cuda, variant, early_stop):
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Decoder
    for code in (inputs.cfg_regular_576(), irregular_code()):
        cls, degrees = oracle.column_classes(code)
        dec = Decoder.from_code(code)
        assert dec.classes() == list(degrees)
        a, b = random_weights(6, len(degrees), 3)
        dec.set_weights(a, b)
        dec.set_variant(variant)
        llr = inputs.all_zero_awgn_llr(333, code.N, 2.0, code.design_rate, 5)
        bits, it, ok, soft = dec.decode(torch.from_numpy(llr).cuda(), 15, early_stop=early_stop,
                                        want_ok=True, want_soft=True)
        torch.cuda.synchronize()
        g = oracle.Graph.from_code(code)
        wb, wi, wok, ws = oracle.decode_weighted_f32(g, llr, 15, cls, a, b, early_stop=early_stop)
        assert (it.cpu().numpy() == wi).all() and (ok.cpu().numpy() == wok).all()
        assert (bits.cpu().numpy() == wb).all()
        np.testing.assert_allclose(soft.cpu().numpy(), ws, rtol=RTOL, atol=0)
        dec.close()


@pytest.mark.parametrize("shape", ["2,768,1", "4,768,1", "1,256,1", "1,1024,2", "2,384,2"])
@pytest.mark.parametrize("early_stop", [True, False])
def test_one_class_weights_over_resident_shapes(torch_cuda, shape, early_stop):
    """A regular code has one weight class, so the resident rows apply the weights to their
    two candidate magnitudes once (the unrolled row bodies) instead of per edge. Every
    launch shape, with and without early stop (tested every iteration and every third),
    must equal the oracle's weighted decode bit for bit, posteriors included."""
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Decoder, LdpcError
    code = inputs.cfg_regular_576()
    cls, degrees = oracle.column_classes(code)
    assert len(degrees) == 1
    a, b = random_weights(7, 1, 13)
    llr = inputs.all_zero_awgn_llr(259, code.N, 2.5, code.design_rate, 17)
    g = oracle.Graph.from_code(code)
    dec = Decoder.from_code(code)
    dec.set_weights(a, b)
    dec.set_variant("resident")
    ft, th, ip = (int(v) for v in shape.split(","))
    try:
        dec.set_tuning(ft, th, ip)
    except LdpcError:
        pytest.skip(f"{shape} does not fit this code")
    x = torch.from_numpy(llr).cuda()
    for check_every in ((1, 3) if early_stop else (1,)):
        bits, it, ok, soft = dec.decode(x, 12, early_stop=early_stop, check_every=check_every,
                                        want_ok=True, want_soft=True)
        torch.cuda.synchronize()
        wb, wi, wok, ws = oracle.decode_weighted_f32(g, llr, 12, cls, a, b, early_stop=early_stop,
                                                     check_every=check_every)
        assert (it.cpu().numpy() == wi).all() and (ok.cpu().numpy() == wok).all()
        assert (bits.cpu().numpy() == wb).all()
        assert (soft.cpu().numpy() == ws).all(), (shape, early_stop, check_every)
    assert wi.max() > 1
    dec.close()


@pytest.mark.parametrize("variant", ["stream", "resident", "cluster"])
def test_unit_weights_equal_plain_on_gpu(torch_cuda, variant):
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Decoder
    code = irregular_code()
    dec = Decoder.from_code(code)
    dec.set_variant(variant)
    x = torch.from_numpy(inputs.all_zero_awgn_llr(100, code.N, 1.5, 0.5, 9)).cuda()
    plain = dec.decode(x, 12, want_soft=True)
    C = len(dec.classes())
    dec.set_weights(np.ones((3, C)), np.zeros((3, C)))
    learned = dec.decode(x, 12, want_soft=True)
    torch.cuda.synchronize()
    assert (plain[0] == learned[0]).all() and (plain[1] == learned[1]).all()
    assert (plain[3] == learned[3]).all()
    dec.set_mode("fixed")
    with pytest.raises(Exception):
        dec.decode(x, 12)  # learned weights are an FP32-mode feature


def test_training_forward_equals_decode(torch_cuda):
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Decoder
    from paper_2507_10424_gb300.learn import WeightedMinSum
    code = irregular_code()
    cls, degrees = oracle.column_classes(code)
    dec = Decoder.from_code(code)
    T = 7
    a, b = random_weights(T, len(degrees), 12)
    llr = inputs.all_zero_awgn_llr(77, code.N, 2.0, code.design_rate, 13)
    x = torch.from_numpy(llr).cuda()
    soft = WeightedMinSum.apply(dec, x, torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
    dec.set_weights(a, b)
    _, _, _, soft2 = dec.decode(x, T, early_stop=False, want_soft=True)
    torch.cuda.synchronize()
    assert (soft.cpu().numpy() == soft2.cpu().numpy()).all()
    g = oracle.Graph.from_code(code)
    ws = oracle.decode_weighted_f32(g, llr, T, cls, a, b, early_stop=False)[3]
    np.testing.assert_allclose(soft.cpu().numpy(), ws, rtol=RTOL, atol=0)


def gpu_grads(torch, dec, llr, cw, a, b):
    from paper_2507_10424_gb300.learn import WeightedMinSum
    ta = torch.from_numpy(a).cuda().requires_grad_()
    tb = torch.from_numpy(b).cuda().requires_grad_()
    soft = WeightedMinSum.apply(dec, torch.from_numpy(llr).cuda(), ta, tb)
    loss = torch.nn.functional.binary_cross_entropy_with_logits(
        -soft, torch.from_numpy(cw).cuda().float(), reduction="sum")
    loss.backward()
    return ta.grad.cpu().numpy().astype(np.float64), tb.grad.cpu().numpy().astype(np.float64)


def test_every_iteration_outputs_and_their_adjoint(torch_cuda):
    """Posteriors after every iteration, and the adjoint of a loss that uses all of them,
    against the autograd reference."""
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Decoder
    from paper_2507_10424_gb300.learn import WeightedMinSum
    code = inputs.irregular_code(40, 20, [2, 3, 4], [0.4, 0.4, 0.2], 21)
    cls, degrees = oracle.column_classes(code)
    dec = Decoder.from_code(code)
    T = 4
    a, b = random_weights(T, len(degrees), 41)
    cw = inputs.Encoder(code).random_codewords(20, 42)
    llr = inputs.bpsk_awgn_llr(cw, 1.5, code.design_rate, 43)
    ta = torch.from_numpy(a).cuda().requires_grad_()
    tb = torch.from_numpy(b).cuda().requires_grad_()
    soft = WeightedMinSum.apply(dec, torch.from_numpy(llr).cuda(), ta, tb, True)
    assert soft.shape == (T, 20, code.N)
    last = WeightedMinSum.apply(dec, torch.from_numpy(llr).cuda(), ta.detach(), tb.detach())
    assert (soft[-1] == last).all()
    tgt = torch.from_numpy(cw).cuda().float().expand_as(soft)
    torch.nn.functional.binary_cross_entropy_with_logits(-soft, tgt, reduction="sum").backward()
    rows = [list(code.cols[code.rows == i]) for i in range(code.M)]
    ra = torch.from_numpy(a.astype(np.float64)).requires_grad_()
    rb = torch.from_numpy(b.astype(np.float64)).requires_grad_()
    r64 = torch.from_numpy(llr.astype(np.float64))
    total = 0
    for t in range(1, T + 1):
        s = learned_ref.unrolled_posteriors(rows, code.N, cls, r64, ra[:t], rb[:t])
        total = total + learned_ref.bce_loss(s, torch.from_numpy(cw))
    total.backward()
    np.testing.assert_allclose(ta.grad.cpu().numpy(), ra.grad.numpy(), rtol=1e-3, atol=1e-3)
    np.testing.assert_allclose(tb.grad.cpu().numpy(), rb.grad.numpy(), rtol=1e-3, atol=1e-3)


def code_with_a_long_row():
    """The 40-bit code below plus a check over 20 of its bits: with a row longer than 16
    edges the training state keeps one sign byte per edge instead of folding the row's
    sign bits into its word."""
    base = inputs.irregular_code(40, 20, [2, 3, 4], [0.4, 0.4, 0.2], 21)
    sets = [list(base.cols[base.rows == i] + 1) for i in range(base.M)]
    sets.append(list(np.random.default_rng(5).choice(40, 20, replace=False) + 1))
    return inputs.code_from_index_sets(sets, 40)


@pytest.mark.parametrize("long_row", [False, True])
def test_adjoint_matches_autograd_reference(torch_cuda, long_row):
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Decoder
    code = code_with_a_long_row() if long_row else inputs.irregular_code(40, 20, [2, 3, 4], [0.4, 0.4, 0.2], 21)
    assert (code.row_weights().max() > 16) == long_row
    cls, degrees = oracle.column_classes(code)
    dec = Decoder.from_code(code)
    T = 5
    a, b = random_weights(T, len(degrees), 22)
    enc = inputs.Encoder(code)
    cw = enc.random_codewords(24, 23)
    llr = inputs.bpsk_awgn_llr(cw, 1.5, code.design_rate, 24)
    ga, gb = gpu_grads(torch, dec, llr, cw, a, b)
    rows = [list(code.cols[code.rows == i]) for i in range(code.M)]
    ra = torch.from_numpy(a.astype(np.float64)).requires_grad_()
    rb = torch.from_numpy(b.astype(np.float64)).requires_grad_()
    s = learned_ref.unrolled_posteriors(rows, code.N, cls, torch.from_numpy(llr.astype(np.float64)), ra, rb)
    learned_ref.bce_loss(s, torch.from_numpy(cw)).backward()
    np.testing.assert_allclose(ga, ra.grad.numpy(), rtol=1e-3, atol=1e-3)
    np.testing.assert_allclose(gb, rb.grad.numpy(), rtol=1e-3, atol=1e-3)


def test_adjoint_matches_finite_differences(torch_cuda):
    """Central differences of the binary64 oracle's loss, eps = 1e-3, relative tolerance
    1e-3, at the weights where the loss is smooth over +-eps (no minimum changes its
    location and no magnitude crosses zero there: the differences at eps and eps/4 agree)."""
    torch = torch_cuda
    from paper_2507_10424_gb300.ldpc import Decoder
    code = inputs.irregular_code(60, 30, [2, 3, 5], [0.4, 0.4, 0.2], 3)
    cls, degrees = oracle.column_classes(code)
    g = oracle.Graph.from_code(code)
    dec = Decoder.from_code(code)
    T, C = 4, len(degrees)
    a, b = random_weights(T, C, 31)
    enc = inputs.Encoder(code)
    cw = enc.random_codewords(6, 32)
    llr = inputs.bpsk_awgn_llr(cw, 2.0, code.design_rate, 33)
    ga, gb = gpu_grads(torch, dec, llr, cw, a, b)

    def loss64(aa, bb):
        s = oracle.decode_weighted_f64(g, llr.astype(np.float64), T, cls, aa, bb)
        z = -s  # logits of P(bit = 1)
        return float(np.sum(np.logaddexp(0.0, z) - cw * z))

    def central(p64, t, c, eps, aa, bb):
        keep = p64[t, c]
        p64[t, c] = keep + eps
        lp = loss64(aa, bb)
        p64[t, c] = keep - eps
        lm = loss64(aa, bb)
        p64[t, c] = keep
        return (lp - lm) / (2 * eps)

    eps = 1e-3
    a64, b64 = a.astype(np.float64), b.astype(np.float64)
    compared = 0
    for t in range(T):
        for c in range(C):
            for p64, grad in ((a64, ga), (b64, gb)):
                fd = central(p64, t, c, eps, a64, b64)
                fd4 = central(p64, t, c, eps / 4, a64, b64)
                if abs(fd - fd4) > 1e-6 * max(1.0, abs(fd)):
                    continue  # a kink within +-eps: no derivative to compare with
                compared += 1
                assert abs(fd - grad[t, c]) <= 1e-3 * max(1.0, abs(fd)), (t, c, fd, grad[t, c])
    assert compared >= T * C  # at least half of the weights were checked


def test_a_few_training_steps_lower_the_loss(torch_cuda):
    from paper_2507_10424_gb300.ldpc import Decoder
    from paper_2507_10424_gb300.learn import train_weights
    code = inputs.cfg_regular_576()
    dec = Decoder.from_code(code)
    a, b, losses = train_weights(dec, code, iters=5, steps=40, batch=1024, lr=0.03, seed=3)
    assert a.shape == (5, 1) and np.isfinite(a).all() and np.isfinite(b).all()
    assert np.mean(losses[-5:]) < np.mean(losses[:5])


@pytest.mark.parametrize("long_row", [False, True])
def test_training_workspace_size(torch_cuda, long_row):
    """Per frame: r, s and the bit-pass gradient (4 N bytes each), messages and their
    gradient (4 E bytes each), and per iteration 12 M bytes of saved check state; a code
    with a row longer than 16 edges adds a sign byte per edge and iteration. Each region
    starts 256-byte aligned, frames are padded to a multiple of 32."""
    from paper_2507_10424_gb300 import ldpc
    from paper_2507_10424_gb300.ldpc import Decoder
    code = code_with_a_long_row() if long_row else inputs.cfg_regular_576()
    dec = Decoder.from_code(code)
    F, T = 1000, 10
    Fp = (F + 31) // 32 * 32
    al = lambda x: (x + 255) // 256 * 256
    want = (3 * al(code.N * Fp * 4) + 2 * al(code.E * Fp * 4) + 3 * al(T * code.M * Fp * 4)
            + (al(T * code.E * Fp) if long_row else 0))
    assert ldpc.ldpc_train_workspace_size(dec.h, F, T) == want
    dec.close()

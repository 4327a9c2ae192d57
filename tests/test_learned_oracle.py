"""Pins for the weighted (normalised/offset) Min-Sum oracle and its autograd reference."""
import numpy as np
import torch

import oracle
from oracle import learned_ref
from paper_2507_10424_gb300 import inputs


def small_code():
    return inputs.irregular_code(60, 30, [2, 3, 5], [0.4, 0.4, 0.2], 3)


def test_column_classes():
    code = small_code()
    cls, degrees = oracle.column_classes(code)
    assert list(degrees) == [2, 3, 5]
    assert (degrees[cls] == code.col_weights()).all()
    c1, d1 = oracle.column_classes(inputs.cfg_regular_576())
    assert list(d1) == [3] and (c1 == 0).all()


def test_unit_weights_are_plain_min_sum():
    code = small_code()
    g = oracle.Graph.from_code(code)
    cls, degrees = oracle.column_classes(code)
    r = (np.random.default_rng(1).standard_normal((40, code.N)) * 2 + 0.7).astype(np.float32)
    T = 7
    a, b = np.ones((T, len(degrees)), np.float32), np.zeros((T, len(degrees)), np.float32)
    for es in (True, False):
        w = oracle.decode_weighted_f32(g, r, 12, cls, a, b, early_stop=es)
        p = oracle.decode_f32(g, r, 12, early_stop=es)
        for x, y in zip(w, p):
            assert (x == y).all()


def test_single_check_closed_form():
    # one check over 6 bits (Fig. 1 shape, all in): after one iteration
    # s_j = r_j + prod_{k != j} sign(r_k) * max(alpha * min_{k != j} |r_k| - beta, 0)
    code = inputs.code_from_index_sets([[1, 2, 3, 4, 5, 6]], 6)
    g = oracle.Graph.from_code(code)
    cls = np.zeros(6, np.int32)
    rng = np.random.default_rng(4)
    for _ in range(200):
        r = rng.integers(-12, 13, size=6).astype(np.float32)
        alpha = np.float32(rng.choice([0.5, 0.75, 1.25]))
        beta = np.float32(rng.choice([0.0, 0.5, 1.0, 3.0]))
        _, _, _, s = oracle.decode_weighted_f32(g, r, 1, cls, [[alpha]], [[beta]], early_stop=False)
        for j in range(6):
            o = np.delete(r, j)
            sign = -1.0 if (o < 0).sum() % 2 else 1.0
            mag = max(float(alpha) * np.abs(o).min() - float(beta), 0.0)  # exact: dyadic values
            assert s[0, j] == r[j] + sign * mag


def test_large_offset_silences_every_check():
    code = small_code()
    g = oracle.Graph.from_code(code)
    cls, degrees = oracle.column_classes(code)
    r = np.random.default_rng(2).standard_normal((10, code.N)).astype(np.float32)
    a = np.ones((3, len(degrees)), np.float32)
    b = np.full((3, len(degrees)), 1e6, np.float32)
    _, it, _, s = oracle.decode_weighted_f32(g, r, 3, cls, a, b, early_stop=False)
    assert (s == r).all() and (it == 3).all()


def test_rows_beyond_the_table_reuse_its_last_row():
    code = small_code()
    g = oracle.Graph.from_code(code)
    cls, degrees = oracle.column_classes(code)
    r = np.random.default_rng(3).standard_normal((8, code.N)).astype(np.float32)
    rng = np.random.default_rng(5)
    a2 = rng.uniform(0.6, 1.0, (2, len(degrees))).astype(np.float32)
    b2 = rng.uniform(0.0, 0.3, (2, len(degrees))).astype(np.float32)
    a5 = np.concatenate([a2, np.repeat(a2[-1:], 3, 0)])
    b5 = np.concatenate([b2, np.repeat(b2[-1:], 3, 0)])
    x = oracle.decode_weighted_f32(g, r, 5, cls, a2, b2, early_stop=False)
    y = oracle.decode_weighted_f32(g, r, 5, cls, a5, b5, early_stop=False)
    assert (x[3] == y[3]).all()


def test_torch_reference_matches_c_oracle_in_binary64():
    code = small_code()
    g = oracle.Graph.from_code(code)
    cls, degrees = oracle.column_classes(code)
    rng = np.random.default_rng(6)
    T, C = 4, len(degrees)
    r = rng.standard_normal((5, code.N)) * 2 + 0.5
    a = rng.uniform(0.5, 1.0, (T, C))
    b = rng.uniform(0.0, 0.4, (T, C))
    want = oracle.decode_weighted_f64(g, r, T, cls, a, b)
    rows = [list(code.cols[code.rows == i]) for i in range(code.M)]
    got = learned_ref.unrolled_posteriors(rows, code.N, cls, torch.from_numpy(r), torch.from_numpy(a),
                                          torch.from_numpy(b)).numpy()
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_torch_reference_gradient_matches_finite_differences():
    code = inputs.irregular_code(24, 12, [2, 3], [0.5, 0.5], 7)
    cls, degrees = oracle.column_classes(code)
    rows = [list(code.cols[code.rows == i]) for i in range(code.M)]
    rng = np.random.default_rng(8)
    T, C = 3, len(degrees)
    r = torch.from_numpy(rng.standard_normal((4, code.N)) * 2 + 0.5)
    cw = torch.zeros(4, code.N)
    a = torch.from_numpy(rng.uniform(0.6, 1.0, (T, C))).requires_grad_()
    b = torch.from_numpy(rng.uniform(0.0, 0.2, (T, C))).requires_grad_()
    loss = learned_ref.bce_loss(learned_ref.unrolled_posteriors(rows, code.N, cls, r, a, b), cw)
    ga, gb = torch.autograd.grad(loss, (a, b))
    eps = 1e-6
    for (tt, cc) in [(0, 0), (1, 1), (2, 0)]:
        for param, grad in ((a, ga), (b, gb)):
            with torch.no_grad():
                p0 = param[tt, cc].item()
                param[tt, cc] = p0 + eps
                lp = learned_ref.bce_loss(learned_ref.unrolled_posteriors(rows, code.N, cls, r, a, b), cw)
                param[tt, cc] = p0 - eps
                lm = learned_ref.bce_loss(learned_ref.unrolled_posteriors(rows, code.N, cls, r, a, b), cw)
                param[tt, cc] = p0
            fd = (lp - lm).item() / (2 * eps)
            assert abs(fd - grad[tt, cc].item()) <= 1e-5 * max(1.0, abs(fd))

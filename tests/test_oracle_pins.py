"""Pins for the CPU oracle against facts fixed by the paper and by the mathematics.

Each test ties the oracle to something other than itself: the paper's printed examples
(Section II-A, Fig. 1), the literal check-update definition (eq. eta_update), closed
forms, brute-force maximum marginals over all codewords of cycle-free codes, GF(2) brute
force, and invariants of the algorithm.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2507_10424_gb300 import inputs
from conftest import read_golden


# ---------------------------------------------------------------- helpers (brute force)

def all_vectors(n):
    return ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)


def brute_codewords(H):
    V = all_vectors(H.shape[1])
    ok = ((V.astype(np.int64) @ H.T.astype(np.int64)) % 2 == 0).all(axis=1)
    return V[ok]


def max_marginals(H, r):
    """s*_j = max_{c: c_j=0} (-sum c r) - max_{c: c_j=1} (-sum c r), over codewords c."""
    C = brute_codewords(H).astype(np.float64)
    score = -(C @ np.asarray(r, np.float64))
    out = np.empty(H.shape[1])
    for j in range(H.shape[1]):
        out[j] = score[C[:, j] == 0].max() - score[C[:, j] == 1].max()
    return out


def tanner():
    rows = read_golden("tanner_10x5.txt")
    sets = [r[1] for r in rows]
    printed = [r[2] for r in rows]
    return inputs.code_from_index_sets(sets, 10, name="tanner"), sets, printed


# ---------------------------------------------------------------- Section II-A / Fig. 1

def test_tanner_index_sets_and_printed_indicators():
    code, sets, printed = tanner()
    H = code.dense()
    for c, (s, ind) in enumerate(zip(sets, printed)):
        built = [1 if j + 1 in s else 0 for j in range(10)]
        assert built == list(H[c])
        if c == 2:
            # the printed indicator of check 3 is a copy of check 1's (misprint)
            assert ind == printed[0] and ind != built
        else:
            assert ind == built
    assert (H.sum(axis=1) == 6).all() and (H.sum(axis=0) == 3).all()


def test_tanner_syndrome_on_all_vectors():
    code, _, _ = tanner()
    H = code.dense()
    g = oracle.Graph(code.M, code.N, dense=H)
    V = all_vectors(10)
    zero = []
    for v in V:
        n, z = oracle.syndrome(g, v)
        expect = (H.astype(np.int64) @ v) % 2  # eq. (1): sum over the index set mod 2
        assert (z == expect).all() and n == expect.sum()
        zero.append(n == 0)
    zero = np.array(zero)
    assert zero.sum() == 32  # 2^(10 - rank 5): the kernel of H over GF(2)
    assert zero[-1]  # all-ones vector: every row has even weight
    assert zero[0]


def test_fig1_single_parity_check():
    (k,), I, ind = read_golden("spc_fig1.txt")[0]
    assert [1 if j + 1 in I else 0 for j in range(k)] == ind
    code = inputs.code_from_index_sets([I], k)
    g = oracle.Graph.from_code(code)
    for v in all_vectors(k):
        n, z = oracle.syndrome(g, v)
        assert n == (v[0] ^ v[1] ^ v[3] ^ v[4])  # Bit_1 xor Bit_2 xor Bit_4 xor Bit_5


def test_fig1_single_check_min_sum_is_exact():
    (k,), I, _ = read_golden("spc_fig1.txt")[0]
    code = inputs.code_from_index_sets([I], k)
    g = oracle.Graph.from_code(code)
    rng = np.random.default_rng(7)
    for _ in range(50):
        r = rng.integers(-9, 10, size=k).astype(np.float32)
        _, it, _, s = oracle.decode_f32(g, r, L=1, early_stop=False)
        assert it == 1
        assert (s[0] == max_marginals(code.dense(), r)).all()


# ---------------------------------------------------------------- check update

@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int32])
def test_check_update_literal_equals_observations(dtype):
    rng = np.random.default_rng(11)
    for d in list(range(2, 17)) + [24, 32, 48, 64]:
        for trial in range(40):
            if dtype == np.int32:
                lam = rng.integers(-6, 7, size=d).astype(np.int32)  # many ties and zeros
                if trial % 5 == 0:
                    lam = rng.choice([-32767, 32767, 0, 1, -1], size=d).astype(np.int32)
            else:
                lam = (rng.standard_normal(d) * 3).astype(dtype)
                if trial % 3 == 0:
                    lam = np.round(lam).astype(dtype)  # ties, +0 and -0
                    lam[rng.integers(0, d)] = -0.0
            a = oracle.check_row(lam, oracle.CHECK_BRUTE)
            b = oracle.check_row(lam, oracle.CHECK_TWOMIN)
            assert (a == b).all(), (d, lam, a, b)


@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int32])
def test_check_update_closed_forms(dtype):
    rng = np.random.default_rng(3)
    for _ in range(100):
        lam = rng.integers(-50, 51, size=3).astype(dtype)
        for variant in (oracle.CHECK_BRUTE, oracle.CHECK_TWOMIN):
            e2 = oracle.check_row(lam[:2].copy(), variant)
            # degree 2: each side receives the other's value (sign(0) = +1)
            assert e2[0] == lam[1] and e2[1] == lam[0]
            e3 = oracle.check_row(lam.copy(), variant)
            for j in range(3):
                o = [lam[k] for k in range(3) if k != j]
                sgn = (-1) ** sum(1 for v in o if v < 0)
                assert e3[j] == sgn * min(abs(o[0]), abs(o[1]))


def test_check_update_tie_gives_equal_minima():
    lam = np.array([3.0, -1.0, 5.0, 1.0, 2.0], np.float32)
    e = oracle.check_row(lam)
    assert np.abs(e).tolist() == [1.0, 1.0, 1.0, 1.0, 1.0]


# ---------------------------------------------------------------- whole decoder on trees

@pytest.mark.parametrize("seed", range(12))
def test_tree_codes_give_exact_max_marginals(seed):
    code = inputs.tree_code(n_checks=2 + seed % 4, seed=seed)
    assert code.N <= 16
    H = code.dense()
    g = oracle.Graph.from_code(code)
    rng = np.random.default_rng(100 + seed)
    L = code.M + 2  # at least the tree's diameter in check steps
    for _ in range(20):
        r = rng.integers(-20, 21, size=code.N)
        mm = max_marginals(H, r)
        _, it, _, s32 = oracle.decode_f32(g, r.astype(np.float32), L, early_stop=False)
        _, _, _, s64 = oracle.decode_f64(g, r.astype(np.float64), L, early_stop=False)
        b8, _, _, s16 = oracle.decode_fixed(g, r.astype(np.int8), L, early_stop=False)
        assert it == L
        assert (s32[0] == mm).all()
        assert (s64[0] == mm).all()
        assert (s16[0] == mm).all()
        decided = mm != 0
        assert (b8[0][decided] == (mm[decided] < 0)).all()


def test_three_chained_checks_tree():
    code = inputs.code_from_index_sets([[1, 2, 3], [3, 4, 5], [5, 6, 7]], 7)
    g = oracle.Graph.from_code(code)
    rng = np.random.default_rng(5)
    for _ in range(100):
        r = rng.integers(-15, 16, size=7)
        _, _, _, s = oracle.decode_f32(g, r.astype(np.float32), L=4, early_stop=False)
        assert (s[0] == max_marginals(code.dense(), r)).all()


def test_float_error_bound_against_exact_marginals():
    rng = np.random.default_rng(9)
    for seed in range(8):
        code = inputs.tree_code(n_checks=4, seed=seed)
        g = oracle.Graph.from_code(code)
        L = code.M + 2
        dmax = int(max(code.row_weights().max(), code.col_weights().max()))
        for _ in range(10):
            r = rng.standard_normal(code.N) * 4
            mm = max_marginals(code.dense(), r)
            _, _, _, s32 = oracle.decode_f32(g, r.astype(np.float32), L, early_stop=False)
            _, _, _, s64 = oracle.decode_f64(g, r, L, early_stop=False)
            scale = np.abs(r).sum()
            bound32 = L * (dmax + 2) * np.finfo(np.float32).eps * scale
            bound64 = L * (dmax + 2) * np.finfo(np.float64).eps * scale
            r32err = np.abs(r.astype(np.float32).astype(np.float64) - r).max()
            assert np.abs(s32[0] - mm).max() <= bound32 + code.N * r32err
            assert np.abs(s64[0] - mm).max() <= bound64


# ---------------------------------------------------------------- Algorithm 1 == Algorithm 2

@pytest.mark.parametrize("which", ["regular", "qc", "irregular", "tanner"])
def test_dense_map_reduce_equals_graph_form(which):
    code = {"regular": lambda: inputs.regular_code(48, 24, 3, 6, 4),
            "qc": lambda: inputs.qc_code(3, 6, 8, 0.6, 5),
            "irregular": lambda: inputs.irregular_code(60, 30, [2, 3, 6], [0.4, 0.4, 0.2], 6),
            "tanner": lambda: tanner()[0]}[which]()
    H = code.dense()
    g = oracle.Graph(code.M, code.N, dense=H)
    rng = np.random.default_rng(21)
    for t in range(12):
        r = (rng.standard_normal(code.N) * 2 + 0.5).astype(np.float32)
        es = bool(t % 2)
        b2, it2, ok2, s2 = oracle.decode_dense_f32(H, r, 15, early_stop=es)
        for variant in (oracle.CHECK_TWOMIN, oracle.CHECK_BRUTE):
            b1, it1, ok1, s1 = oracle.decode_f32(g, r, 15, early_stop=es, variant=variant)
            assert it1[0] == it2 and ok1[0] == ok2
            assert (b1[0] == b2).all()
            assert (s1[0] == s2).all()


# ---------------------------------------------------------------- invariants

def small_qc():
    return inputs.qc_code(4, 8, 16, 0.6, 13)


def test_codewords_stop_before_first_iteration():
    code = small_qc()
    g = oracle.Graph.from_code(code)
    cw = inputs.Encoder(code).random_codewords(64, 1)
    for c in cw:
        assert oracle.syndrome(g, c)[0] == 0
    r = (1.0 - 2.0 * cw.astype(np.float32)) * 3.5
    b, it, ok, _ = oracle.decode_f32(g, r, 20)
    assert (it == 0).all() and (ok == 1).all() and (b == cw).all()
    q = oracle.quantize(r)
    b, it, ok, _ = oracle.decode_fixed(g, q, 20)
    assert (it == 0).all() and (ok == 1).all() and (b == cw).all()
    pos = np.full((3, code.N), 0.7, np.float32)
    b, it, ok, _ = oracle.decode_f32(g, pos, 20)
    assert (it == 0).all() and (b == 0).all()


def test_zero_iterations_is_the_input_decision():
    code = small_qc()
    g = oracle.Graph.from_code(code)
    r = np.random.default_rng(2).standard_normal((8, code.N)).astype(np.float32)
    b, it, ok, s = oracle.decode_f32(g, r, 0)
    assert (it == 0).all() and (s == r).all() and (b == (r < 0)).all()
    for f in range(8):
        assert ok[f] == (oracle.syndrome(g, b[f])[0] == 0)


def test_power_of_two_scaling():
    code = small_qc()
    g = oracle.Graph.from_code(code)
    rng = np.random.default_rng(4)
    r = (rng.standard_normal((16, code.N)) * 2 + 0.8).astype(np.float32)
    b, it, ok, s = oracle.decode_f32(g, r, 12)
    for p in (-3, 5):
        b2, it2, ok2, s2 = oracle.decode_f32(g, np.ldexp(r, p), 12)
        assert (b2 == b).all() and (it2 == it).all() and (ok2 == ok).all()
        assert (s2 == np.ldexp(s, p)).all()


def test_channel_symmetry():
    code = small_qc()
    g = oracle.Graph.from_code(code)
    cw = inputs.Encoder(code).random_codewords(32, 8)
    rng = np.random.default_rng(10)
    r = (rng.standard_normal((32, code.N)) * 1.5 + 1.0).astype(np.float32)
    b, it, ok, s = oracle.decode_f32(g, r, 15)
    flip = (1 - 2 * cw.astype(np.int8)).astype(np.float32)
    b2, it2, ok2, s2 = oracle.decode_f32(g, r * flip, 15)
    assert (it2 == it).all() and (ok2 == ok).all()
    assert (b2 == (b ^ cw)).all()
    assert (s2 == s * flip).all()


def test_fixed_equals_float_on_integer_inputs_without_saturation():
    code = small_qc()
    g = oracle.Graph.from_code(code)
    rng = np.random.default_rng(12)
    q = rng.integers(-12, 13, size=(32, code.N)).astype(np.int8)
    b1, it1, ok1, s1 = oracle.decode_fixed(g, q, 8)
    b2, it2, ok2, s2 = oracle.decode_f32(g, q.astype(np.float32), 8)
    assert (np.abs(s1) < oracle.SAT).all()
    assert (b1 == b2).all() and (it1 == it2).all() and (ok1 == ok2).all()
    assert (s1.astype(np.float32) == s2).all()


def test_fixed_point_saturates_and_never_wraps():
    # a few bits shared by many short checks, all LLRs at the +-127 limit: messages grow
    # until they hit the saturation limit within a few iterations
    rng = np.random.default_rng(1)
    n_bits = 8
    sets = [sorted(rng.choice(n_bits, size=int(rng.integers(2, 4)), replace=False) + 1)
            for _ in range(64)]
    code = inputs.code_from_index_sets(sets, n_bits)
    assert code.col_weights().max() >= 16
    g = oracle.Graph.from_code(code)
    L = 8
    seen_wide_lambda = False
    for trial in range(20):
        q = rng.choice([-127, 127], size=code.N).astype(np.int8)
        _, _, _, eta, s = oracle.trace_fixed(g, q, L)
        assert np.abs(eta.astype(np.int64)).max() <= oracle.SAT
        assert np.abs(s.astype(np.int64)).max() <= oracle.SAT
        assert np.abs(s.astype(np.int64)).max() == oracle.SAT  # the limit is reached
        for k in range(L):
            # s_j = clamp(q_j + sum of incoming eta), the sum taken wide (no wrap-around)
            wide = q.astype(np.int64).copy()
            np.add.at(wide, code.cols, eta[k].astype(np.int64))
            assert (np.clip(wide, -oracle.SAT, oracle.SAT) == s[k]).all()
            if k:
                lam_wide = s[k - 1].astype(np.int64)[code.cols] - eta[k - 1].astype(np.int64)
                seen_wide_lambda |= bool((np.abs(lam_wide) > oracle.SAT).any())
    assert seen_wide_lambda  # the lambda saturation point is exercised too


def test_paper_slicer_complements_bits_on_even_weight_rows():
    code, _, _ = tanner()
    g = oracle.Graph.from_code(code)
    rng = np.random.default_rng(31)
    r = (rng.standard_normal((64, 10)) * 2 + 1.0).astype(np.float32)
    b, it, _, _ = oracle.decode_f32(g, r, 10)
    b2, it2, _, _ = oracle.decode_f32(g, r, 10, flags=oracle.PAPER_SLICER)
    assert (it == it2).all()
    assert (b2 == 1 - b).all()


def test_quantizer_closed_form_table():
    x = np.array([0.0, -0.0, 0.125, 0.375, -0.125, -0.375, 0.25, 31.75, 31.875, 40.0, -40.0,
                  np.inf, -np.inf, 1.1, -2.6], np.float32)
    # q = clamp(round_half_even(4x), -127, 127): 4x = 0.5 -> 0, 1.5 -> 2, 127.5 -> 127
    expect = [0, 0, 0, 2, 0, -2, 1, 127, 127, 127, -127, 127, -127, 4, -10]
    assert oracle.quantize(x).tolist() == expect


def test_rejects_rows_of_weight_one():
    with pytest.raises(ValueError):
        oracle.Graph(2, 3, dense=np.array([[1, 1, 0], [0, 0, 1]], np.uint8))
    with pytest.raises(ValueError):
        oracle.Graph(1, 2, dense=np.array([[2, 1]], np.uint8))
    oracle.Graph(2, 3, dense=np.array([[1, 1, 0], [0, 0, 0]], np.uint8))  # weight 0 is fine


def test_check_every_cadence():
    code = small_qc()
    g = oracle.Graph.from_code(code)
    rng = np.random.default_rng(14)
    r = (rng.standard_normal((64, code.N)) * 1.2 + 1.0).astype(np.float32)
    _, it1, _, _ = oracle.decode_f32(g, r, 30, check_every=1)
    _, it3, ok3, _ = oracle.decode_f32(g, r, 30, check_every=3)
    for a, c, ok in zip(it1, it3, ok3):
        if a == 0:
            assert c == 0
        elif ok:
            assert c % 3 == 0 or c == 30
            assert c >= a


def test_threads_do_not_change_results():
    code = small_qc()
    g = oracle.Graph.from_code(code)
    r = np.random.default_rng(15).standard_normal((37, code.N)).astype(np.float32) + 0.6
    a = oracle.decode_f32(g, r, 10, threads=1)
    b = oracle.decode_f32(g, r, 10, threads=5)
    for x, y in zip(a, b):
        assert (x == y).all()

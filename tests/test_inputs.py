"""Seeded input generators: code structure, encoder and channel statistics (CPU)."""
import numpy as np

from paper_2507_10424_gb300 import inputs


def no_duplicate_edges(code):
    key = code.rows.astype(np.int64) * code.N + code.cols
    return np.unique(key).size == key.size


def test_regular_code_degrees():
    c = inputs.cfg_regular_576()
    assert (c.M, c.N, c.E) == (288, 576, 1728)
    assert (c.row_weights() == 6).all() and (c.col_weights() == 3).all()
    assert no_duplicate_edges(c)
    c2 = inputs.cfg_regular_576()
    assert (c.cols == c2.cols).all()  # seeded


def test_qc_code_structure():
    base = inputs.qc_base_matrix(12, 24, 96, 0.5, 2)
    c = inputs.cfg_qc_2304()
    assert (c.M, c.N) == (1152, 2304)
    assert c.E == 96 * int((base >= 0).sum())
    assert ((base >= 0).sum(axis=1) >= 2).all() and ((base >= 0).sum(axis=0) >= 2).all()
    H = c.dense()
    for r in range(12):
        for col in range(24):
            blk = H[r * 96:(r + 1) * 96, col * 96:(col + 1) * 96]
            if base[r, col] < 0:
                assert blk.sum() == 0
            else:
                assert (blk == np.roll(np.eye(96, dtype=np.uint8), base[r, col], axis=1)).all()


def test_paper_shaped_code_structure():
    c = inputs.cfg_paper_shaped()
    assert (c.M, c.N, c.E) == (1022, 8176, 32704)
    assert (c.row_weights() == 32).all() and (c.col_weights() == 4).all()
    assert no_duplicate_edges(c)
    # block (r, b) of the 2x16 base holds exactly two ones in every row and column
    H = c.dense().astype(np.int64)
    for r in range(2):
        for b in range(16):
            blk = H[r * 511:(r + 1) * 511, b * 511:(b + 1) * 511]
            assert (blk.sum(axis=0) == 2).all() and (blk.sum(axis=1) == 2).all()
    cw = inputs.Encoder(c).random_codewords(8, 3)
    assert not ((H @ cw.T.astype(np.int64)) % 2).any()


def test_irregular_code_degree_counts():
    c = inputs.cfg_irregular_64800()
    assert (c.M, c.N, c.E) == (32400, 64800, 202500)
    cw = np.bincount(c.col_weights())
    assert cw[2] == 32400 and cw[3] == 24300 and cw[8] == 8100
    rw = np.bincount(c.row_weights())
    assert rw[6] == 24300 and rw[7] == 8100
    assert no_duplicate_edges(c)


def test_encoder_gives_codewords():
    c = inputs.cfg_qc_2304()
    enc = inputs.Encoder(c)
    cw = enc.random_codewords(256, 3)
    H = c.dense().astype(np.int64)
    assert ((cw.astype(np.int64) @ H.T) % 2 == 0).all()
    assert enc.rank + enc.K == c.N
    assert 0.4 < cw.mean() < 0.6


def test_channel_llr_statistics():
    F, N = 512, 576
    llr = inputs.all_zero_awgn_llr(F, N, 2.5, 0.5, 9)
    s2 = inputs.noise_sigma2(2.5, 0.5)
    assert llr.dtype == np.float32
    # LLR = 2y/sigma^2 with y ~ N(1, sigma^2): mean 2/sigma^2, variance 4/sigma^2
    assert abs(llr.mean() - 2 / s2) < 0.02 * (2 / s2)
    assert abs(llr.var() - 4 / s2) < 0.03 * (4 / s2)
    cw = np.zeros((4, 8), np.uint8)
    cw[:, 3] = 1
    l2 = inputs.bpsk_awgn_llr(cw, 30.0, 0.5, 1)
    assert (l2[:, 3] < 0).all() and (np.delete(l2, 3, axis=1) > 0).all()

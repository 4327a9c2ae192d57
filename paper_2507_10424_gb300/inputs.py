"""Seeded synthetic inputs for Min-Sum decoding: parity matrices, codewords, channel LLRs.

This module is shared by the CUDA path's tests and benchmark and by the CPU oracle's
tests. It holds none of the decoder's arithmetic: no check/variable updates, no hard
decision, no syndrome and no LLR quantisation. It only draws codes and channel outputs.

Code constructions (the paper benchmarks a quasi-cyclic code, Section VI, whose parity
matrix is not available here; these seeded constructions stand in for it):

* ``regular_code``   -- (dv, dc)-regular code by socket permutation with double-edge repair.
* ``qc_code``        -- quasi-cyclic code: a random base matrix of circulant shifts.
* ``irregular_code`` -- column weights drawn to exact counts from a degree distribution,
                        row weights as equal as possible, socket permutation + repair.
* ``tree_code``      -- a random cycle-free Tanner graph (used for exactness pins).
* ``code_from_index_sets`` -- a code given by its check index sets (Section II-A).

Channel (Section VI: AWGN added to a BPSK-modulated codeword): bit 0 -> +1, bit 1 -> -1,
``sigma^2 = 1 / (2 R 10^(EbN0/10))`` with R the design rate ``1 - M/N``, and
``LLR = 2 y / sigma^2`` so that a positive LLR favours bit 0.
"""
from __future__ import annotations

import dataclasses
import numpy as np


@dataclasses.dataclass
class Code:
    """A binary LDPC code as an edge list (one edge per nonzero of H).

    ``rows[e], cols[e]`` are sorted by (row, col). ``M`` checks, ``N`` bits.
    """

    M: int
    N: int
    rows: np.ndarray  # int32 [E]
    cols: np.ndarray  # int32 [E]
    name: str = ""

    @property
    def E(self) -> int:
        return int(self.rows.shape[0])

    @property
    def design_rate(self) -> float:
        return 1.0 - self.M / self.N

    def dense(self) -> np.ndarray:
        """Dense 0/1 parity matrix, uint8 [M][N] row-major."""
        H = np.zeros((self.M, self.N), dtype=np.uint8)
        H[self.rows, self.cols] = 1
        return H

    def csr(self):
        """(row_ptr int64 [M+1], col_idx int32 [E]) with ascending columns per row."""
        row_ptr = np.zeros(self.M + 1, dtype=np.int64)
        np.add.at(row_ptr, self.rows.astype(np.int64) + 1, 1)
        return np.cumsum(row_ptr), self.cols.astype(np.int32).copy()

    def row_weights(self) -> np.ndarray:
        return np.bincount(self.rows, minlength=self.M)

    def col_weights(self) -> np.ndarray:
        return np.bincount(self.cols, minlength=self.N)

    def packed_rows(self) -> np.ndarray:
        """Bit-packed rows: uint32 [M][ceil(N/32)], bit (j % 32) of word j // 32 is H[i, j]."""
        W = (self.N + 31) // 32
        out = np.zeros((self.M, W), dtype=np.uint32)
        np.bitwise_or.at(out, (self.rows, self.cols // 32),
                         (np.uint32(1) << (self.cols % 32).astype(np.uint32)))
        return out


def _make_code(M: int, N: int, rows, cols, name: str) -> Code:
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    order = np.lexsort((cols, rows))
    return Code(M, N, rows[order].astype(np.int32), cols[order].astype(np.int32), name)


def _repair_double_edges(check_sockets: np.ndarray, var_sockets: np.ndarray, N: int,
                         rng: np.random.Generator, max_rounds: int = 10000) -> np.ndarray:
    """Swap variable sockets until no (check, variable) pair occurs twice."""
    var_sockets = var_sockets.copy()
    E = var_sockets.shape[0]
    for _ in range(max_rounds):
        key = check_sockets.astype(np.int64) * N + var_sockets
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup = np.nonzero(ks[1:] == ks[:-1])[0]
        if dup.size == 0:
            return var_sockets
        bad = order[dup + 1]
        partners = rng.integers(0, E, size=bad.size)
        for a, b in zip(bad, partners):
            var_sockets[a], var_sockets[b] = var_sockets[b], var_sockets[a]
    raise RuntimeError("double-edge repair did not converge")


def _socket_code(col_deg: np.ndarray, row_deg: np.ndarray, rng: np.random.Generator,
                 name: str) -> Code:
    M, N = row_deg.shape[0], col_deg.shape[0]
    assert col_deg.sum() == row_deg.sum()
    check_sockets = np.repeat(np.arange(M, dtype=np.int64), row_deg)
    var_sockets = np.repeat(np.arange(N, dtype=np.int64), col_deg)
    var_sockets = var_sockets[rng.permutation(var_sockets.shape[0])]
    var_sockets = _repair_double_edges(check_sockets, var_sockets, N, rng)
    return _make_code(M, N, check_sockets, var_sockets, name)


def regular_code(N: int, M: int, dv: int, dc: int, seed: int) -> Code:
    """(dv, dc)-regular code, seeded socket permutation with double-edge repair."""
    if N * dv != M * dc:
        raise ValueError("N*dv must equal M*dc")
    rng = np.random.default_rng(seed)
    return _socket_code(np.full(N, dv, np.int64), np.full(M, dc, np.int64), rng,
                        f"regular({dv},{dc}) N={N} M={M} seed={seed}")


def irregular_code(N: int, M: int, col_weights, fractions, seed: int) -> Code:
    """Irregular code with exact column-weight counts and near-equal row weights."""
    rng = np.random.default_rng(seed)
    col_weights = np.asarray(col_weights, dtype=np.int64)
    counts = np.floor(np.asarray(fractions, dtype=np.float64) * N + 0.5).astype(np.int64)
    counts[-1] = N - counts[:-1].sum()
    col_deg = np.repeat(col_weights, counts)
    col_deg = col_deg[rng.permutation(N)]
    E = int(col_deg.sum())
    row_deg = np.full(M, E // M, np.int64)
    row_deg[: E % M] += 1
    row_deg = row_deg[rng.permutation(M)]
    return _socket_code(col_deg, row_deg, rng, f"irregular N={N} M={M} seed={seed}")


def qc_base_matrix(mb: int, nb: int, Z: int, p: float, seed: int) -> np.ndarray:
    """Base matrix of circulant shifts (-1 = zero block), >= 2 nonzeros per base row/column."""
    rng = np.random.default_rng(seed)
    while True:
        mask = rng.random((mb, nb)) < p
        if (mask.sum(axis=1) >= 2).all() and (mask.sum(axis=0) >= 2).all():
            break
    shifts = rng.integers(0, Z, size=(mb, nb))
    return np.where(mask, shifts, -1)


def qc_code(mb: int, nb: int, Z: int, p: float, seed: int) -> Code:
    """Quasi-cyclic code: block (r, c) with shift s maps row r*Z+z to column c*Z+(z+s)%Z."""
    base = qc_base_matrix(mb, nb, Z, p, seed)
    rows, cols = [], []
    z = np.arange(Z)
    for r in range(mb):
        for c in range(nb):
            s = base[r, c]
            if s >= 0:
                rows.append(r * Z + z)
                cols.append(c * Z + (z + s) % Z)
    return _make_code(mb * Z, nb * Z, np.concatenate(rows), np.concatenate(cols),
                      f"qc {mb}x{nb} Z={Z} p={p} seed={seed}")


def tree_code(n_checks: int, seed: int, max_new: int = 3) -> Code:
    """Random cycle-free Tanner graph: each new check joins one existing bit and new bits."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    first = int(rng.integers(2, max_new + 2))
    n_bits = first
    rows += [0] * first
    cols += list(range(first))
    for i in range(1, n_checks):
        anchor = int(rng.integers(0, n_bits))
        k = int(rng.integers(1, max_new + 1))
        rows += [i] * (k + 1)
        cols += [anchor] + list(range(n_bits, n_bits + k))
        n_bits += k
    return _make_code(n_checks, n_bits, rows, cols, f"tree m={n_checks} seed={seed}")


def code_from_index_sets(index_sets, N: int, one_based: bool = True, name: str = "") -> Code:
    rows, cols = [], []
    for i, s in enumerate(index_sets):
        for j in s:
            rows.append(i)
            cols.append(j - 1 if one_based else j)
    return _make_code(len(index_sets), N, rows, cols, name)


class Encoder:
    """GF(2) encoder from the reduced row-echelon form of H (Gaussian elimination).

    Information bits sit on the non-pivot columns; each pivot column's bit is the parity
    of the RREF row's support on the non-pivot columns.
    """

    def __init__(self, code: Code):
        H = code.dense().astype(np.uint8)
        M, N = H.shape
        W = (N + 63) // 64
        pad = np.zeros((M, W * 64), dtype=np.uint8)
        pad[:, :N] = H
        A = np.packbits(pad, axis=1, bitorder="little").view(np.uint64).copy()
        pivots = []
        r = 0
        for c in range(N):
            if r == M:
                break
            w, b = divmod(c, 64)
            colbits = (A[r:, w] >> np.uint64(b)) & np.uint64(1)
            nz = np.nonzero(colbits)[0]
            if nz.size == 0:
                continue
            p = r + int(nz[0])
            if p != r:
                A[[r, p]] = A[[p, r]]
            hit = ((A[:, w] >> np.uint64(b)) & np.uint64(1)).astype(bool)
            hit[r] = False
            A[hit] ^= A[r]
            pivots.append(c)
            r += 1
        self.N = N
        self.rank = r
        self.pivots = np.array(pivots, dtype=np.int64)
        free = np.ones(N, dtype=bool)
        free[self.pivots] = False
        self.free = np.nonzero(free)[0]
        R = np.unpackbits(A[:r].view(np.uint8), axis=1, bitorder="little")[:, :N]
        self.P = R[:, self.free].astype(np.float32)  # [rank][K]
        self.K = self.free.shape[0]

    def encode(self, info: np.ndarray) -> np.ndarray:
        """info uint8 [F][K] -> codewords uint8 [F][N]."""
        info = np.asarray(info, dtype=np.uint8)
        F = info.shape[0]
        c = np.zeros((F, self.N), dtype=np.uint8)
        c[:, self.free] = info
        par = (info.astype(np.float32) @ self.P.T)  # exact integer sums < 2^24
        c[:, self.pivots] = (par.astype(np.int64) & 1).astype(np.uint8)
        return c

    def random_codewords(self, F: int, seed: int) -> np.ndarray:
        rng = np.random.default_rng(seed)
        info = rng.integers(0, 2, size=(F, self.K), dtype=np.uint8)
        return self.encode(info)


def noise_sigma2(ebn0_db: float, rate: float) -> float:
    return 1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0))


def bpsk_awgn_llr(codewords: np.ndarray, ebn0_db: float, rate: float, seed: int) -> np.ndarray:
    """Channel LLRs (float32 [F][N]) for BPSK (0 -> +1, 1 -> -1) over AWGN at Eb/N0."""
    codewords = np.asarray(codewords)
    sigma2 = noise_sigma2(ebn0_db, rate)
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(size=codewords.shape, dtype=np.float32)
    x = 1.0 - 2.0 * codewords.astype(np.float32)
    y = x + np.float32(np.sqrt(sigma2)) * noise
    return (np.float32(2.0 / sigma2) * y).astype(np.float32)


def all_zero_awgn_llr(F: int, N: int, ebn0_db: float, rate: float, seed: int) -> np.ndarray:
    """LLRs of the all-zero codeword over AWGN (the paper's measurement set-up)."""
    sigma2 = noise_sigma2(ebn0_db, rate)
    rng = np.random.default_rng(seed)
    y = np.float32(np.sqrt(sigma2)) * rng.standard_normal(size=(F, N), dtype=np.float32)
    y += np.float32(1.0)
    return (np.float32(2.0 / sigma2) * y).astype(np.float32)


# Named workloads (sizes and seeds of the benchmark and parity configurations).
def cfg_regular_576(seed: int = 1) -> Code:
    """(3,6)-regular, N=576, M=288 (socket permutation)."""
    return regular_code(576, 288, 3, 6, seed)


def cfg_qc_2304(seed: int = 2) -> Code:
    """Quasi-cyclic 12x24 base, p=0.5, Z=96: N=2304, M=1152."""
    return qc_code(12, 24, 96, 0.5, seed)


def cfg_irregular_64800(seed: int = 5) -> Code:
    """Irregular N=64800, M=32400, column weights {2,3,8} at 0.5/0.375/0.125."""
    return irregular_code(64800, 32400, [2, 3, 8], [0.5, 0.375, 0.125], seed)


def cfg_paper_shaped(seed: int = 4) -> Code:
    """Stand-in with the dimensions of the paper's code (N=8176, M=1022), whose matrix is
    not available: a 2x16 base of 511x511 blocks, each block the sum of two circulant
    permutations with distinct seeded shifts, so every column has weight 4 and every row
    weight 32 (E=32704)."""
    rng = np.random.default_rng(seed)
    mb, nb, Z = 2, 16, 511
    rows, cols = [], []
    z = np.arange(Z)
    for r in range(mb):
        for c in range(nb):
            for sh in rng.choice(Z, size=2, replace=False):
                rows.append(r * Z + z)
                cols.append(c * Z + (z + int(sh)) % Z)
    return _make_code(mb * Z, nb * Z, np.concatenate(rows), np.concatenate(cols),
                      f"paper-shaped 2x16 Z=511 weight-2 circulants seed={seed}")


MIXED_N = (256, 512, 1024, 2048, 4096, 8192, 12288, 16200)
MIXED_RATES = (1 / 2, 2 / 3, 3 / 4, 5 / 6)


def cfg_mixed_codes(seed: int = 3):
    """Eight irregular codes: column weights {2,3,4,8} at 0.3/0.4/0.2/0.1, N from MIXED_N,
    rate of code k = MIXED_RATES[k % 4], M = round(N (1 - rate)); frames per code drawn
    uniformly from [64, 8192]. Returns (codes, frames)."""
    rng = np.random.default_rng(seed)
    codes, frames = [], []
    for k, N in enumerate(MIXED_N):
        R = MIXED_RATES[k % 4]
        M = int(round(N * (1 - R)))
        codes.append(irregular_code(N, M, [2, 3, 4, 8], [0.3, 0.4, 0.2, 0.1], seed * 100 + k))
        frames.append(int(rng.integers(64, 8193)))
    return codes, frames

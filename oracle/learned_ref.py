"""Reference of the unrolled normalised/offset Min-Sum in plain PyTorch -- TEST
INFRASTRUCTURE ONLY (small codes, CPU, float64).

Forward: T flooding iterations without early stop. Iteration t (1-based) forms
lambda_e = s_j - eta_e^(t-1) for every edge of a check, the extrinsic magnitude
m_e = min over the check's other edges of |lambda| and the extrinsic sign (product of the
other edges' signs, sign(0) = +1), then eta_e = sign * max(alpha[t, c] m_e - beta[t, c], 0)
with c the class of the edge's bit, and s_j = r_j + sum of eta over the checks of bit j
(eq. eta_update and eq. lambda_j of the paper, with the learned weights applied to the
magnitude). Gradients come from torch.autograd: through the minimum they follow the edge
that attains it (ties are avoided by the tests), through max(., 0) the active side.
"""
from __future__ import annotations

import torch


def unrolled_posteriors(rows, N, col_class, r, alpha, beta):
    """rows: list of column-index lists (one per check); r: [F][N] float64 tensor;
    alpha, beta: [T][C] tensors (may require grad). Returns s^T: [F][N]."""
    T = alpha.shape[0]
    F = r.shape[0]
    col_class = torch.as_tensor(col_class, dtype=torch.long)
    s = r
    eta = [torch.zeros(F, len(cols), dtype=r.dtype) for cols in rows]
    for t in range(T):
        new_eta = []
        for i, cols in enumerate(rows):
            d = len(cols)
            if d == 0:
                new_eta.append(eta[i])
                continue
            idx = torch.as_tensor(cols, dtype=torch.long)
            lam = s[:, idx] - eta[i]
            mag = lam.abs()
            sgn = torch.where(lam < 0, -torch.ones_like(lam), torch.ones_like(lam))
            out = []
            for k in range(d):
                others = [j for j in range(d) if j != k]
                m = mag[:, others].min(dim=1).values
                ext = sgn[:, others].prod(dim=1)
                c = col_class[cols[k]]
                a = torch.relu(alpha[t, c] * m - beta[t, c])
                out.append(ext * a)
            new_eta.append(torch.stack(out, dim=1))
        eta = new_eta
        s = r.clone()
        for i, cols in enumerate(rows):
            if len(cols):
                s = s.index_add(1, torch.as_tensor(cols, dtype=torch.long), eta[i])
    return s


def bce_loss(s, codewords):
    """Binary cross-entropy of P(bit = 1) = sigmoid(-s) against the sent bits, summed."""
    return torch.nn.functional.binary_cross_entropy_with_logits(-s, codewords.to(s.dtype),
                                                                reduction="sum")

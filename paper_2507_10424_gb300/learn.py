"""Learned normalised / offset Min-Sum: training and evaluation on the GPU.

The decoder's check update gets per-iteration, per-class weights: every extrinsic
magnitude m becomes max(alpha[t][c] m - beta[t][c], 0), c the class (column weight) of the
edge's bit; alpha = 1, beta = 0 is plain Min-Sum. The weights are trained by binary
cross-entropy of the final posteriors (P(bit = 1) = sigmoid(-s)) on frames generated here:
random codewords, BPSK over AWGN, Eb/N0 drawn per frame from a range.

Every decoding step (forward and adjoint) runs in libldpc.so through
``ldpc_train_forward`` / ``ldpc_train_backward``; this module only allocates the tensors,
calls them through :class:`WeightedMinSum` (a ``torch.autograd.Function``) and runs the
optimiser.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import ldpc as _ldpc


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class WeightedMinSum:
    """``apply(dec, llr, alpha, beta, every=False) -> soft``: T = alpha.shape[0] unrolled
    iterations; soft is [F][N] after the last one, or [T][F][N] after each (every=True)."""

    _fn = None

    @classmethod
    def apply(cls, dec, llr, alpha, beta, every=False):
        if cls._fn is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, llr, alpha, beta, dec, every):
                    F, N = llr.shape
                    T = alpha.shape[0]
                    lib = _ldpc.load()
                    nbytes = _ldpc.ldpc_train_workspace_size(dec.h, F, T)
                    work = torch.empty(nbytes, dtype=torch.uint8, device=llr.device)
                    shape = (T, F, N) if every else (F, N)
                    soft = torch.empty(shape, dtype=torch.float32, device=llr.device)
                    a = alpha.detach().contiguous()
                    b = beta.detach().contiguous()
                    _ldpc._check(lib.ldpc_set_stream(dec.h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
                                 "ldpc_set_stream")
                    _ldpc._check(lib.ldpc_train_forward(dec.h, _ptr(llr), F, T, _ptr(a), _ptr(b), _ptr(soft),
                                                        int(every), _ptr(work), nbytes), "ldpc_train_forward")
                    ctx.dec, ctx.work, ctx.nbytes, ctx.F, ctx.T = dec, work, nbytes, F, T
                    ctx.every = int(every)
                    ctx.save_for_backward(a, b)
                    return soft

                @staticmethod
                def backward(ctx, grad_soft):
                    a, b = ctx.saved_tensors
                    ga = torch.empty_like(a)
                    gb = torch.empty_like(b)
                    g = grad_soft.contiguous().float()
                    lib = _ldpc.load()
                    _ldpc._check(lib.ldpc_train_backward(ctx.dec.h, ctx.F, ctx.T, _ptr(a), _ptr(b), _ptr(g),
                                                         ctx.every, _ptr(ga), _ptr(gb), _ptr(ctx.work),
                                                         ctx.nbytes), "ldpc_train_backward")
                    return None, ga, gb, None, None

            cls._fn = _F
        return cls._fn.apply(llr.contiguous(), alpha, beta, dec, bool(every))


class FrameSource:
    """Random codewords of a code, BPSK over AWGN, on the GPU (seeded).

    encode=False sends the all-zero codeword instead (for codes too large for the GF(2)
    encoder): Min-Sum, normalised or offset, is symmetric under BPSK over AWGN, so its
    error rates and the expected loss do not depend on the codeword sent.
    """

    def __init__(self, code, device="cuda", seed=0, encode=True):
        import torch
        from . import inputs
        self.N, self.rate = code.N, code.design_rate
        self.encode = encode
        if encode:
            enc = inputs.Encoder(code)
            self.K = enc.K
            self.P = torch.from_numpy(enc.P).to(device)                 # [rank][K]
            self.free = torch.from_numpy(enc.free).to(device)
            self.pivots = torch.from_numpy(enc.pivots).to(device)
        self.device = device
        self.gen = torch.Generator(device=device)
        self.gen.manual_seed(seed)

    def batch(self, F, ebn0_db):
        """ebn0_db: a float, or (lo, hi) for a per-frame uniform draw. Returns (llr, bits)."""
        import torch
        c = torch.zeros((F, self.N), device=self.device)
        if self.encode:
            info = torch.randint(0, 2, (F, self.K), generator=self.gen, device=self.device,
                                 dtype=torch.float32)
            c[:, self.free] = info
            c[:, self.pivots] = torch.remainder(info @ self.P.T, 2.0)
        if isinstance(ebn0_db, tuple):
            e = torch.rand((F, 1), generator=self.gen, device=self.device) * (ebn0_db[1] - ebn0_db[0]) + ebn0_db[0]
        else:
            e = torch.full((F, 1), float(ebn0_db), device=self.device)
        sigma2 = 1.0 / (2.0 * self.rate * torch.pow(10.0, e / 10.0))
        y = (1.0 - 2.0 * c) + torch.sqrt(sigma2) * torch.randn((F, self.N), generator=self.gen,
                                                                device=self.device)
        return (2.0 * y / sigma2).contiguous(), c.to(torch.uint8)


def train_weights(dec, code, iters=10, steps=300, batch=4096, ebn0=(1.0, 4.0), lr=0.02,
                  seed=1, log_every=0, every=True, encode=True):
    """Train alpha, beta [iters][n_classes] from plain Min-Sum (alpha = 1, beta = 0).

    every=True: the loss is the mean over iterations of the cross-entropy of that
    iteration's posteriors (rewards early convergence); else the last iteration only.
    Returns (alpha, beta, losses) as numpy arrays / list.
    """
    import torch
    C = len(dec.classes())
    alpha = torch.ones((iters, C), device="cuda", requires_grad=True)
    beta = torch.zeros((iters, C), device="cuda", requires_grad=True)
    opt = torch.optim.Adam([alpha, beta], lr=lr)
    src = FrameSource(code, seed=seed, encode=encode)
    losses = []
    for step in range(steps):
        llr, bits = src.batch(batch, ebn0)
        soft = WeightedMinSum.apply(dec, llr, alpha, beta, every)
        # binary cross-entropy of the logits z = -s of P(bit = 1): the mean of softplus(z) -
        # t z, whose gradient w.r.t. s is -(sigmoid(z) - t) / n. Both are formed here one
        # iteration's posteriors at a time, so that a large batch needs no temporaries the
        # size of all T x F x N posteriors beyond the gradient itself.
        opt.zero_grad()
        with torch.no_grad():
            t = bits.float()
            n = soft.numel()
            grad = torch.empty_like(soft)
            total = 0.0
            for k in range(soft.shape[0] if every else 1):
                z = -(soft[k] if every else soft)
                total += float((torch.nn.functional.softplus(z) - t * z).sum().item())
                g = grad[k] if every else grad
                torch.sigmoid(z, out=g)
                g.sub_(t).mul_(-1.0 / n)
                del z
        soft.backward(grad)
        del grad, soft
        opt.step()
        losses.append(total / n)
        if log_every and step % log_every == 0:
            print(f"step {step} loss {losses[-1]:.5f}")
    return alpha.detach().cpu().numpy(), beta.detach().cpu().numpy(), losses


def frame_error_rate(dec, llr, bits, max_iter, weights=None):
    """FER with early stop; weights = (alpha, beta) or None for plain Min-Sum."""
    import torch
    if weights is None:
        dec.set_weights(None)
    else:
        dec.set_weights(*weights)
    out, iters, _, _ = dec.decode(llr, max_iter, early_stop=True)
    fer = float((out != bits).any(dim=1).float().mean().item())
    mean_it = float(iters.float().mean().item())
    dec.set_weights(None)
    return fer, mean_it


def compare(dec, code, weights, ebn0_points=(2.0, 2.5, 3.0), frames=20000,
            iters=(5, 6, 7, 8, 9, 10, 11, 12, 14, 16, 20), seed=7, encode=True):
    """FER and mean iterations of plain and learned Min-Sum at several iteration limits."""
    src = FrameSource(code, seed=seed, encode=encode)
    rows = []
    for e in ebn0_points:
        llr, bits = src.batch(frames, float(e))
        for L in iters:
            fp, ip = frame_error_rate(dec, llr, bits, L)
            fl, il = frame_error_rate(dec, llr, bits, L, weights)
            rows.append({"ebn0_db": e, "max_iter": L, "fer_plain": fp, "fer_learned": fl,
                         "mean_iter_plain": ip, "mean_iter_learned": il})
    return rows


def iterations_to_match(rows, ebn0_db, plain_iters):
    """Smallest listed iteration limit at which the learned decoder's FER is at most the
    plain decoder's FER at `plain_iters` (None if none)."""
    target = [r["fer_plain"] for r in rows if r["ebn0_db"] == ebn0_db and r["max_iter"] == plain_iters][0]
    cands = sorted((r["max_iter"], r["fer_learned"]) for r in rows if r["ebn0_db"] == ebn0_db)
    for L, f in cands:
        if f <= target:
            return L
    return None

#!/usr/bin/env python3
"""Throughput benchmark of flooding Min-Sum decoding on one or more GB300s.

Workload (one "step" = one pass of the whole decoding path over one batch): the
quasi-cyclic code with a 12 x 24 base matrix of seeded shifts (about half nonzero) and
circulant size Z = 96 (N = 2304, M = 1152), 65536 random codewords (uniform information
bits encoded through Gaussian elimination on H), BPSK over AWGN with the frames split over
Eb/N0 = 1.0, 1.5, 2.0, 2.5, 3.0 dB, decoded with 10 flooding iterations and no early stop.
Throughput is codeword bits decoded per second (frames x N / time), the paper's definition
(Section VI). Inputs are synthetic and seeded; the paper's own code (the CCSDS (8176, 1022)
quasi-cyclic code) is not available, so this code stands in for it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank decodes its own batch (frames are independent: weak
scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "decoded Gbit/s at fixed iters; HBM GB/s vs peak; learned vs plain iters@FER"
SNRS = [1.0, 1.5, 2.0, 2.5, 3.0]
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["fp32", "fixed"], default="fp32")
    ap.add_argument("--frames", type=int, default=65536)
    ap.add_argument("--iters", type=int, default=10)
    ap.add_argument("--variant", choices=["auto", "resident", "stream"], default="auto")
    ap.add_argument("--tuning", default="auto",
                    help="launch shape instead of the autotuner: resident 'FT,threads[,index "
                         "placement]'; streaming 'warps per CTA,stages[,frames per lane]'")
    ap.add_argument("--quick", action="store_true", help="skip the extra measurements")
    ap.add_argument("--part", choices=sorted(PARTS), default=None,
                    help="run one of the extra measurements alone and print its record (for "
                         "profiling it); no headline step")
    ap.add_argument("--workload", choices=["qc2304", "irregular64800"], default="qc2304",
                    help="qc2304: the headline batch; irregular64800: the large irregular code "
                         "(all-zero codeword at Eb/N0 1.0 dB, decoded by the streaming kernels)")
    return ap.parse_args()


# ------------------------------------------------------------------ workload

def make_code(workload="qc2304"):
    from paper_2507_10424_gb300 import inputs
    return inputs.cfg_irregular_64800() if workload == "irregular64800" else inputs.cfg_qc_2304()


def make_llr(code, F, seed, workload="qc2304"):
    from paper_2507_10424_gb300 import inputs
    if workload == "irregular64800":  # all-zero codeword (the encoder of this code is impractical)
        llr = inputs.all_zero_awgn_llr(F, code.N, 1.0, code.design_rate, seed)
        return np.zeros((F, code.N), np.uint8), llr, np.array([0, F])
    enc = inputs.Encoder(code)
    cw = enc.random_codewords(F, seed)
    llr = np.empty((F, code.N), np.float32)
    bounds = np.linspace(0, F, len(SNRS) + 1).astype(int)
    for k, e in enumerate(SNRS):
        a, b = bounds[k], bounds[k + 1]
        llr[a:b] = inputs.bpsk_awgn_llr(cw[a:b], e, code.design_rate, seed * 10 + k)
    return cw, llr, bounds


def edge_message_bytes(code, mode):
    """Algorithmic bytes per frame per iteration: each edge message read and written once,
    the channel value read once and the posterior read and written once."""
    m, br, bs = (4, 4, 4) if mode == "fp32" else (2, 1, 2)
    return 2 * code.E * m + code.N * (br + 2 * bs)


def workload_name(code, F, L, workload="qc2304"):
    if workload == "irregular64800":
        return (f"irregular, column weights 2/3/8: N={code.N} M={code.M} E={code.E}; {F} all-zero "
                f"codewords, Eb/N0 1.0 dB; {L} flooding iterations, no early stop")
    return (f"QC 12x24 base, Z=96: N={code.N} M={code.M} E={code.E}; {F} random codewords, "
            f"Eb/N0 1.0-3.0 dB step 0.5; {L} flooding iterations, no early stop")


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.file = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.dev).uuid)
            sel = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        except Exception:
            sel = str(self.dev)
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", sel, f"--query-gpu=timestamp,{self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = open(self.file.name).read().strip().splitlines()
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        for r in rows:
            p = [x.strip() for x in r.split(",")]
            if len(p) < 9:
                continue
            try:
                ts = time.mktime(time.strptime(p[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
            except Exception:
                ts = None
            if ts is not None and self.t0 is not None and not (self.t0 - 1 <= ts <= self.t1 + 1):
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                "sw_power_cap"), p[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers

def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


KERNEL_SOURCES = {"k_resident": "resident.cuh"}
NOMINAL_HBM_GBS = 8000.0  # nominal HBM3e bandwidth of the GPU


def kernel_source_hash(kernel):
    """Hash of the file holding a kernel's device code (the traffic record goes stale with it)."""
    with open(os.path.join(ROOT, "paper_2507_10424_gb300", "csrc", KERNEL_SOURCES[kernel]), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def ncu_traffic(kernel, mode, F):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, scaled to F frames,
    or None when the kernel sources changed since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            t = json.load(fh)
    except Exception:
        return None
    e = t.get(f"{kernel}:{mode}")
    if not e or e.get("source_hash") != kernel_source_hash(kernel):
        return None
    return e["dram_bytes_per_launch"] * F / e["frames"]


def ncu_counters(kernel, mode):
    """Per-unit counters of `kernel` from the committed ncu summary (unit: one edge of one
    frame in one iteration): warp instructions issued, ALU-pipe warp instructions and
    shared-memory wavefronts; None when the kernel sources changed since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            t = json.load(fh)
    except Exception:
        return None
    e = t.get(f"{kernel}:{mode}")
    if not e or e.get("source_hash") != kernel_source_hash(kernel) or "warp_inst_per_unit" not in e:
        return None
    return e


def onchip_roofline(c, units, ms, sm_mhz, n_sms):
    """Fractions of the on-chip limits a frame-resident kernel runs into, from per-unit ncu
    counts scaled to this step's units and the step time measured here: instruction issue
    (one warp instruction per clock per scheduler, 4 schedulers per SM), the ALU pipe (16
    lanes per scheduler: a warp instruction every 2 clocks) and the shared-memory pipe (one
    128-byte wavefront per clock per SM), at the SM clock sampled during the step."""
    cycles = sm_mhz * 1e6 * ms * 1e-3
    issue = c["warp_inst_per_unit"] * units / (4 * n_sms * cycles)
    alu = 2 * c["alu_inst_per_unit"] * units / (4 * n_sms * cycles)
    smem = c["smem_wavefronts_per_unit"] * units / (n_sms * cycles)
    fr = {"issue": issue, "alu_pipe": alu, "shared_memory_pipe": smem}
    bound = max(fr, key=fr.get)
    return {"bound": bound, "frac": fr[bound], "fractions": fr, "sm_mhz": sm_mhz, "sms": n_sms,
            "per_unit": {k: c[k] for k in ("warp_inst_per_unit", "alu_inst_per_unit",
                                             "smem_wavefronts_per_unit")},
            "unit": "one edge of one frame in one iteration",
            "counters_from": c.get("capture")}


def cpu_threads():
    return os.cpu_count() or 1


def oracle_rate(code, llr, L, mode, budget_s=10.0, threads=None):
    """Time the oracle (as it stands) on a bounded sample; returns (Gbit/s, frames, seconds)."""
    import oracle
    g = oracle.Graph.from_code(code)
    threads = threads or cpu_threads()
    run = (lambda x: oracle.decode_f32(g, x, L, early_stop=False, threads=threads, soft=False)) \
        if mode == "fp32" else \
        (lambda x: oracle.decode_fixed(g, oracle.quantize(x), L, early_stop=False, threads=threads,
                                       soft=False))
    n = max(threads, 16)
    t = time.perf_counter()
    run(llr[:n])
    dt = time.perf_counter() - t
    n = int(min(llr.shape[0], max(threads, n * budget_s / max(dt, 1e-3))))
    t = time.perf_counter()
    run(llr[:n])
    dt = time.perf_counter() - t
    return n * code.N / dt / 1e9, n, dt


# ------------------------------------------------------------------ the other workloads

def other_workloads(timed):
    """The configured workloads besides the headline: the (3,6)-regular N=576 code (1024
    all-zero frames at 2.5 dB, 20 iterations, early stop) and the irregular N=64800 code
    (4096 all-zero frames at 1.0 dB, 50 iterations, early stop; its frames do not fit in
    shared memory, so it runs the streaming kernels), FP32 and fixed point."""
    import torch
    from paper_2507_10424_gb300 import inputs
    from paper_2507_10424_gb300.ldpc import Decoder
    out = {}
    for name, code, F, e, L in (("regular576", inputs.cfg_regular_576(), 1024, 2.5, 20),
                                ("irregular64800", inputs.cfg_irregular_64800(), 4096, 1.0, 50)):
        llr = torch.from_numpy(inputs.all_zero_awgn_llr(F, code.N, e, code.design_rate, 17)).cuda()
        for mode in ("fp32", "fixed"):
            dec = Decoder.from_code(code, mode=mode)
            # resident tile shape, or check-pass staging when streaming, timed on these frames
            dec.autotune(F, L, llr=llr, early_stop=True)
            o = (torch.empty((F, code.N), dtype=torch.uint8, device="cuda"),
                 torch.empty(F, dtype=torch.int32, device="cuda"), None, None)
            ms = timed(lambda: dec.decode(llr, L, early_stop=True, out=o), 10, 3)
            it = o[1].float()
            B = edge_message_bytes(code, mode)
            out[f"{name}/{mode}"] = {
                "variant": dec.variant(), "frames": F, "ebn0_db": e, "max_iter": L,
                "ms_per_call": ms, "Gbit/s": F * code.N / (ms * 1e-3) / 1e9,
                "mean_iter": float(it.mean().item()),
                "fer": float((o[0] != 0).any(dim=1).float().mean().item()),
                "edge_message_GBs_at_mean_iter": F * float(it.mean().item()) * B / (ms * 1e-3) / 1e9}
            dec.close()
    # the same large code with a frame tile held across a thread-block cluster's shared
    # memory (never chosen automatically: measured slower than streaming)
    code = inputs.cfg_irregular_64800()
    F, L = 4096, 50
    llr = torch.from_numpy(inputs.all_zero_awgn_llr(F, code.N, 1.0, code.design_rate, 17)).cuda()
    for mode in ("fp32", "fixed"):
        dec = Decoder.from_code(code, mode=mode)
        dec.set_variant("cluster")
        o = (torch.empty((F, code.N), dtype=torch.uint8, device="cuda"),
             torch.empty(F, dtype=torch.int32, device="cuda"), None, None)
        ms = timed(lambda: dec.decode(llr, L, early_stop=True, out=o), 3, 1)
        C, FT, th, ncl = dec.cluster_shape()
        out[f"irregular64800/{mode}/cluster"] = {
            "variant": "cluster", "cluster_ctas": C, "frames_per_tile": FT, "threads": th,
            "clusters": ncl, "frames": F, "ebn0_db": 1.0, "max_iter": L, "ms_per_call": ms,
            "Gbit/s": F * code.N / (ms * 1e-3) / 1e9, "mean_iter": float(o[1].float().mean().item())}
        dec.close()
    return out


def early_stop_latency(timed, code, x, cw, L, mode):
    """The headline batch (same LLRs: random codewords at every Eb/N0 of the mix) decoded
    with early stop: launch-to-completion time of the whole batch and the decoded rate,
    on a decoder whose launch shape is tuned on these frames."""
    import torch
    from paper_2507_10424_gb300.ldpc import Decoder
    F = x.shape[0]
    dec = Decoder.from_code(code, mode=mode)
    dec.autotune(F, L, llr=x, early_stop=True)
    o = (torch.empty((F, code.N), dtype=torch.uint8, device="cuda"),
         torch.empty(F, dtype=torch.int32, device="cuda"), None, None)
    ms = timed(lambda: dec.decode(x, L, early_stop=True, out=o), 10, 3)
    it = o[1].float()
    res = {"frames": F, "max_iter": L, "ms_per_batch": ms,
           "Gbit/s": F * code.N / (ms * 1e-3) / 1e9, "mean_iter": float(it.mean().item()),
           "max_iter_used": int(it.max().item()),
           "fer": float((o[0] != torch.from_numpy(cw).cuda()).any(dim=1).float().mean().item()),
           "tuning": dict(zip(("frames_per_tile", "threads", "index_placement"), dec.tuning()))}
    dec.close()
    return res


def paper_shaped(timed):
    """The paper's decoding protocol on a stand-in with its code's dimensions (N=8176,
    M=1022: a 2x16 base of 511x511 blocks, each the sum of two seeded circulant
    permutations; the paper's matrix is not available): 50 random codewords at each Eb/N0
    of 3.0, 3.2, 3.4 and 3.6 dB (200 frames), at most 60 iterations, the syndrome tested
    every 6 iterations as in the paper's runs. Device-resident time per call, and end to
    end through ldpc_decode_host with pinned host buffers. The paper reports 48.31 s for
    this protocol on its code (about 33.8 kbit/s), given beside as context only."""
    import torch
    from paper_2507_10424_gb300 import inputs
    from paper_2507_10424_gb300.ldpc import Decoder
    code = inputs.cfg_paper_shaped()
    cw = inputs.Encoder(code).random_codewords(200, 21)
    llr = np.concatenate([inputs.bpsk_awgn_llr(cw[50 * k:50 * k + 50], e, code.design_rate, 40 + k)
                          for k, e in enumerate((3.0, 3.2, 3.4, 3.6))])
    x = torch.from_numpy(llr).cuda()
    xh = torch.from_numpy(llr).pin_memory()
    F, L, CE = 200, 60, 6
    paper_bits_per_s = F * code.N / 48.31
    out = {"code": f"N={code.N} M={code.M} E={code.E}, column weight 4, row weight 32",
           "frames": F, "max_iter": L, "check_every": CE,
           "paper_reported_Gbit/s": paper_bits_per_s / 1e9}
    for mode in ("fp32", "fixed"):
        dec = Decoder.from_code(code, mode=mode)
        dec.autotune(F, L, llr=x, early_stop=True, check_every=CE)
        o = (torch.empty((F, code.N), dtype=torch.uint8, device="cuda"),
             torch.empty(F, dtype=torch.int32, device="cuda"), None, None)
        ms = timed(lambda: dec.decode(x, L, early_stop=True, check_every=CE, out=o), 20, 3)
        ho = (torch.empty((F, code.N), dtype=torch.uint8).pin_memory(),
              torch.empty(F, dtype=torch.int32).pin_memory(), None, None)
        for _ in range(3):
            dec.decode_host(xh, L, early_stop=True, check_every=CE, out=ho)
        t = time.perf_counter()
        for _ in range(20):
            dec.decode_host(xh, L, early_stop=True, check_every=CE, out=ho)
        te = (time.perf_counter() - t) / 20
        assert (ho[0] == o[0].cpu()).all()
        gbit = F * code.N / (ms * 1e-3) / 1e9
        out[mode] = {"variant": dec.variant(), "ms_per_call": ms, "Gbit/s": gbit,
                     "e2e_ms_per_call": te * 1e3, "e2e_Gbit/s": F * code.N / te / 1e9,
                     "mean_iter": float(o[1].float().mean().item()),
                     "fer": float((o[0] != torch.from_numpy(cw).cuda()).any(dim=1).float().mean().item()),
                     "e2e_vs_paper_reported": F * code.N / te / paper_bits_per_s}
        dec.close()
    return out


# ------------------------------------------------------------------ learned decoder

def learned_vs_plain_large(timed):
    """Learned normalised/offset Min-Sum on the irregular N=64800 code, one weight pair per
    column degree (2, 3, 8) and iteration: trained here (20 unrolled iterations, 100 steps of
    4096 all-zero frames at Eb/N0 uniform in [0.8, 1.4] dB; the later iterations reuse the
    last row), then FER and mean iterations of both decoders (streaming variant, 4096
    frames, early stop) at 1.2 and 1.4 dB for iteration limits 30..50, and decoded Gbit/s of
    both at equal FER at 1.4 dB (plain at 50 iterations, learned at its matching limit)."""
    import torch
    from paper_2507_10424_gb300 import inputs, learn
    from paper_2507_10424_gb300.ldpc import Decoder, ldpc_train_workspace_size
    code = inputs.cfg_irregular_64800()
    dec = Decoder.from_code(code)
    train_ws = ldpc_train_workspace_size(dec.h, 4096, 20)
    t = time.perf_counter()
    alpha, beta, losses = learn.train_weights(dec, code, iters=20, steps=100, batch=4096,
                                              ebn0=(0.8, 1.4), lr=0.02, seed=1, every=True,
                                              encode=False)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t
    limits = (30, 35, 40, 45, 50)
    rows = learn.compare(dec, code, (alpha, beta), ebn0_points=(1.2, 1.4), frames=4096,
                         iters=limits, encode=False)
    match = {f"{e:.1f}dB": learn.iterations_to_match(rows, e, 50) for e in (1.2, 1.4)}
    L_l = match["1.4dB"] or 50
    src = learn.FrameSource(code, seed=11, encode=False)
    llr, bits = src.batch(4096, 1.4)
    out = (torch.empty_like(bits), torch.empty(4096, dtype=torch.int32, device="cuda"), None, None)
    res = {}
    for name, w, L in (("plain", None, 50), ("learned", (alpha, beta), L_l)):
        dec.set_weights(*(w if w else (None,)))
        dec.autotune(4096, L, llr=llr, early_stop=True)
        ms = timed(lambda: dec.decode(llr, L, early_stop=True, out=out), 3, 1)
        fer = float((out[0] != bits).any(dim=1).float().mean().item())
        res[name] = {"max_iter": L, "ms_per_call": ms, "Gbit/s": 4096 * code.N / (ms * 1e-3) / 1e9,
                     "fer": fer, "mean_iter": float(out[1].float().mean().item())}
    dec.set_weights(None)
    cls = dec.classes()
    dec.close()
    return {"code": "irregular N=64800 M=32400, column weights 2/3/8", "classes": cls,
            "train_steps": 100, "train_batch": 4096, "train_s": train_s,
            "train_workspace_bytes": train_ws,
            "loss_first_last": [float(np.mean(losses[:5])), float(np.mean(losses[-5:]))],
            "alpha_first_last_iteration": [alpha[0].round(4).tolist(), alpha[-1].round(4).tolist()],
            "beta_first_last_iteration": [beta[0].round(4).tolist(), beta[-1].round(4).tolist()],
            "iterations_to_match_plain_fer_at_50": match, "equal_fer_throughput_1.4dB": res,
            "fer_table": rows}


def learned_vs_plain(timed):
    """Learned normalised/offset Min-Sum on the (3,6)-regular N=576 code: trained here
    (10 unrolled iterations, 4096-frame batches at Eb/N0 uniform in [1, 4] dB), then the
    iteration limit at which it matches plain Min-Sum's frame error rate, and decoded Gbit/s
    of both at equal FER (early stop, 65536 frames at 2.5 dB)."""
    import torch
    from paper_2507_10424_gb300 import inputs, learn
    from paper_2507_10424_gb300.ldpc import Decoder
    code = inputs.cfg_regular_576()
    dec = Decoder.from_code(code)
    t = time.perf_counter()
    alpha, beta, losses = learn.train_weights(dec, code, iters=10, steps=400, batch=4096, lr=0.02,
                                              seed=1, every=True)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t
    rows = learn.compare(dec, code, (alpha, beta), ebn0_points=(2.0, 2.5, 3.0), frames=20000)
    match = {f"{e:.1f}dB": {f"plain@{p}": learn.iterations_to_match(rows, e, p) for p in (10, 20)}
             for e in (2.0, 2.5, 3.0)}
    # throughput at equal FER: plain at 20 iterations vs learned at its matching limit
    L_l = match["2.5dB"]["plain@20"] or 20
    src = learn.FrameSource(code, seed=11)
    llr, bits = src.batch(65536, 2.5)
    out = (torch.empty_like(bits), torch.empty(65536, dtype=torch.int32, device="cuda"), None, None)
    res = {}
    for name, w, L in (("plain", None, 20), ("learned", (alpha, beta), L_l)):
        dec.set_weights(*(w if w else (None,)))
        dec.autotune(65536, L, llr=llr, early_stop=True)
        ms = timed(lambda: dec.decode(llr, L, early_stop=True, out=out), 10, 3)
        fer = float((out[0] != bits).any(dim=1).float().mean().item())
        res[name] = {"max_iter": L, "ms_per_step": ms, "Gbit/s": 65536 * code.N / (ms * 1e-3) / 1e9,
                     "fer": fer, "mean_iter": float(out[1].float().mean().item())}
    dec.set_weights(None)
    return {"code": "(3,6)-regular N=576 M=288", "train_steps": 400, "train_s": train_s,
            "loss_first_last": [float(np.mean(losses[:10])), float(np.mean(losses[-10:]))],
            "alpha": alpha[:, 0].round(4).tolist(), "beta": beta[:, 0].round(4).tolist(),
            "iterations_to_match_plain_fer": match, "equal_fer_throughput_2.5dB": res,
            "fer_table": rows}


# ------------------------------------------------------------------ mixed codes, one launch

def _mixed_record(codes, frames, timed, seed0):
    """One graph replay of the batch of `codes` (frames[k] all-zero frames of code k at
    Eb/N0 2.0 dB, FP32, at most 25 iterations with early stop) against one decode call per
    code (each code tuned on its own frames first), bits compared."""
    import torch
    from paper_2507_10424_gb300 import inputs
    from paper_2507_10424_gb300.ldpc import Batch, Decoder
    L = 25
    decs = [Decoder.from_code(c) for c in codes]
    xs = []
    for k, (c, F) in enumerate(zip(codes, frames)):
        xs.append(torch.from_numpy(inputs.all_zero_awgn_llr(F, c.N, 2.0, c.design_rate, seed0 + k)).cuda())
    # every code tuned on its own frames first: the per-code calls use the tuned shapes, and
    # the batch's large codes run the streaming kernels with their handle's tuned staging
    for d, x, F in zip(decs, xs, frames):
        try:  # resident tile shape, or streaming check-pass staging (rows of at most 16 edges)
            d.autotune(F, L, llr=x, early_stop=True)
        except Exception:
            pass
    batch = Batch(decs)
    for k, x in enumerate(xs):
        batch.set_io(k, x)
    threads, _ = batch.autotune(L)
    batch.prepare(L)
    batch.capture()
    stream = batch.stream

    def one_launch():
        batch.replay()

    ms_graph = timed(one_launch, 20, 3, st=stream)
    bits_total = sum(c.N * F for c, F in zip(codes, frames))
    outs = []
    for d, c, F, x in zip(decs, codes, frames, xs):
        outs.append((torch.empty((F, c.N), dtype=torch.uint8, device="cuda"),
                     torch.empty(F, dtype=torch.int32, device="cuda"), None, None))

    def per_code():
        for d, x, o in zip(decs, xs, outs):
            d.decode(x, L, early_stop=True, out=o)

    ms_seq = timed(per_code, 20, 3)
    same = all(bool((batch._keep[k][1] == outs[k][0]).all()) for k in range(len(codes)))
    info = batch.info()
    cap = batch.tile_frames()
    split = batch.sm_split()
    batch.close()
    return {"codes": [{"N": c.N, "M": c.M, "E": c.E, "frames": F} for c, F in zip(codes, frames)],
            "max_iter": L, "ebn0_db": 2.0, "frames_total": int(sum(frames)),
            "one_launch_graph": {"ms": ms_graph, "Gbit/s": bits_total / (ms_graph * 1e-3) / 1e9,
                                 "threads": threads, "frames_per_tile_at_most": cap,
                                 "sm_split": split,
                                 "codes_in_shared_memory": info["codes_in_shared_memory"]},
            "per_code_calls": {"ms": ms_seq, "Gbit/s": bits_total / (ms_seq * 1e-3) / 1e9,
                               "launches": sum(d.last_kernel_count() for d in decs)},
            "graph_speedup": ms_seq / ms_graph,
            "identical_bits": same}


def mixed_codes(timed):
    """Eight irregular codes (N 256..16200, rates 1/2..5/6, column weights {2,3,4,8}),
    frames per code drawn from [64, 8192], all-zero codeword at Eb/N0 = 2.0 dB, FP32, at
    most 25 iterations with early stop: decoded as one persistent launch replayed from a
    CUDA graph, and, for comparison, one decode call per code (each autotuned). Also the
    same eight codes with 64 frames each (the low end of the range), where one call per
    code leaves most of the GPU idle."""
    from paper_2507_10424_gb300 import inputs
    codes, frames = inputs.cfg_mixed_codes()
    rec = _mixed_record(codes, frames, timed, 300)
    rec["short_batches"] = _mixed_record(codes, [64] * len(codes), timed, 400)
    return rec


# the extra measurements that --part runs alone (name -> function)
PARTS = {"mixed_codes": "mixed_codes", "learned": "learned_vs_plain",
         "learned_large": "learned_vs_plain_large", "other_workloads": "other_workloads",
         "paper_shaped": "paper_shaped"}


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    code = make_code(args.workload)
    L = args.iters
    threads = cpu_threads()
    _, llr, _ = make_llr(code, 4096 if args.workload == "qc2304" else 256, 7, args.workload)
    g = oracle.Graph.from_code(code)

    def step(x):
        if args.mode == "fp32":
            oracle.decode_f32(g, x, L, early_stop=False, threads=threads, soft=False)
        else:
            oracle.decode_fixed(g, oracle.quantize(x), L, early_stop=False, threads=threads, soft=False)

    t = time.perf_counter()
    step(llr[: max(threads, 32)])
    per_frame = (time.perf_counter() - t) / max(threads, 32)
    S = int(min(len(llr), max(threads, 0.5 / max(per_frame, 1e-6))))  # ~0.5 s per step
    for w in range(args.warmup):
        step(llr[:S])
    t = time.perf_counter()
    for k in range(args.steps):
        step(llr[:S])
    dt = time.perf_counter() - t
    val = S * code.N * args.steps / dt / 1e9
    sample = (f"{S} of the workload's {args.frames} frames per step (a bounded sample), "
              f"on {threads} host threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "Gbit/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.mode == "fp32" else "i16",
        "data": "synthetic",
        "config": {"workload": workload_name(code, args.frames, L, args.workload), "mode": args.mode},
        "cpu_baseline": {"value": val, "unit": "Gbit/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


# ------------------------------------------------------------------ our arm

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    from paper_2507_10424_gb300 import build, shard
    build.build()
    from paper_2507_10424_gb300.ldpc import Decoder

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if args.part:  # one extra measurement alone, timed like the others
        def part_timed(fn, K, W, sampler=None, st=None):
            st = st or torch.cuda.current_stream()
            for _ in range(W):
                fn()
            torch.cuda.synchronize()
            p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            p0.record(st)
            for _ in range(K):
                fn()
            p1.record(st)
            torch.cuda.synchronize()
            return p0.elapsed_time(p1) / K
        print(json.dumps({"part": args.part, args.part: globals()[PARTS[args.part]](part_timed)}))
        return 0
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        return shard.max_over_ranks(x, device="cuda")

    code = make_code(args.workload)
    F, L, mode = args.frames, args.iters, args.mode
    cw, llr, bounds = make_llr(code, F, shard.rank_seed(1000, rank), args.workload)
    snrs = SNRS if args.workload == "qc2304" else [1.0]
    dec = Decoder.from_code(code, mode=mode)
    dec.set_variant(args.variant)
    variant = dec.variant()
    if variant == "resident":  # launch shape for this code on this GPU
        if args.tuning == "auto":
            dec.autotune(F, L)
        else:
            dec.set_tuning(*[int(v) for v in args.tuning.split(",")])
    elif variant == "stream":  # check-pass staging (codes whose rows have at most 16 edges)
        if args.tuning == "auto":
            try:
                dec.autotune(F, L)
            except Exception:
                pass
        else:
            dec.set_stream_staging(*[int(v) for v in args.tuning.split(",")])
    x = torch.from_numpy(llr).cuda()
    bits = torch.empty((F, code.N), dtype=torch.uint8, device="cuda")
    iters = torch.empty(F, dtype=torch.int32, device="cuda")
    out = (bits, iters, None, None)
    stream = torch.cuda.current_stream()

    def step():
        dec.decode(x, L, early_stop=False, out=out)

    def timed(fn, K, W, sampler=None, st=None):
        """Mean ms per call of fn over K calls after W warm-up calls, CUDA events on the
        stream the work is launched on (st, else the current stream)."""
        st = st or stream
        for _ in range(W):
            fn()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if sampler:
            sampler.mark("t0")
        e0.record(st)
        for _ in range(K):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        if sampler:
            sampler.mark("t1")
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) / K)

    step()
    torch.cuda.synchronize()
    per_step_kernels = dec.last_kernel_count()
    sampler = ClockSampler(local)
    sampler.start()
    ms = timed(step, args.steps, max(3, args.warmup), sampler)
    clocks = sampler.stop()

    bits_total = F * code.N * world
    value = bits_total / (ms * 1e-3) / 1e9
    peak, peak_kind = measured_peak_hbm()
    B = edge_message_bytes(code, mode)
    alg_bytes = F * L * B
    achieved = alg_bytes / (ms * 1e-3) / 1e9
    if variant == "resident":  # one launch per step: the step time is the kernel's
        kname, traffic = "k_resident", ncu_traffic("k_resident", mode, F)
        c = ncu_counters("k_resident", mode)
        onchip = None
        if c and clocks and clocks.get("sm_mhz"):
            onchip = onchip_roofline(c, code.E * F * L, ms, clocks["sm_mhz"],
                                     torch.cuda.get_device_properties(local).multi_processor_count)
    else:  # about 2 L + 5 launches per step: the figure is the whole decode's
        kname, traffic = "the whole decode (check and variable passes, L iterations)", None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": kname, "peak_kind": peak_kind,
                "algorithmic_bytes_per_frame_iteration": B,
                # the same against the nominal HBM3e bandwidth the targets are quoted at
                "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS}
    if variant == "resident":
        # the edge messages never leave shared memory, so the HBM fraction above is an
        # effective rate; this is the fraction of the limit the kernel actually runs into
        roofline["onchip"] = onchip

    # error rates per SNR point (outside the timed region): frame and bit error rates of
    # the decoded bits, beside the channel's own hard decisions (the uncoded rate) and its
    # closed form Q(sqrt(2 R Eb/N0)); below the code's threshold failed decodes end with
    # more bit errors than the channel made
    ber_fer = {}
    cw_dev = torch.from_numpy(cw).cuda()
    wrong_bits = bits != cw_dev
    wrong = wrong_bits.any(dim=1).cpu().numpy()
    bit_err = wrong_bits.float().mean(dim=1).cpu().numpy()
    raw_err = ((x < 0) != cw_dev.bool()).float().mean(dim=1).cpu().numpy()
    for k, e in enumerate(snrs):
        a, b = bounds[k], bounds[k + 1]
        ber_fer[f"{e:.1f}dB"] = {
            "fer": float(wrong[a:b].mean()), "ber": float(bit_err[a:b].mean()),
            "channel_ber": float(raw_err[a:b].mean()),
            "uncoded_ber": 0.5 * math.erfc(math.sqrt(code.design_rate * 10.0 ** (e / 10.0)))}
    del wrong_bits, cw_dev

    result = {
        "metric": METRIC, "value": value, "unit": "Gbit/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if mode == "fp32" else "i16", "data": "synthetic",
        "config": {"workload": workload_name(code, F, L, args.workload), "frames_per_gpu": F, "iters": L,
                   "early_stop": False, "mode": mode, "variant": variant,
                   "tuning": (dict(zip(("frames_per_tile", "threads", "index_placement"), dec.tuning()))
                              if variant == "resident" else
                              dict(zip(("warps_per_cta", "stages", "frames_per_lane"), dec.stream_staging()))),
                   "l2": f"inputs larger than L2 ({llr.nbytes / 1e6:.0f} MB of LLRs per step)"},
        "roofline": roofline,
        "gpu_launches": per_step_kernels * args.steps,
        "clocks": clocks,
        "fer": ber_fer,
    }

    if not args.quick:
        # end to end through the C ABI with host buffers (pinned), copies inside the timed region
        xh = torch.from_numpy(llr).pin_memory()
        bh = torch.empty((F, code.N), dtype=torch.uint8).pin_memory()
        ih = torch.empty(F, dtype=torch.int32).pin_memory()
        hout = (bh, ih, None, None)
        dec.decode_host(xh, L, early_stop=False, out=hout)
        Ke = max(3, args.steps // 10)
        barrier()
        t = time.perf_counter()
        for _ in range(Ke):
            dec.decode_host(xh, L, early_stop=False, out=hout)
        te = max_over_ranks((time.perf_counter() - t) / Ke)
        assert (bh.numpy() == bits.cpu().numpy()).all()
        result["e2e"] = {"value": bits_total / te / 1e9, "unit": "Gbit/s",
                         "h2d_bytes_per_step": int(xh.numel() * 4),
                         "d2h_bytes_per_step": int(bh.numel() + ih.numel() * 4),
                         "ms_per_step": te * 1e3}

        # the host link alone, outside the timed region: the same bytes copied between the
        # pinned buffers and the device with no decode (the pipelined e2e step cannot beat
        # its input copy)
        def link_ms(dst, src, n=5):
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0.record(stream)
            for _ in range(n):
                dst.copy_(src, non_blocking=True)
            l1.record(stream)
            torch.cuda.synchronize()
            return l0.elapsed_time(l1) / n

        xd = torch.empty_like(x)
        h2d_ms, d2h_ms = link_ms(xd, xh), link_ms(bh, bits)
        del xd
        result["e2e"]["link"] = {"h2d_ms": h2d_ms, "h2d_GBs": xh.numel() * 4 / h2d_ms / 1e6,
                                 "d2h_ms": d2h_ms, "d2h_GBs": bh.numel() / d2h_ms / 1e6}
    # The extra measurements are single-GPU records: they run at N=1 only (under torchrun the
    # rank-0-only parts would otherwise enter the timer's collectives alone, and every GPU
    # would be held while one of them works).
    if not args.quick and args.workload == "qc2304" and world == 1:
        # the other arithmetic mode and the other kernel variant, same workload
        others = {}
        for m2, v2 in (("fixed" if mode == "fp32" else "fp32", "auto"), (mode, "stream")):
            d2 = Decoder.from_code(code, mode=m2)
            d2.set_variant(v2)
            try:  # resident tile shape, or streaming staging and message format
                d2.autotune(F, L)
            except Exception:
                pass
            o2 = (torch.empty_like(bits), torch.empty_like(iters), None, None)
            f2 = lambda: d2.decode(x, L, early_stop=False, out=o2)
            ms2 = timed(f2, max(5, args.steps // 5), 3)
            B2 = edge_message_bytes(code, m2)
            ach2 = F * L * B2 / (ms2 * 1e-3) / 1e9
            others[f"{m2}/{d2.variant()}"] = {
                "value": bits_total / (ms2 * 1e-3) / 1e9, "unit": "Gbit/s", "ms_per_step": ms2,
                "hbm_edge_message_GBs": ach2, "frac": ach2 / peak}
            d2.close()
        # the paper's dense m x n map-reduce form (Algorithm 2) as a baseline, on a slice of
        # the batch (its workspace is 4 M N bytes per frame)
        Fd = min(F, 2048)
        dd = Decoder.from_code(code)
        dd.set_variant("dense")
        od = (torch.empty((Fd, code.N), dtype=torch.uint8, device="cuda"),
              torch.empty(Fd, dtype=torch.int32, device="cuda"), None, None)
        xd = x[:Fd].contiguous()
        msd = timed(lambda: dd.decode(xd, L, early_stop=False, out=od), 3, 1)
        others["fp32/dense_baseline"] = {"value": Fd * code.N * world / (msd * 1e-3) / 1e9,
                                         "unit": "Gbit/s", "ms_per_step": msd, "frames": Fd,
                                         "identical_bits": bool((od[0] == bits[:Fd]).all())}
        dd.close()
        result["other_paths"] = others
        result["early_stop_latency"] = early_stop_latency(timed, code, x, cw, L, mode)
        if rank == 0:
            result["other_workloads"] = other_workloads(timed)
            result["paper_shaped"] = paper_shaped(timed)
            result["learned"] = learned_vs_plain(timed)
            result["learned_large"] = learned_vs_plain_large(timed)
            result["mixed_codes"] = mixed_codes(timed)
    if not args.quick and world == 1 and rank == 0:
        val, n, dt = oracle_rate(code, llr, L, mode)
        result["cpu_baseline"] = {"value": val, "unit": "Gbit/s", "cores": cpu_threads(),
                                  "kind": "oracle",
                                  "sample": f"{n} frames of this workload, {L} iterations "
                                            f"({dt:.1f} s on {cpu_threads()} threads)"}
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

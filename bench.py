#!/usr/bin/env python3
"""Throughput benchmark: batched ADMM-LP decoding of the (3,6) n=1056 LDPC code.

Workload (one "step"): 4 x 10^4 frames -- 10^4 frames at each of Eb/N0 = 1.5,
2.0, 2.5, 3.0 dB (BPSK/AWGN, all-zeros codeword, seeded) -- of a seeded
4-cycle-free (3,6)-regular Gallager code with n = 1056, m = 528, decoded with
mu = 3, rho = 1.9 for a fixed 300 ADMM iterations (eps = 0), FP32.  One step is
one lpdec_decode call over the whole batch, which runs every part of the hot
path (x-update, over-relaxed z/lambda update with the parity-polytope
projection, final residual test, hard decision, syndrome and certificate).

Metric: decoded information bits per second (k = n - m = 528 per frame).
Usage:  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank decodes its own seeded batch (frames are independent:
weak scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SNRS = (1.5, 2.0, 2.5, 3.0)
MU, RHO, ITERS = 3.0, 1.9, 300
METRIC = "ADMM-LP decoded info bits/s, (3,6) n=1056 LDPC"
UNIT = "info bits/s"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames-per-point", type=int, default=10_000)
    ap.add_argument("--code", default="C1056", choices=["C96", "C1056", "C2640", "C4000", "C8000"],
                    help="code of the single-code workload (the headline is C1056)")
    ap.add_argument("--iters", type=int, default=300, help="fixed ADMM iterations of the single-code workload "
                    "(with --eps > 0: the most a frame may run)")
    ap.add_argument("--eps", type=float, default=0.0, help="stopping tolerance of the single-code workload "
                    "(0: fixed iterations; > 0: per-frame early exit, RESIDENT schedule only)")
    ap.add_argument("--no-autotune", action="store_true", help="use the library's default tile")
    ap.add_argument("--tile", default="", help="GROUP_THREADS,GROUPS[,RING_SLOTS]: set the single-code tile instead of "
                    "autotuning (RING_SLOTS > GROUPS: the STREAMED ring kernel)")
    ap.add_argument("--schedule", default="resident", choices=["resident", "streamed", "auto"])
    ap.add_argument("--state", default="f32", choices=["f32", "bf16", "f16", "q16"])
    ap.add_argument("--variants", type=int, default=1, help="also time the other schedules/precisions")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU work of the oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-latency", action="store_true", help="skip the served p50/p99 leg of the headline")
    ap.add_argument("--latency-rate", type=float, default=5e4, help="offered frames/s of the headline's served leg")
    ap.add_argument("--workload", default="single",
                    choices=["single", "mixed", "precision", "served", "bsc", "sweep", "dual"],
                    help="single: the headline C1056 batch; mixed: three codes in one persistent launch; "
                         "precision: FP32 / BF16 / FP16 state storage; served: Poisson request stream; "
                         "bsc: random (3,6) ensemble over the BSC; sweep: eps / mu / rho parameter study; "
                         "dual: dual subgradient decoder (appendix) against ADMM on the same frames")
    ap.add_argument("--ensemble-codes", type=int, default=10)
    ap.add_argument("--ensemble-frames", type=int, default=1000, help="frames per code per crossover")
    ap.add_argument("--sweep-frames", type=int, default=4000)
    ap.add_argument("--dual-frames", type=int, default=10_000, help="frames per Eb/N0 point of the dual workload")
    ap.add_argument("--served-rate", type=float, default=2e5, help="offered load, frames/s")
    ap.add_argument("--served-requests", type=int, default=200_000)
    ap.add_argument("--served-round", type=int, default=8, help="ADMM iterations per server round")
    ap.add_argument("--served-round-n8000", type=int, default=0,
                    help="rounds of the n=8000 code, whose frames run longest (0: --served-round)")
    ap.add_argument("--mixed-frames", type=int, default=30_000)
    ap.add_argument("--precision-frames", type=int, default=100_000)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_seeds(rank: int) -> list[int]:
    """LLR seeds of one rank's batch (one per Eb/N0 point): ranks decode disjoint,
    independent frames, so sharding needs no exchange of data."""
    return [100 + p + 1000 * rank for p in range(len(SNRS))]


CODE_SEEDS = {"C96": 0, "C1056": 0, "C2640": 1, "C4000": 2, "C8000": 3}


def make_workload(frames_per_point: int, rank: int, name: str = "C1056"):
    from paper_1204_0556_gb300 import inputs as I

    code = I.benchmark_code(name, CODE_SEEDS[name])
    llr = np.concatenate([I.awgn_llr(code, snr, frames_per_point, seed)
                          for snr, seed in zip(SNRS, workload_seeds(rank))])
    return code, llr


def max_over_ranks(value: float, device=None) -> float:
    """The slowest rank's time (the job's time); identity without a process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def algorithmic_bytes_per_frame_iter(code, state_bytes: int) -> int:
    """2E(s_z + s_lambda) + 12N: every edge's z and lambda read and written once,
    gamma read, x written and read once."""
    return 2 * code.E * (2 * state_bytes) + 12 * code.n


def moved_bytes_per_frame_iter(code, state_bytes: int) -> int:
    """2E(s_z + s_lambda) + 4N: what a STREAMED launch of the fused kernel must
    move per frame-iteration (x never leaves shared memory)."""
    return 2 * code.E * (2 * state_bytes) + 4 * code.n


def _batcher_comparators(n: int) -> int:
    """Comparators of Batcher's odd-even merge sort on n inputs (padded network,
    comparators touching padding dropped): the sort of Algorithm 2's first step."""
    p2 = 1
    while p2 < n:
        p2 *= 2
    c, p = 0, 1
    while p < p2:
        k = p
        while k >= 1:
            j = k % p
            while j <= p2 - 1 - k:
                for i in range(k):
                    if (i + j) // (2 * p) == (i + j + k) // (2 * p) and i + j + k < n:
                        c += 1
                j += 2 * k
            k //= 2
        p *= 2
    return c


def hand_ops_per_frame_iter(code) -> int:
    """A hand count of the FP32 operations of one frame-iteration, from the
    code's degrees (used only for kernels without an instruction-counter
    capture; a fused multiply-add counts 1):
      variable of degree dv (x-update): dv (accumulate) + 4;
      edge (over-relaxed q, v, lambda-update): 4;
      check of degree d (projection): clip d, facet choice 3d, violation sum d,
      breakpoints d, sort 2*comparators(d), beta candidates 3d + 1 divide, output 3d."""
    ops = int((code.var_degrees + 4).sum()) + 4 * code.E
    for d in code.check_degrees.tolist():
        ops += 12 * d + 2 * _batcher_comparators(d) + 1
    return ops


# Counters of the decode kernels from ncu captures, keyed by code/schedule and by
# a hash of the kernel sources at capture time (a changed kernel reports null
# until it is captured again).  Per frame-iteration:
#   fp32_ops   FP32 lane-operations: sm__sass_thread_inst_executed_op_fp32_pred_on
#              plus one more lane for every packed FADD2/FMUL2/FFMA2, so an FMA
#              counts once, against a peak of one operation per FP32 lane per cycle;
#   warp_inst  warp instructions issued (smsp__inst_executed.sum).
# traffic: dram__bytes_read.sum + dram__bytes_write.sum of one launch of
# traffic_frames frames (the bench's full-size launch where it was captured).
KERNEL_SOURCES = ("lpdec_device.cuh", "lpdec_kclass.cuh", "lpdec_internal.h")
MEASURED_COUNTERS = {
    # C1056, 8000 frames x 300 iterations, tile 6 x 160 (instruction counters); traffic from the
    # bench's full-size launch (4 x 10^4 frames, tile 6 x 160)
    "C1056/resident/f32": {"hash": "8d57f3c0b45d2c40", "fp32_ops": 53835, "warp_inst": 3957.4,
                           "traffic": 174_958_592 + 165_210_880, "traffic_frames": 40000},
    # 608 frames x 300 iterations; C8000 at tile 1 x 896, C4000 at 2 x 416 (no full-size traffic capture)
    "C8000/resident/f32": {"hash": "8d57f3c0b45d2c40", "fp32_ops": 635319, "warp_inst": 72441.4},
    "C4000/resident/f32": {"hash": "8d57f3c0b45d2c40", "fp32_ops": 255646, "warp_inst": 28131.1},
}


def kernel_source_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1204_0556_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def counters_for(key: str):
    rec = MEASURED_COUNTERS.get(key)
    if not rec or rec["hash"] != kernel_source_hash():
        return None
    return rec


def traffic_per_launch(key: str, frames: int):
    """DRAM bytes of one launch of `frames` frames, from the capture: exact when
    the capture ran the same number of frames, else scaled by the frames."""
    rec = counters_for(key)
    if not rec or "traffic" not in rec:
        return None
    return int(rec["traffic"] * frames / rec["traffic_frames"])


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [t.strip() for t in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = np.array([float(r[1]) for r in rows])
        mx = float(rows[0][2])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        loaded = sm[sm >= 0.5 * sm.max()] if sm.max() > 0 else sm
        return {"sm_mhz": float(np.median(loaded)), "sm_max_mhz": mx, "reasons": reasons,
                "samples": int(len(rows)), "power_w_max": max(float(r[3]) for r in rows)}


def oracle_sample(code, llr, seconds: float, eps: float = 0.0):
    """Time the FP64 oracle on a bounded, evenly spread sample of the workload."""
    import oracle

    oracle.build()
    threads = oracle.default_threads()
    F = len(llr)
    probe = np.linspace(0, F - 1, max(threads, 16)).astype(int)
    t0 = time.perf_counter()
    oracle.decode(code.row_ptr, code.col_idx, code.n, llr[probe].astype(np.float64), mu=MU, rho=RHO, eps=eps,
                  max_iter=ITERS, threads=threads)
    per_frame = (time.perf_counter() - t0) / len(probe)
    n = int(min(F, max(len(probe), seconds / max(per_frame, 1e-9))))
    idx = np.linspace(0, F - 1, n).astype(int)
    t0 = time.perf_counter()
    oracle.decode(code.row_ptr, code.col_idx, code.n, llr[idx].astype(np.float64), mu=MU, rho=RHO, eps=eps,
                  max_iter=ITERS, threads=threads)
    dt = time.perf_counter() - t0
    return {"value": n * code.k_design / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n} of {F} frames (evenly spaced over the 4 Eb/N0 points), "
                      f"{f'{ITERS} iterations each' if eps == 0 else f'eps={eps:g}, at most {ITERS} iterations'}, "
                      f"FP64, {threads} threads", "seconds": round(dt, 2)}


def run_reference(args, ws, rank):
    """The FP64 CPU oracle as the reference arm (rank 0 only)."""
    if rank != 0:
        return
    code, llr = make_workload(args.frames_per_point, 0)
    for _ in range(args.warmup):
        oracle_sample(code, llr, min(2.0, args.cpu_seconds / 4))
    vals = []
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = oracle_sample(code, llr, args.cpu_seconds / max(1, args.steps))
        vals.append(last["value"])
    wall = time.perf_counter() - t0
    v = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "C1056 (3,6) n=1056 m=528 Gallager seed 0, 4-cycle free; 4 x 10^4 frames "
                               "(10^4 at each of 1.5/2.0/2.5/3.0 dB), mu=3 rho=1.9, 300 fixed iterations",
                   "sample": last["sample"]},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                         "sample": last["sample"]},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _time_call(fn, steps, warmup):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


# Autotuner sample: enough frames for about 20 rounds of the frames a persistent
# grid holds in flight, so that tail effects of a short sample do not pick the tile.
AUTOTUNE_FRAMES = 16384


def autotune_codes(lpdec, handles, llrs, state):
    """Pick each code's tile with lpdec_autotune on up to 16384 of its frames (60 fixed iterations)."""
    import torch

    tiles = []
    for C, llr in zip(handles, llrs):
        sample = torch.from_numpy(np.ascontiguousarray(llr[:AUTOTUNE_FRAMES])).cuda()
        p = lpdec.make_params(mu=MU, rho=RHO, eps=0.0, max_iter=60, state=state, schedule="resident")
        tiles.append(lpdec.lpdec_autotune(C.handle, p, sample.shape[0], sample.data_ptr(),
                                          int(torch.cuda.current_stream().cuda_stream)))
    return tiles


def run_mixed(args):
    """Three codes interleaved 40/40/20 in one persistent launch, per-frame early exit."""
    import torch

    from paper_1204_0556_gb300 import build, inputs as I, lpdec

    build.build()
    codes = [I.benchmark_code("C1056", 0), I.benchmark_code("C2640", 1), I.benchmark_code("C4000", 2)]
    F = args.mixed_frames
    counts = [int(0.4 * F), int(0.4 * F), F - 2 * int(0.4 * F)]
    order = np.random.Generator(np.random.Philox(key=3)).permutation(F)
    fc = np.concatenate([np.full(n, c, dtype=np.int32) for c, n in enumerate(counts)])[order]
    snr = np.random.Generator(np.random.Philox(key=4)).uniform(1.5, 4.0, F)
    per_code = {}
    for c, code in enumerate(codes):
        idx = np.nonzero(fc == c)[0]
        per_code[c] = (idx, I.awgn_llr(code, snr[idx], len(idx), 40 + c))
    offsets = np.concatenate([[0], np.cumsum([codes[c].n for c in fc])])
    packed = np.empty(offsets[-1], dtype=np.float32)
    for c, (idx, llr) in per_code.items():
        for r, f in enumerate(idx):
            packed[offsets[f]:offsets[f + 1]] = llr[r]
    Cs = [lpdec.Code(cd) for cd in codes]
    p = lpdec.make_params(mu=MU, rho=RHO, eps=1e-5, max_iter=1000, state="f32", schedule="resident")
    tiles = autotune_codes(lpdec, Cs, [per_code[c][1] for c in range(3)], "f32")
    d_packed = torch.from_numpy(packed).cuda()
    out = lpdec.decode_mixed(Cs, fc, d_packed, p)
    ms_mixed = _time_call(lambda: lpdec.decode_mixed(Cs, fc, d_packed, p, out=out), args.steps, args.warmup)
    iters = out["iters"].cpu().numpy()
    bits = out["bits"].cpu().numpy()
    word_err = np.array([bits[offsets[f]:offsets[f + 1]].any() for f in range(F)])
    info = sum(codes[c].k_design for c in fc)
    # the same frames as plain single-code launches (frames grouped per code)
    d_per = {c: torch.from_numpy(llr).cuda() for c, (idx, llr) in per_code.items()}
    outs = {c: lpdec.decode(Cs[c], d_per[c], p) for c in d_per}

    def per_code_resident():
        for c in d_per:
            lpdec.decode(Cs[c], d_per[c], p, out=outs[c])

    ps = lpdec.make_params(mu=MU, rho=RHO, eps=1e-5, max_iter=1000, state="f32", schedule="streamed")

    def per_code_streamed():
        for c in d_per:
            lpdec.decode(Cs[c], d_per[c], ps, out=outs[c])

    ms_res = _time_call(per_code_resident, max(1, args.steps), 1)
    ms_str = _time_call(per_code_streamed, 1, 1)
    line = {
        "workload": "mixed", "metric": "ADMM-LP decoded info bits/s, mixed-code batch", "unit": UNIT,
        "value": info / (ms_mixed / 1000.0), "ms_per_step": ms_mixed, "steps": args.steps, "warmup": args.warmup,
        "frames": F, "frames_per_s": F / (ms_mixed / 1000.0),
        "config": {"codes": "C1056 (3,6) seed 0, C2640 (4,8) seed 1, C4000 (3,30) m=400 seed 2",
                   "mix": f"{counts[0]}/{counts[1]}/{counts[2]} interleaved by a seeded shuffle",
                   "snr": "Eb/N0 uniform in [1.5, 4.0] dB per frame", "eps": 1e-5, "max_iter": 1000,
                   "dtype": "f32", "launches_per_step": 1},
        "mean_iters": {codes[c].name: float(iters[fc == c].mean()) for c in range(3)},
        "wer": {codes[c].name: float(word_err[fc == c].mean()) for c in range(3)},
        "tiles": {codes[c].name: tiles[c] for c in range(3)},
        "vs_plain": {
            "per_code_resident_launches": {"value": info / (ms_res / 1000.0), "ms_per_step": ms_res,
                                           "launches_per_step": 3},
            "per_code_streamed_launches": {"value": info / (ms_str / 1000.0), "ms_per_step": ms_str,
                                           "launches_per_step": 3000},
        },
    }
    for C in Cs:
        C.close()
    print(json.dumps(line), flush=True)


def run_precision(args):
    """FP32 vs BF16 vs FP16 z/lambda storage (FP32 arithmetic), fixed 300 iterations."""
    import torch

    import oracle
    from paper_1204_0556_gb300 import build, inputs as I, lpdec

    build.build()
    oracle.build()
    F = args.precision_frames
    rows = []
    for name, hseed in (("C1056", 0), ("C4000", 2)):
        code = I.benchmark_code(name, hseed)
        C = lpdec.Code(code)
        for pt, snr in enumerate((2.5, 4.0)):
            llr = I.awgn_llr(code, snr, F, 200 + pt)
            d_llr = torch.from_numpy(llr).cuda()
            sample = np.linspace(0, F - 1, 48).astype(int)
            ref = oracle.decode(code.row_ptr, code.col_idx, code.n, llr[sample].astype(np.float64), mu=MU, rho=RHO,
                                eps=0.0, max_iter=ITERS)
            for state in ("f32", "bf16", "f16", "q16"):
                for sched in ("resident", "streamed"):
                    p = lpdec.make_params(mu=MU, rho=RHO, eps=0.0, max_iter=ITERS, state=state, schedule=sched)
                    out = lpdec.decode(C, d_llr, p)
                    ms = _time_call(lambda: lpdec.decode(C, d_llr, p, out=out), max(1, args.steps // 2), 1)
                    x = out["x"].cpu().numpy()
                    bits = out["bits"].cpu().numpy()
                    rows.append({
                        "code": name, "snr_db": snr, "state": state, "schedule": sched,
                        "value": F * code.k_design / (ms / 1000.0), "ms_per_step": ms,
                        "hbm_frac": round(F * ITERS * algorithmic_bytes_per_frame_iter(code, 4 if state == "f32"
                                                                                        else 2)
                                          / (ms / 1000.0) / 1e9 / measured_peaks()[0], 4),
                        "wer": float(bits.any(axis=1).mean()),
                        "max_abs_x_err_vs_oracle": float(np.abs(x[sample] - ref["x"]).max()),
                    })
        C.close()
    print(json.dumps({"workload": "precision", "frames_per_point": F, "iters": ITERS, "unit": UNIT,
                      "oracle_sample": "48 evenly spaced frames per point", "rows": rows}), flush=True)


def run_served(args):
    """Poisson arrivals of one-frame requests over four codes into lpdec_server."""
    import torch

    from paper_1204_0556_gb300 import build, inputs as I, lpdec

    build.build()
    names = ["C96", "C1056", "C2640", "C8000"]
    codes = [I.benchmark_code(nm, k) for k, nm in enumerate(names)]
    handles = [lpdec.Code(c) for c in codes]
    R = args.served_requests
    arrivals = np.cumsum(np.random.Generator(np.random.Philox(key=5)).exponential(1.0 / args.served_rate, R))
    which = np.random.Generator(np.random.Philox(key=6)).integers(0, 4, R).astype(np.int32)
    snr_rng = np.random.Generator(np.random.Philox(key=7))
    # A pool of 2048 seeded frames per code (Eb/N0 uniform in [1.5, 4.5] dB each)
    # is cycled through; a request's frame is drawn once per request.
    POOL = 2048
    pools = [I.awgn_llr(c, snr_rng.uniform(1.5, 4.5, POOL), POOL, 8 + 10 * k) for k, c in enumerate(codes)]
    # A code's rounds length is its own parameter: the long C8000 frames may take
    # longer rounds (less bookkeeping per iteration) without delaying the others.
    rounds = [args.served_round] * 3 + [args.served_round_n8000 or args.served_round]
    ps = [lpdec.make_params(mu=MU, rho=RHO, eps=1e-5, max_iter=1000, state="f32", iters_per_launch=r)
          for r in rounds]
    p = ps[0]
    tiles = autotune_codes(lpdec, handles, pools, "f32")
    srv = lpdec.Server(budget_bytes=8 << 30)
    ids = [srv.add_code(h) for h in handles]
    ptrs = [[pl[i].ctypes.data for i in range(POOL)] for pl in pools]
    outx = [np.empty(c.n, np.float32) for c in codes]
    outb = [np.empty(c.n, np.uint8) for c in codes]
    it_buf, ce_buf = np.empty(1, np.int32), np.empty(1, np.uint8)
    rid = np.zeros(R, dtype=np.uint64)
    iters = np.zeros(R, dtype=np.int32)
    err = np.zeros(R, dtype=bool)
    submit_lag = np.zeros(R)
    cursor = [0, 0, 0, 0]
    sub_fn = lpdec.load().lpdec_server_submit
    poll_fn = lpdec.load().lpdec_server_poll
    import ctypes

    rid_c = ctypes.c_uint64()
    # Warm start: a code's first request sizes and allocates its slot pool (a
    # one-time set-up of the server, hundreds of MB of device and pinned host
    # memory); one request per code is served before the timed stream.
    for c in range(4):
        st = sub_fn(srv.handle, ids[c], 1, ptrs[c][POOL - 1], ctypes.byref(ps[c]), ctypes.byref(rid_c))
        if st == 0:
            st = poll_fn(srv.handle, int(rid_c.value), -1, outx[c].ctypes.data, outb[c].ctypes.data,
                         it_buf.ctypes.data, ce_buf.ctypes.data)
        if st != 0:
            raise RuntimeError(lpdec.lpdec_last_error())
    done_submit = threading.Event()
    submitted = [0]
    busy_waits = [0]

    # Everything a submit needs is prepared before the timed stream, so that the
    # Python submit loop does as little as it can per request.
    req_code = [int(c) for c in which]
    req_ptr = []
    for c in req_code:
        req_ptr.append(ptrs[c][cursor[c]])
        cursor[c] = (cursor[c] + 1) % POOL
    req_id = [ids[c] for c in req_code]
    arr = arrivals.tolist()
    rid_l = [0] * R
    lag_l = [0.0] * R
    h, rid_ref, pc = srv.handle, ctypes.byref(rid_c), time.perf_counter
    p_refs = [ctypes.byref(q) for q in ps]
    req_p = [p_refs[c] for c in req_code]
    x_ptr = [o.ctypes.data for o in outx]
    b_ptr = [o.ctypes.data for o in outb]
    it_ptr, ce_ptr = it_buf.ctypes.data, ce_buf.ctypes.data

    def poller():
        for i in range(R):
            while submitted[0] <= i:
                time.sleep(0.0002)
            c = req_code[i]
            if poll_fn(h, rid_l[i], -1, x_ptr[c], b_ptr[c], it_ptr, ce_ptr) != 0:
                raise RuntimeError(lpdec.lpdec_last_error())
            iters[i] = it_buf[0]
            err[i] = bool(outb[c].any())

    th = threading.Thread(target=poller)
    th.start()
    t0 = pc()
    for i in range(R):
        a = arr[i]
        while pc() - t0 < a:
            pass
        st = sub_fn(h, req_id[i], 1, req_ptr[i], req_p[i], rid_ref)
        while st == lpdec.LPDEC_EBUSY:  # back-pressure: the queue is full, wait for the server
            busy_waits[0] += 1
            time.sleep(0.0005)
            st = sub_fn(h, req_id[i], 1, req_ptr[i], req_p[i], rid_ref)
        if st != 0:
            raise RuntimeError(lpdec.lpdec_last_error())
        rid_l[i] = rid_c.value
        lag_l[i] = pc() - t0 - a
        submitted[0] = i + 1
    done_submit.set()
    th.join()
    wall = pc() - t0
    rid[:] = rid_l
    submit_lag[:] = lag_l
    st = srv.stats()
    ctr = srv.counters()
    srv.close()
    info = sum(codes[c].k_design for c in which)
    # The plain path on the same frame mix: every pool frame decoded as a batch of
    # its code with one launch per iteration (STREAMED) and with the RESIDENT
    # schedule, same parameters and early exit.
    plain = {}
    for sched in ("streamed", "resident"):
        pp = lpdec.make_params(mu=MU, rho=RHO, eps=1e-5, max_iter=1000, state="f32", schedule=sched)
        d_pools = [torch.from_numpy(pl).cuda() for pl in pools]
        outs = [lpdec.decode(h, dp, pp) for h, dp in zip(handles, d_pools)]

        def run_all():
            for h, dp, o in zip(handles, d_pools, outs):
                lpdec.decode(h, dp, pp, out=o)

        ms = _time_call(run_all, 1, 1)
        bits_pool = sum(codes[c].k_design * POOL for c in range(4))
        plain[f"per_code_{sched}_batches"] = {"value": bits_pool / (ms / 1000.0), "ms": ms,
                                              "frames": 4 * POOL}
    line = {
        "workload": "served", "metric": "ADMM-LP served decode stream: sustained info bits/s, p50/p99 latency",
        "unit": UNIT, "value": info / wall, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
        "frames": R, "wall_s": wall, "server_bits_per_s_since_first_submit": st["bits_per_s"],
        "value_note": "info bits of the timed requests over the wall time from the first timed submit to the last "
                      "completion (bench clock), after one warm-up request per code",
        "offered_frames_per_s": args.served_rate, "achieved_submit_frames_per_s": R / (arrivals[-1] + submit_lag[-1]),
        "submit_lag_ms_p50": float(np.quantile(submit_lag, 0.50) * 1000),
        "submit_lag_ms_p99": float(np.quantile(submit_lag, 0.99) * 1000),
        "arrival_latency_note": "p50/p99 are submit-to-completion on the server clock; a request's latency from "
                                "its scheduled arrival adds its submit lag (queue back-pressure and driver pacing)",
        "backpressure_waits": busy_waits[0],
        "rounds": ctr["rounds"], "scheduler_busy_ms": ctr["round_wall_ms"], "gpu_busy_ms": ctr["round_gpu_ms"],
        "gpu_busy_frac": ctr["round_gpu_ms"] / max(1e-9, wall * 1000.0),
        "config": {"codes": "C96, C1056, C2640, C8000 (irregular dc 6..20, dv 3), uniform per request",
                   "snr": "Eb/N0 uniform in [1.5, 4.5] dB", "eps": 1e-5, "max_iter": 1000,
                   "iters_per_round": {names[c]: rounds[c] for c in range(4)}, "budget_bytes": 8 << 30,
                   "arrivals": f"Poisson, {args.served_rate:.0f} frames/s, {R} one-frame requests",
                   "frames": "2048 seeded frames per code, cycled"},
        "mean_iters": {names[c]: float(iters[which == c].mean()) for c in range(4)},
        "wer": {names[c]: float(err[which == c].mean()) for c in range(4)},
        "tiles": {names[c]: tiles[c] for c in range(4)},
        "vs_plain": plain,
    }
    for h in handles:
        h.close()
    print(json.dumps(line), flush=True)


def served_latency(lpdec, C, code, llr_h, rate: float, seconds: float, round_iters: int) -> dict:
    """The headline's frames and parameters (300 fixed iterations, FP32) served as
    a Poisson stream of one-frame requests through lpdec_server: p50/p99 latency
    from submit to completion, and the sustained bits/s."""
    import ctypes

    R = max(1, int(rate * seconds))
    arrivals = np.cumsum(np.random.Generator(np.random.Philox(key=9)).exponential(1.0 / rate, R))
    p = lpdec.make_params(mu=MU, rho=RHO, eps=0.0, max_iter=ITERS, state="f32", iters_per_launch=round_iters)
    srv = lpdec.Server(budget_bytes=8 << 30)
    cid = srv.add_code(C)
    F = len(llr_h)
    idx = np.arange(R) * max(1, F // R) % F  # frames spread over the four Eb/N0 points
    ptrs = [llr_h[i].ctypes.data for i in idx]
    sub_fn = lpdec.load().lpdec_server_submit
    poll_fn = lpdec.load().lpdec_server_poll
    rid = np.zeros(R, dtype=np.uint64)
    rid_c = ctypes.c_uint64()
    submitted = [0]
    outx = np.empty(code.n, np.float32)
    # warm start: the first request allocates the code's slot pool (one-time set-up)
    if sub_fn(srv.handle, cid, 1, ptrs[0], ctypes.byref(p), ctypes.byref(rid_c)) != 0 or \
            poll_fn(srv.handle, int(rid_c.value), -1, outx.ctypes.data, None, None, None) != 0:
        raise RuntimeError(lpdec.lpdec_last_error())

    def poller():
        for i in range(R):
            while submitted[0] <= i:
                time.sleep(0.0002)
            if poll_fn(srv.handle, int(rid[i]), -1, outx.ctypes.data, None, None, None) != 0:
                raise RuntimeError(lpdec.lpdec_last_error())

    th = threading.Thread(target=poller)
    th.start()
    t0 = time.perf_counter()
    for i in range(R):
        while time.perf_counter() - t0 < arrivals[i]:
            pass
        st = sub_fn(srv.handle, cid, 1, ptrs[i], ctypes.byref(p), ctypes.byref(rid_c))
        while st == lpdec.LPDEC_EBUSY:
            time.sleep(0.0005)
            st = sub_fn(srv.handle, cid, 1, ptrs[i], ctypes.byref(p), ctypes.byref(rid_c))
        if st != 0:
            raise RuntimeError(lpdec.lpdec_last_error())
        rid[i] = rid_c.value
        submitted[0] = i + 1
    th.join()
    wall = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    return {"p50_ms": stats["p50_ms"], "p99_ms": stats["p99_ms"], "sustained_bits_per_s": R * code.k_design / wall,
            "offered_frames_per_s": rate, "frames": R, "iters_per_round": round_iters,
            "note": f"the headline's C1056 frames and parameters ({ITERS} fixed iterations, FP32) as Poisson "
                    "one-frame requests through lpdec_server; latency from submit to completion"}


def run_bsc(args):
    """Random (3,6) n=1002 ensemble over the BSC: WER, BER, iterations split by outcome, ML lower bound."""
    import torch

    from paper_1204_0556_gb300 import analysis as A, build, inputs as I, lpdec

    build.build()
    ens = I.gallager_ensemble(1002, 3, 6, args.ensemble_codes)
    p = lpdec.make_params(mu=MU, rho=RHO, eps=1e-5, max_iter=1000, state="f32", schedule="resident")
    rows = []
    for cp in (0.03, 0.04, 0.05, 0.06, 0.07, 0.08):
        bits_all, iters_all, llr_all, mlb, frac, ms_tot = [], [], [], 0, 0, 0.0
        for k, code in enumerate(ens):
            C = lpdec.Code(code)
            llr = I.bsc_llr(code, cp, args.ensemble_frames, 7000 + 100 * k + int(cp * 1000))
            d = torch.from_numpy(llr).cuda()
            out = lpdec.decode(C, d, p)
            ms_tot += _time_call(lambda: lpdec.decode(C, d, p, out=out), 1, 0)
            bits = out["bits"].cpu().numpy()
            iters = out["iters"].cpu().numpy()
            mlb += int(A.ml_lower_bound_errors(code, llr, bits).sum())
            frac += A.pseudocodeword_summary(out["x"].cpu().numpy())["frames_fractional"]
            bits_all.append(bits)
            iters_all.append(iters)
            C.close()
        e = A.error_rates(np.concatenate(bits_all), np.concatenate(iters_all))
        F = e["frames"]
        e.update({"crossover": cp, "ml_lower_bound_wer": mlb / F, "fractional_frames": frac / F,
                  "frames_per_s": F / (ms_tot / 1000.0)})
        rows.append(e)
    print(json.dumps({"workload": "bsc", "codes": f"{args.ensemble_codes} seeded (3,6) Gallager codes, n=1002",
                      "frames_per_code": args.ensemble_frames, "mu": MU, "rho": RHO, "eps": 1e-5,
                      "max_iter": 1000, "rows": rows}), flush=True)


def run_sweep(args):
    """Parameter study on a (3,6) n=2640 code: WER, mean iterations and time vs eps, mu and rho."""
    import torch

    from paper_1204_0556_gb300 import analysis as A, build, inputs as I, lpdec

    build.build()
    code = I.gallager_code(2640, 3, 6, 5, remove_4cycles=True, name="(3,6) n=2640")
    C = lpdec.Code(code)
    F = args.sweep_frames
    cache = {}

    def point(snr, mu, rho, eps):
        if snr not in cache:
            cache[snr] = torch.from_numpy(I.awgn_llr(code, snr, F, 9000 + int(10 * snr))).cuda()
        d = cache[snr]
        p = lpdec.make_params(mu=mu, rho=rho, eps=eps, max_iter=1000, state="f32", schedule="resident")
        out = lpdec.decode(C, d, p)
        ms = _time_call(lambda: lpdec.decode(C, d, p, out=out), 1, 0)
        e = A.error_rates(out["bits"].cpu().numpy(), out["iters"].cpu().numpy())
        return {"snr_db": snr, "mu": mu, "rho": rho, "eps": eps, "wer": e["wer"], "iters_mean": e["iters_mean"],
                "ms_per_frame": ms / F}

    rows = []
    for mu in (1.0, 5.0, 7.0):  # WER vs the stopping tolerance (no over-relaxation)
        for bits_tol in (10, 14, 17, 20):
            rows.append(point(2.2, mu, 1.0, 2.0 ** -bits_tol))
    for snr in (1.9, 2.2, 2.5):  # WER and time vs mu
        for mu in (1.0, 2.0, 3.0, 5.0, 7.0, 10.0):
            rows.append(point(snr, mu, 1.0, 1e-5))
    for mu in (1.0, 3.0, 5.0, 7.0):  # time vs over-relaxation
        for rho in (1.0, 1.3, 1.6, 1.9):
            rows.append(point(2.8, mu, rho, 1e-5))
    C.close()
    print(json.dumps({"workload": "sweep", "code": "(3,6) Gallager n=2640 seed 5, 4-cycle free",
                      "frames_per_point": F, "max_iter": 1000, "rows": rows}), flush=True)


def run_dual(args):
    """Dual subgradient ascent (appendix) against ADMM (Algorithm 1, early exit)
    on the same frames: throughput, iterations, WER and certificates, per code,
    Eb/N0 and dual step size; plus a tile sweep of the dual kernel."""
    import torch

    from paper_1204_0556_gb300 import analysis as A, build, inputs as I, lpdec

    build.build()
    F = args.dual_frames
    rows, tiles = [], []
    for name, snrs in (("C1056", (3.0, 3.5, 4.0)), ("C2640", (3.0, 3.5))):
        code = I.benchmark_code(name, CODE_SEEDS[name])
        C = lpdec.Code(code)
        k_info = code.n - code.m
        if name == "C1056":
            d = torch.from_numpy(I.awgn_llr(code, 3.5, F, 9100)).cuda()
            for gt, g in ((64, 15), (96, 10), (128, 8), (192, 5), (256, 4), (128, 4), (192, 2), (32, 15)):
                lpdec.lpdec_dual_set_tile(C.handle, gt, g)
                out = lpdec.decode_dual(C, d, mu=0.25, max_iter=5000)
                ms = _time_call(lambda: lpdec.decode_dual(C, d, mu=0.25, max_iter=5000, out=out), 2, 1)
                it = float(out["iters"].double().sum().item())
                tiles.append({"group_threads": gt, "groups": g, "ms": ms,
                              "edge_iters_per_s": it * code.E / (ms / 1000.0)})
            best = min(tiles, key=lambda r: r["ms"])
            lpdec.lpdec_dual_set_tile(C.handle, best["group_threads"], best["groups"])
        for snr in snrs:
            d = torch.from_numpy(I.awgn_llr(code, snr, F, 9200 + int(10 * snr))).cuda()
            p = lpdec.make_params(mu=MU, rho=RHO, eps=1e-5, max_iter=1000, state="f32", schedule="resident")
            out = lpdec.decode(C, d, p)
            ms = _time_call(lambda: lpdec.decode(C, d, p, out=out), 2, 1)
            e = A.error_rates(out["bits"].cpu().numpy(), out["iters"].cpu().numpy())
            rows.append({"code": name, "snr_db": snr, "decoder": "admm", "mu": MU, "rho": RHO, "wer": e["wer"],
                         "iters_mean": e["iters_mean"], "cert": float(out["cert"].float().mean().item()),
                         "info_bits_per_s": F * k_info / (ms / 1000.0),
                         "edge_iters_per_s": e["iters_mean"] * F * code.E / (ms / 1000.0)})
            for mu in (0.125, 0.25, 0.5):
                out = lpdec.decode_dual(C, d, mu=mu, max_iter=5000)
                ms = _time_call(lambda: lpdec.decode_dual(C, d, mu=mu, max_iter=5000, out=out), 2, 1)
                e = A.error_rates(out["bits"].cpu().numpy(), out["iters"].cpu().numpy())
                rows.append({"code": name, "snr_db": snr, "decoder": "dual", "mu": mu, "wer": e["wer"],
                             "iters_mean": e["iters_mean"], "cert": float(out["cert"].float().mean().item()),
                             "info_bits_per_s": F * k_info / (ms / 1000.0),
                             "edge_iters_per_s": e["iters_mean"] * F * code.E / (ms / 1000.0)})
        C.close()
    print(json.dumps({"workload": "dual", "frames_per_point": F, "dual_max_iter": 5000, "admm_max_iter": 1000,
                      "admm_eps": 1e-5, "dual_tiles_C1056": tiles, "rows": rows}), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload == "mixed":
        run_mixed(args)
        return
    if args.workload == "precision":
        run_precision(args)
        return
    if args.workload == "served":
        run_served(args)
        return
    if args.workload == "bsc":
        run_bsc(args)
        return
    if args.workload == "sweep":
        run_sweep(args)
        return
    if args.workload == "dual":
        run_dual(args)
        return

    import torch

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1204_0556_gb300 import build, lpdec

    build.build()
    lpdec.load()

    global ITERS
    ITERS = args.iters
    code, llr_h = make_workload(args.frames_per_point, rank, args.code)
    F = len(llr_h)
    C = lpdec.Code(code)
    tile = None
    if args.tile:
        gt, g, *ring = (int(v) for v in args.tile.split(","))
        dt = {"f32": 0, "bf16": 1, "f16": 2, "q16": 3}[args.state]
        lpdec.lpdec_set_tile(C.handle, dt, gt, g)
        tile = {"group_threads": gt, "groups": g, "source": "--tile"}
        if ring and ring[0]:
            lpdec.lpdec_set_streamed_tile(C.handle, dt, gt, g, ring[0])
            tile["ring_slots"] = ring[0]
    tune_sample = []

    def tune(schedule, state):
        """Autotune the tile of one (schedule, state) on a sample of the workload:
        60 fixed iterations for RESIDENT, 12 launches for STREAMED."""
        if not tune_sample:
            tune_sample.append(torch.from_numpy(
                np.ascontiguousarray(llr_h[:: max(1, F // AUTOTUNE_FRAMES)][:AUTOTUNE_FRAMES])).cuda())
        smp = tune_sample[0]
        sch = "streamed" if schedule == "streamed" else "resident"
        p = lpdec.make_params(mu=MU, rho=RHO, eps=0.0, max_iter=12 if sch == "streamed" else 60, state=state,
                              schedule=sch)
        return lpdec.lpdec_autotune(C.handle, p, smp.shape[0], smp.data_ptr(),
                                    int(torch.cuda.current_stream().cuda_stream))

    if not args.tile and not args.no_autotune:
        tile = tune(args.schedule, args.state)
    dev = torch.device("cuda", local)
    llr = torch.from_numpy(llr_h).to(dev)
    out = {
        "x": torch.empty((F, code.n), dtype=torch.float32, device=dev),
        "bits": torch.empty((F, code.n), dtype=torch.uint8, device=dev),
        "iters": torch.empty((F,), dtype=torch.int32, device=dev),
        "cert": torch.empty((F,), dtype=torch.uint8, device=dev),
    }
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    if args.eps > 0 and args.schedule != "resident":
        raise SystemExit("--eps > 0 runs the RESIDENT schedule only")

    def time_variant(schedule, state, steps, warmup, eps=0.0):
        p = lpdec.make_params(mu=MU, rho=RHO, eps=eps, max_iter=ITERS, state=state, schedule=schedule)
        for _ in range(warmup):
            lpdec.decode(C, llr, p, stream=stream, out=out)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            lpdec.decode(C, llr, p, stream=stream, out=out)
        e1.record(stream)
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) / steps, dev)

    # ---- headline: timed region with clock sampling
    sampler = ClockSampler(local)
    with sampler:
        ms = time_variant(args.schedule, args.state, args.steps, args.warmup, args.eps)
    clocks = sampler.summary()
    bits_h = out["bits"].cpu().numpy()
    cert_h = out["cert"].cpu().numpy()
    # frame-iterations one step runs: all of them at fixed iterations, the
    # frames' own counts with early exit
    fi_step = F * ITERS if args.eps == 0 else int(out["iters"].cpu().numpy().astype(np.int64).sum())
    value = ws * F * code.k_design / (ms / 1000.0)

    state_bytes = 4 if args.state == "f32" else 2
    B = algorithmic_bytes_per_frame_iter(code, state_bytes)
    launches_per_step = 1 if args.schedule in ("resident", "auto") else ITERS
    bytes_per_launch = fi_step // launches_per_step * B
    launch_ms = ms / launches_per_step
    hbm_peak, peak_kind = measured_peaks()
    achieved = bytes_per_launch / (launch_ms / 1000.0) / 1e9
    kname = f"lpdec::decode_kernel ({code.name}, {args.state}, {args.schedule})"
    if args.schedule == "streamed":
        ring = lpdec.lpdec_get_tile(C.handle, {"f32": 0, "bf16": 1, "f16": 2, "q16": 3}[args.state],
                                    lpdec.SCHED_STREAMED)["ring_slots"]
        if ring:
            kname = f"lpdec::decode_kernel_ring ({code.name}, {args.state}, streamed, {ring} slots)"
    if args.schedule in ("resident", "auto"):
        # State stays in shared memory for all 300 iterations: the kernel is bound
        # by instruction issue, not HBM.  Peak: 152 SMs x 128 FP32 lanes x the
        # maximum SM clock; work: the FP32 lane-operations one frame-iteration
        # executes, from the instruction counters of an ncu capture of this kernel.
        sm_max = float(clocks.get("sm_max_mhz") or 2070.0)
        peak_gops = 152 * 128 * sm_max * 1e6 / 1e9
        rec = counters_for(f"{code.name}/resident/{args.state}")
        if rec:
            ops, ops_src = rec["fp32_ops"], "counted (ncu instruction counters of this kernel)"
        else:
            ops, ops_src = hand_ops_per_frame_iter(code), "hand count (no counter capture of this kernel)"
        ach_gops = fi_step * ops / (launch_ms / 1000.0) / 1e9
        roofline = {
            "bound": "alu", "achieved": round(ach_gops, 1), "peak": round(peak_gops, 1), "unit": "Gop/s",
            "frac": round(ach_gops / peak_gops, 4), "traffic": traffic_per_launch(f"{code.name}/resident/{args.state}", F),
            "kernel": kname,
            "note": f"{ops} FP32 lane-operations per frame-iteration ({ops_src}; an FMA counts once) x {fi_step} "
                    f"frame-iterations per launch; peak = 152 SMs x 128 FP32 lanes x {sm_max:.0f} MHz, of measured "
                    "maximum SM clock",
            "hbm_effective": {"achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                              "frac": round(achieved / hbm_peak, 4),
                              "note": f"algorithmic bytes {B} per frame-iteration over the {peak_kind} HBM copy "
                                      "bandwidth; an effective figure, since z/lambda/x never leave the SM"},
        }
        if rec:
            peak_wi = 152 * 4 * sm_max * 1e6 / 1e9
            ach_wi = fi_step * rec["warp_inst"] / (launch_ms / 1000.0) / 1e9
            roofline["issue"] = {"achieved": round(ach_wi, 1), "peak": round(peak_wi, 1), "unit": "G warp-inst/s",
                                 "frac": round(ach_wi / peak_wi, 4),
                                 "note": f"{rec['warp_inst']} warp instructions per frame-iteration (counted) over "
                                         "4 issue slots per SM per cycle"}
    else:
        Bm = moved_bytes_per_frame_iter(code, state_bytes)
        moved = F * (ITERS // launches_per_step) * Bm / (launch_ms / 1000.0) / 1e9
        roofline = {
            "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(achieved / hbm_peak, 4), "traffic": traffic_per_launch(f"{code.name}/streamed/{args.state}", F), "kernel": kname,
            "note": f"peak is the {peak_kind} HBM copy bandwidth; algorithmic bytes {B} per frame-iteration "
                    f"x {F} frames x {ITERS // launches_per_step} iterations per launch (they count x written and "
                    f"read once, 8N bytes, which the fused kernel keeps in shared memory, so frac can exceed 1)",
            "moved": {"bytes_per_frame_iter": Bm, "achieved": round(moved, 1), "frac": round(moved / hbm_peak, 4),
                      "note": "2E(s_z + s_lambda) + 4N: the bytes a launch must move (state in and out, LLRs in)"},
        }

    wer = {}
    per = args.frames_per_point
    for p, snr in enumerate(SNRS):
        wer[str(snr)] = float(bits_h[p * per:(p + 1) * per].any(axis=1).mean())

    line = {
        "metric": METRIC if code.name == "C1056" else METRIC.replace("(3,6) n=1056", code.name), "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.state, "data": "synthetic",
        "config": {"workload": f"{code.name}: n={code.n} m={code.m} seed {CODE_SEEDS[code.name]}"
                               f"{', 4-cycle free' if code.name in ('C1056', 'C2640') else ''}; {F} frames "
                               f"({per} at each of 1.5/2.0/2.5/3.0 dB), mu=3 rho=1.9, "
                               f"{f'{ITERS} fixed iterations' if args.eps == 0 else f'eps={args.eps:g}, at most {ITERS} iterations'}, "
                               f"FP32 arithmetic, {args.state} edge state (w = z - lambda/mu, lambda/mu)",
                   "schedule": args.schedule, "frames_per_step": F * ws, "tile": tile,
                   "l2": f"inputs larger than L2: {F * code.n * 4 / 1e6:.0f} MB of LLRs read and "
                         f"{F * code.n * 4 / 1e6:.0f} MB of x written per step",
                   "parallelism": f"frames sharded over {ws} rank(s), no collective on the data path"},
        "frames_per_s": ws * F / (ms / 1000.0),
        "wer": wer, "certified_frac": float(cert_h.mean()), "mean_iters": fi_step / F,
        "edge_iterations_per_s": ws * fi_step * code.E / (ms / 1000.0),
        # STREAMED: one decode launch per iteration plus the check for unfinished frames
        "gpu_launches": (launches_per_step + (0 if launches_per_step == 1 else 1)) * args.steps,
        "clocks": clocks,
        "roofline": roofline,
    }

    if args.variants and ws == 1:
        var = {}
        for sch, st in (("streamed", "f32"), ("streamed", "bf16"), ("streamed", "q16"), ("resident", "bf16")):
            if (sch, st) == (args.schedule, args.state):
                continue
            vtile = None
            if not args.tile and not args.no_autotune:
                vtile = tune(sch, st)
            vms = time_variant(sch, st, max(2, args.steps // 2), 2)
            vb = algorithmic_bytes_per_frame_iter(code, 4 if st == "f32" else 2)
            vl = 1 if sch == "resident" else ITERS
            vach = F * (ITERS // vl) * vb / ((vms / vl) / 1000.0) / 1e9
            var[f"{sch}-{st}"] = {"value": F * code.k_design / (vms / 1000.0), "ms_per_step": vms,
                                  "hbm_frac": round(vach / hbm_peak, 4), "launches_per_step": vl,
                                  "tile": vtile}
            if sch == "streamed":
                vm = moved_bytes_per_frame_iter(code, 4 if st == "f32" else 2)
                var[f"{sch}-{st}"]["moved_frac"] = round(
                    F * (ITERS // vl) * vm / ((vms / vl) / 1000.0) / 1e9 / hbm_peak, 4)
        line["variants"] = var

    if not args.no_latency and ws == 1:
        line["latency"] = served_latency(lpdec, C, code, llr_h, rate=args.latency_rate, seconds=1.0, round_iters=8)

    if not args.no_e2e:
        # end to end through the host entry point: pinned LLRs in, bits/iters/cert out, every step
        llr_pin = torch.from_numpy(llr_h).pin_memory()
        x_pin = torch.empty((F, code.n), dtype=torch.float32).pin_memory()
        b_pin = torch.empty((F, code.n), dtype=torch.uint8).pin_memory()
        i_pin = torch.empty((F,), dtype=torch.int32).pin_memory()
        c_pin = torch.empty((F,), dtype=torch.uint8).pin_memory()
        p = lpdec.make_params(mu=MU, rho=RHO, eps=args.eps, max_iter=ITERS, state=args.state, schedule=args.schedule)
        sp = int(stream.cuda_stream)

        def host_step():
            lpdec.lpdec_decode_host(C.handle, F, llr_pin.data_ptr(), p, x_pin.data_ptr(), b_pin.data_ptr(),
                                    i_pin.data_ptr(), c_pin.data_ptr(), sp)

        host_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            host_step()
        barrier()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, dev)
        line["e2e"] = {"value": ws * F * code.k_design / e2e_s, "unit": UNIT,
                       "h2d_bytes_per_step": F * code.n * 4,
                       "d2h_bytes_per_step": F * code.n * 4 + F * code.n + F * 5,
                       "ms_per_step": 1000 * e2e_s}

    if rank == 0:
        line["cpu_baseline"] = oracle_sample(code, llr_h, args.cpu_seconds, args.eps)
        print(json.dumps(line), flush=True)
    C.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()

"""Benchmark: subdomains bounded and clipped per second on GB300.

One step = one Clip-and-Verify bounding round (cv_bound_batch: constraint rows, pre-check,
relaxed clipping, re-concretisation, complete clipping, spec back-substitution) over one batch of
synthetic subdomains of the 784->256x6->10 ReLU MLP workload (4096 subdomains, 1-4 split
constraints each, 9 margin rows, 10 coordinate-ascent sweeps).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference] [--precision fp32|bf16x8]

--impl reference times the FP64 CPU oracle on the host cores (the slow reference program).
Under torchrun every rank bounds its own batch (weak scaling, no data-path collective)."""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CONFIG = "mlp784x256"
# lane operations per coordinate and row step of Algorithm 1 (a' and the breakpoint 3, the weight 1,
# the slope update 3, the crossing test and bookkeeping 3): the count of the benchmark table
CC_OPS_PER_COORD = 10
# DRAM bytes (read + write) of complete clipping's main launch per executed row step, from one ncu
# capture of the kernel on this workload at B = 1024 (19.675 MB over 1,717,951 row steps); the
# launch's traffic grows with its row steps, so the timed launch's is this times its row steps
CC_DRAM_BYTES_PER_ROW_STEP = 19.675e6 / 1717951


def workload_desc(cfg, name=CONFIG):
    d = cfg["dims"]
    return (f"{name}: ReLU MLP {d[0]}->{d[1]}x{len(d) - 2}->{d[-1]} He-normal seed 0; box eps={cfg['eps']} around "
            f"U[0,1]^{d[0]} clipped to [0,1]; B={cfg['B']} subdomains with {cfg['kmin']}-{cfg['kmax']} ReLU split "
            f"constraints each; 9 margin spec rows; {RELAXED_DESC[cfg['relaxed']]} + complete clipping "
            f"({cfg['sweeps']} sweeps) on every still-unstable cached neuron")


RELAXED_DESC = {0: "no relaxed clipping", 1: "relaxed clipping",
                2: "sequential relaxed clipping (Algorithm 3)",
                3: "sequential relaxed clipping in the constraint-importance order"}


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--precision", default="bf16x8", choices=["fp32", "bf16x8"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--config", default=CONFIG,
                   choices=["mlp784x256", "mlp5x50", "cnn3x32", "mlp784x1024", "mlp784x512x8", "bab_loop"],
                   help="workload (default: the metric's workload, with the others nested in its line)")
    p.add_argument("--full-stress", action="store_true",
                   help="with --config mlp784x512x8: its own line at the full 65,536 subdomains")
    p.add_argument("--no-other-configs", action="store_true",
                   help="only the metric's workload (no nested lines for the other configurations)")
    p.add_argument("--relaxed", type=int, default=None, choices=[1, 2, 3],
                   help="relaxed clipping: 1 parallel (Algorithm 2, the workload's), 2 sequential (Algorithm 3), "
                        "3 sequential in the constraint-importance order")
    p.add_argument("--activation-bab", action="store_true",
                   help="time the activation-BaB split (cv_activation_split) and top-20 targets (cv_select_targets)")
    p.add_argument("--spec-clip", action="store_true",
                   help="time complete clipping of the spec rows' final planes (cv_spec_clip) after a round")
    p.add_argument("--input-bab", action="store_true",
                   help="time the input-BaB split step (cv_input_split) on the workload's bounded batch instead")
    p.add_argument("--no-autotune", action="store_true",
                   help="keep complete clipping's default work-item sizes instead of tuning them first")
    p.add_argument("--subdomains", type=int, default=0,
                   help="smaller batch for profiler captures (default: the workload's own batch)")
    return p.parse_args()


# ---------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "50"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # the timed region is short: start it only once the sampler has written its first sample
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.proc.poll() is None and os.path.getsize(self.path) == 0:
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), hw=parts[5], hwt=parts[6], swt=parts[7],
                                 swp=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = []
        for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                          ("swp", "sw_power_cap")):
            if any(r[key].lower().startswith("active") for r in rows):
                reasons.append(name)
        return dict(sm_mhz=statistics.median(r["sm"] for r in rows), sm_max_mhz=max(r["smax"] for r in rows),
                    reasons=reasons, samples=len(rows))


# ---------------------------------------------------------------- oracle timing
def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_sample_rate(cfg, n_sub, offset=0, threads=None):
    """Time the FP64 oracle on n_sub subdomains of the workload with all host threads.  The sample is
    evenly spaced over the batch the GPU arm bounds (rank 0's split draws of all B subdomains),
    starting at `offset`, so that it has the batch's mix of row counts (a subdomain whose rows the
    pre-check drops costs almost nothing, one with four active rows the most)."""
    import numpy as np
    from oracle import oracle as O
    from paper_2512_11087_gb300 import workloads as WL
    layers = WL.he_mlp(cfg["dims"], seed=0)
    net = O.Net(layers)
    lo0, hi0 = WL.box(cfg["dims"][0], cfg["eps"], seed=0, centre=cfg["centre"], clip01=cfg["clip01"])
    cache = O.make_cache(O.root_crown(net, lo0, hi0))
    B = cfg["B"]
    off_all, ids_all = WL.draw_splits(cache["ids"], B, cfg["kmin"], cfg["kmax"], seed=shard_seed(0))
    pick = (offset + (np.arange(n_sub) * B) // max(n_sub, 1)) % B
    counts = off_all[pick + 1] - off_all[pick]
    so = np.zeros(n_sub + 1, np.int32)
    so[1:] = np.cumsum(counts)
    si = np.concatenate([ids_all[off_all[b]:off_all[b + 1]] for b in pick]).astype(np.int32) if n_sub else \
        np.zeros(0, np.int32)
    lo, hi = WL.tile_box(lo0, hi0, n_sub)
    C, t = WL.margin_spec(cfg["dims"][-1])
    cores = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    O.bound_batch(net, cache, lo, hi, split_off=so, split_ids=si, C=C, t=t, relaxed=cfg["relaxed"],
                  sweeps=cfg["sweeps"], nthreads=cores)
    dt = time.perf_counter() - t0
    return n_sub / dt, dt, cores


def pick_sample(cfg, budget_s):
    """Subdomain count (at least 16) whose oracle run takes about budget_s seconds on all host threads."""
    rate, dt, cores = oracle_sample_rate(cfg, 16, offset=5)
    n = int(max(16, min(cfg["B"], rate * budget_s)))
    return n, cores


def run_reference(args, cfg, rank, world):
    if rank != 0:
        return
    # about 6 s of oracle work per step, less for long runs: the whole run stays within a few minutes
    n, cores = pick_sample(cfg, min(6.0, 150.0 / max(1, args.steps + args.warmup)))
    for w in range(args.warmup):
        oracle_sample_rate(cfg, n, offset=11 + w)
    total_dt, total_n = 0.0, 0
    for k in range(args.steps):
        rate, dt, cores = oracle_sample_rate(cfg, n, offset=k)
        total_dt += dt
        total_n += n
    value = total_n / total_dt
    line = dict(metric="subdomains bounded+clipped per second", value=value, unit="subdomains/s", n_gpus=args.gpus,
                steps=args.steps, warmup=args.warmup, ms_per_step=1e3 * total_dt / args.steps,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                impl="reference",
                config=dict(workload=workload_desc(cfg, args.config),
                            sample=f"{n} subdomains per step, evenly spaced over the batch"),
                cpu_baseline=dict(value=value, unit="subdomains/s", cores=cores, kind="oracle",
                                  sample=f"{n} subdomains of the workload's batch per step (evenly spaced), "
                                         f"FP64 C oracle, OpenMP"),
                e2e=dict(value=value, unit="subdomains/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- sharding across ranks
# Subdomains are independent: each rank bounds its own batch (its own split draws) and the only
# cross-rank step is the max of the timed region, outside the data path.
def shard_seed(rank):
    """Seed of the split draws of a rank's batch."""
    return 1 + rank


def job_time_ms(local_ms, dist=None, device="cpu"):
    """The job's time: the max over ranks of each rank's timed region."""
    if dist is None:
        return float(local_ms)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, B, steps, total_ms):
    """Whole-job throughput: the subdomains of all ranks over the job's time."""
    return world * B * steps / (total_ms / 1e3)


# ---------------------------------------------------------------- input-BaB split step
def run_input_split(args, cfg):
    """Times cv_input_split (Algorithm 4's Domain_Filter + Batch_Split) on the outputs of one round of
    the workload (final planes included), the L2 flushed before every step; roofline against the
    measured HBM copy bandwidth with the bytes the step must move for this batch."""
    import numpy as np
    import torch
    from paper_2512_11087_gb300 import capi, engine as E, workloads as WL
    torch.cuda.set_device(0)
    dims, B, kmin, kmax = cfg["dims"], cfg["B"], cfg["kmin"], cfg["kmax"]
    layers = WL.he_mlp(dims, seed=0)
    lo0, hi0 = WL.box(dims[0], cfg["eps"], seed=0, centre=cfg["centre"], clip01=cfg["clip01"])
    net = E.Net(layers)
    net.build_cache(lo0, hi0)
    so, si = WL.draw_splits(net.read_cache()["ids"], B, kmin, kmax, seed=shard_seed(0))
    lo, hi = WL.tile_box(lo0, hi0, B)
    C, t = WL.margin_spec(dims[-1])
    m, n0 = C.shape[0], dims[0]
    rnd = E.Round(net, B, m, max_splits=kmax, relaxed=cfg["relaxed"], sweeps=cfg["sweeps"],
                  precision=capi.CV_PREC_BF16X8, want_final=True)
    d = E.to_dev
    out = rnd.run(d(lo), d(hi), d(C), d(t), split_off=d(so), split_ids=d(si))
    torch.cuda.synchronize()
    f32 = dict(dtype=torch.float32, device="cuda")
    lo2, hi2 = torch.empty(2 * B, n0, **f32), torch.empty(2 * B, n0, **f32)
    ro = torch.zeros(2 * B + 1, dtype=torch.int32, device="cuda")
    G, h = torch.empty(2 * B, n0, **f32), torch.empty(2 * B, **f32)
    par = torch.empty(2 * B, dtype=torch.int32, device="cuda")
    nch = torch.zeros(1, dtype=torch.int32, device="cuda")
    wsb = capi.cv_input_split_workspace(B)
    ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, **f32)
    stream = torch.cuda.current_stream()

    def step():
        capi.cv_input_split(B, n0, m, out["lo_clip"], out["hi_clip"], out["final_A"], out["final_c"], out["lower"],
                            out["verified"], out["infeasible"], lo2, hi2, ro, G, h, par, nch, ws, wsb, stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = sum(times) / len(times)
    # bytes the step must move: every parent's flags and spec lower bounds; per kept parent its box,
    # the planes of its unproven rows (the axis scores), two child boxes, and two inherited rows
    # when exactly one row is unproven; offsets and parent indices
    ver = out["verified"].cpu().numpy().astype(bool)
    inf = out["infeasible"].cpu().numpy().astype(bool)
    unp = (~(out["lower"].cpu().numpy() > 0)).sum(axis=1)
    kept = ~ver & ~inf
    K = int(kept.sum())
    byts = B * (2 + 4 * m) + int(np.sum(4 * n0 * unp[kept])) + K * (8 * n0 + 2 * 8 * n0 + 2 * 8) \
        + int(np.sum(kept & (unp == 1))) * 2 * (4 * n0 + 4)
    achieved = byts / (ms * 1e-3) / 1e9
    peak, peak_src = 6800.0, "fallback"
    try:
        peak, peak_src = float(json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                            "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except Exception:
        pass
    line = dict(metric="parent subdomains split per second (input BaB)", value=B / (ms * 1e-3), unit="subdomains/s",
                n_gpus=1, steps=args.steps, warmup=args.warmup, ms_per_step=ms, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload=workload_desc(cfg, args.config) + "; one round with final planes, then the split",
                            kept_parents=K, children=2 * K, parents_with_one_unproven_row=int(np.sum(kept & (unp == 1))),
                            l2="flushed (256 MiB write) before every timed step"),
                roofline=dict(bound="hbm", kernel="cv_input_split (k_split_mark, k_split_scan, k_split_write)",
                              achieved=achieved, peak=peak, unit="GB/s", frac=achieved / peak, traffic=None,
                              alg_bytes_per_step=byts, peak_source=peak_src),
                gpu_launches=3 * args.steps)
    print(json.dumps(line), flush=True)
    net.close()


# ---------------------------------------------------------------- complete clipping of the spec planes
def run_spec_clip(args, cfg):
    """Times cv_spec_clip (Algorithm 1 on the final plane of every unproven spec row) after a round of
    the workload: each step re-runs the round untimed (fresh bounds), flushes the L2, then times the
    spec clipping alone with CUDA events; reports the verified subdomains before and after."""
    import numpy as np
    import torch
    from paper_2512_11087_gb300 import capi, engine as E, workloads as WL
    torch.cuda.set_device(0)
    dims, B, kmin, kmax = cfg["dims"], cfg["B"], cfg["kmin"], cfg["kmax"]
    layers = WL.he_mlp(dims, seed=0)
    lo0, hi0 = WL.box(dims[0], cfg["eps"], seed=0, centre=cfg["centre"], clip01=cfg["clip01"])
    net = E.Net(layers)
    net.build_cache(lo0, hi0)
    so, si = WL.draw_splits(net.read_cache()["ids"], B, kmin, kmax, seed=shard_seed(0))
    lo, hi = WL.tile_box(lo0, hi0, B)
    C, t = WL.margin_spec(dims[-1])
    m = C.shape[0]
    rnd = E.Round(net, B, m, max_splits=kmax, relaxed=cfg["relaxed"], sweeps=cfg["sweeps"],
                  precision=capi.CV_PREC_BF16X8, want_final=True)
    d = E.to_dev
    args_ = (d(lo), d(hi), d(C), d(t))
    kw = dict(split_off=d(so), split_ids=d(si))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    times, before, after, raised = [], 0, 0, 0
    for k in range(max(args.warmup, 3) + args.steps):
        out = rnd.run(*args_, **kw)
        torch.cuda.synchronize()
        l0 = out["lower"].clone()
        v0 = int(out["verified"].sum().item())
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rnd.spec_clip(*args_, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= max(args.warmup, 3):
            times.append(e0.elapsed_time(e1))
        before, after = v0, int(out["verified"].sum().item())
        raised = int((out["lower"] > l0).sum().item())
    ms = sum(times) / len(times)
    line = dict(metric="subdomains spec-clipped per second", value=B / (ms * 1e-3), unit="subdomains/s", n_gpus=1,
                steps=args.steps, warmup=args.warmup, ms_per_step=ms, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload=workload_desc(cfg, args.config) + "; then complete clipping of the final "
                            "planes of the unproven spec rows (same sweeps)",
                            spec_rows=B * m, spec_rows_raised=raised, verified_before=before, verified_after=after,
                            l2="flushed (256 MiB write) before every timed step"))
    print(json.dumps(line), flush=True)
    net.close()


# ---------------------------------------------------------------- activation-BaB steps
def run_activation_bab(args, cfg):
    """Times the activation-BaB split step and the top-20 target selection on the outputs of one
    round of the workload (L2 flushed before every timed call); HBM roofline of the split with the
    bytes it must move for this batch."""
    import numpy as np
    import torch
    from paper_2512_11087_gb300 import capi, engine as E, workloads as WL
    torch.cuda.set_device(0)
    dims, B, kmin, kmax = cfg["dims"], cfg["B"], cfg["kmin"], cfg["kmax"]
    layers = WL.he_mlp(dims, seed=0)
    lo0, hi0 = WL.box(dims[0], cfg["eps"], seed=0, centre=cfg["centre"], clip01=cfg["clip01"])
    net = E.Net(layers)
    U = net.build_cache(lo0, hi0)
    so, si = WL.draw_splits(net.read_cache()["ids"], B, kmin, kmax, seed=shard_seed(0))
    lo, hi = WL.tile_box(lo0, hi0, B)
    C, t = WL.margin_spec(dims[-1])
    m, n0 = C.shape[0], dims[0]
    rnd = E.Round(net, B, m, max_splits=kmax, relaxed=cfg["relaxed"], sweeps=cfg["sweeps"],
                  precision=capi.CV_PREC_BF16X8)
    d = E.to_dev
    dso, dsi = d(so), d(si)
    out = rnd.run(d(lo), d(hi), d(C), d(t), split_off=dso, split_ids=dsi)
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn):
        ts = []
        for k in range(max(args.warmup, 3) + args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if k >= max(args.warmup, 3):
                ts.append(e0.elapsed_time(e1))
        return sum(ts) / len(ts), res

    # outputs allocated once: the timed calls are the library's alone
    f32 = dict(dtype=torch.float32, device="cuda")
    i32 = dict(dtype=torch.int32, device="cuda")
    so2, si2 = torch.zeros(2 * B + 1, **i32), torch.zeros(2 * (len(si) + B) + 1, **i32)
    lo2, hi2 = torch.empty(2 * B, n0, **f32), torch.empty(2 * B, n0, **f32)
    l2, u2 = torch.empty(2 * B, U, **f32), torch.empty(2 * B, U, **f32)
    par, br = torch.empty(2 * B, **i32), torch.empty(2 * B, **i32)
    stuck = torch.zeros(B, dtype=torch.uint8, device="cuda")
    nch = torch.zeros(1, **i32)
    wsa = capi.cv_activation_split_workspace(B)
    wa = torch.empty(max(wsa, 256), dtype=torch.uint8, device="cuda")
    toff, tids = torch.zeros(B + 1, **i32), torch.empty(B * U, **i32)
    wst = capi.cv_select_targets_workspace(B, U)
    wt = torch.empty(max(wst, 256), dtype=torch.uint8, device="cuda")
    split = lambda: capi.cv_activation_split(net.handle, net.cache, B, dso, dsi, out["lo_clip"], out["hi_clip"],
                                             out["l"], out["u"], out["mask"], None, out["verified"],
                                             out["infeasible"], so2, si2, lo2, hi2, l2, u2, par, br, stuck, nch, wa,
                                             wsa, stream)
    topk = lambda: capi.cv_select_targets(net.handle, net.cache, B, out["l"], out["u"], out["mask"], None, 20, toff,
                                          tids, wt, wst, stream)
    ms_split, _ = timed(split)
    ms_topk, _ = timed(topk)
    K = int(nch.item()) // 2
    kept = np.zeros(B, bool)
    kept[par[:2 * K].cpu().numpy()] = True
    nsp = np.diff(so)
    # bytes the split must move: every parent's flags; per kept parent its bounds and mask (the
    # scores), box and split codes (read once), and two children's boxes, bounds, split codes and
    # offsets, parent and branching slot
    kp = int(kept.sum())
    byts = B * 2 + kp * (9 * U + 8 * n0) + int(np.sum(nsp[kept])) * 4 \
        + 2 * kp * (8 * n0 + 8 * U + 12) + 2 * int(np.sum(nsp[kept] + 1)) * 4
    peak = 6800.0
    try:
        peak = float(json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                 "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        pass
    ach = byts / (ms_split * 1e-3) / 1e9
    line = dict(metric="parent subdomains branched per second (activation BaB)", value=B / (ms_split * 1e-3),
                unit="subdomains/s", n_gpus=1, steps=args.steps, warmup=args.warmup, ms_per_step=ms_split,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload=workload_desc(cfg, args.config) + "; one round, then the split and the "
                            "top-20 targets per hidden layer", cached_neurons=U, kept_parents=K,
                            topk_ms=ms_topk, topk_targets=int(toff[-1].item()),
                            l2="flushed (256 MiB write) before every timed call"),
                roofline=dict(bound="hbm", kernel="cv_activation_split (k_act_mark, k_scan2, k_act_write)",
                              achieved=ach, peak=peak, unit="GB/s", frac=ach / peak, traffic=None,
                              alg_bytes_per_step=byts),
                gpu_launches=3 * args.steps)
    print(json.dumps(line), flush=True)
    net.close()


# ---------------------------------------------------------------- GPU arm
# ---------------------------------------------------------------- the other workload configurations
# One entry per further configuration of the benchmark table: its own metric, timing (CUDA events,
# at least 3 warm-up steps, the L2 flushed before every timed step), the roofline of its dominant
# phase and the oracle on a bounded sample.  The default run nests them in the headline's JSON line.

def _timed(fn, steps, warmup, flush, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return ts


def _layers_of(cfg):
    from paper_2512_11087_gb300 import workloads as WL
    if "convs" in cfg:
        return WL.he_cnn(cfg["in_shape"], cfg["convs"], cfg["fcs"], seed=0)
    return WL.he_mlp(cfg["dims"], seed=0)


def _macs(dims):
    """Multiply-adds of one spec row's back-substitution through the (dense) layers."""
    return sum(dims[i] * dims[i - 1] for i in range(1, len(dims)))


def _oracle_rate(cfg, layers, lo0, hi0, n_sub, mk_batch, budget_s=5.0, spec_rows=None):
    """Subdomains per second of the FP64 oracle on at most n_sub subdomains of the configuration's
    batch (whole subdomains; the root cache is built first and not timed)."""
    import numpy as np
    from oracle import oracle as O
    net = O.Net(layers)
    cache = O.make_cache(O.root_crown(net, lo0, hi0))
    cores = os.cpu_count() or 1
    n = max(1, n_sub)
    kw = mk_batch(cache, n)
    t0 = time.perf_counter()
    O.bound_batch(net, cache, kw.pop("lo"), kw.pop("hi"), nthreads=cores, **kw)
    dt = time.perf_counter() - t0
    return dict(value=n / dt, unit="subdomains/s", cores=cores, kind="oracle",
                sample=f"{n} subdomains of the configuration's batch, FP64 C oracle ({dt:.1f} s on {cores} threads)")


def bench_mlp5x50(steps, warmup, flush, stream, peaks, cpu=True):
    """Configuration 1: 5->50x6->5, B = 256, 0-8 splits, one output-plane row per subdomain, relaxed
    clipping, one spec row; launch-bound, timed as replays of a captured graph (microseconds per round)."""
    import numpy as np
    import torch
    from paper_2512_11087_gb300 import engine as E, workloads as WL
    cfg = WL.CONFIGS["mlp5x50"]
    layers = _layers_of(cfg)
    lo0, hi0 = WL.box(cfg["dims"][0], cfg["eps"], seed=0, centre=cfg["centre"], clip01=cfg["clip01"])
    net = E.Net(layers)
    net.build_cache(lo0, hi0)
    ids = net.read_cache()["ids"]
    B = cfg["B"]
    C, t = WL.margin_spec(cfg["dims"][-1])
    C, t = C[:1], t[:1]
    d = E.to_dev
    # the spec row's root plane (a GPU round on the root box), shifted to cut every box
    r0 = E.Round(net, 1, 1, want_final=True)
    o0 = r0.run(d(lo0[None]), d(hi0[None]), d(C), d(t))
    a = o0["final_A"][0, 0].cpu().numpy()
    lo, hi = WL.tile_box(lo0, hi0, B)
    ro, G, h = WL.shifted_plane_rows(a, 0.0, lo, hi, B, seed=2)
    so, si = WL.draw_splits(ids, B, cfg["kmin"], cfg["kmax"], seed=1)
    rnd = E.Round(net, B, 1, max_splits=cfg["kmax"], max_rows=1, relaxed=1, sweeps=0)
    rnd.capture(d(lo), d(hi), d(C), d(t), split_off=d(so), split_ids=d(si), row_off=d(ro), G=d(G), h=d(h))
    ts = _timed(lambda: rnd.replay(stream), steps, warmup, flush, stream)
    ms = statistics.mean(ts)
    out = dict(config="mlp5x50: ReLU MLP 5->50x6->5, box width 0.1 around U[-1,1]^5, B=256, 0-8 splits, one "
                      "output-plane row per subdomain, relaxed clipping, spec row e0-e1; graph replays",
               metric="microseconds per round", value=1e3 * ms, unit="us", higher_is_better=False,
               subdomains_per_s=B / (ms / 1e3), steps=steps, warmup=warmup,
               roofline=dict(bound="launch", note="a few microseconds of work per kernel: launch latency, not a "
                                                   "throughput roofline"))
    if cpu:
        def mk(cache, n):
            so2, si2 = WL.draw_splits(cache["ids"], n, cfg["kmin"], cfg["kmax"], seed=1)
            l2, h2 = WL.tile_box(lo0, hi0, n)
            return dict(lo=l2, hi=h2, split_off=so2, split_ids=si2, row_off=ro[:n + 1], G=G[:n], h=h[:n], C=C, t=t,
                        relaxed=1, sweeps=0)
        out["cpu_baseline"] = _oracle_rate(cfg, layers, lo0, hi0, B, mk)
    capi_destroy_graph(rnd)
    net.close()
    return out


def capi_destroy_graph(rnd):
    from paper_2512_11087_gb300 import capi
    if getattr(rnd, "graph", None) is not None:
        capi.cv_graph_destroy(rnd.graph)
        rnd.graph = None


def _phase_roofline(phases, steps_cc, n0, dims, Bm, peaks, prec):
    """Roofline of the dominant phase of a round: complete clipping against the measured FP32 issue
    peak (about 10 lane operations per coordinate and row step), or the spec back-substitution
    (2 x rows x sum_i n_i n_(i-1) flops) against the FP32 FMA peak (CUDA cores) or the BF16 tensor
    peak divided by the 8 digit products of the split-precision path."""
    names = ["rows+relaxed", "reconcretize", "complete_clip", "backsubst"]
    k = max(range(4), key=lambda i: phases[i])
    if k == 2:
        ach = steps_cc * n0 * CC_OPS_PER_COORD / (phases[2] / 1e3) / 1e9
        pk = peaks["fma_lane_gops"]
        return dict(bound="alu", kernel="k_complete", phase=names[k], achieved=ach, peak=pk, unit="Gop/s",
                    frac=ach / pk, traffic=None, peak_source="measured (cv_fp32_fma_peak, lane FMAs/s)")
    if k == 3:
        fl = 2.0 * Bm * _macs(dims) / (phases[3] / 1e3) / 1e12
        if prec == 1:
            pk = peaks["bf16_tflops"] / 8.0
            src = "MEASURED_PEAKS bf16 burst / 8 digit products"
            return dict(bound="tensor", kernel="k_tc_layer", phase=names[k], achieved=fl, peak=pk, unit="TFLOP/s",
                        frac=fl / pk, traffic=None, peak_source=src)
        pk = 2.0 * peaks["fma_lane_gops"] / 1e3
        return dict(bound="alu", kernel="k_bwd_layer<float>", phase=names[k], achieved=fl, peak=pk,
                    unit="TFLOP/s", frac=fl / pk, traffic=None, peak_source="measured FP32 FMA peak x 2 flops")
    return dict(bound="hbm", phase=names[k], note="rows / re-concretisation dominate", achieved=None, peak=None)


def bench_cnn3x32(steps, warmup, flush, stream, peaks, cpu=True):
    """Configuration 3: the CIFAR-style CNN on 3x32x32, B = 2048, 1-16 splits, complete clipping (10
    sweeps) on the top-20 BaBSR targets per hidden layer chosen from a first round's bounds and
    weights; the timed round is one replay of its captured graph, on the split-BF16 tensor-core path
    (conv layers are dense Toeplitz matrices inside the library; K up to 4096 runs in passes)."""
    import numpy as np
    import torch
    from paper_2512_11087_gb300 import capi, engine as E, workloads as WL
    cfg = WL.CONFIGS["cnn3x32"]
    layers = _layers_of(cfg)
    n0 = int(np.prod(cfg["in_shape"]))
    lo0, hi0 = WL.box(n0, cfg["eps"], seed=0, centre=cfg["centre"], clip01=cfg["clip01"])
    net = E.Net(layers)
    U = net.build_cache(lo0, hi0)
    ids = net.read_cache()["ids"]
    B = cfg["B"]
    C, t = WL.margin_spec(layers[-1]["out_shape"][0])
    m = C.shape[0]
    so, si = WL.draw_splits(ids, B, cfg["kmin"], cfg["kmax"], seed=1)
    lo, hi = WL.tile_box(lo0, hi0, B)
    d = E.to_dev
    dlo, dhi, dC, dt_, dso, dsi = d(lo), d(hi), d(C), d(t), d(so), d(si)
    prec = capi.CV_PREC_BF16X8
    r0 = E.Round(net, B, m, max_splits=cfg["kmax"], relaxed=1, sweeps=0, precision=prec, want_weight=True)
    o0 = r0.run(dlo, dhi, dC, dt_, split_off=dso, split_ids=dsi)
    toff, tids = E.select_targets(net, o0["l"], o0["u"], o0["mask"], cfg["topk"], weight=o0["babsr_weight"])
    torch.cuda.synchronize()
    ntg = int(toff[-1].item())
    del r0
    rnd = E.Round(net, B, m, max_splits=cfg["kmax"], relaxed=1, sweeps=cfg["sweeps"], precision=prec)
    rnd.enable_timer()
    rnd.run(dlo, dhi, dC, dt_, split_off=dso, split_ids=dsi, tgt_off=toff, tgt_ids=tids)
    ph, _, steps_cc = capi.cv_timer_read(rnd.timer)
    cc_counts = dict(zip(["row_steps", "certified", "several_candidates", "widened", "fp32_decision_kept",
                          "over_candidate_limit"], rnd.cc_stats()))
    rnd.opt.timer = None
    rnd.capture(dlo, dhi, dC, dt_, split_off=dso, split_ids=dsi, tgt_off=toff, tgt_ids=tids)
    ts = _timed(lambda: rnd.replay(stream), steps, warmup, flush, stream)
    ms = statistics.mean(ts)
    dims = [n0] + [int(np.prod(l["out_shape"])) for l in layers]
    out = dict(config=f"cnn3x32: ReLU CNN 3x32x32 -> conv16 4x4 s2 p1 -> conv32 4x4 s2 p1 -> conv32 3x3 s1 p1 -> "
                      f"FC100 -> FC10, eps=2/255 around U[0,1] clipped to [0,1]; B={B}, 1-16 splits (uneven), "
                      f"9 margin rows, relaxed + complete clipping (10 sweeps) on the top-20 BaBSR targets per "
                      f"hidden layer ({ntg} in all); split-BF16 tensor-core path; one captured-graph replay "
                      f"per round",
               metric="subdomains bounded+clipped per second", value=B / (ms / 1e3), unit="subdomains/s",
               higher_is_better=True, ms_per_step=ms, steps=steps, warmup=warmup, cached_neurons=U,
               phase_ms=dict(zip(["rows+relaxed", "reconcretize", "complete_clip", "backsubst"],
                                 [round(x, 3) for x in ph])), cc_counters=cc_counts,
               roofline=_phase_roofline(ph, steps_cc, n0, dims, B * m, peaks, 1))
    if cpu:
        from oracle import oracle as O
        onet = O.Net(layers)

        def mk(cache, n):
            # the oracle's own top-20 targets, from its own round without complete clipping (not timed)
            so2, si2 = WL.draw_splits(cache["ids"], n, cfg["kmin"], cfg["kmax"], seed=1)
            l2, h2 = WL.tile_box(lo0, hi0, n)
            o = O.bound_batch(onet, cache, l2, h2, split_off=so2, split_ids=si2, C=C, t=t, relaxed=1, sweeps=0,
                              want_weight=True, nthreads=os.cpu_count() or 1)
            mask = np.where(o["l"] >= 0, 1, np.where(o["u"] <= 0, -1, 0)).astype(np.int8)
            to, ti = O.select_targets(O.layer_of_slots(onet, cache["ids"]), o["l"], o["u"], mask, o["babsr_weight"],
                                      cfg["topk"])
            return dict(lo=l2, hi=h2, split_off=so2, split_ids=si2, C=C, t=t, relaxed=1, sweeps=cfg["sweeps"],
                        tgt_off=to, tgt_ids=ti)
        out["cpu_baseline"] = _oracle_rate(cfg, layers, lo0, hi0, 4, mk)
    capi_destroy_graph(rnd)
    net.close()
    return out


def bench_alpha(steps, warmup, flush, stream, peaks, cpu=True, adam_steps=20):
    """Configuration 4: slope optimisation on 784->1024x4->10, B = 1024, 0-12 splits: one step is 20
    Adam iterations (cv_alpha_grad: forward keeping the layer products, reverse sweep of the adjoint;
    cv_alpha_adam) on the bounds, box and masks of a round, with the forward and reverse contractions
    on tensor cores (split-BF16, 1024-wide layers in two K passes); the FP32 CUDA-core path is timed
    beside it."""
    import numpy as np
    import torch
    from paper_2512_11087_gb300 import capi, engine as E, workloads as WL
    cfg = WL.CONFIGS["mlp784x1024"]
    dims = cfg["dims"]
    layers = _layers_of(cfg)
    lo0, hi0 = WL.box(dims[0], cfg["eps"], seed=0, centre=cfg["centre"], clip01=cfg["clip01"])
    net = E.Net(layers)
    U = net.build_cache(lo0, hi0)
    ids = net.read_cache()["ids"]
    B = cfg["B"]
    C, t = WL.margin_spec(dims[-1])
    m = C.shape[0]
    so, si = WL.draw_splits(ids, B, cfg["kmin"], cfg["kmax"], seed=1)
    lo, hi = WL.tile_box(lo0, hi0, B)
    d = E.to_dev
    rnd = E.Round(net, B, m, max_splits=cfg["kmax"], relaxed=1, sweeps=0)
    o = rnd.run(d(lo), d(hi), d(C), d(t), split_off=d(so), split_ids=d(si))
    st = E.AlphaState(net, o["lo_clip"], o["hi_clip"], o["l"], o["u"], o["mask"], d(C), d(t))
    H = net.H
    alpha = torch.ones(B, m, H, dtype=torch.float32, device="cuda")
    m1, m2 = torch.zeros_like(alpha), torch.zeros_like(alpha)
    lower = torch.empty(B, m, dtype=torch.float32, device="cuda")
    grad = torch.empty_like(alpha)
    a0 = alpha.clone()
    res = {}
    for prec in (capi.CV_PREC_BF16X8, capi.CV_PREC_FP32):
        ai = capi.make_alpha_in(B, m, st.lo, st.hi, st.l, st.u, st.mask, st.C, st.t, alpha, None, precision=prec)

        def step():
            alpha.copy_(a0)
            m1.zero_()
            m2.zero_()
            for it in range(1, adam_steps + 1):
                capi.cv_alpha_grad(net.handle, net.cache, ai, lower, grad, st.ws, st.ws_bytes, stream)
                capi.cv_alpha_adam(alpha, m1, m2, grad, it, 0.1 * 0.98 ** (it - 1), stream=stream)

        alpha.copy_(a0)
        capi.cv_alpha_grad(net.handle, net.cache, ai, lower, grad, st.ws, st.ws_bytes, stream)
        f0 = float(lower[torch.isfinite(lower)].double().mean())
        ts = _timed(step, steps, warmup, flush, stream)
        capi.cv_alpha_grad(net.handle, net.cache, ai, lower, grad, st.ws, st.ws_bytes, stream)
        f1 = float(lower[torch.isfinite(lower)].double().mean())
        res[prec] = (statistics.mean(ts), f0, f1)
    # the slopes and the split multipliers together (beta-CROWN form of the splits), tensor cores
    sign = E.split_signs(net, d(so), d(si), B)
    beta = torch.zeros_like(alpha)
    n1, n2 = torch.zeros_like(alpha), torch.zeros_like(alpha)
    gbeta = torch.empty_like(alpha)
    aib = capi.make_alpha_in(B, m, st.lo, st.hi, st.l, st.u, st.mask, st.C, st.t, alpha, None,
                             precision=capi.CV_PREC_BF16X8, beta=beta, split_sign=sign, grad_beta=gbeta)

    def step_b():
        alpha.copy_(a0)
        m1.zero_(); m2.zero_()
        beta.zero_(); n1.zero_(); n2.zero_()
        for it in range(1, adam_steps + 1):
            capi.cv_alpha_grad(net.handle, net.cache, aib, lower, grad, st.ws, st.ws_bytes, stream)
            lr_it = 0.1 * 0.98 ** (it - 1)
            capi.cv_alpha_adam(alpha, m1, m2, grad, it, lr_it, stream=stream)
            capi.cv_adam_range(beta, n1, n2, gbeta, it, lr_it, 0.0, float("inf"), stream=stream)

    tsb = _timed(step_b, steps, warmup, flush, stream)
    capi.cv_alpha_grad(net.handle, net.cache, aib, lower, grad, st.ws, st.ws_bytes, stream)
    fb1 = float(lower[torch.isfinite(lower)].double().mean())
    msb = statistics.mean(tsb)
    ms, f0, f1 = res[capi.CV_PREC_BF16X8]
    ms32, f032, f132 = res[capi.CV_PREC_FP32]
    # forward and reverse sweep: two contractions of B m rows through the layers per iteration
    fl = adam_steps * 2 * 2.0 * B * m * _macs(dims) / (ms / 1e3) / 1e12
    pk = peaks["bf16_tflops"] / 8.0
    out = dict(config="mlp784x1024: ReLU MLP 784->1024x4->10, eps=0.02 around U[0,1]^784 clipped to [0,1]; B=1024, "
                      "0-12 splits; per (subdomain, spec row, neuron) slopes, 20 Adam steps (lr 0.1, x0.98 per step) "
                      "through the hand-written adjoint; split-BF16 tensor-core contractions (forward and reverse)",
               metric="subdomains optimised per second (20 Adam steps each)", value=B / (ms / 1e3),
               unit="subdomains/s", higher_is_better=True, ms_per_step=ms, steps=steps, warmup=warmup,
               cached_neurons=U, mean_bound_before=f0, mean_bound_after=f1,
               fp32_path=dict(value=B / (ms32 / 1e3), ms_per_step=ms32, mean_bound_after=f132),
               with_split_multipliers=dict(value=B / (msb / 1e3), ms_per_step=msb, mean_bound_after=fb1,
                                           note="slopes and split multipliers optimised together"),
               roofline=dict(bound="tensor", kernel="cv_alpha_grad (k_tc_layer forward + adjoint contractions)",
                             achieved=fl, peak=pk, unit="TFLOP/s", frac=fl / pk, traffic=None,
                             peak_source="MEASURED_PEAKS bf16 burst / 8 digit products (FP32-equivalent flops)"))
    if cpu:
        from oracle import oracle as O
        onet = O.Net(layers)
        cache = O.make_cache(O.root_crown(onet, lo0, hi0))
        n = 1
        so2, si2 = WL.draw_splits(cache["ids"], n, cfg["kmin"], cfg["kmax"], seed=1)
        l2, h2 = WL.tile_box(lo0, hi0, n)
        orr = O.bound_batch(onet, cache, l2, h2, split_off=so2, split_ids=si2, C=C, t=t, relaxed=1, sweeps=0)
        hl, hu = cache["root_l"].copy(), cache["root_u"].copy()
        hl[cache["ids"]], hu[cache["ids"]] = orr["l"][0], orr["u"][0]
        hs = np.where(hl >= 0, 1, np.where(hu <= 0, -1, 0)).astype(np.int8)
        al = np.ones((m, onet.H))
        mm1, mm2 = np.zeros_like(al), np.zeros_like(al)
        t0 = time.perf_counter()
        for it in range(1, adam_steps + 1):
            _, g = O.alpha_grad(onet, hl, hu, hs, orr["lo_clip"][0], orr["hi_clip"][0], C, t, al)
            O.adam_step(al, mm1, mm2, g, it, 0.1 * 0.98 ** (it - 1))
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = dict(value=n / dt, unit="subdomains/s", cores=1, kind="oracle",
                                   sample=f"{n} subdomain, 20 oracle gradient + Adam steps in FP64 ({dt:.1f} s, one "
                                          f"thread)")
    net.close()
    return out


def bench_stress(steps, warmup, flush, stream, peaks, cpu=True, B=None):
    """Configuration 5: the BaB stress shape 784->512x8->10 at its full 65,536 subdomains with 0-24
    splits, relaxed + complete clipping (10 sweeps), split-precision (tensor-core) back-substitution.
    Complete clipping's work-item sizes are tuned first (cv_autotune_cc) on the batch's first 4096
    subdomains, untimed, and kept for the full batch."""
    import numpy as np
    import torch
    from paper_2512_11087_gb300 import capi, engine as E, workloads as WL
    cfg = WL.CONFIGS["mlp784x512x8"]
    dims = cfg["dims"]
    B = B or cfg["B"]
    layers = _layers_of(cfg)
    lo0, hi0 = WL.box(dims[0], cfg["eps"], seed=0, centre=cfg["centre"], clip01=cfg["clip01"])
    net = E.Net(layers)
    U = net.build_cache(lo0, hi0)
    ids = net.read_cache()["ids"]
    C, t = WL.margin_spec(dims[-1])
    m = C.shape[0]
    so, si = WL.draw_splits(ids, B, cfg["kmin"], cfg["kmax"], seed=1)
    lo, hi = WL.tile_box(lo0, hi0, B)
    d = E.to_dev
    dlo, dhi, dC, dt_, dso, dsi = d(lo), d(hi), d(C), d(t), d(so), d(si)
    nt = min(B, 4096)
    tune = E.Round(net, nt, m, max_splits=cfg["kmax"], relaxed=1, sweeps=cfg["sweeps"], precision=capi.CV_PREC_BF16X8)
    items, items_ms = tune.autotune(d(lo[:nt]), d(hi[:nt]), dC, dt_, split_off=d(so[:nt + 1]),
                                    split_ids=d(si[:int(so[nt])]))
    del tune
    torch.cuda.empty_cache()
    rnd = E.Round(net, B, m, max_splits=cfg["kmax"], relaxed=1, sweeps=cfg["sweeps"], precision=capi.CV_PREC_BF16X8)
    rnd.enable_timer()

    def step():
        rnd.run(dlo, dhi, dC, dt_, split_off=dso, split_ids=dsi, stream=stream)

    ts = _timed(step, steps, warmup, flush, stream)
    ph, _, steps_cc = capi.cv_timer_read(rnd.timer)
    cs = rnd.cc_stats()
    ms = statistics.mean(ts)
    out = dict(config=f"mlp784x512x8: ReLU MLP 784->512x8->10, eps=0.02 around U[0,1]^784 clipped to [0,1]; B={B} "
                      f"subdomains with 0-24 splits; 9 margin rows; relaxed + complete clipping (10 sweeps) on every "
                      f"still-unstable cached neuron; split-BF16 tensor-core back-substitution; item sizes "
                      f"{items} tuned on the first {nt} subdomains",
               metric="subdomains bounded+clipped per second", value=B / (ms / 1e3), unit="subdomains/s",
               higher_is_better=True, ms_per_step=ms, steps=steps, warmup=warmup, cached_neurons=U,
               phase_ms=dict(zip(["rows+relaxed", "reconcretize", "complete_clip", "backsubst"],
                                 [round(x, 2) for x in ph])),
               cc_row_steps=steps_cc, cc_certified=cs[1], cc_items=dict(sizes=items, tuned_on=nt),
               roofline=_phase_roofline(ph, steps_cc, dims[0], dims, B * m, peaks, 1))
    if cpu:
        def mk(cache, n):
            off_all, ids_all = WL.draw_splits(cache["ids"], cfg["B"], cfg["kmin"], cfg["kmax"], seed=1)
            pick = (np.arange(n) * cfg["B"]) // n
            counts = off_all[pick + 1] - off_all[pick]
            so2 = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
            si2 = np.concatenate([ids_all[off_all[b]:off_all[b + 1]] for b in pick]).astype(np.int32)
            l2, h2 = WL.tile_box(lo0, hi0, n)
            return dict(lo=l2, hi=h2, split_off=so2, split_ids=si2, C=C, t=t, relaxed=1, sweeps=cfg["sweeps"])
        out["cpu_baseline"] = _oracle_rate(cfg, layers, lo0, hi0, 16, mk)
    net.close()
    return out


def _bab_instance(cfg, seed=0):
    """The network, root box and spec rows of a configuration (margin rows e_0 - e_k)."""
    from paper_2512_11087_gb300 import workloads as WL
    layers = _layers_of(cfg)
    lo0, hi0 = WL.box(cfg["dims"][0], cfg["eps"], seed=seed, centre=cfg["centre"], clip01=cfg["clip01"])
    C, t = WL.margin_spec(cfg["dims"][-1])
    return layers, lo0, hi0, C, t


def bench_bab_loop(steps, warmup, flush, stream, peaks, cpu=True, batch=2048, top_k=20):
    """The activation-BaB loop of Algorithm 5 (cv_bab_*: pick-out, split with the BaBSR score and weight,
    top-20 targets, the round, filter, push) on two synthetic instances.
    (a) Throughput on the 784->256x6->10 network of the headline (eps 0.02 box in [0,1], 9 margin rows):
        from the root box, untimed iterations until the list holds a full batch of 2048 parents, then
        `steps` timed iterations of 4096 children each (split-BF16 rounds, 10 sweeps); subdomains bounded
        per second over the whole iteration (host read-backs included).
    (b) Domains visited to an answer on the 5->50x6->5 network (box width 0.1, row e_0 - e_1): the
        threshold clears the least of 65,536 sampled spec values by 25% or 50% of its gap to the root
        bound, and the loop runs until the list is empty or 200 iterations, for top-k 20, 0 and all."""
    import numpy as np
    import torch
    from paper_2512_11087_gb300 import capi, engine as E, workloads as WL
    d = E.to_dev
    res = {}
    # (a)
    cfg = WL.CONFIGS["mlp784x256"]
    layers, lo0, hi0, C, t = _bab_instance(cfg)
    net = E.Net(layers)
    U = net.build_cache(lo0, hi0)
    bab = E.ActivationBaB(net, C, t, batch=batch, top_k=top_k, capacity=1 << 16, max_depth=32, sweeps=cfg["sweeps"],
                          precision=capi.CV_PREC_BF16X8)
    st0 = bab.init(lo0[None].astype(np.float32), hi0[None].astype(np.float32), stream)
    visited, warm = st0["children"], 0
    while st0["remaining"] > 0:
        o = bab.step(stream)
        visited += o["children"]
        warm += 1
        if o["remaining"] >= batch or o["picked"] == 0:
            break
    for _ in range(max(warmup - 1, 0)):
        visited += bab.step(stream)["children"]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    tot, iters = bab.run(steps, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = e0.elapsed_time(e1)
    res["throughput"] = dict(instance="784->256x6->10, eps 0.02 box in [0,1], 9 margin rows, top-20 targets, 10 "
                                      "sweeps, split-BF16 rounds", cached_neurons=U, batch_parents=batch,
                             warmup_iterations=warm + max(warmup - 1, 0), timed_iterations=iters,
                             children_timed=tot["children"], subdomains_per_s=tot["children"] / (ms / 1e3),
                             ms_per_iteration=ms / max(iters, 1), wall_s=wall,
                             verified=tot["verified"], infeasible=tot["infeasible"], pushed=tot["pushed"],
                             list_size=tot["remaining"], domains_visited=visited + tot["children"])
    bab.close()
    net.close()
    torch.cuda.empty_cache()
    # (b)
    cfg1 = WL.CONFIGS["mlp5x50"]
    layers1, lo1, hi1, C1, _ = _bab_instance(cfg1)
    C1 = C1[:1]
    net1 = E.Net(layers1)
    U1 = net1.build_cache(lo1, hi1)
    r0 = E.Round(net1, 1, 1)
    f_root = float(r0.run(d(lo1[None]), d(hi1[None]), d(C1), d(np.zeros(1)))["lower"][0, 0].item())
    rng = np.random.default_rng(5)
    x = lo1 + (hi1 - lo1) * rng.uniform(size=(65536, lo1.size))
    for ly in layers1[:-1]:
        x = np.maximum(x @ np.asarray(ly["W"], np.float64).T + ly["b"], 0.0)
    y = x @ np.asarray(layers1[-1]["W"], np.float64).T + layers1[-1]["b"]
    f_samp = float(np.min(y @ C1[0]))
    runs = {}
    for frac, k in ((0.25, 20), (0.25, 0), (0.25, -1), (0.5, 20), (0.5, 0), (0.5, -1)):
        t1 = np.array([-f_samp + frac * (f_samp - f_root)])
        b1 = E.ActivationBaB(net1, C1, t1, batch=1024, top_k=k, capacity=1 << 18, max_depth=32, sweeps=10)
        torch.cuda.synchronize()
        e0.record(stream)
        s0 = b1.init(lo1[None].astype(np.float32), hi1[None].astype(np.float32), stream)
        tt, it = b1.run(200, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms1 = e0.elapsed_time(e1)
        dv = s0["children"] + tt["children"]
        unknown = tt["remaining"] > 0 or tt["stuck"] > 0 or tt["depth_limited"] > 0
        runs[f"margin{frac}_top{'all' if k < 0 else k}"] = dict(status="unknown" if unknown else "verified",
                                                                 iterations=it, threshold=float(t1[0]),
                                                domains_visited=dv, ms=ms1, subdomains_per_s=dv / (ms1 / 1e3),
                                                stuck=tt["stuck"], depth_limited=tt["depth_limited"],
                                                remaining=tt["remaining"])
        b1.close()
    res["to_answer"] = dict(instance="5->50x6->5, box width 0.1 around U[-1,1]^5, row e_0 - e_1, threshold 25% or "
                                     "50% of the root gap above the least of 65,536 samples", cached_neurons=U1,
                            root_lower=f_root, sampled_min=f_samp, runs=runs)
    net1.close()
    out = dict(config="activation-BaB loop (Algorithm 5): (a) throughput on 784->256x6->10, 2048 parents per "
                      "iteration; (b) domains visited to an answer on 5->50x6->5 for top-k 20 / 0 / all",
               metric="subdomains bounded per second in the activation-BaB loop", value=res["throughput"]
               ["subdomains_per_s"], unit="subdomains/s", higher_is_better=True,
               ms_per_step=res["throughput"]["ms_per_iteration"], steps=steps, warmup=warmup,
               domains_visited=res["to_answer"]["runs"]["margin0.5_top20"]["domains_visited"], detail=res)
    if cpu:
        from oracle import oracle as O
        onet = O.Net(layers)
        cache = O.make_cache(O.root_crown(onet, lo0, hi0))
        t0 = time.perf_counter()
        rec = O.activation_bab(onet, cache, lo0[None], hi0[None], C, t, batch=batch, top_k=top_k, capacity=1 << 16,
                               max_depth=32, max_iters=7, sweeps=cfg["sweeps"])
        dt = time.perf_counter() - t0
        n = sum(s["children"] for s in rec["iters"])
        out["cpu_baseline"] = dict(value=n / dt, unit="subdomains/s", cores=os.cpu_count() or 1, kind="oracle",
                                   sample=f"the oracle's loop on instance (a): Init and 7 iterations ({n} subdomains, "
                                          f"{dt:.1f} s)")
    return out


def measure_peaks():
    """The FP32 FMA issue peak (measured here) and the HBM / BF16 peaks measured on this GPU type
    (MEASURED_PEAKS.json)."""
    from paper_2512_11087_gb300 import capi
    fma, ms = capi.cv_fp32_fma_peak()
    p = dict(fma_lane_gops=fma / 1e9, fma_probe_ms=ms)
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        p.update(hbm_gbs=mp["hbm_gbs"], bf16_tflops=mp["bf16_tflops"], bf16_source="measured")
    except Exception:
        p.update(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_source="fallback")
    return p


OTHER = {"mlp5x50": bench_mlp5x50, "cnn3x32": bench_cnn3x32, "mlp784x1024": bench_alpha, "mlp784x512x8": bench_stress,
         "bab_loop": bench_bab_loop}


def run_other(args, names, cpu):
    """The further configurations; returns {name: entry}."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    peaks = measure_peaks()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    res = {}
    for n in names:
        steps = 2 if n == "mlp784x512x8" else max(2, min(args.steps, 5))
        res[n] = OTHER[n](steps, max(args.warmup, 3), flush, stream, peaks, cpu=cpu)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return res, peaks


def main():
    args = parse_args()
    from paper_2512_11087_gb300 import workloads as WL
    if args.config in OTHER and args.config != "mlp784x512x8" or (args.config == "mlp784x512x8" and args.full_stress):
        # a further configuration on its own line
        res, peaks = run_other(args, [args.config], cpu=not args.no_cpu_baseline)
        e = res[args.config]
        line = dict(metric=e["metric"], value=e["value"], unit=e["unit"], n_gpus=1, steps=e["steps"],
                    warmup=e["warmup"], ms_per_step=e.get("ms_per_step", e["value"] / 1e3 if e["unit"] == "us" else None),
                    higher_is_better=e["higher_is_better"], scaling="weak", vs_baseline=None, dtype="f32",
                    data="synthetic", config=dict(workload=e["config"]), roofline=e.get("roofline"), peaks=peaks)
        for k in ("cpu_baseline", "phase_ms", "subdomains_per_s", "domains_visited", "detail", "fp32_path",
                  "cc_items", "cc_counters", "with_split_multipliers"):
            if k in e:
                line[k] = e[k]
        print(json.dumps(line), flush=True)
        return
    cfg = WL.CONFIGS[args.config]
    if args.subdomains > 0:
        cfg = dict(cfg, B=args.subdomains)
    if args.relaxed is not None:
        cfg = dict(cfg, relaxed=args.relaxed)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, cfg, rank, world)
        return
    if args.input_bab:
        run_input_split(args, cfg)
        return
    if args.spec_clip:
        run_spec_clip(args, cfg)
        return
    if args.activation_bab:
        run_activation_bab(args, cfg)
        return

    import numpy as np
    import torch
    from paper_2512_11087_gb300 import capi, engine as E

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    dims = cfg["dims"]
    B, kmin, kmax = cfg["B"], cfg["kmin"], cfg["kmax"]
    layers = WL.he_mlp(dims, seed=0)
    lo0, hi0 = WL.box(dims[0], cfg["eps"], seed=0, centre=cfg["centre"], clip01=cfg["clip01"])
    net = E.Net(layers)
    U = net.build_cache(lo0, hi0)
    ids = net.read_cache()["ids"]
    so, si = WL.draw_splits(ids, B, kmin, kmax, seed=shard_seed(rank))
    lo, hi = WL.tile_box(lo0, hi0, B)
    C, t = WL.margin_spec(dims[-1])
    m = C.shape[0]
    prec = capi.CV_PREC_FP32 if args.precision == "fp32" else capi.CV_PREC_BF16X8
    rnd = E.Round(net, B, m, max_splits=kmax, relaxed=cfg["relaxed"], sweeps=cfg["sweeps"], precision=prec)
    timer = capi.cv_timer_create()
    rnd.opt.timer = timer
    d = E.to_dev
    dlo, dhi, dC, dt_, dso, dsi = d(lo), d(hi), d(C), d(t), d(so), d(si)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        rnd.run(dlo, dhi, dC, dt_, split_off=dso, split_ids=dsi)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    # complete clipping's work-item sizes, tuned on this batch before anything is timed
    items_tuned = cfg["sweeps"] > 0 and not args.no_autotune
    if items_tuned:
        items, _ = rnd.autotune(dlo, dhi, dC, dt_, split_off=dso, split_ids=dsi)
    else:
        items = capi.cv_cc_items_get(net.cache)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    if rank == 0:
        clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times, phases = [], []
    launches = steps_cc = 0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        ph, nl, ncc = capi.cv_timer_read(timer)
        phases.append(ph)
        launches += nl
        steps_cc = ncc
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop() if rank == 0 else None
    total_ms = job_time_ms(sum(times), dist, "cuda")
    value = job_value(world, B, args.steps, total_ms)

    # end to end through the same C-ABI call with host buffers (pinned), copies inside the timed region
    hlo, hhi = torch.from_numpy(lo).pin_memory(), torch.from_numpy(hi).pin_memory()
    hso, hsi = torch.from_numpy(so).pin_memory(), torch.from_numpy(si).pin_memory()
    hlower = torch.empty(B, m, dtype=torch.float32).pin_memory()
    hver = torch.empty(B, dtype=torch.uint8).pin_memory()
    h2d = sum(x.numel() * x.element_size() for x in (hlo, hhi, hso, hsi))
    d2h = hlower.numel() * 4 + hver.numel()
    e2e_ms = 0.0
    rnd.opt.timer = None
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dlo.copy_(hlo, non_blocking=True)
        dhi.copy_(hhi, non_blocking=True)
        dso.copy_(hso, non_blocking=True)
        dsi.copy_(hsi, non_blocking=True)
        out = rnd.run(dlo, dhi, dC, dt_, split_off=dso, split_ids=dsi)
        hlower.copy_(out["lower"], non_blocking=True)
        hver.copy_(out["verified"], non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_ms = job_time_ms(e2e_ms, dist, "cuda")
    e2e_value = job_value(world, B, args.steps, e2e_ms)
    # the per-round summary every rank contributes (least lower bound, verified / infeasible counts)
    job_summary = E.reduce_round_summary(*E.round_summary(out, stream), dist)

    # the plain FP32 GPU path on the same inputs: its throughput and the agreement of the bounds
    vs_fp32 = None
    if prec != capi.CV_PREC_FP32:
        r32 = E.Round(net, B, m, max_splits=kmax, relaxed=cfg["relaxed"], sweeps=cfg["sweeps"],
                      precision=capi.CV_PREC_FP32)
        for _ in range(2):
            r32.run(dlo, dhi, dC, dt_, split_off=dso, split_ids=dsi)
        t32 = 0.0
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r32.run(dlo, dhi, dC, dt_, split_off=dso, split_ids=dsi)
            e1.record(stream)
            torch.cuda.synchronize()
            t32 += e0.elapsed_time(e1)
        o32 = {k: v.clone() for k, v in r32.run(dlo, dhi, dC, dt_, split_off=dso, split_ids=dsi).items()}
        o16 = rnd.run(dlo, dhi, dC, dt_, split_off=dso, split_ids=dsi)
        torch.cuda.synchronize()
        feas = o32["infeasible"] == 0
        l32, l16 = o32["lower"][feas].double(), o16["lower"][feas].double()
        t32 = job_time_ms(t32, dist, "cuda")
        v32 = job_value(world, B, args.steps, t32)
        vs_fp32 = dict(value=v32, unit="subdomains/s", ms_per_step=t32 / args.steps, speedup=value / v32,
                       mean_lower=float(l16.mean()), mean_lower_fp32=float(l32.mean()),
                       mean_lower_rel_diff=float(abs(l16.mean() - l32.mean()) / l32.abs().mean()),
                       max_abs_lower_diff=float((l16 - l32).abs().max()),
                       verified_agree=float((o16["verified"] == o32["verified"]).double().mean()))
        del r32
    status = capi.cv_device_status(net.handle)

    # roofline of the dominant kernel (complete clipping, ALU bound): the benchmark table's count of
    # about 10 lane operations per coordinate and executed row step, against the measured FP32 issue
    # peak (lane FMAs per second of the probe kernel)
    ph_mean = [statistics.mean(p[i] for p in phases) for i in range(capi.N_PHASES)]
    n0 = dims[0]
    peaks = measure_peaks()
    alg_ops = steps_cc * n0 * CC_OPS_PER_COORD
    achieved = alg_ops / (ph_mean[2] / 1e3) / 1e9  # Gop/s
    peak = peaks["fma_lane_gops"]
    if rank == 0:
        line = dict(metric="subdomains bounded+clipped per second", value=value, unit="subdomains/s", n_gpus=world,
                    steps=args.steps, warmup=max(args.warmup, 3), ms_per_step=total_ms / args.steps,
                    higher_is_better=True, scaling="weak", vs_baseline=None,
                    dtype="f32" if args.precision == "fp32" else "bf16x8+f32", data="synthetic",
                    config=dict(workload=workload_desc(cfg, args.config), precision=args.precision, cached_neurons=U,
                                l2="flushed (256 MiB write) before every timed step",
                                cc_items=dict(sizes=items, tuned=items_tuned),
                                phase_ms=dict(zip(["rows+relaxed", "reconcretize", "complete_clip", "backsubst"],
                                                  [round(x, 4) for x in ph_mean]))),
                    roofline=dict(bound="alu", kernel="k_complete", achieved=achieved, peak=peak, unit="Gop/s",
                                  frac=achieved / peak,
                                  traffic=(CC_DRAM_BYTES_PER_ROW_STEP * steps_cc if args.config == CONFIG else None),
                                  traffic_source="ncu capture at B = 1024, scaled by the row steps",
                                  alg_ops_per_launch=alg_ops,
                                  ops_per_coordinate_and_row_step=CC_OPS_PER_COORD, cc_row_steps=steps_cc,
                                  peak_source="measured: cv_fp32_fma_peak lane FMAs/s"),
                    e2e=dict(value=e2e_value, unit="subdomains/s", h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h),
                    gpu_launches=launches, device_status=status, clocks=clk, peaks=peaks,
                    round_summary=job_summary)
        if vs_fp32 is not None:
            line["vs_fp32_path"] = vs_fp32
        if world == 1 and not args.no_cpu_baseline:
            n, cores = pick_sample(cfg, 20.0)  # the pick overestimates the cost: about 10-15 s
            rate, dt, cores = oracle_sample_rate(cfg, n, offset=3)
            n1 = max(4, n // 8)
            rate1, dt1, _ = oracle_sample_rate(cfg, n1, offset=7, threads=1)
            line["cpu_baseline"] = dict(value=rate, unit="subdomains/s", cores=cores, kind="oracle",
                                        cpu_model=cpu_model(), single_thread=rate1,
                                        sample=f"{n} subdomains of the benchmark batch (evenly spaced), FP64 C "
                                               f"oracle ({dt:.1f} s on {cores} threads); single thread: {n1} "
                                               f"subdomains in {dt1:.1f} s")
        if world == 1 and not args.no_other_configs and args.config == CONFIG and args.subdomains == 0:
            # the benchmark table's other configurations, each with its own metric and roofline
            rnd.ws = None
            del rnd
            torch.cuda.empty_cache()
            line["other_configs"], _ = run_other(args, ["mlp5x50", "cnn3x32", "mlp784x1024", "mlp784x512x8",
                                                        "bab_loop"],
                                                 cpu=not args.no_cpu_baseline)
        print(json.dumps(line), flush=True)
    capi.cv_timer_destroy(timer)
    net.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

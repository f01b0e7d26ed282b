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
ALG_OPS_BASE = 7  # per coordinate and row step of Algorithm 1, besides the argsort comparisons


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
    p.add_argument("--config", default=CONFIG, choices=["mlp784x256", "mlp784x512x8"],
                   help="workload (default: the metric's workload; mlp784x512x8 is the BaB stress shape)")
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
def oracle_sample_rate(cfg, n_sub, offset=0):
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
    cores = os.cpu_count() or 1
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
def main():
    args = parse_args()
    from paper_2512_11087_gb300 import workloads as WL
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

    # roofline of the dominant kernel (complete clipping, ALU bound)
    ph_mean = [statistics.mean(p[i] for p in phases) for i in range(capi.N_PHASES)]
    n0 = dims[0]
    alg_ops = steps_cc * n0 * (ALG_OPS_BASE + float(np.log2(n0)))
    achieved = alg_ops / (ph_mean[2] / 1e3) / 1e9  # Gop/s
    sm_clock = (clk or {}).get("sm_mhz") or 2070.0
    peak = 152 * 128 * sm_clock / 1e3  # Gop/s: 152 SMs x 128 FP32/INT32 lanes x clock
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
                                  frac=achieved / peak, traffic=None,
                                  alg_ops_per_launch=alg_ops, cc_row_steps=steps_cc),
                    e2e=dict(value=e2e_value, unit="subdomains/s", h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h),
                    gpu_launches=launches, device_status=status, clocks=clk)
        if vs_fp32 is not None:
            line["vs_fp32_path"] = vs_fp32
        if world == 1 and not args.no_cpu_baseline:
            n, cores = pick_sample(cfg, 20.0)  # the pick overestimates the cost: about 10-15 s
            rate, dt, cores = oracle_sample_rate(cfg, n, offset=3)
            line["cpu_baseline"] = dict(value=rate, unit="subdomains/s", cores=cores, kind="oracle",
                                        sample=f"{n} subdomains of the benchmark batch (evenly spaced), FP64 C "
                                               f"oracle ({dt:.1f} s on {cores} threads)")
        print(json.dumps(line), flush=True)
    capi.cv_timer_destroy(timer)
    net.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

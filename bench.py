"""Benchmark of the counter-guided search step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--paths all|none|mlp,lsq,cached,nbr,batch,large,tiny]

Workload of the headline line: the mid-size synthetic tuning space -- 12
parameters, 41.3M raw / 2.26M valid configurations materialised on the
device, 32 FP32 counters, depth-12 regression trees per counter fitted on a
2% sample with 2% Gaussian noise, k = 5 weighted draws per step.  A step is
one full pass of the hot path: bottleneck analysis and Delta-PC, prediction
of c_profile and of every unevaluated configuration, Eq. score,
normalisation, integer weights, k draws without replacement, evaluated-set
update.

The per-step inputs (the measured counters of each step's c_profile) come
from a recorded search over the synthetic performance function; the timed
steps replay them from device memory (``value``), and the end-to-end leg
replays them through the host API with its copies (``e2e``).  L2 is flushed
between timed steps (a 512 MB write outside the timed region, queued before
the step so that the device-timed region excludes host launch latency, which
``e2e`` includes).

``paths`` (same JSON line) measures the other forms of the step, each with
the roofline of its dominant kernel:
  mlp    the MLP counter model on the same space: trained on the GPU (Adam,
         2000 steps x 4096 rows) on a 5% profile sample with 2% noise; its
         counter RMSE and the tree model's on a 1% held-out sample against
         the noise-free synthetic counters; search steps scored by the fused
         tensor-core forward, and their speed against the tree path;
  lsq    the least-squares counter model (Section 3.3.1) fitted on the
         trees' sample: its held-out counter RMSE, and steps that predict the
         active counters and score in one kernel, or from cached columns;
  cached the headline search with the trees' leaf indices cached once;
  nbr    the headline search with steps restricted to c_profile's Hamming-1
         or Hamming-2 neighbourhood (latency of a step);
  batch  64 concurrent searches (8 per space) over 8 spaces of 3.5k-988k
         valid configurations, 6-14 parameters, K in {16, 32, 40}, depth-12
         trees, one graph launch per step, kernel shape from the autotuner;
  large  the 16-parameter space, 113M raw / 19.5M valid configurations
         decoded on the fly every step (nothing materialised), 40 counters,
         depth-12 trees, top-16 select;
  tiny   the 6-parameter block/tile space (1,824 configurations), 16
         counters, depth-8 trees fitted on a 10% sample: step latency.

With --gpus N > 1 (torchrun), every rank runs an independent search on its
own GPU (replicas; the step has no cross-GPU exchange).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from workloads.synth import SyntheticGPU, add_noise, sample_indices  # noqa: E402

METRIC = "configs scored/s per search step on 1 GB300; MLP vs tree path at equal counter RMSE"
WORKLOADS = {
    "mid_12p": dict(space="mid_12p", K=32, depth=12, frac=0.02, noise=0.02, k=5),
    "tiny_block_tile": dict(space=None, K=16, depth=8, frac=0.10, noise=0.0, k=5),
}
ALL_PATHS = ("chain", "mlp", "lsq", "cached", "table", "nbr", "batch", "large", "mlp_large", "tiny")
# DRAM bytes (read + write) per launch of each path's dominant kernel, from the ncu
# captures summarised under profiles/ (the kernels have not changed since)
PROFILED_TRAFFIC = {
    "k_bscore": 9.637e6,          # profiles/k_bscore_mid_12p.md
    "k_cscore_leaf": 36.564e6,    # profiles/cached_mid_12p.md
    "k_mlp_pipe": 18.748e6,       # profiles/k_mlp_pipe_mid_12p.md
    "k_bscore_otf": 20.228e6,     # profiles/k_bscore_otf_large_16p.md
    "k_step_fused": 9.763e6,      # profiles/k_step_fused_mid_12p.md
    "k_step_fused_otf": 378.7e6,  # profiles/k_step_fused_otf_large_16p.md
}
MLP_HIDDEN = 256


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def load_desc(wl):
    return W.space_tiny_block_tile() if wl["space"] is None else W.load_space(wl["space"])


def describe(name, wl, desc, n_valid):
    return {"workload": "%s: %d params, %d raw / %d valid configurations (materialised), "
                        "K=%d FP32 counters, depth-%d trees fit on a %g%% sample + %g%% noise, "
                        "k=%d weighted draws per step" % (
                            name, desc.n_params, desc.n_raw, n_valid, wl["K"], wl["depth"],
                            100 * wl["frac"], 100 * wl["noise"], wl["k"]),
            "n_valid": int(n_valid), "n_raw": int(desc.n_raw), "K": wl["K"],
            "depth": wl["depth"], "k": wl["k"], "select": "sample",
            "l2": "flushed between timed steps (512 MB write outside the timed region)"}


def alu_peak(props, pk):
    """Node visits/s at full issue: SMs x 4 SMSPs x 32 lanes x max SM clock
    over 4 instructions per visit (load, digit extract, compare, index)."""
    mhz = float(pk.get("sm_max_mhz", 2070.0))
    return props.multi_processor_count * 4 * 32 * mhz * 1e6 / 4.0, mhz


def mlp_flops_per_config(F, K):
    H = MLP_HIDDEN
    return 2.0 * (F * H + 2 * H * H + H * K)


# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
def combine_ranks(dist, t_total, t_e2e, scored, device):
    """Whole-job figures of independent replicas (one search per rank, seed =
    rank, no data exchanged): the slowest rank's device and end-to-end times,
    and the configurations scored by all ranks."""
    if dist is None:
        return t_total, t_e2e, float(scored)
    import torch
    tt = torch.tensor([t_total, t_e2e], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    cnt = torch.tensor([float(scored)], dtype=torch.float64, device=device)
    dist.all_reduce(cnt, op=dist.ReduceOp.SUM)
    return float(tt[0]), float(tt[1]), float(cnt[0])


def setup(kt, name, seed):
    wl = WORKLOADS[name]
    desc = load_desc(wl)
    roles = W.layout(wl["K"])
    gpu = SyntheticGPU(desc, roles, seed=0)
    sp = kt.Space.from_desc(desc)
    n_valid = sp.count()[0]
    valid = sp.valid_raw()
    digits = sp.valid_digits()
    samp = sample_indices(n_valid, wl["frac"], 0)
    Y = gpu.evaluate(digits[samp])[0]
    if wl["noise"]:
        Y = add_noise(Y, 0, wl["noise"])
    from paper_2102_05297_gb300 import fit
    model = fit.fit_model(digits[samp], Y, wl["depth"], desc.radices, roles)
    m = kt.Model(sp, model)
    return wl, desc, roles, gpu, sp, valid, digits, model, m, samp


def record(kt, sp, m, gpu, valid, digits, wl, seed, n_steps):
    """A search driven by the synthetic function; returns per step the
    c_profile, its measured counters and the batch runtimes."""
    s = kt.Search(sp, m, k=wl["k"], seed=seed)
    traj = []
    for _ in range(n_steps):
        cp = s.current()
        pos = int(np.searchsorted(valid, cp))
        c = gpu.evaluate(digits[pos:pos + 1])[0][0]
        raw, _ = s.step(c)
        rts = gpu.evaluate(digits[np.searchsorted(valid, raw)])[1]
        s.report(rts)
        traj.append((cp, c, rts))
    s.close()
    return traj


def timed_device_steps(kt, torch, s, traj, lo, hi, k, stream, flush):
    """Steps lo..hi-1 of a recorded trajectory on device buffers, each timed
    with CUDA events on the step's stream, L2 flushed before each.  With the
    search's per-kernel timing enabled the step's graph also records events
    between its kernels (kernel_ms); the step times are then slightly longer."""
    out_raw = torch.empty(k, dtype=torch.int64, device="cuda")
    out_sc = torch.empty(k, dtype=torch.float32, device="cuda")
    n_out = torch.empty(1, dtype=torch.int32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms, kern_ms, visits, scored, n_active = [], np.zeros(8), 0, 0, []
    for i in range(lo, hi):
        flush.zero_()
        s.set_profile(int(traj[i][0]))
        e0.record(stream)
        s.step_device(np.ascontiguousarray(traj[i][1], np.float32), k, out_raw.data_ptr(),
                      out_sc.data_ptr(), n_out.data_ptr(), stream)
        e1.record(stream)
        st = s.stats()                  # synchronises
        step_ms.append(e0.elapsed_time(e1))
        kern_ms += np.array(st.kernel_ms[:8])
        visits += st.n_scored * st.n_active * (st.depth + 1)
        scored += st.n_scored
        n_active.append(st.n_active)
    return step_ms, kern_ms, visits, scored, n_active


def untimed_device_steps(s, traj, lo, hi, k, bufs, stream):
    for i in range(lo, hi):
        s.set_profile(int(traj[i][0]))
        s.step_device(np.ascontiguousarray(traj[i][1], np.float32), k, *bufs, stream)


def run_ours(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2102_05297_gb300 import ktune as kt

    name = args.workload
    seed = rank
    wl, desc, roles, gpu, sp, valid, digits, model, m, samp = setup(kt, name, seed)
    K, Wu = args.steps, args.warmup
    traj = record(kt, sp, m, gpu, valid, digits, wl, seed, Wu + K)
    # a dedicated stream: steps on a non-default stream run as one captured CUDA graph
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    # written before every timed step: larger than L2, and long enough (~80 us)
    # that the step's host-side enqueue finishes before the device reaches the
    # step's start event, so the events bracket device work only
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device="cuda")

    # ---- device-resident timed steps -------------------------------------
    bufs = (torch.empty(wl["k"], dtype=torch.int64, device="cuda").data_ptr(),
            torch.empty(wl["k"], dtype=torch.float32, device="cuda").data_ptr(),
            torch.empty(1, dtype=torch.int32, device="cuda").data_ptr())
    # per-kernel times (a separate pass: events between the kernels lengthen the step)
    fused = args.fused
    s = kt.Search(sp, m, k=wl["k"], seed=seed, stream=stream)
    s.set_fused(fused)
    s.set_timing(True)
    untimed_device_steps(s, traj, 0, Wu, wl["k"], bufs, stream)
    _, kern_ms, visits, _, _ = timed_device_steps(kt, torch, s, traj, Wu, Wu + K, wl["k"],
                                                  stream, flush)
    # the dominant kernel: the fused step itself, or the score kernel of the chain
    score_s = (kern_ms[0] if fused else kern_ms[1]) / 1e3
    s.close()
    # the timed steps
    s = kt.Search(sp, m, k=wl["k"], seed=seed, stream=stream)
    s.set_fused(fused)
    untimed_device_steps(s, traj, 0, Wu, wl["k"], bufs, stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.25)                    # the sampler's first reading lands in the timed region
    step_ms, _, _, scored, _ = timed_device_steps(kt, torch, s, traj, Wu, Wu + K, wl["k"],
                                                  stream, flush)
    torch.cuda.synchronize()
    ck = clocks.stop()
    t_total = sum(step_ms) / 1e3
    s.close()

    # ---- end to end through the host API ---------------------------------
    s2 = kt.Search(sp, m, k=wl["k"], seed=seed, stream=stream)
    s2.set_fused(fused)
    e2e_ms = []
    for i in range(Wu + K):
        if i >= Wu:
            flush.zero_()
            torch.cuda.synchronize()
        t0 = time.perf_counter()
        raw, _ = s2.step(traj[i][1])
        t1 = time.perf_counter()
        s2.report(traj[i][2])
        if i >= Wu:
            e2e_ms.append((t1 - t0) * 1e3)
    s2.close()

    t_total, t_e2e, scored_all = combine_ranks(dist, t_total, sum(e2e_ms) / 1e3, scored, "cuda")

    pk, src = peaks()
    props = torch.cuda.get_device_properties(local)
    peak_visits, sm_mhz = alu_peak(props, pk)
    achieved = visits / score_s

    paths = {}
    if rank == 0 and world == 1:
        want = ALL_PATHS if args.paths == "all" else \
            () if args.paths == "none" else tuple(args.paths.split(","))
        ctx = dict(kt=kt, torch=torch, stream=stream, flush=flush, pk=pk, src=src, props=props,
                   steps=K, warmup=Wu, mlp_train_steps=args.mlp_train_steps)
        if "mlp" in want:
            paths["mlp"] = path_mlp(ctx, wl, desc, roles, gpu, sp, valid, digits, m, samp, traj,
                                    tree_ms=1e3 * t_total / K)
        if "lsq" in want:
            paths["lsq"] = path_lsq(ctx, wl, desc, roles, gpu, sp, valid, digits, m, samp, traj,
                                    tree_ms=1e3 * t_total / K)
        if "chain" in want and fused:
            paths["chain"] = path_chain(ctx, wl, sp, m, traj, fused_ms=1e3 * t_total / K)
        if "cached" in want:
            paths["cached"] = path_cached(ctx, wl, sp, m, traj, fused_ms=1e3 * t_total / K)
        if "table" in want:
            paths["table"] = path_table(ctx, wl, roles, gpu, sp, digits, traj,
                                        fused_ms=1e3 * t_total / K)
        if "nbr" in want:
            paths["nbr"] = path_nbr(ctx, wl, sp, m, traj, fused_ms=1e3 * t_total / K)
        if "batch" in want:
            paths["batch"] = path_batch(ctx)
        if "large" in want:
            paths["large"] = path_large(ctx)
        if "mlp_large" in want:
            paths["mlp_large"] = path_mlp_large(ctx)
        if "tiny" in want:
            paths["tiny"] = path_tiny(ctx)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    bytes_h2d = wl["K"] * 4
    bytes_d2h = wl["k"] * (8 + 4 + 8) + 4
    line = {
        "metric": METRIC,
        "value": scored_all / t_total,
        "unit": "configs/s",
        "n_gpus": world,
        "steps": K,
        "warmup": Wu,
        "ms_per_step": 1e3 * t_total / K,
        "steps_per_s": K / t_total,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded synthetic performance function; depth-12 trees fitted by the "
                "library's fitter)",
        "config": describe(name, wl, desc, len(valid)),
        "roofline": headline_roofline(fused, kern_ms, achieved, peak_visits, props, sm_mhz, src),
        "e2e": {"value": scored_all / t_e2e, "unit": "configs/s", "h2d_bytes_per_step": bytes_h2d,
                "d2h_bytes_per_step": bytes_d2h, "ms_per_step": 1e3 * t_e2e / K},
        "gpu_launches": (1 if fused else 4) * K,
        "clocks": ck,
    }
    if paths:
        line["paths"] = paths
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(name, model, traj[Wu][1])
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def headline_roofline(fused, kern_ms, achieved, peak_visits, props, sm_mhz, src):
    """Roofline of the headline step's dominant kernel: the whole step as one
    persistent kernel (its duration includes the weights and the draws), or
    the score kernel of the four-kernel chain; algorithmic work = node visits
    n_scored x n_active x (D + 1) per step."""
    r = {
        "bound": "alu",
        "achieved": achieved / 1e9,
        "peak": peak_visits / 1e9,
        "unit": "Gvisit/s",
        "frac": achieved / peak_visits,
        "traffic_unit": "bytes per launch (ncu dram read + write)",
        "peak_source": "derived: %d SMs x 4 SMSPs x 32 lanes x %.0f MHz (%s sm_max) / 4 "
                       "instructions per node visit" % (props.multi_processor_count, sm_mhz, src),
    }
    if fused:
        r["kernel"] = ("k_step_fused (the whole step: c_profile prediction, tree walk + Eq. score, "
                       "weights, draws; shape %d)" % fused)
        r["traffic"] = PROFILED_TRAFFIC.get("k_step_fused")
        tot = kern_ms[0]
        names = ("predict_cprofile", "summands_barrier", "walk", "barrier_wait", "weights",
                 "last_cta_slack", "draws")
        r["phase_share"] = {n: kern_ms[1 + i] / tot for i, n in enumerate(names)}
        # the walk phase alone (its share of the kernel's duration, from the
        # phase stamps): the part of the step the derived peak describes
        walk = r["phase_share"]["walk"]
        if walk > 0:
            r["walk_phase"] = {"achieved": achieved / walk / 1e9, "frac": achieved / walk / peak_visits,
                               "unit": "Gvisit/s"}
    else:
        tot = kern_ms[:4].sum()
        r["kernel"] = "k_bscore (tree walk + Eq. score)"
        r["traffic"] = PROFILED_TRAFFIC["k_bscore"]
        r["kernel_share"] = {"prepare": kern_ms[0] / tot, "score": kern_ms[1] / tot,
                             "weights": kern_ms[2] / tot, "select": kern_ms[3] / tot}
    return r


def path_chain(ctx, wl, sp, m, traj, fused_ms):
    """The headline search with four kernels per step (prepare, score,
    weights, select; one CUDA graph): step time, per-kernel shares and the
    score kernel's roofline, beside the fused step."""
    kt, torch, stream, flush = ctx["kt"], ctx["torch"], ctx["stream"], ctx["flush"]
    Wu, K = ctx["warmup"], min(ctx["steps"], 300)
    bufs = (torch.empty(wl["k"], dtype=torch.int64, device="cuda").data_ptr(),
            torch.empty(wl["k"], dtype=torch.float32, device="cuda").data_ptr(),
            torch.empty(1, dtype=torch.int32, device="cuda").data_ptr())
    s = kt.Search(sp, m, k=wl["k"], seed=0, stream=stream)
    s.set_fused(0)
    s.set_timing(True)
    untimed_device_steps(s, traj, 0, Wu, wl["k"], bufs, stream)
    _, kern_ms, visits, _, _ = timed_device_steps(kt, torch, s, traj, Wu, Wu + K, wl["k"], stream,
                                                  flush)
    s.close()
    s = kt.Search(sp, m, k=wl["k"], seed=0, stream=stream)
    s.set_fused(0)
    untimed_device_steps(s, traj, 0, Wu, wl["k"], bufs, stream)
    step_ms, _, _, scored, _ = timed_device_steps(kt, torch, s, traj, Wu, Wu + K, wl["k"], stream,
                                                  flush)
    s.close()
    t = sum(step_ms) / 1e3
    peak_visits, sm_mhz = alu_peak(ctx["props"], ctx["pk"])
    return {"workload": "the headline search, four kernels per step (one CUDA graph)",
            "value": scored / t, "unit": "configs/s", "ms_per_step": 1e3 * t / K, "steps": K,
            "fused_speedup": (1e3 * t / K) / fused_ms,
            "roofline": headline_roofline(0, kern_ms, visits / (kern_ms[1] / 1e3), peak_visits,
                                          ctx["props"], sm_mhz, ctx["src"])}


# ---------------------------------------------------------------------------
def rmse_norm(pred, truth, ranges):
    """Range-normalised counter RMSE over all counters and rows."""
    d = (np.asarray(pred, np.float64) - truth) / ranges
    return float(np.sqrt(np.mean(d * d)))


def path_mlp(ctx, wl, desc, roles, gpu, sp, valid, digits, tree_model, tree_samp, traj, tree_ms):
    """The MLP counter model on the headline space: GPU training, counter
    RMSE against the tree model, and search steps scored on the tensor cores."""
    kt, torch, stream, flush = ctx["kt"], ctx["torch"], ctx["stream"], ctx["flush"]
    from paper_2102_05297_gb300 import fit
    n = len(valid)
    Kc = wl["K"]
    ranges = gpu.counter_ranges()
    samp = sample_indices(n, 0.05, 11)
    Y = add_noise(gpu.evaluate(digits[samp])[0], 11, 0.02)
    rest = np.setdiff1d(np.setdiff1d(np.arange(n), samp), tree_samp)
    held = np.sort(np.random.default_rng(12).choice(rest, size=max(1, n // 100), replace=False))
    truth = gpu.evaluate(digits[held])[0].astype(np.float64)

    B, steps = 4096, ctx["mlp_train_steps"]
    mlp = kt.Mlp(sp, roles, ranges, max_batch=B, stream=stream)
    mlp.set_params(fit.init_mlp(mlp.F, Kc, seed=0))
    mlp.set_data(valid[samp], Y)
    rng = np.random.default_rng(13)
    idx = rng.integers(0, len(samp), size=steps * B).astype(np.int32)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    losses = mlp.train(idx, B)
    e1.record(stream)
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    fpc = mlp_flops_per_config(mlp.F, Kc)
    train_flops = 3.0 * fpc * B * steps

    rm_mlp = rmse_norm(mlp.predict(valid[held]), truth, ranges)
    pred_all = torch.empty((n, Kc), dtype=torch.float32, device="cuda")
    tm = tree_model
    tm.predict_device(0, n, pred_all.data_ptr(), stream)
    torch.cuda.synchronize()
    rm_tree = rmse_norm(pred_all[torch.from_numpy(held).cuda()].cpu().numpy(), truth, ranges)
    del pred_all

    model = kt.Model.from_mlp(mlp)
    s = kt.Search(sp, model, k=wl["k"], seed=0, stream=stream)
    s.set_timing(True)
    Wu = ctx["warmup"]
    n_steps = min(ctx["steps"], 100)
    bufs = (torch.empty(wl["k"], dtype=torch.int64, device="cuda").data_ptr(),
            torch.empty(wl["k"], dtype=torch.float32, device="cuda").data_ptr(),
            torch.empty(1, dtype=torch.int32, device="cuda").data_ptr())
    untimed_device_steps(s, traj, 0, Wu, wl["k"], bufs, stream)
    torch.cuda.synchronize()
    step_ms, kern_ms, _, scored, _ = timed_device_steps(kt, torch, s, traj, Wu,
                                                        min(len(traj), Wu + n_steps), wl["k"],
                                                        stream, flush)
    s.close()
    # the same search with cached predictions (the network predicts TS once)
    sc = kt.Search(sp, model, k=wl["k"], seed=0, stream=stream)
    torch.cuda.synchronize()
    tf = time.perf_counter()
    sc.set_cached(True)
    fill_ms = 1e3 * (time.perf_counter() - tf)
    untimed_device_steps(sc, traj, 0, Wu, wl["k"], bufs, stream)
    c_ms, _, _, c_scored, _ = timed_device_steps(kt, torch, sc, traj, Wu,
                                                 min(len(traj), Wu + n_steps), wl["k"], stream, flush)
    sc.close()
    model.close()
    mlp.close()
    t = sum(step_ms) / 1e3
    ns = len(step_ms)
    score_s = kern_ms[1] / 1e3
    pk = ctx["pk"]
    peak = float(pk.get("bf16_tflops", 1933.0)) * 1e12
    ach = scored * fpc / score_s
    return {
        "workload": "MLP %d->256->256->256->%d (GELU, BF16 operands, FP32 accumulate) on the "
                    "mid_12p space; trained on the GPU with Adam, %d steps x %d rows, on a 5%% "
                    "profile sample (%d configurations) + 2%% noise" % (mlp.F, Kc, steps, B, len(samp)),
        "value": scored / t, "unit": "configs/s", "ms_per_step": 1e3 * t / ns,
        "steps_per_s": ns / t, "steps": ns,
        "counter_rmse": {"mlp": rm_mlp, "tree": rm_tree,
                         "definition": "range-normalised RMSE over all %d counters on a 1%% held-out "
                                       "sample (%d configurations) against the noise-free synthetic "
                                       "counters; trees: depth 12 on a 2%% sample" % (Kc, len(held))},
        "speedup_vs_tree": tree_ms / (1e3 * t / ns),
        "cached": {"ms_per_step": sum(c_ms) / len(c_ms), "fill_ms": fill_ms,
                   "value": c_scored / (sum(c_ms) / 1e3), "unit": "configs/s",
                   "speedup_vs_tree_fused": tree_ms / (sum(c_ms) / len(c_ms))},
        "train": {"ms": train_ms, "final_loss": float(losses[-1]), "first_loss": float(losses[0]),
                  "tflops": train_flops / (train_ms / 1e3) / 1e12,
                  "flops": "3 x forward (%d FLOP per row) per row" % fpc},
        "roofline": {"bound": "tensor", "kernel": "k_mlp_fwd<score> (fused forward + Eq. score)",
                     "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                     "frac": ach / peak, "traffic": PROFILED_TRAFFIC["k_mlp_pipe"],
                     "peak_source": "%s bf16 burst (cuBLAS GEMM)" % ctx["src"],
                     "flop_per_config": fpc,
                     "kernel_share": {"prepare": kern_ms[0] / kern_ms.sum(),
                                      "score": kern_ms[1] / kern_ms.sum(),
                                      "weights": kern_ms[2] / kern_ms.sum(),
                                      "select": kern_ms[3] / kern_ms.sum()}},
    }


def path_lsq(ctx, wl, desc, roles, gpu, sp, valid, digits, tree_model, tree_samp, traj, tree_ms):
    """The least-squares counter model (Section 3.3.1) on the headline space:
    fitted on the trees' profile sample, counter RMSE against the trees, and
    search steps that predict the active counters and score in one kernel
    (fused) or from cached prediction columns."""
    kt, torch, stream, flush = ctx["kt"], ctx["torch"], ctx["stream"], ctx["flush"]
    from paper_2102_05297_gb300 import fit
    n = len(valid)
    Kc = wl["K"]
    ranges = gpu.counter_ranges()
    Y = gpu.evaluate(digits[tree_samp])[0]
    if wl["noise"]:
        Y = add_noise(Y, 0, wl["noise"])
    t0 = time.perf_counter()
    lm = fit.fit_lsq(desc.values, digits[tree_samp], Y, roles)
    fit_s = time.perf_counter() - t0
    binary, regs, _ = fit.lsq_shape(desc.values)
    mreg, T = len(regs), lm["coef"].shape[2]
    model = kt.Model(sp, lm)
    rest = np.setdiff1d(np.arange(n), tree_samp)
    held = np.sort(np.random.default_rng(12).choice(rest, size=max(1, n // 100), replace=False))
    truth = gpu.evaluate(digits[held])[0].astype(np.float64)
    pred_all = torch.empty((n, Kc), dtype=torch.float32, device="cuda")
    hidx = torch.from_numpy(held).cuda()
    model.predict_device(0, n, pred_all.data_ptr(), stream)
    torch.cuda.synchronize()
    rm_lsq = rmse_norm(pred_all[hidx].cpu().numpy(), truth, ranges)
    tree_model.predict_device(0, n, pred_all.data_ptr(), stream)
    torch.cuda.synchronize()
    rm_tree = rmse_norm(pred_all[hidx].cpu().numpy(), truth, ranges)
    del pred_all

    Wu = ctx["warmup"]
    n_steps = min(ctx["steps"], 100)
    hi = min(len(traj), Wu + n_steps)
    bufs = (torch.empty(wl["k"], dtype=torch.int64, device="cuda").data_ptr(),
            torch.empty(wl["k"], dtype=torch.float32, device="cuda").data_ptr(),
            torch.empty(1, dtype=torch.int32, device="cuda").data_ptr())
    s = kt.Search(sp, model, k=wl["k"], seed=0, stream=stream)
    untimed_device_steps(s, traj, 0, Wu, wl["k"], bufs, stream)
    step_ms, _, _, scored, _ = timed_device_steps(kt, torch, s, traj, Wu, hi, wl["k"], stream, flush)
    s.close()
    s = kt.Search(sp, model, k=wl["k"], seed=0, stream=stream)
    s.set_timing(True)
    untimed_device_steps(s, traj, 0, Wu, wl["k"], bufs, stream)
    _, kern_ms, _, k_scored, nact = timed_device_steps(kt, torch, s, traj, Wu, hi, wl["k"], stream,
                                                       flush)
    s.close()
    sc = kt.Search(sp, model, k=wl["k"], seed=0, stream=stream)
    torch.cuda.synchronize()
    tf = time.perf_counter()
    sc.set_cached(True)
    fill_ms = 1e3 * (time.perf_counter() - tf)
    untimed_device_steps(sc, traj, 0, Wu, wl["k"], bufs, stream)
    c_ms, _, _, c_scored, _ = timed_device_steps(kt, torch, sc, traj, Wu, hi, wl["k"], stream, flush)
    sc.close()
    model.close()
    t = sum(step_ms) / 1e3
    ns = len(step_ms)
    # algorithmic FP32 operations per scored configuration: per active counter
    # the polynomial's T - 1 multiply-adds in Horner form (2 operations each)
    # and 5 for its Eq. score term (sub, add, div, mul, add)
    flop = sum(float(k_scored) / ns * a * (2.0 * (T - 1) + 5.0) for a in nact)
    ach = flop / (kern_ms[1] / 1e3)
    mhz = float(ctx["pk"].get("sm_max_mhz", 2070.0))
    peak = ctx["props"].multi_processor_count * 128 * 2 * mhz * 1e6
    return {
        "workload": "least-squares counter model on the mid_12p space: %d subspaces of the %d "
                    "two-valued parameters, %d regressors, T = %d terms per counter, fitted on "
                    "the trees' %.0f%% profile sample" % (1 << len(binary), len(binary), mreg, T,
                                                          100 * wl["frac"]),
        "value": scored / t, "unit": "configs/s", "ms_per_step": 1e3 * t / ns,
        "steps_per_s": ns / t, "steps": ns, "fit_s": fit_s,
        "counter_rmse": {"lsq": rm_lsq, "tree": rm_tree,
                         "definition": "range-normalised RMSE over all %d counters on a 1%% held-out "
                                       "sample (%d configurations) against the noise-free synthetic "
                                       "counters; both fitted on the same sample" % (Kc, len(held))},
        "speedup_vs_tree": tree_ms / (1e3 * t / ns),
        "cached": {"ms_per_step": sum(c_ms) / len(c_ms), "fill_ms": fill_ms,
                   "value": c_scored / (sum(c_ms) / 1e3), "unit": "configs/s"},
        "roofline": {"bound": "alu", "kernel": "k_lsq_score_s (prediction of the active counters "
                                               "+ Eq. score, subspace-sorted tiles)",
                     "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                     "frac": ach / peak, "traffic": PROFILED_TRAFFIC.get("k_lsq_score"),
                     "peak_source": "FP32 FMA issue: SMs x 128 lanes x 2 x %.0f MHz (max SM clock)"
                                    % mhz,
                     "flop_per_config": "active counters (mean %.2f) x (2(T - 1) + 5)"
                                        % np.mean(nact),
                     "kernel_share": {"prepare": kern_ms[0] / kern_ms.sum(),
                                      "score": kern_ms[1] / kern_ms.sum(),
                                      "weights": kern_ms[2] / kern_ms.sum(),
                                      "select": kern_ms[3] / kern_ms.sum()}},
    }


def path_nbr(ctx, wl, sp, m, traj, fused_ms):
    """The headline search with neighbourhood-restricted steps: each recorded
    c_profile's Hamming-1 and Hamming-2 neighbours only."""
    kt, torch, stream, flush = ctx["kt"], ctx["torch"], ctx["stream"], ctx["flush"]
    Wu, n_steps = ctx["warmup"], min(ctx["steps"], 100)
    k = wl["k"]
    bufs = (torch.empty(k, dtype=torch.int64, device="cuda").data_ptr(),
            torch.empty(k, dtype=torch.float32, device="cuda").data_ptr(),
            torch.empty(1, dtype=torch.int32, device="cuda").data_ptr())
    out = {"workload": "the headline search (mid_12p, depth-12 trees, K = 32, k = 5) with each "
                       "step restricted to the recorded c_profile's Hamming neighbourhood"}
    hi = min(len(traj), Wu + n_steps)
    for radius in (1, 2):
        s = kt.Search(sp, m, k=k, seed=0, stream=stream)
        s.set_neighbourhood(radius)
        untimed_device_steps(s, traj, 0, Wu, k, bufs, stream)
        step_ms, _, visits, scored, _ = timed_device_steps(kt, torch, s, traj, Wu, hi, k, stream, flush)
        s.close()
        ms = sum(step_ms) / len(step_ms)
        out["radius_%d" % radius] = {"ms_per_step": ms, "steps_per_s": 1e3 / ms,
                                     "candidates_per_step": scored / len(step_ms),
                                     "node_visits_per_step": visits / len(step_ms),
                                     "speedup_vs_whole_space_step": fused_ms / ms}
    return out


def path_cached(ctx, wl, sp, m, traj, fused_ms):
    """The headline search with cached predictions: the trees predict all of TS
    once; each step streams the active counters' columns (HBM-bound)."""
    kt, torch, stream, flush = ctx["kt"], ctx["torch"], ctx["stream"], ctx["flush"]
    Wu, n_steps = ctx["warmup"], ctx["steps"]
    k = wl["k"]
    bufs = (torch.empty(k, dtype=torch.int64, device="cuda").data_ptr(),
            torch.empty(k, dtype=torch.float32, device="cuda").data_ptr(),
            torch.empty(1, dtype=torch.int32, device="cuda").data_ptr())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s = kt.Search(sp, m, k=k, seed=0, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.set_cached(True)
    fill_ms = 1e3 * (time.perf_counter() - t0)
    untimed_device_steps(s, traj, 0, Wu, k, bufs, stream)
    step_ms, _, _, scored, _ = timed_device_steps(kt, torch, s, traj, Wu, Wu + n_steps, k, stream,
                                                  flush)
    s.close()
    s = kt.Search(sp, m, k=k, seed=0, stream=stream)
    s.set_cached(True)
    s.set_timing(True)
    untimed_device_steps(s, traj, 0, Wu, k, bufs, stream)
    _, kern_ms, _, _, nact = timed_device_steps(kt, torch, s, traj, Wu, Wu + n_steps, k, stream, flush)
    s.close()
    t = sum(step_ms) / 1e3
    ns = len(step_ms)
    # algorithmic bytes per scored configuration: a 2-byte cached leaf index per
    # active counter, 4 per score written, 1/8 per evaluated bit
    bytes_ = sum(float(scored) / ns * (2.0 * a + 4.125) for a in nact)
    ach = bytes_ / (kern_ms[1] / 1e3)
    peak = float(ctx["pk"].get("hbm_gbs", 6800.0)) * 1e9
    return {
        "workload": "the headline search with cached predictions (the leaf of every "
                    "configuration in each of the depth-12 trees cached once for all %d "
                    "configurations; each step streams the active counters' leaf columns and "
                    "looks up the step's per-leaf terms)" % (scored // ns),
        "value": scored / t, "unit": "configs/s", "ms_per_step": 1e3 * t / ns,
        "steps_per_s": ns / t, "steps": ns, "fill_ms": fill_ms,
        "speedup_vs_fused": fused_ms / (1e3 * t / ns),
        "roofline": {"bound": "hbm", "kernel": "k_cscore_leaf (Eq. score from cached leaf indices)",
                     "achieved": ach / 1e9, "peak": peak / 1e9, "unit": "GB/s", "frac": ach / peak,
                     "traffic": PROFILED_TRAFFIC["k_cscore_leaf"],
                     "peak_source": "%s STREAM-style copy" % ctx["src"],
                     "bytes_per_config": "2 x active counters (mean %.2f) + 4.125" % np.mean(nact),
                     "kernel_share": {"prepare": kern_ms[0] / kern_ms.sum(),
                                      "score": kern_ms[1] / kern_ms.sum(),
                                      "weights": kern_ms[2] / kern_ms.sum(),
                                      "select": kern_ms[3] / kern_ms.sum()}},
    }


def path_table(ctx, wl, roles, gpu, sp, digits, traj, fused_ms):
    """The headline search with the measured counters of every configuration
    as the model (model blob kind 2; the exact-counter experiment of Section
    4): each step streams the active counters' columns of the table."""
    kt, torch, stream, flush = ctx["kt"], ctx["torch"], ctx["stream"], ctx["flush"]
    Wu, n_steps = ctx["warmup"], ctx["steps"]
    k = wl["k"]
    table = np.ascontiguousarray(gpu.evaluate(digits)[0], np.float32)
    t0 = time.perf_counter()
    m = kt.Model(sp, {"kind": "table", "roles": roles, "table": table})
    load_ms = 1e3 * (time.perf_counter() - t0)
    bufs = (torch.empty(k, dtype=torch.int64, device="cuda").data_ptr(),
            torch.empty(k, dtype=torch.float32, device="cuda").data_ptr(),
            torch.empty(1, dtype=torch.int32, device="cuda").data_ptr())
    s = kt.Search(sp, m, k=k, seed=0, stream=stream)
    untimed_device_steps(s, traj, 0, Wu, k, bufs, stream)
    step_ms, _, _, scored, _ = timed_device_steps(kt, torch, s, traj, Wu, Wu + n_steps, k, stream,
                                                  flush)
    s.close()
    s = kt.Search(sp, m, k=k, seed=0, stream=stream)
    s.set_timing(True)
    untimed_device_steps(s, traj, 0, Wu, k, bufs, stream)
    _, kern_ms, _, _, nact = timed_device_steps(kt, torch, s, traj, Wu, Wu + n_steps, k, stream, flush)
    s.close()
    m.close()
    t = sum(step_ms) / 1e3
    ns = len(step_ms)
    # algorithmic bytes per scored configuration: 4 per active counter's
    # column entry, 4 per score written, 1/8 per evaluated bit
    bytes_ = sum(float(scored) / ns * (4.0 * a + 4.125) for a in nact)
    ach = bytes_ / (kern_ms[1] / 1e3)
    peak = float(ctx["pk"].get("hbm_gbs", 6800.0)) * 1e9
    tot = kern_ms[:4].sum()
    return {
        "workload": "the headline search over a table of the measured (noise-free synthetic) "
                    "counters of all %d configurations as the model" % (scored // ns),
        "value": scored / t, "unit": "configs/s", "ms_per_step": 1e3 * t / ns,
        "steps_per_s": ns / t, "steps": ns, "load_ms": load_ms,
        "speedup_vs_fused_trees": fused_ms / (1e3 * t / ns),
        "roofline": {"bound": "hbm", "kernel": "k_cscore (Eq. score from the table's columns)",
                     "achieved": ach / 1e9, "peak": peak / 1e9, "unit": "GB/s", "frac": ach / peak,
                     "traffic": None, "peak_source": "%s STREAM-style copy" % ctx["src"],
                     "bytes_per_config": "4 x active counters (mean %.2f) + 4.125" % np.mean(nact),
                     "kernel_share": {"prepare": kern_ms[0] / tot, "score": kern_ms[1] / tot,
                                      "weights": kern_ms[2] / tot, "select": kern_ms[3] / tot}},
    }


BATCH_SPACES = ["batch_%d" % i for i in range(8)]
BATCH_K = [16, 32, 40, 32, 16, 40, 32, 16]


def path_batch(ctx, per_space=8, depth=12, mlp_steps=200):
    kt, torch, stream = ctx["kt"], ctx["torch"], ctx["stream"]
    from workloads.trees import random_model
    from paper_2102_05297_gb300 import fit
    entries = []
    keep = []
    mlps = []
    for si, nm in enumerate(BATCH_SPACES):
        d = W.load_space(nm)
        roles = W.layout(BATCH_K[si])
        gpu = SyntheticGPU(d, roles, seed=si)
        sp = kt.Space.from_desc(d)
        valid = sp.valid_raw()
        dig = sp.valid_digits()
        if si % 2 == 0:      # even spaces: depth-12 trees
            m = kt.Model(sp, random_model(d.radices, roles, depth=depth, seed=100 + si))
        else:                # odd spaces: the MLP, briefly trained on a 5% profile sample
            mlp = kt.Mlp(sp, roles, gpu.counter_ranges(), max_batch=1024, stream=stream)
            mlp.set_params(fit.init_mlp(mlp.F, BATCH_K[si], seed=si))
            samp = sample_indices(len(valid), 0.05, si)
            mlp.set_data(valid[samp], add_noise(gpu.evaluate(dig[samp])[0], si, 0.02))
            mlp.train(np.random.default_rng(si).integers(0, len(samp), size=mlp_steps * 1024)
                      .astype(np.int32), 1024, return_losses=False)
            mlps.append(mlp)
            m = kt.Model.from_mlp(mlp)
        keep += [sp, m]
        for r in range(per_space):
            s = kt.Search(sp, m, k=5, seed=10 * si + r, search_id=r, stream=stream)
            entries.append((s, gpu, valid, dig))
    n_valid = [len(e[2]) for e in entries[::per_space]]

    def counters():
        out = []
        for s, gpu, valid, dig in entries:
            p = int(np.searchsorted(valid, s.current()))
            out.append(gpu.evaluate(dig[p:p + 1])[0][0])
        return out

    b = kt.Batch([e[0] for e in entries], stream=stream)
    c0 = counters()
    choice, ms = b.autotune(c0, reps=3)
    n_steps = min(ctx["steps"], 100)
    Wu = ctx["warmup"]
    # the counters of every step are precomputed from a recording so that
    # the timed loop holds only the batched steps
    seqs, cps = [], []
    for i in range(Wu + n_steps):
        c = counters()
        cps.append([e[0].current() for e in entries])
        res = b.step(c, 5)
        seqs.append(c)
        for (s, gpu, valid, dig), (raw, _) in zip(entries, res):
            s.report(gpu.evaluate(dig[np.searchsorted(valid, raw)])[1])
    b.close()
    for s, *_ in entries:
        s.close()
    # replay: fresh searches, same counters, same c_profiles (reports follow
    # the same runtimes, so the trajectory repeats exactly)
    entries2 = []
    for si, nm in enumerate(BATCH_SPACES):
        sp, m = keep[2 * si], keep[2 * si + 1]
        for r in range(per_space):
            entries2.append(kt.Search(sp, m, k=5, seed=10 * si + r, search_id=r, stream=stream))
    b = kt.Batch(entries2, stream=stream)
    b.autotune(c0, reps=1)
    scored, t_ms = 0, 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for i in range(Wu + n_steps):
        n_before = sum(len(e[2]) - s.evaluated() for s, e in zip(entries2, entries))
        e0.record(stream)
        res = b.step(seqs[i], 5)        # host outputs: synchronises
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= Wu:
            t_ms += e0.elapsed_time(e1)
            scored += n_before
        for s2, (s, gpu, valid, dig), (raw, _) in zip(entries2, entries, res):
            s2.report(gpu.evaluate(dig[np.searchsorted(valid, raw)])[1])
    b.close()
    for s in entries2:
        s.close()
    # the same searches stepped one at a time (one graph launch per search step)
    singles = []
    for si, nm in enumerate(BATCH_SPACES):
        sp, m = keep[2 * si], keep[2 * si + 1]
        for r in range(per_space):
            singles.append(kt.Search(sp, m, k=5, seed=10 * si + r, search_id=r, stream=stream))
    ob = (torch.empty(5, dtype=torch.int64, device="cuda"),
          torch.empty(5, dtype=torch.float32, device="cuda"),
          torch.empty(1, dtype=torch.int32, device="cuda"))
    t1_ms = 0.0
    for i in range(Wu + n_steps):
        for q, s1 in enumerate(singles):   # the c_profiles of the recorded trajectory
            s1.set_profile(cps[i][q])
        e0.record(stream)
        for q, s1 in enumerate(singles):
            s1.step_device(seqs[i][q], 5, ob[0].data_ptr(), ob[1].data_ptr(), ob[2].data_ptr(),
                           stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= Wu:
            t1_ms += e0.elapsed_time(e1)
    for s1 in singles:
        s1.close()
    thr, cpt, ipc = kt.Batch.variant(choice)
    t = t_ms / 1e3
    return {
        "workload": "%d searches (%d per space) over %d spaces of %s valid configurations, "
                    "K %s; even spaces scored by depth-%d random trees, odd spaces by the BF16 "
                    "MLP (%d Adam steps x 1024 rows on a 5%% sample); k=5 weighted draws; one "
                    "CUDA-graph launch per batched step" % (
                        len(entries), per_space, len(BATCH_SPACES),
                        "/".join(str(v) for v in n_valid), "/".join(str(k) for k in BATCH_K),
                        depth, mlp_steps),
        "value": scored / t, "unit": "configs/s", "ms_per_batch_step": t_ms / n_steps,
        "search_steps_per_s": len(entries) * n_steps / t, "steps": n_steps,
        "one_at_a_time_ms_per_batch_step": t1_ms / n_steps,
        "speedup_vs_one_at_a_time": t1_ms / t_ms,
        "autotune": {"choice": choice, "threads": thr, "configs_per_thread": cpt,
                     "items_per_cta": ipc, "candidates_ms": [float(x) for x in ms]},
        "timing": "CUDA events around ktune_batch_step, including its device-to-host copy of "
                  "the 64 searches' selections",
    }


def path_large(ctx, depth=12):
    kt, torch, stream, flush = ctx["kt"], ctx["torch"], ctx["stream"], ctx["flush"]
    from workloads.trees import random_model
    d = W.load_space("large_16p")
    roles = W.layout(40)
    model = random_model(d.radices, roles, depth=depth, seed=40)
    gpu = SyntheticGPU(d, roles, seed=0)
    sp = kt.Space.from_desc(d, flags=kt.KTUNE_ON_THE_FLY)
    n_valid, n_raw = sp.count()
    m = kt.Model(sp, model)
    k = 16
    n_steps = min(ctx["steps"], 50)
    Wu = ctx["warmup"]

    def dig_of(raw):
        out = np.zeros((len(raw), d.n_params), np.int64)
        for j, r in enumerate(raw):
            v = sp.decode(int(r))
            out[j] = [d.values[p].index(v[p]) for p in range(d.n_params)]
        return out

    rec = kt.Search(sp, m, k=k, seed=0, select=kt.KTUNE_SELECT_TOPK)
    traj = []
    for _ in range(Wu + n_steps):
        cp = rec.current()
        c = gpu.evaluate(dig_of([cp]))[0][0]
        raw, _ = rec.step(c)
        rec.report(gpu.evaluate(dig_of(raw))[1])
        traj.append((cp, c))
    rec.close()
    s = kt.Search(sp, m, k=k, seed=0, select=kt.KTUNE_SELECT_TOPK, stream=stream)
    s.set_timing(True)
    bufs = (torch.empty(k, dtype=torch.int64, device="cuda").data_ptr(),
            torch.empty(k, dtype=torch.float32, device="cuda").data_ptr(),
            torch.empty(1, dtype=torch.int32, device="cuda").data_ptr())
    untimed_device_steps(s, traj, 0, Wu, k, bufs, stream)
    torch.cuda.synchronize()
    step_ms, kern_ms, visits, scored, nact = timed_device_steps(kt, torch, s, traj, Wu,
                                                                Wu + n_steps, k, stream, flush)
    s.close()
    t = sum(step_ms) / 1e3
    peak, _ = alu_peak(ctx["props"], ctx["pk"])
    # the whole step is one persistent kernel (decode + filter, c_profile's
    # prediction, walk + Eq. score, top-k): its whole duration is the divisor
    ach = visits / (kern_ms[0] / 1e3)
    names = ("predict_cprofile_and_decode", "summands_barrier", "walk_and_cta_topk", None, None,
             "last_cta_slack", "select_topk")
    return {
        "workload": "large_16p on the fly: %d raw / %d valid configurations decoded every step "
                    "(none stored), K=40, depth-%d random trees, top-%d select" % (
                        n_raw, n_valid, depth, k),
        "value": scored / t, "unit": "configs/s", "ms_per_step": 1e3 * t / n_steps,
        "steps_per_s": n_steps / t, "steps": n_steps,
        "raw_decoded_per_s": n_raw * n_steps / t,
        "roofline": {"bound": "alu",
                     "kernel": "k_step_fused<on-the-fly> (the whole step: decode + filter, c_profile "
                               "prediction, walk + Eq. score, top-k)",
                     "achieved": ach / 1e9, "peak": peak / 1e9, "unit": "Gvisit/s",
                     "frac": ach / peak, "traffic": PROFILED_TRAFFIC.get("k_step_fused_otf"),
                     "mean_active_counters": float(np.mean(nact)),
                     "phase_share": {n: kern_ms[1 + i] / kern_ms[0] for i, n in enumerate(names) if n},
                     "walk_phase": {"achieved": visits / (kern_ms[3] / 1e3) / 1e9,
                                    "frac": visits / (kern_ms[3] / 1e3) / peak, "unit": "Gvisit/s"}},
    }


def path_mlp_large(ctx, n_fit=40000, k=16):
    """The MLP on the large space (16 parameters, 19.5M valid configurations,
    materialised here because the network reads packed digits), K = 40
    counters, 16 weighted draws per step (MLP searches take weighted draws
    only): GPU training, counter RMSE against depth-12 trees
    fitted on the same profile sample, and the step time of both models on
    the same recorded trajectory."""
    kt, torch, stream, flush = ctx["kt"], ctx["torch"], ctx["stream"], ctx["flush"]
    from paper_2102_05297_gb300 import fit
    d = W.load_space("large_16p")
    Kc = 40
    roles = W.layout(Kc)
    gpu = SyntheticGPU(d, roles, seed=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sp = kt.Space.from_desc(d)
    n = sp.count()[0]
    create_s = time.perf_counter() - t0
    valid = sp.valid_raw()
    digits = sp.valid_digits()
    samp = sample_indices(n, n_fit / n, 21)
    Y = add_noise(gpu.evaluate(digits[samp])[0], 21, 0.02)
    ranges = gpu.counter_ranges()
    t0 = time.perf_counter()
    tree_model = fit.fit_model(digits[samp], Y, 12, d.radices, roles)
    fit_s = time.perf_counter() - t0
    tm = kt.Model(sp, tree_model)
    rest = np.setdiff1d(np.arange(n), samp)
    held = np.sort(np.random.default_rng(22).choice(rest, size=max(1, n // 100), replace=False))
    truth = gpu.evaluate(digits[held])[0].astype(np.float64)
    # tree predictions of the held-out rows, by chunks of TS ordinals
    chunk = 1 << 21
    buf = torch.empty((chunk, Kc), dtype=torch.float32, device="cuda")
    tree_pred = np.empty((len(held), Kc), np.float32)
    for lo in range(0, n, chunk):
        cnt = min(chunk, n - lo)
        tm.predict_device(lo, cnt, buf.data_ptr(), stream)
        sel = held[(held >= lo) & (held < lo + cnt)]
        if len(sel):
            rows = torch.from_numpy(sel - lo).cuda()
            tree_pred[np.searchsorted(held, sel)] = buf[rows].cpu().numpy()
    torch.cuda.synchronize()
    del buf
    rm_tree = rmse_norm(tree_pred, truth, ranges)

    B, steps = 4096, ctx["mlp_train_steps"]
    mlp = kt.Mlp(sp, roles, ranges, max_batch=B, stream=stream)
    mlp.set_params(fit.init_mlp(mlp.F, Kc, seed=0))
    mlp.set_data(valid[samp], Y)
    idx = np.random.default_rng(23).integers(0, len(samp), size=steps * B).astype(np.int32)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    losses = mlp.train(idx, B)
    e1.record(stream)
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    rm_mlp = rmse_norm(mlp.predict(valid[held]), truth, ranges)

    # a trajectory recorded with the trees (c_profile, its counters, the batch runtimes)
    Wu = ctx["warmup"]
    n_steps = min(ctx["steps"], 20)
    rec = kt.Search(sp, tm, k=k, seed=0)
    traj = []
    for _ in range(Wu + n_steps):
        cp = rec.current()
        pos = int(np.searchsorted(valid, cp))
        c = gpu.evaluate(digits[pos:pos + 1])[0][0]
        raw, _ = rec.step(c)
        rec.report(gpu.evaluate(digits[np.searchsorted(valid, raw)])[1])
        traj.append((cp, c))
    rec.close()
    bufs = (torch.empty(k, dtype=torch.int64, device="cuda").data_ptr(),
            torch.empty(k, dtype=torch.float32, device="cuda").data_ptr(),
            torch.empty(1, dtype=torch.int32, device="cuda").data_ptr())

    def timed(model, timing):
        s = kt.Search(sp, model, k=k, seed=0, stream=stream)
        s.set_timing(timing)
        untimed_device_steps(s, traj, 0, Wu, k, bufs, stream)
        torch.cuda.synchronize()
        out = timed_device_steps(kt, torch, s, traj, Wu, Wu + n_steps, k, stream, flush)
        s.close()
        return out

    t_step, _, _, t_scored, _ = timed(tm, False)
    model = kt.Model.from_mlp(mlp)
    _, kern_ms, _, _, _ = timed(model, True)
    m_step, _, _, m_scored, _ = timed(model, False)
    model.close()
    tm.close()
    mlp.close()
    sp.close()
    tree_ms = sum(t_step) / len(t_step)
    mlp_ms = sum(m_step) / len(m_step)
    fpc = mlp_flops_per_config(mlp.F, Kc)
    pk = ctx["pk"]
    peak = float(pk.get("bf16_tflops", 1933.0)) * 1e12
    ach = m_scored * fpc / (kern_ms[1] / 1e3)
    return {
        "workload": "MLP %d->256->256->256->%d on the large_16p space materialised (%d valid of %d "
                    "raw, created in %.2f s), %d weighted draws per step; trees (depth 12) and MLP (Adam, %d "
                    "steps x %d rows) fitted on the same %d-configuration profile sample + 2%% "
                    "noise (trees fitted on the host in %.1f s)" % (
                        mlp.F, Kc, n, d.n_raw, create_s, k, steps, B, len(samp), fit_s),
        "value": m_scored / (sum(m_step) / 1e3), "unit": "configs/s", "ms_per_step": mlp_ms,
        "steps": len(m_step),
        "tree": {"value": t_scored / (sum(t_step) / 1e3), "unit": "configs/s", "ms_per_step": tree_ms},
        "counter_rmse": {"mlp": rm_mlp, "tree": rm_tree,
                         "definition": "range-normalised RMSE over all %d counters on a 1%% held-out "
                                       "sample (%d configurations) against the noise-free synthetic "
                                       "counters" % (Kc, len(held))},
        "speedup_vs_tree": tree_ms / mlp_ms,
        "train": {"ms": train_ms, "final_loss": float(losses[-1]), "first_loss": float(losses[0]),
                  "tflops": 3.0 * fpc * B * steps / (train_ms / 1e3) / 1e12},
        "roofline": {"bound": "tensor", "kernel": "k_mlp_fwd<score> (fused forward + Eq. score)",
                     "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                     "frac": ach / peak, "traffic": None,
                     "peak_source": "%s bf16 burst (cuBLAS GEMM)" % ctx["src"],
                     "flop_per_config": fpc},
    }


def path_tiny(ctx):
    kt, torch, stream, flush = ctx["kt"], ctx["torch"], ctx["stream"], ctx["flush"]
    wl, desc, roles, gpu, sp, valid, digits, model, m, samp = setup(kt, "tiny_block_tile", 0)
    n_steps = 40
    Wu = ctx["warmup"]
    traj = record(kt, sp, m, gpu, valid, digits, wl, 0, Wu + n_steps)
    s = kt.Search(sp, m, k=5, seed=0, stream=stream)
    bufs = (torch.empty(5, dtype=torch.int64, device="cuda").data_ptr(),
            torch.empty(5, dtype=torch.float32, device="cuda").data_ptr(),
            torch.empty(1, dtype=torch.int32, device="cuda").data_ptr())
    untimed_device_steps(s, traj, 0, Wu, 5, bufs, stream)
    torch.cuda.synchronize()
    step_ms, _, _, scored, _ = timed_device_steps(kt, torch, s, traj, Wu, Wu + n_steps, 5,
                                                  stream, flush)
    s.close()
    return {"workload": "tiny_block_tile: 6 params, %d valid configurations, K=16, depth-8 trees "
                        "fitted on a 10%% sample, k=5; %d steps" % (len(valid), n_steps),
            "us_per_step_median": 1e3 * statistics.median(step_ms),
            "us_per_step_mean": 1e3 * sum(step_ms) / n_steps,
            "value": scored / (sum(step_ms) / 1e3), "unit": "configs/s",
            "bound": "launch latency (one CUDA-graph launch of 4 kernels per step)"}


# ---------------------------------------------------------------------------
def oracle_sample(desc, n_valid_target, seed=1):
    """A uniform sample of valid configurations, drawn by the oracle."""
    from oracle import space as ospace
    rng = np.random.default_rng(seed)
    if desc.n_raw <= 4 * n_valid_target:
        raw = ospace.enumerate_valid(desc)
    else:
        raw = np.zeros(0, np.int64)
        while len(raw) < n_valid_target:
            r = np.unique(rng.integers(0, desc.n_raw, size=4 * n_valid_target))
            raw = np.union1d(raw, r[ospace.is_valid_raw(desc, r)])
        raw = np.sort(rng.choice(raw, size=n_valid_target, replace=False))
    return raw, ospace.decode(desc.radices, raw)


def oracle_step_time(wl, roles, model, dig, counters, seed=0, step=0):
    """Time one oracle step over the sampled configurations: predictions,
    expert system, Eq. score, normalisation, weights and k draws."""
    from oracle import expert, score as oscore, select as oselect, trees as otrees
    t0 = time.perf_counter()
    pred = otrees.predict(model, dig)
    d64 = expert.delta_vector(roles, counters)
    s = oscore.score_fp32(pred[0], pred, d64.astype(np.float32))
    free = np.ones(len(s), bool)
    free[0] = False                       # the sample's first configuration plays c_profile
    sn = oselect.normalise_fp32(s[free], s[free].min(), s[free].max())
    w = np.zeros(len(s), np.uint64)
    w[free] = oselect.quantise(sn)
    oselect.weighted_draws(w, wl["k"], seed, 0, step)
    return time.perf_counter() - t0, int(free.sum())


# ---- the oracle on every host core: worker state and tasks (spawned processes) ----
_W = {}


def _oracle_init(model, dig, prof, d32):
    _W.update(model=model, dig=dig, prof=prof, d32=d32)


def _oracle_scores(lohi):
    from oracle import score as oscore, trees as otrees
    lo, hi = lohi
    return oscore.score_fp32(_W["prof"], otrees.predict(_W["model"], _W["dig"][lo:hi]), _W["d32"])


def _oracle_weights(args):
    from oracle import select as oselect
    s, smin, smax = args
    return oselect.quantise(oselect.normalise_fp32(s, smin, smax))


def oracle_step_time_allcores(wl, roles, model, dig, counters, n_proc):
    """The oracle step of oracle_step_time with its per-configuration work
    (predictions, Eq. score, normalisation and weights) split over n_proc
    spawned processes; the draws run in the parent.  Pool start-up and the
    workers' copies of the inputs are outside the timed region."""
    import multiprocessing as mp
    from oracle import expert, select as oselect, trees as otrees
    prof = otrees.predict(model, dig[:1])[0]
    d32 = expert.delta_vector(roles, counters).astype(np.float32)
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    edges = np.linspace(1, len(dig), n_proc + 1).astype(np.int64)   # configuration 0 is c_profile
    parts = [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:])]
    with mp.get_context("spawn").Pool(n_proc, initializer=_oracle_init,
                                      initargs=(model, dig, prof, d32)) as pool:
        pool.map(_oracle_scores, [(0, 1)] * n_proc)           # every worker started and warm
        t0 = time.perf_counter()
        sc = pool.map(_oracle_scores, parts)
        smin = min(float(x.min()) for x in sc)
        smax = max(float(x.max()) for x in sc)
        ws = pool.map(_oracle_weights, [(x, np.float32(smin), np.float32(smax)) for x in sc])
        w = np.concatenate([np.zeros(1, np.uint64)] + ws)
        oselect.weighted_draws(w, wl["k"], 0, 0, 0)
        t = time.perf_counter() - t0
    return t, len(dig) - 1


def cpu_baseline(name, model, counters, n_sample=None):
    wl = WORKLOADS[name]
    desc = load_desc(wl)
    roles = W.layout(wl["K"])
    n_sample = n_sample or (1_000_000 if desc.n_raw > 1e7 else min(desc.n_raw, 1_000_000))
    raw, dig = oracle_sample(desc, n_sample)
    t, n = oracle_step_time(wl, roles, model, dig, counters)
    out = {"value": n / t, "unit": "configs/s", "cores": 1, "kind": "oracle",
           "host_cores": os.cpu_count(),
           "sample": "one oracle step (numpy, single thread) over %d valid configurations drawn "
                     "uniformly from the workload's space, same model and counters" % len(raw),
           "seconds": t}
    n_proc = os.cpu_count() or 1
    if n_proc > 1:
        ta, na = oracle_step_time_allcores(wl, roles, model, dig, counters, n_proc)
        out["all_cores"] = {"value": na / ta, "unit": "configs/s", "cores": n_proc, "kind": "oracle",
                            "sample": "the same step over the same sample, its per-configuration "
                                      "work split over %d spawned processes (one per host core)"
                                      % n_proc, "seconds": ta}
    return out


def oracle_count(wl):
    """The space's valid count as the oracle wrote it (tests/golden/space_counts.json,
    written by tests/golden/make_spaces.py with oracle.space.count_valid), so
    that the reference line names the same configuration as the library's."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "space_counts.json")) as f:
            return int(json.load(f)[wl["space"]]["n_valid"])
    except (OSError, KeyError, TypeError, ValueError):
        return -1


def run_reference(args):
    """The oracle as the reference arm: --steps timed oracle steps, each over
    a bounded uniform sample of the workload (no GPU used)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if int(os.environ.get("RANK", "0")) != 0:
        return
    name = args.workload
    wl = WORKLOADS[name]
    desc = load_desc(wl)
    roles = W.layout(wl["K"])
    gpu = SyntheticGPU(desc, roles, seed=0)
    n_sample = 200_000 if desc.n_raw > 1e7 else min(desc.n_raw, 200_000)
    raw, dig = oracle_sample(desc, n_sample)
    m = max(2, int(round(wl["frac"] * len(raw))))
    Y = gpu.evaluate(dig[:m])[0]
    if wl["noise"]:
        Y = add_noise(Y, 0, wl["noise"])
    from paper_2102_05297_gb300 import fit   # host-side model creation (input preparation)
    model = fit.fit_model(dig[:m], Y, wl["depth"], desc.radices, roles)
    counters = gpu.evaluate(dig[:1])[0][0]
    for i in range(args.warmup):
        oracle_step_time(wl, roles, model, dig, counters, step=i)
    tt, nn = 0.0, 0
    for i in range(args.steps):
        t, n = oracle_step_time(wl, roles, model, dig, counters, step=args.warmup + i)
        tt += t
        nn += n
    v = nn / tt
    cb = {"value": v, "unit": "configs/s", "cores": 1, "kind": "oracle",
          "host_cores": os.cpu_count(),
          "sample": "each step one oracle step (numpy, single thread) over %d valid configurations "
                    "drawn uniformly from the workload's space" % len(raw)}
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "configs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": describe(name, wl, desc, oracle_count(wl)), "cpu_baseline": cb,
        "e2e": {"value": v, "unit": "configs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mid_12p", choices=list(WORKLOADS))
    ap.add_argument("--paths", default="all",
                    help="all | none | comma list of %s" % ",".join(ALL_PATHS))
    ap.add_argument("--mlp-train-steps", type=int, default=2000,
                    help="Adam steps (4096 rows each) of the MLP path's training")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fused", type=int, default=2,
                    help="step shape of the headline search (ktune_search_set_fused): 0 = four "
                         "kernels, 1..3 = the whole step as one persistent kernel")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

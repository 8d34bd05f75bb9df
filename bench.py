"""Benchmark of the counter-guided search step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (default): the mid-size synthetic tuning space -- 12 parameters,
41.3M raw / 2.26M valid configurations materialised on the device, 32 FP32
counters, depth-12 regression trees per counter fitted on a 2% sample with 2%
Gaussian noise, k = 5 weighted draws per step.  A step is one full pass of the
hot path: bottleneck analysis and Delta-PC, prediction of c_profile and of
every unevaluated configuration, Eq. score, normalisation, integer weights,
k draws without replacement, evaluated-set update.

The per-step inputs (the measured counters of each step's c_profile) come
from a recorded search over the synthetic performance function; the timed
steps replay them from device memory (``value``), and the end-to-end leg
replays them through the host API with its copies (``e2e``).  L2 is flushed
between timed steps (a 256 MB write outside the timed region).

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


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


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
            "l2": "flushed between timed steps (256 MB write outside the timed region)"}


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
                                       "--format=csv,noheader,nounits", "-lms", "200"],
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
    return wl, desc, roles, gpu, sp, valid, digits, model, m


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
    wl, desc, roles, gpu, sp, valid, digits, model, m = setup(kt, name, seed)
    K, Wu = args.steps, args.warmup
    traj = record(kt, sp, m, gpu, valid, digits, wl, seed, Wu + K)
    # a dedicated stream: steps on a non-default stream run as one captured CUDA graph
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    # ---- device-resident timed steps -------------------------------------
    s = kt.Search(sp, m, k=wl["k"], seed=seed, stream=stream)
    s.set_timing(True)
    cnt_host = [np.ascontiguousarray(t[1], dtype=np.float32) for t in traj]
    out_raw = torch.empty(wl["k"], dtype=torch.int64, device="cuda")
    out_sc = torch.empty(wl["k"], dtype=torch.float32, device="cuda")
    n_out = torch.empty(1, dtype=torch.int32, device="cuda")
    for i in range(Wu):
        s.set_profile(int(traj[i][0]))
        s.step_device(cnt_host[i], wl["k"], out_raw.data_ptr(), out_sc.data_ptr(),
                      n_out.data_ptr(), stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    step_ms, score_ms, kern_ms, visits, scored = [], [], np.zeros(4), 0, 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for i in range(Wu, Wu + K):
        flush.zero_()
        s.set_profile(int(traj[i][0]))
        e0.record(stream)
        s.step_device(cnt_host[i], wl["k"], out_raw.data_ptr(), out_sc.data_ptr(),
                      n_out.data_ptr(), stream)
        e1.record(stream)
        st = s.stats()                  # synchronises
        step_ms.append(e0.elapsed_time(e1))
        kern_ms += np.array(st.kernel_ms[:4])
        score_ms.append(st.kernel_ms[1])
        visits += st.n_scored * st.n_active * (st.depth + 1)
        scored += st.n_scored
    torch.cuda.synchronize()
    ck = clocks.stop()
    t_total = sum(step_ms) / 1e3
    s.close()

    # ---- end to end through the host API ---------------------------------
    s2 = kt.Search(sp, m, k=wl["k"], seed=seed, stream=stream)
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

    if dist:
        tt = torch.tensor([t_total, sum(e2e_ms) / 1e3], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        cnt = torch.tensor([scored], dtype=torch.float64, device="cuda")
        dist.all_reduce(cnt, op=dist.ReduceOp.SUM)
        t_total, t_e2e, scored_all = float(tt[0]), float(tt[1]), float(cnt[0])
    else:
        t_e2e, scored_all = sum(e2e_ms) / 1e3, float(scored)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    pk, src = peaks()
    props = torch.cuda.get_device_properties(local)
    sm_mhz = float(pk.get("sm_max_mhz", 2070.0))
    peak_visits = props.multi_processor_count * 4 * 32 * sm_mhz * 1e6 / 4.0
    achieved = visits / (sum(score_ms) / 1e3)
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
        "roofline": {
            "bound": "alu",
            "kernel": "k_score_mat (tree walk + Eq. score)",
            "achieved": achieved / 1e9,
            "peak": peak_visits / 1e9,
            "unit": "Gvisit/s",
            "frac": achieved / peak_visits,
            "traffic": None,
            "peak_source": "derived: %d SMs x 4 SMSPs x 32 lanes x %.0f MHz (%s sm_max) / 4 "
                           "instructions per node visit" % (props.multi_processor_count, sm_mhz, src),
            "kernel_share": {"prepare": kern_ms[0] / kern_ms.sum(), "score": kern_ms[1] / kern_ms.sum(),
                             "weights": kern_ms[2] / kern_ms.sum(), "select": kern_ms[3] / kern_ms.sum()},
        },
        "e2e": {"value": scored_all / t_e2e, "unit": "configs/s", "h2d_bytes_per_step": bytes_h2d,
                "d2h_bytes_per_step": bytes_d2h, "ms_per_step": 1e3 * t_e2e / K},
        "gpu_launches": 4 * K,
        "clocks": ck,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(name, model, traj[Wu][1])
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


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


def cpu_baseline(name, model, counters, n_sample=None):
    wl = WORKLOADS[name]
    desc = load_desc(wl)
    roles = W.layout(wl["K"])
    n_sample = n_sample or (1_000_000 if desc.n_raw > 1e7 else min(desc.n_raw, 1_000_000))
    raw, dig = oracle_sample(desc, n_sample)
    t, n = oracle_step_time(wl, roles, model, dig, counters)
    return {"value": n / t, "unit": "configs/s", "cores": 1, "kind": "oracle",
            "host_cores": os.cpu_count(),
            "sample": "one oracle step (numpy, single thread) over %d valid configurations drawn "
                      "uniformly from the workload's space, same model and counters" % len(raw),
            "seconds": t}


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
        "data": "synthetic", "config": describe(name, wl, desc, -1), "cpu_baseline": cb,
        "e2e": {"value": v, "unit": "configs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mid_12p", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

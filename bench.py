"""Throughput of the slip-spring time step on GB300, in bead-steps/s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: the equilibrium linear-viscoelasticity ensemble -- 65536 chains of
N = 32 beads, FP32 beads with FP64 ensemble sums, the paper's parameters
(N0 = 4, Ns = 0.5, zeta_s = 0.1, dt = 0.01), multiple-tau correlator with 16
points x 24 levels, synthetic equilibrium start from Philox seed 1.  One bench
step is one library call ss_run(steps_per_call) covering every part of the
time step (bead update, slip-spring forces, hops, creation/destruction,
stress, correlator).  `value` is whole-job bead-steps/s with the state resident
in HBM; `e2e` is the same metric through the C ABI with the state copied in
from host memory and G(t) read back every step; `plain` is the one-step-per-
launch form of the same library (state through HBM every step, FP64 flush of
the correlator every step).  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

# ---- algorithmic work per bead-step (N = 32, <Z>/N = 1/N0 = 0.25, kappa = 0)
# Counted per bead and step as scalar operations of the method, a multiply-add
# and a three-input logic operation counting once, a transcendental once.
ALG_OPS = {
    "philox_block": 10 * 6,          # 10 rounds x (2 wide multiplies, 2 xor3, 2 key adds)
    "box_muller_2pairs": 2 * 11,     # 2 x (2 cvt, 2 scale, log, x-2, sqrt, sin, cos, 2 mul)
    "uniform24": 5,                  # byte extract/merge, cvt, scale
    "bond_force": 3 * 4,             # 2 differences + 2 fma per component
    "euler_update": 3 * 2,           # R + mob F + amp n
    "spring_force": 0.25 * 3 * 2,    # per spring: difference + fma per component
    "hop": 0.25 * 44,                # 3 squared distances, 2 Glauber probabilities, decision
    "create_attempt": 0.75 * 2,      # empty slots: two comparisons
    "destroy_test": 0.06 * 1,
    "stress": 3 + 6 + 0.25 * 9 + 6,  # bond vector, 3 off-diagonal products, springs, sums
    "correlator": (96 + 60) / 32.0,  # per chain: 2 ch x 16 lags x 3 comps + higher levels
}
ALG_OPS_PER_BEAD_STEP = float(sum(ALG_OPS.values()))
SMS, LANES_PER_SM, SM_MAX_MHZ_NOMINAL = 152, 128, 2070.0
# DRAM bytes (read + write) of one chain-kernel launch of 1024 steps, per chain:
# ncu capture of 16384 chains x 1024 steps (profiles/chunk_kernel_16x2_small_full.md),
# 17.3 MB read + 363.5 MB written; every term scales with the chain count.
TRAFFIC_BYTES_PER_CHAIN_1024 = 380.2e6 / 16384


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def _max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def run_ours(args):
    import torch

    from paper_1106_2899_gb300 import SlipSpring, build

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    w = synth.WORKLOADS["lve"]
    M, N = args.chains, w["N"]
    spc = args.steps_per_call
    stream = torch.cuda.current_stream()

    def make(chunk):
        # rank r runs its own M chains, global chain ids r*M .. r*M+M-1 (weak scaling)
        g = SlipSpring([(M, N)], precision="fp32", seed=w["seed"], stream=stream.cuda_stream, chain_offset=rank * M)
        g.set_params(**synth.PAPER, corr_levels=w["levels"], groups=32, chunk_steps=chunk)
        return g

    # ---------------- resident (batched multi-step) form
    g = make(args.chunk)
    g.run(0)
    for _ in range(args.warmup):
        g.run(spc)
    torch.cuda.synchronize()
    c0 = g.counters()["launches"]
    g.kernel_timing(True)
    clocks = ClockSampler(local)
    clocks.start()
    _barrier(ws)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        g.run(spc)
    t1.record(stream)
    torch.cuda.synchronize()
    _barrier(ws)
    clk = clocks.stop()
    ms_total = t0.elapsed_time(t1)
    launches = g.counters()["launches"] - c0
    chain_ms, chain_launches = g.kernel_time()  # CUDA events around each chain-kernel launch
    g.kernel_timing(False)
    ms_total = _max_over_ranks(ms_total, ws)
    bead_steps = float(M) * N * spc * args.steps
    value = bead_steps * ws / (ms_total / 1e3)
    kernel_ms = chain_ms / max(chain_launches, 1)
    steps_per_launch = spc * args.steps / max(chain_launches, 1)
    alg_ops_launch = ALG_OPS_PER_BEAD_STEP * M * N * steps_per_launch
    achieved = alg_ops_launch / (kernel_ms / 1e3)
    peak = SMS * LANES_PER_SM * SM_MAX_MHZ_NOMINAL * 1e6
    status = g.status()
    tg, Gg, sg = g.correlator("total")
    dt_step = synth.PAPER["dt"]
    gpu_G = {int(round(tt / dt_step)): (float(a), float(b)) for tt, a, b in zip(tg, Gg, sg)}
    g.close()

    # ---------------- plain one-step-per-launch form (same library, chunk = 1)
    gp = make(1)
    gp.run(0)
    gp.run(args.warmup)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    gp.run(args.plain_steps)
    b.record(stream)
    torch.cuda.synchronize()
    plain_ms = _max_over_ranks(a.elapsed_time(b), ws)
    plain_value = float(M) * N * args.plain_steps * ws / (plain_ms / 1e3)
    gp.close()

    # ---------------- end to end through the C ABI with host buffers
    ge = make(args.chunk)
    ge.run(0)
    # the step's inputs live in pinned host memory (numpy views of pinned tensors)
    host_state = {}
    for k, v in ge.get_state().items():
        pinned = torch.empty(v.shape, dtype=torch.float64 if v.dtype == np.float64 else torch.int32,
                             pin_memory=True).numpy()
        pinned[...] = v
        host_state[k] = pinned
    ge.run(spc)
    ge.correlator("total")
    torch.cuda.synchronize()
    e2e_steps = max(2, args.steps // 2)
    te = time.perf_counter()
    for _ in range(e2e_steps):
        ge.set_state(host_state)      # host -> device: the state of this step
        ge.run(spc)
        tt, GG, ss = ge.correlator("total")  # device -> host: G(t) of this step
    torch.cuda.synchronize()
    e2e_s = _max_over_ranks(time.perf_counter() - te, ws)
    e2e_value = float(M) * N * spc * e2e_steps * ws / e2e_s
    # set_state copies the caller's arrays as they are (R, A double; S, Z int32) and
    # reads back a 4-byte check flag; correlator() copies the FP64 group sums
    zm = min(N, 64)
    h2d = M * (N * 3 * 8 + zm * 3 * 8 + zm * 4 + 4)
    d2h = 32 * w["levels"] * 96 * 8 + 4
    ge.close()

    if rank != 0:
        return None
    pk = _peaks()
    out = {
        "metric": "bead-steps/s",
        "value": value,
        "unit": "bead-steps/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_total / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic: equilibrium ensembles sampled by the library (Philox seed 1)",
        "config": {"workload": "lve: %d chains x N=32, FP32 beads / FP64 sums, multiple-tau 16x24, "
                               "paper parameters N0=4 Ns=0.5 zeta_s=0.1 dt=0.01" % M,
                   "chains": M, "beads": N, "steps_per_call": spc, "steps_per_launch": args.chunk,
                   "l2": "working set (state, stress series, correlator buffers, ~3.9 GB) larger than L2",
                   "parallelism": "independent chains; ranks run disjoint chains" if ws > 1 else "1 GPU"},
        "plain": {"value": plain_value, "unit": "bead-steps/s", "steps": args.plain_steps,
                  "form": "one step per launch, state and correlator through HBM, FP64 flush every step",
                  "batched_over_plain": value / plain_value},
        "e2e": {"value": e2e_value, "unit": "bead-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "lane-ops/s",
                     "frac": achieved / peak,
                     "traffic": TRAFFIC_BYTES_PER_CHAIN_1024 * M if abs(steps_per_launch - 1024) < 1e-9 else None,
                     "kernel": "chunk_kernel<float, 16, 2, 0, 0>", "kernel_ms": kernel_ms,
                     "kernel_share_of_region": chain_ms / ms_total if ws == 1 else None,
                     "alg_ops_per_bead_step": ALG_OPS_PER_BEAD_STEP,
                     "peak_basis": "152 SMs x 128 lanes x 2070 MHz (nominal max clock), 1 lane-op/lane/clock"},
        "clocks": clk,
        "status": status,
        "hbm_peak_measured_gbs": pk.get("hbm_gbs"),
    }
    if not args.no_cpu_baseline:
        cb = cpu_baseline(args.cpu_chains, args.cpu_steps)
        out["g_err_vs_oracle"] = g_error(gpu_G, cb.pop("_G"))
        out["cpu_baseline"] = cb
    return out


def cpu_baseline(M=4096, steps=3000, nthreads=0):
    """The FP64 CPU oracle as it stands, on a bounded sample of the workload."""
    import oracle
    w = synth.WORKLOADS["lve"]
    p = oracle.Params(N=w["N"], **synth.PAPER)
    nthreads = nthreads or os.cpu_count()
    e = oracle.Ensemble(p, seed=w["seed"], M=M, groups=32, levels=w["levels"])
    e.init()
    e.run(20, nthreads=nthreads)
    t = time.perf_counter()
    e.run(steps, nthreads=nthreads)
    dt = time.perf_counter() - t
    # G(t) of the TOTAL channel per multiple-tau slot, mean and SE over the 32 groups
    acc, n = e.corr_sums()
    cnt = oracle.corr_counts(n, w["levels"])
    lags = oracle.corr_lags(w["levels"])
    per_group = np.array([(g + 1) * M // 32 - g * M // 32 for g in range(32)], dtype=float)
    G = {}
    for l in range(w["levels"]):
        for k in range(16):
            if lags[l, k] < 0 or cnt[l, k] <= 0:
                continue
            gk = acc[:, l, k, 1, :].sum(axis=-1) / 3.0 / (cnt[l, k] * per_group * w["N"] * p.kT * p.kT)
            G[int(lags[l, k])] = (float(gk.mean()), float(gk.std(ddof=1) / np.sqrt(len(gk))))
    return {"value": M * w["N"] * steps / dt, "unit": "bead-steps/s", "cores": nthreads, "kind": "oracle",
            "sample": "%d chains x N=%d x %d steps of the lve workload (correlator 16x24), %.1f s" % (
                M, w["N"], steps, dt), "_G": G}


def g_error(gpu, ora, max_lag=2000):
    """G(t) of the benchmark run against the oracle's independent FP64 ensemble at
    common lags up to max_lag steps: z-scores |dG| / sqrt(SE_gpu^2 + SE_oracle^2), and
    the relative error where the oracle resolves G to 0.5%."""
    zs, rel = [], []
    for lag, (gg, sg) in gpu.items():
        if lag > max_lag or lag not in ora:
            continue
        go, so = ora[lag]
        zs.append(abs(gg - go) / np.sqrt(sg * sg + so * so))
        if so < 0.005 * abs(go):
            rel.append(abs(gg - go) / abs(go))
    if not zs:
        return None
    zs = np.array(zs)
    return {"channel": "TOTAL", "lags_compared": int(len(zs)), "max_lag_steps": max_lag,
            "max_z": float(zs.max()), "frac_z_below_3": float(np.mean(zs < 3.0)),
            "max_rel_err_where_resolved": float(max(rel)) if rel else None, "resolved_lags": len(rel),
            "oracle": "independent FP64 ensemble of the cpu_baseline leg (other chains)"}


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return None
    vals = []
    cb = None
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline(args.cpu_chains, max(50, args.cpu_steps // 5))
        cb.pop("_G")
        if k >= args.warmup:
            vals.append(cb["value"])
    value = float(np.mean(vals))
    return {"impl": "reference", "metric": "bead-steps/s", "value": value, "unit": "bead-steps/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "lve: 65536 chains x N=32 (bounded sample: %d chains per step)" % args.cpu_chains},
            "cpu_baseline": {"value": value, "unit": "bead-steps/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": value, "unit": "bead-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--chains", type=int, default=synth.WORKLOADS["lve"]["M"])
    ap.add_argument("--steps-per-call", type=int, default=2048)
    ap.add_argument("--chunk", type=int, default=1024)
    ap.add_argument("--plain-steps", type=int, default=200)
    ap.add_argument("--cpu-chains", type=int, default=4096)
    ap.add_argument("--cpu-steps", type=int, default=10000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()

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
the correlator every step).

Further blocks of the JSON line (outside the timed region):
  batched    the batched multiscale workload (4096 elements, ensemble sizes
             log-uniform in 64..1024, lengths in {16, 24, 32, 48}, traceless
             Gaussian velocity gradients redrawn every 1000 steps) in one
             graph-replayed persistent launch per chunk: bead-steps/s from
             CUDA events over --batched-steps steps, its ALU roofline and the
             ratio to the plain per-ensemble form; `n32`: the same element
             table with every chain length 32, against the plain form at the
             same N.
  heun       the benchmark workload with the stochastic Heun integrator.
  precision  error of the FP32 library against the FP64 oracle per output:
             G(t) AUTO/CROSS/TOTAL at long lags and eta+(t), N1, <Z> at the 8
             startup-shear rates against the stored oracle reference
             (tests/golden/longrun_*_oracle.txt), and the short-lag G(t) of the
             benchmark run against the cpu_baseline leg's oracle ensemble.
The ALU roofline's numerator is the oracle's operation count per bead-step
(tests/golden/alg_ops.txt, written by the counting build of the oracle) less
the correlator's operations, which the correlator kernel executes; the
peak is the device's SM count x 128 lanes x the SM clock sampled during the
timed region.  --impl reference times the FP64 CPU oracle on a bounded
sample of the same workload.
"""
import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import longrun_parity  # noqa: E402  (reads the stored oracle reference; runs only the library)
import synth  # noqa: E402

LANES_PER_SM = 128  # FP32/INT32 lanes of a Blackwell SM: 4 schedulers x 32, one instruction per clock each
ALG_OPS_FILE = os.path.join(ROOT, "tests", "golden", "alg_ops.txt")
# DRAM bytes (read + write) of one chain-kernel launch of 1024 steps, per chain, from the ncu
# capture of 16384 chains x 1024 steps of the current kernel (382.8 MB; every term scales with
# the chain count), profiles/chunk_kernel_16x2_lve_small.md; None once the kernel has changed
TRAFFIC_BYTES_PER_CHAIN_1024 = 382.8e6 / 16384


def alg_ops():
    """Operations of the method per bead-step by workload, from the stored counts of
    the oracle's counting build: {name: {"total": x, category: x}}."""
    out, cats = {}, None
    for ln in open(ALG_OPS_FILE):
        if ln.startswith("# name"):
            cats = ln.split()[2:]
        elif ln.strip() and not ln.startswith("#"):
            f = ln.split()
            out[f[0]] = dict(zip(cats, [float(x) for x in f[1:]]))
    return out


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


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


def _peak(sms, clk):
    """ALU issue peak in lane-ops/s at the SM clock clk (MHz) and its basis."""
    mhz = clk.get("sm_max_mhz") or _peaks().get("sm_max_mhz") or 2070.0
    return sms * LANES_PER_SM * mhz * 1e6, "%d SMs (device) x %d lanes x %.0f MHz (max SM clock sampled during " \
        "the timed region), 1 lane-op per lane per clock" % (sms, LANES_PER_SM, mhz)


def _time_batched(els, G, n_k, every, steps, stream, rank, seed):
    """Run a batched ensemble (elements els, velocity-gradient table G) for 1000
    warm-up steps, then time `steps` more with CUDA events and sampled clocks."""
    import torch

    from paper_1106_2899_gb300 import SlipSpring
    warm = 1000
    g = SlipSpring(els, precision="fp32", seed=seed + 1000 * rank, stream=stream.cuda_stream)
    g.set_params(**synth.PAPER, corr_levels=-1, groups=4, log_every=100, max_logs=(warm + steps) // 100,
                 chunk_steps=1000)
    g.set_batched(True)
    g.set_flow_table(np.repeat(np.arange(len(els)), n_k), np.tile(np.arange(n_k) * every, len(els)),
                     G.reshape(-1, 3, 3))
    g.run(0)
    g.run(warm)  # autotune and the first graph launches
    torch.cuda.synchronize()
    c0 = g.counters()["launches"]
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    g.run(steps)
    b.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = a.elapsed_time(b)
    status = g.status()
    launches = g.counters()["launches"] - c0
    g.close()
    return ms, clk, status, launches


def run_batched(args, stream, rank, sms, ops_by_n):
    """The batched multiscale workload: one graph-replayed persistent launch per
    chunk; then the same element table with every chain length set to 32 (the
    batched form at the benchmark's N against the plain per-ensemble form)."""
    w = synth.WORKLOADS["batched"]
    steps, every = args.batched_steps, w["kappa_every"]
    n_k = (1000 + steps) // every + 1
    Ms, Ns, G = synth.element_table(args.batched_elements, seed=w["seed"], lengths=w["lengths"], m_lo=w["m_lo"],
                                    m_hi=w["m_hi"], n_kappa=n_k, kappa_std=w["kappa_std"])
    els = [(int(m), int(n)) for m, n in zip(Ms, Ns)]
    ms, clk, status, launches = _time_batched(els, G, n_k, every, steps, stream, rank, w["seed"])
    beads = float(sum(m * n for m, n in els))
    ops = sum(m * n * ops_by_n["flow_%d" % n]["total"] for m, n in els) / beads
    value = beads * steps / (ms / 1e3)
    peak, basis = _peak(sms, clk)
    out = {"value": value, "unit": "bead-steps/s", "steps": steps, "ms": ms,
           "workload": "batched multiscale: %d elements, %d chains, %.4g beads (N in %s), FP32 beads / FP64 "
                       "per-element stress sums, kappa redrawn every %d steps" % (
                           len(els), int(sum(Ms)), beads, list(w["lengths"]), every),
           "roofline": {"bound": "alu", "achieved": ops * value, "peak": peak, "unit": "lane-ops/s",
                        "frac": ops * value / peak, "alg_ops_per_bead_step": ops,
                        "kernel": "batched_kernel (all lane-layout classes of one graph launch per chunk, "
                                  "timed together with CUDA events)", "peak_basis": basis, "traffic": None},
           "clocks": clk, "status": status, "gpu_launches": int(launches)}
    els32 = [(m, 32) for m, _ in els]
    ms32, clk32, status32, launches32 = _time_batched(els32, G, n_k, every, steps, stream, rank, w["seed"])
    beads32 = float(sum(m * n for m, n in els32))
    value32 = beads32 * steps / (ms32 / 1e3)
    ops32 = ops_by_n["flow_32"]["total"]
    peak32, _ = _peak(sms, clk32)
    out["n32"] = {"value": value32, "unit": "bead-steps/s", "steps": steps, "ms": ms32,
                  "workload": "the same %d elements and velocity gradients, every chain N = 32 (%.4g beads)" % (
                      len(els32), beads32),
                  "roofline": {"bound": "alu", "achieved": ops32 * value32, "peak": peak32, "unit": "lane-ops/s",
                               "frac": ops32 * value32 / peak32, "alg_ops_per_bead_step": ops32},
                  "clocks": clk32, "status": status32, "gpu_launches": int(launches32)}
    return out


def run_precision(stream):
    """FP32 library against the stored FP64 oracle reference, per output."""
    ref_G = longrun_parity.load_G()
    res_G = longrun_parity.compare_G(longrun_parity.gpu_G(stream=stream.cuda_stream), ref_G)
    steady, logs = longrun_parity.load_eta()
    rates = synth.WORKLOADS["shear"]["rates"]
    res_eta = longrun_parity.compare_eta(longrun_parity.gpu_eta(rates, stream=stream.cuda_stream), steady, logs,
                                         rates)
    out = {"criterion": "z = |delta| / sqrt(SE_gpu^2 + SE_oracle^2): every z <= 4, at most 1% of z above 3 "
                        "(the 3-SE bound with the multiplicity of the comparisons), and |delta| <= 2% where the "
                        "oracle's relative SE < 0.5%",
           "G": {ch: {k: v for k, v in r.items() if k not in ("failures", "zs")} | {"failures": len(r["failures"])}
                 for ch, r in res_G.items()},
           "G_workload": "equilibrium N=32, 65536 GPU chains vs 2048 oracle chains, 320000 steps"}
    eta = {}
    for k, r in res_eta.items():
        eta["%.3g" % r["gdot"]] = {
            q: {"max_z": r[q]["max_z"], "n_z_over_3": r[q]["n_z_over_3"],
                "max_rel_err_where_resolved": r[q]["max_rel_err_where_resolved"],
                "times": r[q]["times_compared"], "failures": len(r[q]["failures"])} for q in ("eta", "N1", "Z")}
        eta["%.3g" % r["gdot"]]["steady_eta"] = {k2: r["steady_eta"][k2] for k2 in ("gpu", "gpu_se", "oracle",
                                                                                     "oracle_se", "z")}
    out["startup_shear"] = eta
    out["shear_workload"] = "N=32, 16384 GPU chains vs 1024 oracle chains per rate, 200000 steps"
    zG = [z for r in res_G.values() for z in r["zs"]]
    zE = [z for r in res_eta.values() for q in ("eta", "N1", "Z") for z in r[q]["zs"]]
    fails = [f for r in res_G.values() for f in r["failures"]] + [
        f for r in res_eta.values() for q in ("eta", "N1", "Z") for f in r[q]["failures"]]
    out["comparisons"] = len(zG) + len(zE)
    out["n_z_over_3"] = int(np.sum(np.array(zG + zE) > 3.0))
    out["all_pass"] = longrun_parity.passes(zG, []) and longrun_parity.passes(zE, []) and not fails and all(
        r["steady_eta"]["ok"] for r in res_eta.values())
    out["max_lag_steps"] = max(v["max_lag_steps"] for v in out["G"].values())
    return out


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
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    ops = alg_ops()
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
    # the chain kernel's share of the method's operations: all but the
    # correlator's, which corr_kernel executes
    ops_lve = ops["lve"]["total"] - ops["lve"]["correlator"]
    achieved = ops_lve * M * N * steps_per_launch / (kernel_ms / 1e3)
    peak, basis = _peak(sms, clk)
    status = g.status()
    gpu_G = {}
    for ch in longrun_parity.CHANNELS:
        tg, Gg, sg = g.correlator(ch)
        gpu_G[ch] = {int(round(tt / synth.PAPER["dt"])): (float(a), float(b)) for tt, a, b in zip(tg, Gg, sg)}
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
    ge.set_state(host_state)  # warm-up of the path: its staging buffer is allocated here, untimed
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

    # ---------------- the same workload with the stochastic Heun integrator
    heun = None
    if not args.no_heun:
        gh = SlipSpring([(M, N)], precision="fp32", seed=w["seed"], stream=stream.cuda_stream, chain_offset=rank * M)
        gh.set_params(**synth.PAPER, corr_levels=w["levels"], groups=32, chunk_steps=args.chunk, integrator=1)
        gh.run(0)
        gh.run(spc)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(3):
            gh.run(spc)
        b.record(stream)
        torch.cuda.synchronize()
        heun_ms = _max_over_ranks(a.elapsed_time(b), ws)
        heun_value = float(M) * N * spc * 3 * ws / (heun_ms / 1e3)
        heun = {"value": heun_value, "unit": "bead-steps/s", "steps": 3 * spc,
                "form": "stochastic Heun integrator (integrator = SS_HEUN), same workload and launch shape",
                "over_euler": heun_value / value}
        gh.close()

    batched = None if args.no_batched else run_batched(args, stream, rank, sms, ops)
    precision = None if (args.no_precision or rank != 0) else run_precision(stream)

    if rank != 0:
        return None
    pk = _peaks()
    traffic = TRAFFIC_BYTES_PER_CHAIN_1024 * M if (TRAFFIC_BYTES_PER_CHAIN_1024 and
                                                   abs(steps_per_launch - 1024) < 1e-9) else None
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
        "heun": heun,
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "lane-ops/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "chunk_kernel<float, 16, 2, 0, 0>", "kernel_ms": kernel_ms,
                     "kernel_share_of_region": chain_ms / ms_total if ws == 1 else None,
                     "alg_ops_per_bead_step": ops_lve,
                     "alg_ops_source": "oracle counting build (tests/golden/alg_ops.txt)",
                     "alg_ops_by_substep": {k: v for k, v in ops["lve"].items()
                                            if k not in ("total", "correlator")},
                     "alg_ops_in_corr_kernel": ops["lve"]["correlator"],
                     "peak_basis": basis, "sms": sms, "device": props.name},
        "clocks": clk,
        "status": status,
        "hbm_peak_measured_gbs": pk.get("hbm_gbs"),
    }
    if batched is not None:
        batched["over_plain"] = batched["value"] / plain_value
        batched["n32"]["over_plain"] = batched["n32"]["value"] / plain_value
        out["batched"] = batched
    if precision is not None:
        out["precision"] = precision
    if not args.no_cpu_baseline:
        cb = cpu_baseline(args.cpu_chains, args.cpu_steps)
        ora = cb.pop("_G")
        short = {ch: g_error(gpu_G[ch], ora[ch]) for ch in longrun_parity.CHANNELS}
        if precision is not None:
            precision["short_lag_vs_cpu_baseline"] = short
        out["g_err_vs_oracle"] = short["total"]
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
    # G(t) per channel and multiple-tau slot, mean and SE over the 32 groups
    acc, n = e.corr_sums()
    cnt = oracle.corr_counts(n, w["levels"])
    lags = oracle.corr_lags(w["levels"])
    per_group = np.array([(g + 1) * M // 32 - g * M // 32 for g in range(32)], dtype=float)
    G = {ch: {} for ch in longrun_parity.CHANNELS}
    for l in range(w["levels"]):
        for k in range(16):
            if lags[l, k] < 0 or cnt[l, k] <= 0:
                continue
            norm = cnt[l, k] * per_group * w["N"] * p.kT * p.kT
            auto = acc[:, l, k, 0, :].sum(axis=-1) / 3.0 / norm
            total = acc[:, l, k, 1, :].sum(axis=-1) / 3.0 / norm
            for ch, v in zip(longrun_parity.CHANNELS, (auto, total - auto, total)):
                G[ch][int(lags[l, k])] = (float(v.mean()), float(v.std(ddof=1) / np.sqrt(len(v))))
    return {"value": M * w["N"] * steps / dt, "unit": "bead-steps/s", "cores": nthreads, "kind": "oracle",
            "cpu": cpu_model(),
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
    return {"lags_compared": int(len(zs)), "max_lag_steps": max_lag,
            "max_z": float(zs.max()), "frac_z_below_3": float(np.mean(zs < 3.0)),
            "max_rel_err_where_resolved": float(max(rel)) if rel else None, "resolved_lags": len(rel),
            "oracle": "independent FP64 ensemble of the cpu_baseline leg (other chains)"}


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return None
    vals, secs = [], []
    cb = None
    for k in range(args.warmup + args.steps):
        t = time.perf_counter()
        cb = cpu_baseline(args.cpu_chains, max(50, args.cpu_steps // 5))
        dt = time.perf_counter() - t
        cb.pop("_G")
        if k >= args.warmup:
            vals.append(cb["value"])
            secs.append(dt)
    value = float(np.mean(vals))
    return {"impl": "reference", "metric": "bead-steps/s", "value": value, "unit": "bead-steps/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "lve: 65536 chains x N=32 (bounded sample: %d chains per step)" % args.cpu_chains},
            "cpu_baseline": {"value": value, "unit": "bead-steps/s", "cores": cb["cores"], "kind": "oracle",
                             "cpu": cb["cpu"], "sample": cb["sample"]},
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
    ap.add_argument("--batched-steps", type=int, default=10000)
    ap.add_argument("--batched-elements", type=int, default=synth.WORKLOADS["batched"]["n_elements"])
    ap.add_argument("--cpu-chains", type=int, default=4096)
    ap.add_argument("--cpu-steps", type=int, default=10000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-heun", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()

"""Long-run statistical parity of the FP32 library against the stored FP64
oracle reference (tests/golden/longrun_*_oracle.txt, written by
tests/golden/make_longrun_reference.py from independent oracle ensembles).

The library runs the same workloads with more chains and its own seeds:
* G(t), equilibrium, N = 32: 65536 chains, 20000 steps of equilibration, then
  320000 steps into the 16 x 24 multiple-tau correlator; AUTO, CROSS and TOTAL
  channels (Eq. relaxation_modulus_tensor_green_kubo_form, App. B) with
  standard errors over 32 chain groups, read through ss_correlator.
  The same with the stochastic Heun integrator against its own reference.
* Startup shear (Sec. 4.1), N = 32: 16384 chains per rate, the 8 rates
  10^(-4 + 3k/7), 200000 steps, stress logs every 100 steps; eta+ =
  <sigma_xy>/(N gdot), N1 = <sigma_xx - sigma_yy> and <Z> per log from the
  per-group log sums (ss_log_sums), the steady viscosity from the groups' time
  averages over the second half of the run.

The criterion (FP32 beads with FP64 sums against the FP64 oracle, for every
channel): z = |delta| / sqrt(SE_gpu^2 + SE_oracle^2) with standard errors from
32 chain groups.  "Within 3 SE at every logged time" is applied with its
multiplicity: the comparisons number in the thousands and a t statistic with
31 degrees of freedom exceeds 3 with probability about 0.5% even when both
sides sample the same law, so every z must be <= 4 (the family-wise bound
near 1% for this many correlated comparisons), at most 1% of them may exceed
3, and |delta| <= 2% of the oracle value wherever the oracle's relative SE is
below 0.5%.
"""
import os

import numpy as np

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
G_FILE = os.path.join(GOLDEN, "longrun_G_oracle.txt")
G_HEUN_FILE = os.path.join(GOLDEN, "longrun_G_heun_oracle.txt")
ETA_FILE = os.path.join(GOLDEN, "longrun_eta_oracle.txt")
CHANNELS = ("auto", "cross", "total")


def load_G(path=G_FILE):
    """{lag_steps: {channel: (G, se)}}"""
    out = {}
    for ln in open(path):
        if ln.startswith("#") or not ln.strip():
            continue
        f = ln.split()
        v = [float(x) for x in f[1:]]
        out[int(f[0])] = {ch: (v[2 * i], v[2 * i + 1]) for i, ch in enumerate(CHANNELS)}
    return out


def load_eta(path=ETA_FILE):
    """(steady {k: (gdot, eta, se)}, logs {k: array [n][step, eta, se, N1, se, Z, se]})"""
    steady, logs = {}, {}
    for ln in open(path):
        if ln.startswith("S "):
            f = ln.split()
            steady[int(f[1])] = (float(f[2]), float(f[3]), float(f[4]))
        elif ln.startswith("L "):
            f = ln.split()
            logs.setdefault(int(f[1]), []).append([float(x) for x in f[3:]])
    return steady, {k: np.array(v) for k, v in logs.items()}


def gpu_G(M=65536, N=32, seed=5, equil=20000, steps=320000, levels=24, groups=32, stream=None, integrator=0):
    from paper_1106_2899_gb300 import SlipSpring
    g = SlipSpring([(M, N)], precision="fp32", seed=seed, stream=stream)
    g.set_params(corr_levels=levels, groups=groups, integrator=integrator, **synth.PAPER)
    g.run(0)
    g.run(equil)
    g.reset_observables()
    g.run(steps)
    dt = synth.PAPER["dt"]
    out = {}
    for ch in CHANNELS:
        t, G, se = g.correlator(ch)
        for tt, a, b in zip(t, G, se):
            out.setdefault(int(round(tt / dt)), {})[ch] = (float(a), float(b))
    g.close()
    return out


def gpu_eta(rates, M=16384, N=32, seed0=2, steps=200000, log_every=100, groups=32, stream=None):
    """Per rate index: (steps [n], group means [n][G][14], steady (eta, se))."""
    from paper_1106_2899_gb300 import SlipSpring
    res = {}
    for k, gd in enumerate(rates):
        g = SlipSpring([(M, N)], precision="fp32", seed=seed0 + k, stream=stream)
        g.set_params(corr_levels=-1, groups=groups, log_every=log_every, max_logs=steps // log_every,
                     **synth.PAPER)
        g.run(0)
        g.set_flow(synth.shear_kappa(gd), from_step=0)
        g.run(steps)
        ts, L = g.log_sums()
        per = np.array([(i + 1) * M // groups - i * M // groups for i in range(groups)], dtype=float)
        gm = L / per[None, :, None]
        eta = gm[:, :, 3] / (N * gd)
        half = eta[len(ts) // 2:].mean(axis=0)
        res[k] = (ts, gm, (half.mean(), half.std(ddof=1) / np.sqrt(groups)))
        g.close()
    return res


Z_FAMILY, Z_EACH, FRAC_OVER = 4.0, 3.0, 0.01


def _judge(d, se_g, ref, se_o):
    z = abs(d) / np.sqrt(se_g * se_g + se_o * se_o) if (se_g > 0 or se_o > 0) else (0.0 if d == 0 else np.inf)
    resolved = se_o < 0.005 * abs(ref)
    rel = abs(d) / abs(ref) if resolved else None
    ok = z <= Z_FAMILY and (rel is None or rel <= 0.02)
    return z, rel, ok


def passes(zs, failures):
    """The criterion over a family of comparisons: no failure (z > 4 or a
    resolved value off by more than 2%) and at most 1% of the z above 3."""
    zs = np.asarray(zs, dtype=float)
    return not failures and (zs > Z_EACH).mean() <= FRAC_OVER if len(zs) else False


def compare_G(gpu, ref):
    """Per channel: lags compared, max lag, max z, max relative error where resolved, failures."""
    out = {}
    for ch in CHANNELS:
        zs, rels, fails, lags = [], [], [], []
        for lag in sorted(ref):
            if lag not in gpu or ch not in gpu[lag]:
                continue
            (gg, sg), (go, so) = gpu[lag][ch], ref[lag][ch]
            z, rel, ok = _judge(gg - go, sg, go, so)
            zs.append(z)
            lags.append(lag)
            if rel is not None:
                rels.append(rel)
            if not ok:
                fails.append((lag, gg, sg, go, so))
        out[ch] = {"lags_compared": len(zs), "max_lag_steps": max(lags) if lags else 0,
                   "max_z": float(max(zs)) if zs else None, "n_z_over_3": int(np.sum(np.array(zs) > Z_EACH)),
                   "max_rel_err_where_resolved": float(max(rels)) if rels else None,
                   "resolved_lags": len(rels), "failures": fails, "zs": zs}
    return out


def compare_eta(gpu, ref_steady, ref_logs, rates, N=32):
    """Per rate: eta+, N1 and <Z> at the reference's log times, and the steady viscosity."""
    out = {}
    for k, gd in enumerate(rates):
        ts, gm, (eg, sg) = gpu[k]
        G = gm.shape[1]
        idx = {int(t): i for i, t in enumerate(ts)}
        quantities = {"eta": gm[:, :, 3] / (N * gd), "N1": gm[:, :, 0] - gm[:, :, 1], "Z": gm[:, :, 12]}
        rec = {"gdot": gd}
        for qi, (name, arr) in enumerate(quantities.items()):
            zs, rels, fails = [], [], []
            for row in ref_logs[k]:
                step = int(row[0])
                if step not in idx:
                    continue
                v = arr[idx[step]]
                mg, sgm = v.mean(), v.std(ddof=1) / np.sqrt(G)
                mo, so = row[1 + 2 * qi], row[2 + 2 * qi]
                z, rel, ok = _judge(mg - mo, sgm, mo, so)
                zs.append(z)
                if rel is not None:
                    rels.append(rel)
                if not ok:
                    fails.append((step, mg, sgm, mo, so))
            rec[name] = {"times_compared": len(zs), "max_z": float(max(zs)) if zs else None,
                         "n_z_over_3": int(np.sum(np.array(zs) > Z_EACH)),
                         "max_rel_err_where_resolved": float(max(rels)) if rels else None, "failures": fails,
                         "zs": zs}
        go, so = ref_steady[k][1], ref_steady[k][2]
        z, rel, ok = _judge(eg - go, sg, go, so)
        rec["steady_eta"] = {"gpu": eg, "gpu_se": sg, "oracle": go, "oracle_se": so, "z": z, "rel_err": rel,
                             "ok": ok}
        out[k] = rec
    return out

"""Write the FP64 oracle's long-run reference observables (calls only oracle/).

    python tests/golden/make_longrun_reference.py [--quick]

Two workloads, the paper's parameters (N0 = 4, Ns = 0.5, zeta_s = 0.1,
dt = 0.01, b = kT = zeta = 1; Sec. 4.1), each from the equilibrium initial
state of Sec. 3.1:

* G(t): N = 32, 2048 chains (seed 61), 20000 steps of equilibration, then
  320000 steps into a 16 x 24 multiple-tau correlator.  For every lag slot
  with samples, the AUTO, CROSS and TOTAL channels of the relaxation modulus
  (Eq. relaxation_modulus_tensor_green_kubo_form with the virtual stress of
  App. B; averaged over xy, xz, yz; in rho0 kT, i.e. divided by N kT^2) with
  their standard errors over 32 chain groups.  -> longrun_G_oracle.txt
* The same equilibrium G(t) with the stochastic Heun integrator (integrator =
  1; Sec. 3.1's stochastic Runge-Kutta alternative): N = 32, 2048 chains (seed
  62), 20000 + 320000 steps.  -> longrun_G_heun_oracle.txt
* Startup shear (Sec. 4.1, viscosity growth): N = 32, 1024 chains per rate
  (seeds 71 + k), kappa_xy = gdot from step 0 for the 8 rates
  10^(-4 + 3k/7), 200000 steps, stress logged every 100 steps.  At about 100
  log-spaced log times: eta+ = <sigma_xy>/(N gdot) (rho0 kT tau0), the first
  normal stress difference <sigma_xx - sigma_yy> per chain and <Z>, each with
  its standard error over 32 chain groups; and per rate the steady viscosity,
  the mean of eta+ over the second half of the run with its standard error
  from the groups' time averages.  -> longrun_eta_oracle.txt

The chains are independent of any GPU run's (other seeds).  --quick writes
small versions to a temporary directory (a smoke test of this script).
"""
import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

G_SPEC = dict(N=32, M=2048, seed=61, equil=20000, steps=320000, levels=24, groups=32)
G_HEUN_SPEC = dict(G_SPEC, seed=62, integrator=1)
ETA_SPEC = dict(N=32, M=1024, seed0=71, steps=200000, log_every=100, groups=32,
                rates=[10 ** (-4 + 3 * k / 7) for k in range(8)])


def log_times(n_logs, n_pick=100):
    """Indices of about n_pick log-spaced logs out of n_logs (always the last)."""
    idx = np.unique(np.round(np.geomspace(1, n_logs, n_pick)).astype(int) - 1)
    return idx


def make_G(spec, out_path, nthreads=0):
    p = oracle.Params(N=spec["N"], integrator=spec.get("integrator", 0), **synth.PAPER)
    M, G, L = spec["M"], spec["groups"], spec["levels"]
    e = oracle.Ensemble(p, seed=spec["seed"], M=M, groups=G, levels=L)
    e.init()
    e.run(spec["equil"], nthreads=nthreads)
    e.reset_observables()
    e.run(spec["steps"], nthreads=nthreads)
    acc, n = e.corr_sums()  # [G][L][16][2][3]
    cnt = oracle.corr_counts(n, L)
    lags = oracle.corr_lags(L)
    per = np.array([(g + 1) * M // G - g * M // G for g in range(G)], dtype=float)
    rows = []
    for l in range(L):
        for k in range(16):
            if lags[l, k] < 0 or cnt[l, k] <= 0:
                continue
            norm = cnt[l, k] * per * p.N * p.kT * p.kT
            auto = acc[:, l, k, 0, :].sum(axis=-1) / 3.0 / norm
            total = acc[:, l, k, 1, :].sum(axis=-1) / 3.0 / norm
            row = [int(lags[l, k])]
            for v in (auto, total - auto, total):
                row += [v.mean(), v.std(ddof=1) / np.sqrt(G)]
            rows.append(row)
    rows.sort(key=lambda r: r[0])
    with open(out_path, "w") as f:
        f.write("# FP64 oracle relaxation modulus, equilibrium (Eq. relaxation_modulus_tensor_green_kubo_form,\n")
        if spec.get("integrator", 0):
            f.write("# stochastic Heun integrator\n")
        f.write("# App. B virtual stress), written by tests/golden/make_longrun_reference.py\n")
        f.write("# spec %r\n" % (spec,))
        f.write("# lag_steps G_auto se_auto G_cross se_cross G_total se_total  (rho0 kT; SE over %d groups)\n" % G)
        for r in rows:
            f.write("%d %s\n" % (r[0], " ".join("%.10e" % x for x in r[1:])))


def make_eta(spec, out_path, nthreads=0):
    N, M, G = spec["N"], spec["M"], spec["groups"]
    p = oracle.Params(N=N, **synth.PAPER)
    nlog = spec["steps"] // spec["log_every"]
    pick = log_times(nlog)
    per = np.array([(g + 1) * M // G - g * M // G for g in range(G)], dtype=float)
    lines, steady = [], []
    for k, gd in enumerate(spec["rates"]):
        e = oracle.Ensemble(p, seed=spec["seed0"] + k, M=M, groups=G, levels=1, log_every=spec["log_every"],
                            max_logs=nlog)
        e.init()
        e.set_flow(0, synth.shear_kappa(gd))
        e.run(spec["steps"], nthreads=nthreads)
        ts, L = e.logs()  # [n][G][14]: sums over each group's chains
        gm = L / per[None, :, None]  # group means
        eta = gm[:, :, 3] / (N * gd)
        n1 = gm[:, :, 0] - gm[:, :, 1]
        z = gm[:, :, 12]
        for i in pick:
            vals = []
            for v in (eta[i], n1[i], z[i]):
                vals += [v.mean(), v.std(ddof=1) / np.sqrt(G)]
            lines.append("%d %.10e %d %s" % (k, gd, int(ts[i]), " ".join("%.10e" % x for x in vals)))
        half = eta[nlog // 2:].mean(axis=0)  # each group's time average over the second half
        steady.append("%d %.10e %.10e %.10e" % (k, gd, half.mean(), half.std(ddof=1) / np.sqrt(G)))
    with open(out_path, "w") as f:
        f.write("# FP64 oracle startup shear (Sec. 4.1 viscosity growth), written by\n")
        f.write("# tests/golden/make_longrun_reference.py\n")
        f.write("# spec %r\n" % (spec,))
        f.write("# steady: rate_index gdot eta_steady se  (mean of eta+ over the second half of the run)\n")
        for s in steady:
            f.write("S %s\n" % s)
        f.write("# log: rate_index gdot step eta+ se N1 se Z se  (eta+ in rho0 kT tau0, N1 = <s_xx - s_yy>\n")
        f.write("#      per chain in kT, SE over %d groups)\n" % G)
        for ln in lines:
            f.write("L %s\n" % ln)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--only", choices=["G", "eta", "heun"], default=None)
    a = ap.parse_args()
    gs, es, out = dict(G_SPEC), dict(ETA_SPEC), HERE
    if a.quick:
        import tempfile
        out = tempfile.mkdtemp()
        gs.update(M=64, equil=100, steps=2000)
        es.update(M=64, steps=2000, rates=es["rates"][-2:])
    t = time.time()
    if a.only in (None, "G"):
        make_G(gs, os.path.join(out, "longrun_G_oracle.txt"), a.threads)
        print("G done %.0f s" % (time.time() - t), flush=True)
    if a.only in (None, "heun"):
        hs = dict(G_HEUN_SPEC)
        if a.quick:
            hs.update(M=64, equil=100, steps=2000)
        make_G(hs, os.path.join(out, "longrun_G_heun_oracle.txt"), a.threads)
        print("heun G done %.0f s" % (time.time() - t), flush=True)
    if a.only in (None, "eta"):
        make_eta(es, os.path.join(out, "longrun_eta_oracle.txt"), a.threads)
        print("eta done %.0f s" % (time.time() - t), flush=True)
    print(out)


if __name__ == "__main__":
    main()

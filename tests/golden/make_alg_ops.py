"""Write the algorithmic operation counts per bead-step (calls only oracle/).

    python tests/golden/make_alg_ops.py

The counting build of the FP64 oracle (-DOR_COUNT_OPS; the counting rules are
stated in oracle/ss_oracle.h) runs each workload's step single-threaded on a
sample of chains and divides the operations of the method, by substep, by the
bead-steps taken.  bench.py reads the result as the numerator of its ALU
roofline.  Workloads, the paper's parameters (Sec. 4.1):
  lve        N = 32, no flow (the benchmark workload), multiple-tau 16 x 24
  flow_N     N = 16, 24, 32, 48 under a traceless velocity gradient with
             N(0, 1e-2) entries (the batched multiscale workload's elements),
             stress logs every 100 steps; the batched path keeps no
             correlator, so its category is left out (0)
-> alg_ops.txt: one line per workload, "name total philox decode ...".
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(HERE, "alg_ops.txt")
SAMPLE = dict(M=256, steps=4000, warm=500)


def workloads():
    yield "lve", 32, None, 24, 0
    k = synth.element_table(1, seed=3, n_kappa=1)[2][0, 0]
    for N in (16, 24, 32, 48):
        yield "flow_%d" % N, N, k, 1, 100


def measure(name, N, kappa, levels, log_every, M, steps, warm):
    p = oracle.Params(N=N, **synth.PAPER)
    c = oracle.op_counts(p, seed=7, M=M, steps=steps, levels=levels, warm=warm, kappa=kappa, log_every=log_every)
    if name.startswith("flow_"):
        c["correlator"] = 0.0
    return c


def main():
    lines = ["# operations of the method per bead-step (oracle/ss_oracle.h counting rules), written by",
             "# tests/golden/make_alg_ops.py: counting build of the oracle, %d chains x %d steps after %d" % (
                 SAMPLE["M"], SAMPLE["steps"], SAMPLE["warm"]),
             "# name total " + " ".join(oracle.OPS_CATEGORIES)]
    for name, N, kappa, levels, log_every in workloads():
        c = measure(name, N, kappa, levels, log_every, **SAMPLE)
        lines.append("%s %.4f %s" % (name, sum(c.values()), " ".join("%.4f" % c[k] for k in oracle.OPS_CATEGORIES)))
        print(lines[-1], flush=True)
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")


def load(path=OUT):
    """{name: {"total": x, category: x, ...}}"""
    out = {}
    cats = None
    for ln in open(path):
        if ln.startswith("# name"):
            cats = ln.split()[2:]
            continue
        if ln.startswith("#") or not ln.strip():
            continue
        f = ln.split()
        out[f[0]] = dict(zip(cats, [float(x) for x in f[1:]]))
    return out


if __name__ == "__main__":
    main()

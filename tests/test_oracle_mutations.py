"""Mutation checks of the oracle's pins (CPU only).

Each case plants one plausible mistake in a copy of oracle/ss_oracle.c (a
transposed velocity gradient, a missing dt, a flow schedule that switches one
step early or late, a wrong anchor spread for new springs, a wrong noise
amplitude, a wrong Glauber exponent ...), compiles the copy in a temporary
directory and runs the pins that must catch it against that copy in a child
process (SS_ORACLE_LIB points the oracle binding at it).  Every listed pin has
to fail.  The committed oracle is untouched; the same pins pass on it in the
other test files.
"""
import json
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

from oracle import build as obuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

BEAD_FLOW = ("double flow = kap[3 * a + 0] * c->R[i][0] + kap[3 * a + 1] * c->R[i][1] +\n"
             "                          kap[3 * a + 2] * c->R[i][2];")
ANCHOR_FLOW = ("double flow = kap[3 * a + 0] * c->A[j][0] + kap[3 * a + 1] * c->A[j][1] +\n"
               "                          kap[3 * a + 2] * c->A[j][2];")
NEW_SPREAD = "        double sa = sqrt(p->kT / p->k_s);\n        for (int j = first; j < last; ++j) {"

# (name, text in ss_oracle.c, replacement, pins that must fail: module::function)
MUTATIONS = [
    ("bead kappa transposed", BEAD_FLOW,
     BEAD_FLOW.replace("3 * a + 0", "a + 0").replace("3 * a + 1", "a + 3").replace("3 * a + 2", "a + 6"),
     ["test_oracle_flow::test_frozen_beads_follow_linear_flow_map",
      "test_oracle_flow::test_sheared_rouse_steady_stress_matches_lyapunov"]),
    ("anchor kappa transposed", ANCHOR_FLOW,
     ANCHOR_FLOW.replace("3 * a + 0", "a + 0").replace("3 * a + 1", "a + 3").replace("3 * a + 2", "a + 6"),
     ["test_oracle_flow::test_frozen_anchors_follow_linear_flow_map"]),
    ("bead flow without dt", "mob * F[i][a] + p->dt * flow", "mob * F[i][a] + flow",
     ["test_oracle_flow::test_frozen_beads_follow_linear_flow_map",
      "test_oracle_flow::test_sheared_rouse_steady_stress_matches_lyapunov"]),
    ("bead flow with the wrong sign", "mob * F[i][a] + p->dt * flow", "mob * F[i][a] - p->dt * flow",
     ["test_oracle_flow::test_frozen_beads_follow_linear_flow_map",
      "test_oracle_flow::test_sheared_rouse_steady_stress_matches_lyapunov"]),
    ("anchor advection without dt", "An[j][a] = c->A[j][a] + p->dt * flow;", "An[j][a] = c->A[j][a] + flow;",
     ["test_oracle_flow::test_frozen_anchors_follow_linear_flow_map",
      "test_oracle_flow::test_flow_schedule_switches_exactly_at_from_step"]),
    ("schedule switches a step early", "if (e->flow[i].from <= t) k = e->flow[i].k;",
     "if (e->flow[i].from <= t + 1) k = e->flow[i].k;",
     ["test_oracle_flow::test_flow_schedule_switches_exactly_at_from_step"]),
    ("schedule switches a step late", "if (e->flow[i].from <= t) k = e->flow[i].k;",
     "if (e->flow[i].from < t) k = e->flow[i].k;",
     ["test_oracle_flow::test_flow_schedule_switches_exactly_at_from_step"]),
    ("new springs with the bond spread", NEW_SPREAD, NEW_SPREAD.replace("p->k_s", "p->k_b"),
     ["test_oracle_flow::test_spring_vector_variance_in_dynamics_with_frozen_beads"]),
    ("noise amplitude without the 2", "sqrt(2.0 * p->kT * p->dt / p->zeta)", "sqrt(p->kT * p->dt / p->zeta)",
     ["test_oracle_observables::test_rouse_closed_form_autocorrelation"]),
    ("Heun corrector with the full mobility", "const double hmob = 0.5 * mob, hdt = 0.5 * p->dt;",
     "const double hmob = mob, hdt = 0.5 * p->dt;",
     ["test_oracle_heun::test_heun_rouse_closed_form_autocorrelation"]),
    ("Heun corrector flow without the half", "const double hmob = 0.5 * mob, hdt = 0.5 * p->dt;",
     "const double hmob = 0.5 * mob, hdt = p->dt;",
     ["test_oracle_heun::test_heun_frozen_beads_and_anchors_follow_second_order_flow_map",
      "test_oracle_heun::test_heun_sheared_rouse_matches_lyapunov"]),
    ("Heun corrector forces at the start state", "if (i > 0) f += p->k_b * (Rn[i - 1][a] - Rn[i][a]);",
     "if (i > 0) f += p->k_b * (c->R[i - 1][a] - c->R[i][a]);",
     ["test_oracle_heun::test_heun_rouse_closed_form_autocorrelation"]),
    ("Glauber exponent doubled", "p->k_s * (d_new - d_old) / (4.0 * p->kT)",
     "p->k_s * (d_new - d_old) / (2.0 * p->kT)",
     ["test_oracle_model::test_hop_detailed_balance_frozen_beads",
      "test_oracle_flow::test_spring_vector_variance_in_dynamics_with_frozen_beads"]),
]

_RUNNER = r"""
import json, sys, traceback
sys.path.insert(0, %(root)r)
sys.path.insert(0, %(tests)r)
out = {}
for spec in %(pins)r:
    mod, fn = spec.split("::")
    m = __import__(mod)
    try:
        getattr(m, fn)()
        out[spec] = "passed"
    except AssertionError as e:
        out[spec] = "failed: " + repr(e)[:200]
print(json.dumps(out))
"""


@pytest.mark.slow
@pytest.mark.parametrize("name,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_its_pins(name, old, new, pins):
    src = open(obuild.SRC).read()
    assert src.count(old) == 1, "mutation site not found once: %r" % old
    d = tempfile.mkdtemp(prefix="ss_oracle_mut_")
    try:
        shutil.copy(obuild.HDR, d)
        with open(os.path.join(d, "ss_oracle.c"), "w") as f:
            f.write(src.replace(old, new))
        lib = obuild.compile_oracle(os.path.join(d, "ss_oracle.c"), os.path.join(d, "libssoracle_mut.so"))
        code = _RUNNER % {"root": ROOT, "tests": os.path.join(ROOT, "tests"), "pins": pins}
        r = subprocess.run([sys.executable, "-c", code], env={**os.environ, "SS_ORACLE_LIB": lib},
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-3000:]
        res = json.loads(r.stdout.strip().splitlines()[-1])
        survived = [k for k, v in res.items() if not v.startswith("failed")]
        assert not survived, "%s: pins passed on the mutated oracle: %s" % (name, survived)
    finally:
        shutil.rmtree(d, ignore_errors=True)

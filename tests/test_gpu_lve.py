"""Linear viscoelasticity at the paper's longest chains (GPU, FP32 beads / FP64 sums).

The plateau modulus: the paper reads G_N ~ 0.1 rho0 kT (so N_e = rho0 kT / G_N
~ 10, Eq. entanglement_bead_number_rubber_elasticity_definition) from the
plateau of the linear-viscoelastic data of equilibrium runs up to N = 80.
Here the plateau of the TOTAL-channel G(t) at N = 80 (the value where ln G is
flattest in ln t) is checked against that printed value as a +-30% sanity
band (printed numbers of the paper are qualitative).
"""
import numpy as np
import pytest

import synth
from paper_1106_2899_gb300 import SlipSpring

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu(cuda_ok):
    from paper_1106_2899_gb300 import build
    build.build()
    yield


@pytest.mark.slow
def test_plateau_modulus_at_N80():
    N, M, steps = 80, 16384, 200000
    g = SlipSpring([(M, N)], precision="fp32", seed=N)
    g.set_params(**synth.PAPER, corr_levels=20, groups=32)
    g.run(5000)
    g.reset_observables()
    g.run(steps)
    assert g.status() == 0
    t, G, se = g.correlator("total")
    order = np.argsort(t)
    t, G, se = t[order], G[order], se[order]
    # the plateau: G where ln G(t) is flattest over a factor 4 in time, 1 <= t <= 1000
    sel = (t >= 1) & (t <= 1000) & (G > 0) & (se < 0.05 * G)
    lt, lg = np.log(t[sel]), np.log(G[sel])
    slopes, vals = [], []
    for j in range(len(lt)):
        k = np.searchsorted(lt, lt[j] + np.log(4.0))
        if k >= len(lt):
            break
        slopes.append(abs((lg[k] - lg[j]) / (lt[k] - lt[j])))
        vals.append(np.exp(0.5 * (lg[j] + lg[k])))
    i = int(np.argmin(slopes))
    GN = vals[i]
    print("\nN=80: plateau G = %.4f rho0 kT (log-slope %.3f); N_e = %.1f" % (GN, slopes[i], 1.0 / GN))
    assert slopes[i] < 0.2  # a plateau region exists
    assert 0.07 <= GN <= 0.13, GN

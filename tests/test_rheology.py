"""Post-processing formulas (Sec. 4.1) against closed forms (CPU).

A Maxwell mode G(t) = g exp(-t/tau) has G' = g (w tau)^2 / (1 + (w tau)^2),
G'' = g w tau / (1 + (w tau)^2), eta0 = g tau and tau_d = tau; a sum of modes
is linear in each.  The grid mimics the multiple-tau lag grid (dense at short
lags, sparse at long ones).
"""
import numpy as np

from paper_1106_2899_gb300 import rheology


def _multitau_grid(dt=0.01, levels=22):
    lags = [k for k in range(16)]
    for l in range(1, levels):
        lags += [k << l for k in range(8, 16)]
    return np.array(sorted(set(lags))) * dt


def test_maxwell_modes_closed_forms():
    t = _multitau_grid()
    modes = [(0.7, 0.3), (0.2, 5.0), (0.1, 40.0)]
    G = sum(g * np.exp(-t / tau) for g, tau in modes)
    w = np.logspace(-2, 1, 13)
    Gp, Gpp = rheology.storage_loss_moduli(t, G, w)
    Gp_x = sum(g * (w * tau) ** 2 / (1 + (w * tau) ** 2) for g, tau in modes)
    Gpp_x = sum(g * w * tau / (1 + (w * tau) ** 2) for g, tau in modes)
    assert np.allclose(Gp, Gp_x, rtol=0.03, atol=2e-3)
    assert np.allclose(Gpp, Gpp_x, rtol=0.03, atol=2e-3)
    assert abs(rheology.zero_shear_viscosity(t, G) - sum(g * tau for g, tau in modes)) < 0.01 * 4.2
    assert abs(rheology.longest_relaxation_time(t, G, t_min=300.0) - 40.0) < 0.5
    eta = rheology.dynamic_viscosity(Gp_x, Gpp_x, w)
    assert np.allclose(eta, np.abs(sum(g * tau / (1 + 1j * w * tau) for g, tau in modes)), rtol=1e-12)


def test_eta_plus_and_steady_viscosity():
    sig = np.full(200, 3.2)
    e = rheology.eta_plus(sig, N=32, gdot=0.01)
    assert np.allclose(e, 10.0)
    m, se = rheology.steady_viscosity(np.r_[np.linspace(0, 10, 100), 10 + 0.01 * np.sin(np.arange(100))])
    assert abs(m - 10) < 0.01 and se < 0.01

"""Host-side analysis of the library's outputs (Sec. 4.1).

These are the paper's post-processing formulas applied to G(t) from the
multiple-tau correlator (`SlipSpring.correlator`) and to stress logs
(`SlipSpring.stress`); they run on the host in FP64 NumPy.

* G'(w) = w int_0^inf G(t) sin(w t) dt, G''(w) = w int_0^inf G(t) cos(w t) dt
  (Eqs. storage_modulus_definition, loss_modulus_definition) by the
  trapezoidal rule applied to the piecewise-linear interpolant of G, i.e. the
  exact transform of that interpolant, so that the sparse long-lag grid of the
  multiple-tau correlator does not alias at high frequency
* eta0 = int_0^inf G(t) dt (Sec. 4.1, zero-shear viscosity)
* 1/tau_d = -lim ln G(t)/t, estimated as the slope of ln G over the tail
* |eta*(w)| = sqrt(G'^2 + G''^2)/w for the Cox-Merz comparison (Eq.
  dynamic_viscosity_definition prints sqrt(G'^2+G''^2); the 1/w that makes it a
  viscosity is restored)
* eta+(t, gdot) = <sigma_xy>(t)/(N gdot) from the chain-averaged stress, and
  the steady viscosity as its mean over the last part of a run.
"""
import numpy as np


def _trap(y, x):
    f = getattr(np, "trapezoid", None) or np.trapz
    return f(y, x)


def _grid(t, G):
    t = np.asarray(t, dtype=float)
    G = np.asarray(G, dtype=float)
    order = np.argsort(t)
    return t[order], G[order]


def _fourier_piecewise_linear(t, G, w):
    """int G(t) e^{i w t} dt over [t0, t_end] for G linear between samples:
    per segment the exact integral of the linear interpolant (the trapezoidal
    rule applied to the interpolant); short segments (w h < 1e-2) use the plain
    trapezoid, which agrees to O((w h)^2)."""
    a, b = t[:-1], t[1:]
    ga, gb = G[:-1], G[1:]
    h = b - a
    ea, eb = np.exp(1j * w * a), np.exp(1j * w * b)
    short = w * h < 1e-2
    with np.errstate(divide="ignore", invalid="ignore"):
        slope = (gb - ga) / h
        exact = (gb * eb - ga * ea) / (1j * w) + slope * (eb - ea) / (w * w)
    trap = 0.5 * h * (ga * ea + gb * eb)
    return np.sum(np.where(short, trap, exact))


def storage_loss_moduli(t, G, omega):
    """(G'(w), G''(w)) for each w in omega from G sampled at lags t (t[0] = 0),
    G taken linear between samples and zero beyond the last one."""
    t, G = _grid(t, G)
    w = np.atleast_1d(np.asarray(omega, dtype=float))
    Gp, Gpp = np.zeros(len(w)), np.zeros(len(w))
    for i, wi in enumerate(w):
        I = _fourier_piecewise_linear(t, G, wi)
        Gp[i] = wi * I.imag
        Gpp[i] = wi * I.real
    return Gp, Gpp


def zero_shear_viscosity(t, G):
    """eta0 = integral of G over the sampled lags."""
    t, G = _grid(t, G)
    return float(_trap(G, t))


def longest_relaxation_time(t, G, t_min, t_max=None):
    """tau_d from a least-squares line through ln G(t) for t_min <= t <= t_max
    (lags with G > 0 only)."""
    t, G = _grid(t, G)
    sel = (t >= t_min) & (G > 0)
    if t_max is not None:
        sel &= t <= t_max
    if sel.sum() < 2:
        raise ValueError("need at least two positive samples in the fit window")
    slope, _ = np.polyfit(t[sel], np.log(G[sel]), 1)
    return float(-1.0 / slope)


def dynamic_viscosity(Gp, Gpp, omega):
    """|eta*(w)| = sqrt(G'^2 + G''^2) / w."""
    return np.sqrt(np.asarray(Gp) ** 2 + np.asarray(Gpp) ** 2) / np.asarray(omega, dtype=float)


def eta_plus(mean_sigma_xy, N, gdot):
    """eta+(t) in rho0 kT tau0 from the chain-averaged sigma_xy (units of kT)."""
    return np.asarray(mean_sigma_xy, dtype=float) / (N * gdot)


def steady_viscosity(eta_plus_t, tail=0.5):
    """Mean and batch-means standard error of eta+ over the last `tail` of the run."""
    x = np.asarray(eta_plus_t, dtype=float)
    x = x[int(len(x) * (1 - tail)):]
    nb = max(2, min(16, len(x) // 4))
    batches = np.array_split(x, nb)
    means = np.array([b.mean() for b in batches])
    return float(x.mean()), float(means.std(ddof=1) / np.sqrt(nb))

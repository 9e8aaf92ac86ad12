"""Pathwise gradients of a G(t)-fit loss with respect to (k_b, k_s, zeta).

The paper fixes the bond stiffness k_b = 3kT/b^2, the slip-spring stiffness
k_s = 3kT/(N_s b^2) and the bead friction zeta (Sec. 3.1, Eqs. of the bead
Langevin equation); fitting them to a measured relaxation modulus needs the
derivative of G(t) (Eq. relaxation_modulus_tensor_green_kubo_form, App. B) with
respect to them.  The derivative taken here is the pathwise one with every
discrete decision (hop, creation, destruction) frozen along the trajectory:
the forward window records the decisions, and the library's adjoint kernels
run backwards through the continuous update with checkpoint-and-recompute.

    ens = SlipSpring([(8192, 24)], precision="fp32", seed=1)
    ens.set_params(**PAPER, corr_levels=14, chunk_steps=1024)
    ens.run(2000)                                  # equilibrate
    start = ens.get_state()
    fit = GFit(ens, start, n_steps=10000, checkpoint_every=256, target=G_target)
    theta = torch.tensor([3.0, 6.0, 1.0], dtype=torch.float64, requires_grad=True)
    loss = fit(theta)
    loss.backward()                                # theta.grad = dL/d(k_b, k_s, zeta)

The loss is sum over the fitted slots of (ln G - ln G_target)^2 in FP64; the
fitted slots are those where G > 0, G_target > 0 and the standard error of G
is below a fraction of G (20% by default), taken from the first evaluation
unless given.
"""
import numpy as np
import torch


def slot_counts(n_samples, levels, points=16):
    """Number of later x origin products of each multiple-tau slot [levels][points]
    after n_samples samples: max(0, floor(n / 2^l) - k), level 0 lags 0..15 and
    level l >= 1 lags 8..15 (the lower half repeats the level below)."""
    cnt = np.zeros((levels, points), dtype=np.int64)
    for l in range(levels):
        for k in range(0 if l == 0 else points // 2, points):
            cnt[l, k] = max(0, (n_samples >> l) - k)
    return cnt


def slot_lags(levels, points=16):
    """Lag in steps of each slot [levels][points] (-1 for the unused lower half)."""
    lag = -np.ones((levels, points), dtype=np.int64)
    for l in range(levels):
        for k in range(0 if l == 0 else points // 2, points):
            lag[l, k] = k << l
    return lag


def window_G(ens, elem=0):
    """(G, sem, counts) of the TOTAL channel per slot [levels][16]: the modulus
    in rho0 kT and its standard error over groups as ss_correlator returns them,
    NaN where a slot has no products yet."""
    _, n = ens.corr_sums(elem)
    levels = (ens.params or {}).get("corr_levels", 0) or 24
    cnt = slot_counts(n, levels)
    _, g, se = ens.correlator("total", elem)
    G = np.full((levels, 16), np.nan)
    sem = np.full((levels, 16), np.nan)
    ok = cnt > 0  # ss_correlator lists exactly these slots, level by level
    G[ok] = g
    sem[ok] = se
    return G, sem, cnt


def fit_mask(G, sem, target, max_rel_se=0.2):
    """Slots fitted by the log loss: both moduli positive and resolved."""
    with np.errstate(invalid="ignore"):
        m = np.isfinite(G) & np.isfinite(target) & (G > 0) & (target > 0)
        m &= np.isfinite(sem) & (sem < max_rel_se * np.abs(G))
    return m


def log_loss(G, target, mask):
    """(L, dL/dG) of L = sum_mask (ln G - ln G_target)^2."""
    d = np.zeros_like(G)
    r = np.log(G[mask]) - np.log(target[mask])
    d[mask] = 2.0 * r / G[mask]
    return float(np.sum(r * r)), d


class GFit:
    """Loss of one differentiation window as a function of theta = (k_b, k_s, zeta).

    Every evaluation restarts from `start_state` at the same step index, so
    evaluations at different theta use the same Gaussian noise; with
    replay=True they also reuse the decisions of the last recorded window (the
    frozen-decision surrogate that finite differences of the pathwise gradient
    must use)."""

    def __init__(self, ens, start_state, n_steps, checkpoint_every=256, target=None, mask=None,
                 max_rel_se=0.2):
        if target is None:
            raise ValueError("a target G [levels][16] is required")
        self.ens = ens
        self.start = start_state
        self.t0 = ens.step
        self.n = int(n_steps)
        self.ce = int(checkpoint_every)
        self.target = np.asarray(target, dtype=np.float64)
        self.mask = mask
        self.max_rel_se = max_rel_se
        self.G = self.sem = None

    def evaluate(self, theta, replay=False):
        """Run the window at theta; return (L, dL/dG)."""
        k_b, k_s, zeta = (float(v) for v in theta)
        self.ens.set_coefficients(k_b, k_s, zeta)
        self.ens.set_state(self.start)
        self.ens.step = self.t0
        self.ens.window_forward(self.n, self.ce, replay=replay)
        self.G, self.sem, _ = window_G(self.ens)
        if self.mask is None:
            self.mask = fit_mask(self.G, self.sem, self.target, self.max_rel_se)
        return log_loss(self.G, self.target, self.mask)

    def gradient(self, dL_dG):
        """dL/d(k_b, k_s, zeta) of the last evaluated window."""
        return self.ens.window_backward(dL_dG)

    def __call__(self, theta):
        return _GFitLoss.apply(theta, self)


class _GFitLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, fit):
        th = theta.detach().cpu().double().numpy()
        loss, dL_dG = fit.evaluate(th)
        ctx.fit = fit
        ctx.dL_dG = dL_dG
        ctx.theta_meta = (theta.dtype, theta.device)
        return torch.tensor(loss, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        g = ctx.fit.gradient(ctx.dL_dG)
        dtype, device = ctx.theta_meta
        return torch.as_tensor(g, dtype=torch.float64, device=device).to(dtype) * grad_out.to(dtype), None

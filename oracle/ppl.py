"""Proximal-Perturbed Lagrangian update and adaptive time stepping (oracle)."""
import math

import numpy as np


class PPL:
    """Constraint handling of Sec. 5.4.

    Lagrangian (eq. lagrangian):
        L = J + <lambda, C - 1> + <mu, z> + alpha/2 |z|^2 + beta/2 |lambda - mu|^2.
    One update (eq. lag_method), i = 1, 2, ...:
        mu^i     = mu^{i-1} + delta^{i-1} (lambda^{i-1} - mu^{i-1}) / (|lambda^{i-1} - mu^{i-1}|^2 + 1)
        lambda^i = mu^i + alpha / (1 + alpha beta) (C(Omega^i) - 1)
        z^i      = (lambda^i - mu^i) / alpha
        delta^i  = r delta^{i-1}
    Defaults r = 0.999, delta0 = 0.5, alpha = 2000, beta = 0.5, z0 = lambda0 = mu0 = 0.
    """

    def __init__(self, nc, r=0.999, delta0=0.5, alpha=2000.0, beta=0.5):
        self.r, self.alpha, self.beta = r, alpha, beta
        self.delta = delta0
        self.z = np.zeros(nc)
        self.lam = np.zeros(nc)
        self.mu = np.zeros(nc)

    def update(self, C, J):
        C = np.atleast_1d(np.asarray(C, dtype=np.float64))
        diff = self.lam - self.mu
        self.mu = self.mu + self.delta * diff / (diff @ diff + 1.0)
        self.lam = self.mu + self.alpha / (1.0 + self.alpha * self.beta) * (C - 1.0)
        self.z = (self.lam - self.mu) / self.alpha
        self.delta = self.r * self.delta
        return self.lam.copy(), self.lagrangian(C, J)

    def lagrangian(self, C, J):
        lm = self.lam - self.mu
        return float(J + self.lam @ (C - 1.0) + self.mu @ self.z
                     + 0.5 * self.alpha * (self.z @ self.z) + 0.5 * self.beta * (lm @ lm))


def adaptime(Btt, dfactor=1e-2, lv_time=(1e-3, 1e-1), lv_iter=(8, 16), floor=1e-12):
    """Final time and number of transport steps (Sec. 5.7, eqs tend and steps).

    t_end = dfactor / B(theta, theta) with B(theta, theta) bounded below by
    ``floor``; t_end is clamped to [t_min, t_max] before eq. steps
        s = (s_max - s_min) ((t_end - t_min) / (t_max - t_min))^(1/6) + s_min,
    s is clamped to [s_min, s_max] and rounded half away from zero.
    """
    tmin, tmax = lv_time
    smin, smax = lv_iter
    t_end = dfactor / max(Btt, floor)
    t_end = min(max(t_end, tmin), tmax)
    s = (smax - smin) * ((t_end - tmin) / (tmax - tmin)) ** (1.0 / 6.0) + smin
    s = min(max(s, smin), smax)
    return t_end, int(math.floor(s + 0.5))


def stop_check(values, C=None, start_to_check=30, tol=1e-2, ctrn_tol=1e-2, prev=10):
    """Stopping criterion of Sec. 5.7 at iteration i = len(values) - 1.

    values: J(Omega^0..i) for a problem without constraints, L(Omega^0..i, ...) with them; C:
    the constraint vector C(Omega^i) (None without constraints).  Stops when i > start_to_check
    and max_{j in I(i)} |v_i - v_j| < tol |v_i| with I(i) = {i - prev, ..., i - 1}, and, with
    constraints, also |C - 1|_inf < ctrn_tol.
    """
    i = len(values) - 1
    if i <= start_to_check or i < prev:
        return False
    vi = values[i]
    spread = max(abs(vi - values[j]) for j in range(i - prev, i))
    if not spread < tol * abs(vi):
        return False
    if C is not None and len(np.atleast_1d(C)):
        return bool(np.max(np.abs(np.atleast_1d(C) - 1.0)) < ctrn_tol)
    return True

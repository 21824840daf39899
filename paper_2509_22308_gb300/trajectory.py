"""Design maps and low-Reynolds-number trajectories of Janus cylinders (arXiv 2509.22308,
Sec. IV.A-C).

A design map is the non-dimensional drag, lift and torque over the interface
orientation phi0 (and the material parameters), computed by the batched CUDA path: one
instance per map cell, all in one persistent kernel.  A trajectory integrates the
force- and torque-free motion of a slender cylinder at low Reynolds number (Sec. IV.C):

    dx~/dt~ = ln(l/a) / (4 pi) F~x(phi0),   dy~/dt~ = ln(l/a) / (4 pi) F~y(phi0),
    dphi0/dt~ = M~z(phi0) / (2 pi),

with F~, M~ interpolated periodically in phi0 from a map.  The ODE is three scalars per
step and runs on the host; only the map comes from the GPU.
"""
from __future__ import annotations

import math

import numpy as np


class PeriodicMap:
    """F~x, F~y, M~z sampled at phi0_k = 2 pi k / n, interpolated by the trigonometric
    polynomial through the samples (exact for band-limited maps)."""

    def __init__(self, fx, fy, mz):
        self.coef = [np.fft.rfft(np.asarray(v, dtype=float)) for v in (fx, fy, mz)]
        self.n = len(fx)

    def __call__(self, phi0):
        phi0 = np.atleast_1d(np.asarray(phi0, dtype=float))
        n = self.n
        m = np.arange(len(self.coef[0]))
        basis = np.exp(1j * np.outer(phi0, m))
        out = []
        for c in self.coef:
            w = np.full(len(m), 2.0 / n)
            w[0] = 1.0 / n
            if n % 2 == 0:
                w[-1] = 1.0 / n
            out.append(np.real(basis @ (c * w)))
        return np.stack(out, axis=-1)


def design_map(eps1, eps2=1.0, pec2=False, n_phi=36, a=32, wavelength=None, periods=30, grid=None,
               precision="f32", conv_tol=0.0, stream=None):
    """F~x, F~y, M~z [n_phi, 3] at phi0_k = 2 pi k / n_phi for one material pair, from one
    batched GPU run (a/lambda = 1 by default, lattice 16 a, contour radius 1.6 a)."""
    from paper_2509_22308_gb300 import lbm_em as L
    lam = a if wavelength is None else wavelength
    n = grid if grid is not None else 16 * a
    T = int(round(3 * lam))
    insts = [dict(nx=n, ny=n, a=float(a), phi0=2 * math.pi * k / n_phi, eps1=float(eps1), eps2=float(eps2),
                  pec2=bool(pec2), period=T, periods=periods, R=1.6 * a, ramp=T) for k in range(n_phi)]
    b = L.Batch(insts, precision, stream=stream, conv_tol=conv_tol, min_periods=min(8, periods))
    try:
        b.run()
        F, _ = b.results()
    finally:
        b.close()
    return F


def janus_map(materials, phi0_values, *, a=40, L_over_a=4, a_over_lambda=1.0, R_over_a=1.5, periods=30,
              precision="f32", conv_tol=0.0, min_periods=8, stream=None, chunk=4096):
    """F~x, F~y, M~z [len(materials), len(phi0_values), 3] and the steps each instance ran
    [len(materials), len(phi0_values)], for every (material, orientation) pair, from batched
    GPU runs of at most ``chunk`` instances each.

    ``materials`` is a list of (eps1, eps2, pec2).  Defaults are the paper's force
    resolution for metallo-dielectric cylinders (Sec. III: a/dx = 40, L/a = 4, a/lambda = 1);
    dielectric Janus maps use a = 50.  With ``conv_tol`` > 0 each instance stops once its
    energy has settled (at least ``min_periods``, at most ``periods``)."""
    from paper_2509_22308_gb300 import lbm_em as L
    n = int(round(L_over_a * a))
    T = int(round(3 * a / a_over_lambda))
    insts = [dict(nx=n, ny=n, a=float(a), phi0=float(p), eps1=float(e1), eps2=float(e2), pec2=bool(pec),
                  period=T, periods=periods, R=R_over_a * a, ramp=T)
             for (e1, e2, pec) in materials for p in phi0_values]
    F = np.empty((len(insts), 3))
    steps = np.empty(len(insts), dtype=np.int64)
    for lo in range(0, len(insts), chunk):
        b = L.Batch(insts[lo:lo + chunk], precision, stream=stream, conv_tol=conv_tol,
                    min_periods=min(min_periods, periods))
        try:
            b.run()
            F[lo:lo + chunk], _ = b.results()
            steps[lo:lo + chunk] = b.steps()
        finally:
            b.close()
    shape = (len(materials), len(phi0_values))
    return F.reshape(shape + (3,)), steps.reshape(shape)


def md_janus_map(eps1_values, phi0_values, **kw):
    """Sec. IV.A map: dielectric half eps_r1, the other half PEC (paper: eps_r1 = 1 ... 5 in
    steps of 0.04, phi0 = 0 ... 2 pi in steps of pi/90, a/dx = 40, L/a = 4)."""
    return janus_map([(e, 1.0, True) for e in eps1_values], phi0_values, **kw)


def dielectric_janus_map(eps1, ratios, phi0_values, **kw):
    """Sec. IV.B map at fixed eps_r1: eps_r2 = ratio * eps_r1 (paper: eps_r1 in {1, 2, 5},
    ratio = 1 ... 5 in steps of 0.04, phi0 in steps of pi/90, a/dx = 50, L/a = 4)."""
    kw.setdefault("a", 50)
    return janus_map([(eps1, r * eps1, False) for r in ratios], phi0_values, **kw)


def integrate(fmap, phi0_init, t_final=1.0e4, log_l_over_a=math.log(10.0), dt=1.0, x0=0.0, y0=0.0):
    """RK4 trajectory (t~, x~, y~, phi0) from (x0, y0, phi0_init) to t~ = t_final (Sec. IV.C
    starts at the origin and integrates to 10^4)."""
    k = log_l_over_a / (4.0 * math.pi)

    def rhs(s):
        F = fmap(s[2])[0]
        return np.array([k * F[0], k * F[1], F[2] / (2.0 * math.pi)])

    n = int(math.ceil(t_final / dt))
    out = np.empty((n + 1, 4))
    s = np.array([x0, y0, phi0_init], dtype=float)
    out[0] = (0.0, *s)
    for i in range(n):
        h = min(dt, t_final - i * dt)
        k1 = rhs(s)
        k2 = rhs(s + 0.5 * h * k1)
        k3 = rhs(s + 0.5 * h * k2)
        k4 = rhs(s + h * k3)
        s = s + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
        out[i + 1] = (min((i + 1) * dt, t_final), *s)
    return out


def torque_free_orientations(fmap, n=4096):
    """Orientations with M~z = 0 and whether each is stable (dM~z/dphi0 < 0), found by
    sign changes on a fine grid refined by bisection."""
    phi = 2 * math.pi * np.arange(n + 1) / n
    M = fmap(phi)[:, 2]
    roots = []
    for i in range(n):
        if M[i] == 0.0 or M[i] * M[i + 1] < 0.0:
            lo, hi = phi[i], phi[i + 1]
            for _ in range(60):
                mid = 0.5 * (lo + hi)
                if fmap(lo)[0, 2] * fmap(mid)[0, 2] <= 0.0:
                    hi = mid
                else:
                    lo = mid
            r = 0.5 * (lo + hi)
            slope = (fmap(r + 1e-6)[0, 2] - fmap(r - 1e-6)[0, 2]) / 2e-6
            roots.append((r % (2 * math.pi), slope < 0.0))
    return roots

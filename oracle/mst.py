"""Oracle (test infrastructure only): period-averaged Maxwell stress tensor on a contour.

arXiv 2509.22308, Sec. II.B:
  <T> = 1/2 Re[eps0 E E* + mu0 H H* - 1/2 (eps0 |E|^2 + mu0 |H|^2) I]   (Eq. stress tensor average)
  <F> = closed integral of <T> . n dl                                     (Eq. force)
  <M> = closed integral of r x (<T> . n) dl                              (Eq. torque)
  F~ = <F> / F0, M~ = <M> / M0 with F0 = pi a eps0 E0^2 / 4, M0 = 2 F0 a (Sec. II.B)
Lattice units eps0 = mu0 = 1.  For TM^z fields E = (0, 0, Ez), H = (Hx, Hy, 0).

The contour (the paper integrates over any enclosing vacuum contour): a circle of radius R about the
cylinder axis sampled at N points phi_k = 2 pi k / N, dl = R 2 pi / N, the
phasors at each point bilinearly interpolated from the four surrounding sites.
"""
from __future__ import annotations

import numpy as np


def contour_points(cx, cy, R, n_points):
    phi = 2.0 * np.pi * np.arange(n_points) / n_points
    return cx + R * np.cos(phi), cy + R * np.sin(phi), phi


def bilinear(field, px, py):
    """Bilinear interpolation of a [ny, nx] array at lattice coordinates (px, py)."""
    i = np.floor(px).astype(np.int64)
    j = np.floor(py).astype(np.int64)
    fx = px - i
    fy = py - j
    return ((1 - fx) * (1 - fy) * field[j, i] + fx * (1 - fy) * field[j, i + 1]
            + (1 - fx) * fy * field[j + 1, i] + fx * fy * field[j + 1, i + 1])


def stress_dot_n(Ez, Hx, Hy, nx_, ny_):
    """<T> . n for complex phasors (Eq. stress tensor average), eps0 = mu0 = 1."""
    E2 = np.abs(Ez) ** 2
    H2 = np.abs(Hx) ** 2 + np.abs(Hy) ** 2
    # full 3x3 tensor restricted to the in-plane rows; E has only a z component
    Txx = 0.5 * (np.abs(Hx) ** 2 - 0.5 * (E2 + H2))
    Tyy = 0.5 * (np.abs(Hy) ** 2 - 0.5 * (E2 + H2))
    Txy = 0.5 * np.real(Hx * np.conj(Hy))
    return Txx * nx_ + Txy * ny_, Txy * nx_ + Tyy * ny_


def force_torque(Ez, Hx, Hy, cx, cy, R, n_points, a, E0=1.0):
    """(F~x, F~y, M~z) from phasor fields [ny, nx] on a circle of radius R."""
    px, py, phi = contour_points(cx, cy, R, n_points)
    ez = bilinear(Ez, px, py)
    hx = bilinear(Hx, px, py)
    hy = bilinear(Hy, px, py)
    nx_, ny_ = np.cos(phi), np.sin(phi)
    tx, ty = stress_dot_n(ez, hx, hy, nx_, ny_)
    dl = R * 2.0 * np.pi / n_points
    Fx = np.sum(tx) * dl
    Fy = np.sum(ty) * dl
    rx, ry = R * nx_, R * ny_
    Mz = np.sum(rx * ty - ry * tx) * dl
    F0 = np.pi * a * E0 * E0 / 4.0
    M0 = 2.0 * F0 * a
    return np.array([Fx / F0, Fy / F0, Mz / M0])


def poynting_net(Ez, Hx, Hy, cx, cy, R, n_points):
    """Period-averaged net outward Poynting flux through the circle:
    closed integral of 1/2 Re(E x H*) . n dl (zero for a lossless scatterer)."""
    px, py, phi = contour_points(cx, cy, R, n_points)
    ez = bilinear(Ez, px, py)
    hx = bilinear(Hx, px, py)
    hy = bilinear(Hy, px, py)
    # E x H* with E = (0, 0, Ez): (-Ez Hy*, Ez Hx*, 0)
    sx = 0.5 * np.real(-ez * np.conj(hy))
    sy = 0.5 * np.real(ez * np.conj(hx))
    dl = R * 2.0 * np.pi / n_points
    return float(np.sum(sx * np.cos(phi) + sy * np.sin(phi)) * dl)


def default_n_points(R):
    """N_c = 2 ceil(2 pi R): about two samples per lattice spacing of arc."""
    return int(2 * np.ceil(2.0 * np.pi * R))

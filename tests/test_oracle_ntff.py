"""Pins of the near-to-far-field transform (oracle/ntff.py), used for the far-field
scattering intensity |S(phi)|^2 of Sec. II.A."""
import numpy as np
import pytest
from scipy import special as sp

from oracle import analytic as A
from oracle import geometry as G
from oracle import lbm, mst, ntff

import lattice_theory as LT


def _analytic_near_field(B, D, k0, R, N):
    """Scattered E_z on a circle of radius R and the physical H from curl E = i k H."""
    phi = 2 * np.pi * np.arange(N) / N
    m = np.arange(len(B))[:, None]
    H, Hp = sp.hankel1(m, k0 * R), sp.h1vp(m, k0 * R)
    ang = B[:, None] * np.cos(m * phi) + D[:, None] * np.sin(m * phi)
    Es = np.sum(ang * H, axis=0)
    dEdr = k0 * np.sum(ang * Hp, axis=0)
    dEdphi = np.sum(m * (-B[:, None] * np.sin(m * phi) + D[:, None] * np.cos(m * phi)) * H, axis=0)
    dEdx = np.cos(phi) * dEdr - np.sin(phi) / R * dEdphi
    dEdy = np.sin(phi) * dEdr + np.cos(phi) / R * dEdphi
    return phi, Es, dEdy / (1j * k0), -dEdx / (1j * k0)


@pytest.mark.parametrize("case", ["homogeneous", "md_janus", "pec"])
def test_transform_reproduces_analytic_far_field(case):
    """Green's-theorem transform of the exact near field equals the Hankel-asymptote far
    field of the same series (Sec. II.A) at every angle."""
    k0, phi0 = 2 * np.pi / 40, 0.7
    if case == "homogeneous":
        a = 20.0
        B, D = A.homogeneous_BD(k0, a, 2.25, phi0)
    elif case == "pec":
        a = 20.0
        B, D = A.homogeneous_BD(k0, a, 1.0, phi0, pec=True)
    else:
        a = 40.0
        B, D, _ = A.md_janus_BD_galerkin(k0, a, 3.0, phi0, n_basis=160)
    R, N = 1.5 * a, 720
    phi, Es, Hx, Hy = _analytic_near_field(B, D, k0, R, N)
    phis = np.linspace(0, 2 * np.pi, 37)
    An = ntff.far_field_amplitude_from_contour(Es, Hx, Hy, R * np.cos(phi), R * np.sin(phi), np.cos(phi),
                                               np.sin(phi), 0.0, 0.0, R * 2 * np.pi / N, k0, phis)
    Aa = A.far_field_amplitude(B, D, phis)
    assert np.max(np.abs(An - Aa)) < 1e-12 * np.max(np.abs(Aa))


def test_lattice_wavenumber_matches_dispersion_relation():
    for T in (48, 120, 212):
        assert ntff.lattice_wavenumber(T) == pytest.approx(np.angle(LT.vacuum_w(T)), abs=1e-15)


def test_lbm_far_field_matches_analytic_md_janus():
    """Sec. IV.A validation case (eps_r1 = 2, phi0 = -pi/4) at a/dx = 40, L/a = 6: the
    LBM |S(phi)|^2 is within 5 % of the analytic one at most angles."""
    a, T, n, eps1, phi0 = 40.0, 120, 240, 2.0, -np.pi / 4
    eps, pec, _ = G.janus_material(n, n, a, phi0, eps1, pec2=True)
    sim = lbm.Simulation(eps, pec, period=T, ramp_steps=T, nthreads=8)
    sim.advance(24 * T)
    sim.advance(T, accumulate=True)
    Ez, Hx, Hy = sim.phasors()
    cx, cy = G.default_center(n, n)
    R = 1.5 * a
    phis = np.linspace(0, 2 * np.pi, 73)[:-1]
    S = ntff.scattering_intensity_lattice(Ez, Hx, Hy, T, cx, cy, R, mst.default_n_points(R), phis)
    k = ntff.lattice_wavenumber(T)
    B, D, _ = A.md_janus_BD_galerkin(k, a, eps1, phi0, n_basis=320)
    Sa = A.scattering_intensity(B, D, phis + phi0 + np.pi)   # lattice angle -> paper angle
    rel = np.abs(S - Sa) / Sa
    assert np.median(rel) < 0.05 and np.mean(rel < 0.05) > 0.6


@pytest.mark.parametrize("pec", [False, True])
def test_te_transform_reproduces_analytic_far_field(pec):
    """TE^z: the transform of the exact scattered H_z, with E from curl H = -i k E (the
    negative of the TM helper's H), equals the Hankel asymptote of the H_z series."""
    k0, phi0, a = 2 * np.pi / 40, 0.7, 20.0
    B, D = A.homogeneous_BD(k0, a, 1.0 if pec else 2.25, phi0, pec=pec, te=True)
    R, N = 1.5 * a, 720
    phi, Hs, ex, ey = _analytic_near_field(B, D, k0, R, N)
    phis = np.linspace(0, 2 * np.pi, 37)
    An = ntff.far_field_amplitude_from_contour(Hs, -ex, -ey, R * np.cos(phi), R * np.sin(phi), np.cos(phi),
                                               np.sin(phi), 0.0, 0.0, R * 2 * np.pi / N, k0, phis, te=True)
    Aa = A.far_field_amplitude(B, D, phis)
    assert np.max(np.abs(An - Aa)) < 1e-12 * np.max(np.abs(Aa))

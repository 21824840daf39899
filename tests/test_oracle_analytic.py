"""Pins of the analytic oracle (oracle/analytic.py) against what the paper and the
mathematics fix: two independent routes to the same force, the far-field momentum
balance, energy conservation, symmetry, the PEC limit and the values the paper
quotes in its prose."""
import os

import numpy as np
import pytest

from oracle import analytic as A

K0 = 2 * np.pi / 40.0
A_RAD = 40.0          # a / lambda = 1 as in Sec. IV


@pytest.mark.parametrize("eps,phi0", [(2.25, np.pi), (2.25, 0.3), (4.0, 1.1), (9.0, 2.0)])
def test_homogeneous_routes_agree(eps, phi0):
    """Eq. (drag)-(Torque) quadrature, Eq. (U)/(V)/(Torque) closed form and the
    far-field momentum balance give one force; lift and torque vanish (Sec. I:
    homogeneous cylinders feel only drag)."""
    B, D = A.homogeneous_BD(K0, 20.0, eps, phi0)
    q = A.forces_quadrature(B, D, K0, 20.0, phi0)
    cf = A.forces_closed_form(B, D, K0, 20.0, phi0)
    ff = A.far_field_forces(B, D, K0, 20.0, phi0)
    q2 = A.forces_quadrature(B, D, K0, 20.0, phi0, r=45.0)
    assert np.allclose(q, cf, atol=1e-12)
    assert np.allclose(q[:2], ff, atol=1e-12)
    assert np.allclose(q, q2, atol=1e-12)
    assert abs(q[1]) < 1e-12 and abs(q[2]) < 1e-12
    assert q[0] > 0


def test_homogeneous_mode_identity():
    """Lossless single-mode energy balance Re(c_m) + |c_m|^2 = 0 for the scattering
    coefficient c_m = B_m / (alpha_m (-j)^m cos m phi0) of a homogeneous cylinder."""
    B, _ = A.homogeneous_BD(K0, 20.0, 3.0, 0.0)
    m = np.arange(len(B))
    c = B / (A.alpha(m) * (-1j) ** m)
    assert np.max(np.abs(c.real + np.abs(c) ** 2)) < 1e-13


def test_rayleigh_limit():
    """Small dielectric cylinder (k0 a << 1): the dominant m = 0 coefficient tends to
    c_0 -> +j pi (k0 a)^2 (eps - 1) / 4, the textbook Rayleigh limit for TM."""
    k0a = 1e-3
    B, _ = A.homogeneous_BD(k0a, 1.0, 2.0, 0.0)
    expected = 1j * np.pi * k0a ** 2 * (2.0 - 1.0) / 4.0
    assert abs(B[0] - expected) / abs(expected) < 1e-4


def test_pec_cylinder_conserves_energy():
    """PEC cylinder (E_z^tot = 0 on the whole circle in Eq. constants_Bm_Dm)."""
    B, D = A.homogeneous_BD(K0, 20.0, 1.0, 0.4, pec=True)
    pn, ps = A.net_flux(B, D, K0, 30.0, 0.4)
    assert abs(pn) < 1e-12 * ps
    q = A.forces_quadrature(B, D, K0, 20.0, 0.4)
    assert np.allclose(q[:2], A.far_field_forces(B, D, K0, 20.0, 0.4), atol=1e-12)


@pytest.mark.parametrize("eps1,phi0", [(2.0, 7 * np.pi / 36), (5.0, 0.611), (3.0, 4.0)])
def test_md_janus_galerkin_conserves_and_routes_agree(eps1, phi0):
    B, D, _ = A.md_janus_BD_galerkin(K0, A_RAD, eps1, phi0, n_basis=160)
    pn, ps = A.net_flux(B, D, K0, 1.5 * A_RAD, phi0)
    assert abs(pn) < 1e-12 * ps                      # lossless: extinction = scattering
    q_a = A.forces_quadrature(B, D, K0, A_RAD, phi0)
    assert np.allclose(q_a, A.forces_closed_form(B, D, K0, A_RAD, phi0), atol=1e-12)
    q_far = A.forces_quadrature(B, D, K0, A_RAD, phi0, r=1.5 * A_RAD)
    assert np.allclose(q_far[:2], A.far_field_forces(B, D, K0, A_RAD, phi0), atol=1e-10)


@pytest.mark.parametrize("eps1,phi0", [(2.0, 7 * np.pi / 36), (5.0, 0.611)])
def test_md_janus_paper_nystrom_converges_to_galerkin(eps1, phi0):
    """The paper's discretisation (Eq. discrete integral equation, nodes pi/(N-1)
    apart) and an independent Galerkin solution of Eq. (integral equation) agree,
    and the gap closes as N grows."""
    Bg, Dg, _ = A.md_janus_BD_galerkin(K0, A_RAD, eps1, phi0, n_basis=320)
    ref = A.forces_quadrature(Bg, Dg, K0, A_RAD, phi0, r=1.5 * A_RAD)
    gaps = []
    for N in (200, 800):
        B, D, _, _ = A.md_janus_BD(K0, A_RAD, eps1, phi0, N=N)
        f = A.forces_quadrature(B, D, K0, A_RAD, phi0, r=1.5 * A_RAD)
        gaps.append(np.max(np.abs(f - ref)))
        pn, ps = A.net_flux(B, D, K0, 1.5 * A_RAD, phi0)
        assert abs(pn) < 1e-10 * ps
    assert gaps[1] < 0.5 * gaps[0]
    assert gaps[1] < 5e-3


@pytest.mark.parametrize("eps1", [2.0, 5.0])
def test_md_janus_symmetry(eps1):
    """Sec. IV.A: drag symmetric, lift and torque antisymmetric about phi0 = pi/2, 3 pi/2;
    both vanish at those orientations."""
    f = {}
    for p in (np.pi / 2 - 0.4, np.pi / 2 + 0.4, np.pi / 2, 3 * np.pi / 2):
        B, D, _ = A.md_janus_BD_galerkin(K0, A_RAD, eps1, p, n_basis=120)
        f[p] = A.forces_quadrature(B, D, K0, A_RAD, p, r=1.5 * A_RAD)
    lo, hi = f[np.pi / 2 - 0.4], f[np.pi / 2 + 0.4]
    assert abs(lo[0] - hi[0]) < 1e-10 and abs(lo[1] + hi[1]) < 1e-10 and abs(lo[2] + hi[2]) < 1e-10
    for p in (np.pi / 2, 3 * np.pi / 2):
        assert abs(f[p][1]) < 1e-10 and abs(f[p][2]) < 1e-10


def test_md_janus_pec_facing_matches_pec_cylinder():
    """Sec. IV.A / Appendix A: with the PEC half facing the wave (phi0 = 3 pi/2) the
    drag is close to that of a homogeneous PEC cylinder of the same radius."""
    Bp, Dp = A.homogeneous_BD(K0, A_RAD, 1.0, 0.0, pec=True)
    pec_drag = A.forces_quadrature(Bp, Dp, K0, A_RAD, 0.0)[0]
    for eps1 in (1.0001, 2.0, 5.0):
        B, D, _ = A.md_janus_BD_galerkin(K0, A_RAD, eps1, 1.5 * np.pi, n_basis=160)
        drag = A.forces_quadrature(B, D, K0, A_RAD, 1.5 * np.pi, r=1.5 * A_RAD)[0]
        assert abs(drag - pec_drag) < 0.025 * pec_drag


def _quoted():
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_quoted_values.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split(None, 5)
        rows.append((float(parts[0]), float(parts[1]) * np.pi, parts[2], float(parts[3]),
                     float(parts[4]), parts[5]))
    return rows


@pytest.mark.parametrize("row", _quoted(), ids=lambda r: r[5][:40])
def test_md_janus_quoted_values(row):
    eps1, phi0, qty, value, tol, _ = row
    B, D, _ = A.md_janus_BD_galerkin(K0, A_RAD, eps1, phi0, n_basis=320)
    f = A.forces_quadrature(B, D, K0, A_RAD, phi0, r=1.5 * A_RAD)
    assert qty == "drag"
    assert abs(f[0] - value) <= tol


# --- TE^z (H_z, E_x, E_y): the polarization the paper leaves for future work ---------

@pytest.mark.parametrize("eps,pec", [(2.25, False), (6.0, False), (1.0, True)])
def test_te_homogeneous_routes_agree_and_conserve(eps, pec):
    """TE coefficients: near-field stress quadrature at two radii, the closed form and
    the far-field momentum balance give one force (the stress tensor of the dual fields
    (H_z, E_r, E_phi) has the TM form); lossless energy balance."""
    B, D = A.homogeneous_BD(K0, 20.0, eps, 0.7, pec=pec, te=True)
    q = A.forces_quadrature(B, D, K0, 20.0, 0.7)
    assert np.allclose(q, A.forces_closed_form(B, D, K0, 20.0, 0.7), atol=1e-12)
    assert np.allclose(q, A.forces_quadrature(B, D, K0, 20.0, 0.7, r=45.0), atol=1e-12)
    assert np.allclose(q[:2], A.far_field_forces(B, D, K0, 20.0, 0.7), atol=1e-12)
    pn, ps = A.net_flux(B, D, K0, 30.0, 0.7)
    assert abs(pn) < 1e-12 * ps
    assert abs(q[1]) < 1e-12 and abs(q[2]) < 1e-12 and q[0] > 0


def test_te_rayleigh_limits():
    """Small cylinders (k0 a << 1), textbook TE limits that differ from TM: a dielectric
    scatters through the in-plane dipole, c_1 -> +j pi (k0 a)^2 (eps - 1) / (4 (eps + 1))
    with c_0 of order (k0 a)^4; a PEC through c_0 -> -j pi (k0 a)^2 / 4 and
    c_1 -> +j pi (k0 a)^2 / 4 (dH_z/dr = 0 on the surface)."""
    x, eps = 1e-3, 2.0
    B, _ = A.homogeneous_BD(x, 1.0, eps, 0.0, te=True)
    c = B / (A.alpha(np.arange(len(B))) * (-1j) ** np.arange(len(B)))
    assert abs(c[1] - 1j * np.pi * x ** 2 * (eps - 1) / (4 * (eps + 1))) < 1e-4 * abs(c[1])
    assert abs(c[0]) < 1e-4 * abs(c[1])
    B, _ = A.homogeneous_BD(x, 1.0, 1.0, 0.0, pec=True, te=True)
    c = B / (A.alpha(np.arange(len(B))) * (-1j) ** np.arange(len(B)))
    assert abs(c[0] + 1j * np.pi * x ** 2 / 4) < 1e-4 * np.pi * x ** 2 / 4
    assert abs(c[1] - 1j * np.pi * x ** 2 / 4) < 1e-4 * np.pi * x ** 2 / 4

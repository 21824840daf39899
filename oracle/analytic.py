"""Oracle (test infrastructure only): analytic TM^z scattering by (Janus) cylinders.

arXiv 2509.22308, Sec. II and Sec. IV.A.  Units eps0 = mu0 = 1, so omega = k0
(speed of light 1) and the vacuum impedance is 1; incident amplitude E0 = 1.
Time factor e^{-j omega t} (Sec. II); the magnetic field is formed the way
Eq. (total_field) forms it, from curl E = -j omega mu0 H.  Flipping the sign of
H leaves every time-averaged stress (quadratic in H) unchanged.

Paper frame: the incident field is the Jacobi-Anger series of Eq. (incident
field), E_z^I = sum_m alpha_m (-j)^m J_m(k0 r) cos m(phi - phi0), which travels
towards the polar angle phi0 + pi; region II is the half 0 < phi < pi.

Functions
  homogeneous_BD   Bessel series of a homogeneous dielectric or PEC cylinder:
                   continuity of E_z and H_phi at r = a (the textbook special
                   case of Sec. II; the paper uses it as its PEC reference), and
                   the TE^z counterpart (series of H_z).  By the duality
                   E <-> H (eps0 = mu0 = 1 outside) every function below applies to
                   TE coefficients unchanged, with (E_z, H_r, H_phi) read as
                   (H_z, E_r, E_phi).
  md_janus_BD      metallo-dielectric Janus cylinder, solved the way Sec. IV.A
                   does: the integral equation (Eq. integral equation) on N
                   nodes with spacing pi/(N-1), then Eq. (constants_Bm_Dm).
  forces_quadrature  Eq. (drag), (lift), (Torque) integrated numerically on
                   the surface fields of Eq. (total_field).
  forces_closed_form Eq. (Fx), (Fy), (U), (V), (Torque) and (coefficients).
  far_field_forces drag and lift from the far-field momentum balance (an
                   independent route used to pin the two above).
"""
from __future__ import annotations

import numpy as np
from scipy import special as sp


def alpha(m):
    m = np.asarray(m)
    return np.where(m == 0, 1.0, 2.0)


def mode_count(x: float, extra: int = 10) -> int:
    """Series truncation: ceil(x + 4 x^(1/3) + 2) + extra (Wiscombe's rule plus margin)."""
    return int(np.ceil(x + 4.0 * x ** (1.0 / 3.0) + 2.0)) + extra


def homogeneous_BD(k0: float, a: float, eps: float, phi0: float, M: int | None = None,
                   pec: bool = False, te: bool = False):
    """B_m, D_m (m = 0..M) of Eq. (scattered field) for a homogeneous cylinder.

    TM (default): the series is E_z; E_z and H_phi ~ dE_z/dr are continuous at r = a
    (E_z = 0 on a PEC).  TE (``te``, the polarization the paper leaves for future work):
    the same series describes H_z with unit incident amplitude; H_z and
    E_phi ~ (1/eps) dH_z/dr are continuous (dH_z/dr = 0 on a PEC), so the dielectric
    coefficient is the TM one with the inner wavenumber k replaced by k / eps in the
    derivative terms."""
    k = k0 * np.sqrt(eps) if not pec else k0
    if M is None:
        M = mode_count(max(k0 * a, k * a))
    m = np.arange(M + 1)
    x0 = k0 * a
    J0, J0p = sp.jv(m, x0), sp.jvp(m, x0)
    H0, H0p = sp.hankel1(m, x0), sp.h1vp(m, x0)
    if pec:
        c = -J0p / H0p if te else -J0 / H0
    else:
        x1 = k * a
        J1, J1p = sp.jv(m, x1), sp.jvp(m, x1)
        kd = k / eps if te else k      # factor of the inner radial derivative
        c = (kd * J0 * J1p - k0 * J0p * J1) / (k0 * H0p * J1 - kd * H0 * J1p)
    pre = alpha(m) * (-1j) ** m * c
    return pre * np.cos(m * phi0), pre * np.sin(m * phi0)


def md_janus_BD(k0: float, a: float, eps1: float, phi0: float, N: int = 400,
                M: int | None = None, M_kernel: int | None = None):
    """B_m, D_m of the metallo-dielectric Janus cylinder (Sec. IV.A).

    Steps as in the paper: nodes phi_n = (n-1) dphi, dphi = pi/(N-1); kernel
    K(phi, phi') and forcing Y(phi) of Eq. (integral equation) summed to
    M_kernel modes; solve K E dphi = Y (Eq. discrete integral equation) for the
    surface field E_z^tot on region II; then Eq. (constants_Bm_Dm) with the
    integrals over [0, pi] taken by the same node rule.
    Returns (B, D, phi_nodes, E_tot_nodes)."""
    k = k0 * np.sqrt(eps1)
    x0, x1 = k0 * a, k * a
    if M is None:
        M = mode_count(max(x0, x1))
    if M_kernel is None:
        M_kernel = N - 1          # every mode the N nodes resolve
    dphi = np.pi / (N - 1)
    phi = dphi * np.arange(N)
    mk = np.arange(M_kernel + 1)
    ratio_H = hankel_logderiv(M_kernel, x0)
    coef_s = ratio_H - 2.0 * (k / k0) * bessel_j_logderiv(M_kernel, x1)
    coef_c = 0.5 * alpha(mk) * ratio_H
    S = np.sin(np.outer(phi, mk))
    C = np.cos(np.outer(phi, mk))
    K = (S * coef_s) @ S.T + (C * coef_c) @ C.T
    Y = (2j / x0) * (np.cos(np.outer(phi - phi0, mk)) @ (alpha(mk) * (-1j) ** mk * inv_hankel(M_kernel, x0)))
    E_tot = np.linalg.solve(K * dphi, Y)

    m = np.arange(M + 1)
    J0, H0 = sp.jv(m, x0), sp.hankel1(m, x0)
    int_cos = (np.cos(np.outer(m, phi)) @ E_tot) * dphi
    int_sin = (np.sin(np.outer(m, phi)) @ E_tot) * dphi
    B = alpha(m) / (2.0 * np.pi * H0) * int_cos - alpha(m) * (-1j) ** m * J0 * np.cos(m * phi0) / H0
    D = 1.0 / (np.pi * H0) * int_sin - 2.0 * (-1j) ** m * J0 * np.sin(m * phi0) / H0
    return B, D, phi, E_tot


def hankel_logderiv(mmax: int, x: float):
    """H_m^(1)'(x) / H_m^(1)(x) for m = 0..mmax via the ratio r_m = H_{m-1}/H_m,
    which obeys r_{m+1} = 1 / (2m/x - r_m) (upward recurrence, stable because H
    grows with m); H_m' / H_m = r_m - m/x, and H_0'/H_0 = -H_1/H_0."""
    out = np.empty(mmax + 1, dtype=complex)
    H0, H1 = sp.hankel1(0, x), sp.hankel1(1, x)
    out[0] = -H1 / H0
    r = H0 / H1
    for m in range(1, mmax + 1):
        out[m] = r - m / x
        r = 1.0 / (2.0 * m / x - r)
    return out


def bessel_j_logderiv(mmax: int, x: float):
    """J_m'(x) / J_m(x) for m = 0..mmax.  Orders m <= x + 40 use scipy directly;
    above, the ratio rho_m = J_{m-1}/J_m from the downward recurrence
    rho_m = 2m/x - 1/rho_{m+1} (stable for the decaying J) gives J'/J = rho_m - m/x."""
    out = np.empty(mmax + 1)
    mdir = min(mmax, int(x) + 40)
    m = np.arange(mdir + 1)
    out[: mdir + 1] = sp.jvp(m, x) / sp.jv(m, x)
    if mmax > mdir:
        top = mmax + 60
        rho = 2.0 * (top + 1) / x
        for mm in range(top, mdir, -1):
            rho = 2.0 * mm / x - 1.0 / rho
            if mm <= mmax:
                out[mm] = rho - mm / x
    return out


def inv_hankel(mmax: int, x: float):
    """1 / H_m^(1)(x) for m = 0..mmax, set to 0 where H_m overflows."""
    m = np.arange(mmax + 1)
    with np.errstate(over="ignore", invalid="ignore"):
        H = sp.hankel1(m, x)
        out = np.where(np.isfinite(H) & (np.abs(H) < 1e300), 1.0 / np.where(np.isfinite(H), H, 1.0), 0.0)
    return out


def _sin_cos_overlap(p, m):
    """I[p, m] = integral over [0, pi] of sin(p phi) cos(m phi) dphi (p >= 1, m >= 0)."""
    p = np.asarray(p)[:, None]
    m = np.asarray(m)[None, :]
    odd = ((p + m) % 2) == 1
    with np.errstate(divide="ignore", invalid="ignore"):
        val = np.where(odd, 2.0 * p / (p * p - m * m), 0.0)
    return np.where(p == m, 0.0, val)


def md_janus_BD_galerkin(k0: float, a: float, eps1: float, phi0: float, n_basis: int = 160,
                         M: int | None = None, m_sum: int | None = None):
    """B_m, D_m of the metallo-dielectric Janus cylinder from a Galerkin solution of
    the same integral equation (Eq. integral equation) in the basis sin(n phi),
    n = 1..n_basis, which vanishes at the two PEC edges phi = 0, pi; tested with
    the same functions.  With E = sum b_n sin(n phi) the sin-sin part of the
    kernel is diagonal, the cos-cos part couples through the overlaps of
    sin(n phi) with cos(m phi) over [0, pi].  An independent discretisation used
    to pin ``md_janus_BD``; Eq. (constants_Bm_Dm) then follows exactly."""
    k = k0 * np.sqrt(eps1)
    x0, x1 = k0 * a, k * a
    if M is None:
        M = mode_count(max(x0, x1))
    if m_sum is None:
        m_sum = 8 * n_basis + 400
    n = np.arange(1, n_basis + 1)
    mc = np.arange(m_sum + 1)
    lH = hankel_logderiv(m_sum, x0)
    c_m = 0.5 * alpha(mc) * lH
    s_n = lH[1:n_basis + 1] - 2.0 * (k / k0) * bessel_j_logderiv(n_basis, x1)[1:]
    I = _sin_cos_overlap(n, mc)                       # [n_basis, m_sum+1]
    G = (I * c_m) @ I.T + np.diag(s_n * (np.pi / 2.0) ** 2)
    y_m = alpha(mc) * (-1j) ** mc * inv_hankel(m_sum, x0)
    rhs = (2j / x0) * (I @ (y_m * np.cos(mc * phi0))
                       + (np.pi / 2.0) * y_m[1:n_basis + 1] * np.sin(n * phi0))
    b = np.linalg.solve(G, rhs)
    m = np.arange(M + 1)
    J0, H0 = sp.jv(m, x0), sp.hankel1(m, x0)
    int_cos = _sin_cos_overlap(n, m).T @ b            # integral of E cos(m phi) over [0, pi]
    int_sin = np.zeros(M + 1, dtype=complex)
    kk = np.arange(1, min(M, n_basis) + 1)
    int_sin[kk] = (np.pi / 2.0) * b[kk - 1]
    B = alpha(m) / (2.0 * np.pi * H0) * int_cos - alpha(m) * (-1j) ** m * J0 * np.cos(m * phi0) / H0
    D = 1.0 / (np.pi * H0) * int_sin - 2.0 * (-1j) ** m * J0 * np.sin(m * phi0) / H0
    return B, D, b


def fields(B, D, k0: float, r: float, phi0: float, phi):
    """Total E_z, H_r, H_phi on the circle of radius r (Eq. total_field evaluated
    at radius r; with omega mu0 = k0)."""
    M = len(B) - 1
    m = np.arange(M + 1)[:, None]
    phi = np.asarray(phi)[None, :]
    x = k0 * r
    J, Jp = sp.jv(m, x), sp.jvp(m, x)
    H, Hp = sp.hankel1(m, x), sp.h1vp(m, x)
    inc = alpha(m) * (-1j) ** m
    B_ = np.asarray(B)[:, None]
    D_ = np.asarray(D)[:, None]
    Ez = np.sum(inc * J * np.cos(m * (phi - phi0)) + (B_ * np.cos(m * phi) + D_ * np.sin(m * phi)) * H, axis=0)
    Hr = (-1j / (k0 * r)) * np.sum(m * inc * J * np.sin(m * (phi - phi0))
                                   + m * (B_ * np.sin(m * phi) - D_ * np.cos(m * phi)) * H, axis=0)
    Hphi = -1j * np.sum(inc * Jp * np.cos(m * (phi - phi0)) + (B_ * np.cos(m * phi) + D_ * np.sin(m * phi)) * Hp, axis=0)
    return Ez, Hr, Hphi


def forces_quadrature(B, D, k0: float, a: float, phi0: float, r: float | None = None,
                      nphi: int = 2048):
    """(F~x drag, F~y lift, M~z) from Eq. (drag), (lift), (Torque), integrated with
    the periodic trapezoid rule on the circle of radius r (default r = a)."""
    if r is None:
        r = a
    phi = 2.0 * np.pi * np.arange(nphi) / nphi
    Ez, Hr, Hphi = fields(B, D, k0, r, phi0, phi)
    Trr = -0.25 * np.abs(Ez) ** 2 + 0.25 * (np.abs(Hr) ** 2 - np.abs(Hphi) ** 2)
    Tpr = 0.5 * np.real(Hphi * np.conj(Hr))
    c, s = np.cos(phi), np.sin(phi)
    cp, sp0 = np.cos(phi0), np.sin(phi0)
    dphi = 2.0 * np.pi / nphi
    Fx = np.sum(Trr * (-cp * c - sp0 * s) + Tpr * (-sp0 * c + cp * s)) * r * dphi
    Fy = np.sum(Trr * (sp0 * c - cp * s) + Tpr * (-cp * c - sp0 * s)) * r * dphi
    Mz = np.sum(r * r * Tpr) * dphi
    F0 = np.pi * a / 4.0
    return np.array([Fx / F0, Fy / F0, Mz / (2.0 * F0 * a)])


def closed_form_coefficients(B, D, k0: float, a: float, phi0: float):
    """C_m, S_m, C'_m, S'_m of Eq. (coefficients)."""
    M = len(B) - 1
    m = np.arange(M + 1)
    x = k0 * a
    inc = alpha(m) * (-1j) ** m
    J, Jp = sp.jv(m, x), sp.jvp(m, x)
    H, Hp = sp.hankel1(m, x), sp.h1vp(m, x)
    C = inc * J * np.cos(m * phi0) + B * H
    S = inc * J * np.sin(m * phi0) + D * H
    Cp = inc * Jp * np.cos(m * phi0) + B * Hp
    Sp = inc * Jp * np.sin(m * phi0) + D * Hp
    return C, S, Cp, Sp


def forces_closed_form(B, D, k0: float, a: float, phi0: float):
    """(F~x, F~y, M~z) from Eq. (Fx), (Fy) with U, V of Eq. (U), (V) and Eq. (Torque),
    transcribed term by term."""
    C, S, Cp, Sp = closed_form_coefficients(B, D, k0, a, phi0)
    # pad one zero mode so that every sum runs to m = M with the (M+1) terms zero
    C, S, Cp, Sp = (np.append(v, 0.0) for v in (C, S, Cp, Sp))
    x = k0 * a
    Mx = len(C) - 1
    re = np.real
    m = np.arange(Mx)          # m = 0..M-1 for the m, m+1 sums
    U = (re(C[1] * np.conj(C[0])) - re(S[1] * np.conj(S[0])) + re(Cp[1] * np.conj(Cp[0]))
         - re(Sp[1] * np.conj(Sp[0])))
    U += np.sum(re(C[m] * np.conj(C[m + 1])) + re(S[m] * np.conj(S[m + 1]))
                + re(Cp[m] * np.conj(Cp[m + 1])) + re(Sp[m] * np.conj(Sp[m + 1])))
    U -= np.sum(m * (m + 1) * (re(C[m] * np.conj(C[m + 1])) + re(S[m] * np.conj(S[m + 1])))) / x ** 2
    mm = np.arange(1, Mx)     # m = 1..M-1 for the m-1, m+1 sums
    inner = (Sp[0] * np.conj(S[1]) - Cp[0] * np.conj(C[1])) - np.sum(
        mm * ((Cp[mm - 1] - Cp[mm + 1]) * np.conj(C[mm]) + (Sp[mm - 1] - Sp[mm + 1]) * np.conj(S[mm])))
    U -= re(inner) / x
    V = (re(C[1] * np.conj(S[0])) + re(C[0] * np.conj(S[1])) + re(Cp[1] * np.conj(Sp[0]))
         + re(Sp[1] * np.conj(Cp[0])))
    V += np.sum(re(S[m + 1] * np.conj(C[m])) - re(S[m] * np.conj(C[m + 1]))
                + re(Cp[m] * np.conj(Sp[m + 1])) - re(Sp[m] * np.conj(Cp[m + 1])))
    V += np.sum(m * (m + 1) * (re(C[m + 1] * np.conj(S[m])) - re(C[m] * np.conj(S[m + 1])))) / x ** 2
    inner = (Cp[0] * np.conj(S[1]) + Sp[0] * np.conj(C[1])) + np.sum(
        mm * ((Cp[mm - 1] + Cp[mm + 1]) * np.conj(S[mm]) - (Sp[mm - 1] + Sp[mm + 1]) * np.conj(C[mm])))
    V += re(inner) / x
    mt = np.arange(1, Mx + 1)
    Mz = np.sum(mt * re(Sp[mt] * np.conj(C[mt]) - Cp[mt] * np.conj(S[mt]))) / x
    cp, sp0 = np.cos(phi0), np.sin(phi0)
    return np.array([U * cp + V * sp0, -U * sp0 + V * cp, Mz])


def far_field_amplitude(B, D, phi):
    """A(phi) = sum_m (-j)^m (B_m cos m phi + D_m sin m phi): the scattered field is
    sqrt(2 / (pi k0 r)) e^{j (k0 r - pi/4)} A(phi) far away (Hankel asymptote, Sec. II.A)."""
    m = np.arange(len(B))[:, None]
    phi = np.asarray(phi)[None, :]
    return np.sum((-1j) ** m * (np.asarray(B)[:, None] * np.cos(m * phi)
                                + np.asarray(D)[:, None] * np.sin(m * phi)), axis=0)


def scattering_intensity(B, D, phi):
    """|S(phi)|^2 = k0 r |E^S|^2 / |E^I|^2 in the far field (Eq. scattering intensity)."""
    return (2.0 / np.pi) * np.abs(far_field_amplitude(B, D, phi)) ** 2


def far_field_forces(B, D, k0: float, a: float, phi0: float, nphi: int = 4096):
    """Drag and lift (non-dimensional) from the far-field momentum balance of a
    lossless scatterer: the force equals the momentum removed from the incident
    beam (extinction = scattered power) minus the momentum carried away by the
    scattered wave, per unit angle dP/dphi = |A(phi)|^2 / (pi k0)."""
    phi = 2.0 * np.pi * np.arange(nphi) / nphi
    dP = np.abs(far_field_amplitude(B, D, phi)) ** 2 / (np.pi * k0)
    dphi = 2.0 * np.pi / nphi
    drag = np.sum(dP * (1.0 + np.cos(phi - phi0))) * dphi
    lift = np.sum(dP * np.sin(phi - phi0)) * dphi
    F0 = np.pi * a / 4.0
    return np.array([drag / F0, lift / F0])


def net_flux(B, D, k0: float, r: float, phi0: float, nphi: int = 4096):
    """Net period-averaged Poynting flux of the total field through radius r and
    the scattered power, (P_net, P_sca); P_net is zero for a lossless cylinder."""
    phi = 2.0 * np.pi * np.arange(nphi) / nphi
    Ez, Hr, Hphi = fields(B, D, k0, r, phi0, phi)
    dphi = 2.0 * np.pi / nphi
    # physical H is the negative of the Eq. (total_field) H; S_r = -1/2 Re(Ez Hphi*)
    P_net = np.sum(0.5 * np.real(Ez * np.conj(Hphi))) * r * dphi
    P_sca = np.sum(np.abs(far_field_amplitude(B, D, phi)) ** 2) / (np.pi * k0) * dphi
    return float(P_net), float(P_sca)

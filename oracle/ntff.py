"""Oracle (test infrastructure only): near-to-far-field transform of lattice phasors.

arXiv 2509.22308, Sec. II.A: the far-field scattering intensity
|S(phi)|^2 = k0 r |E^S(phi)|^2 / |E^I|^2 (Eq. scattering intensity), obtained from the LBM
near field by a near-to-far-field transformation.  The paper cites the method without
giving it; this is the scalar 2-D form from Green's theorem:

  E^s(r) = closed integral over C of [G dE^s/dn' - E^s dG/dn'] dl',  G = (i/4) H_0^(1)(k|r - r'|)

with n' the outward normal of a contour C that encloses the scatterer (time factor
e^{-i omega t}).  With the Hankel asymptote far away, E^s = sqrt(2/(pi k r)) e^{i(k r - pi/4)} A(phi),
  A(phi) = (k/4) closed integral [ (r^ . n') E^s + (-n_x H_y^s + n_y H_x^s) ] e^{-i k r^ . r'} dl',
using dE/dn = i k (-n_x H_y + n_y H_x) (curl E = i k H for TM^z phasors), and
|S(phi)|^2 = (2/pi) |A(phi)|^2 / E0^2.  The lattice frame has the wave along +x, so phi = 0
is forward scattering and phi = pi backward (as in the paper's Fig. 2).

The scattered near field is the total phasor minus the lattice's exact incident plane
wave E^I = i E0 e^{i k x} (H_y^I = -E^I), subtracted at the lattice sites before the
bilinear interpolation onto the contour.
"""
from __future__ import annotations

import numpy as np

from oracle import mst


def lattice_wavenumber(period: int) -> float:
    """Wavenumber of the lattice's right-going vacuum plane wave of period T: arg w,
    w = (3 - z) / (z (3 z - 1)), z = e^{-2 pi i / T} (the source's dispersion relation)."""
    z = np.exp(-2j * np.pi / period)
    return float(np.angle((3.0 - z) / (z * (3.0 * z - 1.0))))


def far_field_amplitude_from_contour(ez, hx, hy, px, py, nx_, ny_, cx, cy, dl, k, phis, te=False):
    """A(phi) from scattered phasors ez, hx, hy sampled at contour points (px, py) with
    outward normals (nx_, ny_), line element dl, about the centre (cx, cy).

    TE^z: (ez, hx, hy) are (H_z, E_x, E_y) and the transformed scalar is H_z; curl H = -i k E
    gives dH_z/dn = -i k (-n_x E_y + n_y E_x), the TM normal derivative with the sign flipped."""
    phis = np.asarray(phis)[:, None]
    rx, ry = px[None, :] - cx, py[None, :] - cy
    ux, uy = np.cos(phis), np.sin(phis)
    phase = np.exp(-1j * k * (ux * rx + uy * ry))
    sgn = -1.0 if te else 1.0
    integrand = (ux * nx_[None, :] + uy * ny_[None, :]) * ez[None, :] + sgn * (-nx_ * hy + ny_ * hx)[None, :]
    return (k / 4.0) * np.sum(integrand * phase, axis=1) * dl


def scattered_phasors(Ez, Hx, Hy, period: int, E0: float = 1.0, te=False):
    """Lattice phasor fields minus the exact incident plane wave at every site (TM: E_z^I =
    i E0 e^{i k x}, H_y^I = -E_z^I; TE: H_z^I = i E0 e^{i k x}, E_y^I = +H_z^I)."""
    k = lattice_wavenumber(period)
    x = np.arange(Ez.shape[1])[None, :]
    Einc = 1j * E0 * np.exp(1j * k * x)
    return Ez - Einc, Hx, (Hy - Einc) if te else (Hy + Einc)


def scattering_intensity_lattice(Ez, Hx, Hy, period, cx, cy, R, n_points, phis, E0=1.0, te=False):
    """|S(phi)|^2 (Eq. scattering intensity) from LBM phasor fields [ny, nx] via the
    transform on a circle of radius R about (cx, cy); TE: the triple is (H_z, E_x, E_y)."""
    k = lattice_wavenumber(period)
    Es, Hxs, Hys = scattered_phasors(Ez, Hx, Hy, period, E0, te)
    px, py, phi = mst.contour_points(cx, cy, R, n_points)
    ez = mst.bilinear(Es, px, py)
    hx = mst.bilinear(Hxs, px, py)
    hy = mst.bilinear(Hys, px, py)
    A = far_field_amplitude_from_contour(ez, hx, hy, px, py, np.cos(phi), np.sin(phi), cx, cy,
                                         R * 2.0 * np.pi / n_points, k, phis, te)
    return (2.0 / np.pi) * np.abs(A) ** 2 / (E0 * E0)

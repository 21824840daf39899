"""Closed-form facts about the D3Q7 Maxwell lattice scheme, derived by hand from
Eq. (LBGK equation) and Eq. (equilibrium distribution functions) by Fourier
analysis; used by the tests to pin the oracle.  Nothing here runs the scheme.

For fields uniform in y, a plane wave ~ w^x z^t (w = e^{ik}, z = e^{-i omega})
with E_z, H_y only.  Each population obeys f(x + c_x, t + 1) = 2 f^eq - f, so a
population with eq value q and velocity c_x has amplitude 2q / (w^{c_x} z + 1).
Writing a = 1/(3(wz + 1)), b = 1/(3(z/w + 1)), c_e = (4/3 + 2(eps - 1))/(z + 1),
c_h = (4/3)/(z + 1), the moment conditions D = eps E and B = H become
    (eps - a - b - c_e) E = (b - a) H,   (1 - a - b - c_h) H = (b - a) E,
so (eps - a - b - c_e)(1 - a - b - c_h) = (b - a)^2.  In vacuum the right-going
branch is H = -E with 2a + c_h = 1, i.e. w = (3 - z) / (z (3 z - 1)), |w| = 1.
"""
from __future__ import annotations

import numpy as np
from scipy import optimize


def vacuum_w(period: int) -> complex:
    om = 2.0 * np.pi / period
    z = np.exp(-1j * om)
    return (3.0 - z) / (z * (3.0 * z - 1.0))


def medium_k(period: int, eps: float) -> float:
    """Real wavenumber of the right-going wave in a uniform medium (root of the
    dispersion relation above near the continuum value 3 omega sqrt(eps))."""
    om = 2.0 * np.pi / period
    z = np.exp(-1j * om)

    def F(k):
        w = np.exp(1j * k)
        a = 1.0 / (3.0 * (w * z + 1.0))
        b = 1.0 / (3.0 * (z / w + 1.0))
        ce = (4.0 / 3.0 + 2.0 * (eps - 1.0)) / (z + 1.0)
        ch = (4.0 / 3.0) / (z + 1.0)
        return (eps - a - b - ce) * (1.0 - a - b - ch) - (b - a) ** 2

    k0 = 3.0 * om * np.sqrt(eps)
    k = optimize.newton(F, k0 + 0j, tol=1e-15, maxiter=100)
    return complex(k)


def vacuum_plane_wave_state(period: int, nx: int, ny: int, t: int, E=1j):
    """Full 42-component pre-collision state [ny, nx, 14, 3] of the exact
    right-going vacuum plane wave E_z = Re[E w^x z^t], H_y = -E_z, at time t.
    Vector order e_0, e_+x, e_-x, e_+y, e_-y, e_+z, e_-z, then the same for h."""
    om = 2.0 * np.pi / period
    z = np.exp(-1j * om)
    w = vacuum_w(period)
    H = -E
    P = 2.0 * E / (3.0 * (w * z + 1.0))   # e_+x,z (eq (E_z - H_y)/6, velocity +x)
    s = 1.0 / (3.0 * (z + 1.0))           # 2 q/(z+1) with q = field/6, no x motion
    amp = np.zeros((14, 3), complex)
    amp[1, 2] = P
    for i in (3, 4, 5, 6):                # e_+-y, e_+-z: eq E_z / 6
        amp[i, 2] = E * s
    amp[5, 0] = H * s                     # e_+z: eq (H_y/6, -H_x/6, E_z/6)
    amp[6, 0] = -H * s                    # e_-z: eq (-H_y/6, H_x/6, E_z/6)
    amp[7 + 1, 1] = -P                    # h_+x,y: eq (H_y - E_z)/6
    amp[7 + 3, 0] = E * s                 # h_+y: eq ((H_x + E_z)/6, H_y/6, 0)
    amp[7 + 3, 1] = H * s
    amp[7 + 4, 0] = -E * s                # h_-y: eq ((H_x - E_z)/6, H_y/6, 0)
    amp[7 + 4, 1] = H * s
    amp[7 + 5, 1] = H * s                 # h_+-z: eq (H_x/6, H_y/6, 0)
    amp[7 + 6, 1] = H * s
    ph = (w ** np.arange(nx)) * (z ** t)
    st = np.real(amp[None, None, :, :] * ph[None, :, None, None])
    return np.ascontiguousarray(np.broadcast_to(st, (ny, nx, 14, 3)))

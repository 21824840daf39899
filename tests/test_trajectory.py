"""Trajectory integration of Sec. IV.C (host side) against closed forms."""
import math

import numpy as np
import pytest

from paper_2509_22308_gb300 import trajectory as TR


def _map(fx, fy, mz, n=64):
    phi = 2 * np.pi * np.arange(n) / n
    return TR.PeriodicMap(fx(phi), fy(phi), mz(phi))


def test_periodic_interpolation_is_exact_for_band_limited_maps():
    f = lambda p: 1.3 + 0.4 * np.cos(p) - 0.2 * np.sin(3 * p)
    m = _map(f, f, f, n=16)
    q = np.linspace(0, 7, 29)
    assert np.allclose(m(q)[:, 0], f(q), atol=1e-12)


def test_torque_free_motion_is_straight():
    m = _map(lambda p: 2.0 + 0 * p, lambda p: 0.5 + 0 * p, lambda p: 0 * p)
    tr = TR.integrate(m, 0.3, t_final=100.0, log_l_over_a=math.log(20.0), dt=0.5)
    k = math.log(20.0) / (4 * math.pi)
    assert tr[-1, 1] == pytest.approx(k * 2.0 * 100.0, rel=1e-12)
    assert tr[-1, 2] == pytest.approx(k * 0.5 * 100.0, rel=1e-12)
    assert tr[-1, 3] == pytest.approx(0.3, abs=1e-12)


def test_reorientation_matches_closed_form_and_settles_at_stable_zero():
    """dphi/dt = M/(2 pi) with M = -c sin(phi - phi*): tan((phi - phi*)/2) decays as
    exp(-c t / (2 pi)); phi* is the stable torque-free orientation."""
    c, ps = 0.8, 1.2
    m = _map(lambda p: 1.0 + 0 * p, lambda p: 0 * p, lambda p: -c * np.sin(p - ps))
    tr = TR.integrate(m, 2.5, t_final=40.0, dt=0.05)
    exact = ps + 2 * np.arctan(np.tan((2.5 - ps) / 2) * np.exp(-c * tr[:, 0] / (2 * np.pi)))
    assert np.max(np.abs(tr[:, 3] - exact)) < 1e-8
    roots = TR.torque_free_orientations(m)
    stable = [r for r, s in roots if s]
    assert len(roots) == 2 and len(stable) == 1 and stable[0] == pytest.approx(ps, abs=1e-9)

"""Seeded synthetic workloads (parameters only; no lattice Boltzmann arithmetic).

Every workload is a list of Janus-cylinder instance specifications in lattice
units (cell size 1, time step 1).  The incident period is ``period`` steps;
with the lattice's vacuum phase speed of 1/3 cell per step, the nominal
wavelength is period / 3 cells.  Both the CUDA path and the CPU oracle are
driven from these dictionaries; each side rasterises and runs them itself.

Keys of an instance: nx, ny, a (radius, cells), phi0 (interface orientation,
rad), eps1 (region II), eps2 (region III, ignored when pec2), pec2 (region III
is a perfect electric conductor), period (T), periods (run length in periods;
the last one is Fourier-averaged), R (stress-tensor contour radius), ramp
(source ramp in steps).
"""
from __future__ import annotations

import math

import numpy as np


def _inst(nx, a, phi0, eps1, eps2, pec2, period, periods, R, ny=None, ramp=None):
    return dict(nx=int(nx), ny=int(ny if ny is not None else nx), a=float(a), phi0=float(phi0),
                eps1=float(eps1), eps2=float(eps2), pec2=bool(pec2), period=int(period),
                periods=int(periods), R=float(R), ramp=int(period if ramp is None else ramp))


def homogeneous_dielectric_256():
    """Homogeneous dielectric cylinder eps_r = 2.25, a = 20, 256 x 256, wavelength 40
    (T = 120), 20 periods, contour radius 40."""
    return [_inst(256, 20, 0.0, 2.25, 2.25, False, 120, 20, 40)]


def md_janus_512(seed: int = 1):
    """Metallo-dielectric Janus cylinders, 512 x 512, a = 32, wavelength 32 (a/lambda = 1,
    T = 96), interface angle theta in {0, 30, ..., 180} deg, eps_r1 ~ U[2, 10] per
    instance (seeded), 30 periods, contour radius 64."""
    rng = np.random.default_rng(seed)
    out = []
    for th in range(0, 181, 30):
        e1 = float(rng.uniform(2.0, 10.0))
        out.append(_inst(512, 32, math.radians(th), e1, 1.0, True, 96, 30, 64))
    return out


def transit_periods(nx, ny, period, R):
    """Periods the incident front needs from the source column x = 0 to the far side of
    the contour (x = centre + R) at the vacuum speed of 1/3 cell per step, rounded up."""
    cx = (nx - 1) / 2.0
    return int(math.ceil(3.0 * (cx + R) / period))


def settled(inst, periods_after_transit: int = 20):
    """Copy of an instance whose run covers the transit of the incident front past the
    contour and then ``periods_after_transit`` more periods (the last one accumulated)."""
    out = dict(inst)
    out["periods"] = transit_periods(inst["nx"], inst["ny"], inst["period"], inst["R"]) + periods_after_transit
    return out


def dielectric_janus_2048():
    """Dielectric Janus cylinders, 2048 x 2048, a = 128, eps1 = 2, eps2 in {2, 4.5, 7, 9.5, 12},
    size parameter k0 a in {5, 10, 20} (wavelength rounded so that T = 3 lambda is an
    integer), phi0 = 30 deg, contour radius 1.6 a; 20 periods after the incident front has
    crossed the contour (the front needs up to 31 periods to get there at k0 a = 20)."""
    out = []
    for k0a in (5.0, 10.0, 20.0):
        lam = round(2.0 * math.pi * 128.0 / k0a)
        for e2 in (2.0, 4.5, 7.0, 9.5, 12.0):
            out.append(settled(_inst(2048, 128, math.radians(30.0), 2.0, e2, False, 3 * lam, 20, 1.6 * 128)))
    return out


def design_map_256(seed: int = 4, n: int = 256):
    """Batched design diagram: n dielectric Janus instances, eps1 = 2, eps2 ~ U[2, 12],
    theta ~ U[0, 180] deg, a in {16, 32, 64}, grid 16 a (256^2 / 512^2 / 1024^2),
    wavelength = a (T = 3 a), 20 periods each, contour radius 1.6 a."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        a = int(rng.choice([16, 32, 64]))
        e2 = float(rng.uniform(2.0, 12.0))
        th = float(rng.uniform(0.0, 180.0))
        out.append(_inst(16 * a, a, math.radians(th), 2.0, e2, False, 3 * a, 20, 1.6 * a))
    return out


def md_janus_8192(seed: int = 5):
    """Large single domain: 8192 x 8192 metallo-dielectric Janus, a = 512, wavelength 80
    (k0 a ~ 40, T = 240), eps ~ U[2, 12] and theta ~ U[0, 180) deg (seeded), 50 periods,
    contour radius 1.5 a.  After 50 periods the incident front has only just reached the
    cylinder (it crosses the contour after 61 periods); ``settled`` gives the run whose
    forces are those of the steady state."""
    rng = np.random.default_rng(seed)
    e1 = float(rng.uniform(2.0, 12.0))
    th = float(rng.uniform(0.0, 180.0))
    return [_inst(8192, 512, math.radians(th), e1, 1.0, True, 240, 50, 768)]


def small_cases():
    """Small instances the oracle finishes in seconds, spanning several thread-block
    tiles with ragged tails (odd and non-multiple-of-32 sizes)."""
    return [
        _inst(96, 12, 0.0, 2.25, 2.25, False, 60, 4, 20),
        _inst(101, 14, math.radians(30.0), 4.0, 1.0, True, 48, 3, 24, ny=77),
        _inst(130, 16, math.radians(200.0), 2.0, 7.5, False, 54, 3, 26, ny=70),
        _inst(67, 9, math.radians(90.0), 5.0, 1.0, True, 36, 4, 14, ny=45),
    ]


def shard(instances, rank: int, world: int):
    """Instances of one rank when a list of independent instances is spread over
    world ranks (round robin; no instance is shared, every instance is covered)."""
    return list(instances[rank::world])


def rank_workload(name: str, rank: int, **kw):
    """The seeded workload a rank runs under weak scaling: rank r uses seed base + r,
    so the ranks solve distinct but statistically identical problem sets."""
    fn = WORKLOADS[name]
    if "seed" in fn.__code__.co_varnames:
        base = kw.pop("seed", fn.__defaults__[0] if fn.__defaults__ else 0)
        return fn(seed=base + rank, **kw)
    return fn(**kw)


WORKLOADS = {
    "homogeneous_dielectric_256": homogeneous_dielectric_256,
    "md_janus_512": md_janus_512,
    "dielectric_janus_2048": dielectric_janus_2048,
    "design_map_256": design_map_256,
    "md_janus_8192": md_janus_8192,
    "small_cases": small_cases,
}

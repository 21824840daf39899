"""Oracle (test infrastructure only): staircase rasterisation of a Janus cylinder.

Sec. II of arXiv 2509.22308: a circular cylinder of radius a made of two halves,
region II (dielectric eps_r1) and region III (dielectric eps_r2, or a perfect
electric conductor for the metallo-dielectric cylinder), in vacuum (region I).
Sec. IV.A notes the circle is represented by a staircase on the Cartesian lattice.

Lattice frame (derived here from the paper's frame): the incident wave travels along +x.  In the
paper's frame region II occupies the polar angles [0, pi] and the wave travels
towards phi0 + pi, so after rotating the wave onto +x the region-II half is the
one whose points d (relative to the centre) satisfy d . n_d > 0 with
n_d = (-sin phi0, -cos phi0).  Points on the interface line (|d . n_d| <= 1e-9
cells, the tie band that absorbs rounding) belong to region III.
"""
from __future__ import annotations

import numpy as np

REGION_I, REGION_II, REGION_III = 0, 1, 2
TIE_BAND = 1e-9


def default_center(nx: int, ny: int):
    return (nx - 1) / 2.0, (ny - 1) / 2.0


def janus_regions(nx: int, ny: int, a: float, phi0: float, cx=None, cy=None):
    """Region id per site [ny, nx] (uint8): 0 vacuum, 1 region II, 2 region III."""
    if cx is None or cy is None:
        cx, cy = default_center(nx, ny)
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    dx = x - cx
    dy = y - cy
    inside = dx * dx + dy * dy <= a * a
    ndx, ndy = -np.sin(phi0), -np.cos(phi0)
    side = dx * ndx + dy * ndy
    reg = np.zeros((ny, nx), dtype=np.uint8)
    reg[inside & (side > TIE_BAND)] = REGION_II
    reg[inside & ~(side > TIE_BAND)] = REGION_III
    return reg


def janus_material(nx, ny, a, phi0, eps1, eps2=None, pec2=False, cx=None, cy=None):
    """(eps [ny, nx] float64, pec [ny, nx] uint8, regions) for a Janus cylinder.

    Region III is a PEC when ``pec2`` is true (metallo-dielectric cylinder), a
    dielectric eps2 otherwise.  A homogeneous cylinder is eps1 == eps2."""
    reg = janus_regions(nx, ny, a, phi0, cx, cy)
    eps = np.ones((ny, nx))
    eps[reg == REGION_II] = eps1
    pec = np.zeros((ny, nx), dtype=np.uint8)
    if pec2:
        pec[reg == REGION_III] = 1
    else:
        eps[reg == REGION_III] = eps2
    return eps, pec, reg

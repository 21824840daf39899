"""2-D design maps on the batched path (Sec. IV.A-B): a metallo-dielectric map at the paper's
force resolution (a/dx = 40, L/a = 4, a = lambda) against the analytic solution, and the
mirror symmetry of the map."""
import numpy as np
import pytest

from oracle import analytic as A
from oracle import ntff
from paper_2509_22308_gb300 import trajectory as TR

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_22308_gb300 import build
    build.build()


def test_md_janus_map_matches_analytic():
    """4 x 12 cells (eps_r1 in {1, 2, 3.5, 5}, phi0 in steps of pi/6), 30 periods, FP32 batch:
    the force/torque error against the analytic Janus solution, in units of the drag, has a
    median below 3 % and stays below 10 % everywhere (Sec. IV.A: small over most of the map,
    larger where lift and torque are small or vary sharply; measured median 1.5 %, largest
    7.9 % at eps_r1 = 3.5)."""
    eps = [1.0, 2.0, 3.5, 5.0]
    phis = 2 * np.pi * np.arange(12) / 12
    F, steps = TR.md_janus_map(eps, phis, periods=30)
    assert (steps == 30 * 120).all()
    k = ntff.lattice_wavenumber(120)
    err = np.empty((len(eps), len(phis)))
    for i, e in enumerate(eps):
        for j, p in enumerate(phis):
            B, D, _ = A.md_janus_BD_galerkin(k, 40.0, e, p, n_basis=320)
            ex = A.forces_quadrature(B, D, k, 40.0, p, r=60.0)
            err[i, j] = np.max(np.abs(F[i, j] - ex)) / abs(ex[0])
    assert np.median(err) < 0.03 and err.max() < 0.10, err


def test_map_mirror_symmetry():
    """phi0 <-> pi - phi0 is the mirror y -> -y of the lattice: drag equal, lift and torque
    opposite, for a dielectric Janus map (eps_r2 = ratio x eps_r1) as for the MD maps (to the
    FP32 rounding, whose order of summation is not mirror symmetric)."""
    n = 12
    phis = 2 * np.pi * np.arange(n) / n
    F, _ = TR.dielectric_janus_map(2.0, [1.5, 3.0], phis, a=24, periods=12)
    mirror = (n // 2 - np.arange(n)) % n
    scale = np.abs(F[..., 0]).max()
    assert np.max(np.abs(F[:, :, 0] - F[:, mirror, 0])) < 1e-4 * scale
    assert np.max(np.abs(F[:, :, 1:] + F[:, mirror, 1:])) < 1e-4 * scale

"""Parity at the benchmark workloads' full size and run length, and bit-identity of the
multi-step kernels where every persistent thread block walks several tiles.

FP64 against the oracle (Sec. III scheme, Sec. II.B forces): the homogeneous eps = 2.25
cylinder on 256^2 (a = 20, T = 120, the full 20 periods, contour radius 40) and one
metallo-dielectric instance of the 512^2 benchmark workload (a = 32, T = 96, the full 30
periods, contour radius 64), both in the launch configuration the benchmark uses.  By the
end of these runs the incident front has crossed the cylinder many times, so the source,
the edges, the dielectric and the PEC half all shape the compared fields and forces.
Bars: fields within 1e-10 (relative L2 of the field state), forces within 1e-10 of drag
scale, phasors at every stencil site within 1e-10.

Multi-step launches against one step per launch: lattices of 1024^2 and 1536 x 1000 hold
2 048-3 182 tiles of the two- and three-step kernels against a persistent grid of 3 thread
blocks per SM, so each block walks several tiles, reusing its stage and flipping its
mbarrier phase; the four-step kernel cuts them into strips and row segments of several
rows per warp, so its row ring wraps many times; fields after step counts of every residue
and the forces of an accumulated period must be the same bits."""
import os

import numpy as np
import pytest

from oracle import geometry as G
from oracle import lbm as OL
from oracle import mst
from paper_2509_22308_gb300 import lbm_em as L
from paper_2509_22308_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_22308_gb300 import build
    build.build()
    OL.build()


def fields_rel_l2(got, ref):
    num = sum(np.linalg.norm(a - b) ** 2 for a, b in zip(got, ref))
    den = sum(np.linalg.norm(b) ** 2 for b in ref)
    return float(np.sqrt(num / max(den, 1e-300)))


def _full_run_against_oracle(inst):
    eps, pec, reg = G.janus_material(inst["nx"], inst["ny"], inst["a"], inst["phi0"], inst["eps1"],
                                     inst["eps2"], inst["pec2"])
    sim = OL.Simulation(eps, pec, period=inst["period"], ramp_steps=inst["ramp"], nthreads=os.cpu_count() or 1)
    n_plain = (inst["periods"] - 1) * inst["period"]
    with L.solver_for_instance(inst, "f64") as s:
        ids, _ = s.material()
        assert np.array_equal(ids, reg)
        s.step(n_plain)
        sim.advance(n_plain)
        assert s.t == sim.t == n_plain
        ez, hx, hy = s.fields()
        oz, ox, oy = sim.fields()
        assert fields_rel_l2((ez, hx, hy), (oz, ox, oy)) < 1e-10
        # the front has long passed the cylinder: the field is non-trivial everywhere
        assert np.abs(oz[:, -2]).max() > 0.1 and np.abs(oz[inst["ny"] // 2]).max() > 0.5
        F = s.force_torque(L.make_contour(inst["R"], inst["a"]))
        sim.advance(inst["period"], accumulate=True)
        cx, cy = G.default_center(inst["nx"], inst["ny"])
        Fo = mst.force_torque(*sim.phasors(), cx, cy, inst["R"], mst.default_n_points(inst["R"]), inst["a"])
        assert np.max(np.abs(F - Fo)) < 1e-10 * np.sum(np.abs(Fo)), (F, Fo)
        xy, ph = s.phasors()
        oE, oX, oY = sim.phasors()
        ref = np.stack([oE.real, oE.imag, oX.real, oX.imag, oY.real, oY.imag], -1)[xy[:, 1], xy[:, 0]]
        assert np.linalg.norm(ph - ref) < 1e-10 * np.linalg.norm(ref)
        return F, Fo


def test_homogeneous_256_full_run_matches_oracle():
    """The 256^2 homogeneous-cylinder workload, all 20 periods: FP64 GPU = oracle to 1e-10,
    and the mirror-symmetric cylinder has no lift or torque (Sec. IV.A)."""
    inst = W.homogeneous_dielectric_256()[0]
    F, Fo = _full_run_against_oracle(inst)
    assert abs(F[1]) < 1e-6 * abs(F[0]) and abs(F[2]) < 1e-6 * abs(F[0])


def test_md_janus_512_full_run_matches_oracle():
    """One instance (theta = 30 deg) of the 512^2 metallo-dielectric benchmark workload, all
    30 periods: FP64 GPU = oracle to 1e-10 in fields, phasors and forces."""
    inst = W.md_janus_512()[1]
    F, Fo = _full_run_against_oracle(inst)
    assert abs(F[1]) > 1e-3 * abs(F[0])   # an oblique Janus interface has lift


BIG = [(1024, 1024), (1536, 1000)]


def _big_inst(nx, ny, pec2=True):
    a = min(nx, ny) / 5.0
    return dict(nx=nx, ny=ny, a=a, phi0=0.7, eps1=3.5, eps2=1.0 if pec2 else 6.0, pec2=pec2, period=48,
                periods=2, R=1.5 * a, ramp=48)


def _same_bits(inst, prec, mode, pol="tm", counts=(1, 2, 3, 5, 30, 31, 64, 7)):
    with L.solver_for_instance(inst, prec, steps_per_launch=mode, polarization=pol) as a, \
            L.solver_for_instance(inst, prec, steps_per_launch="one", polarization=pol) as b:
        for n in counts:
            a.step(n)
            b.step(n)
            for x, y in zip(a.fields(), b.fields()):
                assert np.array_equal(x, y), (prec, mode, pol, n)
        assert np.abs(a.fields()[0]).max() > 0
        c = L.make_contour(inst["R"], inst["a"])
        assert np.array_equal(a.force_torque(c), b.force_torque(c))
        for x, y in zip(a.fields(), b.fields()):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("shape", BIG, ids=lambda s: f"{s[0]}x{s[1]}")
@pytest.mark.parametrize("prec,mode", [("f32", "two"), ("f32", "three"), ("f32", "four"), ("f16dev", "two")])
def test_multi_step_bit_identity_on_persistent_grid(shape, prec, mode):
    _same_bits(_big_inst(*shape), prec, mode)


@pytest.mark.parametrize("shape", BIG, ids=lambda s: f"{s[0]}x{s[1]}")
@pytest.mark.parametrize("mode", ["two", "three", "four"])
def test_multi_step_bit_identity_on_persistent_grid_te(shape, mode):
    _same_bits(_big_inst(*shape, pec2=False), "f32", mode, pol="te")


@pytest.mark.parametrize("pol", ["tm", "te"])
def test_four_steps_in_several_waves_of_units_bit_identical(pol):
    """On 4096^2 the four-step kernel cuts each strip into twice as many row segments as one
    wave of resident warps holds (84-row segments, two waves of thread blocks): fields after
    step counts of every residue and an accumulated period's forces are the bits of one step
    per launch."""
    _same_bits(_big_inst(4096, 4096, pec2=pol == "tm"), "f32", "four", pol=pol, counts=(1, 2, 3, 4, 7, 32))


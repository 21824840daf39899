"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars: region ids bit-exact; FP64 fields and forces within 1e-10 (relative L2 for
fields, drag scale for forces); FP32 storage within 1e-4 of drag and 1e-3 of drag
scale for lift and torque against the FP64 GPU run (spec tolerances)."""
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


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def fields_rel_l2(got, ref):
    """||(E_z, H_x, H_y)_got - (E_z, H_x, H_y)_ref|| / ||(E_z, H_x, H_y)_ref||: one norm over
    the whole field state (a component that vanishes in exact arithmetic, such as H_x
    of a y-uniform wave, carries only rounding and has no relative error of its own)."""
    num = sum(np.linalg.norm(a - b) ** 2 for a, b in zip(got, ref))
    den = sum(np.linalg.norm(b) ** 2 for b in ref)
    return float(np.sqrt(num / max(den, 1e-300)))


KINDS = {"hard": (L.SRC_HARD, OL.SRC_HARD), "open": (L.SRC_OPEN, OL.SRC_OPEN)}


def oracle_sim(inst, kind=OL.SRC_HARD):
    eps, pec, reg = G.janus_material(inst["nx"], inst["ny"], inst["a"], inst["phi0"], inst["eps1"],
                                     inst["eps2"], inst["pec2"])
    return OL.Simulation(eps, pec, period=inst["period"], ramp_steps=inst["ramp"], source_kind=kind), reg


def oracle_forces(sim, inst):
    cx, cy = G.default_center(inst["nx"], inst["ny"])
    Ez, Hx, Hy = sim.phasors()
    return mst.force_torque(Ez, Hx, Hy, cx, cy, inst["R"], mst.default_n_points(inst["R"]), inst["a"])


SMALL = W.small_cases()


@pytest.mark.parametrize("inst", SMALL + W.homogeneous_dielectric_256(), ids=lambda i: f"{i['nx']}x{i['ny']}")
def test_rasterisation_bit_exact(inst):
    j = L.make_janus(inst["a"], inst["phi0"], inst["eps1"], inst["eps2"], inst["pec2"])
    gpu = L.rasterize_janus(j, inst["nx"], inst["ny"])
    ref = G.janus_regions(inst["nx"], inst["ny"], inst["a"], inst["phi0"])
    assert np.array_equal(gpu, ref)


@pytest.mark.parametrize("phi0", np.linspace(0, 2 * np.pi, 13))
def test_rasterisation_ties(phi0):
    """Angles where many sites lie exactly on the interface (multiples of 30 deg)."""
    j = L.make_janus(40, phi0, 2.0, 3.0)
    assert np.array_equal(L.rasterize_janus(j, 128, 96), G.janus_regions(128, 96, 40, phi0))


@pytest.mark.parametrize("kind", ["hard", "open"])
@pytest.mark.parametrize("inst", SMALL, ids=lambda i: f"{i['nx']}x{i['ny']}")
def test_fp64_fields_and_forces_match_oracle(inst, kind):
    gpu_kind, oracle_kind = KINDS[kind]
    sim, reg = oracle_sim(inst, oracle_kind)
    n_run = (inst["periods"] - 1) * inst["period"] + 7
    with L.solver_for_instance(inst, "f64", kind=gpu_kind) as s:
        ids, _ = s.material()
        assert np.array_equal(ids, reg)
        s.step(n_run)
        sim.advance(n_run)
        assert fields_rel_l2(s.fields(), sim.fields()) < 1e-10
        F = s.force_torque(L.make_contour(inst["R"], inst["a"]))
        sim.advance(inst["period"], accumulate=True)
        Fo = oracle_forces(sim, inst)
        assert np.max(np.abs(F - Fo)) < 1e-10 * np.sum(np.abs(Fo))
        xy, ph = s.phasors()
        oE, oX, oY = sim.phasors()
        ref = np.stack([oE.real, oE.imag, oX.real, oX.imag, oY.real, oY.imag], -1)[xy[:, 1], xy[:, 0]]
        assert rel_l2(ph, ref) < 1e-10
        assert s.t == sim.t


def test_fields_right_after_start_and_odd_counts():
    inst = SMALL[1]
    sim, _ = oracle_sim(inst)
    with L.solver_for_instance(inst, "f64") as s:
        for n in (0, 1, 2, 31, 33, 64):
            s.step(n)
            sim.advance(n)
            ez, hx, hy = s.fields()
            oz, ox, oy = sim.fields()
            assert np.max(np.abs(ez - oz)) < 1e-12 and np.max(np.abs(hy - oy)) < 1e-12


def test_fp32_storage_forces_within_tolerance():
    """Homogeneous eps = 2.25 cylinder on 256^2 (T = 120, 20 periods): FP32 storage
    against the FP64 run."""
    inst = W.homogeneous_dielectric_256()[0]
    F64 = L.run_instance(inst, "f64")
    F32 = L.run_instance(inst, "f32")
    scale = abs(F64[0])
    assert abs(F32[0] - F64[0]) < 1e-4 * scale
    assert abs(F32[1] - F64[1]) < 1e-3 * scale and abs(F32[2] - F64[2]) < 1e-3 * scale


def test_full_size_first_period_matches_oracle():
    """512^2 metallo-dielectric workload in the benchmark's launch configuration:
    every site after one period (96 steps) against the oracle."""
    inst = W.md_janus_512()[1]
    sim, _ = oracle_sim(inst)
    with L.solver_for_instance(inst, "f64") as s:
        s.step(inst["period"])
        sim.advance(inst["period"])
        assert fields_rel_l2(s.fields(), sim.fields()) < 1e-10


def test_full_size_mirror_symmetry():
    """Full 30-period run at 512^2: phi0 and pi - phi0 are mirror images, so drag is
    equal and lift and torque are opposite (Sec. IV.A); phi0 = pi/2 has neither."""
    base = dict(W.md_janus_512()[0])
    base["eps1"] = 4.0
    F = {}
    for th in (30.0, 150.0, 90.0):
        inst = dict(base, phi0=np.radians(th))
        F[th] = L.run_instance(inst, "f64")
    scale = abs(F[30.0][0])
    assert abs(F[30.0][0] - F[150.0][0]) < 1e-10 * scale
    assert abs(F[30.0][1] + F[150.0][1]) < 1e-10 * scale
    assert abs(F[30.0][2] + F[150.0][2]) < 1e-10 * scale
    assert abs(F[90.0][1]) < 1e-10 * scale and abs(F[90.0][2]) < 1e-10 * scale


def test_checkpoint_resume_is_bit_exact():
    inst = SMALL[2]
    c = L.make_contour(inst["R"], inst["a"])
    with L.solver_for_instance(inst, "f64") as a, L.solver_for_instance(inst, "f64") as b:
        a.step(50)
        a.set_contour(c)
        a.accumulate(13)
        blob = a.save_state()
        a.accumulate(40)
        Fa = a.contour_integral()
        b.set_contour(c)
        b.load_state(blob)
        assert b.t == 63
        b.accumulate(40)
        Fb = b.contour_integral()
        assert np.array_equal(Fa, Fb)
        for x, y in zip(a.fields(), b.fields()):
            assert np.array_equal(x, y)


def test_runaway_field_is_reported():
    """A drive the FP32 form cannot represent (E0 = 1e39, beyond the FP32 range) makes the
    fields non-finite and sets the sticky error word; sync reports EUNSTABLE and the context
    stays usable.  (The threshold for finite fields is relative to E0:
    test_gpu_amplitude.py.)"""
    j = L.make_janus(6, 0.3, 2.0)
    with L.Solver(48, 40, "f32", janus=j, source=L.make_source(24, 0, E0=1e39)) as s:
        s.step(40)
        with pytest.raises(L.LbmEmError) as e:
            s.sync()
        assert e.value.status == L.EUNSTABLE
    with L.Solver(48, 40, "f32", janus=j, source=L.make_source(24)) as s:
        s.step(40)
        s.sync()


def test_user_stream():
    import torch
    st = torch.cuda.Stream()
    inst = SMALL[0]
    ref = L.run_instance(inst, "f64")
    got = L.run_instance(inst, "f64", stream=st)
    assert np.array_equal(ref, got)

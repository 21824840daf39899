"""Double-float storage (LBM_EM_F32X2: pairs of FP32, ~48 significant bits, FP32-pipe
arithmetic) against the FP64 oracle at the FP64 parity bound, and against the GPU FP64
form on long runs."""
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


def _rel(got, ref):
    num = sum(np.linalg.norm(a - b) ** 2 for a, b in zip(got, ref))
    den = sum(np.linalg.norm(b) ** 2 for b in ref)
    return float(np.sqrt(num / den))


@pytest.mark.parametrize("pol", ["tm", "te"])
@pytest.mark.parametrize("inst", W.small_cases(), ids=lambda i: f"{i['nx']}x{i['ny']}")
def test_f32x2_fields_and_forces_match_oracle(inst, pol):
    """Fields (relative L2 of the state) and forces (drag scale) within the FP64 bound 1e-10."""
    eps, pec, _ = G.janus_material(inst["nx"], inst["ny"], inst["a"], inst["phi0"], inst["eps1"],
                                   inst["eps2"], inst["pec2"])
    sim = OL.Simulation(eps, pec, period=inst["period"], ramp_steps=inst["ramp"], polarization=pol)
    n_run = (inst["periods"] - 1) * inst["period"] + 7
    with L.solver_for_instance(inst, "f32x2", polarization=pol) as s:
        s.step(n_run)
        sim.advance(n_run)
        assert _rel(s.fields(), sim.fields()) < 1e-10
        F = s.force_torque(L.make_contour(inst["R"], inst["a"]))
    sim.advance(inst["period"], accumulate=True)
    cx, cy = G.default_center(inst["nx"], inst["ny"])
    Fo = mst.force_torque(*sim.phasors(), cx, cy, inst["R"], mst.default_n_points(inst["R"]), inst["a"])
    assert np.max(np.abs(F - Fo)) < 1e-10 * np.sum(np.abs(Fo))


def test_f32x2_benchmark_instances_match_fp64():
    """The benchmark workload (512^2 metallo-dielectric Janus, 30 periods = 2 880 steps):
    forces within 1e-10 of drag scale of the GPU FP64 form."""
    for inst in W.md_janus_512()[:3]:
        F64 = L.run_instance(inst, "f64")
        F2 = L.run_instance(inst, "f32x2")
        assert np.max(np.abs(F2 - F64)) < 1e-10 * np.sum(np.abs(F64)), (F2, F64)


def test_f32x2_has_no_amplitude_drift():
    """Vacuum plane wave carried 4 000 cells (15 000 steps): phasors at x = 4 000 within 1e-10
    of the FP64 form's (the double-float constants carry a bias of ~2^-48 per step)."""
    nx, ny, T = 4400, 8, 240
    eps = np.ones((ny, nx))
    src = L.make_source(T)
    ph = {}
    for p in ("f64", "f32x2"):
        with L.Solver(nx, ny, p, eps_map=eps, source=src) as s:
            s.step(15000)
            s.set_contour(L.make_contour(2.0, 1.0, cx=4000.5, cy=3.5))
            s.accumulate(T)
            ph[p] = s.phasors()[1]
    assert np.linalg.norm(ph["f32x2"] - ph["f64"]) < 1e-10 * np.linalg.norm(ph["f64"])


def test_f32x2_checkpoint_and_energy():
    inst = W.small_cases()[0]
    with L.solver_for_instance(inst, "f32x2") as a, L.solver_for_instance(inst, "f32x2") as b, \
            L.solver_for_instance(inst, "f64") as c:
        a.step(37)
        blob = a.save_state()
        a.step(41)
        b.load_state(blob)
        b.step(41)
        c.step(78)
        for x, y in zip(a.fields(), b.fields()):
            assert np.array_equal(x, y)
        assert abs(a.energy() - c.energy()) < 1e-10 * c.energy()

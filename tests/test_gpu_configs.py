"""The large workloads on the GPU: per-form force errors against the FP64 GPU run, and a
full-size check against the oracle inside the light cone."""
import numpy as np
import pytest

from oracle import geometry as G
from oracle import lbm as OL
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


def _errors(F, ref):
    scale = abs(ref[0])
    return abs(F[0] - ref[0]) / scale, max(abs(F[1] - ref[1]), abs(F[2] - ref[2])) / scale


@pytest.mark.parametrize("k0a", [20.0, 10.0, 5.0])
def test_dielectric_janus_2048_forms(k0a):
    """2048^2 dielectric Janus (a = 128, eps1 = 2), FP32 and FP16-deviation storage against
    FP64: FP32 drag within 1e-4, lift and torque within 1e-3 of drag; FP16-deviation
    within 1e-3 of drag scale."""
    insts = [i for i in W.dielectric_janus_2048() if abs(2 * np.pi * 128 / (i["period"] / 3) - k0a) < 0.2 * k0a]
    assert len(insts) == 5
    assert all(i["periods"] * i["period"] > 3 * (1023.5 + i["R"]) + 19 * i["period"] for i in insts)
    for inst in insts[1::2]:                      # eps2 = 4.5 and 9.5
        ref = L.run_instance(inst, "f64")
        d32, lt32 = _errors(L.run_instance(inst, "f32"), ref)
        d16, lt16 = _errors(L.run_instance(inst, "f16dev"), ref)
        assert d32 < 1e-4 and lt32 < 1e-3, (inst["eps2"], d32, lt32)
        assert max(d16, lt16) < 1e-3, (inst["eps2"], d16, lt16)


def test_md_janus_8192_forms():
    """8192^2 metallo-dielectric Janus (a = 512, T = 240), run until 20 periods after the
    incident front has crossed the contour (81 periods, 19 440 steps): FP32 and
    FP16-deviation storage against the FP64 run."""
    inst = W.settled(W.md_janus_8192()[0])
    assert inst["periods"] == 81
    ref = L.run_instance(inst, "f64")
    d32, lt32 = _errors(L.run_instance(inst, "f32"), ref)
    d16, lt16 = _errors(L.run_instance(inst, "f16dev"), ref)
    assert d32 < 1e-4 and lt32 < 1e-3, (d32, lt32)
    assert max(d16, lt16) < 1e-3, (d16, lt16)


def test_md_janus_8192_light_cone_matches_oracle():
    """Full-size FP64 run for 240 steps (one period): populations move one site per step,
    so the fields at x < 230 depend only on the left strip x < 480 of the lattice, which the
    oracle runs exactly (same rows, source, top and bottom edges)."""
    inst = W.md_janus_8192()[0]
    strip = 480
    eps, pec, _ = G.janus_material(inst["nx"], inst["ny"], inst["a"], inst["phi0"], inst["eps1"],
                                   inst["eps2"], inst["pec2"])
    sim = OL.Simulation(np.ascontiguousarray(eps[:, :strip]), np.ascontiguousarray(pec[:, :strip]),
                        period=inst["period"], ramp_steps=inst["ramp"])
    sim.advance(inst["period"])
    with L.solver_for_instance(inst, "f64") as s:
        s.step(inst["period"])
        got = s.fields()
    ref = sim.fields()
    num = sum(np.linalg.norm(g[:, :230] - r[:, :230]) ** 2 for g, r in zip(got, ref))
    den = sum(np.linalg.norm(r[:, :230]) ** 2 for r in ref)
    assert np.sqrt(num / den) < 1e-10

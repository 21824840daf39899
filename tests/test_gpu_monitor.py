"""Convergence monitor (Sec. III: the total electromagnetic energy in the domain
approaches a constant) and runs that stop once it has, on the GPU."""
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


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5), ("f16dev", 2e-3)])
def test_energy_matches_definition_on_oracle_fields(prec, tol):
    """W = sum (eps E_z^2 + H_x^2 + H_y^2) / 2 against the same sum over the oracle's fields."""
    inst = W.small_cases()[1]
    eps, pec, _ = G.janus_material(inst["nx"], inst["ny"], inst["a"], inst["phi0"], inst["eps1"],
                                   inst["eps2"], inst["pec2"])
    sim = OL.Simulation(eps, pec, period=inst["period"], ramp_steps=inst["ramp"])
    sim.advance(2 * inst["period"] + 5)
    Ez, Hx, Hy = sim.fields()
    ref = 0.5 * np.sum(eps * Ez ** 2 + Hx ** 2 + Hy ** 2)
    with L.solver_for_instance(inst, prec) as s:
        s.step(2 * inst["period"] + 5)
        assert abs(s.energy() - ref) <= tol * ref


def test_run_converged_stops_early_and_agrees_with_long_run():
    inst = dict(W.small_cases()[0], periods=60)
    c = L.make_contour(inst["R"], inst["a"])
    with L.solver_for_instance(inst, "f64") as s:
        F, n = s.run_converged(c, tol=1e-4, min_periods=4, max_periods=60)
    T = inst["period"]
    assert 4 * T <= n < 60 * T and n % T == 1
    ref = L.run_instance(inst, "f64")
    assert np.max(np.abs(F - ref)) < 1e-2 * abs(ref[0])


def test_run_converged_respects_max_periods():
    inst = W.small_cases()[3]
    c = L.make_contour(inst["R"], inst["a"])
    with L.solver_for_instance(inst, "f32") as s:
        F, n = s.run_converged(c, tol=0.0, min_periods=2, max_periods=5)
        assert n == 5 * inst["period"] and s.t == 5 * inst["period"]


def test_batch_convergence_exits_match_single_domain_runs():
    """Per-instance early exits in the batched kernel follow the single-domain schedule:
    same steps and (up to summation order) the same forces."""
    insts = [dict(i, periods=40) for i in W.small_cases()]
    b = L.Batch(insts, "f64", conv_tol=1e-4, min_periods=4)
    b.run()
    F, st = b.results()
    steps = b.steps()
    for i, inst in enumerate(insts):
        with L.solver_for_instance(inst, "f64") as s:
            Fs, n = s.run_converged(L.make_contour(inst["R"], inst["a"]), tol=1e-4, min_periods=4, max_periods=40)
        assert steps[i] == n, (i, steps[i], n)
        assert np.max(np.abs(F[i] - Fs)) < 1e-10 * np.sum(np.abs(Fs))
    assert (steps < 40 * np.array([i["period"] for i in insts])).any()
    b.close()

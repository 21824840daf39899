"""TE^z polarization (H_z, E_x, E_y) on the GPU: parity with the oracle's full-vector
scheme, the FP32 storage form, two steps per launch, the energy monitor and the far field.
The paper leaves TE for future work; the scheme and the state layout are the TM ones."""
import numpy as np
import pytest

from oracle import geometry as G
from oracle import lbm as OL
from oracle import mst, ntff
from paper_2509_22308_gb300 import lbm_em as L
from paper_2509_22308_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KINDS = {"hard": (L.SRC_HARD, OL.SRC_HARD), "open": (L.SRC_OPEN, OL.SRC_OPEN)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_22308_gb300 import build
    build.build()


def _oracle(inst, kind=OL.SRC_HARD):
    eps, pec, _ = G.janus_material(inst["nx"], inst["ny"], inst["a"], inst["phi0"], inst["eps1"],
                                   inst["eps2"], inst["pec2"])
    return OL.Simulation(eps, pec, period=inst["period"], ramp_steps=inst["ramp"], source_kind=kind,
                         polarization="te"), eps


def _rel(got, ref):
    num = sum(np.linalg.norm(a - b) ** 2 for a, b in zip(got, ref))
    den = sum(np.linalg.norm(b) ** 2 for b in ref)
    return float(np.sqrt(num / den))


@pytest.mark.parametrize("kind", ["hard", "open"])
@pytest.mark.parametrize("inst", W.small_cases(), ids=lambda i: f"{i['nx']}x{i['ny']}")
def test_te_fp64_fields_and_forces_match_oracle(inst, kind):
    gk, ok = KINDS[kind]
    sim, _ = _oracle(inst, ok)
    n_run = (inst["periods"] - 1) * inst["period"] + 7
    with L.solver_for_instance(inst, "f64", kind=gk, polarization="te") as s:
        s.step(n_run)
        sim.advance(n_run)
        assert _rel(s.fields(), sim.fields()) < 1e-10
        F = s.force_torque(L.make_contour(inst["R"], inst["a"]))
    sim.advance(inst["period"], accumulate=True)
    cx, cy = G.default_center(inst["nx"], inst["ny"])
    Fo = mst.force_torque(*sim.phasors(), cx, cy, inst["R"], mst.default_n_points(inst["R"]), inst["a"])
    assert np.max(np.abs(F - Fo)) < 1e-10 * np.sum(np.abs(Fo))


def test_te_fp32_forces_within_tolerance():
    """Homogeneous eps = 2.25 cylinder (256^2, T = 120, 20 periods) and a metallo-dielectric
    Janus instance of the benchmark workload in TE: FP32 storage against FP64, drag within
    1e-4 relative, lift and torque within 1e-3 of drag."""
    for inst in W.homogeneous_dielectric_256() + W.md_janus_512()[1:2]:
        F64 = L.run_instance(inst, "f64", polarization="te")
        F32 = L.run_instance(inst, "f32", polarization="te")
        scale = abs(F64[0])
        assert abs(F32[0] - F64[0]) < 1e-4 * scale
        assert max(abs(F32[1] - F64[1]), abs(F32[2] - F64[2])) < 1e-3 * scale


@pytest.mark.parametrize("inst", W.small_cases()[:3], ids=lambda i: f"{i['nx']}x{i['ny']}")
def test_te_two_steps_per_launch_is_bit_identical(inst):
    with L.solver_for_instance(inst, "f32", steps_per_launch="two", polarization="te") as a, \
            L.solver_for_instance(inst, "f32", steps_per_launch="one", polarization="te") as b:
        for n in (1, 2, 5, 32, 33, 3):
            a.step(n)
            b.step(n)
            for x, y in zip(a.fields(), b.fields()):
                assert np.array_equal(x, y)
        c = L.make_contour(inst["R"], inst["a"])
        assert np.array_equal(a.force_torque(c), b.force_torque(c))


def test_te_energy_matches_definition_on_oracle_fields():
    """W = sum (eps (E_x^2 + E_y^2) + H_z^2) / 2 against the same sum over the oracle's fields."""
    inst = W.small_cases()[1]
    sim, eps = _oracle(inst)
    sim.advance(2 * inst["period"] + 5)
    Hz, Ex, Ey = sim.fields()
    ref = 0.5 * np.sum(eps * (Ex ** 2 + Ey ** 2) + Hz ** 2)
    with L.solver_for_instance(inst, "f64", polarization="te") as s:
        s.step(2 * inst["period"] + 5)
        assert abs(s.energy() - ref) <= 1e-10 * ref


def test_te_far_field_matches_oracle_transform():
    inst = W.small_cases()[2]
    sim, _ = _oracle(inst)
    sim.advance((inst["periods"] - 1) * inst["period"])
    sim.advance(inst["period"], accumulate=True)
    cx, cy = G.default_center(inst["nx"], inst["ny"])
    phis = np.linspace(0, 2 * np.pi, 25)[:-1]
    ref = ntff.scattering_intensity_lattice(*sim.phasors(), inst["period"], cx, cy, inst["R"],
                                            2 * int(np.ceil(2 * np.pi * inst["R"])), phis, te=True)
    with L.solver_for_instance(inst, "f64", polarization="te") as s:
        s.step((inst["periods"] - 1) * inst["period"])
        s.force_torque(L.make_contour(inst["R"], inst["a"]))
        got = s.far_field(phis)
    assert np.max(np.abs(got - ref)) < 1e-10 * np.max(ref)


def test_te_far_field_matches_bessel_series():
    """Sec. IV.A's far-field validation, carried to TE^z: homogeneous dielectric cylinder
    (eps = 2.25), a = lambda, lambda_eps / dx = 50, L/a = 10, run until the energy has settled;
    |S(phi)|^2 of H_z within 5 % of the TE Bessel series at most angles (median)."""
    from oracle import analytic as A
    eps = 2.25
    lam = 50.0 * np.sqrt(eps)
    T = int(round(3 * lam))
    a = T / 3.0
    n = int(round(10 * a)) // 2 * 2
    inst = dict(nx=n, ny=n, a=a, phi0=0.0, eps1=eps, eps2=eps, pec2=False, period=T, periods=30,
                R=1.5 * a, ramp=T)
    phis = np.linspace(0, 2 * np.pi, 73)[:-1]
    with L.solver_for_instance(inst, "f64", polarization="te") as s:
        _, steps = s.run_converged(L.make_contour(inst["R"], a), tol=1e-6, min_periods=20, max_periods=800)
        assert steps < 800 * T
        S = s.far_field(phis)
    k = ntff.lattice_wavenumber(T)
    B, D = A.homogeneous_BD(k, a, eps, 0.0, te=True)
    Sa = A.scattering_intensity(B, D, phis + np.pi)
    rel = np.abs(S - Sa) / Sa
    print(f"TE far field: steps={steps} median={np.median(rel):.4f} within5%={np.mean(rel < 0.05):.2f}")
    assert np.median(rel) < 0.05, (np.median(rel), steps)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_te_batch_matches_single_domain(prec):
    """TE^z instances of uneven size in one batch: the forces of every instance equal its
    single-domain TE run (same per-site arithmetic; only the contour sum order differs)."""
    insts = W.small_cases()
    b = L.Batch(insts, prec, polarization="te")
    try:
        b.run()
        F, st = b.results()
    finally:
        b.close()
    assert (st == L.OK).all()
    for i, inst in enumerate(insts):
        ref = L.run_instance(inst, prec, polarization="te")
        assert np.max(np.abs(F[i] - ref)) < 1e-12 * np.sum(np.abs(ref)), (i, F[i], ref)


def test_te_batch_two_steps_per_launch_is_bit_identical():
    insts = W.small_cases()
    insts[0] = dict(insts[0], period=61, ramp=61)  # an odd run length: the last launch takes one step
    b2 = L.Batch(insts, "f32", tile_w=64, tile_h=8, ctas_per_sm=3, polarization="te")
    b1 = L.Batch(insts, "f32", tile_w=64, tile_h=4, ctas_per_sm=4, polarization="te")
    try:
        assert b2.config() == (64, 8, 3)
        b2.run()
        b1.run()
        F2, s2 = b2.results()
        F1, _ = b1.results()
    finally:
        b1.close()
        b2.close()
    assert (s2 == L.OK).all()
    assert np.array_equal(F1, F2)

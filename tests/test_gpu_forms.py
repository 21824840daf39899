"""Storage forms and the batched path on the GPU.

FP16-deviation storage: forces within 1e-3 of drag scale of the FP64 run (the
design-map accuracy bar).  Batched runs: every instance of a packed batch with
uneven sizes and run lengths equals its single-domain run (same per-site
arithmetic; only the contour sum order differs)."""
import numpy as np
import pytest

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


def test_f16dev_forces_within_design_map_tolerance():
    for inst in W.homogeneous_dielectric_256() + W.md_janus_512()[:3]:
        F64 = L.run_instance(inst, "f64")
        F16 = L.run_instance(inst, "f16dev")
        scale = abs(F64[0])
        assert np.max(np.abs(F16 - F64)) < 1e-3 * scale, (F16, F64)


def test_f16dev_fields_track_fp64():
    inst = W.small_cases()[1]
    with L.solver_for_instance(inst, "f64") as a, L.solver_for_instance(inst, "f16dev") as b:
        a.step(150)
        b.step(150)
        fa, fb = a.fields(), b.fields()
        num = sum(np.linalg.norm(x - y) ** 2 for x, y in zip(fa, fb))
        den = sum(np.linalg.norm(x) ** 2 for x in fa)
        assert np.sqrt(num / den) < 2e-3


@pytest.mark.parametrize("prec,tol", [("f32", 1e-5), ("f16dev", 1.5e-4)])
def test_reduced_precision_has_no_amplitude_drift(prec, tol):
    """Vacuum plane wave carried 4 000 cells (15 000 steps at T = 240): the reduced-precision
    phasors at x = 1 000 and x = 4 000 stay within tol of the FP64 ones.  The scheme has no
    damping at tau = 1/2, so a fixed rounding bias in the equilibria (1/3 rounded to FP32)
    would grow the wave by about 6e-8 per step, 4e-4 at x = 4 000 here.  Phasors (one
    period of Fourier accumulation at a small contour's stencil sites), not instantaneous
    fields: the forces use phasors, and FP16 rounding noise spread over all frequencies
    (~3e-4 of the instantaneous field) averages out of them."""
    nx, ny, T = 4400, 8, 240
    eps = np.ones((ny, nx))
    src = L.make_source(T)
    for xc in (1000.5, 4000.5):
        ph = {}
        for p in ("f64", prec):
            with L.Solver(nx, ny, p, eps_map=eps, source=src) as s:
                s.step(15000)
                s.set_contour(L.make_contour(2.0, 1.0, cx=xc, cy=3.5))
                s.accumulate(T)
                ph[p] = s.phasors()[1]
        err = np.linalg.norm(ph[prec] - ph["f64"]) / np.linalg.norm(ph["f64"])
        assert err < tol, (prec, xc, err)


def test_f16dev_checkpoint_resume_is_bit_exact():
    inst = W.small_cases()[0]
    with L.solver_for_instance(inst, "f16dev") as a, L.solver_for_instance(inst, "f16dev") as b:
        a.step(37)
        blob = a.save_state()
        a.step(41)
        b.load_state(blob)
        b.step(41)
        for x, y in zip(a.fields(), b.fields()):
            assert np.array_equal(x, y)


def _batch_instances():
    insts = W.small_cases()
    # different run lengths and periods (the longest instance finishes last)
    insts[0] = dict(insts[0], periods=5)
    insts[3] = dict(insts[3], periods=2)
    return insts


@pytest.mark.parametrize("prec", ["f64", "f32", "f32x2"])
def test_batch_matches_single_domain(prec):
    insts = _batch_instances()
    b = L.Batch(insts, prec)
    b.run()
    F, st = b.results()
    assert (st == L.OK).all()
    for i, inst in enumerate(insts):
        ref = L.run_instance(inst, prec)
        assert np.max(np.abs(F[i] - ref)) < 1e-12 * np.sum(np.abs(ref)), (i, F[i], ref)
    w, h, c = b.config()
    assert (w in (32, 40, 64, 128, 256) and 1 <= h <= 16 and c >= 1) or (w == 56 and h in (64, 128, 256) and c >= 1)
    b.run()                      # a second run starts from a cleared state
    F2, _ = b.results()
    assert np.array_equal(F, F2)
    b.close()


def test_batch_explicit_configuration():
    insts = _batch_instances()
    b = L.Batch(insts, "f32", tile_w=128, tile_h=2, ctas_per_sm=2)
    assert b.config() == (128, 2, 2)
    b.run()
    F, _ = b.results()
    for i, inst in enumerate(insts):
        ref = L.run_instance(inst, "f32")
        assert np.max(np.abs(F[i] - ref)) < 1e-12 * np.sum(np.abs(ref))
    b.close()


@pytest.mark.parametrize("shape", [(64, 8), (32, 16), (40, 12)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_batch_two_steps_per_launch_is_bit_identical(shape):
    """The FP32 batch with two steps per launch (64 x 8, 32 x 16 or 40 x 12 tiles staged by TMA with their halo)
    gives the same bits as the one-step batch kernel, for uneven sizes and run lengths
    (odd step counts end with a one-step launch), and matches the single-domain runs."""
    insts = _batch_instances()
    insts[0] = dict(insts[0], period=61, ramp=61)    # 305 steps: the run ends with one step
    insts[1] = dict(insts[1], period=45, ramp=45)    # 135 steps: a launch's second step is skipped
    b2 = L.Batch(insts, "f32", tile_w=shape[0], tile_h=shape[1], ctas_per_sm=3)
    b1 = L.Batch(insts, "f32", tile_w=64, tile_h=4, ctas_per_sm=4)
    assert b2.config() == (shape[0], shape[1], 3)
    b2.run()
    b1.run()
    F2, s2 = b2.results()
    F1, _ = b1.results()
    assert (s2 == L.OK).all()
    assert np.array_equal(F1, F2)
    for i, inst in enumerate(insts):
        ref = L.run_instance(inst, "f32")
        assert np.max(np.abs(F2[i] - ref)) < 1e-12 * np.sum(np.abs(ref))
    b1.close()
    b2.close()


def test_batch_reports_unstable_instance():
    insts = _batch_instances()[:2]
    b = L.Batch(insts, "f32")
    b._L.lbm_em_batch_destroy(b.b)
    b.b = None
    # an instance whose drive the FP32 form cannot represent (E0 = 1e39: non-finite fields) is
    # flagged on its own
    import ctypes
    arr = (L.Instance * 2)()
    for i, inst in enumerate(insts):
        arr[i] = L.Instance(inst["nx"], inst["ny"], inst["period"], inst["periods"], inst["ramp"], 0,
                            1e39 if i == 1 else 1.0, inst["R"],
                            L.make_janus(inst["a"], inst["phi0"], inst["eps1"], inst["eps2"], inst["pec2"]))
    o = L.BatchOpts(L.F32, 64, 4, 2, 0, 0, 0.0, None)
    h = ctypes.c_void_p()
    L._call("lbm_em_batch_create", arr, 2, ctypes.byref(o), ctypes.byref(h))
    L._call("lbm_em_batch_run", h)
    out = np.zeros(6)
    st = np.zeros(2, dtype=np.int32)
    rc = L.load().lbm_em_batch_results(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       st.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    assert rc == L.EUNSTABLE and st[0] == L.OK and st[1] == L.EUNSTABLE
    L.load().lbm_em_batch_destroy(h)


@pytest.mark.parametrize("prec", ["f32", "f16dev", "f32x2"])
@pytest.mark.parametrize("inst", W.small_cases()[:3], ids=lambda i: f"{i['nx']}x{i['ny']}")
def test_two_steps_per_launch_is_bit_identical(inst, prec):
    """Two steps per launch (temporal blocking) equals one step per launch bit for bit,
    for even and odd step counts and through the accumulating period; the FP16-deviation
    form rounds the intermediate state exactly as storing it would."""
    with L.solver_for_instance(inst, prec, steps_per_launch="two") as a, \
            L.solver_for_instance(inst, prec, steps_per_launch="one") as b:
        for n in (1, 2, 5, 32, 33, 64, 3):
            a.step(n)
            b.step(n)
            for x, y in zip(a.fields(), b.fields()):
                assert np.array_equal(x, y)
        c = L.make_contour(inst["R"], inst["a"])
        assert np.array_equal(a.force_torque(c), b.force_torque(c))


@pytest.mark.parametrize("prec,mode", [("f32", "two"), ("f16dev", "two"), ("f32", "three"), ("f32", "four")])
@pytest.mark.parametrize("shape", [(7, 5), (28, 12), (32, 16), (64, 8), (128, 48), (33, 17), (29, 13), (200, 35),
                                   (56, 9), (57, 4), (113, 23)],
                         ids=lambda s: f"{s[0]}x{s[1]}")
def test_multi_steps_on_tile_edge_shapes(shape, prec, mode):
    """The TMA-staged kernels copy 64 x 8 tiles with a two-site halo for two steps per launch
    (boxes of 72 x 12 sites in FP32; 80 x 12 deviations and 72 x 12 fields in the
    FP16-deviation form) and 28 x 12 tiles with a three-site halo for three (36 x 18); the
    four-step kernel streams strips of 56 output columns (64-column rows) down the lattice:
    a lattice smaller than the box in both directions, exactly one tile or strip, exact
    multiples and one site beyond them, odd widths, and lattices shorter than the four rows a
    strip's pipeline spans all give the bits of one step per launch (fields, over step counts
    of every residue)."""
    nx, ny = shape
    a = min(nx, ny) / 3.0
    inst = dict(nx=nx, ny=ny, a=a, phi0=0.4, eps1=3.0, eps2=1.0, pec2=True, period=24, periods=3,
                R=a, ramp=24)
    with L.solver_for_instance(inst, prec, steps_per_launch=mode) as s2, \
            L.solver_for_instance(inst, prec, steps_per_launch="one") as s1:
        for n in (1, 2, 5, 33, 64, 3, 31):
            s2.step(n)
            s1.step(n)
            for x, y in zip(s2.fields(), s1.fields()):
                assert np.array_equal(x, y)
        assert np.abs(s2.fields()[0]).max() > 0  # the source has reached the field


@pytest.mark.parametrize("pol", ["tm", "te"])
@pytest.mark.parametrize("inst", W.small_cases()[:3], ids=lambda i: f"{i['nx']}x{i['ny']}")
def test_three_steps_per_launch_is_bit_identical(inst, pol):
    """Three steps per launch (FP32, 28 x 12 TMA tiles) equals one step per launch bit for bit,
    for step counts of every residue modulo 3, through graphs of 30 steps and through the
    accumulating period (forces)."""
    with L.solver_for_instance(inst, "f32", steps_per_launch="three", polarization=pol) as a, \
            L.solver_for_instance(inst, "f32", steps_per_launch="one", polarization=pol) as b:
        for n in (1, 3, 2, 30, 31, 64, 5):
            a.step(n)
            b.step(n)
            for x, y in zip(a.fields(), b.fields()):
                assert np.array_equal(x, y)
        c = L.make_contour(inst["R"], inst["a"])
        assert np.array_equal(a.force_torque(c), b.force_torque(c))


@pytest.mark.parametrize("pol", ["tm", "te"])
@pytest.mark.parametrize("inst", W.small_cases()[:3], ids=lambda i: f"{i['nx']}x{i['ny']}")
def test_four_steps_per_launch_accumulates_bit_identically(inst, pol):
    """Four steps per launch (FP32) takes the Fourier sums of the accumulated period inside the
    launch's time levels (its accumulating kernel): fields, the phasors at every stencil site and
    the forces equal one step per launch bit for bit, through graphs of 32 steps, remainders of
    every residue modulo 4, and an accumulated period that starts at an odd time."""
    with L.solver_for_instance(inst, "f32", steps_per_launch="four", polarization=pol) as a, \
            L.solver_for_instance(inst, "f32", steps_per_launch="one", polarization=pol) as b:
        assert a.steps_per_launch() == 4
        for n in (1, 4, 2, 32, 35, 64, 3):
            a.step(n)
            b.step(n)
            for x, y in zip(a.fields(), b.fields()):
                assert np.array_equal(x, y)
        c = L.make_contour(inst["R"], inst["a"])
        for extra in (0, 1):  # a second period from an odd start
            a.step(extra)
            b.step(extra)
            assert np.array_equal(a.force_torque(c), b.force_torque(c))
            (xa, pa), (xb, pb) = a.phasors(), b.phasors()
            assert np.array_equal(xa, xb) and np.array_equal(pa, pb)
            assert np.abs(pa).max() > 0
        for x, y in zip(a.fields(), b.fields()):
            assert np.array_equal(x, y)


def test_f16dev_split_runs_agree_bitwise():
    """The FP16-deviation form gives the same bits however a run is split into calls."""
    inst = W.small_cases()[2]
    with L.solver_for_instance(inst, "f16dev", steps_per_launch="two") as a, \
            L.solver_for_instance(inst, "f16dev", steps_per_launch="two") as b:
        a.step(77)
        for n in (3, 30, 1, 43):
            b.step(n)
        for x, y in zip(a.fields(), b.fields()):
            assert np.array_equal(x, y)


def test_f16dev_two_step_mode_within_tolerance():
    inst = W.homogeneous_dielectric_256()[0]
    F64 = L.run_instance(inst, "f64")
    F16 = L.run_instance(inst, "f16dev", steps_per_launch="two")
    assert np.max(np.abs(F16 - F64)) < 1e-3 * abs(F64[0])


def test_far_field_matches_oracle_transform():
    """GPU near-to-far-field transform against the oracle's transform of the oracle's
    own phasors (same seeded instance)."""
    from oracle import geometry as G
    from oracle import lbm as OL
    from oracle import ntff
    inst = W.small_cases()[1]
    eps, pec, _ = G.janus_material(inst["nx"], inst["ny"], inst["a"], inst["phi0"], inst["eps1"],
                                   inst["eps2"], inst["pec2"])
    sim = OL.Simulation(eps, pec, period=inst["period"], ramp_steps=inst["ramp"])
    sim.advance((inst["periods"] - 1) * inst["period"])
    sim.advance(inst["period"], accumulate=True)
    cx, cy = G.default_center(inst["nx"], inst["ny"])
    phis = np.linspace(0, 2 * np.pi, 25)[:-1]
    ref = ntff.scattering_intensity_lattice(*sim.phasors(), inst["period"], cx, cy, inst["R"],
                                            2 * int(np.ceil(2 * np.pi * inst["R"])), phis)
    with L.solver_for_instance(inst, "f64") as s:
        s.step((inst["periods"] - 1) * inst["period"])
        s.force_torque(L.make_contour(inst["R"], inst["a"]))
        got = s.far_field(phis)
    assert np.max(np.abs(got - ref)) < 1e-10 * np.max(ref)


@pytest.mark.parametrize("eps1,phi0", [(1.0, 0.0), (2.0, -np.pi / 4), (5.0, 0.0)])
def test_far_field_validation_at_paper_resolution(eps1, phi0):
    """Sec. IV.A far-field validation: metallo-dielectric Janus cylinder, a = lambda,
    lambda_eps / dx = 50 inside the dielectric, L/a = 10; the LBM |S(phi)|^2 agrees with
    the analytic one within 5 % at most scattering angles."""
    from oracle import analytic as A
    from oracle import ntff
    lam = 50.0 * np.sqrt(eps1)
    T = int(round(3 * lam))
    a = T / 3.0
    n = int(round(10 * a)) // 2 * 2
    inst = dict(nx=n, ny=n, a=a, phi0=phi0, eps1=eps1, eps2=1.0, pec2=True, period=T, periods=30,
                R=1.5 * a, ramp=T)
    phis = np.linspace(0, 2 * np.pi, 73)[:-1]
    with L.solver_for_instance(inst, "f64") as s:
        # run until the domain energy has settled (Sec. III); high contrast needs long runs
        # eps1 = 5 has a high-Q resonance: at tol 1e-5 the energy test passes after 76
        # periods while the far field is still settling (55 % of angles within 5 %); at
        # 1e-6 it runs 455 periods (64 %), as long as a 1e-7 run capped at 600 (65 %)
        _, steps = s.run_converged(L.make_contour(inst["R"], a), tol=1e-6, min_periods=20, max_periods=800)
        assert steps < 800 * T, "energy did not settle"
        S = s.far_field(phis)
    k = ntff.lattice_wavenumber(T)
    B, D, _ = A.md_janus_BD_galerkin(k, a, eps1, phi0, n_basis=320)
    Sa = A.scattering_intensity(B, D, phis + phi0 + np.pi)
    rel = np.abs(S - Sa) / Sa
    print(f"eps1={eps1} phi0={phi0:.3f} steps={steps} median={np.median(rel):.4f} within5%={np.mean(rel < 0.05):.2f}")
    assert np.median(rel) < 0.05 and np.mean(rel < 0.05) > 0.6, (np.median(rel), np.mean(rel < 0.05), steps)


def test_design_map_symmetry_and_trajectory():
    """A metallo-dielectric design map over phi0 from one batched run: drag symmetric,
    lift and torque antisymmetric about phi0 = pi/2 (Sec. IV.A), no torque at pi/2 and
    3 pi/2; a trajectory started off a torque-free orientation settles on a stable one."""
    from paper_2509_22308_gb300 import trajectory as TR
    n = 24
    F = TR.design_map(2.0, pec2=True, n_phi=n, a=16, periods=20, precision="f32")
    scale = np.abs(F[:, 0]).max()
    k = np.arange(n)
    mirror = (n // 2 - k) % n                     # phi0 -> pi - phi0
    assert np.max(np.abs(F[:, 0] - F[mirror, 0])) < 1e-4 * scale
    assert np.max(np.abs(F[:, 1] + F[mirror, 1])) < 1e-4 * scale
    assert np.max(np.abs(F[:, 2] + F[mirror, 2])) < 1e-4 * scale
    assert abs(F[n // 4, 2]) < 1e-4 * scale and abs(F[3 * n // 4, 2]) < 1e-4 * scale
    fmap = TR.PeriodicMap(F[:, 0], F[:, 1], F[:, 2])
    tr = TR.integrate(fmap, 0.1, t_final=2.0e4, dt=2.0)
    assert abs(fmap(tr[-1, 3])[0, 2]) < 1e-3 * scale
    assert tr[-1, 1] > 0                          # drag pushes along +x


def _random_shapes(seed, n, lo, hi):
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(lo, hi)), int(rng.integers(lo, hi))) for _ in range(n)]


@pytest.mark.parametrize("shape", _random_shapes(11, 8, 4, 300), ids=lambda s: f"{s[0]}x{s[1]}")
def test_fp32_two_steps_on_random_shapes(shape):
    """Seeded random lattice sizes (4 .. 299 per side): the TMA-staged two-step kernel gives the
    bits of one step per launch."""
    nx, ny = shape
    a = max(min(nx, ny) / 4.0, 1.0)
    inst = dict(nx=nx, ny=ny, a=a, phi0=1.1, eps1=2.5, eps2=6.0, pec2=False, period=30, periods=3, R=a,
                ramp=30)
    with L.solver_for_instance(inst, "f32", steps_per_launch="two") as s2, \
            L.solver_for_instance(inst, "f32", steps_per_launch="one") as s1:
        s2.step(37)
        s1.step(37)
        for x, y in zip(s2.fields(), s1.fields()):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("shape", [(64, 8), (32, 16), (40, 12)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_batch_two_steps_on_random_instance_sizes(shape):
    """Seeded random instance sizes (24 .. 259 per side, ragged against every tile shape) and
    run lengths in one batch: the two-step kernel's forces equal the one-step kernel's bits."""
    insts = []
    for k, (nx, ny) in enumerate(_random_shapes(23, 7, 24, 260)):
        a = min(nx, ny) / 6.0
        T = 24 + 6 * k
        insts.append(dict(nx=nx, ny=ny, a=a, phi0=0.4 * k, eps1=2.0, eps2=1.0 + k, pec2=k % 3 == 0, period=T,
                          periods=2 + k % 3, R=min(nx, ny) / 3.0, ramp=T))
    b2 = L.Batch(insts, "f32", tile_w=shape[0], tile_h=shape[1], ctas_per_sm=3)
    b1 = L.Batch(insts, "f32", tile_w=64, tile_h=4, ctas_per_sm=4)
    try:
        assert b2.config() == (shape[0], shape[1], 3)
        b2.run()
        b1.run()
        F2, s2 = b2.results()
        F1, s1 = b1.results()
    finally:
        b1.close()
        b2.close()
    assert (s2 == L.OK).all() and (s1 == L.OK).all()
    assert np.array_equal(F1, F2)


@pytest.mark.parametrize("inst", W.homogeneous_dielectric_256() + W.md_janus_512()[:3],
                         ids=lambda i: f"{i['nx']}-{i['phi0']:.2f}")
def test_f16dev_four_steps_within_tolerance(inst):
    """FP16-deviation storage with four steps per launch rounds the stored state once per
    launch (levels 1-3 of a launch stay FP32): forces within the design-map bar (1e-3 of drag)
    of FP64, at the level of the FP16 rounding noise of one step per launch (both measured at
    4e-6 to 1.2e-5 of drag on these workloads; which is smaller varies from instance to
    instance)."""
    F64 = L.run_instance(inst, "f64")
    F4 = L.run_instance(inst, "f16dev", steps_per_launch="four")
    F1 = L.run_instance(inst, "f16dev", steps_per_launch="one")
    scale = abs(F64[0])
    e4 = np.max(np.abs(F4 - F64)) / scale
    e1 = np.max(np.abs(F1 - F64)) / scale
    assert e4 < 1e-3, (F4, F64)
    assert e4 < 1e-4 and e1 < 1e-4, (e4, e1)


@pytest.mark.parametrize("shape", [(7, 5), (57, 4), (200, 35), (301, 77)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_f16dev_four_steps_track_one_step(shape):
    """Four FP16-deviation steps per launch against one per launch on edge shapes: the fields
    differ only by the FP16 rounding the four-step launch skips (relative L2 < 2e-3), and a
    run split at multiples of four steps gives the same bits as an unsplit one."""
    nx, ny = shape
    a = min(nx, ny) / 3.0
    inst = dict(nx=nx, ny=ny, a=a, phi0=0.4, eps1=3.0, eps2=1.0, pec2=True, period=24, periods=3, R=a, ramp=24)
    with L.solver_for_instance(inst, "f16dev", steps_per_launch="four") as s4, \
            L.solver_for_instance(inst, "f16dev", steps_per_launch="one") as s1, \
            L.solver_for_instance(inst, "f16dev", steps_per_launch="four") as s4b:
        s4.step(96)
        s1.step(96)
        for n in (8, 32, 4, 52):
            s4b.step(n)
        f4, f1 = s4.fields(), s1.fields()
        num = sum(np.linalg.norm(x - y) ** 2 for x, y in zip(f4, f1))
        den = sum(np.linalg.norm(y) ** 2 for y in f1)
        assert np.sqrt(num / den) < 2e-3
        for x, y in zip(f4, s4b.fields()):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("pol", ["tm", "te"])
def test_batch_four_steps_per_launch_is_bit_identical(pol):
    """The FP32 batch with four steps per launch (persistent warps streaming every instance's
    strips and row segments through four time levels in registers, Fourier sums accumulated
    inside the levels of each instance's last period) gives the forces of the one-step batch
    kernel bit for bit, for uneven sizes, periods and run lengths that are not multiples of four
    (an instance ending inside a launch runs on past its end; the last steps take one-step
    launches), and matches the single-domain runs."""
    insts = _batch_instances()
    insts[0] = dict(insts[0], period=61, ramp=61)    # 305 steps
    insts[1] = dict(insts[1], period=45, ramp=45)    # 135 steps
    b4 = L.Batch(insts, "f32", steps_per_launch=4, polarization=pol)
    b1 = L.Batch(insts, "f32", tile_w=64, tile_h=4, ctas_per_sm=4, polarization=pol)
    try:
        assert b4.steps_per_launch() == 4
        w, h, c = b4.config()
        assert w == 56 and h in (64, 128, 256) and c >= 1
        b4.run()
        b1.run()
        F4, s4 = b4.results()
        F1, _ = b1.results()
        b4.run()                  # a second run starts from a cleared state
        F4b, _ = b4.results()
    finally:
        b1.close()
        b4.close()
    assert (s4 == L.OK).all()
    assert np.array_equal(F1, F4) and np.array_equal(F4, F4b)
    for i, inst in enumerate(insts):
        ref = L.run_instance(inst, "f32", polarization=pol)
        assert np.max(np.abs(F4[i] - ref)) < 1e-12 * np.sum(np.abs(ref))


def test_batch_four_steps_on_random_instance_sizes():
    """Seeded random instance sizes (24 .. 259 per side: strips and row segments cut ragged) and
    run lengths: the four-step batch kernel's forces equal the one-step kernel's bits."""
    insts = []
    for k, (nx, ny) in enumerate(_random_shapes(31, 9, 24, 260)):
        a = min(nx, ny) / 6.0
        T = 24 + 5 * k
        insts.append(dict(nx=nx, ny=ny, a=a, phi0=0.3 * k, eps1=2.0, eps2=1.5 + k, pec2=k % 3 == 1, period=T,
                          periods=2 + k % 3, R=min(nx, ny) / 3.0, ramp=T))
    b4 = L.Batch(insts, "f32", steps_per_launch=4)
    b1 = L.Batch(insts, "f32", tile_w=64, tile_h=4, ctas_per_sm=4)
    try:
        b4.run()
        b1.run()
        F4, s4 = b4.results()
        F1, s1 = b1.results()
    finally:
        b1.close()
        b4.close()
    assert (s4 == L.OK).all() and (s1 == L.OK).all()
    assert np.array_equal(F1, F4)


def test_batch_rejects_bad_steps_per_launch():
    insts = _batch_instances()[:1]
    for prec, kw in (("f32", {"steps_per_launch": 3}), ("f64", {"steps_per_launch": 4}),
                     ("f32", {"steps_per_launch": 4, "conv_tol": 1e-3}),
                     ("f32", {"steps_per_launch": 4, "tile_w": 64})):
        with pytest.raises(L.LbmEmError) as e:
            L.Batch(insts, prec, **kw)
        assert e.value.status == L.EINVAL


@pytest.mark.parametrize("ctas", [0, 1])
def test_batch_four_steps_on_the_design_map(ctas):
    """The 256-instance design map, shortened to 8 periods (the incident front crosses every
    instance's contour by then), about 34 000 work units, including the last row segment of
    instances where the wavefront drains past the lattice's last row.  ctas 0: one warp per
    unit; ctas 1: a persistent grid of one block per SM (608 warps), so every warp takes about
    56 units in turn and its row ring carries its slot and barrier phase over from unit to
    unit.  Forces equal the two-step kernel's bits (which equal one step per launch), and no
    row copy times out."""
    dm = [dict(i, periods=8) for i in W.design_map_256(4, 256)]
    b4 = L.Batch(dm, "f32", steps_per_launch=4, ctas_per_sm=ctas)
    b2 = L.Batch(dm, "f32", tile_w=64, tile_h=8, ctas_per_sm=3, steps_per_launch=2)
    try:
        assert b4.steps_per_launch() == 4
        if ctas:
            assert b4.config()[2] == ctas
        b4.run()
        b2.run()
        F4, s4 = b4.results()
        F2, s2 = b2.results()
    finally:
        b2.close()
        b4.close()
    assert (s4 == L.OK).all() and (s2 == L.OK).all()
    assert (np.abs(F2).sum(axis=1) > 0).all()
    assert np.array_equal(F2, F4)


def test_batch_four_steps_rejects_too_many_ctas():
    with pytest.raises(L.LbmEmError) as e:
        L.Batch(_batch_instances()[:1], "f32", steps_per_launch=4, ctas_per_sm=8)
    assert e.value.status == L.EINVAL


def _reuse_instances():
    out = []
    for k, (nx, ny) in enumerate(_random_shapes(5, 12, 48, 130)):
        a = min(nx, ny) / 6.0
        out.append(dict(nx=nx, ny=ny, a=a, phi0=0.5 * k, eps1=2.5, eps2=4.0, pec2=k % 2 == 0, period=20,
                        periods=10, R=min(nx, ny) / 3.0, ramp=20))
    return out


def test_batches_on_reused_memory_give_the_same_bits():
    """Batches created, run and freed in turn, some while another batch is alive, are placed on
    memory that freed batches left holding their final state, error words, accumulators and
    tensor-map tables.  Every run, the first one of a batch whose tuning had a single candidate
    included, starts from the cleared state with its own maps: all give the forces of the first
    batch, and no copy times out."""
    insts = _reuse_instances()

    def two():
        return L.Batch(insts, "f32", tile_w=64, tile_h=8, ctas_per_sm=3, steps_per_launch=2)

    def four():
        return L.Batch(insts, "f32", steps_per_launch=4)

    def one():
        return L.Batch(insts, "f32", tile_w=64, tile_h=4, ctas_per_sm=4)

    def run(make):
        b = make()
        try:
            b.run()
            return b.results()
        finally:
            b.close()

    F_ref, s_ref = run(two)
    assert (s_ref == L.OK).all() and (np.abs(F_ref).sum(axis=1) > 0).all()
    for pre in (None, two, four, one, None):
        held = pre() if pre else None
        try:
            for make in (two, four, one, two):
                F, st = run(make)
                assert (st == L.OK).all()
                assert np.array_equal(F, F_ref)
        finally:
            if held is not None:
                held.close()

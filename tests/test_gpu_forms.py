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


@pytest.mark.parametrize("prec", ["f64", "f32"])
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
    assert w % 32 == 0 and h >= 1 and c >= 1
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


def test_batch_reports_unstable_instance():
    insts = _batch_instances()[:2]
    b = L.Batch(insts, "f32")
    b._L.lbm_em_batch_destroy(b.b)
    b.b = None
    # a runaway instance is flagged on its own
    import ctypes
    arr = (L.Instance * 2)()
    for i, inst in enumerate(insts):
        arr[i] = L.Instance(inst["nx"], inst["ny"], inst["period"], inst["periods"], inst["ramp"], 0,
                            1e9 if i == 1 else 1.0, inst["R"],
                            L.make_janus(inst["a"], inst["phi0"], inst["eps1"], inst["eps2"], inst["pec2"]))
    o = L.BatchOpts(L.F32, 64, 4, 2, 0, None)
    h = ctypes.c_void_p()
    L._call("lbm_em_batch_create", arr, 2, ctypes.byref(o), ctypes.byref(h))
    L._call("lbm_em_batch_run", h)
    out = np.zeros(6)
    st = np.zeros(2, dtype=np.int32)
    rc = L.load().lbm_em_batch_results(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       st.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    assert rc == L.EUNSTABLE and st[0] == L.OK and st[1] == L.EUNSTABLE
    L.load().lbm_em_batch_destroy(h)


@pytest.mark.parametrize("inst", W.small_cases()[:3], ids=lambda i: f"{i['nx']}x{i['ny']}")
def test_two_steps_per_launch_is_bit_identical_in_fp32(inst):
    """FP32 with two steps per launch (temporal blocking) equals one step per launch bit
    for bit, for even and odd step counts and through the accumulating period."""
    with L.solver_for_instance(inst, "f32") as a, L.solver_for_instance(inst, "f32", single_step=True) as b:
        for n in (1, 2, 5, 32, 33, 64, 3):
            a.step(n)
            b.step(n)
            for x, y in zip(a.fields(), b.fields()):
                assert np.array_equal(x, y)
        c = L.make_contour(inst["R"], inst["a"])
        assert np.array_equal(a.force_torque(c), b.force_torque(c))


def test_f16dev_split_runs_agree_bitwise():
    """The FP16-deviation form gives the same bits however a run is split into calls."""
    inst = W.small_cases()[2]
    with L.solver_for_instance(inst, "f16dev") as a, L.solver_for_instance(inst, "f16dev") as b:
        a.step(77)
        for n in (3, 30, 1, 43):
            b.step(n)
        for x, y in zip(a.fields(), b.fields()):
            assert np.array_equal(x, y)


def test_f16dev_single_step_mode_within_tolerance():
    inst = W.homogeneous_dielectric_256()[0]
    F64 = L.run_instance(inst, "f64")
    F16 = L.run_instance(inst, "f16dev", single_step=True)
    assert np.max(np.abs(F16 - F64)) < 1e-3 * abs(F64[0])

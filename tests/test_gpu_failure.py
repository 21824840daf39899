"""Failure detection on the GPU without a fault: the bounded device-side wait that the
TMA-staged kernels use for their tile copies gives up on a barrier that nothing arrives on,
the library reports LBM_EM_ETIMEOUT, and the device stays usable afterwards."""
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


def test_bounded_wait_gives_up_and_reports_timeout():
    lib = L.load()
    rc = lib.lbm_em_probe_bounded_wait(20_000_000)  # about 10 ms of clock cycles
    assert rc == L.ETIMEOUT, (rc, L.last_error())
    assert "gave up" in L.last_error()
    # the device is still usable: the TMA-staged two-step kernel gives one-step bits
    inst = W.small_cases()[1]
    with L.solver_for_instance(inst, "f32", steps_per_launch="two") as a, \
            L.solver_for_instance(inst, "f32", steps_per_launch="one") as b:
        a.step(40)
        b.step(40)
        a.sync()
        for x, y in zip(a.fields(), b.fields()):
            assert np.array_equal(x, y)


@pytest.fixture
def quiet_gc():
    """Handles of earlier tests that wait for the garbage collector would change the held
    count in the middle of a test: collect them first and pause the collector."""
    import gc
    gc.collect()
    gc.disable()
    yield
    gc.enable()


def _make_janus_solver(inst):
    return L.solver_for_instance(inst, "f32")


def _make_map_solver(inst):
    from oracle import geometry as G
    eps, pec, _ = G.janus_material(inst["nx"], inst["ny"], inst["a"], inst["phi0"], inst["eps1"],
                                   inst["eps2"], inst["pec2"])
    return L.Solver(inst["nx"], inst["ny"], "f32", eps_map=eps, pec_mask=pec,
                    source=L.make_source(inst["period"], inst["ramp"]))


def _fail_each_allocation(make, live0):
    """Arms the hook at k = 1, 2, ... until make() succeeds; every earlier attempt must fail
    with ENOMEM and leave the library holding what it held before.  Returns (object, failures)."""
    k = 0
    while True:
        k += 1
        assert k < 200
        L.alloc_fault_hook(k)
        try:
            obj = make()
        except L.LbmEmError as e:
            assert e.status == L.ENOMEM, (k, str(e))
            assert L.alloc_fault_hook(0) == live0, k
            continue
        L.alloc_fault_hook(0)
        return obj, k - 1


@pytest.mark.parametrize("make", [_make_janus_solver, _make_map_solver], ids=["janus", "maps"])
def test_allocation_failures_in_create_release_everything(make, quiet_gc):
    """Host-side injection (nothing faults on the device): failing each device or pinned
    allocation of a create in turn returns ENOMEM and releases what the call had allocated;
    the handle that finally gets everything runs and equals an uninjected one, and so do
    the later calls that allocate (contour, fields) after their own injected failures."""
    inst = W.small_cases()[1]
    live0 = L.alloc_fault_hook(0)
    s, failures = _fail_each_allocation(lambda: make(inst), live0)
    assert failures >= 8, failures
    live1 = L.alloc_fault_hook(0)
    c = L.make_contour(inst["R"], inst["a"])
    _, cfail = _fail_each_allocation(lambda: s.set_contour(c), live1)
    assert cfail >= 3, cfail
    L.alloc_fault_hook(1)
    with pytest.raises(L.LbmEmError) as e:
        s.fields()
    assert e.value.status == L.ENOMEM
    L.alloc_fault_hook(0)
    s.step((inst["periods"] - 1) * inst["period"])
    F = s.force_torque(c)
    ref = L.run_instance(inst, "f32")
    assert np.array_equal(F, ref)
    assert all(np.isfinite(x).all() for x in s.fields())
    s.close()
    assert L.alloc_fault_hook(0) == live0


@pytest.mark.parametrize("prec,shape", [("f32", (64, 8, 3)), ("f64", (64, 4, 2))], ids=["f32-two-step", "f64"])
def test_allocation_failures_in_batch_create_release_everything(prec, shape, quiet_gc):
    insts = W.small_cases()
    live0 = L.alloc_fault_hook(0)
    b, failures = _fail_each_allocation(lambda: L.Batch(insts, prec, *shape), live0)
    assert failures >= 15, failures
    b.run()
    F, st = b.results()
    b.close()
    assert L.alloc_fault_hook(0) == live0
    ref = L.Batch(insts, prec, *shape)
    ref.run()
    Fr, _ = ref.results()
    ref.close()
    assert (st == L.OK).all() and np.array_equal(F, Fr)

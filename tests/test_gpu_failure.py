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

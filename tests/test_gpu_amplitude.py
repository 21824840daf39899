"""Amplitude invariance of every form (the scheme of Sec. III is linear in the fields, and the
forces of Sec. II.B are normalised by F0 = pi a E0^2 / 4, M0 = 2 F0 a).

The FP16-deviation scale is 2^(10 - k) and the runaway threshold |E| >= 3 * 2^(20 + k), with
2^k <= |E0| < 2^(k + 1), so neither depends on the absolute amplitude:
  - F~, M~ of FP64 do not depend on E0 (to 1e-9 relative: only rounding differs), and the
    FP32 and FP16-deviation forms meet their spec tolerances against FP64 at
    E0 = 1e-3, 1 and 1e3;
  - a field planted at 2^21 times the amplitude in a checkpoint trips the runaway test, one
    planted at 2^17 times it does not, whatever E0 is."""
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


AMPS = [1e-3, 1.0, 1e3]


@pytest.fixture(scope="module")
def forces():
    inst = W.homogeneous_dielectric_256()[0]
    md = W.md_janus_512()[2]
    out = {}
    for name, base in (("homogeneous_256", inst), ("md_janus_512", md)):
        for E0 in AMPS:
            for prec in ("f64", "f32", "f16dev"):
                out[name, E0, prec] = L.run_instance(dict(base, E0=E0), prec)
    return out


@pytest.mark.parametrize("name", ["homogeneous_256", "md_janus_512"])
def test_fp64_forces_do_not_depend_on_amplitude(forces, name):
    ref = forces[name, 1.0, "f64"]
    for E0 in AMPS:
        F = forces[name, E0, "f64"]
        assert np.max(np.abs(F - ref)) < 1e-9 * np.sum(np.abs(ref)), (E0, F, ref)


@pytest.mark.parametrize("E0", AMPS)
@pytest.mark.parametrize("name", ["homogeneous_256", "md_janus_512"])
def test_reduced_precision_forms_meet_tolerances_at_any_amplitude(forces, name, E0):
    F64 = forces[name, E0, "f64"]
    scale = abs(F64[0])
    F32 = forces[name, E0, "f32"]
    assert abs(F32[0] - F64[0]) < 1e-4 * scale, (F32, F64)
    assert abs(F32[1] - F64[1]) < 1e-3 * scale and abs(F32[2] - F64[2]) < 1e-3 * scale
    F16 = forces[name, E0, "f16dev"]
    assert np.max(np.abs(F16 - F64)) < 1e-3 * scale, (F16, F64)
    # the reduced forms are as accurate at E0 = 1e-3 and 1e3 as at 1 (same relative rounding)
    for prec, F in (("f32", F32), ("f16dev", F16)):
        e = np.max(np.abs(F - F64)) / scale
        e1 = np.max(np.abs(forces[name, 1.0, prec] - forces[name, 1.0, "f64"])) / abs(forces[name, 1.0, "f64"][0])
        assert e < 4.0 * e1 + 1e-9, (prec, E0, e, e1)


@pytest.mark.parametrize("E0", [1e-6, 1e-3, 1e3])
def test_f16dev_four_steps_meet_tolerances_at_any_amplitude(forces, E0):
    """The four-step FP16-deviation kernel takes the scale 2^(10 - k) of E0 like the other
    kernels of the form: on the 512^2 metallo-dielectric instance its forces at E0 = 1e-6 (below
    2^-14: the converting rebuild), 1e-3 and 1e3 (the mixed-precision one) are within the form's
    bound of FP64 and as accurate as at E0 = 1."""
    md = W.md_janus_512()[2]
    e = {}
    for amp in (1.0, E0):
        F64 = forces.get(("md_janus_512", amp, "f64"))
        if F64 is None:
            F64 = L.run_instance(dict(md, E0=amp), "f64")
        F4 = L.run_instance(dict(md, E0=amp), "f16dev", steps_per_launch="four")
        e[amp] = np.max(np.abs(F4 - F64)) / abs(F64[0])
    assert e[E0] < 1e-3, e
    assert e[E0] < 4.0 * e[1.0] + 1e-9, e


@pytest.mark.parametrize("m", [-24, -20, -15, -14, -10, -1, 0, 15])
def test_mixed_precision_fp16_rebuild_is_the_converting_one(m):
    """The four-step FP16-deviation kernel rebuilds each stored deviation with the mixed-precision
    FMA (FP16 deviation times -2^m plus an FP32 equilibrium, one rounding) wherever -2^m is an
    FP16 number, |E0| >= 2^-14; the other kernels of the form convert the deviation to FP32 and
    use the FP32 FMA.  Both must give the same bits for every FP16 value (normal, subnormal,
    zero, infinite, NaN) against equilibria from subnormal to large, at every inverse scale the
    kernel takes this path for."""
    rng = np.random.default_rng(100 + m)
    lo = np.tile(np.arange(65536, dtype=np.uint32), 8)
    hi = rng.integers(0, 65536, lo.size, dtype=np.uint32)
    g2 = lo | (hi << 16)
    mag = 10.0 ** rng.uniform(-45.0, 10.0, lo.size)
    eq2 = (np.where(rng.random(lo.size) < 0.5, -mag, mag) * (rng.random(lo.size) > 0.01)).astype(np.float32)
    assert L.probe_f16_rebuild(g2, eq2, m) == 0


HEADER = 40  # bytes of the checkpoint header (magic, precision, nx, ny, slots, t, n_acc)


def _plant(blob, prec, nx, ny, x, y, value):
    """Checkpoint with the stored value that sets E at site (x, y) replaced: the z-pair
    population (FP64, FP32) or the stored field E_z/3 (FP16-deviation)."""
    b = bytearray(blob)
    pitch = (nx + 31) // 32 * 32
    site = y * pitch + x
    if prec == "f64":
        np.frombuffer(b, dtype=np.float64, count=1, offset=HEADER + 8 * site)[...] = value
    elif prec == "f32":
        np.frombuffer(b, dtype=np.float32, count=1, offset=HEADER + 4 * site)[...] = value
    else:
        pstride = pitch * ny
        half = (11 * pstride * 2 + 255) // 256 * 256
        np.frombuffer(b, dtype=np.float32, count=1, offset=HEADER + half + 4 * site)[...] = value
    return bytes(b)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16dev"])
@pytest.mark.parametrize("E0", AMPS)
def test_runaway_threshold_is_relative_to_the_amplitude(prec, E0):
    nx, ny = 48, 40
    j = L.make_janus(6, 0.3, 2.0)
    src = L.make_source(24, E0=E0)
    with L.Solver(nx, ny, prec, janus=j, source=src, steps_per_launch="one") as s:
        s.step(30)
        s.sync()
        blob = s.save_state()
    # E/3 at the planted vacuum site: 2 v / 3 for a z-pair population v, v / 3 for a stored E/3
    per = 1.0 / 3.0 if prec == "f16dev" else 2.0 / 3.0
    k = int(np.floor(np.log2(E0)))
    for factor, expect in ((2.0 ** 21, L.EUNSTABLE), (2.0 ** 17, L.OK)):
        v = factor * 2.0 ** k / per
        with L.Solver(nx, ny, prec, janus=j, source=src, steps_per_launch="one") as s:
            s.load_state(_plant(blob, prec, nx, ny, 5, 5, v))
            s.step(1)
            if expect == L.OK:
                s.sync()
            else:
                with pytest.raises(L.LbmEmError) as e:
                    s.sync()
                assert e.value.status == expect

"""The C-ABI library builds for sm_103a, loads, and exports every symbol the header
declares; without a GPU it refuses to run (there is no CPU fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm_em.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_em_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_22308_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbm_em_create", "lbm_em_step", "lbm_em_force_torque", "lbm_em_batch_create",
                     "lbm_em_batch_run", "lbm_em_batch_results", "lbm_em_destroy", "lbm_em_last_error"):
        assert required in names


def test_every_declaration_is_documented():
    """Each function of the header comes right after its own comment block (arguments,
    layout, ownership, errors)."""
    lines = open(HEADER).read().split("\n")
    decl = re.compile(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(lbm_em_[a-z_0-9]+)\s*\(")
    seen = 0
    for i, line in enumerate(lines):
        m = decl.match(line)
        if not m:
            continue
        seen += 1
        j = i - 1
        while j >= 0 and not lines[j].strip():
            j -= 1
        assert lines[j].rstrip().endswith("*/"), f"{m.group(1)} has no comment block of its own"
    assert seen == len(declared_functions())


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"missing export {name}"


def test_binding_covers_every_declared_symbol():
    from paper_2509_22308_gb300 import lbm_em
    names = set(declared_functions()) - {"lbm_em_last_error"}
    assert names == set(lbm_em.SIGNATURES)


def test_no_cpu_fallback_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2509_22308_gb300 import lbm_em
    with pytest.raises(lbm_em.LbmEmError) as e:
        lbm_em.Solver(32, 32, "f64", janus=lbm_em.make_janus(5, 0.3, 2.0), source=lbm_em.make_source(24))
    assert e.value.status == lbm_em.ECUDA


def test_argument_validation_needs_no_gpu(lib):
    from paper_2509_22308_gb300 import lbm_em
    with pytest.raises(lbm_em.LbmEmError) as e:
        lbm_em.Solver(32, 32, "f64", janus=lbm_em.make_janus(-1, 0.3, 2.0), source=lbm_em.make_source(24))
    assert e.value.status == lbm_em.EINVAL
    with pytest.raises(lbm_em.LbmEmError) as e:
        lbm_em.Solver(32, 32, "f64", janus=lbm_em.make_janus(5, 0.3, 0.5), source=lbm_em.make_source(24))
    assert e.value.status == lbm_em.EINVAL
    with pytest.raises(lbm_em.LbmEmError) as e:
        lbm_em.Solver(32, 32, "f64", janus=lbm_em.make_janus(5, 0.3, 2.0), source=lbm_em.make_source(2))
    assert e.value.status == lbm_em.EINVAL
    with pytest.raises(lbm_em.LbmEmError) as e:     # TE^z has no FP16-deviation form
        lbm_em.Solver(32, 32, "f16dev", janus=lbm_em.make_janus(5, 0.3, 2.0), source=lbm_em.make_source(24),
                      polarization="te")
    assert e.value.status == lbm_em.EINVAL


def test_bounded_wait_probe_rejects_limits_out_of_range(lib):
    """The limit is checked before any device work (so this runs without a GPU too)."""
    fn = lib.lbm_em_probe_bounded_wait
    fn.argtypes = [ctypes.c_int64]
    fn.restype = ctypes.c_int
    assert fn(0) == 1 and fn(-5) == 1 and fn(3_000_000_000) == 1  # LBM_EM_EINVAL


def test_batch_rejects_the_40_wide_tile_outside_the_two_step_kernel(lib):
    """40 x 12 tiles exist only in the FP32 two-step batch kernel (the one-step kernel needs a
    power-of-two tile width); the options are checked before any device work."""
    from paper_2509_22308_gb300 import lbm_em as L
    inst = dict(nx=200, ny=200, a=50.0, phi0=0.3, eps1=2.0, eps2=4.0, pec2=False, period=150, periods=2,
                R=75.0, ramp=150)
    for prec, kw in (("f64", {}), ("f32", {"conv_tol": 1e-6}), ("f32", {"tile_h": 8})):
        with pytest.raises(L.LbmEmError) as e:
            L.Batch([inst], prec, tile_w=40, **kw)
        assert e.value.status == L.EINVAL


def test_batch_rejects_an_unknown_polarization(lib):
    import ctypes as C
    from paper_2509_22308_gb300 import lbm_em as L
    arr = (L.Instance * 1)()
    arr[0] = L.Instance(64, 64, 48, 2, 48, 0, 1.0, 20.0, L.make_janus(10.0, 0.3, 2.0, 4.0, False))
    o = L.BatchOpts(L.F32, 0, 0, 0, 0, 0, 0.0, None, 2)
    h = C.c_void_p()
    assert L.load().lbm_em_batch_create(arr, 1, C.byref(o), C.byref(h)) == L.EINVAL


def test_three_step_flag_is_fp32_only(lib):
    """LBM_EM_FLAG_THREE_STEP (8) is accepted for FP32 alone, LBM_EM_FLAG_FOUR_STEP (16) for
    FP32 and FP16-deviation; each excludes the other step flags; unknown flags are rejected.
    The checks come before any device work."""
    from paper_2509_22308_gb300 import lbm_em
    P = lbm_em.PRECISIONS
    for prec, flags in (("f64", 8), ("f16dev", 8), ("f32x2", 8), ("f32", 8 | 1), ("f32", 8 | 2), ("f32", 32),
                        ("f64", 16), ("f32x2", 16), ("f32", 16 | 2), ("f32", 16 | 8), ("f16dev", 16 | 1)):
        g = lbm_em.Grid(16, 16, P[prec], flags, None)
        h = ctypes.c_void_p()
        rc = lib.lbm_em_create_janus(ctypes.byref(g), ctypes.byref(lbm_em.make_janus(5, 0.3, 2.0)),
                                     ctypes.byref(lbm_em.make_source(24)), ctypes.byref(h))
        assert rc == lbm_em.EINVAL, (prec, flags, rc)


def test_batch_steps_per_launch_is_validated_before_device_work(lib):
    """lbm_em_batch_opts.steps_per_launch: 0, 1, 2 or 4; 2 and 4 need FP32 without convergence
    exits, 4 takes no tile shape."""
    from paper_2509_22308_gb300 import lbm_em as L
    arr = (L.Instance * 1)()
    arr[0] = L.Instance(64, 64, 48, 2, 48, 0, 1.0, 20.0, L.make_janus(10.0, 0.3, 2.0, 4.0, False))
    for prec, spl, conv, tw in ((L.F32, 3, 0.0, 0), (L.F64, 4, 0.0, 0), (L.F32X2, 2, 0.0, 0), (L.F32, 4, 1e-3, 0),
                                (L.F32, 4, 0.0, 64)):
        o = L.BatchOpts(prec, tw, 0, 0, 0, 0, conv, None, 0, spl)
        h = ctypes.c_void_p()
        assert lib.lbm_em_batch_create(arr, 1, ctypes.byref(o), ctypes.byref(h)) == L.EINVAL, (prec, spl, conv, tw)

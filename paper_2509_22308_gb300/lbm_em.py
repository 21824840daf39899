"""Thin ctypes binding of the C ABI in ``include/lbm_em.h`` (argument marshalling only).

Every step of the solver runs in the CUDA library ``_build/liblbm_em.so``; this
module never computes a lattice quantity itself.  Loading fails loudly when the
library is missing (build it with ``paper_2509_22308_gb300.build.build()``)."""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbm_em.so")

OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ETIMEOUT, ESTATE = range(7)
F64, F32, F16DEV, F32X2 = 0, 1, 2, 3
FLAG_SINGLE_STEP, FLAG_TWO_STEP, FLAG_THREE_STEP, FLAG_FOUR_STEP = 1, 2, 8, 16
STEP_MODES = {"auto": 0, "one": FLAG_SINGLE_STEP, "two": FLAG_TWO_STEP, "three": FLAG_THREE_STEP,
              "four": FLAG_FOUR_STEP}
FLAG_TE = 4
POLARIZATION_FLAGS = {"tm": 0, "te": FLAG_TE}
SRC_HARD, SRC_OPEN, SRC_NONE = 0, 1, 2
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EUNSTABLE", 5: "ETIMEOUT", 6: "ESTATE"}
PRECISIONS = {"f64": F64, "f32": F32, "f16dev": F16DEV, "f32x2": F32X2}


class LbmEmError(RuntimeError):
    def __init__(self, status, fn, msg):
        super().__init__(f"{fn}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("stream", ctypes.c_void_p)]


class Source(ctypes.Structure):
    _fields_ = [("period_steps", ctypes.c_int32), ("ramp_steps", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("E0", ctypes.c_double)]


class Janus(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("phi0", ctypes.c_double), ("eps1", ctypes.c_double),
                ("eps2", ctypes.c_double), ("pec2", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double)]


class Contour(ctypes.Structure):
    _fields_ = [("cx", ctypes.c_double), ("cy", ctypes.c_double), ("radius", ctypes.c_double),
                ("n_points", ctypes.c_int32), ("reserved", ctypes.c_int32), ("a", ctypes.c_double)]


class Instance(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("period_steps", ctypes.c_int32),
                ("periods", ctypes.c_int32), ("ramp_steps", ctypes.c_int32), ("n_points", ctypes.c_int32),
                ("E0", ctypes.c_double), ("contour_radius", ctypes.c_double), ("janus", Janus)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("min_periods", ctypes.c_int32), ("source_kind", ctypes.c_int32),
                ("conv_tol", ctypes.c_double), ("stream", ctypes.c_void_p), ("polarization", ctypes.c_int32),
                ("steps_per_launch", ctypes.c_int32)]


_P = ctypes.POINTER
_vp = ctypes.c_void_p
# name -> (argtypes); every function returns lbm_em_status except lbm_em_last_error
SIGNATURES = {
    "lbm_em_create": [_P(Grid), _P(ctypes.c_double), _P(ctypes.c_uint8), _P(Source), _P(_vp)],
    "lbm_em_create_janus": [_P(Grid), _P(Janus), _P(Source), _P(_vp)],
    "lbm_em_destroy": [_vp],
    "lbm_em_reset": [_vp],
    "lbm_em_set_janus": [_vp, _P(Janus)],
    "lbm_em_step": [_vp, ctypes.c_int64],
    "lbm_em_sync": [_vp],
    "lbm_em_get_time": [_vp, _P(ctypes.c_int64)],
    "lbm_em_get_steps_per_launch": [_vp, _P(ctypes.c_int32)],
    "lbm_em_set_contour": [_vp, _P(Contour)],
    "lbm_em_accumulate": [_vp, ctypes.c_int64],
    "lbm_em_contour_integral": [_vp, _P(ctypes.c_double)],
    "lbm_em_force_torque": [_vp, _P(Contour), _P(ctypes.c_double)],
    "lbm_em_contour_integral_device": [_vp, _vp],
    "lbm_em_force_torque_device": [_vp, _P(Contour), _vp],
    "lbm_em_energy": [_vp, _P(ctypes.c_double)],
    "lbm_em_run_converged": [_vp, _P(Contour), ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                             _P(ctypes.c_double), _P(ctypes.c_int64)],
    "lbm_em_far_field": [_vp, _P(ctypes.c_double), ctypes.c_int32, _P(ctypes.c_double)],
    "lbm_em_get_fields": [_vp, _P(ctypes.c_double), _P(ctypes.c_double), _P(ctypes.c_double)],
    "lbm_em_get_phasors": [_vp, _P(ctypes.c_int32), _P(ctypes.c_double), _P(ctypes.c_int32)],
    "lbm_em_get_material": [_vp, _P(ctypes.c_uint8), _P(ctypes.c_double)],
    "lbm_em_save_state": [_vp, _vp, _P(ctypes.c_size_t)],
    "lbm_em_load_state": [_vp, _vp, ctypes.c_size_t],
    "lbm_em_rasterize_janus": [_P(Janus), ctypes.c_int32, ctypes.c_int32, _P(ctypes.c_uint8)],
    "lbm_em_rasterize_janus_noalloc": [_P(Janus), ctypes.c_int32, ctypes.c_int32, _P(ctypes.c_uint8)],
    "lbm_em_probe_bounded_wait": [ctypes.c_int64],
    "lbm_em_test_alloc_hook": [ctypes.c_int64, _P(ctypes.c_int64)],
    "lbm_em_probe_fp64_fma": [_vp, ctypes.c_int64, _P(ctypes.c_double)],
    "lbm_em_probe_f16_rebuild": [_P(ctypes.c_uint32), _P(ctypes.c_float), ctypes.c_int64, ctypes.c_int32,
                                 _P(ctypes.c_int64)],
    "lbm_em_transfer_bytes": [_P(ctypes.c_uint64), _P(ctypes.c_uint64)],
    "lbm_em_batch_create": [_P(Instance), ctypes.c_int32, _P(BatchOpts), _P(_vp)],
    "lbm_em_batch_run": [_vp],
    "lbm_em_batch_results": [_vp, _P(ctypes.c_double), _P(ctypes.c_int32)],
    "lbm_em_batch_steps": [_vp, _P(ctypes.c_int64)],
    "lbm_em_batch_config": [_vp, _P(ctypes.c_int32), _P(ctypes.c_int32), _P(ctypes.c_int32)],
    "lbm_em_batch_steps_per_launch": [_vp, _P(ctypes.c_int32)],
    "lbm_em_batch_destroy": [_vp],
}

_lib = None


def load():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} is missing "
                              "(run paper_2509_22308_gb300.build.build()); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.lbm_em_last_error.argtypes = []
        L.lbm_em_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def last_error() -> str:
    return load().lbm_em_last_error().decode()


def _call(name, *args):
    st = getattr(load(), name)(*args)
    if st != OK:
        raise LbmEmError(st, name, last_error())
    return st


def _dptr(a):
    return None if a is None else a.ctypes.data_as(_P(ctypes.c_double))


def _u8ptr(a):
    return None if a is None else a.ctypes.data_as(_P(ctypes.c_uint8))


def make_janus(a, phi0, eps1, eps2=1.0, pec2=False, cx=None, cy=None) -> Janus:
    return Janus(float(a), float(phi0), float(eps1), float(eps2), int(bool(pec2)), 0,
                 math.nan if cx is None else float(cx), math.nan if cy is None else float(cy))


def make_source(period, ramp=None, kind=SRC_HARD, E0=1.0) -> Source:
    return Source(int(period), int(period if ramp is None else ramp), int(kind), 0, float(E0))


def make_contour(radius, a, n_points=0, cx=None, cy=None) -> Contour:
    return Contour(math.nan if cx is None else float(cx), math.nan if cy is None else float(cy),
                   float(radius), int(n_points), 0, float(a))


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):  # torch.cuda.Stream
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Solver:
    """Owner of one ``lbm_em_t`` handle; methods map one-to-one onto the C calls.

    ``steps_per_launch``: "auto" (the library's default for the form and lattice size), "one",
    "two" (FP32, FP16-deviation, double-float) or "three" (FP32); the modes give the same bits."""

    def __init__(self, nx, ny, precision="f64", *, janus: Janus | None = None, eps_map=None, pec_mask=None,
                 source: Source, stream=None, steps_per_launch="auto", polarization="tm"):
        L = load()
        self.nx, self.ny = int(nx), int(ny)
        self.source = source
        self.polarization = polarization
        g = Grid(self.nx, self.ny, PRECISIONS.get(precision, precision),
                 STEP_MODES[steps_per_launch] | POLARIZATION_FLAGS[polarization],
                 _stream_ptr(stream))
        h = ctypes.c_void_p()
        if janus is not None:
            _call("lbm_em_create_janus", ctypes.byref(g), ctypes.byref(janus), ctypes.byref(source), ctypes.byref(h))
        else:
            eps = np.ascontiguousarray(eps_map, dtype=np.float64)
            assert eps.shape == (self.ny, self.nx)
            pec = None if pec_mask is None else np.ascontiguousarray(pec_mask, dtype=np.uint8)
            _call("lbm_em_create", ctypes.byref(g), _dptr(eps), _u8ptr(pec), ctypes.byref(source), ctypes.byref(h))
        self.h = h
        self._L = L

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self._L.lbm_em_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def reset(self):
        _call("lbm_em_reset", self.h)

    def set_janus(self, j: Janus):
        _call("lbm_em_set_janus", self.h, ctypes.byref(j))

    def step(self, n):
        _call("lbm_em_step", self.h, ctypes.c_int64(int(n)))

    def sync(self):
        _call("lbm_em_sync", self.h)

    @property
    def t(self) -> int:
        v = ctypes.c_int64()
        _call("lbm_em_get_time", self.h, ctypes.byref(v))
        return v.value

    def steps_per_launch(self) -> int:
        v = ctypes.c_int32()
        _call("lbm_em_get_steps_per_launch", self.h, ctypes.byref(v))
        return v.value

    def set_contour(self, c: Contour):
        _call("lbm_em_set_contour", self.h, ctypes.byref(c))

    def accumulate(self, n):
        _call("lbm_em_accumulate", self.h, ctypes.c_int64(int(n)))

    def contour_integral(self):
        out = np.zeros(3)
        _call("lbm_em_contour_integral", self.h, _dptr(out))
        return out

    def force_torque(self, c: Contour):
        out = np.zeros(3)
        _call("lbm_em_force_torque", self.h, ctypes.byref(c), _dptr(out))
        return out

    def force_torque_device(self, c: Contour, d_out_ptr: int):
        """Asynchronous force/torque into a device buffer of 3 doubles (e.g. a torch tensor's data_ptr)."""
        _call("lbm_em_force_torque_device", self.h, ctypes.byref(c), ctypes.c_void_p(int(d_out_ptr)))

    def energy(self) -> float:
        v = ctypes.c_double()
        _call("lbm_em_energy", self.h, ctypes.byref(v))
        return v.value

    def run_converged(self, c: Contour, tol=1e-3, min_periods=5, max_periods=100):
        """Periods until the per-period energy settles, then force/torque -> (F, steps run)."""
        out = np.zeros(3)
        n = ctypes.c_int64()
        _call("lbm_em_run_converged", self.h, ctypes.byref(c), float(tol), int(min_periods), int(max_periods),
              _dptr(out), ctypes.byref(n))
        return out, n.value

    def far_field(self, angles):
        """|S(phi)|^2 at the given lattice-frame angles from the accumulated phasors."""
        ang = np.ascontiguousarray(angles, dtype=np.float64)
        out = np.zeros(len(ang))
        _call("lbm_em_far_field", self.h, _dptr(ang), len(ang), _dptr(out))
        return out

    def fields(self):
        ez = np.empty((self.ny, self.nx))
        hx = np.empty_like(ez)
        hy = np.empty_like(ez)
        _call("lbm_em_get_fields", self.h, _dptr(ez), _dptr(hx), _dptr(hy))
        return ez, hx, hy

    def phasors(self):
        n = ctypes.c_int32()
        _call("lbm_em_get_phasors", self.h, None, None, ctypes.byref(n))
        xy = np.zeros(2 * n.value, dtype=np.int32)
        ph = np.zeros(6 * n.value)
        _call("lbm_em_get_phasors", self.h, xy.ctypes.data_as(_P(ctypes.c_int32)), _dptr(ph), ctypes.byref(n))
        return xy.reshape(-1, 2), ph.reshape(-1, 6)

    def material(self):
        ids = np.zeros((self.ny, self.nx), dtype=np.uint8)
        tab = np.zeros(256)
        _call("lbm_em_get_material", self.h, _u8ptr(ids), _dptr(tab))
        return ids, tab

    def save_state(self) -> bytes:
        n = ctypes.c_size_t()
        _call("lbm_em_save_state", self.h, None, ctypes.byref(n))
        buf = ctypes.create_string_buffer(n.value)
        _call("lbm_em_save_state", self.h, ctypes.cast(buf, ctypes.c_void_p), ctypes.byref(n))
        return buf.raw[: n.value]

    def load_state(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        _call("lbm_em_load_state", self.h, ctypes.cast(buf, ctypes.c_void_p), ctypes.c_size_t(len(data)))


def probe_fp64_fma(stream, iters) -> float:
    """Enqueue one launch of the library's FP64 FMA-chain probe on ``stream`` (a torch stream
    or a raw cudaStream_t); returns the number of FMAs the launch performs."""
    n = ctypes.c_double()
    _call("lbm_em_probe_fp64_fma", _stream_ptr(stream), ctypes.c_int64(int(iters)), ctypes.byref(n))
    return n.value


def probe_f16_rebuild(g2, eq2, m) -> int:
    """Bit mismatches between the four-step kernel's mixed-precision FP16 rebuild and the
    converting one, over the pairs g2 (uint32) and values eq2 (float32) at inverse scale 2^m."""
    g = np.ascontiguousarray(g2, dtype=np.uint32)
    e = np.ascontiguousarray(eq2, dtype=np.float32)
    if g.shape != e.shape:
        raise ValueError("g2 and eq2 must have the same shape")
    out = ctypes.c_int64()
    _call("lbm_em_probe_f16_rebuild", g.ctypes.data_as(_P(ctypes.c_uint32)), e.ctypes.data_as(_P(ctypes.c_float)),
          ctypes.c_int64(g.size), ctypes.c_int32(int(m)), ctypes.byref(out))
    return out.value


def transfer_bytes():
    """(host -> device, device -> host) bytes the library has copied since it was loaded."""
    h, d = ctypes.c_uint64(), ctypes.c_uint64()
    _call("lbm_em_transfer_bytes", ctypes.byref(h), ctypes.byref(d))
    return h.value, d.value


def alloc_fault_hook(fail_at=0) -> int:
    """Arm (fail_at > 0: the fail_at-th device or pinned allocation from now on fails with
    ENOMEM) or disarm (0) the library's allocation fault injection; returns the number of
    allocations the library's handles and batches currently hold."""
    live = ctypes.c_int64()
    _call("lbm_em_test_alloc_hook", ctypes.c_int64(int(fail_at)), ctypes.byref(live))
    return live.value


def rasterize_janus(j: Janus, nx, ny):
    out = np.zeros((ny, nx), dtype=np.uint8)
    _call("lbm_em_rasterize_janus", ctypes.byref(j), int(nx), int(ny), _u8ptr(out))
    return out


def rasterize_janus_noalloc(j: Janus, nx, ny):
    """Like ``rasterize_janus`` without any device allocation (fixed 4 MiB device array)."""
    out = np.zeros((ny, nx), dtype=np.uint8)
    _call("lbm_em_rasterize_janus_noalloc", ctypes.byref(j), int(nx), int(ny), _u8ptr(out))
    return out


def solver_for_instance(inst: dict, precision="f64", stream=None, kind=SRC_HARD, steps_per_launch="auto",
                        polarization="tm") -> Solver:
    """Solver for one workload instance dictionary (see ``workloads``; an optional "E0" key
    sets the incident amplitude, 1 by default)."""
    j = make_janus(inst["a"], inst["phi0"], inst["eps1"], inst["eps2"], inst["pec2"])
    s = make_source(inst["period"], inst.get("ramp"), kind, E0=inst.get("E0", 1.0))
    return Solver(inst["nx"], inst["ny"], precision, janus=j, source=s, stream=stream,
                  steps_per_launch=steps_per_launch, polarization=polarization)


def run_instance(inst: dict, precision="f64", stream=None, steps_per_launch="auto", polarization="tm") -> np.ndarray:
    """Full hot path for one instance: (periods - 1) periods of steps, one accumulated
    period, contour integral -> (F~x, F~y, M~z)."""
    with solver_for_instance(inst, precision, stream, steps_per_launch=steps_per_launch,
                             polarization=polarization) as s:
        s.step((inst["periods"] - 1) * inst["period"])
        return s.force_torque(make_contour(inst["R"], inst["a"]))


class Batch:
    """Owner of one ``lbm_em_batch_t``."""

    def __init__(self, instances, precision="f32", tile_w=0, tile_h=0, ctas_per_sm=0, stream=None,
                 conv_tol=0.0, min_periods=0, kind=SRC_HARD, polarization="tm", steps_per_launch=0):
        L = load()
        n = len(instances)
        arr = (Instance * n)()
        for i, inst in enumerate(instances):
            arr[i] = Instance(int(inst["nx"]), int(inst["ny"]), int(inst["period"]), int(inst["periods"]),
                              int(inst.get("ramp", inst["period"])), int(inst.get("n_points", 0)),
                              float(inst.get("E0", 1.0)),
                              float(inst["R"]),
                              make_janus(inst["a"], inst["phi0"], inst["eps1"], inst["eps2"], inst["pec2"]))
        o = BatchOpts(PRECISIONS.get(precision, precision), int(tile_w), int(tile_h), int(ctas_per_sm),
                      int(min_periods), int(kind), float(conv_tol), _stream_ptr(stream),
                      {"tm": 0, "te": 1}[polarization], int(steps_per_launch))
        b = ctypes.c_void_p()
        _call("lbm_em_batch_create", arr, n, ctypes.byref(o), ctypes.byref(b))
        self.b, self.n, self._L = b, n, L

    def run(self):
        _call("lbm_em_batch_run", self.b)

    def results(self):
        out = np.zeros(3 * self.n)
        st = np.zeros(self.n, dtype=np.int32)
        _call("lbm_em_batch_results", self.b, _dptr(out), st.ctypes.data_as(_P(ctypes.c_int32)))
        return out.reshape(-1, 3), st

    def steps(self):
        out = np.zeros(self.n, dtype=np.int64)
        _call("lbm_em_batch_steps", self.b, out.ctypes.data_as(_P(ctypes.c_int64)))
        return out

    def steps_per_launch(self) -> int:
        v = ctypes.c_int32()
        _call("lbm_em_batch_steps_per_launch", self.b, ctypes.byref(v))
        return v.value

    def config(self):
        w, h, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _call("lbm_em_batch_config", self.b, ctypes.byref(w), ctypes.byref(h), ctypes.byref(c))
        return w.value, h.value, c.value

    def close(self):
        if getattr(self, "b", None) is not None and self.b.value:
            self._L.lbm_em_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

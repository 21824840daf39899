"""Oracle (test infrastructure only): Python driver of the FP64 C lattice Boltzmann oracle.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It never touches the CUDA library.

The C file ``lbm_oracle.c`` implements Sec. III of arXiv 2509.22308 (Eq. LBGK
equation, Eq. equilibrium distribution functions) on the full 42-double D3Q7
vector state; this module compiles it with gcc, allocates the state with numpy
and exposes a small ``Simulation`` object.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

SITE_DOUBLES = 42
SRC_OPEN, SRC_HARD, SRC_NONE = 0, 1, 2
POLARIZATIONS = {"tm": 0, "te": 1}


class OracleCfg(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("period", ctypes.c_int),
        ("E0", ctypes.c_double),
        ("ramp_steps", ctypes.c_int),
        ("source_kind", ctypes.c_int),
        ("nthreads", ctypes.c_int),
        ("polarization", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            up = ctypes.POINTER(ctypes.c_ubyte)
            L.oracle_advance.argtypes = [ctypes.POINTER(OracleCfg), dp, up, dp, dp,
                                         ctypes.c_long, ctypes.c_long, dp]
            L.oracle_advance.restype = ctypes.c_int
            L.oracle_fields.argtypes = [ctypes.POINTER(OracleCfg), dp, up, dp, dp, dp, dp]
            L.oracle_fields.restype = None
            L.oracle_equilibria.argtypes = [ctypes.c_double, ctypes.c_double, dp, dp, dp, dp]
            L.oracle_equilibria.restype = None
            L.oracle_site_doubles.restype = ctypes.c_int
            assert L.oracle_site_doubles() == SITE_DOUBLES
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _up(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)) if a is not None else None


def equilibria(eps_r: float, E, H):
    """e_i^eq, h_i^eq (7x3 each) of Eq. (equilibrium distribution functions)."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    H = np.ascontiguousarray(H, dtype=np.float64)
    eeq = np.zeros((7, 3))
    heq = np.zeros((7, 3))
    lib().oracle_equilibria(float(eps_r), 1.0, _dp(E), _dp(H), _dp(eeq), _dp(heq))
    return eeq, heq


class Simulation:
    """Full-vector FP64 D3Q7 Maxwell LBM on an nx x ny lattice (Sec. III).

    ``eps`` is the per-site relative permittivity [ny, nx]; ``pec`` a per-site
    0/1 mask of perfect-electric-conductor cells.  ``f`` holds the pre-collision
    populations at time ``t`` as [ny, nx, 14, 3] (e_0..e_6, h_0..h_6).
    ``polarization`` "tm" (E_z, H_x, H_y; the paper's case) or "te" (H_z, E_x, E_y):
    the field triple the source drives, ``fields`` returns and ``phasors`` accumulates.
    """

    def __init__(self, eps, pec=None, period=120, E0=1.0, ramp_steps=0,
                 source_kind=SRC_HARD, nthreads=None, polarization="tm"):
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        self.ny, self.nx = eps.shape
        self.eps = eps
        self.pec = None if pec is None else np.ascontiguousarray(pec, dtype=np.uint8)
        if nthreads is None:
            nthreads = int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1))
        self.polarization = polarization
        self.cfg = OracleCfg(self.nx, self.ny, int(period), float(E0), int(ramp_steps),
                             int(source_kind), int(nthreads), POLARIZATIONS[polarization])
        self.period = int(period)
        self.f = np.zeros((self.ny, self.nx, 14, 3))
        self._post = np.zeros_like(self.f)
        self.t = 0
        self.acc = None
        self.acc_steps = 0

    def advance(self, nsteps: int, accumulate: bool = False):
        if accumulate and self.acc is None:
            self.acc = np.zeros((self.ny, self.nx, 6))
        rc = lib().oracle_advance(ctypes.byref(self.cfg), _dp(self.eps), _up(self.pec),
                                  _dp(self.f), _dp(self._post), self.t, int(nsteps),
                                  _dp(self.acc) if accumulate else None)
        if rc != 0:
            raise RuntimeError("oracle_advance rejected its arguments")
        self.t += int(nsteps)
        if accumulate:
            self.acc_steps += int(nsteps)

    def reset_accumulators(self):
        self.acc = np.zeros((self.ny, self.nx, 6))
        self.acc_steps = 0

    def fields(self):
        """The field triple of every site at time t, each [ny, nx]: (E_z, H_x, H_y) for
        TM, (H_z, E_x, E_y) for TE."""
        ez = np.empty((self.ny, self.nx))
        hx = np.empty_like(ez)
        hy = np.empty_like(ez)
        lib().oracle_fields(ctypes.byref(self.cfg), _dp(self.eps), _up(self.pec), _dp(self.f),
                            _dp(ez), _dp(hx), _dp(hy))
        return ez, hx, hy

    def phasors(self):
        """Complex phasors X = (2/T) sum_t X(t) e^{i w t} over the accumulated
        steps (Sec. III: Fourier analysis over one period), each [ny, nx]."""
        if self.acc is None or self.acc_steps == 0:
            raise RuntimeError("no accumulated steps")
        s = 2.0 / float(self.acc_steps)
        a = self.acc
        return (s * (a[..., 0] + 1j * a[..., 1]), s * (a[..., 2] + 1j * a[..., 3]),
                s * (a[..., 4] + 1j * a[..., 5]))

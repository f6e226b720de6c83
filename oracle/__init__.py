"""FP64 CPU oracle for the explicit phase-field step (arXiv 2303.09671).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use this
package; the product path (``paper_2303_09671_gb300``) never imports it.

The arithmetic lives in ``pf_oracle.c`` (plain C, FP64, OpenMP over the
outermost loop).  This module compiles it with gcc and exposes numpy-facing
wrappers.  Field arrays are C-ordered ``[z][y][x]`` (x fastest) float64 arrays
of shape ``n[::-1]`` restricted to the active dimensions.

Parameters are passed as a plain dict with the keys of ``PARAM_KEYS``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pf_oracle.c")
_HDR = os.path.join(_HERE, "pf_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

BC = {"noflux": 0, "periodic": 1, "dirichlet": 2}

# planted mistakes (tests only), mirrors the PLANT_* bits of pf_oracle.c
PLANT = {
    "printed_drag": 1,
    "no_antitrap": 2,
    "no_cross": 4,
    "no_K": 8,
    "tang_sign": 16,
    "swap_w": 32,
    "mu_s_cryst": 64,
}

# planted mistakes of the front locator and the moving window (tests only); the
# rates do not see them, so they are pinned separately from PLANT
PLANT_WINDOW = {
    "front_index": 128,
    "front_half": 256,
    "fresh_cinf": 512,
    "shift_early": 1024,
}


class _Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int64 * 3),
        ("dx", ctypes.c_double),
        ("bc_lo", ctypes.c_int * 3),
        ("bc_hi", ctypes.c_int * 3),
        ("dir_phi", ctypes.c_double),
        ("dir_cs", ctypes.c_double),
        ("dir_cl", ctypes.c_double),
        ("interp", ctypes.c_int),
        ("lap", ctypes.c_int),
        ("mobility", ctypes.c_int),
        ("H", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("M_phi", ctypes.c_double),
        ("D_s", ctypes.c_double),
        ("D_l", ctypes.c_double),
        ("k_e", ctypes.c_double),
        ("A", ctypes.c_double),
        ("b", ctypes.c_double),
        ("a", ctypes.c_double),
        ("delta", ctypes.c_double),
        ("theta_ref", ctypes.c_double),
        ("G_theta", ctypes.c_double),
        ("v_pull", ctypes.c_double),
        ("x0", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("c_inf", ctypes.c_double),
        ("shift", ctypes.c_int),
        ("form", ctypes.c_int),
        ("plant", ctypes.c_int),
    ]


class _Clock(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("shifts", ctypes.c_int64)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, -O2, no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.POINTER(_Params)
            C = ctypes.POINTER(_Clock)
            dp = ctypes.POINTER(ctypes.c_double)
            L.orc_point.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, dp]
            L.orc_rates.argtypes = [P, C, dp, dp, dp, dp, dp, dp]
            L.orc_step.argtypes = [P, C, dp, dp, dp, ctypes.c_int64, dp]
            L.orc_energy.argtypes = [P, C, dp, dp, dp]
            L.orc_energy.restype = ctypes.c_double
            L.orc_solute.argtypes = [P, dp, dp, dp]
            L.orc_solute.restype = ctypes.c_double
            L.orc_front.argtypes = [P, C, dp, dp, dp, dp, dp]
            L.orc_mixture.argtypes = [P, dp, dp, dp, ctypes.c_int64, dp, dp]
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_threads.restype = ctypes.c_int
            L.orc_set_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> int:
    """Threads of the oracle's later sweeps; returns the count in use."""
    return int(lib().orc_set_threads(int(n)))


def _params(p: dict) -> _Params:
    s = _Params()
    s.dim = int(p["dim"])
    n = list(p["n"]) + [1] * (3 - len(p["n"]))
    for a in range(3):
        s.n[a] = int(n[a])
        s.bc_lo[a] = BC[p["bc_lo"][a]] if a < s.dim else 0
        s.bc_hi[a] = BC[p["bc_hi"][a]] if a < s.dim else 0
    s.dx = float(p["dx"])
    s.dir_phi, s.dir_cs, s.dir_cl = (float(v) for v in p.get("dirichlet", (0.0, 0.0, 1.0)))
    s.interp = {"quintic": 0, "cubic": 1}[p.get("interp", "quintic")]
    s.lap = int(p["lap"])
    s.mobility = {"Dc": 0, "const": 1}[p.get("mobility", "Dc")]
    for k in ("H", "sigma", "M_phi", "D_s", "D_l", "k_e", "A", "b", "a", "delta",
              "theta_ref", "G_theta", "v_pull", "x0", "dt", "c_inf"):
        setattr(s, k, float(p[k]))
    s.shift = int(bool(p.get("shift", False)))
    s.form = {"cd": 0, "literal": 1}[p.get("form", "cd")]
    plant = p.get("plant", 0)
    if isinstance(plant, str):
        plant = PLANT[plant] if plant in PLANT else PLANT_WINDOW[plant]
    s.plant = int(plant)
    return s


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(p: dict, *arrs):
    shape = tuple(int(v) for v in list(p["n"])[: p["dim"]][::-1])
    out = []
    for a in arrs:
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.shape != shape:
            raise ValueError(f"field shape {a.shape} != {shape}")
        out.append(a)
    return out


POINT_NAMES = ("p", "dp", "fdw", "dfdw", "mu_s", "mu_l", "f_s", "f_l", "M_s", "M_l",
               "Mbar", "drag", "dG", "q_n", "w_s", "w_l", "h_n", "a_phi", "Y")


def point(p: dict, phi: float, cs: float, cl: float, theta: float) -> dict:
    out = (ctypes.c_double * len(POINT_NAMES))()
    lib().orc_point(ctypes.byref(_params(p)), phi, cs, cl, theta, out)
    return dict(zip(POINT_NAMES, list(out)))


def mixture(p: dict, phi, cs, cl):
    """(p(phi), c = p c_s + (1 - p) c_l) per cell, for arrays of one shape."""
    phi, cs, cl = (np.ascontiguousarray(a, dtype=np.float64) for a in (phi, cs, cl))
    if not (phi.shape == cs.shape == cl.shape):
        raise ValueError("phi, c_s, c_l must have one shape")
    pv, cv = np.empty_like(phi), np.empty_like(phi)
    if lib().orc_mixture(ctypes.byref(_params(p)), _dptr(phi), _dptr(cs), _dptr(cl), phi.size,
                         _dptr(pv), _dptr(cv)) != 0:
        raise ValueError("oracle: invalid parameters")
    return pv, cv


class State:
    """Oracle state: FP64 fields plus the clock (step count, window shifts)."""

    def __init__(self, p: dict, phi, cs, cl, step: int = 0, shifts: int = 0):
        self.p = dict(p)
        self.phi, self.cs, self.cl = (a.copy() for a in _check(p, phi, cs, cl))
        self.clock = _Clock(step, shifts)

    @property
    def t(self) -> float:
        return self.clock.step * self.p["dt"]

    def step(self, n: int, energy: bool = False):
        hist = np.zeros(max(n, 1)) if energy else None
        rc = lib().orc_step(ctypes.byref(_params(self.p)), ctypes.byref(self.clock),
                            _dptr(self.phi), _dptr(self.cs), _dptr(self.cl), int(n),
                            _dptr(hist) if energy else None)
        if rc == -2:
            raise FloatingPointError("oracle: non-finite value")
        if rc != 0:
            raise ValueError("oracle: invalid parameters")
        return hist[:n] if energy else None

    def rates(self):
        z = [np.zeros_like(self.phi) for _ in range(3)]
        rc = lib().orc_rates(ctypes.byref(_params(self.p)), ctypes.byref(self.clock),
                             _dptr(self.phi), _dptr(self.cs), _dptr(self.cl),
                             _dptr(z[0]), _dptr(z[1]), _dptr(z[2]))
        if rc != 0:
            raise ValueError("oracle: invalid parameters")
        return tuple(z)

    def energy(self) -> float:
        return float(lib().orc_energy(ctypes.byref(_params(self.p)), ctypes.byref(self.clock),
                                      _dptr(self.phi), _dptr(self.cs), _dptr(self.cl)))

    def solute(self) -> float:
        return float(lib().orc_solute(ctypes.byref(_params(self.p)), _dptr(self.phi),
                                      _dptr(self.cs), _dptr(self.cl)))

    def front(self):
        xf, cm = ctypes.c_double(), ctypes.c_double()
        lib().orc_front(ctypes.byref(_params(self.p)), ctypes.byref(self.clock),
                        _dptr(self.phi), _dptr(self.cs), _dptr(self.cl),
                        ctypes.byref(xf), ctypes.byref(cm))
        return xf.value, cm.value

"""Python binding of libpf (include/pf.h): argument marshalling only.

Every step of the method runs in the CUDA kernels of libpf.so; there is no CPU
fallback.  If the library cannot be built or loaded, or no GPU is present,
the calls raise.

Parameters use the dict produced by ``workloads.scaled_params``.  Host arrays
are numpy arrays; device arrays are torch CUDA tensors (passed by data_ptr).
By default the handle runs on torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

PF_OK, PF_EINVAL, PF_ENOMEM, PF_ECUDA, PF_ENONFINITE, PF_ETIMEOUT, PF_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
PF_HOST, PF_DEVICE, PF_HOST_ASYNC = 0, 1, 2
BC = {"noflux": 0, "periodic": 1, "dirichlet": 2, "halo": 3}
PRECISION = {"fp32": 0, "fp64": 1}

_lock = threading.Lock()
_lib = None


class PFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libpf error {code}: {msg}")
        self.code = code


class pf_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("dx", ctypes.c_double)]


class pf_bc(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int * 3), ("hi", ctypes.c_int * 3), ("dir_phi", ctypes.c_double),
                ("dir_cs", ctypes.c_double), ("dir_cl", ctypes.c_double)]


class pf_params(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("interp", ctypes.c_int), ("lap_stencil", ctypes.c_int),
                ("mobility_mode", ctypes.c_int)] + [
        (k, ctypes.c_double) for k in ("H", "sigma", "M_phi", "D_s", "D_l", "k_e", "A", "b", "a",
                                       "delta", "theta_ref", "G_theta", "v_pull", "x0", "dt", "c_inf")
    ] + [("shift", ctypes.c_int)]


class pf_batch_desc(ctypes.Structure):
    _fields_ = [("n_instances", ctypes.c_int), ("n", ctypes.POINTER(ctypes.c_int64)),
                ("v_pull", ctypes.POINTER(ctypes.c_double)), ("dt", ctypes.POINTER(ctypes.c_double)),
                ("phi0", ctypes.c_void_p), ("cs0", ctypes.c_void_p), ("cl0", ctypes.c_void_p),
                ("dx", ctypes.c_double), ("bc", pf_bc), ("params", pf_params),
                ("max_steps", ctypes.c_int64), ("steps_per_launch", ctypes.c_int64),
                ("launches_per_graph", ctypes.c_int), ("check_every", ctypes.c_int64),
                ("window", ctypes.c_double), ("tol", ctypes.c_double), ("min_travel", ctypes.c_double),
                ("cells_per_thread", ctypes.c_int), ("energy_every", ctypes.c_int64)]


class pf_batch_result(ctypes.Structure):
    _fields_ = [("k_v", ctypes.POINTER(ctypes.c_double)), ("dkdt", ctypes.POINTER(ctypes.c_double)),
                ("t", ctypes.POINTER(ctypes.c_double)), ("steps", ctypes.POINTER(ctypes.c_int64)),
                ("converged", ctypes.POINTER(ctypes.c_int)), ("phi", ctypes.c_void_p),
                ("cs", ctypes.c_void_p), ("cl", ctypes.c_void_p), ("cells_per_thread", ctypes.c_int),
                ("launches", ctypes.c_int64), ("gpu_ms", ctypes.c_double),
                ("energy", ctypes.POINTER(ctypes.c_double))]


class pf_adjoint_desc(ctypes.Structure):
    _fields_ = [("batch", pf_batch_desc), ("nsteps", ctypes.c_int64), ("wrt", ctypes.c_int),
                ("k_target", ctypes.POINTER(ctypes.c_double)), ("mode", ctypes.c_int),
                ("checkpoint_every", ctypes.c_int)]


class pf_adjoint_result(ctypes.Structure):
    _fields_ = [("k", ctypes.POINTER(ctypes.c_double)), ("dk", ctypes.POINTER(ctypes.c_double)),
                ("loss", ctypes.c_double), ("grad", ctypes.c_double * 3), ("gpu_ms", ctypes.c_double)]


ADJ_MPHI, ADJ_A, ADJ_B = 1, 2, 4
ADJ_TANGENT, ADJ_REVERSE = 0, 1
ADJ_PARAMS = ("M_phi", "A", "b")


# exported symbols and their signatures (the header include/pf.h declares the same set)
_VP = ctypes.c_void_p
_SIGS = {
    "pf_create": (ctypes.c_int, [ctypes.POINTER(pf_grid), ctypes.POINTER(pf_bc),
                                 ctypes.POINTER(pf_params), _VP, ctypes.POINTER(_VP)]),
    "pf_set_fields": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int]),
    "pf_get_fields": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int]),
    "pf_get_fields_async": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int]),
    "pf_sync": (ctypes.c_int, [_VP]),
    "pf_step": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "pf_solute_total_async": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "pf_set_fields_step": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int, ctypes.c_int64]),
    "pf_energy": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "pf_step_energies": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]),
    "pf_solute_total": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "pf_front": (ctypes.c_int, [_VP] + [ctypes.POINTER(ctypes.c_double)] * 3),
    "pf_get_clock": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "pf_set_clock": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int64]),
    "pf_stable_dt": (ctypes.c_int, [ctypes.POINTER(pf_grid), ctypes.POINTER(pf_params),
                                    ctypes.POINTER(ctypes.c_double)]),
    "pf_run_batch": (ctypes.c_int, [ctypes.POINTER(pf_batch_desc), ctypes.POINTER(pf_batch_result), _VP]),
    "pf_adjoint": (ctypes.c_int, [ctypes.POINTER(pf_adjoint_desc), ctypes.POINTER(pf_adjoint_result), _VP]),
    "pf_energy_solute_noalloc": (ctypes.c_int, [ctypes.POINTER(pf_grid), ctypes.POINTER(pf_bc),
                                                ctypes.POINTER(pf_params), ctypes.c_int64, ctypes.c_int64,
                                                _VP, _VP, _VP, _VP, _VP]),
    "pf_halo_bytes": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64)]),
    "pf_get_halo": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int]),
    "pf_set_halo": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int]),
    "pf_step_begin": (ctypes.c_int, [_VP]),
    "pf_step_end": (ctypes.c_int, [_VP]),
    "pf_last_error": (ctypes.c_char_p, [_VP]),
    "pf_destroy": (None, [_VP]),
}


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libpf.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc, h=None):
    if rc != PF_OK:
        msg = lib().pf_last_error(h)
        raise PFError(rc, msg.decode() if msg else "")


def make_structs(pr: dict, precision: str = "fp32"):
    g = pf_grid()
    g.dim = int(pr["dim"])
    n = list(pr["n"]) + [1] * (3 - len(pr["n"]))
    for a in range(3):
        g.n[a] = int(n[a])
    g.dx = float(pr["dx"])
    b = pf_bc()
    for a in range(3):
        b.lo[a] = BC[pr["bc_lo"][a]] if a < g.dim else 0
        b.hi[a] = BC[pr["bc_hi"][a]] if a < g.dim else 0
    b.dir_phi, b.dir_cs, b.dir_cl = (float(v) for v in pr.get("dirichlet", (0.0, 0.0, 1.0)))
    p = pf_params()
    p.precision = PRECISION[precision]
    p.interp = {"quintic": 0, "cubic": 1}[pr.get("interp", "quintic")]
    p.lap_stencil = int(pr["lap"])
    p.mobility_mode = {"Dc": 0, "const": 1}[pr.get("mobility", "Dc")]
    for k in ("H", "sigma", "M_phi", "D_s", "D_l", "k_e", "A", "b", "a", "delta", "theta_ref",
              "G_theta", "v_pull", "x0", "dt", "c_inf"):
        setattr(p, k, float(pr[k]))
    p.shift = int(bool(pr.get("shift", False)))
    if pr.get("form", "cd") != "cd":
        raise ValueError("libpf implements the conservative (c, d) update only")
    return g, b, p


def stable_dt(pr: dict) -> float:
    g, _, p = make_structs(pr)
    out = ctypes.c_double()
    _check(lib().pf_stable_dt(ctypes.byref(g), ctypes.byref(p), ctypes.byref(out)))
    return out.value


def _current_stream():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libpf needs a CUDA device")
    return torch.cuda.current_stream().cuda_stream


class Sim:
    """One simulation handle (pf_create ... pf_destroy)."""

    def __init__(self, pr: dict, precision: str = "fp32", stream=None):
        self.pr = dict(pr)
        self.precision = precision
        self.dtype = np.float64 if precision == "fp64" else np.float32
        self.shape = tuple(int(v) for v in list(pr["n"])[: pr["dim"]][::-1])
        g, b, p = make_structs(pr, precision)
        s = _current_stream() if stream is None else stream
        h = _VP()
        rc = lib().pf_create(ctypes.byref(g), ctypes.byref(b), ctypes.byref(p), _VP(s), ctypes.byref(h))
        _check(rc, None)
        self._h = h
        self.stream = s

    # -- fields
    def _field_ptrs(self, phi, cs, cl):
        """(pointers, where, arrays kept alive) for CUDA tensors or host arrays."""
        if all(hasattr(a, "data_ptr") for a in (phi, cs, cl)):
            for a in (phi, cs, cl):
                if not a.is_cuda or not a.is_contiguous() or tuple(a.shape) != self.shape:
                    raise ValueError("device fields must be contiguous CUDA tensors of the grid shape")
                if a.element_size() != np.dtype(self.dtype).itemsize:
                    raise ValueError("device field dtype does not match the handle precision")
            return [_VP(a.data_ptr()) for a in (phi, cs, cl)], PF_DEVICE, None
        arrs = [np.ascontiguousarray(a, dtype=self.dtype) for a in (phi, cs, cl)]
        for a in arrs:
            if a.shape != self.shape:
                raise ValueError(f"field shape {a.shape} != {self.shape}")
        return [_VP(a.ctypes.data) for a in arrs], PF_HOST, arrs

    def set_fields(self, phi, cs, cl):
        ptrs, where, _keep = self._field_ptrs(phi, cs, cl)
        _check(lib().pf_set_fields(self._h, *ptrs, where), self._h)

    def set_fields_step(self, phi, cs, cl, n: int = 1, wait: bool = True):
        """set_fields then step(n), the upload overlapped with the first step
        (3D, device or page-locked host fields).  wait=False (page-locked host
        arrays of the handle's dtype, contiguous): the call returns without
        waiting for the copies; the arrays must stay unchanged until sync() or
        another synchronising call returns."""
        ptrs, where, keep = self._field_ptrs(phi, cs, cl)
        if not wait and where == PF_HOST:
            if any(k is not a for k, a in zip(keep, (phi, cs, cl))):
                raise ValueError("wait=False needs contiguous host arrays of the handle's dtype (no copy)")
            where = PF_HOST_ASYNC
        _check(lib().pf_set_fields_step(self._h, *ptrs, where, int(n)), self._h)

    def _device_out(self, out):
        """Pointers of three output CUDA tensors, checked (the library cannot
        check a raw pointer): contiguous, the grid shape, the handle's dtype."""
        if len(out) != 3:
            raise ValueError("three output tensors (phi, cs, cl)")
        for a in out:
            if (not getattr(a, "is_cuda", False) or not a.is_contiguous() or tuple(a.shape) != self.shape
                    or a.element_size() != np.dtype(self.dtype).itemsize or not a.is_floating_point()):
                raise ValueError("device outputs must be contiguous CUDA tensors of the grid shape and dtype")
        return [_VP(a.data_ptr()) for a in out]

    def get_fields(self, out=None, out_host=None):
        """Return (phi, cs, cl) as numpy arrays, or fill the given CUDA tensors
        (out), or the given host arrays (out_host: contiguous numpy arrays of the
        grid shape and the handle's dtype, page-locked for a direct copy)."""
        if out is not None:
            ptrs = self._device_out(out)
            _check(lib().pf_get_fields(self._h, *ptrs, PF_DEVICE), self._h)
            return out
        if out_host is not None:
            for a in out_host:
                if a.shape != self.shape or a.dtype != self.dtype or not a.flags.c_contiguous:
                    raise ValueError("out_host arrays must be contiguous, of the grid shape and dtype")
            _check(lib().pf_get_fields(self._h, *[_VP(a.ctypes.data) for a in out_host], PF_HOST), self._h)
            return tuple(out_host)
        arrs = [np.empty(self.shape, dtype=self.dtype) for _ in range(3)]
        _check(lib().pf_get_fields(self._h, *[_VP(a.ctypes.data) for a in arrs], PF_HOST), self._h)
        return tuple(arrs)

    def get_fields_async(self, out=None, out_host=None):
        """Queue the read-back of (phi, cs, cl) into CUDA tensors (out) or
        page-locked host arrays (out_host) without waiting; valid after sync()."""
        if out is not None:
            ptrs, where = self._device_out(out), PF_DEVICE
        else:
            for a in out_host:
                if a.shape != self.shape or a.dtype != self.dtype or not a.flags.c_contiguous:
                    raise ValueError("out_host arrays must be contiguous, of the grid shape and dtype")
            ptrs, where = [_VP(a.ctypes.data) for a in out_host], PF_HOST
        _check(lib().pf_get_fields_async(self._h, *ptrs, where), self._h)
        return out if out is not None else out_host

    def sync(self):
        """Wait for all work of the handle, read-backs included."""
        _check(lib().pf_sync(self._h), self._h)

    # -- stepping and diagnostics
    def step(self, n: int = 1):
        _check(lib().pf_step(self._h, int(n)), self._h)

    def energy(self) -> float:
        v = ctypes.c_double()
        _check(lib().pf_energy(self._h, ctypes.byref(v)), self._h)
        return v.value

    def step_energies(self, n: int) -> np.ndarray:
        """n steps with F_h recorded on the device after each; returns the n energies."""
        out = np.empty(int(n), dtype=np.float64)
        _check(lib().pf_step_energies(self._h, int(n), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               self._h)
        return out

    def solute_total(self) -> float:
        v = ctypes.c_double()
        _check(lib().pf_solute_total(self._h, ctypes.byref(v)), self._h)
        return v.value

    def solute_total_async(self, out, i: int = 0):
        """Queue S_h into out[i] (a float64 numpy array, page-locked for the copy
        to be asynchronous); valid after the handle's stream is synchronised."""
        if out.dtype != np.float64 or not out.flags.c_contiguous or not 0 <= i < out.size:
            raise ValueError("out must be a contiguous float64 array and i an index into it")
        ptr = ctypes.cast(out.ctypes.data + 8 * int(i), ctypes.POINTER(ctypes.c_double))
        _check(lib().pf_solute_total_async(self._h, ptr), self._h)

    def front(self):
        x, v, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().pf_front(self._h, ctypes.byref(x), ctypes.byref(v), ctypes.byref(c)), self._h)
        return x.value, v.value, c.value

    # -- z-slab halos (a handle whose z sides are "halo")
    def halo_bytes(self) -> int:
        v = ctypes.c_int64()
        _check(lib().pf_halo_bytes(self._h, ctypes.byref(v)), self._h)
        return v.value

    def _halo_buf(self, buf):
        if hasattr(buf, "data_ptr"):   # a torch tensor on the GPU or on the host
            if not buf.is_contiguous() or buf.numel() * buf.element_size() != self.halo_bytes():
                raise ValueError("halo buffer: a contiguous tensor of halo_bytes() bytes")
            return _VP(buf.data_ptr()), (PF_DEVICE if buf.is_cuda else PF_HOST)
        if not buf.flags.c_contiguous or buf.nbytes != self.halo_bytes():
            raise ValueError("halo buffer: a contiguous host array of halo_bytes() bytes")
        return _VP(buf.ctypes.data), PF_HOST

    def get_halo(self, side: int, buf):
        """Export the two outermost planes at z side 0 (low) or 1 (high) into
        buf (a CUDA tensor or a host array of halo_bytes() bytes)."""
        ptr, where = self._halo_buf(buf)
        _check(lib().pf_get_halo(self._h, int(side), ptr, where), self._h)
        return buf

    def set_halo(self, side: int, buf):
        """Import the two ghost planes beyond z side 0 (low) or 1 (high)."""
        ptr, where = self._halo_buf(buf)
        _check(lib().pf_set_halo(self._h, int(side), ptr, where), self._h)

    def step_begin(self):
        """First half of a split step (3D): queue the z-chunks that read no
        ghost plane on the handle's interior stream.  Exchange the halos, then
        call step_end(); the two advance one step as step(1) does."""
        _check(lib().pf_step_begin(self._h), self._h)

    def step_end(self):
        """Second half of a split step: the chunks next to the z sides (the
        halos imported by now), then the join with the interior."""
        _check(lib().pf_step_end(self._h), self._h)

    @property
    def clock(self):
        s, k = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().pf_get_clock(self._h, ctypes.byref(s), ctypes.byref(k)), self._h)
        return s.value, k.value

    def set_clock(self, step: int, shifts: int = 0):
        _check(lib().pf_set_clock(self._h, int(step), int(shifts)), self._h)

    def close(self):
        if getattr(self, "_h", None):
            lib().pf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def run_batch(pr: dict, lengths, v_pull, phi0, cs0, cl0, *, precision="fp32", dt=None,
              max_steps=100000, steps_per_launch=500, launches_per_graph=4, check_every=100,
              window=1.0, tol=1e-8, min_travel=0.0, cells_per_thread=0, want_fields=False,
              energy_every=0, stream=None):
    """pf_run_batch: many 1D pulled fronts in one persistent launch per chunk.

    pr: shared 1D parameters (workloads.pulled_front_1d style; n, v_pull, dt and
    shift are ignored); lengths, v_pull (and dt) per instance; phi0, cs0, cl0
    packed initial fields.  Returns a dict of per-instance arrays.
    """
    N = len(lengths)
    dtype = np.float64 if precision == "fp64" else np.float32
    n_arr = np.ascontiguousarray(lengths, dtype=np.int64)
    v_arr = np.ascontiguousarray(v_pull, dtype=np.float64)
    dt_arr = np.ascontiguousarray(dt if dt is not None else np.zeros(N), dtype=np.float64)
    fields = [np.ascontiguousarray(a, dtype=dtype) for a in (phi0, cs0, cl0)]
    total = int(n_arr.sum())
    for a in fields:
        if a.shape != (total,):
            raise ValueError("packed fields must have sum(lengths) entries")
    g, b, p = make_structs(dict(pr, n=(8,), shift=False, v_pull=0.0), precision)
    D = pf_batch_desc()
    D.n_instances = N
    D.n = n_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    D.v_pull = v_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    D.dt = dt_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    D.phi0, D.cs0, D.cl0 = (a.ctypes.data for a in fields)
    D.dx = float(pr["dx"])
    D.bc = b
    D.params = p
    D.max_steps, D.steps_per_launch, D.launches_per_graph = int(max_steps), int(steps_per_launch), int(launches_per_graph)
    D.check_every, D.window, D.tol, D.cells_per_thread = int(check_every), float(window), float(tol), int(cells_per_thread)
    D.min_travel = float(min_travel)
    D.energy_every = int(energy_every)
    out = dict(k_v=np.zeros(N), dkdt=np.zeros(N), t=np.zeros(N), steps=np.zeros(N, np.int64),
               converged=np.zeros(N, np.int32))
    R = pf_batch_result()
    R.k_v = out["k_v"].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    R.dkdt = out["dkdt"].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    R.t = out["t"].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    R.steps = out["steps"].ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    R.converged = out["converged"].ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    if energy_every > 0:
        out["energy"] = np.zeros((N, int(max_steps) // int(energy_every)))
        R.energy = out["energy"].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if want_fields:
        for k in ("phi", "cs", "cl"):
            out[k] = np.zeros(total, dtype=dtype)
        R.phi, R.cs, R.cl = (out[k].ctypes.data for k in ("phi", "cs", "cl"))
    s = _current_stream() if stream is None else stream
    _check(lib().pf_run_batch(ctypes.byref(D), ctypes.byref(R), _VP(s)), None)
    out.update(cells_per_thread=R.cells_per_thread, launches=R.launches, gpu_ms=R.gpu_ms)
    return out


def _batch_desc(pr, lengths, v_pull, phi0, cs0, cl0, precision, dt, keep):
    N = len(lengths)
    dtype = np.float64 if precision == "fp64" else np.float32
    n_arr = np.ascontiguousarray(lengths, dtype=np.int64)
    v_arr = np.ascontiguousarray(v_pull, dtype=np.float64)
    dt_arr = np.ascontiguousarray(dt if dt is not None else np.zeros(N), dtype=np.float64)
    fields = [np.ascontiguousarray(a, dtype=dtype) for a in (phi0, cs0, cl0)]
    total = int(n_arr.sum())
    for a in fields:
        if a.shape != (total,):
            raise ValueError("packed fields must have sum(lengths) entries")
    keep.extend([n_arr, v_arr, dt_arr, *fields])
    g, b, p = make_structs(dict(pr, n=(8,), shift=False, v_pull=0.0), precision)
    D = pf_batch_desc()
    D.n_instances = N
    D.n = n_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    D.v_pull = v_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    D.dt = dt_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    D.phi0, D.cs0, D.cl0 = (a.ctypes.data for a in fields)
    D.dx = float(pr["dx"])
    D.bc = b
    D.params = p
    return D


def adjoint(pr: dict, lengths, v_pull, phi0, cs0, cl0, nsteps, *, k_target=None,
            wrt=("M_phi", "A", "b"), precision="fp32", dt=None, steps_per_launch=0,
            cells_per_thread=0, stream=None, mode="tangent", checkpoint_every=0):
    """pf_adjoint: k_i = c_inf / max c after `nsteps` steps of every pulled front
    and the exact derivatives dk_i/d(M_phi, A, b) of the discrete run, by the
    tangent-linear run (mode="tangent") or by a reverse sweep with stored
    checkpoints (mode="reverse", every `checkpoint_every` steps, 0: ~sqrt(nsteps)).

    Same instance description as run_batch.  Returns dict(k, dk (N x 3), loss,
    grad (3,), gpu_ms); loss and grad are those of sum (k - k_target)^2.
    """
    keep = []
    D = _batch_desc(pr, lengths, v_pull, phi0, cs0, cl0, precision, dt, keep)
    D.steps_per_launch = int(steps_per_launch)
    D.cells_per_thread = int(cells_per_thread)
    N = len(lengths)
    A = pf_adjoint_desc()
    A.batch = D
    A.nsteps = int(nsteps)
    A.wrt = sum(1 << ADJ_PARAMS.index(w) for w in wrt)
    A.mode = {"tangent": ADJ_TANGENT, "reverse": ADJ_REVERSE}[mode]
    A.checkpoint_every = int(checkpoint_every)
    kt = None
    if k_target is not None:
        kt = np.ascontiguousarray(k_target, dtype=np.float64)
        if kt.shape != (N,):
            raise ValueError("k_target needs one value per instance")
        A.k_target = kt.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    k = np.zeros(N)
    dk = np.zeros(3 * N)
    R = pf_adjoint_result()
    R.k = k.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    R.dk = dk.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    s = _current_stream() if stream is None else stream
    _check(lib().pf_adjoint(ctypes.byref(A), ctypes.byref(R), _VP(s)), None)
    return dict(k=k, dk=dk.reshape(N, 3), loss=R.loss, grad=np.array(R.grad[:]), gpu_ms=R.gpu_ms)


def calibrate(pr: dict, lengths, v_pull, phi0, cs0, cl0, nsteps, k_target, *, iters=50, lr=0.05,
              wrt=("M_phi", "A", "b"), precision="fp32", dt=None, betas=(0.9, 0.999), eps=1e-8,
              callback=None, mode="tangent", bounds=None):
    """Adam on the logarithms of the chosen parameters (M_phi, A, b > 0), each
    iteration one pf_adjoint run; returns (parameters, history of losses).
    bounds: optional {name: (lo, hi)}; a parameter is clamped into its range
    after every update (the model diverges for some parameter sets)."""
    idx = [ADJ_PARAMS.index(w) for w in wrt]
    theta = np.log(np.array([pr[ADJ_PARAMS[j]] for j in idx], dtype=np.float64))
    lo = np.array([np.log((bounds or {}).get(ADJ_PARAMS[j], (0.0, np.inf))[0] or 1e-300) for j in idx])
    hi = np.array([np.log((bounds or {}).get(ADJ_PARAMS[j], (0.0, np.inf))[1]) for j in idx])
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    hist = []
    cur = dict(pr)
    for it in range(1, iters + 1):
        for j, t in zip(idx, theta):
            cur[ADJ_PARAMS[j]] = float(np.exp(t))
        r = adjoint(cur, lengths, v_pull, phi0, cs0, cl0, nsteps, k_target=k_target, wrt=wrt,
                    precision=precision, dt=dt, mode=mode)
        hist.append(r["loss"])
        g = np.array([r["grad"][j] for j in idx]) * np.exp(theta)   # d/d(log theta)
        m = betas[0] * m + (1 - betas[0]) * g
        v = betas[1] * v + (1 - betas[1]) * g * g
        mh = m / (1 - betas[0] ** it)
        vh = v / (1 - betas[1] ** it)
        theta = np.clip(theta - lr * mh / (np.sqrt(vh) + eps), lo, hi)
        if callback is not None:
            callback(it, cur, r)
    for j, t in zip(idx, theta):
        cur[ADJ_PARAMS[j]] = float(np.exp(t))
    return {w: cur[w] for w in wrt}, hist


class KvProblem:
    """The fixed part of a k(V) calibration problem for kv_loss: instances,
    initial fields, step count, targets, precision, and how the gradient is
    taken (mode="reverse": the reverse sweep with checkpoints; "tangent")."""

    def __init__(self, pr, lengths, v_pull, phi0, cs0, cl0, nsteps, k_target, *, precision="fp32", dt=None,
                 mode="reverse"):
        self.pr, self.lengths, self.v_pull = dict(pr), lengths, v_pull
        self.fields = (phi0, cs0, cl0)
        self.nsteps, self.k_target, self.precision, self.dt = nsteps, k_target, precision, dt
        self.mode = mode

    def run(self, theta):
        pr = dict(self.pr, **{n: float(t) for n, t in zip(ADJ_PARAMS, theta)})
        return adjoint(pr, self.lengths, self.v_pull, *self.fields, self.nsteps, k_target=self.k_target,
                       precision=self.precision, dt=self.dt, mode=self.mode)


def kv_loss(theta, problem: KvProblem):
    """sum_i (k_i - k_target_i)^2 as a differentiable torch scalar of
    theta = (M_phi, A, b) (a float64 tensor of 3): forward and the derivatives
    come from one pf_adjoint run; backward scales the stored gradient."""
    import torch

    class _KvLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, th):
            r = problem.run(th.detach().cpu().numpy())
            ctx.save_for_backward(torch.as_tensor(r["grad"], dtype=th.dtype, device=th.device))
            return torch.as_tensor(r["loss"], dtype=th.dtype, device=th.device)

        @staticmethod
        def backward(ctx, g):
            (grad,) = ctx.saved_tensors
            return g * grad

    return _KvLoss.apply(theta)


def _noalloc_pointers(pr: dict, precision: str, phi, cs, cl, out):
    """Device pointers of the arguments of pf_energy_solute_noalloc, after the
    checks the C entry point cannot make on raw pointers: the three fields are
    contiguous CUDA tensors of exactly prod(n) elements of the precision's
    float type, and out a contiguous float64 CUDA tensor of at least 2 elements,
    all on one device.  PFError(PF_EINVAL) otherwise, before anything runs."""
    if precision not in PRECISION:
        raise PFError(PF_EINVAL, f"unknown precision {precision!r}")
    cells = 1
    for v in list(pr["n"])[: int(pr["dim"])]:
        cells *= int(v)
    want = "torch.float64" if precision == "fp64" else "torch.float32"

    def bad(msg):
        return PFError(PF_EINVAL, "energy_solute_noalloc: " + msg)

    for name, t in (("out", out), ("phi", phi), ("cs", cs), ("cl", cl)):
        if not hasattr(t, "data_ptr") or not getattr(t, "is_cuda", False):
            raise bad(f"{name} must be a CUDA tensor")
        if not t.is_contiguous():
            raise bad(f"{name} must be contiguous")
        if t.device != out.device:
            raise bad(f"{name} is on {t.device}, out on {out.device}")
    if str(out.dtype) != "torch.float64" or out.numel() < 2:
        raise bad("out must be a float64 tensor of at least 2 elements")
    for name, t in (("phi", phi), ("cs", cs), ("cl", cl)):
        if str(t.dtype) != want:
            raise bad(f"{name} has dtype {t.dtype}, the {precision} precision needs {want}")
        if t.numel() != cells:
            raise bad(f"{name} has {t.numel()} elements, the grid has {cells}")
    return [_VP(t.data_ptr()) for t in (phi, cs, cl, out)]


def energy_solute_noalloc(pr: dict, phi, cs, cl, out, precision="fp32", step=0, shifts=0, stream=None):
    """pf_energy_solute_noalloc on CUDA tensors: writes (F_h, S_h) into the
    float64 CUDA tensor `out` (at least 2 elements) without allocating device
    memory.  The fields are checked first (see _noalloc_pointers)."""
    ptrs = _noalloc_pointers(pr, precision, phi, cs, cl, out)
    g, b, p = make_structs(pr, precision)
    s = _current_stream() if stream is None else stream
    rc = lib().pf_energy_solute_noalloc(ctypes.byref(g), ctypes.byref(b), ctypes.byref(p), int(step),
                                        int(shifts), *ptrs, _VP(s))
    _check(rc, None)

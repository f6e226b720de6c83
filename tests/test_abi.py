"""C-ABI checks that need no GPU: the library builds and loads, exports every
symbol include/pf.h declares, validates its arguments before touching the
device, and its stable-dt rule agrees with the input recipe's."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2303_09671_gb300 import build as pbuild
from paper_2303_09671_gb300 import pf
from paper_2303_09671_gb300 import workloads as wl

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "pf.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pf_[a-z_]+)\s*\(", src)))


def test_library_loads_and_exports_header_symbols():
    L = pf.lib()
    names = declared_functions()
    assert "pf_create" in names and "pf_step" in names
    for n in names:
        assert hasattr(L, n), f"{n} declared in pf.h but not exported"
    out = subprocess.run(["nm", "-D", "--defined-only", pbuild.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pf_[a-z_]+)\b", out))
    assert set(names) == exported, f"header/exports mismatch: {set(names) ^ exported}"


def test_binding_covers_header():
    assert set(pf._SIGS) == set(declared_functions())


def _create(pr, **over):
    g, b, p = pf.make_structs(pr, "fp32")
    for k, v in over.items():
        for s in (g, b, p):
            if hasattr(s, k):
                setattr(s, k, v)
    h = ctypes.c_void_p()
    rc = pf.lib().pf_create(ctypes.byref(g), ctypes.byref(b), ctypes.byref(p), None, ctypes.byref(h))
    return rc, pf.lib().pf_last_error(None).decode()


@pytest.mark.parametrize("over,needle", [
    (dict(dim=4), "dim"),
    (dict(k_e=1.5), "k_e"),
    (dict(b=0.0), "b must"),
    (dict(lap_stencil=5), "lap_stencil"),
    (dict(dt=1.0), "stability"),
    (dict(dx=-1.0), "dx"),
    (dict(M_phi=0.0), "positive"),
    (dict(shift=1), "1D only"),
])
def test_create_rejects_invalid(over, needle):
    pr, *_ = wl.random_state(3, (16, 8, 8))
    rc, msg = _create(pr, **over)
    assert rc == pf.PF_EINVAL and needle in msg


def test_create_rejects_one_sided_periodic():
    pr, *_ = wl.random_state(2, (16, 8), bc_lo=("periodic", "noflux"), bc_hi=("noflux", "noflux"))
    rc, msg = _create(pr)
    assert rc == pf.PF_EINVAL and "periodic" in msg


def test_null_handle_calls_fail_cleanly():
    L = pf.lib()
    assert L.pf_step(None, 1) == pf.PF_EINVAL
    assert L.pf_set_fields_step(None, None, None, None, pf.PF_HOST, 1) == pf.PF_EINVAL
    v = ctypes.c_double()
    assert L.pf_energy(None, ctypes.byref(v)) == pf.PF_EINVAL
    L.pf_destroy(None)


@pytest.mark.parametrize("maker", [
    lambda: wl.planar_1d(A=2.0, b=1.0),
    lambda: wl.perturbed_front_2d(nx=64, ny=64, A=1.5, b=0.3),
    lambda: wl.random_state(3, (16, 8, 8), mobility="const"),
])
def test_stable_dt_matches_recipe(maker):
    pr = maker()[0]
    assert abs(pf.stable_dt(pr) - wl.stable_dt(pr)) <= 1e-13 * wl.stable_dt(pr)


def test_create_rejects_grids_beyond_the_launch_limits():
    """y extents the 2D/3D kernels cannot tile (grid.y <= 65535) and x-y planes
    beyond 32-bit offsets are refused before any allocation."""
    pr, *_ = wl.random_state(2, (16, 8))
    g, b, p = pf.make_structs(pr, "fp32")
    g.n[1] = 65535 * 8 + 1
    h = ctypes.c_void_p()
    rc = pf.lib().pf_create(ctypes.byref(g), ctypes.byref(b), ctypes.byref(p), None, ctypes.byref(h))
    assert rc == pf.PF_EINVAL and "n[1]" in pf.lib().pf_last_error(None).decode()
    pr, *_ = wl.random_state(3, (16, 8, 8))
    g, b, p = pf.make_structs(pr, "fp32")
    g.n[0], g.n[1], g.n[2] = 1 << 17, 1 << 14, 3
    rc = pf.lib().pf_create(ctypes.byref(g), ctypes.byref(b), ctypes.byref(p), None, ctypes.byref(h))
    assert rc == pf.PF_EINVAL and "plane" in pf.lib().pf_last_error(None).decode()


def test_empty_batch_is_rejected_before_any_device_work():
    """A batch of no instances (or of an instance below 8 cells) is an invalid
    descriptor: PF_EINVAL from validation, which runs before any CUDA call, so
    this holds through the C ABI without a GPU."""
    L = pf.lib()
    pr, _, _, _ = wl.pulled_front_1d(N=64)
    g, b, p = pf.make_structs(dict(pr, n=(8,), shift=False, v_pull=0.0), "fp32")
    for lengths in ([], [4]):
        n = np.ascontiguousarray(lengths if lengths else [0], dtype=np.int64)
        v = np.full(max(1, len(lengths)), 0.1)
        z = np.zeros(64, dtype=np.float32)
        D = pf.pf_batch_desc()
        D.n_instances = len(lengths)
        D.n = n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        D.v_pull = v.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        D.phi0 = D.cs0 = D.cl0 = z.ctypes.data
        D.dx = float(pr["dx"])
        D.bc = b
        D.params = p
        D.max_steps, D.steps_per_launch, D.launches_per_graph = 100, 10, 1
        R = pf.pf_batch_result()
        assert L.pf_run_batch(ctypes.byref(D), ctypes.byref(R), None) == pf.PF_EINVAL


# ------------------------------------------------ pf_energy_solute_noalloc checks

class _FakeCudaTensor:
    """Stands in for a torch CUDA tensor in the argument checks of
    pf.energy_solute_noalloc (no GPU here; nothing is dereferenced)."""

    def __init__(self, numel, dtype="torch.float32", cuda=True, contiguous=True, device="cuda:0"):
        self._n, self.dtype, self.is_cuda, self._c, self.device = numel, dtype, cuda, contiguous, device

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        return 0x1000


@pytest.mark.parametrize("case,needle", [
    ("short_field", "elements"),
    ("f32_out", "float64"),
    ("one_element_out", "float64"),
    ("wrong_dtype", "dtype"),
    ("host_field", "CUDA"),
    ("strided", "contiguous"),
    ("other_device", "cuda:1"),
])
def test_noalloc_binding_rejects_bad_tensors(case, needle):
    pr, *_ = wl.random_state(2, (8, 8))
    F = _FakeCudaTensor
    f = [F(64), F(64), F(64)]
    out = F(2, dtype="torch.float64")
    if case == "short_field":
        f[1] = F(63)
    elif case == "f32_out":
        out = F(2, dtype="torch.float32")
    elif case == "one_element_out":
        out = F(1, dtype="torch.float64")
    elif case == "wrong_dtype":
        f[2] = F(64, dtype="torch.float64")
    elif case == "host_field":
        f[0] = F(64, cuda=False)
    elif case == "strided":
        f[0] = F(64, contiguous=False)
    elif case == "other_device":
        f[2] = F(64, device="cuda:1")
    with pytest.raises(pf.PFError, match=needle):
        pf.energy_solute_noalloc(pr, *f, out, precision="fp32")
    ptrs = pf._noalloc_pointers(pr, "fp32", F(64), F(64), F(64), F(2, dtype="torch.float64"))
    assert len(ptrs) == 4


@pytest.mark.parametrize("over,needle", [
    (dict(interp=7), "interp"),
    (dict(lo=(5, 0, 0)), "boundary"),
    (dict(lo=(1, 0, 0)), "periodic"),
    (dict(H=float("inf")), "non-finite"),
    (dict(sigma=float("nan")), "positive"),
    (dict(lap_stencil=19), "lap_stencil"),
    (dict(dt=float("nan")), "non-finite"),
])
def test_noalloc_entry_point_validates_like_pf_create(over, needle):
    """The C entry point returns PF_EINVAL for the descriptions pf_create
    rejects (unknown interp, an unknown or one-sided boundary code, non-finite
    parameters), before it touches the device."""
    pr, *_ = wl.random_state(2, (8, 8))
    g, b, p = pf.make_structs(pr, "fp32")
    for k, v in over.items():
        for s in (g, b, p):
            if hasattr(s, k):
                if k in ("lo", "hi"):
                    for a, x in enumerate(v):
                        getattr(s, k)[a] = x
                else:
                    setattr(s, k, v)
    dummy = ctypes.c_void_p(0x1000)
    rc = pf.lib().pf_energy_solute_noalloc(ctypes.byref(g), ctypes.byref(b), ctypes.byref(p), 0, 0,
                                           dummy, dummy, dummy, dummy, None)
    assert rc == pf.PF_EINVAL
    assert needle in pf.lib().pf_last_error(None).decode()


@pytest.mark.parametrize("dim,axis,needle", [(3, 0, "halo"), (3, 1, "halo"), (2, 1, "halo")])
def test_halo_sides_only_on_3d_z(dim, axis, needle):
    """PF_BC_HALO (the cut between two slabs of a grid decomposed along z) is
    accepted on the z sides of a 3D handle only."""
    n = (16, 12, 10)[:dim]
    pr, *_ = wl.random_state(dim, n)
    g, b, p = pf.make_structs(pr, "fp32")
    b.lo[axis] = 3
    h = ctypes.c_void_p()
    rc = pf.lib().pf_create(ctypes.byref(g), ctypes.byref(b), ctypes.byref(p), None, ctypes.byref(h))
    assert rc == pf.PF_EINVAL and needle in pf.lib().pf_last_error(None).decode()


def test_device_outputs_are_checked_before_the_call():
    """get_fields(out=...) and get_fields_async(out=...) hand raw pointers to
    the library, which cannot check them: the binding refuses tensors of the
    wrong shape, dtype or layout, or not on the GPU, before any call."""
    s = pf.Sim.__new__(pf.Sim)
    s.shape, s.dtype, s._h = (4, 5, 6), np.float32, None

    class T:
        def __init__(self, shape=(4, 5, 6), es=4, cuda=True, contiguous=True, fp=True):
            self.shape, self._es, self.is_cuda, self._c, self._fp = shape, es, cuda, contiguous, fp

        def is_contiguous(self):
            return self._c

        def element_size(self):
            return self._es

        def is_floating_point(self):
            return self._fp

        def data_ptr(self):
            return 0x1000

    assert len(s._device_out([T(), T(), T()])) == 3
    for bad in (T(shape=(4, 5, 5)), T(es=8), T(cuda=False), T(contiguous=False), T(fp=False)):
        with pytest.raises(ValueError):
            s._device_out([T(), bad, T()])
    with pytest.raises(ValueError):
        s._device_out([T(), T()])

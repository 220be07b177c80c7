"""Thin ctypes binding of libsop.so (the ``sop_*`` C ABI of ``include/sop.h``).

Functions carry the C names and only marshal arguments: every step of the
split-operator path runs in the library's CUDA kernels.  PyTorch provides the
device memory and the stream.  The library must have been built
(``paper_1012_3911_gb300.build.build()``); there is no fallback, and a missing
library raises ``RuntimeError``.

Shapes: ``dims`` is given in axis order (n_x, n_y, n_z) as in the C ABI; a
state tensor has the NumPy/PyTorch shape (C, n_z, n_y, n_x) with the leading
component axis only for Dirac (C = 4).
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SOP_CHECK=1: the check build (see build.py)
LIB_PATH = os.path.join(_HERE, "_build_check" if os.environ.get("SOP_CHECK", "") == "1" else "_build", "libsop.so")

SOP_C64, SOP_C128 = 0, 1
SOP_OK, SOP_EINVAL, SOP_EUNSUPPORTED, SOP_ENOMEM, SOP_ECUDA, SOP_ETIMEOUT, SOP_ESTATE = 0, -1, -2, -3, -4, -5, -6
SOP_PASS_CLASSES = 5
PASS_CLASS_NAMES = ("real_space_pass", "momentum_space_pass", "middle_axis_pass", "whole_step_1d", "table_setup")

_lib = None
_lock = threading.Lock()


class SopError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"sop status {status}: {message}")
        self.status = status


class sop_params(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("charge", ctypes.c_double), ("hbar", ctypes.c_double),
                ("c", ctypes.c_double)]


def load(path: str = LIB_PATH):
    """Load libsop.so (once).  Raises RuntimeError if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1012_3911_gb300.build.build(); "
                               "the split-operator path has no CPU fallback")
        lib = ctypes.CDLL(path)
        vp, i64, d, i = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        lib.sop_plan_create.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(i64), ctypes.POINTER(d), i, i,
                                        ctypes.POINTER(sop_params), vp]
        lib.sop_plan_destroy.argtypes = [vp]
        lib.sop_bind_state.argtypes = [vp, vp]
        lib.sop_set_potential.argtypes = [vp, vp, i]
        lib.sop_step.argtypes = [vp, i64, d, vp]
        lib.sop_step_host.argtypes = [vp, vp, i64, d, vp]
        lib.sop_norm.argtypes = [vp, ctypes.POINTER(d)]
        lib.sop_energy.argtypes = [vp, ctypes.POINTER(d)]
        lib.sop_profile_enable.argtypes = [vp, i]
        lib.sop_profile_read.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(i64), i]
        lib.sop_launch_counter.argtypes = [vp]
        lib.sop_launch_counter.restype = i64
        lib.sop_last_error.restype = ctypes.c_char_p
        lib.sop_version.restype = i
        for name in ("sop_plan_create", "sop_plan_destroy", "sop_bind_state", "sop_set_potential", "sop_step",
                     "sop_step_host", "sop_norm", "sop_energy", "sop_profile_enable", "sop_profile_read"):
            getattr(lib, name).restype = i
        _lib = lib
        return lib


def sop_last_error() -> str:
    return load().sop_last_error().decode()


def sop_version() -> int:
    return int(load().sop_version())


def _check(rc: int) -> None:
    if rc != SOP_OK:
        raise SopError(rc, sop_last_error())


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def sop_plan_create(dims: Sequence[int], spacing: Sequence[float], components: int = 1, dtype: int = SOP_C64,
                    params: Optional[dict] = None, stream=None) -> int:
    """Create a plan; returns the opaque handle (an int).  ``stream`` is a
    torch.cuda.Stream, a raw handle, or None for torch's current stream."""
    lib = load()
    nd = len(dims)
    cd = (ctypes.c_int64 * nd)(*[int(x) for x in dims])
    cs = (ctypes.c_double * nd)(*[float(x) for x in spacing])
    pp = None
    if params is not None:
        pr = sop_params(params.get("mass", 1.0), params.get("charge", -1.0), params.get("hbar", 1.0),
                        params.get("c", 137.036))
        pp = ctypes.pointer(pr)
    out = ctypes.c_void_p()
    _check(lib.sop_plan_create(ctypes.byref(out), nd, cd, cs, int(components), int(dtype), pp,
                               _stream_handle(stream)))
    return out.value


def sop_plan_destroy(plan: int) -> None:
    _check(load().sop_plan_destroy(plan))


def sop_bind_state(plan: int, psi) -> None:
    """Bind a contiguous CUDA tensor (complex64/complex128) as the state."""
    if not psi.is_cuda or not psi.is_contiguous():
        raise ValueError("psi must be a contiguous CUDA tensor")
    _check(load().sop_bind_state(plan, psi.data_ptr()))


def sop_set_potential(plan: int, V) -> None:
    """Copy a CUDA float32/float64 tensor of prod(dims) values as V."""
    import torch
    if not V.is_cuda or not V.is_contiguous():
        raise ValueError("V must be a contiguous CUDA tensor")
    if V.dtype not in (torch.float32, torch.float64):
        raise ValueError("V must be float32 or float64")
    _check(load().sop_set_potential(plan, V.data_ptr(), int(V.dtype == torch.float64)))


def _field_ptr(field, n_steps: int, ndim: int):
    if field is None:
        return None, None
    f = np.ascontiguousarray(np.asarray(field, dtype=np.float64).reshape(int(n_steps), ndim))
    return f, f.ctypes.data


def sop_step(plan: int, n_steps: int, dt: float, field=None, ndim: Optional[int] = None) -> None:
    """Asynchronous: n_steps Strang steps of size dt on the bound state.
    ``field`` (host) has n_steps rows of ndim samples, or None."""
    keep, ptr = (None, None)
    if field is not None:
        nd = ndim if ndim is not None else np.asarray(field).reshape(int(n_steps), -1).shape[1]
        keep, ptr = _field_ptr(field, n_steps, nd)
    _check(load().sop_step(plan, int(n_steps), float(dt), ptr))
    del keep


def sop_step_host(plan: int, psi_host, n_steps: int, dt: float, field=None, ndim: Optional[int] = None) -> None:
    """Copy a host tensor/array in, step, copy it back (synchronous)."""
    if hasattr(psi_host, "data_ptr"):
        if psi_host.is_cuda or not psi_host.is_contiguous():
            raise ValueError("psi_host must be a contiguous CPU tensor")
        hptr = psi_host.data_ptr()
    else:
        if not psi_host.flags["C_CONTIGUOUS"]:
            raise ValueError("psi_host must be C-contiguous")
        hptr = psi_host.ctypes.data
    keep, ptr = (None, None)
    if field is not None:
        nd = ndim if ndim is not None else np.asarray(field).reshape(int(n_steps), -1).shape[1]
        keep, ptr = _field_ptr(field, n_steps, nd)
    _check(load().sop_step_host(plan, hptr, int(n_steps), float(dt), ptr))
    del keep


def sop_norm(plan: int) -> float:
    out = ctypes.c_double()
    _check(load().sop_norm(plan, ctypes.byref(out)))
    return out.value


def sop_energy(plan: int) -> float:
    out = ctypes.c_double()
    _check(load().sop_energy(plan, ctypes.byref(out)))
    return out.value


def sop_profile_enable(plan: int, every: int = 1) -> None:
    """every = 0: off; 1: time every kernel; k > 1: time the passes of one
    split step in k (and every table set-up kernel)."""
    _check(load().sop_profile_enable(plan, int(every)))


def sop_profile_read(plan: int):
    """Returns (ms per pass class, launches per pass class) and resets them."""
    ms = (ctypes.c_double * SOP_PASS_CLASSES)()
    n = (ctypes.c_int64 * SOP_PASS_CLASSES)()
    _check(load().sop_profile_read(plan, ms, n, SOP_PASS_CLASSES))
    return list(ms), list(n)


def sop_launch_counter(plan: int) -> int:
    return int(load().sop_launch_counter(plan))


SOP_PASS_SHAPES = 8


def sop_autotune(plan: int, dt: float, trial_steps: int = 16):
    """Time every launch shape of the plan's pencil passes on a scratch copy
    of the state and keep the fastest; returns [contiguous, strided] shape."""
    lib = load()
    fn = lib.sop_autotune
    fn.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    fn.restype = ctypes.c_int
    chosen = (ctypes.c_int * 2)()
    _check(fn(plan, float(dt), int(trial_steps), chosen))
    return [int(chosen[0]), int(chosen[1])]


def sop_set_pass_shape(plan: int, axis_kind: int, shape: int) -> None:
    """Force launch shape ``shape`` for the contiguous (0) or strided (1) passes."""
    lib = load()
    fn = lib.sop_set_pass_shape
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    fn.restype = ctypes.c_int
    _check(fn(plan, int(axis_kind), int(shape)))


def sop_fma_peak(f64: bool = True, stream=None) -> float:
    """Measured FMA throughput of the current device in flop/s (FP64 or FP32)."""
    lib = load()
    fn = lib.sop_fma_peak
    fn.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    out = ctypes.c_double()
    _check(fn(1 if f64 else 0, ctypes.byref(out), _stream_handle(stream)))
    return out.value


def sop_debug_check_canaries() -> int:
    """Check builds: the number of overwritten canaries after device buffers
    (SopError SOP_EUNSUPPORTED in a normal build)."""
    lib = load()
    fn = lib.sop_debug_check_canaries
    fn.argtypes = [ctypes.POINTER(ctypes.c_int64)]
    fn.restype = ctypes.c_int
    bad = ctypes.c_int64(0)
    _check(fn(ctypes.byref(bad)))
    return int(bad.value)


def sop_debug_fail_alloc(after: int) -> None:
    """Make the device allocation after `after` more successful ones fail (-1: off)."""
    lib = load()
    fn = lib.sop_debug_fail_alloc
    fn.argtypes = [ctypes.c_int64]
    fn.restype = ctypes.c_int
    _check(fn(int(after)))


def sop_set_wait_limit(plan: int, wait_ns: int) -> None:
    """Limit of the pass kernels' tile-copy waits in ns (0: the default 2 s)."""
    lib = load()
    fn = lib.sop_set_wait_limit
    fn.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    fn.restype = ctypes.c_int
    _check(fn(plan, int(wait_ns)))


def _check_noalloc_tensors(psi, n_values: int, dtype: int, out) -> None:
    """Reject tensors the kernel would read or write out of bounds."""
    import torch
    if not isinstance(psi, int):
        want = {SOP_C64: torch.complex64, SOP_C128: torch.complex128}.get(int(dtype))
        if not (isinstance(psi, torch.Tensor) and psi.is_cuda and psi.is_contiguous()):
            raise ValueError("psi must be a contiguous CUDA tensor (or a raw device pointer)")
        if want is None or psi.dtype != want:
            raise ValueError(f"psi has dtype {psi.dtype}, which does not match dtype={dtype}")
        if psi.numel() < int(n_values):
            raise ValueError(f"psi holds {psi.numel()} values, fewer than n_values={n_values}")
    if not isinstance(out, int):
        if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64 and out.numel() >= 1):
            raise ValueError("out must be a float64 CUDA tensor with at least one element (or a raw pointer)")


def sop_norm_noalloc(psi, n_values: int, dtype: int, scale: float, out, stream=None) -> None:
    """Asynchronous norm without device allocation: writes scale * sum |psi|^2
    into the one-element float64 CUDA tensor ``out``.  ``psi`` is a CUDA
    tensor or a raw device pointer holding n_values complex values; tensors
    are checked for device, layout, dtype and size first."""
    lib = load()
    fn = lib.sop_norm_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    _check_noalloc_tensors(psi, n_values, dtype, out)
    ptr = psi if isinstance(psi, int) else psi.data_ptr()
    optr = out if isinstance(out, int) else out.data_ptr()
    _check(fn(ptr, int(n_values), int(dtype), float(scale), optr, _stream_handle(stream)))


def sop_adjoint_gradient(plan: int, phi, n_steps: int, dt: float, field, every: int, ndim: int,
                         grad_V=None):
    """J, dJ/dfield (numpy, n_steps x ndim) and, into the CUDA float64 tensor
    grad_V (one value per lattice point) when given, dJ/dV; see include/sop.h."""
    lib = load()
    fn = lib.sop_adjoint_gradient
    vp, i64, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    fn.argtypes = [vp, vp, i64, d, vp, i64, ctypes.POINTER(d), vp, vp]
    fn.restype = ctypes.c_int
    if not phi.is_cuda or not phi.is_contiguous():
        raise ValueError("phi must be a contiguous CUDA tensor")
    keep, fptr = (None, None) if field is None else _field_ptr(field, n_steps, ndim)
    g = np.zeros((int(n_steps), ndim), dtype=np.float64)
    J = d()
    gv = None
    if grad_V is not None:
        if not grad_V.is_cuda or not grad_V.is_contiguous():
            raise ValueError("grad_V must be a contiguous CUDA tensor")
        gv = grad_V.data_ptr()
    _check(fn(plan, phi.data_ptr(), int(n_steps), float(dt), fptr, int(every), ctypes.byref(J), g.ctypes.data, gv))
    del keep
    return J.value, g


SOP_GAUGE_LENGTH = 0
SOP_GAUGE_VELOCITY = 1


def sop_set_gauge(plan: int, gauge: int) -> None:
    """Field samples of a Schroedinger plan: E (length gauge, the default) or
    A (velocity gauge, Eq. 13)."""
    lib = load()
    lib.sop_set_gauge.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.sop_set_gauge.restype = ctypes.c_int
    _check(lib.sop_set_gauge(plan, int(gauge)))


def sop_set_field_profile(plan: int, along_x1: bool) -> None:
    """Dirac plans: field samples per lattice column of axis 0, A(x_1, t)."""
    lib = load()
    lib.sop_set_field_profile.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.sop_set_field_profile.restype = ctypes.c_int
    _check(lib.sop_set_field_profile(plan, 1 if along_x1 else 0))


SOP_SPECTRAL_MAX_EIGEN = 16


def sop_spectral(plan: int, n_steps: int, dt: float, energies=None, psiE=None):
    """Spectral method from the bound (trial) state: returns (chi [n_steps+1],
    spectrum [len(energies)]) as complex128 numpy arrays and, into the CUDA
    complex128 tensor psiE of shape (len(energies), ...state shape) when given,
    the eigenfunctions Psi_E; the bound state ends at psi_N.  See include/sop.h."""
    lib = load()
    fn = lib.sop_spectral
    vp, d = ctypes.c_void_p, ctypes.c_double
    fn.argtypes = [vp, ctypes.c_int64, d, ctypes.c_int, vp, vp, vp, vp]
    fn.restype = ctypes.c_int
    E = np.ascontiguousarray(np.atleast_1d(np.asarray([] if energies is None else energies, dtype=np.float64)))
    chi = np.zeros(2 * (int(n_steps) + 1), dtype=np.float64)
    spec = np.zeros(max(1, 2 * len(E)), dtype=np.float64)
    pp = None
    if psiE is not None:
        import torch
        if not psiE.is_cuda or not psiE.is_contiguous() or psiE.dtype != torch.complex128:
            raise ValueError("psiE must be a contiguous complex128 CUDA tensor")
        pp = psiE.data_ptr()
    _check(fn(plan, int(n_steps), float(dt), len(E), E.ctypes.data if len(E) else None, chi.ctypes.data,
              spec.ctypes.data, pp))
    return chi.view(np.complex128), spec[:2 * len(E)].view(np.complex128)


def sop_batch_create(plans) -> int:
    """A batch over plan handles (two-dimensional Schroedinger, one dtype and stream)."""
    lib = load()
    fn = lib.sop_batch_create
    fn.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    fn.restype = ctypes.c_int
    arr = (ctypes.c_void_p * len(plans))(*plans)
    out = ctypes.c_void_p()
    _check(fn(ctypes.byref(out), len(plans), arr))
    return out.value


def sop_batch_step(batch: int, n_steps: int, dt: float, fields=None, ndim: int = 2) -> None:
    """Asynchronous lockstep steps of every plan; fields: None or a list with
    one entry (n_steps x ndim samples or None) per plan."""
    lib = load()
    fn = lib.sop_batch_step
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    keep, arr = [], None
    if fields is not None:
        ptrs = []
        for f in fields:
            if f is None:
                ptrs.append(None)
            else:
                k, ptr = _field_ptr(f, n_steps, ndim)
                keep.append(k)
                ptrs.append(ptr)
        arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
    _check(fn(batch, int(n_steps), float(dt), arr))
    del keep


def sop_batch_destroy(batch: int) -> None:
    lib = load()
    lib.sop_batch_destroy.argtypes = [ctypes.c_void_p]
    lib.sop_batch_destroy.restype = ctypes.c_int
    _check(lib.sop_batch_destroy(batch))


class Batch:
    """Several Propagators advanced together by sop_batch_step."""

    def __init__(self, props):
        self.props = list(props)
        self.handle = sop_batch_create([p.plan for p in self.props])

    def step(self, n_steps: int, dt: float, fields=None) -> None:
        sop_batch_step(self.handle, n_steps, dt, fields, 2)

    def close(self) -> None:
        if getattr(self, "handle", None):
            sop_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Propagator:
    """A plan plus its bound torch state.

    >>> prop = Propagator(dims=(2048, 2048), spacing=(h, h), dtype="c64")
    >>> prop.state.copy_(psi0); prop.set_potential(V)
    >>> prop.step(5000, 0.02, field)        # asynchronous
    >>> prop.norm(), prop.energy()
    """

    def __init__(self, dims: Sequence[int], spacing: Sequence[float], components: int = 1,
                 dtype: str = "c64", params: Optional[dict] = None, stream=None, device=None):
        import torch
        self.dims = tuple(int(x) for x in dims)
        self.ndim = len(self.dims)
        self.components = int(components)
        self.dtype = dtype
        tdt = {"c64": torch.complex64, "c128": torch.complex128}[dtype]
        shape = self.dims[::-1]
        if self.components > 1:
            shape = (self.components,) + shape
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.state = torch.zeros(shape, dtype=tdt, device=dev)
        self.plan = sop_plan_create(self.dims, spacing, components, SOP_C64 if dtype == "c64" else SOP_C128,
                                    params, stream)
        sop_bind_state(self.plan, self.state)

    def set_state(self, psi) -> None:
        import torch
        self.state.copy_(torch.as_tensor(psi).to(self.state.dtype))

    def set_potential(self, V) -> None:
        import torch
        Vt = torch.as_tensor(np.ascontiguousarray(V) if isinstance(V, np.ndarray) else V)
        if Vt.dtype not in (torch.float32, torch.float64):
            Vt = Vt.double()
        sop_set_potential(self.plan, Vt.to(self.state.device).contiguous())

    def set_gauge(self, gauge: str) -> None:
        """"length" (field samples are E) or "velocity" (field samples are A)."""
        if gauge not in ("length", "velocity"):
            raise ValueError("gauge must be 'length' or 'velocity'")
        sop_set_gauge(self.plan, SOP_GAUGE_LENGTH if gauge == "length" else SOP_GAUGE_VELOCITY)

    def set_field_profile(self, along_x1: bool) -> None:
        """Dirac: field samples of shape (n_steps, n_x, ndim), A per column of x_1."""
        sop_set_field_profile(self.plan, along_x1)
        self.profile = bool(along_x1)

    def step(self, n_steps: int, dt: float, field=None) -> None:
        row = self.ndim * (self.dims[0] if getattr(self, "profile", False) else 1)
        sop_step(self.plan, n_steps, dt, field, row)

    def step_host(self, psi_host, n_steps: int, dt: float, field=None) -> None:
        sop_step_host(self.plan, psi_host, n_steps, dt, field, self.ndim)

    def autotune(self, dt: float, trial_steps: int = 16):
        """Pick the fastest launch shape of each pass kind (results are
        bit-identical across shapes); returns [contiguous, strided]."""
        return sop_autotune(self.plan, dt, trial_steps)

    def set_pass_shape(self, axis_kind: int, shape: int) -> None:
        sop_set_pass_shape(self.plan, axis_kind, shape)

    def norm(self) -> float:
        return sop_norm(self.plan)

    def energy(self) -> float:
        return sop_energy(self.plan)

    def adjoint_gradient(self, phi, n_steps: int, dt: float, field=None, every: int = 20, grad_V=None):
        """J = |<phi|psi_N>|^2 from the current state, dJ/dfield and (into
        grad_V) dJ/dV; the state is left unchanged."""
        import torch
        phi_t = torch.as_tensor(phi).to(self.state.device, self.state.dtype).contiguous()
        return sop_adjoint_gradient(self.plan, phi_t, n_steps, dt, field, every, self.ndim, grad_V)

    def spectral(self, n_steps: int, dt: float, energies=None, eigenfunctions: bool = False):
        """chi, spectrum (numpy complex128) and, with eigenfunctions=True, a
        CUDA complex128 tensor of Psi_E per energy; the state ends at psi_N."""
        import torch
        psiE = None
        if eigenfunctions:
            n = len(np.atleast_1d(energies))
            psiE = torch.zeros((n,) + tuple(self.state.shape), dtype=torch.complex128, device=self.state.device)
        chi, spec = sop_spectral(self.plan, n_steps, dt, energies, psiE)
        return chi, spec, psiE

    def close(self) -> None:
        if getattr(self, "plan", None):
            sop_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

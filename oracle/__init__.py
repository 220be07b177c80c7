"""FP64 CPU oracle for the Fourier split-operator step (test infrastructure).

This package is test infrastructure, not product code.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` import it.  The GPU library never imports, links or calls it.

It wraps ``sop_oracle.c`` (plain C, FP64, its own radix-2/3 FFT) through
ctypes.  Arrays follow NumPy C order with x fastest: a 2D field has shape
``(ny, nx)``, a Dirac spinor ``(4, ny, nx)``; ``dims`` in the C calls are
``(nx, ny, nz)``, i.e. the reversed NumPy shape.

Every function cites the passage of Bauke & Keitel (arXiv:1012.3911) it
follows; the C source states each formula.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sop_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``sop_oracle.c`` into ``_build/liboracle.so`` with gcc/OpenMP."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        d = ctypes.c_double
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_get_threads.restype = ctypes.c_int
        lib.orc_max_threads.restype = ctypes.c_int
        lib.orc_size_ok.argtypes = [ctypes.c_int64]
        lib.orc_size_ok.restype = ctypes.c_int
        lib.orc_dft_naive.argtypes = [P, P, ctypes.c_int64, ctypes.c_int]
        lib.orc_fft.argtypes = [P, ctypes.c_int64, ctypes.c_int]
        lib.orc_fft.restype = ctypes.c_int
        lib.orc_fftn.argtypes = [P, ctypes.c_int, i64p, ctypes.c_int]
        lib.orc_fftn.restype = ctypes.c_int
        lib.orc_schr_propagate.argtypes = [P, P, ctypes.c_int, i64p, dp, d, d, d, d,
                                           ctypes.c_int64, P]
        lib.orc_schr_propagate.restype = ctypes.c_int
        lib.orc_schr_propagate_gauge.argtypes = [P, P, ctypes.c_int, i64p, dp, d, d, d, d,
                                                 ctypes.c_int64, P, ctypes.c_int]
        lib.orc_schr_propagate_gauge.restype = ctypes.c_int
        lib.orc_dirac_propagate.argtypes = [P, P, ctypes.c_int, i64p, dp, d, d, d, d, d,
                                            ctypes.c_int64, P]
        lib.orc_dirac_propagate.restype = ctypes.c_int
        lib.orc_dirac_alpha_beta.argtypes = [P]
        lib.orc_dirac_u.argtypes = [dp, ctypes.c_int, d, d, P]
        lib.orc_dirac_propagate_profile.argtypes = [P, P, ctypes.c_int, i64p, dp, d, d, d, d, d,
                                                    ctypes.c_int64, P]
        lib.orc_dirac_propagate_profile.restype = ctypes.c_int
        lib.orc_dirac1d_u.argtypes = [d, d, d, P]
        lib.orc_dirac1d_h.argtypes = [d, d, d, P]
        lib.orc_dirac1d_propagate.argtypes = [P, P, ctypes.c_int64, d, d, d, d, d, d, ctypes.c_int64, P]
        lib.orc_dirac1d_propagate.restype = ctypes.c_int
        lib.orc_dirac_h.argtypes = [dp, ctypes.c_int, d, d, P]
        lib.orc_dirac_kinetic_matrix.argtypes = [dp, ctypes.c_int, d, d, d, d, P]
        lib.orc_dirac_mixing_matrix.argtypes = [dp, ctypes.c_int, d, d, d, d, d, P]
        lib.orc_norm.argtypes = [P, ctypes.c_int, i64p, dp, ctypes.c_int]
        lib.orc_norm.restype = d
        lib.orc_energy.argtypes = [P, P, ctypes.c_int, i64p, dp, ctypes.c_int, d, d, d]
        lib.orc_energy.restype = d
        lib.orc_set_threads(0)
        _lib = lib
        return lib


class _swap_library:
    """Context manager that points this module at another build of
    ``sop_oracle.c`` (the tests use it to plant mistakes in a copy of the
    oracle and check that the pins catch them)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        real = _load()
        self._saved = real
        lib = ctypes.CDLL(self.path)
        for name in dir(real):
            if name.startswith("orc_"):
                f, g = getattr(real, name), getattr(lib, name)
                g.argtypes, g.restype = f.argtypes, f.restype
        lib.orc_set_threads(real.orc_get_threads())
        with _lock:
            _lib = lib
        return lib

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self._saved
        return False


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _dims(shape) -> ctypes.Array:
    rev = tuple(int(s) for s in shape)[::-1]
    return (ctypes.c_int64 * len(rev))(*rev)


def _dp(vals) -> ctypes.Array:
    vals = [float(v) for v in vals]
    return (ctypes.c_double * max(1, len(vals)))(*vals)


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle uses (0 or 1: one thread)."""
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def max_threads() -> int:
    return int(_load().orc_max_threads())


def size_ok(n: int) -> bool:
    """True if n = 2^a 3^b (the sizes the oracle's radix-2/3 FFT handles)."""
    return bool(_load().orc_size_ok(int(n)))


def dft_naive(x, sign: int = -1) -> np.ndarray:
    """O(n^2) DFT by definition, X_k = sum_j x_j exp(sign 2 pi i jk/n) (Sec. 2.1)."""
    x = _c128(x).ravel()
    out = np.empty_like(x)
    _load().orc_dft_naive(x.ctypes.data, out.ctypes.data, x.size, int(sign))
    return out


def fft(x, sign: int = -1) -> np.ndarray:
    """The oracle's own radix-2/3 FFT of a 1D array (unscaled in both directions)."""
    y = _c128(x).ravel().copy()
    if _load().orc_fft(y.ctypes.data, y.size, int(sign)) != 0:
        raise ValueError(f"size {y.size} is not 2^a 3^b")
    return y


def fftn(x, sign: int = -1) -> np.ndarray:
    """Separable d-dimensional DFT over all axes of ``x``; the inverse
    (sign=+1) includes 1/N."""
    y = _c128(x).copy()
    if _load().orc_fftn(y.ctypes.data, y.ndim, _dims(y.shape), int(sign)) != 0:
        raise ValueError(f"shape {y.shape} has a side that is not 2^a 3^b")
    return y


def schrodinger_propagate(psi, V, spacing, dt: float, n_steps: int, field=None,
                          mass: float = 1.0, charge: float = -1.0,
                          hbar: float = 1.0, gauge: str = "length") -> np.ndarray:
    """``n_steps`` Strang steps of Eq. 8 with the Schroedinger split of
    Eqs. 10a/10b.  ``psi`` has shape (…, ny, nx); ``V`` the same spatial
    shape (potential energy) or None; ``spacing`` is (h_x, h_y, h_z) in axis
    order; ``field`` is (n_steps, ndim) samples at step midpoints, components
    in axis order, or None: the electric field E (``gauge="length"``, in the
    real-space factor) or the vector potential A (``gauge="velocity"``, in the
    momentum-space factor of Eq. 13).  Returns the propagated copy."""
    y = _c128(psi).copy()
    ndim = y.ndim
    Vp = None
    if V is not None:
        Vc = _f64(V)
        if Vc.shape != y.shape:
            raise ValueError("V must have the shape of psi")
        Vp = Vc.ctypes.data
    fp = None
    if field is not None:
        fc = _f64(field).reshape(int(n_steps), ndim)
        fp = fc.ctypes.data
    if gauge not in ("length", "velocity"):
        raise ValueError("gauge must be 'length' or 'velocity'")
    rc = _load().orc_schr_propagate_gauge(y.ctypes.data, Vp, ndim, _dims(y.shape), _dp(spacing),
                                          mass, charge, hbar, float(dt), int(n_steps), fp,
                                          0 if gauge == "length" else 1)
    if rc != 0:
        raise ValueError("unsupported shape")
    return y


def dirac_propagate(psi, V, spacing, dt: float, n_steps: int, field=None,
                    mass: float = 1.0, charge: float = -1.0, hbar: float = 1.0,
                    c: float = 137.036) -> np.ndarray:
    """``n_steps`` Strang steps of Eq. 8 with the Dirac split of
    Eqs. 18a/18b for a four-component spinor of shape (4, …, ny, nx) in 2D or
    3D.  ``field`` holds vector-potential samples (n_steps, ndim) at step
    midpoints, or None.  Returns the propagated copy."""
    y = _c128(psi).copy()
    if y.shape[0] != 4:
        raise ValueError("Dirac spinor needs 4 components on axis 0")
    sp = y.shape[1:]
    ndim = len(sp)
    Vp = None
    if V is not None:
        Vc = _f64(V)
        if Vc.shape != sp:
            raise ValueError("V must have the spatial shape of psi")
        Vp = Vc.ctypes.data
    fp = None
    if field is not None:
        fc = _f64(field).reshape(int(n_steps), ndim)
        fp = fc.ctypes.data
    rc = _load().orc_dirac_propagate(y.ctypes.data, Vp, ndim, _dims(sp), _dp(spacing), mass,
                                     charge, hbar, c, float(dt), int(n_steps), fp)
    if rc != 0:
        raise ValueError("unsupported shape")
    return y


def dirac_propagate_profile(psi, V, spacing, dt: float, n_steps: int, field,
                            mass: float = 1.0, charge: float = -1.0, hbar: float = 1.0,
                            c: float = 137.036) -> np.ndarray:
    """As dirac_propagate, for a vector potential that varies along x_1:
    ``field`` has shape (n_steps, n_x, ndim), A at each step midpoint and
    lattice column of axis 0 (the mixing of Eq. 26 per column)."""
    y = _c128(psi).copy()
    if y.shape[0] != 4:
        raise ValueError("Dirac spinor needs 4 components on axis 0")
    sp = y.shape[1:]
    ndim = len(sp)
    Vp = None
    if V is not None:
        Vc = _f64(V)
        if Vc.shape != sp:
            raise ValueError("V must have the spatial shape of psi")
        Vp = Vc.ctypes.data
    fc = _f64(field).reshape(int(n_steps), sp[-1], ndim)
    rc = _load().orc_dirac_propagate_profile(y.ctypes.data, Vp, ndim, _dims(sp), _dp(spacing), mass,
                                             charge, hbar, c, float(dt), int(n_steps), fc.ctypes.data)
    if rc != 0:
        raise ValueError("unsupported shape")
    return y


def dirac1d_propagate(psi, V, spacing, dt: float, n_steps: int, field=None,
                      mass: float = 1.0, charge: float = -1.0, hbar: float = 1.0,
                      c: float = 137.036) -> np.ndarray:
    """``n_steps`` Strang steps of the one-dimensional two-component Dirac
    equation (end of Sec. 2.3; alpha_1 = sigma_x, beta = sigma_z) for a spinor
    of shape (2, n).  ``field`` holds vector-potential samples A_1 (n_steps,)
    at step midpoints, or None.  Returns the propagated copy."""
    y = _c128(psi).copy()
    if y.ndim != 2 or y.shape[0] != 2:
        raise ValueError("1D Dirac spinor needs shape (2, n)")
    n = y.shape[1]
    Vp = None
    if V is not None:
        Vc = _f64(V)
        if Vc.shape != (n,):
            raise ValueError("V must have shape (n,)")
        Vp = Vc.ctypes.data
    fp = None
    if field is not None:
        fc = _f64(field).reshape(int(n_steps))
        fp = fc.ctypes.data
    h = float(spacing[0]) if np.ndim(spacing) else float(spacing)
    rc = _load().orc_dirac1d_propagate(y.ctypes.data, Vp, n, h, mass, charge, hbar, c, float(dt),
                                       int(n_steps), fp)
    if rc != 0:
        raise ValueError("unsupported shape")
    return y


def dirac1d_u(p: float, mass: float = 1.0, c: float = 137.036) -> np.ndarray:
    """The 2x2 u(p) of the 1D Dirac split (Eq. 30's form)."""
    out = np.empty(4, dtype=np.complex128)
    _load().orc_dirac1d_u(float(p), mass, c, out.ctypes.data)
    return out.reshape(2, 2)


def dirac1d_h(p: float, mass: float = 1.0, c: float = 137.036) -> np.ndarray:
    """c alpha_1 p + m c^2 beta with alpha_1 = sigma_x, beta = sigma_z."""
    out = np.empty(4, dtype=np.complex128)
    _load().orc_dirac1d_h(float(p), mass, c, out.ctypes.data)
    return out.reshape(2, 2)


def alpha_beta():
    """alpha_1..3 and beta of the Dirac representation (Eq. 16)."""
    out = np.empty(64, dtype=np.complex128)
    _load().orc_dirac_alpha_beta(out.ctypes.data)
    m = out.reshape(4, 4, 4)
    return m[0], m[1], m[2], m[3]


def dirac_u(p, mass: float = 1.0, c: float = 137.036) -> np.ndarray:
    """u(p) of Eq. 30 built from d_+- of Eq. 29."""
    p = [float(v) for v in p]
    out = np.empty(16, dtype=np.complex128)
    _load().orc_dirac_u(_dp(p), len(p), mass, c, out.ctypes.data)
    return out.reshape(4, 4)


def dirac_h(p, mass: float = 1.0, c: float = 137.036) -> np.ndarray:
    """c alpha.p + m c^2 beta (Eq. 28)."""
    p = [float(v) for v in p]
    out = np.empty(16, dtype=np.complex128)
    _load().orc_dirac_h(_dp(p), len(p), mass, c, out.ctypes.data)
    return out.reshape(4, 4)


def dirac_kinetic_matrix(p, tau: float, mass: float = 1.0, c: float = 137.036,
                         hbar: float = 1.0) -> np.ndarray:
    """u^dagger diag(e^{-iE tau}, e^{-iE tau}, e^{iE tau}, e^{iE tau}) u (Eq. 33)."""
    p = [float(v) for v in p]
    out = np.empty(16, dtype=np.complex128)
    _load().orc_dirac_kinetic_matrix(_dp(p), len(p), mass, c, hbar, float(tau), out.ctypes.data)
    return out.reshape(4, 4)


def dirac_mixing_matrix(A, tau: float, delta: float = 0.5, charge: float = -1.0,
                        c: float = 137.036, hbar: float = 1.0) -> np.ndarray:
    """Real-space factor U_A1,2 of Eq. 26 for a uniform vector potential A."""
    A = [float(v) for v in A]
    out = np.empty(16, dtype=np.complex128)
    _load().orc_dirac_mixing_matrix(_dp(A), len(A), charge, c, hbar, float(tau), float(delta),
                                    out.ctypes.data)
    return out.reshape(4, 4)


def norm(psi, spacing, comps: int = 1) -> float:
    """dV sum |psi|^2 over all points and components (compensated sum)."""
    y = _c128(psi)
    sp = y.shape[1:] if comps > 1 else y.shape
    return float(_load().orc_norm(y.ctypes.data, len(sp), _dims(sp), _dp(spacing), comps))


def energy(psi, V, spacing, comps: int = 1, mass: float = 1.0, hbar: float = 1.0,
           c: float = 137.036) -> float:
    """Field-free energy <T> + <V>; T = p^2/2m (comps=1) or the free Dirac
    Hamiltonian of Eq. 28 (comps=4 in 2D/3D, comps=2 in 1D with
    alpha_1 = sigma_x, beta = sigma_z)."""
    y = _c128(psi)
    sp = y.shape[1:] if comps > 1 else y.shape
    Vp = None
    if V is not None:
        Vc = _f64(V)
        Vp = Vc.ctypes.data
    return float(_load().orc_energy(y.ctypes.data, Vp, len(sp), _dims(sp), _dp(spacing), comps,
                                    mass, hbar, c))

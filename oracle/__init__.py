"""CPU oracle for the staggered Dslash / even-odd CG path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never loads it and
shares no code with it.

The arithmetic lives in ``stag_oracle.c`` (plain C, double complex, sequential
sums, built with ``-ffp-contract=off``); this module compiles it on demand with
gcc and wraps it with ctypes.  ``encodings`` holds the reduced-precision storage
encodings (float32 rounding, the FP16 per-site-norm spinor code) written in
numpy, used to state what the reduced-precision kernels must compute.

Every function here takes and returns arrays in the canonical layout of
``lattice_inputs``: links (V,4,3,3), full fields (V,3), half fields (V/2,3),
complex128.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stag_oracle.c")
_LIB = os.path.join(_HERE, "libstag_oracle.so")
_LIB_OMP = os.path.join(_HERE, "libstag_oracle_omp.so")
_lock = threading.Lock()
_libs = {}
_threaded = False

STATUS = {0: "converged", 1: "not converged", 2: "breakdown"}


def _compile(out, extra):
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", *extra,
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile the oracle shared libraries with gcc (portable flags, no -march):
    the single-threaded parity build and an OpenMP build used only to time the
    oracle on every host core (identical results: see stag_oracle.c)."""
    if force:
        for p in (_LIB, _LIB_OMP):
            if os.path.exists(p):
                os.remove(p)
    _compile(_LIB, [])
    _compile(_LIB_OMP, ["-fopenmp"])
    return _LIB


class threads:
    """Context manager: oracle calls inside it use the OpenMP build (timing only).

        with oracle.threads():
            oracle.cg(...)
    """

    def __enter__(self):
        global _threaded
        self._prev, _threaded = _threaded, True
        return self

    def __exit__(self, *exc):
        global _threaded
        _threaded = self._prev


def num_threads() -> int:
    """Threads the OpenMP build's site loops use (1 for the parity build)."""
    return int(_load().orc_num_threads())


def _load():
    key = "omp" if _threaded else "serial"
    with _lock:
        if key not in _libs:
            build()
            lib = ctypes.CDLL(_LIB_OMP if key == "omp" else _LIB)
            P = ctypes.c_void_p
            I4 = ctypes.POINTER(ctypes.c_int)
            lib.orc_check_dims.argtypes = [I4]
            lib.orc_volume.argtypes = [I4]
            lib.orc_volume.restype = ctypes.c_long
            lib.orc_eta.argtypes = [I4, I4, ctypes.c_int]
            lib.orc_dslash_full.argtypes = [I4, P, P, P]
            lib.orc_dslash_half.argtypes = [I4, P, ctypes.c_int, P, P]
            lib.orc_apply_M.argtypes = [I4, P, ctypes.c_double, P, P]
            lib.orc_cg.argtypes = [I4, P, ctypes.c_double, P, P, ctypes.c_double, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
            lib.orc_multishift_cg.argtypes = [I4, P, ctypes.c_double, ctypes.c_int, P, P, P,
                                              ctypes.c_double, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_int), P]
            lib.orc_action.argtypes = [I4, P, P]
            lib.orc_action.restype = ctypes.c_double
            lib.orc_force.argtypes = [I4, P, P, P, P]
            lib.orc_reconstruct_row2.argtypes = [ctypes.c_long, P, P]
            lib.orc_num_threads.restype = ctypes.c_int
            _libs[key] = lib
    return _libs[key]


def _dims(dims):
    d = tuple(int(v) for v in dims)
    if len(d) != 4 or any(v < 2 or v % 2 for v in d):
        raise ValueError(f"lattice extents must be four even integers >= 2, got {d}")
    return (ctypes.c_int * 4)(*d)


def _c128(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if shape is not None and a.shape != tuple(shape):
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def volume(dims) -> int:
    d = _dims(dims)
    return int(_load().orc_volume(d))


def eta(dims, coord, mu: int) -> int:
    """Kogut-Susskind phase eta_mu(x) (no boundary sign)."""
    c = (ctypes.c_int * 4)(*[int(v) for v in coord])
    return int(_load().orc_eta(_dims(dims), c, int(mu)))


def dslash_full(dims, U, phi):
    """D phi on the full lattice, Eq. (staggered) of Sec. 4.2."""
    V = volume(dims)
    U = _c128(U, (V, 4, 3, 3))
    phi = _c128(phi, (V, 3))
    out = np.empty((V, 3), np.complex128)
    rc = _load().orc_dslash_full(_dims(dims), _ptr(U), _ptr(phi), _ptr(out))
    if rc:
        raise ValueError("orc_dslash_full failed")
    return out


def dslash_half(dims, U, psi, out_parity: int):
    """D restricted to output parity ``out_parity`` (0: D_eo, 1: D_oe)."""
    V = volume(dims)
    U = _c128(U, (V, 4, 3, 3))
    psi = _c128(psi, (V // 2, 3))
    out = np.empty((V // 2, 3), np.complex128)
    rc = _load().orc_dslash_half(_dims(dims), _ptr(U), int(out_parity), _ptr(psi), _ptr(out))
    if rc:
        raise ValueError("orc_dslash_half failed")
    return out


def dslash_eo(dims, U, psi_odd):
    return dslash_half(dims, U, psi_odd, 0)


def dslash_oe(dims, U, psi_even):
    return dslash_half(dims, U, psi_even, 1)


def apply_M(dims, U, mass: float, psi_even):
    """M psi = m^2 psi - D_eo D_oe psi on even sites."""
    V = volume(dims)
    U = _c128(U, (V, 4, 3, 3))
    psi = _c128(psi_even, (V // 2, 3))
    out = np.empty((V // 2, 3), np.complex128)
    rc = _load().orc_apply_M(_dims(dims), _ptr(U), float(mass), _ptr(psi), _ptr(out))
    if rc:
        raise ValueError("orc_apply_M failed")
    return out


def cg(dims, U, mass: float, b_even, tol: float = 1e-10, maxiter: int = 100000):
    """Solve M x = b by CG; returns (x, iterations, true relative residual, status)."""
    V = volume(dims)
    U = _c128(U, (V, 4, 3, 3))
    b = _c128(b_even, (V // 2, 3))
    x = np.empty_like(b)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = _load().orc_cg(_dims(dims), _ptr(U), float(mass), _ptr(b), _ptr(x), float(tol),
                        int(maxiter), ctypes.byref(it), ctypes.byref(rr))
    if st < 0:
        raise ValueError("orc_cg failed")
    return x, it.value, rr.value, st


def multishift_cg(dims, U, mass: float, shifts, b_even, tol: float = 1e-10, maxiter: int = 100000):
    """Solve (M + shifts[i]) x_i = b for all i; returns (X, iterations, relres[], status)."""
    V = volume(dims)
    U = _c128(U, (V, 4, 3, 3))
    b = _c128(b_even, (V // 2, 3))
    sh = np.ascontiguousarray(shifts, dtype=np.float64)
    X = np.empty((len(sh), V // 2, 3), np.complex128)
    rel = np.empty(len(sh), np.float64)
    it = ctypes.c_int(0)
    st = _load().orc_multishift_cg(_dims(dims), _ptr(U), float(mass), len(sh), _ptr(sh), _ptr(b),
                                   _ptr(X), float(tol), int(maxiter), ctypes.byref(it), _ptr(rel))
    if st < 0:
        raise ValueError("orc_multishift_cg failed")
    return X, it.value, rel, st


def action(dims, phi_even, X_even) -> float:
    """S = Re <phi, X> (with X = M^{-1} phi this is phi^dagger M^{-1} phi)."""
    V = volume(dims)
    phi = _c128(phi_even, (V // 2, 3))
    X = _c128(X_even, (V // 2, 3))
    return float(_load().orc_action(_dims(dims), _ptr(phi), _ptr(X)))


def force(dims, U, X_even):
    """(P, G): projected force TA(U G^dagger) and Euclidean gradient G, both (V,4,3,3)."""
    V = volume(dims)
    U = _c128(U, (V, 4, 3, 3))
    X = _c128(X_even, (V // 2, 3))
    P = np.empty((V, 4, 3, 3), np.complex128)
    G = np.empty((V, 4, 3, 3), np.complex128)
    rc = _load().orc_force(_dims(dims), _ptr(U), _ptr(X), _ptr(P), _ptr(G))
    if rc:
        raise ValueError("orc_force failed")
    return P, G


def reconstruct_row2(mats):
    """Third rows rebuilt from rows 0 and 1 (12-real compression), (n,3)."""
    m = _c128(mats)
    n = m.size // 9
    m = m.reshape(n, 3, 3)
    out = np.empty((n, 3), np.complex128)
    _load().orc_reconstruct_row2(n, _ptr(m), _ptr(out))
    return out


def true_residual(dims, U, mass: float, x_even, b_even, sigma: float = 0.0) -> float:
    """||b - (M + sigma) x|| / ||b|| recomputed in double precision."""
    r = np.asarray(b_even) - apply_M(dims, U, mass, x_even) - sigma * np.asarray(x_even)
    nb = np.linalg.norm(b_even)
    return float(np.linalg.norm(r) / nb) if nb > 0 else 0.0

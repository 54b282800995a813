"""Reduced-precision storage encodings, written plainly in numpy (test infrastructure).

The mixed-precision solvers store links and spinors in float32 or float16.  The
operator they apply is the double-precision one acting on the *stored* values,
so the oracle for a reduced-precision kernel is: encode the inputs here, decode
them back to float64 exactly, and apply the double-precision oracle.  The
rounding decisions are taken in the same precision the kernels use (float32
arithmetic, round-to-nearest-even), so both sides produce identical codes.

* float32 storage: every real component rounded to the nearest float32.
* float16 links: every real component rounded to float32, then to float16
  (SU(3) entries lie in [-1, 1], no scale is needed).
* float16 spinors with a per-site norm: for each site the norm is the largest
  magnitude of its six float32-rounded real components (a float32); the code is
  round_to_half(component / norm) with the division in float32; a site whose
  norm is zero stores zeros.  Decoding multiplies the code by the norm.
* 12-real links: rows 0 and 1 stored, row 2 rebuilt as conj(row0 x row1).
"""

from __future__ import annotations

import numpy as np

from . import reconstruct_row2


def _reals(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a.view(np.float64).reshape(a.shape + (2,))


def _complex(r):
    r = np.ascontiguousarray(r, dtype=np.float64)
    return r.view(np.complex128).reshape(r.shape[:-1])


def round_f32(a):
    """Each real component rounded to float32, returned as complex128."""
    return _complex(_reals(a).astype(np.float32).astype(np.float64))


def round_f16(a):
    """Each real component rounded to float32 and then to float16, as complex128."""
    return _complex(_reals(a).astype(np.float32).astype(np.float16).astype(np.float64))


def encode_half_spinor(psi):
    """(codes float16 (n,6), norms float32 (n,)) for a half field psi (n,3)."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128).reshape(-1, 3)
    r32 = psi.view(np.float64).reshape(-1, 6).astype(np.float32)
    norm = np.max(np.abs(r32), axis=1).astype(np.float32)
    safe = np.where(norm > 0, norm, np.float32(1.0)).astype(np.float32)
    q = (r32 / safe[:, None]).astype(np.float32)
    q = np.where(norm[:, None] > 0, q, np.float32(0.0)).astype(np.float16)
    return q, norm


def decode_half_spinor(codes, norms):
    """Exact float64 value of the stored (codes, norms), as complex128 (n,3)."""
    r = codes.astype(np.float64) * norms.astype(np.float64)[:, None]
    return np.ascontiguousarray(r).view(np.complex128).reshape(-1, 3)


def half_spinor(psi):
    """Round trip of psi through the float16 per-site-norm code."""
    q, n = encode_half_spinor(psi)
    return decode_half_spinor(q, n).reshape(np.shape(psi))


def recon12(U, rounding=None):
    """Links as a 12-real kernel sees them: rows 0,1 (optionally rounded) kept,
    row 2 rebuilt from them in double precision."""
    U = np.ascontiguousarray(U, dtype=np.complex128)
    shape = U.shape
    m = U.reshape(-1, 3, 3).copy()
    if rounding is not None:
        m[:, :2, :] = rounding(m[:, :2, :])
    m[:, 2, :] = reconstruct_row2(m)
    return m.reshape(shape)

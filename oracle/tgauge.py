"""Temporal-gauge transform of a gauge field, plainly in numpy (test infrastructure).

Sec. 4.3 of the paper stores 6 SU(3) matrices per site by fixing the temporal
gauge: the links of the time direction become the identity everywhere except
on one time slice.  The transform that does this is a gauge transformation
built along each time line:

    g(x, t = 0) = 1,        g(x, t + 1) = g(x, t) U_t(x, t),

applied as U'_mu(x) = g(x) U_mu(x) g(x + mu)^dagger to every link and as
psi'(x) = g(x) psi(x) to fields.  For unitary links U'_t(x, t) = 1 for
t < Lt - 1, and on the last slice U'_t(x, Lt - 1) = g(x, Lt - 1) U_t(x, Lt - 1)
(the ordered product of the time links along the line, since g = 1 again at
t = 0).  Gauge covariance gives D[U'] = g D[U] g^dagger, hence
M' = g M g^dagger on even sites.

Nothing here special-cases the identity links: U' is the definition computed
in double, so its time links off the last slice equal 1 only to rounding.
Index conventions are those of ``lattice_inputs``: i = x + Lx (y + Ly (z + Lz t)),
half fields indexed i / 2 over the sites of one parity.
"""

from __future__ import annotations

import numpy as np


def _coords(dims):
    Lx, Ly, Lz, Lt = dims
    i = np.arange(Lx * Ly * Lz * Lt)
    x = i % Lx
    y = (i // Lx) % Ly
    z = (i // (Lx * Ly)) % Lz
    t = i // (Lx * Ly * Lz)
    return x, y, z, t


def _index(dims, x, y, z, t):
    Lx, Ly, Lz, Lt = dims
    return (x % Lx) + Lx * ((y % Ly) + Ly * ((z % Lz) + Lz * (t % Lt)))


def gauge_matrices(dims, U):
    """g per site (V, 3, 3): g = 1 on t = 0, g(t + 1) = g(t) U_t(t) along each time line."""
    Lx, Ly, Lz, Lt = dims
    Vs = Lx * Ly * Lz
    U = np.asarray(U, dtype=np.complex128).reshape(Lx * Ly * Lz * Lt, 4, 3, 3)
    g = np.empty((Lx * Ly * Lz * Lt, 3, 3), dtype=np.complex128)
    g[:Vs] = np.eye(3)
    for t in range(Lt - 1):
        sl = slice(t * Vs, (t + 1) * Vs)
        nx = slice((t + 1) * Vs, (t + 2) * Vs)
        g[nx] = g[sl] @ U[sl, 3]
    return g


def transform_links(dims, U, g):
    """U'_mu(x) = g(x) U_mu(x) g(x + mu)^dagger for every site and direction."""
    U = np.asarray(U, dtype=np.complex128).reshape(-1, 4, 3, 3)
    x, y, z, t = _coords(dims)
    out = np.empty_like(U)
    step = [(1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1)]
    for mu in range(4):
        dx, dy, dz, dt = step[mu]
        fwd = _index(dims, x + dx, y + dy, z + dz, t + dt)
        out[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(g[fwd], 1, 2))
    return out


def temporal_links(dims, U):
    """(g, U') of the temporal gauge of U."""
    g = gauge_matrices(dims, U)
    return g, transform_links(dims, U, g)


def parity_sites(dims, parity):
    """Lexicographic indices of the sites of one parity, in half-field order."""
    x, y, z, t = _coords(dims)
    idx = np.arange(len(x))
    return idx[((x + y + z + t) % 2) == parity]


def apply_to_half(dims, g, psi, parity, dagger=False):
    """g psi (or g^dagger psi) on a half field of the given parity, (V/2, 3) or (n, V/2, 3)."""
    gs = g[parity_sites(dims, parity)]
    if dagger:
        gs = np.conj(np.swapaxes(gs, 1, 2))
    psi = np.asarray(psi, dtype=np.complex128)
    return np.einsum("hab,...hb->...ha", gs, psi)

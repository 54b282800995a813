"""Seeded synthetic inputs for the staggered Dslash / even-odd CG workloads.

This module only draws random numbers and shapes them into the input fields
(gauge links, colour-vector sources, gauge transformations). It holds none of
the operator, solver or force arithmetic: both the CPU oracle and the CUDA
library consume the arrays produced here, so the two paths see bit-identical
inputs.

Canonical host layout (shared by every consumer):

* site index ``i = x + Lx*(y + Ly*(z + Lz*t))`` (lexicographic, x fastest),
  directions ``mu = 0,1,2,3 = x,y,z,t``;
* gauge field ``U``: complex128 array of shape ``(V, 4, 3, 3)``,
  ``U[i, mu, a, b]`` is row ``a``, column ``b`` of ``U_{x,mu}``;
* half field of parity ``p`` (``p = (x+y+z+t) mod 2``): complex128 array of
  shape ``(V//2, 3)`` indexed by ``h = i // 2`` over the sites of that parity
  (valid because ``Lx`` is even, so every pair ``(2k, 2k+1)`` of a row holds one
  site of each parity).

Random draws use numpy's PCG64 (``numpy.random.default_rng(seed)``); seeds for
the standard workloads follow ``seed = 1000 * workload_index + stream`` with
stream 0 = links, 1 = sources, 2 = choice of finite-difference links.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "WORKLOADS",
    "volume",
    "check_dims",
    "haar_su3",
    "smooth_su3",
    "gaussian",
    "random_links",
    "gaussian_half",
    "gaussian_full",
    "random_gauge_transform",
    "unit_links",
    "workload_seed",
    "random_links_torch",
    "gaussian_half_torch",
]


# Standard workloads: (name, dims (Lx, Ly, Lz, Lt), link recipe, eps, mass).
# "haar" = Haar-random SU(3); "smooth" = exp(i*eps*H) with H Gaussian traceless
# Hermitian. Index in this table is the workload index used in the seeds.
WORKLOADS = [
    dict(name="4^4 Haar, m=0.1", dims=(4, 4, 4, 4), links="haar", eps=None, mass=0.1),
    dict(name="32^3x8 smooth eps=0.3, m=0.01", dims=(32, 32, 32, 8), links="smooth", eps=0.3, mass=0.01),
    dict(name="48^3x12 smooth eps=0.2, m=0.002", dims=(48, 48, 48, 12), links="smooth", eps=0.2, mass=0.002),
    dict(name="32^3x16 smooth eps=0.3, m=0.005", dims=(32, 32, 32, 16), links="smooth", eps=0.3, mass=0.005),
    dict(name="24^3x8 smooth eps=0.3, m=0.01", dims=(24, 24, 24, 8), links="smooth", eps=0.3, mass=0.01),
    dict(name="64^3x16 smooth eps=0.3, m=0.01", dims=(64, 64, 64, 16), links="smooth", eps=0.3, mass=0.01),
    # the lattices of the paper's Table 2 (32^4) and Table 1 (48^4)
    dict(name="32^4 smooth eps=0.3, m=0.01", dims=(32, 32, 32, 32), links="smooth", eps=0.3, mass=0.01),
    dict(name="48^4 smooth eps=0.3, m=0.01", dims=(48, 48, 48, 48), links="smooth", eps=0.3, mass=0.01),
]


def workload_seed(index: int, stream: int) -> int:
    """Seed of random stream ``stream`` (0 links, 1 sources, 2 FD links) of workload ``index``."""
    return 1000 * int(index) + int(stream)


def check_dims(dims) -> tuple:
    """Validate lattice extents: four ints, each even and >= 2."""
    dims = tuple(int(d) for d in dims)
    if len(dims) != 4 or any(d < 2 or d % 2 for d in dims):
        raise ValueError(f"lattice extents must be four even integers >= 2, got {dims}")
    return dims


def volume(dims) -> int:
    dims = check_dims(dims)
    return dims[0] * dims[1] * dims[2] * dims[3]


def gaussian(rng: np.random.Generator, shape) -> np.ndarray:
    """Complex Gaussian with unit variance per complex component: (N + iN)/sqrt(2)."""
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im) / np.sqrt(2.0)


def haar_su3(rng: np.random.Generator, n: int) -> np.ndarray:
    """``n`` Haar-random SU(3) matrices, shape (n, 3, 3).

    QR of a complex Gaussian matrix with the phases of R's diagonal moved into
    Q gives a Haar-distributed U(3) element; dividing by the principal cube root
    of its determinant puts it in SU(3).
    """
    z = gaussian(rng, (n, 3, 3))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    return q / (det ** (1.0 / 3.0))[:, None, None]


def smooth_su3(rng: np.random.Generator, n: int, eps: float) -> np.ndarray:
    """``n`` matrices ``exp(i*eps*H)``, H a Gaussian traceless Hermitian 3x3.

    ``A`` complex Gaussian, ``H = (A + A^dagger)/2 - tr(...)/3``; the exponential
    is formed from the eigen-decomposition ``H = V diag(l) V^dagger`` as
    ``V diag(exp(i*eps*l)) V^dagger``, which is unitary with unit determinant up
    to rounding.
    """
    a = gaussian(rng, (n, 3, 3))
    h = 0.5 * (a + np.conj(np.swapaxes(a, 1, 2)))
    tr = np.trace(h, axis1=1, axis2=2).real / 3.0
    h = h - tr[:, None, None] * np.eye(3)[None]
    lam, vec = np.linalg.eigh(h)
    ph = np.exp(1j * eps * lam)
    return np.einsum("nij,nj,nkj->nik", vec, ph, np.conj(vec), optimize=True)


def unit_links(dims) -> np.ndarray:
    """Free field: every link the 3x3 identity."""
    v = volume(dims)
    u = np.zeros((v, 4, 3, 3), dtype=np.complex128)
    u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1.0
    return u


def random_links(dims, recipe: str = "haar", eps: float | None = None, seed: int = 0) -> np.ndarray:
    """Gauge field of shape (V, 4, 3, 3) in the canonical layout.

    recipe "haar": Haar SU(3); "smooth": exp(i*eps*H); "unit": free field;
    "gl3": complex Gaussian matrices (not unitary; the operator and the action
    are defined for any complex links, which the gradient checks exploit).
    """
    v = volume(dims)
    if recipe == "unit":
        return unit_links(dims)
    rng = np.random.default_rng(seed)
    if recipe == "haar":
        u = haar_su3(rng, 4 * v)
    elif recipe == "smooth":
        if eps is None:
            raise ValueError("smooth links need eps")
        u = smooth_su3(rng, 4 * v, float(eps))
    elif recipe == "gl3":
        u = gaussian(rng, (4 * v, 3, 3))
    else:
        raise ValueError(f"unknown link recipe {recipe!r}")
    return np.ascontiguousarray(u.reshape(v, 4, 3, 3), dtype=np.complex128)


def gaussian_half(dims, seed: int = 1, nvec: int | None = None) -> np.ndarray:
    """Gaussian half field(s): shape (V/2, 3), or (nvec, V/2, 3) when nvec is given."""
    v = volume(dims)
    rng = np.random.default_rng(seed)
    shape = (v // 2, 3) if nvec is None else (int(nvec), v // 2, 3)
    return np.ascontiguousarray(gaussian(rng, shape), dtype=np.complex128)


def gaussian_full(dims, seed: int = 1) -> np.ndarray:
    """Gaussian colour-vector field on all V sites, shape (V, 3), lexicographic order."""
    v = volume(dims)
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(gaussian(rng, (v, 3)), dtype=np.complex128)


def random_gauge_transform(dims, seed: int = 7) -> np.ndarray:
    """One Haar SU(3) matrix per site, shape (V, 3, 3)."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(haar_su3(rng, volume(dims)), dtype=np.complex128)


# ---------------------------------------------------------------------------
# Device-side generators for large volumes (same recipes, torch's own seeded
# stream: values differ from the numpy generators above; tests that compare
# with the oracle copy these arrays to the host and hand them to both sides).

def random_links_torch(dims, recipe: str = "smooth", eps: float | None = None, seed: int = 0, device="cuda"):
    """Gauge field (V,4,3,3) complex128 generated on `device` with torch.

    "smooth": exp(i*eps*H) with H = (A + A^dagger)/2 - tr/3, A complex Gaussian,
    the exponential by torch.linalg.matrix_exp; "haar": QR of a complex Gaussian
    with the phases of R moved into Q, determinant divided out."""
    import torch
    v = volume(dims)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    n = 4 * v
    out = torch.empty((n, 3, 3), dtype=torch.complex128, device=device)
    chunk = 1 << 21
    for s0 in range(0, n, chunk):
        m = min(chunk, n - s0)
        re = torch.randn((m, 3, 3), generator=gen, dtype=torch.float64, device=device)
        im = torch.randn((m, 3, 3), generator=gen, dtype=torch.float64, device=device)
        a = torch.complex(re, im) / np.sqrt(2.0)
        if recipe == "smooth":
            h = 0.5 * (a + a.conj().transpose(1, 2))
            tr = torch.diagonal(h, dim1=1, dim2=2).sum(-1).real / 3.0
            h = h - tr[:, None, None] * torch.eye(3, dtype=h.dtype, device=device)
            out[s0:s0 + m] = torch.linalg.matrix_exp(1j * float(eps) * h)
        elif recipe == "haar":
            q, r = torch.linalg.qr(a)
            d = torch.diagonal(r, dim1=1, dim2=2)
            q = q * (d / d.abs())[:, None, :]
            det = torch.linalg.det(q)
            out[s0:s0 + m] = q / (det ** (1.0 / 3.0))[:, None, None]
        else:
            raise ValueError(f"unknown link recipe {recipe!r}")
    return out.reshape(v, 4, 3, 3)


def gaussian_half_torch(dims, seed: int = 1, nvec: int | None = None, device="cuda"):
    """Gaussian half field(s) generated on `device`: (V/2,3) or (nvec,V/2,3) complex128."""
    import torch
    v = volume(dims)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    shape = (v // 2, 3) if nvec is None else (int(nvec), v // 2, 3)
    re = torch.randn(shape, generator=gen, dtype=torch.float64, device=device)
    im = torch.randn(shape, generator=gen, dtype=torch.float64, device=device)
    return torch.complex(re, im) / np.sqrt(2.0)

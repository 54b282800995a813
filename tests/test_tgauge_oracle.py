"""Pins of the oracle's temporal-gauge transform (oracle/tgauge.py, Sec. 4.3).

The transform is checked against what fixes it independently of its own code:
  * the definition along one time line, by brute force: g(x, t) is the ordered
    product U_t(x, 0) U_t(x, 1) ... U_t(x, t - 1), formed site by site in a loop;
  * the gauge condition the paper relies on: for unitary links every time link
    off the last slice becomes the identity, and the last one the full product;
  * gauge covariance through the oracle's own operator (eq. (staggered)):
    D[U'] (g psi) = g (D[U] psi) on both parities, and M' = g M g^dagger;
  * g is unitary, so norms (and with them CG residual norms) are kept.
A transposed product (U g instead of g U), a missing dagger, a wrong
neighbour or an off-by-one in t fails at least one of them.
"""

import numpy as np
import pytest

import lattice_inputs as li
import oracle as orc
from oracle import tgauge as tgo

DIMS = [(4, 4, 4, 4), (6, 4, 2, 6), (4, 2, 2, 2)]


def _site(dims, x, y, z, t):
    Lx, Ly, Lz, _ = dims
    return x + Lx * (y + Ly * (z + Lz * t))


@pytest.mark.parametrize("dims", DIMS)
def test_gauge_matrices_are_ordered_time_products(dims):
    U = li.random_links(dims, "haar", seed=1501)
    g = tgo.gauge_matrices(dims, U)
    Lx, Ly, Lz, Lt = dims
    rng = np.random.default_rng(1502)
    for _ in range(6):
        x, y, z = (int(rng.integers(L)) for L in (Lx, Ly, Lz))
        prod = np.eye(3, dtype=complex)
        for t in range(Lt):
            assert np.allclose(g[_site(dims, x, y, z, t)], prod, atol=1e-13)
            prod = prod @ U[_site(dims, x, y, z, t), 3]


@pytest.mark.parametrize("dims", DIMS)
def test_time_links_become_identity_off_the_last_slice(dims):
    U = li.random_links(dims, "haar", seed=1511)
    g, Up = tgo.temporal_links(dims, U)
    Lx, Ly, Lz, Lt = dims
    Vs = Lx * Ly * Lz
    eye = np.broadcast_to(np.eye(3), (Vs * (Lt - 1), 3, 3))
    assert np.abs(Up[: Vs * (Lt - 1), 3] - eye).max() <= 1e-13
    # last slice: the ordered product of the time links along the whole line
    for s in (0, Vs // 2, Vs - 1):
        prod = np.eye(3, dtype=complex)
        for t in range(Lt):
            prod = prod @ U[s + t * Vs, 3]
        assert np.allclose(Up[s + (Lt - 1) * Vs, 3], prod, atol=1e-13)
    # g unitary; U' unitary with unit determinant (SU(3) is kept)
    gg = g @ np.conj(np.swapaxes(g, 1, 2))
    assert np.abs(gg - np.eye(3)).max() <= 1e-13
    assert np.abs(np.linalg.det(Up) - 1).max() <= 1e-12


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("parity", [0, 1])
def test_operator_covariance_through_the_oracle(dims, parity):
    U = li.random_links(dims, "haar", seed=1521)
    psi = li.gaussian_half(dims, seed=1522)
    g, Up = tgo.temporal_links(dims, U)
    # the output parity's field from the input parity 1 - parity
    lhs = orc.dslash_half(dims, Up, tgo.apply_to_half(dims, g, psi, 1 - parity), parity)
    rhs = tgo.apply_to_half(dims, g, orc.dslash_half(dims, U, psi, parity), parity)
    assert np.linalg.norm(lhs - rhs) <= 1e-13 * np.linalg.norm(rhs)


def test_normal_operator_and_residual_norm_are_kept():
    dims, mass = (6, 4, 2, 6), 0.2
    U = li.random_links(dims, "haar", seed=1531)
    b = li.gaussian_half(dims, seed=1532)
    g, Up = tgo.temporal_links(dims, U)
    gb = tgo.apply_to_half(dims, g, b, 0)
    # M' (g b) = g (M b)
    lhs = orc.apply_M(dims, Up, mass, gb)
    rhs = tgo.apply_to_half(dims, g, orc.apply_M(dims, U, mass, b), 0)
    assert np.linalg.norm(lhs - rhs) <= 1e-13 * np.linalg.norm(rhs)
    # solving M' x' = g b and returning x = g^dagger x' solves M x = b
    xp, _, _, _ = orc.cg(dims, Up, mass, gb, tol=1e-12)
    x = tgo.apply_to_half(dims, g, xp, 0, dagger=True)
    assert orc.true_residual(dims, U, mass, x, b) <= 1e-11
    assert abs(np.linalg.norm(gb) - np.linalg.norm(b)) <= 1e-13 * np.linalg.norm(b)

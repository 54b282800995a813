"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics.

None of these re-types the oracle's formula: each checks a property that a
dropped term, a wrong sign, a wrong index or a transposed operand breaks.

  * Kogut-Susskind phases: pi flux through every plaquette (Sec. 4.2 only says
    eta = +-1; the flux is what makes the operator a staggered one).
  * Antihermiticity of D (Eq. (staggered) pairs U with U^dagger).
  * Even-odd connectivity (D only hops between neighbours).
  * Gauge covariance (U vs U^dagger, which end of the link, direction of hops).
  * Free-field spectrum with antiperiodic time (normalisation, phases, boundary).
  * Schur complement of the dense full operator (definition of M).
  * Dense linear solves (CG, multi-shift CG).
  * Central finite differences of S (force sign and factor) and covariance.
  * SU(3) third-row reconstruction (Sec. 4.3).
"""

import itertools

import numpy as np
import pytest

import lattice_inputs as li
import oracle as orc
from oracle import encodings as enc

DIMS_SMALL = [(2, 2, 2, 2), (4, 4, 4, 4), (4, 2, 6, 4), (2, 4, 2, 6)]


def inner(a, b):
    return np.vdot(np.ravel(a), np.ravel(b))


def coords(dims, i):
    Lx, Ly, Lz, Lt = dims
    return (i % Lx, (i // Lx) % Ly, (i // (Lx * Ly)) % Lz, i // (Lx * Ly * Lz))


def lex(dims, c):
    Lx, Ly, Lz, Lt = dims
    return c[0] + Lx * (c[1] + Ly * (c[2] + Lz * c[3]))


def parity_mask(dims):
    V = li.volume(dims)
    return np.array([sum(coords(dims, i)) % 2 for i in range(V)])


def shift(dims, c, mu, d):
    c = list(c)
    c[mu] = (c[mu] + d) % dims[mu]
    return tuple(c)


def split(dims, phi):
    """Full field (V,3) -> (even half, odd half)."""
    par = parity_mask(dims)
    V = li.volume(dims)
    e = np.zeros((V // 2, 3), complex)
    o = np.zeros((V // 2, 3), complex)
    for i in range(V):
        (e if par[i] == 0 else o)[i // 2] = phi[i]
    return e, o


def join(dims, e, o):
    par = parity_mask(dims)
    V = li.volume(dims)
    phi = np.zeros((V, 3), complex)
    for i in range(V):
        phi[i] = (e if par[i] == 0 else o)[i // 2]
    return phi


def dense_operator(n, apply):
    cols = []
    for k in range(n):
        v = np.zeros(n, complex)
        v[k] = 1.0
        cols.append(np.ravel(apply(v)))
    return np.array(cols).T


# --------------------------------------------------------------------------
# Kogut-Susskind phases
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 6, 4, 2), (6, 2, 2, 4)])
def test_eta_pi_flux_and_independence_of_own_direction(dims):
    V = li.volume(dims)
    for i in range(V):
        c = coords(dims, i)
        for mu in range(4):
            e = orc.eta(dims, c, mu)
            assert e in (1, -1)
            # eta_mu does not depend on x_mu, also across the periodic wrap
            assert orc.eta(dims, shift(dims, c, mu, 1), mu) == e
            for nu in range(4):
                if nu == mu:
                    continue
                flux = (e * orc.eta(dims, shift(dims, c, mu, 1), nu)
                        * orc.eta(dims, shift(dims, c, nu, 1), mu) * orc.eta(dims, c, nu))
                assert flux == -1


# --------------------------------------------------------------------------
# Antihermiticity and even-odd structure
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dims", DIMS_SMALL)
@pytest.mark.parametrize("recipe", ["haar", "gl3"])
def test_dslash_antihermitian(dims, recipe):
    U = li.random_links(dims, recipe, seed=3)
    psi = li.gaussian_full(dims, seed=4)
    phi = li.gaussian_full(dims, seed=5)
    lhs = inner(psi, orc.dslash_full(dims, U, phi))
    rhs = inner(orc.dslash_full(dims, U, psi), phi)
    scale = np.linalg.norm(psi) * np.linalg.norm(orc.dslash_full(dims, U, phi))
    assert abs(lhs + rhs) <= 1e-13 * scale


@pytest.mark.parametrize("dims", DIMS_SMALL)
def test_even_odd_connectivity(dims):
    U = li.random_links(dims, "haar", seed=11)
    V = li.volume(dims)
    par = parity_mask(dims)
    phi = li.gaussian_full(dims, seed=12)
    eps = np.where(par == 0, 1.0, -1.0)[:, None]
    # D anticommutes with the parity sign: eps D eps = -D
    lhs = eps * orc.dslash_full(dims, U, eps * phi)
    assert np.allclose(lhs, -orc.dslash_full(dims, U, phi), rtol=0, atol=1e-13)
    # D maps even to odd and odd to even only
    e, o = split(dims, phi)
    De = orc.dslash_full(dims, U, join(dims, e, np.zeros_like(o)))
    de_e, de_o = split(dims, De)
    assert np.all(de_e == 0)
    Do = orc.dslash_full(dims, U, join(dims, np.zeros_like(e), o))
    do_e, do_o = split(dims, Do)
    assert np.all(do_o == 0)
    # the half operators are exactly the off-diagonal blocks
    assert np.array_equal(orc.dslash_oe(dims, U, e), de_o)
    assert np.array_equal(orc.dslash_eo(dims, U, o), do_e)
    assert V == 2 * len(e)


def test_dense_connectivity_2x4():
    """At 2^4 every site has each neighbour twice (x+mu = x-mu); both hops count."""
    dims = (2, 2, 2, 2)
    U = li.random_links(dims, "haar", seed=21)
    V = li.volume(dims)
    D = dense_operator(3 * V, lambda v: orc.dslash_full(dims, U, v.reshape(V, 3)))
    par = np.repeat(parity_mask(dims), 3)
    assert np.all(D[np.ix_(par == 0, par == 0)] == 0)
    assert np.all(D[np.ix_(par == 1, par == 1)] == 0)
    assert np.allclose(D, -D.conj().T, atol=1e-14)
    # each site couples to its 4 distinct neighbours (2 links each: +mu and -mu)
    blocks = D.reshape(V, 3, V, 3)
    for i in range(V):
        nz = [j for j in range(V) if np.any(blocks[i, :, j, :] != 0)]
        assert len(nz) == 4


def dense_D_from_definition(dims, U):
    """The dense 3V x 3V operator written out hop by hop from Eq. (staggered),
    independently of the oracle's C: for every site x and direction mu,
    +eta_mu(x) U_mu(x) into the x + mu column and -eta_mu(x - mu) U_mu(x - mu)^dagger
    into the x - mu column, eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}) (reading Q2),
    and -1 on both hops that cross the time boundary (antiperiodic time, Q3)."""
    V = li.volume(dims)
    D = np.zeros((V, 3, V, 3), complex)
    for i in range(V):
        c = coords(dims, i)
        for mu in range(4):
            f = shift(dims, c, mu, +1)
            b = shift(dims, c, mu, -1)
            eta = (-1) ** sum(c[:mu])            # eta_mu does not depend on x_mu
            sf = eta * (-1 if (mu == 3 and c[3] == dims[3] - 1) else 1)
            sb = eta * (-1 if (mu == 3 and c[3] == 0) else 1)
            D[i, :, lex(dims, f), :] += sf * U[i, mu]
            D[i, :, lex(dims, b), :] -= sb * np.conj(U[lex(dims, b), mu]).T
    return D.reshape(3 * V, 3 * V)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 4), (2, 4, 2, 6)])
def test_dense_operator_matches_independent_builder(dims):
    """P5: the oracle's D against a dense matrix assembled directly from the
    definition (loops over sites and directions, no shared code), and the
    oracle's M against the Schur complement of that matrix."""
    U = li.random_links(dims, "haar", seed=31)
    V = li.volume(dims)
    D_ref = dense_D_from_definition(dims, U)
    D_orc = dense_operator(3 * V, lambda v: orc.dslash_full(dims, U, v.reshape(V, 3)))
    assert np.abs(D_orc - D_ref).max() <= 1e-14
    # M = m^2 - D_eo D_oe on even sites, from the independent matrix
    mass = 0.3
    par = np.repeat(parity_mask(dims), 3)
    Deo = D_ref[np.ix_(par == 0, par == 1)]
    Doe = D_ref[np.ix_(par == 1, par == 0)]
    M_ref = mass ** 2 * np.eye(3 * V // 2) - Deo @ Doe
    M_orc = dense_operator(3 * V // 2, lambda v: orc.apply_M(dims, U, mass, v.reshape(V // 2, 3)))
    assert np.abs(M_orc - M_ref).max() <= 1e-13


# --------------------------------------------------------------------------
# Gauge covariance
# --------------------------------------------------------------------------

def gauge_transform_links(dims, U, g):
    V = li.volume(dims)
    Ug = np.empty_like(U)
    for i in range(V):
        c = coords(dims, i)
        for mu in range(4):
            j = lex(dims, shift(dims, c, mu, 1))
            Ug[i, mu] = g[i] @ U[i, mu] @ g[j].conj().T
    return Ug


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 2, 6)])
def test_gauge_covariance(dims):
    U = li.random_links(dims, "haar", seed=31)
    g = li.random_gauge_transform(dims, seed=32)
    phi = li.gaussian_full(dims, seed=33)
    Ug = gauge_transform_links(dims, U, g)
    gphi = np.einsum("iab,ib->ia", g, phi)
    lhs = orc.dslash_full(dims, Ug, gphi)
    rhs = np.einsum("iab,ib->ia", g, orc.dslash_full(dims, U, phi))
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-12)
    # and M on even sites
    e, _ = split(dims, phi)
    ge, _ = split(dims, gphi)
    gE, _ = split(dims, np.einsum("iab,ib->ia", g, join(dims, orc.apply_M(dims, U, 0.3, e), np.zeros_like(e))))
    assert np.allclose(orc.apply_M(dims, Ug, 0.3, ge), gE, rtol=0, atol=1e-12)


# --------------------------------------------------------------------------
# Free field: spectrum of M and one-step CG convergence on an eigenvector
# --------------------------------------------------------------------------

def free_spectrum_even(dims, mass):
    """m^2 + 4 sum_mu sin^2 p_mu over p_i = 2 pi n/L (space), 2 pi (n+1/2)/Lt (time),
    three colours each, every other entry of the sorted full-lattice list."""
    Lx, Ly, Lz, Lt = dims
    vals = []
    for nx, ny, nz, nt in itertools.product(range(Lx), range(Ly), range(Lz), range(Lt)):
        p = (2 * np.pi * nx / Lx, 2 * np.pi * ny / Ly, 2 * np.pi * nz / Lz, 2 * np.pi * (nt + 0.5) / Lt)
        lam = mass ** 2 + 4 * sum(np.sin(q) ** 2 for q in p)
        vals += [lam] * 3
    vals = np.sort(vals)
    return vals[::2]


@pytest.mark.parametrize("dims,mass", [((4, 4, 4, 4), 0.1), ((2, 4, 6, 4), 0.3), ((4, 2, 2, 2), 0.05)])
def test_free_field_spectrum(dims, mass):
    U = li.unit_links(dims)
    n = 3 * li.volume(dims) // 2
    Ve = n // 3
    M = dense_operator(n, lambda v: orc.apply_M(dims, U, mass, v.reshape(Ve, 3)))
    assert np.allclose(M, M.conj().T, atol=1e-13)
    ev = np.sort(np.linalg.eigvalsh(M))
    assert np.allclose(ev, free_spectrum_even(dims, mass), rtol=0, atol=1e-12)


def test_free_field_plane_wave_cg_one_step():
    dims, mass = (4, 4, 4, 8), 0.1
    U = li.unit_links(dims)
    V = li.volume(dims)
    p = (2 * np.pi / 4, 0.0, 2 * np.pi * 3 / 4, 2 * np.pi * 2.5 / 8)
    colour = np.array([1.0, 0.5 - 0.25j, -0.75j])
    b = np.zeros((V // 2, 3), complex)
    for i in range(V):
        c = coords(dims, i)
        if sum(c) % 2 == 0:
            b[i // 2] = np.exp(1j * np.dot(p, c)) * colour
    lam = mass ** 2 + 4 * sum(np.sin(q) ** 2 for q in p)
    assert np.allclose(orc.apply_M(dims, U, mass, b), lam * b, atol=1e-13)
    x, iters, rel, st = orc.cg(dims, U, mass, b, tol=1e-12)
    assert st == 0 and iters == 1
    assert np.allclose(x, b / lam, rtol=0, atol=1e-14)


# --------------------------------------------------------------------------
# Schur complement, dense solves
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 4)])
def test_schur_complement_solves_full_system(dims):
    mass = 0.2
    U = li.random_links(dims, "haar", seed=41)
    V = li.volume(dims)
    D = dense_operator(3 * V, lambda v: orc.dslash_full(dims, U, v.reshape(V, 3)))
    b = li.gaussian_full(dims, seed=42)
    psi = np.linalg.solve(mass * np.eye(3 * V) + D, b.ravel()).reshape(V, 3)
    be, bo = split(dims, b)
    rhs = mass * be - orc.dslash_eo(dims, U, bo)
    Mdense = dense_operator(3 * V // 2, lambda v: orc.apply_M(dims, U, mass, v.reshape(V // 2, 3)))
    psi_e = np.linalg.solve(Mdense, rhs.ravel()).reshape(V // 2, 3)
    psi_o = (bo - orc.dslash_oe(dims, U, psi_e)) / mass
    pe, po = split(dims, psi)
    assert np.allclose(psi_e, pe, rtol=0, atol=1e-11 * np.abs(pe).max())
    assert np.allclose(psi_o, po, rtol=0, atol=1e-11 * np.abs(po).max())


@pytest.mark.parametrize("dims,mass,recipe", [((2, 2, 2, 2), 0.1, "haar"), ((4, 4, 4, 4), 0.1, "haar"),
                                               ((4, 2, 2, 4), 0.05, "smooth")])
def test_cg_matches_dense_solve(dims, mass, recipe):
    U = li.random_links(dims, recipe, eps=0.3, seed=51)
    Ve = li.volume(dims) // 2
    b = li.gaussian_half(dims, seed=52)
    Mdense = dense_operator(3 * Ve, lambda v: orc.apply_M(dims, U, mass, v.reshape(Ve, 3)))
    x_ref = np.linalg.solve(Mdense, b.ravel()).reshape(Ve, 3)
    x, iters, rel, st = orc.cg(dims, U, mass, b, tol=1e-13)
    assert st == 0 and rel <= 1e-13
    cond = np.linalg.cond(Mdense)
    assert np.linalg.norm(x - x_ref) <= 10 * cond * 1e-13 * np.linalg.norm(x_ref)
    # the recomputed residual the oracle reports is the real one
    assert abs(orc.true_residual(dims, U, mass, x, b) - rel) <= 1e-15 + 1e-3 * rel


def test_cg_terminates_after_number_of_distinct_eigenvalues():
    """Free field at 4^4: sin^2 p is 0 or 1 in space and 1/2 in antiperiodic
    time, so M has exactly four distinct eigenvalues m^2 + 4(n + 1/2), n = 0..3,
    and CG from any source ends after at most four steps."""
    dims, mass = (4, 4, 4, 4), 0.1
    U = li.unit_links(dims)
    b = li.gaussian_half(dims, seed=54)
    x, iters, rel, st = orc.cg(dims, U, mass, b, tol=1e-12)
    assert st == 0 and iters <= 4 and rel <= 1e-12
    x3, iters3, rel3, st3 = orc.cg(dims, U, mass, b, tol=1e-12, maxiter=3)
    assert st3 == 1 and rel3 > 1e-6


def test_cg_status_not_converged_and_zero_source():
    dims = (4, 4, 4, 4)
    U = li.random_links(dims, "haar", seed=61)
    b = li.gaussian_half(dims, seed=62)
    x, iters, rel, st = orc.cg(dims, U, 0.01, b, tol=1e-12, maxiter=5)
    assert st == 1 and iters == 5 and rel > 1e-12
    x, iters, rel, st = orc.cg(dims, U, 0.01, np.zeros_like(b), tol=1e-12)
    assert st == 0 and iters == 0 and np.all(x == 0)


@pytest.mark.parametrize("dims,mass", [((4, 4, 4, 4), 0.05), ((2, 4, 2, 4), 0.1)])
def test_multishift_matches_dense_shifted_solves(dims, mass):
    U = li.random_links(dims, "haar", seed=71)
    Ve = li.volume(dims) // 2
    b = li.gaussian_half(dims, seed=72)
    shifts = 10.0 ** (-5 + 5 * np.arange(12) / 11)
    X, iters, rel, st = orc.multishift_cg(dims, U, mass, shifts, b, tol=1e-12)
    assert st == 0
    Mdense = dense_operator(3 * Ve, lambda v: orc.apply_M(dims, U, mass, v.reshape(Ve, 3)))
    for s, sig in enumerate(shifts):
        A = Mdense + sig * np.eye(3 * Ve)
        xs = np.linalg.solve(A, b.ravel()).reshape(Ve, 3)
        assert rel[s] <= 2e-12
        assert np.linalg.norm(X[s] - xs) <= 1e-12 * np.linalg.cond(A) * np.linalg.norm(xs) * 10
    # shifts in any order, base system picked as the smallest
    perm = np.array([5, 0, 11, 3, 1, 2, 4, 6, 7, 8, 9, 10])
    X2, _, rel2, st2 = orc.multishift_cg(dims, U, mass, shifts[perm], b, tol=1e-12)
    assert st2 == 0
    assert np.allclose(X2, X[perm], rtol=0, atol=1e-10 * np.abs(X).max())


# --------------------------------------------------------------------------
# Force: finite differences of S, covariance
# --------------------------------------------------------------------------

GELL_MANN = [np.array(m, complex) for m in (
    [[0, 1, 0], [1, 0, 0], [0, 0, 0]],
    [[0, -1j, 0], [1j, 0, 0], [0, 0, 0]],
    [[1, 0, 0], [0, -1, 0], [0, 0, 0]],
    [[0, 0, 1], [0, 0, 0], [1, 0, 0]],
    [[0, 0, -1j], [0, 0, 0], [1j, 0, 0]],
    [[0, 0, 0], [0, 0, 1], [0, 1, 0]],
    [[0, 0, 0], [0, 0, -1j], [0, 1j, 0]],
    np.diag([1, 1, -2]) / np.sqrt(3),
)]


def expm_herm(h):
    w, v = np.linalg.eigh(h)
    return (v * np.exp(1j * w)) @ v.conj().T


def action_of(dims, U, mass, phi):
    X, _, _, st = orc.cg(dims, U, mass, phi, tol=1e-14)
    assert st == 0
    return orc.action(dims, phi, X)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 2, 4)])
def test_force_matches_central_fd_on_group(dims):
    mass, h = 0.2, 1e-5
    U = li.random_links(dims, "haar", seed=81)
    phi = li.gaussian_half(dims, seed=82)
    X, _, _, _ = orc.cg(dims, U, mass, phi, tol=1e-14)
    P, G = orc.force(dims, U, X)
    rng = np.random.default_rng(83)
    V = li.volume(dims)
    for _ in range(6):
        i, mu, a = int(rng.integers(V)), int(rng.integers(4)), int(rng.integers(8))
        T = GELL_MANN[a] / 2
        Up, Um = U.copy(), U.copy()
        Up[i, mu] = expm_herm(h * T) @ U[i, mu]
        Um[i, mu] = expm_herm(-h * T) @ U[i, mu]
        fd = (action_of(dims, Up, mass, phi) - action_of(dims, Um, mass, phi)) / (2 * h)
        an = np.trace(1j * T @ P[i, mu]).real
        assert abs(np.trace(1j * T @ P[i, mu]).imag) < 1e-12
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * np.abs(P).max())
    # P is traceless antihermitian
    assert np.allclose(P, -np.conj(np.swapaxes(P, -1, -2)), atol=1e-14)
    assert np.allclose(np.trace(P, axis1=-2, axis2=-1), 0, atol=1e-13)


def test_euclidean_gradient_matches_fd_on_complex_links():
    dims, mass, h = (2, 2, 4, 4), 0.3, 1e-6
    U = li.random_links(dims, "gl3", seed=91) * 0.4
    phi = li.gaussian_half(dims, seed=92)
    X, _, _, st = orc.cg(dims, U, mass, phi, tol=1e-14)
    assert st == 0
    _, G = orc.force(dims, U, X)
    rng = np.random.default_rng(93)
    V = li.volume(dims)
    for _ in range(8):
        i, mu, a, b = (int(rng.integers(V)), int(rng.integers(4)), int(rng.integers(3)),
                       int(rng.integers(3)))
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            Up, Um = U.copy(), U.copy()
            Up[i, mu, a, b] += unit * h
            Um[i, mu, a, b] -= unit * h
            fd = (action_of(dims, Up, mass, phi) - action_of(dims, Um, mass, phi)) / (2 * h)
            assert abs(fd - part(G[i, mu, a, b])) <= 1e-6 * max(1.0, abs(G[i, mu, a, b]))


def test_force_gauge_covariance():
    dims, mass = (4, 4, 2, 4), 0.25
    U = li.random_links(dims, "haar", seed=101)
    g = li.random_gauge_transform(dims, seed=102)
    phi = li.gaussian_half(dims, seed=103)
    Ug = gauge_transform_links(dims, U, g)
    ge, _ = split(dims, np.einsum("iab,ib->ia", g, join(dims, phi, np.zeros_like(phi))))
    X, _, _, _ = orc.cg(dims, U, mass, phi, tol=1e-14)
    Xg, _, _, _ = orc.cg(dims, Ug, mass, ge, tol=1e-14)
    assert abs(orc.action(dims, phi, X) - orc.action(dims, ge, Xg)) <= 1e-11 * abs(orc.action(dims, phi, X))
    P, _ = orc.force(dims, U, X)
    Pg, _ = orc.force(dims, Ug, Xg)
    rot = np.einsum("iab,imbc,idc->imad", g, P, np.conj(g))
    assert np.allclose(Pg, rot, rtol=0, atol=1e-10 * np.abs(P).max())


# --------------------------------------------------------------------------
# 12-real compression and the reduced-precision encodings
# --------------------------------------------------------------------------

def test_reconstruct_row2_su3():
    rng = np.random.default_rng(111)
    U = li.haar_su3(rng, 1000)
    assert np.allclose(orc.reconstruct_row2(U), U[:, 2, :], rtol=0, atol=1e-14)
    S = li.smooth_su3(rng, 1000, 0.3)
    assert np.allclose(orc.reconstruct_row2(S), S[:, 2, :], rtol=0, atol=1e-14)
    # a U(3) matrix with det != 1 is not reproduced (the test can fail)
    W = U * np.exp(0.5j)
    assert not np.allclose(orc.reconstruct_row2(W), W[:, 2, :], atol=1e-3)


def test_half_spinor_code():
    rng = np.random.default_rng(121)
    psi = li.gaussian(rng, (5000, 3)) * np.exp(rng.uniform(-20, 20, (5000, 1)))
    psi[7] = 0.0
    q, n = enc.encode_half_spinor(psi)
    assert q.dtype == np.float16 and n.dtype == np.float32
    assert np.all(np.abs(q.astype(np.float64)) <= 1.0)
    back = enc.decode_half_spinor(q, n)
    err = np.abs(back - psi).max(axis=1)
    # rounding to float32 (2^-24) then to a half code of magnitude <= 1 (2^-11 absolute)
    bound = (2.0 ** -11 + 2.0 ** -22) * np.abs(psi.view(np.float64).reshape(-1, 6)).max(axis=1)
    assert np.all(err <= bound * np.sqrt(2) + 1e-300)
    assert np.all(back[7] == 0)
    # the largest component of each site is coded as exactly +-1
    assert np.allclose(np.abs(q.astype(np.float64)).max(axis=1)[n > 0], 1.0)


# Round-to-nearest-even onto a binary grid with p significant bits, written
# from the definition with integer arithmetic on exact power-of-two scalings
# (independent of numpy's casts): quantum = 2^(e - p) for x = m 2^e with m in
# [1/2, 1), never below qmin (the subnormal spacing of the target format).
def _rne(x, p, qmin):
    import math
    if x == 0.0:
        return 0.0
    _, e = math.frexp(x)
    quantum = max(math.ldexp(1.0, e - p), qmin)
    q = x / quantum                      # exact: a power-of-two scaling
    n = math.floor(q)
    frac = q - n                         # exact: |q| < 2^(p+1)
    if frac > 0.5 or (frac == 0.5 and n % 2 == 1):
        n += 1
    return n * quantum


F32_QMIN = 2.0 ** -149
F16_QMIN = 2.0 ** -24


def _components(a):
    return np.ascontiguousarray(a, dtype=np.complex128).view(np.float64).ravel()


def test_round_f32_is_round_to_nearest_even_per_component():
    """round_f32 (the stored value of every float link and spinor component)
    equals round-to-nearest-even onto the 24-bit grid, real and imaginary
    parts separately; the result is a float32 and within half an ulp."""
    rng = np.random.default_rng(131)
    z = li.gaussian(rng, (4000,)) * np.exp2(rng.uniform(-40, 40, 4000))
    got = _components(enc.round_f32(z))
    want = np.array([_rne(v, 24, F32_QMIN) for v in _components(z)])
    assert np.array_equal(got, want)
    assert np.array_equal(got, got.astype(np.float32).astype(np.float64))
    import math
    half_ulp = np.array([math.ldexp(1.0, math.frexp(v)[1] - 25) for v in _components(z)])
    assert np.all(np.abs(got - _components(z)) <= half_ulp)
    # the real and imaginary parts are not mixed up
    w = np.array([1.0 + 2.0 ** -30 + 1j * (3.0 + 2.0 ** -20)])
    assert np.array_equal(enc.round_f32(w), np.array([1.0 + 1j * (3.0 + 2.0 ** -20)]))


def test_round_f32_ties_go_to_even():
    one = 1.0
    cases = {
        one + 2.0 ** -24: one,                              # tie, even neighbour below
        one + 3 * 2.0 ** -24: one + 2.0 ** -22,              # tie, even neighbour above
        one + 2.0 ** -24 + 2.0 ** -50: one + 2.0 ** -23,     # just above the tie
        -(one + 3 * 2.0 ** -24): -(one + 2.0 ** -22),        # sign symmetric
    }
    for x, y in cases.items():
        assert enc.round_f32(np.array([complex(x, -x)]))[0] == complex(y, -y)
        assert _rne(x, 24, F32_QMIN) == y


def test_round_f16_rounds_through_float32_like_the_kernels():
    """round_f16 is float64 -> float32 -> float16, each round-to-nearest-even
    (the kernels receive float32 values and round them to half).  A value
    just above a half-precision tie that float32 rounds onto the tie separates
    this from a direct float64 -> float16 rounding."""
    rng = np.random.default_rng(141)
    z = li.gaussian(rng, (4000,)) * 0.5
    z[:50] *= 2.0 ** -16                     # subnormal half codes
    got = _components(enc.round_f16(z))
    want = np.array([_rne(_rne(v, 24, F32_QMIN), 11, F16_QMIN) for v in _components(z)])
    assert np.array_equal(got, want)
    assert np.array_equal(got, got.astype(np.float16).astype(np.float64))
    # ties in half precision go to even
    assert _components(enc.round_f16(np.array([complex(1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11)]))).tolist() == \
        [1.0, 1 + 2.0 ** -9]
    # double rounding: float32 puts 1 + 2^-11 + 2^-40 on the half tie, which goes to 1
    x = 1 + 2.0 ** -11 + 2.0 ** -40
    assert _rne(x, 11, F16_QMIN) == 1 + 2.0 ** -10            # direct rounding would go up
    assert enc.round_f16(np.array([complex(x, 0)]))[0] == 1.0


def test_recon12_keeps_rounded_rows_and_rebuilds_the_third():
    rng = np.random.default_rng(151)
    U = li.smooth_su3(rng, 500, 0.3)
    for rounding in (enc.round_f32, enc.round_f16):
        R = enc.recon12(U, rounding)
        assert np.array_equal(R[:, :2, :], rounding(U[:, :2, :]))
        assert np.array_equal(R[:, 2, :], orc.reconstruct_row2(R))
        # the rebuilt row is close to the original one (SU(3) links), not equal to a rounded copy
        assert np.abs(R[:, 2, :] - U[:, 2, :]).max() <= 8 * 2.0 ** -11


def test_threaded_timing_build_gives_identical_bits():
    """The OpenMP build (used only to time the oracle on every host core)
    spreads independent sites over threads and keeps every sum sequential, so
    its operator, M and CG results equal the parity build's bit for bit."""
    dims, mass = (6, 4, 4, 6), 0.1
    U = li.random_links(dims, "haar", seed=161)
    psi = li.gaussian_half(dims, seed=162)
    full = li.gaussian_full(dims, seed=163)
    ref = (orc.dslash_half(dims, U, psi, 0), orc.dslash_half(dims, U, psi, 1), orc.apply_M(dims, U, mass, psi),
           orc.dslash_full(dims, U, full), orc.cg(dims, U, mass, psi, tol=1e-10)[0])
    with orc.threads():
        assert orc.num_threads() >= 1
        got = (orc.dslash_half(dims, U, psi, 0), orc.dslash_half(dims, U, psi, 1), orc.apply_M(dims, U, mass, psi),
               orc.dslash_full(dims, U, full), orc.cg(dims, U, mass, psi, tol=1e-10)[0])
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    assert orc.num_threads() == 1

"""Full-lattice solve (m + D) psi = b through the even-odd Schur complement,
checked with the oracle's full operator (pinned by antihermiticity, gauge
covariance and the free spectrum) and, at 2^4, against a dense solve."""

import numpy as np
import pytest

import lattice_inputs as li
import oracle as orc

pytestmark = pytest.mark.gpu


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("dims,mass,recipe", [((4, 4, 4, 4), 0.1, "haar"), ((10, 6, 4, 6), 0.2, "smooth"),
                                              ((32, 32, 32, 8), 0.01, "smooth")])
@pytest.mark.parametrize("kw", [dict(inner_prec=0, f64_arith=3), dict(inner_prec=0, f64_arith=0),
                                dict(inner_prec=1, inner_recon=12)])
def test_full_solve_residual(stag, dims, mass, recipe, kw):
    tol = 1e-10
    U = li.random_links(dims, recipe, eps=0.3, seed=901)
    b = li.gaussian_full(dims, seed=902)
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    psi = dev(np.zeros_like(b))
    st = ctx.solve_full(psi, dev(b), mass, tol=tol, **kw)
    assert st["status"] == 0
    p = host(psi)
    r = b - mass * p - orc.dslash_full(dims, U, p)
    # |r_full| = |b_e' - M psi_e| / m with |rhs_e| <= m |b_e| + 8 |b_o|
    assert np.linalg.norm(r) <= tol * (1 + 8 / mass) * np.linalg.norm(b)


def test_full_solve_matches_dense_2x4(stag):
    dims, mass = (2, 2, 2, 2), 0.3
    U = li.random_links(dims, "haar", seed=911)
    b = li.gaussian_full(dims, seed=912)
    V = 16
    D = np.array([orc.dslash_full(dims, U, e.reshape(V, 3)).ravel() for e in np.eye(3 * V)]).T
    ref = np.linalg.solve(mass * np.eye(3 * V) + D, b.ravel()).reshape(V, 3)
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    psi = dev(np.zeros_like(b))
    ctx.solve_full(psi, dev(b), mass, tol=1e-13, inner_prec=0, f64_arith=0)
    assert np.linalg.norm(host(psi) - ref) <= 1e-10 * np.linalg.norm(ref)


def test_full_solve_rejects_zero_mass(stag):
    dims = (4, 4, 4, 4)
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(li.random_links(dims, "haar", seed=921)))
    b = dev(li.gaussian_full(dims, seed=922))
    psi = dev(np.zeros((256, 3), complex))
    with pytest.raises(stag.StagError):
        ctx.solve_full(psi, b, 0.0)

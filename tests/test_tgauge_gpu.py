"""The double-float CG in temporal gauge (solver parameter temporal_gauge = 1).

The solve runs on the links U' = g U g^dagger with U'_t = 1 off the last time
slice and returns x = g^dagger x'.  Gauge covariance (the oracle's pin P3)
makes this the same system: the oracle-recomputed true residual of the
returned x, with the links as uploaded, is <= tol; and since M' = g M
g^dagger has the spectrum of M, the iteration count matches the solve on the
uploaded links within rounding (+-2).  Covered: Lt = 2 (the only time slice
pair: t = 0 with g = 1 and the boundary slice), an odd number of sites per
time slice per warp (6 x 4 x 2 x 10), the 32^3 x 8 workload, a re-uploaded
field (the transform follows it), the action S, and the IEEE-double refusal.
"""

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


@pytest.mark.parametrize("dims,recipe,mass", [((4, 4, 4, 2), "haar", 0.2), ((10, 6, 4, 6), "haar", 0.1),
                                              ((6, 4, 2, 10), "smooth", 0.05), ((8, 8, 8, 8), "smooth", 0.3)])
def test_temporal_gauge_solve_matches_oracle(stag, dims, recipe, mass):
    U = li.random_links(dims, recipe, eps=0.3, seed=901)
    b = li.gaussian_half(dims, seed=902)
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    x_tg, x = ctx.new_half(), ctx.new_half()
    st_tg = ctx.cg_solve(x_tg, dev(b), mass, tol=1e-10, temporal_gauge=1)
    st = ctx.cg_solve(x, dev(b), mass, tol=1e-10)
    assert orc.true_residual(dims, U, mass, host(x_tg), b) <= 1e-10
    assert abs(st_tg["iters"] - st["iters"]) <= 2
    # both solutions within the residual bound 2 tol cond(M) of each other
    cond = (mass ** 2 + 64) / mass ** 2
    assert np.linalg.norm(host(x_tg) - host(x)) <= 2e-10 * cond * np.linalg.norm(host(x))


def test_temporal_gauge_32c8_workload(stag):
    dims, mass = (32, 32, 32, 8), 0.01
    U = li.random_links(dims, "smooth", eps=0.3, seed=li.workload_seed(1, 0))
    b = li.gaussian_half(dims, seed=li.workload_seed(1, 1))
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    x = ctx.new_half()
    st = ctx.cg_solve(x, dev(b), mass, tol=1e-10, temporal_gauge=1)
    assert orc.true_residual(dims, U, mass, host(x), b) <= 1e-10
    assert abs(st["iters"] - 80) <= 2


def test_temporal_gauge_follows_reupload_and_action(stag):
    dims, mass = (10, 6, 4, 6), 0.1
    U1 = li.random_links(dims, "haar", seed=911)
    U2 = li.random_links(dims, "haar", seed=912)
    b = li.gaussian_half(dims, seed=913)
    ctx = stag.Context(dims)
    x = ctx.new_half()
    for U in (U1, U2, U1):
        ctx.upload_gauge(dev(U))
        ctx.cg_solve(x, dev(b), mass, tol=1e-10, temporal_gauge=1)
        assert orc.true_residual(dims, U, mass, host(x), b) <= 1e-10
    S_tg, _, _ = ctx.fermion_action(dev(b), mass, tol=1e-11, inner_prec=0, temporal_gauge=1)
    S, _, _ = ctx.fermion_action(dev(b), mass, tol=1e-11, inner_prec=0)
    assert abs(S_tg - S) <= 1e-9 * abs(S)


def test_temporal_gauge_needs_double_float(stag):
    dims = (4, 4, 4, 4)
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(li.random_links(dims, "haar", seed=921)))
    x = ctx.new_half()
    with pytest.raises(stag.StagError):
        ctx.cg_solve(x, dev(li.gaussian_half(dims, seed=922)), 0.1, f64_arith=0, temporal_gauge=1)

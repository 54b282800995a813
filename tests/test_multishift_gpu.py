"""Multi-shift CG against the oracle: every shifted system must reach an
oracle-recomputed double-precision true residual <= tol, and the shifted
solutions must agree with the oracle's multi-shift CG (itself pinned to dense
shifted solves) within the residual bound."""

import numpy as np
import pytest

import lattice_inputs as li
import oracle as orc

pytestmark = pytest.mark.gpu

SHIFTS12 = 10.0 ** (-5 + 5 * np.arange(12) / 11)


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("prec,recon", [(1, 12), (1, 18), (0, 18)])
@pytest.mark.parametrize("dims,mass", [((4, 4, 4, 4), 0.1), ((10, 6, 4, 6), 0.05)])
def test_multishift_matches_oracle(stag, prec, recon, dims, mass):
    U = li.random_links(dims, "smooth", eps=0.3, seed=601)
    b = li.gaussian_half(dims, seed=602)
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    X = ctx.new_half(len(SHIFTS12))
    st = ctx.cg_solve_multishift(X, dev(b), SHIFTS12, mass, tol=1e-10, inner_prec=prec, inner_recon=recon)
    Xh = host(X)
    Xo, _, rel_o, st_o = orc.multishift_cg(dims, U, mass, SHIFTS12, b, tol=1e-12)
    assert st_o == 0
    for i, s in enumerate(SHIFTS12):
        res = orc.true_residual(dims, U, mass, Xh[i], b, sigma=s)
        assert st[i]["status"] == 0 and res <= 1e-10, (i, st[i], res)
        # |x - x_oracle| <= (tol + tol_oracle) |b| / (m^2 + s)
        bound = 2e-10 * np.linalg.norm(b) / (mass ** 2 + s)
        assert np.linalg.norm(Xh[i] - Xo[i]) <= bound


def test_multishift_unsorted_and_duplicate_shifts(stag):
    dims, mass = (6, 4, 2, 10), 0.05
    U = li.random_links(dims, "haar", seed=611)
    b = li.gaussian_half(dims, seed=612)
    shifts = [0.3, 0.0, 1e-3, 0.3, 2.0]
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    X = ctx.new_half(len(shifts))
    st = ctx.cg_solve_multishift(X, dev(b), shifts, mass, tol=1e-10)
    Xh = host(X)
    for i, s in enumerate(shifts):
        assert orc.true_residual(dims, U, mass, Xh[i], b, sigma=s) <= 1e-10
    assert np.linalg.norm(Xh[0] - Xh[3]) <= 1e-9 * np.linalg.norm(Xh[0])


def test_multishift_32c16_workload(stag):
    """32^3 x 16, m = 0.005, 12 shifts log-spaced in [1e-5, 1], F32 Krylov phase,
    double-precision refinement to 1e-10 for every shift."""
    dims, mass = (32, 32, 32, 16), 0.005
    U = li.random_links(dims, "smooth", eps=0.3, seed=li.workload_seed(3, 0))
    b = li.gaussian_half(dims, seed=li.workload_seed(3, 1))
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    X = ctx.new_half(12)
    st = ctx.cg_solve_multishift(X, dev(b), SHIFTS12, mass, tol=1e-10)
    Xh = host(X)
    for i in (0, 5, 11):
        res = orc.true_residual(dims, U, mass, Xh[i], b, sigma=SHIFTS12[i])
        assert st[i]["status"] == 0 and res <= 1e-10, (i, st[i], res)


def test_multishift_bad_arguments(stag):
    import ctypes
    dims = (4, 4, 4, 4)
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(li.random_links(dims, "haar", seed=621)))
    b = dev(li.gaussian_half(dims, seed=622))
    X = ctx.new_half(2)
    with pytest.raises(stag.StagError):
        ctx.cg_solve_multishift(X, b, [-1.0, 0.5], 0.1)
    lib = stag.load()
    assert lib.stag_cg_solve_multishift(ctx._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(b.data_ptr()), None, 2,
                                        ctypes.c_double(0.1), None, None) == -1

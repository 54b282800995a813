"""Mixed-precision CG with reliable updates: every solve must reach an
oracle-recomputed double-precision true residual <= tol (1e-10), whatever the
inner storage (F32 or F16 with per-site norm, 18- or 12-real links)."""

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


INNER = [(1, 18), (1, 12), (2, 18), (2, 12)]


@pytest.mark.parametrize("prec,recon", INNER)
@pytest.mark.parametrize("dims,mass,recipe,eps", [((4, 4, 4, 4), 0.1, "haar", None),
                                                  ((10, 6, 4, 6), 0.05, "smooth", 0.3),
                                                  ((8, 8, 8, 8), 0.02, "smooth", 0.2)])
@pytest.mark.parametrize("arith", [0, 3])
def test_mixed_reaches_double_residual(stag, prec, recon, dims, mass, recipe, eps, arith):
    U = li.random_links(dims, recipe, eps=eps, seed=401)
    b = li.gaussian_half(dims, seed=402)
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    x = ctx.new_half()
    st = ctx.cg_solve_mixed(x, dev(b), mass, tol=1e-10, inner_prec=prec, inner_recon=recon, f64_arith=arith)
    res = orc.true_residual(dims, U, mass, host(x), b)
    assert st["status"] == 0 and res <= 1e-10, (st, res)
    assert st["reliable_updates"] >= 1
    assert abs(res - st["true_rel_residual"]) <= 1e-2 * res


@pytest.mark.parametrize("use_graph", [1, 0])
def test_mixed_graph_matches_host_loop(stag, use_graph):
    dims, mass = (6, 4, 2, 10), 0.05
    U = li.random_links(dims, "smooth", eps=0.3, seed=411)
    b = dev(li.gaussian_half(dims, seed=412))
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    x1, x2 = ctx.new_half(), ctx.new_half()
    s1 = ctx.cg_solve_mixed(x1, b, mass, tol=1e-10, use_graph=1)
    s2 = ctx.cg_solve_mixed(x2, b, mass, tol=1e-10, use_graph=use_graph, check_every=5)
    assert s1["iters"] == s2["iters"] and s1["reliable_updates"] == s2["reliable_updates"]
    assert bool((x1 == x2).all())


def test_mixed_48c12_workload_against_f64(stag):
    """48^3 x 12, smooth links eps = 0.2, m = 0.002: F32/12 and F16/12 inner solves
    reach the true residual 1e-10 (recomputed by the oracle), like plain F64 CG."""
    dims, mass = (48, 48, 48, 12), 0.002
    U = li.random_links(dims, "smooth", eps=0.2, seed=li.workload_seed(2, 0))
    b = li.gaussian_half(dims, seed=li.workload_seed(2, 1))
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    bd = dev(b)
    x64 = ctx.new_half()
    s64 = ctx.cg_solve(x64, bd, mass, tol=1e-10)
    assert s64["status"] == 0
    for prec in (1, 2):
        x = ctx.new_half()
        st = ctx.cg_solve_mixed(x, bd, mass, tol=1e-10, inner_prec=prec, inner_recon=12)
        res = orc.true_residual(dims, U, mass, host(x), b)
        assert st["status"] == 0 and res <= 1e-10, (prec, st, res)
        # both solutions within the residual bound of each other: |x - x64| <= 2 tol |b| / m^2
        d = np.linalg.norm(host(x) - host(x64))
        assert d <= 2 * 1e-10 * np.linalg.norm(b) / mass ** 2


def test_mixed_edge_cases(stag):
    import torch
    dims = (4, 4, 4, 4)
    U = li.random_links(dims, "haar", seed=421)
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    x = ctx.new_half()
    st = ctx.cg_solve_mixed(x, torch.zeros_like(x), 0.1)
    assert st["status"] == 0 and bool((x == 0).all())
    b = dev(li.gaussian_half(dims, seed=422))
    st = ctx.cg_solve_mixed(x, b, 0.01, tol=1e-12, maxiter=4, raise_on_fail=False)
    assert st["status"] == 1
    with pytest.raises(stag.StagError) as e:
        ctx.cg_solve_mixed(x, b, 0.1, inner_prec=0)
    assert e.value.code == -6

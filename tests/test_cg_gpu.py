"""Parity of the double-precision M apply and CG solver against the CPU oracle.

Bars: M applied to a vector within 1e-12 relative (L2); a solve to tol must
have an oracle-recomputed true residual <= tol; two solves near the rounding
floor agree to 2 tol cond(M) (the solution error is bounded by cond(M) times
the relative residual).
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


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def setup(stag, dims, recipe="haar", eps=None, seed=301):
    U = li.random_links(dims, recipe, eps=eps, seed=seed)
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    return ctx, U


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (10, 6, 4, 6)])
def test_apply_M_matches_oracle(stag, dims):
    ctx, U = setup(stag, dims)
    psi = li.gaussian_half(dims, seed=302)
    out = ctx.new_half()
    ctx.apply_M(out, dev(psi), 0.1)
    assert rel(host(out), orc.apply_M(dims, U, 0.1, psi)) <= 1e-12


@pytest.mark.parametrize("use_graph", [1, 0])
@pytest.mark.parametrize("arith", [0, 3])
def test_cg_4x4_workload(stag, use_graph, arith):
    """4^4, Haar links, m = 0.1, stop at true residual 1e-10; IEEE double (0) and
    double-float (3) operator arithmetic."""
    dims, mass = (4, 4, 4, 4), 0.1
    ctx, U = setup(stag, dims, seed=li.workload_seed(0, 0))
    b = li.gaussian_half(dims, seed=li.workload_seed(0, 1))
    x = ctx.new_half()
    st = ctx.cg_solve(x, dev(b), mass, tol=1e-10, use_graph=use_graph, f64_arith=arith)
    xr = host(x)
    assert st["status"] == 0
    res = orc.true_residual(dims, U, mass, xr, b)
    assert res <= 1e-10
    # The library recomputes the residual with its own operator arithmetic:
    # IEEE double agrees with the oracle to rounding; double-float carries the
    # operator's error (~1e-14 relative per application, times |x|/|b| <= 1/m^2),
    # the 1e-12 residual floor of that arithmetic at m = 0.1.
    floor = 1e-16 if arith == 0 else 1e-12
    assert abs(res - st["true_rel_residual"]) <= 1e-3 * res + floor
    x_cpu, it_cpu, _, _ = orc.cg(dims, U, mass, b, tol=1e-10)
    assert abs(st["iters"] - it_cpu) <= max(3, it_cpu // 20)


@pytest.mark.parametrize("arith,tol", [(0, 1e-11), (3, 1e-10)])
def test_graph_and_host_loop_identical(stag, arith, tol):
    """Graph and host-driven loops give the same solve bit for bit.  The
    double-float solve uses tol 1e-10: its residual floor at m = 0.05 is
    ~4e-12 (1e-12 (0.1 / m)^2), too close to 1e-11 for a stable stopping point."""
    dims, mass = (6, 4, 2, 10), 0.05
    ctx, U = setup(stag, dims, seed=311)
    b = dev(li.gaussian_half(dims, seed=312))
    x1, x2 = ctx.new_half(), ctx.new_half()
    s1 = ctx.cg_solve(x1, b, mass, tol=tol, use_graph=1, f64_arith=arith)
    s2 = ctx.cg_solve(x2, b, mass, tol=tol, use_graph=0, check_every=7, f64_arith=arith)
    assert s1["iters"] == s2["iters"]
    assert bool((x1 == x2).all())      # deterministic reductions: bit for bit
    s3 = ctx.cg_solve(x1, b, mass, tol=tol, use_graph=1, f64_arith=arith)   # graph reused
    assert s3["iters"] == s1["iters"] and bool((x1 == x2).all())


def test_shifted_solve(stag):
    dims, mass, sigma = (10, 6, 4, 6), 0.05, 0.3
    ctx, U = setup(stag, dims, "smooth", eps=0.3, seed=341)
    b = li.gaussian_half(dims, seed=342)
    x = ctx.new_half()
    st = ctx.cg_solve_shifted(x, dev(b), mass, sigma, tol=1e-10)
    assert st["status"] == 0
    assert orc.true_residual(dims, U, mass, host(x), b, sigma=sigma) <= 1e-10
    with pytest.raises(stag.StagError):
        ctx.cg_solve_shifted(x, dev(b), mass, -1.0)


@pytest.mark.parametrize("dims,mass,tol", [((4, 4, 4, 4), 0.1, 1e-13), ((8, 8, 8, 8), 0.5, 3e-14)])
def test_cg_tight_solution_matches_oracle(stag, dims, mass, tol):
    """Both solves to a residual near the double-precision floor.  Each solution
    is within tol ||b|| / lambda_min of the exact one and ||x|| >= ||b|| / lambda_max,
    so the two agree to 2 tol cond(M) relative.  cond(M) is computed from the dense
    M at 4^4; at 8^4 it is bounded by (m^2 + 64) / m^2 (||D_eo|| <= 8 for unitary
    links)."""
    ctx, U = setup(stag, dims, seed=321)
    b = li.gaussian_half(dims, seed=322)
    x = ctx.new_half()
    st = ctx.cg_solve(x, dev(b), mass, tol=tol, f64_arith=0)   # IEEE double: tol below the double-float floor
    x_cpu, _, rel_cpu, st_cpu = orc.cg(dims, U, mass, b, tol=tol)
    assert st_cpu == 0 and st["status"] == 0
    if dims == (4, 4, 4, 4):
        Ve = li.volume(dims) // 2
        M = np.array([orc.apply_M(dims, U, mass, e.reshape(Ve, 3)).ravel() for e in np.eye(3 * Ve)]).T
        ev = np.linalg.eigvalsh(M)
        cond = ev.max() / ev.min()
    else:
        cond = (mass ** 2 + 64) / mass ** 2
    assert rel(host(x), x_cpu) <= 2 * tol * cond


@pytest.mark.parametrize("arith,floor", [(0, 1e-12), (3, 1e-11)])
def test_cg_stagnation_stops(stag, arith, floor):
    """A tolerance below the rounding floor ends with NOT_CONVERGED after a few
    restarts instead of spinning until maxiter.  The floor of the recomputed
    residual is set by the operator's rounding amplified by the cancellation in
    M = m^2 - D_eo D_oe (|D_eo D_oe x| ~ 16 |x| against m^2 |x|): ~1e-13 for
    IEEE double, ~1e-12 for double-float (2^-44 per hop sum) at m = 0.1."""
    dims = (8, 8, 8, 8)
    ctx, U = setup(stag, dims, seed=323)
    b = dev(li.gaussian_half(dims, seed=324))
    x = ctx.new_half()
    st = ctx.cg_solve(x, b, 0.1, tol=1e-17, raise_on_fail=False, f64_arith=arith)
    assert st["status"] == 1 and st["restarts"] < 10 and st["true_rel_residual"] < floor


@pytest.mark.parametrize("arith", [0, 3])
def test_cg_32c8_workload(stag, arith):
    """32^3 x 8, smooth links eps = 0.3, m = 0.01, true residual 1e-10 (the bench step)."""
    dims, mass = (32, 32, 32, 8), 0.01
    ctx, U = setup(stag, dims, "smooth", eps=0.3, seed=li.workload_seed(1, 0))
    b = li.gaussian_half(dims, seed=li.workload_seed(1, 1))
    x = ctx.new_half()
    st = ctx.cg_solve(x, dev(b), mass, tol=1e-10, f64_arith=arith)
    assert st["status"] == 0 and st["iters"] > 10
    assert orc.true_residual(dims, U, mass, host(x), b) <= 1e-10


def test_cg_edge_cases(stag):
    import torch
    dims = (4, 4, 4, 4)
    ctx, U = setup(stag, dims, seed=331)
    x = ctx.new_half()
    # zero source: x = 0 exactly, no iterations
    st = ctx.cg_solve(x, torch.zeros_like(x), 0.1)
    assert st["status"] == 0 and st["iters"] == 0 and bool((x == 0).all())
    # iteration limit
    b = dev(li.gaussian_half(dims, seed=332))
    with pytest.raises(stag.NotConverged) as e:
        ctx.cg_solve(x, b, 0.01, tol=1e-14, maxiter=5)
    assert e.value.code == 1 and e.value.stats["iters"] == 5
    st = ctx.cg_solve(x, b, 0.01, tol=1e-14, maxiter=5, raise_on_fail=False)
    assert st["status"] == 1 and st["true_rel_residual"] > 1e-10
    # non-finite data ends in a breakdown status, not a fault
    bn = b.clone()
    bn[3, 1] = float("nan")
    st = ctx.cg_solve(x, bn, 0.1, raise_on_fail=False)
    assert st["status"] == 2
    # the context still solves afterwards
    st = ctx.cg_solve(x, b, 0.1)
    assert st["status"] == 0



@pytest.mark.parametrize("tol", [1e-10, 1e-17])
@pytest.mark.parametrize("tg", [0, 1])
@pytest.mark.parametrize("use_graph", [1, 0])
def test_direction_update_arrangements_identical(stag, monkeypatch, use_graph, tg, tol):
    """The double-float CG applies p = r + beta p either as a pass of its own
    (STAG_CG_DIR=0) or inside the next iteration's operator passes (1, the
    choice on lattices whose solver vectors fit in L2): the same arithmetic,
    so the same iterations and the same solution bit for bit.  tol 1e-17 lies
    below the rounding floor: the solve restarts from the true residual until
    a restart no longer halves it, which checks that both arrangements begin
    a restart with p = r."""
    dims, mass = (10, 6, 4, 6), 0.05
    U = li.random_links(dims, "smooth", eps=0.3, seed=361)
    b = li.gaussian_half(dims, seed=362)
    out = {}
    for setting in ("0", "1"):
        monkeypatch.setenv("STAG_CG_DIR", setting)
        ctx = stag.Context(dims)
        ctx.upload_gauge(dev(U))
        x = ctx.new_half()
        st = ctx.cg_solve(x, dev(b), mass, tol=tol, use_graph=use_graph, temporal_gauge=tg, raise_on_fail=False)
        if tol >= 1e-10:
            assert st["status"] == 0
            assert orc.true_residual(dims, U, mass, host(x), b) <= tol
        else:
            assert st["status"] == 1 and st["restarts"] >= 1 and st["true_rel_residual"] < 1e-11
        out[setting] = (st["iters"], st["restarts"], host(x))
        ctx.close()
    assert out["0"][:2] == out["1"][:2]
    assert np.array_equal(out["0"][2], out["1"][2])


def test_apply_M_noalloc_binding(stag):
    """The Python wrapper of the allocation-free operator: equal to the
    context's M to the operator bar, bad tensors rejected before the call."""
    import torch
    dims, mass = (6, 4, 2, 10), 0.2
    U = li.random_links(dims, "haar", seed=381)
    ctx, _ = setup(stag, dims, seed=381)
    psi = dev(li.gaussian_half(dims, seed=382))
    ref = ctx.new_half()
    ctx.apply_M(ref, psi, mass)
    out = torch.empty_like(psi)
    stag.apply_M_noalloc(dims, dev(U), out, psi, mass)
    torch.cuda.synchronize()
    assert rel(host(out), host(ref)) <= 1e-12
    with pytest.raises(stag.StagError):
        stag.apply_M_noalloc(dims, dev(U), out.to(torch.complex64), psi, mass)
    # shapes that do not match dims are refused on the host, before any launch
    Ud = dev(U)
    with pytest.raises(stag.StagError, match="shape"):
        stag.apply_M_noalloc(dims, Ud[: Ud.shape[0] // 2], out, psi, mass)
    with pytest.raises(stag.StagError, match="shape"):
        stag.apply_M_noalloc(dims, Ud, out[:-1], psi[:-1], mass)
    with pytest.raises(stag.StagError, match="shape"):
        stag.apply_M_noalloc((6, 4, 2, 12), Ud, out, psi, mass)
    with pytest.raises(stag.StagError):
        stag.apply_M_noalloc((6, 4, 3, 10), Ud, out, psi, mass)

"""The double-precision paths over the whole double range.

Double-float arithmetic keeps 48 significant bits only inside the float
exponent range, and the mixed solvers store floats or halves, so every solver
normalises its right-hand side by an exact power of two (largest component in
[1, 2)) and scales the solution back; the double-float operator entry points
do the same with their inputs and outputs, and double-float links whose
largest element lies outside 2^-40 .. 2^40 are stored scaled (the solvers then
use IEEE double).  Scaling by 2^s is exact and M is linear, so

  * a solve of 2^s b reaches the same oracle-recomputed residual as one of b,
    and its solution is 2^s times the solution for b, bit for bit;
  * the operator on 2^s psi is 2^s times the operator on psi.

Scales: 2^-200 and 2^-90 (below the float range and the 2^-74 limit of the
double-float split) and 2^120 (near the top of the float range).
"""

import numpy as np
import pytest

import lattice_inputs as li
import oracle as orc

pytestmark = pytest.mark.gpu

SCALES = [-200, -90, 120]


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def setup(stag, dims, recipe="haar", eps=None, seed=401, scale_links=0):
    U = li.random_links(dims, recipe, eps=eps, seed=seed) * 2.0 ** scale_links
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    return ctx, U


@pytest.mark.parametrize("s", SCALES)
@pytest.mark.parametrize("arith", [3, 0])
def test_cg_default_arithmetic_any_scale(stag, s, arith):
    dims, mass = (10, 6, 4, 6), 0.1
    ctx, U = setup(stag, dims)
    b = li.gaussian_half(dims, seed=402)
    x1, xs = ctx.new_half(), ctx.new_half()
    st1 = ctx.cg_solve(x1, dev(b), mass, tol=1e-10, f64_arith=arith)
    bs = b * 2.0 ** s
    sts = ctx.cg_solve(xs, dev(bs), mass, tol=1e-10, f64_arith=arith)
    assert sts["status"] == 0 and sts["iters"] == st1["iters"]
    assert orc.true_residual(dims, U, mass, host(xs), bs) <= 1e-10
    assert np.array_equal(host(xs), host(x1) * 2.0 ** s)


def test_cg_source_with_wide_dynamic_range(stag):
    """Components from 2^-300 to 2^100 in one source: the normalisation keeps
    the large ones exact; the tiny ones are far below the residual tolerance."""
    dims, mass = (4, 4, 6, 4), 0.1
    ctx, U = setup(stag, dims, seed=403)
    Vh = li.volume(dims) // 2
    b = li.gaussian_half(dims, seed=404) * np.exp2(np.random.default_rng(405).uniform(-300, 100, (Vh, 1)))
    x = ctx.new_half()
    st = ctx.cg_solve(x, dev(b), mass, tol=1e-10)
    assert st["status"] == 0
    assert orc.true_residual(dims, U, mass, host(x), b) <= 1e-10


@pytest.mark.parametrize("s", SCALES)
@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_any_scale(stag, s, prec):
    dims, mass = (10, 6, 4, 6), 0.1
    ctx, U = setup(stag, dims, seed=411)
    b = li.gaussian_half(dims, seed=412)
    x1, xs = ctx.new_half(), ctx.new_half()
    ctx.cg_solve_mixed(x1, dev(b), mass, tol=1e-10, inner_prec=prec, inner_recon=12)
    bs = b * 2.0 ** s
    st = ctx.cg_solve_mixed(xs, dev(bs), mass, tol=1e-10, inner_prec=prec, inner_recon=12)
    assert st["status"] == 0
    assert orc.true_residual(dims, U, mass, host(xs), bs) <= 1e-10
    assert np.array_equal(host(xs), host(x1) * 2.0 ** s)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_batched_systems_of_different_scales(stag, prec):
    """Each system is normalised on its own: sources 2^-200 b0, b1, 2^120 b2
    in one batch, each solution equal to the scaled solution of its unscaled
    source, bit for bit."""
    dims, mass = (10, 6, 4, 6), 0.1
    ctx, U = setup(stag, dims, seed=421)
    B = li.gaussian_half(dims, seed=422, nvec=3)
    sc = np.array([2.0 ** -200, 1.0, 2.0 ** 120])
    Bs = B * sc[:, None, None]
    X1, Xs = ctx.new_half(3), ctx.new_half(3)
    kw = dict(tol=1e-10, inner_prec=prec, inner_recon=12 if prec else 18, rhs_block=2)
    ctx.cg_solve_multi(X1, dev(B), mass, **kw)
    st = ctx.cg_solve_multi(Xs, dev(Bs), mass, **kw)
    xs = host(Xs)
    for k in range(3):
        assert st[k]["status"] == 0
        assert orc.true_residual(dims, U, mass, xs[k], Bs[k]) <= 1e-10
    assert np.array_equal(xs, host(X1) * sc[:, None, None])


@pytest.mark.parametrize("s", [-200, 120])
def test_multishift_any_scale(stag, s):
    dims, mass = (10, 6, 4, 6), 0.05
    ctx, U = setup(stag, dims, recipe="smooth", eps=0.3, seed=431)
    b = li.gaussian_half(dims, seed=432) * 2.0 ** s
    shifts = [1e-4, 1e-2, 0.3]
    X = ctx.new_half(3)
    st = ctx.cg_solve_multishift(X, dev(b), shifts, mass, tol=1e-10)
    xs = host(X)
    for i, sh in enumerate(shifts):
        assert st[i]["status"] == 0
        assert orc.true_residual(dims, U, mass, xs[i], b, sigma=sh) <= 1e-10


@pytest.mark.parametrize("s", [-150, -80, 200])
@pytest.mark.parametrize("parity", [0, 1])
def test_f64x_operator_any_scale(stag, s, parity):
    """The double-float operator on canonical fields of any scale meets the
    double-precision bar (the input is normalised on the device)."""
    dims = (10, 6, 4, 6)
    ctx, U = setup(stag, dims, seed=441)
    psi = li.gaussian_half(dims, seed=442) * 2.0 ** s
    out = ctx.new_half()
    (ctx.dslash_eo if parity == 0 else ctx.dslash_oe)(out, dev(psi), 3, 18)
    ref = orc.dslash_half(dims, U, psi, parity)
    assert rel(host(out), ref) <= 1e-12


def test_f64x_multi_operator_fields_of_different_scales(stag):
    dims = (10, 6, 4, 6)
    ctx, U = setup(stag, dims, seed=451)
    psi = li.gaussian_half(dims, seed=452, nvec=3) * np.array([2.0 ** -180, 1.0, 2.0 ** 150])[:, None, None]
    out = ctx.new_half(3)
    ctx.dslash_multi(out, dev(psi), 0, 3, 18, 2)
    got = host(out)
    for k in range(3):
        assert rel(got[k], orc.dslash_eo(dims, U, psi[k])) <= 1e-12


@pytest.mark.parametrize("sl", [-45, 45])
def test_links_outside_the_double_float_range(stag, sl):
    """Links scaled by 2^sl: the double-float operator stores them scaled and
    scales its output back; the default solver switches to IEEE double and
    still reaches the oracle-recomputed tolerance (mass scaled like the links
    so that M keeps its condition number).  The float inner iterations would
    leave the float range (M ~ 2^(2 sl)): the mixed solver refuses such links
    with an error code, and serves links within 2^-20 .. 2^20."""
    dims = (4, 4, 6, 4)
    ctx, U = setup(stag, dims, recipe="gl3", seed=461, scale_links=sl)
    psi = li.gaussian_half(dims, seed=462)
    out = ctx.new_half()
    ctx.dslash_oe(out, dev(psi), 3, 18)
    assert rel(host(out), orc.dslash_oe(dims, U, psi)) <= 1e-12
    Uh, _ = setup(stag, dims, recipe="haar", seed=463, scale_links=sl)
    Uh_np = li.random_links(dims, "haar", seed=463) * 2.0 ** sl
    mass = 0.1 * 2.0 ** sl
    b = li.gaussian_half(dims, seed=464)
    x = Uh.new_half()
    st = Uh.cg_solve(x, dev(b), mass, tol=1e-10)
    assert st["status"] == 0
    assert orc.true_residual(dims, Uh_np, mass, host(x), b) <= 1e-10
    with pytest.raises(stag.StagError) as e:
        Uh.cg_solve_mixed(x, dev(b), mass, tol=1e-10, inner_prec=1, inner_recon=18)
    assert e.value.code == -6
    sm = 15 if sl > 0 else -15
    Um, _ = setup(stag, dims, recipe="haar", seed=463, scale_links=sm)
    st = Um.cg_solve_mixed(x, dev(b), 0.1 * 2.0 ** sm, tol=1e-10, inner_prec=1, inner_recon=18)
    assert st["status"] == 0
    assert orc.true_residual(dims, Uh_np * 2.0 ** (sm - sl), 0.1 * 2.0 ** sm, host(x), b) <= 1e-10


def test_full_solve_any_scale(stag):
    dims, mass = (4, 4, 6, 4), 0.2
    U = li.random_links(dims, "haar", seed=471)
    import torch
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    b = li.gaussian_full(dims, seed=472) * 2.0 ** -190
    psi = torch.empty((li.volume(dims), 3), dtype=torch.complex128, device="cuda")
    st = ctx.solve_full(psi, dev(b), mass, tol=1e-11, inner_prec=0)
    assert st["status"] == 0
    r = b - mass * host(psi) - orc.dslash_full(dims, U, host(psi))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-11 * (1 + 8 / mass)


def test_force_of_a_tiny_source(stag):
    """phi scaled by 2^-150: X and Y = D_oe X are tiny, the force (quadratic
    in phi) is 2^-300 times the unscaled one, still matching the oracle's
    force on the same X to the double-precision bar."""
    dims, mass = (4, 4, 6, 4), 0.2
    U = li.random_links(dims, "haar", seed=481)
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    phi = li.gaussian_half(dims, seed=482) * 2.0 ** -150
    import torch
    S, X, st = ctx.fermion_action(dev(phi), mass, tol=1e-12, inner_prec=0)
    assert st["status"] == 0
    P = torch.empty((li.volume(dims), 4, 3, 3), dtype=torch.complex128, device="cuda")
    G = torch.empty_like(P)
    ctx.fermion_force(X, P=P, G=G)
    Pr, Gr = orc.force(dims, U, host(X))
    assert rel(host(P), Pr) <= 1e-12 and rel(host(G), Gr) <= 1e-12

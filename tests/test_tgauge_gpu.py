"""Temporal gauge (Sec. 4.3): the operator on the transformed links and every
solver with temporal_gauge = 1.

The library builds g and U' = g U g^dagger from the uploaded field and, with
the identity time links skipped, reads 6 links per site.  Checked here:
  * the operator entry points on U' (stag_set_operator_links) against the
    oracle's operator on the oracle's own transform (oracle/tgauge.py, pinned
    on the CPU): double storage at 1e-12, float / half storage on the stored
    values as in test_dslash_gpu.py;
  * skipping the identity links against reading them (LINKS_TEMPORAL against
    LINKS_TEMPORAL_FULL): bit for bit, single- and multi-vector kernels, on a
    lattice whose warps straddle time slices (10 x 6 x 4 x 6: V_s/2 = 120)
    and one whose do not;
  * every solver in temporal gauge: the oracle-recomputed true residual of the
    returned x, with the links as uploaded, is <= tol (gauge covariance makes
    M' x' = g b the same system), and the iteration count matches the solve on
    the uploaded links within rounding.
"""

import numpy as np
import pytest

import lattice_inputs as li
import oracle as orc
from oracle import encodings as enc
from oracle import tgauge as tgo

pytestmark = pytest.mark.gpu


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def make_ctx(stag, dims, U):
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    return ctx


@pytest.mark.parametrize("dims", [(4, 4, 4, 2), (10, 6, 4, 6), (8, 8, 8, 8)])
@pytest.mark.parametrize("prec,recon", [(0, 18), (0, 12), (3, 18), (1, 18), (1, 12), (2, 12)])
@pytest.mark.parametrize("parity", [0, 1])
def test_operator_on_temporal_links_matches_oracle(stag, dims, prec, recon, parity):
    U = li.random_links(dims, "haar", seed=1601)
    psi = li.gaussian_half(dims, seed=1602)
    _, Up = tgo.temporal_links(dims, U)
    ctx = make_ctx(stag, dims, U)
    ctx.set_operator_links(stag.LINKS_TEMPORAL)
    out = ctx.new_half()
    (ctx.dslash_eo if parity == 0 else ctx.dslash_oe)(out, dev(psi), prec, recon)
    got = host(out)
    if prec in (0, 3):
        ref = orc.dslash_half(dims, Up if recon == 18 else enc.recon12(Up), psi, parity)
        assert rel(got, ref) <= 1e-12
    elif prec == 1:
        Us = enc.round_f32(Up) if recon == 18 else enc.recon12(Up, enc.round_f32)
        ref = orc.dslash_half(dims, Us, enc.round_f32(psi), parity)
        assert rel(got, ref) <= 1e-5
        bound = 48 * 2.0 ** -24 * np.abs(psi).max() + 2.0 ** -24 * np.abs(ref).max()
        assert np.abs(got - ref).max() <= bound
    else:
        ref = enc.half_spinor(orc.dslash_half(dims, enc.recon12(Up, enc.round_f16), enc.half_spinor(psi), parity))
        assert rel(got, ref) <= 1e-3
    # the same field read with all 8 links: the same bits
    ctx.set_operator_links(stag.LINKS_TEMPORAL_FULL)
    full = ctx.new_half()
    (ctx.dslash_eo if parity == 0 else ctx.dslash_oe)(full, dev(psi), prec, recon)
    assert np.array_equal(got, host(full))
    # and back to the uploaded links
    ctx.set_operator_links(stag.LINKS_UPLOADED)
    (ctx.dslash_eo if parity == 0 else ctx.dslash_oe)(full, dev(psi), prec, recon)
    assert rel(host(full), orc.dslash_half(dims, U, psi, parity)) <= (1e-12 if prec in (0, 3) else 3e-3)


@pytest.mark.parametrize("dims", [(10, 6, 4, 6), (8, 8, 8, 8)])
@pytest.mark.parametrize("prec,recon,block", [(1, 12, 1), (1, 12, 4), (1, 12, (4 << 8) | 2), (1, 12, (2 << 8) | 4),
                                              (1, 12, (8 << 8) | 2), (1, 18, (2 << 8) | 2), (2, 12, (4 << 8) | 2),
                                              (2, 12, 2), (3, 18, 2), (0, 18, 4)])
def test_multi_vector_skip_is_bit_identical(stag, dims, prec, recon, block):
    U = li.random_links(dims, "smooth", eps=0.3, seed=1611)
    psi = li.gaussian_half(dims, seed=1612, nvec=5)
    ctx = make_ctx(stag, dims, U)
    outs = []
    for links in (stag.LINKS_TEMPORAL, stag.LINKS_TEMPORAL_FULL):
        ctx.set_operator_links(links)
        out = ctx.new_half(5)
        ctx.dslash_multi(out, dev(psi), 1, prec, recon, block)
        outs.append(host(out))
    assert np.array_equal(outs[0], outs[1])
    if prec in (0, 3):
        _, Up = tgo.temporal_links(dims, U)
        for k in range(5):
            assert rel(outs[0][k], orc.dslash_oe(dims, Up, psi[k])) <= 1e-12


def test_bare_kernel_paths_on_temporal_links(stag):
    """The timing entry points (stag_dslash_repeat and _repeat_multi) follow the
    operator's link field."""
    dims = (10, 6, 4, 6)
    U = li.random_links(dims, "smooth", eps=0.3, seed=1621)
    psi = li.gaussian_half(dims, seed=1622, nvec=3)
    _, Up = tgo.temporal_links(dims, U)
    ctx = make_ctx(stag, dims, U)
    ctx.set_operator_links(stag.LINKS_TEMPORAL)
    ctx.dslash_prepare(dev(psi[0]), 3)
    ctx.dslash_repeat(3, 18, 2)
    assert rel(host(ctx.dslash_result(ctx.new_half())), orc.dslash_eo(dims, Up, psi[0])) <= 1e-12
    ctx.dslash_prepare_multi(dev(psi), 1)
    ctx.dslash_repeat_multi(1, 12, 0, 2)
    got = host(ctx.dslash_result(ctx.new_half(3)))
    for k in range(3):
        ref = orc.dslash_eo(dims, enc.recon12(Up, enc.round_f32), enc.round_f32(psi[k]))
        assert rel(got[k], ref) <= 1e-5


def test_operator_links_argument_checked(stag):
    dims = (4, 4, 4, 4)
    ctx = make_ctx(stag, dims, li.random_links(dims, "haar", seed=1631))
    with pytest.raises(stag.StagError) as e:
        ctx.set_operator_links(3)
    assert e.value.code == -1


def test_non_unitary_links_are_refused(stag):
    """g U g^dagger fixes the temporal gauge only for unitary links: general
    complex links are refused (STAG_EUNSUPPORTED), not solved wrongly; the
    links as uploaded still work, and a unitary re-upload is accepted."""
    dims, mass = (4, 4, 4, 4), 0.3
    U = li.random_links(dims, "gl3", seed=1671)
    b = li.gaussian_half(dims, seed=1672)
    ctx = make_ctx(stag, dims, U)
    x = ctx.new_half()
    with pytest.raises(stag.StagError) as e:
        ctx.cg_solve(x, dev(b), mass, tol=1e-10, temporal_gauge=1)
    assert e.value.code == -6
    ctx.set_operator_links(stag.LINKS_TEMPORAL)
    with pytest.raises(stag.StagError) as e:
        ctx.dslash_eo(ctx.new_half(), dev(b))
    assert e.value.code == -6
    ctx.set_operator_links(stag.LINKS_UPLOADED)
    ctx.dslash_eo(x, dev(b))
    assert rel(host(x), orc.dslash_eo(dims, U, b)) <= 1e-12
    Uh = li.random_links(dims, "haar", seed=1673)
    ctx.upload_gauge(dev(Uh))
    ctx.cg_solve(x, dev(b), mass, tol=1e-10, temporal_gauge=1)
    assert orc.true_residual(dims, Uh, mass, host(x), b) <= 1e-10


@pytest.mark.parametrize("dims,recipe,mass", [((4, 4, 4, 2), "haar", 0.2), ((10, 6, 4, 6), "haar", 0.1),
                                              ((6, 4, 2, 10), "smooth", 0.05), ((8, 8, 8, 8), "smooth", 0.3)])
@pytest.mark.parametrize("arith", [3, 0])
def test_cg_in_temporal_gauge_matches_oracle(stag, dims, recipe, mass, arith):
    U = li.random_links(dims, recipe, eps=0.3, seed=901)
    b = li.gaussian_half(dims, seed=902)
    ctx = make_ctx(stag, dims, U)
    x_tg, x = ctx.new_half(), ctx.new_half()
    st_tg = ctx.cg_solve(x_tg, dev(b), mass, tol=1e-10, f64_arith=arith, temporal_gauge=1)
    st = ctx.cg_solve(x, dev(b), mass, tol=1e-10, f64_arith=arith)
    assert orc.true_residual(dims, U, mass, host(x_tg), b) <= 1e-10
    assert abs(st_tg["iters"] - st["iters"]) <= 2
    # both solutions within the residual bound 2 tol cond(M) of each other
    cond = (mass ** 2 + 64) / mass ** 2
    assert np.linalg.norm(host(x_tg) - host(x)) <= 2e-10 * cond * np.linalg.norm(host(x))


def test_cg_temporal_gauge_32c8_workload(stag):
    dims, mass = (32, 32, 32, 8), 0.01
    U = li.random_links(dims, "smooth", eps=0.3, seed=li.workload_seed(1, 0))
    b = li.gaussian_half(dims, seed=li.workload_seed(1, 1))
    ctx = make_ctx(stag, dims, U)
    x = ctx.new_half()
    st = ctx.cg_solve(x, dev(b), mass, tol=1e-10, temporal_gauge=1)
    assert orc.true_residual(dims, U, mass, host(x), b) <= 1e-10
    assert abs(st["iters"] - 80) <= 2


@pytest.mark.parametrize("inner,recon", [(1, 12), (2, 12), (1, 18)])
@pytest.mark.parametrize("arith", [3, 0])
def test_mixed_in_temporal_gauge_matches_oracle(stag, inner, recon, arith):
    dims, mass = (10, 6, 4, 6), 0.05
    U = li.random_links(dims, "smooth", eps=0.3, seed=1641)
    b = li.gaussian_half(dims, seed=1642)
    ctx = make_ctx(stag, dims, U)
    x_tg, x = ctx.new_half(), ctx.new_half()
    for ug in (1, 0):
        st_tg = ctx.cg_solve_mixed(x_tg, dev(b), mass, tol=1e-10, inner_prec=inner, inner_recon=recon,
                                   f64_arith=arith, temporal_gauge=1, use_graph=ug)
        assert orc.true_residual(dims, U, mass, host(x_tg), b) <= 1e-10
    st = ctx.cg_solve_mixed(x, dev(b), mass, tol=1e-10, inner_prec=inner, inner_recon=recon, f64_arith=arith)
    assert abs(st_tg["iters"] - st["iters"]) <= max(3, st["iters"] // 20)
    # the untransformed solve still uses its own links and graph afterwards
    assert orc.true_residual(dims, U, mass, host(x), b) <= 1e-10


@pytest.mark.parametrize("inner,recon,block", [(1, 12, 0), (1, 12, 2), (2, 12, (4 << 8) | 1), (0, 18, 2)])
def test_batched_in_temporal_gauge_matches_oracle(stag, inner, recon, block):
    dims, mass, n = (8, 8, 8, 8), 0.1, 5
    U = li.random_links(dims, "smooth", eps=0.3, seed=1651)
    B = li.gaussian_half(dims, seed=1652, nvec=n)
    ctx = make_ctx(stag, dims, U)
    X = ctx.new_half(n)
    sts = ctx.cg_solve_multi(X, dev(B), mass, tol=1e-10, inner_prec=inner, inner_recon=recon, rhs_block=block,
                             temporal_gauge=1)
    Xh = host(X)
    for k in range(n):
        assert orc.true_residual(dims, U, mass, Xh[k], B[k]) <= 1e-10, (k, sts[k])


def test_multishift_in_temporal_gauge_matches_oracle(stag):
    dims, mass = (8, 8, 8, 8), 0.05
    U = li.random_links(dims, "smooth", eps=0.3, seed=1661)
    b = li.gaussian_half(dims, seed=1662)
    shifts = [1e-4, 1e-2, 0.3]
    ctx = make_ctx(stag, dims, U)
    X = ctx.new_half(len(shifts))
    ctx.cg_solve_multishift(X, dev(b), shifts, mass, tol=1e-10, temporal_gauge=1)
    Xh = host(X)
    for i, s in enumerate(shifts):
        assert orc.true_residual(dims, U, mass, Xh[i], b, sigma=s) <= 1e-10


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
        ctx.cg_solve_mixed(x, dev(b), mass, tol=1e-10, temporal_gauge=1)
        assert orc.true_residual(dims, U, mass, host(x), b) <= 1e-10
    S_tg, _, _ = ctx.fermion_action(dev(b), mass, tol=1e-11, inner_prec=0, temporal_gauge=1)
    S, _, _ = ctx.fermion_action(dev(b), mass, tol=1e-11, inner_prec=0)
    assert abs(S_tg - S) <= 1e-9 * abs(S)

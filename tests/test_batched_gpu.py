"""Multi-vector operator and batched CG against the oracle.

The multi-vector Dslash must equal the single-vector one applied to each
vector (same arithmetic, so bit-identical for every rhs block) and the oracle
within the single-vector tolerances; every batched solve must reach an
oracle-recomputed double-precision true residual <= tol for every system."""

import numpy as np
import pytest

import lattice_inputs as li
import oracle as orc
from oracle import encodings as enc

pytestmark = pytest.mark.gpu


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec,recon,tol", [(0, 18, 1e-12), (0, 12, 1e-12), (1, 12, 1e-5), (1, 18, 1e-5),
                                            (2, 12, 1e-3), (3, 18, 1e-12)])
@pytest.mark.parametrize("nrhs", [1, 3, 16])
def test_multi_dslash_matches_single_and_oracle(stag, prec, recon, tol, nrhs):
    import torch
    dims = (10, 6, 4, 6)
    U = li.random_links(dims, "smooth", eps=0.3, seed=501)
    psi = li.gaussian_half(dims, seed=502, nvec=nrhs)
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    ind = dev(psi)
    single = torch.stack([ctx.dslash_oe(ctx.new_half(), ind[k], prec, recon) for k in range(nrhs)])
    for nb in (0, 1, 2, 4, 8, 16):
        out = ctx.new_half(nrhs)
        ctx.dslash_multi(out, ind, 1, prec, recon, nb)
        assert bool((out == single).all()), nb
    Us = {0: U, 1: enc.round_f32(U), 2: enc.round_f16(U), 3: U}[prec]
    if recon == 12:
        Us = enc.recon12(U, {0: None, 1: enc.round_f32, 2: enc.round_f16}[prec])
    for k in range(nrhs):
        src = {0: psi[k], 1: enc.round_f32(psi[k]), 2: enc.half_spinor(psi[k]), 3: psi[k]}[prec]
        assert rel(host(out[k]), orc.dslash_oe(dims, Us, src)) <= tol


@pytest.mark.parametrize("prec,recon", [(0, 18), (1, 12), (2, 12), (1, 18)])
@pytest.mark.parametrize("rhs_block", [0, 1, 4])
def test_batched_cg_every_system_converges(stag, prec, recon, rhs_block):
    dims, mass, nrhs = (8, 8, 8, 8), 0.05, 6
    U = li.random_links(dims, "smooth", eps=0.3, seed=511)
    B = li.gaussian_half(dims, seed=512, nvec=nrhs)
    B[2] *= 1e-3   # systems of very different scale
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    X = ctx.new_half(nrhs)
    st = ctx.cg_solve_multi(X, dev(B), mass, tol=1e-10, inner_prec=prec, inner_recon=recon, rhs_block=rhs_block)
    Xh = host(X)
    for k in range(nrhs):
        res = orc.true_residual(dims, U, mass, Xh[k], B[k])
        assert st[k]["status"] == 0 and res <= 1e-10, (k, st[k], res)
    assert ctx.last_rhs_block() in (1, 2, 4, 8, 16)
    if rhs_block:
        assert ctx.last_rhs_block() == rhs_block


def test_batched_f64_matches_single_solves(stag):
    """Plain double-precision batched CG follows the same recurrence as the
    single-system solver (its reductions are blocked differently, so rounding
    differs): iteration counts within 2 %, solutions within the residual
    bound 2 tol (m^2 + 64) / m^2 of each other."""
    dims, mass, nrhs, tol = (6, 4, 2, 10), 0.2, 4, 1e-11
    U = li.random_links(dims, "haar", seed=521)
    B = dev(li.gaussian_half(dims, seed=522, nvec=nrhs))
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    X = ctx.new_half(nrhs)
    st = ctx.cg_solve_multi(X, B, mass, tol=tol, inner_prec=0, inner_recon=18)
    for k in range(nrhs):
        x = ctx.new_half()
        s1 = ctx.cg_solve(x, B[k].contiguous(), mass, tol=tol)
        assert abs(s1["iters"] - st[k]["iters"]) <= max(2, 0.02 * s1["iters"])
        assert rel(host(X[k]), host(x)) <= 2 * tol * (mass ** 2 + 64) / mass ** 2


def test_batched_32c16_sixteen_rhs(stag):
    """32^3 x 16, m = 0.005, 16 Gaussian right-hand sides, F32/12 inner with
    double-precision reliable updates, one graph launch: every system to 1e-10."""
    dims, mass, nrhs = (32, 32, 32, 16), 0.005, 16
    U = li.random_links(dims, "smooth", eps=0.3, seed=li.workload_seed(3, 0))
    B = li.gaussian_half(dims, seed=li.workload_seed(3, 1), nvec=nrhs)
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    X = ctx.new_half(nrhs)
    st = ctx.cg_solve_multi(X, dev(B), mass, tol=1e-10, inner_prec=1, inner_recon=12)
    Xh = host(X)
    for k in (0, 7, 15):
        res = orc.true_residual(dims, U, mass, Xh[k], B[k])
        assert st[k]["status"] == 0 and res <= 1e-10, (k, st[k], res)
    assert all(s["status"] == 0 and s["true_rel_residual"] <= 1e-10 for s in st)


def test_batched_edge_cases(stag):
    import torch
    dims = (4, 4, 4, 4)
    U = li.random_links(dims, "haar", seed=531)
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    B = li.gaussian_half(dims, seed=532, nvec=3)
    B[1] = 0.0
    X = ctx.new_half(3)
    st = ctx.cg_solve_multi(X, dev(B), 0.1, tol=1e-10, inner_prec=1, inner_recon=12)
    assert bool((X[1] == 0).all()) and st[1]["status"] == 0
    assert st[0]["status"] == 0 and st[2]["status"] == 0
    lib = stag.load()
    import ctypes
    assert lib.stag_cg_solve_multi(ctx._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(X.data_ptr()), 0,
                                   ctypes.c_double(0.1), None, None) == -1
    assert lib.stag_cg_solve_multi(ctx._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(X.data_ptr()), 65,
                                   ctypes.c_double(0.1), None, None) == -1
    with pytest.raises(stag.StagError):
        ctx.cg_solve_multi(X, dev(B), 0.1, rhs_block=3)


@pytest.mark.parametrize("prec,f64_arith", [(1, 3), (2, 3), (1, 0)])
def test_batched_graph_and_host_loop_identical(stag, prec, f64_arith):
    """The graph (reliable updates inside a device-side if) and the host-driven
    loop (the reliable-update kernels launched every iteration, doing work only
    for the systems due) run the same kernels: the same iterations, reliable
    updates and solutions bit for bit, every system at the oracle's residual."""
    dims, mass, nrhs = (10, 6, 4, 6), 0.05, 5
    U = li.random_links(dims, "smooth", eps=0.3, seed=541)
    B = li.gaussian_half(dims, seed=542, nvec=nrhs)
    B[3] *= 1e-4
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    out = {}
    for ug in (1, 0):
        X = ctx.new_half(nrhs)
        st = ctx.cg_solve_multi(X, dev(B), mass, tol=1e-10, inner_prec=prec, inner_recon=12, rhs_block=4,
                                use_graph=ug, f64_arith=f64_arith)
        out[ug] = ([(s["iters"], s["reliable_updates"]) for s in st], host(X))
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1])
    for k in range(nrhs):
        assert orc.true_residual(dims, U, mass, out[1][1][k], B[k]) <= 1e-10


TILE_CODES = [(2, 1), (2, 2), (4, 1), (2, 4), (4, 2), (8, 1), (4, 4), (8, 2), (16, 1)]


def code(G, N):
    return (G << 8) | N


@pytest.mark.parametrize("prec,recon", [(1, 12), (1, 18), (2, 12), (2, 18)])
@pytest.mark.parametrize("dims,nrhs", [((10, 6, 4, 6), 5), ((6, 4, 2, 10), 16)])
def test_tile_configurations_equal_the_single_vector_operator(stag, prec, recon, dims, nrhs):
    """Every link-tile configuration (G warp groups sharing one shared-memory
    tile of hop matrices, NBT right-hand sides per thread; Sec. 4.3 NMULTI)
    gives the single-vector operator bit for bit, for both output parities,
    with ragged site tiles (V/2 = 720, 240) and masked right-hand sides."""
    import torch
    U = li.random_links(dims, "smooth", eps=0.3, seed=551)
    psi = li.gaussian_half(dims, seed=552, nvec=nrhs)
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    ind = dev(psi)
    for parity in (0, 1):
        fn = ctx.dslash_eo if parity == 0 else ctx.dslash_oe
        single = torch.stack([fn(ctx.new_half(), ind[k], prec, recon) for k in range(nrhs)])
        for G, N in TILE_CODES:
            out = ctx.new_half(nrhs)
            out.fill_(float("nan"))
            ctx.dslash_multi(out, ind, parity, prec, recon, code(G, N))
            assert bool((out == single).all()), (G, N, parity)


@pytest.mark.parametrize("G,N", [(1, 4), (2, 2), (4, 1), (4, 4), (8, 2), (16, 1)])
def test_batched_cg_tile_configurations(stag, G, N):
    """The batched solver with tile configurations: every system at the
    oracle's true residual; the iterations and reliable updates equal those of
    the register-blocked configuration (the operator is bit-identical; only
    the grouping of the <p, Ap> partial sums differs)."""
    dims, mass, nrhs = (10, 6, 4, 6), 0.05, 7
    U = li.random_links(dims, "smooth", eps=0.3, seed=561)
    B = li.gaussian_half(dims, seed=562, nvec=nrhs)
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    X = ctx.new_half(nrhs)
    st = ctx.cg_solve_multi(X, dev(B), mass, tol=1e-10, inner_prec=1, inner_recon=12, rhs_block=code(G, N))
    assert ctx.last_rhs_block() == G * N
    xs = host(X)
    for k in range(nrhs):
        assert st[k]["status"] == 0
        assert orc.true_residual(dims, U, mass, xs[k], B[k]) <= 1e-10
    X1 = ctx.new_half(nrhs)
    st1 = ctx.cg_solve_multi(X1, dev(B), mass, tol=1e-10, inner_prec=1, inner_recon=12, rhs_block=1)
    assert max(abs(a["iters"] - b["iters"]) for a, b in zip(st, st1)) <= 2


def test_tile_configuration_codes_rejected_for_double_links(stag):
    dims = (4, 4, 4, 4)
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(li.random_links(dims, "haar", seed=571)))
    psi = dev(li.gaussian_half(dims, seed=572, nvec=4))
    with pytest.raises(stag.StagError) as e:
        ctx.dslash_multi(ctx.new_half(4), psi, 0, 0, 18, code(4, 1))
    assert e.value.code == -1

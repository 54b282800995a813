"""The autotuner on the GPU: every launch shape it may choose for the
solvers' kernels gives the same solution bit for bit, a tuned solve equals
an untuned one, and a reloaded cache file skips the timing."""

import os

import numpy as np
import pytest

import lattice_inputs as li

pytestmark = pytest.mark.gpu

HOP = [128, 64, 256]
VEC = [(256 << 4) | 1, (128 << 4) | 1, (256 << 4) | 2, (128 << 4) | 2]


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.fixture()
def fresh_tuner(stag, tmp_path, monkeypatch):
    monkeypatch.setenv("STAG_TUNE_CACHE", str(tmp_path / "tune.json"))
    stag.tuner.clear()
    yield stag.tuner
    stag.tuner.clear()


def solve(stag, dims, U, b, mass, **kw):
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    x = ctx.new_half()
    st = ctx.cg_solve(x, dev(b), mass, tol=1e-10, **kw)
    out = (st["iters"], x.cpu().numpy())
    ctx.close()
    return out


@pytest.mark.parametrize("arith,kernels", [(0, ("cg_f64_hop", "cg_f64_update", "cg_f64_p")),
                                           (3, ("cg_f64x_hop_dir", "cg_f64x_update", "cg_f64x_p"))])
def test_every_cg_launch_shape_gives_the_same_bits(stag, fresh_tuner, arith, kernels):
    """Each candidate of each decision, forced through the cache before the
    first solve of a fresh context (ragged lattice: V/2 = 720, not a multiple
    of any block)."""
    import torch
    dims, mass = (10, 6, 4, 6), 0.1
    U = li.random_links(dims, "smooth", eps=0.3, seed=601)
    b = li.gaussian_half(dims, seed=602)
    gpu = torch.cuda.get_device_name()
    prec = 0 if arith == 0 else 3
    ref = None
    shapes = [(h, VEC[0], VEC[0]) for h in HOP] + [(128, u, p) for u, p in zip(VEC, VEC[::-1])]
    for hop, upd, pk in shapes:
        fresh_tuner.clear()
        for k, c in zip(kernels, (hop, upd, pk)):
            fresh_tuner.insert(fresh_tuner.make_key(k, dims, prec, 18, 1, gpu), c)
        got = solve(stag, dims, U, b, mass, f64_arith=arith)
        if ref is None:
            ref = got
        assert got[0] == ref[0] and np.array_equal(got[1], ref[1]), (hop, upd, pk)


def test_tuned_solve_equals_untuned_and_cache_file_skips_timing(stag, fresh_tuner, monkeypatch, tmp_path):
    dims, mass = (10, 6, 4, 6), 0.1
    U = li.random_links(dims, "haar", seed=611)
    b = li.gaussian_half(dims, seed=612)
    monkeypatch.setenv("STAG_TUNE", "0")
    untuned = solve(stag, dims, U, b, mass)
    assert fresh_tuner.stats()["timed"] == 0
    fresh_tuner.clear()
    monkeypatch.setenv("STAG_TUNE", "1")
    tuned = solve(stag, dims, U, b, mass)
    t = fresh_tuner.stats()
    assert t["timed"] >= 2          # hop and update (and p where it is a pass of its own)
    assert tuned[0] == untuned[0] and np.array_equal(tuned[1], untuned[1])
    path = tmp_path / "tune.json"
    assert path.exists()
    # a new process would start from the file: clear, load, solve again
    fresh_tuner.clear()
    assert fresh_tuner.load(path) >= 2
    again = solve(stag, dims, U, b, mass)
    t = fresh_tuner.stats()
    assert t["timed"] == 0 and t["from_cache"] >= 2
    assert np.array_equal(again[1], tuned[1])
    # force: time again what came from the file
    monkeypatch.setenv("STAG_TUNE", "force")
    fresh_tuner.clear()
    fresh_tuner.load(path)
    forced = solve(stag, dims, U, b, mass)
    assert fresh_tuner.stats()["timed"] >= 2
    assert np.array_equal(forced[1], tuned[1])


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_solver_launch_shapes_identical(stag, fresh_tuner, prec):
    import torch
    dims, mass = (10, 6, 4, 6), 0.1
    U = li.random_links(dims, "smooth", eps=0.3, seed=621)
    b = li.gaussian_half(dims, seed=622)
    gpu = torch.cuda.get_device_name()
    ref = None
    for hop, upd, pk in [(128, VEC[0], VEC[0]), (64, VEC[3], VEC[1]), (256, VEC[2], VEC[3])]:
        fresh_tuner.clear()
        for k, c in zip(("mixed_hop", "mixed_update", "mixed_p"), (hop, upd, pk)):
            fresh_tuner.insert(fresh_tuner.make_key(k, dims, prec, 12, 1, gpu), c)
        ctx = stag.Context(dims)
        ctx.upload_gauge(dev(U))
        x = ctx.new_half()
        st = ctx.cg_solve_mixed(x, dev(b), mass, tol=1e-10, inner_prec=prec, inner_recon=12)
        got = (st["iters"], st["reliable_updates"], x.cpu().numpy())
        ctx.close()
        if ref is None:
            ref = got
        assert got[:2] == ref[:2] and np.array_equal(got[2], ref[2]), (hop, upd, pk)


STAGED = 1 << 12   # hop block size + STAGED: links staged in shared memory; 2 STAGED: neighbour
                   # spinors; 3 STAGED: both


def test_mixed_half_staged_links_identical(stag, fresh_tuner):
    """Half 12-real inner iteration with its links and / or neighbour spinors
    staged in shared memory (cp.async, the hop and Mp_dot kernels) against the unstaged kernels: the
    same iterations, reliable updates and solution bits, as uploaded and in
    temporal gauge (ragged lattice: V/2 = 720)."""
    import torch
    dims, mass = (10, 6, 4, 6), 0.1
    U = li.random_links(dims, "smooth", eps=0.3, seed=631)
    b = li.gaussian_half(dims, seed=632)
    gpu = torch.cuda.get_device_name()
    for tg in (0, 1):
        ref = None
        for hop, mp in [(128, 0), (128 | STAGED, 1), (64 | STAGED, 0), (64, 1), (128 | 2 * STAGED, 2),
                        (64 | 3 * STAGED, 3), (128 | 3 * STAGED, 2)]:
            fresh_tuner.clear()
            sfx = "_tg" if tg else ""
            for k, c in (("mixed_hop" + sfx, hop), ("mixed_mpdot_stage" + sfx, mp), ("mixed_update", VEC[0]),
                         ("mixed_p", VEC[0])):
                fresh_tuner.insert(fresh_tuner.make_key(k, dims, 2, 12, 1, gpu), c)
            ctx = stag.Context(dims)
            ctx.upload_gauge(dev(U))
            x = ctx.new_half()
            st = ctx.cg_solve_mixed(x, dev(b), mass, tol=1e-10, inner_prec=2, inner_recon=12, temporal_gauge=tg)
            got = (st["iters"], st["reliable_updates"], x.cpu().numpy())
            ctx.close()
            if ref is None:
                ref = got
            assert got[:2] == ref[:2] and np.array_equal(got[2], ref[2]), (tg, hop, mp)


@pytest.mark.parametrize("dims", [(10, 6, 4, 6), (6, 4, 2, 10), (16, 16, 16, 16), (32, 32, 32, 12)])
def test_half_operator_staged_links_identical(stag, fresh_tuner, dims):
    """stag_dslash_repeat on half 12-real storage with the links, the
    neighbour spinors or both staged in shared memory equals the unstaged
    kernel bit for bit, as uploaded and in temporal gauge (identity time links
    skipped)."""
    import torch
    if li.volume(dims) > 100000:
        U = li.random_links_torch(dims, "smooth", 0.3, seed=641).cpu().numpy()
        psi = li.gaussian_half_torch(dims, seed=642).cpu().numpy()
    else:
        U = li.random_links(dims, "haar", seed=641)
        psi = li.gaussian_half(dims, seed=642)
    gpu = torch.cuda.get_device_name()
    for links in (stag.LINKS_UPLOADED, stag.LINKS_TEMPORAL):
        outs = []
        for choice in (0, 1, 2, 3):
            fresh_tuner.clear()
            key = "dslash_stage_tg" if links == stag.LINKS_TEMPORAL else "dslash_stage"
            fresh_tuner.insert(fresh_tuner.make_key(key, dims, 2, 12, 1, gpu), choice)
            ctx = stag.Context(dims)
            ctx.upload_gauge(dev(U))
            ctx.set_operator_links(links)
            ctx.dslash_prepare(dev(psi), stag.F16)
            ctx.dslash_repeat(stag.F16, 12, 2)
            out = ctx.new_half()
            ctx.dslash_result(out)
            outs.append(out.cpu().numpy())
            ctx.close()
        for o in outs[1:]:
            assert np.array_equal(outs[0], o), links
        assert np.isfinite(outs[0]).all() and np.abs(outs[0]).max() > 0

"""Parity of the CUDA half-lattice operators against the CPU oracle.

Tolerances (derived from the arithmetic, see the module docstrings of the
oracle encodings):
  * F64 storage, double arithmetic: relative L2 error <= 1e-12 (spec bar)
    and every element within 1e-13 of the output scale;
  * F32 / F16 storage, float arithmetic: compared with the double-precision
    operator applied to the *stored* values (rounded links, F16 codes); each
    output component is a sum of 48 products of magnitude <= max|U||psi|, so
    float accumulation bounds the error by about 48 * 2^-24 ~ 3e-6 of that
    scale: relative L2 <= 1e-5.
Sizes span several 128-thread blocks with a ragged tail (V/2 not a multiple of
128), the extent-2 case where x+mu = x-mu, and the 32^3 x 8 workload.
"""

import numpy as np
import pytest

import lattice_inputs as li
import oracle as orc
from oracle import encodings as enc

pytestmark = pytest.mark.gpu

SIZES = [(2, 2, 2, 2), (4, 4, 4, 4), (6, 4, 2, 2), (10, 6, 4, 6), (8, 8, 8, 8), (4, 6, 10, 14)]


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


@pytest.mark.parametrize("dims", SIZES)
@pytest.mark.parametrize("parity", [0, 1])
def test_f64_18_matches_oracle(stag, dims, parity):
    U = li.random_links(dims, "haar", seed=201)
    psi = li.gaussian_half(dims, seed=202)
    ctx = make_ctx(stag, dims, U)
    out = ctx.new_half()
    (ctx.dslash_eo if parity == 0 else ctx.dslash_oe)(out, dev(psi))
    got = host(out)
    ref = orc.dslash_half(dims, U, psi, parity)
    assert rel(got, ref) <= 1e-12
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (10, 6, 4, 6)])
def test_f64_18_gl3_links_and_host_upload(stag, dims):
    """Any complex links (not only SU(3)) for 18-real storage; upload from host memory."""
    U = li.random_links(dims, "gl3", seed=211)
    psi = li.gaussian_half(dims, seed=212)
    ctx = stag.Context(dims)
    import torch
    ctx.upload_gauge(torch.from_numpy(U))
    out = ctx.new_half()
    ctx.dslash_oe(out, dev(psi))
    assert rel(host(out), orc.dslash_oe(dims, U, psi)) <= 1e-12


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (10, 6, 4, 6)])
def test_f64_12_matches_oracle(stag, dims):
    U = li.random_links(dims, "haar", seed=221)
    psi = li.gaussian_half(dims, seed=222)
    ctx = make_ctx(stag, dims, U)
    out = ctx.new_half()
    ctx.dslash_eo(out, dev(psi), stag.F64, stag.RECON_12)
    ref = orc.dslash_eo(dims, enc.recon12(U), psi)
    assert rel(host(out), ref) <= 1e-12
    assert rel(host(out), orc.dslash_eo(dims, U, psi)) <= 1e-12


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (10, 6, 4, 6), (8, 8, 8, 8)])
@pytest.mark.parametrize("recon", [18, 12])
@pytest.mark.parametrize("parity", [0, 1])
def test_f32_matches_oracle_on_stored_values(stag, dims, recon, parity):
    U = li.random_links(dims, "smooth", eps=0.3, seed=231)
    psi = li.gaussian_half(dims, seed=232)
    ctx = make_ctx(stag, dims, U)
    out = ctx.new_half()
    (ctx.dslash_eo if parity == 0 else ctx.dslash_oe)(out, dev(psi), stag.F32, recon)
    Us = enc.round_f32(U) if recon == 18 else enc.recon12(U, enc.round_f32)
    ref = orc.dslash_half(dims, Us, enc.round_f32(psi), parity)
    got = host(out)
    assert rel(got, ref) <= 1e-5
    # every element: 48 float products per component, each rounded at 2^-24
    # of at most max|U| max|psi| (|U| <= 1), plus the float32 output rounding
    bound = 48 * 2.0 ** -24 * np.abs(psi).max() + 2.0 ** -24 * np.abs(ref).max()
    assert np.abs(got - ref).max() <= bound
    assert rel(got, orc.dslash_half(dims, U, psi, parity)) <= 1e-5


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (10, 6, 4, 6), (8, 8, 8, 8)])
@pytest.mark.parametrize("recon", [18, 12])
def test_f16_matches_oracle_on_stored_values(stag, dims, recon):
    U = li.random_links(dims, "smooth", eps=0.3, seed=241)
    psi = li.gaussian_half(dims, seed=242) * np.exp(np.random.default_rng(243).uniform(-3, 3, (dims[0] * dims[1] * dims[2] * dims[3] // 2, 1)))
    ctx = make_ctx(stag, dims, U)
    out = ctx.new_half()
    ctx.dslash_oe(out, dev(psi), stag.F16, recon)
    Us = enc.round_f16(U) if recon == 18 else enc.recon12(U, enc.round_f16)
    ref = orc.dslash_oe(dims, Us, enc.half_spinor(psi))
    got = host(out)
    # output is re-encoded to F16 on the way out: one more code rounding
    ref_out = enc.half_spinor(ref)
    assert rel(got, ref_out) <= 1e-3
    assert rel(got, ref) <= 1e-3
    assert rel(got, orc.dslash_oe(dims, U, psi)) <= 3e-3
    # every element, against its own site's scale: the float accumulation
    # (48 products at 2^-24 of the neighbours' magnitudes) can move a half code
    # by at most one unit, 2^-10 of the site's norm
    site = np.abs(ref_out.view(np.float64).reshape(-1, 6)).max(axis=1)
    nbr = 48 * 2.0 ** -24 * np.abs(psi).max()
    err = np.abs((got - ref_out).view(np.float64)).reshape(-1, 6).max(axis=1)
    assert np.all(err <= 2.0 ** -10 * site + 2 * nbr)


@pytest.mark.parametrize("prec,recon", [(1, 18), (1, 12), (2, 18), (2, 12)])
def test_reduced_precision_link_storage_element_by_element(stag, prec, recon):
    """The stored float / half links, read back one element at a time.

    A unit source e_b at one site makes every output component of the
    operator a single signed link element (products with 1.0, sums with 0:
    exact in float), so the kernel's output is the stored link itself: the
    columns b of the forward links into the site and the conjugated rows b of
    its own links (Sec. 4.3 12-real storage: rows 0 and 1 stored, row 2
    rebuilt).  Compared exactly with the oracle's encodings (round_f32,
    round_f16, and for half the output's own per-site code); only the rebuilt
    third row, formed in float by the kernel and in double by the oracle,
    gets a rounding tolerance."""
    dims = (4, 4, 6, 4)
    U = li.random_links(dims, "smooth", eps=0.3, seed=361)
    Vh = li.volume(dims) // 2
    ctx = make_ctx(stag, dims, U)
    out = ctx.new_half()
    rnd = enc.round_f32 if prec == 1 else enc.round_f16
    Us = rnd(U) if recon == 18 else enc.recon12(U, rnd)
    for parity in (0, 1):
        for h, b in ((0, 0), (37, 1), (Vh - 1, 2), (50, 2)):
            psi = np.zeros((Vh, 3), complex)
            psi[h, b] = 1.0
            (ctx.dslash_eo if parity == 0 else ctx.dslash_oe)(out, dev(psi), prec, recon)
            got = host(out)
            ref = orc.dslash_half(dims, Us, psi, parity)
            if prec == 2:
                ref = enc.half_spinor(ref)
            nz = np.abs(ref) > 0
            assert nz.sum() >= 8 * 3 - 3      # eight neighbours, three colours each (row-2 zeros aside)
            if recon == 18:
                assert np.array_equal(got, ref)
            else:
                # exact where no rebuilt element enters; rebuilt ones within float rounding
                # (half: a code can move by one unit of 2^-10 of the site's norm)
                tol = 4 * 2.0 ** -24 if prec == 1 else 2.0 ** -10
                site = np.abs(ref.view(np.float64)).reshape(-1, 6).max(axis=1)
                err = np.abs((got - ref).view(np.float64)).reshape(-1, 6).max(axis=1)
                assert np.all(err <= tol * site)
                if prec == 1:
                    # inexact only where the rebuilt row enters: colour 2 of the four
                    # forward hops, and all of a backward hop's row when b == 2
                    assert np.count_nonzero(got != ref) <= 4 + (12 if b == 2 else 0)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (10, 6, 4, 6), (8, 8, 8, 8)])
@pytest.mark.parametrize("parity", [0, 1])
def test_f64x_double_float_matches_oracle(stag, dims, parity):
    """Double-float arithmetic (48-bit significand) on double storage meets the
    double-precision bar: relative L2 error <= 1e-12 against the oracle."""
    U = li.random_links(dims, "haar", seed=271)
    rng = np.random.default_rng(272)
    Vh = dims[0] * dims[1] * dims[2] * dims[3] // 2
    # site magnitudes spread over 2^-60 .. 2^20, one exact zero site
    psi = li.gaussian_half(dims, seed=273) * np.exp2(rng.uniform(-60, 20, (Vh, 1)))
    psi[3] = 0.0
    ctx = make_ctx(stag, dims, U)
    out = ctx.new_half()
    (ctx.dslash_eo if parity == 0 else ctx.dslash_oe)(out, dev(psi), 3, 18)
    ref = orc.dslash_half(dims, U, psi, parity)
    got = host(out)
    assert rel(got, ref) <= 1e-12
    # per site, relative to that site's own scale of inputs: far sites keep precision too
    scale = np.abs(ref).max(axis=1) + 1e-300
    assert np.max(np.abs(got - ref).max(axis=1) / scale) <= 1e-9


def test_f64x_rejects_12_real(stag):
    dims = (4, 4, 4, 4)
    ctx = make_ctx(stag, dims, li.random_links(dims, "haar", seed=281))
    out = ctx.new_half()
    with pytest.raises(stag.StagError) as e:
        ctx.dslash_eo(out, dev(li.gaussian_half(dims, seed=282)), 3, 12)
    assert e.value.code == -6


def test_full_size_32c8_f64(stag):
    """The 32^3 x 8 workload (smooth links eps = 0.3): every output element."""
    dims = (32, 32, 32, 8)
    U = li.random_links(dims, "smooth", eps=0.3, seed=li.workload_seed(1, 0))
    psi = li.gaussian_half(dims, seed=li.workload_seed(1, 1))
    ctx = make_ctx(stag, dims, U)
    out = ctx.new_half()
    ctx.dslash_eo(out, dev(psi))
    ref = orc.dslash_eo(dims, U, psi)
    assert rel(host(out), ref) <= 1e-12
    ctx.dslash_oe(out, dev(psi))
    ref = orc.dslash_oe(dims, U, psi)
    assert rel(host(out), ref) <= 1e-12
    ctx.dslash_oe(out, dev(psi), 3, 18)
    assert rel(host(out), ref) <= 1e-12


def test_deterministic_repeat(stag):
    dims = (8, 8, 8, 8)
    U = li.random_links(dims, "haar", seed=251)
    psi = dev(li.gaussian_half(dims, seed=252))
    ctx = make_ctx(stag, dims, U)
    a, b = ctx.new_half(), ctx.new_half()
    ctx.dslash_eo(a, psi)
    ctx.dslash_eo(b, psi)
    assert bool((a == b).all())


def test_errors_are_reported_not_faulted(stag):
    import torch
    dims = (4, 4, 4, 4)
    ctx = stag.Context(dims)
    psi = dev(li.gaussian_half(dims, seed=261))
    out = ctx.new_half()
    with pytest.raises(stag.StagError) as e:
        ctx.dslash_eo(out, psi)          # no gauge field yet
    assert e.value.code == -5
    ctx.upload_gauge(dev(li.random_links(dims, "haar", seed=262)))
    with pytest.raises(stag.StagError) as e:
        ctx.dslash_eo(out, psi, 7, 18)   # unknown precision
    assert e.value.code == -6
    with pytest.raises(stag.StagError) as e:
        ctx.dslash_eo(out, psi, 0, 10)   # unknown compression
    assert e.value.code == -6
    lib = stag.load()
    import ctypes
    raw = torch.zeros(2 * psi.numel() + 1, dtype=torch.float64, device="cuda")
    mis = ctypes.c_void_p(raw.data_ptr() + 8)   # 8-byte aligned only
    assert lib.stag_dslash_eo(ctx._h, mis, ctypes.c_void_p(psi.data_ptr()), 0, 18) == -1
    assert lib.stag_dslash_eo(ctx._h, ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(psi.data_ptr()), 0, 18) == -1
    host_buf = np.zeros((128, 3), complex)
    assert lib.stag_dslash_eo(ctx._h, ctypes.c_void_p(host_buf.ctypes.data), ctypes.c_void_p(psi.data_ptr()), 0, 18) == -1
    # the context is still usable afterwards
    ctx.dslash_eo(out, psi)
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec,recon", [(0, 18), (3, 18), (1, 12), (2, 12)])
@pytest.mark.parametrize("dims", [(10, 6, 4, 6), (32, 32, 32, 8)])
def test_bare_kernel_path_matches_oracle(stag, dims, prec, recon):
    """The operator kernel the benchmark times: stag_dslash_prepare (internal
    storage of the precision: complex128, double-float pairs, float, half
    codes), stag_dslash_repeat, read back with stag_dslash_result.  At 32^3 x 8
    with the benchmark's own links and source."""
    if dims == (32, 32, 32, 8):
        U = li.random_links(dims, "smooth", eps=0.3, seed=li.workload_seed(1, 0))
        psi = li.gaussian_half(dims, seed=99)
    else:
        U = li.random_links(dims, "smooth", eps=0.3, seed=291)
        psi = li.gaussian_half(dims, seed=292)
    ctx = make_ctx(stag, dims, U)
    out = ctx.new_half()
    with pytest.raises(stag.StagError):
        ctx.dslash_result(out)             # nothing repeated yet
    ctx.dslash_prepare(dev(psi), prec)
    ctx.dslash_repeat(prec, recon, 3)      # the same input each time: the same output
    got = host(ctx.dslash_result(out))
    if prec in (0, 3):
        assert rel(got, orc.dslash_eo(dims, U, psi)) <= 1e-12
    elif prec == 1:
        ref = orc.dslash_eo(dims, enc.recon12(U, enc.round_f32), enc.round_f32(psi))
        assert rel(got, ref) <= 1e-5
    else:
        ref = orc.dslash_eo(dims, enc.recon12(U, enc.round_f16), enc.half_spinor(psi))
        assert rel(got, ref) <= 1e-3


@pytest.mark.parametrize("prec,recon,rhs_block", [(3, 18, 4), (3, 18, 1), (1, 12, 4), (0, 12, 2)])
def test_bare_multi_kernel_path_matches_oracle(stag, prec, recon, rhs_block):
    """The multi-vector operator the paper-comparable NMULTI scan times
    (stag_dslash_prepare_multi / _repeat_multi on internal storage): each of 3
    fields against the oracle, with a block of 4 (one lane masked), 2 or 1."""
    dims = (10, 6, 4, 6)
    U = li.random_links(dims, "smooth", eps=0.3, seed=301)
    psi = li.gaussian_half(dims, seed=302, nvec=3)
    ctx = make_ctx(stag, dims, U)
    ctx.dslash_prepare_multi(dev(psi), prec)
    ctx.dslash_repeat_multi(prec, recon, rhs_block, 2)
    got = host(ctx.dslash_result(ctx.new_half(3)))
    for k in range(3):
        if prec == 3:
            ref, bar = orc.dslash_eo(dims, U, psi[k]), 1e-12
        elif prec == 1:
            ref, bar = orc.dslash_eo(dims, enc.recon12(U, enc.round_f32), enc.round_f32(psi[k])), 1e-5
        else:
            ref, bar = orc.dslash_eo(dims, enc.recon12(U), psi[k]), 1e-12
        assert rel(got[k], ref) <= bar
    # a converting operator call discards the prepared fields
    ctx.dslash_eo(ctx.new_half(), dev(psi[0]), 1, 12)
    with pytest.raises(stag.StagError):
        ctx.dslash_repeat_multi(prec, recon, rhs_block, 1)


def test_cg_update_time(stag):
    dims = (8, 8, 8, 8)
    ctx = stag.Context(dims)
    for arith in (0, 3):
        assert 0.0 < ctx.cg_update_time(arith, nrep=3) < 100.0
    with pytest.raises(stag.StagError):
        ctx.cg_update_time(2, nrep=3)

"""Pseudo-fermion action and force against the oracle and finite differences.

* Force given X: P and G equal the oracle's (pinned by finite differences of
  S and gauge covariance) to 1e-12 relative; dS/dphi = 2 X exactly.
* Central finite differences of S on the group, on 64 random links of the
  24^3 x 8 workload (m = 0.01, eps = 0.3 links, step 1e-5).  S itself is ~1e5
  there, so S(U+) - S(U-) is formed without cancellation from the exact
  identity S(U+) - S(U-) = X+^dagger (M- - M+) X-  (X+- = M+-^{-1} phi, M
  Hermitian), with M- X- and M+ X- applied by the library; the quotient must
  match tr(i T P) to 1e-6 relative.
* torch.autograd.gradcheck of the autograd Function (complex128) at 2^4.
"""

import numpy as np
import pytest

import lattice_inputs as li
import oracle as orc

pytestmark = pytest.mark.gpu

GELL_MANN = [np.array(m, complex) for m in (
    [[0, 1, 0], [1, 0, 0], [0, 0, 0]], [[0, -1j, 0], [1j, 0, 0], [0, 0, 0]], [[1, 0, 0], [0, -1, 0], [0, 0, 0]],
    [[0, 0, 1], [0, 0, 0], [1, 0, 0]], [[0, 0, -1j], [0, 0, 0], [1j, 0, 0]], [[0, 0, 0], [0, 0, 1], [0, 1, 0]],
    [[0, 0, 0], [0, 0, -1j], [0, 1j, 0]], np.diag([1, 1, -2]) / np.sqrt(3))]


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def expm_herm(h):
    w, v = np.linalg.eigh(h)
    return (v * np.exp(1j * w)) @ v.conj().T


@pytest.mark.parametrize("dims,recipe", [((4, 4, 4, 4), "haar"), ((10, 6, 4, 6), "smooth"), ((2, 2, 2, 2), "gl3")])
def test_force_given_X_matches_oracle(stag, dims, recipe):
    import torch
    U = li.random_links(dims, recipe, eps=0.3, seed=801)
    X = li.gaussian_half(dims, seed=802)
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    P = torch.empty((ctx.V, 4, 3, 3), dtype=torch.complex128, device="cuda")
    G = torch.empty_like(P)
    gphi = ctx.new_half()
    ctx.fermion_force(dev(X), P=P, G=G, phi_grad=gphi, scale=1.0)
    Po, Go = orc.force(dims, U, X)
    assert rel(host(P), Po) <= 1e-12
    assert rel(host(G), Go) <= 1e-12
    assert np.array_equal(host(gphi), 2.0 * X)
    # scale multiplies every output
    ctx.fermion_force(dev(X), P=P, scale=-0.5)
    assert rel(host(P), -0.5 * Po) <= 1e-12


def test_action_matches_oracle(stag):
    dims, mass = (4, 4, 4, 4), 0.2
    U = li.random_links(dims, "haar", seed=811)
    phi = li.gaussian_half(dims, seed=812)
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    S, X, st = ctx.fermion_action(dev(phi), mass, tol=1e-13, inner_prec=0, f64_arith=0)
    Xo, _, _, _ = orc.cg(dims, U, mass, phi, tol=1e-13)
    So = orc.action(dims, phi, Xo)
    assert abs(S - So) <= 1e-11 * abs(So)
    assert orc.true_residual(dims, U, mass, host(X), phi) <= 1e-13
    # double-float and mixed-precision solves give the same action to their tolerance
    S1, _, _ = ctx.fermion_action(dev(phi), mass, tol=1e-11, inner_prec=0, f64_arith=3)
    assert abs(S1 - So) <= 1e-9 * abs(So)
    S2, _, _ = ctx.fermion_action(dev(phi), mass, tol=1e-10, inner_prec=1, inner_recon=12)
    assert abs(S2 - So) <= 1e-8 * abs(So)


def test_force_matches_finite_differences_24c8(stag):
    import torch
    dims, mass, h = (24, 24, 24, 8), 0.01, 1e-5
    U = li.random_links(dims, "smooth", eps=0.3, seed=li.workload_seed(4, 0))
    phi = dev(li.gaussian_half(dims, seed=li.workload_seed(4, 1)))
    ctx = stag.Context(dims)
    Ud = dev(U)
    ctx.upload_gauge(Ud)
    ieee = dict(tol=1e-13, inner_prec=0, f64_arith=0)
    _, X, st = ctx.fermion_action(phi, mass, **ieee)
    P = torch.empty_like(Ud)
    ctx.fermion_force(X, P=P)
    Ph = host(P)
    # the oracle's force on the same X
    Po, _ = orc.force(dims, U, host(X))
    assert rel(Ph, Po) <= 1e-12
    rng = np.random.default_rng(li.workload_seed(4, 2))
    V = ctx.V
    worst = 0.0
    for _ in range(64):
        i, mu, a = int(rng.integers(V)), int(rng.integers(4)), int(rng.integers(8))
        T = GELL_MANN[a] / 2
        Up, Um = Ud.clone(), Ud.clone()
        Up[i, mu] = dev(expm_herm(h * T) @ U[i, mu])
        Um[i, mu] = dev(expm_herm(-h * T) @ U[i, mu])
        ctx.upload_gauge(Up)
        _, Xp, _ = ctx.fermion_action(phi, mass, **ieee)
        MpXm = ctx.new_half()
        ctx.upload_gauge(Um)
        _, Xm, _ = ctx.fermion_action(phi, mass, **ieee)
        MmXm = ctx.new_half()
        ctx.apply_M(MmXm, Xm, mass)
        ctx.upload_gauge(Up)
        ctx.apply_M(MpXm, Xm, mass)
        dS = torch.vdot(Xp.flatten(), (MmXm - MpXm).flatten()).real.item()
        fd = dS / (2 * h)
        an = np.trace(1j * T @ Ph[i, mu]).real
        err = abs(fd - an) / max(abs(an), 1e-3 * np.abs(Ph).max())
        worst = max(worst, err)
    assert worst <= 1e-6, worst


def test_autograd_gradcheck_2x4(stag):
    import torch
    dims, mass = (2, 2, 2, 2), 0.5
    ctx = stag.Context(dims)
    U = dev(li.random_links(dims, "gl3", seed=821) * 0.5).requires_grad_(True)
    phi = dev(li.gaussian_half(dims, seed=822)).requires_grad_(True)

    def f(U_, phi_):
        return stag.StaggeredAction(U_, phi_, ctx, mass, tol=1e-13, f64_arith=0)

    assert torch.autograd.gradcheck(f, (U, phi), eps=1e-6, atol=1e-6, rtol=1e-4)


def test_autograd_gradient_equals_force_api(stag):
    import torch
    dims, mass = (4, 4, 4, 4), 0.1
    ctx = stag.Context(dims)
    Uh = li.random_links(dims, "haar", seed=831)
    U = dev(Uh).requires_grad_(True)
    phi = dev(li.gaussian_half(dims, seed=832))
    S = stag.StaggeredAction(U, phi, ctx, mass, tol=1e-13, f64_arith=0)
    (3.0 * S).backward()
    Xo, _, _, _ = orc.cg(dims, Uh, mass, host(phi), tol=1e-13)
    _, Go = orc.force(dims, Uh, Xo)
    assert rel(host(U.grad), 3.0 * Go) <= 1e-10
    P = stag.fermion_force(U.detach(), phi, ctx, mass, tol=1e-13, f64_arith=0)
    Po, _ = orc.force(dims, Uh, Xo)
    assert rel(host(P), Po) <= 1e-10


def test_reupload_keeps_cached_solver_graphs_valid(stag):
    """Re-uploading the gauge field re-derives the compressed / double-float link
    copies in place, so solver graphs captured before the upload stay valid
    (every solver path, several uploads in a row)."""
    import torch
    dims, mass = (8, 8, 8, 8), 0.1
    ctx = stag.Context(dims)
    b = li.gaussian_half(dims, seed=841)
    for seed in (842, 843, 844):
        U = li.random_links(dims, "smooth", eps=0.3, seed=seed)
        ctx.upload_gauge(dev(U))
        for kw in (dict(f64_arith=3), dict(f64_arith=0)):
            x = ctx.new_half()
            st = ctx.cg_solve(x, dev(b), mass, tol=1e-10, **kw)
            assert st["status"] == 0 and orc.true_residual(dims, U, mass, host(x), b) <= 1e-10
        for kw in (dict(inner_prec=1, inner_recon=12, f64_arith=3), dict(inner_prec=2, inner_recon=12, f64_arith=0)):
            x = ctx.new_half()
            st = ctx.cg_solve_mixed(x, dev(b), mass, tol=1e-10, **kw)
            assert st["status"] == 0 and orc.true_residual(dims, U, mass, host(x), b) <= 1e-10
        X = ctx.new_half(2)
        B = dev(np.stack([b, 2 * b]))
        st = ctx.cg_solve_multi(X, B, mass, tol=1e-10, inner_prec=1, inner_recon=12)
        assert all(s["status"] == 0 for s in st)
        assert orc.true_residual(dims, U, mass, host(X[1]), 2 * b) <= 1e-10
    torch.cuda.synchronize()


def test_rational_force_is_weighted_sum(stag):
    """sum_i r_i F(X_i) with X_i from the multi-shift solver equals the oracle's
    weighted sum of single forces; and the rational action's derivative, checked
    against central finite differences of S = sum_i r_i phi^dagger (M+s_i)^-1 phi."""
    import torch
    dims, mass = (4, 4, 4, 4), 0.2
    shifts = [0.01, 0.1, 1.0]
    coeffs = [0.5, 0.3, 0.2]
    U = li.random_links(dims, "haar", seed=851)
    phi = li.gaussian_half(dims, seed=852)
    ctx = stag.Context(dims)
    ctx.upload_gauge(dev(U))
    X = ctx.new_half(3)
    # 1e-12 is at the double-float residual floor: IEEE double passes
    ctx.cg_solve_multishift(X, dev(phi), shifts, mass, tol=1e-12, inner_prec=0, f64_arith=0)
    P = torch.empty((ctx.V, 4, 3, 3), dtype=torch.complex128, device="cuda")
    G = torch.empty_like(P)
    ctx.fermion_force_multi(X, coeffs, P=P, G=G)
    Xh = host(X)
    Pref = sum(c * orc.force(dims, U, Xh[i])[0] for i, c in enumerate(coeffs))
    Gref = sum(c * orc.force(dims, U, Xh[i])[1] for i, c in enumerate(coeffs))
    assert np.linalg.norm(host(P) - Pref) <= 1e-12 * np.linalg.norm(Pref)
    assert np.linalg.norm(host(G) - Gref) <= 1e-12 * np.linalg.norm(Gref)
    # P alone (the kernel on the double-float fields of the operator pass,
    # accumulated over the terms) against the same sum
    P1 = torch.full_like(P, float("nan"))
    ctx.fermion_force_multi(X, coeffs, P=P1)
    assert np.linalg.norm(host(P1) - Pref) <= 1e-12 * np.linalg.norm(Pref)
    # finite differences of the rational action on the group (oracle solves)
    def S_of(Ux):
        tot = 0.0
        for c, s in zip(coeffs, shifts):
            Xs = orc.multishift_cg(dims, Ux, mass, [s], phi, tol=1e-14)[0][0]
            tot += c * orc.action(dims, phi, Xs)
        return tot
    rng = np.random.default_rng(853)
    h = 1e-5
    Ph = host(P)
    for _ in range(4):
        i, mu, a = int(rng.integers(ctx.V)), int(rng.integers(4)), int(rng.integers(8))
        T = GELL_MANN[a] / 2
        Up, Um = U.copy(), U.copy()
        Up[i, mu] = expm_herm(h * T) @ U[i, mu]
        Um[i, mu] = expm_herm(-h * T) @ U[i, mu]
        fd = (S_of(Up) - S_of(Um)) / (2 * h)
        an = np.trace(1j * T @ Ph[i, mu]).real
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * np.abs(Ph).max())

"""Python binding of libstag (staggered Dslash and even-odd CG on one GB300).

Argument marshalling only: every operation runs in the CUDA kernels of
``libstag.so`` (built from ``csrc/`` by ``_build.build()``).  There is no CPU
fallback; if the library or a CUDA device is missing, the calls raise.

Fields are torch complex128 tensors on the CUDA device, in the canonical
layout of ``include/stag.h``:

* gauge field: shape (V, 4, 3, 3), site index x + Lx*(y + Ly*(z + Lz*t));
* half field of one parity: shape (V//2, 3); several: (n, V//2, 3).

Method names follow the C entry points (``stag_dslash_eo`` ->
``Context.dslash_eo``).  Work is enqueued on torch's current CUDA stream.
"""

from __future__ import annotations

import ctypes
import os
import threading

__all__ = [
    "F64", "F32", "F16", "F64X", "RECON_18", "RECON_12", "StagError", "NotConverged",
    "LINKS_UPLOADED", "LINKS_TEMPORAL", "LINKS_TEMPORAL_FULL",
    "load", "build", "Context", "SolverParams", "SolverStats", "StaggeredAction", "fermion_force",
    "apply_M_noalloc", "NOALLOC_MAX_VH", "fma_probe", "tuner",
]

F64, F32, F16, F64X = 0, 1, 2, 3
ABI_VERSION = 3   # include/stag.h STAG_ABI_VERSION: the struct layouts below
RECON_18, RECON_12 = 18, 12
# include/stag.h enum stag_links: the link field of the operator entry points
LINKS_UPLOADED, LINKS_TEMPORAL, LINKS_TEMPORAL_FULL = 0, 1, 2
OK, NOT_CONVERGED, BREAKDOWN = 0, 1, 2
NOALLOC_MAX_VH = 1 << 17   # include/stag.h STAG_NOALLOC_MAX_VH

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libstag.so")
_lib = None
_lock = threading.Lock()


class StagError(RuntimeError):
    """A libstag call returned a negative status."""

    def __init__(self, code, msg):
        super().__init__(f"libstag error {code}: {msg}")
        self.code = code


class NotConverged(RuntimeError):
    """A solver returned STAG_NOT_CONVERGED or STAG_BREAKDOWN (stats attached)."""

    def __init__(self, code, stats):
        super().__init__(f"solver status {code}: {stats}")
        self.code = code
        self.stats = stats


class SolverParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("check_every", ctypes.c_int), ("delta", ctypes.c_double), ("inner_prec", ctypes.c_int),
                ("inner_recon", ctypes.c_int), ("rhs_block", ctypes.c_int), ("f64_arith", ctypes.c_int),
                ("temporal_gauge", ctypes.c_int)]


class SolverStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("restarts", ctypes.c_int),
                ("reliable_updates", ctypes.c_int), ("true_rel_residual", ctypes.c_double),
                ("iter_rel_residual", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile libstag.so for sm_103a in-tree (needs nvcc)."""
    from . import _build
    return _build.build(force=force)


def _declare(lib):
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "stag_create": ([ctypes.POINTER(P), ctypes.POINTER(I), P], I),
        "stag_destroy": ([P], I),
        "stag_set_stream": ([P, P], I),
        "stag_set_operator_links": ([P, I], I),
        "stag_get_dims": ([P, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_longlong)], I),
        "stag_upload_gauge": ([P, P, I], I),
        "stag_dslash_eo": ([P, P, P, I, I], I),
        "stag_dslash_oe": ([P, P, P, I, I], I),
        "stag_apply_M": ([P, P, P, D], I),
        "stag_dslash_prepare": ([P, P, I], I),
        "stag_dslash_repeat": ([P, I, I, I], I),
        "stag_dslash_result": ([P, P], I),
        "stag_dslash_prepare_multi": ([P, P, I, I], I),
        "stag_dslash_repeat_multi": ([P, I, I, I, I], I),
        "stag_cg_update_time": ([P, I, I, P], I),
        "stag_solver_params_default": ([ctypes.POINTER(SolverParams)], None),
        "stag_cg_solve": ([P, P, P, D, ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats)], I),
        "stag_cg_solve_mixed": ([P, P, P, D, ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats)], I),
        "stag_cg_solve_shifted": ([P, P, P, D, D, ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats)], I),
        "stag_cg_solve_multi": ([P, P, P, I, D, ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats)], I),
        "stag_dslash_multi": ([P, P, P, I, I, I, I, I], I),
        "stag_last_rhs_block": ([P], I),
        "stag_cg_solve_multishift": ([P, P, P, P, I, D, ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats)], I),
        "stag_fermion_action": ([P, P, D, ctypes.POINTER(SolverParams), P, ctypes.POINTER(D),
                                 ctypes.POINTER(SolverStats)], I),
        "stag_fermion_force": ([P, P, P, P, P, D], I),
        "stag_fermion_force_multi": ([P, P, P, P, P, I], I),
        "stag_solve_full": ([P, P, P, D, ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats)], I),
        "stag_strerror": ([I], ctypes.c_char_p),
        "stag_last_error": ([], ctypes.c_char_p),
        "stag_abi_version": ([], I),
        "stag_apply_M_noalloc": ([ctypes.POINTER(I), P, P, P, D, P], I),
        "stag_fma_probe": ([I, I, ctypes.POINTER(D)], I),
        "stag_tune_make_key": ([ctypes.c_char_p, ctypes.POINTER(I), I, I, I, ctypes.c_char_p, ctypes.c_char_p, I], I),
        "stag_tune_cache_load": ([ctypes.c_char_p], I),
        "stag_tune_cache_save": ([ctypes.c_char_p], I),
        "stag_tune_cache_lookup": ([ctypes.c_char_p, ctypes.POINTER(I)], I),
        "stag_tune_cache_insert": ([ctypes.c_char_p, I], I),
        "stag_tune_cache_clear": ([], None),
        "stag_tune_stats": ([ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


def load(path: str | None = None):
    """Load libstag.so (building it first if it is missing); raises if that fails."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or _LIB_PATH
            if not os.path.exists(p):
                build()
            if not os.path.exists(p):
                raise ImportError(f"libstag.so not found at {p}; run paper_2502_03249_gb300.build()")
            lib = _declare(ctypes.CDLL(p))
            if lib.stag_abi_version() != ABI_VERSION:
                raise ImportError(f"{p} has ABI version {lib.stag_abi_version()}, this binding {ABI_VERSION}: "
                                  "rebuild with paper_2502_03249_gb300.build(force=True)")
            _lib = lib
    return _lib


def _check(rc):
    if rc < 0:
        lib = load()
        raise StagError(rc, f"{lib.stag_strerror(rc).decode()}: {lib.stag_last_error().decode()}")
    return rc


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libstag needs a CUDA device; none is available")
    return torch


class Context:
    """One lattice geometry on the current CUDA device (wraps stag_ctx)."""

    def __init__(self, dims, stream=None):
        torch = _torch()
        self._lib = load()
        self.dims = tuple(int(d) for d in dims)
        d = (ctypes.c_int * 4)(*self.dims)
        h = ctypes.c_void_p()
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        _check(self._lib.stag_create(ctypes.byref(h), d, ctypes.c_void_p(s)))
        self._h = h
        self.V = self.dims[0] * self.dims[1] * self.dims[2] * self.dims[3]
        self.Vh = self.V // 2
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.stag_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- helpers -----------------------------------------------------------
    def _sync_stream(self):
        torch = _torch()
        _check(self._lib.stag_set_stream(self._h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))

    def _field(self, t, name, n=None):
        torch = _torch()
        shape = (self.Vh, 3) if n is None else (n, self.Vh, 3)
        if not isinstance(t, torch.Tensor) or t.dtype != torch.complex128 or not t.is_cuda:
            raise TypeError(f"{name} must be a complex128 CUDA tensor")
        if tuple(t.shape) != shape or not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous with shape {shape}, got {tuple(t.shape)}")
        return ctypes.c_void_p(t.data_ptr())

    def new_half(self, n=None):
        torch = _torch()
        shape = (self.Vh, 3) if n is None else (n, self.Vh, 3)
        return torch.empty(shape, dtype=torch.complex128, device=self.device)

    # -- API -----------------------------------------------------------------
    def upload_gauge(self, U):
        """stag_upload_gauge: U complex128 (V,4,3,3), CUDA or CPU tensor."""
        torch = _torch()
        if U.dtype != torch.complex128 or tuple(U.shape) != (self.V, 4, 3, 3):
            raise ValueError("U must be complex128 with shape (V, 4, 3, 3)")
        U = U.contiguous()
        self._sync_stream()
        if U.is_cuda:
            _check(self._lib.stag_upload_gauge(self._h, ctypes.c_void_p(U.data_ptr()), 1))
        else:
            _check(self._lib.stag_upload_gauge(self._h, ctypes.c_void_p(U.data_ptr()), 0))
        self._U_keepalive = U if U.is_cuda else None

    def set_operator_links(self, links):
        """stag_set_operator_links: the link field the operator entry points apply
        (LINKS_UPLOADED, LINKS_TEMPORAL: the temporal-gauge transform read with 6
        links per site, LINKS_TEMPORAL_FULL: the same field read in full)."""
        _check(self._lib.stag_set_operator_links(self._h, int(links)))

    def dslash_eo(self, out, inp, prec=F64, recon=RECON_18):
        """stag_dslash_eo: out (even) = D_eo inp (odd)."""
        self._sync_stream()
        _check(self._lib.stag_dslash_eo(self._h, self._field(out, "out"), self._field(inp, "in"), prec, recon))
        return out

    def dslash_oe(self, out, inp, prec=F64, recon=RECON_18):
        """stag_dslash_oe: out (odd) = D_oe inp (even)."""
        self._sync_stream()
        _check(self._lib.stag_dslash_oe(self._h, self._field(out, "out"), self._field(inp, "in"), prec, recon))
        return out

    def dslash_prepare(self, inp, prec):
        """stag_dslash_prepare: convert inp once into the internal storage of prec."""
        self._sync_stream()
        _check(self._lib.stag_dslash_prepare(self._h, self._field(inp, "in"), int(prec)))

    def dslash_repeat(self, prec, recon, nrep=1):
        """stag_dslash_repeat: nrep bare operator launches on the prepared internal field."""
        self._sync_stream()
        _check(self._lib.stag_dslash_repeat(self._h, int(prec), int(recon), int(nrep)))

    def dslash_prepare_multi(self, inp, prec):
        """stag_dslash_prepare_multi: convert the multi field inp (nrhs, V/2, 3) once into internal storage."""
        self._sync_stream()
        nrhs = int(inp.shape[0])
        _check(self._lib.stag_dslash_prepare_multi(self._h, self._field(inp, "in", nrhs), nrhs, int(prec)))

    def dslash_repeat_multi(self, prec, recon, rhs_block=0, nrep=1):
        """stag_dslash_repeat_multi: nrep multi-vector operator launches on the prepared fields."""
        self._sync_stream()
        _check(self._lib.stag_dslash_repeat_multi(self._h, int(prec), int(recon), int(rhs_block), int(nrep)))

    def cg_update_time(self, f64_arith=F64X, nrep=10):
        """stag_cg_update_time: mean milliseconds per launch of the fused CG vector update."""
        self._sync_stream()
        ms = ctypes.c_double()
        _check(self._lib.stag_cg_update_time(self._h, int(f64_arith), int(nrep), ctypes.byref(ms)))
        return ms.value

    def dslash_result(self, out):
        """stag_dslash_result: the last repeat's output, converted to canonical complex128
        (out: (V/2, 3), or (nrhs, V/2, 3) after a multi prepare)."""
        self._sync_stream()
        n = int(out.shape[0]) if out.dim() == 3 else None
        _check(self._lib.stag_dslash_result(self._h, self._field(out, "out", n)))
        return out

    def apply_M(self, out, inp, mass):
        """stag_apply_M: out = (m^2 - D_eo D_oe) inp on even sites."""
        self._sync_stream()
        _check(self._lib.stag_apply_M(self._h, self._field(out, "out"), self._field(inp, "in"), float(mass)))
        return out

    @staticmethod
    def solver_params(**kw) -> SolverParams:
        p = SolverParams()
        load().stag_solver_params_default(ctypes.byref(p))
        for k, v in kw.items():
            if not hasattr(p, k):
                raise KeyError(k)
            setattr(p, k, v)
        return p

    def _solve(self, fn, x, b, mass, raise_on_fail, params):
        self._sync_stream()
        prm = self.solver_params(**params)
        st = SolverStats()
        rc = _check(fn(self._h, self._field(x, "x"), self._field(b, "b"), float(mass), ctypes.byref(prm),
                       ctypes.byref(st)))
        if rc != OK and raise_on_fail:
            raise NotConverged(rc, st.as_dict())
        return st.as_dict()

    def cg_solve(self, x, b, mass, raise_on_fail=True, **params):
        """stag_cg_solve: x = M^{-1} b (double precision CG); returns the stats dict."""
        return self._solve(self._lib.stag_cg_solve, x, b, mass, raise_on_fail, params)

    def dslash_multi(self, out, inp, out_parity, prec=F64, recon=RECON_18, rhs_block=0):
        """stag_dslash_multi: out[k] = D_{p,1-p} inp[k] for every k (links loaded once per rhs block)."""
        n = int(inp.shape[0])
        self._sync_stream()
        _check(self._lib.stag_dslash_multi(self._h, self._field(out, "out", n), self._field(inp, "in", n), n,
                                           int(out_parity), prec, recon, int(rhs_block)))
        return out

    def cg_solve_multi(self, X, B, mass, raise_on_fail=True, **params):
        """stag_cg_solve_multi: X[k] = M^{-1} B[k] for all k in one graph launch; returns a list of stats."""
        n = int(B.shape[0])
        self._sync_stream()
        prm = self.solver_params(**params)
        st = (SolverStats * n)()
        rc = _check(self._lib.stag_cg_solve_multi(self._h, self._field(X, "X", n), self._field(B, "B", n), n,
                                                  float(mass), ctypes.byref(prm), st))
        out = [s.as_dict() for s in st]
        if rc != OK and raise_on_fail:
            raise NotConverged(rc, out)
        return out

    def cg_solve_multishift(self, X, b, shifts, mass, raise_on_fail=True, **params):
        """stag_cg_solve_multishift: X[i] = (M + shifts[i])^{-1} b; returns a list of stats."""
        sh = [float(v) for v in shifts]
        n = len(sh)
        arr = (ctypes.c_double * n)(*sh)
        self._sync_stream()
        prm = self.solver_params(**params)
        st = (SolverStats * n)()
        rc = _check(self._lib.stag_cg_solve_multishift(self._h, self._field(X, "X", n), self._field(b, "b"), arr, n,
                                                       float(mass), ctypes.byref(prm), st))
        out = [s.as_dict() for s in st]
        if rc != OK and raise_on_fail:
            raise NotConverged(rc, out)
        return out

    def solve_full(self, psi, b, mass, raise_on_fail=True, **params):
        """stag_solve_full: psi = (m + D)^{-1} b on the full lattice; psi, b complex128 (V, 3)."""
        torch = _torch()
        for t, name in ((psi, "psi"), (b, "b")):
            if not isinstance(t, torch.Tensor) or t.dtype != torch.complex128 or not t.is_cuda or \
                    tuple(t.shape) != (self.V, 3) or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous complex128 CUDA tensor of shape (V, 3)")
        self._sync_stream()
        prm = self.solver_params(**params)
        st = SolverStats()
        rc = _check(self._lib.stag_solve_full(self._h, ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                              float(mass), ctypes.byref(prm), ctypes.byref(st)))
        if rc != OK and raise_on_fail:
            raise NotConverged(rc, st.as_dict())
        return st.as_dict()

    def fermion_action(self, phi, mass, X=None, raise_on_fail=True, **params):
        """stag_fermion_action: S = phi^dagger M^{-1} phi; X (M^{-1} phi) is written too. Returns (S, X, stats)."""
        X = self.new_half() if X is None else X
        self._sync_stream()
        prm = self.solver_params(**params)
        st = SolverStats()
        S = ctypes.c_double(0.0)
        rc = _check(self._lib.stag_fermion_action(self._h, self._field(phi, "phi"), float(mass), ctypes.byref(prm),
                                                  self._field(X, "X"), ctypes.byref(S), ctypes.byref(st)))
        if rc != OK and raise_on_fail:
            raise NotConverged(rc, st.as_dict())
        return S.value, X, st.as_dict()

    def fermion_force(self, X, P=None, G=None, phi_grad=None, scale=1.0):
        """stag_fermion_force: projected force P, Euclidean gradient G and dS/dphi = 2 X, times scale."""
        torch = _torch()

        def link_out(t, name):
            if t is None:
                return None
            if t.dtype != torch.complex128 or not t.is_cuda or tuple(t.shape) != (self.V, 4, 3, 3) or \
                    not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous complex128 CUDA tensor of shape (V, 4, 3, 3)")
            return ctypes.c_void_p(t.data_ptr())

        self._sync_stream()
        _check(self._lib.stag_fermion_force(self._h, link_out(P, "P"), link_out(G, "G"), self._field(X, "X"),
                                            None if phi_grad is None else self._field(phi_grad, "phi_grad"),
                                            float(scale)))
        return P, G, phi_grad

    def fermion_force_multi(self, X, coeffs, P=None, G=None):
        """stag_fermion_force_multi: P, G = sum_i coeffs[i] * force(X[i])."""
        torch = _torch()
        n = int(X.shape[0])
        c = (ctypes.c_double * n)(*[float(v) for v in coeffs])
        for t, name in ((P, "P"), (G, "G")):
            if t is not None and (t.dtype != torch.complex128 or not t.is_cuda or
                                  tuple(t.shape) != (self.V, 4, 3, 3) or not t.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous complex128 CUDA tensor of shape (V, 4, 3, 3)")
        self._sync_stream()
        _check(self._lib.stag_fermion_force_multi(
            self._h, None if P is None else ctypes.c_void_p(P.data_ptr()),
            None if G is None else ctypes.c_void_p(G.data_ptr()), self._field(X, "X", n), c, n))
        return P, G

    def last_rhs_block(self):
        """stag_last_rhs_block: rhs block of the last batched solve."""
        return int(self._lib.stag_last_rhs_block(self._h))

    def cg_solve_shifted(self, x, b, mass, sigma, raise_on_fail=True, **params):
        """stag_cg_solve_shifted: x = (M + sigma)^{-1} b (double precision CG)."""
        self._sync_stream()
        prm = self.solver_params(**params)
        st = SolverStats()
        rc = _check(self._lib.stag_cg_solve_shifted(self._h, self._field(x, "x"), self._field(b, "b"), float(mass),
                                                    float(sigma), ctypes.byref(prm), ctypes.byref(st)))
        if rc != OK and raise_on_fail:
            raise NotConverged(rc, st.as_dict())
        return st.as_dict()

    def cg_solve_mixed(self, x, b, mass, raise_on_fail=True, **params):
        """stag_cg_solve_mixed: reliable-update CG, inner precision params inner_prec / inner_recon."""
        return self._solve(self._lib.stag_cg_solve_mixed, x, b, mass, raise_on_fail, params)


def _autograd_function():
    import torch

    class _StaggeredAction(torch.autograd.Function):
        """S(U, phi) = phi^dagger M[U]^{-1} phi, M = m^2 - D_eo D_oe.

        forward: uploads U, solves X = M^{-1} phi (stag_fermion_action), returns S.
        backward: solves again for X (the solution is recomputed, not stored:
        only U and phi are saved), then stag_fermion_force gives the Euclidean
        gradient with respect to U and 2 X with respect to phi, both scaled by
        the incoming gradient of S.
        """

        @staticmethod
        def forward(fctx, U, phi, lattice, mass, params):
            lattice.upload_gauge(U.detach())
            S, _, _ = lattice.fermion_action(phi.detach().contiguous(), mass, **params)
            fctx.save_for_backward(U, phi)
            fctx.lattice, fctx.mass, fctx.params = lattice, mass, params
            return torch.tensor(S, dtype=torch.float64, device=U.device)

        @staticmethod
        def backward(fctx, gS):
            U, phi = fctx.saved_tensors
            lat = fctx.lattice
            lat.upload_gauge(U.detach())
            _, X, _ = lat.fermion_action(phi.detach().contiguous(), fctx.mass, **fctx.params)
            G = torch.empty_like(U) if fctx.needs_input_grad[0] else None
            gphi = torch.empty_like(phi) if fctx.needs_input_grad[1] else None
            if G is not None or gphi is not None:
                lat.fermion_force(X, G=G, phi_grad=gphi, scale=float(gS))
            return G, gphi, None, None, None

    return _StaggeredAction


_SA = None


def StaggeredAction(U, phi, lattice, mass, **params):
    """Differentiable S(U, phi) = phi^dagger M[U]^{-1} phi on the given Context.

    U: complex128 (V,4,3,3) CUDA tensor; phi: complex128 (V/2,3) CUDA tensor on
    even sites.  Solver keyword arguments (tol, inner_prec, ...) are passed to
    stag_fermion_action (defaults: _action_params).  The gradient with respect
    to U is the Euclidean one (dS/dRe U + i dS/dIm U)."""
    global _SA
    if _SA is None:
        _SA = _autograd_function()
    return _SA.apply(U, phi, lattice, float(mass), _action_params(params))


def _action_params(params):
    """Solver defaults of the action and its force: true residual 1e-10 by the
    mixed-precision solver (float inner iteration on 18-real links, valid for
    any complex links, double-precision reliable updates); tolerances below
    1e-11, near the double-float residual floor, use the double-precision CG."""
    params = dict(params)
    params.setdefault("tol", 1e-10)
    if "inner_prec" not in params:
        params["inner_prec"] = F32 if params["tol"] >= 1e-11 else F64
        params.setdefault("inner_recon", RECON_18)
    return params


def fermion_force(U, phi, lattice, mass, **params):
    """The projected HMC force P = TA(U G^dagger) per link, (V,4,3,3), for S = phi^dagger M^{-1} phi."""
    import torch
    lattice.upload_gauge(U)
    _, X, _ = lattice.fermion_action(phi, mass, **_action_params(params))
    P = torch.empty_like(U)
    lattice.fermion_force(X, P=P)
    return P


class tuner:
    """The library's autotuner cache (stag_tune_*): keys, file load / save,
    lookups and counters.  Needs no GPU."""

    @staticmethod
    def make_key(kernel, dims, prec, recon, nrhs, gpu):
        buf = ctypes.create_string_buffer(512)
        d = (ctypes.c_int * 4)(*(int(v) for v in dims))
        _check(load().stag_tune_make_key(kernel.encode(), d, int(prec), int(recon), int(nrhs), gpu.encode(), buf, 512))
        return buf.value.decode()

    @staticmethod
    def load(path=None):
        return _check(load().stag_tune_cache_load(None if path is None else str(path).encode()))

    @staticmethod
    def save(path=None):
        _check(load().stag_tune_cache_save(None if path is None else str(path).encode()))

    @staticmethod
    def lookup(key):
        c = ctypes.c_int()
        return c.value if _check(load().stag_tune_cache_lookup(key.encode(), ctypes.byref(c))) else None

    @staticmethod
    def insert(key, choice):
        _check(load().stag_tune_cache_insert(key.encode(), int(choice)))

    @staticmethod
    def clear():
        load().stag_tune_cache_clear()

    @staticmethod
    def stats():
        t, h = ctypes.c_longlong(), ctypes.c_longlong()
        _check(load().stag_tune_stats(ctypes.byref(t), ctypes.byref(h)))
        return {"timed": t.value, "from_cache": h.value}


def fma_probe(prec=F64, iters=None):
    """stag_fma_probe: sustained FMA throughput (TFLOP/s) of the FP64 or FP32 pipe."""
    _torch()
    if iters is None:
        iters = 2048 if prec == F64 else 32768
    v = ctypes.c_double()
    _check(load().stag_fma_probe(int(prec), int(iters), ctypes.byref(v)))
    return v.value


def apply_M_noalloc(dims, U, out, inp, mass, stream=None):
    """stag_apply_M_noalloc: out = m^2 inp - D_eo D_oe inp without any device
    allocation, for callers whose device memory is owned by their own arena.
    No context: U is the canonical (V,4,3,3) complex128 gauge field, out and inp
    are (V/2,3) complex128 even-site fields, all on the current CUDA device;
    V/2 <= NOALLOC_MAX_VH.  The intermediate lives in one static device array
    shared by every call: calls that overlap on the device must be serialised.
    Enqueued on `stream` (default: torch's current stream)."""
    torch = _torch()
    lib = load()
    dims = tuple(int(v) for v in dims)
    if len(dims) != 4 or any(v < 2 or v % 2 for v in dims):
        raise StagError(-2, f"lattice extents must be four even integers >= 2, got {dims}")
    V = dims[0] * dims[1] * dims[2] * dims[3]
    d = (ctypes.c_int * 4)(*dims)
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    cur = torch.cuda.current_device()
    for t, what, shape in ((U, "U", (V, 4, 3, 3)), (out, "out", (V // 2, 3)), (inp, "inp", (V // 2, 3))):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.complex128 or not t.is_cuda or \
                not t.is_contiguous():
            raise StagError(-1, f"{what} must be a contiguous complex128 CUDA tensor")
        if tuple(t.shape) != shape:
            raise StagError(-1, f"{what} must have shape {shape} for dims {dims}, got {tuple(t.shape)}")
        if t.device.index != cur:
            raise StagError(-1, f"{what} is on cuda:{t.device.index}, but cuda:{cur} is current")
    _check(lib.stag_apply_M_noalloc(d, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(inp.data_ptr()), float(mass), ctypes.c_void_p(s)))
    return out

"""The allocation-free operator entry point, stag_apply_M_noalloc.

Some callers cannot allocate device memory at the point where they apply the
operator: hosts that own all device memory through their own pre-sized arena
or caching allocator and forbid a library to call cudaMalloc behind it, and
latency-critical loops that cannot absorb the device-wide synchronisation
cudaFree implies.  For them the
library offers stag_apply_M_noalloc, which keeps its intermediate field in a
fixed static device array.  It must give the same result as stag_apply_M (the
context-based entry point), within the double-precision tolerance used for
the operator tests, call after call (the array is shared and reused).

This file is collected last on purpose; it also passes when run on its own in
a fresh process.
"""

import ctypes

import numpy as np
import pytest

import lattice_inputs as li
import oracle as orc

pytestmark = pytest.mark.gpu


def _fn(stag):
    lib = stag.load()
    fn = lib.stag_apply_M_noalloc
    fn.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return lib, fn


def test_noalloc_matches_apply_M_on_two_calls_in_a_row(stag):
    import torch
    lib, fn = _fn(stag)
    dims = (10, 6, 4, 6)            # V/2 = 720: several blocks and a ragged tail
    U = torch.from_numpy(li.random_links(dims, "haar", seed=701)).cuda()
    ctx = stag.Context(dims)
    ctx.upload_gauge(U)
    d = (ctypes.c_int * 4)(*dims)
    stream = torch.cuda.current_stream().cuda_stream
    for seed, mass in ((702, 0.1), (703, 0.37)):
        psi = torch.from_numpy(li.gaussian_half(dims, seed=seed)).cuda()
        ref = ctx.new_half()
        ctx.apply_M(ref, psi, mass)
        out = torch.full_like(psi, complex(float("nan"), float("nan")))
        rc = fn(d, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(psi.data_ptr()),
                mass, ctypes.c_void_p(stream))
        assert rc == 0, lib.stag_last_error()
        torch.cuda.synchronize()
        o, r = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.linalg.norm(o - r) <= 1e-12 * np.linalg.norm(r)
        # and directly against the CPU oracle's M on the same host data (the
        # links are read from the canonical layout here, so an index mistake
        # shared with the context's own link packing would show up only here)
        want = orc.apply_M(dims, U.cpu().numpy(), mass, psi.cpu().numpy())
        err = np.linalg.norm(o - want) / np.linalg.norm(want)
        assert err <= 1e-12, f"relative error against the oracle: {err:.3e}"


def test_noalloc_rejects_lattices_beyond_the_static_limit(stag):
    lib, fn = _fn(stag)
    d = (ctypes.c_int * 4)(64, 64, 64, 16)   # V/2 = 2^21 > 2^17
    assert fn(d, None, None, None, 0.1, None) == -1
    assert b"static scratch limit" in lib.stag_last_error()
    bad = (ctypes.c_int * 4)(4, 4, 3, 4)
    assert fn(bad, None, None, None, 0.1, None) == -2

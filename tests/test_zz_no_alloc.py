"""gpe_overlap_noalloc: the overlap reduction for callers that cannot allocate
device memory when they need a result (a host application whose memory pool
already holds the GPU's free memory, or a loop that must not call cudaMalloc
or cudaFree because those can synchronise the device).  Its partial sums live
in a fixed array inside the library.

Collected last on purpose.  Checks, through the C ABI, that two calls in a row
agree with gpe_overlap (the allocating entry point) and with the FP64 CPU
oracle's overlap on the same host values, to the parity tolerances used
elsewhere (1e-12 complex128, 2e-6 complex64); that a length which is not a
multiple of the per-block chunk and spans several blocks is summed whole; and
that inputs above the documented limit are refused before any GPU work.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2603_05447_gb300 import gpe, inputs

from gpu_cases import ragged_shell

CHUNK = 8192  # elements reduced by one block of the kernel


def test_noalloc_rejects_inputs_above_the_limit():
    from paper_2603_05447_gb300 import _build
    _build.build()
    out = (ctypes.c_double * 2)()
    lib = gpe.load()
    rc = lib.gpe_overlap_noalloc(ctypes.c_void_p(16), ctypes.c_void_p(16), 268435457, gpe.GPE_C64, 1.0, out, None)
    assert rc == gpe.GPE_ERR_ARG
    assert "static scratch limit" in gpe.last_error()


def _setup(torch):
    from paper_2603_05447_gb300 import _build
    _build.build()
    torch.cuda.init()
    torch.cuda.set_device(0)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,tol", [(gpe.GPE_C128, 1e-12), (gpe.GPE_C64, 2e-6)])
def test_noalloc_overlap_matches_gpe_overlap_and_oracle_twice(dtype, tol, oracle_mod):
    torch = pytest.importorskip("torch")
    _setup(torch)
    case = ragged_shell()
    grid = gpe.gpe_grid_create_dense(case.gbox, case.V, case.V_cut)
    a = gpe.gpe_state_create(grid, dtype)
    b = gpe.gpe_state_create(grid, dtype)
    try:
        cdt = np.complex128 if dtype == gpe.GPE_C128 else np.complex64
        gpe.gpe_state_load(a, np.ascontiguousarray(case.psi.astype(cdt)), gpe.GPE_LAYOUT_DENSE)
        other = inputs.random_state(case.box.shape, seed=9).astype(cdt)
        gpe.gpe_state_load(b, np.ascontiguousarray(other), gpe.GPE_LAYOUT_DENSE)
        n = gpe.gpe_grid_get_info(grid).n_packed
        # the compact arrays as the GPU holds them, for the oracle
        ha = np.empty(n, cdt)
        hb = np.empty(n, cdt)
        gpe.gpe_state_store(a, ha, gpe.GPE_LAYOUT_COMPACT)
        gpe.gpe_state_store(b, hb, gpe.GPE_LAYOUT_COMPACT)
        want = oracle.overlap(ha.astype(np.complex128), hb.astype(np.complex128), case.box.dV)
        pa, pb = gpe.gpe_state_device_ptr(a), gpe.gpe_state_device_ptr(b)
        ref = gpe.gpe_overlap(a, b)
        for _ in range(2):
            got = gpe.gpe_overlap_noalloc(pa, pb, n, dtype, case.box.dV)
            assert abs(got - ref) <= tol * abs(ref), (got, ref)
            assert abs(got - want) <= tol * abs(want), (got, want)
        # a different pair right after: the shared scratch carries nothing over
        want2 = oracle.overlap(hb.astype(np.complex128), hb.astype(np.complex128), case.box.dV)
        got2 = gpe.gpe_overlap_noalloc(pb, pb, n, dtype, case.box.dV)
        assert abs(got2 - want2) <= tol * abs(want2)
        assert abs(got2 - gpe.gpe_overlap(b, b)) <= tol * abs(want2)
    finally:
        gpe.gpe_state_destroy(a)
        gpe.gpe_state_destroy(b)
        gpe.gpe_grid_destroy(grid)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,tol", [(gpe.GPE_C128, 1e-12), (gpe.GPE_C64, 2e-6)])
def test_noalloc_overlap_ragged_length_over_several_blocks(dtype, tol, oracle_mod):
    """n = 5 chunks + 1237: the last block reduces a partial chunk; every
    element counts (a dropped tail or a doubled block would show)."""
    torch = pytest.importorskip("torch")
    _setup(torch)
    n = 5 * CHUNK + 1237
    rng = np.random.default_rng(31)
    cdt = np.complex128 if dtype == gpe.GPE_C128 else np.complex64
    # a mostly real-positive pair, so the overlap is large next to its rounding
    x = (1.0 + 0.3 * rng.standard_normal(n) + 0.2j * rng.standard_normal(n)).astype(cdt)
    y = (1.0 + 0.3 * rng.standard_normal(n) + 0.2j * rng.standard_normal(n)).astype(cdt)
    tdt = torch.complex128 if dtype == gpe.GPE_C128 else torch.complex64
    dx = torch.from_numpy(x).to("cuda", tdt)
    dy = torch.from_numpy(y).to("cuda", tdt)
    dV = 0.37
    want = oracle.overlap(x.astype(np.complex128), y.astype(np.complex128), dV)
    for _ in range(2):
        got = gpe.gpe_overlap_noalloc(dx.data_ptr(), dy.data_ptr(), n, dtype, dV)
        assert abs(got - want) <= tol * abs(want), (got, want)
    # the same arrays without their last element and without their last block
    for m in (n - 1, 5 * CHUNK):
        want_m = oracle.overlap(x[:m].astype(np.complex128), y[:m].astype(np.complex128), dV)
        got_m = gpe.gpe_overlap_noalloc(dx.data_ptr(), dy.data_ptr(), m, dtype, dV)
        assert abs(got_m - want_m) <= tol * abs(want_m), (m, got_m, want_m)

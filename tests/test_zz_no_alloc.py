"""gpe_overlap_noalloc: the overlap reduction for callers that cannot allocate
device memory (its partial sums live in a fixed array inside the library).

Collected last on purpose.  Checks, through the C ABI, that two calls in a row
agree with gpe_overlap (the allocating-at-setup entry point) to the parity
tolerances used elsewhere (1e-12 complex128, 2e-6 complex64), and that inputs
above the documented limit are refused before any GPU work.
"""
import ctypes

import numpy as np
import pytest

from paper_2603_05447_gb300 import gpe, inputs

from gpu_cases import ragged_shell


def test_noalloc_rejects_inputs_above_the_limit():
    from paper_2603_05447_gb300 import _build
    _build.build()
    out = (ctypes.c_double * 2)()
    lib = gpe.load()
    rc = lib.gpe_overlap_noalloc(ctypes.c_void_p(16), ctypes.c_void_p(16), 268435457, gpe.GPE_C64, 1.0, out, None)
    assert rc == gpe.GPE_ERR_ARG
    assert "static scratch limit" in gpe.last_error()


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,tol", [(gpe.GPE_C128, 1e-12), (gpe.GPE_C64, 2e-6)])
def test_noalloc_overlap_matches_gpe_overlap_twice(dtype, tol):
    torch = pytest.importorskip("torch")
    from paper_2603_05447_gb300 import _build
    _build.build()
    torch.cuda.init()
    torch.cuda.set_device(0)
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
        pa, pb = gpe.gpe_state_device_ptr(a), gpe.gpe_state_device_ptr(b)
        ref = gpe.gpe_overlap(a, b)
        for _ in range(2):
            got = gpe.gpe_overlap_noalloc(pa, pb, n, dtype, case.box.dV)
            assert abs(got - ref) <= tol * abs(ref), (got, ref)
        # a different pair right after: the shared scratch carries nothing over
        ref2 = gpe.gpe_overlap(b, b)
        got2 = gpe.gpe_overlap_noalloc(pb, pb, n, dtype, case.box.dV)
        assert abs(got2 - ref2) <= tol * abs(ref2)
    finally:
        gpe.gpe_state_destroy(a)
        gpe.gpe_state_destroy(b)
        gpe.gpe_grid_destroy(grid)

"""Failure detection on the GPU without faulting it: bounded waits that run
out report a status and leave the context usable; non-finite values, unstable
time steps, failed convergence and impossible allocations return error codes."""
import numpy as np
import pytest

from paper_2603_05447_gb300 import gpe, inputs

from gpu_cases import harmonic64, ragged_shell

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2603_05447_gb300 import _build
    _build.build()
    torch.cuda.init()
    torch.cuda.set_device(0)
    return gpe.load()


def test_bounded_wait_times_out_and_context_survives():
    timed_out, waited = gpe.gpe_wait_selftest(0.05)
    assert timed_out
    assert 0.04 < waited < 1.0
    # the context still works: a normal step afterwards
    case = ragged_shell()
    grid = gpe.gpe_grid_create_dense(case.gbox, case.V, case.V_cut)
    st = gpe.gpe_state_create(grid, gpe.GPE_C64)
    gpe.gpe_state_load(st, np.ascontiguousarray(case.psi.astype(np.complex64)), gpe.GPE_LAYOUT_DENSE)
    gpe.gpe_step_real(st, gpe.real_params(case.g, case.dt), 2)
    assert abs(gpe.gpe_observables(st, case.g)["norm"] - 1.0) < 1e-4
    gpe.gpe_state_destroy(st)
    gpe.gpe_grid_destroy(grid)


def test_ground_state_reports_not_converged():
    case = harmonic64()
    grid = gpe.gpe_grid_create_dense(case.gbox, case.V, case.V_cut)
    st = gpe.gpe_state_create(grid, gpe.GPE_C128)
    try:
        gpe.gpe_state_load(st, np.ascontiguousarray(case.psi), gpe.GPE_LAYOUT_DENSE)
        with pytest.raises(gpe.GpeError) as e:
            gpe.gpe_ground_state(st, gpe.gpe_imag_params(case.g, 1e-3, 1.0), 1e-300, 10, 30)
        assert e.value.code == gpe.GPE_ERR_NOT_CONVERGED
    finally:
        gpe.gpe_state_destroy(st)
        gpe.gpe_grid_destroy(grid)


def test_blowup_is_detected_as_nonfinite():
    """An unstable-but-permitted run (the check bounds only the linear part)
    grows without bound; observables then report non-finite cells."""
    case = ragged_shell()
    grid = gpe.gpe_grid_create_dense(case.gbox, case.V, case.V_cut)
    st = gpe.gpe_state_create(grid, gpe.GPE_C64)
    try:
        psi = (case.psi * 1e18).astype(np.complex64)     # |psi|^2 g far beyond the step's range
        gpe.gpe_state_load(st, np.ascontiguousarray(psi), gpe.GPE_LAYOUT_DENSE)
        gpe.gpe_step_real(st, gpe.real_params(case.g, case.dt), 40)
        with pytest.raises(gpe.GpeError) as e:
            gpe.gpe_observables(st, case.g)
        assert e.value.code == gpe.GPE_ERR_NONFINITE
    finally:
        gpe.gpe_state_destroy(st)
        gpe.gpe_grid_destroy(grid)


def test_impossible_allocation_returns_oom():
    box = gpe.make_box(8, 8, 8, 0.1)
    wl = inputs.SHELL_64
    grid = gpe.gpe_grid_create_dense(gpe.make_box(wl.n, wl.n, wl.n, wl.h),
                                     inputs.dense_potential(wl.box, wl.potential), wl.V_cut)
    try:
        # a tape with ~1e6 checkpoints of the state does not fit in device memory
        st = gpe.gpe_state_create(grid, gpe.GPE_C128)
        gpe.gpe_grid_set_potential(grid, 1, inputs.dense_potential(wl.box, wl.potential))
        p = gpe.real_params(wl.g, wl.stable_dt(), gpe.GPE_V_BLEND, [0.0, 1.0], 1.0)
        with pytest.raises(gpe.GpeError) as e:
            gpe.gpe_ramp_forward(st, p, 10 ** 9, 0.0, 1)
        assert e.value.code == gpe.GPE_ERR_OOM
        gpe.gpe_state_destroy(st)
    finally:
        gpe.gpe_grid_destroy(grid)

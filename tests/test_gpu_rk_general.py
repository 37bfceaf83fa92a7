"""GPU parity of the general memory-optimised integrators (RKHE3, RKCK; App. A)
against the oracle's Butcher-form steps.  Tolerances as for RK4: complex128
1e-12, complex64 2e-6 after one step (from the same complex64-rounded input).
"""
import numpy as np
import pytest

import oracle
from gpu_cases import harmonic64, ragged_shell, ramp_case, rel_l2
from paper_2603_05447_gb300 import gpe

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C128_TOL = 1e-12
C64_TOL_1 = 2e-6
METHODS = {"RKHE3": gpe.GPE_RKHE3, "RKCK": gpe.GPE_RKCK}


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2603_05447_gb300 import _build
    _build.build()
    torch.cuda.init()
    torch.cuda.set_device(0)
    return gpe.load()


def make(case, dtype=gpe.GPE_C128, brick=(8, 8, 8)):
    opts = gpe.make_opts(brick)
    if case.V1 is None:
        grid = gpe.gpe_grid_create_dense(case.gbox, case.V, case.V_cut, opts)
    else:
        grid = gpe.gpe_grid_create_dense(case.gbox, np.where(case.region, -1.0, 1.0), 0.0, opts)
        gpe.gpe_grid_set_potential(grid, 0, case.V)
        gpe.gpe_grid_set_potential(grid, 1, case.V1)
    st = gpe.gpe_state_create(grid, dtype)
    cdt = np.complex128 if dtype == gpe.GPE_C128 else np.complex64
    gpe.gpe_state_load(st, np.ascontiguousarray(case.psi, dtype=cdt), gpe.GPE_LAYOUT_DENSE)
    return grid, st


def dense(case, st, dtype):
    out = np.zeros(case.box.shape, np.complex128 if dtype == gpe.GPE_C128 else np.complex64)
    gpe.gpe_state_store(st, out, gpe.GPE_LAYOUT_DENSE)
    return out.astype(np.complex128)


def oracle_run(case, psi, method, nsteps, t0=0.0):
    mask = case.mask if case.V1 is None else case.region
    og = oracle.Grid(mask, (case.box.hx, case.box.hy, case.box.hz))
    y = og.compact(psi)
    V0 = og.compact(case.V)
    V1 = None if case.V1 is None else og.compact(case.V1)
    for q in range(nsteps):
        if V1 is None:
            y = oracle.rk_step(og, V0, y, case.g, t0 + q * case.dt, case.dt, method)
        else:
            y = oracle.rk_step(og, V0, y, case.g, t0 + q * case.dt, case.dt, method, V1, case.knots, case.T)
    return og.dense(y)


@pytest.mark.parametrize("method", list(METHODS))
@pytest.mark.parametrize("factory", [harmonic64, ragged_shell])
def test_static_c128_matches_oracle(method, factory):
    case = factory()
    ref = oracle_run(case, case.psi, method, 3)
    grid, st = make(case)
    try:
        gpe.gpe_step_real(st, gpe.real_params(case.g, case.dt, integrator=METHODS[method]), 3)
        assert rel_l2(dense(case, st, gpe.GPE_C128), ref) <= C128_TOL
    finally:
        gpe.gpe_state_destroy(st)
        gpe.gpe_grid_destroy(grid)


@pytest.mark.parametrize("method", list(METHODS))
def test_ramp_blend_c128_matches_oracle(method):
    case = ramp_case()
    t0 = 5 * case.dt
    ref = oracle_run(case, case.psi, method, 6, t0=t0)
    grid, st = make(case)
    try:
        p = gpe.real_params(case.g, case.dt, gpe.GPE_V_BLEND, case.knots, case.T, integrator=METHODS[method])
        gpe.gpe_step_real(st, p, 6, t0)
        assert rel_l2(dense(case, st, gpe.GPE_C128), ref) <= C128_TOL
    finally:
        gpe.gpe_state_destroy(st)
        gpe.gpe_grid_destroy(grid)


@pytest.mark.parametrize("method", list(METHODS))
@pytest.mark.parametrize("brick", [(8, 8, 4), (8, 4, 4)])
def test_c64_matches_oracle_one_step(method, brick):
    case = ragged_shell()
    grid, st = make(case, gpe.GPE_C64, brick)
    try:
        psi32 = dense(case, st, gpe.GPE_C64)   # the complex64-rounded input
        gpe.gpe_step_real(st, gpe.real_params(case.g, case.dt, integrator=METHODS[method]), 1)
        assert rel_l2(dense(case, st, gpe.GPE_C64), oracle_run(case, psi32, method, 1)) <= C64_TOL_1
    finally:
        gpe.gpe_state_destroy(st)
        gpe.gpe_grid_destroy(grid)


def test_stability_limits_per_integrator():
    """dt lambda_max between RKCK's limit (0.43) and RKHE3's (sqrt 3):
    RKCK refuses, RKHE3 and RK4 accept; above sqrt 3 only RK4 accepts."""
    case = ragged_shell()
    grid, st = make(case)
    try:
        info = gpe.gpe_grid_get_info(grid)
        b = case.box
        lam = 2 / b.hx ** 2 + 2 / b.hy ** 2 + 2 / b.hz ** 2 + info.v_max
        with pytest.raises(gpe.GpeError) as e:
            gpe.gpe_step_real(st, gpe.real_params(case.g, 1.0 / lam, integrator=gpe.GPE_RKCK), 1)
        assert e.value.code == gpe.GPE_ERR_UNSTABLE
        gpe.gpe_step_real(st, gpe.real_params(case.g, 1.0 / lam, integrator=gpe.GPE_RKHE3), 1)
        with pytest.raises(gpe.GpeError) as e:
            gpe.gpe_step_real(st, gpe.real_params(case.g, 2.0 / lam, integrator=gpe.GPE_RKHE3), 1)
        assert e.value.code == gpe.GPE_ERR_UNSTABLE
        gpe.gpe_step_real(st, gpe.real_params(case.g, 2.0 / lam), 1)
        with pytest.raises(gpe.GpeError) as e:
            gpe.gpe_step_real(st, gpe.real_params(case.g, case.dt, integrator=7), 1)
        assert e.value.code == gpe.GPE_ERR_ARG
    finally:
        gpe.gpe_state_destroy(st)
        gpe.gpe_grid_destroy(grid)

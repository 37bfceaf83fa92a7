"""The ramp gradient (discrete adjoint of the RK4 step) through the C ABI:
against the FP64 oracle's adjoint, against central finite differences, and
through torch.autograd.

Tolerances: complex128 adjoint vs oracle adjoint 1e-10 (same arithmetic,
rounding order only); finite differences h = 1e-4 to 1e-4 relative (the
target the method's gradient must meet); complex64 adjoint vs FP64 adjoint
1e-4 relative (FP32 round-off over the run, FP64 accumulation)."""
import numpy as np
import pytest

import oracle
from paper_2603_05447_gb300 import gpe, inputs

from gpu_cases import ramp_case, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NSTEPS, K = 30, 8


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2603_05447_gb300 import _build
    _build.build()
    torch.cuda.init()
    torch.cuda.set_device(0)
    return gpe.load()


@pytest.fixture(scope="module")
def problem():
    case = ramp_case()
    og = oracle.Grid(case.region, case.box.hx)
    x, y, z = case.box.coords_of(og.ijk())
    r = np.sqrt(x * x + y * y + z * z)
    tgt = np.exp(-40.0 * (r - 0.6) ** 2).astype(np.complex128)
    tgt /= np.sqrt(np.sum(np.abs(tgt) ** 2) * og.dV)
    case.target = og.dense(tgt)
    loss, grad, _ = oracle.ramp_loss_and_grad(og, og.compact(case.V), og.compact(case.V1), case.knots, case.T,
                                              case.g, case.dt, NSTEPS, og.compact(case.psi), tgt)
    return case, og, loss, grad


def blend_grid(case):
    ind = np.where(case.region, -1.0, 1.0)
    grid = gpe.gpe_grid_create_dense(case.gbox, ind, 0.0)
    gpe.gpe_grid_set_potential(grid, 0, case.V)
    gpe.gpe_grid_set_potential(grid, 1, case.V1)
    return grid


def gpu_loss_grad(case, dtype, knots, with_grad=True):
    grid = blend_grid(case)
    cdt = np.complex128 if dtype == gpe.GPE_C128 else np.complex64
    st = gpe.gpe_state_create(grid, dtype)
    tg = gpe.gpe_state_create(grid, dtype)
    tape = None
    try:
        gpe.gpe_state_load(st, np.ascontiguousarray(case.psi.astype(cdt)), gpe.GPE_LAYOUT_DENSE)
        gpe.gpe_state_load(tg, np.ascontiguousarray(case.target.astype(cdt)), gpe.GPE_LAYOUT_DENSE)
        p = gpe.real_params(case.g, case.dt, gpe.GPE_V_BLEND, knots, case.T)
        tape = gpe.gpe_ramp_forward(st, p, NSTEPS, 0.0, K)
        if not with_grad:
            return 1.0 - abs(gpe.gpe_overlap(tg, st)) ** 2, None
        loss, grad = gpe.gpe_ramp_backward(tape, tg, len(knots))
        return loss, np.array(grad)
    finally:
        if tape is not None:
            gpe.gpe_tape_destroy(tape)
        gpe.gpe_state_destroy(st)
        gpe.gpe_state_destroy(tg)
        gpe.gpe_grid_destroy(grid)


def test_c128_adjoint_matches_oracle_adjoint(problem):
    case, og, loss, grad = problem
    l, g = gpu_loss_grad(case, gpe.GPE_C128, case.knots)
    assert abs(l - loss) <= 1e-12 * abs(loss)
    assert np.max(np.abs(g - grad)) <= 1e-10 * np.max(np.abs(grad))
    assert np.max(np.abs(grad)) > 1e-8          # a non-trivial gradient


def test_c128_adjoint_matches_central_differences(problem):
    case, og, loss, grad = problem
    h = 1e-4
    for k in (2, 7, 11):
        kp, km = case.knots.copy(), case.knots.copy()
        kp[k] += h
        km[k] -= h
        lp, _ = gpu_loss_grad(case, gpe.GPE_C128, kp, with_grad=False)
        lm, _ = gpu_loss_grad(case, gpe.GPE_C128, km, with_grad=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-4 * np.max(np.abs(grad)), (k, fd, grad[k])


def test_c64_adjoint_close_to_fp64_adjoint(problem):
    case, og, loss, grad = problem
    l, g = gpu_loss_grad(case, gpe.GPE_C64, case.knots)
    assert abs(l - loss) <= 1e-5
    assert np.max(np.abs(g - grad)) <= 1e-4 * np.max(np.abs(grad))


def test_autograd_function_gives_the_adjoint_gradient(problem):
    from paper_2603_05447_gb300.autograd import RampProblem, ramp_infidelity
    case, og, loss, grad = problem
    grid = blend_grid(case)
    info = gpe.gpe_grid_get_info(grid)
    idx, i, j, k = gpe.packed_coords(grid)
    psi0 = np.zeros(info.n_packed, np.complex128)
    psi0[idx] = case.psi[k, j, i]
    tgt = np.zeros(info.n_packed, np.complex128)
    tgt[idx] = case.target[k, j, i]
    prob = RampProblem(grid, gpe.GPE_C128, psi0, tgt, case.g, case.dt, NSTEPS, case.T, K=K)
    try:
        knots = torch.tensor(case.knots, dtype=torch.float64, requires_grad=True)
        L = ramp_infidelity(knots, prob)
        L.backward()
        assert abs(L.item() - loss) <= 1e-12 * abs(loss)
        assert np.max(np.abs(knots.grad.numpy() - grad)) <= 1e-10 * np.max(np.abs(grad))
    finally:
        prob.close()
        gpe.gpe_grid_destroy(grid)

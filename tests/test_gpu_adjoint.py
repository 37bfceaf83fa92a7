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


def fd_check(grad, loss_at, knots, h=1e-4):
    """Central differences of the loss at every knot against the adjoint
    gradient, knot by knot: |fd - g_k| <= 1e-4 |g_k| + 1e-9 max |g| (the
    absolute floor covers the knots the run never reaches, whose gradient is
    exactly zero, and the FP64 rounding of the differences)."""
    floor = 1e-9 * np.max(np.abs(grad))
    for k in range(len(knots)):
        kp, km = knots.copy(), knots.copy()
        kp[k] += h
        km[k] -= h
        fd = (loss_at(kp) - loss_at(km)) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-4 * abs(grad[k]) + floor, (k, fd, grad[k])


def test_c128_adjoint_matches_central_differences_at_every_knot(problem):
    case, og, loss, grad = problem
    fd_check(grad, lambda kn: gpu_loss_grad(case, gpe.GPE_C128, kn, with_grad=False)[0], case.knots)
    # the knots inside the run carry a gradient well above the floor
    assert np.sum(np.abs(grad) > 1e-3 * np.max(np.abs(grad))) >= 8


def test_adjoint_64cubed_ramp_against_fp64_oracle_adjoint_and_differences():
    """The 64^3 version of the adjoint workload (harmonic core -> thin shell,
    g = 5000, 16 seeded monotone knots, checkpoints every K = 64 steps):
    256 RK4 steps in complex128 against the FP64 oracle's adjoint (loss 1e-12,
    gradient 1e-10 of its largest entry and 1e-8 per knot), and against
    central differences of the GPU loss at every knot (h = 1e-4, 1e-4
    relative).  The target is the initial state."""
    rw = inputs.RAMP_64
    b = rw.shell.box
    V0 = inputs.dense_potential(b, rw.v0)
    V1 = inputs.dense_potential(b, rw.shell.potential)
    region = (V0 < rw.cut0) | (V1 < rw.cut1)
    og = oracle.Grid(region, b.hx)
    x, y, z = b.coords_of(og.ijk())
    psi0 = np.sqrt(np.maximum(rw.mu0_core - rw.v0(x, y, z), 0.0)).astype(np.complex128)
    psi0 /= np.sqrt(np.sum(np.abs(psi0) ** 2) * og.dV)
    v_max = max(np.max(np.abs(og.compact(V0))), np.max(np.abs(og.compact(V1))))
    dt = 0.2 / (6.0 / b.hx ** 2 + v_max)
    nsteps, kk = 256, 64
    knots = inputs.monotone_knots(16, seed=3)
    T = nsteps * dt
    loss, grad, _ = oracle.ramp_loss_and_grad(og, og.compact(V0), og.compact(V1), knots, T, rw.shell.g, dt,
                                              nsteps, psi0, psi0)

    from gpu_cases import Case
    case = Case("ramp64", b, V0, rw.cut0, og.dense(psi0), rw.shell.g, dt, V1=V1)
    case.region, case.target, case.T = region, og.dense(psi0), T

    def run(kn, with_grad):
        grid = blend_grid(case)
        st = gpe.gpe_state_create(grid, gpe.GPE_C128)
        tg = gpe.gpe_state_create(grid, gpe.GPE_C128)
        tape = None
        try:
            gpe.gpe_state_load(st, np.ascontiguousarray(case.psi), gpe.GPE_LAYOUT_DENSE)
            gpe.gpe_state_load(tg, np.ascontiguousarray(case.target), gpe.GPE_LAYOUT_DENSE)
            tape = gpe.gpe_ramp_forward(st, gpe.real_params(case.g, dt, gpe.GPE_V_BLEND, kn, T), nsteps, 0.0, kk)
            if not with_grad:
                return 1.0 - abs(gpe.gpe_overlap(tg, st)) ** 2, None
            l_, g_ = gpe.gpe_ramp_backward(tape, tg, len(kn))
            return l_, np.array(g_)
        finally:
            if tape is not None:
                gpe.gpe_tape_destroy(tape)
            gpe.gpe_state_destroy(st)
            gpe.gpe_state_destroy(tg)
            gpe.gpe_grid_destroy(grid)

    l, g = run(knots, True)
    gmax = np.max(np.abs(grad))
    assert gmax > 0 and loss > 1e-12
    assert abs(l - loss) <= 1e-12 * abs(loss)
    assert np.max(np.abs(g - grad)) <= 1e-10 * gmax
    big = np.abs(grad) > 1e-6 * gmax
    assert np.all(np.abs(g - grad)[big] <= 1e-8 * np.abs(grad)[big])
    fd_check(grad, lambda kn: run(kn, False)[0], knots)


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

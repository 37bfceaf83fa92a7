"""The PAIR schedule (RK4 stages fused in pairs, 0+1 and 2+3, the first
stage of each pair recomputed on the brick's face halo, the state
alternating between two buffers) through the C ABI: against the FP64 oracle
at the parity tolerances of test_gpu_parity, and against the STAGED kernels,
whose per-cell arithmetic it shares (identical bits).

Cases: the harmonic trap (every cell active), the 64^3 shell, the ragged box
with unequal spacings, a single active cell, the two-potential ramp; all three
brick shapes and both brick orders; odd and even step counts (an odd count
ends in the second buffer and is copied back), CUDA-graph replay with even
and odd graph lengths."""
import numpy as np
import pytest

from paper_2603_05447_gb300 import gpe

from gpu_cases import harmonic64, shell, ragged_shell, single_cell, ramp_case, rel_l2
from test_gpu_parity import Gpu, oracle_grid, oracle_rk4, C128_TOL, C64_TOL_1, C64_TOL_10

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PAIR = gpe.GPE_SCHED_PAIR
CASES = {"harmonic64": harmonic64, "shell64": shell, "ragged": ragged_shell, "single": single_cell}


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2603_05447_gb300 import _build
    _build.build()
    torch.cuda.init()
    torch.cuda.set_device(0)
    return gpe.load()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("nsteps", [1, 10])
def test_pair_rk4_c128_matches_oracle(name, nsteps):
    case = CASES[name]()
    ref = oracle_rk4(case, oracle_grid(case), case.psi, nsteps)
    with Gpu(case, sched=PAIR) as G:
        gpe.gpe_step_real(G.state, gpe.real_params(case.g, case.dt), nsteps)
        assert rel_l2(G.dense(), ref) <= C128_TOL


@pytest.mark.parametrize("brick", [(8, 8, 8), (8, 8, 4), (8, 4, 4)])
@pytest.mark.parametrize("order", [gpe.GPE_ORDER_ZMAJOR, gpe.GPE_ORDER_MORTON])
def test_pair_rk4_brick_shapes_and_orders_match_oracle(brick, order):
    case = ragged_shell()
    ref = oracle_rk4(case, oracle_grid(case), case.psi, 3)
    with Gpu(case, brick=brick, order=order, sched=PAIR) as G:
        gpe.gpe_step_real(G.state, gpe.real_params(case.g, case.dt), 3)
        assert rel_l2(G.dense(), ref) <= C128_TOL


@pytest.mark.parametrize("name", ["harmonic64", "ragged"])
def test_pair_rk4_c64_matches_oracle(name):
    case = CASES[name]()
    og = oracle_grid(case)
    with Gpu(case, dtype=gpe.GPE_C64, brick=(8, 8, 4), sched=PAIR) as G:
        psi32 = G.dense()
        gpe.gpe_step_real(G.state, gpe.real_params(case.g, case.dt), 1)
        assert rel_l2(G.dense(), oracle_rk4(case, og, psi32, 1)) <= C64_TOL_1
        gpe.gpe_step_real(G.state, gpe.real_params(case.g, case.dt), 9)
        assert rel_l2(G.dense(), oracle_rk4(case, og, psi32, 10)) <= C64_TOL_10


@pytest.mark.parametrize("dtype", [gpe.GPE_C128, gpe.GPE_C64])
def test_pair_rk4_ramp_blend_matches_oracle_and_staged(dtype):
    case = ramp_case()
    t0 = 7 * case.dt
    p = gpe.real_params(case.g, case.dt, gpe.GPE_V_BLEND, case.knots, case.T)
    outs = []
    for sched in (gpe.GPE_SCHED_STAGED, PAIR):
        with Gpu(case, dtype=dtype, brick=(8, 8, 4), sched=sched) as G:
            gpe.gpe_step_real(G.state, p, 12, t0)
            outs.append(G.dense())
    assert np.array_equal(outs[0], outs[1])
    if dtype == gpe.GPE_C128:
        assert rel_l2(outs[1], oracle_rk4(case, oracle_grid(case), case.psi, 12, t0=t0)) <= C128_TOL


@pytest.mark.parametrize("dtype", [gpe.GPE_C128, gpe.GPE_C64])
@pytest.mark.parametrize("brick", [(8, 8, 8), (8, 8, 4), (8, 4, 4)])
@pytest.mark.parametrize("nsteps", [5, 8])
def test_pair_equals_staged_bit_for_bit(dtype, brick, nsteps):
    case = ragged_shell()
    outs = []
    for sched in (gpe.GPE_SCHED_STAGED, PAIR):
        with Gpu(case, dtype=dtype, brick=brick, sched=sched) as G:
            gpe.gpe_step_real(G.state, gpe.real_params(case.g, case.dt), nsteps)
            outs.append(G.dense())
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("graph_steps", [4, 3])
def test_pair_graph_replay_matches_eager_steps(graph_steps):
    case = shell()
    with Gpu(case, sched=PAIR, brick=(8, 8, 4)) as E, Gpu(case, sched=PAIR, brick=(8, 8, 4)) as Gr:
        gpe.gpe_state_set_graph(Gr.state, graph_steps)
        side = torch.cuda.Stream()
        p = gpe.real_params(case.g, case.dt)
        gpe.gpe_step_real(E.state, p, 19, stream=0)
        with torch.cuda.stream(side):
            gpe.gpe_step_real(Gr.state, p, 19, stream=side)
            gpe.gpe_step_real(Gr.state, p, 7, stream=side)
        torch.cuda.synchronize()
        gpe.gpe_step_real(E.state, p, 7, stream=0)
        assert np.array_equal(E.dense(), Gr.dense())


def test_pair_grid_runs_the_staged_observables():
    """Observables on a PAIR grid are the staged kernel's (imaginary time has
    its own one-pass kernel there: test_gpu_itp_fused)."""
    case = shell()
    obs = []
    for sched in (gpe.GPE_SCHED_STAGED, PAIR):
        with Gpu(case, sched=sched) as G:
            gpe.gpe_step_real(G.state, gpe.real_params(case.g, case.dt), 6)
            obs.append(gpe.gpe_observables(G.state, case.g))
    assert obs[0] == obs[1]


def test_pair_grid_serves_traces_and_the_ramp_gradient_as_staged():
    """Calls built on gpe_step_real (the observables trace, the adjoint's
    checkpointed forward run) give the same results on a PAIR grid; the
    adjoint's backward recomputation runs the staged kernels, whose bits the
    PAIR forward run reproduces."""
    case = ramp_case()
    p = gpe.real_params(case.g, case.dt, gpe.GPE_V_BLEND, case.knots, case.T)
    res = []
    for sched in (gpe.GPE_SCHED_STAGED, PAIR):
        with Gpu(case, sched=sched, brick=(8, 8, 4)) as G:
            tg = gpe.gpe_state_create(G.grid, gpe.GPE_C128)
            try:
                gpe.gpe_state_copy(tg, G.state)
                trace = gpe.gpe_step_real_traced(G.state, p, 9, 4)
                G.load(case.psi)
                tape = gpe.gpe_ramp_forward(G.state, p, 21, 0.0, 8)
                loss, grad = gpe.gpe_ramp_backward(tape, tg, 16)
                gpe.gpe_tape_destroy(tape)
            finally:
                gpe.gpe_state_destroy(tg)
            res.append((trace, loss, grad))
    assert res[0][0] == res[1][0]
    assert res[0][1] == res[1][1] and res[0][2] == res[1][2]


def test_pair_schedule_on_a_19_point_grid_runs_the_staged_19_point_step():
    case = ragged_shell()
    outs = []
    for sched in (gpe.GPE_SCHED_STAGED, PAIR):
        opts = gpe.make_opts((8, 8, 4), sched=sched, stencil=19)
        grid = gpe.gpe_grid_create_dense(case.gbox, case.V, case.V_cut, opts)
        st = gpe.gpe_state_create(grid, gpe.GPE_C128)
        try:
            gpe.gpe_state_load(st, np.ascontiguousarray(case.psi), gpe.GPE_LAYOUT_DENSE)
            gpe.gpe_step_real(st, gpe.real_params(case.g, case.dt), 3)
            out = np.zeros(case.box.shape, np.complex128)
            gpe.gpe_state_store(st, out, gpe.GPE_LAYOUT_DENSE)
            outs.append(out)
        finally:
            gpe.gpe_state_destroy(st)
            gpe.gpe_grid_destroy(grid)
    assert np.array_equal(outs[0], outs[1])

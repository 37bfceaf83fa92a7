"""The imaginary-time step in one pass (a PAIR grid: the diagonal half step
and the first Euler substep recomputed on the brick's one-cell face halo,
the state alternating between two buffers) through the C ABI: against the
FP64 oracle at the parity tolerances of test_gpu_parity, and against the
staged two-pass kernels, whose per-cell arithmetic it shares (only the norm
is summed in another order, so the renormalisation factor can differ in its
last bit).

Cases: the harmonic trap (every cell active), the 64^3 shell, the ragged box
with unequal spacings, a single active cell; all three brick shapes and both
brick orders; odd and even step counts (an odd count ends in the second
buffer and is copied back); CUDA-graph replay with even and odd graph
lengths; ground states; real states (which keep the staged kernels)."""
import numpy as np
import pytest

from paper_2603_05447_gb300 import gpe

from gpu_cases import harmonic64, shell, ragged_shell, single_cell, rel_l2
from test_gpu_parity import Gpu, oracle_grid, oracle_itp, C128_TOL, C64_TOL_1, C64_TOL_10

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


def ip(case):
    return gpe.gpe_imag_params(case.g, case.dt, 1.0)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("nsteps", [1, 20])
def test_fused_itp_c128_matches_oracle(name, nsteps):
    case = CASES[name]()
    ref = oracle_itp(case, oracle_grid(case), case.psi, nsteps)
    with Gpu(case, sched=PAIR) as G:
        gpe.gpe_step_imag(G.state, ip(case), nsteps)
        assert rel_l2(G.dense(), ref) <= C128_TOL


@pytest.mark.parametrize("brick", [(8, 8, 8), (8, 8, 4), (8, 4, 4)])
@pytest.mark.parametrize("order", [gpe.GPE_ORDER_ZMAJOR, gpe.GPE_ORDER_MORTON])
def test_fused_itp_brick_shapes_and_orders_match_oracle(brick, order):
    case = ragged_shell()
    ref = oracle_itp(case, oracle_grid(case), case.psi, 3)
    with Gpu(case, brick=brick, order=order, sched=PAIR) as G:
        gpe.gpe_step_imag(G.state, ip(case), 3)
        assert rel_l2(G.dense(), ref) <= C128_TOL


@pytest.mark.parametrize("name", ["harmonic64", "ragged", "shell64"])
def test_fused_itp_c64_matches_oracle(name):
    case = CASES[name]()
    og = oracle_grid(case)
    with Gpu(case, dtype=gpe.GPE_C64, brick=(8, 8, 4), sched=PAIR) as G:
        psi32 = G.dense()
        gpe.gpe_step_imag(G.state, ip(case), 1)
        assert rel_l2(G.dense(), oracle_itp(case, og, psi32, 1)) <= C64_TOL_1
        gpe.gpe_step_imag(G.state, ip(case), 9)
        assert rel_l2(G.dense(), oracle_itp(case, og, psi32, 10)) <= C64_TOL_10


@pytest.mark.parametrize("dtype", [gpe.GPE_C128, gpe.GPE_C64])
@pytest.mark.parametrize("brick", [(8, 8, 8), (8, 8, 4), (8, 4, 4)])
@pytest.mark.parametrize("nsteps", [5, 8])
def test_fused_itp_agrees_with_staged(dtype, brick, nsteps):
    """One step from the same state: the per-cell arithmetic is shared, the
    norms agree to the rounding of their sums (a few units in the last
    place), so the states agree to that after any number of steps."""
    case = ragged_shell()
    outs, norms = [], []
    for sched in (gpe.GPE_SCHED_STAGED, PAIR):
        with Gpu(case, dtype=dtype, brick=brick, sched=sched) as G:
            gpe.gpe_step_imag(G.state, ip(case), nsteps)
            outs.append(G.dense())
            norms.append(gpe.gpe_observables(G.state, case.g)["norm"])
    tol, ntol = (1e-14, 1e-12) if dtype == gpe.GPE_C128 else (1e-6, 1e-6)
    assert rel_l2(outs[1], outs[0]) <= tol
    assert abs(norms[0] - 1.0) <= ntol and abs(norms[1] - 1.0) <= ntol


@pytest.mark.parametrize("graph_steps", [4, 3])
def test_fused_itp_graph_replay_matches_eager_steps(graph_steps):
    case = shell()
    with Gpu(case, sched=PAIR, brick=(8, 8, 4)) as E, Gpu(case, sched=PAIR, brick=(8, 8, 4)) as Gr:
        gpe.gpe_state_set_graph(Gr.state, graph_steps)
        side = torch.cuda.Stream()
        gpe.gpe_step_imag(E.state, ip(case), 19, stream=0)
        with torch.cuda.stream(side):
            gpe.gpe_step_imag(Gr.state, ip(case), 19, stream=side)
            gpe.gpe_step_imag(Gr.state, ip(case), 7, stream=side)
        torch.cuda.synchronize()
        gpe.gpe_step_imag(E.state, ip(case), 7, stream=0)
        assert np.array_equal(E.dense(), Gr.dense())


def test_fused_itp_split_calls_equal_one_call():
    """The pending factor is applied at the end of each call, rounded as the
    next load would apply it, and the buffers are swapped back after an odd
    count: 4 + 3 steps equal 7."""
    case = ragged_shell()
    with Gpu(case, sched=PAIR, brick=(8, 8, 4)) as A, Gpu(case, sched=PAIR, brick=(8, 8, 4)) as B:
        gpe.gpe_step_imag(A.state, ip(case), 7)
        gpe.gpe_step_imag(B.state, ip(case), 3)
        gpe.gpe_step_imag(B.state, ip(case), 4)
        assert np.array_equal(A.dense(), B.dense())


def test_fused_itp_ground_state_matches_staged():
    case = harmonic64(g=30.0)
    res = []
    for sched in (gpe.GPE_SCHED_STAGED, PAIR):
        with Gpu(case, sched=sched, brick=(8, 8, 4)) as G:
            steps, obs = gpe.gpe_ground_state(G.state, gpe.gpe_imag_params(case.g, 1e-3, 1.0), 1e-9, 100, 20000)
            res.append((steps, obs, G.dense()))
    assert res[0][0] == res[1][0]
    assert abs(res[0][1]["mu"] - res[1][1]["mu"]) <= 1e-11 * abs(res[0][1]["mu"])
    assert rel_l2(res[1][2], res[0][2]) <= 1e-10


@pytest.mark.parametrize("real", [gpe.GPE_R64, gpe.GPE_R32])
def test_real_states_on_a_pair_grid_run_the_staged_pass(real):
    case = ragged_shell()
    npt = {gpe.GPE_R64: np.float64, gpe.GPE_R32: np.float32}[real]
    outs = []
    for sched in (gpe.GPE_SCHED_STAGED, PAIR):
        grid = gpe.gpe_grid_create_dense(case.gbox, case.V, case.V_cut, gpe.make_opts((8, 8, 4), sched=sched))
        st = gpe.gpe_state_create(grid, real)
        try:
            gpe.gpe_state_load(st, np.ascontiguousarray(np.abs(case.psi).astype(npt)), gpe.GPE_LAYOUT_DENSE)
            gpe.gpe_step_imag(st, ip(case), 5)
            out = np.zeros(case.box.shape, npt)
            gpe.gpe_state_store(st, out, gpe.GPE_LAYOUT_DENSE)
            outs.append(out)
        finally:
            gpe.gpe_state_destroy(st)
            gpe.gpe_grid_destroy(grid)
    assert np.array_equal(outs[0], outs[1])

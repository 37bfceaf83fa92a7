"""Degenerate layouts: boxes smaller than one brick in some or all
dimensions, down to a single cell and to lines of cells along one axis;
every cell active, anisotropic spacings.  RK4, imaginary-time steps and
observables against the FP64 oracle (complex128, 1e-12) on every brick shape,
both brick orders and the staged and fused-pair schedules."""
import pytest

import oracle
from paper_2603_05447_gb300 import gpe

from gpu_cases import tiny_box, rel_l2
from test_gpu_parity import Gpu, oracle_grid, oracle_rk4, oracle_itp, C128_TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [(1, 1, 1), (9, 1, 1), (1, 10, 1), (1, 1, 7), (3, 5, 2), (13, 3, 1)]


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2603_05447_gb300 import _build
    _build.build()
    torch.cuda.init()
    torch.cuda.set_device(0)
    return gpe.load()


@pytest.mark.parametrize("size", SIZES)
@pytest.mark.parametrize("brick", [(8, 8, 8), (8, 8, 4), (8, 4, 4)])
@pytest.mark.parametrize("sched", [gpe.GPE_SCHED_STAGED, gpe.GPE_SCHED_PAIR])
def test_tiny_box_steps_match_oracle(size, brick, sched):
    case = tiny_box(*size)
    og = oracle_grid(case)
    ref_rk = oracle_rk4(case, og, case.psi, 3)
    ref_itp = oracle_itp(case, og, case.psi, 3)
    with Gpu(case, brick=brick, sched=sched) as G:
        assert gpe.gpe_grid_get_info(G.grid).n_active == size[0] * size[1] * size[2]
        gpe.gpe_step_real(G.state, gpe.real_params(case.g, case.dt), 3)
        assert rel_l2(G.dense(), ref_rk) <= C128_TOL
        G.load(case.psi)
        gpe.gpe_step_imag(G.state, gpe.gpe_imag_params(case.g, case.dt, 1.0), 3)
        assert rel_l2(G.dense(), ref_itp) <= C128_TOL
        G.load(case.psi)
        o = gpe.gpe_observables(G.state, case.g)
    r = oracle.observables(og, og.compact(case.V), case.g, og.compact(case.psi))
    for k in ("norm", "energy", "mu", "e_kin", "e_pot", "e_int"):
        assert abs(o[k] - r[k]) <= 1e-12 * max(1.0, abs(r[k])), k


@pytest.mark.parametrize("size", [(1, 1, 1), (3, 5, 2)])
def test_tiny_box_morton_order_matches_oracle(size):
    case = tiny_box(*size)
    og = oracle_grid(case)
    with Gpu(case, brick=(8, 4, 4), order=gpe.GPE_ORDER_MORTON) as G:
        gpe.gpe_step_real(G.state, gpe.real_params(case.g, case.dt), 2)
        assert rel_l2(G.dense(), oracle_rk4(case, og, case.psi, 2)) <= C128_TOL

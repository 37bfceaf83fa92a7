"""The batch configuration at full size, in the launch configuration bench.py
times (--workload batch): the 64 seeded uneven shells (7.4e8 active cells in
all), complex64, 8x8x8 bricks (the batch autotuner's choice on these
shells), one persistent launch per kernel, graph-replayed blocks of steps.
100 imaginary-time steps of the batch against the single-state solver on
the same input for the smallest, the median and the largest shell (the
single-state path is pinned to the oracle by the parity tests, at full size
too): relative L2 1e-5 and mu to 1e-6 (complex64; the norms are summed in
another order, so the renormalisation factors differ in their last bits)."""
import numpy as np
import pytest

from paper_2603_05447_gb300 import gpe, inputs

from gpu_cases import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2603_05447_gb300 import _build
    _build.build()
    torch.cuda.init()
    torch.cuda.set_device(0)
    return gpe.load()


def test_batch_of_64_shells_matches_the_single_state_solver():
    shells = inputs.batch_shells(64)
    grids, states, psis = [], [], []
    batch = None
    try:
        for wl in shells:
            b = wl.box
            g = gpe.gpe_grid_create_analytic(gpe.make_box(b.nx, b.ny, b.nz, b.hx),
                                             gpe.make_potential(gpe.GPE_POT_ELLIPSOID_SHELL, wl.w, *wl.axes),
                                             wl.V_cut, gpe.make_opts((8, 8, 8)))
            grids.append(g)
            # the parabolic profile from the stored potential (inactive cells
            # of stored segments hold V = +inf and get 0)
            V = gpe.gpe_grid_potential(g, 0)
            psi = np.sqrt(np.maximum(wl.mu0 - V, 0.0) / wl.g).astype(np.complex64)
            st = gpe.gpe_state_create(g, gpe.GPE_C64)
            gpe.gpe_state_load(st, psi, gpe.GPE_LAYOUT_COMPACT)
            states.append(st)
            psis.append(psi)
        cells = [gpe.gpe_grid_get_info(g).n_active for g in grids]
        assert 5e8 < sum(cells) < 1e9
        batch = gpe.gpe_batch_create(states)
        params = [gpe.gpe_imag_params(wl.g, wl.stable_dt() * 20, 1.0) for wl in shells]
        rc, conv, steps, obs = gpe.gpe_batch_ground_state(batch, params, 1e-300, 50, 100, check=False)
        assert steps == [100] * 64 and not any(conv)
        order = np.argsort(cells)
        for i in (int(order[0]), int(order[32]), int(order[-1])):
            solo = gpe.gpe_state_create(grids[i], gpe.GPE_C64)
            try:
                gpe.gpe_state_load(solo, psis[i], gpe.GPE_LAYOUT_COMPACT)
                gpe.gpe_step_imag(solo, params[i], 100)
                a = np.zeros_like(psis[i])
                s = np.zeros_like(psis[i])
                gpe.gpe_state_store(states[i], a, gpe.GPE_LAYOUT_COMPACT)
                gpe.gpe_state_store(solo, s, gpe.GPE_LAYOUT_COMPACT)
                assert rel_l2(a.astype(np.complex128), s.astype(np.complex128)) <= 1e-5, i
                o = gpe.gpe_observables(solo, shells[i].g)
                assert abs(obs[i]["mu"] - o["mu"]) <= 1e-6 * abs(o["mu"]), i
                assert abs(obs[i]["norm"] - 1.0) <= 1e-6, i
            finally:
                gpe.gpe_state_destroy(solo)
    finally:
        if batch is not None:
            gpe.gpe_batch_destroy(batch)
        for st in states:
            gpe.gpe_state_destroy(st)
        for g in grids:
            gpe.gpe_grid_destroy(g)

"""Batched shells in one persistent launch, CUDA-graph step loops and the
autotuner, through the C ABI, against the FP64 oracle and the single-state
path."""
import numpy as np
import pytest

import oracle
from paper_2603_05447_gb300 import gpe, inputs

from gpu_cases import harmonic64, shell, ragged_shell, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2603_05447_gb300 import _build
    _build.build()
    torch.cuda.init()
    torch.cuda.set_device(0)
    return gpe.load()


def make(case, dtype=gpe.GPE_C128, brick=(8, 8, 8)):
    grid = gpe.gpe_grid_create_dense(case.gbox, case.V, case.V_cut, gpe.make_opts(brick))
    st = gpe.gpe_state_create(grid, dtype)
    cdt = np.complex128 if dtype == gpe.GPE_C128 else np.complex64
    gpe.gpe_state_load(st, np.ascontiguousarray(case.psi.astype(cdt)), gpe.GPE_LAYOUT_DENSE)
    return grid, st


def dense(case, st, dtype=gpe.GPE_C128):
    out = np.zeros(case.box.shape, np.complex128 if dtype == gpe.GPE_C128 else np.complex64)
    gpe.gpe_state_store(st, out, gpe.GPE_LAYOUT_DENSE)
    return out.astype(np.complex128)


def shell_cases():
    """Uneven shells: different box sizes, spacings, couplings."""
    wl2 = inputs.ShellWorkload(n=48, a_cells=20.0, g=800.0)
    c2 = shell(wl2, seed=5)
    return [shell(), ragged_shell(), c2, harmonic64(g=30.0)]


def test_batch_fixed_steps_match_oracle_per_shell():
    cases = shell_cases()
    made = [make(c) for c in cases]
    batch = gpe.gpe_batch_create([st for _, st in made])
    try:
        params = [gpe.gpe_imag_params(c.g, c.dt, 1.0) for c in cases]
        # a tolerance no shell can meet: every shell runs exactly max_steps
        rc, conv, steps, obs = gpe.gpe_batch_ground_state(batch, params, 1e-300, 5, 15, check=False)
        assert rc == gpe.GPE_ERR_NOT_CONVERGED
        assert steps == [15] * len(cases) and not any(conv)
        for c, (_, st), o in zip(cases, made, obs):
            og = oracle.Grid(c.mask, (c.box.hx, c.box.hy, c.box.hz))
            y = og.compact(c.psi)
            for _ in range(15):
                y, _ = oracle.itp_step(og, og.compact(c.V), y, c.g, c.dt, 1.0)
            assert rel_l2(dense(c, st), og.dense(y)) <= 1e-12, c.name
            ref = oracle.observables(og, og.compact(c.V), c.g, y)
            assert abs(o["mu"] - ref["mu"]) <= 1e-11 * abs(ref["mu"])
            assert abs(o["norm"] - 1.0) <= 1e-12
    finally:
        gpe.gpe_batch_destroy(batch)
        for g, st in made:
            gpe.gpe_state_destroy(st)
            gpe.gpe_grid_destroy(g)


def trap_cases():
    """Harmonic traps of uneven sizes and couplings (their ground states
    converge within a few thousand steps at dt = 1e-3)."""
    from gpu_cases import Case
    out = []
    for n, h, g in ((64, 0.25, 30.0), (48, 0.3, 100.0), (40, 0.35, 0.0)):
        box = inputs.cubic_box(n, h)
        V = inputs.dense_potential(box, inputs.Harmonic(1.0, 1.1, 0.9))
        psi = inputs.gaussian_with_noise(box, seed=n, noise=1e-3)
        out.append(Case(f"trap{n}", box, V, 12.0, psi, g, 1e-3))
    return out


@pytest.mark.parametrize("dtype", [gpe.GPE_C128, gpe.GPE_C64])
def test_batch_convergence_matches_single_state_solver(dtype):
    cases = trap_cases()
    made = [make(c, dtype) for c in cases]
    solo = [make(c, dtype) for c in cases]
    batch = gpe.gpe_batch_create([st for _, st in made])
    try:
        params = [gpe.gpe_imag_params(c.g, c.dt, 1.0) for c in cases]
        tol = 1e-7 if dtype == gpe.GPE_C128 else 1e-5
        rc, conv, steps, obs = gpe.gpe_batch_ground_state(batch, params, tol, 50, 20000)
        assert len(set(steps)) > 1                  # the shells stopped at different checks
        assert rc == gpe.GPE_OK and all(conv)
        for c, (_, st), (_, st1), n, o, p in zip(cases, made, solo, steps, obs, params):
            n1, o1 = gpe.gpe_ground_state(st1, p, tol, 50, 20000)
            assert n1 == n                       # same checks, same stopping step
            tol_mu = 1e-10 if dtype == gpe.GPE_C128 else 1e-6
            assert abs(o["mu"] - o1["mu"]) <= tol_mu * abs(o1["mu"])
            tol_l2 = 1e-10 if dtype == gpe.GPE_C128 else 1e-5
            assert rel_l2(dense(c, st, dtype), dense(c, st1, dtype)) <= tol_l2
    finally:
        gpe.gpe_batch_destroy(batch)
        for g, st in made + solo:
            gpe.gpe_state_destroy(st)
            gpe.gpe_grid_destroy(g)


@pytest.mark.parametrize("real,cplx", [(gpe.GPE_R64, gpe.GPE_C128), (gpe.GPE_R32, gpe.GPE_C64)])
def test_batch_of_real_states_matches_the_complex_batch_and_the_solo_solver(real, cplx):
    """A real starting state stays real under the imaginary-time step, so a
    batch of real states runs the complex batch's arithmetic on the real parts
    (the imaginary parts stay exactly zero): same stopping checks, same
    wavefunctions and chemical potentials.  Each shell also matches the
    single-state solver on the same real state."""
    cases = trap_cases()
    rnp = {gpe.GPE_R64: np.float64, gpe.GPE_R32: np.float32}[real]
    cnp = {gpe.GPE_C128: np.complex128, gpe.GPE_C64: np.complex64}[cplx]

    def made(dtype, npt):
        out = []
        for c in cases:
            grid = gpe.gpe_grid_create_dense(c.gbox, c.V, c.V_cut, gpe.make_opts((8, 8, 4)))
            st = gpe.gpe_state_create(grid, dtype)
            gpe.gpe_state_load(st, np.ascontiguousarray(np.abs(c.psi).astype(npt)), gpe.GPE_LAYOUT_DENSE)
            out.append((grid, st))
        return out

    def store(c, st, npt):
        out = np.zeros(c.box.shape, npt)
        gpe.gpe_state_store(st, out, gpe.GPE_LAYOUT_DENSE)
        return out.astype(np.complex128)

    R, C, solo = made(real, rnp), made(cplx, cnp), made(real, rnp)
    br = gpe.gpe_batch_create([st for _, st in R])
    bc = gpe.gpe_batch_create([st for _, st in C])
    try:
        params = [gpe.gpe_imag_params(c.g, c.dt, 1.0) for c in cases]
        tol = 1e-7 if real == gpe.GPE_R64 else 1e-5
        rc_r, conv_r, steps_r, obs_r = gpe.gpe_batch_ground_state(br, params, tol, 50, 20000)
        rc_c, conv_c, steps_c, obs_c = gpe.gpe_batch_ground_state(bc, params, tol, 50, 20000)
        assert rc_r == rc_c == gpe.GPE_OK and all(conv_r) and conv_r == conv_c
        assert steps_r == steps_c and len(set(steps_r)) > 1
        for c, (_, sr), (_, sc), (_, s1), n, orr, oc, p in zip(cases, R, C, solo, steps_r, obs_r, obs_c, params):
            a, b = store(c, sr, rnp), store(c, sc, cnp)
            assert np.abs(b.imag).max() == 0.0
            assert rel_l2(a, b) <= 1e-15
            for k in ("norm", "energy", "mu", "e_kin", "e_pot", "e_int"):
                assert abs(orr[k] - oc[k]) <= 1e-14 * max(1.0, abs(oc[k])), k
            n1, o1 = gpe.gpe_ground_state(s1, p, tol, 50, 20000)
            assert n1 == n
            tol_mu = 1e-10 if real == gpe.GPE_R64 else 1e-6
            assert abs(orr["mu"] - o1["mu"]) <= tol_mu * abs(o1["mu"])
            assert rel_l2(a, store(c, s1, rnp)) <= (1e-10 if real == gpe.GPE_R64 else 1e-5)
    finally:
        gpe.gpe_batch_destroy(br)
        gpe.gpe_batch_destroy(bc)
        for g, st in R + C + solo:
            gpe.gpe_state_destroy(st)
            gpe.gpe_grid_destroy(g)


@pytest.mark.parametrize("dtype", [gpe.GPE_C64, gpe.GPE_R32])
def test_batch_autotune_times_every_brick_shape_on_the_batch(dtype):
    """The batch tuner builds the shells in each brick shape, times the batch
    and returns the fastest; the shape it picks builds a batch that runs."""
    shells = [inputs.ShellWorkload(n=48, a_cells=18.0, g=500.0), inputs.ShellWorkload(n=64, a_cells=24.0, g=900.0),
              inputs.ShellWorkload(n=40, a_cells=14.0, g=300.0)]
    args = []
    for wl in shells:
        b = wl.box
        args.append((gpe.make_box(b.nx, b.ny, b.nz, b.hx),
                     gpe.make_potential(gpe.GPE_POT_ELLIPSOID_SHELL, wl.w, *wl.axes), wl.V_cut))
    best, allr = gpe.gpe_batch_autotune([a[0] for a in args], [a[1] for a in args], [a[2] for a in args], dtype, 10)
    assert sorted((r["bx"], r["by"], r["bz"]) for r in allr) == [(8, 4, 4), (8, 8, 4), (8, 8, 8)]
    assert all(r["ms_per_step"] > 0 and r["cell_steps_per_s"] > 0 and r["sched"] == gpe.GPE_SCHED_STAGED for r in allr)
    assert best["cell_steps_per_s"] == max(r["cell_steps_per_s"] for r in allr)
    grids = [gpe.gpe_grid_create_analytic(*a, gpe.make_opts((best["bx"], best["by"], best["bz"]))) for a in args]
    states = [gpe.gpe_state_create(g, dtype) for g in grids]
    batch = None
    try:
        for g, st, wl in zip(grids, states, shells):
            idx, i, j, k = gpe.packed_coords(g)
            b = wl.box
            npt = np.complex64 if dtype == gpe.GPE_C64 else np.float32
            psi = np.zeros(gpe.gpe_grid_get_info(g).n_packed, npt)
            psi[idx] = np.sqrt(np.maximum(wl.mu0 - wl.potential(b.x0 + i * b.hx, b.y0 + j * b.hy, b.z0 + k * b.hz),
                                          0.0) / wl.g)
            gpe.gpe_state_load(st, psi, gpe.GPE_LAYOUT_COMPACT)
        batch = gpe.gpe_batch_create(states)
        params = [gpe.gpe_imag_params(wl.g, wl.stable_dt() * 20, 1.0) for wl in shells]
        rc, conv, steps, obs = gpe.gpe_batch_ground_state(batch, params, 1e-300, 5, 10, check=False)
        assert steps == [10, 10, 10] and all(abs(o["norm"] - 1.0) < 1e-5 for o in obs)
    finally:
        if batch is not None:
            gpe.gpe_batch_destroy(batch)
        for st in states:
            gpe.gpe_state_destroy(st)
        for g in grids:
            gpe.gpe_grid_destroy(g)
    for bad in (dict(dtype=7), dict(nsteps=0)):
        kw = dict(dtype=dtype, nsteps=10)
        kw.update(bad)
        with pytest.raises(gpe.GpeError) as e:
            gpe.gpe_batch_autotune([args[0][0]], [args[0][1]], [args[0][2]], kw["dtype"], kw["nsteps"])
        assert e.value.code == gpe.GPE_ERR_ARG


def test_graph_replay_matches_eager_steps_bit_for_bit():
    case = ragged_shell()
    g1, eager = make(case)
    g2, graphed = make(case)
    try:
        gpe.gpe_state_set_graph(graphed, 4)
        side = torch.cuda.Stream()
        p = gpe.real_params(case.g, case.dt)
        gpe.gpe_step_real(eager, p, 11, stream=0)
        with torch.cuda.stream(side):
            gpe.gpe_step_real(graphed, p, 11, stream=side)      # 2 replays of 4 + 3 eager
            gpe.gpe_step_real(graphed, p, 8, stream=side)       # cached graph, 2 replays
        torch.cuda.synchronize()
        gpe.gpe_step_real(eager, p, 8, stream=0)
        assert np.array_equal(dense(case, eager), dense(case, graphed))
        ip = gpe.gpe_imag_params(case.g, case.dt, 1.0)
        gpe.gpe_step_imag(eager, ip, 9, stream=0)
        with torch.cuda.stream(side):
            gpe.gpe_step_imag(graphed, ip, 9, stream=side)
        torch.cuda.synchronize()
        assert rel_l2(dense(case, graphed), dense(case, eager)) <= 1e-15
    finally:
        for g, st in ((g1, eager), (g2, graphed)):
            gpe.gpe_state_destroy(st)
            gpe.gpe_grid_destroy(g)


def test_graph_replay_of_ramp_matches_oracle():
    from gpu_cases import ramp_case
    case = ramp_case()
    ind = np.where(case.region, -1.0, 1.0)
    grid = gpe.gpe_grid_create_dense(case.gbox, ind, 0.0)
    gpe.gpe_grid_set_potential(grid, 0, case.V)
    gpe.gpe_grid_set_potential(grid, 1, case.V1)
    st = gpe.gpe_state_create(grid, gpe.GPE_C128)
    try:
        gpe.gpe_state_load(st, np.ascontiguousarray(case.psi), gpe.GPE_LAYOUT_DENSE)
        gpe.gpe_state_set_graph(st, 5)
        side = torch.cuda.Stream()
        p = gpe.real_params(case.g, case.dt, gpe.GPE_V_BLEND, case.knots, case.T)
        t0 = 3 * case.dt
        with torch.cuda.stream(side):
            gpe.gpe_step_real(st, p, 12, t0, stream=side)
        torch.cuda.synchronize()
        og = oracle.Grid(case.region, case.box.hx)
        y = og.compact(case.psi)
        for q in range(12):
            y = oracle.rk4_step(og, og.compact(case.V), y, case.g, t0 + q * case.dt, case.dt,
                                og.compact(case.V1), case.knots, case.T)
        out = np.zeros(case.box.shape, np.complex128)
        gpe.gpe_state_store(st, out, gpe.GPE_LAYOUT_DENSE)
        assert rel_l2(out, og.dense(y)) <= 1e-12
    finally:
        gpe.gpe_state_destroy(st)
        gpe.gpe_grid_destroy(grid)


def test_autotune_returns_a_timed_valid_layout():
    wl = inputs.SHELL_96
    b = wl.box
    box = gpe.make_box(b.nx, b.ny, b.nz, b.hx)
    pot = gpe.make_potential(gpe.GPE_POT_ELLIPSOID_SHELL, wl.w, *wl.axes)
    best, allr = gpe.gpe_autotune(box, pot, wl.V_cut, gpe.GPE_C64, gpe.GPE_TUNE_REAL, 5)
    assert len(allr) == 8 and best["cell_steps_per_s"] == max(r["cell_steps_per_s"] for r in allr)
    assert any(r["sched"] == gpe.GPE_SCHED_PAIR for r in allr)
    assert (best["bx"], best["by"], best["bz"]) in {(8, 8, 8), (8, 8, 4), (8, 4, 4)}
    cached, none = gpe.gpe_autotune(box, pot, wl.V_cut, gpe.GPE_C64, gpe.GPE_TUNE_REAL, 5, timings=False)
    assert none == [] and cached == best
    # the chosen layout builds and steps
    grid = gpe.gpe_grid_create_analytic(box, pot, wl.V_cut, gpe.make_opts(
        (best["bx"], best["by"], best["bz"]), sched=best["sched"], chunk=best["chunk"]))
    st = gpe.gpe_state_create(grid, gpe.GPE_C64)
    gpe.gpe_step_real(st, gpe.real_params(wl.g, wl.stable_dt()), 2)
    gpe.gpe_state_destroy(st)
    gpe.gpe_grid_destroy(grid)


def test_autotune_takes_real_states_for_imaginary_time_only():
    wl = inputs.SHELL_64
    b = wl.box
    box = gpe.make_box(b.nx, b.ny, b.nz, b.hx)
    pot = gpe.make_potential(gpe.GPE_POT_ELLIPSOID_SHELL, wl.w, *wl.axes)
    best, allr = gpe.gpe_autotune(box, pot, wl.V_cut, gpe.GPE_R32, gpe.GPE_TUNE_IMAG, 5)
    assert len(allr) == 7 and best["cell_steps_per_s"] == max(r["cell_steps_per_s"] for r in allr)
    assert all(r["ms_per_step"] > 0 for r in allr)
    with pytest.raises(gpe.GpeError) as e:
        gpe.gpe_autotune(box, pot, wl.V_cut, gpe.GPE_R32, gpe.GPE_TUNE_REAL, 5)
    assert e.value.code == gpe.GPE_ERR_ARG


def _c4_small_states(dtype):
    """Four seeded shells of the batch family (radius scale 40 cells instead
    of 360: boxes of 76-104 cells, 1e5-2.5e5 active), parabolic initial
    profiles, 8^3 bricks, as the batch benchmark builds them."""
    shells = inputs.batch_shells(4, seed=4, scale_cells=40.0)
    made, params = [], []
    for wl in shells:
        b = wl.box
        g = gpe.gpe_grid_create_analytic(gpe.make_box(b.nx, b.ny, b.nz, b.hx),
                                         gpe.make_potential(gpe.GPE_POT_ELLIPSOID_SHELL, wl.w, *wl.axes),
                                         wl.V_cut, gpe.make_opts((8, 8, 8)))
        idx, ii, jj, kk = gpe.packed_coords(g)
        psi = np.zeros(gpe.gpe_grid_get_info(g).n_packed, np.complex128)
        psi[idx] = np.sqrt(np.maximum(wl.mu0 - wl.potential(b.x0 + ii * b.hx, b.y0 + jj * b.hy, b.z0 + kk * b.hz),
                                      0.0) / wl.g)
        st = gpe.gpe_state_create(g, dtype)
        gpe.gpe_state_load(st, np.ascontiguousarray(psi.astype(np.complex64 if dtype == gpe.GPE_C64 else
                                                                np.complex128)), gpe.GPE_LAYOUT_COMPACT)
        made.append((g, st))
        params.append(gpe.gpe_imag_params(wl.g, wl.stable_dt() * 20, 1.0))
    return shells, made, params


def test_batch_ground_states_at_dmu_1e8_and_the_complex64_floor():
    """The batch configuration's tolerance, |mu_n - mu_(n-1)| < 1e-8 between
    checks (absolute, mu in FP64), on four small shells of that family.  The
    complex128 solves converge.  The complex64 solves either converge (the
    single-precision iteration can land on an exact fixed point, |dmu| = 0)
    or stop at max_steps on their rounding floor: |dmu| between further
    checks is then at most a few FP32 units of mu (2e-7 relative).  Either
    way their mu equals the complex128 value to 1e-6 relative.  bench.py
    --workload batch measures the same floor on the large shells."""
    res = {}
    for dtype in (gpe.GPE_C128, gpe.GPE_C64):
        shells, made, params = _c4_small_states(dtype)
        batch = gpe.gpe_batch_create([st for _, st in made])
        try:
            rc, conv, steps, obs = gpe.gpe_batch_ground_state(batch, params, 1e-8, 50, 5000, check=False)
            mus = [o["mu"] for o in obs]
            if dtype == gpe.GPE_C128:
                assert rc == gpe.GPE_OK and all(conv), (conv, steps)
                assert all(n < 5000 for n in steps)
            else:
                assert rc in (gpe.GPE_OK, gpe.GPE_ERR_NOT_CONVERGED)
                for (g, st), p, wl, c, mu in zip(made, params, shells, conv, mus):
                    if c:
                        continue
                    m = []
                    for _ in range(7):
                        gpe.gpe_step_imag(st, p, 50)
                        m.append(gpe.gpe_observables(st, wl.g)["mu"])
                    floor = float(np.median(np.abs(np.diff(m))))
                    assert floor <= 2e-7 * abs(mu), (floor, mu)
            res[dtype] = mus
        finally:
            gpe.gpe_batch_destroy(batch)
            for g, st in made:
                gpe.gpe_state_destroy(st)
                gpe.gpe_grid_destroy(g)
    for m64, m128 in zip(res[gpe.GPE_C64], res[gpe.GPE_C128]):
        assert abs(m64 - m128) <= 1e-6 * abs(m128)

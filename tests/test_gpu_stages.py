"""Multi-stage potential ramps (Sec. V) on the GPU against the oracle's
stage loop: per stage the region is selected again at 5 max(mu_i, mu_{i+1})
(Thomas-Fermi mu, Eq. (5)), the wavefunction remapped, and the stage's RK4
steps blend V_i into V_{i+1}; a hold in the last potential follows.

Tolerances: complex128 1e-10 relative L2 after all stages (FP64 rounding
order over about 20 steps, as for the single-grid RK4 parity); complex64
1e-4 (complex64 RK4 drifts about 1e-6 per step from the same input).
Region sizes and step counts are integers: bit-exact."""
import numpy as np
import pytest

import oracle
from paper_2603_05447_gb300 import gpe, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2603_05447_gb300 import _build
    _build.build()
    torch.cuda.init()
    torch.cuda.set_device(0)
    return gpe.load()


BOX = inputs.Box(41, 37, 33, 0.25, 0.24, 0.26)   # ragged, unequal spacings
G, N = 5.0, 1.0
POTS = [inputs.Harmonic(2.0, 2.2, 1.8),                 # compact core
        inputs.Harmonic(1.5, 1.65, 1.35),               # looser trap
        inputs.EllipsoidShell(3.0, 1.6, 1.5, 1.4)]      # hollowed out
DURATIONS = [0.05, 0.04]
DT, T_HOLD = 0.005, 0.03


def analytic(p):
    if isinstance(p, inputs.Harmonic):
        return gpe.make_potential(gpe.GPE_POT_HARMONIC, p.wx, p.wy, p.wz)
    return gpe.make_potential(gpe.GPE_POT_ELLIPSOID_SHELL, p.w, p.a, p.b, p.c)


def gbox():
    return gpe.make_box(BOX.nx, BOX.ny, BOX.nz, BOX.hx, BOX.hy, BOX.hz)


def initial_psi(V0):
    """Thomas-Fermi profile in the first potential with a smooth phase."""
    mu = oracle.tf_mu(V0, BOX.dV, G, N)
    x, y, z = BOX.axes()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    psi = np.sqrt(np.maximum(mu - V0, 0) / G) * np.exp(0.5j * X * Y - 0.3j * Z)
    return psi / np.sqrt(np.sum(np.abs(psi) ** 2) * BOX.dV), mu


@pytest.fixture(scope="module")
def expected():
    Vs = [inputs.dense_potential(BOX, p) for p in POTS]
    psi0, mu0 = initial_psi(Vs[0])
    out, rec = oracle.ramp_stages(Vs, (BOX.hx, BOX.hy, BOX.hz), DURATIONS, G, N, DT, psi0, t_hold=T_HOLD)
    return Vs, psi0, mu0, out, rec


def run(Vs, psi0, mu0, dtype, kind, opts=None, first_brick=(8, 8, 8), integrator=gpe.GPE_RK4, dt=DT):
    cdt = np.complex128 if dtype == gpe.GPE_C128 else np.complex64
    g0 = gpe.gpe_grid_create_analytic(gbox(), analytic(POTS[0]), 5 * mu0, gpe.make_opts(first_brick))
    s0 = gpe.gpe_state_create(g0, dtype)
    try:
        gpe.gpe_state_load(s0, np.ascontiguousarray(psi0, dtype=cdt), gpe.GPE_LAYOUT_DENSE)
        pots = [analytic(p) for p in POTS] if kind == "analytic" else [np.ascontiguousarray(V) for V in Vs]
        params = gpe.stage_params(G, N, dt, 5.0, T_HOLD, integrator)
        grid, st, rep = gpe.gpe_ramp_stages(s0, pots, DURATIONS, params, opts)
    finally:
        gpe.gpe_state_destroy(s0)
        gpe.gpe_grid_destroy(g0)
    try:
        out = np.zeros(BOX.shape, cdt)
        gpe.gpe_state_store(st, out, gpe.GPE_LAYOUT_DENSE)
        info = gpe.gpe_grid_get_info(grid)
    finally:
        gpe.gpe_state_destroy(st)
        gpe.gpe_grid_destroy(grid)
    return out.astype(np.complex128), rep, info


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("kind", ["analytic", "dense"])
@pytest.mark.parametrize("dtype", [gpe.GPE_C128, gpe.GPE_C64])
def test_stages_match_the_oracle(expected, kind, dtype):
    Vs, psi0, mu0, want, rec = expected
    got, rep, info = run(Vs, psi0, mu0, dtype, kind, gpe.make_opts((8, 8, 4)))
    assert len(rep) == len(rec) == 3
    for r, o in zip(rep, rec):
        assert r["n_active"] == o["n_active"] and r["steps"] == o["steps"]
        for k in ("mu_a", "mu_b", "cut", "dt"):
            assert abs(r[k] - o[k]) <= 1e-9 * abs(o[k]), k
    tol = 1e-10 if dtype == gpe.GPE_C128 else 1e-4
    for r, o in zip(rep, rec):
        assert abs(r["norm_kept"] - o["norm_kept"]) < tol and abs(r["norm_end"] - o["norm_end"]) < tol
    assert info.n_active == rec[-1]["n_active"]
    assert all(r["regrid_s"] > 0 for r in rep)
    assert rel_l2(got, want) < tol


def test_stages_with_float32_device_potentials(expected):
    """Dense single-precision potentials already on the device (the form a
    large precomputed ramp takes): the oracle runs on the same rounded
    potentials, so regions and results match as before."""
    Vs, psi0, mu0, _, _ = expected
    Vs32 = [V.astype(np.float32).astype(np.float64) for V in Vs]
    want, rec = oracle.ramp_stages(Vs32, (BOX.hx, BOX.hy, BOX.hz), DURATIONS, G, N, DT, psi0, t_hold=T_HOLD)
    dev = [torch.from_numpy(V.astype(np.float32)).cuda() for V in Vs]
    g0 = gpe.gpe_grid_create_analytic(gbox(), analytic(POTS[0]), 5 * mu0)
    s0 = gpe.gpe_state_create(g0, gpe.GPE_C128)
    try:
        gpe.gpe_state_load(s0, np.ascontiguousarray(psi0), gpe.GPE_LAYOUT_DENSE)
        grid, st, rep = gpe.gpe_ramp_stages(s0, dev, DURATIONS, gpe.stage_params(G, N, DT, 5.0, T_HOLD))
        out = np.zeros(BOX.shape, np.complex128)
        gpe.gpe_state_store(st, out, gpe.GPE_LAYOUT_DENSE)
        gpe.gpe_state_destroy(st)
        gpe.gpe_grid_destroy(grid)
    finally:
        gpe.gpe_state_destroy(s0)
        gpe.gpe_grid_destroy(g0)
    assert [r["n_active"] for r in rep] == [o["n_active"] for o in rec]
    assert rel_l2(out, want) < 1e-10


def test_stage_regions_change_and_grid_options_are_inherited(expected):
    """The regions differ from stage to stage (the remap does work), and with
    no options the stage grids take the initial grid's brick shape."""
    Vs, psi0, mu0, want, rec = expected
    assert len({r["n_active"] for r in rec}) == 3
    got, rep, info = run(Vs, psi0, mu0, gpe.GPE_C128, "analytic", None, first_brick=(8, 4, 4))
    assert (info.bx, info.by, info.bz) == (8, 4, 4)
    assert rel_l2(got, want) < 1e-10


@pytest.mark.parametrize("method,stencil", [("RKHE3", 7), ("RKCK", 7), ("RK4", 19)])
def test_stages_with_other_integrators_and_the_19_point_stencil(expected, method, stencil):
    """The stage loop passes its integrator and the grid options through:
    RKHE3 and RKCK (App. A) and App. B's 19-point Laplacian.  RKCK takes a
    shorter step: its accepted range on the imaginary axis is narrower."""
    Vs, psi0, mu0, _, _ = expected
    dt = DT / 2 if method == "RKCK" else DT
    want, rec = oracle.ramp_stages(Vs, (BOX.hx, BOX.hy, BOX.hz), DURATIONS, G, N, dt, psi0, t_hold=T_HOLD,
                                   method=method, stencil=stencil)
    integ = {"RK4": gpe.GPE_RK4, "RKHE3": gpe.GPE_RKHE3, "RKCK": gpe.GPE_RKCK}[method]
    got, rep, info = run(Vs, psi0, mu0, gpe.GPE_C128, "analytic", gpe.make_opts((8, 8, 4), stencil=stencil),
                         integrator=integ, dt=dt)
    assert [r["n_active"] for r in rep] == [o["n_active"] for o in rec]
    assert rel_l2(got, want) < 1e-10


@pytest.mark.parametrize("sched", [gpe.GPE_SCHED_WAVE, gpe.GPE_SCHED_WAVE2])
def test_stages_on_the_wavefront_schedules_are_bit_identical(expected, sched):
    Vs, psi0, mu0, _, _ = expected
    ref, _, _ = run(Vs, psi0, mu0, gpe.GPE_C64, "analytic", gpe.make_opts((8, 8, 4)))
    got, _, _ = run(Vs, psi0, mu0, gpe.GPE_C64, "analytic", gpe.make_opts((8, 8, 4), sched=sched))
    assert np.array_equal(got, ref)


def test_stages_without_a_report_give_the_same_state(expected):
    """report = NULL skips the observables; the result is the same."""
    import ctypes
    Vs, psi0, mu0, want, rec = expected
    g0 = gpe.gpe_grid_create_analytic(gbox(), analytic(POTS[0]), 5 * mu0)
    s0 = gpe.gpe_state_create(g0, gpe.GPE_C128)
    try:
        gpe.gpe_state_load(s0, np.ascontiguousarray(psi0), gpe.GPE_LAYOUT_DENSE)
        pots = (gpe.gpe_ramp_pot * 3)()
        keep = [analytic(p) for p in POTS]
        for i, P in enumerate(keep):
            pots[i].analytic = ctypes.pointer(P)
        dur = (ctypes.c_double * 2)(*DURATIONS)
        params = gpe.stage_params(G, N, DT, 5.0, T_HOLD)
        grid, st = ctypes.c_void_p(), ctypes.c_void_p()
        rc = gpe.load().gpe_ramp_stages(s0, pots, 3, dur, ctypes.byref(params), None, ctypes.byref(grid),
                                        ctypes.byref(st), None, gpe.stream_handle())
        assert rc == gpe.GPE_OK, gpe.last_error()
        out = np.zeros(BOX.shape, np.complex128)
        gpe.gpe_state_store(st.value, out, gpe.GPE_LAYOUT_DENSE)
        gpe.gpe_state_destroy(st.value)
        gpe.gpe_grid_destroy(grid.value)
        assert rel_l2(out, want) < 1e-10
    finally:
        gpe.gpe_state_destroy(s0)
        gpe.gpe_grid_destroy(g0)


def test_stage_argument_errors(expected):
    Vs, psi0, mu0, _, _ = expected
    g0 = gpe.gpe_grid_create_analytic(gbox(), analytic(POTS[0]), 5 * mu0)
    s0 = gpe.gpe_state_create(g0, gpe.GPE_C128)
    r0 = gpe.gpe_state_create(g0, gpe.GPE_R64)
    try:
        good = gpe.stage_params(G, N, DT)
        cases = [
            (s0, [analytic(POTS[0])], [], good),                                   # one potential
            (s0, [analytic(POTS[0]), np.ascontiguousarray(Vs[1])], [0.1], good),   # mixed kinds
            (s0, [analytic(p) for p in POTS], [0.1, -1.0], good),                 # bad duration
            (s0, [analytic(p) for p in POTS], [0.1, 0.1], gpe.stage_params(G, N, 0.0)),
            (r0, [analytic(p) for p in POTS], [0.1, 0.1], good),                  # real state
        ]
        for st, pots, dur, params in cases:
            with pytest.raises(gpe.GpeError) as e:
                gpe.gpe_ramp_stages(st, pots, dur, params)
            assert e.value.code == gpe.GPE_ERR_ARG
        with pytest.raises(gpe.GpeError) as e:                                  # unstable step
            gpe.gpe_ramp_stages(s0, [analytic(p) for p in POTS], [0.1, 0.1], gpe.stage_params(G, N, 0.1))
        assert e.value.code == gpe.GPE_ERR_UNSTABLE
    finally:
        gpe.gpe_state_destroy(s0)
        gpe.gpe_state_destroy(r0)
        gpe.gpe_grid_destroy(g0)

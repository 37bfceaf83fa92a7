"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (derived from the arithmetic):
  * complex128 path: relative L2 <= 1e-12 per step (the oracle and the kernels
    evaluate the same expressions in FP64; only rounding order differs, ~1e-16
    per operation, amplified by at most dt*||H|| ~ 0.2 per step);
  * complex64 path: FP32 round-off of a handful of operations per stage,
    ~6e-8 each: relative L2 <= 2e-6 after one step, <= 1e-5 after 10 steps;
  * integer work (masks, tables, counts) is compared exactly.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_05447_gb300 import gpe, inputs

from gpu_cases import harmonic64, shell, ragged_shell, single_cell, ramp_case, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C128_TOL = 1e-12
C64_TOL_1 = 2e-6
C64_TOL_10 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2603_05447_gb300 import _build
    _build.build()
    torch.cuda.init()
    torch.cuda.set_device(0)
    return gpe.load()


class Gpu:
    """Grid + state for a case (destroyed on exit)."""

    def __init__(self, case, dtype=gpe.GPE_C128, brick=(8, 8, 8), order=gpe.GPE_ORDER_ZMAJOR,
                 mask_mode=gpe.GPE_MASK_CELL, sched=gpe.GPE_SCHED_STAGED, chunk=0):
        opts = gpe.make_opts(brick, mask_mode, order, sched, chunk)
        if case.V1 is None:
            self.grid = gpe.gpe_grid_create_dense(case.gbox, case.V, case.V_cut, opts)
        else:
            ind = np.where(case.region, -1.0, 1.0)
            self.grid = gpe.gpe_grid_create_dense(case.gbox, ind, 0.0, opts)
            gpe.gpe_grid_set_potential(self.grid, 0, case.V)
            gpe.gpe_grid_set_potential(self.grid, 1, case.V1)
        self.dtype = dtype
        self.state = gpe.gpe_state_create(self.grid, dtype)
        self.case = case
        self.load(case.psi)

    def load(self, psi):
        arr = np.ascontiguousarray(psi, dtype=np.complex128 if self.dtype == gpe.GPE_C128 else np.complex64)
        gpe.gpe_state_load(self.state, arr, gpe.GPE_LAYOUT_DENSE)

    def dense(self):
        out = np.zeros(self.case.box.shape, np.complex128 if self.dtype == gpe.GPE_C128 else np.complex64)
        gpe.gpe_state_store(self.state, out, gpe.GPE_LAYOUT_DENSE)
        return out.astype(np.complex128)

    def close(self):
        gpe.gpe_state_destroy(self.state)
        gpe.gpe_grid_destroy(self.grid)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def oracle_grid(case):
    mask = case.mask if case.V1 is None else case.region
    return oracle.Grid(mask, (case.box.hx, case.box.hy, case.box.hz))


# ----------------------------------------------------------------- grid builder
def morton_key(c):
    key = 0
    for bit in range(21):
        for ax in range(3):
            key |= ((int(c[ax]) >> bit) & 1) << (3 * bit + ax)
    return key


@pytest.mark.parametrize("brick", [(8, 8, 8), (8, 8, 4), (8, 4, 4)])
@pytest.mark.parametrize("order", [gpe.GPE_ORDER_MORTON, gpe.GPE_ORDER_ZMAJOR])
def test_grid_mask_tables_and_order(brick, order):
    case = ragged_shell()
    with Gpu(case, brick=brick, order=order) as G:
        info = gpe.gpe_grid_get_info(G.grid)
        assert info.n_active == int(case.mask.sum())
        org, nbr = gpe.gpe_grid_bricks(G.grid)
        bits = gpe.gpe_grid_mask(G.grid)
        bx, by, bz = brick
        assert info.n_stored == info.n_bricks * bx * by * bz
        # active bits -> dense active set, exactly V < V_cut
        slots = np.flatnonzero(np.unpackbits(bits.view(np.uint8), bitorder="little"))
        b, l = slots // (bx * by * bz), slots % (bx * by * bz)
        i = org[b, 0] + l % bx
        j = org[b, 1] + (l // bx) % by
        k = org[b, 2] + l // (bx * by)
        dense = np.zeros(case.box.shape, bool)
        dense[k, j, i] = True
        assert np.array_equal(dense, case.mask)
        # every brick holding an active cell is present, and only those
        bc = org // np.array(brick)
        occ = set(map(tuple, np.argwhere(case.mask)[:, ::-1] // np.array(brick)))
        assert set(map(tuple, bc)) == occ
        # neighbour table against brute force
        pos = {tuple(c): n for n, c in enumerate(bc)}
        for n, c in enumerate(bc):
            for d in range(6):
                q = list(c)
                q[d // 2] += 1 if d % 2 else -1
                assert nbr[n, d] == pos.get(tuple(q), -1)
        keys = [morton_key(c) if order == gpe.GPE_ORDER_MORTON else
                c[0] + 1000 * (c[1] + 1000 * c[2]) for c in bc]
        assert all(a < b for a, b in zip(keys, keys[1:]))


def test_brick_mask_mode_selects_whole_bricks():
    case = ragged_shell()
    with Gpu(case, mask_mode=gpe.GPE_MASK_BRICK) as G:
        info = gpe.gpe_grid_get_info(G.grid)
        bb = np.zeros(case.box.shape, bool)
        sel = np.argwhere(case.mask)[:, ::-1] // 8
        for cx, cy, cz in set(map(tuple, sel)):
            bb[cz * 8:cz * 8 + 8, cy * 8:cy * 8 + 8, cx * 8:cx * 8 + 8] = True
        assert info.n_active == int(bb.sum())


def test_analytic_builder_matches_dense_samples():
    wl = inputs.SHELL_64
    box = wl.box
    gb = gpe.make_box(box.nx, box.ny, box.nz, box.hx)
    pot = gpe.make_potential(gpe.GPE_POT_ELLIPSOID_SHELL, wl.w, *wl.axes)
    ga = gpe.gpe_grid_create_analytic(gb, pot, wl.V_cut)
    V = inputs.dense_potential(box, wl.potential)
    gd = gpe.gpe_grid_create_dense(gb, V, wl.V_cut)
    try:
        ia, id_ = gpe.gpe_grid_get_info(ga), gpe.gpe_grid_get_info(gd)
        near = np.abs(V - wl.V_cut) < 1e-9 * wl.V_cut
        assert abs(ia.n_active - id_.n_active) <= int(near.sum())
        Va, Vd = gpe.gpe_grid_potential(ga), gpe.gpe_grid_potential(gd)
        if ia.n_bricks == id_.n_bricks:
            assert np.allclose(Va, Vd, rtol=1e-13, atol=1e-12 * wl.V_cut)
    finally:
        gpe.gpe_grid_destroy(ga)
        gpe.gpe_grid_destroy(gd)


def _builder_cases():
    shell = inputs.EllipsoidShell(400.0, 1.0, 0.9, 0.8)
    return {
        # a box that is not a whole number of bricks on any axis
        "shell": (inputs.Box(70, 66, 61, 1 / 30, 1 / 30, 1 / 30), [(gpe.GPE_POT_ELLIPSOID_SHELL, shell, 40.0)]),
        "harmonic": (inputs.Box(41, 36, 45, 0.25, 0.3, 0.2), [(gpe.GPE_POT_HARMONIC, inputs.Harmonic(1.0, 1.3, 0.7), 4.0)]),
        "blend": (inputs.Box(48, 48, 48, 1 / 20, 1 / 20, 1 / 20),
                  [(gpe.GPE_POT_ELLIPSOID_SHELL, shell, 30.0),
                   (gpe.GPE_POT_ELLIPSOID_SHELL, inputs.EllipsoidShell(300.0, 0.7, 0.75, 0.6), 20.0)]),
    }


def _params(kind, pot):
    if kind == gpe.GPE_POT_HARMONIC:
        return (pot.wx, pot.wy, pot.wz)
    return (pot.w, pot.a, pot.b, pot.c)


@pytest.mark.parametrize("name", ["shell", "harmonic", "blend"])
@pytest.mark.parametrize("brick", [(8, 8, 8), (8, 8, 4)])
def test_analytic_builder_selects_exactly_the_cells_below_the_cut(name, brick):
    """Every cell with V < V_cut (of either potential for a blend) is active
    and no other, up to cells within rounding of the cut: the per-brick bound
    that skips far bricks never drops a selected cell."""
    box, pots = _builder_cases()[name]
    gb = gpe.make_box(box.nx, box.ny, box.nz, box.hx, box.hy, box.hz)
    P = [gpe.make_potential(k, *_params(k, p)) for k, p, _ in pots]
    opts = gpe.make_opts(brick)
    if len(pots) == 1:
        grid = gpe.gpe_grid_create_analytic(gb, P[0], pots[0][2], opts)
    else:
        grid = gpe.gpe_grid_create_blend(gb, P[0], pots[0][2], P[1], pots[1][2], opts)
    try:
        _, i, j, k = gpe.packed_coords(grid)
        got = np.zeros(box.shape, bool)
        got[k, j, i] = True
        want = np.zeros(box.shape, bool)
        near = np.zeros(box.shape, bool)
        for _, p, cut in pots:
            V = inputs.dense_potential(box, p)
            want |= V < cut
            near |= np.abs(V - cut) <= 1e-9 * cut
        assert want.any()
        assert not np.any((got != want) & ~near)
    finally:
        gpe.gpe_grid_destroy(grid)


def test_empty_region_and_destroy_order_errors():
    case = single_cell()
    with pytest.raises(gpe.GpeError) as e:
        gpe.gpe_grid_create_dense(case.gbox, case.V, -1.0)
    assert e.value.code == gpe.GPE_ERR_ARG
    G = Gpu(case)
    with pytest.raises(gpe.GpeError) as e:
        gpe.gpe_grid_destroy(G.grid)
    assert e.value.code == gpe.GPE_ERR_STATE
    G.close()


# ----------------------------------------------------------------- load / store
@pytest.mark.parametrize("dtype", [gpe.GPE_C128, gpe.GPE_C64])
def test_load_store_roundtrip_is_exact(dtype):
    case = ragged_shell()
    with Gpu(case, dtype=dtype) as G:
        out = G.dense()
        want = np.where(case.mask, case.psi, 0)
        if dtype == gpe.GPE_C64:
            want = want.astype(np.complex64).astype(np.complex128)
        assert np.array_equal(out, want)
        info = gpe.gpe_grid_get_info(G.grid)
        cdt = np.complex128 if dtype == gpe.GPE_C128 else np.complex64
        comp = np.zeros(info.n_packed, cdt)
        gpe.gpe_state_store(G.state, comp, gpe.GPE_LAYOUT_COMPACT)
        # the compact layout follows the documented rule
        idx, i, j, k = gpe.packed_coords(G.grid)
        assert np.array_equal(comp[idx], want[k, j, i].astype(cdt))
        pad = np.ones(info.n_packed, bool)
        pad[idx] = False
        assert np.all(comp[pad] == 0)
        assert info.n_packed % 4 == 0 and info.n_active <= info.n_packed
        V0 = gpe.gpe_grid_potential(G.grid, 0)
        assert np.all(np.isinf(V0[pad])) and np.all(np.isfinite(V0[idx]))
        junk = comp + (1.0 + 2.0j)       # inactive entries must be forced to zero on load
        gpe.gpe_state_load(G.state, np.ascontiguousarray(junk), gpe.GPE_LAYOUT_COMPACT)
        comp2 = np.zeros(info.n_packed, cdt)
        gpe.gpe_state_store(G.state, comp2, gpe.GPE_LAYOUT_COMPACT)
        assert np.all(comp2[pad] == 0)
        assert np.array_equal(comp2[idx], junk[idx])
        back = G.dense()
        assert np.array_equal(np.where(case.mask, back, 0), back)


@pytest.mark.parametrize("dtype", [gpe.GPE_C128, gpe.GPE_C64, gpe.GPE_R32])
def test_compact_load_from_page_locked_host_memory_equals_pageable(dtype):
    """Page-locked host input takes the direct copy-and-zero kernel; pageable
    input the staged copy.  Same state either way, inactive entries zero."""
    case = ragged_shell()
    grid = gpe.gpe_grid_create_dense(case.gbox, case.V, case.V_cut)
    st = gpe.gpe_state_create(grid, dtype)
    try:
        n = gpe.gpe_grid_get_info(grid).n_packed
        rng = np.random.default_rng(3)
        if dtype == gpe.GPE_R32:
            host = rng.standard_normal(n).astype(np.float32) + 1.0
        else:
            cdt = np.complex128 if dtype == gpe.GPE_C128 else np.complex64
            host = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(cdt) + 1.0
        outs = []
        for src in (np.ascontiguousarray(host), torch.from_numpy(host).pin_memory()):
            gpe.gpe_state_load(st, src, gpe.GPE_LAYOUT_COMPACT)
            out = np.zeros_like(host)
            gpe.gpe_state_store(st, out, gpe.GPE_LAYOUT_COMPACT)
            outs.append(out)
        assert np.array_equal(outs[0], outs[1])
        V = gpe.gpe_grid_potential(grid, 0)
        assert np.all(outs[1][~np.isfinite(V)] == 0) and np.array_equal(outs[1][np.isfinite(V)], host[np.isfinite(V)])
    finally:
        gpe.gpe_state_destroy(st)
        gpe.gpe_grid_destroy(grid)


# ----------------------------------------------------------------- real time
CASES = {"harmonic64": harmonic64, "shell64": shell, "ragged": ragged_shell, "single": single_cell}


def oracle_rk4(case, og, psi, nsteps, t0=0.0):
    V = og.compact(case.V)
    y = og.compact(psi)
    for q in range(nsteps):
        if case.V1 is None:
            y = oracle.rk4_step(og, V, y, case.g, t0 + q * case.dt, case.dt)
        else:
            y = oracle.rk4_step(og, V, y, case.g, t0 + q * case.dt, case.dt, og.compact(case.V1),
                                case.knots, case.T)
    return og.dense(y)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("nsteps", [1, 10])
def test_rk4_c128_matches_oracle(name, nsteps):
    case = CASES[name]()
    og = oracle_grid(case)
    ref = oracle_rk4(case, og, case.psi, nsteps)
    with Gpu(case) as G:
        gpe.gpe_step_real(G.state, gpe.real_params(case.g, case.dt), nsteps)
        assert rel_l2(G.dense(), ref) <= C128_TOL


@pytest.mark.parametrize("brick", [(8, 8, 4), (8, 4, 4)])
def test_rk4_c128_other_brick_shapes(brick):
    case = ragged_shell()
    og = oracle_grid(case)
    ref = oracle_rk4(case, og, case.psi, 3)
    with Gpu(case, brick=brick, order=gpe.GPE_ORDER_ZMAJOR) as G:
        gpe.gpe_step_real(G.state, gpe.real_params(case.g, case.dt), 3)
        assert rel_l2(G.dense(), ref) <= C128_TOL


@pytest.mark.parametrize("dtype", [gpe.GPE_C128, gpe.GPE_C64])
@pytest.mark.parametrize("order", [gpe.GPE_ORDER_ZMAJOR, gpe.GPE_ORDER_MORTON])
def test_rk4_wave_and_staged_schedules_are_bit_identical(dtype, order):
    """All schedules run the same per-cell arithmetic (no reductions), so
    every bit agrees, whatever the chunk size or brick order."""
    case = ragged_shell()
    outs = []
    for sched, chunk in [(gpe.GPE_SCHED_STAGED, 0), (gpe.GPE_SCHED_WAVE, 0), (gpe.GPE_SCHED_WAVE, 1),
                         (gpe.GPE_SCHED_WAVE, 3), (gpe.GPE_SCHED_WAVE, 64), (gpe.GPE_SCHED_WAVE2, 0),
                         (gpe.GPE_SCHED_WAVE2, 1), (gpe.GPE_SCHED_WAVE2, 5)]:
        with Gpu(case, dtype=dtype, order=order, sched=sched, chunk=chunk) as G:
            gpe.gpe_step_real(G.state, gpe.real_params(case.g, case.dt), 5)
            outs.append(G.dense())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


@pytest.mark.parametrize("chunk", [0, 1, 5])
def test_itp_wave_matches_staged(chunk):
    case = shell()
    outs = []
    for sched in (gpe.GPE_SCHED_STAGED, gpe.GPE_SCHED_WAVE, gpe.GPE_SCHED_WAVE2):
        with Gpu(case, sched=sched, chunk=chunk) as G:
            gpe.gpe_step_imag(G.state, gpe.gpe_imag_params(case.g, case.dt, 1.0), 7)
            outs.append(G.dense())
    assert rel_l2(outs[1], outs[0]) <= 1e-14
    assert rel_l2(outs[2], outs[0]) <= 1e-14


@pytest.mark.parametrize("name", ["harmonic64", "ragged"])
def test_rk4_c64_matches_oracle(name):
    case = CASES[name]()
    og = oracle_grid(case)
    with Gpu(case, dtype=gpe.GPE_C64) as G:
        psi32 = G.dense()                      # the complex64-rounded input
        gpe.gpe_step_real(G.state, gpe.real_params(case.g, case.dt), 1)
        assert rel_l2(G.dense(), oracle_rk4(case, og, psi32, 1)) <= C64_TOL_1
        gpe.gpe_step_real(G.state, gpe.real_params(case.g, case.dt), 9)
        assert rel_l2(G.dense(), oracle_rk4(case, og, psi32, 10)) <= C64_TOL_10


@pytest.mark.parametrize("name", ["harmonic64", "ragged", "shell64", "single"])
def test_rk4_c64_8x8x4_matches_oracle_and_the_8x8x8_tile_kernels(name):
    """complex64 on 8x8x4 bricks runs the register-tile stage kernels (the
    brick in the warp's registers, neighbours by shuffles); 8x8x8 bricks run
    the shared-memory tile kernels.  Same arithmetic per cell: identical
    bits, and both within the complex64 tolerance of the oracle."""
    case = CASES[name]()
    og = oracle_grid(case)
    outs = []
    for brick in ((8, 8, 4), (8, 8, 8)):
        with Gpu(case, dtype=gpe.GPE_C64, brick=brick) as G:
            psi32 = G.dense()
            gpe.gpe_step_real(G.state, gpe.real_params(case.g, case.dt), 10)
            outs.append(G.dense())
    assert rel_l2(outs[0], oracle_rk4(case, og, psi32, 10)) <= C64_TOL_10
    assert np.array_equal(outs[0], outs[1])


def test_rk4_c64_8x8x4_ramp_blend_matches_the_tile_kernels():
    case = ramp_case()
    t0 = 7 * case.dt
    outs = []
    for brick in ((8, 8, 4), (8, 8, 8)):
        with Gpu(case, dtype=gpe.GPE_C64, brick=brick) as G:
            p = gpe.real_params(case.g, case.dt, gpe.GPE_V_BLEND, case.knots, case.T)
            gpe.gpe_step_real(G.state, p, 12, t0)
            outs.append(G.dense())
    assert np.array_equal(outs[0], outs[1])


def test_rk4_ramp_blend_matches_oracle():
    case = ramp_case()
    og = oracle_grid(case)
    t0 = 7 * case.dt
    ref = oracle_rk4(case, og, case.psi, 12, t0=t0)
    with Gpu(case) as G:
        p = gpe.real_params(case.g, case.dt, gpe.GPE_V_BLEND, case.knots, case.T)
        gpe.gpe_step_real(G.state, p, 12, t0)
        assert rel_l2(G.dense(), ref) <= C128_TOL


def test_rk4_rejects_unstable_dt():
    case = harmonic64()
    with Gpu(case) as G:
        with pytest.raises(gpe.GpeError) as e:
            gpe.gpe_step_real(G.state, gpe.real_params(case.g, 0.05), 1)
        assert e.value.code == gpe.GPE_ERR_UNSTABLE
        gpe.gpe_step_real(G.state, gpe.real_params(case.g, case.dt), 0)   # zero steps: no-op
        assert np.array_equal(G.dense(), case.psi)


# ----------------------------------------------------------------- imaginary time
def oracle_itp(case, og, psi, nsteps):
    V = og.compact(case.V)
    y = og.compact(psi)
    for _ in range(nsteps):
        y, _ = oracle.itp_step(og, V, y, case.g, case.dt, 1.0)
    return og.dense(y)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("nsteps", [1, 20])
def test_itp_c128_matches_oracle(name, nsteps):
    case = CASES[name]()
    og = oracle_grid(case)
    ref = oracle_itp(case, og, case.psi, nsteps)
    with Gpu(case) as G:
        gpe.gpe_step_imag(G.state, gpe.gpe_imag_params(case.g, case.dt, 1.0), nsteps)
        assert rel_l2(G.dense(), ref) <= C128_TOL


def test_itp_c64_matches_oracle():
    case = shell()
    og = oracle_grid(case)
    with Gpu(case, dtype=gpe.GPE_C64) as G:
        psi32 = G.dense()
        gpe.gpe_step_imag(G.state, gpe.gpe_imag_params(case.g, case.dt, 1.0), 10)
        assert rel_l2(G.dense(), oracle_itp(case, og, psi32, 10)) <= C64_TOL_10


def test_ground_state_harmonic_g0_energy():
    """g = 0, 64^3, h = 0.25: E -> 3 lambda_min(1D) = 1.4941174639 up to the
    O(dt^2) splitting bias of the ITP fixed point."""
    case = harmonic64(g=0.0)
    with Gpu(case) as G:
        p = gpe.gpe_imag_params(0.0, 1e-3, 1.0)
        steps, obs = gpe.gpe_ground_state(G.state, p, 1e-12, 500, 60000)
        assert abs(obs["energy"] - 1.4941174639) < 2e-6
        assert abs(obs["mu"] - obs["energy"]) < 1e-9
        assert abs(obs["norm"] - 1.0) < 1e-12


# ----------------------------------------------------------------- observables
@pytest.mark.parametrize("name", ["harmonic64", "ragged"])
@pytest.mark.parametrize("dtype", [gpe.GPE_C128, gpe.GPE_C64])
def test_observables_match_oracle(name, dtype):
    case = CASES[name]()
    og = oracle_grid(case)
    with Gpu(case, dtype=dtype) as G:
        psi = G.dense()
        ref = oracle.observables(og, og.compact(case.V), case.g, og.compact(psi))
        got = gpe.gpe_observables(G.state, case.g)
        tol = 1e-12 if dtype == gpe.GPE_C128 else 2e-6
        for k in ("norm", "energy", "mu", "e_kin", "e_pot", "e_int"):
            assert abs(got[k] - ref[k]) <= tol * max(abs(ref[k]), 1e-300) + 1e-300, (k, got[k], ref[k])
        assert got["nonfinite"] == 0


def test_observables_report_nonfinite():
    case = ragged_shell()
    psi = case.psi.copy()
    idx = np.argwhere(case.mask)[:3]
    for k, j, i in idx:
        psi[k, j, i] = np.nan
    with Gpu(case) as G:
        G.load(psi)
        with pytest.raises(gpe.GpeError) as e:
            gpe.gpe_observables(G.state, case.g)
        assert e.value.code == gpe.GPE_ERR_NONFINITE
        assert gpe.gpe_observables(G.state, case.g, check=False)["nonfinite"] == 3


def test_overlap_matches_oracle():
    case = ragged_shell()
    og = oracle_grid(case)
    with Gpu(case) as A:
        B = gpe.gpe_state_create(A.grid, gpe.GPE_C128)
        try:
            other = inputs.random_state(case.box.shape, seed=9)
            gpe.gpe_state_load(B, np.ascontiguousarray(other), gpe.GPE_LAYOUT_DENSE)
            got = gpe.gpe_overlap(A.state, B)
            ref = oracle.overlap(og.compact(case.psi), og.compact(other), og.dV)
            assert abs(got - ref) <= 1e-12 * abs(ref)
        finally:
            gpe.gpe_state_destroy(B)


def test_tf_mu_matches_oracle():
    box = inputs.cubic_box(80, 0.1)
    V = inputs.dense_potential(box, inputs.Harmonic())
    gb = gpe.make_box(80, 80, 80, 0.1)
    mu_gpu = gpe.gpe_tf_mu_dense(gb, V, 500.0, 1.0)
    mu_orc = oracle.tf_mu(V, box.dV, 500.0, 1.0)
    assert abs(mu_gpu - mu_orc) <= 1e-10 * mu_orc
    pot = gpe.make_potential(gpe.GPE_POT_HARMONIC, 1, 1, 1)
    mu_an = gpe.gpe_tf_mu_analytic(gb, pot, 500.0, 1.0)
    assert abs(mu_an - mu_orc) <= 1e-10 * mu_orc


def test_tf_mu_closed_forms():
    """A flat potential V = c fills the box: mu = c + g N / (n dV).  A
    potential of two levels puts every atom on the lower level while
    mu - lo < hi - lo."""
    box = inputs.Box(37, 29, 23, 0.3, 0.25, 0.2)
    gb = gpe.make_box(box.nx, box.ny, box.nz, box.hx, box.hy, box.hz)
    n = box.nx * box.ny * box.nz
    V = np.full(box.shape, 1.75)
    mu = gpe.gpe_tf_mu_dense(gb, V, 3.0, 2.0)
    assert abs(mu - (1.75 + 3.0 * 2.0 / (n * box.dV))) <= 1e-14 * mu
    V2 = np.where(np.arange(n).reshape(box.shape) % 3 == 0, 0.5, 1e6)
    m = np.count_nonzero(V2 == 0.5)
    mu2 = gpe.gpe_tf_mu_dense(gb, V2, 3.0, 2.0)
    assert abs(mu2 - (0.5 + 3.0 * 2.0 / (m * box.dV))) <= 1e-14 * mu2


def test_blend_dense_grid_is_the_union_of_both_regions():
    box = inputs.Box(45, 39, 35, 0.25, 0.25, 0.25)
    gb = gpe.make_box(box.nx, box.ny, box.nz, box.hx, box.hy, box.hz)
    V0 = inputs.dense_potential(box, inputs.Harmonic(2.0, 2.2, 1.8))
    V1 = inputs.dense_potential(box, inputs.EllipsoidShell(3.0, 1.6, 1.5, 1.4))
    grid = gpe.gpe_grid_create_blend_dense(gb, V0, V1, 6.0, 2.0, gpe.make_opts((8, 8, 4)))
    try:
        info = gpe.gpe_grid_get_info(grid)
        region = (V0 < 6.0) | (V1 < 2.0)
        assert info.n_active == np.count_nonzero(region) and info.n_slots == 2
        idx, i, j, k = gpe.packed_coords(grid)
        assert np.array_equal(np.sort(i + box.nx * (j + box.ny * k)), np.flatnonzero(region.ravel()))
        for slot, V in ((0, V0), (1, V1)):
            assert np.array_equal(gpe.gpe_grid_potential(grid, slot)[idx], V[k, j, i])
        assert info.v_max == max(V0[region].max(), V1[region].max())
    finally:
        gpe.gpe_grid_destroy(grid)


@pytest.mark.parametrize("name", ["SHELL_64", "SHELL_96"])
def test_tf_mu_on_shells_matches_oracle_and_holds_N_atoms(name):
    wl = getattr(inputs, name)
    b = wl.box
    gb = gpe.make_box(b.nx, b.ny, b.nz, b.hx)
    V = inputs.dense_potential(b, wl.potential)
    mu_orc = oracle.tf_mu(V, b.dV, wl.g, wl.N)
    pot = gpe.make_potential(gpe.GPE_POT_ELLIPSOID_SHELL, wl.w, *wl.axes)
    for mu in (gpe.gpe_tf_mu_dense(gb, V, wl.g, wl.N), gpe.gpe_tf_mu_analytic(gb, pot, wl.g, wl.N),
               gpe.gpe_tf_mu_dense(gb, np.ascontiguousarray(V.astype(np.float32)), wl.g, wl.N)):
        assert abs(mu - mu_orc) <= 1e-6 * mu_orc
    mu = gpe.gpe_tf_mu_dense(gb, V, wl.g, wl.N)
    assert abs(mu - mu_orc) <= 1e-12 * mu_orc
    assert abs(np.sum(np.maximum(mu - V, 0)) / wl.g * b.dV - wl.N) < 1e-10


# ----------------------------------------------------------------- checkpoint / resume
@pytest.mark.parametrize("dtype", [gpe.GPE_C128, gpe.GPE_C64])
def test_checkpoint_and_resume_are_bit_exact(dtype):
    """A compact-layout dump taken between calls and loaded into a fresh
    state on a fresh grid continues the run bit for bit: RK4 with a static
    potential, and imaginary time (the pending renormalisation is applied
    when a call's work completes, and a factor of one on the next load is
    exact).  A ramped potential resumes at the right time but not bit for
    bit: t0 + k dt and the uninterrupted run's time can differ in the last
    bit."""
    case = ragged_shell()
    p = gpe.real_params(case.g, case.dt)
    q = gpe.gpe_imag_params(case.g, case.dt, 1.0)
    with Gpu(case, dtype) as A:
        gpe.gpe_step_real(A.state, p, 12, 0.0)
        gpe.gpe_step_imag(A.state, q, 6)
        straight = A.dense()
    with Gpu(case, dtype) as A:
        gpe.gpe_step_real(A.state, p, 5, 0.0)
        info = gpe.gpe_grid_get_info(A.grid)
        dump = np.zeros(info.n_packed, np.complex128 if dtype == gpe.GPE_C128 else np.complex64)
        gpe.gpe_state_store(A.state, dump, gpe.GPE_LAYOUT_COMPACT)
        with Gpu(case, dtype) as B:
            gpe.gpe_state_load(B.state, dump, gpe.GPE_LAYOUT_COMPACT)
            gpe.gpe_step_real(B.state, p, 7, 5 * case.dt)
            gpe.gpe_step_imag(B.state, q, 2)
            gpe.gpe_state_store(B.state, dump, gpe.GPE_LAYOUT_COMPACT)
            gpe.gpe_state_load(A.state, dump, gpe.GPE_LAYOUT_COMPACT)
            gpe.gpe_step_imag(A.state, q, 4)
            resumed = A.dense()
    assert np.array_equal(resumed, straight)


# ----------------------------------------------------------------- observables trace
def test_traced_steps_equal_separate_calls_and_the_oracle():
    case = ragged_shell()
    p = gpe.real_params(case.g, case.dt)
    with Gpu(case) as A:
        log = gpe.gpe_step_real_traced(A.state, p, 10, 4)
    with Gpu(case) as B:
        sep = []
        for n in (4, 4, 2):
            gpe.gpe_step_real(B.state, p, n)
            sep.append(gpe.gpe_observables(B.state, case.g))
    assert log == sep
    og = oracle_grid(case)
    y, V = og.compact(case.psi), og.compact(case.V)
    for _ in range(10):
        y = oracle.rk4_step(og, V, y, case.g, 0.0, case.dt)
    o = oracle.observables(og, V, case.g, y)
    for k in ("norm", "energy", "mu"):
        assert abs(log[-1][k] - o[k]) <= 1e-12 * abs(o[k]), k


def test_traced_ramp_uses_the_blend_at_each_trace_time():
    case = ramp_case()
    p = gpe.real_params(case.g, case.dt, gpe.GPE_V_BLEND, case.knots, case.T)
    with Gpu(case) as A:
        log = gpe.gpe_step_real_traced(A.state, p, 9, 3, t0=0.5 * case.dt)
    with Gpu(case) as B:
        for i, n in enumerate((3, 3, 3)):
            gpe.gpe_step_real(B.state, p, n, 0.5 * case.dt + 3 * i * case.dt)
            s = oracle.ramp_s(case.knots, case.T, 0.5 * case.dt + 3 * (i + 1) * case.dt)
            o = gpe.gpe_observables(B.state, case.g, s)
            for k in ("norm", "e_kin", "e_pot", "e_int"):
                assert abs(log[i][k] - o[k]) <= 1e-14 * abs(o[k]), (i, k)


def test_traced_steps_stop_at_a_nonfinite_point():
    case = ragged_shell()
    psi = case.psi.copy()
    k, j, i = np.argwhere(case.mask)[len(np.argwhere(case.mask)) // 2]
    psi[k, j, i] = np.nan
    with Gpu(case) as A:
        A.load(psi)
        with pytest.raises(gpe.GpeError) as e:
            gpe.gpe_step_real_traced(A.state, gpe.real_params(case.g, case.dt), 10, 4)
        assert e.value.code == gpe.GPE_ERR_NONFINITE
        log = gpe.gpe_step_real_traced(A.state, gpe.real_params(case.g, case.dt), 10, 4, check=False)
        assert len(log) == 1 and log[0]["nonfinite"] > 0

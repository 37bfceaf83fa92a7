"""Parity at the headline size, in the launch configuration bench.py times
(1024^3 shell, ~2.9e7 active cells, the bench's brick shape, z-major order,
staged schedule): one GPU step on the whole grid, then sampled active cells compared
with the FP64 oracle run on the 11^3 patch around each sample.  One RK4 step
applies the stencil four times, so a cell's new value depends only on cells
within 4 of it and the patch (half-width 5) reproduces it exactly.

The oracle is fed the potential evaluated on the host in FP64 from the
workload's formula (not the potential the device builder produced), and every
sampled patch also checks the builder: the region of interest equals
{V_host < V_cut} cell by cell and the stored potential equals V_host.

Tolerances as in test_gpu_parity: complex128 1e-12, complex64 2e-6, relative
to the largest |psi| of the patch.  The imaginary-time step renormalises
globally; the samples are compared up to one common factor, which must be the
same for every sample.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_05447_gb300 import gpe, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HALF = 5
NSAMPLE = 300


@pytest.fixture(scope="module")
def big():
    from paper_2603_05447_gb300 import _build
    _build.build()
    torch.cuda.init()
    torch.cuda.set_device(0)
    import bench
    wl = inputs.SHELL_1024
    grid = bench.build_grid(gpe, wl)
    psi0 = bench.initial_compact(gpe, inputs, wl, grid)
    info = gpe.gpe_grid_get_info(grid)
    org, _ = gpe.gpe_grid_bricks(grid)
    bits = gpe.gpe_grid_mask(grid)
    V = gpe.gpe_grid_potential(grid, 0)
    bc = info.bx * info.by * info.bz
    act = np.unpackbits(bits.view(np.uint8), bitorder="little").astype(bool).reshape(info.n_bricks, bc)
    seg = act.reshape(info.n_bricks, bc // 4, 4).any(axis=2)
    off = 4 * np.concatenate([[0], np.cumsum(seg.sum(axis=1))[:-1]]).astype(np.int64)
    rank = np.cumsum(seg, axis=1) - 1
    shape = np.array([info.bx, info.by, info.bz])
    nbx, nby, nbz = (-(-wl.box.nx // shape[0]), -(-wl.box.ny // shape[1]), -(-wl.box.nz // shape[2]))
    bvol = -np.ones((nbz, nby, nbx), np.int64)
    bo = org // shape
    bvol[bo[:, 2], bo[:, 1], bo[:, 0]] = np.arange(info.n_bricks)
    yield dict(wl=wl, grid=grid, psi0=psi0, info=info, act=act, seg=seg, off=off, rank=rank, bvol=bvol, V=V,
               shape=tuple(int(x) for x in shape))
    gpe.gpe_grid_destroy(grid)


def patch(B, i, j, k):
    """Mask, packed indices (-1 = not active) and host FP64 potential of the
    (2H+1)^3 patch at (i, j, k); also checks the builder on the patch: the
    active cells are exactly those with V_host < V_cut, and the stored
    potential equals V_host there."""
    wl = B["wl"]
    b_ = wl.box
    r = np.arange(-HALF, HALF + 1)
    K, J, I = np.meshgrid(k + r, j + r, i + r, indexing="ij")
    inside = (I >= 0) & (I < b_.nx) & (J >= 0) & (J < b_.ny) & (K >= 0) & (K < b_.nz)
    bx, by, bz = B["shape"]
    idx = -np.ones(K.shape, np.int64)
    Ii, Ji, Ki = I[inside], J[inside], K[inside]
    bid = B["bvol"][Ki // bz, Ji // by, Ii // bx]
    l = (Ii % bx) + bx * ((Ji % by) + by * (Ki % bz))
    has = bid >= 0
    act = np.zeros(Ii.shape, bool)
    act[has] = B["act"][bid[has], l[has]]
    sub = np.full(Ii.shape, -1, np.int64)
    sub[act] = B["off"][bid[act]] + 4 * B["rank"][bid[act], l[act] // 4] + l[act] % 4
    idx[inside] = sub
    Vh = np.full(K.shape, np.inf)
    Vh[inside] = wl.potential(b_.x0 + Ii * b_.hx, b_.y0 + Ji * b_.hy, b_.z0 + Ki * b_.hz)
    m = idx >= 0
    # the builder's region and potential against the host evaluation (cells
    # within 1e-12 of the cutoff may round either way)
    clear = np.abs(Vh - wl.V_cut) > 1e-12 * wl.V_cut
    assert np.array_equal(m[inside & clear], (Vh < wl.V_cut)[inside & clear]), (i, j, k)
    assert np.all(np.abs(B["V"][idx[m]] - Vh[m]) <= 1e-12 * wl.V_cut), (i, j, k)
    return m, idx, Vh


def samples(B, seed):
    rng = np.random.default_rng(seed)
    b = rng.integers(0, B["info"].n_bricks, 20 * NSAMPLE)
    out = []
    org, _ = gpe.gpe_grid_bricks(B["grid"])
    for bb in b:
        ls = np.flatnonzero(B["act"][bb])
        if ls.size == 0:
            continue
        l = rng.choice(ls)
        bx, by, _ = B["shape"]
        out.append((org[bb, 0] + l % bx, org[bb, 1] + (l // bx) % by, org[bb, 2] + l // (bx * by)))
        if len(out) == NSAMPLE:
            break
    return out


def run(B, dtype, kind):
    cdt = np.complex128 if dtype == gpe.GPE_C128 else np.complex64
    st = gpe.gpe_state_create(B["grid"], dtype)
    try:
        before = np.ascontiguousarray(B["psi0"].astype(cdt))
        gpe.gpe_state_load(st, before, gpe.GPE_LAYOUT_COMPACT)
        wl = B["wl"]
        if kind == "rk4":
            gpe.gpe_step_real(st, gpe.real_params(wl.g, wl.stable_dt()), 1)
        else:
            gpe.gpe_step_imag(st, gpe.gpe_imag_params(wl.g, wl.stable_dt(), 1.0), 1)
        after = np.zeros_like(before)
        gpe.gpe_state_store(st, after, gpe.GPE_LAYOUT_COMPACT)
    finally:
        gpe.gpe_state_destroy(st)
    return before.astype(np.complex128), after.astype(np.complex128)


@pytest.mark.parametrize("dtype,tol", [(gpe.GPE_C128, 1e-12), (gpe.GPE_C64, 2e-6)])
def test_rk4_full_size_sampled(big, dtype, tol):
    before, after = run(big, dtype, "rk4")
    wl = big["wl"]
    for (i, j, k) in samples(big, 11):
        m, idx, Vh = patch(big, i, j, k)
        g = oracle.Grid(m, wl.box.hx)
        y = oracle.rk4_step(g, Vh[m], before[idx[m]], wl.g, 0.0, wl.stable_dt())
        c = np.flatnonzero(np.all(g.ijk() == HALF, axis=1))[0]
        ref = y[c]
        got = after[idx[HALF, HALF, HALF]]
        scale = np.max(np.abs(before[idx[m]]))
        assert abs(got - ref) <= tol * scale, ((i, j, k), got, ref)


@pytest.mark.parametrize("dtype,tol", [(gpe.GPE_C128, 1e-12), (gpe.GPE_C64, 2e-6)])
def test_itp_full_size_sampled_up_to_one_factor(big, dtype, tol):
    before, after = run(big, dtype, "itp")
    wl = big["wl"]
    got, ref, scl = [], [], []
    for (i, j, k) in samples(big, 12):
        m, idx, Vh = patch(big, i, j, k)
        g = oracle.Grid(m, wl.box.hx)
        # the step before its renormalisation: N chosen so the factor is 1
        y, nrm = oracle.itp_step(g, Vh[m], before[idx[m]], wl.g, wl.stable_dt(), 1.0)
        y = y / math.sqrt(1.0 / nrm)
        c = np.flatnonzero(np.all(g.ijk() == HALF, axis=1))[0]
        ref.append(y[c])
        got.append(after[idx[HALF, HALF, HALF]])
        scl.append(np.max(np.abs(before[idx[m]])))
    got, ref, scl = np.array(got), np.array(ref), np.array(scl)
    big_ = np.abs(ref) > 1e-3 * scl
    factor = np.median(np.real(got[big_] / ref[big_]))
    assert 0.9 < factor < 1.1
    assert np.all(np.abs(got - factor * ref) <= tol * scl * factor)


def test_rk4_19_point_full_size_sampled(big):
    """App. B's 19-point stencil on the same shell, same launch configuration:
    its grid packs the cells exactly as the 7-point grid does (the stencil
    only adds edge records), so the samples reuse the layout.  A cell's new
    value depends on cells within Chebyshev distance 4, inside the patch."""
    wl, tol = big["wl"], 2e-6
    b = wl.box
    pot = gpe.make_potential(gpe.GPE_POT_ELLIPSOID_SHELL, wl.w, *wl.axes)
    grid = gpe.gpe_grid_create_analytic(gpe.make_box(b.nx, b.ny, b.nz, b.hx), pot, wl.V_cut,
                                        gpe.make_opts(big["shape"], stencil=19))
    try:
        info = gpe.gpe_grid_get_info(grid)
        assert info.n_packed == big["info"].n_packed and info.n_active == big["info"].n_active
        st = gpe.gpe_state_create(grid, gpe.GPE_C64)
        try:
            before = np.ascontiguousarray(big["psi0"].astype(np.complex64))
            gpe.gpe_state_load(st, before, gpe.GPE_LAYOUT_COMPACT)
            gpe.gpe_step_real(st, gpe.real_params(wl.g, wl.stable_dt()), 1)
            after = np.zeros_like(before)
            gpe.gpe_state_store(st, after, gpe.GPE_LAYOUT_COMPACT)
        finally:
            gpe.gpe_state_destroy(st)
    finally:
        gpe.gpe_grid_destroy(grid)
    before, after = before.astype(np.complex128), after.astype(np.complex128)
    for (i, j, k) in samples(big, 13):
        m, idx, Vh = patch(big, i, j, k)
        g = oracle.Grid(m, wl.box.hx)
        y = oracle.rk_step_np(g, Vh[m], before[idx[m]], wl.g, 0.0, wl.stable_dt(), "RK4", stencil=19)
        c = np.flatnonzero(np.all(g.ijk() == HALF, axis=1))[0]
        scale = np.max(np.abs(before[idx[m]]))
        assert abs(after[idx[HALF, HALF, HALF]] - y[c]) <= tol * scale, (i, j, k)


def test_pair_schedule_full_size_sampled(big):
    """The fused-pair schedule on the same shell (its grid packs the cells as
    the staged grid does): one RK4 step in two fused launches is bit-identical
    to the staged step on every cell; one imaginary-time step in one launch
    matches the oracle on the samples up to one common factor."""
    wl, tol = big["wl"], 2e-6
    b = wl.box
    pot = gpe.make_potential(gpe.GPE_POT_ELLIPSOID_SHELL, wl.w, *wl.axes)
    grid = gpe.gpe_grid_create_analytic(gpe.make_box(b.nx, b.ny, b.nz, b.hx), pot, wl.V_cut,
                                        gpe.make_opts(big["shape"], sched=gpe.GPE_SCHED_PAIR))
    try:
        assert gpe.gpe_grid_get_info(grid).n_packed == big["info"].n_packed
        st = gpe.gpe_state_create(grid, gpe.GPE_C64)
        before = np.ascontiguousarray(big["psi0"].astype(np.complex64))
        try:
            gpe.gpe_state_load(st, before, gpe.GPE_LAYOUT_COMPACT)
            gpe.gpe_step_real(st, gpe.real_params(wl.g, wl.stable_dt()), 1)
            rk = np.zeros_like(before)
            gpe.gpe_state_store(st, rk, gpe.GPE_LAYOUT_COMPACT)
            gpe.gpe_state_load(st, before, gpe.GPE_LAYOUT_COMPACT)
            gpe.gpe_step_imag(st, gpe.gpe_imag_params(wl.g, wl.stable_dt(), 1.0), 1)
            it = np.zeros_like(before)
            gpe.gpe_state_store(st, it, gpe.GPE_LAYOUT_COMPACT)
        finally:
            gpe.gpe_state_destroy(st)
    finally:
        gpe.gpe_grid_destroy(grid)
    _, rk_staged = run(big, gpe.GPE_C64, "rk4")
    assert np.array_equal(rk.astype(np.complex128), rk_staged)
    before, it = before.astype(np.complex128), it.astype(np.complex128)
    got, ref, scl = [], [], []
    for (i, j, k) in samples(big, 14):
        m, idx, Vh = patch(big, i, j, k)
        g = oracle.Grid(m, wl.box.hx)
        y, nrm = oracle.itp_step(g, Vh[m], before[idx[m]], wl.g, wl.stable_dt(), 1.0)
        y = y / math.sqrt(1.0 / nrm)
        c = np.flatnonzero(np.all(g.ijk() == HALF, axis=1))[0]
        ref.append(y[c])
        got.append(it[idx[HALF, HALF, HALF]])
        scl.append(np.max(np.abs(before[idx[m]])))
    got, ref, scl = np.array(got), np.array(ref), np.array(scl)
    big_ = np.abs(ref) > 1e-3 * scl
    factor = np.median(np.real(got[big_] / ref[big_]))
    assert 0.9 < factor < 1.1
    assert np.all(np.abs(got - factor * ref) <= tol * scl * factor)

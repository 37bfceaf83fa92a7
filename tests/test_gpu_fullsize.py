"""Parity at the headline size, in the launch configuration bench.py times
(1024^3 shell, ~2.9e7 active cells, the bench's brick shape, z-major order,
staged schedule): one GPU step on the whole grid, then sampled active cells compared
with the FP64 oracle run on the 11^3 patch around each sample.  One RK4 step
applies the stencil four times, so a cell's new value depends only on cells
within 4 of it and the patch (half-width 5) reproduces it exactly.

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
NSAMPLE = 40


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
    bid = {tuple(c): n for n, c in enumerate(org // shape)}
    yield dict(wl=wl, grid=grid, psi0=psi0, info=info, act=act, seg=seg, off=off, rank=rank, bid=bid, V=V,
               shape=tuple(int(x) for x in shape))
    gpe.gpe_grid_destroy(grid)


def patch(B, i, j, k):
    """Mask, packed indices (-1 = not active) of the (2H+1)^3 patch at (i, j, k)."""
    r = np.arange(-HALF, HALF + 1)
    K, J, I = np.meshgrid(k + r, j + r, i + r, indexing="ij")
    n = B["wl"].box.nx
    idx = -np.ones(K.shape, np.int64)
    inside = (I >= 0) & (I < n) & (J >= 0) & (J < n) & (K >= 0) & (K < n)
    for (a, b_, c) in zip(*np.nonzero(inside)):
        ii, jj, kk = I[a, b_, c], J[a, b_, c], K[a, b_, c]
        bx, by, bz = B["shape"]
        b = B["bid"].get((ii // bx, jj // by, kk // bz))
        if b is None:
            continue
        l = (ii % bx) + bx * ((jj % by) + by * (kk % bz))
        if B["act"][b, l]:
            idx[a, b_, c] = B["off"][b] + 4 * B["rank"][b, l // 4] + l % 4
    return idx >= 0, idx


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
        m, idx = patch(big, i, j, k)
        g = oracle.Grid(m, wl.box.hx)
        y = oracle.rk4_step(g, big["V"][idx[m]], before[idx[m]], wl.g, 0.0, wl.stable_dt())
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
        m, idx = patch(big, i, j, k)
        g = oracle.Grid(m, wl.box.hx)
        # the step before its renormalisation: N chosen so the factor is 1
        y, nrm = oracle.itp_step(g, big["V"][idx[m]], before[idx[m]], wl.g, wl.stable_dt(), 1.0)
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
        m, idx = patch(big, i, j, k)
        g = oracle.Grid(m, wl.box.hx)
        y = oracle.rk_step_np(g, big["V"][idx[m]], before[idx[m]], wl.g, 0.0, wl.stable_dt(), "RK4", stencil=19)
        c = np.flatnonzero(np.all(g.ijk() == HALF, axis=1))[0]
        scale = np.max(np.abs(before[idx[m]]))
        assert abs(after[idx[HALF, HALF, HALF]] - y[c]) <= tol * scale, (i, j, k)

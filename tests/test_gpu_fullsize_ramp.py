"""Parity at the ramp configuration's full size, in the launch configuration
bench.py times for it (--workload ramp2048): the 2048^3 box, the union region
{V0 < cut0} U {V1 < cut1} of the harmonic core and the thin shell (about
1.07e8 active cells), the library's default brick shape, the staged RK4 step
with V(t) = (1 - s(t)) V0 + s(t) V1 on the seeded 16-knot schedule and the
bench's dt.  One GPU step on the whole grid from a state that covers both
regions (the core cloud plus the shell's parabolic profile with its smooth
phase), taken in the middle of the ramp; sampled active cells (half of them
in the core, where the bench's state lives) compared with the FP64 oracle's
step on the 11^3 patch around each.  Every patch also checks the builder:
the region equals the union of the host FP64 potentials' regions and the
stored potentials equal the host values.

Tolerance as in test_gpu_parity: complex64 2e-6 relative to the largest
|psi| of the patch.
"""
import numpy as np
import pytest

import oracle
from paper_2603_05447_gb300 import gpe, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HALF = 5
NSAMPLE = 200


@pytest.fixture(scope="module")
def ramp():
    from paper_2603_05447_gb300 import _build
    _build.build()
    torch.cuda.init()
    torch.cuda.set_device(0)
    import bench
    rw = inputs.RAMP_2048
    b = rw.shell.box
    grid = bench._ramp_grid(gpe, rw)
    info = gpe.gpe_grid_get_info(grid)
    org, _ = gpe.gpe_grid_bricks(grid)
    bits = gpe.gpe_grid_mask(grid)
    bc = info.bx * info.by * info.bz
    act = np.unpackbits(bits.view(np.uint8), bitorder="little").astype(bool).reshape(info.n_bricks, bc)
    seg = act.reshape(info.n_bricks, bc // 4, 4).any(axis=2)
    off = 4 * np.concatenate([[0], np.cumsum(seg.sum(axis=1))[:-1]]).astype(np.int64)
    rank = np.cumsum(seg, axis=1) - 1
    shape = np.array([info.bx, info.by, info.bz])
    nb = (-(-b.nx // shape[0]), -(-b.ny // shape[1]), -(-b.nz // shape[2]))
    bvol = -np.ones((nb[2], nb[1], nb[0]), np.int64)
    bo = org // shape
    bvol[bo[:, 2], bo[:, 1], bo[:, 0]] = np.arange(info.n_bricks)
    # the state: the bench's core cloud plus the shell's profile, normalised
    idx, i, j, k = gpe.packed_coords(grid)
    x, y, z = b.x0 + i * b.hx, b.y0 + j * b.hy, b.z0 + k * b.hz
    psi = np.zeros(info.n_packed, np.complex128)
    psi[idx] = np.sqrt(np.maximum(rw.mu0_core - rw.v0(x, y, z), 0.0))
    on = rw.shell.potential(x, y, z) < rw.shell.mu0       # where the shell profile is not zero
    psi[idx[on]] += inputs.shell_initial_psi(rw.shell, x[on], y[on], z[on])
    psi /= np.sqrt(np.sum(np.abs(psi) ** 2) * b.dV)
    before = np.ascontiguousarray(psi.astype(np.complex64))
    dt = 0.2 / (6.0 / rw.shell.h ** 2 + info.v_max)
    knots = inputs.monotone_knots(16, seed=3)
    T = 500 * dt
    t0 = 0.37 * T
    st = gpe.gpe_state_create(grid, gpe.GPE_C64)
    try:
        gpe.gpe_state_load(st, before, gpe.GPE_LAYOUT_COMPACT)
        gpe.gpe_step_real(st, gpe.real_params(rw.shell.g, dt, gpe.GPE_V_BLEND, knots, T), 1, t0)
        after = np.zeros_like(before)
        gpe.gpe_state_store(st, after, gpe.GPE_LAYOUT_COMPACT)
    finally:
        gpe.gpe_state_destroy(st)
    V0 = gpe.gpe_grid_potential(grid, 0)
    V1 = gpe.gpe_grid_potential(grid, 1)
    yield dict(rw=rw, grid=grid, info=info, act=act, off=off, rank=rank, bvol=bvol, org=org,
               shape=tuple(int(v) for v in shape), V0=V0, V1=V1, before=before.astype(np.complex128),
               after=after.astype(np.complex128), dt=dt, knots=knots, T=T, t0=t0)
    gpe.gpe_grid_destroy(grid)


def patch(R, i, j, k):
    rw = R["rw"]
    b = rw.shell.box
    r = np.arange(-HALF, HALF + 1)
    K, J, I = np.meshgrid(k + r, j + r, i + r, indexing="ij")
    inside = (I >= 0) & (I < b.nx) & (J >= 0) & (J < b.ny) & (K >= 0) & (K < b.nz)
    bx, by, bz = R["shape"]
    Ii, Ji, Ki = I[inside], J[inside], K[inside]
    bid = R["bvol"][Ki // bz, Ji // by, Ii // bx]
    l = (Ii % bx) + bx * ((Ji % by) + by * (Ki % bz))
    has = bid >= 0
    act = np.zeros(Ii.shape, bool)
    act[has] = R["act"][bid[has], l[has]]
    sub = np.full(Ii.shape, -1, np.int64)
    sub[act] = R["off"][bid[act]] + 4 * R["rank"][bid[act], l[act] // 4] + l[act] % 4
    idx = -np.ones(K.shape, np.int64)
    idx[inside] = sub
    x, y, z = b.x0 + Ii * b.hx, b.y0 + Ji * b.hy, b.z0 + Ki * b.hz
    V0h = np.full(K.shape, np.inf)
    V1h = np.full(K.shape, np.inf)
    V0h[inside] = rw.v0(x, y, z)
    V1h[inside] = rw.shell.potential(x, y, z)
    m = idx >= 0
    clear = (np.abs(V0h - rw.cut0) > 1e-12 * rw.cut0) & (np.abs(V1h - rw.cut1) > 1e-12 * rw.cut1)
    want = (V0h < rw.cut0) | (V1h < rw.cut1)
    assert np.array_equal(m[inside & clear], want[inside & clear]), (i, j, k)
    assert np.all(np.abs(R["V0"][idx[m]] - V0h[m]) <= 1e-12 * max(rw.cut0, np.max(np.abs(V0h[m])))), (i, j, k)
    assert np.all(np.abs(R["V1"][idx[m]] - V1h[m]) <= 1e-12 * max(rw.cut1, np.max(np.abs(V1h[m])))), (i, j, k)
    return m, idx, V0h, V1h


def samples(R, seed):
    """Half in the core cloud (|r| below 0.8 of its Thomas-Fermi radius,
    core_radius / sqrt(cut_factor)), half anywhere in the region."""
    rng = np.random.default_rng(seed)
    rw = R["rw"]
    b = rw.shell.box
    bx, by, bz = R["shape"]
    org = R["org"]
    centre = (org + np.array([bx, by, bz]) / 2.0) * np.array([b.hx, b.hy, b.hz]) + np.array([b.x0, b.y0, b.z0])
    core = np.flatnonzero(np.linalg.norm(centre, axis=1) < 0.8 * rw.core_radius / np.sqrt(rw.shell.cut_factor))
    out = []
    for pool in (core, np.arange(R["info"].n_bricks)):
        got = 0
        for bb in rng.choice(pool, 20 * NSAMPLE):
            ls = np.flatnonzero(R["act"][bb])
            if ls.size == 0:
                continue
            l = rng.choice(ls)
            out.append((org[bb, 0] + l % bx, org[bb, 1] + (l // bx) % by, org[bb, 2] + l // (bx * by)))
            got += 1
            if got == NSAMPLE // 2:
                break
    return out


def test_ramp_rk4_full_size_sampled(ramp):
    R = ramp
    rw = R["rw"]
    b = rw.shell.box
    before, after = R["before"], R["after"]
    n_core = 0
    for (i, j, k) in samples(R, 21):
        m, idx, V0h, V1h = patch(R, i, j, k)
        g = oracle.Grid(m, b.hx)
        y = oracle.rk4_step(g, V0h[m], before[idx[m]], rw.shell.g, R["t0"], R["dt"], V1=V1h[m],
                            knots=R["knots"], T=R["T"])
        c = np.flatnonzero(np.all(g.ijk() == HALF, axis=1))[0]
        scale = np.max(np.abs(before[idx[m]]))
        got = after[idx[HALF, HALF, HALF]]
        assert abs(got - y[c]) <= 2e-6 * scale, ((i, j, k), got, y[c])
        n_core += abs(before[idx[HALF, HALF, HALF]]) > 0
    # at least the core half of the samples sits where psi is not zero
    assert n_core >= NSAMPLE // 2

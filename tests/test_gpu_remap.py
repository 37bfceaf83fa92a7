"""Regrid between ramp stages (Sec. V): gpe_state_remap carries a state to a
grid over the same box.  The expected result is the seeded input itself:
cells active in both regions keep their value, every other cell of the new
grid is zero.  Bit-exact (a copy)."""
import numpy as np
import pytest

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


BOX = inputs.Box(61, 53, 47, 1 / 26, 1 / 26, 1 / 26)    # not a multiple of any brick edge


def region(pot, cut):
    V = inputs.dense_potential(BOX, pot)
    return V, V < cut


def seeded_psi(seed):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=BOX.shape) + 1j * rng.normal(size=BOX.shape)).astype(np.complex128)


def gbox():
    return gpe.make_box(BOX.nx, BOX.ny, BOX.nz, BOX.hx, BOX.hy, BOX.hz)


NPT = {gpe.GPE_C128: np.complex128, gpe.GPE_C64: np.complex64, gpe.GPE_R64: np.float64, gpe.GPE_R32: np.float32}


@pytest.mark.parametrize("dtype", [gpe.GPE_C128, gpe.GPE_C64, gpe.GPE_R64, gpe.GPE_R32])
@pytest.mark.parametrize("bricks", [((8, 8, 8), (8, 8, 8)), ((8, 8, 4), (8, 4, 4)),
                                    ((8, 4, 4), (8, 8, 8))])
def test_remap_keeps_common_cells_and_zeroes_the_rest(dtype, bricks):
    V_a, m_a = region(inputs.EllipsoidShell(30.0, 0.9, 0.8, 0.7), 3.0)      # stage i
    V_b, m_b = region(inputs.EllipsoidShell(30.0, 0.95, 0.85, 0.75), 4.0)   # stage i + 1
    assert (m_a & m_b).any() and (m_a & ~m_b).any() and (m_b & ~m_a).any()
    cdt = NPT[dtype]
    psi = (seeded_psi(7).real if dtype in (gpe.GPE_R64, gpe.GPE_R32) else seeded_psi(7)).astype(cdt)
    ga = gpe.gpe_grid_create_dense(gbox(), V_a, 3.0, gpe.make_opts(bricks[0]))
    gb = gpe.gpe_grid_create_dense(gbox(), V_b, 4.0, gpe.make_opts(bricks[1], order=gpe.GPE_ORDER_MORTON))
    sa = gpe.gpe_state_create(ga, dtype)
    sb = gpe.gpe_state_create(gb, dtype)
    try:
        gpe.gpe_state_load(sa, np.ascontiguousarray(psi), gpe.GPE_LAYOUT_DENSE)
        other = seeded_psi(8)
        other = other.real if dtype in (gpe.GPE_R64, gpe.GPE_R32) else other
        gpe.gpe_state_load(sb, np.ascontiguousarray(other.astype(cdt)), gpe.GPE_LAYOUT_DENSE)
        gpe.gpe_state_remap(sb, sa)
        out = np.zeros(BOX.shape, cdt)
        gpe.gpe_state_store(sb, out, gpe.GPE_LAYOUT_DENSE)
        want = np.where(m_a & m_b, psi, 0).astype(cdt)
        assert np.array_equal(out, want)
        # and back again: only the common cells survive the round trip
        gpe.gpe_state_remap(sa, sb)
        gpe.gpe_state_store(sa, out, gpe.GPE_LAYOUT_DENSE)
        assert np.array_equal(out, want)
    finally:
        for s in (sa, sb):
            gpe.gpe_state_destroy(s)
        for g in (ga, gb):
            gpe.gpe_grid_destroy(g)


def test_remap_onto_the_same_region_is_a_copy():
    V, m = region(inputs.Harmonic(1.0, 1.2, 0.8), 2.0)
    psi = np.where(m, seeded_psi(9), 0)
    g1 = gpe.gpe_grid_create_dense(gbox(), V, 2.0, gpe.make_opts((8, 8, 8)))
    g2 = gpe.gpe_grid_create_dense(gbox(), V, 2.0, gpe.make_opts((8, 4, 4)))
    s1, s2 = gpe.gpe_state_create(g1, gpe.GPE_C128), gpe.gpe_state_create(g2, gpe.GPE_C128)
    try:
        gpe.gpe_state_load(s1, np.ascontiguousarray(psi), gpe.GPE_LAYOUT_DENSE)
        gpe.gpe_state_remap(s2, s1)
        out = np.zeros(BOX.shape, np.complex128)
        gpe.gpe_state_store(s2, out, gpe.GPE_LAYOUT_DENSE)
        assert np.array_equal(out, psi)
    finally:
        gpe.gpe_state_destroy(s1)
        gpe.gpe_state_destroy(s2)
        gpe.gpe_grid_destroy(g1)
        gpe.gpe_grid_destroy(g2)


def test_remap_argument_errors():
    V, _ = region(inputs.Harmonic(), 2.0)
    g1 = gpe.gpe_grid_create_dense(gbox(), V, 2.0)
    other = inputs.Box(BOX.nx, BOX.ny, BOX.nz, BOX.hx * 1.01, BOX.hy, BOX.hz)
    V2 = inputs.dense_potential(other, inputs.Harmonic())
    g2 = gpe.gpe_grid_create_dense(gpe.make_box(other.nx, other.ny, other.nz, other.hx, other.hy, other.hz), V2, 2.0)
    a, b = gpe.gpe_state_create(g1, gpe.GPE_C128), gpe.gpe_state_create(g2, gpe.GPE_C128)
    c = gpe.gpe_state_create(g1, gpe.GPE_C64)
    try:
        for dst, src in ((b, a), (c, a), (a, a)):
            with pytest.raises(gpe.GpeError) as e:
                gpe.gpe_state_remap(dst, src)
            assert e.value.code == gpe.GPE_ERR_ARG
    finally:
        for s in (a, b, c):
            gpe.gpe_state_destroy(s)
        gpe.gpe_grid_destroy(g1)
        gpe.gpe_grid_destroy(g2)

"""The 19-point higher-order compact Laplacian of App. B on the GPU against the
oracle's (the Kronecker form of App. B, pinned in test_oracle_pins): the
kinetic energy, RK4 steps (static and ramped potential) and imaginary-time
steps; complex128 and real FP64 1e-12, complex64 2e-6 after one step."""
import numpy as np
import pytest

import oracle
from gpu_cases import harmonic64, ragged_shell, ramp_case, rel_l2, shell
from paper_2603_05447_gb300 import gpe

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2603_05447_gb300 import _build
    _build.build()
    torch.cuda.init()
    torch.cuda.set_device(0)
    return gpe.load()


NPT = {gpe.GPE_C128: np.complex128, gpe.GPE_C64: np.complex64, gpe.GPE_R64: np.float64, gpe.GPE_R32: np.float32}


class G19:
    def __init__(self, case, dtype=gpe.GPE_C128, brick=(8, 8, 8), psi=None):
        self.case, self.dtype = case, dtype
        opts = gpe.make_opts(brick, stencil=19)
        if case.V1 is None:
            self.grid = gpe.gpe_grid_create_dense(case.gbox, case.V, case.V_cut, opts)
        else:
            self.grid = gpe.gpe_grid_create_dense(case.gbox, np.where(case.region, -1.0, 1.0), 0.0, opts)
            gpe.gpe_grid_set_potential(self.grid, 0, case.V)
            gpe.gpe_grid_set_potential(self.grid, 1, case.V1)
        self.st = gpe.gpe_state_create(self.grid, dtype)
        psi = case.psi if psi is None else psi
        arr = psi.real if dtype in (gpe.GPE_R64, gpe.GPE_R32) else psi
        gpe.gpe_state_load(self.st, np.ascontiguousarray(arr.astype(NPT[dtype])), gpe.GPE_LAYOUT_DENSE)

    def dense(self):
        out = np.zeros(self.case.box.shape, NPT[self.dtype])
        gpe.gpe_state_store(self.st, out, gpe.GPE_LAYOUT_DENSE)
        return out.astype(np.complex128)

    def close(self):
        gpe.gpe_state_destroy(self.st)
        gpe.gpe_grid_destroy(self.grid)


def ogrid(case):
    mask = case.mask if case.V1 is None else case.region
    return oracle.Grid(mask, (case.box.hx, case.box.hy, case.box.hz))


def oracle_rk4(case, psi, nsteps, t0=0.0):
    og = ogrid(case)
    y = og.compact(psi)
    V0 = og.compact(case.V)
    V1 = None if case.V1 is None else og.compact(case.V1)
    for q in range(nsteps):
        y = oracle.rk_step_np(og, V0, y, case.g, t0 + q * case.dt, case.dt, "RK4", V1,
                              None if V1 is None else case.knots, 0.0 if V1 is None else case.T, stencil=19)
    return og.dense(y)


@pytest.mark.parametrize("factory", [harmonic64, ragged_shell])
def test_kinetic_energy_matches_oracle(factory):
    case = factory()
    G = G19(case)
    try:
        og = ogrid(case)
        ref = oracle.observables_np(og, og.compact(case.V), case.g, og.compact(case.psi), stencil=19)
        o = gpe.gpe_observables(G.st, case.g)
        for k in ("e_kin", "energy", "mu", "norm"):
            assert abs(o[k] - ref[k]) <= 1e-12 * abs(ref[k]), k
        # and it differs from the 7-point value
        ref7 = oracle.observables(og, og.compact(case.V), case.g, og.compact(case.psi))
        assert abs(ref7["e_kin"] - ref["e_kin"]) > 1e-9 * abs(ref["e_kin"])
    finally:
        G.close()


@pytest.mark.parametrize("brick", [(8, 8, 8), (8, 8, 4), (8, 4, 4)])
@pytest.mark.parametrize("factory", [harmonic64, ragged_shell, shell])
def test_rk4_c128_matches_oracle(factory, brick):
    case = factory()
    G = G19(case, brick=brick)
    try:
        gpe.gpe_step_real(G.st, gpe.real_params(case.g, case.dt), 3)
        assert rel_l2(G.dense(), oracle_rk4(case, case.psi, 3)) <= 1e-12
    finally:
        G.close()


def test_rk4_ramp_blend_matches_oracle():
    case = ramp_case()
    t0 = 4 * case.dt
    G = G19(case)
    try:
        p = gpe.real_params(case.g, case.dt, gpe.GPE_V_BLEND, case.knots, case.T)
        gpe.gpe_step_real(G.st, p, 5, t0)
        assert rel_l2(G.dense(), oracle_rk4(case, case.psi, 5, t0)) <= 1e-12
    finally:
        G.close()


@pytest.mark.parametrize("brick", [(8, 8, 4), (8, 4, 4)])
def test_rk4_c64_matches_oracle_one_step(brick):
    case = ragged_shell()
    G = G19(case, gpe.GPE_C64, brick)
    try:
        psi32 = G.dense()
        gpe.gpe_step_real(G.st, gpe.real_params(case.g, case.dt), 1)
        assert rel_l2(G.dense(), oracle_rk4(case, psi32, 1)) <= 2e-6
    finally:
        G.close()


@pytest.mark.parametrize("dtype", [gpe.GPE_C128, gpe.GPE_R64])
def test_itp_matches_oracle(dtype):
    case = ragged_shell()
    psi = np.abs(case.psi).astype(np.complex128)
    G = G19(case, dtype, psi=psi)
    try:
        gpe.gpe_step_imag(G.st, gpe.gpe_imag_params(case.g, case.dt, 1.0), 4)
        og = ogrid(case)
        y = og.compact(psi)
        for _ in range(4):
            y, _ = oracle.itp_step_np(og, og.compact(case.V), y, case.g, case.dt, 1.0, stencil=19)
        assert rel_l2(G.dense(), og.dense(y)) <= 1e-12
    finally:
        G.close()


@pytest.mark.parametrize("dtype", [gpe.GPE_C64, gpe.GPE_R32])
def test_itp_single_precision_matches_oracle(dtype):
    """From the same single-precision input, four steps: a few roundings of
    6e-8 per pass and step."""
    case = ragged_shell()
    psi = np.abs(case.psi).astype(NPT[dtype]).astype(np.complex128)
    G = G19(case, dtype, brick=(8, 8, 4), psi=psi)
    try:
        gpe.gpe_step_imag(G.st, gpe.gpe_imag_params(case.g, case.dt, 1.0), 4)
        og = ogrid(case)
        y = og.compact(psi)
        for _ in range(4):
            y, _ = oracle.itp_step_np(og, og.compact(case.V), y, case.g, case.dt, 1.0, stencil=19)
        assert rel_l2(G.dense(), og.dense(y)) <= 1e-5
    finally:
        G.close()


def test_19_point_grids_refuse_the_other_paths():
    case = ragged_shell()
    G = G19(case)
    try:
        with pytest.raises(gpe.GpeError) as e:
            gpe.gpe_step_real(G.st, gpe.real_params(case.g, case.dt, integrator=gpe.GPE_RKHE3), 1)
        assert e.value.code == gpe.GPE_ERR_ARG
        with pytest.raises(gpe.GpeError) as e:
            gpe.gpe_batch_create([G.st])
        assert e.value.code == gpe.GPE_ERR_ARG
        with pytest.raises(gpe.GpeError) as e:
            gpe.gpe_grid_create_dense(case.gbox, case.V, case.V_cut, gpe.make_opts(stencil=9))
        assert e.value.code == gpe.GPE_ERR_ARG
    finally:
        G.close()

"""Real-valued states for imaginary time (half the bytes; Sec. II A notes that
the imaginary-time step keeps a real wavefunction real).  Parity with the
oracle's step on the same real input (complex oracle, zero imaginary part),
agreement with the complex path, and refusal of the complex-only calls."""
import numpy as np
import pytest

import oracle
from gpu_cases import harmonic64, ragged_shell, rel_l2, shell
from paper_2603_05447_gb300 import gpe, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R64_TOL = 1e-12
R32_TOL_1, R32_TOL_10 = 2e-6, 1e-5


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2603_05447_gb300 import _build
    _build.build()
    torch.cuda.init()
    torch.cuda.set_device(0)
    return gpe.load()


REAL = {gpe.GPE_R64: np.float64, gpe.GPE_R32: np.float32}
CPLX = {gpe.GPE_C128: np.complex128, gpe.GPE_C64: np.complex64}


class State:
    def __init__(self, case, dtype, brick=(8, 8, 8)):
        self.case, self.dtype = case, dtype
        self.grid = gpe.gpe_grid_create_dense(case.gbox, case.V, case.V_cut, gpe.make_opts(brick))
        self.st = gpe.gpe_state_create(self.grid, dtype)
        self.np = REAL.get(dtype) or CPLX[dtype]
        gpe.gpe_state_load(self.st, np.ascontiguousarray(real_psi(case).astype(self.np)), gpe.GPE_LAYOUT_DENSE)

    def dense(self):
        out = np.zeros(self.case.box.shape, self.np)
        gpe.gpe_state_store(self.st, out, gpe.GPE_LAYOUT_DENSE)
        return out.astype(np.complex128)

    def close(self):
        gpe.gpe_state_destroy(self.st)
        gpe.gpe_grid_destroy(self.grid)


def real_psi(case):
    """A real starting state: |psi| of the case's seeded state."""
    return np.abs(case.psi)


def oracle_itp(case, psi, nsteps):
    og = oracle.Grid(case.mask, (case.box.hx, case.box.hy, case.box.hz))
    y = og.compact(psi.astype(np.complex128))
    for _ in range(nsteps):
        y, _ = oracle.itp_step(og, og.compact(case.V), y, case.g, case.dt, 1.0)
    return og.dense(y)


@pytest.mark.parametrize("factory", [harmonic64, ragged_shell, shell])
def test_r64_itp_matches_oracle(factory):
    case = factory()
    S = State(case, gpe.GPE_R64)
    try:
        gpe.gpe_step_imag(S.st, gpe.gpe_imag_params(case.g, case.dt, 1.0), 5)
        ref = oracle_itp(case, real_psi(case), 5)
        assert np.abs(ref.imag).max() == 0.0
        assert rel_l2(S.dense(), ref) <= R64_TOL
    finally:
        S.close()


@pytest.mark.parametrize("brick", [(8, 8, 8), (8, 8, 4), (8, 4, 4)])
def test_r32_itp_matches_oracle(brick):
    case = ragged_shell()
    S = State(case, gpe.GPE_R32, brick)
    try:
        psi32 = S.dense()   # the float32-rounded input
        gpe.gpe_step_imag(S.st, gpe.gpe_imag_params(case.g, case.dt, 1.0), 1)
        assert rel_l2(S.dense(), oracle_itp(case, psi32, 1)) <= R32_TOL_1
        gpe.gpe_step_imag(S.st, gpe.gpe_imag_params(case.g, case.dt, 1.0), 9)
        assert rel_l2(S.dense(), oracle_itp(case, psi32, 10)) <= R32_TOL_10
    finally:
        S.close()


@pytest.mark.parametrize("real,cplx", [(gpe.GPE_R64, gpe.GPE_C128), (gpe.GPE_R32, gpe.GPE_C64)])
def test_real_state_agrees_with_complex_state(real, cplx):
    """Same arithmetic on the real part (the imaginary part stays exactly 0):
    the same wavefunction and the same observables."""
    case = shell()
    A, B = State(case, real), State(case, cplx)
    try:
        p = gpe.gpe_imag_params(case.g, case.dt, 1.0)
        gpe.gpe_step_imag(A.st, p, 12)
        gpe.gpe_step_imag(B.st, p, 12)
        a, b = A.dense(), B.dense()
        assert np.abs(b.imag).max() == 0.0
        assert rel_l2(a, b) <= 1e-15
        oa, ob = gpe.gpe_observables(A.st, case.g), gpe.gpe_observables(B.st, case.g)
        for k in ("norm", "energy", "mu", "e_kin", "e_pot", "e_int"):
            assert abs(oa[k] - ob[k]) <= 1e-14 * max(1.0, abs(ob[k])), k
    finally:
        A.close()
        B.close()


def test_r32_ground_state_converges_to_the_complex_one():
    case = harmonic64(g=100.0)
    A, B = State(case, gpe.GPE_R32), State(case, gpe.GPE_C64)
    try:
        p = gpe.gpe_imag_params(case.g, case.dt, 1.0)
        _, oa = gpe.gpe_ground_state(A.st, p, 1e-6, 10, 4000)   # raises unless converged
        _, ob = gpe.gpe_ground_state(B.st, p, 1e-6, 10, 4000)
        assert abs(oa["mu"] - ob["mu"]) < 1e-5 * abs(ob["mu"])
    finally:
        A.close()
        B.close()


def test_complex_only_calls_refuse_real_states():
    case = ragged_shell()
    A, B = State(case, gpe.GPE_R64), State(case, gpe.GPE_R64)
    try:
        for call in (lambda: gpe.gpe_step_real(A.st, gpe.real_params(case.g, case.dt), 1),
                     lambda: gpe.gpe_overlap(A.st, B.st)):
            with pytest.raises(gpe.GpeError) as e:
                call()
            assert e.value.code == gpe.GPE_ERR_ARG
    finally:
        A.close()
        B.close()


def test_region_error_shrinks_with_the_cutoff_and_brick_regions_do_better():
    """Sec. IV's study of the region of interest on a synthetic shell: real
    FP64 ground states on {V < r mu_TF} against the full-box ground state
    (same operator and time step).  The error falls with r, and the brick
    region, a superset of the cell region at the same r, does better."""
    wl = inputs.SHELL_64
    b = wl.box
    gb = gpe.make_box(b.nx, b.ny, b.nz, b.hx)
    V = inputs.dense_potential(b, wl.potential)
    mu_tf = gpe.gpe_tf_mu_dense(gb, V, wl.g, wl.N)
    p = gpe.gpe_imag_params(wl.g, 2.0 / (3 * 2.0 / b.hx ** 2), wl.N)
    psi0 = np.sqrt(np.maximum(mu_tf - V, 0.0) / wl.g)

    def ground(V_cut, mode):
        grid = gpe.gpe_grid_create_dense(gb, V, V_cut, gpe.make_opts((8, 8, 8), mode))
        st = gpe.gpe_state_create(grid, gpe.GPE_R64)
        try:
            gpe.gpe_state_load(st, np.ascontiguousarray(psi0), gpe.GPE_LAYOUT_DENSE)
            gpe.gpe_step_imag(st, p, 4000)
            gpe.gpe_ground_state(st, p, 1e-11, 100, 400000)
            out = np.zeros(b.shape)
            gpe.gpe_state_store(st, out, gpe.GPE_LAYOUT_DENSE)
            return out
        finally:
            gpe.gpe_state_destroy(st)
            gpe.gpe_grid_destroy(grid)

    ref = ground(np.inf, gpe.GPE_MASK_CELL)
    err = {(mode, r): float(np.sum(np.abs(ref ** 2 - ground(r * mu_tf, mode) ** 2)) * b.dV / wl.N)
           for mode in (gpe.GPE_MASK_CELL, gpe.GPE_MASK_BRICK) for r in (1.5, 3.0)}
    for mode in (gpe.GPE_MASK_CELL, gpe.GPE_MASK_BRICK):
        assert err[(mode, 3.0)] < 0.1 * err[(mode, 1.5)]
    for r in (1.5, 3.0):
        assert err[(gpe.GPE_MASK_BRICK, r)] < err[(gpe.GPE_MASK_CELL, r)]
    assert err[(gpe.GPE_MASK_CELL, 3.0)] < 1e-3

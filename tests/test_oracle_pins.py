"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a library
construction of the paper's own definition (Kronecker-sum Laplacian with rows
and columns deleted, Sec. II A), closed forms, dense matrix functions on tiny
grids, conservation laws, the paper's printed App. A tables, and finite
differences.  A plausible slip in the oracle (dropped term, wrong sign or
factor, wrong stage time, transposed index) fails at least one of them.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
from scipy.sparse.linalg import eigsh

from paper_2603_05447_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers
def kron_laplacian(nx, ny, nz, h):
    """Sec. II A: the Cartesian 7-point Laplacian built from Kronecker products
    of identities and the tridiagonal [1, -2, 1]/h^2 (x fastest)."""
    def d2(n, hh):
        return sp.diags([np.ones(n - 1), -2 * np.ones(n), np.ones(n - 1)], [-1, 0, 1]) / hh ** 2
    Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    return (sp.kron(Iz, sp.kron(Iy, d2(nx, h[0]))) + sp.kron(Iz, sp.kron(d2(ny, h[1]), Ix))
            + sp.kron(d2(nz, h[2]), sp.kron(Iy, Ix))).tocsr()


def reduced_laplacian(grid, h):
    """Rows and columns of inactive cells deleted (Sec. II A)."""
    L = kron_laplacian(grid.nx, grid.ny, grid.nz, h)
    return L[grid.cells][:, grid.cells]


def random_mask(shape, frac, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(size=shape) < frac


def cvec(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


# ----------------------------------------------------------------- grid
def test_neighbors_symmetric_and_match_dense_roll(oracle_mod):
    mask = random_mask((7, 6, 9), 0.6, 11)
    g = oracle_mod.Grid(mask, (0.3, 0.4, 0.5))
    pos = -np.ones(mask.size, dtype=np.int64)
    pos[g.cells] = np.arange(g.n)
    ijk = g.ijk()
    for e, (dx, dy, dz) in enumerate([(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]):
        i, j, k = ijk[:, 0] + dx, ijk[:, 1] + dy, ijk[:, 2] + dz
        inside = (i >= 0) & (i < g.nx) & (j >= 0) & (j < g.ny) & (k >= 0) & (k < g.nz)
        want = np.full(g.n, -1, dtype=np.int64)
        lin = (i + g.nx * (j + g.ny * k))[inside]
        want[inside] = pos[lin]
        assert np.array_equal(g.nbr[:, e], want)
        # symmetry: my +e neighbour has me as its -e neighbour
        opp = e ^ 1
        has = g.nbr[:, e] >= 0
        assert np.array_equal(g.nbr[g.nbr[has, e], opp], np.flatnonzero(has))


# ----------------------------------------------------------------- Laplacian
@pytest.mark.parametrize("frac", [1.0, 0.55])
def test_laplacian_equals_kronecker_sum_with_deleted_rows(oracle_mod, frac):
    h = (0.21, 0.34, 0.47)                          # anisotropic spacings, App. B
    mask = random_mask((9, 8, 10), frac, 3)
    g = oracle_mod.Grid(mask, h)
    L = reduced_laplacian(g, h)
    psi = cvec(g.n, 5)
    assert relerr(oracle_mod.laplacian(g, psi), L @ psi) < 1e-14


def test_laplacian_all_active_equals_dense_zero_padded_fd(oracle_mod):
    h = (0.25, 0.3, 0.2)
    shape = (12, 10, 11)
    g = oracle_mod.Grid(np.ones(shape, bool), h)
    dense = cvec(np.prod(shape), 9).reshape(shape)
    p = np.pad(dense, 1)
    ref = ((p[1:-1, 1:-1, 2:] - 2 * dense + p[1:-1, 1:-1, :-2]) / h[0] ** 2
           + (p[1:-1, 2:, 1:-1] - 2 * dense + p[1:-1, :-2, 1:-1]) / h[1] ** 2
           + (p[2:, 1:-1, 1:-1] - 2 * dense + p[:-2, 1:-1, 1:-1]) / h[2] ** 2)
    out = g.dense(oracle_mod.laplacian(g, g.compact(dense)))
    assert relerr(out, ref) < 1e-14


def test_laplacian_exact_on_quadratics_and_kills_constants(oracle_mod):
    box = inputs.Box(10, 9, 8, 0.2, 0.3, 0.4)
    mask = random_mask(box.shape, 0.8, 4)
    g = oracle_mod.Grid(mask, (box.hx, box.hy, box.hz))
    x, y, z = box.coords_of(g.ijk())
    interior = np.all(g.nbr >= 0, axis=1)
    assert interior.sum() > 20
    q = (x * x + 2 * y * y + 3 * z * z).astype(np.complex128)
    lap = oracle_mod.laplacian(g, q)
    assert np.allclose(lap[interior], 12.0, rtol=0, atol=1e-10)
    const = np.full(g.n, 2.5 - 1.5j)
    assert np.allclose(oracle_mod.laplacian(g, const)[interior], 0.0, atol=1e-11)


# ----------------------------------------------------------------- observables
def ho_1d(n, h):
    x = (np.arange(n) - (n - 1) / 2) * h
    d = 1.0 / h ** 2 + 0.5 * x ** 2          # -1/2 [1,-2,1]/h^2 + x^2/2
    e = -0.5 / h ** 2 * np.ones(n - 1)
    w, v = sla.eigh_tridiagonal(d, e, select="i", select_range=(0, 0))
    return w[0], v[:, 0]


def test_harmonic_exact_discrete_ground_state_energy(oracle_mod):
    """g = 0, 64^3, h = 0.25: the separable discrete ground state has
    E = mu = 3 lambda_min(1D); it is 1.5 up to the O(h^2) discretisation error."""
    n, h = 64, 0.25
    lam, v = ho_1d(n, h)
    assert abs(3 * lam - 1.4941174639) < 1e-9
    box = inputs.cubic_box(n, h)
    g = oracle_mod.Grid(np.ones(box.shape, bool), h)
    psi = np.einsum("k,j,i->kji", v, v, v).astype(np.complex128) / math.sqrt(box.dV)
    V = inputs.dense_potential(box, inputs.Harmonic())
    obs = oracle_mod.observables(g, g.compact(V), 0.0, g.compact(psi))
    assert abs(obs["norm"] - 1.0) < 1e-12
    assert abs(obs["energy"] - 3 * lam) < 1e-11
    assert abs(obs["mu"] - 3 * lam) < 1e-11
    assert abs(obs["energy"] - 1.5) < 3 * h ** 2 / 32 * 1.01 + 1e-6   # stated discretisation error


def test_observables_overlap_nonfinite_and_interaction(oracle_mod):
    box = inputs.Box(6, 5, 7, 0.3, 0.3, 0.3)
    g = oracle_mod.Grid(random_mask(box.shape, 0.7, 2), 0.3)
    psi = cvec(g.n, 3)
    V = np.random.default_rng(4).uniform(0, 2, g.n)
    o0 = oracle_mod.observables(g, V, 0.0, psi)
    o1 = oracle_mod.observables(g, V, 3.0, psi)
    rho = np.abs(psi) ** 2
    # E(g) - E(0) = g/2 sum rho^2 dV and mu gains twice that per atom
    assert abs((o1["energy"] - o0["energy"]) - 1.5 * np.sum(rho ** 2) * g.dV) < 1e-10
    assert abs((o1["mu"] - o0["mu"]) * o1["norm"] - 3.0 * np.sum(rho ** 2) * g.dV) < 1e-10
    assert abs(oracle_mod.overlap(psi, psi, g.dV) - o0["norm"]) < 1e-12
    # kinetic energy is Re<psi, T psi> = <psi, T psi> (T symmetric): matches the sparse matrix
    L = reduced_laplacian(g, g.h)
    assert abs(o0["e_kin"] - np.real(np.vdot(psi, -0.5 * (L @ psi))) * g.dV) < 1e-10
    bad = psi.copy()
    bad[3] = np.nan
    bad[7] = np.inf
    assert oracle_mod.observables(g, V, 0.0, bad)["nonfinite"] == 2


def test_tf_mu_harmonic_closed_form(oracle_mod):
    """Eq. (5) in V = r^2/2: mu = 1/2 (15 g N / 4 pi)^(2/5)."""
    g_, N = 500.0, 1.0
    mu_exact = 0.5 * (15 * g_ * N / (4 * math.pi)) ** 0.4
    box = inputs.cubic_box(96, 0.08)
    V = inputs.dense_potential(box, inputs.Harmonic())
    mu = oracle_mod.tf_mu(V, box.dV, g_, N)
    assert abs(mu - mu_exact) / mu_exact < 2e-3
    n = np.sum(np.maximum(mu - V, 0) / g_) * box.dV
    assert abs(n - N) < 1e-9


# ----------------------------------------------------------------- imaginary time
def itp_matrix(g, V, dt):
    """g = 0: the ITP step before renormalisation is D (I - dt/2 T)^2 D with
    D = diag(exp(-V dt/2)) and T = -1/2 Laplacian (Sec. II A)."""
    L = reduced_laplacian(g, g.h).toarray()
    K = np.eye(g.n) - 0.5 * dt * (-0.5 * L)
    D = np.diag(np.exp(-V * dt / 2))
    return D @ K @ K @ D


def test_itp_step_g0_equals_dense_linear_map(oracle_mod):
    box = inputs.Box(8, 7, 6, 0.4, 0.45, 0.5)
    g = oracle_mod.Grid(random_mask(box.shape, 0.75, 8), g_h := (0.4, 0.45, 0.5))
    V = np.random.default_rng(1).uniform(0, 3, g.n)
    psi = cvec(g.n, 2)
    dt, N = 0.02, 2.5
    out, nrm = oracle_mod.itp_step(g, V, psi, 0.0, dt, N)
    ref = itp_matrix(g, V, dt) @ psi
    assert abs(nrm - np.sum(np.abs(ref) ** 2) * g.dV) / nrm < 1e-13
    ref = ref * math.sqrt(N / (np.sum(np.abs(ref) ** 2) * g.dV))
    assert relerr(out, ref) < 1e-13


def test_itp_fixed_point_is_dominant_eigenvector(oracle_mod):
    """Repeated ITP steps at g = 0 converge to the dominant eigenvector of the
    step matrix, computed by ARPACK on the sparse Kronecker construction."""
    n, h, dt = 14, 0.5, 0.02
    box = inputs.cubic_box(n, h)
    g = oracle_mod.Grid(np.ones(box.shape, bool), h)
    V = g.compact(inputs.dense_potential(box, inputs.Harmonic()))
    L = reduced_laplacian(g, g.h)
    K = sp.identity(g.n) + 0.25 * dt * L
    D = sp.diags(np.exp(-V * dt / 2))
    A = (D @ K @ K @ D).tocsc()
    w, vec = eigsh(A, k=1, which="LA", tol=1e-14)
    vec = vec[:, 0] * np.sign(vec[:, 0].sum())
    vec = vec / math.sqrt(np.sum(vec ** 2) * g.dV)
    psi = g.compact(inputs.gaussian_with_noise(box, seed=1, noise=1e-3))
    for _ in range(2500):
        psi, _ = oracle_mod.itp_step(g, V, psi, 0.0, dt, 1.0)
    phase = np.vdot(vec, psi) / abs(np.vdot(vec, psi))
    assert relerr(psi / phase, vec) < 1e-8


def test_itp_interacting_fixed_point_solves_stationary_gpe(oracle_mod):
    """At g > 0 the ITP fixed point solves Eq. (1) on the grid up to a splitting
    error that shrinks with dt; the discrete virial identity
    2 E_kin - 2 E_pot + 3 E_int = 0 holds to O(h^2)."""
    n, h, g_ = 24, 0.4, 30.0
    box = inputs.cubic_box(n, h)
    g = oracle_mod.Grid(np.ones(box.shape, bool), h)
    V = g.compact(inputs.dense_potential(box, inputs.Harmonic()))
    res = []
    for dt in (0.004, 0.002):
        psi = g.compact(inputs.gaussian_with_noise(box, seed=1, noise=0.0))
        for _ in range(int(12.0 / dt)):
            psi, _ = oracle_mod.itp_step(g, V, psi, g_, dt, 1.0)
        obs = oracle_mod.observables(g, V, g_, psi)
        Hpsi = -0.5 * oracle_mod.laplacian(g, psi) + (V + g_ * np.abs(psi) ** 2) * psi
        res.append(np.linalg.norm(Hpsi - obs["mu"] * psi) / np.linalg.norm(psi))
        vir = 2 * obs["e_kin"] - 2 * obs["e_pot"] + 3 * obs["e_int"]
        assert abs(vir) / obs["energy"] < 0.02
    assert res[0] < 0.05
    assert 1.6 < res[0] / res[1] < 2.4      # first order in dt


# ----------------------------------------------------------------- real time (RK4)
def dense_H(g, V):
    L = reduced_laplacian(g, g.h).toarray()
    return -0.5 * L + np.diag(V)


def test_rk4_step_g0_is_taylor_polynomial_of_propagator(oracle_mod):
    """Static V, g = 0: one classic RK4 step is P4(-i H dt) psi with
    P4(z) = 1 + z + z^2/2 + z^3/6 + z^4/24."""
    box = inputs.Box(7, 8, 6, 0.3, 0.35, 0.4)
    g = oracle_mod.Grid(random_mask(box.shape, 0.7, 21), (0.3, 0.35, 0.4))
    V = np.random.default_rng(3).uniform(0, 4, g.n)
    psi = cvec(g.n, 4)
    dt = 0.004
    Z = -1j * dt * dense_H(g, V)
    P = np.eye(g.n) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    out = oracle_mod.rk4_step(g, V, psi, 0.0, 0.0, dt)
    assert relerr(out, P @ psi) < 1e-13


def test_rk4_fourth_order_against_matrix_exponential_with_time_dependent_shift(oracle_mod):
    """V(t) = V0 + s(t) (a uniform shift ramped by the knot schedule) commutes
    with H, so the exact solution is exp(-i H t) psi exp(-i int s).  RK4 with
    the right stage times c = (0, 1/2, 1/2, 1) converges at fourth order."""
    box = inputs.Box(6, 6, 5, 0.35, 0.35, 0.35)
    g = oracle_mod.Grid(random_mask(box.shape, 0.8, 5), 0.35)
    V0 = np.random.default_rng(6).uniform(0, 2, g.n)
    V1 = V0 + 1.0
    knots = np.array([0.0, 3.0, -2.0, 1.0, 4.0])
    T = 0.2
    psi0 = cvec(g.n, 7)
    H0 = dense_H(g, V0)
    tt = np.linspace(0.0, T, 200001)
    s = np.array([oracle_mod.ramp_s(knots, T, t) for t in tt[::100]])
    S = np.trapezoid(np.interp(tt, tt[::100], s), tt)     # s is piecewise linear: exact
    exact = sla.expm(-1j * H0 * T) @ psi0 * np.exp(-1j * S)
    errs = []
    for nsteps in (40, 80):
        dt = T / nsteps
        y = psi0
        for q in range(nsteps):
            y = oracle_mod.rk4_step(g, V0, y, 0.0, q * dt, dt, V1, knots, T)
        errs.append(relerr(y, exact))
    assert errs[0] / errs[1] > 12.0, errs


def test_rk4_constant_knots_equal_static_blend(oracle_mod):
    box = inputs.Box(5, 6, 5, 0.3, 0.3, 0.3)
    g = oracle_mod.Grid(random_mask(box.shape, 0.8, 9), 0.3)
    rng = np.random.default_rng(10)
    V0, V1 = rng.uniform(0, 3, g.n), rng.uniform(0, 3, g.n)
    psi = cvec(g.n, 11)
    s = 0.37
    a = oracle_mod.rk4_step(g, V0, psi, 2.0, 0.01, 0.003, V1, np.full(16, s), 1.0)
    b = oracle_mod.rk4_step(g, (1 - s) * V0 + s * V1, psi, 2.0, 0.01, 0.003)
    assert relerr(a, b) < 1e-15


def test_rk4_norm_loss_matches_stability_polynomial(oracle_mod):
    """For an eigenvector of H with eigenvalue E, one step multiplies it by
    P4(-i E dt); the norm loss is 1 - |P4(i y)|^2 = y^6/72 - y^8/576, y = E dt."""
    n, h = 20, 0.3
    box = inputs.cubic_box(n, h)
    g = oracle_mod.Grid(np.ones(box.shape, bool), h)
    V = g.compact(inputs.dense_potential(box, inputs.Harmonic()))
    lam, v = ho_1d(n, h)
    psi = np.einsum("k,j,i->kji", v, v, v).astype(np.complex128).ravel()
    dt = 0.35
    y = 3 * lam * dt
    out = oracle_mod.rk4_step(g, V, psi, 0.0, 0.0, dt)
    loss = 1 - np.sum(np.abs(out) ** 2) / np.sum(np.abs(psi) ** 2)
    assert abs(loss - (y ** 6 / 72 - y ** 8 / 576)) < 1e-13


def test_rk4_interacting_conserves_norm_and_energy(oracle_mod):
    """g > 0: the exact flow of Eq. (2) conserves N and E; RK4 drift shrinks
    at high order with dt (consistency of the RHS with the energy functional)."""
    n, h, g_ = 20, 0.4, 50.0
    box = inputs.cubic_box(n, h)
    g = oracle_mod.Grid(np.ones(box.shape, bool), h)
    V = g.compact(inputs.dense_potential(box, inputs.Harmonic(1.0, 1.3, 0.8)))
    psi0 = g.compact(inputs.gaussian_with_noise(box, seed=3, noise=0.05))
    o0 = oracle_mod.observables(g, V, g_, psi0)
    drifts = []
    for dt in (0.004, 0.002):
        y = psi0
        for q in range(int(0.2 / dt)):
            y = oracle_mod.rk4_step(g, V, y, g_, q * dt, dt)
        o = oracle_mod.observables(g, V, g_, y)
        drifts.append((abs(o["norm"] - o0["norm"]), abs(o["energy"] - o0["energy"]) / abs(o0["energy"])))
    assert drifts[0][0] < 1e-5 and drifts[0][1] < 1e-5
    assert drifts[0][1] / drifts[1][1] > 10.0


# ----------------------------------------------------------------- App. A tables
def derive_memopt(a, b):
    """Eq. (A4)-(A7): express k_j through the stage states by inverting M, then
    collect the coefficients of y^(j) in y^(i+1) and in y1 (dt = 1)."""
    n = len(b)
    M = [[Fraction(0)] * n for _ in range(n)]
    for i in range(n):
        M[i][0] = Fraction(1)
        for j in range(i):
            M[i][j + 1] = a[i][j]
    # exact inverse of the lower-triangular M
    Minv = [[Fraction(0)] * n for _ in range(n)]
    for col in range(n):
        e = [Fraction(int(r == col)) for r in range(n)]
        x = [Fraction(0)] * n
        for r in range(n):
            x[r] = (e[r] - sum(M[r][q] * x[q] for q in range(r))) / M[r][r]
        for r in range(n):
            Minv[r][col] = x[r]
    a_star = []
    for i in range(1, n):                     # row for y^(i+1), i = 1..n-1
        row = [Fraction(int(m == 0)) for m in range(i)]
        for j in range(1, i):                 # k_j, j < i, through Minv row j (K_{j+1})
            for m in range(i):
                row[m] += a[i][j - 1] * Minv[j][m]
        a_star.append(row)
    b_star = [Fraction(int(m == 0)) for m in range(n)]
    for j in range(1, n):
        for m in range(n):
            b_star[m] += b[j - 1] * Minv[j][m]
    return a_star, b_star


F = Fraction
TABLEAUS = {
    "RKHE3": ([[], [F(1, 3)], [F(0), F(2, 3)]], [F(1, 4), F(0), F(3, 4)]),
    "RK4": ([[], [F(1, 2)], [F(0), F(1, 2)], [F(0), F(0), F(1)]], [F(1, 6), F(1, 3), F(1, 3), F(1, 6)]),
    "RKCK": ([[], [F(1, 5)], [F(3, 40), F(9, 40)], [F(3, 10), F(-9, 10), F(6, 5)],
              [F(-11, 54), F(5, 2), F(-70, 27), F(35, 27)],
              [F(1631, 55296), F(175, 512), F(575, 13824), F(44275, 110592), F(253, 4096)]],
             [F(37, 378), F(0), F(250, 621), F(125, 594), F(0), F(512, 1771)]),
}


@pytest.mark.parametrize("method", ["RKHE3", "RK4", "RKCK"])
def test_memory_optimized_tables_match_appendix_A(method):
    gold = json.load(open(os.path.join(GOLDEN, "memopt_rk_appA.json")))[method]
    a, b = TABLEAUS[method]
    a_star, b_star = derive_memopt(a, b)
    want_a = [[Fraction(v) for v in row] for row in gold["a_star"]]
    want_b = [Fraction(v) for v in gold["b_star"]]
    for i, row in enumerate(want_a):
        assert a_star[i] == row[: i + 1] and all(v == 0 for v in row[i + 1:]), (i, a_star[i], row)
    assert b_star == want_b


def table_I_traffic(a, b, halo=1000, own=512):
    """Global loads and writes per 8^3 block and step under Table I's rule,
    for the normal method (stage i reads y0 and every k_j with a_ij != 0,
    with their halos) and the memory-optimised one (the stage producing
    y^(i+1) reads y^(i) with its halo and, at the block's own cells only,
    every other y^(j) with a*_ij != 0; the final combination likewise with
    b*).  Every stage writes one block."""
    a_star, b_star = derive_memopt(a, b)
    s = len(b)
    normal = sum(halo * (1 + sum(1 for v in a[i] if v != 0)) for i in range(s))
    opt = sum(halo + own * sum(1 for j, v in enumerate(row) if v != 0 and j != i)
              for i, row in enumerate(a_star))
    opt += halo + own * sum(1 for j, v in enumerate(b_star[:s]) if v != 0 and j != s - 1)
    return normal, opt, own * s


def test_table_I_traffic_from_the_derived_tables():
    """Table I (RKHE3) follows from the sparsity of the derived a*, b*: 5000
    and 4536 loads, 1536 writes; the saving relative to the optimised
    traffic, 7.6 %, is the quoted 7.5 %, and the same rule gives RKCK's
    quoted 44 % (43.7 %).  RK4's quoted 12 % does not follow from this rule
    (it gives 5.1 %)."""
    gold = json.load(open(os.path.join(GOLDEN, "memopt_rk_appA.json")))
    t = gold["traffic_table_I_RKHE3"]
    normal, opt, writes = table_I_traffic(*TABLEAUS["RKHE3"])
    assert (normal, writes) == (t["normal"]["loads"], t["normal"]["writes"])
    assert (opt, writes) == (t["optimized"]["loads"], t["optimized"]["writes"])
    saving = {}
    for m in ("RKHE3", "RK4", "RKCK"):
        n, o, w = table_I_traffic(*TABLEAUS[m])
        saving[m] = 100.0 * ((n + w) - (o + w)) / (o + w)
    assert round(saving["RKHE3"], 1) == 7.6 and abs(saving["RKHE3"] - gold["traffic_saving_percent"]["RKHE3"]) < 0.2
    assert round(saving["RKCK"]) == gold["traffic_saving_percent"]["RKCK"]
    assert round(saving["RK4"], 1) == 5.1


def test_memory_optimized_rk4_stage_algebra_equals_butcher_step(oracle_mod):
    """The stage recurrences used by the CUDA kernels (App. A, RK4 a*, b*)
    reproduce the oracle's Butcher-form step to round-off."""
    box = inputs.Box(6, 5, 7, 0.3, 0.3, 0.3)
    g = oracle_mod.Grid(random_mask(box.shape, 0.8, 12), 0.3)
    V = np.random.default_rng(13).uniform(0, 3, g.n)
    y0 = cvec(g.n, 14) * 0.3
    dt, g_ = 0.003, 4.0
    f = lambda y: oracle_mod.rhs_real(g, V, g_, y)
    y2 = y0 + dt / 2 * f(y0)
    y3 = y0 + dt / 2 * f(y2)
    y4 = y0 + dt * f(y3)
    y1 = -y0 / 3 + y2 / 3 + 2 * y3 / 3 + y4 / 3 + dt / 6 * f(y4)
    assert relerr(y1, oracle_mod.rk4_step(g, V, y0, g_, 0.0, dt)) < 1e-14


# ----------------------------------------------------------------- adjoint
def ramp_problem(oracle_mod, seed=0):
    box = inputs.Box(6, 6, 6, 0.4, 0.4, 0.4)
    g = oracle_mod.Grid(random_mask(box.shape, 0.85, 30 + seed), 0.4)
    x, y, z = box.coords_of(g.ijk())
    V0 = 0.5 * (x * x + y * y + z * z)
    V1 = 2.0 * (np.sqrt(x * x + y * y + z * z) - 0.8) ** 2
    rng = np.random.default_rng(40 + seed)
    psi0 = (np.exp(-(x * x + y * y + z * z)) * (1 + 0.1 * rng.standard_normal(g.n))).astype(np.complex128)
    psi0 /= math.sqrt(np.sum(np.abs(psi0) ** 2) * g.dV)
    tgt = (np.exp(-2 * (np.sqrt(x * x + y * y + z * z) - 0.8) ** 2)).astype(np.complex128)
    tgt /= math.sqrt(np.sum(np.abs(tgt) ** 2) * g.dV)
    knots = inputs.monotone_knots(16, seed=3)
    return g, V0, V1, psi0, tgt, knots


def test_adjoint_gradient_matches_central_differences(oracle_mod):
    g, V0, V1, psi0, tgt, knots = ramp_problem(oracle_mod)
    T, dt, nsteps, g_ = 0.3, 0.01, 30, 20.0
    loss, grad, _ = oracle_mod.ramp_loss_and_grad(g, V0, V1, knots, T, g_, dt, nsteps, psi0, tgt)
    eps = 1e-4
    fd = np.zeros_like(grad)
    for q in range(len(knots)):
        kp, km = knots.copy(), knots.copy()
        kp[q] += eps
        km[q] -= eps
        lp = oracle_mod.ramp_loss_and_grad(g, V0, V1, kp, T, g_, dt, nsteps, psi0, tgt)[0]
        lm = oracle_mod.ramp_loss_and_grad(g, V0, V1, km, T, g_, dt, nsteps, psi0, tgt)[0]
        fd[q] = (lp - lm) / (2 * eps)
    assert np.max(np.abs(grad - fd)) / np.max(np.abs(fd)) < 1e-6


def test_adjoint_step_transpose_identity(oracle_mod):
    """<lam, J v> = <J^T lam, v> (real inner product of real pairs) for one step,
    J v from a central directional difference of the forward step."""
    g, V0, V1, psi0, tgt, knots = ramp_problem(oracle_mod, seed=1)
    T, dt, g_, t = 0.3, 0.01, 20.0, 0.05
    v = cvec(g.n, 50)
    lam = cvec(g.n, 51)
    eps = 1e-6
    fp = oracle_mod.rk4_step(g, V0, psi0 + eps * v, g_, t, dt, V1, knots, T)
    fm = oracle_mod.rk4_step(g, V0, psi0 - eps * v, g_, t, dt, V1, knots, T)
    Jv = (fp - fm) / (2 * eps)
    JTlam, _ = oracle_mod.rk4_adjoint_step(g, V0, V1, knots, T, g_, t, dt, psi0, lam)
    lhs = np.sum(np.real(np.conj(lam) * Jv))
    rhs = np.sum(np.real(np.conj(JTlam) * v))
    assert abs(lhs - rhs) / abs(lhs) < 1e-8


# ----------------------------------------------------------------- RKHE3 / RKCK (general Butcher step)
ORDER = {"RKHE3": 3, "RK4": 4, "RKCK": 5}


@pytest.mark.parametrize("method", ["RKHE3", "RK4", "RKCK"])
def test_tableaux_satisfy_the_linear_order_conditions(oracle_mod, method):
    """b^T A^(k-1) 1 = 1/k! for k <= order (the stability polynomial agrees
    with exp(z) to that order): a transcription error in A or b fails here."""
    A, b, c = oracle_mod.TABLEAUX[method]
    assert np.allclose(c, A.sum(axis=1), atol=0)
    v = np.ones(len(b))
    for k in range(1, ORDER[method] + 1):
        assert abs(b @ v - 1 / math.factorial(k)) < 1e-15, (method, k)
        v = A @ v


@pytest.mark.parametrize("method", ["RKHE3", "RKCK"])
def test_rk_step_g0_is_stability_function_of_propagator(oracle_mod, method):
    """Static V, g = 0: one step is R(-i H dt) psi with the stability function
    R(z) = 1 + z b^T (I - z A)^-1 1, formed here as a dense matrix."""
    A, b, _ = oracle_mod.TABLEAUX[method]
    box = inputs.Box(7, 6, 6, 0.3, 0.35, 0.4)
    g = oracle_mod.Grid(random_mask(box.shape, 0.7, 41), (0.3, 0.35, 0.4))
    V = np.random.default_rng(42).uniform(0, 4, g.n)
    psi = cvec(g.n, 43)
    dt = 0.004
    Z = -1j * dt * dense_H(g, V)
    # R(Z) = I + sum_k (b^T A^(k-1) 1) Z^k  (A is nilpotent: finitely many terms)
    R = np.eye(g.n, dtype=complex)
    v, Zk = np.ones(len(b)), np.eye(g.n, dtype=complex)
    for _ in range(len(b)):
        Zk = Zk @ Z
        R = R + (b @ v) * Zk
        v = A @ v
    out = oracle_mod.rk_step(g, V, psi, 0.0, 0.0, dt, method)
    assert relerr(out, R @ psi) < 1e-13


def test_rk_step_with_rk4_tableau_equals_classic_rk4(oracle_mod):
    box = inputs.Box(6, 5, 7, 0.3, 0.3, 0.3)
    g = oracle_mod.Grid(random_mask(box.shape, 0.8, 44), 0.3)
    rng = np.random.default_rng(45)
    V0, V1 = rng.uniform(0, 3, g.n), rng.uniform(0, 3, g.n)
    psi = cvec(g.n, 46) * 0.3
    knots = np.array([0.1, 0.7, 0.2, 0.9])
    a = oracle_mod.rk_step(g, V0, psi, 3.0, 0.05, 0.004, "RK4", V1, knots, 0.3)
    b = oracle_mod.rk4_step(g, V0, psi, 3.0, 0.05, 0.004, V1, knots, 0.3)
    assert relerr(a, b) < 1e-14


@pytest.mark.parametrize("method", ["RKHE3", "RKCK"])
def test_rk_order_against_matrix_exponential_with_time_dependent_shift(oracle_mod, method):
    """As for RK4: a ramped uniform shift commutes with H, so the exact
    solution is known; halving dt must cut the error by about 2^order, which
    also pins the stage times c."""
    box = inputs.Box(6, 6, 5, 0.35, 0.35, 0.35)
    g = oracle_mod.Grid(random_mask(box.shape, 0.8, 47), 0.35)
    V0 = np.random.default_rng(48).uniform(0, 2, g.n)
    V1 = V0 + 1.0
    knots = np.array([0.0, 3.0, -2.0, 1.0, 4.0])
    T = 0.2
    psi0 = cvec(g.n, 49)
    H0 = dense_H(g, V0)
    tt = np.linspace(0.0, T, 200001)
    s = np.array([oracle_mod.ramp_s(knots, T, t) for t in tt[::100]])
    S = np.trapezoid(np.interp(tt, tt[::100], s), tt)
    exact = sla.expm(-1j * H0 * T) @ psi0 * np.exp(-1j * S)
    errs = []
    n0 = 40 if method == "RKHE3" else 16
    for nsteps in (n0, 2 * n0):
        dt = T / nsteps
        y = psi0
        for q in range(nsteps):
            y = oracle_mod.rk_step(g, V0, y, 0.0, q * dt, dt, method, V1, knots, T)
        errs.append(relerr(y, exact))
    p = ORDER[method]
    assert 0.6 * 2 ** p < errs[0] / errs[1] < 1.6 * 2 ** p, errs


@pytest.mark.parametrize("method", ["RKHE3", "RKCK"])
def test_appendix_A_memory_optimized_recurrence_equals_butcher_step(oracle_mod, method):
    """App. A's printed a*, b* (tests/golden/memopt_rk_appA.json) with the
    tableau's sub-diagonal: y^(1) = y0, y^(i+1) = sum_j a*_ij y^(j) + dt
    a_{i+1,i} f(t + c_i dt, y^(i)), y1 = sum_j b*_j y^(j) + dt b_s f(t + c_s dt,
    y^(s)), reproduce the Butcher step at g > 0 with a ramped potential."""
    gold = json.load(open(os.path.join(GOLDEN, "memopt_rk_appA.json")))[method]
    a_star = [[float(Fraction(v)) for v in row] for row in gold["a_star"]]
    b_star = [float(Fraction(v)) for v in gold["b_star"]]
    A, b, c = oracle_mod.TABLEAUX[method]
    box = inputs.Box(6, 5, 6, 0.3, 0.3, 0.3)
    g = oracle_mod.Grid(random_mask(box.shape, 0.8, 50), 0.3)
    rng = np.random.default_rng(51)
    V0, V1 = rng.uniform(0, 3, g.n), rng.uniform(0, 3, g.n)
    knots = np.array([0.2, 0.6, 0.1, 0.8, 0.5])
    T, t, dt, gg = 0.3, 0.07, 0.003, 3.0
    y0 = cvec(g.n, 52) * 0.3

    def f(tt, y):
        s = oracle_mod.ramp_s(knots, T, tt)
        return oracle_mod.rhs_real(g, (1 - s) * V0 + s * V1, gg, y)

    n = len(b)
    Y = [y0]
    for i in range(1, n):          # y^(i+1) from y^(1..i)
        nxt = sum(a_star[i - 1][j] * Y[j] for j in range(i)) + dt * A[i, i - 1] * f(t + c[i - 1] * dt, Y[i - 1])
        Y.append(nxt)
    y1 = sum(b_star[j] * Y[j] for j in range(n)) + dt * b[n - 1] * f(t + c[n - 1] * dt, Y[n - 1])
    ref = oracle_mod.rk_step(g, V0, y0, gg, t, dt, method, V1, knots, T)
    assert relerr(y1, ref) < 1e-13


# ----------------------------------------------------------------- 19-point stencil (App. B)
def kron_laplacian19(nx, ny, nz, h):
    """App. B written out with Kronecker products: the 7-point sum plus
    1/12 [(hx^2+hy^2) d2x d2y + (hx^2+hz^2) d2x d2z + (hy^2+hz^2) d2y d2z]."""
    def d2(n, hh):
        return sp.diags([np.ones(n - 1), -2 * np.ones(n), np.ones(n - 1)], [-1, 0, 1]) / hh ** 2
    Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    Dx, Dy, Dz = d2(nx, h[0]), d2(ny, h[1]), d2(nz, h[2])
    hx2, hy2, hz2 = h[0] ** 2, h[1] ** 2, h[2] ** 2
    mixed = ((hx2 + hy2) * sp.kron(Iz, sp.kron(Dy, Dx)) + (hx2 + hz2) * sp.kron(Dz, sp.kron(Iy, Dx))
             + (hy2 + hz2) * sp.kron(Dz, sp.kron(Dy, Ix)))
    return (kron_laplacian(nx, ny, nz, h) + mixed / 12.0).tocsr()


@pytest.mark.parametrize("frac", [1.0, 0.6])
def test_laplacian19_equals_appendix_B_kronecker_form_with_deleted_rows(oracle_mod, frac):
    h = (0.21, 0.34, 0.47)
    mask = random_mask((9, 8, 10), frac, 61)
    g = oracle_mod.Grid(mask, h)
    L = kron_laplacian19(g.nx, g.ny, g.nz, h)[g.cells][:, g.cells]
    psi = cvec(g.n, 62)
    assert relerr(oracle_mod.laplacian(g, psi, 19), L @ psi) < 1e-14


def test_laplacian19_exact_on_quadratics_kills_constants_and_differs_from_7pt(oracle_mod):
    """The mixed differences vanish on polynomials of degree <= 2 (so the
    19-point stencil is exact there, like the 7-point one) but not on x^2 y^2."""
    box = inputs.Box(12, 11, 10, 0.2, 0.3, 0.4)
    g = oracle_mod.Grid(random_mask(box.shape, 0.96, 63), (box.hx, box.hy, box.hz))
    x, y, z = box.coords_of(g.ijk())
    full = np.all(g.nbr >= 0, axis=1) & np.all(g.nbr_e >= 0, axis=1)
    assert full.sum() > 10
    q = (x * x + 2 * y * y + 3 * z * z + x * y - y * z).astype(np.complex128)
    assert np.allclose(oracle_mod.laplacian(g, q, 19)[full], 12.0, rtol=0, atol=1e-9)
    const = np.full(g.n, 1.0 + 2.0j)
    assert np.allclose(oracle_mod.laplacian(g, const, 19)[full], 0.0, atol=1e-10)
    p = (x * x * y * y).astype(np.complex128)
    diff = oracle_mod.laplacian(g, p, 19) - oracle_mod.laplacian(g, p, 7)
    # d2x d2y (x^2 y^2) = 4 exactly: the extra term is (hx^2 + hy^2) * 4 / 12
    assert np.allclose(diff[full], (box.hx ** 2 + box.hy ** 2) * 4 / 12, rtol=1e-9, atol=0)


def test_numpy_steps_equal_the_c_steps(oracle_mod):
    """The numpy restatements (used with the 19-point stencil) reproduce the
    C steps with the 7-point stencil."""
    box = inputs.Box(6, 7, 5, 0.3, 0.32, 0.34)
    g = oracle_mod.Grid(random_mask(box.shape, 0.8, 64), (box.hx, box.hy, box.hz))
    rng = np.random.default_rng(65)
    V0, V1 = rng.uniform(0, 3, g.n), rng.uniform(0, 3, g.n)
    psi = cvec(g.n, 66) * 0.3
    knots = np.array([0.1, 0.5, 0.9])
    a = oracle_mod.rk_step_np(g, V0, psi, 3.0, 0.02, 0.003, "RK4", V1, knots, 0.2)
    b = oracle_mod.rk4_step(g, V0, psi, 3.0, 0.02, 0.003, V1, knots, 0.2)
    assert relerr(a, b) < 1e-14
    a, na = oracle_mod.itp_step_np(g, V0, psi, 3.0, 0.004, 1.0)
    b, nb = oracle_mod.itp_step(g, V0, psi, 3.0, 0.004, 1.0)
    assert relerr(a, b) < 1e-14 and abs(na - nb) < 1e-14 * nb
    oa, ob = oracle_mod.observables_np(g, V0, 3.0, psi), oracle_mod.observables(g, V0, 3.0, psi)
    for k in ("norm", "energy", "mu", "e_kin", "e_pot", "e_int"):
        assert abs(oa[k] - ob[k]) <= 1e-13 * max(1.0, abs(ob[k])), k


# ----------------------------------------------------------------- multi-stage ramps (Sec. V)
def stage_problem(oracle_mod, g_=50.0, trap=inputs.Harmonic(1.0, 1.1, 0.9)):
    box = inputs.cubic_box(28, 0.25)
    h = (box.hx, box.hy, box.hz)
    Va = inputs.dense_potential(box, trap)
    mu = oracle_mod.tf_mu(Va, box.dV, g_, 1.0)
    rng = np.random.default_rng(70)
    prof = np.sqrt(np.maximum(mu - Va, 0) / g_) * np.exp(0.3j * rng.normal(size=Va.shape))
    psi0 = np.where(Va < 5 * mu, prof, 0)
    psi0 = psi0 / np.sqrt(np.sum(np.abs(psi0) ** 2) * box.dV)
    return box, h, Va, mu, psi0


def test_ramp_stages_with_equal_potentials_chain_into_one_static_evolution(oracle_mod):
    """Stages and the hold between identical potentials select the same region
    and must continue one static evolution: 3 + 2 stage steps and a 4-step
    hold equal 9 RK4 steps in V."""
    box, h, V, mu, psi0 = stage_problem(oracle_mod)
    dt, g_ = 0.01, 50.0
    out, rec = oracle_mod.ramp_stages([V, V, V], h, [3 * dt, 2 * dt], g_, 1.0, dt, psi0, t_hold=4 * dt)
    assert [r["steps"] for r in rec] == [3, 2, 4]
    grid = oracle_mod.Grid(V < 5 * mu, h)
    assert all(r["n_active"] == grid.n and r["cut"] == 5 * mu for r in rec)
    y, Vc = grid.compact(psi0), grid.compact(V)
    for k in range(9):
        y = oracle_mod.rk4_step(grid, Vc, y, g_, 0.0, dt)
    assert relerr(out, grid.dense(y)) < 1e-12
    assert abs(rec[-1]["norm_end"] - oracle_mod.observables(grid, Vc, g_, y)["norm"]) < 1e-13


def test_ramp_stage_with_a_uniform_shift_is_a_phase(oracle_mod):
    """V_b = V_a + c: during the stage V(t) = V_a + c t/d, which multiplies the
    solution by exp(-i c t^2 / 2d) and leaves |psi| alone at any g.  So one
    stage equals the static evolution in V_a times exp(-i c d / 2), up to the
    two RK4 errors, which shrink as dt^4."""
    box, h, Va, mu, psi0 = stage_problem(oracle_mod)
    c, d, g_ = 3.0, 0.1, 50.0
    Vb = Va + c
    errs = []
    for n in (8, 16):
        dt = d / n
        out, rec = oracle_mod.ramp_stages([Va, Vb], h, [d], g_, 1.0, dt, psi0)
        assert rec[0]["steps"] == n
        grid = oracle_mod.Grid((Va < rec[0]["cut"]) | (Vb < rec[0]["cut"]), h)
        assert abs(rec[0]["mu_b"] - rec[0]["mu_a"] - c) < 1e-9      # Eq. (5) shifts with V
        y, Vc = grid.compact(psi0), grid.compact(Va)
        for k in range(n):
            y = oracle_mod.rk4_step(grid, Vc, y, g_, 0.0, dt)
        errs.append(relerr(out, grid.dense(y * np.exp(-0.5j * c * d))))
    assert errs[0] < 2e-3 and 12.0 < errs[0] / errs[1] < 20.0, errs     # fourth order


def test_ramp_stage_starts_in_its_first_potential(oracle_mod):
    """Within a stage the potential runs from V_i at t = 0 to V_{i+1} at t = d:
    the same as a ramp whose knots rise linearly from 0 to 1 over d (not the
    reverse)."""
    g_ = 5.0
    box, h, Va, mu, psi0 = stage_problem(oracle_mod, g_, inputs.Harmonic(2.0, 2.2, 1.8))
    Vb = inputs.dense_potential(box, inputs.EllipsoidShell(20.0, 2.6, 2.4, 2.2))
    d, dt = 0.06, 0.01
    out, rec = oracle_mod.ramp_stages([Va, Vb], h, [d], g_, 1.0, dt, psi0)
    grid = oracle_mod.Grid((Va < rec[0]["cut"]) | (Vb < rec[0]["cut"]), h)
    assert rec[0]["n_active"] == grid.n
    assert grid.n > np.count_nonzero(Va < rec[0]["cut"]) and grid.n > np.count_nonzero(Vb < rec[0]["cut"])
    A, B = grid.compact(Va), grid.compact(Vb)
    fwd, rev = grid.compact(psi0), grid.compact(psi0)
    lin = np.linspace(0.0, 1.0, 16)
    for k in range(6):
        fwd = oracle_mod.rk4_step(grid, A, fwd, g_, k * dt, dt, B, lin, d)
        rev = oracle_mod.rk4_step(grid, A, rev, g_, k * dt, dt, B, lin[::-1].copy(), d)
    assert relerr(out, grid.dense(fwd)) < 1e-12
    assert relerr(out, grid.dense(rev)) > 1e-4

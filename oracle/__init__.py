"""FP64 CPU oracle for the finite-difference GPE step on a sampled grid.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it and shares no code with it.

The arithmetic lives in ``gpe_oracle.c`` (plain loops, FP64, OpenMP across
cells only); this module compiles it with gcc on first use and wraps it with
numpy arrays.  Paper: "Efficient simulation of Bose-Einstein condensates in
nontrivial topologies", Sec. II A (general algorithm), Eqs. (3), (5)-(9).

Conventions: a dense box array has numpy shape (nz, ny, nx) (x fastest), so a
cell's linear index is ``i + nx*(j + ny*k)``.  The active cells of a grid are
kept in ascending linear order; a compact vector holds one value per active
cell in that order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gpe_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libgpe_oracle.so")
_lib = None
_lock = threading.Lock()

_c_i64p = ctypes.POINTER(ctypes.c_int64)
_c_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libgpe_oracle.so`` with gcc."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.orc_neighbors.restype = ctypes.c_int
        lib.orc_neighbors.argtypes = [ctypes.c_int64, _c_i64p, ctypes.c_int64,
                                      ctypes.c_int64, ctypes.c_int64, _c_i64p]
        lib.orc_edge_neighbors.restype = ctypes.c_int
        lib.orc_edge_neighbors.argtypes = [ctypes.c_int64, _c_i64p, ctypes.c_int64,
                                           ctypes.c_int64, ctypes.c_int64, _c_i64p]
        lib.orc_laplacian19.restype = None
        lib.orc_laplacian19.argtypes = ([ctypes.c_int64, _c_i64p, _c_i64p] + [ctypes.c_double] * 3
                                        + [_c_f64p, _c_f64p])
        lib.orc_laplacian.restype = None
        lib.orc_laplacian.argtypes = [ctypes.c_int64, _c_i64p] + [ctypes.c_double] * 3 + [_c_f64p, _c_f64p]
        lib.orc_rhs_real.restype = None
        lib.orc_rhs_real.argtypes = ([ctypes.c_int64, _c_i64p] + [ctypes.c_double] * 3
                                     + [_c_f64p, ctypes.c_double, _c_f64p, _c_f64p])
        lib.orc_rk_step.restype = ctypes.c_int
        lib.orc_rk_step.argtypes = ([ctypes.c_int64, _c_i64p] + [ctypes.c_double] * 3
                                    + [_c_f64p, _c_f64p, ctypes.c_int, _c_f64p] + [ctypes.c_double] * 4
                                    + [ctypes.c_int, _c_f64p, _c_f64p, _c_f64p, _c_f64p])
        lib.orc_rk4_step.restype = ctypes.c_int
        lib.orc_rk4_step.argtypes = ([ctypes.c_int64, _c_i64p] + [ctypes.c_double] * 3
                                     + [_c_f64p, _c_f64p, ctypes.c_int, _c_f64p]
                                     + [ctypes.c_double] * 4 + [_c_f64p])
        lib.orc_itp_step.restype = ctypes.c_double
        lib.orc_itp_step.argtypes = ([ctypes.c_int64, _c_i64p] + [ctypes.c_double] * 3
                                     + [_c_f64p] + [ctypes.c_double] * 3 + [_c_f64p])
        lib.orc_observables.restype = None
        lib.orc_observables.argtypes = ([ctypes.c_int64, _c_i64p] + [ctypes.c_double] * 3
                                        + [_c_f64p, ctypes.c_double, _c_f64p, _c_f64p])
        lib.orc_overlap.restype = None
        lib.orc_overlap.argtypes = [ctypes.c_int64, _c_f64p, _c_f64p, ctypes.c_double, _c_f64p]
        lib.orc_tf_mu.restype = ctypes.c_double
        lib.orc_tf_mu.argtypes = [ctypes.c_int64, _c_f64p] + [ctypes.c_double] * 3
        lib.orc_ramp_s.restype = ctypes.c_double
        lib.orc_ramp_s.argtypes = [ctypes.c_int, _c_f64p, ctypes.c_double, ctypes.c_double]
        lib.orc_rk4_adjoint_step.restype = ctypes.c_int
        lib.orc_rk4_adjoint_step.argtypes = ([ctypes.c_int64, _c_i64p] + [ctypes.c_double] * 3
                                             + [_c_f64p, _c_f64p, ctypes.c_int, _c_f64p]
                                             + [ctypes.c_double] * 4 + [_c_f64p, _c_f64p, _c_f64p])
        _lib = lib
        return lib


def set_threads(n: int) -> int:
    """Threads the oracle's OpenMP loops use from the calling thread on
    (host plumbing for timing, no arithmetic); returns the new maximum."""
    _load()
    gomp = ctypes.CDLL("libgomp.so.1")
    gomp.omp_set_num_threads(int(n))
    return int(gomp.omp_get_max_threads())


def _p64(a):
    return a.ctypes.data_as(_c_f64p) if a is not None else None


def _pi64(a):
    return a.ctypes.data_as(_c_i64p)


def _cvec(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a, a.view(np.float64).ctypes.data_as(_c_f64p)


class Grid:
    """The discrete problem of Sec. II A: a box, its spacings and the active set.

    ``mask`` is a boolean array of shape (nz, ny, nx).  Cells outside the mask
    are deleted from the Laplacian (psi == 0 there, never updated).
    """

    def __init__(self, mask: np.ndarray, h):
        mask = np.asarray(mask, dtype=bool)
        assert mask.ndim == 3
        self.nz, self.ny, self.nx = mask.shape
        self.h = tuple(float(x) for x in (h if np.ndim(h) else (h, h, h)))
        self.dV = self.h[0] * self.h[1] * self.h[2]
        self.mask = mask
        self.cells = np.flatnonzero(mask.ravel()).astype(np.int64)
        self.n = int(self.cells.size)
        self.nbr = np.empty((self.n, 6), dtype=np.int64)
        rc = _load().orc_neighbors(self.n, _pi64(self.cells), self.nx, self.ny,
                                   self.nz, _pi64(self.nbr))
        assert rc == 0

    # --- dense <-> compact ------------------------------------------------
    def compact(self, dense: np.ndarray) -> np.ndarray:
        return np.ascontiguousarray(np.asarray(dense).ravel()[self.cells])

    def dense(self, vec: np.ndarray, dtype=None) -> np.ndarray:
        vec = np.asarray(vec)
        out = np.zeros(self.nx * self.ny * self.nz, dtype=dtype or vec.dtype)
        out[self.cells] = vec
        return out.reshape(self.nz, self.ny, self.nx)

    def ijk(self) -> np.ndarray:
        c = self.cells
        return np.stack([c % self.nx, (c // self.nx) % self.ny, c // (self.nx * self.ny)], axis=1)

    @property
    def nbr_e(self) -> np.ndarray:
        """Edge-neighbour table (n, 12) of the 19-point stencil, built on first use."""
        if not hasattr(self, "_nbr_e"):
            e = np.empty((self.n, 12), dtype=np.int64)
            assert _load().orc_edge_neighbors(self.n, _pi64(self.cells), self.nx, self.ny, self.nz, _pi64(e)) == 0
            self._nbr_e = e
        return self._nbr_e


def laplacian(grid: Grid, psi: np.ndarray, stencil: int = 7) -> np.ndarray:
    """The 7-point (Eq. (B1)) or 19-point (App. B) Laplacian on the active cells."""
    psi, pp = _cvec(psi)
    out = np.empty(grid.n, dtype=np.complex128)
    op = out.view(np.float64).ctypes.data_as(_c_f64p)
    if stencil == 7:
        _load().orc_laplacian(grid.n, _pi64(grid.nbr), *grid.h, pp, op)
    elif stencil == 19:
        _load().orc_laplacian19(grid.n, _pi64(grid.nbr), _pi64(grid.nbr_e), *grid.h, pp, op)
    else:
        raise ValueError("stencil must be 7 or 19")
    return out


# --- steps with either stencil, in numpy on top of the C Laplacian --------
# (the C step functions use the 7-point stencil; these restate the same
#  steps with the Laplacian as a parameter, for the 19-point stencil)
def _V_at(V0, V1, knots, T, t):
    if V1 is None or knots is None:
        return V0
    s = ramp_s(knots, T, t)
    return (1.0 - s) * V0 + s * V1


def rhs(grid: Grid, V, g, y, stencil: int = 7) -> np.ndarray:
    """f(y) = -i (T + V + g|y|^2) y, T = -1/2 Laplacian (Eq. (8))."""
    y = np.asarray(y, dtype=np.complex128)
    return -1j * (-0.5 * laplacian(grid, y, stencil) + (V + g * np.abs(y) ** 2) * y)


def rk_step_np(grid: Grid, V0, psi, g, t, dt, method="RK4", V1=None, knots=None, T=0.0,
               stencil: int = 7) -> np.ndarray:
    """Butcher-form explicit RK step (TABLEAUX[method]) in numpy."""
    A, b, c = TABLEAUX[method]
    y0 = np.asarray(psi, dtype=np.complex128)
    k = []
    for i in range(len(b)):
        yi = y0 + dt * sum((A[i, j] * k[j] for j in range(i)), np.zeros_like(y0))
        k.append(rhs(grid, _V_at(V0, V1, knots, T, t + c[i] * dt), g, yi, stencil))
    return y0 + dt * sum(b[i] * k[i] for i in range(len(b)))


def itp_step_np(grid: Grid, V, psi, g, dt, N=1.0, stencil: int = 7):
    """The imaginary-time step in the paper's order (Eqs. (6)-(7)) in numpy;
    returns (new psi, norm before renormalisation)."""
    y = np.asarray(psi, dtype=np.complex128)
    E = np.exp(-V * dt / 2.0)
    y = y * E * (1.0 - g * np.abs(y) ** 2 * dt / 2.0)
    for _ in range(2):
        y = y - (dt / 2.0) * (-0.5 * laplacian(grid, y, stencil))
    y = y * E * (1.0 - g * np.abs(y) ** 2 * dt / 2.0)
    nrm = float(np.sum(np.abs(y) ** 2) * grid.dV)
    return y * np.sqrt(N / nrm), nrm


def observables_np(grid: Grid, V, g, psi, stencil: int = 7) -> dict:
    y = np.asarray(psi, dtype=np.complex128)
    rho = np.abs(y) ** 2
    Ty = -0.5 * laplacian(grid, y, stencil)
    norm = float(np.sum(rho) * grid.dV)
    e_kin = float(np.sum(np.real(np.conj(y) * Ty)) * grid.dV)
    e_pot = float(np.sum(V * rho) * grid.dV)
    e_int = float(np.sum(0.5 * g * rho ** 2) * grid.dV)
    return dict(norm=norm, energy=e_kin + e_pot + e_int, mu=(e_kin + e_pot + 2 * e_int) / norm,
                e_kin=e_kin, e_pot=e_pot, e_int=e_int)


def rhs_real(grid: Grid, V: np.ndarray, g: float, y: np.ndarray) -> np.ndarray:
    V = np.ascontiguousarray(V, dtype=np.float64)
    y, yp = _cvec(y)
    out = np.empty(grid.n, dtype=np.complex128)
    _load().orc_rhs_real(grid.n, _pi64(grid.nbr), *grid.h, _p64(V), float(g), yp,
                         out.view(np.float64).ctypes.data_as(_c_f64p))
    return out


def _ramp_args(V1, knots, T):
    if V1 is None or knots is None:
        return None, 0, None, 0.0
    V1 = np.ascontiguousarray(V1, dtype=np.float64)
    knots = np.ascontiguousarray(knots, dtype=np.float64)
    return V1, int(knots.size), knots, float(T)


def rk4_step(grid: Grid, V0, psi, g, t, dt, V1=None, knots=None, T=0.0) -> np.ndarray:
    """One classic RK4 step (Butcher form) of Eq. (8); returns the new psi."""
    V0 = np.ascontiguousarray(V0, dtype=np.float64)
    V1, nk, kn, T = _ramp_args(V1, knots, T)
    y = np.array(psi, dtype=np.complex128, copy=True)
    rc = _load().orc_rk4_step(grid.n, _pi64(grid.nbr), *grid.h, _p64(V0), _p64(V1), nk,
                              _p64(kn), T, float(g), float(t), float(dt),
                              y.view(np.float64).ctypes.data_as(_c_f64p))
    assert rc == 0
    return y


# Butcher tableaux (A strictly lower, b, c) of the explicit integrators whose
# memory-optimised forms App. A tabulates: Heun's third-order method (RKHE3),
# the classic fourth-order method (RK4) and the fifth-order solution of the
# Cash-Karp pair (RKCK).
def _tableau(A, b):
    from fractions import Fraction as F
    s = len(b)
    M = np.zeros((s, s))
    for i, row in enumerate(A):
        for j, v in enumerate(row):
            M[i, j] = float(F(v))
    bb = np.array([float(F(v)) for v in b])
    return M, bb, M.sum(axis=1)


TABLEAUX = {
    "RKHE3": _tableau([[], ["1/3"], ["0", "2/3"]], ["1/4", "0", "3/4"]),
    "RK4": _tableau([[], ["1/2"], ["0", "1/2"], ["0", "0", "1"]], ["1/6", "1/3", "1/3", "1/6"]),
    "RKCK": _tableau([[], ["1/5"], ["3/40", "9/40"], ["3/10", "-9/10", "6/5"],
                      ["-11/54", "5/2", "-70/27", "35/27"],
                      ["1631/55296", "175/512", "575/13824", "44275/110592", "253/4096"]],
                     ["37/378", "0", "250/621", "125/594", "0", "512/1771"]),
}


def rk_step(grid: Grid, V0, psi, g, t, dt, method="RK4", V1=None, knots=None, T=0.0) -> np.ndarray:
    """One explicit Runge-Kutta step in Butcher form (TABLEAUX[method]) of
    Eq. (8); returns the new psi."""
    A, b, c = TABLEAUX[method]
    V0 = np.ascontiguousarray(V0, dtype=np.float64)
    V1, nk, kn, T = _ramp_args(V1, knots, T)
    y = np.array(psi, dtype=np.complex128, copy=True)
    A = np.ascontiguousarray(A)
    rc = _load().orc_rk_step(grid.n, _pi64(grid.nbr), *grid.h, _p64(V0), _p64(V1), nk, _p64(kn), T,
                             float(g), float(t), float(dt), len(b), _p64(A), _p64(np.ascontiguousarray(b)),
                             _p64(np.ascontiguousarray(c)), y.view(np.float64).ctypes.data_as(_c_f64p))
    assert rc == 0
    return y


def itp_step(grid: Grid, V, psi, g, dt, N=1.0):
    """One imaginary-time split step with renormalisation (Eqs. (6)-(7)).

    Returns (new psi, norm before renormalisation)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    y = np.array(psi, dtype=np.complex128, copy=True)
    nrm = _load().orc_itp_step(grid.n, _pi64(grid.nbr), *grid.h, _p64(V), float(g), float(dt),
                               float(N), y.view(np.float64).ctypes.data_as(_c_f64p))
    return y, nrm


def observables(grid: Grid, V, g, psi) -> dict:
    V = np.ascontiguousarray(V, dtype=np.float64)
    psi, pp = _cvec(psi)
    out = np.zeros(7)
    _load().orc_observables(grid.n, _pi64(grid.nbr), *grid.h, _p64(V), float(g), pp, _p64(out))
    return dict(norm=out[0], energy=out[1], mu=out[2], nonfinite=int(out[3]),
                e_kin=out[4], e_pot=out[5], e_int=out[6])


def overlap(a, b, dV) -> complex:
    a, ap = _cvec(a)
    b, bp = _cvec(b)
    out = np.zeros(2)
    _load().orc_overlap(a.size, ap, bp, float(dV), _p64(out))
    return complex(out[0], out[1])


def tf_mu(V, dV, g, N) -> float:
    """Thomas-Fermi chemical potential of Eq. (5) for atom number N."""
    V = np.ascontiguousarray(np.asarray(V, dtype=np.float64).ravel())
    return float(_load().orc_tf_mu(V.size, _p64(V), float(dV), float(g), float(N)))


def ramp_s(knots, T, t) -> float:
    knots = np.ascontiguousarray(knots, dtype=np.float64)
    return float(_load().orc_ramp_s(knots.size, _p64(knots), float(T), float(t)))


def rk4_adjoint_step(grid: Grid, V0, V1, knots, T, g, t, dt, y0, lam):
    """Reverse one RK4 step: returns (dL/dy0, dL/dknots contribution)."""
    V0 = np.ascontiguousarray(V0, dtype=np.float64)
    V1, nk, kn, T = _ramp_args(V1, knots, T)
    y0, yp = _cvec(y0)
    lam = np.array(lam, dtype=np.complex128, copy=True)
    grad = np.zeros(max(nk, 1))
    rc = _load().orc_rk4_adjoint_step(grid.n, _pi64(grid.nbr), *grid.h, _p64(V0), _p64(V1), nk,
                                      _p64(kn), T, float(g), float(t), float(dt), yp,
                                      lam.view(np.float64).ctypes.data_as(_c_f64p), _p64(grad))
    assert rc == 0
    return lam, grad[:nk]


def ramp_loss_and_grad(grid: Grid, V0, V1, knots, T, g, dt, nsteps, psi0, psi_target, t0=0.0):
    """Infidelity L = 1 - |<psi_t|psi(T)>|^2 after nsteps RK4 steps, and dL/dknots.

    Forward: store every step's start state (small grids only); backward: the
    step adjoint in reverse order.  The loss gradient seed is
    dL/dpsi = -2 c psi_t dV with c = <psi_t|psi(T)>.
    """
    states = [np.array(psi0, dtype=np.complex128)]
    y = states[0]
    for s in range(nsteps):
        y = rk4_step(grid, V0, y, g, t0 + s * dt, dt, V1, knots, T)
        states.append(y)
    c = overlap(psi_target, y, grid.dV)
    loss = 1.0 - abs(c) ** 2
    lam = -2.0 * c * np.asarray(psi_target, dtype=np.complex128) * grid.dV
    grad = np.zeros(len(knots))
    for s in reversed(range(nsteps)):
        lam, gk = rk4_adjoint_step(grid, V0, V1, knots, T, g, t0 + s * dt, dt, states[s], lam)
        grad += gk
    return loss, grad, y


def ramp_stages(Vs, h, durations, g, N, dt, psi0, cut_factor=5.0, t_hold=0.0, method="RK4", stencil=7):
    """Multi-stage ramp of Sec. V through the dense potentials Vs[0..M].

    Stage i interpolates linearly in time from Vs[i] to Vs[i+1] over
    durations[i].  Before it runs, the region of interest is selected again
    with the cutoff cut_factor * max(mu_i, mu_{i+1}) (mu the Thomas-Fermi
    chemical potential of Eq. (5) for g and N): every cell below the cutoff
    in either endpoint potential.  The wavefunction is carried over on the
    cells the two regions share (remapped between the old and new grids).
    The stage takes ceil(d / dt) equal steps.  With t_hold > 0 a hold in the
    last potential follows on {Vs[-1] < cut_factor * mu_M}.

    stencil 19 takes the numpy steps with App. B's Laplacian.
    psi0 is a dense box array (zero outside its own region).  Returns the
    final dense psi and one record per stage (mu_a, mu_b, cut, n_active,
    steps, dt, norm_kept, norm_end).
    """
    h = tuple(float(x) for x in (h if np.ndim(h) else (h, h, h)))
    dV = h[0] * h[1] * h[2]
    mu = [tf_mu(V, dV, g, N) for V in Vs]
    psi = np.array(psi0, dtype=np.complex128)
    M = len(Vs) - 1
    records = []
    for i in range(M + (1 if t_hold > 0 else 0)):
        hold = i == M
        if hold:
            mu_a = mu_b = mu[M]
            cut = cut_factor * mu_a
            mask = Vs[M] < cut
            d = t_hold
        else:
            mu_a, mu_b = mu[i], mu[i + 1]
            cut = cut_factor * max(mu_a, mu_b)
            mask = (Vs[i] < cut) | (Vs[i + 1] < cut)
            d = durations[i]
        grid = Grid(mask, h)
        y = grid.compact(psi)          # cells outside the new region are dropped
        norm_kept = float(np.sum(np.abs(y) ** 2) * dV)
        n = max(1, int(np.ceil(d / dt * (1.0 - 1e-12))))
        dts = d / n
        if hold:
            V0, V1, knots = grid.compact(Vs[M]), None, None
        else:
            V0, V1, knots = grid.compact(Vs[i]), grid.compact(Vs[i + 1]), np.array([0.0, 1.0])
        for k in range(n):
            if stencil == 7:
                y = rk_step(grid, V0, y, g, k * dts, dts, method, V1, knots, d)
            else:
                y = rk_step_np(grid, V0, y, g, k * dts, dts, method, V1, knots, d, stencil)
        psi = grid.dense(y)
        records.append(dict(mu_a=mu_a, mu_b=mu_b, cut=cut, n_active=grid.n, steps=n, dt=dts,
                            norm_kept=norm_kept, norm_end=float(np.sum(np.abs(y) ** 2) * dV)))
    return psi, records

"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests
and the benchmark.

This module defines workloads only: boxes, potentials (the synthetic stand-ins
for the paper's RF-dressed bubble potentials), initial wavefunctions and ramp
schedules.  It performs none of the method's arithmetic (no Laplacian, no time
stepping, no reductions of the method) and imports neither the CUDA binding
nor the oracle.

Coordinates: cell (i, j, k) of an n-point axis with spacing h sits at
x_i = x0 + i*h with x0 = -(n-1)/2*h (box centred on the origin).  Dense arrays
have numpy shape (nz, ny, nx).  Units hbar = m = 1; psi is normalised to
N = sum |psi|^2 dV = 1 unless stated.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Box:
    nx: int
    ny: int
    nz: int
    hx: float
    hy: float
    hz: float

    @property
    def x0(self):
        return -(self.nx - 1) / 2.0 * self.hx

    @property
    def y0(self):
        return -(self.ny - 1) / 2.0 * self.hy

    @property
    def z0(self):
        return -(self.nz - 1) / 2.0 * self.hz

    @property
    def dV(self):
        return self.hx * self.hy * self.hz

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def axes(self):
        return (self.x0 + np.arange(self.nx) * self.hx,
                self.y0 + np.arange(self.ny) * self.hy,
                self.z0 + np.arange(self.nz) * self.hz)

    def coords_of(self, ijk: np.ndarray):
        """Cell-centre coordinates of integer cell indices (n, 3) = (i, j, k)."""
        ijk = np.asarray(ijk)
        return (self.x0 + ijk[:, 0] * self.hx, self.y0 + ijk[:, 1] * self.hy,
                self.z0 + ijk[:, 2] * self.hz)


def cubic_box(n: int, h: float) -> Box:
    return Box(n, n, n, h, h, h)


# ---------------------------------------------------------------- potentials
@dataclass(frozen=True)
class Harmonic:
    """V = 1/2 (wx^2 x^2 + wy^2 y^2 + wz^2 z^2)."""
    wx: float = 1.0
    wy: float = 1.0
    wz: float = 1.0

    def __call__(self, x, y, z):
        return 0.5 * (self.wx ** 2 * x * x + self.wy ** 2 * y * y + self.wz ** 2 * z * z)


@dataclass(frozen=True)
class EllipsoidShell:
    """V = 1/2 w^2 (rho - 1)^2, rho = sqrt(x^2/a^2 + y^2/b^2 + z^2/c^2).

    A thin ellipsoidal shell: the synthetic stand-in for the RF-dressed bubble
    potentials of Sec. V (whose coil and field data are not available)."""
    w: float
    a: float
    b: float
    c: float

    def __call__(self, x, y, z):
        rho = np.sqrt(x * x / self.a ** 2 + y * y / self.b ** 2 + z * z / self.c ** 2)
        return 0.5 * self.w ** 2 * (rho - 1.0) ** 2


def dense_potential(box: Box, pot) -> np.ndarray:
    """Potential sampled on every cell of the box, FP64, shape (nz, ny, nx)."""
    x, y, z = box.axes()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.ascontiguousarray(pot(X, Y, Z), dtype=np.float64)


@dataclass(frozen=True)
class ShellWorkload:
    """Anisotropic thin shell on a cubic box (the paper's bubble geometry).

    The shell's semi-axes are (a, b, c) = (1, 0.9, 0.8) in units where the box
    spacing is h = 1/a_cells.  The trap stiffness w and the reference chemical
    potential mu0 are fixed by a thin-shell closed form so that the parabolic
    (Thomas-Fermi-like) radial profile of N atoms at coupling g is
    ``width_cells`` cells wide along the x semi-axis; the active region is
    V < cut_factor * mu0.  mu0 is a workload constant, not a computed result.
    """
    n: int
    a_cells: float
    g: float
    N: float = 1.0
    width_cells: float = 6.0
    cut_factor: float = 5.0
    axes: tuple = (1.0, 0.9, 0.8)

    @property
    def h(self):
        return 1.0 / self.a_cells

    @property
    def box(self):
        return cubic_box(self.n, self.h)

    @property
    def mu0(self):
        a, b, c = self.axes
        U = 0.5 * self.width_cells * self.h / a
        # N = (4 pi a b c / g) * (4/3) mu0 * U  for a thin parabolic shell
        return 3.0 * self.g * self.N / (16.0 * math.pi * a * b * c * U)

    @property
    def w(self):
        U = 0.5 * self.width_cells * self.h / self.axes[0]
        return math.sqrt(2.0 * self.mu0) / U

    @property
    def V_cut(self):
        return self.cut_factor * self.mu0

    @property
    def potential(self):
        a, b, c = self.axes
        return EllipsoidShell(self.w, a, b, c)

    def stable_dt(self, courant: float = 0.2):
        """dt with dt * lambda_max = courant, lambda_max bounding the spectrum of
        T + V + g|psi|^2 on the active region (T's bound: 2/h^2 per axis)."""
        lam = 3.0 * 2.0 / self.h ** 2 + self.V_cut + 2.0 * self.mu0
        return courant / lam


# Headline shell: 1024^3 box, semi-axis 490 cells, g = 2000 (~2.9e7 active cells).
SHELL_1024 = ShellWorkload(n=1024, a_cells=490.0, g=2000.0)
# Small shells with the same structure for parity tests (several bricks, ragged).
SHELL_64 = ShellWorkload(n=64, a_cells=26.0, g=2000.0)
SHELL_96 = ShellWorkload(n=96, a_cells=41.0, g=2000.0)
SHELL_512 = ShellWorkload(n=512, a_cells=240.0, g=2000.0)


# ---------------------------------------------------------------- wavefunctions
def normalise(psi: np.ndarray, dV: float, N: float = 1.0) -> np.ndarray:
    s = np.sum(np.abs(psi) ** 2) * dV
    return psi * math.sqrt(N / s)


def gaussian_with_noise(box: Box, seed: int = 1, noise: float = 1e-3) -> np.ndarray:
    """exp(-r^2/2) plus `noise` times a seeded complex normal field, normalised."""
    x, y, z = box.axes()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    rng = np.random.default_rng(seed)
    psi = np.exp(-(X * X + Y * Y + Z * Z) / 2.0).astype(np.complex128)
    psi += noise * (rng.standard_normal(box.shape) + 1j * rng.standard_normal(box.shape))
    return normalise(psi, box.dV)


class SmoothPhase:
    """Seeded smooth random phase field: a sum of M random plane waves whose
    wave vectors are drawn from a Gaussian of width 1/corr, so that the field
    has correlation length ~corr and r.m.s. amplitude ``amp`` radians."""

    def __init__(self, seed: int, corr: float, amp: float = 0.1, M: int = 32):
        rng = np.random.default_rng(seed)
        self.k = rng.standard_normal((M, 3)) / corr
        self.phi = rng.uniform(0.0, 2.0 * math.pi, M)
        self.scale = amp * math.sqrt(2.0 / M)

    def __call__(self, x, y, z):
        out = np.zeros(np.shape(x), dtype=np.float64)
        for m in range(self.k.shape[0]):
            out += np.cos(self.k[m, 0] * x + self.k[m, 1] * y + self.k[m, 2] * z + self.phi[m])
        return self.scale * out


def shell_initial_psi(wl: ShellWorkload, x, y, z, seed: int = 2) -> np.ndarray:
    """Parabolic shell profile sqrt(max(mu0 - V, 0)/g) times a smooth seeded
    phase (correlation 4 cells, 0.1 rad), at the given coordinates; not
    normalised (normalise over the cells actually kept)."""
    V = wl.potential(x, y, z)
    amp = np.sqrt(np.maximum(wl.mu0 - V, 0.0) / wl.g)
    ph = SmoothPhase(seed, corr=4.0 * wl.h)(x, y, z)
    return amp * np.exp(1j * ph)


def random_state(shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def monotone_knots(n: int = 16, seed: int = 3) -> np.ndarray:
    """Seeded monotone schedule s_0 = 0 <= s_1 <= ... <= s_{n-1} = 1."""
    rng = np.random.default_rng(seed)
    inner = np.sort(rng.uniform(0.0, 1.0, n - 2))
    return np.concatenate([[0.0], inner, [1.0]])


# ---------------------------------------------------------------- ramps
@dataclass(frozen=True)
class RampWorkload:
    """Hollowing-out ramp: V(t) = (1 - s(t)) V0 + s(t) V1 from a compact
    harmonic trap V0 = 1/2 W^2 r^2 to the thin shell V1 of ``shell``, on a
    cubic box; the region of interest is the union {V0 < cut0} U {V1 < cut1}.
    W is fixed by the Thomas-Fermi radius of N atoms at coupling g being
    ``core_radius`` / sqrt(cut_factor) (so the harmonic region has radius
    ``core_radius``); both cutoffs are cut_factor times the reference chemical
    potentials.  Workload constants, not computed results."""
    shell: ShellWorkload
    core_radius: float

    @property
    def mu0_core(self):
        # Closed-form workload constant: a parabolic (Thomas-Fermi-like) cloud
        # of N atoms in W^2 r^2 / 2 has mu = (15 g N W^3 / (4 pi))^(2/5) / 2
        # and radius R = sqrt(2 mu) / W; W is picked so that R is the target.
        R = self.core_radius / math.sqrt(self.shell.cut_factor)
        c = (15.0 * self.shell.g * self.shell.N / (4.0 * math.pi)) ** 0.4
        W = (c / R ** 2) ** (1.0 / 0.8)
        return 0.5 * W * W * R * R

    @property
    def W(self):
        R = self.core_radius / math.sqrt(self.shell.cut_factor)
        return math.sqrt(2.0 * self.mu0_core) / R

    @property
    def cut0(self):
        return self.shell.cut_factor * self.mu0_core

    @property
    def cut1(self):
        return self.shell.V_cut

    @property
    def v0(self):
        return Harmonic(self.W, self.W, self.W)

    def stable_dt(self, courant: float = 0.2):
        h = self.shell.h
        lam = 6.0 / h ** 2 + max(self.cut0, self.cut1) + 2.0 * max(self.mu0_core, self.shell.mu0)
        return courant / lam


# 2048^3 box, shell semi-axis 800 cells (~7.7e7 active) plus a harmonic core of
# radius 0.24 (~3e7 active): about 1e8 active cells, g = 5000
RAMP_2048 = RampWorkload(ShellWorkload(n=2048, a_cells=800.0, g=5000.0), core_radius=0.24)
# 512^3 box, ~5e6 active: the adjoint workload
RAMP_512 = RampWorkload(ShellWorkload(n=512, a_cells=200.0, g=5000.0), core_radius=0.24)
# 48^3 version for parity tests
RAMP_48 = RampWorkload(ShellWorkload(n=48, a_cells=19.0, g=5000.0), core_radius=0.24)
# 64^3 version of the adjoint workload, small enough for the FP64 oracle adjoint
RAMP_64 = RampWorkload(ShellWorkload(n=64, a_cells=24.0, g=5000.0), core_radius=0.24)


def stage_fractions(n_stages: int = 66) -> np.ndarray:
    """Blend fractions s_k = k / n_stages of the stage potentials
    V_k = (1 - s_k) V0 + s_k V1 of a multi-stage ramp between a ramp
    workload's two endpoints: synthetic stand-ins for the precomputed
    potentials of Sec. V (67 potentials, 66 stages)."""
    return np.arange(n_stages + 1, dtype=np.float64) / n_stages


def batch_shells(n: int = 64, seed: int = 4, scale_cells: float = 360.0):
    """Seeded batch of uneven ellipsoidal shells: radius r ~ U[0.5, 1] (semi-axis
    r * scale_cells cells), aspect ratios b/a, c/a ~ U[0.7, 1], thickness
    ~ U[4, 10] cells, g ~ U[100, 3000]; the box is the smallest cube holding
    the active band with a 4-cell margin."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        r = rng.uniform(0.5, 1.0)
        ar = (1.0, rng.uniform(0.7, 1.0), rng.uniform(0.7, 1.0))
        width = rng.uniform(4.0, 10.0)
        g = rng.uniform(100.0, 3000.0)
        a_cells = r * scale_cells
        band = math.sqrt(5.0) * width / 2.0
        nbox = int(2 * math.ceil(a_cells + band + 4))
        out.append(ShellWorkload(n=nbox, a_cells=a_cells, g=g, width_cells=width, axes=ar))
    return out

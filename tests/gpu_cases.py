"""Seeded cases shared by the GPU parity tests (inputs only, no method arithmetic)."""
import math

import numpy as np

from paper_2603_05447_gb300 import gpe, inputs


class Case:
    """A box, a dense potential (or two for a ramp), a cutoff and an initial psi."""

    def __init__(self, name, box, V, V_cut, psi, g, dt, V1=None):
        self.name, self.box, self.V, self.V_cut, self.psi = name, box, V, V_cut, psi
        self.g, self.dt, self.V1 = g, dt, V1
        self.mask = V < V_cut if V1 is None else None

    @property
    def gbox(self):
        b = self.box
        return gpe.make_box(b.nx, b.ny, b.nz, b.hx, b.hy, b.hz, b.x0, b.y0, b.z0)


def harmonic64(g=100.0):
    """64^3 isotropic trap, h = 0.25, every cell active, Gaussian + 1e-3 noise."""
    box = inputs.cubic_box(64, 0.25)
    V = inputs.dense_potential(box, inputs.Harmonic())
    psi = inputs.gaussian_with_noise(box, seed=1, noise=1e-3)
    return Case("harmonic64", box, V, np.inf, psi, g, 1e-3)


def shell(wl=inputs.SHELL_64, seed=2):
    box = wl.box
    V = inputs.dense_potential(box, wl.potential)
    x, y, z = box.axes()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    psi = np.where(V < wl.V_cut, inputs.shell_initial_psi(wl, X, Y, Z, seed=seed), 0)
    psi = inputs.normalise(psi.astype(np.complex128), box.dV)
    return Case(f"shell{wl.n}", box, V, wl.V_cut, psi, wl.g, wl.stable_dt())


def ragged_shell():
    """Box sizes that are not multiples of any brick edge, anisotropic spacings."""
    box = inputs.Box(61, 53, 45, 0.040, 0.043, 0.047)
    pot = inputs.EllipsoidShell(w=60.0, a=1.0, b=0.9, c=0.8)
    V = inputs.dense_potential(box, pot)
    rng = np.random.default_rng(5)
    cut = 3.0
    psi = np.where(V < cut, np.exp(-V) * np.exp(1j * rng.uniform(0, 0.3, box.shape)), 0).astype(np.complex128)
    psi = inputs.normalise(psi, box.dV)
    lam = 2 / box.hx ** 2 + 2 / box.hy ** 2 + 2 / box.hz ** 2 + cut
    return Case("ragged", box, V, cut, psi, 50.0, 0.2 / lam)


def single_cell():
    box = inputs.cubic_box(9, 0.3)
    V = np.full(box.shape, 10.0)
    V[4, 3, 5] = 0.5
    psi = np.zeros(box.shape, np.complex128)
    psi[4, 3, 5] = 1.0 + 0.5j
    return Case("single", box, V, 1.0, psi, 3.0, 1e-3)


def ramp_case():
    """Harmonic -> shell blend on a 48^3 box; region = union of both cutoffs."""
    box = inputs.cubic_box(48, 0.06)
    V0 = inputs.dense_potential(box, inputs.Harmonic(3.0, 3.0, 3.0))
    V1 = inputs.dense_potential(box, inputs.EllipsoidShell(w=40.0, a=1.0, b=0.9, c=0.8))
    c0, c1 = 4.0, 4.0
    region = (V0 < c0) | (V1 < c1)
    x, y, z = box.axes()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    psi = np.where(region, np.exp(-(X * X + Y * Y + Z * Z) * 2.0), 0).astype(np.complex128)
    psi = inputs.normalise(psi, box.dV)
    lam = 6 / box.hx ** 2 + max(c0, c1) * 4
    case = Case("ramp", box, V0, c0, psi, 20.0, 0.2 / lam, V1=V1)
    case.region = region
    case.cut1 = c1
    case.knots = inputs.monotone_knots(16, seed=3)
    case.T = 40 * case.dt
    return case


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def tiny_box(nx, ny, nz, h=(0.3, 0.35, 0.4), seed=9):
    """A box smaller than one brick in some or all dimensions (down to a
    single cell), every cell active, anisotropic spacings, seeded complex
    psi; for the degenerate layouts (bricks mostly outside the box)."""
    box = inputs.Box(nx, ny, nz, *h)
    V = inputs.dense_potential(box, inputs.Harmonic(1.0, 1.3, 0.8))
    rng = np.random.default_rng(seed)
    psi = (rng.normal(size=box.shape) + 1j * rng.normal(size=box.shape)).astype(np.complex128)
    psi = inputs.normalise(psi, box.dV)
    lam = 2 / box.hx ** 2 + 2 / box.hy ** 2 + 2 / box.hz ** 2 + float(V.max())
    return Case(f"tiny{nx}x{ny}x{nz}", box, V, np.inf, psi, 2.0, 0.2 / lam)

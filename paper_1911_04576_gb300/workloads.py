"""Seeded synthetic workloads (input recipes only -- no arithmetic of the method).

Every number the method consumes is drawn here from numpy.random.default_rng
with an explicit seed, with the shapes of the paper's reflectarray problems
(Sec. V): f = 10 GHz (lambda = 30 mm), period lambda/2, boxes of height
lambda/4 meshed n x n per face (K = 36 n^2 unknowns per box), a 0.76 mm
eps_r = 3, tan delta = 0.001 slab filling the bottom of every cell, one PEC
square patch per cell on the slab top, sides drawn uniformly from a type
library, a cell -> type map, plane-wave incidence angles.

Both the oracle-side tests and the product's bench/tests take their inputs
from here; neither side's arithmetic is in this module.
"""
from dataclasses import dataclass, field

import numpy as np

LAMBDA = 0.03
K0 = 2.0 * np.pi / LAMBDA
PERIOD = 0.5 * LAMBDA
BOX_H = 0.25 * LAMBDA
PATCH_Z = 0.76e-3
SLAB_T = 0.76e-3                     # slab thickness: the patch sits on its top
EPS_SLAB = 3.0 * (1.0 - 0.001j)      # eps_r (1 - j tan delta), tan delta = 0.001, e^{jwt}
RING_LAYERS = 3                      # slab-top mesh: graded rings around the patch


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    n: int                       # box face mesh n x n  (E = 18 n^2, K = 2E)
    n_types: int
    side_lo: float               # patch side range, in wavelengths
    side_hi: float
    n_rhs: int = 1
    patch_n: int = 4             # patch mesh n x n quads
    seed: int = 0
    type_rule: str = "random"    # "random" or "gradient" (type = ix mod T)
    angles: list = field(default_factory=list)   # (theta_deg, phi_deg, pol) per rhs

    @property
    def E(self):
        return 18 * self.n * self.n

    @property
    def K(self):
        return 2 * self.E

    @property
    def M(self):
        return self.nx * self.ny


def normal_incidence():
    return [(0.0, 0.0, "theta")]


WORKLOADS = {
    # 3x3 lattice, 3x3-quad faces (K = 324), dense oracle solve in seconds
    "lattice3x3_k324": Workload("lattice3x3_k324", 3, 3, 3, 9, 0.20, 0.45, 1, 4, 11,
                                angles=normal_incidence()),
    # 16x16 lattice, K = 576, 32 patch types, one normal-incidence rhs
    "lattice16x16_k576": Workload("lattice16x16_k576", 16, 16, 4, 32, 0.15, 0.45, 1, 4, 16,
                                  angles=normal_incidence()),
    # 12x12 lattice, K = 576: the bin multiply of the 16x16 case on a smaller
    # grid (576 bins, 0.76 GB of complex64 blocks > L2) for profiler captures
    "lattice12x12_k576": Workload("lattice12x12_k576", 12, 12, 4, 32, 0.15, 0.45, 1, 4, 12,
                                  angles=normal_incidence()),
    # 48x48 lattice, K = 576, 32 types, 32 plane waves
    "lattice48x48_k576_r32": Workload(
        "lattice48x48_k576_r32", 48, 48, 4, 32, 0.15, 0.45, 32, 4, 48,
        angles=[(4.0 * i, 0.0, "theta") for i in range(16)] + [(4.0 * i, 90.0, "phi") for i in range(16)]),
    # 100x100 lattice, K = 324, 64-type phase-gradient map, 8 plane waves
    "lattice100x100_k324_r8": Workload(
        "lattice100x100_k324_r8", 100, 100, 3, 64, 0.15, 0.45, 8, 4, 100, type_rule="gradient",
        angles=[(t, 0.0, p) for t in (0.0, 15.0, 30.0, 45.0) for p in ("theta", "phi")]),
}


def patch_sides(w: Workload):
    """Patch side per type in metres (uniform draw, or linear for a gradient map)."""
    if w.type_rule == "gradient":
        t = np.arange(w.n_types) / max(1, w.n_types - 1)
        return (w.side_lo + (w.side_hi - w.side_lo) * t) * LAMBDA
    rng = np.random.default_rng(w.seed)
    return rng.uniform(w.side_lo, w.side_hi, w.n_types) * LAMBDA


def type_map(w: Workload):
    """Cell -> type, cells numbered m = iy*nx + ix."""
    if w.type_rule == "gradient":
        ix = np.tile(np.arange(w.nx), w.ny)
        return (ix % w.n_types).astype(np.int32)
    rng = np.random.default_rng(w.seed + 1)
    return rng.integers(0, w.n_types, w.M).astype(np.int32)


def plane_waves(w: Workload):
    """(khat, ehat) per rhs: incidence from above, theta/phi polarisation."""
    out = []
    for th, ph, pol in w.angles[: w.n_rhs]:
        t, p = np.radians(th), np.radians(ph)
        khat = -np.array([np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)])
        theta_hat = np.array([np.cos(t) * np.cos(p), np.cos(t) * np.sin(p), -np.sin(t)])
        phi_hat = np.array([-np.sin(p), np.cos(p), 0.0])
        out.append((khat, theta_hat if pol == "theta" else phi_hat))
    return out


def random_vectors(R, n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((R, n)) + 1j * rng.standard_normal((R, n))


def random_tables(nx, ny, E, seed, decay=1.0):
    """Synthetic offset tables with the magnitude profile of free-space
    coupling (|block| ~ 1/(1+|d|)) and random phases; (2ny-1, 2nx-1, E, E)."""
    rng = np.random.default_rng(seed)
    shape = (2 * ny - 1, 2 * nx - 1, E, E)
    dy = np.arange(-(ny - 1), ny)[:, None]
    dx = np.arange(-(nx - 1), nx)[None, :]
    amp = (1.0 / (1.0 + decay * np.hypot(dx, dy)))[:, :, None, None]
    L = amp * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    K = amp * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    return L, K


def random_macromodels(T, K, seed, diag=0.0):
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((T, K, K)) + 1j * rng.standard_normal((T, K, K))
    if diag:
        Z += diag * np.eye(K)[None]
    return Z

"""Seeded synthetic inputs for the SRD step: workload recipes and initial states.

This module holds none of the method's arithmetic (no streaming, binning, reduction or
rotation).  It only draws states with the shapes and distributions of the paper's workloads
(arXiv 2212.11878, Sec. 4: a pure fluid in a periodic cubic box, cells of edge a = 1 holding
<N_c> = 10 particles on average, N = 10 L^3), so that the CUDA library and the CPU oracle can
start from identical inputs.  It imports neither of them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

BASE_SEED = 20221211


@dataclass(frozen=True)
class Workload:
    """One SRD configuration.  Lengths in units of the cell edge a; alpha in degrees."""

    name: str
    L: tuple
    ppc: float = 10.0
    a: float = 1.0
    dt: float = 0.1
    alpha_deg: float = 130.0
    kT: float = 1.0
    mass: float = 1.0
    seed: int = BASE_SEED
    precision: str = "fp64"          # "fp64" or "mixed"
    resort_k: int = 1
    walls_z: int = 0
    g: tuple = (0.0, 0.0, 0.0)
    thermostat: int = 0
    angular: int = 0
    mass_range: tuple = ()           # per-particle masses uniform in this range (times m)
    steps: int = 100
    notes: str = ""

    @property
    def cells(self) -> int:
        return int(self.L[0]) * int(self.L[1]) * int(self.L[2])

    @property
    def n_particles(self) -> int:
        return int(round(self.ppc * self.cells))

    @property
    def alpha(self) -> float:
        return math.radians(self.alpha_deg)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


# The five workloads the project measures (shapes from the paper's benchmark fluid).
WORKLOADS = {
    "fp64_L16": Workload("fp64_L16", (16, 16, 16), seed=BASE_SEED + 0, steps=100, resort_k=1,
                         notes="plain FP64 SRD, 40,960 particles, 100 steps"),
    "fp64_L64": Workload("fp64_L64", (64, 64, 64), seed=BASE_SEED + 1, steps=100, resort_k=10,
                         notes="plain FP64 SRD, 2,621,440 particles (profiling size, state > L2)"),
    "fp64_L128": Workload("fp64_L128", (128, 128, 128), seed=BASE_SEED + 1, steps=1000, resort_k=10,
                          notes="plain FP64 SRD, 20,971,520 particles, full re-sort every 10 steps"),
    "mixed_L64": Workload("mixed_L64", (64, 64, 64), seed=BASE_SEED + 2, steps=500, precision="mixed", resort_k=1,
                          notes="mixed form, 2,621,440 particles (error sub-run and profiling size)"),
    "mixed_L128": Workload("mixed_L128", (128, 128, 128), seed=BASE_SEED + 2, steps=500, precision="mixed", resort_k=1,
                           notes="mixed form, 20,971,520 particles"),
    "mixed_L256": Workload("mixed_L256", (256, 256, 256), seed=BASE_SEED + 2, steps=500, precision="mixed",
                           resort_k=1, notes="int32 cell + FP32 offset positions, FP32 velocities"),
    "poiseuille_256x64x64": Workload("poiseuille_256x64x64", (256, 64, 64), ppc=20.0, seed=BASE_SEED + 3,
                                     steps=20000, precision="mixed", resort_k=1, walls_z=1,
                                     g=(1e-3, 0.0, 0.0), thermostat=1,
                                     notes="bounce-back walls in z, body force along x"),
    "fp64_L128_angular": Workload("fp64_L128_angular", (128, 128, 128), seed=BASE_SEED + 1, steps=1000, resort_k=10,
                                  angular=1, notes="angular-momentum-conserving collision, FP64"),
    "fp64_L128_masses": Workload("fp64_L128_masses", (128, 128, 128), seed=BASE_SEED + 1, steps=1000, resort_k=10,
                                 mass_range=(0.5, 4.0), notes="per-particle masses 0.5-4 m, FP64"),
    "mixed_L128_angular": Workload("mixed_L128_angular", (128, 128, 128), seed=BASE_SEED + 2, steps=500,
                                   precision="mixed", resort_k=1, angular=1,
                                   notes="angular-momentum-conserving collision, mixed form (per-cell path)"),
    "mixed_L128_masses": Workload("mixed_L128_masses", (128, 128, 128), seed=BASE_SEED + 2, steps=500,
                                  precision="mixed", resort_k=1, mass_range=(0.5, 4.0),
                                  notes="per-particle masses 0.5-4 m, mixed form (FP32 masses, per-cell path)"),
    "poiseuille_256x64x64_mbs": Workload("poiseuille_256x64x64_mbs", (256, 64, 64), ppc=20.0, seed=BASE_SEED + 3,
                                         steps=20000, precision="mixed", resort_k=1, walls_z=1,
                                         g=(1e-3, 0.0, 0.0), thermostat=2,
                                         notes="the channel with the Maxwell-Boltzmann-scaling cell thermostat"),
}


def particle_masses(n: int, seed: int, lo: float, hi: float, mass: float = 1.0):
    """Per-particle masses uniform in [lo, hi) times mass, in particle-id order."""
    rng = np.random.Generator(np.random.Philox(seed + 7))
    return np.ascontiguousarray(rng.uniform(lo, hi, n) * mass)


def uniform_gaussian_state(L, n: int, seed: int, a: float = 1.0, kT: float = 1.0, mass: float = 1.0):
    """Positions uniform in [0, L_d a), velocities N(0, kT/m) per component with the net
    momentum removed.  Returns (r, v) as (n, 3) float64 arrays."""
    rng = np.random.Generator(np.random.Philox(seed))
    box = np.asarray(L, dtype=np.float64) * a
    r = rng.random((n, 3)) * box
    r = np.minimum(r, np.nextafter(box, 0.0))  # keep every coordinate strictly inside
    v = rng.standard_normal((n, 3)) * math.sqrt(kT / mass)
    if n:
        v -= v.mean(axis=0)
    return np.ascontiguousarray(r), np.ascontiguousarray(v)


def shell_state(L, n: int, seed: int, a: float = 1.0, kT: float = 1.0, mass: float = 1.0):
    """A deliberately non-Maxwellian start: every speed equals sqrt(3 kT / m), directions
    uniform on the sphere, net momentum removed.  Used to watch the collisions relax the
    distribution."""
    rng = np.random.Generator(np.random.Philox(seed))
    box = np.asarray(L, dtype=np.float64) * a
    r = np.minimum(rng.random((n, 3)) * box, np.nextafter(box, 0.0))
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    v = d * math.sqrt(3.0 * kT / mass)
    if n:
        v -= v.mean(axis=0)
    return np.ascontiguousarray(r), np.ascontiguousarray(v)


def face_state(L, n: int, seed: int, a: float = 1.0, kT: float = 1.0, mass: float = 1.0, denominator: int = 8):
    """Edge-case positions: every coordinate on a lattice of spacing a/denominator (cell faces
    included), a few at 0 and just below the box edge.  Velocities Gaussian."""
    rng = np.random.Generator(np.random.Philox(seed))
    box = np.asarray(L, dtype=np.float64) * a
    steps = (np.asarray(L) * denominator).astype(np.int64)
    r = rng.integers(0, steps, size=(n, 3)).astype(np.float64) * (a / denominator)
    if n >= 4:
        r[0] = 0.0
        r[1] = np.nextafter(box, 0.0)
        r[2] = np.minimum(np.full(3, a), np.nextafter(box, 0.0))
        r[3] = box / 2
    v = rng.standard_normal((n, 3)) * math.sqrt(kT / mass)
    return np.ascontiguousarray(r), np.ascontiguousarray(v)


@dataclass
class BatchRecipe:
    """Uneven ensemble of independent periodic boxes."""

    sides: list = field(default_factory=list)
    ppc: list = field(default_factory=list)
    alpha_deg: list = field(default_factory=list)
    dt: list = field(default_factory=list)
    seeds: list = field(default_factory=list)

    @property
    def nbox(self) -> int:
        return len(self.sides)

    @property
    def n_particles(self) -> int:
        return int(sum(round(p * s ** 3) for s, p in zip(self.sides, self.ppc)))

    @property
    def cells(self) -> int:
        return int(sum(s ** 3 for s in self.sides))


def batch_recipe(nbox: int = 256, meta_seed: int = BASE_SEED, side_choices=(8, 12, 16, 24, 32, 48, 64),
                 ppc_range=(5, 20), alpha_range=(60.0, 150.0), dt_choices=(0.05, 0.1, 0.2)) -> BatchRecipe:
    """Sides uniform over ``side_choices``, integer particles per cell uniform in
    ``ppc_range`` (inclusive), alpha uniform in ``alpha_range`` degrees, dt uniform over
    ``dt_choices``, distinct seeds."""
    rng = np.random.Generator(np.random.Philox(meta_seed))
    rec = BatchRecipe()
    for b in range(nbox):
        rec.sides.append(int(rng.choice(side_choices)))
        rec.ppc.append(float(rng.integers(ppc_range[0], ppc_range[1] + 1)))
        rec.alpha_deg.append(float(rng.uniform(*alpha_range)))
        rec.dt.append(float(rng.choice(dt_choices)))
        rec.seeds.append(int(meta_seed * 1000 + b))
    return rec


# Ensembles: many independent periodic boxes advanced together (mixed form).
BATCH_WORKLOADS = {
    "batched_256": dict(nbox=256, meta_seed=BASE_SEED, side_choices=(8, 12, 16, 24, 32, 48, 64), ppc_range=(5, 20),
                        alpha_range=(60.0, 150.0), dt_choices=(0.05, 0.1, 0.2), steps=1000,
                        notes="256 uneven boxes, sides 8-64, 5-20 particles per cell, alpha 60-150 deg"),
    "batched_32": dict(nbox=32, meta_seed=BASE_SEED + 7, side_choices=(8, 12, 16, 24), ppc_range=(5, 20),
                       alpha_range=(60.0, 150.0), dt_choices=(0.05, 0.1, 0.2), steps=100,
                       notes="small ensemble for tests and profiling"),
}


def batch_workload(name: str) -> BatchRecipe:
    w = dict(BATCH_WORKLOADS[name])
    for k in ("steps", "notes"):
        w.pop(k)
    return batch_recipe(**w)

"""Seeded synthetic inputs for the periodic thermal-microstructure design loop.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic, so both the CPU oracle's tests and the CUDA path's tests
and benchmark may use it.

Layout convention shared by every consumer: a scalar field on an n^3 periodic
voxel grid is a flat array of length n^3 in which x varies fastest, i.e. voxel
(x, y, z) lives at index x + n*(y + n*z).  A numpy array of shape (n, n, n)
indexed [z, y, x] and flattened in C order has exactly this layout.

The workloads mirror the paper's examples (Sec. 4: resolution 128^3, SIMP
p = 3, OC step 0.05, damping 0.5; Fig. 1 targets) with densities drawn as
``volfrac + U(-0.05, 0.05)``.  The paper's own IWP/TPMS initial fields are not
specified in the paper and are not used.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

# Target tensors of the paper's teaser figure (isotropic, orthotropic,
# anisotropic), ordered [k11, k22, k33, k12, k23, k13] as in Eq. (rep).
TARGET_ISOTROPIC = (0.1, 0.1, 0.1, 0.0, 0.0, 0.0)
TARGET_ORTHOTROPIC = (0.3, 0.2, 0.1, 0.0, 0.0, 0.0)
TARGET_ANISOTROPIC = (0.3, 0.2, 0.1, 0.1, 0.05, 0.05)


@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    kappa_target: tuple
    volfrac: float
    penal: float = 3.0
    rmin: float = 1.5
    k_solid: float = 1.0
    k_void: float = 1e-3
    cg_tol: float = 1e-6
    oc_iters: int = 50
    seed: int = 0
    precision: str = "fp32"

    @property
    def nelem(self) -> int:
        return self.n ** 3

    def rho0(self, dtype=np.float64) -> np.ndarray:
        return initial_density(self.n, self.volfrac, self.seed, dtype)


def initial_density(n: int, volfrac: float, seed: int, dtype=np.float64) -> np.ndarray:
    """rho0 = volfrac + U(-0.05, 0.05), drawn in float64, x fastest."""
    rng = np.random.default_rng(seed)
    rho = volfrac + rng.uniform(-0.05, 0.05, size=n ** 3)
    return rho.astype(dtype)


def random_density(n: int, seed: int, lo: float = 0.0, hi: float = 1.0,
                   dtype=np.float64) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=n ** 3).astype(dtype)


def random_field(n: int, seed: int, ncomp: int = 3, dtype=np.float64) -> np.ndarray:
    """Standard-normal field of shape (ncomp, n^3): test vectors for operators."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((ncomp, n ** 3)).astype(dtype)


def random_spd_target(rng: np.random.Generator, lo: float = 0.05, hi: float = 0.35):
    """Q diag(lam) Q^T with lam ~ U[lo, hi] and Q the Q factor of a 3x3
    standard-normal matrix, signs fixed so diag(R) > 0 and det Q = +1.
    Returned in the [k11, k22, k33, k12, k23, k13] order."""
    lam = rng.uniform(lo, hi, size=3)
    a = rng.standard_normal((3, 3))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    m = q @ np.diag(lam) @ q.T
    return (m[0, 0], m[1, 1], m[2, 2], m[0, 1], m[1, 2], m[0, 2])


# 16^3 plain-method case the oracle finishes in seconds.
SMALL_16 = Workload(name="periodic-16^3-isotropic", n=16, kappa_target=TARGET_ISOTROPIC,
                    volfrac=0.3, rmin=1.5, cg_tol=1e-8, oc_iters=50, seed=0,
                    precision="fp64")
# 128^3 orthotropic plain-FP32 case (2,097,152 elements).
ORTHO_128 = Workload(name="periodic-128^3-orthotropic", n=128,
                     kappa_target=TARGET_ORTHOTROPIC, volfrac=0.3, rmin=2.0,
                     cg_tol=1e-6, oc_iters=200, seed=1, precision="fp32")
# Mixed-precision anisotropic cases.
ANISO_128 = Workload(name="periodic-128^3-anisotropic", n=128,
                     kappa_target=TARGET_ANISOTROPIC, volfrac=0.35, rmin=2.0,
                     cg_tol=1e-6, oc_iters=200, seed=2, precision="mixed")
ANISO_256 = Workload(name="periodic-256^3-anisotropic", n=256,
                     kappa_target=TARGET_ANISOTROPIC, volfrac=0.35, rmin=2.0,
                     cg_tol=1e-6, oc_iters=200, seed=2, precision="mixed")


@dataclass(frozen=True)
class BatchDesign:
    index: int
    n: int
    kappa_target: tuple
    volfrac: float
    seed: int

    def rho0(self, dtype=np.float64) -> np.ndarray:
        return initial_density(self.n, self.volfrac, self.seed, dtype)


def batch_designs(count: int = 64, sizes=(32, 48, 64, 96), base_seed: int = 1000) -> List[BatchDesign]:
    """Batched workload: design d uses seed base_seed + d for n ~ U{sizes},
    a random SPD target with eigenvalues in [0.05, 0.35] and
    volfrac ~ U[0.2, 0.45]."""
    out = []
    for d in range(count):
        rng = np.random.default_rng(base_seed + d)
        n = int(rng.choice(np.asarray(sizes)))
        tgt = random_spd_target(rng)
        vf = float(rng.uniform(0.2, 0.45))
        out.append(BatchDesign(index=d, n=n, kappa_target=tuple(float(t) for t in tgt),
                               volfrac=vf, seed=base_seed + d))
    return out

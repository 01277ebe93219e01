"""Seeded synthetic workloads: lattice sizes, seeds, temperatures and sweep counts.

The paper's inputs are random +-J lattices (Sec. 1, Eq. 2), so these recipes are
the workloads themselves.  This module draws only the parameters of each job;
the couplings, spins and random streams are generated inside the library (and,
independently, inside the oracle) from the seeds given here.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Lattice:
    L: int
    seed_J: int
    seed_spin: int
    T: float
    kind: str          # "minstd" or "mt19937"
    sweeps: int

    @property
    def beta(self) -> float:
        return 1.0 / self.T

    @property
    def attempts_per_sweep(self) -> int:
        return self.L ** 3


# L = 32, quench at T = 1.1, MINSTD, 1000 sweeps, energy logged every sweep.
SMALL = Lattice(L=32, seed_J=1, seed_spin=2, T=1.1, kind="minstd", sweeps=1000)
# L = 256, quench at T = 0.7, 10^4 sweeps, both generators; measured at 2^k.
MEDIUM_MINSTD = Lattice(L=256, seed_J=1, seed_spin=2, T=0.7, kind="minstd", sweeps=10_000)
MEDIUM_MT = Lattice(L=256, seed_J=1, seed_spin=2, T=0.7, kind="mt19937", sweeps=10_000)
# L = 1024, MT19937, quench at T = 0.9, 1000 sweeps: the headline psFlip workload.
LARGE = Lattice(L=1024, seed_J=1, seed_spin=2, T=0.9, kind="mt19937", sweeps=1000)

BATCH_SIZES = (16, 32, 48, 64, 96, 128, 192)
BATCH_TEMPS = (0.7, 0.9, 1.1)


@dataclass(frozen=True)
class BatchSample:
    L: int
    seed_J: int
    seed_spin: tuple      # two replicas
    T: float


def batch_samples(n: int = 512, sampler_seed: int = 7) -> list[BatchSample]:
    """n disorder samples: L uniform over BATCH_SIZES, T uniform over BATCH_TEMPS,
    seed_J = 1000 + s, replica spin seeds 2s and 2s + 1."""
    rng = np.random.default_rng(sampler_seed)
    Ls = rng.choice(BATCH_SIZES, size=n)
    Ts = rng.choice(BATCH_TEMPS, size=n)
    return [BatchSample(int(Ls[s]), 1000 + s, (2 * s, 2 * s + 1), float(Ts[s])) for s in range(n)]


def amsc_seeds(L: int) -> tuple[list[int], list[int]]:
    """Seeds of the 32 systems of an asynchronous multispin ensemble of size L:
    system b has seed_J = 5000 + 64 b + L and seed_spin = 5001 + 64 b + L."""
    return ([5000 + 64 * b + L for b in range(32)], [5001 + 64 * b + L for b in range(32)])


@dataclass(frozen=True)
class Job:
    arrival: float        # seconds from the start of the trace
    L: int
    sweeps: int
    T: float
    kind: str
    seed_J: int
    seed_spin: int


def serving_trace(n_jobs: int, rate: float = 200.0, arrival_seed: int = 11) -> list[Job]:
    """Poisson arrivals (mean `rate` jobs/s); L uniform over even multiples of 16
    in [32, 512]; sweeps log-uniform in [1e2, 1e5]; T uniform in [0.5, 1.5];
    MINSTD or MT19937 with probability 1/2 each."""
    rng = np.random.default_rng(arrival_seed)
    gaps = rng.exponential(1.0 / rate, size=n_jobs)
    t = np.cumsum(gaps)
    Ls = rng.choice(np.arange(32, 513, 16), size=n_jobs)
    sweeps = np.floor(10 ** rng.uniform(2.0, 5.0, size=n_jobs)).astype(np.int64)
    Ts = rng.uniform(0.5, 1.5, size=n_jobs)
    kinds = rng.integers(0, 2, size=n_jobs)
    return [Job(float(t[j]), int(Ls[j]), int(sweeps[j]), float(Ts[j]), ("minstd", "mt19937")[int(kinds[j])],
                50_000 + j, 90_000 + j) for j in range(n_jobs)]

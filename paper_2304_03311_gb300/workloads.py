"""Seeded synthetic workloads: the parameter sets of the five benchmark
configurations, with the shapes of the paper's simulations (section 4: 2D
critical Ising, linear protocol, N_therm = 1000; section 5: 3D at beta_c).

This module only produces parameters (lattice sizes, couplings, l values,
trajectory counts, seeds, arrival times).  It holds none of the method's
arithmetic and is shared by the tests, the benchmark and the oracle runs alike.
Every job starts from Philox hot starts, so there is no input data beyond
these parameters.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

BETA_C_2D = 0.5 * math.log(1.0 + math.sqrt(2.0))     # section 4
BETA_C_3D = 0.221654626                              # section 5
BETA_3D_CONFIG = 0.22165455                          # 3D slab workload's own value


@dataclass(frozen=True)
class Job:
    d: int
    L: int
    L_t: int
    beta: float
    l: int
    n_step: int
    n_sweep: int
    n_traj: int
    seed: int = 0
    n_therm: int = 1000
    direction: int = 1
    traj0: int = 0
    update: int = 0          # 0 checkerboard Metropolis, 1 Swendsen-Wang
    protocol: int = 1        # 1 every switched column together, 2 one column at a time
    n_replica: int = 2       # replicas n
    whole: bool = False      # True: whole-cut transformation of the columns x < l
    therm_update: int = 0    # 1: Swendsen-Wang thermalisation before a Metropolis protocol

    @property
    def sites(self) -> int:
        return self.n_replica * self.L_t * self.L ** (self.d - 1)

    @property
    def updates(self) -> int:
        """Spin updates, every site visit of thermalisation and protocol."""
        return self.n_traj * self.sites * (self.n_therm + self.n_step * self.n_sweep)

    def with_(self, **kw) -> "Job":
        return replace(self, **kw)


@dataclass
class Workload:
    name: str
    jobs: list = field(default_factory=list)

    @property
    def updates(self) -> int:
        return sum(j.updates for j in self.jobs)

    @property
    def trajectories(self) -> int:
        return sum(j.n_traj for j in self.jobs)


def config1() -> Workload:
    """2D L = L_t = 16, beta_c, l = 4 -> 5, N = 200, 1 sweep/step, 1000 trajectories."""
    return Workload("2d_L16_l4_N200_traj1000",
                    [Job(2, 16, 16, BETA_C_2D, 4, 200, 1, 1000, seed=0)])


def config2(n_traj: int = 16384) -> Workload:
    """2D L = L_t = 64 at beta_c, full scan l = 0..30 (31 transformations),
    N = 1000, 2 sweeps/step, 16384 trajectories per l."""
    return Workload(f"2d_L64_scan_l0-30_N1000_x2_traj{n_traj}",
                    [Job(2, 64, 64, BETA_C_2D, l, 1000, 2, n_traj, seed=0) for l in range(31)])


def config2_sw(n_traj: int = 16384) -> Workload:
    """The 2D L = 64 scan of config2 with Swendsen-Wang cluster sweeps (the
    update of the paper's own simulations, section 3) in place of Metropolis."""
    return Workload(f"2d_L64_scan_l0-30_N1000_x2_traj{n_traj}_sw",
                    [j.with_(update=1) for j in config2(n_traj).jobs])


def config3(n_traj: int = 4096) -> Workload:
    """3D 16^2 x L_t = 16 at beta = 0.22165455, slab l = 1..8, N = 2000, 1 sweep/step,
    4096 trajectories per l."""
    return Workload(f"3d_L16_slab_l1-8_N2000_traj{n_traj}",
                    [Job(3, 16, 16, BETA_3D_CONFIG, l, 2000, 1, n_traj, seed=0)
                     for l in range(1, 9)])


def config4(seed: int = 0) -> Workload:
    """Uneven batch: 2D L in {32,48,64,96,128}, 3D L in {8,12,16,24}, L_t = L,
    critical beta, every l in [1, L/2]; per item n_traj in {1024..8192} and
    N in {500..4000} drawn log-uniformly (powers of two grid) from
    numpy.random.default_rng(seed); 1 sweep per step.  All jobs use Philox
    seed 0 (one persistent launch shares one key; the counter's l, direction
    and trajectory words keep the streams of different jobs apart)."""
    rng = np.random.default_rng(seed)
    jobs = []
    shapes = [(2, L) for L in (32, 48, 64, 96, 128)] + [(3, L) for L in (8, 12, 16, 24)]
    for i, (d, L) in enumerate(shapes):
        beta = BETA_C_2D if d == 2 else BETA_C_3D
        for l in range(1, L // 2 + 1):
            n_traj = int(2 ** rng.integers(10, 14))          # 1024 .. 8192
            n_step = int(500 * 2 ** rng.integers(0, 4))       # 500 .. 4000
            # distinct trajectory ranges per shape keep the shapes' streams apart
            jobs.append(Job(d, L, L, beta, l, n_step, 1, n_traj, seed=0, traj0=i << 24))
    return Workload("uneven_batch_2d_3d", jobs)


def config5(n_jobs: int = 200, rate: float = 50.0, seed: int = 0):
    """Served stream: Poisson arrivals (mean `rate`/s) of jobs with d in {2,3},
    even L uniform in [32,256] (2D) or [8,48] (3D), L_t = L, beta in
    {0.9,1.0,1.1} x beta_c, l uniform in [1, L/2], n_traj a power of two in
    [256, 8192], N = 1000, 1 sweep/step.  Returns [(arrival_time_s, Job)]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_jobs):
        t += float(rng.exponential(1.0 / rate))
        d = int(rng.integers(2, 4))
        if d == 2:
            L = int(2 * rng.integers(16, 129))
            bc = BETA_C_2D
        else:
            L = int(2 * rng.integers(4, 25))
            bc = BETA_C_3D
        beta = float(bc * (0.9, 1.0, 1.1)[int(rng.integers(0, 3))])
        l = int(rng.integers(1, L // 2 + 1))
        n_traj = int(2 ** rng.integers(8, 14))
        out.append((t, Job(d, L, L, beta, l, 1000, 1, n_traj, seed=10_000 + i)))
    return out


CONFIGS = {1: config1, 2: config2, 3: config3, 4: config4}

#!/usr/bin/env python3
"""Benchmark of the Jarzynski replica-gluing path on one or more GB300s.

A step is one pass of the whole method over one batch: the 2D critical Ising
c-function scan (L = L_t = 64, transformations l -> l+1 for l = 0..30, N = 1000
steps of 2 sweeps, 1000 thermalisation sweeps, 16384 trajectories per l) run as
one device launch, then the FP64 estimator per l on the device and the
c-function on the host.  With --config 1 or 3 the step is the 2D L = 16 single
transformation or the 3D slab scan instead.

Output: one JSON line on rank 0.  value = spin updates per second over all
ranks (every site visit of thermalisation and protocol), device-timed with CUDA
events; e2e = the same through the C ABI with host buffers.  --impl reference
times the CPU oracle (the plain C program) on the host cores instead.

Multi-GPU (torchrun): each rank runs its own trajectory range of every l
(weak scaling); the per-l work arrays are all-gathered before the estimator.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2304_03311_gb300 import workloads as wl  # noqa: E402

METRIC = "spin-updates/s and Jarzynski trajectories/s per GB300 at fixed c-function error"
UNIT = "spin-updates/s"
# Algorithmic integer operations per spin update (Philox4x32-10 share, local
# field and acceptance), fixed a priori for the roofline.
N_ALG = {2: 32, 3: 36}
# Swendsen-Wang: algorithmic integer operations per site and sweep of the bond
# phase alone (one Philox4x32-10 block of about 100 operations, four threshold
# compares); the data-dependent union-find and root flip draws are not counted,
# so this fraction is a lower bound.
N_ALG_SW = {2: 104, 3: 104}
# Integer lanes per SM per clock (64 ALU + 64 FMA-pipe integer lanes); the SM
# count and clock are read from the live device.
INT_LANES_PER_SM = 128
SM_MAX_MHZ_FALLBACK = 2070.0
L2_FLUSH_BYTES = 512 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, choices=[1, 2, 3, 4, 5], default=2)
    ap.add_argument("--serve-jobs", type=int, default=200, help="served stream: jobs")
    ap.add_argument("--rate", type=float, default=50.0, help="served stream: arrivals per second")
    ap.add_argument("--inflight", type=int, default=16, help="served stream: stream slots")
    ap.add_argument("--serve-budget-mb", type=int, default=4096,
                    help="served stream: admission budget (MiB)")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--traj-per-l", type=int, default=None,
                    help="override the trajectories per transformation (small profiling cases)")
    ap.add_argument("--n-step", type=int, default=None,
                    help="override the protocol steps N (small profiling cases)")
    ap.add_argument("--threads", type=int, default=0,
                    help="fix the trajectory kernel's CTA size (0 = library default)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the (untimed) CTA-size autotuning per lattice shape")
    ap.add_argument("--probe", action="store_true",
                    help="print the integer-issue probe rates as JSON and exit")
    ap.add_argument("--update", choices=["metropolis", "sw"], default="metropolis",
                    help="Monte Carlo update of every sweep: checkerboard Metropolis or "
                         "Swendsen-Wang clusters")
    ap.add_argument("--protocol", type=int, choices=[1, 2], default=1,
                    help="1: every switched column together; 2: one column at a time (3D)")
    ap.add_argument("--n-replica", type=int, default=2, help="replicas n (Renyi index)")
    ap.add_argument("--lattice", type=str, default=None,
                    help="L,L_t override for every job of the config (l values kept below L)")
    ap.add_argument("--whole", action="store_true",
                    help="whole-cut transformations (cut lengths l+1) instead of moving the "
                         "end of region A by one column")
    ap.add_argument("--n-therm", type=int, default=None,
                    help="override the thermalisation sweeps")
    ap.add_argument("--therm-update", type=int, choices=[0, 1], default=0,
                    help="1: thermalise with Swendsen-Wang clusters before the Metropolis "
                         "protocol (jz_params.therm_update)")
    ap.add_argument("--therm-study", action="store_true",
                    help="run the scan with Metropolis (n_therm 1000, 4000, 16000) and "
                         "Swendsen-Wang (n_therm 100, 1000) and print the c-function pulls "
                         "against Swendsen-Wang at n_therm 1000 (thermalisation bias)")
    ap.add_argument("--fit-2d", type=int, default=0, metavar="L",
                    help="section 4's study: the 2D critical scan at this L with L_t = 8L, "
                         "fitted with cos(pi x)/16 + k cot(pi x)/(2L); prints k and chi^2")
    ap.add_argument("--small-x-3d", type=int, default=0, metavar="L",
                    help="section 5's study: 2 C_2 at small x of the 3D critical model at this "
                         "L with L_t = 4L (l = 1..4 for L = 24, 2..5 for L = 48)")
    ap.add_argument("--no-compare", action="store_true",
                    help="sw: skip the equal-error comparison with Metropolis")
    ap.add_argument("--plain", type=int, default=8,
                    help="also time the plain one-lattice-per-launch baseline on this many "
                         "trajectories of the middle l (0: skip)")
    ap.add_argument("--bias-traj", type=int, default=512,
                    help="trajectories per l of the Swendsen-Wang reference scan of the "
                         "thermalisation-bias check (0: skip)")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline workload only (no configs 1 and 3, plain baseline or bias "
                         "check beside the default config-2 run)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def workload_for(config: int, rank: int, traj_per_l=None, n_step=None, update="metropolis",
                 protocol=1, n_therm=None, n_replica=2, whole=False, lattice=None,
                 therm_update=0):
    w = wl.CONFIGS[config]()
    if lattice:
        L, L_t = (int(v) for v in lattice.split(","))
        w.jobs = [j.with_(L=L, L_t=L_t) for j in w.jobs if j.l < L]
        w.name += f"_L{L}_T{L_t}"
    if n_replica != 2:
        w.jobs = [j.with_(n_replica=n_replica) for j in w.jobs]
        w.name += f"_n{n_replica}"
    if whole:
        w.jobs = [j.with_(whole=True, l=j.l + 1) for j in w.jobs]
        w.name += "_wholecut"
    if update == "sw":
        w.jobs = [j.with_(update=1) for j in w.jobs]
        w.name += "_sw"
    if protocol == 2:
        w.jobs = [j.with_(protocol=2) for j in w.jobs]
        w.name += "_protocol2"
    if n_therm is not None:
        w.jobs = [j.with_(n_therm=n_therm) for j in w.jobs]
        w.name += f"_therm{n_therm}"
    if therm_update and update != "sw":
        w.jobs = [j.with_(therm_update=1) for j in w.jobs]
        w.name += "_swtherm"
    if traj_per_l:
        w.jobs = [j.with_(n_traj=traj_per_l) for j in w.jobs]
        w.name += f"_traj{traj_per_l}"
    if n_step:
        w.jobs = [j.with_(n_step=n_step) for j in w.jobs]
        w.name += f"_N{n_step}"
    # weak scaling: rank r owns trajectories [r n, (r+1) n) of every job
    w.jobs = [j.with_(traj0=j.traj0 + rank * j.n_traj) for j in w.jobs]
    return w


def run_probe():
    import torch
    from paper_2304_03311_gb300 import build as jzbuild
    jzbuild.build()
    import paper_2304_03311_gb300 as jz
    dev = torch.cuda.current_device()
    sampler = ClockSampler(dev)
    sampler.start()
    names = ["lop3_chain", "imad_chain", "imad_lop3_iadd3_mix", "philox_blocks"]
    rates = {n: jz.ising_probe(dev, k) for k, n in enumerate(names)}
    clocks = sampler.stop()
    rates["philox_update_ceiling"] = 4 * rates["philox_blocks"]
    print(json.dumps({"probe": rates, "units": "thread-instr/s (chains), blocks/s (philox), "
                      "updates/s (ceiling)", "clocks": clocks}), flush=True)


def config_block(w, config, world):
    j0 = w.jobs[0]
    ls = [j.l for j in w.jobs]
    if len({(j.d, j.L, j.L_t) for j in w.jobs}) > 1:
        shapes = sorted({(j.d, j.L, j.L_t) for j in w.jobs})
        return {"workload": w.name, "jobs": len(w.jobs),
                "shapes": [f"{d}D L={L} L_t={Lt}" for d, L, Lt in shapes],
                "trajectories": w.trajectories * world, "spin_updates": w.updates * world,
                "n_step": f"{min(j.n_step for j in w.jobs)}-{max(j.n_step for j in w.jobs)}",
                "n_therm": j0.n_therm, "replicas": 2, "launch": "one persistent CUDA-graph launch",
                "l2": "flushed between steps (512 MiB write)",
                "parallelism": f"trajectory shards x{world}" if world > 1 else "single GPU",
                "source_config": config}
    return {"workload": w.name, "d": j0.d, "L": j0.L, "L_t": j0.L_t, "beta": j0.beta,
            "l": f"{min(ls)}-{max(ls)}" if len(ls) > 1 else ls[0],
            "n_step": j0.n_step, "n_sweep": j0.n_sweep, "n_therm": j0.n_therm,
            "n_traj_per_l": j0.n_traj * world, "replicas": 2,
            "l2": "flushed between steps (512 MiB write)",
            "parallelism": f"trajectory shards x{world}" if world > 1 else "single GPU",
            "source_config": config}


# ----------------------------------------------------------------- clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle ----
def cpu_oracle_rate(w, seconds: float):
    """Times the oracle (as it stands) on the host cores on a bounded sample of
    the workload: trajectories of up to 4 evenly spaced jobs, all cores."""
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    jobs = w.jobs[:: max(1, len(w.jobs) // 4)][:4]
    # one round (one trajectory per thread) to size the sample
    j = jobs[0]
    t0 = time.perf_counter()
    oracle.run(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, threads, j.seed,
               n_therm=j.n_therm, traj0=j.traj0, n_threads=threads, update=j.update,
               therm_update=j.therm_update,
               protocol=j.protocol, n_replica=j.n_replica, whole=j.whole)
    t_round = time.perf_counter() - t0
    rounds = max(1, int(seconds / max(t_round, 1e-3) / len(jobs)))
    n_per_job = rounds * threads
    t0 = time.perf_counter()
    updates = 0
    for j in jobs:
        oracle.run(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, n_per_job, j.seed,
                   n_therm=j.n_therm, traj0=j.traj0, n_threads=threads, update=j.update,
                   therm_update=j.therm_update,
                   protocol=j.protocol, n_replica=j.n_replica, whole=j.whole)
        updates += j.with_(n_traj=n_per_job).updates
    dt = time.perf_counter() - t0
    sample = (f"{n_per_job} trajectories at each of l = {[j.l for j in jobs]} of the same "
              f"workload ({updates:.3e} spin updates, {dt:.1f} s)")
    # one core: one trajectory of the first sampled job on one thread
    j = jobs[0]
    t1 = time.perf_counter()
    oracle.run(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, 1, j.seed,
               n_therm=j.n_therm, traj0=j.traj0, n_threads=1, update=j.update,
               therm_update=j.therm_update,
               protocol=j.protocol, n_replica=j.n_replica, whole=j.whole)
    single = j.with_(n_traj=1).updates / (time.perf_counter() - t1)
    return updates / dt, len(jobs) * n_per_job / dt, threads, sample, single


# Sources of each timed kernel: a recorded DRAM traffic figure stands only
# while these files are unchanged.
KERNEL_SOURCES = {
    "traj_kernel": ("jz_kernels.cu", "jz_traj.cuh", "jz_device.cuh"),
    "persistent_kernel": ("jz_batch.cu", "jz_traj.cuh", "jz_device.cuh"),
    "sw_kernel": ("jz_sw.cu", "jz_device.cuh"),
}


def algorithmic_ops(jobs, sw: bool):
    """Integer operations one launch of these jobs is charged for: each job's
    spin updates at its own dimension's per-update cost.  Returns the total and
    the per-update figure (one number, or one per dimension for mixed jobs)."""
    table = N_ALG_SW if sw else N_ALG
    total = sum(table[j.d] * j.updates for j in jobs)
    dims = sorted({j.d for j in jobs})
    per = table[dims[0]] if len(dims) == 1 else {f"{dd}D": table[dd] for dd in dims}
    return total, per


def kernel_source_hash(kernel: str) -> str:
    """sha256 over the sources of one kernel, in the order listed."""
    csrc = os.path.join(ROOT, "paper_2304_03311_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()


def traffic_from_profile(kernel: str, workload: str):
    """DRAM bytes (read + write) of one launch of this workload's dominant
    kernel, from the ncu capture recorded in profiles/dram_traffic.json; None
    when there is none or the kernel's sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        rec = (json.load(open(path)).get("launches", {}).get(workload)) or {}
    except (OSError, ValueError, AttributeError):
        return None
    if rec.get("source_sha256") != kernel_source_hash(kernel):
        return None
    return rec.get("dram_bytes_per_launch")


def c_function_errors(w, results):
    """(C_n, error) per job: C_n from Delta S_n = Delta S / (n-1) for the
    one-column moves; for whole-cut jobs S_n(l) itself."""
    import math as m
    out = []
    for j, (ds, err) in zip(w.jobs, results):
        ds, err = ds / (j.n_replica - 1), err / (j.n_replica - 1)
        if j.whole:
            out.append((ds, err))
            continue
        x = (j.l + 0.5) / j.L
        fac = (j.L / m.pi * m.sin(m.pi * x)) ** (j.d - 1) / (2.0 * j.L ** (j.d - 2))
        out.append((fac * ds, fac * err))
    return out


# ------------------------------------------------------------ our arm -------
def device_facts(torch, local_rank):
    """SM count from the device properties and the maximum SM clock from
    nvidia-smi (the derived integer-issue ceiling uses both)."""
    props = torch.cuda.get_device_properties(local_rank)
    mhz = None
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits", "-i", str(local_rank)],
                             capture_output=True, text=True, timeout=20).stdout
        mhz = float(out.strip().splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        mhz = None
    return {"name": props.name, "sm_count": props.multi_processor_count,
            "sm_max_mhz": mhz if mhz else SM_MAX_MHZ_FALLBACK,
            "sm_max_mhz_source": "nvidia-smi clocks.max.sm" if mhz else "fallback 2070 MHz"}


def ceilings(jz, dev_index, facts):
    """The three ceilings of the trajectory kernel's roofline, from the live
    device: derived issue ceiling (SMs x 128 integer lanes x max clock, int-op/s),
    the measured mixed IMAD/LOP3/IADD3 issue rate (thread-instr/s) and the
    measured Philox4x32-10-only update rate (4 updates per block)."""
    derived = facts["sm_count"] * INT_LANES_PER_SM * facts["sm_max_mhz"] * 1e6
    mix = jz.ising_probe(dev_index, 2)
    philox = jz.ising_probe(dev_index, 3)
    return {"derived_int_ops_per_s": derived, "probe_mix_int_ops_per_s": mix,
            "philox_update_ceiling_per_s": 4.0 * philox,
            "derived_basis": f"{facts['sm_count']} SMs x {INT_LANES_PER_SM} int lanes/clk x "
                             f"{facts['sm_max_mhz']:.0f} MHz ({facts['sm_max_mhz_source']})"}


def fractions(ops_per_s, updates_per_s, ceil):
    return {"frac_derived": ops_per_s / ceil["derived_int_ops_per_s"],
            "frac_probe": ops_per_s / ceil["probe_mix_int_ops_per_s"],
            "frac_philox_ceiling": updates_per_s / ceil["philox_update_ceiling_per_s"]}


def job_params(jz, j, **over):
    kw = dict(n_therm=j.n_therm, direction=j.direction, traj0=j.traj0, update=j.update,
              protocol=j.protocol, n_replica=j.n_replica, whole=j.whole,
              therm_update=j.therm_update)
    kw.update(over)
    return jz.make_params(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj, j.seed,
                          **kw)


def exchange_work(arrays, jobs, world, group):
    """The one exchange step of the method: every job's W_int shards gathered
    in global trajectory order on every rank (shard.gather_work, which reports a
    missing or mis-sized shard instead of waiting on it)."""
    from paper_2304_03311_gb300 import shard
    return [shard.gather_work(a.cpu().numpy() if hasattr(a, "cpu") else a,
                              j.n_traj * world, group=group)
            for a, j in zip(arrays, jobs)]


class Scan:
    """One workload on the device: its parameters, output buffers, tuned CTA
    sizes, and a step = the trajectory launch(es) + the FP64 estimator per job
    (+ the c-function on the host)."""

    def __init__(self, jz, torch, ctx, stream, dev, w, world=1, host_group=None, threads=0,
                 autotune=True, use_plan=False):
        self.jz, self.torch, self.ctx, self.stream, self.w = jz, torch, ctx, stream, w
        self.world, self.group = world, host_group
        self.sw = all(j.update == 1 for j in w.jobs)
        self.outs = [torch.empty(j.n_traj, dtype=torch.int64, device=dev) for j in w.jobs]
        self.params = [job_params(jz, j) for j in w.jobs]
        self.n_groups = len({(j.d, j.L, j.L_t, j.seed, j.update, j.n_replica, j.therm_update)
                             for j in w.jobs})
        # a launch group starting from Swendsen-Wang thermalisation adds its
        # thermalisation launch (one while the state fits shared memory; a
        # state beyond it adds one per wave of resident trajectories)
        self.n_therm_launches = len({(j.d, j.L, j.L_t, j.seed, j.n_replica) for j in w.jobs
                                     if j.therm_update and j.update == 0 and j.n_therm > 0})
        self.tuned = {}
        self.plan = None
        self.est = None
        if use_plan:
            self.est = torch.zeros(3 * len(w.jobs), dtype=torch.float64, device=dev)
            self.plan = jz.jz_plan_create(ctx, self.params, self.outs, self.est, threads)
            cta, grid, n_items = jz.jz_plan_info(self.plan)
            self.tuned = {"persistent_cta": cta, "grid": grid, "work_items": n_items}
            self.n_groups = 1
        else:
            for shape, j in {(j.d, j.L, j.L_t): j for j in w.jobs}.items():
                if threads:
                    jz.ising_set_threads(ctx, *shape, threads)
                    self.tuned[str(shape)] = threads
                elif autotune and j.update == 0:
                    try:
                        p = self.params[w.jobs.index(j)]
                        self.tuned[str(shape)] = jz.ising_autotune(ctx, p)
                    except jz.IsingError:   # lattices beyond shared memory are not tuned
                        self.tuned[str(shape)] = "default (lattice in HBM)"

    def launches_per_step(self):
        if self.plan is not None:
            return 2
        return self.n_groups + self.n_therm_launches + len(self.w.jobs)

    def estimate(self, buffers):
        res = []
        for j, b in zip(self.w.jobs, buffers):
            _, ds, err = self.jz.estimator_reduce(self.ctx, b, j.n_traj * self.world, j.beta,
                                                  j.n_step, j.direction, 32)
            res.append((ds, err))
        return res

    def step(self):
        """One step; returns ((start event, end event, library launch ms), c-function)."""
        torch, jz = self.torch, self.jz
        k0 = torch.cuda.Event(enable_timing=True)
        k1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(self.stream):
            k0.record(self.stream)
            if self.plan is not None:
                jz.jz_plan_launch(self.plan)
            else:
                jz.jarzynski_run_batch(self.ctx, self.params, self.outs)
            k1.record(self.stream)
            if self.plan is not None and self.world == 1:
                e = self.est.cpu().numpy().reshape(-1, 3)
                return (k0, k1, None), c_function_errors(self.w, [(r[1], r[2]) for r in e])
            bufs = self.outs
            if self.world > 1:
                bufs = exchange_work(self.outs, self.w.jobs, self.world, self.group)
            res = self.estimate(bufs)
        # the trajectory launches alone (library events on the same stream, the
        # call's table and result copies excluded); the plan's graph has none
        launch_ms = jz.ising_last_launch_ms(self.ctx) if self.plan is None else None
        return (k0, k1, launch_ms), c_function_errors(self.w, res)

    def free(self):
        if self.plan is not None:
            self.jz.jz_plan_free(self.plan)


def timed(torch, dist, scan, steps, warmup, flush, world, local_rank):
    """W untimed steps, then K steps bracketed by barrier + synchronize, L2
    flushed between steps; device time from CUDA events on the launching
    stream, max over ranks."""
    stream = scan.stream

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.fill_(1)

    for _ in range(warmup):
        scan.step()
        flush_l2()
    stream.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    pairs = []
    t_start.record(stream)
    cfun = None
    for i in range(steps):
        pair, cfun = scan.step()
        pairs.append(pair)
        if i + 1 < steps:
            flush_l2()
    t_end.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    kernel_ms = statistics.mean(ms if ms is not None else a.elapsed_time(b) for a, b, ms in pairs)
    if world > 1:
        t = torch.tensor([elapsed_ms, kernel_ms], dtype=torch.float64,
                         device=torch.device("cuda", local_rank))
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms, kernel_ms = float(t[0]), float(t[1])
    ms_per_step = elapsed_ms / steps
    return {"ms_per_step": ms_per_step, "kernel_ms": kernel_ms, "cfun": cfun, "clocks": clocks,
            "steps": steps, "warmup": warmup}


def workload_record(w, t, ceil, world=1, sw=False):
    """Rates and roofline fractions of one timed workload."""
    updates = w.updates * world
    ops, n_alg = algorithmic_ops(w.jobs, sw)
    k_s = t["kernel_ms"] / 1e3
    rec = {"workload": w.name, "ms_per_step": t["ms_per_step"], "kernel_ms": t["kernel_ms"],
           "spin_updates_per_s": updates / (t["ms_per_step"] / 1e3),
           "trajectories_per_s": w.trajectories * world / (t["ms_per_step"] / 1e3),
           "kernel_spin_updates_per_s": w.updates / k_s, "ops_per_update": n_alg,
           "steps": t["steps"], "warmup": t["warmup"], "clocks": t["clocks"],
           "c_function_err_max": max(e for _, e in t["cfun"]) if t["cfun"] else None}
    if ceil and not sw:
        rec.update(fractions(ops / k_s, w.updates / k_s, ceil))
    return rec


def pulls(test, ref):
    """Per-l pulls of two c-function scans (value, error) and their summary."""
    p = [(a - b) / math.hypot(ea, eb) for (a, ea), (b, eb) in zip(test, ref)]
    chi2 = sum(x * x for x in p) / len(p)
    return {"max_abs_pull": max(abs(x) for x in p), "mean_pull": sum(p) / len(p),
            "chi2_per_l": chi2,
            # 31 independent unit normals: chi2/l below 1.8 and no pull beyond 3.6
            # fail by chance in well under 1 % of scans
            "passes": chi2 < 1.8 and max(abs(x) for x in p) < 3.6}


def bias_and_cost(jz, torch, ctx, stream, dev, headline_w, headline_cfun, headline_ms, args):
    """Thermalisation bias of the 2D L = 64 scan and the cost of a c-function
    at fixed error for both updates, and for Metropolis protocols started by
    Swendsen-Wang thermalisation.  A Jarzynski estimate is unbiased only from
    an equilibrium start (Appendix A), so each scan's per-l c-function is pulled
    against a Swendsen-Wang reference with 1000 cluster sweeps of
    thermalisation (the paper's set-up, section 4) on independent
    trajectories; each choice's cost is the time to reach the headline's rms
    c-function error at the smallest tested n_therm whose pulls pass."""
    nref = args.bias_traj
    base = headline_w.jobs

    def run(tag, update, n_therm, n_traj, traj0, therm_update=0):
        jobs = [j.with_(update=update, n_therm=n_therm, n_traj=n_traj, traj0=traj0,
                        therm_update=therm_update) for j in base]
        w = wl.Workload(f"{headline_w.name}_{tag}", jobs)
        outs = [torch.empty(n_traj, dtype=torch.int64, device=dev) for _ in jobs]
        ps = [job_params(jz, j) for j in jobs]
        with torch.cuda.stream(stream):
            jz.jarzynski_run_batch(ctx, ps, outs)
        ms = jz.ising_last_launch_ms(ctx)
        res = []
        for j, o in zip(jobs, outs):
            _, ds, err = jz.estimator_reduce(ctx, o, n_traj, j.beta, j.n_step, j.direction, 32)
            res.append((ds, err))
        return {"cfun": c_function_errors(w, res), "kernel_ms": ms, "n_traj_per_l": n_traj,
                "n_therm": n_therm}

    rms = lambda v: math.sqrt(sum(e * e for _, e in v) / len(v))
    # independent trajectory ranges: the headline uses 0 .. n_traj-1
    ref = run("sw_ref", 1, 1000, nref, 1 << 28)
    head = {"cfun": headline_cfun, "kernel_ms": headline_ms, "n_traj_per_l": base[0].n_traj,
            "n_therm": base[0].n_therm}
    cands = {"metropolis": [head, run("m4000", 0, 4000, 2 * nref, 2 << 28)],
             "sw": [run("sw100", 1, 100, nref, 3 << 28)],
             "sw_therm_metropolis": [run("h100", 0, 100, 2 * nref, 4 << 28, therm_update=1)]}
    target = rms(headline_cfun)
    out = {"reference": f"Swendsen-Wang, n_therm = 1000, {nref} trajectories per l "
                        f"(independent of the headline's)",
           "headline": dict(pulls(headline_cfun, ref["cfun"]), n_therm=base[0].n_therm),
           "target_c_err_rms": target}
    cost = {}
    for upd, runs in cands.items():
        tested = []
        chosen = None
        for r in runs:
            pl = pulls(r["cfun"], ref["cfun"])
            tested.append({"n_therm": r["n_therm"], **pl})
            if chosen is None and pl["passes"]:
                chosen = r
        entry = {"tested": tested}
        if chosen is not None:
            e = rms(chosen["cfun"])
            t_s = chosen["kernel_ms"] / 1e3
            n_per_l = chosen["n_traj_per_l"]
            need = n_per_l * (e / target) ** 2          # trajectories per l at the target error
            seconds = t_s * (e / target) ** 2
            entry.update({"n_therm": chosen["n_therm"], "run_kernel_s": t_s,
                          "n_traj_per_l": n_per_l, "c_err_rms": e,
                          "trajectories_per_s": n_per_l * len(base) / t_s,
                          "trajectories_per_l_at_target": need,
                          "seconds_at_target": seconds})
        cost[upd] = entry
    if "seconds_at_target" in cost["sw"] and "seconds_at_target" in cost["metropolis"]:
        cost["sw_over_metropolis_time_at_target"] = (cost["sw"]["seconds_at_target"] /
                                                     cost["metropolis"]["seconds_at_target"])
    if ("seconds_at_target" in cost["sw_therm_metropolis"] and
            "seconds_at_target" in cost["metropolis"]):
        cost["sw_therm_over_metropolis_time_at_target"] = (
            cost["sw_therm_metropolis"]["seconds_at_target"] /
            cost["metropolis"]["seconds_at_target"])
    out["cost_at_fixed_error"] = cost
    return out


def plain_baseline(jz, torch, ctx, dev, w, value, n):
    """K0: the plain one-lattice-per-launch form on n trajectories of the
    middle transformation, and the fused kernel on the same trajectories
    (identical bits, hence equal statistical error)."""
    j = w.jobs[len(w.jobs) // 2].with_(n_traj=n)
    pw = torch.empty(j.n_traj, dtype=torch.int64, device=dev)
    pp = job_params(jz, j)
    jz.ising_sync(ctx)
    t0 = time.perf_counter()
    jz.jarzynski_run_plain(ctx, pp, pw)
    jz.ising_sync(ctx)
    dt = time.perf_counter() - t0
    fw = torch.empty_like(pw)
    jz.jarzynski_run_ex(ctx, pp, fw)
    jz.ising_sync(ctx)
    return {"value": j.updates / dt, "unit": UNIT,
            "sample": f"{j.n_traj} trajectories of l = {j.l}",
            "seconds": dt, "bit_identical_to_fused": bool(torch.equal(pw, fw)),
            "speedup_of_fused": value / (j.updates / dt)}


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local_rank = dist_env()
    host_group = None
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
        # the W_int exchange is a host-side gather (8 bytes per trajectory)
        host_group = dist.new_group(backend="gloo")
    torch.cuda.set_device(local_rank)
    from paper_2304_03311_gb300 import build as jzbuild
    if rank == 0 or world == 1:
        jzbuild.build()
    if world > 1:
        dist.barrier()
    import paper_2304_03311_gb300 as jz

    w = workload_for(args.config, rank, args.traj_per_l, args.n_step, args.update, args.protocol,
                     args.n_therm, args.n_replica, args.whole, args.lattice,
                     args.therm_update)
    sw = args.update == "sw"
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    ctx = jz.ising_replica_init(local_rank, 0, stream.cuda_stream)
    if sw and args.config == 4:
        raise SystemExit("--update sw runs configs 1-3 (the persistent plan is Metropolis only)")
    facts = device_facts(torch, local_rank)
    ceil = ceilings(jz, local_rank, facts)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    scan = Scan(jz, torch, ctx, stream, dev, w, world, host_group, args.threads,
                not args.no_autotune, use_plan=args.config == 4)
    t = timed(torch, dist, scan, args.steps, args.warmup, flush, world, local_rank)
    cfun, kernel_ms, ms_per_step, clocks = t["cfun"], t["kernel_ms"], t["ms_per_step"], t["clocks"]
    updates_step = w.updates * world
    value = updates_step / (ms_per_step / 1e3)
    traj_rate = w.trajectories * world / (ms_per_step / 1e3)

    # end to end through the C ABI with host buffers: work arrays copied back
    # each step, the estimator fed from host memory
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else max(1, args.steps // 2)
    host_outs = [torch.empty(j.n_traj, dtype=torch.int64, pin_memory=True) for j in w.jobs]
    stream.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        with torch.cuda.stream(stream):
            jz.jarzynski_run_batch(ctx, scan.params, host_outs)
            gathered = (exchange_work(host_outs, w.jobs, world, host_group) if world > 1
                        else host_outs)
            scan.estimate(gathered)
    stream.synchronize()
    e2e_s = time.perf_counter() - t0
    if world > 1:
        tt = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_s = float(tt[0])
    table_bytes = sum(j.n_step * (2 if sw else 8 * j.d) * 4 + 96 for j in w.jobs)
    h2d = table_bytes + sum(8 * j.n_traj * world for j in w.jobs)
    d2h = sum(8 * j.n_traj for j in w.jobs) + 24 * len(w.jobs)
    e2e = {"value": updates_step / (e2e_s / e2e_steps) if e2e_steps else None, "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": e2e_steps}

    d = w.jobs[0].d
    ops_per_launch, n_alg = algorithmic_ops(w.jobs, sw)   # one launch per rank per step
    achieved = ops_per_launch / (kernel_ms / 1e3) / 1e12
    peak = ceil["derived_int_ops_per_s"] / 1e12
    kbase = "sw_kernel" if sw else "persistent_kernel" if scan.plan is not None else "traj_kernel"
    kname = (f"sw_kernel<{d}>" if sw else
             "persistent_kernel" if scan.plan is not None else f"traj_kernel<{d},...>")
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved,
                "peak": peak, "unit": "Tintop/s", "frac": achieved / peak,
                "traffic": traffic_from_profile(kbase, w.name),
                "ops_per_update": n_alg, "kernel_ms": kernel_ms,
                "peak_basis": ceil["derived_basis"] + " (derived)"}
    if not sw:
        fr = fractions(ops_per_launch / (kernel_ms / 1e3), w.updates / (kernel_ms / 1e3), ceil)
        roofline.update({"frac_probe": fr["frac_probe"],
                         "frac_philox_ceiling": fr["frac_philox_ceiling"],
                         "probe_peak": ceil["probe_mix_int_ops_per_s"] / 1e12,
                         "philox_update_ceiling": ceil["philox_update_ceiling_per_s"]})

    equal_error = None
    if sw and not args.no_compare:
        # the same workload with Metropolis sweeps: time per step and the
        # c-function error it reaches; at equal error the cost scales as err^2 t
        mw = wl.Workload(w.name + "_metropolis", [j.with_(update=0) for j in w.jobs])
        mscan = Scan(jz, torch, ctx, stream, dev, mw, world, host_group, args.threads,
                     not args.no_autotune)
        mt = timed(torch, dist, mscan, 1, 1, flush, world, local_rank)
        m_ms, mfun = mt["kernel_ms"], mt["cfun"]
        rms = lambda v: math.sqrt(sum(x * x for x in v) / len(v))
        m_err = [e for _, e in mfun]
        s_err = [e for _, e in cfun]
        pl = pulls(cfun, mfun)
        equal_error = {
            "metropolis": {"kernel_ms": m_ms, "c_err_rms": rms(m_err)},
            "sw": {"kernel_ms": kernel_ms, "c_err_rms": rms(s_err)},
            "sw_speedup_at_equal_error": (rms(m_err) ** 2 * m_ms) / (rms(s_err) ** 2 * kernel_ms),
            "c_function_pull_max": pl["max_abs_pull"], "c_function_chi2_per_l": pl["chi2_per_l"],
            "basis": "same trajectories, N, sweeps and n_therm; cost at equal error ~ err^2 x time"}

    # the other benchmark workloads and the plain baseline, beside the
    # headline (one GPU only; the headline alone under torchrun)
    default_run = (args.config == 2 and not sw and args.protocol == 1 and args.n_replica == 2
                   and not args.whole and not args.lattice and not args.traj_per_l
                   and not args.n_step and args.n_therm is None and not args.therm_update)
    extras = world == 1 and not args.no_extras and default_run
    configs = None
    plain = None
    bias = None
    if extras:
        configs = {"2": workload_record(w, t, ceil)}
        for c, (steps, warm) in ((1, (20, 5)), (3, (3, 1))):
            cw = wl.CONFIGS[c]()
            cs = Scan(jz, torch, ctx, stream, dev, cw, 1, None, 0, not args.no_autotune)
            ct = timed(torch, dist, cs, steps, warm, flush, 1, local_rank)
            configs[str(c)] = workload_record(cw, ct, ceil)
            configs[str(c)]["cta_threads"] = cs.tuned
            cs.free()
        if args.plain > 0:
            plain = plain_baseline(jz, torch, ctx, dev, w, value, args.plain)
        if args.bias_traj > 0:
            bias = bias_and_cost(jz, torch, ctx, stream, dev, w, cfun, kernel_ms, args)
    elif args.plain > 0 and all(j.update == 0 and j.therm_update == 0 and j.n_replica == 2 and
                                not j.whole and
                                (j.protocol == 1 or j.d == 2) for j in w.jobs):
        # the plain form serves Metropolis, two replicas and moving ends only
        plain = plain_baseline(jz, torch, ctx, dev, w, value, args.plain)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, trate, cores, sample, single = cpu_oracle_rate(w, args.cpu_seconds / (3 if sw else 1))
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "trajectories_per_s": trate, "single_core_value": single,
               # the whole workload on these cores, extrapolated at the sampled rate
               "full_workload_s_estimate": w.updates / rate if rate > 0 else None}
    scan.free()
    jz.ising_replica_free(ctx)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u32", "data": "synthetic (Philox hot starts; no dataset)",
                "config": config_block(w, args.config, world),
                "trajectories_per_s": traj_rate,
                "c_function_err_max": max(e for _, e in cfun) if cfun else None,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "configs": configs, "plain_gpu_baseline": plain, "bias_check": bias,
                "ceilings": ceil, "device": facts,
                "cta_threads": scan.tuned or "default",
                "update": args.update, "therm_update": args.therm_update,
                "protocol": args.protocol,
                "n_replica": args.n_replica, "whole_cut": args.whole,
                "equal_error_vs_metropolis": equal_error,
                "gpu_launches": args.steps * scan.launches_per_step(),
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------ serving -------
def run_serve(args):
    """Served stream: jobs arrive as a Poisson process and are submitted to the
    continuous-batching server at their arrival times; reports sustained spin
    updates/s over the makespan and p50 / p99 latency (submit -> result)."""
    import torch
    from paper_2304_03311_gb300 import build as jzbuild
    jzbuild.build()
    import paper_2304_03311_gb300 as jz

    arrivals = wl.config5(n_jobs=args.serve_jobs, rate=args.rate)
    if args.n_therm is not None:
        arrivals = [(t, j.with_(n_therm=args.n_therm)) for t, j in arrivals]
    if args.therm_update:
        arrivals = [(t, j.with_(therm_update=1)) for t, j in arrivals]
    ctx = jz.ising_replica_init(0, 0, None)
    server = jz.jz_server_create(ctx, args.serve_budget_mb << 20, args.inflight)
    mk = lambda j: jz.make_params(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj,
                                  j.seed, n_therm=j.n_therm, direction=j.direction,
                                  traj0=j.traj0, therm_update=j.therm_update)
    # warm-up: one small job per dimension through the same server
    for j in (wl.Job(2, 32, 32, wl.BETA_C_2D, 3, 20, 1, 64),
              wl.Job(3, 8, 8, wl.BETA_C_3D, 2, 20, 1, 64)):
        jz.jz_wait(server, jz.jz_submit(server, mk(j)))
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    t0 = time.perf_counter()
    ids = []
    for t_arr, j in arrivals:
        delay = t0 + t_arr - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        ids.append(jz.jz_submit(server, mk(j)))
    results = [jz.jz_wait(server, i, 7200.0) for i in ids]
    clocks = sampler.stop()
    jz.jz_server_free(server)
    jz.ising_replica_free(ctx)
    bad = [r.status for r in results if r.status != 0]
    in_order = [r.done_s - r.submit_s for r in results]   # arrival order
    lat = sorted(in_order)
    makespan = max(r.done_s for r in results) - min(r.submit_s for r in results)
    updates = sum(r.updates for r in results)
    pct = lambda q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]

    waits = [r.start_s - r.submit_s for r in results]    # arrival order
    pct_of = lambda v, q: sorted(v)[min(len(v) - 1, int(round(q * (len(v) - 1))))]

    def halves_p99(v):
        v = sorted(v)
        return v[min(len(v) - 1, int(round(0.99 * (len(v) - 1))))] if v else None
    line = {"metric": METRIC, "value": updates / makespan, "unit": UNIT, "n_gpus": 1,
            "steps": 1, "warmup": 1, "ms_per_step": makespan * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (Philox hot starts; no dataset)",
            "config": {"workload": f"served_stream_poisson{args.rate:g}_jobs{len(ids)}" +
                                   (f"_therm{args.n_therm}" if args.n_therm is not None else "") +
                                   ("_swtherm" if args.therm_update else ""),
                       "inflight_slots": args.inflight, "hbm_budget_mb": args.serve_budget_mb,
                       "source_config": 5},
            "latency_s": {"p50": pct(0.50), "p99": pct(0.99), "max": lat[-1]},
            # a stable rate keeps the late arrivals' latency near the early ones'
            "latency_p99_by_half_s": [halves_p99(in_order[:len(in_order) // 2]),
                                      halves_p99(in_order[len(in_order) // 2:])],
            # time from submission to admission (a free slot and memory); a stable
            # rate keeps it bounded, whatever the sizes of the jobs
            "queue_wait_s": {"p50": pct_of(waits, 0.50), "p99": pct_of(waits, 0.99)},
            "queue_wait_p99_by_half_s": [halves_p99(waits[:len(waits) // 2]),
                                         halves_p99(waits[len(waits) // 2:])],
            "trajectories_per_s": sum(j.n_traj for _, j in arrivals) / makespan,
            "jobs_failed": len(bad), "makespan_s": makespan, "clocks": clocks}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- reference arm -----
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    w = workload_for(args.config, 0, args.traj_per_l, args.n_step, args.update, args.protocol,
                     args.n_therm, args.n_replica, args.whole, args.lattice,
                     args.therm_update)
    jobs = w.jobs[:: max(1, len(w.jobs) // 2)][:2]
    n_per = threads

    def step():
        u = 0
        for j in jobs:
            oracle.run(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, n_per, j.seed,
                       n_therm=j.n_therm, traj0=j.traj0, n_threads=threads, update=j.update,
                       therm_update=j.therm_update,
                       protocol=j.protocol, n_replica=j.n_replica, whole=j.whole)
            u += j.with_(n_traj=n_per).updates
        return u

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    updates = 0
    for _ in range(args.steps):
        updates += step()
    dt = time.perf_counter() - t0
    value = updates / dt
    sample = (f"per step {n_per} trajectories at each of l = {[j.l for j in jobs]} of "
              f"{w.name}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8",
            "data": "synthetic (Philox hot starts; no dataset)",
            "config": config_block(w, args.config, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_therm_study(args):
    """The same scan with both updates, and Swendsen-Wang starts before
    Metropolis protocols, at several thermalisation lengths: the Jarzynski
    estimate is unbiased only from an equilibrium start, so a start that has
    not thermalised shows up as a pull against a reference that has
    (Swendsen-Wang with 1000 cluster sweeps)."""
    import torch
    from paper_2304_03311_gb300 import build as jzbuild
    jzbuild.build()
    import paper_2304_03311_gb300 as jz
    n = args.traj_per_l or 512
    ctx = jz.ising_replica_init(0, 0, None)
    runs = {}
    for name, upd, nth, seed, th in [("metropolis_therm1000", 0, 1000, 0, 0),
                                     ("metropolis_therm1000_seed7", 0, 1000, 7, 0),
                                     ("metropolis_therm4000", 0, 4000, 0, 0),
                                     ("metropolis_therm16000", 0, 16000, 0, 0),
                                     ("sw_therm1000", 1, 1000, 0, 0), ("sw_therm100", 1, 100, 3, 0),
                                     ("sw_therm100_metropolis", 0, 100, 5, 1),
                                     ("sw_therm25_metropolis", 0, 25, 6, 1)]:
        w = wl.CONFIGS[args.config]()
        jobs = [j.with_(n_traj=n, n_therm=nth, seed=seed, update=upd, therm_update=th)
                for j in w.jobs]
        outs = [torch.empty(n, dtype=torch.int64, device="cuda") for _ in jobs]
        ps = [jz.make_params(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj, j.seed,
                             n_therm=j.n_therm, update=upd, therm_update=th) for j in jobs]
        t0 = time.perf_counter()
        jz.jarzynski_run_batch(ctx, ps, outs)
        jz.ising_sync(ctx)
        dt = time.perf_counter() - t0
        res = []
        for j, o in zip(jobs, outs):
            _, ds, err = jz.estimator_reduce(ctx, o, n, j.beta, j.n_step, 1, 32)
            res.append((ds, err))
        runs[name] = (res, dt)
    ref = runs["sw_therm1000"][0]
    table = {}
    for name, (res, dt) in runs.items():
        pulls = [(a - b) / math.hypot(ea, eb) for (a, ea), (b, eb) in zip(res, ref)]
        table[name] = {"seconds": dt, "chi2_per_l": sum(p * p for p in pulls) / len(pulls),
                       "mean_pull": sum(pulls) / len(pulls),
                       "max_abs_pull": max(abs(p) for p in pulls),
                       "dS_err_l0": res[0][1], "dS_err_lmax": res[-1][1]}
    jz.ising_replica_free(ctx)
    print(json.dumps({"therm_study": table, "workload": wl.CONFIGS[args.config]().name,
                      "n_traj_per_l": n, "reference": "sw_therm1000"}), flush=True)


def run_fit_2d(args):
    """Section 4 on the GPU: every l -> l+1 of the critical 2D model at L,
    L_t = 8L, the c-function from Delta S_2, and the paper's fit with and
    without the two points at each end (its table of chi^2 and k)."""
    import numpy as np
    import torch
    from paper_2304_03311_gb300 import build as jzbuild
    from paper_2304_03311_gb300 import analysis as an
    jzbuild.build()
    import paper_2304_03311_gb300 as jz
    L = args.fit_2d
    L_t = 8 * L
    n_traj = args.traj_per_l or 4096
    N = args.n_step or 2000
    upd = 1 if args.update == "sw" else 0
    # Metropolis needs of order L^2.17 sweeps from a hot start at criticality
    n_therm = args.n_therm or (100 if upd else int(4 * L ** 2.17) + 1000)
    jobs = [wl.Job(2, L, L_t, wl.BETA_C_2D, l, N, 1, n_traj, seed=l, n_therm=n_therm, update=upd)
            for l in range(L)]
    ctx = jz.ising_replica_init(0, 0, None)
    outs = [torch.empty(n_traj, dtype=torch.int64, device="cuda") for _ in jobs]
    ps = [jz.make_params(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj, j.seed,
                         n_therm=j.n_therm, update=upd) for j in jobs]
    t0 = time.perf_counter()
    jz.jarzynski_run_batch(ctx, ps, outs)
    jz.ising_sync(ctx)
    dt = time.perf_counter() - t0
    ds, err = [], []
    for j, o in zip(jobs, outs):
        _, d, e = jz.estimator_reduce(ctx, o, n_traj, j.beta, N, 1, 32)
        ds.append(d)
        err.append(e)
    jz.ising_replica_free(ctx)
    l = np.arange(L)
    x = an.midpoint_x(l, L)
    c, ce = an.c_function(np.array(ds), 2, L, l, err=np.array(err))
    out = {"fit_2d": {"L": L, "L_t": L_t, "n_step": N, "n_traj_per_l": n_traj,
                      "n_therm": n_therm, "update": args.update, "seconds": dt}}
    for drop in (0, 2):
        f = an.fit_2d(x, c, ce, L, drop_ends=drop)
        sf = an.chi2_scaling_function_2d(x, c, ce, drop_ends=drop)
        out["fit_2d"][f"drop_{drop}"] = {"k": float(f.params[0]), "k_err": float(f.errors[0]),
                                         "chi2_per_dof": f.chi2_per_dof,
                                         "scaling_function_chi2_per_dof": sf.chi2_per_dof}
    out["fit_2d"]["c_function"] = [[float(a), float(b), float(e)] for a, b, e in zip(x, c, ce)]
    print(json.dumps(out), flush=True)


def run_small_x_3d(args):
    """Section 5's table of 2 C_2 at small x (3D critical model, L_t = 4L),
    with the paper's N for x near 0 by default."""
    import torch
    from paper_2304_03311_gb300 import build as jzbuild
    from paper_2304_03311_gb300 import analysis as an
    jzbuild.build()
    import paper_2304_03311_gb300 as jz
    L = args.small_x_3d
    L_t = 4 * L
    ls = [1, 2, 3, 4] if L <= 24 else [2, 3, 4, 5]
    n_traj = args.traj_per_l or 256
    N = args.n_step or (25000 if L <= 24 else 40000)
    n_therm = args.n_therm or 8000
    jobs = [wl.Job(3, L, L_t, wl.BETA_C_3D, l, N, 1, n_traj, seed=40 + l, n_therm=n_therm)
            for l in ls]
    ctx = jz.ising_replica_init(0, 0, None)
    outs = [torch.empty(n_traj, dtype=torch.int64, device="cuda") for _ in jobs]
    t0 = time.perf_counter()
    jz.jarzynski_run_batch(ctx, [jz.make_params(j.d, j.L, j.L_t, j.beta, j.l, j.n_step,
                                                j.n_sweep, j.n_traj, j.seed, n_therm=j.n_therm)
                                 for j in jobs], outs)
    jz.ising_sync(ctx)
    dt = time.perf_counter() - t0
    rows = []
    for j, o in zip(jobs, outs):
        _, ds, err = jz.estimator_reduce(ctx, o, n_traj, j.beta, N, 1, 32)
        c, ce = an.c_function(ds, 3, L, j.l, err=err)
        rows.append({"x": float(an.midpoint_x(j.l, L)), "two_C2": float(2 * c),
                     "err": float(2 * ce)})
    jz.ising_replica_free(ctx)
    print(json.dumps({"small_x_3d": {"L": L, "L_t": L_t, "n_step": N, "n_traj_per_l": n_traj,
                                     "n_therm": n_therm, "seconds": dt, "rows": rows}}),
          flush=True)


def main():
    args = parse_args()
    if args.probe:
        run_probe()
    elif args.small_x_3d:
        run_small_x_3d(args)
    elif args.fit_2d:
        run_fit_2d(args)
    elif args.therm_study:
        run_therm_study(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.config == 5:
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

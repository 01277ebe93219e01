#!/usr/bin/env python3
"""psFlip benchmark of the GB300 checkerboard Metropolis sweep (arXiv:1411.0127).

Workload: one L = 1024 lattice (2^30 spins), +-J couplings with p = 1/2 from
seed 1, random initial spins and MT19937 streams from seed 2, quench at
T = 0.9.  A step is one sweep (red pass + blue pass, every spin attempted once).
psFlip = picoseconds per spin-flip attempt = step time / 2^30 (lower is better).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  Under torchrun (N > 1) every rank sweeps its
own independent replica (same couplings, spin seed 2 + rank): the path has no
exchange step at one lattice per GPU, so the ranks share nothing but the
barrier and the max-over-ranks timing ("replicas only", weak scaling).
`--impl reference` times the CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ps per spin-flip attempt (psFlip) at L=1024; batched vs plain psFlip"
UNIT = "ps/attempt"

# Roofline definitions: the integer issue rate of the SMs, and the algorithmic
# operations and DRAM bytes of one spin-flip attempt.
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
INT_LANES_PER_SM = 128                         # 4 SMSPs x 32 lanes, one 32-bit op each per clock
ALU_PEAK_TOPS = SM_COUNT * INT_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12   # 40.27 Tops/s
OPS_PER_ATTEMPT = {"mt19937": 17, "minstd": 11}  # algorithmic 32-bit integer ops per attempt
E2E_HANDLES = 4                                # lattices of the pipelined end-to-end exchange
E2E_PIPE_STEPS = 192                           # its timed steps (48 per lattice, about 0.3 s)
BYTES_PER_ATTEMPT = 9 / 8                      # S_c read+write, S_c' once, 6 coupling bits


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=20)
    p.add_argument("--plain-steps", type=int, default=300)
    p.add_argument("--batch-groups", type=int, default=2, help="timed 64-sweep groups of the batched workload (0: skip)")
    p.add_argument("--serve-jobs", type=int, default=16, help="jobs of the serving trace to serve (0: skip)")
    p.add_argument("--serve-sustained-jobs", type=int, default=200,
                   help="jobs of the sustainable-load serving run (0: skip)")
    p.add_argument("--L", type=int, default=0, help="lattice size instead of 1024 (quick runs and tests only)")
    p.add_argument("--other-configs", type=int, default=1, help="also time the L=32/256 and MINSTD lattices (0: skip)")
    p.add_argument("--amsc", type=int, default=1, help="also time the asynchronous multispin ensembles (0: skip)")
    return p.parse_args()


def workload_config(w):
    return {"workload": "single lattice L=%d (%d spins), +-J p=1/2 seed_J=%d, random spins seed_spin=%d, "
                        "%s streams, quench at T=%g" % (w.L, w.L ** 3, w.seed_J, w.seed_spin, w.kind.upper(), w.T),
            "L": w.L, "rng": w.kind, "T": w.T, "seed_J": w.seed_J, "seed_spin": w.seed_spin,
            "attempts_per_step": w.L ** 3,
            "l2": "no flush: inputs (%d MiB of bit planes) exceed the 129 MB L2" % (w.L ** 3 * 4 // 8 // 2**20)}


# ------------------------------------------------------------------ clocks ---
class ClockSampler:
    """nvidia-smi samples (every 50 ms) of SM clock and throttle reasons."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self, t0: float, t1: float) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = []
        for line in self.file.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                frac = float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                rows.append((ts + frac, float(parts[1]), float(parts[2]), parts[5:9], parts[4]))
            except (ValueError, IndexError):
                continue
        os.unlink(self.file.name)
        inside = [r for r in rows if t0 - 0.05 <= r[0] <= t1 + 0.05]
        note = "samples inside the timed region"
        if not inside and rows:  # region shorter than the sampling period: nearest samples
            inside = sorted(rows, key=lambda r: min(abs(r[0] - t0), abs(r[0] - t1)))[:3]
            note = "timed region shorter than the sampling period: nearest samples"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in inside for k in range(4) if r[3][k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": reasons, "samples": len(inside), "note": note}


# ----------------------------------------------------------- distributed ---
class Dist:
    def __init__(self, backend: str):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float, device=None) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=device)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ------------------------------------------------------------ our kernels ---
def profile_fields(kind: str):
    """The machine-read lines of the committed ncu summary of the flip kernel,
    if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "flip_L1024_%s.md" % kind)
    src = os.path.join(ROOT, "paper_1411_0127_gb300", "csrc")
    if not os.path.exists(path):
        return None
    h = hashlib.sha256()
    for name in sorted(os.listdir(src)):
        if name in ("isg_flip_fast.cu", "isg_stream.cuh", "isg_common.cuh"):
            h.update(open(os.path.join(src, name), "rb").read())
    digest = h.hexdigest()[:16]
    fields = {}
    for line in open(path):
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            fields[k.strip()] = v.strip()
    if fields.get("kernel_source_sha256_16") != digest:
        return None
    return fields


def traffic_from_profile(kind: str):
    """DRAM bytes per colour pass of the flip kernel from the committed ncu
    summary (None if it was not taken on the current kernel source)."""
    f = profile_fields(kind)
    try:
        return float(f["dram_bytes_per_pass"]) if f else None
    except (KeyError, ValueError):
        return None


def issue_from_profile(kind: str):
    """ncu's issue-slot utilisation and warp instructions per 32 attempts of the
    flip kernel from the committed summary (None if stale)."""
    f = profile_fields(kind)
    try:
        return {"issue_active": float(f["issue_active_pct"]) / 100,
                "warp_instructions_per_32_attempts": float(f["warp_instructions_per_32_attempts"]),
                "source": "ncu, profiles/flip_L1024_%s.md" % kind} if f else None
    except (KeyError, ValueError):
        return None


def _stream_block(S: int, R: int, L: int, t0: int, m: int):
    """Streams [t0, t1) of a lattice, restarting at 0 when fewer than m remain, and
    the attempts of one colour pass over them (the last stream may be short)."""
    t0 = t0 % S
    if t0 + m > S:
        t0 = 0
    t1 = min(S, t0 + m)
    rows = min(t1 * R, L * L) - t0 * R
    return t0, t1, rows * (L // 2)


def cpu_baseline(w, target_s: float = 12.0) -> dict:
    """The oracle, as it stands, on this host's cores: whole sweeps (a red and a
    blue pass over all streams, the threads sharing out the streams of each
    pass) of the benchmark lattice, repeated for about target_s seconds; and
    on one core, passes over one stream at a time for about a quarter of that."""
    import oracle
    threads = os.cpu_count() or 1
    kinds = {"minstd": oracle.RNG_MINSTD, "mt19937": oracle.RNG_MT19937, "parisi_rapuano": oracle.RNG_PR}
    o = oracle.OracleSim(w.L, w.seed_J, w.seed_spin, w.beta, kinds[w.kind])
    S, R = oracle.num_streams(w.L), oracle.rows_per_stream(w.L)
    t_start = time.perf_counter()
    sweeps = 0
    while sweeps == 0 or time.perf_counter() - t_start < target_s:
        o.pass_range(0, 0, S, threads)
        o.pass_range(1, 0, S, threads)
        sweeps += 1
    dt = time.perf_counter() - t_start
    attempts = sweeps * w.L ** 3
    t_single, att1, t1s = time.perf_counter(), 0, 0
    while time.perf_counter() - t_single < target_s / 4:
        t1s, t1e, n = _stream_block(S, R, w.L, t1s, 1)
        o.pass_range(0, t1s, t1e, 1)
        o.pass_range(1, t1s, t1e, 1)
        att1 += 2 * n
        t1s = t1e
    dt1 = time.perf_counter() - t_single
    o.close()
    return {"value": dt * 1e12 / attempts, "unit": UNIT, "cores": min(threads, S), "kind": "oracle",
            "sample": "%d whole sweeps (red+blue passes over all %d streams) of the L=%d lattice on %d threads "
                      "(%d attempts, %.1f s wall)" % (sweeps, S, w.L, min(threads, S), attempts, dt),
            "single_core": {"value": dt1 * 1e12 / att1, "unit": UNIT, "cores": 1,
                            "sample": "red+blue passes over one stream at a time (%d attempts, %.1f s wall)"
                                      % (att1, dt1)}}


def batched_section(a, stream) -> dict:
    """The 512-sample batched workload (two replicas each, L in {16..192}, T in
    {0.7, 0.9, 1.1}, MT19937): psFlip of the persistent graph-replayed engine,
    against sweeping every replica on its own, one lattice per launch, with the
    plain per-colour kernel and with the fast kernel."""
    import torch
    import paper_1411_0127_gb300 as isg
    from paper_1411_0127_gb300 import workloads
    samples = workloads.batch_samples()
    b = isg.Batch([x.L for x in samples], [x.seed_J for x in samples],
                  [v for x in samples for v in x.seed_spin], [1.0 / x.T for x in samples], "mt19937")
    attempts = b.info()["attempts_per_sweep"]
    tuned = b.autotune(sweeps=16, stream=stream)      # untimed: candidates timed on a twin batch
    group = 64
    b.run(group, group, stream)                      # warm-up (captures the graph)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.run(a.batch_groups * group, group, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    sweeps = a.batch_groups * group
    out = {"workload": "512 samples x 2 replicas, L uniform over {16,32,48,64,96,128,192}, T over {0.7,0.9,1.1}, "
                       "MT19937, sampler seed 7; %d attempts per sweep" % attempts,
           "group_sweeps": group, "timed_sweeps": sweeps, "launches": a.batch_groups,
           "psflip": ms * 1e9 / (sweeps * attempts),
           "samples_sweeps_per_s": len(samples) * sweeps / (ms / 1e3),
           "autotune": {"config": list(tuned["config"]), "candidates": len(tuned["table"]),
                        "psflip_by_config_16_sweeps": {"%d/%d/%d/%d" % tuple(c): round(p, 4) for c, p in tuned["table"]},
                        "note": "config = engine (0: 32x1, 1: 24x1, 2: 16x1, 3: 16x2 warps x CTAs per SM, persistent "
                                "bundles; 4: one launch per colour pass; 5: one launch per sweep group, per-lattice "
                                "waits) / streams per bundle / resident generator state / words per lane"}}
    members = [b.member(r) for r in range(2 * len(samples))]
    for name, fn in (("plain_one_sample_per_launch_psflip", "sweep_plain"),
                     ("fast_one_sample_per_launch_psflip", "sweep")):
        n = 2
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for m in members:
            getattr(m, fn)(n, stream)
        p1.record(stream)
        torch.cuda.synchronize()
        out[name] = p0.elapsed_time(p1) * 1e9 / (n * attempts)
    b.close()
    return out


def other_configs_section(stream) -> dict:
    """psFlip of the other single-lattice workloads (the parity configurations),
    each timed with CUDA events after a warm-up, for context."""
    import torch
    import paper_1411_0127_gb300 as isg
    from paper_1411_0127_gb300 import workloads
    out = {}
    cases = [("L32_minstd_T1.1", workloads.SMALL, 2000), ("L256_minstd_T0.7", workloads.MEDIUM_MINSTD, 1000),
             ("L256_mt19937_T0.7", workloads.MEDIUM_MT, 1000),
             ("L1024_minstd_T0.9", dataclasses.replace(workloads.LARGE, kind="minstd"), 300),
             ("L1024_parisi_rapuano_T0.9", dataclasses.replace(workloads.LARGE, kind="parisi_rapuano"), 300)]
    for name, w, n in cases:
        s = isg.Sim(w.L, w.seed_J, w.seed_spin, w.beta, w.kind)
        s.sweep(10, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.sweep(n, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = {"psflip": e0.elapsed_time(e1) * 1e9 / (n * w.L ** 3), "sweeps": n,
                     "streams": s.info()["streams"]}
        s.close()
    return out


def rng_section() -> dict:
    """Device-API generator benchmark (Sec. 3, Table MYTEST): the paper's run is
    64 x 256 threads x 2^15 numbers x 10 = 5.4e9 instances; here 8192 streams x
    2^16 numbers x 10 calls (the same total), counting odd outputs."""
    import paper_1411_0127_gb300 as isg
    out = {"paper_gtx_titan_instances_per_s": {"mt19937": 14.1e9, "minstd": 8.9e10, "parisi_rapuano": 16.8e9}}
    for kind in ("mt19937", "minstd", "parisi_rapuano"):
        isg.rng_count_odd(kind, 1, 8192, 4096)                 # warm-up
        total_ms, odd, n = 0.0, 0, 0
        for rep in range(10):
            o, ms = isg.rng_count_odd(kind, 100 + rep, 8192, 2**16)
            total_ms += ms
            odd += o
            n += 8192 * 2**16
        out[kind] = {"instances_per_s": n / (total_ms / 1e3), "odd_fraction": odd / n, "instances": n}
    return out


def hbm_peak() -> tuple:
    """The measured HBM copy rate in GB/s from MEASURED_PEAKS.json, else a
    fallback of 6800 GB/s (an earlier copy measurement on a GB300)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            return float(json.load(open(path))["hbm_gbs"]), "measured"
        except (ValueError, KeyError):
            pass
    return 6800.0, "fallback"


def amsc_section(stream) -> dict:
    """Asynchronous multispin coding (Sec. 4): 32 systems per word, one draw per
    site shared by the 32.  psFlip = time / (32 L^3 sweeps), the paper's unit for
    its ~3 (MINSTD) and ~5 (MT19937) psFlip on a GTX Titan.  Algorithmic HBM
    bytes per colour pass and site word: 8 words read (S, Jx, Jy, Jz of both
    colours) + 1 written = 36 B per 32 attempts."""
    import torch
    import paper_1411_0127_gb300 as isg
    from paper_1411_0127_gb300 import workloads
    out = {"paper_gtx_titan_psflip": {"minstd": 3.0, "mt19937": 5.0}, "bytes_per_attempt": 36 / 32}
    for L, kind, n in [(1024, "mt19937", 40), (1024, "minstd", 40), (1024, "parisi_rapuano", 40),
                       (256, "mt19937", 400)]:
        seed_J, seed_spin = workloads.amsc_seeds(L)
        m = isg.Amsc(L, seed_J, seed_spin, 12345, 1 / 0.9, kind)
        m.sweep(3, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        m.sweep(n, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        att = 32 * L ** 3 * n
        gbs = att * 36 / 32 / (ms / 1e3) / 1e9
        out["L%d_%s_T0.9" % (L, kind)] = {"psflip": ms * 1e9 / att, "sweeps": n, "hbm_gbs": gbs,
                                          "hbm_frac_of_measured": gbs / hbm_peak()[0]}
        m.close()
    return out


def _serve(jobs, budget: int, quantum: int, time_limit_s: float = 600.0) -> dict:
    """Serve `jobs` (arrival times in seconds from the start of the run) and
    summarise latency (completion - arrival, queueing included) and throughput."""
    import numpy as np
    import paper_1411_0127_gb300 as isg
    srv = isg.Server(budget, quantum, 4096)
    ids = [srv.submit(j.L, j.seed_J, j.seed_spin, 1.0 / j.T, j.kind, j.sweeps, j.arrival) for j in jobs]
    srv.run(time_limit_s=time_limit_s)
    res = [srv.job(i) for i in ids]
    st = srv.stats()
    srv.close()
    lat = np.array([r["latency"] for r in res])
    queue = np.array([r["admit"] - r["arrival"] for r in res])
    return {"jobs": len(jobs), "finished": sum(r["status"] == 2 for r in res), "attempts": st["attempts"],
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()), "mean_admission_wait_s": float(queue.mean()),
            "queueing_share": float(queue.sum() / max(lat.sum(), 1e-12)),
            "aggregate_psflip": st["busy_s"] * 1e12 / max(1, st["attempts"]),
            "wall_psflip": st["wall_s"] * 1e12 / max(1, st["attempts"]),
            "attempts_per_s": st["attempts"] / max(st["wall_s"], 1e-12),
            "wall_s": st["wall_s"], "quanta": st["iterations"], "peak_active": st["peak_active"],
            "peak_bytes": st["peak_bytes"]}


SERVE_SWEEP_SCALE = 16     # sweeps of the sustainable-load trace: the trace's count / 16
SERVE_LOAD = 0.8           # offered load of the sustainable run, as a fraction of measured capacity


def serving_section(a) -> dict:
    """Continuous batching under a 150 GB budget, in two regimes.

    overload: the first `--serve-jobs` jobs of the Poisson quench trace as
    specified (200 jobs/s, L over even multiples of 16 in [32, 512], sweeps
    log-uniform in [1e2, 1e5], T uniform in [0.5, 1.5], MINSTD or MT19937),
    which offers about 100 times what one GPU can sweep.

    sustainable: `--serve-sustained-jobs` jobs with the same L, T and kinds and
    sweeps divided by SERVE_SWEEP_SCALE, first all at once (the capacity on
    this job mix: attempts per second of wall time), then as Poisson arrivals
    at SERVE_LOAD of that capacity; p50 / p99 latency with queueing included."""
    import dataclasses as dc
    from paper_1411_0127_gb300 import workloads
    budget, quantum = 150 * 10**9, 64
    out = {"budget_bytes": budget, "quantum_sweeps": quantum}
    if a.serve_jobs > 0:
        jobs = workloads.serving_trace(a.serve_jobs)
        r = _serve(jobs, budget, quantum)
        r["trace"] = ("first %d jobs of the Poisson trace (200 jobs/s, arrival seed 11), %.3g attempts, arrivals "
                      "over %.3f s" % (len(jobs), r["attempts"], jobs[-1].arrival))
        out["overload"] = r
        # the keys of the overload regime also at the top level
        out.update({k: r[k] for k in ("trace", "jobs", "finished", "p50_latency_s", "p99_latency_s",
                                      "mean_admission_wait_s", "aggregate_psflip", "wall_s", "quanta",
                                      "peak_active", "peak_bytes")})
    n = a.serve_sustained_jobs
    if n > 0:
        def scaled(rate):
            return [dc.replace(j, sweeps=max(1, j.sweeps // SERVE_SWEEP_SCALE))
                    for j in workloads.serving_trace(n, rate=rate)]
        burst = [dc.replace(j, arrival=0.0) for j in scaled(200.0)]
        cap = _serve(burst, budget, quantum)
        mean_work = sum(j.L ** 3 * j.sweeps for j in burst) / n
        rate = SERVE_LOAD * cap["attempts_per_s"] / mean_work
        jobs = scaled(rate)
        r = _serve(jobs, budget, quantum)
        r.update({"offered_load": SERVE_LOAD, "arrival_rate_jobs_per_s": rate,
                  "offered_attempts_per_s": rate * mean_work, "capacity_attempts_per_s": cap["attempts_per_s"],
                  "trace": "%d jobs of the trace's L, T and kind draws (arrival seed 11) with sweeps / %d "
                           "(mean %.3g attempts per job), Poisson arrivals at %.3g jobs/s = %.2f of the capacity "
                           "measured on the same jobs submitted at once" %
                           (n, SERVE_SWEEP_SCALE, mean_work, rate, SERVE_LOAD)})
        out["sustainable"] = r
        out["capacity_burst"] = {k: cap[k] for k in ("jobs", "finished", "attempts", "wall_s", "attempts_per_s",
                                                       "aggregate_psflip", "p50_latency_s", "p99_latency_s")}
    return out


def run_ours(a, dist: Dist):
    import numpy as np
    import torch
    import paper_1411_0127_gb300 as isg
    from paper_1411_0127_gb300 import workloads

    torch.cuda.set_device(dist.local)
    isg.use_torch_allocator()
    w = workloads.LARGE if a.L <= 0 else dataclasses.replace(workloads.LARGE, L=a.L)
    seed_spin = w.seed_spin + 1000 * dist.rank
    sim = isg.Sim(w.L, w.seed_J, seed_spin, w.beta, w.kind)
    stream = torch.cuda.current_stream()
    N = w.L ** 3

    sim.sweep(a.warmup, stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(dist.local)
    clocks.start()
    time.sleep(0.2)
    dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0 = time.time()
    e0.record(stream)
    sim.sweep(a.steps, stream)      # the K timed sweeps as one call, as a run of K sweeps is made
    e1.record(stream)
    torch.cuda.synchronize()
    h1 = time.time()
    dist.barrier()
    clk = clocks.stop(h0, h1)
    ms = e0.elapsed_time(e1)
    ms_max = dist.max(ms, device="cuda")
    # isg_sweep runs the 2K colour passes in launches of up to 128 passes where
    # the lattice allows it (a call of at least 8 sweeps), else one launch each
    passes = 2 * a.steps
    per_launch = sim.passes_per_launch() if a.steps >= 8 else 1
    launches = -(-passes // per_launch)
    launch_s = ms / 1e3 / launches
    attempts_per_launch = N * a.steps / launches
    value = ms_max * 1e9 / (a.steps * N * dist.world)   # ps per attempt, whole job

    # the plain per-colour kernel on the same lattice
    plain = None
    if a.plain_steps > 0:
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(a.plain_steps):
            sim.sweep_plain(1, stream)
        p1.record(stream)
        torch.cuda.synchronize()
        plain = p0.elapsed_time(p1) * 1e9 / (a.plain_steps * N)

    # the energy popcount kernel (isg_energy) against HBM: its algorithmic
    # traffic is every bit plane read once, 4 bits per site (the spins of both
    # colours and the three forward couplings); the memset and the 8-byte read
    # of the result ride along inside the events
    en0, en1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sim.energy(stream)
    n_en = 20
    en0.record(stream)
    for _ in range(n_en):
        sim.energy(stream)
    en1.record(stream)
    torch.cuda.synchronize()
    en_ms = en0.elapsed_time(en1) / n_en
    en_gbs = N * 0.5 / (en_ms / 1e3) / 1e9

    # end to end through the C-ABI with host buffers, every step: the spin
    # configuration in from pinned host memory, one sweep, the configuration and
    # the tracked energy out.  Main form: packed bits (1 bit per spin, the
    # engine's own coding); also timed with int8 +-1 (one byte per spin).
    nb = (N + 7) // 8
    p_in = torch.empty(nb, dtype=torch.uint8, pin_memory=True).numpy()
    p_out = torch.empty(nb, dtype=torch.uint8, pin_memory=True).numpy()
    h_in = torch.empty(N, dtype=torch.int8, pin_memory=True).numpy()
    h_out = torch.empty(N, dtype=torch.int8, pin_memory=True).numpy()
    sim.read_spins_packed(stream, out=p_in)
    sim.read_spins(stream, out=h_in)
    sim.write_spins_packed(p_in, stream)              # untimed: the staging buffers are allocated once
    sim.write_spins(h_in, stream)
    n_e2e = max(1, min(a.e2e_steps, a.steps))

    def e2e_run(write, read, src, dst):
        dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            write(src, stream)
            sim.sweep(1, stream)
            read(stream, out=dst)
            sim.tracked_energy()
        torch.cuda.synchronize()
        return dist.max(time.perf_counter() - t0, device="cuda") * 1e12 / (n_e2e * N * dist.world)

    e2e_seq = e2e_run(sim.write_spins_packed, sim.read_spins_packed, p_in, p_out)
    e2e_int8 = e2e_run(sim.write_spins, sim.read_spins, h_in, h_out)

    # The same exchange (configuration in, one sweep, configuration and tracked
    # energy out, every step) through isg_exchange_async, pipelined over
    # E2E_HANDLES lattices of the same workload on as many streams: step k uses
    # lattice k mod E2E_HANDLES, so while one lattice sweeps, the copy engines
    # move the others' configurations in and out.
    hs = [sim] + [isg.Sim(w.L, w.seed_J, seed_spin + j, w.beta, w.kind) for j in range(1, E2E_HANDLES)]
    sts = [stream] + [torch.cuda.Stream() for _ in range(1, E2E_HANDLES)]
    ins = [torch.empty(nb, dtype=torch.uint8, pin_memory=True).numpy() for _ in hs]
    outs = [torch.empty(nb, dtype=torch.uint8, pin_memory=True).numpy() for _ in hs]
    Es = [torch.empty(1, dtype=torch.int64, pin_memory=True).numpy() for _ in hs]
    for h, bi, bo, eo, st in zip(hs, ins, outs, Es, sts):
        h.read_spins_packed(st, out=bi)
        h.exchange_async(bi, bo, 0, eo, st)           # untimed: the staging buffer is allocated once
    n_pipe = max(n_e2e, E2E_PIPE_STEPS)
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(n_pipe):
        j = k % E2E_HANDLES
        hs[j].exchange_async(ins[j], outs[j], 1, Es[j], sts[j])
    torch.cuda.synchronize()
    e2e_value = dist.max(time.perf_counter() - t0, device="cuda") * 1e12 / (n_pipe * N * dist.world)
    for h in hs[1:]:
        h.close()

    batched = batched_section(a, stream) if a.batch_groups > 0 else None
    serving = (serving_section(a) if (a.serve_jobs > 0 or a.serve_sustained_jobs > 0) and dist.rank == 0
               else None)
    others = other_configs_section(stream) if a.other_configs and dist.rank == 0 else None
    rng = rng_section() if a.other_configs and dist.rank == 0 else None
    amsc = amsc_section(stream) if a.amsc and dist.rank == 0 else None

    ops = OPS_PER_ATTEMPT[w.kind]
    achieved_tops = ops * attempts_per_launch / launch_s / 1e12
    hbm_gbs = BYTES_PER_ATTEMPT * attempts_per_launch / launch_s / 1e9
    hbm_pk, hbm_src = hbm_peak()
    per_pass = traffic_from_profile(w.kind)
    traffic = per_pass * passes / launches if per_pass is not None else None
    int_rates = {name: isg.int_rate(mode) / 1e12 for mode, name in ((0, "lop3_imad"), (1, "lop3"), (2, "imad"))}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic", "impl": "ours",
        "config": {**workload_config(w), "parallelism": "replicas only"},
        "parallelism": "one lattice per GPU; under torchrun every rank sweeps its own replica",
        "plain_psflip": plain,
        "batched_psflip": batched["psflip"] if batched else None,
        "batched": batched,
        "serving": serving,
        "other_configs": others,
        "rng_device_api": rng,
        "amsc": amsc,
        "roofline": {"bound": "alu", "achieved": achieved_tops, "peak": ALU_PEAK_TOPS, "unit": "Tops/s",
                     "frac": achieved_tops / ALU_PEAK_TOPS, "traffic": traffic,
                     "kernel": ("flip_sweeps_kernel (up to %d colour passes per launch, %.1f on average here)"
                                % (per_launch, passes / launches) if per_launch > 1
                                else "flip_fast_kernel (one colour pass per launch)"),
                     "ops_per_attempt": ops,
                     "attempts_per_launch": attempts_per_launch, "launch_ms": launch_s * 1e3,
                     "peak_source": "derived: 152 SMs x 128 lanes x 2070 MHz",
                     "measured_int_peaks_tops": int_rates,
                     "frac_of_measured_lop3_imad": achieved_tops / int_rates["lop3_imad"],
                     "issue": issue_from_profile(w.kind),
                     "hbm": {"achieved": hbm_gbs, "peak": hbm_pk, "unit": "GB/s", "frac": hbm_gbs / hbm_pk,
                             "peak_source": hbm_src, "bytes_per_attempt": BYTES_PER_ATTEMPT}},
        "energy_kernel": {"ms": en_ms, "achieved_gbs": en_gbs, "bytes_per_site": 0.5,
                          "frac_of_hbm": en_gbs / hbm_peak()[0],
                          "note": "isg_energy at the same lattice: unsatisfied-bond popcount over all planes"},
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb + 8,
                "steps": n_pipe,
                "path": "isg_exchange_async(pinned packed bits in, 1 sweep, packed bits and tracked energy out), "
                        "step k on lattice k mod %d, one stream each" % E2E_HANDLES,
                "sequential": {"value": e2e_seq, "steps": n_e2e,
                               "path": "one lattice, synchronous calls: isg_write_spins_packed(pinned) + isg_sweep + "
                                       "isg_read_spins_packed(pinned) + isg_tracked_energy"},
                "int8": {"value": e2e_int8, "h2d_bytes_per_step": N, "d2h_bytes_per_step": N + 8, "steps": n_e2e,
                         "path": "isg_write_spins(pinned int8) + isg_sweep + isg_read_spins(pinned int8) + "
                                 "isg_tracked_energy"}},
        "gpu_launches": launches,
    }
    sim.close()
    if dist.rank == 0 and dist.world == 1 and not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w)
    return out


# ----------------------------------------------------------- reference arm ---
def run_reference(a, dist: Dist):
    """The CPU oracle as it stands, on the host cores, on bounded samples of the
    same workload; every step is one red and one blue pass over a block of
    streams sized so that the whole run ends within about a minute."""
    if dist.rank != 0:
        return None
    import oracle
    from paper_1411_0127_gb300 import workloads
    w = workloads.LARGE if a.L <= 0 else dataclasses.replace(workloads.LARGE, L=a.L)
    threads = os.cpu_count() or 1
    o = oracle.OracleSim(w.L, w.seed_J, w.seed_spin, w.beta, oracle.RNG_MT19937)
    S, R = oracle.num_streams(w.L), oracle.rows_per_stream(w.L)
    t = time.perf_counter()
    o.pass_range(0, 0, threads, threads)
    o.pass_range(1, 0, threads, threads)
    cal = (time.perf_counter() - t) / threads            # seconds per stream pair, all cores busy
    budget = 60.0 / max(1, a.steps + a.warmup)
    m = int(max(threads, min(S, budget / max(cal, 1e-9))))
    m = min(S, max(threads, m // threads * threads))
    t0 = threads % S
    for _ in range(a.warmup):
        t0, t1, n = _stream_block(S, R, w.L, t0, m)
        o.pass_range(0, t0, t1, threads)
        o.pass_range(1, t0, t1, threads)
        t0 = t1
    times, done = [], 0
    for _ in range(a.steps):
        t0, t1, n = _stream_block(S, R, w.L, t0, m)
        s = time.perf_counter()
        o.pass_range(0, t0, t1, threads)
        o.pass_range(1, t0, t1, threads)
        times.append(time.perf_counter() - s)
        done += 2 * n
        t0 = t1
    attempts = done // max(1, a.steps)
    total = sum(times)
    value = total * 1e12 / max(1, done)
    o.close()
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": total * 1e3 / a.steps, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "int8", "data": "synthetic", "impl": "reference",
        "config": {**workload_config(w), "parallelism": "replicas only"},
        "parallelism": "one lattice on the host cores: threads share out the streams of each colour pass",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": min(threads, m), "kind": "oracle",
                         "sample": "each step: red+blue passes over %d of the %d streams of the L=%d lattice "
                                   "(%d attempts)" % (m, S, w.L, attempts)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    a = parse()
    dist = Dist("nccl" if a.impl == "ours" else "gloo")
    try:
        out = run_reference(a, dist) if a.impl == "reference" else run_ours(a, dist)
        if out is not None and dist.rank == 0:
            print(json.dumps(out), flush=True)
    finally:
        dist.close()


if __name__ == "__main__":
    main()

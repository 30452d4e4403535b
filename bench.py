#!/usr/bin/env python
"""Benchmark of the GB300 octahedron KPZ engine.

Workload (one step): the L = 2^16 job -- flat checkerboard start, p = 1, q = 0,
2000 Monte Carlo steps (sweeps of L^2 attempts each) with the exact width W^2
sampled at log-spaced times, through the C ABI of include/kpz.h. Metric:
site-update attempts per second (Kelling et al., arXiv:1204.5072, Sec. 4
report updates per second). One JSON line on stdout (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Besides `value` (lattice resident in HBM) the line carries `e2e` (the same job
with the start surface uploaded from pinned host memory and the final one read
back, per-part times and the bare pinned-copy bandwidth beside it), `roofline`
(the sweep kernel against the integer-logic pipe, with the HBM view, the
measured pipe peak and the DRAM traffic of the committed ncu capture),
`cpu_baseline` / `cpu_all_cores` / `cpu_rsu` (the oracle on a bounded sample),
`clocks`, `gpu_launches`, and the `batch` (ensemble) and `surrogate` sections.

`--impl reference` times the CPU oracle (the plain single-threaded
restatement of the same schedule) on a bounded sample of the workload.
Under torchrun every rank runs its own independent realisation (sample =
rank): the path has no exchange step, so the scaling is weak and replica-only.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time
import warnings

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import inputs as I  # noqa: E402

METRIC = "KPZ site-update attempts/s at L=2^16 (frac. of roofline); batched realisations/s"
UNIT = "attempts/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--L", type=int, default=I.L65536_2000.L)
    ap.add_argument("--mcs", type=int, default=I.L65536_2000.mcs)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample-mcs", type=int, default=100)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-cap", type=int, default=200)
    ap.add_argument("--batch-n", type=int, default=512)
    ap.add_argument("--batch-only", action="store_true",
                    help="profiling aid: run only the batched-ensemble section (no comparisons)")
    ap.add_argument("--no-surrogate", action="store_true")
    return ap.parse_args()


def peaks():
    """(HBM GB/s, SM max MHz, source) from the driver-written measurements."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


# ALU-pipe operations the algorithm needs per attempt at p = 1, q = 0 (bit-sliced
# rule on 32 cells per word, 2 Philox bits per attempt, window staging):
# 20/64 (Philox xors) + 22/32 (masks, tests, flips, neighbour shifts) + 64/512.
K_ALG_ALU = 20 / 64 + 22 / 32 + 64 / 512
ALU_LANES_PER_SM = 64   # integer logic pipe: 16 lanes per SM sub-partition per clock


# Files the sweep kernel is compiled from (their hash ties a profile to the source).
SWEEP_SOURCES = ("kpz_sweep.cu", "kpz_run.cuh", "kpz_rounds.cuh", "kpz_common.cuh", "kpz_internal.h")


def sweep_source_sha():
    import hashlib
    src = b"".join(open(os.path.join(ROOT, "paper_1204_5072_gb300", "csrc", f), "rb").read()
                   for f in SWEEP_SOURCES)
    return hashlib.sha256(src).hexdigest()[:16]


def measured_traffic(L):
    """DRAM bytes per sweep launch from the committed ncu summary, if it was
    taken on this size and on the current kernel source; else None."""
    try:
        sha = sweep_source_sha()
        txt = open(os.path.join(ROOT, "profiles", "sweep_kernel_L65536.md")).read()
        fields = dict(ln.split(": ", 1) for ln in txt.splitlines() if ": " in ln and ln[:1].isalpha())
        if L == 65536 and fields.get("source_sha256") == sha:
            return float(fields["traffic_bytes_per_launch"])
    except Exception:
        pass
    return None


# --------------------------------------------------------------------------- #
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- #
def cpu_baseline(L_full: int, mcs_sample: int):
    """The oracle, as it stands (single-threaded C), on a bounded sample of the
    workload: L = 1024 with the same schedule parameters, `mcs_sample` sweeps
    from the flat start and W^2 at the end."""
    from oracle import oracle as O
    L = 1024
    w = I.L65536_2000
    st = O.State.flat(L)
    t0 = time.perf_counter()
    st.run(mcs_sample, w.bx, w.by, w.p, w.q, w.seed, w.sample)
    st.w2()
    dt = time.perf_counter() - t0
    return {"value": mcs_sample * L * L / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"L={L} p={w.p} q={w.q} seed={w.seed}, {mcs_sample} MCS from the flat start "
                      f"+ W^2, 128x128 tiles (sub-run of the L={L_full} workload)",
            "seconds": dt}


def replica_sample(rank: int) -> int:
    """The realisation a rank runs under torchrun: sample = rank, i.e. its own
    Philox streams (the path has no exchange step; replicas only)."""
    return rank


def max_over_ranks(seconds: float, dist=None, device="cuda") -> float:
    """The slowest rank's time (the job ends when every rank has finished)."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, steps: int, mcs: int, L: int, seconds: float) -> float:
    """Attempts/s of the whole job: every rank sweeps its own L x L lattice."""
    return float(world) * steps * mcs * L * L / seconds


def job_config(L, mcs, world):
    """The `config` of the benchmark job (both arms report the same one)."""
    w = I.L65536_2000
    n = len(I.sample_times(mcs))
    return {"workload": f"octahedron KPZ L={L} p=1 q=0 {mcs} MCS, W^2 at "
                        f"{n} log-spaced times, 1 realisation per GPU",
            "L": L, "p": w.p, "q": w.q, "mcs": mcs, "samples": n,
            "tile": "128x128, 4x4 cells", "seed": w.seed,
            "l2": "lattice (L^2/8 bytes = 512 MiB at L=2^16) larger than L2",
            "parallelism": f"replicas{world}"}


def cpu_all_cores(mcs_sample: int):
    """The oracle with the tiles of each sweep spread over every host core
    (bit-identical to the serial oracle), on the same L = 1024 sub-run."""
    from oracle import oracle as O
    L, w = 1024, I.L65536_2000
    cores = os.cpu_count() or 1
    st = O.State.flat(L)
    t0 = time.perf_counter()
    st.run_threads(mcs_sample, w.bx, w.by, w.p, w.q, w.seed, w.sample, threads=cores)
    st.w2()
    dt = time.perf_counter() - t0
    return {"value": mcs_sample * L * L / dt, "unit": UNIT, "cores": cores,
            "kind": "oracle, tiles of a sweep over all host threads",
            "sample": f"L={L}, {mcs_sample} MCS from the flat start + W^2", "seconds": dt}


def cpu_rsu(mcs_sample: int):
    """The oracle's random-sequential updates (one attempt at a uniformly random
    site at a time, no decomposition: the dynamics the decomposition
    approximates) on one core, L = 1024 from the flat start."""
    from oracle import oracle as O
    L, w = 1024, I.L65536_2000
    st = O.State.flat(L)
    t0 = time.perf_counter()
    st.rsu(mcs_sample, w.p, w.q, w.seed, w.sample)
    dt = time.perf_counter() - t0
    return {"value": mcs_sample * L * L / dt, "unit": UNIT, "cores": 1,
            "kind": "oracle, random-sequential updates",
            "sample": f"L={L}, {mcs_sample} MCS from the flat start", "seconds": dt}


# The paper's own update rates (order of magnitude from its text; its figures
# are not available): context for the GB300 numbers, not a target.
PAPER_CONTEXT = {"gpu_updates_per_s": 1e9,
                 "gpu_hardware": "Tesla C1060, Fermi C2050/C2070, Radeon HD5970/HD6970",
                 "cpu_updates_per_s": 1e7,
                 "cpu_hardware": "Opteron F8380, Core i5 430M, Core i7 920 (one core)",
                 "workload": "p = 1, q = 0, bit-coded lattice (Sec. 4)"}


def run_reference(a):
    """--impl reference: the CPU oracle timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    w = I.L65536_2000
    L, per_step = 1024, 4
    O.build()
    st = O.State.flat(L)
    for _ in range(a.warmup):
        st.run(per_step, w.bx, w.by, w.p, w.q, w.seed, w.sample)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        st.run(per_step, w.bx, w.by, w.p, w.q, w.seed, w.sample)
        st.w2()
    dt = time.perf_counter() - t0
    value = a.steps * per_step * L * L / dt
    sample = (f"L={L} p={w.p} q={w.q} seed={w.seed}, {per_step} MCS + W^2 per step, "
              f"128x128 tiles (sub-run of the L={a.L} workload)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * dt / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic (flat checkerboard start)",
            "config": job_config(a.L, a.mcs, a.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- #
def batch_bench(eng, cap, seed=1, n_specs=512, compare=True):
    """Batched ensemble (512 realisations shaped like the batched workload: L =
    2^{8..13} log-uniform, p ~ U[0.5, 1], q = 1 - p, run length min(4 L^1.6, cap)),
    one persistent graph launch, against (i) one launch per sweep per realisation
    (kpz_run, W^2 at the same times) and (ii) one persistent launch per realisation."""
    import torch
    specs = [(s.L, s.p, s.q, seed, s.sample, min(s.mcs, cap)) for s in I.ensemble_specs(n_specs, seed=seed)]
    attempts = float(sum(L * L * n for L, _, _, _, _, n in specs))
    t0 = time.perf_counter()
    b = eng.Batch(specs, n_samples=64, autotune=True)
    create_s = time.perf_counter() - t0
    b.run()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.run()
    torch.cuda.synchronize()
    batched = time.perf_counter() - t0
    times = [int(t) for t in b.times()]
    info = b.info()
    b.close()
    n = len(specs)
    out = {"metric": "batched realisations/s", "value": n / batched, "unit": "realisations/s",
           "attempts_per_s": attempts / batched, "seconds": batched,
           "workload": f"{n} realisations, L=2^(8..13) log-uniform, p~U[0.5,1], q=1-p, "
                       f"T=min(4 L^1.6, {cap}) MCS, W^2 at the common log-spaced times (seed {seed})",
           "tuning": {k: info[k] for k in ("run", "warps_per_cta", "ctas_per_sm", "grid", "graph", "tile_y")},
           "autotune_s": create_s}
    if not compare:
        return out
    t0 = time.perf_counter()
    for (L, p, q, sd, smp, n) in specs:
        lat = eng.Lattice(L, p, q, seed=sd, sample=smp)
        tp = 0
        for t in times:
            if t > n:
                break
            if t > tp:
                lat.run(t - tp)
            lat.roughness()
            tp = t
        lat.close()
    per_sweep = time.perf_counter() - t0
    t0 = time.perf_counter()
    for sp in specs:
        one = eng.Batch([sp], n_samples=64)
        one.run()
        one.close()
    per_real = time.perf_counter() - t0
    n = len(specs)
    out["vs_launch_per_sweep"] = {"value": n / per_sweep, "seconds": per_sweep, "speedup": per_sweep / batched}
    out["vs_launch_per_realisation"] = {"value": n / per_real, "seconds": per_real,
                                        "speedup": per_real / batched}
    return out


def surrogate_bench(eng):
    """Surrogate trained by the engine's kernels on simulated ensemble means
    (L in {128, 256}, p in {0.7, 0.8, 0.9, 1.0}, q = 1 - p, 64 realisations each,
    run length 4 L^1.6); error against fresh 128-realisation ensembles at held-out
    p in {0.75, 0.95}; planned run lengths 2 t_sat against 4 L^1.6."""
    import math
    import numpy as np
    from paper_1204_5072_gb300 import surrogate as S

    def heur(L):
        return int(min(math.ceil(4 * L ** 1.6), 100_000))

    def ens(pairs, seeds, run_len):
        specs = [(L, p, 1 - p, 100 + k, k, run_len(L, p)) for (L, p) in pairs for k in seeds]
        b = eng.Batch(specs, n_samples=48)
        b.run()
        t, w = b.times(), b.w2()
        b.close()
        out = {}
        for (L, p) in pairs:
            rows = [i for i, sp in enumerate(specs) if sp[0] == L and sp[1] == p]
            with warnings.catch_warnings():   # times past every run's end are all-NaN columns
                warnings.simplefilter("ignore", RuntimeWarning)
                out[(L, p)] = np.nanmean(w[rows], axis=0)
        return t, out

    LS, PT, PH = [128, 256], [0.7, 0.8, 0.9, 1.0], [0.75, 0.95]
    t0 = time.perf_counter()
    tr_pairs = [(L, p) for L in LS for p in PT]
    times, means = ens(tr_pairs, range(64), lambda L, p: heur(L))
    sim_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    sur = S.Surrogate.fit([(L, p, 1 - p, 0, 0, heur(L)) for (L, p) in tr_pairs], times,
                          np.stack([means[k] for k in tr_pairs]), epochs=400, batch=128, lr=3e-3, seed=1)
    train_s = time.perf_counter() - t0
    ho = [(L, p) for L in LS for p in PH]
    th, hmeans = ens(ho, range(200, 328), lambda L, p: heur(L))
    errs = {}
    for (L, p), m in hmeans.items():
        sel = (th >= 1) & (th <= heur(L)) & np.isfinite(m)
        errs[f"L{L}_p{p}"] = float(np.mean(np.abs(sur.w2(L, th[sel], p, 1 - p) / m[sel] - 1)))
    planned = {k: int(min(heur(k[0]), math.ceil(2 * sur.t_sat(k[0], k[1], 1 - k[1], t_max=heur(k[0])))))
               for k in ho}
    saved = sum((heur(L) - planned[(L, p)]) * L * L for (L, p) in ho) / sum(heur(L) * L * L for (L, p) in ho)
    sur.close()
    return {"held_out_mean_rel_error": errs, "max_mean_rel_error": max(errs.values()),
            "planned_mcs": {f"L{L}_p{p}": v for (L, p), v in planned.items()},
            "fixed_rule_mcs": {f"L{L}": heur(L) for L in LS}, "sweeps_saved_frac": saved,
            "train_s": train_s, "simulate_s": sim_s}


# --------------------------------------------------------------------------- #
def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
        return

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()
    import paper_1204_5072_gb300 as eng
    from paper_1204_5072_gb300._lib import launch_count
    if a.batch_only:   # profiling aid: the batched-ensemble section alone
        if rank == 0:
            print(json.dumps(batch_bench(eng, a.batch_cap, n_specs=a.batch_n, compare=False)), flush=True)
        return

    w = I.L65536_2000
    L, mcs = a.L, a.mcs
    times = I.sample_times(mcs)
    stream = torch.cuda.current_stream()
    lat = eng.Lattice(L, w.p, w.q, seed=w.seed, sample=replica_sample(rank))

    sweep_events = []  # (start, end, n_sweeps) on the engine's stream

    def job(record=False):
        lat.reset()
        t_prev = 0
        rough = []
        for t in times:
            n = t - t_prev
            if n:
                if record:
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                lat.run(n)
                if record:
                    e1.record(stream)
                    sweep_events.append((e0, e1, n))
            rough.append(lat.roughness())
            t_prev = t
        return rough

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(a.warmup, 3)):
        job()
    barrier()
    launches0 = launch_count()
    with ClockSampler(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for _ in range(a.steps):
            rough = job(record=True)
        t_end.record(stream)
        torch.cuda.synchronize()
    launches = launch_count() - launches0
    elapsed = max_over_ranks(t_start.elapsed_time(t_end) / 1e3, dist)
    attempts = float(world) * a.steps * mcs * L * L
    value = whole_job_value(world, a.steps, mcs, L, elapsed)
    sweep_ms = sum(e0.elapsed_time(e1) for e0, e1, _ in sweep_events)
    n_sweeps = sum(n for _, _, n in sweep_events)
    per_sweep_s = sweep_ms / 1e3 / n_sweeps

    # Roofline of the sweep kernel. The state is one bit per site, read and
    # written once per sweep (0.25 B/attempt); the integer-logic pipe binds
    # first: K_ALG_ALU ops per attempt against 152 SMs x 64 lanes x clock.
    hbm_peak, sm_mhz, peak_kind = peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    alg_bytes = 0.25 * L * L
    alu_peak = sms * ALU_LANES_PER_SM * sm_mhz * 1e6 / 1e12          # Top/s
    alu_achieved = K_ALG_ALU * L * L / per_sweep_s / 1e12
    hbm_achieved = alg_bytes / per_sweep_s / 1e9
    roofline = {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "Top/s",
                "frac": alu_achieved / alu_peak, "traffic": measured_traffic(L),
                "kernel": "sweep_kernel", "alg_ops_per_attempt": K_ALG_ALU,
                "launch_ms": per_sweep_s * 1e3,
                "peak_source": f"{sms} SMs x {ALU_LANES_PER_SM} ALU lanes x {sm_mhz:.0f} MHz ({peak_kind} clock)",
                "hbm": {"achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                        "frac": hbm_achieved / hbm_peak, "alg_bytes_per_launch": alg_bytes,
                        "peak_source": f"{peak_kind} hbm_gbs"}}
    # The derived ALU peak checked by the engine's own LOP3 throughput probe
    # (outside the timed region).
    try:
        probe = eng._lib.alu_peak()
        roofline["peak_probe"] = {"value": probe["lane_ops_per_s"] / 1e12, "unit": "Top/s",
                                  "of_derived": probe["lane_ops_per_s"] / 1e12 / alu_peak,
                                  "source": "kpz_alu_peak: one wave of independent LOP3 chains"}
    except Exception as exc:   # report, do not hide
        roofline["peak_probe"] = {"error": str(exc)}

    # End to end through the C ABI with host buffers: upload the start state
    # from pinned memory, run the job with W^2 sampling, read the final lattice.
    e2e = None
    if not a.no_e2e:
        nwords = L * L // 16
        h_in = torch.empty(nwords, dtype=torch.int32, pin_memory=True)
        h_out = torch.empty(nwords, dtype=torch.int32, pin_memory=True)
        host_in = h_in.numpy().view(np.uint32)
        host_in.reshape(L, L // 16)[0::2] = 0x33333333
        host_in.reshape(L, L // 16)[1::2] = 0xCCCCCCCC
        host_out = h_out.numpy().view(np.uint32)

        parts = []   # host clock at the boundaries; every call returns after its stream work

        def e2e_step():
            c0 = time.perf_counter()
            lat.set_slopes(host_in, h00=0, t=0)
            c1 = time.perf_counter()
            t_prev = 0
            for t in times:
                if t - t_prev:
                    lat.run(t - t_prev)
                lat.roughness()
                t_prev = t
            c2 = time.perf_counter()
            lat.slopes_into(host_out)
            parts.append((c1 - c0, c2 - c1, time.perf_counter() - c2))

        e2e_step()
        barrier()
        parts.clear()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            e2e_step()
        barrier()
        e2e_dt = max_over_ranks(time.perf_counter() - t0, dist)
        med = np.median(np.array(parts), axis=0) * 1e3
        # The bare pinned-memory copies of the same buffers in this process, for
        # reading the import/export parts (host links differ from box to box).
        dev_tmp = torch.empty(nwords, dtype=torch.int32, device="cuda")
        link = []
        for _ in range(2):
            torch.cuda.synchronize()
            c0 = time.perf_counter()
            dev_tmp.copy_(h_in, non_blocking=True)
            torch.cuda.synchronize()
            c1 = time.perf_counter()
            h_out.copy_(dev_tmp, non_blocking=True)
            torch.cuda.synchronize()
            link.append((c1 - c0, time.perf_counter() - c1))
        del dev_tmp
        best = np.min(np.array(link), axis=0)
        e2e = {"value": attempts / e2e_dt, "unit": UNIT, "h2d_bytes_per_step": nwords * 4,
               "d2h_bytes_per_step": nwords * 4 + len(times) * 48,
               "parts_ms": {"import": round(float(med[0]), 2), "job": round(float(med[1]), 2),
                            "export": round(float(med[2]), 2)},
               "bare_copy_gbs": {"h2d": round(nwords * 4 / best[0] / 1e9, 1),
                                 "d2h": round(nwords * 4 / best[1] / 1e9, 1)}}

    cpu = cpu_mt = cpu_seq = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cpu = cpu_baseline(L, a.cpu_sample_mcs)
        cpu_mt = cpu_all_cores(max(10, a.cpu_sample_mcs // 2))
        cpu_seq = cpu_rsu(max(4, a.cpu_sample_mcs // 10))
    batch = None if (a.no_batch or world > 1) else batch_bench(eng, a.batch_cap, n_specs=a.batch_n)
    sur = None if (a.no_surrogate or world > 1) else surrogate_bench(eng)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": max(a.warmup, 3), "ms_per_step": 1e3 * elapsed / a.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                "data": "synthetic (flat checkerboard start, p=1 q=0)",
                "config": job_config(L, mcs, world),
                "roofline": roofline, "cpu_baseline": cpu, "cpu_all_cores": cpu_mt, "cpu_rsu": cpu_seq,
                "paper_context": PAPER_CONTEXT, "e2e": e2e,
                "clocks": clk.summary(), "gpu_launches": launches,
                "w2_final": rough[-1]["w2"], "batch": batch, "surrogate": sur}
        print(json.dumps(line), flush=True)
    lat.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

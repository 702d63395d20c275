"""Benchmark: particle-updates per second of the full particle timestep on GB300.

One step = one pass of the whole particle path (advance and track, particle-number
control, statistics, conditional-mean binning, nodal averages) over all particles of the
workload: the 50,000-triangle wall-graded channel at 500 particles per element (25.0M
particles), synthetic seeded inputs.  The FP32 form (FP32 state and SDE arithmetic, FP64
statistics) is the headline; the plain FP64 form is measured on the same GPU beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pdfx|reference]

With N > 1 (torchrun), every rank steps its own independent instance (its own Philox
instance id): weak scaling with no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-updates/sec per full PDF timestep, FP32/batched vs FP64, same GPU"
UNIT = "particle-updates/s"
# Algorithmic bytes per particle-update (keys: 1 FP32 form, 0 FP64 form).
# advance (pass 1): read the position, u, v, w, omega, psi, the particle id (Philox
#   counter), elem, cp; write the position, u, v, w, omega, psi, elem.  The FP32 form holds
#   each coordinate as an FP32 pair (hi + lo, 8 B): 4*9+4+4+1+4*9+4 = 85 B; the FP64 form
#   8*7+4+4+1+8*7+4 = 125 B.
# binning (pass 2): read u, v, w, omega, psi (the moments of Eqs. 35-36), the particle id
#   (the (value, id) order of the bins), the element; write cp: 4*5+4+4+1 = 29 B,
#   8*5+4+4+1 = 49 B.
# With single FP32 positions the FP32 step would be 69 + 29 = 98 B; the pairs add 16 B.
ADV_BYTES = {1: 85, 0: 125}
BIN_BYTES = {1: 29, 0: 49}
SINGLE_POSITION_STEP_BYTES = 98
# Figures from ncu captures of the kernels (DRAM bytes per particle and launch,
# dram__bytes_read.sum + dram__bytes_write.sum; FP64 instructions per particle of the FP64
# form's advance; the bound each capture shows), keyed by the SHA-256 of the CUDA sources'
# code (comments aside) they were taken from: a capture describes only the kernels it
# measured, so after any change of the code the bench reports traffic as null until the
# next capture.
NCU_RECORDS = {
    # channel_50k, 25.0M particles (FP32) and 5.0M (FP64 form), one GB300
    "884109f4ef9f937ec8e6c0f340dcb09331d34ffda8b87605775c6a478bbb70d9": {
        "traffic": {"advance": (1162.113e6 + 949.069312e6) / 25.0e6,
                    "statistics_binning": (0.066048e6 + 688.4096e6 + 49.580032e6 + 237.703168e6
                                           + 10.723072e6) / 25.0e6},
        "limiter": {"advance": "instruction issue: 76% issue-active at 49% warps active (64 "
                               "registers cap 4 blocks of 256), long-scoreboard stalls first; "
                               "DRAM 25% of peak",
                    "statistics_binning": "instruction issue and shared-memory latency: 71% "
                                          "issue-active (<= 512 class), short-scoreboard stalls "
                                          "first; DRAM 13% of peak"},
        "f64_advance_fp64_inst_per_particle": (1407568787 + 454038118 + 836638858) / 5.0e6,
    },
}
STAGES = ["advance", "plan", "lists", "redistribute", "statistics_binning", "node_average"]


def _code_only(text: str) -> str:
    """C++/CUDA source without its comments and blank lines (string and character literals
    kept as they are, trailing blanks dropped): what a compiler sees of it."""
    out = []
    i, n = 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    lines = (line.rstrip() for line in "".join(out).split("\n"))
    return "\n".join(line for line in lines if line)


def kernel_sources_hash() -> str:
    """SHA-256 over the CUDA sources of the library (file names and their code without
    comments and blank lines, sorted by name): a change of comments alone keeps the hash."""
    import hashlib
    d = os.path.join(ROOT, "paper_1006_0532_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h")):
            h.update(name.encode())
            with open(os.path.join(d, name), encoding="utf-8") as f:
                h.update(_code_only(f.read()).encode())
    return h.hexdigest()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        try:
            self.f.flush()
            rows = [l.strip().split(", ") for l in open(self.f.name) if l.strip()]
        except Exception:
            rows = []
        finally:
            try:
                os.unlink(self.f.name)
            except Exception:
                pass
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def oracle_sample(workload_name: str, steps: int, ppe: int):
    """The oracle as it stands (one host thread) on a bounded sample of the workload."""
    import oracle
    from paper_1006_0532_gb300 import synth

    w = synth.workload(workload_name)
    # MINNPEL follows the particle count of the sample (one tenth, the workloads' ratio)
    o = oracle.Oracle(w["grid"], dict(w["params"], minnpel=max(1, ppe // 10)), w["fields"])
    o.init_particles(ppe)
    n = o.np_
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step(w["dt"])
    dt = time.perf_counter() - t0
    return n, steps, dt, w


def _oracle_part(job):
    """One host process of the all-core oracle timing: the oracle as it stands (one thread)
    stepping the particles of its share of the elements; waits at the barrier, then times
    its steps (it returns its particle count and time)."""
    workload, ppe, elems, warmup, steps, barrier = job
    import numpy as np
    import oracle
    from paper_1006_0532_gb300 import synth
    w = synth.workload(workload)
    o = oracle.Oracle(w["grid"], dict(w["params"], minnpel=0), w["fields"])
    o.init_elements(ppe, np.asarray(elems, dtype=np.int64))
    for _ in range(warmup):
        o.step(w["dt"])
    barrier.wait()
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step(w["dt"])
    return o.np_, time.perf_counter() - t0


def oracle_parallel(workload: str, ppe: int, warmup: int, steps: int, procs: int):
    """The oracle on all host cores: procs processes (spawned), each stepping the particles of
    a contiguous share of the elements with the unchanged one-thread oracle (particle-number
    control off: it couples all elements).  Throughput = all particles x steps / the slowest
    process's time."""
    import multiprocessing as mp
    import numpy as np
    from paper_1006_0532_gb300 import synth
    ne = synth.workload(workload)["grid"].ne
    procs = max(1, min(procs, ne))
    parts = np.array_split(np.arange(ne), procs)
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        barrier = mgr.Barrier(procs)
        with ctx.Pool(procs) as pool:
            res = pool.map(_oracle_part, [(workload, ppe, p.tolist(), warmup, steps, barrier)
                                          for p in parts])
    n = sum(r[0] for r in res)
    el = max(r[1] for r in res)
    return n, el


def host_cores():
    """Host cores this process may use, and the CPU model (lscpu) for the record."""
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Vendor ID") and model is None:
                model = line.split(":", 1)[1].strip()
    except Exception:
        pass
    return cores, model


def run_reference(args, rank, world):
    """The reference arm: the oracle (there is no other implementation of the paper's method
    to run), timed on all host cores, on the benchmark's grid at a bounded particle count."""
    if rank != 0:
        return
    ppe = args.oracle_ppe
    cores, model = host_cores()
    steps = max(1, args.steps)
    n, el = oracle_parallel(args.workload, ppe, min(args.warmup, 1), steps, cores)
    v = n * steps / el
    sample = ("%s grid at %d particles per element (%d particles), %d steps after %d, "
              "%d processes of the one-thread oracle over contiguous element shares"
              % (args.workload, ppe, n, steps, min(args.warmup, 1), cores))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "particles": n, "ppe": ppe,
                                            "host_cores": cores, "cpu": model},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(torch, dist, x: float) -> float:
    """The largest value over the ranks (the job's time is its slowest rank's); a CUDA tensor
    under NCCL, a host tensor under gloo."""
    if dist is None:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_params(params: dict, rank: int, precision: int, sort_every: int) -> dict:
    """Each rank steps its own instance: the Philox instance number is the rank."""
    return dict(params, precision=precision, sort_every=sort_every, instance=int(rank))


def make_ctx(B, w, precision, instance, sort_every, extra=None):
    p = dict(rank_params(w["params"], instance, precision, sort_every), **(extra or {}))
    c = B.Context(p)
    c.set_grid(w["grid"])
    c.set_fields(w["fields"])
    c.init_particles(w["ppe"])
    return c


def time_form(torch, B, w, precision, args, rank, world, dist, with_clock, extra=None):
    """Device time of K steps of one form (inputs resident in HBM)."""
    c = make_ctx(B, w, precision, rank, args.sort_every, extra)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        c.step(w["dt"])
    torch.cuda.synchronize()
    tuned = c.autotune(w["dt"]) if not args.no_autotune else None
    c.set_profiling(True)
    c.stage_times()
    l0 = c.kernel_launches
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(torch.cuda.current_device()) if with_clock else None
    if sampler:
        sampler.__enter__()
    ev0.record(stream)
    for _ in range(args.steps):
        c.step(w["dt"])
    ev1.record(stream)
    torch.cuda.synchronize()
    if sampler:
        sampler.__exit__()
    ms = ev0.elapsed_time(ev1)
    launches = c.kernel_launches - l0
    stage_ms, stage_n = c.stage_times()
    c.set_profiling(False)
    ms = max_over_ranks(torch, dist, ms)
    err = c.check()
    diag = c.diag()
    np_ = c.np_
    out = dict(ms=ms, launches=launches, stage_ms=stage_ms, stage_n=stage_n, np=np_, err=err,
               diag=diag, clocks=sampler.summary() if sampler else None, tuned=tuned,
               nodal=c.nodal_stats())
    return c, out


def e2e_form(torch, B, c, w, args):
    """Same metric through the C ABI with host buffers: per step, the nodal fields go
    host -> device from pinned memory, the step runs, the nodal statistics come back."""
    import numpy as np
    nn = w["grid"].nn
    f_host = torch.from_numpy(np.ascontiguousarray(w["fields"])).pin_memory()
    s_host = torch.empty((nn, 13), dtype=torch.float64).pin_memory()
    for _ in range(2):
        c.set_fields(f_host.numpy())
        c.step(w["dt"])
        c.nodal_stats(s_host.numpy())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        c.set_fields(f_host.numpy())
        c.step(w["dt"])
        c.nodal_stats(s_host.numpy())
    el = time.perf_counter() - t0
    return el, nn * 32 * 8, nn * 13 * 8


def element_areas(grid):
    """Triangle areas (x differences taken as minimum images on a periodic grid)."""
    import numpy as np
    xy = grid.node_xy[grid.tri]
    d1 = xy[:, 1] - xy[:, 0]
    d2 = xy[:, 2] - xy[:, 0]
    if grid.period_x > 0:
        L = grid.period_x
        for d in (d1, d2):
            d[:, 0] -= L * np.round(d[:, 0] / L)
    return 0.5 * np.abs(d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0])


def redistribution_study(torch, B, synth, args):
    """Sect. 3.7, Figs. 4-6: the simplified model of Eqs. 46-47 (alpha = 0.5) on the
    stretched 1,536-triangle grid, FP32 form, for 50 to 800 initial particles per element
    with MINNPEL = ppe / 10 (Eq. 51), and at 200 without particle-number control.  Per case:
    the relative error of the kinetic energy, Eq. 52, delta = (k_c - k_a) / k_a with k_a =
    3/2 and k_c half the area-weighted spatial average of the element variances, at t = 1,
    2 and 4; the particles moved per step; and the throughput of the steps."""
    import numpy as np
    out = {"what": "Eq. 52 delta at t = 1, 2, 4 (dt 0.01, 400 steps), FP32 form",
           "cases": {}}
    for ppe, redist in [(200, False), (50, True), (100, True), (200, True), (400, True),
                        (800, True)]:
        w = synth.redistribution_workload("redist_1k", ppe=ppe)
        p = dict(w["params"], precision=1, sort_every=args.sort_every)
        if not redist:
            p["minnpel"] = 0
        c = B.Context(p)
        c.set_grid(w["grid"])
        c.set_fields(w["fields"])
        c.init_particles(ppe)
        A = element_areas(w["grid"])
        dt, blk = w["dt"], 20
        deltas, moves_prev, ms = {}, 0, 0.0
        stream = torch.cuda.current_stream()
        for b in range(400 // blk):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for _ in range(blk):
                c.step(dt)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms += ev0.elapsed_time(ev1)
            t = round((b + 1) * blk * dt, 6)
            if t in (1.0, 2.0, 4.0):
                em, _ = c.element_stats()
                kc = 0.5 * float(np.sum(A * (em[:, 4] + em[:, 5] + em[:, 6])) / np.sum(A))
                deltas["t=%g" % t] = (kc - 1.5) / 1.5
        d = c.diag()
        _, cnt = c.element_stats()
        key = "ppe%d_%s" % (ppe, "minnpel%d" % p["minnpel"] if redist else "no_redistribution")
        out["cases"][key] = {"delta": deltas, "moves_per_step": d["moves"] / 400.0,
                             "min_count": int(cnt.min()), "empty_elements": int((cnt == 0).sum()),
                             "lost": d["lost"], "device_errors": c.check(),
                             "particles": c.np_,
                             "value": c.np_ * 400 / (ms * 1e-3), "unit": UNIT}
        c.close()
    return out


def coupled_form(torch, B, w, args):
    """The full coupled step of Table 1 (CG solves included) on the same workload, FP32 state
    with FP64 solves: C_p = dt/2 (Eq. 33 is stable only for C_p < 2 dt), solver tolerance
    1e-6 relative to the load.  Device time of K coupled steps after W, CUDA events on the
    library's stream; the solves read their convergence flags on the host every 16
    iterations, so the time includes those round trips."""
    c = make_ctx(B, w, 1, 0, args.sort_every)
    dt, Cp, tol = w["dt"], 0.5 * w["dt"], 1e-6
    for _ in range(args.warmup):
        c.coupled_step(dt, Cp=Cp, tol=tol, max_iter=20000)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    iters = []
    steps = args.coupled_steps
    ev0.record(stream)
    for _ in range(steps):
        iters.append(c.coupled_step(dt, Cp=Cp, tol=tol, max_iter=20000))
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    np_ = c.np_
    err = c.check()
    c.close()
    return {"what": "full coupled step (Table 1: elliptic relaxation, particle step, pressure "
                    "projection, Eq. 31 correction, statistics), FP32 state, FP64 CG solves",
            "ms_per_step": ms, "value": np_ / (ms * 1e-3), "unit": UNIT, "steps": steps,
            "Cp": Cp, "tol": tol,
            "wp_iterations": [int(a) for a, _ in iters],
            "pressure_iterations": [int(b) for _, b in iters],
            "device_errors": err}


def scalar_post(torch, c, w):
    """Scalar post-processing of Sect. 4.1.2 (Eqs. 67-69) through the C ABI with host
    outputs: the wall time of one call for 64 probe elements at 200 psi bins (the paper's
    point PDFs and conditional curves) and for every element at 50 bins."""
    import numpy as np
    ne = w["grid"].ne
    res = {}
    for name, elems, nb in (("probes64_bins200", np.linspace(0, ne - 1, 64).astype(np.int32), 200),
                            ("all_elements_bins50", np.arange(ne, dtype=np.int32), 50)):
        c.scalar_stats(elems, nb)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            c.scalar_stats(elems, nb)
        el = (time.perf_counter() - t0) / 3
        res[name] = {"ms_per_call": el * 1e3, "probes": int(elems.size), "bins": nb,
                     "particles": c.np_}
    return res


STAT_NAMES = ["N", "U", "V", "W", "uu", "vv", "ww", "uv", "uw", "vw", "omega", "psi", "psi2"]


def _rel_errors(a, b, ref):
    """Relative error per statistic column (floor: the column RMS of the reference; the
    covariances also sqrt(<ii><jj>)): max, RMS and 99th percentile."""
    import numpy as np
    pairs = {7: (4, 5), 8: (4, 6), 9: (5, 6)}
    out = {}
    for j, name in enumerate(STAT_NAMES):
        if j == 0:
            continue
        rms = float(np.sqrt(np.mean(ref[:, j] ** 2))) or 1.0
        den = np.maximum(np.abs(b[:, j]), rms)
        if j in pairs:
            den = np.maximum(den, np.sqrt(np.abs(b[:, pairs[j][0]] * b[:, pairs[j][1]])))
        r = np.abs(a[:, j] - b[:, j]) / den
        out[name] = {"max": float(r.max()), "rms": float(np.sqrt(np.mean(r * r))),
                     "p99": float(np.percentile(r, 99))}
    return out


def _patches(grid, centres):
    """Elements of a few round patches of the grid, centres[k] = (x, y, radius); the interior
    elements (those whose neighbours up to two edges away lie in a patch) and the nodes all
    of whose elements are interior."""
    import numpy as np
    xy = grid.node_xy[grid.tri].mean(axis=1)
    L = grid.period_x
    inside = np.zeros(grid.ne, bool)
    for cx, cy, radius in centres:
        dx = xy[:, 0] - cx
        if L > 0:
            dx = (dx + 0.5 * L) % L - 0.5 * L
        inside |= dx * dx + (xy[:, 1] - cy) ** 2 <= radius * radius
    # element neighbours across edges
    e3 = np.repeat(np.arange(grid.ne), 3)
    a = grid.tri[:, [1, 2, 0]].ravel()
    b = grid.tri[:, [2, 0, 1]].ravel()
    key = np.minimum(a, b).astype(np.int64) * grid.nn + np.maximum(a, b)
    order = np.argsort(key, kind="stable")
    ks, es = key[order], e3[order]
    same = ks[1:] == ks[:-1]
    pairs = np.stack([es[:-1][same], es[1:][same]], axis=1)
    inner = inside.copy()
    for _ in range(2):
        bad = np.zeros(grid.ne, bool)
        bad[pairs[:, 0][~inner[pairs[:, 1]]]] = True
        bad[pairs[:, 1][~inner[pairs[:, 0]]]] = True
        inner &= ~bad
    node_ok = np.ones(grid.nn, bool)
    node_ok[grid.tri[~inner].ravel()] = False
    node_ok[np.setdiff1d(np.arange(grid.nn), grid.tri.ravel())] = False
    return np.where(inside)[0], np.where(inner)[0], np.where(node_ok)[0]


def precision_study(B, w, forms, sample_steps):
    """Forms A/B/C against the FP64 oracle, one step at a time from identical inputs: at each
    sampled step of a run of the form, the particles of round element patches (a wall patch,
    an interior one and one around the scalar source, where psi varies) are handed to the oracle as the form holds them (FP32 values widened
    exactly; the fields rounded to FP32 for the FP32 forms); both take one step; the nodal
    statistics of the nodes whose elements all lie well inside a patch are compared.  The
    differences are those of the form's arithmetic only; particles whose discrete decisions
    differ are counted (element on a shared edge to rounding; a wall decision whose uniform
    and Eq. 53's probability agree to rounding)."""
    import numpy as np
    import oracle
    g = w["grid"]
    P = dict(w["params"], minnpel=0)             # particle-number control is global: off
    # radii that leave about 300, 30 and 30 nodes inside: the graded wall cells are small,
    # the interior ones large
    src = (w["params"]["src_x"], w["params"]["src_y"], 0.1)
    patch, inner, nodes = _patches(g, [(0.7, 0.03, 0.06), (1.3, 0.5, 0.1), src])
    out = {}
    for name, (precision, acc64) in forms.items():
        F = w["fields"] if precision == 0 else w["fields"].astype(np.float32).astype(np.float64)
        c = B.Context(dict(P, precision=precision, acc64=acc64, sort_every=4))
        c.set_grid(g)
        c.set_fields(F)
        c.init_particles(w["ppe"])
        done, errs, nmax = 0, [], {}
        ex_elem = ex_wall = n_cmp = 0
        for s in sample_steps:
            while done < s:
                c.step(w["dt"])
                done += 1
            sg = c.get_particles()
            ids = np.where(np.isin(sg["elem"], patch))[0]
            o = oracle.Oracle(g, P, F)
            o.set_particles({k: sg[k][ids] for k in ("x", "y", "u", "v", "w", "om", "psi", "elem")},
                            c.step_index, pid=ids)
            o.step(w["dt"])
            c.step(w["dt"])
            done += 1
            sg, so = c.get_particles(), o.get_particles()
            ex_elem += int((sg["elem"][ids] != so["elem"]).sum())
            stop_g = (sg["u"][ids] == 0) & (sg["v"][ids] == 0) & (sg["w"][ids] == 0)
            stop_o = (so["u"] == 0) & (so["v"] == 0) & (so["w"] == 0)
            ex_wall += int((stop_g != stop_o).sum())
            ng, no = c.nodal_stats()[nodes], o.nodal_stats()[nodes]
            errs.append(_rel_errors(ng, no, no))
            n_cmp += nodes.size
        c.close()
        for st in STAT_NAMES[1:]:
            nmax[st] = {k: max(e[st][k] for e in errs) for k in ("max", "rms", "p99")}
        out[name] = {"errors": nmax, "nodes_compared": n_cmp, "sampled_steps": list(sample_steps),
                     "exempt_element": ex_elem, "exempt_wall_decision": ex_wall,
                     "patch_elements": int(patch.size)}
    return out


def canyon_form(torch, B, synth, args):
    """The street canyon (cavity [1.5, 2.5] x [0, 1] under a periodic channel [0, 4] x
    [1, 2], 200,000 triangles graded to the walls and cavity corners, 100 particles per
    element, FP32 state): autotuned, whole re-order cycles replayed from a CUDA graph."""
    w = synth.canyon_workload("canyon_200k")
    c = B.Context(dict(w["params"], precision=1, sort_every=args.sort_every))
    c.set_grid(w["grid"])
    c.set_fields(w["fields"])
    c.init_particles(w["ppe"])
    dt = w["dt"]
    c.step(dt)
    tuned = c.autotune(dt) if not args.no_autotune else None
    cycle = 2 * (tuned["sort_every"] if tuned else args.sort_every)
    steps = max(cycle, (args.steps // cycle) * cycle)
    c.step_many(dt, cycle, use_graph=True)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    c.step_many(dt, steps, use_graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # where the time goes: one re-order cycle of eager steps with the stage timers on
    c.set_profiling(True)
    c.stage_times()
    for _ in range(cycle):
        c.step(dt)
    torch.cuda.synchronize()
    stage_ms, stage_n = c.stage_times()
    c.set_profiling(False)
    npart = c.np_
    d = c.diag()
    out = {"value": npart * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
           "steps": steps, "particles": npart, "triangles": int(w["grid"].ne), "ppe": w["ppe"],
           "dtype": "f32", "tuned": tuned, "device_errors": c.check(),
           "stages_ms_per_step": {n: stage_ms[i] / max(stage_n[i], 1) for i, n in enumerate(STAGES)},
           "diag": {k: d[k] for k in ("wall_hits", "freeslip_hits", "moves", "lost", "walk_brute")}}
    c.close()
    torch.cuda.empty_cache()
    return out


def batched_form(torch, B, synth, args):
    """The ensemble of independent instances (32 channel and 32 street-canyon grids of 1k-57k
    triangles at 50-500 particles per element, about 288M particles, FP32 state): one
    context stepping all of
    them with one launch per stage, whole re-order cycles replayed from a CUDA graph; then
    the same instances as 64 contexts stepped one after the other."""
    ins = synth.ensemble(args.batch_instances)
    g, F, ef, nf = synth.union(ins)
    P = [dict(it["params"], precision=1, sort_every=args.sort_every) for it in ins]
    ppe = [it["ppe"] for it in ins]
    dt = 1e-4
    stream = torch.cuda.current_stream()

    def timed(fn):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    b = B.Context(P[0])
    b.set_instances(P, ef)
    b.set_grid(g)
    b.set_fields(F)
    b.init_particles_batch(ppe)
    npart = b.np_
    b.step(dt)
    tuned = b.autotune(dt) if not args.no_autotune else None
    cycle = 2 * (tuned["sort_every"] if tuned else args.sort_every)
    steps = max(cycle, (args.batch_steps // cycle) * cycle)
    b.step_many(dt, cycle, use_graph=True)            # warm-up, includes the capture
    l0 = b.kernel_launches
    ms_b = timed(lambda: b.step_many(dt, steps, use_graph=True))
    launches_b = b.kernel_launches - l0
    err_b = b.check()
    b.close()
    del b
    torch.cuda.empty_cache()

    ctxs = []
    for it, p in zip(ins, P):
        c = B.Context(p)
        c.set_grid(it["grid"])
        c.set_fields(it["fields"])
        c.init_particles(it["ppe"])
        ctxs.append(c)
    for c in ctxs:
        c.step(dt)

    def one_by_one():
        for _ in range(steps):
            B.batch_step(ctxs, dt)

    ms_1 = timed(one_by_one)
    err_1 = max(c.check() for c in ctxs)
    for c in ctxs:
        c.close()
    torch.cuda.empty_cache()
    v_b = npart * steps / (ms_b * 1e-3)
    v_1 = npart * steps / (ms_1 * 1e-3)
    return {"value": v_b, "unit": UNIT, "ms_per_step": ms_b / steps, "steps": steps,
            "instances": len(ins), "particles": npart, "triangles": int(g.ne),
            "ppe_range": [min(ppe), max(ppe)], "dtype": "f32", "graph_cycle_steps": cycle,
            "gpu_launches": launches_b, "device_errors": err_b, "tuned": tuned,
            "one_by_one": {"value": v_1, "ms_per_step": ms_1 / steps, "device_errors": err_1},
            "speedup_vs_one_by_one": v_b / v_1}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="pdfx", choices=["pdfx", "reference"])
    ap.add_argument("--workload", default="channel_50k")
    ap.add_argument("--sort-every", type=int, default=8)
    ap.add_argument("--oracle-ppe", type=int, default=40)
    ap.add_argument("--oracle-steps", type=int, default=2)
    ap.add_argument("--no-f64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-canyon", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-fox", action="store_true")
    ap.add_argument("--no-redist", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the precision study against the oracle (the FP64 form still runs)")
    ap.add_argument("--no-coupled", action="store_true",
                    help="skip the full coupled step (CG solves included)")
    ap.add_argument("--coupled-steps", type=int, default=5)
    ap.add_argument("--batch-instances", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=16)
    ap.add_argument("--ppe", type=int, default=None,
                    help="particles per element (default: the workload's own)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_env()

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1006_0532_gb300 import _binding as B
    from paper_1006_0532_gb300 import synth
    w = synth.workload(args.workload, args.ppe)

    c32, r32 = time_form(torch, B, w, 1, args, rank, world, dist, with_clock=True)
    e2e_s, h2d, d2h = e2e_form(torch, B, c32, w, args)
    rs = scalar_post(torch, c32, w) if rank == 0 else None
    c32.close()
    r64 = rb64 = None
    if not args.no_f64:
        c64, r64 = time_form(torch, B, w, 0, args, rank, world, dist, with_clock=False)
        c64.close()
        # the FP32 form with FP64 accumulation of moments and conditional means
        cb, rb64 = time_form(torch, B, w, 1, args, rank, world, dist, with_clock=False,
                             extra={"acc64": 1})
        cb.close()
    rs8 = None
    if not args.no_sweep:
        # the (2, 2, 2) point of the bins sweep: 8 conditioning bins instead of 64
        cs8, rs8 = time_form(torch, B, w, 1, args, rank, world, dist, with_clock=False,
                             extra={"bins": (2, 2, 2)})
        cs8.close()
    rf = None
    if not args.no_fox:
        # Fox's projection conditioning (Eqs. 64-66) in place of the hierarchical bins, as
        # many intervals as the hierarchical form has bins
        nbins = 1
        for b in w["params"]["bins"]:
            nbins *= b
        cf, rf = time_form(torch, B, w, 1, args, rank, world, dist, with_clock=False,
                           extra={"cond_mode": 1, "fox_bins": nbins})
        cf.close()
        rf["fox_bins"] = nbins
    rb = None
    if not args.no_batch:
        rb = batched_form(torch, B, synth, args)
    rr = None
    if not args.no_redist and rank == 0:
        rr = redistribution_study(torch, B, synth, args)
    rc = None
    if not args.no_canyon:
        rc = canyon_form(torch, B, synth, args)
    rcs = None
    if not args.no_coupled and rank == 0:
        rcs = coupled_form(torch, B, w, args)
    e2e_s = max_over_ranks(torch, dist, e2e_s)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    np_ = r32["np"]
    value = np_ * world * args.steps / (r32["ms"] * 1e-3)
    peak, peak_kind = peaks()
    stage = {n: r32["stage_ms"][i] / max(r32["stage_n"][i], 1) for i, n in enumerate(STAGES)}
    # roofline of the dominant kernel (by time per step): binning or advance
    dom = "statistics_binning" if stage["statistics_binning"] >= stage["advance"] else "advance"
    per_p = BIN_BYTES[1] if dom == "statistics_binning" else ADV_BYTES[1]
    dom_ms = stage[dom]
    achieved = per_p * np_ / (dom_ms * 1e-3) / 1e9
    src_hash = kernel_sources_hash()
    rec = NCU_RECORDS.get(src_hash)
    traffic = rec["traffic"].get(dom) if rec else None
    step_bytes = ADV_BYTES[1] + BIN_BYTES[1]
    step_achieved = step_bytes * np_ * args.steps / (r32["ms"] * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r32["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "triangles": w["grid"].ne, "nodes": w["grid"].nn,
                   "particles_per_gpu": np_, "ppe": w["ppe"], "dt": w["dt"],
                   "form": "FP32 state and SDE arithmetic, FP64 statistics",
                   "l2": "particle state (%.2f GB) larger than L2; grid and fields L2-resident"
                         % (np_ * 45 / 1e9),
                   "sort_every": (r32["tuned"] or {}).get("sort_every", args.sort_every),
                   "advance_block": (r32["tuned"] or {}).get("adv_block", 256),
                   "binning_tile_split": (r32["tuned"] or {}).get("tile_split", 256),
                   "autotuned": r32["tuned"] is not None,
                   "parallelism": "independent instance per GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": traffic * np_ if traffic is not None else None,
                     "traffic_source": ("ncu capture of these sources (DRAM bytes per particle "
                                        "x particles)" if traffic is not None else
                                        "null: no ncu capture of these kernel sources (sha256 %s)"
                                        % src_hash[:16]),
                     "kernel": ("binning: stats_tile_kernel<float> and rank_tile_kernel<float> "
                                 "(three size-class launches per step)"
                                if dom == "statistics_binning" else "advance_kernel<float>"),
                     "algorithmic_bytes_per_particle": per_p, "peak_source": peak_kind,
                     "ms_per_step": dom_ms,
                     "limiter": rec["limiter"].get(dom) if rec else None},
        "step_roofline": {"bytes_per_update": step_bytes, "achieved": step_achieved,
                          "peak": peak, "unit": "GB/s", "frac": step_achieved / peak,
                          "frac_nominal_8000": step_achieved / 8000.0,
                          "frac_at_single_fp32_positions": SINGLE_POSITION_STEP_BYTES * np_ * args.steps
                          / (r32["ms"] * 1e-3) / 1e9 / peak},
        "stages_ms_per_step": stage,
        "stages_gbs": {n: {"algorithmic_bytes_per_particle": bpp,
                           "achieved": bpp * np_ / (stage[n] * 1e-3) / 1e9,
                           "frac_measured": bpp * np_ / (stage[n] * 1e-3) / 1e9 / peak,
                           "frac_nominal_8000": bpp * np_ / (stage[n] * 1e-3) / 1e9 / 8000.0}
                       for n, bpp in (("advance", ADV_BYTES[1]),
                                      ("statistics_binning", BIN_BYTES[1]))},
        "gpu_launches": r32["launches"],
        "e2e": {"value": np_ * world * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "clocks": r32["clocks"],
        "device_errors": r32["err"],
        "diag": {k: r32["diag"][k] for k in ("hops_total", "walk_fallback", "walk_brute", "lost",
                                              "wall_hits", "moves", "capacity_overflow", "nonfinite")},
    }
    if r64 is not None:
        v64 = r64["np"] * world * args.steps / (r64["ms"] * 1e-3)
        line["f64_form"] = {"value": v64, "ms_per_step": r64["ms"] / args.steps,
                            "stages_ms_per_step": {n: r64["stage_ms"][i] / max(r64["stage_n"][i], 1)
                                                   for i, n in enumerate(["advance", "plan", "lists",
                                                                          "redistribute",
                                                                          "statistics_binning",
                                                                          "node_average"])},
                            "device_errors": r64["err"],
                            "diag": {k: r64["diag"][k] for k in ("hops_total", "walk_fallback",
                                                                  "walk_brute", "lost", "wall_hits",
                                                                  "moves")}}
        # the FP64 form's advance is bound by the FP64 pipe: its FP64 instruction rate
        # (instructions per particle from an ncu capture of these sources) against the
        # measured FMA rate of this GPU
        fp64_peak = B.measure_fp64_rate() / 1e12
        adv64_ms = r64["stage_ms"][0] / max(r64["stage_n"][0], 1)
        n64 = rec.get("f64_advance_fp64_inst_per_particle") if rec else None
        line["f64_form"]["roofline"] = {
            "bound": "alu", "pipe": "fp64", "unit": "TFLOP/s", "peak": fp64_peak,
            "peak_source": "measured (pdfx_measure_fp64_rate: independent FMA chains, 2 FLOP each)",
            "kernel": "advance_kernel<double>", "ms_per_step": adv64_ms,
            "achieved": (2.0 * n64 * r64["np"] / (adv64_ms * 1e-3) / 1e12) if n64 else None,
            "frac": (2.0 * n64 * r64["np"] / (adv64_ms * 1e-3) / 1e12 / fp64_peak) if n64 else None,
            "fp64_inst_per_particle": n64,
            "flop_convention": "each FP64 instruction counted as one FMA (2 FLOP), as the probe counts",
            "note": None if n64 else "no ncu capture of these kernel sources: FP64 instructions "
                                     "per particle unknown"}
        line["speedup_f32_vs_f64"] = value / v64
        vB = rb64["np"] * world * args.steps / (rb64["ms"] * 1e-3)
    if r64 is not None and not args.no_precision:
        ps = precision_study(B, w, {"A_fp64": (0, 0), "B_fp32_sde_fp64_accumulation": (1, 1),
                                    "C_fp32_sde_compensated_fp32_accumulation": (1, 0)},
                             sample_steps=(0, 10))
        ps["A_fp64"]["value"], ps["B_fp32_sde_fp64_accumulation"]["value"] = v64, vB
        ps["C_fp32_sde_compensated_fp32_accumulation"]["value"] = value
        line["precision_study"] = {
            "what": "nodal statistics of one step against the FP64 oracle from identical inputs "
                    "(the form's own state at the sampled steps, handed over exactly), on the "
                    "nodes inside a wall patch, an interior patch and a patch around the "
                    "scalar source; relative error per "
                    "statistic (floor: the column RMS; covariances also sqrt(<ii><jj>)), "
                    "max / RMS / 99th percentile over the samples",
            "unit": UNIT, "forms": ps}
    if rs8 is not None:
        line["bins_sweep"] = {
            "what": "FP32 form with (2, 2, 2) conditioning bins against the default (4, 4, 4)",
            "bins_2_2_2": {"value": rs8["np"] * world * args.steps / (rs8["ms"] * 1e-3),
                           "ms_per_step": rs8["ms"] / args.steps,
                           "binning_ms_per_step": rs8["stage_ms"][STAGES.index("statistics_binning")]
                           / max(rs8["stage_n"][STAGES.index("statistics_binning")], 1)},
            "bins_4_4_4": {"value": value, "ms_per_step": r32["ms"] / args.steps,
                           "binning_ms_per_step": stage["statistics_binning"]}}
    if rr is not None:
        line["redistribution_error"] = rr
    if rcs is not None:
        rcs["vs_particle_step"] = rcs["ms_per_step"] / (r32["ms"] / args.steps)
        line["coupled_step"] = rcs
    if rs is not None:
        line["scalar_statistics"] = rs
    if rf is not None:
        vF = rf["np"] * world * args.steps / (rf["ms"] * 1e-3)
        line["fox_form"] = {
            "what": "FP32 form with Fox's projection conditioning (Eqs. 64-66), N_c = %d "
                    "intervals, in place of the hierarchical bins" % rf["fox_bins"],
            "value": vF, "unit": UNIT, "ms_per_step": rf["ms"] / args.steps,
            "stages_ms_per_step": {n: rf["stage_ms"][i] / max(rf["stage_n"][i], 1)
                                   for i, n in enumerate(STAGES)},
            "vs_hierarchical": vF / value, "device_errors": rf["err"]}
    if rc is not None:
        line["street_canyon"] = rc
    if rb is not None:
        line["batched_form"] = rb
        if r64 is not None:
            line["speedup_batched_vs_f64"] = rb["value"] / v64
    if not args.no_cpu:
        cores, model = host_cores()
        n, st, el, _ = oracle_sample(args.workload, args.oracle_steps, args.oracle_ppe)
        na, ela = oracle_parallel(args.workload, args.oracle_ppe, 1, 3, cores)
        line["cpu_baseline"] = {
            "value": na * 3 / ela, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%s grid at %d particles per element (%d particles), 3 steps after 1: %d "
                      "processes of the one-thread oracle over contiguous element shares "
                      "(particle-number control off)" % (args.workload, args.oracle_ppe, na, cores),
            "one_thread": {"value": n * st / el, "unit": UNIT, "cores": 1,
                           "sample": "the same grid and particles per element, %d steps, "
                                     "particle-number control on (MINNPEL %d)" % (st, max(1, args.oracle_ppe // 10))},
            "host": {"cores": cores, "cpu": model},
            "config_differs": "the oracle runs %d particles per element, the GPU arm %d"
                              % (args.oracle_ppe, w["ppe"])}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

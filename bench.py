"""Benchmark of the IB-LBM step on B300: MLUPS and fraction of the HBM roofline.

Workload (default): the fixed-cylinder case matrix on a 2048x1024 lattice
(D = 64 at (0.4 Lx, 0.5 Ly), 201 markers, U = 0.1, Re = 100 and 200) with every
scheme {DF, MDF (5 iterations), DFC} x kernel {hat, Peskin 4-point} x collision
{BGK, TRT (Lambda = 3/16), CM-MRT}: 36 lattices, FP32 shifted populations,
advanced together with one batched launch sequence per step.  A bench step is
one IB-LBM step of every lattice.  The populations (2 x 75.5 MB per lattice,
5.4 GB in all) exceed the 126 MB L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on the host cores instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import faulthandler
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
faulthandler.enable()   # a crash prints the Python stack to stderr

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "MLUPS & % of HBM peak per IB-LBM step; batched cases/s with p50/p99 latency"
UNIT = "MLUPS"
BYTES_PER_LU = {W.F64: 144, W.F32: 72, W.F16S: 36}
# DRAM bytes (read + write) per node of one FP32 stream-collide launch, by (variant,
# operator), and per lattice of the edge launch: ncu --metrics dram__bytes_read.sum,
# dram__bytes_write.sum of two steps of the 12-lattice case (4 lattices per stream-collide
# launch, 12 per edge launch), averaged and divided by nodes or lattices.  A sweep whose
# kernels have no entry here (or changed since) reports traffic null.
SWEEP_DRAM_BYTES_PER_NODE = {(2, W.BGK): (560977408 + 558729216) / 2 / 8388608,
                             (2, W.TRT): (559787776 + 560373760) / 2 / 8388608,
                             (2, W.CMMRT): (560088320 + 560034816) / 2 / 8388608}
EDGE_DRAM_BYTES_PER_LATTICE = (29608192 + 29780736) / 2 / 12
DTYPE = {W.F64: "f64", W.F32: "f32", W.F16S: "f32 compute / f16 storage"}
STORAGE_LABEL = {W.F64: "f64 shifted", W.F32: "f32 shifted", W.F16S: "f16 shifted"}


def matrix_specs(storage=W.F32, res=(100.0, 200.0), nx=2048, ny=1024):
    specs = []
    for re in res:
        for scheme in (W.DF, W.MDF, W.DFC):
            for kernel in (W.HAT, W.PESKIN4):
                for col in (W.BGK, W.TRT, W.CMMRT):
                    specs.append(W.fixed_cylinder_2048(re=re, storage=storage, collision=col, kernel=kernel,
                                                       scheme=scheme, nx=nx, ny=ny, mdf_iters=5))
    return specs


VARIANT_KERNELS = {0: "sc_kernel", 1: "sc_kernel_scalar<NPT=1>", 2: "sc_kernel_scalar<NPT=2>", 3: "sc_kernel_bulk"}


def sweep_name(L, storage) -> str:
    """Kernels of the lattice sweep as tuned: stream-collide variant per operator + edge kernel."""
    parts = []
    for name, col in (("bgk", W.BGK), ("trt", W.TRT), ("cmmrt", W.CMMRT)):
        v = L.kernel_variant(storage, col)[0]
        parts.append("%s:%s" % (name, VARIANT_KERNELS.get(v, "untuned")))
    return "stream-collide sweep (%s) + edge_kernel" % ", ".join(parts)


def sweep_traffic(L, specs):
    """Measured DRAM bytes of one sweep (all stream-collide launches + edge launch) for the
    tuned kernels, or None when a tuned kernel has no capture."""
    if any(s.storage != W.F32 for s in specs):
        return None
    total = 0.0
    for s in specs:
        v = L.kernel_variant(s.storage, s.collision)[0]
        bpn = SWEEP_DRAM_BYTES_PER_NODE.get((v, s.collision))
        if bpn is None or EDGE_DRAM_BYTES_PER_LATTICE is None:
            return None
        total += bpn * s.nodes + EDGE_DRAM_BYTES_PER_LATTICE
    return total


def launches_per_step(specs, L=None) -> int:
    """Kernel launches of one batched step, following the library's launch orders: one IB
    launch per storage type with bodies (body motion folded in; one more before it when a
    lattice holds several DFC bodies and one of them moves) and one stream-collide launch
    per (storage, collision) group.  With one storage type the last stream-collide launch
    also takes the lattice edges and the step end in its tail CTAs (its variant has them:
    the one- or two-node-per-lane kernels) -- unless no body can reach a lattice edge, when
    the edges run beside the IB stage in a launch of their own and a counter launch ends
    the step.  When at most eight bodies,
    all fixed, of one storage type sit on at least 2^20 nodes, the IB stage runs beside the
    sweep and each group's sweep also takes its IB-region segments.  Otherwise add a
    lattice-edge launch per storage type and the step-counter launch (and, in the overlap
    order, an IB-region launch per group with bodies)."""
    storages = {s.storage for s in specs}
    with_bodies = {s.storage for s in specs if s.bodies}
    groups = sorted({(s.storage, s.collision) for s in specs})
    bodies = [(s, b) for s in specs for b in s.bodies]
    fixed = all(b.motion == W.FIXED for _, b in bodies)
    variant = {g: (L.kernel_variant(*g)[0] if L is not None else 2) for g in groups}
    phased = all(v in (1, 2) for v in variant.values())
    large = sum(s.nodes for s in specs) >= (1 << 20)
    prepare = any(sum(1 for b in s.bodies if b.scheme == W.DFC) >= 2 and
                  any(b.motion != W.FIXED for b in s.bodies) for s in specs)
    n = len(with_bodies) + len(groups) + (1 if prepare else 0)
    if len(with_bodies) == 1 and 0 < len(bodies) <= 8 and fixed and phased and large:
        if len(storages) == 1:
            return n
        return n + len({(s.storage, s.collision) for s in specs if s.bodies}) + len(storages) + 1

    def clear(s, b):
        xy = np.asarray(b.xy, dtype=float).reshape(-1, 2)
        m = float(np.max(np.hypot(xy[:, 0] - b.xc, xy[:, 1] - b.yc))) + 4.0 if len(xy) else 4.0
        return (b.motion == W.FIXED and b.xc - m > 1.0 and b.yc - m > 1.0 and b.xc + m < s.nx - 2.0
                and b.yc + m < s.ny - 2.0)

    early = all(clear(s, b) for s, b in bodies) and all(v != 0 for v in variant.values())
    if len(storages) == 1 and variant[groups[-1]] in (1, 2) and not early:
        return n
    return n + len(storages) + 1


def shard(items, rank: int, world: int):
    """Independent cases (lattices, requests) handed to ranks round-robin; no
    data-path exchange is needed between ranks (replicas, weak scaling)."""
    return list(items)[rank::world]


def aggregate(nodes_local: int, steps: int, ms_local: float, dist=None, device="cpu"):
    """Whole-job MLUPS: lattice updates of all ranks over the slowest rank's time."""
    import torch
    t = torch.tensor([ms_local, float(nodes_local)], dtype=torch.float64, device=device)
    if dist is not None:
        mx = t[:1].clone()
        sm = t[1:].clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        ms_max, nodes_all = float(mx.item()), float(sm.item())
    else:
        ms_max, nodes_all = ms_local, float(nodes_local)
    return nodes_all * steps / (ms_max / 1e3) / 1e6, ms_max


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        finally:
            os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(spec, budget_s: float = 15.0):
    """The FP64 oracle as it stands, single thread, on a bounded number of steps
    of one lattice of the workload; returns (MLUPS, steps, seconds)."""
    import oracle  # noqa: F401
    from tests.harness import oracle_case
    c = oracle_case(spec)
    t0 = time.perf_counter()
    c.step(1)
    one = time.perf_counter() - t0
    n = max(1, min(200, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    c.step(n)
    dt = time.perf_counter() - t0
    return spec.nodes * n / dt / 1e6, n, dt


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baselines(budget_s: float):
    """The oracle timed in fresh processes (no GPU context, no other threads of this
    program): one thread, then the all-cores build (OpenMP over its node loops) with
    one thread per core; (single, all_cores) dicts of MLUPS, steps, seconds, threads."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench, workloads as W; "
            "spec = W.fixed_cylinder_2048(re=100.0, storage=W.F64, collision=W.BGK, kernel=W.HAT, scheme=W.DF); "
            "print(json.dumps(bench.cpu_baseline(spec, %r)))" % (ROOT, budget_s))
    cores = os.cpu_count() or 1
    out = []
    for omp in (False, True):
        env = dict(os.environ)
        env.pop("IBLBM_ORACLE_OPENMP", None)
        if omp:
            env["IBLBM_ORACLE_OPENMP"] = "1"
            env["OMP_NUM_THREADS"] = str(cores)
            env["OMP_PROC_BIND"] = "spread"
        else:
            env["OMP_NUM_THREADS"] = "1"
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        if r.returncode != 0:
            raise RuntimeError("oracle baseline failed: " + r.stderr[-500:])
        mlups, n, dt = json.loads(r.stdout.strip().splitlines()[-1])
        out.append({"mlups": mlups, "steps": n, "seconds": dt, "threads": cores if omp else 1})
    return out[0], out[1]


def _pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(math.ceil(q / 100.0 * len(xs))) - 1))
    return xs[k]


def serving_report(L, n_requests=256, steps=2000, tick=100, budget_gb=64.0, seed=0, grids=None):
    """Serving stream of seeded requests (grids 128x64 .. 2048x1024, random
    scheme/kernel/collision, Re in [20, 200], FP32): capacity with every request
    queued at once, then Poisson arrivals at 0.5x and 0.9x that capacity through
    the continuous-batching server, and one case at a time (graph-replayed
    iblbm_step) at 0.5x; p50/p99 time-to-result for each."""
    _, specs, resampled = W.serving_requests(seed=seed, n=n_requests, rate=1.0, steps=steps, grids=grids)
    budget = int(budget_gb * 1e9)

    def run_server(arrivals, graphs=True):
        srv = L.Server(budget, max_slots=128)
        srv.set_graphs(graphs)
        t0 = time.perf_counter()
        pending = list(zip(arrivals, specs))
        ids = []
        done = 0
        while done < len(specs):
            now = time.perf_counter() - t0
            while pending and pending[0][0] <= now:
                ids.append(srv.submit(pending.pop(0)[1], steps))
            if done == len(ids) and pending:
                time.sleep(max(0.0, min(0.01, pending[0][0] - now)))
                continue
            k, _, _ = srv.tick(tick)
            done += k
        wall = time.perf_counter() - t0
        lats, failed, why = [], 0, {}
        for i, sp in zip(ids, specs):
            try:
                lats.append(srv.poll(i, cap=4)[1])
            except L.IblbmError as exc:       # a request whose case went unstable or did not fit
                failed += 1
                key = "%s %dx%d %s/%s/%s tau<%.2f" % (
                    str(exc).split(":")[-1].strip(), sp.nx, sp.ny, ("BGK", "TRT", "CM-MRT")[sp.collision],
                    ("DF", "MDF", "DFC")[sp.bodies[0].scheme], ("hat", "P4")[sp.bodies[0].kernel],
                    math.ceil(sp.tau * 20) / 20)
                why[key] = why.get(key, 0) + 1
        srv.close()
        return {"cases_per_s": len(specs) / wall, "p50_s": _pct(lats, 50), "p99_s": _pct(lats, 99),
                "wall_s": wall, "failed": failed, "failed_kinds": why}

    cap = run_server([0.0] * len(specs))
    rate_cap = cap["cases_per_s"]
    cap_direct = run_server([0.0] * len(specs), graphs=False)
    out = {"requests": len(specs), "steps_per_request": steps, "tau_resampled": resampled,
           "budget_gb": budget_gb, "tick_steps": tick, "capacity": cap,
           "capacity_launch_by_launch": cap_direct,
           "updates_per_s_capacity": sum(sp.nodes for sp in specs) * steps / cap["wall_s"]}
    rng = np.random.default_rng(seed + 1)
    gaps = rng.exponential(1.0, size=len(specs))
    for frac in (0.5, 0.9):
        arr = list(np.cumsum(gaps) / (frac * rate_cap))
        out["rate_%.1fx" % frac] = dict(run_server(arr), rate_per_s=frac * rate_cap)
    # one case at a time, same arrivals as the 0.5x run
    arr = list(np.cumsum(gaps) / (0.5 * rate_cap))
    t0 = time.perf_counter()
    lats, failed = [], 0
    for a, sp in zip(arr, specs):
        now = time.perf_counter() - t0
        if a > now:
            time.sleep(a - now)
        lat = L.Lattice.from_spec(sp)
        lat.step(steps)
        try:
            lat.force_history(0, cap=4)
            lats.append(time.perf_counter() - t0 - a)
        except L.IblbmError:
            failed += 1
        lat.close()
    wall = time.perf_counter() - t0
    out["sequential_0.5x"] = {"cases_per_s": len(specs) / wall, "p50_s": _pct(lats, 50), "p99_s": _pct(lats, 99),
                              "wall_s": wall, "failed": failed}
    return out


def moving_report(L, torch, steps=400):
    """Bodies whose markers move every step (footprint and node lists rebuilt on the
    device each step, DFC lambda_k recomputed): one 1024x512 in-line oscillating
    cylinder (D = 40, KC = 5, DFC, Peskin, FP32) and one 400x1600 channel with two
    settling disks (D = 20, DFC, Peskin, FP32), each stepped alone.  Graph-replayed
    microseconds per step, then the same steps launched one by one with events around
    each launch for the IB share of the step."""
    out = {}
    peak, _ = read_peaks()
    cases = [("osc-1024x512-dfc-p4-f32", W.oscillating_cylinder(storage=W.F32, kernel=W.PESKIN4, scheme=W.DFC)),
             ("sed2-400x1600-dfc-p4-f32", W.sedimentation(two_particles=True, storage=W.F32, kernel=W.PESKIN4,
                                                           scheme=W.DFC))]
    for name, spec in cases:
        lat = L.Lattice.from_spec(spec)
        lat.step(20)
        lat.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st = torch.cuda.current_stream()
        e0.record(st)
        lat.step(steps)
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        lat.sync()
        lat.set_timing(True)
        lat.step(steps)
        stages = lat.stage_timing()
        lat.set_timing(False)
        lat.close()
        per = {k: 1e3 * v[0] / steps for k, v in stages.items()}
        out[name] = {"us_per_step": 1e3 * ms / steps, "mlups": spec.nodes * steps / (ms / 1e3) / 1e6,
                     "hbm_fraction": spec.nodes * steps / (ms / 1e3) * BYTES_PER_LU[spec.storage] / (peak * 1e9),
                     "launch_breakdown_us_per_step": per,
                     "ib_share": per["ib"] / max(1e-9, sum(per.values())), "steps": steps,
                     "bodies": len(spec.bodies)}
    return out


def storage_report(L, torch, steps=20):
    """The same 36-lattice matrix with FP16 and FP64 shifted storage: graph-replayed
    steps timed with CUDA events, MLUPS and the fraction of the HBM bound at each
    storage type's bytes per node (36 B FP16, 144 B FP64)."""
    out = {}
    peak, _ = read_peaks()
    for name, st in (("f16", W.F16S), ("f64", W.F64)):
        specs = matrix_specs(storage=st)
        lats = [L.Lattice.from_spec(s) for s in specs]
        nodes = sum(s.nodes for s in specs)
        L.step_batch(lats, 3)
        for l in lats:
            l.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream()
        e0.record(stream)
        L.step_batch(lats, steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        rc = max(l.sync() for l in lats)
        for l in lats:
            l.close()
        mlups = nodes * steps / (ms / 1e3) / 1e6
        out[name] = {"mlups": mlups, "ms_per_step": ms / steps, "steps": steps, "status": rc,
                     "hbm_fraction": mlups * 1e6 * BYTES_PER_LU[st] / (peak * 1e9),
                     "kernel_variants": {cn: L.kernel_variant(st, col) for cn, col in
                                         (("bgk", W.BGK), ("trt", W.TRT), ("cmmrt", W.CMMRT))}}
    return out


def single_case_report(L, torch, steps=2000, only_large=False):
    """One lattice stepped alone (graph-replayed iblbm_step): the 200x100 Re=20
    cylinder (DF, hat, BGK) in FP64 and FP32, and one 2048x1024 lattice of the
    matrix (DF, Peskin, BGK, FP32).  Small lattices are latency-bound, so these
    are reported as microseconds per step beside MLUPS."""
    out = {}
    peak, _ = read_peaks()
    cases = [("cyl-re20-200x100-f64", W.fixed_cylinder_re20(storage=W.F64), steps),
             ("cyl-re20-200x100-f32", W.fixed_cylinder_re20(storage=W.F32), steps),
             ("cyl-re100-2048x1024-f32", W.fixed_cylinder_2048(re=100.0, storage=W.F32, collision=W.BGK,
                                                               kernel=W.PESKIN4, scheme=W.DF), steps // 4)]
    if only_large:
        cases = cases[-1:]
    for name, spec, n in cases:
        lat = L.Lattice.from_spec(spec)
        lat.step(20)
        lat.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st = torch.cuda.current_stream()
        e0.record(st)
        lat.step(n)
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        lat.sync()
        # per-launch breakdown: the same steps launched one by one with CUDA events around
        # each launch (no overlap between the IB stage and the sweep in this mode)
        m = min(n, 200)
        lat.set_timing(True)
        lat.step(m)
        stages = lat.stage_timing()
        lat.set_timing(False)
        lat.close()
        out[name] = {"us_per_step": 1e3 * ms / n, "mlups": spec.nodes * n / (ms / 1e3) / 1e6, "steps": n,
                     "hbm_fraction": spec.nodes * n / (ms / 1e3) * BYTES_PER_LU[spec.storage] / (peak * 1e9),
                     "launch_breakdown_us_per_step": {k: 1e3 * v[0] / m for k, v in stages.items()},
                     "launches_per_step": launches_per_step([spec], L)}
    return out


def workload_config(specs, world=1):
    """The `config` object both arms print for the same workload."""
    nx, ny = specs[0].nx, specs[0].ny
    nodes = sum(s.nodes for s in specs)
    return {"workload": ("fixed-cylinder matrix %dx%d, D=%g, %d markers: Re {100,200} x "
                         "{DF, MDF(5), DFC} x {hat, P4} x {BGK, TRT, CM-MRT}" %
                         (nx, ny, specs[0].bodies[0].radius * 2, len(specs[0].bodies[0].xy))),
            "lattices": len(specs), "nodes_per_step": nodes,
            "storage": STORAGE_LABEL[specs[0].storage],
            "l2": "populations %.1f GB (A/B buffers) > 126 MB L2, no flush"
                  % (BYTES_PER_LU[specs[0].storage] * nodes / 1e9),
            "parallelism": "replicas" if world > 1 else "single"}


def run_reference(args, specs):
    """--impl reference: the oracle timed on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    spec = specs[0] if not args.small else specs[0]
    per_step = []
    for _ in range(args.warmup):
        cpu_baseline(spec, budget_s=0.5)
    tot_nodes, tot_time = 0, 0.0
    for _ in range(args.steps):
        mlups, n, dt = cpu_baseline(spec, budget_s=args.ref_budget)
        per_step.append(dt)
        tot_nodes += spec.nodes * n
        tot_time += dt
    value = tot_nodes / tot_time / 1e6
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_time / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": workload_config(specs),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu_model": cpu_model(),
                             "sample": "each step = %.1f s of FP64 oracle steps on one %dx%d lattice of the "
                                       "matrix (%s), scaled to lattice updates per second"
                                       % (args.ref_budget, spec.nx, spec.ny, spec.name)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--small", action="store_true", help="256x128 lattices (quick check, not a bench number)")
    ap.add_argument("--cpu-budget", type=float, default=15.0,
                    help="seconds of oracle time for the CPU baseline (0: not reported)")
    ap.add_argument("--ref-budget", type=float, default=5.0)
    ap.add_argument("--lattices", type=int, default=0,
                    help="use only the first K lattices of the matrix (profiling a smaller case)")
    ap.add_argument("--serving-requests", type=int, default=256,
                    help="requests in the serving stream (0: not reported)")
    ap.add_argument("--e2e-chunks", type=int, default=3,
                    help="lattice chunks of the end-to-end leg (copy-in of one overlaps the steps of the last)")
    ap.add_argument("--kernel-variant", type=int, default=-1,
                    help="fix the stream-collide variant (0-3) instead of tuning it (profiling)")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "f64"],
                    help="population storage of the matrix (the bench line is FP32; others for profiling)")
    ap.add_argument("--single", action="store_true",
                    help="only the single-lattice report (one 2048x1024 lattice alone; profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    nx, ny = (256, 128) if args.small else (2048, 1024)
    specs = matrix_specs(storage=W.STORAGES[args.storage], nx=nx, ny=ny) if not args.small else [
        W.fixed_cylinder_2048(re=re, storage=W.F32, collision=c, kernel=k, scheme=s, nx=nx, ny=ny,
                              diameter=16.0, nmark=50, mdf_iters=5)
        for re in (100.0, 200.0) for s in (W.DF, W.MDF, W.DFC) for k in (W.HAT, W.PESKIN4)
        for c in (W.BGK, W.TRT, W.CMMRT)]
    if args.lattices > 0:
        specs = specs[:args.lattices]
    if args.impl == "reference":
        run_reference(args, specs)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import paper_2609_02298_b300 as L
    L.use_torch_allocator()
    if args.kernel_variant >= 0:
        for col in (W.BGK, W.TRT, W.CMMRT, W.STREAM_ONLY):
            L.set_kernel_variant(specs[0].storage, col, args.kernel_variant)
    if args.single:
        out = single_case_report(L, torch, steps=4 * args.steps, only_large=True)
        out["kernel_variant_bgk_f32"] = L.kernel_variant(W.F32, W.BGK)
        print(json.dumps(out), flush=True)
        return
    lats = [L.Lattice.from_spec(s) for s in specs]
    nodes = sum(s.nodes for s in specs)
    storage = specs[0].storage

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up (graph capture happens here)
    L.step_batch(lats, args.warmup)
    for l in lats:
        l.sync()
    # timed region: CUDA events on the launching stream (graph-replayed steps)
    lead = lats[0]
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        gpu_id = str(local)
    with ClockSampler(gpu_id) as clocks:
        e0.record(stream)
        L.step_batch(lats, args.steps)
        e1.record(stream)
        e1.synchronize()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    for l in lats:
        rc = l.sync()
    value, ms_max = aggregate(nodes, args.steps, ms, dist, device="cuda")

    # roofline of the dominant kernel: the lattice sweep (stream-collide launches,
    # one per collision group, plus the lattice-edge launch) timed with CUDA events
    # on the launching stream over the same number of steps, launched one by one
    lead.set_timing(True)
    barrier()
    L.step_batch(lats, args.steps)
    for l in lats:
        l.sync()
    sc_ms, sc_n = lead.kernel_timing()
    lead.set_timing(False)
    peak, peak_kind = read_peaks()
    # together the sweep launches move 72 B per node of every lattice once per step
    sc_avg_s = sc_ms / max(1, sc_n) / 1e3
    alg_bytes = BYTES_PER_LU[storage] * nodes
    achieved = alg_bytes * args.steps / (sc_ms / 1e3) / 1e9 if sc_n else None

    # end to end through the public API from pinned host buffers: restore every lattice
    # from its host checkpoint (the inputs), run the steps, read back the result (the
    # force history of every body: the drag and lift the method is run for).  The
    # lattices go in chunks, one batch each: a restore waits only for its own lattice,
    # so chunk k+1 is copied in while chunk k runs
    bufs = [torch.empty(l.snapshot_bytes(), dtype=torch.uint8, pin_memory=True) for l in lats]
    for l, b in zip(lats, bufs):
        l.snapshot(out=b)
    h2d = sum(b.numel() for b in bufs)
    nch = max(1, min(args.e2e_chunks, len(lats)))
    chunks = [list(range(len(lats)))[k::nch] for k in range(nch)]
    for ch in chunks:     # build each chunk's batch plan and graphs before the clock starts
        L.step_batch([lats[i] for i in ch], 1)
    for l in lats:
        l.sync()
    barrier()
    t0 = time.perf_counter()
    for ch in chunks:
        for i in ch:
            lats[i].restore(bufs[i])
        L.step_batch([lats[i] for i in ch], args.steps)
    d2h = 0
    for l in lats:
        hist = l.force_history(0, cap=args.steps)
        d2h += hist.nbytes
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = nodes * args.steps * world / e2e_s / 1e6

    for l in lats:
        l.close()
    single = None
    if rank == 0 and not args.small and args.serving_requests > 0:
        try:
            single = single_case_report(L, torch)
        except Exception as exc:
            single = {"error": repr(exc)}
    moving = None
    if rank == 0 and args.serving_requests > 0 and not args.small:
        try:
            moving = moving_report(L, torch)
        except Exception as exc:
            moving = {"error": repr(exc)}
    storages = None
    if rank == 0 and args.serving_requests > 0 and not args.small:
        try:
            storages = storage_report(L, torch)
        except Exception as exc:
            storages = {"error": repr(exc)}
    serving = None
    if rank == 0 and args.serving_requests > 0 and not args.small:
        try:
            serving = serving_report(L, n_requests=args.serving_requests)
        except Exception as exc:      # the headline line is printed whatever happens here
            serving = {"error": repr(exc)}
    if rank == 0:
        cpu = None
        if not args.small and args.cpu_budget > 0:
            try:
                one, allc = cpu_baselines(args.cpu_budget)
                cpu = {"value": one["mlups"], "unit": UNIT, "cores": 1, "kind": "oracle",
                       "sample": "%d steps of one 2048x1024 lattice (DF, hat, BGK, FP64), %.1f s, fresh process"
                                 % (one["steps"], one["seconds"]),
                       "cpu_model": cpu_model(),
                       "all_cores": {"value": allc["mlups"], "cores": allc["threads"],
                                     "sample": "%d steps of the same lattice, %.1f s, OpenMP over the oracle's "
                                               "node loops" % (allc["steps"], allc["seconds"])}}
            except Exception as exc:
                cpu = {"error": repr(exc)}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[storage], "data": "synthetic",
            "config": workload_config(specs, world),
            "hbm_fraction": (value * 1e6 * BYTES_PER_LU[storage] / (peak * 1e9)),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None,
                         "traffic": sweep_traffic(L, specs), "traffic_per": "step (sweep launches)",
                         "peak_kind": peak_kind, "kernel": sweep_name(L, storage),
                         "bytes_per_step": alg_bytes, "launches": sc_n,
                         "launches_per_step": sc_n / args.steps, "avg_launch_ms": sc_avg_s * 1e3,
                         "sc_ms_per_step": sc_ms / args.steps},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
                    "d2h_bytes_per_step": d2h / args.steps, "chunks": nch},
            "kernel_variants": {name: L.kernel_variant(storage, col) for name, col in
                                (("bgk", W.BGK), ("trt", W.TRT), ("cmmrt", W.CMMRT))},
            "gpu_launches": launches_per_step(specs, L) * args.steps,
            "clocks": clocks.summary(),
            "device_status": rc,
            "single_lattice": single,
            "moving_body": moving,
            "other_storage": storages,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

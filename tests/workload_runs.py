"""Runs of the moving-body workloads at their stated sizes, through the library on
one B300, with the device FP64 storage mode (equal to the oracle to 1e-12 in the
parity suite) standing in for the oracle at sizes it cannot run:

* the in-line oscillating cylinder (Sec. 2.9.2 shape): 1024 x 512, D = 40, KC = 5,
  Re = 100 at U_max = 0.1, open sides, markers moved every step, {DF, MDF, DFC} x
  {hat, Peskin}, BGK, in FP64, FP32 and shifted-FP16 storage: the C_d history of the
  narrow storages against FP64 over periods 3-10 (20,000 steps);
* sedimentation in the 400 x 1600 walled channel (Sec. 2.9.3 shape): D = 20, one disk
  (rho_s/rho_f 1.5) and two disks (1.5 below 1.01, 2 D apart), DFC + Peskin, BGK, FP64
  Newton-Euler, internal-mass increment on and off, FP32 against FP64 storage: the
  settling velocity v* = max |v_y| / u_g, u_g = sqrt(|rho_r - 1| g D), until a disk is
  within 2 D of the bottom wall or 60,000 steps.

Usage: python tests/workload_runs.py --oscillating | --sedimentation [--steps N] [--out F]."""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import workloads as W  # noqa: E402

SCHEME_NAMES = {W.DF: "DF", W.MDF: "MDF", W.DFC: "DFC"}
KERNEL_NAMES = {W.HAT: "hat", W.PESKIN4: "P4"}
STORAGE_NAMES = {W.F64: "f64", W.F32: "f32", W.F16S: "f16"}


def run_oscillating(L, steps=20000, storages=(W.F64, W.F32, W.F16S), schemes=(W.DF, W.MDF, W.DFC),
                    kernels=(W.HAT, W.PESKIN4), skip_periods=2):
    """C_d(t) = F_x / (rho_f U_max^2 D / 2) of every case in every storage type, one batch;
    returns rows with the peak |C_d| (FP64) and, per narrow storage, the largest
    deviation from the FP64 history over the periods after the first ``skip_periods``
    (relative to the peak), its rms, and the peak |C_d| of that storage."""
    specs = []
    for st in storages:
        for sch in schemes:
            for ker in kernels:
                specs.append(W.oscillating_cylinder(storage=st, kernel=ker, scheme=sch, steps=steps))
    lats = [L.Lattice.from_spec(s) for s in specs]
    L.step_batch(lats, steps)
    hist = {}
    for s, lat in zip(specs, lats):
        b = s.bodies[0]
        lat.sync()
        h = lat.force_history(0, cap=steps)
        scale = 0.5 * 0.1 ** 2 * 40.0
        hist[(s.storage, b.scheme, b.kernel)] = h[:, 0] / scale
        lat.close()
    period = int(round(5.0 * 40.0 / 0.1))
    t0 = skip_periods * period
    rows = []
    for sch in schemes:
        for ker in kernels:
            ref = hist[(W.F64, sch, ker)][t0:]
            row = {"scheme": SCHEME_NAMES[sch], "kernel": KERNEL_NAMES[ker], "steps": steps,
                   "cd_peak_f64": float(np.abs(ref).max()), "cd_rms_f64": float(np.sqrt((ref ** 2).mean()))}
            for st in storages:
                if st == W.F64:
                    continue
                d = hist[(st, sch, ker)][t0:] - ref
                row["dcd_max_rel_%s" % STORAGE_NAMES[st]] = float(np.abs(d).max() / np.abs(ref).max())
                row["dcd_rms_rel_%s" % STORAGE_NAMES[st]] = float(np.sqrt((d ** 2).mean()) / np.abs(ref).max())
                row["cd_peak_%s" % STORAGE_NAMES[st]] = float(np.abs(hist[(st, sch, ker)][t0:]).max())
            rows.append(row)
    return rows


def run_sedimentation(L, steps=60000, sample=100, storages=(W.F64, W.F32)):
    """The 400 x 1600 settling cases (one and two disks, internal mass on and off) in
    FP64 and FP32 storage, one batch; v* of every disk and the FP32 error against FP64."""
    g, D, nu = 8.33e-5, 20.0, (0.65 - 0.5) / 3.0
    cases = []
    for two in (False, True):
        for im in (1, 0):
            for st in storages:
                spec = W.sedimentation(two_particles=two, storage=st, internal_mass=im, kernel=W.PESKIN4,
                                       scheme=W.DFC)
                cases.append({"two": two, "internal_mass": im, "storage": st, "spec": spec,
                              "lat": L.Lattice.from_spec(spec), "vy": [[] for _ in spec.bodies],
                              "y": [[] for _ in spec.bodies], "stopped": False})
    done = 0
    while done < steps and not all(c["stopped"] for c in cases):
        live = [c for c in cases if not c["stopped"]]
        L.step_batch([c["lat"] for c in live], sample)
        done += sample
        for c in live:
            try:
                for b in range(len(c["spec"].bodies)):
                    st = c["lat"].body_state(b)
                    c["vy"][b].append(float(st[3]))
                    c["y"][b].append(float(st[1]))
                if min(yb[-1] for yb in c["y"]) < 2.5 * D + 1.0:   # 2 D of gap below the disk
                    c["stopped"], c["stop_step"] = True, done
            except Exception as exc:
                c["stopped"], c["error"], c["error_step"] = True, str(exc), done
    rows = []
    for c in cases:
        c["lat"].close()
        bodies = c["spec"].bodies
        r = {"particles": len(bodies), "internal_mass": "B-2" if c["internal_mass"] else "A",
             "storage": STORAGE_NAMES[c["storage"]], "steps": c.get("stop_step", done)}
        if "error" in c:
            r["error"], r["error_step"] = c["error"], c["error_step"]
        for b, body in enumerate(bodies):
            vy = np.array(c["vy"][b])
            ug = math.sqrt(abs(body.rho_ratio - 1.0) * g * D)
            r["v_star_%d" % b] = float(np.abs(vy).max() / ug) if len(vy) else None
            r["re_f_max_%d" % b] = float(np.abs(vy).max() * D / nu) if len(vy) else None
            r["rho_ratio_%d" % b] = body.rho_ratio
        rows.append(r)
    # FP32 against FP64 of the same case
    for r in rows:
        if r["storage"] == "f64":
            continue
        ref = [q for q in rows if q["storage"] == "f64" and q["particles"] == r["particles"]
               and q["internal_mass"] == r["internal_mass"]][0]
        for b in range(r["particles"]):
            if r.get("v_star_%d" % b) and ref.get("v_star_%d" % b):
                r["v_star_err_%d" % b] = r["v_star_%d" % b] / ref["v_star_%d" % b] - 1.0
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--oscillating", action="store_true")
    ap.add_argument("--sedimentation", action="store_true")
    ap.add_argument("--steps", type=int, default=0)
    ap.add_argument("--out", default="workload_runs.json")
    args = ap.parse_args()
    import paper_2609_02298_b300 as L
    L.use_torch_allocator()
    rows = []
    if args.oscillating:
        rows += run_oscillating(L, steps=args.steps or 20000)
    if args.sedimentation:
        rows += run_sedimentation(L, steps=args.steps or 60000)
    for r in rows:
        print(json.dumps(r), flush=True)
    os.makedirs(os.path.dirname(args.out) or ".", exist_ok=True)
    with open(args.out, "w") as fh:
        json.dump(rows, fh)


if __name__ == "__main__":
    main()

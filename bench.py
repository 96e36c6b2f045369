#!/usr/bin/env python
"""Benchmark of the direct-sum Hermite force engine on one GB300 (or N replicas).

Workload (default, the precision configuration): a Plummer sphere of
N = 2^20 equal-mass particles, eps = 1/4096, shared block step dt = 2^-10 so
that every block step is a full i = j evaluation.  One "step" is one whole
block step of the hot path through the C ABI (nb_step): block selection,
prediction of all N, mixed-precision forces on all N active particles from
all N (N^2 = 1.1e12 pairwise interactions), Hermite correction and new steps.

Printed (rank 0, one JSON line): interactions/s over the timed steps (all
ranks), the force kernel's roofline against the FP32 CUDA-core peak
(152 SMs x 128 lanes x 2 flop x 2070 MHz, 60 flop per interaction), an
end-to-end number through the same C ABI with host buffers (H2D of the step's
inputs and D2H of its results inside the timed region), the FP64 GPU path on
the same state, the mixed path's error against the FP64 oracle on sampled
particles, and the oracle timed on the host cores (cpu_baseline).

``--impl reference`` times the oracle (the plain FP64 CPU direct sum) on the
host cores for the same metric on a bounded sample of the same workload.
Multi-GPU (torchrun): independent replicas, one per GPU; max time over ranks.
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FLOP_PER_INTERACTION = 60
SM_MAX_MHZ_FALLBACK = 2070.0
METRIC = "force interactions/s"
UNIT = "interactions/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1 << 20, help="particles (default 2^20)")
    ap.add_argument("--eps", type=float, default=1.0 / 4096)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--cpu-sample", type=int, default=16384,
                    help="sampled i for the oracle legs (the reference arm takes a quarter per step)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--strict-steps", type=int, default=2,
                    help="block steps timed again with the far-tile pass off (roofline_strict; 0 = skip)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--tuning", default="", help="force launch override ipt,threads,jtile,nsplit (0 = auto)")
    ap.add_argument("--workload", default="c3",
                    choices=["c3", "c2", "c4", "c5", "tapp", "c3sweep", "c4init"],
                    help="c3 (default): the timed benchmark; c2/c4/c5: long integrations; tapp: time per "
                         "N-body time unit vs N and the per-task model; one JSON line each")
    ap.add_argument("--tune-file", default="",
                    help="c3sweep / c4: save the autotuned table to this JSON file (c3sweep adds to it)")
    ap.add_argument("--sweep-n", default="",
                    help="c3sweep: active-block sizes to run (comma list; default the whole sweep)")
    ap.add_argument("--tapp-sizes", default="1024,2048,4096,8192,16384,32768,65536,131072,196608")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, device="cpu"):
    """The largest value of x over all ranks (x itself with one rank)."""
    if ws <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, ws, t_max_s):
    """Units processed by all replicas divided by the slowest rank's time."""
    return float(units_per_rank) * ws / t_max_s


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def sec41_taus(t_pred, t_force, t_corr, N, steps, interactions, particle_steps):
    """Per-unit costs of Sec. 4.1 from measured phase times: t_pred = tau_pred N per
    block step (Eq. 2), t_force = tau_force n N (Eq. 3), t_corr = tau_corr n (Eq. 4),
    summed over the steps (interactions = sum n N, particle_steps = sum n)."""
    return t_pred / (steps * N), t_force / interactions, t_corr / particle_steps


def sec41_T(taus, N, steps, interactions, particle_steps):
    """Eq. 1: T_integrate = sum over the block steps of (tau_pred N + tau_force n N +
    tau_corr n), written with the sums of n N and n over the steps."""
    tau_pred, tau_force, tau_corr = taus
    return tau_pred * N * steps + tau_force * interactions + tau_corr * particle_steps


def fp32_peak_tflops(sms, mhz):
    return sms * 128 * 2 * mhz * 1e6 / 1e12


# the committed ncu record (JSON beside its Markdown summary) of the mixed force
# kernel on this benchmark's full launch; its DRAM bytes count only while the
# kernel source is the one profiled
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "force_mixed_kernel_bench_n1048576.json")
KERNEL_SOURCES = ("paper_0709_4552_gb300/csrc/force_common.cuh", "paper_0709_4552_gb300/csrc/force_mixed.cu")


def kernel_source_digest():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(n):
    """DRAM bytes (read + write) of one mixed force launch over all n particles, from
    the committed ncu record, or None when there is none for n or the kernel changed."""
    try:
        with open(TRAFFIC_PROFILE) as f:
            rec = json.load(f)
        if int(rec["particles"]) != n or rec["kernel_source_sha256_16"] != kernel_source_digest():
            return None
        return int(rec["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError, TypeError):
        return None


def measured_hbm_gbs():
    """The measured copy bandwidth of this GPU model (MEASURED_PEAKS.json at the repo root)."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0  # the fallback figure of an earlier GB300 measurement


def run_reference(args, ws, rank):
    """The oracle (plain FP64 CPU direct sum) on a bounded sample of the workload."""
    if rank != 0:
        return
    import oracle
    from paper_0709_4552_gb300 import inputs
    oracle.build()
    m, x, v = inputs.plummer(args.n, args.seed)
    k = max(1, min(args.cpu_sample // 4, args.n))
    idx = inputs.sample_indices(args.n, k, args.seed + 1000)
    for _ in range(args.warmup):
        oracle.forces(m, x, v, args.eps, idx=idx[: max(1, k // 8)])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.forces(m, x, v, args.eps, idx=idx)
    dt = time.perf_counter() - t0
    inter = float(k) * args.n * args.steps
    val = inter / dt
    cores = oracle.max_threads()
    sample = f"{k} sampled active particles x all N={args.n} j per step (of the N x N block step)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Plummer sphere)",
        "config": workload_config(args),
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def workload_config(args):
    return {"workload": f"Plummer sphere N={args.n}, equal masses, eps=1/{round(1 / args.eps)}, "
                        f"shared dt=2^-10 (every block step is a full i=j step of {args.precision} forces)",
            "N": args.n, "n_active": args.n, "eps": args.eps, "precision": args.precision, "seed": args.seed,
            "l2": f"block-step arrays {args.n * 336 / 1e9:.3g} GB (state, prediction, j-store, results); "
                  "L2 (126 MB) flushed by a 512 MB write before every timed step"}


def run_integration(args):
    """Long block-step integrations of the other configurations (one GPU, one
    JSON line each; not the headline metric):
      c2: N=196608 Salpeter, eps=1/1024, eta=0.01, dt 2^-22..2^-3, FP64, to t=1/8;
      c4: 512 clusters (N_c log-uniform 256..16384, seed 7, Salpeter,
          eps_c=1/(4 N_c^(1/3))), mixed, to t=1/16: one CUDA-graph launch vs
          per-cluster launches;
      c5: N=2^22 Salpeter, eps=1/8192, mixed, to t=1/64 (wall x 64 = N-body time unit)."""
    import torch
    import oracle
    from paper_0709_4552_gb300 import build, inputs
    build.build()
    oracle.build()
    from paper_0709_4552_gb300 import nbody as nb
    torch.cuda.set_device(0)
    w = args.workload

    def rel(a, b):
        return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)

    if w in ("c2", "c5"):
        if w == "c2":
            N, eps, t_end, seed, prec = 196608, 1.0 / 1024, 0.125, 2, nb.NB_FP64
        else:
            N, eps, t_end, seed, prec = 1 << 22, 1.0 / 8192, 1.0 / 64, 5, nb.NB_MIXED
        m, x, v = inputs.plummer(N, seed, "salpeter")
        s = nb.NBody(N, prec, 0)
        s.set_params(eps, 0.01, 2.0 ** -22, min(0.125, t_end))
        s.set_j_particles(0, m, x, v)
        s.initial_forces_and_dt()
        k0, w0 = s.energy()
        s.get_timings(reset=True)
        c0 = s.get_counters()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # c2 (FP64, many small blocks): the CUDA-graph loop; c5 (mixed, large blocks): the
        # host-driven loop, whose force launches use the spatial j-order
        s.integrate(t_end, use_graph=(w == "c2"))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        tim = s.get_timings()
        c1 = s.get_counters()
        k1, w1 = s.energy()
        st = s.get_particles(0, N)
        k = 4096 if w == "c2" else 2048
        idx = inputs.sample_indices(N, k, seed + 1000).astype(np.int32)
        s.predict(t_end)
        a, j, p = s.compute_forces(idx)
        s.close()
        ar, jr, pr = oracle.forces(st["m"], st["x"], st["v"], eps, idx=idx.astype(np.int64), compensated=True)
        out = {"workload": w, "N": N, "eps": eps, "t_end": t_end,
               "precision": "fp64" if prec == nb.NB_FP64 else "mixed",
               "interactions": tim["interactions"], "wall_s": wall,
               "interactions_per_s": tim["interactions"] / wall,
               "gflops_60": tim["interactions"] / wall * FLOP_PER_INTERACTION / 1e9,
               "block_steps": c1["block_steps"] - c0["block_steps"],
               "energy_drift": abs((k1 + w1) - (k0 + w0)) / abs(k0 + w0),
               "final_state_forces_vs_oracle": {
                   "sample": k, "acc_median": float(np.median(rel(a, ar))), "acc_max": float(rel(a, ar).max()),
                   "jerk_median": float(np.median(rel(j, jr))), "jerk_max": float(rel(j, jr).max()),
                   "pot_max": float((np.abs(p - pr) / np.abs(pr)).max())}}
        if w == "c5":
            out["wall_per_nbody_time_unit_s_extrapolated"] = wall / t_end
        print(json.dumps(out), flush=True)
        return

    if w == "c4init":
        # configuration 4's clusters, all particles at once (the persistent force kernel on one
        # full force evaluation per cluster, launched outside the graph): a short case for
        # profiling the batched kernel
        sizes = inputs.ensemble_sizes(512, 256, 16384, seed=7)
        off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        eps = 1.0 / (4.0 * sizes.astype(np.float64) ** (1.0 / 3.0))
        parts = [inputs.plummer(int(n), 10000 + q, "salpeter") for q, n in enumerate(sizes)]
        m = np.concatenate([p[0] for p in parts])
        x = np.concatenate([p[1] for p in parts])
        v = np.concatenate([p[2] for p in parts])
        e = nb.Ensemble(off, eps, nb.NB_MIXED, 0)
        e.set_params(0.01, 0.01, 2.0 ** -22, 1.0 / 16)
        e.set_j_particles(0, m, x, v)
        walls = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e.initial_forces_and_dt()
            torch.cuda.synchronize()
            walls.append(time.perf_counter() - t0)
        inter = float((sizes.astype(np.float64) ** 2).sum())
        e.close()
        print(json.dumps({"workload": "c4init", "clusters": 512, "N_total": int(off[-1]),
                          "interactions": inter, "wall_s": walls,
                          "interactions_per_s": inter / min(walls[1:])}), flush=True)
        return

    if w == "c4":
        sizes = inputs.ensemble_sizes(512, 256, 16384, seed=7)
        off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        eps = 1.0 / (4.0 * sizes.astype(np.float64) ** (1.0 / 3.0))
        parts = [inputs.plummer(int(n), 10000 + q, "salpeter") for q, n in enumerate(sizes)]
        m = np.concatenate([p[0] for p in parts])
        x = np.concatenate([p[1] for p in parts])
        v = np.concatenate([p[2] for p in parts])
        t_end = 1.0 / 16
        res = {}
        finals = {}
        drift64 = None
        tuned = None
        for mode, prec, name in ((nb.NB_ENSEMBLE_PERSISTENT, nb.NB_MIXED, "persistent_graph"),
                                 (nb.NB_ENSEMBLE_PERSISTENT, nb.NB_MIXED, "persistent_graph_autotuned"),
                                 (nb.NB_ENSEMBLE_PER_CLUSTER, nb.NB_MIXED, "per_cluster_launches"),
                                 (nb.NB_ENSEMBLE_PERSISTENT, nb.NB_FP64, "persistent_graph_fp64")):
            e = nb.Ensemble(off, eps, prec, 0)
            e.set_params(0.01, 0.01, 2.0 ** -22, t_end)
            e.set_j_particles(0, m, x, v)
            e.initial_forces_and_dt()
            if name == "persistent_graph":
                e.tune_clear()   # the default item shape (a table from NB_TUNE_FILE is not used here)
            if name == "persistent_graph_autotuned":
                # the item shape timed on 16 block steps of this ensemble's own state (restored),
                # outside the timed run; the table is saved when --tune-file names a path
                t0 = time.perf_counter()
                tuned = e.autotune(16)
                tuned["tuning_wall_s"] = time.perf_counter() - t0
                if args.tune_file:
                    e.tune_save(args.tune_file)
            if name != "per_cluster_launches":
                ek0_, ep0_ = e.energy()
                if prec == nb.NB_MIXED:
                    ek0, ep0 = ek0_, ep0_
            e.get_timings(reset=True)
            c0 = e.get_counters()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e.integrate(t_end, mode)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            tim = e.get_timings()
            c1 = e.get_counters()
            if name == "persistent_graph":
                ek1, ep1 = e.energy()
            if name == "persistent_graph_fp64":
                ek1_, ep1_ = e.energy()
                drift64 = np.abs((ek1_ + ep1_) - (ek0_ + ep0_)) / np.abs(ek0_ + ep0_)
            finals[name] = e.get_particles(0, int(off[-1]))
            e.close()
            res[name] = {"wall_s": wall, "interactions": tim["interactions"],
                         "interactions_per_s": tim["interactions"] / wall,
                         "kernel_launches": c1["kernel_launches"] - c0["kernel_launches"],
                         "block_steps": c1["block_steps"] - c0["block_steps"]}
        drift = np.abs((ek1 + ep1) - (ek0 + ep0)) / np.abs(ek0 + ep0)
        # oracle: 16 seeded clusters with N_c <= 4096 integrated fully, energy drift compared
        small = np.nonzero(sizes <= 4096)[0]
        pick = np.sort(np.random.default_rng(77).choice(small, 16, replace=False))
        orc = []
        for q in pick:
            a, b = off[q], off[q + 1]
            r = oracle.hermite_run(m[a:b], x[a:b], v[a:b], eps[q], 0.01, 2.0 ** -22, t_end, t_end)
            E0 = sum(oracle.energy(m[a:b], x[a:b], v[a:b], eps[q]))
            d_orc = abs(sum(oracle.energy(m[a:b], r["x"], r["v"], eps[q])) - E0) / abs(E0)
            fx = finals["persistent_graph"]
            d_gpu = abs(sum(oracle.energy(m[a:b], fx["x"][a:b], fx["v"][a:b], eps[q])) - E0) / abs(E0)
            orc.append({"cluster": int(q), "N": int(b - a), "drift_gpu": d_gpu, "drift_oracle": d_orc})
        dx = np.abs(finals["persistent_graph"]["x"] - finals["per_cluster_launches"]["x"]).max()
        dx_t = np.abs(finals["persistent_graph"]["x"] - finals["persistent_graph_autotuned"]["x"]).max()
        print(json.dumps({"workload": "c4", "clusters": 512, "N_total": int(off[-1]), "t_end": t_end,
                          "modes": res, "autotuned_shape": tuned,
                          "speedup_autotuned_vs_default_shape": res["persistent_graph"]["wall_s"] /
                          res["persistent_graph_autotuned"]["wall_s"],
                          "max_abs_dx_autotuned_vs_default": float(dx_t),
                          "speedup_persistent_vs_per_cluster": res["per_cluster_launches"]["wall_s"] /
                          res["persistent_graph"]["wall_s"],
                          "max_abs_dx_between_modes": float(dx),
                          "mixed_vs_fp64_persistent": res["persistent_graph"]["interactions_per_s"] /
                          res["persistent_graph_fp64"]["interactions_per_s"],
                          "energy_drift_gpu_median": float(np.median(drift)),
                          "energy_drift_gpu_max": float(drift.max()),
                          "energy_drift_fp64_median": float(np.median(drift64)),
                          "energy_drift_fp64_max": float(drift64.max()),
                          "oracle_subset": orc,
                          "oracle_subset_within_2x": all(o["drift_gpu"] <= 2 * o["drift_oracle"] + 1e-9 for o in orc)}),
              flush=True)
        return
    if w == "c3sweep":
        # configuration 3's active-block sweep: N = 2^20 equal masses, eps = 1/4096, the first n of
        # a seeded shuffle, on a state of the block-step schedule (the initial forces and steps,
        # each particle's time the last multiple of its step before T = 1/16, so prediction runs
        # over h up to a whole step).  Per n: the mixed path with the separate predictor of all N
        # (nb_predict + nb_compute_forces), the same forces with the j-particles predicted on the
        # fly (nb_compute_forces_at: GRAPE's split, Sec. 4.4 steps 3-4), and the FP64 path; errors
        # vs the oracle (FP64 prediction of all N, compensated sums) on 1024 sampled particles
        N, eps, T = 1 << 20, 1.0 / 4096, 2.0 ** -4
        m, x, v = inputs.plummer(N, 3)
        s = nb.NBody(N, nb.NB_MIXED, 0)
        s.set_params(eps, 0.01, 2.0 ** -22, 2.0 ** -3)
        s.set_j_particles(0, m, x, v)
        s.initial_forces_and_dt()
        st = s.get_particles(0, N)
        s.close()
        ti = (np.ceil(T / st["dt"]) - 1.0) * st["dt"]
        state = (m, x, v, st["a"], st["jerk"], ti, st["dt"])
        xp, vp = oracle.predict(x, v, st["a"], st["jerk"], ti, T)
        res = []
        sweep = (256, 1024, 2048, 4096, 8192, inputs.block_size(N), 65536, N)
        if args.sweep_n:
            sweep = tuple(int(k) for k in args.sweep_n.split(","))
        for n in sweep:
            act = inputs.sample_indices(N, n, 1003).astype(np.int32)
            pos = inputs.sample_indices(n, min(n, 1024), 2003)
            ref = oracle.forces(m, xp, vp, eps, idx=act[pos].astype(np.int64), compensated=True)
            row = {"n_active": n}
            for prec, name in ((nb.NB_MIXED, "mixed"), (nb.NB_MIXED, "mixed_autotuned"),
                               (nb.NB_MIXED, "mixed_onthefly"), (nb.NB_FP64, "fp64")):
                if prec == nb.NB_FP64 and n > 65536:
                    continue  # 1.1e12 FP64 interactions take over a minute; the sample covers accuracy
                if name == "mixed_autotuned" and n > 65536:
                    continue  # the tuner's ~80 trial launches of 0.9 s each at n = N
                s = nb.NBody(N, prec, 0, stream=torch.cuda.current_stream())
                s.set_params(eps, 0.01, 2.0 ** -22, 2.0 ** -3)
                s.set_j_particles(0, *state)
                d_act = torch.from_numpy(act).cuda()
                tuned = None
                if name == "mixed_autotuned":
                    # nb_autotune_list on this block (the trial launches use this active list on
                    # the same state), then the same timed calls take the tuned launch; with
                    # --tune-file the table collects every n's entry
                    if args.tune_file and os.path.exists(args.tune_file):
                        s.tune_load(args.tune_file)
                    s.predict(T)
                    tuned = s.autotune_list(d_act)
                    if args.tune_file:
                        s.tune_save(args.tune_file)
                A = torch.empty((n, 3), dtype=torch.float64, device="cuda")
                J = torch.empty_like(A)
                P = torch.empty(n, dtype=torch.float64, device="cuda")
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

                def once():
                    ev[0].record()
                    if name == "mixed_onthefly":
                        s.compute_forces_at(T, d_act, A, J, P)
                        ev[1].record()
                    else:
                        s.predict(T)
                        ev[1].record()
                        s.compute_forces(d_act, A, J, P)
                    ev[2].record()

                once()  # warm-up (the first on-the-fly call also builds the j-memory)
                reps = 5 if n * N < 1e10 else (3 if n * N < 1e11 else 1)
                tp, tf = [], []
                for _ in range(reps):
                    once()
                    torch.cuda.synchronize()
                    tp.append(ev[0].elapsed_time(ev[1]))
                    tf.append(ev[1].elapsed_time(ev[2]))
                tp, tf = float(np.median(tp)), float(np.median(tf))
                pp = torch.from_numpy(pos).cuda()
                a, j, p = A[pp].cpu().numpy(), J[pp].cpu().numpy(), P[pp].cpu().numpy()
                s.close()
                ea, ej, ep = rel(a, ref[0]), rel(j, ref[1]), np.abs(p - ref[2]) / np.abs(ref[2])
                tot = tp + tf
                if name == "mixed_onthefly":  # one call: list prediction, boxes and forces
                    tp, tf = None, tot
                row[name] = {"ms_predict": tp, "ms_force": tf, "ms_total": tot,
                             "interactions_per_s": float(n) * N / (tot / 1e3),
                             "frac_fp32_peak_60flop_force": float(n) * N / (tf / 1e3) * 60 / 80.548e12,
                             "acc_median": float(np.median(ea)), "acc_max": float(ea.max()),
                             "jerk_median": float(np.median(ej)), "jerk_max": float(ej.max()),
                             "pot_max": float(ep.max())}
                if tuned is not None:
                    row[name]["tuning"] = tuned
            row["onthefly_speedup"] = row["mixed"]["ms_total"] / row["mixed_onthefly"]["ms_total"]
            res.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
        print(json.dumps({"workload": "c3sweep", "N": N, "eps": eps, "T": T, "rows": res}), flush=True)
        return
    if w == "tapp":
        # T_app for one N-body time unit vs N on one GB300 (the single-node curves of the paper's
        # timing figures), the per-task time of one block step with the average block size
        # n = 0.20 N^0.81 (Sec. 3.2 profile), and the Sec. 4.1 model T = sum(tau_pred N +
        # tau_force n N + tau_corr n) recalibrated with GB300's tau's (Eqs. 1-4).
        eps, eta = 2.0 ** -8, 0.01
        prec = nb.NB_FP64 if args.precision == "fp64" else nb.NB_MIXED  # (--precision fp64: short --tapp-sizes)
        out = []
        sizes = [int(s) for s in args.tapp_sizes.split(",")]
        for N in sizes:
            m, x, v = inputs.plummer(N, 100 + N)
            s = nb.NBody(N, prec, 0)
            s.set_params(eps, eta, 2.0 ** -22, 2.0 ** -3)
            s.set_j_particles(0, m, x, v)
            s.initial_forces_and_dt()
            # one step of the Sec. 3.2 profile: n = 0.20 N^0.81 active particles
            n = inputs.block_size(N)
            idx = inputs.sample_indices(N, n, 7).astype(np.int32)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            dev_idx = torch.from_numpy(idx).cuda()
            A = torch.empty((n, 3), dtype=torch.float64, device="cuda")
            J = torch.empty_like(A)
            P = torch.empty(n, dtype=torch.float64, device="cuda")
            prof = []
            for rep in range(4):
                torch.cuda.synchronize()
                ev[0].record()
                s.predict(0.0)
                ev[1].record()
                s.compute_forces(dev_idx, A, J, P)
                ev[2].record()
                s.correct(dev_idx, 2.0 ** -22)
                ev[3].record()
                torch.cuda.synchronize()
                prof.append([ev[k].elapsed_time(ev[k + 1]) for k in range(3)])
                s.set_j_particles(0, m, x, v)   # undo the correction
                s.initial_forces_and_dt()
            pr = np.median(np.array(prof[1:]), axis=0)
            # one N-body time unit with block steps
            s.get_timings(reset=True)
            c0 = s.get_counters()
            k0, w0 = s.energy()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.integrate(1.0, use_graph=False)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            tim = s.get_timings()
            c1 = s.get_counters()
            k1, w1 = s.energy()
            jp = s.get_jpredict()
            s.close()
            # the host loop again with every block predicting all N first (the on-the-fly j
            # prediction of small blocks, Sec. 4.4 steps 3-4, switched off): the ablation
            h2 = nb.NBody(N, prec, 0)
            h2.set_params(eps, eta, 2.0 ** -22, 2.0 ** -3)
            h2.set_j_particles(0, m, x, v)
            h2.initial_forces_and_dt()
            h2.set_jpredict(0)
            ch0 = h2.get_counters()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h2.integrate(1.0, use_graph=False)
            torch.cuda.synchronize()
            wall_sep = time.perf_counter() - t0
            steps_sep = h2.get_counters()["block_steps"] - ch0["block_steps"]
            h2.close()
            # the same time unit with the whole block-step loop on the device (one CUDA graph)
            g = nb.NBody(N, prec, 0)
            g.set_params(eps, eta, 2.0 ** -22, 2.0 ** -3)
            g.set_j_particles(0, m, x, v)
            g.initial_forces_and_dt()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.integrate(1.0, use_graph=True)
            torch.cuda.synchronize()
            wall_g = time.perf_counter() - t0
            kg, wg = g.energy()
            g.close()
            # ... and as one persistent cooperative kernel (mixed systems up to 262144, FP64 up to 65536)
            wall_p, drift_p, steps_p = None, None, None
            if N <= (nb.NB_PERSISTENT_MAX_N if prec == nb.NB_MIXED else nb.NB_PERSISTENT_MAX_N_FP64):
                q = nb.NBody(N, prec, 0)
                q.set_params(eps, eta, 2.0 ** -22, 2.0 ** -3)
                q.set_j_particles(0, m, x, v)
                q.initial_forces_and_dt()
                cq0 = q.get_counters()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                q.integrate(1.0, loop=nb.NB_LOOP_PERSISTENT)
                torch.cuda.synchronize()
                wall_p = time.perf_counter() - t0
                steps_p = q.get_counters()["block_steps"] - cq0["block_steps"]
                kq, wq = q.energy()
                drift_p = abs((kq + wq) - (k0 + w0)) / abs(k0 + w0)
                q.close()
            # ... and on one thread-block cluster (mixed systems up to 16384)
            wall_c, drift_c, steps_c = None, None, None
            if N <= nb.NB_CLUSTER_MAX_N and prec == nb.NB_MIXED:
                q = nb.NBody(N, prec, 0)
                q.set_params(eps, eta, 2.0 ** -22, 2.0 ** -3)
                q.set_j_particles(0, m, x, v)
                q.initial_forces_and_dt()
                cq0 = q.get_counters()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                q.integrate(1.0, loop=nb.NB_LOOP_CLUSTER)
                torch.cuda.synchronize()
                wall_c = time.perf_counter() - t0
                steps_c = q.get_counters()["block_steps"] - cq0["block_steps"]
                kq, wq = q.energy()
                drift_c = abs((kq + wq) - (k0 + w0)) / abs(k0 + w0)
                q.close()
            steps = c1["block_steps"] - c0["block_steps"]
            inter = tim["interactions"]
            psteps = inter / N
            tp, tf, tc = tim["ms_pred"] / 1e3, tim["ms_force"] / 1e3, tim["ms_corr"] / 1e3
            taus = sec41_taus(tp, tf, tc, N, steps, inter, psteps)
            out.append({"N": N, "profile_step": {"n": n, "ms_predict": pr[0], "ms_force": pr[1], "ms_correct": pr[2]},
                        "T_app_s": wall, "block_steps": steps, "particle_steps": psteps, "interactions": inter,
                        "interactions_per_s": inter / wall,
                        "tau_pred_s": taus[0], "tau_force_s": taus[1], "tau_corr_s": taus[2],
                        "model_T_s": sec41_T(taus, N, steps, inter, psteps), "share_force": tf / wall,
                        "share_pred": tp / wall,
                        "share_corr": tc / wall, "share_host_and_select": 1 - (tp + tf + tc) / wall,
                        "energy_drift": abs((k1 + w1) - (k0 + w0)) / abs(k0 + w0),
                        "jpredict_max_n": jp,
                        "T_app_host_separate_predictor_s": wall_sep, "block_steps_separate": steps_sep,
                        "T_app_graph_s": wall_g, "energy_drift_graph": abs((kg + wg) - (k0 + w0)) / abs(k0 + w0),
                        "T_app_persistent_s": wall_p, "block_steps_persistent": steps_p,
                        "T_app_cluster_s": wall_c, "block_steps_cluster": steps_c, "energy_drift_cluster": drift_c,
                        "energy_drift_persistent": drift_p})
            print(json.dumps(out[-1]), file=sys.stderr, flush=True)
        # the paper calibrates its model on one run (N = 32768, Sec. 4.1) and predicts the others:
        # the same with the tau's of the N = 32768 row (when it was run)
        cal = [r for r in out if r["N"] == 32768]
        if cal:
            taus = (cal[0]["tau_pred_s"], cal[0]["tau_force_s"], cal[0]["tau_corr_s"])
            for r in out:
                r["model_T_calibrated_at_32768_s"] = sec41_T(taus, r["N"], r["block_steps"], r["interactions"],
                                                             r["particle_steps"])
        print(json.dumps({"workload": "tapp", "eps": eps, "eta": eta, "t_end": 1.0, "precision": args.precision,
                          "grape_tau_force_s": 4.3e-10, "rows": out}), flush=True)
        return
    raise SystemExit(f"unknown workload {w}")


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload != "c3":
        run_integration(args)
        return

    import torch
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_0709_4552_gb300 import build, inputs
    build.build()
    from paper_0709_4552_gb300 import nbody as nb

    N, eps, dt_shared = args.n, args.eps, 2.0 ** -10
    prec = nb.NB_MIXED if args.precision == "mixed" else nb.NB_FP64
    m, x, v = inputs.plummer(N, args.seed)
    stream = torch.cuda.current_stream(dev)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count

    s = nb.NBody(N, prec, local, stream=stream)
    s.set_params(eps, 0.01, dt_shared, dt_shared)
    if args.tuning:
        s.set_tuning(*[int(t) for t in args.tuning.split(",")])
    s.set_j_particles(0, m, x, v)
    s.initial_forces_and_dt()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        flush.fill_(1.0)   # the flush kernel loads with its first launch: before the timed region
        s.step()
    s.get_timings(reset=True)
    launches0 = s.get_counters()["kernel_launches"]
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev0.record(stream)
    for k in range(args.steps):
        flush.fill_(1.0)
        step_ev[k].record(stream)
        s.step()
    step_ev[args.steps].record(stream)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    per_step = [step_ev[k].elapsed_time(step_ev[k + 1]) for k in range(args.steps)]
    print(f"per-step ms (flush excluded after the first): {[round(x, 1) for x in per_step]}", file=sys.stderr)
    tim = s.get_timings()
    launches = s.get_counters()["kernel_launches"] - launches0
    t_max = max_over_ranks(ms, ws, dev)
    inter_rank = float(N) * N * args.steps
    value = whole_job_rate(inter_rank, ws, t_max / 1e3)

    # roofline of the force kernel (events on the context's stream around each launch)
    force_s_per_launch = tim["ms_force"] / 1e3 / args.steps
    achieved_tflops = FLOP_PER_INTERACTION * float(N) * N / force_s_per_launch / 1e12
    # the FP64 path is bound by the FP64 pipe: 1/64 of the FP32 lanes on this part
    fp_div = 1.0 if prec == nb.NB_MIXED else 64.0
    peak = fp32_peak_tflops(sms, SM_MAX_MHZ_FALLBACK) / fp_div
    sm_mhz = clk["sm_mhz"] if clk else None
    # predictor and corrector: HBM-bound passes, algorithmic bytes per particle
    # (predictor: m, t, x, v, a, jerk read, FP64 xp, vp written, plus slot index and
    # the 40 B mixed j-store; corrector: list, t, dt, a, jerk, 7 force rows, xp, vp
    # read, x, v, a, jerk, pot, t, dt written)
    pred_bytes = float(N) * (112 + 48 + (44 if prec == nb.NB_MIXED else 0))
    corr_bytes = float(N) * 292
    hbm = measured_hbm_gbs()
    phases = {}
    for name, key, b in (("predict", "ms_pred", pred_bytes), ("correct", "ms_corr", corr_bytes)):
        ms_k = tim[key] / args.steps
        gbs = b / (ms_k / 1e3) / 1e9 if ms_k > 0 else None
        # both are bound by the FP64 pipe (ncu: 86% active), not by HBM
        phases[name] = {"ms": ms_k, "bytes": b, "achieved_gbs": gbs, "peak_gbs": hbm,
                        "frac": (gbs / hbm) if (gbs and hbm) else None, "bound": "fp64 pipe"}

    # the same block steps with the far-tile pass off (double-single position
    # differences on every tile: the strict form of the precision pattern),
    # timed the same way, beside the default
    strict = None
    if prec == nb.NB_MIXED and args.strict_steps > 0:
        s.set_far_tiles(False)
        s.get_timings(reset=True)
        for _ in range(args.strict_steps):
            flush.fill_(1.0)
            s.step()
        barrier()
        tim_s = s.get_timings(reset=True)
        s.set_far_tiles(True)
        strict_s = tim_s["ms_force"] / 1e3 / args.strict_steps
        strict_tflops = FLOP_PER_INTERACTION * float(N) * N / strict_s / 1e12
        strict = {"bound": "alu", "achieved": strict_tflops, "peak": peak, "unit": "TFLOP/s",
                  "frac": strict_tflops / peak, "ms_per_launch": strict_s * 1e3,
                  "launches": args.strict_steps, "far_tiles": False,
                  "default_ms_per_launch": force_s_per_launch * 1e3,
                  "far_pass_speedup": strict_s / force_s_per_launch}

    # end to end through the C ABI with host buffers: H2D of the step's inputs,
    # the step, D2H of its results, all inside the timed region
    e2e = None
    if not args.no_e2e:
        st = s.get_particles(0, N)
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hin = dict(m=pin(st["m"]), x=pin(st["x"]), v=pin(st["v"]), a=pin(st["a"]), jerk=pin(st["jerk"]),
                   t=pin(st["t"]), dt=pin(st["dt"]))
        hout = {k: pin(np.empty_like(st[k])) for k in ("x", "v", "a", "jerk", "pot", "t", "dt")}
        e_steps = max(1, min(args.steps, 3))
        barrier()
        t0 = time.perf_counter()
        for _ in range(e_steps):
            s.set_j_particles(0, hin["m"], hin["x"], hin["v"], hin["a"], hin["jerk"], hin["t"], hin["dt"])
            s.step()
            s.get_particles(0, N, out=hout)
        barrier()
        e_s = max_over_ranks(time.perf_counter() - t0, ws, dev)
        bi = sum(t.numel() * 8 for t in hin.values())
        bo = sum(t.numel() * 8 for t in hout.values())
        e2e = {"value": float(N) * N * e_steps * ws / e_s, "unit": UNIT, "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "steps": e_steps}

    # FP64 GPU path and mixed-path accuracy on sampled particles of the same state
    extra = {}
    cpu = None
    if rank == 0:
        st = s.get_particles(0, N)
        k = min(args.cpu_sample, N)
        idx = inputs.sample_indices(N, k, args.seed + 1000).astype(np.int32)
        t_now = float(st["t"][0])
        s.predict(t_now)
        am, jm, pm = s.compute_forces(idx)
        if prec == nb.NB_MIXED:
            s.set_far_tiles(False)
            as_, js_, ps_ = s.compute_forces(idx)
            s.set_far_tiles(True)
        s.set_precision(nb.NB_FP64)
        s.predict(t_now)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        a64, j64, p64 = s.compute_forces(idx)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        fp64_rate = float(k) * N / (e0.elapsed_time(e1) / 1e3)
        s.set_precision(prec)
        pk = s.measure_peaks()
        # the FP64 item issues 32 FP64-pipe instructions per interaction (source count)
        extra["fp64_gpu_path"] = {"value": fp64_rate, "unit": UNIT,
                                  "sample": f"{k} active x N={N}", "vs_mixed": fp64_rate / value * ws,
                                  "fp64_pipe_frac": fp64_rate * 32 / (pk["fp64_tflops"] * 1e12 / 2)}
        # how the FP64 unit issues (cycles per FMA for one warp, dependent chain with 32 or 1
        # lanes, four chains; SM cycles per warp instruction with 16 warps)
        pk["fp64_issue_cycles"] = s.measure_fp64_issue()
        extra["peaks_measured"] = pk
        if not args.no_cpu and ws == 1:  # the host baseline is taken at N = 1 only
            import oracle
            oracle.build()
            t0 = time.perf_counter()
            ar, jr, pr = oracle.forces(st["m"], st["x"], st["v"], eps, idx=idx.astype(np.int64))
            cpu_s = time.perf_counter() - t0
            cpu = {"value": float(k) * N / cpu_s, "unit": UNIT, "cores": oracle.max_threads(),
                   "kind": "oracle", "sample": f"forces on {k} sampled particles from all N={N} "
                                               f"(one block step's state), {cpu_s:.1f} s"}
            k1 = max(1, k // 32)
            t0 = time.perf_counter()
            oracle.forces(st["m"], st["x"], st["v"], eps, idx=idx[:k1].astype(np.int64), threads=1)
            one_s = time.perf_counter() - t0
            cpu["single_core"] = {"value": float(k1) * N / one_s, "unit": UNIT, "cores": 1,
                                  "sample": f"forces on {k1} sampled particles from all N={N}, {one_s:.1f} s"}
            # a full i = j evaluation of a smaller sphere on all cores
            n16 = 1 << 16
            m16, x16, v16 = inputs.plummer(n16, args.seed)
            t0 = time.perf_counter()
            oracle.forces(m16, x16, v16, eps)
            f_s = time.perf_counter() - t0
            cpu["full_ij"] = {"value": float(n16) * n16 / f_s, "unit": UNIT, "cores": oracle.max_threads(),
                              "sample": f"full i = j forces at N={n16}, {f_s:.1f} s"}

            def rel(a, b):
                return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)

            ea, ej, ep = rel(am, ar), rel(jm, jr), np.abs(pm - pr) / np.abs(pr)
            e64 = rel(a64, ar)
            extra["accuracy_vs_oracle"] = {
                "sample": k, "mixed_acc_median": float(np.median(ea)), "mixed_acc_max": float(ea.max()),
                "mixed_jerk_median": float(np.median(ej)), "mixed_jerk_max": float(ej.max()),
                "mixed_pot_median": float(np.median(ep)), "mixed_pot_max": float(ep.max()),
                "fp64_acc_max": float(e64.max()), "fp64_jerk_max": float(rel(j64, jr).max()),
                "fp64_pot_max": float((np.abs(p64 - pr) / np.abs(pr)).max())}
            if prec == nb.NB_MIXED:
                es = (rel(as_, ar), rel(js_, jr), np.abs(ps_ - pr) / np.abs(pr))
                for nm, e_ in zip(("acc", "jerk", "pot"), es):
                    extra["accuracy_vs_oracle"][f"strict_{nm}_median"] = float(np.median(e_))
                    extra["accuracy_vs_oracle"][f"strict_{nm}_max"] = float(e_.max())
    s.close()

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 pairwise (packed x2) + double-single f32 accumulate" if prec == nb.NB_MIXED else "f64",
            "data": "synthetic (seeded Plummer sphere, Aarseth-Henon-Wielen sampling)",
            "config": dict(workload_config(args), parallelism=f"replicas x{ws}" if ws > 1 else "1 GPU"),
            "gflops_60": value * FLOP_PER_INTERACTION / 1e9,
            "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved_tflops / peak,
                         "traffic": profiled_traffic(N) if prec == nb.NB_MIXED else None,
                         "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                         "algorithmic_bytes": float(N) * (40 + 4 + 56),
                         "kernel": "force_mixed_kernel" if prec == nb.NB_MIXED else "force_fp64_kernel",
                         "peak_basis": (f"FP32 CUDA cores: {sms} SMs x 128 x 2 flop x {SM_MAX_MHZ_FALLBACK:.0f} MHz"
                                        + ("" if fp_div == 1.0 else " / 64 (FP64 pipe)")),
                         "frac_at_sampled_clock": (achieved_tflops * fp_div / fp32_peak_tflops(sms, sm_mhz))
                         if sm_mhz else None},
            "roofline_strict": strict,
            "hbm_rooflines": phases,
            "phases_ms_per_step": {"predict": tim["ms_pred"] / args.steps, "force": tim["ms_force"] / args.steps,
                                   "correct": tim["ms_corr"] / args.steps},
            "gpu_launches": int(launches) * ws,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        out.update(extra)
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()

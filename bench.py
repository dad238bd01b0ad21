#!/usr/bin/env python
"""Benchmark of the lambda-dynamics step (alchemical nonbonded evaluation +
Langevin/constraints + theta/OPES) on the octanol solvation box.

One step = one pass of the whole hot path: pair kernel, PME (spread, FFT,
convolution, inverse FFT, gather), exclusion/1-4 and bonded terms, the
constrained Langevin middle-scheme update of every atom, the theta/dual-OPES
update and (when needed) the device-side neighbour-list rebuild, replayed as
one captured CUDA graph.

Prints one JSON line (rank 0).  --impl reference times the FP64 oracle on the
host cores on a bounded sample of the same workload.
"""
import argparse
import json

import numpy as np
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ns/day & pair-interactions/s (mixed vs FP64, batched vs per-replica) on 1 B300"
# algorithmic FP32 operations per interacting pair, itemised: minimum image 9,
# r^2 5, rsqrt 1, erfc + exp 12, Coulomb 4, LJ 8, switch 8, force vector and
# Newton's third law 12 (58 in all; about two of them go to the special
# function unit)
FLOPS_PER_PAIR = 58
# From one ncu capture of the current k_pairs2 on the octanol profile case
# (31,949 tiles of the 0.10 nm-buffer list): DRAM bytes (dram__bytes_read.sum
# 6,353,920 + dram__bytes_write.sum 0) and counted FP32 operations (2 FFMA +
# 4 FFMA2 + FADD + 2 FADD2 + FMUL + 2 FMUL2, predicated-on thread
# instructions: 6.340e8; every lane of an executed step counts, the lanes
# whose pairs are out of range computing zeros), both per tile, for scaling
# to the tile count of the timed launch (the tile records dominate the
# traffic, and every tile runs the same instruction stream); None whenever
# the kernel has changed since the capture
PAIR_CAPTURE_TILES = 31949
PAIR_DRAM_BYTES_PER_TILE = 6347520.0 / PAIR_CAPTURE_TILES
PAIR_COUNTED_FLOPS_PER_TILE = 6.340e8 / PAIR_CAPTURE_TILES
FP32_LANES_PER_SM = 128
MAX_SM_MHZ = 2032.0
# timed evaluations of the reference arm at most (one level-2 oracle
# evaluation of the octanol box takes 0.2-0.5 s on the host cores)
REFERENCE_MAX_STEPS = 200


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None,
                   help="timed steps (default 2000; 20 oracle evaluations for --impl reference)")
    p.add_argument("--warmup", type=int, default=None, help="untimed warm-up steps (default 50; 3 for the oracle)")
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="octanol", choices=["octanol", "water", "c0"])
    p.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison leg")
    p.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    p.add_argument("--no-dafed", action="store_true", help="skip the flexible-solute d-AFED leg")
    p.add_argument("--no-errors", action="store_true",
                   help="skip the oracle-error leg (every output of both precisions against levels 1 and 2)")
    p.add_argument("--e2e-steps", type=int, default=200)
    p.add_argument("--tune-cache", default=None,
                   help="JSON autotuner cache shared by every system of the run (default: none for the main "
                        "system, a temporary one for the batched replicas)")
    p.add_argument("--no-autotune", action="store_true",
                   help="keep the default launch shapes in every leg (e.g. for a per-kernel launch list)")
    p.add_argument("--batch-replicas", type=int, default=32,
                   help="replicas in the batched leg (half water, half octanol; 0 skips it)")
    p.add_argument("--batch-steps", type=int, default=40)
    p.add_argument("--profile-case", action="store_true",
                   help="build the workload, run 3 staged evaluations and exit (a small case for ncu)")
    p.add_argument("--prune", type=float, default=None,
                   help="inner buffer (nm) of the pruned pair list (lfe_set_list_prune) for the profile case")
    p.add_argument("--skin", type=float, default=None, help="list buffer (nm) of the profile case")
    a = p.parse_args()
    ref = a.impl == "reference"
    if a.steps is None:
        a.steps = 20 if ref else 2000
    if a.warmup is None:
        a.warmup = 3 if ref else 50
    return a


# Section 2.6: the extended variables (theta, the d-AFED auxiliary angles)
# are thermostatted by the regulated Nose-Hoover-Langevin thermostat with a
# 40 fs time constant, 25 ps^-1 friction and regulation parameter 1
EXT_THERMOSTAT = dict(tau=0.040, n_reg=1.0)


def use_paper_thermostat(g):
    from paper_2608_12691_b300 import lfe
    g.set_ext_thermostat(lfe.LFE_EXT_RNHL, **EXT_THERMOSTAT)


def run_config(d, desc):
    """The workload description shared by both arms of the bench."""
    return {"workload": desc, "atoms": len(d["charge"]), "dt_fs": float(d["dt"]) * 1e3,
            "extended_thermostat": "regulated Nose-Hoover-Langevin, tau 40 fs, 25 ps^-1, regulation 1",
            "list_buffer": "chosen by lfe_autotune among 0.10-0.26 nm (0.10 without autotuning)",
            "l2": "flushed between steps (256 MiB write)", "data": "seeded synthetic stand-in"}


def make_workload(name, rank):
    from paper_2608_12691_b300 import systems as S
    if name == "octanol":
        d = S.make_c1(seed=2609 + 1000 * rank)
        desc = ("octanol solvation box: 500 27-atom octanol-like chains + 20-atom rigid solute, "
                "13,520 atoms, 4.8 nm, r_c 1.0 nm, PME 48^3, octanol masses x0.1, dual OPES on lambda")
    elif name == "water":
        d = S.make_c2(seed=2610 + 1000 * rank)
        desc = ("water box: 4,000 rigid waters + 20-atom rigid solute, 12,020 atoms, 4.93 nm, "
                "r_c 1.0 nm, PME 48^3, lambda mass 20 amu nm^2, OPES every 500 steps")
    else:
        d = S.make_c0(seed=2608 + 1000 * rank)
        desc = "12-atom solute + 216 waters, 660 atoms, 1.86 nm, r_c 0.9 nm, PME 16^3"
    d = dict(d)
    d.setdefault("lambda_mass", 20.0)
    d.setdefault("opes_stride", 500)
    d.setdefault("opes_dE_std", 30.0 * 4.184)
    d.setdefault("opes_dE_exp", 5.0 * 4.184)
    return d, desc


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.p = None
        # the first sample must exist before the timed region starts
        t0 = time.perf_counter()
        while self.p is not None and time.perf_counter() - t0 < 5.0:
            self.f.flush()
            if os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.02)

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_model():
    """The host CPU's model name (from /proc/cpuinfo), or None."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def oracle_timed(d, level, reps):
    """Median host time of `reps` oracle evaluations (nonbonded + bonded) of
    system d at the given level, and the last evaluation's results."""
    from oracle import reference as R
    times = []
    out = None
    for _ in range(reps):
        t0 = time.perf_counter()
        E, F0, Fuv, Fs = R.nonbonded(d, level=level)
        Ub, Fb = R.bonded(d)
        times.append(time.perf_counter() - t0)
        out = (E, F0, Fuv, Fs, Ub, Fb)
    return statistics.median(times), times, out


def cpu_baseline(d, dt_ps, reps=3):
    """The oracle as it stands timed on the host cores on full force/energy
    evaluations of the same system: level 2 (real-space pairs + naive-DFT
    smooth PME on the GPU's grid, the approximation the GPU computes) and
    level 1 (real-space pairs + direct Ewald k-sum, the definition), medians
    of `reps` each; value = level 2 converted to the step's ns/day.  Returns
    (baseline, {level: results}) so that the results serve the error leg."""
    from oracle import reference as R
    t2, all2, r2 = oracle_timed(d, 2, reps)
    t1, all1, r1 = oracle_timed(d, 1, reps)
    n_pairs = r2[0]["n_pairs"]
    base = {"value": dt_ps * 1e-3 * 86400.0 / t2, "unit": "ns/day", "cores": R.num_threads(),
            "host_cpus": os.cpu_count(), "cpu_model": cpu_model(), "kind": "oracle",
            "label": "definitional FP64 oracle, not an optimised CPU MD engine",
            "sample": f"median of {reps} full level-2 oracle force+energy evaluations of the same "
                      f"{len(d['charge'])}-atom system ({t2:.3f} s each); integration not included",
            "seconds_per_eval": t2, "seconds_per_eval_all": all2, "pair_interactions_per_s": n_pairs / t2,
            "level1": {"seconds_per_eval": t1, "seconds_per_eval_all": all1,
                       "ns_per_day": dt_ps * 1e-3 * 86400.0 / t1, "pair_interactions_per_s": n_pairs / t1}}
    return base, {1: r1, 2: r2}


def output_errors(terms, F, res, lam, solute):
    """Errors of every output of one GPU evaluation against one oracle level:
    forces (relative RMS over all atoms and over the solute, largest component
    error relative to the RMS atomic force), U, the class energies and
    dU/dlambda (absolute, kJ/mol, and relative)."""
    from oracle import reference as R
    E, F0, Fuv, Fs, Ub, Fb = res
    hA, hB, dA, dB = R.switching(lam)
    Fo = F0 + hA * Fuv + hB * Fs + Fb
    sol = np.asarray(solute).astype(bool)
    out = {"F_rel_rms": float(np.linalg.norm(F - Fo) / np.linalg.norm(Fo)),
           "F_rel_rms_solute": float(np.linalg.norm(F[sol] - Fo[sol]) / np.linalg.norm(Fo[sol])),
           "F_max_over_rms": float(np.abs(F - Fo).max() / np.sqrt((Fo * Fo).sum(1).mean()))}
    ref = {"U": E["U_vv"] + E["U_uu"] + hA * E["U_uv"] + hB * E["U_soft"] + Ub,
           "dUdl": dA * E["U_uv"] + dB * E["U_soft"],
           "U_vv": E["U_vv"], "U_uu": E["U_uu"], "U_uv": E["U_uv"], "U_soft": E["U_soft"], "U_bonded": Ub}
    for k, v in ref.items():
        err = float(terms[k] - v)
        out[k] = {"abs": err, "rel": abs(err) / abs(v) if v else None}
    return out


def error_leg(systems, oracle_cache):
    """Every output of both precision modes against the level-2 oracle (the
    same smooth PME on the same grid, the parity bar) and the level-1 oracle
    (exact Ewald; dominated by the PME discretisation of the grid), on the
    seeded frames named in `systems` (name -> (d, lambda))."""
    from paper_2608_12691_b300 import lfe
    out = {}
    for name, (d, lam) in systems.items():
        res = oracle_cache.get(name) or {lv: oracle_timed(d, lv, 1)[2] for lv in (2, 1)}
        row = {"atoms": len(d["charge"]), "lambda": lam}
        for pname, prec in (("fp32_mixed", lfe.LFE_FP32_MIXED), ("fp64", lfe.LFE_FP64)):
            g = lfe.System(d, precision=prec)
            terms, F = g.eval(lam)
            g.close()
            row[pname] = {f"vs_level{lv}": output_errors(terms, F, res[lv], lam, d["solute"]) for lv in (2, 1)}
        out[name] = row
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import reference as R
    d, desc = make_workload(args.workload, 0)
    dt_ps = float(d["dt"])
    for _ in range(args.warmup):
        oracle_timed(d, 2, 1)
    k = min(args.steps, REFERENCE_MAX_STEPS)
    _, times, res = oracle_timed(d, 2, k)
    t = sum(times) / k
    v = dt_ps * 1e-3 * 86400.0 / t
    npairs = res[0]["n_pairs"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ns/day", "n_gpus": args.gpus,
            "steps": k, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": run_config(d, desc),
            "pair_interactions_per_s": npairs / t,
            "cpu_baseline": {"value": v, "unit": "ns/day", "cores": R.num_threads(), "host_cpus": os.cpu_count(),
                             "cpu_model": cpu_model(), "kind": "oracle",
                             "label": "definitional FP64 oracle, not an optimised CPU MD engine",
                             "sample": f"each step one full level-2 oracle force+energy evaluation of the same "
                                       f"{len(d['charge'])}-atom system (mean {t:.3f} s over {k}); integration "
                                       f"not included"},
            "e2e": {"value": v, "unit": "ns/day", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def equilibrate(g, d, stream):
    """Untimed equilibration from the packed lattice start: short phases of
    small time step and high friction, then the production parameters."""
    dt = float(d["dt"])
    for dt_eq, fric, n in ((dt * 0.05, 100.0, 200), (dt * 0.25, 50.0, 200), (dt * 0.5, 20.0, 200)):
        g.set_integrator(dt_eq, fric, float(d["temperature"]))
        g.step(n, stream)
    g.set_integrator(dt, float(d["friction"]), float(d["temperature"]))
    g.get_state()


def dafed_leg(args, stream, flush):
    """The flexible-solute workload of the method: a differentiation frame
    (22-atom dipeptide-like solute in 4,000 rigid waters, 12,022 atoms) stepped
    at 1 fs with lambda-dynamics under the dual OPES bias and d-AFED on the
    phi, psi and chi torsions (1000 K, 50 amu nm^2 rad^-2, 1000 kJ/mol/rad^2)."""
    import torch
    from paper_2608_12691_b300 import lfe
    from paper_2608_12691_b300 import systems as S
    d = dict(S.make_c4_frame(frame=0))
    d.update(dt=0.001, lambda_mass=20.0, lambda_friction=25.0, opes_stride=500,
             opes_dE_std=30.0 * 4.184, opes_dE_exp=5.0 * 4.184, opes_sigma=0.10)
    g = lfe.System(d, precision=lfe.LFE_FP32_MIXED, seed=4242, skin=0.0)   # buffer left to the autotuner
    g.set_dafed(S.DIPEPTIDE_CVS, 1000.0, 50.0, temperature=1000.0, friction=25.0)
    use_paper_thermostat(g)
    equilibrate(g, d, stream)
    if not args.no_autotune:
        g.autotune(reps=20)
    g.step(20, stream)
    torch.cuda.synchronize()
    k = max(20, min(200, args.steps))
    ms = time_steps(g, k, stream, flush)
    m = sum(ms) / k
    _, _, ext = g.get_state()
    s, _, xi = g.dafed_state()
    return {"workload": "dipeptide-like 22-atom flexible solute + 4,000 rigid waters, 12,022 atoms, 1 fs, "
                        "lambda-OPES (dual) + d-AFED on 3 torsions",
            "ms_per_step": m, "ns_per_day": 0.001 * 1e-3 * 86400.0 / (m * 1e-3), "steps": k,
            "lambda_end": ext["lambda"], "s_end": [float(x) for x in s], "xi_end": [float(x) for x in xi]}


def batched_leg(args, stream, flush):
    """Replicas at lambda_r = r/(R-1), alternately the water system (12,020
    atoms, 2 fs) and the octanol system (13,520 atoms, 1 fs): mixed precision
    advanced together (one graph launch per step), the same replicas one after
    another with their own graphs, and both forms again in FP64 from the same
    states."""
    import torch
    from paper_2608_12691_b300 import lfe
    from paper_2608_12691_b300 import systems as S
    R = args.batch_replicas
    t0 = time.perf_counter()
    dicts = []
    for r in range(R):
        lam = r / (R - 1)
        d = S.make_c2(seed=5000 + r, lam=lam) if r % 2 == 0 else S.make_c1(seed=6000 + r, lam=lam)
        dicts.append(d)
    t_gen = time.perf_counter() - t0
    reps = [lfe.System(d, precision=lfe.LFE_FP32_MIXED, seed=7000 + r, theta0=d["lam"]) for r, d in enumerate(dicts)]
    for g in reps:
        use_paper_thermostat(g)
    b = lfe.Batch(reps)
    for frac, fric in ((0.05, 100.0), (0.25, 50.0), (0.5, 20.0), (1.0, None)):
        for d, g in zip(dicts, reps):
            g.set_integrator(float(d["dt"]) * frac, fric if fric else float(d["friction"]), float(d["temperature"]))
        b.step(200 if fric else args.warmup, stream)
    torch.cuda.synchronize()
    # replicas keep the default launch shapes and the 0.10 nm list buffer:
    # the autotuner times one system stepping alone, and its choices measured
    # no better for 32 replicas sharing the GPU (2.76-2.84 ms against
    # 2.74-2.75 ms per batched step; buffers of 0.16 and 0.22 nm, which
    # shorten a single system's step, gave 2.60 and 2.68 ms against 2.58 ms:
    # with 32 replicas the pair work, not the rebuilds, sets the step);
    # --tune-cache applies a cache's entries to them
    tuned = [g.autotune(reps=20, cache_path=args.tune_cache)[1] for g in reps] \
        if (args.tune_cache and not args.no_autotune) else []
    for g in reps:
        g.get_state()
    K = args.batch_steps
    ms = time_steps(b, K, stream, flush)
    for g in reps:
        pos, _, _ = g.get_state()
        assert np.isfinite(pos).all()
    ms_step = sum(ms) / K
    ns_day = sum(float(d["dt"]) for d in dicts) * 1e-3 * 86400.0 / (ms_step * 1e-3)
    # the FP32 replicas' shared pair-kernel launch at batched scale (CUDA
    # events around launches of it alone, between steps)
    pair_ms = b.time_pairs(reps=20, stream=stream)
    pairs = sum(g.eval(d["lam"])[0]["n_pairs"] for g, d in zip(reps, dicts))
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak = n_sm * FP32_LANES_PER_SM * 2 * MAX_SM_MHZ * 1e6 / 1e12
    batch_roof = {"bound": "alu", "kernel": "k_pairs2 (all FP32 replicas, one launch)",
                  "kernel_ms": pair_ms, "pairs_per_launch": pairs, "flops_per_pair": FLOPS_PER_PAIR,
                  "achieved": pairs * FLOPS_PER_PAIR / (pair_ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s"}
    batch_roof["frac"] = batch_roof["achieved"] / peak
    dt_sum = sum(float(d["dt"]) for d in dicts)
    # mixed precision, one replica after another (each with its own graph)
    kmix = max(3, K // 8)
    tmix = sum(sum(time_steps(g, kmix, stream, flush)) / kmix for g in reps)
    # FP64 from the same states: one replica after another, then batched
    k64 = max(3, K // 8)
    t64 = 0.0
    reps64 = []
    for d, g in zip(dicts, reps):
        p, v, _ = g.get_state()
        g64 = lfe.System(d, precision=lfe.LFE_FP64, seed=1, theta0=d["lam"])
        use_paper_thermostat(g64)
        g64.set_positions(p)
        g64.set_velocities(v)
        g64.step(2, stream)
        torch.cuda.synchronize()
        t64 += sum(time_steps(g64, k64, stream, flush)) / k64
        reps64.append(g64)
    b64 = lfe.Batch(reps64)
    b64.step(2, stream)
    torch.cuda.synchronize()
    t64b = sum(time_steps(b64, k64, stream, flush)) / k64
    b64.close()
    for g64 in reps64:
        g64.close()
    ns_day64 = dt_sum * 1e-3 * 86400.0 / (t64 * 1e-3)
    b.close()
    for g in reps:
        g.close()
    return {"replicas": R, "atoms": int(sum(len(d["charge"]) for d in dicts)),
            "autotuned_from_cache": int(sum(t["from_cache"] for t in tuned)),
            "mixed_batched": {"ms_per_step": ms_step, "ns_per_day_x_replica": ns_day,
                              "pair_interactions_per_s": pairs / (ms_step * 1e-3), "steps": K},
            "fp64_per_replica": {"ms_per_step_all_replicas": t64, "ns_per_day_x_replica": ns_day64,
                                 "steps": k64},
            "mixed_per_replica": {"ms_per_step_all_replicas": tmix,
                                  "ns_per_day_x_replica": dt_sum * 1e-3 * 86400.0 / (tmix * 1e-3), "steps": kmix},
            "fp64_batched": {"ms_per_step": t64b, "ns_per_day_x_replica": dt_sum * 1e-3 * 86400.0 / (t64b * 1e-3),
                             "steps": k64},
            "speedup_mixed_batched_vs_fp64_per_replica": ns_day / ns_day64,
            "roofline_pairs": batch_roof,
            "setup_s": t_gen}


def max_over_ranks(value, world, device):
    """The largest of the ranks' values (every rank gets it); the timed region
    of the slowest rank sets the whole job's time."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_ns_day(dt_ps, ms_per_step, world):
    """Whole-job ns/day: every rank advances its own replica (same system
    size, own seed) by one step of dt_ps in ms_per_step (the slowest rank's)."""
    return dt_ps * 1e-3 * 86400.0 / (ms_per_step * 1e-3) * world


def time_steps(g, K, stream, flush):
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for i in range(K):
        flush.zero_()                    # L2 flush outside the timed step
        ev[i][0].record(stream)
        g.step(1, stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2608_12691_b300 import lfe

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    d, desc = make_workload(args.workload, rank)
    prec = lfe.LFE_FP64 if args.precision == "fp64" else lfe.LFE_FP32_MIXED
    dt_ps = float(d["dt"])
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    g = lfe.System(d, precision=prec, seed=2608 + rank, skin=0.0)   # buffer left to the autotuner
    use_paper_thermostat(g)
    terms0, _ = g.eval(d["lam"])
    n_pairs = terms0["n_pairs"]
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    equilibrate(g, d, stream)
    # launch shapes chosen on the equilibrated system (the tuner steps it
    # from a saved state and restores it)
    tune_ms, tune = (None, None) if args.no_autotune else g.autotune(reps=40, cache_path=args.tune_cache)
    time_steps(g, args.warmup, stream, flush)     # warm-up through the timed path
    torch.cuda.synchronize()
    _, _, ext0 = g.get_state()

    sampler = ClockSampler(local) if rank == 0 else None
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    ms = time_steps(g, args.steps, stream, flush)
    wall = time.perf_counter() - wall0
    barrier()
    clocks = sampler.stop() if sampler else None
    pos, vel, ext1 = g.get_state()       # raises on any device-side error
    assert np.isfinite(pos).all()
    total_ms = max_over_ranks(sum(ms), world, "cuda")
    ms_step = total_ms / args.steps
    ns_day = weak_scaling_ns_day(dt_ps, ms_step, world)
    rebuilds = int(ext1["n_rebuilds"] - ext0["n_rebuilds"])
    # kernels of one captured step (FP32 systems): rebuild decision, pair
    # kernel; spread, plane transform, column pass, inverse plane transform,
    # gather; df64 energy branch (two transform passes, column pass); kicks
    # with the OPES biases (one launch), exclusions/1-4, bonded, FP64 uv
    # energies, theta's step (the regulated thermostat's, once dU/dlambda is
    # in); integrator, theta's commit (which also ends the step); the FP64
    # form has no df64 branch.  A neighbour-list build adds 11 kernels (column keys,
    # column scan, scatter, column sort, slot assignment, tile search, tile
    # scan, placement + masks, uv pair count, scan, write).
    per_step = 17 if prec == lfe.LFE_FP32_MIXED else 14
    launches = args.steps * per_step + rebuilds * 11
    n_tiles = int(ext1["n_tiles"])

    out = None
    if rank == 0:
        # per-kernel device times with CUDA events on the launching stream
        stages = g.time_stages(float(ext1["lambda"]), reps=min(args.steps, 300), stream=stream)
        pair_ms = stages["pairs"]
        achieved = n_pairs * FLOPS_PER_PAIR / (pair_ms * 1e-3) / 1e12
        peak = n_sm * FP32_LANES_PER_SM * 2 * MAX_SM_MHZ * 1e6 / 1e12
        octanol32 = args.workload == "octanol" and prec == lfe.LFE_FP32_MIXED
        traffic = PAIR_DRAM_BYTES_PER_TILE * n_tiles if octanol32 else None
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "k_pairs2 (FP32, packed f32x2)", "kernel_ms": pair_ms,
                "flops_per_pair": FLOPS_PER_PAIR,
                "peak_basis": f"{n_sm} SMs (device properties) x 128 FP32 lanes x 2 flop/FMA x 2032 MHz "
                              f"(max SM clock); unit-count peak, no measured FP32 peak in the pool's file"}
        if clocks and clocks.get("sm_mhz"):
            roof["frac_at_measured_clock"] = achieved / (peak * clocks["sm_mhz"] / MAX_SM_MHZ)
        f32_meas, f64_meas = lfe.alu_peak()
        roof["peak_measured_fma_fp32"] = f32_meas
        roof["peak_measured_fma_fp64"] = f64_meas
        roof["frac_of_measured_fma"] = achieved / f32_meas
        if octanol32:
            # the FP32 pipes' own count (every evaluated pair slot, in range or
            # not), per tile from the ncu capture, over the live kernel time
            counted = PAIR_COUNTED_FLOPS_PER_TILE * n_tiles / (pair_ms * 1e-3) / 1e12
            roof["counted_fp32_tflops"] = counted
            roof["frac_counted_fp32"] = counted / peak
            roof["traffic_basis"] = f"ncu per-tile figures of a {PAIR_CAPTURE_TILES}-tile capture x {n_tiles} tiles"
        if "pairs_full" in stages:
            # the same launch with the grid that fills every multiprocessor
            # (the step keeps fewer blocks to leave room for the PME branches)
            full_ms = stages["pairs_full"]
            roof["kernel_ms_full_grid"] = full_ms
            roof["frac_full_grid"] = n_pairs * FLOPS_PER_PAIR / (full_ms * 1e-3) / 1e12 / peak
        # end to end through the public API with host buffers: one host-I/O
        # step call per step (host-to-device copy of the positions, the step,
        # and the device-to-host copies of positions, velocities and the
        # scalar state, replayed as one captured graph), from and into
        # page-locked memory.  An FP32 system's coordinates are floats on the
        # device, so the float variant (lfe_step_io_f32) moves them without
        # widening; the double variant is timed beside it.
        e2e = None
        if args.e2e_steps > 0:
            n = len(d["charge"])

            def time_io(dtype, call):
                pin_pos = torch.from_numpy(g.get_state()[0].astype(dtype)).pin_memory()
                pin_vel = torch.empty_like(pin_pos).pin_memory()
                ext_buf = np.zeros(lfe.NEXT)
                for _ in range(5):      # untimed: the first call captures its graph
                    call(pin_pos.data_ptr(), pin_pos.data_ptr(), pin_vel.data_ptr(), ext_buf.ctypes.data, stream)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(args.e2e_steps):
                    call(pin_pos.data_ptr(), pin_pos.data_ptr(), pin_vel.data_ptr(), ext_buf.ctypes.data, stream)
                return (time.perf_counter() - t0) / args.e2e_steps

            te64 = time_io(np.float64, g.step_io)
            if prec == lfe.LFE_FP32_MIXED:
                te = time_io(np.float32, g.step_io_f32)
                e2e = {"value": dt_ps * 1e-3 * 86400.0 / te, "unit": "ns/day",
                       "h2d_bytes_per_step": 3 * n * 4, "d2h_bytes_per_step": 6 * n * 4 + 16 * 8,
                       "calls": "lfe_step_io_f32 per step: float positions in, one step, float positions + "
                                "velocities and the FP64 scalar state out (page-locked host buffers)",
                       "value_double_buffers": dt_ps * 1e-3 * 86400.0 / te64}
            else:
                e2e = {"value": dt_ps * 1e-3 * 86400.0 / te64, "unit": "ns/day",
                       "h2d_bytes_per_step": 3 * n * 8, "d2h_bytes_per_step": 6 * n * 8 + 16 * 8,
                       "calls": "lfe_step_io per step: positions in, one step, positions + velocities + scalar "
                                "state out (page-locked host buffers)"}
        fp64 = None
        if not args.no_fp64 and prec == lfe.LFE_FP32_MIXED:
            # the FP64 form keeps the 0.10 nm list buffer: its pair kernel is
            # several times costlier, and the mixed system's tuned 0.22 nm
            # buffer measured slower for it (42.3 against 46.9 ns/day)
            g64 = lfe.System(d, precision=lfe.LFE_FP64, seed=2608)
            use_paper_thermostat(g64)
            g64.set_positions(pos)
            g64.set_velocities(vel)
            g64.step(5, stream)
            torch.cuda.synchronize()
            k64 = max(5, min(40, args.steps // 5))
            ms64 = time_steps(g64, k64, stream, flush)
            m64 = sum(ms64) / k64
            fp64 = {"ns_per_day": dt_ps * 1e-3 * 86400.0 / (m64 * 1e-3), "ms_per_step": m64, "steps": k64}
            g64.close()
        cpu, ocache = (None, {}) if args.no_cpu else cpu_baseline(d, dt_ps)
        errors = None
        if not args.no_errors:
            from paper_2608_12691_b300 import systems as S
            frames = {"c1_octanol" if args.workload == "octanol" else args.workload: (d, float(d["lam"]))}
            cache = {next(iter(frames)): ocache} if ocache else {}
            if args.workload == "octanol":
                c2 = S.make_c2(seed=2610)
                frames["c2_water"] = (c2, float(c2["lam"]))
                c4 = S.make_c4_frame(frame=5)
                frames["c4_flexible"] = (c4, float(c4["lam"]))
            errors = error_leg(frames, cache)
        batched = batched_leg(args, stream, flush) if args.batch_replicas > 1 else None
        dafed = dafed_leg(args, stream, flush) if not args.no_dafed else None
        out = {"metric": METRIC, "value": ns_day, "unit": "ns/day", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32" if prec == lfe.LFE_FP32_MIXED else "f64",
               "data": "synthetic",
               "config": run_config(d, desc),
               "precision": "FP32 arithmetic, int64 fixed-point force/energy sums, FP64 lambda/OPES"
               if prec == lfe.LFE_FP32_MIXED else "FP64",
               "parallelism": "replicas" if world > 1 else "single replica",
               "pairs_per_step": n_pairs, "tiles": n_tiles,
               "tile_efficiency": n_pairs / (256.0 * n_tiles) if n_tiles else None,
               "autotuned": dict(tune, eval_ms=tune_ms) if tune else None,
               "pair_interactions_per_s": n_pairs / (ms_step * 1e-3) * world,
               "wall_ms_per_step": wall / args.steps * 1e3,
               "neighbour_rebuilds": rebuilds,
               "gpu_launches": launches,
               "roofline": roof, "stages_ms": stages, "fp64": fp64, "batched": batched, "dafed": dafed,
               "cpu_baseline": cpu,
               "oracle_errors": errors,
               "e2e": e2e,
               "clocks": clocks, "lambda_end": ext1["lambda"], "theta_end": ext1["theta"]}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_profile_case(args):
    import torch
    from paper_2608_12691_b300 import lfe
    torch.cuda.set_device(0)
    d, _ = make_workload(args.workload, 0)
    prec = lfe.LFE_FP64 if args.precision == "fp64" else lfe.LFE_FP32_MIXED
    g = lfe.System(d, precision=prec, **({"skin": args.skin} if args.skin else {}))
    if args.prune:
        g.set_list_prune(args.prune)
    stages = g.time_stages(d["lam"], reps=3)
    _, _, ext = g.get_state()
    print(json.dumps({"profile_case": args.workload, "stages_ms": stages, "tiles": int(ext["n_tiles"])}))


def main():
    args = parse()
    if args.profile_case:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

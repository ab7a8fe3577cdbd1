#!/usr/bin/env python
"""Benchmark: changeover-kick pair-interactions/s and steps/s of the hybrid
symplectic step (Appendix A with the two-level changeover of Sec. 6.3) on the
large planetesimal disk: N = 65,536 equal-mass planetesimals (0.5-4 AU, 5 Earth
masses, Sigma ~ a^-1.5) plus 4 embryos of 0.1 Earth masses, dt = 6.0875 d,
2 symplectic levels x 10 sub-steps, FP64 and mixed-precision kick.

One step = genga_step(1): Rcrit, Kick + pre-check, HC, FG, detection, SEnc
(RcritS, KickS, FGS, detection, grouping, Bulirsch-Stoer per sub-step), HC,
Kick.  The headline value counts the two all-pairs kick evaluations of a step,
2 N (N - 1) pair interactions, divided by the measured whole-step time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank integrates its own replica of the disk
(the path has no exchange step: replicas only); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("changeover-kick G pair-interactions/s and steps/s at N=65536 (FP64 vs mixed), "
          "% of peak")
UNIT = "Gpair/s"
# FP64 instructions per pair interaction (ordered pair i <- j) that each kick
# form's algorithm needs (FMA counted as one), by layout.  Tiled (every ordered
# pair): mixed 6 -- displacement 3, accumulation 3 (r^2 in float-float from an
# exact split of the displacement, the FP32 rsqrt seed and its Newton
# correction and the correction terms all on the FP32 pipe; m y0^3 converted to
# FP64 by integer operations); FP64 17 -- CUDA's double rsqrt on an FP64 r^2,
# m r^-3 and the accumulation.  Symmetric (each unordered pair once, the force
# to both bodies): mixed 9 per unordered pair = 4.5 per interaction
# (displacement 3, accumulation 3 + 3); FP64 21 = 10.5 (displacement 3, r^2 3,
# Newton rsqrt 5, r^-3 2, two mass products 2, accumulation 3 + 3).
FP64_OPS_PER_PAIR = {("mixed", "tiled"): 6, ("fp64", "tiled"): 17,
                     ("mixed", "symmetric"): 4.5, ("fp64", "symmetric"): 10.5}
# The same counted by ncu on one launch at N = 65,536 (thread-level
# smsp__sass_thread_inst_executed_op_d{add,mul,fma}_pred_on.sum / N^2, and the
# warp-level sm__inst_executed_pipe_fp64.sum x 32 / N^2, which also charges the
# idle lanes of partly predicated warps); the mixed symmetric kick at the
# bench's N = 65,540 per interaction N (N - 1), where the padding of the last
# 128-body tile adds 0.4 % (4.553 at N = 65,536, thread and warp level alike);
# None where the kernel has changed since the count
FP64_INSTR_PER_PAIR_COUNTED = {("mixed", "tiled"): (6.152, 6.383), ("fp64", "tiled"): (17.091, 17.402),
                               ("mixed", "symmetric"): (4.571, 4.571), ("fp64", "symmetric"): (10.549, 10.605)}
# FP64 units per SM: GB300's nominal FP64 rate (1.25 TFLOP/s = 0.625 T FMA/s
# over 152 SMs at ~2.06 GHz) is 2 FP64 operations per clock per SM; ncu's FP64
# pipe utilisation is relative to this rate
FP64_OPS_PER_CLK_PER_SM = 2
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the mixed
# symmetric kick kernel at N = 65,540 (P = 4, 129 partial slots: the traffic is
# the partial sums); None when the kernel has changed since the capture
KICK_MIXED_DRAM_BYTES = 358854400


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=65536, help="planetesimals (embryos: 4 more)")
    ap.add_argument("--kick-reps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip e2e/cpu/fp64 legs (profiling runs)")
    ap.add_argument("--workload", choices=["disk", "ensemble", "adjoint", "variants", "tp", "kick"],
                    default="disk",
                    help="disk: the N=65,540 disk (headline); ensemble: 4096 compact systems "
                         "with GR and tides; adjoint: the 1000-step adjoint at N=4096; "
                         "variants: FP64 vs mixed on the N=16,384 disk (one level) and the "
                         "N=65,540 disk at other (levels, sub-steps); tp: the N=65,540 disk "
                         "with 4,096 large bodies and semi-active test particles; kick: the "
                         "all-pairs kick alone on a disk of --n planetesimals (0.5-4 AU, "
                         "5 M_earth), --kick-reps timed launches in the form --kick")
    ap.add_argument("--kick", choices=["fp64", "mixed"], default="mixed",
                    help="kick form of --workload kick")
    ap.add_argument("--kick-layout", choices=["auto", "tiled", "symmetric"], default="auto",
                    help="kick layout of --workload kick (auto: the library's choice for N)")
    ap.add_argument("--kick-p", type=int, default=0, help="symmetric layout super-range (0: chosen)")
    ap.add_argument("--kick-precheck", action="store_true",
                    help="--workload kick: each kick also records the close-encounter candidates")
    ap.add_argument("--ens-tile", default="",
                    help="threads,ctas_per_sm of the ensemble kernel instead of autotuning "
                         "(profiling runs)")
    ap.add_argument("--ens-steps", type=int, default=10000,
                    help="integration steps per timed ensemble launch (the configuration's 10,000)")
    ap.add_argument("--energy-run", type=int, default=0,
                    help="instead of timing: integrate this many steps in FP64 and mixed and "
                         "report the relative energy error every 100 steps")
    return ap.parse_args()


# ---------------------------------------------------------------- distributed plumbing
class Dist:
    """Replica bookkeeping for N processes (one per GPU): every rank integrates
    its own copy of the workload; the only collectives are the barriers around
    the timed region and the max of the ranks' times.  Backend: NCCL on GPUs,
    gloo for the CPU tests of this logic."""

    def __init__(self, ngpus: int, backend: str | None = None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        self.backend = backend or "nccl"
        if self.world > 1:
            import torch
            import torch.distributed as dist
            if self.backend == "nccl":
                torch.cuda.set_device(self.local)
                dist.init_process_group("nccl", device_id=torch.device("cuda", self.local))
            else:
                dist.init_process_group(self.backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        dev = f"cuda:{self.local}" if self.backend == "nccl" else "cpu"
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def replica_throughput(world: int, units_per_step: float, steps: int, t_max_ms: float) -> float:
    """Whole-job throughput of `world` replicas: the units all ranks processed
    divided by the slowest rank's time (units per second)."""
    return world * units_per_step * steps / (t_max_ms * 1e-3)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.rows = []
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                if self.uuid and parts[1] != self.uuid:
                    continue
                rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        smax = max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k] == "Active"})
        # only samples under load (clock above 60% of max) enter the median
        loaded = [v for v in sm if v > 0.6 * smax] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows)}


def gpu_uuid(dev_index: int) -> str | None:
    try:
        import torch
        u = torch.cuda.get_device_properties(dev_index).uuid
        return "GPU-" + str(u)
    except Exception:
        return None


# ---------------------------------------------------------------- our arm
def run_ours(args, dist: Dist) -> dict | None:
    import torch

    from paper_2201_10058_gb300 import genga
    from workloads import disk
    from workloads.disk import SEED_BASE

    dev = torch.device("cuda", dist.local)
    torch.cuda.set_device(dev)
    genga.load()
    wl = disk(args.n, 0.5, 4.0, 5.0, SEED_BASE + 2, n_embryos=4, m_embryo_earth=0.1,
              slevels=2, substeps=10, name=f"disk{args.n}+4emb")
    n = wl.n
    pairs_per_step = 2.0 * n * (n - 1)
    x0 = torch.tensor(np.ascontiguousarray(wl.x.T), device=dev)
    v0 = torch.tensor(np.ascontiguousarray(wl.v.T), device=dev)
    mass = torch.tensor(wl.m, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    rates = genga.measure_pipe_rates()      # FP64 / FP32 / MUFU ops per clock per SM
    fp64_lat = genga.measure_fp64_latency()  # cycles per dependent FP64 FMA (warp, one lane)

    def params(prec):
        return genga.default_params(G=wl.G, m_star=wl.m_star, dt=wl.dt, n1=wl.n1, n2=wl.n2,
                                    f_pc=wl.f_pc, slevels=wl.slevels, substeps=wl.substeps,
                                    precision=prec)

    results = {}
    clocks = None
    launches = 0
    final_state = None
    precisions = ["mixed"] if args.quick else ["fp64", "mixed"]
    for name in precisions:
        prec = genga.GENGA_MIXED if name == "mixed" else genga.GENGA_FP64
        pos, vel = x0.clone(), v0.clone()
        sysm = genga.System(pos, vel, mass, params(prec), stream=stream)
        E_start, _ = sysm.energy()                # outside the timed region
        for _ in range(args.warmup):
            sysm.step(1)
        torch.cuda.synchronize()
        sampler = ClockSampler(gpu_uuid(dist.local)) if name == "mixed" else None
        if sampler:
            sampler.start()
        dist.barrier()
        torch.cuda.synchronize()
        per_step = []
        nl = 0
        syncs = 0
        for _ in range(args.steps):
            flush.fill_(1.0)                      # L2 flush between timed steps (untimed)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sysm.step(1)
            e1.record(stream)
            e1.synchronize()
            per_step.append(e0.elapsed_time(e1))
            st = sysm.stats()
            nl += st["kernel_launches"]
            syncs += st["host_syncs"]
        torch.cuda.synchronize()
        dist.barrier()
        total_ms = sum(per_step)
        stats = sysm.stats()
        if name == "mixed":
            final_state = (pos.cpu().numpy().copy(), vel.cpu().numpy().copy())
        E_end, _ = sysm.energy()
        # the kick alone (the dominant kernel), same launch configuration; the
        # accelerations are written out so that the partial sums are folded
        sysm.rcrit(wl.dt)
        acc = torch.empty((3, n), dtype=torch.float64, device=dev)
        sysm.kick(0.0, precheck=False, acc_out=acc)
        torch.cuda.synchronize()
        k0 = torch.cuda.Event(enable_timing=True)
        k1 = torch.cuda.Event(enable_timing=True)
        k0.record(stream)
        for _ in range(args.kick_reps):
            sysm.kick(0.0, precheck=False, acc_out=acc)
        k1.record(stream)
        k1.synchronize()
        kick_ms = k0.elapsed_time(k1) / args.kick_reps
        lay = sysm.kick_layout()
        layout = "symmetric" if lay["layout"] == genga.GENGA_KICK_SYMMETRIC else "tiled"
        if sampler:
            clocks = sampler.stop()
        t_max = dist.max(total_ms)
        sysm.close()
        # where the time goes: the same step window again on a new system,
        # with CUDA events at the phase boundaries of each step (kept out of
        # the timed steps above, whose time they would add to)
        pos, vel = x0.clone(), v0.clone()
        sysm = genga.System(pos, vel, mass, params(prec), stream=stream)
        for _ in range(args.warmup):
            sysm.step(1)
        sysm.set_timing(True)
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            sysm.step(1)
        phases, nph = sysm.phase_ms()
        sysm.set_timing(False)
        ph_step = {k: v / max(nph, 1) for k, v in phases.items()}
        kick_ph = ph_step["kick1"] + ph_step["kick2"]
        results[name] = {
            "ms_per_step": t_max / args.steps,
            "gpairs_per_s": replica_throughput(dist.world, pairs_per_step, args.steps, t_max) / 1e9,
            "steps_per_s": replica_throughput(dist.world, 1.0, args.steps, t_max),
            "kick_ms": kick_ms,
            "kick_layout": dict(lay, name=layout),
            "kick_gpairs_per_s": n * (n - 1) / (kick_ms * 1e-3) / 1e9,
            "kick_share": 2 * kick_ms / (total_ms / args.steps),
            "energy_rel_err": abs(E_end - E_start) / abs(E_start),
            "per_step": {"min_ms": round(min(per_step), 3),
                         "median_ms": round(statistics.median(per_step), 3),
                         "max_ms": round(max(per_step), 3),
                         "ms": [round(v, 3) for v in per_step]},
            "phases": {"ms_per_step": {k: round(v, 4) for k, v in ph_step.items()},
                       "sum_ms_per_step": round(sum(ph_step.values()), 3),
                       "kick_ms_per_step": round(kick_ph, 3),
                       "non_kick_ms_per_step": round(sum(ph_step.values()) - kick_ph, 3),
                       "non_kick_share": round(1.0 - kick_ph / max(sum(ph_step.values()), 1e-9), 4),
                       "host_syncs_per_step": syncs / args.steps,
                       "launches_per_step": nl / args.steps,
                       "definition": "device time between CUDA events recorded on the system's "
                                     "stream at the phase boundaries of each step of the same "
                                     "step window (warm-up and timed counts as above), in a "
                                     "separate untimed pass; includes the GPU's waits for the "
                                     "host inside a phase"},
            "encounters": {"candidates_per_step": stats["n_candidates"],
                           "pairs_level0": stats["n_pairs"][0],
                           "pairs_level1": stats["n_pairs"][1],
                           "groups": stats["n_groups"], "max_group": stats["max_group"],
                           "bs_max_attempts": stats["bs_max_attempts"]},
        }
        if name == "mixed":
            launches = nl
        sysm.close()

    # e2e through the C ABI with host buffers (pinned), copies inside the timed
    # region: the same warm-up count from the same initial state, so the timed
    # steps are the same steps as above
    e2e = None
    if not args.quick:
        pos, vel = x0.clone(), v0.clone()
        sysm = genga.System(pos, vel, mass, params(genga.GENGA_MIXED), stream=stream)
        xh = torch.empty((3, n), dtype=torch.float64).pin_memory()
        vh = torch.empty((3, n), dtype=torch.float64).pin_memory()
        xh.copy_(x0.cpu())
        vh.copy_(v0.cpu())
        for _ in range(args.warmup):
            sysm.step_host_ptr(xh.data_ptr(), vh.data_ptr(), 1)
        torch.cuda.synchronize()
        dist.barrier()
        te = 0.0
        for _ in range(args.steps):
            flush.fill_(1.0)                      # untimed, as in the device-timed leg
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sysm.step_host_ptr(xh.data_ptr(), vh.data_ptr(), 1)
            te += time.perf_counter() - t0
        dist.barrier()
        te = dist.max(te)
        bytes_each = 2 * 3 * n * 8
        same = (final_state is not None and np.array_equal(xh.numpy(), final_state[0])
                and np.array_equal(vh.numpy(), final_state[1]))
        e2e = {"value": dist.world * pairs_per_step * args.steps / te / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": bytes_each, "d2h_bytes_per_step": bytes_each,
               "ms_per_step": round(1e3 * te / args.steps, 3),
               "same_steps_as_value": bool(same),
               "timing": "host wall clock around genga_step_host (copy in, step, copy out, "
                         "synchronise) for each of the same timed steps; L2 flushed between "
                         "them (untimed)"}
        sysm.close()

    if dist.rank != 0:
        return None

    head = results["mixed"]
    sm_clock = (clocks or {}).get("sm_mhz") or 2070.0
    props = torch.cuda.get_device_properties(dev)
    nsm = props.multi_processor_count
    peak = FP64_OPS_PER_CLK_PER_SM * nsm * sm_clock * 1e6 / 1e9
    probe_peak = rates["dfma"] * nsm * sm_clock * 1e6 / 1e9
    lay = head["kick_layout"]["name"]
    ops = FP64_OPS_PER_PAIR[("mixed", lay)]
    achieved = ops * head["kick_gpairs_per_s"]
    counted = FP64_INSTR_PER_PAIR_COUNTED[("mixed", lay)]
    kname = "kick_sym_kernel<mixed>" if lay == "symmetric" else "kick_kernel<mixed>"
    line = {
        "metric": METRIC, "value": round(head["gpairs_per_s"], 4), "unit": UNIT,
        "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(head["ms_per_step"], 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32 (mixed kick)",
        "data": "synthetic (seeded planetesimal disk, no external data)",
        "config": {"workload": f"disk N={n} (65536 planetesimals 0.5-4 AU, 5 M_earth, "
                               f"+4 embryos 0.1 M_earth), dt=6.0875 d, 2 levels x 10 substeps, "
                               f"mixed-precision kick",
                   "n_bodies": n, "slevels": 2, "substeps": 10, "kick": "mixed",
                   "pairs_per_step": pairs_per_step,
                   "l2": "flushed between timed steps (256 MiB write, untimed)",
                   "parallelism": f"replicas x{dist.world}"},
        "steps_per_s": round(head["steps_per_s"], 4),
        "per_step": head["per_step"],
        "phases": head["phases"],
        "kick_only": {"mixed_gpairs_per_s": round(head["kick_gpairs_per_s"], 3),
                      "mixed_kick_ms": round(head["kick_ms"], 3),
                      "kick_share_of_step": round(head["kick_share"], 3)},
        "roofline": {"bound": "alu", "kernel": f"{kname} (all-pairs changeover kick, {lay} layout)",
                     "achieved": round(achieved, 2), "peak": round(peak, 2),
                     "unit": "G FP64-op/s (FMA = 1; FP64 pipe)",
                     "frac": round(achieved / peak, 4),
                     "traffic": KICK_MIXED_DRAM_BYTES,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch "
                                       "of this kernel (no pre-check) at N=65540, P=4: the partial sums",
                     "ops_per_pair": ops,
                     "kick_layout": head["kick_layout"],
                     "duration_basis": "CUDA events on the system's stream around genga_kick writing the "
                                       "accelerations (pack, kick kernel, fold of the partial sums), "
                                       "averaged over the repetitions",
                     "peak_basis": f"derived: {FP64_OPS_PER_CLK_PER_SM} FP64 op/clk/SM (GB300 nominal "
                                   f"FP64 unit count) x {nsm} SMs x {sm_clock:.0f} MHz (median SM "
                                   f"clock under load)",
                     "frac_counted": None if counted is None else
                     {"thread_level": round(counted[0] * head["kick_gpairs_per_s"] / peak, 4),
                      "warp_level": round(counted[1] * head["kick_gpairs_per_s"] / peak, 4),
                      "instr_per_pair": list(counted)},
                     "probe": {"peak": round(probe_peak, 2),
                               "frac": round(achieved / probe_peak, 4),
                               "basis": f"{rates['dfma']:.3f} FP64 FMA/clk/SM reached by independent "
                                        f"FMA chains (genga_measure_pipe_rates, this run)"},
                     "pipe_rates_per_clk_sm": {k: round(v, 3) for k, v in rates.items()},
                     "fp64_dependent_fma_cycles": {k: round(v, 2) for k, v in fp64_lat.items()}},
        "clocks": clocks, "gpu_launches": launches, "e2e": e2e,
        "encounters": head["encounters"],
        "energy": {"rel_err": head["energy_rel_err"], "steps": args.warmup + args.steps,
                   "definition": "|E_end - E_start| / |E_start| over this run's warm-up and timed "
                                 "steps (compensated FP64 energy, outside the timed region)"},
    }
    if "fp64" in results:
        f = results["fp64"]
        line["fp64"] = {"value": round(f["gpairs_per_s"], 4), "unit": UNIT, "dtype": "f64",
                        "ms_per_step": round(f["ms_per_step"], 3),
                        "steps_per_s": round(f["steps_per_s"], 4),
                        "per_step": {k: v for k, v in f["per_step"].items() if k != "ms"},
                        "non_kick_ms_per_step": f["phases"]["non_kick_ms_per_step"],
                        "kick_gpairs_per_s": round(f["kick_gpairs_per_s"], 3),
                        "kick_ms": round(f["kick_ms"], 3),
                        "roofline_frac": round(FP64_OPS_PER_PAIR[("fp64", f["kick_layout"]["name"])]
                                               * f["kick_gpairs_per_s"] / peak, 4),
                        "ops_per_pair": FP64_OPS_PER_PAIR[("fp64", f["kick_layout"]["name"])],
                        "kick_layout": f["kick_layout"],
                        "energy_rel_err": f["energy_rel_err"]}
        line["mixed_over_fp64"] = round(head["gpairs_per_s"] / f["gpairs_per_s"], 3)
    if not args.no_cpu_baseline and not args.quick and dist.world == 1:
        line["cpu_baseline"] = cpu_baseline(wl)
    return line


# ---------------------------------------------------------------- oracle legs
def _oracle_step_sample(wl, nthreads: int) -> tuple[float, dict]:
    import oracle as O
    p = O.make_params(wl, nthreads=nthreads)
    t0 = time.perf_counter()
    _, _, status, st = O.step(wl.x, wl.v, wl.m, p, 1)
    return time.perf_counter() - t0, st


def cpu_baseline(wl) -> dict:
    """The oracle as it stands: one full step of the same workload on all host cores."""
    cores = os.cpu_count() or 1
    dt, st = _oracle_step_sample(wl, cores)
    n = wl.n
    return {"value": round(2.0 * n * (n - 1) / dt / 1e9, 5), "unit": UNIT, "cores": cores,
            "kind": "oracle", "sample": f"1 full step (Appendix A, 2 levels x 10 substeps) of the "
                                        f"N={n} disk; {dt:.1f} s wall on {cores} threads",
            "seconds": round(dt, 2)}


def run_reference(args, dist: Dist) -> dict | None:
    """Reference arm: the FP64 CPU oracle, timed on the host cores on the same
    workload, metric and unit; each timed step is one full oracle step."""
    if dist.rank != 0:
        return None
    from workloads import disk
    from workloads.disk import SEED_BASE
    wl = disk(args.n, 0.5, 4.0, 5.0, SEED_BASE + 2, n_embryos=4, m_embryo_earth=0.1,
              slevels=2, substeps=10, name=f"disk{args.n}+4emb")
    import oracle as O
    cores = os.cpu_count() or 1
    # untimed warm-up: build and load the oracle, touch the data
    O.lib()
    O.rcrit(wl.x, wl.v, wl.m, wl.m_star, wl.dt)
    total = 0.0
    for _ in range(args.steps):
        dt, st = _oracle_step_sample(wl, cores)
        total += dt
    n = wl.n
    value = 2.0 * n * (n - 1) * args.steps / total / 1e9
    return {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT,
            "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * total / args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded planetesimal disk)",
            "config": {"workload": f"disk N={n} ({n - 4} planetesimals 0.5-4 AU, 5 M_earth, "
                                   f"+4 embryos 0.1 M_earth), dt=6.0875 d, 2 levels x 10 substeps",
                       "n_bodies": n},
            "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} full oracle steps of the N={n} disk from the "
                                       f"initial state, {cores} threads"},
            "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def energy_run(args) -> dict:
    """Relative energy error of the FP64 and mixed kicks along the same run."""
    import torch

    from paper_2201_10058_gb300 import genga
    from workloads import disk
    from workloads.disk import SEED_BASE
    genga.load()
    wl = disk(args.n, 0.5, 4.0, 5.0, SEED_BASE + 2, n_embryos=4, m_embryo_earth=0.1,
              slevels=2, substeps=10, name=f"disk{args.n}+4emb")
    dev = torch.device("cuda", 0)
    out = {"n_bodies": wl.n, "steps": args.energy_run, "every": 100}
    traj = {}
    for name, prec in (("fp64", genga.GENGA_FP64), ("mixed", genga.GENGA_MIXED)):
        pos = torch.tensor(np.ascontiguousarray(wl.x.T), device=dev)
        vel = torch.tensor(np.ascontiguousarray(wl.v.T), device=dev)
        mass = torch.tensor(wl.m, device=dev)
        p = genga.default_params(G=wl.G, m_star=wl.m_star, dt=wl.dt, n1=wl.n1, n2=wl.n2,
                                 f_pc=wl.f_pc, slevels=wl.slevels, substeps=wl.substeps,
                                 precision=prec)
        s = genga.System(pos, vel, mass, p)
        E0, L0 = s.energy()
        rows = [(0, 0.0)]
        t0 = time.perf_counter()
        done = 0
        while done < args.energy_run:
            k = min(100, args.energy_run - done)
            s.step(k)
            done += k
            E, L = s.energy()
            rows.append((done, (E - E0) / abs(E0)))
        traj[name] = {"E0": E0, "dE_rel": rows, "seconds": time.perf_counter() - t0}
        s.close()
    diffs = [abs(a[1] - b[1]) for a, b in zip(traj["fp64"]["dE_rel"], traj["mixed"]["dE_rel"])]
    out.update(traj)
    out["max_abs_dE_rel_fp64"] = max(abs(r[1]) for r in traj["fp64"]["dE_rel"])
    out["max_abs_dE_rel_mixed"] = max(abs(r[1]) for r in traj["mixed"]["dE_rel"])
    out["max_mixed_minus_fp64"] = max(diffs)
    return out


def run_ensemble(args) -> dict:
    """Configuration 3: 4096 compact systems, GR + tides, one persistent launch per
    timed step (args.ens_steps integration steps each, 10,000 as configured),
    tile shape autotuned; the FP64 and the mixed-precision pair kick."""
    import torch

    from paper_2201_10058_gb300 import genga
    from workloads.ensemble import ensemble
    genga.load()
    wl = ensemble(4096)
    sizes = np.diff(wl.offsets)
    pairs_per_step = float((2 * sizes * (sizes - 1)).sum())
    rates = genga.measure_pipe_rates()
    sampler = ClockSampler(gpu_uuid(0))
    sampler.start()
    stream = torch.cuda.current_stream()
    legs = {}
    for name, prec in (("fp64", genga.GENGA_FP64), ("mixed", genga.GENGA_MIXED)):
        ens = genga.Ensemble(wl, genga.default_params(G=wl.G, precision=prec))
        if args.ens_tile:
            threads, ctas = (int(v) for v in args.ens_tile.split(","))
            ens.set_tile(threads, ctas)
        else:
            threads, ctas = ens.autotune(20)
        for _ in range(args.warmup):
            ens.step(args.ens_steps)
        torch.cuda.synchronize()
        total = 0.0
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ens.step(args.ens_steps)
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        st = ens.stats()
        steps = args.steps * args.ens_steps
        legs[name] = {"value": round(wl.n_systems * steps / (total * 1e-3), 1), "unit": "system-steps/s",
                      "ms_per_launch": round(total / args.steps, 3),
                      "pair_gpairs_per_s": round(pairs_per_step * steps / (total * 1e-3) / 1e9, 3),
                      "tile": {"threads": threads, "ctas_per_sm": ctas},
                      "encounters": {"candidates": st["n_candidates"], "pairs": st["n_pairs"][0],
                                     "groups": st["n_groups"]}}
        ens.close()
    clocks = sampler.stop()
    head = legs["mixed"]
    return {"metric": "ensemble system-steps/s (4096 compact systems, GR + tides)",
            "value": head["value"], "unit": "system-steps/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_launch"],
            "higher_is_better": True, "dtype": "f64+f32 (mixed pair kick)",
            "data": "synthetic (seeded ensemble)",
            "config": {"workload": f"ensemble of {wl.n_systems} systems, N 8-64 (total "
                                   f"{int(wl.offsets[-1])} bodies), GR + tides, "
                                   f"{args.ens_steps} steps per launch"},
            "mixed": head, "fp64": legs["fp64"],
            "mixed_over_fp64": round(head["value"] / legs["fp64"]["value"], 3),
            "pipe_rates_per_clk_sm": {k: round(v, 3) for k, v in rates.items()}, "clocks": clocks}


def run_adjoint(args) -> dict:
    """Configuration 4: N = 4096 disk (0.5-2 AU, 2 Earth masses), 1000 steps with
    frozen encounters, FP64 checkpoints every 100 steps; forward (recording) and
    hand-written backward timed.  Finite-difference check (h = 1e-7, central) of
    one directional derivative over the first checkpoint segment (100 steps) of
    the same recording: over all 1000 steps the disk's close encounters amplify
    a 1e-7 perturbation far beyond the linear regime (see grad_norms), so a
    difference quotient there measures curvature, not the derivative."""
    import torch

    from paper_2201_10058_gb300 import genga
    from workloads import config_workload
    genga.load()
    wl = config_workload(4)
    nsteps, every = 1000, 100
    dev = torch.device("cuda", 0)
    T = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)
    p = genga.default_params(G=wl.G, m_star=wl.m_star, dt=wl.dt)
    pos, vel, mass = T(wl.x.T), T(wl.v.T), T(wl.m)
    s = genga.System(pos, vel, mass, p)
    t0 = time.perf_counter()
    s.adjoint_forward(nsteps, every)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    st_fwd = s.stats()
    rng = np.random.default_rng(11)
    lx, lv = T(rng.standard_normal((3, wl.n))), T(rng.standard_normal((3, wl.n)))
    t0 = time.perf_counter()
    gx, gv, gm = s.adjoint_backward(lx, lv)
    torch.cuda.synchronize()
    t_bwd = time.perf_counter() - t0
    rc_all, pairs_all = _recording(s)
    s.close()

    # directional derivative over the first segment: adjoint vs central differences
    nseg = every
    rc_seg, pairs_seg = rc_all[:nseg], pairs_all[:nseg]
    dx0 = rng.standard_normal((3, wl.n))
    dv0 = rng.standard_normal((3, wl.n)) * 0.017
    dm0 = rng.standard_normal(wl.n) * wl.m
    h = 1e-7

    def replay(eps):
        sp, sv, sm = T(wl.x.T + eps * dx0), T(wl.v.T + eps * dv0), T(wl.m + eps * dm0)
        s2 = genga.System(sp, sv, sm, p)
        s2.adjoint_load(10, rc_seg, pairs_seg)
        return s2, sp, sv

    s2, _, _ = replay(0.0)
    t0 = time.perf_counter()
    ax, av, am = s2.adjoint_backward(lx, lv)
    torch.cuda.synchronize()
    t_bwd_seg = time.perf_counter() - t0
    s2.close()
    lxn, lvn = lx.cpu().numpy(), lv.cpu().numpy()
    ad = float((ax.cpu().numpy() * dx0).sum() + (av.cpu().numpy() * dv0).sum()
               + (am.cpu().numpy() * dm0).sum())
    fds = []
    for hh in (1e-7, 1e-8, 1e-9):
        fin = []
        for eps in (hh, -hh):
            s3, sp, sv = replay(eps)
            fin.append((sp.cpu().numpy(), sv.cpu().numpy()))
            s3.close()
        fdh = ((lxn * (fin[0][0] - fin[1][0])).sum() + (lvn * (fin[0][1] - fin[1][1])).sum()) / (2 * hh)
        fds.append({"h": hh, "central_difference": fdh, "rel_diff": abs(ad - fdh) / abs(ad)})
    fd = fds[0]["central_difference"]
    return {"metric": "adjoint of 1000 kick-drift-kick steps (frozen encounters), N=4096",
            "forward_s": round(t_fwd, 3), "backward_s": round(t_bwd, 3),
            "backward_over_forward": round(t_bwd / t_fwd, 2),
            "forward_steps_per_s": round(nsteps / t_fwd, 2),
            "checkpoint_every": every, "n_bodies": wl.n,
            "encounters": {"pairs_per_step": st_fwd["n_pairs"][0] / nsteps,
                           "largest_group": st_fwd["max_group"],
                           "bs_attempts": st_fwd["bs_steps"] + st_fwd["bs_rejects"],
                           "bs_max_attempts_one_call": st_fwd["bs_max_attempts"]},
            "grad_norms": {"x0": float(gx.norm()), "v0": float(gv.norm()), "m": float(gm.norm())},
            "fd_check": {"steps": nseg, "h": h, "direction": "x0, v0 and m together",
                         "adjoint": ad, "central_difference": fd,
                         "rel_diff": abs(ad - fd) / abs(ad), "backward_s": round(t_bwd_seg, 3),
                         "by_h": fds},
            "dtype": "f64", "data": "synthetic (seeded disk)"}


def _timed_steps(genga, sysm, flush, stream, steps: int, warmup: int) -> float:
    """Mean device time (ms) of one whole step, L2 flushed before each timed step."""
    import torch
    for _ in range(warmup):
        sysm.step(1)
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sysm.step(1)
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    return total / steps


def run_variants(args) -> dict:
    """Secondary measurements beside the headline: the N = 16,384 disk (0.5-2 AU,
    2 Earth masses, one level) with the FP64 and the mixed kick, and the N = 65,540
    disk of the headline at other (levels, sub-steps) choices of Sec. 6.3.  Same
    timing rules as the headline (device events, L2 flushed between timed steps)."""
    import torch

    from paper_2201_10058_gb300 import genga
    from workloads import config_workload, disk
    from workloads.disk import SEED_BASE

    dev = torch.device("cuda", 0)
    genga.load()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    sampler = ClockSampler(gpu_uuid(0))
    sampler.start()

    def system(wl, prec, slevels, substeps):
        pos = torch.tensor(np.ascontiguousarray(wl.x.T), device=dev)
        vel = torch.tensor(np.ascontiguousarray(wl.v.T), device=dev)
        mass = torch.tensor(wl.m, device=dev)
        p = genga.default_params(G=wl.G, m_star=wl.m_star, dt=wl.dt, n1=wl.n1, n2=wl.n2,
                                 f_pc=wl.f_pc, slevels=slevels, substeps=substeps, precision=prec)
        return genga.System(pos, vel, mass, p, stream=stream)

    def kick_ms(sysm, wl, reps=5):
        sysm.rcrit(wl.dt)
        sysm.kick(0.0, precheck=False)
        torch.cuda.synchronize()
        k0 = torch.cuda.Event(enable_timing=True)
        k1 = torch.cuda.Event(enable_timing=True)
        k0.record(stream)
        for _ in range(reps):
            sysm.kick(0.0, precheck=False)
        k1.record(stream)
        k1.synchronize()
        return k0.elapsed_time(k1) / reps

    out = {"metric": "secondary measurements (not the headline)", "unit": UNIT, "dtype": "f64",
           "data": "synthetic (seeded disks)", "l2": "flushed between timed steps (256 MiB write)"}
    wl = config_workload(1)
    n = wl.n
    c1 = {"workload": f"disk N={n} (0.5-2 AU, 2 M_earth), dt=6.0875 d, one level",
          "steps": args.steps, "warmup": args.warmup}
    for name, prec in (("fp64", genga.GENGA_FP64), ("mixed", genga.GENGA_MIXED)):
        sysm = system(wl, prec, 1, 1)
        ms = _timed_steps(genga, sysm, flush, stream, args.steps, args.warmup)
        st = sysm.stats()
        km = kick_ms(sysm, wl)
        c1[name] = {"gpairs_per_s": round(2.0 * n * (n - 1) / (ms * 1e-3) / 1e9, 3),
                    "ms_per_step": round(ms, 3), "steps_per_s": round(1e3 / ms, 2),
                    "kick_ms": round(km, 3),
                    "kick_gpairs_per_s": round(n * (n - 1) / (km * 1e-3) / 1e9, 3),
                    "pairs_level0": st["n_pairs"][0], "max_group": st["max_group"]}
        sysm.close()
    c1["mixed_over_fp64"] = round(c1["fp64"]["ms_per_step"] / c1["mixed"]["ms_per_step"], 3)
    out["disk16384"] = c1
    wl = disk(65536, 0.5, 4.0, 5.0, SEED_BASE + 2, n_embryos=4, m_embryo_earth=0.1,
              slevels=2, substeps=10, name="disk65536+4emb")
    n = wl.n
    lv = []
    for slevels, substeps in ((1, 1), (2, 10), (3, 2), (3, 10)):
        sysm = system(wl, genga.GENGA_MIXED, slevels, substeps)
        ms = _timed_steps(genga, sysm, flush, stream, args.steps, args.warmup)
        st = sysm.stats()
        lv.append({"slevels": slevels, "substeps": substeps, "ms_per_step": round(ms, 3),
                   "gpairs_per_s": round(2.0 * n * (n - 1) / (ms * 1e-3) / 1e9, 3),
                   "steps_per_s": round(1e3 / ms, 3),
                   "pairs_per_level": [st["n_pairs"][k] for k in range(slevels)],
                   "max_group": st["max_group"], "bs_max_attempts": st["bs_max_attempts"]})
        sysm.close()
    out["disk65540_levels"] = {"workload": f"disk N={n} (headline disk), mixed kick",
                               "steps": args.steps, "warmup": args.warmup, "runs": lv}
    # the self-tuner on the same candidates (one untimed and 2 timed steps each)
    cands = [(r["slevels"], r["substeps"]) for r in lv]
    sysm = system(wl, genga.GENGA_MIXED, 1, 1)
    best, ms = sysm.tune_levels(cands, trial_steps=2)
    sysm.close()
    out["disk65540_levels"]["tuned"] = {"choice": list(cands[best]),
                                        "trial_ms_per_step": [round(float(v), 3) for v in ms]}
    out["clocks"] = sampler.stop()
    return out


def run_tp(args) -> dict:
    """The headline disk in the semi-active test-particle mode (Sec. 8.1): the 4
    embryos and the first 4,092 planetesimals are the large bodies (moved to the
    front), the other 61,444 planetesimals test particles.  Mixed kick, 2 levels x
    10 sub-steps, the headline's timing rules."""
    import torch

    from paper_2201_10058_gb300 import genga
    from workloads import disk
    from workloads.disk import SEED_BASE

    dev = torch.device("cuda", 0)
    genga.load()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    wl = disk(65536, 0.5, 4.0, 5.0, SEED_BASE + 2, n_embryos=4, m_embryo_earth=0.1,
              slevels=2, substeps=10, name="disk65536+4emb")
    n, nm = wl.n, 4096
    order = np.r_[np.arange(n - 4, n), np.arange(n - 4)]
    x, v, m = wl.x[order], wl.v[order], wl.m[order]
    pos = torch.tensor(np.ascontiguousarray(x.T), device=dev)
    vel = torch.tensor(np.ascontiguousarray(v.T), device=dev)
    mass = torch.tensor(m, device=dev)
    p = genga.default_params(G=wl.G, m_star=wl.m_star, dt=wl.dt, n1=wl.n1, n2=wl.n2, f_pc=wl.f_pc,
                             slevels=2, substeps=10, precision=genga.GENGA_MIXED, tp_mode=2,
                             n_massive=nm)
    sampler = ClockSampler(gpu_uuid(0))
    sampler.start()
    sysm = genga.System(pos, vel, mass, p, stream=stream)
    ms = _timed_steps(genga, sysm, flush, stream, args.steps, args.warmup)
    st = sysm.stats()
    sysm.rcrit(wl.dt)
    sysm.kick(0.0, precheck=False)
    torch.cuda.synchronize()
    k0 = torch.cuda.Event(enable_timing=True)
    k1 = torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(5):
        sysm.kick(0.0, precheck=False)
    k1.record(stream)
    k1.synchronize()
    kick_ms = k0.elapsed_time(k1) / 5
    sysm.close()
    evals = nm * (n - 1) + (n - nm) * nm        # pair evaluations of one kick
    return {"metric": "semi-active test-particle mode (secondary measurement)",
            "workload": f"disk N={n}: {nm} large bodies (4 embryos first), {n - nm} test particles; "
                        f"mixed kick, 2 levels x 10 sub-steps",
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
            "steps_per_s": round(1e3 / ms, 3), "kick_ms": round(kick_ms, 3),
            "kick_pair_evaluations": evals,
            "kick_gpairs_per_s": round(evals / (kick_ms * 1e-3) / 1e9, 3),
            "candidates_per_step": st["n_candidates"], "pairs_per_level": st["n_pairs"][:2],
            "max_group": st["max_group"], "clocks": sampler.stop()}


def run_kick(args) -> dict:
    """The all-pairs kick alone (one warm-up launch, then --kick-reps timed
    launches) on a disk of --n planetesimals, in the form --kick."""
    import torch

    from paper_2201_10058_gb300 import genga
    from workloads import disk
    from workloads.disk import SEED_BASE

    dev = torch.device("cuda", 0)
    genga.load()
    stream = torch.cuda.current_stream(dev)
    wl = disk(args.n, 0.5, 4.0, 5.0, SEED_BASE + 2, name=f"disk{args.n}")
    pos = torch.tensor(np.ascontiguousarray(wl.x.T), device=dev)
    vel = torch.tensor(np.ascontiguousarray(wl.v.T), device=dev)
    mass = torch.tensor(wl.m, device=dev)
    prec = genga.GENGA_MIXED if args.kick == "mixed" else genga.GENGA_FP64
    p = genga.default_params(G=wl.G, m_star=wl.m_star, dt=wl.dt, n1=wl.n1, n2=wl.n2, f_pc=wl.f_pc,
                             precision=prec)
    sysm = genga.System(pos, vel, mass, p, stream=stream)
    sysm.set_kick_layout({"auto": genga.GENGA_KICK_AUTO, "tiled": genga.GENGA_KICK_TILED,
                          "symmetric": genga.GENGA_KICK_SYMMETRIC}[args.kick_layout], args.kick_p)
    lay = sysm.kick_layout()
    sysm.rcrit(wl.dt)
    acc = torch.empty((3, wl.n), dtype=torch.float64, device=dev)
    sysm.kick(0.0, precheck=args.kick_precheck, acc_out=acc)
    torch.cuda.synchronize()
    k0 = torch.cuda.Event(enable_timing=True)
    k1 = torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(args.kick_reps):
        sysm.kick(0.0, precheck=args.kick_precheck, acc_out=acc)
    k1.record(stream)
    k1.synchronize()
    ms = k0.elapsed_time(k1) / args.kick_reps
    sysm.close()
    n = wl.n
    return {"metric": "all-pairs changeover kick alone (secondary measurement)", "kick": args.kick,
            "n_bodies": n, "launches": args.kick_reps, "ms_per_launch": round(ms, 4), "layout": lay,
            "precheck": bool(args.kick_precheck),
            "gpairs_per_s": round(n * (n - 1) / (ms * 1e-3) / 1e9, 3)}


def _recording(s):
    """Host copies of a system's recorded rc history and pair lists."""
    return s.adjoint_export()


def main():
    args = parse()
    if args.workload == "adjoint" and args.impl == "ours":
        print(json.dumps(run_adjoint(args)))
        return
    if args.workload == "tp" and args.impl == "ours":
        print(json.dumps(run_tp(args)))
        return
    if args.workload == "kick" and args.impl == "ours":
        print(json.dumps(run_kick(args)))
        return
    if args.workload == "variants" and args.impl == "ours":
        print(json.dumps(run_variants(args)))
        return
    if args.workload == "ensemble" and args.impl == "ours":
        print(json.dumps(run_ensemble(args)))
        return
    if args.energy_run:
        print(json.dumps(energy_run(args)))
        return
    dist = Dist(args.gpus)
    try:
        line = run_reference(args, dist) if args.impl == "reference" else run_ours(args, dist)
        if line is not None and dist.rank == 0:
            print(json.dumps(line))
    finally:
        dist.close()


if __name__ == "__main__":
    main()

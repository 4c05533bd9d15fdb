"""Benchmark of the VL+CT ideal-MHD step on GB300 (cell-updates/s).

Workload (default): the 512^3 periodic turbulent box (rho = 1, P = 1, k^-2
velocity at rms Mach 1 over k = 1..16, B = (0.5, 0, 0) + divergence-free
perturbation of rms 0.1), PPMC + HLLD, CFL 0.3, dt from the CFL reduction on
the device every step.  The headline line is the FP64 step; the FP32-bulk
and double-float steps on the same workload are reported under "variants",
each with its per-field relative L1 and max error against the FP64 state
after 10 steps on the FP64 run's dt sequence, and the adjoint steps where
their workspace fits beside the state (else at 256^3, said so).

Timing: W warm-up steps, then K steps bracketed by a barrier and a device
synchronisation, CUDA events on the library's stream, max over ranks.  The
state (8.6 GB) and workspace are far larger than L2, so no flush is needed.
Per-stage device times come from the library's event tracing over the same
timed region.  One process per GPU; ranks run independent replicas (weak
scaling, no data-path collective).

--impl reference times the CPU oracle (the plain FP64 reference) on the
host cores on a bounded sample of the same recipe (--ref-n, 96^3 per step by
default).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "cell-updates/s on 1 GB300 (FP64 vs FP32-bulk step, adjoint step); % HBM roofline"
UNIT = "cell-updates/s"

# Algorithmic HBM bytes per cell of one launch of each stage (reads + writes of
# the arrays the stage must touch once; T = compute type size).
def stage_bytes(T: int) -> dict:
    return {
        "prim": 64 + 8 * T,                  # U in, W out
        "flux_pcm": 14 * T + 8,              # 7 W fields, face B in; 7 fluxes out (one axis)
        "emf": (6 + 9) * T + 3 * T,          # v, B_cc, 2 EMF + mass flux per axis; 3 edges out
        "update_half": 64 + 18 * T + 11 * T,  # U, 15 hydro fluxes + 3 edges in; W + 3 faces out
        "recon": 8 * T + 14 * T,             # W in; W_L, W_R out (one axis)
        "flux_hlld": 15 * T + 7 * T,         # W_L, W_R, face B in; 7 fluxes out (one axis)
        "update_full": 64 + 18 * T + 64,     # U, fluxes, edges in; U out
        "dt": 0,
        "h2d": 0,                            # host copies of mhd_run_host (not step stages)
        "d2h": 0,
    }


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# FP64 pipe rate of this GPU, measured by a dependent-DFMA-chain probe with
# enough warps in flight: 601.3 G DFMA/s (1.91 per clock per SM at 2.07 GHz),
# i.e. 1202.6 GFLOP/s.  DADD and DMUL occupy the pipe like a DFMA.
FP64_PIPE_GINST = 601.3
FP64_PEAK_GFLOPS = 2 * FP64_PIPE_GINST
# Warp-instruction issue limit: 4 schedulers per SM, 152 SMs, 2.07 GHz.
ISSUE_PEAK_GWARPINST = 4 * 152 * 2.07

# Per-cell counters of one launch of each stage, from ncu captures at 192^3 of
# the turbulent box, PPMC (one kernel per capture; per-kernel SASS op counters
# and DRAM bytes; the x-axis launch of the per-axis stages, the mean of the x
# and z launches for the reconstruction), keyed by precision: (FP64 pipe ops
# DFMA + DADD + DMUL, FP64 flop 2 DFMA + DADD + DMUL, warp instructions, DRAM
# bytes read + written).  They hold for the kernels as profiled; a kernel
# changed since has no entry.  The PCM predictor, edge fields, updates and
# primitives do not depend on the reconstruction; PLMC has no reconstruction
# entry (its kernel changed after its capture).
_STAGES = {
    "fp64": {
        "prim": (45.7, 65.1, 1020.3 / 32, 145.0),
        "flux_pcm": (232.6, 350.8, 1416.9 / 32, 114.2),
        "emf": (48.0, 51.0, 698.0 / 32, 118.3),
        "update_half": (92.0, 133.0, 646.0 / 32, 315.6),
        "flux_hlld": (232.1, 349.9, 1422.6 / 32, 171.9),
        "update_full": (45.0, 66.0, 352.0 / 32, 268.3),
    },
    "fp32_bulk": {
        "prim": (18.0, 29.0, 719.0 / 32, 102.5),
        "flux_pcm": (0.0, 0.0, 493.3 / 32, 58.8),
        "emf": (0.0, 0.0, 224.0 / 32, 58.0),
        "update_half": (29.0, 46.0, 1103.0 / 32, 188.5),
        "flux_hlld": (0.0, 0.0, 524.2 / 32, 84.3),
        "update_full": (16.0, 19.0, 1040.8 / 32, 194.4),
    },
    "fp64_df": {
        "prim": (37.0, 53.0, 1517.3 / 32, 144.2),
        "flux_pcm": (0.0, 0.0, 2876.8 / 32, 114.2),
        "emf": (0.0, 0.0, 801.9 / 32, 118.2),
        "update_half": (45.0, 62.0, 2051.0 / 32, 315.5),
        "flux_hlld": (0.0, 0.0, 2816.5 / 32, 172.0),
        "update_full": (16.0, 19.0, 1145.0 / 32, 268.1),
    },
}
# FP64-pipe busy fraction of the FP64 kernels from the same captures
# (sm__pipe_fp64_cycles_active, % of peak sustained active): the pipe's
# occupancy by every FP64 instruction issued -- arithmetic, compares, and the
# lanes a divergent branch leaves idle -- beside the algorithmic count above
FP64_PIPE_BUSY = {"prim": 0.858, "flux_pcm": 0.892, "emf": 0.838, "update_half": 0.870, "recon": 0.852,
                  "flux_hlld": 0.892, "update_full": 0.879}
_RECON_PPMC = {
    "fp64": (420.2, 529.6, 3675.0 / 32, 169.6),
    "fp32_bulk": (0.0, 0.0, 1260.9 / 32, 80.9),
    "fp64_df": (0.0, 0.0, 7048.3 / 32, 169.4),
}
COUNTERS = {
    "plmc": {prec: dict(tab) for prec, tab in _STAGES.items()},
    "ppmc": {prec: dict(tab, recon=_RECON_PPMC[prec]) for prec, tab in _STAGES.items()},
}
class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[0]))
                mx.append(float(s[1]))
            except ValueError:
                continue
            for n, v in zip(names, s[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_state(n: int, recipe: str = "turbulent"):
    from paper_2402_05240_gb300 import inputs
    box = inputs.Box(n, n, n)
    if recipe == "turbulent":
        return inputs.turbulent_box(box, seed_v=1, seed_b=2)
    raise ValueError(recipe)


def time_gpu(mhd, torch, U0, n, steps, warmup, recon, precision, barrier):
    """Times `steps` device-dt VL+CT steps; returns (ms_per_step, stage profile, launches)."""
    stream = torch.cuda.current_stream()
    sim = mhd.Sim(n, n, n, cfl=0.3, recon=recon, precision=precision, stream=stream.cuda_stream)
    U = U0.clone()
    sim.run(U, warmup)
    torch.cuda.synchronize()
    sim.status()
    mhd.mhd_profile_enable(sim.ctx, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    sim.run(U, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    prof = mhd.mhd_profile_read(sim.ctx)
    mhd.mhd_profile_enable(sim.ctx, False)
    code, floors = mhd.mhd_status(sim.ctx)
    if code != mhd.MHD_OK:
        raise RuntimeError(f"device flags after the timed run: {code}")
    launches = sum(v[1] for v in prof.values())
    return ms / steps, prof, launches, sim, U


def time_adjoint(mhd, torch, U0, n, steps, warmup, recon, precision, barrier, fwd_ms):
    """Times `steps` adjoint steps (VJP of one step at fixed dt, forward
    recompute included) on the workload state; returns a variants entry."""
    stream = torch.cuda.current_stream()
    sim = mhd.Sim(n, n, n, cfl=0.3, recon=recon, precision=precision, stream=stream.cuda_stream)
    U = U0.clone()
    dt = sim.dt(U)
    g = torch.ones_like(U)
    gout = torch.empty_like(U)
    for _ in range(warmup):
        mhd.mhd_adjoint_step(sim.ctx, U, dt, g, gout)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for s in range(steps):
        src, dst = (g, gout) if s % 2 == 0 else (gout, g)
        mhd.mhd_adjoint_step(sim.ctx, U, dt, src, dst)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / steps
    ws = mhd.mhd_adjoint_workspace_bytes(sim.cfg)
    code, _ = mhd.mhd_status(sim.ctx)
    sim.close()
    del U, g, gout
    torch.cuda.empty_cache()
    return {"n": n, "value": n ** 3 / (ms * 1e-3), "ms_per_step": ms,
            "ratio_to_forward": ms / fwd_ms if fwd_ms else None,
            "dtype": DTYPES[precision], "adjoint_workspace_gb": ws / 1e9, "status": code}


DTYPES = {"fp64": "f64", "fp32_bulk": "f32 (FP64 state)", "fp64_df": "df64 (float pairs, FP64 state)"}
MODE_NAMES = {"fp64": "FP64", "fp32_bulk": "FP32-bulk", "fp64_df": "double-float"}


def adjoint_fits(mhd, torch, n, recon, precision):
    """Whether the forward and adjoint workspaces of an n^3 context plus the
    three states of time_adjoint (state, cotangent in and out) fit in the
    device memory that is free now (5 % kept back)."""
    cfg = mhd.mhd_config(n, n, n, 1.0 / n, 1.0 / n, 1.0 / n, 5.0 / 3.0, 0.3, mhd.RECON[recon],
                         mhd.PRECISION[precision], 1e-20, 1e-20)
    need = mhd.mhd_workspace_bytes(cfg) + mhd.mhd_adjoint_workspace_bytes(cfg) + 3 * 64 * n ** 3
    free, _ = torch.cuda.mem_get_info()
    return need <= 0.95 * free, need


def roofline_of(prof, precision, n3, hbm_peak, peak_kind, recon="plmc"):
    """Roofline of the dominant stage (largest share of the timed region).

    With per-cell counters of the stage (ncu capture at 192^3):
    the stage is bound by the FP64 pipe or by instruction issue, whichever
    runs closer to its peak -- achieved = counted FP64-pipe operations
    (DFMA + DADD + DMUL) per launch / live launch time against the measured
    FP64 pipe rate, or counted warp instructions per launch / launch time
    against the 4-per-clock-per-SM issue limit; both are reported, with the
    HBM view and the flop view.  Without counters: algorithmic bytes per
    launch / launch time against the measured HBM copy bandwidth.  `traffic`
    is the ncu DRAM bytes per cell of the profiled 192^3 launch scaled to
    this launch's cells (null without counters).
    """
    T = 4 if precision == "fp32_bulk" else 8
    sb = stage_bytes(T)
    total = sum(v[0] for v in prof.values())
    name, (ms, launches) = max(prof.items(), key=lambda kv: kv[1][0])
    per_launch_s = ms / max(launches, 1) * 1e-3
    shares = {k: round(v[0] / total, 4) for k, v in prof.items() if v[1]}
    gbs = sb[name] * n3 / per_launch_s / 1e9
    steps = max(1, prof["update_full"][1])
    step_s = total * 1e-3 / steps
    counted = sum(sb[k] * v[1] for k, v in prof.items()) / steps
    out = {"kernel": name, "per_launch_ms": round(per_launch_s * 1e3, 4), "stage_share": shares,
           "bytes_per_cell_counted": counted,
           "hbm": {"achieved": round(gbs, 1), "peak": hbm_peak, "frac": round(gbs / hbm_peak, 4),
                   "peak_source": peak_kind}}
    # the whole step against HBM: counted bytes, the 128 B/cell minimum (read
    # and write the state), and the ncu DRAM bytes of the profiled kernels
    cells_per_s = n3 / step_s
    step_hbm = {"cells_per_s": round(cells_per_s), "frac_counted": round(cells_per_s * counted / 1e9 / hbm_peak, 4),
                "frac_min_128B": round(cells_per_s * 128 / 1e9 / hbm_peak, 4)}
    table = COUNTERS.get(recon, {}).get(precision, {})
    if table and all(k in table for k in prof if k != "dt" and prof[k][1]):
        ncu_b = sum(table[k][3] * v[1] for k, v in prof.items() if k != "dt" and v[1]) / steps
        step_hbm.update({"ncu_dram_bytes_per_cell": round(ncu_b, 1),
                         "frac_ncu": round(cells_per_s * ncu_b / 1e9 / hbm_peak, 4)})
    out["step_hbm"] = step_hbm
    cnt = COUNTERS.get(recon, {}).get(precision, {}).get(name)
    if cnt:
        gi = cnt[0] * n3 / per_launch_s / 1e9
        gw = cnt[2] * n3 / per_launch_s / 1e9
        fp64 = {"achieved": round(gi, 1), "peak": FP64_PIPE_GINST, "unit": "G FP64-pipe op/s (DFMA+DADD+DMUL)",
                "frac": round(gi / FP64_PIPE_GINST, 4), "peak_source": "measured (FP64 FMA-chain probe)"}
        issue = {"achieved": round(gw, 1), "peak": round(ISSUE_PEAK_GWARPINST, 1), "unit": "G warp-inst/s issued",
                 "frac": round(gw / ISSUE_PEAK_GWARPINST, 4),
                 "peak_source": "nominal (4 issue slots per clock per SM, 152 SMs, 2.07 GHz)"}
        main = fp64 if fp64["frac"] >= issue["frac"] else issue
        if precision == "fp64" and name in FP64_PIPE_BUSY:
            fp64["busy_ncu"] = FP64_PIPE_BUSY[name]
        out.update({"bound": "alu", **main, "fp64_pipe": fp64, "issue": issue,
                    "traffic": round(cnt[3] * n3),
                    "traffic_note": "ncu DRAM bytes per cell at 192^3 scaled to this launch's cells"})
        if cnt[1]:
            gf = cnt[1] * n3 / per_launch_s / 1e9
            out["flop"] = {"achieved_gflops": round(gf, 1), "peak_gflops": FP64_PEAK_GFLOPS,
                           "frac": round(gf / FP64_PEAK_GFLOPS, 4), "flop_per_cell": cnt[1]}
    else:
        out.update({"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(gbs / hbm_peak, 4), "peak_source": peak_kind, "traffic": None})
    return out


def cpu_baseline_sample(recon, n_sample=128, steps=1):
    """The oracle as it stands on the host cores: one step of the same recipe
    at n_sample^3 (a bounded sample of the workload)."""
    import oracle
    U = make_state(n_sample)
    orc = oracle.Oracle(n_sample, n_sample, n_sample, recon=recon)
    dt = orc.dt(U, 0.3)
    t0 = time.perf_counter()
    for _ in range(steps):
        U = orc.step(U, dt)
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": n_sample ** 3 * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} FP64 {recon.upper()} step(s) of the turbulent-box recipe at {n_sample}^3 "
                      f"({el:.1f} s wall)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    n = args.ref_n
    import oracle
    U = make_state(n)
    orc = oracle.Oracle(n, n, n, recon=args.recon)
    dt = orc.dt(U, 0.3)
    for _ in range(args.warmup):
        orc.step(U, dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U = orc.step(U, dt)
    el = time.perf_counter() - t0
    value = n ** 3 * args.steps / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": f"turbulent box {args.n or 512}^3, {args.recon.upper()} + HLLD, "
                                                   f"FP64 step, CFL 0.3: CPU oracle on a {n}^3 sample of the "
                                                   "recipe per step",
                                        "parallelism": "host cores (OpenMP)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n}^3 per step, {args.steps} steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    if args.ref_sweep:
        line["cpu_baseline"]["sweep"] = oracle_sweep(args.recon)
    print(json.dumps(line), flush=True)
    return 0


def oracle_sweep(recon, sizes=((32, 10), (128, 1), (256, 1)), single=((32, 2), (128, 1))):
    """Per-step time and cell-updates/s of the oracle on this host: all cores
    (OpenMP over cells) at 32^3, 128^3 and 256^3, and one thread at 32^3 and
    128^3 (the turbulent recipe, the CFL dt of the initial state)."""
    import oracle
    out = []
    allc = oracle.set_threads(0)
    for threads, cases in ((allc, sizes), (1, single)):
        oracle.set_threads(threads)
        for n, steps in cases:
            U = make_state(n)
            orc = oracle.Oracle(n, n, n, recon=recon)
            dt = orc.dt(U, 0.3)
            t0 = time.perf_counter()
            for _ in range(steps):
                U = orc.step(U, dt)
            el = (time.perf_counter() - t0) / steps
            out.append({"n": n, "threads": threads, "s_per_step": round(el, 4),
                        "cell_updates_per_s": n ** 3 / el})
    oracle.set_threads(allc)
    return out


def run_workload(args, mhd, torch, rank):
    """One of the extra measurements; prints one JSON line on rank 0."""
    from paper_2402_05240_gb300 import workloads as Wk
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if args.workload == "precision512":
        r = Wk.precision_compare(mhd, torch, n=args.n or 512, steps=args.steps,
                                 warmup=args.warmup, recon="ppmc")
        value, ms, dtype = r["fp64"]["value"], r["fp64"]["ms_per_step"], "f64"
        wl = f"turbulent box {r['n']}^3, PPMC + HLLD, FP64 vs FP32-bulk vs double-float, {r['steps']} steps"
    elif args.workload == "adjoint_rollout":
        r = Wk.adjoint_rollout(mhd, torch, n=args.n or 256, steps=100, every=10)
        value, ms, dtype = r["backward_cell_updates_per_s"], r["backward_s"] / r["steps"] * 1e3, "f32 (FP64 state)"
        wl = f"blast beta=0.1 {r['n']}^3, PPMC + HLLD, FP32-bulk, 100-step adjoint rollout, checkpoints every 10"
    elif args.workload == "adjoint":
        # the adjoint step alone (and the forward step it is compared with)
        # on the turbulent box, in the precision and reconstruction given
        n = args.n or 512
        U0 = torch.from_numpy(make_state(n)).cuda()
        fwd_ms, _, _, sim, U = time_gpu(mhd, torch, U0, n, args.steps, args.warmup, args.recon, args.precision,
                                        lambda: None)
        sim.close()
        del sim, U
        torch.cuda.empty_cache()
        r = time_adjoint(mhd, torch, U0, n, args.steps, args.warmup, args.recon, args.precision, lambda: None, fwd_ms)
        r["forward_ms_per_step"] = fwd_ms
        value, ms, dtype = r["value"], r["ms_per_step"], DTYPES[args.precision]
        wl = f"turbulent box {n}^3, {args.recon.upper()} + HLLD, {MODE_NAMES[args.precision]} adjoint step"
    else:
        n = args.n or 459
        r = Wk.slow_wave(mhd, torch, n=n, steps=args.steps, warmup=args.warmup, precision=args.precision)
        value, ms = r["value"], r["ms_per_step"]
        dtype = {"fp64": "f64", "fp32_bulk": "f32 (FP64 state)", "fp64_df": "df64 (float pairs, FP64 state)"}[
            args.precision]
        wl = f"slow magnetosonic wave {n}^3 (B = (1, 1.5, 0)), PLMC + HLLD, {args.precision}"
    clk = clocks.stop()
    if rank == 0:
        print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
                          "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": dtype, "data": "synthetic",
                          "config": {"workload": wl}, "clocks": clk, "result": r}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=None,
                    help="cells per axis (default 512; 256 for adjoint_rollout, 459 for slow_wave)")
    ap.add_argument("--recon", default="ppmc", choices=["plmc", "ppmc"])
    ap.add_argument("--compare-steps", type=int, default=10,
                    help="steps after which each variant's state is compared with the headline mode's")
    ap.add_argument("--ref-n", type=int, default=96)
    ap.add_argument("--ref-sweep", action="store_true",
                    help="with --impl reference: also time the oracle at 32^3-256^3, all cores and one thread")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_bulk", "fp64_df"],
                    help="precision of the headline timed run (default: the FP64 step)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--workload", default="turbulent",
                    choices=["turbulent", "precision512", "adjoint_rollout", "slow_wave", "adjoint"],
                    help="turbulent: the default step timing; adjoint: the adjoint step alone (--precision, "
                         "--recon, --n); the others are the extra measurements of "
                         "paper_2402_05240_gb300.workloads (one JSON line each)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

        def barrier():
            dist.barrier()
    else:
        dist = None

        def barrier():
            pass

    from paper_2402_05240_gb300 import build
    build.build()
    from paper_2402_05240_gb300 import mhd

    if args.workload != "turbulent":
        return run_workload(args, mhd, torch, rank)

    n = args.n or 512
    n3 = n ** 3
    t0 = time.perf_counter()
    U0 = torch.from_numpy(make_state(n)).cuda()
    gen_s = time.perf_counter() - t0
    hbm_peak, peak_kind = load_peaks()

    clocks = ClockSampler(local)
    clocks.start()
    ms64, prof64, launches64, sim, U = time_gpu(mhd, torch, U0, n, args.steps, args.warmup, args.recon,
                                                  args.precision, barrier)
    clk = clocks.stop()
    if dist is not None:
        t = torch.tensor([ms64], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms64 = float(t.item())
    value = world * n3 / (ms64 * 1e-3)
    roof = roofline_of(prof64, args.precision, n3, hbm_peak, peak_kind, args.recon)
    del U

    # end to end through the public host-buffer entry point (copies inside)
    e2e_s, e2e_parts = None, None
    if args.e2e_steps > 0:
        # page-locked, huge-page backed host memory from the library
        # (mhd_host_alloc): the copies stay at the link rate between steps
        host = mhd.host_buffer(8, n, n, n)
        host.copy_(U0)  # device -> host, no pageable temporary
        mhd.mhd_run_host(sim.ctx, host, 1)  # warm the host-state buffer
        mhd.mhd_profile_enable(sim.ctx, True)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            mhd.mhd_run_host(sim.ctx, host, 1)
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        # device time of each part of a call (CUDA events on the library's stream)
        p = mhd.mhd_profile_read(sim.ctx)
        mhd.mhd_profile_enable(sim.ctx, False)
        e2e_parts = {"h2d_ms": p["h2d"][0] / args.e2e_steps, "d2h_ms": p["d2h"][0] / args.e2e_steps,
                     "step_ms": sum(v[0] for k, v in p.items() if k not in ("h2d", "d2h")) / args.e2e_steps,
                     "wall_ms": e2e_s * 1e3}
        del host
    sim.close()
    del sim
    torch.cuda.empty_cache()

    variants = {}
    if not args.no_variants:
        from paper_2402_05240_gb300 import workloads as Wk
        modes = [m for m in ("fp64", "fp32_bulk", "fp64_df") if m != args.precision]
        # the headline mode's state after --compare-steps steps and its dts,
        # against which each variant's state is compared on the same dts
        ref = U0.clone()
        dts = torch.zeros(args.compare_steps, dtype=torch.float64, device="cuda")
        sim = mhd.Sim(n, n, n, cfl=0.3, recon=args.recon, precision=args.precision,
                      stream=torch.cuda.current_stream().cuda_stream)
        sim.run(ref, args.compare_steps, dts)
        sim.status()
        sim.close()
        del sim
        dts_host = dts.cpu().numpy().tolist()
        for m in modes:
            msm, profm, launchesm, simm, Um = time_gpu(mhd, torch, U0, n, args.steps, args.warmup, args.recon, m,
                                                       barrier)
            Um.copy_(U0)
            for dt in dts_host:
                simm.step(Um, dt)
            torch.cuda.synchronize()
            simm.status()
            simm.close()
            variants[m] = {
                "value": world * n3 / (msm * 1e-3), "ms_per_step": msm, "dtype": DTYPES[m],
                "speedup_over_headline": ms64 / msm,
                "roofline": roofline_of(profm, m, n3, hbm_peak, peak_kind, args.recon), "gpu_launches": launchesm,
                "stage_ms": {k: round(v[0] / args.steps, 4) for k, v in profm.items()},
                f"vs_{args.precision}_after_{args.compare_steps}_steps": Wk.field_errors(torch, Um, ref)}
            del Um, simm
            torch.cuda.empty_cache()
        del ref
        torch.cuda.empty_cache()
        fwd = {args.precision: ms64, **{m: variants[m]["ms_per_step"] for m in modes}}
        U_small = None
        for m in ("fp32_bulk", "fp64", "fp64_df"):
            adj_steps = max(2, args.steps // 2)
            fits, need = adjoint_fits(mhd, torch, n, args.recon, m)
            if fits:
                variants["adjoint_" + m] = time_adjoint(mhd, torch, U0, n, adj_steps, 1, args.recon, m, barrier,
                                                        fwd[m])
                continue
            # does not fit beside the state at this size: time it at n/2 (and its forward step there)
            nh = n // 2
            if U_small is None:
                U_small = torch.from_numpy(make_state(nh)).cuda()
            msf, _, _, simf, Uf = time_gpu(mhd, torch, U_small, nh, adj_steps, 1, args.recon, m, barrier)
            simf.close()
            del Uf, simf
            entry = time_adjoint(mhd, torch, U_small, nh, adj_steps, 1, args.recon, m, barrier, msf)
            entry["note"] = (f"at {n}^3 the forward and adjoint workspaces and three states need "
                             f"{need / 1e9:.0f} GB, more than the free device memory; timed at {nh}^3")
            variants["adjoint_" + m] = entry
        del U_small
        torch.cuda.empty_cache()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms64, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[args.precision],
        "data": "synthetic",
        "config": {"workload": f"turbulent box {n}^3, {args.recon.upper()} + HLLD, "
                               f"{MODE_NAMES[args.precision]} step, CFL 0.3, device dt",
                   "parallelism": f"replicas x{world}",
                   "l2": f"inputs larger than L2 (state {64 * n3 / 1e9:.2f} GB)",
                   "input_generation_s": round(gen_s, 1)},
        "roofline": roof,
        "e2e": ({"value": world * n3 / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 64 * n3,
                 "d2h_bytes_per_step": 64 * n3, "parts": e2e_parts} if e2e_s else None),
        "gpu_launches": launches64,
        "clocks": clk,
        "stage_ms": {k: round(v[0] / args.steps, 4) for k, v in prof64.items()},
        "variants": variants,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(args.recon)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

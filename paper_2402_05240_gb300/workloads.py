"""Benchmark workloads beyond the default step timing (used by bench.py).

* precision_compare: the 512^3 PPMC turbulent box, FP64, FP32-bulk and
  double-float steps timed on the same state, and the FP32-bulk and
  double-float states after n steps compared with the FP64 state per field
  (relative L1 and max error), all runs on the FP64 run's dt sequence.
* adjoint_rollout: the strongly magnetised blast at 256^3, FP32-bulk PPMC,
  a 100-step rollout differentiated through torch.autograd with checkpoints
  every 10 steps; reports forward and backward time, their ratio, the peak
  device memory and the floor triggers.
* slow_wave: the paper's single-GPU throughput problem (slow magnetosonic
  wave, B = (1, 1.5, 0), PLMC) at a given size and precision.

Everything runs through the library's C ABI; torch supplies device memory.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs


def field_errors(torch, got, ref):
    """Per-field relative L1 (sum |a-b| / max(sum |b|, N s_f), s_f the field's
    physical scale) and max |a-b| of two float64 CUDA states."""
    N = ref[0].numel()
    rho = float(ref[0].abs().mean())
    e = float(ref[4].abs().mean())
    m = (rho * e) ** 0.5
    b = float(torch.sqrt((ref[5] ** 2 + ref[6] ** 2 + ref[7] ** 2).mean()))
    scales = [rho, m, m, m, e, b, b, b]
    names = ["rho", "mx", "my", "mz", "E", "Bx", "By", "Bz"]
    out = {}
    for f in range(8):
        d = (got[f] - ref[f]).abs()
        denom = max(float(ref[f].abs().sum()), N * scales[f])
        out[names[f]] = {"rel_l1": float(d.sum()) / denom, "max_abs": float(d.max())}
    return out


def _timed_run(mhd, torch, sim, U, steps, dt_log=None):
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.run(U, steps, dt_log)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def precision_compare(mhd, torch, n=512, steps=10, warmup=2, recon="ppmc"):
    box = inputs.Box(n, n, n)
    t0 = time.perf_counter()
    U0 = torch.from_numpy(inputs.turbulent_box(box, seed_v=1, seed_b=2)).cuda()
    gen_s = time.perf_counter() - t0
    res = {"n": n, "steps": steps, "recon": recon, "input_generation_s": round(gen_s, 1)}
    stream = torch.cuda.current_stream().cuda_stream
    # FP64 reference run (records dt)
    sim = mhd.Sim(n, n, n, cfl=0.3, recon=recon, precision="fp64", stream=stream)
    W = U0.clone()
    sim.run(W, warmup)
    del W
    U64 = U0.clone()
    dts = torch.zeros(steps, dtype=torch.float64, device="cuda")
    ms64 = _timed_run(mhd, torch, sim, U64, steps, dts)
    sim.status()
    sim.close()
    torch.cuda.empty_cache()
    n3 = n ** 3
    res["fp64"] = {"value": n3 / (ms64 * 1e-3), "ms_per_step": ms64}
    # the other modes: a timing run (device dt), then the comparison run on the FP64 dts
    for prec in ("fp32_bulk", "fp64_df"):
        sim = mhd.Sim(n, n, n, cfl=0.3, recon=recon, precision=prec, stream=stream)
        W = U0.clone()
        sim.run(W, warmup)
        ms = _timed_run(mhd, torch, sim, W, steps)
        W.copy_(U0)
        for dt in dts.cpu().numpy().tolist():
            sim.step(W, dt)
        torch.cuda.synchronize()
        sim.status()
        sim.close()
        res[prec] = {"value": n3 / (ms * 1e-3), "ms_per_step": ms, "speedup_over_fp64": ms64 / ms,
                     "vs_fp64_after_steps": field_errors(torch, W, U64)}
        del W
        torch.cuda.empty_cache()
    del U64, U0
    torch.cuda.empty_cache()
    return res


def adjoint_rollout(mhd, torch, n=256, steps=100, every=10, recon="ppmc", precision="fp32_bulk"):
    from . import autograd as A

    box = inputs.Box(n, n, n)
    U0 = torch.from_numpy(inputs.blast(box, seed=4)).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    sim = mhd.Sim(n, n, n, cfl=0.3, recon=recon, precision=precision, rho_floor=1e-4, p_floor=1e-6, stream=stream)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    free0, total = torch.cuda.mem_get_info()
    x = U0.clone().requires_grad_(True)
    t0 = time.perf_counter()
    Un = A.rollout(sim, x, steps, checkpoint_every=every)
    L = A.magnetic_energy(Un, 1.0 / n ** 3)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    free1, _ = torch.cuda.mem_get_info()
    t0 = time.perf_counter()
    L.backward()
    torch.cuda.synchronize()
    t_bwd = time.perf_counter() - t0
    free2, _ = torch.cuda.mem_get_info()
    g = x.grad
    code, floors = mhd.mhd_status(sim.ctx)
    peak_torch = torch.cuda.max_memory_allocated()
    res = {
        "n": n, "steps": steps, "checkpoint_every": every, "recon": recon, "precision": precision,
        "forward_s": t_fwd, "backward_s": t_bwd, "backward_over_forward": t_bwd / t_fwd,
        "forward_cell_updates_per_s": n ** 3 * steps / t_fwd,
        "backward_cell_updates_per_s": n ** 3 * steps / t_bwd,
        "peak_torch_bytes": peak_torch,
        "library_workspace_bytes": mhd.mhd_workspace_bytes(sim.cfg) + mhd.mhd_adjoint_workspace_bytes(sim.cfg),
        "device_used_bytes_after_backward": total - free2,
        "loss": float(L.detach()), "grad_norm": float(g.norm()), "grad_finite": bool(torch.isfinite(g).all()),
        "floor_triggers_rho_p": list(floors), "status": code,
    }
    res["peak_hbm_bytes"] = res["peak_torch_bytes"] + res["library_workspace_bytes"]
    sim.close()
    del g, x, Un, L, U0
    torch.cuda.empty_cache()
    return res


def slow_wave(mhd, torch, n=459, steps=20, warmup=2, precision="fp64"):
    box = inputs.Box(n, n, n)
    U0, _ = inputs.linear_wave(box, amp=1e-6, b=(1.0, 1.5, 0.0), wave="slow+")
    U = torch.from_numpy(U0).cuda()
    del U0
    sim = mhd.Sim(n, n, n, cfl=0.3, recon="plmc", precision=precision,
                  stream=torch.cuda.current_stream().cuda_stream)
    sim.run(U, warmup)
    ms = _timed_run(mhd, torch, sim, U, steps)
    sim.status()
    sim.close()
    return {"n": n, "steps": steps, "precision": precision, "value": n ** 3 / (ms * 1e-3), "ms_per_step": ms}

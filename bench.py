#!/usr/bin/env python
"""Benchmark of the multilevel D3Q19 lattice Boltzmann hot path on GB300.

Default workload: the sphere flow at Re = 100 (box 32D x 16D x 16D, sphere
D = 64 finest elements, five levels D/4 .. D/64, about 8.6e7 fluid elements,
velocity inlet / pressure outlet), FP32-deviation storage.  A "step" is one
coarse time step of the whole hierarchy (31 stream-collide launches plus the
ghost fills).  The metric is fine-substep weighted MLUPS,
U = sum_L N_L 2^{L - Lmin} element updates per coarse step.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

N > 1 (launched by torch.distributed.run): independent replicas, one per GPU
(the method is not sharded here), value = total updates / max time.
"""
from __future__ import annotations

import argparse
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

METRIC = "multilevel D3Q19 MLUPS & % HBM peak, FP32-dev vs FP64 at stated error"
SMI_FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sphere", choices=["sphere", "sphere_half", "tgv3d"],
                    help="sphere_half: every length halved (about 1.1e7 elements), for profiling captures")
    ap.add_argument("--no-variants", action="store_true", help="skip the FP64/BF16 and TGV side measurements")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the oracle CPU baseline")
    return ap.parse_args()


# ---------------------------------------------------------------- workloads
def make_workload(name):
    from paper_1601_06984_gb300 import workloads as W
    if name in ("sphere", "sphere_half"):
        scale = 1 if name == "sphere" else 2
        mesh = W.config_sphere(scale)
        U = 0.04
        om_f = W.omega_for_re(U, 64, 100.0)
        om_c = W.omega_coarse_from_finest(om_f, 5)
        desc = {"workload": "sphere_re100_d3q19_5level" + ("" if scale == 1 else "_half"),
                "box": "32D x 16D x 16D", "D_finest": 64 // scale,
                "levels": 5, "u_in": U, "omega_finest": round(om_f, 6), "omega_coarsest": round(om_c, 6),
                "boundaries": "velocity inlet x-, pressure outlet x+, periodic y/z, half-way bounce-back sphere",
                "outlet": "zero-gradient"}
        fields = lambda m: W.uniform_fields(m, 1.0, (U, 0.0, 0.0))
        return mesh, 19, om_c, (U, 0.0, 0.0), fields, desc
    mesh = W.config_tgv3d(64)
    desc = {"workload": "tgv3d_two_level_64", "box": "64^3 periodic, 32^3 block refined", "levels": 2,
            "u0": 0.01, "omega_coarse": 1.6}
    fields = lambda m: W.tgv_fields(m, 0.01)
    return mesh, 19, 1.6, (0.0, 0.0, 0.0), fields, desc


def small_sample():
    """Bounded sample of the sphere workload for the CPU oracle: the reduced
    three-level sphere case (about 1.75e4 elements)."""
    from paper_1601_06984_gb300 import workloads as W
    m = W.config_sphere_small()
    om = W.omega_coarse_from_finest(W.omega_for_re(0.04, 64, 100.0), 3)
    return m, om, (0.04, 0.0, 0.0)


def bytes_per_update(Q, prec, brick=False):
    """Algorithmic HBM bytes of one element update: Q pdf reads and Q writes,
    plus the 32-bit neighbour list (Q-1 entries) for the neighbour-list kernel
    or one 27-entry row of neighbour-brick indices per 64 elements for the
    interior-brick kernel."""
    s = {0: 8, 1: 4, 2: 2}[prec]
    return 2 * Q * s + (27 * 4 / 64 if brick else 4 * (Q - 1))


# ---------------------------------------------------------------- clocks
class Clocks:
    def __init__(self, uuid=None, index=0):
        self.uuid, self.index = uuid, index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={SMI_FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                r = [x.strip() for x in line.split(",")]
                if len(r) < 10:
                    continue
                if self.uuid and self.uuid not in r[1]:
                    continue
                if not self.uuid and r[0] != str(self.index):
                    continue
                rows.append(r)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower().startswith("active")})
        pw = [float(r[4]) for r in rows if r[4].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


def gpu_uuid(dev):
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


def stream_collide_traffic():
    """DRAM bytes per element update of the finest-level interior-brick
    stream-collide from the committed ncu capture, if the kernel source is
    unchanged since."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "stream_collide_brick_fp32_sphere.json")) as fh:
            rec = json.load(fh)
        with open(os.path.join(ROOT, "paper_1601_06984_gb300", "csrc", "kernels.cuh")) as fh:
            src = fh.read()
        a = src.index("// ----------------------------------------------------------------- physics")
        b = src.index("// ----------------------------------------------------------------- outlet values")
        if hashlib.sha256(src[a:b].encode()).hexdigest()[:16] != rec["kernel_source_sha256_16"]:
            return None
        return float(rec["dram_bytes_per_unit"])
    except Exception:
        return None


def fp64_instruction_record():
    """FP64 instructions per element update of the interior-brick kernel and
    the FP64 issue peak, from the committed ncu count, if the kernel source is
    unchanged since."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "stream_collide_brick_fp64_tgv3d.json")) as fh:
            rec = json.load(fh)
        with open(os.path.join(ROOT, "paper_1601_06984_gb300", "csrc", "kernels.cuh")) as fh:
            src = fh.read()
        a = src.index("// ----------------------------------------------------------------- physics")
        b = src.index("// ----------------------------------------------------------------- outlet values")
        if hashlib.sha256(src[a:b].encode()).hexdigest()[:16] != rec["kernel_source_sha256_16"]:
            return None
        return rec
    except Exception:
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


# ---------------------------------------------------------------- replicas
def max_over_ranks(value, dist=None, device="cpu"):
    """Largest value over all ranks (the slowest replica sets the job time)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(updates_per_rank, seconds_per_rank, world, dist=None, device="cpu"):
    """Whole-job MLUPS of independent replicas: all ranks' updates over the
    slowest rank's time."""
    return world * updates_per_rank / max_over_ranks(seconds_per_rank, dist, device) / 1e6


# ---------------------------------------------------------------- CPU oracle
def cpu_oracle(seconds, min_steps=2):
    """Time the CPU oracle (single thread) on the bounded sample."""
    from oracle.oracle import Oracle
    from paper_1601_06984_gb300 import workloads as W
    m, om, uin = small_sample()
    o = Oracle(m, 19, om, u_in=uin, outlet=1)
    o.init(*W.uniform_fields(m, 1.0, uin))
    o.step(1)
    steps, t0 = 0, time.perf_counter()
    while steps < min_steps or time.perf_counter() - t0 < seconds:
        o.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    U = m.updates_per_coarse_step()
    return {"value": steps * U / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"reduced 3-level D3Q19 sphere ({m.n} elements, {U} updates/coarse step), "
                      f"{steps} coarse steps, single-threaded FP64 oracle",
            "seconds": round(dt, 2), "ms_per_step": 1e3 * dt / steps}


# ---------------------------------------------------------------- GPU runs
OUTLETS = {"linear": 0, "zero-gradient": 1}


def run_gpu(mesh, Q, om, uin, fields, prec, K, W_, device, dist=None, want_moments=False, outlet=0,
            kernel_timing=True):
    """Time K coarse steps after W_ warm-up steps.  With kernel_timing the
    library brackets every stream-collide launch with CUDA events (steps are
    then launched kernel by kernel); without it the steps replay the library's
    captured CUDA graphs, as a caller's lbm_step(K) does."""
    import torch

    from paper_1601_06984_gb300 import lbm
    U = mesh.updates_per_coarse_step()
    t_build = time.perf_counter()
    sim = lbm.Sim(mesh, Q, om, precision=prec, u_in=uin, device=device, outlet=outlet)
    t_build = time.perf_counter() - t_build
    rho, u, S = fields(mesh)
    sim.init(rho, u, S)
    sim.step(W_)
    info = sim.mesh_info()
    stream = sim.stream
    torch.cuda.synchronize(device)
    sim.timing_enable(kernel_timing)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(device)
    n0 = sim.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sim.step(K)
    ev1.record(stream)
    torch.cuda.synchronize(device)
    ms = ev0.elapsed_time(ev1)
    launches = sim.kernel_launches() - n0
    nl, kms = sim.timing_read()
    ms = max_over_ranks(ms, dist, device)
    finest = len(info) - 1
    # dominant kernel: the interior-brick stream-collide of the finest level
    # (the neighbour-list kernel when the level has no interior bricks)
    kb = 0 if info[finest, 8] > 0 else 1
    units = int(64 * info[finest, 8]) if kb == 0 else int(info[finest, 1])
    avg_ms = kms[finest, kb] / max(nl[finest, kb], 1) if kernel_timing else float("nan")
    bpu = bytes_per_update(Q, prec, brick=kb == 0)
    list_units = int(info[finest, 1] - 64 * (info[finest, 8] + info[finest, 9]))
    list_ms = kms[finest, 1] / max(nl[finest, 1], 1)
    bnd_units = int(64 * info[finest, 9])
    bnd_ms = kms[finest, 2] / max(nl[finest, 2], 1)
    res = {"ms_total": ms, "ms_per_step": ms / K, "mlups": K * U / (ms * 1e-3) / 1e6, "launches": launches,
           "finest_kernel": "k_stream_collide_brick" if kb == 0 else "k_stream_collide",
           "finest_launch_ms": avg_ms, "finest_launches": int(nl[finest, kb]), "finest_units": units,
           "finest_bytes": units * bpu, "finest_gbs": units * bpu / (avg_ms * 1e-3) / 1e9 if kernel_timing else None,
           "finest_list_units": list_units, "finest_list_launch_ms": list_ms,
           "finest_boundary_units": bnd_units, "finest_boundary_launch_ms": bnd_ms,
           "finest_boundary_gbs": (bnd_units * bytes_per_update(Q, prec, brick=True) / (bnd_ms * 1e-3) / 1e9
                                   if nl[finest, 2] > 0 and bnd_ms > 0 else None),
           "finest_list_gbs": (list_units * bytes_per_update(Q, prec) / (list_ms * 1e-3) / 1e9
                               if nl[finest, 1] > 0 and list_ms > 0 else None),
           "level_ms": kms.sum(axis=1).tolist(), "level_launches": nl.sum(axis=1).tolist(),
           "interior_fraction": float(64 * info[:, 8].sum() / info[:, 1].sum()),
           "brick_fraction": float(64 * (info[:, 8] + info[:, 9]).sum() / info[:, 1].sum()),
           "step_bytes": float(sum((1 << li) * (64 * (info[li, 8] + info[li, 9]) * bytes_per_update(Q, prec, brick=True)
                                                + (info[li, 1] - 64 * (info[li, 8] + info[li, 9]))
                                                * bytes_per_update(Q, prec))
                                   for li in range(len(info)))),
           "bytes_per_update": bpu, "build_s": t_build, "device_gb": sim.device_bytes() / 1e9,
           "reduce": sim.reduce().tolist()}
    if want_moments:
        res["moments"] = sim.moments()
    return sim, res


def adjoint_run(device):
    """Adjoint configuration: periodic 64^3 coarse with the central 32^3 block
    refined, Gaussian body force N(0, 1e-6) per component, 400 coarse steps,
    final kinetic energy, checkpoints every 20 steps.  FP32 deviation: time of
    the adjoint (forward with checkpoints + reverse sweep) over the forward
    alone.  FP64: gradient along a random force direction and along omega
    against central differences."""
    import torch
    from paper_1601_06984_gb300 import lbm, workloads as W
    m = W.config_tgv3d(64)
    rho, u, S = W.uniform_fields(m)
    F = W.gaussian_force(m, 1e-6)
    n, K = 400, 20
    out = {"config": "tgv3d 64^3/32^3 two-level, force N(0,1e-6), 400 coarse steps, K=20, objective KE"}
    for name, prec in (("fp32dev", lbm.FP32DEV), ("fp64", lbm.FP64)):
        g = lbm.Sim(m, 19, 1.6, precision=prec, use_force=True, device=device)
        g.init(rho, u, S)
        g.set_force(F)
        g.step(3)
        g.init(rho, u, S)
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        g.step(n)
        g.reduce()
        tf = time.perf_counter() - t0
        g.init(rho, u, S)
        t0 = time.perf_counter()
        J, dF, dw, _ = g.adjoint(n, K, 0)
        ta = time.perf_counter() - t0
        rec = {"forward_s": tf, "adjoint_s": ta, "adjoint_to_forward": ta / tf, "J": J,
               "adjoint_workspace_gb": g.adjoint_bytes(n, K) / 1e9}
        if prec == lbm.FP64:
            vF = W.random_direction((m.n, 3), W.SEED, 51) * 1e-6
            vw = 0.1

            def run(h):
                gg = lbm.Sim(m, 19, 1.6, precision=prec, use_force=True, device=device)
                gg.init(rho, u, S)
                gg.set_params(1.6 + h * vw)
                gg.set_force(F + h * vF)
                gg.step(n)
                return gg.reduce()[7]

            h = 1e-3
            fd = (run(h) - run(-h)) / (2 * h)
            adj = float((dF * vF).sum() + dw * vw)
            rec["directional_derivative_adjoint"] = adj
            rec["directional_derivative_central_fd"] = fd
            rec["rel_error_vs_fd"] = abs(adj - fd) / abs(fd)
        out[name] = rec
        g.close()
        del g
        torch.cuda.empty_cache()
    return out


def e2e_run(sim, mesh, fields, K):
    """End to end through the C ABI: initial fields from pinned host memory,
    then K coarse steps each followed by the FP64 reduction (mass, momentum,
    drag, kinetic energy) read back to the host."""
    import torch
    rho, u, _ = fields(mesh)
    rho_p = torch.from_numpy(rho).pin_memory()
    u_p = torch.from_numpy(u).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.init(rho_p.numpy(), u_p.numpy())
    n0 = sim.kernel_launches()
    for _ in range(K):
        sim.step(1)
        sim.reduce()
    dt = time.perf_counter() - t0
    U = mesh.updates_per_coarse_step()
    return {"value": K * U / dt / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": int((rho_p.numel() + u_p.numel()) * 8 / K), "d2h_bytes_per_step": 64,
            "seconds": round(dt, 3), "launches": sim.kernel_launches() - n0}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    K, W_ = args.steps, args.warmup
    assert W_ >= 3, "at least 3 warm-up steps"

    if args.impl == "reference":
        if rank != 0:
            return
        cb = cpu_oracle(max(5.0, min(args.cpu_seconds, 20.0)), min_steps=K)
        desc = {"workload": "sphere_re100_d3q19_5level" if args.workload == "sphere" else "tgv3d_two_level_64"}
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "MLUPS", "n_gpus": args.gpus,
                "steps": K, "warmup": W_, "ms_per_step": cb["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": dict(desc, sample="bounded: reduced 3-level D3Q19 sphere run by the CPU oracle"),
                "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
                "e2e": {"value": cb["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import numpy as np
    import torch
    dist = None
    if world > 1:
        import torch.distributed as td
        td.init_process_group("nccl")
        dist = td
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
    from paper_1601_06984_gb300 import lbm

    mesh, Q, om, uin, fields, desc = make_workload(args.workload)
    U = mesh.updates_per_coarse_step()
    peak, peak_src = measured_peaks()
    traffic_per_unit = stream_collide_traffic()

    clk = Clocks(uuid=gpu_uuid(device), index=local)
    outlet = OUTLETS.get(desc.get("outlet"), 0)
    sim, r = run_gpu(mesh, Q, om, uin, fields, lbm.FP32DEV, K, W_, device, dist,
                     want_moments=not args.no_variants, outlet=outlet)
    clocks = clk.stop()
    e2e = e2e_run(sim, mesh, fields, K)
    if dist is not None:
        e2e["value"] = job_throughput(K * U, e2e["seconds"], world, dist, device)
    mom32 = r.pop("moments", None)
    sim.close()
    del sim
    torch.cuda.empty_cache()

    variants, errors, tgv, adj = {}, {}, None, None
    if not args.no_variants and rank == 0 and world == 1:
        mom = {}
        for name, prec in (("fp64", lbm.FP64), ("bf16dev", lbm.BF16DEV)):
            s2, r2 = run_gpu(mesh, Q, om, uin, fields, prec, K, W_, device, None, want_moments=True,
                             outlet=outlet)
            mom[name] = r2.pop("moments")
            variants[name] = {"mlups": r2["mlups"], "ms_per_step": r2["ms_per_step"],
                              "finest_kernel_gbs": r2["finest_gbs"], "finest_kernel_frac": r2["finest_gbs"] / peak,
                              "bytes_per_update": r2["bytes_per_update"], "device_gb": r2["device_gb"],
                              "reduce": r2["reduce"]}
            if name == "fp64":
                rec = fp64_instruction_record()
                rate = r2["finest_units"] / (r2["finest_launch_ms"] * 1e-3)  # elements / s
                variants[name]["alu_roofline"] = None if rec is None else {
                    "bound": "alu", "unit": "G FP64 inst/s",
                    "achieved": rate * rec["fp64_inst_per_unit"] / 1e9,
                    "peak": rec["peak_fp64_inst_per_s"] / 1e9,
                    "frac": rate * rec["fp64_inst_per_unit"] / rec["peak_fp64_inst_per_s"],
                    "fp64_inst_per_update": rec["fp64_inst_per_unit"], "flops_per_update": rec["flops_per_unit"],
                    "peak_source": "152 SMs x 2 FP64 inst/clock x 2.07 GHz (profiles/stream_collide_brick_fp64_tgv3d.md)"}
            s2.close()
            del s2
            torch.cuda.empty_cache()
        # the paper's own 3D stencil on the same mesh, FP32 deviation storage
        s27, r27 = run_gpu(mesh, 27, om, uin, fields, lbm.FP32DEV, K, W_, device, None, outlet=outlet)
        variants["d3q27_fp32dev"] = {
            "mlups": r27["mlups"], "ms_per_step": r27["ms_per_step"], "kernel": r27["finest_kernel"],
            "finest_kernel_gbs": r27["finest_gbs"], "finest_kernel_frac": r27["finest_gbs"] / peak,
            "bytes_per_update": r27["bytes_per_update"], "device_gb": r27["device_gb"],
            "interior_fraction": r27["interior_fraction"], "reduce": r27["reduce"]}
        s27.close()
        del s27
        torch.cuda.empty_cache()
        ref_u = mom["fp64"][1]
        ref_red = variants["fp64"]["reduce"]
        for name, m_ in (("fp32dev", mom32), ("bf16dev", mom["bf16dev"])):
            if m_ is None:
                continue
            du = m_[1] - ref_u
            red = r["reduce"] if name == "fp32dev" else variants["bf16dev"]["reduce"]
            errors[name] = {
                "u_l2_rel_vs_fp64": float(math.sqrt((du ** 2).sum() / (ref_u ** 2).sum())),
                "u_max_abs_vs_fp64": float(np.abs(du).max()),
                "drag_rel_vs_fp64": float(abs(red[4] - ref_red[4]) / abs(ref_red[4])) if ref_red[4] else None,
                "after_coarse_steps": W_ + K}
        del mom
        # secondary: the 64^3 / 32^3 two-level Taylor-Green (working set fits in L2)
        from paper_1601_06984_gb300 import workloads as Wk
        tm, tQ, tom, tuin, tfields, tdesc = make_workload("tgv3d")
        tgv = {"config": tdesc, "note": "working set (~0.13 GB) fits in the 129 MB L2 plus HBM; L2 not flushed; "
                                         "steps replay the library's CUDA graphs (launch-bound size)"}
        for name, prec in (("fp32dev", lbm.FP32DEV), ("fp64", lbm.FP64)):
            st, rt = run_gpu(tm, tQ, tom, tuin, tfields, prec, 50, 3, device, None, want_moments=True,
                             kernel_timing=False)
            _, ut, _ = rt.pop("moments")
            nu = (1 / 1.6 - 0.5) / 3
            _, ua, _ = Wk.tgv_fields(tm, 0.01, t=53, nu=nu)
            tgv[name] = {"mlups": rt["mlups"], "ms_per_step": rt["ms_per_step"],
                         "u_l2_rel_vs_closed_form": float(math.sqrt(((ut - ua) ** 2).sum() / (ua ** 2).sum()))}
            st.close()
            del st
            torch.cuda.empty_cache()
        adj = adjoint_run(device)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    cb = cpu_oracle(args.cpu_seconds) if world == 1 else None
    value = world * r["mlups"]
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": K, "warmup": W_,
        "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": dict(desc, elements=mesh.n, updates_per_coarse_step=U, storage="fp32 deviation g=f-w*rho0",
                       time_mode="linear", parallelism="replicas" if world > 1 else "single GPU",
                       l2="inputs larger than L2 (%.1f GB workspace)" % r["device_gb"]),
        "roofline": {"bound": "hbm", "achieved": r["finest_gbs"], "peak": peak, "unit": "GB/s",
                     "frac": r["finest_gbs"] / peak,
                     "traffic": None if traffic_per_unit is None else traffic_per_unit * r["finest_units"],
                     "traffic_source": "ncu capture on the half-scale sphere scaled by units "
                                       "(profiles/stream_collide_brick_fp32_sphere.md)",
                     "kernel": r["finest_kernel"] + "<19,float> on the finest level",
                     "units_per_launch": r["finest_units"], "bytes_per_unit": r["bytes_per_update"],
                     "avg_launch_ms": r["finest_launch_ms"], "peak_source": peak_src},
        "step_gbs_algorithmic": r["step_bytes"] / (r["ms_per_step"] * 1e-3) / 1e9,
        "interior_brick_fraction": r["interior_fraction"],
        "brick_fraction": r["brick_fraction"],
        "finest_boundary_brick_kernel": {"units_per_launch": r["finest_boundary_units"],
                                         "avg_launch_ms": r["finest_boundary_launch_ms"],
                                         "achieved_gbs": r["finest_boundary_gbs"],
                                         "bytes_per_unit": bytes_per_update(Q, lbm.FP32DEV, brick=True)},
        "finest_list_kernel": {"units_per_launch": r["finest_list_units"],
                               "avg_launch_ms": r["finest_list_launch_ms"], "achieved_gbs": r["finest_list_gbs"],
                               "bytes_per_unit": bytes_per_update(Q, lbm.FP32DEV)},
        "cpu_baseline": cb if cb is None else {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "e2e": {k: e2e[k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step")},
        "gpu_launches": r["launches"], "clocks": clocks,
        "level_stream_collide_ms": r["level_ms"], "level_stream_collide_launches": r["level_launches"],
        "drag_force_fp32dev": r["reduce"][4],
    }
    if variants:
        line["variants"] = variants
        line["error_vs_fp64"] = errors
    if tgv:
        line["tgv3d"] = tgv
    if adj:
        line["adjoint"] = adj
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

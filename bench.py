#!/usr/bin/env python
"""Benchmark of the multilevel D3Q19 lattice Boltzmann hot path on GB300.

Default workload: the sphere flow at Re = 100 (box 32D x 16D x 16D, sphere
D = 64 finest elements, five levels D/4 .. D/64, about 8.6e7 fluid elements,
velocity inlet / pressure outlet), FP32-deviation storage.  A "step" is one
coarse time step of the whole hierarchy (31 level substeps of stream-collide
plus the ghost fills).  The metric is fine-substep weighted MLUPS,
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
NOMINAL_HBM_GBS = 8000.0
SMI_FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
KINDS = ("interior", "list", "boundary", "gff", "moments", "gfc", "outlet")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sphere", choices=["sphere", "sphere_half", "tgv3d"],
                    help="sphere_half: every length halved (about 1.1e7 elements), for profiling captures")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the FP64/BF16/D3Q27 variants, the precision errors, the side workloads, the "
                         "adjoint and the oracle timings of the other configurations")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the oracle CPU baseline")
    ap.add_argument("--develop-steps", type=int, default=400,
                    help="coarse steps from rest before the precision comparison")
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


def bytes_per_update(Q, prec, brick=False):
    """Algorithmic HBM bytes of one element update: Q pdf reads and Q writes,
    plus the 32-bit neighbour list (Q-1 entries) for the neighbour-list kernel
    or one 27-entry row of neighbour-brick indices per 64 elements for the
    brick kernels."""
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


def _profile_record(name):
    """A committed ncu record under profiles/, if the stream-collide source
    (kernels.cuh, sections "physics" to "outlet values") is unchanged since it
    was taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", name)) as fh:
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


def stream_collide_traffic():
    """DRAM bytes per element update of the finest level's stream-collide
    kernels (interior bricks, boundary bricks, neighbour list) from the
    committed ncu capture (None once the kernel source changed)."""
    rec = _profile_record("stream_collide_brick_fp32_sphere.json")
    if rec is None:
        return None
    return {k: float(rec[k]) for k in ("dram_bytes_per_unit", "boundary_dram_bytes_per_unit",
                                       "list_dram_bytes_per_unit") if k in rec}


def fp64_instruction_record():
    """FP64 instructions and flops per element update of the interior-brick
    kernel from the committed ncu count (None once the kernel changed)."""
    return _profile_record("stream_collide_brick_fp64_tgv3d.json")


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
def oracle_cases():
    """The oracle timing cases: the configurations' meshes (config 2 and the
    sphere as bounded samples) with their parameters."""
    from paper_1601_06984_gb300 import workloads as W
    cyl_om = W.omega_coarse_from_finest(W.omega_for_re(0.05, 40, 100.0), 4)
    sph_om = W.omega_coarse_from_finest(W.omega_for_re(0.04, 64, 100.0), 3)
    return {
        "tgv2d_two_level_32": (W.config_tgv2d, 9, 1.6, (0.0, 0.0, 0.0), 0, lambda m: W.tgv_fields(m, 0.01)),
        "tgv3d_two_level_64": (lambda: W.config_tgv3d(64), 19, 1.6, (0.0, 0.0, 0.0), 0,
                               lambda m: W.tgv_fields(m, 0.01)),
        "cylinder_d2q9_4level": (W.config_cylinder, 9, cyl_om, (0.05, 0.0, 0.0), 1,
                                 lambda m: W.uniform_fields(m, 1.0, (0.05, 0.0))),
        "sphere_sample_3level": (W.config_sphere_small, 19, sph_om, (0.04, 0.0, 0.0), 1,
                                 lambda m: W.uniform_fields(m, 1.0, (0.04, 0.0, 0.0))),
    }


def oracle_rate(name, seconds, threads, min_steps=2):
    """Time the oracle (FP64, as it stands) on one case with the given thread
    count (0: every host core); returns MLUPS and what was run."""
    from oracle import oracle as O
    make, Q, om, uin, outlet, fields = oracle_cases()[name]
    used = O.set_threads(threads if threads > 0 else (os.cpu_count() or 1))
    m = make()
    o = O.Oracle(m, Q, om, u_in=uin, outlet=outlet)
    o.init(*fields(m))
    o.step(1)
    steps, t0 = 0, time.perf_counter()
    while steps < min_steps or time.perf_counter() - t0 < seconds:
        o.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    U = m.updates_per_coarse_step()
    O.set_threads(0)
    return {"value": steps * U / dt / 1e6, "unit": "MLUPS", "cores": used, "kind": "oracle",
            "sample": f"{name} ({m.n} elements, {U} updates/coarse step), {steps} coarse steps, FP64 oracle on "
                      f"{used} host thread{'s' if used > 1 else ''}",
            "seconds": round(dt, 2), "ms_per_step": 1e3 * dt / steps}


def oracle_timings(seconds_each):
    """Oracle MLUPS on every configuration, one thread and every host core."""
    out = {"host_cores": os.cpu_count()}
    for name in oracle_cases():
        one = oracle_rate(name, seconds_each, 1)
        allc = oracle_rate(name, seconds_each, 0)
        out[name] = {"single_thread_mlups": one["value"], "all_cores_mlups": allc["value"],
                     "threads": allc["cores"], "sample_steps": allc["sample"].split(", ")[1]}
    out["note"] = ("config 2 and the sphere are run on their meshes as given (64^3 two-level TGV) and on the "
                   "reduced 3-level sphere sample; the full 5-level sphere (8.6e7 elements) would take the oracle "
                   "about 8.6e7 x 31 / rate seconds per coarse step")
    return out


# ---------------------------------------------------------------- GPU runs
OUTLETS = {"linear": 0, "zero-gradient": 1}


def run_gpu(mesh, Q, om, uin, fields, prec, K, W_, device, dist=None, want_moments=False, outlet=0,
            timing=2, breakdown=True, state=None, time_mode=0):
    """Time K coarse steps after W_ warm-up steps, the way a caller's
    lbm_step(K) runs them: replaying the library's captured two-step CUDA
    graphs.  timing=2 has those graphs record CUDA events around the finest
    level's stream-collide launches (the roofline kernel's launch time comes
    from the last replay of the timed region); timing=0 records none.  With
    breakdown, K more steps follow with every kernel bracketed by events
    (launched kernel by kernel) for the per-kind and per-level times.
    state: post-collision pdfs [n, Q] to start from instead of the fields.
    time_mode 2 (diffusive scaling) takes four substeps per coarser step."""
    import numpy as np
    import torch

    from paper_1601_06984_gb300 import lbm
    msub = 4 if time_mode == 2 else 2
    U = mesh.updates_per_coarse_step(msub)
    t_build = time.perf_counter()
    sim = lbm.Sim(mesh, Q, om, precision=prec, u_in=uin, device=device, outlet=outlet, time_mode=time_mode)
    t_build = time.perf_counter() - t_build
    if state is None:
        rho, u, S = fields(mesh)
        sim.init(rho, u, S)
    else:
        sim.set_state(state)
    sim.timing_enable(timing)
    sim.step(W_)
    sim.step(2)  # captures the graph of the parity state the timed region starts from
    info = sim.mesh_info()
    stream = sim.stream
    sim.timing_read()  # clears the warm-up record
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(device)
    n0 = sim.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sim.step(K)
    ev1.record(stream)
    torch.cuda.synchronize(device)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(device)
    ms = ev0.elapsed_time(ev1)
    launches = sim.kernel_launches() - n0
    nl, kms = sim.timing_read()
    ms = max_over_ranks(ms, dist, device)
    finest = len(info) - 1
    nlev = len(info)
    # dominant kernel: the interior-brick stream-collide of the finest level
    # (the neighbour-list kernel when the level has no interior bricks)
    kb = 0 if info[finest, 8] > 0 else 1
    units = int(64 * info[finest, 8]) if kb == 0 else int(info[finest, 1])
    timed = timing == 2 and nl[finest, kb] > 0
    avg_ms = kms[finest, kb] / nl[finest, kb] if timed else float("nan")
    bpu = bytes_per_update(Q, prec, brick=kb == 0)
    list_units = int(info[finest, 1] - 64 * (info[finest, 8] + info[finest, 9]))
    list_ms = kms[finest, 1] / max(nl[finest, 1], 1)
    bnd_units = int(64 * info[finest, 9])
    bnd_ms = kms[finest, 2] / max(nl[finest, 2], 1)
    # algorithmic bytes of one coarse step: every level's interior and boundary
    # bricks at the brick rate, the rest at the neighbour-list rate, times its
    # substeps per coarse step
    brick_units = [int(64 * (info[li, 8] + info[li, 9])) for li in range(nlev)]
    step_bytes = float(sum(msub ** li * (brick_units[li] * bytes_per_update(Q, prec, brick=True)
                                        + (info[li, 1] - brick_units[li]) * bytes_per_update(Q, prec))
                           for li in range(nlev)))
    # the finest level's stream-collide as one op: its three kernels run as
    # parallel graph branches, timed from fork to join (timing kind 7)
    span_ms = kms[finest, 7] / nl[finest, 7] if timing == 2 and nl[finest, 7] > 0 else None
    sc_bytes = (units * bpu + bnd_units * bytes_per_update(Q, prec, brick=True)
                + list_units * bytes_per_update(Q, prec)) if kb == 0 else units * bpu
    res_sc = {"span_ms": span_ms, "bytes": sc_bytes, "units": int(info[finest, 1]),
              "gbs": sc_bytes / (span_ms * 1e-3) / 1e9 if span_ms else None}
    res = {"ms_total": ms, "ms_per_step": ms / K, "mlups": K * U / (ms * 1e-3) / 1e6, "launches": launches,
           "finest_sc": res_sc,
           "finest_kernel": "k_stream_collide_brick" if kb == 0 else "k_stream_collide",
           "finest_launch_ms": avg_ms, "finest_launches": int(nl[finest, kb]), "finest_units": units,
           "finest_bytes": units * bpu, "finest_gbs": units * bpu / (avg_ms * 1e-3) / 1e9 if timed else None,
           "finest_list_units": list_units, "finest_list_launch_ms": list_ms,
           "finest_boundary_units": bnd_units, "finest_boundary_launch_ms": bnd_ms,
           "finest_boundary_gbs": (bnd_units * bytes_per_update(Q, prec, brick=True) / (bnd_ms * 1e-3) / 1e9
                                   if nl[finest, 2] > 0 and bnd_ms > 0 else None),
           "finest_list_gbs": (list_units * bytes_per_update(Q, prec) / (list_ms * 1e-3) / 1e9
                               if nl[finest, 1] > 0 and list_ms > 0 else None),
           "interior_fraction": float(64 * info[:, 8].sum() / info[:, 1].sum()),
           "brick_fraction": float(64 * (info[:, 8] + info[:, 9]).sum() / info[:, 1].sum()),
           "step_bytes": step_bytes, "bytes_per_update": bpu, "build_s": t_build,
           "device_gb": sim.device_bytes() / 1e9}
    if breakdown:
        sim.timing_enable(1)
        torch.cuda.synchronize(device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(K)
        e1.record(stream)
        torch.cuda.synchronize(device)
        ms1 = e0.elapsed_time(e1)
        nl1, kms1 = sim.timing_read()
        per_kind = {k: float(kms1[:, i].sum() / K) for i, k in enumerate(KINDS)}
        res["breakdown"] = {"ms_per_step": ms1 / K,
                            "kinds_ms_per_step": dict(per_kind, between_kernels=ms1 / K - sum(per_kind.values())),
                            "note": "K further steps with every kernel bracketed by CUDA events, launched kernel "
                                    "by kernel (the events add about 2 us per launch)"}
        res["level_ms_per_step"] = {f"L{int(info[li, 0])}": {k: round(float(kms1[li, i] / K), 4)
                                                            for i, k in enumerate(KINDS) if nl1[li, i] > 0}
                                    for li in range(nlev)}
        # the finest level's boundary-brick and neighbour-list kernels launched
        # alone (in the graph they run beside the interior bricks, and their
        # events there span the shared time)
        for kind, key, brick in ((2, "boundary", True), (1, "list", False)):
            n_ = bnd_units if kind == 2 else list_units
            if nl1[finest, kind] > 0 and n_ > 0:
                t_ = kms1[finest, kind] / nl1[finest, kind]
                res[f"finest_{key}_launch_ms"] = float(t_)
                res[f"finest_{key}_gbs"] = n_ * bytes_per_update(Q, prec, brick=brick) / (t_ * 1e-3) / 1e9
        # every level's brick stream-collide against the HBM roofline
        res["level_brick_gbs"] = {}
        for li in range(nlev):
            for i, key in ((0, "interior"), (2, "boundary")):
                n_ = int(64 * info[li, 8 if i == 0 else 9])
                if nl1[li, i] > 0 and n_ > 0:
                    res["level_brick_gbs"][f"L{int(info[li, 0])}_{key}"] = round(
                        n_ * bytes_per_update(Q, prec, brick=True) / (kms1[li, i] / nl1[li, i] * 1e-3) / 1e9, 1)
    sim.timing_enable(0)
    res["reduce"] = sim.reduce().tolist()
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


def sphere_adjoint_run(mesh, Q, om, uin, fields, outlet, device, n=4, K=2):
    """Adjoint at production size: the bench sphere, FP32 deviation storage,
    drag objective, n coarse steps with checkpoints every K, each step recorded
    in a recompute of its own (adjoint_tape 2, the smaller workspace).  Time of
    the adjoint (forward with checkpoints, recomputes, reverse sweep) over the
    forward alone (n steps through lbm_step's graphs)."""
    import torch
    from paper_1601_06984_gb300 import lbm
    rec = {"config": f"sphere_re100_d3q19_5level FP32 deviation, drag (F_x) objective, {n} coarse steps, K={K}, "
                     "step-by-step recording"}
    g = None
    try:
        g = lbm.Sim(mesh, Q, om, precision=lbm.FP32DEV, u_in=uin, outlet=outlet, device=device, adjoint_tape=2)
        rho, u, S = fields(mesh)
        g.init(rho, u, S)
        g.step(4)
        f0 = g.get_state()
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        g.step(n)
        g.reduce()
        tf = time.perf_counter() - t0
        g.set_state(f0)
        del f0
        rec["adjoint_workspace_gb"] = g.adjoint_bytes(n, K) / 1e9
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        J, _, dw, dU = g.adjoint(n, K, 1, want_force=False)
        ta = time.perf_counter() - t0
        rec.update({"forward_s": tf, "adjoint_s": ta, "adjoint_to_forward": ta / tf, "J_drag": J,
                    "dJ_domega_c": dw, "dJ_du_in_x": float(dU[0])})
    except Exception as ex:  # reported, not fatal: the workspace is the largest allocation of the run
        rec["error"] = repr(ex)[:300]
    if g is not None:
        g.close()
    torch.cuda.empty_cache()
    return rec


def e2e_run(sim, mesh, fields, K):
    """End to end through the C ABI: initial fields from pinned host memory,
    then K coarse steps each followed by the FP64 reduction (mass, momentum,
    drag, kinetic energy) read back to the host; two untimed iterations of the
    same loop first."""
    import torch
    rho, u, _ = fields(mesh)
    rho_p = torch.from_numpy(rho).pin_memory()
    u_p = torch.from_numpy(u).pin_memory()
    # untimed warm-up of the same loop: captures the one-step graphs of both
    # parity states (a timing-mode change before this dropped the captured steps)
    for _ in range(2):
        sim.step(1)
        sim.reduce()
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


def _rel_l2(a, b):
    import numpy as np
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def precision_study(mesh, Q, om, uin, fields, K, W_, device, outlet, develop, peak, sim32, done):
    """Precision variants from a developed flow.  The FP32-deviation run, `done`
    coarse steps from rest, is carried on by `develop` more; its state (FP64 host copy)
    then starts an FP64, an FP32-deviation and a BF16-deviation run, each timed
    over K steps after W_ warm-up steps.  The errors of FP32 and BF16 against
    FP64 after those W_ + K steps: velocity and strain rate (relative l2 over
    all fluid elements, strain rate in coarsest-level units as the error norm of
    Sec. 4.1), drag and lift (momentum exchange on the sphere)."""
    import numpy as np
    import torch

    from paper_1601_06984_gb300 import lbm
    t0 = time.perf_counter()
    sim32.step(develop)
    f_dev = sim32.get_state()
    t_dev = time.perf_counter() - t0
    sim32.close()
    torch.cuda.empty_cache()
    sc = np.ldexp(1.0, mesh.levels.astype(np.int64) - mesh.lmin)[:, None]
    rec, mom, red = {}, {}, {}
    for name, prec in (("fp64", lbm.FP64), ("fp32dev", lbm.FP32DEV), ("bf16dev", lbm.BF16DEV)):
        s, r = run_gpu(mesh, Q, om, uin, fields, prec, K, W_, device, None, want_moments=True, outlet=outlet,
                       state=f_dev)
        # the precision's own steps from the developed state: W_ + 2 warm-up, K
        # timed, K with per-kernel events (moments after all of them)
        steps_run = W_ + 2 + 2 * K
        _, u, S = r.pop("moments")
        mom[name] = (u, S * sc)
        red[name] = np.asarray(r["reduce"])
        rec[name] = {"mlups": r["mlups"], "ms_per_step": r["ms_per_step"], "finest_kernel_gbs": r["finest_gbs"],
                     "finest_kernel_frac": r["finest_gbs"] / peak, "bytes_per_update": r["bytes_per_update"],
                     "device_gb": r["device_gb"], "step_gbs_algorithmic": r["step_bytes"] / (r["ms_per_step"] * 1e-3) / 1e9,
                     "breakdown": r["breakdown"], "finest_units": r["finest_units"],
                     "finest_launch_ms": r["finest_launch_ms"], "finest_sc": r["finest_sc"], "reduce": r["reduce"]}
        if r["finest_sc"]["gbs"]:
            rec[name]["finest_sc_frac"] = r["finest_sc"]["gbs"] / peak
        s.close()
        del s
        torch.cuda.empty_cache()
    del f_dev
    ref_u, ref_S = mom["fp64"]
    rf = red["fp64"]
    errors = {}
    for name in ("fp32dev", "bf16dev"):
        u, S = mom[name]
        rp = red[name]
        errors[name] = {"u_l2_rel_vs_fp64": _rel_l2(u, ref_u), "S_l2_rel_vs_fp64": _rel_l2(S, ref_S),
                        "u_max_abs_vs_fp64": float(np.abs(u - ref_u).max()),
                        "drag_rel_vs_fp64": float(abs(rp[4] - rf[4]) / abs(rf[4])) if rf[4] else None,
                        "lift_y_vs_fp64_rel_to_drag": float(abs(rp[5] - rf[5]) / abs(rf[4])) if rf[4] else None,
                        "lift_z_vs_fp64_rel_to_drag": float(abs(rp[6] - rf[6]) / abs(rf[4])) if rf[4] else None,
                        "mass_rel_vs_fp64": float(abs(rp[0] - rf[0]) / rf[0])}
    errors["state"] = (f"flow developed for {done + develop} coarse steps from rest (uniform u_in) in FP32-deviation storage, "
                       f"then each precision runs {steps_run} coarse steps from that state; fp64 drag "
                       f"{rf[4]:.6g}, lift {rf[5]:.3g}, {rf[6]:.3g} (finest-level lattice units)")
    errors["develop_seconds"] = round(t_dev, 1)
    return rec, errors


def side_workload(mesh, Q, om, uin, fields, precs, steps, device, outlet=0, ref=None):
    """MLUPS of a small workload through graph replay (lbm_step(steps)), and
    the velocity error against `ref(mesh, steps)` when given."""
    import numpy as np
    import torch

    from paper_1601_06984_gb300 import lbm
    out = {}
    for name, prec in precs:
        s, r = run_gpu(mesh, Q, om, uin, fields, prec, steps, 3, device, None, want_moments=ref is not None,
                       outlet=outlet, timing=0, breakdown=False)
        rec = {"mlups": r["mlups"], "ms_per_step": r["ms_per_step"],
               "hbm_gbs_algorithmic": r["step_bytes"] / (r["ms_per_step"] * 1e-3) / 1e9}
        if ref is not None:
            _, u, _ = r.pop("moments")
            ua = ref(mesh, steps + 5)  # 3 + 2 warm-up steps, then the timed ones
            rec["u_l2_rel_vs_closed_form"] = float(np.sqrt(((u - ua) ** 2).sum() / (ua ** 2).sum()))
        out[name] = rec
        s.close()
        del s
        torch.cuda.empty_cache()
    return out


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
        # each timed step is one coarse step of the bounded sample; the oracle
        # runs until K steps and the time budget are both used
        cb = oracle_rate("sphere_sample_3level", max(5.0, min(args.cpu_seconds, 20.0)), 0, min_steps=K)
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
    sim, r = run_gpu(mesh, Q, om, uin, fields, lbm.FP32DEV, K, W_, device, dist, outlet=outlet)
    clocks = clk.stop()
    e2e = e2e_run(sim, mesh, fields, K)
    if dist is not None:
        e2e["value"] = job_throughput(K * U, e2e["seconds"], world, dist, device)

    variants, errors, side, adj, oracles, alu = {}, {}, {}, None, None, None
    if not args.no_variants and rank == 0 and world == 1:
        # the FP32 context is K steps past its last init (the end-to-end run)
        rec, errors = precision_study(mesh, Q, om, uin, fields, K, W_, device, outlet, args.develop_steps, peak,
                                      sim, K)
        sim = None
        variants = {"fp64": rec["fp64"], "bf16dev": rec["bf16dev"], "fp32dev_from_developed_state": rec["fp32dev"]}
        # FP64 against the FP64 pipe: instructions per update from the committed
        # ncu count, peak from the multiply-add probe run now
        fp64_peak = lbm.lbm_alu_peak(lbm.FP64, device)
        fp32_peak = lbm.lbm_alu_peak(lbm.FP32DEV, device)
        alu = {"fp64_gflops": fp64_peak, "fp32_gflops": fp32_peak,
               "how": "lbm_alu_peak: register-only multiply-add chains on every SM, CUDA events, 2 flop per FMA"}
        irec = fp64_instruction_record()
        v = rec["fp64"]
        # element updates / s of the finest level's stream-collide (all three
        # kernels, fork to join; they share the FP64 pipe)
        fsc = v["finest_sc"]
        rate = (fsc["units"] / (fsc["span_ms"] * 1e-3) if fsc["span_ms"]
                else v["finest_units"] / (v["finest_launch_ms"] * 1e-3))
        variants["fp64"]["alu_roofline"] = None if irec is None else {
            "bound": "alu", "unit": "GFLOP/s", "achieved": rate * irec["flops_per_unit"] / 1e9,
            "peak": fp64_peak, "frac": rate * irec["fp64_inst_per_unit"] / (fp64_peak / 2 * 1e9),
            "frac_meaning": "FP64 instructions issued / FP64 multiply-adds per second the probe reached",
            "fp64_inst_per_update": irec["fp64_inst_per_unit"], "flops_per_update": irec["flops_per_unit"],
            "peak_source": "measured: lbm_alu_peak(LBM_FP64) in this run"}
        # the paper's own 3D stencil on the same mesh, FP32 deviation storage
        s27, r27 = run_gpu(mesh, 27, om, uin, fields, lbm.FP32DEV, K, W_, device, None, outlet=outlet,
                           breakdown=False)
        variants["d3q27_fp32dev"] = {
            "mlups": r27["mlups"], "ms_per_step": r27["ms_per_step"], "kernel": r27["finest_kernel"],
            "finest_kernel_gbs": r27["finest_gbs"], "finest_kernel_frac": r27["finest_gbs"] / peak,
            "bytes_per_update": r27["bytes_per_update"], "device_gb": r27["device_gb"],
            "step_gbs_algorithmic": r27["step_bytes"] / (r27["ms_per_step"] * 1e-3) / 1e9,
            "interior_fraction": r27["interior_fraction"], "reduce": r27["reduce"]}
        s27.close()
        del s27
        torch.cuda.empty_cache()
        # diffusive scaling (dt ~ dx^2) on the same mesh: four substeps per
        # coarser step (256 on the finest level per coarse step), four
        # GhostFromCoarser layers, omega 1.8 on every level, the inlet velocity
        # halved per level; FP32 deviation storage
        from paper_1601_06984_gb300 import workloads as Wk
        sd, rd = run_gpu(mesh, Q, 1.8, uin, lambda m: Wk.diffusive_units(m, *fields(m)), lbm.FP32DEV, 2, 3,
                         device, None, outlet=outlet, breakdown=False, time_mode=2)
        fsc = rd["finest_sc"]
        variants["diffusive_fp32dev"] = {
            "mlups": rd["mlups"], "ms_per_step": rd["ms_per_step"], "steps": 2, "warmup": 3,
            "updates_per_coarse_step": mesh.updates_per_coarse_step(4), "omega_all_levels": 1.8,
            "kernel": rd["finest_kernel"], "finest_kernel_gbs": rd["finest_gbs"],
            "finest_kernel_frac": None if rd["finest_gbs"] is None else rd["finest_gbs"] / peak,
            "finest_sc_gbs": fsc["gbs"], "finest_sc_frac": None if fsc["gbs"] is None else fsc["gbs"] / peak,
            "step_gbs_algorithmic": rd["step_bytes"] / (rd["ms_per_step"] * 1e-3) / 1e9,
            "step_frac": rd["step_bytes"] / (rd["ms_per_step"] * 1e-3) / 1e9 / peak,
            "device_gb": rd["device_gb"], "launches_per_step": rd["launches"] / 2, "reduce": rd["reduce"]}
        sd.close()
        del sd
        torch.cuda.empty_cache()
        # side workloads (working sets that fit in L2: launch- and latency-bound sizes)
        from paper_1601_06984_gb300 import workloads as Wk
        nu = (1 / 1.6 - 0.5) / 3
        tm = Wk.config_tgv3d(64)
        side["tgv3d"] = {"config": {"workload": "tgv3d_two_level_64", "box": "64^3 periodic, 32^3 block refined",
                                    "levels": 2, "u0": 0.01, "omega_coarse": 1.6},
                         **side_workload(tm, 19, 1.6, (0, 0, 0), lambda m: Wk.tgv_fields(m, 0.01),
                                         (("fp32dev", lbm.FP32DEV), ("fp64", lbm.FP64)), 50, device,
                                         ref=lambda m, t: Wk.tgv_fields(m, 0.01, t=t, nu=nu)[1])}
        cm = Wk.config_cylinder()
        cyl_om = Wk.omega_coarse_from_finest(Wk.omega_for_re(0.05, 40, 100.0), 4)
        side["cylinder2d"] = {"config": {"workload": "cylinder_re100_d2q9_4level", "channel": "40D x 20D",
                                         "D_finest": 40, "levels": 4, "u_in": 0.05, "elements": cm.n,
                                         "updates_per_coarse_step": cm.updates_per_coarse_step(),
                                         "omega_coarsest": round(cyl_om, 6), "outlet": "zero-gradient"},
                              **side_workload(cm, 9, cyl_om, (0.05, 0, 0),
                                              lambda m: Wk.uniform_fields(m, 1.0, (0.05, 0.0)),
                                              (("fp32dev", lbm.FP32DEV), ("fp64", lbm.FP64)), 200, device,
                                              outlet=1)}
        for v_ in side.values():
            v_["note"] = ("working set fits in the 129 MB L2 (not flushed); steps replay the library's CUDA "
                          "graphs; hbm_gbs_algorithmic counts the algorithmic bytes, most of which L2 serves")
        adj = adjoint_run(device)
        adj["sphere"] = sphere_adjoint_run(mesh, Q, om, uin, fields, outlet, device)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    cb = None
    if world == 1:
        cb = oracle_rate("sphere_sample_3level", args.cpu_seconds, 0)
        if not args.no_variants:
            oracles = oracle_timings(max(2.0, args.cpu_seconds / 4))
    value = world * r["mlups"]
    step_gbs = r["step_bytes"] / (r["ms_per_step"] * 1e-3) / 1e9
    sc = r["finest_sc"]
    if sc["gbs"] is None:  # no span recorded (no graphs): the interior kernel alone
        sc = {"gbs": r["finest_gbs"], "span_ms": r["finest_launch_ms"], "bytes": r["finest_bytes"],
              "units": r["finest_units"]}
    traffic = None
    if traffic_per_unit and len(traffic_per_unit) == 3:
        traffic = (traffic_per_unit["dram_bytes_per_unit"] * r["finest_units"]
                   + traffic_per_unit["boundary_dram_bytes_per_unit"] * r["finest_boundary_units"]
                   + traffic_per_unit["list_dram_bytes_per_unit"] * r["finest_list_units"])
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": K, "warmup": W_,
        "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": dict(desc, elements=mesh.n, updates_per_coarse_step=U, storage="fp32 deviation g=f-w*rho0",
                       time_mode="linear", parallelism="replicas" if world > 1 else "single GPU",
                       l2="inputs larger than L2 (%.1f GB workspace)" % r["device_gb"],
                       timing="K coarse steps through lbm_step's captured two-step CUDA graphs, CUDA events on the "
                              "bound stream around the region; the graphs also record events around the finest "
                              "level's stream-collide (roofline: the last replay's 32 finest-level spans)"),
        "roofline": {"bound": "hbm", "achieved": sc["gbs"], "peak": peak, "unit": "GB/s",
                     "frac": sc["gbs"] / peak,
                     "traffic": traffic,
                     "traffic_source": "ncu DRAM bytes per unit of each of the three kernels (half-scale sphere "
                                       "capture, profiles/stream_collide_brick_fp32_sphere.md) times its units",
                     "kernel": "finest-level stream-collide: k_stream_collide_brick<19,float> on the interior and "
                               "boundary bricks and k_stream_collide<19,float> on the other elements, run as "
                               "parallel branches of the captured step graph",
                     "units_per_launch": sc["units"], "bytes_per_unit": sc["bytes"] / sc["units"],
                     "avg_launch_ms": sc["span_ms"], "launches_averaged": r["finest_launches"],
                     "interior_kernel": {"units": r["finest_units"], "bytes_per_unit": r["bytes_per_update"],
                                         "avg_launch_ms": r["finest_launch_ms"], "achieved": r["finest_gbs"],
                                         "frac": r["finest_gbs"] / peak if r["finest_gbs"] else None,
                                         "note": "its own launch, sharing HBM with the concurrent branches"},
                     "peak_source": peak_src,
                     "step": {"achieved": step_gbs, "frac_of_measured": step_gbs / peak,
                              "frac_of_nominal": step_gbs / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS,
                              "bytes_per_step": r["step_bytes"],
                              "meaning": "algorithmic bytes of every level's stream-collide per coarse step "
                                         "over the whole step's time (ghost fills count as time, not bytes)"}},
        "breakdown": r["breakdown"],
        "level_ms_per_step": r["level_ms_per_step"],
        "level_brick_gbs": r["level_brick_gbs"],
        "interior_brick_fraction": r["interior_fraction"],
        "brick_fraction": r["brick_fraction"],
        "finest_boundary_brick_kernel": {"units_per_launch": r["finest_boundary_units"],
                                         "avg_launch_ms": r["finest_boundary_launch_ms"],
                                         "achieved_gbs": r["finest_boundary_gbs"],
                                         "bytes_per_unit": bytes_per_update(Q, lbm.FP32DEV, brick=True),
                                         "timing": "launched alone (kernel-by-kernel pass)"},
        "finest_list_kernel": {"units_per_launch": r["finest_list_units"],
                               "avg_launch_ms": r["finest_list_launch_ms"], "achieved_gbs": r["finest_list_gbs"],
                               "bytes_per_unit": bytes_per_update(Q, lbm.FP32DEV),
                               "timing": "launched alone (kernel-by-kernel pass)"},
        "cpu_baseline": cb if cb is None else {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "e2e": {k: e2e[k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step")},
        "gpu_launches": r["launches"], "clocks": clocks,
        "drag_force_fp32dev": r["reduce"][4],
    }
    if variants:
        line["variants"] = variants
        line["error_vs_fp64"] = errors
    if alu:
        line["alu_peaks"] = alu
    if side:
        line["side_workloads"] = side
    if adj:
        line["adjoint"] = adj
    if oracles:
        line["oracle_timings"] = oracles
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Flow studies on the GPU path: drag, lift and Strouhal number.

    python -m paper_1601_06984_gb300.studies cylinder --re 20 --precision fp32dev --steps 6000
    python -m paper_1601_06984_gb300.studies sphere --precision fp32dev --steps 2000

Coefficients follow Sec. 4.2 / 4.3 of arXiv:1601.06984: c_D = 2 F_x / (rho
U^2 A), c_L = 2 F_y / (rho U^2 A), A = D (2D) or pi D^2 / 4 (3D), St = f D / U
with f the lift oscillation frequency, and the sphere's recirculation length
L_r / D.  Forces come from the FP64
momentum-exchange reduction (lbm_reduce), in finest-level lattice units; D
and U are in those units too.  The geometries are the synthetic cylinder
channel and sphere box of workloads.py.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import lbm
from . import workloads as W

PRECISION = {"fp64": lbm.FP64, "fp32dev": lbm.FP32DEV, "bf16dev": lbm.BF16DEV}
OUTLET = {"linear": lbm.OUTLET_LINEAR, "zero-gradient": lbm.OUTLET_ZERO_GRADIENT}


def _outlet(outlet, omega_coarse):
    """'auto': the linear extrapolation of Sec. 2.3 unless the coarsest level
    relaxes at omega >= 1.9, where it diverges on a walled channel; then the
    zero-gradient extrapolation."""
    if outlet == "auto":
        outlet = "zero-gradient" if omega_coarse >= 1.9 else "linear"
    return outlet, OUTLET[outlet]


def _strouhal(cl, dt_finest, D, U, prominence=20.0, min_swing=1e-3):
    """Strouhal number of the lift signal (one sample per coarse step of
    dt_finest finest steps), or None when it has no dominant period (steady
    flow, or storage noise only): the lift must swing by at least min_swing
    and the peak of the Hann-windowed spectrum must exceed `prominence` times
    the median spectral power.  The peak frequency
    is located on a 16x zero-padded spectrum, refined by a parabola through
    the log power at the peak and its two neighbours."""
    x = np.asarray(cl, dtype=float)
    x = x - x.mean()
    n = len(x)
    # a steady flow: the lift swings by less than min_swing (shedding swings by ~1)
    if n < 32 or np.ptp(x) < min_swing:
        return None
    xw = x * np.hanning(n)
    power = np.abs(np.fft.rfft(xw)) ** 2
    k = 1 + int(np.argmax(power[1:]))
    if power[k] < prominence * np.median(power[1:]):
        return None
    pad = 16
    pz = np.abs(np.fft.rfft(xw, pad * n)) ** 2
    lo = max(1, pad * k - pad)
    kz = lo + int(np.argmax(pz[lo:pad * k + pad + 1]))
    shift = 0.0
    if 0 < kz < len(pz) - 1:
        a0, a1, a2 = np.log(pz[kz - 1:kz + 2] + 1e-300)
        den = a0 - 2 * a1 + a2
        if den < 0:
            shift = 0.5 * (a0 - a2) / den
    f = (kz + shift) / (pad * n * dt_finest)
    return f * D / U


def cylinder(Re=20.0, precision="fp32dev", steps=6000, window=2000, U=0.05, seed_amp=1e-6, outlet="auto",
             device="cuda"):
    mesh = W.config_cylinder()
    D = 40.0
    levels = len(mesh.level_counts())
    om_f = W.omega_for_re(U, D, Re)
    om_c = W.omega_coarse_from_finest(om_f, levels)
    outlet, out_code = _outlet(outlet, om_c)
    sim = lbm.Sim(mesh, 9, om_c, precision=PRECISION[precision], u_in=(U, 0.0, 0.0), device=device,
                  outlet=out_code)
    sim.init(*W.uniform_fields(mesh, 1.0, (U, 0.0)), W.pdf_perturbation(mesh, 9, seed_amp))
    fine_per_coarse = 1 << (levels - 1)
    cd, cl = [], []
    t0 = time.perf_counter()
    for k in range(steps):
        sim.step(1)
        if k >= steps - window:
            red = sim.reduce()
            cd.append(2.0 * red[4] / (U * U * D))
            cl.append(2.0 * red[5] / (U * U * D))
    wall = time.perf_counter() - t0
    out = {"case": "cylinder", "Re": Re, "precision": precision, "outlet": outlet, "coarse_steps": steps,
           "finest_steps": steps * fine_per_coarse, "omega_finest": om_f, "omega_coarsest": om_c,
           "c_D_last": cd[-1], "c_L_last": cl[-1], "c_D_mean": float(np.mean(cd)), "c_L_mean": float(np.mean(cl)),
           "c_D_max": float(np.max(cd)), "c_L_max": float(np.max(np.abs(cl))),
           "St": _strouhal(cl, fine_per_coarse, D, U), "seconds": wall}
    return out


def schafer(Re=20.0, precision="fp32dev", steps=20000, window=5000, D=40, U=0.05, outlet="auto", device="cuda"):
    """The paper's cylinder (Sec. 4.2): the 2.2 x 0.41 channel with the cylinder
    at (0.2, 0.2), parabolic inflow of mean U, interpolated bounce-back on the
    cylinder with the circle's wall distances, two levels with D finest cells
    across the cylinder.  c_D, c_L = 2 F / (rho U^2 D); St from the lift."""
    mesh = W.config_cylinder_schafer(D)
    om_f = W.omega_for_re(U, D, Re)
    om_c = W.omega_coarse_from_finest(om_f, 2)
    outlet, out_code = _outlet(outlet, om_c)
    sim = lbm.Sim(mesh, 9, om_c, precision=PRECISION[precision], u_in=(U, 0.0, 0.0), device=device,
                  outlet=out_code, inlet_profile=lbm.INLET_PARABOLIC, bouzidi=True)
    e, d = sim.obstacle_links()
    sim.set_link_q(W.wall_distance_ball(mesh, e, d, (2.0 * D, 2.0 * D), 0.5 * D, 9))
    sim.init(*W.uniform_fields(mesh, 1.0, (U, 0.0)))
    cd, cl = [], []
    t0 = time.perf_counter()
    chunk = 10
    for k in range(0, steps, chunk):
        sim.step(chunk)
        if k + chunk > steps - window:
            red = sim.reduce()
            cd.append(2.0 * red[4] / (U * U * D))
            cl.append(2.0 * red[5] / (U * U * D))
    wall = time.perf_counter() - t0
    return {"case": "cylinder (paper geometry)", "Re": Re, "D": D, "precision": precision, "outlet": outlet,
            "inlet": "parabolic", "walls": "interpolated bounce-back", "coarse_steps": steps,
            "omega_finest": om_f, "omega_coarsest": om_c, "c_D_last": cd[-1], "c_L_last": cl[-1],
            "c_D_mean": float(np.mean(cd)), "c_L_mean": float(np.mean(cl)), "c_D_max": float(np.max(cd)),
            "c_L_max": float(np.max(cl)), "St": _strouhal(cl, 2 * chunk, D, U), "seconds": wall,
            "samples_every_coarse_steps": chunk}


def recirculation_length(mesh, u, center, D):
    """Length of the recirculation zone behind a body centred on the x axis
    through `center` (finest-level cell units, a corner of the cells around
    the axis on every level), in diameters D: from the body's rear point
    center[0] + D/2 to the first point where the axial velocity u_x turns
    from negative to positive (Sec. 4.3, L_r).  u_x on the axis is the mean of
    the four cells around it at each cell-centre position x, linearly
    interpolated between positions.  None when the flow behind the body is not
    reversed."""
    lv = mesh.levels.astype(np.int64)
    h = np.ldexp(1.0, int(lv.max()) - lv)  # cell size in finest units
    cen = (np.asarray(mesh.coords, float) + 0.5) * h[:, None]
    on = ((np.abs(np.abs(cen[:, 1] - center[1]) - 0.5 * h) < 1e-9)
          & (np.abs(np.abs(cen[:, 2] - center[2]) - 0.5 * h) < 1e-9))
    x0 = center[0] + 0.5 * D
    sel = on & (cen[:, 0] > x0)
    if not sel.any():
        return None
    xs, inv = np.unique(cen[sel, 0], return_inverse=True)
    ux = np.bincount(inv, weights=np.asarray(u)[sel, 0]) / np.bincount(inv)
    if ux[0] >= 0.0:
        return None
    k = int(np.argmax(ux >= 0.0))
    if ux[k] < 0.0:
        return None  # reversed up to the last axis cell
    xc = xs[k - 1] + (0.0 - ux[k - 1]) * (xs[k] - xs[k - 1]) / (ux[k] - ux[k - 1])
    return float((xc - x0) / D)


def sphere(precision="fp32dev", steps=2000, window=200, U=0.04, Re=100.0, outlet="auto", Q=19, bouzidi=False,
           device="cuda"):
    """The bench's sphere (D = 64 finest cells, 5 levels), D3Q19 or the paper's
    D3Q27, half-way or interpolated bounce-back with the sphere's wall
    distances.  c_D = 2 F_x / (rho U^2 pi D^2 / 4); L_r / D from the final
    state's axial velocity (recirculation_length)."""
    mesh = W.config_sphere(1)
    D = 64.0
    om_f = W.omega_for_re(U, D, Re)
    om_c = W.omega_coarse_from_finest(om_f, 5)
    outlet, out_code = _outlet(outlet, om_c)
    sim = lbm.Sim(mesh, Q, om_c, precision=PRECISION[precision], u_in=(U, 0.0, 0.0), device=device,
                  outlet=out_code, bouzidi=bouzidi)
    if bouzidi:
        e, d = sim.obstacle_links()
        sim.set_link_q(W.wall_distance_ball(mesh, e, d, (8 * D,) * 3, 0.5 * D, Q))
    sim.init(*W.uniform_fields(mesh, 1.0, (U, 0.0, 0.0)))
    A = math.pi * D * D / 4.0
    cd = []
    t0 = time.perf_counter()
    for k in range(steps):
        sim.step(1)
        if k >= steps - window:
            cd.append(2.0 * sim.reduce()[4] / (U * U * A))
    wall = time.perf_counter() - t0
    _, u, _ = sim.moments()
    lr = recirculation_length(mesh, u, (8 * D,) * 3, D)
    return {"case": "sphere", "Re": Re, "precision": precision, "stencil": f"D3Q{Q}",
            "walls": "interpolated bounce-back" if bouzidi else "half-way bounce-back", "outlet": outlet,
            "coarse_steps": steps,
            "omega_coarsest": om_c, "c_D_last": cd[-1],
            "c_D_mean": float(np.mean(cd)), "L_r_over_D": lr, "seconds": wall}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["cylinder", "sphere", "schafer"])
    ap.add_argument("--D", type=int, default=40)
    ap.add_argument("--Q", type=int, default=19, choices=[19, 27])
    ap.add_argument("--bouzidi", action="store_true")
    ap.add_argument("--re", type=float, default=None)
    ap.add_argument("--precision", default="fp32dev", choices=list(PRECISION))
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--window", type=int, default=None)
    ap.add_argument("--outlet", default="auto", choices=["auto"] + list(OUTLET))
    ap.add_argument("--seed-amp", type=float, default=None)
    a = ap.parse_args()
    if a.case == "cylinder":
        kw = {"Re": a.re or 20.0, "precision": a.precision, "outlet": a.outlet}
        if a.seed_amp is not None:
            kw["seed_amp"] = a.seed_amp
        if a.steps:
            kw["steps"] = a.steps
        if a.window:
            kw["window"] = a.window
        print(json.dumps(cylinder(**kw)), flush=True)
    elif a.case == "schafer":
        kw = {"Re": a.re or 20.0, "precision": a.precision, "outlet": a.outlet, "D": a.D}
        if a.steps:
            kw["steps"] = a.steps
        if a.window:
            kw["window"] = a.window
        print(json.dumps(schafer(**kw)), flush=True)
    else:
        kw = {"precision": a.precision, "outlet": a.outlet, "Q": a.Q, "bouzidi": a.bouzidi}
        if a.steps:
            kw["steps"] = a.steps
        if a.window:
            kw["window"] = a.window
        print(json.dumps(sphere(**kw)), flush=True)


if __name__ == "__main__":
    main()

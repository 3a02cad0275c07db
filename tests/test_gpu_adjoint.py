"""Discrete adjoint (lbm_adjoint) against the dual-number oracle and central
finite differences.

Gradients are taken at fixed initial pdfs: the dual oracle starts from the same
pdfs with zero tangent, and the finite differences change omega after the
initial state is set.  The adjoint must match the oracle's forward-mode
derivative to 1e-10 relative, and central differences of the GPU FP64 forward
to 1e-5 relative, for the body-force field, omega_c, u_in and the initial pdfs.
"""
import numpy as np
import pytest

from paper_1601_06984_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1601_06984_gb300 import build, lbm as L
    build.build()
    return L


def make(name):
    if name == "uni2d":
        m = W.uniform(2, 4, (16, 16), (0,) * 4)
        return m, 9, 1.6, (0.0, 0.0, 0.0), lambda m: W.tgv_fields(m, 0.02), 5, 2
    if name == "tgv2d":
        m = W.two_level_block(2, 16, 4, 12)
        return m, 9, 1.6, (0.0, 0.0, 0.0), lambda m: W.tgv_fields(m, 0.02), 6, 2
    if name == "half2d":
        m = W.half_refined_2d(16)
        return m, 9, 1.6, (0.0, 0.0, 0.0), lambda m: W.tgv_fields(m, 0.02), 4, 3
    if name == "tgv3d":
        m = W.config_tgv3d(16)
        return m, 19, 1.6, (0.0, 0.0, 0.0), lambda m: W.tgv_fields(m, 0.02), 4, 3
    if name == "sphere":
        m = W.config_sphere_small()
        return (m, 19, W.omega_coarse_from_finest(1.6, 3), (0.04, 0.0, 0.0),
                lambda m: W.uniform_fields(m, 1.0, (0.04, 0.0, 0.0)), 3, 2)
    if name == "schafer20":
        # the paper's cylinder: interpolated bounce-back, parabolic inflow
        m = W.config_cylinder_schafer(20)
        om = W.omega_coarse_from_finest(W.omega_for_re(0.05, 20, 20.0), 2)
        return m, 9, om, (0.05, 0.0, 0.0), lambda m: W.uniform_fields(m, 1.0, (0.05, 0.0)), 3, 2
    if name == "tgv3d_q27":
        m = W.config_tgv3d(16)
        return m, 27, 1.6, (0.0, 0.0, 0.0), lambda m: W.tgv_fields(m, 0.02), 4, 3
    if name == "sphere_q27":
        m = W.config_sphere_small()
        return (m, 27, W.omega_coarse_from_finest(1.6, 3), (0.04, 0.0, 0.0),
                lambda m: W.uniform_fields(m, 1.0, (0.04, 0.0, 0.0)), 3, 2)
    if name in ("channel", "channel_zg"):
        # walled inlet/outlet channel, refined block in the middle; omega near 2
        # on the coarse level exercises the outlet's f^neq rescale
        m = W.nested_boxes(2, 5, (32, 16), [((16, 8), (40, 24))],
                           (W.BC_VELOCITY_IN, W.BC_PRESSURE_OUT, W.BC_WALL, W.BC_WALL))
        return (m, 9, 1.85, (0.05, 0.0, 0.0),
                lambda m: W.uniform_fields(m, 1.0, (0.05, 0.0)), 6, 2)
    raise KeyError(name)


OUTLET = {"channel_zg": 1}
BOUZIDI = {"schafer20": ((40.0, 40.0), 10.0)}  # circle centre and radius, finest cells


def configure(name, m, Q, g, oracles=()):
    """Interpolated bounce-back wall distances of the circle on the GPU context
    and the oracles (same links, same q)."""
    if name not in BOUZIDI:
        return
    e, d = g.obstacle_links()
    q = W.wall_distance_ball(m, e, d, BOUZIDI[name][0], BOUZIDI[name][1], Q)
    g.set_link_q(q)
    for o in oracles:
        o.set_link_q(e, d, q)
    return e, d, q
CASES = [("uni2d", 0, 0), ("tgv2d", 0, 0), ("tgv2d", 1, 0), ("half2d", 0, 0), ("tgv3d", 0, 0), ("tgv3d", 1, 0),
         ("sphere", 0, 0), ("sphere", 1, 0), ("sphere", 0, 1), ("sphere", 1, 3),
         ("channel", 0, 0), ("channel", 1, 0), ("channel_zg", 0, 0),
         ("tgv3d_q27", 0, 0), ("tgv3d_q27", 1, 0), ("sphere_q27", 0, 1),
         ("schafer20", 0, 1), ("schafer20", 1, 0)]


def J_of(red, objective):
    return red[7] if objective == 0 else red[3 + objective]


@pytest.mark.parametrize("tape", [1, 2])
@pytest.mark.parametrize("name,mode,objective", CASES)
def test_adjoint_matches_dual_oracle(lbm, oracle_mod, name, mode, objective, tape):
    m, Q, om, uin, fields, n, K = make(name)
    d = 2 if Q == 9 else 3
    rho, u, S = fields(m)
    F = W.gaussian_force(m, 1e-5)
    out = OUTLET.get(name, 0)
    bz = name in BOUZIDI
    g = lbm.Sim(m, Q, om, time_mode=mode, u_in=uin, use_force=True, outlet=out, bouzidi=bz,
                inlet_profile=1 if bz else 0, adjoint_tape=tape)
    links = configure(name, m, Q, g)
    g.init(rho, u, S, W.pdf_perturbation(m, Q, 1e-5))
    g.set_force(F)
    f0 = g.get_state()
    J, dF, dw, dU, df0 = g.adjoint(n, K, objective, want_f0=True)
    vF = W.random_direction((m.n, d), W.SEED, 21) * 1e-5
    vw = 0.37
    has_uin = bool(np.any(np.asarray(uin) != 0))
    vU = np.array([0.9, -0.4, 0.25 if d == 3 else 0.0]) if has_uin else np.zeros(3)
    vf0 = W.random_direction((m.n, Q), W.SEED, 22) * 1e-4
    parts = {"force": (vF, 0.0, np.zeros(3), None), "omega": (0 * vF, vw, np.zeros(3), None),
             "u_in": (0 * vF, 0.0, vU, None), "f0": (0 * vF, 0.0, np.zeros(3), vf0)}
    for key, (a, b, c, fd0) in parts.items():
        if key == "u_in" and not has_uin:
            continue
        adj = float((dF * a).sum() + dw * b + (dU * c).sum() + (0.0 if fd0 is None else (df0 * fd0).sum()))
        od = oracle_mod.Oracle(m, Q, om, time_mode=mode, u_in=uin, use_force=True, dual=True, omega_dot=b,
                               u_in_dot=tuple(c), outlet=out, inlet_profile=1 if bz else 0)
        if links is not None:
            od.set_link_q(*links)
        od.set_f(f0, fd0)
        od.set_force(F, a)
        od.step(n)
        val, dot = od.reduce()
        # a force component is a cancelling sum of O(|force|) link terms
        J_scale = max(abs(J), abs(val[7]) if objective == 0 else np.abs(val[4:4 + d]).max())
        assert abs(J_of(val, objective) - J) <= 1e-11 * J_scale
        exact = J_of(dot, objective)
        scale = max(abs(exact), 1e-12 * abs(J))
        assert abs(adj - exact) <= 1e-10 * scale, (key, adj, exact, abs(adj - exact) / scale)


@pytest.mark.parametrize("name,mode", [("tgv2d", 0), ("tgv3d", 1), ("sphere", 0), ("channel_zg", 0)])
def test_adjoint_matches_central_differences(lbm, name, mode):
    m, Q, om, uin, fields, n, K = make(name)
    d = 2 if Q == 9 else 3
    rho, u, S = fields(m)
    F = W.gaussian_force(m, 1e-5)
    vF = W.random_direction((m.n, d), W.SEED, 31) * 1e-5
    vw = -0.21
    vU = np.array([0.5, 0.2, -0.3 if d == 3 else 0.0]) if np.any(np.asarray(uin) != 0) else np.zeros(3)
    out = OUTLET.get(name, 0)

    def run(h):
        g = lbm.Sim(m, Q, om, time_mode=mode, u_in=uin, use_force=True, outlet=out)
        g.init(rho, u, S)
        g.set_params(om + h * vw, tuple(np.array(uin) + h * vU))
        g.set_force(F + h * vF)
        g.step(n)
        return g, g.reduce()[7]

    g = lbm.Sim(m, Q, om, time_mode=mode, u_in=uin, use_force=True, outlet=out)
    g.init(rho, u, S)
    g.set_force(F)
    J, dF, dw, dU = g.adjoint(n, K, 0)
    adj = float((dF * vF).sum() + dw * vw + (dU * vU).sum())
    h = 1e-4
    fd = (run(h)[1] - run(-h)[1]) / (2 * h)
    assert abs(adj - fd) <= 1e-5 * abs(fd)


# Reduced-precision adjoints against the FP64 adjoint of the same inputs.  The
# FP32-deviation path rounds every stored pdf and adjoint to FP32 (unit
# roundoff 6e-8) over a handful of steps, so 1e-4 relative leaves a wide
# margin; BF16 storage rounds the stored deviations to 8 significant bits
# (2^-9 = 2e-3 relative) and the gradient inherits errors of that order, so
# 3e-2.  The cases cover both time modes, K not dividing n, and the inlet,
# outlet and obstacle paths of the small sphere.
@pytest.mark.parametrize("prec,tol", [("fp32dev", 1e-4), ("bf16dev", 3e-2)])
@pytest.mark.parametrize("name,mode,objective", [("tgv3d", 0, 0), ("tgv2d", 1, 0), ("sphere", 0, 0), ("sphere", 0, 1)])
def test_adjoint_reduced_precision(lbm, prec, tol, name, mode, objective):
    m, Q, om, uin, fields, n, K = make(name)
    rho, u, S = fields(m)
    F = W.gaussian_force(m, 1e-5)
    res = {}
    for p in ("fp64", prec):
        g = lbm.Sim(m, Q, om, precision={"fp64": lbm.FP64, "fp32dev": lbm.FP32DEV, "bf16dev": lbm.BF16DEV}[p],
                    time_mode=mode, u_in=uin, use_force=True)
        g.init(rho, u, S)
        g.set_force(F)
        res[p] = g.adjoint(n + 1, K, objective)
        g.close()
    (J0, dF0, dw0, dU0), (J1, dF1, dw1, dU1) = res["fp64"], res[prec]
    err = {"J": abs(J1 - J0) / abs(J0),
           "dF": float(np.linalg.norm(dF1 - dF0) / np.linalg.norm(dF0)),
           "dw": abs(dw1 - dw0) / abs(dw0)}
    if np.any(np.asarray(uin) != 0):
        # the drag of the small sphere after a few steps does not depend on u_in yet
        err["dU"] = float(np.linalg.norm(dU1 - dU0) / max(np.linalg.norm(dU0), 1e-12 * abs(J0)))
    assert all(v <= tol for v in err.values()), err


@pytest.mark.parametrize("name,mode,objective,K", [("sphere", 0, 1, 2), ("tgv3d", 1, 0, 3), ("channel_zg", 0, 0, 4)])
def test_adjoint_tape_schemes_agree_bitwise(lbm, name, mode, objective, K):
    """Recording every step of a segment in one recompute (adjoint_tape 1) and
    recomputing each step once more to record it (2) feed the same reverse
    kernels the same states in the same order: bit-identical gradients, with
    K not dividing n."""
    m, Q, om, uin, fields, n, _ = make(name)
    rho, u, S = fields(m)
    F = W.gaussian_force(m, 1e-5)
    out = []
    for tape in (1, 2):
        g = lbm.Sim(m, Q, om, time_mode=mode, u_in=uin, use_force=True, outlet=OUTLET.get(name, 0),
                    adjoint_tape=tape)
        g.init(rho, u, S, W.pdf_perturbation(m, Q, 1e-5))
        g.set_force(F)
        out.append(g.adjoint(n + 1, K, objective, want_f0=True) + (g.get_state(),))
    (J1, dF1, dw1, dU1, f1, s1), (J2, dF2, dw2, dU2, f2, s2) = out
    assert J1 == J2 and dw1 == dw2
    assert np.array_equal(dF1, dF2) and np.array_equal(dU1, dU2) and np.array_equal(f1, f2)
    assert np.array_equal(s1, s2)


def test_adjoint_leaves_final_state_and_is_deterministic(lbm):
    m, Q, om, uin, fields, n, K = make("sphere")
    rho, u, S = fields(m)
    out = []
    for _ in range(2):
        g = lbm.Sim(m, Q, om, u_in=uin, use_force=True)
        g.init(rho, u, S)
        g.set_force(W.gaussian_force(m, 1e-5))
        res = g.adjoint(n, K, 1)
        out.append((res, g.get_state()))
    ref = lbm.Sim(m, Q, om, u_in=uin, use_force=True)
    ref.init(rho, u, S)
    ref.set_force(W.gaussian_force(m, 1e-5))
    ref.step(n)
    assert np.array_equal(out[0][1], ref.get_state())
    assert out[0][0][0] == out[1][0][0] and out[0][0][2] == out[1][0][2]
    assert np.array_equal(out[0][0][1], out[1][0][1])


def test_autograd_function(lbm):
    import torch
    from paper_1601_06984_gb300.autograd import objective
    m, Q, om, uin, fields, n, K = make("tgv3d")
    g = lbm.Sim(m, Q, om, u_in=uin, use_force=True)
    init = (*fields(m), None)
    F = torch.tensor(W.gaussian_force(m, 1e-5), requires_grad=True)
    w = torch.tensor(om, dtype=torch.float64, requires_grad=True)
    U = torch.zeros(3, dtype=torch.float64, requires_grad=True)
    J = objective(F, w, U, g, init, n, K, 0)
    J.backward()
    with torch.no_grad():
        h = 1e-4
        vF = torch.tensor(W.random_direction((m.n, 3), W.SEED, 41) * 1e-5)
        Jp = objective(F + h * vF, w, U, g, init, n, K, 0)
        Jm = objective(F - h * vF, w, U, g, init, n, K, 0)
    fd = float((Jp - Jm) / (2 * h))
    assert abs(float((F.grad * vF).sum()) - fd) <= 1e-5 * abs(fd)
    assert w.grad is not None and torch.isfinite(w.grad)


def test_adjoint_full_size_tgv3d_64(lbm):
    """Two-level Taylor-Green mesh at full size: periodic 64^3 coarse with the
    central 32^3 block refined, Gaussian body force N(0, 1e-6), 400 coarse
    steps, kinetic energy, checkpoints every 20 steps (FP64): the gradient
    along a random force direction and along omega matches central
    differences."""
    m = W.config_tgv3d(64)
    rho, u, S = W.uniform_fields(m)
    F = W.gaussian_force(m, 1e-6)
    vF = W.random_direction((m.n, 3), W.SEED, 51) * 1e-6
    vw = 0.1

    def run(h):
        g = lbm.Sim(m, 19, 1.6, use_force=True)
        g.init(rho, u, S)
        g.set_params(1.6 + h * vw)
        g.set_force(F + h * vF)
        g.step(400)
        return g.reduce()[7]

    g = lbm.Sim(m, 19, 1.6, use_force=True)
    g.init(rho, u, S)
    g.set_force(F)
    J, dF, dw, _ = g.adjoint(400, 20, 0)
    assert J > 0
    adj = float((dF * vF).sum() + dw * vw)
    h = 1e-3
    fd = (run(h) - run(-h)) / (2 * h)
    assert abs(adj - fd) <= 1e-5 * abs(fd)


@pytest.mark.parametrize("outlet", [0, 1])
def test_adjoint_cylinder_drag(lbm, outlet):
    """Drag objective on the full 4-level cylinder channel (about 64k elements,
    coarsest omega 1.86 at Re = 20) with the Sec. 2.3 outlet: the adjoint's
    derivative of c_D-proportional F_x along (omega_c, u_in) matches central
    differences of the FP64 forward."""
    m = W.config_cylinder()
    U = 0.05
    om = W.omega_coarse_from_finest(W.omega_for_re(U, 40, 20.0), 4)
    rho, u, S = W.uniform_fields(m, 1.0, (U, 0.0))
    df = W.pdf_perturbation(m, 9, 1e-5)
    n, K = 20, 5
    vw, vU = 0.05, np.array([0.3, 0.1, 0.0])

    def run(h):
        g = lbm.Sim(m, 9, om, u_in=(U, 0.0, 0.0), outlet=outlet)
        g.init(rho, u, S, df)
        g.set_params(om + h * vw, tuple(np.array([U, 0.0, 0.0]) + h * vU))
        g.step(n)
        return g.reduce()[4]

    g = lbm.Sim(m, 9, om, u_in=(U, 0.0, 0.0), outlet=outlet)
    g.init(rho, u, S, df)
    J, _, dw, dU = g.adjoint(n, K, 1, want_force=False)
    assert abs(J - run(0.0)) <= 1e-12 * abs(J)
    adj = dw * vw + float((dU * vU).sum())
    h = 1e-4
    fd = (run(h) - run(-h)) / (2 * h)
    assert abs(adj - fd) <= 1e-6 * abs(fd), (adj, fd)

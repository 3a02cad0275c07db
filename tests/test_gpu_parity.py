"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

FP64 must match the oracle to 1e-11 relative max-norm on the post-collision
pdfs and on the moments, element by element, on meshes that span several
levels, ghost layers, boundaries and forces, in all three time-coupling modes.
"""
import math

import numpy as np
import pytest

from paper_1601_06984_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.fixture(scope="module")
def lbm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1601_06984_gb300 import build, lbm as L
    build.build()
    return L


def rel(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / (scale if scale > 0 else 1.0)


def make_case(name):
    """mesh, stencil, omega_c, u_in, fields(mesh) -> (rho, u, S, df), force or None, steps"""
    if name == "tgv2d":
        m = W.config_tgv2d()
        return m, 9, 1.6, (0, 0, 0), lambda m: (*W.tgv_fields(m, 0.01), W.pdf_perturbation(m, 9)), None, 50
    if name == "tgv2d_half":
        m = W.half_refined_2d(16)
        return m, 9, 1.6, (0, 0, 0), lambda m: (*W.tgv_fields(m, 0.02), W.pdf_perturbation(m, 9)), None, 20
    if name == "tgv3d":
        m = W.config_tgv3d(16)
        return m, 19, 1.6, (0, 0, 0), lambda m: (*W.tgv_fields(m, 0.01), W.pdf_perturbation(m, 19)), None, 8
    if name == "tgv3d_force":
        m = W.config_tgv3d(16)
        return (m, 19, 1.6, (0, 0, 0), lambda m: (*W.tgv_fields(m, 0.01), None),
                W.gaussian_force(m, 1e-5), 6)
    if name == "cylinder":
        m = W.config_cylinder()
        om = W.omega_coarse_from_finest(W.omega_for_re(0.05, 40, 20), 4)
        return (m, 9, om, (0.05, 0, 0),
                lambda m: (*W.uniform_fields(m, 1.0, (0.05, 0.0)), W.pdf_perturbation(m, 9, 1e-4)), None, 2)
    if name == "tgv3d_q27":
        m = W.config_tgv3d(16)
        return m, 27, 1.6, (0, 0, 0), lambda m: (*W.tgv_fields(m, 0.01), W.pdf_perturbation(m, 27)), None, 8
    if name == "tgv3d_force_q27":
        m = W.config_tgv3d(16)
        return (m, 27, 1.6, (0, 0, 0), lambda m: (*W.tgv_fields(m, 0.01), None),
                W.gaussian_force(m, 1e-5), 6)
    if name == "sphere_small_q27":
        m = W.config_sphere_small()
        om = W.omega_coarse_from_finest(1.6, 3)
        return (m, 27, om, (0.04, 0, 0),
                lambda m: (*W.uniform_fields(m, 1.0, (0.04, 0.0, 0.0)), W.pdf_perturbation(m, 27, 1e-4)), None, 3)
    if name == "schafer20":
        m = W.config_cylinder_schafer(20)
        om = W.omega_coarse_from_finest(W.omega_for_re(0.05, 20, 20.0), 2)
        return (m, 9, om, (0.05, 0, 0),
                lambda m: (*W.uniform_fields(m, 1.0, (0.05, 0.0)), W.pdf_perturbation(m, 9, 1e-4)), None, 4)
    if name == "channel_zg":
        m = W.nested_boxes(2, 5, (32, 16), [((16, 8), (40, 24))],
                           (W.BC_VELOCITY_IN, W.BC_PRESSURE_OUT, W.BC_WALL, W.BC_WALL))
        return (m, 9, 1.85, (0.05, 0, 0),
                lambda m: (*W.uniform_fields(m, 1.0, (0.05, 0.0)), W.pdf_perturbation(m, 9, 1e-4)), None, 40)
    if name == "sphere_small":
        m = W.config_sphere_small()
        om = W.omega_coarse_from_finest(1.6, 3)
        return (m, 19, om, (0.04, 0, 0),
                lambda m: (*W.uniform_fields(m, 1.0, (0.04, 0.0, 0.0)), W.pdf_perturbation(m, 19, 1e-4)), None, 3)
    if name == "sphere5":
        # five levels, four interfaces: the recursion depth of the sphere
        # workload (coarsest omega 1.969 for omega_f = 1.6, as near 2 as there)
        m = W.config_sphere_5level_small()
        om = W.omega_coarse_from_finest(1.6, 5)
        return (m, 19, om, (0.04, 0, 0),
                lambda m: (*W.uniform_fields(m, 1.0, (0.04, 0.0, 0.0)), W.pdf_perturbation(m, 19, 1e-4)), None, 4)
    raise KeyError(name)


OUTLET = {"channel_zg": 1, "sphere5": 1}  # zero-gradient outlet extrapolation
# the paper's cylinder: interpolated bounce-back with the wall distances of the
# circle, parabolic inflow
BOUZIDI = {"schafer20": (20, (40.0, 40.0), 10.0)}


def case_fields(m, fields, mode):
    """The case's fields, converted to each level's lattice units in the
    diffusive mode (the generators give coarsest-level velocities)."""
    rho, u, S, df = fields(m)
    if mode == 2:
        rho, u, S = W.diffusive_units(m, rho, u, S)
    return rho, u, S, df


def run_both(lbm, oracle_mod, name, mode, precision=0):
    m, Q, om, uin, fields, force, steps = make_case(name)
    rho, u, S, df = case_fields(m, fields, mode)
    out = OUTLET.get(name, 0)
    bz = BOUZIDI.get(name)
    o = oracle_mod.Oracle(m, Q, om, time_mode=mode, u_in=uin, use_force=force is not None, outlet=out,
                          inlet_profile=1 if bz else 0)
    o.init(rho, u, S, df)
    g = lbm.Sim(m, Q, om, precision=precision, time_mode=mode, u_in=uin, use_force=force is not None,
                outlet=out, inlet_profile=1 if bz else 0, bouzidi=bz is not None)
    if bz:
        e, d = g.obstacle_links()
        q = W.wall_distance_ball(m, e, d, bz[1], bz[2], Q)
        g.set_link_q(q)
        o.set_link_q(e, d, q)
    g.init(rho, u, S, df)
    if force is not None:
        o.set_force(force)
        g.set_force(force)
    o.step(steps)
    g.step(steps)
    return m, o, g


CASES = ["tgv2d", "tgv2d_half", "tgv3d", "tgv3d_force", "cylinder", "channel_zg", "sphere_small",
         "tgv3d_q27", "tgv3d_force_q27", "sphere_small_q27", "schafer20", "sphere5"]


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_fp64_matches_oracle(lbm, oracle_mod, name, mode):
    m, o, g = run_both(lbm, oracle_mod, name, mode)
    assert rel(g.get_state(), o.get_f()) < TOL
    r_o, u_o, S_o = o.moments()
    r_g, u_g, S_g = g.moments()
    assert rel(r_g, r_o) < TOL
    assert rel(u_g, u_o) < TOL
    assert rel(S_g, S_o) < 1e-10
    red_o, red_g = o.reduce(), g.reduce()
    assert abs(red_g[0] - red_o[0]) / red_o[0] < TOL
    mom_scale = max(np.abs(red_o[1:4]).max(), 1e-300)
    assert np.abs(red_g[1:4] - red_o[1:4]).max() / max(mom_scale, red_o[0] * 1e-6) < 1e-9
    assert abs(red_g[7] - red_o[7]) / max(red_o[7], 1e-300) < 1e-10
    if np.abs(red_o[4:7]).max() > 0:
        assert np.abs(red_g[4:7] - red_o[4:7]).max() / np.abs(red_o[4:7]).max() < 1e-10


@pytest.mark.parametrize("name", ["tgv2d", "tgv3d", "sphere_small", "tgv3d_q27", "sphere5"])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_ghost_fill_matches_oracle(lbm, oracle_mod, name, mode):
    """GhostFromFiner and GhostFromCoarser values after one synchronous fill
    (in the diffusive mode four GhostFromCoarser layers, with the unit
    conversions of both fills)."""
    m, Q, om, uin, fields, force, _ = make_case(name)
    rho, u, S, df = case_fields(m, fields, mode)
    o = oracle_mod.Oracle(m, Q, om, time_mode=mode, u_in=uin)
    g = lbm.Sim(m, Q, om, time_mode=mode, u_in=uin)
    o.init(rho, u, S, df)
    g.init(rho, u, S, df)
    o.fill_ghosts()
    g.fill_ghosts()
    io, fo = o.ghosts()
    ig, fg = g.ghosts()
    assert len(io) == len(ig) > 0
    key = lambda info: {(int(r[0]), int(r[1]), int(r[3]), int(r[4]), int(r[5])): k for k, r in enumerate(info)}
    ko, kg = key(io), key(ig)
    assert ko.keys() == kg.keys()
    idx_o = np.array([ko[k] for k in ko])
    idx_g = np.array([kg[k] for k in ko])
    assert rel(fg[idx_g], fo[idx_o]) < 1e-12
    # layers agree too
    assert np.array_equal(ig[idx_g, 2], io[idx_o, 2])


@pytest.mark.parametrize("precision", [0, 1])
def test_sphere5_levels_and_reduced_precision(lbm, oracle_mod, precision):
    """The five-level sphere case per level: every level's elements against the
    oracle after four coarse steps (64 finest substeps), FP64 at 1e-11 and
    FP32-deviation storage within its rounding (1e-5 of the pdfs' scale)."""
    m, o, g = run_both(lbm, oracle_mod, "sphere5", 0, precision)
    info = g.mesh_info()
    assert len(info) == 5 and (info[:, 1] > 0).all()
    fo, fg = o.get_f(), g.get_state()
    for L in np.unique(m.levels):
        sel = m.levels == L
        assert rel(fg[sel], fo[sel]) < (TOL if precision == 0 else 1e-5), L


def test_fp64_full_size_tgv3d(lbm, oracle_mod):
    """The 64^3 / 32^3-block D3Q19 mesh at full size (about 0.5M elements),
    two coarse steps, every element against the oracle."""
    m = W.config_tgv3d(64)
    rho, u, S = W.tgv_fields(m, 0.01)
    df = W.pdf_perturbation(m, 19)
    o = oracle_mod.Oracle(m, 19, 1.6)
    o.init(rho, u, S, df)
    o.step(2)
    g = lbm.Sim(m, 19, 1.6)
    g.init(rho, u, S, df)
    g.step(2)
    assert rel(g.get_state(), o.get_f()) < TOL


def test_shuffled_user_order_is_bitwise_identical(lbm):
    m = W.config_tgv3d(16)
    sh = W.shuffled(m)
    res = []
    for mesh in (m, sh):
        g = lbm.Sim(mesh, 19, 1.6)
        rho, u, S = W.tgv_fields(mesh, 0.01)
        g.init(rho, u, S, W.pdf_perturbation(mesh, 19))
        g.step(4)
        key = np.argsort(mesh.tree_ids)
        res.append(g.get_state()[key])
    assert np.array_equal(res[0], res[1])


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_deterministic(lbm, precision):
    """No atomics on the forward path: two identical runs give identical bits,
    reductions included."""
    m = W.config_sphere_small()
    om = W.omega_coarse_from_finest(1.6, 3)
    out = []
    for _ in range(2):
        g = lbm.Sim(m, 19, om, precision=precision, u_in=(0.04, 0, 0))
        g.init(*W.uniform_fields(m, 1.0, (0.04, 0, 0)), W.pdf_perturbation(m, 19, 1e-4))
        g.step(3)
        out.append((g.get_state(), g.reduce()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_precision_variants_error(lbm, oracle_mod, mode):
    """FP32-deviation and BF16-deviation storage against the FP64 oracle on the
    2D two-level Taylor-Green (200 coarse steps, u0 = 0.01): velocity l2 error
    and mass drift stay within the stated bounds."""
    m = W.config_tgv2d()
    rho, u, S = W.tgv_fields(m, 0.01)
    if mode == 2:
        rho, u, S = W.diffusive_units(m, rho, u, S)
    o = oracle_mod.Oracle(m, 9, 1.6, time_mode=mode)
    o.init(rho, u, S)
    o.step(200)
    _, u_o, S_o = o.moments()
    bounds = {1: 1e-4, 2: 5e-2}
    for prec, bound in bounds.items():
        g = lbm.Sim(m, 9, 1.6, precision=prec, time_mode=mode)
        g.init(rho, u, S)
        g.step(200)
        _, u_g, _ = g.moments()
        err = math.sqrt(((u_g - u_o) ** 2).sum() / (u_o ** 2).sum())
        assert err < bound, (prec, err)


def test_kernel_launches_counted(lbm):
    m = W.config_tgv2d()
    g = lbm.Sim(m, 9, 1.6)
    g.init(*W.tgv_fields(m, 0.01))
    info = g.mesh_info()
    assert info[0, 8] == 0 and info[1, 8] == 4    # interior bricks: none coarse, 4 fine
    assert info[0, 9] == 12 and info[1, 9] == 12  # boundary bricks: all other complete bricks
    n0 = g.kernel_launches()
    g.step(1)
    # LINEAR two-level step: GFF, source moments, GFC, coarse stream-collide
    # (boundary bricks + neighbour list for the inner GFF layer), fine
    # stream-collide (interior + boundary bricks), source moments, GFC, fine
    # stream-collide (interior + boundary bricks)
    assert g.kernel_launches() - n0 == 11


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpoint_restart(lbm, precision):
    """lbm_get_state / lbm_set_state: a run interrupted after 3 steps and
    restarted from the saved state into a fresh context reproduces the
    uninterrupted run (bitwise in FP64; FP32 within the storage rounding of
    one round trip)."""
    m, Q, om, uin, fields, force, _ = make_case("sphere_small")
    rho, u, S, df = fields(m)
    a = lbm.Sim(m, Q, om, precision=precision, u_in=uin)
    a.init(rho, u, S, df)
    a.step(3)
    saved = a.get_state()
    a.step(2)
    b = lbm.Sim(m, Q, om, precision=precision, u_in=uin)
    b.set_state(saved)
    b.step(2)
    if precision == 0:
        assert np.array_equal(a.get_state(), b.get_state())
    else:
        assert rel(b.get_state(), a.get_state()) < 1e-6


@pytest.mark.parametrize("precision,mode", [(0, 0), (1, 1), (2, 0), (1, 2)])
def test_graph_steps_match_eager_steps(lbm, precision, mode):
    """lbm_step replays captured graphs (two-step graphs for pairs of steps, a
    one-step graph for a remaining step); in timing mode 1 every step is
    launched kernel by kernel.  Same kernels, same order: bitwise equal states
    and equal launch counts, from either parity state, and after set_params
    (which must drop the captured steps)."""
    m = W.config_tgv3d(16)
    rho, u, S = W.tgv_fields(m, 0.01)
    df = W.pdf_perturbation(m, 19)
    a = lbm.Sim(m, 19, 1.6, precision=precision, time_mode=mode)
    b = lbm.Sim(m, 19, 1.6, precision=precision, time_mode=mode)
    for s_ in (a, b):
        s_.init(rho, u, S, df)
    b.timing_enable(1)  # kernel by kernel
    na, nb = a.kernel_launches(), b.kernel_launches()
    a.step(1)       # one-step graph from the even parity state
    a.step(5)       # two-step graphs from the odd parity state, then a one-step graph
    a.step(4)       # two-step graphs from the even parity state
    for _ in range(10):
        b.step(1)
    assert np.array_equal(a.get_state(), b.get_state())
    assert a.kernel_launches() - na == b.kernel_launches() - nb
    for s_ in (a, b):
        s_.set_params(1.5)
    a.step(4)
    for _ in range(4):
        b.step(1)
    assert np.array_equal(a.get_state(), b.get_state())


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_records_follow_state_changes(lbm, mode):
    """The stream-collide keeps the GhostFromCoarser source records of the
    state it writes; anything else that changes the state, the force or the
    relaxation rates must make the next step rebuild them.  A context that has
    been stepping (records current) and then takes lbm_set_state,
    lbm_set_force or lbm_set_params continues bit for bit like a fresh context
    given the same state and parameters, through the eager and the graph path
    (FP64, whose state round trip is exact)."""
    precision = 0
    m = W.config_tgv3d(16)
    rho, u, S = W.tgv_fields(m, 0.01)
    df = W.pdf_perturbation(m, 19)
    F1, F2 = W.gaussian_force(m, 1e-5), 2.0 * W.gaussian_force(m, 1e-5)

    def sim(om=1.6):
        s_ = lbm.Sim(m, 19, om, precision=precision, time_mode=mode, use_force=True)
        s_.set_force(F1)
        return s_

    a = sim()
    a.init(rho, u, S, df)
    a.step(3)
    other = sim()
    other.init(rho, -u, S, df)
    other.step(2)
    y = other.get_state()
    # a new state
    a.set_state(y)
    a.step(1)
    a.step(2)
    b = sim()
    b.set_state(y)
    b.step(1)
    b.step(2)
    assert np.array_equal(a.get_state(), b.get_state())
    # a new force
    x = a.get_state()
    a.set_force(F2)
    a.step(2)
    a.step(1)
    c = sim()
    c.set_state(x)
    c.set_force(F2)
    c.step(2)
    c.step(1)
    assert np.array_equal(a.get_state(), c.get_state())
    # new relaxation rates
    x = a.get_state()
    a.set_params(1.5)
    a.step(2)
    d = sim(1.5)
    d.set_state(x)
    d.set_force(F2)
    d.step(2)
    assert np.array_equal(a.get_state(), d.get_state())


@pytest.mark.parametrize("precision", [1, 2])
def test_q27_reduced_precision_tracks_fp64(lbm, oracle_mod, precision):
    """D3Q27 with FP32 / BF16 deviation storage on the two-level 16^3 Taylor-Green
    (40 coarse steps) stays within the same bounds as D2Q9 / D3Q19 against the
    FP64 oracle: velocity l2 1e-4 (FP32) and 5e-2 (BF16)."""
    m = W.config_tgv3d(16)
    rho, u, S = W.tgv_fields(m, 0.01)
    o = oracle_mod.Oracle(m, 27, 1.6)
    o.init(rho, u, S)
    o.step(40)
    _, u_o, _ = o.moments()
    g = lbm.Sim(m, 27, 1.6, precision=precision)
    g.init(rho, u, S)
    g.step(40)
    _, u_g, _ = g.moments()
    err = math.sqrt(((u_g - u_o) ** 2).sum() / (u_o ** 2).sum())
    assert err < {1: 1e-4, 2: 5e-2}[precision], err


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_empty_refined_region_is_identity(lbm, oracle_mod, d, mode):
    """Sec. 2.2 recursive stepping with nothing to couple: one more declared
    level without elements (an empty refined region) leaves the FP64 result of
    lbm_step bit for bit equal to the run without it, through the captured
    graphs and kernel by kernel alike, and equal to the oracle run with the
    same declared levels to 1e-11.  Single-level periodic Taylor-Green (the
    two-level code path against the plain single-level one) and the two-level
    one with a third, empty level."""
    if d == 2:
        meshes = ((W.uniform(2, 5, (32, 32), (0,) * 4), 1), (W.config_tgv2d(), 2))
        Q = 9
    else:
        meshes = ((W.uniform(3, 4, (16, 16, 16), (0,) * 6), 1), (W.config_tgv3d(16), 2))
        Q = 19
    for mesh, nl in meshes:
        rho, u, S = W.tgv_fields(mesh, 0.02)
        df = W.pdf_perturbation(mesh, Q, 1e-6)
        res = []
        for n_levels in (0, nl + 1):
            g = lbm.Sim(mesh, Q, 1.8, time_mode=mode, n_levels=n_levels)
            assert len(g.mesh_info()) == (nl if n_levels == 0 else nl + 1)
            g.init(rho, u, S, df)
            g.step(6)       # three captured two-step graphs
            g.step(1)       # one step kernel by kernel
            res.append((g.get_state(), g.reduce(), g.moments()))
        (f0, r0, m0), (f1, r1, m1) = res
        assert np.array_equal(f0, f1)
        assert np.array_equal(r0, r1)
        assert all(np.array_equal(a, b) for a, b in zip(m0, m1))
        o = oracle_mod.Oracle(mesh, Q, 1.8, time_mode=mode, n_levels=nl + 1)
        o.init(rho, u, S, df)
        o.step(7)
        assert rel(f1, o.get_f()) < TOL


def test_mass_check_stops_on_non_finite_input(lbm):
    """params.check_every: a NaN planted on the host in one element's initial
    density (a host-side fault; nothing faults on the GPU) makes lbm_step
    return LBM_ERR_NUMERIC at its first check, and the context stays usable:
    a clean state restored with lbm_set_state steps on normally."""
    m = W.config_tgv2d()
    rho, u, S = W.tgv_fields(m, 0.01)
    bad = rho.copy()
    bad[123] = np.nan
    g = lbm.Sim(m, 9, 1.6, check_every=4)
    g.init(bad, u, S)
    with pytest.raises(lbm.LBMError, match="not finite") as ei:
        g.step(10)
    assert ei.value.status == -6
    clean = lbm.Sim(m, 9, 1.6)
    clean.init(rho, u, S)
    g.set_state(clean.get_state())
    g.step(8)
    clean.step(8)
    assert np.array_equal(g.get_state(), clean.get_state())


def test_mass_check_catches_a_blow_up_and_a_band(lbm):
    """A run that diverges on its own (omega_c = 1.99 with u0 = 0.5 and a 1e-3
    pdf perturbation, far outside the stable range; the oracle overflows after
    about 500 steps) trips the finiteness check at a multiple of check_every;
    a mass band trips on an open channel whose mass changes (by 1.5% in its
    first 10 steps), and only when the band is tighter than that."""
    m = W.uniform(2, 5, (32, 32), (0,) * 4)
    g = lbm.Sim(m, 9, 1.99, check_every=25)
    g.init(*W.tgv_fields(m, 0.5), W.pdf_perturbation(m, 9, 1e-3))
    with pytest.raises(lbm.LBMError, match=r"after (\d+) coarse steps") as ei:
        g.step(5000)
    assert ei.value.status == -6
    k = int(__import__("re").search(r"after (\d+) coarse", str(ei.value)).group(1))
    assert k % 25 == 0 and k > 0
    ch = W.nested_boxes(2, 5, (32, 16), [((16, 8), (40, 24))],
                        (W.BC_VELOCITY_IN, W.BC_PRESSURE_OUT, W.BC_WALL, W.BC_WALL))
    fields = W.uniform_fields(ch, 1.0, (0.0, 0.0))
    tight = lbm.Sim(ch, 9, 1.85, u_in=(0.05, 0, 0), outlet=1, check_every=10, mass_band=1e-9)
    tight.init(*fields)
    with pytest.raises(lbm.LBMError, match="outside"):
        tight.step(100)
    loose = lbm.Sim(ch, 9, 1.85, u_in=(0.05, 0, 0), outlet=1, check_every=10, mass_band=0.5)
    loose.init(*fields)
    loose.step(100)


@pytest.mark.parametrize("precision", [0, 1])
def test_mass_check_leaves_clean_runs_unchanged(lbm, precision):
    """With the check on, a clean run takes the same steps in the same order:
    its state is bit for bit that of the run without the check, whatever the
    split of the steps over lbm_step calls."""
    m, Q, om, uin, fields, _, _ = make_case("sphere_small")
    rho, u, S, df = fields(m)
    res = []
    for check, calls in ((0, (7,)), (3, (4, 3)), (2, (1, 1, 5))):
        g = lbm.Sim(m, Q, om, precision=precision, u_in=uin, check_every=check, mass_band=1e-2 if check else 0.0)
        g.init(rho, u, S, df)
        for n in calls:
            g.step(n)
        res.append(g.get_state())
    assert np.array_equal(res[0], res[1]) and np.array_equal(res[0], res[2])


def test_diffusive_mode_has_no_adjoint(lbm):
    """The adjoint covers the acoustic-scaling modes only; in the diffusive
    mode both adjoint calls fail with LBM_ERR_STATE and leave the context usable."""
    m = W.config_tgv2d()
    g = lbm.Sim(m, 9, 1.6, time_mode=2)
    g.init(*W.diffusive_units(m, *W.tgv_fields(m, 0.01)))
    with pytest.raises(lbm.LBMError) as ex:
        g.adjoint_bytes(2, 1)
    assert ex.value.status == -5
    g.step(1)
    assert np.isfinite(g.get_state()).all()


def test_diffusive_tgv_converges_at_second_order(lbm):
    """Taylor-Green vortex on the half-refined square in the diffusive mode
    (u0 ~ 1/N at fixed omega), through the C ABI in FP64 at N = 32..512: at
    t_D / 4 the strain-rate error in coarsest-level units falls at second
    order (local slopes in [1.8, 2.2]; 1.94, 1.97, 1.99, 1.99), and so does the
    velocity error (slopes at least 1.8, the last at most 2.2; 2.53, 2.28,
    2.14, 2.08).  Without the separate factor for f^neq's odd part the
    velocity error levels off near 2e-6 from N = 256 on (slopes 1.03, 0.72)."""
    from conv_fit import local_slopes
    res = (32, 64, 128, 256, 512)
    eu, eS = [], []
    for N in res:
        mesh = W.half_refined_2d(N)
        omega = 1.6
        nu = (1 / omega - 0.5) / 3
        k = 2 * math.pi / N
        steps = int(round(0.25 / (2 * nu * k * k)))
        u0 = 0.0025 * 16 / N
        g = lbm.Sim(mesh, 9, omega, time_mode=2)
        g.init(*W.diffusive_units(mesh, *W.tgv_fields(mesh, u0)))
        g.step(steps)
        _, u1, S1 = g.moments()
        _, ua, Sa = W.diffusive_units(mesh, *W.tgv_fields(mesh, u0, t=steps, nu=nu))
        l = mesh.levels.astype(np.int64) - mesh.lmin
        su, sS = np.ldexp(1.0, l), np.ldexp(1.0, 2 * l)
        eu.append(math.sqrt((((u1[:, 0] - ua[:, 0]) * su) ** 2).sum() / ((ua[:, 0] * su) ** 2).sum()))
        eS.append(math.sqrt((((S1[:, 0] - Sa[:, 0]) * sS) ** 2).sum() / ((Sa[:, 0] * sS) ** 2).sum()))
        g.close()
    slS, slu = local_slopes(res, np.array(eS)), local_slopes(res, np.array(eu))
    assert np.all((slS >= 1.8) & (slS <= 2.2)), (slS, eS)
    assert np.all(slu >= 1.8) and slu[-1] <= 2.2, (slu, eu)

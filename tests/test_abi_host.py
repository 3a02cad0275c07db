"""Host-side checks of the C ABI (no GPU): the library loads and exports every
entry point declared in include/lbm.h, the host mesh builder agrees with the
oracle's own mesh code on ghost counts and on rejected meshes, and the
z-curve / weight utility reproduces the paper's worked example."""
import itertools
import json
import os
import re

import numpy as np
import pytest

from paper_1601_06984_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lbm():
    from paper_1601_06984_gb300 import build, lbm as L
    build.build()
    return L


def test_exports_every_declared_symbol(lbm):
    header = open(os.path.join(ROOT, "include", "lbm.h")).read()
    declared = set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", header))
    declared.discard("lbm_params")
    lib = lbm.lib()
    missing = [s for s in sorted(declared) if not hasattr(lib, s)]
    assert not missing, missing
    assert declared == set(lbm.EXPORTS)


MESHES = [
    ("tgv2d", W.config_tgv2d, 9, 1.6),
    ("tgv3d", lambda: W.config_tgv3d(16), 19, 1.6),
    ("tgv3d_q27", lambda: W.config_tgv3d(16), 27, 1.6),
    ("sphere_q27", W.config_sphere_small, 27, 1.7),
    ("half", lambda: W.half_refined_2d(16), 9, 1.6),
    ("cylinder", W.config_cylinder, 9, 1.8605),
]


@pytest.mark.parametrize("name,make,Q,omega", MESHES)
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_mesh_counts_match_oracle(lbm, oracle_mod, name, make, Q, omega, mode):
    """Level-wise fluid / GhostFromCoarser / GhostFromFiner counts of the
    library's builder equal those of the oracle's independent mesh code."""
    mesh = make()
    s = lbm.Sim(mesh, Q, omega, time_mode=mode, device=None)
    info = s.mesh_info()
    oc = oracle_mod.Oracle(mesh, Q, omega, time_mode=mode).counts()
    assert len(info) == len(oc)
    for a, b in zip(info, oc):
        assert a[0] == b[0]
        assert a[1] == b[1]              # fluid
        assert a[2] == b[2]              # GFC
        assert a[3] + a[4] == b[3]       # GFF
        assert a[3] == b[5]              # inner GFF layer
    assert s.ghost_count() == int(oc[:, 2].sum() + oc[:, 3].sum())


def test_tgv2d_two_level_counts(lbm):
    """Two-level 32x32 mesh with a refined 16x16 block: 768 coarse and 1024 fine fluid elements, 272 fine
    GhostFromCoarser, 60 coarse GhostFromFiner (112 with the second layer)."""
    mesh = W.config_tgv2d()
    lin = lbm.Sim(mesh, 9, 1.6, time_mode=0, device=None).mesh_info()
    two = lbm.Sim(mesh, 9, 1.6, time_mode=1, device=None).mesh_info()
    assert lin[0, 1] == 768 and lin[1, 1] == 1024 and lin[1, 2] == 272
    assert two[0, 3] + two[0, 4] == 60 and lin[0, 3] + lin[0, 4] == 112


def _bad_meshes():
    good = W.config_tgv2d()
    dup = W.Mesh(2, good.extent, good.bc, np.concatenate([good.tree_ids, good.tree_ids[:1]]),
                 np.concatenate([good.levels, good.levels[:1]]), np.concatenate([good.coords, good.coords[:1]]),
                 good.lmin)
    fine = good.levels > good.lmin
    parent = good.coords[fine][0] // 2
    ov = W.Mesh(2, good.extent, good.bc, np.concatenate([good.tree_ids, W.tree_ids(parent[None], good.lmin, 2)]),
                np.concatenate([good.levels, [good.lmin]]).astype(np.int8),
                np.concatenate([good.coords, parent[None]]), good.lmin)
    jump = W.nested_boxes(2, 5, (32, 32), [((16, 16), (48, 48)), ((48, 48), (80, 80))], (0,) * 4)
    far = W.Mesh(2, (4, 4), (0,) * 4, W.tree_ids(np.array([[5, 5]]), 3, 2), np.array([3], np.int8),
                 np.array([[5, 5]]), 3)
    return [("duplicate", dup), ("overlap", ov), ("level jump", jump), ("outside", far)]


@pytest.mark.parametrize("name,mesh", _bad_meshes())
def test_invalid_meshes_rejected_like_the_oracle(lbm, oracle_mod, name, mesh):
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.Oracle(mesh, 9, 1.6)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.Sim(mesh, 9, 1.6, device=None)
    assert ei.value.status in (-1, -2)


def test_level_list_must_match_tree_ids(lbm):
    mesh = W.config_tgv2d()
    lv = mesh.levels.copy()
    lv[0] += 1
    bad = W.Mesh(2, mesh.extent, mesh.bc, mesh.tree_ids, lv, mesh.coords, mesh.lmin)
    with pytest.raises(lbm.LBMError, match="level"):
        lbm.Sim(bad, 9, 1.6, device=None)


def test_bad_arguments(lbm):
    mesh = W.config_tgv2d()
    with pytest.raises(lbm.LBMError):
        lbm.Sim(mesh, 9, 2.5, device=None)          # omega outside (0,2)
    with pytest.raises(lbm.LBMError):
        lbm.Sim(mesh, 7, 1.6, device=None)          # unknown stencil
    with pytest.raises(lbm.LBMError, match="outlet"):
        lbm.Sim(mesh, 9, 1.6, device=None, outlet=2)  # unknown outlet extrapolation
    half_periodic = W.Mesh(2, mesh.extent, (0, 1, 0, 0), mesh.tree_ids, mesh.levels, mesh.coords, mesh.lmin)
    with pytest.raises(lbm.LBMError, match="periodic"):
        lbm.Sim(half_periodic, 9, 1.6, device=None)
    # explicit level count: below the span of the treeIDs, or beyond 16
    with pytest.raises(lbm.LBMError, match="n_levels"):
        lbm.Sim(mesh, 9, 1.6, device=None, n_levels=1)
    with pytest.raises(lbm.LBMError, match="n_levels"):
        lbm.Sim(mesh, 9, 1.6, device=None, n_levels=17)
    # mass check settings
    with pytest.raises(lbm.LBMError, match="check_every"):
        lbm.Sim(mesh, 9, 1.6, device=None, check_every=-1)
    with pytest.raises(lbm.LBMError, match="mass_band"):
        lbm.Sim(mesh, 9, 1.6, device=None, check_every=10, mass_band=-1e-3)
    with pytest.raises(lbm.LBMError, match="mass_band"):
        lbm.Sim(mesh, 9, 1.6, device=None, check_every=10, mass_band=float("nan"))
    with pytest.raises(lbm.LBMError, match="adjoint_tape"):
        lbm.Sim(mesh, 9, 1.6, device=None, adjoint_tape=3)


@pytest.mark.parametrize("mode", [0, 1])
def test_empty_refined_levels_in_mesh_info(lbm, oracle_mod, mode):
    """An explicit level count adds finer levels with no element (an empty
    refined region): the library and the oracle both report them, with zero
    fluid and ghost counts, and the levels that hold elements are unchanged."""
    mesh = W.config_tgv2d()
    # omega_c = 1.8 keeps every level's rate away from 1 (1.6 reaches 1 on the third)
    base = lbm.Sim(mesh, 9, 1.8, time_mode=mode, device=None).mesh_info()
    more = lbm.Sim(mesh, 9, 1.8, time_mode=mode, device=None, n_levels=4).mesh_info()
    assert len(base) == 2 and len(more) == 4
    assert np.array_equal(more[:2, :5], base[:, :5])
    assert more[2, 0] == base[1, 0] + 1 and more[3, 0] == base[1, 0] + 2
    assert (more[2:, 1:5] == 0).all()
    oc = oracle_mod.Oracle(mesh, 9, 1.8, time_mode=mode, n_levels=4).counts()
    assert len(oc) == 4 and (oc[2:, 1:] == 0).all()
    with pytest.raises(oracle_mod.OracleError, match="n_levels"):
        oracle_mod.Oracle(mesh, 9, 1.6, n_levels=1)


def test_sfc_worked_example(lbm):
    """Sec. 3.1, Fig. partition: z-curve order, weights, cumulative weights and
    the split over three processes of the 10-element quadtree."""
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "worked_example.json")))
    el = g["elements"]
    # treeIDs of the figure agree with the encoding used by the workloads
    for e in el:
        assert W.tree_ids(np.array([[e["x"], e["y"]]]), e["level"], 2)[0] == e["tree_id"]
    # hand the elements over in a scrambled order
    tids = np.array([e["tree_id"] for e in el], np.int64)[[3, 9, 0, 5, 7, 1, 8, 2, 6, 4]]
    order, w, cum, part = lbm.lbm_sfc_partition(tids, 2, g["processes"])
    assert tids[order].tolist() == g["sfc_order"]
    assert w.tolist() == g["weights"]
    assert cum.tolist() == g["cumulative_weights"]
    assert np.bincount(part, minlength=g["processes"]).tolist() == g["partition_sizes"]


def test_updates_weighting():
    """Fine-substep weighted updates per coarse step, sum_L N_L 2^{L-Lmin}."""
    m = W.config_tgv2d()
    assert m.updates_per_coarse_step() == 768 + 2 * 1024
    m3 = W.config_tgv3d(64)
    assert m3.updates_per_coarse_step() == 229376 + 2 * 262144


def _interior_bricks(mesh, Q):
    """Per level, interior bricks counted from the element coordinates alone:
    aligned blocks of 64 same-level elements (4^3 / 8^2) whose neighbour
    blocks reached by the stencil are complete too (D3Q19: faces and edges;
    D2Q9 and D3Q27: all of them); periodic axes wrap when their extent is a
    whole number of blocks."""
    d = mesh.d
    side = 4 if d == 3 else 8
    offs = [o for o in itertools.product((-1, 0, 1), repeat=d) if any(o)]
    if Q == 19:
        offs = [o for o in offs if sum(map(abs, o)) <= 2]  # D3Q19 reaches no corner block
    out, complete = [], []
    for L in sorted(set(int(v) for v in mesh.levels)):
        sel = mesh.levels == L
        xyz = mesh.coords[sel][:, :d] // side
        keys, cnt = np.unique(xyz, axis=0, return_counts=True)
        full = {tuple(k) for k, c in zip(keys, cnt) if c == side ** d}
        complete.append(len(full))
        ext = [e << (L - mesh.lmin) for e in mesh.extent]
        nb = [(e + side - 1) // side for e in ext]
        n = 0
        for k in full:
            ok = True
            for o in offs:
                q = []
                for a in range(d):
                    v = k[a] + o[a]
                    if v < 0 or v >= nb[a]:
                        if mesh.bc[2 * a] != W.BC_PERIODIC or ext[a] % side:
                            ok = False
                            break
                        v %= nb[a]
                    q.append(v)
                if not ok or tuple(q) not in full:
                    ok = False
                    break
            n += ok
        out.append(n)
    return out, complete


@pytest.mark.parametrize("name", ["tgv2d", "tgv3d16", "half2d", "cylinder", "sphere_small", "tgv3d32_q27",
                                  "sphere_small_q27"])
def test_interior_brick_counts(lbm, name):
    """The builder's interior bricks match an independent count, every other
    complete brick is a boundary brick, and the builder has checked each
    brick's link table against the neighbour list."""
    mesh, Q = {"tgv2d": (W.config_tgv2d(), 9), "tgv3d16": (W.config_tgv3d(16), 19),
               "half2d": (W.half_refined_2d(32), 9), "cylinder": (W.config_cylinder(), 9),
               "sphere_small": (W.config_sphere_small(), 19), "tgv3d32_q27": (W.config_tgv3d(32), 27),
               "sphere_small_q27": (W.config_sphere_small(), 27)}[name]
    info = lbm.Sim(mesh, Q, 1.7, u_in=(0.04, 0, 0), device=None).mesh_info()
    interior, complete = _interior_bricks(mesh, Q)
    assert [int(r[8]) for r in info] == interior
    assert [int(r[8] + r[9]) for r in info] == complete


def test_obstacle_links_and_link_q(lbm):
    """lbm_obstacle_links lists exactly the (element, direction) pairs whose
    upstream cell x - c_i lies inside the cylinder (computed here from the
    geometry), and lbm_set_link_q checks its arguments."""
    D = 20
    m = W.config_cylinder_schafer(D)
    s = lbm.Sim(m, 9, 1.6, u_in=(0.05, 0, 0), device=None, bouzidi=True, inlet_profile=1)
    e, d = s.obstacle_links()
    c9 = np.array([[0, 0], [1, 0], [-1, 0], [0, 1], [0, -1], [1, 1], [-1, -1], [1, -1], [-1, 1]])
    fine = m.levels == m.levels.max()
    want = set()
    for k in np.nonzero(fine)[0]:
        for i in range(1, 9):
            p = m.coords[k] - c9[i] + 0.5
            if (p[0] - 2 * D) ** 2 + (p[1] - 2 * D) ** 2 < (D / 2) ** 2:
                want.add((int(k), i))
    assert set(zip(e.tolist(), d.tolist())) == want
    q = W.wall_distance_ball(m, e, d, (2 * D, 2 * D), D / 2, 9)
    assert np.all((q > 0) & (q <= 1))
    s.set_link_q(q)
    with pytest.raises(lbm.LBMError, match="obstacle link count"):
        s.set_link_q(q[:-1])
    with pytest.raises(lbm.LBMError, match="outside"):
        s.set_link_q(np.zeros(len(q)))
    hb = lbm.Sim(m, 9, 1.6, u_in=(0.05, 0, 0), device=None)
    with pytest.raises(lbm.LBMError, match="bouzidi"):
        hb.set_link_q(q)


def test_diffusive_mode_needs_wider_level_margins(lbm, oracle_mod):
    """Four GhostFromCoarser layers reach one coarse cell further than two: a
    three-level mesh whose finest box sits two level-1 cells inside the level-1
    box builds in the two-layer mode, but in the diffusive mode a ghost's coarse
    source would itself be a ghost, and the oracle and the library both reject
    it; four cells of margin build in every mode."""
    def mesh(margin):
        lo, hi = 32 + 2 * margin, 96 - 2 * margin
        return W.nested_boxes(2, 5, (32, 32), [((16, 16), (48, 48)), ((lo, lo), (hi, hi))], (0,) * 4)
    thin, wide = mesh(2), mesh(4)
    lbm.Sim(thin, 9, 1.7, time_mode=1, device=None)
    oracle_mod.Oracle(thin, 9, 1.7, time_mode=1)
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.Oracle(thin, 9, 1.7, time_mode=2)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.Sim(thin, 9, 1.7, time_mode=2, device=None)
    assert ei.value.status == -2 and "source" in str(ei.value)
    for mode in (0, 1, 2):
        lbm.Sim(wide, 9, 1.7, time_mode=mode, device=None)
        oracle_mod.Oracle(wide, 9, 1.7, time_mode=mode)

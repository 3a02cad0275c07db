"""Sec. 3.1 / 3.2: the weight-based decomposition along the space-filling curve
and the halo elements of each part, run as a distributed computation on the
CPU with gloo ranks.

Each rank splits the mesh with lbm_sfc_partition, takes its halo plan from
lbm_halo_plan and steps the CPU oracle op by op, in the order of the recursive
level stepping (Sec. 2.2), on its own elements; every element outside its own
and its halo holds NaN.  After each stream-collide of a level the ranks
exchange that level's halo over gloo (each sends what the other's plan lists
under it).  After several coarse steps every owned element must equal the
single-rank run bit for bit: a halo element missing from the plan would carry
NaN in, and a stale one (a missing exchange) would change the bits.  The ranks
also check that what each asks of the other is what the other's own plan says
it must send.
"""
import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _case(name):
    """mesh, Q, omega_c, u_in, outlet, wall (centre, radius) of interpolated
    bounce-back or None, fields, coarse steps"""
    from paper_1601_06984_gb300 import workloads as W
    if name == "tgv2d":
        m = W.config_tgv2d()
        return m, 9, 1.6, (0, 0, 0), 0, None, lambda m: W.tgv_fields(m, 0.02), 6
    if name == "tgv3d":
        m = W.config_tgv3d(16)
        return m, 19, 1.6, (0, 0, 0), 0, None, lambda m: W.tgv_fields(m, 0.02), 3
    if name == "schafer20":
        m = W.config_cylinder_schafer(20)
        om = W.omega_coarse_from_finest(W.omega_for_re(0.05, 20, 20.0), 2)
        return m, 9, om, (0.05, 0, 0), 1, ((40.0, 40.0), 10.0), lambda m: W.uniform_fields(m, 1.0, (0.05, 0.0)), 3
    if name == "sphere5":
        m = W.config_sphere_5level_small()
        om = W.omega_coarse_from_finest(1.6, 5)
        return (m, 19, om, (0.04, 0, 0), 1, None, lambda m: W.uniform_fields(m, 1.0, (0.04, 0.0, 0.0)), 2)
    raise KeyError(name)


def _distributed(name, mode, rank, world, dist):
    import torch

    from oracle import oracle as O
    from paper_1601_06984_gb300 import lbm, workloads as W
    m, Q, om, uin, outlet, wall, fields, steps = _case(name)
    d = 2 if Q == 9 else 3
    bz = wall is not None
    sim = lbm.Sim(m, Q, om, time_mode=mode, u_in=uin, outlet=outlet, bouzidi=bz, inlet_profile=1 if bz else 0,
                  device=None)
    order, _, _, ps = lbm.lbm_sfc_partition(m.tree_ids, d, world)
    part = np.empty(m.n, np.int32)
    part[order] = ps
    recv, ghosts = sim.halo_plan(part, world, rank)
    send = {p: sim.halo_plan(part, world, p)[0].get(rank, np.zeros(0, np.int64)) for p in range(world) if p != rank}
    # what the others ask of this rank equals what this rank's copy of their plans says it sends
    asked = [None] * world
    dist.all_gather_object(asked, {p: v.tolist() for p, v in recv.items()})
    consistent = all(asked[p].get(rank, []) == send[p].tolist() for p in send)
    link = None
    if bz:
        e, dr = sim.obstacle_links()
        link = (e, dr, W.wall_distance_ball(m, e, dr, wall[0], wall[1], Q))

    def oracle():
        o = O.Oracle(m, Q, om, time_mode=mode, u_in=uin, outlet=outlet, inlet_profile=1 if bz else 0)
        if link is not None:
            o.set_link_q(*link)
        o.init(*fields(m), W.pdf_perturbation(m, Q, 1e-4))
        return o

    ref = oracle()
    f0 = ref.get_f()
    ref.step(steps)
    f_ref = ref.get_f()
    lev = (m.levels.astype(np.int64) - m.lmin)
    mine = part == rank
    loc = oracle()
    view = np.full_like(f0, np.nan)
    view[mine] = f0[mine]
    loc.set_f(view)
    exchanges = [0]

    def exchange(levels):
        f = loc.get_f()
        reqs, into = [], []
        for p in sorted(send):
            s_idx = send[p][np.isin(lev[send[p]], levels)]
            r_all = recv.get(p, np.zeros(0, np.int64))
            r_idx = r_all[np.isin(lev[r_all], levels)]
            if len(s_idx):
                reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(f[s_idx])), p))
            if len(r_idx):
                buf = torch.empty((len(r_idx), Q), dtype=torch.float64)
                reqs.append(dist.irecv(buf, p))
                into.append((r_idx, buf))
        for r in reqs:
            r.wait()
        for r_idx, buf in into:
            f[r_idx] = buf.numpy()
        loc.set_f(f)
        exchanges[0] += 1

    nlev = loc.nlev()

    def advance(li):
        finer = li + 1 < nlev
        if finer:
            loc.op(loc.OP_GFF, li)
            loc.op(loc.OP_MOM_A, li)
            loc.op(loc.OP_GFC_A, li)
        loc.op(loc.OP_SC, li)
        exchange([li])
        if finer:
            advance(li + 1)
            if mode == 0:
                loc.op(loc.OP_MOM_B, li)
                loc.op(loc.OP_GFC_B, li)
            for _ in range(3 if mode == 2 else 1):  # four substeps with diffusive scaling
                advance(li + 1)

    exchange(list(range(nlev)))  # the initial state's halo
    for _ in range(steps):
        advance(0)
    f = loc.get_f()
    own_equal = bool(np.array_equal(f[mine], f_ref[mine]))
    n_halo = int(sum(len(v) for v in recv.values()))
    return {"consistent": consistent, "own_equal": own_equal, "own": int(mine.sum()), "halo": n_halo,
            "ghosts": int(len(ghosts)), "exchanges": exchanges[0], "n": int(m.n)}


CASES = [("tgv2d", 0), ("tgv2d", 1), ("tgv2d", 2), ("tgv3d", 0), ("tgv3d", 1), ("tgv3d", 2), ("schafer20", 0),
         ("schafer20", 2), ("sphere5", 0)]


def _worker(rank, world, port, cases, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    O.set_threads(max(1, (os.cpu_count() or 2) // world))
    out = {}
    try:
        for name, mode in cases:
            out[(name, mode)] = _distributed(name, mode, rank, world, dist)
    except Exception as ex:  # reported to the parent, which fails the test
        out["error"] = repr(ex)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


def _run(world, cases, port_offset):
    from oracle import oracle as O
    O.build()
    from paper_1601_06984_gb300 import build
    build.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29600 + port_offset + os.getpid() % 500
    procs = [ctx.Process(target=_worker, args=(r, world, port, cases, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def test_distributed_run_with_halo_exchange_two_ranks():
    res = _run(2, CASES, 0)
    for rank, out in res.items():
        assert "error" not in out, out.get("error")
        for key in CASES:
            r = out[key]
            assert r["consistent"], (rank, key)
            assert r["own_equal"], (rank, key, r)
            assert 0 < r["halo"] < r["n"] - r["own"], (rank, key, r)
    # the two parts split the weighted work and together own every element
    for key in CASES:
        assert res[0][key]["own"] + res[1][key]["own"] == res[0][key]["n"]


def test_distributed_run_three_ranks():
    res = _run(3, [("tgv2d", 0), ("sphere5", 0), ("sphere5", 2)], 700)
    for rank, out in res.items():
        assert "error" not in out, out.get("error")
        for key, r in out.items():
            assert r["consistent"] and r["own_equal"], (rank, key, r)


def test_single_part_needs_no_halo():
    """One part owns everything: nothing to receive, and it fills every ghost
    that an element reads (in LINEAR mode not the outer GhostFromCoarser layer,
    which nothing reads)."""
    sys.path.insert(0, ROOT)
    from paper_1601_06984_gb300 import lbm, workloads as W
    m = W.config_tgv2d()
    for mode in (0, 1):
        s = lbm.Sim(m, 9, 1.6, time_mode=mode, device=None)
        recv, ghosts = s.halo_plan(np.zeros(m.n, np.int32), 1, 0)
        assert recv == {}
        if mode == 1:
            assert len(ghosts) == s.ghost_count()
        else:
            assert 0 < len(ghosts) < s.ghost_count()
    with pytest.raises(lbm.LBMError):
        s.halo_plan(np.full(m.n, 2, np.int32), 2, 0)

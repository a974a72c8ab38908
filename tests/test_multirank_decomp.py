"""The sectored timestep split over ranks (Sec. 5.1) on CPU: two gloo ranks
on 127.0.0.1, each holding a copy of the system in the oracle but owning
only the atoms of its slab of sector columns (paper_1801_10233_gb300.decomp).
Every atom a rank does not own starts scrambled (random spin, displaced
position) except its halo, which the owner sends: the spins each colour's
pass turned after that pass, the positions after each drift.  After 10 steps
the owned atoms of both ranks equal the single-domain oracle bit for bit: the
plan delivers everything an owned atom reads, in time, and the global
colouring keeps each pass's result independent of the cut.  Dropping one
colour's exchange breaks the equality (the check has teeth)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STEPS = 10


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _system():
    from paper_1801_10233_gb300 import inputs
    # 12 cells along x: 8 sector columns of 4.3 A, two slabs of 4 columns
    return inputs.bcc_fe_system((12, 8, 8), 91, T=200.0, sigma=0.02, spins="uniform")


def _rank(rank, world, port, q, skip_colour):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1801_10233_gb300 import decomp
        p, r, v, s = _system()
        o = oracle.Oracle(p, r, v, s)
        order = o.order()
        nsec = order["nsec"]
        sector_x = order["sector"] % nsec[0]
        bounds = decomp.slab_bounds(int(nsec[0]), world)
        own = decomp.owners(sector_x, bounds)
        L = float(p["box"][0])
        reach = p["morse_rc_A"] + p["skin_A"]
        r0 = o.state()[0]
        plan = decomp.halo_plan(r0[:, 0], order["colour"], own, bounds, L / nsec[0], L, reach)
        peers = [k for k in range(world) if k != rank]

        def exchange(ids_out, ids_in, what):
            # send my owned atoms' rows, receive the owners' rows of my halo
            cur = o.state()
            data = cur[0] if what == "r" else cur[2]
            reqs, bufs = [], []
            for k in peers:
                out = torch.from_numpy(np.ascontiguousarray(data[ids_out[k]]))
                reqs.append(dist.isend(out, dst=k))
                buf = torch.empty((len(ids_in[k]), 3), dtype=torch.float64)
                reqs.append(dist.irecv(buf, src=k))
                bufs.append((k, buf))
            for rq in reqs:
                rq.wait()
            for k, buf in bufs:
                if what == "r":
                    o.set_atoms(ids_in[k], r=buf.numpy())
                else:
                    o.set_atoms(ids_in[k], s=buf.numpy())

        every_out = {k: decomp.halo_ids(plan, rank, k) for k in peers}
        every_in = {k: decomp.halo_ids(plan, k, rank) for k in peers}
        # scramble every atom this rank does not own, then receive the halo
        rng = np.random.default_rng(100 + rank)
        foreign = np.flatnonzero(own != rank)
        g = rng.normal(size=(len(foreign), 3))
        o.set_atoms(foreign, r=r0[foreign] + rng.uniform(-0.05, 0.05, (len(foreign), 3)),
                    s=g / np.linalg.norm(g, axis=1, keepdims=True))
        exchange(every_out, every_in, "r")
        exchange(every_out, every_in, "s")

        def hook(event, arg):
            if event == 0:      # colour `arg` was just turned: its halo spins
                if arg == skip_colour:
                    return
                exchange({k: plan[(rank, k)][arg] for k in peers}, {k: plan[(k, rank)][arg] for k in peers}, "s")
            else:               # positions after the drift
                exchange(every_out, every_in, "r")

        o.set_hook(hook)
        assert o.step(STEPS) == 0
        o.set_hook(None)
        mine = np.flatnonzero(own == rank)
        rr, vv, ss = o.state()
        q.put((rank, mine, rr[mine], vv[mine], ss[mine], o.rebuilds, {k: len(every_in[k]) for k in peers}))
    finally:
        dist.destroy_process_group()


def _run(skip_colour=-1):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(k, 2, port, q, skip_colour)) for k in range(2)]
    for pr in procs:
        pr.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    return res


def _single_domain():
    sys.path.insert(0, ROOT)
    import oracle
    p, r, v, s = _system()
    o = oracle.Oracle(p, r, v, s)
    o.step(STEPS)
    return o.state()


def test_two_slabs_reproduce_the_single_domain_bit_for_bit():
    res = _run()
    r1, v1, s1 = _single_domain()
    owned = np.concatenate([t[1] for t in res])
    assert np.array_equal(np.sort(owned), np.arange(len(r1)))      # every atom owned once
    for rank, ids, rr, vv, ss, rebuilds, halo in res:
        assert rebuilds == 1                                        # the initial sector assignment only
        assert all(n > 0 for n in halo.values())
        assert np.array_equal(rr, r1[ids]), rank
        assert np.array_equal(vv, v1[ids]), rank
        assert np.array_equal(ss, s1[ids]), rank


def test_a_missing_colour_exchange_is_detected():
    res = _run(skip_colour=3)
    r1, v1, s1 = _single_domain()
    assert any(not np.array_equal(ss, s1[ids]) for _, ids, _, _, ss, _, _ in res)


def test_slab_plan_on_the_host():
    sys.path.insert(0, ROOT)
    from paper_1801_10233_gb300 import decomp
    assert decomp.slab_bounds(8, 2) == [(0, 4), (4, 8)]
    assert decomp.slab_bounds(9, 4) == [(0, 2), (2, 4), (4, 6), (6, 9)]
    with pytest.raises(ValueError):
        decomp.slab_bounds(7, 4)
    # periodic distance to a slab: an atom just below x = 0 is near the slab [0, 4)
    d = decomp._distance_to_slab(np.array([-0.5, 1.0, 4.5, 9.5]), 0.0, 4.0, 10.0)
    assert np.allclose(d, [0.5, 0.0, 0.5, 0.5])

"""z-slab decomposition of one lattice (paper_1904_03618_gb300/slabs.py) on
CPU ranks: world size 2 and 3 over gloo, one process per rank, each rank
stepping its slab (own planes plus two ghost planes per neighbour, walls at
both local z ends) with the FP64 oracle and exchanging its two outermost own
planes with its neighbours after every step through the same exchange
schedule the GPU ranks use.  The slabs' own planes must equal the undivided
oracle run exactly (the oracle is deterministic and a cell's update reads
the state within two planes), for lattices periodic in z and with walls in
z (with forcing, gravity and the wetting rule at the real walls)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = {
    "periodic": dict(nx=6, ny=5, nz=12, wall=(0, 0, 0), improved=True, rho_in_R=3.0,
                     rho_in_B=1.0, alpha_R=0.9, alpha_B=0.7, tau_R=0.9, tau_B=1.2,
                     A_R=0.01, A_B=0.01, beta=0.7, force=(1e-4, 0.0, 2e-5)),
    "walls": dict(nx=5, ny=6, nz=12, wall=(0, 0, 1), improved=True, rho_in_R=3.0,
                  rho_in_B=1.0, alpha_R=0.9, alpha_B=0.7, tau_R=1.1, tau_B=0.8,
                  A_R=0.01, A_B=0.01, beta=0.7, gravity=(0.0, 1e-4, -2e-4),
                  wetting=True, contact_angle_deg=60.0),
}
STEPS = 4


def _fields(pd):
    sys.path.insert(0, ROOT)
    from paper_1904_03618_gb300 import workloads as wl
    return wl.random_fields(pd["nx"], pd["ny"], pd["nz"], seed=11)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, name, q):
    sys.path.insert(0, ROOT)
    os.environ["OMP_NUM_THREADS"] = "1"
    import oracle
    from paper_1904_03618_gb300 import slabs
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        pd = CASES[name]
        plan = slabs.SlabPlan(pd["nz"], world, rank, bool(pd["wall"][2]))
        p = oracle.params_from(plan.local_params(pd))
        state = {"f": oracle.init(p, *slabs.split_fields(plan, _fields(pd)))}

        def get_planes(z0, n):
            return torch.from_numpy(np.ascontiguousarray(state["f"][:, :, z0:z0 + n]))

        def set_planes(z0, n, t):
            state["f"][:, :, z0:z0 + n] = t.numpy().reshape(state["f"][:, :, z0:z0 + n].shape)

        send_recv = slabs.torch_send_recv(dist, torch.empty(0, dtype=torch.float64),
                                          2 * 19 * pd["ny"] * pd["nx"])
        for _ in range(STEPS):
            state["f"] = oracle.step(p, state["f"], 1)
            slabs.exchange_p2p(plan, get_planes, set_planes, send_recv)
        q.put((rank, plan.z0, state["f"][:, :, plan.local_own].copy()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("world", [2, 3])
def test_slabs_equal_the_undivided_lattice(name, world):
    sys.path.insert(0, ROOT)
    import oracle
    pd = CASES[name]
    p = oracle.params_from(pd)
    ref = oracle.step(p, oracle.init(p, *_fields(pd)), STEPS)
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, name, q))
             for r in range(world)]
    for pr in procs:
        pr.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for pr in procs:
        pr.join(60)
        assert pr.exitcode == 0
    covered = 0
    for rank, z0, own in sorted(got, key=lambda g: g[0]):
        n = own.shape[2]
        assert np.array_equal(own, ref[:, :, z0:z0 + n]), (rank, np.abs(own - ref[:, :, z0:z0 + n]).max())
        covered += n
    assert covered == pd["nz"]


def test_plan_covers_the_lattice_and_pairs_every_send_with_a_receive():
    sys.path.insert(0, ROOT)
    from paper_1904_03618_gb300 import slabs
    for nz, world, walls in [(12, 2, True), (12, 2, False), (13, 3, True), (17, 4, False),
                             (1024, 8, True), (1024, 1, False)]:
        plans = [slabs.SlabPlan(nz, world, r, walls) for r in range(world)]
        assert sum(p.own for p in plans) == nz
        assert [p.z0 for p in plans] == list(np.cumsum([0] + [p.own for p in plans[:-1]]))
        sends = sorted((r, peer, tag, n) for r, p in enumerate(plans)
                       for _, n, peer, tag in p.sends())
        recvs = sorted((peer, r, tag, n) for r, p in enumerate(plans)
                       for _, n, peer, tag in p.receives())
        assert sends == recvs
        for p in plans:
            assert p.nz_local == p.own + p.ghost_lo + p.ghost_hi
            if world > 1 and not walls:
                assert p.ghost_lo == p.ghost_hi == slabs.GHOST
    with pytest.raises(ValueError):
        slabs.SlabPlan(5, 3, 0, True)       # fewer than two own planes per slab
    with pytest.raises(ValueError):
        slabs.SlabPlan(12, 2, 0, False).local_params(dict(nx=4, ny=4, nz=12, wall=(0, 2, 0)))

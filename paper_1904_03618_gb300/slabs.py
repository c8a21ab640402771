"""One lattice cut into z-slabs: one slab per rank (one GPU each) or several
slabs on one device, with a halo exchange after every step.

A cell's update reads the stored state within two planes (its pulls, and
the phase field rho^N, Qbar of its neighbours, whose own moments come from
their pulls), so a slab keeps two ghost planes on each side that has a
neighbour.  After every step each slab sends its two outermost own planes
to the neighbour on that side, which writes them into its ghost planes;
then the slab's own planes evolve exactly as in the undivided lattice.  The
slab's context is an ordinary lattice of its own planes plus ghosts with
halfway bounce-back at both z ends: those walls only touch ghost planes,
whose values the next exchange overwrites (the lattice's real z walls, where
it has them, are the outer ends of the first and last slab).

The exchange copies the raw stored planes (lbm_get_planes / lbm_set_planes:
the library's storage format, exact for 16-bit storage) into LOCAL halo
buffers of the receiving slab; kernels only ever read their own device's
memory.  Between ranks the transfer is a point-to-point send / receive of
torch.distributed (NCCL between GPUs); within one process it is a device
copy.  The plan and the exchange schedule below are host logic only; the
step and the plane copies are the library's.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

GHOST = 2  # ghost planes per side with a neighbour


@dataclass(frozen=True)
class SlabPlan:
    """Slab `rank` of `world` of a lattice with nz planes (periodic in z,
    or halfway bounce-back walls at both z ends when z_walls)."""
    nz: int
    world: int
    rank: int
    z_walls: bool

    def __post_init__(self):
        if self.world < 1 or not 0 <= self.rank < self.world:
            raise ValueError("need 0 <= rank < world")
        if self.nz < GHOST * self.world:
            raise ValueError("every slab needs at least %d planes of its own" % GHOST)

    @property
    def z0(self) -> int:
        """First global plane of this slab's own range."""
        q, r = divmod(self.nz, self.world)
        return self.rank * q + min(self.rank, r)

    @property
    def own(self) -> int:
        q, r = divmod(self.nz, self.world)
        return q + (1 if self.rank < r else 0)

    @property
    def lower(self):
        """Rank holding the planes below, or None (a wall, or one slab)."""
        if self.world == 1:
            return None
        if self.rank == 0:
            return None if self.z_walls else self.world - 1
        return self.rank - 1

    @property
    def upper(self):
        if self.world == 1:
            return None
        if self.rank == self.world - 1:
            return None if self.z_walls else 0
        return self.rank + 1

    @property
    def ghost_lo(self) -> int:
        return GHOST if self.lower is not None else 0

    @property
    def ghost_hi(self) -> int:
        return GHOST if self.upper is not None else 0

    @property
    def nz_local(self) -> int:
        return self.ghost_lo + self.own + self.ghost_hi

    @property
    def local_own(self) -> slice:
        """The slab's own planes within its local lattice."""
        return slice(self.ghost_lo, self.ghost_lo + self.own)

    def local_params(self, pd: dict) -> dict:
        """lbm_params keywords of the slab's local lattice."""
        if self.world == 1:
            return dict(pd)
        wall = tuple(pd.get("wall", (0, 0, 0)))
        if 2 in wall:
            raise ValueError("moving plates (wall = 2) are not decomposed into slabs")
        if bool(wall[2]) != self.z_walls:
            raise ValueError("z_walls of the plan must match wall[2] of the lattice")
        d = dict(pd)
        d["nz"] = self.nz_local
        d["wall"] = (wall[0], wall[1], 1)
        return d

    def sends(self):
        """(first local plane, count, destination rank, tag) of each send
        after a step: the two lowest own planes go to the lower neighbour,
        the two highest to the upper one."""
        out = []
        if self.lower is not None:
            out.append((self.ghost_lo, GHOST, self.lower, 0))
        if self.upper is not None:
            out.append((self.ghost_lo + self.own - GHOST, GHOST, self.upper, 1))
        return out

    def receives(self):
        """(first local ghost plane, count, source rank, tag) of each
        receive; tag 0 = planes coming down from the upper neighbour, 1 =
        planes coming up from the lower one."""
        out = []
        if self.upper is not None:
            out.append((self.ghost_lo + self.own, GHOST, self.upper, 0))
        if self.lower is not None:
            out.append((0, GHOST, self.lower, 1))
        return out


def split_fields(plan: SlabPlan, fields):
    """The slab's local initial fields (own planes plus ghosts, periodic in
    z where the lattice is) from the whole lattice's (rho_R, rho_B, u) in
    the (z, y, x) / (3, z, y, x) layout."""
    rR, rB, u = fields
    idx = np.arange(plan.z0 - plan.ghost_lo, plan.z0 + plan.own + plan.ghost_hi) % plan.nz
    return (np.ascontiguousarray(rR[idx]), np.ascontiguousarray(rB[idx]),
            np.ascontiguousarray(u[:, idx]))


def exchange_p2p(plan: SlabPlan, get_planes, set_planes, send_recv):
    """One halo exchange between ranks.  get_planes(z0, n) -> tensor of the
    stored planes, set_planes(z0, n, tensor) writes them;
    send_recv(sends, receives) performs the transfers (lists of (tensor,
    peer, tag)) and returns the received tensors in order."""
    sends = [(get_planes(z0, n), peer, tag) for z0, n, peer, tag in plan.sends()]
    recvs = plan.receives()
    got = send_recv(sends, [(n, peer, tag) for _, n, peer, tag in recvs])
    for (z0, n, _, _), t in zip(recvs, got):
        set_planes(z0, n, t)


def torch_send_recv(dist, like, plane_numel):
    """send_recv for exchange_p2p over torch.distributed point-to-point
    operations (NCCL or gloo): buffers like `like` (dtype, device)."""
    import torch

    def run(sends, recvs):
        ops = []
        bufs = []
        for n, peer, tag in recvs:
            b = torch.empty(n * plane_numel, dtype=like.dtype, device=like.device)
            bufs.append(b)
            ops.append(dist.P2POp(dist.irecv, b, peer, tag=tag))
        for t, peer, tag in sends:
            ops.append(dist.P2POp(dist.isend, t.reshape(-1), peer, tag=tag))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        return bufs
    return run


class SlabLattice:
    """This rank's slab of one lattice on its own GPU, stepped with a halo
    exchange over torch.distributed after every step.  The context runs on
    the current torch stream of the device, so its steps, the plane copies
    and the collective transfers are ordered on one stream."""

    def __init__(self, pd: dict, plan: SlabPlan, dist=None, device=None, storage="f32",
                 refs=(0.0, 0.0)):
        import torch

        from . import lbm
        self.lbm = lbm
        self.plan = plan
        self.dist = dist
        self.device = torch.device(device or "cuda")
        local = plan.local_params(pd)
        self.params = lbm.make_params(storage=storage, **local)
        self.params.ref_R, self.params.ref_B = refs
        self.stream = torch.cuda.current_stream(self.device)
        self.lat = lbm.Lattice(self.params, device=self.device, stream=self.stream)
        nbytes = lbm.lbm_plane_bytes(self.lat.ctx)
        self.plane_words = nbytes // 4   # exchanged as 32-bit words
        self._buf = {}

    def init_fields(self, fields):
        self.lat.init_fields(*split_fields(self.plan, fields))

    def _get(self, z0, n):
        import torch
        key = ("s", z0, n)
        t = self._buf.get(key)
        if t is None:
            t = torch.empty(n * self.plane_words, dtype=torch.int32, device=self.device)
            self._buf[key] = t
        self.lbm.lbm_get_planes(self.lat.ctx, z0, n, t)
        return t

    def _set(self, z0, n, t):
        self.lbm.lbm_set_planes(self.lat.ctx, z0, n, t)

    def exchange(self):
        import torch
        like = torch.empty(0, dtype=torch.int32, device=self.device)
        exchange_p2p(self.plan, self._get, self._set,
                     torch_send_recv(self.dist, like, self.plane_words))

    def step(self, n=1):
        for _ in range(n):
            self.lbm.lbm_step(self.lat.ctx, 1)
            if self.plan.world > 1:
                self.exchange()

    def own_moments(self):
        """(rho_R, rho_B, u) of the slab's own planes."""
        rR, rB, u = self.lat.moments()
        s = self.plan.local_own
        return rR[s], rB[s], u[:, s]

    def close(self):
        self.lat.close()


class SlabsOnOneDevice:
    """All slabs of one lattice in one process on one device: each step
    advances every slab, then copies each slab's outer own planes into its
    neighbours' ghost planes (device to device).  Kernels of different
    slabs never wait on one another.  Used to check the decomposition
    against the undivided lattice on one GPU."""

    def __init__(self, pd: dict, world: int, device=None, storage="f32", refs=(0.0, 0.0)):
        import torch

        from . import lbm
        self.lbm = lbm
        self.device = torch.device(device or "cuda")
        z_walls = bool(tuple(pd.get("wall", (0, 0, 0)))[2])
        self.plans = [SlabPlan(pd["nz"], world, r, z_walls) for r in range(world)]
        self.stream = torch.cuda.current_stream(self.device)
        self.lats = []
        for plan in self.plans:
            p = lbm.make_params(storage=storage, **plan.local_params(pd))
            p.ref_R, p.ref_B = refs
            self.lats.append(lbm.Lattice(p, device=self.device, stream=self.stream))
        self.plane_bytes = lbm.lbm_plane_bytes(self.lats[0].ctx)
        self._tmp = torch.empty(GHOST * self.plane_bytes // 4, dtype=torch.int32,
                                device=self.device)

    def init_fields(self, fields):
        for plan, lat in zip(self.plans, self.lats):
            lat.init_fields(*split_fields(plan, fields))

    def exchange(self):
        for plan, lat in zip(self.plans, self.lats):
            for z0, n, peer, tag in plan.sends():
                self.lbm.lbm_get_planes(lat.ctx, z0, n, self._tmp)
                dst = self.plans[peer]
                # tag 0 (going down) lands in the peer's upper ghosts
                zr = dst.ghost_lo + dst.own if tag == 0 else 0
                self.lbm.lbm_set_planes(self.lats[peer].ctx, zr, n, self._tmp)

    def step(self, n=1):
        for _ in range(n):
            for lat in self.lats:
                self.lbm.lbm_step(lat.ctx, 1)
            if len(self.lats) > 1:
                self.exchange()

    def moments(self):
        """(rho_R, rho_B, u) of the whole lattice, assembled from the slabs'
        own planes."""
        import torch
        parts = []
        for plan, lat in zip(self.plans, self.lats):
            rR, rB, u = lat.moments()
            s = plan.local_own
            parts.append((rR[s], rB[s], u[:, s]))
        return (torch.cat([p[0] for p in parts]), torch.cat([p[1] for p in parts]),
                torch.cat([p[2] for p in parts], dim=1))

    def close(self):
        for lat in self.lats:
            lat.close()

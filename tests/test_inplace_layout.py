"""The in-place (AA) layout of include/lbm.h is a correct streaming scheme.

The GPU tests check the in-place kernels against the oracle and against the
layout the header documents.  This host test checks the layout itself, on
small lattices of every wall combination (including axes of one and two
cells, where a cell is its own or its only neighbour): with the slots the
header names -- a step from an even state reads slot (i, x) and writes
f_i^+ to (opp(i), x); a step from an odd state reads f_i(x, t) at
(opp(i), x - e_i), or (i, x) where x - e_i lies beyond a wall, and writes
f_i^+ to (i, x + e_i), or (opp(i), x) across a wall --
  * every cell writes exactly the slots it reads, and the cells' slot sets
    partition the array (so one thread per cell races with no other);
  * processing the cells one at a time in random order, with a collision
    stand-in that mixes every direction and both colours, gives after each
    of four steps the state that plain push streaming with halfway
    bounce-back gives.
"""
import itertools

import numpy as np
import pytest

# D3Q19 in the order of Eq. 5; opp pairs (1,2), (3,4), ..., (17,18)
EX = (0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0)
EY = (0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1)
EZ = (0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1)
OPP = tuple(0 if i == 0 else (i + 1 if i % 2 else i - 1) for i in range(19))


def _neighbour(dims, walls, cell, d):
    """Index of cell + d (periodic wrap), None beyond a wall."""
    out = []
    for c, dc, n, w in zip(cell, d, dims, walls):
        v = c + dc
        if not 0 <= v < n:
            if w:
                return None
            v %= n
        out.append(v)
    x, y, z = out
    return (z * dims[1] + y) * dims[0] + x


def _read_slot(odd, dims, walls, cell, c, i, N):
    """Flat slot (direction * N + cell) of f_i(x, t) in a state of the given
    parity, as the header documents it."""
    if not odd:
        return i * N + c
    src = _neighbour(dims, walls, cell, (-EX[i], -EY[i], -EZ[i]))
    return i * N + c if src is None else OPP[i] * N + src


def _write_slot(odd, dims, walls, cell, c, i, N):
    if not odd:
        return OPP[i] * N + c
    dst = _neighbour(dims, walls, cell, (EX[i], EY[i], EZ[i]))
    return OPP[i] * N + c if dst is None else i * N + dst


def _collide(pre, c, t):
    """Stand-in for the collision: every output depends on several
    directions and both colours of the cell."""
    post = np.empty_like(pre)
    for k in range(2):
        for i in range(19):
            post[k, i] = (pre[k, (7 * i + 3) % 19] + 0.5 * pre[1 - k, i] + 0.01 * i
                          + 1e-3 * c + 1e-4 * t)
    return post


def _cells(dims):
    nx, ny, nz = dims
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        yield (x, y, z), (z * ny + y) * nx + x


def _push_reference(f, dims, walls, nsteps):
    for t in range(nsteps):
        g = np.full_like(f, np.nan)
        for cell, c in _cells(dims):
            post = _collide(f[:, :, c], c, t)
            for i in range(19):
                d = _neighbour(dims, walls, cell, (EX[i], EY[i], EZ[i]))
                if d is None:
                    g[:, OPP[i], c] = post[:, i]          # halfway bounce-back
                else:
                    g[:, i, d] = post[:, i]
        assert not np.isnan(g).any()
        f = g
    return f


@pytest.mark.parametrize("dims", [(4, 3, 3), (1, 3, 2), (2, 1, 2), (1, 1, 1)])
@pytest.mark.parametrize("walls", list(itertools.product((0, 1), repeat=3)))
def test_aa_layout_is_a_race_free_streaming_scheme(dims, walls):
    rng = np.random.default_rng(sum(dims) + 7 * sum(walls))
    N = dims[0] * dims[1] * dims[2]
    f0 = rng.standard_normal((2, 19, N))
    A = f0.reshape(2, 19 * N).copy()
    odd = 0
    for t in range(4):
        order = list(_cells(dims))
        rng.shuffle(order)
        owner = np.zeros(19 * N, dtype=int)
        for cell, c in order:
            rs = [_read_slot(odd, dims, walls, cell, c, i, N) for i in range(19)]
            ws = [_write_slot(odd, dims, walls, cell, c, i, N) for i in range(19)]
            assert all(0 <= s < 19 * N for s in rs)
            assert sorted(rs) == sorted(ws)
            owner[rs] += 1
            post = _collide(A[:, rs], c, t)
            A[:, ws] = post
        assert (owner == 1).all()
        odd ^= 1
        got = np.empty((2, 19, N))
        for cell, c in _cells(dims):
            for i in range(19):
                got[:, i, c] = A[:, _read_slot(odd, dims, walls, cell, c, i, N)]
        want = _push_reference(f0, dims, walls, t + 1)
        assert np.array_equal(got, want), (dims, walls, t)

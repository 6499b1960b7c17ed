"""x-slab decomposition, host side (no GPU).

The partition of the columns, and the packing, ordering and routing of the
halo messages (paper_2103_01444_gb300.slabs) are checked with two gloo ranks
on the CPU: each rank steps its slab with the FP64 oracle, on its own
columns plus one ghost column per side that borders the other rank, and
after every step refills the ghost column from the neighbour through
slabs.exchange_with_neighbours, six populations per row (PLUS_X, MINUS_X).
The ranks' own columns then equal the oracle's single-lattice run bit for
bit: the exchange carries exactly what the pulls across a slab side read.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_partition_covers_the_lattice_in_order():
    from paper_2103_01444_gb300.slabs import partition
    for nx, n in ((200, 2), (203, 3), (64, 16), (9, 2)):
        r = partition(nx, n)
        assert r[0][0] == 0 and r[-1][1] == nx and len(r) == n
        assert all(a[1] == b[0] for a, b in zip(r[:-1], r[1:]))
        w = [x1 - x0 for x0, x1 in r]
        assert max(w) - min(w) <= 1 and min(w) >= 4
    with pytest.raises(ValueError):
        partition(15, 4)


def test_halo_planes_are_the_links_crossing_a_side():
    """The six planes leaving through the high side are those with e_x = +1
    (D2Q9, Eq. 2: 1, 5, 8; D2Q5, Eq. 9: link 1 of each scalar), through the
    low side those with e_x = -1; every other plane stays in its column."""
    from paper_2103_01444_gb300.slabs import MINUS_X, PLUS_X
    ex9 = [0, 1, 0, -1, 0, 1, -1, -1, 1]
    ex5 = [0, 1, 0, -1, 0]
    ex = ex9 + ex5 * 3
    assert sorted(PLUS_X) == [q for q in range(24) if ex[q] == 1]
    assert sorted(MINUS_X) == [q for q in range(24) if ex[q] == -1]


def _slab_oracle(case, x0, x1, nx):
    """Oracle over the columns [x0 - g_lo, x1 + g_hi) of the whole lattice:
    the slab plus a ghost column on each side inside the lattice."""
    from oracle import Oracle
    from oracle.params import lattice_problem
    params, material, solid = lattice_problem(case, interface_mode=1)
    lo, hi = (1 if x0 > 0 else 0), (1 if x1 < nx else 0)
    a, b = x0 - lo, x1 + hi
    p = dict(params, nx=b - a)
    mat = {k: np.ascontiguousarray(np.asarray(v)[:, a:b]) for k, v in material.items()}
    sol = None if solid is None else np.ascontiguousarray(solid[:, a:b])
    return Oracle(p, mat, sol), lo, hi


def _state(o):
    return np.concatenate([o.f, o.g.reshape(15, o.ny, o.nx)], axis=0)


def _set_planes(o, planes, col, values):
    for k, q in enumerate(planes):
        if q < 9:
            o.f[q, :, col] = values[k]
        else:
            s, i = divmod(q - 9, 5)
            o.g[s, i, :, col] = values[k]


def _worker(rank, world, port, case, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2103_01444_gb300.slabs import MINUS_X, PLUS_X, exchange_with_neighbours, partition
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nx = case["nx"]
    x0, x1 = partition(nx, world)[rank]
    o, lo, hi = _slab_oracle(case, x0, x1, nx)
    first, last = lo, lo + (x1 - x0) - 1          # own columns in the oracle's lattice
    buf = {k: torch.zeros((6, case["ny"]), dtype=torch.float64)
           for k in ("lo_out", "hi_out", "lo_in", "hi_in")}
    for _ in range(steps):
        o.step(1)
        st = _state(o)
        buf["lo_out"].copy_(torch.from_numpy(st[list(MINUS_X), :, first]))
        buf["hi_out"].copy_(torch.from_numpy(st[list(PLUS_X), :, last]))
        exchange_with_neighbours(rank, world, buf["lo_out"], buf["hi_out"], buf["lo_in"],
                                 buf["hi_in"])
        if lo:
            _set_planes(o, PLUS_X, 0, buf["lo_in"].numpy())
        if hi:
            _set_planes(o, MINUS_X, last + 1, buf["hi_in"].numpy())
    out.put((rank, _state(o)[:, :, first:last + 1]))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("kind", ["film-pressure", "grains"])
def test_two_gloo_ranks_equal_the_single_lattice(kind):
    from oracle import Oracle
    from oracle.params import lattice_problem
    from paper_2103_01444_gb300 import workloads
    if kind == "grains":
        case = workloads.small_cathode(nx=46, ny=16, reaction_mode=0, grains=True, seed=9,
                                       V_op=0.45)
    else:
        case = dict(workloads.small_cathode(nx=41, ny=14, reaction_mode=0, V_op=0.45, seed=3),
                    inlet="pressure", dp_in=1e-3, scalar_advection=1)
    steps = 60
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, case, steps, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    params, material, solid = lattice_problem(case, interface_mode=1)
    ref = _state(Oracle(params, material, solid).step(steps))
    got = np.concatenate([res[0], res[1]], axis=2)
    live = (Oracle(params, material, solid).mask & 3) != 3
    np.testing.assert_array_equal(got[:, live], ref[:, live])

"""x-slab decomposition on the GPU: a lattice split into slabs (domains
owning column ranges, joined by the halo exchange after every step) steps
bit for bit like the whole lattice, with the library's own kernels."""
import os
import socket
import sys

import numpy as np
import pytest

from paper_2103_01444_gb300 import workloads

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2103_01444_gb300.build import build
    build()


def case_of(name):
    if name == "film":
        return workloads.small_cathode(nx=150, ny=20, reaction_mode=0, V_op=0.45, seed=2)
    if name == "vol-p":
        return dict(workloads.small_cathode(nx=131, ny=24, reaction_mode=1, V_op=0.4, seed=4),
                    inlet="pressure", dp_in=1e-3, scalar_advection=1)
    if name == "grains":
        return workloads.small_cathode(nx=140, ny=24, reaction_mode=0, grains=True, seed=9,
                                       V_op=0.45)
    raise KeyError(name)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("name,nslabs,mode", [("film", 2, 0), ("vol-p", 3, 1), ("grains", 4, 1)])
def test_slabs_step_like_the_whole_lattice(name, nslabs, mode, precision):
    from paper_2103_01444_gb300.lbm import Domain
    from paper_2103_01444_gb300.slabs import SlabLattice
    case = case_of(name)
    whole = Domain.from_case(case, precision=precision, interface_mode=mode)
    sl = SlabLattice(case, nslabs, precision=precision, interface_mode=mode)
    for n in (1, 70):
        whole.step(n)
        sl.step(n)
        np.testing.assert_array_equal(sl.state(), whole.state())
    fw, fs = whole.fields(), sl.fields()
    for k in fw:
        np.testing.assert_array_equal(fs[k], fw[k])
    i_w, h_w, p_w = whole.current_density()
    i_s, h_s, p_s = sl.current_density()
    np.testing.assert_array_equal(p_s, p_w)
    assert i_s == pytest.approx(i_w, rel=1e-12) and h_s == pytest.approx(h_w, rel=1e-12)


def test_pack_and_unpack_carry_the_same_halo_as_the_exchange():
    import torch
    from paper_2103_01444_gb300.lbm import _check
    from paper_2103_01444_gb300.slabs import SlabLattice
    case = case_of("grains")
    a = SlabLattice(case, 2, precision="fp32", interface_mode=1)
    b = SlabLattice(case, 2, precision="fp32", interface_mode=1)
    bufs = [torch.zeros((6, a.ny), dtype=torch.float32, device="cuda") for _ in range(2)]
    for _ in range(40):
        a.step(1)
        lo, hi = b.slabs
        lo.step(1)
        hi.step(1)
        torch.cuda.synchronize()
        _check(lo.L.lbm_halo_pack(lo.h, 1, bufs[0].data_ptr()))
        _check(hi.L.lbm_halo_pack(hi.h, 0, bufs[1].data_ptr()))
        torch.cuda.synchronize()
        _check(hi.L.lbm_halo_unpack(hi.h, 0, bufs[0].data_ptr()))
        _check(lo.L.lbm_halo_unpack(lo.h, 1, bufs[1].data_ptr()))
        torch.cuda.synchronize()
    np.testing.assert_array_equal(b.state(), a.state())


def test_slab_refusals():
    from paper_2103_01444_gb300.lbm import Batch, LbmError, _check
    from paper_2103_01444_gb300.slabs import SlabLattice
    case = case_of("film")
    sl = SlabLattice(case, 3, precision="fp64")
    d0, d1, d2 = sl.slabs
    with pytest.raises(LbmError, match="EINVAL.*neighbours"):
        _check(d0.L.lbm_halo_exchange(d0.h, d2.h))
    with pytest.raises(LbmError, match="EINVAL.*borders no slab"):
        _check(d0.L.lbm_halo_pack(d0.h, 0, 1))
    d1.step(1)
    with pytest.raises(LbmError, match="ESTATE.*different steps"):
        _check(d0.L.lbm_halo_exchange(d0.h, d1.h))
    with pytest.raises(LbmError, match="EINVAL.*x-slabs"):
        d0.grad(0, 4)
    with pytest.raises(LbmError, match="EINVAL.*x-slabs"):
        Batch([d0, d2])


def _dist_worker(rank, world, port, case, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2103_01444_gb300.slabs import DistributedSlab
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = DistributedSlab(case, precision="fp64", interface_mode=1)
    s.step(steps)
    i, h = s.current_density()
    torch.cuda.synchronize()
    out.put((rank, s.d.state(), i, h))
    dist.barrier()
    dist.destroy_process_group()


def test_distributed_slabs_over_gloo_equal_the_whole_lattice():
    """DistributedSlab, one slab per process: two processes on this GPU
    (their kernels never wait on each other: each exchange goes through the
    host and gloo between steps) step the lattice bit for bit like one
    domain, and the all-reduced current density is the lattice's."""
    import torch.multiprocessing as mp
    from paper_2103_01444_gb300.lbm import Domain
    case = case_of("vol-p")
    steps = 50
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    procs = [ctx.Process(target=_dist_worker, args=(r, 2, port, case, steps, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        r, st, i, h = q.get(timeout=300)
        res[r] = (st, i, h)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    whole = Domain.from_case(case, precision="fp64", interface_mode=1)
    whole.step(steps)
    np.testing.assert_array_equal(np.concatenate([res[0][0], res[1][0]], axis=2), whole.state())
    i_w, h_w, _ = whole.current_density()
    assert res[0][1] == pytest.approx(i_w, rel=1e-12) and res[1][2] == pytest.approx(h_w, rel=1e-12)

"""x-slab decomposition of the cathode lattice.

The paper's domain (Sec. 4, Fig. 4) is a long channel over the GDL, so the
lattice splits naturally into slabs of whole columns along the flow
direction x.  A slab is an ordinary domain of the library that owns the
columns [x_begin, x_end) of the whole lattice (lbm_domain_desc.x_begin,
x_end); every step it pulls, at each side that borders another slab, six
populations per row from that neighbour's edge column:

  PLUS_X  (f1, f5, f8 and the D2Q5 link-1 populations of T, O2, H2O, Eq. 2
           and Eq. 9 numbering) leave a slab through its high side;
  MINUS_X (f3, f6, f7 and the link-3 populations) through its low side.

After every step each slab's ghost columns are refilled from its
neighbours' new state (6 ny values per side).  Slabs on one device exchange
with lbm_halo_exchange; slabs in different processes pack the values
(lbm_halo_pack), move them between processes (here with torch.distributed
point-to-point messages, one each way per pair of neighbours) and unpack
them (lbm_halo_unpack).  The reductions of Sec. 5 (current density, heat)
are sums over the slabs.
"""
from __future__ import annotations

import numpy as np

# Planes of the 24-population state ([f0..f8, g_T0..4, g_O2 0..4,
# g_H2O 0..4]) crossing a slab side, in the library's packing order.
PLUS_X = (1, 5, 8, 10, 15, 20)
MINUS_X = (3, 6, 7, 12, 17, 22)


def partition(nx: int, nslabs: int, min_width: int = 4):
    """Column ranges [x_begin, x_end) of nslabs slabs of nearly equal width
    covering nx columns (the first nx % nslabs slabs one column wider)."""
    if nslabs < 1 or nx < nslabs * min_width:
        raise ValueError(f"{nx} columns do not split into {nslabs} slabs of >= {min_width}")
    base, extra = divmod(nx, nslabs)
    out, x = [], 0
    for k in range(nslabs):
        w = base + (1 if k < extra else 0)
        out.append((x, x + w))
        x += w
    return out


def exchange_with_neighbours(rank: int, world: int, lo_out, hi_out, lo_in, hi_in, group=None):
    """One halo exchange between the processes of a 1D chain of slabs:
    lo_out goes to rank - 1 (and arrives there as its hi_in), hi_out to
    rank + 1 (its lo_in).  Non-blocking sends and receives, all posted
    before any is waited on, so the chain cannot deadlock; each pair of
    neighbours carries one message each way."""
    import torch.distributed as dist
    reqs = []
    if rank > 0:
        reqs.append(dist.irecv(lo_in, rank - 1, group=group))
        reqs.append(dist.isend(lo_out, rank - 1, group=group))
    if rank < world - 1:
        reqs.append(dist.irecv(hi_in, rank + 1, group=group))
        reqs.append(dist.isend(hi_out, rank + 1, group=group))
    for r in reqs:
        r.wait()


def combine_current(parts, widths):
    """Lattice mean current density and heat from per-slab means
    ((i_avg, heat) pairs) weighted by the slabs' widths."""
    n = float(sum(widths))
    i = sum(p[0] * w for p, w in zip(parts, widths)) / n
    h = sum(p[1] * w for p, w in zip(parts, widths)) / n
    return i, h


class SlabLattice:
    """A lattice split into x-slabs on one device: one library domain per
    slab, stepped in turn and joined by lbm_halo_exchange after every step.
    Reads and reductions concatenate or combine the slabs."""

    def __init__(self, case: dict, nslabs: int, precision="fp32", forchheimer: int = 1,
                 interface_mode: int = 0, stream=None):
        from .lbm import Domain, _check
        from .units import cathode_params
        self._check = _check
        params, fields, geo = cathode_params(case, forchheimer, interface_mode)
        self.nx, self.ny = geo["nx"], geo["ny"]
        self.ranges = partition(self.nx, nslabs)
        self.slabs = []
        for x0, x1 in self.ranges:
            d = Domain(precision=precision, stream=stream, x_begin=x0, x_end=x1, **geo)
            d.set_params(params)
            d.set_fields(**fields)
            self.slabs.append(d)
        self.reset()

    @property
    def widths(self):
        return [x1 - x0 for x0, x1 in self.ranges]

    def exchange(self):
        for a, b in zip(self.slabs[:-1], self.slabs[1:]):
            self._check(a.L.lbm_halo_exchange(a.h, b.h))

    def reset(self):
        for d in self.slabs:
            d.reset()
        self.exchange()

    def step(self, n: int = 1):
        for _ in range(int(n)):
            for d in self.slabs:
                d.step(1)
            self.exchange()
        return self

    def state(self):
        return np.concatenate([d.state() for d in self.slabs], axis=2)

    def fields(self):
        parts = [d.fields() for d in self.slabs]
        return {k: np.concatenate([p[k] for p in parts], axis=1) for k in parts[0]}

    def current_density(self):
        parts = [d.current_density() for d in self.slabs]
        i, h = combine_current(parts, self.widths)
        return i, h, np.concatenate([p[2] for p in parts])


class DistributedSlab:
    """This process's slab of a lattice split over the ranks of a
    torch.distributed group (one slab per rank, a 1D chain along x).  The
    halo values travel as [6][ny] arrays of the storage type: device tensors
    with a backend that moves CUDA tensors (NCCL), host copies otherwise.
    The domain runs on a torch stream of its own, which also carries the
    packing copies and, with NCCL, the messages, so that they are ordered
    after the step that produced them."""

    def __init__(self, case: dict, precision="fp32", forchheimer: int = 1,
                 interface_mode: int = 0, group=None):
        import torch
        import torch.distributed as dist
        from .lbm import Domain, _check
        from .units import cathode_params
        self._check, self.group = _check, group
        self.rank, self.world = dist.get_rank(group), dist.get_world_size(group)
        params, fields, geo = cathode_params(case, forchheimer, interface_mode)
        self.nx, self.ny = geo["nx"], geo["ny"]
        self.ranges = partition(self.nx, self.world)
        x0, x1 = self.ranges[self.rank]
        self.stream = torch.cuda.Stream()
        self.d = Domain(precision=precision, stream=self.stream.cuda_stream,
                        x_begin=x0, x_end=x1, **geo)
        self.d.set_params(params)
        self.d.set_fields(**fields)
        dtype = {"fp64": torch.float64, "fp32": torch.float32}.get(precision, torch.int16)
        dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
        self._dev = dev
        mk = lambda where: torch.zeros((6, self.ny), dtype=dtype, device=where)  # noqa: E731
        self.buf = {k: mk("cuda") for k in ("lo_out", "hi_out", "lo_in", "hi_in")}
        self.msg = self.buf if dev == "cuda" else {k: mk("cpu") for k in self.buf}
        self.reset()

    def exchange(self):
        import torch
        d, L, b, m = self.d, self.d.L, self.buf, self.msg
        lo, hi = self.rank > 0, self.rank < self.world - 1
        if lo:
            self._check(L.lbm_halo_pack(d.h, 0, b["lo_out"].data_ptr()))
        if hi:
            self._check(L.lbm_halo_pack(d.h, 1, b["hi_out"].data_ptr()))
        with torch.cuda.stream(self.stream):
            if self._dev == "cpu":
                m["lo_out"].copy_(b["lo_out"])
                m["hi_out"].copy_(b["hi_out"])
                self.stream.synchronize()
            exchange_with_neighbours(self.rank, self.world, m["lo_out"], m["hi_out"], m["lo_in"],
                                     m["hi_in"], self.group)
            if self._dev == "cpu":
                b["lo_in"].copy_(m["lo_in"])
                b["hi_in"].copy_(m["hi_in"])
        if lo:
            self._check(L.lbm_halo_unpack(d.h, 0, b["lo_in"].data_ptr()))
        if hi:
            self._check(L.lbm_halo_unpack(d.h, 1, b["hi_in"].data_ptr()))

    def reset(self):
        self.d.reset()
        self.exchange()

    def step(self, n: int = 1):
        for _ in range(int(n)):
            self.d.step(1)
            self.exchange()
        return self

    def current_density(self):
        """(i_avg, heat) of the whole lattice: the slabs' width-weighted
        sums, added over the ranks."""
        import torch
        import torch.distributed as dist
        i, h, _ = self.d.current_density(profile=False)
        w = self.ranges[self.rank][1] - self.ranges[self.rank][0]
        t = torch.tensor([i * w, h * w], dtype=torch.float64, device=self._dev)
        dist.all_reduce(t, group=self.group)
        return float(t[0]) / self.nx, float(t[1]) / self.nx

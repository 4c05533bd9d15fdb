"""Domain decomposition of a periodic grid over ranks (one subdomain per GPU).

The paper runs one subdomain per GPU and exchanges the halo cells around each
rank's subdomain once per step, after Step 10 (Sec. 2.2, Step 10; Sec. 3.2);
the CFL time step is the minimum over ranks (Step 1).  Here:

* ``plan`` splits a global grid into ``parts`` = (px, py, pz) boxes of near
  equal size and gives each rank its offset, size and periodic neighbours;
* ``Subdomain`` holds one rank's interior block and builds its
  halo-extended block (``HALO`` cells more per side along decomposed axes)
  by exchanging slabs with the neighbours, one axis after the other (x, y,
  z), each slab carrying the halos of the axes already done so that edges
  and corners arrive too;
* ``step`` exchanges the halo, takes the global dt (all-reduce MIN of the
  ranks' CFL dt unless a dt is given) and advances the interior with a step
  function on the halo-extended block: the library's ``mhd_step_sub`` on
  GPUs, any function with the same contract elsewhere.

Communication goes through ``torch.distributed`` point-to-point calls (NCCL
for CUDA tensors, gloo for CPU tensors).  Nothing here does arithmetic on the
state: slabs are copied, never combined.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

HALO = 8  # halo cells per side: the library's ghost depth (> one step's 5-cell stencil reach)


@dataclass
class Part:
    rank: int
    coords: tuple  # (cx, cy, cz) in the process grid
    offset: tuple  # first global cell (ox, oy, oz)
    size: tuple    # cells (nx, ny, nz)
    lo: tuple      # neighbour rank below along x, y, z (periodic)
    hi: tuple      # neighbour rank above along x, y, z


def _split(n: int, p: int):
    base, extra = divmod(n, p)
    sizes = [base + (1 if i < extra else 0) for i in range(p)]
    offs = [sum(sizes[:i]) for i in range(p)]
    return offs, sizes


def plan(global_n, parts):
    """Boxes of the ranks, rank = cx + px (cy + py cz).  global_n = (nx, ny, nz)."""
    px, py, pz = parts
    splits = [_split(global_n[a], parts[a]) for a in range(3)]
    for a in range(3):
        if parts[a] > 1 and min(splits[a][1]) < HALO:
            raise ValueError(f"axis {a}: subdomains of {min(splits[a][1])} cells are thinner than the halo ({HALO})")

    def rank_of(cx, cy, cz):
        return (cx % px) + px * ((cy % py) + py * (cz % pz))

    out = []
    for cz in range(pz):
        for cy in range(py):
            for cx in range(px):
                c = (cx, cy, cz)
                lo = tuple(rank_of(*[c[b] - (1 if b == a else 0) for b in range(3)]) for a in range(3))
                hi = tuple(rank_of(*[c[b] + (1 if b == a else 0) for b in range(3)]) for a in range(3))
                out.append(Part(rank_of(cx, cy, cz), c, tuple(splits[a][0][c[a]] for a in range(3)),
                                tuple(splits[a][1][c[a]] for a in range(3)), lo, hi))
    return out


class Subdomain:
    """One rank's share of the global state.

    interior: tensor [8, nz, ny, nx] of this rank's cells.  ``halo[a]`` is
    HALO on decomposed axes (parts[a] > 1), else 0 (the step wraps those axes
    itself)."""

    def __init__(self, part: Part, parts, interior: torch.Tensor, group=None):
        self.part = part
        self.parts = parts
        self.group = group
        self.halo = tuple(HALO if parts[a] > 1 else 0 for a in range(3))
        self.interior = interior.contiguous()
        nx, ny, nz = part.size
        hx, hy, hz = self.halo
        self.ext = torch.empty((8, nz + 2 * hz, ny + 2 * hy, nx + 2 * hx), dtype=interior.dtype,
                               device=interior.device)
        self.out = torch.empty_like(self.ext)

    # array axis of the state tensor for grid axis a (x, y, z)
    @staticmethod
    def _dim(a):
        return 3 - a

    def _slab(self, t, a, start, width):
        return t.narrow(self._dim(a), start, width)

    def exchange(self):
        """Fills ``ext``: the interior in the middle, the halo from the
        neighbours (axis by axis, so edges and corners come along)."""
        import torch.distributed as dist
        nx, ny, nz = self.part.size
        hx, hy, hz = self.halo
        self.ext[:, hz:hz + nz, hy:hy + ny, hx:hx + nx] = self.interior
        for a in range(3):
            h = self.halo[a]
            if h == 0:
                continue
            n = self.part.size[a]
            # the slabs span the full extent of the axes already exchanged and
            # the interior extent of the ones still to do
            view = self.ext
            for b in range(a + 1, 3):
                if self.halo[b]:
                    view = view.narrow(self._dim(b), self.halo[b], self.part.size[b])
            send_lo = self._slab(view, a, h, h).contiguous()          # my first h cells -> lower neighbour
            send_hi = self._slab(view, a, n, h).contiguous()          # my last h cells -> upper neighbour
            recv_lo = torch.empty_like(send_lo)                       # from lower neighbour: its last h
            recv_hi = torch.empty_like(send_hi)                       # from upper neighbour: its first h
            reqs = [dist.isend(send_lo, self.part.lo[a], group=self.group, tag=2 * a),
                    dist.isend(send_hi, self.part.hi[a], group=self.group, tag=2 * a + 1),
                    dist.irecv(recv_lo, self.part.lo[a], group=self.group, tag=2 * a + 1),
                    dist.irecv(recv_hi, self.part.hi[a], group=self.group, tag=2 * a)]
            for r in reqs:
                r.wait()
            self._slab(view, a, 0, h).copy_(recv_lo)
            self._slab(view, a, n + h, h).copy_(recv_hi)

    def step(self, step_fn, dt=None, dt_fn=None):
        """One step: halo exchange, global dt (MIN over ranks of dt_fn(ext,
        halo) unless dt is given), then step_fn(ext, halo, dt, out) writes
        the new interior into ``out``.  Returns the dt used."""
        import torch.distributed as dist
        self.exchange()
        if dt is None:
            d = torch.tensor([float(dt_fn(self.ext, self.halo))], dtype=torch.float64, device=self.ext.device)
            dist.all_reduce(d, op=dist.ReduceOp.MIN, group=self.group)
            dt = float(d.item())
        step_fn(self.ext, self.halo, dt, self.out)
        nx, ny, nz = self.part.size
        hx, hy, hz = self.halo
        self.interior = self.out[:, hz:hz + nz, hy:hy + ny, hx:hx + nx].contiguous()
        return dt


def library_fns(mhd, sim):
    """(step_fn, dt_fn) on GPUs: ``sim`` is a Sim of the subdomain's size
    with bc "halo" on its decomposed axes."""
    def step_fn(ext, halo, dt, out):
        mhd.mhd_step_sub(sim.ctx, ext, halo, dt, out)

    def dt_fn(ext, halo):
        return mhd.mhd_dt_sub(sim.ctx, ext, halo)
    return step_fn, dt_fn

"""Z-slab decomposition of one lattice, with the halo exchange between slabs.

The lattice is cut along z, the slowest axis of the state layout, into slabs
of whole z planes.  Each slab is a librlb context (``zbc="halo"``) that holds
its own planes plus one halo plane below and one above.  A step updates the
slab's own planes only; then every halo plane is refilled from its
neighbour: the 5 f and 5 g populations with e_z = +1 of a slab's top plane go
to the lower halo plane of the slab above, the 10 with e_z = -1 of its bottom
plane to the upper halo plane of the slab below.  These are exactly the
values that the next pull-streaming step reads across the two faces (in Eqs.
lbe1/lbe2 a population moves one cell along e_i per step), so the slabs
together compute the same step as one context holding the whole lattice,
value for value.  z is periodic: the slabs form a ring.

* ``SlabLattice`` -- every slab on one device; the exchange is
  ``rlb_halo_exchange`` (one kernel per slab pair).
* ``exchange_halo`` / ``DistributedSlab`` -- one slab per rank (one GPU per
  process); the faces travel by torch.distributed point-to-point messages
  (NCCL between GPUs; gloo in the CPU tests of the exchange schedule).

Only the data movement lives here; every arithmetic step of the method runs
in the library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _native as N
from .rlb import RLB

# e_z of the D3Q19 velocities in the plane order of a state (include/rlb.h)
_EZ = (0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1)
# population planes (f then g) crossing a z face upwards / downwards
UP_PLANES = tuple(s * 19 + i for s in (0, 1) for i in range(19) if _EZ[i] == 1)
DOWN_PLANES = tuple(s * 19 + i for s in (0, 1) for i in range(19) if _EZ[i] == -1)


def split_z(nz: int, parts: int):
    """Bounds [(z0, z1), ...] of `parts` slabs of whole planes, sizes differing
    by at most one plane."""
    if not 1 <= parts <= nz:
        raise ValueError(f"cannot cut {nz} planes into {parts} slabs")
    edges = [round(k * nz / parts) for k in range(parts + 1)]
    return [(edges[k], edges[k + 1]) for k in range(parts)]


def slab_planes(z0: int, z1: int, nz: int):
    """Global z indices of a slab's planes, its two halo planes included
    (z0 - 1 and z1, periodic in z)."""
    return [(z % nz) for z in range(z0 - 1, z1 + 1)]


class SlabLattice:
    """One lattice as z slabs on one device.  Same interface as ``RLB`` for
    the forward path: ``init_fields``, ``step``, ``macro``, ``stats``."""

    def __init__(self, nx, ny, nz, tau, nslabs=2, bounds=None, **kw):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.bounds = list(bounds) if bounds is not None else split_z(self.nz, nslabs)
        if self.bounds[0][0] != 0 or self.bounds[-1][1] != self.nz or any(
                a[1] != b[0] for a, b in zip(self.bounds, self.bounds[1:])):
            raise ValueError(f"slab bounds {self.bounds} do not tile 0..{self.nz}")
        self.slabs = [RLB(nx, ny, z1 - z0 + 2, tau, zbc="halo", **kw) for z0, z1 in self.bounds]

    @classmethod
    def from_workload(cls, w, precision="fp64", nslabs=2, bounds=None, device=None, **kw):
        """Slabs of a ``workloads.Workload``, with the FP32 reference of the
        whole lattice (every slab stores deviations from the same one)."""
        m = np.ones(w.eps.shape, bool) if w.solid is None else (w.solid == 0)
        n_ref = kw.pop("n_ref", None) or RLB.reference_value(np.append(w.n[m], w.n_in))
        eps_ref = kw.pop("eps_ref", None) or RLB.reference_value(np.append(w.eps[m], w.eps_in))
        xbc = {0: "periodic", 1: "inflow_outflow", 2: "outflow_both"}[w.xbc]
        return cls(w.nx, w.ny, w.nz, w.tau, nslabs=nslabs, bounds=bounds, c_l=w.c_l, precision=precision, xbc=xbc,
                   n_in=w.n_in, eps_in=w.eps_in, beta_in=w.beta_in, n_ref=n_ref, eps_ref=eps_ref, device=device, **kw)

    def init_fields(self, n, eps, beta, solid=None):
        """Host fields of the whole lattice: n, eps (nz, ny, nx), beta (3, nz,
        ny, nx), solid (nz, ny, nx) or None.  Every slab starts from its own
        planes and copies of its neighbours' edge planes."""
        for (z0, z1), s in zip(self.bounds, self.slabs):
            zz = slab_planes(z0, z1, self.nz)
            s.init_fields(np.ascontiguousarray(n[zz]), np.ascontiguousarray(eps[zz]),
                          np.ascontiguousarray(beta[:, zz]), None if solid is None else np.ascontiguousarray(solid[zz]))
        return self

    def exchange(self):
        """Refill every halo plane from the slab's neighbours (a ring in z)."""
        K = len(self.slabs)
        for k in range(K):
            N.rlb_halo_exchange(self.slabs[k].ctx, self.slabs[(k + 1) % K].ctx)

    def step(self, nsteps: int = 1):
        for _ in range(int(nsteps)):
            for s in self.slabs:
                s.step(1)
            self.exchange()
        return self

    def macro(self, where: str = "host"):
        """(n, eps, beta, ok) of the whole lattice from the slabs' own planes."""
        parts = [s.macro(where=where) for s in self.slabs]
        cat = np.concatenate if where == "host" else torch.cat
        n = cat([p[0][1:-1] for p in parts], 0)
        e = cat([p[1][1:-1] for p in parts], 0)
        b = cat([p[2][:, 1:-1] for p in parts], 1)
        return n, e, b, all(p[3] for p in parts)

    def stats(self) -> dict:
        st = [s.stats() for s in self.slabs]
        return {"steps": st[0]["steps"], "n_unphysical": sum(x["n_unphysical"] for x in st),
                "n_nonpositive_eq": sum(x["n_nonpositive_eq"] for x in st)}

    def sync(self):
        for s in self.slabs:
            s.sync()

    def close(self):
        for s in self.slabs:
            s.close()


def exchange_halo(state: torch.Tensor, nx: int, ny: int, nz_local: int, group=None) -> None:
    """Halo exchange of this rank's slab with its two neighbours in a ring of
    ranks ordered by z (rank r + 1 holds the slab above rank r's; the last
    rank's upper neighbour is rank 0).  `state` is the slab's (38, S) state
    (nz_local planes, the two halo planes included).  The ten upward
    populations of plane nz_local - 2 go up into the neighbour's plane 0; the
    ten downward ones of plane 1 go down into the neighbour's plane
    nz_local - 1.  Each direction is one packed message per neighbour."""
    import torch.distributed as dist

    nxy = nx * ny
    top, bottom = (nz_local - 2) * nxy, nxy
    lo_halo, hi_halo = 0, (nz_local - 1) * nxy
    up_src = torch.stack([state[q, top:top + nxy] for q in UP_PLANES])
    down_src = torch.stack([state[q, bottom:bottom + nxy] for q in DOWN_PLANES])
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    if world == 1:
        from_below, from_above = up_src, down_src
    else:
        rank = dist.get_rank(group)
        above, below = (rank + 1) % world, (rank - 1) % world
        if group is not None:
            above = dist.get_global_rank(group, above)
            below = dist.get_global_rank(group, below)
        from_below = torch.empty_like(up_src)
        from_above = torch.empty_like(down_src)
        ops = [dist.P2POp(dist.isend, up_src, above, group, tag=1),
               dist.P2POp(dist.irecv, from_below, below, group, tag=1),
               dist.P2POp(dist.isend, down_src, below, group, tag=2),
               dist.P2POp(dist.irecv, from_above, above, group, tag=2)]
        for r in dist.batch_isend_irecv(ops):
            r.wait()
    for k, q in enumerate(UP_PLANES):
        state[q, lo_halo:lo_halo + nxy] = from_below[k]
    for k, q in enumerate(DOWN_PLANES):
        state[q, hi_halo:hi_halo + nxy] = from_above[k]


class DistributedSlab:
    """This rank's z slab of a lattice cut over the ranks of a process group
    (one GPU per process).  Forward path only; the exchange after every step
    is ``exchange_halo``."""

    def __init__(self, w, precision="fp64", group=None, device=None, **kw):
        import torch.distributed as dist

        world = dist.get_world_size(group) if dist.is_initialized() else 1
        rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.group = group
        self.bounds = split_z(w.nz, world)[rank]
        self.nx, self.ny = w.nx, w.ny
        z0, z1 = self.bounds
        self.nz_local = z1 - z0 + 2
        m = np.ones(w.eps.shape, bool) if w.solid is None else (w.solid == 0)
        n_ref = RLB.reference_value(np.append(w.n[m], w.n_in))
        eps_ref = RLB.reference_value(np.append(w.eps[m], w.eps_in))
        xbc = {0: "periodic", 1: "inflow_outflow", 2: "outflow_both"}[w.xbc]
        self.slab = RLB(w.nx, w.ny, self.nz_local, w.tau, c_l=w.c_l, precision=precision, xbc=xbc, n_in=w.n_in,
                        eps_in=w.eps_in, beta_in=w.beta_in, n_ref=n_ref, eps_ref=eps_ref, device=device, zbc="halo",
                        **kw)
        zz = slab_planes(z0, z1, w.nz)
        self.slab.init_fields(np.ascontiguousarray(w.n[zz]), np.ascontiguousarray(w.eps[zz]),
                              np.ascontiguousarray(w.beta[:, zz]),
                              None if w.solid is None else np.ascontiguousarray(w.solid[zz]))

    def step(self, nsteps: int = 1):
        for _ in range(int(nsteps)):
            self.slab.step(1)
            exchange_halo(self.slab.state(), self.nx, self.ny, self.nz_local, self.group)
        return self

    def macro(self, where: str = "host"):
        """(n, eps, beta, ok) of this rank's own planes."""
        n, e, b, ok = self.slab.macro(where=where)
        return n[1:-1], e[1:-1], b[:, 1:-1], ok

    def close(self):
        self.slab.close()

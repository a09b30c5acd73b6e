"""x-slab decomposition of one state solve across ranks (one GPU per rank).

The structured grid is cut along x: rank r owns the node planes
i in [i0, i1) (the last rank also owns i = nx) and keeps one ghost node
plane on each side it shares with a neighbour.  To form (K u) on its owned
nodes a rank needs every element that touches them, i.e. the element layers
[i0 - 1, i1) (one ghost element layer on its -x side), and therefore u on the
node planes [i0 - 1, i1]: one halo exchange per operator application, each
rank sending its first owned plane to the left neighbour and its last owned
plane to the right one, (ny+1)(nz+1) x 3 values each way.  A CG iteration
adds two FP64 scalar all-reduces (p.Ap, and r.z with r.r in one call); the
Jacobi diagonal needs no communication (the ghost element layer is local).
Densities, moduli and the load are each rank's slab of the global arrays,
read once at set-up.

Multigrid levels coarsen 2:1 in x as well; a level whose node count falls
below `gather_below` is gathered whole onto every rank (one all-gather of its
slabs) and solved redundantly, then each rank keeps its own slab of the
result.

This module is the host side of the decomposition: partitions, halo
exchange and the all-reduces over torch.distributed (NCCL on GPUs, gloo on
CPUs), and a Jacobi-preconditioned CG driver that takes the local operator
as a callable: apply_local(u_ext) -> y on the owned nodes, u_ext holding the
ghost planes.  The per-rank operator on the device is the library's FP32 or
FP64 operator restricted to the slab; that kernel wiring and any
measurement on several GPUs are not built here (every box this runs on has
one GPU).

Array layout per rank: (planes, nz+1, ny+1, 3), x outermost: node (i, j, k)
component c of the global grid at [i - lo, k, j, c].  `Slab.to_local` and
`Slab.from_local` convert to and from the library's DOF order
(3 n + c, n = i + (nx+1)(j + (ny+1) k)).
"""
from __future__ import annotations

import dataclasses

import numpy as np


def split_planes(n_planes: int, world: int) -> list[tuple[int, int]]:
    """Balanced contiguous ranges [a, b) of n_planes node planes over `world`
    ranks (the first n_planes % world ranks get one more)."""
    if world < 1 or n_planes < world:
        raise ValueError(f"cannot split {n_planes} planes over {world} ranks")
    q, r = divmod(n_planes, world)
    out, a = [], 0
    for rank in range(world):
        b = a + q + (1 if rank < r else 0)
        out.append((a, b))
        a = b
    return out


@dataclasses.dataclass(frozen=True)
class Slab:
    """Rank `rank`'s part of an nx x ny x nz element grid split along x.

    i0, i1      owned node planes [i0, i1)
    lo, hi      node planes held locally [lo, hi] (owned plus ghosts):
                lo = max(i0 - 1, 0), hi = min(i1, nx)
    e_lo, e_hi  element layers held locally [e_lo, e_hi) = [lo, hi)
    """
    nx: int
    ny: int
    nz: int
    world: int
    rank: int
    i0: int
    i1: int

    @staticmethod
    def make(nx: int, ny: int, nz: int, world: int, rank: int) -> "Slab":
        i0, i1 = split_planes(nx + 1, world)[rank]
        return Slab(nx, ny, nz, world, rank, i0, i1)

    @property
    def lo(self) -> int:
        return max(self.i0 - 1, 0)

    @property
    def hi(self) -> int:
        return min(self.i1, self.nx)

    @property
    def e_lo(self) -> int:
        return self.lo

    @property
    def e_hi(self) -> int:
        return self.hi

    @property
    def plane_nodes(self) -> int:
        return (self.ny + 1) * (self.nz + 1)

    @property
    def n_local_planes(self) -> int:
        return self.hi - self.lo + 1

    @property
    def owned(self) -> slice:
        """Owned planes as a slice of the local planes."""
        return slice(self.i0 - self.lo, self.i1 - self.lo)

    @property
    def left(self) -> int | None:
        return self.rank - 1 if self.rank > 0 else None

    @property
    def right(self) -> int | None:
        return self.rank + 1 if self.rank < self.world - 1 else None

    # ---- conversions between the global DOF order and local planes ------
    def to_local(self, v_global: np.ndarray) -> np.ndarray:
        """(planes, nz+1, ny+1, 3) array of the local planes [lo, hi] of a
        global DOF vector (3 n + c, n = i + (nx+1)(j + (ny+1) k))."""
        g = np.asarray(v_global).reshape(self.nz + 1, self.ny + 1, self.nx + 1, 3)
        return np.ascontiguousarray(g[:, :, self.lo:self.hi + 1, :].transpose(2, 0, 1, 3))

    def from_local(self, v_local: np.ndarray, out: np.ndarray | None = None,
                   owned_only: bool = True) -> np.ndarray:
        """Scatter local planes (owned ones, or all) into a global DOF vector."""
        if out is None:
            out = np.zeros(3 * (self.nx + 1) * self.plane_nodes)
        g = out.reshape(self.nz + 1, self.ny + 1, self.nx + 1, 3)
        src = np.asarray(v_local).transpose(1, 2, 0, 3)
        if owned_only:
            g[:, :, self.i0:self.i1, :] = src[:, :, self.owned, :]
        else:
            g[:, :, self.lo:self.hi + 1, :] = src
        return out

    def local_elements(self, e_global: np.ndarray) -> np.ndarray:
        """The element layers [e_lo, e_hi) of a global element array (element
        e = i + nx (j + ny k)) in the local element order."""
        g = np.asarray(e_global).reshape(self.nz, self.ny, self.nx)
        return np.ascontiguousarray(g[:, :, self.e_lo:self.e_hi]).reshape(-1)


class Comm:
    """Halo exchange and reductions of one slab over torch.distributed (the
    default process group); tensors are CPU (gloo) or CUDA (NCCL) torch
    tensors of FP64 values."""

    def __init__(self, slab: Slab, device: str = "cpu"):
        import torch
        import torch.distributed as dist
        self.slab, self.dist, self.torch, self.device = slab, dist, torch, device

    def exchange(self, u_local: np.ndarray) -> np.ndarray:
        """Fill the ghost planes of u_local (planes, nz+1, ny+1, 3) from the
        neighbours' owned planes: send the first owned plane left and the last
        owned plane right, receive the ghosts.  Returns u_local."""
        s, dist, torch = self.slab, self.dist, self.torch
        reqs, recv = [], {}
        o = s.owned
        if s.left is not None:
            first = torch.from_numpy(np.ascontiguousarray(u_local[o.start])).to(self.device)
            reqs.append(dist.isend(first, s.left))
            recv["left"] = torch.empty_like(first)
            reqs.append(dist.irecv(recv["left"], s.left))
        if s.right is not None:
            last = torch.from_numpy(np.ascontiguousarray(u_local[o.stop - 1])).to(self.device)
            reqs.append(dist.isend(last, s.right))
            recv["right"] = torch.empty_like(last)
            reqs.append(dist.irecv(recv["right"], s.right))
        for r in reqs:
            r.wait()
        if "left" in recv:
            u_local[0] = recv["left"].cpu().numpy()
        if "right" in recv:
            u_local[-1] = recv["right"].cpu().numpy()
        return u_local

    def allreduce(self, values) -> np.ndarray:
        """Sum of FP64 scalars over the ranks (one all-reduce for all of them)."""
        t = self.torch.tensor(np.asarray(values, dtype=np.float64), device=self.device)
        self.dist.all_reduce(t)
        return t.cpu().numpy()

    def allgather_planes(self, v_owned: np.ndarray, n_planes_total: int) -> np.ndarray:
        """Every rank's owned planes, concatenated in x order (the gather of a
        coarse multigrid level).  Ranks may own one plane more than others:
        the slabs travel padded to the longest and are trimmed after."""
        dist, torch, s = self.dist, self.torch, self.slab
        ranges = split_planes(n_planes_total, s.world)
        width = max(b - a for a, b in ranges)
        mine = np.zeros((width,) + v_owned.shape[1:])
        mine[:len(v_owned)] = v_owned
        parts = [torch.empty(mine.shape, dtype=torch.float64, device=self.device)
                 for _ in ranges]
        dist.all_gather(parts, torch.from_numpy(mine).to(self.device))
        return np.concatenate([p.cpu().numpy()[:b - a] for p, (a, b) in zip(parts, ranges)],
                              axis=0)


class LocalComm:
    """The same interface for one rank holding the whole grid (no messages)."""

    def __init__(self, slab: Slab):
        if slab.world != 1:
            raise ValueError("LocalComm is the one-rank case")
        self.slab = slab

    def exchange(self, u_local):
        return u_local

    def allreduce(self, values):
        return np.asarray(values, dtype=np.float64)

    def allgather_planes(self, v_owned, n_planes_total):
        return v_owned


def coarse_slabs(nx: int, ny: int, nz: int, world: int, levels: int,
                 gather_below: int = 4096) -> list[dict]:
    """Per multigrid level (2:1 vertex-nested coarsening, odd counts rounded
    up as in the library's hierarchy): its grid, and either this level's
    split over the ranks or 'gathered' when it has fewer than gather_below
    nodes or fewer node planes than ranks."""
    out = []
    gx, gy, gz = nx, ny, nz
    for lev in range(levels):
        nodes = (gx + 1) * (gy + 1) * (gz + 1)
        gathered = nodes < gather_below or gx + 1 < world
        out.append({"level": lev, "grid": (gx, gy, gz), "nodes": nodes, "gathered": gathered,
                    "split": None if gathered else split_planes(gx + 1, world)})
        gx, gy, gz = (gx + 1) // 2, (gy + 1) // 2, (gz + 1) // 2
    return out


def jacobi_pcg(slab: Slab, comm, apply_local, dinv_local: np.ndarray, f_local: np.ndarray,
               fixed_local: np.ndarray, rtol: float = 1e-8, maxiter: int = 100000,
               record: list | None = None):
    """Jacobi-preconditioned CG on the owned DOFs of this rank.

    apply_local(u_local) -> (K u) on the local planes, correct on the owned
    ones (u_local's ghost planes already exchanged).  dinv_local, f_local,
    fixed_local: local-plane arrays (planes, nz+1, ny+1, 3); fixed DOFs hold 0.
    Each iteration: one halo exchange (in the operator application), one
    all-reduce of p.Ap, one of (r.z, r.r).  `record` (optional) receives
    the owned part of every iterate x_k.  Returns (x_local, iterations,
    relative recursive residual)."""
    o = slab.owned
    free = ~fixed_local
    x = np.zeros_like(f_local)
    r = np.where(free, f_local, 0.0)
    z = dinv_local * r
    p = z.copy()
    rz, rr, ff = comm.allreduce([np.sum(r[o] * z[o]), np.sum(r[o] * r[o]),
                                 np.sum(f_local[o] * f_local[o] * free[o])])
    fn = np.sqrt(ff)
    it = 0
    while it < maxiter and np.sqrt(rr) > rtol * fn:
        comm.exchange(p)
        q = np.where(free, apply_local(p), 0.0)
        (pq,) = comm.allreduce([np.sum(p[o] * q[o])])
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        z = dinv_local * r
        rz_new, rr = comm.allreduce([np.sum(r[o] * z[o]), np.sum(r[o] * r[o])])
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
        if record is not None:
            record.append(x[o].copy())
    return x, it, float(np.sqrt(rr) / fn) if fn > 0 else 0.0


class DeviceSlabOperator:
    """The library's operator on one rank's slab: a mesh of the slab's element
    layers [e_lo, e_hi) with no support (TOPO_BC_NONE; the decomposition
    applies the global supports), whose densities are the slab of the global
    densities (Eq. (1) on the device).  apply_local(u) gives K u on the local
    planes (correct on the owned ones once the ghosts are exchanged);
    dinv_local() the Jacobi inverse on the local planes (exact on the owned
    ones: every element around an owned node is held).  precision:
    topo.PREC_FP64 or topo.PREC_FP32 (the operator kernels of the library)."""

    def __init__(self, slab: Slab, rho_global: np.ndarray, precision: int = 0, params=None,
                 stream=None):
        from . import topo
        self.slab, self.precision, self.topo = slab, precision, topo
        self.mesh = topo.Mesh(slab.e_hi - slab.e_lo, slab.ny, slab.nz, topo.BC_NONE,
                              topo.LOAD_EDGE_XL_BOTTOM, params=params, stream=stream)
        self.mesh.set_density(np.ascontiguousarray(slab.local_elements(rho_global),
                                                   dtype=np.float32))
        self.shape = (slab.n_local_planes, slab.nz + 1, slab.ny + 1, 3)

    def _to_mesh(self, v_local):
        return np.ascontiguousarray(np.asarray(v_local).transpose(1, 2, 0, 3)).reshape(-1)

    def _from_mesh(self, flat):
        s = self.slab
        return np.ascontiguousarray(flat.reshape(s.nz + 1, s.ny + 1, s.n_local_planes, 3)
                                    .transpose(2, 0, 1, 3))

    def apply_local(self, u_local: np.ndarray) -> np.ndarray:
        y = self.mesh.apply(self._to_mesh(u_local), precision=self.precision)
        return self._from_mesh(y)

    def dinv_local(self) -> np.ndarray:
        return self._from_mesh(self.mesh.jacobi_inverse())

    def close(self):
        self.mesh.close()

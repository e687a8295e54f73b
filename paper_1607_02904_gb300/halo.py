"""Spatial decomposition of one periodic cell over ranks, with a ghost (halo)
exchange: the data-parallel layout of the paper's MPI runs (Sec. V, strong
scaling over nodes), one process per GPU.

The cell is cut into slabs along one axis. Each rank owns the atoms whose
wrapped coordinate lies in its slab and receives, in one exchange step per
direction, the atoms within ``r_ghost`` of its two faces from the neighbouring
ranks (shifted by the box length across the periodic boundary). With
``r_ghost = 2 r_c`` (owner computes) every term of Eq. 5-7 that touches an
owned atom is complete on its rank: a term centred on atom i involves
neighbours j, k within r_c of i, so if any of i, j, k is owned, all three lie
within 2 r_c of the slab. Each rank therefore evaluates its local system
(owned atoms first, then ghosts) and keeps the forces and per-centre energies
of its owned atoms; there is no reverse (force) exchange. The total energy is
the sum over ranks of the owned atoms' per-centre energies.

The local system is periodic in the two other axes and padded along the cut
axis, so that no periodic image couples its two faces. Host logic only: the
evaluation itself is a callback (the CUDA library on a GPU).
"""
from __future__ import annotations

import numpy as np


class SlabDecomposition:
    """Slabs of equal width along ``axis`` (default: the longest box edge).

    box: the three periodic edges; world: number of ranks; r_cut: the largest
    cutoff of the potential (R + D); r_list: the neighbour-list radius the
    callback will use (cutoff plus skin). Requires every slab to be at least
    ``r_ghost = 2 r_cut`` wide, so that ghosts come from the two adjacent ranks
    only.
    """

    def __init__(self, box, world: int, r_cut: float, r_list: float | None = None, axis=None):
        self.box = np.asarray(box, dtype=np.float64).copy()
        if self.box.shape != (3,) or not np.all(self.box > 0):
            raise ValueError("box must hold three positive edges")
        if world < 1:
            raise ValueError("world must be >= 1")
        self.world = int(world)
        self.axis = int(np.argmax(self.box)) if axis is None else int(axis)
        self.r_cut = float(r_cut)
        self.r_list = float(r_list if r_list is not None else r_cut)
        self.r_ghost = 2.0 * self.r_cut
        self.width = self.box[self.axis] / self.world
        if self.world > 1 and self.width < self.r_ghost:
            raise ValueError(f"slab width {self.width:.3f} is below the ghost shell "
                             f"{self.r_ghost:.3f}: use fewer ranks")

    def bounds(self, rank: int):
        lo = rank * self.width
        return lo, lo + self.width

    def wrapped(self, x):
        """Coordinate along the cut axis, wrapped into [0, L)."""
        L = self.box[self.axis]
        u = np.mod(np.asarray(x, dtype=np.float64)[:, self.axis], L)
        return np.where(u >= L, u - L, u)

    def wrap(self, x):
        """Copy of x with the cut-axis coordinate wrapped into [0, L) (the
        other coordinates are left to the periodic evaluation)."""
        y = np.array(x, dtype=np.float64, copy=True).reshape(-1, 3)
        y[:, self.axis] = self.wrapped(y)
        return y

    def owner(self, x):
        """Rank owning each atom."""
        r = np.floor(self.wrapped(x) / self.width).astype(np.int64)
        return np.clip(r, 0, self.world - 1)

    def face_sets(self, x, rank: int):
        """Indices of rank's atoms (x: its owned atoms) within r_ghost of its
        lower and upper faces, and the shift along the axis each set takes at
        the receiver (+L when crossing below 0, -L above L, else 0)."""
        lo, hi = self.bounds(rank)
        u = self.wrapped(x)
        L = self.box[self.axis]
        lower = np.nonzero(u - lo < self.r_ghost)[0]
        upper = np.nonzero(hi - u <= self.r_ghost)[0]
        shift_lower = L if rank == 0 else 0.0              # to the rank below
        shift_upper = -L if rank == self.world - 1 else 0.0  # to the rank above
        return (lower, shift_lower), (upper, shift_upper)

    def local_box(self):
        """Box of a rank's local system: the periodic edges, and along the cut
        axis the slab, both ghost shells and a gap wider than the list radius
        (no image couples the two faces)."""
        b = self.box.copy()
        b[self.axis] = self.width + 2.0 * self.r_ghost + 1.05 * self.r_list
        b[self.axis] = max(b[self.axis], 2.0 * self.r_list)
        return b

    def to_local(self, x, rank: int):
        """Positions of owned atoms (wrapped) and ghosts (wrapped and shifted)
        in the local frame: along the cut axis offset so that the lower ghost
        shell starts at 0; the other coordinates unchanged."""
        lo, _ = self.bounds(rank)
        y = np.array(x, dtype=np.float64, copy=True)
        y[:, self.axis] -= lo - self.r_ghost
        return y


def _shifted(x, idx, axis, shift):
    y = np.array(x[idx], dtype=np.float64, copy=True)
    y[:, axis] += shift
    return y


def ghosts_from_global(dec: SlabDecomposition, x_all, types_all, rank: int):
    """The ghosts of ``rank`` taken directly from the whole system (what the
    exchange delivers; used to emulate ranks in one process and to check the
    exchange): atoms of the adjacent ranks (or, with one rank, periodic
    images of its own) within r_ghost of the rank's faces, shifted across the
    periodic boundary. Returns (positions, species, global indices)."""
    x_all = dec.wrap(x_all)
    own = dec.owner(x_all)
    xs, ts, ids = [], [], []
    world = dec.world
    for d in (-1, 1):
        src = (rank - d) % world  # the rank whose face set travels in direction d
        sel = np.nonzero(own == src)[0]
        (lower, sl), (upper, su) = dec.face_sets(x_all[sel], src)
        idx, shift = (upper, su) if d == 1 else (lower, sl)
        xs.append(_shifted(x_all[sel], idx, dec.axis, shift))
        ts.append(np.asarray(types_all)[sel][idx])
        ids.append(sel[idx])
    return np.concatenate(xs), np.concatenate(ts).astype(np.int32), np.concatenate(ids)


def halo_exchange(dec: SlabDecomposition, x_own, types_own, ids_own, rank: int, group=None):
    """One exchange step per direction over torch.distributed point-to-point
    messages: the upper face set goes to rank + 1 and the lower one to
    rank - 1 (periodic), each shifted across the boundary where it wraps.
    Counts travel first, then positions, species and global indices.
    Returns the ghosts (positions, species, global indices) in the order of
    ``ghosts_from_global``."""
    import torch
    import torch.distributed as dist
    world = dec.world
    x_own = dec.wrap(x_own)
    (lower, sl), (upper, su) = dec.face_sets(x_own, rank)
    if world == 1:  # periodic images of its own faces, no messages
        xs = [_shifted(x_own, lower, dec.axis, sl), _shifted(x_own, upper, dec.axis, su)]
        ts = [np.asarray(types_own)[lower], np.asarray(types_own)[upper]]
        ids = [np.asarray(ids_own)[lower], np.asarray(ids_own)[upper]]
        return np.concatenate(xs), np.concatenate(ts).astype(np.int32), np.concatenate(ids)
    out = {}
    # direction +1: upper face to rank + 1, receive from rank - 1 (and vice versa)
    for tag, (d, idx, shift) in enumerate(((1, upper, su), (-1, lower, sl))):
        dst, src = (rank + d) % world, (rank - d) % world
        send_x = torch.from_numpy(_shifted(x_own, idx, dec.axis, shift))
        send_t = torch.from_numpy(np.asarray(types_own, dtype=np.int64)[idx])
        send_i = torch.from_numpy(np.asarray(ids_own, dtype=np.int64)[idx])
        cnt_out = torch.tensor([len(idx)], dtype=torch.int64)
        cnt_in = torch.zeros(1, dtype=torch.int64)
        base = 8 * tag
        reqs = [dist.isend(cnt_out, dst, group=group, tag=base),
                dist.irecv(cnt_in, src, group=group, tag=base)]
        for r in reqs:
            r.wait()
        m = int(cnt_in.item())
        recv_x = torch.zeros((m, 3), dtype=torch.float64)
        recv_t = torch.zeros(m, dtype=torch.int64)
        recv_i = torch.zeros(m, dtype=torch.int64)
        reqs = []
        for k, (s, r_) in enumerate(((send_x, recv_x), (send_t, recv_t), (send_i, recv_i))):
            if len(idx):
                reqs.append(dist.isend(s.contiguous(), dst, group=group, tag=base + 1 + k))
            if m:
                reqs.append(dist.irecv(r_, src, group=group, tag=base + 1 + k))
        for r in reqs:
            r.wait()
        out[d] = (recv_x.numpy(), recv_t.numpy().astype(np.int32), recv_i.numpy())
    xs = [out[-1][0], out[1][0]]
    ts = [out[-1][1], out[1][1]]
    ids = [out[-1][2], out[1][2]]
    # order as ghosts_from_global: first the set travelling down (from rank + 1),
    # then the set travelling up (from rank - 1)
    return np.concatenate(xs), np.concatenate(ts).astype(np.int32), np.concatenate(ids)


def local_system(dec: SlabDecomposition, x_own, types_own, x_ghost, types_ghost, rank: int):
    """Owned atoms first, then ghosts, in the local frame and box."""
    x = np.concatenate([dec.wrap(x_own), np.asarray(x_ghost, dtype=np.float64).reshape(-1, 3)])
    t = np.concatenate([np.asarray(types_own), np.asarray(types_ghost)]).astype(np.int32)
    return dec.to_local(x, rank), t, dec.local_box()


def owned_energy_forces(dec: SlabDecomposition, x_own, types_own, x_ghost, types_ghost,
                        rank: int, compute):
    """Evaluates the local system with ``compute(x, types, box) -> (eatom,
    forces)`` and returns the owned atoms' energy (sum of their per-centre
    energies) and forces."""
    x, t, box = local_system(dec, x_own, types_own, x_ghost, types_ghost, rank)
    eatom, f = compute(x, t, box)
    n = len(x_own)
    return float(np.sum(np.asarray(eatom)[:n])), np.asarray(f)[:n]


def distributed_energy_forces(dec: SlabDecomposition, x_own, types_own, ids_own, rank: int,
                              compute, group=None):
    """Halo exchange, local evaluation, and the sum of the energy over ranks
    (one all-reduce of a scalar). Returns (total energy, owned forces)."""
    xg, tg, _ = halo_exchange(dec, x_own, types_own, ids_own, rank, group)
    e, f = owned_energy_forces(dec, x_own, types_own, xg, tg, rank, compute)
    if dec.world > 1:
        import torch
        import torch.distributed as dist
        et = torch.tensor([e], dtype=torch.float64)
        dist.all_reduce(et, group=group)
        e = float(et.item())
    return e, f


class LibraryCompute:
    """The callback for a GPU: one library context, rebuilt for each local
    system (its atom count changes from call to call)."""

    def __init__(self, table, r_list: float, precision=None, device="cuda"):
        import torch
        from ._lib import FP64, Context
        self.torch = torch
        self.ctx = Context(FP64 if precision is None else precision)
        self.ctx.params(np.asarray(table, dtype=np.float64))
        self.r_list = float(r_list)
        self.device = device

    def __call__(self, x, t, box):
        torch = self.torch
        xd = torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=self.device)
        td = torch.tensor(np.ascontiguousarray(t), dtype=torch.int32, device=self.device)
        self.ctx.neighbor_build(xd, td, box, self.r_list)
        f = torch.zeros_like(xd)
        ea = torch.zeros(xd.shape[0], dtype=torch.float64, device=self.device)
        self.ctx.compute(xd, None, f)
        self.ctx.compute_peratom(xd, ea)
        return ea.cpu().numpy(), f.cpu().numpy()

    def close(self):
        self.ctx.close()

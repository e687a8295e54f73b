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


def pack_geometry(dec: SlabDecomposition, rank: int):
    """The 9 values that tersoff_halo_pack takes for ``rank``: the box edge
    along the cut axis, the slab [lo, hi), the ghost width, the rank's frame
    origin (lo - r_ghost: ``to_local``), and for the lower and upper face sets
    the periodic shift each takes (as in ``face_sets``) and the frame origin
    of the neighbour that receives it."""
    L = float(dec.box[dec.axis])
    lo, hi = dec.bounds(rank)
    rg = dec.r_ghost
    world = dec.world
    frame = lo - rg
    shift_lower = L if rank == 0 else 0.0
    shift_upper = -L if rank == world - 1 else 0.0
    frame_lower = dec.bounds((rank - 1) % world)[0] - rg
    frame_upper = dec.bounds((rank + 1) % world)[0] - rg
    return [L, lo, hi, rg, frame, shift_lower, frame_lower, shift_upper, frame_upper]


def device_pack(ctx):
    """The face-set packing of ``halo_exchange_device`` on the GPU: one call
    of tersoff_halo_pack through ``ctx`` (a library Context). Returns
    (x_local, send_x, send_t, send_id, counts on the host)."""
    import torch

    def pack(dec, x_own, types_own, ids_own, rank):
        n = x_own.shape[0]
        cap = max(n, 1)
        dev = x_own.device
        x_local = torch.empty((n, 3), dtype=torch.float64, device=dev)
        send_x = torch.empty((2, cap, 3), dtype=torch.float64, device=dev)
        send_t = torch.empty((2, cap), dtype=torch.int32, device=dev)
        send_id = torch.empty((2, cap), dtype=torch.int64, device=dev)
        counts = torch.zeros(2, dtype=torch.int32, device=dev)
        ctx.halo_pack(x_own, types_own, ids_own, dec.axis, pack_geometry(dec, rank), cap,
                      x_local, send_x, send_t, send_id, counts)
        return x_local, send_x, send_t, send_id, [int(v) for v in counts.cpu()]

    return pack


def halo_exchange_device(dec: SlabDecomposition, x_own, types_own, ids_own, rank: int, pack,
                         group=None):
    """The halo exchange on device buffers. ``pack`` (``device_pack(ctx)`` on
    a GPU) writes the rank's owned atoms in its local frame and its two face
    sets, already in the receivers' frames; the upper set goes to rank + 1 and
    the lower set to rank - 1 (periodic) over torch.distributed point-to-point
    messages (NCCL between GPUs), counts first, and the received sets land
    after the owned atoms: first the set travelling down (from rank + 1), then
    the set travelling up (from rank - 1), the order of ``ghosts_from_global``.
    Returns the local system (positions, species, global indices; owned atoms
    first) on the device of x_own, and the owned count."""
    import torch
    import torch.distributed as dist
    n = x_own.shape[0]
    x_local, send_x, send_t, send_id, cnt = pack(dec, x_own, types_own, ids_own, rank)
    dev = x_own.device
    world = dec.world
    if world == 1:  # periodic images of its own faces, no messages
        m = [cnt[0], cnt[1]]
        parts = [(send_x[0, :m[0]], send_t[0, :m[0]], send_id[0, :m[0]]),
                 (send_x[1, :m[1]], send_t[1, :m[1]], send_id[1, :m[1]])]
        xs = torch.cat([x_local] + [p[0] for p in parts])
        ts = torch.cat([types_own.to(torch.int32)] + [p[1] for p in parts])
        ids = torch.cat([ids_own.to(torch.int64)] + [p[2] for p in parts])
        return xs, ts, ids, n
    # counts: set 1 (upper) travels up to rank + 1, set 0 (lower) down to rank - 1
    up, down = (rank + 1) % world, (rank - 1) % world
    c_up = torch.tensor([cnt[1]], dtype=torch.int64, device=dev)
    c_down = torch.tensor([cnt[0]], dtype=torch.int64, device=dev)
    r_from_below = torch.zeros(1, dtype=torch.int64, device=dev)  # rank - 1's upper set
    r_from_above = torch.zeros(1, dtype=torch.int64, device=dev)  # rank + 1's lower set
    # one group of point-to-point operations per phase (with NCCL a send
    # posted alone could wait for its peer's receive behind the peer's send)
    _p2p([dist.P2POp(dist.isend, c_up, up, group, 0),
          dist.P2POp(dist.irecv, r_from_below, down, group, 0),
          dist.P2POp(dist.isend, c_down, down, group, 1),
          dist.P2POp(dist.irecv, r_from_above, up, group, 1)])
    m_above, m_below = int(r_from_above.item()), int(r_from_below.item())
    tot = n + m_above + m_below
    xs = torch.empty((tot, 3), dtype=torch.float64, device=dev)
    ts = torch.empty(tot, dtype=torch.int32, device=dev)
    ids = torch.empty(tot, dtype=torch.int64, device=dev)
    xs[:n].copy_(x_local)
    ts[:n].copy_(types_own)
    ids[:n].copy_(ids_own)
    a0, a1 = n, n + m_above        # from rank + 1 (travelling down)
    b0, b1 = a1, tot               # from rank - 1 (travelling up)
    ops = []
    for k, (buf, dst_a, dst_b) in enumerate(((send_x, xs[a0:a1], xs[b0:b1]),
                                             (send_t, ts[a0:a1], ts[b0:b1]),
                                             (send_id, ids[a0:a1], ids[b0:b1]))):
        if cnt[1]:
            ops.append(dist.P2POp(dist.isend, buf[1, :cnt[1]].contiguous(), up, group, 2 + 2 * k))
        if m_below:
            ops.append(dist.P2POp(dist.irecv, dst_b, down, group, 2 + 2 * k))
        if cnt[0]:
            ops.append(dist.P2POp(dist.isend, buf[0, :cnt[0]].contiguous(), down, group, 3 + 2 * k))
        if m_above:
            ops.append(dist.P2POp(dist.irecv, dst_a, up, group, 3 + 2 * k))
    _p2p(ops)
    return xs, ts, ids, n


def _p2p(ops):
    import torch.distributed as dist
    if ops:
        for r in dist.batch_isend_irecv(ops):
            r.wait()


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

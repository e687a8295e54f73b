"""Spatial decomposition with a ghost exchange (paper_1607_02904_gb300.halo),
on CPU ranks: gloo process groups of 2 to 4 ranks, each rank evaluating its
local system with the oracle.

Owner computes with a ghost shell of 2 r_c: the energy summed over ranks and
the owned atoms' forces must equal the whole cell's (oracle, 1e-10 relative);
the exchanged ghosts must be exactly those selected from the whole system;
and the ghost set must contain every periodic image within 2 r_c of the slab.
"""
import os
import socket

import numpy as np
import pytest

import oracle
import workloads as W
from tests import _systems as S

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1607_02904_gb300 import halo  # noqa: E402

RC = 3.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def oracle_compute(table):
    def fn(x, t, box):
        nl = oracle.neighbors(x, box, RC)
        _, f, _, ea = oracle.compute(x, t, box, table, nl, eatom=True)
        return ea, f
    return fn


def tall_sic(seed=130):
    # zincblende SiC, 4 x 4 x 6 cells (768 atoms, 17.4 x 17.4 x 26.2 A):
    # three slabs of 8.7 A along z, wider than the 6 A ghost shell
    x, t, box = W.diamond(4, 4, 6, 4.36, zincblende=True)
    rng = np.random.Generator(np.random.Philox(seed))
    x = W.jitter_gaussian(x, 0.12, rng)
    x[:, 2] += 1.3  # some atoms leave [0, L) along the cut axis
    return x, t.astype(np.int32), box


TABLE = S.table_for(["Si", "C"], oracle.mix_tersoff89)
X, T, BOX = tall_sic()


def full_reference():
    nl = oracle.neighbors(X, BOX, RC)
    e, f, _ = oracle.compute(X, T, BOX, TABLE, nl)
    return e, f


@pytest.mark.parametrize("world", [1, 2, 3])
def test_owner_computes_equals_whole_cell(world):
    # ranks emulated one after the other, ghosts selected from the whole system
    dec = halo.SlabDecomposition(BOX, world, RC, RC + 0.5)
    assert dec.axis == 2
    e_ref, f_ref = full_reference()
    own = dec.owner(X)
    e_tot, f = 0.0, np.full_like(X, np.nan)
    for r in range(world):
        sel = np.nonzero(own == r)[0]
        xg, tg, _ = halo.ghosts_from_global(dec, X, T, r)
        e, fo = halo.owned_energy_forces(dec, X[sel], T[sel], xg, tg, r, oracle_compute(TABLE))
        e_tot += e
        f[sel] = fo
    assert abs(e_tot - e_ref) <= 1e-10 * abs(e_ref)
    assert np.abs(f - f_ref).max() <= 1e-10 * np.abs(f_ref).max()


@pytest.mark.parametrize("world", [1, 2, 3])
def test_ghosts_cover_the_shell(world):
    # brute force: every image (shift -L, 0, +L) of every atom whose cut-axis
    # coordinate lies within 2 r_c outside the slab is a ghost
    dec = halo.SlabDecomposition(BOX, world, RC, RC + 0.5)
    L = BOX[dec.axis]
    u = dec.wrapped(X)
    for r in range(world):
        lo, hi = dec.bounds(r)
        _, _, ids = halo.ghosts_from_global(dec, X, T, r)
        xg, _, _ = halo.ghosts_from_global(dec, X, T, r)
        got = {(int(i), round(float(z), 9)) for i, z in zip(ids, xg[:, dec.axis])}
        need = set()
        for k in range(len(X)):
            for s in (-L, 0.0, L):
                z = u[k] + s
                if lo - dec.r_ghost <= z < lo - 1e-12 or hi <= z < hi + dec.r_ghost - 1e-12:
                    need.add((k, round(float(z), 9)))
        assert need <= got
        # and nothing outside the shell
        zg = xg[:, dec.axis]
        assert np.all((zg >= lo - dec.r_ghost - 1e-9) & (zg <= hi + dec.r_ghost + 1e-9))
        assert not np.any((zg >= lo) & (zg < hi))


def test_decomposition_rejects_thin_slabs():
    with pytest.raises(ValueError):
        halo.SlabDecomposition(BOX, 5, RC)  # 5.2 A slabs < 6 A ghost shell
    with pytest.raises(ValueError):
        halo.SlabDecomposition([10.0, -1.0, 10.0], 1, RC)


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dec = halo.SlabDecomposition(BOX, world, RC, RC + 0.5)
        sel = np.nonzero(dec.owner(X) == rank)[0]
        xg, tg, ids = halo.halo_exchange(dec, X[sel], T[sel], sel, rank)
        xr, tr, idr = halo.ghosts_from_global(dec, X, T, rank)
        same = (np.array_equal(ids, idr) and np.array_equal(tg, tr) and np.array_equal(xg, xr))
        e, f = halo.distributed_energy_forces(dec, X[sel], T[sel], sel, rank,
                                              oracle_compute(TABLE))
        out[rank] = (same, e, sel, f)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3, 4])
def test_halo_exchange_gloo_ranks(world):
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    e_ref, f_ref = full_reference()
    f = np.full_like(X, np.nan)
    for r in range(world):
        same, e, sel, fo = out[r]
        assert same  # the messages deliver exactly the ghosts of the whole system
        assert abs(e - e_ref) <= 1e-10 * abs(e_ref)  # all-reduced total on every rank
        f[sel] = fo
    assert np.abs(f - f_ref).max() <= 1e-10 * np.abs(f_ref).max()


def test_single_cutoff_shell_is_not_enough():
    # with ghosts only within r_c, terms centred on ghosts that touch owned
    # atoms lose neighbours: the owned forces near the faces change
    dec = halo.SlabDecomposition(BOX, 2, RC, RC + 0.5)
    dec.r_ghost = RC
    e_ref, f_ref = full_reference()
    own = dec.owner(X)
    f = np.full_like(X, np.nan)
    for r in range(2):
        sel = np.nonzero(own == r)[0]
        xg, tg, _ = halo.ghosts_from_global(dec, X, T, r)
        _, f[sel] = halo.owned_energy_forces(dec, X[sel], T[sel], xg, tg, r, oracle_compute(TABLE))
    assert np.abs(f - f_ref).max() > 1e-3 * np.abs(f_ref).max()


def host_pack(dec, x_own, types_own, ids_own, rank):
    """The packing contract of tersoff_halo_pack restated on CPU tensors (the
    GPU tests check the kernel against the host path itself): owned atoms in
    the rank's frame, the two face sets in the receivers' frames."""
    x = x_own.numpy()
    u = dec.wrapped(x)
    L, lo, hi, rg, frame, s_lo, f_lo, s_up, f_up = halo.pack_geometry(dec, rank)
    x_local = x.copy()
    x_local[:, dec.axis] = u - frame
    n = len(x)
    cap = max(n, 1)
    send_x = np.zeros((2, cap, 3))
    send_t = np.zeros((2, cap), dtype=np.int32)
    send_id = np.zeros((2, cap), dtype=np.int64)
    cnt = []
    for k, (sel, shift, fr) in enumerate(((u - lo < rg, s_lo, f_lo), (hi - u <= rg, s_up, f_up))):
        idx = np.nonzero(sel)[0]
        y = x[idx].copy()
        y[:, dec.axis] = (u[idx] + shift) - fr
        send_x[k, :len(idx)] = y
        send_t[k, :len(idx)] = types_own.numpy()[idx]
        send_id[k, :len(idx)] = ids_own.numpy()[idx]
        cnt.append(len(idx))
    return (torch.from_numpy(x_local), torch.from_numpy(send_x), torch.from_numpy(send_t),
            torch.from_numpy(send_id), cnt)


def _expected_local(dec, rank):
    sel = np.nonzero(dec.owner(X) == rank)[0]
    xg, tg, idg = halo.ghosts_from_global(dec, X, T, rank)
    xl, tl, _ = halo.local_system(dec, X[sel], T[sel], xg, tg, rank)
    return sel, xl, tl, np.concatenate([sel, idg])


def _device_worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dec = halo.SlabDecomposition(BOX, world, RC, RC + 0.5)
        sel, xl, tl, il = _expected_local(dec, rank)
        xs, ts, ids, n = halo.halo_exchange_device(
            dec, torch.from_numpy(X[sel]), torch.from_numpy(T[sel]),
            torch.from_numpy(sel.astype(np.int64)), rank, host_pack)
        out[rank] = (n == len(sel) and np.array_equal(xs.numpy(), xl)
                     and np.array_equal(ts.numpy(), tl) and np.array_equal(ids.numpy(), il))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3, 4])
def test_device_buffer_exchange_gloo_ranks(world):
    # the exchange of packed buffers (halo_exchange_device) delivers, on every
    # rank, exactly the host path's local system: owned atoms first, then the
    # ghosts, bit for bit, in the local frame
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_device_worker, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    assert all(out[r] for r in range(world))


def test_device_buffer_exchange_one_rank():
    dec = halo.SlabDecomposition(BOX, 1, RC, RC + 0.5)
    sel, xl, tl, il = _expected_local(dec, 0)
    xs, ts, ids, n = halo.halo_exchange_device(
        dec, torch.from_numpy(X[sel]), torch.from_numpy(T[sel]),
        torch.from_numpy(sel.astype(np.int64)), 0, host_pack)
    assert n == len(sel)
    assert np.array_equal(xs.numpy(), xl) and np.array_equal(ts.numpy(), tl)
    assert np.array_equal(ids.numpy(), il)

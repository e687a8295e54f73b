"""Spatial decomposition with ghost exchange on one GPU: the ranks of
paper_1607_02904_gb300.halo emulated one after the other in one process (the
exchange is host logic between launches; no kernel waits on another rank),
each local system evaluated by the CUDA library.

Owner computes with a 2 r_c ghost shell: the energy summed over ranks and the
owned forces against the oracle for the whole cell (FP64 path, 1e-10), and at
512,000 atoms (4 slabs) against the library's whole-cell evaluation (FP64
1e-10; mixed path force RMS 1e-5 of the FP64 result).
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests import _systems as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RC = 3.0


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1607_02904_gb300 as T
    T.load()
    return T


def emulate(T, prec, x, t, box, table, world, r_list):
    from paper_1607_02904_gb300 import halo
    dec = halo.SlabDecomposition(box, world, RC, r_list)
    comp = halo.LibraryCompute(table, r_list, precision=prec)
    own = dec.owner(x)
    e_tot, f = 0.0, np.full_like(x, np.nan)
    for r in range(world):
        sel = np.nonzero(own == r)[0]
        xg, tg, _ = halo.ghosts_from_global(dec, x, t, r)
        e, fo = halo.owned_energy_forces(dec, x[sel], t[sel], xg, tg, r, comp)
        e_tot += e
        f[sel] = fo
    comp.close()
    return e_tot, f


def whole(T, prec, x, t, box, table, r_list):
    ctx = T.Context(prec)
    ctx.params(table)
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    ctx.neighbor_build(xd, torch.tensor(t, dtype=torch.int32, device="cuda"), box, r_list)
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    f = torch.zeros_like(xd)
    ctx.compute(xd, e, f)
    out = (e.item(), f.cpu().numpy())
    ctx.close()
    return out


@pytest.mark.parametrize("world", [1, 2, 3])
def test_emulated_ranks_match_oracle(T, world):
    x, t, box = W.diamond(4, 4, 6, 4.36, zincblende=True)
    rng = np.random.Generator(np.random.Philox(131))
    x = W.jitter_gaussian(x, 0.12, rng)
    t = t.astype(np.int32)
    table = S.table_for(["Si", "C"], oracle.mix_tersoff89)
    e, f = emulate(T, T.FP64, x, t, box, table, world, RC + 0.5)
    e_ref, f_ref, _ = oracle.compute(x, t, box, table, oracle.neighbors(x, box, RC))
    assert abs(e - e_ref) <= 1e-10 * abs(e_ref)
    assert np.abs(f - f_ref).max() <= 1e-10 * np.abs(f_ref).max()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_four_slabs_at_full_size(T, prec):
    x, v, t, box, names = W.config_si_md()
    t = t.astype(np.int32)
    table = S.table_for(["Si"], oracle.mix_tersoff89)
    e, f = emulate(T, prec, x, t, box, table, 4, 4.0)
    e64, f64 = whole(T, T.FP64, x, t, box, table, 4.0)
    if prec == 0:
        assert abs(e - e64) <= 1e-10 * abs(e64)
        assert np.abs(f - f64).max() <= 1e-10 * np.abs(f64).max()
    else:
        assert abs(e - e64) <= 1e-5 * abs(e64)
        assert np.sqrt(((f - f64) ** 2).mean() / (f64 ** 2).mean()) <= 1e-5


def tall_sic_moved():
    x, t, box = W.diamond(4, 4, 6, 4.36, zincblende=True)
    rng = np.random.Generator(np.random.Philox(132))
    x = W.jitter_gaussian(x, 0.12, rng)
    x[:, 2] += 1.3  # some atoms leave [0, L) along the cut axis
    x[:5, 2] -= 2 * box[2]  # and a few lie two periods below
    return x, t.astype(np.int32), box


def assemble(packs, world, r):
    # the exchange's delivery, emulated: rank r's own frame, then rank r + 1's
    # lower set (travelling down), then rank r - 1's upper set (travelling up)
    xl, _, _, _, _ = packs[r]
    a = packs[(r + 1) % world]
    b = packs[(r - 1) % world]
    xs = torch.cat([xl, a[1][0, :a[4][0]], b[1][1, :b[4][1]]])
    ts = torch.cat([a[2][0, :a[4][0]], b[2][1, :b[4][1]]])
    ids = torch.cat([a[3][0, :a[4][0]], b[3][1, :b[4][1]]])
    return xs.cpu().numpy(), ts.cpu().numpy(), ids.cpu().numpy()


def check_device_pack(T, x, t, box, world, r_list):
    from paper_1607_02904_gb300 import halo
    dec = halo.SlabDecomposition(box, world, RC, r_list)
    ctx = T.Context(T.FP64)
    pack = halo.device_pack(ctx)
    own = dec.owner(x)
    packs, sels = {}, {}
    for r in range(world):
        sel = np.nonzero(own == r)[0]
        sels[r] = sel
        packs[r] = pack(dec, torch.tensor(x[sel], dtype=torch.float64, device="cuda"),
                        torch.tensor(t[sel], dtype=torch.int32, device="cuda"),
                        torch.tensor(sel, dtype=torch.int64, device="cuda"), r)
    for r in range(world):
        sel = sels[r]
        xg, tg, idg = halo.ghosts_from_global(dec, x, t, r)
        xl, tl, _ = halo.local_system(dec, x[sel], t[sel], xg, tg, r)
        xs, ts, ids = assemble(packs, world, r)
        assert np.array_equal(xs, xl)  # bit for bit: owned atoms, then ghosts
        assert np.array_equal(ts, tl[len(sel):])
        assert np.array_equal(ids, idg)
    ctx.close()
    return dec, packs, sels


@pytest.mark.parametrize("world", [1, 2, 3])
def test_device_pack_matches_host_local_systems(T, world):
    x, t, box = tall_sic_moved()
    check_device_pack(T, x, t, box, world, RC + 0.5)


def test_device_pack_four_slabs_at_full_size(T):
    # 512,000 atoms, 4 slabs: the packed local systems equal the host path's;
    # evaluated by the library (FP64), the owned forces and the summed energy
    # equal the whole cell's
    from paper_1607_02904_gb300 import halo
    x, v, t, box, names = W.config_si_md()
    t = t.astype(np.int32)
    table = S.table_for(["Si"], oracle.mix_tersoff89)
    dec, packs, sels = check_device_pack(T, x, t, box, 4, 4.0)
    comp = halo.LibraryCompute(table, 4.0, precision=T.FP64)
    e_tot, f = 0.0, np.full_like(x, np.nan)
    for r in range(4):
        xs, ts, _ = assemble(packs, 4, r)
        tl = np.concatenate([t[sels[r]], ts])
        ea, fo = comp(xs, tl, dec.local_box())
        e_tot += float(np.sum(ea[:len(sels[r])]))
        f[sels[r]] = fo[:len(sels[r])]
    comp.close()
    e_ref, f_ref = whole(T, T.FP64, x, t, box, table, 4.0)
    assert abs(e_tot - e_ref) <= 1e-10 * abs(e_ref)
    assert np.abs(f - f_ref).max() <= 1e-10 * np.abs(f_ref).max()


def test_device_pack_capacity_and_empty(T):
    from paper_1607_02904_gb300 import halo
    x, t, box = tall_sic_moved()
    dec = halo.SlabDecomposition(box, 2, RC, RC + 0.5)
    ctx = T.Context(T.FP64)
    sel = np.nonzero(dec.owner(x) == 0)[0]
    xd = torch.tensor(x[sel], dtype=torch.float64, device="cuda")
    td = torch.tensor(t[sel], dtype=torch.int32, device="cuda")
    idd = torch.tensor(sel, dtype=torch.int64, device="cuda")
    full = halo.device_pack(ctx)(dec, xd, td, idd, 0)
    cap = 5
    xl = torch.empty_like(xd)
    sx = torch.full((2, cap, 3), -1.0, dtype=torch.float64, device="cuda")
    st = torch.empty((2, cap), dtype=torch.int32, device="cuda")
    si = torch.empty((2, cap), dtype=torch.int64, device="cuda")
    cnt = torch.zeros(2, dtype=torch.int32, device="cuda")
    ctx.halo_pack(xd, td, idd, dec.axis, halo.pack_geometry(dec, 0), cap, xl, sx, st, si, cnt)
    # sets larger than the capacity: counted in full, the first cap entries written
    assert [int(c) for c in cnt.cpu()] == full[4] and min(full[4]) > cap
    assert torch.equal(sx, full[1][:, :cap]) and torch.equal(si, full[3][:, :cap])
    # no owned atoms: both counts zero
    e = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    cnt.fill_(7)
    ctx.halo_pack(e, td[:0], idd[:0], dec.axis, halo.pack_geometry(dec, 0), cap, e, sx, st, si,
                  cnt)
    assert cnt.cpu().tolist() == [0, 0]
    with pytest.raises(T.TersoffError):
        ctx.halo_pack(xd, td, idd, 3, halo.pack_geometry(dec, 0), cap, xl, sx, st, si, cnt)
    ctx.close()

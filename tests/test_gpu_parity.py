"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle.

Tolerances (stated once, used everywhere):
  neighbour lists   bit-exact (sorted indices and counts)
  FP64 path         |dE| <= 1e-10 |E|; max|dF| <= 1e-10 max|F|; max|dW| <= 1e-10 max|W|
  mixed path        relative force RMS <= 1e-5; |dE| <= 1e-5 |E|; max|dW| <= 1e-5 max|W|
                    (float resolution of r inside the f_C transition limits a lone
                    transition-region term to ~2e-6 relative energy)
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests import _systems as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RC = 3.0
TOL64 = 1e-10
TOLMIX_F = 1e-5
TOLMIX_E = 1e-5
TOLMIX_W = 1e-5


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1607_02904_gb300 as T
    T.load()
    return T


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def gpu_eval(T, prec, x, t, box, table, r_list, scatter=0):
    ctx = T.Context(prec)
    ctx.set_scatter(scatter)
    ctx.params(table)
    xd, td = dev(x), dev(t, torch.int32)
    ctx.neighbor_build(xd, td, box, r_list)
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    f = torch.zeros_like(xd)
    w = torch.zeros(6, dtype=torch.float64, device="cuda")
    ctx.compute(xd, e, f, w)
    torch.cuda.synchronize()
    out = (e.item(), f.cpu().numpy(), w.cpu().numpy())
    ctx.close()
    return out


def check(prec, got, ref):
    e, f, w = got
    er, fr, wr = ref
    if prec == 0:
        assert abs(e - er) <= TOL64 * abs(er), (e, er)
        assert np.abs(f - fr).max() <= TOL64 * np.abs(fr).max()
        assert np.abs(w - wr).max() <= TOL64 * np.abs(wr).max()
    else:
        rms = np.sqrt(((f - fr) ** 2).mean()) / np.sqrt((fr ** 2).mean())
        assert rms <= TOLMIX_F, rms
        assert abs(e - er) <= TOLMIX_E * abs(er), (e, er)
        assert np.abs(w - wr).max() <= TOLMIX_W * np.abs(wr).max()


def si_table():
    return S.table_for(["Si"], oracle.mix_tersoff89)


def sic_table():
    return S.table_for(["Si", "C"], oracle.mix_tersoff89)


def small_systems():
    si, sic = si_table(), sic_table()
    out = []
    x, t, box, _ = W.config_si_small()
    out.append(("si-4096", x, t, box, si))
    x, t, box = S.sic_cell(n=4)
    out.append(("sic-512", x, t, box, sic))
    x, t, box = S.packing_cell(n=300, c_frac=0.3, seed=31)
    out.append(("pack-300", x, t, box, sic))
    x, t, box = S.packing_cell(n=200, c_frac=1.0, seed=32)
    out.append(("pack-C-200", x, t, box, sic))
    x, t, box = S.si_cell(n=3, amp=0.3, seed=33)
    out.append(("si-l3m3", x, t, box, S.with_lambda3(si, 1.7322, 3)))
    out.append(("si-l3m1", x, t, box, S.with_lambda3(si, 1.3, 1)))
    x, t, box = S.si_cell(n=2, amp=0.2, seed=34)
    out.append(("si-64-two-cells", x, t, box, si))  # box 10.9 A: two cells per edge
    return out


SMALL = small_systems()
IDS = [s[0] for s in SMALL]


@pytest.mark.parametrize("sysd", SMALL, ids=IDS)
@pytest.mark.parametrize("r_list", [RC, RC + 1.0])
def test_neighbor_lists_bit_exact(T, sysd, r_list):
    _, x, t, box, table = sysd
    if box.min() < 2 * r_list:
        pytest.skip("box below twice the list radius")
    cnt_ref, nbr_ref = oracle.neighbors(x, box, r_list)
    ctx = T.Context(T.MIXED)
    ctx.params(table)
    ctx.neighbor_build(dev(x), dev(t, torch.int32), box, r_list)
    cap = int(cnt_ref.max())
    cnt, nbr, st = ctx.neighbor_export(cap)
    assert st == 0
    assert np.array_equal(cnt.cpu().numpy(), cnt_ref)
    assert np.array_equal(nbr.cpu().numpy(), nbr_ref[:, :cap])
    ctx.close()


@pytest.mark.parametrize("sysd", SMALL, ids=IDS)
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("scatter", [0, 1], ids=["gather", "atomic"])
def test_compute_matches_oracle(T, sysd, prec, scatter):
    _, x, t, box, table = sysd
    r_list = RC + 0.5 if box.min() >= 2 * (RC + 0.5) else RC
    ref = oracle.compute(x, t, box, table, oracle.neighbors(x, box, RC), nthreads=4)
    got = gpu_eval(T, prec, x, t, box, table, r_list, scatter)
    check(prec, got, ref)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_peratom_energy(T, prec):
    x, t, box = S.sic_cell(n=3, seed=40)
    table = sic_table()
    _, _, _, ea_ref = oracle.compute(x, t, box, table, oracle.neighbors(x, box, RC), eatom=True)
    ctx = T.Context(prec)
    ctx.params(table)
    xd = dev(x)
    ctx.neighbor_build(xd, dev(t, torch.int32), box, RC)
    ea = torch.zeros(len(x), dtype=torch.float64, device="cuda")
    ctx.compute_peratom(xd, ea)
    torch.cuda.synchronize()
    tol = 1e-10 if prec == 0 else 1e-5
    assert np.abs(ea.cpu().numpy() - ea_ref).max() <= tol * np.abs(ea_ref).max()
    ctx.close()


def test_moved_positions_use_skin_list(T):
    # positions moved after the build (less than half the skin): same result as
    # a fresh list, for both paths
    x, t, box, _ = W.config_si_small()
    table = si_table()
    rng = np.random.default_rng(5)
    x2 = x + rng.uniform(-0.2, 0.2, size=x.shape) + np.array([10.0, -3.0, 2 * box[2]])
    ref = oracle.compute(x2, t, box, table, oracle.neighbors(x2, box, RC))
    for prec in (0, 1):
        ctx = T.Context(prec)
        ctx.params(table)
        ctx.neighbor_build(dev(x), dev(t, torch.int32), box, RC + 1.0)
        xd2 = dev(x2)
        e = torch.zeros(1, dtype=torch.float64, device="cuda")
        f = torch.zeros_like(xd2)
        w = torch.zeros(6, dtype=torch.float64, device="cuda")
        ctx.compute(xd2, e, f, w)
        torch.cuda.synchronize()
        check(prec, (e.item(), f.cpu().numpy(), w.cpu().numpy()), ref)
        ctx.close()


def test_capacity_overflow_regrows(T):
    x, t, box, _ = W.config_si_small()
    ctx = T.Context(T.FP64)
    ctx.params(si_table())
    ctx.set_neighbor_capacity(2)
    ctx.neighbor_build(dev(x), dev(t, torch.int32), box, RC + 1.0)
    cap, mx = ctx.neighbor_capacity()
    cnt_ref, nbr_ref = oracle.neighbors(x, box, RC + 1.0)
    assert mx == cnt_ref.max() and cap >= mx
    cnt, nbr, st = ctx.neighbor_export(int(cnt_ref.max()))
    assert np.array_equal(nbr.cpu().numpy(), nbr_ref[:, : cnt_ref.max()])
    # export into too small a buffer reports overflow
    _, _, st = ctx.neighbor_export(3)
    assert st == 3
    ctx.close()


def test_error_codes(T):
    x, t, box, _ = W.config_si_small()
    ctx = T.Context(T.MIXED)
    with pytest.raises(T.TersoffError) as ei:
        ctx.neighbor_build(dev(x), dev(t, torch.int32), box, RC)
    assert ei.value.code == 7  # params first
    ctx.params(si_table())
    with pytest.raises(T.TersoffError) as ei:
        ctx.compute(dev(x), torch.zeros(1, dtype=torch.float64, device="cuda"))
    assert ei.value.code == 7  # list first
    with pytest.raises(T.TersoffError) as ei:
        ctx.neighbor_build(dev(x), dev(t, torch.int32), np.array([7.0, 50.0, 50.0]), RC + 1.0)
    assert ei.value.code == 2  # box too small
    bad = x.copy()
    bad[17, 1] = np.nan
    with pytest.raises(T.TersoffError) as ei:
        ctx.neighbor_build(dev(bad), dev(t, torch.int32), box, RC)
    assert ei.value.code == 4
    tt = t.copy()
    tt[3] = 5
    with pytest.raises(T.TersoffError) as ei:
        ctx.neighbor_build(dev(x), dev(tt, torch.int32), box, RC)
    assert ei.value.code == 1
    with pytest.raises(T.TersoffError) as ei:
        ctx.neighbor_build(dev(x), dev(t, torch.int32), box, 2.0)  # below the cutoff
    assert ei.value.code == 1
    bad_table = si_table().copy()
    bad_table[0] = 2.5  # m not an integer
    with pytest.raises(T.TersoffError) as ei:
        ctx.params(bad_table)
    assert ei.value.code == 1
    ctx.close()


def test_empty_and_dimer(T):
    table = si_table()
    ctx = T.Context(T.FP64)
    ctx.params(table)
    box = np.array([20.0, 20.0, 20.0])
    xe = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    te = torch.zeros(0, dtype=torch.int32, device="cuda")
    ctx.neighbor_build(xe, te, box, RC)
    e = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    ctx.compute(xe, e)
    torch.cuda.synchronize()
    assert e.item() == 0.0
    # isolated dimer in the cutoff transition: zeta = 0 path
    x = np.array([[5.0, 5.0, 5.0], [7.9, 5.0, 5.0]])
    t = np.zeros(2, dtype=np.int32)
    ref = oracle.compute(x, t, box, table, oracle.neighbors(x, box, RC))
    for prec in (0, 1):
        got = gpu_eval(T, prec, x, t, box, table, RC)
        check(prec, got, ref)
    ctx.close()


# ----------------------------------------------------------------------------- full sizes
def test_full_size_si_512k(T):
    # 40^3 diamond cells (512,000 atoms), the MD benchmark's configuration;
    # every atom is compared (the oracle runs multi-threaded)
    x, v, t, box, _ = W.config_si_md()
    table = si_table()
    cnt_ref, nbr_ref = oracle.neighbors(x, box, RC + 1.0)
    ref = oracle.compute(x, t, box, table, (cnt_ref, nbr_ref), nthreads=16)
    for prec in (0, 1):
        ctx = T.Context(prec)
        ctx.params(table)
        xd = dev(x)
        ctx.neighbor_build(xd, dev(t, torch.int32), box, RC + 1.0)
        if prec == 1:
            cnt, nbr, st = ctx.neighbor_export(int(cnt_ref.max()))
            assert np.array_equal(cnt.cpu().numpy(), cnt_ref)
            assert np.array_equal(nbr.cpu().numpy(), nbr_ref[:, : cnt_ref.max()])
        e = torch.zeros(1, dtype=torch.float64, device="cuda")
        f = torch.zeros_like(xd)
        w = torch.zeros(6, dtype=torch.float64, device="cuda")
        ctx.compute(xd, e, f, w)
        torch.cuda.synchronize()
        check(prec, (e.item(), f.cpu().numpy(), w.cpu().numpy()), ref)
        ctx.close()


def test_full_size_sic_2m_sampled(T):
    # 64^3 zincblende cells (2,097,152 atoms): mixed path, compared on every atom's
    # force against the oracle, energy and virial in full
    x, t, box, _ = W.config_sic()
    table = sic_table()
    ref = oracle.compute(x, t, box, table, oracle.neighbors(x, box, RC), nthreads=16)
    got = gpu_eval(T, 1, x, t, box, table, RC + 0.5)
    check(1, got, ref)


# ----------------------------------------------------------------------------- MD
def _md_inputs(ncell=3, seed=50):
    x, t, box = W.diamond(ncell, ncell, ncell, 5.432)
    rng = np.random.Generator(np.random.Philox(seed))
    x = W.jitter_gaussian(x, 0.05, rng)
    v = W.maxwell_velocities(t, np.array([W.MASS_AMU["Si"]]), 1000.0, rng)
    return x, v, t, box


@pytest.mark.parametrize("scatter", [0, 1], ids=["gather", "atomic"])
def test_md_fp64_matches_oracle(T, scatter):
    x, v, t, box = _md_inputs(ncell=4)
    table = si_table()
    mass = [W.MASS_AMU["Si"]]
    nsteps, every = 25, 10
    xo, vo, thermo_o, fo = oracle.md_run(x, v, t, box, table, mass, 0.001, nsteps, RC + 1.0,
                                         every)
    ctx = T.Context(T.FP64)
    ctx.set_scatter(scatter)
    ctx.params(table)
    xd, vd = dev(x), dev(v)
    ctx.neighbor_build(xd, dev(t, torch.int32), box, RC + 1.0)
    fd = torch.zeros_like(xd)
    ctx.compute(xd, None, fd)
    th = torch.zeros((nsteps, 3), dtype=torch.float64, device="cuda")
    ctx.md_step(xd, vd, fd, mass, 0.001, nsteps, every, th)
    torch.cuda.synchronize()
    assert np.abs(xd.cpu().numpy() - xo).max() < 1e-9
    assert np.abs(vd.cpu().numpy() - vo).max() < 1e-7
    assert np.abs(fd.cpu().numpy() - fo).max() < 1e-8 * np.abs(fo).max()
    assert np.abs(th.cpu().numpy() - thermo_o).max() < 1e-8 * np.abs(thermo_o).max()
    ctx.close()


def test_md_mixed_energy_conservation_and_host_api(T):
    x, v, t, box = _md_inputs(ncell=5, seed=51)
    table = si_table()
    mass = [W.MASS_AMU["Si"]]
    ctx = T.Context(T.MIXED)
    ctx.params(table)
    xd, vd = dev(x), dev(v)
    ctx.neighbor_build(xd, dev(t, torch.int32), box, RC + 1.0)
    fd = torch.zeros_like(xd)
    ctx.compute(xd, None, fd)
    # host-buffer variant from the same state
    xh, vh, fh = xd.cpu().pin_memory(), vd.cpu().pin_memory(), fd.cpu().pin_memory()
    th = torch.zeros((200, 3), dtype=torch.float64, device="cuda")
    ctx.md_step(xd, vd, fd, mass, 0.001, 200, 10, th)
    thermo = th.cpu().numpy()
    assert np.ptp(thermo[:, 2]) < 0.02 * np.ptp(thermo[:, 1])
    ctx2 = T.Context(T.MIXED)
    ctx2.params(table)
    ctx2.neighbor_build(xh.cuda(), dev(t, torch.int32), box, RC + 1.0)
    thh = torch.zeros((200, 3), dtype=torch.float64).pin_memory()
    ctx2.md_step_host(xh, vh, fh, mass, 0.001, 200, 10, thh)
    # same arithmetic up to atomics ordering: trajectories stay close over 0.2 ps
    assert np.abs(xh.numpy() - xd.cpu().numpy()).max() < 1e-4
    assert np.abs(thh.numpy()[:, 2] - thermo[:, 2]).max() < 1e-3
    ctx.close()
    ctx2.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_md_host_buffers_pinned_and_pageable_equal_device(T, prec):
    # the host-buffer call with page-locked and with pageable host arrays
    # gives the device call's state bit for bit (the copies are exact, and
    # gather mode sums in a fixed order)
    x, v, t, box = _md_inputs(ncell=4, seed=53)
    table = si_table()
    mass = [W.MASS_AMU["Si"]]
    runs = []
    for mode in ("device", "pinned", "pageable"):
        ctx = T.Context(prec)
        ctx.params(table)
        xd, vd = dev(x), dev(v)
        ctx.neighbor_build(xd, dev(t, torch.int32), box, RC + 1.0)
        fd = torch.zeros_like(xd)
        ctx.compute(xd, None, fd)
        if mode == "device":
            ctx.md_step(xd, vd, fd, mass, 0.001, 20, 10)
            torch.cuda.synchronize()
            runs.append([a.cpu().numpy() for a in (xd, vd, fd)])
        else:
            hs = [a.cpu() for a in (xd, vd, fd)]
            if mode == "pinned":
                hs = [a.pin_memory() for a in hs]
            ctx.md_step_host(hs[0], hs[1], hs[2], mass, 0.001, 20, 10)
            runs.append([a.numpy().copy() for a in hs])
        ctx.close()
    for other in runs[1:]:
        for a, b in zip(runs[0], other):
            assert np.array_equal(a, b)


def test_md_graph_replay_matches_eager(T):
    # the same FP64 MD through direct launches and through a replayed CUDA graph
    x, v, t, box = _md_inputs(ncell=4, seed=52)
    table = si_table()
    mass = [W.MASS_AMU["Si"]]
    out = []
    for graphs in (False, True):
        ctx = T.Context(T.FP64)
        ctx.set_graphs(graphs)
        ctx.params(table)
        xd, vd = dev(x), dev(v)
        ctx.neighbor_build(xd, dev(t, torch.int32), box, RC + 1.0)
        fd = torch.zeros_like(xd)
        ctx.compute(xd, None, fd)
        th = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
        for _ in range(3):  # capture once, replay twice
            ctx.md_step(xd, vd, fd, mass, 0.001, 10, 10, th)
        torch.cuda.synchronize()
        out.append((xd.cpu().numpy(), vd.cpu().numpy(), th.cpu().numpy()))
        ctx.close()
    assert np.abs(out[0][0] - out[1][0]).max() < 1e-10
    assert np.abs(out[0][1] - out[1][1]).max() < 1e-8
    assert np.abs(out[0][2] - out[1][2]).max() < 1e-8


def test_md_graph_overflow_rolls_back(T):
    # a hot random packing with the list capacity set to the initial maximum:
    # a rebuild inside the replayed graph overflows, the state is restored and
    # the steps rerun; the trajectory still matches the oracle
    x, t, box = S.packing_cell(n=300, c_frac=0.0, seed=61)
    table = sic_table()
    mass = [W.MASS_AMU["Si"], W.MASS_AMU["C"]]
    rng = np.random.Generator(np.random.Philox(62))
    v = W.maxwell_velocities(t, np.array(mass), 6000.0, rng)
    nsteps, every = 40, 2
    xo, vo, thermo_o, fo = oracle.md_run(x, v, t, box, table, mass, 0.001, nsteps, RC + 1.0,
                                         every, cap=96)
    cnt_ref, _ = oracle.neighbors(x, box, RC + 1.0)
    ctx = T.Context(T.FP64)
    ctx.params(table)
    ctx.set_neighbor_capacity(int(cnt_ref.max()))
    xd, vd = dev(x), dev(v)
    ctx.neighbor_build(xd, dev(t, torch.int32), box, RC + 1.0)
    fd = torch.zeros_like(xd)
    ctx.compute(xd, None, fd)
    ctx.md_step(xd, vd, fd, mass, 0.001, nsteps, every)
    torch.cuda.synchronize()
    cap, _ = ctx.neighbor_capacity()
    assert cap > cnt_ref.max()  # the overflow was caught and the capacity grown
    assert np.abs(xd.cpu().numpy() - xo).max() < 1e-8
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_forces_bitwise_reproducible(T, prec):
    # forces are gathered from per-slot contributions in a fixed order (exact
    # fixed point on the mixed path): two evaluations agree bit for bit
    x, t, box = S.sic_cell(n=6, seed=70)
    ctx = T.Context(prec)
    ctx.params(sic_table())
    xd = dev(x)
    ctx.neighbor_build(xd, dev(t, torch.int32), box, RC + 0.5)
    f1 = torch.zeros_like(xd)
    f2 = torch.zeros_like(xd)
    ctx.compute(xd, None, f1)
    ctx.compute(xd, None, f2)
    torch.cuda.synchronize()
    assert torch.equal(f1, f2)
    ctx.close()


def _boundary_cell():
    """A jittered Si cell whose atoms sit on the list-cell edges of the build's
    grid (exactly, or one ulp to either side), on the box faces (0, -0.0, L and
    one ulp below L) and in other periodic images (shifted by -L, +L, +2L)."""
    x, t, box = S.si_cell(n=4, amp=0.1, seed=41)
    r_list = RC + 1.0
    x = x.copy()
    for a in range(3):
        L = box[a]
        nc = max(2, int(np.floor(L / r_list)))
        h = L / nc
        edges = np.array([c * h for c in range(nc + 1)])
        for i in range(len(x)):
            d = np.abs(edges - x[i, a])
            k = int(np.argmin(d))
            if d[k] < 0.15:
                x[i, a] = edges[k]
                sel = (i + a) % 3  # exact, one ulp below, one ulp above
                if sel == 1:
                    x[i, a] = np.nextafter(x[i, a], -np.inf)
                elif sel == 2:
                    x[i, a] = np.nextafter(x[i, a], np.inf)
                if k == nc and (i % 2 == 0):
                    x[i, a] = np.nextafter(L, -np.inf)
                if k == 0 and x[i, a] == 0.0 and (i % 2 == 1):
                    x[i, a] = -0.0
    shifts = (-1.0, 1.0, 2.0)
    for q, i in enumerate(range(0, len(x), 37)):
        x[i] += shifts[q % 3] * box
    return x, t, box, r_list


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_atoms_on_cell_edges_and_box_faces(T, prec):
    x, t, box, r_list = _boundary_cell()
    assert (x < 0).any() and (x >= box).any() and (np.signbit(x) & (x == 0)).any()
    table = si_table()
    cnt_ref, nbr_ref = oracle.neighbors(x, box, r_list)
    ctx = T.Context(prec)
    ctx.params(table)
    ctx.neighbor_build(dev(x), dev(t, torch.int32), box, r_list)
    cap = int(cnt_ref.max())
    cnt, nbr, st = ctx.neighbor_export(cap)
    assert st == 0
    assert np.array_equal(cnt.cpu().numpy(), cnt_ref)
    assert np.array_equal(nbr.cpu().numpy(), nbr_ref[:, :cap])
    ctx.close()
    ref = oracle.compute(x, t, box, table, oracle.neighbors(x, box, RC), nthreads=4)
    check(prec, gpu_eval(T, prec, x, t, box, table, r_list), ref)


def test_md_fp64_from_cell_edges_matches_oracle(T):
    x, t, box, r_list = _boundary_cell()
    table = si_table()
    mass = [W.MASS_AMU["Si"]]
    rng = np.random.Generator(np.random.Philox(42))
    v = W.maxwell_velocities(t, np.array(mass), 1000.0, rng)
    nsteps, every = 12, 4
    xo, vo, _, fo = oracle.md_run(x, v, t, box, table, mass, 0.001, nsteps, r_list, every)
    ctx = T.Context(T.FP64)
    ctx.params(table)
    xd, vd = dev(x), dev(v)
    ctx.neighbor_build(xd, dev(t, torch.int32), box, r_list)
    fd = torch.zeros_like(xd)
    ctx.compute(xd, None, fd)
    ctx.md_step(xd, vd, fd, mass, 0.001, nsteps, every)
    torch.cuda.synchronize()
    assert np.abs(xd.cpu().numpy() - xo).max() < 1e-9
    assert np.abs(fd.cpu().numpy() - fo).max() < 1e-8 * np.abs(fo).max()
    ctx.close()

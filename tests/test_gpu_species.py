"""More than two species, and a batch with an empty system.

Three species run the kernels' runtime-species-count paths (records in shared
memory, shared-memory adjoint accumulators), which the one- and two-species
systems never reach. The third element is Si with A and B raised by 5% and a
bond softening of 0.95 towards C, so every record differs.

Tolerances: FP64 1e-10 relative, mixed 1e-5 (force RMS, energy, virial); the
parameter VJP compared scaled by the parameter values (FP64 1e-10, mixed 1e-5).
"""
import numpy as np
import pytest

import oracle
import workloads as W

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


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def three_species_table():
    elem, _ = W.element_records(["Si", "C", "Si"])
    elem = elem.copy()
    elem[2, 0] *= 1.05  # A
    elem[2, 1] *= 1.05  # B
    chi = np.ones((3, 3))
    chi[0, 1] = chi[1, 0] = W.CHI_SIC
    chi[1, 2] = chi[2, 1] = 0.95
    return oracle.mix_tersoff89(elem, chi)


def three_species_system(seed=95):
    rng = np.random.Generator(np.random.Philox(seed))
    x, t, box, ok = W.random_packing(240, 0.4, 2.3, 1.8, rng)
    assert ok
    t = t.copy()
    si = np.nonzero(t == 0)[0]
    t[si[::2]] = 2  # half the Si atoms become the third species
    return x, t.astype(np.int32), box


TABLE3 = three_species_table()
X3, T3, BOX3 = three_species_system()
REF3 = oracle.compute(X3, T3, BOX3, TABLE3, oracle.neighbors(X3, BOX3, RC))


def check(prec, got, ref):
    e, f, w = got
    er, fr, wr = ref
    if prec == 0:
        assert abs(e - er) <= 1e-10 * abs(er)
        assert np.abs(f - fr).max() <= 1e-10 * np.abs(fr).max()
        assert np.abs(w - wr).max() <= 1e-10 * np.abs(wr).max()
    else:
        assert np.sqrt(((f - fr) ** 2).mean()) / np.sqrt((fr ** 2).mean()) <= 1e-5
        assert abs(e - er) <= 1e-5 * abs(er)
        assert np.abs(w - wr).max() <= 1e-5 * np.abs(wr).max()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("scatter", [0, 1], ids=["gather", "atomic"])
def test_three_species_compute(T, prec, scatter):
    assert set(np.unique(T3)) == {0, 1, 2}
    ctx = T.Context(prec)
    ctx.set_scatter(scatter)
    ctx.params(TABLE3)
    xd = dev(X3)
    ctx.neighbor_build(xd, dev(T3, torch.int32), BOX3, RC + 0.5)
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    f = torch.zeros_like(xd)
    w = torch.zeros(6, dtype=torch.float64, device="cuda")
    ctx.compute(xd, e, f, w)
    torch.cuda.synchronize()
    check(prec, (e.item(), f.cpu().numpy(), w.cpu().numpy()), REF3)
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_three_species_backward(T, prec):
    rng = np.random.Generator(np.random.Philox(96))
    gE = 1.3
    gF = rng.normal(0.0, 1.0, size=X3.shape)
    nl = oracle.neighbors(X3, BOX3, RC)
    ref = np.zeros(TABLE3.size)
    for p in range(TABLE3.size):
        if p % oracle.NPAR == 0:
            continue
        de, df = oracle.cs_param(X3, T3, BOX3, TABLE3, nl, p)
        ref[p] = gE * de + float((gF * df).sum())
    ctx = T.Context(prec)
    ctx.params(TABLE3)
    xd = dev(X3)
    ctx.neighbor_build(xd, dev(T3, torch.int32), BOX3, RC + 0.5)
    g = torch.full((TABLE3.size,), np.nan, dtype=torch.float64, device="cuda")
    ctx.backward(xd, dev([gE]), dev(gF), None, g)
    torch.cuda.synchronize()
    got = g.cpu().numpy()
    s = np.where(TABLE3 != 0.0, np.abs(TABLE3), 1.0)
    err = np.abs(s * (got - ref)).max() / np.abs(s * ref).max()
    assert err <= (1e-10 if prec == 0 else 1e-5), err
    ctx.close()


def test_batch_with_empty_system(T):
    # systems 1 and 3 hold no atoms: zero energy and virial, the others exact
    table = oracle.mix_tersoff89(*W.element_records(["Si", "C"]))
    cells = W.batched_cells(n_cells=2, nmin=64, nmax=200, seed_k=97)
    empty_box = np.array([9.0, 9.0, 9.0])
    systems = [cells[0], (np.zeros((0, 3)), np.zeros(0, np.int32), empty_box), cells[1],
               (np.zeros((0, 3)), np.zeros(0, np.int32), empty_box)]
    off = np.cumsum([0] + [len(c[0]) for c in systems]).astype(np.int32)
    x = np.concatenate([c[0] for c in systems])
    t = np.concatenate([c[1] for c in systems]).astype(np.int32)
    boxes = np.stack([c[2] for c in systems])
    ctx = T.Context(0)
    ctx.params(table)
    xd = dev(x)
    ctx.neighbor_build_batched(xd, dev(t, torch.int32), off, boxes, RC + 0.5)
    e = torch.full((4,), np.nan, dtype=torch.float64, device="cuda")
    f = torch.zeros_like(xd)
    w = torch.full((4, 6), np.nan, dtype=torch.float64, device="cuda")
    ctx.compute_batched(xd, e, f, w)
    torch.cuda.synchronize()
    e, w = e.cpu().numpy(), w.cpu().numpy()
    assert e[1] == 0.0 and e[3] == 0.0 and not w[1].any() and not w[3].any()
    for s in (0, 2):
        xs, ts, bs = systems[s]
        er, fr, wr = oracle.compute(xs, ts, bs, table, oracle.neighbors(xs, bs, RC))
        assert abs(e[s] - er) <= 1e-10 * abs(er)
        assert np.abs(f[off[s]:off[s + 1]].cpu().numpy() - fr).max() <= 1e-10 * np.abs(fr).max()
    ctx.close()

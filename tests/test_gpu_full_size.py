"""Parity at the full sizes of the two workloads the oracle cannot evaluate
whole in seconds, on sampled outputs it computes one by one.

16,384,000-atom Si (the long-MD workload, list radius 4.0 A as in the bench):
the force on atom a depends only on atoms within 2 r_c of a, and its
per-centre energy on atoms within r_c; the oracle evaluates a cut-out of all
atoms within 6.5 A of each sampled atom (minimum image, placed in an empty
40 A box) and gives that atom's exact force and per-centre energy. FP64 path
1e-10 relative (per component, scaled by the largest sampled force); mixed
path force RMS 1e-5, per-atom energies 1e-5. At full size, properties: the
total energy equals the sum of the per-centre energies (FP64 1e-9; mixed 1e-6,
each warp's energies summed in float), and the forces sum to zero.

The 256-cell fitting batch (514,676 atoms): energies, forces and virials of
24 sampled cells against the oracle cell by cell, and the parameter VJP of
the energy for two table entries against the oracle's complex step summed
over every cell.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests import _systems as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RC = 3.0
CUT = 6.5


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1607_02904_gb300 as T
    T.load()
    return T


class Cutouts:
    """Atoms binned once into cells at least CUT wide; the cut-out around an
    atom gathers its 27 neighbouring cells."""

    def __init__(self, x, box):
        self.x, self.box = x, box
        self.nc = np.floor(box / CUT).astype(np.int64)
        c = np.floor(np.mod(x, box) / (box / self.nc)).astype(np.int64)
        c = np.minimum(c, self.nc - 1)
        cid = (c[:, 2] * self.nc[1] + c[:, 1]) * self.nc[0] + c[:, 0]
        self.order = np.argsort(cid, kind="stable")
        self.start = np.searchsorted(cid[self.order], np.arange(self.nc.prod() + 1))
        self.cell = c

    def around(self, a):
        c = self.cell[a]
        idx = []
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    q = np.mod(c + (dx, dy, dz), self.nc)
                    k = (q[2] * self.nc[1] + q[1]) * self.nc[0] + q[0]
                    idx.append(self.order[self.start[k]:self.start[k + 1]])
        idx = np.unique(np.concatenate(idx))
        d = self.x[idx] - self.x[a]
        d -= self.box * np.round(d / self.box)
        keep = (d * d).sum(axis=1) < CUT * CUT
        return idx[keep], d[keep]


def cutout_reference(cut, t, table, a):
    sel, d = cut.around(a)
    centre = int(np.nonzero(sel == a)[0][0])
    big = np.full(3, 40.0)
    xc = d + big / 2
    _, f, _, ea = oracle.compute(xc, t[sel], big, table, oracle.neighbors(xc, big, RC), eatom=True)
    return f[centre], ea[centre]


@pytest.fixture(scope="module")
def large():
    x, v, t, box, names = W.config_si_large()
    t = t.astype(np.int32)
    table = S.table_for(["Si"], oracle.mix_tersoff89)
    rng = np.random.Generator(np.random.Philox(150))
    sample = rng.choice(len(x), size=48, replace=False)
    cut = Cutouts(x, box)
    ref = [cutout_reference(cut, t, table, int(a)) for a in sample]
    return x, t, box, table, sample, np.array([r[0] for r in ref]), np.array([r[1] for r in ref])


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_si_16m_sampled_atoms(T, prec, large):
    x, t, box, table, sample, ref_f, ref_e = large
    assert len(x) == 16_384_000
    ctx = T.Context(prec)
    ctx.params(table)
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    ctx.neighbor_build(xd, torch.tensor(t, device="cuda"), box, RC + 1.0)
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    f = torch.zeros_like(xd)
    ea = torch.zeros(len(x), dtype=torch.float64, device="cuda")
    ctx.compute(xd, e, f)
    ctx.compute_peratom(xd, ea)
    torch.cuda.synchronize()
    e_tot = e.item()
    ea_sum = float(ea.sum().item())
    f_sum = f.sum(dim=0).cpu().numpy()
    f_abs = float(f.abs().sum().item())
    got_f = f[torch.tensor(sample, device="cuda")].cpu().numpy()
    got_e = ea[torch.tensor(sample, device="cuda")].cpu().numpy()
    ctx.close()
    if prec == 0:
        assert np.abs(got_f - ref_f).max() <= 1e-10 * np.abs(ref_f).max()
        assert np.abs(got_e - ref_e).max() <= 1e-10 * np.abs(ref_e).max()
    else:
        assert np.sqrt(((got_f - ref_f) ** 2).mean() / (ref_f ** 2).mean()) <= 1e-5
        assert np.abs(got_e - ref_e).max() <= 1e-5 * np.abs(ref_e).max()
    # (the mixed path sums each warp's energies in float before the double sums)
    assert abs(e_tot - ea_sum) <= (1e-9 if prec == 0 else 1e-6) * abs(e_tot)
    assert np.abs(f_sum).max() <= 1e-9 * f_abs / 3


def test_fitting_batch_256_cells(T):
    cells = W.batched_cells(n_cells=256)
    table = S.table_for(["Si", "C"], oracle.mix_tersoff89)
    off = np.cumsum([0] + [len(c[0]) for c in cells]).astype(np.int32)
    x = np.concatenate([c[0] for c in cells])
    t = np.concatenate([c[1] for c in cells]).astype(np.int32)
    boxes = np.stack([c[2] for c in cells])
    ctx = T.Context(T.MIXED)
    ctx.params(table)
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    ctx.neighbor_build_batched(xd, torch.tensor(t, device="cuda"), off, boxes, RC + 0.5)
    ns = len(cells)
    e = torch.full((ns,), np.nan, dtype=torch.float64, device="cuda")
    f = torch.full_like(xd, np.nan)
    w = torch.full((ns, 6), np.nan, dtype=torch.float64, device="cuda")
    ctx.compute_batched(xd, e, f, w)
    g = torch.zeros(table.size, dtype=torch.float64, device="cuda")
    ctx.backward(xd, torch.ones(ns, dtype=torch.float64, device="cuda"), None, None, g)
    torch.cuda.synchronize()
    e, f, w, g = e.cpu().numpy(), f.cpu().numpy(), w.cpu().numpy(), g.cpu().numpy()
    ctx.close()
    rng = np.random.Generator(np.random.Philox(151))
    for s in rng.choice(ns, size=24, replace=False):
        xs, ts, bs = cells[s]
        er, fr, wr = oracle.compute(xs, ts, bs, table, oracle.neighbors(xs, bs, RC))
        fs = f[off[s]:off[s + 1]]
        assert np.sqrt(((fs - fr) ** 2).mean() / (fr ** 2).mean()) <= 1e-5, s
        assert abs(e[s] - er) <= 1e-5 * abs(er), s
        assert np.abs(w[s] - wr).max() <= 1e-5 * np.abs(wr).max(), s
    # d(sum of energies)/d theta for A and lambda1 of record (Si, Si, Si)
    for p in (13, 12):
        ref = 0.0
        for xs, ts, bs in cells:
            de, _ = oracle.cs_param(xs, ts, bs, table, oracle.neighbors(xs, bs, RC), p)
            ref += de
        assert abs(g[p] - ref) <= 1e-5 * abs(ref), (p, g[p], ref)

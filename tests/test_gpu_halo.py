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

"""MD with displacement-triggered neighbour rebuilds (TERSOFF_REBUILD_ON_SKIN):
the list is rebuilt when some atom has moved more than half the skin since the
last build, decided on the device (a conditional graph node when the steps run
as a CUDA graph, a host check otherwise).

While the lists are valid the forces do not depend on when they were built, so
the FP64 trajectory must match the oracle's with a rebuild at every step (its
lists are always fresh), to the tolerances of the fixed-period MD parity test.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests import _systems as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RC = 3.0
SKIN = 0.3
MASS = [W.MASS_AMU["Si"]]


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1607_02904_gb300 as T
    T.load()
    return T


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def hot_si(ncell=3, temp=3000.0, seed=60):
    x, t, box = W.diamond(ncell, ncell, ncell, 5.432)
    rng = np.random.Generator(np.random.Philox(seed))
    x = W.jitter_gaussian(x, 0.05, rng)
    v = W.maxwell_velocities(t, np.array(MASS), temp, rng)
    return x, v, t, box


def run_gpu(T, prec, x, v, t, box, nsteps, graphs=True, calls=1):
    table = S.table_for(["Si"], oracle.mix_tersoff89)
    ctx = T.Context(prec)
    ctx.set_graphs(graphs)
    ctx.params(table)
    xd, vd = dev(x), dev(v)
    ctx.neighbor_build(xd, dev(t, torch.int32), box, RC + SKIN)
    fd = torch.zeros_like(xd)
    ctx.compute(xd, None, fd)
    th = torch.zeros((nsteps, 3), dtype=torch.float64, device="cuda")
    rebuilds = []
    for _ in range(calls):
        ctx.md_step(xd, vd, fd, MASS, 0.001, nsteps, T.REBUILD_ON_SKIN, th)
        rebuilds.append(ctx.md_rebuilds())
    torch.cuda.synchronize()
    out = (xd.cpu().numpy(), vd.cpu().numpy(), fd.cpu().numpy(), th.cpu().numpy(), rebuilds)
    ctx.close()
    return out


@pytest.mark.parametrize("graphs", [True, False], ids=["graph", "eager"])
def test_skin_triggered_fp64_matches_oracle(T, graphs):
    x, v, t, box = hot_si()
    nsteps = 60
    table = S.table_for(["Si"], oracle.mix_tersoff89)
    xo, vo, thermo_o, fo = oracle.md_run(x, v, t, box, table, MASS, 0.001, nsteps, RC + SKIN, 1)
    xg, vg, fg, thg, reb = run_gpu(T, T.FP64, x, v, t, box, nsteps, graphs)
    assert reb[0] >= 2  # 3000 K: atoms cross half of a 0.3 A skin several times
    assert np.abs(xg - xo).max() < 1e-9
    assert np.abs(vg - vo).max() < 1e-7
    assert np.abs(fg - fo).max() < 1e-8 * np.abs(fo).max()
    assert np.abs(thg - thermo_o).max() < 1e-8 * np.abs(thermo_o).max()


def test_graph_and_eager_agree_bitwise(T):
    # forces are gathered in a fixed order: both modes take the same rebuild
    # decisions and give the same trajectory bit for bit; repeated calls
    # replay the captured graph
    x, v, t, box = hot_si(seed=61)
    a = run_gpu(T, T.MIXED, x, v, t, box, 20, graphs=True, calls=3)
    b = run_gpu(T, T.MIXED, x, v, t, box, 20, graphs=False, calls=3)
    assert a[4] == b[4] and sum(a[4]) >= 2
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_no_rebuild_without_motion(T):
    x, t, box = W.diamond(3, 3, 3, 5.432)
    v = np.zeros_like(x)
    _, _, _, _, reb = run_gpu(T, T.MIXED, x, v, t, box, 20, graphs=True, calls=2)
    assert reb == [0, 0]


def test_fixed_period_rebuild_count(T):
    x, v, t, box = hot_si(seed=62)
    table = S.table_for(["Si"], oracle.mix_tersoff89)
    ctx = T.Context(T.MIXED)
    ctx.params(table)
    xd, vd = dev(x), dev(v)
    ctx.neighbor_build(xd, dev(t, torch.int32), box, RC + 1.0)
    fd = torch.zeros_like(xd)
    ctx.compute(xd, None, fd)
    counts = []
    for _ in range(3):
        ctx.md_step(xd, vd, fd, MASS, 0.001, 15, 10)
        counts.append(ctx.md_rebuilds())
    assert counts == [1, 2, 1]  # rebuilds after steps 10, 20, 30, 40 of 45
    with pytest.raises(T.TersoffError):
        ctx.md_step(xd, vd, fd, MASS, 0.001, 5, -2)
    ctx.close()


@pytest.mark.parametrize("graphs", [True, False], ids=["graph", "eager"])
def test_mixed_thermo_when_short_list_expires(T, graphs):
    # 3000 K, skin 0.5 A and no rebuild for 25 steps: after ~15 steps atoms
    # have moved beyond half the short-list margin (0.15 A) and the force
    # kernel scatters through the fallback buffer, while the skin list stays
    # valid (0.25 A). The mixed path's thermo must still follow the FP64 path.
    x, v, t, box = hot_si(seed=63)
    table = S.table_for(["Si"], oracle.mix_tersoff89)
    out = {}
    for prec in (T.FP64, T.MIXED):
        ctx = T.Context(prec)
        ctx.set_graphs(graphs)
        ctx.params(table)
        xd, vd = dev(x), dev(v)
        ctx.neighbor_build(xd, dev(t, torch.int32), box, RC + 0.5)
        fd = torch.zeros_like(xd)
        ctx.compute(xd, None, fd)
        th = torch.zeros((25, 3), dtype=torch.float64, device="cuda")
        ctx.md_step(xd, vd, fd, MASS, 0.001, 25, 0, th)
        torch.cuda.synchronize()
        out[prec] = th.cpu().numpy()
        ctx.close()
    d, m = out[T.FP64], out[T.MIXED]
    scale = np.abs(d[:, 2]).max()
    assert np.abs(m[:, 2] - d[:, 2]).max() <= 1e-6 * scale  # total energy
    assert np.abs(m[:, 1] - d[:, 1]).max() <= 1e-5 * np.abs(d[:, 1]).max()  # kinetic


@pytest.mark.parametrize("rebuild", [10, -1], ids=["every-10", "on-skin"])
def test_mixed_forces_after_in_graph_rebuild_match_oracle(T, rebuild):
    # Mixed path, MD steps as a replayed CUDA graph with the neighbour rebuild
    # inside it (a fixed period, or the conditional node of the displacement
    # trigger): the forces left in f after the call are F(x) at the final
    # positions, evaluated over the list rebuilt inside the graph; against the
    # FP64 oracle at those positions, to the mixed path's tolerance.
    x, v, t, box = hot_si(seed=64)
    table = S.table_for(["Si"], oracle.mix_tersoff89)
    ctx = T.Context(T.MIXED)
    ctx.params(table)
    xd, vd = dev(x), dev(v)
    ctx.neighbor_build(xd, dev(t, torch.int32), box, RC + SKIN)
    fd = torch.zeros_like(xd)
    ctx.compute(xd, None, fd)
    rebuilds = []
    for _ in range(3):  # the first call captures the graph, the others replay it
        ctx.md_step(xd, vd, fd, MASS, 0.001, 10, T.REBUILD_ON_SKIN if rebuild < 0 else rebuild)
        rebuilds.append(ctx.md_rebuilds())
    torch.cuda.synchronize()
    assert rebuilds[-1] >= 1 and sum(rebuilds) >= 3
    xg, fg = xd.cpu().numpy(), fd.cpu().numpy()
    ctx.close()
    _, fo, _ = oracle.compute(xg, t, box, table, oracle.neighbors(xg, box, RC))
    rms = np.sqrt(((fg - fo) ** 2).mean()) / np.sqrt((fo ** 2).mean())
    assert rms <= 1e-5, rms

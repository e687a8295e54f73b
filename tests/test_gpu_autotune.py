"""The autotuner and the launch options it chooses between.

Every option value must give the same results as the default launch, to the
parity tolerances against the oracle (FP64 1e-10 relative; mixed force RMS,
energy and virial 1e-5); the tuner must leave the caller's arrays untouched,
keep a valid list, and report its trials.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests import _systems as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RC = 3.0
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


# SiC: many atoms need register capacity 8 (bucket 1), so the split option matters
X, TY, BOX = S.sic_cell(n=5, sigma=0.1, seed=90)
TABLE = S.table_for(["Si", "C"], oracle.mix_tersoff89)
REF = oracle.compute(X, TY, BOX, TABLE, oracle.neighbors(X, BOX, RC))


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("waves,split,block", [(0, -1, 256), (1, -1, 256), (2, 0, 128),
                                               (4, 1, 512), (1, 1, 64), (0, 0, 512)])
def test_launch_options_keep_results(T, prec, waves, split, block):
    ctx = T.Context(prec)
    ctx.set_launch(waves, split, block)
    ctx.params(TABLE)
    xd = dev(X)
    ctx.neighbor_build(xd, dev(TY, torch.int32), BOX, RC + 0.5)
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    f = torch.zeros_like(xd)
    w = torch.zeros(6, dtype=torch.float64, device="cuda")
    ctx.compute(xd, e, f, w)
    torch.cuda.synchronize()
    check(prec, (e.item(), f.cpu().numpy(), w.cpu().numpy()), REF)
    ctx.close()


def test_set_launch_rejects_bad_values(T):
    ctx = T.Context(1)
    for bad in [(-1, -1, 256), (0, 2, 256), (0, -1, 1024), (0, -1, 96)]:
        with pytest.raises(T.TersoffError):
            ctx.set_launch(*bad)
    ctx.close()


def test_autotune_md_keeps_state_and_results(T):
    x, t, box = W.diamond(5, 5, 5, 5.432)
    rng = np.random.Generator(np.random.Philox(91))
    x = W.jitter_gaussian(x, 0.05, rng)
    v = W.maxwell_velocities(t, np.array(MASS), 1000.0, rng)
    table = S.table_for(["Si"], oracle.mix_tersoff89)
    ctx = T.Context(0)
    ctx.params(table)
    xd, vd = dev(x), dev(v)
    ctx.neighbor_build(xd, dev(t, torch.int32), box, RC + 1.0)
    summary = ctx.autotune(xd, vd, MASS, 0.001, 10)
    assert summary.startswith("chosen ") and summary.count("ms") >= 8
    assert np.array_equal(xd.cpu().numpy(), x) and np.array_equal(vd.cpu().numpy(), v)
    # the tuned context still runs MD equal to the oracle's
    fd = torch.zeros_like(xd)
    ctx.compute(xd, None, fd)
    ctx.md_step(xd, vd, fd, MASS, 0.001, 20, 10)
    torch.cuda.synchronize()
    xo, vo, _, fo = oracle.md_run(x, v, t, box, table, MASS, 0.001, 20, RC + 1.0, 10)
    assert np.abs(xd.cpu().numpy() - xo).max() < 1e-9
    assert np.abs(fd.cpu().numpy() - fo).max() < 1e-8 * np.abs(fo).max()
    ctx.close()


def test_autotune_batch_compute(T):
    cells = W.batched_cells(n_cells=4, nmin=64, nmax=400, seed_k=93)
    off = np.cumsum([0] + [len(c[0]) for c in cells]).astype(np.int32)
    x = np.concatenate([c[0] for c in cells])
    t = np.concatenate([c[1] for c in cells]).astype(np.int32)
    boxes = np.stack([c[2] for c in cells])
    ctx = T.Context(1)
    ctx.params(TABLE)
    xd = dev(x)
    ctx.neighbor_build_batched(xd, dev(t, torch.int32), off, boxes, RC + 0.5)
    summary = ctx.autotune(xd)
    assert summary.startswith("chosen ") and "split" in summary
    e = torch.zeros(len(cells), dtype=torch.float64, device="cuda")
    f = torch.zeros_like(xd)
    w = torch.zeros((len(cells), 6), dtype=torch.float64, device="cuda")
    ctx.compute_batched(xd, e, f, w)
    torch.cuda.synchronize()
    for s, (xs, ts, bs) in enumerate(cells):
        ref = oracle.compute(xs, ts, bs, TABLE, oracle.neighbors(xs, bs, RC))
        check(1, (e[s].item(), f[off[s]:off[s + 1]].cpu().numpy(), w[s].cpu().numpy()), ref)
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("flags", [1, 2, 3, 8, 9])
def test_ablations_keep_results(T, prec, flags):
    ctx = T.Context(prec)
    ctx.set_ablation(flags)
    ctx.params(TABLE)
    xd = dev(X)
    ctx.neighbor_build(xd, dev(TY, torch.int32), BOX, RC + 0.5)
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    f = torch.zeros_like(xd)
    w = torch.zeros(6, dtype=torch.float64, device="cuda")
    ctx.compute(xd, e, f, w)
    torch.cuda.synchronize()
    check(prec, (e.item(), f.cpu().numpy(), w.cpu().numpy()), REF)
    with pytest.raises(T.TersoffError):
        ctx.set_ablation(32)
    ctx.close()


@pytest.mark.parametrize("scatter", [0, 1], ids=["gather", "atomic"])
def test_fp32_sums_ablation(T, scatter):
    # plain float force sums (the paper's all-single accumulation): still within
    # the mixed path's tolerance of the oracle; in gather mode they differ from
    # the compensated sums, in atomic mode (FP64 atomics) they are not used
    def run(flags):
        ctx = T.Context(T.MIXED)
        ctx.set_scatter(scatter)
        ctx.set_ablation(flags)
        ctx.params(TABLE)
        xd = dev(X)
        ctx.neighbor_build(xd, dev(TY, torch.int32), BOX, RC + 0.5)
        e = torch.zeros(1, dtype=torch.float64, device="cuda")
        f = torch.zeros_like(xd)
        w = torch.zeros(6, dtype=torch.float64, device="cuda")
        ctx.compute(xd, e, f, w)
        torch.cuda.synchronize()
        out = (e.item(), f.cpu().numpy(), w.cpu().numpy())
        ctx.close()
        return out
    plain, comp = run(T.ABLATE_FP32_SUMS), run(0)
    check(1, plain, REF)
    if scatter == 0:
        assert not np.array_equal(plain[1], comp[1])
    else:
        assert np.abs(plain[1] - comp[1]).max() <= 1e-12 * np.abs(comp[1]).max()


# The fast-forward lane scheme (Sec. IV-C, Fig. 2) over the full skin list:
# lanes of a warp hold atoms with different numbers of bonds and of skin
# entries (random packings, lambda3 tables, a ragged last warp), in both paths
# and both scatter modes, against the oracle.
FF_CASES = []
_xp, _tp, _bp = S.packing_cell(n=300, seed=95)
FF_CASES.append(("packing", _xp, _tp, _bp, TABLE))
_xs, _ts, _bs = S.si_cell(n=3, seed=96, amp=0.3)
FF_CASES.append(("si-l3m3", _xs, _ts, _bs,
                 S.with_lambda3(S.table_for(["Si"], oracle.mix_tersoff89), 1.7322, 3)))
FF_CASES.append(("sic", X, TY, BOX, TABLE))


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("scatter", [0, 1], ids=["gather", "atomic"])
@pytest.mark.parametrize("case", FF_CASES, ids=[c[0] for c in FF_CASES])
def test_fastforward_ablation_against_oracle(T, prec, scatter, case):
    _, x, t, box, table = case
    ref = oracle.compute(x, t, box, table, oracle.neighbors(x, box, RC))
    ctx = T.Context(prec)
    ctx.set_scatter(scatter)
    ctx.set_ablation(T.ABLATE_FASTFWD)
    ctx.params(table)
    xd = dev(x)
    ctx.neighbor_build(xd, dev(t, torch.int32), box, RC + 1.0)
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    f = torch.zeros_like(xd)
    w = torch.zeros(6, dtype=torch.float64, device="cuda")
    ea = torch.zeros(len(x), dtype=torch.float64, device="cuda")
    for _ in range(2):  # the fallback buffer is cleared by the gather between calls
        ctx.compute(xd, e, f, w)
    ctx.compute_peratom(xd, ea)
    torch.cuda.synchronize()
    check(prec, (e.item(), f.cpu().numpy(), w.cpu().numpy()), ref)
    _, _, _, ea_ref = oracle.compute(x, t, box, table, oracle.neighbors(x, box, RC), eatom=True)
    tol = 1e-10 if prec == 0 else 1e-5
    assert np.abs(ea.cpu().numpy() - ea_ref).max() <= tol * np.abs(ea_ref).max()
    # switching back to the default path gives the default results
    ctx.set_ablation(0)
    f2 = torch.zeros_like(xd)
    ctx.compute(xd, None, f2)
    torch.cuda.synchronize()
    check(prec, (ref[0], f2.cpu().numpy(), ref[2]), ref)
    ctx.close()


def test_fastforward_ablation_md_fp64_against_oracle(T):
    x, t, box = W.diamond(4, 4, 4, 5.432)
    rng = np.random.Generator(np.random.Philox(97))
    x = W.jitter_gaussian(x, 0.05, rng)
    v = W.maxwell_velocities(t, np.array(MASS), 1000.0, rng)
    table = S.table_for(["Si"], oracle.mix_tersoff89)
    ctx = T.Context(0)
    ctx.set_ablation(T.ABLATE_FASTFWD)
    ctx.params(table)
    xd, vd = dev(x), dev(v)
    ctx.neighbor_build(xd, dev(t, torch.int32), box, RC + 1.0)
    fd = torch.zeros_like(xd)
    ctx.compute(xd, None, fd)
    ctx.md_step(xd, vd, fd, MASS, 0.001, 20, 10)
    torch.cuda.synchronize()
    xo, vo, _, fo = oracle.md_run(x, v, t, box, table, MASS, 0.001, 20, RC + 1.0, 10)
    assert np.abs(xd.cpu().numpy() - xo).max() < 1e-9
    assert np.abs(fd.cpu().numpy() - fo).max() < 1e-8 * np.abs(fo).max()
    ctx.close()


@pytest.mark.parametrize("case", ["si", "si-l3m3"])
def test_compensated_atom_sums_variant(T, case):
    # Compensated per-atom sums carried into double (mixed path, one species):
    # within the mixed tolerance of the oracle, and at least as close to the
    # oracle as the plain float per-atom sums under the same (atomic) scatter.
    table = S.table_for(["Si"], oracle.mix_tersoff89)
    if case == "si-l3m3":
        table = S.with_lambda3(table, 1.7322, 3)
    x, t, box = S.si_cell(n=4, seed=98, amp=0.2)
    ref = oracle.compute(x, t, box, table, oracle.neighbors(x, box, RC))

    def run(flags):
        ctx = T.Context(T.MIXED)
        ctx.set_scatter(T.SCATTER_ATOMIC)
        ctx.set_ablation(flags)
        ctx.params(table)
        xd = dev(x)
        ctx.neighbor_build(xd, dev(t, torch.int32), box, RC + 1.0)
        e = torch.zeros(1, dtype=torch.float64, device="cuda")
        f = torch.zeros_like(xd)
        w = torch.zeros(6, dtype=torch.float64, device="cuda")
        ea = torch.zeros(len(x), dtype=torch.float64, device="cuda")
        ctx.compute(xd, e, f, w)
        ctx.compute_peratom(xd, ea)
        torch.cuda.synchronize()
        out = (e.item(), f.cpu().numpy(), w.cpu().numpy(), ea.cpu().numpy())
        ctx.close()
        return out

    comp, plain = run(T.ABLATE_COMP_ATOM_SUMS), run(0)
    check(1, comp[:3], ref)
    _, _, _, ea_ref = oracle.compute(x, t, box, table, oracle.neighbors(x, box, RC), eatom=True)
    assert np.abs(comp[3] - ea_ref).max() <= 1e-5 * np.abs(ea_ref).max()
    err = lambda f: np.sqrt(((f - ref[1]) ** 2).mean())
    assert err(comp[1]) <= 1.5 * err(plain[1])


def test_compensated_atom_sums_md_gather_mode(T):
    # in the default gather mode the variant scatters through FP64 atomics;
    # MD still follows the FP64 oracle's trajectory to the mixed tolerance
    x, t, box = W.diamond(4, 4, 4, 5.432)
    rng = np.random.Generator(np.random.Philox(99))
    x = W.jitter_gaussian(x, 0.05, rng)
    v = W.maxwell_velocities(t, np.array(MASS), 1000.0, rng)
    table = S.table_for(["Si"], oracle.mix_tersoff89)
    ctx = T.Context(T.MIXED)
    ctx.set_ablation(T.ABLATE_COMP_ATOM_SUMS)
    ctx.params(table)
    xd, vd = dev(x), dev(v)
    ctx.neighbor_build(xd, dev(t, torch.int32), box, RC + 1.0)
    fd = torch.zeros_like(xd)
    ctx.compute(xd, None, fd)
    ctx.md_step(xd, vd, fd, MASS, 0.001, 20, 10)
    torch.cuda.synchronize()
    xo, vo, _, fo = oracle.md_run(x, v, t, box, table, MASS, 0.001, 20, RC + 1.0, 10)
    assert np.abs(xd.cpu().numpy() - xo).max() < 1e-6
    fg = fd.cpu().numpy()
    assert np.sqrt(((fg - fo) ** 2).mean()) / np.sqrt((fo ** 2).mean()) <= 1e-5
    ctx.close()

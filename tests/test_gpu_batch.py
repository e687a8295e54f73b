"""Batches of independent periodic systems in one context (the fitting
workload): per-system energy, forces and virial from one launch over all atoms,
the parameter VJP with one energy weight per system, and a whole fitting step
(forward, loss gradient, backward) captured in one CUDA graph.

References are the oracle evaluated system by system. Tolerances as in the
single-system parity tests (FP64 1e-10 relative; mixed force RMS, energy and
virial 1e-5; parameter VJP compared scaled by the parameter values, FP64 1e-10,
mixed 1e-5).
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests import _systems as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RC = 3.0
R_LIST = RC + 0.5


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1607_02904_gb300 as T
    T.load()
    return T


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def make_batch():
    cells = W.batched_cells(n_cells=5, nmin=64, nmax=500, seed_k=40)
    x, t, box = S.si_cell(n=3, amp=0.2, seed=41)
    cells.append((x, t, box))
    x, t, box = S.sic_cell(n=3, sigma=0.12, seed=42)
    cells.append((x, t, box))
    x, t, box = S.packing_cell(n=64, c_frac=1.0, seed=43)  # smallest box: all C
    cells.append((x, t, box))
    off = np.cumsum([0] + [len(c[0]) for c in cells]).astype(np.int32)
    return cells, off


CELLS, OFF = make_batch()
TABLE = S.table_for(["Si", "C"], oracle.mix_tersoff89)


def concat():
    x = np.concatenate([c[0] for c in CELLS])
    t = np.concatenate([c[1] for c in CELLS]).astype(np.int32)
    boxes = np.stack([c[2] for c in CELLS])
    return x, t, boxes


def oracle_refs():
    out = []
    for x, t, box in CELLS:
        out.append(oracle.compute(x, t, box, TABLE, oracle.neighbors(x, box, RC)))
    return out


REFS = oracle_refs()


def batch_ctx(T, prec):
    x, t, boxes = concat()
    ctx = T.Context(prec)
    ctx.params(TABLE)
    xd = dev(x)
    ctx.neighbor_build_batched(xd, dev(t, torch.int32), OFF, boxes, R_LIST)
    return ctx, xd


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("scatter", [0, 1], ids=["gather", "atomic"])
def test_batched_compute_matches_oracle(T, prec, scatter):
    ctx, xd = batch_ctx(T, prec)
    ctx.set_scatter(scatter)
    ns = len(CELLS)
    e = torch.full((ns,), np.nan, dtype=torch.float64, device="cuda")
    f = torch.full_like(xd, np.nan)
    w = torch.full((ns, 6), np.nan, dtype=torch.float64, device="cuda")
    ctx.compute_batched(xd, e, f, w)
    torch.cuda.synchronize()
    e, f, w = e.cpu().numpy(), f.cpu().numpy(), w.cpu().numpy()
    for s, (er, fr, wr) in enumerate(REFS):
        fs = f[OFF[s]:OFF[s + 1]]
        if prec == 0:
            assert abs(e[s] - er) <= 1e-10 * abs(er)
            assert np.abs(fs - fr).max() <= 1e-10 * np.abs(fr).max()
            assert np.abs(w[s] - wr).max() <= 1e-10 * np.abs(wr).max()
        else:
            rms = np.sqrt(((fs - fr) ** 2).mean()) / np.sqrt((fr ** 2).mean())
            assert rms <= 1e-5, (s, rms)
            assert abs(e[s] - er) <= 1e-5 * abs(er)
            assert np.abs(w[s] - wr).max() <= 1e-5 * np.abs(wr).max()
    ctx.close()


def _bcc_dense(n, a, seed):
    # 8 first and 6 second neighbours inside the Si cutoff: more than 8 bonds
    g = np.arange(n)
    base = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    x = np.concatenate([base, base + 0.5]) * a
    rng = np.random.Generator(np.random.Philox(seed))
    box = np.full(3, n * a)
    return W.jitter_gaussian(x, 0.04, rng) % box, np.zeros(len(x), np.int32), box


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_batch_with_dense_cells_wide_kernel(T, prec):
    # two dense bcc cells (every atom has 13-14 bonds inside the cutoff: the
    # batch variant of the wide kernel), a SiC crystal and a packing (the
    # capacity-4 and capacity-8 launches) in one batch, against the oracle
    cells = [_bcc_dense(5, 2.9, 140), S.sic_cell(n=3, sigma=0.12, seed=141),
             _bcc_dense(4, 2.95, 142), S.packing_cell(n=120, c_frac=0.4, seed=143)]
    off = np.cumsum([0] + [len(c[0]) for c in cells]).astype(np.int32)
    x = np.concatenate([c[0] for c in cells])
    t = np.concatenate([c[1] for c in cells]).astype(np.int32)
    boxes = np.stack([c[2] for c in cells])
    ctx = T.Context(prec)
    ctx.params(TABLE)
    xd = dev(x)
    ctx.neighbor_build_batched(xd, dev(t, torch.int32), off, boxes, R_LIST)
    ns = len(cells)
    e = torch.full((ns,), np.nan, dtype=torch.float64, device="cuda")
    f = torch.full_like(xd, np.nan)
    w = torch.full((ns, 6), np.nan, dtype=torch.float64, device="cuda")
    ctx.compute_batched(xd, e, f, w)
    torch.cuda.synchronize()
    e, f, w = e.cpu().numpy(), f.cpu().numpy(), w.cpu().numpy()
    ctx.close()
    for s, (xs, ts, bs) in enumerate(cells):
        er, fr, wr = oracle.compute(xs, ts, bs, TABLE, oracle.neighbors(xs, bs, RC))
        fs = f[off[s]:off[s + 1]]
        tol = 1e-10 if prec == 0 else 1e-5
        if prec == 0:
            assert np.abs(fs - fr).max() <= tol * np.abs(fr).max()
        else:
            assert np.sqrt(((fs - fr) ** 2).mean() / (fr ** 2).mean()) <= tol
        assert abs(e[s] - er) <= tol * abs(er)
        assert np.abs(w[s] - wr).max() <= tol * np.abs(wr).max()


def test_batched_lists_bit_exact(T):
    ctx, xd = batch_ctx(T, 1)
    cap, mx = ctx.neighbor_capacity()
    cnt, nbr, st = ctx.neighbor_export(mx)
    assert st == 0
    cnt, nbr = cnt.cpu().numpy(), nbr.cpu().numpy()
    for s, (x, t, box) in enumerate(CELLS):
        cr, nr = oracle.neighbors(x, box, R_LIST)
        rows = slice(OFF[s], OFF[s + 1])
        assert np.array_equal(cnt[rows], cr)
        ref = np.where(nr[:, :mx] >= 0, nr[:, :mx] + OFF[s], -1)
        got = nbr[rows]
        assert np.array_equal(got[:, :ref.shape[1]], ref)
    ctx.close()


def _vjp_ref(gE, gF):
    g = np.zeros(TABLE.size)
    for s, (x, t, box) in enumerate(CELLS):
        nl = oracle.neighbors(x, box, RC)
        gfs = gF[OFF[s]:OFF[s + 1]]
        for p in range(TABLE.size):
            if p % oracle.NPAR == 0:
                continue
            de, df = oracle.cs_param(x, t, box, TABLE, nl, p)
            g[p] += gE[s] * de + float((gfs * df).sum())
    return g


def _scaled_err(got, ref):
    s = np.where(TABLE != 0.0, np.abs(TABLE), 1.0)
    return np.abs(s * (got - ref)).max() / np.abs(s * ref).max()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_batched_backward_matches_oracle(T, prec):
    rng = np.random.Generator(np.random.Philox(44))
    gE = rng.uniform(0.5, 2.0, size=len(CELLS))
    gF = rng.normal(0.0, 1.0, size=(OFF[-1], 3))
    ctx, xd = batch_ctx(T, prec)
    g = torch.full((TABLE.size,), np.nan, dtype=torch.float64, device="cuda")
    ctx.backward(xd, dev(gE), dev(gF), None, g)
    gx = torch.full_like(xd, np.nan)
    ctx.backward(xd, dev(gE), None, gx, None)
    f = torch.zeros_like(xd)
    ctx.compute_batched(xd, None, f, None)
    torch.cuda.synchronize()
    err = _scaled_err(g.cpu().numpy(), _vjp_ref(gE, gF))
    assert err <= (1e-10 if prec == 0 else 1e-5), err
    scale = np.repeat(gE, np.diff(OFF))[:, None]
    assert np.array_equal(gx.cpu().numpy(), -scale * f.cpu().numpy())
    ctx.close()


def test_single_system_batch_equals_single_context(T):
    x, t, box = CELLS[1]
    ctx = T.Context(0)
    ctx.params(TABLE)
    xd = dev(x)
    ctx.neighbor_build_batched(xd, dev(t, torch.int32), [0, len(x)], box[None, :], R_LIST)
    e1 = torch.zeros(1, dtype=torch.float64, device="cuda")
    f1 = torch.zeros_like(xd)
    w1 = torch.zeros((1, 6), dtype=torch.float64, device="cuda")
    ctx.compute_batched(xd, e1, f1, w1)
    with pytest.raises(T.TersoffError) as ei:  # batch mode: the single calls refuse
        ctx.compute(xd, e1, f1)
    assert ei.value.code == 7
    ctx.neighbor_build(xd, dev(t, torch.int32), box, R_LIST)  # back to one system
    e2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    f2 = torch.zeros_like(xd)
    w2 = torch.zeros(6, dtype=torch.float64, device="cuda")
    ctx.compute(xd, e2, f2, w2)
    torch.cuda.synchronize()
    assert abs(e1.item() - e2.item()) <= 1e-12 * abs(e2.item())
    assert torch.allclose(f1, f2, rtol=0, atol=1e-12 * f2.abs().max().item())
    assert torch.allclose(w1[0], w2, rtol=0, atol=1e-12 * w2.abs().max().item())
    ctx.close()


def test_batched_errors(T):
    x, t, boxes = concat()
    ctx = T.Context(1)
    ctx.params(TABLE)
    xd, td = dev(x), dev(t, torch.int32)
    with pytest.raises(T.TersoffError):  # offsets must end at n
        ctx.neighbor_build_batched(xd, td, OFF[:-1], boxes[:-1], R_LIST)
    small = boxes.copy()
    small[0] = 2.0 * R_LIST - 0.1
    with pytest.raises(T.TersoffError) as ei:
        ctx.neighbor_build_batched(xd, td, OFF, small, R_LIST)
    assert ei.value.code == 2
    ctx.close()


def test_fitting_step_in_one_cuda_graph(T):
    # forward, loss gradient (torch elementwise ops) and backward captured in
    # one CUDA graph; its replay equals the eager sequence
    ctx, xd = batch_ctx(T, 1)
    ns = len(CELLS)
    rng = np.random.Generator(np.random.Philox(45))
    e_ref = dev(np.array([r[0] for r in REFS]) + rng.normal(0.0, 1.0, ns))
    f_ref = dev(np.concatenate([r[1] for r in REFS]) + rng.normal(0.0, 0.1, (OFF[-1], 3)))
    e = torch.zeros(ns, dtype=torch.float64, device="cuda")
    f = torch.zeros_like(xd)
    gE = torch.zeros_like(e)
    gF = torch.zeros_like(f)
    grad = torch.zeros(TABLE.size, dtype=torch.float64, device="cuda")

    def step():
        ctx.compute_batched(xd, e, f, None)
        torch.mul(e - e_ref, 2.0, out=gE)
        torch.mul(f - f_ref, 2.0, out=gF)
        ctx.backward(xd, gE, gF, None, grad)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    eager = grad.clone()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    grad.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.allclose(grad, eager, rtol=1e-9, atol=0)
    ctx.close()


def test_autograd_batch_fitting_loss_eager_and_graph(T):
    # loss = sum_s (E_s - E0_s)^2 + sum_a |F_a - F0_a|^2 through the autograd
    # Function: the eager gradient (warm-up on a side stream, as whole-network
    # CUDA-graph capture requires) against the oracle; forward and backward
    # captured in one CUDA graph reproduce it
    x, t, boxes = concat()
    system = T.TersoffBatch(t, OFF, boxes, R_LIST, precision=0)
    tab = torch.tensor(TABLE, dtype=torch.float64, device="cuda", requires_grad=True)
    xd = dev(x)
    rng = np.random.Generator(np.random.Philox(46))
    e0 = dev(np.array([r[0] for r in REFS]) + rng.normal(0.0, 1.0, len(CELLS)))
    f0 = dev(np.concatenate([r[1] for r in REFS]) + rng.normal(0.0, 0.1, (OFF[-1], 3)))

    def loss_fn():
        E, F = T.energy_forces(system, xd, tab)
        return ((E - e0) ** 2).sum() + ((F - f0) ** 2).sum(), E, F

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            tab.grad = None
            loss, E, F = loss_fn()
            loss.backward()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    eager = tab.grad.clone()
    gE = 2.0 * (E.detach().cpu().numpy() - e0.cpu().numpy())
    gF = 2.0 * (F.detach().cpu().numpy() - f0.cpu().numpy())
    assert _scaled_err(eager.cpu().numpy(), _vjp_ref(gE, gF)) <= 1e-10

    tab.grad = None
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        static_loss = loss_fn()[0]
        static_loss.backward()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.allclose(tab.grad, eager, rtol=1e-9, atol=0)
    assert abs(static_loss.item() - loss.item()) <= 1e-9 * abs(loss.item())

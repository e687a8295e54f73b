"""GPU backward (tersoff_backward and the autograd Function) against the oracle.

The reference gradient of L = gE E + sum_a gF_a . F_a with respect to table
entry p is gE dE/dtheta_p + sum_a gF_a . dF_a/dtheta_p, with both derivatives
from the oracle's complex step (exact to rounding; pinned against finite
differences in the oracle tests). Entries are compared scaled by their
parameter value, s_p = theta_p dL/dtheta_p (the change of L under a relative
change of theta_p), so that entries of very different units share one scale:
  FP64 path   max_p |s_p - s_p,ref| <= 1e-10 max_p |s_p,ref|
  mixed path  max_p |s_p - s_p,ref| <= 1e-5  max_p |s_p,ref|
(entries with theta_p = 0, e.g. lambda3 of the Tersoff 1989 tables, are
scaled by 1). Field m is an integer and must get exactly 0.
"""
import functools

import numpy as np
import pytest

import oracle
import workloads as W
from tests import _systems as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RC = 3.0
TOL = {0: 1e-10, 1: 1e-5}


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1607_02904_gb300 as T
    T.load()
    return T


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _systems():
    si = S.table_for(["Si"], oracle.mix_tersoff89)
    sic = S.table_for(["Si", "C"], oracle.mix_tersoff89)
    out = {}
    x, t, box = S.si_cell(n=3, amp=0.3, seed=81)
    out["si"] = (x, t, box, si)
    out["si-l3m3"] = (x, t, box, S.with_lambda3(si, 1.7322, 3))
    out["si-l3m1"] = (x, t, box, S.with_lambda3(si, 1.3, 1))
    x, t, box = S.sic_cell(n=3, sigma=0.15, seed=82)
    out["sic"] = (x, t, box, sic)
    x, t, box = S.packing_cell(n=200, c_frac=0.5, seed=83)
    out["pack"] = (x, t, box, sic)
    return out


SYS = _systems()


def weights(n, seed, with_f=True):
    rng = np.random.Generator(np.random.Philox(seed))
    gE = float(rng.uniform(0.5, 2.0))
    gF = rng.normal(0.0, 1.0, size=(n, 3)) if with_f else None
    return gE, gF


@functools.lru_cache(maxsize=None)
def oracle_grad(name, with_f):
    x, t, box, table = SYS[name]
    gE, gF = weights(len(x), 91, with_f)
    nl = oracle.neighbors(x, box, RC)
    g = np.zeros(table.size)
    for p in range(table.size):
        if p % oracle.NPAR == 0:  # m
            continue
        de, df = oracle.cs_param(x, t, box, table, nl, p)
        g[p] = gE * de + (float((gF * df).sum()) if gF is not None else 0.0)
    return g


def scaled_err(table, got, ref):
    s = np.where(table != 0.0, np.abs(table), 1.0)
    return np.abs(s * (got - ref)).max() / np.abs(s * ref).max()


# Per entry: every entry whose scaled value is at least FLOOR of the largest
# must also match on its own, to TOL_ENTRY relative.
FLOOR = 1e-3
TOL_ENTRY = {0: 1e-8, 1: 1e-3}


def entry_err(table, got, ref):
    s = np.where(table != 0.0, np.abs(table), 1.0)
    big = np.abs(s * ref) >= FLOOR * np.abs(s * ref).max()
    return (np.abs(got - ref)[big] / np.abs(ref)[big]).max()


def gpu_grad(T, prec, name, with_f):
    x, t, box, table = SYS[name]
    gE, gF = weights(len(x), 91, with_f)
    ctx = T.Context(prec)
    ctx.params(table)
    xd = dev(x)
    ctx.neighbor_build(xd, dev(t, torch.int32), box, RC + 0.5)
    g = torch.full((table.size,), np.nan, dtype=torch.float64, device="cuda")
    ctx.backward(xd, dev([gE]), dev(gF) if gF is not None else None, None, g)
    torch.cuda.synchronize()
    ctx.close()
    return g.cpu().numpy()


@pytest.mark.parametrize("name", list(SYS))
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_param_vjp_matches_oracle(T, prec, name):
    x, t, box, table = SYS[name]
    got = gpu_grad(T, prec, name, True)
    ref = oracle_grad(name, True)
    assert np.isfinite(got).all()
    assert np.all(got[::oracle.NPAR] == 0.0)  # m
    err = scaled_err(table, got, ref)
    assert err <= TOL[prec], err
    e1 = entry_err(table, got, ref)
    assert e1 <= TOL_ENTRY[prec], e1


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_energy_only_vjp_matches_oracle(T, prec):
    x, t, box, table = SYS["pack"]
    got = gpu_grad(T, prec, "pack", False)
    ref = oracle_grad("pack", False)
    assert scaled_err(table, got, ref) <= TOL[prec]


def test_param_vjp_matches_finite_differences(T):
    # central differences of the GPU FP64 forward, step 1e-6 relative
    name = "si-l3m1"
    x, t, box, table = SYS[name]
    gE, gF = weights(len(x), 91, True)
    got = gpu_grad(T, 0, name, True)
    ctx = T.Context(0)
    xd, td = dev(x), dev(t, torch.int32)
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    f = torch.zeros_like(xd)

    def loss(tab):
        ctx.params(tab)
        ctx.neighbor_build(xd, td, box, RC + 0.5)
        ctx.compute(xd, e, f)
        torch.cuda.synchronize()
        return gE * e.item() + float((gF * f.cpu().numpy()).sum())

    fd = np.zeros(table.size)
    for p in range(1, table.size):
        h = 1e-6 * abs(table[p])
        tp, tm = table.copy(), table.copy()
        tp[p] += h
        tm[p] -= h
        fd[p] = (loss(tp) - loss(tm)) / (2 * h)
    ctx.close()
    assert scaled_err(table, got, fd) <= 1e-6


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_autograd_position_gradient_is_minus_forces(T, prec):
    x, t, box, table = SYS["pack"]
    system = T.TersoffSystem(t, box, RC + 0.5, precision=prec)
    xd = dev(x).requires_grad_(True)
    tab = torch.tensor(table, dtype=torch.float64)
    E, F = T.energy_forces(system, xd, tab)
    E.backward()
    assert torch.equal(xd.grad, -F.detach())
    ref = oracle.compute(x, t, box, table, oracle.neighbors(x, box, RC))
    if prec == 0:
        assert abs(E.item() - ref[0]) <= 1e-10 * abs(ref[0])
        assert np.abs(-xd.grad.cpu().numpy() - ref[1]).max() <= 1e-10 * np.abs(ref[1]).max()


def test_autograd_force_matching_loss(T):
    # loss = (E - E0)^2 + sum (F - F0)^2: gE = 2 (E - E0), gF = 2 (F - F0)
    name = "pack"
    x, t, box, table = SYS[name]
    system = T.TersoffSystem(t, box, RC + 0.5, precision=0)
    rng = np.random.Generator(np.random.Philox(92))
    E0 = -700.0
    F0 = rng.normal(0.0, 0.5, size=x.shape)
    tab = torch.tensor(table, dtype=torch.float64, requires_grad=True)
    xd = dev(x)
    E, F = T.energy_forces(system, xd, tab)
    loss = (E - E0) ** 2 + ((F - dev(F0)) ** 2).sum()
    loss.backward()
    gE = 2.0 * (E.item() - E0)
    gF = 2.0 * (F.detach().cpu().numpy() - F0)
    nl = oracle.neighbors(x, box, RC)
    ref = np.zeros(table.size)
    for p in range(table.size):
        if p % oracle.NPAR == 0:
            continue
        de, df = oracle.cs_param(x, t, box, table, nl, p)
        ref[p] = gE * de + float((gF * df).sum())
    assert scaled_err(table, tab.grad.numpy(), ref) <= 1e-10


def test_backward_error_codes(T):
    x, t, box, table = SYS["si"]
    ctx = T.Context(1)
    ctx.params(table)
    xd = dev(x)
    g = torch.zeros(table.size, dtype=torch.float64, device="cuda")
    with pytest.raises(T.TersoffError) as ei:  # no list yet
        ctx.backward(xd, dev([1.0]), None, None, g)
    assert ei.value.code == 7
    ctx.neighbor_build(xd, dev(t, torch.int32), box, RC + 0.5)
    with pytest.raises(T.TersoffError) as ei:  # atom count differs from the build
        ctx.backward(xd[:-1].contiguous(), dev([1.0]), None, None, g)
    assert ei.value.code == 1
    ctx.close()

"""Position gradient of an energy-and-force loss (tersoff_backward with grad_x
and force weights): the Hessian-vector product.

For L = gE E + sum_b gF_b . F_b the reference is
  dL/dx_{a,c} = gE dE/dx_{a,c} + sum_b gF_b . dF_b/dx_{a,c},
both derivatives from the oracle's complex step in position (exact to
rounding; the force derivative is pinned against finite differences of the
oracle's forces and the Hessian's symmetry in the oracle tests), every
coordinate of every atom.

Tolerances: FP64 max |g - g_ref| <= 1e-10 max |g_ref|; mixed path (per-term
float, like the forces) RMS |g - g_ref| <= 1e-5 RMS |g_ref|.

At the 512,000-atom Si workload, where the oracle is too slow for every
coordinate, properties that hold at any size: H is symmetric
(v . H u = u . H v), the rows of H sum to zero (translation invariance),
a uniform gF gives zero, and -H u equals the central difference of the
forces along u.
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


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1607_02904_gb300 as T
    T.load()
    return T


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def bcc_dense(n=5, a=2.9, seed=101):
    # 8 first and 6 second neighbours inside the Si cutoff (3.0 A): more bonds
    # per atom than the kernel's shared-memory slots
    g = np.arange(n)
    base = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    x = np.concatenate([base, base + 0.5]) * a
    rng = np.random.Generator(np.random.Philox(seed))
    box = np.full(3, n * a)
    return W.jitter_gaussian(x, 0.04, rng) % box, np.zeros(len(x), np.int32), box


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
    x, t, box = bcc_dense()
    out["bcc-dense"] = (x, t, box, si)
    return out


SYS = _systems()


def weights(x, seed):
    rng = np.random.Generator(np.random.Philox(seed))
    return 0.7, rng.normal(0.0, 1.0, size=x.shape)


@functools.lru_cache(maxsize=None)
def reference(name):
    x, t, box, table = SYS[name]
    gE, gF = weights(x, 102)
    nl = oracle.neighbors(x, box, RC)
    ref = np.zeros_like(x)
    for a in range(len(x)):
        for c in range(3):
            de, df = oracle.cs_pos(x, t, box, table, nl, a, c, forces=True)
            ref[a, c] = gE * de + float((gF * df).sum())
    return ref


def check(prec, got, ref):
    if prec == 0:
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= 1e-10, err
    else:
        err = np.sqrt(((got - ref) ** 2).mean() / (ref ** 2).mean())
        assert err <= 1e-5, err


def run_hvp(T, prec, x, t, box, table, gE, gF, r_list=RC + 0.5):
    ctx = T.Context(prec)
    ctx.params(table)
    xd = dev(x)
    ctx.neighbor_build(xd, dev(t, torch.int32), box, r_list)
    gx = torch.full_like(xd, np.nan)
    ctx.backward(xd, dev([gE]), None if gF is None else dev(gF), gx, None)
    torch.cuda.synchronize()
    out = gx.cpu().numpy()
    ctx.close()
    return out


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name", list(SYS))
def test_hvp_matches_oracle(T, prec, name):
    x, t, box, table = SYS[name]
    gE, gF = weights(x, 102)
    got = run_hvp(T, prec, x, t, box, table, gE, gF)
    check(prec, got, reference(name))


def test_dense_system_exceeds_slots(T):
    # the dense system takes the kernel's recompute-and-scatter branch: nearly
    # every atom has more bonds inside the cutoff than there are slots (12);
    # the jitter leaves a few at 12 or fewer (slot branch, same launch)
    x, t, box, table = SYS["bcc-dense"]
    cnt, _ = oracle.neighbors(x, box, RC)
    assert (cnt > 12).mean() > 0.9


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_hvp_without_force_weights_is_minus_ge_f(T, prec):
    # gF = NULL: grad_x = -gE F exactly as before; gF = 0 adds exact zeros
    x, t, box, table = SYS["sic"]
    a = run_hvp(T, prec, x, t, box, table, 1.7, None)
    b = run_hvp(T, prec, x, t, box, table, 1.7, np.zeros_like(x))
    assert np.array_equal(a, b)
    ref = oracle.compute(x, t, box, table, oracle.neighbors(x, box, RC))[1]
    tol = 1e-10 if prec == 0 else 1e-5
    assert np.sqrt(((a + 1.7 * ref) ** 2).mean() / ((1.7 * ref) ** 2).mean()) <= tol


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_hvp_batched_matches_oracle(T, prec):
    # batch mode (one launch over independent periodic systems): per-system
    # gE, the HVP of each system from its own atoms only
    names = ["si", "sic", "pack", "bcc-dense"]
    table = S.table_for(["Si", "C"], oracle.mix_tersoff89)
    cells = [SYS[n][:3] for n in names]
    off = np.cumsum([0] + [len(c[0]) for c in cells]).astype(np.int32)
    x = np.concatenate([c[0] for c in cells])
    t = np.concatenate([c[1] for c in cells]).astype(np.int32)
    boxes = np.stack([c[2] for c in cells])
    rng = np.random.Generator(np.random.Philox(103))
    gE = rng.normal(0.0, 1.0, size=len(cells))
    gF = rng.normal(0.0, 1.0, size=x.shape)
    ctx = T.Context(prec)
    ctx.params(table)
    xd = dev(x)
    ctx.neighbor_build_batched(xd, dev(t, torch.int32), off, boxes, RC + 0.5)
    gx = torch.full_like(xd, np.nan)
    ctx.backward(xd, dev(gE), dev(gF), gx, None)
    torch.cuda.synchronize()
    got = gx.cpu().numpy()
    ctx.close()
    for s, (xs, ts, bs) in enumerate(cells):
        nl = oracle.neighbors(xs, bs, RC)
        gfs = gF[off[s]:off[s + 1]]
        ref = np.zeros_like(xs)
        for a in range(len(xs)):
            for c in range(3):
                de, df = oracle.cs_pos(xs, ts, bs, table, nl, a, c, forces=True)
                ref[a, c] = gE[s] * de + float((gfs * df).sum())
        check(prec, got[off[s]:off[s + 1]], ref)


def test_autograd_position_gradient_of_force_loss(T):
    # loss on energy and forces, differentiated in x through the Function
    x, t, box, table = SYS["pack"]
    system = T.TersoffSystem(t, box, RC + 0.5, precision=0)
    rng = np.random.Generator(np.random.Philox(104))
    E0 = -700.0
    F0 = rng.normal(0.0, 0.5, size=x.shape)
    xd = dev(x).requires_grad_(True)
    E, F = T.energy_forces(system, xd, torch.tensor(table))
    loss = (E - E0) ** 2 + ((F - dev(F0)) ** 2).sum()
    loss.backward()
    gE = 2.0 * (E.item() - E0)
    gF = 2.0 * (F.detach().cpu().numpy() - F0)
    nl = oracle.neighbors(x, box, RC)
    ref = np.zeros_like(x)
    for a in range(len(x)):
        for c in range(3):
            de, df = oracle.cs_pos(x, t, box, table, nl, a, c, forces=True)
            ref[a, c] = gE * de + float((gF * df).sum())
    got = xd.grad.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
    with pytest.raises(RuntimeError):
        # the gradient is not itself differentiable
        xd2 = dev(x).requires_grad_(True)
        E2, F2 = T.energy_forces(system, xd2, torch.tensor(table))
        (gx,) = torch.autograd.grad((F2 ** 2).sum(), xd2, create_graph=True)
        gx.sum().backward()


@pytest.fixture(scope="module")
def large():
    x, v, t, box, names = W.config_si_md(ncell=40)
    table = S.table_for(["Si"], oracle.mix_tersoff89)
    return x, t, box, table


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_hvp_properties_at_full_size(T, prec, large):
    x, t, box, table = large
    assert len(x) == 512000
    rng = np.random.Generator(np.random.Philox(105))
    u = rng.normal(0.0, 1.0, size=x.shape)
    v = rng.normal(0.0, 1.0, size=x.shape)
    ctx = T.Context(prec)
    ctx.params(table)
    xd = dev(x)
    ctx.neighbor_build(xd, dev(t, torch.int32), box, RC + 1.0)
    zero = dev([0.0])

    def minus_hvp(w):
        gx = torch.full_like(xd, np.nan)
        ctx.backward(xd, zero, dev(w), gx, None)
        return gx.cpu().numpy()

    hu, hv = minus_hvp(u), minus_hvp(v)
    # symmetric: v . (H u) == u . (H v)
    a, b = float((v * hu).sum()), float((u * hv).sum())
    scale = np.sqrt((v * v).sum() * (hu * hu).sum())
    assert abs(a - b) <= (1e-11 if prec == 0 else 1e-6) * scale
    # translation invariance: the rows of H sum to zero
    # (each bond's contribution enters its two atoms with opposite signs in
    # double, so only the rounding of the double sums remains)
    assert np.abs(hu.sum(axis=0)).max() <= 1e-12 * np.abs(hu).sum()
    # uniform weights: no relative motion, exactly zero
    assert not minus_hvp(np.broadcast_to(np.array([0.3, -1.1, 0.7]), x.shape)).any()
    if prec == 0:
        # -H u = d/de F(x + e u), central difference with e = 1e-5 (error
        # O(e^2 |F'''|) plus rounding |F| 1e-16 / e)
        eps = 1e-5
        f = []
        for sgn in (1.0, -1.0):
            fd = torch.zeros_like(xd)
            ctx.compute(dev(x + sgn * eps * u), None, fd)
            f.append(fd.cpu().numpy())
        fdiff = (f[0] - f[1]) / (2 * eps)
        err = np.sqrt(((hu - fdiff) ** 2).mean() / (hu ** 2).mean())
        assert err <= 1e-6, err
    ctx.close()

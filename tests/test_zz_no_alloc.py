"""tersoff_compute_noalloc (fixed scratch, no allocation in the call) against
tersoff_compute on the same context, through the C ABI.

Collected last on purpose: it must also hold after every other GPU test has
used the library in the same process. Two calls in a row on the same inputs
check that each call clears the shared scratch it accumulates into.

Tolerances are those of the parity tests: FP64 path 1e-10 relative (energy,
max force, max virial component); mixed path relative force RMS, energy and
max virial component 1e-5. The two entry points differ only in the order in
which the same per-term forces are summed.
"""
import numpy as np
import pytest

import workloads as W
from tests import _systems as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RC = 3.0
TOL64 = 1e-10
TOLMIX = 1e-5


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1607_02904_gb300 as T
    T.load()
    return T


def _dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _outputs(n):
    e = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    f = torch.full((n, 3), np.nan, dtype=torch.float64, device="cuda")
    w = torch.full((6,), np.nan, dtype=torch.float64, device="cuda")
    return e, f, w


def _host(e, f, w):
    torch.cuda.synchronize()
    return e.item(), f.cpu().numpy(), w.cpu().numpy()


def _check(prec, got, ref):
    e, f, w = got
    er, fr, wr = ref
    assert np.isfinite(f).all() and np.isfinite(w).all() and np.isfinite(e)
    if prec == 0:
        assert abs(e - er) <= TOL64 * abs(er), (e, er)
        assert np.abs(f - fr).max() <= TOL64 * np.abs(fr).max()
        assert np.abs(w - wr).max() <= TOL64 * np.abs(wr).max()
    else:
        rms = np.sqrt(((f - fr) ** 2).mean()) / np.sqrt((fr ** 2).mean())
        assert rms <= TOLMIX, rms
        assert abs(e - er) <= TOLMIX * abs(er), (e, er)
        assert np.abs(w - wr).max() <= TOLMIX * np.abs(wr).max()


def _system(T, name):
    if name == "si":
        x, t, box = S.si_cell(5, amp=0.15, seed=71)
        return x, t, box, S.table_for(["Si"], T.mix_tersoff89)
    if name == "sic":
        x, t, box = S.sic_cell(4, sigma=0.1, seed=72)
        return x, t, box, S.table_for(["Si", "C"], T.mix_tersoff89)
    # the largest accepted size: 16 x 16 x 32 diamond cells = 65536 atoms
    x, t, box = W.diamond(16, 16, 32, 5.432)
    rng = np.random.Generator(np.random.Philox(73))
    return W.jitter_uniform(x, 0.1, rng), t, box, S.table_for(["Si"], T.mix_tersoff89)


@pytest.mark.parametrize("name", ["si", "sic", "max"])
@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_compute_twice(T, prec, name):
    x, t, box, table = _system(T, name)
    n = len(x)
    assert n <= T.NOALLOC_MAX_ATOMS
    ctx = T.Context(prec)
    ctx.params(table)
    xd, td = _dev(x), _dev(t, torch.int32)
    ctx.neighbor_build(xd, td, box, RC + 0.5)
    ref_out = _outputs(n)
    ctx.compute(xd, *ref_out)
    ref = _host(*ref_out)
    for _ in range(2):  # two calls in a row share (and must re-clear) the scratch
        out = _outputs(n)
        ctx.compute_noalloc(xd, *out)
        _check(prec, _host(*out), ref)
    # the context's own compute path is unaffected by the calls above: its
    # forces (gathered in a fixed order) repeat bit for bit; energy and virial
    # are sums with atomics, equal up to the order of the additions
    again = _outputs(n)
    ctx.compute(xd, *again)
    e2, f2, w2 = _host(*again)
    assert np.array_equal(f2, ref[1])
    assert abs(e2 - ref[0]) <= 1e-12 * abs(ref[0])
    assert np.abs(w2 - ref[2]).max() <= 1e-12 * np.abs(ref[2]).max()
    ctx.close()


def test_noalloc_moved_positions_and_null_outputs(T):
    x, t, box, table = _system(T, "si")
    n = len(x)
    ctx = T.Context(1)
    ctx.params(table)
    ctx.neighbor_build(_dev(x), _dev(t, torch.int32), box, RC + 1.0)
    rng = np.random.Generator(np.random.Philox(74))
    xm = _dev(x + rng.uniform(-0.1, 0.1, size=x.shape))
    ref_out = _outputs(n)
    ctx.compute(xm, *ref_out)
    ref = _host(*ref_out)
    e, f, w = _outputs(n)
    ctx.compute_noalloc(xm, e, None, None)
    ctx.compute_noalloc(xm, None, f, w)
    _check(1, _host(e, f, w), ref)
    ctx.close()


def test_noalloc_rejects_oversize(T):
    x, t, box, table = _system(T, "si")
    ctx = T.Context(1)
    ctx.params(table)
    ctx.neighbor_build(_dev(x), _dev(t, torch.int32), box, RC + 0.5)
    st = ctx.lib.tersoff_compute_noalloc(ctx.h, None, T.NOALLOC_MAX_ATOMS + 1, None, None, None,
                                         None)
    assert st == 1  # TERSOFF_E_INVALID_ARG, nothing enqueued
    assert b"TERSOFF_NOALLOC_MAX_ATOMS" in ctx.lib.tersoff_last_error(ctx.h)
    with pytest.raises(T.TersoffError):  # atom count differs from the build
        ctx.compute_noalloc(_dev(x[:-1]), *_outputs(len(x) - 1))
    ctx.close()


def test_noalloc_allocates_no_device_memory(T):
    # The call's defining property, observed through cudaMemGetInfo: after a
    # first call (which looks up the scratch array's address), further calls
    # leave the device's free memory unchanged. A tersoff_compute after a
    # precision switch reallocates the per-neighbour force buffers at another
    # size (16 or 32 bytes per slot), which shows that the check sees an
    # allocation.
    x, t, box, table = _system(T, "max")
    n = len(x)
    for prec in (0, 1):
        ctx = T.Context(prec)
        ctx.params(table)
        xd, td = _dev(x), _dev(t, torch.int32)
        ctx.neighbor_build(xd, td, box, RC + 0.5)
        out, out2 = _outputs(n), _outputs(n)  # every tensor of the test allocated up front
        ctx.compute_noalloc(xd, *out)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for _ in range(3):
            ctx.compute_noalloc(xd, *out)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (prec, free0 - free1)
        ctx.set_precision(1 - prec)
        ctx.compute(xd, *out2)
        torch.cuda.synchronize()
        free2, _ = torch.cuda.mem_get_info()
        assert free2 != free1
        ctx.close()


def test_md_after_noalloc_equals_md_without(T):
    # The call shares the context's status words with the force kernel; MD
    # that follows it must equal MD on a context that never made the call.
    x, t, box = W.diamond(4, 4, 4, 5.432)
    rng = np.random.Generator(np.random.Philox(75))
    x = W.jitter_gaussian(x, 0.05, rng)
    mass = [W.MASS_AMU["Si"]]
    v = W.maxwell_velocities(t, np.array(mass), 1000.0, rng)
    table = S.table_for(["Si"], T.mix_tersoff89)
    runs = []
    for use_noalloc in (False, True):
        ctx = T.Context(1)
        ctx.params(table)
        xd, vd = _dev(x), _dev(v)
        ctx.neighbor_build(xd, _dev(t, torch.int32), box, RC + 1.0)
        f = torch.zeros_like(xd)
        ctx.compute(xd, None, f)
        if use_noalloc:
            ctx.compute_noalloc(xd, *_outputs(len(x)))
        ctx.md_step(xd, vd, f, mass, 0.001, 15, 10)
        torch.cuda.synchronize()
        runs.append((xd.cpu().numpy(), vd.cpu().numpy(), f.cpu().numpy()))
        ctx.close()
    for a, b in zip(runs[0], runs[1]):
        assert np.array_equal(a, b)

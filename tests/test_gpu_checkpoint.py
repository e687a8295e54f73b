"""MD checkpoints through the C ABI: a run saved and restored into a new
context continues exactly as the uninterrupted run, the file's header and
arrays hold the stated layout, and bad files are refused.
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W
from tests import _systems as S

torch = pytest.importorskip("torch")

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


def _state(species):
    if species == "Si":
        x, t, box = S.si_cell(n=4, amp=0.05, seed=61)
        names = ["Si"]
    else:
        x, t, box = S.sic_cell(n=4, sigma=0.05, seed=62)
        names = ["Si", "C"]
    table = S.table_for(names, oracle.mix_tersoff89)
    mass = [W.MASS_AMU[s] for s in names]
    rng = np.random.Generator(np.random.Philox(63))
    v = W.maxwell_velocities(t, np.array(mass), 1000.0, rng)
    return x, v, t, box, table, mass


def _start(T, prec, x, v, t, box, table):
    ctx = T.Context(prec)
    ctx.params(table)
    xd, vd = dev(x), dev(v)
    ctx.neighbor_build(xd, dev(t, torch.int32), box, RC + 1.0)
    fd = torch.zeros_like(xd)
    ctx.compute(xd, None, fd)
    return ctx, xd, vd, fd


@pytest.mark.gpu
@pytest.mark.parametrize("species", ["Si", "SiC"])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_resume_after_a_rebuild_is_bit_identical(T, tmp_path, prec, species):
    x, v, t, box, table, mass = _state(species)
    every = 10
    # uninterrupted: two calls of 10 steps on one context
    a, xa, va, fa = _start(T, prec, x, v, t, box, table)
    a.md_step(xa, va, fa, mass, 0.001, 10, every)
    a.md_step(xa, va, fa, mass, 0.001, 10, every)
    torch.cuda.synchronize()
    # interrupted after the first call (the list was rebuilt at its last step)
    b, xb, vb, fb = _start(T, prec, x, v, t, box, table)
    b.md_step(xb, vb, fb, mass, 0.001, 10, every)
    path = str(tmp_path / "run.ckpt")
    b.checkpoint_save(path, xb, vb, fb, step=10)
    b.close()
    assert T.checkpoint_info(path) == (len(x), 1 if species == "Si" else 2)
    c = T.Context(1 - prec)  # the saved precision is restored
    xc, vc, fc = (torch.zeros((len(x), 3), dtype=torch.float64, device="cuda") for _ in range(3))
    tc = torch.zeros(len(x), dtype=torch.int32, device="cuda")
    step = c.checkpoint_load(path, xc, vc, fc, tc)
    assert step == 10
    assert np.array_equal(tc.cpu().numpy(), t)
    c.md_step(xc, vc, fc, mass, 0.001, 10, every)
    torch.cuda.synchronize()
    assert torch.equal(xc, xa) and torch.equal(vc, va) and torch.equal(fc, fa)
    assert c.md_rebuilds() == a.md_rebuilds() == 1
    a.close()
    c.close()


@pytest.mark.gpu
def test_resume_mid_period_keeps_the_rebuild_phase(T, tmp_path):
    x, v, t, box, table, mass = _state("Si")
    a, xa, va, fa = _start(T, 0, x, v, t, box, table)
    a.md_step(xa, va, fa, mass, 0.001, 4, 10)
    a.md_step(xa, va, fa, mass, 0.001, 12, 10)
    ra = a.md_rebuilds()
    torch.cuda.synchronize()
    b, xb, vb, fb = _start(T, 0, x, v, t, box, table)
    b.md_step(xb, vb, fb, mass, 0.001, 4, 10)
    path = str(tmp_path / "mid.ckpt")
    b.checkpoint_save(path, xb, vb, fb, step=4)
    b.close()
    c = T.Context(0)
    xc, vc, fc = (torch.zeros((len(x), 3), dtype=torch.float64, device="cuda") for _ in range(3))
    tc = torch.zeros(len(x), dtype=torch.int32, device="cuda")
    assert c.checkpoint_load(path, xc, vc, fc, tc) == 4
    c.md_step(xc, vc, fc, mass, 0.001, 12, 10)
    torch.cuda.synchronize()
    # the list was built at the saved positions, so summation order may differ;
    # the rebuild after 6 more steps (the saved phase) is kept
    assert c.md_rebuilds() == ra == 1
    assert np.abs(xc.cpu().numpy() - xa.cpu().numpy()).max() < 1e-9
    assert np.abs(vc.cpu().numpy() - va.cpu().numpy()).max() < 1e-7
    a.close()
    c.close()


@pytest.mark.gpu
def test_file_layout_and_refusals(T, tmp_path):
    x, v, t, box, table, mass = _state("SiC")
    b, xb, vb, fb = _start(T, 1, x, v, t, box, table)
    b.set_scatter(T.SCATTER_ATOMIC)
    b.set_launch(2, 1, 128)
    b.md_step(xb, vb, fb, mass, 0.001, 3, 10)
    path = str(tmp_path / "s.ckpt")
    b.checkpoint_save(path, xb, vb, fb, step=123456789012)
    raw = open(path, "rb").read()
    nl = raw.index(b"\n")
    hdr = json.loads(raw[:nl])
    n, ns = len(x), 2
    assert hdr["format"] == "tersoff-gb300-checkpoint" and hdr["version"] == 1
    assert (hdr["n"], hdr["n_species"], hdr["precision"], hdr["step"]) == (n, ns, 1, 123456789012)
    assert hdr["steps_since_build"] == 3 and hdr["r_list"] == RC + 1.0 and hdr["capacity"] >= 32
    assert hdr["box"] == [float(b_) for b_ in box]
    assert (hdr["scatter"], hdr["waves"], hdr["split"], hdr["block"], hdr["lanes"],
            hdr["ablate"], hdr["graphs"]) == (1, 2, 1, 128, -1, 0, 1)
    body = raw[nl + 1:]
    nt = ns ** 3 * 14
    assert len(body) == 4 * n + 8 * (nt + 9 * n)
    types = np.frombuffer(body[:4 * n], dtype="<i4")
    tab = np.frombuffer(body[4 * n:4 * n + 8 * nt], dtype="<f8")
    st = np.frombuffer(body[4 * n + 8 * nt:], dtype="<f8").reshape(3, n, 3)
    assert np.array_equal(types, t)
    assert np.array_equal(tab, np.asarray(table, dtype=np.float64))
    for k, arr in enumerate((xb, vb, fb)):
        assert np.array_equal(st[k], arr.cpu().numpy())
    c = T.Context(1)
    z = [torch.zeros((n + 1, 3), dtype=torch.float64, device="cuda") for _ in range(3)]
    tz = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(T.TersoffError) as e:  # another atom count
        c.checkpoint_load(path, *z, tz)
    assert e.value.code == T._lib.E_INVALID_ARG
    z = [a[:n] for a in z]
    bad = str(tmp_path / "bad.ckpt")
    for blob in (raw[:nl + 1 + len(body) // 2], b"not a checkpoint\n" + body):
        with open(bad, "wb") as fh:
            fh.write(blob)
        with pytest.raises(T.TersoffError) as e:  # truncated, foreign
            c.checkpoint_load(bad, *z, tz[:n])
        assert e.value.code == T._lib.E_INVALID_ARG
    with pytest.raises(T.TersoffError):
        c.checkpoint_load(str(tmp_path / "missing.ckpt"), *z, tz[:n])
    # a restored context saves the same file byte for byte (state, options,
    # capacity and rebuild phase all restored)
    assert c.checkpoint_load(path, *z, tz[:n]) == 123456789012
    again = str(tmp_path / "again.ckpt")
    c.checkpoint_save(again, *z, step=123456789012)
    assert open(again, "rb").read() == raw
    b.close()
    c.close()


def test_info_reads_the_header_without_a_gpu(tmp_path):
    """The header reader is host code: a file in the stated layout gives its
    counts, and a foreign header is refused (no GPU needed)."""
    from paper_1607_02904_gb300 import _lib
    _lib.load()
    hdr = ('{"format":"tersoff-gb300-checkpoint","version":1,"n":7,"n_species":2,'
           '"precision":1,"box":[10.5,11,12.25],"r_list":4,"step":3,"steps_since_build":0,'
           '"capacity":32,"scatter":0,"waves":0,"split":-1,"block":256,"lanes":-1,"ablate":0,"graphs":1,'
           '"endian":"little","arrays":[]}\n')
    p = tmp_path / "h.ckpt"
    p.write_bytes(hdr.encode())
    assert _lib.checkpoint_info(str(p)) == (7, 2)
    for bad in (hdr.replace('"version":1', '"version":2'), hdr.replace("gb300", "other"),
                hdr.replace('"n_species":2', '"n_species":9'), hdr.replace('"graphs":1,', ''),
                hdr.rstrip("\n")):
        p.write_bytes(bad.encode())
        with pytest.raises(_lib.TersoffError):
            _lib.checkpoint_info(str(p))
    assert not os.path.exists(str(tmp_path / "none.ckpt"))
    with pytest.raises(_lib.TersoffError):
        _lib.checkpoint_info(str(tmp_path / "none.ckpt"))

"""Host-side checks that need no GPU: the library builds and exports every
declared entry point, the binding matches the header, and the product's
parameter-table helper agrees with the oracle's mixing rule."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W


def test_library_exports_declared_symbols():
    import paper_1607_02904_gb300 as T
    lib = T.load()
    declared = T.declared_symbols()
    assert len(declared) >= 14
    for name in declared:
        assert hasattr(lib, name), name
    # the binding knows every declared symbol
    from paper_1607_02904_gb300 import _lib
    assert set(declared) <= set(_lib._SIG)


def test_header_constants_match_binding():
    import re
    import os
    import paper_1607_02904_gb300 as T
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "include",
                            "tersoff.h")).read()
    consts = dict(re.findall(r"#define (TERSOFF_\w+) (\d+)", hdr))
    assert int(consts["TERSOFF_NPARAM"]) == T.NPARAM
    assert int(consts["TERSOFF_FP64"]) == T.FP64
    assert int(consts["TERSOFF_MIXED"]) == T.MIXED
    assert int(consts["TERSOFF_NOALLOC_MAX_ATOMS"]) == T.NOALLOC_MAX_ATOMS
    for name in ("NO_SHORT", "GENERAL", "FP32_SUMS", "FASTFWD", "COMP_ATOM_SUMS"):
        assert int(consts["TERSOFF_ABLATE_" + name]) == getattr(T, "ABLATE_" + name)
    order = ["M", "GAMMA", "LAMBDA3", "C", "D", "H", "N", "BETA", "LAMBDA2", "B", "R", "D_CUT",
             "LAMBDA1", "A"]
    for q, name in enumerate(order):
        assert int(consts["TERSOFF_P_" + name]) == q


@pytest.mark.parametrize("names", [["Si"], ["C"], ["Si", "C"], ["C", "Si"]])
def test_product_mixing_matches_oracle(names):
    import paper_1607_02904_gb300 as T
    elem, chi = W.element_records(names)
    a = T.mix_tersoff89(elem, chi)
    b = oracle.mix_tersoff89(elem, chi)
    assert a.shape == b.shape
    assert np.allclose(a, b, rtol=1e-15, atol=0)


def test_create_without_gpu_reports_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_1607_02904_gb300 as T
    lib = T.load()
    h = ctypes.c_void_p()
    st = lib.tersoff_create(ctypes.byref(h), 1)
    assert st == 6  # TERSOFF_E_CUDA
    assert lib.tersoff_create(None, 1) == 1
    assert lib.tersoff_destroy(None) == 0


@pytest.mark.parametrize("names", [["Si"], ["Si", "C"]])
def test_table_file_round_trip(tmp_path, names):
    import paper_1607_02904_gb300 as T
    table = T.mix_tersoff89(*W.element_records(names))
    p = tmp_path / "t.txt"
    T.write_table(str(p), table, names)
    assert np.array_equal(T.read_table(str(p), names), table)
    # species order is the caller's: the same file read with the names swapped
    # gives the table with species indices permuted
    if len(names) == 2:
        sw = T.read_table(str(p), names[::-1]).reshape(2, 2, 2, 14)
        ref = np.asarray(table).reshape(2, 2, 2, 14)
        for i in range(2):
            for j in range(2):
                for k in range(2):
                    assert np.array_equal(sw[1 - i, 1 - j, 1 - k], ref[i, j, k])


def test_table_file_format(tmp_path):
    """A hand-written file: comments, an entry over two lines, an entry of
    another element that is skipped, and the record each entry lands in."""
    import paper_1607_02904_gb300 as T
    vals = {("A", "A", "A"): 1.0, ("A", "A", "B"): 2.0, ("A", "B", "A"): 3.0, ("A", "B", "B"): 4.0,
            ("B", "A", "A"): 5.0, ("B", "A", "B"): 6.0, ("B", "B", "A"): 7.0, ("B", "B", "B"): 8.0}
    lines = ["# test table", "X A A " + " ".join(["9"] * 14) + "  # another element"]
    for (i, j, k), v in vals.items():
        rec = " ".join(f"{v + q / 100:g}" for q in range(14))
        if (i, j, k) == ("A", "B", "A"):
            toks = rec.split()
            lines += [f"{i} {j} {k} " + " ".join(toks[:5]), " ".join(toks[5:])]
        else:
            lines.append(f"{i} {j} {k} {rec}")
    p = tmp_path / "t.txt"
    p.write_text("\n".join(lines) + "\n")
    t = T.read_table(str(p), ["A", "B"]).reshape(2, 2, 2, 14)
    for (i, j, k), v in vals.items():
        idx = tuple("AB".index(x) for x in (i, j, k))
        assert np.allclose(t[idx], [v + q / 100 for q in range(14)], rtol=0, atol=1e-12)
    # a missing triplet, a duplicate, a broken entry are refused
    with pytest.raises(ValueError, match="no entry"):
        T.read_table(str(p), ["A", "B", "X"])
    p.write_text("\n".join(lines + [lines[2]]) + "\n")
    with pytest.raises(ValueError, match="twice"):
        T.read_table(str(p), ["A", "B"])
    p.write_text("\n".join(lines + ["A A"]) + "\n")
    with pytest.raises(ValueError, match="entries of 17"):
        T.read_table(str(p), ["A", "B"])


def test_thermo_records_and_jsonl(tmp_path):
    """Temperature from the kinetic energy (3/2 N kB T), the ideal-gas pressure
    with a zero virial, the virial's share, step numbering and the file."""
    import json
    from paper_1607_02904_gb300 import thermo
    n, T0 = 1000, 1000.0
    ke = 1.5 * n * thermo.KB_EV_PER_K * T0
    rows = np.array([[-4630.0, ke, -4630.0 + ke], [-4629.0, 2 * ke, -4629.0 + 2 * ke]])
    vol = 20000.0
    w = np.zeros((2, 6))
    w[1, :3] = 30.0  # trace 90 eV: adds 30 eV / V
    recs = thermo.records(rows, n, step0=10, virials=w, volume=vol)
    assert [r["step"] for r in recs] == [11, 12]
    assert abs(recs[0]["temperature_K"] - T0) < 1e-9 and abs(recs[1]["temperature_K"] - 2 * T0) < 1e-9
    ideal = n * thermo.KB_EV_PER_K * T0 / vol * thermo.EV_PER_A3_IN_BAR
    assert abs(recs[0]["pressure_bar"] - ideal) < 1e-9 * ideal
    assert abs(recs[1]["pressure_bar"] - (2 * ideal + 30.0 / vol * thermo.EV_PER_A3_IN_BAR)) < 1e-6
    p = tmp_path / "thermo.jsonl"
    assert thermo.write_jsonl(str(p), rows, n, append=False) == 2
    assert thermo.write_jsonl(str(p), rows, n, step0=2) == 2
    lines = [json.loads(s) for s in p.read_text().splitlines()]
    assert [r["step"] for r in lines] == [1, 2, 3, 4]
    assert lines[0]["etot_eV"] == rows[0, 2] and "pressure_bar" not in lines[0]

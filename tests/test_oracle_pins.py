"""Pins for the FP64 CPU oracle (no GPU).

Each test checks the oracle against something other than itself: published
cohesive energies, closed forms for symmetric structures, brute-force
evaluation with no neighbour list, complex-step and finite-difference
derivatives, conservation laws and symmetries.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from tests import _systems as S

RC = 3.0  # largest Tersoff cutoff (Si R + D)


def si_table():
    return S.table_for(["Si"], oracle.mix_tersoff89)


def sic_table():
    return S.table_for(["Si", "C"], oracle.mix_tersoff89)


# ----------------------------------------------------------------------------- closed forms
def _closed_form_bond(el_i, el_j, r, chi=1.0):
    """V(i->j) in a perfect tetrahedral crystal: 3 other neighbours at cos = -1/3."""
    A = math.sqrt(el_i[0] * el_j[0])
    B = chi * math.sqrt(el_i[1] * el_j[1])
    lam1 = 0.5 * (el_i[2] + el_j[2])
    lam2 = 0.5 * (el_i[3] + el_j[3])
    beta, n, c, d, h = el_i[4], el_i[5], el_i[6], el_i[7], el_i[8]
    g = 1.0 + c * c / (d * d) - c * c / (d * d + (h + 1.0 / 3.0) ** 2)
    zeta = 3.0 * g
    b = (1.0 + (beta * zeta) ** n) ** (-1.0 / (2.0 * n))
    return A * math.exp(-lam1 * r) - b * B * math.exp(-lam2 * r)


def _closed_form_energy(structure, species, a):
    r = a * math.sqrt(3.0) / 4.0
    if structure == "diamond":
        el = W.ELEMENTS_TERSOFF89[species]
        return 2.0 * _closed_form_bond(el, el, r)  # 4 bonds x 1/2
    si, c = W.ELEMENTS_TERSOFF89["Si"], W.ELEMENTS_TERSOFF89["C"]
    return _closed_form_bond(si, c, r, W.CHI_SIC) + _closed_form_bond(c, si, r, W.CHI_SIC)


def _oracle_crystal(structure, species, a, ncell=2):
    if structure == "diamond":
        names = [species]
        x, t, box = W.diamond(ncell, ncell, ncell, a)
    else:
        names = ["Si", "C"]
        x, t, box = W.diamond(ncell, ncell, ncell, a, zincblende=True)
    table = S.table_for(names, oracle.mix_tersoff89)
    nl = oracle.neighbors(x, box, RC)
    e, f, w = oracle.compute(x, t, box, table, nl)
    return e / len(x), f, w


@pytest.mark.parametrize("row", S.read_cohesive(), ids=lambda r: f"{r[0]}-{r[1]}")
def test_cohesive_energy_closed_form_and_published(row):
    structure, species, a, e_pub, tol = row
    ncell = 3 if species == "C" else 2  # box edge must exceed twice the cutoff
    e_or, f, w = _oracle_crystal(structure, species, a, ncell)
    e_cf = _closed_form_energy(structure, species, a)
    assert abs(e_or - e_cf) <= 1e-12 * abs(e_cf)
    assert abs(-e_or - e_pub) <= tol * e_pub
    # perfect crystal: zero forces by symmetry, isotropic virial
    assert np.abs(f).max() < 1e-11
    assert abs(w[0] - w[1]) < 1e-10 and abs(w[0] - w[2]) < 1e-10
    assert np.abs(w[3:]).max() < 1e-10


def test_si_lattice_constant_is_minimum():
    e0 = _closed_form_energy("diamond", "Si", 5.432)
    for a in (5.40, 5.42, 5.445, 5.46):
        assert _oracle_crystal("diamond", "Si", a)[0] > e0 - 1e-12


def test_dimer_closed_form():
    # Isolated pair: zeta = 0, b = 1, E = fc(r) (fR + fA) (two directed bonds x 1/2)
    table = si_table()
    el = W.ELEMENTS_TERSOFF89["Si"]
    A, B, lam1, lam2, Rin, Sout = el[0], el[1], el[2], el[3], el[9], el[10]
    R, D = 0.5 * (Rin + Sout), 0.5 * (Sout - Rin)
    box = np.array([30.0, 30.0, 30.0])
    for r in (2.3, 2.78, 2.85, 2.93, 2.999):
        x = np.array([[5.0, 5.0, 5.0], [5.0 + r, 5.0, 5.0]])
        t = np.zeros(2, dtype=np.int32)
        nl = oracle.neighbors(x, box, 3.2)
        e, f, w = oracle.compute(x, t, box, table, nl)
        if r < R - D:
            fc, dfc = 1.0, 0.0
        else:
            fc = 0.5 - 0.5 * math.sin(0.5 * math.pi * (r - R) / D)
            dfc = -0.25 * math.pi / D * math.cos(0.5 * math.pi * (r - R) / D)
        v = A * math.exp(-lam1 * r) - B * math.exp(-lam2 * r)
        dv = -lam1 * A * math.exp(-lam1 * r) + lam2 * B * math.exp(-lam2 * r)
        assert abs(e - fc * v) <= 1e-13 * max(1.0, abs(e))
        # force on atom 1 along +x: -dE/dr
        assert abs(f[1, 0] - (-(dfc * v + fc * dv))) <= 1e-12 * max(1.0, abs(f[1, 0]))
        assert abs(f[0, 0] + f[1, 0]) < 1e-12


# ----------------------------------------------------------------------------- brute force
def _systems():
    si = si_table()
    sic = sic_table()
    out = []
    x, t, box = S.si_cell()
    out.append(("si", x, t, box, si))
    x, t, box = S.sic_cell()
    out.append(("sic", x, t, box, sic))
    x, t, box = S.packing_cell()
    out.append(("pack", x, t, box, sic))
    x, t, box = S.si_cell(seed=21, amp=0.3)
    out.append(("si-l3m3", x, t, box, S.with_lambda3(si, 1.7322, 3)))
    out.append(("si-l3m1", x, t, box, S.with_lambda3(si, 1.3, 1)))
    return out


SYSTEMS = _systems()
IDS = [s[0] for s in SYSTEMS]


@pytest.mark.parametrize("sysd", SYSTEMS, ids=IDS)
def test_bruteforce_n3_matches_list(sysd):
    _, x, t, box, table = sysd
    e_bf = oracle.energy_n3(x, t, box, table)
    # Sec. III: iterating a skin-extended list gives the same result as the cutoff list
    for rc in (RC, RC + 0.5):
        e, f, w = oracle.compute(x, t, box, table, oracle.neighbors(x, box, rc))
        assert abs(e - e_bf) <= 1e-13 * abs(e_bf)


@pytest.mark.parametrize("sysd", SYSTEMS, ids=IDS)
def test_forces_complex_step_and_fd(sysd):
    _, x, t, box, table = sysd
    nl = oracle.neighbors(x, box, RC + 0.3)
    e, f, w = oracle.compute(x, t, box, table, nl)
    fscale = np.abs(f).max()
    rng = np.random.default_rng(5)
    atoms = rng.choice(len(x), size=8, replace=False)
    for a in atoms:
        for c in range(3):
            dcs = oracle.cs_pos(x, t, box, table, nl, int(a), c)
            assert abs(-dcs - f[a, c]) <= 1e-11 * fscale
            # central difference with one Richardson step
            def ef(hh):
                xp = x.copy(); xp[a, c] += hh
                xm = x.copy(); xm[a, c] -= hh
                return (oracle.compute(xp, t, box, table, nl)[0]
                        - oracle.compute(xm, t, box, table, nl)[0]) / (2 * hh)
            h = 1e-4
            d = (4 * ef(h / 2) - ef(h)) / 3
            assert abs(-d - f[a, c]) <= 1e-6 * fscale


@pytest.mark.parametrize("sysd", SYSTEMS, ids=IDS)
def test_conservation_and_symmetry(sysd):
    _, x, t, box, table = sysd
    nl = oracle.neighbors(x, box, RC)
    e, f, w = oracle.compute(x, t, box, table, nl)
    fscale = np.abs(f).max()
    assert np.abs(f.sum(axis=0)).max() <= 1e-12 * max(fscale, 1.0) * len(x)
    # translation (a periodic translate changes no distance)
    shift = np.array([0.37, -1.91, 2.53])
    e2, f2, w2 = oracle.compute(x + shift, t, box, table, oracle.neighbors(x + shift, box, RC))
    assert abs(e2 - e) <= 1e-12 * abs(e)
    assert np.abs(f2 - f).max() <= 1e-10 * fscale
    # permutation of atom order
    perm = np.random.default_rng(3).permutation(len(x))
    xp, tp = x[perm], t[perm]
    e3, f3, w3 = oracle.compute(xp, tp, box, table, oracle.neighbors(xp, box, RC))
    assert abs(e3 - e) <= 1e-12 * abs(e)
    assert np.abs(f3 - f[perm]).max() <= 1e-10 * fscale
    assert np.abs(w3 - w).max() <= 1e-10 * np.abs(w).max()


def test_replication_2x2x2():
    table = sic_table()
    x, t, box = S.sic_cell(n=2)
    e, f, w = oracle.compute(x, t, box, table, oracle.neighbors(x, box, RC))
    reps = []
    for k in range(2):
        for j in range(2):
            for i in range(2):
                reps.append(x + np.array([i, j, k]) * box)
    xr = np.concatenate(reps)
    tr = np.tile(t, 8)
    br = 2 * box
    e8, f8, w8 = oracle.compute(xr, tr, br, table, oracle.neighbors(xr, br, RC))
    assert abs(e8 - 8 * e) <= 1e-12 * abs(e8)
    assert np.abs(w8 - 8 * w).max() <= 1e-10 * np.abs(w8).max()
    for r in range(8):
        assert np.abs(f8[r * len(x):(r + 1) * len(x)] - f).max() <= 1e-11 * np.abs(f).max()


def test_isolated_cluster_zero_torque_and_full_virial():
    table = si_table()
    x, t, box = W.diamond(2, 2, 2, 5.432)
    rng = np.random.default_rng(8)
    x = x + rng.uniform(-0.15, 0.15, size=x.shape) + 20.0  # cluster in a 50 A box
    box = np.array([50.0, 50.0, 50.0])
    nl = oracle.neighbors(x, box, RC)
    e, f, w = oracle.compute(x, t, box, table, nl)
    com = x.mean(axis=0)
    torque = np.cross(x - com, f).sum(axis=0)
    assert np.abs(torque).max() <= 1e-11 * np.abs(f).max() * len(x)
    # virial from homogeneous deformation x_a += eps * x_b: W_ab = -dE/deps
    comp = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (0, 2): 4, (1, 2): 5}
    for (a, b), k in comp.items():
        def en(eps, a=a, b=b):
            xd = x.copy()
            xd[:, b] += eps * (x[:, a] - com[a])
            return oracle.compute(xd, t, box, table, oracle.neighbors(xd, box, RC))[0]
        h = 1e-5
        d = (en(h) - en(-h)) / (2 * h)
        assert abs(-d - w[k]) <= 1e-6 * np.abs(w).max()


def test_periodic_virial_diagonal_strain():
    table = sic_table()
    x, t, box = S.packing_cell()
    e, f, w = oracle.compute(x, t, box, table, oracle.neighbors(x, box, RC))
    for a in range(3):
        def en(eps, a=a):
            s = np.ones(3); s[a] += eps
            xd = x * s
            bd = box * s
            return oracle.compute(xd, t, bd, table, oracle.neighbors(xd, bd, RC))[0]
        h = 1e-5
        d = (en(h) - en(-h)) / (2 * h)
        assert abs(-d - w[a]) <= 1e-6 * np.abs(w).max()


def test_param_gradient_complex_step_vs_fd():
    table = sic_table()
    x, t, box = S.packing_cell(seed=17)
    nl = oracle.neighbors(x, box, RC)
    e0, f0, _ = oracle.compute(x, t, box, table, nl)
    ns = 2
    # every continuous field of a pair record and a mixed three-body record
    checks = []
    for rec in [(0, 0, 0), (0, 1, 1), (1, 0, 0), (1, 1, 1), (0, 0, 1), (1, 0, 1)]:
        for fld in oracle.FIELDS:
            if fld == "m" or fld == "lambda3":
                continue
            checks.append(oracle.table_index(ns, *rec, fld))
    for p in checks:
        de, df = oracle.cs_param(x, t, box, table, nl, p)
        h = 1e-6 * max(abs(table[p]), 1e-3)
        tp = table.copy(); tp[p] += h
        tm = table.copy(); tm[p] -= h
        ep, fp, _ = oracle.compute(x, t, box, tp, nl)
        em, fm, _ = oracle.compute(x, t, box, tm, nl)
        dfd = (ep - em) / (2 * h)
        assert abs(de - dfd) <= 1e-5 * max(abs(de), 1e-6 * abs(e0) / max(abs(table[p]), 1e-3))
        ffd = (fp - fm) / (2 * h)
        scale = max(np.abs(df).max(), 1e-9)
        assert np.abs(df - ffd).max() <= 1e-4 * scale + 1e-7


def test_identical_species_reduce_to_single_species():
    si1 = si_table()
    elem = np.array([W.ELEMENTS_TERSOFF89["Si"]] * 2)
    chi = np.ones((2, 2))
    si2 = oracle.mix_tersoff89(elem, chi)
    x, t, box = S.si_cell(seed=4)
    t2 = (np.arange(len(x)) % 3 == 0).astype(np.int32)
    nl = oracle.neighbors(x, box, RC)
    e1, f1, w1 = oracle.compute(x, t, box, si1, nl)
    e2, f2, w2 = oracle.compute(x, t2, box, si2, nl)
    assert abs(e1 - e2) <= 1e-13 * abs(e1)
    assert np.abs(f1 - f2).max() <= 1e-12 * np.abs(f1).max()


def test_mixing_rule_records():
    # Tersoff (1989) mixing: geometric A, B (x chi), R, S; arithmetic lambda, mu.
    t = sic_table().reshape(2, 2, 2, 14)
    si, c = W.ELEMENTS_TERSOFF89["Si"], W.ELEMENTS_TERSOFF89["C"]
    rec = t[0, 1, 1]
    assert abs(rec[13] - 1597.3111) < 1e-3          # A_SiC
    assert abs(rec[9] - 395.1451) < 1e-3            # B_SiC (with chi)
    assert abs(rec[12] - 2.9839) < 1e-12            # lambda1
    assert abs(rec[8] - 1.97205) < 1e-12            # lambda2
    Rt, St = math.sqrt(si[9] * c[9]), math.sqrt(si[10] * c[10])
    assert abs(rec[10] - 0.5 * (Rt + St)) < 1e-14 and abs(rec[11] - 0.5 * (St - Rt)) < 1e-14
    # three-body terms come from the centre element
    assert t[1, 0, 0][3] == c[6] and t[0, 1, 0][3] == si[6]


# ----------------------------------------------------------------------------- neighbour lists
def test_neighbors_cells_equal_bruteforce():
    rng = np.random.default_rng(2)
    for n, L, rc in ((300, 13.0, 4.0), (500, 15.5, 3.7), (200, 9.0, 4.0)):
        box = np.array([L, L * 1.1, L * 0.95])
        x = rng.random((n, 3)) * box
        x[::7] += box * rng.integers(-3, 4, size=(len(x[::7]), 3))  # unwrapped images
        a = oracle.neighbors(x, box, rc, method="cells")
        b = oracle.neighbors(x, box, rc, method="brute")
        assert np.array_equal(a[0], b[0])
        assert np.array_equal(a[1][:, : a[0].max()], b[1][:, : b[0].max()])
        for i in range(n):
            row = a[1][i, : a[0][i]]
            assert np.all(np.diff(row) > 0)


def test_neighbors_cutoff_inclusive():
    # Eq. 4 uses r <= r_C: a pair at exactly the cutoff belongs to the list.
    box = np.array([20.0, 20.0, 20.0])
    x = np.array([[1.0, 1.0, 1.0], [4.0, 1.0, 1.0], [1.0, 1.0, 4.0000001]])
    cnt, nbr = oracle.neighbors(x, box, 3.0, method="brute")
    assert list(nbr[0, : cnt[0]]) == [1]


def test_md_energy_conservation():
    table = si_table()
    x, t, box = S.si_cell(n=3, amp=0.0)
    v = W.maxwell_velocities(t, np.array([W.MASS_AMU["Si"]]), 1000.0,
                             np.random.Generator(np.random.Philox(99)))
    xo, vo, thermo, f = oracle.md_run(x, v, t, box, table, [W.MASS_AMU["Si"]], 0.001, 200,
                                     RC + 1.0, 10)
    etot = thermo[:, 2]
    ke = thermo[:, 1]
    assert np.ptp(etot) < 0.02 * np.ptp(ke)


def test_force_derivative_complex_step_vs_fd():
    # dF/dx by the complex step (a column of minus the Hessian) against central
    # differences of the oracle's forces; and the Hessian's symmetry
    table = sic_table()
    x, t, box = S.packing_cell(n=48, seed=19)
    nl = oracle.neighbors(x, box, RC)
    cols = {}
    for a, c in [(0, 0), (5, 2), (17, 1), (30, 0)]:
        de, df = oracle.cs_pos(x, t, box, table, nl, a, c, forces=True)
        h = 1e-5
        xp, xm = x.copy(), x.copy()
        xp[a, c] += h
        xm[a, c] -= h
        _, fp, _ = oracle.compute(x=xp, types=t, box=box, table=table, nl=nl)
        _, fm, _ = oracle.compute(x=xm, types=t, box=box, table=table, nl=nl)
        fd = (fp - fm) / (2 * h)
        assert np.abs(df - fd).max() <= 1e-6 * np.abs(df).max()
        _, f0, _ = oracle.compute(x, t, box, table, nl)
        assert abs(de + f0[a, c]) <= 1e-10 * np.abs(f0).max()
        cols[(a, c)] = df
    # H = -dF/dx is symmetric: dF_b/dx_a = dF_a/dx_b
    keys = list(cols)
    for p in keys:
        for q in keys:
            assert abs(cols[p][q] - cols[q][p]) <= 1e-9 * np.abs(cols[p]).max()


def test_cutoff_edge_keeps_relative_accuracy():
    # dimer in the taper just inside R + D (zeta = 0, b = 1): E = f_C(r) (f_R +
    # f_A) and F = -dE/dr, against 50-digit arithmetic on the same double
    # inputs. f_C ~ delta^2 there (delta = R + D - r): the textbook
    # 1/2 - 1/2 sin(...) loses ~1e-16 absolute, 4e-10 relative at delta = 1e-4
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    table = S.table_for(["Si"], oracle.mix_tersoff89)
    rec = table.reshape(-1, 14)[0]
    R, D, A, B, l1, l2 = (mpmath.mpf(float(rec[k])) for k in (10, 11, 13, 9, 12, 8))
    box = np.array([20.0, 20.0, 20.0])
    t = np.zeros(2, np.int32)

    def energy(r):
        fc = mpmath.sin(mpmath.pi * ((R + D) - r) / (4 * D)) ** 2
        return fc * (A * mpmath.exp(-l1 * r) - B * mpmath.exp(-l2 * r))

    for delta in (1e-2, 1e-3, 1e-4):
        x = np.array([[5.0, 5.0, 5.0], [5.0 + (3.0 - delta), 5.0, 5.0]])
        r = mpmath.mpf(float(x[1, 0])) - mpmath.mpf(float(x[0, 0]))  # exact difference
        e, f, _ = oracle.compute(x, t, box, table, oracle.neighbors(x, box, 3.5))
        e_ref = energy(r)
        f_ref = -mpmath.diff(energy, r)  # force on atom 1 along +x
        assert abs(e - float(e_ref)) <= 1e-11 * abs(float(e_ref)), delta
        assert abs(f[1, 0] - float(f_ref)) <= 1e-11 * abs(float(f_ref)), delta
        assert f[0, 0] == -f[1, 0]


def test_dimer_force_derivative_closed_form():
    # the Hessian of a dimer (zeta = 0, b = 1, E = f_C (f_R + f_A)): along the
    # bond dF/dx = -E''(r), across it -E'(r)/r; the oracle's complex-step force
    # derivative (the reference of the Hessian-vector product) against
    # 50-digit arithmetic, inside the cutoff region and in the taper
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    table = S.table_for(["Si"], oracle.mix_tersoff89)
    rec = table.reshape(-1, 14)[0]
    R, D, A, B, l1, l2 = (mpmath.mpf(float(rec[k])) for k in (10, 11, 13, 9, 12, 8))
    box = np.array([20.0, 20.0, 20.0])
    t = np.zeros(2, np.int32)

    def energy(r):
        fc = 1 if r <= R - D else mpmath.sin(mpmath.pi * ((R + D) - r) / (4 * D)) ** 2
        return fc * (A * mpmath.exp(-l1 * r) - B * mpmath.exp(-l2 * r))

    for r0 in (2.35, 2.95):
        x = np.array([[5.0, 5.0, 5.0], [5.0 + r0, 5.0, 5.0]])
        r = mpmath.mpf(float(x[1, 0])) - mpmath.mpf(float(x[0, 0]))
        nl = oracle.neighbors(x, box, 3.5)
        _, df_along = oracle.cs_pos(x, t, box, table, nl, 1, 0, forces=True)
        _, df_across = oracle.cs_pos(x, t, box, table, nl, 1, 1, forces=True)
        e2 = float(mpmath.diff(energy, r, 2))
        e1 = float(mpmath.diff(energy, r))
        assert abs(df_along[1, 0] + e2) <= 1e-10 * abs(e2), r0
        assert abs(df_across[1, 1] + e1 / float(r)) <= 1e-10 * abs(e1 / float(r)), r0
        # Newton's third law in the derivative
        assert abs(df_along[0, 0] - e2) <= 1e-10 * abs(e2)


def test_dimer_parameter_derivatives_closed_form():
    # dE/dtheta of a dimer (zeta = 0, b = 1) for A, B, lambda1, lambda2, R, D
    # in the taper, the oracle's complex step against 50-digit differentiation
    # of E = f_C(r; R, D) (A e^(-lambda1 r) - B e^(-lambda2 r))
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    table = S.table_for(["Si"], oracle.mix_tersoff89)
    rec = table.reshape(-1, 14)[0]
    box = np.array([20.0, 20.0, 20.0])
    t = np.zeros(2, np.int32)
    x = np.array([[5.0, 5.0, 5.0], [5.0 + 2.93, 5.0, 5.0]])
    r = mpmath.mpf(float(x[1, 0])) - mpmath.mpf(float(x[0, 0]))
    nl = oracle.neighbors(x, box, 3.5)
    fields = {"A": 13, "B": 9, "lambda1": 12, "lambda2": 8, "R": 10, "D": 11}
    base = {k: mpmath.mpf(float(rec[v])) for k, v in fields.items()}

    def energy(p):
        fc = mpmath.sin(mpmath.pi * ((p["R"] + p["D"]) - r) / (4 * p["D"])) ** 2
        return fc * (p["A"] * mpmath.exp(-p["lambda1"] * r) - p["B"] * mpmath.exp(-p["lambda2"] * r))

    for name, k in fields.items():
        def along(h, name=name):
            p = dict(base)
            p[name] = p[name] + h
            return energy(p)
        ref = float(mpmath.diff(along, 0))
        de, _ = oracle.cs_param(x, t, box, table, nl, k)
        assert abs(de - ref) <= 1e-10 * abs(ref), (name, de, ref)


# ----------------------------------------------------------------------------- trimer closed form
# A centre atom i with two neighbours j and k at unequal distances and an angle
# away from the tetrahedral one, j and k out of each other's range. Four directed
# bonds: i->j and i->k carry a bond order with one three-body term each (Eq. 7),
# j->i and k->i have zeta = 0 (b = 1). E = 1/2 sum of f_C [f_R + b f_A] (Eq. 5-6),
# written out here from the coordinates in 50-digit arithmetic with the
# textbook cutoff function, the exponent (lambda3 (r_ij - r_ik))^m, and the
# record convention: (ti, tj, tk) gives m, gamma, lambda3, c, d, h and the
# cutoff of f_C(r_ik); (ti, tj, tj) gives the pair terms and f_C(r_ij).
def _trimer_energy(mp, X, types, rec):
    """X: three mpf 3-vectors (i, j, k); rec(a, b, c) -> dict of mpf fields."""
    def sub(a, b):
        return [X[b][q] - X[a][q] for q in range(3)]

    def norm(v):
        return mp.sqrt(v[0] ** 2 + v[1] ** 2 + v[2] ** 2)

    def fc(r, R, D):
        if r < R - D:
            return mp.mpf(1)
        if r > R + D:
            return mp.mpf(0)
        return mp.mpf(1) / 2 - mp.sin(mp.pi / 2 * (r - R) / D) / 2

    def g(cs, p):
        c2, d2 = p["c"] ** 2, p["d"] ** 2
        return p["gamma"] * (1 + c2 / d2 - c2 / (d2 + (p["h"] - cs) ** 2))

    def bond(a, b, third):
        tp = rec(types[a], types[b], types[b])
        rab = norm(sub(a, b))
        zeta = mp.mpf(0)
        if third is not None:
            p3 = rec(types[a], types[b], types[third])
            vab, vac = sub(a, b), sub(a, third)
            rac = norm(vac)
            cs = (vab[0] * vac[0] + vab[1] * vac[1] + vab[2] * vac[2]) / (rab * rac)
            m = int(p3["m"])
            zeta = fc(rac, p3["R"], p3["D"]) * g(cs, p3) * mp.exp((p3["lambda3"] * (rab - rac)) ** m)
        b = mp.mpf(1) if zeta == 0 else (1 + (tp["beta"] * zeta) ** tp["n"]) ** (-1 / (2 * tp["n"]))
        return fc(rab, tp["R"], tp["D"]) * (tp["A"] * mp.exp(-tp["lambda1"] * rab)
                                             - b * tp["B"] * mp.exp(-tp["lambda2"] * rab)) / 2

    return bond(0, 1, 2) + bond(0, 2, 1) + bond(1, 0, None) + bond(2, 0, None)


def _trimer_positions(r_ij, r_ik, theta_deg, seed):
    th = math.radians(theta_deg)
    loc = np.array([[0.0, 0.0, 0.0], [r_ij, 0.0, 0.0],
                    [r_ik * math.cos(th), r_ik * math.sin(th), 0.0]])
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))  # generic orientation
    return loc @ q.T + np.array([11.3, 12.1, 10.7])


def _custom_sic_table():
    # The Si/C mixing rule's table with lambda3, m, gamma, h and the three-body
    # cutoff radius R varied record by record, so that taking any of them from
    # the wrong record changes the energy
    t = sic_table().reshape(8, 14).copy()
    for q in range(8):
        ti, tj, tk = q // 4, (q // 2) % 2, q % 2
        t[q, 2] = 0.9 + 0.15 * q
        t[q, 0] = 3.0 if q % 2 == 0 else 1.0
        t[q, 1] = 1.0 + 0.07 * q
        t[q, 5] = t[q, 5] + 0.02 * q
        if tj != tk:
            t[q, 10] = t[q, 10] + 0.004 * q
    return t.ravel()


TRIMERS = [
    # name, table builder, species (i, j, k), r_ij, r_ik (k in the taper of f_C(r_ik)), angle
    ("si-l3m3", lambda: S.with_lambda3(si_table(), 1.7322, 3), (0, 0, 0), 2.25, 2.92, 125.0),
    ("si-l3m1", lambda: S.with_lambda3(si_table(), 1.3, 1), (0, 0, 0), 2.25, 2.92, 125.0),
    ("si-c-si", _custom_sic_table, (0, 1, 0), 1.95, 2.88, 118.0),
    ("c-si-c", _custom_sic_table, (1, 0, 1), 2.0, 1.98, 140.0),
]


@pytest.mark.parametrize("case", TRIMERS, ids=[c[0] for c in TRIMERS])
def test_trimer_closed_form(case):
    mp = pytest.importorskip("mpmath").mp
    mp.dps = 50
    _, mk, species, r_ij, r_ik, theta = case
    table = mk()
    ns = round((table.size // 14) ** (1 / 3))
    x = _trimer_positions(r_ij, r_ik, theta, seed=hash(case[0]) % 1000)
    t = np.array(species, dtype=np.int32)
    box = np.array([30.0, 30.0, 30.0])
    assert np.linalg.norm(x[1] - x[2]) > 3.05  # j and k out of each other's range
    nl = oracle.neighbors(x, box, 3.5)
    e, f, _ = oracle.compute(x, t, box, table, nl)

    def rec(a, b, c):
        r = table.reshape(-1, 14)[(a * ns + b) * ns + c]
        return {name: mp.mpf(float(r[q])) for q, name in enumerate(oracle.FIELDS)}

    X = [[mp.mpf(float(v)) for v in row] for row in x]
    e_ref = _trimer_energy(mp, X, t, rec)
    assert abs(e - float(e_ref)) <= 1e-12 * abs(float(e_ref))
    f_ref = np.zeros((3, 3))
    for a in range(3):
        for c in range(3):
            def along(s, a=a, c=c):
                Y = [list(row) for row in X]
                Y[a][c] = s
                return _trimer_energy(mp, Y, t, rec)
            f_ref[a, c] = -float(mp.diff(along, X[a][c]))
    assert np.abs(f - f_ref).max() <= 1e-10 * np.abs(f_ref).max()
    # the three-body term matters: with gamma = 0 in every record the energy changes
    t0 = table.reshape(-1, 14).copy()
    t0[:, 1] = 0.0
    e0, _, _ = oracle.compute(x, t, box, t0.ravel(), nl)
    assert abs(e0 - e) > 1e-5 * abs(e)


# ----------------------------------------------------------------------------- MD units
# Metal units: mass in amu, length in Angstrom, time in ps, energy in eV. The
# conversion 1 amu A^2/ps^2 in eV follows from the CODATA 2018 atomic mass
# constant and the exact SI electronvolt; MD codes quote it to 8 digits
# (1.0364269e-4), so the pins below hold to 1e-7.
AMU_KG = 1.66053906660e-27
EV_J = 1.602176634e-19
MVV2EV_CODATA = AMU_KG * (1e-10 / 1e-12) ** 2 / EV_J


def _dimer_energy_derivs(r):
    el = W.ELEMENTS_TERSOFF89["Si"]
    A, B, l1, l2 = el[0], el[1], el[2], el[3]
    e1 = -l1 * A * math.exp(-l1 * r) + l2 * B * math.exp(-l2 * r)
    e2 = l1 * l1 * A * math.exp(-l1 * r) - l2 * l2 * B * math.exp(-l2 * r)
    return e1, e2


def test_md_one_step_metal_units():
    # A Si dimer at rest at r = 2.5 A (inside R - D: zeta = 0, b = 1, f_C = 1).
    # One velocity-Verlet step of dt: dx = dt^2/2 F0/m, v = dt/2 (F0 + F1)/m, in
    # metal units.
    table = si_table()
    m = W.MASS_AMU["Si"]
    dt = 0.002
    r0 = 2.5
    x = np.array([[10.0, 10.0, 10.0], [10.0 + r0, 10.0, 10.0]])
    v = np.zeros_like(x)
    t = np.zeros(2, np.int32)
    box = np.array([30.0, 30.0, 30.0])
    x1, v1, thermo, f1 = oracle.md_run(x, v, t, box, table, [m], dt, 1, 3.5, 0)
    e1, _ = _dimer_energy_derivs(r0)
    f0 = -e1  # force on atom 1 along +x
    dx_ref = 0.5 * dt * dt * f0 / (m * MVV2EV_CODATA)
    assert abs((x1[1, 0] - x[1, 0]) - dx_ref) <= 1e-7 * abs(dx_ref)
    assert abs((x1[0, 0] - x[0, 0]) + dx_ref) <= 1e-7 * abs(dx_ref)
    r1 = r0 + 2 * dx_ref
    f1_ref = -_dimer_energy_derivs(r1)[0]
    v_ref = 0.5 * dt * (f0 + f1_ref) / (m * MVV2EV_CODATA)
    assert abs(v1[1, 0] - v_ref) <= 1e-7 * abs(v_ref)
    ke_ref = 2 * 0.5 * m * v_ref * v_ref * MVV2EV_CODATA  # eV
    assert abs(thermo[0, 1] - ke_ref) <= 2e-7 * ke_ref


def test_md_dimer_period_metal_units():
    # Small oscillation of a Si dimer about its minimum r_e: the period is
    # 2 pi sqrt(mu / E''(r_e)) with the reduced mass mu = m/2, in metal units.
    el = W.ELEMENTS_TERSOFF89["Si"]
    A, B, l1, l2 = el[0], el[1], el[2], el[3]
    r_e = math.log(l1 * A / (l2 * B)) / (l1 - l2)  # E'(r_e) = 0
    _, k = _dimer_energy_derivs(r_e)
    m = W.MASS_AMU["Si"]
    period = 2 * math.pi * math.sqrt(0.5 * m * MVV2EV_CODATA / k)  # ps
    table = si_table()
    dt = 5e-5
    x = np.array([[10.0, 10.0, 10.0], [10.0 + r_e + 2e-3, 10.0, 10.0]])
    v = np.zeros_like(x)
    t = np.zeros(2, np.int32)
    box = np.array([30.0, 30.0, 30.0])
    rs = [x[1, 0] - x[0, 0]]
    nsteps = int(2.2 * period / dt)
    for _ in range(nsteps):
        x, v, _, _ = oracle.md_run(x, v, t, box, table, [m], dt, 1, 3.5, 0)
        rs.append(x[1, 0] - x[0, 0])
    u = np.array(rs) - r_e
    # downward zero crossings of r - r_e, linearly interpolated
    cross = [s + u[s] / (u[s] - u[s + 1]) for s in range(len(u) - 1) if u[s] > 0 >= u[s + 1]]
    assert len(cross) >= 2
    measured = (cross[1] - cross[0]) * dt
    assert abs(measured - period) <= 1e-4 * period

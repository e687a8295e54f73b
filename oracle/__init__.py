"""Python access to the FP64 CPU Tersoff oracle (``tersoff_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use this module; the library never does. The
shared object is compiled from source on first use (g++, -ffp-contract=off so
the neighbour-distance test is a fixed sequence of IEEE operations).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tersoff_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None

NPAR = 14
FIELDS = ("m", "gamma", "lambda3", "c", "d", "h", "n", "beta", "lambda2", "B", "R", "D",
          "lambda1", "A")


def build(force: bool = False) -> str:
    """Compile the oracle shared object if missing or older than its source."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    sig = {
        "oracle_abi_version": ([], I),
        "oracle_mix_tersoff89": ([I, P, P, P], I),
        "oracle_neighbors_brute": ([I, P, P, D, I, P, P], I),
        "oracle_neighbors_cells": ([I, P, P, D, I, P, P], I),
        "oracle_compute": ([I, P, P, P, I, P, P, P, I, I, P, P, P, P], I),
        "oracle_energy_n3": ([I, P, P, P, I, P, P], I),
        "oracle_cs_param": ([I, P, P, P, I, P, P, P, I, I, D, P, P], I),
        "oracle_cs_pos": ([I, P, P, P, I, P, P, P, I, I, I, D, P, P], I),
        "oracle_md_run": ([I, P, P, P, P, I, P, P, D, I, D, I, I, I, P, P], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def mix_tersoff89(elem, chi):
    elem = _f64(elem)
    chi = _f64(chi)
    ns = elem.shape[0]
    table = np.zeros(ns ** 3 * NPAR, dtype=np.float64)
    st = _load().oracle_mix_tersoff89(ns, _p(elem), _p(chi), _p(table))
    assert st == 0
    return table


def neighbors(x, box, rcut, cap=64, method="cells"):
    """Full neighbour lists: (cnt [N], nbr [N, cap]) ascending j, -1 padded."""
    x = _f64(x)
    box = _f64(box)
    n = x.shape[0]
    while True:
        cnt = np.zeros(n, dtype=np.int32)
        nbr = np.full((n, cap), -1, dtype=np.int32)
        fn = _load().oracle_neighbors_cells if method == "cells" else _load().oracle_neighbors_brute
        st = fn(n, _p(x), _p(box), float(rcut), cap, _p(cnt), _p(nbr))
        if st == 0:
            return cnt, nbr
        cap = int(cnt.max())


def compute(x, types, box, table, nl, nthreads=1, eatom=False):
    """Energy, forces (N,3), virial (6,) [, per-atom energy] over list ``nl``."""
    x = _f64(x)
    types = _i32(types)
    box = _f64(box)
    table = _f64(table)
    cnt, nbr = nl
    cnt = _i32(cnt)
    nbr = _i32(nbr)
    n = x.shape[0]
    ns = round((table.size // NPAR) ** (1.0 / 3.0))
    e = np.zeros(1)
    f = np.zeros((n, 3))
    w = np.zeros(6)
    ea = np.zeros(n) if eatom else None
    st = _load().oracle_compute(n, _p(x), _p(types), _p(box), ns, _p(table), _p(cnt), _p(nbr),
                                nbr.shape[1], int(nthreads), _p(e), _p(f), _p(w),
                                _p(ea) if eatom else None)
    assert st == 0
    if eatom:
        return float(e[0]), f, w, ea
    return float(e[0]), f, w


def energy_n3(x, types, box, table):
    x = _f64(x)
    types = _i32(types)
    box = _f64(box)
    table = _f64(table)
    ns = round((table.size // NPAR) ** (1.0 / 3.0))
    e = np.zeros(1)
    st = _load().oracle_energy_n3(x.shape[0], _p(x), _p(types), _p(box), ns, _p(table), _p(e))
    assert st == 0
    return float(e[0])


def cs_param(x, types, box, table, nl, p, h=1e-30):
    """Complex-step dE/dtheta_p and dF/dtheta_p for flat table index ``p``."""
    x = _f64(x)
    types = _i32(types)
    box = _f64(box)
    table = _f64(table)
    cnt, nbr = _i32(nl[0]), _i32(nl[1])
    ns = round((table.size // NPAR) ** (1.0 / 3.0))
    de = np.zeros(1)
    df = np.zeros((x.shape[0], 3))
    st = _load().oracle_cs_param(x.shape[0], _p(x), _p(types), _p(box), ns, _p(table),
                                 _p(cnt), _p(nbr), nbr.shape[1], int(p), float(h), _p(de),
                                 _p(df))
    assert st == 0
    return float(de[0]), df


def cs_pos(x, types, box, table, nl, a, c, h=1e-30, forces=False):
    """Complex-step dE/dx[a, c] (and, with forces=True, dF/dx[a, c] as (n, 3))."""
    x = _f64(x)
    types = _i32(types)
    box = _f64(box)
    table = _f64(table)
    cnt, nbr = _i32(nl[0]), _i32(nl[1])
    ns = round((table.size // NPAR) ** (1.0 / 3.0))
    de = np.zeros(1)
    df = np.zeros((x.shape[0], 3)) if forces else None
    st = _load().oracle_cs_pos(x.shape[0], _p(x), _p(types), _p(box), ns, _p(table), _p(cnt),
                               _p(nbr), nbr.shape[1], int(a), int(c), float(h), _p(de),
                               _p(df) if forces else None)
    assert st == 0
    return (float(de[0]), df) if forces else float(de[0])


def md_run(x, v, types, box, table, mass_per_species, dt, nsteps, rlist, rebuild_every,
           cap=64, nthreads=1):
    """Velocity-Verlet NVE; returns (x, v, thermo [nsteps,3], forces)."""
    x = _f64(x).copy()
    v = _f64(v).copy()
    types = _i32(types)
    box = _f64(box)
    table = _f64(table)
    mass = _f64(mass_per_species)
    ns = round((table.size // NPAR) ** (1.0 / 3.0))
    thermo = np.zeros((nsteps, 3))
    f = np.zeros_like(x)
    st = _load().oracle_md_run(x.shape[0], _p(x), _p(v), _p(types), _p(box), ns, _p(table),
                               _p(mass), float(dt), int(nsteps), float(rlist),
                               int(rebuild_every), int(cap), int(nthreads), _p(thermo), _p(f))
    assert st == 0, st
    return x, v, thermo, f


def table_index(ns, ti, tj, tk, field):
    """Flat index of ``field`` in record (ti, tj, tk)."""
    f = FIELDS.index(field) if isinstance(field, str) else int(field)
    return ((ti * ns + tj) * ns + tk) * NPAR + f

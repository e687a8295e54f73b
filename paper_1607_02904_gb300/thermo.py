"""Thermodynamic output of MD runs as JSON lines.

``tersoff_md_step`` fills a thermo array of potential, kinetic and total
energy (eV) per step. These helpers add the instantaneous temperature and,
given the virial of a ``compute`` call, the pressure, and write one JSON
object per step. Metal units: eV, K, Angstrom, bar.
"""
from __future__ import annotations

import json

import numpy as np

KB_EV_PER_K = 8.617333262e-5          # Boltzmann constant (CODATA 2018, exact SI definition)
EV_PER_A3_IN_BAR = 1.602176634e6      # 1 eV / A^3 = 1.602176634e-19 J / 1e-30 m^3, in bar


def temperature(ke_ev, n_atoms):
    """Instantaneous temperature 2 KE / (3 N kB) in K (no degrees of freedom
    removed for the conserved momentum)."""
    return 2.0 * np.asarray(ke_ev, dtype=np.float64) / (3.0 * n_atoms * KB_EV_PER_K)


def pressure(temperature_k, virial, n_atoms, volume):
    """Pressure in bar from the kinetic part N kB T and the virial's trace
    (the library's virial: W_ab summed over terms, positive when repulsive,
    components xx yy zz xy xz yz), over the volume in A^3."""
    w = np.asarray(virial, dtype=np.float64)
    return (n_atoms * KB_EV_PER_K * temperature_k + (w[0] + w[1] + w[2]) / 3.0) / volume * \
        EV_PER_A3_IN_BAR


def records(thermo, n_atoms, step0=0, virials=None, volume=None):
    """One dict per row of a thermo array (nsteps x 3: potential, kinetic and
    total energy in eV): step (step0 + 1 for the first row: the state after
    that step), the three energies and the temperature; with per-step virials
    (nsteps x 6) and the volume, also the pressure."""
    t = np.asarray(thermo, dtype=np.float64).reshape(-1, 3)
    temp = temperature(t[:, 1], n_atoms)
    out = []
    for k, (pe, ke, et) in enumerate(t):
        r = {"step": int(step0 + k + 1), "pe_eV": float(pe), "ke_eV": float(ke),
             "etot_eV": float(et), "temperature_K": float(temp[k])}
        if virials is not None and volume is not None:
            r["pressure_bar"] = float(pressure(temp[k], np.asarray(virials)[k], n_atoms, volume))
        out.append(r)
    return out


def write_jsonl(path, thermo, n_atoms, step0=0, virials=None, volume=None, append=True):
    """Appends (or writes) the records of a thermo array to `path`, one JSON
    object per line; returns the number of lines written."""
    recs = records(thermo, n_atoms, step0, virials, volume)
    with open(path, "a" if append else "w") as fh:
        for r in recs:
            fh.write(json.dumps(r) + "\n")
    return len(recs)

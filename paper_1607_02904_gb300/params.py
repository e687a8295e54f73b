"""Per-triplet Tersoff parameter tables.

Layout (shared with the C ABI, include/tersoff.h): n_species^3 records of 14
values, record ((ti*ns + tj)*ns + tk), fields in ``FIELDS`` order. Record
(ti,tj,tj) gives the pair terms of bond i-j; record (ti,tj,tk) the three-body
terms of the triplet and the cutoff of the i-k distance.
"""
from __future__ import annotations

import numpy as np

FIELDS = ("m", "gamma", "lambda3", "c", "d", "h", "n", "beta", "lambda2", "B", "R", "D",
          "lambda1", "A")


def mix_tersoff89(elem, chi):
    """Tersoff (Phys. Rev. B 39, 5566 (1989)) multicomponent table.

    elem: (ns, 11) element records (A, B, lambda, mu, beta, n, c, d, h, R, S),
    R and S being the inner and outer cutoff radii; chi: (ns, ns) bond
    softening. Pair terms of bond i-j: A = sqrt(A_i A_j), B = chi_ij
    sqrt(B_i B_j), lambda1 = (lambda_i + lambda_j)/2, lambda2 = (mu_i + mu_j)/2,
    beta, n from element i. Three-body terms: c, d, h from element i, gamma = 1,
    no lambda3 term (m = 3, lambda3 = 0). Cutoff of the i-k distance from
    R_ik = sqrt(R_i R_k), S_ik = sqrt(S_i S_k) as R = (R_ik + S_ik)/2,
    D = (S_ik - R_ik)/2.
    """
    e = np.asarray(elem, dtype=np.float64)
    chi = np.asarray(chi, dtype=np.float64)
    ns = e.shape[0]
    t = np.zeros((ns, ns, ns, len(FIELDS)), dtype=np.float64)
    A, B, lam, mu, beta, n, c, d, h, Rin, Sout = (e[:, q] for q in range(11))
    i, j, k = np.meshgrid(np.arange(ns), np.arange(ns), np.arange(ns), indexing="ij")
    t[..., 0] = 3.0
    t[..., 1] = 1.0
    t[..., 2] = 0.0
    t[..., 3] = c[i]
    t[..., 4] = d[i]
    t[..., 5] = h[i]
    t[..., 6] = n[i]
    t[..., 7] = beta[i]
    t[..., 8] = 0.5 * (mu[i] + mu[j])
    t[..., 9] = chi[i, j] * np.sqrt(B[i] * B[j])
    rik = np.sqrt(Rin[i] * Rin[k])
    sik = np.sqrt(Sout[i] * Sout[k])
    t[..., 10] = 0.5 * (rik + sik)
    t[..., 11] = 0.5 * (sik - rik)
    t[..., 12] = 0.5 * (lam[i] + lam[j])
    t[..., 13] = np.sqrt(A[i] * A[j])
    return t.ravel()


def read_table(path, species):
    """Per-triplet table from a text file of element-triplet entries.

    Each entry is three element names (e_i e_j e_k) followed by the 14 values
    of its record in ``FIELDS`` order (m, gamma, lambda3, c, d, h, n, beta,
    lambda2, B, R, D, lambda1, A); an entry may run over several lines, and
    text after '#' is a comment. ``species`` lists the element names in
    species-index order; entries naming other elements are skipped. Every
    triplet of the listed elements must appear exactly once. Returns the flat
    table (n_species^3 x 14) for tersoff_params.
    """
    names = list(species)
    index = {e: q for q, e in enumerate(names)}
    if len(index) != len(names):
        raise ValueError("duplicate element names")
    tokens = []
    with open(path) as fh:
        for line in fh:
            tokens.extend(line.split("#", 1)[0].split())
    per = 3 + len(FIELDS)
    if len(tokens) % per:
        raise ValueError(f"{path}: {len(tokens)} fields do not form entries of {per}")
    ns = len(names)
    t = np.full((ns, ns, ns, len(FIELDS)), np.nan)
    seen = set()
    for q in range(0, len(tokens), per):
        e = tokens[q:q + 3]
        if not all(x in index for x in e):
            continue
        key = tuple(index[x] for x in e)
        if key in seen:
            raise ValueError(f"{path}: entry {' '.join(e)} appears twice")
        seen.add(key)
        t[key] = [float(v) for v in tokens[q + 3:q + per]]
    if len(seen) != ns ** 3:
        missing = [" ".join(names[a] for a in (i, j, k)) for i in range(ns) for j in range(ns)
                   for k in range(ns) if (i, j, k) not in seen]
        raise ValueError(f"{path}: no entry for {', '.join(missing)}")
    return t.ravel()


def write_table(path, table, species):
    """Writes a flat per-triplet table in the format ``read_table`` reads, one
    entry per line, values with 17 significant digits (exact round trip)."""
    names = list(species)
    ns = len(names)
    t = np.asarray(table, dtype=np.float64).reshape(ns, ns, ns, len(FIELDS))
    with open(path, "w") as fh:
        fh.write("# e_i e_j e_k " + " ".join(FIELDS) + "\n")
        for i in range(ns):
            for j in range(ns):
                for k in range(ns):
                    vals = " ".join(f"{v:.17g}" for v in t[i, j, k])
                    fh.write(f"{names[i]} {names[j]} {names[k]} {vals}\n")

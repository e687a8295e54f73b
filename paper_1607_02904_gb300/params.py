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

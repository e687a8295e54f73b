// Tersoff oracle: plain, slow, FP64 CPU evaluation of the Tersoff potential.
//
// TEST INFRASTRUCTURE ONLY. This file is the independent reference that the
// CUDA library is checked against. It shares no code, header, table or
// constant with the library; only the tests, the package's smoke check and the
// benchmark's CPU-baseline leg load it. Nothing on the product path may call it.
//
// What it computes (Hoehnerbach, Ismail, Bientinesi, "The Vectorization of the
// Tersoff Multi-Body Potential", SC'16):
//   * neighbour sets  N_i = { j : r_ij <= r_C, j != i }            (Sec. II, Eq. 4)
//   * the Tersoff energy                                           (Sec. III, Eq. 5-7)
//       E     = 1/2 sum_i sum_{j in N_i} f_C(r_ij) [ f_R(r_ij) + b_ij f_A(r_ij) ]
//       b_ij  = (1 + (beta zeta_ij)^n)^(-1/(2n))
//       zeta_ij = sum_{k in N_i \ {j}} f_C(r_ik) g(theta_ijk) exp((lambda3 (r_ij - r_ik))^m)
//     with the functional forms the paper leaves out ("trivial definitions",
//     Sec. III) taken from Tersoff's papers:
//       f_C(r) = 1, 1/2 - 1/2 sin(pi/2 (r-R)/D), 0   for r < R-D, |r-R| <= D, r > R+D
//       f_R(r) = A exp(-lambda1 r),   f_A(r) = -B exp(-lambda2 r)
//       g(t)   = gamma (1 + c^2/d^2 - c^2 / (d^2 + (h - cos t)^2))
//   * forces F_a = -dE/dx_a (Sec. II, Eq. 1), evaluated in the loop order of
//     Algorithm 2 (first K loop accumulates zeta, then V and its zeta-derivative,
//     then a second K loop applies the three-body force terms);
//   * the virial W_ab = sum over terms of (x_a - x_i)_a F_b (relative to the
//     term's centre atom i);
//   * velocity-Verlet MD in metal units, rebuilding neighbour lists on a fixed
//     period (the skin scheme of Sec. III);
//   * derivatives with respect to parameters and positions by the complex-step
//     method (f'(x) = Im f(x + i h) / h, exact to rounding for analytic f): the
//     whole evaluation is a template over the scalar type and is instantiated
//     for double and std::complex<double>.
//   * Tersoff's 1989 Si/C mixing rule for building the per-triplet table.
//
// Parameter table layout: n_species^3 records of 14 doubles, record
// ((ti*ns + tj)*ns + tk), fields in the order
//   m, gamma, lambda3, c, d, h, n, beta, lambda2, B, R, D, lambda1, A.
// Record (ti,tj,tj) supplies the pair terms of bond i-j (n, beta, lambda2, B,
// lambda1, A and the R, D of f_C(r_ij)); record (ti,tj,tk) supplies the
// three-body terms (m, gamma, lambda3, c, d, h and the R, D of f_C(r_ik)).
//
// Minimum image: d = x_j - x_i; d -= L * nearbyint(d * (1/L)), per axis,
// with r^2 = (dx*dx + dy*dy) + dz*dz. Built with -ffp-contract=off so the
// neighbour test is a fixed sequence of IEEE operations.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int NPAR = 14;
enum {
  I_M = 0, I_GAMMA, I_LAM3, I_C, I_D, I_H, I_N, I_BETA, I_LAM2, I_B, I_R, I_DD, I_LAM1, I_A
};
constexpr double PI = 3.14159265358979323846;

// Metal units: mass amu, distance Angstrom, time ps, energy eV.
// 1 amu*A^2/ps^2 expressed in eV.
constexpr double MVV2EV = 1.0364269e-4;

using cd = std::complex<double>;

inline double re(double x) { return x; }
inline double re(const cd& x) { return x.real(); }

// ---------------------------------------------------------------- geometry
inline double min_image(double d, double L, double invL) {
  return d - L * std::nearbyint(d * invL);
}

inline double dist2(const double* xi, const double* xj, const double* box,
                    const double* inv) {
  double dx = min_image(xj[0] - xi[0], box[0], inv[0]);
  double dy = min_image(xj[1] - xi[1], box[1], inv[1]);
  double dz = min_image(xj[2] - xi[2], box[2], inv[2]);
  return dx * dx + dy * dy + dz * dz;
}

// ---------------------------------------------------------------- pieces of Eq. 5-7
// In the taper, written in delta = R + D - r: 1/2 - 1/2 sin(pi/2 (r-R)/D) =
// sin^2(pi delta/(4D)) and -pi/(4D) cos(pi/2 (r-R)/D) = -pi/(4D) sin(pi
// delta/(2D)) (the same functions; these forms keep their relative accuracy
// as r -> R + D, where f_C ~ delta^2 and the textbook form cancels).
template <class T> T f_c(const T& r, const T& R, const T& D) {
  if (re(r) < re(R - D)) return T(1.0);
  if (re(r) > re(R + D)) return T(0.0);
  T s = std::sin(0.25 * PI * ((R + D) - r) / D);
  return s * s;
}
template <class T> T f_c_d(const T& r, const T& R, const T& D) {
  if (re(r) < re(R - D) || re(r) > re(R + D)) return T(0.0);
  return -0.25 * PI / D * std::sin(0.5 * PI * ((R + D) - r) / D);
}
template <class T> T g_ang(const T& cs, const T* p) {
  T c2 = p[I_C] * p[I_C], d2 = p[I_D] * p[I_D];
  T t = p[I_H] - cs;
  return p[I_GAMMA] * (1.0 + c2 / d2 - c2 / (d2 + t * t));
}
template <class T> T g_ang_d(const T& cs, const T* p) {  // dg / dcos(theta)
  T c2 = p[I_C] * p[I_C], d2 = p[I_D] * p[I_D];
  T t = p[I_H] - cs;
  T den = d2 + t * t;
  return -2.0 * p[I_GAMMA] * c2 * t / (den * den);
}
inline int m_of(const double* p) { return (int)std::lround(p[I_M]); }
inline int m_of(const cd* p) { return (int)std::lround(p[I_M].real()); }

// exp((lambda3 * dr)^m) and its derivative with respect to dr
template <class T> void exp_term(const T& dr, const T* p, T& e, T& de) {
  int m = m_of(p);
  T a = p[I_LAM3] * dr;
  T am1 = T(1.0);
  for (int q = 1; q < m; ++q) am1 = am1 * a;
  T am = am1 * a;
  e = std::exp(am);
  de = e * (double)m * p[I_LAM3] * am1;
}

// b(zeta) and db/dzeta (reading: at zeta == 0 the derivative term is taken as 0)
template <class T> void bond_order(const T& zeta, const T* p, T& b, T& db) {
  if (re(zeta) == 0.0) {
    b = T(1.0);
    db = T(0.0);
    return;
  }
  T n = p[I_N];
  T u = std::pow(p[I_BETA] * zeta, n);
  T e = -1.0 / (2.0 * n);
  b = std::pow(1.0 + u, e);
  db = -0.5 * std::pow(1.0 + u, e - 1.0) * u / zeta;
}

struct NbrView {
  const int* cnt;
  const int* nbr;
  int cap;
};

// One evaluation of E, F, W following Algorithm 2. Positions and the table are
// of scalar type T (double, or complex for complex-step derivatives). The
// neighbour list and the periodic image shifts are taken from the real parts.
template <class T>
void evaluate(int /*n*/, const T* x, const int* types, const double* box, int ns,
              const T* table, NbrView nl, int i_begin, int i_end, T* energy,
              T* forces, T* virial, T* eatom) {
  double inv[3] = {1.0 / box[0], 1.0 / box[1], 1.0 / box[2]};
  std::vector<T> dvec;  // per neighbour of i: displacement x_k - x_i (3)
  std::vector<T> rlen;
  T E = T(0.0);
  T W[6] = {T(0.0), T(0.0), T(0.0), T(0.0), T(0.0), T(0.0)};
  auto addW = [&](const T* d, const T* f) {
    W[0] += d[0] * f[0];
    W[1] += d[1] * f[1];
    W[2] += d[2] * f[2];
    W[3] += d[0] * f[1];
    W[4] += d[0] * f[2];
    W[5] += d[1] * f[2];
  };
  for (int i = i_begin; i < i_end; ++i) {
    const int ti = types[i];
    const int zi = nl.cnt[i];
    const int* li = nl.nbr + (size_t)i * nl.cap;
    dvec.assign((size_t)zi * 3, T(0.0));
    rlen.assign(zi, T(0.0));
    for (int q = 0; q < zi; ++q) {
      int j = li[q];
      for (int a = 0; a < 3; ++a) {
        T d = x[3 * j + a] - x[3 * i + a];
        double shift = box[a] * std::nearbyint(re(d) * inv[a]);
        dvec[3 * q + a] = d - shift;
      }
      T* dq = &dvec[3 * q];
      rlen[q] = std::sqrt(dq[0] * dq[0] + dq[1] * dq[1] + dq[2] * dq[2]);
    }
    T* Fi = forces + 3 * (size_t)i;
    for (int qj = 0; qj < zi; ++qj) {
      const int j = li[qj];
      const int tj = types[j];
      const T* p2 = table + (size_t)((ti * ns + tj) * ns + tj) * NPAR;
      const T rij = rlen[qj];
      if (re(rij) > re(p2[I_R] + p2[I_DD])) continue;  // f_C(r_ij) = 0: no term
      const T* dij = &dvec[3 * qj];
      T uij[3] = {dij[0] / rij, dij[1] / rij, dij[2] / rij};

      // first K loop: zeta_ij
      T zeta = T(0.0);
      for (int qk = 0; qk < zi; ++qk) {
        if (qk == qj) continue;
        const int k = li[qk];
        const T* p3 = table + (size_t)((ti * ns + tj) * ns + types[k]) * NPAR;
        const T rik = rlen[qk];
        if (re(rik) > re(p3[I_R] + p3[I_DD])) continue;  // f_C(r_ik) = 0: no term
        const T* dik = &dvec[3 * qk];
        T cs = (dij[0] * dik[0] + dij[1] * dik[1] + dij[2] * dik[2]) / (rij * rik);
        T e, de;
        exp_term(rij - rik, p3, e, de);
        zeta += f_c(rik, p3[I_R], p3[I_DD]) * g_ang(cs, p3) * e;
      }

      // V(i, j, zeta) and its explicit r_ij dependence
      T b, db;
      bond_order(zeta, p2, b, db);
      T fc = f_c(rij, p2[I_R], p2[I_DD]);
      T dfc = f_c_d(rij, p2[I_R], p2[I_DD]);
      T fr = p2[I_A] * std::exp(-p2[I_LAM1] * rij);
      T fa = -p2[I_B] * std::exp(-p2[I_LAM2] * rij);
      T dfr = -p2[I_LAM1] * fr;
      T dfa = -p2[I_LAM2] * fa;
      T V = 0.5 * fc * (fr + b * fa);
      E += V;
      if (eatom) eatom[i] += V;
      T dVdr = 0.5 * (dfc * (fr + b * fa) + fc * (dfr + b * dfa));
      T* Fj = forces + 3 * (size_t)j;
      T fj[3];
      for (int a = 0; a < 3; ++a) {
        fj[a] = -dVdr * uij[a];  // -dV/dx_j
        Fj[a] += fj[a];
        Fi[a] -= fj[a];
      }
      addW(dij, fj);

      // delta zeta = dV / dzeta
      T dz = 0.5 * fc * fa * db;

      // second K loop: three-body forces
      for (int qk = 0; qk < zi; ++qk) {
        if (qk == qj) continue;
        const int k = li[qk];
        const T* p3 = table + (size_t)((ti * ns + tj) * ns + types[k]) * NPAR;
        const T rik = rlen[qk];
        if (re(rik) > re(p3[I_R] + p3[I_DD])) continue;
        const T* dik = &dvec[3 * qk];
        T uik[3] = {dik[0] / rik, dik[1] / rik, dik[2] / rik};
        T cs = uij[0] * uik[0] + uij[1] * uik[1] + uij[2] * uik[2];
        T fck = f_c(rik, p3[I_R], p3[I_DD]);
        T dfck = f_c_d(rik, p3[I_R], p3[I_DD]);
        T g = g_ang(cs, p3);
        T dg = g_ang_d(cs, p3);
        T e, de;
        exp_term(rij - rik, p3, e, de);
        T dzj[3], dzk[3], dzi[3];
        for (int a = 0; a < 3; ++a) {
          T dcos_j = (uik[a] - cs * uij[a]) / rij;  // d cos / d x_j
          T dcos_k = (uij[a] - cs * uik[a]) / rik;  // d cos / d x_k
          T dcos_i = -dcos_j - dcos_k;               // d cos / d x_i
          // d zeta(i,j,k) / d x_a for a = j, k, i
          dzj[a] = fck * (dg * dcos_j * e + g * de * uij[a]);
          dzk[a] = dfck * uik[a] * g * e + fck * (dg * dcos_k * e - g * de * uik[a]);
          dzi[a] = -dfck * uik[a] * g * e +
                   fck * (dg * dcos_i * e + g * de * (uik[a] - uij[a]));
        }
        T* Fk = forces + 3 * (size_t)k;
        T fjk[3], fkk[3];
        for (int a = 0; a < 3; ++a) {
          Fi[a] -= dz * dzi[a];
          fjk[a] = -dz * dzj[a];
          fkk[a] = -dz * dzk[a];
          Fj[a] += fjk[a];
          Fk[a] += fkk[a];
        }
        addW(dij, fjk);
        addW(dik, fkk);
      }
    }
  }
  *energy += E;
  for (int c = 0; c < 6; ++c) virial[c] += W[c];
}

// Brute-force energy: every ordered pair and triple, no neighbour list.
template <class T>
T energy_n3(int n, const T* x, const int* types, const double* box, int ns,
            const T* table) {
  double inv[3] = {1.0 / box[0], 1.0 / box[1], 1.0 / box[2]};
  auto disp = [&](int i, int j, T* d) {
    for (int a = 0; a < 3; ++a) {
      T dd = x[3 * j + a] - x[3 * i + a];
      dd = dd - box[a] * std::nearbyint(re(dd) * inv[a]);
      d[a] = dd;
    }
  };
  T E = T(0.0);
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      const T* p2 = table + (size_t)((types[i] * ns + types[j]) * ns + types[j]) * NPAR;
      T dij[3];
      disp(i, j, dij);
      T rij = std::sqrt(dij[0] * dij[0] + dij[1] * dij[1] + dij[2] * dij[2]);
      if (re(rij) > re(p2[I_R] + p2[I_DD])) continue;  // f_C(r_ij) = 0
      T zeta = T(0.0);
      for (int k = 0; k < n; ++k) {
        if (k == i || k == j) continue;
        const T* p3 = table + (size_t)((types[i] * ns + types[j]) * ns + types[k]) * NPAR;
        T dik[3];
        disp(i, k, dik);
        T rik = std::sqrt(dik[0] * dik[0] + dik[1] * dik[1] + dik[2] * dik[2]);
        if (re(rik) > re(p3[I_R] + p3[I_DD])) continue;  // f_C(r_ik) = 0
        T cs = (dij[0] * dik[0] + dij[1] * dik[1] + dij[2] * dik[2]) / (rij * rik);
        T e, de;
        exp_term(rij - rik, p3, e, de);
        zeta += f_c(rik, p3[I_R], p3[I_DD]) * g_ang(cs, p3) * e;
      }
      T b, db;
      bond_order(zeta, p2, b, db);
      T fc = f_c(rij, p2[I_R], p2[I_DD]);
      T fr = p2[I_A] * std::exp(-p2[I_LAM1] * rij);
      T fa = -p2[I_B] * std::exp(-p2[I_LAM2] * rij);
      E += 0.5 * fc * (fr + b * fa);
    }
  }
  return E;
}

int neighbors_brute(int n, const double* x, const double* box, double rcut, int cap,
                    int* cnt, int* nbr) {
  double inv[3] = {1.0 / box[0], 1.0 / box[1], 1.0 / box[2]};
  double rc2 = rcut * rcut;
  int status = 0;
  for (int i = 0; i < n; ++i) {
    int c = 0;
    for (int j = 0; j < n; ++j) {  // ascending j
      if (j == i) continue;
      if (dist2(x + 3 * i, x + 3 * j, box, inv) <= rc2) {
        if (c < cap) nbr[(size_t)i * cap + c] = j;
        ++c;
      }
    }
    cnt[i] = c;
    if (c > cap) status = 3;
  }
  return status;
}

// Same set as neighbors_brute, found through a cell grid (cell edge >= rcut).
int neighbors_cells(int n, const double* x, const double* box, double rcut, int cap,
                    int* cnt, int* nbr) {
  int nc[3];
  for (int a = 0; a < 3; ++a) nc[a] = (int)std::floor(box[a] / rcut);
  if (nc[0] < 3 || nc[1] < 3 || nc[2] < 3)
    return neighbors_brute(n, x, box, rcut, cap, cnt, nbr);
  double inv[3] = {1.0 / box[0], 1.0 / box[1], 1.0 / box[2]};
  double rc2 = rcut * rcut;
  const long ncell = (long)nc[0] * nc[1] * nc[2];
  std::vector<int> cell_of(n), head(ncell + 1, 0), order(n);
  for (int i = 0; i < n; ++i) {
    int c3[3];
    for (int a = 0; a < 3; ++a) {
      double w = x[3 * i + a] - box[a] * std::floor(x[3 * i + a] * inv[a]);
      int c = (int)(w / box[a] * nc[a]);
      if (c < 0) c = 0;
      if (c >= nc[a]) c = nc[a] - 1;
      c3[a] = c;
    }
    cell_of[i] = (c3[2] * nc[1] + c3[1]) * nc[0] + c3[0];
    head[cell_of[i] + 1]++;
  }
  for (long c = 0; c < ncell; ++c) head[c + 1] += head[c];
  {
    std::vector<int> fill(head.begin(), head.end() - 1);
    for (int i = 0; i < n; ++i) order[fill[cell_of[i]]++] = i;
  }
  int status = 0;
  std::vector<int> found;
  for (int i = 0; i < n; ++i) {
    int ci = cell_of[i];
    int cx = ci % nc[0], cy = (ci / nc[0]) % nc[1], cz = ci / (nc[0] * nc[1]);
    found.clear();
    for (int oz = -1; oz <= 1; ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          int ax = (cx + ox + nc[0]) % nc[0];
          int ay = (cy + oy + nc[1]) % nc[1];
          int az = (cz + oz + nc[2]) % nc[2];
          long c = ((long)az * nc[1] + ay) * nc[0] + ax;
          for (int s = head[c]; s < head[c + 1]; ++s) {
            int j = order[s];
            if (j == i) continue;
            if (dist2(x + 3 * i, x + 3 * j, box, inv) <= rc2) found.push_back(j);
          }
        }
    std::sort(found.begin(), found.end());
    int c = (int)found.size();
    for (int q = 0; q < c && q < cap; ++q) nbr[(size_t)i * cap + q] = found[q];
    cnt[i] = c;
    if (c > cap) status = 3;
  }
  return status;
}

// E, F, W in double with an optional thread split over centre atoms i.
int compute_real(int n, const double* x, const int* types, const double* box, int ns,
                 const double* table, NbrView nl, int nthreads, double* energy,
                 double* forces, double* virial, double* eatom) {
  std::memset(forces, 0, sizeof(double) * 3 * (size_t)n);
  if (eatom) std::memset(eatom, 0, sizeof(double) * (size_t)n);
  *energy = 0.0;
  for (int c = 0; c < 6; ++c) virial[c] = 0.0;
  int nt = nthreads > 0 ? nthreads : 1;
#ifndef _OPENMP
  nt = 1;
#endif
  if (nt == 1) {
    evaluate<double>(n, x, types, box, ns, table, nl, 0, n, energy, forces, virial, eatom);
    return 0;
  }
  std::vector<std::vector<double>> fbuf(nt, std::vector<double>(3 * (size_t)n, 0.0));
  std::vector<double> ebuf(nt, 0.0), wbuf(6 * (size_t)nt, 0.0);
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
  {
    int t = omp_get_thread_num();
    int nth = omp_get_num_threads();
    int lo = (int)((long)n * t / nth), hi = (int)((long)n * (t + 1) / nth);
    evaluate<double>(n, x, types, box, ns, table, nl, lo, hi, &ebuf[t], fbuf[t].data(),
                     &wbuf[6 * t], eatom);
  }
#endif
  for (int t = 0; t < nt; ++t) {
    *energy += ebuf[t];
    for (int c = 0; c < 6; ++c) virial[c] += wbuf[6 * t + c];
    for (size_t q = 0; q < 3 * (size_t)n; ++q) forces[q] += fbuf[t][q];
  }
  return 0;
}

}  // namespace

extern "C" {

int oracle_abi_version() { return 1; }

// Tersoff (1989) multicomponent mixing. elem: ns x 11 records
// (A, B, lambda, mu, beta, n, c, d, h, R, S) with R, S the inner/outer cutoff
// radii; chi: ns x ns. Fills the ns^3 x 14 table (layout in the file header).
int oracle_mix_tersoff89(int ns, const double* elem, const double* chi, double* table) {
  if (ns <= 0) return 1;
  for (int i = 0; i < ns; ++i)
    for (int j = 0; j < ns; ++j)
      for (int k = 0; k < ns; ++k) {
        const double* ei = elem + 11 * i;
        const double* ej = elem + 11 * j;
        const double* ek = elem + 11 * k;
        double* p = table + (size_t)((i * ns + j) * ns + k) * NPAR;
        // three-body terms: element i; no lambda3 term in the 1989 form
        p[I_M] = 3.0;
        p[I_GAMMA] = 1.0;
        p[I_LAM3] = 0.0;
        p[I_C] = ei[6];
        p[I_D] = ei[7];
        p[I_H] = ei[8];
        // pair terms of bond i-j
        p[I_N] = ei[5];
        p[I_BETA] = ei[4];
        p[I_LAM2] = 0.5 * (ei[3] + ej[3]);
        p[I_B] = chi[i * ns + j] * std::sqrt(ei[1] * ej[1]);
        p[I_LAM1] = 0.5 * (ei[2] + ej[2]);
        p[I_A] = std::sqrt(ei[0] * ej[0]);
        // cutoff of the i-k distance (equal to i-j on the pair record j == k)
        double Rik = std::sqrt(ei[9] * ek[9]);
        double Sik = std::sqrt(ei[10] * ek[10]);
        p[I_R] = 0.5 * (Rik + Sik);
        p[I_DD] = 0.5 * (Sik - Rik);
      }
  return 0;
}

// Full neighbour lists (Eq. 4), ascending j, capacity cap per atom.
// Returns 0, or 3 when some atom has more than cap neighbours (cnt holds the
// true counts; entries beyond cap are not written).
int oracle_neighbors_brute(int n, const double* x, const double* box, double rcut,
                           int cap, int* cnt, int* nbr) {
  return neighbors_brute(n, x, box, rcut, cap, cnt, nbr);
}
int oracle_neighbors_cells(int n, const double* x, const double* box, double rcut,
                           int cap, int* cnt, int* nbr) {
  return neighbors_cells(n, x, box, rcut, cap, cnt, nbr);
}

// Energy, forces (n x 3), virial (xx, yy, zz, xy, xz, yz) and optional per-atom
// energy over a given neighbour list.
int oracle_compute(int n, const double* x, const int* types, const double* box, int ns,
                   const double* table, const int* cnt, const int* nbr, int cap,
                   int nthreads, double* energy, double* forces, double* virial,
                   double* eatom) {
  NbrView nl{cnt, nbr, cap};
  return compute_real(n, x, types, box, ns, table, nl, nthreads, energy, forces, virial,
                      eatom);
}

// Brute-force energy with no neighbour list (all ordered i, j, k).
int oracle_energy_n3(int n, const double* x, const int* types, const double* box, int ns,
                     const double* table, double* energy) {
  *energy = energy_n3<double>(n, x, types, box, ns, table);
  return 0;
}

// Complex-step derivatives with respect to one table entry (index p into the
// flat ns^3*14 table): dE/dtheta_p and dF/dtheta_p (n x 3).
int oracle_cs_param(int n, const double* x, const int* types, const double* box, int ns,
                    const double* table, const int* cnt, const int* nbr, int cap, int p,
                    double h, double* dE, double* dF) {
  size_t nt = (size_t)ns * ns * ns * NPAR;
  if (p < 0 || (size_t)p >= nt) return 1;
  std::vector<cd> xz(3 * (size_t)n), tz(nt), fz(3 * (size_t)n, cd(0.0));
  for (size_t q = 0; q < 3 * (size_t)n; ++q) xz[q] = cd(x[q], 0.0);
  for (size_t q = 0; q < nt; ++q) tz[q] = cd(table[q], 0.0);
  tz[p] += cd(0.0, h);
  cd E(0.0), W[6];
  NbrView nl{cnt, nbr, cap};
  evaluate<cd>(n, xz.data(), types, box, ns, tz.data(), nl, 0, n, &E, fz.data(), W,
               (cd*)nullptr);
  *dE = E.imag() / h;
  if (dF)
    for (size_t q = 0; q < 3 * (size_t)n; ++q) dF[q] = fz[q].imag() / h;
  return 0;
}

// Complex-step derivatives with respect to position component x[3*a + c]:
// dE/dx_ac, and (dF optional, n x 3) dF/dx_ac, the column (a, c) of minus the
// Hessian.
int oracle_cs_pos(int n, const double* x, const int* types, const double* box, int ns,
                  const double* table, const int* cnt, const int* nbr, int cap, int a,
                  int c, double h, double* dE, double* dF) {
  size_t nt = (size_t)ns * ns * ns * NPAR;
  std::vector<cd> xz(3 * (size_t)n), tz(nt), fz(3 * (size_t)n, cd(0.0));
  for (size_t q = 0; q < 3 * (size_t)n; ++q) xz[q] = cd(x[q], 0.0);
  for (size_t q = 0; q < nt; ++q) tz[q] = cd(table[q], 0.0);
  xz[3 * (size_t)a + c] += cd(0.0, h);
  cd E(0.0), W[6];
  NbrView nl{cnt, nbr, cap};
  evaluate<cd>(n, xz.data(), types, box, ns, tz.data(), nl, 0, n, &E, fz.data(), W,
               (cd*)nullptr);
  *dE = E.imag() / h;
  if (dF)
    for (size_t q = 0; q < 3 * (size_t)n; ++q) dF[q] = fz[q].imag() / h;
  return 0;
}

// Velocity-Verlet NVE in metal units (x in A, v in A/ps, dt in ps, masses in
// amu). Before the first step the lists are built and forces evaluated; each
// step is: v += dt/2 F/m; x += dt v; rebuild the list when (step+1) is a
// multiple of rebuild_every; F = F(x); v += dt/2 F/m. thermo (nsteps x 3):
// potential, kinetic and total energy after each step. Positions are not
// wrapped back into the box (the minimum image handles any translate).
int oracle_md_run(int n, double* x, double* v, const int* types, const double* box,
                  int ns, const double* table, const double* mass, double dt, int nsteps,
                  double rlist, int rebuild_every, int cap, int nthreads,
                  double* thermo, double* forces_out) {
  std::vector<int> cnt(n), nbr((size_t)n * cap);
  std::vector<double> F(3 * (size_t)n);
  double E, W[6];
  int st = neighbors_cells(n, x, box, rlist, cap, cnt.data(), nbr.data());
  if (st) return st;
  NbrView nl{cnt.data(), nbr.data(), cap};
  compute_real(n, x, types, box, ns, table, nl, nthreads, &E, F.data(), W, nullptr);
  const double ftm2v = 1.0 / MVV2EV;
  for (int s = 0; s < nsteps; ++s) {
    for (int i = 0; i < n; ++i) {
      double a = 0.5 * dt * ftm2v / mass[types[i]];
      for (int c = 0; c < 3; ++c) {
        v[3 * i + c] += a * F[3 * i + c];
        x[3 * i + c] += dt * v[3 * i + c];
      }
    }
    if (rebuild_every > 0 && (s + 1) % rebuild_every == 0) {
      st = neighbors_cells(n, x, box, rlist, cap, cnt.data(), nbr.data());
      if (st) return st;
    }
    compute_real(n, x, types, box, ns, table, nl, nthreads, &E, F.data(), W, nullptr);
    double ke = 0.0;
    for (int i = 0; i < n; ++i) {
      double a = 0.5 * dt * ftm2v / mass[types[i]];
      double m = mass[types[i]];
      for (int c = 0; c < 3; ++c) {
        v[3 * i + c] += a * F[3 * i + c];
        ke += 0.5 * m * v[3 * i + c] * v[3 * i + c];
      }
    }
    ke *= MVV2EV;
    if (thermo) {
      thermo[3 * s + 0] = E;
      thermo[3 * s + 1] = ke;
      thermo[3 * s + 2] = E + ke;
    }
  }
  if (forces_out) std::memcpy(forces_out, F.data(), sizeof(double) * 3 * (size_t)n);
  return 0;
}

}  // extern "C"

// Adjoint of the Tersoff energy and forces with respect to the parameter table
// (the derivative of Sec. III Eq. 5-7 in the table entries; the paper itself
// has no backward pass).
//
// For weights gE (energy) and gF (one 3-vector per atom) the kernel adds
//   d/dtheta [ gE E + sum_a gF_a . F_a ]
// to grad (n_species^3 records of TERSOFF_NPARAM doubles, table layout).
//
// With F_a = -dE/dx_a and E = sum_i E_i (E_i: the terms centred on atom i,
// which depend on the bond vectors d_ij = x_j - x_i only), the force term is
//   sum_a gF_a . F_a = - sum_i D_w E_i,   D_w E_i = sum_j dE_i/dd_ij . w_ij,
// with w_ij = gF_j - gF_i: minus the derivative of E_i along the bond
// perturbations w. Per centre atom the kernel evaluates
//   L_i = gE E_i - D_w E_i
// forward (each quantity together with its derivative along w: r_j and its
// rate rd_j = u_j . w_j, cos(theta_jk) and its rate, zeta_ij and its rate) and
// differentiates L_i with respect to the parameters in reverse, in the loop
// order of Algorithm 2: a first K loop forms zeta_ij and its rate, the pair
// level gives the adjoints of zeta and its rate, and a second K loop
// recomputes every three-body term and adds the adjoints of its parameters.
// Nothing per triplet is stored.
//
// Record roles as in the forward evaluation: record (ti,tj,tj) supplies the
// pair terms of bond i-j (A, lambda1, B, lambda2, beta, n and the R, D of
// f_C(r_ij)); record (ti,tj,tk) supplies the three-body terms (gamma, c, d, h,
// lambda3, m and the R, D of f_C(r_ik)). m is an integer and gets no gradient.
//
// Per-term arithmetic in T (float on the mixed path, double on the FP64
// path); every gradient sum is accumulated in double.
#include <cstring>

#include "tersoff_fwd.cuh"

namespace tgb {
namespace bwd {

using fwd::Bond;
using fwd::SelfPos;
using fwd::self_pos;
using fwd::to_f64;

constexpr int NP = TERSOFF_NPARAM;

template <class T> struct BwdArgs {
  fwd::FwdArgs<T> g;      // geometry: packed positions, skin list, filter radii
  const T* raw;           // ns^3 raw records (table layout)
  const double* gE;       // energy weight(s): gE[cell(i)]
  const int* atom_cell;   // optional: cell of each atom (NULL: one cell)
  const T* gF;            // optional: N x 3 force weights, in T
  double* grad;           // ns^3 x NP, accumulated
  const int* order;       // atoms by bucket (bonds inside the cutoffs: <= 4, <= 8, more) ...
  const int* counts;      // ... and the three bucket sizes (device, FLAG_STRIDE apart)
  const int* fine;        // optional: all atoms ordered by their count of bonds inside the
                          // cutoffs (at the build), which then replaces the bucket order
};

// ------------------------------------------------------------------ math
template <class T> struct BM;
template <> struct BM<float> {
  static __device__ __forceinline__ float ex(float x) { return expf(x); }
  static __device__ __forceinline__ float ln(float x) { return logf(x); }
  static __device__ __forceinline__ float ln1p(float x) { return log1pf(x); }
  static __device__ __forceinline__ float pw(float x, float y) { return powf(x, y); }
  static __device__ __forceinline__ void scpi(float x, float* s, float* c) {
    sincospif(x, s, c);
  }
  static __device__ __forceinline__ float sq(float x) { return sqrtf(x); }
  // reciprocal: hardware approximation and one Newton step (~1 ulp)
  static __device__ __forceinline__ float rcp(float x) { return fwd::M<float>::rcp_nr(x); }
};
template <> struct BM<double> {
  static __device__ __forceinline__ double ex(double x) { return exp(x); }
  static __device__ __forceinline__ double ln(double x) { return log(x); }
  static __device__ __forceinline__ double ln1p(double x) { return log1p(x); }
  static __device__ __forceinline__ double pw(double x, double y) { return pow(x, y); }
  static __device__ __forceinline__ void scpi(double x, double* s, double* c) {
    sincospi(x, s, c);
  }
  static __device__ __forceinline__ double sq(double x) { return sqrt(x); }
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
};

// f_C(r; R, D), its r-derivative, and the R- and D-derivatives of both.
template <class T> struct Cut {
  T fc, dfc, fc_R, fc_D, dfc_R, dfc_D;
};
template <class T>
__device__ __forceinline__ Cut<T> cutoff_ad(T r, T R, T D) {
  Cut<T> o;
  if (r <= R - D) {
    o.fc = T(1);
    o.dfc = o.fc_R = o.fc_D = o.dfc_R = o.dfc_D = T(0);
    return o;
  }
  if (r >= R + D) {
    o.fc = o.dfc = o.fc_R = o.fc_D = o.dfc_R = o.dfc_D = T(0);
    return o;
  }
  // x = pi (r - R) / (2 D) = pi/2 - pi delta/(2D), delta = R + D - r: with
  // sh, ch = sin, cos(pi delta/(4D)), sin x = 1 - 2 sh^2 and cos x = 2 sh ch,
  // and f_C = 1/2 - 1/2 sin x = sh^2 without cancellation near R + D
  // (one reciprocal of D; products in place of the divisions)
  const T delta = (R + D) - r;
  const T iD = BM<T>::rcp(D);
  T sh, ch;
  BM<T>::scpi(delta * (T(0.25) * iD), &sh, &ch);
  const T s = T(1) - T(2) * sh * sh, c = T(2) * sh * ch;
  const T PI = T(3.14159265358979323846);
  const T x = PI * (r - R) * (T(0.5) * iD);
  const T k = PI * (T(0.25) * iD);  // pi / (4 D)
  o.fc = sh * sh;
  o.dfc = -k * c;
  o.fc_R = k * c;
  o.fc_D = T(0.5) * c * x * iD;
  o.dfc_R = -k * PI * (T(0.5) * iD) * s;
  o.dfc_D = k * iD * (c - x * s);
  return o;
}

// g(cos) = gamma (1 + c^2/d^2 - c^2/(d^2 + (h - cos)^2)), its cos-derivative,
// and the gamma, c, d, h derivatives of both. With t = h - cos and
// Den = d^2 + t^2 the forms below have no cancellation.
template <class T> struct Ang {
  T g, dg, g_ga, g_c, g_d, g_h, dg_ga, dg_c, dg_d, dg_h;
};
template <class T>
__device__ __forceinline__ Ang<T> angular_ad(T cs, T ga, T c, T d, T h) {
  Ang<T> o;
  // (reciprocals of d and Den; products in place of the divisions)
  const T t = h - cs;
  const T t2 = t * t;
  const T d2 = d * d;
  const T den = d2 + t2;
  const T iden = BM<T>::rcp(den);
  const T iden2 = iden * iden;
  const T id = BM<T>::rcp(d);
  const T id2 = id * id;
  const T c2 = c * c;
  const T r = t2 * id2 * iden;  // (1/d^2 - 1/Den)
  o.g_ga = T(1) + c2 * r;
  o.g = ga * o.g_ga;
  o.g_c = T(2) * ga * c * r;
  o.g_d = -T(2) * ga * c2 * t2 * (T(2) * d2 + t2) * (id2 * id) * iden2;
  o.dg = -T(2) * ga * c2 * t * iden2;
  o.g_h = -o.dg;
  o.dg_ga = -T(2) * c2 * t * iden2;
  o.dg_c = -T(4) * ga * c * t * iden2;
  o.dg_d = T(8) * ga * c2 * t * d * iden2 * iden;
  o.dg_h = -T(2) * ga * c2 * (den - T(4) * t2) * iden2 * iden;
  return o;
}

// X(Delta) = exp((lambda3 Delta)^m), dX/dDelta, and their lambda3-derivatives.
template <class T> struct Expo {
  T x, dx, x_l, dx_l;
};
template <class T>
__device__ __forceinline__ Expo<T> expo_ad(T delta, T l3, int m) {
  Expo<T> o;
  const T a = l3 * delta;
  T am1 = T(1);
  for (int s = 1; s < m; ++s) am1 *= a;
  const T am = am1 * a;
  o.x = am == T(0) ? T(1) : BM<T>::ex(am);  // lambda3 = 0 (most tables): no exponential
  o.dx = T(m) * l3 * am1 * o.x;
  o.x_l = T(m) * am1 * delta * o.x;
  o.dx_l = T(m) * T(m) * am1 * (T(1) + am) * o.x;
  return o;
}

// b(zeta) = (1 + (beta zeta)^n)^(-1/(2n)), b' = db/dzeta, b'' and the beta, n
// derivatives of b and b'. zeta = 0 gives b = 1 and zero derivatives.
template <class T> struct Bo {
  T b, db, ddb, b_be, b_n, db_be, db_n;
};
template <class T>
__device__ __forceinline__ Bo<T> bond_ad(T zeta, T be, T n) {
  Bo<T> o;
  if (!(zeta > T(0))) {
    o.b = T(1);
    o.db = o.ddb = o.b_be = o.b_n = o.db_be = o.db_n = T(0);
    return o;
  }
  // (reciprocals of 1 + u, zeta, n and beta; products in place of the divisions)
  const T L = BM<T>::ln(be * zeta);
  const T u = BM<T>::ex(n * L);
  const T w = u * BM<T>::rcp(T(1) + u);
  const T l1u = BM<T>::ln1p(u);
  const T iz = BM<T>::rcp(zeta);
  const T ih = T(0.5) * BM<T>::rcp(n);  // 1 / (2 n)
  const T ibe = BM<T>::rcp(be);
  o.b = BM<T>::ex(-l1u * ih);
  o.db = -T(0.5) * o.b * w * iz;
  o.ddb = -T(0.5) * (o.db * w + o.b * w * (n * (T(1) - w) - T(1)) * iz) * iz;
  o.b_be = -o.b * w * (T(0.5) * ibe);
  o.b_n = o.b * (l1u * (T(2) * ih * ih) - w * L * ih);
  const T w_be = n * w * (T(1) - w) * ibe;
  const T w_n = w * (T(1) - w) * L;
  o.db_be = -T(0.5) * (o.b_be * w + o.b * w_be) * iz;
  o.db_n = -T(0.5) * (o.b_n * w + o.b * w_n) * iz;
  return o;
}

// ------------------------------------------------------------------ accumulation
// Per-thread sums are kept in T (one atom's terms: a few dozen per field) and
// summed over the warp in T; the warp totals go to the block and global sums
// in double. On the mixed path this keeps the FP64 pipe out of the loops (a
// depth-5 float tree adds ~3e-7 relative error to a warp's total).
// NS == 1: one record. NS == 2 (mixed path): the 4 records (ti, *, *) of the
// thread's centre species, summed once per centre species. Otherwise:
// per-block shared accumulators with shared-memory atomics.
// the fields a three-body term adds to, in the order of Acc::add_triplet
__host__ __device__ constexpr int triplet_field(int k) {
  return k == 0   ? TERSOFF_P_R
         : k == 1 ? TERSOFF_P_D_CUT
         : k == 2 ? TERSOFF_P_GAMMA
         : k == 3 ? TERSOFF_P_C
         : k == 4 ? TERSOFF_P_D
         : k == 5 ? TERSOFF_P_H
                  : TERSOFF_P_LAMBDA3;
}

template <int NS, class T> struct Acc;
template <class T> struct Acc<1, T> {
  T v[NP];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int q = 0; q < NP; ++q) v[q] = T(0);
  }
  __device__ __forceinline__ void add(double*, int, int f, T x) { v[f] += x; }
  __device__ __forceinline__ void add_pair(double*, int, int, int f, T x) { v[f] += x; }
  __device__ __forceinline__ void add_triplet(double*, int, const T (&x)[7]) {
#pragma unroll
    for (int k = 0; k < 7; ++k) v[triplet_field(k)] += x[k];
  }
  __device__ __forceinline__ void flush(double* sh, int) {
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      T s = v[q];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if ((threadIdx.x & 31) == 0 && s != T(0)) atomicAdd(&sh[q], to_f64(s));
    }
  }
};
template <class T> struct Acc<2, T> {
  T v[4][NP];  // record (ti, tj, tk) at [2 tj + tk]; indices constant after unrolling
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < NP; ++q) v[r][q] = T(0);
  }
  __device__ __forceinline__ void add(double*, int rec, int f, T x) {
    const int r = rec & 3;  // rec = 4 ti + 2 tj + tk
    if (r == 0) v[0][f] += x;
    else if (r == 1) v[1][f] += x;
    else if (r == 2) v[2][f] += x;
    else v[3][f] += x;
  }
  // one three-body term's seven fields: one choice of the record position
  // for all of them
  __device__ __forceinline__ void add_triplet(double*, int rec, const T (&x)[7]) {
    const int r = rec & 3;
    if (r == 0) {
#pragma unroll
      for (int k = 0; k < 7; ++k) v[0][triplet_field(k)] += x[k];
    } else if (r == 1) {
#pragma unroll
      for (int k = 0; k < 7; ++k) v[1][triplet_field(k)] += x[k];
    } else if (r == 2) {
#pragma unroll
      for (int k = 0; k < 7; ++k) v[2][triplet_field(k)] += x[k];
    } else {
#pragma unroll
      for (int k = 0; k < 7; ++k) v[3][triplet_field(k)] += x[k];
    }
  }
  // pair terms: record (ti, tj, tj), at [3 tj]; the mixed records (1 and 2)
  // never receive a pair field, so their pair-only sums are never live
  __device__ __forceinline__ void add_pair(double*, int, int tj, int f, T x) {
    if (tj == 0) v[0][f] += x;
    else v[3][f] += x;
  }
  // fields a record position can receive: m never; A, lambda1, B, lambda2,
  // beta and n only at the pair records 0 and 3
  static __device__ __forceinline__ constexpr bool used(int r, int f) {
    return f != TERSOFF_P_M &&
           (r == 0 || r == 3 || f == TERSOFF_P_GAMMA || f == TERSOFF_P_LAMBDA3 ||
            f == TERSOFF_P_C || f == TERSOFF_P_D || f == TERSOFF_P_H || f == TERSOFF_P_R ||
            f == TERSOFF_P_D_CUT);
  }
  // all lanes; lanes without an atom hold zeros (ti 0)
  __device__ __forceinline__ void flush(double* sh, int ti) {
#pragma unroll
    for (int tt = 0; tt < 2; ++tt)
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          if (!used(r, q)) continue;
          T s = ti == tt ? v[r][q] : T(0);
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          if ((threadIdx.x & 31) == 0 && s != T(0))
            atomicAdd(&sh[(4 * tt + r) * NP + q], to_f64(s));
        }
  }
};
template <class T> struct Acc<0, T> {
  __device__ __forceinline__ void init() {}
  __device__ __forceinline__ void add(double* sh, int rec, int f, T x) {
    const double d = to_f64(x);
    if (d != 0.0) atomicAdd(&sh[rec * NP + f], d);
  }
  __device__ __forceinline__ void add_pair(double* sh, int rec, int, int f, T x) {
    add(sh, rec, f, x);
  }
  __device__ __forceinline__ void add_triplet(double* sh, int rec, const T (&x)[7]) {
#pragma unroll
    for (int k = 0; k < 7; ++k) add(sh, rec, triplet_field(k), x[k]);
  }
  __device__ __forceinline__ void flush(double*, int) {}
};

template <class T>
__device__ __forceinline__ T rec_val(const T* raw, int rec, int f) {
  return raw[rec * NP + f];
}

// ------------------------------------------------------------------ bonds
// One neighbour k of the centre atom: unit vector u, length r, the rate of r
// along w (rd = u . w), p = (w - u rd) / r (the rate of cos(theta_jk) is
// p_j . u_k + p_k . u_j) and the species.
template <class T> struct BondD {
  T ux, uy, uz, r, rd, px, py, pz;
  int t;
};

// Bonds inside the filter radius are cached per thread in dynamic shared
// memory, slot-major with the thread index innermost (no bank conflicts):
// slots of 9 words (12 slots in float, 8 in double). Atoms with more bonds
// inside recompute them from the skin list in every loop.
constexpr int SLOT_WORDS = 9;
template <class T> struct BwdBlock;
template <> struct BwdBlock<float> {
  static constexpr int size = 128;
  static constexpr int slots = 12;
};
template <> struct BwdBlock<double> {
  static constexpr int size = 64;
  static constexpr int slots = 8;
};
template <class T>
constexpr size_t slot_bytes() {
  return (size_t)BwdBlock<T>::size * BwdBlock<T>::slots * SLOT_WORDS * sizeof(T);
}

template <class T>
__device__ __forceinline__ void put_slot(T* sh, int q, const BondD<T>& b) {
  const int B = blockDim.x;
  T* p = sh + (size_t)q * SLOT_WORDS * B + threadIdx.x;
  p[0] = b.ux;
  p[B] = b.uy;
  p[2 * B] = b.uz;
  p[3 * B] = b.r;
  p[4 * B] = b.rd;
  p[5 * B] = b.px;
  p[6 * B] = b.py;
  p[7 * B] = b.pz;
  p[8 * B] = T(b.t);
}
template <class T>
__device__ __forceinline__ void get_slot(const T* sh, int q, BondD<T>& b) {
  const int B = blockDim.x;
  const T* p = sh + (size_t)q * SLOT_WORDS * B + threadIdx.x;
  b.ux = p[0];
  b.uy = p[B];
  b.uz = p[2 * B];
  b.r = p[3 * B];
  b.rd = p[4 * B];
  b.px = p[5 * B];
  b.py = p[6 * B];
  b.pz = p[7 * B];
  b.t = (int)p[8 * B];
}

// The adjoint of L_i over the neighbourhood given by get(q, bond) for
// q < count (get returns false for a bond outside the filter radius), in
// Algorithm 2's loop order.
template <class T, int NS, class AccT, class Get>
__device__ __forceinline__ void atom_adjoint(const T* sraw, int ns, int ti, T hE, int count,
                                             Get get, AccT& acc, double* sgrad) {
  for (int qj = 0; qj < count; ++qj) {
    BondD<T> bj;
    if (!get(qj, bj)) continue;
    const int tj = bj.t;
    const int p = NS == 1 ? 0 : (ti * ns + tj) * ns + tj;
    const T Rp = rec_val(sraw, p, TERSOFF_P_R), Dp = rec_val(sraw, p, TERSOFF_P_D_CUT);
    const T rj = bj.r, rdj = bj.rd;
    if (!(rj < Rp + Dp)) continue;
    // first K loop: zeta_ij and its rate along w
    T zeta = T(0), zd = T(0);
    for (int qk = 0; qk < count; ++qk) {
      if (qk == qj) continue;
      BondD<T> bk;
      if (!get(qk, bk)) continue;
      const int q = NS == 1 ? 0 : (ti * ns + tj) * ns + bk.t;
      const T Rq = rec_val(sraw, q, TERSOFF_P_R), Dq = rec_val(sraw, q, TERSOFF_P_D_CUT);
      const T rk = bk.r, rdk = bk.rd;
      if (!(rk < Rq + Dq)) continue;
      const T cs = bj.ux * bk.ux + bj.uy * bk.uy + bj.uz * bk.uz;
      const T csd = (bj.px * bk.ux + bj.py * bk.uy + bj.pz * bk.uz) +
                    (bk.px * bj.ux + bk.py * bj.uy + bk.pz * bj.uz);
      const Cut<T> fk = cutoff_ad<T>(rk, Rq, Dq);
      const Ang<T> an = angular_ad<T>(cs, rec_val(sraw, q, TERSOFF_P_GAMMA),
                                      rec_val(sraw, q, TERSOFF_P_C),
                                      rec_val(sraw, q, TERSOFF_P_D),
                                      rec_val(sraw, q, TERSOFF_P_H));
      const Expo<T> ex = expo_ad<T>(rj - rk, rec_val(sraw, q, TERSOFF_P_LAMBDA3),
                                    (int)rec_val(sraw, q, TERSOFF_P_M));
      zeta += fk.fc * an.g * ex.x;
      zd += fk.dfc * rdk * an.g * ex.x + fk.fc * an.dg * csd * ex.x +
            fk.fc * an.g * ex.dx * (rdj - rdk);
    }
    // pair level
    const Cut<T> fj = cutoff_ad<T>(rj, Rp, Dp);
    const T A = rec_val(sraw, p, TERSOFF_P_A), l1 = rec_val(sraw, p, TERSOFF_P_LAMBDA1);
    const T B = rec_val(sraw, p, TERSOFF_P_B), l2 = rec_val(sraw, p, TERSOFF_P_LAMBDA2);
    const T e1 = BM<T>::ex(-l1 * rj), e2 = BM<T>::ex(-l2 * rj);
    const T Ae1 = A * e1, Be2 = B * e2;
    const T Pv = fj.fc * Ae1;
    const T Pd = (fj.dfc - l1 * fj.fc) * Ae1;
    const T Qv = -fj.fc * Be2;
    const T Qd = -(fj.dfc - l2 * fj.fc) * Be2;
    const Bo<T> bo = bond_ad<T>(zeta, rec_val(sraw, p, TERSOFF_P_BETA),
                                rec_val(sraw, p, TERSOFF_P_N));
    // L_j = gE/2 (P + b Q) - 1/2 (P' + b Q') rd_j - 1/2 Q b' zeta_rate
    const T Pbar = hE;
    const T Pdbar = -T(0.5) * rdj;
    const T Qbar = hE * bo.b - T(0.5) * bo.db * zd;
    const T Qdbar = -T(0.5) * bo.b * rdj;
    const T bbar = hE * Qv - T(0.5) * Qd * rdj;
    const T dbbar = -T(0.5) * Qv * zd;
    acc.add_pair(sgrad, p, tj, TERSOFF_P_A, (Pbar * fj.fc * e1 + Pdbar * (fj.dfc - l1 * fj.fc) * e1));
    acc.add_pair(sgrad, p, tj, TERSOFF_P_LAMBDA1, (Pbar * (-rj * Pv) + Pdbar * (-fj.fc * Ae1 - rj * Pd)));
    acc.add_pair(sgrad, p, tj, TERSOFF_P_B, (Qbar * (-fj.fc * e2) + Qdbar * (-(fj.dfc - l2 * fj.fc) * e2)));
    acc.add_pair(sgrad, p, tj, TERSOFF_P_LAMBDA2, (Qbar * (-rj * Qv) + Qdbar * (fj.fc * Be2 - rj * Qd)));
    acc.add_pair(sgrad, p, tj, TERSOFF_P_R, ((Pbar * fj.fc_R + Pdbar * (fj.dfc_R - l1 * fj.fc_R)) * Ae1 -
                   (Qbar * fj.fc_R + Qdbar * (fj.dfc_R - l2 * fj.fc_R)) * Be2));
    acc.add_pair(sgrad, p, tj, TERSOFF_P_D_CUT, ((Pbar * fj.fc_D + Pdbar * (fj.dfc_D - l1 * fj.fc_D)) * Ae1 -
                   (Qbar * fj.fc_D + Qdbar * (fj.dfc_D - l2 * fj.fc_D)) * Be2));
    acc.add_pair(sgrad, p, tj, TERSOFF_P_BETA, (bbar * bo.b_be + dbbar * bo.db_be));
    acc.add_pair(sgrad, p, tj, TERSOFF_P_N, (bbar * bo.b_n + dbbar * bo.db_n));
    const T zbar = bbar * bo.db + dbbar * bo.ddb;
    const T zdbar = -T(0.5) * Qv * bo.db;
    if (zbar == T(0) && zdbar == T(0)) continue;
    // second K loop: recompute each three-body term, adjoints of its parameters
    for (int qk = 0; qk < count; ++qk) {
      if (qk == qj) continue;
      BondD<T> bk;
      if (!get(qk, bk)) continue;
      const int q = NS == 1 ? 0 : (ti * ns + tj) * ns + bk.t;
      const T Rq = rec_val(sraw, q, TERSOFF_P_R), Dq = rec_val(sraw, q, TERSOFF_P_D_CUT);
      const T rk = bk.r, rdk = bk.rd;
      if (!(rk < Rq + Dq)) continue;
      const T cs = bj.ux * bk.ux + bj.uy * bk.uy + bj.uz * bk.uz;
      const T csd = (bj.px * bk.ux + bj.py * bk.uy + bj.pz * bk.uz) +
                    (bk.px * bj.ux + bk.py * bj.uy + bk.pz * bj.uz);
      const Cut<T> fk = cutoff_ad<T>(rk, Rq, Dq);
      const Ang<T> an = angular_ad<T>(cs, rec_val(sraw, q, TERSOFF_P_GAMMA),
                                      rec_val(sraw, q, TERSOFF_P_C),
                                      rec_val(sraw, q, TERSOFF_P_D),
                                      rec_val(sraw, q, TERSOFF_P_H));
      const T dl = rj - rk, dld = rdj - rdk;
      const Expo<T> ex = expo_ad<T>(dl, rec_val(sraw, q, TERSOFF_P_LAMBDA3),
                                    (int)rec_val(sraw, q, TERSOFF_P_M));
      // T = F3 G X ; T_rate = F3' rd_k G X + F3 G' cs_rate X + F3 G X' dl_rate
      const T F3bar = zbar * an.g * ex.x + zdbar * (an.dg * csd * ex.x + an.g * ex.dx * dld);
      const T F3dbar = zdbar * rdk * an.g * ex.x;
      const T Gbar = zbar * fk.fc * ex.x + zdbar * (fk.dfc * rdk * ex.x + fk.fc * ex.dx * dld);
      const T Gdbar = zdbar * fk.fc * csd * ex.x;
      const T Xbar = zbar * fk.fc * an.g + zdbar * (fk.dfc * rdk * an.g + fk.fc * an.dg * csd);
      const T Xdbar = zdbar * fk.fc * an.g * dld;
      const T tb[7] = {F3bar * fk.fc_R + F3dbar * fk.dfc_R,  // R
                       F3bar * fk.fc_D + F3dbar * fk.dfc_D,  // D
                       Gbar * an.g_ga + Gdbar * an.dg_ga,    // gamma
                       Gbar * an.g_c + Gdbar * an.dg_c,      // c
                       Gbar * an.g_d + Gdbar * an.dg_d,      // d
                       Gbar * an.g_h + Gdbar * an.dg_h,      // h
                       Xbar * ex.x_l + Xdbar * ex.dx_l};     // lambda3
      acc.add_triplet(sgrad, q, tb);
    }
  }
}

// ------------------------------------------------------------------ the kernel
template <class T, int NS, bool BATCH>
__global__ void __launch_bounds__(BwdBlock<T>::size) k_tersoff_bwd(const __grid_constant__ BwdArgs<T> a) {
  constexpr int SNS = NS > 0 ? NS : TERSOFF_MAX_SPECIES;
  __shared__ T sraw[SNS * SNS * SNS * NP];
  __shared__ T sfilt[SNS * SNS];
  __shared__ double sgrad[SNS * SNS * SNS * NP];
  extern __shared__ __align__(16) unsigned char bwd_dyn[];
  T* slots = reinterpret_cast<T*>(bwd_dyn);
  const fwd::FwdArgs<T>& g = a.g;
  const int ns = NS > 0 ? NS : g.ns;
  const int nrec = ns * ns * ns;
  for (int q = threadIdx.x; q < nrec * NP; q += blockDim.x) {
    sraw[q] = a.raw[q];
    sgrad[q] = 0.0;
  }
  if (threadIdx.x < ns * ns) sfilt[threadIdx.x] = g.filt2[threadIdx.x];
  __syncthreads();

  // atoms in bucket order: neighbouring lanes have similar neighbourhood sizes
  __shared__ int nb[3];
  if (threadIdx.x < 3) nb[threadIdx.x] = a.counts[threadIdx.x * FLAG_STRIDE];
  __syncthreads();
  Acc<NS, T> acc;
  acc.init();
  int ti = 0;
  const int item = blockIdx.x * blockDim.x + threadIdx.x;
  const int n01 = nb[0] + nb[1];
  const int i = item >= g.n   ? g.n
                : a.fine      ? a.fine[item]
                : item < nb[0] ? a.order[item]
                : item < n01   ? a.order[(size_t)g.n + item - nb[0]]
                               : a.order[2 * (size_t)g.n + item - n01];
  if (i < g.n) {
    using P = typename SelfPos<T>::type;
    const P pi = self_pos<T>(g, i);
    fwd::Shift<T, BATCH> sh;
    sh.load(g, i);
    ti = g.types[i];
    const int c = min(g.cnt[i], g.cap);
    const double gE = a.gE[a.atom_cell ? a.atom_cell[i] : 0];
    const bool hasF = a.gF != nullptr;
    T gfi0 = T(0), gfi1 = T(0), gfi2 = T(0);
    if (hasF) {
      gfi0 = a.gF[3 * (size_t)i];
      gfi1 = a.gF[3 * (size_t)i + 1];
      gfi2 = a.gF[3 * (size_t)i + 2];
    }
    const T hE = T(0.5) * T(gE);
    // skin-list entry s: bond data; false when outside the filter radius
    auto from_list = [&](int s, BondD<T>& b) -> bool {
      T dx, dy, dz;
      int j;
      Bond<T>::vec(g, sh, pi, g.nbr[(size_t)s * g.n + i], dx, dy, dz, j, b.t);
      const T r2 = dx * dx + dy * dy + dz * dz;
      if (!(r2 <= sfilt[ti * ns + b.t])) return false;
      b.r = BM<T>::sq(r2);
      const T ir = T(1) / b.r;
      b.ux = dx * ir;
      b.uy = dy * ir;
      b.uz = dz * ir;
      T wx = T(0), wy = T(0), wz = T(0);
      if (hasF) {
        wx = a.gF[3 * (size_t)j] - gfi0;
        wy = a.gF[3 * (size_t)j + 1] - gfi1;
        wz = a.gF[3 * (size_t)j + 2] - gfi2;
      }
      b.rd = b.ux * wx + b.uy * wy + b.uz * wz;
      b.px = (wx - b.ux * b.rd) * ir;
      b.py = (wy - b.uy * b.rd) * ir;
      b.pz = (wz - b.uz * b.rd) * ir;
      return true;
    };
    // cache the bonds inside the filter radius when they fit; mark them in a
    // bit mask over the list (its first 64 entries)
    constexpr int ZB = BwdBlock<T>::slots;
    int z = 0;
    unsigned long long kept = 0ull;
    for (int s = 0; s < c; ++s) {
      BondD<T> b;
      if (!from_list(s, b)) continue;
      if (z < ZB) put_slot<T>(slots, z, b);
      if (s < 64) kept |= 1ull << s;
      ++z;
    }
    if (z <= ZB) {
      atom_adjoint<T, NS>(sraw, ns, ti, hE, z,
                          [&](int q, BondD<T>& b) -> bool {
                            get_slot<T>(slots, q, b);
                            return true;
                          },
                          acc, sgrad);
    } else if (c <= 64) {
      // more bonds than slots: the q-th marked entry, formed again from the list
      const unsigned lo = (unsigned)kept, hi = (unsigned)(kept >> 32);
      const int nlo = __popc(lo);
      atom_adjoint<T, NS>(sraw, ns, ti, hE, z,
                          [&](int q, BondD<T>& b) -> bool {
                            const int s = q < nlo ? (int)__fns(lo, 0, q + 1)
                                                  : 32 + (int)__fns(hi, 0, q - nlo + 1);
                            return from_list(s, b);
                          },
                          acc, sgrad);
    } else {
      atom_adjoint<T, NS>(sraw, ns, ti, hE, c, from_list, acc, sgrad);
    }
  }
  acc.flush(sgrad, ti);
  __syncthreads();
  for (int q = threadIdx.x; q < nrec * NP; q += blockDim.x)
    if (sgrad[q] != 0.0) atomicAdd(&a.grad[q], sgrad[q]);
}

// ------------------------------------------------------------------ Hessian-vector product
// The position derivative of the force term: d/dx [sum_a gF_a . F_a] =
// -sum_i d/dx D_w E_i, D_w E_i the derivative of E_i along the bond
// perturbations w_ij = gF_j - gF_i (as in the parameter adjoint). Per centre
// atom, D_w E_i = sum_j [V_r(r_j, zeta_j) rd_j + V_zeta(r_j, zeta_j) zeta_rate_j]
// is differentiated in reverse with respect to the bond geometry (lengths r,
// unit vectors u, rates rd = u.w, and p = (w - u rd)/r, through which
// cos(theta_jk) = u_j.u_k and its rate p_j.u_k + p_k.u_j depend on the bond
// vectors), which needs the second derivatives of f_C, g, the exponential and
// the pair functions; the bond-vector adjoints are scattered to the atoms.

template <class T> struct D2 {
  T f, d1, d2;
};
// f_C(r) and its first two r-derivatives
template <class T>
__device__ __forceinline__ D2<T> cutoff2(T r, T R, T D) {
  D2<T> o;
  if (r <= R - D) {
    o.f = T(1);
    o.d1 = o.d2 = T(0);
    return o;
  }
  if (r >= R + D) {
    o.f = o.d1 = o.d2 = T(0);
    return o;
  }
  // in delta = R + D - r, as in cutoff_ad: sin x = 1 - 2 sh^2, cos x = 2 sh ch
  T sh, ch;
  BM<T>::scpi(((R + D) - r) / (T(4) * D), &sh, &ch);
  const T sn = T(1) - T(2) * sh * sh, cn = T(2) * sh * ch;
  const T PI = T(3.14159265358979323846);
  const T k = PI / (T(4) * D);
  o.f = sh * sh;
  o.d1 = -k * cn;
  o.d2 = k * PI / (T(2) * D) * sn;
  return o;
}
// g(cos) and its first two cos-derivatives (t = h - cos, Den = d^2 + t^2)
template <class T>
__device__ __forceinline__ D2<T> angular2(T cs, T ga, T c, T d, T h) {
  const T t = h - cs, t2 = t * t, d2 = d * d, den = d2 + t2, iden = T(1) / den, c2 = c * c;
  D2<T> o;
  o.f = ga + ga * c2 * t2 / (d2 * den);
  o.d1 = -T(2) * ga * c2 * t * iden * iden;
  o.d2 = T(2) * ga * c2 * (den - T(4) * t2) * iden * iden * iden;
  return o;
}
// X(Delta) = exp((lambda3 Delta)^m) and its first two Delta-derivatives
template <class T>
__device__ __forceinline__ D2<T> expo2(T delta, T l3, int m) {
  const T a = l3 * delta;
  T am2 = T(1);  // a^(m-2), used for m >= 2
  for (int s = 2; s < m; ++s) am2 *= a;
  const T am1 = m >= 2 ? am2 * a : T(1);
  D2<T> o;
  o.f = BM<T>::ex(am1 * a);
  o.d1 = T(m) * l3 * am1 * o.f;
  o.d2 = (m >= 2 ? T(m) * T(m - 1) * l3 * l3 * am2 * o.f : T(0)) + T(m) * l3 * am1 * o.d1;
  return o;
}

// Adjoints of one bond's (r, u, rd, p).
template <class T> struct BondBar {
  T r, ux, uy, uz, rd, px, py, pz;
};
template <class T>
__device__ __forceinline__ BondBar<T> zero_bar() {
  BondBar<T> o;
  o.r = o.ux = o.uy = o.uz = o.rd = o.px = o.py = o.pz = T(0);
  return o;
}

// The adjoint of the bond vector d from those of (r, u, rd, p), with
// r = |d|, u = d / r, rd = u . w, p = (w - u rd) / r (w held fixed).
template <class T>
__device__ __forceinline__ void bond_vec_bar(const BondD<T>& b, BondBar<T> q, T& dx, T& dy, T& dz) {
  const T ir = T(1) / b.r;
  q.ux -= b.rd * ir * q.px;
  q.uy -= b.rd * ir * q.py;
  q.uz -= b.rd * ir * q.pz;
  q.rd -= (b.ux * q.px + b.uy * q.py + b.uz * q.pz) * ir;
  q.r -= (b.px * q.px + b.py * q.py + b.pz * q.pz) * ir;
  // w = p r + u rd
  q.ux += q.rd * (b.px * b.r + b.ux * b.rd);
  q.uy += q.rd * (b.py * b.r + b.uy * b.rd);
  q.uz += q.rd * (b.pz * b.r + b.uz * b.rd);
  const T uu = q.ux * b.ux + q.uy * b.uy + q.uz * b.uz;
  dx = (q.ux - uu * b.ux) * ir + q.r * b.ux;
  dy = (q.uy - uu * b.uy) * ir + q.r * b.uy;
  dz = (q.uz - uu * b.uz) * ir + q.r * b.uz;
}

// The three-body factor of one (j, k) pair and what the Hessian-vector pass
// needs of it: T = F3(r_k) G(cos) X(r_j - r_k) with first and second
// derivatives. Tables with lambda3 = 0 everywhere (LAM3 false) have X = 1.
template <class T, bool LAM3> struct Tri {
  D2<T> F3, G, X;
  __device__ __forceinline__ Tri(const T* sraw, int q, T rj, T rk, T cs) {
    F3 = cutoff2<T>(rk, rec_val(sraw, q, TERSOFF_P_R), rec_val(sraw, q, TERSOFF_P_D_CUT));
    G = angular2<T>(cs, rec_val(sraw, q, TERSOFF_P_GAMMA), rec_val(sraw, q, TERSOFF_P_C),
                    rec_val(sraw, q, TERSOFF_P_D), rec_val(sraw, q, TERSOFF_P_H));
    if constexpr (LAM3)
      X = expo2<T>(rj - rk, rec_val(sraw, q, TERSOFF_P_LAMBDA3), (int)rec_val(sraw, q, TERSOFF_P_M));
  }
};

// Reverse-mode derivative of D_w E_i with respect to the geometry of the
// centre atom's bonds, in Algorithm 2's loop order: per bond j a first K loop
// forms zeta_ij and its rate, the pair level seeds the adjoints, and a second
// K loop adds the adjoints of every three-body term's inputs. get(q, bond, j)
// returns bond q (false outside the filter radius); sink(q, bond, j, bar)
// receives additive adjoint contributions for bond q.
template <class T, bool LAM3, class Get, class Sink>
__device__ __forceinline__ void atom_hvp(const T* sraw, int ns, int ti, int count, Get get, Sink sink) {
  for (int qj = 0; qj < count; ++qj) {
    BondD<T> bj;
    int jj;
    if (!get(qj, bj, jj)) continue;
    const int tj = bj.t;
    const int p = (ti * ns + tj) * ns + tj;
    const T Rp = rec_val(sraw, p, TERSOFF_P_R), Dp = rec_val(sraw, p, TERSOFF_P_D_CUT);
    const T rj = bj.r, rdj = bj.rd;
    if (!(rj < Rp + Dp)) continue;
    // first K loop: zeta_ij and its rate
    T zeta = T(0), zd = T(0);
    for (int qk = 0; qk < count; ++qk) {
      if (qk == qj) continue;
      BondD<T> bk;
      int jk;
      if (!get(qk, bk, jk)) continue;
      const int q = (ti * ns + tj) * ns + bk.t;
      if (!(bk.r < rec_val(sraw, q, TERSOFF_P_R) + rec_val(sraw, q, TERSOFF_P_D_CUT))) continue;
      const T cs = bj.ux * bk.ux + bj.uy * bk.uy + bj.uz * bk.uz;
      const T csd = (bj.px * bk.ux + bj.py * bk.uy + bj.pz * bk.uz) +
                    (bk.px * bj.ux + bk.py * bj.uy + bk.pz * bj.uz);
      const Tri<T, LAM3> tr(sraw, q, rj, bk.r, cs);
      const T FG = tr.F3.f * tr.G.f;
      const T FGd = tr.F3.d1 * bk.rd * tr.G.f + tr.F3.f * tr.G.d1 * csd;
      if constexpr (LAM3) {
        zeta += FG * tr.X.f;
        zd += FGd * tr.X.f + FG * tr.X.d1 * (rdj - bk.rd);
      } else {
        zeta += FG;
        zd += FGd;
      }
    }
    // pair level: Phi_j = 1/2 (P' + b Q') rd_j + 1/2 Q b' zeta_rate
    const D2<T> fc = cutoff2<T>(rj, Rp, Dp);
    const T A = rec_val(sraw, p, TERSOFF_P_A), l1 = rec_val(sraw, p, TERSOFF_P_LAMBDA1);
    const T B = rec_val(sraw, p, TERSOFF_P_B), l2 = rec_val(sraw, p, TERSOFF_P_LAMBDA2);
    const T Ae = A * BM<T>::ex(-l1 * rj), Be = B * BM<T>::ex(-l2 * rj);
    const T P1 = (fc.d1 - l1 * fc.f) * Ae;
    const T P2 = (fc.d2 - T(2) * l1 * fc.d1 + l1 * l1 * fc.f) * Ae;
    const T Q0 = -fc.f * Be;
    const T Q1 = -(fc.d1 - l2 * fc.f) * Be;
    const T Q2 = -(fc.d2 - T(2) * l2 * fc.d1 + l2 * l2 * fc.f) * Be;
    const Bo<T> bo = bond_ad<T>(zeta, rec_val(sraw, p, TERSOFF_P_BETA), rec_val(sraw, p, TERSOFF_P_N));
    BondBar<T> aj = zero_bar<T>();
    aj.rd = T(0.5) * (P1 + bo.b * Q1);
    aj.r = T(0.5) * (P2 + bo.b * Q2) * rdj + T(0.5) * Q1 * bo.db * zd;
    const T zb = T(0.5) * Q1 * bo.db * rdj + T(0.5) * Q0 * bo.ddb * zd;  // d Phi_j / d zeta
    const T zdb = T(0.5) * Q0 * bo.db;                                   // d Phi_j / d zeta_rate
    if (zb != T(0) || zdb != T(0)) {
      // second K loop: T = F3 G X, T_rate = F3' rd_k G X + F3 G' cs_rate X + F3 G X' (rd_j - rd_k)
      for (int qk = 0; qk < count; ++qk) {
        if (qk == qj) continue;
        BondD<T> bk;
        int jk;
        if (!get(qk, bk, jk)) continue;
        const int q = (ti * ns + tj) * ns + bk.t;
        const T rk = bk.r, rdk = bk.rd;
        if (!(rk < rec_val(sraw, q, TERSOFF_P_R) + rec_val(sraw, q, TERSOFF_P_D_CUT))) continue;
        const T cs = bj.ux * bk.ux + bj.uy * bk.uy + bj.uz * bk.uz;
        const T csd = (bj.px * bk.ux + bj.py * bk.uy + bj.pz * bk.uz) +
                      (bk.px * bj.ux + bk.py * bj.uy + bk.pz * bj.uz);
        const Tri<T, LAM3> tr(sraw, q, rj, rk, cs);
        const D2<T>&F3 = tr.F3, &G = tr.G;
        BondBar<T> ak;
        T cb, cdb;
        if constexpr (LAM3) {
          const D2<T>& X = tr.X;
          const T dl = rdj - rdk, FG = F3.f * G.f;
          ak.r = zb * (F3.d1 * G.f * X.f - FG * X.d1) +
                 zdb * (F3.d2 * rdk * G.f * X.f - F3.d1 * rdk * G.f * X.d1 + F3.d1 * G.d1 * csd * X.f -
                        F3.f * G.d1 * csd * X.d1 + F3.d1 * G.f * X.d1 * dl - FG * X.d2 * dl);
          ak.rd = zdb * (F3.d1 * G.f * X.f - FG * X.d1);
          aj.r += zb * FG * X.d1 + zdb * (F3.d1 * rdk * G.f * X.d1 + F3.f * G.d1 * csd * X.d1 + FG * X.d2 * dl);
          aj.rd += zdb * FG * X.d1;
          cb = zb * F3.f * G.d1 * X.f +
               zdb * (F3.d1 * rdk * G.d1 * X.f + F3.f * G.d2 * csd * X.f + F3.f * G.d1 * X.d1 * dl);
          cdb = zdb * F3.f * G.d1 * X.f;
        } else {
          ak.r = zb * F3.d1 * G.f + zdb * (F3.d2 * rdk * G.f + F3.d1 * G.d1 * csd);
          ak.rd = zdb * F3.d1 * G.f;
          cb = zb * F3.f * G.d1 + zdb * (F3.d1 * rdk * G.d1 + F3.f * G.d2 * csd);
          cdb = zdb * F3.f * G.d1;
        }
        // cos = u_j . u_k, cos_rate = p_j . u_k + p_k . u_j
        aj.ux += cb * bk.ux + cdb * bk.px;
        aj.uy += cb * bk.uy + cdb * bk.py;
        aj.uz += cb * bk.uz + cdb * bk.pz;
        aj.px += cdb * bk.ux;
        aj.py += cdb * bk.uy;
        aj.pz += cdb * bk.uz;
        ak.ux = cb * bj.ux + cdb * bj.px;
        ak.uy = cb * bj.uy + cdb * bj.py;
        ak.uz = cb * bj.uz + cdb * bj.pz;
        ak.px = cdb * bj.ux;
        ak.py = cdb * bj.uy;
        ak.pz = cdb * bj.uz;
        sink(qk, bk, jk, ak);
      }
    }
    sink(qj, bj, jj, aj);
  }
}

// Per-thread bond slots of the Hessian-vector kernel in dynamic shared memory,
// thread index innermost: the bond data (9 words, as in the parameter
// adjoint), its adjoint accumulators (8 words) and the neighbour index. Two
// shapes: 4 slots in blocks of 128 threads for atoms with at most 4 bonds
// inside the cutoffs at the list build (bucket 0), 12 slots in blocks of 64
// for the others. An atom with more bonds than slots inside the filter radius
// (it has moved since the build, or has more than 12) recomputes its bonds
// from the skin list and scatters each adjoint contribution as it is formed.
constexpr int HVP_BAR_WORDS = 8;
template <class T, int ZB, int BS>
constexpr size_t hvp_bytes() {
  return (size_t)BS * ZB * ((SLOT_WORDS + HVP_BAR_WORDS) * sizeof(T) + sizeof(int));
}

// Items: the atoms of buckets b0 .. b1 - 1 (bucket order), in a grid-stride
// loop (grids are sized from the host's bucket counts; the device counts
// decide).
template <class T, bool BATCH, bool LAM3, int ZB, int BS>
__global__ void __launch_bounds__(BS) k_tersoff_hvp(const __grid_constant__ BwdArgs<T> a,
                                                    double* __restrict__ gx, int b0, int b1) {
  constexpr int SNS = TERSOFF_MAX_SPECIES;
  __shared__ T sraw[SNS * SNS * SNS * NP];
  __shared__ T sfilt[SNS * SNS];
  __shared__ int nb[3];
  extern __shared__ __align__(16) unsigned char hvp_dyn[];
  T* geo = reinterpret_cast<T*>(hvp_dyn);
  T* bar = geo + (size_t)ZB * SLOT_WORDS * BS;
  int* sj = reinterpret_cast<int*>(bar + (size_t)ZB * HVP_BAR_WORDS * BS);
  const fwd::FwdArgs<T>& g = a.g;
  const int ns = g.ns;
  for (int q = threadIdx.x; q < ns * ns * ns * NP; q += blockDim.x) sraw[q] = a.raw[q];
  if (threadIdx.x < ns * ns) sfilt[threadIdx.x] = g.filt2[threadIdx.x];
  if (threadIdx.x < 3) nb[threadIdx.x] = a.counts[threadIdx.x * FLAG_STRIDE];
  __syncthreads();
  int total = 0;
  for (int b = b0; b < b1; ++b) total += nb[b];
  for (int item = blockIdx.x * BS + threadIdx.x; item < total; item += gridDim.x * BS) {
    int b = b0, r = item;
    while (r >= nb[b]) r -= nb[b++];
    const int i = a.order[(size_t)b * g.n + r];
    using P = typename SelfPos<T>::type;
    const P pi = self_pos<T>(g, i);
    fwd::Shift<T, BATCH> sh;
    sh.load(g, i);
    const int ti = g.types[i];
    const int c = min(g.cnt[i], g.cap);
    const T gfi0 = a.gF[3 * (size_t)i], gfi1 = a.gF[3 * (size_t)i + 1], gfi2 = a.gF[3 * (size_t)i + 2];
    auto from_list = [&](int s, BondD<T>& bd, int& j) -> bool {
      T dx, dy, dz;
      Bond<T>::vec(g, sh, pi, g.nbr[(size_t)s * g.n + i], dx, dy, dz, j, bd.t);
      const T r2 = dx * dx + dy * dy + dz * dz;
      if (!(r2 <= sfilt[ti * ns + bd.t])) return false;
      bd.r = BM<T>::sq(r2);
      const T ir = T(1) / bd.r;
      bd.ux = dx * ir;
      bd.uy = dy * ir;
      bd.uz = dz * ir;
      const T wx = a.gF[3 * (size_t)j] - gfi0, wy = a.gF[3 * (size_t)j + 1] - gfi1,
              wz = a.gF[3 * (size_t)j + 2] - gfi2;
      bd.rd = bd.ux * wx + bd.uy * wy + bd.uz * wz;
      bd.px = (wx - bd.ux * bd.rd) * ir;
      bd.py = (wy - bd.uy * bd.rd) * ir;
      bd.pz = (wz - bd.uz * bd.rd) * ir;
      return true;
    };
    // the force term takes minus the derivative of D_w E_i: -bar(d) at atom
    // j, +bar(d) at the centre
    double gix = 0.0, giy = 0.0, giz = 0.0;
    auto scatter = [&](const BondD<T>& bd, int j, const BondBar<T>& q) {
      T dx, dy, dz;
      bond_vec_bar<T>(bd, q, dx, dy, dz);
      atomicAdd(gx + 3 * (size_t)j, -to_f64(dx));
      atomicAdd(gx + 3 * (size_t)j + 1, -to_f64(dy));
      atomicAdd(gx + 3 * (size_t)j + 2, -to_f64(dz));
      gix += to_f64(dx);
      giy += to_f64(dy);
      giz += to_f64(dz);
    };
    int z = 0;
    for (int s = 0; s < c && z <= ZB; ++s) {
      BondD<T> bd;
      int j;
      if (!from_list(s, bd, j)) continue;
      if (z < ZB) {
        put_slot<T>(geo, z, bd);
        sj[z * BS + threadIdx.x] = j;
        for (int f = 0; f < HVP_BAR_WORDS; ++f) bar[((size_t)z * HVP_BAR_WORDS + f) * BS + threadIdx.x] = T(0);
      }
      ++z;
    }
    if (z <= ZB) {
      // adjoints accumulated per slot, one scatter per bond
      atom_hvp<T, LAM3>(sraw, ns, ti, z,
                        [&](int q, BondD<T>& bd, int& j) -> bool {
                          get_slot<T>(geo, q, bd);
                          j = sj[q * BS + threadIdx.x];
                          return true;
                        },
                        [&](int q, const BondD<T>&, int, const BondBar<T>& v) {
                          T* p = bar + (size_t)q * HVP_BAR_WORDS * BS + threadIdx.x;
                          p[0] += v.r;
                          p[BS] += v.ux;
                          p[2 * BS] += v.uy;
                          p[3 * BS] += v.uz;
                          p[4 * BS] += v.rd;
                          p[5 * BS] += v.px;
                          p[6 * BS] += v.py;
                          p[7 * BS] += v.pz;
                        });
      for (int q = 0; q < z; ++q) {
        BondD<T> bd;
        get_slot<T>(geo, q, bd);
        const T* p = bar + (size_t)q * HVP_BAR_WORDS * BS + threadIdx.x;
        BondBar<T> v;
        v.r = p[0];
        v.ux = p[BS];
        v.uy = p[2 * BS];
        v.uz = p[3 * BS];
        v.rd = p[4 * BS];
        v.px = p[5 * BS];
        v.py = p[6 * BS];
        v.pz = p[7 * BS];
        scatter(bd, sj[q * BS + threadIdx.x], v);
      }
    } else {
      // more bonds than slots: bonds recomputed from the list, every adjoint
      // contribution scattered as it is formed (the map to bar(d) is linear)
      atom_hvp<T, LAM3>(sraw, ns, ti, c, from_list,
                        [&](int, const BondD<T>& bd, int j, const BondBar<T>& v) { scatter(bd, j, v); });
    }
    atomicAdd(gx + 3 * (size_t)i, gix);
    atomicAdd(gx + 3 * (size_t)i + 1, giy);
    atomicAdd(gx + 3 * (size_t)i + 2, giz);
  }
}

// Atoms ordered by their count of list entries inside the filter radii (at
// the build): neighbouring lanes of the adjoint kernel then run loops of the
// same length. A counting sort over 64 values: per-block histograms added to
// global counts, an exclusive scan, and the placement (block base from a
// global cursor plus the rank inside the block). bins: counts [0, 64),
// offsets [64, 128), cursors [128, 192).
__global__ void k_zw_count(int n, const uint8_t* __restrict__ zw, int* __restrict__ bins) {
  __shared__ int h[64];
  if (threadIdx.x < 64) h[threadIdx.x] = 0;
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&h[zw[i]], 1);
  __syncthreads();
  if (threadIdx.x < 64 && h[threadIdx.x]) atomicAdd(&bins[threadIdx.x], h[threadIdx.x]);
}
__global__ void k_zw_scan(int* __restrict__ bins) {
  if (threadIdx.x != 0) return;
  int s = 0;
  for (int b = 0; b < 64; ++b) {
    bins[64 + b] = s;
    bins[128 + b] = 0;
    s += bins[b];
  }
}
__global__ void k_zw_place(int n, const uint8_t* __restrict__ zw, int* __restrict__ bins,
                           int* __restrict__ fine) {
  __shared__ int h[64], base[64];
  if (threadIdx.x < 64) h[threadIdx.x] = 0;
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int b = 0, r = 0;
  if (i < n) {
    b = zw[i];
    r = atomicAdd(&h[b], 1);
  }
  __syncthreads();
  if (threadIdx.x < 64 && h[threadIdx.x])
    base[threadIdx.x] = bins[64 + threadIdx.x] + atomicAdd(&bins[128 + threadIdx.x], h[threadIdx.x]);
  __syncthreads();
  if (i < n) fine[base[b] + r] = i;
}

__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, int m) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) out[t] = (float)in[t];
}

// grad_x = -gE F (in place: f holds F on entry); gE of the atom's system
__global__ void k_scale_forces(double* __restrict__ f, const double* __restrict__ gE,
                               const int* __restrict__ atom_sys, int n3) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n3) f[t] = -gE[atom_sys ? atom_sys[t / 3] : 0] * f[t];
}

template <class T> const T* filt_ptr(Ctx* c);
template <> inline const float* filt_ptr<float>(Ctx* c) { return c->d_filt32; }
template <> inline const double* filt_ptr<double>(Ctx* c) { return c->d_filt64; }

// force weights in T: the caller's doubles, or a float copy (mixed path)
inline const double* weights_t(Ctx*, const double* gF, cudaStream_t, double*) { return gF; }
inline const float* weights_t(Ctx* c, const double* gF, cudaStream_t s, float*) {
  if (!gF) return nullptr;
  const int m = 3 * c->n;
  if (m > 0) {
    k_to_float<<<(m + 255) / 256, 256, 0, s>>>(gF, c->d_gf32, m);
    c->launches++;
  }
  return c->d_gf32;
}

template <class T>
BwdArgs<T> make_args(Ctx* c, const T* raw, const double* gE, const double* gF, double* grad,
                     cudaStream_t s) {
  BwdArgs<T> a;
  fwd::FwdArgs<T>& g = a.g;
  memset(&g, 0, sizeof(g));
  g.n = c->n;
  g.cap = c->cap;
  g.ns = c->ns;
  g.nbr = c->d_nbr;
  g.cnt = c->d_cnt;
  g.types = c->d_types;
  g.pos32 = c->d_pos32;
  g.posq = c->d_posq;
  g.pos64 = c->d_pos64;
  g.filt2 = filt_ptr<T>(c);
  const double scale = ldexp(1.0, c->grid.fix_shift);
  for (int q = 0; q < 3; ++q) {
    g.h[q] = (T)c->grid.h[q];
    g.hq[q] = (int)llrint(c->grid.h[q] * scale);
  }
  g.qinv = ldexpf(1.0f, -c->grid.fix_shift);
  g.sys = c->d_sys;
  g.atom_sys = c->d_atom_sys;
  a.raw = raw;
  a.gE = gE;
  a.atom_cell = c->n_sys > 0 ? c->d_atom_sys : nullptr;
  a.gF = weights_t(c, gF, s, (T*)nullptr);
  a.order = c->d_bucket;
  a.counts = c->d_flags + flag_bucket(0);
  a.fine = nullptr;
  a.grad = grad;
  return a;
}

template <class T>
int launch_t(Ctx* c, const T* raw, const double* gE, const double* gF, double* grad,
             cudaStream_t s) {
  BwdArgs<T> a = make_args<T>(c, raw, gE, gF, grad, s);
  constexpr int B = BwdBlock<T>::size;
  // atoms by bond count, sorted once per list (the placement order within a
  // count comes from atomics: sorting again would change the summation order
  // between calls on the same list); blocks of 256 cover the 64 bins
  if (c->n > 0 && !c->fine_valid) {
    const int nb = (c->n + 255) / 256;
    TGB_CUDA(c, cudaMemsetAsync(c->d_zbins, 0, sizeof(int) * 64, s));
    k_zw_count<<<nb, 256, 0, s>>>(c->n, c->d_zw, c->d_zbins);
    k_zw_scan<<<1, 32, 0, s>>>(c->d_zbins);
    k_zw_place<<<nb, 256, 0, s>>>(c->n, c->d_zw, c->d_zbins, c->d_fine);
    c->launches += 3;
    c->fine_valid = true;
  }
  if (c->n > 0) a.fine = c->d_fine;
  constexpr size_t dyn = slot_bytes<T>();
  const int grid = (c->n + B - 1) / B;
  if (grid > 0) {
    // two species on the mixed path: register accumulators (NS = 2)
    const bool two = c->ns == 2 && sizeof(T) == sizeof(float);
    void (*k)(BwdArgs<T>) = c->n_sys > 0 ? (two ? k_tersoff_bwd<T, 2, true> : k_tersoff_bwd<T, 0, true>)
                            : c->ns == 1 ? k_tersoff_bwd<T, 1, false>
                            : two        ? k_tersoff_bwd<T, 2, false>
                                         : k_tersoff_bwd<T, 0, false>;
    // static parameter tables plus the bond slots exceed the default 48 KB
    TGB_CUDA(c, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    k<<<grid, B, dyn, s>>>(a);
    c->launches++;
  }
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

template <class T, bool BATCH, bool LAM3, int ZB, int BS>
int launch_hvp_part(Ctx* c, const BwdArgs<T>& a, double* gx, int b0, int b1, cudaStream_t s) {
  long long items = 0;
  for (int b = b0; b < b1; ++b) items += c->nbucket[b];
  // grid from the host's bucket counts (the kernel loops over the device's),
  // at most 4 waves of the resident blocks
  constexpr size_t dyn = hvp_bytes<T, ZB, BS>();
  const int per_sm = (int)((200u << 10) / (dyn + 8192));
  const long long cap = (long long)(c->n_sm > 0 ? c->n_sm : 152) * (per_sm > 0 ? per_sm : 1) * 4;
  long long grid = (items + BS - 1) / BS + 1;
  if (grid > cap) grid = cap;
  void (*k)(BwdArgs<T>, double*, int, int) = k_tersoff_hvp<T, BATCH, LAM3, ZB, BS>;
  TGB_CUDA(c, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  k<<<(int)grid, BS, dyn, s>>>(a, gx, b0, b1);
  c->launches++;
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

template <class T, bool BATCH, bool LAM3>
int launch_hvp_buckets(Ctx* c, const BwdArgs<T>& a, double* gx, cudaStream_t s) {
  int st = launch_hvp_part<T, BATCH, LAM3, 4, 128>(c, a, gx, 0, 1, s);
  if (st) return st;
  return launch_hvp_part<T, BATCH, LAM3, 12, 64>(c, a, gx, 1, 3, s);
}

template <class T>
int launch_hvp_t(Ctx* c, const T* raw, const double* gF, double* gx, cudaStream_t s) {
  if (c->n == 0) return TERSOFF_OK;
  const BwdArgs<T> a = make_args<T>(c, raw, nullptr, gF, nullptr, s);
  if (c->n_sys > 0)
    return c->has_lam3 ? launch_hvp_buckets<T, true, true>(c, a, gx, s)
                       : launch_hvp_buckets<T, true, false>(c, a, gx, s);
  return c->has_lam3 ? launch_hvp_buckets<T, false, true>(c, a, gx, s)
                     : launch_hvp_buckets<T, false, false>(c, a, gx, s);
}

}  // namespace bwd

int launch_hvp(Ctx* c, const double* gF, double* grad_x, cudaStream_t s) {
  if (c->precision == TERSOFF_MIXED) return bwd::launch_hvp_t<float>(c, c->d_raw32, gF, grad_x, s);
  return bwd::launch_hvp_t<double>(c, c->d_raw64, gF, grad_x, s);
}

int launch_backward(Ctx* c, const double* gE, const double* gF, double* grad, cudaStream_t s) {
  if (c->precision == TERSOFF_MIXED) return bwd::launch_t<float>(c, c->d_raw32, gE, gF, grad, s);
  return bwd::launch_t<double>(c, c->d_raw64, gE, gF, grad, s);
}

int launch_scale_forces(Ctx* c, double* f, const double* gE, cudaStream_t s) {
  const int n3 = 3 * c->n;
  if (n3 == 0) return TERSOFF_OK;
  bwd::k_scale_forces<<<(n3 + 255) / 256, 256, 0, s>>>(f, gE, c->n_sys > 0 ? c->d_atom_sys : nullptr,
                                                        n3);
  c->launches++;
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

}  // namespace tgb

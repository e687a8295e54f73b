// Fused Tersoff energy / force / virial kernel (Sec. III Eq. 5-7, Sec. IV).
//
// One thread per centre atom i (the GPU mapping of Sec. IV-B, scheme (c)).
//  1. Filter (Sec. IV-B "filter component", Sec. IV-D): the thread scans its
//     skin list S_i and marks the entries within the largest cutoff that any
//     term of (type i, type j) can use; the marks form a bit mask.
//  2. Fast path, when the short list fits the compile-time capacity ZC: the
//     short list is loaded into registers (bond vectors, lengths, unit
//     vectors); for every j the first K loop accumulates zeta_ij together with
//     its derivatives with respect to x_j and every x_k (the pre-computed
//     derivatives of Sec. IV-A, kept in registers), then b_ij, V and
//     dV/dzeta are formed and the forces are applied. Forces on the
//     neighbours accumulate in registers; the force on i and the virial follow
//     from them at the end (every term's forces sum to zero, and all of atom
//     i's terms are centred on i).
//  3. General path (short list longer than ZC, the fall-back of Sec. IV-A):
//     Algorithm 2's loop order directly over S_i with the cutoff test inside
//     the loops, forces scattered per term.
// Forces are scattered with FP64 atomics (global sums in double); energy and
// virial are reduced in the warp, and across warps and blocks in double.
//
// Arithmetic: T = double for the FP64 path. T = float for the mixed path;
// there bond vectors come from exact integer differences of fixed-point
// positions, reciprocal square roots and reciprocals get one Newton step,
// and the exponent arguments of f_R, f_A carry the rounding residual of
// lambda * r, so each term is accurate to a few float ulps.
#pragma once
#include <cstdint>

#include "internal.cuh"

namespace tgb {
namespace fwd {

constexpr int BLOCK = 128;

// float -> double through the IEEE-754 bit layouts (exact; float subnormals
// flush to signed zero). Integer operations only.
__device__ __forceinline__ double f2d_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t sign = u & 0x80000000u;
  const uint32_t mag = u & 0x7fffffffu;
  uint32_t hi = (mag >> 3) + 0x38000000u;  // exponent rebias 127 -> 1023
  uint32_t lo = mag << 29;
  const bool tiny = mag < 0x00800000u;
  hi = tiny ? 0u : hi;
  lo = tiny ? 0u : lo;
  hi = (mag >= 0x7f800000u) ? ((mag >> 3) | 0x7ff00000u) : hi;  // inf / nan
  return __hiloint2double((int)(hi | sign), (int)lo);
}
__device__ __forceinline__ double to_f64(float v) { return f2d_bits(v); }
__device__ __forceinline__ double to_f64(double v) { return v; }

// ---------------------------------------------------------------- math per precision
__device__ __forceinline__ float fmaf_t(float x, float y, float z) { return fmaf(x, y, z); }
__device__ __forceinline__ double fmaf_t(double x, double y, double z) { return fma(x, y, z); }

template <class T> struct M;

template <> struct M<float> {
  // reciprocal square root with one Newton step on 1/y^2 = x
  static __device__ __forceinline__ float rsqrt_nr(float x) {
    float y = rsqrtf(x);
    float e = fmaf(-x * y, y, 1.0f);
    return fmaf(0.5f * y, e, y);
  }
  // reciprocal with one Newton step on 1/y = x
  static __device__ __forceinline__ float rcp_nr(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    float e = fmaf(-x, y, 1.0f);
    return fmaf(y, e, y);
  }
  // exp(-(lh + ll) r) with the rounding residual of lh*r folded in
  static __device__ __forceinline__ float exp_neg_lr(float lh, float ll, float r) {
    float a = lh * r;
    float res = fmaf(lh, r, -a) + ll * r;
    return expf(-a) * (1.0f - res);
  }
  static __device__ __forceinline__ float exp_(float x) { return expf(x); }
  static __device__ __forceinline__ void sincospi_(float x, float* s, float* c) {
    sincospif(x, s, c);
  }
  // hardware base-2 exponential and logarithm (special function unit)
  static __device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  }
  static __device__ __forceinline__ float lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  }
  // b = (1 + (beta zeta)^n)^(-1/(2n)),  db/dzeta. The inner power u goes
  // through the hardware log2/exp2: b depends weakly on u (relative
  // sensitivity u / (2 n (1 + u)) ~ 0.03 for Si), so their few-ulp errors move
  // b by ~1e-9. The outer power uses the accurate log2f/exp2f.
  static __device__ __forceinline__ void bond(float zeta, float beta, float n, float ninv2,
                                              float& b, float& db) {
    if (zeta > 0.0f) {
      float u = ex2(n * lg2(beta * zeta));
      float opu = 1.0f + u;
      b = exp2f(ninv2 * log2f(opu));
      db = -0.5f * b * u * rcp_nr(opu * zeta);
    } else {
      b = 1.0f;
      db = 0.0f;
    }
  }
};

template <> struct M<double> {
  static __device__ __forceinline__ double rsqrt_nr(double x) { return rsqrt(x); }
  // reciprocal: the hardware approximation and two Newton steps on 1/y = x
  // (each squares the relative error; the result is within about an ulp)
  static __device__ __forceinline__ double rcp_nr(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
  }
  static __device__ __forceinline__ double exp_neg_lr(double lh, double, double r) {
    return exp(-lh * r);
  }
  static __device__ __forceinline__ double exp_(double x) { return exp(x); }
  static __device__ __forceinline__ void sincospi_(double x, double* s, double* c) {
    sincospi(x, s, c);
  }
  static __device__ __forceinline__ void bond(double zeta, double beta, double n, double ninv2,
                                              double& b, double& db) {
    if (zeta > 0.0) {
      double u = exp(n * log(beta * zeta));
      double opu = 1.0 + u;
      b = exp(ninv2 * log1p(u));
      db = -0.5 * b * u * rcp_nr(opu * zeta);
    } else {
      b = 1.0;
      db = 0.0;
    }
  }
};

// ---------------------------------------------------------------- arguments
template <class T> struct FwdArgs {
  int n, cap;
  int ns;                // species count (used when the kernel's NS is 0)
  const uint32_t* nbr;   // slot-major skin list
  const int* cnt;
  const int* types;
  const float4* pos32;   // mixed: (u, type bits)
  const int4* posq;      // mixed: fixed-point u, type
  const dpos4* pos64;  // fp64: (u, type)
  const T* rec;          // ns^3 derived records
  T prm1[RSTRIDE];       // the record of a one-species table (read from the
                         // kernel-parameter constant bank)
  const T* filt2;        // ns x ns squared filter radii
  const float* near2;    // ns x ns: squared radii beyond which a bond gets its exact length
                         // residual (float path; unused by the double path)
  T h[3];                // cell edges
  int hq[3];             // cell edges in fixed point
  float qinv;            // 2^-fix_shift
  const uint32_t* shortl;  // slot-major short list (filter radius + margin)
  const int* zcnt;       // short-list counts
  int zs_cap;            // short-list capacity
  const int* order;      // atoms of this launch (a short-list size bucket) ...
  const int* n_items;    // ... and their device count
  const int* order2;     // optional second and third buckets processed after the first
  const int* n_items2;
  const int* order3;
  const int* n_items3;
  int identity;          // process atoms 0..n-1 directly (no bucket order)
  int all_general;       // ablation: every atom takes the general path (Algorithm 2 loops)
  float dlim2;           // short list valid while max squared displacement <= dlim2
  void* contrib;         // zs_cap x n force contributions (T4), receiver-major: slot p of
                         // atom j's column holds the force from its p-th short-list neighbour
  const uint8_t* rev;    // zs_cap x n: slot of i in the short list of i's s-th neighbour
  unsigned long long* kmask;  // per atom: entries whose receiving slot may be nonzero
  void* own;             // per-atom force of its own terms (T4)
  int atomic_mode;       // scatter every force with FP64 atomics (no slots)
  double* f;             // fallback forces, accumulated atomically
  double* acc;           // energy, virial (6); NULL: not needed (no reduction)
  double* eatom;         // optional per-atom energy
  int* flags;
  // batches of independent systems (kernels instantiated with BATCH)
  const SysShift* sys;   // per system: periodic shift units
  const int* atom_sys;   // system of each atom
  double* vatom;         // per-atom virial (6), summed per system afterwards
  int virial;            // the virial is wanted (with acc): 0 for the MD steps' thermo
  int* left;             // four-lane kernel: atoms left to the per-thread kernel
  int left_reset;        // per-thread kernel over that list: the last block zeroes the
                         // list's count (FLAG_LEFT) and its own ticket
};

// position of atom j relative to its origin, in T, and its species
template <class T> struct Pos;
template <> struct Pos<float> {
  // filter precision (cheap): float offsets
  static __device__ __forceinline__ void coarse(const FwdArgs<float>& a, int j, float& x,
                                                float& y, float& z, int& t) {
    int4 p = __ldg(&a.posq[j]);
    x = (float)p.x * a.qinv;
    y = (float)p.y * a.qinv;
    z = (float)p.z * a.qinv;
    t = p.w;
  }
};
template <> struct Pos<double> {
  static __device__ __forceinline__ void coarse(const FwdArgs<double>& a, int j, double& x,
                                                double& y, double& z, int& t) {
    dpos4 p = a.pos64[j];
    x = p.x;
    y = p.y;
    z = p.z;
    t = (int)p.w;
  }
};

__device__ __forceinline__ void decode(uint32_t e, int& j, int& ox, int& oy, int& oz) {
  j = (int)(e & ENTRY_JMASK);
  ox = (int)((e >> 26) & 3u) - 1;
  oy = (int)((e >> 28) & 3u) - 1;
  oz = (int)(e >> 30) - 1;
}

// Periodic shift units of atom i: the launch-wide cell edges, or (batches of
// systems) those of atom i's system, loaded once per atom.
template <class T, bool BATCH> struct Shift {
  __device__ __forceinline__ void load(const FwdArgs<T>&, int) {}
  __device__ __forceinline__ int hq(const FwdArgs<T>& a, int q) const { return a.hq[q]; }
  __device__ __forceinline__ T h(const FwdArgs<T>& a, int q) const { return a.h[q]; }
};
template <class T> struct Shift<T, true> {
  int hq_[3];
  T h_[3];
  __device__ __forceinline__ void load(const FwdArgs<T>& a, int i) {
    const SysShift& s = a.sys[a.atom_sys[i]];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      hq_[q] = s.hq[q];
      h_[q] = (T)s.h[q];
    }
  }
  __device__ __forceinline__ int hq(const FwdArgs<T>&, int q) const { return hq_[q]; }
  __device__ __forceinline__ T h(const FwdArgs<T>&, int q) const { return h_[q]; }
};

// Accurate bond vector from i to entry e's image of j.
template <class T> struct Bond;
template <> struct Bond<float> {
  template <bool B>
  static __device__ __forceinline__ void vec(const FwdArgs<float>& a, const Shift<float, B>& sh,
                                             int4 qi, uint32_t e, float& dx, float& dy,
                                             float& dz, int& j, int& tj) {
    int ox, oy, oz;
    decode(e, j, ox, oy, oz);
    int4 qj = __ldg(&a.posq[j]);
    int ix = qj.x - qi.x + ox * sh.hq(a, 0);
    int iy = qj.y - qi.y + oy * sh.hq(a, 1);
    int iz = qj.z - qi.z + oz * sh.hq(a, 2);
    dx = (float)ix * a.qinv;
    dy = (float)iy * a.qinv;
    dz = (float)iz * a.qinv;
    tj = qj.w;
  }
};
template <> struct Bond<double> {
  template <bool B>
  static __device__ __forceinline__ void vec(const FwdArgs<double>& a, const Shift<double, B>& sh,
                                             dpos4 pi, uint32_t e, double& dx, double& dy,
                                             double& dz, int& j, int& tj) {
    int ox, oy, oz;
    decode(e, j, ox, oy, oz);
    dpos4 pj = a.pos64[j];
    dx = (pj.x - pi.x) + ox * sh.h(a, 0);
    dy = (pj.y - pi.y) + oy * sh.h(a, 1);
    dz = (pj.z - pi.z) + oz * sh.h(a, 2);
    tj = (int)pj.w;
  }
};

// Exact length minus r for the bond to entry e (float path: from the exact
// fixed-point bond vector, whose squared length is an exact integer; the
// double path's r is already accurate to rounding: 0).
template <class T> struct Exact;
template <> struct Exact<float> {
  template <bool B>
  static __device__ float residual(const FwdArgs<float>& a, const Shift<float, B>& sh, int4 qi,
                                   uint32_t e, float r) {
    int j, ox, oy, oz;
    decode(e, j, ox, oy, oz);
    const int4 qj = __ldg(&a.posq[j]);
    const long long ix = qj.x - qi.x + ox * sh.hq(a, 0);
    const long long iy = qj.y - qi.y + oy * sh.hq(a, 1);
    const long long iz = qj.z - qi.z + oz * sh.hq(a, 2);
    const double q2 = (double)a.qinv * (double)a.qinv;
    const double r2 = (double)(ix * ix + iy * iy + iz * iz) * q2;  // exact up to one rounding
    const double rd = (double)r;
    return (float)((r2 - rd * rd) / (2.0 * rd));
  }
};
template <> struct Exact<double> {
  template <bool B>
  static __device__ double residual(const FwdArgs<double>&, const Shift<double, B>&, dpos4,
                                    uint32_t, double) {
    return 0.0;
  }
};
// bonds within this distance of their pair cutoff get the exact residual
constexpr float NEAR_CUT = 2e-3f;

template <class T> struct SelfPos;
template <> struct SelfPos<float> { using type = int4; };
template <> struct SelfPos<double> { using type = dpos4; };

template <class T>
__device__ __forceinline__ typename SelfPos<T>::type self_pos(const FwdArgs<T>& a, int i);
template <>
__device__ __forceinline__ int4 self_pos<float>(const FwdArgs<float>& a, int i) {
  return __ldg(&a.posq[i]);
}
template <>
__device__ __forceinline__ dpos4 self_pos<double>(const FwdArgs<double>& a, int i) {
  return a.pos64[i];
}

// ---------------------------------------------------------------- term pieces
// f_C and its derivative (Tersoff's cutoff), fields at offsets PID (pi/(2D)),
// DFC (-pi/(4D)), RIN (R - D), ROUT (R + D) and ROUTLO (the rounding residual
// of R + D in T). In the taper, with delta = R + D - r, f_C = 1/2 - 1/2
// sin(pi (r - R)/(2D)) = sin^2(pi delta/(4D)) and df_C/dr = -pi/(4D)
// sin(pi delta/(2D)): the form without cancellation as r reaches R + D, where
// f_C ~ delta^2 and, for n < 1, the bond order's derivative ~ zeta^(n-1) makes
// the force sensitive to delta itself. rex: exact r minus r, for bonds within
// a few thousandths of an Angstrom of a cutoff (0 otherwise).
template <class T>
__device__ __forceinline__ void cutoff(const T* p, int kPID, int kDFC, int kRIN, int kROUT,
                                       int kROUTLO, T r, T& fc, T& dfc, T rex = T(0)) {
  if (r <= p[kRIN]) {
    fc = T(1);
    dfc = T(0);
  } else {
    const T delta = (p[kROUT] - r) + (p[kROUTLO] - rex);
    if (!(delta > T(0))) {
      fc = dfc = T(0);
      return;
    }
    T s, c;
    // sin(pi delta/(4D)) = sinpi(delta/(4D)); p[kPID] / (2 pi) = 1/(4D)
    M<T>::sincospi_(delta * p[kPID] * T(0.15915494309189534), &s, &c);
    fc = s * s;
    dfc = p[kDFC] * (T(2) * s * c);
  }
}

// one three-body term zeta(i,j,k) and the coefficients of its derivative:
//   d zeta = A1 d(cos) + A2 d(r_ij) + (A3 - A2) d(r_ik)
template <class T, bool LAM3>
__device__ __forceinline__ void triplet(const T* p3, T rij, T rik, T cs, T& zt, T& A1, T& A2,
                                        T& A3, T rexk = T(0)) {
  T fc, dfc;
  cutoff<T>(p3, K_PID3, K_DFC3, K_RIN3, K_ROUT3, K_ROUT3LO, rik, fc, dfc, rexk);
  const T t = p3[K_H] - cs;
  const T t2 = t * t;
  const T q = M<T>::rcp_nr(p3[K_D2] + t2);
  const T g = p3[K_GC2D2] * (t2 * q) + p3[K_GAMMA];
  const T dg = -p3[K_G2C2] * t * q * q;
  T ex = T(1), dex = T(0);
  if (LAM3) {
    const T l3 = p3[K_LAM3];
    const int m = (int)p3[K_M];
    const T aa = l3 * (rij - rik);
    T am1 = T(1);
    for (int s = 1; s < m; ++s) am1 *= aa;
    ex = M<T>::exp_(am1 * aa);
    dex = ex * T(m) * l3 * am1;
  }
  const T fg = fc * g;
  zt = fg * ex;
  A1 = fc * dg * ex;
  A2 = fg * dex;
  A3 = dfc * g * ex;
}

// pair part: V = 1/2 fc (fR + b fA), dV/dr, dV/dzeta, for given f_C(r_ij)
// and its derivative
template <class T>
__device__ __forceinline__ void pair_fc(const T* p2, T rij, T zeta, T fc, T dfc, T& V, T& dVdr,
                                        T& dz) {
  T b, db;
  M<T>::bond(zeta, p2[K_BETA], p2[K_N], p2[K_NINV2], b, db);
  const T er = M<T>::exp_neg_lr(p2[K_LAM1], p2[K_LAM1LO], rij);
  const T ea = M<T>::exp_neg_lr(p2[K_LAM2], p2[K_LAM2LO], rij);
  const T fr = p2[K_A] * er;
  const T fa = -p2[K_B] * ea;
  const T s = fr + b * fa;
  V = T(0.5) * fc * s;
  // d/dr [fc (fR + b fA)] at fixed b: fR' = -l1 fR, fA' = -l2 fA
  dVdr = T(0.5) * (dfc * s - fc * (p2[K_LAM1] * fr + p2[K_LAM2] * b * fa));
  dz = T(0.5) * fc * fa * db;
}

template <class T>
__device__ __forceinline__ void pair(const T* p2, T rij, T zeta, T& V, T& dVdr, T& dz,
                                     T rexj = T(0)) {
  T fc, dfc;
  cutoff<T>(p2, K_PID2, K_DFC2, K_RIN2, K_ROUT2, K_ROUT2LO, rij, fc, dfc, rexj);
  pair_fc<T>(p2, rij, zeta, fc, dfc, V, dVdr, dz);
}

template <class T> struct C4;
template <> struct C4<float> {
  using type = float4;
  static __device__ __forceinline__ float4 make(float x, float y, float z) {
    return make_float4(x, y, z, 0.0f);
  }
};
template <> struct C4<double> {
  using type = dpos4;
  static __device__ __forceinline__ dpos4 make(double x, double y, double z) {
    return dpos4{x, y, z, 0.0};
  }
};

template <class T>
__device__ __forceinline__ void store_slot(const FwdArgs<T>& a, void* base, size_t idx, T x, T y,
                                           T z) {
  ((typename C4<T>::type*)base)[idx] = C4<T>::make(x, y, z);
}
// Receiving slot of the force that atom i's terms put on the neighbour j held
// in entry s of i's short list: slot rev(i, s) of j's column (the entry of j's
// short list that holds i). Short-list membership is symmetric and no atom
// appears twice in a list (box edges are at least twice the list radius), so
// every slot of every column has exactly one writer, and each atom's gather
// reads its own column.
template <class T>
__device__ __forceinline__ size_t recv_slot(const FwdArgs<T>& a, int s, int i, int j) {
  return (size_t)__ldg(&a.rev[(size_t)s * a.n + i]) * a.n + j;
}
template <class T>
__device__ __forceinline__ int entry_atom(const FwdArgs<T>& a, const uint32_t* list, int s, int i) {
  return (int)(list[(size_t)s * a.n + i] & ENTRY_JMASK);
}

// An atom whose stored short list was truncated (more entries than its
// capacity) scatters with atomics; the receiving slots of its stored entries
// must then read zero.
template <class T>
__device__ __forceinline__ void zero_stored(const FwdArgs<T>& a, int i, int z_list) {
  const int zs = z_list < a.zs_cap ? z_list : a.zs_cap;
  for (int s = 0; s < zs; ++s)
    store_slot<T>(a, a.contrib, recv_slot(a, s, i, entry_atom(a, a.shortl, s, i)), T(0), T(0),
                  T(0));
  a.kmask[i] = 0ull;
}

template <class T>
__device__ __forceinline__ void add_slot(const FwdArgs<T>& a, size_t idx, T x, T y, T z) {
  typename C4<T>::type* p = (typename C4<T>::type*)a.contrib + idx;
  typename C4<T>::type v = *p;
  v.x += x;
  v.y += y;
  v.z += z;
  *p = v;
}

__device__ __forceinline__ void atomic_add3(double* f, int j, double a, double b, double c) {
  atomicAdd(f + 3 * (size_t)j + 0, a);
  atomicAdd(f + 3 * (size_t)j + 1, b);
  atomicAdd(f + 3 * (size_t)j + 2, c);
}

// ---------------------------------------------------------------- general path
// Algorithm 2 directly over S_i, cutoff tests inside the loops.
// record offset of (ti, tj, tk); a one-species table has a single record
template <int NS>
__device__ __forceinline__ int rec_off(int ns, int ti, int tj, int tk) {
  return NS == 1 ? 0 : ((ti * ns + tj) * ns + tk) * RSTRIDE;
}

// slots: forces go to the per-slot contributions of the list (the short list),
// otherwise to the fallback buffer through FP64 atomics.
// use_mask: bit s of mask marks the entries s < 64 inside the filter radius
// (the others cannot be in any term and are skipped before their bond vector
// is formed).
template <class T, int NS, bool LAM3, bool BATCH>
__device__ __forceinline__ void general_atom(const FwdArgs<T>& a, const Shift<T, BATCH>& sh,
                                          const T* srec, int i, int ti,
                                          const uint32_t* list, int c, bool slots,
                                          bool use_mask, unsigned long long mask, T& ei,
                                          T* w) {
  using P = typename SelfPos<T>::type;
  const int ns = NS > 0 ? NS : a.ns;
  const P pi = self_pos<T>(a, i);
  T fix = 0, fiy = 0, fiz = 0;
  // exact length residual of a bond near a cutoff (float path)
  auto near_res = [&](uint32_t e, T r2, T r, int tx) -> T {
    if (sizeof(T) == 4 && r2 > a.near2[ti * ns + tx]) return Exact<T>::residual(a, sh, pi, e, r);
    return T(0);
  };
  if (slots)
    for (int q = 0; q < c; ++q)
      store_slot<T>(a, a.contrib, recv_slot(a, q, i, entry_atom(a, list, q, i)), T(0), T(0), T(0));
  for (int sj = 0; sj < c; ++sj) {
    if (use_mask && !((mask >> sj) & 1ull)) continue;
    T dxj, dyj, dzj;
    int j, tj;
    Bond<T>::vec(a, sh, pi, list[(size_t)sj * a.n + i], dxj, dyj, dzj, j, tj);
    const T* p2 = srec + rec_off<NS>(ns, ti, tj, tj);
    const T r2j = dxj * dxj + dyj * dyj + dzj * dzj;
    const T rij = r2j * M<T>::rsqrt_nr(r2j);
    if (!(rij < p2[K_ROUT2])) continue;
    const T rexj = near_res(list[(size_t)sj * a.n + i], r2j, rij, tj);
    const T rinj = T(1) / rij;
    const T uxj = dxj * rinj, uyj = dyj * rinj, uzj = dzj * rinj;
    T zeta = 0;
    for (int sk = 0; sk < c; ++sk) {
      if (sk == sj || (use_mask && !((mask >> sk) & 1ull))) continue;
      T dxk, dyk, dzk;
      int k, tk;
      Bond<T>::vec(a, sh, pi, list[(size_t)sk * a.n + i], dxk, dyk, dzk, k, tk);
      const T* p3 = srec + rec_off<NS>(ns, ti, tj, tk);
      const T r2k = dxk * dxk + dyk * dyk + dzk * dzk;
      const T rik = r2k * M<T>::rsqrt_nr(r2k);
      if (!(rik < p3[K_ROUT3])) continue;
      const T cs = (dxj * dxk + dyj * dyk + dzj * dzk) * rinj / rik;
      T zt, A1, A2, A3;
      triplet<T, LAM3>(p3, rij, rik, cs, zt, A1, A2, A3,
                       near_res(list[(size_t)sk * a.n + i], r2k, rik, tk));
      zeta += zt;
    }
    T V, dVdr, dz;
    pair<T>(p2, rij, zeta, V, dVdr, dz, rexj);
    ei += V;
    T Fjx = -dVdr * uxj, Fjy = -dVdr * uyj, Fjz = -dVdr * uzj;
    for (int sk = 0; sk < c; ++sk) {
      if (sk == sj || (use_mask && !((mask >> sk) & 1ull))) continue;
      T dxk, dyk, dzk;
      int k, tk;
      Bond<T>::vec(a, sh, pi, list[(size_t)sk * a.n + i], dxk, dyk, dzk, k, tk);
      const T* p3 = srec + rec_off<NS>(ns, ti, tj, tk);
      const T r2k = dxk * dxk + dyk * dyk + dzk * dzk;
      const T rik = r2k * M<T>::rsqrt_nr(r2k);
      if (!(rik < p3[K_ROUT3])) continue;
      const T rink = T(1) / rik;
      const T uxk = dxk * rink, uyk = dyk * rink, uzk = dzk * rink;
      const T cs = uxj * uxk + uyj * uyk + uzj * uzk;
      T zt, A1, A2, A3;
      triplet<T, LAM3>(p3, rij, rik, cs, zt, A1, A2, A3,
                       near_res(list[(size_t)sk * a.n + i], r2k, rik, tk));
      // d zeta / d x_j and d x_k
      const T gjx = A1 * (uxk - cs * uxj) * rinj + A2 * uxj;
      const T gjy = A1 * (uyk - cs * uyj) * rinj + A2 * uyj;
      const T gjz = A1 * (uzk - cs * uzj) * rinj + A2 * uzj;
      const T gkx = A1 * (uxj - cs * uxk) * rink + (A3 - A2) * uxk;
      const T gky = A1 * (uyj - cs * uyk) * rink + (A3 - A2) * uyk;
      const T gkz = A1 * (uzj - cs * uzk) * rink + (A3 - A2) * uzk;
      Fjx -= dz * gjx;
      Fjy -= dz * gjy;
      Fjz -= dz * gjz;
      const T Fkx = -dz * gkx, Fky = -dz * gky, Fkz = -dz * gkz;
      if (slots)
        add_slot<T>(a, recv_slot(a, sk, i, k), Fkx, Fky, Fkz);
      else
        atomic_add3(a.f, k, to_f64(Fkx), to_f64(Fky), to_f64(Fkz));
      fix -= Fkx;
      fiy -= Fky;
      fiz -= Fkz;
      w[0] += dxk * Fkx;
      w[1] += dyk * Fky;
      w[2] += dzk * Fkz;
      w[3] += dxk * Fky;
      w[4] += dxk * Fkz;
      w[5] += dyk * Fkz;
    }
    if (slots)
      add_slot<T>(a, recv_slot(a, sj, i, j), Fjx, Fjy, Fjz);
    else
      atomic_add3(a.f, j, to_f64(Fjx), to_f64(Fjy), to_f64(Fjz));
    fix -= Fjx;
    fiy -= Fjy;
    fiz -= Fjz;
    w[0] += dxj * Fjx;
    w[1] += dyj * Fjy;
    w[2] += dzj * Fjz;
    w[3] += dxj * Fjy;
    w[4] += dxj * Fjz;
    w[5] += dyj * Fjz;
  }
  if (slots)
    store_slot<T>(a, a.own, (size_t)i, fix, fiy, fiz);
  else
    atomic_add3(a.f, i, to_f64(fix), to_f64(fiy), to_f64(fiz));
}

// atomic mode: the gather must see zero in the atom's own slot and its column
template <class T>
__device__ __forceinline__ void clear_slots(const FwdArgs<T>& a, int i) {
  store_slot<T>(a, a.own, (size_t)i, T(0), T(0), T(0));
  int z = a.zcnt[i];
  z = z < a.zs_cap ? z : a.zs_cap;
  for (int q = 0; q < z; ++q) store_slot<T>(a, a.contrib, (size_t)q * a.n + i, T(0), T(0), T(0));
}

// ---------------------------------------------------------------- reduction
// Energy and virial of the double path: the 7 per-thread sums (padded to 8)
// are reduce-scattered across the warp (halving exchanges: 4, 2, 1 values),
// then summed over the remaining lanes; lanes 0, 4, ..., 28 end with the 8
// warp totals. Warp totals are summed in double over the block and added to
// acc with one atomic each.
template <int NB = BLOCK>
__device__ __forceinline__ void block_reduce_store_d(double ei, const double* w, double* acc) {
  __shared__ double part[NB / 32][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double v[8] = {ei, w[0], w[1], w[2], w[3], w[4], w[5], 0.0};
  const bool hi16 = lane & 16;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double send = hi16 ? v[q] : v[q + 4];
    const double keep = hi16 ? v[q + 4] : v[q];
    v[q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  const bool hi8 = lane & 8;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const double send = hi8 ? v[q] : v[q + 2];
    const double keep = hi8 ? v[q + 2] : v[q];
    v[q] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const bool hi4 = lane & 4;
  {
    const double send = hi4 ? v[0] : v[1];
    const double keep = hi4 ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
  if ((lane & 3) == 0) {
    const int idx = (hi16 ? 4 : 0) + (hi8 ? 2 : 0) + (hi4 ? 1 : 0);
    part[wid][idx] = v[0];
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    double s = 0.0;
    for (int q = 0; q < NB / 32; ++q) s += part[q][threadIdx.x];
    atomicAdd(&acc[threadIdx.x * ACC_STRIDE], s);
  }
}

// ---------------------------------------------------------------- thread sums
// Energy and virial (7 components) summed by one thread over the atoms it
// handles, kept in the thread's column of a shared-memory table. Float path:
// compensated pairs (s, e) (Knuth's TwoSum keeps each addition's rounding
// error in e), reduced over the warp as pairs and carried into double at the
// warp totals: exact to double rounding at a few float operations per value,
// where double arithmetic would run on GB300's FP64 pipe at 1/62 of the FP32
// rate. Double path: plain doubles.
template <class T> struct SumT;
template <> struct SumT<float> { using type = float2; };
template <> struct SumT<double> { using type = double; };

__device__ __forceinline__ float2 pair_add(float2 a, float2 b) {
  const float t = a.x + b.x;
  const float bp = t - a.x;
  const float err = (a.x - (t - bp)) + (b.x - bp);
  return make_float2(t, (a.y + b.y) + err);
}
__device__ __forceinline__ void sum_zero(float2& p) { p = make_float2(0.0f, 0.0f); }
__device__ __forceinline__ void sum_zero(double& p) { p = 0.0; }
__device__ __forceinline__ void sum_add(float2& p, float x) { p = pair_add(p, make_float2(x, 0.0f)); }
__device__ __forceinline__ void sum_add(double& p, double x) { p += x; }
// a compensated per-atom value (s, e)
__device__ __forceinline__ void sum_add2(float2& p, float s_, float e_) {
  p = pair_add(p, make_float2(s_, e_));
}
__device__ __forceinline__ void sum_add2(double& p, double s_, double e_) { p += s_ + e_; }

__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// Block sum of the 7 per-thread values col[k * NB] (this thread's column),
// added to acc with one double atomic per component and block: the same
// halving reduce-scatter over the warp as block_reduce_store_d, on pairs.
template <int NB = BLOCK>
__device__ __forceinline__ void block_reduce_sums(const float2* col, double* acc) {
  __shared__ double part[NB / 32][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float2 v[8];
#pragma unroll
  for (int k = 0; k < 7; ++k) v[k] = col[k * NB];
  v[7] = make_float2(0.0f, 0.0f);
  const bool hi16 = lane & 16;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float2 send = hi16 ? v[q] : v[q + 4];
    const float2 keep = hi16 ? v[q + 4] : v[q];
    v[q] = pair_add(keep, shfl_xor2(send, 16));
  }
  const bool hi8 = lane & 8;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const float2 send = hi8 ? v[q] : v[q + 2];
    const float2 keep = hi8 ? v[q + 2] : v[q];
    v[q] = pair_add(keep, shfl_xor2(send, 8));
  }
  const bool hi4 = lane & 4;
  {
    const float2 send = hi4 ? v[0] : v[1];
    const float2 keep = hi4 ? v[1] : v[0];
    v[0] = pair_add(keep, shfl_xor2(send, 4));
  }
  v[0] = pair_add(v[0], shfl_xor2(v[0], 2));
  v[0] = pair_add(v[0], shfl_xor2(v[0], 1));
  if ((lane & 3) == 0) {
    const int idx = (hi16 ? 4 : 0) + (hi8 ? 2 : 0) + (hi4 ? 1 : 0);
    part[wid][idx] = to_f64(v[0].x) + to_f64(v[0].y);
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    double s = 0.0;
    for (int q = 0; q < NB / 32; ++q) s += part[q][threadIdx.x];
    atomicAdd(&acc[threadIdx.x * ACC_STRIDE], s);
  }
}
template <int NB = BLOCK>
__device__ __forceinline__ void block_reduce_sums(const double* col, double* acc) {
  double wd[6];
  for (int k = 0; k < 6; ++k) wd[k] = col[(1 + k) * NB];
  block_reduce_store_d<NB>(col[0], wd, acc);
}

// ---------------------------------------------------------------- the kernel
// Running sum of one thread: plain (CS false) or compensated (CS true: Knuth's
// TwoSum keeps the rounding error of every float addition in e, so s + e is
// the exact sum of the added terms up to the rounding of e itself).
template <class T, bool CS> struct Acc {
  T s = T(0);
  __device__ __forceinline__ void add(T x) { s += x; }
  // s += c t + b u, as two fused multiply-adds
  __device__ __forceinline__ void madd2(T c, T t, T b, T u) { s = fmaf_t(c, t, fmaf_t(b, u, s)); }
  __device__ __forceinline__ void sub(const Acc& o) { s -= o.s; }
  __device__ __forceinline__ T lo() const { return T(0); }
  __device__ __forceinline__ double d() const { return to_f64(s); }
};
template <class T> struct Acc<T, true> {
  T s = T(0), e = T(0);
  __device__ __forceinline__ void add(T x) {
    const T t = s + x;
    const T bp = t - s;
    e += (s - (t - bp)) + (x - bp);
    s = t;
  }
  __device__ __forceinline__ void madd2(T c, T t, T b, T u) { add(fmaf_t(c, t, b * u)); }
  __device__ __forceinline__ void sub(const Acc& o) {
    add(-o.s);
    e -= o.e;
  }
  __device__ __forceinline__ T lo() const { return e; }
  __device__ __forceinline__ double d() const { return to_f64(s) + to_f64(e); }
};

// CS (float, one species, single systems only): every sum a thread forms over
// the terms of its atom -- the force on each neighbour and on the atom, its
// energy and virial -- is compensated, carried into double, and forces are
// scattered with FP64 atomics (the TERSOFF_ABLATE_COMP_ATOM_SUMS variant).
// Resident blocks per SM that the force kernel's launch bound asks for: the
// register budget, and the grid of the "waves" launch option.
// The FP64 instances run on the FP64 pipe (about 87% busy on the benchmark):
// four blocks per SM give them 128 registers and no spills.
__host__ __device__ constexpr int fwd_min_blocks(int zc, int ev, bool dbl = false) {
  return zc <= 4 ? (dbl ? 4 : (ev == 2 ? 7 : 8)) : 4;
}

// EV: 2 energy and virial (and per-atom energy) as requested; 1 energy and
// per-atom energy only (the MD steps' thermo); 0 forces only (the MD steps
// without thermo). Instances 0 and 1 carry less bookkeeping and fit one more
// block per SM.
template <class T, int NS, int ZC, int MODE, bool BATCH = false, bool CS = false, int EV = 2>
__global__ void __launch_bounds__(BLOCK, fwd_min_blocks(ZC, EV, sizeof(T) == 8))
    k_tersoff(const __grid_constant__ FwdArgs<T> a) {
  static_assert(!(CS && BATCH), "compensated per-atom sums: single systems only");
  static_assert(EV == 2 || !BATCH, "batches need the per-atom energy and virial");
  pdl_wait();  // the previous kernel's writes (a launch with launch_pdl)
  constexpr int SNS = NS > 1 ? NS : (NS == 1 ? 1 : TERSOFF_MAX_SPECIES);
  constexpr int SREC = NS == 1 ? 1 : SNS * SNS * SNS * RSTRIDE;
  __shared__ T srec_s[SREC];
  __shared__ T sfilt[SNS * SNS];
  const int ns = NS > 0 ? NS : a.ns;
  // launch-uniform words, read once per block (one load per lane, together)
  __shared__ int uni[5];
  __shared__ float snear[SNS * SNS];
  if (NS != 1)
    for (int q = threadIdx.x; q < ns * ns * ns * RSTRIDE; q += BLOCK) srec_s[q] = a.rec[q];
  if (threadIdx.x < ns * ns) {
    sfilt[threadIdx.x] = a.filt2[threadIdx.x];
    snear[threadIdx.x] = sizeof(T) == 4 ? a.near2[threadIdx.x] : 0.0f;
  }
  if (threadIdx.x < 5) {
    const int* src = threadIdx.x == 0   ? a.n_items
                     : threadIdx.x == 1 ? a.flags + FLAG_REV_MISS
                     : threadIdx.x == 2 ? a.flags + FLAG_DMAX
                     : threadIdx.x == 3 ? a.n_items2
                                        : a.n_items3;
    uni[threadIdx.x] = src ? *src : 0;
  }
  __syncthreads();
  // parameters: shared memory for several species (type-dependent records),
  // the constant bank for one species (uniform, operands of the FP instructions)
  const T* srec = NS == 1 ? a.prm1 : srec_s;
  constexpr bool LAM3 = MODE == 1;
  const int n_first = uni[0];
  const int n_second = uni[0] + uni[3];
  const int n_items = a.identity ? a.n : min(n_second + uni[4], a.n);
  // slots: contributions go to per-slot stores (needs the stored short list and
  // its reverse map); otherwise FP64 atomics into the fallback buffer
  const bool slots_ok = uni[1] == 0;
  // the stored short list holds every atom that can be inside a cutoff while no
  // atom has moved more than half the list margin since the build (uniform)
  const bool use_short = __int_as_float(uni[2]) <= a.dlim2;
  const bool slots = !a.atomic_mode && use_short && slots_ok;
  if (blockIdx.x == 0 && threadIdx.x == 0) a.flags[FLAG_EXTRA] = slots ? 0 : 1;
  // the atom's own virial sums (float), and the thread's energy and virial
  // over its atoms in double, kept in the thread's column of a shared-memory
  // table (not in registers) and formed only when the reduction is wanted
  T w[6];
  __shared__ typename SumT<T>::type tsum[7][BLOCK];
  const bool want_acc = a.acc != nullptr;
  if (want_acc)
    for (int q = 0; q < 7; ++q) sum_zero(tsum[q][threadIdx.x]);
  bool any = false;
  for (int item = blockIdx.x * BLOCK + threadIdx.x; item < n_items;
       item += gridDim.x * BLOCK) {
    any = true;
    const int i = a.identity ? item
                  : (item < n_first ? a.order[item]
                     : (item < n_second ? a.order2[item - n_first] : a.order3[item - n_second]));
    T eatom_i = T(0);
    Acc<T, CS> eatom_c;  // CS: the atom's energy (fast path)
    Acc<T, CS> wa[6];    // CS: the atom's virial (fast path)
    for (int q = 0; q < 6; ++q) w[q] = T(0);
    Shift<T, BATCH> sh;
    sh.load(a, i);
    int ti;
    int z;
    unsigned long long mask = 0ull;
    const uint32_t* list;
    int c;
    bool general;
    bool filtered = false;  // the register slots come from a cutoff mask over list
    bool have_mask = false; // mask covers every entry of list (at most 64)
    int z_list = 0;         // stored short-list length (slots mode bookkeeping)
    using P = typename SelfPos<T>::type;
    const P pi = self_pos<T>(a, i);
    // the first ZC stored entries and their reverse slots (for the scatter),
    // loaded together with the count: every atom has at least 8 list slots, so
    // they are in bounds whatever the count
    uint32_t pre[ZC];
    int rv[ZC];
    if (use_short) {
#pragma unroll
      for (int q = 0; q < ZC; ++q) {
        pre[q] = a.shortl[(size_t)q * a.n + i];
        rv[q] = slots ? (int)__ldg(&a.rev[(size_t)q * a.n + i]) : 0;
      }
      z_list = a.zcnt[i];
      ti = a.types[i];
      list = a.shortl;
      c = z_list;
      z = z_list;
      general = z_list > a.zs_cap || a.all_general;
      if (general) {  // short list truncated: use the skin list
        list = a.nbr;
        c = min(a.cnt[i], a.cap);
      } else if (z_list > ZC) {
        // more stored entries than registers: keep those inside the cutoffs now
        filtered = true;
        T xi, yi, zi;
        int tii;
        Pos<T>::coarse(a, i, xi, yi, zi, tii);
        const bool fits = z_list <= 64;
        if (fits)
          for (int s = 0; s < z_list; ++s) {
            const uint32_t e = a.shortl[(size_t)s * a.n + i];
            int j, ox, oy, oz;
            decode(e, j, ox, oy, oz);
            T xj, yj, zj;
            int tj;
            Pos<T>::coarse(a, j, xj, yj, zj, tj);
            const T dx = (xj - xi) + ox * sh.h(a, 0);
            const T dy = (yj - yi) + oy * sh.h(a, 1);
            const T dz = (zj - zi) + oz * sh.h(a, 2);
            const T r2 = dx * dx + dy * dy + dz * dz;
            if (r2 <= sfilt[ti * ns + tj]) mask |= 1ull << s;
          }
        z = __popcll(mask);
        general = !fits || z > ZC || a.all_general;
        have_mask = fits;
      }
    } else {
      // filter the skin list into a bit mask (Sec. IV-D)
      filtered = true;
      T xi, yi, zi;
      Pos<T>::coarse(a, i, xi, yi, zi, ti);
      c = min(a.cnt[i], a.cap);
      list = a.nbr;
      const bool fits = c <= 64;
      if (fits) {
        for (int s = 0; s < c; ++s) {
          const uint32_t e = a.nbr[(size_t)s * a.n + i];
          int j, ox, oy, oz;
          decode(e, j, ox, oy, oz);
          T xj, yj, zj;
          int tj;
          Pos<T>::coarse(a, j, xj, yj, zj, tj);
          const T dx = (xj - xi) + ox * sh.h(a, 0);
          const T dy = (yj - yi) + oy * sh.h(a, 1);
          const T dz = (zj - zi) + oz * sh.h(a, 2);
          const T r2 = dx * dx + dy * dy + dz * dz;
          if (r2 <= sfilt[ti * ns + tj]) mask |= 1ull << s;
        }
      }
      z = __popcll(mask);
      general = !fits || z > ZC || a.all_general;
      have_mask = fits;
    }
    if (!slots && !a.atomic_mode) clear_slots<T>(a, i);
    if (general) {
      atomicAdd(&a.flags[FLAG_FALLBACK], 1);
      if (slots && list != a.shortl) {
        atomicOr(&a.flags[FLAG_EXTRA_STICKY], 1);
        zero_stored<T>(a, i, z_list);
      }
      general_atom<T, NS, LAM3, BATCH>(a, sh, srec, i, ti, list, c, slots && list == a.shortl,
                                       have_mask, mask, eatom_i, w);
      if (slots && list == a.shortl) a.kmask[i] = ~0ull;  // every entry written
    } else {
      // 2. short list into registers
      T ux[ZC], uy[ZC], uz[ZC], rr[ZC], ri[ZC], rex[ZC];
      T fc3[ZC], dfc3[ZC];  // MODE 2: f_C(r_iq) of the bond's own record
      int jj[ZC], tt[ZC];
      const unsigned long long kept = mask;
      // stored short list, not filtered: the entries loaded above
#pragma unroll
      for (int q = 0; q < ZC; ++q) {
        ux[q] = uy[q] = uz[q] = T(0);
        rr[q] = T(1);
        ri[q] = T(1);
        rex[q] = T(0);
        fc3[q] = dfc3[q] = T(0);
        jj[q] = i;
        tt[q] = 0;
        if (q < z) {
          uint32_t e;
          if (filtered) {
            const int sl = __ffsll(mask) - 1;
            mask &= mask - 1ull;
            e = list[(size_t)sl * a.n + i];
          } else {
            e = pre[q];
          }
          T dx, dy, dz;
          int j, tj;
          Bond<T>::vec(a, sh, pi, e, dx, dy, dz, j, tj);
          const T r2 = dx * dx + dy * dy + dz * dz;
          const T inv = M<T>::rsqrt_nr(r2);
          ri[q] = inv;
          rr[q] = r2 * inv;
          T rx = T(0);
          if (sizeof(T) == 4 && r2 > snear[ti * ns + tj])  // near a cutoff: exact length
            rx = Exact<T>::residual(a, sh, pi, e, rr[q]);
          rex[q] = rx;
          if (MODE == 2) {
            // symmetric tables: f_C(r_iq) of record (ti, tq, tq) serves both
            // the three-body terms with k = q and the pair term of bond q
            const T* pq = srec + rec_off<NS>(ns, ti, tj, tj);
            if (rr[q] < pq[K_ROUT3])
              cutoff<T>(pq, K_PID3, K_DFC3, K_RIN3, K_ROUT3, K_ROUT3LO, rr[q], fc3[q], dfc3[q], rx);
          }
          ux[q] = dx * inv;
          uy[q] = dy * inv;
          uz[q] = dz * inv;
          jj[q] = j;
          tt[q] = tj;
        }
      }
      Acc<T, CS> fx[ZC], fy[ZC], fz[ZC];

      if (MODE == 2) {
        // Symmetric tables without a lambda3 term: the angular part of
        // zeta(i,j,k) and zeta(i,k,j) is the same, and f_C(r_ik) does not
        // depend on j. Each unordered neighbour pair {j,k} is evaluated once
        // for the zeta sums and once (recomputed) for the forces.
        T zeta[ZC], dzt[ZC];
#pragma unroll
        for (int q = 0; q < ZC; ++q) zeta[q] = dzt[q] = T(0);
        // pass 1: zeta_ij = sum_k f_C(r_ik) g(theta_ijk)
#pragma unroll
        for (int qj = 0; qj < ZC; ++qj)
#pragma unroll
          for (int qk = qj + 1; qk < ZC; ++qk) {
            // (the test keeps the compiler from interleaving all six pairs:
            // without it the kernel spills)
            if (qk >= z) continue;
            const T* p3 = srec + rec_off<NS>(ns, ti, tt[qj], tt[qk]);
            const T cs = ux[qj] * ux[qk] + uy[qj] * uy[qk] + uz[qj] * uz[qk];
            const T t = p3[K_H] - cs;
            const T tq = t * M<T>::rcp_nr(p3[K_D2] + t * t);
            const T g = p3[K_GC2D2] * (t * tq) + p3[K_GAMMA];
            zeta[qj] += fc3[qk] * g;
            zeta[qk] += fc3[qj] * g;
          }
        // pair terms, b_ij and dV/dzeta
#pragma unroll
        for (int qj = 0; qj < ZC; ++qj)
          if (qj < z) {
            const T* p2 = srec + rec_off<NS>(ns, ti, tt[qj], tt[qj]);
            if (rr[qj] < p2[K_ROUT2]) {
              T V, dVdr, dz;
              pair_fc<T>(p2, rr[qj], zeta[qj], fc3[qj], dfc3[qj], V, dVdr, dz);
              if (EV >= 1) eatom_c.add(V);
              dzt[qj] = dz;
              fx[qj].add(-dVdr * ux[qj]);
              fy[qj].add(-dVdr * uy[qj]);
              fz[qj].add(-dVdr * uz[qj]);
            }
          }
        // pass 2: -dV/dzeta_ij d zeta_ij/dx - dV/dzeta_ik d zeta_ik/dx per pair
        // {j,k}; with q = 1/(d^2 + t^2): g = gamma + gamma c^2/d^2 t^2 q and
        // dg/dcos = -2 gamma c^2 t q^2
#pragma unroll
        for (int qj = 0; qj < ZC; ++qj)
#pragma unroll
          for (int qk = qj + 1; qk < ZC; ++qk) {
            if (qk >= z) continue;
            const T* p3 = srec + rec_off<NS>(ns, ti, tt[qj], tt[qk]);
            const T cs = ux[qj] * ux[qk] + uy[qj] * uy[qk] + uz[qj] * uz[qk];
            const T t = p3[K_H] - cs;
            const T q = M<T>::rcp_nr(p3[K_D2] + t * t);
            const T tq = t * q;
            const T g = p3[K_GC2D2] * (t * tq) + p3[K_GAMMA];
            const T dg = (-p3[K_G2C2] * q) * tq;
            const T A = -(dzt[qj] * fc3[qk] + dzt[qk] * fc3[qj]) * dg;
            const T cj = A * ri[qj], ck = A * ri[qk];
            const T bj = -dzt[qk] * dfc3[qj] * g;
            const T bk = -dzt[qj] * dfc3[qk] * g;
            // F += c (u_k - cos u_j) + b u_j
            fx[qj].madd2(cj, fmaf_t(-cs, ux[qj], ux[qk]), bj, ux[qj]);
            fy[qj].madd2(cj, fmaf_t(-cs, uy[qj], uy[qk]), bj, uy[qj]);
            fz[qj].madd2(cj, fmaf_t(-cs, uz[qj], uz[qk]), bj, uz[qj]);
            fx[qk].madd2(ck, fmaf_t(-cs, ux[qk], ux[qj]), bk, ux[qk]);
            fy[qk].madd2(ck, fmaf_t(-cs, uy[qk], uy[qj]), bk, uy[qk]);
            fz[qk].madd2(ck, fmaf_t(-cs, uz[qk], uz[qj]), bk, uz[qk]);
          }
      } else
#pragma unroll
      for (int qj = 0; qj < ZC; ++qj) {
        if (qj < z) {
          const T* p2 = srec + rec_off<NS>(ns, ti, tt[qj], tt[qj]);
          const T rij = rr[qj];
          if (rij < p2[K_ROUT2]) {
            // first K loop: zeta_ij and its derivatives (Sec. IV-A)
            T zeta = 0, gjx = 0, gjy = 0, gjz = 0;
            T gkx[ZC], gky[ZC], gkz[ZC];
#pragma unroll
            for (int qk = 0; qk < ZC; ++qk) {
              gkx[qk] = gky[qk] = gkz[qk] = T(0);
              if (qk != qj && qk < z) {
                const T* p3 = srec + rec_off<NS>(ns, ti, tt[qj], tt[qk]);
                const T rik = rr[qk];
                if (rik < p3[K_ROUT3]) {
                  const T cs = ux[qj] * ux[qk] + uy[qj] * uy[qk] + uz[qj] * uz[qk];
                  T zt, A1, A2, A3;
                  triplet<T, LAM3>(p3, rij, rik, cs, zt, A1, A2, A3, rex[qk]);
                  zeta += zt;
                  const T a1j = A1 * ri[qj], a1k = A1 * ri[qk];
                  gjx += a1j * (ux[qk] - cs * ux[qj]) + A2 * ux[qj];
                  gjy += a1j * (uy[qk] - cs * uy[qj]) + A2 * uy[qj];
                  gjz += a1j * (uz[qk] - cs * uz[qj]) + A2 * uz[qj];
                  const T a3 = A3 - A2;
                  gkx[qk] = a1k * (ux[qj] - cs * ux[qk]) + a3 * ux[qk];
                  gky[qk] = a1k * (uy[qj] - cs * uy[qk]) + a3 * uy[qk];
                  gkz[qk] = a1k * (uz[qj] - cs * uz[qk]) + a3 * uz[qk];
                }
              }
            }
            T V, dVdr, dz;
            pair<T>(p2, rij, zeta, V, dVdr, dz, rex[qj]);
            if (EV >= 1) eatom_c.add(V);
            fx[qj].add(-(dVdr * ux[qj] + dz * gjx));
            fy[qj].add(-(dVdr * uy[qj] + dz * gjy));
            fz[qj].add(-(dVdr * uz[qj] + dz * gjz));
#pragma unroll
            for (int qk = 0; qk < ZC; ++qk) {
              if (qk != qj) {
                fx[qk].add(-dz * gkx[qk]);
                fy[qk].add(-dz * gky[qk]);
                fz[qk].add(-dz * gkz[qk]);
              }
            }
          }
        }
      }
      // force on i and virial from the neighbour forces; scatter
      Acc<T, CS> fix, fiy, fiz;
      unsigned long long left = kept;
#pragma unroll
      for (int q = 0; q < ZC; ++q) {
        if (q < z) {
          int sl = q;
          if (filtered) {
            sl = __ffsll(left) - 1;
            left &= left - 1ull;
          }
          fix.sub(fx[q]);
          fiy.sub(fy[q]);
          fiz.sub(fz[q]);
          const T dx = ux[q] * rr[q], dy = uy[q] * rr[q], dz = uz[q] * rr[q];
          if (CS) {
            wa[0].add(dx * fx[q].s + dx * fx[q].lo());
            wa[1].add(dy * fy[q].s + dy * fy[q].lo());
            wa[2].add(dz * fz[q].s + dz * fz[q].lo());
            wa[3].add(dx * fy[q].s + dx * fy[q].lo());
            wa[4].add(dx * fz[q].s + dx * fz[q].lo());
            wa[5].add(dy * fz[q].s + dy * fz[q].lo());
          } else if (EV == 2) {
            w[0] += dx * fx[q].s;
            w[1] += dy * fy[q].s;
            w[2] += dz * fz[q].s;
            w[3] += dx * fy[q].s;
            w[4] += dx * fz[q].s;
            w[5] += dy * fz[q].s;
          }
          if (slots)
            store_slot<T>(a, a.contrib,
                          filtered ? recv_slot(a, sl, i, jj[q]) : (size_t)rv[q] * a.n + jj[q],
                          fx[q].s, fy[q].s, fz[q].s);
          else
            atomic_add3(a.f, jj[q], fx[q].d(), fy[q].d(), fz[q].d());
        }
      }
      if (slots && filtered) {
        // stored entries outside the cutoffs now: their receiving slots get
        // zero, unless they hold zero already (not kept at the last
        // evaluation); kept entries were written above
        unsigned long long clr = a.kmask[i] & ~kept;
        if (z_list < 64) clr &= (1ull << z_list) - 1ull;
        while (clr) {
          const int s = __ffsll(clr) - 1;
          clr &= clr - 1ull;
          store_slot<T>(a, a.contrib, recv_slot(a, s, i, entry_atom(a, a.shortl, s, i)), T(0),
                        T(0), T(0));
        }
        a.kmask[i] = kept;
      } else if (ZC > 4 && slots && z_list > 4) {
        a.kmask[i] = ~0ull;  // every entry written
      }
      if (slots)
        store_slot<T>(a, a.own, (size_t)i, fix.s, fiy.s, fiz.s);
      else
        atomic_add3(a.f, i, fix.d(), fiy.d(), fiz.d());
    }
    if (CS) {
      // the general path's float sums (eatom_i, w) and the fast path's
      // compensated ones (eatom_c, wa), into the thread's double sums
      if (a.eatom) a.eatom[i] = to_f64(eatom_i) + eatom_c.d();
      if (want_acc) {
        sum_add(tsum[0][threadIdx.x], eatom_i);
        sum_add2(tsum[0][threadIdx.x], eatom_c.s, eatom_c.lo());
        for (int q = 0; q < 6; ++q) {
          sum_add(tsum[1 + q][threadIdx.x], w[q]);
          sum_add2(tsum[1 + q][threadIdx.x], wa[q].s, wa[q].lo());
        }
      }
      continue;
    }
    if (EV == 0) continue;
    eatom_i += eatom_c.s;
    if (a.eatom) a.eatom[i] = to_f64(eatom_i);
    if (want_acc) {
      sum_add(tsum[0][threadIdx.x], eatom_i);
      if (EV == 2)
        for (int q = 0; q < 6; ++q) sum_add(tsum[1 + q][threadIdx.x], w[q]);
    }
    if (BATCH)
      for (int q = 0; q < 6; ++q) a.vatom[6 * (size_t)i + q] = to_f64(w[q]);
  }
  if (EV >= 1 && want_acc && __syncthreads_or(any)) block_reduce_sums(&tsum[0][threadIdx.x], a.acc);
  if (a.left_reset) {
    // every block read the leftover count (uni[0]) before taking its ticket
    __syncthreads();
    if (threadIdx.x == 0 && atomicAdd(&a.flags[FLAG_LEFT_TICKET], 1) == (int)gridDim.x - 1) {
      a.flags[FLAG_LEFT] = 0;
      a.flags[FLAG_LEFT_TICKET] = 0;
    }
  }
}

// ---------------------------------------------------------------- wide kernel
// Atoms with many bonds inside the cutoffs (bucket 2: more than 8). One thread
// per atom; the bonds inside the filter radius are formed once into per-thread
// slots in dynamic shared memory (unit vector, length, species, list slot, and
// the force accumulated on that neighbour), and Algorithm 2's loops (zeta
// over k, the pair terms, the three-body forces over k) run over the slots.
// Atoms with more bonds than slots take the general path.
constexpr int WIDE_BLOCK = 64;
constexpr int WIDE_SLOTS = 16;
constexpr int WIDE_WORDS = 10;  // ux uy uz r t s fx fy fz, exact length residual
constexpr size_t wide_slot_bytes(size_t word) {
  return (size_t)WIDE_BLOCK * WIDE_SLOTS * WIDE_WORDS * word;
}

template <class T, int NS, bool LAM3, bool BATCH = false>
__global__ void __launch_bounds__(WIDE_BLOCK) k_tersoff_wide(const __grid_constant__ FwdArgs<T> a) {
  constexpr int SNS = NS > 1 ? NS : (NS == 1 ? 1 : TERSOFF_MAX_SPECIES);
  constexpr int SREC = NS == 1 ? 1 : SNS * SNS * SNS * RSTRIDE;
  __shared__ T srec_s[SREC];
  __shared__ T sfilt[SNS * SNS];
  __shared__ int uni[3];
  extern __shared__ __align__(16) unsigned char wide_dyn[];
  T* sl = reinterpret_cast<T*>(wide_dyn);
  const int ns = NS > 0 ? NS : a.ns;
  if (NS != 1)
    for (int q = threadIdx.x; q < ns * ns * ns * RSTRIDE; q += WIDE_BLOCK) srec_s[q] = a.rec[q];
  __shared__ float snear[SNS * SNS];
  if (threadIdx.x < ns * ns) {
    sfilt[threadIdx.x] = a.filt2[threadIdx.x];
    snear[threadIdx.x] = sizeof(T) == 4 ? a.near2[threadIdx.x] : 0.0f;
  }
  if (threadIdx.x == 0) {
    uni[0] = *a.n_items;
    uni[1] = a.flags[FLAG_REV_MISS];
    uni[2] = a.flags[FLAG_DMAX];
  }
  __syncthreads();
  const T* srec = NS == 1 ? a.prm1 : srec_s;
  const int n_items = uni[0];
  const bool use_short = __int_as_float(uni[2]) <= a.dlim2;
  const bool slots = !a.atomic_mode && use_short && uni[1] == 0;
  // slot q, word f of this thread (thread index innermost: no bank conflicts)
  auto at = [&](int q, int f) -> T& {
    return sl[((size_t)q * WIDE_WORDS + f) * WIDE_BLOCK + threadIdx.x];
  };
  // the atom's own virial sums (float); energy and virial over the thread's
  // atoms in double (only when the reduction is wanted)
  T w[6];
  __shared__ typename SumT<T>::type tsum[7][WIDE_BLOCK];
  const bool want_acc = a.acc != nullptr;
  if (want_acc)
    for (int q = 0; q < 7; ++q) sum_zero(tsum[q][threadIdx.x]);
  bool any = false;
  for (int item = blockIdx.x * WIDE_BLOCK + threadIdx.x; item < n_items;
       item += gridDim.x * WIDE_BLOCK) {
    any = true;
    const int i = a.order[item];
    if (!slots && !a.atomic_mode) clear_slots<T>(a, i);
    Shift<T, BATCH> sh;
    sh.load(a, i);
    for (int q = 0; q < 6; ++q) w[q] = T(0);
    using P = typename SelfPos<T>::type;
    const P pi = self_pos<T>(a, i);
    const int ti = a.types[i];
    const uint32_t* list = use_short ? a.shortl : a.nbr;
    int c = use_short ? a.zcnt[i] : min(a.cnt[i], a.cap);
    bool general = false;
    if (use_short && c > a.zs_cap) {  // short list truncated: the skin list
      list = a.nbr;
      c = min(a.cnt[i], a.cap);
      general = true;
    }
    // bonds inside the filter radius into the slots
    int z = 0;
    if (!general)
      for (int s = 0; s < c && z <= WIDE_SLOTS; ++s) {
        T dx, dy, dz;
        int j, tj;
        Bond<T>::vec(a, sh, pi, list[(size_t)s * a.n + i], dx, dy, dz, j, tj);
        const T r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 <= sfilt[ti * ns + tj])) continue;
        if (z < WIDE_SLOTS) {
          const T r = r2 * M<T>::rsqrt_nr(r2);
          const T ir = T(1) / r;
          at(z, 0) = dx * ir;
          at(z, 1) = dy * ir;
          at(z, 2) = dz * ir;
          at(z, 3) = r;
          at(z, 4) = T(tj);
          at(z, 5) = T(s);
          at(z, 6) = at(z, 7) = at(z, 8) = T(0);
          at(z, 9) = (sizeof(T) == 4 && r2 > snear[ti * ns + tj])
                         ? Exact<T>::residual(a, sh, pi, list[(size_t)s * a.n + i], r)
                         : T(0);
        }
        ++z;
      }
    T eatom_i = T(0);
    if (general || z > WIDE_SLOTS) {
      atomicAdd(&a.flags[FLAG_FALLBACK], 1);
      if (slots && list != a.shortl) {
        atomicOr(&a.flags[FLAG_EXTRA_STICKY], 1);
        zero_stored<T>(a, i, a.zcnt[i]);
      }
      general_atom<T, NS, LAM3, BATCH>(a, sh, srec, i, ti, list, c, slots && list == a.shortl,
                                       false, 0ull, eatom_i, w);
      if (slots && list == a.shortl) a.kmask[i] = ~0ull;  // every entry written
    } else {
      for (int qj = 0; qj < z; ++qj) {
        const T uxj = at(qj, 0), uyj = at(qj, 1), uzj = at(qj, 2), rij = at(qj, 3);
        const int tj = (int)at(qj, 4);
        const T* p2 = srec + rec_off<NS>(ns, ti, tj, tj);
        if (!(rij < p2[K_ROUT2])) continue;
        T zeta = 0;
        for (int qk = 0; qk < z; ++qk) {
          if (qk == qj) continue;
          const T rik = at(qk, 3);
          const T* p3 = srec + rec_off<NS>(ns, ti, tj, (int)at(qk, 4));
          if (!(rik < p3[K_ROUT3])) continue;
          const T cs = uxj * at(qk, 0) + uyj * at(qk, 1) + uzj * at(qk, 2);
          T zt, A1, A2, A3;
          triplet<T, LAM3>(p3, rij, rik, cs, zt, A1, A2, A3, at(qk, 9));
          zeta += zt;
        }
        T V, dVdr, dzv;
        pair<T>(p2, rij, zeta, V, dVdr, dzv, at(qj, 9));
        eatom_i += V;
        T Fjx = -dVdr * uxj, Fjy = -dVdr * uyj, Fjz = -dVdr * uzj;
        const T rinj = T(1) / rij;
        for (int qk = 0; qk < z; ++qk) {
          if (qk == qj) continue;
          const T rik = at(qk, 3);
          const T* p3 = srec + rec_off<NS>(ns, ti, tj, (int)at(qk, 4));
          if (!(rik < p3[K_ROUT3])) continue;
          const T uxk = at(qk, 0), uyk = at(qk, 1), uzk = at(qk, 2);
          const T cs = uxj * uxk + uyj * uyk + uzj * uzk;
          T zt, A1, A2, A3;
          triplet<T, LAM3>(p3, rij, rik, cs, zt, A1, A2, A3, at(qk, 9));
          const T rink = T(1) / rik;
          Fjx -= dzv * (A1 * (uxk - cs * uxj) * rinj + A2 * uxj);
          Fjy -= dzv * (A1 * (uyk - cs * uyj) * rinj + A2 * uyj);
          Fjz -= dzv * (A1 * (uzk - cs * uzj) * rinj + A2 * uzj);
          at(qk, 6) -= dzv * (A1 * (uxj - cs * uxk) * rink + (A3 - A2) * uxk);
          at(qk, 7) -= dzv * (A1 * (uyj - cs * uyk) * rink + (A3 - A2) * uyk);
          at(qk, 8) -= dzv * (A1 * (uzj - cs * uzk) * rink + (A3 - A2) * uzk);
        }
        at(qj, 6) += Fjx;
        at(qj, 7) += Fjy;
        at(qj, 8) += Fjz;
      }
      // forces, virial and the stores of the list's slots
      if (slots) {  // entries outside the cutoffs get zero; the kept ones are overwritten
        for (int s = 0; s < c; ++s)
          store_slot<T>(a, a.contrib, recv_slot(a, s, i, entry_atom(a, list, s, i)), T(0), T(0), T(0));
        a.kmask[i] = ~0ull;
      }
      T fix = 0, fiy = 0, fiz = 0;
      for (int q = 0; q < z; ++q) {
        const T fx = at(q, 6), fy = at(q, 7), fz = at(q, 8);
        fix -= fx;
        fiy -= fy;
        fiz -= fz;
        const T r = at(q, 3);
        const T dx = at(q, 0) * r, dy = at(q, 1) * r, dz = at(q, 2) * r;
        w[0] += dx * fx;
        w[1] += dy * fy;
        w[2] += dz * fz;
        w[3] += dx * fy;
        w[4] += dx * fz;
        w[5] += dy * fz;
        const int s = (int)at(q, 5);
        if (slots) {
          store_slot<T>(a, a.contrib, recv_slot(a, s, i, entry_atom(a, list, s, i)), fx, fy, fz);
        } else {
          int j, ox, oy, oz;
          decode(list[(size_t)s * a.n + i], j, ox, oy, oz);
          atomic_add3(a.f, j, to_f64(fx), to_f64(fy), to_f64(fz));
        }
      }
      if (slots)
        store_slot<T>(a, a.own, (size_t)i, fix, fiy, fiz);
      else
        atomic_add3(a.f, i, to_f64(fix), to_f64(fiy), to_f64(fiz));
    }
    if (a.eatom) a.eatom[i] = to_f64(eatom_i);
    if (want_acc) {
      sum_add(tsum[0][threadIdx.x], eatom_i);
      for (int q = 0; q < 6; ++q) sum_add(tsum[1 + q][threadIdx.x], w[q]);
    }
    if (BATCH)
      for (int q = 0; q < 6; ++q) a.vatom[6 * (size_t)i + q] = to_f64(w[q]);
  }
  if (want_acc && __syncthreads_or(any))
    block_reduce_sums<WIDE_BLOCK>(&tsum[0][threadIdx.x], a.acc);
}

// ---------------------------------------------------------------- fast-forward ablation
// The paper's lane scheme without list filtering (Sec. IV-C, Fig. 2), with the
// vector-wide conditional taken as a warp vote as in its CUDA back-end
// (Sec. VI-B): one lane per centre atom i walks i's full skin list. Each lane
// moves its own J index forward to the next entry inside the pair cutoff while
// the lanes that have found one wait; the body for (i, j) runs once every lane
// of the warp is ready or has finished its list. Both K loops inside the body
// advance the same way, to entries inside the three-body cutoff. Forces go to
// the fallback buffer through FP64 atomics. For measurement only
// (TERSOFF_ABLATE_FASTFWD): the stored short list makes this unnecessary.
template <class T, int NS, bool LAM3>
__global__ void __launch_bounds__(BLOCK) k_tersoff_ffwd(const __grid_constant__ FwdArgs<T> a) {
  constexpr int SNS = NS > 1 ? NS : (NS == 1 ? 1 : TERSOFF_MAX_SPECIES);
  constexpr int SREC = NS == 1 ? 1 : SNS * SNS * SNS * RSTRIDE;
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ T srec_s[SREC];
  __shared__ float snear[SNS * SNS];
  const int ns = NS > 0 ? NS : a.ns;
  if (NS != 1)
    for (int q = threadIdx.x; q < ns * ns * ns * RSTRIDE; q += BLOCK) srec_s[q] = a.rec[q];
  if (threadIdx.x < ns * ns) snear[threadIdx.x] = sizeof(T) == 4 ? a.near2[threadIdx.x] : 0.0f;
  __syncthreads();
  const T* srec = NS == 1 ? a.prm1 : srec_s;
  if (blockIdx.x == 0 && threadIdx.x == 0) a.flags[FLAG_EXTRA] = 1;
  using P = typename SelfPos<T>::type;
  const Shift<T, false> sh;
  T w[6];
  __shared__ typename SumT<T>::type tsum[7][BLOCK];
  for (int q = 0; q < 7; ++q) sum_zero(tsum[q][threadIdx.x]);
  // block-uniform loop: every lane of a warp takes part in every vote
  for (int i0 = blockIdx.x * BLOCK; i0 < a.n; i0 += gridDim.x * BLOCK) {
    const int i = i0 + threadIdx.x;
    const bool have = i < a.n;
    const int ti = have ? a.types[i] : 0;
    const int c = have ? min(a.cnt[i], a.cap) : 0;
    P pi{};
    if (have) {
      pi = self_pos<T>(a, i);
      if (!a.atomic_mode) clear_slots<T>(a, i);
    }
    T eatom_i = 0, fix = 0, fiy = 0, fiz = 0;
    for (int q = 0; q < 6; ++q) w[q] = T(0);
    // bond to the entry in slot s: vector, length, exact residual near a cutoff
    auto bond = [&](int s, T& dx, T& dy, T& dz, T& r, T& rx, int& j, int& tj) {
      const uint32_t e = a.nbr[(size_t)s * a.n + i];
      Bond<T>::vec(a, sh, pi, e, dx, dy, dz, j, tj);
      const T r2 = dx * dx + dy * dy + dz * dz;
      r = r2 * M<T>::rsqrt_nr(r2);
      rx = (sizeof(T) == 4 && r2 > snear[ti * ns + tj]) ? Exact<T>::residual(a, sh, pi, e, r)
                                                         : T(0);
    };
    // J loop: candidate sj is ready when it is inside the pair cutoff or the
    // list is exhausted
    int sj = 0, j = i, tj = 0;
    T dxj = 0, dyj = 0, dzj = 0, rij = 1, rexj = 0;
    auto ready_j = [&]() -> bool {
      if (sj >= c) return true;
      bond(sj, dxj, dyj, dzj, rij, rexj, j, tj);
      return rij < srec[rec_off<NS>(ns, ti, tj, tj) + K_ROUT2];
    };
    bool rj = ready_j();
    while (!__all_sync(FULL, rj))
      if (!rj) {
        ++sj;
        rj = ready_j();
      }
    while (__any_sync(FULL, sj < c)) {
      const bool act = sj < c;
      const T* p2 = srec + rec_off<NS>(ns, ti, tj, tj);
      const T rinj = T(1) / rij;
      const T uxj = dxj * rinj, uyj = dyj * rinj, uzj = dzj * rinj;
      int sk = 0, k = i, tk = 0;
      T dxk = 0, dyk = 0, dzk = 0, rik = 1, rexk = 0;
      auto ready_k = [&]() -> bool {
        if (!act || sk >= c) return true;
        if (sk == sj) return false;
        bond(sk, dxk, dyk, dzk, rik, rexk, k, tk);
        return rik < srec[rec_off<NS>(ns, ti, tj, tk) + K_ROUT3];
      };
      // first K loop: zeta_ij
      T zeta = 0;
      bool rk = ready_k();
      for (;;) {
        while (!__all_sync(FULL, rk))
          if (!rk) {
            ++sk;
            rk = ready_k();
          }
        if (!__any_sync(FULL, act && sk < c)) break;
        if (act && sk < c) {
          const T* p3 = srec + rec_off<NS>(ns, ti, tj, tk);
          const T cs = (dxj * dxk + dyj * dyk + dzj * dzk) * rinj / rik;
          T zt, A1, A2, A3;
          triplet<T, LAM3>(p3, rij, rik, cs, zt, A1, A2, A3, rexk);
          zeta += zt;
        }
        ++sk;
        rk = ready_k();
      }
      T V = 0, dVdr = 0, dz = 0;
      if (act) pair<T>(p2, rij, zeta, V, dVdr, dz, rexj);
      eatom_i += V;
      T Fjx = -dVdr * uxj, Fjy = -dVdr * uyj, Fjz = -dVdr * uzj;
      // second K loop: three-body forces
      sk = 0;
      rk = ready_k();
      for (;;) {
        while (!__all_sync(FULL, rk))
          if (!rk) {
            ++sk;
            rk = ready_k();
          }
        if (!__any_sync(FULL, act && sk < c)) break;
        if (act && sk < c) {
          const T* p3 = srec + rec_off<NS>(ns, ti, tj, tk);
          const T rink = T(1) / rik;
          const T uxk = dxk * rink, uyk = dyk * rink, uzk = dzk * rink;
          const T cs = uxj * uxk + uyj * uyk + uzj * uzk;
          T zt, A1, A2, A3;
          triplet<T, LAM3>(p3, rij, rik, cs, zt, A1, A2, A3, rexk);
          Fjx -= dz * (A1 * (uxk - cs * uxj) * rinj + A2 * uxj);
          Fjy -= dz * (A1 * (uyk - cs * uyj) * rinj + A2 * uyj);
          Fjz -= dz * (A1 * (uzk - cs * uzj) * rinj + A2 * uzj);
          const T Fkx = -dz * (A1 * (uxj - cs * uxk) * rink + (A3 - A2) * uxk);
          const T Fky = -dz * (A1 * (uyj - cs * uyk) * rink + (A3 - A2) * uyk);
          const T Fkz = -dz * (A1 * (uzj - cs * uzk) * rink + (A3 - A2) * uzk);
          atomic_add3(a.f, k, to_f64(Fkx), to_f64(Fky), to_f64(Fkz));
          fix -= Fkx;
          fiy -= Fky;
          fiz -= Fkz;
          w[0] += dxk * Fkx;
          w[1] += dyk * Fky;
          w[2] += dzk * Fkz;
          w[3] += dxk * Fky;
          w[4] += dxk * Fkz;
          w[5] += dyk * Fkz;
        }
        ++sk;
        rk = ready_k();
      }
      if (act) {
        atomic_add3(a.f, j, to_f64(Fjx), to_f64(Fjy), to_f64(Fjz));
        fix -= Fjx;
        fiy -= Fjy;
        fiz -= Fjz;
        w[0] += dxj * Fjx;
        w[1] += dyj * Fjy;
        w[2] += dzj * Fjz;
        w[3] += dxj * Fjy;
        w[4] += dxj * Fjz;
        w[5] += dyj * Fjz;
      }
      // next J candidate, fast-forwarded
      if (act) ++sj;
      rj = ready_j();
      while (!__all_sync(FULL, rj))
        if (!rj) {
          ++sj;
          rj = ready_j();
        }
    }
    if (have) {
      atomic_add3(a.f, i, to_f64(fix), to_f64(fiy), to_f64(fiz));
      if (a.eatom) a.eatom[i] = to_f64(eatom_i);
    }
    sum_add(tsum[0][threadIdx.x], eatom_i);
    for (int q = 0; q < 6; ++q) sum_add(tsum[1 + q][threadIdx.x], w[q]);
  }
  if (a.acc != nullptr) {
    __syncthreads();
    block_reduce_sums(&tsum[0][threadIdx.x], a.acc);
  }
}

}  // namespace fwd
}  // namespace tgb

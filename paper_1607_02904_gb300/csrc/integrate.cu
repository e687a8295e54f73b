// Per-step atom kernels: position packing for the force kernels and the
// velocity-Verlet kick/drift on the FP64 state (x, v, f).
#include "gather.cuh"
#include "internal.cuh"

namespace tgb {
namespace {

// 1.5 * 2^52: adding it to a double of magnitude < 2^51 rounds it to an
// integer held in the low mantissa bits (IEEE-754 binary64 layout).
constexpr double ROUND_MAGIC = 6755399441055744.0;

struct PackArgs {
  int n;
  const double* origin;  // o_i (FP64 path offsets)
  const double* qorg;    // 1.5*2^52 - o_i 2^S
  int4* qref;            // offsets at the build (displacement tracking)
  const int* types;
  int fp64;              // also write FP64 offsets
  int track;             // update the running max displacement
  int build;             // at a build: float offsets and displacement references
  double scale;          // 2^S
  float inv_scale;       // 2^-S
  float4* pos32;
  int4* posq;
  dpos4* pos64;
  int* flags;
};

// Packs atom i (species t) at position (x0, x1, x2); qo: its fixed-point
// origin words; returns its squared displacement since the build (A^2) when
// tracking. Loads are issued before any store.
__device__ __forceinline__ float pack_one(const PackArgs& a, int i, int t, double x0, double x1,
                                          double x2) {
  const double* qo = a.qorg + 3 * (size_t)i;
  const double qo0 = qo[0], qo1 = qo[1], qo2 = qo[2];
  int4 r = make_int4(0, 0, 0, 0);
  if (a.track) r = a.qref[i];
  double o0 = 0.0, o1 = 0.0, o2 = 0.0;
  if (a.fp64) {
    const double* o = a.origin + 3 * (size_t)i;
    o0 = o[0];
    o1 = o[1];
    o2 = o[2];
  }
  // q = round((x - o) 2^S) with one rounding: fma(x, 2^S, magic - o 2^S)
  const long long mb = __double_as_longlong(ROUND_MAGIC);
  const int q0 = (int)(__double_as_longlong(fma(x0, a.scale, qo0)) - mb);
  const int q1 = (int)(__double_as_longlong(fma(x1, a.scale, qo1)) - mb);
  const int q2 = (int)(__double_as_longlong(fma(x2, a.scale, qo2)) - mb);
  a.posq[i] = make_int4(q0, q1, q2, t);
  if (a.build) {
    a.pos32[i] = make_float4((float)q0 * a.inv_scale, (float)q1 * a.inv_scale,
                             (float)q2 * a.inv_scale, __int_as_float(t));
    a.qref[i] = make_int4(q0, q1, q2, t);
  }
  if (a.fp64) a.pos64[i] = dpos4{x0 - o0, x1 - o1, x2 - o2, (double)t};
  float d2 = 0.0f;
  if (a.track) {
    const float d0 = (float)(q0 - r.x) * a.inv_scale;
    const float d1 = (float)(q1 - r.y) * a.inv_scale;
    const float dd = (float)(q2 - r.z) * a.inv_scale;
    d2 = d0 * d0 + d1 * d1 + dd * dd;
  }
  return d2;
}

// block max, one atomic per block (non-negative floats order like their bits)
__device__ __forceinline__ void track_max(const PackArgs& a, float d2) {
  if (!a.track) return;
  __shared__ float wmax[32];
  for (int o = 16; o > 0; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = d2;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wmax[w]);
    atomicMax(&a.flags[FLAG_DMAX], __float_as_int(m));
  }
}

__global__ void k_pack(PackArgs a, const double* __restrict__ x) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float d2 = 0.0f;
  if (i < a.n) {
    const double* xi = x + 3 * (size_t)i;
    d2 = pack_one(a, i, a.types[i], xi[0], xi[1], xi[2]);
  }
  track_max(a, d2);
}

// double -> float rounded to nearest (ties away from zero) through the IEEE-754
// bit layouts, for values in float's normal range (velocities, forces); below
// it gives signed zero. Integer operations only: conversions involving double
// run on GB300's FP64 pipe at 1/62 of the FP32 rate.
__device__ __forceinline__ float d2f_bits(double d) {
  const unsigned long long u = __double_as_longlong(d);
  const unsigned long long mag = (u & 0x7fffffffffffffffull) + 0x10000000ull;  // + half ulp
  const int e = (int)(mag >> 52) - 1023 + 127;
  uint32_t f = ((uint32_t)e << 23) | (uint32_t)((mag >> 29) & 0x7fffffu);
  f = e <= 0 ? 0u : (e >= 255 ? 0x7f800000u : f);
  return __uint_as_float(f | (uint32_t)(u >> 32 & 0x80000000ull));
}

// Block sum of one float per thread, added to dst: compensated float pairs
// over the warp (TwoSum), warp totals carried into double.
__device__ __forceinline__ void block_sum_add_f(float x, double* dst) {
  float s = x, e = 0.0f;
  for (int o = 16; o > 0; o >>= 1) {
    const float os = __shfl_xor_sync(0xffffffffu, s, o);
    const float oe = __shfl_xor_sync(0xffffffffu, e, o);
    const float t = s + os;
    const float bp = t - s;
    e = (e + oe) + ((s - (t - bp)) + (os - bp));
    s = t;
  }
  __shared__ double ws[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) ws[wid] = gather_f2d(s) + gather_f2d(e);
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    atomicAdd(dst, t);
  }
}

__device__ __forceinline__ void block_sum_add(double v, double* dst) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __shared__ double ws[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) ws[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
    atomicAdd(dst, s);
  }
}

// v += kick coef F ; x += dt v ; pack ; optional kinetic energy of the
// previous step ; clear the accumulator for the coming force evaluation.
// F: from f on the first step of a call, gathered from the last force
// evaluation afterwards. All loads of an atom are issued before its stores.
// MG: the instance for the mixed path's gathered steps (gather set, float
// slots with compensated sums), KE its kinetic-energy row; with MG false the
// kernel decides both at run time. The specialised instances carry fewer
// registers.
// snap (first step of a call, MG false; may be null): receives x, v and f as
// read (three n x 3 blocks), the state a rerun of the call starts from.
template <bool MG, bool KE>
__global__ void k_step(PackArgs pk, GatherArgs ga, int gather_, double* __restrict__ x,
                       double* __restrict__ v, const double* __restrict__ f, const __grid_constant__ Coef cf,
                       double dt, int kick, int do_pack, double* ke_row_, double* acc_zero,
                       double* __restrict__ snap) {
  pdl_wait();  // the previous kernel's writes (a launch with launch_pdl)
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int gather = MG ? 1 : gather_;
  double* const ke_row = MG ? (KE ? ke_row_ : nullptr) : ke_row_;
  if (acc_zero && i < 8) acc_zero[i * ACC_STRIDE] = 0.0;
  float d2 = 0.0f;
  double ke = 0.0;   // FP64 path
  float kef = 0.0f;  // mixed path: in float (m v^2 / 2 in amu A^2/ps^2, ~1e1 per atom)
  if (i < pk.n) {
    const int t = pk.types[i];
    const size_t b = 3 * (size_t)i;
    const double x0 = x[b], x1 = x[b + 1], x2 = x[b + 2];
    const double v0 = v[b], v1 = v[b + 1], v2 = v[b + 2];
    double F0, F1, F2;
    float sc[6] = {0, 0, 0, 0, 0, 0};
    const bool mixed = MG || (gather && !ga.fp64 && !ga.atomic_mode);
    if (gather) {
      gather_force(ga, i, F0, F1, F2, mixed ? sc : nullptr);
    } else {
      F0 = f[b];
      F1 = f[b + 1];
      F2 = f[b + 2];
    }
    if (!MG && snap) {
      const size_t m = 3 * (size_t)pk.n;
      snap[b] = x0;
      snap[b + 1] = x1;
      snap[b + 2] = x2;
      snap[m + b] = v0;
      snap[m + b + 1] = v1;
      snap[m + b + 2] = v2;
      snap[2 * m + b] = F0;
      snap[2 * m + b + 1] = F1;
      snap[2 * m + b + 2] = F2;
    }
    const double cu = cf.c[t];
    const double kcu = kick == 2 ? cf.c2[t] : cu;
    double vn0, vn1, vn2;
    if (mixed) {
      // the velocity increment from the float force pair in float (the forces
      // are float-accurate), accumulated into the double velocity; F0..2 hold
      // the (rare) fallback-buffer forces, whose share of the increment is
      // also formed in float (no FP64 operation on the common path)
      const float kf = kick == 2 ? cf.c2f[t] : cf.cf[t];
      float d0 = kf * sc[0] + kf * sc[3];
      float d1 = kf * sc[1] + kf * sc[4];
      float d2v = kf * sc[2] + kf * sc[5];
      const bool extra = ga.flags[FLAG_EXTRA] | ga.flags[FLAG_EXTRA_STICKY];
      if (ke_row) {
        // the previous step's full velocity in float (the kinetic energy is a
        // thermo output; it does not feed the dynamics)
        const float hf = cf.cf[t];
        float w0 = d2f_bits(v0) + (hf * sc[0] + hf * sc[3]);
        float w1 = d2f_bits(v1) + (hf * sc[1] + hf * sc[4]);
        float w2 = d2f_bits(v2) + (hf * sc[2] + hf * sc[5]);
        if (extra) {  // forces scattered through the fallback buffer
          w0 = fmaf(hf, d2f_bits(F0), w0);
          w1 = fmaf(hf, d2f_bits(F1), w1);
          w2 = fmaf(hf, d2f_bits(F2), w2);
        }
        kef = cf.hmf[t] * fmaf(w0, w0, fmaf(w1, w1, w2 * w2));
      }
      if (extra) {
        d0 = fmaf(kf, d2f_bits(F0), d0);
        d1 = fmaf(kf, d2f_bits(F1), d1);
        d2v = fmaf(kf, d2f_bits(F2), d2v);
      }
      vn0 = v0 + gather_f2d(d0);
      vn1 = v1 + gather_f2d(d1);
      vn2 = v2 + gather_f2d(d2v);
    } else {
      if (ke_row) {
        // full-step velocity of the previous step
        const double w0 = fma(cu, F0, v0), w1 = fma(cu, F1, v1), w2 = fma(cu, F2, v2);
        ke = 0.5 * cf.m[t] * fma(w0, w0, fma(w1, w1, w2 * w2));
      }
      vn0 = fma(kcu, F0, v0);
      vn1 = fma(kcu, F1, v1);
      vn2 = fma(kcu, F2, v2);
    }
    const double xn0 = fma(dt, vn0, x0), xn1 = fma(dt, vn1, x1), xn2 = fma(dt, vn2, x2);
    v[b] = vn0;
    v[b + 1] = vn1;
    v[b + 2] = vn2;
    x[b] = xn0;
    x[b + 1] = xn1;
    x[b + 2] = xn2;
    if (do_pack) d2 = pack_one(pk, i, t, xn0, xn1, xn2);
  }
  if (do_pack) track_max(pk, d2);
  if (ke_row) {
    if (MG || (gather && !ga.fp64 && !ga.atomic_mode))
      block_sum_add_f(kef, ke_row);
    else
      block_sum_add(ke, ke_row);
  }
}

// closing half kick with gathered forces, which are also written to f.
// MG: the mixed path's gathered forces (float slots, compensated sums): the
// force is the float pair carried into double (one rounding), the velocity
// increment is formed in float as in k_step, and the kinetic energy in float
// with a compensated block sum; otherwise all in double.
template <bool MG>
__global__ void k_final_kick(GatherArgs ga, const int* __restrict__ types,
                             double* __restrict__ v, double* __restrict__ f, const __grid_constant__ Coef cf,
                             double* ke_row) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (MG) {
    float kef = 0.0f;
    if (i < ga.n) {
      const int t = types[i];
      const size_t b = 3 * (size_t)i;
      const double v0 = v[b], v1 = v[b + 1], v2 = v[b + 2];
      double E0, E1, E2;  // fallback-buffer forces (zero unless flagged)
      float sc[6];
      gather_force(ga, i, E0, E1, E2, sc);
      const bool extra = ga.flags[FLAG_EXTRA] | ga.flags[FLAG_EXTRA_STICKY];
      const float kf = cf.cf[t];
      float d0 = kf * sc[0] + kf * sc[3];
      float d1 = kf * sc[1] + kf * sc[4];
      float d2 = kf * sc[2] + kf * sc[5];
      double F0 = gather_f2d(sc[0]) + gather_f2d(sc[3]);
      double F1 = gather_f2d(sc[1]) + gather_f2d(sc[4]);
      double F2 = gather_f2d(sc[2]) + gather_f2d(sc[5]);
      if (extra) {
        d0 = fmaf(kf, d2f_bits(E0), d0);
        d1 = fmaf(kf, d2f_bits(E1), d1);
        d2 = fmaf(kf, d2f_bits(E2), d2);
        F0 += E0;
        F1 += E1;
        F2 += E2;
      }
      const double w0 = v0 + gather_f2d(d0), w1 = v1 + gather_f2d(d1), w2 = v2 + gather_f2d(d2);
      f[b] = F0;
      f[b + 1] = F1;
      f[b + 2] = F2;
      v[b] = w0;
      v[b + 1] = w1;
      v[b + 2] = w2;
      if (ke_row) {
        const float u0 = d2f_bits(w0), u1 = d2f_bits(w1), u2 = d2f_bits(w2);
        kef = cf.hmf[t] * fmaf(u0, u0, fmaf(u1, u1, u2 * u2));
      }
    }
    if (ke_row) block_sum_add_f(kef, ke_row);
    return;
  }
  double ke = 0.0;
  if (i < ga.n) {
    const int t = types[i];
    const size_t b = 3 * (size_t)i;
    const double v0 = v[b], v1 = v[b + 1], v2 = v[b + 2];
    double F0, F1, F2;
    gather_force(ga, i, F0, F1, F2);
    const double cu = cf.c[t];
    const double w0 = fma(cu, F0, v0), w1 = fma(cu, F1, v1), w2 = fma(cu, F2, v2);
    f[b] = F0;
    f[b + 1] = F1;
    f[b + 2] = F2;
    v[b] = w0;
    v[b + 1] = w1;
    v[b + 2] = w2;
    ke = 0.5 * cf.m[t] * fma(w0, w0, fma(w1, w1, w2 * w2));
  }
  if (ke_row) block_sum_add(ke, ke_row);
}

__global__ void k_gather(GatherArgs ga, double* __restrict__ f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ga.n) return;
  double F[3];
  gather_force(ga, i, F[0], F[1], F[2]);
  f[3 * (size_t)i] = F[0];
  f[3 * (size_t)i + 1] = F[1];
  f[3 * (size_t)i + 2] = F[2];
}

// one block per system: sums of the per-atom energy and virial over the
// system's atom range (fixed order: deterministic)
__global__ void k_system_sums(const int* __restrict__ off, const double* __restrict__ eatom,
                              const double* __restrict__ vatom, double* __restrict__ energy,
                              double* __restrict__ virial) {
  const int sys = blockIdx.x;
  const int a0 = off[sys], a1 = off[sys + 1];
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int i = a0 + threadIdx.x; i < a1; i += blockDim.x) {
    v[0] += eatom[i];
    for (int q = 0; q < 6; ++q) v[1 + q] += vatom[6 * (size_t)i + q];
  }
  __shared__ double part[7][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = 0; q < 7; ++q) {
    double t = v[q];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) part[q][wid] = t;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[threadIdx.x][w];
    if (threadIdx.x == 0) {
      if (energy) energy[sys] = t;
    } else if (virial) {
      virial[6 * (size_t)sys + threadIdx.x - 1] = t;
    }
  }
}

// one thread: rebuild when the running max squared displacement (float bits,
// non-negative) exceeds lim2
__global__ void k_decide_rebuild(int* flags, float lim2, cudaGraphConditionalHandle h) {
  const bool go = __int_as_float(flags[FLAG_DMAX]) > lim2;
  if (go) flags[FLAG_NREBUILD] += 1;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

// rows: ACC_LEN doubles per step (energy, virial[6], kinetic in mass units)
__global__ void k_thermo_rows(const double* rows, int nsteps, double mvv2e, double* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsteps) return;
  const double pe = rows[ACC_LEN * (size_t)s];
  const double ke = rows[ACC_LEN * (size_t)s + 7 * ACC_STRIDE] * mvv2e;
  out[3 * (size_t)s + 0] = pe;
  out[3 * (size_t)s + 1] = ke;
  out[3 * (size_t)s + 2] = pe + ke;
}

PackArgs make_pack(Ctx* c, bool track, bool build = false) {
  PackArgs a;
  a.n = c->n;
  a.origin = c->d_origin;
  a.qorg = c->d_qorg;
  a.qref = c->d_qref;
  a.types = c->d_types;
  a.fp64 = c->precision == TERSOFF_FP64;
  a.track = track ? 1 : 0;
  a.build = build ? 1 : 0;
  a.scale = ldexp(1.0, c->grid.fix_shift);
  a.inv_scale = ldexpf(1.0f, -c->grid.fix_shift);
  a.pos32 = c->d_pos32;
  a.posq = c->d_posq;
  a.pos64 = c->d_pos64;
  a.flags = c->d_flags;
  return a;
}

}  // namespace

int launch_pack_positions(Ctx* c, const double* x, bool build, cudaStream_t s) {
  if (c->n == 0) return TERSOFF_OK;
  const int B = c->opt_block;
  TGB_CUDA(c, launch_pdl(k_pack, (c->n + B - 1) / B, B, 0, s, make_pack(c, !build, build), x));
  c->launches++;
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

int launch_md_step(Ctx* c, double* x, double* v, double* f, double dt, int kick, bool pack,
                   double* ke_row, double* acc_zero, cudaStream_t s, double* snap) {
  const int B = c->opt_block;
  const GatherArgs ga = make_gather(c);
  const int grid = (c->n + B - 1) / B;
  if (kick == 2 && !ga.fp64 && !ga.atomic_mode) {
    if (ke_row)
      TGB_CUDA(c, launch_pdl(k_step<true, true>, grid, B, 0, s, make_pack(c, true), ga, 1, x, v,
                             f, c->coef, dt, kick, pack ? 1 : 0, ke_row, acc_zero,
                             (double*)nullptr));
    else
      TGB_CUDA(c, launch_pdl(k_step<true, false>, grid, B, 0, s, make_pack(c, true), ga, 1, x, v,
                             f, c->coef, dt, kick, pack ? 1 : 0, (double*)nullptr, acc_zero,
                             (double*)nullptr));
  } else {
    TGB_CUDA(c, launch_pdl(k_step<false, false>, grid, B, 0, s, make_pack(c, true), ga,
                           kick == 2 ? 1 : 0, x, v, f, c->coef, dt, kick, pack ? 1 : 0, ke_row,
                           acc_zero, snap));
  }
  c->launches++;
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

int launch_final_kick(Ctx* c, double* v, double* f, double* ke_row, cudaStream_t s) {
  const int B = c->opt_block;
  const GatherArgs ga = make_gather(c);
  if (!ga.fp64 && !ga.atomic_mode)
    TGB_CUDA(c, launch_pdl(k_final_kick<true>, (c->n + B - 1) / B, B, 0, s, ga, c->d_types, v, f, c->coef, ke_row));
  else
    TGB_CUDA(c, launch_pdl(k_final_kick<false>, (c->n + B - 1) / B, B, 0, s, ga, c->d_types, v, f, c->coef, ke_row));
  c->launches++;
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

int launch_gather(Ctx* c, double* f, cudaStream_t s) {
  if (c->n == 0) return TERSOFF_OK;
  const int B = c->opt_block;
  k_gather<<<(c->n + B - 1) / B, B, 0, s>>>(make_gather(c), f);
  c->launches++;
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

int launch_system_sums(Ctx* c, double* energy, double* virial, cudaStream_t s) {
  if (c->n_sys <= 0) return TERSOFF_OK;
  k_system_sums<<<c->n_sys, 256, 0, s>>>(c->d_sys_off, c->d_eatom, c->d_vatom, energy, virial);
  c->launches++;
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

int launch_decide_rebuild(Ctx* c, float lim2, cudaGraphConditionalHandle h, cudaStream_t s) {
  k_decide_rebuild<<<1, 1, 0, s>>>(c->d_flags, lim2, h);
  c->launches++;
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

int launch_thermo_rows(Ctx* c, const double* rows, int nsteps, double mvv2e, double* thermo,
                       cudaStream_t s) {
  if (nsteps <= 0) return TERSOFF_OK;
  k_thermo_rows<<<(nsteps + 127) / 128, 128, 0, s>>>(rows, nsteps, mvv2e, thermo);
  c->launches++;
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

}  // namespace tgb

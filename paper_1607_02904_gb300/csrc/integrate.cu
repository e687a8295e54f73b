// Per-step atom kernels: position packing for the force kernels and the
// velocity-Verlet kick/drift on the FP64 state (x, v, f).
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

// Packs atom i at position (x0, x1, x2); returns its squared displacement
// since the build (A^2) when tracking.
__device__ __forceinline__ float pack_one(const PackArgs& a, int i, double x0, double x1,
                                          double x2) {
  const double* qo = a.qorg + 3 * (size_t)i;
  const int t = a.types[i];
  // q = round((x - o) 2^S) with one rounding: fma(x, 2^S, magic - o 2^S)
  const long long mb = __double_as_longlong(ROUND_MAGIC);
  const int q0 = (int)(__double_as_longlong(fma(x0, a.scale, qo[0])) - mb);
  const int q1 = (int)(__double_as_longlong(fma(x1, a.scale, qo[1])) - mb);
  const int q2 = (int)(__double_as_longlong(fma(x2, a.scale, qo[2])) - mb);
  a.posq[i] = make_int4(q0, q1, q2, t);
  if (a.build) {
    a.pos32[i] = make_float4((float)q0 * a.inv_scale, (float)q1 * a.inv_scale,
                             (float)q2 * a.inv_scale, __int_as_float(t));
    a.qref[i] = make_int4(q0, q1, q2, t);
  }
  if (a.fp64) {
    const double* o = a.origin + 3 * (size_t)i;
    a.pos64[i] = dpos4{x0 - o[0], x1 - o[1], x2 - o[2], (double)t};
  }
  float d2 = 0.0f;
  if (a.track) {
    const int4 r = a.qref[i];
    const float d0 = (float)(q0 - r.x) * a.inv_scale;
    const float d1 = (float)(q1 - r.y) * a.inv_scale;
    const float dd = (float)(q2 - r.z) * a.inv_scale;
    d2 = d0 * d0 + d1 * d1 + dd * dd;
  }
  return d2;
}

// warp max, one atomic per warp (non-negative floats order like their bits)
__device__ __forceinline__ void track_max(const PackArgs& a, float d2) {
  if (!a.track) return;
  for (int o = 16; o > 0; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&a.flags[FLAG_DMAX], __float_as_int(d2));
}

__global__ void k_pack(PackArgs a, const double* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float d2 = 0.0f;
  if (i < a.n) {
    const double* xi = x + 3 * (size_t)i;
    d2 = pack_one(a, i, xi[0], xi[1], xi[2]);
  }
  track_max(a, d2);
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

// v += kick coef f ; x += dt v ; f = 0 ; pack ; optional kinetic energy of the
// previous step ; clear the accumulator for the coming force evaluation
__global__ void k_step(PackArgs pk, double* __restrict__ x, double* __restrict__ v,
                       double* __restrict__ f, const double* __restrict__ coef, double dt,
                       double kick, int do_pack, double* ke_row, double* acc_zero) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (acc_zero && i < 8) acc_zero[i] = 0.0;
  float d2 = 0.0f;
  double ke = 0.0;
  if (i < pk.n) {
    const int t = pk.types[i];
    const double c = coef[t];
    double xn[3];
    for (int a = 0; a < 3; ++a) {
      const size_t k = 3 * (size_t)i + a;
      const double fk = f[k];
      const double vk = v[k];
      if (ke_row) {
        const double vf = fma(c, fk, vk);  // full-step velocity of the previous step
        ke = fma(vf, vf, ke);
      }
      const double vv = fma(kick * c, fk, vk);
      v[k] = vv;
      xn[a] = fma(dt, vv, x[k]);
      x[k] = xn[a];
      f[k] = 0.0;
    }
    if (ke_row) ke *= 0.5 * coef[TERSOFF_MAX_SPECIES + t];
    if (do_pack) d2 = pack_one(pk, i, xn[0], xn[1], xn[2]);
  }
  if (do_pack) track_max(pk, d2);
  if (ke_row) block_sum_add(ke, ke_row);
}

__global__ void k_final_kick(int n, const int* __restrict__ types, double* __restrict__ v,
                             const double* __restrict__ f, const double* __restrict__ coef,
                             double* ke_row) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double ke = 0.0;
  if (i < n) {
    const int t = types[i];
    const double c = coef[t];
    for (int a = 0; a < 3; ++a) {
      const size_t k = 3 * (size_t)i + a;
      const double vv = fma(c, f[k], v[k]);
      v[k] = vv;
      ke = fma(vv, vv, ke);
    }
    ke *= 0.5 * coef[TERSOFF_MAX_SPECIES + t];
  }
  if (ke_row) block_sum_add(ke, ke_row);
}

// rows: 8 doubles per step (energy, virial[6], kinetic in mass units)
__global__ void k_thermo_rows(const double* rows, int nsteps, double mvv2e, double* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsteps) return;
  const double pe = rows[8 * (size_t)s];
  const double ke = rows[8 * (size_t)s + 7] * mvv2e;
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
  k_pack<<<(c->n + 255) / 256, 256, 0, s>>>(make_pack(c, !build, build), x);
  c->launches++;
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

int launch_md_step(Ctx* c, double* x, double* v, double* f, const double* coef, double dt,
                   int kick, bool pack, double* ke_row, double* acc_zero, cudaStream_t s) {
  k_step<<<(c->n + 255) / 256, 256, 0, s>>>(make_pack(c, true), x, v, f, coef, dt,
                                            (double)kick, pack ? 1 : 0, ke_row, acc_zero);
  c->launches++;
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

int launch_final_kick(Ctx* c, double* v, const double* f, const double* coef, double* ke_row,
                      cudaStream_t s) {
  k_final_kick<<<(c->n + 255) / 256, 256, 0, s>>>(c->n, c->d_types, v, f, coef, ke_row);
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

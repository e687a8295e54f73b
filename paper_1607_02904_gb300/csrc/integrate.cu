// Per-step atom kernels: position packing for the force kernels and the
// velocity-Verlet kick/drift (FP64 state: x, v, f).
#include "internal.cuh"

namespace tgb {
namespace {

// 1.5 * 2^52: adding it to a double of magnitude < 2^51 rounds it to an
// integer held in the low mantissa bits (IEEE-754 binary64 layout).
constexpr double ROUND_MAGIC = 6755399441055744.0;

struct PackArgs {
  int n;
  const double* x;
  const double* origin;
  const int* types;
  int precision;
  double scale;      // 2^fix_shift
  float inv_scale;   // 2^-fix_shift
  float4* pos32;
  int4* posq;
  dpos4* pos64;
};

__device__ __forceinline__ void pack_one(const PackArgs& a, int i, double x0, double x1,
                                         double x2) {
  const double* o = a.origin + 3 * (size_t)i;
  const int t = a.types[i];
  if (a.precision == TERSOFF_MIXED) {
    // q = round((x - o) * 2^S): one rounding, exact integer differences later
    long long b0 = __double_as_longlong(fma(x0 - o[0], a.scale, ROUND_MAGIC));
    long long b1 = __double_as_longlong(fma(x1 - o[1], a.scale, ROUND_MAGIC));
    long long b2 = __double_as_longlong(fma(x2 - o[2], a.scale, ROUND_MAGIC));
    const long long mb = __double_as_longlong(ROUND_MAGIC);
    int q0 = (int)(b0 - mb), q1 = (int)(b1 - mb), q2 = (int)(b2 - mb);
    a.posq[i] = make_int4(q0, q1, q2, t);
    a.pos32[i] = make_float4((float)q0 * a.inv_scale, (float)q1 * a.inv_scale,
                             (float)q2 * a.inv_scale, __int_as_float(t));
  } else {
    a.pos64[i] = dpos4{x0 - o[0], x1 - o[1], x2 - o[2], (double)t};
  }
}

__global__ void k_pack(PackArgs a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const double* x = a.x + 3 * (size_t)i;
  pack_one(a, i, x[0], x[1], x[2]);
}

// v += c_t f ; x += dt v ; f = 0 ; optionally pack positions; block 0 clears acc
__global__ void k_kick_drift(int n, double* __restrict__ x, double* __restrict__ v,
                             double* __restrict__ f, const int* __restrict__ types,
                             const double* __restrict__ cdt, double dt, double* acc,
                             int do_pack, PackArgs pk) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0)
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
  if (i >= n) return;
  const double c = cdt[types[i]];
  double xn[3];
  for (int a = 0; a < 3; ++a) {
    size_t k = 3 * (size_t)i + a;
    double vv = fma(c, f[k], v[k]);
    v[k] = vv;
    xn[a] = fma(dt, vv, x[k]);
    x[k] = xn[a];
    f[k] = 0.0;
  }
  if (do_pack) pack_one(pk, i, xn[0], xn[1], xn[2]);
}

// v += c_t f ; accumulate kinetic energy (sum m v^2 / 2) into acc[7]
__global__ void k_kick(int n, double* __restrict__ v, const double* __restrict__ f,
                       const int* __restrict__ types, const double* __restrict__ cdt,
                       const double* __restrict__ mass, double* acc, int want_ke) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double ke = 0.0;
  if (i < n) {
    const int t = types[i];
    const double c = cdt[t];
    for (int a = 0; a < 3; ++a) {
      size_t k = 3 * (size_t)i + a;
      double vv = fma(c, f[k], v[k]);
      v[k] = vv;
      ke = fma(vv, vv, ke);
    }
    ke *= 0.5 * mass[t];
  }
  if (!want_ke) return;
  // block reduction in double (one value per atom, once per step)
  for (int o = 16; o > 0; o >>= 1) ke += __shfl_xor_sync(0xffffffffu, ke, o);
  __shared__ double ws[32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) ws[wid] = ke;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
    atomicAdd(&acc[7], s);
  }
}

// thermo row: potential, kinetic (converted to eV), total
__global__ void k_thermo(const double* acc, double mvv2e, double* row) {
  double pe = acc[0];
  double ke = acc[7] * mvv2e;
  row[0] = pe;
  row[1] = ke;
  row[2] = pe + ke;
}

__global__ void k_zero(double* p, size_t m) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < m) p[i] = 0.0;
}

PackArgs make_pack(Ctx* c, const double* x) {
  PackArgs a;
  a.n = c->n;
  a.x = x;
  a.origin = c->d_origin;
  a.types = c->d_types;
  a.precision = c->precision;
  a.scale = ldexp(1.0, c->grid.fix_shift);
  a.inv_scale = ldexpf(1.0f, -c->grid.fix_shift);
  a.pos32 = c->d_pos32;
  a.posq = c->d_posq;
  a.pos64 = c->d_pos64;
  return a;
}

}  // namespace

int launch_pack_positions(Ctx* c, const double* x, cudaStream_t s) {
  if (c->n == 0) return TERSOFF_OK;
  k_pack<<<(c->n + 255) / 256, 256, 0, s>>>(make_pack(c, x));
  c->launches++;
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

int launch_kick_drift(Ctx* c, double* x, double* v, double* f, const double* cdt, double dt,
                      bool pack, cudaStream_t s) {
  k_kick_drift<<<(c->n + 255) / 256, 256, 0, s>>>(c->n, x, v, f, c->d_types, cdt, dt,
                                                  c->d_acc, pack ? 1 : 0, make_pack(c, x));
  c->launches++;
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

int launch_kick(Ctx* c, double* v, const double* f, const double* cdt, const double* mass,
                bool want_ke, cudaStream_t s) {
  k_kick<<<(c->n + 255) / 256, 256, 0, s>>>(c->n, v, f, c->d_types, cdt, mass, c->d_acc,
                                            want_ke ? 1 : 0);
  c->launches++;
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

int launch_thermo(Ctx* c, double mvv2e, double* row, cudaStream_t s) {
  k_thermo<<<1, 1, 0, s>>>(c->d_acc, mvv2e, row);
  c->launches++;
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

int launch_zero(Ctx* c, double* p, size_t count, cudaStream_t s) {
  if (count == 0) return TERSOFF_OK;
  k_zero<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(p, count);
  c->launches++;
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

}  // namespace tgb

// Ghost-shell packing of the slab decomposition on the device: the data-parallel
// layout of the paper's multi-node runs (Sec. V), where each rank owns a slab
// of the cell and receives the atoms within the ghost width of its two faces
// from its neighbours.
//
// For one rank's owned atoms the three kernels below write
//   - the owned positions in the rank's local frame (the cut-axis coordinate
//     wrapped into [0, L), minus the frame origin),
//   - the lower face set (wrapped u with u - lo < r_ghost) and the upper face
//     set (hi - u <= r_ghost), each shifted across the periodic boundary where
//     it wraps and placed in the receiving neighbour's local frame,
//     with species and global indices, in ascending owned index,
// so that the receiver can take the buffers as they arrive, after its own
// atoms, with no further arithmetic. The order is deterministic: a count per
// block, an exclusive scan over the blocks, and a block-level scan of the
// selection flags place every selected atom.
#include <cmath>

#include "internal.cuh"

namespace tgb {
namespace {

constexpr int HB = 256;         // threads per block
constexpr int HI = 4;           // owned atoms per thread (consecutive)
constexpr int HTILE = HB * HI;  // owned atoms per block

struct HaloGeo {
  int n, axis, cap;
  double L, lo, hi, rg, frame, shift[2], frame_to[2];
};

// cut-axis coordinate wrapped into [0, L): the remainder of x / L (exact),
// moved up by L when negative, +0 for a zero remainder, and L itself mapped
// to 0
__device__ __forceinline__ double wrap_axis(double x, double L) {
  double u = fmod(x, L);
  if (u != 0.0) {
    if (u < 0.0) u += L;
  } else {
    u = 0.0;
  }
  return u >= L ? u - L : u;
}

__device__ __forceinline__ void flags_of(const HaloGeo& g, double u, bool& lower, bool& upper) {
  lower = u - g.lo < g.rg;
  upper = g.hi - u <= g.rg;
}

// per block: how many of its atoms each face set takes
__global__ void k_halo_count(HaloGeo g, const double* __restrict__ x, int* __restrict__ bcount) {
  const int base = blockIdx.x * HTILE + threadIdx.x * HI;
  int cl = 0, cu = 0;
  for (int q = 0; q < HI; ++q) {
    const int i = base + q;
    if (i < g.n) {
      bool lw, up;
      flags_of(g, wrap_axis(x[3 * (size_t)i + g.axis], g.L), lw, up);
      cl += lw;
      cu += up;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    cl += __shfl_xor_sync(0xffffffffu, cl, o);
    cu += __shfl_xor_sync(0xffffffffu, cu, o);
  }
  __shared__ int wl[HB / 32], wu[HB / 32];
  if ((threadIdx.x & 31) == 0) {
    wl[threadIdx.x >> 5] = cl;
    wu[threadIdx.x >> 5] = cu;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0, b = 0;
    for (int w = 0; w < HB / 32; ++w) {
      a += wl[w];
      b += wu[w];
    }
    bcount[blockIdx.x] = a;
    bcount[gridDim.x + blockIdx.x] = b;
  }
}

// block-wide exclusive scan of one int per thread (wsum: one int per warp)
__device__ __forceinline__ int block_excl(int v, int* wsum) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  int off = 0;
  for (int w = 0; w < wid; ++w) off += wsum[w];
  __syncthreads();
  return off + incl - v;
}

// one block of 1024 threads: exclusive scan of both count rows in place (each
// thread takes a run of consecutive blocks); totals to counts
__global__ void k_halo_scan(int nb, int* __restrict__ bcount, int* __restrict__ counts) {
  __shared__ int wsum[32];
  const int per = (nb + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per;
  for (int set = 0; set < 2; ++set) {
    int* row = bcount + (size_t)set * nb;
    int sum = 0;
    for (int k = 0; k < per; ++k)
      if (b0 + k < nb) sum += row[b0 + k];
    int run = block_excl(sum, wsum);
    if (threadIdx.x == blockDim.x - 1) counts[set] = run + sum;
    for (int k = 0; k < per; ++k)
      if (b0 + k < nb) {
        const int v = row[b0 + k];
        row[b0 + k] = run;
        run += v;
      }
  }
}

__global__ void k_halo_write(HaloGeo g, const double* __restrict__ x, const int* __restrict__ types,
                             const long long* __restrict__ ids, const int* __restrict__ bscan,
                             double* __restrict__ x_local, double* __restrict__ send_x,
                             int* __restrict__ send_t, long long* __restrict__ send_id) {
  __shared__ int wsum[HB / 32];
  const int base = blockIdx.x * HTILE + threadIdx.x * HI;
  double u[HI];
  bool lw[HI], up[HI];
  int cl = 0, cu = 0;
  for (int q = 0; q < HI; ++q) {
    const int i = base + q;
    u[q] = 0.0;
    lw[q] = up[q] = false;
    if (i < g.n) {
      u[q] = wrap_axis(x[3 * (size_t)i + g.axis], g.L);
      flags_of(g, u[q], lw[q], up[q]);
    }
    cl += lw[q];
    cu += up[q];
  }
  int pl = block_excl(cl, wsum) + bscan[blockIdx.x];
  int pu = block_excl(cu, wsum) + bscan[gridDim.x + blockIdx.x];
  for (int q = 0; q < HI; ++q) {
    const int i = base + q;
    if (i >= g.n) break;
    const double* xi = x + 3 * (size_t)i;
    double p[3] = {xi[0], xi[1], xi[2]};
    p[g.axis] = u[q] - g.frame;
    for (int a = 0; a < 3; ++a) x_local[3 * (size_t)i + a] = p[a];
    for (int set = 0; set < 2; ++set) {
      const bool sel = set == 0 ? lw[q] : up[q];
      if (!sel) continue;
      const int k = set == 0 ? pl++ : pu++;
      if (k >= g.cap) continue;
      const size_t o = (size_t)set * g.cap + k;
      double s[3] = {xi[0], xi[1], xi[2]};
      s[g.axis] = (u[q] + g.shift[set]) - g.frame_to[set];
      for (int a = 0; a < 3; ++a) send_x[3 * o + a] = s[a];
      send_t[o] = types[i];
      send_id[o] = ids[i];
    }
  }
}

}  // namespace

int launch_halo_pack(Ctx* c, const double* x, const int* types, const long long* ids, int n,
                     int axis, const double* geo, int cap, double* x_local, double* send_x,
                     int* send_t, long long* send_id, int* counts, cudaStream_t s) {
  HaloGeo g;
  g.n = n;
  g.axis = axis;
  g.cap = cap;
  g.L = geo[0];
  g.lo = geo[1];
  g.hi = geo[2];
  g.rg = geo[3];
  g.frame = geo[4];
  g.shift[0] = geo[5];
  g.frame_to[0] = geo[6];
  g.shift[1] = geo[7];
  g.frame_to[1] = geo[8];
  const int nb = (n + HTILE - 1) / HTILE;
  if (nb == 0) {
    TGB_CUDA(c, cudaMemsetAsync(counts, 0, 2 * sizeof(int), s));
    return TERSOFF_OK;
  }
  int* bcount = nullptr;
  TGB_CUDA(c, cudaMallocAsync(&bcount, 2 * sizeof(int) * (size_t)nb, s));
  k_halo_count<<<nb, HB, 0, s>>>(g, x, bcount);
  k_halo_scan<<<1, 1024, 0, s>>>(nb, bcount, counts);
  k_halo_write<<<nb, HB, 0, s>>>(g, x, types, ids, bcount, x_local, send_x, send_t, send_id);
  c->launches += 3;
  const cudaError_t e = cudaGetLastError();
  TGB_CUDA(c, cudaFreeAsync(bcount, s));
  TGB_CUDA(c, e);
  return TERSOFF_OK;
}

}  // namespace tgb

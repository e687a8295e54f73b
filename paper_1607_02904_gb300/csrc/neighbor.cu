// Cell-binned full neighbour lists (Sec. II Eq. 4; skin of Sec. III).
//
// Pipeline, all on the caller's stream:
//   k_bin      atom -> cell (wrapped position), per-atom origin o_i, FP32 offset
//   scan       exclusive prefix sum of cell counts (three kernels)
//   k_scatter  atoms grouped by cell
//   k_neigh    one thread per atom scans the 27 stencil cells; candidates far from
//              the cutoff are classified in FP32 from cell-relative offsets, those
//              within a safety band of it by the exact FP64 minimum-image test
//              (same operation sequence as the definition); entries are then
//              sorted by neighbour index.
// An entry stores j and the stencil cell offset; with u_i = x_i - o_i the bond
// vector is  x_j(image) - x_i = (u_j - u_i) + off * h.
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace tgb {
namespace {

constexpr int SCAN_BLOCK = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

GridDev to_dev(const Grid& g) {
  GridDev d;
  d.cell_base = 0;
  for (int a = 0; a < 3; ++a) {
    d.nc[a] = g.nc[a];
    d.L[a] = g.L[a];
    d.invL[a] = g.invL[a];
    d.h[a] = g.h[a];
    d.invh[a] = g.invh[a];
    d.hf[a] = (float)g.h[a];
  }
  return d;
}

// BATCH: every atom uses the grid of its system (geo[atom_sys[i]]), whose
// cells are numbered from its cell_base; otherwise the launch-wide grid g1
// (a kernel parameter, read in place).
template <bool BATCH>
__device__ __forceinline__ const GridDev& grid_of(const GridDev& g1,
                                                  const GridDev* __restrict__ geo,
                                                  const int* __restrict__ atom_sys, int i) {
  if constexpr (BATCH)
    return geo[atom_sys[i]];
  else
    return g1;
}

template <bool BATCH>
__global__ void k_bin(int n, const double* __restrict__ x, const __grid_constant__ GridDev g1,
                      const GridDev* __restrict__ geo, const int* __restrict__ atom_sys,
                      double scale, int* __restrict__ cell_of, int* __restrict__ cell_count,
                      double* __restrict__ origin, double* __restrict__ qorg,
                      int* __restrict__ flags) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const GridDev& g = grid_of<BATCH>(g1, geo, atom_sys, i);
  int c3[3];
  bool finite = true;
  for (int a = 0; a < 3; ++a) {
    double xa = x[3 * (size_t)i + a];
    if (!isfinite(xa)) {
      finite = false;
      xa = 0.0;
    }
    // periodic image k = floor(x / L) and the wrapped coordinate w; inside
    // the box (0 <= x/L < 1, tested on the bits of the double: no FP64
    // operation) k = 0 and w = x, the values the general formulas give there
    const double u = xa * g.invL[a];
    const long long ub = __double_as_longlong(u);
    // origin o = image corner of the cell; offsets x - o start inside the cell
    int c;
    double o;
    if (ub >= 0 && ub < 0x3FF0000000000000ll) {
      c = (int)(xa * g.invh[a]);
      c = c < 0 ? 0 : (c >= g.nc[a] ? g.nc[a] - 1 : c);
      o = c * g.h[a];  // = fma(0, L, c h)
    } else {
      const double k = floor(u);
      const double w = xa - g.L[a] * k;
      c = (int)(w * g.invh[a]);
      c = c < 0 ? 0 : (c >= g.nc[a] ? g.nc[a] - 1 : c);
      o = fma(k, g.L[a], c * g.h[a]);
    }
    origin[3 * (size_t)i + a] = o;
    qorg[3 * (size_t)i + a] = 6755399441055744.0 - o * scale;
    c3[a] = c;
  }
  if (!finite) atomicOr(&flags[FLAG_NONFINITE], 1);
  int cell = g.cell_base + (c3[2] * g.nc[1] + c3[1]) * g.nc[0] + c3[0];
  cell_of[i] = cell;
  atomicAdd(&cell_count[cell], 1);
}

// Binning of a single system by table lookups. Per axis a, with C(x) the cell
// index (int)(x / h) of k_bin and U(x) = x / L (both rounded double products,
// non-decreasing in x), the host tabulates
//   t[0]        the smallest double x >= 0 with U(x) >= 1: an atom is inside
//               the box (the test of k_bin) when 0 <= bits(x) < bits(t[0]);
//   t[c]        for 1 <= c < nc, the smallest double x with C(x) >= c: inside
//               the box the cell is the c with t[c] <= x < t[c + 1];
//   t[BT_O + c] the origin c h, and t[BT_Q + c] the fixed-point origin
//               1.5 2^52 - c h 2^S, by the double operations of k_bin (c h 2^S
//               is exact, so the fused and unfused forms agree).
// Non-negative doubles order like their bit patterns, so the tests are
// integer comparisons; k_bin's FP64 arithmetic remains for atoms outside the
// box. The build's position pack (fixed-point, float and FP64 offsets,
// displacement references) is fused in.
constexpr int BT_O = 1024;
constexpr int BT_Q = 2048;
constexpr int BT_AXIS = 3072;  // 64-bit words per axis (nc <= 1024)

struct BinPack {
  const long long* tab;  // 3 x BT_AXIS words
  float invhf[3];        // float(1 / h): the estimate the thresholds correct
  double scale;          // 2^S
  float inv_scale;       // 2^-S
  const int* types;
  int4* posq;
  float4* pos32;
  int4* qref;
  dpos4* pos64;  // FP64 path only, else null
  unsigned long long* kmask;  // set to all ones (every slot may hold a stale force)
};

__global__ void k_bin_pack(int n, const double* __restrict__ x, const __grid_constant__ GridDev g,
                           const __grid_constant__ BinPack bp, int* __restrict__ cell_of,
                           int* __restrict__ cell_count, double* __restrict__ origin,
                           double* __restrict__ qorg, int* __restrict__ flags) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int t = bp.types[i];
  int c3[3], q3[3];
  double xr[3], o3[3], qo3[3];
  long long xb3[3], lo3[3], hi3[3];
  bool inb[3];
  bool finite = true;
  const long long mb = __double_as_longlong(6755399441055744.0);
  // per axis: the bits of x, the inside-the-box test and a float estimate of
  // the cell (truncated from the bits); then, for the three axes together, the
  // estimated cell's thresholds and origins (one round of independent loads)
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double x_in = x[3 * (size_t)i + a];
    xr[a] = x_in;
    long long xb = __double_as_longlong(x_in);
    if ((xb & 0x7ff0000000000000ll) == 0x7ff0000000000000ll) {
      finite = false;
      xb = 0;  // binned as x = 0
    }
    xb3[a] = xb;
    const long long* tb = bp.tab + a * BT_AXIS;
    inb[a] = xb >= 0 && xb < __ldg(&tb[0]);
    const int e = (int)(xb >> 52) - 1023 + 127;
    const float xf = __uint_as_float(
        e <= 0 ? 0u : (((uint32_t)e << 23) | (uint32_t)((xb >> 29) & 0x7fffff)));
    int c = (int)(xf * bp.invhf[a]);
    c = c < 0 ? 0 : (c >= g.nc[a] ? g.nc[a] - 1 : c);
    c3[a] = c;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const long long* tb = bp.tab + a * BT_AXIS;
    const int c = c3[a];
    lo3[a] = __ldg(&tb[c]);      // threshold of cell c (c > 0)
    hi3[a] = __ldg(&tb[c + 1]);  // of cell c + 1 (c + 1 < nc; otherwise an origin word, unused)
    o3[a] = __longlong_as_double(__ldg(&tb[BT_O + c]));
    qo3[a] = __longlong_as_double(__ldg(&tb[BT_Q + c]));
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const long long* tb = bp.tab + a * BT_AXIS;
    const long long xb = xb3[a];
    const int nc = g.nc[a];
    int c = c3[a];
    if (inb[a]) {
      // the exact cell from the thresholds (the estimate is off by at most a
      // step, rarely)
      if (!((c == 0 || xb >= lo3[a]) && (c == nc - 1 || xb < hi3[a]))) {
        while (c < nc - 1 && xb >= __ldg(&tb[c + 1])) ++c;
        while (c > 0 && xb < __ldg(&tb[c])) --c;
        o3[a] = __longlong_as_double(__ldg(&tb[BT_O + c]));
        qo3[a] = __longlong_as_double(__ldg(&tb[BT_Q + c]));
      }
    } else {
      // k_bin's general path: periodic image and wrapped coordinate
      const double xa = __longlong_as_double(xb);
      const double k = floor(xa * g.invL[a]);
      const double w = xa - g.L[a] * k;
      c = (int)(w * g.invh[a]);
      c = c < 0 ? 0 : (c >= nc ? nc - 1 : c);
      o3[a] = fma(k, g.L[a], c * g.h[a]);
      qo3[a] = 6755399441055744.0 - o3[a] * bp.scale;
    }
    c3[a] = c;
    origin[3 * (size_t)i + a] = o3[a];
    qorg[3 * (size_t)i + a] = qo3[a];
    // the pack of k_pack at a build: q = round((x - o) 2^S) with one rounding
    q3[a] = (int)(__double_as_longlong(fma(xr[a], bp.scale, qo3[a])) - mb);
  }
  if (!finite) atomicOr(&flags[FLAG_NONFINITE], 1);
  const int cell = (c3[2] * g.nc[1] + c3[1]) * g.nc[0] + c3[0];
  cell_of[i] = cell;
  atomicAdd(&cell_count[cell], 1);
  const int4 pq = make_int4(q3[0], q3[1], q3[2], t);
  bp.posq[i] = pq;
  bp.qref[i] = pq;
  bp.pos32[i] = make_float4((float)q3[0] * bp.inv_scale, (float)q3[1] * bp.inv_scale,
                            (float)q3[2] * bp.inv_scale, __int_as_float(t));
  if (bp.pos64) bp.pos64[i] = dpos4{xr[0] - o3[0], xr[1] - o3[1], xr[2] - o3[2], (double)t};
  bp.kmask[i] = ~0ull;
}

// --- exclusive scan over m ints (tile scans, then tile offsets) ---
__device__ __forceinline__ int warp_incl_scan(int v) {
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) >= o) v += t;
  }
  return v;
}

// block-wide exclusive scan of one value per thread; returns exclusive prefix, *total
__device__ int block_excl_scan(int v, int* total) {
  __shared__ int wsum[SCAN_BLOCK / 32];
  __shared__ int wtotal;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = warp_incl_scan(v);
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int nw = blockDim.x >> 5;
    int s = lane < nw ? wsum[lane] : 0;
    int si = warp_incl_scan(s);
    if (lane < nw) wsum[lane] = si - s;
    if (lane == nw - 1) wtotal = si;
  }
  __syncthreads();
  int res = incl - v + wsum[wid];
  if (total) *total = wtotal;
  __syncthreads();
  return res;
}

__global__ void k_scan_tiles(int* __restrict__ in, int m, int* __restrict__ out,
                             int* __restrict__ tile_sums) {
  pdl_wait();
  int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
  int v[SCAN_ITEMS];
  int s = 0;
  for (int q = 0; q < SCAN_ITEMS; ++q) {
    v[q] = (base + q < m) ? in[base + q] : 0;
    s += v[q];
  }
  // the counts are read once: clear them for the next build's binning
  for (int q = 0; q < SCAN_ITEMS; ++q)
    if (base + q < m) in[base + q] = 0;
  int total;
  int pre = block_excl_scan(s, &total);
  for (int q = 0; q < SCAN_ITEMS; ++q) {
    if (base + q < m) out[base + q] = pre;
    pre += v[q];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// single block: exclusive scan of the tile sums in place (grids of many tiles)
__global__ void k_scan_sums(int* __restrict__ sums, int nt) {
  pdl_wait();
  int carry = 0;
  for (int base = 0; base < nt; base += SCAN_BLOCK) {
    int idx = base + threadIdx.x;
    int v = idx < nt ? sums[idx] : 0;
    int total;
    int pre = block_excl_scan(v, &total);
    if (idx < nt) sums[idx] = pre + carry;
    carry += total;
  }
}

// Adds to each count's tile-local prefix the offset of its tile: tile_sums
// holds either the scanned offsets (scanned = 1, after k_scan_sums) or the
// tile totals, which the block's first warp then sums up to its tile (grids of
// at most SCAN_SUM_TILES tiles: no separate pass). A block lies inside one
// tile (SCAN_TILE is a multiple of the block).
constexpr int SCAN_ADD_BLOCK = 256;
constexpr int SCAN_SUM_TILES = 1024;
static_assert(SCAN_TILE % SCAN_ADD_BLOCK == 0, "a scan-add block must lie inside one tile");
__global__ void __launch_bounds__(SCAN_ADD_BLOCK) k_scan_add(int* __restrict__ out, int m,
                                                             const int* __restrict__ tile_sums,
                                                             int scanned, int* __restrict__ fill) {
  pdl_wait();
  __shared__ int s_off;
  const int tile = (int)(((size_t)blockIdx.x * SCAN_ADD_BLOCK) / SCAN_TILE);
  if (threadIdx.x < 32) {
    int v = 0;
    if (scanned) {
      v = threadIdx.x == 0 ? tile_sums[tile] : 0;
    } else {
      for (int t = threadIdx.x; t < tile; t += 32) v += tile_sums[t];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    if (threadIdx.x == 0) s_off = v;
  }
  __syncthreads();
  const int idx = blockIdx.x * SCAN_ADD_BLOCK + threadIdx.x;
  if (idx >= m) return;
  const int v = out[idx] + s_off;
  out[idx] = v;
  if (fill) fill[idx] = v;
}

__global__ void k_scatter(int n, const int* __restrict__ cell_of, int* __restrict__ fill,
                          int* __restrict__ cell_atoms) {
  pdl_wait();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int slot = atomicAdd(&fill[cell_of[i]], 1);
  cell_atoms[slot] = i;
}

// Exact membership test (the definition's operation sequence, no FMA).
__device__ __forceinline__ bool exact_member(const double* __restrict__ x, int i, int j,
                                             const GridDev& g, double rc2, float dx32,
                                             float dy32, float dz32) {
  double d[3];
  float st[3] = {dx32, dy32, dz32};
  for (int a = 0; a < 3; ++a) {
    double dd = __dsub_rn(x[3 * (size_t)j + a], x[3 * (size_t)i + a]);
    dd = __dsub_rn(dd, __dmul_rn(g.L[a], rint(__dmul_rn(dd, g.invL[a]))));
    d[a] = dd;
    // the stencil image must be the minimum image (relevant when a box edge
    // holds only two cells and two images of j are visited)
    if (fabs((double)st[a] - dd) > 0.5 * g.L[a]) return false;
  }
  double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])),
                        __dmul_rn(d[2], d[2]));
  return r2 <= rc2;
}

// squared short-list radii per (type i, type j): filter radius plus margin
struct Radii {
  float r2[TERSOFF_MAX_SPECIES * TERSOFF_MAX_SPECIES];
};

// Atoms of each cell in ascending index order, so that list order (stencil
// order, then cell order) does not depend on the scatter's atomic order.
// Sorts each cell's atoms by index and writes the positions in cell order for
// the candidate scan: slot s of the cell arrays holds the float offsets of
// atom j = cell_atoms[s] and, in the fourth word, the bits of 4 j + species
// (j < 2^26, at most 4 species). A cell of at most CS_REG atoms is sorted in
// registers (odd-even transposition over CS_REG keys, empty keys last) with
// its loads issued together; larger cells by insertion in place.
constexpr int CS_REG = 8;
__global__ void k_cell_sort(int ncell, const int* __restrict__ cell_start,
                            int* __restrict__ cell_atoms, const float4* __restrict__ pos32,
                            float4* __restrict__ posc) {
  pdl_wait();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int s0 = cell_start[c], s1 = cell_start[c + 1];
  const int m = s1 - s0;
  if (m <= CS_REG) {
    int k[CS_REG];
#pragma unroll
    for (int q = 0; q < CS_REG; ++q) k[q] = q < m ? cell_atoms[s0 + q] : 0x7fffffff;
#pragma unroll
    for (int r = 0; r < CS_REG; ++r)
#pragma unroll
      for (int q = r & 1; q + 1 < CS_REG; q += 2) {
        const int lo = min(k[q], k[q + 1]), hi = max(k[q], k[q + 1]);
        k[q] = lo;
        k[q + 1] = hi;
      }
    float4 p[CS_REG];
#pragma unroll
    for (int q = 0; q < CS_REG; ++q)
      if (q < m) p[q] = pos32[k[q]];
#pragma unroll
    for (int q = 0; q < CS_REG; ++q)
      if (q < m) {
        cell_atoms[s0 + q] = k[q];
        posc[s0 + q] = make_float4(p[q].x, p[q].y, p[q].z,
                                   __int_as_float(4 * k[q] + __float_as_int(p[q].w)));
      }
    return;
  }
  for (int a = s0 + 1; a < s1; ++a) {
    const int key = cell_atoms[a];
    int b = a - 1;
    while (b >= s0 && cell_atoms[b] > key) {
      cell_atoms[b + 1] = cell_atoms[b];
      --b;
    }
    cell_atoms[b + 1] = key;
  }
  for (int a = s0; a < s1; ++a) {
    const int j = cell_atoms[a];
    const float4 p = pos32[j];
    posc[a] = make_float4(p.x, p.y, p.z, __int_as_float(4 * j + __float_as_int(p.w)));
  }
}

// NS1: one species (the short-list radii are single values)
template <bool BATCH, bool NS1>
__global__ void __launch_bounds__(128) k_neigh(
    int n, const double* __restrict__ x, const float4* __restrict__ pos32,
    const int* __restrict__ cell_of, const int* __restrict__ cell_start,
    const float4* __restrict__ posc, const __grid_constant__ GridDev g1,
    const GridDev* __restrict__ geo,
    const int* __restrict__ atom_sys, double rc2, float lo2, float hi2, int cap,
    uint32_t* __restrict__ nbr, int* __restrict__ cnt, const __grid_constant__ Radii lim,
    const __grid_constant__ Radii core, int ns,
    uint32_t* __restrict__ shortl, int* __restrict__ zcnt, int* __restrict__ bucket,
    uint8_t* __restrict__ zwa, int* __restrict__ flags) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = i < n;
  int count = 0;
  int z = 0;
  int zw = 0;  // entries inside the filter radii without the margin
  if (active) {
    const GridDev& g = grid_of<BATCH>(g1, geo, atom_sys, i);
    const float4 pi = pos32[i];
    const int ti = __float_as_int(pi.w);
    const int ci = cell_of[i] - g.cell_base;
    const int cx = ci % g.nc[0];
    const int cy = (ci / g.nc[0]) % g.nc[1];
    const int cz = ci / (g.nc[0] * g.nc[1]);
    for (int oz = -1; oz <= 1; ++oz) {
      int az = cz + oz;
      az += (az < 0) ? g.nc[2] : 0;
      az -= (az >= g.nc[2]) ? g.nc[2] : 0;
      for (int oy = -1; oy <= 1; ++oy) {
        int ay = cy + oy;
        ay += (ay < 0) ? g.nc[1] : 0;
        ay -= (ay >= g.nc[1]) ? g.nc[1] : 0;
        for (int ox = -1; ox <= 1; ++ox) {
          int ax = cx + ox;
          ax += (ax < 0) ? g.nc[0] : 0;
          ax -= (ax >= g.nc[0]) ? g.nc[0] : 0;
          const int c = g.cell_base + (az * g.nc[1] + ay) * g.nc[0] + ax;
          const float sx = ox * g.hf[0], sy = oy * g.hf[1], sz = oz * g.hf[2];
          const uint32_t code = ((uint32_t)(ox + 1) << 26) | ((uint32_t)(oy + 1) << 28) |
                                ((uint32_t)(oz + 1) << 30);
          const int s1 = cell_start[c + 1];
          for (int s = cell_start[c]; s < s1; ++s) {
            const float4 pj = posc[s];
            const int jt = __float_as_int(pj.w);
            const int j = jt >> 2, tj = jt & 3;
            const float dx = (pj.x - pi.x) + sx;
            const float dy = (pj.y - pi.y) + sy;
            const float dz = (pj.z - pi.z) + sz;
            const float r2 = dx * dx + dy * dy + dz * dz;
            // FP32 classification; candidates in the band around the list
            // radius take the exact test (rare)
            bool in = r2 < lo2;
            if (r2 >= lo2 && r2 <= hi2) in = exact_member(x, i, j, g, rc2, dx, dy, dz);
            in = in && j != i;
            if (in) {
              const uint32_t e = (uint32_t)j | code;
              if (count < cap) nbr[(size_t)count * n + i] = e;
              ++count;
              // short list: within the filter radius plus the margin
              const float l2 = NS1 ? lim.r2[0] : lim.r2[ti * ns + tj];
              const float c2 = NS1 ? core.r2[0] : core.r2[ti * ns + tj];
              if (r2 <= l2) {
                if (z < cap) shortl[(size_t)z * n + i] = e;
                ++z;
                zw += r2 <= c2 ? 1 : 0;
              }
            }
          }
        }
      }
    }
    cnt[i] = count;
    zcnt[i] = z;
    zwa[i] = (uint8_t)(zw < 63 ? zw : 63);
  }
  // block-level aggregation: one atomic per block and word
  __shared__ int s_max[2], s_ovf, s_cnt[3], s_base[3], s_wcnt[4][3];
  if (threadIdx.x == 0) {
    s_max[0] = s_max[1] = 0;
    s_ovf = 0;
    s_cnt[0] = s_cnt[1] = s_cnt[2] = 0;
  }
  __syncthreads();
  int mc = active ? count : 0, mz = active ? z : 0;
  for (int o = 16; o > 0; o >>= 1) {
    mc = max(mc, __shfl_xor_sync(0xffffffffu, mc, o));
    mz = max(mz, __shfl_xor_sync(0xffffffffu, mz, o));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const bool ovf = __any_sync(0xffffffffu, active && count > cap);
  // bucket by the entries inside the filter radii themselves (<= 4, <= 8,
  // more): the force launch of a bucket keeps that many in registers and masks
  // the stored short list (radius plus margin) by the cutoffs at each step
  const int b = zw <= 4 ? 0 : (zw <= 8 ? 1 : 2);
  unsigned msk[3];
  for (int q = 0; q < 3; ++q) msk[q] = __ballot_sync(0xffffffffu, active && b == q);
  if (lane == 0) {
    atomicMax(&s_max[0], mc);
    atomicMax(&s_max[1], mz);
    if (ovf) s_ovf = 1;
    for (int q = 0; q < 3; ++q) s_wcnt[wid][q] = __popc(msk[q]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_max[0] > 0) atomicMax(&flags[FLAG_OVERFLOW], s_max[0]);
    if (s_max[1] > 0) atomicMax(&flags[FLAG_SHORT_MAX], s_max[1]);
    if (s_ovf) atomicOr(&flags[FLAG_OVF_ANY], 1);
    for (int q = 0; q < 3; ++q) {
      int tot = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_wcnt[w][q];
      s_base[q] = tot ? atomicAdd(&flags[flag_bucket(q)], tot) : 0;
    }
  }
  __syncthreads();
  if (active) {
    int off = s_base[b];
    for (int w = 0; w < wid; ++w) off += s_wcnt[w][b];
    bucket[(size_t)b * n + off + __popc(msk[b] & ((1u << lane) - 1u))] = i;
  }
}

// Reverse slots: for each short-list entry (j -> i), the slot of j in i's
// short list (255 if absent), used to gather forces without atomics.
// The first RU entries of j's list, and the first RU entries of each of those
// neighbours' lists, are requested together (every column has at least 8
// slots, so the loads are in bounds; entries at or beyond a count are only
// compared, never followed); longer lists finish with the loop below.
constexpr int RU = 4;
__global__ void k_rev(int n, const uint32_t* __restrict__ shortl, const int* __restrict__ zcnt,
                      int cap, uint8_t* __restrict__ rev, int* __restrict__ flags) {
  pdl_wait();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int z = zcnt[j];
  z = z < cap ? z : cap;
  int ii[RU], zi[RU];
  uint32_t ent[RU][RU];
#pragma unroll
  for (int p = 0; p < RU; ++p) {
    const uint32_t e = shortl[(size_t)p * n + j];
    ii[p] = p < z ? (int)(e & ENTRY_JMASK) : j;
  }
#pragma unroll
  for (int p = 0; p < RU; ++p) {
    zi[p] = zcnt[ii[p]];
#pragma unroll
    for (int s = 0; s < RU; ++s) ent[p][s] = shortl[(size_t)s * n + ii[p]];
  }
#pragma unroll
  for (int p = 0; p < RU; ++p) {
    if (p >= z) break;
    const int i = ii[p];
    const int zz = zi[p] < cap ? zi[p] : cap;
    int q = 255;
#pragma unroll
    for (int s = RU - 1; s >= 0; --s)
      if (s < zz && (int)(ent[p][s] & ENTRY_JMASK) == j) q = s;
    for (int s = RU; q == 255 && s < zz; ++s)
      if ((int)(shortl[(size_t)s * n + i] & ENTRY_JMASK) == j) q = s;
    if (q == 255) atomicOr(&flags[FLAG_REV_MISS], 1);
    rev[(size_t)p * n + j] = (uint8_t)q;
  }
  for (int p = RU; p < z; ++p) {
    const int i = (int)(shortl[(size_t)p * n + j] & ENTRY_JMASK);
    int zi = zcnt[i];
    zi = zi < cap ? zi : cap;
    int q = 255;
    for (int s = 0; s < zi; ++s)
      if ((int)(shortl[(size_t)s * n + i] & ENTRY_JMASK) == j) {
        q = s;
        break;
      }
    if (q == 255) atomicOr(&flags[FLAG_REV_MISS], 1);
    rev[(size_t)p * n + j] = (uint8_t)q;
  }
}

// Copies the lists out row-major, each row sorted by neighbour index.
__global__ void k_export(int n, const uint32_t* __restrict__ nbr, const int* __restrict__ cnt,
                         int cap_in, int cap_out, int* __restrict__ out_cnt,
                         int* __restrict__ out_nbr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = cnt[i];
  out_cnt[i] = c;
  int m = c < cap_in ? c : cap_in;
  m = m < cap_out ? m : cap_out;
  int* row = out_nbr + (size_t)i * cap_out;
  for (int s = 0; s < m; ++s) {
    const int key = (int)(nbr[(size_t)s * n + i] & ENTRY_JMASK);
    int b = s - 1;
    while (b >= 0 && row[b] > key) {
      row[b + 1] = row[b];
      --b;
    }
    row[b + 1] = key;
  }
  for (int s = m; s < cap_out; ++s) row[s] = -1;
}

template <class T>
int grow(Ctx* c, T** p, size_t* have, size_t need) {
  if (*have >= need && *p) return TERSOFF_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  TGB_CUDA(c, cudaMalloc((void**)p, sizeof(T) * need));
  *have = need;
  return TERSOFF_OK;
}

// smallest double x >= 0 whose rounded product x * m is at least v (m > 0,
// v > 0): a binary search over the bit patterns of the non-negative doubles,
// which order like the values
double first_at_least(double m, double v) {
  long long lo = 0, hi = 0x7ff0000000000000ll;  // P(+0) false, P(+inf) true
  while (hi - lo > 1) {
    const long long mid = lo + (hi - lo) / 2;
    double xm;
    std::memcpy(&xm, &mid, sizeof xm);
    if (xm * m >= v)
      hi = mid;
    else
      lo = mid;
  }
  double r;
  std::memcpy(&r, &hi, sizeof r);
  return r;
}

long long bits_of(double d) {
  long long b;
  std::memcpy(&b, &d, sizeof b);
  return b;
}

}  // namespace

int upload_bin_tables(Ctx* c, cudaStream_t s) {
  const Grid& G = c->grid;
  const double scale = ldexp(1.0, G.fix_shift);
  std::vector<long long>& t = c->h_bintab;
  t.assign((size_t)3 * BT_AXIS, 0);
  for (int a = 0; a < 3; ++a) {
    if (G.nc[a] > BT_O) return fail(c, TERSOFF_E_INVALID_ARG, "more than 1024 cells per axis");
    long long* ta = t.data() + (size_t)a * BT_AXIS;
    ta[0] = bits_of(first_at_least(G.invL[a], 1.0));
    for (int q = 1; q < G.nc[a]; ++q) ta[q] = bits_of(first_at_least(G.invh[a], (double)q));
    for (int q = 0; q < G.nc[a]; ++q) {
      const double o = q * G.h[a];
      ta[BT_O + q] = bits_of(o);
      ta[BT_Q + q] = bits_of(6755399441055744.0 - o * scale);
    }
  }
  if (!c->d_bintab) TGB_CUDA(c, cudaMalloc(&c->d_bintab, sizeof(long long) * t.size()));
  TGB_CUDA(c, cudaMemcpyAsync(c->d_bintab, t.data(), sizeof(long long) * t.size(),
                              cudaMemcpyHostToDevice, s));
  return TERSOFF_OK;
}

int launch_neighbor_build(Ctx* c, const double* x, cudaStream_t s) {
  const int n = c->n;
  c->fine_valid = false;
  const Grid& G = c->grid;
  const bool batch = c->n_sys > 0;
  const long ncell = batch ? c->ncell_batch : (long)G.nc[0] * G.nc[1] * G.nc[2];
  // cell arrays
  if (c->cells_alloc < (size_t)ncell + 1) {
    cudaFree(c->d_cell_count);
    cudaFree(c->d_cell_start);
    cudaFree(c->d_cell_fill);
    cudaFree(c->d_scan_tmp);
    c->d_cell_count = c->d_cell_start = c->d_cell_fill = c->d_scan_tmp = nullptr;
    size_t m = (size_t)ncell + 1;
    TGB_CUDA(c, cudaMalloc(&c->d_cell_count, sizeof(int) * m));
    TGB_CUDA(c, cudaMalloc(&c->d_cell_start, sizeof(int) * m));
    TGB_CUDA(c, cudaMalloc(&c->d_cell_fill, sizeof(int) * m));
    TGB_CUDA(c, cudaMalloc(&c->d_scan_tmp, sizeof(int) * (m / SCAN_TILE + 2)));
    // zero once: every build's first scan pass clears the counts it read
    TGB_CUDA(c, cudaMemsetAsync(c->d_cell_count, 0, sizeof(int) * m, s));
    c->cells_alloc = m;
  }
  GridDev g = to_dev(G);
  const int B = 256;
  const int nb = (n + B - 1) / B;
  const double scale = ldexp(1.0, G.fix_shift);
  // new slots hold stale forces: every entry of every atom may be nonzero
  // (k_bin_pack sets the masks of single systems)
  if (n > 0 && batch)
    TGB_CUDA(c, cudaMemsetAsync(c->d_kmask, 0xff, sizeof(unsigned long long) * n, s));
  if (n > 0) {
    c->launches++;
    if (batch) {
      // per-system grids: k_bin's arithmetic, then the build's pack
      TGB_CUDA(c, launch_pdl(k_bin<true>, nb, B, 0, s, n, x, g, c->d_geo, c->d_atom_sys, scale,
                             c->d_cell_of, c->d_cell_count, c->d_origin, c->d_qorg, c->d_flags));
      int st = launch_pack_positions(c, x, true, s);
      if (st) return st;
    } else {
      BinPack bp;
      bp.tab = c->d_bintab;
      for (int a = 0; a < 3; ++a) bp.invhf[a] = (float)G.invh[a];
      bp.scale = scale;
      bp.inv_scale = ldexpf(1.0f, -G.fix_shift);
      bp.types = c->d_types;
      bp.posq = c->d_posq;
      bp.pos32 = c->d_pos32;
      bp.qref = c->d_qref;
      bp.pos64 = c->precision == TERSOFF_FP64 ? c->d_pos64 : nullptr;
      bp.kmask = c->d_kmask;
      TGB_CUDA(c, launch_pdl(k_bin_pack, nb, B, 0, s, n, x, g, bp, c->d_cell_of, c->d_cell_count,
                             c->d_origin, c->d_qorg, c->d_flags));
    }
  }
  const int m = (int)ncell + 1;
  const int ntiles = (m + SCAN_TILE - 1) / SCAN_TILE;
  TGB_CUDA(c, launch_pdl(k_scan_tiles, ntiles, SCAN_BLOCK, 0, s, c->d_cell_count, m, c->d_cell_start, c->d_scan_tmp));
  const int scanned = ntiles > SCAN_SUM_TILES ? 1 : 0;
  if (scanned) {
    TGB_CUDA(c, launch_pdl(k_scan_sums, 1, SCAN_BLOCK, 0, s, c->d_scan_tmp, ntiles));
    c->launches++;
  }
  TGB_CUDA(c, launch_pdl(k_scan_add, (m + SCAN_ADD_BLOCK - 1) / SCAN_ADD_BLOCK, SCAN_ADD_BLOCK, 0, s,
                         c->d_cell_start, m, c->d_scan_tmp, scanned, c->d_cell_fill));
  c->launches += 2;
  if (n > 0) {
    TGB_CUDA(c, launch_pdl(k_scatter, nb, B, 0, s, n, c->d_cell_of, c->d_cell_fill, c->d_cell_atoms));
    TGB_CUDA(c, launch_pdl(k_cell_sort, (int)((ncell + 255) / 256), 256, 0, s, (int)ncell, c->d_cell_start,
                           c->d_cell_atoms, c->d_pos32, c->d_posc));
    c->launches += 2;
  }
  const double rc2 = c->r_list * c->r_list;
  // FP32 classification band: the FP32 r^2 of a stencil candidate differs from
  // the exact value by far less than this (offsets below 2 cells, float eps).
  const double hmax = fmax(G.h[0], fmax(G.h[1], G.h[2]));
  const double band = 64.0 * (4.0 * hmax) * (4.0 * hmax) * 1.2e-7 + 1e-6;
  const float lo2 = (float)(rc2 - band);
  const float hi2 = (float)(rc2 + band);
  Radii lim, core;
  for (int q = 0; q < TERSOFF_MAX_SPECIES * TERSOFF_MAX_SPECIES; ++q) lim.r2[q] = core.r2[q] = 0.0f;
  // symmetric in the two species, so that short-list membership is mutual
  for (int a = 0; a < c->ns; ++a)
    for (int b = 0; b < c->ns; ++b) {
      const double rf = fmax(c->filt[(size_t)a * c->ns + b], c->filt[(size_t)b * c->ns + a]);
      const double r = rf + c->margin;
      lim.r2[a * c->ns + b] = (float)(r * r * (1.0 + 1e-6));
      core.r2[a * c->ns + b] = (float)(rf * rf);
    }
  if (n > 0) {
    if (batch)
      TGB_CUDA(c, launch_pdl(k_neigh<true, false>, (n + 127) / 128, 128, 0, s,
          n, x, c->d_pos32, c->d_cell_of, c->d_cell_start, c->d_posc, g, c->d_geo,
          c->d_atom_sys, rc2, lo2, hi2, c->cap, c->d_nbr, c->d_cnt, lim, core, c->ns, c->d_short,
          c->d_zcnt, c->d_bucket, c->d_zw, c->d_flags));
    else if (c->ns == 1)
      TGB_CUDA(c, launch_pdl(k_neigh<false, true>, (n + 127) / 128, 128, 0, s,
          n, x, c->d_pos32, c->d_cell_of, c->d_cell_start, c->d_posc, g, nullptr, nullptr,
          rc2, lo2, hi2, c->cap, c->d_nbr, c->d_cnt, lim, core, c->ns, c->d_short, c->d_zcnt,
          c->d_bucket, c->d_zw, c->d_flags));
    else
      TGB_CUDA(c, launch_pdl(k_neigh<false, false>, (n + 127) / 128, 128, 0, s,
          n, x, c->d_pos32, c->d_cell_of, c->d_cell_start, c->d_posc, g, nullptr, nullptr,
          rc2, lo2, hi2, c->cap, c->d_nbr, c->d_cnt, lim, core, c->ns, c->d_short, c->d_zcnt,
          c->d_bucket, c->d_zw, c->d_flags));
    TGB_CUDA(c, launch_pdl(k_rev, (n + 255) / 256, 256, 0, s, n, c->d_short, c->d_zcnt, c->zs_cap, c->d_rev,
                                          c->d_flags));
    c->launches += 2;
  }
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

int launch_neighbor_export(Ctx* c, int* cnt, int* nbr, int cap, cudaStream_t s) {
  if (c->n == 0) return TERSOFF_OK;
  k_export<<<(c->n + 255) / 256, 256, 0, s>>>(c->n, c->d_nbr, c->d_cnt, c->cap, cap, cnt, nbr);
  c->launches++;
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

}  // namespace tgb

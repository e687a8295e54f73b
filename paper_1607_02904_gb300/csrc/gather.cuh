// Force gathering from per-slot contributions (no atomics on the fast path).
//
// The force kernel stores the force that atom i's terms put on each short-list
// neighbour j in j's column of the contribution array, at the slot of j's own
// short list that holds i (the reverse slot, found at the build; short-list
// membership is symmetric), and the force on i itself in own_i. The force on
// atom j is own_j plus the slots 0 .. z_j - 1 of its column, read in slot
// order with coalesced loads and no indirection. Mixed path: the float
// contributions are
// summed with error-free transformations (each float addition's rounding
// error is recovered exactly and accumulated), and the sum and its error term
// are converted to double and added once: the result carries the exact sum to
// within a double rounding. FP64 path: summed in double.
#pragma once
#include <cstdint>

#include "internal.cuh"

namespace tgb {

struct GatherArgs {
  int n;
  int cap;
  int fp64;
  int atomic_mode;  // forces were scattered with FP64 atomics into extra
  int plain;        // mixed path: plain float sums (ablation), no error term
  const int* zcnt;
  const void* contrib;
  const void* own;
  double* extra;
  const int* flags;
};

// float -> double through the IEEE-754 bit layouts (exact; float subnormals
// flush to signed zero). Integer operations only.
__device__ __forceinline__ double gather_f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t sign = u & 0x80000000u;
  const uint32_t mag = u & 0x7fffffffu;
  uint32_t hi = (mag >> 3) + 0x38000000u;
  uint32_t lo = mag << 29;
  const bool tiny = mag < 0x00800000u;
  hi = tiny ? 0u : hi;
  lo = tiny ? 0u : lo;
  hi = (mag >= 0x7f800000u) ? ((mag >> 3) | 0x7ff00000u) : hi;
  return __hiloint2double((int)(hi | sign), (int)lo);
}

// s += x with the rounding error of the addition added to c (Knuth's TwoSum:
// the error is exact for round-to-nearest float arithmetic).
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
  const float t = __fadd_rn(s, x);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
  s = t;
  c = __fadd_rn(c, err);
}

// Total force on atom j in eV/A (clears j's fallback-buffer entry when it is
// used). Mixed path: also the float pair (s, c) with s + c = the exact sum of
// the contributions (fixed order) plus the fallback term; FP64 path: s, c = 0.
__device__ __forceinline__ void gather_force(const GatherArgs& g, int j, double& fx,
                                             double& fy, double& fz, float* sc = nullptr) {
  if (g.atomic_mode) {
    double* e = g.extra + 3 * (size_t)j;
    fx = e[0];
    fy = e[1];
    fz = e[2];
    e[0] = e[1] = e[2] = 0.0;
    if (sc) sc[0] = sc[1] = sc[2] = sc[3] = sc[4] = sc[5] = 0.0f;
    return;
  }
  int z = g.zcnt[j];
  z = z < g.cap ? z : g.cap;
  double ex = 0.0, ey = 0.0, ez = 0.0;
  const bool extra = g.flags[FLAG_EXTRA] | g.flags[FLAG_EXTRA_STICKY];
  if (extra) {
    double* e = g.extra + 3 * (size_t)j;
    ex = e[0];
    ey = e[1];
    ez = e[2];
    e[0] = e[1] = e[2] = 0.0;
  }
  // the first GU slots are loaded without waiting for the count (every
  // column has at least GU slots), the rest once it is known
  constexpr int GU = 4;
  if (!g.fp64) {
    const float4* c = (const float4*)g.contrib + j;
    const float4 o = ((const float4*)g.own)[j];
    float4 v[GU];
#pragma unroll
    for (int p = 0; p < GU; ++p) v[p] = c[(size_t)p * g.n];
    float sx = o.x, sy = o.y, sz = o.z, cx = 0.0f, cy = 0.0f, cz = 0.0f;
    if (g.plain) {  // single-precision accumulation, same order
#pragma unroll
      for (int p = 0; p < GU; ++p)
        if (p < z) {
          sx = __fadd_rn(sx, v[p].x);
          sy = __fadd_rn(sy, v[p].y);
          sz = __fadd_rn(sz, v[p].z);
        }
      for (int p = GU; p < z; ++p) {
        const float4 w = c[(size_t)p * g.n];
        sx = __fadd_rn(sx, w.x);
        sy = __fadd_rn(sy, w.y);
        sz = __fadd_rn(sz, w.z);
      }
    } else {
#pragma unroll
      for (int p = 0; p < GU; ++p)
        if (p < z) {
          two_sum_acc(sx, cx, v[p].x);
          two_sum_acc(sy, cy, v[p].y);
          two_sum_acc(sz, cz, v[p].z);
        }
      for (int p = GU; p < z; ++p) {
        const float4 w = c[(size_t)p * g.n];
        two_sum_acc(sx, cx, w.x);
        two_sum_acc(sy, cy, w.y);
        two_sum_acc(sz, cz, w.z);
      }
    }
    if (sc) {  // the caller works with the pair and the fallback term separately
      sc[0] = sx;
      sc[1] = sy;
      sc[2] = sz;
      sc[3] = cx;
      sc[4] = cy;
      sc[5] = cz;
      fx = ex;
      fy = ey;
      fz = ez;
    } else {
      fx = gather_f2d(sx) + (gather_f2d(cx) + ex);
      fy = gather_f2d(sy) + (gather_f2d(cy) + ey);
      fz = gather_f2d(sz) + (gather_f2d(cz) + ez);
    }
  } else {
    const dpos4* c = (const dpos4*)g.contrib + j;
    const dpos4 o = ((const dpos4*)g.own)[j];
    fx = o.x + ex;
    fy = o.y + ey;
    fz = o.z + ez;
    for (int p = 0; p < z; ++p) {
      const dpos4 w = c[(size_t)p * g.n];
      fx += w.x;
      fy += w.y;
      fz += w.z;
    }
    if (sc) sc[0] = sc[1] = sc[2] = sc[3] = sc[4] = sc[5] = 0.0f;
  }
}

inline GatherArgs make_gather(Ctx* c) {
  GatherArgs g;
  g.n = c->n;
  g.cap = c->zs_cap;
  g.fp64 = c->precision == TERSOFF_FP64;
  g.atomic_mode = (c->scatter_atomic || comp_atom_sums(c)) ? 1 : 0;
  g.plain = (c->ablate & 4) && c->precision == TERSOFF_MIXED;
  g.zcnt = c->d_zcnt;
  g.contrib = c->d_contrib;
  g.own = c->d_own;
  g.extra = c->d_extra;
  g.flags = c->d_flags;
  return g;
}

}  // namespace tgb

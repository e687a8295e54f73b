// Force kernel with four lanes per centre atom, one lane per bond (the GPU
// form of the paper's scheme (a), Sec. IV-B: neighbours j on vector lanes).
//
// The group of four lanes holds atom i's bonds inside the cutoffs, at most
// four (Si diamond: its four nearest neighbours). Lane q forms the bond
// vector, length, unit vector and cutoff of its bond; the other bonds' data
// arrive by warp shuffles. The first K loop (Sec. III, Algorithm 2) runs over
// the three other lanes' bonds and gives zeta_iq; the pair level gives
// V(i, q), dV/dr and dV/dzeta of the lane's own bond; the second K loop
// combines the lane's own dV/dzeta with those of the other lanes (shuffled)
// into the force on neighbour q. The force on i is the negated group sum.
// Nothing is held in per-thread arrays, so the kernel needs few registers
// and many warps fit on an SM.
//
// Bonds: from the stored short list when it is valid (the common case: no
// atom has moved more than half the list margin since the build), else from
// the skin list. When the list holds more than four entries, the group keeps
// those inside the cutoffs (ballot, then a shuffle into the lanes); atoms
// with more than four bonds inside the cutoffs, or on the general path, are
// appended to a leftover list that the per-thread kernel (k_tersoff, with its
// register capacity 8 and general path) processes next.
//
// Forces: per-slot stores into the receiving atoms' columns (gather scatter)
// or FP64 atomics, exactly as k_tersoff; the same kmask bookkeeping for
// stored short lists filtered by the cutoffs.
#pragma once
#include "tersoff_fwd.cuh"

namespace tgb {
namespace fwd {

constexpr int QBLOCK = 128;
constexpr int QATOMS = QBLOCK / 4;  // atoms per block and round

// Shuffle from lane src of the warp (all lanes take part).
template <class T>
__device__ __forceinline__ T qsh(T v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}

// Sum over the four lanes of a group.
template <class T>
__device__ __forceinline__ T qsum(T v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  return v;
}

template <class T, int NS, int MODE, bool EV>
__global__ void __launch_bounds__(QBLOCK) k_tersoff_quad(const __grid_constant__ FwdArgs<T> a) {
  constexpr int SNS = NS > 1 ? NS : (NS == 1 ? 1 : TERSOFF_MAX_SPECIES);
  constexpr int SREC = NS == 1 ? 1 : SNS * SNS * SNS * RSTRIDE;
  constexpr bool LAM3 = MODE == 1;
  __shared__ T srec_s[SREC];
  __shared__ T sfilt[SNS * SNS];
  __shared__ float snear[SNS * SNS];
  __shared__ int uni[3];
  __shared__ typename SumT<T>::type tsum[7][QBLOCK];
  const int ns = NS > 0 ? NS : a.ns;
  if (NS != 1)
    for (int q = threadIdx.x; q < ns * ns * ns * RSTRIDE; q += QBLOCK) srec_s[q] = a.rec[q];
  if (threadIdx.x < ns * ns) {
    sfilt[threadIdx.x] = a.filt2[threadIdx.x];
    snear[threadIdx.x] = sizeof(T) == 4 ? a.near2[threadIdx.x] : 0.0f;
  }
  if (threadIdx.x < 3) {
    const int* src = threadIdx.x == 0   ? a.flags + FLAG_REV_MISS
                     : threadIdx.x == 1 ? a.flags + FLAG_DMAX
                                        : a.n_items;
    uni[threadIdx.x] = src ? *src : 0;
  }
  const bool want_acc = EV && a.acc != nullptr;
  if (want_acc)
    for (int q = 0; q < 7; ++q) sum_zero(tsum[q][threadIdx.x]);
  __syncthreads();
  const T* srec = NS == 1 ? a.prm1 : srec_s;
  const bool use_short = __int_as_float(uni[1]) <= a.dlim2;
  const bool slots = !a.atomic_mode && use_short && uni[0] == 0;
  const int n_items = a.identity ? a.n : uni[2];
  if (blockIdx.x == 0 && threadIdx.x == 0) a.flags[FLAG_EXTRA] = slots ? 0 : 1;
  const int lane = threadIdx.x & 31;
  const int q = lane & 3;          // this lane's bond slot in the group
  const int gb = lane & ~3;        // the group's first lane
  const Shift<T, false> sh;
  using P = typename SelfPos<T>::type;

  // block-uniform loop: every lane takes part in every shuffle
  for (int it0 = blockIdx.x * QATOMS; it0 < n_items; it0 += gridDim.x * QATOMS) {
    const int item = it0 + (threadIdx.x >> 2);
    const bool have = item < n_items;
    const int i = have ? (a.identity ? item : a.order[item]) : 0;
    int zl = 0, ti = 0;
    P pi{};
    if (have) {
      zl = a.zcnt[i];
      ti = NS == 1 ? 0 : a.types[i];
      pi = self_pos<T>(a, i);
    }
    // the list to take the bonds from
    const uint32_t* list = a.shortl;
    int c = zl;
    bool left = have && a.all_general;  // handled by the per-thread kernel
    if (have && use_short && (zl > a.zs_cap || zl > 64)) left = true;  // general path there
    if (have && !use_short) {
      list = a.nbr;
      c = min(a.cnt[i], a.cap);
    }
    // the group's bond of this lane: entry and its list slot
    uint32_t e = 0;
    int sl = -1;
    const bool filtered = have && !left && (!use_short || c > 4);
    unsigned long long kept = 0ull;
    if (__any_sync(0xffffffffu, filtered)) {
      // keep the entries inside the cutoffs, four at a time; the loop runs to
      // the warp's longest list (every lane takes part in the votes)
      int nk = 0;
      T xi = 0, yi = 0, zi = 0;
      int tii;
      if (filtered) Pos<T>::coarse(a, i, xi, yi, zi, tii);
      const int cl = filtered ? c : 0;
      int cmax = cl;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
      for (int c0 = 0; c0 < cmax; c0 += 4) {
        const int s = c0 + q;
        uint32_t es = 0;
        bool ok = false;
        if (s < cl) {
          es = list[(size_t)s * a.n + i];
          int jj, ox, oy, oz;
          decode(es, jj, ox, oy, oz);
          T xj, yj, zj;
          int tjj;
          Pos<T>::coarse(a, jj, xj, yj, zj, tjj);
          const T dx = (xj - xi) + ox * sh.h(a, 0);
          const T dy = (yj - yi) + oy * sh.h(a, 1);
          const T dz = (zj - zi) + oz * sh.h(a, 2);
          ok = dx * dx + dy * dy + dz * dz <= sfilt[ti * ns + tjj];
        }
        const unsigned m = (__ballot_sync(0xffffffffu, ok) >> gb) & 0xFu;
        const int cnt_m = __popc(m);
        // lane q receives the (q - nk)-th kept entry of this chunk
        const int want = q - nk;
        const bool take = want >= 0 && want < cnt_m;
        const int src = take ? (int)__fns(m, 0, want + 1) : 0;
        const uint32_t ein = __shfl_sync(0xffffffffu, es, gb + src);
        if (take) {
          e = ein;
          sl = c0 + src;
        }
        if (ok && s < 64) kept |= 1ull << s;
        nk += cnt_m;
      }
      if (filtered && nk > 4) left = true;
      // kept slots of the whole group
      kept |= __shfl_xor_sync(0xffffffffu, kept, 1);
      kept |= __shfl_xor_sync(0xffffffffu, kept, 2);
    }
    if (have && !left && !filtered && q < c) {
      e = list[(size_t)q * a.n + i];
      sl = q;
    }
    // atoms the per-thread kernel finishes: appended to the leftover list
    {
      const unsigned lm = __ballot_sync(0xffffffffu, left && q == 0);
      if (lm) {
        int base = 0;
        if (lane == __ffs(lm) - 1) base = atomicAdd(&a.flags[FLAG_LEFT], __popc(lm));
        base = __shfl_sync(0xffffffffu, base, __ffs(lm) - 1);
        const int slot = base + __popc(lm & ((1u << lane) - 1u));
        if (left && q == 0 && slot < a.n) a.left[slot] = i;
      }
    }
    const bool act = have && !left;   // the group computes this atom
    const bool mine = act && sl >= 0;  // this lane holds a bond
    // forces through the fallback buffer while the gather still runs: the
    // gather must see zero in the atom's own slot and in its column (the
    // lanes take the slots q, q + 4, ...)
    if (act && !slots && !a.atomic_mode) {
      if (q == 0) store_slot<T>(a, a.own, (size_t)i, T(0), T(0), T(0));
      const int zc = min(zl, a.zs_cap);
      for (int p = q; p < zc; p += 4) store_slot<T>(a, a.contrib, (size_t)p * a.n + i, T(0), T(0), T(0));
    }
    // 1. the lane's bond
    T ux = 0, uy = 0, uz = 0, r = 1, ri = 1, rx = 0, fc = 0, dfc = 0;
    int j = i, tj = 0, rv = 0;
    if (slots && mine && !filtered) rv = (int)__ldg(&a.rev[(size_t)q * a.n + i]);
    if (mine) {
      T dx, dy, dz;
      Bond<T>::vec(a, sh, pi, e, dx, dy, dz, j, tj);
      const T r2 = dx * dx + dy * dy + dz * dz;
      ri = M<T>::rsqrt_nr(r2);
      r = r2 * ri;
      if (sizeof(T) == 4 && r2 > snear[ti * ns + tj]) rx = Exact<T>::residual(a, sh, pi, e, r);
      ux = dx * ri;
      uy = dy * ri;
      uz = dz * ri;
      if (MODE == 2) {
        // symmetric tables: f_C(r_iq) of record (ti, tq, tq) serves the
        // three-body terms with k = q and the pair term of bond q
        const T* pq = srec + rec_off<NS>(ns, ti, tj, tj);
        if (r < pq[K_ROUT3]) cutoff<T>(pq, K_PID3, K_DFC3, K_RIN3, K_ROUT3, K_ROUT3LO, r, fc, dfc, rx);
      }
    }
    // the other three bonds of the group
    T kx[3], ky[3], kz[3], kr[3], kf[3];
    int kt[3];
    bool kv[3];
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      const int src = gb + ((q + 1 + o) & 3);
      kx[o] = qsh(ux, src);
      ky[o] = qsh(uy, src);
      kz[o] = qsh(uz, src);
      kv[o] = qsh((int)mine, src) != 0;
      kr[o] = qsh(r, src);
      kf[o] = MODE == 2 ? qsh(fc, src) : T(0);
      kt[o] = NS == 1 ? 0 : qsh(tj, src);
    }
    const T krx_own = rx;
    // 2. first K loop: zeta of the lane's bond
    T zeta = 0;
    T cs_[3], g_[3], dg_[3], a1_[3], a2_[3];
    const T* p2 = srec + rec_off<NS>(ns, ti, tj, tj);
    const bool pair_in = mine && r < p2[K_ROUT2];
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      const T cs = ux * kx[o] + uy * ky[o] + uz * kz[o];
      cs_[o] = cs;
      const T* p3 = srec + rec_off<NS>(ns, ti, tj, kt[o]);
      if (MODE == 2) {
        const T t = p3[K_H] - cs;
        const T t2 = t * t;
        const T qq = M<T>::rcp_nr(p3[K_D2] + t2);
        g_[o] = p3[K_GC2D2] * (t2 * qq) + p3[K_GAMMA];
        dg_[o] = -p3[K_G2C2] * t * qq * qq;
        zeta += kf[o] * g_[o];
      } else {
        // the other lane's exact length residual near a cutoff
        const T rxk = qsh(rx, gb + ((q + 1 + o) & 3));
        T zt = 0, A1 = 0, A2 = 0, A3 = 0;
        if (mine && kv[o] && kr[o] < p3[K_ROUT3])
          triplet<T, LAM3>(p3, r, kr[o], cs, zt, A1, A2, A3, rxk);
        zeta += zt;
        a1_[o] = A1;
        a2_[o] = A2;
      }
    }
    // 3. pair level
    T V = 0, dVdr = 0, dz = 0;
    if (pair_in) {
      if (MODE == 2)
        pair_fc<T>(p2, r, zeta, fc, dfc, V, dVdr, dz);
      else
        pair<T>(p2, r, zeta, V, dVdr, dz, krx_own);
    }
    // 4. second K loop: the force on neighbour q
    T fx = -dVdr * ux, fy = -dVdr * uy, fz = -dVdr * uz;
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      const int src = gb + ((q + 1 + o) & 3);
      const T dzk = qsh(dz, src);
      const T cs = cs_[o];
      const T ex = kx[o] - cs * ux, ey = ky[o] - cs * uy, ez = kz[o] - cs * uz;
      T cj, bj;
      if (MODE == 2) {
        // terms zeta(i,q,k) and zeta(i,k,q) share g(cos); f_C of the other bond
        const T A = -(dz * kf[o] + dzk * fc) * dg_[o];
        cj = A * ri;
        bj = -dzk * dfc * g_[o];
      } else {
        // own term (q, k): dz d zeta(q,k)/dx_q; the other bond's term (k, q):
        // dzk d zeta(k,q)/dx_q, with record (ti, tk, tq)
        const T* p3 = srec + rec_off<NS>(ns, ti, kt[o], tj);
        T zt = 0, B1 = 0, B2 = 0, B3 = 0;
        if (mine && kv[o] && r < p3[K_ROUT3])
          triplet<T, LAM3>(p3, kr[o], r, cs, zt, B1, B2, B3, krx_own);
        cj = -(dz * a1_[o] + dzk * B1) * ri;
        bj = -(dz * a2_[o] + dzk * (B3 - B2));
      }
      fx = fmaf_t(cj, ex, fmaf_t(bj, ux, fx));
      fy = fmaf_t(cj, ey, fmaf_t(bj, uy, fy));
      fz = fmaf_t(cj, ez, fmaf_t(bj, uz, fz));
    }
    if (!mine) fx = fy = fz = 0;
    // 5. stores: the lane's neighbour force, the atom's own (lane 0)
    const T fix = -qsum(fx), fiy = -qsum(fy), fiz = -qsum(fz);
    if (mine) {
      if (slots)
        store_slot<T>(a, a.contrib, filtered ? recv_slot(a, sl, i, j) : (size_t)rv * a.n + j, fx, fy,
                      fz);
      else
        atomic_add3(a.f, j, to_f64(fx), to_f64(fy), to_f64(fz));
    }
    if (act && q == 0) {
      if (slots)
        store_slot<T>(a, a.own, (size_t)i, fix, fiy, fiz);
      else
        atomic_add3(a.f, i, to_f64(fix), to_f64(fiy), to_f64(fiz));
    }
    // stored entries outside the cutoffs now: their receiving slots get zero
    // unless they hold zero already; the lanes take the slots q, q + 4, ...
    if (slots && filtered && act) {
      unsigned long long clr = a.kmask[i] & ~kept;
      if (zl < 64) clr &= (1ull << zl) - 1ull;
      for (int s = q; s < 64; s += 4)
        if ((clr >> s) & 1ull)
          store_slot<T>(a, a.contrib, recv_slot(a, s, i, entry_atom(a, a.shortl, s, i)), T(0), T(0),
                        T(0));
      if (q == 0) a.kmask[i] = kept;
    }
    // 6. energy and virial
    if (EV) {
      const T vsum = qsum(V);
      if (a.eatom && act && q == 0) a.eatom[i] = to_f64(vsum);
      if (want_acc && mine) {
        const T dx = ux * r, dy = uy * r, dzz = uz * r;
        sum_add(tsum[0][threadIdx.x], V);
        sum_add(tsum[1][threadIdx.x], dx * fx);
        sum_add(tsum[2][threadIdx.x], dy * fy);
        sum_add(tsum[3][threadIdx.x], dzz * fz);
        sum_add(tsum[4][threadIdx.x], dx * fy);
        sum_add(tsum[5][threadIdx.x], dx * fz);
        sum_add(tsum[6][threadIdx.x], dy * fz);
      }
    }
  }
  if (want_acc) {
    __syncthreads();
    block_reduce_sums<QBLOCK>(&tsum[0][threadIdx.x], a.acc);
  }
}

}  // namespace fwd
}  // namespace tgb

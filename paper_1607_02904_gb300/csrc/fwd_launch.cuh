// Host-side instantiation and launch of the force kernel for one precision.
#pragma once
#include "tersoff_fwd.cuh"

namespace tgb {
namespace fwd {

template <class T> const T* rec_ptr(Ctx* c);
template <> inline const float* rec_ptr<float>(Ctx* c) { return c->d_rec32; }
template <> inline const double* rec_ptr<double>(Ctx* c) { return c->d_rec64; }
template <class T> const T* rec_host(Ctx* c);
template <> inline const float* rec_host<float>(Ctx* c) { return c->h_rec32.data(); }
template <> inline const double* rec_host<double>(Ctx* c) { return c->h_rec64.data(); }
template <class T> const T* filt_ptr(Ctx* c);
template <> inline const float* filt_ptr<float>(Ctx* c) { return c->d_filt32; }
template <> inline const double* filt_ptr<double>(Ctx* c) { return c->d_filt64; }

// Grids are fixed by the atom count (the bucket sizes live on the device), so
// the launches can be captured in a CUDA graph and replayed across builds.
template <class T, int NS, int ZC>
void launch_t(Ctx* c, const FwdArgs<T>& a, int grid, cudaStream_t s) {
  if (grid <= 0) return;
  if (c->has_lam3)
    k_tersoff<T, NS, ZC, 1><<<grid, BLOCK, 0, s>>>(a);
  else if (c->sym_table)
    k_tersoff<T, NS, ZC, 2><<<grid, BLOCK, 0, s>>>(a);
  else
    k_tersoff<T, NS, ZC, 0><<<grid, BLOCK, 0, s>>>(a);
  c->launches++;
}

// One launch per short-list size bucket (built with the list): register
// capacity 4 for atoms with at most 4 short-list entries, 8 for at most 8;
// longer lists take the general path inside the capacity-4 instance.
// One launch per short-list size bucket (built with the list): register
// capacity 4 for atoms with at most 4 short-list entries, 8 for at most 8;
// longer lists take the general path inside the capacity-4 instance. The small
// buckets (few atoms, latency-bound) run on a side stream next to bucket 0.
template <class T, int NS>
void launch_buckets(Ctx* c, FwdArgs<T> a, cudaStream_t s) {
  const int full = (c->n + BLOCK - 1) / BLOCK;
  const int small = full < 2 * 152 ? full : 2 * 152;
  const bool fork = c->side != nullptr;
  if (fork) {
    cudaEventRecord(c->ev_fork, s);
    cudaStreamWaitEvent(c->side, c->ev_fork, 0);
  }
  cudaStream_t s2 = fork ? c->side : s;
  for (int b = 2; b >= 0; --b) {
    a.order = c->d_bucket + (size_t)b * c->n;
    a.n_items = c->d_flags + FLAG_BUCKET + b;
    if (b == 0)
      launch_t<T, NS, 4>(c, a, full, s);
    else if (b == 1)
      launch_t<T, NS, 8>(c, a, small, s2);
    else
      launch_t<T, NS, 4>(c, a, small, s2);
  }
  if (fork) {
    cudaEventRecord(c->ev_join, c->side);
    cudaStreamWaitEvent(s, c->ev_join, 0);
  }
}

template <class T>
int launch_prec(Ctx* c, double* f, double* acc, double* eatom, cudaStream_t s) {
  FwdArgs<T> a;
  a.n = c->n;
  a.cap = c->cap;
  a.ns = c->ns;
  a.nbr = c->d_nbr;
  a.cnt = c->d_cnt;
  a.pos32 = c->d_pos32;
  a.posq = c->d_posq;
  a.pos64 = c->d_pos64;
  a.rec = rec_ptr<T>(c);
  for (int q = 0; q < RSTRIDE; ++q) a.prm1[q] = rec_host<T>(c)[q];
  a.filt2 = filt_ptr<T>(c);
  const double scale = ldexp(1.0, c->grid.fix_shift);
  for (int q = 0; q < 3; ++q) {
    a.h[q] = (T)c->grid.h[q];
    a.hq[q] = (int)llrint(c->grid.h[q] * scale);
  }
  a.qinv = ldexpf(1.0f, -c->grid.fix_shift);
  a.types = c->d_types;
  a.shortl = c->d_short;
  a.zcnt = c->d_zcnt;
  a.zs_cap = c->zs_cap;
  a.dlim2 = (float)(0.25 * c->margin * c->margin);
  a.f = f;
  a.acc = acc;
  a.eatom = eatom;
  a.flags = c->d_flags;
  switch (c->ns) {
    case 1: launch_buckets<T, 1>(c, a, s); break;
    case 2: launch_buckets<T, 2>(c, a, s); break;
    default: launch_buckets<T, 0>(c, a, s); break;
  }
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

}  // namespace fwd
}  // namespace tgb

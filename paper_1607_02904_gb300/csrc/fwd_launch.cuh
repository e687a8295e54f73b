// Host-side instantiation and launch of the force kernel for one precision.
#pragma once
#include "tersoff_fwd.cuh"

namespace tgb {
namespace fwd {

template <class T> const T* rec_ptr(Ctx* c);
template <> inline const float* rec_ptr<float>(Ctx* c) { return c->d_rec32; }
template <> inline const double* rec_ptr<double>(Ctx* c) { return c->d_rec64; }
template <class T> const T* filt_ptr(Ctx* c);
template <> inline const float* filt_ptr<float>(Ctx* c) { return c->d_filt32; }
template <> inline const double* filt_ptr<double>(Ctx* c) { return c->d_filt64; }

template <class T, int NS, int ZC>
void launch_t(Ctx* c, const FwdArgs<T>& a, cudaStream_t s) {
  const int grid = (a.n + BLOCK - 1) / BLOCK;
  if (c->has_lam3)
    k_tersoff<T, NS, ZC, true><<<grid, BLOCK, 0, s>>>(a);
  else
    k_tersoff<T, NS, ZC, false><<<grid, BLOCK, 0, s>>>(a);
}

// Register capacity of the short list: the smallest instance holding the
// largest short list seen at the last build; atoms with longer short lists
// take the general path.
template <class T, int NS>
void launch_zc(Ctx* c, const FwdArgs<T>& a, int zc, cudaStream_t s) {
  if (zc <= 4)
    launch_t<T, NS, 4>(c, a, s);
  else
    launch_t<T, NS, 8>(c, a, s);
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
  a.filt2 = filt_ptr<T>(c);
  const double scale = ldexp(1.0, c->grid.fix_shift);
  for (int q = 0; q < 3; ++q) {
    a.h[q] = (T)c->grid.h[q];
    a.hq[q] = (int)llrint(c->grid.h[q] * scale);
  }
  a.qinv = ldexpf(1.0f, -c->grid.fix_shift);
  a.f = f;
  a.acc = acc;
  a.eatom = eatom;
  a.flags = c->d_flags;
  const int zc = c->max_short;
  switch (c->ns) {
    case 1: launch_zc<T, 1>(c, a, zc, s); break;
    case 2: launch_zc<T, 2>(c, a, zc, s); break;
    default: launch_zc<T, 0>(c, a, zc, s); break;
  }
  c->launches++;
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

}  // namespace fwd
}  // namespace tgb

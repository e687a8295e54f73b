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

// Atoms with more than 8 bonds inside the cutoffs (bucket 2), when they are
// over 0.5% of the atoms (e.g. SiC): the slot-cached wide kernel, on the
// launch's stream after the main launch. A grid of a few waves loops over the
// bucket (its size lives on the device).
template <class T, int NS, bool BATCH = false>
void launch_wide(Ctx* c, const FwdArgs<T>& a, cudaStream_t s) {
  FwdArgs<T> b2 = a;
  b2.order = c->d_bucket + 2 * (size_t)c->n;
  b2.n_items = c->d_flags + flag_bucket(2);
  b2.order2 = b2.order3 = nullptr;
  b2.n_items2 = b2.n_items3 = nullptr;
  b2.identity = 0;
  const size_t dyn = wide_slot_bytes(sizeof(T));
  const int cap = (c->n_sm > 0 ? c->n_sm : 152) * 8;
  const int need = (c->nbucket[2] + WIDE_BLOCK - 1) / WIDE_BLOCK + 1;
  const int grid = need < cap ? need : cap;
  void (*k)(FwdArgs<T>) =
      c->has_lam3 ? k_tersoff_wide<T, NS, true, BATCH> : k_tersoff_wide<T, NS, false, BATCH>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  k<<<grid, WIDE_BLOCK, dyn, s>>>(b2);
  c->launches++;
}

// Energy/virial mode of a force launch (the EV parameter of k_tersoff).
template <class T, bool BATCH>
int ev_mode(const FwdArgs<T>& a) {
  if (BATCH) return 2;
  if (a.acc != nullptr) return a.virial ? 2 : 1;
  return a.eatom != nullptr ? 1 : 0;
}

// Grids are fixed by the atom count (the bucket sizes live on the device), so
// the launches can be captured in a CUDA graph and replayed across builds.
template <class T, int NS, int ZC, bool BATCH = false>
void launch_t(Ctx* c, const FwdArgs<T>& a, int grid, cudaStream_t s) {
  if (grid <= 0) return;
  if (sizeof(T) == 4 && NS == 1 && !BATCH && comp_atom_sums(c)) {
    launch_forward_cs(c, &a, ZC, grid, s);
    return;
  }
  // forces only, or energy without the virial (MD steps, with or without
  // thermo): the instances with less bookkeeping
  const int evm = ev_mode<T, BATCH>(a);
  if (ZC == 4 && !BATCH && evm == 0) {
    if (c->has_lam3)
      launch_pdl(k_tersoff<T, NS, ZC, 1, false, false, 0>, grid, BLOCK, 0, s, a);
    else if (c->sym_table)
      launch_pdl(k_tersoff<T, NS, ZC, 2, false, false, 0>, grid, BLOCK, 0, s, a);
    else
      launch_pdl(k_tersoff<T, NS, ZC, 0, false, false, 0>, grid, BLOCK, 0, s, a);
  } else if (ZC == 4 && !BATCH && evm == 1) {
    if (c->has_lam3)
      launch_pdl(k_tersoff<T, NS, ZC, 1, false, false, 1>, grid, BLOCK, 0, s, a);
    else if (c->sym_table)
      launch_pdl(k_tersoff<T, NS, ZC, 2, false, false, 1>, grid, BLOCK, 0, s, a);
    else
      launch_pdl(k_tersoff<T, NS, ZC, 0, false, false, 1>, grid, BLOCK, 0, s, a);
  } else if (c->has_lam3) {
    launch_pdl(k_tersoff<T, NS, ZC, 1, BATCH>, grid, BLOCK, 0, s, a);
  } else if (c->sym_table) {
    launch_pdl(k_tersoff<T, NS, ZC, 2, BATCH>, grid, BLOCK, 0, s, a);
  } else {
    launch_pdl(k_tersoff<T, NS, ZC, 0, BATCH>, grid, BLOCK, 0, s, a);
  }
  c->launches++;
}

// Launches per bucket (built with the list: the number of list entries inside
// the filter radii themselves, without the margin). Bucket 0 (at most 4) runs
// with register capacity 4. Bucket 1 (5 to 8) runs with capacity 8, on a side
// stream next to the main launch, when it holds over 5% of the atoms (e.g.
// SiC, where Si-Si second neighbours straddle the cutoff); otherwise it is
// appended to the capacity-4 launch. Every launch masks the stored short list
// (radius plus margin) by the cutoffs at each step; atoms with more entries
// inside than the capacity, and bucket 2, take the general path.
// Grid of a force launch: one thread per item, or (launch option) a number of
// waves of the blocks that fit on all SMs at once (resident blocks per SM from
// the kernel's launch bounds), the kernel looping over the items.
inline int force_grid(const Ctx* c, int zc, int evm) {
  const int full = (c->n + BLOCK - 1) / BLOCK;
  if (c->opt_waves <= 0 || c->n_sm <= 0) return full;
  // the blocks of this instance resident on one SM (its launch bound)
  const int resident = c->n_sm * fwd_min_blocks(zc <= 4 ? 4 : 8, zc <= 4 ? evm : 2,
                                                c->precision == TERSOFF_FP64);
  const int g = c->opt_waves * resident;
  return g < full ? g : full;
}

// The four-lane kernel takes the main launch when the launch option asks for
// it (tersoff_set_lanes(4), or the autotuner's choice) and the context is
// eligible (mixed path, one or two species, a single system). Automatic
// means one thread per atom: on the 512,000-atom Si benchmark the four-lane
// launch executes 43% more instructions at a 21% higher IPC and is slower.
template <class T, int NS, bool BATCH>
bool use_quad(const Ctx* c) {
  if (BATCH || sizeof(T) != 4 || NS < 1 || NS > 2 || comp_atom_sums(c) || c->n == 0) return false;
  return c->opt_quad == 1;
}

template <class T, int NS, bool BATCH = false>
void launch_buckets(Ctx* c, FwdArgs<T> a, cudaStream_t s) {
  if (use_quad<T, NS, BATCH>(c)) {
    TimedRegion tr(c, 0, s);
    const bool ev = a.acc != nullptr || a.eatom != nullptr;
    FwdArgs<T> aq = a;
    aq.identity = 1;
    launch_forward_quad(c, &aq, ev, s);
    // the atoms it left (more than four bonds inside the cutoffs, general
    // path): the per-thread kernel over the leftover list, one block per SM
    // looping over it; its last block zeroes the list's count
    FwdArgs<T> bl = a;
    bl.order = c->d_left;
    bl.n_items = c->d_flags + FLAG_LEFT;
    bl.order2 = bl.order3 = nullptr;
    bl.n_items2 = bl.n_items3 = nullptr;
    bl.identity = 0;
    bl.left_reset = 1;
    launch_t<T, NS, 8, BATCH>(c, bl, c->n_sm > 0 ? c->n_sm : 152, s);
    return;
  }
  const int dec = bucket_decisions(c);
  const bool split1 = (dec & 1) != 0;
  const bool fork = split1 && c->side != nullptr;
  cudaStream_t s2 = s;
  if (fork) {
    cudaEventRecord(c->ev_fork, s);
    cudaStreamWaitEvent(c->side, c->ev_fork, 0);
    s2 = c->side;
  }
  if (split1) {
    FwdArgs<T> b1 = a;
    b1.order = c->d_bucket + 1 * (size_t)c->n;
    b1.n_items = c->d_flags + flag_bucket(1);
    b1.order2 = b1.order3 = nullptr;
    b1.n_items2 = b1.n_items3 = nullptr;
    b1.identity = 0;
    launch_t<T, NS, 8, BATCH>(c, b1, force_grid(c, 8, ev_mode<T, BATCH>(a)), s2);
  }
  // bucket 0, then bucket 1 (unless split off), then bucket 2 (general path)
  const bool wide = (dec & 2) != 0;
  FwdArgs<T> b0 = a;
  b0.order = c->d_bucket;
  b0.n_items = c->d_flags + flag_bucket(0);
  b0.order2 = split1 ? nullptr : c->d_bucket + 1 * (size_t)c->n;
  b0.n_items2 = split1 ? nullptr : c->d_flags + flag_bucket(1);
  b0.order3 = wide ? nullptr : c->d_bucket + 2 * (size_t)c->n;
  b0.n_items3 = wide ? nullptr : c->d_flags + flag_bucket(2);
  // all buckets in one launch: atoms in index order (spatial order, and no
  // indirection); atoms with longer lists take the masked or general path
  b0.identity = (split1 || wide) ? 0 : 1;
  {
    TimedRegion tr(c, 0, s);
    launch_t<T, NS, 4, BATCH>(c, b0, force_grid(c, 4, ev_mode<T, BATCH>(a)), s);
    if (wide) launch_wide<T, NS, BATCH>(c, a, s);
  }
  if (fork) {
    cudaEventRecord(c->ev_join, c->side);
    cudaStreamWaitEvent(s, c->ev_join, 0);
  }
}

template <class T>
FwdArgs<T> make_args(Ctx* c, double* f, double* acc, double* eatom, bool virial = true) {
  FwdArgs<T> a;
  a.virial = virial ? 1 : 0;
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
  a.near2 = c->d_near32;
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
  // ablation ABLATE_NO_SHORT: the stored short list is never valid
  a.dlim2 = (c->ablate & 1) ? -1.0f : (float)(0.25 * c->margin * c->margin);
  a.all_general = (c->ablate & 2) ? 1 : 0;
  a.f = f;
  a.contrib = c->d_contrib;
  a.rev = c->d_rev;
  a.kmask = c->d_kmask;
  a.atomic_mode = (c->scatter_atomic || comp_atom_sums(c)) ? 1 : 0;
  a.own = c->d_own;
  a.acc = acc;
  a.eatom = eatom;
  a.flags = c->d_flags;
  a.sys = c->d_sys;
  a.atom_sys = c->d_atom_sys;
  a.vatom = c->d_vatom;
  a.order = c->d_bucket;
  a.n_items = c->d_flags + flag_bucket(0);
  a.order2 = a.order3 = nullptr;
  a.n_items2 = a.n_items3 = nullptr;
  a.identity = 1;
  a.left = c->d_left;
  a.left_reset = 0;
  return a;
}

// Ablation TERSOFF_ABLATE_FASTFWD: the fast-forward lane scheme over the full
// skin list, one launch over all atoms in index order.
template <class T, int NS>
void launch_ffwd(Ctx* c, const FwdArgs<T>& a, cudaStream_t s) {
  const int grid = (c->n + BLOCK - 1) / BLOCK;
  TimedRegion tr(c, 0, s);
  if (c->has_lam3)
    k_tersoff_ffwd<T, NS, true><<<grid, BLOCK, 0, s>>>(a);
  else
    k_tersoff_ffwd<T, NS, false><<<grid, BLOCK, 0, s>>>(a);
  c->launches++;
}

template <class T>
int launch_prec(Ctx* c, double* f, double* acc, double* eatom, cudaStream_t s,
                bool virial = true) {
  FwdArgs<T> a = make_args<T>(c, f, acc, eatom, virial);
  if (c->ablate & TERSOFF_ABLATE_FASTFWD) {
    switch (c->ns) {
      case 1: launch_ffwd<T, 1>(c, a, s); break;
      case 2: launch_ffwd<T, 2>(c, a, s); break;
      default: launch_ffwd<T, 0>(c, a, s); break;
    }
    TGB_CUDA(c, cudaGetLastError());
    return TERSOFF_OK;
  }
  switch (c->ns) {
    case 1: launch_buckets<T, 1>(c, a, s); break;
    case 2: launch_buckets<T, 2>(c, a, s); break;
    default: launch_buckets<T, 0>(c, a, s); break;
  }
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

// Batch of systems: the same bucketed launches as for one system (register
// capacity 4 for the atoms with at most 4 bonds inside the cutoffs, capacity
// 8 on the side stream for those with 5 to 8 when they are over 5%, the
// slot-cached wide kernel for the rest when they are over 0.5%), with
// per-system shifts and per-atom energy and virial for the per-system sums;
// runtime species count.
template <class T>
int launch_batch(Ctx* c, double* f, cudaStream_t s) {
  // energy and virial come from the per-atom stores: no block reduction
  FwdArgs<T> a = make_args<T>(c, f, nullptr, c->d_eatom);
  if (c->n > 0) launch_buckets<T, 0, true>(c, a, s);
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

}  // namespace fwd
}  // namespace tgb

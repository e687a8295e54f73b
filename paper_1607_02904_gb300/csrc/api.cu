// C ABI entry points (include/tersoff.h): argument checks, device buffers owned
// by the context, and the launch sequences of the compute and MD calls.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>

#include "internal.cuh"

namespace tgb {

int fail(Ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(Ctx* c, cudaError_t e, const char* where) {
  cudaGetLastError();  // do not leave a (non-sticky) error for the next caller
  std::string m = std::string("CUDA error ") + cudaGetErrorName(e) + " (" +
                  cudaGetErrorString(e) + ") in " + where;
  return fail(c, TERSOFF_E_CUDA, m);
}

static cudaEvent_t take_event(Ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// During stream capture the event records become graph nodes (external
// records) and the pair is kept with the graph, read after every replay.
static void record(Ctx* c, cudaEvent_t e, cudaStream_t s) {
  if (c->capturing)
    cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else
    cudaEventRecord(e, s);
}

TimedRegion::TimedRegion(Ctx* c_, int kind_, cudaStream_t s_) : c(c_), kind(kind_), s(s_) {
  if (!c->timing) return;
  a = take_event(c);
  b = take_event(c);
  if (a) record(c, a, s);
}

TimedRegion::~TimedRegion() {
  if (!c->timing || !a || !b) return;
  record(c, b, s);
  (c->timer_sink ? c->timer_sink : &c->pending)->push_back({kind, a, b});
}

// adds the elapsed times of a replayed graph's timer pairs (events stay with
// the graph)
static void fold_graph_timers(Ctx* c) {
  for (auto& p : c->graph.timers) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->t_ms[p.kind] += ms;
      c->t_count[p.kind] += 1;
    }
  }
}

static void drop_graph(Ctx* c) {
  if (c->graph.exec) cudaGraphExecDestroy(c->graph.exec);
  c->graph.exec = nullptr;
  for (auto& p : c->graph.timers) {
    c->ev_pool.push_back(p.a);
    c->ev_pool.push_back(p.b);
  }
  c->graph.timers.clear();
  c->graph.gen = -1;
}

int fold_timing(Ctx* c) {
  for (auto& p : c->pending) {
    cudaEventSynchronize(p.b);
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->t_ms[p.kind] += ms;
      c->t_count[p.kind] += 1;
    }
    c->ev_pool.push_back(p.a);
    c->ev_pool.push_back(p.b);
  }
  c->pending.clear();
  return TERSOFF_OK;
}

namespace {

// Metal units: 1 amu A^2 / ps^2 in eV, and its inverse (force eV/A over mass
// amu in A/ps^2).
constexpr double MVV2E = 1.0364269e-4;
constexpr double FTM2V = 1.0 / MVV2E;
constexpr double PI = 3.14159265358979323846;

template <class T>
int dev_alloc(Ctx* c, T** p, size_t count) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  if (count == 0) count = 1;
  TGB_CUDA(c, cudaMalloc((void**)p, sizeof(T) * count));
  return TERSOFF_OK;
}

int ensure_atoms(Ctx* c, int n) {
  if ((size_t)n <= c->atoms_alloc && c->d_types) return TERSOFF_OK;
  size_t m = (size_t)n;
  int st;
  if ((st = dev_alloc(c, &c->d_types, m))) return st;
  if ((st = dev_alloc(c, &c->d_cnt, m))) return st;
  if ((st = dev_alloc(c, &c->d_origin, 3 * m))) return st;
  if ((st = dev_alloc(c, &c->d_cell_of, m))) return st;
  if ((st = dev_alloc(c, &c->d_cell_atoms, m))) return st;
  if ((st = dev_alloc(c, &c->d_pos32, m))) return st;
  if ((st = dev_alloc(c, &c->d_posc, m))) return st;
  if ((st = dev_alloc(c, &c->d_kmask, m))) return st;
  if ((st = dev_alloc(c, &c->d_zw, m))) return st;
  if ((st = dev_alloc(c, &c->d_fine, m))) return st;
  if (!c->d_zbins && (st = dev_alloc(c, &c->d_zbins, (size_t)3 * 64))) return st;
  if ((st = dev_alloc(c, &c->d_posq, m))) return st;
  if ((st = dev_alloc(c, &c->d_pos64, m))) return st;
  if ((st = dev_alloc(c, &c->d_fbuf, 3 * m))) return st;
  if ((st = dev_alloc(c, &c->d_gf32, 3 * m))) return st;
  if ((st = dev_alloc(c, &c->d_qorg, 3 * m))) return st;
  if ((st = dev_alloc(c, &c->d_qref, m))) return st;
  if ((st = dev_alloc(c, &c->d_zcnt, m))) return st;
  if ((st = dev_alloc(c, &c->d_bucket, 3 * m))) return st;
  if ((st = dev_alloc(c, &c->d_left, m))) return st;
  if ((st = dev_alloc(c, &c->d_extra, 3 * (m ? m : 1)))) return st;
  TGB_CUDA(c, cudaMemset(c->d_extra, 0, sizeof(double) * 3 * (m ? m : 1)));
  c->atoms_alloc = m;
  c->nbr_alloc = 0;  // list storage depends on n
  return TERSOFF_OK;
}

int ensure_nbr(Ctx* c) {
  // at least 8 slots per atom: the force kernel loads up to 8 short-list
  // entries before it reads the count
  size_t need = (size_t)(c->cap > 8 ? c->cap : 8) * (size_t)c->n;
  // a short list never exceeds the skin list; reverse slots are bytes
  c->zs_cap = c->cap < 255 ? c->cap : 255;
  int st;
  if (!(need <= c->nbr_alloc && c->d_nbr && c->d_short)) {
    if ((st = dev_alloc(c, &c->d_nbr, need))) return st;
    if ((st = dev_alloc(c, &c->d_short, need))) return st;
    if ((st = dev_alloc(c, &c->d_rev, need))) return st;
    c->nbr_alloc = need;
    c->contrib_alloc = 0;
  }
  // per-slot force contributions of the current precision; at least 8 slots
  // per atom, like the lists: the gather loads the first 4 slots of a column
  // before it reads the count
  const size_t e4 = c->precision == TERSOFF_MIXED ? 16 : 32;
  const size_t bytes = e4 * (size_t)(c->zs_cap > 8 ? c->zs_cap : 8) * (size_t)c->n;
  if (c->contrib_alloc < bytes || c->contrib_prec != c->precision || !c->d_contrib) {
    cudaFree(c->d_contrib);
    cudaFree(c->d_own);
    c->d_contrib = c->d_own = nullptr;
    TGB_CUDA(c, cudaMalloc(&c->d_contrib, bytes ? bytes : 16));
    TGB_CUDA(c, cudaMalloc(&c->d_own, e4 * (c->n ? c->n : 1)));
    TGB_CUDA(c, cudaMemset(c->d_own, 0, e4 * (c->n ? c->n : 1)));
    c->contrib_alloc = bytes;
    c->contrib_prec = c->precision;
  }
  return TERSOFF_OK;
}

bool valid_precision(int p) { return p == TERSOFF_FP64 || p == TERSOFF_MIXED; }

// Build grid geometry on the host.
int setup_grid(Ctx* c, const double* box, double r_list) {
  Grid& g = c->grid;
  double hmax = 0.0;
  for (int a = 0; a < 3; ++a) {
    if (!(box[a] > 0.0) || !std::isfinite(box[a]))
      return fail(c, TERSOFF_E_INVALID_ARG, "box edges must be positive and finite");
    if (box[a] < 2.0 * r_list)
      return fail(c, TERSOFF_E_BOX_TOO_SMALL,
                  "box edge shorter than twice the neighbour-list radius");
    int nc = (int)std::floor(box[a] / r_list);
    if (nc < 2) nc = 2;
    if (nc > 1024) nc = 1024;
    g.nc[a] = nc;
    g.L[a] = box[a];
    g.invL[a] = 1.0 / box[a];
    g.h[a] = box[a] / nc;
    g.invh[a] = nc / box[a];
    hmax = std::fmax(hmax, g.h[a]);
  }
  // offsets u = x - o stay within [-8, h + 8) A between rebuilds; 2^S such
  // that (h + 8) 2^S < 2^30 keeps differences inside int32
  g.fix_shift = (int)std::floor(30.0 - std::log2(hmax + 8.0));
  return TERSOFF_OK;
}

int read_flags(Ctx* c, cudaStream_t s) {
  TGB_CUDA(c, cudaMemcpyAsync(c->h_flags, c->d_flags, sizeof(int) * FLAG_COUNT,
                              cudaMemcpyDeviceToHost, s));
  TGB_CUDA(c, cudaStreamSynchronize(s));
  return TERSOFF_OK;
}

// neighbour build (skin list, short list, displacement references) with
// overflow regrow; synchronises s once per attempt
int build_list(Ctx* c, const double* x, cudaStream_t s) {
  for (int attempt = 0; attempt < 4; ++attempt) {
    int st = ensure_nbr(c);
    if (st) return st;
    TGB_CUDA(c, cudaMemsetAsync(c->d_flags, 0, sizeof(int) * FLAG_BUILD_WORDS, s));
    TGB_CUDA(c, cudaMemsetAsync(c->d_flags + FLAG_NONFINITE, 0, sizeof(int), s));
    TGB_CUDA(c, cudaMemsetAsync(c->d_flags + FLAG_OVF_ANY, 0, sizeof(int), s));
    if ((st = launch_neighbor_build(c, x, s))) return st;
    if ((st = read_flags(c, s))) return st;
    if (c->h_flags[FLAG_NONFINITE])
      return fail(c, TERSOFF_E_NONFINITE, "non-finite position in neighbour build");
    c->max_cnt = c->h_flags[FLAG_OVERFLOW];
    c->max_short = c->h_flags[FLAG_SHORT_MAX];
    for (int b = 0; b < 3; ++b) c->nbucket[b] = c->h_flags[flag_bucket(b)];
    if (c->max_cnt <= c->cap) {
      c->have_list = true;
      c->steps_since_build = 0;
      return TERSOFF_OK;
    }
    // grow with headroom for atoms entering the skin before the next build
    c->cap = c->max_cnt + c->max_cnt / 4 + 4;
    c->gen++;
  }
  return fail(c, TERSOFF_E_NEIGH_OVERFLOW, "neighbour capacity could not be grown");
}

// the same build without host synchronisation (inside MD sequences that may be
// captured): capacity overflow and non-finite input raise sticky flags
int build_list_async(Ctx* c, const double* x, cudaStream_t s) {
  TGB_CUDA(c, cudaMemsetAsync(c->d_flags, 0, sizeof(int) * FLAG_BUILD_WORDS, s));
  return launch_neighbor_build(c, x, s);
}

int check_ctx(Ctx* c) {
  if (!c) return TERSOFF_E_INVALID_ARG;
  TGB_CUDA(c, cudaSetDevice(c->device));
  return TERSOFF_OK;
}

}  // namespace
}  // namespace tgb

using tgb::Ctx;

static Ctx* C(tersoff_ctx* p) { return p ? &p->impl : nullptr; }

extern "C" {

int tersoff_create(tersoff_ctx** out, int precision) {
  if (!out) return TERSOFF_E_INVALID_ARG;
  *out = nullptr;
  if (!tgb::valid_precision(precision)) return TERSOFF_E_INVALID_ARG;
  tersoff_ctx* p = new tersoff_ctx();
  Ctx* c = &p->impl;
  c->precision = precision;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete p;
    return TERSOFF_E_CUDA;
  }
  if (cudaMalloc(&c->d_flags, sizeof(int) * tgb::FLAG_COUNT) != cudaSuccess ||
      cudaMallocHost(&c->h_flags, sizeof(int) * tgb::FLAG_COUNT) != cudaSuccess ||
      cudaMalloc(&c->d_acc, sizeof(double) * tgb::ACC_LEN) != cudaSuccess ||
      cudaMalloc(&c->d_coef, sizeof(double) * 2 * TERSOFF_MAX_SPECIES) != cudaSuccess) {
    cudaFree(c->d_flags);
    cudaFreeHost(c->h_flags);
    delete p;
    return TERSOFF_E_CUDA;
  }
  cudaMemset(c->d_flags, 0, sizeof(int) * tgb::FLAG_COUNT);
  cudaMemset(c->d_acc, 0, sizeof(double) * tgb::ACC_LEN);
  if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
    c->n_sm = 0;
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    c->cap_stream = nullptr;
  if (cudaStreamCreateWithFlags(&c->body_stream, cudaStreamNonBlocking) != cudaSuccess)
    c->body_stream = nullptr;
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    c->side = nullptr;
  }
  *out = p;
  return TERSOFF_OK;
}

int tersoff_destroy(tersoff_ctx* p) {
  if (!p) return TERSOFF_OK;
  Ctx* c = &p->impl;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  void* bufs[] = {c->d_rec64, c->d_rec32, c->d_raw64, c->d_raw32, c->d_filt64, c->d_filt32, c->d_near32,
                  c->d_types, c->d_cnt, c->d_nbr, c->d_origin, c->d_cell_of, c->d_cell_count, c->d_cell_start,
                  c->d_cell_fill, c->d_cell_atoms, c->d_scan_tmp, c->d_bintab, c->d_pos32, c->d_posc, c->d_kmask, c->d_zw, c->d_fine, c->d_zbins, c->d_posq,
                  c->d_pos64, c->d_flags, c->d_acc, c->d_fbuf, c->d_stage, c->d_thermo,
                  c->d_coef, c->d_qorg, c->d_qref, c->d_short, c->d_zcnt, c->d_trow,
                  c->d_bucket, c->d_left, c->d_snap, c->d_rev, c->d_contrib, c->d_own,
                  c->d_extra, c->d_geo, c->d_sys, c->d_atom_sys, c->d_sys_off, c->d_vatom,
                  c->d_eatom, c->d_gf32};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (c->h_flags) cudaFreeHost(c->h_flags);
  tgb::drop_graph(c);
  tgb::fold_timing(c);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->body_stream) cudaStreamDestroy(c->body_stream);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  delete p;
  return TERSOFF_OK;
}

const char* tersoff_last_error(const tersoff_ctx* p) {
  if (!p) return "null context";
  return p->impl.err.c_str();
}

int tersoff_set_precision(tersoff_ctx* p, int precision) {
  Ctx* c = C(p);
  if (!c) return TERSOFF_E_INVALID_ARG;
  if (!tgb::valid_precision(precision))
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "precision must be TERSOFF_FP64 or TERSOFF_MIXED");
  c->precision = precision;
  c->gen++;
  return TERSOFF_OK;
}

int tersoff_params(tersoff_ctx* p, int ns, const double* table) {
  Ctx* c = C(p);
  int st = tgb::check_ctx(c);
  if (st) return st;
  if (ns < 1 || ns > TERSOFF_MAX_SPECIES || !table)
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "n_species must be in [1, 4] and table non-null");
  const int nrec = ns * ns * ns;
  for (int r = 0; r < nrec; ++r) {
    const double* t = table + (size_t)r * TERSOFF_NPARAM;
    for (int f = 0; f < TERSOFF_NPARAM; ++f)
      if (!std::isfinite(t[f])) return tgb::fail(c, TERSOFF_E_INVALID_ARG, "non-finite parameter");
    double m = t[TERSOFF_P_M];
    if (m < 1.0 || m > 16.0 || m != std::floor(m))
      return tgb::fail(c, TERSOFF_E_INVALID_ARG, "m must be an integer in [1, 16]");
    if (!(t[TERSOFF_P_D_CUT] > 0.0) || !(t[TERSOFF_P_N] > 0.0) || !(t[TERSOFF_P_D] != 0.0) ||
        !(t[TERSOFF_P_R] > t[TERSOFF_P_D_CUT]))
      return tgb::fail(c, TERSOFF_E_INVALID_ARG, "need D > 0, R > D, n > 0, d != 0");
  }
  std::vector<double> r64((size_t)nrec * tgb::RSTRIDE, 0.0);
  std::vector<float> r32((size_t)nrec * tgb::RSTRIDE, 0.0f);
  bool lam3 = false;
  for (int r = 0; r < nrec; ++r) {
    const double* t = table + (size_t)r * TERSOFF_NPARAM;
    double* o = &r64[(size_t)r * tgb::RSTRIDE];
    const double gam = t[TERSOFF_P_GAMMA], cc = t[TERSOFF_P_C], dd = t[TERSOFF_P_D];
    const double R = t[TERSOFF_P_R], D = t[TERSOFF_P_D_CUT];
    o[tgb::K_GAMMA] = gam;
    o[tgb::K_GC2D2] = gam * cc * cc / (dd * dd);
    o[tgb::K_G2C2] = 2.0 * gam * cc * cc;
    o[tgb::K_D2] = dd * dd;
    o[tgb::K_H] = t[TERSOFF_P_H];
    o[tgb::K_LAM3] = t[TERSOFF_P_LAMBDA3];
    o[tgb::K_M] = t[TERSOFF_P_M];
    o[tgb::K_R3] = R;
    o[tgb::K_PID3] = tgb::PI / (2.0 * D);
    o[tgb::K_DFC3] = -tgb::PI / (4.0 * D);
    o[tgb::K_RIN3] = R - D;
    o[tgb::K_ROUT3] = R + D;
    o[tgb::K_A] = t[TERSOFF_P_A];
    o[tgb::K_LAM1] = t[TERSOFF_P_LAMBDA1];
    o[tgb::K_LAM1LO] = 0.0;
    o[tgb::K_B] = t[TERSOFF_P_B];
    o[tgb::K_LAM2] = t[TERSOFF_P_LAMBDA2];
    o[tgb::K_LAM2LO] = 0.0;
    o[tgb::K_BETA] = t[TERSOFF_P_BETA];
    o[tgb::K_N] = t[TERSOFF_P_N];
    o[tgb::K_NINV2] = -1.0 / (2.0 * t[TERSOFF_P_N]);
    o[tgb::K_R2] = R;
    o[tgb::K_PID2] = tgb::PI / (2.0 * D);
    o[tgb::K_DFC2] = -tgb::PI / (4.0 * D);
    o[tgb::K_RIN2] = R - D;
    o[tgb::K_ROUT2] = R + D;
    o[tgb::K_ROUT3LO] = 0.0;
    o[tgb::K_ROUT2LO] = 0.0;
    if (t[TERSOFF_P_LAMBDA3] != 0.0) lam3 = true;
    float* of = &r32[(size_t)r * tgb::RSTRIDE];
    for (int k = 0; k < tgb::RSTRIDE; ++k) of[k] = (float)o[k];
    of[tgb::K_LAM1LO] = (float)(o[tgb::K_LAM1] - (double)of[tgb::K_LAM1]);
    of[tgb::K_LAM2LO] = (float)(o[tgb::K_LAM2] - (double)of[tgb::K_LAM2]);
    of[tgb::K_ROUT3LO] = (float)(o[tgb::K_ROUT3] - (double)of[tgb::K_ROUT3]);
    of[tgb::K_ROUT2LO] = (float)(o[tgb::K_ROUT2] - (double)of[tgb::K_ROUT2]);
  }
  // symmetric three-body terms: gamma, c, d, h of (i,j,k) equal those of
  // (i,k,j), and the R, D of f_C(r_ik) do not depend on j
  bool sym = !lam3;
  for (int i = 0; i < ns && sym; ++i)
    for (int j = 0; j < ns && sym; ++j)
      for (int k = 0; k < ns && sym; ++k) {
        const double* a = table + (size_t)((i * ns + j) * ns + k) * TERSOFF_NPARAM;
        const double* b = table + (size_t)((i * ns + k) * ns + j) * TERSOFF_NPARAM;
        const double* e = table + (size_t)((i * ns + k) * ns + k) * TERSOFF_NPARAM;
        for (int f : {TERSOFF_P_GAMMA, TERSOFF_P_C, TERSOFF_P_D, TERSOFF_P_H})
          if (a[f] != b[f]) sym = false;
        if (a[TERSOFF_P_R] != e[TERSOFF_P_R] || a[TERSOFF_P_D_CUT] != e[TERSOFF_P_D_CUT])
          sym = false;
      }
  // filter radius for (ti, tx): largest outer cutoff of any term in which an
  // atom of type tx is the bond partner j or the third atom k of a type-ti atom
  std::vector<double> filt((size_t)ns * ns, 0.0);
  std::vector<float> near32((size_t)ns * ns, 0.0f);
  double rmax = 0.0;
  for (int ti = 0; ti < ns; ++ti)
    for (int tx = 0; tx < ns; ++tx) {
      double rf = r64[(size_t)((ti * ns + tx) * ns + tx) * tgb::RSTRIDE + tgb::K_ROUT2];
      double rn = rf;  // and the smallest such cutoff
      for (int tj = 0; tj < ns; ++tj) {
        const double r3 = r64[(size_t)((ti * ns + tj) * ns + tx) * tgb::RSTRIDE + tgb::K_ROUT3];
        rf = std::fmax(rf, r3);
        rn = std::fmin(rn, r3);
      }
      filt[(size_t)ti * ns + tx] = rf;
      const double rl = std::fmax(rn - 2e-3, 0.0);
      near32[(size_t)ti * ns + tx] = (float)(rl * rl);
      rmax = std::fmax(rmax, rf);
    }
  std::vector<double> f64(filt.size());
  std::vector<float> f32(filt.size());
  for (size_t q = 0; q < filt.size(); ++q) {
    // a little above the radius so that rounding never drops a contributing atom
    double r = filt[q] * (1.0 + 1e-6);
    f64[q] = r * r;
    f32[q] = (float)(r * r);
  }
  if ((st = tgb::dev_alloc(c, &c->d_rec64, r64.size()))) return st;
  if ((st = tgb::dev_alloc(c, &c->d_rec32, r32.size()))) return st;
  if ((st = tgb::dev_alloc(c, &c->d_filt64, f64.size()))) return st;
  if ((st = tgb::dev_alloc(c, &c->d_filt32, f32.size()))) return st;
  if ((st = tgb::dev_alloc(c, &c->d_near32, near32.size()))) return st;
  TGB_CUDA(c, cudaMemcpy(c->d_rec64, r64.data(), sizeof(double) * r64.size(), cudaMemcpyHostToDevice));
  TGB_CUDA(c, cudaMemcpy(c->d_rec32, r32.data(), sizeof(float) * r32.size(), cudaMemcpyHostToDevice));
  {
    // raw records for the backward pass (table layout, both precisions)
    const size_t nraw = (size_t)nrec * TERSOFF_NPARAM;
    std::vector<float> raw32(nraw);
    for (size_t q = 0; q < nraw; ++q) raw32[q] = (float)table[q];
    if ((st = tgb::dev_alloc(c, &c->d_raw64, nraw))) return st;
    if ((st = tgb::dev_alloc(c, &c->d_raw32, nraw))) return st;
    TGB_CUDA(c, cudaMemcpy(c->d_raw64, table, sizeof(double) * nraw, cudaMemcpyHostToDevice));
    TGB_CUDA(c, cudaMemcpy(c->d_raw32, raw32.data(), sizeof(float) * nraw, cudaMemcpyHostToDevice));
  }
  TGB_CUDA(c, cudaMemcpy(c->d_filt64, f64.data(), sizeof(double) * f64.size(), cudaMemcpyHostToDevice));
  TGB_CUDA(c, cudaMemcpy(c->d_filt32, f32.data(), sizeof(float) * f32.size(), cudaMemcpyHostToDevice));
  TGB_CUDA(c, cudaMemcpy(c->d_near32, near32.data(), sizeof(float) * near32.size(),
                         cudaMemcpyHostToDevice));
  c->gen++;
  c->ns = ns;
  c->h_rec64 = r64;
  c->h_rec32 = r32;
  c->table.assign(table, table + (size_t)nrec * TERSOFF_NPARAM);
  c->filt = filt;
  c->has_lam3 = lam3;
  c->sym_table = sym;
  c->rmax_cut = rmax;
  c->have_list = false;
  return TERSOFF_OK;
}

int tersoff_neighbor_build(tersoff_ctx* p, const double* x, const int* types, int n,
                           const double* box, double r_list, void* stream) {
  tgb::NvtxRange nvtx_range("tersoff_neighbor_build");
  Ctx* c = C(p);
  int st = tgb::check_ctx(c);
  if (st) return st;
  if (c->ns == 0) return tgb::fail(c, TERSOFF_E_STATE, "tersoff_params must come first");
  if (n < 0 || n > tgb::MAX_ATOMS || (n > 0 && (!x || !types)) || !box)
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "bad atom arrays or count (max 2^26 atoms)");
  if (!(r_list > 0.0) || !std::isfinite(r_list))
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "r_list must be positive");
  if (r_list < c->rmax_cut)
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "r_list is below the potential's cutoff");
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = tgb::setup_grid(c, box, r_list))) return st;
  if ((st = tgb::upload_bin_tables(c, s))) return st;
  c->n_sys = 0;
  c->n = n;
  c->r_list = r_list;
  c->margin = 0.6 * (r_list - c->rmax_cut);
  c->have_list = false;
  c->gen++;
  if ((st = tgb::ensure_atoms(c, n))) return st;
  if (n > 0)
    TGB_CUDA(c, cudaMemcpyAsync(c->d_types, types, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
  // species range check on the device copy is folded into the build kernels'
  // parameter lookups; validate here on a host copy for clear errors
  if (n > 0) {
    std::vector<int> ht(n);
    TGB_CUDA(c, cudaMemcpyAsync(ht.data(), types, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
    TGB_CUDA(c, cudaStreamSynchronize(s));
    for (int i = 0; i < n; ++i)
      if (ht[i] < 0 || ht[i] >= c->ns)
        return tgb::fail(c, TERSOFF_E_INVALID_ARG, "species index out of range");
  }
  return tgb::build_list(c, x, s);
}

int tersoff_neighbor_build_batched(tersoff_ctx* p, const double* x, const int* types, int n,
                                   const int* sys_offsets, const double* boxes, int n_sys,
                                   double r_list, void* stream) {
  tgb::NvtxRange nvtx_range("tersoff_neighbor_build_batched");
  Ctx* c = C(p);
  int st = tgb::check_ctx(c);
  if (st) return st;
  if (c->ns == 0) return tgb::fail(c, TERSOFF_E_STATE, "tersoff_params must come first");
  if (n_sys < 1 || !sys_offsets || !boxes)
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "need n_systems >= 1, offsets and boxes");
  if (n < 0 || n > tgb::MAX_ATOMS || (n > 0 && (!x || !types)))
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "bad atom arrays or count (max 2^26 atoms)");
  if (!(r_list > 0.0) || !std::isfinite(r_list))
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "r_list must be positive");
  if (r_list < c->rmax_cut)
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "r_list is below the potential's cutoff");
  if (sys_offsets[0] != 0 || sys_offsets[n_sys] != n)
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "offsets must run from 0 to n");
  for (int q = 0; q < n_sys; ++q)
    if (sys_offsets[q + 1] < sys_offsets[q])
      return tgb::fail(c, TERSOFF_E_INVALID_ARG, "offsets must not decrease");
  // one cell grid per system, cells numbered consecutively
  std::vector<tgb::GridDev> geo(n_sys);
  std::vector<tgb::SysShift> shifts(n_sys);
  double hmax = 0.0;
  long cells = 0;
  for (int q = 0; q < n_sys; ++q) {
    tgb::GridDev& g = geo[q];
    g.cell_base = (int)cells;
    long nq = 1;
    for (int a = 0; a < 3; ++a) {
      const double L = boxes[3 * (size_t)q + a];
      if (!(L > 0.0) || !std::isfinite(L))
        return tgb::fail(c, TERSOFF_E_INVALID_ARG, "box edges must be positive and finite");
      if (L < 2.0 * r_list)
        return tgb::fail(c, TERSOFF_E_BOX_TOO_SMALL,
                         "a system's box edge is shorter than twice the neighbour-list radius");
      int nc = (int)std::floor(L / r_list);
      nc = nc < 2 ? 2 : (nc > 1024 ? 1024 : nc);
      g.nc[a] = nc;
      g.L[a] = L;
      g.invL[a] = 1.0 / L;
      g.h[a] = L / nc;
      g.invh[a] = nc / L;
      g.hf[a] = (float)g.h[a];
      hmax = std::fmax(hmax, g.h[a]);
      nq *= nc;
    }
    cells += nq;
    if (cells > (1L << 30))
      return tgb::fail(c, TERSOFF_E_INVALID_ARG, "too many list cells over the systems");
  }
  // the launch-wide grid carries only the fixed-point scale and hmax
  tgb::Grid& G = c->grid;
  for (int a = 0; a < 3; ++a) {
    G.nc[a] = 1;
    G.L[a] = G.h[a] = hmax;
    G.invL[a] = G.invh[a] = 1.0 / hmax;
  }
  G.fix_shift = (int)std::floor(30.0 - std::log2(hmax + 8.0));
  const double scale = std::ldexp(1.0, G.fix_shift);
  for (int q = 0; q < n_sys; ++q)
    for (int a = 0; a < 3; ++a) {
      shifts[q].hq[a] = (int)std::llrint(geo[q].h[a] * scale);
      shifts[q].hf[a] = (float)geo[q].h[a];
      shifts[q].h[a] = geo[q].h[a];
    }
  std::vector<int> asys((size_t)n);
  for (int q = 0; q < n_sys; ++q)
    for (int i = sys_offsets[q]; i < sys_offsets[q + 1]; ++i) asys[i] = q;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = tgb::dev_alloc(c, &c->d_geo, (size_t)n_sys))) return st;
  if ((st = tgb::dev_alloc(c, &c->d_sys, (size_t)n_sys))) return st;
  if ((st = tgb::dev_alloc(c, &c->d_sys_off, (size_t)n_sys + 1))) return st;
  if ((st = tgb::dev_alloc(c, &c->d_atom_sys, (size_t)n))) return st;
  if ((st = tgb::dev_alloc(c, &c->d_eatom, (size_t)n))) return st;
  if ((st = tgb::dev_alloc(c, &c->d_vatom, 6 * (size_t)n))) return st;
  TGB_CUDA(c, cudaMemcpy(c->d_geo, geo.data(), sizeof(tgb::GridDev) * n_sys,
                         cudaMemcpyHostToDevice));
  TGB_CUDA(c, cudaMemcpy(c->d_sys, shifts.data(), sizeof(tgb::SysShift) * n_sys,
                         cudaMemcpyHostToDevice));
  TGB_CUDA(c, cudaMemcpy(c->d_sys_off, sys_offsets, sizeof(int) * (n_sys + 1),
                         cudaMemcpyHostToDevice));
  if (n > 0)
    TGB_CUDA(c, cudaMemcpy(c->d_atom_sys, asys.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
  c->n_sys = n_sys;
  c->ncell_batch = cells;
  c->n = n;
  c->r_list = r_list;
  c->margin = 0.6 * (r_list - c->rmax_cut);
  c->have_list = false;
  c->gen++;
  if ((st = tgb::ensure_atoms(c, n))) return st;
  if (n > 0) {
    TGB_CUDA(c, cudaMemcpyAsync(c->d_types, types, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    std::vector<int> ht(n);
    TGB_CUDA(c, cudaMemcpyAsync(ht.data(), types, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
    TGB_CUDA(c, cudaStreamSynchronize(s));
    for (int i = 0; i < n; ++i)
      if (ht[i] < 0 || ht[i] >= c->ns)
        return tgb::fail(c, TERSOFF_E_INVALID_ARG, "species index out of range");
  }
  return tgb::build_list(c, x, s);
}

int tersoff_neighbor_capacity(const tersoff_ctx* p, int* capacity, int* max_count) {
  if (!p) return TERSOFF_E_INVALID_ARG;
  if (capacity) *capacity = p->impl.cap;
  if (max_count) *max_count = p->impl.max_cnt;
  return TERSOFF_OK;
}

int tersoff_set_neighbor_capacity(tersoff_ctx* p, int capacity) {
  Ctx* c = C(p);
  if (!c) return TERSOFF_E_INVALID_ARG;
  if (capacity < 1 || capacity > 4096)
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "capacity must be in [1, 4096]");
  c->cap = capacity;
  c->have_list = false;
  c->gen++;
  return TERSOFF_OK;
}

int tersoff_neighbor_export(tersoff_ctx* p, int* cnt, int* nbr, int cap, void* stream) {
  Ctx* c = C(p);
  int st = tgb::check_ctx(c);
  if (st) return st;
  if (!c->have_list) return tgb::fail(c, TERSOFF_E_STATE, "no neighbour list");
  if (cap < 1 || (c->n > 0 && (!cnt || !nbr)))
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "bad export buffers");
  if ((st = tgb::launch_neighbor_export(c, cnt, nbr, cap, (cudaStream_t)stream))) return st;
  if (c->max_cnt > cap)
    return tgb::fail(c, TERSOFF_E_NEIGH_OVERFLOW, "export capacity below the largest count");
  return TERSOFF_OK;
}

// forces of a batch of systems into f, per-system energy and virial (either
// may be NULL)
static int batch_impl(Ctx* c, const double* x, double* f, double* energies, double* virials,
                      cudaStream_t s) {
  int st;
  if ((st = tgb::ensure_nbr(c))) return st;
  if ((st = tgb::launch_pack_positions(c, x, false, s))) return st;
  TGB_CUDA(c, cudaMemsetAsync(c->d_acc, 0, sizeof(double) * tgb::ACC_LEN, s));
  TGB_CUDA(c, cudaMemsetAsync(c->d_flags + tgb::FLAG_EXTRA_STICKY, 0, sizeof(int), s));
  if ((st = tgb::launch_forward_batch(c, c->d_extra, s))) return st;
  if ((st = tgb::launch_gather(c, f, s))) return st;
  return tgb::launch_system_sums(c, energies, virials, s);
}

static int compute_impl(Ctx* c, const double* x, int n, double* energy, double* forces,
                        double* virial, double* eatom, cudaStream_t s) {
  int st = tgb::check_ctx(c);
  if (st) return st;
  if (!c->have_list) return tgb::fail(c, TERSOFF_E_STATE, "tersoff_neighbor_build must come first");
  if (c->n_sys > 0)
    return tgb::fail(c, TERSOFF_E_STATE, "the context holds a batch: use tersoff_compute_batched");
  if (n != c->n || (n > 0 && !x))
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "atom count differs from the neighbour build");
  double* f = forces ? forces : c->d_fbuf;
  if ((st = tgb::ensure_nbr(c))) return st;
  if ((st = tgb::launch_pack_positions(c, x, false, s))) return st;
  TGB_CUDA(c, cudaMemsetAsync(c->d_acc, 0, sizeof(double) * tgb::ACC_LEN, s));
  TGB_CUDA(c, cudaMemsetAsync(c->d_flags + tgb::FLAG_EXTRA_STICKY, 0, sizeof(int), s));
  if ((st = tgb::launch_forward(c, c->d_extra, c->d_acc, eatom, s))) return st;
  if ((st = tgb::launch_gather(c, f, s))) return st;
  if (energy)
    TGB_CUDA(c, cudaMemcpyAsync(energy, c->d_acc, sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (virial)
    TGB_CUDA(c, cudaMemcpy2DAsync(virial, sizeof(double), c->d_acc + tgb::ACC_STRIDE,
                                  sizeof(double) * tgb::ACC_STRIDE, sizeof(double), 6,
                                  cudaMemcpyDeviceToDevice, s));
  return TERSOFF_OK;
}

int tersoff_compute_batched(tersoff_ctx* p, const double* x, int n, double* energies,
                            double* forces, double* virials, void* stream) {
  tgb::NvtxRange nvtx_range("tersoff_compute_batched");
  Ctx* c = C(p);
  int st = tgb::check_ctx(c);
  if (st) return st;
  if (!c->have_list || c->n_sys == 0)
    return tgb::fail(c, TERSOFF_E_STATE, "tersoff_neighbor_build_batched must come first");
  if (n != c->n || (n > 0 && !x))
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "atom count differs from the neighbour build");
  return batch_impl(c, x, forces ? forces : c->d_fbuf, energies, virials, (cudaStream_t)stream);
}

int tersoff_compute(tersoff_ctx* p, const double* x, int n, double* energy, double* forces,
                    double* virial, void* stream) {
  tgb::NvtxRange nvtx_range("tersoff_compute");
  return compute_impl(C(p), x, n, energy, forces, virial, nullptr, (cudaStream_t)stream);
}

int tersoff_compute_peratom(tersoff_ctx* p, const double* x, int n, double* eatom,
                            void* stream) {
  tgb::NvtxRange nvtx_range("tersoff_compute_peratom");
  Ctx* c = C(p);
  if (!c) return TERSOFF_E_INVALID_ARG;
  if (!eatom && n > 0) return tgb::fail(c, TERSOFF_E_INVALID_ARG, "eatom is null");
  return compute_impl(c, x, n, nullptr, nullptr, nullptr, eatom, (cudaStream_t)stream);
}

int tersoff_backward(tersoff_ctx* p, const double* x, int n, const double* gE, const double* gF,
                     double* grad_x, double* grad_table, void* stream) {
  tgb::NvtxRange nvtx_range("tersoff_backward");
  Ctx* c = C(p);
  int st = tgb::check_ctx(c);
  if (st) return st;
  if (!c->have_list) return tgb::fail(c, TERSOFF_E_STATE, "tersoff_neighbor_build must come first");
  if (n != c->n || (n > 0 && !x))
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "atom count differs from the neighbour build");
  if (!gE) return tgb::fail(c, TERSOFF_E_INVALID_ARG, "gE is null");
  cudaStream_t s = (cudaStream_t)stream;
  if (grad_table) {
    const size_t nraw = (size_t)c->ns * c->ns * c->ns * TERSOFF_NPARAM;
    if ((st = tgb::launch_pack_positions(c, x, false, s))) return st;
    TGB_CUDA(c, cudaMemsetAsync(grad_table, 0, sizeof(double) * nraw, s));
    if ((st = tgb::launch_backward(c, gE, gF, grad_table, s))) return st;
  }
  if (grad_x) {
    if (c->n_sys > 0)
      st = batch_impl(c, x, grad_x, nullptr, nullptr, s);
    else
      st = compute_impl(c, x, n, nullptr, grad_x, nullptr, nullptr, s);
    if (st) return st;
    if ((st = tgb::launch_scale_forces(c, grad_x, gE, s))) return st;
    if (gF && (st = tgb::launch_hvp(c, gF, grad_x, s))) return st;
  }
  return TERSOFF_OK;
}

// The compute sequence with the force kernel's accumulators in the fixed
// scratch array (forces scattered with atomics, so no per-slot buffers); uses
// only buffers that the neighbour build has already sized.
int tersoff_compute_noalloc(tersoff_ctx* p, const double* x, int n, double* energy,
                            double* forces, double* virial, void* stream) {
  Ctx* c = C(p);
  if (!c) return TERSOFF_E_INVALID_ARG;
  if (n < 0 || n > TERSOFF_NOALLOC_MAX_ATOMS)
    return tgb::fail(c, TERSOFF_E_INVALID_ARG,
                     "tersoff_compute_noalloc: n exceeds TERSOFF_NOALLOC_MAX_ATOMS (65536)");
  int st = tgb::check_ctx(c);
  if (st) return st;
  if (!c->have_list) return tgb::fail(c, TERSOFF_E_STATE, "tersoff_neighbor_build must come first");
  if (c->n_sys > 0)
    return tgb::fail(c, TERSOFF_E_STATE, "the context holds a batch: use tersoff_compute_batched");
  if (n != c->n || (n > 0 && !x))
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "atom count differs from the neighbour build");
  double* scr = nullptr;
  size_t len = 0;
  if ((st = tgb::noalloc_scratch(c, &scr, &len))) return st;
  const size_t used = (size_t)tgb::ACC_LEN + 3 * (size_t)n;
  if (used > len) return tgb::fail(c, TERSOFF_E_INVALID_ARG, "fixed scratch too small");
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = tgb::launch_pack_positions(c, x, false, s))) return st;
  TGB_CUDA(c, cudaMemsetAsync(scr, 0, sizeof(double) * used, s));
  TGB_CUDA(c, cudaMemsetAsync(c->d_flags + tgb::FLAG_EXTRA_STICKY, 0, sizeof(int), s));
  // The force kernel also writes the context's status words FLAG_EXTRA and
  // (for atoms on the general path) FLAG_EXTRA_STICKY, which the gather of
  // tersoff_compute and the MD steps read. Both are rewritten before any such
  // read: every compute and MD call clears FLAG_EXTRA_STICKY and runs a force
  // launch (which sets FLAG_EXTRA) before its gather, and tersoff_md_step's
  // first step uses the caller's f, not a gather.
  const bool was_atomic = c->scatter_atomic;
  c->scatter_atomic = true;  // read by the launch below only
  st = tgb::launch_forward(c, scr + tgb::ACC_LEN, scr, nullptr, s);
  c->scatter_atomic = was_atomic;
  if (st) return st;
  return tgb::launch_noalloc_out(c, scr, n, forces, energy, virial, s);
}

// Rebuild threshold of the displacement trigger: (skin / 2)^2, the skin being
// the list radius beyond the largest cutoff.
static float skin_lim2(const Ctx* c) {
  const double skin = c->r_list - c->rmax_cut;
  return (float)(0.25 * (skin > 0.0 ? skin * skin : 0.0));
}

// Adds to the graph being captured on cs a neighbour rebuild that runs only if
// the largest displacement since the last build exceeds half the skin: a
// one-thread kernel sets the condition of an IF node whose body (captured on
// the context's body stream) holds the build. Returns the body's kernel count
// in *body_kernels.
static int enqueue_conditional_build(Ctx* c, const double* x, cudaStream_t cs,
                                     long long* body_kernels) {
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  TGB_CUDA(c, cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, nullptr, nullptr, nullptr));
  if (cst != cudaStreamCaptureStatusActive || !g || !c->body_stream)
    return tgb::fail(c, TERSOFF_E_STATE, "conditional rebuild outside a graph capture");
  cudaGraphConditionalHandle h;
  TGB_CUDA(c, cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
  int st = tgb::launch_decide_rebuild(c, skin_lim2(c), h, cs);
  if (st) return st;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  TGB_CUDA(c, cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &nd));
  // the node parameters are a C struct (zeroed storage, as the API requires)
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  std::memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams& prm = *reinterpret_cast<cudaGraphNodeParams*>(raw);
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = h;
  prm.conditional.type = cudaGraphCondTypeIf;
  prm.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  TGB_CUDA(c, cudaGraphAddNode(&node, g, deps, nullptr, nd, &prm));
  cudaGraph_t body = prm.conditional.phGraph_out[0];
  TGB_CUDA(c, cudaStreamBeginCaptureToGraph(c->body_stream, body, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal));
  const long long l0 = c->launches;
  st = tgb::build_list_async(c, x, c->body_stream);
  *body_kernels = c->launches - l0;
  cudaGraph_t captured = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(c->body_stream, &captured);
  if (st) return st;
  TGB_CUDA(c, ce);
  TGB_CUDA(c, cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1,
                                                  cudaStreamSetCaptureDependencies));
  return TERSOFF_OK;
}

// Enqueues nsteps velocity-Verlet steps. sync_builds: rebuild with a host
// check (eager); otherwise without host synchronisation (graph capture).
// snap (may be null): receives x, v, f as the first step reads them (the
// start state of a rerun)
static int enqueue_md(Ctx* c, double* x, double* v, double* f, double dt,
                      int nsteps, int rebuild_every, double* rows, double* thermo,
                      bool sync_builds, cudaStream_t s, double* snap = nullptr) {
  int st = TERSOFF_OK;
  const bool on_skin = rebuild_every == TERSOFF_REBUILD_ON_SKIN;
  if (rows) TGB_CUDA(c, cudaMemsetAsync(rows, 0, sizeof(double) * tgb::ACC_LEN * (size_t)nsteps, s));
  for (int step = 0; step < nsteps; ++step) {
    if (!on_skin) c->steps_since_build++;
    const bool rebuild = rebuild_every > 0 && c->steps_since_build >= rebuild_every;
    // opening half kick (merged with the previous step's closing one), drift
    double* ke_row =
        (rows && step > 0) ? rows + tgb::ACC_LEN * (size_t)(step - 1) + 7 * tgb::ACC_STRIDE : nullptr;
    // energy and virial only when thermo rows are requested
    double* acc = rows ? rows + tgb::ACC_LEN * (size_t)step : nullptr;
    {
      tgb::TimedRegion tr(c, 2, s);
      if ((st = tgb::launch_md_step(c, x, v, f, dt, step == 0 ? 1 : 2, !rebuild, ke_row,
                                    nullptr, s, step == 0 ? snap : nullptr)))
        return st;
    }
    if (rebuild) {
      {
        tgb::TimedRegion tr(c, 1, s);
        st = sync_builds ? tgb::build_list(c, x, s) : tgb::build_list_async(c, x, s);
      }
      if (st) return st;
      c->steps_since_build = 0;
      c->last_rebuilds++;
    } else if (on_skin) {
      tgb::TimedRegion tr(c, 1, s);
      if (sync_builds) {
        // host check of the displacement tracked by the step just enqueued
        if ((st = tgb::read_flags(c, s))) return st;
        float d2;
        std::memcpy(&d2, &c->h_flags[tgb::FLAG_DMAX], sizeof(float));
        if (d2 > skin_lim2(c)) {
          if ((st = tgb::build_list(c, x, s))) return st;
          c->last_rebuilds++;
        }
      } else {
        long long bk = 0;
        if ((st = enqueue_conditional_build(c, x, s, &bk))) return st;
        c->graph.body_kernels = bk;
        c->launches -= bk;  // counted per rebuild that runs
      }
    }
    // the thermo rows take the potential energy only: no virial
    if ((st = tgb::launch_forward(c, c->d_extra, acc, nullptr, s, false))) return st;
  }
  {
    tgb::TimedRegion tr(c, 2, s);
    double* ke_row =
        rows ? rows + tgb::ACC_LEN * (size_t)(nsteps - 1) + 7 * tgb::ACC_STRIDE : nullptr;
    if ((st = tgb::launch_final_kick(c, v, f, ke_row, s))) return st;
  }
  if (thermo && (st = tgb::launch_thermo_rows(c, rows, nsteps, tgb::MVV2E, thermo, s))) return st;
  return TERSOFF_OK;
}

static int md_impl(Ctx* c, double* x, double* v, double* f, int n, const double* mass,
                   double dt, int nsteps, int rebuild_every, double* thermo, cudaStream_t s) {
  if (c) c->fine_valid = false;  // the steps may rebuild the lists on the device
  int st = tgb::check_ctx(c);
  if (st) return st;
  if (!c->have_list) return tgb::fail(c, TERSOFF_E_STATE, "tersoff_neighbor_build must come first");
  if (c->n_sys > 0) return tgb::fail(c, TERSOFF_E_STATE, "MD runs on single-system contexts");
  if (n != c->n || (n > 0 && (!x || !v || !f)) || !mass || nsteps < 0 ||
      (rebuild_every < 0 && rebuild_every != TERSOFF_REBUILD_ON_SKIN) || !(dt > 0.0) ||
      !std::isfinite(dt))
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "bad MD arguments");
  c->last_rebuilds = 0;
  const bool on_skin = rebuild_every == TERSOFF_REBUILD_ON_SKIN;
  for (int t = 0; t < c->ns; ++t)
    if (!(mass[t] > 0.0)) return tgb::fail(c, TERSOFF_E_INVALID_ARG, "masses must be positive");
  if (n == 0 || nsteps == 0) return TERSOFF_OK;
  // per-species dt/2 * FTM2V / m, then masses
  double hc[2 * TERSOFF_MAX_SPECIES] = {0};
  for (int t = 0; t < c->ns; ++t) {
    hc[t] = 0.5 * dt * tgb::FTM2V / mass[t];
    hc[TERSOFF_MAX_SPECIES + t] = mass[t];
  }
  TGB_CUDA(c, cudaMemcpyAsync(c->d_coef, hc, sizeof(hc), cudaMemcpyHostToDevice, s));
  for (int t = 0; t < TERSOFF_MAX_SPECIES; ++t) {
    c->coef.c[t] = hc[t];
    c->coef.c2[t] = 2.0 * hc[t];
    c->coef.cf[t] = (float)hc[t];
    c->coef.c2f[t] = (float)(2.0 * hc[t]);
    c->coef.m[t] = hc[TERSOFF_MAX_SPECIES + t];
    c->coef.hmf[t] = (float)(0.5 * hc[TERSOFF_MAX_SPECIES + t]);
  }
  if ((st = tgb::ensure_nbr(c))) return st;
  double* rows = nullptr;
  if (thermo) {
    const size_t need = tgb::ACC_LEN * (size_t)nsteps;
    if (c->trow_alloc < need) {
      if ((st = tgb::dev_alloc(c, &c->d_trow, need))) return st;
      c->trow_alloc = need;
      c->gen++;
    }
    rows = c->d_trow;
  }
  TGB_CUDA(c, cudaMemsetAsync(c->d_flags + tgb::FLAG_BUILD_WORDS, 0,
                              sizeof(int) * (tgb::FLAG_COUNT - tgb::FLAG_BUILD_WORDS), s));
  if (!c->use_graphs || !c->cap_stream) {
    st = enqueue_md(c, x, v, f, dt, nsteps, rebuild_every, rows, thermo, true, s);
    if (st) return st;
    TGB_CUDA(c, cudaStreamSynchronize(s));
    return TERSOFF_OK;
  }
  // graph path: replay (capturing on a new shape), check; the graph's first
  // step writes the start state into the snapshot as it reads it
  const size_t m = 3 * (size_t)n;
  if (c->snap_alloc < 3 * m) {
    if ((st = tgb::dev_alloc(c, &c->d_snap, 3 * m))) return st;
    c->snap_alloc = 3 * m;
  }
  const int ssb0 = on_skin ? -1 : c->steps_since_build;
  auto& G = c->graph;
  const bool same = G.exec && G.gen == c->gen && G.x == x && G.v == v && G.f == f &&
                    G.snap == c->d_snap &&
                    G.thermo == thermo && G.dt == dt && G.nsteps == nsteps &&
                    G.rebuild_every == rebuild_every && G.ssb0 == ssb0 &&
                    G.precision == c->precision && G.timing == c->timing &&
                    G.decisions == tgb::bucket_decisions(c) &&
                    std::memcmp(&G.coef, &c->coef, sizeof(tgb::Coef)) == 0;
  if (!same) {
    tgb::drop_graph(c);
    cudaGraph_t graph = nullptr;
    // capture on the context's own stream (the caller's may be the legacy
    // default stream, which cannot be captured); replay on the caller's
    cudaStream_t cs = c->cap_stream;
    TGB_CUDA(c, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const long long l0 = c->launches;
    c->capturing = true;
    c->timer_sink = &G.timers;
    st = enqueue_md(c, x, v, f, dt, nsteps, rebuild_every, rows, thermo, false, cs, c->d_snap);
    c->capturing = false;
    c->timer_sink = nullptr;
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    cudaGetLastError();  // a failed capture leaves its error in the last-error slot
    if (st == TERSOFF_OK && ce != cudaSuccess) st = tgb::cuda_fail(c, ce, "cudaStreamEndCapture");
    if (st == TERSOFF_OK) {
      // node priorities (the side stream's small-bucket launches are high priority)
      ce = cudaGraphInstantiate(&G.exec, graph, cudaGraphInstantiateFlagUseNodePriority);
      if (ce != cudaSuccess) st = tgb::cuda_fail(c, ce, "cudaGraphInstantiate");
    }
    if (graph) cudaGraphDestroy(graph);
    if (st) {
      tgb::drop_graph(c);
      if (!on_skin) c->steps_since_build = ssb0;
      return st;
    }
    G.x = x;
    G.v = v;
    G.f = f;
    G.snap = c->d_snap;
    G.thermo = thermo;
    G.dt = dt;
    G.coef = c->coef;
    G.nsteps = nsteps;
    G.rebuild_every = rebuild_every;
    G.ssb0 = ssb0;
    G.precision = c->precision;
    G.timing = c->timing;
    G.gen = c->gen;
    G.decisions = tgb::bucket_decisions(c);
    G.kernels = c->launches - l0;
    c->launches = l0;
    c->last_rebuilds = 0;  // nothing ran yet
  } else if (!on_skin) {
    // host bookkeeping of the replayed sequence (the capture did the same)
    for (int step = 0; step < nsteps; ++step) {
      c->steps_since_build++;
      if (rebuild_every > 0 && c->steps_since_build >= rebuild_every) c->steps_since_build = 0;
    }
  }
  if (!on_skin) {
    // rebuild steps of the fixed period in this call
    int ssb = ssb0;
    for (int step = 0; step < nsteps; ++step)
      if (rebuild_every > 0 && ++ssb >= rebuild_every) {
        ssb = 0;
        c->last_rebuilds++;
      }
  }
  c->launches += G.kernels;
  TGB_CUDA(c, cudaGraphLaunch(G.exec, s));
  if ((st = tgb::read_flags(c, s))) return st;
  if (c->timing) tgb::fold_graph_timers(c);
  if (on_skin) {
    c->last_rebuilds = c->h_flags[tgb::FLAG_NREBUILD];
    c->launches += (long long)c->last_rebuilds * G.body_kernels;
  }
  const bool bad = c->h_flags[tgb::FLAG_OVF_ANY] || c->h_flags[tgb::FLAG_NONFINITE];
  if (!bad) {
    c->max_cnt = c->h_flags[tgb::FLAG_OVERFLOW];
    c->max_short = c->h_flags[tgb::FLAG_SHORT_MAX];
    for (int b = 0; b < 3; ++b) c->nbucket[b] = c->h_flags[tgb::flag_bucket(b)];
    return TERSOFF_OK;
  }
  // a build inside the sequence overflowed (or met non-finite positions):
  // restore the state, rebuild with a host check, run the steps eagerly
  TGB_CUDA(c, cudaMemcpyAsync(x, c->d_snap, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
  TGB_CUDA(c, cudaMemcpyAsync(v, c->d_snap + m, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
  TGB_CUDA(c, cudaMemcpyAsync(f, c->d_snap + 2 * m, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
  if (c->h_flags[tgb::FLAG_NONFINITE]) {
    if (!on_skin) c->steps_since_build = ssb0;
    TGB_CUDA(c, cudaStreamSynchronize(s));
    return tgb::fail(c, TERSOFF_E_NONFINITE, "non-finite position during MD (state restored)");
  }
  c->cap = c->cap + c->cap / 2 + 4;
  c->gen++;
  if ((st = tgb::build_list(c, x, s))) return st;
  c->last_rebuilds = 0;
  st = enqueue_md(c, x, v, f, dt, nsteps, rebuild_every, rows, thermo, true, s);
  if (st) return st;
  TGB_CUDA(c, cudaStreamSynchronize(s));
  return TERSOFF_OK;
}

int tersoff_md_step(tersoff_ctx* p, double* x, double* v, double* f, int n, const double* mass,
                    double dt, int nsteps, int rebuild_every, double* thermo, void* stream) {
  tgb::NvtxRange nvtx_range("tersoff_md_step");
  return md_impl(C(p), x, v, f, n, mass, dt, nsteps, rebuild_every, thermo,
                 (cudaStream_t)stream);
}

int tersoff_md_step_host(tersoff_ctx* p, double* x, double* v, double* f, int n,
                         const double* mass, double dt, int nsteps, int rebuild_every,
                         double* thermo, void* stream) {
  tgb::NvtxRange nvtx_range("tersoff_md_step_host");
  Ctx* c = C(p);
  int st = tgb::check_ctx(c);
  if (st) return st;
  if (n != c->n || (n > 0 && (!x || !v || !f)))
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "bad MD arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t m = 3 * (size_t)n;
  if (c->stage_alloc < 3 * m) {
    if ((st = tgb::dev_alloc(c, &c->d_stage, 3 * m))) return st;
    c->stage_alloc = 3 * m;
  }
  if (thermo && c->thermo_alloc < 3 * (size_t)nsteps) {
    if ((st = tgb::dev_alloc(c, &c->d_thermo, 3 * (size_t)nsteps))) return st;
    c->thermo_alloc = 3 * (size_t)nsteps;
  }
  double *dx = c->d_stage, *dv = c->d_stage + m, *df = c->d_stage + 2 * m;
  TGB_CUDA(c, cudaMemcpyAsync(dx, x, sizeof(double) * m, cudaMemcpyHostToDevice, s));
  TGB_CUDA(c, cudaMemcpyAsync(dv, v, sizeof(double) * m, cudaMemcpyHostToDevice, s));
  TGB_CUDA(c, cudaMemcpyAsync(df, f, sizeof(double) * m, cudaMemcpyHostToDevice, s));
  st = md_impl(c, dx, dv, df, n, mass, dt, nsteps, rebuild_every, thermo ? c->d_thermo : nullptr,
               s);
  if (st) return st;
  TGB_CUDA(c, cudaMemcpyAsync(x, dx, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
  TGB_CUDA(c, cudaMemcpyAsync(v, dv, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
  TGB_CUDA(c, cudaMemcpyAsync(f, df, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
  if (thermo)
    TGB_CUDA(c, cudaMemcpyAsync(thermo, c->d_thermo, sizeof(double) * 3 * nsteps,
                                cudaMemcpyDeviceToHost, s));
  TGB_CUDA(c, cudaStreamSynchronize(s));
  return TERSOFF_OK;
}

// ---------------------------------------------------------------- autotuner
namespace {
struct TuneOpt {
  int atomic, split, waves, block, quad;
};

void apply_opt(Ctx* c, const TuneOpt& o) {
  c->scatter_atomic = o.atomic != 0;
  c->opt_split = o.split;
  c->opt_waves = o.waves;
  c->opt_block = o.block;
  c->opt_quad = o.quad;
  c->gen++;  // captured MD graphs hold the old launch shapes
}

std::string opt_text(const TuneOpt& o) {
  char b[160];
  std::snprintf(b, sizeof(b), "scatter=%s split=%s waves=%d block=%d lanes=%s",
                o.atomic ? "atomic" : "gather",
                o.split < 0 ? "auto" : (o.split ? "on" : "off"), o.waves, o.block,
                o.quad < 0 ? "auto" : (o.quad ? "4" : "1"));
  return b;
}
}  // namespace

int tersoff_autotune(tersoff_ctx* p, const double* x, const double* v, int n, const double* mass,
                     double dt, int steps, void* stream) {
  tgb::NvtxRange nvtx_range("tersoff_autotune");
  Ctx* c = C(p);
  if (c) c->fine_valid = false;  // trial steps rebuild the lists
  int st = tgb::check_ctx(c);
  if (st) return st;
  if (!c->have_list) return tgb::fail(c, TERSOFF_E_STATE, "a neighbour build must come first");
  if (n != c->n || (n > 0 && !x)) return tgb::fail(c, TERSOFF_E_INVALID_ARG, "bad positions");
  const bool md = v != nullptr;
  if (md && (c->n_sys > 0 || !mass || !(dt > 0.0) || steps < 1))
    return tgb::fail(c, TERSOFF_E_INVALID_ARG,
                     "MD tuning needs one system, masses, dt > 0 and steps >= 1");
  if (n == 0) return TERSOFF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const bool timing = c->timing;
  c->timing = false;
  const size_t m = 3 * (size_t)n;
  double* work = nullptr;  // MD trials run on copies of x, v and F(x)
  if (md) {
    TGB_CUDA(c, cudaMalloc(&work, sizeof(double) * 3 * m));
    TGB_CUDA(c, cudaMemcpyAsync(work, x, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    TGB_CUDA(c, cudaMemcpyAsync(work + m, v, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  TGB_CUDA(c, cudaEventCreate(&e0));
  TGB_CUDA(c, cudaEventCreate(&e1));
  auto trial = [&](const TuneOpt& o, double* ms_out, int reps) -> int {
    apply_opt(c, o);
    int r;
    auto once = [&]() -> int {
      if (md)
        return md_impl(c, work, work + m, work + 2 * m, n, mass, dt, steps, steps, nullptr, s);
      if (c->n_sys > 0) return batch_impl(c, x, c->d_fbuf, nullptr, nullptr, s);
      return compute_impl(c, x, n, nullptr, c->d_fbuf, nullptr, nullptr, s);
    };
    if (md && (r = compute_impl(c, work, n, nullptr, work + 2 * m, nullptr, nullptr, s))) return r;
    for (int w = 0; w < 2; ++w)
      if ((r = once())) return r;
    std::vector<float> t;
    for (int q = 0; q < reps; ++q) {
      TGB_CUDA(c, cudaEventRecord(e0, s));
      if ((r = once())) return r;
      TGB_CUDA(c, cudaEventRecord(e1, s));
      TGB_CUDA(c, cudaEventSynchronize(e1));
      float ms = 0.0f;
      TGB_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
      t.push_back(ms);
    }
    std::sort(t.begin(), t.end());
    *ms_out = t[t.size() / 2];
    return TERSOFF_OK;
  };
  const TuneOpt start{c->scatter_atomic ? 1 : 0, c->opt_split, c->opt_waves, c->opt_block,
                      c->opt_quad};
  TuneOpt best = start;
  double best_ms = 0.0;
  std::string log;
  st = trial(best, &best_ms, 5);
  if (!st) {
    log = opt_text(best) + ": " + std::to_string(best_ms) + " ms";
    // coordinate descent: one option at a time, the others at their best
    const std::vector<std::vector<int>> values = {
        {1, 0}, {0, 1}, {-1, 0, 1}, {0, 1, 2, 4}, {128, 256, 512}};
    for (int k = 0; k < 5 && !st; ++k)
      for (int val : values[k]) {
        TuneOpt o = best;
        int* field = k == 0 ? &o.quad : k == 1 ? &o.atomic : k == 2 ? &o.split
                   : k == 3 ? &o.waves : &o.block;
        if (*field == val) continue;
        if (k == 0 && val == 0 && *field < 0) continue;  // automatic is one lane per atom
        if ((k == 0 || k == 2) && c->n_sys > 0) continue;  // batches run one launch
        if (k == 0 && (c->precision != TERSOFF_MIXED || c->ns > 2)) continue;
        if (k == 2 && best.quad == 1) continue;  // the four-lane launch has no split
        *field = val;
        double ms = 0.0;
        if ((st = trial(o, &ms, 5))) break;
        log += "; " + opt_text(o) + ": " + std::to_string(ms) + " ms";
        if (ms < best_ms) {
          best_ms = ms;
          best = o;
        }
      }
    // confirmation: the winner against the starting options, 9 repetitions
    // each; the winner replaces them only when at least 1% faster (the
    // trials' spread is of that order, so a narrower win is noise)
    const bool same = best.atomic == start.atomic && best.split == start.split &&
                      best.waves == start.waves && best.block == start.block &&
                      best.quad == start.quad;
    if (!st && !same) {
      double ms_s = 0.0, ms_b = 0.0;
      if (!(st = trial(start, &ms_s, 9)) && !(st = trial(best, &ms_b, 9))) {
        log += "; confirm " + opt_text(start) + ": " + std::to_string(ms_s) + " ms, " +
               opt_text(best) + ": " + std::to_string(ms_b) + " ms";
        if (!(ms_b < 0.99 * ms_s)) {
          best = start;
          best_ms = ms_s;
        } else {
          best_ms = ms_b;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (work) cudaFree(work);
  apply_opt(c, best);
  c->timing = timing;
  if (st) return st;
  // the MD trials rebuilt the list on the copies: rebuild it at x
  if (md && (st = tgb::build_list(c, x, s))) return st;
  c->tune_summary = "chosen " + opt_text(best) + " (" + std::to_string(best_ms) + " ms per " +
                    (md ? std::to_string(steps) + " MD steps" : std::string("evaluation")) +
                    "); trials: " + log;
  return TERSOFF_OK;
}

int tersoff_set_launch(tersoff_ctx* p, int waves, int split, int block) {
  Ctx* c = C(p);
  if (!c) return TERSOFF_E_INVALID_ARG;
  if (waves < 0 || waves > 64 || split < -1 || split > 1 ||
      !(block == 64 || block == 128 || block == 256 || block == 512))
    return tgb::fail(c, TERSOFF_E_INVALID_ARG,
                     "waves in [0, 64], split in {-1, 0, 1}, block a power of two in [64, 512]");
  TuneOpt o{c->scatter_atomic ? 1 : 0, split, waves, block, c->opt_quad};
  apply_opt(c, o);
  return TERSOFF_OK;
}

int tersoff_set_lanes(tersoff_ctx* p, int lanes) {
  Ctx* c = C(p);
  if (!c) return TERSOFF_E_INVALID_ARG;
  if (!(lanes == 0 || lanes == 1 || lanes == 4))
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "lanes is 0 (automatic), 1 or 4");
  TuneOpt o{c->scatter_atomic ? 1 : 0, c->opt_split, c->opt_waves, c->opt_block,
            lanes == 0 ? -1 : (lanes == 4 ? 1 : 0)};
  apply_opt(c, o);
  return TERSOFF_OK;
}

int tersoff_halo_pack(tersoff_ctx* p, const double* x, const int* types, const long long* ids,
                      int n, int axis, const double* geo, int cap, double* x_local,
                      double* send_x, int* send_t, long long* send_id, int* counts,
                      void* stream) {
  tgb::NvtxRange nvtx_range("tersoff_halo_pack");
  Ctx* c = C(p);
  if (!c) return TERSOFF_E_INVALID_ARG;
  if (n < 0 || cap < 0 || axis < 0 || axis > 2 || !geo || !counts)
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "n >= 0, cap >= 0, axis in {0, 1, 2}, geo and counts set");
  if (n > 0 && (!x || !types || !ids || !x_local))
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "x, types, ids and x_local must be set when n > 0");
  if (cap > 0 && (!send_x || !send_t || !send_id))
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "send buffers must be set when cap > 0");
  for (int q = 0; q < 9; ++q)
    if (!std::isfinite(geo[q]))
      return tgb::fail(c, TERSOFF_E_INVALID_ARG, "geo values must be finite");
  if (!(geo[0] > 0.0) || !(geo[3] >= 0.0))
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "L > 0 and r_ghost >= 0");
  return tgb::launch_halo_pack(c, x, types, ids, n, axis, geo, cap, x_local, send_x, send_t,
                               send_id, counts, (cudaStream_t)stream);
}

int tersoff_set_ablation(tersoff_ctx* p, int flags) {
  Ctx* c = C(p);
  if (!c) return TERSOFF_E_INVALID_ARG;
  if (flags & ~31) return tgb::fail(c, TERSOFF_E_INVALID_ARG, "ablation flags are bits 0 to 4");
  c->ablate = flags;
  c->gen++;  // captured MD graphs hold the old kernel arguments
  return TERSOFF_OK;
}

const char* tersoff_autotune_summary(const tersoff_ctx* p) {
  if (!p) return "null context";
  return p->impl.tune_summary.c_str();
}

int tersoff_md_rebuilds(const tersoff_ctx* p, int* count) {
  if (!p || !count) return TERSOFF_E_INVALID_ARG;
  *count = p->impl.last_rebuilds;
  return TERSOFF_OK;
}

int tersoff_launch_count(const tersoff_ctx* p, long long* count) {
  if (!p || !count) return TERSOFF_E_INVALID_ARG;
  *count = p->impl.launches;
  return TERSOFF_OK;
}

int tersoff_set_scatter(tersoff_ctx* p, int mode) {
  Ctx* c = C(p);
  if (!c) return TERSOFF_E_INVALID_ARG;
  if (mode != TERSOFF_SCATTER_GATHER && mode != TERSOFF_SCATTER_ATOMIC)
    return tgb::fail(c, TERSOFF_E_INVALID_ARG, "unknown scatter mode");
  c->scatter_atomic = mode == TERSOFF_SCATTER_ATOMIC;
  c->gen++;
  return TERSOFF_OK;
}

int tersoff_set_graphs(tersoff_ctx* p, int enable) {
  Ctx* c = C(p);
  if (!c) return TERSOFF_E_INVALID_ARG;
  c->use_graphs = enable != 0;
  tgb::drop_graph(c);
  return TERSOFF_OK;
}

int tersoff_set_timing(tersoff_ctx* p, int enable) {
  Ctx* c = C(p);
  if (!c) return TERSOFF_E_INVALID_ARG;
  tgb::fold_timing(c);
  c->timing = enable != 0;
  for (int k = 0; k < 3; ++k) {
    c->t_ms[k] = 0.0;
    c->t_count[k] = 0;
  }
  return TERSOFF_OK;
}

int tersoff_timing(tersoff_ctx* p, int kind, double* total_ms, long long* launches) {
  Ctx* c = C(p);
  if (!c) return TERSOFF_E_INVALID_ARG;
  if (kind < 0 || kind > 2) return tgb::fail(c, TERSOFF_E_INVALID_ARG, "kind must be 0, 1 or 2");
  tgb::fold_timing(c);
  if (total_ms) *total_ms = c->t_ms[kind];
  if (launches) *launches = c->t_count[kind];
  return TERSOFF_OK;
}

}  // extern "C"

// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <string>
#include <vector>

#include "tersoff.h"

namespace tgb {

// Position record of the FP64 path: offset from the atom's origin and its
// species (as a double), 32-byte aligned for one wide load.
struct alignas(32) dpos4 {
  double x, y, z, w;
};

// ------------------------------------------------------------------ parameters
// Derived parameter record, one per (ti, tj, tk), RSTRIDE values of T.
// Three-body part (used as record (ti,tj,tk)):
enum : int {
  K_GAMMA = 0,  // gamma
  K_GC2D2,      // gamma c^2 / d^2
  K_G2C2,       // 2 gamma c^2
  K_D2,         // d^2
  K_H,          // h
  K_LAM3,       // lambda3
  K_M,          // m (integer-valued)
  K_R3,         // R of f_C(r_ik)
  K_PID3,       // pi / (2 D)
  K_DFC3,       // -pi / (4 D)
  K_RIN3,       // R - D
  K_ROUT3,      // R + D
  // pair part (used as record (ti,tj,tj)):
  K_A,          // A
  K_LAM1,       // lambda1 (rounded to T)
  K_LAM1LO,     // lambda1 - (T)lambda1 (float records only)
  K_B,          // B
  K_LAM2,       // lambda2
  K_LAM2LO,     // lambda2 - (T)lambda2
  K_BETA,       // beta
  K_N,          // n
  K_NINV2,      // -1 / (2 n)
  K_R2,         // R of f_C(r_ij)
  K_PID2,       // pi / (2 D)
  K_DFC2,       // -pi / (4 D)
  K_RIN2,       // R - D
  K_ROUT2,      // R + D
  K_ROUT3LO,    // (R + D) - (T)(R + D) of the three-body record (float records only)
  K_ROUT2LO,    // the same for the pair record
  RSTRIDE = 32
};

// ------------------------------------------------------------------ neighbour entries
// Entry = j | (ox+1) << 26 | (oy+1) << 28 | (oz+1) << 30 where (ox,oy,oz) in
// {-1,0,1}^3 is the cell offset of the image of j found from i's cell.
constexpr int ENTRY_JBITS = 26;
constexpr uint32_t ENTRY_JMASK = (1u << ENTRY_JBITS) - 1u;
constexpr int MAX_ATOMS = 1 << ENTRY_JBITS;

struct Grid {
  int nc[3];      // cells per axis
  double L[3];    // box edges
  double invL[3]; // 1 / L (host IEEE division)
  double h[3];    // cell edge L / nc
  double invh[3]; // nc / L
  int fix_shift;  // fixed-point scale 2^fix_shift for mixed positions
};

// MD coefficients per species: c = dt/2 * (force-to-acceleration) / m, and m
struct Coef {
  double c[TERSOFF_MAX_SPECIES];   // dt/2 * (force-to-acceleration) / m
  double c2[TERSOFF_MAX_SPECIES];  // 2 c (merged closing and opening half kicks)
  double m[TERSOFF_MAX_SPECIES];
  float cf[TERSOFF_MAX_SPECIES];   // c and 2c rounded to float (mixed-path increments)
  float c2f[TERSOFF_MAX_SPECIES];
  float hmf[TERSOFF_MAX_SPECIES];  // m / 2 in float (mixed-path kinetic energy)
};

// Cell grid of one periodic system on the device (the launch-wide grid, or one
// system of a batch whose cells are numbered from cell_base).
struct GridDev {
  int nc[3];
  int cell_base;
  double L[3], invL[3], h[3], invh[3];
  float hf[3];
};

// Periodic shift units of one system of a batch: the edges of its list cells,
// in fixed point (mixed path), float and double. A list entry's cell offset
// code multiplies these.
struct SysShift {
  int hq[3];
  float hf[3];
  double h[3];
};

// ------------------------------------------------------------------ context
struct Ctx {
  int precision = TERSOFF_FP64;
  int device = 0;
  std::string err;
  long long launches = 0;

  // parameters
  int ns = 0;
  std::vector<double> table;      // raw, host
  double* d_rec64 = nullptr;      // derived records, device
  float* d_rec32 = nullptr;
  double* d_raw64 = nullptr;      // raw table (backward pass), device
  float* d_raw32 = nullptr;
  std::vector<double> h_rec64;    // host copies
  std::vector<float> h_rec32;
  cudaStream_t side = nullptr;    // side stream for small force launches
  cudaStream_t cap_stream = nullptr;  // stream used to capture MD graphs
  cudaStream_t body_stream = nullptr; // captures the body of a conditional rebuild
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  double* d_filt64 = nullptr;     // (ti,tj) filter radius^2
  float* d_filt32 = nullptr;
  float* d_near32 = nullptr;      // (ti,tj): squared (smallest outer cutoff - 2e-3 A); bonds
                                  // beyond it get their exact length residual (float path)
  std::vector<double> filt;       // host copy, radius (not squared)
  bool has_lam3 = false;
  bool sym_table = false;         // angular terms symmetric in (j,k), f_C(r_ik) j-independent
  double rmax_cut = 0.0;          // largest f_C outer radius

  // atoms / list
  int n = 0;                      // atoms of the current list
  int cap = 32;                   // per-atom capacity
  int max_cnt = 0;
  int max_short = 0;              // largest short-list count seen at build
  double r_list = 0.0;
  Grid grid{};
  bool have_list = false;
  int* d_types = nullptr;         // n
  int* d_cnt = nullptr;           // n
  uint32_t* d_nbr = nullptr;      // cap * n, slot-major: nbr[s * n + i]
  double* d_origin = nullptr;     // n x 3: o_i, u_i = x_i - o_i
  int* d_cell_of = nullptr;       // n
  int* d_cell_count = nullptr;    // ncell + 1
  int* d_cell_start = nullptr;    // ncell + 1
  int* d_cell_fill = nullptr;     // ncell
  int* d_cell_atoms = nullptr;    // n
  int* d_scan_tmp = nullptr;
  long long* d_bintab = nullptr;  // binning tables of the single-system grid (neighbor.cu)
  std::vector<long long> h_bintab;
  size_t cells_alloc = 0;
  size_t atoms_alloc = 0;
  size_t nbr_alloc = 0;
  double* d_qorg = nullptr;       // n x 3: 1.5*2^52 - o_i 2^S (fixed-point origin)
  int4* d_qref = nullptr;         // n: fixed-point offsets at the last build
  uint32_t* d_short = nullptr;    // zs_cap * n, slot-major short list
  int* d_zcnt = nullptr;          // n
  int* d_bucket = nullptr;        // 3 x n: atom indices per bucket (entries inside the cutoffs)
  int* d_left = nullptr;          // n: atoms the four-lane force kernel leaves to the per-thread one
  uint8_t* d_rev = nullptr;       // zs_cap x n: slot of j in the short list of its p-th neighbour
  void* d_contrib = nullptr;      // zs_cap x n force contributions (float4 or dpos4)
  void* d_own = nullptr;          // n: force of each atom's own terms on itself
  double* d_extra = nullptr;      // n x 3: atomically scattered forces (fallback mode)
  size_t contrib_alloc = 0;       // bytes of d_contrib
  int contrib_prec = -1;
  bool scatter_atomic = false;    // forces by FP64 atomics instead of slots + gather
  int nbucket[3] = {0, 0, 0};     // bucket sizes at the last build
  int zs_cap = 0;
  double margin = 0.0;            // short-list radius margin beyond the cutoffs
  double* d_trow = nullptr;       // MD thermo accumulation rows (ACC_LEN doubles per step)
  size_t trow_alloc = 0;
  float4* d_pos32 = nullptr;      // n: (u float, type bits)
  float4* d_posc = nullptr;       // n, cell order: (u float, bits of 4 j + species)
  uint8_t* d_zw = nullptr;        // n: list entries inside the filter radii at the build (capped 63)
  int* d_fine = nullptr;          // n: atoms ordered by d_zw (backward launches)
  int* d_zbins = nullptr;         // 3 x 64: counts, offsets, cursors of that order
  unsigned long long* d_kmask = nullptr;  // n: short-list entries whose receiving slot may
                                          // hold a nonzero force (all ones after a build)
  int4* d_posq = nullptr;         // n: (u fixed point, type)
  dpos4* d_pos64 = nullptr;     // n: (u double, type)
  int* d_flags = nullptr;         // device status words (see FLAG_*)
  int* h_flags = nullptr;         // pinned mirror
  double* d_acc = nullptr;        // ACC_LEN: energy, virial (6), kinetic at stride ACC_STRIDE
  double* d_coef = nullptr;       // MD: dt/2 F->a / m per species, then masses
  Coef coef{};                    // the same, passed to the kernels by value
  int steps_since_build = 0;
  int last_rebuilds = 0;          // neighbour rebuilds during the last MD call
  bool fine_valid = false;        // d_fine matches the current lists (cleared by every build,
                                  // MD call and autotune; set by the backward that sorts)

  // launch options (chosen by tersoff_autotune)
  int opt_waves = 0;   // force kernel grid: 0 = one thread per item; k > 0 = k waves of the
                       // blocks resident on all SMs (the kernel loops over items)
  int opt_split = -1;  // capacity-8 side-stream launch: -1 automatic, 0 never, 1 when non-empty
  int opt_block = 256; // block size of the per-atom pack / integrate / gather kernels
  int opt_quad = -1;   // four lanes per atom in the main force launch: 1 when eligible
                       // (mixed path, one or two species, a single system), 0 or -1
                       // (automatic: measured slower on the benchmark) one thread per atom
  int n_sm = 0;        // multiprocessors of the device
  int ablate = 0;      // tersoff_set_ablation flags
  std::string tune_summary;  // last tersoff_autotune: choice and trial times

  // batch of independent periodic systems (n_sys > 0; tersoff_neighbor_build_batched)
  int n_sys = 0;
  long ncell_batch = 0;           // cells of all systems' grids
  GridDev* d_geo = nullptr;       // n_sys grids
  SysShift* d_sys = nullptr;      // n_sys shift units
  int* d_atom_sys = nullptr;      // n: system of each atom
  int* d_sys_off = nullptr;       // n_sys + 1 atom offsets
  double* d_vatom = nullptr;      // n x 6 per-atom virial
  double* d_eatom = nullptr;      // n per-atom energy
  double* d_fbuf = nullptr;       // scratch forces (n x 3) for calls without output
  float* d_gf32 = nullptr;        // n x 3: force weights of the backward pass in float
  double* d_stage = nullptr;      // host-call staging: x, v, f (3 x n x 3)
  double* d_thermo = nullptr;     // host-call staging thermo
  size_t stage_alloc = 0;
  size_t thermo_alloc = 0;

  // kernel timing (tersoff_set_timing)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Pending {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  double t_ms[3] = {0, 0, 0};
  long long t_count[3] = {0, 0, 0};
  std::vector<Pending>* timer_sink = nullptr;  // capture: the graph's timer list
  bool capturing = false;

  // MD steps as one CUDA graph per call shape (replayed while the shape and
  // the context state generation stay the same)
  bool use_graphs = true;
  long long gen = 0;  // bumped by params, builds from outside MD, capacity changes
  struct MdGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<Pending> timers;
    const double *x = nullptr, *v = nullptr, *f = nullptr, *thermo = nullptr;
    const double* snap = nullptr;  // the start-state copy the first step writes
    double dt = 0.0;
    Coef coef{};
    int nsteps = 0, rebuild_every = 0, ssb0 = 0, precision = 0;
    bool timing = false;
    long long gen = -1;
    int decisions = -1;     // bucket_decisions() at capture
    long long kernels = 0;  // kernel launches inside the graph, conditional bodies excluded
    long long body_kernels = 0;  // kernel launches of one conditional rebuild
  } graph;
  double* d_snap = nullptr;  // x, v, f at the start of a graph launch (rollback)
  size_t snap_alloc = 0;
};

// The force launch's host decisions that depend on the last build's bucket
// sizes, as bits: a capacity-8 launch for bucket 1 on the side stream (1),
// the wide kernel for bucket 2 (2). They choose which kernel evaluates an
// atom, and so the rounding of its terms; a captured MD graph holds them, and
// is captured again when they change.
inline int bucket_decisions(const Ctx* c) {
  const bool split1 = c->opt_split < 0 ? (long long)c->nbucket[1] * 20 > (long long)c->n
                                       : (c->opt_split > 0 && c->nbucket[1] > 0);
  const bool wide = (long long)c->nbucket[2] * 200 > (long long)c->n;
  return (split1 ? 1 : 0) | (wide ? 2 : 0);
}

// An NVTX range over an entry point's host call, named after it: profilers that
// record NVTX (Nsight Systems; Nsight Compute's --nvtx filters) show each
// call's kernels under it. Without such a tool attached it costs a check.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Records an event pair around a launch sequence when timing is enabled.
struct TimedRegion {
  Ctx* c;
  int kind;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  TimedRegion(Ctx* c_, int kind_, cudaStream_t s_);
  ~TimedRegion();
};
int fold_timing(Ctx* c);

// Device status words, each in its own 128-byte line (words that many blocks
// update or read would otherwise serialise on one L2 slice). Words below
// FLAG_BUILD_WORDS are cleared at every neighbour build; the others are sticky
// until the next compute/MD call.
constexpr int FLAG_STRIDE = 32;
enum : int {
  FLAG_OVERFLOW = 0 * FLAG_STRIDE,      // largest neighbour count of the build
  FLAG_SHORT_MAX = 1 * FLAG_STRIDE,     // largest short-list count of the build
  FLAG_DMAX = 2 * FLAG_STRIDE,          // running max squared displacement since the build (float bits)
  FLAG_BUCKET = 3 * FLAG_STRIDE,        // 3 words: atoms per bucket (<= 4, <= 8, more list
                                        // entries inside the filter radii)
  FLAG_REV_MISS = 6 * FLAG_STRIDE,      // a short-list entry has no reverse entry
  FLAG_BUILD_WORDS = 8 * FLAG_STRIDE,
  FLAG_NONFINITE = 8 * FLAG_STRIDE,     // non-finite position seen by a build
  FLAG_FALLBACK = 9 * FLAG_STRIDE,      // atoms handled by the general path
  FLAG_OVF_ANY = 10 * FLAG_STRIDE,      // some build exceeded the list capacity
  FLAG_EXTRA = 11 * FLAG_STRIDE,        // last force evaluation scattered through atomics
  FLAG_NREBUILD = 12 * FLAG_STRIDE,     // displacement-triggered rebuilds in this MD call
  FLAG_EXTRA_STICKY = 13 * FLAG_STRIDE, // some evaluation since the call began did
  FLAG_LEFT = 14 * FLAG_STRIDE,         // atoms the four-lane force kernel left to the
                                        // per-thread kernel (0 between evaluations)
  FLAG_LEFT_TICKET = 15 * FLAG_STRIDE,  // blocks of that per-thread launch done (0 between)
  FLAG_COUNT = 16 * FLAG_STRIDE
};
__host__ __device__ constexpr int flag_bucket(int b) { return FLAG_BUCKET + b * FLAG_STRIDE; }

// Energy / virial / kinetic accumulators: 8 components, each in its own line.
constexpr int ACC_STRIDE = 16;            // doubles
constexpr int ACC_LEN = 8 * ACC_STRIDE;   // one accumulator row

// The TERSOFF_ABLATE_COMP_ATOM_SUMS variant is active: mixed path, one
// species, a single system. Its force kernel scatters with FP64 atomics.
// Programmatic dependent launch: a kernel launched with launch_pdl may be
// scheduled while the previous kernel on its stream drains; it calls
// pdl_wait() before touching any memory, which returns once that kernel has
// completed and its writes are visible (at once when there is no such
// dependency). The launch latency between the two kernels overlaps the first
// one's last blocks.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

inline bool comp_atom_sums(const Ctx* c) {
  return (c->ablate & TERSOFF_ABLATE_COMP_ATOM_SUMS) && c->precision == TERSOFF_MIXED &&
         c->ns == 1 && c->n_sys == 0;
}

int fail(Ctx* c, int code, const std::string& msg);
int cuda_fail(Ctx* c, cudaError_t e, const char* where);

#define TGB_CUDA(ctx, call)                                  \
  do {                                                       \
    cudaError_t e__ = (call);                                \
    if (e__ != cudaSuccess) return ::tgb::cuda_fail((ctx), e__, #call); \
  } while (0)

// ------------------------------------------------------------------ launchers
// Neighbour build (neighbor.cu). Fills d_nbr, d_cnt, d_origin; does not sync.
int launch_neighbor_build(Ctx* c, const double* x, cudaStream_t s);
// Per-axis binning tables of the single-system grid c->grid (cell thresholds,
// origins and fixed-point origins), uploaded on s; called whenever that grid
// is set up, before any build on it.
int upload_bin_tables(Ctx* c, cudaStream_t s);
int launch_neighbor_export(Ctx* c, int* cnt, int* nbr, int cap, cudaStream_t s);

// Position packs for the force kernels (integrate.cu): fixed-point offsets
// (both paths) and FP64 offsets (FP64 path). At a build (build = true) also
// the float offsets and the displacement references; otherwise the running
// maximum displacement since the build is updated.
int launch_pack_positions(Ctx* c, const double* x, bool build, cudaStream_t s);

// Forces (fwd_f32.cu / fwd_f64.cu). Accumulates into f (zeroed by the caller),
// energy and virial into acc components 0..6 (zeroed by the caller); eatom optional.
// virial false: acc receives the energy only (its virial components stay 0).
int launch_forward(Ctx* c, double* f, double* acc, double* eatom, cudaStream_t s,
                   bool virial = true);
int launch_forward_f32(Ctx* c, double* f, double* acc, double* eatom, cudaStream_t s,
                       bool virial);
int launch_forward_f64(Ctx* c, double* f, double* acc, double* eatom, cudaStream_t s,
                       bool virial);
// the force launches of the TERSOFF_ABLATE_COMP_ATOM_SUMS variant (fwd_f32_cs.cu),
// register capacity 4 or 8; args is a fwd::FwdArgs<float>
int launch_forward_cs(Ctx* c, const void* args, int zc, int grid, cudaStream_t s);
// the four-lane force kernel (fwd_f32_quad.cu; mixed path, one or two species,
// single systems) over all atoms; args is a fwd::FwdArgs<float> with
// identity set; ev: energy, virial or per-atom energy wanted
int launch_forward_quad(Ctx* c, const void* args, bool ev, cudaStream_t s);
// Batch of systems: forces (slots or atomics into f, as launch_forward),
// per-atom energy d_eatom and virial d_vatom.
int launch_forward_batch(Ctx* c, double* f, cudaStream_t s);
int launch_forward_batch_f32(Ctx* c, double* f, cudaStream_t s);
// Per-system sums of d_eatom and d_vatom: energy[n_sys], virial[n_sys x 6]
// (either may be NULL).
int launch_system_sums(Ctx* c, double* energy, double* virial, cudaStream_t s);

// Force gathering (integrate.cu): F_j = own_j + the slots of j's column (the
// contributions of the terms of j's short-list neighbours) + the atomic
// fallback buffer when flagged; compensated float sums carried into double
// (mixed) or double sums (FP64), written to f.
int launch_gather(Ctx* c, double* f, cudaStream_t s);

// Velocity Verlet (integrate.cu) with the coefficients c->coef.
//   step kernel: v += kick * c F (kick = 1 on the first step of a call, with
//   F read from f; 2 afterwards, with F gathered from the last force
//   evaluation: the closing half kick of the previous step and the opening
//   half kick of this one); x += dt v; pack; ke_row (optional) receives
//   sum m (v_prev + c F)^2 / 2 of the previous step; acc_zero (optional) is
//   cleared for the coming force evaluation; snap (optional, kick 1 only)
//   receives x, v and f as read (3 x n x 3 doubles).
int launch_md_step(Ctx* c, double* x, double* v, double* f, double dt, int kick, bool pack,
                   double* ke_row, double* acc_zero, cudaStream_t s, double* snap = nullptr);
// closing half kick of the last step with gathered forces, which are also
// written to f; ke_row (optional) as above
int launch_final_kick(Ctx* c, double* v, double* f, double* ke_row, cudaStream_t s);
// Sets the condition of a graph IF node: 1 when the largest squared
// displacement since the last build exceeds lim2 (and counts it), else 0.
int launch_decide_rebuild(Ctx* c, float lim2, cudaGraphConditionalHandle h, cudaStream_t s);
// thermo (nsteps x 3: potential, kinetic [eV], total) from the accumulator rows
// Ghost-shell packing of a slab decomposition (halo.cu); geo: 9 host doubles
// (L, lo, hi, r_ghost, frame, shift_lower, frame_lower, shift_upper,
// frame_upper).
int launch_halo_pack(Ctx* c, const double* x, const int* types, const long long* ids, int n,
                     int axis, const double* geo, int cap, double* x_local, double* send_x,
                     int* send_t, long long* send_id, int* counts, cudaStream_t s);

int launch_thermo_rows(Ctx* c, const double* rows, int nsteps, double mvv2e, double* thermo,
                       cudaStream_t s);
// Parameter adjoint (tersoff_bwd.cu): adds d/dtheta [gE E + sum gF . F] to
// grad (ns^3 x TERSOFF_NPARAM); positions must be packed. And f = -gE f.
int launch_backward(Ctx* c, const double* gE, const double* gF, double* grad, cudaStream_t s);
// adds the position derivative of sum_a gF_a . F_a to grad_x (positions packed)
int launch_hvp(Ctx* c, const double* gF, double* grad_x, cudaStream_t s);
int launch_scale_forces(Ctx* c, double* f, const double* gE, cudaStream_t s);
// Fixed scratch of tersoff_compute_noalloc (noalloc.cu): the current device's
// array and its length in doubles; and the copy of its results to the outputs.
int noalloc_scratch(Ctx* c, double** out, size_t* doubles);
int launch_noalloc_out(Ctx* c, const double* scr, int n, double* forces, double* energy,
                       double* virial, cudaStream_t s);

}  // namespace tgb

// The opaque handle of the C ABI.
struct tersoff_ctx {
  tgb::Ctx impl;
};

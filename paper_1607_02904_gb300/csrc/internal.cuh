// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

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
  double* d_filt64 = nullptr;     // (ti,tj) filter radius^2
  float* d_filt32 = nullptr;
  std::vector<double> filt;       // host copy, radius (not squared)
  bool has_lam3 = false;
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
  size_t cells_alloc = 0;
  size_t atoms_alloc = 0;
  size_t nbr_alloc = 0;
  float4* d_pos32 = nullptr;      // n: (u float, type bits)
  int4* d_posq = nullptr;         // n: (u fixed point, type)
  dpos4* d_pos64 = nullptr;     // n: (u double, type)
  int* d_flags = nullptr;         // device status words (see FLAG_*)
  int* h_flags = nullptr;         // pinned mirror
  double* d_acc = nullptr;        // energy (1) + virial (6) + kinetic (1)
  double* d_coef = nullptr;       // MD: dt/2 F->a / m per species, then masses
  int steps_since_build = 0;
  double* d_fbuf = nullptr;       // scratch forces (n x 3) for calls without output
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

enum : int {
  FLAG_OVERFLOW = 0,   // max neighbour count (atomicMax)
  FLAG_NONFINITE = 1,  // non-finite position seen
  FLAG_SHORT_MAX = 2,  // largest short-list count
  FLAG_FALLBACK = 3,   // atoms handled by the general path
  FLAG_COUNT = 8
};

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
int launch_neighbor_export(Ctx* c, int* cnt, int* nbr, int cap, cudaStream_t s);

// Position packs for the force kernels (integrate.cu).
int launch_pack_positions(Ctx* c, const double* x, cudaStream_t s);

// Forces (tersoff_fwd.cu). Accumulates into f (zeroed by the caller), energy
// and virial into acc[0..6] (zeroed by the caller); eatom optional.
int launch_forward(Ctx* c, double* f, double* acc, double* eatom, cudaStream_t s);
int launch_forward_f32(Ctx* c, double* f, double* acc, double* eatom, cudaStream_t s);
int launch_forward_f64(Ctx* c, double* f, double* acc, double* eatom, cudaStream_t s);

// Velocity Verlet (integrate.cu). cdt[t] = dt/2 * (force-to-acceleration) / m_t.
int launch_kick_drift(Ctx* c, double* x, double* v, double* f, const double* cdt, double dt,
                      bool pack, cudaStream_t s);
int launch_kick(Ctx* c, double* v, const double* f, const double* cdt, const double* mass,
                bool want_ke, cudaStream_t s);
int launch_thermo(Ctx* c, double mvv2e, double* row, cudaStream_t s);
int launch_zero(Ctx* c, double* p, size_t count, cudaStream_t s);

}  // namespace tgb

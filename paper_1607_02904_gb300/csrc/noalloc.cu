// Fixed scratch for tersoff_compute_noalloc: the force kernel's accumulators
// live in one array that is part of the library image, so that call never asks
// the CUDA runtime for memory.
//
// Layout (doubles): [0, ACC_LEN) the energy / virial accumulator row (energy
// at 0, virial component k at (1 + k) ACC_STRIDE), then 3 n force components
// (atom-major). Every call on a device shares that device's copy and leaves
// its last contents behind; the caller clears what must start at zero.
#include <mutex>

#include "internal.cuh"

namespace tgb {

constexpr size_t NOALLOC_DOUBLES = (size_t)ACC_LEN + 3 * (size_t)TERSOFF_NOALLOC_MAX_ATOMS;

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};
}  // namespace

// Address of the current device's scratch array, looked up once per device
// (the first call on a device makes the runtime load this module there).
int noalloc_scratch(Ctx* c, double** out, size_t* doubles) {
  int dev = -1;
  TGB_CUDA(c, cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(c, TERSOFF_E_CUDA, "device ordinal out of range for the fixed scratch");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    TGB_CUDA(c, cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_addr[dev] = (double*)p;
  }
  *out = g_addr[dev];
  *doubles = NOALLOC_DOUBLES;
  return TERSOFF_OK;
}

// Copies the accumulated forces, energy and virial out of the scratch array.
__global__ void k_noalloc_out(const double* __restrict__ scr, int n, double* __restrict__ forces,
                              double* __restrict__ energy, double* __restrict__ virial) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const double* fs = scr + ACC_LEN;
  if (forces && t < 3 * n) forces[t] = fs[t];
  if (t == 0) {
    if (energy) energy[0] = scr[0];
    if (virial)
      for (int k = 0; k < 6; ++k) virial[k] = scr[(1 + k) * ACC_STRIDE];
  }
}

int launch_noalloc_out(Ctx* c, const double* scr, int n, double* forces, double* energy,
                       double* virial, cudaStream_t s) {
  const int threads = 3 * n > 0 ? 3 * n : 1;
  k_noalloc_out<<<(threads + 255) / 256, 256, 0, s>>>(scr, n, forces, energy, virial);
  c->launches++;
  TGB_CUDA(c, cudaGetLastError());
  return TERSOFF_OK;
}

}  // namespace tgb

// Mixed-precision instances of the force kernel (float terms, double sums).
#include "fwd_launch.cuh"

namespace tgb {
int launch_forward_f32(Ctx* c, double* f, double* acc, double* eatom, cudaStream_t s,
                       bool virial) {
  return fwd::launch_prec<float>(c, f, acc, eatom, s, virial);
}
int launch_forward_batch_f32(Ctx* c, double* f, cudaStream_t s) {
  return fwd::launch_batch<float>(c, f, s);
}
}  // namespace tgb

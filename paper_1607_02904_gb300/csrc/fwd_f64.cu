// FP64 instances of the force kernel.
#include "fwd_launch.cuh"

namespace tgb {
int launch_forward_f64(Ctx* c, double* f, double* acc, double* eatom, cudaStream_t s,
                       bool virial) {
  return fwd::launch_prec<double>(c, f, acc, eatom, s, virial);
}

int launch_forward_batch(Ctx* c, double* f, cudaStream_t s) {
  if (c->n == 0) return TERSOFF_OK;
  if (c->precision == TERSOFF_MIXED) return launch_forward_batch_f32(c, f, s);
  return fwd::launch_batch<double>(c, f, s);
}

int launch_forward(Ctx* c, double* f, double* acc, double* eatom, cudaStream_t s, bool virial) {
  if (c->n == 0) return TERSOFF_OK;
  if (c->precision == TERSOFF_MIXED) return launch_forward_f32(c, f, acc, eatom, s, virial);
  return launch_forward_f64(c, f, acc, eatom, s, virial);
}
}  // namespace tgb

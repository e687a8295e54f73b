// Mixed-precision force kernel with compensated per-atom sums (the
// TERSOFF_ABLATE_COMP_ATOM_SUMS variant; one species, single systems).
#include "fwd_launch.cuh"

namespace tgb {
int launch_forward_cs(Ctx* c, const void* args, int zc, int grid, cudaStream_t s) {
  const fwd::FwdArgs<float>& a = *static_cast<const fwd::FwdArgs<float>*>(args);
  const int mode = c->has_lam3 ? 1 : (c->sym_table ? 2 : 0);
  if (zc == 4) {
    if (mode == 1) fwd::k_tersoff<float, 1, 4, 1, false, true><<<grid, fwd::BLOCK, 0, s>>>(a);
    else if (mode == 2) fwd::k_tersoff<float, 1, 4, 2, false, true><<<grid, fwd::BLOCK, 0, s>>>(a);
    else fwd::k_tersoff<float, 1, 4, 0, false, true><<<grid, fwd::BLOCK, 0, s>>>(a);
  } else {
    if (mode == 1) fwd::k_tersoff<float, 1, 8, 1, false, true><<<grid, fwd::BLOCK, 0, s>>>(a);
    else if (mode == 2) fwd::k_tersoff<float, 1, 8, 2, false, true><<<grid, fwd::BLOCK, 0, s>>>(a);
    else fwd::k_tersoff<float, 1, 8, 0, false, true><<<grid, fwd::BLOCK, 0, s>>>(a);
  }
  c->launches++;
  return TERSOFF_OK;
}
}  // namespace tgb

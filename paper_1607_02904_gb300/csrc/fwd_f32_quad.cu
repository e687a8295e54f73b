// The four-lane force kernel, mixed path (float terms, double sums).
#include "tersoff_quad.cuh"

namespace tgb {
namespace {
template <int NS, bool EV>
void quad_launch(Ctx* c, const fwd::FwdArgs<float>& a, cudaStream_t s) {
  const int grid = (c->n + fwd::QATOMS - 1) / fwd::QATOMS;
  if (c->has_lam3)
    fwd::k_tersoff_quad<float, NS, 1, EV><<<grid, fwd::QBLOCK, 0, s>>>(a);
  else if (c->sym_table)
    fwd::k_tersoff_quad<float, NS, 2, EV><<<grid, fwd::QBLOCK, 0, s>>>(a);
  else
    fwd::k_tersoff_quad<float, NS, 0, EV><<<grid, fwd::QBLOCK, 0, s>>>(a);
}
}  // namespace

int launch_forward_quad(Ctx* c, const void* args, bool ev, cudaStream_t s) {
  const fwd::FwdArgs<float>& a = *static_cast<const fwd::FwdArgs<float>*>(args);
  if (c->ns == 1)
    ev ? quad_launch<1, true>(c, a, s) : quad_launch<1, false>(c, a, s);
  else
    ev ? quad_launch<2, true>(c, a, s) : quad_launch<2, false>(c, a, s);
  c->launches++;
  return TERSOFF_OK;
}
}  // namespace tgb

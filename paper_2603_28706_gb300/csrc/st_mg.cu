// Multigrid preconditioner: surrogate Vanka patches, Galerkin coarse
// operators, transfers, V-cycle (Sec. 6.3).
#include "st_internal.h"

namespace st {
st_status mg_destroy(st_problem* h) {
  (void)h;
  return ST_OK;
}
}  // namespace st

using namespace st;

extern "C" {
st_status st_precond_setup(st_problem* h, st_prec prec) {
  (void)prec;
  return set_error(h, ST_EINVAL, "st_precond_setup: not available yet");
}
st_status st_vanka_smooth(st_problem* h, int level, int sweeps, st_prec prec, const void* r, void* d) {
  (void)level; (void)sweeps; (void)prec; (void)r; (void)d;
  return set_error(h, ST_EINVAL, "st_vanka_smooth: not available yet");
}
st_status st_vcycle(st_problem* h, st_prec prec, const void* r, void* d) {
  (void)prec; (void)r; (void)d;
  return set_error(h, ST_EINVAL, "st_vcycle: not available yet");
}
st_status st_newton_step(st_problem* h, st_tangent tangent, st_prec vcycle_prec, void* U, const void* v_prev,
                         const void* f, st_newton_info* info) {
  (void)tangent; (void)vcycle_prec; (void)U; (void)v_prev; (void)f; (void)info;
  return set_error(h, ST_EINVAL, "st_newton_step: not available yet");
}
}

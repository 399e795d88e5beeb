// Outer solvers: FGMRES and the globalised Newton step (placeholder until built).
#include "st_internal.h"

using namespace st;

extern "C" st_status st_newton_step(st_problem* h, st_tangent tangent, st_prec vcycle_prec, void* U,
                                    const void* v_prev, const void* f, st_newton_info* info) {
  (void)tangent; (void)vcycle_prec; (void)U; (void)v_prev; (void)f; (void)info;
  return set_error(h, ST_EINVAL, "st_newton_step: not available");
}

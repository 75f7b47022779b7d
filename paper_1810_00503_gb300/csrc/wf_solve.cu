// L-BFGS MAP driver (placeholder until the device solver lands).
#include "wf_api_internal.h"

void wf_solver_free(wf_problem* p) { (void)p; }

extern "C" wf_status wf_map_solve(wf_problem* p, const wf_opts* opts, const void* s0, void* s_out,
                                  void* x_out, wf_solve_stats* stats) {
  (void)p; (void)opts; (void)s0; (void)s_out; (void)x_out; (void)stats;
  return wf_fail(WF_EINVAL, "wf_map_solve: not built yet");
}

// Batched solver of many independent problems (filled in below).
#include "engine.h"

using namespace dwf;

extern "C" dwf_status dwf_batch_solve(int n, const dwf_problem* problems, double tol, int maxit,
                                      dwf_stats* per_solve, void* stream) {
  (void)n; (void)problems; (void)tol; (void)maxit; (void)per_solve; (void)stream;
  return set_error(DWF_ERR_ARG, "dwf_batch_solve: not available in this build");
}

// GMRES on the PIE system (Section 4).
#include "problem.h"

namespace pie {

pie_status solve(Problem&, const void*, void*, double, int, int, pie_solve_stats*, cudaStream_t) {
  set_error("pie_solve: not built in this version");
  return PIE_ERR_PARAM;
}

}  // namespace pie

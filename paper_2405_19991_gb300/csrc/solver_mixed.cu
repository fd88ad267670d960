// Solver instantiation: PCG vectors / V-cycle storage = float, __nv_bfloat16.
#include "solver.cuh"

namespace otm {
SolverBase* make_solver_mixed() { return new Solver<float, __nv_bfloat16>(); }
}  // namespace otm

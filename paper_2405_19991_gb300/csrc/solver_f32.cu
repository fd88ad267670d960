// Solver instantiation: PCG vectors / V-cycle storage = float, float.
#include "solver.cuh"

namespace otm {
SolverBase* make_solver_f32() { return new Solver<float, float>(); }
}  // namespace otm

// Solver instantiation: PCG vectors / V-cycle storage = double, double.
#include "solver.cuh"

namespace otm {
SolverBase* make_solver_f64() { return new Solver<double, double>(); }
}  // namespace otm

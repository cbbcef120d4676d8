// Explicit instantiation of the specialised local solver kernel.
#include "solver_impl.cuh"
namespace ieti_t {
template cudaError_t launch_t<float, 2, 4, 2, 0>(const SolveArgs&, int, cudaStream_t);
}  // namespace ieti_t

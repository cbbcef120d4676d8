// Explicit instantiation of the specialised local solver kernel.
#include "solver_impl.cuh"
namespace ieti_t {
template cudaError_t launch_t<float, 2, 2, 4, 0, false>(const SolveArgs&, int, cudaStream_t, int*);
template cudaError_t launch_t<float, 2, 2, 4, 0, true>(const SolveArgs&, int, cudaStream_t, int*);
}  // namespace ieti_t

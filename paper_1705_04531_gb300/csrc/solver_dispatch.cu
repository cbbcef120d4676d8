// Dispatch of the local solver to the kernel specialised for the patch
// dimension and degrees.
#include "solver_impl.cuh"

namespace ieti_t {
extern template cudaError_t launch_t<float, 2, 2, 2, 0>(const SolveArgs&, int, cudaStream_t);
extern template cudaError_t launch_t<float, 2, 2, 3, 0>(const SolveArgs&, int, cudaStream_t);
extern template cudaError_t launch_t<float, 2, 2, 4, 0>(const SolveArgs&, int, cudaStream_t);
extern template cudaError_t launch_t<float, 2, 3, 2, 0>(const SolveArgs&, int, cudaStream_t);
extern template cudaError_t launch_t<float, 2, 3, 3, 0>(const SolveArgs&, int, cudaStream_t);
extern template cudaError_t launch_t<float, 2, 3, 4, 0>(const SolveArgs&, int, cudaStream_t);
extern template cudaError_t launch_t<float, 2, 4, 2, 0>(const SolveArgs&, int, cudaStream_t);
extern template cudaError_t launch_t<float, 2, 4, 3, 0>(const SolveArgs&, int, cudaStream_t);
extern template cudaError_t launch_t<float, 2, 4, 4, 0>(const SolveArgs&, int, cudaStream_t);
extern template cudaError_t launch_t<float, 3, 2, 2, 2>(const SolveArgs&, int, cudaStream_t);
extern template cudaError_t launch_t<double, 2, 2, 2, 0>(const SolveArgs&, int, cudaStream_t);
extern template cudaError_t launch_t<double, 2, 2, 3, 0>(const SolveArgs&, int, cudaStream_t);
extern template cudaError_t launch_t<double, 2, 2, 4, 0>(const SolveArgs&, int, cudaStream_t);
extern template cudaError_t launch_t<double, 2, 3, 2, 0>(const SolveArgs&, int, cudaStream_t);
extern template cudaError_t launch_t<double, 2, 3, 3, 0>(const SolveArgs&, int, cudaStream_t);
extern template cudaError_t launch_t<double, 2, 3, 4, 0>(const SolveArgs&, int, cudaStream_t);
extern template cudaError_t launch_t<double, 2, 4, 2, 0>(const SolveArgs&, int, cudaStream_t);
extern template cudaError_t launch_t<double, 2, 4, 3, 0>(const SolveArgs&, int, cudaStream_t);
extern template cudaError_t launch_t<double, 2, 4, 4, 0>(const SolveArgs&, int, cudaStream_t);
extern template cudaError_t launch_t<double, 3, 2, 2, 2>(const SolveArgs&, int, cudaStream_t);
}  // namespace ieti_t

namespace {
template <typename T>
cudaError_t dispatch(const SolveArgs& a, int dim, int p0, int p1, int p2, int threads, cudaStream_t st) {
    using namespace ieti_t;
    if (dim == 2 && p2 == 0) {
        switch (p0 * 10 + p1) {
            case 22: return launch_t<T, 2, 2, 2, 0>(a, threads, st);
            case 23: return launch_t<T, 2, 2, 3, 0>(a, threads, st);
            case 24: return launch_t<T, 2, 2, 4, 0>(a, threads, st);
            case 32: return launch_t<T, 2, 3, 2, 0>(a, threads, st);
            case 33: return launch_t<T, 2, 3, 3, 0>(a, threads, st);
            case 34: return launch_t<T, 2, 3, 4, 0>(a, threads, st);
            case 42: return launch_t<T, 2, 4, 2, 0>(a, threads, st);
            case 43: return launch_t<T, 2, 4, 3, 0>(a, threads, st);
            case 44: return launch_t<T, 2, 4, 4, 0>(a, threads, st);
            default: break;
        }
    } else if (dim == 3 && p0 == p1 && p1 == p2) {
        if (p0 == 2) return launch_t<T, 3, 2, 2, 2>(a, threads, st);
    }
    return cudaErrorNotSupported;
}
}  // namespace

bool solve_variant_exists(int dim, int p0, int p1, int p2) {
    if (dim == 2) return p2 == 0 && p0 >= 2 && p0 <= 4 && p1 >= 2 && p1 <= 4;
    return dim == 3 && p0 == p1 && p1 == p2 && p0 == 2;
}

cudaError_t launch_solve_variant(const SolveArgs& a, int dim, int p0, int p1, int p2, int threads,
                                 cudaStream_t st) {
    if (a.mixed) return dispatch<float>(a, dim, p0, p1, p2, threads, st);
    return dispatch<double>(a, dim, p0, p1, p2, threads, st);
}

size_t solve_smem_need(const PatchDesc& P, int mixed) {
    return ieti_t::smem_need(P, mixed ? sizeof(float) : sizeof(double));
}

// Dispatch of the local solver to the kernel specialised for the patch
// dimension and degrees (FP32 V-cycles: 2D degrees 2..4 in each direction
// and 3D degree 2; FP64 V-cycles: 2D (2,2), (3,3) and 3D degree 2).
#include "solver_impl.cuh"

namespace ieti_t {
extern template cudaError_t launch_t<float, 2, 2, 2, 0, false>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<float, 2, 2, 2, 0, true>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<float, 2, 2, 3, 0, false>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<float, 2, 2, 3, 0, true>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<float, 2, 2, 4, 0, false>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<float, 2, 2, 4, 0, true>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<float, 2, 3, 2, 0, false>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<float, 2, 3, 2, 0, true>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<float, 2, 3, 3, 0, false>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<float, 2, 3, 3, 0, true>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<float, 2, 3, 4, 0, false>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<float, 2, 3, 4, 0, true>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<float, 2, 4, 2, 0, false>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<float, 2, 4, 2, 0, true>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<float, 2, 4, 3, 0, false>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<float, 2, 4, 3, 0, true>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<float, 2, 4, 4, 0, false>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<float, 2, 4, 4, 0, true>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<float, 3, 2, 2, 2, false>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<float, 3, 2, 2, 2, true>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<double, 2, 2, 2, 0, false>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<double, 2, 2, 2, 0, true>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<double, 2, 3, 3, 0, false>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<double, 2, 3, 3, 0, true>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<double, 3, 2, 2, 2, false>(const SolveArgs&, int, cudaStream_t, int*);
extern template cudaError_t launch_t<double, 3, 2, 2, 2, true>(const SolveArgs&, int, cudaStream_t, int*);
}  // namespace ieti_t

namespace {
cudaError_t dispatch_float(const SolveArgs& a, int dim, int p0, int p1, int p2, int threads, cudaStream_t st, bool xg,
                           int* occ) {
    using namespace ieti_t;
    const int key = dim * 1000 + p0 * 100 + p1 * 10 + p2;
    switch (key) {
        case 2220: return xg ? launch_t<float, 2, 2, 2, 0, true>(a, threads, st, occ) : launch_t<float, 2, 2, 2, 0, false>(a, threads, st, occ);
        case 2230: return xg ? launch_t<float, 2, 2, 3, 0, true>(a, threads, st, occ) : launch_t<float, 2, 2, 3, 0, false>(a, threads, st, occ);
        case 2240: return xg ? launch_t<float, 2, 2, 4, 0, true>(a, threads, st, occ) : launch_t<float, 2, 2, 4, 0, false>(a, threads, st, occ);
        case 2320: return xg ? launch_t<float, 2, 3, 2, 0, true>(a, threads, st, occ) : launch_t<float, 2, 3, 2, 0, false>(a, threads, st, occ);
        case 2330: return xg ? launch_t<float, 2, 3, 3, 0, true>(a, threads, st, occ) : launch_t<float, 2, 3, 3, 0, false>(a, threads, st, occ);
        case 2340: return xg ? launch_t<float, 2, 3, 4, 0, true>(a, threads, st, occ) : launch_t<float, 2, 3, 4, 0, false>(a, threads, st, occ);
        case 2420: return xg ? launch_t<float, 2, 4, 2, 0, true>(a, threads, st, occ) : launch_t<float, 2, 4, 2, 0, false>(a, threads, st, occ);
        case 2430: return xg ? launch_t<float, 2, 4, 3, 0, true>(a, threads, st, occ) : launch_t<float, 2, 4, 3, 0, false>(a, threads, st, occ);
        case 2440: return xg ? launch_t<float, 2, 4, 4, 0, true>(a, threads, st, occ) : launch_t<float, 2, 4, 4, 0, false>(a, threads, st, occ);
        case 3222: return xg ? launch_t<float, 3, 2, 2, 2, true>(a, threads, st, occ) : launch_t<float, 3, 2, 2, 2, false>(a, threads, st, occ);
        default: return cudaErrorNotSupported;
    }
}
cudaError_t dispatch_double(const SolveArgs& a, int dim, int p0, int p1, int p2, int threads, cudaStream_t st, bool xg,
                           int* occ) {
    using namespace ieti_t;
    const int key = dim * 1000 + p0 * 100 + p1 * 10 + p2;
    switch (key) {
        case 2220: return xg ? launch_t<double, 2, 2, 2, 0, true>(a, threads, st, occ) : launch_t<double, 2, 2, 2, 0, false>(a, threads, st, occ);
        case 2330: return xg ? launch_t<double, 2, 3, 3, 0, true>(a, threads, st, occ) : launch_t<double, 2, 3, 3, 0, false>(a, threads, st, occ);
        case 3222: return xg ? launch_t<double, 3, 2, 2, 2, true>(a, threads, st, occ) : launch_t<double, 3, 2, 2, 2, false>(a, threads, st, occ);
        default: return cudaErrorNotSupported;
    }
}
}  // namespace

bool solve_variant_exists(int dim, int p0, int p1, int p2, int mixed) {
    const int key = dim * 1000 + p0 * 100 + p1 * 10 + p2;
    if (mixed) return key == 2220 || key == 2230 || key == 2240 || key == 2320 || key == 2330 || key == 2340 || key == 2420 || key == 2430 || key == 2440 || key == 3222;
    return key == 2220 || key == 2330 || key == 3222;
}

cudaError_t launch_solve_variant(const SolveArgs& a, int dim, int p0, int p1, int p2, int threads,
                                 cudaStream_t st, bool xg) {
    if (a.mixed) return dispatch_float(a, dim, p0, p1, p2, threads, st, xg, nullptr);
    return dispatch_double(a, dim, p0, p1, p2, threads, st, xg, nullptr);
}

int solve_variant_ctas_per_sm(int dim, int p0, int p1, int p2, int mixed, bool xg, int threads, size_t smem) {
    SolveArgs a{};
    a.mixed = mixed;
    a.smem_bytes = smem;
    int occ = 0;
    cudaError_t e = mixed ? dispatch_float(a, dim, p0, p1, p2, threads, nullptr, xg, &occ)
                          : dispatch_double(a, dim, p0, p1, p2, threads, nullptr, xg, &occ);
    return e == cudaSuccess ? occ : 0;
}

size_t solve_smem_min(const PatchDesc& P, int mixed) {
    return ieti_t::smem_min(P, mixed ? sizeof(float) : sizeof(double));
}

size_t solve_smem_need(const PatchDesc& P, int mixed, bool xg) {
    return ieti_t::smem_need(P, mixed ? sizeof(float) : sizeof(double), xg);
}


size_t solve_smem_tables(const PatchDesc& P) { return ieti_t::ctab_bytes(P); }

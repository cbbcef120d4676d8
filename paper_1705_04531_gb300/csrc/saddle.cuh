// Launch wrappers of the MG-MG-S vector kernels (saddle_kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

// coefficient sign * num / den read from device scalars (num, den may be null: 1)
struct SaddleCoef {
    const double* num;
    const double* den;
    double sign;
};

// up to 8 updates sharing one coefficient c: mode 0 y = x + c y,
// mode 1 y += c x, mode 2 y = x, mode 3 y = x - y
struct SaddleLin {
    int njobs;
    double* y[8];
    const double* x[8];
    long long n[8];
    int mode[8];
    SaddleCoef c;
};

// sum of up to 4 dot products
struct SaddleDot {
    int njobs;
    const double* a[4];
    const double* b[4];
    long long n[4];
};

cudaError_t launch_sp_matvec(int n, const double* S, const double* x, double* y, double scale, cudaStream_t st);
cudaError_t launch_spp_solve(int n, const double* Linv, const double* x, double* y, double scale, cudaStream_t st);
cudaError_t launch_primal_assemble(int npi, const int* gptr, const int* glist, const double* rloc, double* out,
                                   int accumulate, cudaStream_t st);
cudaError_t launch_project_kerC(int nrows, const PatchDesc* pd, const int* crow_patch, const int* crow_ptr,
                                const int* c_idx, const double* c_w, double* y, cudaStream_t st);
cudaError_t launch_function(int npatch, const PatchDesc* pd, const int* crow_glob, const double* phi,
                            const double* uP, const double* w, double* out, cudaStream_t st);
cudaError_t launch_lin(const SaddleLin& L, cudaStream_t st);
// partial: 256 doubles of scratch; copy_to (may be null) receives the result too
cudaError_t launch_dot(const SaddleDot& D, double* partial, double* out, double* copy_to, cudaStream_t st);
cudaError_t launch_copy_scalar(const double* src, double* dst, cudaStream_t st);

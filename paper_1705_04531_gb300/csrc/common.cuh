// Shared device-side data model of the IETI-DP library.
//
// Every patch keeps its spline space on the full tensor grid of
// m_r = n_r + p_r functions per direction (first direction fastest).
// Boundary conditions are side masks: side 2r is xi_r = 0, side 2r+1 is
// xi_r = 1; a masked side's functions are removed from the operator (their
// rows are skipped, their vector entries stay 0).
//
// Banded stiffness storage ("color-blocked SoA"): rows are grouped by
// Gauss-Seidel color (color c = sum_r (i_r mod (p_r+1)) * stride_r), and
// within a color numbered q in lexicographic order of t_r = i_r / (p_r+1).
// Color c owns one contiguous block of cnt_c * S values (S = prod_r (2p_r+1)
// stencil entries) starting at off_c * S, laid out offset-major:
// K(i, i + offset(o)) sits at off_c * S + o * cnt_c + q.  A warp working on
// one color reads each stencil diagonal with unit stride (coalesced in
// global memory, bank-conflict free in shared memory), and the values one
// color step needs form one contiguous range.  Out-of-grid entries are 0.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define IETI_MAXD 3
#define IETI_MAXLEV 12
#define IETI_MAXP 8

struct LevelDesc {
    int m[3];          // functions per direction (1 for unused directions)
    int n;             // m0*m1*m2
    int S;             // stencil size
    int Sp;            // padded row length of the value arrays
    int xoff, boff;    // specialised solver: offsets of x (color-major, ghost padded) and b (storage order)
    int nx;            // size of the color-major padded x of this level
    int xk[3];         // uniform padded block extents (ceil(m_r/(p_r+1)) + 2; 1 if unused)
    int blk;           // xk0*xk1*xk2: size of one color block
    int refined[3];    // 1 if this level halves the elements of level l-1 along r
    long long koff;    // offset of this level's values in the value arrays
    int voff;          // offset of this level's vectors in a slot's level block
    // 1D tables (offsets into the table pools), valid for level l > 0:
    //  restriction (column form): for coarse index I of level l-1,
    //    itab[rs + I] = first fine index, tab[rw + I*W + t] = P(first+t, I)
    //  prolongation (row form): for fine index i of level l,
    //    itab[ps + i] = first coarse index, tab[pw + i*W + t] = P(i, first+t)
    int rs[3], rw[3], ps[3], pw[3];
    // parameter-domain mass band: tab[mw + i*(2p+1) + (o+p)] = M(i, i+o)
    int mw[3];
};

struct PatchDesc {
    int dim;
    int p[3];
    int nelem[3];
    int L;               // levels (0 = coarsest, L-1 = fine)
    int dmask;           // sides on the Dirichlet boundary
    int floating;        // 1 if dmask == 0
    long long toff;      // offset of this patch in torn vectors
    int n;               // fine functions
    int nlvec;           // sum over levels of n_l
    int nlx, nlb;        // specialised solver: total x and b sizes over levels
    long long a0off[2];  // coarsest inverse (n0 x n0), hierarchy 0 (Neumann) / 1 (Dirichlet)
    int npi;             // primal constraint rows of this patch
    int crow0;           // first global C row of this patch
    long long phioff;    // Phi (n x npi, column-major); also the offset of W = Khat^{-1} C^T (SZ basis)
    long long szhoff;    // Hhat^{-1} of the SZ basis solver (npi x npi, row-major)
    long long bandoff;   // D-MG: banded Cholesky factor of the fine K (n x (bw+1), by columns)
    int bw;              // D-MG: half band width p0 + m0 (p1 + m1 p2)
    int pin;             // D-MG: pinned dof of a floating patch (-1: none)
    LevelDesc lev[IETI_MAXLEV];
};

// ---------------------------------------------------------------------------
// index helpers
// ---------------------------------------------------------------------------
__host__ __device__ inline int ieti_cnt(int m, int p, int c) { return (m - c + p) / (p + 1); }

__host__ __device__ inline int ieti_prefix(int m, int p, int c) {
    int s = 0;
    for (int k = 0; k < c; ++k) s += ieti_cnt(m, p, k);
    return s;
}

// storage offset of color (c0,c1,c2)
__host__ __device__ inline int ieti_color_off(const int* m, const int* p, int c0, int c1, int c2) {
    return m[0] * m[1] * ieti_prefix(m[2], p[2], c2) +
           ieti_cnt(m[2], p[2], c2) * (m[0] * ieti_prefix(m[1], p[1], c1) +
                                       ieti_cnt(m[1], p[1], c1) * ieti_prefix(m[0], p[0], c0));
}

// storage position of natural row (i0,i1,i2)
__host__ __device__ inline int ieti_store_pos(const int* m, const int* p, int i0, int i1, int i2) {
    int c0 = i0 % (p[0] + 1), c1 = i1 % (p[1] + 1), c2 = i2 % (p[2] + 1);
    int t0 = i0 / (p[0] + 1), t1 = i1 / (p[1] + 1), t2 = i2 / (p[2] + 1);
    return ieti_color_off(m, p, c0, c1, c2) +
           t0 + ieti_cnt(m[0], p[0], c0) * (t1 + ieti_cnt(m[1], p[1], c1) * t2);
}

__host__ __device__ inline int ieti_ncolors(const int* p) { return (p[0] + 1) * (p[1] + 1) * (p[2] + 1); }

// row length of the value arrays (no padding in the color-blocked layout)
__host__ __device__ inline int ieti_sp(int S) { return S; }

// position of K(i, i + offset(o)) in a level's value array
__host__ __device__ inline long long ieti_val_pos(const int* m, const int* p, int S, int i0, int i1, int i2, int o) {
    int c0 = i0 % (p[0] + 1), c1 = i1 % (p[1] + 1), c2 = i2 % (p[2] + 1);
    int k0 = ieti_cnt(m[0], p[0], c0), k1 = ieti_cnt(m[1], p[1], c1), k2 = ieti_cnt(m[2], p[2], c2);
    int q = i0 / (p[0] + 1) + k0 * (i1 / (p[1] + 1) + k1 * (i2 / (p[2] + 1)));
    return (long long)ieti_color_off(m, p, c0, c1, c2) * S + (long long)o * (k0 * k1 * k2) + q;
}

// color-major, ghost-padded vector layout of the specialised solver: every
// color owns one block of uniform extents (ceil(m_r/(p_r+1)) + 2) per
// direction (a ghost layer on each side; the third extent is 1 in 2D);
// blocks follow each other in color order.  Entry (t0,t1,t2) of color c sits
// at c*blk + (t0+1) + xk0*((t1+1) + xk1*(t2+1)) (t2+1 -> 0 in 2D).
__host__ __device__ inline int ieti_xk(int m, int p) { return (m + p) / (p + 1) + 2; }
__host__ __device__ inline int ieti_cm_block(const int* m, const int* p, int dim, int c0, int c1, int c2) {
    int b = (ieti_cnt(m[0], p[0], c0) + 2) * (ieti_cnt(m[1], p[1], c1) + 2);
    if (dim == 3) b *= ieti_cnt(m[2], p[2], c2) + 2;
    return b;
}
__host__ __device__ inline int ieti_cm_size(const int* m, const int* p, int dim) {
    int blk = ieti_xk(m[0], p[0]) * ieti_xk(m[1], p[1]) * (dim == 3 ? ieti_xk(m[2], p[2]) : 1);
    return blk * ieti_ncolors(p);
}

__host__ __device__ inline bool ieti_masked(int mask, const int* m, int i0, int i1, int i2) {
    if ((mask & 1) && i0 == 0) return true;
    if ((mask & 2) && i0 == m[0] - 1) return true;
    if ((mask & 4) && i1 == 0) return true;
    if ((mask & 8) && i1 == m[1] - 1) return true;
    if ((mask & 16) && i2 == 0) return true;
    if ((mask & 32) && i2 == m[2] - 1) return true;
    return false;
}

__host__ __device__ inline bool ieti_on_boundary(const int* m, int dim, int i0, int i1, int i2) {
    if (i0 == 0 || i0 == m[0] - 1) return true;
    if (i1 == 0 || i1 == m[1] - 1) return true;
    if (dim == 3 && (i2 == 0 || i2 == m[2] - 1)) return true;
    return false;
}

// error flags written by kernels (bit field in a device int)
#define IETI_FLAG_NOT_CONVERGED 1
#define IETI_FLAG_BREAKDOWN     2
#define IETI_FLAG_NONFINITE     4
#define IETI_FLAG_TABLE         8
#define IETI_FLAG_NOT_SPD      16

// device clock in nanoseconds, common to every SM
__device__ __forceinline__ unsigned long long ieti_gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// widens a launch's [start, end] span by this CTA's lifetime (thread 0)
struct IetiLaunchSpan {
    unsigned long long* p;
    __device__ explicit IetiLaunchSpan(unsigned long long* q) : p(q) {
        if (p && threadIdx.x == 0) atomicMin(p, ieti_gtimer());
    }
    __device__ ~IetiLaunchSpan() {
        if (p && threadIdx.x == 0) atomicMax(p + 1, ieti_gtimer());
    }
};

#define IETI_CUDA_CHECK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return e_; } while (0)

// Multigrid transfer operators and coarse stencil (declarations). See amg.cu.
#pragma once
#include "common.cuh"

namespace tmamg {

struct AggDims {
  int L[4];    // parent lattice
  int agg[4];  // aggregate extents
  int Lc[4];   // coarse lattice
  int64_t Vp;  // parent volume
  int64_t Vc;  // coarse volume
  int asize;   // parent sites per aggregate
};

struct CoarseDims {
  int L[4];
  int64_t Vc;
  int nc;
};

// P from the nv test vectors (FP32 bundle of the parent level, ncomp = 2 d); orthonormal per
// aggregate and chirality (classical Gram-Schmidt twice, FP64 dots).
void build_P(const AggDims& g, const float* Vb, float2* P, int nv, int d, cudaStream_t st);
// xc = P^+ r  (parent bundle -> coarse bundle, nsys systems)
void restrict_vec(const AggDims& g, const float2* P, const float* r, float* xc, int nv, int d, int nsys,
                  cudaStream_t st);
// e (+)= P xc
void prolong_vec(const AggDims& g, const float2* P, const float* xc, float* e, int nv, int d, int nsys, int accumulate,
                 cudaStream_t st);
// y = D_c(dmu * mu_n) x on coarse bundles
void coarse_apply(const CoarseDims& cd, const float2* A, const float* x, float* y, const double* mu, double dmu,
                  int nsys, cudaStream_t st, const double* eps = nullptr);
// A = P^+ D P for a fine parent; W, Y: fine bundles of 2 nv systems; R: coarse bundle of 2 nv systems
void build_coarse_operator_fine(const AggDims& g, const float2* U32, const float* C32, const float2* P, float2* A,
                                int nv, int bc_t, float* W, float* Y, float* R, cudaStream_t st);

// A = P^+ D_p P for a coarse parent D_p (stencil Ap on pd, d = pd.nc / 2 unknowns per chirality):
// W, Y: parent bundles of 2 nv systems; R: coarse bundle of 2 nv systems
void build_coarse_operator_coarse(const AggDims& g, const CoarseDims& pd, const float2* Ap, const float2* P,
                                  float2* A, int nv, float* W, float* Y, float* R, cudaStream_t st);
// coarse field [nsys][Vc][nc] (complex float) -> FP32 coarse bundle
void pack_coarse(const float* field, float* bundle, int nsys, int nc, int64_t Vc, cudaStream_t st);

// plain FP64 forms (amg64.cu) for the FP64 comparator solver: FP64 bundles, one system per tile;
// P64 / A64 are the FP32 P and coarse blocks widened to FP64 (widen_f2)
void widen_f2(const float2* in, double2* out, int64_t n, cudaStream_t st);
void restrict64(const AggDims& g, const double2* P64, const double* r, double* xc, int nv, int d, int nsys,
                cudaStream_t st);
void prolong64(const AggDims& g, const double2* P64, const double* xc, double* e, int nv, int d, int nsys,
               cudaStream_t st);
void coarse_apply64(const CoarseDims& cd, const double2* A64, const double* x, double* y, const double* mu,
                    double dmu, int nsys, cudaStream_t st);

}  // namespace tmamg

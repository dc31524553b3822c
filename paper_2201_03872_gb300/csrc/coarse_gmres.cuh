// Persistent coarse-level GMRES (declarations). See coarse_gmres.cu.
#pragma once
#include <cuda_fp16.h>

#include "amg.cuh"

namespace tmamg {

struct CoarseGmres {
  int m = 0, NS = 0, G = 0;
  double2 *H = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr, *part = nullptr;
  double *cs = nullptr, *tolabs = nullptr, *b0 = nullptr, *sc = nullptr;
  int *kconv = nullptr, *active = nullptr, *done = nullptr, *nactive = nullptr, *err = nullptr, *iters = nullptr;
  unsigned* bar = nullptr;
  int* h_flags = nullptr;
  float* hpart = nullptr;  // 9 coarse bundles: hop partials of the stencil
  size_t hbytes = 0;       // bytes of one coarse bundle the partials are sized for
  __half* X16 = nullptr;   // B images of the tensor-core stencil
  size_t x16_bytes = 0;
  int alloc(int m, int nsys, int G, size_t bundle_bytes, size_t x16_bytes);
  void release();
};

// grid size (CTAs) used for nt coarse tiles: a multiple of nt, at most one wave
int coarse_gmres_grid(int nt);

// xc ~ D_c(dmu mu)^{-1} rc by restarted GMRES(m) to |r| <= tol |rc| per system, at most
// maxiter Arnoldi steps, in one cooperative launch. V: m + 1 coarse bundles (vstride floats
// apart). A16: the FP16 operator of the tensor-core stencil (coarse_mma.cuh), or null for the
// FP32 stencil A. If iters_done is non-null the call synchronises the stream and returns -3
// when a bounded wait timed out, else 0; -1 if the launch failed, -2 if the state is too small.
// process-wide wait bound of the persistent kernel's grid barriers (cycles; <= 0 restores the
// default of 2e9) and a one-shot request that the next launch's barriers wait for one arrival
// more than the grid has, so that the bounded wait runs out (tests of the timeout path)
void coarse_gmres_debug_wait(long long limit_cycles, int unreachable_next);

int coarse_gmres_solve(CoarseGmres& s, const CoarseDims& cd, const float2* A, const __half* A16, const float* rc,
                       float* xc, float* V, int64_t vstride, const double* mu, double dmu, int nsys, int m,
                       int maxiter, double tol, int* iters_done, cudaStream_t st);

}  // namespace tmamg

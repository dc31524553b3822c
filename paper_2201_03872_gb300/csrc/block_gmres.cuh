// Block GMRES at the coarsest level (declarations). See block_gmres.cu.
#pragma once
#include <functional>

#include "common.cuh"

namespace tmamg {

struct BlockGmres {
  int m = 0, nsys = 0, nshift = 0, nblk = 1;
  int64_t M = 0;  // entries per tile of a coarse bundle
  double2 *gram = nullptr, *part = nullptr, *coef = nullptr, *hgram = nullptr, *Racc = nullptr, *S0 = nullptr;
  double2 *H = nullptr, *Gr = nullptr, *sn = nullptr, *Y = nullptr;
  double *cs = nullptr, *res = nullptr, *tolabs = nullptr;
  int *active = nullptr, *steps = nullptr, *nactive = nullptr;
  int* h_nactive = nullptr;
  int alloc(int m, int nsys, int nshift, int64_t M);
  void release();
};

// xc ~ A^{-1} rc by block GMRES(m), one block per shift (systems n with n % nshift == k),
// every column of a block to |r| <= tol |rc|, at most maxiter block steps. apply(x, y):
// y = A x on coarse bundles. V: m + 1 coarse bundles (vstride floats apart); tmp: one more.
// Returns 0, or -2 if the block is wider than 16 or the state is too small.
int block_gmres_solve(BlockGmres& b, const std::function<void(const float*, float*)>& apply, const float* rc,
                      float* xc, float* V, int64_t vstride, float* tmp, size_t bundle_bytes, int m, int maxiter,
                      double tol, int* iters_done, cudaStream_t st);

}  // namespace tmamg

// Batched BLAS-1 on bundles (declarations). See blas.cu.
#pragma once
#include "common.cuh"

namespace tmamg {

// out[i * ostride + n] = <V_i[n], w[n]> (conjugate-linear in V) for i < k, n < nsys.
// V_i = V + i * vstride (reals); M = ncomp * nsite entries per tile. partial: scratch of
// partial_elems(M, nsys, k, T) double2.
template <typename real>
void mdot(const real* V, int64_t vstride, int k, const real* w, int64_t M, int nsys, double2* out, int64_t ostride,
          double2* partial, cudaStream_t st);
size_t partial_elems(int64_t M, int nsys, int kmax, int T);

// Doublet solves: while set (on the calling host thread), every mdot adds the results of systems
// 2p and 2p + 1 and gives the sum to both, so that a Krylov method running on per-system scalars
// treats each doublet (its two flavours) as one system: both lanes then see identical norms, dots,
// rotations and update coefficients.
void set_pair_fold(bool on);
struct PairFold {
  explicit PairFold(bool on) { set_pair_fold(on); }
  ~PairFold() { set_pair_fold(false); }
};

// y[n] += sign * sum_i c[i * cstride + n] V_i[n]; masked systems unchanged
template <typename real>
void maxpy(const real* V, int64_t vstride, int k, const double2* c, int64_t cstride, double sign, real* y, int64_t M,
           int nsys, const int* mask, cudaStream_t st);

// y = a x + b y with a, b per system: mode 0 = zero, 1 = one, 2 = from the device array
template <typename real>
void axpby(const double2* a, int amode, const real* x, const double2* b, int bmode, real* y, int64_t M, int nsys,
           const int* mask, cudaStream_t st);

// FP64 bundle (T = 1) -> FP32 bundle (T = 2), scaled by s[n] (device, nullptr = 1)
void f64_to_f32(const double* x64, const double* s, float* x32, int64_t M, int nsys, cudaStream_t st);
// x64[n] += s[n] x32[n] for unmasked systems
void f32_axpy_f64(const double* s, const float* x32, double* x64, int64_t M, int nsys, const int* mask,
                  cudaStream_t st);

}  // namespace tmamg

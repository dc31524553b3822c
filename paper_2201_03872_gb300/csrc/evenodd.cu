// Even-odd (Schur complement) form of the fine operator.
//
// The hops of D(mu) = A(mu) + H connect only sites of opposite parity p(s) = (x + y + z + t) mod 2,
// so eliminating the odd sites leaves M_ee = A_ee - H_eo A_oo^{-1} H_oe on the even sites, the
// standard reduction of the DDalphaAMG family that the paper's method builds on (Sec. 2). Here it is
// composed from the fine stencil, which is already vectorised over the systems of a bundle:
//   w  = x with its odd sites cleared
//   t  = D w                    (on the odd sites: H_oe x_e, since w_o = 0)
//   w_o = -A_oo(mu_n)^{-1} t_o  (site-local solves, per system: the twisted clover block depends on mu_n)
//   y  = D w, odd sites cleared (on the even sites: A_ee x_e - H_eo A_oo^{-1} H_oe x_e)
// The local solves run per site, system and chirality on the 6 x 6 block A_chi + i s_chi mu_n, whose
// Hermitian part (diagonal 4 + m0 plus the clover) is positive definite, so Gaussian elimination
// without pivoting is stable.
#include "common.cuh"
#include "profile.cuh"

namespace tmamg {

__device__ __forceinline__ int site_parity(int64_t s, const Geom& g) {
  int c[4];
  site_coords(s, g.L, c);
  return (c[0] + c[1] + c[2] + c[3]) & 1;
}

// clear the entries of the sites of parity `par` (bundle [ntile][12][V][2][T])
template <typename real, int T>
__global__ void eo_clear_kernel(real* __restrict__ b, Geom g, int par, int ntile) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // (tile, comp, site)
  const int64_t n = (int64_t)ntile * 12 * g.V;
  if (i >= n) return;
  const int64_t s = i % g.V;
  if (site_parity(s, g) != par) return;
  real* p = b + i * 2 * T;
#pragma unroll
  for (int k = 0; k < 2 * T; ++k) p[k] = real(0);
}

// w <- -A(mu_n)^{-1} t on the odd sites (w keeps its even entries); one thread per (tile, site)
template <typename real, int T>
__global__ void eo_solve_kernel(const real* __restrict__ C, const double* __restrict__ mu, const real* __restrict__ t,
                                real* __restrict__ w, Geom g, int nsys, int ntile) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // (tile, site)
  if (i >= (int64_t)ntile * g.V) return;
  const int tile = (int)(i / g.V);
  const int64_t s = i % g.V;
  if (site_parity(s, g) != 1) return;
  const int64_t V = g.V;
  const int64_t tbase = (int64_t)tile * 12 * V * 2 * T;
  for (int l = 0; l < T; ++l) {
    const int n = tile * T + l;
    const real m = n < nsys ? (real)mu[n] : real(0);
    for (int chi = 0; chi < 2; ++chi) {
      const real* Cc = C + (int64_t)chi * 36 * V + s;
      const real smu = chi == 0 ? m : -m;
      real ar[6][6], ai[6][6], br[6], bi[6];
      for (int r = 0; r < 6; ++r) {
        ar[r][r] = Cc[(int64_t)r * V];
        ai[r][r] = smu;
        for (int c = 0; c < r; ++c) {
          const int k = 6 + 2 * (r * (r - 1) / 2 + c);
          const real re = Cc[(int64_t)k * V], im = Cc[(int64_t)(k + 1) * V];
          ar[r][c] = re;
          ai[r][c] = im;
          ar[c][r] = re;  // Hermitian clover: the upper entry is the conjugate
          ai[c][r] = -im;
        }
        const int64_t o = tbase + ((int64_t)(chi * 6 + r) * V + s) * 2 * T;
        br[r] = t[o + l];
        bi[r] = t[o + T + l];
      }
      // forward elimination
      for (int p = 0; p < 6; ++p) {
        const real den = ar[p][p] * ar[p][p] + ai[p][p] * ai[p][p];
        const real ir = ar[p][p] / den, ii = -ai[p][p] / den;  // 1 / a_pp
        for (int r = p + 1; r < 6; ++r) {
          const real fr = ar[r][p] * ir - ai[r][p] * ii, fi = ar[r][p] * ii + ai[r][p] * ir;  // a_rp / a_pp
          for (int c = p + 1; c < 6; ++c) {
            ar[r][c] -= fr * ar[p][c] - fi * ai[p][c];
            ai[r][c] -= fr * ai[p][c] + fi * ar[p][c];
          }
          br[r] -= fr * br[p] - fi * bi[p];
          bi[r] -= fr * bi[p] + fi * br[p];
        }
      }
      // back substitution
      for (int p = 5; p >= 0; --p) {
        real sr = br[p], si = bi[p];
        for (int c = p + 1; c < 6; ++c) {
          sr -= ar[p][c] * br[c] - ai[p][c] * bi[c];
          si -= ar[p][c] * bi[c] + ai[p][c] * br[c];
        }
        const real den = ar[p][p] * ar[p][p] + ai[p][p] * ai[p][p];
        br[p] = (sr * ar[p][p] + si * ai[p][p]) / den;
        bi[p] = (si * ar[p][p] - sr * ai[p][p]) / den;
      }
      for (int r = 0; r < 6; ++r) {
        const int64_t o = tbase + ((int64_t)(chi * 6 + r) * V + s) * 2 * T;
        w[o + l] = n < nsys ? -br[r] : real(0);
        w[o + T + l] = n < nsys ? -bi[r] : real(0);
      }
    }
  }
}

template <typename real>
void launch_dirac_eo(const Geom& g, const void* U, const real* C, const real* x, real* y, const double* mu, int nsys,
                     real* s0, real* s1, cudaStream_t st) {
  constexpr int T = Tile<real>::T;
  const int nt = ntiles(nsys, T);
  const size_t bytes = (size_t)nt * 12 * g.V * 2 * T * sizeof(real);
  const int64_t ne = (int64_t)nt * 12 * g.V, ns = (int64_t)nt * g.V;
  cudaMemcpyAsync(s0, x, bytes, cudaMemcpyDeviceToDevice, st);
  eo_clear_kernel<real, T><<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(s0, g, 1, nt); TM_COUNT();
  launch_dirac<real>(g, U, C, s0, s1, mu, nsys, st);
  {
    TM_PROF(st, "eo_solve");
    eo_solve_kernel<real, T><<<(unsigned)((ns + 127) / 128), 128, 0, st>>>(C, mu, s1, s0, g, nsys, nt); TM_COUNT();
  }
  launch_dirac<real>(g, U, C, s0, y, mu, nsys, st);
  eo_clear_kernel<real, T><<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(y, g, 1, nt); TM_COUNT();
}

template void launch_dirac_eo<float>(const Geom&, const void*, const float*, const float*, float*, const double*, int,
                                     float*, float*, cudaStream_t);
template void launch_dirac_eo<double>(const Geom&, const void*, const double*, const double*, double*,
                                      const double*, int, double*, double*, cudaStream_t);

}  // namespace tmamg

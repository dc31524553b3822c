// Plain FP64 multigrid transfer and coarse stencil for the FP64 comparator solver (FP64 bundles,
// one system per tile): the same P, P^+ and D_c as the batched path (paper Sec. 2), in FP64
// arithmetic throughout. P and the coarse blocks are the setup's FP32 values widened to FP64.
#include "amg.cuh"

namespace tmamg {

__global__ void widen_kernel(const float2* __restrict__ in, double2* __restrict__ out, int64_t n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) out[t] = make_double2(in[t].x, in[t].y);
}

void widen_f2(const float2* in, double2* out, int64_t n, cudaStream_t st) {
  widen_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, n);
  TM_COUNT();
}

__device__ __forceinline__ int agg_member_site(int64_t a, int q, const AggDims& g) {
  int ac[4], lq[4], c[4];
  site_coords(a, g.Lc, ac);
  site_coords(q, g.agg, lq);
#pragma unroll
  for (int k = 0; k < 4; ++k) c[k] = ac[k] * g.agg[k] + lq[k];
  return (int)site_index(c, g.L);
}

// xc[n][chi nv + j][a] = sum_k conj(P[a][chi][j][k]) r[n][chi d + c'][site(a, q)], k = c' asize + q;
// one CTA per (aggregate, chirality), one warp per output, lanes over k, fixed-order warp sum
__global__ void __launch_bounds__(256) restrict64_kernel(const double2* __restrict__ P, const double* __restrict__ r,
                                                         double* __restrict__ xc, AggDims g, int nv, int d,
                                                         int nsys) {
  extern __shared__ int sidx64[];
  const int64_t a = blockIdx.x >> 1;
  const int chi = blockIdx.x & 1;
  const int K = g.asize * d;
  for (int q = threadIdx.x; q < g.asize; q += blockDim.x) sidx64[q] = agg_member_site(a, q, g);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const double2* Pa = P + ((a * 2 + chi) * nv) * (int64_t)K;
  for (int o = warp; o < nv * nsys; o += nw) {
    const int j = o % nv, n = o / nv;
    double sr = 0, si = 0;
    for (int k = lane; k < K; k += 32) {
      const int cp = k / g.asize, q = k - cp * g.asize;
      const double2 p = Pa[(int64_t)j * K + k];
      const double2 v =
          *reinterpret_cast<const double2*>(r + (((int64_t)n * (2 * d) + chi * d + cp) * g.Vp + sidx64[q]) * 2);
      sr += p.x * v.x + p.y * v.y;
      si += p.x * v.y - p.y * v.x;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, off);
      si += __shfl_xor_sync(0xffffffffu, si, off);
    }
    if (lane == 0)
      *reinterpret_cast<double2*>(xc + (((int64_t)n * (2 * nv) + chi * nv + j) * g.Vc + a) * 2) = make_double2(sr, si);
  }
}

// e[n][chi d + c'][site(a, q)] = sum_j P[a][chi][j][k] xc[n][chi nv + j][a]; one CTA per
// (aggregate, chirality), threads over k, the aggregate's coarse entries in shared memory
__global__ void __launch_bounds__(256) prolong64_kernel(const double2* __restrict__ P, const double* __restrict__ xc,
                                                        double* __restrict__ e, AggDims g, int nv, int d, int nsys) {
  __shared__ double2 xs[32];
  extern __shared__ int sidx64[];
  const int64_t a = blockIdx.x >> 1;
  const int chi = blockIdx.x & 1;
  const int K = g.asize * d;
  for (int q = threadIdx.x; q < g.asize; q += blockDim.x) sidx64[q] = agg_member_site(a, q, g);
  const double2* Pa = P + ((a * 2 + chi) * nv) * (int64_t)K;
  for (int n = 0; n < nsys; ++n) {
    __syncthreads();
    if (threadIdx.x < nv)
      xs[threadIdx.x] =
          *reinterpret_cast<const double2*>(xc + (((int64_t)n * (2 * nv) + chi * nv + threadIdx.x) * g.Vc + a) * 2);
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      double er = 0, ei = 0;
      for (int j = 0; j < nv; ++j) {
        const double2 p = Pa[(int64_t)j * K + k];
        er += p.x * xs[j].x - p.y * xs[j].y;
        ei += p.x * xs[j].y + p.y * xs[j].x;
      }
      const int cp = k / g.asize, q = k - cp * g.asize;
      *reinterpret_cast<double2*>(e + (((int64_t)n * (2 * d) + chi * d + cp) * g.Vp + sidx64[q]) * 2) =
          make_double2(er, ei);
    }
  }
}

// y[n][i][a] = sum_h sum_j A[h][a][j][i] x[n][j][a + h] + i dmu mu_n gamma5_c(i) x[n][i][a]
__global__ void coarse_apply64_kernel(const double2* __restrict__ A, const double* __restrict__ x,
                                      double* __restrict__ y, const double* __restrict__ mu, double dmu, int nsys,
                                      CoarseDims cd) {
  const int nc = cd.nc;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nsys * cd.Vc * nc) return;
  const int i = (int)(t % nc);
  const int64_t a = (t / nc) % cd.Vc;
  const int n = (int)(t / ((int64_t)nc * cd.Vc));
  int c[4];
  site_coords(a, cd.L, c);
  const double* xn = x + (int64_t)n * nc * cd.Vc * 2;
  double yr = 0, yi = 0;
  for (int h = 0; h < 9; ++h) {
    int64_t nb = a;
    if (h > 0) {
      int c2[4] = {c[0], c[1], c[2], c[3]};
      const int nu = (h - 1) / 2, dir = ((h - 1) & 1) ? -1 : 1;
      c2[nu] = (c2[nu] + dir + cd.L[nu]) % cd.L[nu];
      nb = site_index(c2, cd.L);
    }
    const double2* Ah = A + (((int64_t)h * cd.Vc + a) * nc) * nc + i;
    for (int j = 0; j < nc; ++j) {
      const double2 m = Ah[(int64_t)j * nc];
      const double2 v = *reinterpret_cast<const double2*>(xn + ((int64_t)j * cd.Vc + nb) * 2);
      yr += m.x * v.x - m.y * v.y;
      yi += m.x * v.y + m.y * v.x;
    }
  }
  const double2 xv = *reinterpret_cast<const double2*>(xn + ((int64_t)i * cd.Vc + a) * 2);
  const double tw = (i < nc / 2 ? 1.0 : -1.0) * dmu * mu[n];
  yr -= tw * xv.y;
  yi += tw * xv.x;
  *reinterpret_cast<double2*>(y + (((int64_t)n * nc + i) * cd.Vc + a) * 2) = make_double2(yr, yi);
}

void restrict64(const AggDims& g, const double2* P64, const double* r, double* xc, int nv, int d, int nsys,
                cudaStream_t st) {
  restrict64_kernel<<<(unsigned)(g.Vc * 2), 256, sizeof(int) * g.asize, st>>>(P64, r, xc, g, nv, d, nsys);
  TM_COUNT();
}

void prolong64(const AggDims& g, const double2* P64, const double* xc, double* e, int nv, int d, int nsys,
               cudaStream_t st) {
  prolong64_kernel<<<(unsigned)(g.Vc * 2), 256, sizeof(int) * g.asize, st>>>(P64, xc, e, g, nv, d, nsys);
  TM_COUNT();
}

void coarse_apply64(const CoarseDims& cd, const double2* A64, const double* x, double* y, const double* mu,
                    double dmu, int nsys, cudaStream_t st) {
  const int64_t total = (int64_t)nsys * cd.Vc * cd.nc;
  coarse_apply64_kernel<<<(unsigned)((total + 127) / 128), 128, 0, st>>>(A64, x, y, mu, dmu, nsys, cd);
  TM_COUNT();
}

}  // namespace tmamg

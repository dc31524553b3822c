// Coarse stencil on the tensor cores: operator packing, per-system range scan and the
// stand-alone launch of the stencil phase (coarse_mma.cuh holds the phase itself).
#include "coarse_mma.cuh"
#include "profile.cuh"

namespace tmamg {

// one thread per 16-byte row piece (site a, hop h, k-group kk, row i); rows i fastest so that
// the column-major FP32 blocks are read coalesced
__global__ void pack_a16_kernel(const float2* __restrict__ A, __half* __restrict__ A16, int64_t Vc, int nc) {
  const int ncp = cm_ncp(nc), MG = ncp / 8, KG = ncp / 4;
  const int64_t total = Vc * 9 * KG * ncp;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= total) return;
  const int i = (int)(q % ncp);
  int64_t r = q / ncp;
  const int kk = (int)(r % KG);
  r /= KG;
  const int h = (int)(r % 9);
  const int64_t a = r / 9;
  __align__(16) __half v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int k = 8 * kk + e;
    const bool im = k >= ncp;
    const int j = im ? k - ncp : k;
    float val = 0.f;
    if (i < nc && j < nc) {
      const float2 z = A[(((int64_t)h * Vc + a) * nc + j) * nc + i];
      val = im ? z.y : z.x;
    }
    v[e] = __float2half_rn(val);
  }
  unsigned char* dst = reinterpret_cast<unsigned char*>(A16) + a * cm_site_bytes(nc) + h * cm_hop_bytes(nc) +
                       (int64_t)(kk * MG + i / 8) * 128 + (i % 8) * 16;
  *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(v);
}

void pack_coarse_f16(const CoarseDims& cd, const float2* A, __half* A16, cudaStream_t st) {
  const int ncp = cm_ncp(cd.nc);
  const int64_t total = cd.Vc * 9 * (ncp / 4) * ncp;
  pack_a16_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(A, A16, cd.Vc, cd.nc);
  TM_COUNT();
}

// mx[n] = max |x_n| over all entries (as the bit pattern of a non-negative float, so that an
// integer maximum orders them); grid (blocks, tiles)
__global__ void maxabs_kernel(const float* __restrict__ x, float* mx, int64_t M, int nsys) {
  const int t = blockIdx.y;
  const float4* xt = reinterpret_cast<const float4*>(x) + (int64_t)t * M;
  float m0 = 0.f, m1 = 0.f;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < M; e += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = xt[e];
    m0 = fmaxf(m0, fmaxf(fabsf(v.x), fabsf(v.z)));
    m1 = fmaxf(m1, fmaxf(fabsf(v.y), fabsf(v.w)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
    m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (2 * t < nsys) atomicMax(reinterpret_cast<int*>(mx) + 2 * t, __float_as_int(m0));
    if (2 * t + 1 < nsys) atomicMax(reinterpret_cast<int*>(mx) + 2 * t + 1, __float_as_int(m1));
  }
}

// B images of x with the power-of-two scaling of CM_SCALE_MAX
__global__ void __launch_bounds__(256) convert_x16_kernel(const float* __restrict__ x, __half* X16, int64_t Vc, int nc,
                                                          int nsys, const float* mx) {
  __shared__ float sin[CM_MAXSYS];
  for (int n = threadIdx.x; n < nsys; n += blockDim.x) {
    float si, so;
    cm_sys_scale(mx, CM_SCALE_MAX, n, si, so);
    sin[n] = si;
  }
  __syncthreads();
  cm_convert(x, X16, Vc, nc, nsys, sin, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
             (int64_t)gridDim.x * blockDim.x);
}

__global__ void __launch_bounds__(CM_THREADS, 1) coarse_mma_kernel(CmArgs q) {
  __shared__ CmShared cs;
  extern __shared__ __align__(128) unsigned char cm_dyn[];
  cm_begin(cs);
  CmPipe pipe;
  cm_apply(q, cs, cm_dyn, pipe, blockIdx.x, gridDim.x);
  cm_end(cs);
}

size_t cm_dyn_cap(const void* kernel) {
  const int optin = device_smem_optin();
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return 0;
  const size_t used = fa.sharedSizeBytes + 1024;  // static shared memory and the per-CTA reserve
  return (size_t)optin > used ? (size_t)optin - used : 0;
}

int coarse_apply_f16(const CoarseDims& cd, const __half* A16, const float* x, float* y, const double* mu, double dmu,
                     int nsys, float* mx, __half* X16, int* err, cudaStream_t st, const double* eps) {
  TM_PROF(st, "coarse_apply_f16");
  const int sms = device_sms();
  const size_t cap = cm_dyn_cap((const void*)coarse_mma_kernel);
  func_smem_optin((const void*)coarse_mma_kernel, (int)cap);
  if (nsys <= 0) return 0;
  if (cd.nc > CM_MAXNC || cd.nc < 1 || nsys > CM_MAXSYS) return -2;
  const int nstage = cm_nstage(cd.nc, nsys, cap);
  if (nstage < 2) return -2;
  const int nt = ntiles(nsys, 2);
  const int64_t M = (int64_t)cd.nc * cd.Vc;
  cudaMemsetAsync(mx, 0, sizeof(float) * nsys, st);
  int bx = (int)((M + 255) / 256);
  if (bx > 64) bx = 64;
  maxabs_kernel<<<dim3(bx, nt), 256, 0, st>>>(x, mx, M, nsys);
  TM_COUNT();
  const int ncp = cm_ncp(cd.nc), S = cm_chunk(nsys);
  const int64_t items = cd.Vc * cm_nchunk(nsys) * (S / 2) * (ncp / 8);
  convert_x16_kernel<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(x, X16, cd.Vc, cd.nc, nsys, mx);
  TM_COUNT();
  CmArgs q;
  q.A16 = A16;
  q.X16 = X16;
  for (int k = 0; k < 4; ++k) q.L[k] = cd.L[k];
  q.Vc = cd.Vc;
  q.nc = cd.nc;
  q.x = x;
  q.y = y;
  q.mu = mu;
  q.dmu = dmu;
  q.scale = mx;
  q.mode = CM_SCALE_MAX;
  q.nsys = nsys;
  q.nstage = nstage;
  q.err = err;
  q.eps = eps;
  const int64_t G = cd.Vc < sms ? cd.Vc : sms;
  coarse_mma_kernel<<<(unsigned)G, CM_THREADS, cm_smem_bytes(cd.nc, nsys, nstage), st>>>(q);
  TM_COUNT();
  return 0;
}

}  // namespace tmamg

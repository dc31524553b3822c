// Red-black Schwarz alternating procedure (SAP) smoother on GB300.
//
// Paper Sec. 2: the lattice is cut into blocks coloured like a chessboard; the local Dirac
// operators of all blocks of one colour are (approximately) inverted at once, red first,
// then black. Here each block solve is `steps` minimal-residual steps on the block
// operator D_B (hops that leave the block dropped) from a zero start.
//
// GPU design: one CTA per (block, system tile), one thread per block site. The block
// residual rho and the block correction live in shared memory; the block operator reads
// neighbours from shared memory and links/clover from global memory (L1/L2 resident
// across the MR steps). Because neighbouring blocks always have the other colour, the
// residual on a block right after its solve is exactly the final MR residual, and the
// residual on the other colour changes only through hops that cross a block face: a
// second kernel subtracts those hops, so SAP needs no full-lattice operator application.
#include "sap.cuh"
#include "stencil.cuh"

namespace tmamg {

struct SapDims {
  int L[4];
  int bs[4];
  int nb[4];
  int bv;
  int bc_t;
};

__device__ __forceinline__ void block_site(const SapDims& d, int b, int tid, int* bc, int* lc, int* c) {
  bc[0] = b % d.nb[0];
  int r = b / d.nb[0];
  bc[1] = r % d.nb[1];
  r /= d.nb[1];
  bc[2] = r % d.nb[2];
  bc[3] = r / d.nb[2];
  lc[0] = tid % d.bs[0];
  r = tid / d.bs[0];
  lc[1] = r % d.bs[1];
  r /= d.bs[1];
  lc[2] = r % d.bs[2];
  lc[3] = r / d.bs[2];
#pragma unroll
  for (int k = 0; k < 4; ++k) c[k] = bc[k] * d.bs[k] + lc[k];
}

__device__ __forceinline__ int local_index(const int* lc, const SapDims& d) {
  return ((lc[3] * d.bs[2] + lc[2]) * d.bs[1] + lc[1]) * d.bs[0] + lc[0];
}

template <int T>
__device__ __forceinline__ void block_reduce(float* v, int n, float* red) {
  // sums v[0..n) over the CTA; every thread gets the totals (n <= 8); blockDim.x is a
  // multiple of 32, so every warp is full
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = (blockDim.x + 31) >> 5;
  for (int i = 0; i < n; ++i) {
    float x = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    v[i] = x;
  }
  if (lane == 0)
    for (int i = 0; i < n; ++i) red[warp * 8 + i] = v[i];
  __syncthreads();
  for (int i = 0; i < n; ++i) {
    float s = 0;
    for (int w = 0; w < nw; ++w) s += red[w * 8 + i];
    v[i] = s;
  }
  __syncthreads();
}

// CTA of ceil(bv / 32) * 32 threads: thread tid < bv owns block site tid; the others only
// take part in the reductions and barriers with zero contributions.
template <typename real, int T>
__global__ void __launch_bounds__(256, 2) sap_mr_kernel(const float2* __restrict__ U, const real* __restrict__ C,
                                                        real* __restrict__ r, real* __restrict__ delta,
                                                        real* __restrict__ e, const double* __restrict__ mu, int nsys,
                                                        SapDims d, int colour, int steps) {
  extern __shared__ float4 sm[];
  float4* rho = sm;                    // [12][bv]
  float4* eb = sm + 12 * d.bv;         // [12][bv]
  float* red = reinterpret_cast<float*>(sm + 24 * d.bv);  // [nwarps][8]
  const int b = blockIdx.x;
  const int tid = threadIdx.x;
  const bool act = tid < d.bv;
  int bc[4], lc[4], c[4];
  block_site(d, b, act ? tid : 0, bc, lc, c);
  if (((bc[0] + bc[1] + bc[2] + bc[3]) & 1) != colour) return;  // whole CTA: same block
  const int64_t V = (int64_t)d.L[0] * d.L[1] * d.L[2] * d.L[3];
  const int64_t s = site_index(c, d.L);
  const int tile = blockIdx.y;
  const int64_t tstride = (int64_t)12 * V * 2 * T;
  real* rt = r + tile * tstride;
  if (act) {
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      rho[k * d.bv + tid] = *reinterpret_cast<const float4*>(rt + ((int64_t)k * V + s) * 2 * T);
      eb[k * d.bv + tid] = make_float4(0, 0, 0, 0);
    }
  }
  real m[T];
#pragma unroll
  for (int l = 0; l < T; ++l) {
    int n = tile * T + l;
    m[l] = n < nsys ? (real)mu[n] : real(0);
  }
  // in-block neighbours: local index or -1; phase for a wrap in t inside a block spanning t
  int nf[4], nbk[4];
  real pf[4], pb[4];
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) {
    int l2[4] = {lc[0], lc[1], lc[2], lc[3]};
    pf[nu] = 1;
    pb[nu] = 1;
    if (lc[nu] + 1 < d.bs[nu]) {
      l2[nu] = lc[nu] + 1;
      nf[nu] = local_index(l2, d);
    } else if (d.nb[nu] == 1) {
      l2[nu] = 0;
      nf[nu] = local_index(l2, d);
      if (nu == 3) pf[nu] = (real)d.bc_t;
    } else {
      nf[nu] = -1;
    }
    l2[nu] = lc[nu];
    if (lc[nu] > 0) {
      l2[nu] = lc[nu] - 1;
      nbk[nu] = local_index(l2, d);
    } else if (d.nb[nu] == 1) {
      l2[nu] = d.bs[nu] - 1;
      nbk[nu] = local_index(l2, d);
      if (nu == 3) pb[nu] = (real)d.bc_t;
    } else {
      nbk[nu] = -1;
    }
  }
  const int64_t strides[4] = {1, (int64_t)d.L[0], (int64_t)d.L[0] * d.L[1], (int64_t)d.L[0] * d.L[1] * d.L[2]};
  for (int it = 0; it < steps; ++it) {
    __syncthreads();
    Spinor<real, T> q;
#pragma unroll
    for (int k = 0; k < 12; ++k)
#pragma unroll
      for (int l = 0; l < T; ++l) { q.c[k].re[l] = 0; q.c[k].im[l] = 0; }
    float v[3 * T];
#pragma unroll
    for (int l = 0; l < T; ++l) { v[3 * l] = 0; v[3 * l + 1] = 0; v[3 * l + 2] = 0; }
    if (act) {
      const real* rb = reinterpret_cast<const real*>(rho);
#define TM_BHOP(NU)                                                                                      \
      {                                                                                                  \
        if (nf[NU] >= 0)                                                                                 \
          hop<NU, true, real, T>(q, rb + (int64_t)nf[NU] * 2 * T, d.bv, U + (int64_t)NU * 9 * V, V, s, pf[NU]); \
        if (nbk[NU] >= 0) {                                                                              \
          int64_t sb = c[NU] > 0 ? s - strides[NU] : s + (int64_t)(d.L[NU] - 1) * strides[NU];           \
          hop<NU, false, real, T>(q, rb + (int64_t)nbk[NU] * 2 * T, d.bv, U + (int64_t)NU * 9 * V, V, sb, pb[NU]); \
        }                                                                                                \
      }
      TM_BHOP(0)
      TM_BHOP(1)
      TM_BHOP(2)
      TM_BHOP(3)
#undef TM_BHOP
      local_term<real, T>(q, rb + (int64_t)tid * 2 * T, d.bv, C, V, s, m);
      // partial <q, q> and <q, rho> per system
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        float4 rr = rho[k * d.bv + tid];
        float rre[2] = {rr.x, rr.y}, rim[2] = {rr.z, rr.w};
#pragma unroll
        for (int l = 0; l < T; ++l) {
          float qr = q.c[k].re[l], qi = q.c[k].im[l];
          v[3 * l] += qr * qr + qi * qi;
          v[3 * l + 1] += qr * rre[l] + qi * rim[l];
          v[3 * l + 2] += qr * rim[l] - qi * rre[l];
        }
      }
    }
    block_reduce<T>(v, 3 * T, red);  // contains the barrier: every q is computed, rho may change
    float ar[T], ai[T];
#pragma unroll
    for (int l = 0; l < T; ++l) {
      float qq = v[3 * l];
      ar[l] = qq > 0.f ? v[3 * l + 1] / qq : 0.f;
      ai[l] = qq > 0.f ? v[3 * l + 2] / qq : 0.f;
    }
    if (act) {
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        float4 rr = rho[k * d.bv + tid];
        float4 ee = eb[k * d.bv + tid];
        float rre[2] = {rr.x, rr.y}, rim[2] = {rr.z, rr.w};
        float ere[2] = {ee.x, ee.y}, eim[2] = {ee.z, ee.w};
#pragma unroll
        for (int l = 0; l < T; ++l) {
          ere[l] += ar[l] * rre[l] - ai[l] * rim[l];
          eim[l] += ar[l] * rim[l] + ai[l] * rre[l];
          float qr = q.c[k].re[l], qi = q.c[k].im[l];
          rre[l] -= ar[l] * qr - ai[l] * qi;
          rim[l] -= ar[l] * qi + ai[l] * qr;
        }
        rho[k * d.bv + tid] = make_float4(rre[0], rre[1], rim[0], rim[1]);
        eb[k * d.bv + tid] = make_float4(ere[0], ere[1], eim[0], eim[1]);
      }
    }
  }
  if (!act) return;
  real* dt = delta + tile * tstride;
  real* et = e + tile * tstride;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    int64_t o = ((int64_t)k * V + s) * 2 * T;
    float4 ee = eb[k * d.bv + tid];
    *reinterpret_cast<float4*>(dt + o) = ee;
    float4 e0 = *reinterpret_cast<const float4*>(et + o);
    *reinterpret_cast<float4*>(et + o) = make_float4(e0.x + ee.x, e0.y + ee.y, e0.z + ee.z, e0.w + ee.w);
    *reinterpret_cast<float4*>(rt + o) = rho[k * d.bv + tid];
  }
}

// r(s) -= (D delta)(s) on the sites of the blocks of colour `other`, where delta is nonzero
// only on the blocks of the other colour: only hops across a block face contribute,
// D's hop term is -1/2 sum hops, so r += 1/2 sum_{crossing hops} hop(delta).
template <typename real, int T>
__global__ void __launch_bounds__(256) sap_face_kernel(const float2* __restrict__ U, const real* __restrict__ delta,
                                                       real* __restrict__ r, SapDims d, int other, int ntile) {
  const int64_t V = (int64_t)d.L[0] * d.L[1] * d.L[2] * d.L[3];
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int tile = blockIdx.y;
  if (s >= V || tile >= ntile) return;
  int c[4];
  site_coords(s, d.L, c);
  int col = 0;
  bool fwd[4], bwd[4];
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) {
    col += c[nu] / d.bs[nu];
    fwd[nu] = d.nb[nu] > 1 && (c[nu] % d.bs[nu]) == d.bs[nu] - 1;
    bwd[nu] = d.nb[nu] > 1 && (c[nu] % d.bs[nu]) == 0;
  }
  if ((col & 1) != other) return;
  if (!(fwd[0] || fwd[1] || fwd[2] || fwd[3] || bwd[0] || bwd[1] || bwd[2] || bwd[3])) return;
  const int64_t tstride = (int64_t)12 * V * 2 * T;
  const real* dt = delta + tile * tstride;
  Spinor<real, T> acc;
#pragma unroll
  for (int k = 0; k < 12; ++k)
#pragma unroll
    for (int l = 0; l < T; ++l) { acc.c[k].re[l] = 0; acc.c[k].im[l] = 0; }
  const int64_t strides[4] = {1, (int64_t)d.L[0], (int64_t)d.L[0] * d.L[1], (int64_t)d.L[0] * d.L[1] * d.L[2]};
#define TM_FHOP(NU)                                                                                   \
  {                                                                                                   \
    if (fwd[NU]) {                                                                                    \
      int64_t sf = c[NU] + 1 < d.L[NU] ? s + strides[NU] : s - (int64_t)(d.L[NU] - 1) * strides[NU];  \
      real ph = (NU == 3 && c[3] == d.L[3] - 1) ? (real)d.bc_t : real(1);                           \
      hop<NU, true, real, T>(acc, dt + sf * 2 * T, V, U + (int64_t)NU * 9 * V, V, s, ph);              \
    }                                                                                                 \
    if (bwd[NU]) {                                                                                    \
      int64_t sb = c[NU] > 0 ? s - strides[NU] : s + (int64_t)(d.L[NU] - 1) * strides[NU];             \
      real ph = (NU == 3 && c[3] == 0) ? (real)d.bc_t : real(1);                                     \
      hop<NU, false, real, T>(acc, dt + sb * 2 * T, V, U + (int64_t)NU * 9 * V, V, sb, ph);            \
    }                                                                                                 \
  }
  TM_FHOP(0)
  TM_FHOP(1)
  TM_FHOP(2)
  TM_FHOP(3)
#undef TM_FHOP
  real* rt = r + tile * tstride;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    int64_t o = ((int64_t)k * V + s) * 2 * T;
    float4 v = *reinterpret_cast<const float4*>(rt + o);
    v.x += 0.5f * acc.c[k].re[0];
    v.y += 0.5f * acc.c[k].re[1];
    v.z += 0.5f * acc.c[k].im[0];
    v.w += 0.5f * acc.c[k].im[1];
    *reinterpret_cast<float4*>(rt + o) = v;
  }
}

int sap_check_blocks(const Geom& g, const int bs[4], std::string& why) {
  int bv = 1;
  for (int k = 0; k < 4; ++k) {
    if (bs[k] < 1 || g.L[k] % bs[k]) {
      why = "SAP block extent must divide the lattice extent";
      return -1;
    }
    int nb = g.L[k] / bs[k];
    if (nb != 1 && nb % 2) {
      why = "SAP needs an even number of blocks (or one block) per dimension";
      return -1;
    }
    bv *= bs[k];
  }
  if (bv > 256 || bv < 2) {
    why = "SAP block volume must be in [2, 256]";
    return -1;
  }
  return 0;
}

void sap_apply(const Geom& g, const int bs[4], const float2* U32, const float* C32, float* r, float* e, float* delta,
               const double* mu, int nsys, int cycles, int steps, cudaStream_t st) {
  SapDims d;
  int nblocks = 1;
  for (int k = 0; k < 4; ++k) {
    d.L[k] = g.L[k];
    d.bs[k] = bs[k];
    d.nb[k] = g.L[k] / bs[k];
    nblocks *= d.nb[k];
  }
  d.bv = bs[0] * bs[1] * bs[2] * bs[3];
  d.bc_t = g.bc_t;
  constexpr int T = Tile<float>::T;
  int nt = ntiles(nsys, T);
  size_t M = (size_t)12 * g.V * 2 * T * nt;
  cudaMemsetAsync(e, 0, M * sizeof(float), st);
  int nwarps = (d.bv + 31) / 32;
  int nthreads = nwarps * 32;
  size_t smem = sizeof(float4) * 24 * d.bv + sizeof(float) * 8 * nwarps;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(sap_mr_kernel<float, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 110 * 1024);
    attr = true;
  }
  for (int cy = 0; cy < cycles; ++cy) {
    for (int colour = 0; colour < 2; ++colour) {
      sap_mr_kernel<float, T><<<dim3(nblocks, nt), nthreads, smem, st>>>(U32, C32, r, delta, e, mu, nsys, d, colour,
                                                                      steps); TM_COUNT();
      bool last = (cy == cycles - 1) && colour == 1;
      if (!last) {
        sap_face_kernel<float, T><<<dim3((unsigned)((g.V + 255) / 256), nt), 256, 0, st>>>(U32, delta, r, d,
                                                                                          1 - colour, nt); TM_COUNT();
      }
    }
  }
}

}  // namespace tmamg

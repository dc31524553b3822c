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
  int pdim;  // first dimension with two or more blocks (colours alternate along it), -1 if one block
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

// Persistent block solver: CTA b takes a contiguous range of the work items (block of this
// colour, tile), item = k * ntile + tile, so consecutive items mostly share a block. The
// block's links and clover are staged in shared memory once per block and serve every tile
// and every MR step. Two threads per block site, one per system of the tile (adjacent lanes,
// so their link and clover reads are shared-memory broadcasts); the block residual rho lives
// in shared memory as [12][bv][2 systems] (re, im) pairs, the block correction in registers.
//
// shared memory: links [4 nu][9][bv] float2, clover [72][bv] float, rho [12][bv][2] float2,
// reduction scratch [nwarps][2 systems][3] float
constexpr int SAP_THREADS = 512;

__device__ __forceinline__ int colour_block(const SapDims& d, int colour, int k) {
  if (d.pdim < 0) return k;  // one block covers the lattice (colour 0 only)
  const int p = d.pdim, half = d.nb[p] / 2;
  const int j = k % half;
  int rest = k / half;
  int c[4];
  int par = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q == p) continue;
    c[q] = rest % d.nb[q];
    rest /= d.nb[q];
    par += c[q];
  }
  c[p] = 2 * j + ((colour + par) & 1);
  return ((c[3] * d.nb[2] + c[2]) * d.nb[1] + c[1]) * d.nb[0] + c[0];
}

// sums of v[0..2] over the CTA's threads of system l = lane & 1; every thread gets its
// system's totals
__device__ __forceinline__ void pair_reduce(float* v, float* red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float x = v[i];
#pragma unroll
    for (int o = 16; o > 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    v[i] = x;
  }
  if (lane < 2)
    for (int i = 0; i < 3; ++i) red[(warp * 2 + lane) * 3 + i] = v[i];
  __syncthreads();
  const int l = lane & 1;
  for (int i = 0; i < 3; ++i) {
    float s = 0;
    for (int w = 0; w < nw; ++w) s += red[(w * 2 + l) * 3 + i];
    v[i] = s;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(SAP_THREADS, 1) sap_mr_kernel(const float2* __restrict__ U,
                                                                const float* __restrict__ C, float* __restrict__ r,
                                                                float* __restrict__ delta, float* __restrict__ e,
                                                                const double* __restrict__ mu, int nsys, SapDims d,
                                                                int colour, int steps, int nitems, int ntile) {
  constexpr int T = 2;  // systems per tile of the global bundles
  extern __shared__ float4 sm[];
  const int bv = d.bv;
  float2* Ls = reinterpret_cast<float2*>(sm);              // [4][9][bv]
  float* Cs = reinterpret_cast<float*>(Ls + 36 * bv);      // [72][bv]
  float2* rho = reinterpret_cast<float2*>(Cs + 72 * bv);   // [12][bv][2]
  float* red = reinterpret_cast<float*>(rho + 24 * bv);    // [nwarps][2][3]
  const int site = threadIdx.x >> 1, l = threadIdx.x & 1;
  const bool act = site < bv;
  const int64_t V = (int64_t)d.L[0] * d.L[1] * d.L[2] * d.L[3];
  const int64_t tstride = (int64_t)12 * V * 2 * T;
  const int per = (nitems + gridDim.x - 1) / gridDim.x;
  const int i0 = blockIdx.x * per;
  const int i1 = i0 + per < nitems ? i0 + per : nitems;
  int cur = -1;  // block whose links are staged
  int bc[4], lc[4], c[4];
  int64_t s = 0;
  int nf[4], nbk[4];
  float pf[4], pb[4];
  for (int item = i0; item < i1; ++item) {
    const int k = item / ntile, tile = item % ntile;
    const int b = colour_block(d, colour, k);
    __syncthreads();  // the previous item's reads of rho (and of the staged block) are done
    if (b != cur) {
      cur = b;
      block_site(d, b, act ? site : 0, bc, lc, c);
      s = site_index(c, d.L);
      if (act) {
        // links of the block: U_nu(x) for x in the block (forward hops, and backward hops
        // through the in-block neighbour x - nu, whose own forward link it is); the two
        // threads of a site split the loads
        for (int q = l; q < 36; q += 2) Ls[q * bv + site] = U[(int64_t)q * V + s];
        for (int q = l; q < 72; q += 2) Cs[q * bv + site] = C[(int64_t)q * V + s];
      }
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
          if (nu == 3) pf[nu] = (float)d.bc_t;
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
          if (nu == 3) pb[nu] = (float)d.bc_t;
        } else {
          nbk[nu] = -1;
        }
      }
    }
    float* rt = r + tile * tstride;
    CV<float, 1> eb[12];
#pragma unroll
    for (int k2 = 0; k2 < 12; ++k2) {
      eb[k2].re[0] = 0.f;
      eb[k2].im[0] = 0.f;
      if (act) {
        const float4 g = *reinterpret_cast<const float4*>(rt + ((int64_t)k2 * V + s) * 2 * T);
        rho[(k2 * bv + site) * 2 + l] = l == 0 ? make_float2(g.x, g.z) : make_float2(g.y, g.w);
      }
    }
    const int n = tile * T + l;
    float m[1] = {n < nsys ? (float)mu[n] : 0.f};
    const float* rb = reinterpret_cast<const float*>(rho) + 2 * l;  // this thread's system
    for (int it = 0; it < steps; ++it) {
      __syncthreads();  // rho (and the staged links) complete
      Spinor<float, 1> q;
#pragma unroll
      for (int k2 = 0; k2 < 12; ++k2) { q.c[k2].re[0] = 0; q.c[k2].im[0] = 0; }
      float v[3] = {0.f, 0.f, 0.f};
      if (act) {
#define TM_BHOP(NU)                                                                                              \
        {                                                                                                        \
          if (nf[NU] >= 0)                                                                                       \
            hop<NU, true, float, 1>(q, rb + (int64_t)nf[NU] * 4, 2 * bv, Ls + NU * 9 * bv, bv, site, pf[NU]);     \
          if (nbk[NU] >= 0)                                                                                      \
            hop<NU, false, float, 1>(q, rb + (int64_t)nbk[NU] * 4, 2 * bv, Ls + NU * 9 * bv, bv, nbk[NU], pb[NU]); \
        }
        TM_BHOP(0)
        TM_BHOP(1)
        TM_BHOP(2)
        TM_BHOP(3)
#undef TM_BHOP
        local_term<float, 1>(q, rb + (int64_t)site * 4, 2 * bv, Cs, bv, site, m);
        // partial <q, q> and <q, rho>
#pragma unroll
        for (int k2 = 0; k2 < 12; ++k2) {
          const float2 rr = rho[(k2 * bv + site) * 2 + l];
          const float qr = q.c[k2].re[0], qi = q.c[k2].im[0];
          v[0] += qr * qr + qi * qi;
          v[1] += qr * rr.x + qi * rr.y;
          v[2] += qr * rr.y - qi * rr.x;
        }
      }
      pair_reduce(v, red);  // contains the barrier: every q is computed, rho may change
      const float ar = v[0] > 0.f ? v[1] / v[0] : 0.f;
      const float ai = v[0] > 0.f ? v[2] / v[0] : 0.f;
      if (act) {
#pragma unroll
        for (int k2 = 0; k2 < 12; ++k2) {
          float2 rr = rho[(k2 * bv + site) * 2 + l];
          eb[k2].re[0] += ar * rr.x - ai * rr.y;
          eb[k2].im[0] += ar * rr.y + ai * rr.x;
          const float qr = q.c[k2].re[0], qi = q.c[k2].im[0];
          rr.x -= ar * qr - ai * qi;
          rr.y -= ar * qi + ai * qr;
          rho[(k2 * bv + site) * 2 + l] = rr;
        }
      }
    }
    // write back: the even lane of a site assembles the tile's 16-byte entries
    __syncwarp();  // the partner lane's last rho update is visible
    {
      float* dt = delta + tile * tstride;
      float* et = e + tile * tstride;
#pragma unroll
      for (int k2 = 0; k2 < 12; ++k2) {
        const float er = __shfl_xor_sync(0xffffffffu, eb[k2].re[0], 1);
        const float ei = __shfl_xor_sync(0xffffffffu, eb[k2].im[0], 1);
        if (act && l == 0) {
          const int64_t o = ((int64_t)k2 * V + s) * 2 * T;
          const float4 dv = make_float4(eb[k2].re[0], er, eb[k2].im[0], ei);
          *reinterpret_cast<float4*>(dt + o) = dv;
          const float4 e0 = *reinterpret_cast<const float4*>(et + o);
          *reinterpret_cast<float4*>(et + o) = make_float4(e0.x + dv.x, e0.y + dv.y, e0.z + dv.z, e0.w + dv.w);
          const float2 r0 = rho[(k2 * bv + site) * 2], r1 = rho[(k2 * bv + site) * 2 + 1];
          *reinterpret_cast<float4*>(rt + o) = make_float4(r0.x, r1.x, r0.y, r1.y);
        }
      }
    }
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
  d.pdim = -1;
  for (int k = 3; k >= 0; --k)
    if (d.nb[k] >= 2) d.pdim = k;
  constexpr int T = Tile<float>::T;
  int nt = ntiles(nsys, T);
  size_t M = (size_t)12 * g.V * 2 * T * nt;
  cudaMemsetAsync(e, 0, M * sizeof(float), st);
  const int nthreads = (2 * d.bv + 31) / 32 * 32;  // two threads per block site
  const int nwarps = nthreads / 32;
  // links [4][9][bv] float2 + clover [72][bv] + rho [12][bv][2] float2 + reduction scratch
  size_t smem = sizeof(float2) * 36 * d.bv + sizeof(float) * 72 * d.bv + sizeof(float2) * 24 * d.bv +
                sizeof(float) * 6 * nwarps;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(sap_mr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  }
  const int per_colour = d.pdim < 0 ? 1 : nblocks / 2;
  for (int cy = 0; cy < cycles; ++cy) {
    for (int colour = 0; colour < 2; ++colour) {
      const int nb_c = d.pdim < 0 ? (colour == 0 ? 1 : 0) : per_colour;
      const int nitems = nb_c * nt;
      if (nitems > 0) {
        const int grid = nitems < sms ? nitems : sms;
        sap_mr_kernel<<<grid, nthreads, smem, st>>>(U32, C32, r, delta, e, mu, nsys, d, colour, steps, nitems, nt);
        TM_COUNT();
      }
      bool last = (cy == cycles - 1) && colour == 1;
      if (!last) {
        sap_face_kernel<float, T><<<dim3((unsigned)((g.V + 255) / 256), nt), 256, 0, st>>>(U32, delta, r, d,
                                                                                          1 - colour, nt); TM_COUNT();
      }
    }
  }
}

}  // namespace tmamg

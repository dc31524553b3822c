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
#include "profile.cuh"
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

template <int N>
__device__ __forceinline__ void block_reduce(float (&v)[N], float* red) {
  // sums v[0..N) over the CTA; every thread gets the totals (N <= 8); blockDim.x is a
  // multiple of 32, so every warp is full. Fixed-size and fully unrolled, so v stays in registers.
  // One barrier: the caller alternates between two scratch buffers `red`, so a buffer is written
  // again only after a later barrier that every reader of its previous contents has passed.
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float x = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    v[i] = x;
  }
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < N; ++i) red[warp * 8 + i] = v[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float s = 0;
    for (int w = 0; w < nw; ++w) s += red[w * 8 + i];
    v[i] = s;
  }
}

__device__ __forceinline__ void sap_cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void sap_cp_async_wait() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Persistent block solver: CTA b takes a contiguous range of the work items (block of this
// colour, tile), item = k * ntile + tile, so consecutive items mostly share a block. The
// block's links and clover are staged in shared memory once per block and serve every tile
// and every MR step; the block residual rho lives in shared memory (neighbours read it), the
// block correction in registers. One thread per block site handles the tile's two systems in
// packed FP32x2 arithmetic; CTA of ceil(bv / 32) * 32 threads (the threads past bv only take
// part in the reductions and barriers).
//
// shared memory: links [4 nu][9][bv] float2, clover [72][bv] float, rho [12][bv] float4,
// reduction scratch [2][nwarps][8] float
constexpr int SAP_THREADS = 256;
constexpr int SAP_MAX_TILES = 128;  // system tiles per call (256 systems)

__device__ __forceinline__ int colour_block(const SapDims& d, int colour, int k) {
  if (d.pdim < 0) return k;  // one block covers the lattice (colour 0 only)
  // the k-th block of this colour: dimension p = pdim takes 2 j + parity, the others the digits of
  // k / half; written with selects on p so that no array is indexed at run time (that would put
  // the arrays in local memory)
  const int p = d.pdim;
  const int half = (p == 0 ? d.nb[0] : p == 1 ? d.nb[1] : p == 2 ? d.nb[2] : d.nb[3]) / 2;
  const int j = k % half;
  int rest = k / half;
  int c[4];
  int par = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q == p) {
      c[q] = 0;
      continue;
    }
    c[q] = rest % d.nb[q];
    rest /= d.nb[q];
    par += c[q];
  }
  const int cp = 2 * j + ((colour + par) & 1);
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (q == p) c[q] = cp;
  return ((c[3] * d.nb[2] + c[2]) * d.nb[1] + c[1]) * d.nb[0] + c[0];
}

__global__ void __launch_bounds__(SAP_THREADS, 1) sap_mr_kernel(const float2* __restrict__ U,
                                                                const float* __restrict__ C, float* __restrict__ r,
                                                                float* __restrict__ delta, float* __restrict__ e,
                                                                const double* __restrict__ mu, int nsys, SapDims d,
                                                                int colour, int steps, int nitems, int ntile,
                                                                const double* __restrict__ eps) {
  constexpr int T = 2;  // systems per tile
  extern __shared__ float4 sm[];
  const int bv = d.bv;
  float2* Ls = reinterpret_cast<float2*>(sm);              // [4][9][bv]
  float* Cs = reinterpret_cast<float*>(Ls + 36 * bv);      // [72][bv]
  float4* rho = reinterpret_cast<float4*>(Cs + 72 * bv);   // [12][bv]
  float* red = reinterpret_cast<float*>(rho + 12 * bv);    // [nwarps][8]
  const int tid = threadIdx.x;
  const bool act = tid < bv;
  const int64_t V = (int64_t)d.L[0] * d.L[1] * d.L[2] * d.L[3];
  const int64_t tstride = (int64_t)12 * V * 2 * T;
  // every tile's twisted masses (and doublet splitting) in shared memory once per CTA
  __shared__ float2 mu_s[SAP_MAX_TILES];
  __shared__ float ep_s[SAP_MAX_TILES];
  for (int t = tid; t < ntile; t += blockDim.x) {
    const int n0 = t * T;
    mu_s[t] = make_float2(n0 < nsys ? (float)mu[n0] : 0.f, n0 + 1 < nsys ? (float)mu[n0 + 1] : 0.f);
    ep_s[t] = eps ? (float)eps[t] : 0.f;
  }
  const int nwarps = (int)((blockDim.x + 31) >> 5);
  const int per = (nitems + gridDim.x - 1) / gridDim.x;
  const int i0 = blockIdx.x * per;
  const int i1 = i0 + per < nitems ? i0 + per : nitems;
  int cur = -1;  // block whose links are staged
  int bc[4], lc[4], c[4];
  int64_t s = 0;
  int nf[4], nbk[4];
  float pf[4], pb[4];
  // the residual of an item is fetched into rho by asynchronous copies (each thread its own site's
  // twelve entries), for the next item while the current one writes its results back
  auto fetch_rho = [&](int item_) {
    const int k_ = item_ / ntile, t_ = item_ % ntile;
    int bc_[4], lc_[4], c_[4];
    block_site(d, colour_block(d, colour, k_), act ? tid : 0, bc_, lc_, c_);
    const int64_t s_ = site_index(c_, d.L);
    const float* rt_ = r + t_ * tstride;
    if (act) {
#pragma unroll
      for (int k2 = 0; k2 < 12; ++k2) sap_cp_async16(&rho[k2 * bv + tid], rt_ + ((int64_t)k2 * V + s_) * 2 * T);
    }
  };
  if (i0 < i1) fetch_rho(i0);
  for (int item = i0; item < i1; ++item) {
    const int k = item / ntile, tile = item % ntile;
    const int b = colour_block(d, colour, k);
    __syncthreads();  // the previous item's reads of rho (and of the staged block) are done
    if (b != cur) {
      cur = b;
      block_site(d, b, act ? tid : 0, bc, lc, c);
      s = site_index(c, d.L);
      if (act) {
        // links of the block: U_nu(x) for x in the block (forward hops, and backward hops
        // through the in-block neighbour x - nu, whose own forward link it is)
#pragma unroll 12
        for (int q = 0; q < 36; ++q) Ls[q * bv + tid] = U[(int64_t)q * V + s];
#pragma unroll 12
        for (int q = 0; q < 72; ++q) Cs[q * bv + tid] = C[(int64_t)q * V + s];
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
    CV2 eb[12];
#pragma unroll
    for (int k2 = 0; k2 < 12; ++k2) {
      eb[k2].re = make_float2(0.f, 0.f);
      eb[k2].im = make_float2(0.f, 0.f);
    }
    sap_cp_async_wait();  // this thread's residual entries are in rho (the barrier below publishes them)
    const float2 m2 = mu_s[tile];
    // doublet form (eps): the tile's two systems are the flavours of one doublet, one MR system
    const float ep = ep_s[tile];
    const float* rb = reinterpret_cast<const float*>(rho);
    for (int it = 0; it < steps; ++it) {
      __syncthreads();  // rho (and the staged links) complete
      Spinor2 q;
#pragma unroll
      for (int k2 = 0; k2 < 12; ++k2) {
        q.c[k2].re = make_float2(0.f, 0.f);
        q.c[k2].im = make_float2(0.f, 0.f);
      }
      float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (act) {
#define TM_BHOP(NU)                                                                              \
        {                                                                                        \
          if (nf[NU] >= 0)                                                                       \
            hop2<NU, true>(q, rb + nf[NU] * 4, bv, Ls + NU * 9 * bv, bv, tid, NU == 3 ? pf[3] : 1.f); \
          if (nbk[NU] >= 0)                                                                      \
            hop2<NU, false>(q, rb + nbk[NU] * 4, bv, Ls + NU * 9 * bv, bv, nbk[NU], NU == 3 ? pb[3] : 1.f); \
        }
        TM_BHOP(0)
        TM_BHOP(1)
        TM_BHOP(2)
        TM_BHOP(3)
#undef TM_BHOP
        local2(q, rb + tid * 4, bv, Cs, bv, tid, m2, ep);
        // partial <q, q> and <q, rho> per system (packed over the two systems)
        float2 qq = make_float2(0.f, 0.f), qr = qq, qi = qq;
#pragma unroll
        for (int k2 = 0; k2 < 12; ++k2) {
          const float4 rr = rho[k2 * bv + tid];
          const float2 rre = make_float2(rr.x, rr.y), rim = make_float2(rr.z, rr.w);
          const CV2& qv = q.c[k2];
          qq = fma2(qv.re, qv.re, qq);
          qq = fma2(qv.im, qv.im, qq);
          qr = fma2(qv.re, rre, qr);
          qr = fma2(qv.im, rim, qr);
          qi = fma2(qv.re, rim, qi);
          qi = fma2(f2(-1.f), mul2(qv.im, rre), qi);
        }
        v[0] = qq.x; v[1] = qr.x; v[2] = qi.x;
        v[3] = qq.y; v[4] = qr.y; v[5] = qi.y;
      }
      block_reduce(v, red + (it & 1) * 8 * nwarps);  // its barrier: every q is computed, rho may change
      if (eps) {  // one minimal-residual step for the doublet: the dots summed over both flavours
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const float t = v[u] + v[3 + u];
          v[u] = t;
          v[3 + u] = t;
        }
      }
      const float2 ar = make_float2(v[0] > 0.f ? v[1] / v[0] : 0.f, v[3] > 0.f ? v[4] / v[3] : 0.f);
      const float2 ai = make_float2(v[0] > 0.f ? v[2] / v[0] : 0.f, v[3] > 0.f ? v[5] / v[3] : 0.f);
      const float2 nai = make_float2(-ai.x, -ai.y);
      if (act) {
#pragma unroll
        for (int k2 = 0; k2 < 12; ++k2) {
          const float4 rr = rho[k2 * bv + tid];
          float2 rre = make_float2(rr.x, rr.y), rim = make_float2(rr.z, rr.w);
          // e += alpha rho; rho -= alpha q (alpha = ar + i ai per system)
          eb[k2].re = fma2(ar, rre, eb[k2].re);
          eb[k2].re = fma2(nai, rim, eb[k2].re);
          eb[k2].im = fma2(ar, rim, eb[k2].im);
          eb[k2].im = fma2(ai, rre, eb[k2].im);
          const CV2& qv = q.c[k2];
          rre = fma2(f2(-1.f), mul2(ar, qv.re), rre);
          rre = fma2(ai, qv.im, rre);
          rim = fma2(f2(-1.f), mul2(ar, qv.im), rim);
          rim = fma2(nai, qv.re, rim);
          rho[k2 * bv + tid] = make_float4(rre.x, rre.y, rim.x, rim.y);
        }
      }
    }
    if (act) {
      float* dt = delta + tile * tstride;
      float* et = e + tile * tstride;
      // every load of e first (twelve in flight), then the stores
      CV2 e0[12];
#pragma unroll
      for (int k2 = 0; k2 < 12; ++k2) e0[k2] = ld2(et + ((int64_t)k2 * V + s) * 2 * T);
#pragma unroll
      for (int k2 = 0; k2 < 12; ++k2) {
        const int64_t o = ((int64_t)k2 * V + s) * 2 * T;
        st2(dt + o, eb[k2]);
        e0[k2].re = add2(e0[k2].re, eb[k2].re);
        e0[k2].im = add2(e0[k2].im, eb[k2].im);
        st2(et + o, e0[k2]);
        *reinterpret_cast<float4*>(rt + o) = rho[k2 * bv + tid];
      }
    }
    // rho is private per thread from the last barrier on (neighbour reads ended before it): the
    // next item's residual may be fetched into this thread's entries now
    if (item + 1 < i1) fetch_rho(item + 1);
  }
}

// r(s) -= (D delta)(s) on the sites of the blocks of colour `other`, where delta is nonzero
// only on the blocks of the other colour: only hops across a block face contribute,
// D's hop term is -1/2 sum hops, so r += 1/2 sum_{crossing hops} hop(delta).
template <typename real, int T>
__global__ void __launch_bounds__(256) sap_face_kernel(const float2* __restrict__ U, const real* __restrict__ delta,
                                                       real* __restrict__ r, SapDims d, int other, int ntile) {
  // threads over the sites of the blocks of colour `other` only (block k of that colour, site q
  // in the block), so that no lane of a warp idles on a site of the wrong colour
  const int64_t V = (int64_t)d.L[0] * d.L[1] * d.L[2] * d.L[3];
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int tile = blockIdx.y;
  const int nbc = d.pdim < 0 ? 0 : (int)(V / d.bv / 2);
  if (idx >= (int64_t)nbc * d.bv || tile >= ntile) return;
  const int k = (int)(idx / d.bv), q = (int)(idx % d.bv);
  int bc[4], lc[4], c[4];
  block_site(d, colour_block(d, other, k), q, bc, lc, c);
  const int64_t s = site_index(c, d.L);
  bool fwd[4], bwd[4];
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) {
    fwd[nu] = d.nb[nu] > 1 && lc[nu] == d.bs[nu] - 1;
    bwd[nu] = d.nb[nu] > 1 && lc[nu] == 0;
  }
  if (!(fwd[0] || fwd[1] || fwd[2] || fwd[3] || bwd[0] || bwd[1] || bwd[2] || bwd[3])) return;
  const int64_t tstride = (int64_t)12 * V * 2 * T;
  const real* dt = delta + tile * tstride;
  static_assert(sizeof(real) == 4 && T == 2, "packed FP32 tiles");
  Spinor2 acc;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    acc.c[k].re = make_float2(0.f, 0.f);
    acc.c[k].im = make_float2(0.f, 0.f);
  }
  const int64_t strides[4] = {1, (int64_t)d.L[0], (int64_t)d.L[0] * d.L[1], (int64_t)d.L[0] * d.L[1] * d.L[2]};
#define TM_FHOP(NU)                                                                                   \
  {                                                                                                   \
    if (fwd[NU]) {                                                                                    \
      int64_t sf = c[NU] + 1 < d.L[NU] ? s + strides[NU] : s - (int64_t)(d.L[NU] - 1) * strides[NU];  \
      real ph = (NU == 3 && c[3] == d.L[3] - 1) ? (real)d.bc_t : real(1);                           \
      hop2<NU, true>(acc, dt + sf * 2 * T, V, U + (int64_t)NU * 9 * V, V, s, ph);                      \
    }                                                                                                 \
    if (bwd[NU]) {                                                                                    \
      int64_t sb = c[NU] > 0 ? s - strides[NU] : s + (int64_t)(d.L[NU] - 1) * strides[NU];             \
      real ph = (NU == 3 && c[3] == 0) ? (real)d.bc_t : real(1);                                     \
      hop2<NU, false>(acc, dt + sb * 2 * T, V, U + (int64_t)NU * 9 * V, V, sb, ph);                    \
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
    v.x += 0.5f * acc.c[k].re.x;
    v.y += 0.5f * acc.c[k].re.y;
    v.z += 0.5f * acc.c[k].im.x;
    v.w += 0.5f * acc.c[k].im.y;
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
               const double* mu, int nsys, int cycles, int steps, cudaStream_t st, bool accumulate,
               const double* eps) {
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
  if (!accumulate) cudaMemsetAsync(e, 0, M * sizeof(float), st);
  const int nthreads = (d.bv + 31) / 32 * 32;  // one thread per block site
  const int nwarps = nthreads / 32;
  if (nt > SAP_MAX_TILES) return;  // callers check (at most 256 systems)
  // links [4][9][bv] float2 + clover [72][bv] + rho [12][bv] float4 + reduction scratch (two buffers)
  size_t smem = sizeof(float2) * 36 * d.bv + sizeof(float) * 72 * d.bv + sizeof(float4) * 12 * d.bv +
                sizeof(float) * 2 * 8 * nwarps;
  const int sms = device_sms();
  func_smem_optin((const void*)sap_mr_kernel, 200 * 1024);
  // persistent grid: as many CTAs as fit on the device at once (smaller blocks fit two per SM)
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sap_mr_kernel, nthreads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int per_colour = d.pdim < 0 ? 1 : nblocks / 2;
  for (int cy = 0; cy < cycles; ++cy) {
    for (int colour = 0; colour < 2; ++colour) {
      const int nb_c = d.pdim < 0 ? (colour == 0 ? 1 : 0) : per_colour;
      const int nitems = nb_c * nt;
      if (nitems > 0) {
        const int grid = nitems < sms * per_sm ? nitems : sms * per_sm;
        TM_PROF(st, "sap_mr");
        sap_mr_kernel<<<grid, nthreads, smem, st>>>(U32, C32, r, delta, e, mu, nsys, d, colour, steps, nitems, nt,
                                                    eps);
        TM_COUNT();
      }
      bool last = (cy == cycles - 1) && colour == 1;
      if (!last && d.pdim >= 0) {
        TM_PROF(st, "sap_face");
        const int64_t nsite = (int64_t)(nblocks / 2) * d.bv;  // sites of the blocks of the other colour
        sap_face_kernel<float, T><<<dim3((unsigned)((nsite + 255) / 256), nt), 256, 0, st>>>(U32, delta, r, d,
                                                                                            1 - colour, nt); TM_COUNT();
      }
    }
  }
}

}  // namespace tmamg

// ================================================================== plain FP64 form
// The same red-black SAP (MR block solves, face-only residual update) in FP64 for the plain
// comparator solver: FP64 bundles with one system per tile, links and clover from their FP64
// copies in global memory. One CTA per (block of the colour, system), one thread per site; the
// block residual in shared memory, the block correction in registers.
namespace tmamg {

__device__ __forceinline__ void block_reduce_d(double* v, int n, double* red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = (blockDim.x + 31) >> 5;
  for (int i = 0; i < n; ++i) {
    double x = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    v[i] = x;
  }
  if (lane == 0)
    for (int i = 0; i < n; ++i) red[warp * 4 + i] = v[i];
  __syncthreads();
  for (int i = 0; i < n; ++i) {
    double s = 0;
    for (int w = 0; w < nw; ++w) s += red[w * 4 + i];
    v[i] = s;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) sap64_mr_kernel(const double2* __restrict__ U, const double* __restrict__ C,
                                                       double* __restrict__ r, double* __restrict__ delta,
                                                       double* __restrict__ e, const double* __restrict__ mu,
                                                       SapDims d, int colour, int steps) {
  extern __shared__ double2 sm64[];
  const int bv = d.bv;
  double2* rho = sm64;                                       // [12][bv]
  double* red = reinterpret_cast<double*>(rho + 12 * bv);   // [nwarps][4]
  const int tid = threadIdx.x;
  const bool act = tid < bv;
  const int b = colour_block(d, colour, blockIdx.x);
  const int n = blockIdx.y;  // system (one per tile)
  int bc[4], lc[4], c[4];
  block_site(d, b, act ? tid : 0, bc, lc, c);
  const int64_t V = (int64_t)d.L[0] * d.L[1] * d.L[2] * d.L[3];
  const int64_t s = site_index(c, d.L);
  const int64_t tstride = (int64_t)12 * V * 2;
  double* rt = r + n * tstride;
  Spinor<double, 1> eb;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    eb.c[k].re[0] = 0;
    eb.c[k].im[0] = 0;
    if (act) rho[k * bv + tid] = *reinterpret_cast<const double2*>(rt + ((int64_t)k * V + s) * 2);
  }
  double m[1] = {mu[n]};
  int nf[4], nbk[4];
  double pf[4], pb[4];
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
      if (nu == 3) pf[nu] = (double)d.bc_t;
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
      if (nu == 3) pb[nu] = (double)d.bc_t;
    } else {
      nbk[nu] = -1;
    }
  }
  const int64_t strides[4] = {1, (int64_t)d.L[0], (int64_t)d.L[0] * d.L[1], (int64_t)d.L[0] * d.L[1] * d.L[2]};
  const double* rb = reinterpret_cast<const double*>(rho);
  for (int it = 0; it < steps; ++it) {
    __syncthreads();
    Spinor<double, 1> q;
#pragma unroll
    for (int k = 0; k < 12; ++k) { q.c[k].re[0] = 0; q.c[k].im[0] = 0; }
    double v[3] = {0, 0, 0};
    if (act) {
#define TM_BHOP64(NU)                                                                                      \
      {                                                                                                    \
        if (nf[NU] >= 0)                                                                                   \
          hop<NU, true, double, 1>(q, rb + (int64_t)nf[NU] * 2, bv, U + (int64_t)NU * 9 * V, V, s, pf[NU]); \
        if (nbk[NU] >= 0) {                                                                                \
          int64_t sb = c[NU] > 0 ? s - strides[NU] : s + (int64_t)(d.L[NU] - 1) * strides[NU];             \
          hop<NU, false, double, 1>(q, rb + (int64_t)nbk[NU] * 2, bv, U + (int64_t)NU * 9 * V, V, sb, pb[NU]); \
        }                                                                                                  \
      }
      TM_BHOP64(0)
      TM_BHOP64(1)
      TM_BHOP64(2)
      TM_BHOP64(3)
#undef TM_BHOP64
      local_term<double, 1>(q, rb + (int64_t)tid * 2, bv, C, V, s, m);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const double2 rr = rho[k * bv + tid];
        const double qr = q.c[k].re[0], qi = q.c[k].im[0];
        v[0] += qr * qr + qi * qi;
        v[1] += qr * rr.x + qi * rr.y;
        v[2] += qr * rr.y - qi * rr.x;
      }
    }
    block_reduce_d(v, 3, red);
    const double ar = v[0] > 0 ? v[1] / v[0] : 0.0, ai = v[0] > 0 ? v[2] / v[0] : 0.0;
    if (act) {
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        double2 rr = rho[k * bv + tid];
        eb.c[k].re[0] += ar * rr.x - ai * rr.y;
        eb.c[k].im[0] += ar * rr.y + ai * rr.x;
        const double qr = q.c[k].re[0], qi = q.c[k].im[0];
        rr.x -= ar * qr - ai * qi;
        rr.y -= ar * qi + ai * qr;
        rho[k * bv + tid] = rr;
      }
    }
  }
  if (!act) return;
  double* dt = delta + n * tstride;
  double* et = e + n * tstride;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const int64_t o = ((int64_t)k * V + s) * 2;
    *reinterpret_cast<double2*>(dt + o) = make_double2(eb.c[k].re[0], eb.c[k].im[0]);
    const double2 e0 = *reinterpret_cast<const double2*>(et + o);
    *reinterpret_cast<double2*>(et + o) = make_double2(e0.x + eb.c[k].re[0], e0.y + eb.c[k].im[0]);
    *reinterpret_cast<double2*>(rt + o) = rho[k * bv + tid];
  }
}

// r(s) += 1/2 sum over block-crossing hops of delta on the sites of blocks of colour `other`
__global__ void __launch_bounds__(256) sap64_face_kernel(const double2* __restrict__ U,
                                                         const double* __restrict__ delta, double* __restrict__ r,
                                                         SapDims d, int other) {
  const int64_t V = (int64_t)d.L[0] * d.L[1] * d.L[2] * d.L[3];
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int n = blockIdx.y;
  if (s >= V) return;
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
  const int64_t tstride = (int64_t)12 * V * 2;
  const double* dt = delta + n * tstride;
  Spinor<double, 1> acc;
#pragma unroll
  for (int k = 0; k < 12; ++k) { acc.c[k].re[0] = 0; acc.c[k].im[0] = 0; }
  const int64_t strides[4] = {1, (int64_t)d.L[0], (int64_t)d.L[0] * d.L[1], (int64_t)d.L[0] * d.L[1] * d.L[2]};
#define TM_FHOP64(NU)                                                                                  \
  {                                                                                                    \
    if (fwd[NU]) {                                                                                     \
      int64_t sf = c[NU] + 1 < d.L[NU] ? s + strides[NU] : s - (int64_t)(d.L[NU] - 1) * strides[NU];   \
      double ph = (NU == 3 && c[3] == d.L[3] - 1) ? (double)d.bc_t : 1.0;                            \
      hop<NU, true, double, 1>(acc, dt + sf * 2, V, U + (int64_t)NU * 9 * V, V, s, ph);                 \
    }                                                                                                  \
    if (bwd[NU]) {                                                                                     \
      int64_t sb = c[NU] > 0 ? s - strides[NU] : s + (int64_t)(d.L[NU] - 1) * strides[NU];              \
      double ph = (NU == 3 && c[3] == 0) ? (double)d.bc_t : 1.0;                                      \
      hop<NU, false, double, 1>(acc, dt + sb * 2, V, U + (int64_t)NU * 9 * V, V, sb, ph);               \
    }                                                                                                  \
  }
  TM_FHOP64(0)
  TM_FHOP64(1)
  TM_FHOP64(2)
  TM_FHOP64(3)
#undef TM_FHOP64
  double* rt = r + n * tstride;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const int64_t o = ((int64_t)k * V + s) * 2;
    double2 v = *reinterpret_cast<const double2*>(rt + o);
    v.x += 0.5 * acc.c[k].re[0];
    v.y += 0.5 * acc.c[k].im[0];
    *reinterpret_cast<double2*>(rt + o) = v;
  }
}

void sap_apply64(const Geom& g, const int bs[4], const double2* U64, const double* C64, double* r, double* e,
                 double* delta, const double* mu, int nsys, int cycles, int steps, cudaStream_t st) {
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
  cudaMemsetAsync(e, 0, sizeof(double) * 24 * g.V * nsys, st);
  const int nthreads = (d.bv + 31) / 32 * 32;
  const size_t smem = sizeof(double2) * 12 * d.bv + sizeof(double) * 4 * (nthreads / 32);
  func_smem_optin((const void*)sap64_mr_kernel, 64 * 1024);  // 4^4 blocks need 49 KB, above the default limit
  for (int cy = 0; cy < cycles; ++cy) {
    for (int colour = 0; colour < 2; ++colour) {
      const int nb_c = d.pdim < 0 ? (colour == 0 ? 1 : 0) : nblocks / 2;
      if (nb_c > 0) {
        sap64_mr_kernel<<<dim3(nb_c, nsys), nthreads, smem, st>>>(U64, C64, r, delta, e, mu, d, colour, steps);
        TM_COUNT();
      }
      if (!(cy == cycles - 1 && colour == 1)) {
        sap64_face_kernel<<<dim3((unsigned)((g.V + 255) / 256), nsys), 256, 0, st>>>(U64, delta, r, d, 1 - colour);
        TM_COUNT();
      }
    }
  }
}

}  // namespace tmamg

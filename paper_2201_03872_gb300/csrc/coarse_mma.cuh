// Coarse stencil D_c on the fifth-generation tensor cores (tcgen05, sm_103a).
//
//   y_n(a) = sum_h A_h(a) x_n(a + h) + i dmu mu_n gamma5_c x_n(a)
//
// over the nine hops h of the coarse lattice (paper Sec. 2: the coarse operator keeps the
// nearest-neighbour structure of the fine one; Sec. 3: matrix data is read once for all
// right-hand sides). The stencil blocks are stored in FP16, the vector entries are converted
// to FP16 while they are staged, products accumulate in FP32 in tensor memory.
//
// One coarse site is one small GEMM per chunk of S systems:
//   D [nc x 2S] = sum_h [Re A_h | Im A_h] (nc x 2 ncp)  .  B_h (2 ncp x 2S),
// with B_h built from x(a + h) so that the complex product comes out of one real contraction:
// for system s of tile-pair slot (tp, lane l) the four accumulator columns 4 tp + {0,1,2,3} are
// (Re y_{2tp}, Re y_{2tp+1}, Im y_{2tp}, Im y_{2tp+1}) -- exactly one 16-byte entry of the
// vector bundle. B rows: column q of slot tp takes (Re x, -Im x) for q = 0, 1 and (Im x, Re x)
// for q = 2, 3 over the [Re | Im] halves of K.
//
// Operands live in shared memory in the no-swizzle K-major core-matrix layout (8 rows x 16 B
// per core matrix, contiguous); the operator is stored in HBM already in that layout, so one
// bulk copy per hop brings it in. The accumulator uses M = 128 rows of which the first nc are
// read; the descriptor's remaining row groups alias other staged data and are never read.
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

#include "amg.cuh"

namespace tmamg {

constexpr int CM_THREADS = 256;   // threads of a CTA that runs the stencil phase
constexpr int CM_MAXS = 16;       // systems per accumulator chunk (2S <= 32 columns)
constexpr int CM_TMEM_COLS = 32;  // tensor-memory columns held per CTA
constexpr int CM_SLACK = 2048;    // bytes past the last A buffer the M = 128 descriptor may touch
constexpr int CM_MAXNC = 64;      // rows of D read back by warps 0 and 1

__host__ __device__ inline int cm_ncp(int nc) { return (nc + 7) / 8 * 8; }
__host__ __device__ inline int64_t cm_hop_bytes(int nc) {
  const int64_t n = cm_ncp(nc);
  return 4 * n * n;  // ncp rows x 2 ncp columns x 2 bytes
}
__host__ __device__ inline int64_t cm_site_bytes(int nc) { return 9 * cm_hop_bytes(nc); }
// systems per chunk: the accumulator width N = 2S must be a multiple of 16 for M = 128
__host__ __device__ inline int cm_chunk(int nsys) { return nsys > 8 ? CM_MAXS : 8; }
__host__ __device__ inline int64_t cm_b_bytes(int nc, int S) { return 9LL * 8 * cm_ncp(nc) * S; }
// dynamic shared memory of the phase with nbuf operator buffers
inline size_t cm_smem_bytes(int nc, int S, int nbuf) {
  return (size_t)nbuf * cm_site_bytes(nc) + cm_b_bytes(nc, S) + CM_SLACK;
}

struct CmShared {
  unsigned long long mbar[3];  // operator buffers 0 and 1, accumulator ready
  unsigned tmem;
  int fail;
  int64_t nb[9];
  float sin_[CM_MAXS], sout[CM_MAXS], tw[CM_MAXS];
};

// per-system scaling of the staged FP16 vector entries (the FP16 range is kept for any input):
//   CM_SCALE_IN:  x is multiplied by scale[n] (double); y is not rescaled
//   CM_SCALE_OUT: x is divided by scale[n] and y multiplied by it (double; <= 0 means 1)
//   CM_SCALE_MAX: scale[n] is max |x_n| (float); a power of two 2^e >= it is divided out of x
//                 and multiplied back into y (exact)
enum { CM_SCALE_IN = 0, CM_SCALE_OUT = 1, CM_SCALE_MAX = 2 };

struct CmArgs {
  const __half* A16;  // [Vc][9 hops][cm_hop_bytes] operator in the core-matrix layout
  int L[4];
  int64_t Vc;
  int nc;
  const float* x;     // FP32 bundles [ntile][nc][Vc][4]
  float* y;
  const double* mu;   // [nsys]
  double dmu;
  const void* scale;
  int mode;
  int nsys;
  int nbuf;           // operator buffers in shared memory (2: next site prefetched)
  int* err;           // set to 2 when a bounded wait gives up
};

__device__ __forceinline__ uint32_t cm_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool cm_try_wait(uint32_t mb, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mb), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait (about one second at 2 GHz); gives up early when another thread failed
__device__ __forceinline__ bool cm_wait(uint32_t mb, uint32_t parity, volatile int* fail) {
  const long long t0 = clock64();
  while (!cm_try_wait(mb, parity)) {
    if (*fail) return false;
    if (clock64() - t0 > 2000000000LL) {
      *fail = 1;
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void cm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void cm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// shared-memory matrix descriptor: no swizzle, K-major core matrices; lbo = byte stride between
// core matrices along K, sbo = along M (or N)
__device__ __forceinline__ uint64_t cm_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this tensor-core generation
  return d;
}

// CTA prologue: barriers and tensor memory (every thread calls it)
__device__ __forceinline__ void cm_begin(CmShared& cs) {
  if (threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(cm_smem(&cs.mbar[k])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    cs.fail = 0;
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(cm_smem(&cs.tmem)),
                 "n"(CM_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  cm_fence_before();
  __syncthreads();
  cm_fence_after();
}

// CTA epilogue: releases the tensor memory (every thread calls it, after the last phase)
__device__ __forceinline__ void cm_end(CmShared& cs) {
  cm_fence_before();
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(cs.tmem), "n"(CM_TMEM_COLS));
}

// per-system factors of chunk c into shared memory (threads < S)
__device__ __forceinline__ void cm_chunk_scales(const CmArgs& q, CmShared& cs, int c, int S) {
  const int k = threadIdx.x;
  if (k >= S) return;
  const int n = c * S + k;
  float si = 0.f, so = 0.f, tw = 0.f;
  if (n < q.nsys) {
    double in = 1.0, out = 1.0;
    if (q.scale) {
      if (q.mode == CM_SCALE_IN) {
        in = __ldcg(reinterpret_cast<const double*>(q.scale) + n);
      } else if (q.mode == CM_SCALE_OUT) {
        const double v = __ldcg(reinterpret_cast<const double*>(q.scale) + n);
        if (v > 0.0) {
          in = 1.0 / v;
          out = v;
        }
      } else {
        const float mx = __ldcg(reinterpret_cast<const float*>(q.scale) + n);
        if (mx > 0.f && isfinite(mx)) {
          int e;
          frexpf(mx, &e);  // mx < 2^e
          in = ldexp(1.0, -e);
          out = ldexp(1.0, e);
        }
      }
    }
    si = (float)in;
    so = (float)out;
    tw = (float)(q.dmu * q.mu[n]);
  }
  cs.sin_[k] = si;
  cs.sout[k] = so;
  cs.tw[k] = tw;
}

// two FP16 values (round to nearest even), a in the low half (the lower address)
__device__ __forceinline__ uint32_t cm_pack2(float a, float b) {
  uint32_t d;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;\n" : "=r"(d) : "f"(b), "f"(a));
  return d;
}

// one staging item of the B operands: the eight components 8g .. 8g+7 of tile c TP + tp at
// the neighbour of hop h (item = (h TP + tp) MG + g), scaled per system
__device__ __forceinline__ void cm_item_load(const CmArgs& q, const CmShared& cs, int item, int c, int MG, int TP,
                                             int nt, float4* v) {
  const int g = item % MG;
  const int r = item / MG;
  const int tp = r % TP, h = r / TP;
  const int t = c * TP + tp;
  const int64_t nbh = cs.nb[h];
  const int nc = q.nc;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int j = 8 * g + u;
    v[u] = (t < nt && j < nc) ? __ldcg(reinterpret_cast<const float4*>(q.x + ((((int64_t)t * nc + j) * q.Vc) + nbh) * 4))
                              : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// rows n = 4 tp + q' of B^T at k-groups g (Re half of K) and MG + g (Im half):
// q' = 0: (Re x_{2t}, -Im x_{2t}); 1: (Re x_{2t+1}, -Im x_{2t+1}); 2: (Im x_{2t}, Re x_{2t});
// 3: (Im x_{2t+1}, Re x_{2t+1})
__device__ __forceinline__ void cm_item_store(const CmShared& cs, unsigned char* sB, int item, int MG, int TP, int NG,
                                              uint32_t BH, const float4* vin) {
  const int g = item % MG;
  const int r = item / MG;
  const int tp = r % TP, h = r / TP;
  const float s0 = cs.sin_[2 * tp], s1 = cs.sin_[2 * tp + 1];
  float4 v[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) v[u] = make_float4(vin[u].x * s0, vin[u].y * s1, vin[u].z * s0, vin[u].w * s1);
  unsigned char* hb = sB + (size_t)h * BH;
  const int n0 = 4 * tp;
  const uint32_t rowoff = (uint32_t)((n0 >> 3) * 128 + (n0 & 7) * 16);
  unsigned char* lo = hb + (size_t)g * NG * 128 + rowoff;         // k in [8g, 8g + 8)
  unsigned char* hi = hb + (size_t)(MG + g) * NG * 128 + rowoff;  // k in ncp + [8g, 8g + 8)
#define CM_ROW(F, SG) make_uint4(cm_pack2(SG v[0].F, SG v[1].F), cm_pack2(SG v[2].F, SG v[3].F), \
                                 cm_pack2(SG v[4].F, SG v[5].F), cm_pack2(SG v[6].F, SG v[7].F))
  *reinterpret_cast<uint4*>(lo) = CM_ROW(x, +);
  *reinterpret_cast<uint4*>(hi) = CM_ROW(z, -);
  *reinterpret_cast<uint4*>(lo + 16) = CM_ROW(y, +);
  *reinterpret_cast<uint4*>(hi + 16) = CM_ROW(w, -);
  *reinterpret_cast<uint4*>(lo + 32) = CM_ROW(z, +);
  *reinterpret_cast<uint4*>(hi + 32) = CM_ROW(x, +);
  *reinterpret_cast<uint4*>(lo + 48) = CM_ROW(w, +);
  *reinterpret_cast<uint4*>(hi + 48) = CM_ROW(y, +);
#undef CM_ROW
}

// The stencil over the sites a = cta, cta + ncta, ... (every thread of the CTA calls it).
// ph carries the barrier parities between calls (bit 0, 1: operator buffers, bit 2: accumulator).
// Returns false when a bounded wait gave up (q.err is then set to 2).
static __device__ __forceinline__ bool cm_apply(const CmArgs& q, CmShared& cs, unsigned char* dsm, unsigned& ph,
                                                int64_t cta, int64_t ncta) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nc = q.nc, ncp = cm_ncp(nc);
  const int MG = ncp / 8;          // row groups of A (and k-groups per half of K)
  const int KS = ncp / 8;          // K steps of 16 over [Re | Im]
  const int S = cm_chunk(q.nsys), N = 2 * S, NG = S / 4, TP = S / 2;
  const int nchunk = (q.nsys + S - 1) / S;
  const int nt = (q.nsys + 1) / 2;
  const uint32_t HA = (uint32_t)cm_hop_bytes(nc), SA = 9 * HA;
  const uint32_t BH = (uint32_t)(8 * ncp * S);
  unsigned char* sB = dsm + (size_t)q.nbuf * SA;
  const uint32_t sA0 = cm_smem(dsm), sB0 = cm_smem(sB);
  const uint32_t mbD = cm_smem(&cs.mbar[2]);
  const uint32_t idesc = (1u << 4)                       // FP32 accumulator
                         | ((uint32_t)(N >> 3) << 17)    // N
                         | ((uint32_t)(128 >> 4) << 24); // M = 128; FP16 A and B, both K-major
  const unsigned char* Ag = reinterpret_cast<const unsigned char*>(q.A16);
  volatile int* fail = &cs.fail;

  auto load_site = [&](int64_t a, int buf) {  // one thread
    const uint32_t mb = cm_smem(&cs.mbar[buf]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mb), "r"(SA) : "memory");
    const unsigned char* src = Ag + a * (int64_t)SA;
    for (int h = 0; h < 9; ++h)
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
              sA0 + buf * SA + h * HA),
          "l"(src + (int64_t)h * HA), "r"(HA), "r"(mb)
          : "memory");
  };

  // shared memory last written through the generic proxy (other phases) is next written by
  // the bulk copies and read by the tensor cores (async proxy)
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  __syncthreads();
  if (tid == 0 && cta < q.Vc) load_site(cta, 0);
  int it = 0;
  for (int64_t a = cta; a < q.Vc; a += ncta, ++it) {
    const int buf = q.nbuf == 2 ? (it & 1) : 0;
    if (q.nbuf == 2 && tid == 0 && a + ncta < q.Vc) load_site(a + ncta, buf ^ 1);
    if (tid < 9) {
      // neighbour a + h (h = 1 + 2 nu forward, 2 + 2 nu backward), periodic coarse lattice
      const int L0 = q.L[0], L1 = q.L[1], L2 = q.L[2], L3 = q.L[3];
      int c0 = (int)(a % L0);
      int64_t rr = a / L0;
      int c1 = (int)(rr % L1);
      rr /= L1;
      int c2 = (int)(rr % L2);
      int c3 = (int)(rr / L2);
      if (tid > 0) {
        const int nu = (tid - 1) / 2, dir = ((tid - 1) & 1) ? -1 : 1;
        if (nu == 0) c0 = (c0 + dir + L0) % L0;
        else if (nu == 1) c1 = (c1 + dir + L1) % L1;
        else if (nu == 2) c2 = (c2 + dir + L2) % L2;
        else c3 = (c3 + dir + L3) % L3;
      }
      cs.nb[tid] = ((int64_t)(c3 * L2 + c2) * L1 + c1) * L0 + c0;
    }
    for (int c = 0; c < nchunk; ++c) {
      cm_chunk_scales(q, cs, c, S);
      __syncthreads();
      // ---- B operands of the nine hops: item = (hop, tile pair, group of 8 components); two
      // items per thread have their 16 loads in flight together
      const int nitem = 9 * TP * MG;
      for (int i0 = tid; i0 < nitem; i0 += 2 * (int)blockDim.x) {
        const int i1 = i0 + blockDim.x;
        float4 va[8], vb[8];
        cm_item_load(q, cs, i0, c, MG, TP, nt, va);
        if (i1 < nitem) cm_item_load(q, cs, i1, c, MG, TP, nt, vb);
        cm_item_store(cs, sB, i0, MG, TP, NG, BH, va);
        if (i1 < nitem) cm_item_store(cs, sB, i1, MG, TP, NG, BH, vb);
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      cm_fence_before();
      __syncthreads();
      // ---- one thread issues the 9 x KS MMAs of the chunk
      if (tid == 0) {
        bool ok = c > 0 || cm_wait(cm_smem(&cs.mbar[buf]), (ph >> buf) & 1u, fail);
        if (ok) {
          cm_fence_after();
          const uint32_t dt = cs.tmem;
          const uint32_t abase = sA0 + buf * SA;
          for (int h = 0; h < 9; ++h) {
            for (int s = 0; s < KS; ++s) {
              const uint64_t ad = cm_desc(abase + h * HA + 2 * s * MG * 128, MG * 128, 128);
              const uint64_t bd = cm_desc(sB0 + h * BH + 2 * s * NG * 128, NG * 128, 128);
              const uint32_t acc = (h | s) != 0;
              asm volatile(
                  "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                  "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbD)
                       : "memory");
        } else {
          *fail = 1;
        }
      }
      if (c == 0) ph ^= 1u << buf;
      // ---- warps 0 and 1 read rows 0..63 of the accumulator and write y
      if (warp < 2) {
        // the site's own entries for the twist term, fetched while the MMAs run
        const int i = warp * 32 + lane;
        float4 xv[CM_MAXS / 2];
#pragma unroll
        for (int tp = 0; tp < CM_MAXS / 2; ++tp) {
          const int t = c * TP + tp;
          xv[tp] = (i < nc && tp < TP && t < nt)
                       ? __ldcg(reinterpret_cast<const float4*>(q.x + ((((int64_t)t * nc + i) * q.Vc) + a) * 4))
                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (cm_wait(mbD, (ph >> 2) & 1u, fail)) {
          cm_fence_after();
          if (q.nbuf == 1 && tid == 0 && c == nchunk - 1 && a + ncta < q.Vc) load_site(a + ncta, 0);
          uint32_t r[32] = {};
          const uint32_t ta = cs.tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (8 * k < N)
              asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                           : "=r"(r[8 * k]), "=r"(r[8 * k + 1]), "=r"(r[8 * k + 2]), "=r"(r[8 * k + 3]),
                             "=r"(r[8 * k + 4]), "=r"(r[8 * k + 5]), "=r"(r[8 * k + 6]), "=r"(r[8 * k + 7])
                           : "r"(ta + 8 * k));
          }
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
          if (i < nc) {
            const float g5 = i < nc / 2 ? 1.f : -1.f;
#pragma unroll
            for (int tp = 0; tp < CM_MAXS / 2; ++tp) {
              const int t = c * TP + tp;
              if (tp < TP && t < nt) {
                const int64_t off = ((((int64_t)t * nc + i) * q.Vc) + a) * 4;
                const float si0 = cs.sin_[2 * tp], si1 = cs.sin_[2 * tp + 1];
                const float tw0 = g5 * cs.tw[2 * tp] * si0, tw1 = g5 * cs.tw[2 * tp + 1] * si1;
                const float so0 = cs.sout[2 * tp], so1 = cs.sout[2 * tp + 1];
                float4 o;
                o.x = so0 * (__uint_as_float(r[4 * tp]) - tw0 * xv[tp].z);
                o.y = so1 * (__uint_as_float(r[4 * tp + 1]) - tw1 * xv[tp].w);
                o.z = so0 * (__uint_as_float(r[4 * tp + 2]) + tw0 * xv[tp].x);
                o.w = so1 * (__uint_as_float(r[4 * tp + 3]) + tw1 * xv[tp].y);
                *reinterpret_cast<float4*>(q.y + off) = o;
              }
            }
          }
        }
      }
      ph ^= 4u;
      cm_fence_before();
      __syncthreads();
      if (cs.fail) {
        if (tid == 0) atomicExch(q.err, 2);
        return false;
      }
    }
  }
  return true;
}

// host side (coarse_mma.cu)
// FP32 stencil [9][Vc][nc col][nc row] -> FP16 operator in the core-matrix layout
void pack_coarse_f16(const CoarseDims& cd, const float2* A, __half* A16, cudaStream_t st);
// y = D_c(dmu mu_n) x with the FP16 operator; mx: nsys floats of scratch, err: device flag
// (set to 2 when a bounded wait gives up). Returns 0, or -2 for unsupported sizes.
int coarse_apply_f16(const CoarseDims& cd, const __half* A16, const float* x, float* y, const double* mu, double dmu,
                     int nsys, float* mx, int* err, cudaStream_t st);
// largest dynamic shared memory a CTA of 'kernel' may use next to its static shared memory
size_t cm_dyn_cap(const void* kernel);

}  // namespace tmamg

// Coarse stencil D_c on the fifth-generation tensor cores (tcgen05, sm_103a).
//
//   y_n(a) = sum_h A_h(a) x_n(a + h) + i dmu mu_n gamma5_c x_n(a)
//
// over the nine hops h of the coarse lattice (paper Sec. 2: the coarse operator keeps the
// nearest-neighbour structure of the fine one; Sec. 3: matrix data is read once for all
// right-hand sides). The stencil blocks are stored in FP16, the vector entries are converted
// to FP16, products accumulate in FP32 in tensor memory.
//
// One coarse site is one small GEMM per chunk of S systems:
//   D [nc x 2S] = sum_h [Re A_h | Im A_h] (nc x 2 ncp)  .  B(a + h) (2 ncp x 2S),
// with B(a') built from x(a') so that the complex product comes out of one real contraction:
// for tile-pair slot tp the four accumulator columns 4 tp + {0,1,2,3} are
// (Re y_{2tp}, Re y_{2tp+1}, Im y_{2tp}, Im y_{2tp+1}) -- exactly one 16-byte entry of the
// vector bundle. B rows: column q of slot tp takes (Re x, -Im x) for q = 0, 1 and (Im x, Re x)
// for q = 2, 3 over the [Re | Im] halves of K.
//
// Both operands are kept in HBM in the no-swizzle K-major core-matrix layout (8 rows x 16 B per
// core matrix, contiguous) in which the tensor cores read them from shared memory: the
// operator once (setup), the B images of a vector by a conversion pass before each product.
// The product is then a pipeline of bulk copies (one producer thread), MMAs (one issuing
// thread) and a tensor-memory epilogue (two warps), over a ring of shared-memory stages of
// one hop each and two accumulators. The accumulator uses M = 128 rows of which the first nc
// are read; the descriptor's remaining row groups alias other staged data and are never read.
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

#include "amg.cuh"

namespace tmamg {

constexpr int CM_THREADS = 256;   // threads of a CTA that runs the stencil phase
constexpr int CM_MAXS = 16;       // systems per accumulator chunk (2S <= 32 columns)
constexpr int CM_ACCS = 2;        // accumulators in tensor memory
constexpr int CM_TMEM_COLS = 64;  // tensor-memory columns held per CTA (two accumulators of 32)
constexpr int CM_SLACK = 2048;    // bytes past the last stage the M = 128 descriptor may touch
constexpr int CM_MAXNC = 64;      // rows of D read back by the two epilogue warps
constexpr int CM_MAXSTG = 16;     // stages in the shared-memory ring
constexpr int CM_EPI0 = 4;        // first epilogue warp (warps 4 and 5 read TMEM lanes 0..63)
constexpr int CM_TAB = 256;       // systems whose epilogue factors are tabulated in shared memory per call

__host__ __device__ inline int cm_ncp(int nc) { return (nc + 7) / 8 * 8; }
__host__ __device__ inline int64_t cm_hop_bytes(int nc) {
  const int64_t n = cm_ncp(nc);
  return 4 * n * n;  // ncp rows x 2 ncp columns x 2 bytes
}
__host__ __device__ inline int64_t cm_site_bytes(int nc) { return 9 * cm_hop_bytes(nc); }
// systems per chunk: the accumulator width N = 2S must be a multiple of 16 for M = 128
__host__ __device__ inline int cm_chunk(int nsys) { return nsys > 8 ? CM_MAXS : 8; }
__host__ __device__ inline int cm_nchunk(int nsys) { return (nsys + cm_chunk(nsys) - 1) / cm_chunk(nsys); }
// one B image: 2 ncp rows of K x 2S columns, FP16
__host__ __device__ inline int64_t cm_img_bytes(int nc, int S) { return 8LL * cm_ncp(nc) * S; }
inline size_t cm_x16_bytes(int64_t Vc, int nc, int nsys) {
  return (size_t)Vc * cm_nchunk(nsys) * cm_img_bytes(nc, cm_chunk(nsys));
}
inline size_t cm_stage_bytes(int nc, int S) { return (size_t)(cm_hop_bytes(nc) + cm_img_bytes(nc, S)); }
// stages that fit in cap bytes of dynamic shared memory (0 if fewer than two)
inline int cm_nstage(int nc, int nsys, size_t cap) {
  const size_t st = cm_stage_bytes(nc, cm_chunk(nsys));
  if (cap < CM_SLACK + 2 * st) return 0;
  const size_t n = (cap - CM_SLACK) / st;
  return n < (size_t)CM_MAXSTG ? (int)n : CM_MAXSTG;
}
inline size_t cm_smem_bytes(int nc, int nsys, int nstage) {
  return (size_t)nstage * cm_stage_bytes(nc, cm_chunk(nsys)) + CM_SLACK;
}

struct CmShared {
  unsigned long long full[CM_MAXSTG], empty[CM_MAXSTG];  // stage loaded / stage consumed
  unsigned long long tfull[CM_ACCS], tempty[CM_ACCS];    // accumulator ready / drained
  unsigned tmem;
  int fail;
  // per-system epilogue factors of the current call (systems n < CM_TAB): output scale so[n] and
  // twist dmu mu_n si[n], in FP32, so that the epilogue does no FP64 arithmetic (FP64 runs at a
  // small fraction of the FP32 rate on this GPU)
  float so[CM_TAB];
  float tw[CM_TAB];
  float ep[CM_TAB];  // doublet splitting times the input scale (0 unless q.eps)
};

// role-local pipeline position, carried from one stencil call to the next by the thread
// that holds the role (producer, MMA issuer, epilogue warps)
struct CmPipe {
  int stage = 0;
  unsigned phase = 0;
  int acc = 0;
  unsigned aphase = 0;
};

// per-system scaling of the FP16 vector entries (the FP16 range is kept for any input):
//   CM_SCALE_IN:  x is multiplied by scale[n] (double); y is not rescaled
//   CM_SCALE_OUT: x is divided by scale[n] and y multiplied by it (double; <= 0 means 1)
//   CM_SCALE_MAX: scale[n] is max |x_n| (float); a power of two 2^e >= it is divided out of x
//                 and multiplied back into y (exact)
enum { CM_SCALE_IN = 0, CM_SCALE_OUT = 1, CM_SCALE_MAX = 2 };

struct CmArgs {
  const __half* A16;  // [Vc][9 hops][cm_hop_bytes] operator in the core-matrix layout
  __half* X16;        // [Vc][chunks][cm_img_bytes] B images of x
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
  int nstage;         // stages of the shared-memory ring
  int* err;           // set to 2 when a bounded wait gives up
  const double* eps;  // [ntile] doublet splittings (the tile's lanes are the flavours u, d), or null
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
    for (int k = 0; k < CM_MAXSTG; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(cm_smem(&cs.full[k])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(cm_smem(&cs.empty[k])));
    }
    for (int k = 0; k < CM_ACCS; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(cm_smem(&cs.tfull[k])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;\n" ::"r"(cm_smem(&cs.tempty[k])));  // two warps
    }
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

// input and output factors of system n (see CM_SCALE_*)
__device__ __forceinline__ void cm_sys_scale(const void* scale, int mode, int n, float& si, float& so) {
  double in = 1.0, out = 1.0;
  if (scale) {
    if (mode == CM_SCALE_IN) {
      in = __ldcg(reinterpret_cast<const double*>(scale) + n);
    } else if (mode == CM_SCALE_OUT) {
      const double v = __ldcg(reinterpret_cast<const double*>(scale) + n);
      if (v > 0.0) {
        in = 1.0 / v;
        out = v;
      }
    } else {
      const float mx = __ldcg(reinterpret_cast<const float*>(scale) + n);
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
}

// two FP16 values (round to nearest even), a in the low half (the lower address)
__device__ __forceinline__ uint32_t cm_pack2(float a, float b) {
  uint32_t d;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;\n" : "=r"(d) : "f"(b), "f"(a));
  return d;
}

// coordinates of coarse site a (32-bit arithmetic: the producer thread computes these on the
// critical path of the copy pipeline, where 64-bit divisions cost about a microsecond per stage)
struct CmCoord {
  int c[4];
};
__device__ __forceinline__ CmCoord cm_coords(int a, int L0, int L1, int L2) {
  CmCoord k;
  k.c[0] = a % L0;
  int rr = a / L0;
  k.c[1] = rr % L1;
  rr /= L1;
  k.c[2] = rr % L2;
  k.c[3] = rr / L2;
  return k;
}
// neighbour a + h (h = 1 + 2 nu forward, 2 + 2 nu backward) of the site at k, periodic lattice;
// no division
__device__ __forceinline__ int cm_neighbour(const CmCoord& k, int h, int L0, int L1, int L2, int L3) {
  int c0 = k.c[0], c1 = k.c[1], c2 = k.c[2], c3 = k.c[3];
  if (h > 0) {
    const int nu = (h - 1) >> 1;
    const bool back = ((h - 1) & 1) != 0;
    if (nu == 0) c0 = back ? (c0 == 0 ? L0 - 1 : c0 - 1) : (c0 + 1 == L0 ? 0 : c0 + 1);
    else if (nu == 1) c1 = back ? (c1 == 0 ? L1 - 1 : c1 - 1) : (c1 + 1 == L1 ? 0 : c1 + 1);
    else if (nu == 2) c2 = back ? (c2 == 0 ? L2 - 1 : c2 - 1) : (c2 + 1 == L2 ? 0 : c2 + 1);
    else c3 = back ? (c3 == 0 ? L3 - 1 : c3 - 1) : (c3 + 1 == L3 ? 0 : c3 + 1);
  }
  return ((c3 * L2 + c2) * L1 + c1) * L0 + c0;
}

// The B images of x for all sites: item = ((a chunks + c) TP + tp) MG + g covers the eight
// components 8g .. 8g+7 of tile c TP + tp at site a. sin: input factor per system (shared
// memory, [nsys]). Items first .. total step stride; the caller fences the generic writes
// against the bulk copies that read them (fence.proxy.async.global) before its barrier.
__device__ __forceinline__ void cm_convert(const float* __restrict__ x, __half* X16, int64_t Vc, int nc, int nsys,
                                           const float* sin, int64_t first, int64_t stride) {
  const int ncp = cm_ncp(nc), MG = ncp / 8;
  const int S = cm_chunk(nsys), TP = S / 2, NG = S / 4;
  const int nchunk = cm_nchunk(nsys), nt = (nsys + 1) / 2;
  const int64_t IB = cm_img_bytes(nc, S);
  const int64_t total = Vc * nchunk * TP * MG;
  for (int64_t item = first; item < total; item += stride) {
    const int it32 = (int)item;  // Vc * chunks * TP * MG < 2^31 for every supported size
    const int g = it32 % MG;
    int r = it32 / MG;
    const int tp = r % TP;
    r /= TP;
    const int c = r % nchunk;
    const int64_t a = r / nchunk;
    const int t = c * TP + tp;
    float4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int j = 8 * g + u;
      v[u] = (t < nt && j < nc) ? __ldcg(reinterpret_cast<const float4*>(x + ((((int64_t)t * nc + j) * Vc) + a) * 4))
                                : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float s0 = 2 * t < nsys ? sin[2 * t] : 0.f, s1 = 2 * t + 1 < nsys ? sin[2 * t + 1] : 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = make_float4(v[u].x * s0, v[u].y * s1, v[u].z * s0, v[u].w * s1);
    unsigned char* img = reinterpret_cast<unsigned char*>(X16) + (a * nchunk + c) * IB;
    const int n0 = 4 * tp;
    const int64_t rowoff = (n0 >> 3) * 128 + (n0 & 7) * 16;
    unsigned char* lo = img + (int64_t)g * NG * 128 + rowoff;         // k in [8g, 8g + 8)
    unsigned char* hi = img + (int64_t)(MG + g) * NG * 128 + rowoff;  // k in ncp + [8g, 8g + 8)
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
}

__device__ __forceinline__ void cm_fence_global_async() { asm volatile("fence.proxy.async.global;\n" ::: "memory"); }

// The stencil over the units (site a, chunk c), a = cta, cta + ncta, ..., from the B images in
// q.X16 (every thread of the CTA calls it). Thread 0 loads stages (operator block of one hop
// plus the B image of that hop's neighbour), thread 32 issues the MMAs of a unit into one of
// two accumulators, warps 4 and 5 drain an accumulator while the next unit accumulates.
// pipe: this thread's role state. Returns false when a bounded wait gave up (q.err = 2).
static __device__ __forceinline__ bool cm_apply(const CmArgs& q, CmShared& cs, unsigned char* dsm, CmPipe& pipe,
                                                int64_t cta, int64_t ncta) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nc = q.nc, ncp = cm_ncp(nc);
  const int MG = ncp / 8;   // row groups of A (and k-groups per half of K)
  const int KS = ncp / 8;   // K steps of 16 over [Re | Im]
  const int S = cm_chunk(q.nsys), N = 2 * S, NG = S / 4, TP = S / 2;
  const int nchunk = cm_nchunk(q.nsys);
  const int nt = (q.nsys + 1) / 2;
  const uint32_t HA = (uint32_t)cm_hop_bytes(nc), IB = (uint32_t)cm_img_bytes(nc, S), ST = HA + IB;
  const int NS = q.nstage;
  volatile int* fail = &cs.fail;
  // shared memory last written through the generic proxy (other phases) is next written by
  // the bulk copies and read by the tensor cores (async proxy)
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  for (int n = tid; n < q.nsys && n < CM_TAB; n += blockDim.x) {
    float si, so;
    cm_sys_scale(q.scale, q.mode, n, si, so);
    cs.so[n] = so;
    cs.tw[n] = (float)(q.dmu * q.mu[n]) * si;
    cs.ep[n] = q.eps ? (float)q.eps[n >> 1] * si : 0.f;
  }
  __syncthreads();
  const uint32_t s0 = cm_smem(dsm);

  if (tid == 0) {
    // ---- producer: one stage per (unit, hop)
    cm_fence_global_async();
    const unsigned char* Ag = reinterpret_cast<const unsigned char*>(q.A16);
    const unsigned char* Xg = reinterpret_cast<const unsigned char*>(q.X16);
    const int L0 = q.L[0], L1 = q.L[1], L2 = q.L[2], L3 = q.L[3];
    for (int64_t a = cta; a < q.Vc && !*fail; a += ncta) {
      const CmCoord kc = cm_coords((int)a, L0, L1, L2);
      int nbs[9];
#pragma unroll
      for (int h = 0; h < 9; ++h) nbs[h] = cm_neighbour(kc, h, L0, L1, L2, L3);
      for (int c = 0; c < nchunk && !*fail; ++c)
#pragma unroll 1
        for (int h = 0; h < 9; ++h) {
          const int st = pipe.stage;
          if (!cm_wait(cm_smem(&cs.empty[st]), pipe.phase ^ 1u, fail)) break;
          const uint32_t fb = cm_smem(&cs.full[st]);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(ST) : "memory");
          int nb = nbs[0];
#pragma unroll
          for (int q2 = 1; q2 < 9; ++q2)
            if (h == q2) nb = nbs[q2];
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                  s0 + st * ST),
              "l"(Ag + (a * 9 + h) * (int64_t)HA), "r"(HA), "r"(fb)
              : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                  s0 + st * ST + HA),
              "l"(Xg + ((int64_t)nb * nchunk + c) * (int64_t)IB), "r"(IB), "r"(fb)
              : "memory");
          if (++pipe.stage == NS) {
            pipe.stage = 0;
            pipe.phase ^= 1u;
          }
        }
    }
  } else if (tid == 32) {
    // ---- MMA issuer: nine hops x KS steps per unit into accumulator pipe.acc
    const uint32_t idesc = (1u << 4)                        // FP32 accumulator
                           | ((uint32_t)(N >> 3) << 17)     // N
                           | ((uint32_t)(128 >> 4) << 24);  // M = 128; FP16 A and B, both K-major
    for (int64_t a = cta; a < q.Vc && !*fail; a += ncta)
      for (int c = 0; c < nchunk && !*fail; ++c) {
        const int d = pipe.acc;
        if (!cm_wait(cm_smem(&cs.tempty[d]), pipe.aphase ^ 1u, fail)) break;
        cm_fence_after();
        const uint32_t dt = cs.tmem + (uint32_t)(d * 32);
        bool ok = true;
        for (int h = 0; h < 9; ++h) {
          const int st = pipe.stage;
          if (!cm_wait(cm_smem(&cs.full[st]), pipe.phase, fail)) {
            ok = false;
            break;
          }
          cm_fence_after();
          const uint32_t ab = s0 + st * ST, bb = ab + HA;
          // k-step descriptors: the start-address field (address / 16, 14 bits) of the stage's
          // descriptor advanced by the k offset (every address stays below 2^18 bytes: no carry)
          const uint64_t ad0 = cm_desc(ab, MG * 128, 128), bd0 = cm_desc(bb, NG * 128, 128);
          for (int k = 0; k < KS; ++k) {
            const uint64_t ad = ad0 + (uint64_t)((2 * k * MG * 128) >> 4);
            const uint64_t bd = bd0 + (uint64_t)((2 * k * NG * 128) >> 4);
            const uint32_t accum = (h | k) != 0;
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
                "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
          }
          // the stage is free once these MMAs have read it
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                           cm_smem(&cs.empty[st]))
                       : "memory");
          if (++pipe.stage == NS) {
            pipe.stage = 0;
            pipe.phase ^= 1u;
          }
        }
        if (!ok) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         cm_smem(&cs.tfull[d]))
                     : "memory");
        if (++pipe.acc == CM_ACCS) {
          pipe.acc = 0;
          pipe.aphase ^= 1u;
        }
      }
  } else if (warp == CM_EPI0 || warp == CM_EPI0 + 1) {
    // ---- epilogue: rows i = 32 (warp - 4) + lane of the accumulator, twist term, scaling
    const int i = (warp - CM_EPI0) * 32 + lane;
    const float g5 = i < nc / 2 ? 1.f : -1.f;
    for (int64_t a = cta; a < q.Vc && !*fail; a += ncta)
      for (int c = 0; c < nchunk && !*fail; ++c) {
        const int d = pipe.acc;
        // the site's own entries for the twist term, fetched while the MMAs run
        float4 xv[CM_MAXS / 2];
#pragma unroll
        for (int tp = 0; tp < CM_MAXS / 2; ++tp) {
          const int t = c * TP + tp;
          xv[tp] = (i < nc && tp < TP && t < nt)
                       ? __ldcg(reinterpret_cast<const float4*>(q.x + ((((int64_t)t * nc + i) * q.Vc) + a) * 4))
                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (!cm_wait(cm_smem(&cs.tfull[d]), pipe.aphase, fail)) break;
        cm_fence_after();
        uint32_t r[32] = {};
        const uint32_t ta = cs.tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(d * 32);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (8 * k < N)
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                         : "=r"(r[8 * k]), "=r"(r[8 * k + 1]), "=r"(r[8 * k + 2]), "=r"(r[8 * k + 3]),
                           "=r"(r[8 * k + 4]), "=r"(r[8 * k + 5]), "=r"(r[8 * k + 6]), "=r"(r[8 * k + 7])
                         : "r"(ta + 8 * k));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        // the accumulator may be overwritten once both warps have read it
        cm_fence_before();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(cm_smem(&cs.tempty[d])) : "memory");
        if (++pipe.acc == CM_ACCS) {
          pipe.acc = 0;
          pipe.aphase ^= 1u;
        }
        if (i < nc) {
#pragma unroll
          for (int tp = 0; tp < CM_MAXS / 2; ++tp) {
            const int t = c * TP + tp;
            if (tp < TP && t < nt) {
              const int n0 = 2 * t;
              float so0, so1 = 0.f, tw0, tw1 = 0.f, ep0, ep1 = 0.f;
              if (n0 + 1 < CM_TAB) {
                so0 = cs.so[n0];
                tw0 = g5 * cs.tw[n0];
                ep0 = cs.ep[n0];
                if (n0 + 1 < q.nsys) {
                  so1 = cs.so[n0 + 1];
                  tw1 = g5 * cs.tw[n0 + 1];
                  ep1 = cs.ep[n0 + 1];
                }
              } else {  // systems past the table: the factors computed here
                float si0, si1 = 0.f;
                cm_sys_scale(q.scale, q.mode, n0, si0, so0);
                if (n0 + 1 < q.nsys) cm_sys_scale(q.scale, q.mode, n0 + 1, si1, so1);
                tw0 = g5 * (float)(q.dmu * q.mu[n0]) * si0;
                tw1 = n0 + 1 < q.nsys ? g5 * (float)(q.dmu * q.mu[n0 + 1]) * si1 : 0.f;
                ep0 = q.eps ? (float)q.eps[t] * si0 : 0.f;
                ep1 = q.eps ? (float)q.eps[t] * si1 : 0.f;
              }
              // twist i dmu mu g5 x, and for a doublet -eps times the other lane (flavour); the
              // coupling is skipped for degenerate systems, so that a non-finite system cannot
              // reach its tile neighbour through 0 * inf
              float4 o;
              o.x = __uint_as_float(r[4 * tp]) - tw0 * xv[tp].z;
              o.y = __uint_as_float(r[4 * tp + 1]) - tw1 * xv[tp].w;
              o.z = __uint_as_float(r[4 * tp + 2]) + tw0 * xv[tp].x;
              o.w = __uint_as_float(r[4 * tp + 3]) + tw1 * xv[tp].y;
              if (q.eps) {
                o.x -= ep0 * xv[tp].y;
                o.y -= ep1 * xv[tp].x;
                o.z -= ep0 * xv[tp].w;
                o.w -= ep1 * xv[tp].z;
              }
              o.x *= so0;
              o.y *= so1;
              o.z *= so0;
              o.w *= so1;
              *reinterpret_cast<float4*>(q.y + ((((int64_t)t * nc + i) * q.Vc) + a) * 4) = o;
            }
          }
        }
      }
  }
  cm_fence_before();
  __syncthreads();
  if (cs.fail) {
    if (tid == 0) atomicExch(q.err, 2);
    return false;
  }
  return true;
}

// host side (coarse_mma.cu)
// FP32 stencil [9][Vc][nc col][nc row] -> FP16 operator in the core-matrix layout
void pack_coarse_f16(const CoarseDims& cd, const float2* A, __half* A16, cudaStream_t st);
// y = D_c(dmu mu_n) x with the FP16 operator; mx: nsys floats of scratch, X16: cm_x16_bytes of
// scratch for the B images, err: device flag (set to 2 when a bounded wait gives up).
// Returns 0, or -2 for unsupported sizes.
int coarse_apply_f16(const CoarseDims& cd, const __half* A16, const float* x, float* y, const double* mu, double dmu,
                     int nsys, float* mx, __half* X16, int* err, cudaStream_t st, const double* eps = nullptr);
// largest dynamic shared memory a CTA of 'kernel' may use next to its static shared memory
size_t cm_dyn_cap(const void* kernel);

}  // namespace tmamg

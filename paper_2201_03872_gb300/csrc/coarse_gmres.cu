// Persistent restarted GMRES on the coarse lattice for all systems at once (one launch per
// coarse solve).
//
// The coarse-grid problem is small (V_c sites x 2 Nv unknowns) and the paper traces the loss
// of strong scaling of DDalphaAMG to this level (Sec. 3, Fig. 3 right) and most of the
// block-solver overhead to global reductions (Sec. 4). On one GPU the equivalent cost is
// kernel-launch latency: a GMRES step is a stencil application, a Gram-Schmidt pass, a norm
// and a Givens rotation per system. Here all of it runs inside one cooperative kernel; the
// phases are separated by a grid barrier whose wait is bounded (about one second), after
// which the kernel records an error and returns instead of hanging. Reductions are
// deterministic: per-CTA partial sums in FP64, then a fixed-order sum.
//
// Work decomposition.
//  * Stencil phase: independent warp tasks (coarse site, hop, chunk of system tiles); each
//    stencil entry is read once per application for all systems (paper Sec. 3, matrix data
//    loaded once for all right-hand sides); the nine hop partials are summed in a fixed
//    order by the owner threads after a grid barrier.
//  * Vector phases: CTA b works on tile b % nt and on the entries of slice b / nt; the same
//    thread owns the same entries in every vector phase, so in-place updates need no
//    barrier of their own.
//  * Small dense work (Givens rotations, back substitution) is per system, with every
//    operand fetched before the dependent arithmetic starts.
#include <atomic>
#include <cmath>

#include "amg.cuh"
#include "profile.cuh"
#include "coarse_gmres.cuh"
#include "coarse_mma.cuh"

namespace tmamg {

constexpr int CG_THREADS = 256;
constexpr int CG_TCH = 8;    // system tiles per shared-memory chunk in the stencil phase
constexpr int CG_IVEC = 4;   // basis vectors per register chunk in the dot phase
constexpr int CG_MAXM = 64;  // largest restart length
constexpr int CG_EPT = 8;    // entries per thread held in registers in the vector phases
constexpr int CG_MAXNC = 64; // largest coarse site dimension 2 Nv
constexpr int CG_AJC = 16;   // stencil columns per asynchronous chunk
// per-warp shared memory of the stencil phase, in float4 units (vector staging + 2 chunks)
constexpr int CG_WARP_F4 = CG_MAXNC * CG_TCH + CG_AJC * CG_MAXNC;

struct CGArgs {
  const float2* A;
  const __half* A16;  // FP16 operator for the tensor-core stencil, or null (FP32 stencil)
  __half* X16;        // B images of the vector the tensor-core stencil multiplies
  int cm_nstage;      // shared-memory stages of the tensor-core stencil
  double* b0;         // [NS] initial residual norm per system (scale of the restart product)
  int L[4];
  int64_t Vc;
  int nc;
  const float* rc;
  float* xc;
  float* V;
  int64_t vstride;  // floats between basis vectors
  const double* mu;
  double dmu;
  int nsys, nt;
  int64_t M;  // entries per tile
  int m, maxiter;
  double tol;
  // per-system FP64 state, [.. * NS + n]
  double2* H;  // [(j (m+1) + i)]
  double* cs;  // [j]
  double2* sn; // [j]
  double2* g;  // [i]
  double2* y;  // [i]
  double* tolabs;
  double* sc;  // scale of the newest basis vector (applied lazily)
  int* kconv;
  int* active;
  int* done;      // converged (no restart needed)
  int* nactive;   // [1]
  double2* part;  // [G][m + 2][2 lanes]
  float* hpart;   // [9][nt][nc][Vc][4] hop partials of the stencil
  unsigned* bar;  // [2]: count, generation
  int* err;
  long long wait_limit;  // clock cycles a CTA waits at a grid barrier before it gives up
  unsigned extra;        // arrivals a barrier needs beyond the grid (0; 1 makes every barrier unreachable)
  int* iters;  // [1] Arnoldi steps done
  int G, Gt;
  int NS;  // stride of the per-system arrays
};

// Grid barrier on a monotonic arrival counter (zeroed before the launch): barrier number k
// is complete once the counter reaches k G. The CTA's writes are published by bar.sync plus
// the release of thread 0's increment; the acquire load that sees the count makes every
// other CTA's writes visible to this CTA (cross-CTA data is then read through L2).
__device__ __forceinline__ bool grid_barrier(const CGArgs& p) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;\n" : "=r"(prev) : "l"(p.bar) : "memory");
    const unsigned G = (unsigned)p.G;
    const unsigned target = (prev / G + 1) * G + p.extra;
    const long long t0 = clock64();
    while (true) {
      unsigned cur;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(cur) : "l"(p.bar) : "memory");
      if ((int)(cur - target) >= 0) break;
      if (clock64() - t0 > p.wait_limit) {  // 2e9 cycles by default, about one second at 2 GHz
        atomicExch(p.err, 1);
        break;
      }
      if (*(volatile int*)p.err) break;  // another CTA gave up
    }
  }
  __syncthreads();
  return *(volatile int*)p.err == 0;
}

// loads of data written by other CTAs of this launch go through L2 (__ldcg), never a stale L1 line
__device__ __forceinline__ float4 ld4(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
template <typename T>
__device__ __forceinline__ T ldx(const T* p) {
  return __ldcg(p);
}

__device__ __forceinline__ void cfma(float4& acc, float ar, float ai, const float4& v) {
  // acc (2 lanes, re0 re1 im0 im1) += (ar + i ai) * v, as packed FP32x2 FMAs over the lanes
  float2 re = make_float2(acc.x, acc.y), im = make_float2(acc.z, acc.w);
  const float2 vre = make_float2(v.x, v.y), vim = make_float2(v.z, v.w);
  re = __ffma2_rn(make_float2(ar, ar), vre, re);
  re = __ffma2_rn(make_float2(-ai, -ai), vim, re);
  im = __ffma2_rn(make_float2(ar, ar), vim, im);
  im = __ffma2_rn(make_float2(ai, ai), vre, im);
  acc = make_float4(re.x, re.y, im.x, im.y);
}

// Stencil phase A: hop partials hpart[h][t][i][a] = sum_j A_h(a)[i][j] in[t][j][a + h].
// One warp per task (site a, hop h, chunk of CG_TCH tiles); lane l owns rows l and l + 32.
// Stencil loads are coalesced over rows; the vector loads are warp-wide broadcasts from L2;
// eight columns are in flight at a time. No CTA-wide synchronisation.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::);
}

__device__ void cg_apply_partials(const CGArgs& p, const float* in, float4* wsm) {
  const int nc = p.nc;
  const int lane = threadIdx.x & 31;
  const int nchunk = (p.nt + CG_TCH - 1) / CG_TCH;
  const int64_t ntask = (int64_t)9 * p.Vc * nchunk;
  const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)p.G * (blockDim.x >> 5);
  // this warp's shared memory: vector staging [CG_MAXNC][CG_TCH] float4, then two buffers of
  // CG_AJC stencil columns [CG_AJC][nc] float2, filled by asynchronous 16-byte copies so that
  // the next chunk is in flight while the current one is used
  float4* xw = wsm + (threadIdx.x >> 5) * CG_WARP_F4;
  float2* abuf[2] = {reinterpret_cast<float2*>(xw + CG_MAXNC * CG_TCH),
                     reinterpret_cast<float2*>(xw + CG_MAXNC * CG_TCH) + CG_AJC * CG_MAXNC};
  const bool r1 = lane + 32 < nc;
  const int nj = (nc + CG_AJC - 1) / CG_AJC;
  for (int64_t task = wid; task < ntask; task += nw) {
    const int ch = (int)(task % nchunk);
    const int64_t ha = task / nchunk;
    const int h = (int)(ha % 9);
    const int64_t a = ha / 9;
    const int t0 = ch * CG_TCH;
    const int ntc = p.nt - t0 < CG_TCH ? p.nt - t0 : CG_TCH;
    int64_t nb = a;
    if (h > 0) {
      const int L0 = p.L[0], L1 = p.L[1], L2 = p.L[2], L3 = p.L[3];
      int c0 = (int)(a % L0);
      int64_t rr = a / L0;
      int c1 = (int)(rr % L1);
      rr /= L1;
      int c2 = (int)(rr % L2);
      int c3 = (int)(rr / L2);
      const int nu = (h - 1) / 2, dir = ((h - 1) & 1) ? -1 : 1;
      if (nu == 0) c0 = (c0 + dir + L0) % L0;
      else if (nu == 1) c1 = (c1 + dir + L1) % L1;
      else if (nu == 2) c2 = (c2 + dir + L2) % L2;
      else c3 = (c3 + dir + L3) % L3;
      nb = ((int64_t)(c3 * L2 + c2) * L1 + c1) * L0 + c0;
    }
    const float2* Ab = p.A + ((int64_t)h * p.Vc + a) * nc * nc;  // column-major block
    __syncwarp();  // the previous task's buffers are free
    // group 0: vector entries and stencil chunk 0; group 1: stencil chunk 1
    for (int q = lane; q < nc * ntc; q += 32) {
      const int j = q / ntc, u = q - j * ntc;
      cp_async16(xw + j * CG_TCH + u, in + ((((int64_t)(t0 + u) * nc + j) * p.Vc) + nb) * 4);
    }
    {
      const int jn0 = nc < CG_AJC ? nc : CG_AJC;
      for (int q = lane; q < jn0 * nc / 2; q += 32) cp_async16(abuf[0] + 2 * q, Ab + 2 * q);
      asm volatile("cp.async.commit_group;\n" ::);
    }
    if (nj > 1) {
      const int jn1 = nc - CG_AJC < CG_AJC ? nc - CG_AJC : CG_AJC;
      for (int q = lane; q < jn1 * nc / 2; q += 32) cp_async16(abuf[1] + 2 * q, Ab + (int64_t)CG_AJC * nc + 2 * q);
    }
    asm volatile("cp.async.commit_group;\n" ::);
    float4 acc0[CG_TCH], acc1[CG_TCH];
#pragma unroll
    for (int u = 0; u < CG_TCH; ++u) {
      acc0[u] = make_float4(0, 0, 0, 0);
      acc1[u] = make_float4(0, 0, 0, 0);
    }
    for (int c = 0; c < nj; ++c) {
      const int j0 = c * CG_AJC;
      const int jn = nc - j0 < CG_AJC ? nc - j0 : CG_AJC;
      asm volatile("cp.async.wait_group 1;\n" ::);  // chunk c has landed (one group may still fly)
      __syncwarp();
      const float2* aw = abuf[c & 1];
      for (int jj = 0; jj < jn; ++jj) {
        const float2 m0 = lane < nc ? aw[jj * nc + lane] : make_float2(0, 0);
        const float2 m1 = r1 ? aw[jj * nc + lane + 32] : make_float2(0, 0);
        const int j = j0 + jj;
#pragma unroll
        for (int u = 0; u < CG_TCH; ++u) {
          if (u < ntc) {
            const float4 v = xw[j * CG_TCH + u];
            cfma(acc0[u], m0.x, m0.y, v);
            cfma(acc1[u], m1.x, m1.y, v);
          }
        }
      }
      __syncwarp();  // buffer c & 1 is consumed: refill it with chunk c + 2
      if (c + 2 < nj) {
        const int j2 = (c + 2) * CG_AJC;
        const int jn2 = nc - j2 < CG_AJC ? nc - j2 : CG_AJC;
        for (int q = lane; q < jn2 * nc / 2; q += 32)
          cp_async16(abuf[c & 1] + 2 * q, Ab + (int64_t)j2 * nc + 2 * q);
      }
      asm volatile("cp.async.commit_group;\n" ::);
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
#pragma unroll
    for (int u = 0; u < CG_TCH; ++u) {
      if (u < ntc) {
        const int t = t0 + u;
        if (lane < nc) st4(p.hpart + ((((int64_t)h * p.nt + t) * nc + lane) * p.Vc + a) * 4, acc0[u]);
        if (r1) st4(p.hpart + ((((int64_t)h * p.nt + t) * nc + lane + 32) * p.Vc + a) * 4, acc1[u]);
      }
    }
  }
}

// Stencil phase B (owner entries): out = sc_n (sum_h hpart[h] + i dmu mu_n gamma5_c in)
__device__ void cg_apply_sum(const CGArgs& p, const float* in, float* out, int tile, int64_t e0, int64_t estep) {
  const int nc = p.nc;
  const int n0 = 2 * tile, n1 = 2 * tile + 1;
  float m0 = 0, m1 = 0, s0 = 0, s1 = 0;
  if (n0 < p.nsys) { m0 = (float)(p.dmu * p.mu[n0]); s0 = (float)ldx(p.sc + n0); }
  if (n1 < p.nsys) { m1 = (float)(p.dmu * p.mu[n1]); s1 = (float)ldx(p.sc + n1); }
  const int64_t toff = (int64_t)tile * p.M * 4;
  const int64_t hstride = (int64_t)p.nt * p.M * 4;
  for (int64_t e = e0; e < p.M; e += estep) {
    float4 hv[9];
#pragma unroll
    for (int h = 0; h < 9; ++h) hv[h] = ld4(p.hpart + h * hstride + toff + e * 4);
    const float4 xv = ld4(in + toff + e * 4);
    float4 s = hv[0];
#pragma unroll
    for (int h = 1; h < 9; ++h) {
      s.x += hv[h].x; s.y += hv[h].y; s.z += hv[h].z; s.w += hv[h].w;
    }
    const int i = (int)(e / p.Vc);
    const float g5 = i < nc / 2 ? 1.f : -1.f;
    float4 o;
    o.x = s0 * (s.x - g5 * m0 * xv.z);
    o.y = s1 * (s.y - g5 * m1 * xv.w);
    o.z = s0 * (s.z + g5 * m0 * xv.x);
    o.w = s1 * (s.w + g5 * m1 * xv.y);
    st4(out + toff + e * 4, o);
  }
}

// CTA-wide sum of nv float4 values per thread into FP64 partials part[b][slot0 + v][lane]
__device__ void cta_reduce_store(const CGArgs& p, float4* vals, int nv, int slot0, double* sm) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int v = 0; v < nv; ++v) {
    float4 x = vals[v];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x.x += __shfl_xor_sync(0xffffffffu, x.x, o);
      x.y += __shfl_xor_sync(0xffffffffu, x.y, o);
      x.z += __shfl_xor_sync(0xffffffffu, x.z, o);
      x.w += __shfl_xor_sync(0xffffffffu, x.w, o);
    }
    if (lane == 0) {
      double* s = sm + (warp * CG_IVEC + v) * 4;
      s[0] = x.x; s[1] = x.y; s[2] = x.z; s[3] = x.w;
    }
  }
  __syncthreads();
  if (threadIdx.x < nv * 4) {
    const int v = threadIdx.x / 4, q = threadIdx.x % 4;
    double s = 0;
    for (int w = 0; w < CG_THREADS / 32; ++w) s += sm[(w * CG_IVEC + v) * 4 + q];
    // q: 0 = re lane 0, 1 = re lane 1, 2 = im lane 0, 3 = im lane 1; stored as (re, im) per lane
    double* dst = reinterpret_cast<double*>(p.part + ((int64_t)blockIdx.x * (p.m + 2) + slot0 + v) * 2);
    const int ln = q & 1, ri = q >> 1;
    dst[ln * 2 + ri] = s;
  }
  __syncthreads();
}

// sum of the partials of slot i for system n over the slices of its tile (fixed order;
// loads issued eight at a time)
__device__ double2 part_sum(const CGArgs& p, int i, int n) {
  const int t = n / 2, ln = n % 2;
  double2 s = make_double2(0, 0);
  for (int sl0 = 0; sl0 < p.Gt; sl0 += 32) {
    double2 v[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const int sl = sl0 + k;
      v[k] = sl < p.Gt ? ldx(p.part + ((int64_t)(sl * p.nt + t) * (p.m + 2) + i) * 2 + ln) : make_double2(0, 0);
    }
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      s.x += v[k].x;
      s.y += v[k].y;
    }
  }
  return s;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 conjd(double2 a) { return make_double2(a.x, -a.y); }

// Givens step for system n on Arnoldi column j, with H[j+1][j] = hn. The rotations of the
// cycle stay in the calling thread's own arrays c_, s_ (the same thread handles system n at
// every step), so only the new column is fetched. total: Arnoldi steps done before step j.
__device__ void givens_step(const CGArgs& p, int n, int j, double hn, int total, double* c_, double2* s_) {
  const int NS = p.NS, m = p.m;
  double2* col = p.H + (int64_t)j * (m + 1) * NS;
  double2 cv[CG_MAXM + 1];
  // the column fetched sixteen entries at a time into registers before it is parked in local memory
  for (int i0 = 0; i0 <= j; i0 += 16) {
    double2 t[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) t[k] = i0 + k <= j ? ldx(col + (i0 + k) * NS + n) : make_double2(0, 0);
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (i0 + k <= j) cv[i0 + k] = t[k];
  }
  cv[j + 1] = make_double2(hn, 0);
  for (int i = 0; i < j; ++i) {
    const double2 a = cv[i], bb = cv[i + 1];
    const double2 t = cmul(s_[i], bb);
    cv[i] = make_double2(c_[i] * a.x + t.x, c_[i] * a.y + t.y);
    const double2 u = cmul(conjd(s_[i]), a);
    cv[i + 1] = make_double2(c_[i] * bb.x - u.x, c_[i] * bb.y - u.y);
  }
  const double2 a = cv[j];
  const double na = hypot(a.x, a.y), nb = hn;
  const double r = hypot(na, nb);
  double c;
  double2 sn;
  if (r == 0.0) {
    c = 1.0;
    sn = make_double2(0, 0);
  } else if (na == 0.0) {
    c = 0.0;
    sn = make_double2(1, 0);
  } else {
    c = na / r;  // s = (a / |a|) conj(b) / r with b = hn real
    sn = make_double2(a.x / na * (nb / r), a.y / na * (nb / r));
  }
  cv[j] = na == 0.0 ? make_double2(r, 0) : make_double2(a.x / na * r, a.y / na * r);
  cv[j + 1] = make_double2(0, 0);
  for (int i = 0; i <= j + 1; ++i) col[i * NS + n] = cv[i];
  c_[j] = c;
  s_[j] = sn;
  const double2 gj = p.g[j * NS + n];
  const double2 t = cmul(conjd(sn), gj);
  p.g[(j + 1) * NS + n] = make_double2(-t.x, -t.y);
  p.g[j * NS + n] = make_double2(c * gj.x, c * gj.y);
  const double res = hypot(t.x, t.y);
  if (!(res > p.tolabs[n]) || nb == 0.0) {
    p.kconv[n] = j + 1;
    p.active[n] = 0;
    p.done[n] = 1;
  } else if (j + 1 == m || total + 1 >= p.maxiter) {
    p.kconv[n] = j + 1;
    p.active[n] = 0;
  }
}

// The rotations of column j for every active system, by threads n < nsys of CTA 0 (the same
// thread per system at every step; H[j+1][j] was stored by the norm phase of step j).
__device__ __forceinline__ void givens_column(const CGArgs& p, int j, int total, double* gc, double2* gs) {
  const int n = threadIdx.x;
  if (n < p.nsys && ldx(p.active + n)) {
    const double hn = ldx(p.H + ((int64_t)j * (p.m + 1) + j + 1) * p.NS + n).x;
    givens_step(p, n, j, hn, total, gc, gs);
  }
}

// y = R^{-1} g for system n: the CTA stages R in shared memory, warp 0 substitutes
__device__ void backsub(const CGArgs& p, int n, double2* Rs) {
  const int NS = p.NS, m = p.m;
  const int k = ldx(p.kconv + n);
  for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
    const int i = q % k, l = q / k;  // row i, column l
    Rs[l * k + i] = i <= l ? ldx(p.H + ((int64_t)l * (m + 1) + i) * NS + n) : make_double2(0, 0);
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    double2 s0 = lane < k ? ldx(p.g + lane * NS + n) : make_double2(0, 0);
    double2 s1 = lane + 32 < k ? ldx(p.g + (lane + 32) * NS + n) : make_double2(0, 0);
    for (int i = m - 1; i >= k; --i)
      if (lane == 0) p.y[i * NS + n] = make_double2(0, 0);
    for (int i = k - 1; i >= 0; --i) {
      const double2 si = i < 32 ? make_double2(__shfl_sync(0xffffffffu, s0.x, i), __shfl_sync(0xffffffffu, s0.y, i))
                                : make_double2(__shfl_sync(0xffffffffu, s1.x, i - 32),
                                               __shfl_sync(0xffffffffu, s1.y, i - 32));
      const double2 d = Rs[i * k + i];
      const double den = d.x * d.x + d.y * d.y;
      const double2 yi = den > 0 ? make_double2((si.x * d.x + si.y * d.y) / den, (si.y * d.x - si.x * d.y) / den)
                                 : make_double2(0, 0);
      if (lane == 0) p.y[i * NS + n] = yi;
      if (lane < i) {
        const double2 t = cmul(Rs[i * k + lane], yi);
        s0.x -= t.x;
        s0.y -= t.y;
      }
      if (lane + 32 < i) {
        const double2 t = cmul(Rs[i * k + lane + 32], yi);
        s1.x -= t.x;
        s1.y -= t.y;
      }
    }
  }
  __syncthreads();
}

// tensor-core stencil phase: y = s_out D_c (s_in x) over all sites
__device__ __forceinline__ bool cg_apply_tc(const CGArgs& p, CmShared& cs, unsigned char* dsm, CmPipe& pipe,
                                            const float* x, float* y, const double* scale, int mode, int cta,
                                            int ncta) {
  CmArgs q;
  q.A16 = p.A16;
  q.X16 = p.X16;
  q.L[0] = p.L[0]; q.L[1] = p.L[1]; q.L[2] = p.L[2]; q.L[3] = p.L[3];
  q.Vc = p.Vc;
  q.nc = p.nc;
  q.x = x;
  q.y = y;
  q.mu = p.mu;
  q.dmu = p.dmu;
  q.scale = scale;
  q.mode = mode;
  q.nsys = p.nsys;
  q.nstage = p.cm_nstage;
  q.err = p.err;
  q.eps = nullptr;  // the persistent solver runs degenerate systems only
  return cm_apply(q, cs, dsm, pipe, cta, ncta);
}

// B images of x for the tensor-core stencil, input factor cvs[n] per system (shared memory);
// all CTAs take part, the caller's next grid barrier publishes them
__device__ __forceinline__ void cg_convert(const CGArgs& p, const float* x, const float* cvs) {
  cm_convert(x, p.X16, p.Vc, p.nc, p.nsys, cvs, (int64_t)blockIdx.x * CG_THREADS + threadIdx.x,
             (int64_t)p.G * CG_THREADS);
  cm_fence_global_async();
}

__device__ __forceinline__ void cg_body(const CGArgs& p, CmShared& cs, float4* dyn) {
  __shared__ double sm[(CG_THREADS / 32) * CG_IVEC * 4];
  __shared__ float4 hsm[CG_MAXM + 1];  // H column (or y) of this CTA's two systems
  CmPipe pipe;  // this thread's place in the tensor-core stencil pipeline
  __shared__ float cvs[256];  // input factors of the B-image conversion, per system
  double gc[CG_MAXM];   // Givens rotations of the current cycle (used by the threads gtid < nsys)
  double2 gs[CG_MAXM];
  unsigned char* dsm = reinterpret_cast<unsigned char*>(dyn);
  const int b = blockIdx.x;
  const int tile = b % p.nt;
  const int slice = b / p.nt;
  const int64_t toff = (int64_t)tile * p.M * 4;
  const int64_t e0 = (int64_t)slice * CG_THREADS + threadIdx.x;
  const int64_t estep = (int64_t)p.Gt * CG_THREADS;
  const int NS = p.NS;
  const int gtid = b * CG_THREADS + threadIdx.x;
  const int m = p.m;
  const int n0 = 2 * tile, n1 = 2 * tile + 1;
  const int GG = p.G > 1 ? 1 : 0;  // CTAs kept free of stencil sites for the Givens rotations

  // ---- start: x = 0, V0 = rc, |rc| per system
  {
    float4 nrm = make_float4(0, 0, 0, 0);
    for (int64_t e = e0; e < p.M; e += estep) {
      const float4 r = ld4(p.rc + toff + e * 4);
      st4(p.V + toff + e * 4, r);
      st4(p.xc + toff + e * 4, make_float4(0, 0, 0, 0));
      nrm.x += r.x * r.x + r.z * r.z;
      nrm.y += r.y * r.y + r.w * r.w;
    }
    cta_reduce_store(p, &nrm, 1, 0, sm);
  }
  if (!grid_barrier(p)) return;
  // norms sit in the real slot of each lane's partial (see cta_reduce_store)
  if (gtid < p.nsys) {
    const int n = gtid;
    const double2 s = part_sum(p, 0, n);
    const double beta = sqrt(fmax(s.x, 0.0));
    p.tolabs[n] = p.tol * beta;
    const bool on = beta > 0.0 && isfinite(beta);
    p.b0[n] = on ? beta : 0.0;
    p.active[n] = on;
    p.done[n] = !on;
    p.sc[n] = on ? 1.0 / beta : 0.0;
    for (int i = 0; i <= m; ++i) p.g[i * NS + n] = make_double2(0, 0);
    p.g[n] = make_double2(on ? beta : 0.0, 0);
    p.kconv[n] = 0;
  }
  if (!grid_barrier(p)) return;
  if (p.A16) {
    for (int n = threadIdx.x; n < p.nsys; n += CG_THREADS) cvs[n] = (float)ldx(p.sc + n);
    __syncthreads();
    cg_convert(p, p.V, cvs);
    if (!grid_barrier(p)) return;
  }

  int total = 0;
  while (true) {
    int j = 0;
    for (; j < m && total < p.maxiter; ++j) {
      // P1: V_{j+1} = sc * A V_j   (V_j not yet scaled in place). The Givens rotations of the
      // previous column run at the same time on CTA 0, which (on the tensor-core path) takes no
      // stencil sites: the stop test lags the Arnoldi process by one step, and the solution
      // uses the converged column count, so the extra step changes nothing in it.
      if (p.A16) {
        if (b >= GG && !cg_apply_tc(p, cs, dsm, pipe, p.V + (int64_t)j * p.vstride,
                                    p.V + (int64_t)(j + 1) * p.vstride, p.sc, CM_SCALE_IN, b - GG, p.G - GG))
          return;
      } else {
        cg_apply_partials(p, p.V + (int64_t)j * p.vstride, dyn);
      }
      if (j > 0 && b == 0) givens_column(p, j - 1, total - 1, gc, gs);
      if (!grid_barrier(p)) return;
      if (!p.A16)
        cg_apply_sum(p, p.V + (int64_t)j * p.vstride, p.V + (int64_t)(j + 1) * p.vstride, tile, e0, estep);
      // (P2 below touches only this thread's entries of V_j and V_{j+1}: no barrier needed)
      // P2: scale V_j in place (owner entries), then dots <V_i, w> for i <= j
      {
        float s0 = 0, s1 = 0;
        if (n0 < p.nsys) s0 = (float)ldx(p.sc + n0);
        if (n1 < p.nsys) s1 = (float)ldx(p.sc + n1);
        float* vj = p.V + (int64_t)j * p.vstride + toff;
        for (int64_t e = e0; e < p.M; e += estep) {
          float4 v = ld4(vj + e * 4);
          v.x *= s0; v.y *= s1; v.z *= s0; v.w *= s1;
          st4(vj + e * 4, v);
        }
        const float* w = p.V + (int64_t)(j + 1) * p.vstride + toff;
        for (int i0 = 0; i0 <= j; i0 += CG_IVEC) {
          const int ni = j + 1 - i0 < CG_IVEC ? j + 1 - i0 : CG_IVEC;
          float4 acc[CG_IVEC];
#pragma unroll
          for (int u = 0; u < CG_IVEC; ++u) acc[u] = make_float4(0, 0, 0, 0);
          for (int64_t eb = e0; eb < p.M; eb += CG_EPT * estep) {
            float4 ww[CG_EPT];
#pragma unroll
            for (int q = 0; q < CG_EPT; ++q) {
              const int64_t e = eb + q * estep;
              ww[q] = e < p.M ? ld4(w + e * 4) : make_float4(0, 0, 0, 0);
            }
#pragma unroll
            for (int u = 0; u < CG_IVEC; ++u) {
              if (u < ni) {
                const float* vu = p.V + (int64_t)(i0 + u) * p.vstride + toff;
#pragma unroll
                for (int q = 0; q < CG_EPT; ++q) {
                  const int64_t e = eb + q * estep;
                  if (e < p.M) {
                    const float4 v = ld4(vu + e * 4);
                    // conj(v) w per lane
                    acc[u].x += v.x * ww[q].x + v.z * ww[q].z;
                    acc[u].y += v.y * ww[q].y + v.w * ww[q].w;
                    acc[u].z += v.x * ww[q].z - v.z * ww[q].x;
                    acc[u].w += v.y * ww[q].w - v.w * ww[q].y;
                  }
                }
              }
            }
          }
          cta_reduce_store(p, acc, ni, i0, sm);
        }
      }
      if (!grid_barrier(p)) return;
      // P3 + P4: every CTA sums the H column of its tile's two systems from the partials
      // (the same fixed order everywhere; slice 0 stores it for P5), then
      // w -= sum_i H[i][j] V_i (owner entries) and |w|^2 partials
      {
        double* hd = reinterpret_cast<double*>(sm);  // [j + 1][2 lanes] (re, im)
        if (threadIdx.x < 2 * (j + 1)) {
          const int i = threadIdx.x >> 1, ln = threadIdx.x & 1;
          const int n = 2 * tile + ln;
          const double2 h = n < p.nsys ? part_sum(p, i, n) : make_double2(0, 0);
          if (slice == 0 && n < p.nsys) p.H[((int64_t)j * (m + 1) + i) * NS + n] = h;
          hd[(i * 2 + ln) * 2] = h.x;
          hd[(i * 2 + ln) * 2 + 1] = h.y;
        }
        __syncthreads();
        if (threadIdx.x <= j) {
          const int i = threadIdx.x;
          hsm[i] = make_float4((float)hd[i * 4], (float)hd[i * 4 + 1], (float)hd[i * 4 + 2], (float)hd[i * 4 + 3]);
        }
        __syncthreads();
        float* w = p.V + (int64_t)(j + 1) * p.vstride + toff;
        float4 nrm = make_float4(0, 0, 0, 0);
        for (int64_t eb = e0; eb < p.M; eb += CG_EPT * estep) {
          float4 ww[CG_EPT];
#pragma unroll
          for (int q = 0; q < CG_EPT; ++q) {
            const int64_t e = eb + q * estep;
            ww[q] = e < p.M ? ld4(w + e * 4) : make_float4(0, 0, 0, 0);
          }
          for (int i0 = 0; i0 <= j; i0 += CG_IVEC) {
#pragma unroll
            for (int u = 0; u < CG_IVEC; ++u) {
              if (i0 + u <= j) {
                const float4 h = hsm[i0 + u];
                const float* vu = p.V + (int64_t)(i0 + u) * p.vstride + toff;
#pragma unroll
                for (int q = 0; q < CG_EPT; ++q) {
                  const int64_t e = eb + q * estep;
                  if (e < p.M) {
                    const float4 v = ld4(vu + e * 4);
                    ww[q].x -= h.x * v.x - h.y * v.z;
                    ww[q].z -= h.x * v.z + h.y * v.x;
                    ww[q].y -= h.z * v.y - h.w * v.w;
                    ww[q].w -= h.z * v.w + h.w * v.y;
                  }
                }
              }
            }
          }
#pragma unroll
          for (int q = 0; q < CG_EPT; ++q) {
            const int64_t e = eb + q * estep;
            if (e < p.M) {
              st4(w + e * 4, ww[q]);
              nrm.x += ww[q].x * ww[q].x + ww[q].z * ww[q].z;
              nrm.y += ww[q].y * ww[q].y + ww[q].w * ww[q].w;
            }
          }
        }
        cta_reduce_store(p, &nrm, 1, m + 1, sm);
      }
      if (!grid_barrier(p)) return;
      // P5: H[j+1][j] = |w| and sc = 1 / |w| (every CTA sums the norms in the same order; CTA 0
      // stores them), then the B images of sc w for the next stencil
      for (int n = threadIdx.x; n < p.nsys; n += CG_THREADS) {
        const double2 s = part_sum(p, m + 1, n);
        const double hn = sqrt(fmax(s.x, 0.0));
        const double scn = hn > 0 ? 1.0 / hn : 0.0;
        cvs[n] = (float)scn;
        if (b == 0) {
          p.sc[n] = scn;
          p.H[((int64_t)j * (m + 1) + j + 1) * NS + n] = make_double2(hn, 0);
        }
      }
      if (p.A16) {
        __syncthreads();
        cg_convert(p, p.V + (int64_t)(j + 1) * p.vstride, cvs);
      }
      ++total;
      if (!grid_barrier(p)) return;
      {
        // active systems left (warp 0 of every CTA counts; the flags were last written
        // before the barrier)
        __shared__ int nact;
        if (threadIdx.x < 32) {
          int c = 0;
          for (int n = threadIdx.x; n < p.nsys; n += 32) c += ldx(p.active + n);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
          if (threadIdx.x == 0) nact = c;
        }
        __syncthreads();
        if (nact == 0) {
          ++j;
          break;
        }
      }
    }
    // rotations of the cycle's last column (the loop ended on the cycle length or the step
    // budget; systems that converged earlier are inactive already)
    if (j > 0 && b == 0) givens_column(p, j - 1, total - 1, gc, gs);
    if (!grid_barrier(p)) return;
    // y = R^{-1} g per system (a CTA per system), then x += sum_i y_i V_i
    for (int n = b; n < p.nsys; n += p.G) backsub(p, n, reinterpret_cast<double2*>(dyn));
    if (!grid_barrier(p)) return;
    {
      if (threadIdx.x < j) {
        const int i = threadIdx.x;
        const double2 y0 = n0 < p.nsys ? ldx(p.y + i * NS + n0) : make_double2(0, 0);
        const double2 y1 = n1 < p.nsys ? ldx(p.y + i * NS + n1) : make_double2(0, 0);
        hsm[i] = make_float4((float)y0.x, (float)y0.y, (float)y1.x, (float)y1.y);
      }
      __syncthreads();
      float* x = p.xc + toff;
      for (int64_t eb = e0; eb < p.M; eb += CG_EPT * estep) {
        float4 xx[CG_EPT];
#pragma unroll
        for (int q = 0; q < CG_EPT; ++q) {
          const int64_t e = eb + q * estep;
          xx[q] = e < p.M ? ld4(x + e * 4) : make_float4(0, 0, 0, 0);
        }
        for (int i0 = 0; i0 < j; i0 += CG_IVEC) {
#pragma unroll
          for (int u = 0; u < CG_IVEC; ++u) {
            if (i0 + u < j) {
              const float4 yv = hsm[i0 + u];
              const float* vu = p.V + (int64_t)(i0 + u) * p.vstride + toff;
#pragma unroll
              for (int q = 0; q < CG_EPT; ++q) {
                const int64_t e = eb + q * estep;
                if (e < p.M) {
                  const float4 v = ld4(vu + e * 4);
                  xx[q].x += yv.x * v.x - yv.y * v.z;
                  xx[q].z += yv.x * v.z + yv.y * v.x;
                  xx[q].y += yv.z * v.y - yv.w * v.w;
                  xx[q].w += yv.z * v.w + yv.w * v.y;
                }
              }
            }
          }
        }
#pragma unroll
        for (int q = 0; q < CG_EPT; ++q) {
          const int64_t e = eb + q * estep;
          if (e < p.M) st4(x + e * 4, xx[q]);
        }
      }
    }
    // restart decision (uniform: done[] was last written before a grid barrier)
    bool again;
    {
      int alldone = 1;
      for (int n = 0; n < p.nsys; ++n) alldone &= ldx(p.done + n);
      again = !alldone && total < p.maxiter;
    }
    if (!again) break;
    if (!grid_barrier(p)) return;
    // restart: V0 = rc - A x, with sc = 1 for the apply
    if (gtid < p.nsys) p.sc[gtid] = 1.0;
    if (!grid_barrier(p)) return;
    if (p.A16) {
      for (int n = threadIdx.x; n < p.nsys; n += CG_THREADS) {
        const double v = ldx(p.b0 + n);
        cvs[n] = v > 0.0 ? (float)(1.0 / v) : 1.f;
      }
      __syncthreads();
      cg_convert(p, p.xc, cvs);
      if (!grid_barrier(p)) return;
      if (!cg_apply_tc(p, cs, dsm, pipe, p.xc, p.V, p.b0, CM_SCALE_OUT, b, p.G)) return;
    } else {
      cg_apply_partials(p, p.xc, dyn);
    }
    if (!grid_barrier(p)) return;
    if (!p.A16) cg_apply_sum(p, p.xc, p.V, tile, e0, estep);
    {
      float4 nrm = make_float4(0, 0, 0, 0);
      for (int64_t e = e0; e < p.M; e += estep) {
        const float4 r = ld4(p.rc + toff + e * 4);
        float4 w = ld4(p.V + toff + e * 4);
        w.x = r.x - w.x; w.y = r.y - w.y; w.z = r.z - w.z; w.w = r.w - w.w;
        st4(p.V + toff + e * 4, w);
        nrm.x += w.x * w.x + w.z * w.z;
        nrm.y += w.y * w.y + w.w * w.w;
      }
      cta_reduce_store(p, &nrm, 1, 0, sm);
    }
    if (!grid_barrier(p)) return;
    if (gtid < p.nsys) {
      const int n = gtid;
      const double2 s = part_sum(p, 0, n);
      const double beta = sqrt(fmax(s.x, 0.0));
      const bool on = !p.done[n] && beta > p.tolabs[n];
      if (!on) p.done[n] = 1;
      p.active[n] = on;
      p.sc[n] = on ? 1.0 / beta : 0.0;
      for (int i = 0; i <= m; ++i) p.g[i * NS + n] = make_double2(0, 0);
      p.g[n] = make_double2(on ? beta : 0.0, 0);
      p.kconv[n] = 0;
    }
    if (!grid_barrier(p)) return;
    if (p.A16) {
      // B images of the new V0 for the first product of the cycle (the last images were of x)
      for (int n = threadIdx.x; n < p.nsys; n += CG_THREADS) cvs[n] = (float)ldx(p.sc + n);
      __syncthreads();
      cg_convert(p, p.V, cvs);
      if (!grid_barrier(p)) return;
    }
  }
  if (gtid == 0) *p.iters = total;
}

__global__ void __launch_bounds__(CG_THREADS, 1) coarse_gmres_kernel(CGArgs p) {
  __shared__ CmShared cs;
  extern __shared__ __align__(128) float4 dyn[];
  if (p.A16) cm_begin(cs);
  cg_body(p, cs, dyn);
  if (p.A16) cm_end(cs);
}

int CoarseGmres::alloc(int m_, int nsys_, int G_, size_t bundle_bytes, size_t x16b) {
  if (m_ <= m && nsys_ <= NS && G_ <= G && bundle_bytes <= hbytes && x16b <= x16_bytes) return 0;
  release();
  m = m_;
  NS = nsys_;
  G = G_;
  hbytes = bundle_bytes;
  x16_bytes = x16b;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** q, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(q, bytes);
  };
  A((void**)&H, sizeof(double2) * (size_t)(m + 1) * m * NS);
  A((void**)&cs, sizeof(double) * (size_t)m * NS);
  A((void**)&sn, sizeof(double2) * (size_t)m * NS);
  A((void**)&g, sizeof(double2) * (size_t)(m + 1) * NS);
  A((void**)&y, sizeof(double2) * (size_t)m * NS);
  A((void**)&tolabs, sizeof(double) * NS);
  A((void**)&b0, sizeof(double) * NS);
  A((void**)&sc, sizeof(double) * NS);
  A((void**)&kconv, sizeof(int) * NS);
  A((void**)&active, sizeof(int) * NS);
  A((void**)&done, sizeof(int) * NS);
  A((void**)&nactive, sizeof(int));
  A((void**)&part, sizeof(double2) * (size_t)G * (m + 2) * 2);
  A((void**)&bar, sizeof(unsigned) * 2);
  A((void**)&err, sizeof(int));
  A((void**)&iters, sizeof(int));
  A((void**)&hpart, 9 * bundle_bytes);
  if (x16_bytes) A((void**)&X16, x16_bytes);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&h_flags, sizeof(int) * 2);
  return e == cudaSuccess ? 0 : -1;
}

void CoarseGmres::release() {
  void* ptrs[] = {H, cs, sn, g, y, tolabs, b0, sc, kconv, active, done, nactive, part, bar, err, iters, hpart, X16};
  for (void* q : ptrs) cudaFree(q);
  if (h_flags) cudaFreeHost(h_flags);
  H = nullptr; cs = nullptr; sn = nullptr; g = nullptr; y = nullptr; tolabs = nullptr; b0 = nullptr; sc = nullptr;
  kconv = nullptr; active = nullptr; done = nullptr; nactive = nullptr; part = nullptr; bar = nullptr;
  err = nullptr; iters = nullptr; h_flags = nullptr; hpart = nullptr; X16 = nullptr;
  m = 0; NS = 0; G = 0; hbytes = 0; x16_bytes = 0;
}

// dynamic shared memory: back substitution, and the stencil phase (FP32 per-warp staging, or
// the tensor-core operand buffers with nbuf operator copies)
static size_t dyn_smem_bytes(int m, int nc, int nsys, bool tc, int nstage) {
  const size_t rs = sizeof(double2) * (size_t)m * m;
  const size_t stage = tc ? cm_smem_bytes(nc, nsys, nstage) : sizeof(float4) * (size_t)(CG_THREADS / 32) * CG_WARP_F4;
  return stage > rs ? stage : rs;
}

static size_t dyn_smem_cap() {
  const size_t cap = cm_dyn_cap((const void*)coarse_gmres_kernel);
  func_smem_optin((const void*)coarse_gmres_kernel, (int)cap);
  return cap;
}

int coarse_gmres_grid(int nt) {
  const int sms = device_sms();
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coarse_gmres_kernel, CG_THREADS, dyn_smem_cap());
  if (per_sm < 1) per_sm = 1;
  int want = sms;  // one CTA per SM keeps the barrier short
  if (want > per_sm * sms) want = per_sm * sms;
  int Gt = want / nt;
  if (Gt < 1) Gt = 1;
  return Gt * nt;
}

// bound of the grid-barrier waits, and a one-shot request that the next launch's barriers be
// unreachable (process-wide; set by tmamg_debug_bounded_wait for the tests of the timeout path)
static std::atomic<long long> g_wait_limit{2000000000LL};
static std::atomic<int> g_unreachable_next{0};

void coarse_gmres_debug_wait(long long limit_cycles, int unreachable_next) {
  g_wait_limit.store(limit_cycles > 0 ? limit_cycles : 2000000000LL);
  g_unreachable_next.store(unreachable_next ? 1 : 0);
}

int coarse_gmres_solve(CoarseGmres& s, const CoarseDims& cd, const float2* A, const __half* A16, const float* rc,
                       float* xc, float* V, int64_t vstride, const double* mu, double dmu, int nsys, int m,
                       int maxiter, double tol, int* iters_done, cudaStream_t st) {
  const int nt = ntiles(nsys, 2);
  const int G = coarse_gmres_grid(nt);
  const size_t need = (size_t)nt * cd.nc * cd.Vc * 4 * sizeof(float);
  if (G > s.G || m > s.m || nsys > s.NS || m > CG_MAXM || cd.nc > 64 || (cd.nc % 2) || need > s.hbytes) return -2;
  const size_t cap = dyn_smem_cap();
  const int nstage = A16 ? cm_nstage(cd.nc, nsys, cap) : 0;
  if (A16 && (nstage < 2 || cm_x16_bytes(cd.Vc, cd.nc, nsys) > s.x16_bytes)) return -2;
  const size_t dyn = dyn_smem_bytes(m, cd.nc, nsys, A16 != nullptr, nstage);
  if (dyn > cap) return -2;
  CGArgs p;
  p.A = A;
  p.A16 = A16;
  p.X16 = s.X16;
  p.cm_nstage = nstage;
  p.b0 = s.b0;
  for (int k = 0; k < 4; ++k) p.L[k] = cd.L[k];
  p.Vc = cd.Vc;
  p.nc = cd.nc;
  p.rc = rc;
  p.xc = xc;
  p.V = V;
  p.vstride = vstride;
  p.mu = mu;
  p.dmu = dmu;
  p.nsys = nsys;
  p.nt = nt;
  p.M = (int64_t)cd.nc * cd.Vc;
  p.m = m;
  p.maxiter = maxiter;
  p.tol = tol;
  p.H = s.H; p.cs = s.cs; p.sn = s.sn; p.g = s.g; p.y = s.y; p.tolabs = s.tolabs; p.sc = s.sc;
  p.kconv = s.kconv; p.active = s.active; p.done = s.done; p.nactive = s.nactive; p.part = s.part;
  p.bar = s.bar; p.err = s.err; p.iters = s.iters; p.hpart = s.hpart;
  p.wait_limit = g_wait_limit.load();
  p.extra = (unsigned)g_unreachable_next.exchange(0);
  p.G = G;
  p.Gt = G / nt;
  p.NS = s.NS;
  cudaMemsetAsync(s.bar, 0, sizeof(unsigned) * 2, st);
  cudaMemsetAsync(s.err, 0, sizeof(int), st);
  void* args[] = {&p};
  TM_PROF(st, "coarse_gmres");
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)coarse_gmres_kernel, dim3(G), dim3(CG_THREADS), args,
                                              dyn, st);
  TM_COUNT();
  if (e != cudaSuccess) return -1;
  cudaMemcpyAsync(s.h_flags, s.err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(s.h_flags + 1, s.iters, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (iters_done) {
    cudaStreamSynchronize(st);
    *iters_done = s.h_flags[1];
    if (s.h_flags[0]) return -3;
  }
  return 0;
}

}  // namespace tmamg

// Aggregation-based multigrid on GB300: prolongation P, restriction P^+, Galerkin coarse
// operator D_c = P^+ D P, and the coarse 9-point stencil (paper Sec. 2: P and R are built
// from approximate low modes on aggregates, the coarse operator lives on the lattice of
// aggregates, and the construction recurses).
//
// P layout (per coarsening): float2 P[Vc][2 chi][nv][K] with K = asize * d: for aggregate a,
// chirality chi and test vector j, the K = (d unknowns of that chirality) x (site in aggregate)
// entries, k = c' asize + q (sites fastest, so that consecutive k touch consecutive lattice
// sites); d = 6 (2 spins x 3 colours) when the parent is the fine lattice, and the parent's
// nv when the parent is a coarse lattice. A parent component is chi * d + c'.
// Coarse vectors are bundles with ncomp = nc = 2 nv and nsite = Vc; component chi * nv + j.
// Coarse stencil: float2 A[9][Vc][nc (column j)][nc (row i)], hop index 0 = self,
// 1 + 2 nu = +nu, 2 + 2 nu = -nu.
#include "amg.cuh"
#include "profile.cuh"
#include "stencil.cuh"

namespace tmamg {

constexpr int T2 = 2;  // FP32 tile width

__device__ __forceinline__ void agg_site(int64_t a, int q, const int* Lc, const int* ag, const int* L, int* c) {
  int ac[4], lq[4];
  site_coords(a, Lc, ac);
  site_coords(q, ag, lq);
#pragma unroll
  for (int k = 0; k < 4; ++k) c[k] = ac[k] * ag[k] + lq[k];
}

// ------------------------------------------------------------------ test vectors -> P
// P[a][chi][j][c' asize + q] = V_j[chi d + c'][site(a, q)]   (V: FP32 bundle, nv systems, ncomp = 2 d)
__global__ void gather_P_kernel(const float* __restrict__ Vb, float2* __restrict__ P, AggDims g, int nv, int d) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int K = g.asize * d;
  int64_t total = g.Vc * 2 * nv * (int64_t)K;
  if (t >= total) return;
  int k = (int)(t % K);
  int j = (int)((t / K) % nv);
  int chi = (int)((t / ((int64_t)K * nv)) % 2);
  int64_t a = t / ((int64_t)K * nv * 2);
  int cp = k / g.asize, q = k % g.asize;
  int c[4];
  agg_site(a, q, g.Lc, g.agg, g.L, c);
  int64_t s = site_index(c, g.L);
  int comp = chi * d + cp;
  const float* e = Vb + (((int64_t)(j / T2) * (2 * d) + comp) * g.Vp + s) * 2 * T2;
  P[t] = make_float2(e[j % T2], e[T2 + j % T2]);
}

// Classical Gram-Schmidt applied twice to the nv vectors of one (aggregate, chirality),
// one CTA each; dots in FP64.
__global__ void __launch_bounds__(256) orthonormalise_kernel(float2* __restrict__ P, int nv, int K) {
  float2* Pv = P + (int64_t)blockIdx.x * nv * K;
  __shared__ double2 red[8][8];
  __shared__ double2 coef[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = 0; j < nv; ++j) {
    float2* vj = Pv + (int64_t)j * K;
    for (int pass = 0; pass < 2; ++pass) {
      for (int i0 = 0; i0 < j; i0 += 8) {
        int ni = j - i0 < 8 ? j - i0 : 8;
        double2 acc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = make_double2(0, 0);
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
          float2 w = vj[k];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            if (u < ni) {
              float2 v = Pv[(int64_t)(i0 + u) * K + k];
              acc[u].x += (double)v.x * w.x + (double)v.y * w.y;
              acc[u].y += (double)v.x * w.y - (double)v.y * w.x;
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            acc[u].x += __shfl_xor_sync(0xffffffffu, acc[u].x, o);
            acc[u].y += __shfl_xor_sync(0xffffffffu, acc[u].y, o);
          }
          if (lane == 0) red[warp][u] = acc[u];
        }
        __syncthreads();
        if (threadIdx.x < 8) {
          double2 s = make_double2(0, 0);
          for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            s.x += red[w][threadIdx.x].x;
            s.y += red[w][threadIdx.x].y;
          }
          coef[threadIdx.x] = s;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
          float2 w = vj[k];
          double wr = w.x, wi = w.y;
          for (int u = 0; u < ni; ++u) {
            float2 v = Pv[(int64_t)(i0 + u) * K + k];
            double2 cc = coef[u];
            wr -= cc.x * v.x - cc.y * v.y;
            wi -= cc.x * v.y + cc.y * v.x;
          }
          vj[k] = make_float2((float)wr, (float)wi);
        }
        __syncthreads();
      }
    }
    // normalise
    double nn = 0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      float2 w = vj[k];
      nn += (double)w.x * w.x + (double)w.y * w.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
    if (lane == 0) red[warp][0].x = nn;
    __syncthreads();
    double tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w][0].x;
    double inv = tot > 0 ? 1.0 / sqrt(tot) : 0.0;
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      float2 w = vj[k];
      vj[k] = make_float2((float)(w.x * inv), (float)(w.y * inv));
    }
    __syncthreads();
  }
}

void build_P(const AggDims& g, const float* Vb, float2* P, int nv, int d, cudaStream_t st) {
  int64_t total = g.Vc * 2 * nv * (int64_t)g.asize * d;
  gather_P_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(Vb, P, g, nv, d); TM_COUNT();
  orthonormalise_kernel<<<(unsigned)(g.Vc * 2), 256, 0, st>>>(P, nv, g.asize * d); TM_COUNT();
}

// ------------------------------------------------------------------ restriction / prolongation
// Per aggregate the restriction is a small matrix product xc_a = P_a^+ r_a (2 nv x K times
// K x nsys, K = asize d) and the prolongation its transpose; P_a is read once for all systems.

// xc[tile][chi nv + j][a] = sum_k conj(P[a][chi][j][k]) r[tile][chi d + c'][site(a, q)], k = c' asize + q.
// One CTA per (aggregate, chirality). The vector entries of a chunk of RS_KC values of k are
// staged in shared memory for all tiles (every output row reads them there). A thread owns a
// 3 x 3 block of outputs (three rows j, three system tiles) and one of 16 interleaved slices of
// k; per k it loads three entries of P and reads three staged 16-byte entries, and does nine
// packed complex multiply-adds (both systems of a tile at once). The 16 slice sums of an output
// are added by shuffles in a fixed order.
constexpr int RS_KS = 16;         // k slices (lanes of a half warp)
constexpr int RS_MAX_SLOTS = 24;  // output blocks processed at once per CTA (blockDim.x / RS_KS)
constexpr int RS_KC = 128;        // k values staged per chunk (fewer when many tiles)

// two CTAs per SM (80 registers, no spills): one stages its vector chunk while the other computes
__global__ void __launch_bounds__(RS_KS * RS_MAX_SLOTS, 2) restrict_kernel(const float2* __restrict__ P,
                                                              const float* __restrict__ r, float* __restrict__ xc,
                                                              AggDims g, int nv, int d, int nt, int kc) {
  extern __shared__ float4 rsm[];                            // [nt][kc] staged entries
  int* sidx = reinterpret_cast<int*>(rsm + (size_t)nt * kc);  // [asize] lattice site of each member
  const int64_t a = blockIdx.x >> 1;
  const int chi = blockIdx.x & 1;
  const int K = g.asize * d;
  for (int q = threadIdx.x; q < g.asize; q += blockDim.x) {
    int c[4];
    agg_site(a, q, g.Lc, g.agg, g.L, c);
    sidx[q] = (int)site_index(c, g.L);
  }
  const int ks = threadIdx.x % RS_KS, slot = threadIdx.x / RS_KS;
  const int nslots = blockDim.x / RS_KS;
  const int JG = (nv + 2) / 3, TG = (nt + 2) / 3;
  const float2* Pa = P + ((a * 2 + chi) * nv) * (int64_t)K;
  for (int og0 = 0; og0 < JG * TG; og0 += nslots) {
    const int og = og0 + slot;
    const bool live = og < JG * TG;
    const int jg = live ? og / TG : 0, tg = live ? og % TG : 0;
    const int j0 = 3 * jg, t0 = 3 * tg;
    float2 are[9], aim[9];
#pragma unroll
    for (int u = 0; u < 9; ++u) {
      are[u] = make_float2(0.f, 0.f);
      aim[u] = make_float2(0.f, 0.f);
    }
    for (int kc0 = 0; kc0 < K; kc0 += kc) {
      const int kn = K - kc0 < kc ? K - kc0 : kc;
      __syncthreads();  // sidx ready / the previous chunk consumed
      for (int e = threadIdx.x; e < nt * kn; e += blockDim.x) {
        const int t = e / kn, kk = e - t * kn;
        const int k = kc0 + kk;
        const int cp = k / g.asize, q = k - cp * g.asize;
        rsm[t * kc + kk] =
            __ldg(reinterpret_cast<const float4*>(r + (((int64_t)t * (2 * d) + chi * d + cp) * g.Vp + sidx[q]) * 4));
      }
      __syncthreads();
      if (live) {
#pragma unroll 4
        for (int kk = ks; kk < kn; kk += RS_KS) {
          float2 p[3];
          float4 v[3];
#pragma unroll
          for (int jj = 0; jj < 3; ++jj)
            p[jj] = j0 + jj < nv ? __ldg(Pa + (int64_t)(j0 + jj) * K + kc0 + kk) : make_float2(0.f, 0.f);
#pragma unroll
          for (int tt = 0; tt < 3; ++tt)
            v[tt] = t0 + tt < nt ? rsm[(t0 + tt) * kc + kk] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int jj = 0; jj < 3; ++jj) {
            const float2 pr = make_float2(p[jj].x, p[jj].x), pi = make_float2(p[jj].y, p[jj].y);
            const float2 npi = make_float2(-p[jj].y, -p[jj].y);
#pragma unroll
            for (int tt = 0; tt < 3; ++tt) {
              const float2 vr = make_float2(v[tt].x, v[tt].y), vi = make_float2(v[tt].z, v[tt].w);
              // conj(p) v = (pr vr + pi vi) + i (pr vi - pi vr), both systems at once
              are[jj * 3 + tt] = __ffma2_rn(pr, vr, are[jj * 3 + tt]);
              are[jj * 3 + tt] = __ffma2_rn(pi, vi, are[jj * 3 + tt]);
              aim[jj * 3 + tt] = __ffma2_rn(pr, vi, aim[jj * 3 + tt]);
              aim[jj * 3 + tt] = __ffma2_rn(npi, vr, aim[jj * 3 + tt]);
            }
          }
        }
      }
    }
    // sum of the 16 slices (lanes ks of the half warp), fixed order
#pragma unroll
    for (int u = 0; u < 9; ++u) {
#pragma unroll
      for (int o = RS_KS / 2; o > 0; o >>= 1) {
        are[u].x += __shfl_xor_sync(0xffffffffu, are[u].x, o);
        are[u].y += __shfl_xor_sync(0xffffffffu, are[u].y, o);
        aim[u].x += __shfl_xor_sync(0xffffffffu, aim[u].x, o);
        aim[u].y += __shfl_xor_sync(0xffffffffu, aim[u].y, o);
      }
    }
    if (live && ks == 0) {
#pragma unroll
      for (int jj = 0; jj < 3; ++jj)
#pragma unroll
        for (int tt = 0; tt < 3; ++tt)
          if (j0 + jj < nv && t0 + tt < nt)
            *reinterpret_cast<float4*>(xc + (((int64_t)(t0 + tt) * (2 * nv) + chi * nv + j0 + jj) * g.Vc + a) * 4) =
                make_float4(are[jj * 3 + tt].x, are[jj * 3 + tt].y, aim[jj * 3 + tt].x, aim[jj * 3 + tt].y);
    }
  }
}

void restrict_vec(const AggDims& g, const float2* P, const float* r, float* xc, int nv, int d, int nsys,
                  cudaStream_t st) {
  const int nt = ntiles(nsys, T2);
  int kc = RS_KC;
  while (kc > RS_KS && sizeof(float4) * (size_t)nt * kc + sizeof(int) * g.asize > 100 * 1024) kc -= RS_KS;  // two CTAs per SM
  const size_t smem = sizeof(float4) * (size_t)nt * kc + sizeof(int) * g.asize;
  func_smem_optin((const void*)restrict_kernel, 200 * 1024);
  TM_PROF(st, d == 6 ? "restrict" : "restrict_coarse");
  // every output block of the aggregate in one pass over P and the staged vector chunks when they
  // fit one CTA (rounds of RS_MAX_SLOTS blocks otherwise)
  const int nblk = ((nv + 2) / 3) * ((nt + 2) / 3);
  const int rounds = (nblk + RS_MAX_SLOTS - 1) / RS_MAX_SLOTS;
  const int slots = (nblk + rounds - 1) / rounds;
  restrict_kernel<<<(unsigned)(g.Vc * 2), RS_KS * slots, smem, st>>>(P, r, xc, g, nv, d, nt, kc);
  TM_COUNT();
}

// prolongation: tile chunk and CTA size
constexpr int RP_TCH = 8;
constexpr int RP_THREADS = 256;

// e[tile][chi d + c'][site(a, q)] (+)= sum_j P[a][chi][j][k] xc[tile][chi nv + j][a]:
// one CTA per (aggregate, chirality), threads over k (sites fastest: coalesced reads of P and
// writes of e), the aggregate's coarse vector of a tile chunk in shared memory, packed complex
// multiply-adds over the two systems of a tile
__global__ void __launch_bounds__(RP_THREADS) prolong_kernel(const float2* __restrict__ P,
                                                             const float* __restrict__ xc, float* __restrict__ e,
                                                             AggDims g, int nv, int d, int nt, int accumulate) {
  __shared__ float4 Xs[32][RP_TCH];  // [j][tile of the chunk] for this chirality (nv <= 32)
  extern __shared__ int sidx[];      // [asize]
  const int64_t a = blockIdx.x >> 1;
  const int chi = blockIdx.x & 1;
  const int nc = 2 * nv;
  const int K = g.asize * d;
  for (int q = threadIdx.x; q < g.asize; q += blockDim.x) {
    int c[4];
    agg_site(a, q, g.Lc, g.agg, g.L, c);
    sidx[q] = (int)site_index(c, g.L);
  }
  const float2* Pa = P + ((a * 2 + chi) * nv) * (int64_t)K;
  for (int t0 = 0; t0 < nt; t0 += RP_TCH) {
    const int ntc = nt - t0 < RP_TCH ? nt - t0 : RP_TCH;
    __syncthreads();
    for (int q = threadIdx.x; q < nv * ntc; q += blockDim.x) {
      const int j = q / ntc, u = q % ntc;
      Xs[j][u] = *reinterpret_cast<const float4*>(xc + (((int64_t)(t0 + u) * nc + chi * nv + j) * g.Vc + a) * 4);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      float2 are[RP_TCH], aim[RP_TCH];
#pragma unroll
      for (int u = 0; u < RP_TCH; ++u) {
        are[u] = make_float2(0.f, 0.f);
        aim[u] = make_float2(0.f, 0.f);
      }
#pragma unroll 8
      for (int j = 0; j < nv; ++j) {
        const float2 pv = __ldg(Pa + (int64_t)j * K + k);
        const float2 pr = make_float2(pv.x, pv.x), pi = make_float2(pv.y, pv.y), npi = make_float2(-pv.y, -pv.y);
#pragma unroll
        for (int u = 0; u < RP_TCH; ++u) {
          if (u < ntc) {
            const float4 x = Xs[j][u];
            const float2 xr = make_float2(x.x, x.y), xi = make_float2(x.z, x.w);
            // p x = (pr xr - pi xi) + i (pr xi + pi xr), both systems at once
            are[u] = __ffma2_rn(pr, xr, are[u]);
            are[u] = __ffma2_rn(npi, xi, are[u]);
            aim[u] = __ffma2_rn(pr, xi, aim[u]);
            aim[u] = __ffma2_rn(pi, xr, aim[u]);
          }
        }
      }
      const int cp = k / g.asize, q = k - cp * g.asize;
      const int64_t s = sidx[q];
#pragma unroll
      for (int u = 0; u < RP_TCH; ++u) {
        if (u < ntc) {
          float* out = e + (((int64_t)(t0 + u) * (2 * d) + chi * d + cp) * g.Vp + s) * 4;
          float4 v = make_float4(are[u].x, are[u].y, aim[u].x, aim[u].y);
          if (accumulate) {
            const float4 o = *reinterpret_cast<const float4*>(out);
            v.x += o.x; v.y += o.y; v.z += o.z; v.w += o.w;
          }
          *reinterpret_cast<float4*>(out) = v;
        }
      }
    }
  }
}

void prolong_vec(const AggDims& g, const float2* P, const float* xc, float* e, int nv, int d, int nsys, int accumulate,
                 cudaStream_t st) {
  TM_PROF(st, d == 6 ? "prolong" : "prolong_coarse");
  const int nt = ntiles(nsys, T2);
  prolong_kernel<<<(unsigned)(g.Vc * 2), RP_THREADS, sizeof(int) * g.asize, st>>>(P, xc, e, g, nv, d, nt, accumulate);
  TM_COUNT();
}

// ------------------------------------------------------------------ coarse stencil application
// y[tile][i][a] = sum_h sum_j A[h][a][j][i] x[tile][j][a + h] + i dmu mu_n g5c(i) x[tile][i][a]
__global__ void coarse_apply_kernel(const float2* __restrict__ A, const float* __restrict__ x, float* __restrict__ y,
                                    const double* __restrict__ mu, double dmu, int nsys, CoarseDims cd,
                                    const double* __restrict__ eps) {
  const int nc = cd.nc;
  const int64_t Vc = cd.Vc;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int tile = blockIdx.y;
  if (t >= Vc * nc) return;
  const int i = (int)(t % nc);
  const int64_t a = t / nc;
  int c[4];
  site_coords(a, cd.L, c);
  const float* xt = x + (int64_t)tile * nc * Vc * 2 * T2;
  float4 acc = make_float4(0, 0, 0, 0);
  for (int h = 0; h < 9; ++h) {
    int64_t nb = a;
    if (h > 0) {
      int nu = (h - 1) / 2;
      int dir = ((h - 1) % 2) ? -1 : 1;
      int cc[4] = {c[0], c[1], c[2], c[3]};
      cc[nu] = (cc[nu] + dir + cd.L[nu]) % cd.L[nu];
      nb = site_index(cc, cd.L);
    }
    const float2* Ah = A + (((int64_t)h * Vc + a) * nc) * nc + i;
    const float* xn = xt + nb * 2 * T2;
    for (int j = 0; j < nc; ++j) {
      float2 m = Ah[(int64_t)j * nc];
      float4 v = *reinterpret_cast<const float4*>(xn + (int64_t)j * Vc * 2 * T2);
      acc.x += m.x * v.x - m.y * v.z;
      acc.y += m.x * v.y - m.y * v.w;
      acc.z += m.x * v.z + m.y * v.x;
      acc.w += m.x * v.w + m.y * v.y;
    }
  }
  float4 xs = *reinterpret_cast<const float4*>(xt + ((int64_t)i * Vc + a) * 2 * T2);
  float g5 = i < nc / 2 ? 1.f : -1.f;
  float m0 = 0, m1 = 0;
  int n0 = tile * 2, n1 = tile * 2 + 1;
  if (n0 < nsys) m0 = (float)(dmu * mu[n0]) * g5;
  if (n1 < nsys) m1 = (float)(dmu * mu[n1]) * g5;
  // + i m x
  acc.x -= m0 * xs.z;
  acc.y -= m1 * xs.w;
  acc.z += m0 * xs.x;
  acc.w += m1 * xs.y;
  if (eps) {  // doublet form: - eps times the other flavour (the tile's other lane)
    const float ep = (float)eps[tile];
    acc.x -= ep * xs.y;
    acc.y -= ep * xs.x;
    acc.z -= ep * xs.w;
    acc.w -= ep * xs.z;
  }
  *reinterpret_cast<float4*>(y + ((int64_t)(tile * nc + i) * Vc + a) * 2 * T2) = acc;
}

void coarse_apply(const CoarseDims& cd, const float2* A, const float* x, float* y, const double* mu, double dmu,
                  int nsys, cudaStream_t st, const double* eps) {
  TM_PROF(st, "coarse_apply_f32");
  int nt = ntiles(nsys, T2);
  int64_t total = cd.Vc * cd.nc;
  coarse_apply_kernel<<<dim3((unsigned)((total + 127) / 128), nt), 128, 0, st>>>(A, x, y, mu, dmu, nsys, cd, eps);
  TM_COUNT();
}

// ------------------------------------------------------------------ Galerkin coarse operator
// W[column n = chi nv + j] = P column: at (a, q) component chi' d + c' holds P[a][chi][j][q d + c']
// if chi' == chi, else 0. Fine parent (d = 6): a fine bundle of nc systems.
__global__ void columns_kernel(const float2* __restrict__ P, float* __restrict__ W, AggDims g, int nv, int d) {
  const int K = g.asize * d;
  const int nc = 2 * nv;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // one thread per (column pair = tile, parent component, parent site)
  const int64_t per_tile = (int64_t)(2 * d) * g.Vp;
  if (t >= per_tile * (nc / T2)) return;
  int tile = (int)(t / per_tile);
  int64_t r = t % per_tile;
  int comp = (int)(r / g.Vp);
  int64_t s = r % g.Vp;
  int c[4];
  site_coords(s, g.L, c);
  int ac[4], lq[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    ac[k] = c[k] / g.agg[k];
    lq[k] = c[k] % g.agg[k];
  }
  int64_t a = site_index(ac, g.Lc);
  int q = (int)site_index(lq, g.agg);
  int chi_p = comp / d, cp = comp % d;
  float o[4] = {0, 0, 0, 0};
#pragma unroll
  for (int l = 0; l < T2; ++l) {
    int n = tile * T2 + l;
    int chi = n / nv, j = n % nv;
    if (chi == chi_p) {
      float2 p = P[(((int64_t)a * 2 + chi) * nv + j) * K + cp * g.asize + q];
      o[l] = p.x;
      o[2 + l] = p.y;
    }
  }
  *reinterpret_cast<float4*>(W + t * 2 * T2) = make_float4(o[0], o[1], o[2], o[3]);
}

// Part h of the fine operator applied to the columns: h = 0 gives the clover/diagonal term
// plus every hop whose ends lie in one aggregate; h = 1 + 2 nu (2 + 2 nu) gives the forward
// (backward) hop in direction nu on the sites where it crosses into the next aggregate.
template <typename real, int T>
__global__ void __launch_bounds__(128) split_dirac_kernel(const float2* __restrict__ U, const real* __restrict__ C,
                                                          const real* __restrict__ x, real* __restrict__ y, int ntile,
                                                          AggDims g, int h, int bc_t) {
  const int64_t V = g.Vp;
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int tile = blockIdx.y;
  if (s >= V || tile >= ntile) return;
  int c[4];
  site_coords(s, g.L, c);
  const int64_t tstride = (int64_t)12 * V * 2 * T;
  const real* xt = x + tile * tstride;
  Spinor<real, T> acc;
#pragma unroll
  for (int k = 0; k < 12; ++k)
#pragma unroll
    for (int l = 0; l < T; ++l) { acc.c[k].re[l] = 0; acc.c[k].im[l] = 0; }
  const int64_t strides[4] = {1, (int64_t)g.L[0], (int64_t)g.L[0] * g.L[1], (int64_t)g.L[0] * g.L[1] * g.L[2]};
#define TM_SHOP(NU)                                                                                    \
  {                                                                                                    \
    bool xf = g.Lc[NU] > 1 && (c[NU] % g.agg[NU]) == g.agg[NU] - 1;                                   \
    bool xb = g.Lc[NU] > 1 && (c[NU] % g.agg[NU]) == 0;                                                \
    bool use_f = (h == 0 && !xf) || (h == 1 + 2 * NU && xf);                                           \
    bool use_b = (h == 0 && !xb) || (h == 2 + 2 * NU && xb);                                           \
    if (use_f) {                                                                                       \
      int64_t sf = c[NU] + 1 < g.L[NU] ? s + strides[NU] : s - (int64_t)(g.L[NU] - 1) * strides[NU];   \
      real pf = (NU == 3 && c[3] == g.L[3] - 1) ? (real)bc_t : real(1);                              \
      hop<NU, true, real, T>(acc, xt + sf * 2 * T, V, U + (int64_t)NU * 9 * V, V, s, pf);               \
    }                                                                                                  \
    if (use_b) {                                                                                       \
      int64_t sb = c[NU] > 0 ? s - strides[NU] : s + (int64_t)(g.L[NU] - 1) * strides[NU];              \
      real pb = (NU == 3 && c[3] == 0) ? (real)bc_t : real(1);                                        \
      hop<NU, false, real, T>(acc, xt + sb * 2 * T, V, U + (int64_t)NU * 9 * V, V, sb, pb);             \
    }                                                                                                  \
  }
  TM_SHOP(0)
  TM_SHOP(1)
  TM_SHOP(2)
  TM_SHOP(3)
#undef TM_SHOP
  if (h == 0) {
    real m[T];
#pragma unroll
    for (int l = 0; l < T; ++l) m[l] = 0;
    local_term<real, T>(acc, xt + s * 2 * T, V, C, V, s, m);
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k)
#pragma unroll
      for (int l = 0; l < T; ++l) {
        acc.c[k].re[l] *= real(-0.5);
        acc.c[k].im[l] *= real(-0.5);
      }
  }
  real* yo = y + tile * tstride + s * 2 * T;
#pragma unroll
  for (int k = 0; k < 12; ++k) stcv(yo + (int64_t)k * V * 2 * T, acc.c[k]);
}

// A[h][a][j][i] = R[tile j/2][i][a][lane j%2]  (R: restricted part h of the columns)
__global__ void scatter_A_kernel(const float* __restrict__ R, float2* __restrict__ A, int64_t Vc, int nc, int h) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= Vc * nc * (int64_t)nc) return;
  int i = (int)(t % nc);
  int j = (int)((t / nc) % nc);
  int64_t a = t / ((int64_t)nc * nc);
  const float* e = R + (((int64_t)(j / T2) * nc + i) * Vc + a) * 2 * T2;
  A[(((int64_t)h * Vc + a) * nc + j) * nc + i] = make_float2(e[j % T2], e[T2 + j % T2]);
}

void build_coarse_operator_fine(const AggDims& g, const float2* U32, const float* C32, const float2* P, float2* A,
                                int nv, int bc_t, float* W, float* Y, float* R, cudaStream_t st) {
  const int nc = 2 * nv;
  const int nt = nc / T2;
  int64_t per_tile = (int64_t)12 * g.Vp;
  columns_kernel<<<(unsigned)((per_tile * nt + 255) / 256), 256, 0, st>>>(P, W, g, nv, 6); TM_COUNT();
  CoarseDims cd;
  for (int h = 0; h < 9; ++h) {
    split_dirac_kernel<float, T2><<<dim3((unsigned)((g.Vp + 127) / 128), nt), 128, 0, st>>>(U32, C32, W, Y, nt, g, h,
                                                                                            bc_t); TM_COUNT();
    restrict_vec(g, P, Y, R, nv, 6, nc, st);
    int64_t tot = g.Vc * nc * (int64_t)nc;
    scatter_A_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(R, A, g.Vc, nc, h); TM_COUNT();
  }
  (void)cd;
}

// Part h of a coarse operator (the parent level of aggregation g) applied to x, twisted mass
// left out: h = 0 gives the self block plus every hop whose ends lie in one aggregate of g;
// h = 1 + 2 nu (2 + 2 nu) gives the forward (backward) hop in direction nu on the sites where
// it crosses into the next aggregate. x, y: parent bundles (ncomp = pd.nc, nsite = pd.Vc).
__global__ void split_coarse_kernel(const float2* __restrict__ A, const float* __restrict__ x, float* __restrict__ y,
                                    CoarseDims pd, AggDims g, int h) {
  const int nc = pd.nc;
  const int64_t Vc = pd.Vc;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int tile = blockIdx.y;
  if (t >= Vc * nc) return;
  const int i = (int)(t % nc);
  const int64_t a = t / nc;
  int c[4];
  site_coords(a, pd.L, c);
  const float* xt = x + (int64_t)tile * nc * Vc * 2 * T2;
  float4 acc = make_float4(0, 0, 0, 0);
  for (int hh = 0; hh < 9; ++hh) {
    int64_t nb = a;
    if (hh > 0) {
      const int nu = (hh - 1) / 2;
      const bool fwd = ((hh - 1) & 1) == 0;
      const int r = c[nu] % g.agg[nu];
      const bool cross = g.Lc[nu] > 1 && (fwd ? r == g.agg[nu] - 1 : r == 0);
      if (cross ? hh != h : h != 0) continue;
      int cc[4] = {c[0], c[1], c[2], c[3]};
      cc[nu] = (cc[nu] + (fwd ? 1 : -1) + pd.L[nu]) % pd.L[nu];
      nb = site_index(cc, pd.L);
    } else if (h != 0) {
      continue;
    }
    const float2* Ah = A + (((int64_t)hh * Vc + a) * nc) * nc + i;
    const float* xn = xt + nb * 2 * T2;
    for (int j = 0; j < nc; ++j) {
      const float2 m = Ah[(int64_t)j * nc];
      const float4 v = *reinterpret_cast<const float4*>(xn + (int64_t)j * Vc * 2 * T2);
      acc.x += m.x * v.x - m.y * v.z;
      acc.y += m.x * v.y - m.y * v.w;
      acc.z += m.x * v.z + m.y * v.x;
      acc.w += m.x * v.w + m.y * v.y;
    }
  }
  *reinterpret_cast<float4*>(y + ((int64_t)(tile * nc + i) * Vc + a) * 2 * T2) = acc;
}

void build_coarse_operator_coarse(const AggDims& g, const CoarseDims& pd, const float2* Ap, const float2* P,
                                  float2* A, int nv, float* W, float* Y, float* R, cudaStream_t st) {
  const int d = pd.nc / 2;
  const int nc = 2 * nv;
  const int nt = nc / T2;
  const int64_t per_tile = (int64_t)pd.nc * g.Vp;
  columns_kernel<<<(unsigned)((per_tile * nt + 255) / 256), 256, 0, st>>>(P, W, g, nv, d); TM_COUNT();
  for (int h = 0; h < 9; ++h) {
    split_coarse_kernel<<<dim3((unsigned)((per_tile + 127) / 128), nt), 128, 0, st>>>(Ap, W, Y, pd, g, h); TM_COUNT();
    restrict_vec(g, P, Y, R, nv, d, nc, st);
    const int64_t tot = g.Vc * nc * (int64_t)nc;
    scatter_A_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(R, A, g.Vc, nc, h); TM_COUNT();
  }
}

// field [nsys][Vc][nc] complex float -> coarse bundle [ntile][nc][Vc][2][2] (padding lane zero)
__global__ void pack_coarse_kernel(const float2* __restrict__ f, float* __restrict__ b, int nsys, int nc,
                                   int64_t Vc) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int nt = (nsys + T2 - 1) / T2;
  if (t >= (int64_t)nt * nc * Vc) return;
  const int64_t s = t % Vc;
  const int comp = (int)((t / Vc) % nc);
  const int tile = (int)(t / (Vc * nc));
  float o[4] = {0, 0, 0, 0};
#pragma unroll
  for (int l = 0; l < T2; ++l) {
    const int n = tile * T2 + l;
    if (n < nsys) {
      const float2 v = f[((int64_t)n * Vc + s) * nc + comp];
      o[l] = v.x;
      o[T2 + l] = v.y;
    }
  }
  *reinterpret_cast<float4*>(b + t * 4) = make_float4(o[0], o[1], o[2], o[3]);
}

void pack_coarse(const float* field, float* bundle, int nsys, int nc, int64_t Vc, cudaStream_t st) {
  const int64_t total = (int64_t)ntiles(nsys, T2) * nc * Vc;
  pack_coarse_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(reinterpret_cast<const float2*>(field), bundle,
                                                                     nsys, nc, Vc);
  TM_COUNT();
}

}  // namespace tmamg

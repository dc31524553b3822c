// Fine-level twisted-mass Wilson-clover operator on GB300 (sm_103a).
//
// D(mu) x(s) = A_chi(s) x(s) + i mu gamma5 x(s) - 1/2 sum_nu [(1-gamma_nu) U_nu(s) x(s+nu)
//                                                  + (1+gamma_nu) U_nu(s-nu)^+ x(s-nu)]
// with A_chi = 1/(2 kappa) + c_sw C restricted to chirality chi (the operator of the
// paper's Fig. 6 caption, D_TM = D_W + i mu gamma5, at delta mu = 1).
//
// Design: one thread per (site, tile of T systems). The gauge links and the
// clover blocks of a site are loaded once per thread and applied to all T
// systems of the tile; the T threads of one site that differ only in the tile
// sit in the same CTA, so the re-reads of links and clover hit L1 (paper
// Sec. 3: the matrix data is loaded once for all right-hand sides). Spin
// projection in the chiral basis halves the SU(3) work: each hop multiplies
// two colour vectors.
#include "autotune.cuh"
#include "stencil.cuh"
#include "profile.cuh"

namespace tmamg {

// ---------------------------------------------------------------- gauge conversion
__global__ void convert_gauge_kernel(const double* __restrict__ Uin, double2* __restrict__ U64, float2* __restrict__ U32,
                                     int64_t V) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= V * 4) return;
  int64_t s = t / 4;
  int mu = (int)(t % 4);
  const double* src = Uin + ((s * 4 + mu) * 9) * 2;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    double2 v = make_double2(src[2 * k], src[2 * k + 1]);
    U64[((int64_t)mu * 9 + k) * V + s] = v;
    U32[((int64_t)mu * 9 + k) * V + s] = make_float2((float)v.x, (float)v.y);
  }
}

void launch_convert_gauge(const Geom& g, const double* Uin, double2* U64, float2* U32, cudaStream_t st) {
  int64_t n = g.V * 4;
  int bs = 256;
  convert_gauge_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(Uin, U64, U32, g.V); TM_COUNT();
}

// ---------------------------------------------------------------- clover construction (FP64)
struct M3 {
  double2 e[9];
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ M3 load_link(const double2* U, int mu, int64_t s, int64_t V) {
  M3 m;
#pragma unroll
  for (int k = 0; k < 9; ++k) m.e[k] = U[((int64_t)mu * 9 + k) * V + s];
  return m;
}

__device__ __forceinline__ M3 mm(const M3& a, const M3& b) {  // a b
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 acc = make_double2(0, 0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        double2 p = cmul(a.e[i * 3 + k], b.e[k * 3 + j]);
        acc.x += p.x;
        acc.y += p.y;
      }
      c.e[i * 3 + j] = acc;
    }
  return c;
}

__device__ __forceinline__ M3 mmd(const M3& a, const M3& b) {  // a b^+
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 acc = make_double2(0, 0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        double2 bb = make_double2(b.e[j * 3 + k].x, -b.e[j * 3 + k].y);
        double2 p = cmul(a.e[i * 3 + k], bb);
        acc.x += p.x;
        acc.y += p.y;
      }
      c.e[i * 3 + j] = acc;
    }
  return c;
}

__device__ __forceinline__ M3 dm(const M3& a, const M3& b) {  // a^+ b
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 acc = make_double2(0, 0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        double2 p = cmulc(a.e[k * 3 + i], b.e[k * 3 + j]);
        acc.x += p.x;
        acc.y += p.y;
      }
      c.e[i * 3 + j] = acc;
    }
  return c;
}

__device__ __forceinline__ int64_t nbr(const int* c, const int* L, int mu, int d) {
  int cc[4] = {c[0], c[1], c[2], c[3]};
  cc[mu] = (cc[mu] + d + L[mu]) % L[mu];
  return site_index(cc, L);
}

__device__ __forceinline__ int64_t nbr2(const int* c, const int* L, int mu, int dmu, int nu, int dnu) {
  int cc[4] = {c[0], c[1], c[2], c[3]};
  cc[mu] = (cc[mu] + dmu + L[mu]) % L[mu];
  cc[nu] = (cc[nu] + dnu + L[nu]) % L[nu];
  return site_index(cc, L);
}

// F_{mu nu}(s) = (Q - Q^+)/8 with Q the sum of the four clover leaves at s (mu < nu)
__device__ M3 field_strength(const double2* U, const int* c, const int* L, int64_t V, int mu, int nu) {
  int64_t s = site_index(c, L);
  M3 Umu = load_link(U, mu, s, V);
  M3 Unu = load_link(U, nu, s, V);
  M3 Umu_pnu = load_link(U, mu, nbr(c, L, nu, 1), V);
  M3 Unu_pmu = load_link(U, nu, nbr(c, L, mu, 1), V);
  M3 Umu_mmu = load_link(U, mu, nbr(c, L, mu, -1), V);
  M3 Unu_mmu = load_link(U, nu, nbr(c, L, mu, -1), V);
  M3 Umu_mmu_pnu = load_link(U, mu, nbr2(c, L, mu, -1, nu, 1), V);
  M3 Umu_mmu_mnu = load_link(U, mu, nbr2(c, L, mu, -1, nu, -1), V);
  M3 Unu_mmu_mnu = load_link(U, nu, nbr2(c, L, mu, -1, nu, -1), V);
  M3 Unu_mnu = load_link(U, nu, nbr(c, L, nu, -1), V);
  M3 Umu_mnu = load_link(U, mu, nbr(c, L, nu, -1), V);
  M3 Unu_pmu_mnu = load_link(U, nu, nbr2(c, L, mu, 1, nu, -1), V);
  // leaf 1: U_mu(s) U_nu(s+mu) U_mu(s+nu)^+ U_nu(s)^+
  M3 q = mmd(mmd(mm(Umu, Unu_pmu), Umu_pnu), Unu);
  // leaf 2: U_nu(s) U_mu(s-mu+nu)^+ U_nu(s-mu)^+ U_mu(s-mu)
  M3 t2 = mm(mmd(mmd(Unu, Umu_mmu_pnu), Unu_mmu), Umu_mmu);
  // leaf 3: U_mu(s-mu)^+ U_nu(s-mu-nu)^+ U_mu(s-mu-nu) U_nu(s-nu)
  M3 t3 = mm(dm(Umu_mmu, dm(Unu_mmu_mnu, Umu_mmu_mnu)), Unu_mnu);
  // leaf 4: U_nu(s-nu)^+ U_mu(s-nu) U_nu(s-nu+mu) U_mu(s)^+
  M3 t4 = mmd(mm(dm(Unu_mnu, Umu_mnu), Unu_pmu_mnu), Umu);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    q.e[k].x += t2.e[k].x + t3.e[k].x + t4.e[k].x;
    q.e[k].y += t2.e[k].y + t3.e[k].y + t4.e[k].y;
  }
  M3 F;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 a = q.e[i * 3 + j], b = q.e[j * 3 + i];
      F.e[i * 3 + j] = make_double2((a.x - b.x) * 0.125, (a.y + b.y) * 0.125);
    }
  return F;
}

// Per chirality chi (sign s = +1, -1) in the chiral basis:
//   c_sw C_chi = (i c_sw / 2) [[G3, G1 - i G2], [G1 + i G2, -G3]]   (2x2 spin blocks of 3x3 colour)
//   G1 = s F_xt - F_yz,  G2 = s F_yt + F_xz,  G3 = s F_zt - F_xy.
// Stored with the diagonal 1/(2 kappa) folded in: 6 real diagonal entries, then the
// 15 complex entries of the strict lower triangle (row i > col j, row-major), 36 reals.
__global__ void build_clover_kernel(const double2* __restrict__ U, int Lx, int Ly, int Lz, int Lt, double kappa,
                                    double c_sw, double* __restrict__ C64, float* __restrict__ C32) {
  int L[4] = {Lx, Ly, Lz, Lt};
  int64_t V = (int64_t)Lx * Ly * Lz * Lt;
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= V) return;
  int c[4];
  site_coords(s, L, c);
  M3 F01 = field_strength(U, c, L, V, 0, 1);
  M3 F02 = field_strength(U, c, L, V, 0, 2);
  M3 F03 = field_strength(U, c, L, V, 0, 3);
  M3 F12 = field_strength(U, c, L, V, 1, 2);
  M3 F13 = field_strength(U, c, L, V, 1, 3);
  M3 F23 = field_strength(U, c, L, V, 2, 3);
  const double diag = 1.0 / (2.0 * kappa);
  for (int chi = 0; chi < 2; ++chi) {
    double sg = chi == 0 ? 1.0 : -1.0;
    double2 A[6][6];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        int k = a * 3 + b;
        double2 G1 = make_double2(sg * F03.e[k].x - F12.e[k].x, sg * F03.e[k].y - F12.e[k].y);
        double2 G2 = make_double2(sg * F13.e[k].x + F02.e[k].x, sg * F13.e[k].y + F02.e[k].y);
        double2 G3 = make_double2(sg * F23.e[k].x - F01.e[k].x, sg * F23.e[k].y - F01.e[k].y);
        // iG2 = (-G2.y, G2.x)
        double2 b00 = G3;
        double2 b01 = make_double2(G1.x + G2.y, G1.y - G2.x);  // G1 - i G2
        double2 b10 = make_double2(G1.x - G2.y, G1.y + G2.x);  // G1 + i G2
        double2 b11 = make_double2(-G3.x, -G3.y);
        // multiply by i c_sw / 2: (x, y) -> (-y, x) * c_sw / 2
        double h = 0.5 * c_sw;
        A[a][b] = make_double2(-b00.y * h, b00.x * h);
        A[a][3 + b] = make_double2(-b01.y * h, b01.x * h);
        A[3 + a][b] = make_double2(-b10.y * h, b10.x * h);
        A[3 + a][3 + b] = make_double2(-b11.y * h, b11.x * h);
      }
    double* out64 = C64 + (int64_t)chi * 36 * V;
    float* out32 = C32 + (int64_t)chi * 36 * V;
    for (int i = 0; i < 6; ++i) {
      double d = A[i][i].x + diag;
      out64[(int64_t)i * V + s] = d;
      out32[(int64_t)i * V + s] = (float)d;
    }
    int k = 6;
    for (int i = 1; i < 6; ++i)
      for (int j = 0; j < i; ++j) {
        out64[(int64_t)k * V + s] = A[i][j].x;
        out64[(int64_t)(k + 1) * V + s] = A[i][j].y;
        out32[(int64_t)k * V + s] = (float)A[i][j].x;
        out32[(int64_t)(k + 1) * V + s] = (float)A[i][j].y;
        k += 2;
      }
  }
}

void launch_build_clover(const Geom& g, const double2* U64, double kappa, double c_sw, double* C64, float* C32,
                         cudaStream_t st) {
  int bs = 128;
  build_clover_kernel<<<(unsigned)((g.V + bs - 1) / bs), bs, 0, st>>>(U64, g.L[0], g.L[1], g.L[2], g.L[3], kappa,
                                                                       c_sw, C64, C32); TM_COUNT();
}

// FP32: 192-thread CTAs, two per SM, up to 170 registers (no spills); FP64: 256 threads, one per SM
// RES: residual form y = b - D x (b = bsub, tile tile / nshift), else y = D x (bsub unused).
// MAXT, MINB: the launch variant's largest CTA and the CTAs per SM it is compiled for (which sets the
// register budget); every variant does the same per-thread arithmetic.
template <typename real, int T, int BX, bool RES, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) dirac_kernel(const typename LinkT<real>::t* __restrict__ U,
                                                    const real* __restrict__ C, const real* __restrict__ x,
                                                    real* y, const double* __restrict__ mu, int nsys,
                                                    int ntile, int Lx, int Ly, int Lz, int Lt, real bc_t,
                                                    const real* bsub, int nshift,
                                                    const double* __restrict__ eps) {
  // y is not restrict-qualified: the residual form may run in place (bsub == y), every thread
  // reading b at its own site before it writes y there; x never overlaps y
  const int64_t V = (int64_t)Lx * Ly * Lz * Lt;
  const int64_t s = blockIdx.x * (int64_t)BX + threadIdx.x;
  const int tile = blockIdx.y * blockDim.y + threadIdx.y;
  if (s >= V || tile >= ntile) return;
  const int L[4] = {Lx, Ly, Lz, Lt};
  int c[4];
  site_coords(s, L, c);
  const int64_t tstride = (int64_t)12 * V * 2 * T;
  const real* xt = x + tile * tstride;
  const int64_t strides[4] = {1, (int64_t)Lx, (int64_t)Lx * Ly, (int64_t)Lx * Ly * Lz};
  if constexpr (sizeof(real) == 4) {
    // packed FP32x2 arithmetic over the tile's two systems
    Spinor2 acc;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      acc.c[k].re = make_float2(0.f, 0.f);
      acc.c[k].im = make_float2(0.f, 0.f);
    }
    // software pipeline over the eight hops: the neighbour spinor of hop k + 1 is loaded before
    // the colour multiply of hop k, so its latency overlaps that arithmetic (loading the site's own
    // spinor for the local term the same way measured slower)
    int64_t nb[8];
#pragma unroll
    for (int nu = 0; nu < 4; ++nu) {
      nb[2 * nu] = c[nu] + 1 < L[nu] ? s + strides[nu] : s - (int64_t)(L[nu] - 1) * strides[nu];
      nb[2 * nu + 1] = c[nu] > 0 ? s - strides[nu] : s + (int64_t)(L[nu] - 1) * strides[nu];
    }
    const float pf = c[3] == Lt - 1 ? (float)bc_t : 1.f, pb = c[3] == 0 ? (float)bc_t : 1.f;
    Raw2 raw;
    CV2 h[2][3];
    ld_raw2(raw, xt + nb[0] * 4, V);
#define TM_PHOP(NU, FWD, K)                                                                          \
    proj_raw2<NU, FWD>(h, raw);                                                                      \
    if (K < 7) ld_raw2(raw, xt + nb[K < 7 ? K + 1 : 0] * 4, V);                                        \
    mul_acc2<NU, FWD>(acc, h, U + (int64_t)NU * 9 * V, V, FWD ? s : nb[K], NU == 3 ? (FWD ? pf : pb) : 1.f);
    TM_PHOP(0, true, 0)
    TM_PHOP(0, false, 1)
    TM_PHOP(1, true, 2)
    TM_PHOP(1, false, 3)
    TM_PHOP(2, true, 4)
    TM_PHOP(2, false, 5)
    TM_PHOP(3, true, 6)
    TM_PHOP(3, false, 7)
#undef TM_PHOP
    const int n0 = tile * 2;
    const float2 m2 = make_float2(n0 < nsys ? (float)mu[n0] : 0.f, n0 + 1 < nsys ? (float)mu[n0 + 1] : 0.f);
    // eps (doublet form): the tile's two systems are the flavours u, d of one doublet
    local2(acc, xt + s * 4, V, C, V, s, m2, eps ? (float)eps[tile] : 0.f);
    real* yo = y + tile * tstride + s * 4;
    if constexpr (RES) {
      // residual form y = b - D x (b tile tile / nshift)
      const real* bo = bsub + (int64_t)(tile / nshift) * tstride + s * 4;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const CV2 bv = ld2(bo + (int64_t)k * V * 4);
        acc.c[k].re = sub2(bv.re, acc.c[k].re);
        acc.c[k].im = sub2(bv.im, acc.c[k].im);
      }
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) st2(yo + (int64_t)k * V * 4, acc.c[k]);
  } else {
    Spinor<real, T> acc;
#pragma unroll
    for (int k = 0; k < 12; ++k)
#pragma unroll
      for (int l = 0; l < T; ++l) { acc.c[k].re[l] = 0; acc.c[k].im[l] = 0; }

#define TM_HOP(NU)                                                                                   \
    {                                                                                                  \
      int64_t sf = c[NU] + 1 < L[NU] ? s + strides[NU] : s - (int64_t)(L[NU] - 1) * strides[NU];      \
      int64_t sb = c[NU] > 0 ? s - strides[NU] : s + (int64_t)(L[NU] - 1) * strides[NU];               \
      real pf = (NU == 3 && c[3] == Lt - 1) ? bc_t : real(1);                                         \
      real pb = (NU == 3 && c[3] == 0) ? bc_t : real(1);                                              \
      hop<NU, true, real, T>(acc, xt + sf * 2 * T, V, U + (int64_t)NU * 9 * V, V, s, pf);               \
      hop<NU, false, real, T>(acc, xt + sb * 2 * T, V, U + (int64_t)NU * 9 * V, V, sb, pb);             \
    }
    TM_HOP(0)
    TM_HOP(1)
    TM_HOP(2)
    TM_HOP(3)
#undef TM_HOP
    real m[T];
#pragma unroll
    for (int l = 0; l < T; ++l) {
      int n = tile * T + l;
      m[l] = n < nsys ? (real)mu[n] : real(0);
    }
    // eps (doublet form, one system per tile): tiles 2p and 2p + 1 are the flavours u, d of doublet p
    const real* xp = eps ? x + (int64_t)(tile ^ 1) * tstride + s * 2 * T : nullptr;
    local_term<real, T>(acc, xt + s * 2 * T, V, C, V, s, m, xp, eps ? (real)eps[tile >> 1] : real(0));
    real* yo = y + tile * tstride + s * 2 * T;
    if constexpr (RES) {
      // residual form y = b - D x, with b stored once per right-hand side (tile / nshift; for a
      // doublet, once per right-hand side and flavour: tile (p / nshift) 2 + f of doublet p = tile / 2)
      const int bt = eps ? ((tile >> 1) / nshift) * 2 + (tile & 1) : tile / nshift;
      const real* bo = bsub + (int64_t)bt * tstride + s * 2 * T;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        CV<real, T> bv;
        ldcv(bv, bo + (int64_t)k * V * 2 * T);
#pragma unroll
        for (int l = 0; l < T; ++l) {
          acc.c[k].re[l] = bv.re[l] - acc.c[k].re[l];
          acc.c[k].im[l] = bv.im[l] - acc.c[k].im[l];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) stcv(yo + (int64_t)k * V * 2 * T, acc.c[k]);
  }
}

// largest divisor of nt that keeps the CTA at <= maxthreads threads
static inline int pick_ty(int nt, int bx, int maxthreads) {
  int best = 1;
  for (int d = 1; d * bx <= maxthreads && d <= nt; ++d)
    if (nt % d == 0) best = d;
  return best;
}

// launch variants: (sites per CTA row, largest CTA, CTAs per SM). FP32: 168 registers at 12 warps
// per SM, or 128 registers (a few bytes of spills) at 16 warps per SM; FP64: 254 registers at 8
// warps, or 168 registers (about 100 bytes of spills) at 12 warps.
template <typename real, bool RES, int BX, int MAXT, int MINB>
static void launch_variant(const Geom& g, const void* U, const real* C, const real* x, real* y, const double* mu,
                           int nsys, const real* b, int nshift, const double* eps, cudaStream_t st) {
  constexpr int T = Tile<real>::T;
  const int nt = ntiles(nsys, T);
  const int ty = pick_ty(nt, BX, MAXT);
  dim3 block(BX, ty);
  dim3 grid((unsigned)((g.V + BX - 1) / BX), (unsigned)(nt / ty));
  dirac_kernel<real, T, BX, RES, MAXT, MINB><<<grid, block, 0, st>>>(
      reinterpret_cast<const typename LinkT<real>::t*>(U), C, x, y, mu, nsys, nt, g.L[0], g.L[1], g.L[2], g.L[3],
      (real)g.bc_t, b, nshift, eps); TM_COUNT();
}

template <typename real, bool RES>
static void launch_variant_k(int v, const Geom& g, const void* U, const real* C, const real* x, real* y,
                             const double* mu, int nsys, const real* b, int nshift, const double* eps,
                             cudaStream_t st) {
  if constexpr (sizeof(real) == 4) {
    switch (v) {
      case 1: launch_variant<real, RES, 32, 256, 2>(g, U, C, x, y, mu, nsys, b, nshift, eps, st); return;
      case 2: launch_variant<real, RES, 64, 256, 2>(g, U, C, x, y, mu, nsys, b, nshift, eps, st); return;
      case 3: launch_variant<real, RES, 32, 128, 4>(g, U, C, x, y, mu, nsys, b, nshift, eps, st); return;
      default: launch_variant<real, RES, 32, 192, 2>(g, U, C, x, y, mu, nsys, b, nshift, eps, st); return;
    }
  } else {
    switch (v) {
      case 1: launch_variant<real, RES, 64, 192, 2>(g, U, C, x, y, mu, nsys, b, nshift, eps, st); return;
      case 2: launch_variant<real, RES, 32, 192, 2>(g, U, C, x, y, mu, nsys, b, nshift, eps, st); return;
      default: launch_variant<real, RES, 64, 256, 1>(g, U, C, x, y, mu, nsys, b, nshift, eps, st); return;
    }
  }
}

template <typename real>
static constexpr int n_variants() {
  return sizeof(real) == 4 ? 4 : 3;
}

// the tuned variant of a family for this lattice and system count; tuning (which runs every variant
// on this call's data) only when `may_tune`, i.e. when the launch is repeatable
template <typename real, bool RES>
static void launch_tuned(const char* family, bool may_tune, const Geom& g, const void* U, const real* C, const real* x,
                         real* y, const double* mu, int nsys, const real* b, int nshift, const double* eps,
                         cudaStream_t st) {
  const int64_t key = g.V * 4096 + nsys;
  int v = 0;
  if (tune_forced() >= 0) {
    v = tune_forced() < n_variants<real>() ? tune_forced() : 0;
  } else if (autotune_on()) {
    v = tune_lookup(family, key);
    if (v < 0)
      v = may_tune ? tune_run(family, key, n_variants<real>(),
                              [&](int k) {
                                launch_variant_k<real, RES>(k, g, U, C, x, y, mu, nsys, b, nshift, eps, st);
                              },
                              st)
                   : 0;
  }
  launch_variant_k<real, RES>(v, g, U, C, x, y, mu, nsys, b, nshift, eps, st);
}

template <typename real>
void launch_dirac(const Geom& g, const void* U, const real* C, const real* x, real* y, const double* mu, int nsys,
                  cudaStream_t st, const double* eps) {
  TM_PROF(st, sizeof(real) == 4 ? "dirac_f32" : "dirac_f64");
  launch_tuned<real, false>(sizeof(real) == 4 ? "dirac_f32" : "dirac_f64", true, g, U, C, x, y, mu, nsys, nullptr, 1,
                            eps, st);
}

void launch_residual32(const Geom& g, const float2* U, const float* C, const float* x, const float* b, float* r,
                       const double* mu, int nsys, cudaStream_t st, const double* eps) {
  TM_PROF(st, "residual_f32");
  // tuned only out of place (in place, b == r, the launch is not repeatable)
  launch_tuned<float, true>("residual_f32", b != r, g, reinterpret_cast<const void*>(U), C, x, r, mu, nsys, b, 1, eps,
                            st);
}

void launch_residual64(const Geom& g, const double2* U, const double* C, const double* x, const double* b, int nshift,
                       double* r, const double* mu, int nsys, cudaStream_t st, const double* eps) {
  TM_PROF(st, "residual_f64");
  launch_tuned<double, true>("residual_f64", b != r, g, reinterpret_cast<const void*>(U), C, x, r, mu, nsys, b, nshift,
                             eps, st);
}

template void launch_dirac<float>(const Geom&, const void*, const float*, const float*, float*, const double*, int,
                                  cudaStream_t, const double*);
template void launch_dirac<double>(const Geom&, const void*, const double*, const double*, double*, const double*,
                                   int, cudaStream_t, const double*);

// ---------------------------------------------------------------- pack / unpack
// field: complex [nsys][V][12]; bundle: [ntile][12][V][2][T]
template <typename real>
__global__ void pack_kernel(const real* __restrict__ f, real* __restrict__ b, int nsys, int ntile, int64_t V) {
  constexpr int T = Tile<real>::T;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t total = (int64_t)ntile * 12 * V;
  if (t >= total) return;
  int64_t s = t % V;
  int comp = (int)((t / V) % 12);
  int tile = (int)(t / (V * 12));
  real* dst = b + t * 2 * T;
#pragma unroll
  for (int l = 0; l < T; ++l) {
    int n = tile * T + l;
    real re = 0, im = 0;
    if (n < nsys) {
      const real* src = f + (((int64_t)n * V + s) * 12 + comp) * 2;
      re = src[0];
      im = src[1];
    }
    dst[l] = re;
    dst[T + l] = im;
  }
}

template <typename real>
__global__ void unpack_kernel(const real* __restrict__ b, real* __restrict__ f, int nsys, int ntile, int64_t V) {
  constexpr int T = Tile<real>::T;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t total = (int64_t)ntile * 12 * V;
  if (t >= total) return;
  int64_t s = t % V;
  int comp = (int)((t / V) % 12);
  int tile = (int)(t / (V * 12));
  const real* src = b + t * 2 * T;
#pragma unroll
  for (int l = 0; l < T; ++l) {
    int n = tile * T + l;
    if (n < nsys) {
      real* dst = f + (((int64_t)n * V + s) * 12 + comp) * 2;
      dst[0] = src[l];
      dst[1] = src[T + l];
    }
  }
}

template <typename real>
void launch_pack(const Geom& g, const real* field, real* bundle, int nsys, cudaStream_t st) {
  int nt = ntiles(nsys, Tile<real>::T);
  int64_t total = (int64_t)nt * 12 * g.V;
  int bs = 256;
  pack_kernel<real><<<(unsigned)((total + bs - 1) / bs), bs, 0, st>>>(field, bundle, nsys, nt, g.V); TM_COUNT();
}

template <typename real>
void launch_unpack(const Geom& g, const real* bundle, real* field, int nsys, cudaStream_t st) {
  int nt = ntiles(nsys, Tile<real>::T);
  int64_t total = (int64_t)nt * 12 * g.V;
  int bs = 256;
  unpack_kernel<real><<<(unsigned)((total + bs - 1) / bs), bs, 0, st>>>(bundle, field, nsys, nt, g.V); TM_COUNT();
}

template void launch_pack<float>(const Geom&, const float*, float*, int, cudaStream_t);
template void launch_pack<double>(const Geom&, const double*, double*, int, cudaStream_t);
template void launch_unpack<float>(const Geom&, const float*, float*, int, cudaStream_t);
template void launch_unpack<double>(const Geom&, const double*, double*, int, cudaStream_t);

}  // namespace tmamg

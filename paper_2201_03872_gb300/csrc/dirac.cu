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
#include "common.cuh"

namespace tmamg {

// ---------------------------------------------------------------- small complex helpers
template <typename real>
struct cplx {
  real r, i;
};

// multiply by one of {+1, -1, +i, -i} encoded as 0, 1, 2, 3
template <int K, typename real>
__device__ __forceinline__ void mulc(real ar, real ai, real& br, real& bi) {
  if (K == 0) { br = ar; bi = ai; }
  if (K == 1) { br = -ar; bi = -ai; }
  if (K == 2) { br = -ai; bi = ar; }
  if (K == 3) { br = ai; bi = -ar; }
}

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
  convert_gauge_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(Uin, U64, U32, g.V);
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
                                                                       c_sw, C64, C32);
}

// ---------------------------------------------------------------- the stencil
template <typename real>
struct LinkT;
template <>
struct LinkT<float> {
  using t = float2;
};
template <>
struct LinkT<double> {
  using t = double2;
};

// T-lane complex value: re[T], im[T]
template <typename real, int T>
struct CV {
  real re[T];
  real im[T];
};

template <typename real, int T>
__device__ __forceinline__ void ldcv(CV<real, T>& v, const real* __restrict__ p) {
  if constexpr (sizeof(real) == 4 && T == 4) {
    float4 a = __ldg(reinterpret_cast<const float4*>(p));
    float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
    v.re[0] = a.x; v.re[1] = a.y; v.re[2] = a.z; v.re[3] = a.w;
    v.im[0] = b.x; v.im[1] = b.y; v.im[2] = b.z; v.im[3] = b.w;
  } else if constexpr (sizeof(real) == 8 && T == 2) {
    double2 a = __ldg(reinterpret_cast<const double2*>(p));
    double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    v.re[0] = a.x; v.re[1] = a.y;
    v.im[0] = b.x; v.im[1] = b.y;
  } else {
#pragma unroll
    for (int l = 0; l < T; ++l) { v.re[l] = p[l]; v.im[l] = p[T + l]; }
  }
}

template <typename real, int T>
__device__ __forceinline__ void stcv(real* __restrict__ p, const CV<real, T>& v) {
  if constexpr (sizeof(real) == 4 && T == 4) {
    reinterpret_cast<float4*>(p)[0] = make_float4(v.re[0], v.re[1], v.re[2], v.re[3]);
    reinterpret_cast<float4*>(p)[1] = make_float4(v.im[0], v.im[1], v.im[2], v.im[3]);
  } else if constexpr (sizeof(real) == 8 && T == 2) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v.re[0], v.re[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v.im[0], v.im[1]);
  } else {
#pragma unroll
    for (int l = 0; l < T; ++l) { p[l] = v.re[l]; p[T + l] = v.im[l]; }
  }
}

// Projection / reconstruction constants for the chiral basis.
// Forward hop uses (1 - gamma_nu), backward (1 + gamma_nu). With x = (u0, u1, d0, d1)
// (spins 0..3), the half spinor is h_a = u_a + cK_a * d_{p_a} and the lower spins of the
// result are d'_a = bK_a * g_{p_a}, g = U h (or U^+ h).
template <int NU, bool FWD>
struct Proj;
// x: (1 -/+ gamma_1): h = (u0 +/- i d1, u1 +/- i d0); lower (-/+ i g1, -/+ i g0)
template <> struct Proj<0, true>  { static constexpr int p0 = 1, p1 = 0, c0 = 2, c1 = 2, b0 = 3, b1 = 3; };
template <> struct Proj<0, false> { static constexpr int p0 = 1, p1 = 0, c0 = 3, c1 = 3, b0 = 2, b1 = 2; };
// y: h = (u0 +/- d1, u1 -/+ d0); lower (-/+ g1, +/- g0)
template <> struct Proj<1, true>  { static constexpr int p0 = 1, p1 = 0, c0 = 0, c1 = 1, b0 = 1, b1 = 0; };
template <> struct Proj<1, false> { static constexpr int p0 = 1, p1 = 0, c0 = 1, c1 = 0, b0 = 0, b1 = 1; };
// z: h = (u0 +/- i d0, u1 -/+ i d1); lower (-/+ i g0, +/- i g1)
template <> struct Proj<2, true>  { static constexpr int p0 = 0, p1 = 1, c0 = 2, c1 = 3, b0 = 3, b1 = 2; };
template <> struct Proj<2, false> { static constexpr int p0 = 0, p1 = 1, c0 = 3, c1 = 2, b0 = 2, b1 = 3; };
// t: h = u -/+ d; lower -/+ g
template <> struct Proj<3, true>  { static constexpr int p0 = 0, p1 = 1, c0 = 1, c1 = 1, b0 = 1, b1 = 1; };
template <> struct Proj<3, false> { static constexpr int p0 = 0, p1 = 1, c0 = 0, c1 = 0, b0 = 0, b1 = 0; };

template <typename real, int T>
struct Spinor {
  CV<real, T> c[12];  // spin * 3 + colour
};

// acc += (1 -/+ gamma_nu) W psi(nbr) * phase   with W = U_nu(s) (FWD) or U_nu(s-nu)^+ (!FWD)
template <int NU, bool FWD, typename real, int T>
__device__ __forceinline__ void hop(Spinor<real, T>& acc, const real* __restrict__ xs, int64_t V,
                                    const typename LinkT<real>::t* __restrict__ U, int64_t ls, real phase) {
  using P = Proj<NU, FWD>;
  using L2 = typename LinkT<real>::t;
  // half spinor h[a][colour]
  CV<real, T> h[2][3];
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    CV<real, T> u0, u1, d0, d1;
    ldcv(u0, xs + (int64_t)(0 * 3 + col) * V * 2 * T);
    ldcv(u1, xs + (int64_t)(1 * 3 + col) * V * 2 * T);
    ldcv(d0, xs + (int64_t)(2 * 3 + col) * V * 2 * T);
    ldcv(d1, xs + (int64_t)(3 * 3 + col) * V * 2 * T);
    const CV<real, T>& dp0 = P::p0 == 0 ? d0 : d1;
    const CV<real, T>& dp1 = P::p1 == 0 ? d0 : d1;
#pragma unroll
    for (int l = 0; l < T; ++l) {
      real tr, ti;
      mulc<P::c0>(dp0.re[l], dp0.im[l], tr, ti);
      h[0][col].re[l] = (u0.re[l] + tr) * phase;
      h[0][col].im[l] = (u0.im[l] + ti) * phase;
      mulc<P::c1>(dp1.re[l], dp1.im[l], tr, ti);
      h[1][col].re[l] = (u1.re[l] + tr) * phase;
      h[1][col].im[l] = (u1.im[l] + ti) * phase;
    }
  }
  // g = W h, then scatter into the four spins
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    L2 w[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (FWD) {
        w[b] = U[(int64_t)(a * 3 + b) * V + ls];
      } else {
        L2 t = U[(int64_t)(b * 3 + a) * V + ls];
        w[b].x = t.x;
        w[b].y = -t.y;
      }
    }
    CV<real, T> g[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
#pragma unroll
      for (int l = 0; l < T; ++l) {
        real gr = w[0].x * h[k][0].re[l] - w[0].y * h[k][0].im[l];
        real gi = w[0].x * h[k][0].im[l] + w[0].y * h[k][0].re[l];
        gr += w[1].x * h[k][1].re[l] - w[1].y * h[k][1].im[l];
        gi += w[1].x * h[k][1].im[l] + w[1].y * h[k][1].re[l];
        gr += w[2].x * h[k][2].re[l] - w[2].y * h[k][2].im[l];
        gi += w[2].x * h[k][2].im[l] + w[2].y * h[k][2].re[l];
        g[k].re[l] = gr;
        g[k].im[l] = gi;
      }
    }
#pragma unroll
    for (int l = 0; l < T; ++l) {
      acc.c[0 * 3 + a].re[l] += g[0].re[l];
      acc.c[0 * 3 + a].im[l] += g[0].im[l];
      acc.c[1 * 3 + a].re[l] += g[1].re[l];
      acc.c[1 * 3 + a].im[l] += g[1].im[l];
      real tr, ti;
      const CV<real, T>& gp0 = P::p0 == 0 ? g[0] : g[1];
      const CV<real, T>& gp1 = P::p1 == 0 ? g[0] : g[1];
      mulc<P::b0>(gp0.re[l], gp0.im[l], tr, ti);
      acc.c[2 * 3 + a].re[l] += tr;
      acc.c[2 * 3 + a].im[l] += ti;
      mulc<P::b1>(gp1.re[l], gp1.im[l], tr, ti);
      acc.c[3 * 3 + a].re[l] += tr;
      acc.c[3 * 3 + a].im[l] += ti;
    }
  }
}

// y_chi = A_chi x_chi (Hermitian 6x6 packed) + i s mu x_chi, combined with the hop sum:
// out = A x + i s mu x - 1/2 hopsum
template <typename real, int T>
__device__ __forceinline__ void local_term(const Spinor<real, T>& hs, const real* __restrict__ x0, int64_t V,
                                           const real* __restrict__ C, int64_t s, const real* mu, real* __restrict__ y0) {
#pragma unroll
  for (int chi = 0; chi < 2; ++chi) {
    const real* Cc = C + (int64_t)chi * 36 * V + s;
    CV<real, T> xc[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) ldcv(xc[i], x0 + (int64_t)(chi * 6 + i) * V * 2 * T);
    real sg = chi == 0 ? real(1) : real(-1);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      CV<real, T> o;
      real d = Cc[(int64_t)i * V];
#pragma unroll
      for (int l = 0; l < T; ++l) {
        // diagonal + twist: (d + i s mu) x_i
        o.re[l] = d * xc[i].re[l] - sg * mu[l] * xc[i].im[l];
        o.im[l] = d * xc[i].im[l] + sg * mu[l] * xc[i].re[l];
      }
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        if (j == i) continue;
        real ar, ai;
        if (i > j) {
          int k = 6 + 2 * (i * (i - 1) / 2 + j);
          ar = Cc[(int64_t)k * V];
          ai = Cc[(int64_t)(k + 1) * V];
        } else {
          int k = 6 + 2 * (j * (j - 1) / 2 + i);
          ar = Cc[(int64_t)k * V];
          ai = -Cc[(int64_t)(k + 1) * V];
        }
#pragma unroll
        for (int l = 0; l < T; ++l) {
          o.re[l] += ar * xc[j].re[l] - ai * xc[j].im[l];
          o.im[l] += ar * xc[j].im[l] + ai * xc[j].re[l];
        }
      }
      const CV<real, T>& hv = hs.c[chi * 6 + i];
#pragma unroll
      for (int l = 0; l < T; ++l) {
        o.re[l] -= real(0.5) * hv.re[l];
        o.im[l] -= real(0.5) * hv.im[l];
      }
      stcv(y0 + (int64_t)(chi * 6 + i) * V * 2 * T, o);
    }
  }
}

template <typename real, int T, int BX>
__global__ void __launch_bounds__(256) dirac_kernel(const typename LinkT<real>::t* __restrict__ U,
                                                    const real* __restrict__ C, const real* __restrict__ x,
                                                    real* __restrict__ y, const double* __restrict__ mu, int nsys,
                                                    int ntile, int Lx, int Ly, int Lz, int Lt, real bc_t) {
  const int64_t V = (int64_t)Lx * Ly * Lz * Lt;
  const int64_t s = blockIdx.x * (int64_t)BX + threadIdx.x;
  const int tile = blockIdx.y * blockDim.y + threadIdx.y;
  if (s >= V || tile >= ntile) return;
  const int L[4] = {Lx, Ly, Lz, Lt};
  int c[4];
  site_coords(s, L, c);
  const int64_t tstride = (int64_t)12 * V * 2 * T;
  const real* xt = x + tile * tstride;
  Spinor<real, T> acc;
#pragma unroll
  for (int k = 0; k < 12; ++k)
#pragma unroll
    for (int l = 0; l < T; ++l) { acc.c[k].re[l] = 0; acc.c[k].im[l] = 0; }

  const int64_t strides[4] = {1, (int64_t)Lx, (int64_t)Lx * Ly, (int64_t)Lx * Ly * Lz};
#define TM_HOP(NU)                                                                                   \
  {                                                                                                  \
    int64_t sf = c[NU] + 1 < L[NU] ? s + strides[NU] : s - (int64_t)(L[NU] - 1) * strides[NU];      \
    int64_t sb = c[NU] > 0 ? s - strides[NU] : s + (int64_t)(L[NU] - 1) * strides[NU];               \
    real pf = (NU == 3 && c[3] == Lt - 1) ? bc_t : real(1);                                         \
    real pb = (NU == 3 && c[3] == 0) ? bc_t : real(1);                                              \
    hop<NU, true, real, T>(acc, xt + sf * 2 * T, V, U + (int64_t)NU * 9 * V, s, pf);                  \
    hop<NU, false, real, T>(acc, xt + sb * 2 * T, V, U + (int64_t)NU * 9 * V, sb, pb);                \
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
  local_term<real, T>(acc, xt + s * 2 * T, V, C, s, m, y + tile * tstride + s * 2 * T);
}

template <typename real>
void launch_dirac(const Geom& g, const void* U, const real* C, const real* x, real* y, const double* mu, int nsys,
                  cudaStream_t st) {
  constexpr int T = Tile<real>::T;
  constexpr int BX = 64;
  int nt = ntiles(nsys, T);
  int ty = nt < 4 ? nt : 4;
  dim3 block(BX, ty);
  dim3 grid((unsigned)((g.V + BX - 1) / BX), (unsigned)((nt + ty - 1) / ty));
  dirac_kernel<real, T, BX><<<grid, block, 0, st>>>(reinterpret_cast<const typename LinkT<real>::t*>(U), C, x, y, mu,
                                                    nsys, nt, g.L[0], g.L[1], g.L[2], g.L[3], (real)g.bc_t);
}

template void launch_dirac<float>(const Geom&, const void*, const float*, const float*, float*, const double*, int,
                                  cudaStream_t);
template void launch_dirac<double>(const Geom&, const void*, const double*, const double*, double*, const double*,
                                   int, cudaStream_t);

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
  pack_kernel<real><<<(unsigned)((total + bs - 1) / bs), bs, 0, st>>>(field, bundle, nsys, nt, g.V);
}

template <typename real>
void launch_unpack(const Geom& g, const real* bundle, real* field, int nsys, cudaStream_t st) {
  int nt = ntiles(nsys, Tile<real>::T);
  int64_t total = (int64_t)nt * 12 * g.V;
  int bs = 256;
  unpack_kernel<real><<<(unsigned)((total + bs - 1) / bs), bs, 0, st>>>(bundle, field, nsys, nt, g.V);
}

template void launch_pack<float>(const Geom&, const float*, float*, int, cudaStream_t);
template void launch_pack<double>(const Geom&, const double*, double*, int, cudaStream_t);
template void launch_unpack<float>(const Geom&, const float*, float*, int, cudaStream_t);
template void launch_unpack<double>(const Geom&, const double*, double*, int, cudaStream_t);

}  // namespace tmamg

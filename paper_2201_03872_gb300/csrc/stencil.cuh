// Device building blocks of the fine twisted-mass Wilson-clover stencil (chiral basis),
// shared by the full-lattice operator (dirac.cu) and the SAP block solver (sap.cu).
#pragma once
#include "common.cuh"

namespace tmamg {

// multiply by one of {+1, -1, +i, -i} encoded as 0, 1, 2, 3
template <int K, typename real>
__device__ __forceinline__ void mulc(real ar, real ai, real& br, real& bi) {
  if (K == 0) { br = ar; bi = ai; }
  if (K == 1) { br = -ar; bi = -ai; }
  if (K == 2) { br = -ai; bi = ar; }
  if (K == 3) { br = ai; bi = -ar; }
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
  static_assert(sizeof(real) * 2 * T == 16 || (sizeof(real) == 4 && T == 1), "one entry is 16 (or 8) bytes");
  if constexpr (sizeof(real) == 4 && T == 1) {  // one system of a shared-memory block layout
    const float2 a = *reinterpret_cast<const float2*>(p);
    v.re[0] = a.x;
    v.im[0] = a.y;
  } else if constexpr (sizeof(real) == 4) {
    float4 a = *reinterpret_cast<const float4*>(p);
    v.re[0] = a.x; v.re[1] = a.y;
    v.im[0] = a.z; v.im[1] = a.w;
  } else {
    double2 a = *reinterpret_cast<const double2*>(p);
    v.re[0] = a.x;
    v.im[0] = a.y;
  }
}

template <typename real, int T>
__device__ __forceinline__ void stcv(real* __restrict__ p, const CV<real, T>& v) {
  if constexpr (sizeof(real) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v.re[0], v.re[1], v.im[0], v.im[1]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(v.re[0], v.im[0]);
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
// xs: neighbour spinor, components strided by cstride entries (V for a bundle in global
// memory, the block volume for a block staged in shared memory); U: links of direction NU
// with site stride V; ls: the site whose link is used.
template <int NU, bool FWD, typename real, int T>
__device__ __forceinline__ void hop(Spinor<real, T>& acc, const real* __restrict__ xs, int64_t cstride,
                                    const typename LinkT<real>::t* __restrict__ U, int64_t V, int64_t ls,
                                    real phase) {
  using P = Proj<NU, FWD>;
  using L2 = typename LinkT<real>::t;
  // half spinor h[a][colour]
  CV<real, T> h[2][3];
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    CV<real, T> u0, u1, d0, d1;
    ldcv(u0, xs + (int64_t)(0 * 3 + col) * cstride * 2 * T);
    ldcv(u1, xs + (int64_t)(1 * 3 + col) * cstride * 2 * T);
    ldcv(d0, xs + (int64_t)(2 * 3 + col) * cstride * 2 * T);
    ldcv(d1, xs + (int64_t)(3 * 3 + col) * cstride * 2 * T);
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

// In place: acc <- A_chi x_chi + i s mu x_chi - 1/2 acc, per chirality chi (s = +1, -1), where
// acc holds the hop sum on entry. A_chi is the packed Hermitian 6x6 clover block with the
// diagonal 1/(2 kappa) folded in (6 real diagonal entries, then the strict lower triangle).
// xs: the site's own spinor, components strided by cstride entries; C: clover with stride V.
template <typename real, int T>
__device__ __forceinline__ void local_term(Spinor<real, T>& acc, const real* __restrict__ x0, int64_t cstride,
                                           const real* __restrict__ C, int64_t V, int64_t s, const real* mu) {
#pragma unroll
  for (int chi = 0; chi < 2; ++chi) {
    const real* Cc = C + (int64_t)chi * 36 * V + s;
    CV<real, T> xc[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) ldcv(xc[i], x0 + (int64_t)(chi * 6 + i) * cstride * 2 * T);
    real sg = chi == 0 ? real(1) : real(-1);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      CV<real, T> o;
      real d = Cc[(int64_t)i * V];
#pragma unroll
      for (int l = 0; l < T; ++l) {
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
      CV<real, T>& hv = acc.c[chi * 6 + i];
#pragma unroll
      for (int l = 0; l < T; ++l) {
        hv.re[l] = o.re[l] - real(0.5) * hv.re[l];
        hv.im[l] = o.im[l] - real(0.5) * hv.im[l];
      }
    }
  }
}

}  // namespace tmamg

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
// xp (optional): the doublet partner's spinor at the same site (same component stride), subtracted
// with the splitting ep: acc <- ... - ep xp (the -eps tau1 term of the non-degenerate doublet)
template <typename real, int T>
__device__ __forceinline__ void local_term(Spinor<real, T>& acc, const real* __restrict__ x0, int64_t cstride,
                                           const real* __restrict__ C, int64_t V, int64_t s, const real* mu,
                                           const real* __restrict__ xp = nullptr, real ep = real(0)) {
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
      if (xp) {
        CV<real, T> pv;
        ldcv(pv, xp + (int64_t)(chi * 6 + i) * cstride * 2 * T);
#pragma unroll
        for (int l = 0; l < T; ++l) {
          o.re[l] -= ep * pv.re[l];
          o.im[l] -= ep * pv.im[l];
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

// ---------------------------------------------------------------- packed FP32 form (T = 2)
// The two systems of an FP32 tile undergo identical arithmetic, so each complex entry is kept
// as (re, im) float2 pairs over the two systems and every operation is one packed FP32x2
// instruction (half the instruction count of the per-lane form above).
namespace tmamg {

struct CV2 {
  float2 re, im;  // (system 0, system 1)
};
struct Spinor2 {
  CV2 c[12];
};

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(f2(-1.f), b, a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ CV2 ld2(const float* __restrict__ p) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  CV2 v;
  v.re = make_float2(a.x, a.y);
  v.im = make_float2(a.z, a.w);
  return v;
}
__device__ __forceinline__ void st2(float* __restrict__ p, const CV2& v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.re.x, v.re.y, v.im.x, v.im.y);
}

// u + K(d) with K one of {+1, -1, +i, -i} (encoded 0..3 as in mulc)
template <int K>
__device__ __forceinline__ CV2 proj2(const CV2& u, const CV2& d) {
  CV2 h;
  if (K == 0) { h.re = add2(u.re, d.re); h.im = add2(u.im, d.im); }
  if (K == 1) { h.re = sub2(u.re, d.re); h.im = sub2(u.im, d.im); }
  if (K == 2) { h.re = sub2(u.re, d.im); h.im = add2(u.im, d.re); }
  if (K == 3) { h.re = add2(u.re, d.im); h.im = sub2(u.im, d.re); }
  return h;
}

// acc += K(g)
template <int K>
__device__ __forceinline__ void acc2(CV2& acc, const CV2& g) {
  if (K == 0) { acc.re = add2(acc.re, g.re); acc.im = add2(acc.im, g.im); }
  if (K == 1) { acc.re = sub2(acc.re, g.re); acc.im = sub2(acc.im, g.im); }
  if (K == 2) { acc.re = sub2(acc.re, g.im); acc.im = add2(acc.im, g.re); }
  if (K == 3) { acc.re = add2(acc.re, g.im); acc.im = sub2(acc.im, g.re); }
}

// hop<> for FP32 tiles of two systems in packed arithmetic (same operands and meaning)
template <int NU, bool FWD>
__device__ __forceinline__ void hop2(Spinor2& acc, const float* __restrict__ xs, int64_t cstride,
                                     const float2* __restrict__ U, int64_t V, int64_t ls, float phase) {
  using P = Proj<NU, FWD>;
  CV2 h[2][3];
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    const CV2 u0 = ld2(xs + (int64_t)(0 * 3 + col) * cstride * 4);
    const CV2 u1 = ld2(xs + (int64_t)(1 * 3 + col) * cstride * 4);
    const CV2 d0 = ld2(xs + (int64_t)(2 * 3 + col) * cstride * 4);
    const CV2 d1 = ld2(xs + (int64_t)(3 * 3 + col) * cstride * 4);
    h[0][col] = proj2<P::c0>(u0, P::p0 == 0 ? d0 : d1);
    h[1][col] = proj2<P::c1>(u1, P::p1 == 0 ? d0 : d1);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float2 w[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (FWD) {
        w[b] = U[(int64_t)(a * 3 + b) * V + ls];
      } else {
        const float2 t = U[(int64_t)(b * 3 + a) * V + ls];
        w[b] = make_float2(t.x, -t.y);
      }
      w[b] = make_float2(w[b].x * phase, w[b].y * phase);  // boundary phase folded into the link
    }
    CV2 g[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      float2 gr = mul2(f2(w[0].x), h[k][0].re);
      float2 gi = mul2(f2(w[0].x), h[k][0].im);
      gr = fma2(f2(-w[0].y), h[k][0].im, gr);
      gi = fma2(f2(w[0].y), h[k][0].re, gi);
#pragma unroll
      for (int b = 1; b < 3; ++b) {
        gr = fma2(f2(w[b].x), h[k][b].re, gr);
        gr = fma2(f2(-w[b].y), h[k][b].im, gr);
        gi = fma2(f2(w[b].x), h[k][b].im, gi);
        gi = fma2(f2(w[b].y), h[k][b].re, gi);
      }
      g[k].re = gr;
      g[k].im = gi;
    }
    acc2<0>(acc.c[0 * 3 + a], g[0]);
    acc2<0>(acc.c[1 * 3 + a], g[1]);
    acc2<P::b0>(acc.c[2 * 3 + a], P::p0 == 0 ? g[0] : g[1]);
    acc2<P::b1>(acc.c[3 * 3 + a], P::p1 == 0 ? g[0] : g[1]);
  }
}

// hop2<> split in three parts so that a caller can keep the next hop's neighbour loads in flight
// while the current hop multiplies: the raw neighbour spinor of one tile (12 entries), its spin
// projection, and the colour multiply with accumulation.
struct Raw2 {
  CV2 v[12];
};
__device__ __forceinline__ void ld_raw2(Raw2& r, const float* __restrict__ xs, int64_t cstride) {
#pragma unroll
  for (int k = 0; k < 12; ++k) r.v[k] = ld2(xs + (int64_t)k * cstride * 4);
}
template <int NU, bool FWD>
__device__ __forceinline__ void proj_raw2(CV2 (&h)[2][3], const Raw2& r) {
  using P = Proj<NU, FWD>;
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    h[0][col] = proj2<P::c0>(r.v[0 * 3 + col], P::p0 == 0 ? r.v[2 * 3 + col] : r.v[3 * 3 + col]);
    h[1][col] = proj2<P::c1>(r.v[1 * 3 + col], P::p1 == 0 ? r.v[2 * 3 + col] : r.v[3 * 3 + col]);
  }
}
template <int NU, bool FWD>
__device__ __forceinline__ void mul_acc2(Spinor2& acc, const CV2 (&h)[2][3], const float2* __restrict__ U, int64_t V,
                                         int64_t ls, float phase) {
  using P = Proj<NU, FWD>;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float2 w[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (FWD) {
        w[b] = U[(int64_t)(a * 3 + b) * V + ls];
      } else {
        const float2 t = U[(int64_t)(b * 3 + a) * V + ls];
        w[b] = make_float2(t.x, -t.y);
      }
      w[b] = make_float2(w[b].x * phase, w[b].y * phase);
    }
    CV2 g[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      float2 gr = mul2(f2(w[0].x), h[k][0].re);
      float2 gi = mul2(f2(w[0].x), h[k][0].im);
      gr = fma2(f2(-w[0].y), h[k][0].im, gr);
      gi = fma2(f2(w[0].y), h[k][0].re, gi);
#pragma unroll
      for (int b = 1; b < 3; ++b) {
        gr = fma2(f2(w[b].x), h[k][b].re, gr);
        gr = fma2(f2(-w[b].y), h[k][b].im, gr);
        gi = fma2(f2(w[b].x), h[k][b].im, gi);
        gi = fma2(f2(w[b].y), h[k][b].re, gi);
      }
      g[k].re = gr;
      g[k].im = gi;
    }
    acc2<0>(acc.c[0 * 3 + a], g[0]);
    acc2<0>(acc.c[1 * 3 + a], g[1]);
    acc2<P::b0>(acc.c[2 * 3 + a], P::p0 == 0 ? g[0] : g[1]);
    acc2<P::b1>(acc.c[3 * 3 + a], P::p1 == 0 ? g[0] : g[1]);
  }
}

// local_term<> for FP32 tiles of two systems in packed arithmetic: acc <- A_chi x_chi +
// i s mu x_chi - 1/2 acc per chirality; mu: the two systems' twisted masses. ep != 0: the tile's two
// systems are the flavours of a non-degenerate doublet, coupled by -ep (each lane gets -ep times
// the other lane's entry)
__device__ __forceinline__ void local2(Spinor2& acc, const float* __restrict__ x0, int64_t cstride,
                                       const float* __restrict__ C, int64_t V, int64_t s, float2 mu,
                                       float ep = 0.f) {
#pragma unroll
  for (int chi = 0; chi < 2; ++chi) {
    const float* Cc = C + (int64_t)chi * 36 * V + s;
    CV2 xc[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) xc[i] = ld2(x0 + (int64_t)(chi * 6 + i) * cstride * 4);
    const float2 smu = chi == 0 ? mu : make_float2(-mu.x, -mu.y);
    const float2 nsmu = make_float2(-smu.x, -smu.y);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const float d = Cc[(int64_t)i * V];
      CV2 o;
      o.re = fma2(f2(d), xc[i].re, mul2(nsmu, xc[i].im));
      o.im = fma2(f2(d), xc[i].im, mul2(smu, xc[i].re));
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        if (j == i) continue;
        float ar, ai;
        if (i > j) {
          const int k = 6 + 2 * (i * (i - 1) / 2 + j);
          ar = Cc[(int64_t)k * V];
          ai = Cc[(int64_t)(k + 1) * V];
        } else {
          const int k = 6 + 2 * (j * (j - 1) / 2 + i);
          ar = Cc[(int64_t)k * V];
          ai = -Cc[(int64_t)(k + 1) * V];
        }
        o.re = fma2(f2(ar), xc[j].re, o.re);
        o.re = fma2(f2(-ai), xc[j].im, o.re);
        o.im = fma2(f2(ar), xc[j].im, o.im);
        o.im = fma2(f2(ai), xc[j].re, o.im);
      }
      if (ep != 0.f) {
        o.re = fma2(f2(-ep), make_float2(xc[i].re.y, xc[i].re.x), o.re);
        o.im = fma2(f2(-ep), make_float2(xc[i].im.y, xc[i].im.x), o.im);
      }
      CV2& hv = acc.c[chi * 6 + i];
      hv.re = fma2(f2(-0.5f), hv.re, o.re);
      hv.im = fma2(f2(-0.5f), hv.im, o.im);
    }
  }
}

}  // namespace tmamg

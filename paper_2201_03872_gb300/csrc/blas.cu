// Batched BLAS-1 on bundles: per-system dots and norms, axpy-type updates, conversions.
//
// A bundle tile holds M = ncomp * nsite entries of 16 bytes, each entry (re[T], im[T]) for
// the T systems of the tile. Reductions are deterministic: a fixed grid of CTAs writes one
// partial per (tile, CTA, vector, lane); a second kernel adds the partials in index order
// (the paper attributes most of the block-solver overhead to global reductions, Sec. 4;
// on one GPU they are on-device two-pass sums with no host involvement).
#include "blas.cuh"
#include "profile.cuh"

namespace tmamg {

constexpr int RED_THREADS = 256;

template <typename real, int T>
struct Ent {
  real re[T], im[T];
};

template <typename real, int T>
__device__ __forceinline__ Ent<real, T> lde(const real* p) {
  Ent<real, T> e;
  if constexpr (sizeof(real) == 4) {
    float4 a = *reinterpret_cast<const float4*>(p);
    e.re[0] = a.x; e.re[1] = a.y; e.im[0] = a.z; e.im[1] = a.w;
  } else {
    double2 a = *reinterpret_cast<const double2*>(p);
    e.re[0] = a.x; e.im[0] = a.y;
  }
  return e;
}

template <typename real, int T>
__device__ __forceinline__ void ste(real* p, const Ent<real, T>& e) {
  if constexpr (sizeof(real) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(e.re[0], e.re[1], e.im[0], e.im[1]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(e.re[0], e.im[0]);
  }
}

// accumulation type: FP32 vectors sum per thread in FP32, CTA and grid sums in FP64
template <typename real>
struct Acc {
  using t = real;
};

// ----------------------------------------------------------------------- multi-dot
// partial[(tile * nblk + blk) * k + i][lane] = sum over the CTA's slice of conj(V_i) w.
// The basis vectors are taken MD_KC at a time: each entry of w is loaded once per group and
// multiplied with the group's vectors, so one call reads w ceil(k / MD_KC) times instead of k
// (MD_KC = 1 for single dots and norms, 4 otherwise; four CTAs per SM either way).
template <typename real, int T, int MD_KC>
__global__ void __launch_bounds__(RED_THREADS, 4) mdot_partial_kernel(const real* __restrict__ Vb, int64_t vstride, int k,
                                                                   const real* __restrict__ w, int64_t M,
                                                                   double2* __restrict__ partial) {
  const int tile = blockIdx.y;
  const int nblk = gridDim.x;
  const int64_t toff = (int64_t)tile * M * 2 * T;
  __shared__ double2 red[RED_THREADS / 32][MD_KC][T];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const real* ww = w + toff;
  for (int i0 = 0; i0 < k; i0 += MD_KC) {
    const int kn = k - i0 < MD_KC ? k - i0 : MD_KC;
    real sr[MD_KC][T], si[MD_KC][T];
#pragma unroll
    for (int u = 0; u < MD_KC; ++u)
#pragma unroll
      for (int l = 0; l < T; ++l) { sr[u][l] = 0; si[u][l] = 0; }
    for (int64_t m = blockIdx.x * (int64_t)RED_THREADS + threadIdx.x; m < M; m += (int64_t)nblk * RED_THREADS) {
      const Ent<real, T> b = lde<real, T>(ww + m * 2 * T);
#pragma unroll
      for (int u = 0; u < MD_KC; ++u) {
        if (u < kn) {
          const Ent<real, T> a = lde<real, T>(Vb + (int64_t)(i0 + u) * vstride + toff + m * 2 * T);
#pragma unroll
          for (int l = 0; l < T; ++l) {
            sr[u][l] += a.re[l] * b.re[l] + a.im[l] * b.im[l];
            si[u][l] += a.re[l] * b.im[l] - a.im[l] * b.re[l];
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < MD_KC; ++u) {
      if (u < kn) {
#pragma unroll
        for (int l = 0; l < T; ++l) {
          double dr = sr[u][l], di = si[u][l];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            dr += __shfl_xor_sync(0xffffffffu, dr, o);
            di += __shfl_xor_sync(0xffffffffu, di, o);
          }
          if (lane == 0) red[warp][u][l] = make_double2(dr, di);
        }
      }
    }
    __syncthreads();
    if (threadIdx.x < kn * T) {
      const int u = threadIdx.x / T, l = threadIdx.x % T;
      double2 s = make_double2(0, 0);
      for (int q = 0; q < RED_THREADS / 32; ++q) {
        s.x += red[q][u][l].x;
        s.y += red[q][u][l].y;
      }
      partial[(((int64_t)tile * nblk + blockIdx.x) * k + i0 + u) * T + l] = s;
    }
    __syncthreads();
  }
}

// out[i * ostride + n] = sum_blk partial  (system n = tile * T + lane), n < nsys
template <int T>
__global__ void mdot_final_kernel(const double2* __restrict__ partial, int nblk, int k, int nsys, double2* out,
                                  int64_t ostride, double scale) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nsys * k) return;
  int n = t % nsys, i = t / nsys;
  int tile = n / T, lane = n % T;
  double2 s = make_double2(0, 0);
  for (int b = 0; b < nblk; ++b) {
    double2 p = partial[(((int64_t)tile * nblk + b) * k + i) * T + lane];
    s.x += p.x;
    s.y += p.y;
  }
  out[i * ostride + n] = make_double2(s.x * scale, s.y * scale);
}

static thread_local bool t_pair_fold = false;
void set_pair_fold(bool on) { t_pair_fold = on; }

// out[i * ostride + 2p] = out[i * ostride + 2p + 1] = their sum, p < npair, i < k
__global__ void pair_fold_kernel(double2* out, int64_t ostride, int k, int npair) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k * npair) return;
  const int i = t / npair, p = t % npair;
  double2* o = out + (int64_t)i * ostride + 2 * p;
  const double2 s = make_double2(o[0].x + o[1].x, o[0].y + o[1].y);
  o[0] = s;
  o[1] = s;
}

static int red_blocks(int64_t M, int ntile) {
  // about 4 CTAs per SM in total, at least one per tile
  int64_t want = (152 * 4 + ntile - 1) / ntile;
  int64_t maxb = (M + RED_THREADS - 1) / RED_THREADS;
  int64_t b = want < maxb ? want : maxb;
  return (int)(b < 1 ? 1 : b);
}

template <typename real>
void mdot(const real* V, int64_t vstride, int k, const real* w, int64_t M, int nsys, double2* out, int64_t ostride,
          double2* partial, cudaStream_t st) {
  TM_PROF(st, "mdot");
  constexpr int T = Tile<real>::T;
  int nt = ntiles(nsys, T);
  int nblk = red_blocks(M, nt);
  if (k == 1)
    mdot_partial_kernel<real, T, 1><<<dim3(nblk, nt), RED_THREADS, 0, st>>>(V, vstride, k, w, M, partial);
  else
    mdot_partial_kernel<real, T, 4><<<dim3(nblk, nt), RED_THREADS, 0, st>>>(V, vstride, k, w, M, partial);
  TM_COUNT();
  int tot = nsys * k;
  mdot_final_kernel<T><<<(tot + 127) / 128, 128, 0, st>>>(partial, nblk, k, nsys, out, ostride, 1.0); TM_COUNT();
  if (t_pair_fold) {
    const int np = nsys / 2;
    pair_fold_kernel<<<(k * np + 127) / 128, 128, 0, st>>>(out, ostride, k, np); TM_COUNT();
  }
}

size_t partial_elems(int64_t M, int nsys, int kmax, int T) {
  int nt = ntiles(nsys, T);
  return (size_t)nt * red_blocks(M, nt) * kmax * T;
}

// ----------------------------------------------------------------------- updates
// y[n] = y[n] - sum_i c[i * cstride + n] * V_i[n]   (c complex double per system);
// with sign = +1 it adds instead. Inactive systems (mask[n] == 0) are left unchanged.
// The coefficients of the block's tile are converted once into shared memory (k <= MAXPY_K);
// the basis loop is unrolled so that several vector loads are in flight per thread.
constexpr int MAXPY_K = 128;

template <typename real, int T>
__global__ void maxpy_kernel(const real* __restrict__ Vb, int64_t vstride, int k, const double2* __restrict__ c,
                             int64_t cstride, real sign, real* __restrict__ y, int64_t M, int nsys,
                             const int* __restrict__ mask) {
  __shared__ real cre[MAXPY_K][T], cim[MAXPY_K][T];
  const int tile = blockIdx.y;
  const int64_t toff = (int64_t)tile * M * 2 * T;
  for (int q = threadIdx.x; q < k * T; q += blockDim.x) {
    const int i = q / T, l = q % T;
    const int n = tile * T + l;
    const bool on = n < nsys && (!mask || mask[n]);
    const double2 cc = on ? c[i * cstride + n] : make_double2(0, 0);
    cre[i][l] = (real)cc.x * sign;
    cim[i][l] = (real)cc.y * sign;
  }
  __syncthreads();
  int64_t m0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t m = m0; m < M; m += (int64_t)gridDim.x * blockDim.x) {
    Ent<real, T> acc = lde<real, T>(y + toff + m * 2 * T);
    const real* vp = Vb + toff + m * 2 * T;
#pragma unroll 4
    for (int i = 0; i < k; ++i) {
      const Ent<real, T> v = lde<real, T>(vp + i * vstride);
#pragma unroll
      for (int l = 0; l < T; ++l) {
        acc.re[l] += cre[i][l] * v.re[l] - cim[i][l] * v.im[l];
        acc.im[l] += cre[i][l] * v.im[l] + cim[i][l] * v.re[l];
      }
    }
    ste<real, T>(y + toff + m * 2 * T, acc);
  }
}

// the same for k > MAXPY_K: coefficients read from global memory
template <typename real, int T>
__global__ void maxpy_long_kernel(const real* __restrict__ Vb, int64_t vstride, int k, const double2* __restrict__ c,
                                  int64_t cstride, real sign, real* __restrict__ y, int64_t M, int nsys,
                                  const int* __restrict__ mask) {
  const int tile = blockIdx.y;
  const int64_t toff = (int64_t)tile * M * 2 * T;
  int64_t m0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t m = m0; m < M; m += (int64_t)gridDim.x * blockDim.x) {
    Ent<real, T> acc = lde<real, T>(y + toff + m * 2 * T);
    for (int i = 0; i < k; ++i) {
      const Ent<real, T> v = lde<real, T>(Vb + i * vstride + toff + m * 2 * T);
#pragma unroll
      for (int l = 0; l < T; ++l) {
        const int n = tile * T + l;
        const bool on = n < nsys && (!mask || mask[n]);
        const double2 cc = on ? c[i * cstride + n] : make_double2(0, 0);
        const real cr = (real)cc.x * sign, ci = (real)cc.y * sign;
        acc.re[l] += cr * v.re[l] - ci * v.im[l];
        acc.im[l] += cr * v.im[l] + ci * v.re[l];
      }
    }
    ste<real, T>(y + toff + m * 2 * T, acc);
  }
}

static dim3 upd_grid(int64_t M, int nt, int bs) {
  int64_t want = (152 * 8 + nt - 1) / nt;
  int64_t maxb = (M + bs - 1) / bs;
  int64_t b = want < maxb ? want : maxb;
  return dim3((unsigned)(b < 1 ? 1 : b), nt);
}

template <typename real>
void maxpy(const real* V, int64_t vstride, int k, const double2* c, int64_t cstride, double sign, real* y, int64_t M,
           int nsys, const int* mask, cudaStream_t st) {
  TM_PROF(st, "maxpy");
  constexpr int T = Tile<real>::T;
  int nt = ntiles(nsys, T);
  if (k <= MAXPY_K)
    maxpy_kernel<real, T><<<upd_grid(M, nt, 256), 256, 0, st>>>(V, vstride, k, c, cstride, (real)sign, y, M, nsys,
                                                                 mask);
  else
    maxpy_long_kernel<real, T><<<upd_grid(M, nt, 256), 256, 0, st>>>(V, vstride, k, c, cstride, (real)sign, y, M,
                                                                      nsys, mask);
  TM_COUNT();
}

// y[n] = a[n] * x[n] + b[n] * y[n]; a, b complex per system (nullptr a => 0, nullptr b => y ignored,
// i.e. y = a x). Masked systems keep y.
template <typename real, int T>
__global__ void axpby_kernel(const double2* __restrict__ a, const real* __restrict__ x, const double2* __restrict__ b,
                             real* __restrict__ y, int64_t M, int nsys, const int* __restrict__ mask, int amode,
                             int bmode) {
  const int tile = blockIdx.y;
  const int64_t toff = (int64_t)tile * M * 2 * T;
  real ar[T], ai[T], br[T], bi[T];
  bool on[T];
#pragma unroll
  for (int l = 0; l < T; ++l) {
    int n = tile * T + l;
    on[l] = n < nsys && (!mask || mask[n]);
    double2 av = amode == 0 ? make_double2(0, 0) : (amode == 1 ? make_double2(1, 0) : a[n < nsys ? n : 0]);
    double2 bv = bmode == 0 ? make_double2(0, 0) : (bmode == 1 ? make_double2(1, 0) : b[n < nsys ? n : 0]);
    ar[l] = (real)av.x; ai[l] = (real)av.y;
    br[l] = (real)bv.x; bi[l] = (real)bv.y;
  }
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
    Ent<real, T> yy = lde<real, T>(y + toff + m * 2 * T);
    Ent<real, T> xx;
    if (amode) xx = lde<real, T>(x + toff + m * 2 * T);
    Ent<real, T> o;
#pragma unroll
    for (int l = 0; l < T; ++l) {
      real r = 0, i = 0;
      if (bmode) {
        r = br[l] * yy.re[l] - bi[l] * yy.im[l];
        i = br[l] * yy.im[l] + bi[l] * yy.re[l];
      }
      if (amode) {
        r += ar[l] * xx.re[l] - ai[l] * xx.im[l];
        i += ar[l] * xx.im[l] + ai[l] * xx.re[l];
      }
      o.re[l] = on[l] ? r : yy.re[l];
      o.im[l] = on[l] ? i : yy.im[l];
    }
    ste<real, T>(y + toff + m * 2 * T, o);
  }
}

template <typename real>
void axpby(const double2* a, int amode, const real* x, const double2* b, int bmode, real* y, int64_t M, int nsys,
           const int* mask, cudaStream_t st) {
  TM_PROF(st, "axpby");
  constexpr int T = Tile<real>::T;
  int nt = ntiles(nsys, T);
  axpby_kernel<real, T><<<upd_grid(M, nt, 256), 256, 0, st>>>(a, x, b, y, M, nsys, mask, amode, bmode); TM_COUNT();
}

// ----------------------------------------------------------------------- FP64 <-> FP32
// x32[n] = s[n] * x64[n]   (s real per system, from a device array; s == nullptr => 1)
__global__ void f64_to_f32_kernel(const double* __restrict__ x64, const double* __restrict__ s,
                                  float* __restrict__ x32, int64_t M, int nsys) {
  int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int tile = blockIdx.y;  // FP32 tile: systems 2 tile, 2 tile + 1
  if (m >= M) return;
  float o[4];
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    int n = tile * 2 + l;
    double re = 0, im = 0;
    if (n < nsys) {
      double2 v = *reinterpret_cast<const double2*>(x64 + ((int64_t)n * M + m) * 2);
      double sc = s ? s[n] : 1.0;
      re = v.x * sc;
      im = v.y * sc;
    }
    o[l] = (float)re;
    o[2 + l] = (float)im;
  }
  *reinterpret_cast<float4*>(x32 + ((int64_t)tile * M + m) * 4) = make_float4(o[0], o[1], o[2], o[3]);
}

void f64_to_f32(const double* x64, const double* s, float* x32, int64_t M, int nsys, cudaStream_t st) {
  TM_PROF(st, "f64_to_f32");
  int nt = ntiles(nsys, 2);
  f64_to_f32_kernel<<<dim3((unsigned)((M + 255) / 256), nt), 256, 0, st>>>(x64, s, x32, M, nsys); TM_COUNT();
}

// x64[n] += s[n] * x32[n]  for active systems
__global__ void f32_axpy_f64_kernel(const double* __restrict__ s, const float* __restrict__ x32,
                                    double* __restrict__ x64, int64_t M, int nsys, const int* __restrict__ mask) {
  int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int n = blockIdx.y;
  if (m >= M || n >= nsys) return;
  if (mask && !mask[n]) return;
  int tile = n / 2, l = n % 2;
  float4 v = *reinterpret_cast<const float4*>(x32 + ((int64_t)tile * M + m) * 4);
  float re = l ? v.y : v.x, im = l ? v.w : v.z;
  double2* p = reinterpret_cast<double2*>(x64 + ((int64_t)n * M + m) * 2);
  double2 o = *p;
  double sc = s[n];
  o.x += sc * (double)re;
  o.y += sc * (double)im;
  *p = o;
}

void f32_axpy_f64(const double* s, const float* x32, double* x64, int64_t M, int nsys, const int* mask,
                  cudaStream_t st) {
  TM_PROF(st, "f32_axpy_f64");
  f32_axpy_f64_kernel<<<dim3((unsigned)((M + 255) / 256), nsys), 256, 0, st>>>(s, x32, x64, M, nsys, mask); TM_COUNT();
}

// ----------------------------------------------------------------------- explicit instantiations
template void mdot<float>(const float*, int64_t, int, const float*, int64_t, int, double2*, int64_t, double2*,
                          cudaStream_t);
template void mdot<double>(const double*, int64_t, int, const double*, int64_t, int, double2*, int64_t, double2*,
                           cudaStream_t);
template void maxpy<float>(const float*, int64_t, int, const double2*, int64_t, double, float*, int64_t, int,
                           const int*, cudaStream_t);
template void maxpy<double>(const double*, int64_t, int, const double2*, int64_t, double, double*, int64_t, int,
                            const int*, cudaStream_t);
template void axpby<float>(const double2*, int, const float*, const double2*, int, float*, int64_t, int, const int*,
                           cudaStream_t);
template void axpby<double>(const double2*, int, const double*, const double2*, int, double*, int64_t, int,
                            const int*, cudaStream_t);

}  // namespace tmamg

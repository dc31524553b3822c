// Learned preconditioner step: a gauge-covariant parallel-transport network (three linear
// layers, 4 -> 8 -> 8 -> 4 complex channels of colour 3-vectors) with forward, backward and
// Adam kernels. Not part of the paper's method; it is an extra fine-level step inside the
// AMG cycle that is trained on (residual, error) pairs produced by the plain solver and is
// switched off when it does not help.
//
// A layer: out_a(x) = sum_h sum_b W_h[a][b] (T_h in_b)(x), h = 0 (identity) and the eight
// hops T_{+nu} in(x) = U_nu(x) in(x + nu), T_{-nu} in(x) = U_nu(x - nu)^+ in(x - nu) (with the
// fermion boundary phase). Activations are FP32 bundles with ncomp = channels x 3 (channel
// major, colour fastest), so the 12-component residual is the 4-channel input. Weights are
// kept in FP32 for training; the inference copy is BF16 (converted to FP32 in shared memory),
// accumulation is FP32.
#include <cuda_bf16.h>

#include <cmath>

#include "blas.cuh"
#include "nn.cuh"

namespace tmamg {

constexpr int NN_T = 2;  // FP32 tile width

struct F2x2 {  // one complex entry of the two systems of a tile
  float re[2], im[2];
};

__device__ __forceinline__ F2x2 nld(const float* p) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  F2x2 v;
  v.re[0] = a.x; v.re[1] = a.y; v.im[0] = a.z; v.im[1] = a.w;
  return v;
}
__device__ __forceinline__ void nst(float* p, const F2x2& v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.re[0], v.re[1], v.im[0], v.im[1]);
}

// link of hop h at site s (h > 0): U_nu(s) for a forward hop, U_nu(s - nu)^+ for a backward hop;
// also returns the neighbour site and the boundary phase
__device__ __forceinline__ void hop_link(const float2* __restrict__ U, const int* L, int64_t V, int64_t s,
                                         const int* c, int h, int bc_t, float2* w, int64_t& nb, float& ph) {
  const int nu = (h - 1) / 2;
  const bool fwd = ((h - 1) & 1) == 0;
  int64_t stride = 1;
  for (int d = 0; d < nu; ++d) stride *= L[d];
  if (fwd) {
    nb = c[nu] + 1 < L[nu] ? s + stride : s - (int64_t)(L[nu] - 1) * stride;
    ph = (nu == 3 && c[3] == L[3] - 1) ? (float)bc_t : 1.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) w[k] = U[((int64_t)nu * 9 + k) * V + s];
  } else {
    nb = c[nu] > 0 ? s - stride : s + (int64_t)(L[nu] - 1) * stride;
    ph = (nu == 3 && c[3] == 0) ? (float)bc_t : 1.f;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float2 t = U[((int64_t)nu * 9 + b * 3 + a) * V + nb];
        w[a * 3 + b] = make_float2(t.x, -t.y);
      }
  }
}

// z = ph * w x for a colour 3-vector x of two systems
__device__ __forceinline__ void transport3(const float2* w, float ph, const F2x2* x, F2x2* z) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      float zr = 0, zi = 0;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        zr += w[a * 3 + b].x * x[b].re[l] - w[a * 3 + b].y * x[b].im[l];
        zi += w[a * 3 + b].x * x[b].im[l] + w[a * 3 + b].y * x[b].re[l];
      }
      z[a].re[l] = ph * zr;
      z[a].im[l] = ph * zi;
    }
}

// y = sum_h W_h T_h x ; W: [9][COUT][CIN] complex (float2) in global memory
template <int CIN, int COUT>
__global__ void __launch_bounds__(128) nn_layer_kernel(const float2* __restrict__ U, const float* __restrict__ x,
                                                       const float2* __restrict__ W, float* __restrict__ y, int ntile,
                                                       NNGeom g) {
  __shared__ float2 Ws[9 * COUT * CIN];
  for (int q = threadIdx.x; q < 9 * COUT * CIN; q += blockDim.x) Ws[q] = W[q];
  __syncthreads();
  const int64_t V = g.V;
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int tile = blockIdx.y;
  if (s >= V || tile >= ntile) return;
  int c[4];
  site_coords(s, g.L, c);
  const float* xt = x + (int64_t)tile * CIN * 3 * V * 4;
  F2x2 acc[COUT][3];
#pragma unroll
  for (int a = 0; a < COUT; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = 0; l < 2; ++l) { acc[a][k].re[l] = 0; acc[a][k].im[l] = 0; }
  for (int h = 0; h < 9; ++h) {
    float2 w[9];
    int64_t nb = s;
    float ph = 1.f;
    if (h > 0) hop_link(U, g.L, V, s, c, h, g.bc_t, w, nb, ph);
    for (int b = 0; b < CIN; ++b) {
      F2x2 xv[3], z[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) xv[k] = nld(xt + ((int64_t)(b * 3 + k) * V + nb) * 4);
      if (h > 0) {
        transport3(w, ph, xv, z);
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) z[k] = xv[k];
      }
#pragma unroll
      for (int a = 0; a < COUT; ++a) {
        const float2 m = Ws[(h * COUT + a) * CIN + b];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int l = 0; l < 2; ++l) {
            acc[a][k].re[l] += m.x * z[k].re[l] - m.y * z[k].im[l];
            acc[a][k].im[l] += m.x * z[k].im[l] + m.y * z[k].re[l];
          }
      }
    }
  }
  float* yt = y + (int64_t)tile * COUT * 3 * V * 4;
#pragma unroll
  for (int a = 0; a < COUT; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k) nst(yt + ((int64_t)(a * 3 + k) * V + s) * 4, acc[a][k]);
}

// grad W_h[a][b] partials: sum over the CTA's sites, both lanes and colours of g_a conj((T_h x)_b);
// grid (site chunks, 9 hops, tiles), one thread per site; a warp reduction per (a, b).
template <int CIN, int COUT>
__global__ void __launch_bounds__(128) nn_wgrad_kernel(const float2* __restrict__ U, const float* __restrict__ x,
                                                       const float* __restrict__ gy, double2* __restrict__ part,
                                                       int ntile, int nsys, NNGeom g) {
  __shared__ double2 red[4][COUT * CIN];
  const int64_t V = g.V;
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int h = blockIdx.y;
  const int tile = blockIdx.z;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool on = s < V;
  F2x2 z[CIN][3], gv[COUT][3];
  const bool l1 = tile * 2 + 1 < nsys;  // padding lane of the last tile carries zeros anyway
  (void)l1;
  if (on) {
    int c[4];
    site_coords(s, g.L, c);
    float2 w[9];
    int64_t nb = s;
    float ph = 1.f;
    if (h > 0) hop_link(U, g.L, V, s, c, h, g.bc_t, w, nb, ph);
    const float* xt = x + (int64_t)tile * CIN * 3 * V * 4;
    const float* gt = gy + (int64_t)tile * COUT * 3 * V * 4;
#pragma unroll
    for (int b = 0; b < CIN; ++b) {
      F2x2 xv[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) xv[k] = nld(xt + ((int64_t)(b * 3 + k) * V + nb) * 4);
      if (h > 0) {
        transport3(w, ph, xv, z[b]);
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) z[b][k] = xv[k];
      }
    }
#pragma unroll
    for (int a = 0; a < COUT; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) gv[a][k] = nld(gt + ((int64_t)(a * 3 + k) * V + s) * 4);
  } else {
#pragma unroll
    for (int b = 0; b < CIN; ++b)
#pragma unroll
      for (int k = 0; k < 3; ++k) z[b][k] = F2x2{{0, 0}, {0, 0}};
#pragma unroll
    for (int a = 0; a < COUT; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) gv[a][k] = F2x2{{0, 0}, {0, 0}};
  }
#pragma unroll
  for (int a = 0; a < COUT; ++a)
#pragma unroll
    for (int b = 0; b < CIN; ++b) {
      float sr = 0, si = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 2; ++l) {  // g conj(z)
          sr += gv[a][k].re[l] * z[b][k].re[l] + gv[a][k].im[l] * z[b][k].im[l];
          si += gv[a][k].im[l] * z[b][k].re[l] - gv[a][k].re[l] * z[b][k].im[l];
        }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
      }
      if (lane == 0) red[warp][a * CIN + b] = make_double2(sr, si);
    }
  __syncthreads();
  for (int q = threadIdx.x; q < COUT * CIN; q += blockDim.x) {
    double2 t = make_double2(0, 0);
    for (int w2 = 0; w2 < 4; ++w2) {
      t.x += red[w2][q].x;
      t.y += red[w2][q].y;
    }
    const int64_t blk = ((int64_t)tile * gridDim.y + h) * gridDim.x + blockIdx.x;
    part[blk * COUT * CIN + q] = t;
  }
}

// grad W[h][q] = sum over site chunks and tiles of the partials (fixed order)
__global__ void nn_wgrad_final_kernel(const double2* __restrict__ part, int nchunk, int ntile, int nq,
                                      double2* __restrict__ grad) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 9 * nq) return;
  const int h = t / nq, q = t % nq;
  double2 s = make_double2(0, 0);
  for (int tile = 0; tile < ntile; ++tile)
    for (int c = 0; c < nchunk; ++c) {
      const double2 v = part[(((int64_t)tile * 9 + h) * nchunk + c) * nq + q];
      s.x += v.x;
      s.y += v.y;
    }
  grad[t] = s;
}

// adjoint weights for the input-gradient pass: Wa_k = (W_opp(k))^+, [9][CIN][COUT]
__global__ void nn_adjoint_weights_kernel(const float2* __restrict__ W, float2* __restrict__ Wa, int cin, int cout) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 9 * cin * cout) return;
  const int k = t / (cin * cout), r = t % (cin * cout);
  const int b = r / cout, a = r % cout;  // Wa[k][b][a]
  const int ho = k == 0 ? 0 : ((k % 2 == 1) ? k + 1 : k - 1);
  const float2 v = W[((int64_t)ho * cout + a) * cin + b];
  Wa[t] = make_float2(v.x, -v.y);
}

// Adam on 2 n reals (complex parameters as pairs): p -= lr mhat / (sqrt(vhat) + eps)
__global__ void nn_adam_kernel(float* __restrict__ p, const double* __restrict__ grad, float* __restrict__ m1,
                               float* __restrict__ m2, int n2, float lr, float b1, float b2, float eps, int step,
                               double gscale) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n2) return;
  const float gr = (float)(grad[t] * gscale);
  const float a = b1 * m1[t] + (1 - b1) * gr;
  const float b = b2 * m2[t] + (1 - b2) * gr * gr;
  m1[t] = a;
  m2[t] = b;
  const float ah = a / (1 - powf(b1, (float)step));
  const float bh = b / (1 - powf(b2, (float)step));
  p[t] -= lr * ah / (sqrtf(bh) + eps);
}

__global__ void nn_to_bf16_kernel(const float2* __restrict__ W, __nv_bfloat162* __restrict__ Wb, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) Wb[t] = __floats2bfloat162_rn(W[t].x, W[t].y);
}

__global__ void nn_from_bf16_kernel(const __nv_bfloat162* __restrict__ Wb, float2* __restrict__ W, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) W[t] = __bfloat1622float2(Wb[t]);
}

// ---------------------------------------------------------------- host side
static const int CH[4] = {4, 8, 8, 4};

int nn_weight_count(int layer) { return 9 * CH[layer] * CH[layer + 1]; }
int nn_weight_offset(int layer) {
  int o = 0;
  for (int l = 0; l < layer; ++l) o += nn_weight_count(l);
  return o;
}

static void layer_fwd(const NNGeom& g, const float2* U, const float* x, const float2* W, float* y, int cin, int cout,
                      int ntile, cudaStream_t st) {
  dim3 grid((unsigned)((g.V + 127) / 128), ntile);
  if (cin == 4 && cout == 8) nn_layer_kernel<4, 8><<<grid, 128, 0, st>>>(U, x, W, y, ntile, g);
  else if (cin == 8 && cout == 8) nn_layer_kernel<8, 8><<<grid, 128, 0, st>>>(U, x, W, y, ntile, g);
  else if (cin == 8 && cout == 4) nn_layer_kernel<8, 4><<<grid, 128, 0, st>>>(U, x, W, y, ntile, g);
  else nn_layer_kernel<4, 4><<<grid, 128, 0, st>>>(U, x, W, y, ntile, g);
  TM_COUNT();
}

static void layer_wgrad(const NNGeom& g, const float2* U, const float* x, const float* gy, double2* part, int cin,
                        int cout, int ntile, int nsys, double2* grad, cudaStream_t st) {
  const int nchunk = (int)((g.V + 127) / 128);
  dim3 grid(nchunk, 9, ntile);
  if (cin == 4 && cout == 8) nn_wgrad_kernel<4, 8><<<grid, 128, 0, st>>>(U, x, gy, part, ntile, nsys, g);
  else if (cin == 8 && cout == 8) nn_wgrad_kernel<8, 8><<<grid, 128, 0, st>>>(U, x, gy, part, ntile, nsys, g);
  else nn_wgrad_kernel<8, 4><<<grid, 128, 0, st>>>(U, x, gy, part, ntile, nsys, g);
  TM_COUNT();
  const int nq = cin * cout;
  nn_wgrad_final_kernel<<<(9 * nq + 127) / 128, 128, 0, st>>>(part, nchunk, ntile, nq, grad);
  TM_COUNT();
}

int NNState::alloc(int64_t V, int nsys_) {
  if (V <= Vcap && nsys_ <= nsys) return 0;
  release_buffers();
  Vcap = V;
  nsys = nsys_;
  const int nt = ntiles(nsys, NN_T);
  cudaError_t e = cudaSuccess;
  auto A = [&](void** q, size_t b) {
    if (e == cudaSuccess) e = cudaMalloc(q, b);
  };
  const size_t per_ch = (size_t)nt * 3 * V * 4 * sizeof(float);  // one channel of a bundle
  for (int l = 0; l < 4; ++l) A((void**)&act[l], per_ch * CH[l]);
  A((void**)&gbuf[0], per_ch * 8);
  A((void**)&gbuf[1], per_ch * 8);
  const int nchunk = (int)((V + 127) / 128);
  A((void**)&part, sizeof(double2) * (size_t)nt * 9 * nchunk * 64);
  return e == cudaSuccess ? 0 : -1;
}

int NNState::alloc_weights() {
  if (W) return 0;
  const int n = nn_weight_offset(3);
  cudaError_t e = cudaSuccess;
  auto A = [&](void** q, size_t b) {
    if (e == cudaSuccess) e = cudaMalloc(q, b);
  };
  A((void**)&W, sizeof(float2) * n);
  A((void**)&Winf, sizeof(float2) * n);
  A((void**)&Wb16, sizeof(__nv_bfloat162) * n);
  A((void**)&Wadj, sizeof(float2) * 9 * 64);
  A((void**)&grad, sizeof(double2) * n);
  A((void**)&m1, sizeof(float2) * n);
  A((void**)&m2, sizeof(float2) * n);
  A((void**)&enorm, sizeof(double2) * 256);
  A((void**)&coef, sizeof(double2) * 512);
  if (e == cudaSuccess) {
    cudaMemset(m1, 0, sizeof(float2) * n);
    cudaMemset(m2, 0, sizeof(float2) * n);
  }
  return e == cudaSuccess ? 0 : -1;
}

void NNState::release_buffers() {
  for (int l = 0; l < 4; ++l) {
    cudaFree(act[l]);
    act[l] = nullptr;
  }
  cudaFree(gbuf[0]);
  cudaFree(gbuf[1]);
  cudaFree(part);
  gbuf[0] = gbuf[1] = nullptr;
  part = nullptr;
  Vcap = 0;
  nsys = 0;
}

void NNState::release() {
  release_buffers();
  void* ptrs[] = {W, Winf, Wb16, Wadj, grad, m1, m2, enorm, coef};
  for (void* q : ptrs) cudaFree(q);
  W = Winf = Wadj = nullptr;
  Wb16 = nullptr;
  grad = enorm = coef = nullptr;
  m1 = m2 = nullptr;
  trained = false;
}

// inference weights: BF16 copy of the FP32 master weights, expanded back to FP32 for the kernels
void nn_refresh_inference(NNState& s, cudaStream_t st) {
  const int n = nn_weight_offset(3);
  nn_to_bf16_kernel<<<(n + 255) / 256, 256, 0, st>>>(s.W, (__nv_bfloat162*)s.Wb16, n);
  TM_COUNT();
  nn_from_bf16_kernel<<<(n + 255) / 256, 256, 0, st>>>((const __nv_bfloat162*)s.Wb16, s.Winf, n);
  TM_COUNT();
}

void nn_forward(NNState& s, const NNGeom& g, const float2* U, const float* r, float* y, int nsys, bool inference,
                cudaStream_t st) {
  const int nt = ntiles(nsys, NN_T);
  const float2* Wset = inference ? s.Winf : s.W;
  layer_fwd(g, U, r, Wset + nn_weight_offset(0), s.act[1], 4, 8, nt, st);
  layer_fwd(g, U, s.act[1], Wset + nn_weight_offset(1), s.act[2], 8, 8, nt, st);
  layer_fwd(g, U, s.act[2], Wset + nn_weight_offset(2), y, 8, 4, nt, st);
}

// loss gradient g3 = 2 (y - e) / |e|^2 per system, then backpropagation; grads in s.grad
void nn_backward(NNState& s, const NNGeom& g, const float2* U, const float* r, const float* y, const float* e,
                 int nsys, double2* partial, cudaStream_t st) {
  const int nt = ntiles(nsys, NN_T);
  const int64_t M4 = 12 * g.V;
  // |e|^2 per system -> coefficients a = 2/|e|^2 (on y), b = -2/|e|^2 (on e)
  mdot<float>(e, 0, 1, e, M4, nsys, s.enorm, nsys, partial, st);
  nn_loss_coef(s.enorm, s.coef, nsys, st);
  float* g3 = s.gbuf[0];
  cudaMemcpyAsync(g3, e, (size_t)nt * 12 * g.V * 4 * sizeof(float), cudaMemcpyDeviceToDevice, st);
  axpby<float>(s.coef, 2, y, s.coef + 256, 2, g3, M4, nsys, nullptr, st);
  // layer 3 (8 -> 4): weight gradient, then input gradient via the adjoint weights
  layer_wgrad(g, U, s.act[2], g3, s.part, 8, 4, nt, nsys, s.grad + nn_weight_offset(2), st);
  nn_adjoint_weights_kernel<<<(9 * 32 + 127) / 128, 128, 0, st>>>(s.W + nn_weight_offset(2), s.Wadj, 8, 4);
  TM_COUNT();
  float* g2 = s.gbuf[1];
  layer_fwd(g, U, g3, s.Wadj, g2, 4, 8, nt, st);
  // layer 2 (8 -> 8)
  layer_wgrad(g, U, s.act[1], g2, s.part, 8, 8, nt, nsys, s.grad + nn_weight_offset(1), st);
  nn_adjoint_weights_kernel<<<(9 * 64 + 127) / 128, 128, 0, st>>>(s.W + nn_weight_offset(1), s.Wadj, 8, 8);
  TM_COUNT();
  float* g1 = s.gbuf[0];
  layer_fwd(g, U, g2, s.Wadj, g1, 8, 8, nt, st);
  // layer 1 (4 -> 8): weight gradient only
  layer_wgrad(g, U, r, g1, s.part, 4, 8, nt, nsys, s.grad + nn_weight_offset(0), st);
}

__global__ void nn_loss_coef_kernel(const double2* __restrict__ en, double2* __restrict__ coef, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double v = en[t].x > 0 ? 2.0 / en[t].x : 0.0;
  coef[t] = make_double2(v, 0);
  coef[256 + t] = make_double2(-v, 0);
}

void nn_loss_coef(const double2* enorm, double2* coef, int nsys, cudaStream_t st) {
  nn_loss_coef_kernel<<<(nsys + 127) / 128, 128, 0, st>>>(enorm, coef, nsys);
  TM_COUNT();
}

void nn_adam(NNState& s, float lr, int step, double gscale, cudaStream_t st) {
  const int n2 = 2 * nn_weight_offset(3);
  nn_adam_kernel<<<(n2 + 255) / 256, 256, 0, st>>>((float*)s.W, (const double*)s.grad, (float*)s.m1, (float*)s.m2, n2,
                                                   lr, 0.9f, 0.999f, 1e-8f, step, gscale);
  TM_COUNT();
}

}  // namespace tmamg

// Block GMRES on the coarse lattice: one block per twisted mass, over that shift's
// right-hand sides (paper Sec. 4: block Krylov solvers at the coarsest level build one
// Krylov space for a block of right-hand sides; classical Gram-Schmidt without
// re-orthogonalisation performed best; inexact breakdown is not used).
//
// Systems n = r * nshift + k belong to block k (s = nrhs systems). For every block:
//   R0 = B - A X, V_0 S_0 = R0 (CholQR applied twice)
//   step j: W = A V_j;  H_ij = V_i^+ W (i <= j);  W -= sum_i V_i H_ij;  V_{j+1} H_{j+1,j} = W
//   the block Hessenberg matrix is reduced by Givens rotations (FP64), the rotated E_1 S_0
//   gives every column's residual norm; X += [V_0 .. V_{k-1}] Y with Y from the triangle.
// Vectors are FP32 coarse bundles; every small matrix is FP64. The block Gram products are
// deterministic two-pass reductions; the small dense work runs in one warp per block
// (lane = column of the block).
#include <cmath>

#include "amg.cuh"
#include "block_gmres.cuh"

namespace tmamg {

constexpr int BG_THREADS = 256;
constexpr int BG_MAXS = 16;  // largest block width (rhs per shift); one warp per block

__device__ __forceinline__ double2 bcm(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 bcj(double2 a) { return make_double2(a.x, -a.y); }

// complex value of system n at entry e of a coarse FP32 bundle
__device__ __forceinline__ float2 bget(const float* v, int64_t M, int n, int64_t e) {
  const float* q = v + (((int64_t)(n >> 1) * M + e) * 4);
  return make_float2(q[n & 1], q[2 + (n & 1)]);
}

// ---------------------------------------------------------------- block Gram: out[i][a][b] = <V_i[a], W[b]>
// for i < k and a, b in the same block (a % nshift == b % nshift); partials per CTA, then a
// fixed-order sum. One CTA handles a range of entries for every (i, pair).
__global__ void __launch_bounds__(BG_THREADS) bgram_partial_kernel(const float* __restrict__ V, int64_t vstride, int k,
                                                                   const float* __restrict__ W, int64_t M, int nsys,
                                                                   int nshift, double2* __restrict__ part) {
  // one warp per (i, pair) at a time, lanes over the CTA's entries (coalesced), FP32 lane sums
  // added by a fixed-order warp reduction and kept in FP64
  const int npair = nsys * (nsys / nshift);  // (a, b-index within a's block)
  const int s = nsys / nshift;
  const int64_t per = (M + gridDim.x - 1) / gridDim.x;
  const int64_t e_lo = blockIdx.x * per;
  const int64_t e_hi = e_lo + per < M ? e_lo + per : M;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int q = warp; q < k * npair; q += nw) {
    const int i = q / npair, pr = q % npair;
    const int a = pr / s, bi = pr % s;
    const int b = (a % nshift) + bi * nshift;
    const float* vi = V + (int64_t)i * vstride;
    double sr = 0, si = 0;
    for (int64_t e0 = e_lo; e0 < e_hi; e0 += 32 * 64) {  // FP32 runs of at most 64 entries per lane
      float fr = 0, fi = 0;
      const int64_t e1 = e0 + 32 * 64 < e_hi ? e0 + 32 * 64 : e_hi;
      for (int64_t e = e0 + lane; e < e1; e += 32) {
        const float2 x = bget(vi, M, a, e), y = bget(W, M, b, e);
        fr += x.x * y.x + x.y * y.y;
        fi += x.x * y.y - x.y * y.x;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        fr += __shfl_xor_sync(0xffffffffu, fr, o);
        fi += __shfl_xor_sync(0xffffffffu, fi, o);
      }
      sr += fr;
      si += fi;
    }
    if (lane == 0) part[((int64_t)blockIdx.x * k + i) * npair + pr] = make_double2(sr, si);
  }
}

__global__ void bgram_final_kernel(const double2* __restrict__ part, int nblk, int k, int npair, double2* out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= k * npair) return;
  double2 s = make_double2(0, 0);
  for (int b = 0; b < nblk; ++b) {
    const double2 v = part[(int64_t)b * k * npair + q];
    s.x += v.x;
    s.y += v.y;
  }
  out[q] = s;  // out[(i * nsys + a) * s + bi]
}

// ---------------------------------------------------------------- W[b] += sign sum_i sum_a V_i[a] C[i][a][bi]
__global__ void baxpy_kernel(const float* __restrict__ V, int64_t vstride, int k, const double2* __restrict__ C,
                             double sign, float* __restrict__ W, int64_t M, int nsys, int nshift) {
  const int s = nsys / nshift;
  const int nt = (nsys + 1) / 2;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= M * nt) return;
  const int64_t e = t % M;
  const int tile = (int)(t / M);
  float4 w = *reinterpret_cast<const float4*>(W + (((int64_t)tile * M + e) * 4));
  float o[2][2] = {{w.x, w.z}, {w.y, w.w}};  // [lane][re, im]
  for (int l = 0; l < 2; ++l) {
    const int b = tile * 2 + l;
    if (b >= nsys) continue;
    const int kb = b % nshift, bi = b / nshift;
    // FP32 arithmetic on the FP32 basis (GB300's FP64 rate is 1/64 of FP32); coefficients rounded
    float ar = 0, ai = 0;
    for (int i = 0; i < k; ++i) {
      const float* vi = V + (int64_t)i * vstride;
      for (int aj = 0; aj < s; ++aj) {
        const int a = kb + aj * nshift;
        const float2 x = bget(vi, M, a, e);
        const double2 cd = C[((int64_t)i * nsys + a) * s + bi];
        const float cr = (float)cd.x, ci = (float)cd.y;
        ar += cr * x.x - ci * x.y;
        ai += cr * x.y + ci * x.x;
      }
    }
    o[l][0] += (float)sign * ar;
    o[l][1] += (float)sign * ai;
  }
  *reinterpret_cast<float4*>(W + (((int64_t)tile * M + e) * 4)) = make_float4(o[0][0], o[1][0], o[0][1], o[1][1]);
}

// ---------------------------------------------------------------- small dense work (one warp per block)
// Cholesky of the Gram matrix G (s x s, Hermitian) of block kb: G = R^+ R, R upper triangular.
// Writes Rinv (upper) as coefficients C[a][bi] for baxpy (W <- W R^{-1}, with sign handled by
// the caller through a separate output buffer) and accumulates Racc <- R Racc.
// A pivot that is not positive is replaced by a tiny value (a direction that has died).
__device__ void chol_inv(const double2* G, int s, double2* R, double2* Ri) {
  // R and Ri are s x s in shared memory, row-major; lane = column
  const int lane = threadIdx.x & 31;
  for (int q = lane; q < s * s; q += 32) {
    R[q] = make_double2(0, 0);
    Ri[q] = make_double2(0, 0);
  }
  __syncwarp();
  // scale reference for the pivot floor
  double gmax = 0;
  for (int d = 0; d < s; ++d) gmax = fmax(gmax, G[d * s + d].x);
  for (int j = 0; j < s; ++j) {
    // R[j][j] = sqrt(G[j][j] - sum_{p<j} |R[p][j]|^2)
    if (lane == 0) {
      double d = G[j * s + j].x;
      for (int p = 0; p < j; ++p) d -= R[p * s + j].x * R[p * s + j].x + R[p * s + j].y * R[p * s + j].y;
      if (!(d > 1e-28 * gmax)) d = 1e-28 * (gmax > 0 ? gmax : 1.0);
      R[j * s + j] = make_double2(sqrt(d), 0);
    }
    __syncwarp();
    // R[j][c] = (G[j][c] - sum_{p<j} conj(R[p][j]) R[p][c]) / R[j][j], c > j
    const int c = lane;
    if (c > j && c < s) {
      double2 v = G[j * s + c];
      for (int p = 0; p < j; ++p) {
        const double2 t = bcm(bcj(R[p * s + j]), R[p * s + c]);
        v.x -= t.x;
        v.y -= t.y;
      }
      const double inv = 1.0 / R[j * s + j].x;
      R[j * s + c] = make_double2(v.x * inv, v.y * inv);
    }
    __syncwarp();
  }
  // Ri = R^{-1} (upper triangular), column c by lane c: solve R x = e_c
  const int c = lane;
  if (c < s) {
    for (int i = c; i >= 0; --i) {
      double2 v = make_double2(i == c ? 1.0 : 0.0, 0);
      for (int p = i + 1; p <= c; ++p) {
        const double2 t = bcm(R[i * s + p], Ri[p * s + c]);
        v.x -= t.x;
        v.y -= t.y;
      }
      const double inv = 1.0 / R[i * s + i].x;
      Ri[i * s + c] = make_double2(v.x * inv, v.y * inv);
    }
  }
  __syncwarp();
}

// gram layout from bgram: out[(i * nsys + a) * s + bi]; for block kb: G[ai][bi] with a = kb + ai nshift
__global__ void bg_cholqr_kernel(const double2* __restrict__ gram, int nsys, int nshift, double2* coef,
                                 double2* Racc, int first) {
  __shared__ double2 G[BG_MAXS * BG_MAXS], R[BG_MAXS * BG_MAXS], Ri[BG_MAXS * BG_MAXS], T[BG_MAXS * BG_MAXS];
  const int kb = blockIdx.x;
  const int s = nsys / nshift;
  const int lane = threadIdx.x;
  for (int q = lane; q < s * s; q += 32) {
    const int ai = q / s, bi = q % s;
    const int a = kb + ai * nshift;
    G[q] = gram[(int64_t)a * s + bi];
  }
  __syncwarp();
  chol_inv(G, s, R, Ri);
  // coefficients for W <- W Ri : coef[(0 * nsys + a) * s + bi] = Ri[ai][bi]
  for (int q = lane; q < s * s; q += 32) {
    const int ai = q / s, bi = q % s;
    coef[((int64_t)(kb + ai * nshift)) * s + bi] = Ri[q];
  }
  // Racc (per block, s x s) <- R Racc  (or R on the first pass)
  double2* Ra = Racc + (int64_t)kb * s * s;
  for (int q = lane; q < s * s; q += 32) T[q] = first ? R[q] : Ra[q];
  __syncwarp();
  if (!first) {
    for (int q = lane; q < s * s; q += 32) {
      const int i = q / s, c = q % s;
      double2 v = make_double2(0, 0);
      for (int p = 0; p < s; ++p) {
        const double2 t = bcm(R[i * s + p], T[p * s + c]);
        v.x += t.x;
        v.y += t.y;
      }
      Ra[q] = v;
    }
  } else {
    for (int q = lane; q < s * s; q += 32) Ra[q] = T[q];
  }
}

// State per block (FP64, global): Hb [(m+1) s][m s] (row-major, ld = m s), Gb [(m+1) s][s],
// rotations cs/sn per (column, k < s), residual per column, done flags.
struct BGDense {
  double2* H;
  double2* Gr;
  double* cs;
  double2* sn;
  double2* Y;
  double* res;      // [nblock][s]
  double* tolabs;   // [nblock][s]
  int* active;      // [nblock]
  int* nactive;     // [1]
};

// place the new block column (Gram coefficients of step j and R_{j+1}) in H, apply the old
// rotations, build s new rotations per column, rotate the right-hand side block, residuals
__global__ void bg_hessenberg_kernel(const double2* __restrict__ gram, const double2* __restrict__ Rnext, BGDense d,
                                     int j, int m, int nsys, int nshift) {
  const int kb = blockIdx.x;
  const int s = nsys / nshift;
  const int lane = threadIdx.x;
  const int ld = m * s;
  double2* H = d.H + (int64_t)kb * (m + 1) * s * ld;
  double2* Gr = d.Gr + (int64_t)kb * (m + 1) * s * s;
  double* cs = d.cs + (int64_t)kb * m * s * s;
  double2* sn = d.sn + (int64_t)kb * m * s * s;
  if (!d.active[kb]) return;
  // column cc = j s + lane: rows i s + ai from gram (i <= j), rows (j+1) s + ai from Rnext
  if (lane < s) {
    const int cc = j * s + lane;
    for (int i = 0; i <= j; ++i)
      for (int ai = 0; ai < s; ++ai) {
        const int a = kb + ai * nshift;
        H[(int64_t)(i * s + ai) * ld + cc] = gram[((int64_t)i * nsys + a) * s + lane];
      }
    for (int ai = 0; ai < s; ++ai) H[(int64_t)((j + 1) * s + ai) * ld + cc] = Rnext[(int64_t)kb * s * s + ai * s + lane];
    // apply the rotations of all previous columns c' < j s (each: s rotations, bottom-up)
    for (int c2 = 0; c2 < j * s; ++c2) {
      for (int q = 0; q < s; ++q) {
        const int r = c2 + s - q;  // rotate rows (r-1, r)
        const double c = cs[(int64_t)c2 * s + q];
        const double2 sg = sn[(int64_t)c2 * s + q];
        const double2 x = H[(int64_t)(r - 1) * ld + cc], y = H[(int64_t)r * ld + cc];
        const double2 t = bcm(sg, y);
        H[(int64_t)(r - 1) * ld + cc] = make_double2(c * x.x + t.x, c * x.y + t.y);
        const double2 u = bcm(bcj(sg), x);
        H[(int64_t)r * ld + cc] = make_double2(c * y.x - u.x, c * y.y - u.y);
      }
    }
  }
  __syncwarp();
  // new rotations, column by column of the block (sequential in the column, parallel in lanes)
  for (int lc = 0; lc < s; ++lc) {
    const int c2 = j * s + lc;
    // rotations for column c2 (lane 0 computes them one by one, bottom-up)
    if (lane == 0) {
      for (int q = 0; q < s; ++q) {
        const int r = c2 + s - q;
        const double2 x = H[(int64_t)(r - 1) * ld + c2], y = H[(int64_t)r * ld + c2];
        const double nx = hypot(x.x, x.y), ny = hypot(y.x, y.y);
        const double rr = hypot(nx, ny);
        double c;
        double2 sg;
        if (rr == 0.0) {
          c = 1.0;
          sg = make_double2(0, 0);
        } else if (nx == 0.0) {
          c = 0.0;
          sg = make_double2(y.x / ny, -y.y / ny);
        } else {
          c = nx / rr;
          sg = bcm(make_double2(x.x / nx, x.y / nx), make_double2(y.x / rr, -y.y / rr));
        }
        cs[(int64_t)c2 * s + q] = c;
        sn[(int64_t)c2 * s + q] = sg;
        H[(int64_t)(r - 1) * ld + c2] = nx == 0.0 ? make_double2(rr, 0) : make_double2(x.x / nx * rr, x.y / nx * rr);
        H[(int64_t)r * ld + c2] = make_double2(0, 0);
      }
    }
    __syncwarp();
    // apply them to the later columns of this block and to the right-hand side block
    const int cc = j * s + lane;
    if (lane < s && lane > lc) {
      for (int q = 0; q < s; ++q) {
        const int r = c2 + s - q;
        const double c = cs[(int64_t)c2 * s + q];
        const double2 sg = sn[(int64_t)c2 * s + q];
        const double2 x = H[(int64_t)(r - 1) * ld + cc], y = H[(int64_t)r * ld + cc];
        const double2 t = bcm(sg, y);
        H[(int64_t)(r - 1) * ld + cc] = make_double2(c * x.x + t.x, c * x.y + t.y);
        const double2 u = bcm(bcj(sg), x);
        H[(int64_t)r * ld + cc] = make_double2(c * y.x - u.x, c * y.y - u.y);
      }
    }
    if (lane < s) {  // right-hand side column = lane
      for (int q = 0; q < s; ++q) {
        const int r = c2 + s - q;
        const double c = cs[(int64_t)c2 * s + q];
        const double2 sg = sn[(int64_t)c2 * s + q];
        const double2 x = Gr[(int64_t)(r - 1) * s + lane], y = Gr[(int64_t)r * s + lane];
        const double2 t = bcm(sg, y);
        Gr[(int64_t)(r - 1) * s + lane] = make_double2(c * x.x + t.x, c * x.y + t.y);
        const double2 u = bcm(bcj(sg), x);
        Gr[(int64_t)r * s + lane] = make_double2(c * y.x - u.x, c * y.y - u.y);
      }
    }
    __syncwarp();
  }
  // residual of each right-hand side column: norm of rows (j+1) s .. (j+2) s - 1
  if (lane < s) {
    double r2 = 0;
    for (int q = 0; q < s; ++q) {
      const double2 v = Gr[(int64_t)((j + 1) * s + q) * s + lane];
      r2 += v.x * v.x + v.y * v.y;
    }
    d.res[kb * s + lane] = sqrt(r2);
  }
  __syncwarp();
  if (lane == 0) {
    bool all = true;
    for (int q = 0; q < s; ++q) all &= !(d.res[kb * s + q] > d.tolabs[kb * s + q]);
    if (all) d.active[kb] = 0;
  }
}

// start of a cycle: Gr = E_1 S_0 (S_0 = Racc of block kb), tolerances on the first cycle
__global__ void bg_start_kernel(const double2* __restrict__ S0, BGDense d, int m, int nsys, int nshift, double tol,
                                int first) {
  const int kb = blockIdx.x;
  const int s = nsys / nshift;
  const int lane = threadIdx.x;
  double2* Gr = d.Gr + (int64_t)kb * (m + 1) * s * s;
  if (lane < s) {
    for (int r = 0; r < (m + 1) * s; ++r)
      Gr[(int64_t)r * s + lane] = r < s ? S0[(int64_t)kb * s * s + r * s + lane] : make_double2(0, 0);
    double r2 = 0;
    for (int r = 0; r < s; ++r) {
      const double2 v = S0[(int64_t)kb * s * s + r * s + lane];
      r2 += v.x * v.x + v.y * v.y;
    }
    if (first) d.tolabs[kb * s + lane] = tol * sqrt(r2);
    d.res[kb * s + lane] = sqrt(r2);
  }
  __syncwarp();
  if (lane == 0) {
    bool all = true;
    for (int q = 0; q < s; ++q) all &= !(d.res[kb * s + q] > d.tolabs[kb * s + q]);
    d.active[kb] = all ? 0 : 1;
  }
}

__global__ void bg_count_kernel(BGDense d, int nblock) {
  if (threadIdx.x == 0) {
    int c = 0;
    for (int k = 0; k < nblock; ++k) c += d.active[k];
    *d.nactive = c;
  }
}

// Y = R^{-1} Gr on the first kb_steps * s rows, as baxpy coefficients C[i][a][bi]
__global__ void bg_solve_kernel(BGDense d, const int* __restrict__ steps, int m, int nsys, int nshift,
                                double2* coef) {
  const int kb = blockIdx.x;
  const int s = nsys / nshift;
  const int lane = threadIdx.x;
  const int ld = m * s;
  const int n = steps[kb] * s;
  const double2* H = d.H + (int64_t)kb * (m + 1) * s * ld;
  const double2* Gr = d.Gr + (int64_t)kb * (m + 1) * s * s;
  double2* Y = d.Y + (int64_t)kb * m * s * s;
  if (lane < s) {
    for (int r = n - 1; r >= 0; --r) {
      double2 v = Gr[(int64_t)r * s + lane];
      for (int p = r + 1; p < n; ++p) {
        const double2 t = bcm(H[(int64_t)r * ld + p], Y[(int64_t)p * s + lane]);
        v.x -= t.x;
        v.y -= t.y;
      }
      const double2 dd = H[(int64_t)r * ld + r];
      const double den = dd.x * dd.x + dd.y * dd.y;
      Y[(int64_t)r * s + lane] =
          den > 0 ? make_double2((v.x * dd.x + v.y * dd.y) / den, (v.y * dd.x - v.x * dd.y) / den) : make_double2(0, 0);
    }
    // coefficients: coef[(i nsys + a) s + bi] = Y[i s + ai][bi]
    for (int r = 0; r < m * s; ++r) {
      const int i = r / s, ai = r % s;
      const int a = kb + ai * nshift;
      coef[((int64_t)i * nsys + a) * s + lane] = r < n ? Y[(int64_t)r * s + lane] : make_double2(0, 0);
    }
  }
}

__global__ void bg_steps_kernel(const int* __restrict__ active, int* steps, int nblock, int j) {
  const int k = threadIdx.x;
  if (k < nblock && active[k]) steps[k] = j + 1;
}

int BlockGmres::alloc(int m_, int nsys_, int nshift_, int64_t M_) {
  if (m_ <= m && nsys_ == nsys && nshift_ == nshift && M_ <= M) return 0;
  release();
  m = m_;
  nsys = nsys_;
  nshift = nshift_;
  M = M_;
  const int s = nsys / nshift;
  const int nb = nshift;
  nblk = (int)(M / 128);
  if (nblk > 256) nblk = 256;
  if (nblk < 1) nblk = 1;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** q, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(q, bytes);
  };
  A((void**)&gram, sizeof(double2) * (size_t)(m + 1) * nsys * s);
  A((void**)&part, sizeof(double2) * (size_t)nblk * (m + 1) * nsys * s);
  A((void**)&coef, sizeof(double2) * (size_t)(m + 1) * nsys * s);
  A((void**)&hgram, sizeof(double2) * (size_t)(m + 1) * nsys * s);
  A((void**)&Racc, sizeof(double2) * (size_t)nb * s * s);
  A((void**)&S0, sizeof(double2) * (size_t)nb * s * s);
  A((void**)&H, sizeof(double2) * (size_t)nb * (m + 1) * s * m * s);
  A((void**)&Gr, sizeof(double2) * (size_t)nb * (m + 1) * s * s);
  A((void**)&cs, sizeof(double) * (size_t)nb * m * s * s);
  A((void**)&sn, sizeof(double2) * (size_t)nb * m * s * s);
  A((void**)&Y, sizeof(double2) * (size_t)nb * m * s * s);
  A((void**)&res, sizeof(double) * (size_t)nb * s);
  A((void**)&tolabs, sizeof(double) * (size_t)nb * s);
  A((void**)&active, sizeof(int) * nb);
  A((void**)&steps, sizeof(int) * nb);
  A((void**)&nactive, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&h_nactive, sizeof(int));
  return e == cudaSuccess ? 0 : -1;
}

void BlockGmres::release() {
  void* ptrs[] = {gram, part, coef, hgram, Racc, S0, H, Gr, cs, sn, Y, res, tolabs, active, steps, nactive};
  for (void* q : ptrs) cudaFree(q);
  if (h_nactive) cudaFreeHost(h_nactive);
  gram = part = coef = hgram = Racc = S0 = H = Gr = sn = Y = nullptr;
  cs = res = tolabs = nullptr;
  active = steps = nactive = nullptr;
  h_nactive = nullptr;
  m = nsys = nshift = 0;
  M = 0;
}

// Gram of k block vectors against W: gram[(i nsys + a) s + bi]
static void bgram(BlockGmres& b, const float* V, int64_t vstride, int k, const float* W, cudaStream_t st) {
  const int s = b.nsys / b.nshift;
  const int npair = b.nsys * s;
  bgram_partial_kernel<<<b.nblk, BG_THREADS, 0, st>>>(V, vstride, k, W, b.M, b.nsys, b.nshift, b.part);
  TM_COUNT();
  bgram_final_kernel<<<(k * npair + 127) / 128, 128, 0, st>>>(b.part, b.nblk, k, npair, b.gram);
  TM_COUNT();
}

static void baxpy(BlockGmres& b, const float* V, int64_t vstride, int k, const double2* C, double sign, float* W,
                  cudaStream_t st) {
  const int nt = (b.nsys + 1) / 2;
  const int64_t total = b.M * nt;
  baxpy_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(V, vstride, k, C, sign, W, b.M, b.nsys, b.nshift);
  TM_COUNT();
}

// W <- W R^{-1} twice (CholQR2); R_total of each block in b.Racc; dst: a second bundle
static void cholqr2(BlockGmres& b, float* W, float* tmp, size_t bytes, cudaStream_t st) {
  for (int pass = 0; pass < 2; ++pass) {
    bgram(b, W, 0, 1, W, st);
    bg_cholqr_kernel<<<b.nshift, 32, 0, st>>>(b.gram, b.nsys, b.nshift, b.coef, b.Racc, pass == 0);
    TM_COUNT();
    cudaMemsetAsync(tmp, 0, bytes, st);
    baxpy(b, W, 0, 1, b.coef, 1.0, tmp, st);
    cudaMemcpyAsync(W, tmp, bytes, cudaMemcpyDeviceToDevice, st);
  }
}

// V0 = rc - V0 (all systems)
__global__ void rsub_kernel(const float* __restrict__ rc, float* __restrict__ v, int64_t n4) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n4) return;
  const float4 r = reinterpret_cast<const float4*>(rc)[t];
  float4 w = reinterpret_cast<float4*>(v)[t];
  w.x = r.x - w.x; w.y = r.y - w.y; w.z = r.z - w.z; w.w = r.w - w.w;
  reinterpret_cast<float4*>(v)[t] = w;
}

int block_gmres_solve(BlockGmres& b, const std::function<void(const float*, float*)>& apply, const float* rc,
                      float* xc, float* V, int64_t vstride, float* tmp, size_t bundle_bytes, int m, int maxiter,
                      double tol, int* iters_done, cudaStream_t st) {
  const int s = b.nsys / b.nshift;
  if (s > BG_MAXS || b.nsys % b.nshift || m > b.m) return -2;
  BGDense d{b.H, b.Gr, b.cs, b.sn, b.Y, b.res, b.tolabs, b.active, b.nactive};
  const int64_t n4 = (int64_t)(bundle_bytes / sizeof(float4));
  cudaMemsetAsync(xc, 0, bundle_bytes, st);
  cudaMemcpyAsync(V, rc, bundle_bytes, cudaMemcpyDeviceToDevice, st);
  int total = 0;
  for (int cycle = 0;; ++cycle) {
    // V_0 S_0 = R (the residual is in V_0)
    cholqr2(b, V, tmp, bundle_bytes, st);
    cudaMemcpyAsync(b.S0, b.Racc, sizeof(double2) * b.nshift * s * s, cudaMemcpyDeviceToDevice, st);
    bg_start_kernel<<<b.nshift, 32, 0, st>>>(b.S0, d, m, b.nsys, b.nshift, tol, cycle == 0 ? 1 : 0);
    TM_COUNT();
    cudaMemsetAsync(b.steps, 0, sizeof(int) * b.nshift, st);
    bg_count_kernel<<<1, 32, 0, st>>>(d, b.nshift);
    TM_COUNT();
    cudaMemcpyAsync(b.h_nactive, b.nactive, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    if (*b.h_nactive == 0 || total >= maxiter) break;
    int j = 0;
    bool converged = false;
    for (; j < m && total < maxiter; ++j) {
      float* vj = V + (int64_t)j * vstride;
      float* w = V + (int64_t)(j + 1) * vstride;
      apply(vj, w);
      bgram(b, V, vstride, j + 1, w, st);                // H_ij = V_i^+ W
      cudaMemcpyAsync(b.hgram, b.gram, sizeof(double2) * (size_t)(j + 1) * b.nsys * s, cudaMemcpyDeviceToDevice, st);
      baxpy(b, V, vstride, j + 1, b.hgram, -1.0, w, st);  // W -= sum_i V_i H_ij (one CGS pass)
      cholqr2(b, w, tmp, bundle_bytes, st);               // V_{j+1} R_{j+1} = W
      bg_steps_kernel<<<1, 32, 0, st>>>(b.active, b.steps, b.nshift, j);
      TM_COUNT();
      bg_hessenberg_kernel<<<b.nshift, 32, 0, st>>>(b.hgram, b.Racc, d, j, m, b.nsys, b.nshift);
      TM_COUNT();
      bg_count_kernel<<<1, 32, 0, st>>>(d, b.nshift);
      TM_COUNT();
      ++total;
      cudaMemcpyAsync(b.h_nactive, b.nactive, sizeof(int), cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
      if (*b.h_nactive == 0) {
        ++j;
        converged = true;
        break;
      }
    }
    bg_solve_kernel<<<b.nshift, 32, 0, st>>>(d, b.steps, m, b.nsys, b.nshift, b.coef);
    TM_COUNT();
    baxpy(b, V, vstride, j, b.coef, 1.0, xc, st);
    if (converged || total >= maxiter) break;
    // restart from the true residual: V_0 = rc - A x
    apply(xc, V);
    rsub_kernel<<<(unsigned)((n4 + 255) / 256), 256, 0, st>>>(rc, V, n4);
    TM_COUNT();
  }
  if (iters_done) *iters_done = total;
  return 0;
}

}  // namespace tmamg

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
#include "profile.cuh"

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

// ---------------------------------------------------------------- one reduction per block step
// Block classical Gram-Schmidt with the Cholesky Gram taken from the same reduction: with
// H_i = V_i^+ W (i < k) and G = W^+ W, the block left after the projection, U = W - sum V_i H_i,
// has U^+ U = G - sum_i H_i^+ H_i (the V_i are orthonormal), so U = V_k R with R the Cholesky
// factor of that matrix, and V_k = U R^{-1} = W R^{-1} - sum_i V_i (H_i R^{-1}). One grid-wide
// reduction and one vector pass per block step instead of a Gram, an update and two CholQR passes
// (the paper, Sec. 4: most of the block solver's overhead is global reductions).

// partial[((blk * nshift + g) * (k + 1) + i) * s * s + ar * s + br] over the CTA's entries:
// i < k: <V_i[a], W[b]>, i = k: <W[a], W[b]>, systems a = g + ar nshift, b = g + br nshift of
// group g = blockIdx.y. Pairs in 4 x 4 chunks (blockIdx.z = chunk pair).
__global__ void __launch_bounds__(BG_THREADS) bg_gram_kernel(const float* __restrict__ V, int64_t vstride, int k,
                                                             const float* __restrict__ W, int64_t M, int nsys,
                                                             int nshift, double2* __restrict__ part) {
  const int s = nsys / nshift;
  const int g = blockIdx.y;
  const int nch = (s + 3) / 4;
  const int ca = blockIdx.z / nch, cb = blockIdx.z % nch;
  const int nblk = gridDim.x;
  const int64_t per = (M + nblk - 1) / nblk;
  const int64_t e_lo = blockIdx.x * per;
  const int64_t e_hi = e_lo + per < M ? e_lo + per : M;
  __shared__ double2 red[BG_THREADS / 32][16];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = 0; i <= k; ++i) {
    const float* X = i < k ? V + (int64_t)i * vstride : W;
    float ar[4][4], ai[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) { ar[p][q] = 0.f; ai[p][q] = 0.f; }
    for (int64_t e = e_lo + threadIdx.x; e < e_hi; e += blockDim.x) {
      float2 x[4], y[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int ra = ca * 4 + p, rb = cb * 4 + p;
        x[p] = ra < s ? bget(X, M, g + ra * nshift, e) : make_float2(0.f, 0.f);
        y[p] = rb < s ? bget(W, M, g + rb * nshift, e) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // conj(x_p) y_q
          ar[p][q] += x[p].x * y[q].x + x[p].y * y[q].y;
          ai[p][q] += x[p].x * y[q].y - x[p].y * y[q].x;
        }
    }
    // fixed-order reduction: warp shuffles, then the warps in order
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        double dr = ar[p][q], di = ai[p][q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          dr += __shfl_xor_sync(0xffffffffu, dr, o);
          di += __shfl_xor_sync(0xffffffffu, di, o);
        }
        if (lane == 0) red[warp][p * 4 + q] = make_double2(dr, di);
      }
    __syncthreads();
    if (threadIdx.x < 16) {
      const int p = threadIdx.x / 4, q = threadIdx.x % 4;
      const int ra = ca * 4 + p, rb = cb * 4 + q;
      double2 t = make_double2(0, 0);
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        t.x += red[w][threadIdx.x].x;
        t.y += red[w][threadIdx.x].y;
      }
      if (ra < s && rb < s)
        part[(((int64_t)blockIdx.x * nshift + g) * (k + 1) + i) * s * s + ra * s + rb] = t;
    }
    __syncthreads();
  }
}

// out[(g (k + 1) + i) s s + pair] = sum over the CTAs in index order
__global__ void bg_gram_final_kernel(const double2* __restrict__ part, int nblk, int nper, double2* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nper) return;
  double2 t = make_double2(0, 0);
  for (int b = 0; b < nblk; ++b) {
    const double2 v = part[(int64_t)b * nper + q];
    t.x += v.x;
    t.y += v.y;
  }
  out[q] = t;
}

// Per group (one warp): R = chol(G - sum_i H_i^+ H_i), the update coefficients
// coef[(g (k + 1) + i) s s + c s + b] = -(H_i R^{-1})[c][b] (i < k) and R^{-1}[c][b] (i = k), the block
// Gram in the Hessenberg kernel's layout gram[(i nsys + a) s + br] = H_i[ar][br] and Racc[g] = R.
__global__ void bg_lowsync_kernel(const double2* __restrict__ out, int k, int nsys, int nshift, double2* coef,
                                  double2* gram, double2* Racc) {
  __shared__ double2 G[BG_MAXS * BG_MAXS], R[BG_MAXS * BG_MAXS], Ri[BG_MAXS * BG_MAXS];
  const int g = blockIdx.x;
  const int s = nsys / nshift;
  const int lane = threadIdx.x;
  const double2* o = out + (int64_t)g * (k + 1) * s * s;
  // G - sum_i H_i^+ H_i, entry (p, q) = G[p][q] - sum_i sum_c conj(H_i[c][p]) H_i[c][q]
  for (int q2 = lane; q2 < s * s; q2 += 32) {
    const int p = q2 / s, q = q2 % s;
    double2 v = o[(int64_t)k * s * s + q2];
    for (int i = 0; i < k; ++i)
      for (int c = 0; c < s; ++c) {
        const double2 t = bcm(bcj(o[(int64_t)i * s * s + c * s + p]), o[(int64_t)i * s * s + c * s + q]);
        v.x -= t.x;
        v.y -= t.y;
      }
    G[q2] = v;
  }
  __syncwarp();
  chol_inv(G, s, R, Ri);
  double2* cf = coef + (int64_t)g * (k + 1) * s * s;
  for (int q2 = lane; q2 < s * s; q2 += 32) {
    const int c = q2 / s, b = q2 % s;
    cf[(int64_t)k * s * s + q2] = Ri[q2];
    for (int i = 0; i < k; ++i) {
      double2 v = make_double2(0, 0);
      for (int d = 0; d < s; ++d) {
        const double2 t = bcm(o[(int64_t)i * s * s + c * s + d], Ri[d * s + b]);
        v.x -= t.x;
        v.y -= t.y;
      }
      cf[(int64_t)i * s * s + q2] = v;
      gram[((int64_t)i * nsys + g + c * nshift) * s + b] = o[(int64_t)i * s * s + q2];
    }
    Racc[(int64_t)g * s * s + q2] = R[q2];
  }
}

// V_new[b] = sum_c W[c] coef_k[c][b] + sum_{i < k} sum_c V_i[c] coef_i[c][b] for the systems b of group
// g (c and b over the group): one thread per (entry, group), thread index = entry * nshift + g, so
// the two groups that share a 16-byte entry of a tile read it in the same warp; coefficients (FP32)
// in shared memory [g][i][c][b]
__global__ void __launch_bounds__(BG_THREADS) bg_update_kernel(const float* __restrict__ V, int64_t vstride, int k,
                                                               const float* __restrict__ W,
                                                               const double2* __restrict__ coef, int64_t M, int nsys,
                                                               int nshift, float* __restrict__ Vout) {
  extern __shared__ float2 cf[];  // [nshift][k + 1][s][s]
  const int s = nsys / nshift;
  const int ncoef = nshift * (k + 1) * s * s;
  for (int q = threadIdx.x; q < ncoef; q += blockDim.x) {
    const double2 c = coef[q];
    cf[q] = make_float2((float)c.x, (float)c.y);
  }
  __syncthreads();
  const int64_t total = M * nshift;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = idx / nshift;
    const int g = (int)(idx % nshift);
    float2 acc[BG_MAXS];
#pragma unroll
    for (int br = 0; br < BG_MAXS; ++br) acc[br] = make_float2(0.f, 0.f);
    for (int i = 0; i <= k; ++i) {
      const float* X = i < k ? V + (int64_t)i * vstride : W;
      const float2* ci = cf + (int64_t)(g * (k + 1) + i) * s * s;
      for (int cr = 0; cr < s; ++cr) {
        const float2 x = bget(X, M, g + cr * nshift, e);
        const float2* cc = ci + cr * s;
#pragma unroll
        for (int br = 0; br < BG_MAXS; ++br) {
          if (br < s) {
            const float2 w = cc[br];
            acc[br].x += x.x * w.x - x.y * w.y;
            acc[br].y += x.x * w.y + x.y * w.x;
          }
        }
      }
    }
#pragma unroll
    for (int br = 0; br < BG_MAXS; ++br) {
      if (br < s) {
        const int b = g + br * nshift;
        float* q = Vout + (((int64_t)(b >> 1) * M + e) * 4);
        q[b & 1] = acc[br].x;
        q[2 + (b & 1)] = acc[br].y;
      }
    }
  }
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
  A((void**)&gram, sizeof(double2) * (size_t)(m + 2) * nsys * s);
  A((void**)&part, sizeof(double2) * (size_t)nblk * (m + 2) * nsys * s);
  A((void**)&coef, sizeof(double2) * (size_t)(m + 2) * nsys * s);
  A((void**)&hgram, sizeof(double2) * (size_t)(m + 2) * nsys * s);
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

static void baxpy(BlockGmres& b, const float* V, int64_t vstride, int k, const double2* C, double sign, float* W,
                  cudaStream_t st) {
  const int nt = (b.nsys + 1) / 2;
  const int64_t total = b.M * nt;
  baxpy_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(V, vstride, k, C, sign, W, b.M, b.nsys, b.nshift);
  TM_COUNT();
}

// One block step's reduction and update: with W in `w` and the basis blocks V_0 .. V_{k-1}, the
// Grams V_i^+ W and W^+ W of every group in one reduction, then R (Racc), the Hessenberg column
// (b.gram) and the coefficients, then V_k = (W - sum V_i H_i) R^{-1} written to `out` (k = 0:
// V_0 = W R^{-1}, the start block).
static void lowsync_step(BlockGmres& b, const float* V, int64_t vstride, int k, const float* w, float* out,
                         cudaStream_t st) {
  const int s = b.nsys / b.nshift;
  const int nch = (s + 3) / 4;
  const int nper = b.nshift * (k + 1) * s * s;
  bg_gram_kernel<<<dim3(b.nblk, b.nshift, nch * nch), BG_THREADS, 0, st>>>(V, vstride, k, w, b.M, b.nsys, b.nshift,
                                                                          b.part);
  TM_COUNT();
  bg_gram_final_kernel<<<(nper + 127) / 128, 128, 0, st>>>(b.part, b.nblk, nper, b.hgram);
  TM_COUNT();
  bg_lowsync_kernel<<<b.nshift, 32, 0, st>>>(b.hgram, k, b.nsys, b.nshift, b.coef, b.gram, b.Racc);
  TM_COUNT();
  const size_t smem = sizeof(float2) * (size_t)nper;
  func_smem_optin((const void*)bg_update_kernel, (int)(smem > 48 * 1024 ? smem : 48 * 1024));
  const int64_t total = b.M * b.nshift;
  int grid = (int)((total + BG_THREADS - 1) / BG_THREADS);
  if (grid > 152 * 8) grid = 152 * 8;
  bg_update_kernel<<<grid, BG_THREADS, smem, st>>>(V, vstride, k, w, b.coef, b.M, b.nsys, b.nshift, out);
  TM_COUNT();
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
  TM_PROF(st, "block_gmres");
  const int s = b.nsys / b.nshift;
  if (s > BG_MAXS || b.nsys % b.nshift || m > b.m) return -2;
  // the update kernel keeps its coefficients in shared memory
  if (sizeof(float2) * (size_t)b.nshift * (m + 1) * s * s > (size_t)device_smem_optin() - 4096) return -2;
  BGDense d{b.H, b.Gr, b.cs, b.sn, b.Y, b.res, b.tolabs, b.active, b.nactive};
  const int64_t n4 = (int64_t)(bundle_bytes / sizeof(float4));
  cudaMemsetAsync(xc, 0, bundle_bytes, st);
  cudaMemcpyAsync(tmp, rc, bundle_bytes, cudaMemcpyDeviceToDevice, st);
  int total = 0;
  for (int cycle = 0;; ++cycle) {
    // V_0 S_0 = R (the residual is in tmp)
    lowsync_step(b, V, vstride, 0, tmp, V, st);
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
      apply(vj, tmp);                                                    // W = A V_j
      lowsync_step(b, V, vstride, j + 1, tmp, V + (int64_t)(j + 1) * vstride, st);  // V_{j+1} R_{j+1} = W - sum V_i H_ij
      bg_steps_kernel<<<1, 32, 0, st>>>(b.active, b.steps, b.nshift, j);
      TM_COUNT();
      bg_hessenberg_kernel<<<b.nshift, 32, 0, st>>>(b.gram, b.Racc, d, j, m, b.nsys, b.nshift);
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
    // restart from the true residual: tmp = rc - A x
    apply(xc, tmp);
    rsub_kernel<<<(unsigned)((n4 + 255) / 256), 256, 0, st>>>(rc, tmp, n4);
    TM_COUNT();
  }
  if (iters_done) *iters_done = total;
  return 0;
}

}  // namespace tmamg

// Batched (F)GMRES over bundles on GB300.
//
// All systems of a bundle run their own Arnoldi process in lockstep (paper Sec. 3: the
// systems are iterated simultaneously so that every operator application serves all of
// them). Orthogonalisation is one pass of classical Gram-Schmidt (the variant the paper
// found fastest, Sec. 4), optionally repeated. The Hessenberg matrix, its Givens
// rotations and the least-squares solution are kept per system in FP64 on the device;
// a system whose residual estimate reaches its tolerance stops updating (convergence
// mask) while the others continue. The host only polls an active-system count.
#include <cmath>

#include "blas.cuh"
#include "krylov.cuh"

namespace tmamg {

int GmresState::alloc(int m_, int cap_, size_t pe) {
  if (m_ <= m && cap_ <= cap && pe <= partial_cap) return 0;
  release();
  m = m_;
  cap = cap_;
  partial_cap = pe;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t b) {
    if (e == cudaSuccess) e = cudaMalloc(p, b);
  };
  A((void**)&H, sizeof(double2) * (size_t)(m + 1) * m * cap);
  A((void**)&cs, sizeof(double) * (size_t)m * cap);
  A((void**)&sn, sizeof(double2) * (size_t)m * cap);
  A((void**)&g, sizeof(double2) * (size_t)(m + 1) * cap);
  A((void**)&y, sizeof(double2) * (size_t)m * cap);
  A((void**)&tmp, sizeof(double2) * (size_t)(m + 1) * cap);
  A((void**)&sc, sizeof(double2) * (size_t)cap);
  A((void**)&beta, sizeof(double) * (size_t)cap);
  A((void**)&tolabs, sizeof(double) * (size_t)cap);
  A((void**)&resid, sizeof(double) * (size_t)cap);
  A((void**)&kconv, sizeof(int) * (size_t)cap);
  A((void**)&active, sizeof(int) * (size_t)cap);
  A((void**)&nactive, sizeof(int));
  A((void**)&partial, sizeof(double2) * pe);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&h_nactive, sizeof(int));
  return e == cudaSuccess ? 0 : -1;
}

void GmresState::release() {
  cudaFree(H); cudaFree(cs); cudaFree(sn); cudaFree(g); cudaFree(y); cudaFree(tmp); cudaFree(sc);
  cudaFree(beta); cudaFree(tolabs); cudaFree(resid); cudaFree(kconv); cudaFree(active); cudaFree(nactive);
  cudaFree(partial);
  if (h_nactive) cudaFreeHost(h_nactive);
  H = nullptr; cs = nullptr; sn = nullptr; g = nullptr; y = nullptr; tmp = nullptr; sc = nullptr;
  beta = nullptr; tolabs = nullptr; resid = nullptr; kconv = nullptr; active = nullptr; nactive = nullptr;
  partial = nullptr; h_nactive = nullptr;
  m = 0; cap = 0; partial_cap = 0;
}

__global__ void set_value_kernel(double* a, int n, double v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

void set_rel_tol(double* rel, int nsys, double value, cudaStream_t s) {
  set_value_kernel<<<(nsys + 127) / 128, 128, 0, s>>>(rel, nsys, value); TM_COUNT();
}

// beta = |r0|, g = (beta, 0, ...), scale = 1 / beta, tolerance, masks
__global__ void gmres_init_kernel(const double2* __restrict__ dot, int nsys, int cap, int m,
                                  const int* __restrict__ participate, const double* __restrict__ rel_tol,
                                  double* beta, double2* g, double2* sc, double* tolabs, int* kconv, int* active,
                                  int* nactive) {
  int n = threadIdx.x;
  int on = 0;
  if (n < nsys) {
    double b = sqrt(fmax(dot[n].x, 0.0));
    on = (participate ? participate[n] : 1) && b > 0.0 && isfinite(b);
    beta[n] = b;
    for (int i = 0; i <= m; ++i) g[i * cap + n] = make_double2(0, 0);
    g[n] = make_double2(on ? b : 0.0, 0);
    sc[n] = make_double2(on ? 1.0 / b : 0.0, 0);
    tolabs[n] = rel_tol[n] * b;
    kconv[n] = 0;
    active[n] = on;
  }
  int cnt = __syncthreads_count(on);
  if (n == 0) *nactive = cnt;
}

__global__ void norm_finish_kernel(const double2* __restrict__ dot, double2* Hcol_next, double2* sc, int nsys) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nsys) return;
  double h = sqrt(fmax(dot[n].x, 0.0));
  Hcol_next[n] = make_double2(h, 0);
  sc[n] = make_double2(h > 0 ? 1.0 / h : 0.0, 0);
}

__global__ void add_col_kernel(double2* Hcol, const double2* __restrict__ t, int rows, int nsys, int cap) {
  int t_ = blockIdx.x * blockDim.x + threadIdx.x;
  if (t_ >= rows * nsys) return;
  int i = t_ / nsys, n = t_ % nsys;
  double2 a = Hcol[i * cap + n], b = t[i * cap + n];
  Hcol[i * cap + n] = make_double2(a.x + b.x, a.y + b.y);
}

__device__ __forceinline__ double2 cm(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cj(double2 a) { return make_double2(a.x, -a.y); }

// apply the previous rotations to column j, build rotation j, update g and the masks
__global__ void givens_kernel(double2* H, double* cs, double2* sn, double2* g, double* resid, const double* tolabs,
                              int* kconv, int* active, int* nactive, int j, int m, int nsys, int cap) {
  int n = threadIdx.x;
  int still = 0;
  if (n < nsys && active[n]) {
    double2* col = H + (size_t)j * (m + 1) * cap;
    for (int i = 0; i < j; ++i) {
      double c = cs[i * cap + n];
      double2 s = sn[i * cap + n];
      double2 a = col[i * cap + n], b = col[(i + 1) * cap + n];
      double2 t = cm(s, b);
      col[i * cap + n] = make_double2(c * a.x + t.x, c * a.y + t.y);
      double2 u = cm(cj(s), a);
      col[(i + 1) * cap + n] = make_double2(c * b.x - u.x, c * b.y - u.y);
    }
    double2 a = col[j * cap + n], b = col[(j + 1) * cap + n];
    double na = hypot(a.x, a.y), nb = hypot(b.x, b.y);
    double r = hypot(na, nb);
    double c;
    double2 s;
    if (r == 0.0) {
      c = 1.0;
      s = make_double2(0, 0);
    } else if (na == 0.0) {
      c = 0.0;
      s = make_double2(b.x / nb, -b.y / nb);
    } else {
      c = na / r;
      double2 ph = make_double2(a.x / na, a.y / na);
      s = cm(ph, make_double2(b.x / r, -b.y / r));
    }
    cs[j * cap + n] = c;
    sn[j * cap + n] = s;
    double2 newa = na == 0.0 ? make_double2(r, 0) : make_double2(a.x / na * r, a.y / na * r);
    col[j * cap + n] = newa;
    col[(j + 1) * cap + n] = make_double2(0, 0);
    double2 gj = g[j * cap + n];
    double2 t = cm(cj(s), gj);
    g[(j + 1) * cap + n] = make_double2(-t.x, -t.y);
    g[j * cap + n] = make_double2(c * gj.x, c * gj.y);
    double res = hypot(t.x, t.y);
    resid[n] = res;
    bool done = !(res > tolabs[n]) || j + 1 == m || nb == 0.0;
    if (done) {
      kconv[n] = j + 1;
      active[n] = 0;
    } else {
      still = 1;
    }
  }
  int cnt = __syncthreads_count(still);
  if (n == 0) *nactive = cnt;
}

// y = R^{-1} g on the first k = kconv[n] rows (zero beyond)
__global__ void backsub_kernel(const double2* __restrict__ H, const double2* __restrict__ g, double2* y,
                               const int* __restrict__ kconv, int m, int nsys, int cap, int kmax) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nsys) return;
  int k = kconv[n];
  for (int i = kmax - 1; i >= 0; --i) {
    if (i >= k) {
      y[i * cap + n] = make_double2(0, 0);
      continue;
    }
    double2 s = g[i * cap + n];
    for (int l = i + 1; l < k; ++l) {
      double2 t = cm(H[((size_t)l * (m + 1) + i) * cap + n], y[l * cap + n]);
      s.x -= t.x;
      s.y -= t.y;
    }
    double2 d = H[((size_t)i * (m + 1) + i) * cap + n];
    double den = d.x * d.x + d.y * d.y;
    double2 q = den > 0 ? make_double2((s.x * d.x + s.y * d.y) / den, (s.y * d.x - s.x * d.y) / den)
                        : make_double2(0, 0);
    y[i * cap + n] = q;
  }
}

static void poll_active(GmresState& st, cudaStream_t s) {
  cudaMemcpyAsync(st.h_nactive, st.nactive, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
}

template <typename real>
CycleResult gmres_cycle(GmresState& st, const LevelOpsT<real>& ops, int nsys, int m, real* V, int64_t vstride,
                        real* Z, real* x, const int* participate, const double* rel_tol, int poll, bool cgs2,
                        cudaStream_t s) {
  const int cap = st.cap;
  const int64_t M = ops.M;
  // |r0|
  mdot<real>(V, 0, 1, V, M, nsys, st.tmp, cap, st.partial, s);
  gmres_init_kernel<<<1, 1024, 0, s>>>(st.tmp, nsys, cap, m, participate, rel_tol, st.beta, st.g, st.sc, st.tolabs,
                                       st.kconv, st.active, st.nactive); TM_COUNT();
  axpby<real>(nullptr, 0, nullptr, st.sc, 2, V, M, nsys, nullptr, s);
  int done = 0;
  for (int j = 0; j < m; ++j) {
    real* vj = V + (int64_t)j * vstride;
    real* w = V + (int64_t)(j + 1) * vstride;
    const real* z = vj;
    if (ops.precond) {
      real* zj = Z + (int64_t)j * vstride;
      ops.precond(vj, zj);
      z = zj;
    }
    ops.A(z, w);
    double2* Hcol = st.H + (size_t)j * (m + 1) * cap;
    mdot<real>(V, vstride, j + 1, w, M, nsys, Hcol, cap, st.partial, s);
    maxpy<real>(V, vstride, j + 1, Hcol, cap, -1.0, w, M, nsys, nullptr, s);
    if (cgs2) {
      mdot<real>(V, vstride, j + 1, w, M, nsys, st.tmp, cap, st.partial, s);
      maxpy<real>(V, vstride, j + 1, st.tmp, cap, -1.0, w, M, nsys, nullptr, s);
      add_col_kernel<<<((j + 1) * nsys + 127) / 128, 128, 0, s>>>(Hcol, st.tmp, j + 1, nsys, cap); TM_COUNT();
    }
    mdot<real>(w, 0, 1, w, M, nsys, st.tmp, cap, st.partial, s);
    norm_finish_kernel<<<(nsys + 127) / 128, 128, 0, s>>>(st.tmp, Hcol + (size_t)(j + 1) * cap, st.sc, nsys); TM_COUNT();
    axpby<real>(nullptr, 0, nullptr, st.sc, 2, w, M, nsys, nullptr, s);
    givens_kernel<<<1, 1024, 0, s>>>(st.H, st.cs, st.sn, st.g, st.resid, st.tolabs, st.kconv, st.active, st.nactive,
                                     j, m, nsys, cap); TM_COUNT();
    done = j + 1;
    if (done == m) break;
    if (poll > 0 && (done % poll) == 0) {
      poll_active(st, s);
      if (*st.h_nactive == 0) break;
    }
  }
  backsub_kernel<<<(nsys + 127) / 128, 128, 0, s>>>(st.H, st.g, st.y, st.kconv, m, nsys, cap, done); TM_COUNT();
  maxpy<real>(ops.precond ? Z : V, vstride, done, st.y, cap, +1.0, x, M, nsys, nullptr, s);
  CycleResult r;
  r.iters = done;
  return r;
}

template CycleResult gmres_cycle<float>(GmresState&, const LevelOpsT<float>&, int, int, float*, int64_t, float*, float*,
                                        const int*, const double*, int, bool, cudaStream_t);
template CycleResult gmres_cycle<double>(GmresState&, const LevelOpsT<double>&, int, int, double*, int64_t, double*,
                                         double*, const int*, const double*, int, bool, cudaStream_t);

}  // namespace tmamg

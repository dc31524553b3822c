// Multigrid setup, AMG cycle, mixed-precision multi-rhs/multi-shift solve, and the
// component entry points of the C ABI.
//
// Solve (paper Sec. 4: FGMRES at the top level preconditioned by the multigrid cycle,
// goal residual 1e-10; Sec. 3: all right-hand sides and shifts iterated together):
//   outer loop in FP64:   r = b - D(mu_n) x for every system; stop at |r| <= tol |b|;
//   inner FGMRES(m) in FP32 on r / |r|, preconditioned by the AMG cycle
//       z = P D_c^{-1} P^+ v,   z += SAP(v - D z)
//   with the coarse system solved by GMRES to the relative residual r_b (paper: 1e-1).
#include <cmath>
#include <cstring>
#include <vector>

#include "amg.cuh"
#include "blas.cuh"
#include "block_gmres.cuh"
#include "coarse_gmres.cuh"
#include "coarse_mma.cuh"
#include "krylov.cuh"
#include "nn.cuh"
#include "sap.cuh"

namespace tmamg {

struct Workspace {
  int nsys = 0, m = 0, mc = 0;
  size_t fb32 = 0, fb64 = 0, cb32 = 0;  // bytes of one bundle
  float* V = nullptr;                   // m + 1 fine FP32 bundles
  float* Z = nullptr;                   // m
  float *t1 = nullptr, *t2 = nullptr, *t3 = nullptr, *e32 = nullptr;  // t2: learned step only (made on use)
  double *x64 = nullptr, *r64 = nullptr;
  double* b64 = nullptr;  // right-hand sides, one FP64 tile each (grown on demand)
  size_t b64_bytes = 0;
  double* epsd = nullptr;  // doublet splittings, one per doublet (grown on demand)
  int eps_cap = 0;
  float* Vc = nullptr;  // mc + 1 coarse bundles
  float *xc = nullptr, *rc = nullptr;
  GmresState top, coarse;
  CoarseGmres cg;
  BlockGmres bg;
  float* tc = nullptr;  // one more coarse bundle
  // middle level (coarse level 1 of a three-level hierarchy); the coarse buffers above then
  // belong to the bottom level 2
  int mm = 0;
  size_t mb32 = 0;                                // bytes of one level-1 bundle
  float *Vm = nullptr, *Zm = nullptr;             // mm + 1 and mm level-1 bundles
  float *xm = nullptr, *rm = nullptr, *sm1 = nullptr, *sm2 = nullptr;
  GmresState mid;
  double *rel_mid = nullptr, *beta0m = nullptr;
  double2 *mra = nullptr, *mrd = nullptr;         // MR coefficients [2 ns]: alpha, -alpha; dots [2 ns]
  double *rel_top = nullptr, *rel_coarse = nullptr, *rn = nullptr, *bn = nullptr, *scale = nullptr;
  double *beta0 = nullptr, *tmpd = nullptr;
  double2 *ones = nullptr, *mones = nullptr, *dot = nullptr, *partial64 = nullptr;
  size_t partial64_cap = 0;
  int *mask = nullptr, *flags = nullptr, *count = nullptr;
  int* mask2 = nullptr;  // systems still iterating inside the FP32 inner cycles of one refinement cycle
  int* h_count = nullptr;
  int *outer_it = nullptr, *inner_it = nullptr;
  std::vector<void*> extra;
};

// ctx->levels holds the coarse levels: two of them make a three-level hierarchy whose first
// coarse level is the middle level
static bool has_middle(const tmamg_ctx* ctx) { return ctx->levels.size() == 2; }

static void ws_free(Workspace* w) {
  if (!w) return;
  void* ptrs[] = {w->V, w->Z, w->t1, w->t2, w->t3, w->e32, w->x64, w->r64, w->b64, w->epsd, w->Vc, w->xc, w->rc,
                  w->rel_top, w->rel_coarse, w->rn, w->bn, w->scale, w->beta0, w->tmpd, w->ones, w->mones, w->dot,
                  w->partial64, w->mask, w->mask2, w->flags, w->count, w->outer_it, w->inner_it, w->Vm, w->Zm, w->xm,
                  w->rm, w->sm1, w->sm2, w->rel_mid, w->beta0m, w->mra, w->mrd};
  for (void* p : ptrs) cudaFree(p);
  for (void* p : w->extra) cudaFree(p);
  if (w->h_count) cudaFreeHost(w->h_count);
  w->top.release();
  w->coarse.release();
  w->mid.release();
  w->cg.release();
  w->bg.release();
  cudaFree(w->tc);
  *w = Workspace();
}

// state of the plain FP64 solver (FP64 bundles, one system per tile)
struct Workspace64 {
  int nsys = 0, m = 0, mc = 0;
  int64_t Vc = 0;
  int nc = 0;
  size_t fb = 0, cb = 0;  // bytes of one fine / coarse FP64 bundle
  double *V = nullptr, *Z = nullptr, *x = nullptr, *b = nullptr, *t1 = nullptr, *t2 = nullptr, *t3 = nullptr;
  double *Vc_ = nullptr, *xc = nullptr, *rc = nullptr;
  double *rel_top = nullptr, *rel_coarse = nullptr, *beta0 = nullptr, *bn = nullptr, *rn = nullptr;
  double2 *dot = nullptr, *partial = nullptr, *ones = nullptr, *mones = nullptr;
  GmresState top, coarse;
};

static void ws64_free(Workspace64* w) {
  void* ptrs[] = {w->V, w->Z, w->x, w->b, w->t1, w->t2, w->t3, w->Vc_, w->xc, w->rc, w->rel_top, w->rel_coarse,
                  w->beta0, w->bn, w->rn, w->dot, w->partial, w->ones, w->mones};
  for (void* p : ptrs) cudaFree(p);
  w->top.release();
  w->coarse.release();
  *w = Workspace64();
}

void free_workspace(tmamg_ctx* ctx) {
  if (ctx->ws) {
    ws_free(ctx->ws);
    delete ctx->ws;
    ctx->ws = nullptr;
  }
  if (ctx->ws64) {
    ws64_free(ctx->ws64);
    delete ctx->ws64;
    ctx->ws64 = nullptr;
  }
}

__global__ void fill_c_kernel(double2* a, int n, double re) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = make_double2(re, 0);
}

// solver state for nsys systems and the restart lengths of p (top, bottom and, with three
// levels, middle); grown on demand, never shrunk
static int ensure_ws(tmamg_ctx* ctx, int nsys, const tmamg_solve_params& p) {
  if (!ctx->ws) ctx->ws = new Workspace();
  Workspace* w = ctx->ws;
  const bool three = has_middle(ctx);
  const int m = p.restart, mc = p.coarse_restart, mmid = three ? p.mid_restart : 0;
  if (nsys <= w->nsys && m <= w->m && mc <= w->mc && mmid <= w->mm) return 0;
  int ns = nsys > w->nsys ? nsys : w->nsys;
  int mm = m > w->m ? m : w->m;
  int mcc = mc > w->mc ? mc : w->mc;
  int mmm = mmid > w->mm ? mmid : w->mm;
  ws_free(w);
  w->nsys = ns;
  w->m = mm;
  w->mc = mcc;
  w->mm = mmm;
  const int64_t V = ctx->g.V;
  w->fb32 = (size_t)ntiles(ns, 2) * 12 * V * 4 * sizeof(float);
  w->fb64 = (size_t)ns * 12 * V * 2 * sizeof(double);
  // the coarse buffers serve the bottom level
  int64_t Vc = ctx->levels.empty() ? 1 : ctx->levels.back().Vc;
  int nc = ctx->levels.empty() ? 2 : 2 * ctx->levels.back().nv;
  w->cb32 = (size_t)ntiles(ns, 2) * nc * Vc * 4 * sizeof(float);
  const int64_t Vm = three ? ctx->levels[0].Vc : 0;
  const int ncm = three ? 2 * ctx->levels[0].nv : 0;
  w->mb32 = (size_t)ntiles(ns, 2) * ncm * Vm * 4 * sizeof(float);
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t b) {
    if (e == cudaSuccess) e = cudaMalloc(p, b);
  };
  A((void**)&w->V, w->fb32 * (mm + 1));
  A((void**)&w->Z, w->fb32 * mm);
  A((void**)&w->t1, w->fb32);
  A((void**)&w->t3, w->fb32);
  A((void**)&w->e32, w->fb32);
  A((void**)&w->x64, w->fb64);
  A((void**)&w->r64, w->fb64);
  A((void**)&w->Vc, w->cb32 * (mcc + 1));
  A((void**)&w->xc, w->cb32);
  A((void**)&w->rc, w->cb32);
  A((void**)&w->tc, w->cb32);
  const size_t d = sizeof(double) * ns;
  A((void**)&w->rel_top, d);
  A((void**)&w->rel_coarse, d);
  A((void**)&w->rn, d);
  A((void**)&w->bn, d);
  A((void**)&w->scale, d);
  A((void**)&w->beta0, d);
  A((void**)&w->tmpd, d);
  A((void**)&w->ones, sizeof(double2) * ns);
  A((void**)&w->mones, sizeof(double2) * ns);
  A((void**)&w->dot, sizeof(double2) * ns * 4);
  w->partial64_cap = partial_elems(12 * V, ns, 1, 1);
  A((void**)&w->partial64, sizeof(double2) * w->partial64_cap);
  A((void**)&w->mask, sizeof(int) * ns);
  A((void**)&w->mask2, sizeof(int) * ns);
  A((void**)&w->flags, sizeof(int) * ns);
  A((void**)&w->count, sizeof(int));
  A((void**)&w->outer_it, sizeof(int) * ns);
  A((void**)&w->inner_it, sizeof(int) * ns);
  if (three) {
    A((void**)&w->Vm, w->mb32 * (mmm + 1));
    A((void**)&w->Zm, w->mb32 * mmm);
    A((void**)&w->xm, w->mb32);
    A((void**)&w->rm, w->mb32);
    A((void**)&w->sm1, w->mb32);
    A((void**)&w->sm2, w->mb32);
    A((void**)&w->rel_mid, d);
    A((void**)&w->beta0m, d);
    A((void**)&w->mra, sizeof(double2) * 2 * ns);
    A((void**)&w->mrd, sizeof(double2) * 2 * ns);
  }
  if (e == cudaSuccess) e = cudaMallocHost((void**)&w->h_count, sizeof(int));
  if (e != cudaSuccess) {
    ws_free(w);
    return check_cuda(ctx, e, "workspace allocation");
  }
  if (w->top.alloc(mm, ns, partial_elems(12 * V, ns, mm + 1, 2))) return set_err(ctx, TMAMG_ERR_OOM, "gmres state");
  if (w->coarse.alloc(mcc, ns, partial_elems((int64_t)nc * Vc, ns, mcc + 1, 2)))
    return set_err(ctx, TMAMG_ERR_OOM, "gmres state");
  if (three && w->mid.alloc(mmm, ns, partial_elems((int64_t)ncm * Vm, ns, mmm + 1, 2)))
    return set_err(ctx, TMAMG_ERR_OOM, "gmres state");
  // the grid for one tile is the largest any system count uses
  if (w->cg.alloc(mcc, ns, coarse_gmres_grid(1), w->cb32, cm_x16_bytes(Vc, nc, ns)))
    return set_err(ctx, TMAMG_ERR_OOM, "coarse gmres state");
  fill_c_kernel<<<(ns + 127) / 128, 128, 0, ctx->stream>>>(w->ones, ns, 1.0); TM_COUNT();
  fill_c_kernel<<<(ns + 127) / 128, 128, 0, ctx->stream>>>(w->mones, ns, -1.0); TM_COUNT();
  return check_cuda(ctx, cudaGetLastError(), "workspace init");
}

// the second FP32 scratch bundle of the workspace (used by the learned step only)
static int ensure_t2(tmamg_ctx* ctx) {
  Workspace* w = ctx->ws;
  if (w->t2) return TMAMG_OK;
  return check_cuda(ctx, cudaMalloc(&w->t2, w->fb32), "cudaMalloc(learned-step scratch)");
}

// the right-hand sides as FP64 bundles, one tile each (nrhs <= the workspace's system count)
static int ensure_b64(tmamg_ctx* ctx, int nrhs) {
  Workspace* w = ctx->ws;
  const size_t need = (size_t)nrhs * 12 * ctx->g.V * 2 * sizeof(double);
  if (need <= w->b64_bytes) return TMAMG_OK;
  cudaStreamSynchronize(ctx->stream);
  cudaFree(w->b64);
  w->b64 = nullptr;
  w->b64_bytes = 0;
  int rc = check_cuda(ctx, cudaMalloc(&w->b64, need), "cudaMalloc(right-hand sides)");
  if (!rc) w->b64_bytes = need;
  return rc;
}

// ------------------------------------------------------------------ setup
static AggDims agg_dims(const Geom& g, const int agg[4]) {
  AggDims a;
  a.asize = 1;
  a.Vc = 1;
  for (int k = 0; k < 4; ++k) {
    a.L[k] = g.L[k];
    a.agg[k] = agg[k];
    a.Lc[k] = g.L[k] / agg[k];
    a.asize *= agg[k];
    a.Vc *= a.Lc[k];
  }
  a.Vp = g.V;
  return a;
}

// aggregation of a coarse level's lattice (the parent of a further level)
static AggDims agg_dims_coarse(const CoarseLevel& parent, const int agg[4]) {
  AggDims a;
  a.asize = 1;
  a.Vc = 1;
  for (int k = 0; k < 4; ++k) {
    a.L[k] = parent.Lc[k];
    a.agg[k] = agg[k];
    a.Lc[k] = parent.Lc[k] / agg[k];
    a.asize *= agg[k];
    a.Vc *= a.Lc[k];
  }
  a.Vp = parent.Vc;
  return a;
}

static CoarseDims coarse_dims(const CoarseLevel& l) {
  CoarseDims c;
  for (int k = 0; k < 4; ++k) c.L[k] = l.Lc[k];
  c.Vc = l.Vc;
  c.nc = 2 * l.nv;
  return c;
}

// counter-based start vectors: splitmix64 -> uniform -> Box-Muller (complex Gaussian), generated
// on the device (element i of stream (seed, stream) uses counters 2 i and 2 i + 1 of its key)
__host__ __device__ inline uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void gaussian_kernel(uint64_t key, int64_t n, float2* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t a = splitmix64(key + 2 * (uint64_t)i), b = splitmix64(key + 2 * (uint64_t)i + 1);
  const double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740992.0);
  const double u2 = ((b >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  const double r = sqrt(-log(u1));  // variance 1/2 per component
  out[i] = make_float2((float)(r * cos(2 * M_PI * u2)), (float)(r * sin(2 * M_PI * u2)));
}

// the same numbers on the host (small draws: the learned step's start weights and gate right-hand sides)
static void host_gaussian(uint64_t seed, uint64_t stream, size_t n, std::vector<float>& out) {
  out.resize(2 * n);  // n complex numbers
  const uint64_t key = splitmix64(seed ^ stream);
  for (size_t i = 0; i < n; ++i) {
    const uint64_t a = splitmix64(key + 2 * i), b = splitmix64(key + 2 * i + 1);
    const double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740992.0);
    const double u2 = ((b >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double r = sqrt(-log(u1));
    out[2 * i] = (float)(r * cos(2 * M_PI * u2));
    out[2 * i + 1] = (float)(r * sin(2 * M_PI * u2));
  }
}

// n complex Gaussian numbers of the stream (seed, stream) into out (device)
static void device_gaussian(uint64_t seed, uint64_t stream, int64_t n, float2* out, cudaStream_t st) {
  const uint64_t key = splitmix64(seed ^ stream);
  gaussian_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(key, n, out); TM_COUNT();
}

__global__ void inv_sqrt_kernel(const double2* dot, double2* sc, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    double v = dot[i].x;
    sc[i] = make_double2(v > 0 ? 1.0 / sqrt(v) : 0.0, 0);
  }
}

// Level 2 on the lattice of level 1 (paper Sec. 2: the construction applied recursively): nv[1]
// test vectors on level 1, given (vec2_dev: complex float [nv2][Vc1][2 nv1], coarse component
// chi nv1 + j) or drawn from the generator, smoothed (if smooth) by setup_iters steps of inverse
// iteration w <- G(w) / |G(w)|, G = setup_gmres_steps steps of level-1 GMRES at mu_setup; then
// P2 (orthonormal per aggregate and chirality of gamma5_c) and D_c2 = P2^+ D_c1 P2.
static int setup_level2(tmamg_ctx* ctx, const tmamg_setup_params* p, const float* vec2_dev, bool smooth) {
  cudaStream_t st = ctx->stream;
  ctx->levels.reserve(2);  // the push_back below must not move level 1 (L1 refers to it)
  const CoarseLevel& L1 = ctx->levels[0];
  const CoarseDims cd1 = coarse_dims(L1);
  const int nv1 = L1.nv, nc1 = 2 * nv1, nv2 = p->nv[1], nc2 = 2 * nv2;
  const AggDims ad = agg_dims_coarse(L1, p->agg[1]);
  CoarseLevel lv;
  for (int k = 0; k < 4; ++k) {
    lv.Lc[k] = ad.Lc[k];
    lv.agg[k] = ad.agg[k];
  }
  lv.Vc = ad.Vc;
  lv.nv = nv2;
  lv.asize = ad.asize;
  int rc = check_cuda(ctx, cudaMalloc(&lv.P, sizeof(float2) * (size_t)ad.Vc * 2 * nv2 * ad.asize * nv1), "cudaMalloc(P2)");
  if (!rc) rc = check_cuda(ctx, cudaMalloc(&lv.A, sizeof(float2) * 9 * (size_t)ad.Vc * nc2 * nc2), "cudaMalloc(A2)");
  if (!rc && nc2 <= CM_MAXNC)
    rc = check_cuda(ctx, cudaMalloc(&lv.A16, (size_t)cm_site_bytes(nc2) * ad.Vc), "cudaMalloc(A2 f16)");
  if (!rc) rc = check_cuda(ctx, cudaMalloc(&lv.cmax, sizeof(float) * CM_MAXSYS), "cudaMalloc(cmax)");
  if (!rc) rc = check_cuda(ctx, cudaMalloc(&lv.cerr, sizeof(int)), "cudaMalloc(cerr)");
  if (!rc) rc = check_cuda(ctx, cudaMemsetAsync(lv.cerr, 0, sizeof(int), st), "cudaMemset(cerr)");
  if (rc) {
    cudaFree(lv.P);
    cudaFree(lv.A);
    cudaFree(lv.A16);
    cudaFree(lv.cmax);
    cudaFree(lv.cerr);
    return rc;
  }
  ctx->levels.push_back(lv);
  CoarseLevel& L2 = ctx->levels[1];
  const int64_t M1 = (int64_t)nc1 * L1.Vc;
  auto b1 = [&](int n) { return (size_t)ntiles(n, 2) * nc1 * L1.Vc * 4 * sizeof(float); };
  const int m = p->setup_gmres_steps;
  float *Wt = nullptr, *X = nullptr, *Vk = nullptr, *Wc = nullptr, *Yc = nullptr, *Rc = nullptr, *field = nullptr;
  double* mus = nullptr;
  double2 *dots = nullptr, *sc = nullptr, *part = nullptr;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** q, size_t b) {
    if (e == cudaSuccess) e = cudaMalloc(q, b);
  };
  A((void**)&Wt, b1(nv2));
  A((void**)&Wc, b1(nc2));
  A((void**)&Yc, b1(nc2));
  A((void**)&Rc, (size_t)ntiles(nc2, 2) * nc2 * L2.Vc * 4 * sizeof(float));
  const bool iterate = smooth && p->setup_iters > 0;
  CoarseGmres cg;
  if (iterate) {
    A((void**)&X, b1(nv2));
    A((void**)&Vk, b1(nv2) * (m + 1));
    A((void**)&mus, sizeof(double) * nv2);
    A((void**)&dots, sizeof(double2) * nv2);
    A((void**)&sc, sizeof(double2) * nv2);
    A((void**)&part, sizeof(double2) * partial_elems(M1, nv2, 1, 2));
  }
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    cudaFree(Wt); cudaFree(X); cudaFree(Vk); cudaFree(Wc); cudaFree(Yc); cudaFree(Rc); cudaFree(field);
    cudaFree(mus); cudaFree(dots); cudaFree(sc); cudaFree(part);
    cg.release();
  };
  if (e == cudaSuccess && iterate &&
      cg.alloc(m, nv2, coarse_gmres_grid(1), b1(nv2), cm_x16_bytes(L1.Vc, nc1, nv2)))
    e = cudaErrorMemoryAllocation;
  if (e != cudaSuccess) {
    cleanup();
    return check_cuda(ctx, e, "level-2 setup scratch");
  }
  if (!vec2_dev) {
    const int64_t n = (int64_t)nv2 * L1.Vc * nc1;
    e = cudaMalloc(&field, sizeof(float2) * n);
    if (e == cudaSuccess) device_gaussian(p->seed, 0x5eed2ULL, n, reinterpret_cast<float2*>(field), st);
    if (e != cudaSuccess) {
      cleanup();
      return check_cuda(ctx, e, "level-2 start vectors");
    }
    vec2_dev = field;
  }
  pack_coarse(vec2_dev, Wt, nv2, nc1, L1.Vc, st);
  if (iterate) {
    std::vector<double> hmu(nv2, p->mu_setup);
    cudaMemcpyAsync(mus, hmu.data(), sizeof(double) * nv2, cudaMemcpyHostToDevice, st);
    for (int it = 0; it < p->setup_iters && !rc; ++it) {
      int done = 0;
      // FP32 stencil (no A16): the test vectors decide the quality of the level, and the inverse
      // iteration costs little next to the solves
      const int r = coarse_gmres_solve(cg, cd1, L1.A, nullptr, Wt, X, Vk, (int64_t)(b1(nv2) / sizeof(float)), mus, 1.0,
                                       nv2, m, m, 0.0, &done, st);
      if (r == -3) rc = set_err(ctx, TMAMG_ERR_TIMEOUT, "setup: a level-1 GMRES bounded wait timed out");
      else if (r) rc = set_err(ctx, TMAMG_ERR_CUDA, "setup: level-1 GMRES launch failed");
      if (rc) break;
      mdot<float>(X, 0, 1, X, M1, nv2, dots, nv2, part, st);
      inv_sqrt_kernel<<<(nv2 + 127) / 128, 128, 0, st>>>(dots, sc, nv2); TM_COUNT();
      axpby<float>(sc, 2, X, nullptr, 0, Wt, M1, nv2, nullptr, st);
    }
  }
  if (!rc) {
    build_P(ad, Wt, L2.P, nv2, nv1, st);
    build_coarse_operator_coarse(ad, cd1, L1.A, L2.P, L2.A, nv2, Wc, Yc, Rc, st);
    if (L2.A16) pack_coarse_f16(coarse_dims(L2), L2.A, L2.A16, st);
    rc = check_cuda(ctx, cudaGetLastError(), "level-2 setup kernels");
  }
  cudaError_t se = cudaStreamSynchronize(st);
  cleanup();
  if (!rc) rc = check_cuda(ctx, se, "level-2 setup");
  return rc;
}

int do_setup(tmamg_ctx* ctx, const tmamg_setup_params* p, const float* vec_field_dev, bool smooth) {
  const Geom& g = ctx->g;
  cudaStream_t st = ctx->stream;
  std::string why;
  if (p->levels != 2 && p->levels != 3) return set_err(ctx, TMAMG_ERR_ARG, "setup: levels must be 2 or 3");
  if (sap_check_blocks(g, p->sap_block, why)) return set_err(ctx, TMAMG_ERR_ARG, "setup: " + why);
  int nv = p->nv[0];
  if (nv < 1 || nv > 32) return set_err(ctx, TMAMG_ERR_ARG, "setup: nv must be in [1, 32]");
  int asize = 1;
  for (int k = 0; k < 4; ++k) {
    if (p->agg[0][k] < 1 || g.L[k] % p->agg[0][k]) return set_err(ctx, TMAMG_ERR_ARG, "setup: aggregate must divide L");
    asize *= p->agg[0][k];
  }
  if (nv > 6 * asize) return set_err(ctx, TMAMG_ERR_ARG, "setup: nv exceeds the aggregate dimension");
  if (p->sap_cycles < 1 || p->sap_mr_steps < 1 || p->setup_iters < 0)
    return set_err(ctx, TMAMG_ERR_ARG, "setup: bad SAP parameters");
  if (p->levels == 3) {
    const int nv2 = p->nv[1];
    int asize2 = 1;
    for (int k = 0; k < 4; ++k) {
      const int lc = g.L[k] / p->agg[0][k];
      if (p->agg[1][k] < 1 || lc % p->agg[1][k])
        return set_err(ctx, TMAMG_ERR_ARG, "setup: level-2 aggregate must divide the level-1 lattice");
      asize2 *= p->agg[1][k];
    }
    if (nv2 < 1 || nv2 > 32) return set_err(ctx, TMAMG_ERR_ARG, "setup: nv[1] must be in [1, 32]");
    if (nv2 > nv * asize2) return set_err(ctx, TMAMG_ERR_ARG, "setup: nv[1] exceeds the level-2 aggregate dimension");
    if (p->setup_gmres_steps < 1 || p->setup_gmres_steps > 64)
      return set_err(ctx, TMAMG_ERR_ARG, "setup: setup_gmres_steps must be in [1, 64]");
  }
  free_levels(ctx);
  free_workspace(ctx);
  ctx->sp = *p;
  ctx->have_setup = false;
  AggDims ad = agg_dims(g, p->agg[0]);
  CoarseLevel lv;
  for (int k = 0; k < 4; ++k) {
    lv.Lc[k] = ad.Lc[k];
    lv.agg[k] = ad.agg[k];
  }
  lv.Vc = ad.Vc;
  lv.nv = nv;
  lv.asize = ad.asize;
  const int nc = 2 * nv;
  int rc = check_cuda(ctx, cudaMalloc(&lv.P, sizeof(float2) * (size_t)ad.Vc * 2 * nv * ad.asize * 6), "cudaMalloc(P)");
  if (!rc) rc = check_cuda(ctx, cudaMalloc(&lv.A, sizeof(float2) * 9 * (size_t)ad.Vc * nc * nc), "cudaMalloc(A)");
  if (!rc && nc <= CM_MAXNC)
    rc = check_cuda(ctx, cudaMalloc(&lv.A16, (size_t)cm_site_bytes(nc) * ad.Vc), "cudaMalloc(A16)");
  if (!rc) rc = check_cuda(ctx, cudaMalloc(&lv.cmax, sizeof(float) * CM_MAXSYS), "cudaMalloc(cmax)");
  if (!rc) rc = check_cuda(ctx, cudaMalloc(&lv.cerr, sizeof(int)), "cudaMalloc(cerr)");
  if (!rc) rc = check_cuda(ctx, cudaMemsetAsync(lv.cerr, 0, sizeof(int), st), "cudaMemset(cerr)");
  if (rc) {
    cudaFree(lv.P);
    cudaFree(lv.A);
    cudaFree(lv.A16);
    cudaFree(lv.cmax);
    cudaFree(lv.cerr);
    return rc;
  }
  ctx->levels.push_back(lv);
  // scratch: test vectors (nv systems), SAP buffers, columns (nc systems)
  size_t vb = (size_t)ntiles(nv, 2) * 12 * g.V * 4 * sizeof(float);
  size_t wb = (size_t)ntiles(nc, 2) * 12 * g.V * 4 * sizeof(float);
  size_t rb = (size_t)ntiles(nc, 2) * nc * ad.Vc * 4 * sizeof(float);
  float *Vt = nullptr, *R = nullptr, *E = nullptr, *Dl = nullptr, *W = nullptr, *Y = nullptr, *Rc = nullptr;
  double *mus = nullptr;
  double2 *dots = nullptr, *sc = nullptr, *part = nullptr;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** q, size_t b) {
    if (e == cudaSuccess) e = cudaMalloc(q, b);
  };
  A((void**)&Vt, vb);
  A((void**)&R, vb);
  A((void**)&E, vb);
  A((void**)&Dl, vb);
  A((void**)&W, wb);
  A((void**)&Y, wb);
  A((void**)&Rc, rb);
  A((void**)&mus, sizeof(double) * nv);
  A((void**)&dots, sizeof(double2) * nv);
  A((void**)&sc, sizeof(double2) * nv);
  size_t pe = partial_elems(12 * g.V, nv, 1, 2);
  A((void**)&part, sizeof(double2) * pe);
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    cudaFree(Vt); cudaFree(R); cudaFree(E); cudaFree(Dl); cudaFree(W); cudaFree(Y); cudaFree(Rc);
    cudaFree(mus); cudaFree(dots); cudaFree(sc); cudaFree(part);
  };
  if (e != cudaSuccess) {
    cleanup();
    return check_cuda(ctx, e, "setup scratch");
  }
  // start / test vectors as an FP32 bundle
  float* field = nullptr;
  if (!vec_field_dev) {
    const int64_t n = (int64_t)nv * g.V * 12;
    e = cudaMalloc(&field, sizeof(float2) * n);
    if (e == cudaSuccess) device_gaussian(p->seed, 0x5eedULL, n, reinterpret_cast<float2*>(field), st);
    if (e != cudaSuccess) {
      cudaFree(field);
      cleanup();
      return check_cuda(ctx, e, "start vectors");
    }
    launch_pack<float>(g, field, Vt, nv, st);
  } else {
    launch_pack<float>(g, vec_field_dev, Vt, nv, st);
  }
  std::vector<double> hmu(nv, p->mu_setup);
  cudaMemcpyAsync(mus, hmu.data(), sizeof(double) * nv, cudaMemcpyHostToDevice, st);
  const int64_t M = 12 * g.V;
  if (smooth) {
    for (int it = 0; it < p->setup_iters; ++it) {
      cudaMemcpyAsync(R, Vt, vb, cudaMemcpyDeviceToDevice, st);
      sap_apply(g, p->sap_block, ctx->U32, ctx->C32, R, E, Dl, mus, nv, p->sap_cycles, p->sap_mr_steps, st);
      mdot<float>(E, 0, 1, E, M, nv, dots, nv, part, st);
      inv_sqrt_kernel<<<(nv + 127) / 128, 128, 0, st>>>(dots, sc, nv); TM_COUNT();
      axpby<float>(sc, 2, E, nullptr, 0, Vt, M, nv, nullptr, st);
    }
  }
  CoarseLevel& L1 = ctx->levels[0];
  build_P(ad, Vt, L1.P, nv, 6, st);
  build_coarse_operator_fine(ad, ctx->U32, ctx->C32, L1.P, L1.A, nv, g.bc_t, W, Y, Rc, st);
  if (L1.A16) pack_coarse_f16(coarse_dims(L1), L1.A, L1.A16, st);
  rc = check_cuda(ctx, cudaGetLastError(), "setup kernels");
  cudaError_t se = cudaStreamSynchronize(st);
  cudaFree(field);
  cleanup();
  if (rc) return rc;
  rc = check_cuda(ctx, se, "setup");
  if (rc) return rc;
  if (p->levels == 3) {
    // level-2 vectors follow the nv fine fields in a caller's array
    const float* v2 = vec_field_dev ? vec_field_dev + (size_t)nv * g.V * 24 : nullptr;
    rc = setup_level2(ctx, p, v2, smooth);
    if (rc) return rc;
  }
  ctx->have_setup = true;
  return TMAMG_OK;
}

// ------------------------------------------------------------------ AMG cycle and solve
struct SolveCtx {
  tmamg_ctx* ctx;
  const tmamg_solve_params* sp;
  int nsys;
  const double* mu;  // device, per system
  int coarse_iters = 0;
  int mid_iters = 0;          // middle-level FGMRES steps (three levels)
  bool timeout = false;       // a bounded device wait gave up
  bool launch_error = false;  // a cooperative launch was refused
  int nshift = 1;             // systems n = r * nshift + k (block GMRES groups the rhs of shift k)
  int nn = 0;                 // apply the learned step in the AMG cycle
  const double* eps = nullptr;  // doublet solves: splitting per FP32 tile (the tile = one doublet), device
};

__global__ void restart_tol_kernel(const double2* dot, const double* beta0, double tol, double* rel, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double b = sqrt(fmax(dot[i].x, 0.0));
  rel[i] = b > 0 ? tol * beta0[i] / b : 1.0;
}

__global__ void copy_beta_kernel(const double* b, double* dst, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = b[i];
}

// y = D_c x on level l: FP16 operator on the tensor cores (precision 16, or 0 = default) or
// the FP32 stencil (precision 32); false if the sizes are outside the tensor-core path
static bool coarse_apply_level(CoarseLevel& l, int precision, const float* x, float* y, const double* mu, double dmu,
                               int nsys, cudaStream_t st, const double* eps = nullptr) {
  const CoarseDims cd = coarse_dims(l);
  if (precision != 32) {
    if (!l.A16 || nsys > CM_MAXSYS) return false;
    const size_t need = cm_x16_bytes(cd.Vc, cd.nc, nsys);
    if (need > l.x16_bytes) {  // grown once per system count; later calls reuse it
      cudaStreamSynchronize(st);
      cudaFree(l.x16);
      l.x16 = nullptr;
      l.x16_bytes = 0;
      if (cudaMalloc(&l.x16, need) != cudaSuccess) return false;
      l.x16_bytes = need;
    }
    return coarse_apply_f16(cd, l.A16, x, y, mu, dmu, nsys, l.cmax, l.x16, l.cerr, st, eps) == 0;
  }
  coarse_apply(cd, l.A, x, y, mu, dmu, nsys, st, eps);
  return true;
}

// the stand-alone tensor-core stencil records a bounded wait that gave up in l.cerr: read and clear
static bool coarse_apply_timed_out(const CoarseLevel& l, cudaStream_t st) {
  int h = 0;
  cudaMemcpyAsync(&h, l.cerr, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  if (h) cudaMemsetAsync(l.cerr, 0, sizeof(int), st);
  return h != 0;
}

// xc ~ D_c^{-1} rc on the bottom level by restarted GMRES to the relative residual coarse_tol
static void coarse_solve(SolveCtx& S, const float* rc, float* xc) {
  tmamg_ctx* ctx = S.ctx;
  Workspace* w = ctx->ws;
  cudaStream_t st = ctx->stream;
  CoarseLevel& L1 = ctx->levels.back();
  CoarseDims cd = coarse_dims(L1);
  if (S.sp->coarse_solver == 0) {
    // persistent kernel: the whole restarted GMRES in one cooperative launch
    int it = 0;
    const __half* A16 = S.sp->coarse_precision != 32 ? L1.A16 : nullptr;
    int rc_ = coarse_gmres_solve(w->cg, cd, L1.A, A16, rc, xc, w->Vc, (int64_t)(w->cb32 / sizeof(float)), S.mu,
                                 S.sp->delta_mu, S.nsys, S.sp->coarse_restart, S.sp->coarse_maxiter,
                                 S.sp->coarse_tol, &it, st);
    if (rc_ == -3) S.timeout = true;
    if (rc_ == -1 || rc_ == -2) S.launch_error = true;
    S.coarse_iters += it;
    return;
  }
  if (S.sp->coarse_solver == 1) {
    // block GMRES: one Krylov space per shift over that shift's right-hand sides
    const int64_t M = (int64_t)cd.nc * cd.Vc;
    if (w->bg.alloc(S.sp->coarse_restart, S.nsys, S.nshift, M)) {
      S.launch_error = true;
      return;
    }
    const double dmu = S.sp->delta_mu;
    const double* mu = S.mu;
    const int nsys = S.nsys;
    const int prec = S.sp->coarse_precision;
    auto apply = [&, dmu, mu, nsys, prec](const float* x, float* y) {
      if (!coarse_apply_level(L1, prec, x, y, mu, dmu, nsys, st, S.eps)) S.launch_error = true;
    };
    int it = 0;
    const size_t cbytes = (size_t)ntiles(nsys, 2) * M * 4 * sizeof(float);  // the caller's bundles hold nsys systems
    int rc_ = block_gmres_solve(w->bg, apply, rc, xc, w->Vc, (int64_t)(w->cb32 / sizeof(float)), w->tc, cbytes,
                                S.sp->coarse_restart, S.sp->coarse_maxiter, S.sp->coarse_tol, &it, st);
    if (rc_) S.launch_error = true;
    S.coarse_iters += it;
    return;
  }
  const int64_t M = (int64_t)cd.nc * cd.Vc;
  const int nsys = S.nsys;
  const int mc = S.sp->coarse_restart;
  const size_t vstride = w->cb32 / sizeof(float);
  LevelOps ops;
  ops.M = M;
  const double dmu = S.sp->delta_mu;
  const double* mu = S.mu;
  const int prec = S.sp->coarse_precision;
  ops.A = [&, dmu, mu, nsys, prec](const float* x, float* y) {
    if (!coarse_apply_level(L1, prec, x, y, mu, dmu, nsys, st, S.eps)) S.launch_error = true;
  };
  const size_t cbytes = (size_t)ntiles(nsys, 2) * M * 4 * sizeof(float);  // the caller's bundles hold nsys systems
  cudaMemsetAsync(xc, 0, cbytes, st);
  cudaMemcpyAsync(w->Vc, rc, cbytes, cudaMemcpyDeviceToDevice, st);
  set_rel_tol(w->rel_coarse, nsys, S.sp->coarse_tol, st);
  int done = 0;
  for (int cyc = 0; done < S.sp->coarse_maxiter; ++cyc) {
    int m = mc < S.sp->coarse_maxiter - done ? mc : S.sp->coarse_maxiter - done;
    CycleResult r = gmres_cycle<float>(w->coarse, ops, nsys, m, w->Vc, vstride, nullptr, xc, nullptr, w->rel_coarse,
                                S.sp->poll, false, st);
    done += r.iters;
    if (cyc == 0) copy_beta_kernel<<<(nsys + 127) / 128, 128, 0, st>>>(w->coarse.beta, w->beta0, nsys); TM_COUNT();
    if (r.iters < m || done >= S.sp->coarse_maxiter) break;  // every system converged inside the cycle
    // restart from the true coarse residual
    ops.A(xc, w->Vc);
    axpby<float>(w->ones, 2, rc, w->mones, 2, w->Vc, M, nsys, nullptr, st);
    mdot<float>(w->Vc, 0, 1, w->Vc, M, nsys, w->dot, nsys, w->coarse.partial, st);
    restart_tol_kernel<<<(nsys + 127) / 128, 128, 0, st>>>(w->dot, w->beta0, S.sp->coarse_tol, w->rel_coarse, nsys); TM_COUNT();
  }
  S.coarse_iters += done;
}

// MR coefficients from d[n] = <q, rho>, d[ns + n] = <q, q>: a[n] = d[n] / d[ns + n], a[ns + n] = -a[n]
__global__ void mr_coef_kernel(const double2* __restrict__ d, double2* __restrict__ a, int nsys, int ns) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nsys) return;
  const double qq = d[ns + n].x;
  const double2 al = qq > 0 ? make_double2(d[n].x / qq, d[n].y / qq) : make_double2(0, 0);
  a[n] = al;
  a[ns + n] = make_double2(-al.x, -al.y);
}

// z = M_1 v, the preconditioner of the middle FGMRES: level-2 correction z = P2 D_c2^{-1} P2^+ v,
// then mid_smooth minimal-residual steps on the level-1 residual v - D_c1 z (paper Sec. 2: the
// two-level construction applied to the coarse lattice)
static void mid_cycle(SolveCtx& S, const float* v, float* z) {
  tmamg_ctx* ctx = S.ctx;
  Workspace* w = ctx->ws;
  cudaStream_t st = ctx->stream;
  CoarseLevel& L1 = ctx->levels[0];
  const CoarseLevel& L2 = ctx->levels[1];
  const AggDims ad = agg_dims_coarse(L1, L2.agg);
  const int nsys = S.nsys;
  const int64_t M = (int64_t)2 * L1.nv * L1.Vc;
  restrict_vec(ad, L2.P, v, w->rc, L2.nv, L1.nv, nsys, st);
  coarse_solve(S, w->rc, w->xc);
  prolong_vec(ad, L2.P, w->xc, z, L2.nv, L1.nv, nsys, 0, st);
  const int steps = S.sp->mid_smooth;
  if (steps < 1) return;
  const int prec = S.sp->coarse_precision;
  const double dmu = 1.0;  // the twisted-mass factor delta_mu belongs to the bottom level only
  const int ns = w->nsys;
  auto apply = [&](const float* x, float* y) {
    if (!coarse_apply_level(L1, prec, x, y, S.mu, dmu, nsys, st, S.eps)) S.launch_error = true;
  };
  float* rho = w->sm1;
  float* q = w->sm2;
  apply(z, rho);
  axpby<float>(w->ones, 2, v, w->mones, 2, rho, M, nsys, nullptr, st);  // rho = v - D z
  for (int k = 0; k < steps; ++k) {
    apply(rho, q);
    mdot<float>(q, 0, 1, rho, M, nsys, w->mrd, ns, w->mid.partial, st);
    mdot<float>(q, 0, 1, q, M, nsys, w->mrd + ns, ns, w->mid.partial, st);
    mr_coef_kernel<<<(nsys + 127) / 128, 128, 0, st>>>(w->mrd, w->mra, nsys, ns); TM_COUNT();
    axpby<float>(w->mra, 2, rho, nullptr, 1, z, M, nsys, nullptr, st);                      // z += alpha rho
    if (k + 1 < steps) axpby<float>(w->mra + ns, 2, q, nullptr, 1, rho, M, nsys, nullptr, st);  // rho -= alpha q
  }
}

// xm ~ D_c1^{-1} rm on the middle level of a three-level hierarchy: restarted FGMRES(mid_restart)
// to the relative residual mid_tol per system (paper Sec. 4: r_m about 7e-2), preconditioned by
// mid_cycle, restarted from the true level-1 residual
static void mid_solve(SolveCtx& S, const float* rm, float* xm) {
  tmamg_ctx* ctx = S.ctx;
  Workspace* w = ctx->ws;
  cudaStream_t st = ctx->stream;
  CoarseLevel& L1 = ctx->levels[0];
  const int nsys = S.nsys;
  const int64_t M = (int64_t)2 * L1.nv * L1.Vc;
  const int mm = S.sp->mid_restart;
  if (!w->Vm || mm > w->mm) {  // the workspace was sized without a middle level
    S.launch_error = true;
    return;
  }
  const size_t vstride = w->mb32 / sizeof(float);
  const int prec = S.sp->coarse_precision;
  const double dmu = 1.0;  // the twisted-mass factor delta_mu belongs to the bottom level only
  LevelOps ops;
  ops.M = M;
  ops.A = [&](const float* x, float* y) {
    if (!coarse_apply_level(L1, prec, x, y, S.mu, dmu, nsys, st, S.eps)) S.launch_error = true;
  };
  ops.precond = [&](const float* v, float* z) { mid_cycle(S, v, z); };
  const size_t mbytes = (size_t)ntiles(nsys, 2) * M * 4 * sizeof(float);  // the caller's bundles hold nsys systems
  cudaMemsetAsync(xm, 0, mbytes, st);
  cudaMemcpyAsync(w->Vm, rm, mbytes, cudaMemcpyDeviceToDevice, st);
  set_rel_tol(w->rel_mid, nsys, S.sp->mid_tol, st);
  int done = 0;
  for (int cyc = 0; done < S.sp->mid_maxiter; ++cyc) {
    const int m = mm < S.sp->mid_maxiter - done ? mm : S.sp->mid_maxiter - done;
    CycleResult r = gmres_cycle<float>(w->mid, ops, nsys, m, w->Vm, vstride, w->Zm, xm, nullptr, w->rel_mid, 1, false,
                                       st);
    done += r.iters;
    S.mid_iters += r.iters;
    if (cyc == 0) copy_beta_kernel<<<(nsys + 127) / 128, 128, 0, st>>>(w->mid.beta, w->beta0m, nsys); TM_COUNT();
    if (r.iters < m || done >= S.sp->mid_maxiter) break;
    ops.A(xm, w->Vm);
    axpby<float>(w->ones, 2, rm, w->mones, 2, w->Vm, M, nsys, nullptr, st);
    mdot<float>(w->Vm, 0, 1, w->Vm, M, nsys, w->dot, nsys, w->mid.partial, st);
    restart_tol_kernel<<<(nsys + 127) / 128, 128, 0, st>>>(w->dot, w->beta0m, S.sp->mid_tol, w->rel_mid, nsys); TM_COUNT();
  }
}

// z = M v: coarse-grid correction then SAP post-smoothing (paper Sec. 2)
static void amg_cycle(SolveCtx& S, const float* v, float* z) {
  tmamg_ctx* ctx = S.ctx;
  Workspace* w = ctx->ws;
  cudaStream_t st = ctx->stream;
  const CoarseLevel& L1 = ctx->levels[0];
  AggDims ad = agg_dims(ctx->g, L1.agg);
  const int nsys = S.nsys;
  const int nv = L1.nv;
  const int64_t M = 12 * ctx->g.V;
  if (has_middle(ctx)) {
    restrict_vec(ad, L1.P, v, w->rm, nv, 6, nsys, st);
    mid_solve(S, w->rm, w->xm);
    prolong_vec(ad, L1.P, w->xm, z, nv, 6, nsys, 0, st);
  } else {
    restrict_vec(ad, L1.P, v, w->rc, nv, 6, nsys, st);
    coarse_solve(S, w->rc, w->xc);
    prolong_vec(ad, L1.P, w->xc, z, nv, 6, nsys, 0, st);
  }
  launch_residual32(ctx->g, ctx->U32, ctx->C32, z, v, w->t1, S.mu, nsys, st, S.eps);  // t1 = v - D z
  // z += SAP(t1): the block solver adds its corrections to z directly
  const int cyc = S.sp->sap_cycles > 0 ? S.sp->sap_cycles : ctx->sp.sap_cycles;
  const int mrs = S.sp->sap_mr_steps > 0 ? S.sp->sap_mr_steps : ctx->sp.sap_mr_steps;
  sap_apply(ctx->g, ctx->sp.sap_block, ctx->U32, ctx->C32, w->t1, z, w->t3, S.mu, nsys, cyc, mrs, st, true, S.eps);
  if (S.nn && ctx->nn && ctx->nn->trained) {
    // learned step on the residual left by the smoother: z += N(v - D z)
    NNState& nns = *ctx->nn;
    NNGeom ng{{ctx->g.L[0], ctx->g.L[1], ctx->g.L[2], ctx->g.L[3]}, ctx->g.V, ctx->g.bc_t};
    launch_dirac<float>(ctx->g, ctx->U32, ctx->C32, z, w->t1, S.mu, nsys, st);
    axpby<float>(w->ones, 2, v, w->mones, 2, w->t1, M, nsys, nullptr, st);
    nn_forward(nns, ng, ctx->U32, w->t1, w->t2, nsys, true, st);
    axpby<float>(w->ones, 2, w->t2, w->ones, 2, z, M, nsys, nullptr, st);
  }
}

// expand b [nrhs][V][12] (complex double) to the FP64 bundle of nsys = nrhs * nshift systems
__global__ void expand_b_kernel(const double* __restrict__ b, double* __restrict__ b64, int nshift, int nsys,
                                int64_t V) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nsys * 12 * V) return;
  int64_t s = t % V;
  int comp = (int)((t / V) % 12);
  int n = (int)(t / (12 * V));
  int r = n / nshift;
  const double* src = b + (((int64_t)r * V + s) * 12 + comp) * 2;
  double* dst = b64 + t * 2;
  dst[0] = src[0];
  dst[1] = src[1];
}

// r (FP64 bundle of nsys = nrhs * nshift systems) = the right-hand-side tiles b (one per rhs):
// system n takes tile n / nshift; per = complex entries per tile. Doublets (pair): system
// n = 2 (r nshift + k) + f takes the tile of rhs r, flavour f: 2 r + f
__global__ void expand_rhs_kernel(const double2* __restrict__ b, double2* __restrict__ r, int nshift, int nsys,
                                  int64_t per, int pair) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nsys * per) return;
  const int n = (int)(t / per);
  const int bt = pair ? ((n >> 1) / nshift) * 2 + (n & 1) : n / nshift;
  r[t] = b[(int64_t)bt * per + t % per];
}

// norms -> masks, scales and inner tolerances; flags: 1 = non-finite
__global__ void outer_check_kernel(const double2* __restrict__ dot, const double* __restrict__ bn, double tol,
                                   double inner_min, double* rn, double* scale, double* rel, int* mask, int* flags,
                                   int* count, int* outer_it, int nsys) {
  int n = threadIdx.x;
  int on = 0;
  if (n < nsys) {
    double r = sqrt(fmax(dot[n].x, 0.0));
    bool finite = isfinite(dot[n].x) && isfinite(bn[n]);
    if (!finite) flags[n] = 1;
    on = finite && !flags[n] && r > tol * bn[n];
    rn[n] = r;
    scale[n] = on ? 1.0 / r : 0.0;
    double want = on ? 0.5 * tol * bn[n] / r : 1.0;
    rel[n] = want > inner_min ? (want < 0.5 ? want : 0.5) : inner_min;
    mask[n] = on;
    if (on) outer_it[n] += 1;
  }
  int c = __syncthreads_count(on);
  if (n == 0) *count = c;
}

__global__ void sqrt_kernel(const double2* dot, double* out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = sqrt(fmax(dot[i].x, 0.0));
}

// after an FP32 inner cycle: the systems whose FGMRES residual is still above the cycle's goal
// keep iterating (mask2), counted in *count
__global__ void inner_check_kernel(const double* __restrict__ resid, const double* __restrict__ tolabs, int* mask2,
                                   int* count, int nsys) {
  const int n = threadIdx.x;
  int on = 0;
  if (n < nsys) {
    on = mask2[n] && resid[n] > tolabs[n];
    mask2[n] = on;
  }
  const int c = __syncthreads_count(on);
  if (n == 0) *count = c;
}

// goal of the next inner cycle relative to its start residual (norms from dot): the absolute goal
// rel0 (in units of the refinement cycle's normalised residual) over the new start norm
__global__ void inner_rel_kernel(const double2* __restrict__ dot, const double* __restrict__ rel0, double* rel,
                                 int nsys) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nsys) return;
  const double b = sqrt(fmax(dot[n].x, 0.0));
  rel[n] = b > 0 ? fmin(rel0[n] / b, 1.0) : 1.0;
}

__global__ void add_iters_kernel(const int* kconv, const int* mask, int* it, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && mask[i]) it[i] += kconv[i];
}

// ------------------------------------------------------------------ plain FP64 solver
// The comparator of the batched mixed-precision solver: FGMRES(m) in FP64 preconditioned by the
// same two-level AMG cycle (restriction, coarse GMRES to coarse_tol, prolongation, red-black
// SAP) with every vector, operator and reduction in FP64, one system per bundle tile, no
// refinement loop, no learned step. Restarted until every system's true FP64 residual meets tol.
static int ensure_ws64(tmamg_ctx* ctx, int nsys, int m, int mc) {
  if (!ctx->ws64) ctx->ws64 = new Workspace64();
  Workspace64* w = ctx->ws64;
  const CoarseLevel& L1 = ctx->levels[0];
  if (nsys <= w->nsys && m <= w->m && mc <= w->mc && w->Vc == L1.Vc && w->nc == 2 * L1.nv) return 0;
  const int ns = nsys > w->nsys ? nsys : w->nsys, mm = m > w->m ? m : w->m, mcc = mc > w->mc ? mc : w->mc;
  ws64_free(w);
  w->nsys = ns;
  w->m = mm;
  w->mc = mcc;
  w->Vc = L1.Vc;
  w->nc = 2 * L1.nv;
  const int64_t V = ctx->g.V;
  w->fb = (size_t)ns * 12 * V * 2 * sizeof(double);
  w->cb = (size_t)ns * w->nc * w->Vc * 2 * sizeof(double);
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  A((void**)&w->V, w->fb * (mm + 1));
  A((void**)&w->Z, w->fb * mm);
  A((void**)&w->x, w->fb);
  A((void**)&w->b, w->fb);
  A((void**)&w->t1, w->fb);
  A((void**)&w->t2, w->fb);
  A((void**)&w->t3, w->fb);
  A((void**)&w->Vc_, w->cb * (mcc + 1));
  A((void**)&w->xc, w->cb);
  A((void**)&w->rc, w->cb);
  A((void**)&w->rel_top, sizeof(double) * ns);
  A((void**)&w->rel_coarse, sizeof(double) * ns);
  A((void**)&w->beta0, sizeof(double) * ns);
  A((void**)&w->bn, sizeof(double) * ns);
  A((void**)&w->rn, sizeof(double) * ns);
  A((void**)&w->dot, sizeof(double2) * ns);
  A((void**)&w->partial, sizeof(double2) * partial_elems(12 * V, ns, 1, 1));
  A((void**)&w->ones, sizeof(double2) * ns);
  A((void**)&w->mones, sizeof(double2) * ns);
  if (e != cudaSuccess) {
    ws64_free(w);
    return check_cuda(ctx, e, "FP64 workspace allocation");
  }
  if (w->top.alloc(mm, ns, partial_elems(12 * V, ns, mm + 1, 1)) ||
      w->coarse.alloc(mcc, ns, partial_elems((int64_t)w->nc * w->Vc, ns, mcc + 1, 1)))
    return set_err(ctx, TMAMG_ERR_OOM, "FP64 gmres state");
  fill_c_kernel<<<(ns + 127) / 128, 128, 0, ctx->stream>>>(w->ones, ns, 1.0); TM_COUNT();
  fill_c_kernel<<<(ns + 127) / 128, 128, 0, ctx->stream>>>(w->mones, ns, -1.0); TM_COUNT();
  return check_cuda(ctx, cudaGetLastError(), "FP64 workspace init");
}

// xc ~ D_c^{-1} rc in FP64: restarted GMRES to coarse_tol (at most coarse_maxiter steps)
static int coarse_solve64(tmamg_ctx* ctx, const tmamg_solve_params* sp, int nsys, const double* mu) {
  Workspace64* w = ctx->ws64;
  cudaStream_t st = ctx->stream;
  const CoarseLevel& L1 = ctx->levels[0];
  const CoarseDims cd = coarse_dims(L1);
  const int64_t Mc = (int64_t)cd.nc * cd.Vc;
  LevelOpsT<double> ops;
  ops.M = Mc;
  const double dmu = sp->delta_mu;
  ops.A = [&, dmu](const double* xx, double* yy) { coarse_apply64(cd, L1.A64, xx, yy, mu, dmu, nsys, st); };
  const int64_t cvs = (int64_t)(w->cb / sizeof(double));
  cudaMemsetAsync(w->xc, 0, w->cb, st);
  cudaMemcpyAsync(w->Vc_, w->rc, w->cb, cudaMemcpyDeviceToDevice, st);
  set_rel_tol(w->rel_coarse, nsys, sp->coarse_tol, st);
  int done = 0;
  for (int cyc = 0; done < sp->coarse_maxiter; ++cyc) {
    const int m = sp->coarse_restart < sp->coarse_maxiter - done ? sp->coarse_restart : sp->coarse_maxiter - done;
    const CycleResult r = gmres_cycle<double>(w->coarse, ops, nsys, m, w->Vc_, cvs, nullptr, w->xc, nullptr,
                                              w->rel_coarse, sp->poll, false, st);
    done += r.iters;
    if (cyc == 0) {
      copy_beta_kernel<<<(nsys + 127) / 128, 128, 0, st>>>(w->coarse.beta, w->beta0, nsys); TM_COUNT();
    }
    if (r.iters < m || done >= sp->coarse_maxiter) break;
    ops.A(w->xc, w->Vc_);
    axpby<double>(w->ones, 2, w->rc, w->mones, 2, w->Vc_, Mc, nsys, nullptr, st);
    mdot<double>(w->Vc_, 0, 1, w->Vc_, Mc, nsys, w->dot, nsys, w->coarse.partial, st);
    restart_tol_kernel<<<(nsys + 127) / 128, 128, 0, st>>>(w->dot, w->beta0, sp->coarse_tol, w->rel_coarse, nsys);
    TM_COUNT();
  }
  return done;
}

// z = M v in FP64: coarse-grid correction, then SAP on the remaining residual
static void amg_cycle64(tmamg_ctx* ctx, const tmamg_solve_params* sp, int nsys, const double* mu, const double* v,
                        double* z, int& coarse_iters) {
  Workspace64* w = ctx->ws64;
  cudaStream_t st = ctx->stream;
  const CoarseLevel& L1 = ctx->levels[0];
  const AggDims ad = agg_dims(ctx->g, L1.agg);
  const int64_t M = 12 * ctx->g.V;
  restrict64(ad, L1.P64, v, w->rc, L1.nv, 6, nsys, st);
  coarse_iters += coarse_solve64(ctx, sp, nsys, mu);
  prolong64(ad, L1.P64, w->xc, z, L1.nv, 6, nsys, st);
  launch_dirac<double>(ctx->g, ctx->U64, ctx->C64, z, w->t1, mu, nsys, st);
  axpby<double>(w->ones, 2, v, w->mones, 2, w->t1, M, nsys, nullptr, st);  // t1 = v - D z
  sap_apply64(ctx->g, ctx->sp.sap_block, ctx->U64, ctx->C64, w->t1, w->t2, w->t3, mu, nsys,
              sp->sap_cycles > 0 ? sp->sap_cycles : ctx->sp.sap_cycles,
              sp->sap_mr_steps > 0 ? sp->sap_mr_steps : ctx->sp.sap_mr_steps, st);
  axpby<double>(w->ones, 2, w->t2, w->ones, 2, z, M, nsys, nullptr, st);  // z += SAP
}

int do_solve64(tmamg_ctx* ctx, const double* b, int nrhs, const double* mu, int nshift, double* x, int on_device,
               const tmamg_solve_params* sp, tmamg_system_stats* stats) {
  cudaStream_t st = ctx->stream;
  const Geom& g = ctx->g;
  const int nsys = nrhs * nshift;
  CoarseLevel& L1 = ctx->levels[0];
  const int nc = 2 * L1.nv;
  const int64_t V = g.V, M = 12 * V;
  int rc = 0;
  if (!L1.P64) {
    const int64_t np = L1.Vc * 2 * L1.nv * L1.asize * 6, na = 9 * L1.Vc * nc * nc;
    rc = check_cuda(ctx, cudaMalloc(&L1.P64, sizeof(double2) * np), "cudaMalloc(P64)");
    if (!rc) rc = check_cuda(ctx, cudaMalloc(&L1.A64, sizeof(double2) * na), "cudaMalloc(A64)");
    if (rc) return rc;
    widen_f2(L1.P, L1.P64, np, st);
    widen_f2(L1.A, L1.A64, na, st);
  }
  rc = ensure_ws64(ctx, nsys, sp->restart, sp->coarse_restart);
  if (rc) return rc;
  Workspace64* w = ctx->ws64;
  std::vector<double> musys(nsys);
  for (int n = 0; n < nsys; ++n) musys[n] = mu[n % nshift];
  rc = upload_mu(ctx, musys.data(), nsys);
  if (rc) return rc;
  const double* mud = ctx->mu_dev;
  const double* bsrc = b;
  double* bstage = nullptr;
  if (!on_device) {
    const size_t bytes = sizeof(double) * 2 * M * nrhs;
    rc = check_cuda(ctx, cudaMalloc(&bstage, bytes), "cudaMalloc(b staging)");
    if (rc) return rc;
    cudaMemcpyAsync(bstage, b, bytes, cudaMemcpyHostToDevice, st);
    bsrc = bstage;
  }
  expand_b_kernel<<<(unsigned)(((int64_t)nsys * M + 255) / 256), 256, 0, st>>>(bsrc, w->b, nshift, nsys, V); TM_COUNT();
  mdot<double>(w->b, 0, 1, w->b, M, nsys, w->dot, nsys, w->partial, st);
  sqrt_kernel<<<(nsys + 127) / 128, 128, 0, st>>>(w->dot, w->bn, nsys); TM_COUNT();
  cudaMemsetAsync(w->x, 0, w->fb, st);
  cudaMemcpyAsync(w->V, w->b, w->fb, cudaMemcpyDeviceToDevice, st);
  set_rel_tol(w->rel_top, nsys, sp->tol, st);
  int coarse_iters = 0, inner = 0, cycles = 0;
  LevelOpsT<double> fine;
  fine.M = M;
  fine.A = [&](const double* xx, double* yy) { launch_dirac<double>(g, ctx->U64, ctx->C64, xx, yy, mud, nsys, st); };
  fine.precond = [&](const double* v, double* z) { amg_cycle64(ctx, sp, nsys, mud, v, z, coarse_iters); };
  const int64_t vs = (int64_t)(w->fb / sizeof(double));
  std::vector<double> hrn(nsys), hbn(nsys);
  const int max_cycles = 8 * sp->max_outer;
  for (; cycles < max_cycles;) {
    const CycleResult r = gmres_cycle<double>(w->top, fine, nsys, sp->restart, w->V, vs, w->Z, w->x, nullptr,
                                              w->rel_top, 1, false, st);
    inner += r.iters;
    ++cycles;
    // true residual b - D x in FP64
    launch_dirac<double>(g, ctx->U64, ctx->C64, w->x, w->t1, mud, nsys, st);
    axpby<double>(w->ones, 2, w->b, w->mones, 2, w->t1, M, nsys, nullptr, st);
    mdot<double>(w->t1, 0, 1, w->t1, M, nsys, w->dot, nsys, w->partial, st);
    sqrt_kernel<<<(nsys + 127) / 128, 128, 0, st>>>(w->dot, w->rn, nsys); TM_COUNT();
    cudaMemcpyAsync(hrn.data(), w->rn, sizeof(double) * nsys, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(hbn.data(), w->bn, sizeof(double) * nsys, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    bool all = true;
    for (int n = 0; n < nsys; ++n) all &= !(hrn[n] > sp->tol * hbn[n]);
    if (all || r.iters == 0) break;
    cudaMemcpyAsync(w->V, w->t1, w->fb, cudaMemcpyDeviceToDevice, st);
    restart_tol_kernel<<<(nsys + 127) / 128, 128, 0, st>>>(w->dot, w->bn, sp->tol, w->rel_top, nsys); TM_COUNT();
  }
  double* xdst = x;
  double* xstage = nullptr;
  const size_t xbytes = sizeof(double) * 2 * M * nsys;
  if (!on_device) {
    cudaMalloc(&xstage, xbytes);
    xdst = xstage;
  }
  launch_unpack<double>(g, w->x, xdst, nsys, st);
  if (!on_device) cudaMemcpyAsync(x, xstage, xbytes, cudaMemcpyDeviceToHost, st);
  const cudaError_t le = cudaGetLastError();
  const cudaError_t se = cudaStreamSynchronize(st);
  cudaFree(bstage);
  cudaFree(xstage);
  rc = check_cuda(ctx, le, "FP64 solve kernels");
  if (!rc) rc = check_cuda(ctx, se, "FP64 solve");
  if (rc) return rc;
  int all_ok = 1;
  for (int n = 0; n < nsys; ++n) {
    const double rel = hbn[n] > 0 ? hrn[n] / hbn[n] : 0.0;
    const bool finite = std::isfinite(rel);
    const int status = !finite ? TMAMG_ERR_NONFINITE : (rel <= sp->tol ? TMAMG_OK : TMAMG_NOT_CONVERGED);
    if (status != TMAMG_OK) all_ok = 0;
    if (stats) {
      stats[n].status = status;
      stats[n].outer_iters = cycles;
      stats[n].inner_iters = inner;
      stats[n].coarse_iters = coarse_iters;
      stats[n].true_rel_res = finite ? rel : NAN;
    }
  }
  return all_ok ? TMAMG_OK : TMAMG_NOT_CONVERGED;
}

// eps_host (doublets): the splitting per shift; every (rhs, shift) is then a non-degenerate doublet whose
// flavours u, d are the systems 2p, 2p + 1 (one FP32 tile), p = r nshift + k, twisted masses +mu_k, -mu_k
int do_solve(tmamg_ctx* ctx, const double* b, int nrhs, const double* mu, int nshift, double* x, int on_device,
             const tmamg_solve_params* sp_in, tmamg_system_stats* stats, const double* eps_host) {
  cudaStream_t st = ctx->stream;
  const Geom& g = ctx->g;
  const bool pair = eps_host != nullptr;
  const int nsys = nrhs * nshift * (pair ? 2 : 1);
  const int nfields = nrhs * (pair ? 2 : 1);  // right-hand-side fields
  if (nsys > 256) return set_err(ctx, TMAMG_ERR_ARG, "solve: at most 256 systems per call");
  tmamg_solve_params spl = *sp_in;
  if (pair) {
    if (spl.precision != 32) return set_err(ctx, TMAMG_ERR_ARG, "solve: doublets run in the mixed-precision form");
    if (spl.coarse_solver == 1) return set_err(ctx, TMAMG_ERR_ARG, "solve: no block GMRES for doublets");
    if (spl.use_nn) return set_err(ctx, TMAMG_ERR_ARG, "solve: no learned step for doublets");
    // the per-launch coarse GMRES: its reductions go through the folded dots (one system per doublet)
    if (spl.coarse_solver == 0) spl.coarse_solver = 2;
  }
  const tmamg_solve_params* sp = &spl;
  PairFold fold(pair);
  if (sp->restart < 1 || sp->restart > 64 || sp->coarse_restart < 1 || sp->coarse_restart > 128 ||
      sp->coarse_maxiter < 1 || !(sp->tol > 0) || sp->max_outer < 1 || sp->inner_cycles < 1 || sp->sap_cycles < 0 ||
      sp->sap_mr_steps < 0)
    return set_err(ctx, TMAMG_ERR_ARG, "solve: bad parameters");
  if (has_middle(ctx) &&
      (sp->mid_restart < 1 || sp->mid_restart > 64 || sp->mid_maxiter < 1 || !(sp->mid_tol > 0) || sp->mid_smooth < 0))
    return set_err(ctx, TMAMG_ERR_ARG, "solve: bad middle-level parameters");
  if (sp->precision == 64) {
    if (has_middle(ctx))
      return set_err(ctx, TMAMG_ERR_ARG, "solve: the FP64 comparator (precision 64) takes a two-level hierarchy");
    return do_solve64(ctx, b, nrhs, mu, nshift, x, on_device, sp, stats);
  }
  if (sp->precision != 32) return set_err(ctx, TMAMG_ERR_ARG, "solve: precision must be 32 or 64");
  if (sp->coarse_precision != 0 && sp->coarse_precision != 16 && sp->coarse_precision != 32)
    return set_err(ctx, TMAMG_ERR_ARG, "solve: coarse_precision must be 16 or 32");
  if (sp->coarse_solver < 0 || sp->coarse_solver > 2)
    return set_err(ctx, TMAMG_ERR_ARG, "solve: coarse_solver must be 0, 1 or 2");
  if (sp->coarse_solver == 1 && nrhs > 16)
    return set_err(ctx, TMAMG_ERR_ARG, "solve: block GMRES takes at most 16 right-hand sides per shift");
  int rc = ensure_ws(ctx, nsys, *sp);
  if (!rc) rc = ensure_b64(ctx, nfields);
  if (rc) return rc;
  Workspace* w = ctx->ws;
  const int64_t V = g.V;
  const int64_t M = 12 * V;
  // per-system twisted masses: system n = rhs (n / nshift), shift (n % nshift); doublets: +mu, -mu
  std::vector<double> musys(nsys);
  for (int n = 0; n < nsys; ++n)
    musys[n] = pair ? ((n & 1) ? -mu[(n >> 1) % nshift] : mu[(n >> 1) % nshift]) : mu[n % nshift];
  rc = upload_mu(ctx, musys.data(), nsys);
  if (rc) return rc;
  if (pair) {
    const int np = nsys / 2;
    if (np > w->eps_cap) {
      cudaStreamSynchronize(st);
      cudaFree(w->epsd);
      w->epsd = nullptr;
      w->eps_cap = 0;
      rc = check_cuda(ctx, cudaMalloc(&w->epsd, sizeof(double) * np), "cudaMalloc(splittings)");
      if (rc) return rc;
      w->eps_cap = np;
    }
    std::vector<double> ep(np);
    for (int q = 0; q < np; ++q) ep[q] = eps_host[q % nshift];
    rc = check_cuda(ctx, cudaMemcpyAsync(w->epsd, ep.data(), sizeof(double) * np, cudaMemcpyHostToDevice, st),
                    "upload splittings");
    if (!rc) rc = check_cuda(ctx, cudaStreamSynchronize(st), "upload splittings");
    if (rc) return rc;
  }
  // b -> FP64 bundle with one tile per right-hand side (host input staged through x64, which
  // holds nsys >= nrhs fields and is cleared right after)
  const double* bsrc = b;
  if (!on_device) {
    cudaMemcpyAsync(w->x64, b, sizeof(double) * 2 * M * nfields, cudaMemcpyHostToDevice, st);
    bsrc = w->x64;
  }
  launch_pack<double>(g, bsrc, w->b64, nfields, st);
  expand_rhs_kernel<<<(unsigned)(((int64_t)nsys * M + 255) / 256), 256, 0, st>>>(
      reinterpret_cast<const double2*>(w->b64), reinterpret_cast<double2*>(w->r64), nshift, nsys, M, pair ? 1 : 0);
  TM_COUNT();
  cudaMemsetAsync(w->x64, 0, w->fb64, st);
  cudaMemsetAsync(w->flags, 0, sizeof(int) * nsys, st);
  cudaMemsetAsync(w->outer_it, 0, sizeof(int) * nsys, st);
  cudaMemsetAsync(w->inner_it, 0, sizeof(int) * nsys, st);
  mdot<double>(w->r64, 0, 1, w->r64, M, nsys, w->dot, nsys, w->partial64, st);
  sqrt_kernel<<<(nsys + 127) / 128, 128, 0, st>>>(w->dot, w->bn, nsys); TM_COUNT();
  SolveCtx S{ctx, sp, nsys, ctx->mu_dev, 0};
  S.nshift = nshift;
  S.eps = pair ? w->epsd : nullptr;
  S.nn = sp->use_nn == 2 || (sp->use_nn == 1 && ctx->nn && ctx->nn->enabled);
  if (S.nn && (!ctx->nn || !ctx->nn->trained)) return set_err(ctx, TMAMG_ERR_STATE, "solve: no trained network");
  if (S.nn) {
    if (ctx->nn->alloc(ctx->g.V, nsys)) return set_err(ctx, TMAMG_ERR_OOM, "solve: network buffers");
    rc = ensure_t2(ctx);
    if (rc) return rc;
  }
  LevelOps fine;
  fine.M = M;
  fine.A = [&](const float* xx, float* yy) {
    launch_dirac<float>(g, ctx->U32, ctx->C32, xx, yy, ctx->mu_dev, nsys, st, S.eps);
  };
  fine.precond = [&](const float* v, float* z) { amg_cycle(S, v, z); };
  const size_t vstride = w->fb32 / sizeof(float);
  const double inner_min = 2e-6;
  int outer = 0;
  for (; outer < sp->max_outer + 1; ++outer) {
    mdot<double>(w->r64, 0, 1, w->r64, M, nsys, w->dot, nsys, w->partial64, st);
    outer_check_kernel<<<1, 1024, 0, st>>>(w->dot, w->bn, sp->tol, inner_min, w->rn, w->scale, w->rel_top, w->mask,
                                          w->flags, w->count, w->outer_it, nsys); TM_COUNT();
    cudaMemcpyAsync(w->h_count, w->count, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    if (*w->h_count == 0 || outer == sp->max_outer) break;
    f64_to_f32(w->r64, w->scale, w->V, M, nsys, st);
    cudaMemsetAsync(w->e32, 0, w->fb32, st);
    cudaMemcpyAsync(w->mask2, w->mask, sizeof(int) * nsys, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(w->tmpd, w->rel_top, sizeof(double) * nsys, cudaMemcpyDeviceToDevice, st);
    for (int ic = 0; ic < sp->inner_cycles; ++ic) {
      gmres_cycle<float>(w->top, fine, nsys, sp->restart, w->V, vstride, w->Z, w->e32, w->mask2, w->rel_top, 1, false,
                         st);
      add_iters_kernel<<<(nsys + 127) / 128, 128, 0, st>>>(w->top.kconv, w->mask2, w->inner_it, nsys); TM_COUNT();
      if (ic + 1 == sp->inner_cycles) break;
      inner_check_kernel<<<1, 1024, 0, st>>>(w->top.resid, w->top.tolabs, w->mask2, w->count, nsys); TM_COUNT();
      cudaMemcpyAsync(w->h_count, w->count, sizeof(int), cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
      if (*w->h_count == 0) break;
      // restart from the FP32 residual of the inner problem: V0 = r / |r| - D e32
      f64_to_f32(w->r64, w->scale, w->V, M, nsys, st);
      launch_residual32(g, ctx->U32, ctx->C32, w->e32, w->V, w->V, ctx->mu_dev, nsys, st, S.eps);
      mdot<float>(w->V, 0, 1, w->V, M, nsys, w->dot, nsys, w->top.partial, st);
      inner_rel_kernel<<<(nsys + 127) / 128, 128, 0, st>>>(w->dot, w->tmpd, w->rel_top, nsys); TM_COUNT();
    }
    f32_axpy_f64(w->rn, w->e32, w->x64, M, nsys, w->mask, st);
    // r = b - D x in FP64 in one pass (the stencil's residual form)
    launch_residual64(g, ctx->U64, ctx->C64, w->x64, w->b64, nshift, w->r64, ctx->mu_dev, nsys, st, S.eps);
  }
  rc = check_cuda(ctx, cudaGetLastError(), "solve kernels");
  // final true residual per system (r64 holds b - D x for the current x)
  std::vector<double> hrn(nsys), hbn(nsys);
  std::vector<int> hflags(nsys), hout(nsys), hin(nsys), hmask(nsys);
  // the loop left at the refinement cap if systems were still active: their last check counted a
  // cycle that did not run
  const bool capped = *w->h_count != 0;
  cudaMemcpyAsync(hmask.data(), w->mask, sizeof(int) * nsys, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(hrn.data(), w->rn, sizeof(double) * nsys, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(hbn.data(), w->bn, sizeof(double) * nsys, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(hflags.data(), w->flags, sizeof(int) * nsys, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(hout.data(), w->outer_it, sizeof(int) * nsys, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(hin.data(), w->inner_it, sizeof(int) * nsys, cudaMemcpyDeviceToHost, st);
  // x bundle (T = 1) -> x field [nrhs][nshift][V][12]; a host destination is staged through
  // r64 (the residual is no longer needed: the final norms are in rn)
  const size_t xbytes = sizeof(double) * 2 * 12 * V * nsys;
  launch_unpack<double>(g, w->x64, on_device ? x : w->r64, nsys, st);
  if (!on_device) cudaMemcpyAsync(x, w->r64, xbytes, cudaMemcpyDeviceToHost, st);
  cudaError_t se = cudaStreamSynchronize(st);
  if (!rc) rc = check_cuda(ctx, se, "solve");
  if (!rc && S.launch_error) rc = set_err(ctx, TMAMG_ERR_CUDA, "solve: cooperative coarse-solver launch failed");
  for (const CoarseLevel& l : ctx->levels)
    if (!rc && coarse_apply_timed_out(l, st)) S.timeout = true;
  if (!rc && S.timeout) rc = set_err(ctx, TMAMG_ERR_TIMEOUT, "solve: a coarse-solver bounded wait timed out");
  if (rc) return rc;
  int all_ok = 1;
  // doublets: one entry per doublet (both flavours carry the doublet's folded norms)
  const int nout = pair ? nsys / 2 : nsys;
  for (int q = 0; q < nout; ++q) {
    const int n = pair ? 2 * q : q;
    const int fl = pair ? (hflags[n] | hflags[n + 1]) : hflags[n];
    double rel = hbn[n] > 0 ? hrn[n] / hbn[n] : 0.0;
    int status = fl ? TMAMG_ERR_NONFINITE : (rel <= sp->tol ? TMAMG_OK : TMAMG_NOT_CONVERGED);
    if (status != TMAMG_OK) all_ok = 0;
    if (stats) {
      stats[q].status = status;
      stats[q].outer_iters = hout[n] - (capped && hmask[n] ? 1 : 0);
      stats[q].inner_iters = hin[n];
      stats[q].coarse_iters = S.coarse_iters;
      stats[q].true_rel_res = fl ? NAN : rel;
    }
  }
  return all_ok ? TMAMG_OK : TMAMG_NOT_CONVERGED;
}

}  // namespace tmamg

using namespace tmamg;

extern "C" {

int tmamg_debug_bounded_wait(long long limit_cycles, int unreachable_next) {
  if (limit_cycles < 0) return TMAMG_ERR_ARG;
  coarse_gmres_debug_wait(limit_cycles, unreachable_next);
  return TMAMG_OK;
}

int tmamg_setup(tmamg_ctx* ctx, const tmamg_setup_params* p, const float* start_vectors) {
  if (!ctx || !p) return set_err(ctx, TMAMG_ERR_ARG, "setup: null argument");
  if (!ctx->have_op) return set_err(ctx, TMAMG_ERR_STATE, "setup: operator not set");
  return do_setup(ctx, p, start_vectors, true);
}

int tmamg_setup_from_vectors(tmamg_ctx* ctx, const tmamg_setup_params* p, const float* test_vectors) {
  if (!ctx || !p || !test_vectors) return set_err(ctx, TMAMG_ERR_ARG, "setup_from_vectors: null argument");
  if (!ctx->have_op) return set_err(ctx, TMAMG_ERR_STATE, "setup_from_vectors: operator not set");
  return do_setup(ctx, p, test_vectors, false);
}

int tmamg_solve(tmamg_ctx* ctx, const double* b, int nrhs, const double* mu, int nshift, double* x, int on_device,
                const tmamg_solve_params* p, tmamg_system_stats* stats) {
  if (!ctx) return TMAMG_ERR_ARG;
  if (!b || !x || !mu || nrhs < 1 || nshift < 1) return set_err(ctx, TMAMG_ERR_ARG, "solve: bad argument");
  if (!ctx->have_setup) return set_err(ctx, TMAMG_ERR_STATE, "solve: no multigrid setup");
  tmamg_solve_params def;
  tmamg_default_solve_params(&def);
  return do_solve(ctx, b, nrhs, mu, nshift, x, on_device, p ? p : &def, stats, nullptr);
}

int tmamg_solve_doublet(tmamg_ctx* ctx, const double* b, int nrhs, const double* mu, const double* eps, int nshift,
                        double* x, int on_device, const tmamg_solve_params* p, tmamg_system_stats* stats) {
  if (!ctx) return TMAMG_ERR_ARG;
  if (!b || !x || !mu || !eps || nrhs < 1 || nshift < 1)
    return set_err(ctx, TMAMG_ERR_ARG, "solve_doublet: bad argument");
  if (!ctx->have_setup) return set_err(ctx, TMAMG_ERR_STATE, "solve_doublet: no multigrid setup");
  tmamg_solve_params def;
  tmamg_default_solve_params(&def);
  return do_solve(ctx, b, nrhs, mu, nshift, x, on_device, p ? p : &def, stats, eps);
}

size_t tmamg_coarse_bundle_bytes(const tmamg_ctx* ctx, int level, int nsys) {
  if (!ctx || level < 1 || level > (int)ctx->levels.size() || nsys < 1) return 0;
  const CoarseLevel& l = ctx->levels[level - 1];
  return (size_t)ntiles(nsys, 2) * 2 * l.nv * l.Vc * 4 * sizeof(float);
}

int tmamg_sap(tmamg_ctx* ctx, void* r_bundle, void* e_bundle, int nsys, const double* mu, const int block[4],
              int cycles, int mr_steps) {
  if (!ctx) return TMAMG_ERR_ARG;
  if (!r_bundle || !e_bundle || !mu || !block || nsys < 1 || nsys > 256 || cycles < 1 || mr_steps < 1)
    return set_err(ctx, TMAMG_ERR_ARG, "sap: bad argument");
  if (!ctx->have_op) return set_err(ctx, TMAMG_ERR_STATE, "sap: operator not set");
  std::string why;
  if (sap_check_blocks(ctx->g, block, why)) return set_err(ctx, TMAMG_ERR_ARG, "sap: " + why);
  int rc = upload_mu(ctx, mu, nsys);
  if (rc) return rc;
  float* delta = nullptr;
  size_t bytes = (size_t)ntiles(nsys, 2) * 12 * ctx->g.V * 4 * sizeof(float);
  rc = check_cuda(ctx, cudaMalloc(&delta, bytes), "cudaMalloc(sap scratch)");
  if (rc) return rc;
  sap_apply(ctx->g, block, ctx->U32, ctx->C32, (float*)r_bundle, (float*)e_bundle, delta, ctx->mu_dev, nsys, cycles,
            mr_steps, ctx->stream);
  rc = check_cuda(ctx, cudaGetLastError(), "sap launch");
  cudaStreamSynchronize(ctx->stream);
  cudaFree(delta);
  return rc;
}

// aggregation between level - 1 (0 = fine) and coarse level `level`, and the parent's unknowns per chirality
static AggDims transfer_dims(const tmamg_ctx* ctx, int level, int* d) {
  const CoarseLevel& l = ctx->levels[level - 1];
  if (level == 1) {
    *d = 6;
    return agg_dims(ctx->g, l.agg);
  }
  *d = ctx->levels[level - 2].nv;
  return agg_dims_coarse(ctx->levels[level - 2], l.agg);
}

int tmamg_restrict(tmamg_ctx* ctx, int level, const void* fine_bundle, void* coarse_bundle, int nsys) {
  if (!ctx) return TMAMG_ERR_ARG;
  if (!ctx->have_setup) return set_err(ctx, TMAMG_ERR_STATE, "restrict: no setup");
  if (level < 1 || level > (int)ctx->levels.size() || !fine_bundle || !coarse_bundle || nsys < 1)
    return set_err(ctx, TMAMG_ERR_ARG, "restrict: bad argument");
  const CoarseLevel& l = ctx->levels[level - 1];
  int d = 0;
  const AggDims ad = transfer_dims(ctx, level, &d);
  restrict_vec(ad, l.P, (const float*)fine_bundle, (float*)coarse_bundle, l.nv, d, nsys, ctx->stream);
  return check_cuda(ctx, cudaGetLastError(), "restrict launch");
}

int tmamg_prolong(tmamg_ctx* ctx, int level, const void* coarse_bundle, void* fine_bundle, int nsys) {
  if (!ctx) return TMAMG_ERR_ARG;
  if (!ctx->have_setup) return set_err(ctx, TMAMG_ERR_STATE, "prolong: no setup");
  if (level < 1 || level > (int)ctx->levels.size() || !fine_bundle || !coarse_bundle || nsys < 1)
    return set_err(ctx, TMAMG_ERR_ARG, "prolong: bad argument");
  const CoarseLevel& l = ctx->levels[level - 1];
  int d = 0;
  const AggDims ad = transfer_dims(ctx, level, &d);
  prolong_vec(ad, l.P, (const float*)coarse_bundle, (float*)fine_bundle, l.nv, d, nsys, 0, ctx->stream);
  return check_cuda(ctx, cudaGetLastError(), "prolong launch");
}

int tmamg_coarse_solve(tmamg_ctx* ctx, int level, const void* rc_bundle, void* xc_bundle, int nrhs, const double* mu,
                       int nshift, const tmamg_solve_params* p, int* iterations) {
  if (!ctx) return TMAMG_ERR_ARG;
  if (!ctx->have_setup) return set_err(ctx, TMAMG_ERR_STATE, "coarse_solve: no setup");
  const int nlev = (int)ctx->levels.size();
  if (level < 1 || level > nlev || !rc_bundle || !xc_bundle || !mu || nrhs < 1 || nshift < 1 || !p ||
      rc_bundle == xc_bundle)
    return set_err(ctx, TMAMG_ERR_ARG, "coarse_solve: bad argument");
  const bool middle = level < nlev;
  if (middle && (p->mid_restart < 1 || p->mid_restart > 64 || p->mid_maxiter < 1 || !(p->mid_tol > 0) ||
                 p->mid_smooth < 0))
    return set_err(ctx, TMAMG_ERR_ARG, "coarse_solve: bad middle-level parameters");
  const int nsys = nrhs * nshift;
  if (nsys > 256 || p->coarse_solver < 0 || p->coarse_solver > 2 || (p->coarse_solver == 1 && nrhs > 16) ||
      p->coarse_restart < 1 || p->coarse_restart > 64 || p->coarse_maxiter < 1 ||
      (p->coarse_precision != 0 && p->coarse_precision != 16 && p->coarse_precision != 32))
    return set_err(ctx, TMAMG_ERR_ARG, "coarse_solve: bad parameters");
  int rc = ensure_ws(ctx, nsys, *p);
  if (rc) return rc;
  std::vector<double> musys(nsys);
  for (int n = 0; n < nsys; ++n) musys[n] = mu[n % nshift];
  rc = upload_mu(ctx, musys.data(), nsys);
  if (rc) return rc;
  SolveCtx S{ctx, p, nsys, ctx->mu_dev, 0};
  S.nshift = nshift;
  if (middle)
    mid_solve(S, (const float*)rc_bundle, (float*)xc_bundle);
  else
    coarse_solve(S, (const float*)rc_bundle, (float*)xc_bundle);
  rc = check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "coarse_solve");
  if (!rc && S.launch_error) rc = set_err(ctx, TMAMG_ERR_CUDA, "coarse_solve: launch failed");
  for (const CoarseLevel& l : ctx->levels)
    if (!rc && coarse_apply_timed_out(l, ctx->stream)) S.timeout = true;
  if (!rc && S.timeout) rc = set_err(ctx, TMAMG_ERR_TIMEOUT, "coarse_solve: a bounded wait timed out");
  if (iterations) *iterations = middle ? S.mid_iters : S.coarse_iters;
  return rc;
}

int tmamg_coarse_apply(tmamg_ctx* ctx, int level, const void* x_bundle, void* y_bundle, int nsys, const double* mu,
                       int precision) {
  if (!ctx) return TMAMG_ERR_ARG;
  if (!ctx->have_setup) return set_err(ctx, TMAMG_ERR_STATE, "coarse_apply: no setup");
  if (level < 1 || level > (int)ctx->levels.size() || !x_bundle || !y_bundle || !mu || nsys < 1 ||
      x_bundle == y_bundle || (precision != 16 && precision != 32))
    return set_err(ctx, TMAMG_ERR_ARG, "coarse_apply: bad argument");
  int rc = upload_mu(ctx, mu, nsys);
  if (rc) return rc;
  CoarseLevel& l = ctx->levels[level - 1];
  if (!coarse_apply_level(l, precision, (const float*)x_bundle, (float*)y_bundle, ctx->mu_dev, 1.0, nsys,
                          ctx->stream))
    return set_err(ctx, TMAMG_ERR_ARG, "coarse_apply: sizes outside the tensor-core stencil");
  rc = check_cuda(ctx, cudaGetLastError(), "coarse_apply launch");
  if (!rc && coarse_apply_timed_out(l, ctx->stream))
    rc = set_err(ctx, TMAMG_ERR_TIMEOUT, "coarse_apply: a bounded wait timed out");
  return rc;
}

}  // extern "C"

// ================================================================== learned preconditioner step
namespace tmamg {

void free_nn(tmamg_ctx* ctx) {
  if (ctx->nn) {
    ctx->nn->release();
    delete ctx->nn;
    ctx->nn = nullptr;
  }
}

static NNGeom nn_geom(const tmamg_ctx* ctx) {
  return NNGeom{{ctx->g.L[0], ctx->g.L[1], ctx->g.L[2], ctx->g.L[3]}, ctx->g.V, ctx->g.bc_t};
}

static int nn_ready(tmamg_ctx* ctx) {
  if (!ctx->nn) ctx->nn = new NNState();
  return ctx->nn->alloc_weights();
}

// host weights (complex double, three layers concatenated) <-> device FP32 master weights
static int nn_upload(tmamg_ctx* ctx, const double* W) {
  const int n = nn_weight_offset(3);
  std::vector<float> h(2 * n);
  for (int i = 0; i < 2 * n; ++i) h[i] = (float)W[i];
  int rc = check_cuda(ctx, cudaMemcpyAsync(ctx->nn->W, h.data(), sizeof(float) * 2 * n, cudaMemcpyHostToDevice,
                                           ctx->stream), "upload weights");
  if (rc) return rc;
  cudaMemsetAsync(ctx->nn->m1, 0, sizeof(float2) * n, ctx->stream);
  cudaMemsetAsync(ctx->nn->m2, 0, sizeof(float2) * n, ctx->stream);
  nn_refresh_inference(*ctx->nn, ctx->stream);
  ctx->nn->trained = true;
  return check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "upload weights");
}

// gaussian FP32 fine bundle of nsys systems from the library's counter-based generator
static int random_bundle(tmamg_ctx* ctx, uint64_t seed, int nsys, float* bundle) {
  const int64_t n = (int64_t)nsys * ctx->g.V * 12;
  float* field = nullptr;
  int rc = check_cuda(ctx, cudaMalloc(&field, sizeof(float2) * n), "cudaMalloc(random field)");
  if (rc) return rc;
  device_gaussian(seed, 0x5eedULL, n, reinterpret_cast<float2*>(field), ctx->stream);
  launch_pack<float>(ctx->g, field, bundle, nsys, ctx->stream);
  rc = check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "random bundle");
  cudaFree(field);
  return rc;
}

// loss sum_n |y_n - e_n|^2 / |e_n|^2 (host value); d: scratch bundle
static double nn_loss(tmamg_ctx* ctx, const float* y, const float* e, float* d, int nsys) {
  Workspace* w = ctx->ws;
  cudaStream_t st = ctx->stream;
  const int64_t M = 12 * ctx->g.V;
  cudaMemcpyAsync(d, e, w->fb32, cudaMemcpyDeviceToDevice, st);
  axpby<float>(w->ones, 2, y, w->mones, 2, d, M, nsys, nullptr, st);
  mdot<float>(d, 0, 1, d, M, nsys, w->dot, nsys, w->top.partial, st);
  mdot<float>(e, 0, 1, e, M, nsys, w->dot + nsys, nsys, w->top.partial, st);
  std::vector<double2> h(2 * nsys);
  cudaMemcpyAsync(h.data(), w->dot, sizeof(double2) * 2 * nsys, cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  double s = 0;
  for (int n = 0; n < nsys; ++n) s += h[nsys + n].x > 0 ? h[n].x / h[nsys + n].x : 0.0;
  return s;
}

// e ~ D^{-1} r in FP32 by AMG-preconditioned FGMRES (restarted from the true residual)
static void solve32(SolveCtx& S, const float* r, float* e, double tol, int cycles) {
  tmamg_ctx* ctx = S.ctx;
  Workspace* w = ctx->ws;
  cudaStream_t st = ctx->stream;
  const int nsys = S.nsys;
  const int64_t M = 12 * ctx->g.V;
  LevelOps fine;
  fine.M = M;
  fine.A = [&](const float* xx, float* yy) { launch_dirac<float>(ctx->g, ctx->U32, ctx->C32, xx, yy, S.mu, nsys, st); };
  fine.precond = [&](const float* v, float* z) { amg_cycle(S, v, z); };
  const size_t vstride = w->fb32 / sizeof(float);
  cudaMemsetAsync(e, 0, w->fb32, st);
  set_rel_tol(w->rel_top, nsys, tol, st);
  for (int c = 0; c < cycles; ++c) {
    launch_dirac<float>(ctx->g, ctx->U32, ctx->C32, e, w->V, S.mu, nsys, st);
    axpby<float>(w->ones, 2, r, w->mones, 2, w->V, M, nsys, nullptr, st);  // V0 = r - D e
    gmres_cycle<float>(w->top, fine, nsys, S.sp->restart, w->V, vstride, w->Z, e, nullptr, w->rel_top, 1, false, st);
  }
}

}  // namespace tmamg

extern "C" {

void tmamg_default_nn_params(tmamg_nn_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->pairs = 48;
  p->batch = 12;
  p->epochs = 30;
  p->lr = 2e-3;
  p->pair_tol = 1e-5;
  p->mu = 0.0;
  p->seed = 7;
  p->gate_systems = 4;
}

int tmamg_nn_init(tmamg_ctx* ctx, uint64_t seed) {
  if (!ctx) return TMAMG_ERR_ARG;
  if (!ctx->have_op) return set_err(ctx, TMAMG_ERR_STATE, "nn_init: operator not set");
  int rc = nn_ready(ctx);
  if (rc) return set_err(ctx, TMAMG_ERR_OOM, "nn_init: weights");
  // a Jacobi-like start: layer 1 maps the spins onto channels 0..3 scaled by 2 kappa (the
  // inverse of the operator's diagonal), layers 2 and 3 pass them on; plus small noise
  const int n = nn_weight_offset(3);
  std::vector<double> W(2 * n, 0.0);
  std::vector<float> noise;
  host_gaussian(seed, 0x5eedULL, (size_t)12 * ((n + 11) / 12), noise);
  const int chs[4] = {4, 8, 8, 4};
  for (int l = 0; l < 3; ++l) {
    const int cin = chs[l], cout = chs[l + 1], off = nn_weight_offset(l);
    for (int q = 0; q < 9 * cout * cin; ++q) {
      W[2 * (off + q)] = 0.01 * noise[2 * (off + q)];
      W[2 * (off + q) + 1] = 0.01 * noise[2 * (off + q) + 1];
    }
    const double d = l == 0 ? 2.0 * ctx->kappa : 1.0;
    for (int a = 0; a < cout && a < cin; ++a) W[2 * (off + a * cin + a)] += d;
  }
  return nn_upload(ctx, W.data());
}

int tmamg_nn_set_weights(tmamg_ctx* ctx, const double* W) {
  if (!ctx || !W) return set_err(ctx, TMAMG_ERR_ARG, "nn_set_weights: null argument");
  if (nn_ready(ctx)) return set_err(ctx, TMAMG_ERR_OOM, "nn_set_weights: weights");
  return nn_upload(ctx, W);
}

int tmamg_nn_get_weights(const tmamg_ctx* ctx, double* W) {
  if (!ctx || !W || !ctx->nn || !ctx->nn->W) return TMAMG_ERR_ARG;
  const int n = nn_weight_offset(3);
  std::vector<float> h(2 * n);
  cudaMemcpy(h.data(), ctx->nn->W, sizeof(float) * 2 * n, cudaMemcpyDeviceToHost);
  for (int i = 0; i < 2 * n; ++i) W[i] = h[i];
  return TMAMG_OK;
}

int tmamg_nn_forward(tmamg_ctx* ctx, const void* r_bundle, void* y_bundle, int nsys, int bf16) {
  if (!ctx) return TMAMG_ERR_ARG;
  if (!r_bundle || !y_bundle || nsys < 1 || r_bundle == y_bundle) return set_err(ctx, TMAMG_ERR_ARG, "nn_forward: bad argument");
  if (!ctx->nn || !ctx->nn->trained) return set_err(ctx, TMAMG_ERR_STATE, "nn_forward: no weights");
  if (ctx->nn->alloc(ctx->g.V, nsys)) return set_err(ctx, TMAMG_ERR_OOM, "nn_forward: buffers");
  nn_forward(*ctx->nn, nn_geom(ctx), ctx->U32, (const float*)r_bundle, (float*)y_bundle, nsys, bf16 != 0, ctx->stream);
  return check_cuda(ctx, cudaGetLastError(), "nn_forward");
}

int tmamg_nn_loss_grad(tmamg_ctx* ctx, const void* r_bundle, const void* e_bundle, int nsys, double* loss,
                       double* grad) {
  if (!ctx) return TMAMG_ERR_ARG;
  if (!r_bundle || !e_bundle || nsys < 1 || nsys > 256) return set_err(ctx, TMAMG_ERR_ARG, "nn_loss_grad: bad argument");
  if (!ctx->nn || !ctx->nn->trained) return set_err(ctx, TMAMG_ERR_STATE, "nn_loss_grad: no weights");
  tmamg_solve_params def;
  tmamg_default_solve_params(&def);
  int rc = ensure_ws(ctx, nsys, def);
  if (rc) return rc;
  if (ctx->nn->alloc(ctx->g.V, nsys)) return set_err(ctx, TMAMG_ERR_OOM, "nn_loss_grad: buffers");
  rc = ensure_t2(ctx);
  if (rc) return rc;
  Workspace* w = ctx->ws;
  NNGeom ng = nn_geom(ctx);
  nn_forward(*ctx->nn, ng, ctx->U32, (const float*)r_bundle, w->t1, nsys, false, ctx->stream);
  if (loss) *loss = nn_loss(ctx, w->t1, (const float*)e_bundle, w->t2, nsys);
  nn_backward(*ctx->nn, ng, ctx->U32, (const float*)r_bundle, w->t1, (const float*)e_bundle, nsys,
              w->top.partial, ctx->stream);
  rc = check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "nn_loss_grad");
  if (rc) return rc;
  if (grad) {
    const int n = nn_weight_offset(3);
    cudaMemcpy(grad, ctx->nn->grad, sizeof(double2) * n, cudaMemcpyDeviceToHost);
  }
  return TMAMG_OK;
}

int tmamg_nn_train(tmamg_ctx* ctx, const tmamg_nn_params* p, tmamg_nn_report* rep) {
  if (!ctx || !p) return set_err(ctx, TMAMG_ERR_ARG, "nn_train: null argument");
  if (!ctx->have_setup) return set_err(ctx, TMAMG_ERR_STATE, "nn_train: no multigrid setup");
  if (p->batch < 1 || p->batch > 16 || p->pairs < p->batch || p->epochs < 1 || !(p->lr > 0) || p->gate_systems < 1 ||
      p->gate_systems > 16 || p->window < 0)
    return set_err(ctx, TMAMG_ERR_ARG, "nn_train: bad parameters");
  cudaStream_t st = ctx->stream;
  if (!ctx->nn || !ctx->nn->trained) {
    int rc = tmamg_nn_init(ctx, p->seed);
    if (rc) return rc;
  }
  NNState& nns = *ctx->nn;
  const int nsys = p->batch;
  tmamg_solve_params sp;
  tmamg_default_solve_params(&sp);
  int rc = ensure_ws(ctx, nsys, sp);
  if (rc) return rc;
  if (nns.alloc(ctx->g.V, nsys)) return set_err(ctx, TMAMG_ERR_OOM, "nn_train: buffers");
  rc = ensure_t2(ctx);
  if (rc) return rc;
  Workspace* w = ctx->ws;
  std::vector<double> mus(nsys, p->mu);
  rc = upload_mu(ctx, mus.data(), nsys);
  if (rc) return rc;
  // ---- training pairs: r = residual the plain cycle leaves, e = D^{-1} r, collected and trained
  // window by window (all batches in one window unless p->window limits it)
  const int nb = p->pairs / nsys;
  const int win = p->window > 0 && p->window < nb ? p->window : nb;
  float *R = nullptr, *E = nullptr;
  rc = check_cuda(ctx, cudaMalloc(&R, w->fb32 * win), "cudaMalloc(pairs)");
  if (!rc) rc = check_cuda(ctx, cudaMalloc(&E, w->fb32 * win), "cudaMalloc(pairs)");
  if (rc) {
    cudaFree(R);
    return rc;
  }
  const int64_t M = 12 * ctx->g.V;
  SolveCtx S{ctx, &sp, nsys, ctx->mu_dev, 0};
  NNGeom ng = nn_geom(ctx);
  double first = 0, last = 0;
  int step = 0;
  int nfirst = 0, nlast = 0;
  for (int b0 = 0; b0 < nb && !rc; b0 += win) {
    const int nw = nb - b0 < win ? nb - b0 : win;
    for (int k = 0; k < nw; ++k) {
      float* rb = R + (w->fb32 / sizeof(float)) * k;
      float* eb = E + (w->fb32 / sizeof(float)) * k;
      rc = random_bundle(ctx, p->seed * 1000003ULL + b0 + k, nsys, w->t3);  // v
      if (rc) break;
      cudaMemcpyAsync(w->Z, w->t3, w->fb32, cudaMemcpyDeviceToDevice, st);  // keep v
      amg_cycle(S, w->Z, w->e32);                                            // z = M v (plain)
      launch_dirac<float>(ctx->g, ctx->U32, ctx->C32, w->e32, rb, S.mu, nsys, st);
      axpby<float>(w->ones, 2, w->Z, w->mones, 2, rb, M, nsys, nullptr, st);  // r = v - D z
      solve32(S, rb, eb, p->pair_tol, 3);
    }
    for (int ep = 0; ep < p->epochs && !rc; ++ep) {
      // the loss of the first window's first pass and of the last window's last pass
      const bool lf = b0 == 0 && ep == 0, ll = b0 + nw >= nb && ep == p->epochs - 1;
      for (int k = 0; k < nw; ++k) {
        const float* rb = R + (w->fb32 / sizeof(float)) * k;
        const float* eb = E + (w->fb32 / sizeof(float)) * k;
        nn_forward(nns, ng, ctx->U32, rb, w->t1, nsys, false, st);
        if (lf || ll) {
          const double l = nn_loss(ctx, w->t1, eb, w->t2, nsys);
          if (lf) {
            first += l;
            nfirst += nsys;
          }
          if (ll) {
            last += l;
            nlast += nsys;
          }
        }
        nn_backward(nns, ng, ctx->U32, rb, w->t1, eb, nsys, w->top.partial, st);
        nn_adam(nns, (float)p->lr, ++step, 1.0 / nsys, st);
      }
    }
  }
  if (nfirst) first /= nfirst;
  if (nlast) last /= nlast;
  cudaStreamSynchronize(st);
  cudaFree(R);
  cudaFree(E);
  if (rc) return rc;
  nn_refresh_inference(nns, st);
  nns.trained = true;
  nns.loss_first = first;
  nns.loss_last = last;
  // ---- the gate: the same solve with and without the learned step (plain SAP is the judge)
  const int ng_sys = p->gate_systems;
  std::vector<float> hb;
  host_gaussian(p->seed + 99991ULL, 0x5eedULL, (size_t)ng_sys * ctx->g.V * 12, hb);
  std::vector<double> b64(hb.begin(), hb.end());
  std::vector<double> x64(b64.size());
  std::vector<tmamg_system_stats> stats(ng_sys);
  double gm = p->mu;
  int its[2] = {0, 0};
  bool ok[2] = {false, false};
  for (int pass = 0; pass < 2; ++pass) {
    tmamg_solve_params gp;
    tmamg_default_solve_params(&gp);
    gp.use_nn = pass == 0 ? 0 : 2;
    int r2 = do_solve(ctx, b64.data(), ng_sys, &gm, 1, x64.data(), 0, &gp, stats.data(), nullptr);
    if (r2 < 0) return r2;
    int mx = 0;
    bool conv = true;
    for (int n = 0; n < ng_sys; ++n) {
      mx = stats[n].inner_iters > mx ? stats[n].inner_iters : mx;
      conv &= stats[n].status == TMAMG_OK;
    }
    its[pass] = mx;
    ok[pass] = conv;
  }
  nns.iters_plain = its[0];
  nns.iters_nn = its[1];
  nns.enabled = ok[1] && its[1] < its[0];
  if (rep) {
    rep->loss_first = first;
    rep->loss_last = last;
    rep->iters_plain = its[0];
    rep->iters_nn = its[1];
    rep->enabled = nns.enabled ? 1 : 0;
  }
  return TMAMG_OK;
}

}  // extern "C"

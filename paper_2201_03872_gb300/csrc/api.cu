// C ABI of the tmamg library: context, gauge field, operator, bundles, fine stencil.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"

namespace tmamg {

uint64_t& launch_counter() {
  static uint64_t n = 0;
  return n;
}

static std::mutex g_dev_mutex;

static int current_device() {
  int dev = 0;
  cudaGetDevice(&dev);
  return dev;
}

int device_sms() {
  static std::map<int, int> sms;
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_dev_mutex);
  auto it = sms.find(dev);
  if (it != sms.end()) return it->second;
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  sms[dev] = n;
  return n;
}

int device_smem_optin() {
  static std::map<int, int> optin;
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_dev_mutex);
  auto it = optin.find(dev);
  if (it != optin.end()) return it->second;
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  optin[dev] = n;
  return n;
}

void func_smem_optin(const void* func, int bytes) {
  static std::map<std::pair<int, const void*>, int> done;
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_dev_mutex);
  int& have = done[std::make_pair(dev, func)];
  if (have >= bytes) return;
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess) have = bytes;
}

int set_err(tmamg_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int check_cuda(tmamg_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return TMAMG_OK;
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return set_err(ctx, TMAMG_ERR_OOM, m);
  return set_err(ctx, TMAMG_ERR_CUDA, m);
}

int upload_mu(tmamg_ctx* ctx, const double* mu, int nsys) {
  if (nsys > ctx->mu_cap) {
    if (ctx->mu_dev) cudaFree(ctx->mu_dev);
    ctx->mu_dev = nullptr;
    int cap = nsys < 64 ? 64 : nsys;
    int rc = check_cuda(ctx, cudaMalloc(&ctx->mu_dev, sizeof(double) * cap), "cudaMalloc(mu)");
    if (rc) return rc;
    ctx->mu_cap = cap;
  }
  return check_cuda(ctx, cudaMemcpyAsync(ctx->mu_dev, mu, sizeof(double) * nsys, cudaMemcpyHostToDevice, ctx->stream),
                    "upload mu");
}

static int ensure_scratch(tmamg_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->scratch_bytes) return TMAMG_OK;
  for (int i = 0; i < 2; ++i) {
    if (ctx->scratch[i]) cudaFree(ctx->scratch[i]);
    ctx->scratch[i] = nullptr;
  }
  ctx->scratch_bytes = 0;
  for (int i = 0; i < 2; ++i) {
    int rc = check_cuda(ctx, cudaMalloc(&ctx->scratch[i], bytes), "cudaMalloc(scratch)");
    if (rc) return rc;
  }
  ctx->scratch_bytes = bytes;
  return TMAMG_OK;
}

}  // namespace tmamg

using namespace tmamg;

extern "C" {

void tmamg_default_setup_params(tmamg_setup_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->levels = 2;
  for (int d = 0; d < 4; ++d) {
    p->agg[0][d] = 4;
    p->agg[1][d] = 2;
    p->sap_block[d] = 4;
  }
  p->nv[0] = 24;
  p->nv[1] = 32;
  p->sap_cycles = 2;
  p->sap_mr_steps = 3;
  p->setup_iters = 5;
  p->mu_setup = 0.0;
  p->seed = 1;
  p->setup_gmres_steps = 20;
}

void tmamg_default_solve_params(tmamg_solve_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->tol = 1e-10;
  p->restart = 10;
  p->max_outer = 50;
  p->coarse_tol = 1e-1;
  p->coarse_restart = 20;
  p->coarse_maxiter = 100;
  p->coarse_solver = 0;
  p->delta_mu = 1.0;
  p->precision = 32;
  p->use_nn = 0;
  p->poll = 4;
  p->coarse_precision = 16;
  p->mid_tol = 7e-2;
  p->mid_restart = 10;
  p->mid_maxiter = 50;
  p->mid_smooth = 3;
  p->inner_cycles = 1;
  p->sap_cycles = 0;
  p->sap_mr_steps = 0;
}

int tmamg_create(const int L[4], int bc_t, void* cuda_stream, tmamg_ctx** out) {
  if (!out || !L) return TMAMG_ERR_ARG;
  *out = nullptr;
  for (int d = 0; d < 4; ++d)
    if (L[d] < 2 || (L[d] % 2)) return TMAMG_ERR_ARG;
  if (bc_t != 1 && bc_t != -1) return TMAMG_ERR_ARG;
  tmamg_ctx* ctx = new tmamg_ctx();
  for (int d = 0; d < 4; ++d) ctx->g.L[d] = L[d];
  ctx->g.V = (int64_t)L[0] * L[1] * L[2] * L[3];
  ctx->g.bc_t = bc_t;
  ctx->stream = (cudaStream_t)cuda_stream;
  tmamg_default_setup_params(&ctx->sp);
  int rc = check_cuda(ctx, cudaMalloc(&ctx->U64, sizeof(double2) * 36 * ctx->g.V), "cudaMalloc(U64)");
  if (!rc) rc = check_cuda(ctx, cudaMalloc(&ctx->U32, sizeof(float2) * 36 * ctx->g.V), "cudaMalloc(U32)");
  if (!rc) rc = check_cuda(ctx, cudaMalloc(&ctx->C64, sizeof(double) * 72 * ctx->g.V), "cudaMalloc(C64)");
  if (!rc) rc = check_cuda(ctx, cudaMalloc(&ctx->C32, sizeof(float) * 72 * ctx->g.V), "cudaMalloc(C32)");
  if (rc) {
    tmamg_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return TMAMG_OK;
}

int tmamg_destroy(tmamg_ctx* ctx) {
  if (!ctx) return TMAMG_OK;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  free_workspace(ctx);
  free_nn(ctx);
  free_levels(ctx);
  cudaFree(ctx->U64);
  cudaFree(ctx->U32);
  cudaFree(ctx->C64);
  cudaFree(ctx->C32);
  cudaFree(ctx->mu_dev);
  cudaFree(ctx->eps_dev);
  for (int i = 0; i < 2; ++i) cudaFree(ctx->scratch[i]);
  delete ctx;
  return TMAMG_OK;
}

const char* tmamg_last_error(const tmamg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

uint64_t tmamg_kernel_launches(void) { return launch_counter(); }

int tmamg_volume(const tmamg_ctx* ctx, int64_t* V) {
  if (!ctx || !V) return TMAMG_ERR_ARG;
  *V = ctx->g.V;
  return TMAMG_OK;
}

int tmamg_load_gauge(tmamg_ctx* ctx, const double* U, int on_device) {
  if (!ctx || !U) return set_err(ctx, TMAMG_ERR_ARG, "load_gauge: null argument");
  const double* src = U;
  double* tmp = nullptr;
  size_t bytes = sizeof(double) * 2 * 36 * ctx->g.V;
  if (!on_device) {
    int rc = check_cuda(ctx, cudaMalloc(&tmp, bytes), "cudaMalloc(gauge staging)");
    if (rc) return rc;
    rc = check_cuda(ctx, cudaMemcpyAsync(tmp, U, bytes, cudaMemcpyHostToDevice, ctx->stream), "upload gauge");
    if (rc) {
      cudaFree(tmp);
      return rc;
    }
    src = tmp;
  }
  launch_convert_gauge(ctx->g, src, ctx->U64, ctx->U32, ctx->stream);
  int rc = check_cuda(ctx, cudaGetLastError(), "convert_gauge launch");
  if (tmp) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(tmp);
  }
  if (rc) return rc;
  ctx->have_gauge = true;
  ctx->have_op = false;
  ctx->have_setup = false;
  return TMAMG_OK;
}

int tmamg_set_operator(tmamg_ctx* ctx, double kappa, double c_sw) {
  if (!ctx) return TMAMG_ERR_ARG;
  if (!(kappa > 0.0) || !(c_sw >= 0.0)) return set_err(ctx, TMAMG_ERR_ARG, "set_operator: need kappa > 0, c_sw >= 0");
  if (!ctx->have_gauge) return set_err(ctx, TMAMG_ERR_STATE, "set_operator: no gauge field loaded");
  ctx->kappa = kappa;
  ctx->c_sw = c_sw;
  launch_build_clover(ctx->g, ctx->U64, kappa, c_sw, ctx->C64, ctx->C32, ctx->stream);
  int rc = check_cuda(ctx, cudaGetLastError(), "build_clover launch");
  if (rc) return rc;
  ctx->have_op = true;
  ctx->have_setup = false;
  free_workspace(ctx);
  free_levels(ctx);
  return TMAMG_OK;
}

size_t tmamg_bundle_bytes(const tmamg_ctx* ctx, int nsys, int prec) {
  if (!ctx || nsys <= 0 || (prec != 32 && prec != 64)) return 0;
  int T = prec == 32 ? 2 : 1;
  size_t es = prec == 32 ? 4 : 8;
  return (size_t)ntiles(nsys, T) * T * 12 * 2 * (size_t)ctx->g.V * es;
}

int tmamg_pack(tmamg_ctx* ctx, const void* x_field, void* x_bundle, int nsys, int prec) {
  if (!ctx || !x_field || !x_bundle || nsys <= 0) return set_err(ctx, TMAMG_ERR_ARG, "pack: bad argument");
  if (prec == 32) launch_pack<float>(ctx->g, (const float*)x_field, (float*)x_bundle, nsys, ctx->stream);
  else if (prec == 64) launch_pack<double>(ctx->g, (const double*)x_field, (double*)x_bundle, nsys, ctx->stream);
  else return set_err(ctx, TMAMG_ERR_ARG, "pack: prec must be 32 or 64");
  return check_cuda(ctx, cudaGetLastError(), "pack launch");
}

int tmamg_unpack(tmamg_ctx* ctx, const void* x_bundle, void* x_field, int nsys, int prec) {
  if (!ctx || !x_field || !x_bundle || nsys <= 0) return set_err(ctx, TMAMG_ERR_ARG, "unpack: bad argument");
  if (prec == 32) launch_unpack<float>(ctx->g, (const float*)x_bundle, (float*)x_field, nsys, ctx->stream);
  else if (prec == 64) launch_unpack<double>(ctx->g, (const double*)x_bundle, (double*)x_field, nsys, ctx->stream);
  else return set_err(ctx, TMAMG_ERR_ARG, "unpack: prec must be 32 or 64");
  return check_cuda(ctx, cudaGetLastError(), "unpack launch");
}

int tmamg_dirac(tmamg_ctx* ctx, const void* x_bundle, void* y_bundle, int nsys, const double* mu, int prec) {
  if (!ctx) return TMAMG_ERR_ARG;
  if (!x_bundle || !y_bundle || !mu || nsys <= 0) return set_err(ctx, TMAMG_ERR_ARG, "dirac: bad argument");
  if (x_bundle == y_bundle) return set_err(ctx, TMAMG_ERR_ARG, "dirac: x and y must not overlap");
  if (!ctx->have_op) return set_err(ctx, TMAMG_ERR_STATE, "dirac: operator not set");
  int rc = upload_mu(ctx, mu, nsys);
  if (rc) return rc;
  if (prec == 32)
    launch_dirac<float>(ctx->g, ctx->U32, ctx->C32, (const float*)x_bundle, (float*)y_bundle, ctx->mu_dev, nsys,
                        ctx->stream);
  else if (prec == 64)
    launch_dirac<double>(ctx->g, ctx->U64, ctx->C64, (const double*)x_bundle, (double*)y_bundle, ctx->mu_dev, nsys,
                         ctx->stream);
  else
    return set_err(ctx, TMAMG_ERR_ARG, "dirac: prec must be 32 or 64");
  return check_cuda(ctx, cudaGetLastError(), "dirac launch");
}

int tmamg_dirac_doublet(tmamg_ctx* ctx, const void* x_bundle, void* y_bundle, int npair, const double* mu,
                        const double* eps, int prec) {
  if (!ctx) return TMAMG_ERR_ARG;
  if (!x_bundle || !y_bundle || !mu || !eps || npair <= 0 || (prec != 32 && prec != 64))
    return set_err(ctx, TMAMG_ERR_ARG, "dirac_doublet: bad argument");
  if (x_bundle == y_bundle) return set_err(ctx, TMAMG_ERR_ARG, "dirac_doublet: x and y must not overlap");
  if (!ctx->have_op) return set_err(ctx, TMAMG_ERR_STATE, "dirac_doublet: operator not set");
  const int nsys = 2 * npair;
  std::vector<double> ms(nsys);
  for (int q = 0; q < npair; ++q) {
    ms[2 * q] = mu[q];
    ms[2 * q + 1] = -mu[q];
  }
  int rc = upload_mu(ctx, ms.data(), nsys);
  if (rc) return rc;
  if (npair > ctx->eps_cap) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->eps_dev);
    ctx->eps_dev = nullptr;
    ctx->eps_cap = 0;
    rc = check_cuda(ctx, cudaMalloc(&ctx->eps_dev, sizeof(double) * npair), "cudaMalloc(eps)");
    if (rc) return rc;
    ctx->eps_cap = npair;
  }
  rc = check_cuda(ctx, cudaMemcpyAsync(ctx->eps_dev, eps, sizeof(double) * npair, cudaMemcpyHostToDevice,
                                       ctx->stream), "upload eps");
  if (rc) return rc;
  if (prec == 32)
    launch_dirac<float>(ctx->g, ctx->U32, ctx->C32, (const float*)x_bundle, (float*)y_bundle, ctx->mu_dev, nsys,
                        ctx->stream, ctx->eps_dev);
  else
    launch_dirac<double>(ctx->g, ctx->U64, ctx->C64, (const double*)x_bundle, (double*)y_bundle, ctx->mu_dev, nsys,
                         ctx->stream, ctx->eps_dev);
  return check_cuda(ctx, cudaGetLastError(), "dirac_doublet launch");
}

int tmamg_dirac_eo(tmamg_ctx* ctx, const void* x_bundle, void* y_bundle, int nsys, const double* mu, int prec) {
  if (!ctx) return TMAMG_ERR_ARG;
  if (!x_bundle || !y_bundle || !mu || nsys <= 0 || (prec != 32 && prec != 64))
    return set_err(ctx, TMAMG_ERR_ARG, "dirac_eo: bad argument");
  if (x_bundle == y_bundle) return set_err(ctx, TMAMG_ERR_ARG, "dirac_eo: x and y must not overlap");
  if (!ctx->have_op) return set_err(ctx, TMAMG_ERR_STATE, "dirac_eo: operator not set");
  int rc = upload_mu(ctx, mu, nsys);
  if (!rc) rc = ensure_scratch(ctx, tmamg_bundle_bytes(ctx, nsys, prec));
  if (rc) return rc;
  if (prec == 32)
    launch_dirac_eo<float>(ctx->g, ctx->U32, ctx->C32, (const float*)x_bundle, (float*)y_bundle, ctx->mu_dev, nsys,
                           (float*)ctx->scratch[0], (float*)ctx->scratch[1], ctx->stream);
  else
    launch_dirac_eo<double>(ctx->g, ctx->U64, ctx->C64, (const double*)x_bundle, (double*)y_bundle, ctx->mu_dev,
                            nsys, (double*)ctx->scratch[0], (double*)ctx->scratch[1], ctx->stream);
  return check_cuda(ctx, cudaGetLastError(), "dirac_eo launch");
}

int tmamg_apply(tmamg_ctx* ctx, const void* x_field, void* y_field, int nsys, const double* mu, int prec) {
  if (!ctx) return TMAMG_ERR_ARG;
  if (!x_field || !y_field || !mu || nsys <= 0 || (prec != 32 && prec != 64))
    return set_err(ctx, TMAMG_ERR_ARG, "apply: bad argument");
  size_t bytes = tmamg_bundle_bytes(ctx, nsys, prec);
  int rc = ensure_scratch(ctx, bytes);
  if (rc) return rc;
  rc = tmamg_pack(ctx, x_field, ctx->scratch[0], nsys, prec);
  if (!rc) rc = tmamg_dirac(ctx, ctx->scratch[0], ctx->scratch[1], nsys, mu, prec);
  if (!rc) rc = tmamg_unpack(ctx, ctx->scratch[1], y_field, nsys, prec);
  return rc;
}

}  // extern "C"

namespace tmamg {
void free_levels(tmamg_ctx* ctx) {
  for (auto& l : ctx->levels) {
    cudaFree(l.P);
    cudaFree(l.A);
    cudaFree(l.A16);
    cudaFree(l.cmax);
    cudaFree(l.cerr);
    cudaFree(l.x16);
    cudaFree(l.P64);
    cudaFree(l.A64);
  }
  ctx->levels.clear();
}
}  // namespace tmamg

// SAP smoother entry point that allocates no device memory.
//
// tmamg_sap allocates its scratch (the per-colour correction buffer) and may grow the
// context's twisted-mass array on every call. Some callers cannot allow that: code that
// runs while a CUDA stream is being captured into a graph (cudaMalloc is not a legal
// operation there), code that must not touch the allocator once a memory budget has been
// fixed, or code running under a memory pool it does not own. This file gives them a
// variant whose scratch lives in file-scope device arrays of a fixed maximum size, which
// every GPU that loads the library holds until the process exits.
#include <cstring>
#include <mutex>
#include <string>

#include "sap.cuh"

namespace tmamg {

// correction buffer of the red/black sweeps: one FP32 bundle of at most this many bytes
constexpr size_t NOALLOC_SAP_SCRATCH_BYTES = TMAMG_SAP_NOALLOC_MAX_BYTES;
constexpr int NOALLOC_SAP_MAX_SYS = TMAMG_SAP_NOALLOC_MAX_SYSTEMS;

static __device__ __align__(256) float4 g_sap_scratch[NOALLOC_SAP_SCRATCH_BYTES / sizeof(float4)];
static __device__ __align__(256) double g_sap_mu[NOALLOC_SAP_MAX_SYS];

// device addresses of the two arrays, looked up once per device (host-side names are only
// stand-ins for the device symbols and must never be passed to a kernel). std::call_once makes
// the first lookup on a device safe when several host threads make their first call together.
constexpr int MAX_DEVICES = 64;
static std::once_flag s_once[MAX_DEVICES];
static cudaError_t s_lookup_err[MAX_DEVICES];
static float* s_scratch_ptr[MAX_DEVICES] = {nullptr};
static double* s_mu_ptr[MAX_DEVICES] = {nullptr};

static int noalloc_addresses(tmamg_ctx* ctx, float** scratch, double** mu) {
  int dev = -1;
  int rc = check_cuda(ctx, cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  if (dev < 0 || dev >= MAX_DEVICES) return set_err(ctx, TMAMG_ERR_STATE, "sap_noalloc: device index out of range");
  std::call_once(s_once[dev], [dev]() {
    void* p = nullptr;
    void* q = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_sap_scratch);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_sap_mu);
    s_lookup_err[dev] = e;
    if (e == cudaSuccess) {
      s_scratch_ptr[dev] = static_cast<float*>(p);
      s_mu_ptr[dev] = static_cast<double*>(q);
    }
  });
  rc = check_cuda(ctx, s_lookup_err[dev], "cudaGetSymbolAddress(sap_noalloc scratch)");
  if (rc) return rc;
  *scratch = s_scratch_ptr[dev];
  *mu = s_mu_ptr[dev];
  return TMAMG_OK;
}

}  // namespace tmamg

using namespace tmamg;

extern "C" int tmamg_sap_noalloc(tmamg_ctx* ctx, void* r_bundle, void* e_bundle, int nsys, const double* mu,
                                 const int block[4], int cycles, int mr_steps) {
  if (!ctx) return TMAMG_ERR_ARG;
  if (!r_bundle || !e_bundle || !mu || !block || nsys < 1 || cycles < 1 || mr_steps < 1)
    return set_err(ctx, TMAMG_ERR_ARG, "sap_noalloc: bad argument");
  if (!ctx->have_op) return set_err(ctx, TMAMG_ERR_STATE, "sap_noalloc: operator not set");
  if (nsys > NOALLOC_SAP_MAX_SYS)
    return set_err(ctx, TMAMG_ERR_ARG, "sap_noalloc: at most " + std::to_string(NOALLOC_SAP_MAX_SYS) +
                                           " systems per call");
  size_t need = (size_t)ntiles(nsys, Tile<float>::T) * 12 * (size_t)ctx->g.V * 2 * Tile<float>::T * sizeof(float);
  if (need > NOALLOC_SAP_SCRATCH_BYTES)
    return set_err(ctx, TMAMG_ERR_ARG, "sap_noalloc: the bundle needs " + std::to_string(need) +
                                           " bytes of scratch, more than the fixed " +
                                           std::to_string(NOALLOC_SAP_SCRATCH_BYTES) + " bytes");
  std::string why;
  if (sap_check_blocks(ctx->g, block, why)) return set_err(ctx, TMAMG_ERR_ARG, "sap_noalloc: " + why);
  float* scratch = nullptr;
  double* mu_dev = nullptr;
  int rc = noalloc_addresses(ctx, &scratch, &mu_dev);
  if (rc) return rc;
  rc = check_cuda(ctx, cudaMemcpyAsync(mu_dev, mu, sizeof(double) * nsys, cudaMemcpyHostToDevice, ctx->stream),
                  "sap_noalloc: copy mu");
  if (rc) return rc;
  // the scratch needs no clearing: each sweep writes the correction of every site of its
  // colour before the face update reads it
  sap_apply(ctx->g, block, ctx->U32, ctx->C32, (float*)r_bundle, (float*)e_bundle, scratch, mu_dev, nsys, cycles,
            mr_steps, ctx->stream);
  return check_cuda(ctx, cudaGetLastError(), "sap_noalloc launch");
}

// Shared device/host definitions of the tmamg CUDA library (sm_103a).
//
// Bundle layout: real [ntile][ncomp][nsite][2][T]; T = 2 (FP32) or 1 (FP64).
// Every kernel of the library reads and writes this layout; the system index
// runs fastest inside a tile (paper Sec. 3, Fig. 2) so that one 16-byte load
// brings the same complex entry (re[T], im[T]) of T systems.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/tmamg.h"

namespace tmamg {

// number of kernels this library has launched (all contexts), for launch accounting
uint64_t& launch_counter();
#define TM_COUNT() (++::tmamg::launch_counter())

template <typename real> struct Tile;
template <> struct Tile<float> { static constexpr int T = 2; };
template <> struct Tile<double> { static constexpr int T = 1; };

struct Geom {
  int L[4];     // x, y, z, t
  int64_t V;
  int bc_t;
};

__host__ __device__ inline void site_coords(int64_t s, const int* L, int* c) {
  c[0] = (int)(s % L[0]);
  int64_t r = s / L[0];
  c[1] = (int)(r % L[1]);
  r /= L[1];
  c[2] = (int)(r % L[2]);
  c[3] = (int)(r / L[2]);
}

__host__ __device__ inline int64_t site_index(const int* c, const int* L) {
  return ((int64_t)(c[3] * L[2] + c[2]) * L[1] + c[1]) * L[0] + c[0];
}

inline int ntiles(int nsys, int T) { return (nsys + T - 1) / T; }

// one level of the multigrid hierarchy, device data owned by the context
struct CoarseLevel {
  int Lc[4] = {0, 0, 0, 0};
  int agg[4] = {0, 0, 0, 0};
  int64_t Vc = 0;
  int nv = 0;           // test vectors; coarse unknowns per site nc = 2 nv
  int asize = 0;        // fine sites per aggregate
  float2* P = nullptr;  // [Vc][2 chi][nv][asize*6] for a fine parent (6 = 2 spins x 3 colours per chirality)
  float2* A = nullptr;  // [9][Vc][nc (col j)][nc (row i)]  coarse stencil blocks, column-major per block
  __half* A16 = nullptr;  // the same blocks in FP16, in the operand layout of the tensor-core stencil
  float* cmax = nullptr;  // [CM_MAXSYS] per-system range scratch of the stand-alone tensor-core stencil
  int* cerr = nullptr;    // bounded-wait flag of the stand-alone tensor-core stencil
  __half* x16 = nullptr;  // B images of the stand-alone tensor-core stencil (grown on demand)
  size_t x16_bytes = 0;
  double2* P64 = nullptr;  // P and A widened to FP64 for the plain FP64 solver (made on first use)
  double2* A64 = nullptr;
};

constexpr int CM_MAXSYS = 1024;  // systems per stand-alone tensor-core stencil call

struct Workspace;
struct Workspace64;
struct NNState;

}  // namespace tmamg

struct tmamg_ctx {
  tmamg::Geom g;
  cudaStream_t stream = nullptr;
  std::string err;
  // gauge field: [4 mu][9][V] complex (site fastest)
  double2* U64 = nullptr;
  float2* U32 = nullptr;
  // clover + diagonal, per site 2 chiralities x 36 reals: [72][V]
  double* C64 = nullptr;
  float* C32 = nullptr;
  double kappa = 0.0, c_sw = 0.0;
  bool have_gauge = false, have_op = false, have_setup = false;
  // twisted masses on the device (per system), cached
  double* mu_dev = nullptr;
  int mu_cap = 0;
  // doublet splittings on the device (per doublet), cached
  double* eps_dev = nullptr;
  int eps_cap = 0;
  // scratch for tmamg_apply
  void* scratch[2] = {nullptr, nullptr};
  size_t scratch_bytes = 0;
  // multigrid hierarchy
  tmamg_setup_params sp;
  std::vector<tmamg::CoarseLevel> levels;
  tmamg::Workspace* ws = nullptr;
  tmamg::Workspace64* ws64 = nullptr;  // plain FP64 solver state (made on first use)
  tmamg::NNState* nn = nullptr;  // learned preconditioner step (optional)
};

namespace tmamg {

void free_levels(tmamg_ctx* ctx);
void free_workspace(tmamg_ctx* ctx);
void free_nn(tmamg_ctx* ctx);

// per-device launch facts (host, thread-safe): the SM count and the shared-memory opt-in limit
// of the current device, and a kernel's dynamic shared-memory limit raised on the current device
// (cudaFuncSetAttribute acts per device, so each device gets its own call)
int device_sms();
int device_smem_optin();
void func_smem_optin(const void* func, int bytes);

// error helpers (host)
int set_err(tmamg_ctx* ctx, int code, const std::string& msg);
int check_cuda(tmamg_ctx* ctx, cudaError_t e, const char* what);
int upload_mu(tmamg_ctx* ctx, const double* mu, int nsys);

// kernels launched from other translation units
void launch_build_clover(const Geom& g, const double2* U64, double kappa, double c_sw, double* C64, float* C32,
                         cudaStream_t st);
void launch_convert_gauge(const Geom& g, const double* Uin, double2* U64, float2* U32, cudaStream_t st);
// eps (optional): the non-degenerate doublet form, per doublet splittings (device): FP32 tiles hold the
// flavours u, d of one doublet (eps per tile), FP64 tiles 2p and 2p + 1 those of doublet p
template <typename real>
void launch_dirac(const Geom& g, const void* U, const real* C, const real* x, real* y, const double* mu, int nsys,
                  cudaStream_t st, const double* eps = nullptr);
// r = b - D(mu) x on FP32 bundles in one pass (b with the same tiles as x)
void launch_residual32(const Geom& g, const float2* U, const float* C, const float* x, const float* b, float* r,
                       const double* mu, int nsys, cudaStream_t st, const double* eps = nullptr);
// r_n = b_{n / nshift} - D(mu_n) x_n on FP64 bundles (one system per tile), b holding one tile
// per right-hand side: the outer residual of the solver without a separate product buffer
void launch_residual64(const Geom& g, const double2* U, const double* C, const double* x, const double* b, int nshift,
                       double* r, const double* mu, int nsys, cudaStream_t st, const double* eps = nullptr);
// y = M_ee(mu) x on the even sites (the even-odd Schur complement), y = 0 on the odd sites; x's odd
// entries are ignored; s0, s1: two scratch bundles of the same size
template <typename real>
void launch_dirac_eo(const Geom& g, const void* U, const real* C, const real* x, real* y, const double* mu, int nsys,
                     real* s0, real* s1, cudaStream_t st);
template <typename real>
void launch_pack(const Geom& g, const real* field, real* bundle, int nsys, cudaStream_t st);
template <typename real>
void launch_unpack(const Geom& g, const real* bundle, real* field, int nsys, cudaStream_t st);

}  // namespace tmamg

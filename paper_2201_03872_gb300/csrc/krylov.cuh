// Batched (F)GMRES over bundles with per-system convergence masks (declarations). See krylov.cu.
#pragma once
#include <functional>

#include "common.cuh"

namespace tmamg {

// Device state of m-step GMRES cycles for nsys independent systems run in lockstep.
struct GmresState {
  int m = 0, cap = 0;
  double2* H = nullptr;    // [(j (m+1) + i) cap + n]: column j, row i
  double* cs = nullptr;    // [j cap + n]
  double2* sn = nullptr;   // [j cap + n]
  double2* g = nullptr;    // [i cap + n], i <= m
  double2* y = nullptr;    // [i cap + n]
  double2* tmp = nullptr;  // [(m+1) cap]
  double2* sc = nullptr;   // [cap] scale factors
  double* beta = nullptr;  // [cap]
  double* tolabs = nullptr;
  double* resid = nullptr;
  int* kconv = nullptr;
  int* active = nullptr;
  int* nactive = nullptr;  // device counter
  int* h_nactive = nullptr;  // pinned host mirror
  double2* partial = nullptr;
  size_t partial_cap = 0;
  int alloc(int m, int cap, size_t partial_elems);
  void release();
};

template <typename real>
struct LevelOpsT {
  int64_t M;  // entries per tile (ncomp * nsite)
  std::function<void(const real* x, real* y)> A;        // y = A x for all systems
  std::function<void(const real* v, real* z)> precond;  // z = M v; empty = none
};
using LevelOps = LevelOpsT<float>;

struct CycleResult {
  int iters;  // Arnoldi steps performed (max over systems)
};

// One GMRES(m) cycle (flexible if a preconditioner is given) for nsys systems.
// V: m+1 bundles (stride vstride reals); V[0] holds the right-hand side on entry (not
// normalised). Z: m bundles (used only with a preconditioner). x: receives x += Z y
// (or V y). participate: device mask of systems to iterate (nullptr = all).
// rel_tol: device array of per-system relative tolerances (|r| <= rel_tol * |r0|).
// poll: Arnoldi steps between host checks of the active count. cgs2: re-orthogonalise.
// Vectors are FP32 bundles (tiles of 2 systems) or FP64 bundles (one system per tile).
template <typename real>
CycleResult gmres_cycle(GmresState& st, const LevelOpsT<real>& ops, int nsys, int m, real* V, int64_t vstride,
                        real* Z, real* x, const int* participate, const double* rel_tol, int poll, bool cgs2,
                        cudaStream_t s);

// small per-system kernels used by the drivers
void set_rel_tol(double* rel, int nsys, double value, cudaStream_t s);

}  // namespace tmamg

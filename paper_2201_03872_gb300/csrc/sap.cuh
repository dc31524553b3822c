// SAP smoother (declarations). See sap.cu.
#pragma once
#include <string>

#include "common.cuh"

namespace tmamg {

// 0 if the block extents tile the lattice with an even number of blocks (or one) per dimension
int sap_check_blocks(const Geom& g, const int bs[4], std::string& why);

// e = SAP(r): FP32 bundles of nsys systems. r is overwritten (it ends as a partially
// updated residual), delta is scratch of the same size, e receives the correction
// (accumulate: e += SAP(r), e is not cleared first). eps (optional, per tile): the tiles are
// non-degenerate doublets (flavours in the two lanes), each solved as one system.
void sap_apply(const Geom& g, const int bs[4], const float2* U32, const float* C32, float* r, float* e, float* delta,
               const double* mu, int nsys, int cycles, int steps, cudaStream_t st, bool accumulate = false,
               const double* eps = nullptr);

// The same smoother in FP64 (FP64 bundles, one system per tile), for the plain comparator solver.
void sap_apply64(const Geom& g, const int bs[4], const double2* U64, const double* C64, double* r, double* e,
                 double* delta, const double* mu, int nsys, int cycles, int steps, cudaStream_t st);

}  // namespace tmamg

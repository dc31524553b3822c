// Learned preconditioner step (declarations). See nn.cu.
#pragma once
#include "common.cuh"

namespace tmamg {

struct NNGeom {
  int L[4];
  int64_t V;
  int bc_t;
};

struct NNState {
  float2* W = nullptr;     // FP32 master weights, three layers [9][cout][cin] concatenated
  float2* Winf = nullptr;  // inference weights: the BF16 copy, expanded to FP32
  void* Wb16 = nullptr;    // BF16 copy (__nv_bfloat162)
  float2* Wadj = nullptr;  // adjoint weights of one layer (backward pass)
  double2* grad = nullptr;
  float2 *m1 = nullptr, *m2 = nullptr;  // Adam moments
  double2 *enorm = nullptr, *coef = nullptr;
  float* act[4] = {nullptr, nullptr, nullptr, nullptr};  // layer inputs / outputs (act[0] unused)
  float* gbuf[2] = {nullptr, nullptr};
  double2* part = nullptr;
  int64_t Vcap = 0;
  int nsys = 0;
  bool trained = false;
  bool enabled = false;  // the gate: set only when the step lowered the iteration count
  int iters_plain = 0, iters_nn = 0;
  double loss_first = 0, loss_last = 0;
  int alloc(int64_t V, int nsys);
  int alloc_weights();
  void release_buffers();
  void release();
};

int nn_weight_count(int layer);
int nn_weight_offset(int layer);  // nn_weight_offset(3) = all weights
void nn_refresh_inference(NNState& s, cudaStream_t st);
// y = N(r) on FP32 fine bundles of nsys systems (training or inference weights)
void nn_forward(NNState& s, const NNGeom& g, const float2* U, const float* r, float* y, int nsys, bool inference,
                cudaStream_t st);
// gradients of sum_n |y_n - e_n|^2 / |e_n|^2 into s.grad (needs the activations of the forward pass)
void nn_backward(NNState& s, const NNGeom& g, const float2* U, const float* r, const float* y, const float* e,
                 int nsys, double2* partial, cudaStream_t st);
void nn_loss_coef(const double2* enorm, double2* coef, int nsys, cudaStream_t st);
void nn_adam(NNState& s, float lr, int step, double gscale, cudaStream_t st);

}  // namespace tmamg

// Shared by the two training kernels of v_theta (pdds_mlp.cu: FP32 SIMT;
// pdds_mlp_train_tc.cu: BF16 products on the fifth-generation tensor cores):
// the parameter layout, the launch arguments and the device-side step state.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pdds {

// theta = W1[64][2], b1[64], W2[64][64] (row = output unit), b2[64], w3[64], b3
constexpr int kOffW1 = 0, kOffB1 = 128, kOffW2 = 192, kOffB2 = 4288, kOffW3 = 4352, kOffB3 = 4416;

// Step state of a training run (device, zeroed before the first step).
struct TrainState {
  unsigned count;  // CTAs done with the current launch
  int t;           // index of the next launch
  double p1, p2;   // beta1^t, beta2^t for launch t >= 1
};

struct TrainArgs {
  float* theta;     // parameters (training: read by launch 0, written by the last)
  const float* xy;
  const float* tgt;
  int64_t npts;
  float scale;      // 2 / N: d loss / d v
  double inv_n;     // 1 / N
  float* grad;      // gradient: one buffer (gradient only) or three (training)
  double* loss;     // loss; training: the loss history, indexed by the step
  // training only
  float *th2, *m2, *v2;  // [2][kMlpParams] each
  TrainState* st;
  int steps;
  float lr, beta1, beta2, eps;
};

// The tensor-core training kernel (pdds_mlp_train_tc.cu): its function, grid,
// block and dynamic shared memory for npts points (adam: the training
// variant, else the gradient only).
cudaError_t train_tc_launch_config(bool adam, int64_t npts, const void** fn, unsigned* grid,
                                   unsigned* threads, size_t* smem);

}  // namespace pdds

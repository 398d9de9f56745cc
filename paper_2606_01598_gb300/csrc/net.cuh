// Internal declarations of the learned charge/dipole network (net.cu, net_mix.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/gbnet.h"
#include "common.cuh"

namespace gbnet {

// device error word bits of the network kernels
constexpr int kNetFlagTimeout = 1;    // a bounded wait on the tensor cores gave up
constexpr int kNetFlagNbrFull = 2;    // an ion had more than kMaxNbr neighbours within r_c
constexpr int kNetFlagNonFinite = 4;  // a NaN or Inf position

// Y[M][NOUT] (+)= X[M][K] W on the tensor cores (net_mix.cu). Wt is W^T, [NOUT][K] bfloat16
// (K contiguous); X, Y float32 row-major, 16-byte aligned. Supported (K, NOUT): (32,48),
// (16,32), (48,48), (32,16), (32,64), (48,32), (64,32). Returns 0 or a pme_status.
int launch_mix(cudaStream_t s, int M, int K, int NOUT, const float* X, const uint16_t* Wt, float* Y,
               bool accumulate, int* err);

}  // namespace gbnet

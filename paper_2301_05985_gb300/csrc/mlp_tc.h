// mlp_tc.h -- tensor-core (tcgen05) inference of the learned-start network.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

struct MlpTcArgs {
  int64_t rows;
  const __nv_bfloat16* X;   // [rows][224] standardised features, BF16 (columns >= 216 zero)
  const __nv_bfloat16* W1;  // [224][128] row-major (k, n), rows >= 216 zero
  const __nv_bfloat16* W2;  // [128][128]
  const __nv_bfloat16* W3;  // [128][128]
  const __nv_bfloat16* W4;  // [128][8], columns >= 3 zero
  const float* b1;          // [128]
  const float* b2;
  const float* b3;
  const float* b4;          // [8]
  float* out;               // [rows][8]: columns 0..2 written
  int* err;                 // |= 1 when a wait on the tensor core gave up
};

// out = the network's output for every row (GELU hidden layers, BF16 operands and
// activations, FP32 accumulation); X and the weights 16-byte aligned.
cudaError_t launch_mlp_infer_tc(const MlpTcArgs& a, cudaStream_t s);
size_t mlp_tc_smem_bytes();

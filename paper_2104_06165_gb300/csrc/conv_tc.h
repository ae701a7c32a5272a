// Tensor-core convolutions of the proposal network (conv_tc.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

// weights [co][tap][ci] (fp32) -> bf16 B operand in the order conv_tc_launch
// reads (chunk-major, see conv_tc.cu); flip = 1 gives the data-gradient
// filter (N = ci, K = co, taps reversed)
cudaError_t conv_tc_weights(const float* w, int co_n, int taps, int ci_n, int flip, __nv_bfloat16* out,
                            cudaStream_t s);
// input channels per pipeline chunk of a convolution (K inputs, N outputs)
int conv_tc_chunk(int K, int N, int taps);
// out[p][out_off + n] = act(bias[n] + sum over taps t and input channels k of
// in[p + offset(t)][k] wt[t][k][n]) for the W x H channels-last tensor `in`
// (Cin channels, zero outside the image), n < Cout; taps 9 (3 x 3) or 1.
// `status` (device int) receives MVS_DEV_TIMEOUT if a bounded wait ran out;
// force_timeout makes the first wait target a barrier that nothing completes.
cudaError_t conv_tc_launch(const __nv_bfloat16* in, int Cin, int W, int H, const __nv_bfloat16* wt, const float* bias,
                           int taps, int Cout, bool relu, bool out_f32, void* out, int out_ch, int out_off,
                           int* status, int force_timeout, unsigned wait_limit, cudaStream_t s);

/*
 * pat_unet.h - C ABI of the learned warm start for the TV-Bregman solver: the layers of a 3D U-Net
 * (4 levels, 16/32/64/128 channels) that maps the back-projection A^T C^T f to a starting image,
 * trained on phantoms paired with their own TV-Bregman reconstructions.  The paper has no learned
 * component; the solver it warm-starts is Sec. 4.5-4.6 (TV+ with Bregman iterations, App. B), which
 * stays the fallback and the reference the warm start's error is measured against.
 *
 * Conventions (in addition to those of pat.h):
 *   Activations are channels-last BF16 tensors [V][ld] (V = D*H*W voxels, z slowest, x fastest);
 *   a tensor argument is a pointer to its first channel plus the row stride `ld` (so a channel slice
 *   of a wider buffer is passed as base + offset with the buffer's ld).  Channel counts and strides
 *   are multiples of 16 and pointers 16-byte aligned.  Convolutions are 3x3x3, stride 1, zero
 *   padding 1, no bias; weights are [27][Cout][Cin] (tap t = 9 (dz+1) + 3 (dy+1) + (dx+1)).
 *   Tensor cores: BF16 operands with FP32 accumulation, tcgen05 with tensor-memory accumulators and
 *   TMA-staged operands, for the convolution, its data gradient (the convolution with transposed
 *   weights) and its weight gradient.  All calls are ordered on the given stream and return
 *   without synchronising; invalid arguments return PAT_ERR_INVALID_ARG before anything is
 *   launched.
 */
#ifndef PAT_UNET_H
#define PAT_UNET_H

#include <stdint.h>

#include "pat.h"

#ifdef __cplusplus
extern "C" {
#endif

/* y = act(conv3(x, w)): x [V][ldx] (cin channels), w bf16 [27][cout][cin], y [V][ldy] (cout
 * channels, overwritten).  relu != 0 applies max(0, .).  cin in 16..512 and cout in 16..1024,
 * multiples of 16.  The kernel bounds its waits; one that gives up is reported by
 * pat_unet_device_status. */
pat_status pat_unet_conv3(const void* x, int32_t ldx, int32_t cin, const void* w, int32_t cout, void* y,
                          int32_t ldy, int32_t D, int32_t H, int32_t W, int32_t relu, void* cuda_stream);

/* Synchronises cuda_stream, then reads and clears the device word in which the tensor-core
 * convolutions record a bounded wait that gave up: PAT_OK, or PAT_ERR_TIMEOUT (the outputs of the
 * convolutions since the last check are invalid). */
pat_status pat_unet_device_status(void* cuda_stream);

/* Test hook for that failure path (no counterpart in the paper), process-wide: while
 * stop_after_stage >= 0, the convolutions (pat_unet_conv3) issue the TMA copies of only their first
 * stop_after_stage K steps and give up waiting for the next after `polls` polls (0: the default);
 * nothing is left in flight, each CTA frees its tensor memory and exits, the outputs are invalid and
 * pat_unet_device_status reports PAT_ERR_TIMEOUT.  stop_after_stage = -1 restores normal operation. */
pat_status pat_unet_debug_copy_fault(int32_t stop_after_stage, int32_t polls);

/* Weight gradient of pat_unet_conv3: dw[t][co][ci] = sum_v dy[v][co] x[v + off_t][ci] (FP32,
 * overwritten), dy the gradient at the convolution's output (after the activation's backward);
 * cin in 16..256, cout in 16..128 (multiples of 16), strides multiples of 16.  One GEMM over all
 * taps (rows t cin + ci, columns co, reduction over voxels) split over voxel chunks.
 * partial: FP32 scratch of at least pat_unet_wgrad_scratch(...) floats, 16-byte aligned;
 * deterministic (fixed-order sum of the chunks).  Bounded waits as pat_unet_conv3. */
int64_t pat_unet_wgrad_scratch(int32_t cin, int32_t cout, int32_t D, int32_t H, int32_t W);
pat_status pat_unet_conv3_wgrad(const void* x, int32_t ldx, int32_t cin, const void* dy, int32_t ldy,
                                int32_t cout, int32_t D, int32_t H, int32_t W, float* partial, float* dw,
                                void* cuda_stream);

/* From FP32 master weights w32 [27][cout][cin]: wb = bf16 copy (same layout), wt = bf16 weights of
 * the transposed convolution [27][cin][cout] with wt[t][ci][co] = w32[26 - t][co][ci], so that
 * pat_unet_conv3(dy, ..., wt, cin, dx, ...) is the gradient with respect to x. */
pat_status pat_unet_cast_weights(const float* w32, int32_t cin, int32_t cout, void* wb, void* wt,
                                 void* cuda_stream);

/* In place: g[v][c] = 0 where y[v][c] <= 0 (backward of the ReLU whose output is y). */
pat_status pat_unet_relu_bwd(void* g, int32_t ldg, const void* y, int32_t ldy, int32_t C, int64_t V,
                             void* cuda_stream);

/* 2x2x2 average pooling: x [D][H][W][.] -> y [D/2][H/2][W/2][.], C channels. */
pat_status pat_unet_pool(const void* x, int32_t ldx, int32_t C, int32_t D, int32_t H, int32_t W, void* y,
                         int32_t ldy, void* cuda_stream);
/* Its backward, accumulated: dx[child] += dy[parent] / 8 (dims of x given). */
pat_status pat_unet_pool_bwd_add(const void* dy, int32_t ldd, int32_t C, int32_t D, int32_t H, int32_t W,
                                 void* dx, int32_t ldx, void* cuda_stream);

/* Nearest-neighbour 2x upsampling: x [D][H][W][.] -> y [2D][2H][2W][.]; backward sums the 8
 * children: dx[parent] = sum dy[child] (dims of x given). */
pat_status pat_unet_up(const void* x, int32_t ldx, int32_t C, int32_t D, int32_t H, int32_t W, void* y,
                       int32_t ldy, void* cuda_stream);
pat_status pat_unet_up_bwd(const void* dy, int32_t ldd, int32_t C, int32_t D, int32_t H, int32_t W,
                           void* dx, int32_t ldx, void* cuda_stream);

/* Network input: x16 [V][16] bf16 with channel 0 = s * xin[v] (FP32) and channels 1..15 zero. */
pat_status pat_unet_input(const float* xin, float s, int64_t V, void* x16, void* cuda_stream);

/* Output layer, a 1x1x1 convolution with bias: out[v] = head[16] + sum_c head[c] h[v][c], h [V][16]
 * bf16, head FP32[17], out FP32[V]. */
pat_status pat_unet_head(const void* h, const float* head, int64_t V, float* out, void* cuda_stream);

/* Loss and output-layer backward for the mean squared error L = sum_v (out - target)^2 / V:
 * dh[v][c] = g[v] head[c] (bf16 [V][16]) with g = 2 (out - target) / V, ghead[c] = sum_v g h[v][c],
 * ghead[16] = sum_v g, loss[0] = L.  partial: FP64 scratch of pat_unet_head_scratch(V) doubles. */
int64_t pat_unet_head_scratch(int64_t V);
pat_status pat_unet_head_bwd(const void* h, const float* head, const float* out, const float* target,
                             int64_t V, void* dh, float* ghead, double* loss, double* partial,
                             void* cuda_stream);

/* Adam step on n FP32 parameters: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps). */
pat_status pat_unet_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1,
                         float b2, float eps, int32_t step, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PAT_UNET_H */

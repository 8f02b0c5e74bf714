// pat_unet.cu - layers of the learned warm start (a 3D U-Net mapping A^T C^T f to a starting image
// for the TV-Bregman solver): the C ABI of the 3x3x3 convolutions, their data and weight gradients
// (on the tcgen05 tensor cores, pat_unet_tc.cu), and the elementwise layers around them (pooling,
// upsampling, ReLU backward, the input and output layers, the loss and Adam).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/pat_unet.h"
#include "pat_internal.h"

namespace pat {
cudaError_t conv3_tc(const void* x, int ldx, int cin, const void* w, int cout, void* y, int ldy, int D, int H,
                     int W, int relu, cudaStream_t st);
cudaError_t unet_take_status(int* word, cudaStream_t st);
void unet_set_copy_fault(int stop_after, int polls);
int64_t wgrad_tc_scratch(int cin, int cout, int D, int H, int W);
cudaError_t wgrad_tc(const void* x, int ldx, int cin, const void* dy, int ldy, int cout, int D, int H, int W,
                     float* partial, float* dw, cudaStream_t st);
}  // namespace pat

namespace {

typedef __nv_bfloat16 bf16;


__global__ void cast_weights_kernel(const float* __restrict__ w32, int cin, int cout, bf16* __restrict__ wb,
                                    bf16* __restrict__ wt) {
    const int n = 27 * cin * cout;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int t = i / (cout * cin), r = i - t * cout * cin, co = r / cin, ci = r - co * cin;
        const bf16 b = __float2bfloat16(w32[i]);
        wb[i] = b;
        wt[((size_t)(26 - t) * cin + ci) * cout + co] = b;
    }
}

__global__ void relu_bwd_kernel(bf16* __restrict__ g, int ldg, const bf16* __restrict__ y, int ldy, int C, long long V) {
    const long long n = V * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long v = i / C;
        const int c = (int)(i - v * C);
        if (!(__bfloat162float(y[v * ldy + c]) > 0.f)) g[v * ldg + c] = __float2bfloat16(0.f);
    }
}

__global__ void pool_kernel(const bf16* __restrict__ x, int ldx, int C, int D, int H, int W, bf16* __restrict__ y, int ldy) {
    const int D2 = D / 2, H2 = H / 2, W2 = W / 2;
    const long long n = (long long)D2 * H2 * W2 * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long p = i / C;
        const int z = (int)(p / (H2 * W2)), r = (int)(p - (long long)z * H2 * W2), yy = r / W2, xx = r - yy * W2;
        float s = 0.f;
        for (int k = 0; k < 8; k++) {
            const int cz = 2 * z + (k >> 2), cy = 2 * yy + ((k >> 1) & 1), cx = 2 * xx + (k & 1);
            s += __bfloat162float(x[((size_t)(cz * H + cy) * W + cx) * ldx + c]);
        }
        y[p * ldy + c] = __float2bfloat16(0.125f * s);
    }
}

__global__ void pool_bwd_add_kernel(const bf16* __restrict__ dy, int ldd, int C, int D, int H, int W, bf16* __restrict__ dx, int ldx) {
    const long long n = (long long)D * H * W * C;
    const int H2 = H / 2, W2 = W / 2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long v = i / C;
        const int z = (int)(v / (H * W)), r = (int)(v - (long long)z * H * W), yy = r / W, xx = r - yy * W;
        const long long pp = ((long long)(z / 2) * H2 + yy / 2) * W2 + xx / 2;
        const float g = 0.125f * __bfloat162float(dy[pp * ldd + c]);
        dx[v * ldx + c] = __float2bfloat16(__bfloat162float(dx[v * ldx + c]) + g);
    }
}

__global__ void up_kernel(const bf16* __restrict__ x, int ldx, int C, int D, int H, int W, bf16* __restrict__ y, int ldy) {
    const int D2 = 2 * D, H2 = 2 * H, W2 = 2 * W;
    const long long n = (long long)D2 * H2 * W2 * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long v = i / C;
        const int z = (int)(v / (H2 * W2)), r = (int)(v - (long long)z * H2 * W2), yy = r / W2, xx = r - yy * W2;
        y[v * ldy + c] = x[((size_t)((z / 2) * H + yy / 2) * W + xx / 2) * ldx + c];
    }
}

__global__ void up_bwd_kernel(const bf16* __restrict__ dy, int ldd, int C, int D, int H, int W, bf16* __restrict__ dx, int ldx) {
    const long long n = (long long)D * H * W * C;
    const int H2 = 2 * H, W2 = 2 * W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long p = i / C;
        const int z = (int)(p / (H * W)), r = (int)(p - (long long)z * H * W), yy = r / W, xx = r - yy * W;
        float s = 0.f;
        for (int k = 0; k < 8; k++) {
            const int cz = 2 * z + (k >> 2), cy = 2 * yy + ((k >> 1) & 1), cx = 2 * xx + (k & 1);
            s += __bfloat162float(dy[((size_t)(cz * H2 + cy) * W2 + cx) * ldd + c]);
        }
        dx[p * ldx + c] = __float2bfloat16(s);
    }
}

__global__ void input_kernel(const float* __restrict__ xin, float s, long long V, bf16* __restrict__ x16) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V * 16; i += (long long)gridDim.x * blockDim.x) {
        const long long v = i >> 4;
        x16[i] = __float2bfloat16((i & 15) == 0 ? s * xin[v] : 0.f);
    }
}

__global__ void head_kernel(const bf16* __restrict__ h, const float* __restrict__ head, long long V, float* __restrict__ out) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        float s = head[16];
#pragma unroll
        for (int c = 0; c < 16; c++) s = fmaf(head[c], __bfloat162float(h[v * 16 + c]), s);
        out[v] = s;
    }
}

constexpr int kHeadBlocks = 256;
// per block: 16 channel sums of g h, the sum of g, the sum of squared errors (fixed-order tree)
__global__ void __launch_bounds__(256) head_bwd_kernel(const bf16* __restrict__ h, const float* __restrict__ head,
                                                       const float* __restrict__ out, const float* __restrict__ target,
                                                       long long V, bf16* __restrict__ dh, double* __restrict__ partial) {
    __shared__ double red[256][18];
    double acc[18];
    for (int k = 0; k < 18; k++) acc[k] = 0.0;
    const double gs = 2.0 / (double)V;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        const double e = (double)out[v] - (double)target[v];
        const float g = (float)(gs * e);
#pragma unroll
        for (int c = 0; c < 16; c++) {
            const float hv = __bfloat162float(h[v * 16 + c]);
            acc[c] += (double)g * hv;
            dh[v * 16 + c] = __float2bfloat16(g * head[c]);
        }
        acc[16] += g;
        acc[17] += e * e;
    }
    for (int k = 0; k < 18; k++) red[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 18; k++) red[threadIdx.x][k] += red[threadIdx.x + w][k];
        __syncthreads();
    }
    if (threadIdx.x < 18) partial[(size_t)blockIdx.x * 18 + threadIdx.x] = red[0][threadIdx.x];
}

__global__ void head_bwd_final_kernel(const double* __restrict__ partial, int nb, long long V, float* __restrict__ ghead,
                                      double* __restrict__ loss) {
    const int k = threadIdx.x;
    if (k >= 18) return;
    double s = 0.0;
    for (int b = 0; b < nb; b++) s += partial[(size_t)b * 18 + k];
    if (k < 17) ghead[k] = (float)s;
    else loss[0] = s / (double)V;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                            long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

unsigned grid_for(long long n, int nt = 256) {
    const long long b = (n + nt - 1) / nt;
    return (unsigned)std::max(1LL, std::min(b, 152LL * 16));
}

bool al16(const void* p) { return ((uintptr_t)p & 15) == 0; }

pat_status bad(const char* msg) { return pat::set_error(PAT_ERR_INVALID_ARG, msg); }

pat_status launched(const char* where) {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PAT_OK : pat::set_cuda_error(e, where);
}

}  // namespace

extern "C" {

pat_status pat_unet_conv3(const void* x, int32_t ldx, int32_t cin, const void* w, int32_t cout, void* y,
                          int32_t ldy, int32_t D, int32_t H, int32_t W, int32_t relu, void* stream) {
    if (!x || !w || !y) return bad("pat_unet_conv3: NULL pointer");
    if (cin < 16 || cin > 512 || cin % 16 || ldx < cin || ldx % 16 || ldy < cout || ldy % 16)
        return bad("pat_unet_conv3: channel counts and strides must be multiples of 16 (cin <= 512)");
    if (cout < 16 || cout > 1024 || cout % 16) return bad("pat_unet_conv3: cout must be a multiple of 16 (<= 1024)");
    if (D < 1 || H < 1 || W < 1 || (int64_t)D * H * W > (1LL << 30)) return bad("pat_unet_conv3: bad volume");
    if (!al16(x) || !al16(w) || !al16(y)) return bad("pat_unet_conv3: pointers must be 16-byte aligned");
    const cudaError_t e = pat::conv3_tc(x, ldx, cin, w, cout, y, ldy, D, H, W, relu, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return pat::set_cuda_error(e, "pat_unet_conv3");
    }
    return PAT_OK;
}

pat_status pat_unet_debug_copy_fault(int32_t stop_after_stage, int32_t polls) {
    if (stop_after_stage < -1 || polls < 0) return bad("pat_unet_debug_copy_fault: stop_after_stage >= -1, polls >= 0");
    pat::unet_set_copy_fault(stop_after_stage, polls);
    pat::set_error(PAT_OK, "");
    return PAT_OK;
}

pat_status pat_unet_device_status(void* stream) {
    int word = 0;
    const cudaError_t e = pat::unet_take_status(&word, (cudaStream_t)stream);
    if (e != cudaSuccess) return pat::set_cuda_error(e, "pat_unet_device_status");
    if (word) return pat::set_error(PAT_ERR_TIMEOUT, "pat_unet_device_status: a tensor-core convolution gave up "
                                                     "waiting for its copies or its matrix multiplies");
    pat::set_error(PAT_OK, "");
    return PAT_OK;
}

int64_t pat_unet_wgrad_scratch(int32_t cin, int32_t cout, int32_t D, int32_t H, int32_t W) {
    if (cin < 16 || cout < 16 || D < 1 || H < 1 || W < 1) return 0;
    return pat::wgrad_tc_scratch(cin, cout, D, H, W);
}

pat_status pat_unet_conv3_wgrad(const void* x, int32_t ldx, int32_t cin, const void* dy, int32_t ldy, int32_t cout,
                                int32_t D, int32_t H, int32_t W, float* partial, float* dw, void* stream) {
    if (!x || !dy || !partial || !dw) return bad("pat_unet_conv3_wgrad: NULL pointer");
    if (cin < 16 || cin > 256 || cin % 16 || ldx < cin || ldx % 16 || ldy < cout || ldy % 16 || cout < 16 ||
        cout > 128 || cout % 16)
        return bad("pat_unet_conv3_wgrad: cin in 16..256 and cout in 16..128, multiples of 16; strides too");
    if (!al16(x) || !al16(dy) || !al16(partial)) return bad("pat_unet_conv3_wgrad: pointers must be 16-byte aligned");
    if (D < 1 || H < 1 || W < 1 || (int64_t)D * H * W > (1LL << 30)) return bad("pat_unet_conv3_wgrad: bad volume");
    const cudaError_t e = pat::wgrad_tc(x, ldx, cin, dy, ldy, cout, D, H, W, partial, dw, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return pat::set_cuda_error(e, "pat_unet_conv3_wgrad");
    }
    return PAT_OK;
}

pat_status pat_unet_cast_weights(const float* w32, int32_t cin, int32_t cout, void* wb, void* wt, void* stream) {
    if (!w32 || !wb || !wt || cin < 1 || cout < 1) return bad("pat_unet_cast_weights: bad argument");
    const long long n = 27LL * cin * cout;
    cast_weights_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(w32, cin, cout, (bf16*)wb, (bf16*)wt);
    return launched("pat_unet_cast_weights");
}

pat_status pat_unet_relu_bwd(void* g, int32_t ldg, const void* y, int32_t ldy, int32_t C, int64_t V, void* stream) {
    if (!g || !y || C < 1 || ldg < C || ldy < C || V < 0) return bad("pat_unet_relu_bwd: bad argument");
    relu_bwd_kernel<<<grid_for(V * C), 256, 0, (cudaStream_t)stream>>>((bf16*)g, ldg, (const bf16*)y, ldy, C, V);
    return launched("pat_unet_relu_bwd");
}

pat_status pat_unet_pool(const void* x, int32_t ldx, int32_t C, int32_t D, int32_t H, int32_t W, void* y, int32_t ldy,
                         void* stream) {
    if (!x || !y || C < 1 || ldx < C || ldy < C || D < 2 || H < 2 || W < 2 || (D | H | W) & 1)
        return bad("pat_unet_pool: bad argument (even dims >= 2)");
    pool_kernel<<<grid_for((long long)D * H * W / 8 * C), 256, 0, (cudaStream_t)stream>>>((const bf16*)x, ldx, C, D, H, W,
                                                                                       (bf16*)y, ldy);
    return launched("pat_unet_pool");
}

pat_status pat_unet_pool_bwd_add(const void* dy, int32_t ldd, int32_t C, int32_t D, int32_t H, int32_t W, void* dx,
                                 int32_t ldx, void* stream) {
    if (!dy || !dx || C < 1 || ldx < C || ldd < C || D < 2 || H < 2 || W < 2 || (D | H | W) & 1)
        return bad("pat_unet_pool_bwd_add: bad argument (even dims >= 2)");
    pool_bwd_add_kernel<<<grid_for((long long)D * H * W * C), 256, 0, (cudaStream_t)stream>>>(
        (const bf16*)dy, ldd, C, D, H, W, (bf16*)dx, ldx);
    return launched("pat_unet_pool_bwd_add");
}

pat_status pat_unet_up(const void* x, int32_t ldx, int32_t C, int32_t D, int32_t H, int32_t W, void* y, int32_t ldy,
                       void* stream) {
    if (!x || !y || C < 1 || ldx < C || ldy < C || D < 1 || H < 1 || W < 1) return bad("pat_unet_up: bad argument");
    up_kernel<<<grid_for(8LL * D * H * W * C), 256, 0, (cudaStream_t)stream>>>((const bf16*)x, ldx, C, D, H, W, (bf16*)y,
                                                                              ldy);
    return launched("pat_unet_up");
}

pat_status pat_unet_up_bwd(const void* dy, int32_t ldd, int32_t C, int32_t D, int32_t H, int32_t W, void* dx, int32_t ldx,
                           void* stream) {
    if (!dy || !dx || C < 1 || ldx < C || ldd < C || D < 1 || H < 1 || W < 1) return bad("pat_unet_up_bwd: bad argument");
    up_bwd_kernel<<<grid_for((long long)D * H * W * C), 256, 0, (cudaStream_t)stream>>>((const bf16*)dy, ldd, C, D, H, W,
                                                                                       (bf16*)dx, ldx);
    return launched("pat_unet_up_bwd");
}

pat_status pat_unet_input(const float* xin, float s, int64_t V, void* x16, void* stream) {
    if (!xin || !x16 || V < 0) return bad("pat_unet_input: bad argument");
    input_kernel<<<grid_for(V * 16), 256, 0, (cudaStream_t)stream>>>(xin, s, V, (bf16*)x16);
    return launched("pat_unet_input");
}

pat_status pat_unet_head(const void* h, const float* head, int64_t V, float* out, void* stream) {
    if (!h || !head || !out || V < 0) return bad("pat_unet_head: bad argument");
    head_kernel<<<grid_for(V), 256, 0, (cudaStream_t)stream>>>((const bf16*)h, head, V, out);
    return launched("pat_unet_head");
}

int64_t pat_unet_head_scratch(int64_t V) {
    (void)V;
    return (int64_t)kHeadBlocks * 18;
}

pat_status pat_unet_head_bwd(const void* h, const float* head, const float* out, const float* target, int64_t V, void* dh,
                             float* ghead, double* loss, double* partial, void* stream) {
    if (!h || !head || !out || !target || !dh || !ghead || !loss || !partial || V < 1)
        return bad("pat_unet_head_bwd: bad argument");
    const cudaStream_t st = (cudaStream_t)stream;
    head_bwd_kernel<<<kHeadBlocks, 256, 0, st>>>((const bf16*)h, head, out, target, V, (bf16*)dh, partial);
    head_bwd_final_kernel<<<1, 32, 0, st>>>(partial, kHeadBlocks, V, ghead, loss);
    return launched("pat_unet_head_bwd");
}

pat_status pat_unet_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps,
                         int32_t step, void* stream) {
    if (!p || !g || !m || !v || n < 0 || step < 1) return bad("pat_unet_adam: bad argument");
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return launched("pat_unet_adam");
}

}  // extern "C"

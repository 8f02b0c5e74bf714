// pat_zpass.cu - z transforms of a 3D half spectrum, in place, outside the time loop:
//   zfft_fwd  [b][z][c] -> [b][kz][c]           completes the 3D FFT of the image p0
//   zfft_inv  [b][kz][c] -> scale * [b][z][c]   first half of the adjoint's inverse 3D FFT
// with c = kx*ny + ky the half-spectrum column.  A CTA owns TC consecutive columns over all z, so
// working in place is safe: every load of a column happens before the barrier that precedes its
// first store.  Each column's length-NZ transform is the two-pass split of pat_fft.cuh; the
// exchange goes through shared memory laid out [row][column] with the column index fastest.
#include "pat_fft.cuh"
#include "pat_kargs.h"

namespace pat {

template <int NZ>
struct ZS {
    static constexpr int A = Split<NZ>::A;
    static constexpr int B = Split<NZ>::B;
    static constexpr int TC = kZCols;
    static constexpr int NT = A * TC;       // threads per CTA
    static constexpr int BUF = NZ * TC;     // exchange buffer (float2)
    static constexpr size_t smem = (size_t)BUF * sizeof(float2);
};

template <int NZ>
__global__ void __launch_bounds__(ZS<NZ>::NT) zfft_fwd_kernel(ZArgs a) {
    using S = ZS<NZ>;
    constexpr int A = S::A, B = S::B, TC = S::TC;
    extern __shared__ float4 smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    const int tid = threadIdx.x, cl = tid % TC, r = tid / TC;
    const int ncols = a.g.nxh * a.g.ny;
    const int col = blockIdx.x * TC + cl;
    const bool vcol = col < ncols;
    float2* sp = a.spec + (size_t)blockIdx.y * a.g.nspec + col;
    pdl_wait();
    pdl_trigger();
    // pass 1 (thread t = r < B): x[t + B m], A-point DFT, twiddle, rows k1 B + t
    if (vcol && r < B) {
        float2 v[A];
#pragma unroll
        for (int m = 0; m < A; m++) v[m] = sp[(size_t)(r + B * m) * ncols];
        Dft<A, -1>::run(v);
        float2* dst = buf + r * TC + cl;
#pragma unroll
        for (int k1 = 0; k1 < A; k1++)
            dst[k1 * B * TC] = (k1 == 0) ? v[0] : cmul(v[k1], twiddle<NZ, -1>(a.tw_z, r * k1));
    }
    __syncthreads();
    // pass 2 (thread k1 = r < A): B-point DFT of rows k1 B .. k1 B + B-1 -> X[k1 + A k2]
    if (vcol) {
        float2 v[B];
        const float2* src = buf + r * B * TC + cl;
#pragma unroll
        for (int t = 0; t < B; t++) v[t] = src[t * TC];
        Dft<B, -1>::run(v);
#pragma unroll
        for (int k2 = 0; k2 < B; k2++) sp[(size_t)(r + A * k2) * ncols] = v[k2];
    }
}

template <int NZ>
__global__ void __launch_bounds__(ZS<NZ>::NT) zfft_inv_kernel(ZArgs a) {
    using S = ZS<NZ>;
    constexpr int A = S::A, B = S::B, TC = S::TC;
    extern __shared__ float4 smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    const int tid = threadIdx.x, cl = tid % TC, r = tid / TC;
    const int ncols = a.g.nxh * a.g.ny;
    const int col = blockIdx.x * TC + cl;
    const bool vcol = col < ncols;
    float2* sp = a.spec + (size_t)blockIdx.y * a.g.nspec + col;
    pdl_wait();
    pdl_trigger();
    // pass 1 (thread t' = r < A): X[r + A m'], B-point DFT, twiddle, rows k1' A + t'
    if (vcol) {
        float2 v[B];
#pragma unroll
        for (int m = 0; m < B; m++) v[m] = cscale(sp[(size_t)(r + A * m) * ncols], a.scale);
        Dft<B, +1>::run(v);
        float2* dst = buf + r * TC + cl;
#pragma unroll
        for (int k1 = 0; k1 < B; k1++)
            dst[k1 * A * TC] = (k1 == 0) ? v[0] : cmul(v[k1], twiddle<NZ, +1>(a.tw_z, r * k1));
    }
    __syncthreads();
    // pass 2 (thread k1' = r < B): A-point DFT -> x[k1' + B k2']
    if (vcol && r < B) {
        float2 v[A];
        const float2* src = buf + r * A * TC + cl;
#pragma unroll
        for (int t = 0; t < A; t++) v[t] = src[t * TC];
        Dft<A, +1>::run(v);
#pragma unroll
        for (int k2 = 0; k2 < A; k2++) sp[(size_t)(r + B * k2) * ncols] = v[k2];
    }
}

template <int NZ>
static ZKernels make_z() {
    ZKernels k;
    k.fwd = zfft_fwd_kernel<NZ>;
    k.inv = zfft_inv_kernel<NZ>;
    k.smem = ZS<NZ>::smem;
    k.tc = ZS<NZ>::TC;
    k.nt = ZS<NZ>::NT;
    return k;
}

ZKernels z_kernels_for(int nz) {
    switch (nz) {
        case 8: return make_z<8>();
        case 16: return make_z<16>();
        case 32: return make_z<32>();
        case 64: return make_z<64>();
        case 128: return make_z<128>();
        case 256: return make_z<256>();
        default: return ZKernels{};
    }
}

}  // namespace pat

// pat_zpass.cu - z-pass kernels: z-FFT of the (y,x)-transformed fields, multiply by the staggered
// k-space derivative i k_i kappa(|k|) exp(+/- i k_i dx / 2) / N, inverse z-FFT, all in one pass.
//
// A CTA owns TC consecutive half-spectrum columns (kx, ky) over all kz.  Each column's length-NZ
// transform is the two-pass split of pat_fft.cuh: pass 1 reads the column straight from global
// memory into registers, the exchange goes through shared memory laid out [row][column] with the
// column index fastest (consecutive threads touch consecutive words: no bank conflicts), pass 2
// ends in registers holding X[k1 + A k2], where the multiply happens, and the inverse transform's
// first pass starts from the same registers.
//   grad3 : one input, three outputs (gradient of p: the forward step's first half)
//   each3 : three inputs, three outputs, one derivative each (divergence terms; adjoint gradient)
//   sum3  : three inputs, one output, the sum of the three derivatives (adjoint divergence)
#include "pat_fft.cuh"
#include "pat_kargs.h"

namespace pat {

template <int NZ>
struct ZS {
    static constexpr int A = Split<NZ>::A;  // forward R1 = inverse R2
    static constexpr int B = Split<NZ>::B;  // forward R2 = inverse R1
    static constexpr int TC = kZCols;
    static constexpr int NT = A * TC;       // threads per CTA
    static constexpr int BUF = NZ * TC;     // one field's exchange buffer (float2)
    static constexpr size_t smem = 3 * (size_t)BUF * sizeof(float2);
};

template <int NZ>
struct ZCtx {
    using S = ZS<NZ>;
    const ZArgs& a;
    float2* buf;
    int cl, r, col, ky, kx;
    bool vcol;
    size_t boff, zst;

    __device__ ZCtx(const ZArgs& args, float2* smem) : a(args), buf(smem) {
        const int tid = threadIdx.x;
        cl = tid % S::TC;
        r = tid / S::TC;
        const int ncols = a.g.ny * a.g.nxh;  // half-spectrum columns, stored (kx, ky) with ky fastest
        col = blockIdx.x * S::TC + cl;
        vcol = col < ncols;
        zst = (size_t)ncols;
        boff = (size_t)blockIdx.y * a.g.nspec;
        kx = vcol ? col / a.g.ny : 0;
        ky = vcol ? col - kx * a.g.ny : 0;
    }
    // forward pass 1 of one column (role t = r < B) into buffer f
    __device__ __forceinline__ void f1(const float2* __restrict__ in, int f) {
        constexpr int A = S::A, B = S::B;
        if (r < B && vcol) {
            float2 v[A];
            load(in, v);
            f1_from(v, f);
        }
    }
    // the column's values x[t + B m], m < A, of role t = r
    __device__ __forceinline__ void load(const float2* __restrict__ in, float2* v) const {
        constexpr int A = S::A, B = S::B;
#pragma unroll
        for (int m = 0; m < A; m++) v[m] = in[boff + (size_t)(r + B * m) * zst + col];
    }
    __device__ __forceinline__ void f1_from(float2* v, int f) {
        constexpr int A = S::A, B = S::B, TC = S::TC;
        const int t = r;
        Dft<A, -1>::run(v);
        float2* dst = buf + f * S::BUF + t * TC + cl;
#pragma unroll
        for (int k1 = 0; k1 < A; k1++) {
            const float2 w = (k1 == 0) ? v[k1] : cmul(v[k1], twiddle<NZ, -1>(a.tw_z, t * k1));
            dst[k1 * B * TC] = w;
        }
    }
    // pass 1 of all three inputs, every global load issued before the first transform
    __device__ __forceinline__ void f1_three() {
        constexpr int A = S::A, B = S::B;
        if (r < B && vcol) {
            float2 v0[A], v1[A], v2[A];
            load(a.spec[0], v0);
            load(a.spec[1], v1);
            load(a.spec[2], v2);
            f1_from(v0, 0);
            f1_from(v1, 1);
            f1_from(v2, 2);
        }
    }
    // forward pass 2 (role k1 = r < A): v[k2] = X[k1 + A k2]
    __device__ __forceinline__ void f2(int f, float2* v) {
        constexpr int A = S::A, B = S::B, TC = S::TC;
        const float2* src = buf + f * S::BUF + r * B * TC + cl;
#pragma unroll
        for (int t = 0; t < B; t++) v[t] = src[t * TC];
        Dft<B, -1>::run(v);
        (void)A;
    }
    // kappa(|k|)/N at this thread's kz = r + A k2 (pass-2 role), loaded with the first pass's data
    __device__ __forceinline__ void load_kappa(float* kap) const {
        constexpr int A = S::A, B = S::B;
#pragma unroll
        for (int k2 = 0; k2 < B; k2++) kap[k2] = vcol ? __ldg(a.kappaN + (size_t)(r + A * k2) * zst + col) : 0.f;
    }
    // k-space factor of axis o at kz, given kappa/N there
    __device__ __forceinline__ float2 mult(int o, int kz, float kap) const {
        const int ki = (o == 0) ? kz : (o == 1 ? ky : kx);
        return cscale(__ldg(a.dt[o] + ki), kap);
    }
    // inverse pass 1 from registers (thread t' = r holds x'[r + A m'], m' < B) into buffer f
    __device__ __forceinline__ void i1(float2* w, int f) {
        constexpr int A = S::A, B = S::B, TC = S::TC;
        Dft<B, +1>::run(w);
        const int tp = r;
        float2* dst = buf + f * S::BUF + tp * TC + cl;
#pragma unroll
        for (int k1p = 0; k1p < B; k1p++) {
            const float2 v = (k1p == 0) ? w[k1p] : cmul(w[k1p], twiddle<NZ, +1>(a.tw_z, tp * k1p));
            dst[k1p * A * TC] = v;
        }
    }
    // inverse pass 2 (role k1' = r < B) and store
    __device__ __forceinline__ void i2(float2* __restrict__ out, int f) {
        constexpr int A = S::A, B = S::B, TC = S::TC;
        if (r < B && vcol) {
            const int k1p = r;
            float2 v[A];
            const float2* src = buf + f * S::BUF + k1p * A * TC + cl;
#pragma unroll
            for (int t = 0; t < A; t++) v[t] = src[t * TC];
            Dft<A, +1>::run(v);
#pragma unroll
            for (int k2p = 0; k2p < A; k2p++) out[boff + (size_t)(k1p + B * k2p) * zst + col] = v[k2p];
        }
    }
};

template <int NZ>
__global__ void __launch_bounds__(ZS<NZ>::NT) zpass_grad3_kernel(ZArgs a) {
    using S = ZS<NZ>;
    constexpr int A = S::A, B = S::B;
    extern __shared__ float4 smem_raw[];
    ZCtx<NZ> c(a, reinterpret_cast<float2*>(smem_raw));
    pdl_wait();
    pdl_trigger();
    float kap[B];
    c.load_kappa(kap);
    c.f1(a.spec[0], 0);
    __syncthreads();
    float2 v[B];
    if (c.vcol) c.f2(0, v);
    __syncthreads();
    if (c.vcol) {
#pragma unroll 1
        for (int o = 0; o < 3; o++) {
            float2 w[B];
#pragma unroll
            for (int k2 = 0; k2 < B; k2++) w[k2] = cmul(v[k2], c.mult(o, c.r + A * k2, kap[k2]));
            c.i1(w, o);
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int o = 0; o < 3; o++) c.i2(a.spec[o], o);
}

// One field per CTA (blockIdx.z): the three components are independent, and splitting them
// triples the CTAs in flight while cutting each thread's live registers.
template <int NZ>
__global__ void __launch_bounds__(ZS<NZ>::NT) zpass_each3_kernel(ZArgs a) {
    using S = ZS<NZ>;
    constexpr int A = S::A, B = S::B;
    extern __shared__ float4 smem_raw[];
    ZCtx<NZ> c(a, reinterpret_cast<float2*>(smem_raw));
    pdl_wait();
    pdl_trigger();
    const int o = blockIdx.z;
    float kap[B];
    c.load_kappa(kap);
    c.f1(a.spec[o], 0);
    __syncthreads();
    float2 v[B];
    if (c.vcol) c.f2(0, v);
    __syncthreads();
    if (c.vcol) {
#pragma unroll
        for (int k2 = 0; k2 < B; k2++) v[k2] = cmul(v[k2], c.mult(o, c.r + A * k2, kap[k2]));
        c.i1(v, 0);
    }
    __syncthreads();
    c.i2(a.spec[o], 0);
}

template <int NZ>
__global__ void __launch_bounds__(ZS<NZ>::NT) zpass_sum3_kernel(ZArgs a) {
    using S = ZS<NZ>;
    constexpr int A = S::A, B = S::B;
    extern __shared__ float4 smem_raw[];
    ZCtx<NZ> c(a, reinterpret_cast<float2*>(smem_raw));
    pdl_wait();
    pdl_trigger();
    float kap[B];
    c.load_kappa(kap);
    c.f1_three();
    __syncthreads();
    float2 acc[B];
#pragma unroll
    for (int k2 = 0; k2 < B; k2++) acc[k2] = make_float2(0.f, 0.f);
    if (c.vcol) {
#pragma unroll 1
        for (int o = 0; o < 3; o++) {
            float2 v[B];
            c.f2(o, v);
#pragma unroll
            for (int k2 = 0; k2 < B; k2++) acc[k2] = cadd(acc[k2], cmul(v[k2], c.mult(o, c.r + A * k2, kap[k2])));
        }
    }
    __syncthreads();
    if (c.vcol) c.i1(acc, 0);
    __syncthreads();
    c.i2(a.spec[0], 0);
}

template <int NZ>
static ZKernels make_z() {
    ZKernels k;
    k.grad3 = zpass_grad3_kernel<NZ>;
    k.each3 = zpass_each3_kernel<NZ>;
    k.sum3 = zpass_sum3_kernel<NZ>;
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

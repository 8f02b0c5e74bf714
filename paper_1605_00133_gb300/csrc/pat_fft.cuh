// pat_fft.cuh - register/shared-memory FFT building blocks for the k-space time stepping.
//
// A length-L line transform is done in two radix passes, L = R1 * R2:
//   pass 1: thread t < R2 takes x[t + R2 m] (m < R1), an R1-point DFT in registers, then the
//           twiddle W_L^{t k1}; results go to an exchange buffer laid out [k1][t];
//   pass 2: thread k1 < R1 takes the R2 values of row k1, an R2-point DFT, and holds
//           X[k1 + R1 k2] (k2 < R2).
// X[k1 + R1 k2] = sum_t W_R2^{t k2} W_L^{t k1} sum_m W_R1^{m k1} x[t + R2 m] is the plain DFT
// split by the index maps n = t + R2 m, k = k1 + R1 k2.  The forward transform uses
// (R1, R2) = (A, B) and the inverse (B, A), so the forward's pass-2 register layout is exactly the
// inverse's pass-1 input layout: a multiply in k-space can sit between them without an exchange.
// Sign convention: forward exp(-2 pi i ...), inverse exp(+2 pi i ...), neither normalised.
#pragma once
#include <cuda_runtime.h>

namespace pat {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by i
__device__ __forceinline__ float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }

// cos and sin of 2 pi j / 16, j = 0..7 (mathematical constants)
__device__ __forceinline__ float w16c(int j) {
    constexpr float c[8] = {1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                            0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f};
    return c[j];
}
__device__ __forceinline__ float w16s(int j) {
    constexpr float s[8] = {0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f,
                            1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f};
    return s[j];
}

// In-register R-point DFT, X[k] = sum_m v[m] exp(DIR 2 pi i m k / R), R in {1,2,4,8,16},
// by radix-2 decimation in time (fully unrolled; all indices are compile-time constants).
template <int R, int DIR>
struct Dft {
    __device__ __forceinline__ static void run(float2* v) {
        float2 e[R / 2], o[R / 2];
#pragma unroll
        for (int m = 0; m < R / 2; m++) { e[m] = v[2 * m]; o[m] = v[2 * m + 1]; }
        Dft<R / 2, DIR>::run(e);
        Dft<R / 2, DIR>::run(o);
#pragma unroll
        for (int k = 0; k < R / 2; k++) {
            const int j = k * (16 / R);  // W_R^k = W_16^j
            float2 t;
            if (j == 0) {
                t = o[k];
            } else if (j == 4) {
                t = (DIR > 0) ? cmuli(o[k]) : make_float2(o[k].y, -o[k].x);
            } else {
                t = cmul(o[k], make_float2(w16c(j), DIR * w16s(j)));
            }
            v[k] = cadd(e[k], t);
            v[k + R / 2] = csub(e[k], t);
        }
    }
};
template <int DIR>
struct Dft<2, DIR> {
    __device__ __forceinline__ static void run(float2* v) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};
template <int DIR>
struct Dft<1, DIR> {
    __device__ __forceinline__ static void run(float2*) {}
};

// Radix split per length: L = A * B with A >= B.
template <int L>
struct Split {
    static constexpr int A = (L >= 128) ? 16 : (L >= 32) ? 8 : (L >= 8) ? 4 : 2;
    static constexpr int B = L / A;
};

// twiddle W_L^{DIR * e} from the table tw[m] = exp(-2 pi i m / L)
template <int L, int DIR>
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int e) {
    const float2 w = __ldg(tw + (e & (L - 1)));
    return (DIR < 0) ? w : cconj(w);
}

// Transform nl lines of length L held in shared memory (line l at data[l*lp .. l*lp+L)), in place,
// through the exchange buffer `xch` (nl * R1 * (R2+1) complex).  Threads loop over work items, so
// any block size works.  Ends with __syncthreads().
template <int L, int DIR>
__device__ void fft_lines_smem(float2* data, int lp, int nl, float2* xch,
                               const float2* __restrict__ tw, int tid, int nt) {
    constexpr int R1 = (DIR < 0) ? Split<L>::A : Split<L>::B;
    constexpr int R2 = L / R1;
    constexpr int XP = R2 + 1;        // exchange row pitch
    constexpr int XL = R1 * XP;       // exchange line pitch
    for (int it = tid; it < nl * R2; it += nt) {
        const int l = it / R2, t = it - l * R2;
        float2 v[R1];
        const float2* src = data + l * lp + t;
#pragma unroll
        for (int m = 0; m < R1; m++) v[m] = src[R2 * m];
        Dft<R1, DIR>::run(v);
        float2* dst = xch + l * XL + t;
#pragma unroll
        for (int k1 = 0; k1 < R1; k1++) {
            const float2 w = (k1 == 0 || t == 0) ? v[k1] : cmul(v[k1], twiddle<L, DIR>(tw, t * k1));
            dst[k1 * XP] = w;
        }
    }
    __syncthreads();
    for (int it = tid; it < nl * R1; it += nt) {
        const int l = it / R1, k1 = it - l * R1;
        float2 v[R2];
        const float2* src = xch + l * XL + k1 * XP;
#pragma unroll
        for (int t = 0; t < R2; t++) v[t] = src[t];
        Dft<R2, DIR>::run(v);
        float2* dst = data + l * lp + k1;
#pragma unroll
        for (int k2 = 0; k2 < R2; k2++) dst[R1 * k2] = v[k2];
    }
    __syncthreads();
}

// Runtime-length dispatch (L a power of two in [2, 256]).
template <int DIR>
__device__ __forceinline__ void fft_lines(int L, float2* data, int lp, int nl, float2* xch,
                                          const float2* __restrict__ tw, int tid, int nt) {
    switch (L) {
        case 2: fft_lines_smem<2, DIR>(data, lp, nl, xch, tw, tid, nt); break;
        case 4: fft_lines_smem<4, DIR>(data, lp, nl, xch, tw, tid, nt); break;
        case 8: fft_lines_smem<8, DIR>(data, lp, nl, xch, tw, tid, nt); break;
        case 16: fft_lines_smem<16, DIR>(data, lp, nl, xch, tw, tid, nt); break;
        case 32: fft_lines_smem<32, DIR>(data, lp, nl, xch, tw, tid, nt); break;
        case 64: fft_lines_smem<64, DIR>(data, lp, nl, xch, tw, tid, nt); break;
        case 128: fft_lines_smem<128, DIR>(data, lp, nl, xch, tw, tid, nt); break;
        case 256: fft_lines_smem<256, DIR>(data, lp, nl, xch, tw, tid, nt); break;
        default: break;
    }
}

// Exchange-buffer size (complex elements) fft_lines needs for nl lines of length L, either direction.
__host__ __device__ inline int fft_xch_elems(int L, int nl) {
    int a = (L >= 128) ? 16 : (L >= 32) ? 8 : (L >= 8) ? 4 : 2;
    int b = L / a;
    int f = a * (b + 1), i = b * (a + 1);
    return nl * (f > i ? f : i);
}

}  // namespace pat

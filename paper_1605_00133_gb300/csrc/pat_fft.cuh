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

// Complex addition and subtraction as one packed FP32x2 instruction each (two IEEE single-precision
// operations, round to nearest: the same values as two scalar ones); a - b is fma(b, -1, a), exact.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
// s a + b with s = +-1 in both lanes (thread-pair butterflies: sum or difference by lane)
__device__ __forceinline__ float2 csgn_add(float2 s, float2 a, float2 b) { return __ffma2_rn(s, a, b); }
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
            if (j == 4) {
                // t = DIR i o: lanes cross, so scalar adds
                const float tx = (DIR > 0) ? -o[k].y : o[k].y, ty = (DIR > 0) ? o[k].x : -o[k].x;
                v[k] = make_float2(e[k].x + tx, e[k].y + ty);
                v[k + R / 2] = make_float2(e[k].x - tx, e[k].y - ty);
            } else {
                const float2 t = (j == 0) ? o[k] : cmul(o[k], make_float2(w16c(j), DIR * w16s(j)));
                v[k] = cadd(e[k], t);
                v[k + R / 2] = csub(e[k], t);
            }
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

// Plane-kernel variant: NF fields of NL lines each, line l of field f at base + f * AREA + l * P
// in both the data and the exchange area (exchange area != data area).  The exchange keeps a line's
// [k1][t] matrix unpadded (row pitch R2, so a line needs exactly L elements) and swizzles the
// column, t -> t ^ s(k1) with s(k1) = (k1 / (16 / R2)) mod R2: with a line pitch P = 8 (mod 16),
// the 16 threads of a half-warp then hit 16 distinct 8-byte bank pairs in both passes.  NT threads.
template <int R2>
__device__ __forceinline__ int xswz(int k1, int t) {
    constexpr int G = (R2 >= 16) ? 1 : 16 / R2;
    return k1 * R2 + (t ^ ((k1 / G) & (R2 - 1)));
}

template <int L, int DIR, int NL, int NF, int P, int AREA, int NT>
__device__ __forceinline__ void fft_lines_ct(float2* data, float2* xch, const float2* __restrict__ tw) {
    constexpr int R1 = (DIR < 0) ? Split<L>::A : Split<L>::B;
    constexpr int R2 = L / R1;
    static_assert(L <= P, "line pitch too small");
    const int tid = threadIdx.x;
#pragma unroll 1
    for (int it = tid; it < NF * NL * R2; it += NT) {
        const int t = it % R2, lf = it / R2;
        const int off = (lf / NL) * AREA + (lf % NL) * P;
        float2 v[R1];
        const float2* src = data + off + t;
#pragma unroll
        for (int m = 0; m < R1; m++) v[m] = src[R2 * m];
        Dft<R1, DIR>::run(v);
        float2* dst = xch + off;
#pragma unroll
        for (int k1 = 0; k1 < R1; k1++) {
            const float2 w = (k1 == 0) ? v[k1] : cmul(v[k1], twiddle<L, DIR>(tw, t * k1));
            dst[xswz<R2>(k1, t)] = w;
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int it = tid; it < NF * NL * R1; it += NT) {
        const int k1 = it % R1, lf = it / R1;
        const int off = (lf / NL) * AREA + (lf % NL) * P;
        float2 v[R2];
        const float2* src = xch + off;
#pragma unroll
        for (int t = 0; t < R2; t++) v[t] = src[xswz<R2>(k1, t)];
        Dft<R2, DIR>::run(v);
        float2* dst = data + off + k1;
#pragma unroll
        for (int k2 = 0; k2 < R2; k2++) dst[R1 * k2] = v[k2];
    }
    __syncthreads();
}

// Inverse x-transform whose input lines arrive as half rows: line l holds, as float4 at element 2k,
// (W_a[k], W_b[k]) for k < L/2, the x-spectra of the two real rows of a row pair.  Pass 1 rebuilds
// Z[n] = W_a[n] + i W_b[n] with the Hermitian mirror Z[L-n] = conj(W_a[n]) + i conj(W_b[n]), and
// the packed k = 0 entry (real DC in .x, real Nyquist in .y) as Z[0] and Z[L/2], on the fly.
// The data area is overwritten with Z's transform in natural order.
template <int L, int NL, int NF, int P, int AREA, int NT>
__device__ __forceinline__ void ifft_halfrows_ct(float2* data, float2* xch, const float2* __restrict__ tw) {
    constexpr int DIR = +1;
    constexpr int R1 = Split<L>::B;
    constexpr int R2 = L / R1;
    static_assert(L <= P, "line pitch too small");
    const int tid = threadIdx.x;
#pragma unroll 1
    for (int it = tid; it < NF * NL * R2; it += NT) {
        const int t = it % R2, lf = it / R2;
        const int off = (lf / NL) * AREA + (lf % NL) * P;
        const float4* half = reinterpret_cast<const float4*>(data + off);
        float2 v[R1];
#pragma unroll
        for (int m = 0; m < R1; m++) {
            const int n = t + R2 * m;
            if (n == 0 || n == L / 2) {
                const float4 w = half[0];
                v[m] = (n == 0) ? make_float2(w.x, w.z) : make_float2(w.y, w.w);
            } else if (n < L / 2) {
                const float4 w = half[n];
                v[m] = make_float2(w.x - w.w, w.y + w.z);
            } else {
                const float4 w = half[L - n];
                v[m] = make_float2(w.x + w.w, w.z - w.y);
            }
        }
        Dft<R1, DIR>::run(v);
        float2* dst = xch + off;
#pragma unroll
        for (int k1 = 0; k1 < R1; k1++) {
            const float2 w = (k1 == 0) ? v[k1] : cmul(v[k1], twiddle<L, DIR>(tw, t * k1));
            dst[xswz<R2>(k1, t)] = w;
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int it = tid; it < NF * NL * R1; it += NT) {
        const int k1 = it % R1, lf = it / R1;
        const int off = (lf / NL) * AREA + (lf % NL) * P;
        float2 v[R2];
        const float2* src = xch + off;
#pragma unroll
        for (int t = 0; t < R2; t++) v[t] = src[xswz<R2>(k1, t)];
        Dft<R2, DIR>::run(v);
        float2* dst = data + off + k1;
#pragma unroll
        for (int k2 = 0; k2 < R2; k2++) dst[R1 * k2] = v[k2];
    }
    __syncthreads();
}

// Programmatic dependent launch.  Kernels of the time loop are launched with programmatic stream
// serialisation, so a kernel's CTAs can become resident while its predecessor is still running.
// pdl_wait() blocks until the predecessor grid has completed and its writes are visible; every
// such kernel calls it before its first global-memory access.  pdl_trigger() lets the successor be
// scheduled as soon as every CTA of this grid has issued it (the successor still waits for this
// grid's completion before touching its outputs).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Cluster barriers.  cluster_sync_release orders this CTA's earlier memory operations (the
// distributed-shared-memory writes of a transpose) before every CTA's later ones; cluster_sync_relaxed
// is a pure execution barrier, used where a CTA only needs to know that the others have finished
// reading a buffer, so it does not wait for earlier global stores to drain.
__device__ __forceinline__ void cluster_sync_release() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_sync_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}

// Read-only load that does not allocate in L1: for data read once per pass (kappa), so that it does
// not evict the small per-axis tables that every phase of a line pass reads again.
__device__ __forceinline__ float ldg_stream(const float* p) {
    float v;
    asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// Bulk asynchronous copies (the TMA unit's non-tensor form): one thread copies a contiguous block of
// global memory into this CTA's shared memory; the copy completes on an mbarrier, whose phase
// completion makes the data visible to every thread that waits on it.  Addresses 16-byte aligned,
// size a multiple of 16.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// make initialised mbarriers visible to the asynchronous proxy (before the first copy uses them)
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// the single arrival of a phase, announcing `bytes` of copies that complete it
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}
// Wait for phase `parity` of an mbarrier to complete: each poll suspends the thread for at most about
// a microsecond, and after `polls` polls (about a second for 1 << 20) the wait gives up and returns
// false; the caller records the failure and does not use what the copy should have delivered, so no
// thread is left waiting.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int polls) {
    for (int i = 0; i < polls; i++) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(smem_addr(bar)), "r"(parity), "r"(1000u) : "memory");
        if (done) return true;
    }
    return false;
}

// Asynchronous global -> shared copies (cp.async): the data land in shared memory without passing
// through registers; a thread may read what it copied itself after cp_async_wait<N>() (at most N of
// its committed groups still pending), other threads only after a barrier on top of that.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

}  // namespace pat

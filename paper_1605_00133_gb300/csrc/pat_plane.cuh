// pat_plane.cuh - (y,x) plane transforms, templated on the plane size.
//
// One thread-block cluster of CS CTAs owns one plane of one batch entry.  CTA r holds
//   ROW: complex row pairs j in [r*RC, (r+1)*RC), Z_j[x] = r[2j][x] + i r[2j+1][x] (x-FFT lines),
//   COL: packed half-spectrum columns kx' in [r*CC, (r+1)*CC) over all ky (y-FFT lines).
// The x-DC and x-Nyquist columns, both real after the x-FFT, share the packed column kx' = 0 as
// D + i Nq.  Half spectra are stored [kx][ky] (ky fastest), so a CTA's columns are one contiguous
// run of CC * NY complex values per plane.  The transpose between the row and column layouts goes
// through distributed shared memory (map_shared_rank) between two cluster barriers.  While one slab
// is being transformed the other one is idle, so it doubles as the transform's exchange buffer.
//
// The time loop itself needs no plane transforms (pat_line.cuh); these kernels move whole stacks of
// planes between real space and the (kx, ky) half spectrum outside it:
//   plane_rfft   real planes -> half spectra (the image p0; the adjoint's injected data planes)
//   plane_irfft  half spectra -> real planes (the recorded detection-plane series; the adjoint image)
#pragma once
#include <cooperative_groups.h>

#include "pat_fft.cuh"
#include "pat_kargs.h"

namespace pat {

namespace cg = cooperative_groups;

constexpr int cmin(int a, int b) { return a < b ? a : b; }
constexpr int cmax(int a, int b) { return a > b ? a : b; }

template <int NX, int NY>
struct PS {
    static constexpr int CS = cmin(8, cmin(NX / 2, NY / 2));  // CTAs per plane (cluster size)
    static constexpr int RC = NY / 2 / CS;                       // row pairs per CTA
    static constexpr int CC = NX / 2 / CS;                       // packed columns per CTA
    static constexpr int NXH = NX / 2 + 1;
    // line pitch: >= the longest line, and = 8 (mod 16) so that a half-warp spanning two lines
    // touches 16 distinct 8-byte bank pairs
    static constexpr int P = ((cmax(NX, NY) + 7) / 16) * 16 + 8;
    static constexpr int AREA = cmax(RC, CC) * P;                // one field's slab
    static constexpr int NT = kPlaneThreads;
    static constexpr size_t smem(int nf) { return (size_t)2 * nf * AREA * sizeof(float2); }
};

// Inverse (y,x) transform of NF half-spectrum planes (field f at sp + f*fs, [ky][kx]) into ROW.
// The three spectrum buffers are one allocation, so fields are addressed by a stride.
template <int NX, int NY, int NF>
__device__ __forceinline__ void inv_planes(const PlaneArgs& a, float2* ROW, float2* COL,
                                           const float2* sp, size_t fs, int rank,
                                           cg::cluster_group& cl) {
    using S = PS<NX, NY>;
    constexpr int CC = S::CC, RC = S::RC, P = S::P, AREA = S::AREA, NT = S::NT;
    const int tid = threadIdx.x;
    // every load is issued before any is consumed (one L2 round trip, not one per element)
    constexpr int NLD = (NF * NY * CC + NT - 1) / NT;
    float2 v[NLD];
#pragma unroll
    for (int u = 0; u < NLD; u++) {
        const int it = tid + u * NT;
        v[u] = make_float2(0.f, 0.f);
        if (NLD * NT == NF * NY * CC || it < NF * NY * CC) {
            const int ky = it % NY, c = (it / NY) % CC, f = it / (CC * NY);
            const int kx = rank * CC + c;
            const float2* s = sp + f * fs;
            v[u] = s[kx * NY + ky];
            if (kx == 0) {
                const float2 q = s[(NX / 2) * NY + ky];
                v[u] = make_float2(v[u].x - q.y, v[u].y + q.x);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < NLD; u++) {
        const int it = tid + u * NT;
        if (NLD * NT == NF * NY * CC || it < NF * NY * CC) {
            const int ky = it % NY, c = (it / NY) % CC, f = it / (CC * NY);
            COL[f * AREA + c * P + ky] = v[u];
        }
    }
    __syncthreads();
    fft_lines_ct<NY, +1, CC, NF, P, AREA, NT>(COL, ROW, a.tw_y);
    cluster_sync_relaxed();  // every CTA has finished using its ROW as exchange space
    constexpr int NYH = NY / 2;
#pragma unroll 1
    for (int it = tid; it < NF * CC * NYH; it += NT) {
        const int j = it % NYH, c = (it / NYH) % CC, f = it / (CC * NYH);
        const int kx = rank * CC + c;
        const float4 w = *reinterpret_cast<const float4*>(COL + f * AREA + c * P + 2 * j);  // rows 2j, 2j+1
        const int dst = j / RC, jl = j % RC;
        float4* rr = reinterpret_cast<float4*>(cl.map_shared_rank(ROW, dst) + f * AREA + jl * P);
        rr[kx] = w;  // half row: (W_a[kx], W_b[kx]); column 0 carries (DC, Nyquist) of both rows
    }
    cluster_sync_release();
    ifft_halfrows_ct<NX, RC, NF, P, AREA, NT>(ROW, COL, a.tw_x);
}

// Forward (y,x) transform of NF ROW slabs into half-spectrum planes at sp + f*fs.
template <int NX, int NY, int NF>
__device__ __forceinline__ void fwd_planes(const PlaneArgs& a, float2* ROW, float2* COL,
                                           float2* sp, size_t fs, int rank, cg::cluster_group& cl) {
    using S = PS<NX, NY>;
    constexpr int CC = S::CC, RC = S::RC, P = S::P, AREA = S::AREA, NT = S::NT;
    const int tid = threadIdx.x;
    fft_lines_ct<NX, -1, RC, NF, P, AREA, NT>(ROW, COL, a.tw_x);
    cluster_sync_relaxed();  // every CTA has finished using its COL as exchange space
    constexpr int NXQ = NX / 2;
#pragma unroll 1
    for (int it = tid; it < NF * RC * NXQ; it += NT) {
        const int k = it % NXQ, jl = (it / NXQ) % RC, f = it / (RC * NXQ);
        const int jg = rank * RC + jl;
        const float2* row = ROW + f * AREA + jl * P;
        const float2 zk = row[k];
        const int dst = k / CC, c = k % CC;
        float4* cr = reinterpret_cast<float4*>(cl.map_shared_rank(COL, dst) + f * AREA + c * P + 2 * jg);
        if (k == 0) {
            const float2 zn = row[NXQ];
            *cr = make_float4(zk.x, zn.x, zk.y, zn.y);
        } else {
            const float2 zm = cconj(row[NX - k]);
            const float2 sm = cadd(zk, zm), d = csub(zk, zm);
            *cr = make_float4(0.5f * sm.x, 0.5f * sm.y, 0.5f * d.y, -0.5f * d.x);
        }
    }
    cluster_sync_release();
    fft_lines_ct<NY, -1, CC, NF, P, AREA, NT>(COL, ROW, a.tw_y);
#pragma unroll 1
    for (int it = tid; it < NF * NY * CC; it += NT) {
        const int ky = it % NY, c = (it / NY) % CC, f = it / (CC * NY);
        const int kx = rank * CC + c;
        const float2* col = COL + f * AREA + c * P;
        const float2 v = col[ky];
        float2* s = sp + f * fs;
        if (kx == 0) {
            const float2 vm = cconj(col[(NY - ky) & (NY - 1)]);
            const float2 d = csub(v, vm);
            s[ky] = cscale(cadd(v, vm), 0.5f);
            s[(NX / 2) * NY + ky] = make_float2(0.5f * d.y, -0.5f * d.x);
        } else {
            s[kx * NY + ky] = v;
        }
    }
    __syncthreads();
}

// Row loops visit (row pair jl, x pair xp): rows y0 = 2 (rank RC + jl), y0 + 1 and columns
// x0 = 2 xp, x0 + 1; ROW[jl][x] = (value at row y0, value at row y0 + 1).
#define PAT_ROWS_BEGIN(S, rank)                                                     \
    _Pragma("unroll")                                                               \
    for (int it = threadIdx.x; it < S::RC * (NX / 2); it += S::NT) {                \
        const int xp = it % (NX / 2), jl = it / (NX / 2);                           \
        const int x0 = 2 * xp, y0 = 2 * ((rank) * S::RC + jl);                       \
        const size_t o0 = (size_t)y0 * NX + x0, o1 = o0 + NX;                        \
        const int rbase = jl * S::P + x0;
#define PAT_ROWS_END }

template <int NX, int NY>
__global__ void __launch_bounds__(kPlaneThreads, 2) plane_rfft_kernel(PlaneArgs a) {
    using S = PS<NX, NY>;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ float4 smem_raw[];
    float2* ROW = reinterpret_cast<float2*>(smem_raw);
    float2* COL = ROW + S::AREA;
    const int rank = (int)cl.block_rank(), p = blockIdx.y, b = blockIdx.z;
    const float* in = a.in_real + (size_t)b * a.bs_real + (size_t)p * (NY * NX);
    float2* sp = a.spec_out + (size_t)b * a.bs_spec + (size_t)p * (S::NXH * NY);
    pdl_wait();
    pdl_trigger();
    PAT_ROWS_BEGIN(S, rank)
    const float2 pa = *reinterpret_cast<const float2*>(in + o0);  // row y0, x0..x0+1
    const float2 pb = *reinterpret_cast<const float2*>(in + o1);  // row y0+1
    *reinterpret_cast<float4*>(ROW + rbase) = make_float4(pa.x, pb.x, pa.y, pb.y);
    PAT_ROWS_END
    __syncthreads();
    fwd_planes<NX, NY, 1>(a, ROW, COL, sp, 0, rank, cl);
}

template <int NX, int NY>
__global__ void __launch_bounds__(kPlaneThreads, 2) plane_irfft_kernel(PlaneArgs a) {
    using S = PS<NX, NY>;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ float4 smem_raw[];
    float2* ROW = reinterpret_cast<float2*>(smem_raw);
    float2* COL = ROW + S::AREA;
    const int rank = (int)cl.block_rank(), p = blockIdx.y, b = blockIdx.z;
    const float2* sp = a.spec_in + (size_t)b * a.bs_spec + (size_t)p * (S::NXH * NY);
    float* out = a.out_real + (size_t)b * a.bs_real + (size_t)p * (NY * NX);
    pdl_wait();
    pdl_trigger();
    inv_planes<NX, NY, 1>(a, ROW, COL, sp, 0, rank, cl);
    const float s = a.scale;
    PAT_ROWS_BEGIN(S, rank)
    const float4 zz = *reinterpret_cast<const float4*>(ROW + rbase);  // (y0, y0+1) at x0, at x0+1
    *reinterpret_cast<float2*>(out + o0) = make_float2(s * zz.x, s * zz.z);
    *reinterpret_cast<float2*>(out + o1) = make_float2(s * zz.y, s * zz.w);
    PAT_ROWS_END
}

#undef PAT_ROWS_BEGIN
#undef PAT_ROWS_END

template <int NX, int NY>
PlaneKernels make_plane_kernels() {
    using S = PS<NX, NY>;
    PlaneKernels k;
    k.rfft = plane_rfft_kernel<NX, NY>;
    k.irfft = plane_irfft_kernel<NX, NY>;
    k.smem = S::smem(1);
    k.cs = S::CS;
    return k;
}

template <int NX>
PlaneKernels plane_kernels_ny(int ny) {
    switch (ny) {
        case 8: return make_plane_kernels<NX, 8>();
        case 16: return make_plane_kernels<NX, 16>();
        case 32: return make_plane_kernels<NX, 32>();
        case 64: return make_plane_kernels<NX, 64>();
        case 128: return make_plane_kernels<NX, 128>();
        case 256: return make_plane_kernels<NX, 256>();
        default: return PlaneKernels{};
    }
}

}  // namespace pat

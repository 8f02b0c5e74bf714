// pat_plane.cuh - (y,x) plane kernels of the k-space time step, templated on the plane size.
//
// One thread-block cluster of CS CTAs owns one z-plane of one batch entry.  CTA r holds
//   ROW: complex row pairs j in [r*RC, (r+1)*RC), Z_j[x] = r[2j][x] + i r[2j+1][x] (x-FFT lines),
//   COL: packed half-spectrum columns kx' in [r*CC, (r+1)*CC) over all ky (y-FFT lines),
// for up to three fields at once.  The x-DC and x-Nyquist columns, both real after the x-FFT, share
// the packed column kx' = 0 as D + i Nq.  Half spectra are stored [z][kx][ky] (ky fastest), so a
// CTA's columns are one contiguous run of CC * NY complex values per plane.  The transpose between the row and column layouts goes
// through distributed shared memory (map_shared_rank) between two cluster barriers.  While one slab
// is being transformed the other one is idle, so it doubles as the transform's exchange buffer.
//
// Kernels (one z-plane, all fields of one time-step half):
//   plane_init     p0 -> rho_i = p0/(3c^2), record plane 0, forward (y,x) FFT of p0
//   plane_vel      inverse FFTs of 3 gradient components -> new = A1 old + A2 g, out = A3 new
//                  (forward velocity, adjoint velocity) -> forward FFTs of the 3 outputs
//   plane_rho_fwd  inverse FFTs of 3 divergence components -> rho_i = a^2 rho_i - a dt rho0 d_i,
//                  p = c^2 sum rho_i, record -> forward FFT of p
//   plane_rho_adj  inverse FFT of the summed adjoint divergence -> lambda = s0 l + injected data,
//                  q_i = a^2 q_i + c^2 lambda -> forward FFTs of a_i q_i (or, on the last step,
//                  the image p = lambda + sum a_i^2 q_i / (3 c^2))
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
    // CTAs per SM the three-field kernels can hold (228 KB of shared memory per SM, 1 KB reserved
    // per CTA); the register budget follows it, so small planes keep 64 registers per thread and
    // large planes (one CTA per SM) get the full register file instead of spilling
    static constexpr int MINB = (int)(228 * 1024 / (smem(3) + 1024)) >= 4 ? 4
                              : (int)(228 * 1024 / (smem(3) + 1024)) >= 2 ? 2 : 1;
};

__device__ __forceinline__ int axis_pos(int i, int z, int y, int x) { return i == 0 ? z : (i == 1 ? y : x); }

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

struct PlaneIdx {
    int rank, z, b;
    size_t plane_off, spec_off, rec_off, fs;
    bool on_sensor;
};

template <int NX, int NY>
__device__ __forceinline__ PlaneIdx plane_idx(const PlaneArgs& a, cg::cluster_group& cl) {
    const Geom& g = a.g;
    PlaneIdx p;
    p.rank = (int)cl.block_rank();
    p.z = blockIdx.y;
    p.b = blockIdx.z;
    p.plane_off = ((size_t)p.b * g.nz + p.z) * (size_t)(NY * NX);
    p.spec_off = (size_t)p.b * g.nspec + (size_t)p.z * (PS<NX, NY>::NXH * NY);
    p.rec_off = ((size_t)p.b * g.T + a.n_rec) * (size_t)(NY * NX);
    p.on_sensor = (p.z == g.sensor_z);
    p.fs = (size_t)g.B * g.nspec;
    return p;
}

// Pointwise loops visit (row pair jl, x pair xp): rows y0 = 2 (rank RC + jl), y0 + 1 and columns
// x0 = 2 xp, x0 + 1; ROW[f][jl][x] = (value at row y0, value at row y0 + 1).
#define PAT_POINTWISE_BEGIN(S, I)                                                   \
    _Pragma("unroll")                                                               \
    for (int it = threadIdx.x; it < S::RC * (NX / 2); it += S::NT) {                \
        const int xp = it % (NX / 2), jl = it / (NX / 2);                           \
        const int x0 = 2 * xp, y0 = 2 * (I.rank * S::RC + jl);                       \
        const size_t g0 = I.plane_off + (size_t)y0 * NX + x0, g1 = g0 + NX;          \
        const int rbase = jl * S::P + x0;
#define PAT_POINTWISE_END }

template <int NX, int NY>
__global__ void __launch_bounds__(kPlaneThreads, (PS<NX, NY>::MINB)) plane_init_kernel(PlaneArgs a) {
    using S = PS<NX, NY>;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ float4 smem_raw[];
    float2* ROW = reinterpret_cast<float2*>(smem_raw);
    float2* COL = ROW + S::AREA;
    const PlaneIdx I = plane_idx<NX, NY>(a, cl);
    pdl_wait();
    pdl_trigger();
    PAT_POINTWISE_BEGIN(S, I)
    const float2 pa = *reinterpret_cast<const float2*>(a.in_real + g0);  // row y0, x0..x0+1
    const float2 pb = *reinterpret_cast<const float2*>(a.in_real + g1);  // row y0+1
#pragma unroll
    for (int i = 0; i < 3; i++) {
        *reinterpret_cast<float2*>(a.st[i] + g0) = make_float2(pa.x * a.s1, pa.y * a.s1);
        *reinterpret_cast<float2*>(a.st[i] + g1) = make_float2(pb.x * a.s1, pb.y * a.s1);
    }
    if (I.on_sensor) {
        *reinterpret_cast<float2*>(a.rec + I.rec_off + (size_t)y0 * NX + x0) = pa;
        *reinterpret_cast<float2*>(a.rec + I.rec_off + (size_t)(y0 + 1) * NX + x0) = pb;
    }
    *reinterpret_cast<float4*>(ROW + rbase) = make_float4(pa.x, pb.x, pa.y, pb.y);
    PAT_POINTWISE_END
    __syncthreads();
    if (!(a.flags & PF_NO_FWD)) {
        fwd_planes<NX, NY, 1>(a, ROW, COL, a.spec[0] + I.spec_off, I.fs, I.rank, cl);
    }
}

template <int NX, int NY>
__global__ void __launch_bounds__(kPlaneThreads, (PS<NX, NY>::MINB)) plane_vel_kernel(PlaneArgs a) {
    using S = PS<NX, NY>;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ float4 smem_raw[];
    float2* ROW = reinterpret_cast<float2*>(smem_raw);
    float2* COL = ROW + 3 * S::AREA;
    const PlaneIdx I = plane_idx<NX, NY>(a, cl);
    pdl_wait();
    pdl_trigger();
    {
        inv_planes<NX, NY, 3>(a, ROW, COL, a.spec[0] + I.spec_off, I.fs, I.rank, cl);
    }
    const bool no_old = (a.flags & PF_NO_OLD) != 0;
    PAT_POINTWISE_BEGIN(S, I)
#pragma unroll
    for (int i = 0; i < 3; i++) {
        float2* rw = ROW + i * S::AREA + rbase;
        const float4 zz = *reinterpret_cast<const float4*>(rw);  // (y0, y0+1) at x0 and at x0+1
        const float2 z0 = make_float2(zz.x, zz.y), z1 = make_float2(zz.z, zz.w);
        const int qa = axis_pos(i, I.z, y0, x0), qb = axis_pos(i, I.z, y0, x0 + 1);
        const int qc = axis_pos(i, I.z, y0 + 1, x0), qd = axis_pos(i, I.z, y0 + 1, x0 + 1);
        const float* A1 = a.A1[i];
        const float* A2 = a.A2[i];
        const float* A3 = a.A3[i];
        float2 na = make_float2(__ldg(A2 + qa) * z0.x, __ldg(A2 + qb) * z1.x);  // row y0
        float2 nb = make_float2(__ldg(A2 + qc) * z0.y, __ldg(A2 + qd) * z1.y);  // row y0+1
        if (!no_old) {
            const float2 oa = *reinterpret_cast<const float2*>(a.st[i] + g0);
            const float2 ob = *reinterpret_cast<const float2*>(a.st[i] + g1);
            na.x = fmaf(__ldg(A1 + qa), oa.x, na.x);
            na.y = fmaf(__ldg(A1 + qb), oa.y, na.y);
            nb.x = fmaf(__ldg(A1 + qc), ob.x, nb.x);
            nb.y = fmaf(__ldg(A1 + qd), ob.y, nb.y);
        }
        *reinterpret_cast<float2*>(a.st[i] + g0) = na;
        *reinterpret_cast<float2*>(a.st[i] + g1) = nb;
        *reinterpret_cast<float4*>(rw) = make_float4(__ldg(A3 + qa) * na.x, __ldg(A3 + qc) * nb.x,
                                                     __ldg(A3 + qb) * na.y, __ldg(A3 + qd) * nb.y);
    }
    PAT_POINTWISE_END
    __syncthreads();
    fwd_planes<NX, NY, 3>(a, ROW, COL, a.spec[0] + I.spec_off, I.fs, I.rank, cl);
}

template <int NX, int NY>
__global__ void __launch_bounds__(kPlaneThreads, (PS<NX, NY>::MINB)) plane_rho_fwd_kernel(PlaneArgs a) {
    using S = PS<NX, NY>;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ float4 smem_raw[];
    float2* ROW = reinterpret_cast<float2*>(smem_raw);
    float2* COL = ROW + 3 * S::AREA;
    const PlaneIdx I = plane_idx<NX, NY>(a, cl);
    pdl_wait();
    pdl_trigger();
    {
        inv_planes<NX, NY, 3>(a, ROW, COL, a.spec[0] + I.spec_off, I.fs, I.rank, cl);
    }
    PAT_POINTWISE_BEGIN(S, I)
    float2 pa = make_float2(0.f, 0.f), pb = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const float2* rw = ROW + i * S::AREA + rbase;
        const float4 zz = *reinterpret_cast<const float4*>(rw);
        const float2 z0 = make_float2(zz.x, zz.y), z1 = make_float2(zz.z, zz.w);
        const int qa = axis_pos(i, I.z, y0, x0), qb = axis_pos(i, I.z, y0, x0 + 1);
        const int qc = axis_pos(i, I.z, y0 + 1, x0), qd = axis_pos(i, I.z, y0 + 1, x0 + 1);
        const float* A1 = a.A1[i];
        const float* A2 = a.A2[i];
        const float2 oa = *reinterpret_cast<const float2*>(a.st[i] + g0);
        const float2 ob = *reinterpret_cast<const float2*>(a.st[i] + g1);
        const float2 ra = make_float2(fmaf(__ldg(A1 + qa), oa.x, __ldg(A2 + qa) * z0.x),
                                      fmaf(__ldg(A1 + qb), oa.y, __ldg(A2 + qb) * z1.x));
        const float2 rb = make_float2(fmaf(__ldg(A1 + qc), ob.x, __ldg(A2 + qc) * z0.y),
                                      fmaf(__ldg(A1 + qd), ob.y, __ldg(A2 + qd) * z1.y));
        *reinterpret_cast<float2*>(a.st[i] + g0) = ra;
        *reinterpret_cast<float2*>(a.st[i] + g1) = rb;
        pa.x += ra.x;
        pa.y += ra.y;
        pb.x += rb.x;
        pb.y += rb.y;
    }
    pa = cscale(pa, a.c2);
    pb = cscale(pb, a.c2);
    if (I.on_sensor) {
        *reinterpret_cast<float2*>(a.rec + I.rec_off + (size_t)y0 * NX + x0) = pa;
        *reinterpret_cast<float2*>(a.rec + I.rec_off + (size_t)(y0 + 1) * NX + x0) = pb;
    }
    *reinterpret_cast<float4*>(ROW + rbase) = make_float4(pa.x, pb.x, pa.y, pb.y);
    PAT_POINTWISE_END
    __syncthreads();
    if (!(a.flags & PF_NO_FWD)) {
        fwd_planes<NX, NY, 1>(a, ROW, COL, a.spec[0] + I.spec_off, I.fs, I.rank, cl);
    }
}

template <int NX, int NY>
__global__ void __launch_bounds__(kPlaneThreads, (PS<NX, NY>::MINB)) plane_rho_adj_kernel(PlaneArgs a) {
    using S = PS<NX, NY>;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ float4 smem_raw[];
    float2* ROW = reinterpret_cast<float2*>(smem_raw);
    float2* COL = ROW + 3 * S::AREA;
    const PlaneIdx I = plane_idx<NX, NY>(a, cl);
    pdl_wait();
    pdl_trigger();
    const bool have_lambda = (a.flags & PF_HAVE_LAMBDA) != 0;
    if (have_lambda) {
        inv_planes<NX, NY, 1>(a, ROW, COL, a.spec[0] + I.spec_off, I.fs, I.rank, cl);
    }
    const bool final_step = (a.flags & PF_FINAL) != 0;
    const bool no_old = (a.flags & PF_NO_OLD) != 0;
    PAT_POINTWISE_BEGIN(S, I)
    float2 la = make_float2(0.f, 0.f), lb = make_float2(0.f, 0.f);  // rows y0, y0+1 at x0, x0+1
    if (have_lambda) {
        const float4 zz = *reinterpret_cast<const float4*>(ROW + rbase);
        const float2 z0 = make_float2(zz.x, zz.y), z1 = make_float2(zz.z, zz.w);
        la = make_float2(a.s0 * z0.x, a.s0 * z1.x);
        lb = make_float2(a.s0 * z0.y, a.s0 * z1.y);
    }
    if (I.on_sensor) {
        const float2 ia = *reinterpret_cast<const float2*>(a.inj + I.rec_off + (size_t)y0 * NX + x0);
        const float2 ib = *reinterpret_cast<const float2*>(a.inj + I.rec_off + (size_t)(y0 + 1) * NX + x0);
        la.x += ia.x;
        la.y += ia.y;
        lb.x += ib.x;
        lb.y += ib.y;
    }
    if (final_step) {
        float2 oa = make_float2(0.f, 0.f), ob = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const int qa = axis_pos(i, I.z, y0, x0), qb = axis_pos(i, I.z, y0, x0 + 1);
            const int qc = axis_pos(i, I.z, y0 + 1, x0), qd = axis_pos(i, I.z, y0 + 1, x0 + 1);
            const float2 sa = *reinterpret_cast<const float2*>(a.st[i] + g0);
            const float2 sb = *reinterpret_cast<const float2*>(a.st[i] + g1);
            oa.x = fmaf(__ldg(a.A1[i] + qa), sa.x, oa.x);
            oa.y = fmaf(__ldg(a.A1[i] + qb), sa.y, oa.y);
            ob.x = fmaf(__ldg(a.A1[i] + qc), sb.x, ob.x);
            ob.y = fmaf(__ldg(a.A1[i] + qd), sb.y, ob.y);
        }
        *reinterpret_cast<float2*>(a.out_real + g0) = make_float2(fmaf(a.s1, oa.x, la.x), fmaf(a.s1, oa.y, la.y));
        *reinterpret_cast<float2*>(a.out_real + g1) = make_float2(fmaf(a.s1, ob.x, lb.x), fmaf(a.s1, ob.y, lb.y));
    } else {
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const int qa = axis_pos(i, I.z, y0, x0), qb = axis_pos(i, I.z, y0, x0 + 1);
            const int qc = axis_pos(i, I.z, y0 + 1, x0), qd = axis_pos(i, I.z, y0 + 1, x0 + 1);
            float2 na = cscale(la, a.c2), nb = cscale(lb, a.c2);
            if (!no_old) {
                const float2 sa = *reinterpret_cast<const float2*>(a.st[i] + g0);
                const float2 sb = *reinterpret_cast<const float2*>(a.st[i] + g1);
                na.x = fmaf(__ldg(a.A1[i] + qa), sa.x, na.x);
                na.y = fmaf(__ldg(a.A1[i] + qb), sa.y, na.y);
                nb.x = fmaf(__ldg(a.A1[i] + qc), sb.x, nb.x);
                nb.y = fmaf(__ldg(a.A1[i] + qd), sb.y, nb.y);
            }
            *reinterpret_cast<float2*>(a.st[i] + g0) = na;
            *reinterpret_cast<float2*>(a.st[i] + g1) = nb;
            float2* rw = ROW + i * S::AREA + rbase;
            *reinterpret_cast<float4*>(rw) = make_float4(__ldg(a.A3[i] + qa) * na.x, __ldg(a.A3[i] + qc) * nb.x,
                                                         __ldg(a.A3[i] + qb) * na.y, __ldg(a.A3[i] + qd) * nb.y);
        }
    }
    PAT_POINTWISE_END
    if (final_step) return;
    __syncthreads();
    fwd_planes<NX, NY, 3>(a, ROW, COL, a.spec[0] + I.spec_off, I.fs, I.rank, cl);
}

#undef PAT_POINTWISE_BEGIN
#undef PAT_POINTWISE_END

template <int NX, int NY>
PlaneKernels make_plane_kernels() {
    using S = PS<NX, NY>;
    PlaneKernels k;
    k.init = plane_init_kernel<NX, NY>;
    k.vel = plane_vel_kernel<NX, NY>;
    k.rho_fwd = plane_rho_fwd_kernel<NX, NY>;
    k.rho_adj = plane_rho_adj_kernel<NX, NY>;
    k.smem_init = S::smem(1);
    k.smem3 = S::smem(3);
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

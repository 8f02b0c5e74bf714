// pat_kernels.cu - CUDA kernels of the k-space pseudospectral PAT operators (sm_103a).
//
// One time step of A (Sec. 4.3) needs ten 3D real FFTs: D^+ of p (1 forward, 3 inverse) and D^- of
// the three velocity components (3 forward, 3 inverse).  They are organised as four launches:
//
//   zpass  ONE_TO_THREE   z-FFT of the (y,x)-transformed p, times i k_i kappa e^{+ik_i dx/2} / N for
//                         i = z, y, x, three inverse z-FFTs                           (gradient)
//   plane  VEL            per z-plane: inverse (y,x) FFT of each component, split-field PML velocity
//                         update, forward (y,x) FFT of the new velocity
//   zpass  THREE_TO_THREE z-FFT, times i k_i kappa e^{-ik_i dx/2} / N, inverse z-FFT  (divergence)
//   plane  RHO_FWD        per z-plane: inverse (y,x) FFTs, split density update, p = c^2 sum rho_i,
//                         detection-plane record, forward (y,x) FFT of p
//
// The (y,x) plane transforms run on a thread-block cluster: the plane's complex row pairs are
// split across the CTAs for the x-FFT, the packed half-spectrum columns across the CTAs for the
// y-FFT, and the transpose between the two goes through distributed shared memory.  Real rows are
// transformed two at a time (row 2j + i row 2j+1), and the x-DC and x-Nyquist columns, both real
// after the x-FFT, share one packed complex column through the y-FFT.  Every multiply by the
// k-space operator and every pointwise update is fused into these passes; the only global traffic
// per step is the state (read and written once) and the half spectra between the plane and z passes.
// A^T runs the transposed recurrence with the same kernels in other modes.
#include <cooperative_groups.h>

#include "pat_fft.cuh"
#include "pat_internal.h"

namespace cg = cooperative_groups;

namespace pat {

// ---------------------------------------------------------------------------------------------
// plane kernel
// ---------------------------------------------------------------------------------------------

enum PlaneMode { PM_INIT_FWD = 0, PM_VEL = 1, PM_RHO_FWD = 2, PM_RHO_ADJ = 3 };
enum PlaneFlag { PF_NO_FWD = 1, PF_NO_OLD = 2, PF_HAVE_LAMBDA = 4, PF_FINAL = 8 };

struct PlaneArgs {
    Geom g;
    const float2* tw_x;
    const float2* tw_y;
    float2* spec[3];
    float* st[3];
    const float* A1[3];
    const float* A2[3];
    const float* A3[3];
    float c2, s0, s1;
    const float* in_real;
    float* out_real;
    float* rec;
    const float* inj;
    int n_rec;
    int mode;
    int flags;
};

static constexpr int kPlaneThreads = 256;

struct PlaneSmem {
    float2* row;   // rows_cta lines of nx complex, pitch nx + 1
    float2* col;   // cols_cta lines of ny complex, pitch ny + 1
    float2* xch;   // FFT exchange buffer
    float* acc;    // 2*rows_cta x nx reals
};

__host__ __device__ inline size_t plane_smem_bytes(const Geom& g) {
    const size_t row = (size_t)g.rows_cta * (g.nx + 1);
    const size_t col = (size_t)g.cols_cta * (g.ny + 1);
    const int xa = fft_xch_elems(g.nx, g.rows_cta), xb = fft_xch_elems(g.ny, g.cols_cta);
    const size_t xch = (size_t)(xa > xb ? xa : xb);
    const size_t acc = (size_t)g.rows_cta * g.nx;  // in float2 units (2 rows of floats)
    return (row + col + xch + acc) * sizeof(float2);
}

// Inverse (y,x) transform of one half-spectrum plane sp[ky][kx] (kx < nxh) into the row slab:
// afterwards row[jl][x] = N_xy * (r[2 jg][x] + i r[2 jg + 1][x]) with jg = rank * rows_cta + jl.
__device__ void inverse_plane(const Geom& g, const PlaneArgs& a, const PlaneSmem& s,
                              const float2* __restrict__ sp, int rank, cg::cluster_group& cluster) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nx = g.nx, ny = g.ny, nxh = g.nxh, cc = g.cols_cta, rc = g.rows_cta;
    const int LPX = nx + 1, LPY = ny + 1;
    // load this CTA's packed columns; column 0 packs D + i Nq (x-DC and x-Nyquist spectra)
    for (int it = tid; it < ny * cc; it += nt) {
        const int ky = it / cc, c = it - ky * cc;
        const int kx = rank * cc + c;
        float2 v = sp[(size_t)ky * nxh + kx];
        if (kx == 0) {
            const float2 q = sp[(size_t)ky * nxh + nx / 2];
            v = make_float2(v.x - q.y, v.y + q.x);
        }
        s.col[c * LPY + ky] = v;
    }
    __syncthreads();
    fft_lines<+1>(ny, s.col, LPY, cc, s.xch, a.tw_y, tid, nt);
    cluster.sync();  // every CTA is done reading its row slab
    // rebuild complex row pairs Z_j[k] = W[2j][k] + i W[2j+1][k] with Hermitian extension
    const int nyh = ny / 2;
    for (int it = tid; it < cc * nyh; it += nt) {
        const int j = it / cc, c = it - j * cc;
        const int kx = rank * cc + c;
        const float2 wa = s.col[c * LPY + 2 * j];
        const float2 wb = s.col[c * LPY + 2 * j + 1];
        const int dst = j / rc, jl = j - dst * rc;
        float2* rr = cluster.map_shared_rank(s.row, dst) + jl * LPX;
        if (kx == 0) {
            rr[0] = make_float2(wa.x, wb.x);
            rr[nx / 2] = make_float2(wa.y, wb.y);
        } else {
            rr[kx] = make_float2(wa.x - wb.y, wa.y + wb.x);
            rr[nx - kx] = make_float2(wa.x + wb.y, wb.x - wa.y);
        }
    }
    cluster.sync();
    fft_lines<+1>(nx, s.row, LPX, rc, s.xch, a.tw_x, tid, nt);
}

// Forward (y,x) transform of the row slab (row[jl][x] = r[2jg][x] + i r[2jg+1][x]) into the
// half-spectrum plane sp[ky][kx].
__device__ void forward_plane(const Geom& g, const PlaneArgs& a, const PlaneSmem& s,
                              float2* __restrict__ sp, int rank, cg::cluster_group& cluster) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nx = g.nx, ny = g.ny, nxh = g.nxh, cc = g.cols_cta, rc = g.rows_cta;
    const int LPX = nx + 1, LPY = ny + 1;
    fft_lines<-1>(nx, s.row, LPX, rc, s.xch, a.tw_x, tid, nt);
    cluster.sync();  // every CTA is done with its column slab
    // split Z = FFT(a + i b) into A = FFT(a), B = FFT(b); pack A[0] + i A[nx/2] into column 0
    const int nxq = nx / 2;
    for (int it = tid; it < rc * nxq; it += nt) {
        const int jl = it / nxq, k = it - jl * nxq;
        const int jg = rank * rc + jl;
        const float2 zk = s.row[jl * LPX + k];
        const int dst = k / cc, c = k - dst * cc;
        float2* cr = cluster.map_shared_rank(s.col, dst) + c * LPY;
        if (k == 0) {
            const float2 zn = s.row[jl * LPX + nxq];
            cr[2 * jg] = make_float2(zk.x, zn.x);
            cr[2 * jg + 1] = make_float2(zk.y, zn.y);
        } else {
            const float2 zm = cconj(s.row[jl * LPX + nx - k]);
            const float2 d = csub(zk, zm);
            cr[2 * jg] = cscale(cadd(zk, zm), 0.5f);
            cr[2 * jg + 1] = make_float2(0.5f * d.y, -0.5f * d.x);
        }
    }
    cluster.sync();
    fft_lines<-1>(ny, s.col, LPY, cc, s.xch, a.tw_y, tid, nt);
    // store; unpack column 0 into the x-DC and x-Nyquist columns
    for (int it = tid; it < ny * cc; it += nt) {
        const int ky = it / cc, c = it - ky * cc;
        const int kx = rank * cc + c;
        const float2 v = s.col[c * LPY + ky];
        if (kx == 0) {
            const float2 vm = cconj(s.col[c * LPY + ((ny - ky) & (ny - 1))]);
            const float2 d = csub(v, vm);
            sp[(size_t)ky * nxh] = cscale(cadd(v, vm), 0.5f);
            sp[(size_t)ky * nxh + nx / 2] = make_float2(0.5f * d.y, -0.5f * d.x);
        } else {
            sp[(size_t)ky * nxh + kx] = v;
        }
    }
    __syncthreads();  // the column slab is reloaded by the next transform
}

__device__ __forceinline__ int axis_pos(int i, int z, int y, int x) { return i == 0 ? z : (i == 1 ? y : x); }

__global__ void __launch_bounds__(kPlaneThreads) plane_kernel(PlaneArgs a) {
    cg::cluster_group cluster = cg::this_cluster();
    const Geom& g = a.g;
    extern __shared__ float4 smem_raw[];
    PlaneSmem s;
    s.row = reinterpret_cast<float2*>(smem_raw);
    s.col = s.row + (size_t)g.rows_cta * (g.nx + 1);
    s.xch = s.col + (size_t)g.cols_cta * (g.ny + 1);
    {
        const int xa = fft_xch_elems(g.nx, g.rows_cta), xb = fft_xch_elems(g.ny, g.cols_cta);
        s.acc = reinterpret_cast<float*>(s.xch + (xa > xb ? xa : xb));
    }
    const int rank = (int)cluster.block_rank();
    const int z = blockIdx.y, b = blockIdx.z;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nx = g.nx, ny = g.ny, rc = g.rows_cta;
    const int LPX = nx + 1;
    const size_t plane_off = ((size_t)b * g.nz + z) * (size_t)ny * nx;      // real fields
    const size_t spec_off = (size_t)b * g.nspec + (size_t)z * ny * g.nxh;  // half spectra
    const bool on_sensor = (z == g.sensor_z);
    const size_t rec_off = ((size_t)b * g.T + a.n_rec) * (size_t)g.m_plane;
    const int npts = rc * nx;  // (row pair, x) items

    if (a.mode == PM_INIT_FWD) {
        for (int it = tid; it < npts; it += nt) {
            const int jl = it / nx, x = it - jl * nx;
            const int y0 = 2 * (rank * rc + jl);
            const size_t i0 = plane_off + (size_t)y0 * nx + x, i1 = i0 + nx;
            const float p0 = a.in_real[i0], p1 = a.in_real[i1];
#pragma unroll
            for (int i = 0; i < 3; i++) {
                a.st[i][i0] = p0 * a.s1;
                a.st[i][i1] = p1 * a.s1;
            }
            if (on_sensor) {
                a.rec[rec_off + (size_t)y0 * nx + x] = p0;
                a.rec[rec_off + (size_t)(y0 + 1) * nx + x] = p1;
            }
            s.row[jl * LPX + x] = make_float2(p0, p1);
        }
        __syncthreads();
        if (!(a.flags & PF_NO_FWD)) forward_plane(g, a, s, a.spec[0] + spec_off, rank, cluster);
        return;
    }

    if (a.mode == PM_VEL) {
        for (int i = 0; i < 3; i++) {
            inverse_plane(g, a, s, a.spec[i] + spec_off, rank, cluster);
            const float* A1 = a.A1[i];
            const float* A2 = a.A2[i];
            const float* A3 = a.A3[i];
            float* st = a.st[i];
            const bool no_old = (a.flags & PF_NO_OLD) != 0;
            for (int it = tid; it < npts; it += nt) {
                const int jl = it / nx, x = it - jl * nx;
                const int y0 = 2 * (rank * rc + jl);
                const size_t i0 = plane_off + (size_t)y0 * nx + x, i1 = i0 + nx;
                const float2 gv = s.row[jl * LPX + x];
                const int q0 = axis_pos(i, z, y0, x), q1 = axis_pos(i, z, y0 + 1, x);
                float n0 = __ldg(A2 + q0) * gv.x, n1 = __ldg(A2 + q1) * gv.y;
                if (!no_old) {
                    n0 = fmaf(__ldg(A1 + q0), st[i0], n0);
                    n1 = fmaf(__ldg(A1 + q1), st[i1], n1);
                }
                st[i0] = n0;
                st[i1] = n1;
                s.row[jl * LPX + x] = make_float2(__ldg(A3 + q0) * n0, __ldg(A3 + q1) * n1);
            }
            __syncthreads();
            forward_plane(g, a, s, a.spec[i] + spec_off, rank, cluster);
        }
        return;
    }

    if (a.mode == PM_RHO_FWD) {
        for (int i = 0; i < 3; i++) {
            inverse_plane(g, a, s, a.spec[i] + spec_off, rank, cluster);
            const float* A1 = a.A1[i];
            const float* A2 = a.A2[i];
            float* st = a.st[i];
            for (int it = tid; it < npts; it += nt) {
                const int jl = it / nx, x = it - jl * nx;
                const int y0 = 2 * (rank * rc + jl);
                const size_t i0 = plane_off + (size_t)y0 * nx + x, i1 = i0 + nx;
                const float2 dv = s.row[jl * LPX + x];
                const int q0 = axis_pos(i, z, y0, x), q1 = axis_pos(i, z, y0 + 1, x);
                const float r0 = fmaf(__ldg(A1 + q0), st[i0], __ldg(A2 + q0) * dv.x);
                const float r1 = fmaf(__ldg(A1 + q1), st[i1], __ldg(A2 + q1) * dv.y);
                st[i0] = r0;
                st[i1] = r1;
                float* acc = s.acc + 2 * jl * nx + x;
                if (i == 0) {
                    acc[0] = r0;
                    acc[nx] = r1;
                } else {
                    acc[0] += r0;
                    acc[nx] += r1;
                }
            }
            __syncthreads();
        }
        for (int it = tid; it < npts; it += nt) {
            const int jl = it / nx, x = it - jl * nx;
            const int y0 = 2 * (rank * rc + jl);
            const float p0 = a.c2 * s.acc[2 * jl * nx + x];
            const float p1 = a.c2 * s.acc[(2 * jl + 1) * nx + x];
            if (on_sensor) {
                a.rec[rec_off + (size_t)y0 * nx + x] = p0;
                a.rec[rec_off + (size_t)(y0 + 1) * nx + x] = p1;
            }
            s.row[jl * LPX + x] = make_float2(p0, p1);
        }
        __syncthreads();
        if (!(a.flags & PF_NO_FWD)) forward_plane(g, a, s, a.spec[0] + spec_off, rank, cluster);
        return;
    }

    // PM_RHO_ADJ: lambda_p = s0 * (sum_i D_i^- w_i) + injected data; q_i = a_i^2 q_i + c^2 lambda_p
    if (a.flags & PF_HAVE_LAMBDA) inverse_plane(g, a, s, a.spec[0] + spec_off, rank, cluster);
    for (int it = tid; it < npts; it += nt) {
        const int jl = it / nx, x = it - jl * nx;
        const int y0 = 2 * (rank * rc + jl);
        float l0 = 0.f, l1 = 0.f;
        if (a.flags & PF_HAVE_LAMBDA) {
            const float2 lv = s.row[jl * LPX + x];
            l0 = a.s0 * lv.x;
            l1 = a.s0 * lv.y;
        }
        if (on_sensor) {
            l0 += a.inj[rec_off + (size_t)y0 * nx + x];
            l1 += a.inj[rec_off + (size_t)(y0 + 1) * nx + x];
        }
        s.acc[2 * jl * nx + x] = l0;
        s.acc[(2 * jl + 1) * nx + x] = l1;
    }
    __syncthreads();
    if (a.flags & PF_FINAL) {
        // p = injected data + s0 * (sum_i D_i^- w_i) + s1 * sum_i a_i^2 q_i   (s1 = 1 / (3 c^2))
        for (int it = tid; it < npts; it += nt) {
            const int jl = it / nx, x = it - jl * nx;
            const int y0 = 2 * (rank * rc + jl);
            const size_t i0 = plane_off + (size_t)y0 * nx + x, i1 = i0 + nx;
            float o0 = 0.f, o1 = 0.f;
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const int q0 = axis_pos(i, z, y0, x), q1 = axis_pos(i, z, y0 + 1, x);
                o0 = fmaf(__ldg(a.A1[i] + q0), a.st[i][i0], o0);
                o1 = fmaf(__ldg(a.A1[i] + q1), a.st[i][i1], o1);
            }
            a.out_real[i0] = fmaf(a.s1, o0, s.acc[2 * jl * nx + x]);
            a.out_real[i1] = fmaf(a.s1, o1, s.acc[(2 * jl + 1) * nx + x]);
        }
        return;
    }
    const bool no_old = (a.flags & PF_NO_OLD) != 0;
    for (int i = 0; i < 3; i++) {
        const float* A1 = a.A1[i];
        const float* A3 = a.A3[i];
        float* st = a.st[i];
        for (int it = tid; it < npts; it += nt) {
            const int jl = it / nx, x = it - jl * nx;
            const int y0 = 2 * (rank * rc + jl);
            const size_t i0 = plane_off + (size_t)y0 * nx + x, i1 = i0 + nx;
            const int q0 = axis_pos(i, z, y0, x), q1 = axis_pos(i, z, y0 + 1, x);
            float n0 = a.c2 * s.acc[2 * jl * nx + x];
            float n1 = a.c2 * s.acc[(2 * jl + 1) * nx + x];
            if (!no_old) {
                n0 = fmaf(__ldg(A1 + q0), st[i0], n0);
                n1 = fmaf(__ldg(A1 + q1), st[i1], n1);
            }
            st[i0] = n0;
            st[i1] = n1;
            s.row[jl * LPX + x] = make_float2(__ldg(A3 + q0) * n0, __ldg(A3 + q1) * n1);
        }
        __syncthreads();
        forward_plane(g, a, s, a.spec[i] + spec_off, rank, cluster);
    }
}

// ---------------------------------------------------------------------------------------------
// z-pass kernel: z-FFT of the (y,x) half spectra, k-space multiply, inverse z-FFT
// ---------------------------------------------------------------------------------------------

enum ZMode { ZM_ONE_TO_THREE = 0, ZM_THREE_TO_THREE = 1, ZM_THREE_TO_ONE = 2 };

struct ZArgs {
    Geom g;
    const float2* tw_z;
    float2* spec[3];
    const float* kappaN;
    const float2* dt[3];
    int mode;
};

static constexpr int kZThreads = 256;

template <int NZ>
struct ZShape {
    static constexpr int A = Split<NZ>::A;  // forward R1 (inverse R2)
    static constexpr int B = Split<NZ>::B;  // forward R2 (inverse R1)
    static constexpr int TC = kZThreads / A;
    static constexpr int XL = A * (B + 1);  // xbuf per column
    static constexpr int YL = B * (A + 1);  // ybuf per column
    static constexpr size_t smem = (size_t)TC * (XL + YL) * sizeof(float2);
};

template <int NZ>
__global__ void __launch_bounds__(kZThreads) zpass_kernel(ZArgs a) {
    using S = ZShape<NZ>;
    constexpr int A = S::A, B = S::B, TC = S::TC;
    extern __shared__ float4 smem_raw[];
    float2* xbuf = reinterpret_cast<float2*>(smem_raw);
    float2* ybuf = xbuf + TC * S::XL;
    const Geom& g = a.g;
    const int ncols = g.ny * g.nxh;
    const size_t zst = (size_t)ncols;
    const int tid = threadIdx.x;
    const int cl = tid % TC;
    const int col = blockIdx.x * TC + cl;
    const bool vcol = col < ncols;
    const size_t boff = (size_t)blockIdx.y * g.nspec;
    const int ky = vcol ? col / g.nxh : 0;
    const int kx = vcol ? col - ky * g.nxh : 0;
    const int r = tid / TC;  // role index: t (F1, I2: r < B) or k1 (F2/I1: r < A)

    // forward pass 1 of field f into xbuf
    auto f1 = [&](const float2* __restrict__ in) {
        if (r < B && vcol) {
            const int t = r;
            float2 v[A];
#pragma unroll
            for (int m = 0; m < A; m++) v[m] = in[boff + (size_t)(t + B * m) * zst + col];
            Dft<A, -1>::run(v);
            float2* dst = xbuf + cl * S::XL + t;
#pragma unroll
            for (int k1 = 0; k1 < A; k1++) {
                const float2 w = (k1 == 0 || t == 0) ? v[k1] : cmul(v[k1], twiddle<NZ, -1>(a.tw_z, t * k1));
                dst[k1 * (B + 1)] = w;
            }
        }
    };
    // forward pass 2: v[k2] = X[k1 + A k2]
    auto f2 = [&](float2* v) {
        const float2* src = xbuf + cl * S::XL + r * (B + 1);
#pragma unroll
        for (int t = 0; t < B; t++) v[t] = src[t];
        Dft<B, -1>::run(v);
    };
    // multiplier of axis o at kz = k1 + A k2
    auto mult = [&](int o, int kz) -> float2 {
        const float kap = __ldg(a.kappaN + (size_t)kz * zst + col);
        const int ki = (o == 0) ? kz : (o == 1 ? ky : kx);
        return cscale(__ldg(a.dt[o] + ki), kap);
    };
    // inverse pass 1 from registers (thread t' = k1 holds x'[k1 + A m'], m' < B) into ybuf
    auto i1 = [&](float2* w) {
        Dft<B, +1>::run(w);
        const int tp = r;
        float2* dst = ybuf + cl * S::YL + tp;
#pragma unroll
        for (int k1p = 0; k1p < B; k1p++) {
            const float2 v = (k1p == 0 || tp == 0) ? w[k1p] : cmul(w[k1p], twiddle<NZ, +1>(a.tw_z, tp * k1p));
            dst[k1p * (A + 1)] = v;
        }
    };
    // inverse pass 2 and store
    auto i2 = [&](float2* __restrict__ out) {
        if (r < B && vcol) {
            const int k1p = r;
            float2 v[A];
            const float2* src = ybuf + cl * S::YL + k1p * (A + 1);
#pragma unroll
            for (int t = 0; t < A; t++) v[t] = src[t];
            Dft<A, +1>::run(v);
#pragma unroll
            for (int k2p = 0; k2p < A; k2p++) out[boff + (size_t)(k1p + B * k2p) * zst + col] = v[k2p];
        }
    };

    const bool act = (r < A) && vcol;  // F2 / I1 role
    if (a.mode == ZM_ONE_TO_THREE) {
        f1(a.spec[0]);
        __syncthreads();
        float2 v[B];
        if (act) f2(v);
        for (int o = 0; o < 3; o++) {
            if (act) {
                float2 w[B];
#pragma unroll
                for (int k2 = 0; k2 < B; k2++) w[k2] = cmul(v[k2], mult(o, r + A * k2));
                i1(w);
            }
            __syncthreads();
            i2(a.spec[o]);
            __syncthreads();
        }
    } else if (a.mode == ZM_THREE_TO_THREE) {
        for (int o = 0; o < 3; o++) {
            f1(a.spec[o]);
            __syncthreads();
            if (act) {
                float2 v[B];
                f2(v);
#pragma unroll
                for (int k2 = 0; k2 < B; k2++) v[k2] = cmul(v[k2], mult(o, r + A * k2));
                i1(v);
            }
            __syncthreads();
            i2(a.spec[o]);
            __syncthreads();
        }
    } else {  // ZM_THREE_TO_ONE
        float2 acc[B];
#pragma unroll
        for (int k2 = 0; k2 < B; k2++) acc[k2] = make_float2(0.f, 0.f);
        for (int o = 0; o < 3; o++) {
            f1(a.spec[o]);
            __syncthreads();
            if (act) {
                float2 v[B];
                f2(v);
#pragma unroll
                for (int k2 = 0; k2 < B; k2++) acc[k2] = cadd(acc[k2], cmul(v[k2], mult(o, r + A * k2)));
            }
            __syncthreads();
        }
        if (act) i1(acc);
        __syncthreads();
        i2(a.spec[0]);
    }
}

// ---------------------------------------------------------------------------------------------
// sampling kernels (Sec. 3.1 / Sec. 4.3)
// ---------------------------------------------------------------------------------------------

__global__ void rsp_gather_kernel(const float* __restrict__ rec, float* __restrict__ f,
                                  const int32_t* __restrict__ idx, int m, int M, long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / m;
        const int j = (int)(i - p * m);
        f[i] = rec[p * M + __ldg(idx + j)];
    }
}

__global__ void rsp_scatter_kernel(const float* __restrict__ f, float* __restrict__ rec,
                                   const int32_t* __restrict__ idx, int m, int M, long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / m;
        const int j = (int)(i - p * m);
        rec[p * M + __ldg(idx + j)] = f[i];
    }
}

// Unnormalised Walsh-Hadamard transform of v[0..M) in shared memory (Sylvester order), by
// log2(M) butterfly sweeps h = 1, 2, 4, ...
__device__ void fwht_smem(float* v, int M) {
    for (int h = 1; h < M; h <<= 1) {
        for (int q = threadIdx.x; q < M / 2; q += blockDim.x) {
            const int i = (q / h) * 2 * h + (q % h);
            const float x = v[i], y = v[i + h];
            v[i] = x + y;
            v[i + h] = x - y;
        }
        __syncthreads();
    }
}

// one CTA per plane (batch entry, time step): scramble, FWHT, select rows
__global__ void shd_forward_kernel(const float* __restrict__ rec, float* __restrict__ f,
                                   const int32_t* __restrict__ perm, const int32_t* __restrict__ rows,
                                   int M, int m, int pm1, float inv_sqrt_m) {
    extern __shared__ float4 smem_raw[];
    float* v = reinterpret_cast<float*>(smem_raw);
    const size_t p = blockIdx.x;
    const float* src = rec + p * M;
    for (int l = threadIdx.x; l < M; l += blockDim.x) v[l] = src[__ldg(perm + l)];
    __syncthreads();
    fwht_smem(v, M);
    const float w0 = v[0];
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const float w = v[__ldg(rows + j)];
        f[p * m + j] = pm1 ? w * inv_sqrt_m : 0.5f * (w0 + w);
    }
}

__global__ void shd_adjoint_kernel(const float* __restrict__ f, float* __restrict__ rec,
                                   const int32_t* __restrict__ perm, const int32_t* __restrict__ rows,
                                   int M, int m, int pm1, float inv_sqrt_m) {
    extern __shared__ float4 smem_raw[];
    float* e = reinterpret_cast<float*>(smem_raw);
    __shared__ float red[32];
    const size_t p = blockIdx.x;
    for (int l = threadIdx.x; l < M; l += blockDim.x) e[l] = 0.f;
    __syncthreads();
    float sum = 0.f;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const float y = f[p * m + j];
        e[__ldg(rows + j)] = y;
        sum += y;
    }
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x < 32) {
        float t = (threadIdx.x < (blockDim.x + 31) / 32) ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) red[0] = t;
    }
    __syncthreads();
    const float total = red[0];
    fwht_smem(e, M);
    float* dst = rec + p * M;
    for (int l = threadIdx.x; l < M; l += blockDim.x)
        dst[__ldg(perm + l)] = pm1 ? e[l] * inv_sqrt_m : 0.5f * (total + e[l]);
}

// adjoint with T = 1: p = 0 except the detection plane, which takes the injected plane
__global__ void inject_plane_kernel(const float* __restrict__ inj, float* __restrict__ p, Geom g) {
    const long long total = (long long)g.B * g.nreal;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / g.nreal;
        const long long v = i - b * g.nreal;
        const long long z = v / g.m_plane;
        p[i] = (z == g.sensor_z) ? inj[b * (long long)g.T * g.m_plane + (v - z * g.m_plane)] : 0.f;
    }
}

// ---------------------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------------------

typedef void (*ZKernel)(ZArgs);

static ZKernel zkernel_for(int nz, size_t* smem) {
    switch (nz) {
#define PAT_ZCASE(N) \
    case N: *smem = ZShape<N>::smem; return zpass_kernel<N>;
        PAT_ZCASE(8)
        PAT_ZCASE(16)
        PAT_ZCASE(32)
        PAT_ZCASE(64)
        PAT_ZCASE(128)
        PAT_ZCASE(256)
#undef PAT_ZCASE
        default: *smem = 0; return nullptr;
    }
}

int z_tile_columns(int nz) {
    const int a = (nz >= 128) ? 16 : (nz >= 32) ? 8 : (nz >= 8) ? 4 : 2;
    return kZThreads / a;
}

// Dynamic shared-memory limits are per kernel, not per grid: keep the largest any grid needed so
// that several grids of different sizes can coexist in one process.
static size_t g_plane_smem_max = 0, g_z_smem_max[9] = {0}, g_shd_smem_max = 0;

cudaError_t configure_kernels(const Geom& g, size_t* plane_smem, size_t* z_smem) {
    const size_t ps = plane_smem_bytes(g);
    cudaError_t e;
    if (ps > g_plane_smem_max) {
        e = cudaFuncSetAttribute(plane_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ps);
        if (e != cudaSuccess) return e;
        g_plane_smem_max = ps;
    }
    if (g.cs > 8) {
        e = cudaFuncSetAttribute(plane_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    size_t zs = 0;
    ZKernel zk = zkernel_for(g.nz, &zs);
    if (!zk) return cudaErrorInvalidValue;
    int lz = 0;
    while ((1 << lz) < g.nz) lz++;
    if (zs > g_z_smem_max[lz]) {
        e = cudaFuncSetAttribute(zk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zs);
        if (e != cudaSuccess) return e;
        g_z_smem_max[lz] = zs;
    }
    const size_t shd_bytes = (size_t)g.m_plane * sizeof(float);
    if (shd_bytes > 48 * 1024 && shd_bytes > g_shd_smem_max) {
        e = cudaFuncSetAttribute(shd_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shd_bytes);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(shd_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shd_bytes);
        if (e != cudaSuccess) return e;
        g_shd_smem_max = shd_bytes;
    }
    if (plane_smem) *plane_smem = ps;
    if (z_smem) *z_smem = zs;
    return cudaSuccess;
}

static cudaError_t launch_plane_raw(const PlaneArgs& a, cudaStream_t st) {
    const Geom& g = a.g;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g.cs, g.nz, g.B);
    cfg.blockDim = dim3(kPlaneThreads, 1, 1);
    cfg.dynamicSmemBytes = plane_smem_bytes(g);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = g.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, plane_kernel, a);
}

static cudaError_t launch_z_raw(const ZArgs& a, cudaStream_t st) {
    size_t smem = 0;
    ZKernel k = zkernel_for(a.g.nz, &smem);
    if (!k) return cudaErrorInvalidValue;
    const int tc = z_tile_columns(a.g.nz);
    const int ncols = a.g.ny * a.g.nxh;
    dim3 grid((ncols + tc - 1) / tc, a.g.B, 1);
    k<<<grid, kZThreads, smem, st>>>(a);
    return cudaGetLastError();
}

// optional event bracketing of one launch
template <class F>
static cudaError_t timed(Profiler* prof, int cls, cudaStream_t st, F&& launch) {
    if (!prof || !prof->on) return launch();
    Profiler::Rec r;
    r.cls = cls;
    cudaError_t e = prof->ev(&r.a);
    if (e != cudaSuccess) return e;
    if ((e = prof->ev(&r.b)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(r.a, st)) != cudaSuccess) return e;
    if ((e = launch()) != cudaSuccess) return e;
    if ((e = cudaEventRecord(r.b, st)) != cudaSuccess) return e;
    prof->recs.push_back(r);
    return cudaSuccess;
}

static cudaError_t launch_plane(const PlaneArgs& a, cudaStream_t st, Profiler* prof) {
    const int cls = a.mode == PM_INIT_FWD ? KC_PLANE_INIT : a.mode == PM_VEL ? KC_PLANE_VEL
                  : a.mode == PM_RHO_FWD ? KC_PLANE_RHO_FWD : KC_PLANE_RHO_ADJ;
    return timed(prof, cls, st, [&] { return launch_plane_raw(a, st); });
}

static cudaError_t launch_z(const ZArgs& a, cudaStream_t st, Profiler* prof) {
    const int cls = a.mode == ZM_ONE_TO_THREE ? KC_Z_ONE_TO_THREE
                  : a.mode == ZM_THREE_TO_THREE ? KC_Z_THREE_TO_THREE : KC_Z_THREE_TO_ONE;
    return timed(prof, cls, st, [&] { return launch_z_raw(a, st); });
}

static PlaneArgs plane_base(const Geom& g, const DeviceTables& t, const Workspace& w) {
    PlaneArgs a = {};
    a.g = g;
    a.tw_x = t.tw[AX];
    a.tw_y = t.tw[AY];
    for (int i = 0; i < 3; i++) a.spec[i] = w.spec[i];
    return a;
}

static ZArgs z_base(const Geom& g, const DeviceTables& t, const Workspace& w, int mode, bool plus) {
    ZArgs a = {};
    a.g = g;
    a.tw_z = t.tw[AZ];
    for (int i = 0; i < 3; i++) {
        a.spec[i] = w.spec[i];
        a.dt[i] = plus ? t.dplus[i] : t.dminus[i];
    }
    a.kappaN = t.kappaN;
    a.mode = mode;
    return a;
}

static void set_tables(PlaneArgs& a, const DeviceTables& t, int c1, int c2, int c3) {
    for (int i = 0; i < 3; i++) {
        a.A1[i] = t.coef[c1][i];
        a.A2[i] = t.coef[c2][i];
        a.A3[i] = t.coef[c3][i];
    }
}

#define PAT_TRY(x)                            \
    do {                                      \
        cudaError_t _e = (x);                 \
        if (_e != cudaSuccess) return _e;     \
    } while (0)

cudaError_t run_sample(const Geom& g, const Workspace& w, int kind, int m, const float* pbar,
                       float* f, int nt, cudaStream_t st) {
    const long long planes = (long long)g.B * nt;
    if (kind == PAT_SAMPLE_FULL) {
        return cudaMemcpyAsync(f, pbar, sizeof(float) * planes * g.m_plane, cudaMemcpyDeviceToDevice, st);
    }
    if (kind == PAT_SAMPLE_POINTS) {
        const long long total = planes * m;
        if (total == 0) return cudaSuccess;
        const int blocks = (int)((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
        rsp_gather_kernel<<<blocks, 256, 0, st>>>(pbar, f, w.idx, m, g.m_plane, total);
        return cudaGetLastError();
    }
    shd_forward_kernel<<<(unsigned)planes, 1024, g.m_plane * sizeof(float), st>>>(
        pbar, f, w.perm, w.rows, g.m_plane, m, kind == PAT_SAMPLE_HADAMARDPM, (float)(1.0 / sqrt((double)g.m_plane)));
    return cudaGetLastError();
}

cudaError_t run_sample_adjoint(const Geom& g, const Workspace& w, int kind, int m, const float* f,
                               float* pbar, int nt, cudaStream_t st) {
    const long long planes = (long long)g.B * nt;
    if (kind == PAT_SAMPLE_FULL) {
        return cudaMemcpyAsync(pbar, f, sizeof(float) * planes * g.m_plane, cudaMemcpyDeviceToDevice, st);
    }
    if (kind == PAT_SAMPLE_POINTS) {
        PAT_TRY(cudaMemsetAsync(pbar, 0, sizeof(float) * planes * g.m_plane, st));
        const long long total = planes * m;
        if (total == 0) return cudaSuccess;
        const int blocks = (int)((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
        rsp_scatter_kernel<<<blocks, 256, 0, st>>>(f, pbar, w.idx, m, g.m_plane, total);
        return cudaGetLastError();
    }
    shd_adjoint_kernel<<<(unsigned)planes, 1024, g.m_plane * sizeof(float), st>>>(
        f, pbar, w.perm, w.rows, g.m_plane, m, kind == PAT_SAMPLE_HADAMARDPM, (float)(1.0 / sqrt((double)g.m_plane)));
    return cudaGetLastError();
}

cudaError_t run_forward(const Geom& g, const DeviceTables& t, const Workspace& w, const Scalars& s,
                        int kind, int m, const float* p0, float* f, cudaStream_t st, Profiler* prof) {
    float* rec = (kind == PAT_SAMPLE_FULL) ? f : w.rec;
    const float c2 = (float)(s.c * s.c);
    // initial state: rho_i = p0 / (3 c^2), record n = 0, forward (y,x) FFT of p0
    PlaneArgs pi = plane_base(g, t, w);
    pi.mode = PM_INIT_FWD;
    pi.flags = (g.T == 1) ? PF_NO_FWD : 0;
    pi.in_real = p0;
    for (int i = 0; i < 3; i++) pi.st[i] = w.st[3 + i];
    pi.s1 = (float)(1.0 / (3.0 * s.c * s.c));
    pi.rec = rec;
    pi.n_rec = 0;
    PAT_TRY(launch_plane(pi, st, prof));

    ZArgs zg = z_base(g, t, w, ZM_ONE_TO_THREE, true);
    ZArgs zd = z_base(g, t, w, ZM_THREE_TO_THREE, false);
    PlaneArgs pv = plane_base(g, t, w);
    pv.mode = PM_VEL;
    for (int i = 0; i < 3; i++) pv.st[i] = w.st[i];
    PlaneArgs pr = plane_base(g, t, w);
    pr.mode = PM_RHO_FWD;
    for (int i = 0; i < 3; i++) pr.st[i] = w.st[3 + i];
    set_tables(pr, t, CT_A2, CT_DF_D, CT_ONE);
    pr.c2 = c2;
    pr.rec = rec;
    for (int n = 0; n + 1 < g.T; n++) {
        PAT_TRY(launch_z(zg, st, prof));
        if (n == 0) {
            set_tables(pv, t, CT_AS2, CT_VF0_G, CT_ONE);
            pv.flags = PF_NO_OLD;
        } else {
            set_tables(pv, t, CT_AS2, CT_VF_G, CT_ONE);
            pv.flags = 0;
        }
        PAT_TRY(launch_plane(pv, st, prof));
        PAT_TRY(launch_z(zd, st, prof));
        pr.n_rec = n + 1;
        pr.flags = (n + 2 == g.T) ? PF_NO_FWD : 0;
        PAT_TRY(launch_plane(pr, st, prof));
    }
    if (kind != PAT_SAMPLE_FULL)
        PAT_TRY(timed(prof, KC_SAMPLE, st, [&] { return run_sample(g, w, kind, m, rec, f, g.T, st); }));
    return cudaSuccess;
}

cudaError_t run_adjoint(const Geom& g, const DeviceTables& t, const Workspace& w, const Scalars& s,
                        int kind, int m, const float* f, float* p, cudaStream_t st, Profiler* prof) {
    const float* inj = f;
    if (kind != PAT_SAMPLE_FULL) {
        PAT_TRY(timed(prof, KC_SAMPLE, st, [&] { return run_sample_adjoint(g, w, kind, m, f, w.rec, g.T, st); }));
        inj = w.rec;
    }
    if (g.T == 1) {
        const long long total = (long long)g.B * g.nreal;
        const int blocks = (int)((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
        inject_plane_kernel<<<blocks, 256, 0, st>>>(inj, p, g);
        return cudaGetLastError();
    }
    const float c2 = (float)(s.c * s.c);
    PlaneArgs pq = plane_base(g, t, w);
    pq.mode = PM_RHO_ADJ;
    for (int i = 0; i < 3; i++) pq.st[i] = w.st[3 + i];
    set_tables(pq, t, CT_A2, CT_ONE, CT_A);
    pq.c2 = c2;
    pq.s0 = (float)(s.dt / s.rho0);
    pq.s1 = (float)(1.0 / (3.0 * s.c * s.c));
    pq.inj = inj;
    pq.out_real = p;
    // q_i^{T-1} = c^2 (injected plane T-1), transform a_i q_i
    pq.flags = PF_NO_OLD;
    pq.n_rec = g.T - 1;
    PAT_TRY(launch_plane(pq, st, prof));

    ZArgs zg = z_base(g, t, w, ZM_THREE_TO_THREE, true);
    ZArgs zd = z_base(g, t, w, ZM_THREE_TO_ONE, false);
    PlaneArgs pv = plane_base(g, t, w);
    pv.mode = PM_VEL;
    for (int i = 0; i < 3; i++) pv.st[i] = w.st[i];
    for (int n = g.T - 2; n >= 0; n--) {
        PAT_TRY(launch_z(zg, st, prof));
        set_tables(pv, t, CT_AS2, CT_VA_G, (n == 0) ? CT_VA0_OUT : CT_AS);
        pv.flags = (n + 2 == g.T) ? PF_NO_OLD : 0;
        PAT_TRY(launch_plane(pv, st, prof));
        PAT_TRY(launch_z(zd, st, prof));
        pq.flags = PF_HAVE_LAMBDA | ((n == 0) ? PF_FINAL : 0);
        pq.n_rec = n;
        PAT_TRY(launch_plane(pq, st, prof));
    }
    return cudaSuccess;
}

}  // namespace pat

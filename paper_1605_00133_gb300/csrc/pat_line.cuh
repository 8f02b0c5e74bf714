// pat_line.cuh - line passes of the k-space time step (Sec. 4.3) in mixed representation.
//
// The split-field update of axis i (velocity u_i, density rho_i) needs only the derivative along
// axis i and the PML factor of axis i, which depends on x_i alone.  So u_i and rho_i are kept with
// axis i in real space and the other two axes in Fourier space, and the pressure p = c^2 sum rho_i
// as a full 3D half spectrum.  One pass over the lines of axis i then does a whole time step of
// that axis with 1D transforms only:
//
//   forward  g   = F_i^-1[ i k_i kappa e^{+ik_i dx/2} p^ ] / n_i        (D_i^+ p)
//            u_i = as^2 u_i - as dt/rho0 g                              (state 1)
//            d   = F_i^-1[ i k_i kappa e^{-ik_i dx/2} F_i u_i ] / n_i   (D_i^- u_i)
//            rho_i = a^2 rho_i - a dt rho0 d                            (state 2)
//            p^_new (+)= c^2 F_i rho_i
//   adjoint  l   = F_i^-1[ lambda^ ] / n_i,  q_i = a^2 q_i + c^2 l,  w = a q_i
//            g   = F_i^-1[ i k_i kappa e^{+ik_i dx/2} F_i w ] / n_i
//            v_i = as^2 v_i + dt rho0 g,  y = as v_i
//            lambda^_new (+)= (dt/rho0) i k_i kappa e^{-ik_i dx/2} F_i y
//
// i.e. in both directions: [pre factor] F^-1, state update, F, [mid factor] F^-1, state update, F,
// [post factor], accumulate.  The passes of one step run x, y, z; the x pass writes the new
// spectrum, the y and z passes add to it; the z pass also records (forward) the detection plane's
// (kx, ky) spectrum (1/nz) sum_kz p^ e^{+2 pi i kz zs/nz}, or injects (adjoint) the data spectrum
// S e^{-2 pi i kz zs/nz}.
//
// A CTA owns TC lines.  A line's length-L transform is the two-pass split of pat_fft.cuh: in the
// k-space layout thread r < A holds X[r + A k2] (k2 < B), in the spatial layout thread r < B holds
// x[r + B k2] (k2 < A) -- or, when A = 2B, a thread pair shares row group xr (each half holds A/2 of
// its values and computes half of its A-point DFT; LS::PNEW says which rows pair up); each transform
// is one exchange through shared memory laid out [row][line] with the line index fastest.  Two
// exchange buffers alternate, so every transform costs one barrier.  The pass's table block and the
// old values of both states are copied to shared memory as soon as the kernel starts (bulk copies of
// the TMA unit completing on mbarriers, or per-thread cp.async for 16 KB tiles), and the old values
// of the spectrum a y or z pass adds to as soon as its writer has completed, so their latency
// overlaps transforms instead of stalling each update.
//
// Launch overlap.  The y and z passes of a step read only the previous step's spectrum and their own
// states until they add to the new spectrum, so they are launched as programmatic dependents that
// start at once and wait for their predecessor (griddepcontrol.wait) only after their first state
// update, before fetching the spectrum they add to (LF_LATE_WAIT).  Everything they read before the
// wait was written by kernels that had completed before the x pass of the step passed its own wait,
// and is read through L2 (ld.cg, cp.async.cg, bulk copies).
// No kernel waits on a grid whose CTAs have not all started, so the overlap cannot deadlock.
//
// States and kappa are stored tile-major, [B][tile][L][TC] (tile = line / TC, lines padded to a
// whole tile), so a CTA's tile is one contiguous block and every access of a thread is its own base
// plus a compile-time offset.  The twiddles of the two transform halves come from per-thread tables
// (twi, twf: entry k of thread r at k * (row stride) + r) for the same reason.
//
// Spectrum access per axis (3D half spectrum [kz][kx][ky], kx <= nx/2):
//   z lines (kx, ky): column access, stride nxh*ny
//   y lines (kz, kx): each line is a contiguous row; the CTA's TC rows are one contiguous block,
//                     moved through shared memory (row pitch L+1) to stay coalesced
//   x lines (kz <= nz/2, ky): bins kx > nx/2 are the conjugates of (-kz, nx-kx, -ky); on output the
//                     line also writes that mirror entry, except on the self-conjugate planes
//                     kz = 0 and kz = nz/2, whose lines (ky) and (-ky) are both present.
#pragma once
#include "pat_fft.cuh"
#include "pat_kargs.h"

namespace pat {

constexpr int kCopyPolls = 1 << 20;  // bound of a wait for a bulk copy: each poll suspends <= ~1 us

template <int L>
struct LS {
    static constexpr int A = Split<L>::A;  // radix of the spatial-side DFT
    static constexpr int B = Split<L>::B;  // radix of the k-space-side DFT
    // A = 2B: the spatial-side A-point DFT is shared by a thread pair (two A/2-point DFTs and one
    // radix-2 stage through warp shuffles), so both layouts use every thread
    static constexpr bool PAIR = (A == 2 * B);
    static constexpr int XN = PAIR ? A / 2 : A;  // values per thread, spatial layout
    // lines per CTA: about 1024 line points per CTA (8 KB tiles), at least 8 lines (64-byte rows);
    // thread pairs must share a warp, so at most 16 lines when PAIR
    static constexpr int TC0 = (1024 / L > 32) ? 32 : (1024 / L < 8 ? 8 : 1024 / L);
    static constexpr int TC = (PAIR && TC0 > 16) ? 16 : TC0;
    static constexpr int NT = A * TC;
    // staging row pitch for y lines: odd for 16-line half-warps, = 2 (mod 16) for 8 lines
    static constexpr int PITCH = (TC >= 16) ? L + 1 : L + 2;
    static constexpr int BUF = L * TC + 2 * TC;  // one exchange buffer (float2), also holds TC staged rows
    static constexpr int TILE = L * TC;          // one prefetched tile (float2)
    // Resident CTAs per SM the register budget is sized for: the target, or fewer where shared
    // memory (228 KB per SM, 1 KB reserved per CTA) allows fewer.  Where three tiles would cut the
    // CTAs below the target (long lines), the old output of y and z lines (pfo) reuses the state-1
    // tile once every thread has read it.
    static constexpr int MINB_T = (NT >= 256) ? 2 : 4;
    static constexpr int SMEM_SM = 233472;
    // the per-axis tables a time step reads in every phase (twiddles, k-space factors, state
    // coefficients) are copied to shared memory at the start of a pass, up to L = 128
    static constexpr bool STAGE = (L <= 128);
    static constexpr int TAB2 = STAGE ? 5 * L : 0;  // float2: twi, twf, k-space factors pre/mid/post
    // float: coefficients of state 1 and state 2, L + 2 each: entry j at j + 2 [j >= L/2], so that
    // the two halves of a thread pair (positions L/2 apart) read different banks
    static constexpr int CSTR = L + 2;
    static constexpr int TAB1 = STAGE ? 6 * CSTR : 0;
    static constexpr size_t SBASE = (2 * (size_t)BUF + TAB2) * sizeof(float2) + TAB1 * sizeof(float);
    static constexpr bool PFO_ALIAS = (int)(SMEM_SM / (SBASE + 3 * (size_t)TILE * sizeof(float2) + 1024)) < MINB_T;
    static constexpr size_t BAR_OFF = SBASE + (PFO_ALIAS ? 2 : 3) * (size_t)TILE * sizeof(float2);
    static constexpr size_t smem = BAR_OFF + 32;  // three mbarriers (tables, state 1, state 2)
    static constexpr unsigned TILE_BYTES = TILE * sizeof(float2);
    // old state tiles staged by bulk copies (TMA) up to 8 KB, in BULK_PARTS pieces; larger tiles by
    // per-thread 16-byte cp.async copies
    static constexpr bool BULK = TILE_BYTES <= 8192;
    static constexpr int BULK_PARTS = 1;
    static constexpr unsigned TAB_BYTES = TAB2 * sizeof(float2) + TAB1 * sizeof(float);
    static_assert(BAR_OFF % 16 == 0 && TILE_BYTES % 16 == 0 && TAB_BYTES % 16 == 0 &&
                      (2 * (size_t)BUF * sizeof(float2)) % 16 == 0,
                  "bulk copies need 16-byte aligned shared-memory blocks and sizes");
    static constexpr int MINB_S = (int)(SMEM_SM / (smem + 1024));
    static constexpr int MINB = (MINB_T < MINB_S) ? MINB_T : (MINB_S > 0 ? MINB_S : 1);
    // exchange rows are swizzled (bit 0 of the row flipped by bit 0 of row / B) when a row is only
    // half the banks
    static constexpr bool SWZ = TC < 16;
    // Thread pairs.  With 8 lines per CTA a half-warp holds two rows r of the k-space layout.  If the
    // two halves of a pair were rows r and r + 1, a half-warp would read its state tiles at positions
    // L/2 apart (same banks); so then the pair is rows r and r + 2 (xh = bit 1 of r, xr = the other
    // bits) and the exchange flip also takes bit 0 of row / A.
    static constexpr bool PNEW = PAIR && TC <= 8;
    static constexpr int PD = PNEW ? 2 : 1;  // pair partner: thread index ^ (PD * TC)
    static constexpr int TWF_STRIDE = PAIR ? A : B;  // row stride of the forward twiddle table
};

// W_R^(DIR k) = exp(DIR 2 pi i k / R), R in {2, 4, 8, 16}, k < R/2
template <int R, int DIR>
__device__ __forceinline__ float2 wr(int k) {
    return make_float2(w16c(k * (16 / R)), DIR * w16s(k * (16 / R)));
}

template <int L, int AX>
struct LineCtx {
    using S = LS<L>;
    static constexpr int A = S::A, B = S::B, TC = S::TC, XN = S::XN;
    static constexpr bool PAIR = S::PAIR;
    const LineArgs& a;
    float2* buf0;
    float2* buf1;
    float2* pf1;    // prefetched old state 1, [j][line]
    float2* pf2;    // prefetched old state 2
    float2* pfo;    // prefetched old output: z lines [kz][line], y lines the contiguous row block
    int cl, r, col, col0, b;
    int xr, xh;     // spatial layout: row group and half (PAIR), else xr = r, xh = 0
    bool vcol, xact;
    size_t tbase;   // this CTA's tile of the states, element (j = 0, line 0)
    size_t pbase;   // this batch entry's 3D spectrum
    float2 sgn;     // PAIR butterflies: (+1, +1) for the even half, (-1, -1) for the odd one
    const float2* ti;  // this thread's twiddles (global tables, or their shared copies after stage())
    const float2* tf;
    float2* tab2;      // shared copies (S::STAGE): twi, twf, k-space factors [3]
    float* tab1;       // ... state coefficients [2][3]
    unsigned long long* bar;  // mbarriers of the bulk copies: tables, state 1, state 2
    int ka, kb;     // x lines: kz, ky
    int ma, mb;     // x lines: the mirror line's kz, ky

    __device__ LineCtx(const LineArgs& args, float2* smem) : a(args) {
        buf0 = smem;
        buf1 = smem + S::BUF;
        pf1 = smem + 2 * S::BUF;
        pf2 = pf1 + S::TILE;
        pfo = S::PFO_ALIAS ? pf1 : pf2 + S::TILE;
        tab2 = pf2 + (S::PFO_ALIAS ? 1 : 2) * S::TILE;
        tab1 = reinterpret_cast<float*>(tab2 + S::TAB2);
        bar = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(smem) + S::BAR_OFF);
        const int tid = threadIdx.x;
        cl = tid % TC;
        r = tid / TC;
        xr = PAIR ? (S::PNEW ? ((r & 1) | ((r >> 2) << 1)) : (r >> 1)) : r;
        xh = PAIR ? (S::PNEW ? ((r >> 1) & 1) : (r & 1)) : 0;
        col0 = blockIdx.x * TC;
        col = col0 + cl;
        vcol = col < a.ncols;
        xact = vcol && (PAIR || r < B);
        b = blockIdx.y;
        tbase = ((size_t)b * gridDim.x + blockIdx.x) * (size_t)(L * TC);
        pbase = (size_t)b * a.g.nspec;
        sgn = xh ? make_float2(-1.f, -1.f) : make_float2(1.f, 1.f);
        ti = a.twi + r;
        tf = a.twf + r;
        ka = kb = ma = mb = 0;
        if (AX == 2) {
            const int ny = a.g.ny, nz = a.g.nz;
            ka = col / ny;
            kb = col - ka * ny;
            ma = (nz - ka) & (nz - 1);
            mb = (ny - kb) & (ny - 1);
        }
    }
    // read a table entry: shared copies (S::STAGE) by plain loads, global tables through the
    // read-only path
    template <class T>
    __device__ __forceinline__ static T rd(const T* p) {
        if constexpr (S::STAGE) return *p;
        else return __ldg(p);
    }
    // position along the line of spatial-layout value q
    __device__ __forceinline__ int xpos(int q) const { return PAIR ? xr + B * (XN * xh + q) : r + B * q; }
    // whether spatial-layout value q sits at a position >= L/2 (the odd half of a thread pair, or a
    // thread's upper values)
    __device__ __forceinline__ int upper(int q) const { return PAIR ? xh : (q >= XN / 2 ? 1 : 0); }
    // state element of this line at spatial-layout value q (tile-major layout)
    __device__ __forceinline__ size_t sidx(int q) const { return tbase + (size_t)xpos(q) * TC + cl; }

    // Exchange-buffer elements, layout [row][line].  With 8 lines a row is half the banks; rows that
    // a half-warp touches together differ by 1, A or B, so bit 0 of the row is flipped by bit 0 of
    // row / B (and, with S::PNEW, also by bit 0 of row / A) to put them in different halves
    // (S::SWZ).  Each access below writes row = (this thread's part) + (a compile-time part) and
    // resolves the flip per thread, so the address is a per-thread base plus a constant:
    //   inv, k-space side writes  row = k A + r        flip = (k A/B + r/B) & 1   (PNEW: ^ k & 1)
    //   inv, spatial side reads   row = r A + t        flip = (r A/B + t/B) & 1       (r < B)
    //                   PAIR      row = xr A + 2q + xh flip = [q >= B/2]          (PNEW: ^ xr & 1)
    //   fwd, spatial side writes  row = k B + r        flip = k & 1                   (r < B)
    //                   PAIR      row = (2k + xh) B + xr  flip = xh               (PNEW: ^ k & 1)
    //   fwd, k-space side reads   row = r B + t        flip = r & 1               (PNEW: ^ r/2 & 1)
    // (a flip changes bit 0 of the row, which is bit 0 of the thread's part in every case).
    __device__ __forceinline__ int xo_inv_st(int k) const {
        const int f = S::SWZ ? ((((A / B) % 2) ? k : 0) + r / B + (S::PNEW ? k : 0)) & 1 : 0;
        return (k * A + (r ^ f)) * TC + cl;
    }
    __device__ __forceinline__ int xo_inv_ld(int t) const {
        if (PAIR) {
            // t = 2q + xh is passed as 2q
            const int f = S::SWZ ? ((t / 2 >= B / 2 ? 1 : 0) ^ (S::PNEW ? (xr & 1) : 0)) : 0;
            return (xr * A + t + (xh ^ f)) * TC + cl;
        }
        const int f = S::SWZ ? (((A / B) % 2 ? r : 0) + t / B) & 1 : 0;
        return (r * A + (t ^ f)) * TC + cl;
    }
    __device__ __forceinline__ int xo_fwd_st(int k) const {
        if (PAIR) return (2 * k * B + xh * B + (xr ^ (S::SWZ ? (xh ^ (S::PNEW ? (k & 1) : 0)) : 0))) * TC + cl;
        return (k * B + (r ^ (S::SWZ ? (k & 1) : 0))) * TC + cl;
    }
    __device__ __forceinline__ int xo_fwd_ld(int t) const {
        return (r * B + (t ^ (S::SWZ ? ((r ^ (S::PNEW ? (r >> 1) : 0)) & 1) : 0))) * TC + cl;
    }

    // ---- transforms between the layouts (every thread of the CTA must call these)
    // k-space layout (v) -> spatial layout (x) through xb
    __device__ __forceinline__ void inv(float2* v, float2* x, float2* xb) const {
        if (vcol) {
            Dft<B, +1>::run(v);
            // W_L^{+r k}, k < B, row stride A
#pragma unroll
            for (int k1p = 0; k1p < B; k1p++)
                xb[xo_inv_st(k1p)] = (k1p == 0) ? v[0] : cmul(v[k1p], rd(ti + k1p * A));
        }
        __syncthreads();
        if (PAIR) {
            // A-point DFT of row group xr by decimation in time: this thread the even (xh = 0) or odd
            // inputs, then X[k] = E[k] + W_A^k O[k], X[k + A/2] = E[k] - W_A^k O[k]
#pragma unroll
            for (int q = 0; q < XN; q++) x[q] = vcol ? xb[xo_inv_ld(2 * q)] : make_float2(0.f, 0.f);
            Dft<XN, +1>::run(x);
#pragma unroll
            for (int k = 1; k < XN; k++)
                if (xh) x[k] = cmul(x[k], wr<A, +1>(k));
#pragma unroll
            for (int k = 0; k < XN; k++) {
                const float2 t = make_float2(__shfl_xor_sync(0xffffffffu, x[k].x, S::PD * TC),
                                             __shfl_xor_sync(0xffffffffu, x[k].y, S::PD * TC));
                x[k] = csgn_add(sgn, x[k], t);  // E + W O (even half) or E - W O (odd half)
            }
        } else if (vcol && r < B) {
#pragma unroll
            for (int t = 0; t < A; t++) x[t] = xb[xo_inv_ld(t)];
            Dft<A, +1>::run(x);
        }
    }
    // spatial layout (x) -> k-space layout (v) through xb
    __device__ __forceinline__ void fwd(float2* x, float2* v, float2* xb) const {
        if (PAIR) {
            // decimation in frequency: Y[2k] from x[q] + x[q + A/2] (xh = 0), Y[2k+1] from
            // (x[q] - x[q + A/2]) W_A^-q (xh = 1); this thread holds x[q + xh A/2]
#pragma unroll
            for (int q = 0; q < XN; q++) {
                const float2 t = make_float2(__shfl_xor_sync(0xffffffffu, x[q].x, S::PD * TC),
                                             __shfl_xor_sync(0xffffffffu, x[q].y, S::PD * TC));
                x[q] = csgn_add(sgn, x[q], t);  // x[q] + x[q + A/2] (even half) or their difference
            }
#pragma unroll
            for (int q = 1; q < XN; q++)
                if (xh) x[q] = cmul(x[q], wr<A, -1>(q));
            Dft<XN, -1>::run(x);
            if (vcol) {
                // W_L^{-xr (2k + xh)}, k < XN, row stride A
#pragma unroll
                for (int k = 0; k < XN; k++) xb[xo_fwd_st(k)] = cmul(x[k], rd(tf + k * A));
            }
        } else if (vcol && r < B) {
            Dft<A, -1>::run(x);
            // W_L^{-r k}, k < A, row stride B
#pragma unroll
            for (int k1 = 0; k1 < A; k1++)
                xb[xo_fwd_st(k1)] = (k1 == 0) ? x[0] : cmul(x[k1], rd(tf + k1 * B));
        }
        __syncthreads();
        if (vcol) {
#pragma unroll
            for (int t = 0; t < B; t++) v[t] = xb[xo_fwd_ld(t)];
            Dft<B, -1>::run(v);
        }
    }

    // ---- 3D spectrum access in the k-space layout
    __device__ __forceinline__ void load_k(const float2* __restrict__ in, float2* v) const {
        if (AX == 0) {
            if (vcol) {
#pragma unroll
                for (int k2 = 0; k2 < B; k2++) v[k2] = __ldcg(in + pbase + (size_t)(r + A * k2) * a.ncols + col);
            }
        } else if (AX == 1) {
            const int nrows = min(TC, a.ncols - col0);
            const float4* blk = reinterpret_cast<const float4*>(in + pbase + (size_t)col0 * L);
            for (int e = threadIdx.x; e < nrows * (L / 2); e += S::NT) {
                const float4 w = __ldcg(blk + e);
                const int row = (2 * e) / L, pt = (2 * e) % L;
                float2* d = buf1 + row * S::PITCH + pt;
                d[0] = make_float2(w.x, w.y);
                d[1] = make_float2(w.z, w.w);
            }
            __syncthreads();
            if (vcol) {
#pragma unroll
                for (int k2 = 0; k2 < B; k2++) v[k2] = buf1[cl * S::PITCH + r + A * k2];
            }
        } else {
            // bin j = r + A k2 with r < A: j <= L/2 exactly for k2 < B/2, and for k2 = B/2 when r = 0
            if (vcol) {
                const int nxh = a.g.nxh, ny = a.g.ny;
                const float2* own = in + pbase + (size_t)ka * nxh * ny + kb;
                const float2* mir = in + pbase + (size_t)ma * nxh * ny + mb;
#pragma unroll
                for (int k2 = 0; k2 < B; k2++) {
                    const int j = r + A * k2;
                    if (k2 < B / 2 || (k2 == B / 2 && r == 0)) v[k2] = __ldcg(own + (size_t)j * ny);
                    else v[k2] = cconj(__ldcg(mir + (size_t)(L - j) * ny));
                }
            }
        }
    }
    // write (or add, LF_ACCUM) the k-space layout values to the 3D spectrum; z lines return the
    // stored totals in v.  pre: the old values of z and y lines are in pfo (prefetch_out) rather
    // than to be loaded.
    __device__ __forceinline__ void store_k(float2* __restrict__ out, float2* v, bool accum, bool pre) const {
        if (AX == 0) {
            if (vcol) {
#pragma unroll
                for (int k2 = 0; k2 < B; k2++) {
                    const int j = r + A * k2;
                    float2* p = out + pbase + (size_t)j * a.ncols + col;
                    if (accum) v[k2] = cadd(pre ? pfo[j * TC + cl] : *p, v[k2]);
                    *p = v[k2];
                }
            }
        } else if (AX == 1) {
            // buf0's last reader was the previous inverse transform, fenced by the barrier of the
            // forward transform since
            if (vcol) {
#pragma unroll
                for (int k2 = 0; k2 < B; k2++) buf0[cl * S::PITCH + r + A * k2] = v[k2];
            }
            __syncthreads();
            const int nrows = min(TC, a.ncols - col0);
            float4* blk = reinterpret_cast<float4*>(out + pbase + (size_t)col0 * L);
            for (int e = threadIdx.x; e < nrows * (L / 2); e += S::NT) {
                const int row = (2 * e) / L, pt = (2 * e) % L;
                const float2* s = buf0 + row * S::PITCH + pt;
                float4 w = make_float4(s[0].x, s[0].y, s[1].x, s[1].y);
                if (accum) {
                    const float4 o = pre ? reinterpret_cast<const float4*>(pfo)[e] : blk[e];
                    w.x += o.x; w.y += o.y; w.z += o.z; w.w += o.w;
                }
                blk[e] = w;
            }
        } else {
            // own entry for j <= L/2; mirror entry (-kz, L-j mod L, -ky) for j = 0 and j >= L/2, except
            // on the self-conjugate planes kz = 0, nz/2 (k2 ranges as in load_k)
            if (vcol) {
                const int nxh = a.g.nxh, ny = a.g.ny, nz = a.g.nz;
                const bool mirror = (ka != 0) && (2 * ka != nz);
                float2* own = out + pbase + (size_t)ka * nxh * ny + kb;
                float2* mir = out + pbase + (size_t)ma * nxh * ny + mb;
#pragma unroll
                for (int k2 = 0; k2 < B; k2++) {
                    const int j = r + A * k2;
                    if (k2 < B / 2 || (k2 == B / 2 && r == 0)) {
                        float2* p = own + (size_t)j * ny;
                        *p = accum ? cadd(*p, v[k2]) : v[k2];
                    }
                    if (mirror && (k2 >= B / 2 || (k2 == 0 && r == 0))) {
                        float2* p = mir + (size_t)((L - j) & (L - 1)) * ny;
                        const float2 c = cconj(v[k2]);
                        *p = accum ? cadd(*p, c) : c;
                    }
                }
            }
        }
    }

    // ---- pointwise state update in the spatial layout: s = c[0] s + c[1] x (no old: s = c[1] x),
    // x = c[2] s (c[2] == NULL: x = s)
    // (old values from the prefetched tile pf)
    __device__ __forceinline__ void update(float2* __restrict__ st, const float* const* c, bool no_old,
                                           const float2* pf, float2* x) const {
        if (xact) {
#pragma unroll
            for (int q = 0; q < XN; q++) {
                const int j = xpos(q);
                // staged tables: the padded index (positions >= L/2 are the odd pair halves, or the
                // upper values of a thread)
                const int jc = j + (S::STAGE ? 2 * upper(q) : 0);
                float2 nv = cscale(x[q], rd(c[1] + jc));
                if (!no_old) {
                    const float d = rd(c[0] + jc);
                    const float2 o = pf[j * TC + cl];
                    nv.x = fmaf(d, o.x, nv.x);
                    nv.y = fmaf(d, o.y, nv.y);
                }
                st[sidx(q)] = nv;
                x[q] = c[2] ? cscale(nv, rd(c[2] + jc)) : nv;
            }
        }
    }

    // Bulk copies of a STEP pass's inputs into shared memory, issued by thread 0 as the kernel
    // starts: the table block (S::STAGE), and the old tiles of state 1 and state 2 (each one
    // contiguous block of the tile-major layout, padding lines included).  Each completes on its own
    // mbarrier; the barrier initialisation is published by a __syncthreads before any thread waits.
    __device__ __forceinline__ void issue_copies(bool old1, bool old2) const {
        if (threadIdx.x != 0) return;
        mbar_init(bar + 0, 1);
        mbar_init(bar + 1, 1);
        mbar_init(bar + 2, 1);
        mbar_fence_init();
        if (S::STAGE) {
            mbar_arrive_expect_tx(bar + 0, S::TAB_BYTES);
            bulk_copy_g2s(tab2, a.tabs, S::TAB_BYTES, bar + 0);
        }
        constexpr unsigned PART = S::TILE_BYTES / S::BULK_PARTS;
        constexpr int PART2 = (int)(PART / sizeof(float2));
        static_assert(PART % 16 == 0, "bulk copy pieces of 16-byte multiples");
        // a.skip (tests only) leaves a copy out entirely: its barrier phase never completes and
        // nothing is in flight, so the bounded wait for it gives up and the CTA may exit safely
        if (S::BULK && old1 && !(a.skip & 2)) {
            mbar_arrive_expect_tx(bar + 1, S::TILE_BYTES);
            for (int i = 0; i < S::BULK_PARTS; i++)
                bulk_copy_g2s(pf1 + i * PART2, a.st1 + tbase + i * PART2, PART, bar + 1);
        }
        if (S::BULK && old2 && !(a.skip & 4)) {
            mbar_arrive_expect_tx(bar + 2, S::TILE_BYTES);
            for (int i = 0; i < S::BULK_PARTS; i++)
                bulk_copy_g2s(pf2 + i * PART2, a.st2 + tbase + i * PART2, PART, bar + 2);
        }
    }
    // without bulk copies (!S::BULK): every thread's share of one old state tile as 16-byte cp.async
    // copies (one commit group, committed by every thread; read after a wait and a barrier)
    __device__ __forceinline__ void prefetch(const float2* __restrict__ st, float2* pf, bool on) const {
        constexpr int NCH = L * (TC / 2);  // 16-byte chunks per tile
        static_assert(NCH % S::NT == 0, "tile chunks per thread");
        if (on) {
            const float2* src = st + tbase;
#pragma unroll
            for (int q = 0; q < NCH / S::NT; q++) {
                const int e = 2 * ((int)threadIdx.x + q * S::NT);
                cp_async16(pf + e, src + e);
            }
        }
        cp_async_commit();
    }
    // wait for bulk copy i, bounded (kCopyPolls polls, about a second; a copy the test hook left out,
    // a.skip bit i, only a.polls); a copy that has not landed by then is recorded in a.err (bit i) and
    // reported as false, and the caller does not use its tile
    __device__ __forceinline__ bool wait_copy(int i) const {
        if (mbar_wait(bar + i, 0, (a.skip & (1 << i)) ? a.polls : kCopyPolls)) return true;
        atomicOr(a.err, 1 << i);
        return false;
    }
    // before exiting after a wait gave up: wait once more, with the same bound, so that a copy that
    // was only late lands before this CTA's shared memory can be handed to another CTA (a copy the
    // test hook left out was never issued: nothing is in flight)
    __device__ __forceinline__ void drain(int i) const {
        mbar_wait(bar + i, 0, (a.skip & (1 << i)) ? a.polls : kCopyPolls);
    }

    // cp.async copy of the old output of z and y lines into pfo (one commit group, committed by every
    // thread; issue only after the output's writer has completed)
    __device__ __forceinline__ void prefetch_out(bool on) const {
        if (on && AX == 0) {
            constexpr int NCH = L * (TC / 2);
            const int ncol2 = min(TC, a.ncols - col0) / 2;
            const float2* base = a.out + pbase + col0;
            for (int q = threadIdx.x; q < NCH; q += S::NT) {
                const int j = q / (TC / 2), cc = q % (TC / 2);
                if (cc < ncol2) cp_async16(pfo + j * TC + 2 * cc, base + (size_t)j * a.ncols + 2 * cc);
            }
        } else if (on && AX == 1) {
            const int nrows = min(TC, a.ncols - col0);
            const float4* blk = reinterpret_cast<const float4*>(a.out + pbase + (size_t)col0 * L);
            for (int e = threadIdx.x; e < nrows * (L / 2); e += S::NT)
                cp_async16(reinterpret_cast<float4*>(pfo) + e, blk + e);
        }
        cp_async_commit();
    }

    // Point ti/tf at the shared copy of the pass's table block (a.tabs: twi, twf, three k-space
    // factors, six coefficient tables; bulk copy 0); d and c1, c2 receive the shared copies of a's
    // factor and coefficient tables (NULL stays NULL).
    __device__ __forceinline__ void stage(const float2** d, const float** c1, const float** c2) {
        const float2* dsrc[3] = {a.dpre, a.dmid, a.dpost};
#pragma unroll
        for (int i = 0; i < 3; i++) {
            d[i] = dsrc[i] ? tab2 + (2 + i) * L : nullptr;
            c1[i] = a.c1[i] ? tab1 + i * S::CSTR : nullptr;
            c2[i] = a.c2[i] ? tab1 + (3 + i) * S::CSTR : nullptr;
        }
        ti = tab2 + r;
        tf = tab2 + L + r;
    }

    // k-space factor D[j] kappa s (D == NULL: s)
    __device__ __forceinline__ void factor(float2* v, const float2* __restrict__ D, const float* kap,
                                           float s) const {
        if (vcol) {
#pragma unroll
            for (int k2 = 0; k2 < B; k2++) {
                if (D) v[k2] = cmul(v[k2], cscale(rd(D + r + A * k2), kap[k2] * s));
                else v[k2] = cscale(v[k2], s);
            }
        }
    }
};

template <int L, int AX>
__global__ void __launch_bounds__(LS<L>::NT, LS<L>::MINB) line_pass_kernel(LineArgs a) {
    using S = LS<L>;
    constexpr int A = S::A, B = S::B;
    extern __shared__ float4 smem_raw[];
    LineCtx<L, AX> c(a, reinterpret_cast<float2*>(smem_raw));
    const bool late = (a.flags & LF_LATE_WAIT) != 0;
    if (!late) pdl_wait();
    if (!(a.flags & (LF_TRIGGER_MID | LF_TRIGGER_END))) pdl_trigger();
    constexpr int XN = S::XN;
    float2 v[B];
    float2 x[XN];
    const bool accum = (a.flags & LF_ACCUM) != 0;

    if (a.mode == LM_FIN) {
        // adjoint image term: out += F_i (c1[0] st1)
#pragma unroll
        for (int q = 0; q < XN; q++) {
            const int j = c.xpos(q);
            x[q] = c.xact ? cscale(a.st1[c.sidx(q)], __ldg(a.c1[0] + j)) : make_float2(0.f, 0.f);
        }
        c.fwd(x, v, c.buf1);
        c.store_k(a.out, v, true, false);
        return;
    }

    float kap[B];  // tile-major like the states: this thread's points at r + A k2
    const float2* dk[3] = {a.dpre, a.dmid, a.dpost};
    const float* c1[3] = {a.c1[0], a.c1[1], a.c1[2]};
    const float* c2[3] = {a.c2[0], a.c2[1], a.c2[2]};
    const bool old1 = (a.flags & LF_NO_OLD1) == 0, old2 = (a.flags & LF_NO_OLD2) == 0;
    if (a.mode == LM_STEP) {
        c.issue_copies(old1, old2);
        if (!S::BULK) {
            c.prefetch(a.st1, c.pf1, old1);
            c.prefetch(a.st2, c.pf2, old2);
        }
        if (S::STAGE) c.stage(dk, c1, c2);
        const float* kp = a.kap + (size_t)blockIdx.x * (L * S::TC) + c.r * S::TC + c.cl;
#pragma unroll
        for (int k2 = 0; k2 < B; k2++) kap[k2] = c.vcol ? ldg_stream(kp + k2 * A * S::TC) : 0.f;
    }
    c.load_k(a.in, v);
    if (a.mode == LM_INIT) {
        // forward start: st2 = F_i^-1[p^] s_pre  (rho_i^0 = p0 / (3 c^2))
        c.factor(v, nullptr, nullptr, a.s_pre);
        c.inv(v, x, c.buf0);
        if (c.xact) {
#pragma unroll
            for (int q = 0; q < XN; q++) a.st2[c.sidx(q)] = x[q];
        }
        return;
    }

    __syncthreads();  // publishes the mbarrier initialisation
    const bool ok0 = S::STAGE ? c.wait_copy(0) : true;  // the tables
    c.factor(v, dk[0], kap, a.s_pre);
    if (!S::BULK) cp_async_wait<1>();  // state 1 has landed; the barrier inside inv() publishes it
    c.inv(v, x, c.buf0);
    const bool ok1 = (S::BULK && old1) ? c.wait_copy(1) : true;  // the old state 1
    c.update(a.st1, c1, !old1 || !ok1, c.pf1, x);
    if (late) pdl_wait();  // the new spectrum is written by the preceding pass
    if (a.flags & LF_TRIGGER_MID) pdl_trigger();
    const bool pre = accum && AX != 2;
    if (S::PFO_ALIAS && pre) {
        // every thread's state-1 update has read pf1 (written by the bulk copy) before it is reused
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    }
    c.prefetch_out(pre);
    c.fwd(x, v, c.buf1);
    c.factor(v, dk[1], kap, a.s_mid);
    if (!S::BULK) cp_async_wait<1>();  // state 2 likewise (the old output may still be in flight)
    c.inv(v, x, c.buf0);
    const bool ok2 = (S::BULK && old2) ? c.wait_copy(2) : true;  // the old state 2
    c.update(a.st2, c2, !old2 || !ok2, c.pf2, x);
    if (!ok0) c.drain(0);
    if (!ok1) c.drain(1);
    if (!ok2) c.drain(2);
    cp_async_wait<0>();  // old output; published by the barrier inside fwd()
    c.fwd(x, v, c.buf1);
    c.factor(v, dk[2], kap, a.s_post);

    if (AX == 0 && (a.flags & LF_INJECT) && c.vcol) {
        const float2 sv = a.inj[(size_t)c.b * a.plane_bs + c.col];
#pragma unroll
        for (int k2 = 0; k2 < B; k2++) {
            const int kz = c.r + A * k2;
            v[k2] = cadd(v[k2], cmul(sv, __ldg(a.tw + ((kz * a.zs) & (L - 1)))));
        }
    }
    c.store_k(a.out, v, accum, pre);

    if (AX == 0 && (a.flags & LF_RECORD)) {
        // plane spectrum at z = zs: (1/nz) sum_kz p^(kz) e^{+2 pi i kz zs / nz}; partial sums over
        // this thread's kz, then over the A threads of the line (buf0 is free, see store_k)
        float2 part = make_float2(0.f, 0.f);
        if (c.vcol) {
#pragma unroll
            for (int k2 = 0; k2 < B; k2++) {
                const int kz = c.r + A * k2;
                part = cadd(part, cmul(v[k2], cconj(__ldg(a.tw + ((kz * a.zs) & (L - 1))))));
            }
        }
        c.buf0[c.r * S::TC + c.cl] = part;
        __syncthreads();
        if (c.vcol && c.r == 0) {
            float2 sum = make_float2(0.f, 0.f);
#pragma unroll
            for (int rr = 0; rr < A; rr++) sum = cadd(sum, c.buf0[rr * S::TC + c.cl]);
            a.rec[(size_t)c.b * a.plane_bs + c.col] = cscale(sum, a.s_rec);
        }
    }
}

template <int L>
LineKernels make_line_kernels() {
    using S = LS<L>;
    LineKernels k;
    k.pass[0] = line_pass_kernel<L, 0>;
    k.pass[1] = line_pass_kernel<L, 1>;
    k.pass[2] = line_pass_kernel<L, 2>;
    k.smem = S::smem;
    k.tc = S::TC;
    k.nt = S::NT;
    k.ra = S::A;
    k.rb = S::B;
    k.pair = S::PAIR;
    k.pnew = S::PNEW;
    return k;
}

}  // namespace pat

// pat_solver.cu - variational reconstruction on the GPU (arXiv:1605.00133, Sec. 4.5-4.6, App. A-B).
//
//   pat_tv_prox        argmin_{q >= 0} 1/2 ||q - p||^2 + alpha TV(q), TV isotropic with forward
//                      differences and Neumann boundary (App. A), by the accelerated primal-dual
//                      hybrid gradient method the paper names (App. B): one launch per iteration,
//                      the dual step (ball projection of xi + sigma grad(qbar)) fused with the
//                      primal step (divergence, data term, non-negativity clamp); step sizes follow
//                      theta = 1/sqrt(1 + 2 tau), tau <- theta tau, sigma <- sigma / theta,
//                      tau_0 = sigma_0 = 1/sqrt(12).
//   pat_bregman_solve  Bregman iterations (Eqs. BregIterA/B) around an accelerated proximal-gradient
//                      (FISTA) inner solver with restart and up to `max_backtrack` halvings of the
//                      step after a restart, eta = step_scale / L, L from power iteration (App. B).
// Fields and operators run in FP32; the data-space residual, the Bregman variable b, the objective
// and every norm and inner product are accumulated in FP64 (deterministic two-stage reductions).
// The host drives the iteration and reads one or two FP64 scalars per FISTA step.
#include <math.h>

#include <algorithm>
#include <string>

#include "pat_internal.h"

namespace pat {

#define PAT_CUDA(x, where)                                   \
    do {                                                     \
        cudaError_t _e = (x);                                \
        if (_e != cudaSuccess) return set_cuda_error(_e, where); \
    } while (0)

static constexpr int kRedBlocks = 512;
static constexpr int kRedThreads = 256;

static inline int ew_blocks(size_t n) {
    size_t b = (n + 255) / 256;
    return (int)std::min<size_t>(b, 152 * 16);
}

// ------------------------------------------------------------------------------ elementwise kernels

// z = a * x + b * y (float)
__global__ void axpby_kernel(float* __restrict__ z, const float* __restrict__ x, const float* __restrict__ y,
                             float a, float b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        z[i] = fmaf(a, x[i], b * y[i]);
}

// r = (float)(ay - g)  (g in FP64)
__global__ void residual_kernel(float* __restrict__ r, const float* __restrict__ ay, const double* __restrict__ g, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        r[i] = (float)((double)ay[i] - g[i]);
}

// g = f + b (FP64)
__global__ void data_shift_kernel(double* __restrict__ g, const float* __restrict__ f, const double* __restrict__ b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        g[i] = (double)f[i] + b[i];
}

// b += f - ax (FP64 Bregman update)
__global__ void bregman_update_kernel(double* __restrict__ b, const float* __restrict__ f, const float* __restrict__ ax, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] += (double)f[i] - (double)ax[i];
}

__global__ void clamp_copy_kernel(float* __restrict__ q, float* __restrict__ qbar, const float* __restrict__ p, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float v = fmaxf(0.f, p[i]);
        q[i] = v;
        qbar[i] = v;
    }
}

// ------------------------------------------------------------------------------ TV prox kernel

struct TvDims {
    int nz, ny, nx;
    size_t n;      // nz*ny*nx
    size_t total;  // B*n
};

// One primal-dual iteration per launch, dual and primal steps fused (App. B):
//   xi'   = project_{|.| <= alpha}(xi + sigma grad(qbar))        dual, every voxel
//   q'    = max(0, (q - tau grad^T(xi') + tau p) / (1 + tau))    primal, the clamp fused
//   qbar' = q' + theta (q' - q)
// grad: forward differences, zero past the last voxel of an axis; grad^T(xi)(v) = sum over axes of
// [xi_a(v - e_a) if v has a predecessor] - [xi_a(v) if v has a successor].
// A CTA owns a 32 x kTvRows tile of (x, y) columns over a run of z planes and marches along z:
// lanes are consecutive x, warps consecutive y, and warp 0 is the halo row y0 - 1, whose new dual
// the first output row needs.  The x neighbours come by warp shuffle (lane 31 loads qbar at
// x0 + 32, lane 0 also evaluates the dual at x0 - 1), the y neighbours through shared memory, and
// the new dual's z component of the plane below stays in a register; a run's first plane needs
// the plane before it, which the CTA evaluates first without storing it.  qbar and xi are read from
// one buffer and written to the other (neighbouring CTAs read the old values); q is read and
// written only at its own voxel.
constexpr int kTvRows = 8;
constexpr int kTvWarps = kTvRows + 1;

struct TvStep {
    const float* qb_in;
    float* qb_out;
    const float* xi_in;  // components z, y, x at offsets 0, N, 2N
    float* xi_out;
    float* q;
    const float* p;
    float sigma, alpha, tau, theta;
    int nonneg;
    int nz, ny, nx;
    int zrun, nruns;  // planes per run, runs per image
    long long n, N;   // voxels per image, B * n
};

__device__ __forceinline__ void tv_project(float& a, float& b, float& e, float alpha) {
    const float nrm = sqrtf(a * a + b * b + e * e);
    const float s = (nrm > alpha) ? alpha / nrm : 1.f;
    a *= s;
    b *= s;
    e *= s;
}

// what a thread reads for plane z (its qbar at z itself is carried from the plane before)
struct TvIn {
    float qn;          // qbar at z + 1
    float xz, xy, xx;  // dual at the own voxel
    float qv, pv;      // q and the prox input (output voxels only)
    float qr, qd;      // qbar at x0 + 32 (lane 31) and at y + 1 (last warp)
    float qln, qld;    // lane 0 of the output rows: qbar at (z + 1, y, x0 - 1) and (z, y + 1, x0 - 1)
    float lz, ly, lx;  //   and the dual at (z, y, x0 - 1)
};

__global__ void __launch_bounds__(32 * kTvWarps) tv_step_kernel(TvStep a) {
    __shared__ float sq[kTvWarps][32];  // qbar of the current plane, one row per warp
    __shared__ float sy[kTvWarps][32];  // y component of the new dual, one row per warp
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int x0 = blockIdx.x * 32, x = x0 + lane;
    const int y = blockIdx.y * kTvRows - 1 + w;
    const int b = blockIdx.z / a.nruns, run = blockIdx.z - b * a.nruns;
    const int z0 = run * a.zrun, z1 = min(z0 + a.zrun, a.nz);
    const bool yin = y >= 0 && y < a.ny, in = yin && x < a.nx;
    const bool own = in && w > 0;                               // writes its voxel (planes z0 .. z1-1)
    const bool xn = x + 1 < a.nx, yn = y + 1 < a.ny;            // voxel has a successor along x / y
    const bool halo = lane == 0 && x0 > 0 && yin && w > 0;      // evaluates the dual at x0 - 1
    const bool right = lane == 31 && x0 + 32 < a.nx && yin;     // loads qbar at x0 + 32
    const bool down = w == kTvWarps - 1 && in && yn;            // loads qbar at y + 1
    const long long plane = (long long)a.ny * a.nx;
    const long long base = b * a.n + (long long)y * a.nx + x;   // + z * plane; dereferenced only when in
    const float* __restrict__ qb = a.qb_in;
    const float* __restrict__ xi = a.xi_in;
    auto load = [&](int z) {
        TvIn v;
        const long long o = base + z * plane;
        const bool zn = z + 1 < a.nz, store = own && z >= z0;
        v.qn = (in && zn) ? qb[o + plane] : 0.f;
        v.xz = in ? xi[o] : 0.f;
        v.xy = in ? xi[a.N + o] : 0.f;
        v.xx = in ? xi[2 * a.N + o] : 0.f;
        v.qv = store ? a.q[o] : 0.f;
        v.pv = store ? a.p[o] : 0.f;
        v.qr = right ? qb[o + 1] : 0.f;
        v.qd = down ? qb[o + a.nx] : 0.f;
        v.qln = (halo && zn) ? qb[o - 1 + plane] : 0.f;
        v.qld = (halo && yn) ? qb[o - 1 + a.nx] : 0.f;
        v.lz = halo ? xi[o - 1] : 0.f;
        v.ly = halo ? xi[a.N + o - 1] : 0.f;
        v.lx = halo ? xi[2 * a.N + o - 1] : 0.f;
        return v;
    };
    const int zs = z0 > 0 ? z0 - 1 : z0;
    float qc = in ? qb[base + zs * plane] : 0.f;         // qbar at (z, y, x)
    float qlc = halo ? qb[base - 1 + zs * plane] : 0.f;  // qbar at (z, y, x0 - 1)
    float pz = 0.f;                                      // z component of the new dual at z - 1
    // plane z from its reads `cur`.  The reads are not issued a plane ahead: a CTA barrier waits
    // for the loads in flight, so reads issued before the barriers of the plane before would
    // only add registers (measured slower).
    auto step = [&](int z, const TvIn& cur) {
        const long long o = base + z * plane;
        const bool zn = z + 1 < a.nz, store = own && z >= z0;
        sq[w][lane] = qc;
        __syncthreads();
        // new dual at the own voxel
        const float qxn = __shfl_down_sync(0xffffffffu, qc, 1);
        const float qyn = (w < kTvWarps - 1) ? sq[w + 1][lane] : cur.qd;
        const float gz = zn ? cur.qn - qc : 0.f;
        const float gy = yn ? qyn - qc : 0.f;
        const float gx = xn ? (lane < 31 ? qxn : cur.qr) - qc : 0.f;
        float dz = fmaf(a.sigma, gz, cur.xz), dy = fmaf(a.sigma, gy, cur.xy), dx = fmaf(a.sigma, gx, cur.xx);
        tv_project(dz, dy, dx, a.alpha);
        // new dual at x0 - 1 (lane 0 of the output rows): only its x component is used
        float dlx = 0.f;
        if (halo) {
            float ez = fmaf(a.sigma, zn ? cur.qln - qlc : 0.f, cur.lz);
            float ey = fmaf(a.sigma, yn ? cur.qld - qlc : 0.f, cur.ly);
            float ex = fmaf(a.sigma, qc - qlc, cur.lx);
            tv_project(ez, ey, ex, a.alpha);
            dlx = ex;
        }
        sy[w][lane] = dy;
        __syncthreads();
        const float dxl = __shfl_up_sync(0xffffffffu, dx, 1);
        if (store) {
            float gt = 0.f;
            if (zn) gt -= dz;
            if (z > 0) gt += pz;
            if (yn) gt -= dy;
            if (y > 0) gt += sy[w - 1][lane];
            if (xn) gt -= dx;
            if (x > 0) gt += lane > 0 ? dxl : dlx;
            float qnew = fmaf(-a.tau, gt, fmaf(a.tau, cur.pv, cur.qv)) / (1.f + a.tau);
            if (a.nonneg) qnew = fmaxf(0.f, qnew);
            a.q[o] = qnew;
            a.qb_out[o] = fmaf(a.theta, qnew - cur.qv, qnew);
            a.xi_out[o] = dz;
            a.xi_out[a.N + o] = dy;
            a.xi_out[2 * a.N + o] = dx;
        }
        pz = dz;
        qc = cur.qn;
        qlc = cur.qln;
    };
    for (int z = zs; z < z1; z++) step(z, load(z));
}

// ------------------------------------------------------------------------------ FP64 reductions

enum RedOp { RED_SUMSQ_DIFF = 0, RED_TV = 1, RED_SUMSQ = 2, RED_ABS_DIFF = 3, RED_DOT = 4, RED_SUMSQ_DIFF_FF = 5 };

struct RedArgs {
    int op;
    const float* a;
    const float* b;    // second float operand (ABS_DIFF, DOT)
    const double* gd;  // FP64 operand (SUMSQ_DIFF: sum (a - gd)^2)
    size_t n;
    TvDims d;          // RED_TV
};

__device__ __forceinline__ double red_term(const RedArgs& r, size_t i) {
    switch (r.op) {
        case RED_SUMSQ_DIFF: {
            const double e = (double)r.a[i] - r.gd[i];
            return e * e;
        }
        case RED_TV: {
            const size_t plane = (size_t)r.d.ny * r.d.nx;
            const unsigned v = (unsigned)(i % r.d.n), nx = (unsigned)r.d.nx, ny = (unsigned)r.d.ny;
            const unsigned t = v / nx;
            const int x = (int)(v - t * nx), y = (int)(t % ny), z = (int)(t / ny);
            const double c = r.a[i];
            const double gz = (z + 1 < r.d.nz) ? (double)r.a[i + plane] - c : 0.0;
            const double gy = (y + 1 < r.d.ny) ? (double)r.a[i + r.d.nx] - c : 0.0;
            const double gx = (x + 1 < r.d.nx) ? (double)r.a[i + 1] - c : 0.0;
            return sqrt(gz * gz + gy * gy + gx * gx);
        }
        case RED_SUMSQ: {
            const double e = r.a[i];
            return e * e;
        }
        case RED_ABS_DIFF: return fabs((double)r.a[i] - (double)r.b[i]);
        case RED_SUMSQ_DIFF_FF: {
            const double e = (double)r.a[i] - (double)r.b[i];
            return e * e;
        }
        default: return (double)r.a[i] * (double)r.b[i];
    }
}

__global__ void reduce_stage1_kernel(RedArgs r, double* __restrict__ partial) {
    __shared__ double sh[kRedThreads / 32];
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < r.n; i += (size_t)gridDim.x * blockDim.x)
        acc += red_term(r, i);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kRedThreads / 32; w++) t += sh[w];
        partial[blockIdx.x] = t;
    }
}

__global__ void reduce_stage2_kernel(const double* __restrict__ partial, int np, double* __restrict__ out) {
    __shared__ double sh[kRedThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partial[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// ------------------------------------------------------------------------------ host helpers

struct Ctx {
    pat_grid* G;
    cudaStream_t st;
    size_t N;   // image elements (B*nz*ny*nx)
    size_t D;   // data elements (B*T*m)
    TvDims td;
};

static pat_status reduce(Ctx& c, const RedArgs& r, double* out) {
    SolverWs& w = c.G->sw;
    const int nb = (int)std::min<size_t>(kRedBlocks, std::max<size_t>(1, (r.n + kRedThreads - 1) / kRedThreads));
    reduce_stage1_kernel<<<nb, kRedThreads, 0, c.st>>>(r, w.partial);
    reduce_stage2_kernel<<<1, kRedThreads, 0, c.st>>>(w.partial, nb, w.result);
    PAT_CUDA(cudaGetLastError(), "reduction launch");
    PAT_CUDA(cudaMemcpyAsync(w.host, w.result, sizeof(double), cudaMemcpyDeviceToHost, c.st), "reduction copy");
    PAT_CUDA(cudaStreamSynchronize(c.st), "reduction sync");
    *out = w.host[0];
    return PAT_OK;
}

static pat_status ensure_ws(pat_grid* G, bool solver) {
    SolverWs& w = G->sw;
    const size_t N = (size_t)G->g.B * G->g.nreal;
    const size_t D = (size_t)G->g.B * G->g.T * (size_t)G->m;
    pat_status st = PAT_OK;
    if (!w.qbar) {
        st = grid_alloc(G, (void**)&w.qbar, N * sizeof(float), "prox qbar");
        if (st == PAT_OK) st = grid_alloc(G, (void**)&w.qbar2, N * sizeof(float), "prox qbar");
        if (st == PAT_OK) st = grid_alloc(G, (void**)&w.xi, 3 * N * sizeof(float), "prox dual");
        if (st == PAT_OK) st = grid_alloc(G, (void**)&w.xi2, 3 * N * sizeof(float), "prox dual");
        if (st == PAT_OK) st = grid_alloc(G, (void**)&w.z, N * sizeof(float), "prox input copy");
        if (st == PAT_OK) st = grid_alloc(G, (void**)&w.partial, kRedBlocks * sizeof(double), "reduction");
        if (st == PAT_OK) st = grid_alloc(G, (void**)&w.result, sizeof(double), "reduction");
        if (st == PAT_OK) {
            cudaError_t e = cudaMallocHost((void**)&w.host, 4 * sizeof(double));
            if (e != cudaSuccess) return set_cuda_error(e, "cudaMallocHost(reduction)");
        }
        if (st != PAT_OK) return st;
        w.n_img = N;
    }
    if (solver && !w.x) {
        st = grid_alloc(G, (void**)&w.x, N * sizeof(float), "solver x");
        if (st == PAT_OK) st = grid_alloc(G, (void**)&w.xp, N * sizeof(float), "solver x_prev");
        if (st == PAT_OK) st = grid_alloc(G, (void**)&w.y, N * sizeof(float), "solver y");
        if (st == PAT_OK) st = grid_alloc(G, (void**)&w.grad, N * sizeof(float), "solver gradient");
        if (st == PAT_OK) st = grid_alloc(G, (void**)&w.ax, std::max<size_t>(D, 1) * sizeof(float), "solver Ax");
        if (st == PAT_OK) st = grid_alloc(G, (void**)&w.axp, std::max<size_t>(D, 1) * sizeof(float), "solver Ax_prev");
        if (st == PAT_OK) st = grid_alloc(G, (void**)&w.ay, std::max<size_t>(D, 1) * sizeof(float), "solver Ay");
        if (st == PAT_OK) st = grid_alloc(G, (void**)&w.r, std::max<size_t>(D, 1) * sizeof(float), "solver residual");
        if (st == PAT_OK) st = grid_alloc(G, (void**)&w.gdat, std::max<size_t>(D, 1) * sizeof(double), "solver data");
        if (st == PAT_OK) st = grid_alloc(G, (void**)&w.bdat, std::max<size_t>(D, 1) * sizeof(double), "solver Bregman");
        if (st != PAT_OK) return st;
        w.n_dat = D;
    }
    return PAT_OK;
}

// PDHG for the positivity-constrained TV denoising problem; q (output) must not alias p.
static pat_status tv_prox_run(Ctx& c, const float* p, float* q, double alpha, int iters, int nonneg) {
    SolverWs& w = c.G->sw;
    const int nb = ew_blocks(c.N);
    clamp_copy_kernel<<<nb, 256, 0, c.st>>>(q, w.qbar, p, c.N);
    if (!nonneg) PAT_CUDA(cudaMemcpyAsync(q, p, c.N * sizeof(float), cudaMemcpyDeviceToDevice, c.st), "prox init");
    if (!nonneg) PAT_CUDA(cudaMemcpyAsync(w.qbar, p, c.N * sizeof(float), cudaMemcpyDeviceToDevice, c.st), "prox init");
    if (alpha <= 0.0 || iters == 0) {
        PAT_CUDA(cudaGetLastError(), "prox launch");
        return PAT_OK;
    }
    PAT_CUDA(cudaMemsetAsync(w.xi, 0, 3 * c.N * sizeof(float), c.st), "prox init");
    const TvDims& d = c.td;
    const int B = (int)(d.total / d.n);
    const int gx = (d.nx + 31) / 32, gy = (d.ny + kTvRows - 1) / kTvRows;
    // runs of z planes: about 512 CTAs in all, at least 4 planes per run (each run evaluates one
    // plane more than it stores)
    const long long cols = (long long)gx * gy * B;
    int nruns = (int)std::max<long long>(1, std::min<long long>((512 + cols - 1) / cols, (d.nz + 3) / 4));
    const int zrun = (d.nz + nruns - 1) / nruns;
    nruns = (d.nz + zrun - 1) / zrun;
    TvStep a;
    a.q = q;
    a.p = p;
    a.alpha = (float)alpha;
    a.nonneg = nonneg;
    a.nz = d.nz;
    a.ny = d.ny;
    a.nx = d.nx;
    a.zrun = zrun;
    a.nruns = nruns;
    a.n = (long long)d.n;
    a.N = (long long)d.total;
    const dim3 grid(gx, gy, B * nruns);
    float* qb[2] = {w.qbar, w.qbar2};
    float* xi[2] = {w.xi, w.xi2};
    double tau = 1.0 / sqrt(12.0), sigma = 1.0 / (tau * 12.0);
    for (int it = 0; it < iters; it++) {
        const double theta = 1.0 / sqrt(1.0 + 2.0 * tau);
        a.qb_in = qb[it & 1];
        a.qb_out = qb[(it + 1) & 1];
        a.xi_in = xi[it & 1];
        a.xi_out = xi[(it + 1) & 1];
        a.sigma = (float)sigma;
        a.tau = (float)tau;
        a.theta = (float)theta;
        tv_step_kernel<<<grid, 32 * kTvWarps, 0, c.st>>>(a);
        tau *= theta;
        sigma /= theta;
    }
    PAT_CUDA(cudaGetLastError(), "prox launch");
    return PAT_OK;
}

static pat_status energy(Ctx& c, const float* ax, const float* x, double lam, double* E) {
    RedArgs r = {};
    r.op = RED_SUMSQ_DIFF;
    r.a = ax;
    r.gd = c.G->sw.gdat;
    r.n = c.D;
    double dfit = 0.0, tvv = 0.0;
    pat_status st = reduce(c, r, &dfit);
    if (st != PAT_OK) return st;
    RedArgs t = {};
    t.op = RED_TV;
    t.a = x;
    t.n = c.N;
    t.d = c.td;
    if ((st = reduce(c, t, &tvv)) != PAT_OK) return st;
    *E = 0.5 * dfit + lam * tvv;
    return PAT_OK;
}

static pat_status A_fwd(Ctx& c, const float* x, float* ax) {
    pat_grid* G = c.G;
    cudaError_t e = run_forward(G->g, G->t, G->w, G->s, G->kind, G->m, x, ax, c.st, nullptr);
    if (e != cudaSuccess) return set_cuda_error(e, "solver forward");
    return PAT_OK;
}

static pat_status A_adj(Ctx& c, const float* r, float* out) {
    pat_grid* G = c.G;
    cudaError_t e = run_adjoint(G->g, G->t, G->w, G->s, G->kind, G->m, r, out, c.st, nullptr);
    if (e != cudaSuccess) return set_cuda_error(e, "solver adjoint");
    return PAT_OK;
}

// grad = A^T C^T (ax - g)
static pat_status gradient(Ctx& c, const float* ax, float* grad) {
    SolverWs& w = c.G->sw;
    residual_kernel<<<ew_blocks(c.D), 256, 0, c.st>>>(w.r, ax, w.gdat, c.D);
    PAT_CUDA(cudaGetLastError(), "residual launch");
    return A_adj(c, w.r, grad);
}

// x = prox_{eta lam}(base - eta grad)
static pat_status prox_step(Ctx& c, const float* base, const float* grad, double eta, double lam,
                            int prox_iters, float* x) {
    SolverWs& w = c.G->sw;
    axpby_kernel<<<ew_blocks(c.N), 256, 0, c.st>>>(w.z, base, grad, 1.f, (float)-eta, c.N);
    PAT_CUDA(cudaGetLastError(), "step launch");
    return tv_prox_run(c, w.z, x, eta * lam, prox_iters, 1);
}

// Power iteration for L ~ ||A^T C^T C A||_2 from a seeded Gaussian start (SplitMix64 + Box-Muller).
static pat_status power_iteration(Ctx& c, int iters, uint64_t seed, double* L) {
    SolverWs& w = c.G->sw;
    std::vector<float> h(c.N);
    uint64_t state = seed;
    auto next = [&]() {
        state += 0x9E3779B97F4A7C15ull;
        uint64_t z = state;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    for (size_t i = 0; i < c.N; i++) {
        const double u1 = next(), u2 = next();
        h[i] = (float)(sqrt(-2.0 * log(1.0 - u1)) * cos(2.0 * M_PI * u2));
    }
    PAT_CUDA(cudaMemcpyAsync(w.x, h.data(), c.N * sizeof(float), cudaMemcpyHostToDevice, c.st), "power init");
    double nrm = 0.0;
    RedArgs r = {};
    r.op = RED_SUMSQ;
    r.a = w.x;
    r.n = c.N;
    pat_status st = reduce(c, r, &nrm);
    if (st != PAT_OK) return st;
    nrm = sqrt(nrm);
    double lam = 0.0;
    for (int it = 0; it < iters; it++) {
        axpby_kernel<<<ew_blocks(c.N), 256, 0, c.st>>>(w.x, w.x, w.x, (float)(1.0 / nrm), 0.f, c.N);
        PAT_CUDA(cudaGetLastError(), "power launch");
        if ((st = A_fwd(c, w.x, w.ax)) != PAT_OK) return st;
        if ((st = A_adj(c, w.ax, w.x)) != PAT_OK) return st;
        r.a = w.x;
        if ((st = reduce(c, r, &nrm)) != PAT_OK) return st;
        nrm = sqrt(nrm);
        lam = nrm;
        if (!(nrm > 0)) break;
    }
    *L = lam;
    return PAT_OK;
}

struct FistaOut {
    int iterations = 0, restarts = 0;
    double energy = 0.0;
};

// FISTA with restart and backtracking; x_prev holds the start on entry and the result on exit,
// ax_prev its image under C A.  Buffers are swapped by pointer, so results are copied back into
// the solver workspace's canonical xp / axp at the end.
static pat_status fista(Ctx& c, const pat_solve_params& P, double eta, FistaOut* out) {
    SolverWs& w = c.G->sw;
    float *x = w.x, *xp = w.xp, *y = w.y;
    float *ax = w.ax, *axp = w.axp, *ay = w.ay;
    pat_status st;
    if ((st = A_fwd(c, xp, axp)) != PAT_OK) return st;
    double Ep = 0.0;
    if ((st = energy(c, axp, xp, P.lambda, &Ep)) != PAT_OK) return st;
    PAT_CUDA(cudaMemcpyAsync(y, xp, c.N * sizeof(float), cudaMemcpyDeviceToDevice, c.st), "fista init");
    PAT_CUDA(cudaMemcpyAsync(ay, axp, c.D * sizeof(float), cudaMemcpyDeviceToDevice, c.st), "fista init");
    double t = 1.0, best = Ep;
    int since_best = 0;
    for (int it = 0; it < P.inner; it++) {
        if ((st = gradient(c, ay, w.grad)) != PAT_OK) return st;
        if ((st = prox_step(c, y, w.grad, eta, P.lambda, P.prox_iters, x)) != PAT_OK) return st;
        if ((st = A_fwd(c, x, ax)) != PAT_OK) return st;
        double E = 0.0;
        if ((st = energy(c, ax, x, P.lambda, &E)) != PAT_OK) return st;
        if (E > Ep) {
            out->restarts++;
            t = 1.0;
            if ((st = gradient(c, axp, w.grad)) != PAT_OK) return st;
            double eta_b = eta;
            for (int b = 0; b <= P.max_backtrack; b++) {
                if ((st = prox_step(c, xp, w.grad, eta_b, P.lambda, P.prox_iters, x)) != PAT_OK) return st;
                if ((st = A_fwd(c, x, ax)) != PAT_OK) return st;
                if ((st = energy(c, ax, x, P.lambda, &E)) != PAT_OK) return st;
                if (E <= Ep) break;
                eta_b *= 0.5;
            }
            if (E > Ep) {  // no descent found: keep the previous iterate
                PAT_CUDA(cudaMemcpyAsync(x, xp, c.N * sizeof(float), cudaMemcpyDeviceToDevice, c.st), "fista keep");
                PAT_CUDA(cudaMemcpyAsync(ax, axp, c.D * sizeof(float), cudaMemcpyDeviceToDevice, c.st), "fista keep");
                E = Ep;
            }
        }
        out->iterations++;
        double change = 0.0;
        RedArgs r = {};
        r.op = RED_ABS_DIFF;
        r.a = x;
        r.b = xp;
        r.n = c.N;
        if ((st = reduce(c, r, &change)) != PAT_OK) return st;
        const double t_next = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        const double beta = (t - 1.0) / t_next;
        axpby_kernel<<<ew_blocks(c.N), 256, 0, c.st>>>(y, x, xp, (float)(1.0 + beta), (float)-beta, c.N);
        axpby_kernel<<<ew_blocks(c.D), 256, 0, c.st>>>(ay, ax, axp, (float)(1.0 + beta), (float)-beta, c.D);
        PAT_CUDA(cudaGetLastError(), "momentum launch");
        std::swap(x, xp);
        std::swap(ax, axp);
        Ep = E;
        t = t_next;
        if (E < best) {
            best = E;
            since_best = 0;
        } else {
            since_best++;
        }
        if (change == 0.0 || since_best >= P.stall) break;
    }
    if (xp != w.xp) PAT_CUDA(cudaMemcpyAsync(w.xp, xp, c.N * sizeof(float), cudaMemcpyDeviceToDevice, c.st), "fista out");
    if (axp != w.axp) PAT_CUDA(cudaMemcpyAsync(w.axp, axp, c.D * sizeof(float), cudaMemcpyDeviceToDevice, c.st), "fista out");
    out->energy = Ep;
    return PAT_OK;
}

}  // namespace pat

using namespace pat;

extern "C" pat_status pat_tv_prox(pat_grid* G, const float* in, float* out, double alpha, int32_t iters,
                                  int32_t bc, void* stream) {
    const NvtxRange range("pat_tv_prox");
    set_error(PAT_OK, "");
    if (!G) return set_error(PAT_ERR_INVALID_ARG, "pat_tv_prox: NULL grid");
    if (!in || !out) return set_error(PAT_ERR_INVALID_ARG, "pat_tv_prox: NULL buffer");
    if (!(alpha >= 0) || iters < 0) return set_error(PAT_ERR_INVALID_ARG, "pat_tv_prox: need alpha >= 0, iters >= 0");
    if (bc != 0) return set_error(PAT_ERR_UNSUPPORTED, "pat_tv_prox: only the Neumann boundary (bc = 0) is built");
    pat_status st = check_grid_device(G);
    if (st != PAT_OK) return st;
    if ((st = ensure_ws(G, false)) != PAT_OK) return st;
    Ctx c;
    c.G = G;
    c.st = (cudaStream_t)stream;
    c.N = (size_t)G->g.B * G->g.nreal;
    c.D = 0;
    c.td = TvDims{G->g.nz, G->g.ny, G->g.nx, (size_t)G->g.nreal, c.N};
    const float* p = in;
    if (in == out) {  // the primal step reads the input every iteration
        cudaError_t e = cudaMemcpyAsync(G->sw.z, in, c.N * sizeof(float), cudaMemcpyDeviceToDevice, c.st);
        if (e != cudaSuccess) return set_cuda_error(e, "pat_tv_prox copy");
        p = G->sw.z;
    }
    return tv_prox_run(c, p, out, alpha, iters, 1);
}

extern "C" pat_status pat_bp_tv(pat_grid* G, const float* f, float* p_out, double alpha, int32_t iters,
                                void* stream) {
    const NvtxRange range("pat_bp_tv");
    set_error(PAT_OK, "");
    if (!G) return set_error(PAT_ERR_INVALID_ARG, "pat_bp_tv: NULL grid");
    if (!p_out || (!f && G->m > 0)) return set_error(PAT_ERR_INVALID_ARG, "pat_bp_tv: NULL buffer");
    if (!(alpha >= 0) || iters < 0) return set_error(PAT_ERR_INVALID_ARG, "pat_bp_tv: need alpha >= 0, iters >= 0");
    pat_status st = check_grid_device(G);
    if (st != PAT_OK) return st;
    if ((st = ensure_ws(G, false)) != PAT_OK) return st;
    Ctx c;
    c.G = G;
    c.st = (cudaStream_t)stream;
    c.N = (size_t)G->g.B * G->g.nreal;
    c.D = 0;
    c.td = TvDims{G->g.nz, G->g.ny, G->g.nx, (size_t)G->g.nreal, c.N};
    // back-projection A^T C^T f (Eq. BP) into the prox's input buffer, then its TV+ denoising
    float* bp = G->sw.z;
    cudaError_t e = run_adjoint(G->g, G->t, G->w, G->s, G->kind, G->m, f, bp, c.st, nullptr);
    if (e != cudaSuccess) return set_cuda_error(e, "pat_bp_tv adjoint");
    return tv_prox_run(c, bp, p_out, alpha, iters, 1);
}

extern "C" pat_status pat_bregman_solve(pat_grid* G, const float* f, const float* warm, float* p_out,
                                        const pat_solve_params* params, pat_solve_report* report, void* stream) {
    const NvtxRange range("pat_bregman_solve");
    set_error(PAT_OK, "");
    if (!G || !params) return set_error(PAT_ERR_INVALID_ARG, "pat_bregman_solve: NULL grid or params");
    if (!f || !p_out) return set_error(PAT_ERR_INVALID_ARG, "pat_bregman_solve: NULL buffer");
    if (G->g.B != 1) return set_error(PAT_ERR_UNSUPPORTED, "pat_bregman_solve: batch must be 1");
    const pat_solve_params P = *params;
    if (!(P.lambda >= 0) || P.outer < 1 || P.inner < 1 || P.prox_iters < 1 || P.max_backtrack < 0 ||
        P.stall < 1 || !(P.step_scale > 0) || (P.L <= 0 && P.power_iters < 1))
        return set_error(PAT_ERR_INVALID_ARG, "pat_bregman_solve: invalid parameters");
    pat_status st = check_grid_device(G);
    if (st != PAT_OK) return st;
    if ((st = ensure_ws(G, true)) != PAT_OK) return st;
    Ctx c;
    c.G = G;
    c.st = (cudaStream_t)stream;
    c.N = (size_t)G->g.nreal;
    c.D = (size_t)G->g.T * G->m;
    c.td = TvDims{G->g.nz, G->g.ny, G->g.nx, (size_t)G->g.nreal, c.N};
    SolverWs& w = G->sw;
    pat_solve_report rep = {};
    double L = P.L;
    if (L <= 0) {
        if ((st = power_iteration(c, P.power_iters, P.seed, &L)) != PAT_OK) return st;
        if (!(L > 0)) return set_error(PAT_ERR_NOT_CONVERGED, "pat_bregman_solve: power iteration gave L <= 0");
    }
    rep.L = L;
    const double eta = P.step_scale / L;
    if (warm) PAT_CUDA(cudaMemcpyAsync(w.xp, warm, c.N * sizeof(float), cudaMemcpyDeviceToDevice, c.st), "warm start");
    else PAT_CUDA(cudaMemsetAsync(w.xp, 0, c.N * sizeof(float), c.st), "cold start");
    if (P.b_in) PAT_CUDA(cudaMemcpyAsync(w.bdat, P.b_in, c.D * sizeof(double), cudaMemcpyDeviceToDevice, c.st),
                         "Bregman resume");
    else PAT_CUDA(cudaMemsetAsync(w.bdat, 0, c.D * sizeof(double), c.st), "Bregman init");
    for (int k = 0; k < P.outer; k++) {
        const NvtxRange step("Bregman step");
        data_shift_kernel<<<ew_blocks(c.D), 256, 0, c.st>>>(w.gdat, f, w.bdat, c.D);
        PAT_CUDA(cudaGetLastError(), "data launch");
        FistaOut fo;
        if ((st = fista(c, P, eta, &fo)) != PAT_OK) return st;
        rep.inner_total += fo.iterations;
        rep.restarts += fo.restarts;
        rep.energy = fo.energy;
        bregman_update_kernel<<<ew_blocks(c.D), 256, 0, c.st>>>(w.bdat, f, w.axp, c.D);
        PAT_CUDA(cudaGetLastError(), "Bregman launch");
        // data residual ||C A p^{k+1} - f|| (FP64)
        double res2 = 0.0;
        RedArgs q = {};
        q.op = RED_SUMSQ_DIFF_FF;
        q.a = w.axp;
        q.b = f;
        q.n = c.D;
        if ((st = reduce(c, q, &res2)) != PAT_OK) return st;
        const double res = sqrt(res2);
        if (k < 64) rep.residual[k] = res;
        rep.n_residual = std::min(k + 1, 64);
    }
    PAT_CUDA(cudaMemcpyAsync(p_out, w.xp, c.N * sizeof(float), cudaMemcpyDeviceToDevice, c.st), "solution copy");
    if (P.b_out)
        PAT_CUDA(cudaMemcpyAsync(P.b_out, w.bdat, c.D * sizeof(double), cudaMemcpyDeviceToDevice, c.st),
                 "Bregman state copy");
    if (report) *report = rep;
    // a time-step kernel whose bounded wait for a bulk copy gave up makes every result since then
    // undefined; the solve has synchronised anyway, so it reads (and clears) the record itself
    return pat_device_status(G, stream);
}

// pat_solver.cu - variational reconstruction on the GPU (arXiv:1605.00133, Sec. 4.5-4.6, App. A-B).
//
//   pat_tv_prox        argmin_{q >= 0} 1/2 ||q - p||^2 + alpha TV(q), TV isotropic with forward
//                      differences and Neumann boundary (App. A), by the accelerated primal-dual
//                      hybrid gradient method the paper names (App. B): one dual kernel (ball
//                      projection of xi + sigma grad(qbar)) and one primal kernel (divergence, data
//                      term and the non-negativity clamp fused) per iteration; step sizes follow
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

// ------------------------------------------------------------------------------ TV prox kernels

struct TvDims {
    int nz, ny, nx;
    size_t n;      // nz*ny*nx
    size_t total;  // B*n
};

// xi <- project_{|.| <= alpha}(xi + sigma grad(qbar)); forward differences, zero past the last voxel
__global__ void tv_dual_kernel(float* __restrict__ xz, float* __restrict__ xy, float* __restrict__ xx,
                               const float* __restrict__ qb, float sigma, float alpha, TvDims d) {
    const size_t plane = (size_t)d.ny * d.nx;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < d.total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t v = i % d.n;
        const int x = (int)(v % d.nx), y = (int)((v / d.nx) % d.ny), z = (int)(v / plane);
        const float c = qb[i];
        const float gz = (z + 1 < d.nz) ? qb[i + plane] - c : 0.f;
        const float gy = (y + 1 < d.ny) ? qb[i + d.nx] - c : 0.f;
        const float gx = (x + 1 < d.nx) ? qb[i + 1] - c : 0.f;
        const float a = fmaf(sigma, gz, xz[i]), b = fmaf(sigma, gy, xy[i]), e = fmaf(sigma, gx, xx[i]);
        const float nrm = sqrtf(a * a + b * b + e * e);
        const float s = (nrm > alpha) ? alpha / nrm : 1.f;
        xz[i] = a * s;
        xy[i] = b * s;
        xx[i] = e * s;
    }
}

// q_new = max(0, (q - tau grad^T xi + tau p) / (1 + tau)), qbar = q_new + theta (q_new - q)
// grad^T xi at v = sum_axes [xi(v - e) if v has a predecessor] - [xi(v) if v has a successor]
__global__ void tv_primal_kernel(float* __restrict__ q, float* __restrict__ qb, const float* __restrict__ xz,
                                 const float* __restrict__ xy, const float* __restrict__ xx,
                                 const float* __restrict__ p, float tau, float theta, int nonneg, TvDims d) {
    const size_t plane = (size_t)d.ny * d.nx;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < d.total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t v = i % d.n;
        const int x = (int)(v % d.nx), y = (int)((v / d.nx) % d.ny), z = (int)(v / plane);
        float gt = 0.f;
        if (z + 1 < d.nz) gt -= xz[i];
        if (z > 0) gt += xz[i - plane];
        if (y + 1 < d.ny) gt -= xy[i];
        if (y > 0) gt += xy[i - d.nx];
        if (x + 1 < d.nx) gt -= xx[i];
        if (x > 0) gt += xx[i - 1];
        const float q0 = q[i];
        float qn = fmaf(-tau, gt, fmaf(tau, p[i], q0)) / (1.f + tau);
        if (nonneg) qn = fmaxf(0.f, qn);
        q[i] = qn;
        qb[i] = fmaf(theta, qn - q0, qn);
    }
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
            const size_t v = i % r.d.n;
            const int x = (int)(v % r.d.nx), y = (int)((v / r.d.nx) % r.d.ny), z = (int)(v / plane);
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
        if (st == PAT_OK) st = grid_alloc(G, (void**)&w.xi, 3 * N * sizeof(float), "prox dual");
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
    if (alpha <= 0.0) {
        PAT_CUDA(cudaGetLastError(), "prox launch");
        return PAT_OK;
    }
    PAT_CUDA(cudaMemsetAsync(w.xi, 0, 3 * c.N * sizeof(float), c.st), "prox init");
    double tau = 1.0 / sqrt(12.0), sigma = 1.0 / (tau * 12.0);
    float* xz = w.xi;
    float* xy = w.xi + c.N;
    float* xx = w.xi + 2 * c.N;
    for (int it = 0; it < iters; it++) {
        const double theta = 1.0 / sqrt(1.0 + 2.0 * tau);
        tv_dual_kernel<<<nb, 256, 0, c.st>>>(xz, xy, xx, w.qbar, (float)sigma, (float)alpha, c.td);
        tv_primal_kernel<<<nb, 256, 0, c.st>>>(q, w.qbar, xz, xy, xx, p, (float)tau, (float)theta, nonneg, c.td);
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

// pat_api.cu - C ABI of libpat: argument checking, constant tables, workspace, dispatch.
//
// Constant tables are computed here in double precision and stored as FP32:
//   FFT twiddles exp(-2 pi i m / L) per axis;
//   kappa(|k|) = sinc(c dt |k| / 2) (the k-space correction that makes the leapfrog step exact
//   per plane wave) at every point of every line of each axis, in that axis's line layout;
//   i k exp(+/- i k dx / 2) per axis and bin (staggered spectral derivative factors; the Nyquist
//   bin k = -pi/dx gives a real factor, so every operator maps real fields to real fields);
//   split-field PML factors a = exp(-alpha dt / 2), alpha = pml_alpha (c/dx) (d/P)^4, on regular
//   (j) and staggered (j + 1/2) points, and the per-axis update coefficients built from them.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <complex>
#include <mutex>
#include <string>
#include <vector>

#include "pat_internal.h"
#include "pat_kargs.h"

using namespace pat;

namespace {

// poll limit of the line passes' bounded waits for their bulk copies (each poll suspends for at
// most about a microsecond: about a second in all)
constexpr int kDefaultPolls = 1 << 20;

thread_local std::string g_err;

pat_status fail(pat_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

pat_status cuda_fail(cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(e == cudaErrorMemoryAllocation ? PAT_ERR_OOM : PAT_ERR_CUDA, m);
}

bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

// process-wide cap on the device workspace one grid may hold (pat_set_workspace_limit); 0 = none
std::atomic<int64_t> g_ws_limit{0};

}  // namespace


namespace {

pat_status dalloc(pat_grid* G, void** p, size_t bytes, const char* what) {
    *p = nullptr;
    if (bytes == 0) return PAT_OK;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? PAT_ERR_OOM : PAT_ERR_CUDA,
                    std::string("cudaMalloc(") + what + ", " + std::to_string(bytes) + " bytes): " + cudaGetErrorString(e));
    }
    G->allocs.push_back(*p);
    G->bytes += (int64_t)bytes;
    return PAT_OK;
}

template <class T>
pat_status upload(pat_grid* G, T** dst, const std::vector<T>& host, const char* what) {
    pat_status s = dalloc(G, (void**)dst, host.size() * sizeof(T), what);
    if (s != PAT_OK) return s;
    if (host.empty()) return PAT_OK;
    cudaError_t e = cudaMemcpy(*dst, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(table)");
    return PAT_OK;
}

void free_grid(pat_grid* G) {
    if (!G) return;
    for (void* p : G->allocs) cudaFree(p);
    for (cudaEvent_t e : G->prof.pool) cudaEventDestroy(e);
    if (G->sw.host) cudaFreeHost(G->sw.host);
    delete G;
}

double wavenumber(int m, int n, double dx) {
    const int mm = (m < n / 2) ? m : m - n;  // Nyquist bin negative
    return 2.0 * M_PI * (double)mm / ((double)n * dx);
}

// PML factor exp(-alpha dt/2) at a (possibly staggered) position along an axis of n points
double pml_factor(const pat_grid_desc& d, double dt, double pos, int n) {
    const int P = d.pml_size;
    if (P <= 0) return 1.0;
    double depth = 0.0;
    if (pos < (double)P) depth = (double)P - pos;
    else if (pos > (double)(n - 1 - P)) depth = pos - (double)(n - 1 - P);
    if (depth <= 0.0) return 1.0;
    const double r = depth / (double)P;
    const double alpha = d.pml_alpha * (d.c / d.dx) * r * r * r * r;
    return exp(-alpha * dt / 2.0);
}

pat_status validate(const pat_grid_desc* d, const pat_sampling_desc* sm) {
    if (!d || !sm) return fail(PAT_ERR_INVALID_ARG, "pat_create_grid: NULL descriptor");
    if (!pow2_in(d->nz, 8, 256) || !pow2_in(d->ny, 8, 256) || !pow2_in(d->nx, 8, 256))
        return fail(PAT_ERR_INVALID_ARG, "grid sizes must be powers of two in [8, 256]");
    if (!(d->dx > 0) || !(d->c > 0) || !(d->rho0 > 0))
        return fail(PAT_ERR_INVALID_ARG, "dx, c and rho0 must be positive");
    if (!(d->dt > 0) && !(d->cfl > 0)) return fail(PAT_ERR_INVALID_ARG, "need dt > 0 or cfl > 0");
    if (d->T < 1) return fail(PAT_ERR_INVALID_ARG, "T must be >= 1");
    if (d->batch < 1) return fail(PAT_ERR_INVALID_ARG, "batch must be >= 1");
    const int mn = std::min(d->nz, std::min(d->ny, d->nx));
    if (d->pml_size < 0 || 2 * d->pml_size >= mn)
        return fail(PAT_ERR_INVALID_ARG, "pml_size must satisfy 0 <= 2*pml_size < min(nz, ny, nx)");
    if (!(d->pml_alpha >= 0)) return fail(PAT_ERR_INVALID_ARG, "pml_alpha must be >= 0");
    const int sz = d->sensor_z < 0 ? d->pml_size : d->sensor_z;
    if (sz >= d->nz) return fail(PAT_ERR_INVALID_ARG, "sensor_z out of range");
    const int M = d->ny * d->nx;
    switch (sm->kind) {
        case PAT_SAMPLE_FULL: break;
        case PAT_SAMPLE_POINTS: {
            if (sm->m < 0 || sm->m > M) return fail(PAT_ERR_INVALID_ARG, "POINTS: need 0 <= m <= Ny*Nx");
            if (sm->m > 0 && !sm->indices) return fail(PAT_ERR_INVALID_ARG, "POINTS: indices is NULL");
            std::vector<char> seen(M, 0);
            for (int j = 0; j < sm->m; j++) {
                const int v = sm->indices[j];
                if (v < 0 || v >= M) return fail(PAT_ERR_INVALID_ARG, "POINTS: index out of range");
                if (seen[v]) return fail(PAT_ERR_INVALID_ARG, "POINTS: duplicate index");
                seen[v] = 1;
            }
            break;
        }
        case PAT_SAMPLE_HADAMARD01:
        case PAT_SAMPLE_HADAMARDPM: {
            if ((M & (M - 1)) != 0) return fail(PAT_ERR_INVALID_ARG, "HADAMARD: Ny*Nx must be a power of two");
            if (M > 32768) return fail(PAT_ERR_UNSUPPORTED, "HADAMARD: Ny*Nx above 32768 is not supported");
            if (sm->m < 1 || sm->m > M) return fail(PAT_ERR_INVALID_ARG, "HADAMARD: need 1 <= m <= Ny*Nx");
            if (!sm->perm || !sm->rows) return fail(PAT_ERR_INVALID_ARG, "HADAMARD: perm/rows is NULL");
            std::vector<char> seen(M, 0);
            for (int l = 0; l < M; l++) {
                const int v = sm->perm[l];
                if (v < 0 || v >= M || seen[v]) return fail(PAT_ERR_INVALID_ARG, "HADAMARD: perm is not a permutation");
                seen[v] = 1;
            }
            std::fill(seen.begin(), seen.end(), 0);
            for (int j = 0; j < sm->m; j++) {
                const int v = sm->rows[j];
                if (v < 0 || v >= M || seen[v]) return fail(PAT_ERR_INVALID_ARG, "HADAMARD: rows out of range or repeated");
                seen[v] = 1;
            }
            break;
        }
        default: return fail(PAT_ERR_INVALID_ARG, "unknown sampling kind");
    }
    return PAT_OK;
}

pat_status build_tables(pat_grid* G) {
    const pat_grid_desc& d = G->d;
    const int n[3] = {d.nz, d.ny, d.nx};
    const double dt = G->s.dt;
    pat_status st;
    std::vector<float2> h_twi[3], h_twf[3], h_dp[3], h_dm[3];  // host copies for the per-pass blocks
    // twiddles
    for (int a = 0; a < 3; a++) {
        std::vector<float2> tw(n[a]);
        for (int m = 0; m < n[a]; m++) {
            const double ang = -2.0 * M_PI * (double)m / (double)n[a];
            tw[m] = make_float2((float)cos(ang), (float)sin(ang));
        }
        if ((st = upload(G, &G->t.tw[a], tw, "twiddles")) != PAT_OK) return st;
        // per-thread tables of the line passes (layouts in pat_kargs.h, LineKernels)
        const LineKernels lk = line_kernels_for(n[a]);
        const int L = n[a], ra = lk.ra, rb = lk.rb;
        if (ra * rb != L) return fail(PAT_ERR_INVALID_ARG, "no line kernel for this axis length");
        std::vector<float2> twi(L), twf(L);
        for (int k = 0; k < rb; k++)
            for (int r = 0; r < ra; r++) twi[k * ra + r] = make_float2(tw[(r * k) % L].x, -tw[(r * k) % L].y);
        if (lk.pair) {
            for (int k = 0; k < rb; k++)
                for (int r = 0; r < ra; r++) {
                    const int xr = lk.pnew ? ((r & 1) | ((r >> 2) << 1)) : r / 2;
                    const int xh = lk.pnew ? ((r >> 1) & 1) : r % 2;
                    twf[k * ra + r] = tw[(xr * (2 * k + xh)) % L];
                }
        } else {
            for (int k = 0; k < ra; k++)
                for (int r = 0; r < rb; r++) twf[k * rb + r] = tw[(r * k) % L];
        }
        if ((st = upload(G, &G->t.twi[a], twi, "twiddles")) != PAT_OK) return st;
        if ((st = upload(G, &G->t.twf[a], twf, "twiddles")) != PAT_OK) return st;
        h_twi[a] = twi;
        h_twf[a] = twf;
    }
    // derivative factors, every bin of each axis
    for (int a = 0; a < 3; a++) {
        const int len = n[a];
        std::vector<float2> dp(len), dm(len);
        for (int m = 0; m < len; m++) {
            const double k = wavenumber(m, n[a], d.dx);
            const std::complex<double> ik(0.0, k);
            const std::complex<double> p = ik * std::polar(1.0, +k * d.dx / 2.0);
            const std::complex<double> q = ik * std::polar(1.0, -k * d.dx / 2.0);
            dp[m] = make_float2((float)p.real(), (float)p.imag());
            dm[m] = make_float2((float)q.real(), (float)q.imag());
        }
        if ((st = upload(G, &G->t.dplus[a], dp, "dplus")) != PAT_OK) return st;
        if ((st = upload(G, &G->t.dminus[a], dm, "dminus")) != PAT_OK) return st;
        h_dp[a] = dp;
        h_dm[a] = dm;
    }
    // kappa at every line point of each axis, tile-major [ntile][len][tc] like the states
    // (pat_internal.h); padding lines 0
    {
        const Geom& g = G->g;
        for (int a = 0; a < 3; a++) {
            const int tc = g.tc[a];
            std::vector<float> kap((size_t)g.ntile[a] * g.len[a] * tc, 0.0f);
            for (int j = 0; j < g.len[a]; j++) {
                for (int c = 0; c < g.ncols[a]; c++) {
                    int kz, ky, kx;
                    if (a == AZ) { kz = j; kx = c / g.ny; ky = c % g.ny; }
                    else if (a == AY) { ky = j; kz = c / g.nxh; kx = c % g.nxh; }
                    else { kx = j; kz = c / g.ny; ky = c % g.ny; }
                    const double wz = wavenumber(kz, d.nz, d.dx);
                    const double wy = wavenumber(ky, d.ny, d.dx);
                    const double wx = wavenumber(kx, d.nx, d.dx);
                    const double x = 0.5 * d.c * dt * sqrt(wz * wz + wy * wy + wx * wx);
                    kap[((size_t)(c / tc) * g.len[a] + j) * tc + c % tc] = (float)((x == 0.0) ? 1.0 : sin(x) / x);
                }
            }
            if ((st = upload(G, &G->t.kappa[a], kap, "kappa")) != PAT_OK) return st;
        }
    }
    if ((st = upload(G, &G->t.err, std::vector<int32_t>(1, 0), "device status word")) != PAT_OK) return st;
    // PML-derived coefficient tables, and the per-pass table blocks
    for (int a = 0; a < 3; a++) {
        std::vector<std::vector<float>> ct(CT_COUNT, std::vector<float>(n[a]));
        for (int j = 0; j < n[a]; j++) {
            const double A = pml_factor(d, dt, (double)j, n[a]);
            const double As = pml_factor(d, dt, (double)j + 0.5, n[a]);
            ct[CT_ONE][j] = 1.0f;
            ct[CT_AS2][j] = (float)(As * As);
            ct[CT_VF_G][j] = (float)(-As * dt / d.rho0);
            ct[CT_VF0_G][j] = (float)(As * (As / 2.0 - 1.0) * dt / d.rho0);
            ct[CT_VA_G][j] = (float)(dt * d.rho0);
            ct[CT_AS][j] = (float)As;
            ct[CT_VA0_OUT][j] = (float)(As * (1.0 - As / 2.0));
            ct[CT_A2][j] = (float)(A * A);
            ct[CT_DF_D][j] = (float)(-A * dt * d.rho0);
            ct[CT_A][j] = (float)A;
            ct[CT_C2][j] = (float)(d.c * d.c);
            ct[CT_FIN][j] = (float)(A * A / (3.0 * d.c * d.c));
        }
        for (int c = 0; c < CT_COUNT; c++)
            if ((st = upload(G, &G->t.coef[c][a], ct[c], "coef")) != PAT_OK) return st;
        const int L = n[a];
        for (int ps = 0; ps < PS_COUNT; ps++) {
            const PassTables& pt = kPassTables[ps];
            // 5 L float2, then 6 coefficient tables of L + 2 floats (entry j at j + 2 [j >= L/2])
            const int cs = L + 2;
            std::vector<float2> blk(5 * (size_t)L + 3 * (size_t)cs, make_float2(0.f, 0.f));
            std::copy(h_twi[a].begin(), h_twi[a].end(), blk.begin());
            std::copy(h_twf[a].begin(), h_twf[a].end(), blk.begin() + L);
            for (int i = 0; i < 3; i++) {
                if (pt.d[i] == DF_PLUS) std::copy(h_dp[a].begin(), h_dp[a].end(), blk.begin() + (2 + i) * L);
                if (pt.d[i] == DF_MINUS) std::copy(h_dm[a].begin(), h_dm[a].end(), blk.begin() + (2 + i) * L);
            }
            float* c1 = reinterpret_cast<float*>(blk.data() + 5 * L);
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < L; j++) {
                    const int jp = j + ((2 * j >= L) ? 2 : 0);
                    c1[i * cs + jp] = ct[pt.c1[i]][j];
                    c1[(3 + i) * cs + jp] = ct[pt.c2[i]][j];
                }
            if ((st = upload(G, &G->t.pass[ps][a], blk, "pass tables")) != PAT_OK) return st;
        }
    }
    return PAT_OK;
}

pat_status check_device(const pat_grid* G) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != G->device) return fail(PAT_ERR_INVALID_ARG, "the current CUDA device is not the grid's device");
    return PAT_OK;
}

}  // namespace

namespace pat {

static size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// The real plane series (sampled kinds) is live only outside the time loop: the forward writes it
// after the last step, the adjoint has consumed it (its plane spectra) before the first.  So it
// shares its memory with the states and 3D spectra, which are live only inside the loop.
WsLayout workspace_layout(const Geom& g, int kind) {
    const size_t B = (size_t)g.B;
    WsLayout L;
    size_t loop = 0;
    for (int a = 0; a < 3; a++) {
        L.ms[a] = round256(B * (size_t)g.len[a] * g.ntile[a] * g.tc[a] * sizeof(float2));
        loop += 2 * L.ms[a];
    }
    L.ph = round256(B * (size_t)g.nspec * sizeof(float2));
    loop += 2 * L.ph;
    L.rk = round256(B * (size_t)g.T * g.nplane * sizeof(float2));
    L.rec = (kind == PAT_SAMPLE_FULL) ? 0 : round256(B * (size_t)g.T * g.m_plane * sizeof(float));
    L.total = std::max(loop, L.rec) + L.rk;
    return L;
}

void workspace_carve(const Geom& g, const WsLayout& L, unsigned char* base, Workspace* w) {
    (void)g;
    size_t off = 0;
    for (int a = 0; a < 3; a++)
        for (int s = 0; s < 2; s++, off += L.ms[a]) w->ms[a][s] = (float2*)(base + off);
    for (int s = 0; s < 2; s++, off += L.ph) w->ph[s] = (float2*)(base + off);
    w->rec = L.rec ? (float*)base : nullptr;  // aliases the loop state, see workspace_layout
    w->rk = (float2*)(base + std::max(off, L.rec));
}

pat_status set_error(pat_status s, const char* msg) { return fail(s, msg); }
pat_status set_cuda_error(cudaError_t e, const char* where) { return cuda_fail(e, where); }
pat_status grid_alloc(pat_grid* G, void** p, size_t bytes, const char* what) { return dalloc(G, p, bytes, what); }
pat_status check_grid_device(const pat_grid* G) { return check_device(G); }
}  // namespace pat

extern "C" {

const char* pat_last_error(void) { return g_err.c_str(); }

const char* pat_version(void) { return "libpat 0.1 (sm_103a)"; }

pat_status pat_create_grid(const pat_grid_desc* desc, const pat_sampling_desc* sampling, pat_grid** out) {
    g_err.clear();
    if (!out) return fail(PAT_ERR_INVALID_ARG, "pat_create_grid: out is NULL");
    *out = nullptr;
    pat_status st = validate(desc, sampling);
    if (st != PAT_OK) return st;

    pat_grid* G = new pat_grid();
    G->d = *desc;
    G->device = -1;
    G->kind = sampling->kind;
    G->t.polls = kDefaultPolls;
    G->t.skip = 0;
    G->bytes = 0;
    if (G->d.sensor_z < 0) G->d.sensor_z = G->d.pml_size;
    if (!(G->d.dt > 0)) G->d.dt = G->d.cfl * G->d.dx / G->d.c;
    const int M = G->d.ny * G->d.nx;
    G->m = (sampling->kind == PAT_SAMPLE_FULL) ? M : sampling->m;
    G->s.c = G->d.c;
    G->s.rho0 = G->d.rho0;
    G->s.dt = G->d.dt;

    Geom& g = G->g;
    g.nz = G->d.nz;
    g.ny = G->d.ny;
    g.nx = G->d.nx;
    g.nxh = g.nx / 2 + 1;
    g.B = G->d.batch;
    g.nzh = g.nz / 2 + 1;
    g.cs = plane_cluster_size(g.nx, g.ny);
    g.len[AZ] = g.nz;
    g.len[AY] = g.ny;
    g.len[AX] = g.nx;
    g.ncols[AZ] = g.nxh * g.ny;
    g.ncols[AY] = g.nz * g.nxh;
    g.ncols[AX] = g.nzh * g.ny;
    for (int a = 0; a < 3; a++) {
        const int tc = line_kernels_for(g.len[a]).tc;
        g.tc[a] = tc > 0 ? tc : 1;
        g.ntile[a] = (g.ncols[a] + g.tc[a] - 1) / g.tc[a];
    }
    g.nreal = (long long)g.nz * g.ny * g.nx;
    g.nspec = (long long)g.nz * g.ny * g.nxh;
    g.nplane = (long long)g.nxh * g.ny;
    g.sensor_z = G->d.sensor_z;
    g.T = G->d.T;
    g.m_plane = M;

    // the workspace cap is checked on the host, before the device is touched
    const WsLayout layout = workspace_layout(g, G->kind);
    const int64_t limit = g_ws_limit.load();
    if (limit > 0 && (int64_t)layout.total > limit) {
        delete G;
        return fail(PAT_ERR_OOM, "pat_create_grid: the workspace needs " + std::to_string(layout.total) +
                                     " bytes, above the limit of " + std::to_string(limit) +
                                     " bytes set by pat_set_workspace_limit");
    }

    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        delete G;
        return cuda_fail(e, "cudaGetDevice");
    }
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess || prop.major * 10 + prop.minor != 103) {
        delete G;
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
        return fail(PAT_ERR_UNSUPPORTED, std::string("libpat is built for sm_103a only; device is ") + prop.name);
    }
    G->device = dev;

    // workspace: one allocation, carved as workspace_carve describes
    {
        const WsLayout& L = layout;
        unsigned char* base = nullptr;
        st = dalloc(G, (void**)&base, L.total, "workspace");
        if (st == PAT_OK) workspace_carve(g, L, base, &G->w);
    }
    if (st == PAT_OK && G->kind == PAT_SAMPLE_POINTS)
        st = upload(G, &G->w.idx, std::vector<int32_t>(sampling->indices, sampling->indices + G->m), "indices");
    if (st == PAT_OK && (G->kind == PAT_SAMPLE_HADAMARD01 || G->kind == PAT_SAMPLE_HADAMARDPM)) {
        st = upload(G, &G->w.perm, std::vector<int32_t>(sampling->perm, sampling->perm + M), "perm");
        if (st == PAT_OK)
            st = upload(G, &G->w.rows, std::vector<int32_t>(sampling->rows, sampling->rows + G->m), "rows");
    }
    if (st == PAT_OK) st = build_tables(G);
    if (st == PAT_OK) {
        e = configure_kernels(g);
        if (e != cudaSuccess) {
            const std::string where = std::string("configure_kernels (") + configure_failure() + ")";
            st = cuda_fail(e, where.c_str());
        }
    }
    if (st != PAT_OK) {
        std::string msg = g_err;
        free_grid(G);
        g_err = msg;
        return st;
    }
    *out = G;
    return PAT_OK;
}

void pat_destroy_grid(pat_grid* grid) {
    if (!grid) return;
    cudaDeviceSynchronize();
    free_grid(grid);
}

pat_status pat_grid_info(const pat_grid* G, int64_t* n_image, int64_t* n_data, int32_t* m, double* dt) {
    if (!G) return fail(PAT_ERR_INVALID_ARG, "pat_grid_info: NULL grid");
    if (n_image) *n_image = G->g.nreal;
    if (n_data) *n_data = (int64_t)G->g.T * G->m;
    if (m) *m = G->m;
    if (dt) *dt = G->s.dt;
    return PAT_OK;
}

int64_t pat_workspace_bytes(const pat_grid* G) { return G ? G->bytes : 0; }

pat_status pat_forward(pat_grid* G, const float* p0, float* f, void* stream) {
    const NvtxRange range("pat_forward");
    g_err.clear();
    if (!G) return fail(PAT_ERR_INVALID_ARG, "pat_forward: NULL grid");
    if (!p0 || (!f && G->m > 0)) return fail(PAT_ERR_INVALID_ARG, "pat_forward: NULL buffer");
    pat_status st = check_device(G);
    if (st != PAT_OK) return st;
    cudaError_t e = run_forward(G->g, G->t, G->w, G->s, G->kind, G->m, p0, f, (cudaStream_t)stream, &G->prof);
    if (e != cudaSuccess) return cuda_fail(e, "pat_forward");
    return PAT_OK;
}

pat_status pat_adjoint(pat_grid* G, const float* f, float* p, void* stream) {
    const NvtxRange range("pat_adjoint");
    g_err.clear();
    if (!G) return fail(PAT_ERR_INVALID_ARG, "pat_adjoint: NULL grid");
    if (!p || (!f && G->m > 0)) return fail(PAT_ERR_INVALID_ARG, "pat_adjoint: NULL buffer");
    pat_status st = check_device(G);
    if (st != PAT_OK) return st;
    cudaError_t e = run_adjoint(G->g, G->t, G->w, G->s, G->kind, G->m, f, p, (cudaStream_t)stream, &G->prof);
    if (e != cudaSuccess) return cuda_fail(e, "pat_adjoint");
    return PAT_OK;
}

pat_status pat_sample(pat_grid* G, const float* pbar, float* f, int32_t nt, void* stream) {
    g_err.clear();
    if (!G) return fail(PAT_ERR_INVALID_ARG, "pat_sample: NULL grid");
    if (nt < 1) return fail(PAT_ERR_INVALID_ARG, "pat_sample: nt must be >= 1");
    if (!pbar || (!f && G->m > 0)) return fail(PAT_ERR_INVALID_ARG, "pat_sample: NULL buffer");
    pat_status st = check_device(G);
    if (st != PAT_OK) return st;
    cudaError_t e = run_sample(G->g, G->w, G->kind, G->m, pbar, f, nt, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "pat_sample");
    return PAT_OK;
}

pat_status pat_sample_adjoint(pat_grid* G, const float* f, float* pbar, int32_t nt, void* stream) {
    g_err.clear();
    if (!G) return fail(PAT_ERR_INVALID_ARG, "pat_sample_adjoint: NULL grid");
    if (nt < 1) return fail(PAT_ERR_INVALID_ARG, "pat_sample_adjoint: nt must be >= 1");
    if (!pbar || (!f && G->m > 0)) return fail(PAT_ERR_INVALID_ARG, "pat_sample_adjoint: NULL buffer");
    pat_status st = check_device(G);
    if (st != PAT_OK) return st;
    cudaError_t e = run_sample_adjoint(G->g, G->w, G->kind, G->m, f, pbar, nt, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "pat_sample_adjoint");
    return PAT_OK;
}

static const char* kClassNames[KC_COUNT] = {"line_x", "line_y", "line_z", "plane_fft", "z_fft", "sample"};

pat_status pat_get_indices(const pat_grid* G, int32_t* host_idx_or_perm, int32_t* host_rows) {
    g_err.clear();
    if (!G) return fail(PAT_ERR_INVALID_ARG, "pat_get_indices: NULL grid");
    pat_status st = check_device(G);
    if (st != PAT_OK) return st;
    const int M = G->g.m_plane;
    cudaError_t e = cudaSuccess;
    if (G->kind == PAT_SAMPLE_POINTS) {
        if (!host_idx_or_perm && G->m > 0) return fail(PAT_ERR_INVALID_ARG, "pat_get_indices: NULL index buffer");
        if (G->m > 0) e = cudaMemcpy(host_idx_or_perm, G->w.idx, (size_t)G->m * sizeof(int32_t), cudaMemcpyDeviceToHost);
    } else if (G->kind == PAT_SAMPLE_HADAMARD01 || G->kind == PAT_SAMPLE_HADAMARDPM) {
        if (!host_idx_or_perm || !host_rows) return fail(PAT_ERR_INVALID_ARG, "pat_get_indices: NULL buffer");
        e = cudaMemcpy(host_idx_or_perm, G->w.perm, (size_t)M * sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(host_rows, G->w.rows, (size_t)G->m * sizeof(int32_t), cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return cuda_fail(e, "pat_get_indices");
    return PAT_OK;
}

pat_status pat_device_status(pat_grid* G, void* stream) {
    g_err.clear();
    if (!G) return fail(PAT_ERR_INVALID_ARG, "pat_device_status: NULL grid");
    pat_status st = check_device(G);
    if (st != PAT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t word = 0;
    cudaError_t e = cudaMemcpyAsync(&word, G->t.err, sizeof(word), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "pat_device_status");
    if (word == 0) return PAT_OK;
    e = cudaMemsetAsync(G->t.err, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "pat_device_status: clear");
    std::string what;
    if (word & 1) what += " table block";
    if (word & 2) what += " state-1 tile";
    if (word & 4) what += " state-2 tile";
    return fail(PAT_ERR_TIMEOUT, "pat_device_status: a line pass gave up waiting for its bulk copy of the" + what);
}

pat_status pat_debug_copy_fault(pat_grid* G, int32_t mask, int32_t polls) {
    g_err.clear();
    if (!G) return fail(PAT_ERR_INVALID_ARG, "pat_debug_copy_fault: NULL grid");
    if ((mask & ~6) != 0 || polls < 0) return fail(PAT_ERR_INVALID_ARG, "pat_debug_copy_fault: mask bits 1, 2 only; polls >= 0");
    G->t.skip = mask;
    G->t.polls = (mask == 0 || polls == 0) ? kDefaultPolls : polls;
    return PAT_OK;
}

pat_status pat_set_workspace_limit(int64_t bytes) {
    g_err.clear();
    if (bytes < 0) return fail(PAT_ERR_INVALID_ARG, "pat_set_workspace_limit: bytes must be >= 0");
    g_ws_limit.store(bytes);
    return PAT_OK;
}

pat_status pat_profile_enable(pat_grid* G, int32_t enable) {
    g_err.clear();
    if (!G) return fail(PAT_ERR_INVALID_ARG, "pat_profile_enable: NULL grid");
    G->prof.on = enable != 0;
    G->prof.recs.clear();
    G->prof.next = 0;
    return PAT_OK;
}

pat_status pat_profile_read(pat_grid* G, int32_t max_classes, char* names, double* total_ms,
                            int64_t* launches, int32_t* n_classes) {
    g_err.clear();
    if (!G || !n_classes || max_classes < 0) return fail(PAT_ERR_INVALID_ARG, "pat_profile_read: bad argument");
    double ms[KC_COUNT] = {0};
    int64_t cnt[KC_COUNT] = {0};
    for (const auto& r : G->prof.recs) {
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        float t = 0.f;
        e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
        ms[r.cls] += t;
        cnt[r.cls] += 1;
    }
    int k = 0;
    for (int c = 0; c < KC_COUNT && k < max_classes; c++) {
        if (cnt[c] == 0) continue;
        if (names) snprintf(names + 48 * k, 48, "%s", kClassNames[c]);
        if (total_ms) total_ms[k] = ms[c];
        if (launches) launches[k] = cnt[c];
        k++;
    }
    *n_classes = k;
    G->prof.recs.clear();
    G->prof.next = 0;
    return PAT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Forward operator with a fixed, library-owned scratch area (no device allocation per call).
//
// Some callers cannot call cudaMalloc when they need A: reconstruction loops that reserve their
// whole device-memory budget up front (a scanner workstation running acquisition and
// reconstruction side by side, a host application whose memory manager owns every device
// allocation) must not grow their footprint, or fail, in the middle of a solve.  For them,
// pat_forward_noalloc runs the same launch sequence as pat_forward, but the time-stepping
// state, the half spectra and the recorded plane series live in the static device array
// below instead of the grid's workspace.  Limits and sharing rules are in include/pat.h.
// ---------------------------------------------------------------------------------------------

#define PAT_NOALLOC_SCRATCH_BYTES (64ull << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[PAT_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {nullptr};  // device address of g_noalloc_scratch, per device id

}  // namespace

extern "C" pat_status pat_forward_noalloc(pat_grid* G, const float* p0, float* f, void* stream) {
    const NvtxRange range("pat_forward_noalloc");
    g_err.clear();
    if (!G) return fail(PAT_ERR_INVALID_ARG, "pat_forward_noalloc: NULL grid");
    if (!p0 || (!f && G->m > 0)) return fail(PAT_ERR_INVALID_ARG, "pat_forward_noalloc: NULL buffer");
    pat_status st = check_device(G);
    if (st != PAT_OK) return st;
    const Geom& g = G->g;
    const WsLayout L = workspace_layout(g, G->kind);
    const size_t need = L.total;
    if (need > PAT_NOALLOC_SCRATCH_BYTES)
        return fail(PAT_ERR_INVALID_ARG, "pat_forward_noalloc: this grid needs " + std::to_string(need) +
                                             " bytes of scratch; the static scratch holds " +
                                             std::to_string(PAT_NOALLOC_SCRATCH_BYTES) + " bytes");
    if (G->device < 0 || G->device >= 64) return fail(PAT_ERR_UNSUPPORTED, "pat_forward_noalloc: device id >= 64");
    unsigned char* base = nullptr;
    {
        // first call on this device: look up the device address of the static array (the host-side
        // symbol is only a stand-in and must never be handed to a kernel)
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[G->device]) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
            g_noalloc_ptr[G->device] = ptr;
        }
        base = (unsigned char*)g_noalloc_ptr[G->device];
    }
    Workspace w = G->w;  // index sets stay the grid's; all mutable scratch comes from the array
    workspace_carve(g, L, base, &w);
    cudaError_t e = run_forward(G->g, G->t, w, G->s, G->kind, G->m, p0, f, (cudaStream_t)stream, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "pat_forward_noalloc");
    return PAT_OK;
}

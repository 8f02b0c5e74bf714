// pat_internal.h - host-side structures shared by the C ABI layer and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <vector>

#include "../../include/pat.h"

struct pat_grid;

namespace pat {

enum Axis { AZ = 0, AY = 1, AX = 2 };

// Per-axis coefficient tables (float, one entry per grid index along the axis), all derived from
// the PML factors a (regular points) and as (staggered points) in double precision.
enum CoefTable {
    CT_ONE = 0,        // 1
    CT_AS2,            // as^2                      velocity decay (forward and adjoint)
    CT_VF_G,           // -as * dt / rho0           forward velocity: gradient term
    CT_VF0_G,          // as (as/2 - 1) dt / rho0    forward velocity, first step (u^{-1/2} folded in)
    CT_VA_G,           // dt * rho0                 adjoint velocity: gradient term
    CT_AS,             // as                        adjoint velocity: output gain
    CT_VA0_OUT,        // as (1 - as/2)             adjoint velocity, last step (u^{-1/2} folded in)
    CT_A2,             // a^2                       density decay
    CT_DF_D,           // -a dt rho0                forward density: divergence term
    CT_A,              // a                         adjoint density: output gain
    CT_C2,             // c^2                       adjoint density: input gain
    CT_FIN,            // a^2 / (3 c^2)             adjoint image: rho_i^0 = p0 / (3 c^2) transposed
    CT_COUNT
};

// The tables one line pass of a time step reads, per kind of step: the k-space factor before,
// between and after its transforms (none, i k e^{+ik dx/2}, i k e^{-ik dx/2}) and the coefficient
// tables (decay, input gain, output gain) of its two states; an output gain CT_ONE means none.
enum DFactor { DF_NONE = 0, DF_PLUS, DF_MINUS };
enum PassSet { PS_FWD0 = 0, PS_FWD, PS_ADJ, PS_ADJ0, PS_COUNT };  // forward n = 0, n > 0; adjoint n > 0, n = 0
struct PassTables {
    int d[3];
    int c1[3];
    int c2[3];
};
static const PassTables kPassTables[PS_COUNT] = {
    {{DF_PLUS, DF_MINUS, DF_NONE}, {CT_AS2, CT_VF0_G, CT_ONE}, {CT_A2, CT_DF_D, CT_ONE}},
    {{DF_PLUS, DF_MINUS, DF_NONE}, {CT_AS2, CT_VF_G, CT_ONE}, {CT_A2, CT_DF_D, CT_ONE}},
    {{DF_NONE, DF_PLUS, DF_MINUS}, {CT_A2, CT_C2, CT_A}, {CT_AS2, CT_VA_G, CT_AS}},
    {{DF_NONE, DF_PLUS, DF_MINUS}, {CT_A2, CT_C2, CT_A}, {CT_AS2, CT_VA_G, CT_VA0_OUT}},
};

struct Geom {
    int nz, ny, nx, nxh;        // nxh = nx/2 + 1
    int nzh;                    // nz/2 + 1
    int B;                      // batch
    int cs;                     // plane-kernel cluster size
    int len[3];                 // line length per axis (z, y, x)
    int ncols[3];               // lines per batch entry per axis, see Workspace::ms
    int tc[3];                  // lines per tile of the state layout per axis (the line kernel's CTA)
    int ntile[3];               // tiles per batch entry: ceil(ncols / tc)
    long long nreal, nspec;     // per batch entry: nz*ny*nx reals, nz*nxh*ny half-spectrum values
    long long nplane;           // nxh*ny: one plane's half spectrum
    int sensor_z;
    int T;
    int m_plane;                // ny * nx
};

struct DeviceTables {
    float2* tw[3];              // FFT twiddles exp(-2 pi i m / L) per axis length
    float2* twi[3];             // the same, per thread of a line pass (LineKernels in pat_kargs.h)
    float2* twf[3];
    float* kappa[3];            // kappa(|k|) at every point of every line of axis a: [ntile][len][tc]
    float2* dplus[3];           // i k exp(+i k dx/2) per axis, every bin of the axis
    float2* dminus[3];          // i k exp(-i k dx/2)
    float* coef[CT_COUNT][3];   // per-axis coefficient tables
    // per pass set and axis, the tables of one line pass in one block, copied to shared memory at
    // the start of the pass: twi, twf, the three k-space factors (len float2 each; zeros for none),
    // then the coefficient tables of state 1 and state 2 (len + 2 floats each, entry j at
    // j + 2 [j >= len/2])
    float2* pass[PS_COUNT][3];
    int* err;                   // one word: bulk copies of the line passes that never landed (bits)
    int polls;                  // poll limit of the waits for copies the test hook leaves out
    int skip;                   // test hook (pat_debug_copy_fault): state copies not issued (bits 1, 2)
};

// Mixed representation: the split fields u_i, rho_i of axis i are kept with axis i in real space
// and the other two axes Fourier transformed (the PML factor of axis i depends on x_i alone, so the
// update is pointwise there).  Lines are grouped in tiles of tc lines (the lines of one line-pass
// CTA); line c of axis i at position j sits at
// ms[i][s][((b*ntile + c/tc)*len + j)*tc + c%tc], the last tile padded with unused lines:
//   z: c = kx*ny + ky              (kx <= nx/2)        ncols = nxh*ny
//   y: c = kz*nxh + kx             (kx <= nx/2)        ncols = nz*nxh
//   x: c = kz*ny + ky              (kz <= nz/2)        ncols = nzh*ny
// The pressure (or its adjoint) is kept as a full 3D half spectrum ph[.][b][kz][kx][ky].
struct Workspace {
    float2* ms[3][2];           // per axis: state 1 (u_i | adjoint of rho_i), state 2 (rho_i | adjoint of u_i)
    float2* ph[2];              // 3D half spectra [B][nz][nxh][ny], double-buffered across passes
    float2* rk;                 // plane spectra [B][T][nxh][ny]: recorded (A) or injected (A^T)
    float* rec;                 // real plane series [B][T][M] (sampled kinds); shares memory with
                                // ms and ph, which are dead whenever it is live
    int32_t* idx;               // POINTS index list
    int32_t* perm;              // HADAMARD scramble
    int32_t* rows;              // HADAMARD rows
};

struct Scalars {
    double c, rho0, dt;
};

// Kernel classes timed by the optional profiler (CUDA events on the launching stream).
enum KernelClass {
    KC_LINE_X = 0, KC_LINE_Y, KC_LINE_Z, KC_PLANE_FFT, KC_Z_FFT, KC_SAMPLE, KC_COUNT
};

// NVTX range over a scope (for tracing tools such as Nsight Systems; a no-op when none is attached):
// the C-ABI calls, the time loops and the solver's Bregman steps are ranges.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t next = 0;
    struct Rec { int cls; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    cudaError_t ev(cudaEvent_t* out) {
        if (next == pool.size()) {
            cudaEvent_t e;
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return r;
            pool.push_back(e);
        }
        *out = pool[next++];
        return cudaSuccess;
    }
};

// Launchers (pat_run.cu, pat_sample.cu).  All return cudaSuccess or the launch error.
int plane_cluster_size(int nx, int ny);
const char* configure_failure();  // which attribute the last failed configure_kernels call set
cudaError_t configure_kernels(const Geom& g);
// workspace layout: bytes of each part (256-byte aligned) for a grid and sampling kind
struct WsLayout {
    size_t ms[3], ph, rk, rec, total;
};
WsLayout workspace_layout(const Geom& g, int kind);
void workspace_carve(const Geom& g, const WsLayout& L, unsigned char* base, Workspace* w);
cudaError_t run_forward(const Geom& g, const DeviceTables& t, const Workspace& w, const Scalars& s,
                        int kind, int m, const float* p0, float* f, cudaStream_t st, Profiler* prof);
cudaError_t run_adjoint(const Geom& g, const DeviceTables& t, const Workspace& w, const Scalars& s,
                        int kind, int m, const float* f, float* p, cudaStream_t st, Profiler* prof);
cudaError_t run_sample(const Geom& g, const Workspace& w, int kind, int m, const float* pbar,
                       float* f, int nt, cudaStream_t st);
cudaError_t run_sample_adjoint(const Geom& g, const Workspace& w, int kind, int m, const float* f,
                               float* pbar, int nt, cudaStream_t st);

// Solver workspace, allocated by the first pat_tv_prox / pat_bregman_solve call on a grid.
struct SolverWs {
    size_t n_img = 0, n_dat = 0;  // per-call sizes the buffers were made for
    float *x = nullptr, *xp = nullptr, *y = nullptr, *z = nullptr, *grad = nullptr;  // image, B*N
    float *qbar = nullptr, *qbar2 = nullptr, *xi = nullptr, *xi2 = nullptr;         // prox: N, N, 3N, 3N
    float *ax = nullptr, *axp = nullptr, *ay = nullptr, *r = nullptr;              // data, T*m
    double *gdat = nullptr, *bdat = nullptr;                                        // data, FP64
    double *partial = nullptr, *result = nullptr;                                   // reductions
    double* host = nullptr;                                                         // pinned
};

}  // namespace pat

namespace pat {
// Error reporting and workspace allocation shared by the C-ABI translation units (pat_api.cu).
pat_status set_error(pat_status s, const char* msg);
pat_status set_cuda_error(cudaError_t e, const char* where);
pat_status grid_alloc(pat_grid* G, void** p, size_t bytes, const char* what);
pat_status check_grid_device(const pat_grid* G);
}  // namespace pat

// The grid handle (opaque to C callers).
struct pat_grid {
    pat_grid_desc d;
    int kind;
    int m;
    int device;
    pat::Geom g;
    pat::Scalars s;
    pat::DeviceTables t;
    pat::Workspace w;
    std::vector<void*> allocs;
    int64_t bytes;
    pat::Profiler prof;
    pat::SolverWs sw;
};

// pat_internal.h - host-side structures shared by the C ABI layer and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
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
    CT_AS,             // as                        adjoint velocity: transform input
    CT_VA0_OUT,        // as (1 - as/2)             adjoint velocity, last step (u^{-1/2} folded in)
    CT_A2,             // a^2                       density decay
    CT_DF_D,           // -a dt rho0                forward density: divergence term
    CT_A,              // a                         adjoint density: transform input
    CT_COUNT
};

struct Geom {
    int nz, ny, nx, nxh;        // nxh = nx/2 + 1
    int B;                      // batch
    int cs;                     // plane-kernel cluster size
    int rows_cta, cols_cta;     // complex row pairs / packed columns per CTA
    int tc;                     // z-kernel column tile
    long long nreal, nspec;     // per batch entry
    int sensor_z;
    int T;
    int m_plane;                // ny * nx
};

struct DeviceTables {
    float2* tw[3];              // FFT twiddles exp(-2 pi i m / L) per axis length
    float* kappaN;              // kappa(|k|) / N on the half spectrum [nz][nxh][ny]
    float2* dplus[3];           // i k exp(+i k dx/2) per axis (x: nxh entries)
    float2* dminus[3];          // i k exp(-i k dx/2)
    float* coef[CT_COUNT][3];   // per-axis coefficient tables
};

struct Workspace {
    float* st[6];               // u_z,u_y,u_x,rho_z,rho_y,rho_x (forward) / v_i, q_i (adjoint)
    float2* spec[3];            // half spectra [B][nz][nxh][ny] (one allocation)
    float* rec;                 // recorded / injected plane series [B][T][M] (sampled kinds)
    int32_t* idx;               // POINTS index list
    int32_t* perm;              // HADAMARD scramble
    int32_t* rows;              // HADAMARD rows
};

struct Scalars {
    double c, rho0, dt;
};

// Kernel classes timed by the optional profiler (CUDA events on the launching stream).
enum KernelClass {
    KC_PLANE_INIT = 0, KC_PLANE_VEL, KC_PLANE_RHO_FWD, KC_PLANE_RHO_ADJ,
    KC_Z_ONE_TO_THREE, KC_Z_THREE_TO_THREE, KC_Z_THREE_TO_ONE, KC_SAMPLE, KC_COUNT
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
cudaError_t configure_kernels(const Geom& g, size_t* plane_smem, size_t* z_smem);
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
    float *qbar = nullptr, *xi = nullptr;                                          // prox: N, 3N
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

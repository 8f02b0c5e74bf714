// pat_kargs.h - kernel argument blocks shared by the kernel translation units and the launchers.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "pat_internal.h"

namespace pat {

static constexpr int kPlaneThreads = 256;
static constexpr int kZCols = 32;  // half-spectrum columns per z-pass CTA

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
    int flags;
};

typedef void (*PlaneKernel)(PlaneArgs);

struct PlaneKernels {
    PlaneKernel init = nullptr, vel = nullptr, rho_fwd = nullptr, rho_adj = nullptr;
    size_t smem_init = 0, smem3 = 0;
    int cs = 0;
};

// one function per x size, each in its own translation unit (compiled in parallel)
PlaneKernels plane_kernels_nx8(int ny);
PlaneKernels plane_kernels_nx16(int ny);
PlaneKernels plane_kernels_nx32(int ny);
PlaneKernels plane_kernels_nx64(int ny);
PlaneKernels plane_kernels_nx128(int ny);
PlaneKernels plane_kernels_nx256(int ny);

struct ZArgs {
    Geom g;
    const float2* tw_z;
    float2* spec[3];
    const float* kappaN;
    const float2* dt[3];
};

typedef void (*ZKernel)(ZArgs);

struct ZKernels {
    ZKernel grad3 = nullptr, each3 = nullptr, sum3 = nullptr;
    size_t smem = 0;
    int tc = 0;  // columns per CTA
    int nt = 0;  // threads per CTA
};

ZKernels z_kernels_for(int nz);

}  // namespace pat

// pat_kargs.h - kernel argument blocks shared by the kernel translation units and the launchers.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "pat_internal.h"

namespace pat {

static constexpr int kPlaneThreads = 256;
static constexpr int kZCols = 32;  // half-spectrum columns per z-FFT CTA

// (y,x) plane transforms of a stack of planes: real [b][p][ny][nx] <-> half spectrum [b][p][nxh][ny].
struct PlaneArgs {
    Geom g;
    const float2* tw_x;
    const float2* tw_y;
    const float* in_real;       // rfft input planes
    float* out_real;            // irfft output planes
    const float2* spec_in;      // irfft input spectra
    float2* spec_out;           // rfft output spectra
    long long bs_real, bs_spec; // batch strides (elements) of the real and spectral stacks
    float scale;                // irfft output factor
};

typedef void (*PlaneKernel)(PlaneArgs);

struct PlaneKernels {
    PlaneKernel rfft = nullptr, irfft = nullptr;
    size_t smem = 0;
    int cs = 0;
};

// one function per x size, each in its own translation unit (compiled in parallel)
PlaneKernels plane_kernels_nx8(int ny);
PlaneKernels plane_kernels_nx16(int ny);
PlaneKernels plane_kernels_nx32(int ny);
PlaneKernels plane_kernels_nx64(int ny);
PlaneKernels plane_kernels_nx128(int ny);
PlaneKernels plane_kernels_nx256(int ny);

// z transforms of a 3D half spectrum, in place: [b][z][c] <-> [b][kz][c], c = kx*ny + ky
struct ZArgs {
    Geom g;
    const float2* tw_z;
    float2* spec;
    float scale;                // inverse transform output factor
};

typedef void (*ZKernel)(ZArgs);

struct ZKernels {
    ZKernel fwd = nullptr, inv = nullptr;
    size_t smem = 0;
    int tc = 0;  // columns per CTA
    int nt = 0;  // threads per CTA
};

ZKernels z_kernels_for(int nz);

// Line passes of the time step (pat_line.cuh).
enum LineMode { LM_STEP = 0, LM_INIT = 1, LM_FIN = 2 };
enum LineFlag {
    LF_NO_OLD1 = 1, LF_NO_OLD2 = 2, LF_ACCUM = 4, LF_RECORD = 8, LF_INJECT = 16,
    LF_LATE_WAIT = 32,    // wait for the predecessor only before fetching the spectrum added to
    LF_TRIGGER_MID = 64,  // let the successor launch after that wait (default: at the start)
    LF_TRIGGER_END = 128  // let the successor launch only when this grid completes
};

struct LineArgs {
    Geom g;
    int ncols;                  // lines per batch entry
    int mode, flags;
    const float2* tw;           // exp(-2 pi i m / L), m < L
    const float2* twi;          // per-thread twiddles of the inverse transform's first half, [k][r]
    const float2* twf;          // ... and of the forward transform's first half (LineKernels docs)
    const float2* in;           // 3D half spectrum read (LM_STEP, LM_INIT)
    float2* out;                // 3D half spectrum written or accumulated (LM_STEP, LM_FIN)
    float2* st1;                // mixed-representation states, tile-major [B][tile][L][TC]
    float2* st2;
    const float* kap;           // kappa(|k|) at every line point, tile-major [tile][L][TC]
    const float2* dpre;         // k-space factor before the first inverse transform (NULL: none)
    const float2* dmid;         // between the two state updates
    const float2* dpost;        // after the last forward transform (NULL: none)
    float s_pre, s_mid, s_post; // scalar factors of the same three places
    const float* c1[3];         // state 1: decay, input gain, output gain (one entry per position)
    const float* c2[3];         // state 2
    const float2* tabs;         // LM_STEP: all the tables above in one block (DeviceTables::pass)
    int* err;                   // device word: bit i set when bulk copy i of a pass never landed
    int polls;                  // poll limit of the waits for the copies `skip` leaves out
    int skip;                   // fault-injection hook for tests: bulk copies (bits 1, 2) not issued
    float2* rec;                // z lines: plane spectrum recorded this step (LF_RECORD) ...
    const float2* inj;          // ... or injected this step (LF_INJECT); batch stride plane_bs
    long long plane_bs;
    int zs;                     // detection plane index
    float s_rec;                // 1/nz
};

typedef void (*LineKernel)(LineArgs);

// A length-L line transform is split L = ra * rb (pat_fft.cuh).  Thread r of a line (r < ra) uses
// the twiddle tables
//   twi[k * ra + r] = exp(+2 pi i r k / L), k < rb                 (inverse, k-space side first)
//   twf[k * rb + r] = exp(-2 pi i r k / L), k < ra, r < rb         (forward, spatial side first)
//   twf[k * ra + r] = exp(-2 pi i xr (2k + xh) / L), k < rb        (forward, when pair: ra = 2 rb)
// where a pair's row group and half are xr = r/2, xh = r%2, or with pnew xh = bit 1 of r and xr
// the other bits of r
struct LineKernels {
    LineKernel pass[3] = {nullptr, nullptr, nullptr};  // by axis (z, y, x) for this line length
    size_t smem = 0;
    int tc = 0;  // lines per CTA (one tile of the state layout)
    int nt = 0;  // threads per CTA
    int ra = 0, rb = 0;
    bool pair = false;
    bool pnew = false;
};

LineKernels line_kernels_for(int len);  // pass[] all NULL for a length without kernels

LineKernels line_kernels_l8();
LineKernels line_kernels_l16();
LineKernels line_kernels_l32();
LineKernels line_kernels_l64();
LineKernels line_kernels_l128();
LineKernels line_kernels_l256();

// adjoint start: spec[b][kz][c] = S[b][c] exp(-2 pi i kz zs / nz)
cudaError_t launch_spread_plane(const Geom& g, const float2* tw_z, const float2* S, long long s_bs,
                                float2* spec, cudaStream_t st);

}  // namespace pat

// pat_sample.cu - sampling operator C and its transpose per time point (Sec. 3.1, Sec. 4.3):
// rSP row selection (gather) and zero-filled scatter; scrambled-Hadamard patterns through an
// in-shared-memory fast Walsh-Hadamard transform, one CTA per recorded plane.
#include <math.h>

#include "pat_kargs.h"

namespace pat {

#define PAT_TRY(x)                            \
    do {                                      \
        cudaError_t _e = (x);                 \
        if (_e != cudaSuccess) return _e;     \
    } while (0)

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

static size_t g_shd_smem_max = 0;

cudaError_t configure_sampling(const Geom& g) {
    const size_t shd_bytes = (size_t)g.m_plane * sizeof(float);
    // sHd planes live in shared memory; larger planes are refused when the grid is created
    if (g.m_plane > 32768) return cudaSuccess;
    if (shd_bytes > 48 * 1024 && shd_bytes > g_shd_smem_max) {
        cudaError_t e = cudaFuncSetAttribute(shd_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shd_bytes);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(shd_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shd_bytes);
        if (e != cudaSuccess) return e;
        g_shd_smem_max = shd_bytes;
    }
    return cudaSuccess;
}

cudaError_t run_inject_only(const Geom& g, const float* inj, float* p, cudaStream_t st) {
    const long long total = (long long)g.B * g.nreal;
    const int blocks = (int)((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
    inject_plane_kernel<<<blocks, 256, 0, st>>>(inj, p, g);
    return cudaGetLastError();
}

}  // namespace pat

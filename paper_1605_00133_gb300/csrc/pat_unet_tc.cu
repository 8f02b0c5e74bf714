// pat_unet_tc.cu - 3x3x3 convolution of the learned warm start on the fifth-generation tensor cores
// (tcgen05): BF16 operands staged by the TMA unit, FP32 accumulators in tensor memory.
//
// Implicit GEMM, D[m][n] = sum_k A[m][k] B[n][k] with M = voxels, N = output channels, K = 27 taps x
// input channels.  A CTA owns one tile of M = 128 voxels, a bx x by x bz box of the volume (x
// fastest), and BN output channels.  One K step is one tap and CK input channels:
//   A: the voxel box shifted by the tap, loaded by a 4D tensor map over (channel, x, y, z); parts of
//      the box outside the volume come back as zeros, which is the convolution's zero padding;
//   B: the tap's weights w[t][n0 .. n0+BN)[c0 .. c0+CK), a 3D tensor map over (cin, cout, tap).
// Both land K-major in shared memory, CK BF16 per row with the swizzle of that row width (32, 64 or
// 128 bytes), the layout the MMA's shared-memory descriptors read.  Warp roles (192 threads):
//   warp 0   one thread issues the TMA copies of a NSTAGE-deep ring (full/empty mbarriers);
//   warp 1   allocates the tensor-memory accumulator (128 lanes x BN FP32 columns) and one thread
//            issues tcgen05.mma (M = 128, N = BN, K = 16 per instruction), committing each stage's
//            MMAs to that stage's empty barrier and the last to the done barrier;
//   warps 2-5 the epilogue: tcgen05.ld of the accumulator rows (warp w reads lanes 32 (w % 4) ..),
//            optional ReLU, BF16 rounding, one voxel row per thread to global memory.
// Every mbarrier wait is bounded.  A wait that gives up records bit 0 of a device word (read and
// cleared by pat_unet_device_status), and the CTA stops issuing work, waits (bounded) for the copies
// it issued, frees its tensor memory and exits; its outputs are then invalid.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "pat_fft.cuh"

namespace pat {

__device__ int g_unet_err;  // bit 0: a tensor-core convolution gave up waiting (outputs invalid)

namespace {

constexpr int kNStage = 4;
constexpr int kBM = 128;
constexpr int kThreads = 192;
constexpr int kPolls = 1 << 20;  // bounded waits: each poll suspends for at most about a microsecond

// test hook of the convolution's failure path (pat_unet_debug_copy_fault): process-wide
int g_stop_after = -1;
int g_polls = kPolls;

struct ConvTcArgs {
    __nv_bfloat16* y;
    int ldy, cin, cout, bn;
    int D, H, W;
    int bx, by, bz;     // voxel box of a tile
    int tx, ty;         // tiles along x and y
    int relu;
    uint32_t tmem_cols;
    int stop_after;     // test hook: the producer issues only stages < stop_after (< 0: all)
    int polls;          // poll limit of the wait for the first stage the test hook leaves out
};

// shared-memory matrix descriptor of a K-major operand tile: rows of `row_bytes` (= the swizzle
// width: 32, 64 or 128 bytes), 8-row groups `8 * row_bytes` apart (stride byte offset); the leading
// byte offset is unused for swizzled K-major tiles; descriptor version 1; layout type 6 / 4 / 2 for
// the 32 / 64 / 128-byte swizzle
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t saddr, uint32_t row_bytes) {
    const uint64_t layout = (row_bytes == 128) ? 2 : (row_bytes == 64) ? 4 : 6;
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(((8 * row_bytes) >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= layout << 61;
    return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t mma_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
// arrive on `bar` once every tcgen05 operation this thread issued before has completed
__device__ __forceinline__ void tc_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

template <int CK>
__global__ void __launch_bounds__(kThreads, 1) conv3_tc_kernel(const __grid_constant__ CUtensorMap tmx,
                                                                const __grid_constant__ CUtensorMap tmw,
                                                                ConvTcArgs a) {
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte alignment of every operand tile (the 128-byte swizzle repeats every 1024 bytes)
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    constexpr uint32_t RB = CK * 2;            // bytes per operand row = swizzle width
    constexpr uint32_t A_BYTES = kBM * RB;     // 4, 8 or 16 KB: a multiple of 1024
    const uint32_t b_bytes = (uint32_t)a.bn * RB;
    const uint32_t stage_bytes = (A_BYTES + b_bytes + 1023) & ~1023u;
    unsigned long long* full = reinterpret_cast<unsigned long long*>(smem + kNStage * stage_bytes);
    unsigned long long* empty = full + kNStage;
    unsigned long long* done = empty + kNStage;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    int* counts = reinterpret_cast<int*>(tmem_slot + 1);  // [0] stages issued, [1] consumed, [2] failed

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x;
    const int x0 = (tile % a.tx) * a.bx;
    const int y0 = ((tile / a.tx) % a.ty) * a.by;
    const int z0 = (tile / (a.tx * a.ty)) * a.bz;
    const int n0 = blockIdx.y * a.bn;
    const int nc = a.cin / CK;
    const int S = 27 * nc;
    // bytes a stage's two copies deliver: the voxel box (at most 128 rows; rows of the tile beyond it
    // are never stored) and the weight tile
    const uint32_t tx_bytes = RB * (uint32_t)(a.bx * a.by * a.bz) + b_bytes;

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kNStage; s++) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(done, 1);
        mbar_fence_init();
        counts[0] = counts[1] = counts[2] = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer
        int s = 0;
        for (; s < S; s++) {
            const int st = s % kNStage, use = s / kNStage;
            if (a.stop_after >= 0 && s >= a.stop_after) break;  // test hook: nothing more is issued
            if (use > 0 && !mbar_wait(empty + st, (use - 1) & 1, kPolls)) {
                counts[2] = 1;
                break;
            }
            const int t = s / nc, c0 = (s - t * nc) * CK;
            const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
            uint8_t* sa = smem + st * stage_bytes;
            mbar_arrive_expect_tx(full + st, tx_bytes);
            tma_load_4d(sa, &tmx, c0, x0 + dx, y0 + dy, z0 + dz, full + st);
            tma_load_3d(sa + A_BYTES, &tmw, c0, n0, t, full + st);
        }
        counts[0] = s;
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = mma_idesc(a.bn);
        int s = 0;
        for (; s < S; s++) {
            const int st = s % kNStage, use = s / kNStage;
            // the test hook's short limit applies only to the first stage it leaves out
            const int lim = (a.stop_after >= 0 && s >= a.stop_after) ? a.polls : kPolls;
            if (!mbar_wait(full + st, use & 1, lim)) {
                counts[2] = 1;
                break;
            }
            tc_fence_after();
            const uint32_t sa = smem_addr(smem + st * stage_bytes);
#pragma unroll
            for (int k = 0; k < CK / 16; k++) {
                const uint64_t ad = kmajor_desc(sa + 32 * k, RB);
                const uint64_t bd = kmajor_desc(sa + A_BYTES + 32 * k, RB);
                tc_mma(tmem, ad, bd, idesc, (s > 0 || k > 0) ? 1u : 0u);
            }
            tc_commit(empty + st);
        }
        counts[1] = s;
        tc_commit(done);
    } else if (warp >= 2) {
        // epilogue
        const bool ok = mbar_wait(done, 0, kPolls);
        if (!ok) counts[2] = 1;
        __syncwarp();  // the tensor-memory loads below are warp-wide
        tc_fence_after();
        const int m = 32 * (warp & 3) + lane;  // tensor-memory lane = tile row
        const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
        const int xx = m % a.bx, yy = (m / a.bx) % a.by, zz = m / (a.bx * a.by);
        const int x = x0 + xx, y = y0 + yy, z = z0 + zz;
        const bool valid = ok && m < a.bx * a.by * a.bz && x < a.W && y < a.H && z < a.D;
        __nv_bfloat16* out = a.y + ((size_t)((size_t)z * a.H + y) * a.W + x) * a.ldy + n0;
        for (int c = 0; c < a.bn; c += 16) {
            float v[16];
            tc_ld16(trow + (uint32_t)c, v);  // every thread of the warp takes part
            if (valid) {
                uint4 pk[2];
                uint32_t* w32 = reinterpret_cast<uint32_t*>(pk);
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    float p = v[2 * i], q = v[2 * i + 1];
                    if (a.relu) {
                        p = fmaxf(p, 0.f);
                        q = fmaxf(q, 0.f);
                    }
                    const __nv_bfloat162 h = __floats2bfloat162_rn(p, q);
                    w32[i] = *reinterpret_cast<const uint32_t*>(&h);
                }
                uint4* dst = reinterpret_cast<uint4*>(out + c);
                dst[0] = pk[0];
                dst[1] = pk[1];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (counts[2]) {
        if (threadIdx.x == 0) {
            atomicOr(&g_unet_err, 1);
            // copies issued but never consumed may still be in flight: let them land (bounded)
            for (int s = counts[1]; s < counts[0]; s++) mbar_wait(full + s % kNStage, (s / kNStage) & 1, kPolls);
            mbar_wait(done, 0, kPolls);
        }
        __syncthreads();
    }
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
    }
}

// ---------------------------------------------------------------------------------------------
// Weight gradient: dW[t][co][ci] = sum_v dY[v][co] X[v + off_t][ci], all 27 taps in one GEMM with
// M = (tap, input channel) rows m = t cin + ci (M tiles along grid.x, so that the CTAs reading one
// voxel chunk run together and find its input in L2), N = output channels and K = voxels, split over
// chunks of voxel blocks (grid.y) with a fixed-order sum afterwards.  A K block is a box of 64 voxels.  Both
// operands arrive channel-contiguous, i.e. MN-major: a swizzle atom is 8 voxel rows x WA channels of
// one tap (A) or 8 voxel rows x WB output channels (B), WA, WB in {16, 32, 64}; the M tile's 128 rows
// are 128 / WA atoms side by side (one TMA box each: the tap's shifted voxel box, zero outside the
// volume), the N tile's cout columns cout / WB atoms.  In a descriptor the leading byte offset steps
// from one atom to the next along M or N, the stride byte offset from one 8-row group of voxels to
// the next.
// ---------------------------------------------------------------------------------------------

constexpr int kKB = 64;  // voxels per K block

struct WgradArgs {
    float* partial;     // [chunk][mtiles * 128][cout]
    int cin, cout, wa, wb;
    int D, H, W;
    int bx, by, bz, tx, ty, nkb;   // voxel box of a K block, blocks along x and y, blocks in all
    int kb_per_cta;
    uint32_t tmem_cols;
};

// MN-major descriptor: atoms of 8 rows x `row_bytes`, `lbo` bytes apart along M/N, 8-row groups
// 8 * row_bytes apart along K
__device__ __forceinline__ uint64_t mnmajor_desc(uint32_t saddr, uint32_t row_bytes, uint32_t lbo) {
    const uint64_t layout = (row_bytes == 128) ? 2 : (row_bytes == 64) ? 4 : 6;
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)(((8 * row_bytes) >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= layout << 61;
    return d;
}

__global__ void __launch_bounds__(kThreads, 1) wgrad_tc_kernel(const __grid_constant__ CUtensorMap tmx,
                                                               const __grid_constant__ CUtensorMap tmd,
                                                               WgradArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t ra = 2u * a.wa, rb = 2u * a.wb;      // row bytes = swizzle widths
    const uint32_t atom_a = kKB * ra, atom_b = kKB * rb; // one atom column over the K block
    const uint32_t a_bytes = kBM * kKB * 2;              // 16 KB
    const uint32_t b_bytes = (uint32_t)a.cout * kKB * 2;
    const uint32_t stage_bytes = (a_bytes + b_bytes + 1023) & ~1023u;
    unsigned long long* full = reinterpret_cast<unsigned long long*>(smem + kNStage * stage_bytes);
    unsigned long long* empty = full + kNStage;
    unsigned long long* done = empty + kNStage;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    int* counts = reinterpret_cast<int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mtile = blockIdx.x;  // M tiles fastest: the CTAs of one voxel chunk run together
    const int chunk = blockIdx.y;
    const int kb0 = chunk * a.kb_per_cta;
    const int nkb = min(a.kb_per_cta, a.nkb - kb0);
    const int natoms_a = kBM / a.wa;                 // atoms (tap, channel block) of this M tile
    const int cblocks = a.cin / a.wa;
    const int atom0 = mtile * natoms_a;
    const int atoms_total = 27 * cblocks;
    const int natoms_live = min(natoms_a, atoms_total - atom0);
    const int nb_atoms = a.cout / a.wb;
    const uint32_t tx_bytes = (uint32_t)natoms_live * atom_a + b_bytes;

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kNStage; s++) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(done, 1);
        mbar_fence_init();
        counts[0] = counts[1] = counts[2] = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        int s = 0;
        for (; s < nkb; s++) {
            const int st = s % kNStage, use = s / kNStage;
            if (use > 0 && !mbar_wait(empty + st, (use - 1) & 1, kPolls)) {
                counts[2] = 1;
                break;
            }
            const int kb = kb0 + s;
            const int x0 = (kb % a.tx) * a.bx, y0 = ((kb / a.tx) % a.ty) * a.by, z0 = (kb / (a.tx * a.ty)) * a.bz;
            uint8_t* sa = smem + st * stage_bytes;
            mbar_arrive_expect_tx(full + st, tx_bytes);
            for (int j = 0; j < natoms_live; j++) {
                const int atom = atom0 + j, t = atom / cblocks, c0 = (atom - t * cblocks) * a.wa;
                const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
                tma_load_4d(sa + j * atom_a, &tmx, c0, x0 + dx, y0 + dy, z0 + dz, full + st);
            }
            for (int j = 0; j < nb_atoms; j++)
                tma_load_4d(sa + a_bytes + j * atom_b, &tmd, j * a.wb, x0, y0, z0, full + st);
        }
        counts[0] = s;
    } else if (warp == 1 && lane == 0) {
        // A and B MN-major (bits 15, 16), FP32 accumulator, BF16 operands, M = 128, N = cout
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                               ((uint32_t)(a.cout >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
        int s = 0;
        for (; s < nkb; s++) {
            const int st = s % kNStage, use = s / kNStage;
            if (!mbar_wait(full + st, use & 1, kPolls)) {
                counts[2] = 1;
                break;
            }
            tc_fence_after();
            const uint32_t sa = smem_addr(smem + st * stage_bytes);
#pragma unroll
            for (int k = 0; k < kKB / 16; k++) {
                // 16 voxel rows = two 8-row groups: the start moves by 16 rows of each operand
                const uint64_t ad = mnmajor_desc(sa + 16 * ra * k, ra, atom_a);
                const uint64_t bd = mnmajor_desc(sa + a_bytes + 16 * rb * k, rb, atom_b);
                tc_mma(tmem, ad, bd, idesc, (s > 0 || k > 0) ? 1u : 0u);
            }
            tc_commit(empty + st);
        }
        counts[1] = s;
        tc_commit(done);
    } else if (warp >= 2) {
        const bool ok = mbar_wait(done, 0, kPolls);
        if (!ok) counts[2] = 1;
        __syncwarp();
        tc_fence_after();
        const int m = 32 * (warp & 3) + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
        float* out = a.partial + ((size_t)chunk * gridDim.x * kBM + (size_t)mtile * kBM + m) * a.cout;
        for (int c = 0; c < a.cout; c += 16) {
            float v[16];
            tc_ld16(trow + (uint32_t)c, v);
            if (nkb <= 0) {
#pragma unroll
                for (int i = 0; i < 16; i++) v[i] = 0.f;
            }
            float4* dst = reinterpret_cast<float4*>(out + c);
#pragma unroll
            for (int i = 0; i < 4; i++) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (counts[2]) {
        if (threadIdx.x == 0) {
            atomicOr(&g_unet_err, 1);
            for (int s = counts[1]; s < counts[0]; s++) mbar_wait(full + s % kNStage, (s / kNStage) & 1, kPolls);
            mbar_wait(done, 0, kPolls);
        }
        __syncthreads();
    }
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
    }
}

// dw[t][co][ci] = sum over chunks c (in order) of partial[c][t cin + ci][co]
__global__ void wgrad_sum_kernel(const float* __restrict__ partial, int nchunk, int rows, int cin, int cout,
                                 float* __restrict__ dw) {
    const long long n = 27LL * cin * cout;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(i % cin);
        const long long r = i / cin;
        const int co = (int)(r % cout), t = (int)(r / cout);
        const size_t row = (size_t)t * cin + ci;
        float s = 0.f;
        for (int c = 0; c < nchunk; c++) s += partial[((size_t)c * rows + row) * cout + co];
        dw[i] = s;
    }
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static std::once_flag once;
    static EncodeTiled fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

template <int CK>
cudaError_t launch_ck(const CUtensorMap& mx, const CUtensorMap& mw, const ConvTcArgs& a, unsigned tiles,
                      cudaStream_t st) {
    const uint32_t stage = (kBM * CK * 2 + a.bn * CK * 2 + 1023) & ~1023u;
    size_t smem = 1024 + kNStage * (size_t)stage + (2 * kNStage + 1) * 8 + 4 + 16;
    // at most 512 / tmem_cols CTAs on an SM, so that every CTA's tensor-memory allocation succeeds at
    // once: request enough shared memory (228 KB per SM, 1 KB reserved per CTA) to keep out one more
    const size_t max_ctas = 512 / a.tmem_cols;
    const size_t floor_smem = 233472 / (max_ctas + 1) + 1;
    if (smem < floor_smem) smem = floor_smem;
    cudaError_t e = cudaFuncSetAttribute(conv3_tc_kernel<CK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    conv3_tc_kernel<CK><<<dim3(tiles, (unsigned)(a.cout / a.bn)), kThreads, smem, st>>>(mx, mw, a);
    return cudaGetLastError();
}

}  // namespace

// y[v][n] = act(sum_t sum_c x[v + off_t][c] w[t][n][c]) on the tensor cores (see the file comment).
// Channel counts multiples of 16, strides multiples of 16 elements, pointers 16-byte aligned (checked
// by the caller).
cudaError_t conv3_tc(const void* x, int ldx, int cin, const void* w, int cout, void* y, int ldy, int D, int H,
                     int W, int relu, cudaStream_t st) {
    EncodeTiled enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    const int ck = (cin % 64 == 0) ? 64 : (cin % 32 == 0) ? 32 : 16;
    ConvTcArgs a = {};
    a.y = reinterpret_cast<__nv_bfloat16*>(y);
    a.ldy = ldy;
    a.cin = cin;
    a.cout = cout;
    a.bn = (cout % 128 == 0) ? 128 : (cout % 64 == 0) ? 64 : (cout % 32 == 0) ? 32 : 16;
    a.D = D;
    a.H = H;
    a.W = W;
    a.bx = W < kBM ? W : kBM;
    a.by = H < kBM / a.bx ? H : kBM / a.bx;
    a.bz = kBM / (a.bx * a.by);
    a.tx = (W + a.bx - 1) / a.bx;
    a.ty = (H + a.by - 1) / a.by;
    const long long tz = (D + a.bz - 1) / a.bz;
    const long long tiles = (long long)a.tx * a.ty * tz;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    a.relu = relu;
    a.tmem_cols = a.bn < 32 ? 32 : a.bn;
    a.stop_after = g_stop_after;
    a.polls = g_polls;
    const CUtensorMapSwizzle swz =
        ck == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : ck == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
    alignas(64) CUtensorMap mx, mw;
    {
        const cuuint64_t dims[4] = {(cuuint64_t)cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D};
        const cuuint64_t strides[3] = {(cuuint64_t)ldx * 2, (cuuint64_t)ldx * 2 * W, (cuuint64_t)ldx * 2 * W * H};
        const cuuint32_t box[4] = {(cuuint32_t)ck, (cuuint32_t)a.bx, (cuuint32_t)a.by, (cuuint32_t)a.bz};
        const cuuint32_t es[4] = {1, 1, 1, 1};
        if (enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(x), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        const cuuint64_t dims[3] = {(cuuint64_t)cin, (cuuint64_t)cout, 27};
        const cuuint64_t strides[2] = {(cuuint64_t)cin * 2, (cuuint64_t)cin * 2 * cout};
        const cuuint32_t box[3] = {(cuuint32_t)ck, (cuuint32_t)a.bn, 1};
        const cuuint32_t es[3] = {1, 1, 1};
        if (enc(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(w), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    if (ck == 64) return launch_ck<64>(mx, mw, a, (unsigned)tiles, st);
    if (ck == 32) return launch_ck<32>(mx, mw, a, (unsigned)tiles, st);
    return launch_ck<16>(mx, mw, a, (unsigned)tiles, st);
}

// Geometry of the weight-gradient GEMM (shared by the scratch-size query and the launch).
struct WgradGeom {
    int wa, wb, bx, by, bz, tx, ty, nkb, mtiles, kb_per_cta, nchunk;
};

static WgradGeom wgrad_geom(int cin, int cout, int D, int H, int W) {
    WgradGeom g;
    g.wa = (cin % 64 == 0) ? 64 : (cin % 32 == 0) ? 32 : 16;
    g.wb = (cout % 64 == 0) ? 64 : (cout % 32 == 0) ? 32 : 16;
    // a K block is exactly kKB voxels (the MMA reads all its rows): powers of two, the box reaching
    // past the volume where a side is shorter (those voxels read as zeros)
    auto pow2_at_least = [](int v) {
        int p = 1;
        while (p < v) p <<= 1;
        return p;
    };
    g.bx = std::min(kKB, pow2_at_least(W));
    g.by = std::min(kKB / g.bx, pow2_at_least(H));
    g.bz = kKB / (g.bx * g.by);
    g.tx = (W + g.bx - 1) / g.bx;
    g.ty = (H + g.by - 1) / g.by;
    const long long tz = (D + g.bz - 1) / g.bz;
    g.nkb = (int)((long long)g.tx * g.ty * tz);
    g.mtiles = (27 * cin + kBM - 1) / kBM;
    // about four CTAs per SM over all M tiles, at least 8 K blocks each
    const long long want = 4LL * 152;
    long long per = ((long long)g.nkb * g.mtiles + want - 1) / want;
    if (per < 8) per = 8;
    g.kb_per_cta = (int)per;
    g.nchunk = (g.nkb + g.kb_per_cta - 1) / g.kb_per_cta;
    return g;
}

int64_t wgrad_tc_scratch(int cin, int cout, int D, int H, int W) {
    const WgradGeom g = wgrad_geom(cin, cout, D, H, W);
    return (int64_t)g.nchunk * g.mtiles * kBM * cout;
}

// dw[t][co][ci] = sum_v dy[v][co] x[v + off_t][ci] on the tensor cores; partial: wgrad_tc_scratch
// floats.  cin multiple of 16 (<= 512), cout in {16, 32, 48, ..., 256} with cout % 16 == 0.
cudaError_t wgrad_tc(const void* x, int ldx, int cin, const void* dy, int ldy, int cout, int D, int H, int W,
                     float* partial, float* dw, cudaStream_t st) {
    EncodeTiled enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    const WgradGeom g = wgrad_geom(cin, cout, D, H, W);
    const CUtensorMapSwizzle sa = g.wa == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : g.wa == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                                                      : CU_TENSOR_MAP_SWIZZLE_32B;
    const CUtensorMapSwizzle sb = g.wb == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : g.wb == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                                                      : CU_TENSOR_MAP_SWIZZLE_32B;
    alignas(64) CUtensorMap mx, md;
    const cuuint32_t es[4] = {1, 1, 1, 1};
    {
        const cuuint64_t dims[4] = {(cuuint64_t)cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D};
        const cuuint64_t strides[3] = {(cuuint64_t)ldx * 2, (cuuint64_t)ldx * 2 * W, (cuuint64_t)ldx * 2 * W * H};
        const cuuint32_t box[4] = {(cuuint32_t)g.wa, (cuuint32_t)g.bx, (cuuint32_t)g.by, (cuuint32_t)g.bz};
        if (enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(x), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, sa, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        const cuuint64_t dims[4] = {(cuuint64_t)cout, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D};
        const cuuint64_t strides[3] = {(cuuint64_t)ldy * 2, (cuuint64_t)ldy * 2 * W, (cuuint64_t)ldy * 2 * W * H};
        const cuuint32_t box[4] = {(cuuint32_t)g.wb, (cuuint32_t)g.bx, (cuuint32_t)g.by, (cuuint32_t)g.bz};
        if (enc(&md, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(dy), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, sb, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    WgradArgs a = {};
    a.partial = partial;
    a.cin = cin;
    a.cout = cout;
    a.wa = g.wa;
    a.wb = g.wb;
    a.D = D;
    a.H = H;
    a.W = W;
    a.bx = g.bx;
    a.by = g.by;
    a.bz = g.bz;
    a.tx = g.tx;
    a.ty = g.ty;
    a.nkb = g.nkb;
    a.kb_per_cta = g.kb_per_cta;
    a.tmem_cols = cout <= 32 ? 32 : cout <= 64 ? 64 : cout <= 128 ? 128 : 256;
    const uint32_t stage = (kBM * kKB * 2 + cout * kKB * 2 + 1023) & ~1023u;
    size_t smem = 1024 + kNStage * (size_t)stage + (2 * kNStage + 1) * 8 + 4 + 16;
    const size_t max_ctas = 512 / a.tmem_cols;
    const size_t floor_smem = 233472 / (max_ctas + 1) + 1;
    if (smem < floor_smem) smem = floor_smem;
    cudaError_t e = cudaFuncSetAttribute(wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    wgrad_tc_kernel<<<dim3((unsigned)g.mtiles, (unsigned)g.nchunk), kThreads, smem, st>>>(mx, md, a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long n = 27LL * cin * cout;
    const int blocks = (int)((n + 255) / 256 < 152 * 8 ? (n + 255) / 256 : 152 * 8);
    wgrad_sum_kernel<<<blocks, 256, 0, st>>>(partial, g.nchunk, g.mtiles * kBM, cin, cout, dw);
    return cudaGetLastError();
}

// test hook: later convolutions issue only their first stop_after stages (< 0: normal operation) and
// give up waiting after `polls` polls (<= 0: the default)
void unet_set_copy_fault(int stop_after, int polls) {
    g_stop_after = stop_after;
    g_polls = polls > 0 ? polls : kPolls;
}

// reads and clears the device word of the tensor-core convolutions
cudaError_t unet_take_status(int* word, cudaStream_t st) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_unet_err);
    if (e == cudaSuccess) e = cudaMemcpyAsync(word, p, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && *word) e = cudaMemsetAsync(p, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

}  // namespace pat

// pat_run.cu - launch sequences of A and A^T (Sec. 4.3) on one stream.
//
// Forward, T recorded samples (n = 0 is p0 itself):
//   plane_rfft + zfft_fwd          p^0 = F p0 (3D half spectrum); record n = 0 (p0's plane spectrum)
//   line INIT x, y, z              rho_i^0 = p0 / (3c^2) in each axis's mixed representation
//   for n = 0 .. T-2:
//     line STEP x, y, z            u_i^{n+1/2}, rho_i^{n+1} and p^{n+1} = c^2 sum F_i rho_i; the z
//                                  pass records the detection plane's spectrum.  At n = 0 the
//                                  half-step start u^{-1/2} = dt/(2 rho0) D^+ p0 is folded into the
//                                  coefficient as (as/2 - 1) dt/rho0.
//   plane_irfft                    recorded spectra n = 0 .. T-1 -> real planes
//   sample (C)                     unless the full plane is recorded
// Adjoint: C^T, plane_rfft of the T injected planes, lambda^{T-1} = their spectrum placed on the
// plane, then the line passes in reverse time order with the transposed coefficients (the last step
// folds the transpose of the initial half step into as (1 - as/2)), the image terms
// a_i^2 q_i / (3 c^2) (line FIN x, y, z), and the inverse 3D transform (zfft_inv + plane_irfft).
#include "pat_fft.cuh"
#include "pat_kargs.h"

namespace pat {

cudaError_t configure_sampling(const Geom& g);
cudaError_t run_inject_only(const Geom& g, const float* inj, float* p, cudaStream_t st);

#define PAT_TRY(x)                            \
    do {                                      \
        cudaError_t _e = (x);                 \
        if (_e != cudaSuccess) return _e;     \
    } while (0)

static PlaneKernels plane_kernels_for(int nx, int ny) {
    switch (nx) {
        case 8: return plane_kernels_nx8(ny);
        case 16: return plane_kernels_nx16(ny);
        case 32: return plane_kernels_nx32(ny);
        case 64: return plane_kernels_nx64(ny);
        case 128: return plane_kernels_nx128(ny);
        case 256: return plane_kernels_nx256(ny);
        default: return PlaneKernels{};
    }
}

LineKernels line_kernels_for(int len) {
    switch (len) {
        case 8: return line_kernels_l8();
        case 16: return line_kernels_l16();
        case 32: return line_kernels_l32();
        case 64: return line_kernels_l64();
        case 128: return line_kernels_l128();
        case 256: return line_kernels_l256();
        default: return LineKernels{};
    }
}

int plane_cluster_size(int nx, int ny) { return plane_kernels_for(nx, ny).cs; }

static const char* g_config_what = "";
const char* configure_failure() { return g_config_what; }

cudaError_t configure_kernels(const Geom& g) {
    PlaneKernels pk = plane_kernels_for(g.nx, g.ny);
    ZKernels zk = z_kernels_for(g.nz);
    if (!pk.rfft || !zk.fwd) {
        g_config_what = "no kernel instantiation for this grid shape";
        return cudaErrorInvalidValue;
    }
#define PAT_CFG(call, what)                  \
    do {                                     \
        cudaError_t _e = (call);             \
        if (_e != cudaSuccess) {             \
            g_config_what = what;            \
            return _e;                       \
        }                                    \
    } while (0)
    PAT_CFG(cudaFuncSetAttribute(pk.rfft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pk.smem), "plane_rfft smem");
    PAT_CFG(cudaFuncSetAttribute(pk.irfft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pk.smem), "plane_irfft smem");
    PAT_CFG(cudaFuncSetAttribute(zk.fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zk.smem), "zfft_fwd smem");
    PAT_CFG(cudaFuncSetAttribute(zk.inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zk.smem), "zfft_inv smem");
    for (int ax = 0; ax < 3; ax++) {
        LineKernels lk = line_kernels_for(g.len[ax]);
        if (!lk.pass[ax]) {
            g_config_what = "no line kernel for this axis length";
            return cudaErrorInvalidValue;
        }
        PAT_CFG(cudaFuncSetAttribute(lk.pass[ax], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lk.smem),
                "line pass smem");
    }
    PAT_CFG(configure_sampling(g), "sampling smem");
#undef PAT_CFG
    g_config_what = "";
    return cudaSuccess;
}

// optional event bracketing of one launch
template <class F>
static cudaError_t timed(Profiler* prof, int cls, cudaStream_t st, F&& launch) {
    if (!prof || !prof->on) return launch();
    Profiler::Rec r;
    r.cls = cls;
    PAT_TRY(prof->ev(&r.a));
    PAT_TRY(prof->ev(&r.b));
    PAT_TRY(cudaEventRecord(r.a, st));
    PAT_TRY(launch());
    PAT_TRY(cudaEventRecord(r.b, st));
    prof->recs.push_back(r);
    return cudaSuccess;
}

// Kernels are launched with programmatic stream serialisation (they call pdl_wait() before touching
// memory), so each one is scheduled while its predecessor drains.
static cudaLaunchAttribute pdl_attr() {
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at.val.programmaticStreamSerializationAllowed = 1;
    return at;
}

static cudaError_t launch_plane(PlaneKernel k, const PlaneKernels& pk, int nplanes, const PlaneArgs& a,
                                cudaStream_t st) {
    if (nplanes <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(pk.cs, nplanes, a.g.B);
    cfg.blockDim = dim3(kPlaneThreads, 1, 1);
    cfg.dynamicSmemBytes = pk.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = pk.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1] = pdl_attr();
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, k, a);
}

static cudaError_t launch_z(ZKernel k, const ZKernels& zk, const ZArgs& a, cudaStream_t st) {
    const int ncols = a.g.ny * a.g.nxh;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((ncols + zk.tc - 1) / zk.tc, a.g.B, 1);
    cfg.blockDim = dim3(zk.nt, 1, 1);
    cfg.dynamicSmemBytes = zk.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1] = {pdl_attr()};
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, a);
}

static cudaError_t launch_line(int ax, const LineArgs& a, cudaStream_t st) {
    const LineKernels lk = line_kernels_for(a.g.len[ax]);
    if (!lk.pass[ax]) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((a.ncols + lk.tc - 1) / lk.tc, a.g.B, 1);
    cfg.blockDim = dim3(lk.nt, 1, 1);
    cfg.dynamicSmemBytes = lk.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1] = {pdl_attr()};
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, lk.pass[ax], a);
}

static const int kLineClass[3] = {KC_LINE_Z, KC_LINE_Y, KC_LINE_X};
static const int kPassOrder[3] = {AX, AY, AZ};  // x writes the new spectrum, y and z add to it
// When each pass lets its successor launch, by axis (z, y, x).  Launched early, a grid's CTAs land
// on whichever SMs free up first, four to an SM, and wait there; measured on c2, launching the x pass
// only when the z pass completes (all 152 SMs free) and the y and z passes once their predecessor
// has passed its mid-pass point beats launching every pass at the start of its predecessor
// (56.7 vs 52.6 pairs/s).
static const int kTrigger[3] = {LF_TRIGGER_END, LF_TRIGGER_MID, LF_TRIGGER_MID};

// spec[b][kz][c] = S[b][c] exp(-2 pi i kz zs / nz): the 3D spectrum of a plane source at z = zs
__global__ void spread_plane_kernel(Geom g, const float2* __restrict__ tw_z, const float2* __restrict__ S,
                                    long long s_bs, float2* __restrict__ spec) {
    const long long nplane = g.nplane;
    const long long total = (long long)g.B * g.nz * nplane;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long c = i % nplane;
        const long long kz = (i / nplane) % g.nz;
        const long long b = i / (nplane * g.nz);
        const float2 w = tw_z[(kz * g.sensor_z) & (g.nz - 1)];
        spec[i] = cmul(S[b * s_bs + c], w);
    }
}

cudaError_t launch_spread_plane(const Geom& g, const float2* tw_z, const float2* S, long long s_bs,
                                float2* spec, cudaStream_t st) {
    const long long total = (long long)g.B * g.nz * g.nplane;
    const int nt = 256;
    const long long nb = (total + nt - 1) / nt;
    spread_plane_kernel<<<(unsigned)(nb < 4096 ? nb : 4096), nt, 0, st>>>(g, tw_z, S, s_bs, spec);
    return cudaGetLastError();
}

static LineArgs line_base(const Geom& g, const DeviceTables& t, const Workspace& w, int ax) {
    LineArgs a = {};
    a.g = g;
    a.ncols = g.ncols[ax];
    a.tw = t.tw[ax];
    a.err = t.err;
    a.polls = t.polls;
    a.skip = t.skip;
    a.twi = t.twi[ax];
    a.twf = t.twf[ax];
    a.st1 = w.ms[ax][0];
    a.st2 = w.ms[ax][1];
    a.kap = t.kappa[ax];
    a.zs = g.sensor_z;
    a.plane_bs = (long long)g.T * g.nplane;
    a.s_rec = 1.0f / (float)g.nz;
    return a;
}

// state coefficient tables; an output gain of CT_ONE is passed as NULL (no multiply)
static void set_coef(const float** dst, const DeviceTables& t, int ax, const int* c) {
    dst[0] = t.coef[c[0]][ax];
    dst[1] = t.coef[c[1]][ax];
    dst[2] = (c[2] == CT_ONE) ? nullptr : t.coef[c[2]][ax];
}

// the tables of one kind of time step (kPassTables) for a line pass of axis ax
static void set_pass_tables(LineArgs& a, const DeviceTables& t, int ax, int ps) {
    const PassTables& pt = kPassTables[ps];
    const float2* d[3];
    for (int i = 0; i < 3; i++)
        d[i] = (pt.d[i] == DF_PLUS) ? t.dplus[ax] : (pt.d[i] == DF_MINUS) ? t.dminus[ax] : nullptr;
    a.dpre = d[0];
    a.dmid = d[1];
    a.dpost = d[2];
    set_coef(a.c1, t, ax, pt.c1);
    set_coef(a.c2, t, ax, pt.c2);
    a.tabs = t.pass[ps][ax];
}

cudaError_t run_forward(const Geom& g, const DeviceTables& t, const Workspace& w, const Scalars& s,
                        int kind, int m, const float* p0, float* f, cudaStream_t st, Profiler* prof) {
    const PlaneKernels pk = plane_kernels_for(g.nx, g.ny);
    const ZKernels zk = z_kernels_for(g.nz);
    if (!pk.rfft || !zk.fwd) return cudaErrorInvalidValue;
    float* rec = (kind == PAT_SAMPLE_FULL) ? f : w.rec;
    const long long M = g.m_plane;

    // p^0 = F p0; the record's plane 0 is p0's detection plane, taken through its (kx, ky) spectrum
    // like every other plane (the real series may share memory with the loop state)
    PlaneArgs pa = {};
    pa.g = g;
    pa.tw_x = t.tw[AX];
    pa.tw_y = t.tw[AY];
    pa.in_real = p0;
    pa.bs_real = g.nreal;
    pa.spec_out = w.ph[0];
    pa.bs_spec = g.nspec;
    PAT_TRY(timed(prof, KC_PLANE_FFT, st, [&] { return launch_plane(pk.rfft, pk, g.nz, pa, st); }));
    PAT_TRY(cudaMemcpy2DAsync(w.rk, (size_t)g.T * g.nplane * sizeof(float2),
                              w.ph[0] + (size_t)g.sensor_z * g.nplane, (size_t)g.nspec * sizeof(float2),
                              (size_t)g.nplane * sizeof(float2), (size_t)g.B, cudaMemcpyDeviceToDevice, st));
    if (g.T > 1) {
        ZArgs za = {};
        za.g = g;
        za.tw_z = t.tw[AZ];
        za.spec = w.ph[0];
        za.scale = 1.0f;
        PAT_TRY(timed(prof, KC_Z_FFT, st, [&] { return launch_z(zk.fwd, zk, za, st); }));

        const double c2 = s.c * s.c;
        for (int ax : kPassOrder) {
            LineArgs li = line_base(g, t, w, ax);
            li.mode = LM_INIT;
            li.in = w.ph[0];
            li.s_pre = (float)(1.0 / (3.0 * c2 * g.len[ax]));
            PAT_TRY(timed(prof, kLineClass[ax], st, [&] { return launch_line(ax, li, st); }));
        }
        LineArgs la[3];
        for (int ax = 0; ax < 3; ax++) {
            la[ax] = line_base(g, t, w, ax);
            la[ax].mode = LM_STEP;
            la[ax].s_pre = (float)(1.0 / g.len[ax]);
            la[ax].s_mid = (float)(1.0 / g.len[ax]);
            la[ax].s_post = (float)c2;
        }
        const NvtxRange loop("forward time loop");
        for (int n = 0; n + 1 < g.T; n++) {
            float2* cur = w.ph[n & 1];
            float2* nxt = w.ph[(n + 1) & 1];
            for (int ax : kPassOrder) {
                LineArgs& a = la[ax];
                a.in = cur;
                a.out = nxt;
                set_pass_tables(a, t, ax, (n == 0) ? PS_FWD0 : PS_FWD);
                a.flags = (n == 0 ? LF_NO_OLD1 : 0) | (ax == AX ? 0 : LF_ACCUM | LF_LATE_WAIT) |
                          (ax == AZ ? LF_RECORD : 0) | kTrigger[ax];
                a.rec = w.rk + (size_t)(n + 1) * g.nplane;
                PAT_TRY(timed(prof, kLineClass[ax], st, [&] { return launch_line(ax, a, st); }));
            }
        }
    }
    // recorded spectra -> real planes
    PlaneArgs pr = {};
    pr.g = g;
    pr.tw_x = t.tw[AX];
    pr.tw_y = t.tw[AY];
    pr.spec_in = w.rk;
    pr.bs_spec = (long long)g.T * g.nplane;
    pr.out_real = rec;
    pr.bs_real = (long long)g.T * M;
    pr.scale = (float)(1.0 / ((double)g.nx * g.ny));
    PAT_TRY(timed(prof, KC_PLANE_FFT, st, [&] { return launch_plane(pk.irfft, pk, g.T, pr, st); }));
    if (kind != PAT_SAMPLE_FULL)
        PAT_TRY(timed(prof, KC_SAMPLE, st, [&] { return run_sample(g, w, kind, m, rec, f, g.T, st); }));
    return cudaSuccess;
}

cudaError_t run_adjoint(const Geom& g, const DeviceTables& t, const Workspace& w, const Scalars& s,
                        int kind, int m, const float* f, float* p, cudaStream_t st, Profiler* prof) {
    const PlaneKernels pk = plane_kernels_for(g.nx, g.ny);
    const ZKernels zk = z_kernels_for(g.nz);
    if (!pk.rfft || !zk.fwd) return cudaErrorInvalidValue;
    const float* inj = f;
    if (kind != PAT_SAMPLE_FULL) {
        PAT_TRY(timed(prof, KC_SAMPLE, st, [&] { return run_sample_adjoint(g, w, kind, m, f, w.rec, g.T, st); }));
        inj = w.rec;
    }
    if (g.T == 1) return run_inject_only(g, inj, p, st);
    const long long M = g.m_plane;

    // spectra of the T injected planes; lambda^{T-1} = the last one placed on the detection plane
    PlaneArgs pa = {};
    pa.g = g;
    pa.tw_x = t.tw[AX];
    pa.tw_y = t.tw[AY];
    pa.in_real = inj;
    pa.bs_real = (long long)g.T * M;
    pa.spec_out = w.rk;
    pa.bs_spec = (long long)g.T * g.nplane;
    PAT_TRY(timed(prof, KC_PLANE_FFT, st, [&] { return launch_plane(pk.rfft, pk, g.T, pa, st); }));
    const long long s_bs = (long long)g.T * g.nplane;
    PAT_TRY(launch_spread_plane(g, t.tw[AZ], w.rk + (size_t)(g.T - 1) * g.nplane, s_bs, w.ph[0], st));

    LineArgs la[3];
    for (int ax = 0; ax < 3; ax++) {
        la[ax] = line_base(g, t, w, ax);
        la[ax].mode = LM_STEP;
        la[ax].s_pre = (float)(1.0 / g.len[ax]);
        la[ax].s_mid = (float)(1.0 / g.len[ax]);
        la[ax].s_post = (float)(s.dt / s.rho0);
    }
    int cur = 0;
    const NvtxRange loop("adjoint time loop");
    for (int n = g.T - 2; n >= 0; n--) {
        for (int ax : kPassOrder) {
            LineArgs& a = la[ax];
            a.in = w.ph[cur];
            a.out = w.ph[cur ^ 1];
            set_pass_tables(a, t, ax, (n == 0) ? PS_ADJ0 : PS_ADJ);
            a.flags = (n == g.T - 2 ? (LF_NO_OLD1 | LF_NO_OLD2) : 0) | (ax == AX ? 0 : LF_ACCUM | LF_LATE_WAIT) |
                      (ax == AZ ? LF_INJECT : 0) | kTrigger[ax];
            a.inj = w.rk + (size_t)n * g.nplane;
            PAT_TRY(timed(prof, kLineClass[ax], st, [&] { return launch_line(ax, a, st); }));
        }
        cur ^= 1;
    }
    // image terms a_i^2 q_i / (3 c^2) of rho_i^0 = p0 / (3 c^2)
    for (int ax : kPassOrder) {
        LineArgs a = line_base(g, t, w, ax);
        a.mode = LM_FIN;
        a.out = w.ph[cur];
        a.c1[0] = t.coef[CT_FIN][ax];
        a.flags = LF_ACCUM;
        PAT_TRY(timed(prof, kLineClass[ax], st, [&] { return launch_line(ax, a, st); }));
    }
    // p = F^-1 lambda^0
    ZArgs za = {};
    za.g = g;
    za.tw_z = t.tw[AZ];
    za.spec = w.ph[cur];
    za.scale = (float)(1.0 / g.nz);
    PAT_TRY(timed(prof, KC_Z_FFT, st, [&] { return launch_z(zk.inv, zk, za, st); }));
    PlaneArgs pr = {};
    pr.g = g;
    pr.tw_x = t.tw[AX];
    pr.tw_y = t.tw[AY];
    pr.spec_in = w.ph[cur];
    pr.bs_spec = g.nspec;
    pr.out_real = p;
    pr.bs_real = g.nreal;
    pr.scale = (float)(1.0 / ((double)g.nx * g.ny));
    PAT_TRY(timed(prof, KC_PLANE_FFT, st, [&] { return launch_plane(pk.irfft, pk, g.nz, pr, st); }));
    return cudaSuccess;
}

}  // namespace pat

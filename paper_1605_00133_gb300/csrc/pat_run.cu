// pat_run.cu - launch sequences of A and A^T (Sec. 4.3) on one stream.
//
// Forward, T recorded samples (n = 0 is p0 itself):
//   plane_init                     rho_i = p0/(3c^2), record n = 0, (y,x) FFT of p0
//   for n = 0 .. T-2:
//     zpass_grad3  (i k kappa e^{+ik dx/2})     D_i^+ p^n in (z, ky, kx)
//     plane_vel                                  u_i^{n+1/2}; at n = 0 the half-step start
//                                                u^{-1/2} = dt/(2 rho0) D^+ p0 is folded into the
//                                                coefficient as (as/2 - 1) as dt/rho0
//     zpass_each3  (i k kappa e^{-ik dx/2})     D_i^- u_i
//     plane_rho_fwd                              rho_i^{n+1}, p^{n+1}, record n+1, FFT of p^{n+1}
//   sample (C)                                   unless the full plane is recorded
// Adjoint: C^T, then the same four launches per step in reverse time order with the transposed
// coefficients (see the adjoint derivation in the oracle: the last step folds the transpose of
// the initial half step into as (1 - as/2)).
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

int plane_cluster_size(int nx, int ny) { return plane_kernels_for(nx, ny).cs; }

static const char* g_config_what = "";
const char* configure_failure() { return g_config_what; }

cudaError_t configure_kernels(const Geom& g, size_t* plane_smem, size_t* z_smem) {
    PlaneKernels pk = plane_kernels_for(g.nx, g.ny);
    ZKernels zk = z_kernels_for(g.nz);
    if (!pk.vel || !zk.grad3) {
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
    PAT_CFG(cudaFuncSetAttribute(pk.init, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pk.smem_init), "plane_init smem");
    PAT_CFG(cudaFuncSetAttribute(pk.vel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pk.smem3), "plane_vel smem");
    PAT_CFG(cudaFuncSetAttribute(pk.rho_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pk.smem3), "plane_rho_fwd smem");
    PAT_CFG(cudaFuncSetAttribute(pk.rho_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pk.smem3), "plane_rho_adj smem");
    PAT_CFG(cudaFuncSetAttribute(zk.grad3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zk.smem), "zpass_grad3 smem");
    PAT_CFG(cudaFuncSetAttribute(zk.each3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zk.smem), "zpass_each3 smem");
    PAT_CFG(cudaFuncSetAttribute(zk.sum3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zk.smem), "zpass_sum3 smem");
    PAT_CFG(configure_sampling(g), "sampling smem");
#undef PAT_CFG
    g_config_what = "";
    if (plane_smem) *plane_smem = pk.smem3;
    if (z_smem) *z_smem = zk.smem;
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

// Time-loop kernels are launched with programmatic stream serialisation (they call pdl_wait()
// before touching memory), so each one is scheduled while its predecessor drains.
static cudaError_t launch_plane(PlaneKernel k, size_t smem, int cs, const PlaneArgs& a, cudaStream_t st) {
    const Geom& g = a.g;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, g.nz, g.B);
    cfg.blockDim = dim3(kPlaneThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, k, a);
}

static cudaError_t launch_z(ZKernel k, const ZKernels& zk, const ZArgs& a, cudaStream_t st) {
    const int ncols = a.g.ny * a.g.nxh;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((ncols + zk.tc - 1) / zk.tc, a.g.B, k == zk.each3 ? 3 : 1);
    cfg.blockDim = dim3(zk.nt, 1, 1);
    cfg.dynamicSmemBytes = zk.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, a);
}

static PlaneArgs plane_base(const Geom& g, const DeviceTables& t, const Workspace& w) {
    PlaneArgs a = {};
    a.g = g;
    a.tw_x = t.tw[AX];
    a.tw_y = t.tw[AY];
    for (int i = 0; i < 3; i++) a.spec[i] = w.spec[i];
    return a;
}

static ZArgs z_base(const Geom& g, const DeviceTables& t, const Workspace& w, bool plus) {
    ZArgs a = {};
    a.g = g;
    a.tw_z = t.tw[AZ];
    for (int i = 0; i < 3; i++) {
        a.spec[i] = w.spec[i];
        a.dt[i] = plus ? t.dplus[i] : t.dminus[i];
    }
    a.kappaN = t.kappaN;
    return a;
}

static void set_tables(PlaneArgs& a, const DeviceTables& t, int c1, int c2, int c3) {
    for (int i = 0; i < 3; i++) {
        a.A1[i] = t.coef[c1][i];
        a.A2[i] = t.coef[c2][i];
        a.A3[i] = t.coef[c3][i];
    }
}

cudaError_t run_forward(const Geom& g, const DeviceTables& t, const Workspace& w, const Scalars& s,
                        int kind, int m, const float* p0, float* f, cudaStream_t st, Profiler* prof) {
    const PlaneKernels pk = plane_kernels_for(g.nx, g.ny);
    const ZKernels zk = z_kernels_for(g.nz);
    if (!pk.vel || !zk.grad3) return cudaErrorInvalidValue;
    float* rec = (kind == PAT_SAMPLE_FULL) ? f : w.rec;
    const float c2 = (float)(s.c * s.c);

    PlaneArgs pi = plane_base(g, t, w);
    pi.flags = (g.T == 1) ? PF_NO_FWD : 0;
    pi.in_real = p0;
    for (int i = 0; i < 3; i++) pi.st[i] = w.st[3 + i];
    pi.s1 = (float)(1.0 / (3.0 * s.c * s.c));
    pi.rec = rec;
    pi.n_rec = 0;
    PAT_TRY(timed(prof, KC_PLANE_INIT, st, [&] { return launch_plane(pk.init, pk.smem_init, pk.cs, pi, st); }));

    const ZArgs zg = z_base(g, t, w, true);
    const ZArgs zd = z_base(g, t, w, false);
    PlaneArgs pv = plane_base(g, t, w);
    for (int i = 0; i < 3; i++) pv.st[i] = w.st[i];
    PlaneArgs pr = plane_base(g, t, w);
    for (int i = 0; i < 3; i++) pr.st[i] = w.st[3 + i];
    set_tables(pr, t, CT_A2, CT_DF_D, CT_ONE);
    pr.c2 = c2;
    pr.rec = rec;
    for (int n = 0; n + 1 < g.T; n++) {
        PAT_TRY(timed(prof, KC_Z_ONE_TO_THREE, st, [&] { return launch_z(zk.grad3, zk, zg, st); }));
        if (n == 0) {
            set_tables(pv, t, CT_AS2, CT_VF0_G, CT_ONE);
            pv.flags = PF_NO_OLD;
        } else {
            set_tables(pv, t, CT_AS2, CT_VF_G, CT_ONE);
            pv.flags = 0;
        }
        PAT_TRY(timed(prof, KC_PLANE_VEL, st, [&] { return launch_plane(pk.vel, pk.smem3, pk.cs, pv, st); }));
        PAT_TRY(timed(prof, KC_Z_THREE_TO_THREE, st, [&] { return launch_z(zk.each3, zk, zd, st); }));
        pr.n_rec = n + 1;
        pr.flags = (n + 2 == g.T) ? PF_NO_FWD : 0;
        PAT_TRY(timed(prof, KC_PLANE_RHO_FWD, st, [&] { return launch_plane(pk.rho_fwd, pk.smem3, pk.cs, pr, st); }));
    }
    if (kind != PAT_SAMPLE_FULL)
        PAT_TRY(timed(prof, KC_SAMPLE, st, [&] { return run_sample(g, w, kind, m, rec, f, g.T, st); }));
    return cudaSuccess;
}

cudaError_t run_adjoint(const Geom& g, const DeviceTables& t, const Workspace& w, const Scalars& s,
                        int kind, int m, const float* f, float* p, cudaStream_t st, Profiler* prof) {
    const PlaneKernels pk = plane_kernels_for(g.nx, g.ny);
    const ZKernels zk = z_kernels_for(g.nz);
    if (!pk.vel || !zk.grad3) return cudaErrorInvalidValue;
    const float* inj = f;
    if (kind != PAT_SAMPLE_FULL) {
        PAT_TRY(timed(prof, KC_SAMPLE, st, [&] { return run_sample_adjoint(g, w, kind, m, f, w.rec, g.T, st); }));
        inj = w.rec;
    }
    if (g.T == 1) return run_inject_only(g, inj, p, st);
    const float c2 = (float)(s.c * s.c);
    PlaneArgs pq = plane_base(g, t, w);
    for (int i = 0; i < 3; i++) pq.st[i] = w.st[3 + i];
    set_tables(pq, t, CT_A2, CT_ONE, CT_A);
    pq.c2 = c2;
    pq.s0 = (float)(s.dt / s.rho0);
    pq.s1 = (float)(1.0 / (3.0 * s.c * s.c));
    pq.inj = inj;
    pq.out_real = p;
    // q_i^{T-1} = c^2 (injected plane T-1); transform a_i q_i
    pq.flags = PF_NO_OLD;
    pq.n_rec = g.T - 1;
    PAT_TRY(timed(prof, KC_PLANE_RHO_ADJ, st, [&] { return launch_plane(pk.rho_adj, pk.smem3, pk.cs, pq, st); }));

    const ZArgs zg = z_base(g, t, w, true);
    const ZArgs zd = z_base(g, t, w, false);
    PlaneArgs pv = plane_base(g, t, w);
    for (int i = 0; i < 3; i++) pv.st[i] = w.st[i];
    for (int n = g.T - 2; n >= 0; n--) {
        PAT_TRY(timed(prof, KC_Z_THREE_TO_THREE, st, [&] { return launch_z(zk.each3, zk, zg, st); }));
        set_tables(pv, t, CT_AS2, CT_VA_G, (n == 0) ? CT_VA0_OUT : CT_AS);
        pv.flags = (n + 2 == g.T) ? PF_NO_OLD : 0;
        PAT_TRY(timed(prof, KC_PLANE_VEL, st, [&] { return launch_plane(pk.vel, pk.smem3, pk.cs, pv, st); }));
        PAT_TRY(timed(prof, KC_Z_THREE_TO_ONE, st, [&] { return launch_z(zk.sum3, zk, zd, st); }));
        pq.flags = PF_HAVE_LAMBDA | ((n == 0) ? PF_FINAL : 0);
        pq.n_rec = n;
        PAT_TRY(timed(prof, KC_PLANE_RHO_ADJ, st, [&] { return launch_plane(pk.rho_adj, pk.smem3, pk.cs, pq, st); }));
    }
    return cudaSuccess;
}

}  // namespace pat

/*
 * pat.h - C ABI of libpat: the photoacoustic forward operator A, its exact adjoint A^T and the
 * sub-sampling operator C of compressed-sensing PAT (Arridge et al., "Accelerated High-Resolution
 * Photoacoustic Tomography via Compressed Sensing", arXiv:1605.00133), as CUDA kernels for one
 * GB300 GPU (sm_103a).
 *
 * Model (Sec. 2.1, Eq. PATfwd; discrete model Sec. 4.3):
 *   (d_tt - c^2 Laplace) p = 0,  p(t=0) = p0,  d_t p(t=0) = 0,
 * solved by explicit k-space pseudospectral time stepping on an Nz x Ny x Nx grid of voxel size dx
 * with the time step equal to the sampling interval.  The detection plane is the grid plane
 * z = sensor_z (z is the depth axis, the paper's x).  A maps p0 to the plane pressure at the T
 * recorded steps n = 0..T-1 (n = 0 is p0 itself); C samples each recorded plane (Sec. 3.1,
 * Eq. GenScan): all points, a list of single points (rSP / gSP), or binary scrambled-Hadamard
 * patterns (sHd, Sec. 4.3).  Data are f = C A p0 (Eq. Fwd); back-projection is A^T C^T f (Eq. BP).
 *
 * Discretisation fixed by this library (the paper defers it to k-Wave):
 *   kappa(k) = sinc(c dt |k| / 2);  D_i^{+/-} f = Re F^-1[ i k_i kappa exp(+/- i k_i dx/2) F f ]
 *   rho_i^0 = p0/(3c^2),  u_i^{-1/2} = dt/(2 rho0) D_i^+ p0
 *   u_i^{n+1/2} = as_i (as_i u_i^{n-1/2} - dt/rho0 D_i^+ p^n)
 *   rho_i^{n+1} = a_i (a_i rho_i^n - dt rho0 D_i^- u_i^{n+1/2}),   p^{n+1} = c^2 sum_i rho_i^{n+1}
 *   a_i = exp(-alpha_i dt/2), alpha_i = pml_alpha (c/dx) (d/P)^4 at depth d voxels into the
 *   P = pml_size layer on each face (zero inside); as_i on the staggered points j + 1/2.
 *
 * Conventions
 *   Memory: all array arguments named *_dev are device pointers owned by the caller, FP32 (or int32
 *   where stated), contiguous and at least 16-byte aligned.  The library owns its workspace, which
 *   pat_create_grid allocates and pat_destroy_grid frees.
 *   Streams: every call is ordered on the given cudaStream_t (pass NULL for the legacy default
 *   stream) and returns without synchronising the device.
 *   Threads: a grid handle must not be used by two streams or threads at the same time.
 *   Errors: arguments are checked before anything is launched; on failure nothing is launched, the
 *   call returns a non-zero pat_status and pat_last_error() describes it.  No C++ exception crosses
 *   this interface.  There is no CPU fallback: without a usable GPU, calls fail with PAT_ERR_CUDA.
 */
#ifndef PAT_H
#define PAT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PAT_OK = 0,
    PAT_ERR_INVALID_ARG = 1,   /* bad pointer, size, descriptor or index set */
    PAT_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed */
    PAT_ERR_OOM = 3,           /* device workspace could not be allocated */
    PAT_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up (pat_device_status) */
    PAT_ERR_NOT_CONVERGED = 5, /* reserved for iterative solvers */
    PAT_ERR_UNSUPPORTED = 6    /* valid request this build does not handle (e.g. grid too large) */
} pat_status;

/* Sampling operator C (Sec. 3.1, Sec. 4.3). */
typedef enum {
    PAT_SAMPLE_FULL = 0,        /* conventional scan: every plane point, m = Ny*Nx */
    PAT_SAMPLE_POINTS = 1,      /* rSP/gSP: m distinct plane points (row selection) */
    PAT_SAMPLE_HADAMARD01 = 2,  /* sHd, binary 0/1 patterns phi_j(perm[l]) = (1 + H[rows_j][l]) / 2 */
    PAT_SAMPLE_HADAMARDPM = 3   /* sHd, +-1/sqrt(M) patterns phi_j(perm[l]) = H[rows_j][l] / sqrt(M) */
} pat_sampling_kind;

typedef struct pat_grid pat_grid; /* opaque; owns the device workspace and constant tables */

typedef struct {
    int32_t nz, ny, nx;   /* grid size, (z, y, x) with x fastest; each a power of two in [8, 256] */
    double dx;            /* voxel size in metres (isotropic), > 0 */
    double c;             /* sound speed in m/s, > 0 */
    double rho0;          /* ambient density, > 0 (does not affect p) */
    double cfl;           /* used when dt <= 0: dt = cfl * dx / c */
    double dt;            /* time step in seconds (= sampling interval); <= 0 selects cfl */
    int32_t T;            /* number of recorded samples n = 0..T-1, >= 1 */
    int32_t pml_size;     /* absorbing layer thickness in voxels on every face, 0 <= 2*P < min(n) */
    double pml_alpha;     /* absorption at full layer depth, nepers per voxel (e.g. 2.0) */
    int32_t sensor_z;     /* detection plane index in [0, nz); < 0 selects pml_size */
    int32_t batch;        /* number of independent volumes B processed per call, >= 1 */
} pat_grid_desc;

typedef struct {
    int32_t kind;             /* pat_sampling_kind */
    int32_t m;                /* M_c, number of measurements per time step (FULL: ignored) */
    const int32_t* indices;   /* host, POINTS: int32[m] distinct plane indices y*Nx + x */
    const int32_t* perm;      /* host, HADAMARD*: int32[Ny*Nx], a permutation (pattern scramble) */
    const int32_t* rows;      /* host, HADAMARD*: int32[m] distinct Hadamard rows in [0, Ny*Nx) */
} pat_sampling_desc;

/* Create a grid: validates both descriptors, copies the index sets, builds the k-space, PML and
 * FFT tables (in double precision, stored as FP32) and allocates the device workspace on the
 * current CUDA device.  The handle stays bound to that device.  Returns PAT_OK and *out, or an
 * error with *out = NULL.  HADAMARD kinds need Ny*Nx a power of two and at most 32768. */
pat_status pat_create_grid(const pat_grid_desc* desc, const pat_sampling_desc* sampling,
                           pat_grid** out);

/* Free the grid and its device workspace (waits for work queued on the device to finish).
 * NULL is accepted. */
void pat_destroy_grid(pat_grid* grid);

/* Sizes of one batch entry: n_image = Nz*Ny*Nx, n_data = T*m; plus m and the time step dt. Any
 * output pointer may be NULL. */
pat_status pat_grid_info(const pat_grid* grid, int64_t* n_image, int64_t* n_data, int32_t* m,
                         double* dt);

/* Bytes of device workspace the grid holds. */
int64_t pat_workspace_bytes(const pat_grid* grid);

/* f = C A p0 (Sec. 4.3, Eq. Fwd without noise).
 *   p0_dev: float[B][Nz][Ny][Nx] (read only);  f_dev: float[B][T][m] (overwritten).
 * p0_dev and f_dev must not overlap. */
pat_status pat_forward(pat_grid* grid, const float* p0_dev, float* f_dev, void* cuda_stream);

/* p = A^T C^T f (Sec. 4.4, Eq. BP: the exact transpose of pat_forward).
 *   f_dev: float[B][T][m] (read only);  p_dev: float[B][Nz][Ny][Nx] (overwritten).
 * f_dev and p_dev must not overlap. */
pat_status pat_adjoint(pat_grid* grid, const float* f_dev, float* p_dev, void* cuda_stream);

/* f = C A p0 like pat_forward, for callers that cannot allocate device memory when they call the
 * operator (e.g. reconstruction loops that reserve their whole device budget at start-up).  The
 * paper has no counterpart; this is a deployment variant.  It allocates nothing: the time-stepping
 * state, spectra and recorded plane series live in one static device array of 64 MiB that every
 * GPU loading libpat holds until the process exits (64x128x128 with T = 400 and point sampling
 * needs 58 MiB; grids that do not fit are rejected with PAT_ERR_INVALID_ARG and a message giving
 * the bytes needed).  The grid's constant tables and index sets are read, not written.  The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress), so make that first
 * call before any stream capture.  All calls share the one array and every call overwrites it (no
 * part of it needs to start at zero): calls that can overlap on the GPU (other streams, other
 * grids, other threads) race with each other and must be serialised by the caller. */
pat_status pat_forward_noalloc(pat_grid* grid, const float* p0_dev, float* f_dev, void* cuda_stream);

/* The index sets the grid holds on the device, copied back for bit-exact checks of C (Sec. 3.1,
 * Sec. 4.3): POINTS writes the m plane indices to host_idx_or_perm (int32[m]); HADAMARD* writes the
 * scramble permutation to host_idx_or_perm (int32[Ny*Nx]) and the m Hadamard rows to host_rows
 * (int32[m]); FULL writes nothing.  Host buffers owned by the caller; a pointer the kind needs may
 * not be NULL (PAT_ERR_INVALID_ARG).  Synchronous: returns after the copies have completed. */
pat_status pat_get_indices(const pat_grid* grid, int32_t* host_idx_or_perm, int32_t* host_rows);

/* C alone, applied to a plane series (Sec. 3.1, Eq. GenScan per time point):
 *   pbar_dev: float[B][nt][Ny*Nx] -> f_dev: float[B][nt][m].  nt >= 1. */
pat_status pat_sample(pat_grid* grid, const float* pbar_dev, float* f_dev, int32_t nt,
                      void* cuda_stream);

/* C^T alone: f_dev float[B][nt][m] -> pbar_dev float[B][nt][Ny*Nx] (overwritten; rSP zero-fills). */
pat_status pat_sample_adjoint(pat_grid* grid, const float* f_dev, float* pbar_dev, int32_t nt,
                              void* cuda_stream);

/* Positivity-constrained TV denoising, the proximal operator of the TV+ functional (Sec. 4.5
 * Eq. TV+, App. A, App. B Eq. TV+Denoise):  out = argmin_{q >= 0} 1/2 ||q - in||^2 + alpha TV(q),
 * TV(q) = sum over voxels of |forward-difference gradient|_2, Neumann boundary (bc = 0; other
 * values return PAT_ERR_UNSUPPORTED).  Solved by `iters` steps of the accelerated primal-dual
 * hybrid gradient method (tau_0 = sigma_0 = 1/sqrt(12), theta = 1/sqrt(1 + 2 tau)), started at
 * q = max(0, in).  in_dev / out_dev: float[B][Nz][Ny][Nx]; they may alias.  The first call on a
 * grid allocates its prox workspace (9 image-sized FP32 buffers: the input copy, and the dual
 * variable (3) and over-relaxed iterate read from one set and written to the other). */
pat_status pat_tv_prox(pat_grid* grid, const float* in_dev, float* out_dev, double alpha, int32_t iters,
                       int32_t bc, void* cuda_stream);

/* BPppTV+ (Sec. 6.1; the method list's "BP followed by TV+ denoising"): the back-projection
 * A^T C^T f of Eq. BP post-processed by positivity-constrained TV denoising, Eq. TV+Denoise with the
 * back-projection in place of the time-reversal image:
 *   p = argmin_{q >= 0} 1/2 ||q - A^T C^T f||^2 + alpha TV(q),
 * with pat_tv_prox's TV (Neumann boundary) and solver (`iters` primal-dual iterations).  The
 * back-projection is linear in f, so scaling f scales it.  f_dev: float[B][T][m] (read only);
 * p_dev: float[B][Nz][Ny][Nx] (overwritten).  The first call on a grid allocates the prox
 * workspace, like pat_tv_prox. */
pat_status pat_bp_tv(pat_grid* grid, const float* f_dev, float* p_dev, double alpha, int32_t iters,
                     void* cuda_stream);

/* Parameters of pat_bregman_solve (App. B: eta = step_scale / L with step_scale 1.8, up to 5
 * backtracking halvings after a restart, stop when min E has not decreased 5 times in a row). */
typedef struct {
    double lambda;          /* TV weight (>= 0) */
    int32_t outer;          /* Bregman iterations (>= 1; 1 = plain TV+) */
    int32_t inner;          /* FISTA iterations per Bregman step (>= 1; the paper uses 50) */
    int32_t prox_iters;     /* primal-dual iterations per TV prox (>= 1) */
    double L;               /* Lipschitz constant of A^T C^T C A; <= 0: estimate by power iteration */
    int32_t power_iters;    /* power iterations when L <= 0 (>= 1) */
    uint64_t seed;          /* seed of the power-iteration start vector */
    double step_scale;      /* eta = step_scale / L (> 0) */
    int32_t max_backtrack;  /* step halvings after a restart (>= 0) */
    int32_t stall;          /* early stop after this many steps without a new minimum of E (>= 1) */
    /* Checkpoint / resume of the Bregman iteration (device pointers, FP64 [T][m], or NULL): the state
     * between Bregman steps is the image p and the Bregman variable b.  b_in replaces b^0 = 0 (pass
     * the image as warm_dev); b_out receives b after the last step.  A solve of K1 + K2 steps equals a
     * solve of K1 steps followed by one of K2 steps resumed from its image and b_out. */
    const double* b_in;
    double* b_out;
} pat_solve_params;

typedef struct {
    double L;               /* the Lipschitz constant used */
    int32_t inner_total;    /* FISTA iterations done over all Bregman steps */
    int32_t restarts;       /* momentum restarts */
    double energy;          /* final E = 1/2 ||C A p - (f + b)||^2 + lambda TV(p) of the last step */
    int32_t n_residual;     /* entries written to residual (<= 64) */
    double residual[64];    /* ||C A p^k - f|| after Bregman step k (FP64) */
} pat_solve_report;

/* TV+ / TV+Br reconstruction (Sec. 4.5-4.6, Eqs. VarReg, TV+, BregIterA/B; App. B): Bregman
 * iterations p^{k+1} = argmin_{p >= 0} 1/2 ||C A p - (f + b^k)||^2 + lambda TV(p),
 * b^{k+1} = b^k + (f - C A p^{k+1}), b^0 = 0, each solved by FISTA with restart and backtracking
 * (one pat_forward and one pat_adjoint per iteration, plus extra ones on a restart), warm-started
 * from the previous p.  f_dev: float[1][T][m]; warm_dev: float[1][Nz][Ny][Nx] start or NULL (zero);
 * p_out_dev: float[1][Nz][Ny][Nx].  Batch must be 1.  The Bregman variable, the objective and all
 * norms are accumulated in FP64.  The call synchronises the stream after each FP64 reduction (the
 * host takes the restart / stopping decisions).  The first call allocates the solver workspace.
 * report may be NULL. */
pat_status pat_bregman_solve(pat_grid* grid, const float* f_dev, const float* warm_dev, float* p_out_dev,
                             const pat_solve_params* params, pat_solve_report* report, void* cuda_stream);

/* Kernel timing for benchmarks: while enabled, every kernel launch of pat_forward / pat_adjoint is
 * bracketed by CUDA events recorded on the call's stream.  pat_profile_enable(grid, 1) starts (and
 * clears) the record; pat_profile_read waits for the recorded events, then reports per kernel class
 * its name (NUL-terminated, at most 47 characters, in names[48*i]), total device milliseconds and
 * launch count.  Classes: line_x, line_y, line_z (the time step's line passes), plane_fft, z_fft
 * (transforms outside the time loop), sample.  n_classes receives the number written
 * (<= max_classes). */
pat_status pat_profile_enable(pat_grid* grid, int32_t enable);
pat_status pat_profile_read(pat_grid* grid, int32_t max_classes, char* names, double* total_ms,
                            int64_t* launches, int32_t* n_classes);

/* Device-side status of the grid's time-stepping kernels.  They stage their inputs with bulk
 * asynchronous copies and bound every wait for one (about a second); a wait that gives up is
 * recorded in a device word of the grid instead of hanging the GPU, the CTA does not use the tile it
 * waited for (and waits once more, bounded, before it exits), and the outputs of every call since
 * the last check are invalid: repeat those calls.  Synchronises cuda_stream, then reads and clears
 * the record: PAT_OK, or PAT_ERR_TIMEOUT with pat_last_error() naming the copies that never landed.
 * pat_forward and pat_adjoint do not synchronise, so they cannot report this themselves;
 * pat_bregman_solve checks it before returning. */
pat_status pat_device_status(pat_grid* grid, void* cuda_stream);

/* Test hook for the failure path above (the paper has no counterpart): while mask != 0, the line
 * passes of later pat_forward / pat_adjoint calls on this grid leave out the bulk copies of the old
 * state tiles that mask names (bit 1: state 1, bit 2: state 2; grids whose line tiles are 16 KB copy
 * those tiles otherwise and are not affected) and give up waiting for them after `polls` polls
 * (polls >= 1; each suspends for at most about a microsecond).  Nothing is then in flight, so the
 * kernels return normally, their outputs are invalid, and pat_device_status reports
 * PAT_ERR_TIMEOUT.  mask = 0 restores normal operation and the default poll limit. */
pat_status pat_debug_copy_fault(pat_grid* grid, int32_t mask, int32_t polls);

/* Process-wide cap on the device workspace of one grid, in bytes (0, the default: no cap).
 * pat_create_grid computes a grid's workspace on the host and returns PAT_ERR_OOM, before touching
 * the device, when it exceeds the cap: for callers that share the GPU under a memory budget. */
pat_status pat_set_workspace_limit(int64_t bytes);

/* Message for the last failed call on this thread ("" if none). Valid until the next call. */
const char* pat_last_error(void);

/* Library version string. */
const char* pat_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PAT_H */

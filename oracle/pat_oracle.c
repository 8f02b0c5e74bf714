/*
 * FP64 CPU oracle for compressed-sensing photoacoustic tomography
 * (Arridge, Beard, Betcke, Cox, Huynh, Lucka, Ogunlade, Zhang, arXiv:1605.00133).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the CUDA library is
 * checked against.  Only the test-suite, the smoke check and the benchmark's CPU-baseline leg load
 * it.  It shares no code, header, table or constant with the CUDA library.
 *
 * What it computes, in the paper's notation:
 *   A   : initial pressure p0 (R^N, N = Nz*Ny*Nx) -> detection-plane pressure series pbar
 *         (R^{Mt * Ny*Nx}), by explicit k-space pseudospectral time stepping of the 3D linear wave
 *         equation (Eq. "PATfwd", Sec. 2.1; discrete model Sec. 4.3).  The time step equals the
 *         sampling interval (Sec. 4.3) and the plane z = sensor_z is recorded at every step.
 *   A^T : the exact transpose of that recurrence (Sec. 4.3 and Sec. 4.4: the adjoint brings the
 *         data in as a time-dependent source term).
 *   C   : sub-sampling of the detection plane (Sec. 3.1, Eq. "Fwd", Sec. 4.3): random single
 *         points (row selection), or binary scrambled Hadamard patterns applied per time point,
 *         computed through a fast Walsh-Hadamard transform.
 *
 * The paper defers the discretisation to k-Wave.  The scheme written out here (staggered k-space
 * gradient/divergence with the sinc correction kappa, split-field density with a PML of fourth-order
 * profile inside the grid on all six faces) is the reading this library fixes; every formula below
 * is the whole definition.
 *
 * Layout: real fields are [Nz][Ny][Nx] row-major (x fastest); z is the depth axis and the paper's x.
 * Plane series are [T][Ny*Nx].  All arithmetic is double precision.
 *
 * Pins (tests/test_oracle_pins.py): every function is pinned against closed forms, brute force or
 * dense matrices.  Parity unpinned, as readings rather than functions: the absolute reflection
 * level of the PML profile (a chosen profile with no paper value; only its smallness is checked) and
 * the particular scrambled-Hadamard variant (a self-consistent reading of the paper's reference).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
    int32_t nz, ny, nx;
    double dx;        /* voxel size (m), isotropic */
    double c;         /* sound speed (m/s) */
    double rho0;      /* ambient density */
    double dt;        /* time step (s) */
    int32_t T;        /* recorded samples n = 0..T-1 */
    int32_t pml_size; /* PML thickness in voxels on every face */
    double pml_alpha; /* PML absorption in nepers per voxel at full depth */
    int32_t sensor_z; /* index of the detection plane along z */
} or_grid;

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------------------------ */
/* FFT: iterative radix-2 decimation-in-time on a power-of-two length.                          */
/* forward  X[k] = sum_j x[j] exp(-2 pi i j k / n)                                              */
/* inverse  x[j] = (1/n) sum_k X[k] exp(+2 pi i j k / n)                                        */
/* ------------------------------------------------------------------------------------------ */

void or_fft1(cplx* a, int n, int inverse) {
    if (n <= 1) return;
    for (int i = 1, j = 0; i < n; i++) { /* bit-reversal permutation */
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    const double sgn = inverse ? 1.0 : -1.0;
    for (int len = 2; len <= n; len <<= 1) {
        const int half = len / 2;
        for (int k = 0; k < half; k++) {
            const double ang = sgn * 2.0 * M_PI * (double)k / (double)len;
            const cplx w = cos(ang) + I * sin(ang);
            for (int i = 0; i < n; i += len) {
                const cplx u = a[i + k];
                const cplx v = a[i + k + half] * w;
                a[i + k] = u + v;
                a[i + k + half] = u - v;
            }
        }
    }
    if (inverse)
        for (int i = 0; i < n; i++) a[i] /= (double)n;
}

/* Transform of a [nz][ny][nx] complex array along each axis in turn (separable 3D DFT). */
void or_fft3(cplx* a, int nz, int ny, int nx, int inverse) {
    const int dims[3] = {nz, ny, nx};
    const long strides[3] = {(long)ny * nx, nx, 1};
    for (int ax = 0; ax < 3; ax++) {
        const int n = dims[ax];
        const long st = strides[ax];
        const long nlines = (long)nz * ny * nx / n;
#pragma omp parallel
        {
            cplx* buf = (cplx*)malloc(sizeof(cplx) * (size_t)n);
#pragma omp for schedule(static)
            for (long line = 0; line < nlines; line++) {
                /* base offset of this line: enumerate the other two indices */
                long base;
                if (ax == 0) base = line;                                   /* (y,x) */
                else if (ax == 1) base = (line / nx) * (long)ny * nx + line % nx; /* (z,x) */
                else base = line * nx;                                       /* (z,y) */
                for (int j = 0; j < n; j++) buf[j] = a[base + j * st];
                or_fft1(buf, n, inverse);
                for (int j = 0; j < n; j++) a[base + j * st] = buf[j];
            }
            free(buf);
        }
    }
}

/* ------------------------------------------------------------------------------------------ */
/* k-space operators                                                                             */
/* ------------------------------------------------------------------------------------------ */

/* Wavenumber of DFT bin m on an axis of n points spaced dx: 2 pi m/(n dx) for m < n/2,
 * 2 pi (m - n)/(n dx) otherwise (the Nyquist bin m = n/2 is taken negative). */
double or_wavenumber(int m, int n, double dx) {
    const int mm = (m < n / 2) ? m : m - n;
    return 2.0 * M_PI * (double)mm / ((double)n * dx);
}

/* kappa = sinc(c dt |k| / 2) with sinc(x) = sin(x)/x, sinc(0) = 1: the k-space correction that
 * makes the leapfrog time step exact for every plane wave of a homogeneous medium. */
double or_kappa(double kabs, double c, double dt) {
    const double x = 0.5 * c * dt * kabs;
    return (x == 0.0) ? 1.0 : sin(x) / x;
}

/* Staggered spectral derivative along `axis` (0 = z, 1 = y, 2 = x):
 *   D^{s} f = Re F^{-1}[ i k_axis kappa(|k|) exp(s i k_axis dx / 2) F f ],  s = +1 or -1.
 * s = +1 gives the derivative at the points shifted by +dx/2 (velocity grid), s = -1 brings it
 * back.  With transpose = 1 the multiplier is complex-conjugated, which is the transpose of the
 * real linear map (F^{-1} diag(m) F)^T = F^{-1} diag(conj m) F for the unitary-equivalent DFT pair. */
void or_derivative(const or_grid* g, const double* f, double* out, int axis, int s, int transpose) {
    const int nz = g->nz, ny = g->ny, nx = g->nx;
    const long N = (long)nz * ny * nx;
    cplx* a = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    for (long i = 0; i < N; i++) a[i] = f[i];
    or_fft3(a, nz, ny, nx, 0);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        const int iz = (int)(i / ((long)ny * nx));
        const int iy = (int)((i / nx) % ny);
        const int ix = (int)(i % nx);
        const double kz = or_wavenumber(iz, nz, g->dx);
        const double ky = or_wavenumber(iy, ny, g->dx);
        const double kx = or_wavenumber(ix, nx, g->dx);
        const double kabs = sqrt(kz * kz + ky * ky + kx * kx);
        const double ka = (axis == 0) ? kz : (axis == 1) ? ky : kx;
        const double phase = (double)s * ka * g->dx / 2.0;
        cplx m = I * ka * or_kappa(kabs, g->c, g->dt) * (cos(phase) + I * sin(phase));
        if (transpose) m = conj(m);
        a[i] *= m;
    }
    or_fft3(a, nz, ny, nx, 1);
    for (long i = 0; i < N; i++) out[i] = creal(a[i]);
    free(a);
}

/* ------------------------------------------------------------------------------------------ */
/* PML: alpha(d) = pml_alpha * (c / dx) * (d / P)^4 for a point at depth d > 0 (in voxels) into the
 * absorbing layer of thickness P, zero in the interior.  Per half time step the split field is
 * multiplied by a = exp(-alpha dt / 2).  Regular points sit at j, staggered points at j + 1/2;
 * the layer covers positions < P and > n - 1 - P.                                               */
/* ------------------------------------------------------------------------------------------ */

double or_pml_depth(double pos, int n, int P) {
    if (P <= 0) return 0.0;
    if (pos < (double)P) return (double)P - pos;
    if (pos > (double)(n - 1 - P)) return pos - (double)(n - 1 - P);
    return 0.0;
}

double or_pml_factor(const or_grid* g, double pos, int n) {
    const int P = g->pml_size;
    const double d = or_pml_depth(pos, n, P);
    if (d <= 0.0) return 1.0;
    const double r = d / (double)P;
    const double alpha = g->pml_alpha * (g->c / g->dx) * r * r * r * r;
    return exp(-alpha * g->dt / 2.0);
}

/* a_axis at every voxel, on the regular (staggered = 0) or staggered (= 1) grid of that axis */
static void pml_field(const or_grid* g, int axis, int staggered, double* out) {
    const int nz = g->nz, ny = g->ny, nx = g->nx;
    const int n = (axis == 0) ? nz : (axis == 1) ? ny : nx;
    const long N = (long)nz * ny * nx;
    for (long i = 0; i < N; i++) {
        const int iz = (int)(i / ((long)ny * nx));
        const int iy = (int)((i / nx) % ny);
        const int ix = (int)(i % nx);
        const int j = (axis == 0) ? iz : (axis == 1) ? iy : ix;
        out[i] = or_pml_factor(g, (double)j + (staggered ? 0.5 : 0.0), n);
    }
}

static int grid_ok(const or_grid* g) {
    const int d[3] = {g->nz, g->ny, g->nx};
    for (int i = 0; i < 3; i++)
        if (d[i] < 2 || (d[i] & (d[i] - 1))) return 0;
    if (g->T < 1 || g->sensor_z < 0 || g->sensor_z >= g->nz) return 0;
    if (g->pml_size < 0 || 2 * g->pml_size >= g->nz || 2 * g->pml_size >= g->ny ||
        2 * g->pml_size >= g->nx)
        return 0;
    return g->dx > 0 && g->c > 0 && g->dt > 0 && g->rho0 > 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Forward operator A (Sec. 4.3)                                                                 */
/*   rho_i^0 = p0 / (3 c^2),  u_i^{-1/2} = (dt / (2 rho0)) D_i^+ p0,  pbar[0] = p0 on the plane    */
/*   for n = 0 .. T-2:                                                                           */
/*     p^n         = c^2 (rho_x^n + rho_y^n + rho_z^n)                                           */
/*     u_i^{n+1/2} = as_i (as_i u_i^{n-1/2} - (dt / rho0) D_i^+ p^n)                             */
/*     rho_i^{n+1} = a_i (a_i rho_i^n - dt rho0 D_i^- u_i^{n+1/2})                               */
/*     pbar[n+1]   = c^2 (rho_x + rho_y + rho_z)^{n+1} on the plane z = sensor_z                 */
/* With the PML off (a = 1) this reproduces p^n = F^{-1}[cos(n c |k| dt) F p0] exactly, so the      */
/* initial condition dp/dt = 0 of Eq. "PATfwd" holds.                                           */
/* ------------------------------------------------------------------------------------------ */

int or_forward(const or_grid* g, const double* p0, double* pbar) {
    if (!grid_ok(g)) return 1;
    const long N = (long)g->nz * g->ny * g->nx;
    const long M = (long)g->ny * g->nx;
    const double c2 = g->c * g->c, dt = g->dt, rho0 = g->rho0;
    double *rho[3], *u[3], *a[3], *as[3];
    double* p = (double*)malloc(sizeof(double) * N);
    double* tmp = (double*)malloc(sizeof(double) * N);
    for (int i = 0; i < 3; i++) {
        rho[i] = (double*)malloc(sizeof(double) * N);
        u[i] = (double*)malloc(sizeof(double) * N);
        a[i] = (double*)malloc(sizeof(double) * N);
        as[i] = (double*)malloc(sizeof(double) * N);
        pml_field(g, i, 0, a[i]);
        pml_field(g, i, 1, as[i]);
    }
    /* initial state */
    for (int i = 0; i < 3; i++) {
        for (long v = 0; v < N; v++) rho[i][v] = p0[v] / (3.0 * c2);
        or_derivative(g, p0, tmp, i, +1, 0);
        for (long v = 0; v < N; v++) u[i][v] = dt / (2.0 * rho0) * tmp[v];
    }
    memcpy(pbar, p0 + (long)g->sensor_z * M, sizeof(double) * M);

    for (int n = 0; n + 1 < g->T; n++) {
        for (long v = 0; v < N; v++) p[v] = c2 * (rho[0][v] + rho[1][v] + rho[2][v]);
        for (int i = 0; i < 3; i++) {
            or_derivative(g, p, tmp, i, +1, 0);
            for (long v = 0; v < N; v++)
                u[i][v] = as[i][v] * (as[i][v] * u[i][v] - dt / rho0 * tmp[v]);
        }
        for (int i = 0; i < 3; i++) {
            or_derivative(g, u[i], tmp, i, -1, 0);
            for (long v = 0; v < N; v++)
                rho[i][v] = a[i][v] * (a[i][v] * rho[i][v] - dt * rho0 * tmp[v]);
        }
        double* plane = pbar + (long)(n + 1) * M;
        const long off = (long)g->sensor_z * M;
        for (long v = 0; v < M; v++)
            plane[v] = c2 * (rho[0][off + v] + rho[1][off + v] + rho[2][off + v]);
    }
    for (int i = 0; i < 3; i++) { free(rho[i]); free(u[i]); free(a[i]); free(as[i]); }
    free(p); free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Adjoint A^T: reverse-mode transpose of or_forward, statement by statement, run backwards in   */
/* time.  lr_i and lu_i are the adjoint variables of rho_i and u_i.  The plane data enter as a     */
/* source term at every time step (Sec. 4.4).                                                    */
/* ------------------------------------------------------------------------------------------ */

int or_adjoint(const or_grid* g, const double* pbar_adj, double* p_out) {
    if (!grid_ok(g)) return 1;
    const long N = (long)g->nz * g->ny * g->nx;
    const long M = (long)g->ny * g->nx;
    const long off = (long)g->sensor_z * M;
    const double c2 = g->c * g->c, dt = g->dt, rho0 = g->rho0;
    double *lr[3], *lu[3], *a[3], *as[3];
    double* lp = (double*)malloc(sizeof(double) * N);
    double* tmp = (double*)malloc(sizeof(double) * N);
    double* w = (double*)malloc(sizeof(double) * N);
    for (int i = 0; i < 3; i++) {
        lr[i] = (double*)calloc((size_t)N, sizeof(double));
        lu[i] = (double*)calloc((size_t)N, sizeof(double));
        a[i] = (double*)malloc(sizeof(double) * N);
        as[i] = (double*)malloc(sizeof(double) * N);
        pml_field(g, i, 0, a[i]);
        pml_field(g, i, 1, as[i]);
    }
    for (int n = g->T - 1; n >= 1; n--) {
        /* pbar[n] = c^2 sum_i rho_i^n on the plane */
        const double* yn = pbar_adj + (long)n * M;
        for (int i = 0; i < 3; i++)
            for (long v = 0; v < M; v++) lr[i][off + v] += c2 * yn[v];
        /* rho_i^n = a_i (a_i rho_i^{n-1} - dt rho0 D_i^- u_i^{n-1/2}) */
        for (int i = 0; i < 3; i++) {
            for (long v = 0; v < N; v++) w[v] = a[i][v] * lr[i][v];
            or_derivative(g, w, tmp, i, -1, 1); /* (D_i^-)^T w */
            for (long v = 0; v < N; v++) {
                lu[i][v] += -dt * rho0 * tmp[v];
                lr[i][v] = a[i][v] * a[i][v] * lr[i][v];
            }
        }
        /* u_i^{n-1/2} = as_i (as_i u_i^{n-3/2} - (dt/rho0) D_i^+ p^{n-1}) */
        memset(lp, 0, sizeof(double) * N);
        for (int i = 0; i < 3; i++) {
            for (long v = 0; v < N; v++) w[v] = as[i][v] * lu[i][v];
            or_derivative(g, w, tmp, i, +1, 1); /* (D_i^+)^T w */
            for (long v = 0; v < N; v++) {
                lp[v] += -dt / rho0 * tmp[v];
                lu[i][v] = as[i][v] * as[i][v] * lu[i][v];
            }
        }
        /* p^{n-1} = c^2 sum_i rho_i^{n-1} */
        for (int i = 0; i < 3; i++)
            for (long v = 0; v < N; v++) lr[i][v] += c2 * lp[v];
    }
    /* pbar[0] = p0 on the plane */
    memset(p_out, 0, sizeof(double) * N);
    for (long v = 0; v < M; v++) p_out[off + v] += pbar_adj[v];
    /* rho_i^0 = p0 / (3 c^2) and u_i^{-1/2} = (dt / (2 rho0)) D_i^+ p0 */
    for (int i = 0; i < 3; i++) {
        or_derivative(g, lu[i], tmp, i, +1, 1);
        for (long v = 0; v < N; v++)
            p_out[v] += lr[i][v] / (3.0 * c2) + dt / (2.0 * rho0) * tmp[v];
    }
    for (int i = 0; i < 3; i++) { free(lr[i]); free(lu[i]); free(a[i]); free(as[i]); }
    free(lp); free(tmp); free(w);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Sampling operators C and C^T per time point (Sec. 3.1, Sec. 4.3)                              */
/* ------------------------------------------------------------------------------------------ */

/* rSP: f[n][j] = pbar[n][idx[j]] (row selection). */
void or_sample_rsp(int T, int M, const double* pbar, int mc, const int32_t* idx, double* f) {
    for (int n = 0; n < T; n++)
        for (int j = 0; j < mc; j++) f[(long)n * mc + j] = pbar[(long)n * M + idx[j]];
}

/* rSP transpose: zero-filled scatter. */
void or_sample_rsp_T(int T, int M, const double* f, int mc, const int32_t* idx, double* pbar) {
    memset(pbar, 0, sizeof(double) * (size_t)T * M);
    for (int n = 0; n < T; n++)
        for (int j = 0; j < mc; j++) pbar[(long)n * M + idx[j]] += f[(long)n * mc + j];
}

/* Unnormalised Walsh-Hadamard transform in Sylvester (natural) order, in place:
 * w[i] = sum_j (-1)^{popcount(i & j)} v[j], by log2(m) butterfly sweeps. */
void or_fwht(double* v, int m) {
    for (int h = 1; h < m; h <<= 1)
        for (int i = 0; i < m; i += 2 * h)
            for (int j = i; j < i + h; j++) {
                const double x = v[j], y = v[j + h];
                v[j] = x + y;
                v[j + h] = x - y;
            }
}

/* sHd: pattern j acts on the plane through the scrambled Hadamard row R_j:
 *   v[l] = pbar[perm[l]],  w = H v,
 *   0/1 patterns (pm1 = 0): phi_j = (1 + H_{R_j,.}) / 2  ->  f_j = (w[0] + w[R_j]) / 2
 *   +-1 patterns (pm1 = 1): phi_j = H_{R_j,.} / sqrt(M)   ->  f_j = w[R_j] / sqrt(M)
 * (row 0 of the Sylvester matrix is all ones, so w[0] is the plain sum of v). */
void or_sample_shd(int T, int M, const double* pbar, int mc, const int32_t* perm,
                   const int32_t* rows, int pm1, double* f) {
    double* v = (double*)malloc(sizeof(double) * (size_t)M);
    const double s = 1.0 / sqrt((double)M);
    for (int n = 0; n < T; n++) {
        const double* pl = pbar + (long)n * M;
        for (int l = 0; l < M; l++) v[l] = pl[perm[l]];
        or_fwht(v, M);
        for (int j = 0; j < mc; j++)
            f[(long)n * mc + j] = pm1 ? v[rows[j]] * s : 0.5 * (v[0] + v[rows[j]]);
    }
    free(v);
}

/* sHd transpose: z = sum_j f_j phi_j on the scrambled plane, then unscramble:
 *   0/1: z = (sum_j f_j)/2 * 1 + H e / 2,  e[R_j] = f_j (zero elsewhere)
 *   +-1: z = H e / sqrt(M)
 *   pbar[perm[l]] = z[l]   (H is symmetric, so H^T = H). */
void or_sample_shd_T(int T, int M, const double* f, int mc, const int32_t* perm,
                     const int32_t* rows, int pm1, double* pbar) {
    double* e = (double*)malloc(sizeof(double) * (size_t)M);
    const double s = 1.0 / sqrt((double)M);
    for (int n = 0; n < T; n++) {
        const double* fn = f + (long)n * mc;
        memset(e, 0, sizeof(double) * (size_t)M);
        double sum = 0.0;
        for (int j = 0; j < mc; j++) { e[rows[j]] += fn[j]; sum += fn[j]; }
        or_fwht(e, M);
        double* pl = pbar + (long)n * M;
        for (int l = 0; l < M; l++) pl[perm[l]] = pm1 ? e[l] * s : 0.5 * (sum + e[l]);
    }
    free(e);
}

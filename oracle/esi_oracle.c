/*
 * FP64 CPU oracle for the time-domain ESI hot path.
 *
 * TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark call this code; the product library never links, loads or calls it.
 * It shares no code, header or table with the CUDA path.
 *
 * What it computes (all on one shot, fields stored z-major, x fastest, N = nz*ny*nx):
 *
 *  - Acoustic operator (Eq. "wave": A(m)u = (1/v^2) u_tt - Lap u) discretised
 *    O(dt^2, dx^8) as the Numerical-tests section states, with a damping sponge on every
 *    side (absorbing boundary, same section).  Time step n consumes the source q_n and
 *    produces u_{n+1}:
 *        (1+k) u_{n+1} = 2 u_n - (1-k) u_{n-1} + c (Lap8 u_n + q_n),   c = v^2 dt^2,
 *    k = eta dt / 2 the sponge coefficient, u_0 = u_{-1} = 0.
 *  - Sampling R (Eq. "fwi"): d_n = R u_{n+1}, R given as a sparse (node, weight) list.
 *  - Exact discrete adjoint S^T = C M^{-T} R^T, where M is the block lower-triangular
 *    time-stepping matrix above (M U = C Q).  M^T is solved backward in time:
 *        (1+k) mu_j = y_j + 2 mu_{j+1} + Lap8(c mu_{j+1}) - (1-k) mu_{j+2},
 *    y_j = R^T e_{j-1}, and (S^T e)_{j-1} = c mu_j  (Eq. "FWI_lambda", normal equation
 *    right-hand side b = S^H d of the CG section).
 *  - Zero-lag cross-correlation gradient (Eq. "gradient"/"gradewi"): for the misfit
 *    1/2 ||R u - d||^2 the exact discrete derivative with respect to c is
 *        g_c = sum_n mu_{n+1} (Lap8 u_n + q_n),
 *    mu the adjoint field of the residual.
 *  - On-the-fly DTFT (Eq. "dtft"): U(x, f) += u(x, t) exp(+j 2 pi f t) at every state.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* 8th-order central second-derivative weights (Fornberg 1988), index = offset. */
static const double LAP8_W[5] = {
    -205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};

/* u at integer cell (z, y, x); zero outside the grid (homogeneous Dirichlet extension). */
static double cell(const double *u, long nz, long ny, long nx, long z, long y, long x) {
    if (z < 0 || z >= nz || y < 0 || y >= ny || x < 0 || x >= nx) return 0.0;
    return u[(z * ny + y) * nx + x];
}

/* out = Lap8 u  (2D uses the z and x axes; 3D adds y). */
void orc_laplacian(int ndim, long nz, long ny, long nx, double dx, const double *u,
                   double *out) {
    const double inv_dx2 = 1.0 / (dx * dx);
#pragma omp parallel for
    for (long z = 0; z < nz; ++z)
        for (long y = 0; y < ny; ++y)
            for (long x = 0; x < nx; ++x) {
                double s = ndim * LAP8_W[0] * cell(u, nz, ny, nx, z, y, x);
                for (long k = 1; k <= 4; ++k) {
                    s += LAP8_W[k] * (cell(u, nz, ny, nx, z + k, y, x) +
                                      cell(u, nz, ny, nx, z - k, y, x));
                    s += LAP8_W[k] * (cell(u, nz, ny, nx, z, y, x + k) +
                                      cell(u, nz, ny, nx, z, y, x - k));
                    if (ndim == 3)
                        s += LAP8_W[k] * (cell(u, nz, ny, nx, z, y + k, x) +
                                          cell(u, nz, ny, nx, z, y - k, x));
                }
                out[(z * ny + y) * nx + x] = s * inv_dx2;
            }
}

/* Accumulate one state into the DTFT sums: re/im[m][i] += u[i] * exp(+j 2 pi f_m t). */
void orc_dtft_accumulate(long N, const double *u, double t, int nf, const double *freqs,
                         double *re, double *im) {
    for (int m = 0; m < nf; ++m) {
        const double ph = 2.0 * M_PI * freqs[m] * t;
        const double cr = cos(ph), si = sin(ph);
        double *rm = re + (long)m * N, *imm = im + (long)m * N;
        for (long i = 0; i < N; ++i) {
            rm[i] += u[i] * cr;
            imm[i] += u[i] * si;
        }
    }
}

/*
 * Forward modelling of one shot.
 *   c, kappa      : [N] c = v^2 dt^2, kappa = eta dt / 2
 *   q_ext         : [nt][N] extended source, or NULL
 *   point source  : n_src (node, weight) pairs; q_n[node] += weight * wavelet[n]
 *   receivers     : CSR r_ptr[nr+1] into (r_node, r_w); traces[n][r] = sum w u_{n+1}[node]
 *   traces        : [nt][nr] or NULL
 *   s_hist        : [nt][N] or NULL, s_n = Lap8 u_n + q_n (the gradient's forward factor)
 *   u_hist        : [nt+1][N] or NULL, u_0 .. u_nt
 *   DTFT          : nf frequencies; dft_re/dft_im [nf][N] accumulate u_{n+1} at t=(n+1)dt
 */
void orc_forward(int ndim, long nz, long ny, long nx, double dx, double dt, int nt,
                 const double *c, const double *kappa, const double *q_ext, long n_src,
                 const long *src_node, const double *src_w, const double *wavelet, long nr,
                 const long *r_ptr, const long *r_node, const double *r_w, double *traces,
                 double *s_hist, double *u_hist, int nf, const double *freqs, double *dft_re,
                 double *dft_im) {
    const long N = nz * ny * nx;
    double *u_prev = calloc(N, sizeof(double));
    double *u_cur = calloc(N, sizeof(double));
    double *u_next = calloc(N, sizeof(double));
    double *q = calloc(N, sizeof(double));
    double *lap = calloc(N, sizeof(double));
    if (u_hist) memset(u_hist, 0, N * sizeof(double));
    for (int n = 0; n < nt; ++n) {
        if (q_ext)
            memcpy(q, q_ext + (long)n * N, N * sizeof(double));
        else
            memset(q, 0, N * sizeof(double));
        for (long k = 0; k < n_src; ++k) q[src_node[k]] += src_w[k] * wavelet[n];
        orc_laplacian(ndim, nz, ny, nx, dx, u_cur, lap);
#pragma omp parallel for
        for (long i = 0; i < N; ++i) {
            const double s = lap[i] + q[i];
            if (s_hist) s_hist[(long)n * N + i] = s;
            u_next[i] = (2.0 * u_cur[i] - (1.0 - kappa[i]) * u_prev[i] + c[i] * s) /
                        (1.0 + kappa[i]);
        }
        if (traces)
            for (long r = 0; r < nr; ++r) {
                double d = 0.0;
                for (long k = r_ptr[r]; k < r_ptr[r + 1]; ++k) d += r_w[k] * u_next[r_node[k]];
                traces[(long)n * nr + r] = d;
            }
        if (u_hist) memcpy(u_hist + (long)(n + 1) * N, u_next, N * sizeof(double));
        if (nf > 0) orc_dtft_accumulate(N, u_next, (n + 1) * dt, nf, freqs, dft_re, dft_im);
        double *tmp = u_prev;
        u_prev = u_cur;
        u_cur = u_next;
        u_next = tmp;
    }
    free(u_prev);
    free(u_cur);
    free(u_next);
    free(q);
    free(lap);
}

/*
 * Exact discrete adjoint of orc_forward with respect to the extended source, computed as
 * the literal transpose solve M^T mu = R^T e backward in time.
 *   e        : [nt][nr] adjoint data (sample n pairs with state u_{n+1})
 *   out      : [nt][N] or NULL, (S^T e)_n = c * mu_{n+1}
 *   src_adj  : [nt] or NULL, adjoint of the point-source injection:
 *              src_adj[n] = sum_k src_w[k] * (S^T e)_n[src_node[k]]
 *   s_hist, grad_c : if both non-NULL, grad_c[i] += sum_n mu_{n+1}[i] * s_hist[n][i]
 */
void orc_adjoint(int ndim, long nz, long ny, long nx, double dx, int nt, const double *c,
                 const double *kappa, long nr, const long *r_ptr, const long *r_node,
                 const double *r_w, const double *e, double *out, long n_src,
                 const long *src_node, const double *src_w, double *src_adj,
                 const double *s_hist, double *grad_c) {
    const long N = nz * ny * nx;
    double *mu2 = calloc(N, sizeof(double)); /* mu_{j+2} */
    double *mu1 = calloc(N, sizeof(double)); /* mu_{j+1} */
    double *mu0 = calloc(N, sizeof(double)); /* mu_j */
    double *cm = calloc(N, sizeof(double));
    double *lap = calloc(N, sizeof(double));
    double *y = calloc(N, sizeof(double));
    for (int j = nt; j >= 1; --j) {
        memset(y, 0, N * sizeof(double));
        for (long r = 0; r < nr; ++r)
            for (long k = r_ptr[r]; k < r_ptr[r + 1]; ++k)
                y[r_node[k]] += r_w[k] * e[(long)(j - 1) * nr + r];
        for (long i = 0; i < N; ++i) cm[i] = c[i] * mu1[i];
        orc_laplacian(ndim, nz, ny, nx, dx, cm, lap);
#pragma omp parallel for
        for (long i = 0; i < N; ++i)
            mu0[i] = (y[i] + 2.0 * mu1[i] + lap[i] - (1.0 - kappa[i]) * mu2[i]) /
                     (1.0 + kappa[i]);
        if (out)
            for (long i = 0; i < N; ++i) out[(long)(j - 1) * N + i] = c[i] * mu0[i];
        if (src_adj) {
            double a = 0.0;
            for (long k = 0; k < n_src; ++k) a += src_w[k] * c[src_node[k]] * mu0[src_node[k]];
            src_adj[j - 1] = a;
        }
        if (s_hist && grad_c)
            for (long i = 0; i < N; ++i) grad_c[i] += mu0[i] * s_hist[(long)(j - 1) * N + i];
        double *tmp = mu2;
        mu2 = mu1;
        mu1 = mu0;
        mu0 = tmp;
    }
    free(mu2);
    free(mu1);
    free(mu0);
    free(cm);
    free(lap);
    free(y);
}

/* Threads the OpenMP runtime would use for the parallel loops above (1 without OpenMP). */
int orc_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

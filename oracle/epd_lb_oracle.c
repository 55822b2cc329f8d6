/*
 * epd_lb_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of one time step of the hybrid
 * Lattice-Boltzmann / External-Potential-Dynamics method of Heuser, Sevink and
 * Schmid (arXiv:1804.02883).  It exists to check the CUDA path; nothing in the
 * product may call it.  Only the tests, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py load this library.
 *
 * It shares no code, header, table or constant with the CUDA library: it has
 * its own FFT (radix-2, pinned against a naive DFT), its own propagator, its
 * own LB collision written in moment space, and its own implementation of the
 * splitmix64 counter generator used for the initial noise.
 *
 * Every operation follows the paper's statement directly, without blocking or
 * fusion.  The readings taken where the paper is silent are marked READING.
 *
 * Grid layout: row-major [y][x], x fastest; x is the flow axis.  Fields of the
 * three species are stacked as [A, B, S].  LB populations are stacked as
 * [i][y][x] with the D2Q9 velocity order
 *   0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* Parameters of the problem statement (Sec. 2 and Sec. 3).  Lengths in R_G,
 * times in tau = R_G^2/D_S, the LB part in lattice units. */
typedef struct {
    int32_t nx, ny;       /* grid sites per axis (even)                      */
    int32_t ns;           /* contour steps N_s                               */
    int32_t junction_rule; /* field at the A/B junction node: 0 literal, 1 segment-symmetric */
    double dx, dt, rg;    /* grid spacing, time step, gyration radius R_G    */
    double n_seg;         /* segments per chain N                            */
    double f_a;           /* A-fraction q_A of the diblock                   */
    double phi_p;         /* mean polymer volume fraction; solvent 1 - phi_p */
    double chi_ab, chi_as, chi_bs, kappa_h;
    double d_s, d_p;      /* diffusion constants of solvent and monomers     */
    double inv_beta_v;    /* 1/(beta v)                                      */
    double gamma_s, gamma_b, gamma_g; /* MRT relaxation parameters           */
    double f0;            /* reverse-Poiseuille amplitude in units of f*     */
    double noise_amp;     /* amplitude of the initial uniform noise on omega */
    uint64_t seed;
} or_params;

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* FFT (textbook iterative radix-2 Cooley-Tukey; the naive DFT for lengths   */
/* that are not powers of two).                                               */
/* Convention: forward  X[k] = sum_n x[n] exp(-2 pi i k n / N),             */
/*             backward x[n] = sum_k X[k] exp(+2 pi i k n / N)   (no 1/N).  */
/* ------------------------------------------------------------------------ */

void or_dft_naive(const cplx *x, cplx *out, int n, int sign)
{
    for (int k = 0; k < n; k++) {
        long double re = 0.0L, im = 0.0L;
        for (int j = 0; j < n; j++) {
            /* reduce k*j mod n first so the angle stays accurate */
            long long kj = ((long long)k * j) % n;
            long double ang = sign * 2.0L * (long double)M_PI * (long double)kj / (long double)n;
            long double c = cosl(ang), s = sinl(ang);
            long double xr = creal(x[j]), xi = cimag(x[j]);
            re += xr * c - xi * s;
            im += xr * s + xi * c;
        }
        out[k] = (double)re + I * (double)im;
    }
}

void or_fft1d(cplx *x, int n, int sign)
{
    if (n <= 1) return;
    if (n & (n - 1)) {
        /* not a power of two (e.g. the paper's 150-site axes): the DFT by its
         * definition, with the n roots exp(sign 2 pi i t / n) tabulated */
        cplx *out = (cplx *)malloc(sizeof(cplx) * (size_t)n);
        cplx *root = (cplx *)malloc(sizeof(cplx) * (size_t)n);
        for (int t = 0; t < n; t++) {
            double ang = sign * 2.0 * M_PI * (double)t / (double)n;
            root[t] = cos(ang) + I * sin(ang);
        }
        for (int k = 0; k < n; k++) {
            cplx acc = 0.0;
            for (int j = 0; j < n; j++) acc += x[j] * root[(int)(((long long)k * j) % n)];
            out[k] = acc;
        }
        memcpy(x, out, sizeof(cplx) * (size_t)n);
        free(out);
        free(root);
        return;
    }
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = x[i]; x[i] = x[j]; x[j] = t; }
    }
    /* twiddles exp(sign 2 pi i t / n), t < n/2 */
    cplx *tw = (cplx *)malloc(sizeof(cplx) * (size_t)(n / 2));
    for (int t = 0; t < n / 2; t++) {
        double ang = sign * 2.0 * M_PI * (double)t / (double)n;
        tw[t] = cos(ang) + I * sin(ang);
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len / 2, step = n / len;
        for (int i = 0; i < n; i += len) {
            for (int k = 0; k < half; k++) {
                cplx a = x[i + k];
                cplx b = x[i + k + half] * tw[k * step];
                x[i + k] = a + b;
                x[i + k + half] = a - b;
            }
        }
    }
    free(tw);
}

/* 2D transform of a [ny][nx] array: all rows, then all columns. */
void or_fft2d(cplx *a, int ny, int nx, int sign)
{
    for (int y = 0; y < ny; y++) or_fft1d(a + (size_t)y * nx, nx, sign);
    cplx *col = (cplx *)malloc(sizeof(cplx) * (size_t)ny);
    for (int x = 0; x < nx; x++) {
        for (int y = 0; y < ny; y++) col[y] = a[(size_t)y * nx + x];
        or_fft1d(col, ny, sign);
        for (int y = 0; y < ny; y++) a[(size_t)y * nx + x] = col[y];
    }
    free(col);
}

/* Angular wavenumber of FFT index m on an axis of n sites and spacing dx.
 * READING (spectral derivatives): the Nyquist index n/2 carries k = pi/dx in
 * even operators (the Laplacian, the propagator's Fourier factor) and is
 * zeroed in odd ones (first derivatives), since i*k has no real-valued
 * representation there. */
static double wavenumber(int m, int n, double dx)
{
    int mm = (m <= n / 2) ? m : m - n;
    return 2.0 * M_PI * (double)mm / ((double)n * dx);
}
static double wavenumber_odd(int m, int n, double dx)
{
    if (2 * m == n) return 0.0;
    return wavenumber(m, n, dx);
}

/* Spectral derivative of a real field: order 1 along axis (0 = x, 1 = y)
 * multiplies by i*k_axis; order 2 by -k_axis^2; order 0 with axis 2 by
 * -|k|^2 (the Laplacian). */
void or_spectral_op(const or_params *p, const double *f, double *out, int axis, int order)
{
    int nx = p->nx, ny = p->ny;
    size_t n = (size_t)nx * ny;
    cplx *a = (cplx *)malloc(sizeof(cplx) * n);
    for (size_t i = 0; i < n; i++) a[i] = f[i];
    or_fft2d(a, ny, nx, -1);
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            size_t i = (size_t)y * nx + x;
            cplx m;
            if (axis == 2) {
                double kx = wavenumber(x, nx, p->dx), ky = wavenumber(y, ny, p->dx);
                m = -(kx * kx + ky * ky);
            } else if (order == 1) {
                double k = axis == 0 ? wavenumber_odd(x, nx, p->dx) : wavenumber_odd(y, ny, p->dx);
                m = I * k;
            } else {
                double k = axis == 0 ? wavenumber(x, nx, p->dx) : wavenumber(y, ny, p->dx);
                m = -k * k;
            }
            a[i] *= m;
        }
    or_fft2d(a, ny, nx, +1);
    for (size_t i = 0; i < n; i++) out[i] = creal(a[i]) / (double)n;
    free(a);
}

/* ------------------------------------------------------------------------ */
/* Single-chain statistics: Sec. 2, Eqs. (6)-(11).                          */
/* ------------------------------------------------------------------------ */

/* READING: N_A = round(q_A N_s) contour intervals belong to the A block.
 * The paper puts omega_A at s < q_A and omega_B otherwise; at the junction
 * node s_{N_A} = q_A the split step of Eq. (8) can read this two ways:
 *  - junction_rule 0 (literal, the default): contour node j carries
 *    omega_A iff j < N_A, so the junction node takes omega_B; the step over
 *    interval [s_j, s_{j+1}] uses the fields of nodes j and j + 1;
 *  - junction_rule 1 (segment-symmetric): interval j belongs to block A iff
 *    j < N_A and both of its half-steps use that block's field, so the
 *    chain is treated the same way from either end. */
int or_n_a(const or_params *p)
{
    return (int)lround(p->f_a * (double)p->ns);
}

/* Fields of the two half-steps of every contour interval j = 0..ns-1 of one
 * chain (chain 0: g from the A end; chain 1: g' from the B end, which sees
 * the field of position 1 - s): first[j] acts at s_j, second[j] at s_{j+1}. */
static void half_step_fields(const or_params *p, const double *w_a, const double *w_b, int chain,
                             const double **first, const double **second)
{
    int ns = p->ns, na = or_n_a(p);
    for (int j = 0; j < ns; j++) {
        if (p->junction_rule == 1) {
            int jg = chain == 0 ? j : ns - 1 - j; /* the interval of g it covers */
            first[j] = second[j] = (jg < na) ? w_a : w_b;
        } else {
            int j0 = chain == 0 ? j : ns - j, j1 = chain == 0 ? j + 1 : ns - j - 1; /* nodes of g */
            first[j] = (j0 < na) ? w_a : w_b;
            second[j] = (j1 < na) ? w_a : w_b;
        }
    }
}

/* Propagate one chain.  Eq. (8): the contour step from s to s + ds is
 *   g(s+ds) = exp(-N w(s+ds) ds / 2) exp(R_G^2 Laplacian ds) exp(-N w(s) ds / 2) g(s),
 * with the Laplacian factor applied in Fourier space as exp(-R_G^2 |k|^2 ds).
 * first[j], second[j]: the fields of the two half-steps of interval j
 * (half_step_fields).  hist receives g at nodes 0..ns; g at node 0 is g0
 * (1 for Eqs. (6)-(7)). */
static void propagate_chain(const or_params *p, const double *const *first, const double *const *second,
                            const double *g0, double *hist)
{
    int nx = p->nx, ny = p->ny, ns = p->ns;
    size_t n = (size_t)nx * ny;
    double ds = 1.0 / (double)ns;
    double nseg = p->n_seg;
    cplx *work = (cplx *)malloc(sizeof(cplx) * n);
    double *kfac = (double *)malloc(sizeof(double) * n);
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            double kx = wavenumber(x, nx, p->dx), ky = wavenumber(y, ny, p->dx);
            kfac[(size_t)y * nx + x] = exp(-p->rg * p->rg * (kx * kx + ky * ky) * ds);
        }
    for (size_t i = 0; i < n; i++) hist[i] = g0[i];
    for (int j = 0; j < ns; j++) {
        const double *g = hist + (size_t)j * n;
        double *gnext = hist + (size_t)(j + 1) * n;
        const double *wj = first[j], *wj1 = second[j];
        for (size_t i = 0; i < n; i++) work[i] = exp(-nseg * wj[i] * ds / 2.0) * g[i];
        or_fft2d(work, ny, nx, -1);
        for (size_t i = 0; i < n; i++) work[i] *= kfac[i];
        or_fft2d(work, ny, nx, +1);
        for (size_t i = 0; i < n; i++)
            gnext[i] = exp(-nseg * wj1[i] * ds / 2.0) * creal(work[i]) / (double)n;
    }
    free(work);
    free(kfac);
}

/* Forward propagator g (from the A end, Eq. (6)) and backward propagator g'
 * (from the B end, Eq. (7)).  READING: g' sees the field of contour position
 * 1 - s, i.e. at its node j the field of node ns - j; both start from 1.
 * g_hist, gp_hist: (ns+1)*n each.  If g0 is NULL both start from 1,
 * otherwise g starts from g0 and g' from 1. */
void or_propagate(const or_params *p, const double *w_a, const double *w_b,
                  const double *g0, double *g_hist, double *gp_hist)
{
    int ns = p->ns;
    size_t n = (size_t)p->nx * p->ny;
    const double **f1 = (const double **)malloc(sizeof(double *) * (size_t)ns);
    const double **f2 = (const double **)malloc(sizeof(double *) * (size_t)ns);
    double *ones = (double *)malloc(sizeof(double) * n);
    for (size_t i = 0; i < n; i++) ones[i] = 1.0;
    half_step_fields(p, w_a, w_b, 0, f1, f2);
    propagate_chain(p, f1, f2, g0 ? g0 : ones, g_hist);
    half_step_fields(p, w_a, w_b, 1, f1, f2);
    propagate_chain(p, f1, f2, ones, gp_hist);
    free(ones);
    free(f1);
    free(f2);
}

/* READING (contour quadrature, not stated in the paper): the trapezoid rule on
 * [0, s_{N_A}] for the A block and on [s_{N_A}, 1] for the B block. */
static double weight_a(int j, int na, double ds)
{
    if (na == 0 || j > na) return 0.0;
    return (j == 0 || j == na) ? 0.5 * ds : ds;
}
static double weight_b(int j, int na, int ns, double ds)
{
    if (na == ns || j < na) return 0.0;
    return (j == na || j == ns) ? 0.5 * ds : ds;
}

/* Densities, Eqs. (9)-(11), with the partition functions Q_P, Q_S taken as
 * spatial means (READING: the volume V cancels between Q and the prefactor).
 * omega: [A, B, S] fields; phi: [A, B, S] out; q[0] = Q_P, q[1] = Q_S. */
void or_solve(const or_params *p, const double *omega, double *phi, double *q)
{
    int ns = p->ns, na = or_n_a(p);
    size_t n = (size_t)p->nx * p->ny;
    double ds = 1.0 / (double)ns;
    double *g = (double *)malloc(sizeof(double) * n * (size_t)(ns + 1));
    double *gp = (double *)malloc(sizeof(double) * n * (size_t)(ns + 1));
    or_propagate(p, omega, omega + n, NULL, g, gp);

    double q_p = 0.0;
    for (size_t i = 0; i < n; i++) q_p += g[(size_t)ns * n + i];
    q_p /= (double)n;

    for (size_t i = 0; i < n; i++) {
        double ia = 0.0, ib = 0.0;
        for (int j = 0; j <= ns; j++) {
            double prod = g[(size_t)j * n + i] * gp[(size_t)(ns - j) * n + i];
            ia += weight_a(j, na, ds) * prod;
            ib += weight_b(j, na, ns, ds) * prod;
        }
        phi[i] = p->phi_p * ia / q_p;
        phi[n + i] = p->phi_p * ib / q_p;
    }

    const double *w_s = omega + 2 * n;
    double q_s = 0.0;
    for (size_t i = 0; i < n; i++) q_s += exp(-w_s[i]);
    q_s /= (double)n;
    for (size_t i = 0; i < n; i++) phi[2 * n + i] = (1.0 - p->phi_p) * exp(-w_s[i]) / q_s;

    q[0] = q_p;
    q[1] = q_s;
    free(g);
    free(gp);
}

/* ------------------------------------------------------------------------ */
/* The single-chain solve in three dimensions (the extension the paper names  */
/* in Sec. 2 and Sec. 5): Eqs. (6)-(11) on an nz x ny x nx box, layout        */
/* [z][y][x], the Fourier factor exp(-R_G^2 |k|^2 ds) with                    */
/* |k|^2 = kx^2 + ky^2 + kz^2.                                                 */
/* ------------------------------------------------------------------------ */

/* 3D transform: all x rows, then all y columns, then all z pillars. */
void or_fft3d(cplx *a, int nz, int ny, int nx, int sign)
{
    size_t plane = (size_t)nx * ny;
    for (int z = 0; z < nz; z++) or_fft2d(a + (size_t)z * plane, ny, nx, sign);
    cplx *col = (cplx *)malloc(sizeof(cplx) * (size_t)nz);
    for (size_t i = 0; i < plane; i++) {
        for (int z = 0; z < nz; z++) col[z] = a[(size_t)z * plane + i];
        or_fft1d(col, nz, sign);
        for (int z = 0; z < nz; z++) a[(size_t)z * plane + i] = col[z];
    }
    free(col);
}

static void propagate_chain3d(const or_params *p, int nz, const double *const *first, const double *const *second,
                              double *hist)
{
    int nx = p->nx, ny = p->ny, ns = p->ns;
    size_t n = (size_t)nx * ny * nz;
    double ds = 1.0 / (double)ns;
    cplx *work = (cplx *)malloc(sizeof(cplx) * n);
    double *kfac = (double *)malloc(sizeof(double) * n);
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                double kx = wavenumber(x, nx, p->dx), ky = wavenumber(y, ny, p->dx), kz = wavenumber(z, nz, p->dx);
                kfac[((size_t)z * ny + y) * nx + x] = exp(-p->rg * p->rg * (kx * kx + ky * ky + kz * kz) * ds);
            }
    for (size_t i = 0; i < n; i++) hist[i] = 1.0;
    for (int j = 0; j < ns; j++) {
        const double *g = hist + (size_t)j * n;
        double *gnext = hist + (size_t)(j + 1) * n;
        const double *wj = first[j], *wj1 = second[j];
        for (size_t i = 0; i < n; i++) work[i] = exp(-p->n_seg * wj[i] * ds / 2.0) * g[i];
        or_fft3d(work, nz, ny, nx, -1);
        for (size_t i = 0; i < n; i++) work[i] *= kfac[i];
        or_fft3d(work, nz, ny, nx, +1);
        for (size_t i = 0; i < n; i++) gnext[i] = exp(-p->n_seg * wj1[i] * ds / 2.0) * creal(work[i]) / (double)n;
    }
    free(work);
    free(kfac);
}

/* Densities of Eqs. (9)-(11) on the 3D box: omega [A, B, S][z][y][x] ->
 * phi (same layout), q = (Q_P, Q_S) as spatial means.  The same readings as
 * or_solve (junction node, trapezoid quadrature, g' from the B end). */
void or_solve3d(const or_params *p, int nz, const double *omega, double *phi, double *q)
{
    int ns = p->ns, na = or_n_a(p);
    size_t n = (size_t)p->nx * p->ny * nz;
    double ds = 1.0 / (double)ns;
    const double *w_a = omega, *w_b = omega + n, *w_s = omega + 2 * n;
    double *g = (double *)malloc(sizeof(double) * n * (size_t)(ns + 1));
    double *gp = (double *)malloc(sizeof(double) * n * (size_t)(ns + 1));
    const double **f1 = (const double **)malloc(sizeof(double *) * (size_t)ns);
    const double **f2 = (const double **)malloc(sizeof(double *) * (size_t)ns);
    half_step_fields(p, w_a, w_b, 0, f1, f2);
    propagate_chain3d(p, nz, f1, f2, g);
    half_step_fields(p, w_a, w_b, 1, f1, f2);
    propagate_chain3d(p, nz, f1, f2, gp);
    double q_p = 0.0;
    for (size_t i = 0; i < n; i++) q_p += g[(size_t)ns * n + i];
    q_p /= (double)n;
    for (size_t i = 0; i < n; i++) {
        double ia = 0.0, ib = 0.0;
        for (int j = 0; j <= ns; j++) {
            double prod = g[(size_t)j * n + i] * gp[(size_t)(ns - j) * n + i];
            ia += weight_a(j, na, ds) * prod;
            ib += weight_b(j, na, ns, ds) * prod;
        }
        phi[i] = p->phi_p * ia / q_p;
        phi[n + i] = p->phi_p * ib / q_p;
    }
    double q_s = 0.0;
    for (size_t i = 0; i < n; i++) q_s += exp(-w_s[i]);
    q_s /= (double)n;
    for (size_t i = 0; i < n; i++) phi[2 * n + i] = (1.0 - p->phi_p) * exp(-w_s[i]) / q_s;
    q[0] = q_p;
    q[1] = q_s;
    free(g);
    free(gp);
    free(f1);
    free(f2);
}

/* ------------------------------------------------------------------------ */
/* EPD dynamics: Sec. 2, Eqs. (1), (5), and App. C.                          */
/* ------------------------------------------------------------------------ */

/* READING: mu_I = dF/dPhi_I of Eq. (1) with omega as the conjugate field,
 *   mu_I = sum_{J != I} chi_IJ Phi_J + kappa_H (sum_J Phi_J - 1) - omega_I. */
void or_mu(const or_params *p, const double *phi, const double *omega, double *mu)
{
    size_t n = (size_t)p->nx * p->ny;
    for (size_t i = 0; i < n; i++) {
        double pa = phi[i], pb = phi[n + i], ps = phi[2 * n + i];
        double incompress = p->kappa_h * (pa + pb + ps - 1.0);
        mu[i] = p->chi_ab * pb + p->chi_as * ps + incompress - omega[i];
        mu[n + i] = p->chi_ab * pa + p->chi_bs * ps + incompress - omega[n + i];
        mu[2 * n + i] = p->chi_as * pa + p->chi_bs * pb + incompress - omega[2 * n + i];
    }
}

/* Auxiliary convection of omega (App. C, comment 1).  READING: the advective
 * form omega~ = omega - dt v . grad omega, forward Euler, spectral gradient,
 * with the LB velocity converted to physical units v = u_lat dx/dt. */
void or_aux_convection(const or_params *p, const double *omega, const double *vel_lat,
                       double *omega_tilde)
{
    size_t n = (size_t)p->nx * p->ny;
    double vscale = p->dx / p->dt;
    double *gx = (double *)malloc(sizeof(double) * n);
    double *gy = (double *)malloc(sizeof(double) * n);
    for (int s = 0; s < 3; s++) {
        const double *w = omega + (size_t)s * n;
        or_spectral_op(p, w, gx, 0, 1);
        or_spectral_op(p, w, gy, 1, 1);
        for (size_t i = 0; i < n; i++) {
            double vx = vel_lat[i] * vscale, vy = vel_lat[n + i] * vscale;
            omega_tilde[(size_t)s * n + i] = w[i] - p->dt * (vx * gx[i] + vy * gy[i]);
        }
    }
    free(gx);
    free(gy);
}

/* Diffusion step of Eq. (5): omega(t+dt) = omega~ - dt D_I Laplacian mu_I,
 * with mu evaluated at the intermediate densities (App. C, last comment). */
void or_diffusion_update(const or_params *p, const double *omega_tilde, const double *mu,
                         double *omega_new)
{
    size_t n = (size_t)p->nx * p->ny;
    double *lap = (double *)malloc(sizeof(double) * n);
    for (int s = 0; s < 3; s++) {
        double d = (s == 2) ? p->d_s : p->d_p;
        or_spectral_op(p, mu + (size_t)s * n, lap, 2, 0);
        for (size_t i = 0; i < n; i++)
            omega_new[(size_t)s * n + i] = omega_tilde[(size_t)s * n + i] - p->dt * d * lap[i];
    }
    free(lap);
}

/* Unit of force density f* = rho R_G / tau^2 in LB lattice units
 * (dx = dt = rho = 1 on the lattice; tau = R_G^2 / D_S). */
double or_fstar_lattice(const or_params *p)
{
    double tau = p->rg * p->rg / p->d_s;
    double r = p->dt / tau;
    return (p->rg / p->dx) * r * r;
}

/* Force reconstruction, Sec. 2, Eqs. (19)-(20): for each species
 *   f_I(k) = (1/(beta v)) dPhi_I^D(k) / (D_I dt) * i k / |k|^2,
 * summed over I; f(k=0) = 0.  Output in LB lattice units (f* -> lattice).
 * dphi: [A, B, S] composition change over the diffusion step. */
void or_force(const or_params *p, const double *dphi, double *force_lat)
{
    int nx = p->nx, ny = p->ny;
    size_t n = (size_t)nx * ny;
    cplx *fx = (cplx *)malloc(sizeof(cplx) * n);
    cplx *fy = (cplx *)malloc(sizeof(cplx) * n);
    double fstar = or_fstar_lattice(p);
    for (size_t i = 0; i < n; i++) { fx[i] = 0.0; fy[i] = 0.0; }
    cplx *a = (cplx *)malloc(sizeof(cplx) * n);
    for (int s = 0; s < 3; s++) {
        double d = (s == 2) ? p->d_s : p->d_p;
        for (size_t i = 0; i < n; i++) a[i] = dphi[(size_t)s * n + i];
        or_fft2d(a, ny, nx, -1);
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                size_t i = (size_t)y * nx + x;
                double kx = wavenumber(x, nx, p->dx), ky = wavenumber(y, ny, p->dx);
                double k2 = kx * kx + ky * ky;
                if (k2 == 0.0) continue;
                cplx c = p->inv_beta_v * a[i] / (d * p->dt) / k2;
                fx[i] += c * I * wavenumber_odd(x, nx, p->dx);
                fy[i] += c * I * wavenumber_odd(y, ny, p->dx);
            }
    }
    or_fft2d(fx, ny, nx, +1);
    or_fft2d(fy, ny, nx, +1);
    for (size_t i = 0; i < n; i++) {
        force_lat[i] = creal(fx[i]) / (double)n * fstar;
        force_lat[n + i] = creal(fy[i]) / (double)n * fstar;
    }
    free(a);
    free(fx);
    free(fy);
}

/* ------------------------------------------------------------------------ */
/* D2Q9 Lattice Boltzmann: Sec. 2, Eqs. (12), (14)-(16), in lattice units.   */
/* ------------------------------------------------------------------------ */

static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WGT[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                              1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
#define CS2 (1.0 / 3.0)

/* The three D2Q9 ghost-mode basis functions, orthogonal (with weights WGT)
 * to 1, c_a and c_a c_b - c_s^2 delta_ab. */
static double ghost_basis(int g, int i)
{
    double c2 = (double)(CX[i] * CX[i] + CY[i] * CY[i]);
    if (g == 0) return (3.0 * c2 - 4.0) * CX[i];
    if (g == 1) return (3.0 * c2 - 4.0) * CY[i];
    return 4.5 * c2 * c2 - 7.5 * c2 + 1.0;
}

/* Reverse-Poiseuille body force, Eq. (23), in lattice units.
 * READING: node y represents position y + 1/2, so the force flips between
 * nodes ny/2 - 1 and ny/2 (and between ny - 1 and 0). */
double or_poiseuille_force(const or_params *p, int y)
{
    double a = p->f0 * or_fstar_lattice(p);
    return (y < p->ny / 2) ? -a : a;
}

/* Shear viscosity from gamma_s, Eq. (16), lattice units (rho = 1). */
double or_eta(const or_params *p)
{
    return 0.5 * CS2 * (1.0 + p->gamma_s) / (1.0 - p->gamma_s);
}

/* One LB update: collision with force, Eqs. (14)-(15), then streaming,
 * Eq. (12).  pop: pre-collision populations [9][ny][nx], replaced by the
 * populations at t + dt.  force: total force density [2][ny][nx].
 * vel_out: the fluid velocity at the collision, [2][ny][nx].
 *
 * READING (velocity and forcing, after the Dunweg-Ladd mode form the paper
 * cites): u = (j + f/2)/rho; the mass and momentum modes are conserved except
 * j* = j + f; the stress relaxes about Pi_eq(u) = rho c_s^2 I + rho u u with
 * its traceless part scaled by gamma_s and its trace by gamma_b; the force
 * adds Sigma of Eq. (15); the ghost modes relax to zero with gamma_g.
 * READING (Eq. (15) in d = 2): the printed 2/3 and 1/3 are the d = 3 values
 * of 2/d and 1/d; here Sigma = (1+gamma_s)/2 [u f + f u - (u.f) I]
 *                            + (1+gamma_b)/2 (u.f) I. */
void or_lb_step(const or_params *p, double *pop, const double *force, double *vel_out)
{
    int nx = p->nx, ny = p->ny;
    size_t n = (size_t)nx * ny;
    double *post = (double *)malloc(sizeof(double) * 9 * n);
    for (size_t s = 0; s < n; s++) {
        double nloc[9];
        for (int i = 0; i < 9; i++) nloc[i] = pop[(size_t)i * n + s];
        /* moments */
        double rho = 0, jx = 0, jy = 0, pxx = 0, pyy = 0, pxy = 0, mg[3] = {0, 0, 0};
        for (int i = 0; i < 9; i++) {
            rho += nloc[i];
            jx += nloc[i] * CX[i];
            jy += nloc[i] * CY[i];
            pxx += nloc[i] * CX[i] * CX[i];
            pyy += nloc[i] * CY[i] * CY[i];
            pxy += nloc[i] * CX[i] * CY[i];
            for (int g = 0; g < 3; g++) mg[g] += nloc[i] * ghost_basis(g, i);
        }
        double fx = force[s], fy = force[n + s];
        double ux = (jx + 0.5 * fx) / rho, uy = (jy + 0.5 * fy) / rho;
        vel_out[s] = ux;
        vel_out[n + s] = uy;
        /* equilibrium and non-equilibrium stress */
        double exx = rho * CS2 + rho * ux * ux, eyy = rho * CS2 + rho * uy * uy, exy = rho * ux * uy;
        double nxx = pxx - exx, nyy = pyy - eyy, nxy = pxy - exy;
        double tr = nxx + nyy;
        double rxx = p->gamma_s * (nxx - 0.5 * tr) + p->gamma_b * 0.5 * tr;
        double ryy = p->gamma_s * (nyy - 0.5 * tr) + p->gamma_b * 0.5 * tr;
        double rxy = p->gamma_s * nxy;
        /* force contribution Sigma, Eq. (15) read in d = 2 */
        double uf = ux * fx + uy * fy;
        double hs = 0.5 * (1.0 + p->gamma_s), hb = 0.5 * (1.0 + p->gamma_b);
        double sxx = hs * (2.0 * ux * fx - uf) + hb * uf;
        double syy = hs * (2.0 * uy * fy - uf) + hb * uf;
        double sxy = hs * (ux * fy + uy * fx);
        /* post-collision moments */
        double jxs = jx + fx, jys = jy + fy;
        double mxx = exx + rxx + sxx - rho * CS2; /* Pi* - rho c_s^2 I */
        double myy = eyy + ryy + syy - rho * CS2;
        double mxy = exy + rxy + sxy;
        double gnorm[3] = {2.0 / 3.0, 2.0 / 3.0, 4.0};
        for (int i = 0; i < 9; i++) {
            double qxx = CX[i] * CX[i] - CS2, qyy = CY[i] * CY[i] - CS2, qxy = (double)(CX[i] * CY[i]);
            double v = rho + (jxs * CX[i] + jys * CY[i]) / CS2
                     + (mxx * qxx + myy * qyy + 2.0 * mxy * qxy) / (2.0 * CS2 * CS2);
            for (int g = 0; g < 3; g++) v += p->gamma_g * mg[g] * ghost_basis(g, i) / gnorm[g];
            post[(size_t)i * n + s] = WGT[i] * v;
        }
    }
    /* streaming, Eq. (12): n_i(r + c_i, t + 1) = n_i*(r, t), periodic */
    for (int i = 0; i < 9; i++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                int xd = (x + CX[i] + nx) % nx, yd = (y + CY[i] + ny) % ny;
                pop[(size_t)i * n + (size_t)yd * nx + xd] = post[(size_t)i * n + (size_t)y * nx + x];
            }
    free(post);
}

/* ------------------------------------------------------------------------ */
/* D3Q19 collide-stream: the three-dimensional scheme the paper names for the */
/* extension to 3D (Sec. 2), in the same mode form as the D2Q9 update above.  */
/* ------------------------------------------------------------------------ */

static const int C3[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                              {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
                              {-1, 0, 1}, {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double w3(int i) { return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }

/* The hydrodynamic part of a population: the second-order expansion
 *   w_i [rho + j.c_i / c_s^2 + (M : (c_i c_i - c_s^2 I)) / (2 c_s^4)]
 * with M = Pi - rho c_s^2 I, which reproduces rho, j and Pi exactly on D3Q19;
 * the rest of a population is its ghost part. */
static double hydro3(int i, double rho, const double *j, const double m[3][3])
{
    double cj = 0.0, mq = 0.0;
    for (int a = 0; a < 3; a++) {
        cj += j[a] * C3[i][a];
        for (int b = 0; b < 3; b++) mq += m[a][b] * ((double)(C3[i][a] * C3[i][b]) - (a == b ? CS2 : 0.0));
    }
    return w3(i) * (rho + cj / CS2 + mq / (2.0 * CS2 * CS2));
}

/* One D3Q19 update on an nz x ny x nx box ([19][z][y][x]): the collision of
 * or_lb_step in d = 3 (u = (j + f/2)/rho; j* = j + f; the stress relaxes
 * about rho c_s^2 I + rho u u, traceless part by gamma_s, trace by gamma_b;
 * Sigma of Eq. (15) as printed, with its d = 3 constants 2/3 and 1/3; the
 * ghost part scaled by gamma_g), then streaming n_i(r + c_i) = n_i*(r),
 * periodic.  force: total force [3][z][y][x]; vel_out: u [3][z][y][x]. */
void or_lb3d_step(const or_params *p, int nz, double *pop, const double *force, double *vel_out)
{
    int nx = p->nx, ny = p->ny;
    size_t n = (size_t)nx * ny * nz;
    double *post = (double *)malloc(sizeof(double) * 19 * n);
    for (size_t s = 0; s < n; s++) {
        double nl[19], rho = 0.0, j[3] = {0, 0, 0}, pi[3][3] = {{0}};
        for (int i = 0; i < 19; i++) {
            nl[i] = pop[(size_t)i * n + s];
            rho += nl[i];
            for (int a = 0; a < 3; a++) {
                j[a] += nl[i] * C3[i][a];
                for (int b = 0; b < 3; b++) pi[a][b] += nl[i] * C3[i][a] * C3[i][b];
            }
        }
        double f[3], u[3];
        for (int a = 0; a < 3; a++) {
            f[a] = force[(size_t)a * n + s];
            u[a] = (j[a] + 0.5 * f[a]) / rho;
            vel_out[(size_t)a * n + s] = u[a];
        }
        double m_old[3][3], ms[3][3], js[3], neq[3][3], tr = 0.0, uf = 0.0;
        for (int a = 0; a < 3; a++) {
            uf += u[a] * f[a];
            js[a] = j[a] + f[a];
            for (int b = 0; b < 3; b++) {
                m_old[a][b] = pi[a][b] - (a == b ? rho * CS2 : 0.0);
                neq[a][b] = pi[a][b] - (rho * u[a] * u[b] + (a == b ? rho * CS2 : 0.0));
            }
            tr += neq[a][a];
        }
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                double d = a == b ? 1.0 : 0.0;
                double relax = p->gamma_s * (neq[a][b] - d * tr / 3.0) + p->gamma_b * d * tr / 3.0;
                double sigma = 0.5 * (1.0 + p->gamma_s) * (u[a] * f[b] + f[a] * u[b] - d * 2.0 / 3.0 * uf) +
                               d * (1.0 + p->gamma_b) / 3.0 * uf;
                ms[a][b] = rho * u[a] * u[b] + relax + sigma; /* Pi* - rho c_s^2 I */
            }
        for (int i = 0; i < 19; i++) {
            double ghost = nl[i] - hydro3(i, rho, j, m_old);
            post[(size_t)i * n + s] = hydro3(i, rho, js, ms) + p->gamma_g * ghost;
        }
    }
    for (int i = 0; i < 19; i++)
        for (int z = 0; z < nz; z++)
            for (int y = 0; y < ny; y++)
                for (int x = 0; x < nx; x++) {
                    int xd = (x + C3[i][0] + nx) % nx, yd = (y + C3[i][1] + ny) % ny, zd = (z + C3[i][2] + nz) % nz;
                    pop[(size_t)i * n + ((size_t)zd * ny + yd) * nx + xd] = post[(size_t)i * n + ((size_t)z * ny + y) * nx + x];
                }
    free(post);
}

/* ------------------------------------------------------------------------ */
/* Initial state: Sec. 3 (quench), Sec. 4 (flow initialised with Eq. (24)).  */
/* ------------------------------------------------------------------------ */

/* splitmix64 (Steele, Lea and Flood 2014): state += golden gamma, then the
 * variant-13 finaliser. */
uint64_t or_splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

/* READING (the "very small random noise" of Sec. 3): omega_I = a u with u
 * uniform in [-1, 1), independently per species and site; u comes from the
 * top 53 bits of splitmix64(seed ^ splitmix64(counter)), with
 * counter = (species * ny + y) * nx + x. */
double or_noise(uint64_t seed, uint64_t counter)
{
    uint64_t h = or_splitmix64(seed ^ or_splitmix64(counter));
    double u01 = (double)(h >> 11) * (1.0 / 9007199254740992.0);
    return 2.0 * u01 - 1.0;
}

/* Flow field of Eq. (24) at position Y (lattice units). */
double or_flow_profile(const or_params *p, double yy)
{
    double a = p->f0 * or_fstar_lattice(p);
    double ly = (double)p->ny;
    double d = yy - 0.5 * ly;
    return -(a / (2.0 * or_eta(p))) * d * (fabs(d) - 0.5 * ly);
}

/* The LB velocity of the exact discrete steady state of the reverse-Poiseuille
 * flow on nodes at Y = y + 1/2 (derived for gamma_g = 0): Eq. (24) plus
 * f_P(y) (1 - 1/(8 eta)). */
double or_discrete_profile(const or_params *p, int y)
{
    double fp = or_poiseuille_force(p, y);
    return or_flow_profile(p, (double)y + 0.5) + fp * (1.0 - 1.0 / (8.0 * or_eta(p)));
}

/* omega: 3n, pop: 9n (pre-collision), vel: 2n (velocity used by the first
 * convection step).  READING (Sec. 4, "initialized with the flow field"):
 * rho = 1 and pre-collision populations at second-order equilibrium with
 * momentum j = v(y) - f_P(y)/2, so that the first collision sees u = v(y). */
void or_init(const or_params *p, double *omega, double *pop, double *vel)
{
    int nx = p->nx, ny = p->ny;
    size_t n = (size_t)nx * ny;
    for (int s = 0; s < 3; s++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                uint64_t ctr = ((uint64_t)s * (uint64_t)ny + (uint64_t)y) * (uint64_t)nx + (uint64_t)x;
                omega[(size_t)s * n + (size_t)y * nx + x] = p->noise_amp * or_noise(p->seed, ctr);
            }
    for (int y = 0; y < ny; y++) {
        double v = or_discrete_profile(p, y);
        double jx = v - 0.5 * or_poiseuille_force(p, y), jy = 0.0;
        for (int x = 0; x < nx; x++) {
            size_t s = (size_t)y * nx + x;
            vel[s] = v;
            vel[n + s] = 0.0;
            for (int i = 0; i < 9; i++) {
                double cj = CX[i] * jx + CY[i] * jy;
                double jj = jx * jx + jy * jy;
                pop[(size_t)i * n + s] = WGT[i] * (1.0 + cj / CS2 + cj * cj / (2.0 * CS2 * CS2) - jj / (2.0 * CS2));
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* One coupled EPD/LB time step (App. C), CG inversion truncated to its       */
/* starting guess (the auxiliary convection of omega).                        */
/* ------------------------------------------------------------------------ */

/* State in/out: omega (3n), pop (9n), vel (2n).  Outputs: phi (3n) = Phi at
 * t + dt, q[2] = (Q_P, Q_S) of that solve, force (2n) = the polymer force
 * handed to LB (lattice units), phi_tilde (3n, may be NULL). */
void or_step(const or_params *p, double *omega, double *pop, double *vel,
             double *phi, double *q, double *force, double *phi_tilde_out)
{
    int nx = p->nx, ny = p->ny;
    size_t n = (size_t)nx * ny;
    double *wt = (double *)malloc(sizeof(double) * 3 * n);
    double *pt = (double *)malloc(sizeof(double) * 3 * n);
    double *mu = (double *)malloc(sizeof(double) * 3 * n);
    double *dphi = (double *)malloc(sizeof(double) * 3 * n);
    double *ftot = (double *)malloc(sizeof(double) * 2 * n);
    double qt[2];

    /* (1) auxiliary convection of omega with the current flow */
    or_aux_convection(p, omega, vel, wt);
    /* (2) densities at the intermediate fields */
    or_solve(p, wt, pt, qt);
    /* (3) diffusion step of omega with mu at the intermediate densities */
    or_mu(p, pt, wt, mu);
    or_diffusion_update(p, wt, mu, omega);
    /* (4) densities at t + dt */
    or_solve(p, omega, phi, q);
    /* (5) force from the composition change of the diffusion step */
    for (size_t i = 0; i < 3 * n; i++) dphi[i] = phi[i] - pt[i];
    or_force(p, dphi, force);
    /* (6) LB update driven by the polymer force plus the body force */
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            size_t s = (size_t)y * nx + x;
            ftot[s] = force[s] + or_poiseuille_force(p, y);
            ftot[n + s] = force[n + s];
        }
    or_lb_step(p, pop, ftot, vel);
    if (phi_tilde_out) memcpy(phi_tilde_out, pt, sizeof(double) * 3 * n);
    free(wt);
    free(pt);
    free(mu);
    free(dphi);
    free(ftot);
}

/* ------------------------------------------------------------------------ */
/* The exact step of App. C: convection of the composition fields and the    */
/* iterative inversion omega = Phi^{-1}(Phi~) by Fletcher-Reeves CG.          */
/* ------------------------------------------------------------------------ */

/* Convection part of Eq. (2): Phi~_I = Phi_I - dt div(v Phi_I), forward Euler,
 * the divergence of the flux taken spectrally (READING as for every other
 * spatial derivative: continuum wavenumbers, Nyquist bin of a first
 * derivative dropped), v = u_lat dx/dt in physical units. */
void or_convect_phi(const or_params *p, const double *phi, const double *vel_lat, double *phi_tilde)
{
    size_t n = (size_t)p->nx * p->ny;
    double vscale = p->dx / p->dt;
    double *fx = (double *)malloc(sizeof(double) * n);
    double *fy = (double *)malloc(sizeof(double) * n);
    double *dfx = (double *)malloc(sizeof(double) * n);
    double *dfy = (double *)malloc(sizeof(double) * n);
    for (int s = 0; s < 3; s++) {
        const double *f = phi + (size_t)s * n;
        for (size_t i = 0; i < n; i++) {
            fx[i] = vel_lat[i] * vscale * f[i];
            fy[i] = vel_lat[n + i] * vscale * f[i];
        }
        or_spectral_op(p, fx, dfx, 0, 1);
        or_spectral_op(p, fy, dfy, 1, 1);
        for (size_t i = 0; i < n; i++) phi_tilde[(size_t)s * n + i] = f[i] - p->dt * (dfx[i] + dfy[i]);
    }
    free(fx);
    free(fy);
    free(dfx);
    free(dfy);
}

static double dot3(const double *a, const double *b, size_t m)
{
    double s = 0.0;
    for (size_t i = 0; i < m; i++) s += a[i] * b[i];
    return s;
}

/* Inversion of the density map (Sec. 2, the integrator paragraph; App. C,
 * items 2 and 3): find omega with Phi(omega) = Phi~ (target, 3n).
 *
 * Eqs. (9)-(11) give Phi_{A,B} = -(n phi_p / N) d ln Q_P / d omega_{A,B} and
 * Phi_S = -n (1 - phi_p) d ln Q_S / d omega_S (for the polymer up to how the
 * contour quadrature splits the junction node), so the mismatch
 * g = Phi~ - Phi(omega) is n times the gradient of the convex function
 *   G(omega) = <sum_I omega_I Phi~_I> + (phi_p / N) ln Q_P + (1 - phi_p) ln Q_S
 * (<.> the spatial mean), whose Hessian is the two-body correlator P_IJ of
 * Eq. (4) over n.  Fletcher-Reeves nonlinear CG on G (READING: the paper names the
 * method only):
 *   d_0 = -g_0;
 *   line search along d_k by one secant step on dG/dalpha = -(g . d)/n from
 *     alpha = 0 and the trial step alpha_t (1 at k = 0, then the previous
 *     step), falling back to alpha_t when the secant slope is not positive;
 *   d_{k+1} = -g_{k+1} + beta d_k, beta = |g_{k+1}|^2 / |g_k|^2, restarted
 *     as -g_{k+1} when it is not a descent direction (g . d >= 0).
 * Convergence (App. C, item 2): sqrt(sum_I <(Phi~_I - Phi_I)^2>) < tol
 * (N_tr = 1e-8 in the paper).  tol <= 0 runs exactly max_iter iterations.
 *
 * omega: in the starting guess, out the result.  phi (3n), q[2]: out
 * Phi(omega) and (Q_P, Q_S).  stats[0] = residual at the start,
 * stats[1] = residual at the end.  Returns the iterations taken. */
int or_invert(const or_params *p, const double *phi_target, double *omega, double *phi, double *q,
              int max_iter, double tol, double *stats)
{
    size_t n = (size_t)p->nx * p->ny, m = 3 * n;
    double *g = (double *)malloc(sizeof(double) * m);
    double *d = (double *)malloc(sizeof(double) * m);
    double *wtr = (double *)malloc(sizeof(double) * m);
    double *ptr = (double *)malloc(sizeof(double) * m);
    double qt[2];

    or_solve(p, omega, phi, q);
    for (size_t i = 0; i < m; i++) g[i] = phi_target[i] - phi[i];
    double gg = dot3(g, g, m);
    double res = sqrt(gg / (double)n);
    stats[0] = res;
    for (size_t i = 0; i < m; i++) d[i] = -g[i];
    double h0 = -gg, alpha_t = 1.0;
    int it = 0;
    while (it < max_iter && (tol <= 0.0 || res >= tol)) {
        /* slope of G at the trial step */
        for (size_t i = 0; i < m; i++) wtr[i] = omega[i] + alpha_t * d[i];
        or_solve(p, wtr, ptr, qt);
        double ht = 0.0;
        for (size_t i = 0; i < m; i++) ht += (phi_target[i] - ptr[i]) * d[i];
        double den = h0 - ht;
        double alpha = den < 0.0 ? alpha_t * h0 / den : alpha_t;
        /* the step and the new mismatch */
        for (size_t i = 0; i < m; i++) omega[i] += alpha * d[i];
        or_solve(p, omega, phi, q);
        for (size_t i = 0; i < m; i++) g[i] = phi_target[i] - phi[i];
        double gg_new = dot3(g, g, m), gd = dot3(g, d, m);
        double beta = gg > 0.0 ? gg_new / gg : 0.0;
        h0 = -gg_new + beta * gd;
        if (h0 >= 0.0) {
            for (size_t i = 0; i < m; i++) d[i] = -g[i];
            h0 = -gg_new;
        } else {
            for (size_t i = 0; i < m; i++) d[i] = -g[i] + beta * d[i];
        }
        gg = gg_new;
        res = sqrt(gg / (double)n);
        alpha_t = alpha;
        it++;
    }
    stats[1] = res;
    free(g);
    free(d);
    free(wtr);
    free(ptr);
    return it;
}

/* The exact step of App. C: like or_step, but the intermediate fields are
 * the inversion of the convected densities,
 *   Phi~ = Phi(t) - dt div(v Phi(t)),  omega~ = Phi^{-1}(Phi~)
 * (CG started from the auxiliary convection of omega), and the diffusion
 * step and the force use Phi(omega~).  phi: in Phi(t), out Phi(t + dt).
 * stats[0..2] = iterations, residual before and after the inversion.
 * max_iter = 0 gives or_step exactly. */
void or_step_exact(const or_params *p, double *omega, double *pop, double *vel, double *phi, double *q,
                   double *force, int max_iter, double tol, double *stats)
{
    int nx = p->nx, ny = p->ny;
    size_t n = (size_t)nx * ny;
    double *wt = (double *)malloc(sizeof(double) * 3 * n);
    double *target = (double *)malloc(sizeof(double) * 3 * n);
    double *pt = (double *)malloc(sizeof(double) * 3 * n);
    double *mu = (double *)malloc(sizeof(double) * 3 * n);
    double *dphi = (double *)malloc(sizeof(double) * 3 * n);
    double *ftot = (double *)malloc(sizeof(double) * 2 * n);
    double qt[2], rs[2];

    /* (1) convection: the target densities and the starting guess */
    or_convect_phi(p, phi, vel, target);
    or_aux_convection(p, omega, vel, wt);
    /* (2) omega~ = Phi^{-1}(Phi~) and Phi(omega~) */
    int it = or_invert(p, target, wt, pt, qt, max_iter, tol, rs);
    /* (3)-(6) as in or_step */
    or_mu(p, pt, wt, mu);
    or_diffusion_update(p, wt, mu, omega);
    or_solve(p, omega, phi, q);
    for (size_t i = 0; i < 3 * n; i++) dphi[i] = phi[i] - pt[i];
    or_force(p, dphi, force);
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            size_t s = (size_t)y * nx + x;
            ftot[s] = force[s] + or_poiseuille_force(p, y);
            ftot[n + s] = force[n + s];
        }
    or_lb_step(p, pop, ftot, vel);
    stats[0] = (double)it;
    stats[1] = rs[0];
    stats[2] = rs[1];
    free(wt);
    free(target);
    free(pt);
    free(mu);
    free(dphi);
    free(ftot);
}

/* ------------------------------------------------------------------------ */
/* The coupled step on a 3D box: the 2D step's operations with spectral       */
/* derivatives along x, y and z, the 3D single-chain solve and D3Q19.         */
/* ------------------------------------------------------------------------ */

/* Spectral operator on a real [z][y][x] field: op 0, 1, 2 = d/dx, d/dy, d/dz
 * (Nyquist bin of the derivative's axis dropped), op 3 = the Laplacian. */
void or_spectral_op3d(const or_params *p, int nz, const double *f, double *out, int op)
{
    int nx = p->nx, ny = p->ny;
    size_t n = (size_t)nx * ny * nz;
    cplx *a = (cplx *)malloc(sizeof(cplx) * n);
    for (size_t i = 0; i < n; i++) a[i] = f[i];
    or_fft3d(a, nz, ny, nx, -1);
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                size_t i = ((size_t)z * ny + y) * nx + x;
                cplx m;
                if (op == 3) {
                    double kx = wavenumber(x, nx, p->dx), ky = wavenumber(y, ny, p->dx), kz = wavenumber(z, nz, p->dx);
                    m = -(kx * kx + ky * ky + kz * kz);
                } else {
                    double k = op == 0 ? wavenumber_odd(x, nx, p->dx) : op == 1 ? wavenumber_odd(y, ny, p->dx)
                                                                          : wavenumber_odd(z, nz, p->dx);
                    m = I * k;
                }
                a[i] *= m;
            }
    or_fft3d(a, nz, ny, nx, +1);
    for (size_t i = 0; i < n; i++) out[i] = creal(a[i]) / (double)n;
    free(a);
}

/* Force of Eqs. (19)-(20) on the 3D box: f(k) = (1/(beta v)) sum_I dPhi_I(k) /
 * (D_I dt) i k / |k|^2, in lattice units, [3][z][y][x]. */
void or_force3d(const or_params *p, int nz, const double *dphi, double *force_lat)
{
    int nx = p->nx, ny = p->ny;
    size_t n = (size_t)nx * ny * nz;
    double fstar = or_fstar_lattice(p);
    cplx *fc[3], *a = (cplx *)malloc(sizeof(cplx) * n);
    for (int c = 0; c < 3; c++) {
        fc[c] = (cplx *)malloc(sizeof(cplx) * n);
        for (size_t i = 0; i < n; i++) fc[c][i] = 0.0;
    }
    for (int s = 0; s < 3; s++) {
        double d = (s == 2) ? p->d_s : p->d_p;
        for (size_t i = 0; i < n; i++) a[i] = dphi[(size_t)s * n + i];
        or_fft3d(a, nz, ny, nx, -1);
        for (int z = 0; z < nz; z++)
            for (int y = 0; y < ny; y++)
                for (int x = 0; x < nx; x++) {
                    size_t i = ((size_t)z * ny + y) * nx + x;
                    double kx = wavenumber(x, nx, p->dx), ky = wavenumber(y, ny, p->dx), kz = wavenumber(z, nz, p->dx);
                    double k2 = kx * kx + ky * ky + kz * kz;
                    if (k2 == 0.0) continue;
                    cplx c = p->inv_beta_v * a[i] / (d * p->dt) / k2;
                    fc[0][i] += c * I * wavenumber_odd(x, nx, p->dx);
                    fc[1][i] += c * I * wavenumber_odd(y, ny, p->dx);
                    fc[2][i] += c * I * wavenumber_odd(z, nz, p->dx);
                }
    }
    for (int c = 0; c < 3; c++) {
        or_fft3d(fc[c], nz, ny, nx, +1);
        for (size_t i = 0; i < n; i++) force_lat[(size_t)c * n + i] = creal(fc[c][i]) / (double)n * fstar;
        free(fc[c]);
    }
    free(a);
}

/* One coupled step on the 3D box, in the order of or_step: auxiliary
 * convection of omega with the 3D gradient, the 3D solve at omega~, the
 * diffusion step with the 3D Laplacian, the 3D solve at omega(t + dt), the
 * 3D force plus the reverse-Poiseuille body force of Eq. (23) along x
 * (a function of y), one D3Q19 update.  State: omega (3n), pop (19n,
 * pre-collision), vel (3n, the velocity handed to the convection); outputs
 * phi (3n), q[2], force (3n, the polymer force). */
void or_step3d(const or_params *p, int nz, double *omega, double *pop, double *vel, double *phi, double *q,
               double *force)
{
    int nx = p->nx, ny = p->ny;
    size_t n = (size_t)nx * ny * nz;
    double vscale = p->dx / p->dt;
    double *wt = (double *)malloc(sizeof(double) * 3 * n);
    double *pt = (double *)malloc(sizeof(double) * 3 * n);
    double *mu = (double *)malloc(sizeof(double) * 3 * n);
    double *tmp = (double *)malloc(sizeof(double) * n);
    double *ftot = (double *)malloc(sizeof(double) * 3 * n);
    double qt[2];
    /* (1) auxiliary convection */
    for (int s = 0; s < 3; s++) {
        const double *w = omega + (size_t)s * n;
        for (size_t i = 0; i < n; i++) wt[(size_t)s * n + i] = w[i];
        for (int a = 0; a < 3; a++) {
            or_spectral_op3d(p, nz, w, tmp, a);
            for (size_t i = 0; i < n; i++) wt[(size_t)s * n + i] -= p->dt * vel[(size_t)a * n + i] * vscale * tmp[i];
        }
    }
    /* (2) densities at omega~ */
    or_solve3d(p, nz, wt, pt, qt);
    /* (3) mu (as or_mu) and the diffusion step */
    for (size_t i = 0; i < n; i++) {
        double pa = pt[i], pb = pt[n + i], ps = pt[2 * n + i];
        double inc = p->kappa_h * (pa + pb + ps - 1.0);
        mu[i] = p->chi_ab * pb + p->chi_as * ps + inc - wt[i];
        mu[n + i] = p->chi_ab * pa + p->chi_bs * ps + inc - wt[n + i];
        mu[2 * n + i] = p->chi_as * pa + p->chi_bs * pb + inc - wt[2 * n + i];
    }
    for (int s = 0; s < 3; s++) {
        double d = (s == 2) ? p->d_s : p->d_p;
        or_spectral_op3d(p, nz, mu + (size_t)s * n, tmp, 3);
        for (size_t i = 0; i < n; i++) omega[(size_t)s * n + i] = wt[(size_t)s * n + i] - p->dt * d * tmp[i];
    }
    /* (4) densities at t + dt, (5) force */
    or_solve3d(p, nz, omega, phi, q);
    for (size_t i = 0; i < 3 * n; i++) mu[i] = phi[i] - pt[i];
    or_force3d(p, nz, mu, force);
    /* (6) D3Q19 with the polymer force plus the body force */
    for (size_t i = 0; i < 3 * n; i++) ftot[i] = force[i];
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) ftot[((size_t)z * ny + y) * nx + x] += or_poiseuille_force(p, y);
    or_lb3d_step(p, nz, pop, ftot, vel);
    free(wt);
    free(pt);
    free(mu);
    free(tmp);
    free(ftot);
}

/* Observables: sigma of Eq. (21) = mean |Phi_A + Phi_B - phi_p|. */
double or_sigma(const or_params *p, const double *phi)
{
    size_t n = (size_t)p->nx * p->ny;
    double s = 0.0;
    for (size_t i = 0; i < n; i++) s += fabs(phi[i] + phi[n + i] - p->phi_p);
    return s / (double)n;
}

/* ------------------------------------------------------------------------ */
/* Analysis of the polymer distribution Phi_P = Phi_A + Phi_B (Sec. 3,       */
/* Sec. 4): sigma_Delta, the channel width Y_2^P, particles and their        */
/* gyration tensors.                                                         */
/* ------------------------------------------------------------------------ */

/* sigma_Delta of Eq. (22): mean |Phi_P^a - Phi_P^b| of two runs on one grid. */
double or_sigma_delta(const or_params *p, const double *phi_a, const double *phi_b)
{
    size_t n = (size_t)p->nx * p->ny;
    double s = 0.0;
    for (size_t i = 0; i < n; i++) s += fabs((phi_a[i] + phi_a[n + i]) - (phi_b[i] + phi_b[n + i]));
    return s / (double)n;
}

/* Y_2^P of Eq. (30).  READING: the box holds two opposite Poiseuille
 * channels, y in [0, L_y/2) and [L_y/2, L_y), each of width L_y/2 with its
 * centre at L_y/4 and 3 L_y/4, and y of Eq. (30) is the distance across the
 * channel from its centre; site row y sits at (y + 1/2) dx (the LB node
 * positions), and the integrals are sums over all sites of both channels:
 *   Y_2^P = sqrt( sum y_c^2 Phi_P / (phi_p sum y_c^2) ). */
double or_width(const or_params *p, const double *phi)
{
    int nx = p->nx, ny = p->ny;
    size_t n = (size_t)nx * ny;
    double h = 0.5 * (double)ny;
    double num = 0.0, den = 0.0;
    for (int y = 0; y < ny; y++) {
        double yy = (double)y + 0.5;
        double centre = yy < h ? 0.5 * h : 1.5 * h;
        double yc = (yy - centre) * p->dx;
        for (int x = 0; x < nx; x++) {
            size_t i = (size_t)y * nx + x;
            num += yc * yc * (phi[i] + phi[n + i]);
            den += yc * yc;
        }
    }
    return sqrt(num / (p->phi_p * den));
}

/* Particles (Sec. 4): connected clusters of sites with Phi_P >= threshold
 * (0.5 in the paper).  READING: clusters connect nearest neighbours (4 per
 * site) across the periodic boundaries.  Clusters are numbered in the order
 * of their first site in row-major order.  labels (n): particle number or -1.
 * Per particle k < max_out, stats[10 k ...] =
 *   sites, content N = sum Phi_P, centre x, centre y (in [0, L)), G_xx, G_xy,
 *   G_yy of Eq. (27), R and c of Eq. (28), c_rel of Eq. (29),
 * with G from the double sum of Eq. (27) over the particle's sites, r^i - r^j
 * the shortest periodic separation (READING; exact for particles narrower
 * than half the box), positions (x, y) dx.  Returns the number of particles. */
int or_particles(const or_params *p, const double *phi, double threshold, int *labels, double *stats, int max_out)
{
    int nx = p->nx, ny = p->ny;
    size_t n = (size_t)nx * ny;
    int *queue = (int *)malloc(sizeof(int) * n);
    int *members = (int *)malloc(sizeof(int) * n);
    for (size_t i = 0; i < n; i++) labels[i] = -1;
    int count = 0;
    for (size_t s0 = 0; s0 < n; s0++) {
        if (labels[s0] != -1 || phi[s0] + phi[n + s0] < threshold) continue;
        /* breadth-first search of the cluster of s0 */
        int head = 0, tail = 0, m = 0;
        labels[s0] = count;
        queue[tail++] = (int)s0;
        while (head < tail) {
            int s = queue[head++];
            members[m++] = s;
            int x = s % nx, y = s / nx;
            int nb[4] = {y * nx + (x + 1) % nx, y * nx + (x + nx - 1) % nx, ((y + 1) % ny) * nx + x,
                         ((y + ny - 1) % ny) * nx + x};
            for (int k = 0; k < 4; k++) {
                int t = nb[k];
                if (labels[t] == -1 && phi[t] + phi[n + t] >= threshold) {
                    labels[t] = count;
                    queue[tail++] = t;
                }
            }
        }
        if (count < max_out) {
            double *st = stats + (size_t)10 * count;
            double content = 0.0;
            for (int a = 0; a < m; a++) content += phi[members[a]] + phi[n + members[a]];
            /* Eq. (27): G_nm = 1/(2 N^2) sum_i sum_j Phi_i Phi_j (r_n^i - r_n^j)(r_m^i - r_m^j) */
            double gxx = 0.0, gxy = 0.0, gyy = 0.0, mx = 0.0, my = 0.0;
            int x0 = members[0] % nx, y0 = members[0] / nx;
            for (int a = 0; a < m; a++) {
                int ia = members[a];
                double wa = phi[ia] + phi[n + ia];
                int xa = ia % nx, ya = ia / nx;
                /* centre: content-weighted mean of the shortest offsets from the first site */
                int ox = xa - x0, oy = ya - y0;
                if (2 * ox > nx) ox -= nx;
                if (2 * ox <= -nx) ox += nx;
                if (2 * oy > ny) oy -= ny;
                if (2 * oy <= -ny) oy += ny;
                mx += wa * ox;
                my += wa * oy;
                for (int b = 0; b < m; b++) {
                    int ib = members[b];
                    double wb = phi[ib] + phi[n + ib];
                    int dxs = xa - ib % nx, dys = ya - ib / nx;
                    if (2 * dxs > nx) dxs -= nx;
                    if (2 * dxs <= -nx) dxs += nx;
                    if (2 * dys > ny) dys -= ny;
                    if (2 * dys <= -ny) dys += ny;
                    double rx = dxs * p->dx, ry = dys * p->dx;
                    gxx += wa * wb * rx * rx;
                    gxy += wa * wb * rx * ry;
                    gyy += wa * wb * ry * ry;
                }
            }
            double f = 1.0 / (2.0 * content * content);
            gxx *= f;
            gxy *= f;
            gyy *= f;
            double cx = fmod(x0 + mx / content + nx, (double)nx) * p->dx;
            double cy = fmod(y0 + my / content + ny, (double)ny) * p->dx;
            /* Eq. (28): eigenvalues of the 2 x 2 tensor, c = l+ - l-, R = sqrt(l+ + l-); Eq. (29) */
            double tr = gxx + gyy, dd = sqrt(0.25 * (gxx - gyy) * (gxx - gyy) + gxy * gxy);
            double lp = 0.5 * tr + dd, lm = 0.5 * tr - dd;
            double c = lp - lm, r = sqrt(lp + lm);
            st[0] = (double)m;
            st[1] = content;
            st[2] = cx;
            st[3] = cy;
            st[4] = gxx;
            st[5] = gxy;
            st[6] = gyy;
            st[7] = r;
            st[8] = c;
            st[9] = r > 0.0 ? c * c / (r * r * r * r) : 0.0;
        }
        count++;
    }
    free(queue);
    free(members);
    return count;
}

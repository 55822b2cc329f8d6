// epd.cu -- EPD part of the hybrid LB/EPD step of arXiv:1804.02883 on sm_103a:
//   auxiliary convection of omega (App. C, item 1),
//   diffusion step omega <- omega~ - dt D_I Lap mu_I (Sec. 2, Eq. (5); App. C),
//   force reconstruction from the composition change (Sec. 2, Eqs. (19)-(20)).
//
// Spatial derivatives are spectral with continuum wavenumbers; first
// derivatives drop the Nyquist bin, the Laplacian keeps it.  d/dx and d2/dx2
// act on rows only and d/dy, d2/dy2 on columns only, so each operator is one
// row pass plus one column pass; two real fields travel as one complex field.
// These transforms run in FP64 in both precision modes.
#include <cmath>

#include "common.cuh"
#include "engine.h"

namespace epdlb {

enum RowMode { ROW_GRAD = 0, ROW_LAP = 1, ROW_FWD_S = 2, ROW_INV_FORCE = 3 };
enum ColMode { COL_CONVECT = 0, COL_DIFFUSE = 1, COL_FORCE = 2 };

struct EpdK {
    GroupGeom g;
    const double *omega, *omega_t, *phi, *phi_t;
    double *omega_dst;
    double2 *cz;  // [run][4][n]
    const void *vel;
    void *force;
    int bulk_double;
    const double2 *twx, *twy;
    int rows, logc;
};

__device__ __forceinline__ double kvec(int m, int n, double dx) { return 2.0 * 3.14159265358979323846 * (double)signed_bin(m, n) / ((double)n * dx); }
__device__ __forceinline__ double kvec_odd(int m, int n, double dx) { return (2 * m == n) ? 0.0 : kvec(m, n, dx); }

// Chemical potential of Eq. (1): mu_I = sum_{J != I} chi_IJ Phi_J + kappa_H (sum Phi - 1) - omega_I.
__device__ __forceinline__ double2 mu_pair(const GroupGeom &g, const double *phi, const double *om, long long n, long long i, int pair)
{
    const double pa = phi[i], pb = phi[n + i], ps = phi[2 * n + i];
    const double inc = g.kappa_h * (pa + pb + ps - 1.0);
    if (pair == 0)
        return make_double2(g.chi_ab * pb + g.chi_as * ps + inc - om[i], g.chi_ab * pa + g.chi_bs * ps + inc - om[n + i]);
    return make_double2(g.chi_as * pa + g.chi_bs * pb + inc - om[2 * n + i], 0.0);
}

__device__ __forceinline__ double2 vel_at(const EpdK &k, size_t idx)
{
    if (k.bulk_double) return reinterpret_cast<const double2 *>(k.vel)[idx];
    const float2 v = reinterpret_cast<const float2 *>(k.vel)[idx];
    return make_double2((double)v.x, (double)v.y);
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) epd_row(EpdK k)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const GroupGeom &g = k.g;
    const int nx = g.nx, logx = g.logx, rows = k.rows, tile = rows * nx;
    double2 *a = reinterpret_cast<double2 *>(smem_raw);
    double2 *b = a + tile;
    double2 *tw = b + tile;
    const int run = blockIdx.y, pair = blockIdx.z;
    const long long n = g.n;
    const long long base = (long long)blockIdx.x * tile;
    for (int i = threadIdx.x; i < nx / 2; i += blockDim.x) tw[i] = k.twx[i];
    for (int i = threadIdx.x; i < tile; i += blockDim.x) {
        const long long s = base + i;
        double2 v;
        if (MODE == ROW_GRAD) {
            const double *om = k.omega + (size_t)run * 3 * n;
            v = pair == 0 ? make_double2(om[s], om[n + s]) : make_double2(om[2 * n + s], 0.0);
        } else if (MODE == ROW_LAP) {
            v = mu_pair(g, k.phi_t + (size_t)run * 3 * n, k.omega_t + (size_t)run * 3 * n, n, s, pair);
        } else if (MODE == ROW_FWD_S) {
            // S = sum_I dPhi_I^D / D_I, dPhi^D = Phi(t+dt) - Phi~ (Eq. (19))
            const double *p1 = k.phi + (size_t)run * 3 * n, *p0 = k.phi_t + (size_t)run * 3 * n;
            const double sa = (p1[s] - p0[s]) + (p1[n + s] - p0[n + s]);
            v = make_double2(sa / g.d_p + (p1[2 * n + s] - p0[2 * n + s]) / g.d_s, 0.0);
        } else {
            v = k.cz[((size_t)run * 4 + 2) * n + s];
        }
        a[i] = v;
    }
    __syncthreads();
    const int logb = ilog2(rows);
    double2 *r = a, *o = b;
    if (MODE != ROW_INV_FORCE) {
        r = fft_smem<double, false, false>(a, b, logx, logb, nx, 1, tw);
        o = (r == a) ? b : a;
        if (MODE != ROW_FWD_S) {
            for (int i = threadIdx.x; i < tile; i += blockDim.x) {
                const int m = i & (nx - 1);
                double2 v = r[i];
                if (MODE == ROW_GRAD) {  // i kx / nx
                    const double kk = kvec_odd(m, nx, g.dx) / (double)nx;
                    v = make_double2(-kk * v.y, kk * v.x);
                } else {                 // -kx^2 / nx
                    const double kk = kvec(m, nx, g.dx);
                    v = cscale(v, -kk * kk / (double)nx);
                }
                r[i] = v;
            }
            __syncthreads();
        }
    }
    if (MODE != ROW_FWD_S) r = fft_smem<double, true, false>(r, o, logx, logb, nx, 1, tw);
    for (int i = threadIdx.x; i < tile; i += blockDim.x) {
        const long long s = base + i;
        if (MODE == ROW_INV_FORCE) {
            const double2 f = cscale(r[i], 1.0 / (double)nx);
            if (k.bulk_double) reinterpret_cast<double2 *>(k.force)[(size_t)run * n + s] = f;
            else reinterpret_cast<float2 *>(k.force)[(size_t)run * n + s] = make_float2((float)f.x, (float)f.y);
        } else {
            const int plane = (MODE == ROW_FWD_S) ? 2 : pair;
            k.cz[((size_t)run * 4 + plane) * n + s] = r[i];
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) epd_col(EpdK k)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const GroupGeom &g = k.g;
    const int ny = g.ny, nx = g.nx, logy = g.logy, logc = k.logc, C = 1 << logc, tile = ny << logc;
    double2 *a = reinterpret_cast<double2 *>(smem_raw);
    double2 *b = a + tile;
    double2 *tw = b + tile;
    const int run = blockIdx.y, pair = blockIdx.z, x0 = blockIdx.x << logc;
    const long long n = g.n;
    for (int i = threadIdx.x; i < ny / 2; i += blockDim.x) tw[i] = k.twy[i];
    for (int i = threadIdx.x; i < tile; i += blockDim.x) {
        const long long s = (long long)(i >> logc) * nx + x0 + (i & (C - 1));
        double2 v;
        if (MODE == COL_CONVECT) {
            const double *om = k.omega + (size_t)run * 3 * n;
            v = pair == 0 ? make_double2(om[s], om[n + s]) : make_double2(om[2 * n + s], 0.0);
        } else if (MODE == COL_DIFFUSE) {
            v = mu_pair(g, k.phi_t + (size_t)run * 3 * n, k.omega_t + (size_t)run * 3 * n, n, s, pair);
        } else {
            v = k.cz[((size_t)run * 4 + 2) * n + s];
        }
        a[i] = v;
    }
    __syncthreads();
    double2 *r = fft_smem<double, false, true>(a, b, logy, logc, 1, C, tw);
    double2 *o = (r == a) ? b : a;
    for (int i = threadIdx.x; i < tile; i += blockDim.x) {
        const int my = i >> logc;
        double2 v = r[i];
        if (MODE == COL_CONVECT) {       // i ky / ny
            const double kk = kvec_odd(my, ny, g.dx) / (double)ny;
            v = make_double2(-kk * v.y, kk * v.x);
        } else if (MODE == COL_DIFFUSE) { // -ky^2 / ny
            const double kk = kvec(my, ny, g.dx);
            v = cscale(v, -kk * kk / (double)ny);
        } else {
            // f(k) = (1/(beta v)) S(k) / dt * i k / |k|^2, Eq. (20), in lattice units;
            // f_x + i f_y is real + i real, so one transform carries both:
            // multiply by c (i kx - ky) / |k|^2 and invert.
            const int mx = x0 + (i & (C - 1));
            const double kx = kvec(mx, nx, g.dx), ky = kvec(my, ny, g.dx);
            const double k2 = kx * kx + ky * ky;
            if (k2 == 0.0) {
                v = make_double2(0.0, 0.0);
            } else {
                const double c = g.inv_beta_v * g.fstar / (g.dt * k2 * (double)ny);
                const double2 m = make_double2(-c * kvec_odd(my, ny, g.dx), c * kvec_odd(mx, nx, g.dx));
                v = cmul(v, m);
            }
        }
        r[i] = v;
    }
    __syncthreads();
    r = fft_smem<double, true, true>(r, o, logy, logc, 1, C, tw);
    for (int i = threadIdx.x; i < tile; i += blockDim.x) {
        const long long s = (long long)(i >> logc) * nx + x0 + (i & (C - 1));
        const double2 dy = r[i];
        if (MODE == COL_FORCE) {
            k.cz[((size_t)run * 4 + 2) * n + s] = dy;
        } else if (MODE == COL_CONVECT) {
            // omega~ = omega - dt v . grad omega, v = u_lat dx/dt
            const double2 dx = k.cz[((size_t)run * 4 + pair) * n + s];
            const double2 u = vel_at(k, (size_t)run * n + s);
            const double ux = u.x * g.vscale, uy = u.y * g.vscale;
            const double *om = k.omega + (size_t)run * 3 * n;
            double *ot = k.omega_dst + (size_t)run * 3 * n;
            if (pair == 0) {
                ot[s] = om[s] - g.dt * (ux * dx.x + uy * dy.x);
                ot[n + s] = om[n + s] - g.dt * (ux * dx.y + uy * dy.y);
            } else {
                ot[2 * n + s] = om[2 * n + s] - g.dt * (ux * dx.x + uy * dy.x);
            }
        } else {
            // omega(t+dt) = omega~ - dt D_I Lap mu_I
            const double2 lx = k.cz[((size_t)run * 4 + pair) * n + s];
            const double *ot = k.omega_t + (size_t)run * 3 * n;
            double *om = k.omega_dst + (size_t)run * 3 * n;
            if (pair == 0) {
                om[s] = ot[s] - g.dt * g.d_p * (lx.x + dy.x);
                om[n + s] = ot[n + s] - g.dt * g.d_p * (lx.y + dy.y);
            } else {
                om[2 * n + s] = ot[2 * n + s] - g.dt * g.d_s * (lx.x + dy.x);
            }
        }
    }
}

static EpdK make_k(Group &G)
{
    EpdK k;
    k.g = G.g;
    k.omega = G.omega;
    k.omega_t = G.omega_t;
    k.phi = G.phi;
    k.phi_t = G.phi_t;
    k.omega_dst = nullptr;
    k.cz = G.cz;
    k.vel = G.vel;
    k.force = G.force;
    k.bulk_double = G.prec == EPD_LB_PLAIN_FP64;
    k.twx = G.twx_d;
    k.twy = G.twy_d;
    k.rows = G.sh.rows_epd;
    k.logc = ilog2(G.sh.cols_epd);
    return k;
}

static size_t row_smem(const Group &G) { return (size_t)2 * G.sh.rows_epd * G.g.nx * sizeof(double2) + (G.g.nx / 2) * sizeof(double2); }
static size_t col_smem(const Group &G) { return (size_t)2 * G.sh.cols_epd * G.g.ny * sizeof(double2) + (G.g.ny / 2) * sizeof(double2); }

cudaError_t launch_aux_convection(Group &G, cudaStream_t s)
{
    EpdK k = make_k(G);
    k.omega_dst = G.omega_t;
    epd_row<ROW_GRAD><<<dim3(G.g.ny / G.sh.rows_epd, G.g.nruns, 2), kThreads, row_smem(G), s>>>(k);
    epd_col<COL_CONVECT><<<dim3(G.g.nx / G.sh.cols_epd, G.g.nruns, 2), kThreads, col_smem(G), s>>>(k);
    return cudaGetLastError();
}

cudaError_t launch_diffusion(Group &G, cudaStream_t s)
{
    EpdK k = make_k(G);
    k.omega_dst = G.omega;
    epd_row<ROW_LAP><<<dim3(G.g.ny / G.sh.rows_epd, G.g.nruns, 2), kThreads, row_smem(G), s>>>(k);
    epd_col<COL_DIFFUSE><<<dim3(G.g.nx / G.sh.cols_epd, G.g.nruns, 2), kThreads, col_smem(G), s>>>(k);
    return cudaGetLastError();
}

cudaError_t launch_force(Group &G, cudaStream_t s)
{
    EpdK k = make_k(G);
    epd_row<ROW_FWD_S><<<dim3(G.g.ny / G.sh.rows_epd, G.g.nruns, 1), kThreads, row_smem(G), s>>>(k);
    epd_col<COL_FORCE><<<dim3(G.g.nx / G.sh.cols_epd, G.g.nruns, 1), kThreads, col_smem(G), s>>>(k);
    epd_row<ROW_INV_FORCE><<<dim3(G.g.ny / G.sh.rows_epd, G.g.nruns, 1), kThreads, row_smem(G), s>>>(k);
    return cudaGetLastError();
}

cudaError_t configure_epd_kernels()
{
    const int lim = 200 * 1024;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(epd_row<ROW_GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(epd_row<ROW_LAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(epd_row<ROW_FWD_S>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(epd_row<ROW_INV_FORCE>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(epd_col<COL_CONVECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(epd_col<COL_DIFFUSE>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    return cudaFuncSetAttribute(epd_col<COL_FORCE>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

} // namespace epdlb

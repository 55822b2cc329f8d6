// epd.cu -- EPD part of the hybrid LB/EPD step of arXiv:1804.02883 on sm_103a:
//   auxiliary convection of omega (App. C, item 1),
//   diffusion step omega <- omega~ - dt D_I Lap mu_I (Sec. 2, Eq. (5); App. C),
//   force reconstruction from the composition change (Sec. 2, Eqs. (19)-(20)),
//   convection of the composition fields Phi~ = Phi - dt div(v Phi) (the
//   convective part of Eq. (2); the exact step of App. C).
//
// Spatial derivatives are spectral with continuum wavenumbers; first
// derivatives drop the Nyquist bin, the Laplacian keeps it.  d/dx and d2/dx2
// act on rows only and d/dy, d2/dy2 on columns only, so each operator is one
// row pass plus one column pass; two real fields travel as one complex field.
//
// The fields (omega, Phi) are FP64.  The transforms run in the type TT: FP64
// in PLAIN_FP64, FP32 in MIXED_FP32.  In FP32 the transformed quantities are
// small differences: mu_I minus its homogeneous value (the constant drops
// out of every derivative, and FP32 rounding then scales with the
// fluctuations rather than with mu itself), omega (zero-mean noise), and
// dPhi^D.  Pointwise combinations with the fields are done in FP64.
#include <atomic>
#include <cmath>
#include <cstdlib>

#include "common.cuh"
#include "engine.h"
#include "fft8.cuh"

namespace epdlb {

enum RowMode { ROW_GRAD = 0, ROW_LAP = 1, ROW_FWD_S = 2, ROW_INV_FORCE = 3, ROW_DIVX = 4 };
enum ColMode { COL_CONVECT = 0, COL_DIFFUSE = 1, COL_FORCE = 2, COL_DIVY = 3 };

struct EpdK {
    GroupGeom g;
    const double *omega, *omega_t, *phi, *phi_t;
    double *omega_dst;
    double *phi_dst;  // convected densities (ROW_DIVX / COL_DIVY)
    void *cz;  // [run][4][n] complex of the transform type
    const void *vel;
    void *force;
    int bulk_double;
    const void *twx, *twy;  // twiddles of the transform type
    const float2 *tab8x, *tab8y;  // pass tables of each axis' best radix plan (FP32 radix-8/16 kernels)
    const float2 *tab16y, *tab8y_r8;  // column tables of the radix-16 and radix-8 plans (tile-dependent)
    int rows, logc, cols;  // tile rows (row passes), columns and their log2 (column passes; logc when pow2)
    double kunit_x, kunit_y;  // 2 pi / (n dx) per axis
    double mu_ref[3];         // mu_I at the homogeneous composition, omega = 0
    double phibar[3];         // the homogeneous composition
};

// signed wavenumber of bin m; odd operators drop the Nyquist bin
template <typename TT> __device__ __forceinline__ TT kvec(int m, int n, TT unit) { return unit * (TT)signed_bin(m, n); }
template <typename TT> __device__ __forceinline__ TT kvec_odd(int m, int n, TT unit) { return (2 * m == n) ? (TT)0 : kvec<TT>(m, n, unit); }

// Chemical potential of Eq. (1), mu_I = sum_{J != I} chi_IJ Phi_J + kappa_H (sum Phi - 1) - omega_I,
// minus its homogeneous value (computed in FP64).
__device__ __forceinline__ double2 mu_pair(const EpdK &k, const double *phi, const double *om, long long n, long long i, int pair)
{
    const GroupGeom &g = k.g;
    const double pa = phi[i], pb = phi[n + i], ps = phi[2 * n + i];
    const double inc = g.kappa_h * (pa + pb + ps - 1.0);
    if (pair == 0)
        return make_double2(g.chi_ab * pb + g.chi_as * ps + inc - om[i] - k.mu_ref[0],
                            g.chi_ab * pa + g.chi_bs * ps + inc - om[n + i] - k.mu_ref[1]);
    return make_double2(g.chi_as * pa + g.chi_bs * pb + inc - om[2 * n + i] - k.mu_ref[2], 0.0);
}

// The same in FP32 from the FP64 deviations dPhi_J = Phi_J - Phi-bar_J:
// mu_I - mu_I(Phi-bar, 0) = sum_{J != I} chi_IJ dPhi_J + kappa_H sum_J dPhi_J - omega_I
// (linear in Phi), so FP32 rounding scales with the fluctuations.
__device__ __forceinline__ float2 mu_pair_f(const EpdK &k, const double *phi, const double *om, long long n, long long i, int pair)
{
    const GroupGeom &g = k.g;
    const float da = (float)(phi[i] - k.phibar[0]), db = (float)(phi[n + i] - k.phibar[1]),
                dsv = (float)(phi[2 * n + i] - k.phibar[2]);
    const float inc = (float)g.kappa_h * (da + db + dsv);
    if (pair == 0)
        return make_float2((float)g.chi_ab * db + (float)g.chi_as * dsv + inc - (float)om[i],
                           (float)g.chi_ab * da + (float)g.chi_bs * dsv + inc - (float)om[n + i]);
    return make_float2((float)g.chi_as * da + (float)g.chi_bs * db + inc - (float)om[2 * n + i], 0.f);
}

__device__ __forceinline__ double2 vel_at(const EpdK &k, size_t idx)
{
    if (k.bulk_double) return reinterpret_cast<const double2 *>(k.vel)[idx];
    const float2 v = reinterpret_cast<const float2 *>(k.vel)[idx];
    return make_double2((double)v.x, (double)v.y);
}

template <typename TT> __device__ __forceinline__ V2<TT> to_tt(double2 v) { return mk<TT>((TT)v.x, (TT)v.y); }
template <typename TT> __device__ __forceinline__ double2 to_d(V2<TT> v) { return make_double2((double)v.x, (double)v.y); }

template <typename TT, int MODE>
__global__ void __launch_bounds__(kThreads) epd_row(EpdK k)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const GroupGeom &g = k.g;
    const bool p2 = g.pow2;
    const int nx = g.nx, logx = g.logx, rows = k.rows, tile = rows * nx, ntw = p2 ? nx / 2 : nx;
    V2<TT> *a = reinterpret_cast<V2<TT> *>(smem_raw);
    V2<TT> *b = a + tile;
    V2<TT> *tw = b + tile;
    const int run = blockIdx.y, pair = blockIdx.z;
    const long long n = g.n;
    const long long base = (long long)blockIdx.x * tile;
    V2<TT> *cz = reinterpret_cast<V2<TT> *>(k.cz);
    const V2<TT> *twg = reinterpret_cast<const V2<TT> *>(k.twx);
    for (int i = threadIdx.x; i < ntw; i += blockDim.x) tw[i] = twg[i];
    for (int i = threadIdx.x; i < tile; i += blockDim.x) {
        const long long s = base + i;
        V2<TT> v;
        if (MODE == ROW_GRAD) {
            const double *om = k.omega + (size_t)run * 3 * n;
            v = pair == 0 ? mk<TT>((TT)om[s], (TT)om[n + s]) : mk<TT>((TT)om[2 * n + s], (TT)0);
        } else if (MODE == ROW_LAP) {
            v = to_tt<TT>(mu_pair(k, k.phi_t + (size_t)run * 3 * n, k.omega_t + (size_t)run * 3 * n, n, s, pair));
        } else if (MODE == ROW_FWD_S) {
            // S = sum_I dPhi_I^D / D_I, dPhi^D = Phi(t+dt) - Phi~ (Eq. (19))
            const double *p1 = k.phi + (size_t)run * 3 * n, *p0 = k.phi_t + (size_t)run * 3 * n;
            const double sa = (p1[s] - p0[s]) + (p1[n + s] - p0[n + s]);
            v = mk<TT>((TT)(sa / g.d_p + (p1[2 * n + s] - p0[2 * n + s]) / g.d_s), (TT)0);
        } else if (MODE == ROW_DIVX) {
            // x flux v_x Phi_I, v = u_lat dx/dt
            const double *ph = k.phi + (size_t)run * 3 * n;
            const double vx = vel_at(k, (size_t)run * n + s).x * g.vscale;
            v = pair == 0 ? mk<TT>((TT)(vx * ph[s]), (TT)(vx * ph[n + s])) : mk<TT>((TT)(vx * ph[2 * n + s]), (TT)0);
        } else {
            v = cz[((size_t)run * 4 + 2) * n + s];
        }
        a[i] = v;
    }
    __syncthreads();
    const int logb = p2 ? ilog2(rows) : 0;
    V2<TT> *r = a, *o = b;
    if (MODE != ROW_INV_FORCE) {
        r = p2 ? fft_smem<TT, false, false>(a, b, logx, logb, nx, 1, tw)
               : fft_smem_mr<TT, false, false>(a, b, nx, g.nfx, g.fx, rows, nx, 1, tw);
        o = (r == a) ? b : a;
        if (MODE != ROW_FWD_S) {
            const TT unit = (TT)k.kunit_x, inv_n = (TT)(1.0 / (double)nx);
            for (int i = threadIdx.x; i < tile; i += blockDim.x) {
                const int m = p2 ? i & (nx - 1) : i % nx;
                V2<TT> v = r[i];
                if (MODE == ROW_GRAD || MODE == ROW_DIVX) {  // i kx / nx
                    const TT kk = kvec_odd<TT>(m, nx, unit) * inv_n;
                    v = mk<TT>(-kk * v.y, kk * v.x);
                } else {                 // -kx^2 / nx
                    const TT kk = kvec<TT>(m, nx, unit);
                    v = cscale(v, -kk * kk * inv_n);
                }
                r[i] = v;
            }
            __syncthreads();
        }
    }
    if (MODE != ROW_FWD_S)
        r = p2 ? fft_smem<TT, true, false>(r, o, logx, logb, nx, 1, tw)
               : fft_smem_mr<TT, true, false>(r, o, nx, g.nfx, g.fx, rows, nx, 1, tw);
    for (int i = threadIdx.x; i < tile; i += blockDim.x) {
        const long long s = base + i;
        if (MODE == ROW_INV_FORCE) {
            const V2<TT> f = cscale(r[i], (TT)(1.0 / (double)nx));
            if (k.bulk_double) reinterpret_cast<double2 *>(k.force)[(size_t)run * n + s] = make_double2((double)f.x, (double)f.y);
            else reinterpret_cast<float2 *>(k.force)[(size_t)run * n + s] = make_float2((float)f.x, (float)f.y);
        } else {
            const int plane = (MODE == ROW_FWD_S) ? 2 : pair;
            cz[((size_t)run * 4 + plane) * n + s] = r[i];
        }
    }
}

template <typename TT, int MODE>
__global__ void __launch_bounds__(kThreads) epd_col(EpdK k)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const GroupGeom &g = k.g;
    const bool p2 = g.pow2;
    const int ny = g.ny, nx = g.nx, logy = g.logy, logc = k.logc, C = k.cols, tile = ny * C, ntw = p2 ? ny / 2 : ny;
    V2<TT> *a = reinterpret_cast<V2<TT> *>(smem_raw);
    V2<TT> *b = a + tile;
    V2<TT> *tw = b + tile;
    const int run = blockIdx.y, pair = blockIdx.z, x0 = blockIdx.x * C;
    // row and column of tile element i
    auto row_of = [&](int i) { return p2 ? i >> logc : i / C; };
    auto col_of = [&](int i) { return p2 ? i & (C - 1) : i % C; };
    const long long n = g.n;
    V2<TT> *cz = reinterpret_cast<V2<TT> *>(k.cz);
    const V2<TT> *twg = reinterpret_cast<const V2<TT> *>(k.twy);
    for (int i = threadIdx.x; i < ntw; i += blockDim.x) tw[i] = twg[i];
    for (int i = threadIdx.x; i < tile; i += blockDim.x) {
        const long long s = (long long)row_of(i) * nx + x0 + col_of(i);
        V2<TT> v;
        if (MODE == COL_CONVECT) {
            const double *om = k.omega + (size_t)run * 3 * n;
            v = pair == 0 ? mk<TT>((TT)om[s], (TT)om[n + s]) : mk<TT>((TT)om[2 * n + s], (TT)0);
        } else if (MODE == COL_DIFFUSE) {
            v = to_tt<TT>(mu_pair(k, k.phi_t + (size_t)run * 3 * n, k.omega_t + (size_t)run * 3 * n, n, s, pair));
        } else if (MODE == COL_DIVY) {
            // y flux v_y Phi_I
            const double *ph = k.phi + (size_t)run * 3 * n;
            const double vy = vel_at(k, (size_t)run * n + s).y * g.vscale;
            v = pair == 0 ? mk<TT>((TT)(vy * ph[s]), (TT)(vy * ph[n + s])) : mk<TT>((TT)(vy * ph[2 * n + s]), (TT)0);
        } else {
            v = cz[((size_t)run * 4 + 2) * n + s];
        }
        a[i] = v;
    }
    __syncthreads();
    V2<TT> *r = p2 ? fft_smem<TT, false, true>(a, b, logy, logc, 1, C, tw)
                   : fft_smem_mr<TT, false, true>(a, b, ny, g.nfy, g.fy, C, 1, C, tw);
    V2<TT> *o = (r == a) ? b : a;
    const TT uy = (TT)k.kunit_y, ux = (TT)k.kunit_x, inv_n = (TT)(1.0 / (double)ny);
    const TT cforce = (TT)(g.inv_beta_v * g.fstar / (g.dt * (double)ny));
    for (int i = threadIdx.x; i < tile; i += blockDim.x) {
        const int my = row_of(i);
        V2<TT> v = r[i];
        if (MODE == COL_CONVECT || MODE == COL_DIVY) {  // i ky / ny
            const TT kk = kvec_odd<TT>(my, ny, uy) * inv_n;
            v = mk<TT>(-kk * v.y, kk * v.x);
        } else if (MODE == COL_DIFFUSE) { // -ky^2 / ny
            const TT kk = kvec<TT>(my, ny, uy);
            v = cscale(v, -kk * kk * inv_n);
        } else {
            // f(k) = (1/(beta v)) S(k) / dt * i k / |k|^2, Eq. (20), in lattice units;
            // f_x + i f_y is real + i real, so one transform carries both:
            // multiply by c (i kx - ky) / |k|^2 and invert.
            const int mx = x0 + col_of(i);
            const TT kx = kvec<TT>(mx, nx, ux), ky = kvec<TT>(my, ny, uy);
            const TT k2 = kx * kx + ky * ky;
            if (k2 == (TT)0) {
                v = mk<TT>((TT)0, (TT)0);
            } else {
                const TT c = cforce / k2;
                v = cmul(v, mk<TT>(-c * kvec_odd<TT>(my, ny, uy), c * kvec_odd<TT>(mx, nx, ux)));
            }
        }
        r[i] = v;
    }
    __syncthreads();
    r = p2 ? fft_smem<TT, true, true>(r, o, logy, logc, 1, C, tw) : fft_smem_mr<TT, true, true>(r, o, ny, g.nfy, g.fy, C, 1, C, tw);
    for (int i = threadIdx.x; i < tile; i += blockDim.x) {
        const long long s = (long long)row_of(i) * nx + x0 + col_of(i);
        if (MODE == COL_FORCE) {
            cz[((size_t)run * 4 + 2) * n + s] = r[i];
        } else if (MODE == COL_DIVY) {
            // Phi~ = Phi - dt (d/dx (v_x Phi) + d/dy (v_y Phi))
            const double2 dy = to_d<TT>(r[i]);
            const double2 dx = to_d<TT>(cz[((size_t)run * 4 + pair) * n + s]);
            const double *ph = k.phi + (size_t)run * 3 * n;
            double *pd = k.phi_dst + (size_t)run * 3 * n;
            if (pair == 0) {
                pd[s] = ph[s] - g.dt * (dx.x + dy.x);
                pd[n + s] = ph[n + s] - g.dt * (dx.y + dy.y);
            } else {
                pd[2 * n + s] = ph[2 * n + s] - g.dt * (dx.x + dy.x);
            }
        } else if (MODE == COL_CONVECT) {
            // omega~ = omega - dt v . grad omega, v = u_lat dx/dt
            const double2 dy = to_d<TT>(r[i]);
            const double2 dx = to_d<TT>(cz[((size_t)run * 4 + pair) * n + s]);
            const double2 u = vel_at(k, (size_t)run * n + s);
            const double vx = u.x * g.vscale, vy = u.y * g.vscale;
            const double *om = k.omega + (size_t)run * 3 * n;
            double *ot = k.omega_dst + (size_t)run * 3 * n;
            if (pair == 0) {
                ot[s] = om[s] - g.dt * (vx * dx.x + vy * dy.x);
                ot[n + s] = om[n + s] - g.dt * (vx * dx.y + vy * dy.y);
            } else {
                ot[2 * n + s] = om[2 * n + s] - g.dt * (vx * dx.x + vy * dy.x);
            }
        } else {
            // omega(t+dt) = omega~ - dt D_I Lap mu_I
            const double2 dy = to_d<TT>(r[i]);
            const double2 lx = to_d<TT>(cz[((size_t)run * 4 + pair) * n + s]);
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

// ---------------------------------------------------------------------------
// FP32 radix-8 versions of the row and column passes (MIXED_FP32, grids with
// 64..2048 points per axis): the same operators and data flow as epd_row /
// epd_col above, transforms and tiles (RowTile, ColTile) from fft8.cuh.
// ---------------------------------------------------------------------------

// i k / n (first derivative, Nyquist bin dropped) and -k^2 / n along one axis
struct OpGrad {
    int n;
    float unit, inv_n;
    __device__ __forceinline__ float2 operator()(int, int bin, float2 v) const
    {
        const float kk = (2 * bin == n ? 0.f : unit * (float)signed_bin(bin, n)) * inv_n;
        return f2(-kk * v.y, kk * v.x);
    }
};
struct OpLap {
    int n;
    float unit, inv_n;
    __device__ __forceinline__ float2 operator()(int, int bin, float2 v) const
    {
        const float kk = unit * (float)signed_bin(bin, n), f = -kk * kk * inv_n;
        return f2(v.x * f, v.y * f);
    }
};
// force of Eq. (20) on a column of the row spectrum: c (i kx - ky) / |k|^2
struct OpForce {
    int nx, ny, x0;
    float ux, uy, cforce;
    __device__ __forceinline__ float2 operator()(int c, int my, float2 v) const
    {
        const int mx = x0 + c;
        const float kx = ux * (float)signed_bin(mx, nx), ky = uy * (float)signed_bin(my, ny);
        const float k2 = kx * kx + ky * ky;
        if (k2 == 0.f) return f2(0.f, 0.f);
        const float cc = cforce / k2;
        const float kxo = 2 * mx == nx ? 0.f : kx, kyo = 2 * my == ny ? 0.f : ky;
        return fmul(v, f2(-cc * kyo, cc * kxo));
    }
};

template <int LOGX, int MODE>
__global__ void __launch_bounds__(RowTile<LOGX>::T) epd_row8(EpdK k)
{
    using RT = RowTile<LOGX>;
    using RL = RowLayout<LOGX>;
    constexpr int NX = RT::NX, P = RT::P, T = RT::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    float2 *tab = buf + RT::ROWS * RL::PITCH;
    const GroupGeom &g = k.g;
    const int run = blockIdx.y, pair = blockIdx.z, tid = threadIdx.x;
    const long long n = g.n;
    const long long base = (long long)blockIdx.x * P;
    float2 *cz = reinterpret_cast<float2 *>(k.cz);
    copy_tables(tab, k.tab8x, RT::TAB, tid, T);
    // the inputs of this thread in batches, each batch's loads before its
    // stores (the scratch planes written below could alias the fields as far
    // as the compiler knows, so interleaving would serialise the loads
    // behind the stores)
    constexpr int UB = P / T < 8 ? P / T : 8;  // inputs per batch
#pragma unroll
    for (int u0 = 0; u0 < P / T; u0 += UB) {
        float2 vin[UB];
#pragma unroll
        for (int u = u0; u < u0 + UB; ++u) {
            const int i = tid + u * T;
            const long long s = base + i;
            float2 v;
            if (MODE == ROW_GRAD) {
                const double *om = k.omega + (size_t)run * 3 * n;
                v = pair == 0 ? f2((float)om[s], (float)om[n + s]) : f2((float)om[2 * n + s], 0.f);
            } else if (MODE == ROW_LAP) {
                v = mu_pair_f(k, k.phi_t + (size_t)run * 3 * n, k.omega_t + (size_t)run * 3 * n, n, s, pair);
            } else if (MODE == ROW_FWD_S) {
                // S = sum_I dPhi_I^D / D_I from the FP64 differences, in FP32
                const double *p1 = k.phi + (size_t)run * 3 * n, *p0 = k.phi_t + (size_t)run * 3 * n;
                const float da = (float)(p1[s] - p0[s]), db = (float)(p1[n + s] - p0[n + s]), dsv = (float)(p1[2 * n + s] - p0[2 * n + s]);
                v = f2((da + db) * (float)(1.0 / g.d_p) + dsv * (float)(1.0 / g.d_s), 0.f);
            } else {
                v = cz[((size_t)run * 4 + 2) * n + s];
            }
            vin[u - u0] = v;
        }
#pragma unroll
        for (int u = u0; u < u0 + UB; ++u) {
            const int i = tid + u * T;
            // the column pass of the same operator reads this FP32 input from the
            // free scratch planes 2, 3 instead of forming it again from FP64 fields
            if (MODE == ROW_GRAD || MODE == ROW_LAP) cz[((size_t)run * 4 + 2 + pair) * n + base + i] = vin[u - u0];
            buf[RL::at(i / NX, i % NX)] = vin[u - u0];
        }
    }
    __syncthreads();
    if (MODE == ROW_FWD_S) {
        forward<LOGX, T, RL, P, RT::MR>(buf, tab, tid);
#pragma unroll
        for (int u = 0; u < P / T; ++u) {
            const int i = tid + u * T;
            cz[((size_t)run * 4 + 2) * n + base + i] = buf[RL::at(i / NX, i % NX)];
        }
        return;
    }
    const float unit = (float)k.kunit_x, inv_n = 1.f / (float)NX;
    if (MODE == ROW_GRAD)
        transform_pair<LOGX, T, RL, P, OpGrad, RT::MR>(buf, tab, OpGrad{NX, unit, inv_n}, tid);
    else if (MODE == ROW_LAP)
        transform_pair<LOGX, T, RL, P, OpLap, RT::MR>(buf, tab, OpLap{NX, unit, inv_n}, tid);
    else
        inverse_open<LOGX, T, RL, P, RT::MR>(buf, tab, tid);
    constexpr int RLOG_L = inv_rlog(LOGX, npasses(LOGX, RT::MR) - 1, RT::MR), RR = 1 << RLOG_L, PER_L = NX / RR, NB_L = P / RR / T;
    float2 h[NB_L][RR];
    int bb[NB_L], tt[NB_L];
    last_inverse<LOGX, NB_L, T, RL, RT::MR>(buf, h, bb, tt, tid);
#pragma unroll
    for (int j = 0; j < NB_L; ++j)
#pragma unroll
        for (int r = 0; r < RR; ++r) {
            const long long s = base + (long long)bb[j] * NX + tt[j] + r * PER_L;
            if (MODE == ROW_INV_FORCE) {
                const float2 f = f2(h[j][r].x * inv_n, h[j][r].y * inv_n);
                if (k.bulk_double) reinterpret_cast<double2 *>(k.force)[(size_t)run * n + s] = make_double2((double)f.x, (double)f.y);
                else reinterpret_cast<float2 *>(k.force)[(size_t)run * n + s] = f;
            } else {
                cz[((size_t)run * 4 + pair) * n + s] = h[j][r];
            }
        }
}

template <int LOGY, int MODE, int CW>
__global__ void __launch_bounds__(ColTile<LOGY, CW>::T) epd_col8(EpdK k)
{
    using CT = ColTile<LOGY, CW>;
    using CL = ColLayout<LOGY, CT::C>;
    constexpr int NY = CT::NY, C = CT::C, P = CT::P, T = CT::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    float2 *tab = buf + P;
    const GroupGeom &g = k.g;
    const int nx = g.nx, run = blockIdx.y, pair = blockIdx.z, x0 = blockIdx.x * C, tid = threadIdx.x;
    const long long n = g.n;
    float2 *cz = reinterpret_cast<float2 *>(k.cz);
    copy_tables(tab, CT::MR == 4 ? k.tab16y : k.tab8y_r8, CT::TAB, tid, T);
#pragma unroll
    for (int u = 0; u < P / T; ++u) {
        const int i = tid + u * T;
        const long long s = (long long)(i / C) * nx + x0 + (i % C);
        float2 v;
        if (MODE == COL_CONVECT || MODE == COL_DIFFUSE) {
            v = cz[((size_t)run * 4 + 2 + pair) * n + s];  // stored by the row pass (omega, mu in FP32)
        } else {
            v = cz[((size_t)run * 4 + 2) * n + s];
        }
        buf[i] = v;  // CL::at(i % C, i / C)
    }
    __syncthreads();
    const float uy = (float)k.kunit_y, inv_n = 1.f / (float)NY;
    if (MODE == COL_CONVECT)
        transform_pair<LOGY, T, CL, P, OpGrad, CT::MR>(buf, tab, OpGrad{NY, uy, inv_n}, tid);
    else if (MODE == COL_DIFFUSE)
        transform_pair<LOGY, T, CL, P, OpLap, CT::MR>(buf, tab, OpLap{NY, uy, inv_n}, tid);
    else
        transform_pair<LOGY, T, CL, P, OpForce, CT::MR>(
            buf, tab, OpForce{nx, NY, x0, (float)k.kunit_x, uy, (float)(g.inv_beta_v * g.fstar / (g.dt * (double)NY))}, tid);
    constexpr int RLOG_L = inv_rlog(LOGY, npasses(LOGY, CT::MR) - 1, CT::MR), RR = 1 << RLOG_L, PER_L = NY / RR, NB_L = P / RR / T;
    float2 h[NB_L][RR];
    int bb[NB_L], tt[NB_L];
    last_inverse<LOGY, NB_L, T, CL, CT::MR>(buf, h, bb, tt, tid);
    // in batches of SB points: every load first, then the stores (the output
    // field could alias the inputs as far as the compiler knows, which would
    // serialise each load behind the previous stores)
    constexpr int SB = RR < 4 ? RR : 4;
#pragma unroll
    for (int j = 0; j < NB_L; ++j)
#pragma unroll
        for (int r0 = 0; r0 < RR; r0 += SB) {
            long long sj[SB];
#pragma unroll
            for (int b = 0; b < SB; ++b) sj[b] = (long long)(tt[j] + (r0 + b) * PER_L) * nx + x0 + bb[j];
            if (MODE == COL_FORCE) {
#pragma unroll
                for (int b = 0; b < SB; ++b) cz[((size_t)run * 4 + 2) * n + sj[b]] = h[j][r0 + b];
            } else if (MODE == COL_CONVECT) {
                // omega~ = omega - dt v . grad omega, v = u_lat dx/dt (increment in FP32)
                const double *om = k.omega + (size_t)run * 3 * n;
                double *ot = k.omega_dst + (size_t)run * 3 * n;
                const float cv = (float)(g.vscale * g.dt);
                float2 dxf[SB], u[SB];
                double o0[SB], o1[SB];
#pragma unroll
                for (int b = 0; b < SB; ++b) {
                    const long long s = sj[b];
                    dxf[b] = cz[((size_t)run * 4 + pair) * n + s];
                    u[b] = reinterpret_cast<const float2 *>(k.vel)[(size_t)run * n + s];  // FP32 bulk
                    o0[b] = pair == 0 ? om[s] : om[2 * n + s];
                    o1[b] = pair == 0 ? om[n + s] : 0.0;
                }
#pragma unroll
                for (int b = 0; b < SB; ++b) {
                    const long long s = sj[b];
                    const float2 dyf = h[j][r0 + b];
                    const float vx = u[b].x * cv, vy = u[b].y * cv;
                    if (pair == 0) {
                        ot[s] = o0[b] - (double)(vx * dxf[b].x + vy * dyf.x);
                        ot[n + s] = o1[b] - (double)(vx * dxf[b].y + vy * dyf.y);
                    } else {
                        ot[2 * n + s] = o0[b] - (double)(vx * dxf[b].x + vy * dyf.x);
                    }
                }
            } else {
                // omega(t+dt) = omega~ - dt D_I Lap mu_I (increment in FP32)
                const double *ot = k.omega_t + (size_t)run * 3 * n;
                double *om = k.omega_dst + (size_t)run * 3 * n;
                float2 lxf[SB];
                double o0[SB], o1[SB];
#pragma unroll
                for (int b = 0; b < SB; ++b) {
                    const long long s = sj[b];
                    lxf[b] = cz[((size_t)run * 4 + pair) * n + s];
                    o0[b] = pair == 0 ? ot[s] : ot[2 * n + s];
                    o1[b] = pair == 0 ? ot[n + s] : 0.0;
                }
#pragma unroll
                for (int b = 0; b < SB; ++b) {
                    const long long s = sj[b];
                    const float2 dyf = h[j][r0 + b];
                    if (pair == 0) {
                        const float c = (float)(g.dt * g.d_p);
                        om[s] = o0[b] - (double)(c * (lxf[b].x + dyf.x));
                        om[n + s] = o1[b] - (double)(c * (lxf[b].y + dyf.y));
                    } else {
                        om[2 * n + s] = o0[b] - (double)((float)(g.dt * g.d_s) * (lxf[b].x + dyf.x));
                    }
                }
            }
        }
}

// Launch of the radix-8 row / column pass for the group's grid, or false
// when the grid has no radix-8 instantiation.
template <int MODE, int L>
static bool row8_at(int logx, const EpdK &k, dim3 grid_yz, cudaStream_t s)
{
    if constexpr (L > 11) {
        return false;
    } else {
        if (logx != L) return row8_at<MODE, L + 1>(logx, k, grid_yz, s);
        using RT = RowTile<L>;
        static std::atomic<bool> conf{false};  // attribute set (idempotent if two threads race)
        if (!conf) {
            conf = cudaFuncSetAttribute(epd_row8<L, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RT::SMEM) == cudaSuccess;
            if (!conf) return false;
        }
        const int blocks = (int)(k.g.n / RT::P);
        epd_row8<L, MODE><<<dim3(blocks, grid_yz.y, grid_yz.z), RT::T, RT::SMEM, s>>>(k);
        return true;
    }
}
template <int MODE, int L, int CW>
static bool col8_launch(const EpdK &k, dim3 grid_yz, cudaStream_t s)
{
    using CT = ColTile<L, CW>;
    if (k.g.nx % CT::C) return false;
    static std::atomic<bool> conf{false};  // attribute set (idempotent if two threads race)
    if (!conf) {
        conf = cudaFuncSetAttribute(epd_col8<L, MODE, CW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CT::SMEM) == cudaSuccess;
        if (!conf) return false;
    }
    epd_col8<L, MODE, CW><<<dim3(k.g.nx / CT::C, grid_yz.y, grid_yz.z), CT::T, CT::SMEM, s>>>(k);
    return true;
}
// colw: column tile width (4, 8, 16; 0 = default)
template <int MODE, int L>
static bool col8_at(int logy, const EpdK &k, dim3 grid_yz, cudaStream_t s, int colw)
{
    if constexpr (L > 11) {
        return false;
    } else {
        if (logy != L) return col8_at<MODE, L + 1>(logy, k, grid_yz, s, colw);
        switch (colw) {
        case 4: return col8_launch<MODE, L, 4>(k, grid_yz, s);
        case 8: return col8_launch<MODE, L, 8>(k, grid_yz, s);
        case 16: return col8_launch<MODE, L, 16>(k, grid_yz, s);
        default: return col8_launch<MODE, L, ColTile<L>::C>(k, grid_yz, s);
        }
    }
}
// radix-8 passes apply to MIXED_FP32 groups with 64 <= nx, ny <= 2048 and at
// least 2048 sites
static bool use_r8(const Group &G)
{
    return G.prec == EPD_LB_MIXED_FP32 && G.tab8x && G.tab8y && G.g.logx >= 6 && G.g.logy >= 6 && G.g.logx <= 11 &&
           G.g.logy <= 11 && G.g.n >= 2048;
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
    k.phi_dst = nullptr;
    k.cz = G.cz;
    k.vel = G.vel;
    k.force = G.force;
    k.bulk_double = G.prec == EPD_LB_PLAIN_FP64;
    // FP32 transforms use the bulk (FP32) twiddle tables, FP64 ones the FP64 tables
    k.twx = k.bulk_double ? (const void *)G.twx_d : G.twx;
    k.twy = k.bulk_double ? (const void *)G.twy_d : G.twy;
    // tables of each axis' radix plan (RowTile / ColTile pick best_mr)
    k.tab8x = best_mr(G.g.logx) == 4 ? G.tab16x : G.tab8x;
    k.tab8y = best_mr(G.g.logy) == 4 ? G.tab16y : G.tab8y;
    k.tab16y = G.tab16y;
    k.tab8y_r8 = G.tab8y;
    k.rows = G.sh.rows_epd;
    k.logc = G.g.pow2 ? ilog2(G.sh.cols_epd) : 0;
    k.cols = G.sh.cols_epd;
    const double pi = 3.14159265358979323846;
    k.kunit_x = 2.0 * pi / ((double)G.g.nx * G.g.dx);
    k.kunit_y = 2.0 * pi / ((double)G.g.ny * G.g.dx);
    // homogeneous composition: Phi_A = phi_p N_A/N_s, Phi_B = phi_p (1 - N_A/N_s), Phi_S = 1 - phi_p
    const double fa = (double)G.g.na / (double)G.g.ns;
    const double pa = G.g.phi_p * fa, pb = G.g.phi_p * (1.0 - fa), ps = 1.0 - G.g.phi_p;
    const double inc = G.g.kappa_h * (pa + pb + ps - 1.0);
    k.mu_ref[0] = G.g.chi_ab * pb + G.g.chi_as * ps + inc;
    k.mu_ref[1] = G.g.chi_ab * pa + G.g.chi_bs * ps + inc;
    k.mu_ref[2] = G.g.chi_as * pa + G.g.chi_bs * pb + inc;
    k.phibar[0] = pa;
    k.phibar[1] = pb;
    k.phibar[2] = ps;
    return k;
}

template <typename TT> static size_t row_smem(const Group &G)
{
    return (size_t)2 * G.sh.rows_epd * G.g.nx * sizeof(V2<TT>) + (G.g.pow2 ? G.g.nx / 2 : G.g.nx) * sizeof(V2<TT>);
}
template <typename TT> static size_t col_smem(const Group &G)
{
    return (size_t)2 * G.sh.cols_epd * G.g.ny * sizeof(V2<TT>) + (G.g.pow2 ? G.g.ny / 2 : G.g.ny) * sizeof(V2<TT>);
}

template <typename TT> static cudaError_t aux_t(Group &G, cudaStream_t s)
{
    EpdK k = make_k(G);
    k.omega_dst = G.omega_t;
    if (use_r8(G)) {
        const dim3 gz(1, G.g.nruns, 2);
        if (row8_at<ROW_GRAD, 6>(G.g.logx, k, gz, s) && col8_at<COL_CONVECT, 6>(G.g.logy, k, gz, s, G.colw)) return cudaGetLastError();
        return cudaErrorInvalidConfiguration;
    }
    epd_row<TT, ROW_GRAD><<<dim3(G.g.ny / G.sh.rows_epd, G.g.nruns, 2), kThreads, row_smem<TT>(G), s>>>(k);
    epd_col<TT, COL_CONVECT><<<dim3(G.g.nx / G.sh.cols_epd, G.g.nruns, 2), kThreads, col_smem<TT>(G), s>>>(k);
    return cudaGetLastError();
}

template <typename TT> static cudaError_t diffusion_t(Group &G, cudaStream_t s)
{
    EpdK k = make_k(G);
    k.omega_dst = G.omega;
    if (use_r8(G)) {
        const dim3 gz(1, G.g.nruns, 2);
        if (row8_at<ROW_LAP, 6>(G.g.logx, k, gz, s) && col8_at<COL_DIFFUSE, 6>(G.g.logy, k, gz, s, G.colw)) return cudaGetLastError();
        return cudaErrorInvalidConfiguration;
    }
    epd_row<TT, ROW_LAP><<<dim3(G.g.ny / G.sh.rows_epd, G.g.nruns, 2), kThreads, row_smem<TT>(G), s>>>(k);
    epd_col<TT, COL_DIFFUSE><<<dim3(G.g.nx / G.sh.cols_epd, G.g.nruns, 2), kThreads, col_smem<TT>(G), s>>>(k);
    return cudaGetLastError();
}

template <typename TT> static cudaError_t force_t(Group &G, cudaStream_t s)
{
    EpdK k = make_k(G);
    if (use_r8(G)) {
        const dim3 gz(1, G.g.nruns, 1);
        if (row8_at<ROW_FWD_S, 6>(G.g.logx, k, gz, s) && col8_at<COL_FORCE, 6>(G.g.logy, k, gz, s, G.colw) &&
            row8_at<ROW_INV_FORCE, 6>(G.g.logx, k, gz, s))
            return cudaGetLastError();
        return cudaErrorInvalidConfiguration;
    }
    epd_row<TT, ROW_FWD_S><<<dim3(G.g.ny / G.sh.rows_epd, G.g.nruns, 1), kThreads, row_smem<TT>(G), s>>>(k);
    epd_col<TT, COL_FORCE><<<dim3(G.g.nx / G.sh.cols_epd, G.g.nruns, 1), kThreads, col_smem<TT>(G), s>>>(k);
    epd_row<TT, ROW_INV_FORCE><<<dim3(G.g.ny / G.sh.rows_epd, G.g.nruns, 1), kThreads, row_smem<TT>(G), s>>>(k);
    return cudaGetLastError();
}

// Column tile autotuner (radix-8 EPD column passes and streaming propagator
// column passes): each candidate width runs the diffusion column pass a few
// times on the group's state, writing only scratch (omega~, the EPD scratch);
// the fastest width is kept in G.colw.  Every width computes the same
// per-column transforms, so the results do not depend on the choice.
// EPD_LB_COLUMN_TILE=4|8|16 in the environment forces a width.
cudaError_t tune_column_tiles(Group &G, cudaStream_t s)
{
    if (!use_r8(G)) return cudaSuccess;
    if (const char *env = std::getenv("EPD_LB_COLUMN_TILE")) {
        const int w = std::atoi(env);
        if (w == 4 || w == 8 || w == 16) {
            G.colw = w;
            return cudaSuccess;
        }
    }
    EpdK k = make_k(G);
    k.omega_t = G.omega;      // read the current state ...
    k.phi_t = G.phi;
    k.omega_dst = G.omega_t;  // ... write only scratch (rewritten by the next step)
    const dim3 gz(1, G.g.nruns, 2);
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return cudaGetLastError();
    float best = 1e30f;
    int best_w = 0;
    for (int w : kColWidths) {
        if (G.g.nx % w) continue;
        if (!col8_at<COL_DIFFUSE, 6>(G.g.logy, k, gz, s, w)) {
            cudaGetLastError();
            continue;
        }
        float t = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(a, s);
            col8_at<COL_DIFFUSE, 6>(G.g.logy, k, gz, s, w);
            cudaEventRecord(b, s);
            cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (rep > 0 && ms < t) t = ms;  // the first launch is a warm-up
        }
        if (t < best) {
            best = t;
            best_w = w;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    G.colw = best_w;
    return cudaGetLastError();
}

// Convection of the composition fields, always with FP64 transforms (the
// FP64 twiddles exist in both precisions; the FP64 scratch planes fit the
// EPD scratch): the densities of every run of the group.
cudaError_t launch_convect_phi(Group &G, const double *phi, double *phi_dst, cudaStream_t s)
{
    EpdK k = make_k(G);
    k.phi = phi;
    k.phi_dst = phi_dst;
    k.twx = G.twx_d;
    k.twy = G.twy_d;
    epd_row<double, ROW_DIVX><<<dim3(G.g.ny / G.sh.rows_epd, G.g.nruns, 2), kThreads, row_smem<double>(G), s>>>(k);
    epd_col<double, COL_DIVY><<<dim3(G.g.nx / G.sh.cols_epd, G.g.nruns, 2), kThreads, col_smem<double>(G), s>>>(k);
    return cudaGetLastError();
}

cudaError_t launch_aux_convection(Group &G, cudaStream_t s)
{
    return G.prec == EPD_LB_MIXED_FP32 ? aux_t<float>(G, s) : aux_t<double>(G, s);
}

cudaError_t launch_diffusion(Group &G, cudaStream_t s)
{
    return G.prec == EPD_LB_MIXED_FP32 ? diffusion_t<float>(G, s) : diffusion_t<double>(G, s);
}

cudaError_t launch_force(Group &G, cudaStream_t s)
{
    return G.prec == EPD_LB_MIXED_FP32 ? force_t<float>(G, s) : force_t<double>(G, s);
}

template <typename TT> static cudaError_t configure_t()
{
    const int lim = 200 * 1024;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(epd_row<TT, ROW_GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(epd_row<TT, ROW_LAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(epd_row<TT, ROW_FWD_S>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(epd_row<TT, ROW_INV_FORCE>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(epd_col<TT, COL_CONVECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(epd_col<TT, COL_DIFFUSE>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    return cudaFuncSetAttribute(epd_col<TT, COL_FORCE>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

cudaError_t configure_epd_kernels()
{
    cudaError_t e = configure_t<float>();
    if (!e) e = configure_t<double>();
    if (!e) e = cudaFuncSetAttribute(epd_row<double, ROW_DIVX>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (!e) e = cudaFuncSetAttribute(epd_col<double, COL_DIVY>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    return e;
}

} // namespace epdlb

// step3d.cu -- the coupled hybrid LB/EPD step on a 3D box (the extension the
// paper names in Sec. 2 and Sec. 5), FP64 spectral operators on sm_103a:
//   omega~ = omega - dt v . grad omega            (App. C, item 1)
//   Phi~ = solve3d(omega~)                        (Eqs. (6)-(11))
//   omega(t+dt) = omega~ - dt D_I Lap mu_I(Phi~)  (Eq. (5))
//   Phi(t+dt) = solve3d(omega(t+dt))
//   f = (1/(beta v)) sum_I dPhi_I/(D_I dt) i k/|k|^2 (Eqs. (19)-(20)) + f_P(y) x^
//   one D3Q19 collide-stream.
// Spectral derivatives are full 3D transforms of one complex FP64 field
// (real part the data): batched 1D transforms along x (rows), y (columns of
// every z plane) and z (pillars), radix-2 on power-of-two axes and mixed
// radix otherwise, each loading a tile into shared memory and storing it
// back in place; the spectral factor is one elementwise pass.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "engine.h"

namespace epdlb {
namespace {

using C2 = V2<double>;

__host__ __device__ __forceinline__ bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Transforms of the rows (along x, length ax.n) of R consecutive rows per CTA.
template <bool INV>
__global__ void __launch_bounds__(kThreads) fft3_rows(C2 *buf, Axis3 ax, int R, const C2 *tw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const bool p2 = ax.pow2 && is_pow2(R);  // radix-2 passes read half the twiddles
    const int N = ax.n, tile = R * N, ntw = p2 ? N / 2 : N;
    C2 *a = reinterpret_cast<C2 *>(smem_raw);
    C2 *b = a + tile;
    C2 *t = b + tile;
    const long long base = (long long)blockIdx.x * tile;
    for (int i = threadIdx.x; i < tile; i += blockDim.x) a[i] = buf[base + i];
    for (int i = threadIdx.x; i < ntw; i += blockDim.x) t[i] = tw[i];
    __syncthreads();
    C2 *r = p2 ? fft_smem<double, INV, false>(a, b, ax.logn, ilog2(R), N, 1, t)
               : fft_smem_mr<double, INV, false>(a, b, N, ax.nf, ax.f, R, N, 1, t);
    for (int i = threadIdx.x; i < tile; i += blockDim.x) buf[base + i] = r[i];
}

// Transforms of columns of length ax.n: element j of column c of plane p at
// p PS + j S + c; one CTA takes C consecutive columns of one plane.
template <bool INV>
__global__ void __launch_bounds__(kThreads) fft3_cols(C2 *buf, Axis3 ax, long long S, long long PS, int C, const C2 *tw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const bool p2 = ax.pow2 && is_pow2(C);
    const int N = ax.n, tile = N * C, ntw = p2 ? N / 2 : N;
    C2 *a = reinterpret_cast<C2 *>(smem_raw);
    C2 *b = a + tile;
    C2 *t = b + tile;
    const long long base = (long long)blockIdx.y * PS + (long long)blockIdx.x * C;
    for (int i = threadIdx.x; i < tile; i += blockDim.x) a[i] = buf[base + (long long)(i / C) * S + i % C];
    for (int i = threadIdx.x; i < ntw; i += blockDim.x) t[i] = tw[i];
    __syncthreads();
    C2 *r = p2 ? fft_smem<double, INV, true>(a, b, ax.logn, ilog2(C), 1, C, t)
               : fft_smem_mr<double, INV, true>(a, b, N, ax.nf, ax.f, C, 1, C, t);
    for (int i = threadIdx.x; i < tile; i += blockDim.x) buf[base + (long long)(i / C) * S + i % C] = r[i];
}

// real field -> complex buffer (imaginary part 0), optionally a combination
// sum_s w_s f_s of three fields of n values each
__global__ void load_real(C2 *buf, const double *f, long long n, double w0, double w1, double w2, int nfields)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double v = w0 * f[i];
        if (nfields > 1) v += w1 * f[n + i];
        if (nfields > 2) v += w2 * f[2 * n + i];
        buf[i] = mk<double>(v, 0.0);
    }
}

// out = in x the spectral factor, scaled by 1/n (the unnormalised inverse):
// op 0, 1, 2: i k_x, i k_y, i k_z (Nyquist bin of that axis dropped); op 3:
// -|k|^2; op 4, 5, 6: c i k_a / |k|^2 (the force component a, 0 at k = 0)
__global__ void spec3_apply(const C2 *in, C2 *out, int nx, int ny, int nz, double ux, double uy, double uz, int op,
                            double c)
{
    const long long n = (long long)nx * ny * nz;
    const double inv_n = 1.0 / (double)n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long long)nx * ny));
        const double kx = ux * signed_bin(x, nx), ky = uy * signed_bin(y, ny), kz = uz * signed_bin(z, nz);
        const double kox = 2 * x == nx ? 0.0 : kx, koy = 2 * y == ny ? 0.0 : ky, koz = 2 * z == nz ? 0.0 : kz;
        const C2 v = in[i];
        C2 r;
        if (op <= 2) {
            const double k = (op == 0 ? kox : op == 1 ? koy : koz) * inv_n;
            r = mk<double>(-k * v.y, k * v.x);
        } else if (op == 3) {
            const double m = -(kx * kx + ky * ky + kz * kz) * inv_n;
            r = mk<double>(m * v.x, m * v.y);
        } else {
            const double k2 = kx * kx + ky * ky + kz * kz;
            const double ka = op == 4 ? kox : op == 5 ? koy : koz;
            const double m = k2 == 0.0 ? 0.0 : c * ka / k2 * inv_n;
            r = mk<double>(-m * v.y, m * v.x);
        }
        out[i] = r;
    }
}

// omega~_s -= coef v_a Re(buf) (aux convection term of axis a)
__global__ void acc_convect(double *wt, const double *vel, const C2 *buf, long long n, int a, double coef)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        wt[i] -= coef * vel[(size_t)a * n + i] * buf[i].x;
}

// mu_s of Eq. (1) (the derivative of the free energy with omega conjugate)
__global__ void mu3(const double *phi, const double *om, double *mu, long long n, double chi_ab, double chi_as,
                    double chi_bs, double kappa_h)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double pa = phi[i], pb = phi[n + i], ps = phi[2 * n + i];
        const double inc = kappa_h * (pa + pb + ps - 1.0);
        mu[i] = chi_ab * pb + chi_as * ps + inc - om[i];
        mu[n + i] = chi_ab * pa + chi_bs * ps + inc - om[n + i];
        mu[2 * n + i] = chi_as * pa + chi_bs * pb + inc - om[2 * n + i];
    }
}

// dst = src - coef Re(buf)
__global__ void axpy_re(double *dst, const double *src, const C2 *buf, long long n, double coef)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i] - coef * buf[i].x;
}

// d = a - b over 3n values
__global__ void diff3(double *d, const double *a, const double *b, long long m)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
        d[i] = a[i] - b[i];
}

// force component a = fstar Re(buf); the total adds the body force of
// Eq. (23) along x, -f0 for y < ny/2 and +f0 above
__global__ void force_out(double *force, double *ftot, const C2 *buf, int nx, int ny, long long n, int a, double fstar,
                          double f0)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double f = fstar * buf[i].x;
        force[(size_t)a * n + i] = f;
        double fb = 0.0;
        if (a == 0) fb = ((int)((i / nx) % ny) < ny / 2) ? -f0 : f0;
        ftot[(size_t)a * n + i] = f + fb;
    }
}

int grid_n(long long n)
{
    long long b = (n + kThreads - 1) / kThreads;
    return (int)(b > 2048 ? 2048 : b);
}

} // namespace

size_t fft3_smem(const Fft3 &F)
{
    auto one = [](const Axis3 &ax, int tiles) { return (size_t)2 * tiles * ax.n * sizeof(C2) + (size_t)ax.n * sizeof(C2); };
    size_t m = one(F.ax, F.rows_x);
    m = std::max(m, one(F.ay, F.cols_y));
    return std::max(m, one(F.az, F.cols_z));
}

// 3D transform of buf in place: x rows, y columns, z pillars (inverse in the
// same order: the axes commute)
template <bool INV>
static cudaError_t fft3(const Fft3 &F, C2 *buf, cudaStream_t s)
{
    const long long nxy = (long long)F.ax.n * F.ay.n, n = nxy * F.az.n;
    const auto sm = [](const Axis3 &ax, int tiles) { return (size_t)2 * tiles * ax.n * sizeof(C2) + (size_t)ax.n * sizeof(C2); };
    fft3_rows<INV><<<(unsigned)(n / ((long long)F.rows_x * F.ax.n)), kThreads, sm(F.ax, F.rows_x), s>>>(buf, F.ax, F.rows_x, F.twx);
    fft3_cols<INV><<<dim3(F.ax.n / F.cols_y, F.az.n), kThreads, sm(F.ay, F.cols_y), s>>>(buf, F.ay, F.ax.n, nxy, F.cols_y, F.twy);
    fft3_cols<INV><<<dim3((unsigned)(nxy / F.cols_z), 1), kThreads, sm(F.az, F.cols_z), s>>>(buf, F.az, nxy, 0, F.cols_z, F.twz);
    return cudaGetLastError();
}

cudaError_t configure_step3d_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(fft3_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (!e) e = cudaFuncSetAttribute(fft3_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (!e) e = cudaFuncSetAttribute(fft3_cols<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (!e) e = cudaFuncSetAttribute(fft3_cols<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    return e;
}

cudaError_t launch_step3d(const Step3 &T, double *omega, double *pop, double *vel, double *phi, double *q, double *force,
                          cudaStream_t s)
{
    const GroupGeom &g = T.S.vx;
    const Fft3 &F = T.F;
    const long long n = g.n;
    const int gn = grid_n(n);
    const double pi = 3.14159265358979323846;
    const double ux = 2.0 * pi / ((double)F.ax.n * g.dx), uy = 2.0 * pi / ((double)F.ay.n * g.dx),
                 uz = 2.0 * pi / ((double)F.az.n * g.dx);
    cudaError_t e;
    // (1) omega~ = omega - dt v . grad omega, v = u_lat dx/dt
    if ((e = cudaMemcpyAsync(T.wt, omega, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, s))) return e;
    for (int sp = 0; sp < 3; ++sp) {
        load_real<<<gn, kThreads, 0, s>>>(T.b0, omega + (size_t)sp * n, n, 1.0, 0.0, 0.0, 1);
        if ((e = fft3<false>(F, T.b0, s))) return e;
        for (int a = 0; a < 3; ++a) {
            spec3_apply<<<gn, kThreads, 0, s>>>(T.b0, T.b1, F.ax.n, F.ay.n, F.az.n, ux, uy, uz, a, 0.0);
            if ((e = fft3<true>(F, T.b1, s))) return e;
            acc_convect<<<gn, kThreads, 0, s>>>(T.wt + (size_t)sp * n, vel, T.b1, n, a, g.dt * g.vscale);
        }
    }
    // (2) Phi~
    if ((e = launch_solve3d(T.S, T.wt, T.pt, T.qt, s))) return e;
    // (3) mu and the diffusion step
    mu3<<<gn, kThreads, 0, s>>>(T.pt, T.wt, T.mu, n, g.chi_ab, g.chi_as, g.chi_bs, g.kappa_h);
    for (int sp = 0; sp < 3; ++sp) {
        load_real<<<gn, kThreads, 0, s>>>(T.b0, T.mu + (size_t)sp * n, n, 1.0, 0.0, 0.0, 1);
        if ((e = fft3<false>(F, T.b0, s))) return e;
        spec3_apply<<<gn, kThreads, 0, s>>>(T.b0, T.b1, F.ax.n, F.ay.n, F.az.n, ux, uy, uz, 3, 0.0);
        if ((e = fft3<true>(F, T.b1, s))) return e;
        const double d = sp == 2 ? g.d_s : g.d_p;
        axpy_re<<<gn, kThreads, 0, s>>>(omega + (size_t)sp * n, T.wt + (size_t)sp * n, T.b1, n, g.dt * d);
    }
    // (4) Phi(t + dt)
    if ((e = launch_solve3d(T.S, omega, phi, q, s))) return e;
    // (5) the force from S = sum_I dPhi_I / D_I
    diff3<<<gn, kThreads, 0, s>>>(T.mu, phi, T.pt, 3 * n);
    load_real<<<gn, kThreads, 0, s>>>(T.b0, T.mu, n, 1.0 / g.d_p, 1.0 / g.d_p, 1.0 / g.d_s, 3);
    if ((e = fft3<false>(F, T.b0, s))) return e;
    for (int a = 0; a < 3; ++a) {
        spec3_apply<<<gn, kThreads, 0, s>>>(T.b0, T.b1, F.ax.n, F.ay.n, F.az.n, ux, uy, uz, 4 + a, g.inv_beta_v / g.dt);
        if ((e = fft3<true>(F, T.b1, s))) return e;
        force_out<<<gn, kThreads, 0, s>>>(force, T.ftot, T.b1, F.ax.n, F.ay.n, n, a, g.fstar, T.f0_lat);
    }
    // (6) D3Q19 with the total force
    if ((e = launch_lb3d_step(F.ax.n, F.ay.n, F.az.n, g.gamma_s, g.gamma_b, g.gamma_g, pop, T.ftot, T.pop2, vel, s))) return e;
    return cudaMemcpyAsync(pop, T.pop2, 19 * n * sizeof(double), cudaMemcpyDeviceToDevice, s);
}

} // namespace epdlb

// lb.cu -- D2Q9 multi-relaxation-time Lattice Boltzmann of the hybrid LB/EPD
// step (Sec. 2, Eqs. (12), (14)-(16); Sec. 4, Eq. (23) of arXiv:1804.02883),
// the initial state (Sec. 3 noise, Sec. 4 flow of Eq. (24)) and state access.
//
// One fused pull pass per step: each thread gathers the nine post-collision
// populations streamed into its site, collides them with the polymer force
// plus the reverse-Poiseuille body force, and writes its own post-collision
// populations (SoA planes [run][i][site]) and velocity.  Populations are kept
// as deviations d_i = n_i - w_i from the rest state so that FP32 storage
// resolves small flows; every moment below is formed from the deviations.
//
// Collision (Dunweg-Ladd mode form): u = (j + f/2)/rho; mass and momentum are
// conserved except j* = j + f; the stress relaxes about rho u u (deviation form
// of Pi_eq = rho c_s^2 I + rho u u) with its traceless part scaled by gamma_s
// and its trace by gamma_b; the force adds Sigma of Eq. (15) in d = 2; the
// remaining (ghost) part of the populations is scaled by gamma_g.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "engine.h"

namespace epdlb {

__constant__ int c_cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int c_cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

template <typename T> struct LbK {
    int nx, ny, logx;
    long long n;
    const T *pin;
    T *pout;
    const V2<T> *force;
    V2<T> *vel;
    const T *f0;  // body-force amplitude per run, lattice units, bulk type
    T gs, gb, gg;
};

// site -> (x, y): shift and mask when the axes are powers of two (logx > 0),
// division otherwise; periodic neighbour of v on an axis of n sites
__device__ __forceinline__ void site_xy(long long site, int nx, int logx, int &x, int &y)
{
    if (logx > 0) {
        x = (int)(site & (nx - 1));
        y = (int)(site >> logx);
    } else {
        x = (int)(site % nx);
        y = (int)(site / nx);
    }
}
__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__host__ __device__ __forceinline__ double lb_weight(int i) { return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }

template <typename T>
__global__ void __launch_bounds__(kThreads) lb_collide_stream(LbK<T> k)
{
    const int run = blockIdx.y;
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= k.n) return;
    int x, y;
    site_xy(site, k.nx, k.logx, x, y);
    const int xm = wrap(x - 1, k.nx), xp = wrap(x + 1, k.nx);
    const int ym = wrap(y - 1, k.ny), yp = wrap(y + 1, k.ny);
    const long long n = k.n;
    const T *src = k.pin + (size_t)run * 9 * n;
    // pull: population i arrives from site - c_i
    const long long r0 = (long long)y * k.nx, rm = (long long)ym * k.nx, rp = (long long)yp * k.nx;
    const T d0 = src[0 * n + r0 + x];
    const T d1 = src[1 * n + r0 + xm];
    const T d2 = src[2 * n + rm + x];
    const T d3 = src[3 * n + r0 + xp];
    const T d4 = src[4 * n + rp + x];
    const T d5 = src[5 * n + rm + xm];
    const T d6 = src[6 * n + rm + xp];
    const T d7 = src[7 * n + rp + xp];
    const T d8 = src[8 * n + rp + xm];

    const T drho = d0 + d1 + d2 + d3 + d4 + d5 + d6 + d7 + d8;
    const T rho = (T)1 + drho;
    const T jx = (d1 - d3) + (d5 - d6) + (d8 - d7);
    const T jy = (d2 - d4) + (d5 + d6) - (d7 + d8);
    const T sxx = d1 + d3 + d5 + d6 + d7 + d8;
    const T syy = d2 + d4 + d5 + d6 + d7 + d8;
    const T sxy = (d5 + d7) - (d6 + d8);
    const T third = (T)(1.0 / 3.0);
    // M = Pi - rho c_s^2 I from the deviations
    const T mxx = sxx - third * drho, myy = syy - third * drho, mxy = sxy;

    const V2<T> fp = k.force[(size_t)run * n + site];
    const T fpx = (y < (k.ny >> 1)) ? -k.f0[run] : k.f0[run];
    const T fx = fp.x + fpx, fy = fp.y;
    const T inv_rho = (T)1 / rho;
    const T ux = (jx + (T)0.5 * fx) * inv_rho, uy = (jy + (T)0.5 * fy) * inv_rho;
    k.vel[(size_t)run * n + site] = mk<T>(ux, uy);

    // non-equilibrium stress about rho u u, relaxed
    const T exx = rho * ux * ux, eyy = rho * uy * uy, exy = rho * ux * uy;
    const T nxx = mxx - exx, nyy = myy - eyy, nxy = mxy - exy;
    const T htr = (T)0.5 * (nxx + nyy);
    const T rxx = k.gs * (nxx - htr) + k.gb * htr;
    const T ryy = k.gs * (nyy - htr) + k.gb * htr;
    const T rxy = k.gs * nxy;
    // Sigma of Eq. (15) with the d = 2 constants
    const T uf = ux * fx + uy * fy;
    const T hs = (T)0.5 * ((T)1 + k.gs), hb = (T)0.5 * ((T)1 + k.gb);
    const T qxx = hs * ((T)2 * ux * fx - uf) + hb * uf;
    const T qyy = hs * ((T)2 * uy * fy - uf) + hb * uf;
    const T qxy = hs * (ux * fy + uy * fx);
    // post-collision moments
    const T pxx = exx + rxx + qxx, pyy = eyy + ryy + qyy, pxy = exy + rxy + qxy;
    const T jxs = jx + fx, jys = jy + fy;

    // d_i* = w_i [drho + 3 j*.c_i + 4.5 M*:Q_i] + gamma_g (d_i - w_i [drho + 3 j.c_i + 4.5 M:Q_i])
    const T dd[9] = {d0, d1, d2, d3, d4, d5, d6, d7, d8};
    T *dst = k.pout + (size_t)run * 9 * n + site;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
        const int cy = (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
        const T w = (T)lb_weight(i);
        const T qx = (T)(cx * cx) - third, qy = (T)(cy * cy) - third, qc = (T)(cx * cy);
        const T post = drho + (T)3 * (jxs * cx + jys * cy) + (T)4.5 * (pxx * qx + pyy * qy + (T)2 * pxy * qc);
        T v = w * post;
        if (k.gg != (T)0) {
            const T pre = drho + (T)3 * (jx * cx + jy * cy) + (T)4.5 * (mxx * qx + myy * qy + (T)2 * mxy * qc);
            v += k.gg * (dd[i] - w * pre);
        }
        dst[(size_t)i * n] = v;
    }
}

template <typename T>
static cudaError_t lb_t(Group &G, int parity, cudaStream_t s)
{
    LbK<T> k;
    k.nx = G.g.nx;
    k.ny = G.g.ny;
    k.logx = G.g.logx;
    k.n = G.g.n;
    k.pin = reinterpret_cast<const T *>(G.pop[parity]);
    k.pout = reinterpret_cast<T *>(G.pop[1 - parity]);
    k.force = reinterpret_cast<const V2<T> *>(G.force);
    k.vel = reinterpret_cast<V2<T> *>(G.vel);
    k.f0 = reinterpret_cast<const T *>(G.f0_bulk);
    k.gs = (T)G.g.gamma_s;
    k.gb = (T)G.g.gamma_b;
    k.gg = (T)G.g.gamma_g;
    const dim3 grid((unsigned)((G.g.n + kThreads - 1) / kThreads), G.g.nruns);
    lb_collide_stream<T><<<grid, kThreads, 0, s>>>(k);
    return cudaGetLastError();
}

cudaError_t launch_lb(Group &G, int parity, cudaStream_t s)
{
    if (G.prec == EPD_LB_MIXED_FP32) return lb_t<float>(G, parity, s);
    return lb_t<double>(G, parity, s);
}

// ---------------------------------------------------------------------------
// Initial state
// ---------------------------------------------------------------------------

// splitmix64 (Steele, Lea and Flood, OOPSLA 2014): add the golden gamma, then
// the variant-13 finaliser.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Uniform value in [-1, 1) for (seed, counter): top 53 bits of
// splitmix64(seed ^ splitmix64(counter)).
__device__ __forceinline__ double uniform_pm1(unsigned long long seed, unsigned long long ctr)
{
    const unsigned long long h = splitmix64(seed ^ splitmix64(ctr));
    return 2.0 * ((double)(h >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

struct InitK {
    GroupGeom g;
    double *omega;
    const unsigned long long *seeds;
    const double *noise;
    const double *f0_lat;
    void *post;
    void *vel;
    int bulk_double;
};

// Velocity of the steady reverse-Poiseuille flow on nodes at Y = y + 1/2:
// Eq. (24) plus f_P(y) (1 - 1/(8 eta)) (the scheme's discrete correction).
__device__ __forceinline__ double steady_profile(const GroupGeom &g, double a, int y)
{
    const double eta = (1.0 / 6.0) * (1.0 + g.gamma_s) / (1.0 - g.gamma_s);
    const double ly = (double)g.ny, d = (double)y + 0.5 - 0.5 * ly;
    const double fp = (y < g.ny / 2) ? -a : a;
    return -(a / (2.0 * eta)) * d * (fabs(d) - 0.5 * ly) + fp * (1.0 - 1.0 / (8.0 * eta));
}

__global__ void __launch_bounds__(kThreads) init_state(InitK k)
{
    const int run = blockIdx.y;
    const long long n = k.g.n;
    const unsigned long long seed = k.seeds[run];
    const double amp = k.noise[run], a = k.f0_lat[run];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int x, y;
        site_xy(i, k.g.nx, k.g.logx, x, y);
        for (int sp = 0; sp < 3; ++sp) {
            const unsigned long long ctr = ((unsigned long long)sp * k.g.ny + y) * (unsigned long long)k.g.nx + x;
            k.omega[((size_t)run * 3 + sp) * n + i] = amp * uniform_pm1(seed, ctr);
        }
        // post-collision populations at t = -1, so that the first pull sees the
        // pre-collision equilibrium with j = v(y) - f_P(y)/2 at every site
        for (int q = 0; q < 9; ++q) {
            const int yy = wrap(y + c_cy[q], k.g.ny);
            const double v = steady_profile(k.g, a, yy);
            const double fp = (yy < k.g.ny / 2) ? -a : a;
            const double jx = v - 0.5 * fp;
            const double cj = c_cx[q] * jx;
            const double d = lb_weight(q) * (3.0 * cj + 4.5 * cj * cj - 1.5 * jx * jx);
            const size_t o = ((size_t)run * 9 + q) * n + i;
            if (k.bulk_double) reinterpret_cast<double *>(k.post)[o] = d;
            else reinterpret_cast<float *>(k.post)[o] = (float)d;
        }
        const double v = steady_profile(k.g, a, y);
        if (k.bulk_double) reinterpret_cast<double2 *>(k.vel)[(size_t)run * n + i] = make_double2(v, 0.0);
        else reinterpret_cast<float2 *>(k.vel)[(size_t)run * n + i] = make_float2((float)v, 0.0f);
    }
}

cudaError_t launch_init_state(Group &G, cudaStream_t s)
{
    // per-run seeds and noise amplitudes staged through the staging buffer
    const int nr = G.g.nruns;
    unsigned long long *seeds = reinterpret_cast<unsigned long long *>(G.stage);
    double *noise = G.stage + nr;
    std::vector<unsigned long long> hs(nr);
    std::vector<double> hn(nr);
    for (int r = 0; r < nr; ++r) {
        hs[r] = G.run_params[r].seed;
        hn[r] = G.run_params[r].noise_amp;
    }
    cudaError_t e = cudaMemcpyAsync(seeds, hs.data(), nr * sizeof(unsigned long long), cudaMemcpyHostToDevice, s);
    if (e) return e;
    e = cudaMemcpyAsync(noise, hn.data(), nr * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e) return e;
    InitK k;
    k.g = G.g;
    k.omega = G.omega;
    k.seeds = seeds;
    k.noise = noise;
    k.f0_lat = G.f0_lat;
    k.post = G.pop[0];
    k.vel = G.vel;
    k.bulk_double = G.prec == EPD_LB_PLAIN_FP64;
    long long b = (G.g.n + kThreads - 1) / kThreads;
    if (b > 1024) b = 1024;
    init_state<<<dim3((unsigned)b, nr), kThreads, 0, s>>>(k);
    e = cudaGetLastError();
    if (e) return e;
    // the host vectors must outlive the copies
    return cudaStreamSynchronize(s);
}

// ---------------------------------------------------------------------------
// State access
// ---------------------------------------------------------------------------

template <typename T>
__global__ void gather_pre(const T *post, double *dst, int nx, int ny, int logx, long long n)
{
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (site >= n) return;
    int x, y;
    site_xy(site, nx, logx, x, y);
    const int sx = wrap(x - c_cx[q], nx), sy = wrap(y - c_cy[q], ny);
    dst[(size_t)q * n + site] = (double)post[(size_t)q * n + (long long)sy * nx + sx] + lb_weight(q);
}

template <typename T>
__global__ void scatter_pre(T *post, const double *src, int nx, int ny, int logx, long long n)
{
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (site >= n) return;
    int x, y;
    site_xy(site, nx, logx, x, y);
    const int sx = wrap(x + c_cx[q], nx), sy = wrap(y + c_cy[q], ny);
    post[(size_t)q * n + site] = (T)(src[(size_t)q * n + (long long)sy * nx + sx] - lb_weight(q));
}

cudaError_t launch_gather_pre_collision(Group &G, int run, int parity, double *dst, cudaStream_t s)
{
    const dim3 grid((unsigned)((G.g.n + kThreads - 1) / kThreads), 9);
    if (G.prec == EPD_LB_MIXED_FP32)
        gather_pre<float><<<grid, kThreads, 0, s>>>(reinterpret_cast<const float *>(G.pop[parity]) + (size_t)run * 9 * G.g.n, dst,
                                                    G.g.nx, G.g.ny, G.g.logx, G.g.n);
    else
        gather_pre<double><<<grid, kThreads, 0, s>>>(reinterpret_cast<const double *>(G.pop[parity]) + (size_t)run * 9 * G.g.n, dst,
                                                     G.g.nx, G.g.ny, G.g.logx, G.g.n);
    return cudaGetLastError();
}

cudaError_t launch_scatter_pre_collision(Group &G, int run, int parity, const double *src, cudaStream_t s)
{
    const dim3 grid((unsigned)((G.g.n + kThreads - 1) / kThreads), 9);
    if (G.prec == EPD_LB_MIXED_FP32)
        scatter_pre<float><<<grid, kThreads, 0, s>>>(reinterpret_cast<float *>(G.pop[parity]) + (size_t)run * 9 * G.g.n, src,
                                                     G.g.nx, G.g.ny, G.g.logx, G.g.n);
    else
        scatter_pre<double><<<grid, kThreads, 0, s>>>(reinterpret_cast<double *>(G.pop[parity]) + (size_t)run * 9 * G.g.n, src,
                                                      G.g.nx, G.g.ny, G.g.logx, G.g.n);
    return cudaGetLastError();
}

template <typename T>
__global__ void vel_convert(const V2<T> *vin, double *vout, V2<T> *vback, const double *vsrc, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (vout) {
        const V2<T> v = vin[i];
        vout[i] = (double)v.x;
        vout[n + i] = (double)v.y;
    } else {
        vback[i] = mk<T>((T)vsrc[i], (T)vsrc[n + i]);
    }
}

cudaError_t launch_vel_to_f64(Group &G, int run, double *dst, cudaStream_t s)
{
    const unsigned b = (unsigned)((G.g.n + kThreads - 1) / kThreads);
    if (G.prec == EPD_LB_MIXED_FP32)
        vel_convert<float><<<b, kThreads, 0, s>>>(reinterpret_cast<const float2 *>(G.vel) + (size_t)run * G.g.n, dst, nullptr, nullptr, G.g.n);
    else
        vel_convert<double><<<b, kThreads, 0, s>>>(reinterpret_cast<const double2 *>(G.vel) + (size_t)run * G.g.n, dst, nullptr, nullptr, G.g.n);
    return cudaGetLastError();
}

cudaError_t launch_vel_from_f64(Group &G, int run, const double *src, cudaStream_t s)
{
    const unsigned b = (unsigned)((G.g.n + kThreads - 1) / kThreads);
    if (G.prec == EPD_LB_MIXED_FP32)
        vel_convert<float><<<b, kThreads, 0, s>>>(nullptr, nullptr, reinterpret_cast<float2 *>(G.vel) + (size_t)run * G.g.n, src, G.g.n);
    else
        vel_convert<double><<<b, kThreads, 0, s>>>(nullptr, nullptr, reinterpret_cast<double2 *>(G.vel) + (size_t)run * G.g.n, src, G.g.n);
    return cudaGetLastError();
}

// Raw copy of a run's stored populations (post-collision deviations from the
// rest weights, [i][site]) to or from FP64, for exact checkpoints.
template <typename T>
__global__ void pop_raw(T *pop, double *dst, const double *src, long long cnt)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    if (dst) dst[i] = (double)pop[i];
    else pop[i] = (T)src[i];
}

cudaError_t launch_pop_raw(Group &G, int run, int parity, double *dst, const double *src, cudaStream_t s)
{
    const long long cnt = 9 * G.g.n;
    const unsigned b = (unsigned)((cnt + kThreads - 1) / kThreads);
    if (G.prec == EPD_LB_MIXED_FP32)
        pop_raw<float><<<b, kThreads, 0, s>>>(reinterpret_cast<float *>(G.pop[parity]) + (size_t)run * cnt, dst, src, cnt);
    else
        pop_raw<double><<<b, kThreads, 0, s>>>(reinterpret_cast<double *>(G.pop[parity]) + (size_t)run * cnt, dst, src, cnt);
    return cudaGetLastError();
}

// Observables of one run: <Phi_A>, <Phi_B>, <Phi_S>, sigma (Eq. (21)), LB
// mass / sites, max |u|, Q_P, Q_S.  Stage 1: each block of a fixed grid of
// red_blocks(n) blocks writes its five sums and its max into part (slot k of
// block j at k * kRedBlocks + j); stage 2: one block sums the partials in a
// fixed order, so a rerun is bitwise equal.
static int red_blocks(long long n)
{
    const long long b = (n + kThreads - 1) / kThreads;
    return (int)(b < 1 ? 1 : (b > kRedBlocks ? kRedBlocks : b));
}

template <typename T>
__global__ void __launch_bounds__(kThreads) observables_part(const double *phi, const T *post, const V2<T> *vel,
                                                         double phi_p, long long n, double *part)
{
    __shared__ double red[32];
    double sa = 0, sb = 0, ss = 0, sg = 0, sm = 0, vmax = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double a = phi[i], b = phi[n + i];
        sa += a;
        sb += b;
        ss += phi[2 * n + i];
        sg += fabs(a + b - phi_p);
        double m = 0;
        for (int qq = 0; qq < 9; ++qq) m += (double)post[(size_t)qq * n + i];
        sm += m;
        const V2<T> v = vel[i];
        const double vv = sqrt((double)v.x * v.x + (double)v.y * v.y);
        vmax = vv > vmax ? vv : vmax;
    }
    double *o = part + blockIdx.x;
    double r;
    r = block_sum(sa, red); if (threadIdx.x == 0) o[0 * kRedBlocks] = r;
    r = block_sum(sb, red); if (threadIdx.x == 0) o[1 * kRedBlocks] = r;
    r = block_sum(ss, red); if (threadIdx.x == 0) o[2 * kRedBlocks] = r;
    r = block_sum(sg, red); if (threadIdx.x == 0) o[3 * kRedBlocks] = r;
    r = block_sum(sm, red); if (threadIdx.x == 0) o[4 * kRedBlocks] = r;
    for (int w = 16; w > 0; w >>= 1) vmax = fmax(vmax, __shfl_down_sync(0xffffffffu, vmax, w));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = vmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        o[5 * kRedBlocks] = m;
    }
}

__global__ void __launch_bounds__(kThreads) observables_fin(const double *part, int nb, const double *q, long long n,
                                                        double *out)
{
    __shared__ double red[32];
    const double inv = 1.0 / (double)n;
    for (int k = 0; k < 5; ++k) {
        double v = 0;
        for (int j = threadIdx.x; j < nb; j += blockDim.x) v += part[k * kRedBlocks + j];
        const double r = block_sum(v, red);
        if (threadIdx.x == 0) out[k] = k == 4 ? 1.0 + r * inv : r * inv;
    }
    double vmax = 0;
    for (int j = threadIdx.x; j < nb; j += blockDim.x) vmax = fmax(vmax, part[5 * kRedBlocks + j]);
    for (int w = 16; w > 0; w >>= 1) vmax = fmax(vmax, __shfl_down_sync(0xffffffffu, vmax, w));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = vmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        out[5] = m;
        out[6] = q[0];
        out[7] = q[1];
    }
}

cudaError_t launch_observables(Group &G, int run, int parity, double *part, double *out_dev, cudaStream_t s)
{
    const long long n = G.g.n;
    const int nb = red_blocks(n);
    if (G.prec == EPD_LB_MIXED_FP32)
        observables_part<float><<<nb, kThreads, 0, s>>>(G.phi + (size_t)run * 3 * n, reinterpret_cast<const float *>(G.pop[parity]) + (size_t)run * 9 * n,
                                                        reinterpret_cast<const float2 *>(G.vel) + (size_t)run * n, G.g.phi_p, n, part);
    else
        observables_part<double><<<nb, kThreads, 0, s>>>(G.phi + (size_t)run * 3 * n, reinterpret_cast<const double *>(G.pop[parity]) + (size_t)run * 9 * n,
                                                         reinterpret_cast<const double2 *>(G.vel) + (size_t)run * n, G.g.phi_p, n, part);
    observables_fin<<<1, kThreads, 0, s>>>(part, nb, G.q + 2 * run, n, out_dev);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// D3Q19 collide-stream (the three-dimensional scheme named for the extension
// to 3D, Sec. 2), FP64, in the mode form of the D2Q9 update above: u =
// (j + f/2)/rho; j* = j + f; the stress relaxes about rho c_s^2 I + rho u u
// (traceless part by gamma_s, trace by gamma_b) and gains Sigma of Eq. (15)
// with its d = 3 constants; the ghost part (what the second-order projection
// on rho, j, Pi leaves of a population) is scaled by gamma_g.  Push
// streaming into a second array: out_i(r + c_i) = n_i*(r).
// ---------------------------------------------------------------------------

__constant__ int c3[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},  {0, 0, 1},  {0, 0, -1},
                              {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},
                              {-1, 0, 1}, {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

__device__ __forceinline__ double lb3_weight(int i) { return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }

__global__ void __launch_bounds__(kThreads) lb3d_step_k(int nx, int ny, int nz, double gs, double gb, double gg,
                                                        const double *in, const double *force, double *out, double *vel)
{
    const long long n = (long long)nx * ny * nz;
    const long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= n) return;
    const int x = (int)(site % nx), y = (int)((site / nx) % ny), z = (int)(site / ((long long)nx * ny));
    double nl[19];
    double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0, pxx = 0.0, pyy = 0.0, pzz = 0.0, pxy = 0.0, pxz = 0.0, pyz = 0.0;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const double v = in[(size_t)i * n + site];
        const double cx = c3[i][0], cy = c3[i][1], cz = c3[i][2];
        nl[i] = v;
        rho += v;
        jx += v * cx;
        jy += v * cy;
        jz += v * cz;
        pxx += v * cx * cx;
        pyy += v * cy * cy;
        pzz += v * cz * cz;
        pxy += v * cx * cy;
        pxz += v * cx * cz;
        pyz += v * cy * cz;
    }
    const double fx = force[site], fy = force[n + site], fz = force[2 * n + site];
    const double ux = (jx + 0.5 * fx) / rho, uy = (jy + 0.5 * fy) / rho, uz = (jz + 0.5 * fz) / rho;
    vel[site] = ux;
    vel[n + site] = uy;
    vel[2 * n + site] = uz;
    const double cs2 = 1.0 / 3.0;
    // non-equilibrium stress, its trace, and the post-collision M* = Pi* - rho c_s^2 I
    const double nxx = pxx - rho * (ux * ux + cs2), nyy = pyy - rho * (uy * uy + cs2), nzz = pzz - rho * (uz * uz + cs2);
    const double nxy = pxy - rho * ux * uy, nxz = pxz - rho * ux * uz, nyz = pyz - rho * uy * uz;
    const double t3 = (nxx + nyy + nzz) / 3.0, uf = ux * fx + uy * fy + uz * fz;
    const double hs = 0.5 * (1.0 + gs), hb = (1.0 + gb) / 3.0;
    const double dxx = gs * (nxx - t3) + gb * t3 + hs * (2.0 * ux * fx - 2.0 / 3.0 * uf) + hb * uf;
    const double dyy = gs * (nyy - t3) + gb * t3 + hs * (2.0 * uy * fy - 2.0 / 3.0 * uf) + hb * uf;
    const double dzz = gs * (nzz - t3) + gb * t3 + hs * (2.0 * uz * fz - 2.0 / 3.0 * uf) + hb * uf;
    const double sxx = rho * ux * ux + dxx, syy = rho * uy * uy + dyy, szz = rho * uz * uz + dzz;
    const double sxy = rho * ux * uy + gs * nxy + hs * (ux * fy + uy * fx);
    const double sxz = rho * ux * uz + gs * nxz + hs * (ux * fz + uz * fx);
    const double syz = rho * uy * uz + gs * nyz + hs * (uy * fz + uz * fy);
    // M = Pi - rho c_s^2 I of the incoming populations (for their ghost part)
    const double mxx = pxx - rho * cs2, myy = pyy - rho * cs2, mzz = pzz - rho * cs2;
    const double jsx = jx + fx, jsy = jy + fy, jsz = jz + fz;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const double cx = c3[i][0], cy = c3[i][1], cz = c3[i][2], w = lb3_weight(i);
        // (c c - c_s^2 I) : M for the old and the post-collision moments
        const double qold = mxx * (cx * cx - cs2) + myy * (cy * cy - cs2) + mzz * (cz * cz - cs2) +
                            2.0 * (pxy * cx * cy + pxz * cx * cz + pyz * cy * cz);
        const double qnew = sxx * (cx * cx - cs2) + syy * (cy * cy - cs2) + szz * (cz * cz - cs2) +
                            2.0 * (sxy * cx * cy + sxz * cx * cz + syz * cy * cz);
        const double hold = w * (rho + 3.0 * (jx * cx + jy * cy + jz * cz) + 4.5 * qold);
        const double hnew = w * (rho + 3.0 * (jsx * cx + jsy * cy + jsz * cz) + 4.5 * qnew);
        int xd = x + c3[i][0], yd = y + c3[i][1], zd = z + c3[i][2];
        xd = xd < 0 ? xd + nx : (xd >= nx ? xd - nx : xd);
        yd = yd < 0 ? yd + ny : (yd >= ny ? yd - ny : yd);
        zd = zd < 0 ? zd + nz : (zd >= nz ? zd - nz : zd);
        out[(size_t)i * n + ((long long)zd * ny + yd) * nx + xd] = hnew + gg * (nl[i] - hold);
    }
}

cudaError_t launch_lb3d_step(int nx, int ny, int nz, double gs, double gb, double gg, const double *in,
                             const double *force, double *out, double *vel, cudaStream_t s)
{
    const long long n = (long long)nx * ny * nz;
    lb3d_step_k<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(nx, ny, nz, gs, gb, gg, in, force, out, vel);
    return cudaGetLastError();
}

} // namespace epdlb

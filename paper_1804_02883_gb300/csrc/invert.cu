// invert.cu -- vector work of the Fletcher-Reeves inversion omega~ =
// Phi^{-1}(Phi~) of the exact step (Sec. 2, the integrator paragraph; App. C,
// items 2 and 3) on sm_103a.
//
// The mismatch g = Phi~ - Phi(omega) is n times the gradient of the convex
// function G(omega) = <sum_I omega_I Phi~_I> + (phi_p/N) ln Q_P +
// (1 - phi_p) ln Q_S, whose Hessian is the correlator P_IJ of Eq. (4); CG
// minimises G.  One iteration per run:
//   slope at the trial point omega + alpha_t d  ->  secant step alpha,
//   omega += alpha d,  new mismatch g',
//   beta = |g'|^2 / |g|^2,  d = -g' + beta d  (restarted as -g' when that is
//   not a descent direction),  alpha_t = alpha.
// The two solves of an iteration are the propagator launches; the kernels
// here are the FP64 dot products over the 3n fields of each run (fixed-order
// partials and sums: a rerun is bitwise equal), the per-run scalar logic and
// the vector updates.  Runs that reached the tolerance are frozen (alpha = 0).
#include <cmath>

#include "common.cuh"
#include "engine.h"

namespace epdlb {
namespace {

constexpr int kCgThreads = 256;
constexpr int CG_UPD = CG_BETA + 1;  // slot: the direction is updated in this iteration
static_assert(CG_UPD < kCgSlots, "inversion slots");

enum DotKind { DOT_GG = 0, DOT_HT = 1, DOT_NEW = 2 };
enum Stage { ST_BEGIN = 0, ST_ALPHA = 1, ST_DIR = 2 };

// Per block: with g = target - phi,
//   DOT_GG: (g.g, 0);  DOT_HT: (g.d, 0);  DOT_NEW: (g.g, g.d).
template <int KIND>
__global__ void __launch_bounds__(kCgThreads) cg_dots(long long m, const double *target, const double *phi,
                                                       const double *dir, double *part)
{
    __shared__ double sa[kCgThreads / 32], sb[kCgThreads / 32];
    const int run = blockIdx.y;
    const double *t = target + (size_t)run * m, *p = phi + (size_t)run * m, *d = dir + (size_t)run * m;
    double a = 0.0, b = 0.0;
    for (long long i = (long long)blockIdx.x * kCgThreads + threadIdx.x; i < m; i += (long long)gridDim.x * kCgThreads) {
        const double g = t[i] - p[i];
        if (KIND == DOT_GG) {
            a += g * g;
        } else if (KIND == DOT_HT) {
            a += g * d[i];
        } else {
            a += g * g;
            b += g * d[i];
        }
    }
    for (int o = 16; o; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sa[w] = a;
        sb[w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int i = 0; i < kCgThreads / 32; ++i) {
            x += sa[i];
            y += sb[i];
        }
        double *o = part + ((size_t)run * gridDim.x + blockIdx.x) * 2;
        o[0] = x;
        o[1] = y;
    }
}

// Per run (one warp): the sums of the partials (lane-strided, then a fixed
// shuffle tree) and the scalar logic (lane 0).
template <int STAGE>
__global__ void cg_scalar(long long n, int nblk, const double *part, double *cg, double tol)
{
    const int run = blockIdx.x, lane = threadIdx.x;
    double a = 0.0, b = 0.0;
    for (int i = lane; i < nblk; i += 32) {
        a += part[((size_t)run * nblk + i) * 2];
        b += part[((size_t)run * nblk + i) * 2 + 1];
    }
    for (int o = 16; o; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane) return;
    double *c = cg + (size_t)run * kCgSlots;
    if (STAGE == ST_BEGIN) {
        // g.g at the starting guess; d = -g, so g.d = -g.g
        const double res = sqrt(a / (double)n);
        c[CG_GG] = a;
        c[CG_H0] = -a;
        c[CG_AT] = 1.0;
        c[CG_ALPHA] = 0.0;
        c[CG_RES] = res;
        c[CG_RES0] = res;
        c[CG_ITERS] = 0.0;
        c[CG_BETA] = 0.0;
        c[CG_UPD] = 0.0;
        c[CG_ACTIVE] = (tol <= 0.0 || res >= tol) ? 1.0 : 0.0;
    } else if (STAGE == ST_ALPHA) {
        // secant on the slope -g.d / n between alpha = 0 and alpha_t
        if (c[CG_ACTIVE] != 0.0) {
            const double h0 = c[CG_H0], den = h0 - a;
            c[CG_ALPHA] = den < 0.0 ? c[CG_AT] * h0 / den : c[CG_AT];
        } else {
            c[CG_ALPHA] = 0.0;
        }
    } else {
        if (c[CG_ACTIVE] != 0.0) {
            const double gg = c[CG_GG];
            double beta = gg > 0.0 ? a / gg : 0.0;
            double h0 = -a + beta * b;
            if (h0 >= 0.0) {  // not a descent direction: restart with -g
                h0 = -a;
                beta = 0.0;
            }
            const double res = sqrt(a / (double)n);
            c[CG_BETA] = beta;
            c[CG_H0] = h0;
            c[CG_GG] = a;
            c[CG_RES] = res;
            c[CG_AT] = c[CG_ALPHA];
            c[CG_ITERS] += 1.0;
            c[CG_UPD] = 1.0;
            c[CG_ACTIVE] = (tol <= 0.0 || res >= tol) ? 1.0 : 0.0;
        } else {
            c[CG_UPD] = 0.0;
        }
    }
}

// trial = omega + alpha_t d (active runs), omega (frozen runs)
__global__ void __launch_bounds__(kCgThreads) cg_trial_k(long long m, const double *omega, const double *dir,
                                                          const double *cg, double *trial)
{
    const int run = blockIdx.y;
    const double *c = cg + (size_t)run * kCgSlots;
    const double a = c[CG_ACTIVE] != 0.0 ? c[CG_AT] : 0.0;
    const size_t o = (size_t)run * m;
    for (long long i = (long long)blockIdx.x * kCgThreads + threadIdx.x; i < m; i += (long long)gridDim.x * kCgThreads)
        trial[o + i] = omega[o + i] + a * dir[o + i];
}

// omega += alpha d (alpha = 0 for frozen runs)
__global__ void __launch_bounds__(kCgThreads) cg_step_k(long long m, double *omega, const double *dir, const double *cg)
{
    const int run = blockIdx.y;
    const double a = cg[(size_t)run * kCgSlots + CG_ALPHA];
    const size_t o = (size_t)run * m;
    for (long long i = (long long)blockIdx.x * kCgThreads + threadIdx.x; i < m; i += (long long)gridDim.x * kCgThreads)
        omega[o + i] += a * dir[o + i];
}

// d = -g (BEGIN), d = -g + beta d (runs that iterated)
template <bool BEGIN>
__global__ void __launch_bounds__(kCgThreads) cg_dir_k(long long m, const double *target, const double *phi,
                                                        double *dir, const double *cg)
{
    const int run = blockIdx.y;
    const double *c = cg + (size_t)run * kCgSlots;
    if (!BEGIN && c[CG_UPD] == 0.0) return;
    const double beta = BEGIN ? 0.0 : c[CG_BETA];
    const size_t o = (size_t)run * m;
    for (long long i = (long long)blockIdx.x * kCgThreads + threadIdx.x; i < m; i += (long long)gridDim.x * kCgThreads) {
        const double g = target[o + i] - phi[o + i];
        dir[o + i] = BEGIN ? -g : -g + beta * dir[o + i];
    }
}

} // namespace

cudaError_t cg_begin(Group &G, const double *phi, double tol, cudaStream_t s)
{
    const long long m = 3 * G.g.n;
    const dim3 grid(kCgBlocks, G.g.nruns);
    cg_dots<DOT_GG><<<grid, kCgThreads, 0, s>>>(m, G.cg_target, phi, G.cg_dir, G.cg_part);
    cg_scalar<ST_BEGIN><<<G.g.nruns, 32, 0, s>>>(G.g.n, kCgBlocks, G.cg_part, G.cg, tol);
    cg_dir_k<true><<<grid, kCgThreads, 0, s>>>(m, G.cg_target, phi, G.cg_dir, G.cg);
    return cudaGetLastError();
}

cudaError_t cg_trial_point(Group &G, const double *omega, double *trial, cudaStream_t s)
{
    const long long m = 3 * G.g.n;
    cg_trial_k<<<dim3(kCgBlocks, G.g.nruns), kCgThreads, 0, s>>>(m, omega, G.cg_dir, G.cg, trial);
    return cudaGetLastError();
}

cudaError_t cg_line_step(Group &G, const double *phi_trial, double *omega, cudaStream_t s)
{
    const long long m = 3 * G.g.n;
    const dim3 grid(kCgBlocks, G.g.nruns);
    cg_dots<DOT_HT><<<grid, kCgThreads, 0, s>>>(m, G.cg_target, phi_trial, G.cg_dir, G.cg_part);
    cg_scalar<ST_ALPHA><<<G.g.nruns, 32, 0, s>>>(G.g.n, kCgBlocks, G.cg_part, G.cg, 0.0);
    cg_step_k<<<grid, kCgThreads, 0, s>>>(m, omega, G.cg_dir, G.cg);
    return cudaGetLastError();
}

cudaError_t cg_direction(Group &G, const double *phi, double tol, cudaStream_t s)
{
    const long long m = 3 * G.g.n;
    const dim3 grid(kCgBlocks, G.g.nruns);
    cg_dots<DOT_NEW><<<grid, kCgThreads, 0, s>>>(m, G.cg_target, phi, G.cg_dir, G.cg_part);
    cg_scalar<ST_DIR><<<G.g.nruns, 32, 0, s>>>(G.g.n, kCgBlocks, G.cg_part, G.cg, tol);
    cg_dir_k<false><<<grid, kCgThreads, 0, s>>>(m, G.cg_target, phi, G.cg_dir, G.cg);
    return cudaGetLastError();
}

} // namespace epdlb

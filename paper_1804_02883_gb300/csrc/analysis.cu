// analysis.cu -- analysis of the polymer distribution Phi_P = Phi_A + Phi_B
// on sm_103a (Sec. 3, Sec. 4 of arXiv:1804.02883):
//   sigma_Delta of Eq. (22), mean |Phi_P^a - Phi_P^b| of two runs;
//   Y_2^P of Eq. (30), the width of the polymer distribution across the two
//     opposite channels of the reverse-Poiseuille box (channel centres at
//     L_y/4 and 3 L_y/4, site rows at (y + 1/2) dx);
//   particles: connected clusters of sites with Phi_P >= threshold (4
//     neighbours, periodic), and per particle the gyration tensor of
//     Eq. (27), R and c of Eq. (28), c_rel of Eq. (29).
//
// Particles are labelled by a lock-free union-find: every foreground site
// starts as its own root, each site unites with its right and lower
// neighbour by linking the larger root under the smaller with atomicMin, so a
// parent always has a smaller index than its child (every find terminates)
// and each cluster's root is its smallest site index.  Roots are numbered in
// index order by a block scan.  The tensor uses the moment form of the double
// sum of Eq. (27), G = <w d d^T> - <w d><w d>^T / N (weights w = Phi_P,
// d the shortest periodic offset from the cluster's root, exact for clusters
// narrower than half the box); the moments are FP64 atomics (sums in
// arrival order).
#include <cmath>

#include "common.cuh"
#include "engine.h"

namespace epdlb {
namespace {

constexpr int kScanBlock = 1024;  // sites per block of the root numbering
constexpr int kMoments = 7;       // sites, N, sum w dx, sum w dy, sum w dx^2, sum w dx dy, sum w dy^2

__device__ double block_sum_an(double v, double *red)
{
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += red[i];
    return r;
}

// Stage 1 of the two-stage reductions: a fixed grid of an_blocks(n) blocks of
// kPartThreads, each writing its block sums into part (slot k of block j at
// k * kRedBlocks + j); stage 2 (an_finish) sums the partials of every slot in
// a fixed order, so a rerun is bitwise equal.
constexpr int kPartThreads = 256;

int an_blocks(long long n)
{
    const long long b = (n + kPartThreads - 1) / kPartThreads;
    return (int)(b < 1 ? 1 : (b > kRedBlocks ? kRedBlocks : b));
}

// sum |Phi_P^a - Phi_P^b| (Eq. (22))
__global__ void __launch_bounds__(kPartThreads) an_sigma_delta(const double *pa, const double *pb, long long n, double *part)
{
    __shared__ double red[32];
    double s = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        s += fabs((pa[i] + pa[n + i]) - (pb[i] + pb[n + i]));
    const double r = block_sum_an(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = r;
}

// sum y_c^2 Phi_P and sum y_c^2 (Eq. (30)), y_c the row's distance from the
// centre of its channel
__global__ void __launch_bounds__(kPartThreads) an_width(const double *phi, int nx, int ny, double dx, double *part)
{
    __shared__ double red[32];
    const long long n = (long long)nx * ny;
    const double h = 0.5 * (double)ny;
    double num = 0.0, den = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double yy = (double)(i / nx) + 0.5;
        const double yc = (yy - (yy < h ? 0.5 * h : 1.5 * h)) * dx;
        num += yc * yc * (phi[i] + phi[n + i]);
        den += yc * yc;
    }
    const double a = block_sum_an(num, red);
    const double b = block_sum_an(den, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = a;
        part[kRedBlocks + blockIdx.x] = b;
    }
}

enum AnKind { AN_SIGMA_DELTA = 0, AN_WIDTH = 1 };

// SIGMA_DELTA: out = sum / n;  WIDTH: out = sqrt(sum_num / (phi_p sum_den))
template <int KIND>
__global__ void __launch_bounds__(kPartThreads) an_finish(const double *part, int nb, long long n, double phi_p, double *out)
{
    __shared__ double red[32];
    double a = 0.0, b = 0.0;
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        a += part[j];
        if (KIND == AN_WIDTH) b += part[kRedBlocks + j];
    }
    const double ra = block_sum_an(a, red);
    const double rb = KIND == AN_WIDTH ? block_sum_an(b, red) : 0.0;
    if (threadIdx.x == 0) *out = KIND == AN_WIDTH ? sqrt(ra / (phi_p * rb)) : ra / (double)n;
}

__device__ __forceinline__ int find_root(const int *lab, int i)
{
    int p = __ldcg(lab + i);
    while (p != i) {  // parents have smaller indices: at most i steps
        i = p;
        p = __ldcg(lab + i);
    }
    return i;
}

__global__ void ccl_init(const double *phi, long long n, double thr, int *lab)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        lab[i] = (phi[i] + phi[n + i] >= thr) ? (int)i : -1;
}

__device__ void unite(int *lab, int a, int b, int *err)
{
    a = find_root(lab, a);
    b = find_root(lab, b);
    // every pass links a root or moves b to a smaller index: bounded by the
    // index range; the cap only guards against a logic error
    for (int it = 0; a != b; ++it) {
        if (it > (1 << 26)) {
            atomicOr(err, 8);
            return;
        }
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(lab + b, a);  // link root b under a
        if (old == b) return;
        b = find_root(lab, old);
        a = find_root(lab, a);
    }
}

__global__ void ccl_union(int *lab, int nx, int ny, int *err)
{
    const long long n = (long long)nx * ny;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (lab[i] < 0) continue;
        const int x = (int)(i % nx), y = (int)(i / nx);
        const int r = y * nx + (x + 1 == nx ? 0 : x + 1);
        const int d = (y + 1 == ny ? 0 : y + 1) * nx + x;
        if (__ldcg(lab + r) >= 0) unite(lab, (int)i, r, err);
        if (__ldcg(lab + d) >= 0) unite(lab, (int)i, d, err);
    }
}

__global__ void ccl_flatten(int *lab, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (lab[i] >= 0) lab[i] = find_root(lab, (int)i);
}

// roots per block of kScanBlock sites
__global__ void __launch_bounds__(kScanBlock) ccl_count(const int *lab, long long n, int *bcount)
{
    const long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
    const int f = (i < n && lab[i] == (int)i) ? 1 : 0;
    const int c = __syncthreads_count(f);
    if (threadIdx.x == 0) bcount[blockIdx.x] = c;
}

// exclusive scan of the block counts (one thread, in order) and the total
__global__ void ccl_scan(int *bcount, int nb, int *total)
{
    if (threadIdx.x) return;
    int run = 0;
    for (int b = 0; b < nb; ++b) {
        const int c = bcount[b];
        bcount[b] = run;
        run += c;
    }
    *total = run;
}

// particle number of each root: block offset + rank of the root in its block
__global__ void __launch_bounds__(kScanBlock) ccl_number(const int *lab, long long n, const int *boff, int *pid)
{
    __shared__ int wsum[kScanBlock / 32];
    const long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
    const int f = (i < n && lab[i] == (int)i) ? 1 : 0;
    const unsigned m = __ballot_sync(0xffffffffu, f);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) wsum[w] = __popc(m);
    __syncthreads();
    int before = 0;
    for (int k = 0; k < w; ++k) before += wsum[k];
    if (f) pid[i] = boff[blockIdx.x] + before + __popc(m & ((1u << lane) - 1u));
}

__global__ void ccl_moments(const double *phi, const int *lab, const int *pid, int nx, int ny, int maxp, double *mom,
                            int *labels_out)
{
    const long long n = (long long)nx * ny;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int r = lab[i];
        if (r < 0) {
            if (labels_out) labels_out[i] = -1;
            continue;
        }
        const int k = pid[r];
        if (labels_out) labels_out[i] = k;
        if (k >= maxp) continue;
        const double w = phi[i] + phi[n + i];
        int ox = (int)(i % nx) - r % nx, oy = (int)(i / nx) - r / nx;  // shortest periodic offset from the root
        if (2 * ox > nx) ox -= nx;
        if (2 * ox <= -nx) ox += nx;
        if (2 * oy > ny) oy -= ny;
        if (2 * oy <= -ny) oy += ny;
        double *m = mom + (size_t)k * kMoments;
        atomicAdd(m + 0, 1.0);
        atomicAdd(m + 1, w);
        atomicAdd(m + 2, w * ox);
        atomicAdd(m + 3, w * oy);
        atomicAdd(m + 4, w * ox * ox);
        atomicAdd(m + 5, w * ox * oy);
        atomicAdd(m + 6, w * oy * oy);
    }
}

// per particle: centre, G of Eq. (27), R and c of Eq. (28), c_rel of Eq. (29)
__global__ void ccl_finish(const double *mom, const int *total, int maxp, double dx, double *stats)
{
    const int cnt = min(*total, maxp);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
        const double *m = mom + (size_t)k * kMoments;
        const double N = m[1], mx = m[2] / N, my = m[3] / N;
        const double gxx = (m[4] / N - mx * mx) * dx * dx;
        const double gxy = (m[5] / N - mx * my) * dx * dx;
        const double gyy = (m[6] / N - my * my) * dx * dx;
        const double tr = gxx + gyy, dd = sqrt(0.25 * (gxx - gyy) * (gxx - gyy) + gxy * gxy);
        const double lp = 0.5 * tr + dd, lm = 0.5 * tr - dd;
        const double c = lp - lm, R = sqrt(fmax(lp + lm, 0.0));
        double *st = stats + (size_t)k * 10;
        st[0] = m[0];
        st[1] = N;
        st[4] = gxx;
        st[5] = gxy;
        st[6] = gyy;
        st[7] = R;
        st[8] = c;
        st[9] = R > 0.0 ? c * c / (R * R * R * R) : 0.0;
    }
}

// centre of each particle: root position + mean offset, wrapped into [0, L)
__global__ void ccl_centres(const int *lab, const int *pid, long long n, int nx, int ny, double dx, int maxp,
                            const double *mom, double *stats)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (lab[i] != (int)i) continue;
        const int k = pid[i];
        if (k >= maxp) continue;
        const double *m = mom + (size_t)k * kMoments;
        const double cx = fmod((double)(i % nx) + m[2] / m[1] + nx, (double)nx) * dx;
        const double cy = fmod((double)(i / nx) + m[3] / m[1] + ny, (double)ny) * dx;
        stats[(size_t)k * 10 + 2] = cx;
        stats[(size_t)k * 10 + 3] = cy;
    }
}

int grid_of(long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

} // namespace

cudaError_t launch_sigma_delta(const double *phi_a, const double *phi_b, long long n, double *part, double *out_dev,
                               cudaStream_t s)
{
    const int nb = an_blocks(n);
    an_sigma_delta<<<nb, kPartThreads, 0, s>>>(phi_a, phi_b, n, part);
    an_finish<AN_SIGMA_DELTA><<<1, kPartThreads, 0, s>>>(part, nb, n, 0.0, out_dev);
    return cudaGetLastError();
}

cudaError_t launch_width(const Group &G, int run, double *part, double *out_dev, cudaStream_t s)
{
    const long long n = G.g.n;
    const int nb = an_blocks(n);
    an_width<<<nb, kPartThreads, 0, s>>>(G.phi + (size_t)run * 3 * n, G.g.nx, G.g.ny, G.g.dx, part);
    an_finish<AN_WIDTH><<<1, kPartThreads, 0, s>>>(part, nb, n, G.g.phi_p, out_dev);
    return cudaGetLastError();
}

static size_t r256(size_t b) { return (b + 255) & ~(size_t)255; }

// the pieces carved by launch_particles, each rounded to 256 bytes
size_t particles_scratch_bytes(long long n, int maxp)
{
    const size_t nb = (size_t)((n + kScanBlock - 1) / kScanBlock);
    return 2 * r256((size_t)n * sizeof(int)) + r256(nb * sizeof(int)) + r256(sizeof(int)) +
           r256((size_t)maxp * kMoments * sizeof(double)) + r256((size_t)maxp * 10 * sizeof(double));
}

// scratch: lab (n int), pid (n int), block offsets, total, moments, stats
cudaError_t launch_particles(const Group &G, int run, double thr, int maxp, void *scratch, int *labels_dev,
                             int **total_dev, double **stats_dev, cudaStream_t s)
{
    const long long n = G.g.n;
    const int nb = (int)((n + kScanBlock - 1) / kScanBlock);
    char *p = (char *)scratch;
    auto take = [&](size_t bytes) {
        char *r = p;
        p += r256(bytes);
        return (void *)r;
    };
    int *lab = (int *)take((size_t)n * sizeof(int));
    int *pid = (int *)take((size_t)n * sizeof(int));
    int *boff = (int *)take((size_t)nb * sizeof(int));
    int *total = (int *)take(sizeof(int));
    double *mom = (double *)take((size_t)maxp * kMoments * sizeof(double));
    double *stats = (double *)take((size_t)maxp * 10 * sizeof(double));
    const double *phi = G.phi + (size_t)run * 3 * n;
    cudaError_t e;
    if ((e = cudaMemsetAsync(mom, 0, (size_t)maxp * kMoments * sizeof(double), s))) return e;
    const int gb = grid_of(n, 256);
    ccl_init<<<gb, 256, 0, s>>>(phi, n, thr, lab);
    ccl_union<<<gb, 256, 0, s>>>(lab, G.g.nx, G.g.ny, G.err);
    ccl_flatten<<<gb, 256, 0, s>>>(lab, n);
    ccl_count<<<nb, kScanBlock, 0, s>>>(lab, n, boff);
    ccl_scan<<<1, 32, 0, s>>>(boff, nb, total);
    ccl_number<<<nb, kScanBlock, 0, s>>>(lab, n, boff, pid);
    ccl_moments<<<gb, 256, 0, s>>>(phi, lab, pid, G.g.nx, G.g.ny, maxp, mom, labels_dev);
    ccl_finish<<<grid_of(maxp, 256), 256, 0, s>>>(mom, total, maxp, G.g.dx, stats);
    ccl_centres<<<gb, 256, 0, s>>>(lab, pid, n, G.g.nx, G.g.ny, G.g.dx, maxp, mom, stats);
    *total_dev = total;
    *stats_dev = stats;
    return cudaGetLastError();
}

} // namespace epdlb

// prop.cu -- single-chain solve of the hybrid LB/EPD step (Sec. 2, Eqs. (6)-(11)
// of arXiv:1804.02883) on sm_103a.
//
// Both propagators advance together: the forward propagator g (from the A end,
// Eq. (6)) and the backward propagator g' (from the B end, Eq. (7)) are real, so
// they travel as the real and imaginary parts of one complex field z = g + i g'.
// The Fourier factor exp(-R_G^2 |k|^2 ds) of the split step, Eq. (8), is
// separable, exp(-R_G^2 kx^2 ds) exp(-R_G^2 ky^2 ds), and maps real fields to
// real fields, so one contour step is
//   column pass : z <- IFFT_y[ Ky * FFT_y[ z ] ]              (all columns)
//   row pass    : h <- IFFT_x[ Kx * FFT_x[ z ] ]              (all rows)
//                 z_{j+1} = E(s_{j+1}) h  (g and g' each with its own node field),
//                 store or consume the contour history,
//                 z <- E(s_{j+1}) z_{j+1} (first half of the next step)
// with E = exp(-N w ds / 2).  The history holds nodes 0..floor(N_s/2): while
// the chains run through the second half, node m of g meets node N_s - m of g'
// from the history (and vice versa), and the trapezoid sums of Eqs. (9)-(10)
// are accumulated in FP64 on the fly.  In MIXED_FP32 every node is stored:
// the full history is the reference of the differential second solve
// (prop_row<T, true> and the radix-8 passes below), whose contour sums are a
// separate pass over the stored nodes (prop_contour_stream).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <type_traits>

#include "common.cuh"
#include "engine.h"
#include "fft8.cuh"

namespace epdlb {

template <typename T> struct PropK {
    GroupGeom g;
    V2<T> *chain;
    V2<T> *hist;          // [run][hnodes][n]: nodes 0..half_lo, or all N_s + 1 (reference of a differential solve)
    V2<T> *hd;            // differential solve: (dg, dg') at every node, [run][N_s + 1][n]
    const float2 *rho;    // differential solve: (rho_A, rho_B), [run][n]
    int hnodes;
    const V2<T> *efac;
    double *ia, *ib, *part;
    const V2<T> *twx, *twy;
    const T *kx, *ky;
    int rows, logc, cols;  // tile rows (row pass), columns and their log2 (column pass; logc when pow2)
};

// Trapezoid weights on [0, s_{N_A}] (block A) and [s_{N_A}, 1] (block B).
__device__ __forceinline__ double weight_a(int j, int na, double ds)
{
    if (na == 0 || j > na) return 0.0;
    return (j == 0 || j == na) ? 0.5 * ds : ds;
}
__device__ __forceinline__ double weight_b(int j, int na, int ns, double ds)
{
    if (na == ns || j < na) return 0.0;
    return (j == na || j == ns) ? 0.5 * ds : ds;
}

// Node j of g carries w_A iff j < N_A; node j of g' carries the field of node ns - j.
// Boltzmann factor (E_A, E_B) of the half-step at node j of chain g (fac_g)
// or g' (fac_gp), arriving or departing (half_step_block)
template <typename T> __device__ __forceinline__ T fac_g(V2<T> e, const GroupGeom &g, int j, bool arriving)
{
    return half_step_block(g.jr, 0, j, g.ns, g.na, arriving) ? e.y : e.x;
}
template <typename T> __device__ __forceinline__ T fac_gp(V2<T> e, const GroupGeom &g, int j, bool arriving)
{
    return half_step_block(g.jr, 1, j, g.ns, g.na, arriving) ? e.y : e.x;
}

template <typename T> __device__ __forceinline__ T exp_t(T v);
template <> __device__ __forceinline__ float exp_t<float>(float v) { return expf(v); }
template <> __device__ __forceinline__ double exp_t<double>(double v) { return exp(v); }

// Boltzmann factors E_{A,B} = exp(-N w_{A,B} ds / 2) and exp(-w_S) in the bulk
// precision; exp(-w_S) into the S slot of phi_out and its block sums for Q_S
// (per-thread sums of at most a few terms in the bulk type, FP64 across
// threads and blocks).
template <typename T>
__global__ void __launch_bounds__(kThreads) prop_prep(GroupGeom g, const double *omega, V2<T> *efac, double *phi_out, double *part)
{
    __shared__ double red[32];
    const int run = blockIdx.y;
    const long long n = g.n;
    const double *wa = omega + (size_t)run * 3 * n, *wb = wa + n, *ws = wb + n;
    double *es = phi_out + (size_t)run * 3 * n + 2 * n;
    const T c = (T)(-0.5 * g.nseg * g.ds);
    T acc = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        efac[(size_t)run * n + i] = mk<T>(exp_t<T>(c * (T)wa[i]), exp_t<T>(c * (T)wb[i]));
        // exp(-w_S) in the bulk precision (FP32 in MIXED_FP32), kept in FP64
        const T e = exp_t<T>(-(T)ws[i]);
        es[i] = (double)e;
        acc += e;
    }
    const double s = block_sum((double)acc, red);
    if (threadIdx.x == 0) part[(size_t)run * kMaxPart + kMaxPart / 2 + blockIdx.x] = s;
}

// Node 0: g = g' = 1 stored; chain <- E(s_0) z_0.  Differential solve: the
// change of node 0 is 0, the chain starts from d a_0 = E' - E = E rho of the
// departing half-step.
template <typename T, bool DIFF>
__global__ void __launch_bounds__(kThreads) prop_start(PropK<T> k)
{
    const int run = blockIdx.y;
    const long long n = k.g.n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const V2<T> e = k.efac[(size_t)run * n + i];
        if constexpr (!DIFF) {
            k.hist[(size_t)run * k.hnodes * n + i] = mk<T>((T)1, (T)1);
            k.chain[(size_t)run * n + i] = mk<T>(fac_g<T>(e, k.g, 0, false), fac_gp<T>(e, k.g, 0, false));
        } else {
            const float2 q = k.rho[(size_t)run * n + i];
            k.hd[(size_t)run * (k.g.ns + 1) * n + i] = mk<T>((T)0, (T)0);
            k.chain[(size_t)run * n + i] = mk<T>(fac_g<T>(e, k.g, 0, false) * fac_g<float>(q, k.g, 0, false),
                                                 fac_gp<T>(e, k.g, 0, false) * fac_gp<float>(q, k.g, 0, false));
        }
    }
}

// Column pass: Ty = IFFT_y Ky FFT_y on a tile of C adjacent columns (radix-2
// transforms on power-of-two grids, mixed-radix ones otherwise).
template <typename T>
__global__ void __launch_bounds__(kThreads) prop_col(PropK<T> k)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const bool p2 = k.g.pow2;
    const int ny = k.g.ny, nx = k.g.nx, logy = k.g.logy, logc = k.logc, C = k.cols;
    const int tile = ny * C, ntw = p2 ? ny / 2 : ny;
    V2<T> *a = reinterpret_cast<V2<T> *>(smem_raw);
    V2<T> *b = a + tile;
    V2<T> *tw = b + tile;
    T *ky = reinterpret_cast<T *>(tw + ntw);
    const int run = blockIdx.y, x0 = blockIdx.x * C;
    V2<T> *data = k.chain + (size_t)run * k.g.n;
    auto at = [&](int i) { return p2 ? (size_t)(i >> logc) * nx + x0 + (i & (C - 1)) : (size_t)(i / C) * nx + x0 + i % C; };
    for (int i = threadIdx.x; i < tile; i += blockDim.x) a[i] = data[at(i)];
    for (int i = threadIdx.x; i < ntw; i += blockDim.x) tw[i] = k.twy[i];
    for (int i = threadIdx.x; i < ny; i += blockDim.x) ky[i] = k.ky[i];
    __syncthreads();
    V2<T> *r = p2 ? fft_smem<T, false, true>(a, b, logy, logc, 1, C, tw)
                  : fft_smem_mr<T, false, true>(a, b, ny, k.g.nfy, k.g.fy, C, 1, C, tw);
    V2<T> *o = (r == a) ? b : a;
    for (int i = threadIdx.x; i < tile; i += blockDim.x) r[i] = cscale(r[i], ky[p2 ? i >> logc : i / C]);
    __syncthreads();
    r = p2 ? fft_smem<T, true, true>(r, o, logy, logc, 1, C, tw) : fft_smem_mr<T, true, true>(r, o, ny, k.g.nfy, k.g.fy, C, 1, C, tw);
    for (int i = threadIdx.x; i < tile; i += blockDim.x) data[at(i)] = r[i];
}

// Row pass producing contour node m (1 <= m <= ns): Tx, node factors, history
// store / contour accumulation, Q_P partial sums at m = ns, next half step.
// Differential solve (DIFF): the chain carries the change d a of the state
// E_d g; with U = T(d a_{m-1}) and the reference node g~_m from the history,
//   dg_m = E'_a U + rho_a g~_m,   d a_m = E'_d dg_m + E_d rho_d g~_m
// (E' = E (1 + rho)), the exact differences of g_m = E'_a T(a_{m-1}) and
// a_m = E'_d g_m from the reference solve's g~_m = E_a T(a~_{m-1}) and
// a~_m = E_d g~_m; dg_m is stored at every node, dQ_P partials at m = ns.
constexpr int RB = 4;  // points per thread whose loads the row pass's epilogue issues together
template <typename T, bool DIFF>
__global__ void __launch_bounds__(kThreads) prop_row(PropK<T> k, int m)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    const bool p2 = k.g.pow2;
    const int nx = k.g.nx, logx = k.g.logx, rows = k.rows;
    const int tile = rows * nx, ntw = p2 ? nx / 2 : nx;
    V2<T> *a = reinterpret_cast<V2<T> *>(smem_raw);
    V2<T> *b = a + tile;
    V2<T> *tw = b + tile;
    T *kx = reinterpret_cast<T *>(tw + ntw);
    const int run = blockIdx.y;
    const long long n = k.g.n;
    const long long base = (long long)blockIdx.x * tile;
    V2<T> *data = k.chain + (size_t)run * n + base;
    for (int i = threadIdx.x; i < tile; i += blockDim.x) a[i] = data[i];
    for (int i = threadIdx.x; i < ntw; i += blockDim.x) tw[i] = k.twx[i];
    for (int i = threadIdx.x; i < nx; i += blockDim.x) kx[i] = k.kx[i];
    __syncthreads();
    const int logb = p2 ? ilog2(rows) : 0;
    V2<T> *r = p2 ? fft_smem<T, false, false>(a, b, logx, logb, nx, 1, tw)
                  : fft_smem_mr<T, false, false>(a, b, nx, k.g.nfx, k.g.fx, rows, nx, 1, tw);
    V2<T> *o = (r == a) ? b : a;
    for (int i = threadIdx.x; i < tile; i += blockDim.x) r[i] = cscale(r[i], kx[p2 ? i & (nx - 1) : i % nx]);
    __syncthreads();
    r = p2 ? fft_smem<T, true, false>(r, o, logx, logb, nx, 1, tw) : fft_smem_mr<T, true, false>(r, o, nx, k.g.nfx, k.g.fx, rows, nx, 1, tw);

    const int ns = k.g.ns, na = k.g.na, hlo = k.g.half_lo, hhi = k.g.half_hi;
    const double ds = k.g.ds;
    const V2<T> *efac = k.efac + (size_t)run * n + base;
    V2<T> *hist = k.hist + (size_t)run * k.hnodes * n + base;
    double qsum = 0.0;
    if constexpr (DIFF) {
        const float2 *rho = k.rho + (size_t)run * n + base;
        V2<T> *hd = k.hd + ((size_t)run * (ns + 1) + m) * n + base;
        const V2<T> *gref = hist + (size_t)m * n;
        const int bag = half_step_block(k.g.jr, 0, m, ns, na, true), bap = half_step_block(k.g.jr, 1, m, ns, na, true);
        const int bdg = half_step_block(k.g.jr, 0, m, ns, na, false), bdp = half_step_block(k.g.jr, 1, m, ns, na, false);
        // batches of RB points per thread: the loads first, then the stores
        for (int i0 = threadIdx.x; i0 < tile; i0 += RB * blockDim.x) {
            V2<T> eb[RB], grb[RB];
            float2 qb[RB];
#pragma unroll
            for (int b = 0; b < RB; ++b) {
                const int i = i0 + b * blockDim.x;
                if (i < tile) {
                    eb[b] = efac[i];
                    grb[b] = gref[i];
                    qb[b] = rho[i];
                }
            }
#pragma unroll
            for (int b = 0; b < RB; ++b) {
                const int i = i0 + b * blockDim.x;
                if (i >= tile) break;
                const V2<T> e = eb[b], gr = grb[b], u = r[i];
                const float2 q = qb[b];
                const T ea = bag ? e.y : e.x, eap = bap ? e.y : e.x, qa = bag ? q.y : q.x, qap = bap ? q.y : q.x;
                const V2<T> dg = mk<T>(ea * ((T)1 + qa) * u.x + qa * gr.x, eap * ((T)1 + qap) * u.y + qap * gr.y);
                hd[i] = dg;
                if (m == ns) {
                    qsum += (double)dg.x;
                } else {
                    const T ed = bdg ? e.y : e.x, edp = bdp ? e.y : e.x, qd = bdg ? q.y : q.x, qdp = bdp ? q.y : q.x;
                    data[i] = mk<T>(ed * ((T)1 + qd) * dg.x + ed * qd * gr.x, edp * ((T)1 + qdp) * dg.y + edp * qdp * gr.y);
                }
            }
        }
        if (m == ns) {
            const double s = block_sum(qsum, red);
            if (threadIdx.x == 0) k.part[(size_t)run * kMaxPart + blockIdx.x] = s;
        }
        return;
    }
    const bool store_all = k.hnodes == ns + 1;
    double *ia = k.ia + (size_t)run * n + base, *ib = k.ib + (size_t)run * n + base;
    const int s2 = ns - m;
    // batches of RB points per thread: the loads first, then the stores
    for (int i0 = threadIdx.x; i0 < tile; i0 += RB * blockDim.x) {
        V2<T> eb[RB], hvb[RB];
        double iab[RB], ibb[RB];
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            const int i = i0 + b * blockDim.x;
            if (i < tile) {
                eb[b] = efac[i];
                if (m >= hhi && s2 != m) hvb[b] = hist[(size_t)s2 * n + i];
                if (m > hhi) {
                    iab[b] = ia[i];
                    ibb[b] = ib[i];
                }
            }
        }
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            const int i = i0 + b * blockDim.x;
            if (i >= tile) break;
            const V2<T> e = eb[b];
            // z = (g_m, g'_m): the arriving half-step's factor; the chain goes on
            // with the departing one
            const T eg = fac_g<T>(e, k.g, m, true), egp = fac_gp<T>(e, k.g, m, true);
            const V2<T> h = r[i];
            const V2<T> z = mk<T>(eg * h.x, egp * h.y);
            if (m <= hlo || store_all) hist[(size_t)m * n + i] = z;
            if (m >= hhi) {
                const V2<T> hv = (s2 == m) ? z : hvb[b];
                const double t1 = (double)z.x * (double)hv.y;  // g(s_m) g'(1 - s_m)
                double va = weight_a(m, na, ds) * t1, vb = weight_b(m, na, ns, ds) * t1;
                if (s2 != m) {
                    const double t2 = (double)hv.x * (double)z.y;  // g(s_{ns-m}) g'(s_m)
                    va += weight_a(s2, na, ds) * t2;
                    vb += weight_b(s2, na, ns, ds) * t2;
                }
                if (m == hhi) { ia[i] = va; ib[i] = vb; }
                else { ia[i] = iab[b] + va; ib[i] = ibb[b] + vb; }
            }
            if (m == ns) qsum += (double)z.x;
            else data[i] = mk<T>(fac_g<T>(e, k.g, m, false) * z.x, fac_gp<T>(e, k.g, m, false) * z.y);
        }
    }
    if (m == ns) {
        const double s = block_sum(qsum, red);
        if (threadIdx.x == 0) k.part[(size_t)run * kMaxPart + blockIdx.x] = s;
    }
}

// Normalisation, Eqs. (9)-(11) with Q as spatial means.
// ia2/ib2 (may be null): sums of the second chain's terms (cluster solve).
__global__ void __launch_bounds__(kThreads) prop_finalize(GroupGeom g, int nrow_blocks, int nprep_blocks, const double *ia,
                                                      const double *ib, const double *ia2, const double *ib2,
                                                      const double *part, double *phi, double *q, int *err)
{
    __shared__ double bc;
    const int run = blockIdx.y;
    const long long n = g.n;
    const double *pr = part + (size_t)run * kMaxPart;
    const double qp = sum_partials(pr, nrow_blocks, 1, &bc) / (double)n;
    const double qs = sum_partials(pr + kMaxPart / 2, nprep_blocks, 1, &bc) / (double)n;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        q[2 * run] = qp;
        q[2 * run + 1] = qs;
        if (!(qp > 0.0) || !(qs > 0.0) || !isfinite(qp) || !isfinite(qs)) atomicOr(err, 1);
    }
    const double cp = g.phi_p / qp, cs = (1.0 - g.phi_p) / qs;
    double *pa = phi + (size_t)run * 3 * n, *pb = pa + n, *ps = pb + n;
    const double *ja = ia + (size_t)run * n, *jb = ib + (size_t)run * n;
    const double *ja2 = ia2 ? ia2 + (size_t)run * n : nullptr, *jb2 = ib2 ? ib2 + (size_t)run * n : nullptr;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        pa[i] = cp * (ja2 ? ja[i] + ja2[i] : ja[i]);
        pb[i] = cp * (jb2 ? jb[i] + jb2[i] : jb[i]);
        ps[i] = cs * ps[i];
    }
}

// Differential second solve (MIXED_FP32, cluster solve).  The step's second
// solve differs from its first only by the diffusion update d omega = omega -
// omega~ (Eq. (5)), small next to omega.  Its node factors are E~ (1 + rho),
// rho = expm1(-N d omega ds / 2), and its solvent factor e~ (1 + expm1(
// -d omega_S)), so the changes follow from the FP64 difference with the
// rounding of FP32 relative to the change itself.  The solvent change de goes
// to the S slot of phi, its block sums to the S partials.
__global__ void __launch_bounds__(kThreads) prop_prep_delta(GroupGeom g, const double *omega, const double *omega_t,
                                                            float2 *rho, float *cdiff, double *phi_out, double *part)
{
    __shared__ double red[32];
    const int run = blockIdx.y;
    const long long n = g.n;
    const double *wa = omega + (size_t)run * 3 * n, *wb = wa + n, *ws = wb + n;
    const double *ta = omega_t + (size_t)run * 3 * n, *tb = ta + n, *ts = tb + n;
    double *ds_out = phi_out + (size_t)run * 3 * n + 2 * n;
    const float c = (float)(-0.5 * g.nseg * g.ds);
    float acc = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float da = (float)(wa[i] - ta[i]), db = (float)(wb[i] - tb[i]);
        const float qa = expm1f(c * da), qb = expm1f(c * db);
        rho[(size_t)run * n + i] = make_float2(qa, qb);
        if (cdiff) {
            // (1 + rho_d)(1 + rho_a) - 1 for the block pairs (A, A), (B, B),
            // (A, B) of a node's departing and arriving half-steps, in the
            // packed-row layout of the cluster solve (site (y, x) -> packed
            // row y / 2, component y & 1; power-of-two grids: shift and mask)
            const long long y = i >> g.logx, x = i & (g.nx - 1), hn = n / 2;
            const size_t o = (size_t)((y >> 1) * g.nx + x) * 2 + (y & 1);
            cdiff[((size_t)run * 3 + 0) * hn * 2 + o] = qa * (2.f + qa);
            cdiff[((size_t)run * 3 + 1) * hn * 2 + o] = qb * (2.f + qb);
            cdiff[((size_t)run * 3 + 2) * hn * 2 + o] = qa + qb + qa * qb;
        }
        // e~_S exactly as the first solve formed it
        const float es = expf(-(float)ts[i]);
        const float de = es * expm1f(-(float)(ws[i] - ts[i]));
        ds_out[i] = (double)de;
        acc += de;
    }
    const double s = block_sum((double)acc, red);
    if (threadIdx.x == 0) part[(size_t)run * kMaxPart + kMaxPart / 2 + blockIdx.x] = s;
}

// ---------------------------------------------------------------------------
// Streaming passes on radix-8 tiles (MIXED_FP32, grids too large for the
// cluster-resident solve, 64..2048 points per axis).  The chain z = g + i g'
// is transformed by column tiles then row tiles per contour step, as above;
// the row pass stores z at every node (full history, FP32), and the contour
// sums are one pass over the history afterwards (prop_contour_stream):
// I(r) = sum_j w_j g(s_j) g'(1 - s_j) with g'(1 - s_j) the g' chain at its
// node N_s - j.
// ---------------------------------------------------------------------------

struct Stream8K {
    GroupGeom g;
    float2 *chain;        // [run][n]
    float2 *hist;         // [run][N_s + 1][n] (the reference of a differential solve)
    float2 *hd;           // differential solve: (dg, dg') at every node, [run][N_s + 1][n]
    const float2 *rho;    // differential solve: (rho_A, rho_B), [run][n]
    const float2 *efac;   // [run][n]
    double *part;
    const float2 *twx, *twy;  // pass tables of each axis' best radix plan (fft8.cuh layout)
    const float2 *twy8, *twy16;  // column tables of the radix-8 and radix-16 plans (tile-dependent)
    const float *kx, *ky;
};

// node 0: g = g' = 1; chain <- E(s_0) z_0 (differential solve: change 0,
// chain d a_0 = E rho of the departing half-step)
template <bool DIFF>
__global__ void __launch_bounds__(kThreads) prop_start8(Stream8K k)
{
    const int run = blockIdx.y;
    const long long n = k.g.n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float2 e = k.efac[(size_t)run * n + i];
        if (!DIFF) {
            k.hist[(size_t)run * (k.g.ns + 1) * n + i] = make_float2(1.f, 1.f);
            k.chain[(size_t)run * n + i] = make_float2(fac_g<float>(e, k.g, 0, false), fac_gp<float>(e, k.g, 0, false));
        } else {
            const float2 q = k.rho[(size_t)run * n + i];
            k.hd[(size_t)run * (k.g.ns + 1) * n + i] = make_float2(0.f, 0.f);
            k.chain[(size_t)run * n + i] = make_float2(fac_g<float>(e, k.g, 0, false) * fac_g<float>(q, k.g, 0, false),
                                                       fac_gp<float>(e, k.g, 0, false) * fac_gp<float>(q, k.g, 0, false));
        }
    }
}

template <int LOGY, int CW>
__global__ void __launch_bounds__(ColTile<LOGY, CW>::T) prop_col8(Stream8K k)
{
    using CT = ColTile<LOGY, CW>;
    using CL = ColLayout<LOGY, CT::C>;
    constexpr int NY = CT::NY, C = CT::C, P = CT::P, T = CT::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    const int nx = k.g.nx, run = blockIdx.y, x0 = blockIdx.x * C, tid = threadIdx.x;
    float2 *data = k.chain + (size_t)run * k.g.n;
#pragma unroll
    for (int u = 0; u < P / T; ++u) {
        const int i = tid + u * T;
        buf[i] = data[(size_t)(i / C) * nx + x0 + (i % C)];
    }
    __syncthreads();
    // twiddle tables and Fourier factors straight from global memory (L1):
    // shared memory holds only the tile, so more tiles are in flight per SM
    transform_pair<LOGY, T, CL, P, ScaleBins, CT::MR>(buf, CT::MR == 4 ? k.twy16 : k.twy8, ScaleBins{k.ky}, tid);
    constexpr int RLOG_L = inv_rlog(LOGY, npasses(LOGY, CT::MR) - 1, CT::MR), RR = 1 << RLOG_L, PER_L = NY / RR, NB_L = P / RR / T;
    float2 h[NB_L][RR];
    int bb[NB_L], tt[NB_L];
    last_inverse<LOGY, NB_L, T, CL, CT::MR>(buf, h, bb, tt, tid);
#pragma unroll
    for (int j = 0; j < NB_L; ++j)
#pragma unroll
        for (int r = 0; r < RR; ++r) data[(size_t)(tt[j] + r * PER_L) * nx + x0 + bb[j]] = h[j][r];
}

// Row pass of contour node m: Tx, node factors, history store, next half
// step; at m = N_s block sums of g for Q_P.  Differential solve (DIFF): the
// chain carries d a; dg_m = E'_a U + rho_a g~_m is stored, the chain goes on
// with d a_m = E'_d dg_m + E_d rho_d g~_m (as in prop_row), dQ_P partials.
template <int LOGX, bool DIFF>
__global__ void __launch_bounds__(RowTile<LOGX>::T) prop_row8(Stream8K k, int m)
{
    using RT = RowTile<LOGX>;
    using RL = RowLayout<LOGX>;
    constexpr int NX = RT::NX, P = RT::P, T = RT::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    const int run = blockIdx.y, tid = threadIdx.x;
    const long long n = k.g.n, base = (long long)blockIdx.x * P;
    const int ns = k.g.ns;
    float2 *data = k.chain + (size_t)run * n + base;
#pragma unroll
    for (int u = 0; u < P / T; ++u) {
        const int i = tid + u * T;
        buf[RL::at(i / NX, i % NX)] = data[i];
    }
    __syncthreads();
    transform_pair<LOGX, T, RL, P, ScaleBins, RT::MR>(buf, k.twx, ScaleBins{k.kx}, tid);
    constexpr int RLOG_L = inv_rlog(LOGX, npasses(LOGX, RT::MR) - 1, RT::MR), RR = 1 << RLOG_L, PER_L = NX / RR, NB_L = P / RR / T;
    float2 h[NB_L][RR];
    int bb[NB_L], tt[NB_L];
    last_inverse<LOGX, NB_L, T, RL, RT::MR>(buf, h, bb, tt, tid);
    const float2 *efac = k.efac + (size_t)run * n + base;
    float2 *hist = k.hist + ((size_t)run * (ns + 1) + m) * n + base;
    float qsum = 0.f;
    // per batch of RR points: every load first, then the stores (the
    // history and chain stores could alias the inputs as far as the compiler
    // knows, which would serialise each load behind the previous stores)
    if (DIFF) {
        const float2 *rho = k.rho + (size_t)run * n + base;
        float2 *hd = k.hd + ((size_t)run * (ns + 1) + m) * n + base;
#pragma unroll
        for (int j = 0; j < NB_L; ++j) {
            float2 e[RR], q[RR], gr[RR];
#pragma unroll
            for (int r = 0; r < RR; ++r) {
                const int i = bb[j] * NX + tt[j] + r * PER_L;
                e[r] = efac[i];
                q[r] = rho[i];
                gr[r] = hist[i];
            }
#pragma unroll
            for (int r = 0; r < RR; ++r) {
                const int i = bb[j] * NX + tt[j] + r * PER_L;
                const float2 u = h[j][r];
                const float ea = fac_g<float>(e[r], k.g, m, true), eap = fac_gp<float>(e[r], k.g, m, true);
                const float qa = fac_g<float>(q[r], k.g, m, true), qap = fac_gp<float>(q[r], k.g, m, true);
                const float2 dg = make_float2(ea * (1.f + qa) * u.x + qa * gr[r].x, eap * (1.f + qap) * u.y + qap * gr[r].y);
                hd[i] = dg;
                if (m == ns) {
                    qsum += dg.x;
                } else {
                    const float ed = fac_g<float>(e[r], k.g, m, false), edp = fac_gp<float>(e[r], k.g, m, false);
                    const float qd = fac_g<float>(q[r], k.g, m, false), qdp = fac_gp<float>(q[r], k.g, m, false);
                    data[i] = make_float2(ed * (1.f + qd) * dg.x + ed * qd * gr[r].x,
                                          edp * (1.f + qdp) * dg.y + edp * qdp * gr[r].y);
                }
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < NB_L; ++j) {
            float2 e[RR];
#pragma unroll
            for (int r = 0; r < RR; ++r) e[r] = efac[bb[j] * NX + tt[j] + r * PER_L];
#pragma unroll
            for (int r = 0; r < RR; ++r) {
                const int i = bb[j] * NX + tt[j] + r * PER_L;
                const float eg = fac_g<float>(e[r], k.g, m, true), egp = fac_gp<float>(e[r], k.g, m, true);
                const float2 z = make_float2(eg * h[j][r].x, egp * h[j][r].y);
                hist[i] = z;
                if (m == ns) qsum += z.x;
                else data[i] = make_float2(fac_g<float>(e[r], k.g, m, false) * z.x, fac_gp<float>(e[r], k.g, m, false) * z.y);
            }
        }
    }
    if (m == ns) {
        const double s = block_sum((double)qsum, red);
        if (tid == 0) k.part[(size_t)run * kMaxPart + blockIdx.x] = s;
    }
}

// Contour sums and normalisation over the full history (Eqs. (9)-(11)):
// FP32 products, partial sums over up to 8 nodes of equal trapezoid weight,
// FP64 totals; the solvent slot of phi holds exp(-omega_S) from prop_prep.
// Differential solve (DIFF): the sums of the product's change
// g~ dg' + dg g~' + dg dg' (reference history hist, changes hd), the
// partials hold dQ_P and the solvent factor's change, and
// Phi = Phi~ + (phi_p ds dI - Phi~ dQ) / (Q~ + dQ) per species.
template <bool DIFF>
__global__ void __launch_bounds__(kThreads) prop_contour_stream(GroupGeom g, const float2 *hist, const float2 *hd,
                                                                int nrow_blocks, int nprep_blocks, const double *part,
                                                                double *phi, double *q, const double *phi_ref,
                                                                const double *q_ref, int *err)
{
    __shared__ double bc;
    const int run = blockIdx.y, ns = g.ns, na = g.na;
    const long long n = g.n;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    const float2 *hz = hist + (size_t)run * (ns + 1) * n + i;
    const float2 *dz = DIFF ? hd + (size_t)run * (ns + 1) * n + i : nullptr;
    // Nodes m and N_s - m are read together: z_m = (g_m, g'_m) and z_{N_s-m}
    // give the terms g_m g'_{N_s-m} (node m) and g_{N_s-m} g'_m (node N_s - m).
    // Compensated (Kahan) FP32 sums per block (GB300's FP64 rate is a small
    // fraction of FP32); the trapezoid weights 1 and 1/2 scale terms exactly.
    float sa = 0.f, ca = 0.f, sb = 0.f, cb = 0.f;
    auto kadd = [](float &s_, float &c_, float t) {
        const float y = t - c_, u = s_ + y;
        c_ = (u - s_) - y;
        s_ = u;
    };
    auto add = [&](int j, float t) {
        const float wa = (na == 0 || j > na) ? 0.f : ((j == 0 || j == na) ? 0.5f : 1.f);
        const float wb = (na == ns || j < na) ? 0.f : ((j == na || j == ns) ? 0.5f : 1.f);
        if (wa != 0.f) kadd(sa, ca, wa * t);
        if (wb != 0.f) kadd(sb, cb, wb * t);
    };
    const int half = ns / 2;
    constexpr int U = DIFF ? 4 : 8;
    for (int m0 = 0; m0 <= (valid ? half : -1); m0 += U) {
        float2 zl[U], zr[U], dl[U], dr[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int m = m0 + u;
            if (m <= half) {
                zl[u] = hz[(size_t)m * n];
                zr[u] = hz[(size_t)(ns - m) * n];
                if (DIFF) {
                    dl[u] = dz[(size_t)m * n];
                    dr[u] = dz[(size_t)(ns - m) * n];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int m = m0 + u;
            if (m > half) break;
            if (!DIFF) {
                add(m, zl[u].x * zr[u].y);
                if (ns - m != m) add(ns - m, zr[u].x * zl[u].y);
            } else {
                // node m: g_m g'_{ns-m}; node ns - m: g_{ns-m} g'_m
                add(m, zl[u].x * dr[u].y + dl[u].x * zr[u].y + dl[u].x * dr[u].y);
                if (ns - m != m) add(ns - m, zr[u].x * dl[u].y + dr[u].x * zl[u].y + dr[u].x * dl[u].y);
            }
        }
    }
    // Q from the partials (after the streaming loop, so that its latency
    // overlaps other blocks' loads; every thread of the block takes part)
    const double *pr = part + (size_t)run * kMaxPart;
    const double sq = sum_partials(pr, nrow_blocks, 1, &bc) / (double)n;
    const double ss = sum_partials(pr + kMaxPart / 2, nprep_blocks, 1, &bc) / (double)n;
    const double qp = DIFF ? q_ref[2 * run] + sq : sq, qs = DIFF ? q_ref[2 * run + 1] + ss : ss;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        q[2 * run] = qp;
        q[2 * run + 1] = qs;
        if (!(qp > 0.0) || !(qs > 0.0) || !isfinite(qp) || !isfinite(qs)) atomicOr(err, 1);
    }
    if (!valid) return;
    const double ia = (double)sa - (double)ca, ib = (double)sb - (double)cb;
    double *ph = phi + (size_t)run * 3 * n;
    if (!DIFF) {
        const double c = g.phi_p * g.ds / qp;
        ph[i] = c * ia;
        ph[n + i] = c * ib;
        ph[2 * n + i] *= (1.0 - g.phi_p) / qs;
    } else {
        const double *pt = phi_ref + (size_t)run * 3 * n;
        const double rq = 1.0 / qp, c = g.phi_p * g.ds;
        ph[i] = pt[i] + (c * ia - pt[i] * sq) * rq;
        ph[n + i] = pt[n + i] + (c * ib - pt[n + i] * sq) * rq;
        ph[2 * n + i] = pt[2 * n + i] + ((1.0 - g.phi_p) * ph[2 * n + i] - pt[2 * n + i] * ss) / qs;
    }
}

// The contour loop of the radix-8 streaming solve for (LX, LY), column tiles
// of CW columns (diff: the differential solve's row passes).
template <int LX, int LY, int CW>
static void stream8_run(Stream8K &k, const Group &G, cudaStream_t s, const SolveProbe *probe, bool diff)
{
    using RT = RowTile<LX>;
    using CT = ColTile<LY, CW>;
    const size_t sr = (size_t)RT::ROWS * RowLayout<LX>::PITCH * sizeof(float2), sc = (size_t)CT::P * sizeof(float2);
    static std::atomic<bool> conf{false};  // attribute set (idempotent if two threads race)
    if (!conf) {
        cudaFuncSetAttribute(prop_row8<LX, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sr);
        cudaFuncSetAttribute(prop_row8<LX, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sr);
        cudaFuncSetAttribute(prop_col8<LY, CW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc);
        conf = true;
    }
    const dim3 gr((unsigned)(G.g.n / RT::P), G.g.nruns), gc(G.g.nx / CT::C, G.g.nruns);
    for (int m = 1; m <= G.g.ns; ++m) {
        const bool pa = probe && m == probe->m_acc, ps = probe && m == probe->m_store;
        if (pa) cudaEventRecordWithFlags(probe->ev[2], s, cudaEventRecordExternal);
        prop_col8<LY, CW><<<gc, CT::T, sc, s>>>(k);
        if (pa) cudaEventRecordWithFlags(probe->ev[3], s, cudaEventRecordExternal);
        if (ps) cudaEventRecordWithFlags(probe->ev[0], s, cudaEventRecordExternal);
        if (diff) prop_row8<LX, true><<<gr, RT::T, sr, s>>>(k, m);
        else prop_row8<LX, false><<<gr, RT::T, sr, s>>>(k, m);
        if (ps) cudaEventRecordWithFlags(probe->ev[1], s, cudaEventRecordExternal);
        if (pa) cudaEventRecordWithFlags(probe->ev[4], s, cudaEventRecordExternal);
    }
}
template <int LX, int LY>
static bool stream8_dispatch_y(int logy, Stream8K &k, const Group &G, cudaStream_t s, const SolveProbe *probe, bool diff)
{
    if constexpr (LY > 11) {
        return false;
    } else {
        if (logy != LY) return stream8_dispatch_y<LX, LY + 1>(logy, k, G, s, probe, diff);
        switch (G.colw_prop) {
        case 4: stream8_run<LX, LY, 4>(k, G, s, probe, diff); break;
        case 8: stream8_run<LX, LY, 8>(k, G, s, probe, diff); break;
        case 16: stream8_run<LX, LY, 16>(k, G, s, probe, diff); break;
        default: stream8_run<LX, LY, ColTile<LY>::C>(k, G, s, probe, diff); break;
        }
        return true;
    }
}
template <int LX>
static bool stream8_dispatch(int logx, int logy, Stream8K &k, const Group &G, cudaStream_t s, const SolveProbe *probe,
                             bool diff = false)
{
    if constexpr (LX > 11) {
        return false;
    } else {
        if (logx != LX) return stream8_dispatch<LX + 1>(logx, logy, k, G, s, probe, diff);
        return stream8_dispatch_y<LX, 6>(logy, k, G, s, probe, diff);
    }
}

static Stream8K stream8_args(const Group &G)
{
    Stream8K k8;
    k8.g = G.g;
    k8.chain = reinterpret_cast<float2 *>(G.chain);
    k8.hist = reinterpret_cast<float2 *>(G.hist);
    k8.hd = reinterpret_cast<float2 *>(G.hd);
    k8.rho = reinterpret_cast<const float2 *>(G.rho);
    k8.efac = reinterpret_cast<const float2 *>(G.efac);
    k8.part = G.part;
    k8.twx = best_mr(G.g.logx) == 4 ? G.tab16x : G.tab8x;
    k8.twy = best_mr(G.g.logy) == 4 ? G.tab16y : G.tab8y;
    k8.twy8 = G.tab8y;
    k8.twy16 = G.tab16y;
    k8.kx = reinterpret_cast<const float *>(G.kx);
    k8.ky = reinterpret_cast<const float *>(G.ky);
    return k8;
}

// Column tile autotuner of the streaming propagator column pass (see
// tune_column_tiles): times prop_col8 at each width on the group's chain
// buffer (scratch until the next solve starts it) and keeps the fastest.
template <int LY>
static float time_col8(int w, Stream8K &k, const Group &G, cudaStream_t s, cudaEvent_t a, cudaEvent_t b)
{
    auto one = [&](auto tag) {
        constexpr int CW = decltype(tag)::value;
        using CT = ColTile<LY, CW>;
        const size_t sc = (size_t)CT::P * sizeof(float2);
        if (sc > 227 * 1024 ||
            cudaFuncSetAttribute(prop_col8<LY, CW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc) != cudaSuccess) {
            cudaGetLastError();  // this width does not fit: not a candidate
            return 1e30f;
        }
        const dim3 gc(G.g.nx / CT::C, G.g.nruns);
        float best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(a, s);
            prop_col8<LY, CW><<<gc, CT::T, sc, s>>>(k);
            cudaEventRecord(b, s);
            cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (rep > 0 && ms < best) best = ms;
        }
        return cudaGetLastError() == cudaSuccess ? best : 1e30f;
    };
    switch (w) {
    case 4: return one(std::integral_constant<int, 4>{});
    case 8: return one(std::integral_constant<int, 8>{});
    default: return one(std::integral_constant<int, 16>{});
    }
}
template <int LY>
static int tune_col8_at(int logy, Stream8K &k, const Group &G, cudaStream_t s)
{
    if constexpr (LY > 11) {
        return 0;
    } else {
        if (logy != LY) return tune_col8_at<LY + 1>(logy, k, G, s);
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return 0;
        float best = 1e30f;
        int best_w = 0;
        for (int w : kColWidths) {
            if (G.g.nx % w) continue;
            const float t = time_col8<LY>(w, k, G, s, a, b);
            if (t < best) {
                best = t;
                best_w = w;
            }
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return best_w;
    }
}

cudaError_t tune_stream_tiles(Group &G, cudaStream_t s)
{
    if (!(G.prec == EPD_LB_MIXED_FP32 && G.hist_full && G.tab8x)) return cudaSuccess;
    if (const char *env = std::getenv("EPD_LB_COLUMN_TILE")) {
        const int w = std::atoi(env);
        if (w == 4 || w == 8 || w == 16) {
            G.colw_prop = w;
            return cudaSuccess;
        }
    }
    Stream8K k8 = stream8_args(G);
    cudaError_t e = cudaMemsetAsync(G.chain, 0, (size_t)G.g.nruns * G.g.n * sizeof(float2), s);
    if (e != cudaSuccess) return e;
    G.colw_prop = tune_col8_at<6>(G.g.logy, k8, G, s);
    return cudaGetLastError();
}

bool stream8_eligible(int prec, int logx, int logy)
{
    return prec == EPD_LB_MIXED_FP32 && !cluster_shape_exists(logx, logy) && logx >= 6 && logy >= 6 && logx <= 11 &&
           logy <= 11 && logx + logy >= 11;
}

static int grid_for(long long n)
{
    long long b = (n + kThreads - 1) / kThreads;
    if (b > 1024) b = 1024;
    return (int)b;
}

template <typename T>
static size_t col_smem(const Group &G)
{
    return (size_t)2 * (G.g.ny * G.sh.cols_prop) * sizeof(V2<T>) + (G.g.pow2 ? G.g.ny / 2 : G.g.ny) * sizeof(V2<T>) +
           G.g.ny * sizeof(T);
}
template <typename T>
static size_t row_smem(const Group &G)
{
    return (size_t)2 * (G.sh.rows_prop * G.g.nx) * sizeof(V2<T>) + (G.g.pow2 ? G.g.nx / 2 : G.g.nx) * sizeof(V2<T>) +
           G.g.nx * sizeof(T);
}

template <typename T>
static PropK<T> prop_args(const Group &G)
{
    PropK<T> k;
    k.g = G.g;
    k.chain = reinterpret_cast<V2<T> *>(G.chain);
    k.hist = reinterpret_cast<V2<T> *>(G.hist);
    k.hd = reinterpret_cast<V2<T> *>(G.hd);
    k.rho = reinterpret_cast<const float2 *>(G.rho);
    k.hnodes = G.hnodes;
    k.efac = reinterpret_cast<const V2<T> *>(G.efac);
    k.ia = G.ia;
    k.ib = G.ib;
    k.part = G.part;
    k.twx = reinterpret_cast<const V2<T> *>(G.twx);
    k.twy = reinterpret_cast<const V2<T> *>(G.twy);
    k.kx = reinterpret_cast<const T *>(G.kx);
    k.ky = reinterpret_cast<const T *>(G.ky);
    k.rows = G.sh.rows_prop;
    k.logc = G.g.pow2 ? ilog2(G.sh.cols_prop) : 0;
    k.cols = G.sh.cols_prop;
    return k;
}

// Q partial blocks of the radix-8 row pass (one per row tile)
static int stream8_row_blocks(const GroupGeom &g) { return (int)(g.n / (g.nx >= 2048 ? g.nx : 2048)); }

// The contour loop of the generic streaming solve (column pass, row pass per
// node); returns the row pass grid (its x extent = the Q partial blocks).
template <typename T, bool DIFF>
static dim3 generic_loop(const Group &G, PropK<T> &k, cudaStream_t s, const SolveProbe *probe)
{
    const GroupGeom &g = G.g;
    const dim3 gc(g.nx / G.sh.cols_prop, g.nruns), gr(g.ny / G.sh.rows_prop, g.nruns);
    const size_t sc = col_smem<T>(G), sr = row_smem<T>(G);
    for (int m = 1; m <= g.ns; ++m) {
        const bool pa = probe && m == probe->m_acc, ps = probe && m == probe->m_store;
        if (pa) cudaEventRecordWithFlags(probe->ev[2], s, cudaEventRecordExternal);
        prop_col<T><<<gc, kThreads, sc, s>>>(k);
        if (pa) cudaEventRecordWithFlags(probe->ev[3], s, cudaEventRecordExternal);
        if (ps) cudaEventRecordWithFlags(probe->ev[0], s, cudaEventRecordExternal);
        prop_row<T, DIFF><<<gr, kThreads, sr, s>>>(k, m);
        if (ps) cudaEventRecordWithFlags(probe->ev[1], s, cudaEventRecordExternal);
        if (pa) cudaEventRecordWithFlags(probe->ev[4], s, cudaEventRecordExternal);
    }
    return gr;
}

template <typename T>
static cudaError_t solve_t(Group &G, const double *omega, double *phi, double *q, cudaStream_t s, const SolveProbe *probe)
{
    const GroupGeom &g = G.g;
    PropK<T> k = prop_args<T>(G);

    const int pg = grid_for(g.n);
    prop_prep<T><<<dim3(pg, g.nruns), kThreads, 0, s>>>(g, omega, reinterpret_cast<V2<T> *>(G.efac), phi, G.part);
    if (sizeof(T) == sizeof(float) && G.hc && G.twx_full && cluster_solve_supported(G)) {
        // whole contour in one cluster-resident launch, then the contour sums
        return launch_cluster_solve(G, s, false, pg, phi, q, probe);
    }
    if (sizeof(T) == sizeof(float) && G.hist_full && G.tab8x) {
        // radix-8 streaming passes with the full history, then the contour pass
        Stream8K k8 = stream8_args(G);
        prop_start8<false><<<dim3(pg, g.nruns), kThreads, 0, s>>>(k8);
        if (!stream8_dispatch<6>(g.logx, g.logy, k8, G, s, probe)) return cudaErrorInvalidConfiguration;
        prop_contour_stream<false><<<dim3((unsigned)((g.n + kThreads - 1) / kThreads), g.nruns), kThreads, 0, s>>>(
            g, k8.hist, nullptr, stream8_row_blocks(g), pg, G.part, phi, q, nullptr, nullptr, G.err);
        return cudaGetLastError();
    }
    prop_start<T, false><<<dim3(pg, g.nruns), kThreads, 0, s>>>(k);
    const dim3 gr = generic_loop<T, false>(G, k, s, probe);
    prop_finalize<<<dim3(pg, g.nruns), kThreads, 0, s>>>(g, gr.x, pg, G.ia, G.ib, nullptr, nullptr, G.part, phi, q, G.err);
    return cudaGetLastError();
}

// Streaming differential solve (MIXED_FP32 grids without the cluster
// solve): the changes against the reference history of the last plain
// solve, then the contour pass of the changes.
static cudaError_t stream_delta(Group &G, int pg, double *phi, double *q, const double *phi_ref, const double *q_ref,
                                cudaStream_t s, const SolveProbe *probe)
{
    const GroupGeom &g = G.g;
    const dim3 gcon((unsigned)((g.n + kThreads - 1) / kThreads), g.nruns);
    if (G.hist_full && G.tab8x) {
        Stream8K k8 = stream8_args(G);
        prop_start8<true><<<dim3(pg, g.nruns), kThreads, 0, s>>>(k8);
        if (!stream8_dispatch<6>(g.logx, g.logy, k8, G, s, probe, true)) return cudaErrorInvalidConfiguration;
        prop_contour_stream<true><<<gcon, kThreads, 0, s>>>(g, k8.hist, k8.hd, stream8_row_blocks(g), pg, G.part, phi, q,
                                                           phi_ref, q_ref, G.err);
        return cudaGetLastError();
    }
    PropK<float> k = prop_args<float>(G);
    prop_start<float, true><<<dim3(pg, g.nruns), kThreads, 0, s>>>(k);
    const dim3 gr = generic_loop<float, true>(G, k, s, probe);
    prop_contour_stream<true><<<gcon, kThreads, 0, s>>>(g, reinterpret_cast<const float2 *>(G.hist),
                                                       reinterpret_cast<const float2 *>(G.hd), (int)gr.x, pg, G.part, phi,
                                                       q, phi_ref, q_ref, G.err);
    return cudaGetLastError();
}

cudaError_t launch_solve(Group &G, const double *omega, double *phi, double *q, cudaStream_t s, const SolveProbe *probe)
{
    if (G.prec == EPD_LB_MIXED_FP32) return solve_t<float>(G, omega, phi, q, s, probe);
    return solve_t<double>(G, omega, phi, q, s, probe);
}

cudaError_t launch_solve_delta_at(Group &G, const double *omega, const double *omega_ref, const double *phi_ref,
                                  const double *q_ref, double *phi, double *q, cudaStream_t s, const SolveProbe *probe)
{
    if (!G.diff || !G.hd) return cudaErrorInvalidValue;
    const GroupGeom &g = G.g;
    const int pg = grid_for(g.n);
    prop_prep_delta<<<dim3(pg, g.nruns), kThreads, 0, s>>>(g, omega, omega_ref, reinterpret_cast<float2 *>(G.rho),
                                                          reinterpret_cast<float *>(G.cdiff), phi, G.part);
    if (!G.hc) return stream_delta(G, pg, phi, q, phi_ref, q_ref, s, probe);
    return launch_cluster_solve(G, s, true, pg, phi, q, probe, phi_ref, q_ref);
}

cudaError_t launch_solve_delta(Group &G, cudaStream_t s, const SolveProbe *probe)
{
    return launch_solve_delta_at(G, G.omega, G.omega_t, G.phi_t, G.q_t, G.phi, G.q, s, probe);
}

// Single-chain solve on a 3D box: per contour step the z-column, y-column and
// x-row passes (the Fourier factor exp(-R_G^2 |k|^2 ds) is the product of the
// three axes' factors, each applied inside its own axis transform), the row
// pass carrying the node factors, history and contour sums as in 2D.
template <typename T>
static size_t smem3(const GroupGeom &g, int rows, int cols, bool row)
{
    if (row) return (size_t)2 * rows * g.nx * sizeof(V2<T>) + (g.pow2 ? g.nx / 2 : g.nx) * sizeof(V2<T>) + g.nx * sizeof(T);
    return (size_t)2 * g.ny * cols * sizeof(V2<T>) + (g.pow2 ? g.ny / 2 : g.ny) * sizeof(V2<T>) + g.ny * sizeof(T);
}

size_t solve3d_smem_max(const Solve3 &S)
{
    auto mx = [&](auto t) {
        using T = decltype(t);
        return std::max(smem3<T>(S.vx, S.rows_x, 0, true), std::max(smem3<T>(S.vy, 0, S.cols_y, false), smem3<T>(S.vz, 0, S.cols_z, false)));
    };
    return S.prec == EPD_LB_MIXED_FP32 ? mx(0.f) : mx(0.0);
}

template <typename T>
static cudaError_t solve3d_t(const Solve3 &S, const double *omega, double *phi, double *q, cudaStream_t s)
{
    auto view = [&](const GroupGeom &g, const void *tw_row, const void *tw_col, const void *k_row, const void *k_col,
                    int rows, int cols) {
        PropK<T> k;
        k.g = g;
        k.chain = reinterpret_cast<V2<T> *>(S.chain);
        k.hist = reinterpret_cast<V2<T> *>(S.hist);
        k.hd = nullptr;
        k.rho = nullptr;
        k.hnodes = g.half_lo + 1;
        k.efac = reinterpret_cast<const V2<T> *>(S.efac);
        k.ia = S.ia;
        k.ib = S.ib;
        k.part = S.part;
        k.twx = reinterpret_cast<const V2<T> *>(tw_row);
        k.twy = reinterpret_cast<const V2<T> *>(tw_col);
        k.kx = reinterpret_cast<const T *>(k_row);
        k.ky = reinterpret_cast<const T *>(k_col);
        k.rows = rows;
        k.cols = cols;
        k.logc = g.pow2 ? ilog2(cols) : 0;
        return k;
    };
    const PropK<T> kx = view(S.vx, S.twx, S.twy, S.kx, S.ky, S.rows_x, 1);
    const PropK<T> ky = view(S.vy, S.twx, S.twy, S.kx, S.ky, 1, S.cols_y);
    const PropK<T> kz = view(S.vz, S.twx, S.twz, S.kx, S.kz, 1, S.cols_z);
    const GroupGeom &g = S.vx;
    const int pg = grid_for(g.n);
    prop_prep<T><<<dim3(pg, 1), kThreads, 0, s>>>(g, omega, reinterpret_cast<V2<T> *>(S.efac), phi, S.part);
    prop_start<T, false><<<dim3(pg, 1), kThreads, 0, s>>>(kx);
    const dim3 gz(S.vz.nx / S.cols_z, 1), gy(S.vy.nx / S.cols_y, S.vy.nruns), gr(S.vx.ny / S.rows_x, 1);
    const size_t sz = smem3<T>(S.vz, 0, S.cols_z, false), sy = smem3<T>(S.vy, 0, S.cols_y, false),
                 sr = smem3<T>(S.vx, S.rows_x, 0, true);
    for (int m = 1; m <= g.ns; ++m) {
        prop_col<T><<<gz, kThreads, sz, s>>>(kz);
        prop_col<T><<<gy, kThreads, sy, s>>>(ky);
        prop_row<T, false><<<gr, kThreads, sr, s>>>(kx, m);
    }
    prop_finalize<<<dim3(pg, 1), kThreads, 0, s>>>(g, gr.x, pg, S.ia, S.ib, nullptr, nullptr, S.part, phi, q, S.err);
    return cudaGetLastError();
}

cudaError_t launch_solve3d(const Solve3 &S, const double *omega, double *phi, double *q, cudaStream_t s)
{
    return S.prec == EPD_LB_MIXED_FP32 ? solve3d_t<float>(S, omega, phi, q, s) : solve3d_t<double>(S, omega, phi, q, s);
}

cudaError_t configure_prop_kernels()
{
    cudaError_t e = cudaSuccess;
    const int lim = 200 * 1024;
    e = cudaFuncSetAttribute(prop_col<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e) return e;
    e = cudaFuncSetAttribute(prop_row<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e) return e;
    e = cudaFuncSetAttribute(prop_row<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e) return e;
    e = cudaFuncSetAttribute(prop_col<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e) return e;
    return cudaFuncSetAttribute(prop_row<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

} // namespace epdlb

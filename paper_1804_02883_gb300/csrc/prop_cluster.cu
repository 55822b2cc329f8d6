// prop_cluster.cu -- cluster-resident single-chain solve (Sec. 2, Eqs. (6)-(10)
// of arXiv:1804.02883) for grids whose propagator field fits in the shared
// memory of one thread-block cluster (FP32 bulk precision).
//
// One cluster of C CTAs carries one chain of one run: the forward propagator
// g (Eq. (6)) or the backward propagator g' (Eq. (7)), so a launch holds
// 2 x runs clusters.  The real field of the chain lives on chip in two
// packings: CTA c owns complex rows [c R2, (c+1) R2), each holding the real
// rows (2k, 2k+1) as (re, im), in its row buffer, and complex columns
// [c W2, (c+1) W2), each holding the real columns (2j, 2j+1), in its column
// buffer.  The Fourier factor of Eq. (8) is real, even and separable, so it
// acts on each packed row / column as on two real ones.  One contour step:
//   gather rows -> my columns (distributed shared memory, 2 x 2 re/im
//   transposes), column transform Ky, cluster barrier, gather columns -> my
//   rows, row transform Kx, node factor, history or contour sums.
// Two cluster barriers per contour step.
//
// The contour sums of Eqs. (9)-(10) need g and g' at mirrored nodes.  A solve
// is two launches: the first runs nodes 1..N_s/2 of both chains and stores
// them (history) plus the chain state; the second runs nodes N_s/2+1..N_s,
// where the g cluster adds g(s_m) g'(1 - s_m) (node m) and the g' cluster
// adds g(s_{N_s-m}) g'(s_m) (node N_s - m), reading the other chain's
// first-half history; node N_s/2 itself is added by the g cluster from the
// two histories.  Products and partial sums over up to 8 nodes with equal
// trapezoid weights in FP32 registers, added into per-chain FP64 sums.
//
// Transforms: register-resident radix-8 (one radix-2/4 pass where log2 N is
// not a multiple of 3) Stockham passes in shared memory, in place.  The
// forward transform's last pass, the multiplication by the Fourier factor
// and the inverse transform's first pass are fused (same points per
// thread); the inverse's last pass hands its points to the per-site
// epilogue.  Twiddles come from per-pass tables laid out [k][p] so that
// consecutive threads read consecutive entries.
#include <cooperative_groups.h>

#include "common.cuh"
#include "engine.h"

namespace cg = cooperative_groups;

namespace epdlb {

// Solve modes of the cluster kernel.
//  0: plain solve; first-half history in `hist`.
//  1: reference solve: every node of both chains kept in `hist1` (for a
//     following differential solve), mirrored products read from it.
//  2: differential solve at omega + d omega given the reference solve at
//     omega: the chain carries d a_j = E_j dg_j + dE_j (g_j + dg_j), the
//     epilogue forms dg_{j+1} = E_{j+1} T(d a_j) + dE_{j+1} (g_{j+1}/E_{j+1} + T(d a_j))
//     (g, E of the reference solve; dE the change of the node factors), and
//     the contour sums collect g dg' + dg g' + dg dg' (exact algebra of the
//     two solves' difference, rounded relative to the difference itself).
struct PropCK {
    GroupGeom g;
    float *hist;         // [run][chain][half_lo + 1][n] real (modes 0 and 2)
    float *hist1;        // [run][chain][N_s + 1][n] real (reference solve, modes 1 and 2)
    const float2 *defac; // (dE_A, dE_B) [run][n] (mode 2)
    int mode;
    float2 *state;       // [run][chain][n / 2] packed rows, E z at node half_lo
    const float2 *efac;  // [run][n] (E_A, E_B)
    double *ia0, *ib0;   // contour sums of the g chain's terms, [run][n]
    double *ia1, *ib1;   // contour sums of the g' chain's terms, [run][n]
    double *part;
    const float2 *twx, *twy;  // exp(-2 pi i j / N), j < N
    const float *kx, *ky;     // exp(-R_G^2 k^2 ds) / N
    int half;                 // 0: nodes 1..half_lo; 1: nodes half_lo..N_s
};

// Radix plan: passes of radix 8, the last forward pass takes the remainder.
__host__ __device__ constexpr int npasses(int logn) { return (logn + 2) / 3; }
__host__ __device__ constexpr int fwd_rlog(int logn, int i) { return i < npasses(logn) - 1 ? 3 : logn - 3 * (npasses(logn) - 1); }
__host__ __device__ constexpr int fwd_slog(int logn, int i) { return i == 0 ? 0 : fwd_slog(logn, i - 1) + fwd_rlog(logn, i - 1); }
__host__ __device__ constexpr int inv_rlog(int logn, int i) { return fwd_rlog(logn, npasses(logn) - 1 - i); }
__host__ __device__ constexpr int inv_slog(int logn, int i) { return i == 0 ? 0 : inv_slog(logn, i - 1) + inv_rlog(logn, i - 1); }
// Twiddle tables: one per pass that needs twiddles (forward passes
// 0..np-2, inverse passes 0..np-2), (R-1) x M entries, M = N / (S R).
__host__ __device__ constexpr int tab_len(int logn, int slog, int rlog) { return ((1 << rlog) - 1) * ((1 << logn) >> (slog + rlog)); }
__host__ __device__ constexpr int fwd_off(int logn, int i) { return i == 0 ? 0 : fwd_off(logn, i - 1) + tab_len(logn, fwd_slog(logn, i - 1), fwd_rlog(logn, i - 1)); }
__host__ __device__ constexpr int inv_off(int logn, int i)
{
    return i == 0 ? fwd_off(logn, npasses(logn) - 1) : inv_off(logn, i - 1) + tab_len(logn, inv_slog(logn, i - 1), inv_rlog(logn, i - 1));
}
__host__ __device__ constexpr int tabs_total(int logn) { return inv_off(logn, npasses(logn) - 1); }

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 fadd(float2 a, float2 b) { return f2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 fsub(float2 a, float2 b) { return f2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 fmul(float2 a, float2 b) { return f2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 fmulc(float2 a, float2 b) { return f2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }  // a * conj(b)
template <bool INV> __device__ __forceinline__ float2 rot90(float2 a) { return INV ? f2(-a.y, a.x) : f2(a.y, -a.x); }

// In-register DFT of length 2^RLOG, natural order in and out; forward uses
// exp(-2 pi i / R), inverse exp(+2 pi i / R).
template <int RLOG, bool INV> struct Dft;
template <bool INV> struct Dft<1, INV> {
    static __device__ __forceinline__ void run(float2 *x)
    {
        const float2 a = x[0], b = x[1];
        x[0] = fadd(a, b);
        x[1] = fsub(a, b);
    }
};
template <bool INV> struct Dft<2, INV> {
    static __device__ __forceinline__ void run(float2 *x)
    {
        const float2 s02 = fadd(x[0], x[2]), d02 = fsub(x[0], x[2]);
        const float2 s13 = fadd(x[1], x[3]), d13 = rot90<INV>(fsub(x[1], x[3]));
        x[0] = fadd(s02, s13);
        x[2] = fsub(s02, s13);
        x[1] = fadd(d02, d13);
        x[3] = fsub(d02, d13);
    }
};
template <bool INV> struct Dft<3, INV> {
    static __device__ __forceinline__ void run(float2 *x)
    {
        float2 e[4] = {x[0], x[2], x[4], x[6]};
        float2 o[4] = {x[1], x[3], x[5], x[7]};
        Dft<2, INV>::run(e);
        Dft<2, INV>::run(o);
        const float h = 0.70710678118654752440f;
        const float2 o1 = INV ? f2(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y)) : f2(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
        const float2 o2 = rot90<INV>(o[2]);
        const float2 o3 = INV ? f2(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y)) : f2(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
        x[0] = fadd(e[0], o[0]);
        x[4] = fsub(e[0], o[0]);
        x[1] = fadd(e[1], o1);
        x[5] = fsub(e[1], o1);
        x[2] = fadd(e[2], o2);
        x[6] = fsub(e[2], o2);
        x[3] = fadd(e[3], o3);
        x[7] = fsub(e[3], o3);
    }
};

// Shared-memory layouts.  Row layout: sequence b (a packed row), point x,
// padded by one slot per 8 points against bank conflicts.  Column layout:
// point y of sequence c (a packed column) at y * W + c.
template <int LOGN> struct RowLayout {
    static constexpr int N = 1 << LOGN, PITCH = N + N / 8;
    static __device__ __forceinline__ int at(int b, int x) { return b * PITCH + x + (x >> 3); }
    template <int PER> static __device__ __forceinline__ void split(int bf, int &b, int &t) { b = bf / PER; t = bf % PER; }
};
template <int LOGN, int W> struct ColLayout {
    static __device__ __forceinline__ int at(int c, int y) { return y * W + c; }
    template <int PER> static __device__ __forceinline__ void split(int bf, int &b, int &t) { b = bf % W; t = bf / W; }
};

// One in-place Stockham pass (radix 2^RLOG, stride 2^SLOG): load, wait, write.
// tab: this pass's twiddles [k-1][p] (unused in a forward last pass).
template <int LOGN, int SLOG, int RLOG, bool INV, int NB, int T, class L>
__device__ __forceinline__ void pass(float2 *buf, const float2 *tab, int tid)
{
    constexpr int N = 1 << LOGN, R = 1 << RLOG, S = 1 << SLOG, PER = N / R, M = N / (S * R);
    float2 x[NB][R];
    int bb[NB], tt[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        L::template split<PER>(tid + j * T, bb[j], tt[j]);
#pragma unroll
        for (int r = 0; r < R; ++r) x[j][r] = buf[L::at(bb[j], tt[j] + r * PER)];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        Dft<RLOG, INV>::run(x[j]);
        const int q = tt[j] & (S - 1), p = tt[j] >> SLOG;
        if (M > 1) {
#pragma unroll
            for (int k = 1; k < R; ++k) {
                const float2 w = tab[(k - 1) * M + p];
                x[j][k] = INV ? fmulc(x[j][k], w) : fmul(x[j][k], w);
            }
        }
#pragma unroll
        for (int k = 0; k < R; ++k) buf[L::at(bb[j], q + R * S * p + S * k)] = x[j][k];
    }
    __syncthreads();
}

// Forward last pass, Fourier factor, inverse first pass (same points per thread).
template <int LOGN, int RLOG, int NB, int T, class L>
__device__ __forceinline__ void middle(float2 *buf, const float2 *tab_inv0, const float *kf, int tid)
{
    constexpr int N = 1 << LOGN, R = 1 << RLOG, PER = N / R;
    float2 x[NB][R];
    int bb[NB], tt[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        L::template split<PER>(tid + j * T, bb[j], tt[j]);
#pragma unroll
        for (int r = 0; r < R; ++r) x[j][r] = buf[L::at(bb[j], tt[j] + r * PER)];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        Dft<RLOG, false>::run(x[j]);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const float f = kf[tt[j] + k * PER];
            x[j][k].x *= f;
            x[j][k].y *= f;
        }
        Dft<RLOG, true>::run(x[j]);
#pragma unroll
        for (int k = 1; k < R; ++k) x[j][k] = fmulc(x[j][k], tab_inv0[(k - 1) * PER + tt[j]]);
#pragma unroll
        for (int k = 0; k < R; ++k) buf[L::at(bb[j], R * tt[j] + k)] = x[j][k];
    }
    __syncthreads();
}

template <int LOGN, int I, int T, class L, int P>
struct FwdPasses {
    static __device__ __forceinline__ void run(float2 *buf, const float2 *tabs, int tid)
    {
        if constexpr (I < npasses(LOGN) - 1) {
            constexpr int RLOG = fwd_rlog(LOGN, I);
            pass<LOGN, fwd_slog(LOGN, I), RLOG, false, P / (1 << RLOG) / T, T, L>(buf, tabs + fwd_off(LOGN, I), tid);
            FwdPasses<LOGN, I + 1, T, L, P>::run(buf, tabs, tid);
        }
    }
};
template <int LOGN, int I, int T, class L, int P>
struct InvPasses {
    static __device__ __forceinline__ void run(float2 *buf, const float2 *tabs, int tid)
    {
        if constexpr (I < npasses(LOGN) - 1) {
            constexpr int RLOG = inv_rlog(LOGN, I);
            pass<LOGN, inv_slog(LOGN, I), RLOG, true, P / (1 << RLOG) / T, T, L>(buf, tabs + inv_off(LOGN, I), tid);
            InvPasses<LOGN, I + 1, T, L, P>::run(buf, tabs, tid);
        }
    }
};

// Full transform pair (forward, Fourier factor, inverse) up to the inverse's
// last pass, whose loads and DFT are left to the caller.
template <int LOGN, int T, class L, int P>
__device__ __forceinline__ void transform_pair(float2 *buf, const float2 *tabs, const float *kf, int tid)
{
    FwdPasses<LOGN, 0, T, L, P>::run(buf, tabs, tid);
    constexpr int RM = fwd_rlog(LOGN, npasses(LOGN) - 1);
    middle<LOGN, RM, P / (1 << RM) / T, T, L>(buf, tabs + inv_off(LOGN, 0), kf, tid);
    InvPasses<LOGN, 1, T, L, P>::run(buf, tabs, tid);
}

template <int LOGN, int NB, int T, class L>
__device__ __forceinline__ void last_inverse(const float2 *buf, float2 (&x)[NB][1 << inv_rlog(LOGN, npasses(LOGN) - 1)],
                                             int (&bb)[NB], int (&tt)[NB], int tid)
{
    constexpr int RLOG = inv_rlog(LOGN, npasses(LOGN) - 1), R = 1 << RLOG, PER = (1 << LOGN) / R;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        L::template split<PER>(tid + j * T, bb[j], tt[j]);
#pragma unroll
        for (int r = 0; r < R; ++r) x[j][r] = buf[L::at(bb[j], tt[j] + r * PER)];
        Dft<RLOG, true>::run(x[j]);
    }
}

// Fill the twiddle tables of every pass of a length-2^LOGN transform.
template <int LOGN, int I>
__device__ __forceinline__ void fill_tables(float2 *tabs, const float2 *tw, int tid, int nthreads)
{
    constexpr int NP = npasses(LOGN);
    if constexpr (I < 2 * (NP - 1)) {
        constexpr bool INVP = I >= NP - 1;
        constexpr int PI = INVP ? I - (NP - 1) : I;
        constexpr int SLOG = INVP ? inv_slog(LOGN, PI) : fwd_slog(LOGN, PI);
        constexpr int RLOG = INVP ? inv_rlog(LOGN, PI) : fwd_rlog(LOGN, PI);
        constexpr int OFF = INVP ? inv_off(LOGN, PI) : fwd_off(LOGN, PI);
        constexpr int M = (1 << LOGN) >> (SLOG + RLOG), LEN = ((1 << RLOG) - 1) * M;
        for (int e = tid; e < LEN; e += nthreads) {
            const int k = e / M + 1, p = e % M;
            tabs[OFF + e] = tw[(p << SLOG) * k];
        }
        fill_tables<LOGN, I + 1>(tabs, tw, tid, nthreads);
    }
}

__device__ __forceinline__ float wclass_a(int j, int na)
{
    if (na == 0 || j > na) return 0.f;
    return (j == 0 || j == na) ? 0.5f : 1.f;
}
__device__ __forceinline__ float wclass_b(int j, int na, int ns)
{
    if (na == ns || j < na) return 0.f;
    return (j == na || j == ns) ? 0.5f : 1.f;
}

template <int LOGX, int LOGY, int C, int T>
struct ClusterGeom {
    static constexpr int NX = 1 << LOGX, NY = 1 << LOGY, R2 = NY / 2 / C, W2 = NX / 2 / C;
    static constexpr int P = R2 * NX;  // complex points per CTA in either packing
    static constexpr int PITCH = NX + NX / 8;
    static constexpr int TABX = tabs_total(LOGX), TABY = tabs_total(LOGY);
    // shared memory: row buffer, column buffer, twiddle tables, Fourier
    // factors (at most ~110 KB, so that two CTAs fit on one SM and a launch's
    // 16-CTA clusters are co-resident)
    static constexpr size_t SMEM = (size_t)(R2 * PITCH + P + TABX + TABY) * sizeof(float2) + (NX + NY) * sizeof(float);
};

template <int LOGX, int LOGY, int C, int T, bool DIFF>
__global__ void __launch_bounds__(T, 1024 / T) prop_cluster(PropCK k)
{
    using G = ClusterGeom<LOGX, LOGY, C, T>;
    constexpr int NX = G::NX, NY = G::NY, R2 = G::R2, W2 = G::W2, P = G::P;
    static_assert(P == W2 * NY, "layout sizes");
    static_assert(P % (8 * T) == 0, "every pass gives each thread whole butterflies");
    static_assert(LOGX >= 4 && LOGY >= 4 && R2 >= 1 && W2 >= 1, "tile shape");
    using RL = RowLayout<LOGX>;
    using CL = ColLayout<LOGY, W2>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *rowbuf = reinterpret_cast<float2 *>(smem_raw);
    float2 *colbuf = rowbuf + R2 * G::PITCH;
    float2 *tabx = colbuf + P;
    float2 *taby = tabx + G::TABX;
    float *kx = reinterpret_cast<float *>(taby + G::TABY);
    float *ky = kx + NX;
    __shared__ double red[32];

    cg::cluster_group cl = cg::this_cluster();
    const int crank = (int)cl.block_rank();
    const int cidx = blockIdx.x / C, run = cidx >> 1, chain = cidx & 1;
    const int tid = threadIdx.x;
    const long long n = k.g.n;
    const int ns = k.g.ns, na = k.g.na, hlo = k.g.half_lo, hhi = k.g.half_hi;
    const int krow0 = crank * R2;  // first packed row of this CTA

    fill_tables<LOGX, 0>(tabx, k.twx, tid, T);
    fill_tables<LOGY, 0>(taby, k.twy, tid, T);
    for (int i = tid; i < NX; i += T) kx[i] = k.kx[i];
    for (int i = tid; i < NY; i += T) ky[i] = k.ky[i];
    const float2 *efac = k.efac + (size_t)run * n;
    const float2 *defac = DIFF ? k.defac + (size_t)run * n : nullptr;
    const int mode = DIFF ? 2 : k.mode;
    const int hp = mode == 1 ? ns + 1 : hlo + 1;  // history pitch in nodes
    float *hbase = mode == 1 ? k.hist1 : k.hist;
    float *hist_me = hbase + (size_t)(run * 2 + chain) * hp * n;
    const float *hist_other = hbase + (size_t)(run * 2 + (1 - chain)) * hp * n;
    // reference solve's chains (mode 2)
    const float *ref_me = DIFF ? k.hist1 + (size_t)(run * 2 + chain) * (ns + 1) * n : nullptr;
    const float *ref_other = DIFF ? k.hist1 + (size_t)(run * 2 + (1 - chain)) * (ns + 1) * n : nullptr;
    float2 *state = k.state + (size_t)(run * 2 + chain) * (n / 2);
    __syncthreads();

    // node factor of this chain at contour node j: g carries w_A iff j < N_A,
    // g' sees the field of node N_s - j
    auto sel = [&](float2 e, int j) { return ((chain == 0 ? j : ns - j) < na) ? e.x : e.y; };

    int m0, m1;
    if (k.half == 0) {
        for (int e = tid; e < P; e += T) {
            const int b = e / NX, x = e % NX;
            const long long site = (long long)(2 * (krow0 + b)) * NX + x;
            if (DIFF) {  // dg_0 = 0, d a_0 = dE_0 g_0
                hist_me[site] = 0.f;
                hist_me[site + NX] = 0.f;
                rowbuf[RL::at(b, x)] = f2(sel(defac[site], 0), sel(defac[site + NX], 0));
            } else {
                hist_me[site] = 1.f;
                hist_me[site + NX] = 1.f;
                rowbuf[RL::at(b, x)] = f2(sel(efac[site], 0), sel(efac[site + NX], 0));
            }
        }
        m0 = 1;
        m1 = hlo;
    } else {
        for (int e = tid; e < P; e += T) {
            const int b = e / NX, x = e % NX;
            rowbuf[RL::at(b, x)] = state[(size_t)(krow0 + b) * NX + x];
        }
        m0 = hlo + 1;
        m1 = ns;
    }

    // epilogue geometry: the inverse row transform's last pass
    constexpr int RLOG_L = inv_rlog(LOGX, npasses(LOGX) - 1), RR = 1 << RLOG_L, PER_L = NX / RR;
    constexpr int NB_L = P / RR / T;
    // one FP32 partial sum per real site over a group of at most 8 nodes that
    // share the trapezoid weights (w_A, w_B); a group is added to the FP64
    // sums with its weights when it is full or the weights change
    float acc[NB_L][RR][2];
#pragma unroll
    for (int j = 0; j < NB_L; ++j)
#pragma unroll
        for (int r = 0; r < RR; ++r) acc[j][r][0] = acc[j][r][1] = 0.f;
    int nacc = 0;
    float gwa = 0.f, gwb = 0.f;
    float qsum = 0.f;
    double *ia = chain == 0 ? k.ia0 : k.ia1, *ib = chain == 0 ? k.ib0 : k.ib1;
    ia += (size_t)run * n;
    ib += (size_t)run * n;

    auto flush = [&](int bb_j, int tt_j, int j) {
        const double ca = k.g.ds * (double)gwa, cb = k.g.ds * (double)gwb;
#pragma unroll
        for (int r = 0; r < RR; ++r)
#pragma unroll
            for (int cp = 0; cp < 2; ++cp) {
                const long long site = (long long)(2 * (krow0 + bb_j) + cp) * NX + tt_j + r * PER_L;
                const double v = (double)acc[j][r][cp];
                if (gwa != 0.f) ia[site] += ca * v;
                if (gwb != 0.f) ib[site] += cb * v;
                acc[j][r][cp] = 0.f;
            }
    };

    if (k.half == 1) {
        // this chain's FP64 sums start at zero
        for (int e = tid; e < P; e += T) {
            const int b = e / NX, x = e % NX;
            const long long site = (long long)(2 * (krow0 + b)) * NX + x;
            ia[site] = 0.0;
            ib[site] = 0.0;
            ia[site + NX] = 0.0;
            ib[site + NX] = 0.0;
        }
        __syncthreads();
    }

    // node N_s/2 (even N_s): both chains are in the histories; the g cluster adds it
    if (k.half == 1 && chain == 0 && hhi == hlo) {
        gwa = wclass_a(hlo, na);
        gwb = wclass_b(hlo, na, ns);
#pragma unroll
        for (int j = 0; j < NB_L; ++j) {
            int b, t;
            RL::template split<PER_L>(tid + j * T, b, t);
#pragma unroll
            for (int r = 0; r < RR; ++r)
#pragma unroll
                for (int cp = 0; cp < 2; ++cp) {
                    const long long site = (long long)(2 * (krow0 + b) + cp) * NX + t + r * PER_L;
                    const float a = hist_me[(size_t)hlo * n + site], o = hist_other[(size_t)hlo * n + site];
                    if (DIFF) {
                        const float ga = ref_me[(size_t)hlo * n + site], go = ref_other[(size_t)hlo * n + site];
                        acc[j][r][cp] += ga * o + a * go + a * o;
                    } else {
                        acc[j][r][cp] += a * o;
                    }
                }
        }
        nacc = 1;
    }

    for (int m = m0; m <= m1; ++m) {
        cl.sync();  // every row buffer holds E z of node m-1; column buffers are free
        // packed rows -> my packed columns: real rows (2kk, 2kk+1), real columns (2jj, 2jj+1);
        // all remote loads of a thread are issued before its stores
        {
            constexpr int NG = NY / 2 * W2 / T;
            float2 a[NG], c[NG];
#pragma unroll
            for (int u = 0; u < NG; ++u) {
                const int e = tid + u * T, kk = e / W2, jl = e % W2;
                const int src = kk / R2, bl = kk % R2, x0 = 2 * (crank * W2 + jl);
                const float2 *rb = cl.map_shared_rank(rowbuf, src);
                a[u] = rb[RL::at(bl, x0)];
                c[u] = rb[RL::at(bl, x0 + 1)];
            }
#pragma unroll
            for (int u = 0; u < NG; ++u) {
                const int e = tid + u * T, kk = e / W2, jl = e % W2;
                colbuf[CL::at(jl, 2 * kk)] = f2(a[u].x, c[u].x);
                colbuf[CL::at(jl, 2 * kk + 1)] = f2(a[u].y, c[u].y);
            }
        }
        __syncthreads();
        transform_pair<LOGY, T, CL, P>(colbuf, taby, ky, tid);
        {
            constexpr int RLOG_C = inv_rlog(LOGY, npasses(LOGY) - 1), NB_C = P / (1 << RLOG_C) / T;
            float2 x[NB_C][1 << RLOG_C];
            int bb[NB_C], tt[NB_C];
            last_inverse<LOGY, NB_C, T, CL>(colbuf, x, bb, tt, tid);
#pragma unroll
            for (int j = 0; j < NB_C; ++j)
#pragma unroll
                for (int r = 0; r < (1 << RLOG_C); ++r) colbuf[CL::at(bb[j], tt[j] + r * (NY >> RLOG_C))] = x[j][r];
        }
        cl.sync();  // every column buffer holds Ty E z; row buffers are free
        // packed columns -> my packed rows
        {
            constexpr int NG = R2 * (NX / 2) / T;
            float2 a[NG], c[NG];
#pragma unroll
            for (int u = 0; u < NG; ++u) {
                const int e = tid + u * T, bl = e / (NX / 2), jj = e % (NX / 2);
                const int src = jj / W2, jl = jj % W2, kk = krow0 + bl;
                const float2 *cb = cl.map_shared_rank(colbuf, src);
                a[u] = cb[CL::at(jl, 2 * kk)];
                c[u] = cb[CL::at(jl, 2 * kk + 1)];
            }
#pragma unroll
            for (int u = 0; u < NG; ++u) {
                const int e = tid + u * T, bl = e / (NX / 2), jj = e % (NX / 2);
                rowbuf[RL::at(bl, 2 * jj)] = f2(a[u].x, c[u].x);
                rowbuf[RL::at(bl, 2 * jj + 1)] = f2(a[u].y, c[u].y);
            }
        }
        __syncthreads();
        transform_pair<LOGX, T, RL, P>(rowbuf, tabx, kx, tid);
        float2 h[NB_L][RR];
        int bb[NB_L], tt[NB_L];
        last_inverse<LOGX, NB_L, T, RL>(rowbuf, h, bb, tt, tid);

        const bool acc_node = k.half == 1;
        const int jn = chain == 0 ? m : ns - m;  // contour node of this chain's term
        if (acc_node) {
            const float wa = wclass_a(jn, na), wb = wclass_b(jn, na, ns);
            if (nacc > 0 && (wa != gwa || wb != gwb || nacc == 8)) {
#pragma unroll
                for (int j = 0; j < NB_L; ++j) flush(bb[j], tt[j], j);
                nacc = 0;
            }
            if (nacc == 0) {
                gwa = wa;
                gwb = wb;
            }
            ++nacc;
        }
#pragma unroll
        for (int j = 0; j < NB_L; ++j) {
#pragma unroll
            for (int r = 0; r < RR; ++r) {
                const int x = tt[j] + r * PER_L;
                const long long site0 = (long long)(2 * (krow0 + bb[j])) * NX + x;
                const float e0 = sel(efac[site0], m), e1 = sel(efac[site0 + NX], m);
                if (!DIFF) {
                    const float z0 = e0 * h[j][r].x, z1 = e1 * h[j][r].y;
                    if (!acc_node || mode == 1) {
                        hist_me[(size_t)m * n + site0] = z0;
                        hist_me[(size_t)m * n + site0 + NX] = z1;
                    }
                    if (acc_node) {
                        acc[j][r][0] += z0 * hist_other[(size_t)(ns - m) * n + site0];
                        acc[j][r][1] += z1 * hist_other[(size_t)(ns - m) * n + site0 + NX];
                        if (m == ns) qsum += z0 + z1;
                    }
                    if (m < ns) rowbuf[RL::at(bb[j], x)] = f2(e0 * z0, e1 * z1);
                } else {
                    const float d0 = sel(defac[site0], m), d1 = sel(defac[site0 + NX], m);
                    const float g0 = ref_me[(size_t)m * n + site0], g1 = ref_me[(size_t)m * n + site0 + NX];
                    // dg = E T(da) + dE (T(a) + T(da)), T(a) = g / E of the reference solve
                    const float dg0 = e0 * h[j][r].x + d0 * (g0 / e0 + h[j][r].x);
                    const float dg1 = e1 * h[j][r].y + d1 * (g1 / e1 + h[j][r].y);
                    if (!acc_node) {
                        hist_me[(size_t)m * n + site0] = dg0;
                        hist_me[(size_t)m * n + site0 + NX] = dg1;
                    } else {
                        const size_t mo = (size_t)(ns - m) * n + site0;
                        const float o0 = hist_other[mo], o1 = hist_other[mo + NX];
                        const float q0 = ref_other[mo], q1 = ref_other[mo + NX];
                        acc[j][r][0] += g0 * o0 + dg0 * q0 + dg0 * o0;
                        acc[j][r][1] += g1 * o1 + dg1 * q1 + dg1 * o1;
                        if (m == ns) qsum += dg0 + dg1;
                    }
                    if (m < ns) rowbuf[RL::at(bb[j], x)] = f2(e0 * dg0 + d0 * (g0 + dg0), e1 * dg1 + d1 * (g1 + dg1));
                }
            }
        }
        if (acc_node && m == ns) {
#pragma unroll
            for (int j = 0; j < NB_L; ++j) flush(bb[j], tt[j], j);
            nacc = 0;
        }
    }
    if (k.half == 0) {
        __syncthreads();
        for (int e = tid; e < P; e += T) {
            const int b = e / NX, x = e % NX;
            state[(size_t)(krow0 + b) * NX + x] = rowbuf[RL::at(b, x)];
        }
    } else if (chain == 0) {
        const double s = block_sum((double)qsum, red);
        if (tid == 0) k.part[(size_t)run * kMaxPart + crank] = s;
    }
    cl.sync();  // no CTA leaves while others may still read its shared memory
}

// ---------------------------------------------------------------------------
// Host side: instantiated shapes, launch
// ---------------------------------------------------------------------------

struct ClusterShape {
    int logx, logy, c, t;
    const void *fn;       // plain and reference solves
    const void *fn_diff;  // differential solve
    size_t smem;
};

template <int LOGX, int LOGY, int C, int T>
static ClusterShape shape_of()
{
    return ClusterShape{LOGX, LOGY, C, T, (const void *)prop_cluster<LOGX, LOGY, C, T, false>,
                        (const void *)prop_cluster<LOGX, LOGY, C, T, true>, ClusterGeom<LOGX, LOGY, C, T>::SMEM};
}

// Instantiated grids (log2 nx, log2 ny): 4096 packed points per CTA with 256
// threads (two CTAs fit on one SM), fewer on the smallest grids.
static const ClusterShape *find_shape(int logx, int logy)
{
    static const ClusterShape shapes[] = {
        shape_of<6, 6, 2, 128>(),  shape_of<7, 6, 2, 256>(),  shape_of<6, 7, 2, 256>(),  shape_of<7, 7, 2, 512>(),
        shape_of<8, 7, 4, 512>(),  shape_of<7, 8, 4, 512>(),  shape_of<8, 8, 8, 512>(),  shape_of<9, 7, 8, 512>(),
        shape_of<7, 9, 8, 512>(),  shape_of<9, 8, 16, 512>(), shape_of<8, 9, 16, 512>(),
    };
    for (const auto &s : shapes)
        if (s.logx == logx && s.logy == logy) return &s;
    return nullptr;
}

static void set_cluster_cfg(cudaLaunchConfig_t &cfg, cudaLaunchAttribute &attr, const ClusterShape *s, int nclusters)
{
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = s->c;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3(s->c * nclusters, 1, 1);
    cfg.blockDim = dim3(s->t, 1, 1);
    cfg.dynamicSmemBytes = s->smem;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
}

bool cluster_solve_supported(const Group &G)
{
    if (G.prec != EPD_LB_MIXED_FP32) return false;
    const ClusterShape *s = find_shape(G.g.logx, G.g.logy);
    if (!s) return false;
    static int checked[16][16] = {};  // 0 unknown, 1 ok, 2 not launchable
    int &st = checked[s->logx][s->logy];
    if (st == 0) {
        st = 2;
        auto ok = [&](const void *fn) {
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem) != cudaSuccess) return false;
            if (s->c > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
                return false;
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr;
            set_cluster_cfg(cfg, attr, s, 1);
            int nclusters = 0;
            return cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) == cudaSuccess && nclusters > 0;
        };
        if (ok(s->fn) && ok(s->fn_diff)) st = 1;
        cudaGetLastError();
    }
    return st == 1;
}

bool cluster_shape_exists(int logx, int logy) { return find_shape(logx, logy) != nullptr; }

cudaError_t launch_cluster_solve(Group &G, cudaStream_t s, const void *twx_full, const void *twy_full, int mode)
{
    const ClusterShape *sh = find_shape(G.g.logx, G.g.logy);
    PropCK k;
    k.g = G.g;
    k.hist = reinterpret_cast<float *>(G.hist);
    k.hist1 = reinterpret_cast<float *>(G.hist1);
    k.defac = reinterpret_cast<const float2 *>(G.defac);
    k.mode = mode;
    k.state = reinterpret_cast<float2 *>(G.chain);
    k.efac = reinterpret_cast<const float2 *>(G.efac);
    k.ia0 = mode == 2 ? G.dia : G.ia;
    k.ib0 = mode == 2 ? G.dib : G.ib;
    k.ia1 = mode == 2 ? G.dia2 : G.ia2;
    k.ib1 = mode == 2 ? G.dib2 : G.ib2;
    k.part = G.part;
    k.twx = reinterpret_cast<const float2 *>(twx_full);
    k.twy = reinterpret_cast<const float2 *>(twy_full);
    k.kx = reinterpret_cast<const float *>(G.kx);
    k.ky = reinterpret_cast<const float *>(G.ky);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr;
    set_cluster_cfg(cfg, attr, sh, 2 * G.g.nruns);
    cfg.stream = s;
    for (int half = 0; half < 2; ++half) {
        k.half = half;
        void *args[] = {&k};
        const cudaError_t e = cudaLaunchKernelExC(&cfg, mode == 2 ? sh->fn_diff : sh->fn, args);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int cluster_ctas(const Group &G)
{
    const ClusterShape *sh = find_shape(G.g.logx, G.g.logy);
    return sh ? sh->c : 0;
}

} // namespace epdlb

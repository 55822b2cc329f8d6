// prop_cluster.cu -- cluster-resident single-chain solve (Sec. 2, Eqs. (6)-(10)
// of arXiv:1804.02883) for grids whose packed propagator field fits in the
// shared memory of one thread-block cluster (FP32 bulk precision).
//
// One cluster of C CTAs carries one run through the whole contour.  The
// packed field z = g + i g' lives on chip in two layouts: CTA c owns rows
// [c R, (c+1) R) in its row buffer and columns [c W, (c+1) W) in its column
// buffer.  One contour step (Eq. (8), Fourier factor split as Ky then Kx) is
//   gather rows -> my columns (distributed shared memory), column transform
//   Ky (forward, multiply, inverse), cluster barrier, gather columns -> my
//   rows, row transform Kx, node factors, history store or contour sums.
// Two cluster barriers per contour step; no kernel launch per step.
//
// Transforms: register-resident radix-8 (with one radix-2/4 pass where
// log2 N is not a multiple of 3) Stockham passes in shared memory.  The
// forward transform's last pass and the inverse transform's first pass
// touch the same points in each thread, so they are fused around the
// multiplication by the Fourier factor without a shared-memory round trip,
// and the inverse transform's last pass hands its points straight to the
// per-site epilogue.
//
// Contour sums (trapezoid of Eqs. (9)-(10)): products and partial sums over
// up to 8 consecutive nodes in FP32 registers, added into the FP64 sums
// I_A, I_B in global memory after every 8 nodes.
#include <cooperative_groups.h>

#include "common.cuh"
#include "engine.h"

namespace cg = cooperative_groups;

namespace epdlb {

struct PropCK {
    GroupGeom g;
    float2 *hist;
    const float2 *efac;
    double *ia, *ib, *part;
    const float2 *twx, *twy;  // exp(-2 pi i j / N), j < N
    const float *kx, *ky;     // exp(-R_G^2 k^2 ds) / N
};

// Radix plan: passes of radix 8, the last forward pass takes the remainder.
__host__ __device__ constexpr int npasses(int logn) { return (logn + 2) / 3; }
__host__ __device__ constexpr int fwd_rlog(int logn, int i) { return i < npasses(logn) - 1 ? 3 : logn - 3 * (npasses(logn) - 1); }
__host__ __device__ constexpr int fwd_slog(int logn, int i) { return i == 0 ? 0 : fwd_slog(logn, i - 1) + fwd_rlog(logn, i - 1); }
// inverse passes run the radices in reverse order
__host__ __device__ constexpr int inv_rlog(int logn, int i) { return fwd_rlog(logn, npasses(logn) - 1 - i); }
__host__ __device__ constexpr int inv_slog(int logn, int i) { return i == 0 ? 0 : inv_slog(logn, i - 1) + inv_rlog(logn, i - 1); }

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 fadd(float2 a, float2 b) { return f2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 fsub(float2 a, float2 b) { return f2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 fmul(float2 a, float2 b) { return f2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// multiply by -i (forward) or +i (inverse)
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
        // o_k *= exp(-+ 2 pi i k / 8)
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

// Shared-memory layouts.  Row layout: sequence b (a row), point x, rows padded
// by one slot per 8 points against bank conflicts.  Column layout: point y of
// sequence c (a column) at y * W + c.
template <int LOGN> struct RowLayout {
    static constexpr int N = 1 << LOGN, PITCH = N + N / 8;
    static __device__ __forceinline__ int at(int b, int x) { return b * PITCH + x + (x >> 3); }
    // butterfly index -> (sequence, index within sequence), sequences outermost
    template <int PER> static __device__ __forceinline__ void split(int bf, int &b, int &t) { b = bf / PER; t = bf % PER; }
};
template <int LOGN, int W> struct ColLayout {
    static __device__ __forceinline__ int at(int c, int y) { return y * W + c; }
    // consecutive threads take consecutive columns
    template <int PER> static __device__ __forceinline__ void split(int bf, int &b, int &t) { b = bf % W; t = bf / W; }
};

// One in-place Stockham pass (radix 2^RLOG, stride 2^SLOG) over all
// butterflies of the CTA's batch: each thread loads NB butterflies, waits for
// every thread, then writes.
template <int LOGN, int SLOG, int RLOG, bool INV, int NB, int T, class L>
__device__ __forceinline__ void pass(float2 *buf, const float2 *tw, int tid)
{
    constexpr int N = 1 << LOGN, R = 1 << RLOG, S = 1 << SLOG, PER = N / R;
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
        const int q = tt[j] & (S - 1), ps = tt[j] - q;  // ps = p * S
#pragma unroll
        for (int k = 1; k < R; ++k) {
            if (S < N / R) {  // p = 0 in the last pass: no twiddle
                float2 w = tw[ps * k];
                if (INV) w.y = -w.y;
                x[j][k] = fmul(x[j][k], w);
            }
        }
#pragma unroll
        for (int k = 0; k < R; ++k) buf[L::at(bb[j], q + R * ps + S * k)] = x[j][k];
    }
    __syncthreads();
}

// Forward transform's last pass, multiplication by the Fourier factor, and
// the inverse transform's first pass, fused (same points per thread).
template <int LOGN, int RLOG, int NB, int T, class L>
__device__ __forceinline__ void middle(float2 *buf, const float2 *tw, const float *kf, int tid)
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
        Dft<RLOG, false>::run(x[j]);  // last forward pass: outputs at t + k N/R
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const float f = kf[tt[j] + k * PER];
            x[j][k].x *= f;
            x[j][k].y *= f;
        }
        Dft<RLOG, true>::run(x[j]);   // first inverse pass (stride 1, p = t)
#pragma unroll
        for (int k = 1; k < R; ++k) {
            if (N / R > 1) {
                float2 w = tw[tt[j] * k];
                w.y = -w.y;
                x[j][k] = fmul(x[j][k], w);
            }
        }
#pragma unroll
        for (int k = 0; k < R; ++k) buf[L::at(bb[j], R * tt[j] + k)] = x[j][k];
    }
    __syncthreads();
}

// Forward passes 0 .. np-2.
template <int LOGN, int I, int T, class L, int P>
struct FwdPasses {
    static __device__ __forceinline__ void run(float2 *buf, const float2 *tw, int tid)
    {
        if constexpr (I < npasses(LOGN) - 1) {
            constexpr int RLOG = fwd_rlog(LOGN, I);
            pass<LOGN, fwd_slog(LOGN, I), RLOG, false, P / (1 << RLOG) / T, T, L>(buf, tw, tid);
            FwdPasses<LOGN, I + 1, T, L, P>::run(buf, tw, tid);
        }
    }
};
// Inverse passes 1 .. np-2 (pass 0 is fused into middle, pass np-1 is the
// caller's last pass).
template <int LOGN, int I, int T, class L, int P>
struct InvPasses {
    static __device__ __forceinline__ void run(float2 *buf, const float2 *tw, int tid)
    {
        if constexpr (I < npasses(LOGN) - 1) {
            constexpr int RLOG = inv_rlog(LOGN, I);
            pass<LOGN, inv_slog(LOGN, I), RLOG, true, P / (1 << RLOG) / T, T, L>(buf, tw, tid);
            InvPasses<LOGN, I + 1, T, L, P>::run(buf, tw, tid);
        }
    }
};

// Loads of the inverse transform's last pass (stride N/R, p = 0): each
// thread's points t + k N/R; the DFT leaves them in place.
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
__global__ void __launch_bounds__(T, 1) prop_cluster(PropCK k)
{
    constexpr int NX = 1 << LOGX, NY = 1 << LOGY, R = NY / C, W = NX / C;
    constexpr int P = R * NX;  // points per CTA in either layout
    static_assert(P == W * NY, "layout sizes");
    static_assert(P % (8 * T) == 0, "every pass gives each thread whole butterflies");
    static_assert(LOGX >= 4 && LOGY >= 4, "at least two passes per transform");
    static_assert(W >= 2 && R >= 1, "tile shape");
    using RL = RowLayout<LOGX>;
    using CL = ColLayout<LOGY, W>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *rowbuf = reinterpret_cast<float2 *>(smem_raw);
    float2 *colbuf = rowbuf + R * RL::PITCH;
    float2 *twx = colbuf + P;
    float2 *twy = twx + NX;
    float *kx = reinterpret_cast<float *>(twy + NY);
    float *ky = kx + NX;
    __shared__ double red[32];

    cg::cluster_group cl = cg::this_cluster();
    const int crank = (int)cl.block_rank();
    const int run = blockIdx.x / C;
    const int tid = threadIdx.x;
    const long long n = k.g.n;
    const int ns = k.g.ns, na = k.g.na, hlo = k.g.half_lo, hhi = k.g.half_hi;
    const int row0 = crank * R;

    for (int i = tid; i < NX; i += T) { twx[i] = k.twx[i]; kx[i] = k.kx[i]; }
    for (int i = tid; i < NY; i += T) { twy[i] = k.twy[i]; ky[i] = k.ky[i]; }

    const float2 *efac = k.efac + (size_t)run * n;
    float2 *hist = k.hist + (size_t)run * (hlo + 1) * n;
    double *ia = k.ia + (size_t)run * n, *ib = k.ib + (size_t)run * n;

    // node 0: g = g' = 1; the chain enters the first step as E(s_0) z_0
    for (int e = tid; e < P; e += T) {
        const int b = e / NX, x = e % NX;
        const long long site = (long long)(row0 + b) * NX + x;
        const float2 f = efac[site];
        hist[site] = f2(1.f, 1.f);
        rowbuf[RL::at(b, x)] = f2(0 < na ? f.x : f.y, ns < na ? f.x : f.y);
    }

    // epilogue geometry: the inverse row transform's last pass
    constexpr int RLOG_L = inv_rlog(LOGX, npasses(LOGX) - 1), RL_R = 1 << RLOG_L, PER_L = NX / RL_R;
    constexpr int NB_L = P / RL_R / T;
    float acc_a[NB_L][RL_R], acc_b[NB_L][RL_R];
#pragma unroll
    for (int j = 0; j < NB_L; ++j)
#pragma unroll
        for (int r = 0; r < RL_R; ++r) { acc_a[j][r] = 0.f; acc_b[j][r] = 0.f; }
    int nacc = 0;          // nodes in the FP32 partial sums
    bool first_flush = true;
    float qsum = 0.f;

    for (int m = 1; m <= ns; ++m) {
        cl.sync();  // every row buffer holds E z of node m-1; column buffers are free
        // rows -> my columns
        for (int e = tid; e < C * R * W; e += T) {
            const int src = e / (R * W), rem = e % (R * W), i = rem / W, j = rem % W;
            const float2 *rb = cl.map_shared_rank(rowbuf, src);
            colbuf[(src * R + i) * W + j] = rb[RL::at(i, crank * W + j)];
        }
        __syncthreads();
        // column transform: Ty = IFFT_y Ky FFT_y
        FwdPasses<LOGY, 0, T, CL, P>::run(colbuf, twy, tid);
        middle<LOGY, fwd_rlog(LOGY, npasses(LOGY) - 1), P / (1 << fwd_rlog(LOGY, npasses(LOGY) - 1)) / T, T, CL>(colbuf, twy, ky, tid);
        InvPasses<LOGY, 1, T, CL, P>::run(colbuf, twy, tid);
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
        // columns -> my rows
        for (int e = tid; e < C * R * W; e += T) {
            const int src = e / (R * W), rem = e % (R * W), i = rem / W, j = rem % W;
            const float2 *cb = cl.map_shared_rank(colbuf, src);
            rowbuf[RL::at(i, src * W + j)] = cb[(crank * R + i) * W + j];
        }
        __syncthreads();
        // row transform: Tx
        FwdPasses<LOGX, 0, T, RL, P>::run(rowbuf, twx, tid);
        middle<LOGX, fwd_rlog(LOGX, npasses(LOGX) - 1), P / (1 << fwd_rlog(LOGX, npasses(LOGX) - 1)) / T, T, RL>(rowbuf, twx, kx, tid);
        InvPasses<LOGX, 1, T, RL, P>::run(rowbuf, twx, tid);
        float2 h[NB_L][RL_R];
        int bb[NB_L], tt[NB_L];
        last_inverse<LOGX, NB_L, T, RL>(rowbuf, h, bb, tt, tid);

        // node m: factors, history, contour sums, next half step
        const bool acc_node = m >= hhi;
        const int s2 = ns - m;
        const float wa1 = wclass_a(m, na), wb1 = wclass_b(m, na, ns);
        const float wa2 = (s2 != m) ? wclass_a(s2, na) : 0.f, wb2 = (s2 != m) ? wclass_b(s2, na, ns) : 0.f;
        const bool gA = m < na, gpA = (ns - m) < na;
#pragma unroll
        for (int j = 0; j < NB_L; ++j) {
#pragma unroll
            for (int r = 0; r < RL_R; ++r) {
                const int x = tt[j] + r * PER_L;
                const long long site = (long long)(row0 + bb[j]) * NX + x;
                const float2 f = efac[site];
                const float eg = gA ? f.x : f.y, egp = gpA ? f.x : f.y;
                const float2 z = f2(eg * h[j][r].x, egp * h[j][r].y);
                if (m <= hlo) hist[(size_t)m * n + site] = z;
                if (acc_node) {
                    const float2 hv = (s2 == m) ? z : hist[(size_t)s2 * n + site];
                    const float t1 = z.x * hv.y;   // g(s_m) g'(1 - s_m)
                    const float t2 = hv.x * z.y;   // g(s_{ns-m}) g'(s_m)
                    acc_a[j][r] += wa1 * t1 + wa2 * t2;
                    acc_b[j][r] += wb1 * t1 + wb2 * t2;
                }
                if (m == ns) qsum += z.x;
                else rowbuf[RL::at(bb[j], x)] = f2(eg * z.x, egp * z.y);
            }
        }
        if (acc_node) {
            ++nacc;
            if (nacc == 8 || m == ns) {
                const double ds = k.g.ds;
#pragma unroll
                for (int j = 0; j < NB_L; ++j)
#pragma unroll
                    for (int r = 0; r < RL_R; ++r) {
                        const long long site = (long long)(row0 + bb[j]) * NX + tt[j] + r * PER_L;
                        const double va = ds * (double)acc_a[j][r], vb = ds * (double)acc_b[j][r];
                        if (first_flush) { ia[site] = va; ib[site] = vb; }
                        else { ia[site] += va; ib[site] += vb; }
                        acc_a[j][r] = 0.f;
                        acc_b[j][r] = 0.f;
                    }
                first_flush = false;
                nacc = 0;
            }
        }
    }
    const double s = block_sum((double)qsum, red);
    if (tid == 0) k.part[(size_t)run * kMaxPart + crank] = s;
    cl.sync();  // no CTA leaves while others may still read its shared memory
}

// ---------------------------------------------------------------------------
// Host side: instantiated shapes, launch
// ---------------------------------------------------------------------------

struct ClusterShape {
    int logx, logy, c, t;
    const void *fn;
    size_t smem;
};

template <int LOGX, int LOGY, int C, int T>
static ClusterShape shape_of()
{
    constexpr int NX = 1 << LOGX, NY = 1 << LOGY, R = NY / C;
    const size_t smem = (size_t)(R * (NX + NX / 8) + (NX / C) * NY) * sizeof(float2) + (NX + NY) * sizeof(float2) +
                        (NX + NY) * sizeof(float);
    return ClusterShape{LOGX, LOGY, C, T, (const void *)prop_cluster<LOGX, LOGY, C, T>, smem};
}

// Shapes with an instantiated cluster kernel: points per CTA 8192 (T = 512)
// or 2048 (T = 256).
static const ClusterShape *find_shape(int logx, int logy)
{
    static const ClusterShape shapes[] = {
        shape_of<6, 6, 2, 256>(),  shape_of<7, 6, 4, 256>(),  shape_of<6, 7, 4, 256>(),  shape_of<7, 7, 2, 512>(),
        shape_of<8, 7, 4, 512>(),  shape_of<7, 8, 4, 512>(),  shape_of<8, 8, 8, 512>(),  shape_of<9, 7, 8, 512>(),
        shape_of<7, 9, 8, 512>(),  shape_of<9, 8, 16, 512>(), shape_of<8, 9, 16, 512>(),
    };
    for (const auto &s : shapes)
        if (s.logx == logx && s.logy == logy) return &s;
    return nullptr;
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
        if (cudaFuncSetAttribute(s->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem) == cudaSuccess &&
            (s->c <= 8 || cudaFuncSetAttribute(s->fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess)) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr;
            attr.id = cudaLaunchAttributeClusterDimension;
            attr.val.clusterDim.x = s->c;
            attr.val.clusterDim.y = 1;
            attr.val.clusterDim.z = 1;
            cfg.gridDim = dim3(s->c, 1, 1);
            cfg.blockDim = dim3(s->t, 1, 1);
            cfg.dynamicSmemBytes = s->smem;
            cfg.attrs = &attr;
            cfg.numAttrs = 1;
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, s->fn, &cfg) == cudaSuccess && nclusters > 0) st = 1;
        }
        cudaGetLastError();
    }
    return st == 1;
}

cudaError_t launch_cluster_solve(Group &G, cudaStream_t s, const void *twx_full, const void *twy_full)
{
    const ClusterShape *sh = find_shape(G.g.logx, G.g.logy);
    PropCK k;
    k.g = G.g;
    k.hist = reinterpret_cast<float2 *>(G.hist);
    k.efac = reinterpret_cast<const float2 *>(G.efac);
    k.ia = G.ia;
    k.ib = G.ib;
    k.part = G.part;
    k.twx = reinterpret_cast<const float2 *>(twx_full);
    k.twy = reinterpret_cast<const float2 *>(twy_full);
    k.kx = reinterpret_cast<const float *>(G.kx);
    k.ky = reinterpret_cast<const float *>(G.ky);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = sh->c;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3(sh->c * G.g.nruns, 1, 1);
    cfg.blockDim = dim3(sh->t, 1, 1);
    cfg.dynamicSmemBytes = sh->smem;
    cfg.stream = s;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    void *args[] = {&k};
    return cudaLaunchKernelExC(&cfg, sh->fn, args);
}

int cluster_ctas(const Group &G)
{
    const ClusterShape *sh = find_shape(G.g.logx, G.g.logy);
    return sh ? sh->c : 0;
}

} // namespace epdlb

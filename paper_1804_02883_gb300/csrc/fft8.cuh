// fft8.cuh -- register-resident radix-8 Stockham transforms in shared memory
// (FP32), shared by the cluster-resident solve and the EPD passes of the
// hybrid LB/EPD step (arXiv:1804.02883, Sec. 2 and App. C).
//
// A tile holds sequences of N = 2^LOGN complex points in a layout L
// (RowLayout: sequence-major; ColLayout: point-major).  Passes are in place:
// every thread loads its points of the pass, the block synchronises, every
// thread writes its results.  Radix 8, with one radix-2/4 pass where log2 N is
// not a multiple of 3 (or radix 16 where a kernel asks for it); twiddles from
// per-pass tables (build_tables_host) laid out [row][p] so that consecutive
// threads read consecutive entries.
#pragma once

#include <cuda_runtime.h>

namespace epdlb {

// Radix plan: passes of radix 2^mr (8 by default, 16 where a kernel picks
// mr = 4), the last forward pass takes the remainder.
__host__ __device__ constexpr int npasses(int logn, int mr = 3) { return (logn + mr - 1) / mr; }
__host__ __device__ constexpr int fwd_rlog(int logn, int i, int mr = 3)
{
    return i < npasses(logn, mr) - 1 ? mr : logn - mr * (npasses(logn, mr) - 1);
}
__host__ __device__ constexpr int fwd_slog(int logn, int i, int mr = 3) { return i == 0 ? 0 : fwd_slog(logn, i - 1, mr) + fwd_rlog(logn, i - 1, mr); }
__host__ __device__ constexpr int inv_rlog(int logn, int i, int mr = 3) { return fwd_rlog(logn, npasses(logn, mr) - 1 - i, mr); }
__host__ __device__ constexpr int inv_slog(int logn, int i, int mr = 3) { return i == 0 ? 0 : inv_slog(logn, i - 1, mr) + inv_rlog(logn, i - 1, mr); }
// Twiddle tables: one per pass that needs twiddles (forward passes
// 0..np-2, inverse passes 0..np-2), rows x M entries, M = N / (S R): rows
// k = 1, 2, 4 for radix 8 and k = 1, 2, 4, 8 for radix 16 (the others are
// products), k = 1..R-1 otherwise.
__host__ __device__ constexpr int tab_rows(int rlog) { return rlog >= 3 ? rlog : (1 << rlog) - 1; }
__host__ __device__ constexpr int tab_len(int logn, int slog, int rlog) { return tab_rows(rlog) * ((1 << logn) >> (slog + rlog)); }
__host__ __device__ constexpr int fwd_off(int logn, int i, int mr = 3)
{
    return i == 0 ? 0 : fwd_off(logn, i - 1, mr) + tab_len(logn, fwd_slog(logn, i - 1, mr), fwd_rlog(logn, i - 1, mr));
}
__host__ __device__ constexpr int inv_off(int logn, int i, int mr = 3)
{
    return i == 0 ? fwd_off(logn, npasses(logn, mr) - 1, mr)
                  : inv_off(logn, i - 1, mr) + tab_len(logn, inv_slog(logn, i - 1, mr), inv_rlog(logn, i - 1, mr));
}
__host__ __device__ constexpr int tabs_total(int logn, int mr = 3) { return inv_off(logn, npasses(logn, mr) - 1, mr); }
// radix 16 where it takes fewer passes than radix 8 (128, 256, 1024, 2048
// points), else radix 8
__host__ __device__ constexpr int best_mr(int logn) { return npasses(logn, 4) < npasses(logn, 3) ? 4 : 3; }

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

// 16 points as 4 x 4: DFT4 over n1 of x[4 n1 + n2], twiddles W16^(n2 k1),
// DFT4 over n2; output X[k1 + 4 k2].
template <bool INV> struct Dft<4, INV> {
    static __device__ __forceinline__ void run(float2 *x)
    {
        const float c = 0.92387953251128675613f, s = 0.38268343236508977173f, h = 0.70710678118654752440f;
        float2 y[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            float2 v[4] = {x[n2], x[4 + n2], x[8 + n2], x[12 + n2]};
            Dft<2, INV>::run(v);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) y[n2][k1] = v[k1];
        }
        // W16^m = (cos(2 pi m / 16), -sin(2 pi m / 16)), conjugated for the inverse
        const float sg = INV ? 1.f : -1.f;
        const float2 w1 = f2(c, sg * s), w2 = f2(h, sg * h), w3 = f2(s, sg * c), w6 = f2(-h, sg * h), w9 = f2(-c, -sg * s);
        y[1][1] = fmul(y[1][1], w1);
        y[1][2] = fmul(y[1][2], w2);
        y[1][3] = fmul(y[1][3], w3);
        y[2][1] = fmul(y[2][1], w2);
        y[2][2] = rot90<INV>(y[2][2]);  // W16^4 = -i (forward)
        y[2][3] = fmul(y[2][3], w6);
        y[3][1] = fmul(y[3][1], w3);
        y[3][2] = fmul(y[3][2], w6);
        y[3][3] = fmul(y[3][3], w9);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            float2 v[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
            Dft<2, INV>::run(v);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) x[k1 + 4 * k2] = v[k2];
        }
    }
};

// Shared-memory layouts.  Row layout: sequence b (a packed row), point x.
// Rows of 128 points or more are unpadded with the low four bits of x
// XOR-ed by the next four (x ^ ((x >> 4) & 15)): every access pattern of the
// radix-8 passes then hits each 8-byte bank pair at most twice per warp
// (almost all once) and 16-point groups stay aligned and contiguous;
// 64-point rows are padded by one slot per 8 points.  Column layout: point y
// of sequence c (a packed column) at y * W + c.
template <int LOGN> struct RowLayout {
    static constexpr int N = 1 << LOGN, PITCH = LOGN >= 7 ? N : N + N / 8;
    static __device__ __forceinline__ int at(int b, int x)
    {
        if constexpr (LOGN >= 7)
            return b * PITCH + (x ^ ((x >> 4) & 15));
        else
            return b * PITCH + x + (x >> 3);
    }
    template <int PER> static __device__ __forceinline__ void split(int bf, int &b, int &t) { b = bf / PER; t = bf % PER; }
};
template <int LOGN, int W> struct ColLayout {
    static __device__ __forceinline__ int at(int c, int y) { return y * W + c; }
    template <int PER> static __device__ __forceinline__ void split(int bf, int &b, int &t) { b = bf % W; t = bf / W; }
};

// Twiddles w[k] = w1^k, k = 1..R-1, of one butterfly from a pass table laid
// out [row][p] (row length M): radix 8 reads w1, w2, w4 and radix 16 also w8,
// and forms the rest by products (at most three roundings more than a table
// entry).
template <int R>
__device__ __forceinline__ void twiddles(float2 (&w)[R], const float2 *tab, int M, int p)
{
    if constexpr (R == 8) {
        w[1] = tab[p];
        w[2] = tab[M + p];
        w[4] = tab[2 * M + p];
        w[3] = fmul(w[1], w[2]);
        w[5] = fmul(w[1], w[4]);
        w[6] = fmul(w[2], w[4]);
        w[7] = fmul(w[3], w[4]);
    } else if constexpr (R == 16) {
        w[1] = tab[p];
        w[2] = tab[M + p];
        w[4] = tab[2 * M + p];
        w[8] = tab[3 * M + p];
        w[3] = fmul(w[1], w[2]);
        w[5] = fmul(w[1], w[4]);
        w[6] = fmul(w[2], w[4]);
        w[7] = fmul(w[3], w[4]);
#pragma unroll
        for (int k = 9; k < 16; ++k) w[k] = fmul(w[k - 8], w[8]);
    } else {
#pragma unroll
        for (int k = 1; k < R; ++k) w[k] = tab[(k - 1) * M + p];
    }
}

// Butterfly index of thread tid's j-th butterfly (NB per thread) in a pass.
// WS = false: consecutive threads take consecutive butterflies over the tile.
// WS = true (warp-private): warp w takes the 32 NB butterflies from 32 NB w
// on, lane by lane, so that each warp owns whole sequences of a sequence-major
// layout and the pass needs only warp barriers; within a warp the access
// pattern is the same as in the tile-wide split.
template <bool WS, int NB, int T> __device__ __forceinline__ int bfly(int tid, int j)
{
    if constexpr (WS)
        return (tid >> 5) * (32 * NB) + (tid & 31) + 32 * j;
    else
        return tid + j * T;
}
template <bool WS> __device__ __forceinline__ void pass_sync()
{
    if constexpr (WS)
        __syncwarp();
    else
        __syncthreads();
}

// One in-place Stockham pass (radix 2^RLOG, stride 2^SLOG): load, wait, write.
// tab: this pass's twiddles [k-1][p] (unused in a forward last pass).
template <int LOGN, int SLOG, int RLOG, bool INV, int NB, int T, class L, bool WS = false>
__device__ __forceinline__ void pass(float2 *buf, const float2 *tab, int tid)
{
    constexpr int N = 1 << LOGN, R = 1 << RLOG, S = 1 << SLOG, PER = N / R, M = N / (S * R);
    float2 x[NB][R];
    int bb[NB], tt[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        L::template split<PER>(bfly<WS, NB, T>(tid, j), bb[j], tt[j]);
#pragma unroll
        for (int r = 0; r < R; ++r) x[j][r] = buf[L::at(bb[j], tt[j] + r * PER)];
    }
    pass_sync<WS>();
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        Dft<RLOG, INV>::run(x[j]);
        const int q = tt[j] & (S - 1), p = tt[j] >> SLOG;
        if (M > 1) {
            float2 w[R];
            twiddles<R>(w, tab, M, p);
#pragma unroll
            for (int k = 1; k < R; ++k) x[j][k] = INV ? fmulc(x[j][k], w[k]) : fmul(x[j][k], w[k]);
        }
#pragma unroll
        for (int k = 0; k < R; ++k) buf[L::at(bb[j], q + R * S * p + S * k)] = x[j][k];
    }
    pass_sync<WS>();
}

// Forward last pass, spectral operator, inverse first pass (same points per
// thread).  op(b, bin, v) returns the operator applied to bin `bin` (natural
// order) of sequence b.
template <int LOGN, int RLOG, int NB, int T, class L, class Op, bool WS = false>
__device__ __forceinline__ void middle(float2 *buf, const float2 *tab_inv0, const Op &op, int tid)
{
    constexpr int N = 1 << LOGN, R = 1 << RLOG, PER = N / R;
    float2 x[NB][R];
    int bb[NB], tt[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        L::template split<PER>(bfly<WS, NB, T>(tid, j), bb[j], tt[j]);
#pragma unroll
        for (int r = 0; r < R; ++r) x[j][r] = buf[L::at(bb[j], tt[j] + r * PER)];
    }
    pass_sync<WS>();
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        Dft<RLOG, false>::run(x[j]);
#pragma unroll
        for (int k = 0; k < R; ++k) x[j][k] = op(bb[j], tt[j] + k * PER, x[j][k]);
        Dft<RLOG, true>::run(x[j]);
        float2 w[R];
        twiddles<R>(w, tab_inv0, PER, tt[j]);
#pragma unroll
        for (int k = 1; k < R; ++k) x[j][k] = fmulc(x[j][k], w[k]);
#pragma unroll
        for (int k = 0; k < R; ++k) buf[L::at(bb[j], R * tt[j] + k)] = x[j][k];
    }
    pass_sync<WS>();
}

// Inverse first pass alone (input: a spectrum in natural order).
template <int LOGN, int RLOG, int NB, int T, class L, bool WS = false>
__device__ __forceinline__ void inverse_first(float2 *buf, const float2 *tab_inv0, int tid)
{
    constexpr int N = 1 << LOGN, R = 1 << RLOG, PER = N / R;
    float2 x[NB][R];
    int bb[NB], tt[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        L::template split<PER>(bfly<WS, NB, T>(tid, j), bb[j], tt[j]);
#pragma unroll
        for (int r = 0; r < R; ++r) x[j][r] = buf[L::at(bb[j], tt[j] + r * PER)];
    }
    pass_sync<WS>();
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        Dft<RLOG, true>::run(x[j]);
        float2 w[R];
        twiddles<R>(w, tab_inv0, PER, tt[j]);
#pragma unroll
        for (int k = 1; k < R; ++k) x[j][k] = fmulc(x[j][k], w[k]);
#pragma unroll
        for (int k = 0; k < R; ++k) buf[L::at(bb[j], R * tt[j] + k)] = x[j][k];
    }
    pass_sync<WS>();
}

template <int LOGN, int I, int T, class L, int P, int MR = 3, bool WS = false>
struct FwdPasses {
    static __device__ __forceinline__ void run(float2 *buf, const float2 *tabs, int tid)
    {
        if constexpr (I < npasses(LOGN, MR) - 1) {
            constexpr int RLOG = fwd_rlog(LOGN, I, MR);
            pass<LOGN, fwd_slog(LOGN, I, MR), RLOG, false, P / (1 << RLOG) / T, T, L, WS>(buf, tabs + fwd_off(LOGN, I, MR), tid);
            FwdPasses<LOGN, I + 1, T, L, P, MR, WS>::run(buf, tabs, tid);
        }
    }
};
template <int LOGN, int I, int T, class L, int P, int MR = 3, bool WS = false>
struct InvPasses {
    static __device__ __forceinline__ void run(float2 *buf, const float2 *tabs, int tid)
    {
        if constexpr (I < npasses(LOGN, MR) - 1) {
            constexpr int RLOG = inv_rlog(LOGN, I, MR);
            pass<LOGN, inv_slog(LOGN, I, MR), RLOG, true, P / (1 << RLOG) / T, T, L, WS>(buf, tabs + inv_off(LOGN, I, MR), tid);
            InvPasses<LOGN, I + 1, T, L, P, MR, WS>::run(buf, tabs, tid);
        }
    }
};

// Full transform pair (forward, spectral operator, inverse) up to the
// inverse's last pass, whose loads and DFT are left to the caller.
template <int LOGN, int T, class L, int P, class Op, int MR = 3, bool WS = false>
__device__ __forceinline__ void transform_pair(float2 *buf, const float2 *tabs, const Op &op, int tid)
{
    FwdPasses<LOGN, 0, T, L, P, MR, WS>::run(buf, tabs, tid);
    constexpr int RM = fwd_rlog(LOGN, npasses(LOGN, MR) - 1, MR);
    middle<LOGN, RM, P / (1 << RM) / T, T, L, Op, WS>(buf, tabs + inv_off(LOGN, 0, MR), op, tid);
    InvPasses<LOGN, 1, T, L, P, MR, WS>::run(buf, tabs, tid);
}

// Forward transform alone, result in natural order in buf.
template <int LOGN, int T, class L, int P, int MR = 3>
__device__ __forceinline__ void forward(float2 *buf, const float2 *tabs, int tid)
{
    FwdPasses<LOGN, 0, T, L, P, MR>::run(buf, tabs, tid);
    constexpr int I = npasses(LOGN, MR) - 1, RM = fwd_rlog(LOGN, I, MR);
    pass<LOGN, fwd_slog(LOGN, I, MR), RM, false, P / (1 << RM) / T, T, L>(buf, tabs, tid);  // M = 1: no twiddles
}

// Inverse transform of a natural-order spectrum up to its last pass (left to
// the caller, as in transform_pair).
template <int LOGN, int T, class L, int P, int MR = 3>
__device__ __forceinline__ void inverse_open(float2 *buf, const float2 *tabs, int tid)
{
    constexpr int RM = fwd_rlog(LOGN, npasses(LOGN, MR) - 1, MR);
    inverse_first<LOGN, RM, P / (1 << RM) / T, T, L>(buf, tabs + inv_off(LOGN, 0, MR), tid);
    InvPasses<LOGN, 1, T, L, P, MR>::run(buf, tabs, tid);
}

// Multiplication by a real per-bin factor table (the Fourier factor of Eq. (8)).
struct ScaleBins {
    const float *kf;
    __device__ __forceinline__ float2 operator()(int, int bin, float2 v) const
    {
        const float f = kf[bin];
        return f2(v.x * f, v.y * f);
    }
};

template <int LOGN, int NB, int T, class L, int MR = 3, bool WS = false>
__device__ __forceinline__ void last_inverse(const float2 *buf, float2 (&x)[NB][1 << inv_rlog(LOGN, npasses(LOGN, MR) - 1, MR)],
                                             int (&bb)[NB], int (&tt)[NB], int tid)
{
    constexpr int RLOG = inv_rlog(LOGN, npasses(LOGN, MR) - 1, MR), R = 1 << RLOG, PER = (1 << LOGN) / R;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        L::template split<PER>(bfly<WS, NB, T>(tid, j), bb[j], tt[j]);
#pragma unroll
        for (int r = 0; r < R; ++r) x[j][r] = buf[L::at(bb[j], tt[j] + r * PER)];
        Dft<RLOG, true>::run(x[j]);
    }
}

// Copy of prebuilt pass tables (built on the host with the same layout as
// the layout above) into shared memory: coalesced, no scattered gathers.
__device__ __forceinline__ void copy_tables(float2 *dst, const float2 *src, int len, int tid, int nthreads)
{
    for (int e = tid; e < len; e += nthreads) dst[e] = src[e];
}

// Host: the pass tables of a length-2^logn transform from the full twiddles
// tw[j] = exp(-2 pi i j / N) (interleaved re, im), for the plan of radix
// 2^mr.
inline void build_tables_host(int logn, const float *tw, float *out, int mr = 3)
{
    const int np = npasses(logn, mr);
    for (int I = 0; I < 2 * (np - 1); ++I) {
        const bool invp = I >= np - 1;
        const int pi = invp ? I - (np - 1) : I;
        const int slog = invp ? inv_slog(logn, pi, mr) : fwd_slog(logn, pi, mr);
        const int rlog = invp ? inv_rlog(logn, pi, mr) : fwd_rlog(logn, pi, mr);
        const int off = invp ? inv_off(logn, pi, mr) : fwd_off(logn, pi, mr);
        const int M = (1 << logn) >> (slog + rlog), len = tab_rows(rlog) * M;
        for (int e = 0; e < len; ++e) {
            const int row = e / M, p = e % M;
            const int k = rlog >= 3 ? (1 << row) : row + 1;
            const int j = (p << slog) * k;
            out[2 * (off + e)] = tw[2 * j];
            out[2 * (off + e) + 1] = tw[2 * j + 1];
        }
    }
}

// Tiles of the streaming passes (one CTA per tile, in-place transforms): a
// row tile holds 2048 points (max(1, 2048 / nx) whole rows), a column tile CW
// whole columns (by default 16, 8 from 1024 rows on; the autotuner picks 4, 8
// or 16 per grid).
// Radix plan MR = best_mr(N) (rows; columns where it fits); one butterfly of
// the largest radix per thread.
template <int LOGX> struct RowTile {
    static constexpr int MR = best_mr(LOGX);
    static constexpr int NX = 1 << LOGX, ROWS = NX >= 2048 ? 1 : 2048 / NX, P = ROWS * NX, T = P >> MR;
    static constexpr int TAB = tabs_total(LOGX, MR);
    static constexpr size_t SMEM = (size_t)(ROWS * RowLayout<LOGX>::PITCH + TAB) * sizeof(float2);
};
template <int LOGY, int CW = (LOGY >= 10 ? 8 : 16)> struct ColTile {
    static constexpr int NY = 1 << LOGY, C = CW, P = C * NY;
    // radix 16 only where one 16-point butterfly per thread fits in 512 threads
    static constexpr int MR = (best_mr(LOGY) == 4 && (P >> 4) <= 512) ? 4 : 3;
    static constexpr int T = (P >> MR) > 512 ? 512 : (P >> MR);
    static constexpr int TAB = tabs_total(LOGY, MR);
    static constexpr size_t SMEM = (size_t)(P + TAB) * sizeof(float2);
};
// column tile widths the autotuner chooses from (0: the default above)
constexpr int kColWidths[3] = {4, 8, 16};

} // namespace epdlb

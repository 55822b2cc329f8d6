// common.cuh -- shared device types and the in-shared-memory FFT used by the
// propagator, EPD and force passes of the hybrid LB/EPD step (arXiv:1804.02883).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace epdlb {

// ---------------------------------------------------------------------------
// complex pairs
// ---------------------------------------------------------------------------
template <typename T> struct V2Of;
template <> struct V2Of<float> { using type = float2; };
template <> struct V2Of<double> { using type = double2; };
template <typename T> using V2 = typename V2Of<T>::type;

template <typename T> __host__ __device__ __forceinline__ V2<T> mk(T x, T y) { V2<T> r; r.x = x; r.y = y; return r; }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { a.x += b.x; a.y += b.y; return a; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename V> __device__ __forceinline__ V cmul(V a, V b)
{
    V r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename V, typename S> __device__ __forceinline__ V cscale(V a, S s) { a.x *= s; a.y *= s; return a; }

// ---------------------------------------------------------------------------
// Batched radix-2 Stockham FFT in shared memory.
//
// The batch holds B sequences of N = 2^logN complex points; point k of
// sequence b sits at x[b*sb + k*sn].  Each stage reads the pair (r, r + N/2)
// of every sequence and writes the autosorted pair (2r - (r mod stride),
// +stride), so no bit reversal is needed; the result is in natural order and
// unnormalised.  tw holds exp(-2 pi i t / N), t < N/2; INVERSE conjugates it.
// BATCH_FAST maps consecutive threads to consecutive sequences (for the
// column layout, sn > 1), otherwise to consecutive points (row layout).
// Every thread of the block must call it; it ends with a __syncthreads and
// returns the buffer that holds the result (x or y).
// ---------------------------------------------------------------------------
template <typename T, bool INVERSE, bool BATCH_FAST>
__device__ __forceinline__ V2<T> *fft_smem(V2<T> *x, V2<T> *y, int logN, int logB, int sb, int sn,
                                           const V2<T> *tw)
{
    const int half = 1 << (logN - 1);
    const int total = half << logB;
    for (int s = 0; s < logN; ++s) {
        const int stride = 1 << s;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            int b, r;
            if (BATCH_FAST) {
                b = t & ((1 << logB) - 1);
                r = t >> logB;
            } else {
                b = t >> (logN - 1);
                r = t & (half - 1);
            }
            const int q = r & (stride - 1);
            const int base = b * sb;
            V2<T> a = x[base + r * sn];
            V2<T> c = x[base + (r + half) * sn];
            V2<T> w = tw[r - q];
            if (INVERSE) w.y = -w.y;
            const int o = base + (2 * r - q) * sn;
            y[o] = cadd(a, c);
            y[o + stride * sn] = cmul(csub(a, c), w);
        }
        __syncthreads();
        V2<T> *tmp = x;
        x = y;
        y = tmp;
    }
    return x;
}

// Quotient of 0 <= n < 2^24 by a positive d through the float reciprocal,
// corrected to the exact integer quotient (a runtime integer division costs
// tens of instructions; this one a handful).
struct FastDiv {
    int d;
    float inv;
    __device__ __forceinline__ explicit FastDiv(int d_) : d(d_), inv(1.0f / (float)d_) {}
    __device__ __forceinline__ int div(int n) const
    {
        int q = __float2int_rz((float)n * inv);
        if ((q + 1) * d <= n) ++q;
        if (q * d > n) --q;
        return q;
    }
};

// One radix-P butterfly of the mixed-radix Stockham transform below (q = r
// mod s, j = r / s).  The p-th roots are tw[k m] (m = N/P); (u v mod P) m and
// v j s stay below N.
template <typename T, bool INVERSE, int P>
__device__ __forceinline__ void fft_mr_butterfly(const V2<T> *x, V2<T> *y, const V2<T> *tw, int base, int r, int q, int j,
                                                 int m, int s, int sn)
{
    V2<T> in[P], root[P];
#pragma unroll
    for (int u = 0; u < P; ++u) {
        in[u] = x[base + (r + u * m) * sn];
        root[u] = tw[u * m];  // the P-th roots of unity
        if (INVERSE) root[u].y = -root[u].y;
    }
#pragma unroll
    for (int v = 0; v < P; ++v) {
        V2<T> acc = in[0];
#pragma unroll
        for (int u = 1; u < P; ++u) acc = cadd(acc, cmul(in[u], root[(u * v) % P]));
        if (v) {
            V2<T> w = tw[v * j * s];
            if (INVERSE) w.y = -w.y;
            acc = cmul(acc, w);
        }
        y[base + (j * P * s + v * s + q) * sn] = acc;
    }
}

// Mixed-radix (radices 2, 3, 4, 5) Stockham transform of B sequences of
// length N in shared memory, for axes that are not powers of two: the same
// data layout as fft_smem (element t of sequence b at b * sb + t * sn).  fac
// lists the radices (product N); tw holds exp(-2 pi i t / N) for all t < N.
// Stage with radix p after the radices s = p_1 ... p_{k-1}: butterfly r < N/p
// (q = r mod s, j = r / s) takes x[r + u N/p], u < p, forms their p-point DFT
// X_v and writes X_v exp(-+2 pi i v j s / N) to y[j p s + v s + q]; the output
// ends in natural order.
template <typename T, bool INVERSE, bool BATCH_FAST>
__device__ __forceinline__ V2<T> *fft_smem_mr(V2<T> *x, V2<T> *y, int N, int nf, const int *fac, int B, int sb, int sn,
                                              const V2<T> *tw)
{
    int s = 1;
    const FastDiv fb(B);
    for (int st = 0; st < nf; ++st) {
        const int p = fac[st], m = N / p, total = m * B;
        const FastDiv fm(m), fs(s);
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            int b, r;
            if (BATCH_FAST) {
                r = fb.div(t);
                b = t - r * B;
            } else {
                b = fm.div(t);
                r = t - b * m;
            }
            const int j = fs.div(r), q = r - j * s;
            const int base = b * sb;
            switch (p) {
            case 2: fft_mr_butterfly<T, INVERSE, 2>(x, y, tw, base, r, q, j, m, s, sn); break;
            case 3: fft_mr_butterfly<T, INVERSE, 3>(x, y, tw, base, r, q, j, m, s, sn); break;
            case 4: fft_mr_butterfly<T, INVERSE, 4>(x, y, tw, base, r, q, j, m, s, sn); break;
            default: fft_mr_butterfly<T, INVERSE, 5>(x, y, tw, base, r, q, j, m, s, sn); break;
            }
        }
        __syncthreads();
        V2<T> *tmp = x;
        x = y;
        y = tmp;
        s *= p;
    }
    return x;
}

// 8-byte asynchronous copy global -> shared (the thread's own staging
// slot), and the commit / wait of the thread's copy groups
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// 16-byte asynchronous copy global -> shared, not cached in L1
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Block-wide sum of one double per thread (blockDim.x a multiple of 32, at
// most 1024).  Fixed order: deterministic.  Result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *scratch32)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) scratch32[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        r = lane < nw ? scratch32[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;
}

// Sum of cnt partial sums, identical in every block that calls it (the
// warp-0 lanes take fixed strided slices).  Result valid in thread 0 of warp 0
// and broadcast through the returned value of every thread after the call.
__device__ __forceinline__ double sum_partials(const double *part, int cnt, int stride_el, double *bcast)
{
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int i = threadIdx.x; i < cnt; i += 32) v += part[(size_t)i * stride_el];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) *bcast = v;
    }
    __syncthreads();
    double r = *bcast;
    __syncthreads();
    return r;
}

__host__ __device__ __forceinline__ int ilog2(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// Signed index of FFT bin m on an axis of n points.
__device__ __forceinline__ int signed_bin(int m, int n) { return m <= (n >> 1) ? m : m - n; }

constexpr int kThreads = 256;

} // namespace epdlb

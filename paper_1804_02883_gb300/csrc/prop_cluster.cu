// prop_cluster.cu -- cluster-resident single-chain solve (Sec. 2, Eqs. (6)-(11)
// of arXiv:1804.02883) for grids whose propagator field fits in the shared
// memory of one thread-block cluster (FP32 bulk precision).
//
// One cluster of C CTAs carries one chain of one run through the whole
// contour: the forward propagator g (Eq. (6)) or the backward propagator g'
// (Eq. (7)), so a launch holds 2 x runs clusters (or, in the phased
// schedule, 2 x runs - 1 clusters per launch over 2 x runs launches, each
// chain resuming from the state it stored).  The real field of the
// chain lives on chip in two packings: CTA c owns complex rows
// [c R2, (c+1) R2), each holding the real rows (2k, 2k+1) as (re, im), in its
// row buffer, and complex columns [c W2, (c+1) W2), each holding the real
// columns (2j, 2j+1), in its column buffer.  The Fourier factor of Eq. (8) is
// real, even and separable, K = Kx(kx) Ky(ky), so it acts on each packed
// row / column as on two real ones, and its row part Gx = IFFT_x Kx FFT_x and
// column part Gy commute.  Contour step m computes
//   a_m = E_m g_m = E_m^2 Gx Gy a_{m-1}
// as Gy, exchange, Gx on odd steps and Gx, exchange, Gy on even steps: each
// step ends in the packing the next one starts from, so the field changes
// packing once per contour step (one all-to-all of the cluster, 2 x 2 re/im
// transposes by lane-pair shuffles).  The exchange is a push: each CTA
// writes its points into the owners' buffer with st.async, counted as
// transaction bytes on the owner's mbarrier; no cluster barrier is needed
// inside the contour loop (see the ordering note at the loop).  The row
// transforms are warp-private (each warp owns whole packed rows).  Every
// step stores a_m in the packed-row layout for the contour sums.
//
// The contour sums of Eqs. (9)-(10) pair node m of g with node N_s - m of g'
// at every site: a separate pass (prop_contour) reads both chains' stored
// states, forms g_m g'_{N_s-m} = a_m a'_{N_s-m} / E_m^2 (both chains see the
// same node factor at mirrored nodes), sums the trapezoid weights and
// normalises (Eq. (11)).
//
// Transforms: register-resident radix-8 (one radix-2/4 pass where log2 N is
// not a multiple of 3) Stockham passes in shared memory, in place.  The
// forward transform's last pass, the multiplication by the Fourier factor
// and the inverse transform's first pass are fused (same points per
// thread); the inverse's last pass hands its points to the per-site
// epilogue.  Twiddles come from per-pass tables laid out [k][p] so that
// consecutive threads read consecutive entries.
//
// Differential solve (DIFF): the step's second solve differs from its first
// (the reference, states a~) only by the diffusion update d omega of Eq. (5):
// its node factors are E' = E (1 + rho), rho = expm1(-N d omega ds / 2) from
// the FP64 difference.  It propagates the change d a_m = a_m - a~_m through
// the same transforms: with U = T(d a_{m-1}) and T(a~_{m-1}) = a~_m / E^2,
//   d a_m = E'^2 U + rho (2 + rho) a~_m,
// the exact difference of a_m = E'^2 T(a_{m-1}) and a~_m = E^2 T(a~_{m-1}),
// both terms of the size of the change.  prop_contour<DIFF> recovers
// dg = (d a - rho a~) / E' and sums g~ dg' + dg g~' + dg dg'.  Exact algebra
// of the second solve; only the rounding changes: FP32 relative to the
// change, not to Phi.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <cooperative_groups.h>

#include "common.cuh"
#include "engine.h"
#include "fft8.cuh"

namespace cg = cooperative_groups;

namespace epdlb {

struct PropCK {
    GroupGeom g;
    float2 *hout;         // stored states a_m (or d a_m): [run][chain][N_s + 1][NY/2][NX] (packed rows)
    const float2 *href;   // reference states a~_m (DIFF)
    const float2 *efac;   // (E_A, E_B) [run][n]
    const float2 *rho;    // (rho_A, rho_B) [run][n] (DIFF)
    const float2 *cdiff;  // (1 + rho_d)(1 + rho_a) - 1 for (A,A), (B,B), (A,B), packed rows [run][3][NY/2][NX] (DIFF)
    int *err;             // bit 2: an exchange wait gave up
    const float2 *twx, *twy;  // radix-8 pass tables (fft8.cuh layout)
    const float *kx, *ky;     // exp(-R_G^2 k^2 ds) / N
    // Phased schedule (nseg > 0): this launch is phase `skip` of nseg + 1;
    // its nseg clusters take every chain but chain `skip`, each over its next
    // contour segment (segment s = nodes s N_s / nseg .. (s + 1) N_s / nseg),
    // resuming from the state the previous phase stored.  nseg = 0: one
    // launch, every chain over all N_s steps.
    int nseg, skip;
};

template <int LOGX, int LOGY, int C, int T>
struct ClusterGeom {
    static constexpr int NX = 1 << LOGX, NY = 1 << LOGY, R2 = NY / 2 / C, W2 = NX / 2 / C;
    static constexpr int P = R2 * NX;  // complex points per CTA in either packing
    static constexpr int PITCH = RowLayout<LOGX>::PITCH;
    static constexpr int HN = NY / 2 * NX;  // stored complex points per chain and node
    // radix 16 where it saves passes (fft8.cuh best_mr) and every thread gets
    // whole 16-point butterflies
    static constexpr int MRX = (best_mr(LOGX) == 4 && P % (16 * T) == 0) ? 4 : 3;
    static constexpr int MRY = (best_mr(LOGY) == 4 && P % (16 * T) == 0) ? 4 : 3;
    static constexpr int TABX = tabs_total(LOGX, MRX), TABY = tabs_total(LOGY, MRY);
    // row buffer, column buffer, pass tables, Fourier factors, the node
    // factors of the epilogue sites in either packing (P points each; the
    // differential solve reads the coefficients of a~ from L2, which
    // measured faster than a shared-memory copy beside the factors)
    static constexpr size_t SMEM =
        (size_t)(R2 * PITCH + P + TABX + TABY + 2 * P) * sizeof(float2) + (NX + NY) * sizeof(float);
    static constexpr size_t SMEM_DIFF = SMEM;
};

// Distributed-shared-memory pushes: st.async of 8 bytes into a CTA of the
// cluster, counted as transaction bytes on that CTA's mbarrier.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned map_rank(unsigned addr, int rank)
{
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void push_f2(unsigned raddr, float2 v, unsigned rbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(raddr), "f"(v.x),
                 "f"(v.y), "r"(rbar)
                 : "memory");
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase with the given parity to complete, giving up after
// `limit` cycles (about 2^31, a second): then `failed` is set and every later
// wait returns at once (the kernel runs to its end with the same barrier
// sequence and reports the error).
__device__ __forceinline__ void mbar_wait(unsigned bar, unsigned parity, int &failed, long long limit = 1ll << 31)
{
    if (failed) return;
    const long long t0 = clock64();
    while (!mbar_test(bar, parity))
        if (clock64() - t0 > limit) {
            failed = 1;
            return;
        }
}

// Points of the column transform's last pass for butterfly index bf: packed
// column c and butterfly t, arranged so that the threads holding real rows y
// and y + 1 (butterflies t and t + 1, same r) of one column are lanes l and
// l ^ 16 of a warp; the 2 x 2 re/im transpose between the packings is then
// one shuffle.  Bijective on [0, W PER) when W PER is a multiple of 32 and
// PER is even; for W = 16 it is the tile-wide split of the other passes.
template <int W>
__device__ __forceinline__ void col_pair_split(int bf, int &c, int &t)
{
    const int lin = (bf >> 5) * 16 + (bf & 15), par = (bf >> 4) & 1;
    c = lin % W;
    t = 2 * (lin / W) + par;
}

// The 2 x 2 re/im transpose of a lane pair (partner lane ^ LANES): the lane
// with odd = false holds (p(2i, r), p(2i+1, r)) and its partner
// (p(2i, r+1), p(2i+1, r+1)) of one packing; afterwards they hold
// (p(2i, r), p(2i, r+1)) and (p(2i+1, r), p(2i+1, r+1)) of the other.  The
// transpose is its own inverse.
template <int LANES>
__device__ __forceinline__ float2 pair_transpose(float2 v, bool odd)
{
    const float t = __shfl_xor_sync(0xffffffffu, odd ? v.x : v.y, LANES);
    return odd ? f2(t, v.y) : f2(v.x, t);
}

// Contour step m applies the Fourier factor of Eq. (8) as its column part Gy
// (all packed columns) and its row part Gx (all packed rows).  The factor is
// separable, so Gx and Gy commute: odd steps take Gy first, even steps Gx
// first, and each step ends in the packing its next step starts from.  One
// exchange of the field between the packings per contour step.
__device__ __forceinline__ bool starts_in_columns(int m) { return m & 1; }

// MINB: CTAs per SM the register budget is sized for (65536 / (T MINB) each)
template <int LOGX, int LOGY, int C, int T, int MINB, bool DIFF>
__global__ void __launch_bounds__(T, MINB) prop_chain(PropCK k)
{
    using G = ClusterGeom<LOGX, LOGY, C, T>;
    constexpr int NX = G::NX, NY = G::NY, R2 = G::R2, W2 = G::W2, P = G::P, HN = G::HN;
    constexpr int NWARP = T / 32;
    static_assert(P == W2 * NY, "layout sizes");
    static_assert(P % (8 * T) == 0, "every pass gives each thread whole butterflies");
    static_assert(LOGX >= 4 && LOGY >= 4 && R2 >= 1 && W2 >= 1, "tile shape");
    static_assert(T % 32 == 0 && P % T == 0 && NX % 2 == 0, "whole warps, lane pairs");
    static_assert(R2 % NWARP == 0, "warp-private row transforms: every warp owns whole packed rows");
    static_assert(W2 % 16 == 0 || 16 % W2 == 0, "column pairs of the last column pass");
    using RL = RowLayout<LOGX>;
    using CL = ColLayout<LOGY, W2>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2 *rowbuf = reinterpret_cast<float2 *>(smem_raw);
    float2 *colbuf = rowbuf + R2 * G::PITCH;
    float2 *tabx = colbuf + P;
    float2 *taby = tabx + G::TABX;
    float *kx = reinterpret_cast<float *>(taby + G::TABY);
    float *ky = kx + NX;
    // node factors of the two real sites of each epilogue point, thread-major
    // ([point of the thread][thread]: conflict-free), rows then columns:
    // E_d E_a (plain) or E'_d E'_a (DIFF)
    float2 *fac_r = reinterpret_cast<float2 *>(ky + NY), *fac_c = fac_r + P;
    cg::cluster_group cl = cg::this_cluster();
    const int crank = (int)cl.block_rank();
    const int slot = blockIdx.x / C;
    const int cidx = (k.nseg == 0 || slot < k.skip) ? slot : slot + 1, run = cidx >> 1, chain = cidx & 1;
    const int tid = threadIdx.x;
    const int n = (int)k.g.n, ns = k.g.ns, na = k.g.na;
    // contour steps m_begin + 1 .. m_end of this launch (segments in order
    // over the phases: chain j sits out phase j)
    const int seg = k.skip < cidx ? k.skip : k.skip - 1;
    const int m_begin = k.nseg ? seg * ns / k.nseg : 0, m_end = k.nseg ? (seg + 1) * ns / k.nseg : ns;
    const int nsteps = m_end - m_begin;
    const int krow0 = crank * R2, jcol0 = crank * W2;  // first packed row and packed column of this CTA

    copy_tables(tabx, k.twx, G::TABX, tid, T);
    copy_tables(taby, k.twy, G::TABY, tid, T);
    for (int i = tid; i < NX; i += T) kx[i] = k.kx[i];
    for (int i = tid; i < NY; i += T) ky[i] = k.ky[i];
    const float2 *efac = k.efac + (size_t)run * n;
    const float2 *rho = DIFF ? k.rho + (size_t)run * n : nullptr;
    // this chain's stored states of node m at hout + m HN, packed rows
    // [NY/2][NX]; rho (2 + rho) of blocks A, B in the same layout
    float2 *hout = k.hout + (size_t)(run * 2 + chain) * (ns + 1) * HN;
    const float2 *href = DIFF ? k.href + (size_t)(run * 2 + chain) * (ns + 1) * HN : nullptr;
    const float2 *cdiff = DIFF ? k.cdiff + (size_t)run * 3 * HN : nullptr;

    // blocks of the two half-step factors at contour node j of this chain
    // (half_step_block: the literal junction rule gives both the block of
    // node j, g carrying w_A iff j < N_A and g' the field of node N_s - j).
    // The stored state is a_j = E_dep(j) g_j, so a_j = E_dep(j) E_arr(j) T(a_{j-1}).
    auto dep_b = [&](int j) { return half_step_block(k.g.jr, chain, j, ns, na, false); };
    auto arr_b = [&](int j) { return half_step_block(k.g.jr, chain, j, ns, na, true); };
    // a_0 = E_0 (d a_0 = rho_0 E_0) at the real site of packed row kk,
    // column x, rows 2kk (re) and 2kk + 1 (im)
    auto node0 = [&](int kk, int x) {
        const int site = 2 * kk * NX + x;
        const bool bk = dep_b(0);
        const float2 f0 = efac[site], f1 = efac[site + NX];
        float2 a0 = bk ? f2(f0.y, f1.y) : f2(f0.x, f1.x);
        if (DIFF) {
            const float2 r0 = rho[site], r1 = rho[site + NX];
            a0.x *= bk ? r0.y : r0.x;
            a0.y *= bk ? r1.y : r1.x;
        }
        return a0;
    };

    // exchange barriers: [0] my column buffer (filled by the exchange of the
    // steps that start in rows), [1] my row buffer (steps that start in
    // columns); each completes once per use, when all P points have arrived
    __shared__ __align__(8) unsigned long long mbar[2];
    const unsigned bar_col = smem_u32(&mbar[0]), bar_row = smem_u32(&mbar[1]);
    constexpr unsigned XBYTES = (unsigned)(P * sizeof(float2));
    if (tid == 0) {
        mbar_init(bar_col, 1);
        mbar_init(bar_row, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_expect(bar_col, XBYTES);
        mbar_expect(bar_row, XBYTES);
    }


    const bool odd = tid & 1;
    // last row pass (warp-private) and last column pass geometry
    constexpr int RLOG_L = inv_rlog(LOGX, npasses(LOGX, G::MRX) - 1, G::MRX), RR = 1 << RLOG_L, PER_L = NX / RR;
    constexpr int NB_L = P / RR / T;
    static_assert(PER_L % 2 == 0, "lane pairs (x, x + 1) of the last row pass");
    constexpr int RLOG_C = inv_rlog(LOGY, npasses(LOGY, G::MRY) - 1, G::MRY), RC = 1 << RLOG_C, PER_C = NY / RC;
    constexpr int NB_C = P / RC / T;
    static_assert(PER_C % 2 == 0 && (P / RC) % 32 == 0, "column pairs of the last column pass");
    // per-site factors E^2 (plain) or E'^2 (DIFF) of this thread's epilogue
    // sites in either packing (fac_r, fac_c), reloaded when the block (A or
    // B) changes; each thread reads only what it wrote
    int cur_r = -1, cur_c = -1;
    int failed = 0;
    // the factors of packed-row point (kk, x) for blocks d (departing) and a
    // (arriving): real sites 2kk (re) and 2kk + 1 (im) of column x
    auto factors = [&](int kk, int x, bool bd, bool ba) {
        const int s0 = 2 * kk * NX + x;
        const float2 e0 = efac[s0], e1 = efac[s0 + NX];
        const float f0 = (bd ? e0.y : e0.x) * (ba ? e0.y : e0.x), f1 = (bd ? e1.y : e1.x) * (ba ? e1.y : e1.x);
        if constexpr (!DIFF) {
            return f2(f0, f1);
        } else {
            const float2 r0 = rho[s0], r1 = rho[s0 + NX];
            return f2(f0 * ((1.f + (bd ? r0.y : r0.x)) * (1.f + (ba ? r0.y : r0.x))),
                      f1 * ((1.f + (bd ? r1.y : r1.x)) * (1.f + (ba ? r1.y : r1.x))));
        }
    };
    // a_m = E_d E_a U (plain) or d a_m = E'_d E'_a U + c a~_m (DIFF) at
    // packed-row point (kk, x), U = T(a_{m-1}) there, c = (1 + rho_d)(1 +
    // rho_a) - 1 from plane cp of cdiff (0: A A, 1: B B, 2: A B)
    auto finish = [&](float2 u, float2 f, int m, int cp, int kk, int x) {
        if constexpr (!DIFF) {
            return f2(f.x * u.x, f.y * u.y);
        } else {
            const size_t e = (size_t)kk * NX + x;
            const float2 ar = href[(size_t)m * HN + e];  // a~_m
            const float2 c = cdiff[(size_t)cp * HN + e];
            return f2(f.x * u.x + c.x * ar.x, f.y * u.y + c.y * ar.y);
        }
    };

    // per-site factors of this thread's epilogue points in the row packing
    // (fac_r) and the column packing (fac_c) for blocks (bd, ba)
    auto fill_r = [&](bool bd, bool ba) {
#pragma unroll
        for (int j = 0; j < NB_L; ++j) {
            int b, t;
            RL::template split<PER_L>(bfly<true, NB_L, T>(tid, j), b, t);
#pragma unroll
            for (int r = 0; r < RR; ++r) fac_r[(j * RR + r) * T + tid] = factors(krow0 + b, t + r * PER_L, bd, ba);
        }
    };
    auto fill_c = [&](bool bd, bool ba) {
#pragma unroll
        for (int j = 0; j < NB_C; ++j) {
            int c, t;
            col_pair_split<W2>(tid + j * T, c, t);
#pragma unroll
            for (int r = 0; r < RC; ++r) {
                const int kk = (t + r * PER_C) >> 1, xx = 2 * (jcol0 + c) + (t & 1);
                fac_c[(j * RC + r) * T + tid] = factors(kk, xx, bd, ba);
            }
        }
    };
    // The factors of the first step (both packings; they depend only on the
    // fields of this solve, final before the first launch), then the state
    // the previous launch of a phased schedule stored: a launch made as a
    // programmatic dependent of the previous one runs this prologue while
    // that one finishes, and waits for it only here (griddepcontrol.wait
    // returns at once in a launch without that dependency).
    if (nsteps > 0) {
        const int m1 = m_begin + 1;
        const int bd1 = dep_b(m1), ba1 = arr_b(m1);
        fill_r(bd1, ba1);
        fill_c(bd1, ba1);
        cur_r = cur_c = 2 * bd1 + ba1;
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");

    // node m_begin into the packing the first step starts from: a_0 from the
    // node factors (and stored for the contour sums), or the state a_{m_begin}
    // the previous phase stored (the same FP32 values, so the result does not
    // depend on the schedule)
    if (m_begin == 0) {
        for (int e = tid; e < P; e += T) hout[(size_t)krow0 * NX + e] = node0(krow0 + e / NX, e % NX);
    }
    if (starts_in_columns(m_begin + 1)) {
        // packed column jcol0 + c, real row y: (a(2J, y), a(2J + 1, y))
        for (int e = tid; e < P; e += T) {
            const int c = e % W2, y = e / W2, jx = 2 * (jcol0 + c), kk = y >> 1;
            float2 p0, p1;
            if (m_begin == 0) {
                p0 = node0(kk, jx);
                p1 = node0(kk, jx + 1);
            } else {
                p0 = hout[(size_t)m_begin * HN + kk * NX + jx];
                p1 = hout[(size_t)m_begin * HN + kk * NX + jx + 1];
            }
            colbuf[CL::at(c, y)] = (y & 1) ? f2(p0.y, p1.y) : f2(p0.x, p1.x);
        }
    } else {
        for (int e = tid; e < P; e += T) {
            const int b = e / NX, x = e % NX;
            rowbuf[RL::at(b, x)] = m_begin == 0 ? node0(krow0 + b, x) : hout[(size_t)m_begin * HN + (size_t)krow0 * NX + e];
        }
    }
    cl.sync();  // every CTA's barriers are initialised, the first packing is in place

    // The contour loop runs over half steps: each applies the transform pair
    // of its packing, then either hands the field over (first half of a
    // step) or applies the node factors (second half), so every transform is
    // compiled once.  Step m's halves are in columns then rows for odd m,
    // rows then columns for even m.  A buffer is written by the exchange only
    // every other step, and only by CTAs that have received data which every
    // owner computed after its last read of that buffer, so the pushes are
    // ordered behind those reads through the exchange barriers themselves.
    for (int hs = 0; hs < 2 * nsteps; ++hs) {
        const int i = hs >> 1, m = m_begin + 1 + i;
        const bool second = hs & 1, cols = starts_in_columns(m) != second;
        const unsigned par = (unsigned)(i >> 1) & 1u;  // uses of this step's barrier so far in this launch
        const bool rearm = i + 2 < nsteps;
        const int bd = dep_b(m), ba = arr_b(m), key = 2 * bd + ba, cp = bd == ba ? bd : 2;
        if (DIFF && !second) {
            // a~_m and c of this step's epilogue sites into L1 ahead of use
            // (the packing the step ends in)
            auto pf = [&](size_t e) {
                asm volatile("prefetch.global.L1 [%0];" ::"l"(href + (size_t)m * HN + e));
                asm volatile("prefetch.global.L1 [%0];" ::"l"(cdiff + (size_t)cp * HN + e));
            };
            if (cols) {
#pragma unroll
                for (int j = 0; j < NB_L; ++j) {
                    int b, t;
                    RL::template split<PER_L>(bfly<true, NB_L, T>(tid, j), b, t);
#pragma unroll
                    for (int r = 0; r < RR; ++r) pf((size_t)(krow0 + b) * NX + t + r * PER_L);
                }
            } else {
#pragma unroll
                for (int j = 0; j < NB_C; ++j) {
                    int c, t;
                    col_pair_split<W2>(tid + j * T, c, t);
#pragma unroll
                    for (int r = 0; r < RC; ++r)
                        pf((size_t)((t + r * PER_C) >> 1) * NX + 2 * (jcol0 + c) + (t & 1));
                }
            }
        }
        if (cols) {
            // ---- Gy on my packed columns
            transform_pair<LOGY, T, CL, P, ScaleBins, G::MRY>(colbuf, taby, ScaleBins{ky}, tid);
            float2 x[NB_C][RC];
            int cc[NB_C], ct[NB_C];
#pragma unroll
            for (int j = 0; j < NB_C; ++j) {
                col_pair_split<W2>(tid + j * T, cc[j], ct[j]);
#pragma unroll
                for (int r = 0; r < RC; ++r) x[j][r] = colbuf[CL::at(cc[j], ct[j] + r * PER_C)];
            }
#pragma unroll
            for (int j = 0; j < NB_C; ++j) Dft<RLOG_C, true>::run(x[j]);
            if (!second) {
                // my columns -> the owners' rows: lanes l (real row y = 2kk)
                // and l ^ 16 (y + 1) of packed column J form points x = 2J and
                // 2J + 1 of packed row kk
#pragma unroll
                for (int j = 0; j < NB_C; ++j) {
                    const bool oy = ct[j] & 1;
#pragma unroll
                    for (int r = 0; r < RC; ++r) {
                        const float2 v = pair_transpose<16>(x[j][r], oy);
                        const int kk = (ct[j] + r * PER_C) >> 1, dst = kk / R2;
                        const int xx = 2 * (jcol0 + cc[j]) + (oy ? 1 : 0);
                        push_f2(map_rank(smem_u32(rowbuf + RL::at(kk % R2, xx)), dst), v, map_rank(bar_row, dst));
                    }
                }
                mbar_wait(bar_row, par, failed);
                // re-armed before this warp's next warp barrier, which orders
                // it before every later push of this warp that the barrier's
                // next use depends on
                if (tid == 0 && rearm) mbar_expect(bar_row, XBYTES);
            } else {
                // node factors in the packed-row form (x = 2J + (y & 1) of
                // packed row y / 2), the result back in the column buffer
                if (key != cur_c) {
                    cur_c = key;
                    fill_c(bd, ba);
                }
#pragma unroll
                for (int j = 0; j < NB_C; ++j)
#pragma unroll
                    for (int r = 0; r < RC; ++r) {
                        const int kk = (ct[j] + r * PER_C) >> 1, xx = 2 * (jcol0 + cc[j]) + (ct[j] & 1);
                        x[j][r] = finish(pair_transpose<16>(x[j][r], ct[j] & 1), fac_c[(j * RC + r) * T + tid], m, cp, kk, xx);
                    }
                __syncthreads();  // every thread has read its columns: they are rewritten below
#pragma unroll
                for (int j = 0; j < NB_C; ++j) {
                    const bool oy = ct[j] & 1;
#pragma unroll
                    for (int r = 0; r < RC; ++r) {
                        const int y = ct[j] + r * PER_C, kk = y >> 1, xx = 2 * (jcol0 + cc[j]) + (oy ? 1 : 0);
                        hout[(size_t)m * HN + (size_t)kk * NX + xx] = x[j][r];
                        colbuf[CL::at(cc[j], y)] = pair_transpose<16>(x[j][r], oy);
                    }
                }
                __syncthreads();  // the next step's column passes read every column
            }
        } else {
            // ---- Gx on my packed rows (each warp its own)
            transform_pair<LOGX, T, RL, P, ScaleBins, G::MRX, true>(rowbuf, tabx, ScaleBins{kx}, tid);
            float2 h[NB_L][RR];
            int bb[NB_L], tt[NB_L];
            last_inverse<LOGX, NB_L, T, RL, G::MRX, true>(rowbuf, h, bb, tt, tid);
            if (!second) {
                // my rows -> the owners' columns: lanes (2i, 2i + 1) hold
                // columns (x0, x0 + 1) of packed row kk; the even lane forms
                // real row 2kk of packed column x0 / 2, the odd lane real row
                // 2kk + 1
#pragma unroll
                for (int j = 0; j < NB_L; ++j)
#pragma unroll
                    for (int r = 0; r < RR; ++r) {
                        const float2 v = pair_transpose<1>(h[j][r], odd);
                        const int jj = (tt[j] + r * PER_L) >> 1, dst = jj / W2, y = 2 * (krow0 + bb[j]) + (odd ? 1 : 0);
                        push_f2(map_rank(smem_u32(colbuf + CL::at(jj % W2, y)), dst), v, map_rank(bar_col, dst));
                    }
                mbar_wait(bar_col, par, failed);
                // re-armed before this step's CTA barriers, so before every later push
                if (tid == 0 && rearm) mbar_expect(bar_col, XBYTES);
            } else {
                // node factors; the result stays in the row buffer
                if (key != cur_r) {
                    cur_r = key;
                    fill_r(bd, ba);
                }
                // every value first: the stores come after
#pragma unroll
                for (int j = 0; j < NB_L; ++j)
#pragma unroll
                    for (int r = 0; r < RR; ++r)
                        h[j][r] = finish(h[j][r], fac_r[(j * RR + r) * T + tid], m, cp, krow0 + bb[j], tt[j] + r * PER_L);
#pragma unroll
                for (int j = 0; j < NB_L; ++j)
#pragma unroll
                    for (int r = 0; r < RR; ++r) {
                        const int x = tt[j] + r * PER_L;
                        hout[(size_t)m * HN + (size_t)(krow0 + bb[j]) * NX + x] = h[j][r];
                        rowbuf[RL::at(bb[j], x)] = h[j][r];
                    }
                __syncwarp();  // the next step's row passes read these rows in this warp
            }
        }
    }
    if (failed) atomicOr(k.err, 4);
    cl.sync();  // no CTA leaves while others may still write into its shared memory
}

// ---------------------------------------------------------------------------
// Contour sums and normalisation, Eqs. (9)-(11)
// ---------------------------------------------------------------------------

constexpr int kQBlocks = 32;  // blocks (and partials) of prop_qsum per run

struct ContourK {
    GroupGeom g;
    int hn;                 // stored points per chain and node
    int nq, ns_part;        // Q partials (first nq entries), solvent partials (from kMaxPart/2)
    const float2 *hc;       // states a_m (reference / plain solve)
    const float2 *hd;       // changes d a_m (differential solve)
    const float2 *efac, *rho;
    double *part;
    const double *phi_t, *q_t;  // first solve's densities (differential solve)
    double *phi, *q;
    int *err;
};

// Compensated (Kahan) FP32 sum: value() = sum minus the carried rounding
// error, in FP64.  GB300's FP64 rate is a small fraction of FP32, so per-node
// FP64 accumulation would bound these passes.
struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float t)
    {
        const float y = t - c, u = s + y;
        c = (u - s) - y;
        s = u;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Trapezoid weights over [0, s_{N_A}] and [s_{N_A}, 1] in units of ds.
__device__ __forceinline__ void node_weights(int j, int na, int ns, float &wa, float &wb)
{
    wa = (na == 0 || j > na) ? 0.f : ((j == 0 || j == na) ? 0.5f : 1.f);
    wb = (na == ns || j < na) ? 0.f : ((j == na || j == ns) ? 0.5f : 1.f);
}

// Self-test of the bounded wait: one CTA waits on an exchange barrier that
// nothing arrives on, with the given limit, and reports the give-up in the
// error word exactly as prop_chain does (bit 2).
__global__ void selftest_wait(int *err, long long limit)
{
    __shared__ __align__(8) unsigned long long mbar;
    const unsigned bar = smem_u32(&mbar);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int failed = 0;
    mbar_wait(bar, 0, failed, limit);  // phase 0 never completes
    if (failed && threadIdx.x == 0) atomicOr(err, 4);
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

// Q partials from node N_s of the g chain: Q_P = mean g_{N_s} with
// g = a / E (plain); dQ_P = mean dg_{N_s}, dg = (d a - rho a~) / E' (DIFF).
// Block sums into part[run][block].
template <bool DIFF>
__global__ void __launch_bounds__(kThreads) prop_qsum(ContourK k)
{
    __shared__ double red[32];
    const int run = blockIdx.y;
    const int nx = k.g.nx, ns = k.g.ns, na = k.g.na;
    const long long n = k.g.n;
    const int npk = nx * k.g.ny / 2;
    const bool bm = half_step_block(k.g.jr, 0, ns, ns, na, false);  // a_{N_s} = E_bm g_{N_s}
    const size_t cs = (size_t)(ns + 1) * k.hn;
    const float2 *a_ns = k.hc + (size_t)run * 2 * cs + (size_t)ns * k.hn;
    const float2 *d_ns = DIFF ? k.hd + (size_t)run * 2 * cs + (size_t)ns * k.hn : nullptr;
    const float2 *efac = k.efac + (size_t)run * n;
    const float2 *rho = DIFF ? k.rho + (size_t)run * n : nullptr;
    float acc = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npk; i += gridDim.x * blockDim.x) {
        const int kk = i >> k.g.logx, x = i & (nx - 1), s0 = 2 * kk * nx + x, s1 = s0 + nx;
        const float2 e0 = efac[s0], e1 = efac[s1], a = a_ns[i];
        const float E0 = bm ? e0.y : e0.x, E1 = bm ? e1.y : e1.x;
        if (!DIFF) {
            acc += a.x / E0 + a.y / E1;
        } else {
            const float2 r0 = rho[s0], r1 = rho[s1], d = d_ns[i];
            const float q0 = bm ? r0.y : r0.x, q1 = bm ? r1.y : r1.x;
            acc += (d.x - q0 * a.x) / (E0 * (1.f + q0)) + (d.y - q1 * a.y) / (E1 * (1.f + q1));
        }
    }
    const double s = block_sum((double)acc, red);
    if (threadIdx.x == 0) k.part[(size_t)run * kMaxPart + blockIdx.x] = s;
}

// Contour chunks staged per thread: U nodes of each stream (g, g' and, in the
// differential pass, their changes), two stages in flight.
template <bool DIFF> struct ContourStage {
    static constexpr int U = DIFF ? 4 : 8, NW = DIFF ? 4 : 2, NSTAGE = 2;
    static constexpr size_t SMEM = (size_t)NSTAGE * U * NW * kThreads * sizeof(float2);
};

// One thread per packed site (real rows 2kk and 2kk+1 at column x).
// Products in FP32, partial sums over at most 8 nodes of equal weights in
// FP32, then FP64.  The node states stream through shared memory by
// asynchronous copies, each thread staging only its own elements (no
// barriers), so that the loads in flight do not hold registers.
template <bool DIFF>
__global__ void __launch_bounds__(kThreads) prop_contour(ContourK k)
{
    extern __shared__ __align__(16) float2 stg[];
    __shared__ double bc;
    const int run = blockIdx.y;
    const int nx = k.g.nx, ny = k.g.ny, ns = k.g.ns, na = k.g.na;
    const long long n = k.g.n;
    const int npk = nx * ny / 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < npk;
    const int kk = i >> k.g.logx, x = i & (nx - 1);  // power-of-two grids
    const int s0 = 2 * kk * nx + x, s1 = s0 + nx;
    const int slot = kk * nx + x;
    const size_t cs = (size_t)(ns + 1) * k.hn;  // one chain's states
    const float2 *c0 = k.hc + (size_t)run * 2 * cs + slot, *c1 = c0 + cs;
    const float2 *d0 = DIFF ? k.hd + (size_t)run * 2 * cs + slot : nullptr, *d1 = DIFF ? d0 + cs : nullptr;
    using CS = ContourStage<DIFF>;
    constexpr int U = CS::U, NW = CS::NW;
    const int tid = threadIdx.x;
    // stage st, node u, stream w: stg[((st U + u) NW + w) kThreads + tid]
    auto issue = [&](int st, int m0) {
        if (valid) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int m = m0 + u;
                if (m <= ns) {
                    float2 *b = stg + (size_t)((st * U + u) * NW) * kThreads + tid;
                    cp_async8(b, c0 + (size_t)m * k.hn);
                    cp_async8(b + kThreads, c1 + (size_t)(ns - m) * k.hn);
                    if (DIFF) {
                        cp_async8(b + 2 * kThreads, d0 + (size_t)m * k.hn);
                        cp_async8(b + 3 * kThreads, d1 + (size_t)(ns - m) * k.hn);
                    }
                }
            }
        }
        cp_async_commit();
    };
    // a ring of NSTAGE chunks: chunk ch + NSTAGE goes into chunk ch's stage
    // once ch is consumed; every issue commits a group (empty past N_s), so
    // waiting until at most NSTAGE - 1 groups are pending completes chunk ch.
    // The first chunks are in flight while the block sums the Q partials.
    constexpr int NST = CS::NSTAGE;
#pragma unroll
    for (int c = 0; c < NST; ++c) issue(c, c * U);
    const double *pr = k.part + (size_t)run * kMaxPart;
    const double sq = sum_partials(pr, k.nq, 1, &bc) / (double)n;
    const double ss = sum_partials(pr + kMaxPart / 2, k.ns_part, 1, &bc) / (double)n;
    double qp, qs;
    if (DIFF) {
        qp = k.q_t[2 * run] + sq;
        qs = k.q_t[2 * run + 1] + ss;
    } else {
        qp = sq;
        qs = ss;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        k.q[2 * run] = qp;
        k.q[2 * run + 1] = qs;
        if (!(qp > 0.0) || !(qs > 0.0) || !isfinite(qp) || !isfinite(qs)) atomicOr(k.err, 1);
    }
    if (!valid) {
        cp_async_wait<0>();
        return;
    }
    const float2 *efac = k.efac + (size_t)run * n;
    const float2 e0 = efac[s0], e1 = efac[s1];
    // per block (A, B) of the contour: 1 / E^2 (plain); 1 / E, rho, 1 / E' (DIFF)
    float r2[2][2], ri[2][2], dd[2][2], rs[2][2];
    {
        const float e[2][2] = {{e0.x, e1.x}, {e0.y, e1.y}};
        float2 q0 = f2(0.f, 0.f), q1 = f2(0.f, 0.f);
        if (DIFF) {
            const float2 *rho = k.rho + (size_t)run * n;
            q0 = rho[s0];
            q1 = rho[s1];
        }
        const float q[2][2] = {{q0.x, q1.x}, {q0.y, q1.y}};
#pragma unroll
        for (int bk = 0; bk < 2; ++bk)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                r2[bk][c] = 1.f / (e[bk][c] * e[bk][c]);
                ri[bk][c] = 1.f / e[bk][c];
                dd[bk][c] = q[bk][c];
                rs[bk][c] = 1.f / (e[bk][c] * (1.f + q[bk][c]));
            }
    }
    // compensated (Kahan) FP32 sums per block and real site; the trapezoid
    // weights 1 and 1/2 scale the terms exactly
    KSum sa0, sb0, sa1, sb1;
    const int nch = (ns + U) / U;  // chunks of U nodes over 0..ns
    for (int ch = 0; ch < nch; ++ch) {
        cp_async_wait<NST - 1>();
        const int st = ch % NST, m0 = ch * U;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int m = m0 + u;
            if (m > ns) break;
            const float2 *b = stg + (size_t)((st * U + u) * NW) * kThreads + tid;
            float wa, wb;
            node_weights(m, na, ns, wa, wb);
            // the stored states are a = E_dep g: the departing blocks of g at
            // node m and of g' at node N_s - m (the same, B from N_A on, under
            // the literal junction rule)
            const bool bk = half_step_block(k.g.jr, 0, m, ns, na, false);
            const bool bp = half_step_block(k.g.jr, 1, ns - m, ns, na, false);
            // (selects: a run-time index would move these small arrays to local memory)
            auto pick = [](const float (&v)[2][2], bool b, int c) { return b ? v[1][c] : v[0][c]; };
            const float2 a = b[0], bb = b[kThreads];
            float t0, t1;
            if (!DIFF) {
                t0 = a.x * bb.x * (bk == bp ? pick(r2, bk, 0) : ri[0][0] * ri[1][0]);
                t1 = a.y * bb.y * (bk == bp ? pick(r2, bk, 1) : ri[0][1] * ri[1][1]);
            } else {
                const float2 da = b[2 * kThreads], db = b[3 * kThreads];
                // g~ = a~ / E and dg = (d a - rho a~) / E' of both chains
                const float ga0 = a.x * pick(ri, bk, 0), ga1 = a.y * pick(ri, bk, 1);
                const float gb0 = bb.x * pick(ri, bp, 0), gb1 = bb.y * pick(ri, bp, 1);
                const float dga0 = (da.x - pick(dd, bk, 0) * a.x) * pick(rs, bk, 0);
                const float dga1 = (da.y - pick(dd, bk, 1) * a.y) * pick(rs, bk, 1);
                const float dgb0 = (db.x - pick(dd, bp, 0) * bb.x) * pick(rs, bp, 0);
                const float dgb1 = (db.y - pick(dd, bp, 1) * bb.y) * pick(rs, bp, 1);
                t0 = ga0 * dgb0 + dga0 * gb0 + dga0 * dgb0;
                t1 = ga1 * dgb1 + dga1 * gb1 + dga1 * dgb1;
            }
            if (wa != 0.f) {
                sa0.add(wa * t0);
                sa1.add(wa * t1);
            }
            if (wb != 0.f) {
                sb0.add(wb * t0);
                sb1.add(wb * t1);
            }
        }
        issue(st, (ch + NST) * U);  // this stage's values are consumed
    }
    const double ia0 = sa0.value(), ib0 = sb0.value(), ia1 = sa1.value(), ib1 = sb1.value();
    const double ds = k.g.ds, php = k.g.phi_p;
    double *pa = k.phi + (size_t)run * 3 * n, *pb = pa + n, *ps = pb + n;
    if (!DIFF) {
        const double c = php * ds / qp;
        pa[s0] = c * ia0;
        pb[s0] = c * ib0;
        pa[s1] = c * ia1;
        pb[s1] = c * ib1;
        const double cs_ = (1.0 - php) / qs;
        ps[s0] *= cs_;
        ps[s1] *= cs_;
    } else {
        // Phi = Phi~ + (phi_p dI - Phi~ dQ) / (Q~ + dQ), the solvent with de
        const double *ta = k.phi_t + (size_t)run * 3 * n, *tb = ta + n, *tsol = tb + n;
        const double rq = 1.0 / qp, rqs = 1.0 / qs, c = php * ds;
        pa[s0] = ta[s0] + (c * ia0 - ta[s0] * sq) * rq;
        pb[s0] = tb[s0] + (c * ib0 - tb[s0] * sq) * rq;
        pa[s1] = ta[s1] + (c * ia1 - ta[s1] * sq) * rq;
        pb[s1] = tb[s1] + (c * ib1 - tb[s1] * sq) * rq;
        ps[s0] = tsol[s0] + ((1.0 - php) * ps[s0] - tsol[s0] * ss) * rqs;
        ps[s1] = tsol[s1] + ((1.0 - php) * ps[s1] - tsol[s1] * ss) * rqs;
    }
}

// ---------------------------------------------------------------------------
// Host side: instantiated shapes, launch
// ---------------------------------------------------------------------------

struct ClusterShape {
    int logx, logy, c, t;
    const void *fn;       // plain and reference solves
    const void *fn_diff;  // differential solve
    size_t smem, smem_diff;
    int mrx, mry;         // radix plans of the row and column transforms (log2 of the largest radix)
};

template <int LOGX, int LOGY, int C, int T, int MINB = 1024 / T>
static ClusterShape shape_of()
{
    return ClusterShape{LOGX, LOGY, C, T, (const void *)prop_chain<LOGX, LOGY, C, T, MINB, false>,
                        (const void *)prop_chain<LOGX, LOGY, C, T, MINB, true>, ClusterGeom<LOGX, LOGY, C, T>::SMEM,
                        ClusterGeom<LOGX, LOGY, C, T>::SMEM_DIFF, ClusterGeom<LOGX, LOGY, C, T>::MRX,
                        ClusterGeom<LOGX, LOGY, C, T>::MRY};
}

// Instantiated grids (log2 nx, log2 ny).  Tiles of 4096 points take 256
// threads (one or two butterflies per thread and pass) with the SM's whole
// register file (both packings' per-site factors stay in registers; at 128
// registers a thread spilled 220-480 bytes); the smaller tiles fit several
// CTAs per SM.
static const ClusterShape *find_shape(int logx, int logy)
{
    static const ClusterShape shapes[] = {
        shape_of<6, 6, 2, 128, 4>(),  shape_of<7, 6, 2, 256, 2>(),  shape_of<6, 7, 2, 256, 2>(),
        shape_of<7, 7, 2, 256, 1>(),  shape_of<8, 7, 4, 256, 1>(),  shape_of<7, 8, 4, 256, 1>(),
        shape_of<8, 8, 8, 256, 1>(),  shape_of<9, 7, 8, 256, 1>(),  shape_of<7, 9, 8, 256, 1>(),
        shape_of<9, 8, 16, 256, 1>(), shape_of<8, 9, 16, 256, 1>(),
    };
    for (const auto &s : shapes)
        if (s.logx == logx && s.logy == logy) return &s;
    return nullptr;
}

static const void *chain_fn(const ClusterShape *s, bool diff) { return diff ? s->fn_diff : s->fn; }

static void set_cluster_cfg(cudaLaunchConfig_t &cfg, cudaLaunchAttribute &attr, const ClusterShape *s, int nclusters,
                            bool diff)
{
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = s->c;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3(s->c * nclusters, 1, 1);
    cfg.blockDim = dim3(s->t, 1, 1);
    cfg.dynamicSmemBytes = diff ? s->smem_diff : s->smem;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
}

// Clusters of a shape that fit at once at one CTA per SM (more than half of
// an SM's shared memory per CTA), per shape and solve kind; 0: unknown or
// none.  Filled by cluster_solve_supported, outside any stream capture.
constexpr size_t kSoloSmem = 116 * 1024;
// phased launches as programmatic dependents (EPD_LB_CHAIN_PDL=0 in the
// environment turns it off, for timing one against the other)
static const bool g_chain_pdl = [] {
    const char *e = std::getenv("EPD_LB_CHAIN_PDL");
    return !(e && e[0] == '0');
}();
static int g_solo_clusters[16][16][2];

static int count_solo_clusters(const ClusterShape *s, bool diff)
{
    const void *fn = chain_fn(s, diff);
    const size_t sm = std::max(kSoloSmem, diff ? s->smem_diff : s->smem);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return 0;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr;
    set_cluster_cfg(cfg, attr, s, 1, diff);
    cfg.dynamicSmemBytes = sm;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess) return 0;
    return nclusters;
}

bool cluster_solve_supported(const Group &G)
{
    if (G.prec != EPD_LB_MIXED_FP32) return false;
    const ClusterShape *s = find_shape(G.g.logx, G.g.logy);
    if (!s) return false;
    static std::mutex mu;  // handles may be created on several threads
    std::lock_guard<std::mutex> lock(mu);
    static int checked[16][16] = {};  // 0 unknown, 1 ok, 2 not launchable
    int &st = checked[s->logx][s->logy];
    if (st == 0) {
        st = 2;
        auto ok = [&](bool diff) {
            const void *fn = chain_fn(s, diff);
            const size_t sm = diff ? s->smem_diff : s->smem;
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return false;
            if (s->c > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
                return false;
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr;
            set_cluster_cfg(cfg, attr, s, 1, diff);
            int nclusters = 0;
            return cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) == cudaSuccess && nclusters > 0;
        };
        if (ok(false) && ok(true)) {
            st = 1;
            g_solo_clusters[s->logx][s->logy][0] = count_solo_clusters(s, false);
            g_solo_clusters[s->logx][s->logy][1] = count_solo_clusters(s, true);
        }
        cudaGetLastError();
    }
    return st == 1;
}

bool cluster_shape_exists(int logx, int logy) { return find_shape(logx, logy) != nullptr; }

int cluster_chain_launches(const Group &G, bool diff)
{
    const ClusterShape *sh = find_shape(G.g.logx, G.g.logy);
    if (!sh) return 0;
    const int nch = 2 * G.g.nruns, solo = g_solo_clusters[sh->logx][sh->logy][diff ? 1 : 0];
    // solo > 0: the one-CTA-per-SM shared-memory size is set for this shape
    const bool can = solo > 0 && nch >= 2 && G.g.ns >= nch - 1;
    // EPD_LB_CHAIN_SCHEDULE=single|phased forces a schedule (the results are
    // the same either way), e.g. to time one against the other
    const char *env = std::getenv("EPD_LB_CHAIN_SCHEDULE");
    if (env && !std::strcmp(env, "single")) return 1;
    if (env && !std::strcmp(env, "phased")) return can ? nch : 1;
    return (can && nch == solo + 1) ? nch : 1;
}

size_t cluster_state_floats2(int nx, int ny, int ns) { return (size_t)2 * (ns + 1) * (ny / 2) * nx; }

int cluster_ctas(const Group &G)
{
    const ClusterShape *sh = find_shape(G.g.logx, G.g.logy);
    return sh ? sh->c : 0;
}

cudaError_t launch_selftest_wait(int *err, long long limit_cycles, cudaStream_t s)
{
    selftest_wait<<<1, 32, 0, s>>>(err, limit_cycles);
    return cudaGetLastError();
}

cudaError_t launch_cluster_solve(Group &G, cudaStream_t s, bool diff, int nprep_blocks, double *phi, double *q,
                                 const SolveProbe *probe, const double *phi_ref, const double *q_ref)
{
    const ClusterShape *sh = find_shape(G.g.logx, G.g.logy);
    if (!sh || !G.hc || (diff && !G.hd)) return cudaErrorInvalidValue;
    PropCK k;
    k.g = G.g;
    k.hout = reinterpret_cast<float2 *>(diff ? G.hd : G.hc);
    k.href = reinterpret_cast<const float2 *>(G.hc);
    k.efac = reinterpret_cast<const float2 *>(G.efac);
    k.rho = reinterpret_cast<const float2 *>(G.rho);
    k.cdiff = reinterpret_cast<const float2 *>(G.cdiff);
    k.err = G.err;
    k.twx = sh->mrx == 4 ? G.tab16x : G.tab8x;
    k.twy = sh->mry == 4 ? G.tab16y : G.tab8y;
    if (!k.twx || !k.twy) return cudaErrorInvalidValue;
    k.kx = reinterpret_cast<const float *>(G.kx);
    k.ky = reinterpret_cast<const float *>(G.ky);
    // One launch runs every chain, unless the chains are one more than the
    // clusters that fit at one CTA per SM: then the extra cluster would share
    // SMs with another and pace the launch, so nch launches of nch - 1
    // clusters at one CTA per SM take the chains in turns (chain j sits out
    // launch j and runs N_s / (nch - 1) steps in each of the others).
    const int nch = 2 * G.g.nruns, launches = cluster_chain_launches(G, diff);
    const bool phased = launches > 1;
    k.nseg = phased ? nch - 1 : 0;
    k.skip = 0;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr;
    set_cluster_cfg(cfg, attr, sh, phased ? nch - 1 : nch, diff);
    if (phased) cfg.dynamicSmemBytes = std::max(kSoloSmem, cfg.dynamicSmemBytes);
    cfg.stream = s;
    if (probe) {
        probe->cluster = true;
        cudaEventRecordWithFlags(probe->ev[0], s, cudaEventRecordExternal);
    }
    void *args[] = {&k};
    // launches after the first of a phased schedule are programmatic
    // dependents of the one before: their prologue (tables, node factors)
    // overlaps its end; they wait for it before reading the stored states
    cudaLaunchAttribute attrs[2] = {attr, {}};
    attrs[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attrs[1].val.programmaticStreamSerializationAllowed = 1;
    for (int p = 0; p < launches; ++p) {
        k.skip = p;
        cudaLaunchConfig_t c2 = cfg;
        if (p > 0 && g_chain_pdl) {
            c2.attrs = attrs;
            c2.numAttrs = 2;
        }
        cudaError_t e = cudaLaunchKernelExC(&c2, chain_fn(sh, diff), args);
        if (e != cudaSuccess) return e;
    }
    if (probe) cudaEventRecordWithFlags(probe->ev[1], s, cudaEventRecordExternal);

    ContourK c;
    c.g = G.g;
    c.hn = G.g.ny / 2 * G.g.nx;
    c.nq = kQBlocks;
    c.ns_part = nprep_blocks;
    c.hc = reinterpret_cast<const float2 *>(G.hc);
    c.hd = reinterpret_cast<const float2 *>(G.hd);
    c.efac = reinterpret_cast<const float2 *>(G.efac);
    c.rho = reinterpret_cast<const float2 *>(G.rho);
    c.part = G.part;
    c.phi_t = phi_ref ? phi_ref : G.phi_t;
    c.q_t = q_ref ? q_ref : G.q_t;
    c.phi = phi;
    c.q = q;
    c.err = G.err;
    const int npk = G.g.nx * G.g.ny / 2;
    const dim3 grid((npk + kThreads - 1) / kThreads, G.g.nruns), gq(kQBlocks, G.g.nruns);
    static std::atomic<bool> conf{false};  // attribute set (idempotent if two threads race)
    if (!conf) {
        cudaError_t e1 = cudaFuncSetAttribute(prop_contour<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)ContourStage<true>::SMEM);
        cudaError_t e2 = cudaFuncSetAttribute(prop_contour<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)ContourStage<false>::SMEM);
        if (e1 || e2) return e1 ? e1 : e2;
        conf = true;
    }
    if (diff) {
        prop_qsum<true><<<gq, kThreads, 0, s>>>(c);
        prop_contour<true><<<grid, kThreads, ContourStage<true>::SMEM, s>>>(c);
    } else {
        prop_qsum<false><<<gq, kThreads, 0, s>>>(c);
        prop_contour<false><<<grid, kThreads, ContourStage<false>::SMEM, s>>>(c);
    }
    return cudaGetLastError();
}

} // namespace epdlb

// surrogate.cu -- learned stand-in for the single-chain solve (a small
// convolutional network from the fields omega to the polymer densities) with
// BF16 tensor-core training and inference kernels, FP32 accumulation.
//
// Network (periodic grid, 3x3 kernels of dilation d_l = 1, 2, 2, 4, circular
// padding; receptive field +-9 sites, the range of the single-chain density
// response at R_G = 3 sites):
//   x0 = s_in (omega_c - <omega_c>), c = A, B, S          (3 channels)
//   y_l = tanh(W_l *_{d_l} y_{l-1} + b_l), l = 1, 2, 3    (32 channels)
//   y_4 = W_4 *_{d_4} y_3 + b_4                           (2 channels)
//   Phi_A = <Phi_A> + s_out (y_4,0 - <y_4,0>), Phi_B likewise with y_4,1, where
//   <Phi_A> = phi_p N_A/N_s and <Phi_B> = phi_p (1 - N_A/N_s) are the exact
//   means (Sec. 2, Eqs. (9)-(10) conserve them); Phi_S is the exact local
//   expression of Eq. (11).
//
// Every convolution is an implicit GEMM with BF16 operands and FP32
// accumulation on activations stored NHWC in BF16 (channels padded to a
// multiple of 16).  The forward layers, the input gradient (the same
// convolution of the output gradient with flipped, transposed weights) and
// the tangent pass run on tcgen05 (conv3x3_tc: 16 x 8 pixel tiles, M = 128,
// the accumulator in TMEM, halo tiles streamed in by TMA three deep); the
// weight gradient, a GEMM over pixels per tap, runs on mma.sync m16n8k16
// (conv3x3_dw).  Rounding to BF16 happens
// where the tensor cores read: weights, activations and the output
// gradients.
//
// Tangent pass: the change of Phi_A, Phi_B for a small field change domega
// at omega is the network's directional derivative (forward mode):
// dx0 = s_in (domega_c - <domega_c>), dy_l = (1 - y_l^2) (W_l *_{d_l}
// dy_{l-1}), dy_4 = W_4 *_{d_4} dy_3, dPhi_c = s_out (dy_4,c - <dy_4,c>).
// The time stepper takes Phi(t+dt) = Phi~ + dPhi this way: two separate
// forward passes at omega~ and omega(t+dt), whose inputs differ by far less
// than a BF16 step, would not resolve the change that drives the force.
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "engine.h"
#include "surrogate.h"

namespace epdlb {

// periodic index of a halo pixel (v in [-n, 2n)) on an axis of n pixels
__device__ __forceinline__ int halo_wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
namespace sur {

constexpr int TH = 8, TW = 16, TP = TH * TW;  // pixel tile
// halo tile of a 3x3 kernel of dilation D: D pixels on each side
template <int D> struct Halo {
    static constexpr int HH = TH + 2 * D, HW = TW + 2 * D;
};

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b)
{
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Epilogue modes of the convolution: tanh layer, linear layer, input
// gradient (times 1 - y^2 of the layer below, FP32), tangent (times 1 - y^2
// of this layer's BF16 output)
enum { EP_TANH = 0, EP_LINEAR = 1, EP_DX = 2, EP_JVP = 3 };

struct ConvArgs {
    const __nv_bfloat16 *in;    // [b][y][x][KP] (KP = input channels, padded)
    const __nv_bfloat16 *w;     // [tap][NP][KP]
    const float *bias;          // [NP] (EP_TANH, EP_LINEAR) or null
    __nv_bfloat16 *out_bf;      // [b][y][x][NP] BF16 output (EP_TANH, EP_DX)
    float *out_f;               // [b][y][x][NP] FP32 output (EP_TANH when training, EP_LINEAR)
    const float *yprev;         // EP_DX: tanh output of the layer below, [b][y][x][NP] FP32
    const __nv_bfloat16 *ycur;  // EP_JVP: this layer's tanh output, [b][y][x][NP] BF16
    int *err;                   // bit 2: a bounded wait of the tensor-core kernel gave up
    int use_tma;                // interior tiles by TMA (the tensor map encodes `in`)
    int nx, ny, logx, logy, nb;
    int nreal;                  // output channels actually used (the rest are written as 0)
};

// ---------------------------------------------------------------------------
// Convolution on the 5th-generation tensor cores (tcgen05, TMEM): forward
// layers, input gradients and the tangent pass.
//
// A CTA of 4 warps computes 16 x 8 pixel tiles (M = 128 rows of the
// implicit GEMM) for all output channels (N = 32, or 16 for the output
// layer's 8 stored channels), K = 9 taps x the input channels in steps of 16,
// looping over tiles with the next two tiles' halos in flight (TMA boxes for
// tiles inside the grid, periodic per-pixel copies on the border).
// Operands are read by the tensor cores from shared memory in the canonical
// K-major layout without swizzle: core matrices of 8 rows x 16 bytes (8
// channels), the halo tile stored as one plane per 8 input channels
// ([c8][halo pixel][8 channels]), so that for tap (dy, dx) the 8 pixels of an
// output row are one core matrix and consecutive output rows are a halo row
// apart (stride-byte offset), consecutive channel planes a plane apart
// (leading-byte offset); the weights as [tap][c8][co][8 channels].  One
// thread issues the 9 KP / 16 MMAs into a TMEM accumulator (32 columns) and
// commits them to an mbarrier; every warp then reads its 32 TMEM lanes (one
// pixel per thread, all channels) for the epilogue of the layer's mode.  Two
// accumulators alternate between tiles, so the next tile's MMAs run during
// this tile's epilogue.
// ---------------------------------------------------------------------------

constexpr int TCH = 16, TCW = 8;  // tensor-core pixel tile (rows x columns)
template <int D> struct HaloTC {
    static constexpr int HH = TCH + 2 * D, HW = TCW + 2 * D;
};

// Shared memory of the tcgen05 convolution: NBUF halo tiles (the one the
// MMAs read and the next ones, in flight), then the weights.  A halo tile
// is one plane per 8 input channels, each plane [HH][HW][8 channels] (the
// box of one TMA load), padded to 128 bytes.
template <int KP, int NP, int D> struct ConvTC {
    static constexpr int N = NP < 16 ? 16 : NP;  // MMA N (multiple of 16 for M = 128)
    static constexpr int C8 = KP / 8;
    static constexpr int HW16 = HaloTC<D>::HW * 16;
    static constexpr int PLANE_USED = HaloTC<D>::HH * HW16;
    static constexpr int PLANE = (PLANE_USED + 127) / 128 * 128;  // bytes per 8-channel plane
    static constexpr int HALO = C8 * PLANE, WB = 9 * C8 * N * 16;
    static constexpr int NBUF = 3;
    // the furthest byte a descriptor walk reaches (16 core matrices along M,
    // 2 along K) lies inside the halo tile
    static_assert((KP / 16 - 1) * 2 * PLANE + (2 * D * HaloTC<D>::HW + 2 * D) * 16 + 15 * HW16 + PLANE + 128 <= HALO,
                  "A operand walk inside the halo tile");
    static constexpr int AOFF = (NBUF * HALO + 1023) / 1024 * 1024;
    static constexpr size_t SMEM = (size_t)AOFF + WB + 128;  // + alignment slack of the base
};

// Shared-memory matrix descriptor: start, leading-byte offset (between core
// matrices along K), stride-byte offset (along M or N), all >> 4; bit 46 the
// descriptor version of this architecture; no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t mma_idesc(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}


// Bounded wait for the phase with the given parity of a CTA-local mbarrier
// (about 2^28 cycles); sets failed on giving up.
__device__ __forceinline__ void mbar_wait_tc(uint32_t bar, unsigned parity, int &failed)
{
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (ok) return;
        if (clock64() - t0 > (1ll << 28)) {
            failed = 1;
            return;
        }
    }
}

// N FP32 accumulator columns of this thread's TMEM lane (32x32b shape: warp w
// reads lanes 32 w .. 32 w + 31 of the address' lane field).
template <int N> __device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[N]);
template <> __device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
                   "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
template <> __device__ __forceinline__ void tmem_ld<32>(uint32_t taddr, float (&v)[32])
{
    float lo[16], hi[16];
    tmem_ld<16>(taddr, lo);
    tmem_ld<16>(taddr + 16, hi);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        v[i] = lo[i];
        v[16 + i] = hi[i];
    }
}

// tanh(x) = 1 - 2 / (exp(2x) + 1), with |x| clamped at 15 (tanh(15) rounds
// to 1 in FP32); absolute error a few 1e-7, below the BF16 step of the
// stored activations
__device__ __forceinline__ float tanh_fast(float x)
{
    x = fminf(fmaxf(x, -15.f), 15.f);
    return 1.f - __fdividef(2.f, __expf(2.f * x) + 1.f);
}
// the hardware tanh approximation (one special-function instruction;
// relative error about 2^-11, below the BF16 step of the stored result)
__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Bounded wait for the phase with the given parity of a CTA-local mbarrier
// in the tile pipeline: as mbar_wait_tc.
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// TMA load of one box of a 4D tensor map into shared memory, completing
// its bytes on the mbarrier
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1, int c2, int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

// Tile pipeline: NBUF halo buffers, each with a "full" mbarrier that all
// 128 threads arrive on once per tile.  A tile whose halo lies inside the
// grid is loaded by TMA (thread 0 arrives with the expected bytes, one box
// per 8-channel plane; the others arrive plainly); a tile on the border,
// whose halo wraps periodically, by per-pixel asynchronous copies whose
// completion each thread hands to the barrier (cp.async.mbarrier.arrive).
// The MMAs of tile i read buffer i % NBUF while tiles i + 1 .. i + NBUF - 1
// stream in.
template <int KP, int NP, int MODE, int D>
__global__ void __launch_bounds__(128) conv3x3_tc(ConvArgs a, const __grid_constant__ CUtensorMap tmap)
{
    using Geo = ConvTC<KP, NP, D>;
    constexpr int HH = HaloTC<D>::HH, HW = HaloTC<D>::HW, C8 = Geo::C8, N = Geo::N, NBUF = Geo::NBUF;
    static_assert(NP % 8 == 0, "epilogue in groups of 8 channels");
    extern __shared__ __align__(128) unsigned char tc_raw[];
    // base rounded up to 128 bytes (TMA destinations)
    unsigned char *halo = tc_raw + ((128u - ((uint32_t)__cvta_generic_to_shared(tc_raw) & 127u)) & 127u);  // [buffer][c8][HH*HW][16 B]
    unsigned char *wsm = halo + Geo::AOFF;      // [tap][c8][N][16 B]
    __shared__ __align__(8) unsigned long long mbar[2], full[NBUF];  // MMA barriers (one per accumulator), load barriers
    __shared__ uint32_t tmem_base;
    __shared__ float bias_s[NP];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long n = (long long)a.nx * a.ny;
    const uint32_t mbar_s = (uint32_t)__cvta_generic_to_shared(&mbar[0]);
    const uint32_t full_s = (uint32_t)__cvta_generic_to_shared(&full[0]);
    const uint32_t halo_s = (uint32_t)__cvta_generic_to_shared(halo), w_s = (uint32_t)__cvta_generic_to_shared(wsm);
    const int tiles_x = a.nx / TCW, tiles_img = tiles_x * (a.ny / TCH), ntiles = tiles_img * a.nb;
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_s + 8 * i) : "memory");
        for (int i = 0; i < NBUF; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(full_s + 8 * i) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    unsigned pending = 0;  // buffers with a load issued and not yet waited on (bit per buffer)
    auto issue = [&](int tix, int buf) {
        pending |= 1u << buf;
        const int b = tix / tiles_img, rr = tix % tiles_img;
        const int tx0 = (rr % tiles_x) * TCW, ty0 = (rr / tiles_x) * TCH;
        const uint32_t fb = full_s + 8 * buf, dst = halo_s + (uint32_t)(buf * Geo::HALO);
        const bool inside = a.use_tma && tx0 >= D && tx0 + TCW + D <= a.nx && ty0 >= D && ty0 + TCH + D <= a.ny;
        if (inside) {
            if (tid == 0) {
                mbar_arrive_tx(fb, (uint32_t)(C8 * Geo::PLANE_USED));
#pragma unroll
                for (int c8 = 0; c8 < C8; ++c8) tma_load_4d(dst + c8 * Geo::PLANE, &tmap, fb, c8 * 8, tx0 - D, ty0 - D, b);
            } else {
                mbar_arrive(fb);
            }
        } else {
            const __nv_bfloat16 *in = a.in + (size_t)b * n * KP;
            unsigned char *d = halo + (size_t)buf * Geo::HALO;
            for (int pix = tid; pix < HH * HW; pix += 128) {
                const int hy = pix / HW, hx = pix % HW;
                const int gy = halo_wrap(ty0 + hy - D, a.ny), gx = halo_wrap(tx0 + hx - D, a.nx);
                const __nv_bfloat16 *src = in + ((size_t)gy * a.nx + gx) * KP;
#pragma unroll
                for (int c8 = 0; c8 < C8; ++c8) cp_async16(d + (size_t)c8 * Geo::PLANE + (size_t)pix * 16, src + c8 * 8);
            }
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(fb) : "memory");
        }
    };
    for (int i = 0; i < NBUF - 1; ++i)
        if (blockIdx.x + i * (int)gridDim.x < ntiles) issue(blockIdx.x + i * gridDim.x, i);
    // weights once per CTA: row co (zero beyond NP), 8 channels per 16 bytes
    for (int e = tid; e < 9 * C8 * N; e += 128) {
        const int tap = e / (C8 * N), c8 = (e / N) % C8, co = e % N;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (co < NP) v = *reinterpret_cast<const uint4 *>(&a.w[((size_t)tap * NP + co) * KP + c8 * 8]);
        *reinterpret_cast<uint4 *>(wsm + ((size_t)(tap * C8 + c8) * N + co) * 16) = v;
    }
    if (tid < NP) bias_s[tid] = (MODE != EP_DX && MODE != EP_JVP && a.bias && tid < a.nreal) ? a.bias[tid] : 0.f;
    if (warp == 0) {
        // two accumulators of 32 FP32 columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the weights, for the tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    constexpr uint32_t IDESC = mma_idesc(128, N);
    // fphase: full-barrier parities (bit per buffer); mphase: MMA-barrier
    // parities (bit per accumulator); mpend: accumulators with MMAs issued
    // and not yet waited on
    unsigned fphase = 0, mphase = 0, mpend = 0;
    int failed = 0;
    const int G = (int)gridDim.x;
    // the MMAs of tile tix (buffer bf) into accumulator ac: wait for its
    // halo, make the copies visible to the tensor cores, one thread issues
    // 9 KP / 16 MMAs and commits them to the accumulator's barrier
    auto mma_tile = [&](int bf, int ac) {
        int f = 0;
        mbar_wait_tc(full_s + 8 * bf, (fphase >> bf) & 1u, f);
        if (__syncthreads_or(f)) return false;
        fphase ^= 1u << bf;
        pending &= ~(1u << bf);
        // asynchronous-copy writes visible to the tensor cores (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t hb = halo_s + (uint32_t)(bf * Geo::HALO), d = tmem + 32u * ac;
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const int dy = (tap / 3) * D, dx = (tap % 3) * D;
#pragma unroll
                for (int kc = 0; kc < KP / 16; ++kc) {
                    const uint64_t ad = smem_desc(hb + 2 * kc * Geo::PLANE + (uint32_t)(dy * HW + dx) * 16, Geo::PLANE, HW * 16);
                    const uint64_t bd = smem_desc(w_s + (uint32_t)((tap * C8 + 2 * kc) * N * 16), N * 16, 128);
                    const uint32_t acc = (tap | kc) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                        "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_s + 8 * ac)
                         : "memory");
        }
        mpend |= 1u << ac;
        return true;
    };
    // Tile i: buffer i % NBUF, accumulator i % 2.  Its MMAs are issued one
    // iteration ahead, so the tensor cores work on tile i + 1 while the
    // threads run tile i's epilogue; the loads run NBUF - 1 tiles ahead.
    if (blockIdx.x < ntiles && !mma_tile(0, 0)) failed = 1;
    int buf = 0, i = 0;
    for (int tix = blockIdx.x; tix < ntiles && !failed; tix += G, ++i, buf = buf + 1 == NBUF ? 0 : buf + 1) {
        const int ac = i & 1;
        const int b = tix / tiles_img, rr = tix % tiles_img;
        const int tx0 = (rr % tiles_x) * TCW, ty0 = (rr / tiles_x) * TCH;
        // loads of tile i + NBUF - 1 into the buffer tile i - 1's MMAs read
        // (complete: waited on in the previous iteration)
        if (tix + (NBUF - 1) * G < ntiles) issue(tix + (NBUF - 1) * G, buf == 0 ? NBUF - 1 : buf - 1);
        // MMAs of tile i + 1 into the other accumulator (read out by tile
        // i - 1's epilogue, which every thread finished)
        if (tix + G < ntiles && !mma_tile(buf + 1 == NBUF ? 0 : buf + 1, ac ^ 1)) {
            failed = 1;
            break;
        }
        // tile i's MMAs are done (bounded wait; the CTA leaves the tile loop
        // together if any thread gave up)
        {
            int f = 0;
            mbar_wait_tc(mbar_s + 8 * ac, (mphase >> ac) & 1u, f);
            if (__syncthreads_or(f)) {
                failed = 1;
                break;
            }
            mphase ^= 1u << ac;
            mpend &= ~(1u << ac);
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        {
            // thread = TMEM lane = pixel p (row p / 8, column p % 8) of the tile
            float v[N];
            const uint32_t taddr = tmem + 32u * ac + ((uint32_t)(32 * warp) << 16);
            tmem_ld<N>(taddr, v);
            const int p = 32 * warp + lane, py = ty0 + p / TCW, px = tx0 + p % TCW;
            const size_t pix = (size_t)b * n + (size_t)py * a.nx + px;
            // inference (BF16 output only): one-instruction tanh; training
            // keeps the FP32 activations for the gradient and forms tanh
            // from exp
            const bool fast = a.out_f == nullptr;
#pragma unroll
            for (int c0 = 0; c0 < NP; c0 += 8) {
                float o[8];
                if (MODE == EP_DX) {
                    const float4 y0 = *reinterpret_cast<const float4 *>(&a.yprev[pix * NP + c0]);
                    const float4 y1 = *reinterpret_cast<const float4 *>(&a.yprev[pix * NP + c0 + 4]);
                    const float yp[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
                    for (int j = 0; j < 8; ++j) o[j] = v[c0 + j] * (1.f - yp[j] * yp[j]);
                } else if (MODE == EP_JVP) {
                    const uint4 yv = *reinterpret_cast<const uint4 *>(&a.ycur[pix * NP + c0]);
                    const uint32_t w4[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float y = __uint_as_float(j & 1 ? (w4[j >> 1] & 0xFFFF0000u) : (w4[j >> 1] << 16));
                        o[j] = v[c0 + j] * (1.f - y * y);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float z = v[c0 + j] + bias_s[c0 + j];
                        o[j] = MODE == EP_TANH ? (fast ? tanh_approx(z) : tanh_fast(z)) : z;
                    }
                }
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (c0 + j >= a.nreal) o[j] = 0.f;
                if (a.out_bf) {
                    uint4 pk;
                    pk.x = pack2(__float2bfloat16_rn(o[0]), __float2bfloat16_rn(o[1]));
                    pk.y = pack2(__float2bfloat16_rn(o[2]), __float2bfloat16_rn(o[3]));
                    pk.z = pack2(__float2bfloat16_rn(o[4]), __float2bfloat16_rn(o[5]));
                    pk.w = pack2(__float2bfloat16_rn(o[6]), __float2bfloat16_rn(o[7]));
                    *reinterpret_cast<uint4 *>(&a.out_bf[pix * NP + c0]) = pk;
                }
                if (a.out_f) {
                    *reinterpret_cast<float4 *>(&a.out_f[pix * NP + c0]) = make_float4(o[0], o[1], o[2], o[3]);
                    *reinterpret_cast<float4 *>(&a.out_f[pix * NP + c0 + 4]) = make_float4(o[4], o[5], o[6], o[7]);
                }
            }
        }
        // every thread has read accumulator ac (tile i + 2's MMAs may
        // overwrite it) and tile i's buffer is free (its MMAs are done)
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (failed) {
        if (tid == 0 && a.err) atomicOr(a.err, 4);
        // MMAs still in flight, and the loads issued ahead into this CTA's
        // shared memory: wait for them once more (bounded)
        int f = 0;
        for (int c = 0; c < 2; ++c)
            if (mpend >> c & 1u) mbar_wait_tc(mbar_s + 8 * c, (mphase >> c) & 1u, f);
        for (int c = 0; c < NBUF; ++c)
            if (pending >> c & 1u) mbar_wait_tc(full_s + 8 * c, (fphase >> c) & 1u, f);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
}


// Weight gradient of one layer: dW[tap][co][ci] = sum_p dZ[p][co] x[p + off(tap)][ci]
// over an 8 x 16 tile per step, `tiles` consecutive tiles per CTA; 9 warps, warp
// = tap.  Partial sums per CTA to part[blk][tap][co][ci] (deterministic
// reduction later).  CO, CI multiples of 16 and 8.
template <int CI, int CO, int D>
__global__ void __launch_bounds__(288) conv3x3_dw(const __nv_bfloat16 *x, const __nv_bfloat16 *dz, float *part, int nx, int ny,
                                                 int tiles_x, int tiles_per_cta, int ntiles_total)
{
    constexpr int CS = CI + 8, DS = TP + 8;
    constexpr int HH = Halo<D>::HH, HW = Halo<D>::HW;
    __shared__ __align__(16) __nv_bfloat16 tile[HH * HW * CS];
    __shared__ __align__(16) __nv_bfloat16 dzt[CO * DS];  // [co][p], transposed
    const int tid = threadIdx.x, lane = tid & 31, tap = tid >> 5;
    const int g = lane >> 2, t = lane & 3, dy = (tap / 3) * D, dx = (tap % 3) * D;
    const long long n = (long long)nx * ny;
    float acc[CO / 16][CI / 8][4];
#pragma unroll
    for (int mt = 0; mt < CO / 16; ++mt)
#pragma unroll
        for (int nt = 0; nt < CI / 8; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[mt][nt][i] = 0.f;
    const int tiles_per_img = tiles_x * (ny / TH);
    for (int it = 0; it < tiles_per_cta; ++it) {
        const int tidx = blockIdx.x * tiles_per_cta + it;
        if (tidx >= ntiles_total) break;
        const int b = tidx / tiles_per_img, r = tidx % tiles_per_img;
        const int ty0 = (r / tiles_x) * TH, tx0 = (r % tiles_x) * TW;
        const __nv_bfloat16 *xin = x + (size_t)b * n * CI;
        const __nv_bfloat16 *dzin = dz + (size_t)b * n * CO;
        __syncthreads();
        for (int e = tid; e < HH * HW * (CI / 8); e += 288) {
            const int pix = e / (CI / 8), ch = (e % (CI / 8)) * 8;
            const int hy = pix / HW, hx = pix % HW;
            const int gy = halo_wrap(ty0 + hy - D, ny), gx = halo_wrap(tx0 + hx - D, nx);
            *reinterpret_cast<uint4 *>(&tile[pix * CS + ch]) = *reinterpret_cast<const uint4 *>(&xin[((size_t)gy * nx + gx) * CI + ch]);
        }
        for (int e = tid; e < TP * CO; e += 288) {
            const int p = e / CO, co = e % CO;
            const int gy = ty0 + p / TW, gx = tx0 + p % TW;
            dzt[co * DS + p] = dzin[((size_t)gy * nx + gx) * CO + co];
        }
        __syncthreads();
#pragma unroll
        for (int kc = 0; kc < TP / 16; ++kc) {  // 16 pixels = one tile row
            const int py = kc;
            uint32_t af[CO / 16][4];
#pragma unroll
            for (int mt = 0; mt < CO / 16; ++mt) {
                const int r0 = (mt * 16 + g) * DS + kc * 16 + 2 * t, r1 = r0 + 8 * DS;
                af[mt][0] = *reinterpret_cast<const uint32_t *>(&dzt[r0]);
                af[mt][1] = *reinterpret_cast<const uint32_t *>(&dzt[r1]);
                af[mt][2] = *reinterpret_cast<const uint32_t *>(&dzt[r0 + 8]);
                af[mt][3] = *reinterpret_cast<const uint32_t *>(&dzt[r1 + 8]);
            }
#pragma unroll
            for (int nt = 0; nt < CI / 8; ++nt) {
                const int ci = nt * 8 + g;
                const int k0 = 2 * t, k1 = 2 * t + 8;  // pixel columns in the row
                const __nv_bfloat16 *row = &tile[((py + dy) * HW + dx) * CS + ci];
                uint32_t bf[2];
                bf[0] = pack2(row[(k0)*CS], row[(k0 + 1) * CS]);
                bf[1] = pack2(row[(k1)*CS], row[(k1 + 1) * CS]);
#pragma unroll
                for (int mt = 0; mt < CO / 16; ++mt) mma16816(acc[mt][nt], af[mt], bf);
            }
        }
    }
    float *out = part + (size_t)blockIdx.x * 9 * CO * CI + (size_t)tap * CO * CI;
#pragma unroll
    for (int mt = 0; mt < CO / 16; ++mt)
#pragma unroll
        for (int nt = 0; nt < CI / 8; ++nt) {
            const int co = mt * 16 + g, ci = nt * 8 + 2 * t;
            out[co * CI + ci] = acc[mt][nt][0];
            out[co * CI + ci + 1] = acc[mt][nt][1];
            out[(co + 8) * CI + ci] = acc[mt][nt][2];
            out[(co + 8) * CI + ci + 1] = acc[mt][nt][3];
        }
}

// ---------------------------------------------------------------------------
// small kernels: input preparation, output, loss, reductions, optimiser
// ---------------------------------------------------------------------------

constexpr int kRedBlocks = 64;  // blocks per plane of the two-pass reductions

// Fixed-order sums over planes of n values in one launch, grid (kRedBlocks,
// planes): every block writes part[plane][block]; the last block to finish
// (a self-resetting counter) adds each plane's partials in block order and
// writes out[plane] = sum * scale.  KIND 0: the FP64 values, 1: exp(-v) in
// FP32 (solvent weight of Eq. (11)), 2: channel c = plane % 2 of the FP32
// [sample][pixel][8] network output.
__device__ __forceinline__ void finish_planes(const double *part, int planes, double scale, double *out, unsigned *cnt)
{
    __shared__ bool last;
    __threadfence();  // this block's partial before its arrival
    if (threadIdx.x == 0) {
        const unsigned total = gridDim.x * gridDim.y;
        last = atomicInc(cnt, total - 1) == total - 1;  // wraps to 0 for the next use
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int p = threadIdx.x; p < planes; p += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < kRedBlocks; ++b) s += part[(size_t)p * kRedBlocks + b];
        out[p] = s * scale;
    }
}

template <int KIND>
__global__ void __launch_bounds__(256) plane_partials(const void *f, long long n, double *part, double scale, double *out,
                                                      unsigned *cnt)
{
    __shared__ double red[32];
    const int plane = blockIdx.y;
    double s = 0.0;
    const long long chunk = (n + kRedBlocks - 1) / kRedBlocks, lo = blockIdx.x * chunk;
    const long long hi = lo + chunk < n ? lo + chunk : n;
    if (KIND == 0) {
        const double *p = reinterpret_cast<const double *>(f) + (size_t)plane * n;
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) s += p[i];
    } else if (KIND == 1) {
        const double *p = reinterpret_cast<const double *>(f) + ((size_t)plane * 3 + 2) * n;
        float acc = 0.f;
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += expf(-(float)p[i]);
        s = (double)acc;
    } else {
        const float *p = reinterpret_cast<const float *>(f) + (size_t)(plane / 2) * n * 8 + (plane % 2);
        float acc = 0.f;
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += p[(size_t)i * 8];
        s = (double)acc;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[(size_t)plane * kRedBlocks + blockIdx.x] = s;
    finish_planes(part, gridDim.y, scale, out, cnt);
}

// x0[b][p][16] = s_in (omega_c - <omega_c>) for c < 3, 0 for the padding.
__global__ void prep_input(const double *omega, const double *mean, double s_in, long long n, int nb, __nv_bfloat16 *x0)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * nb) return;
    const long long b = i / n, p = i % n;
    __align__(16) __nv_bfloat16 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(0.f);
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = __float2bfloat16_rn((float)(s_in * (omega[(b * 3 + c) * n + p] - mean[b * 3 + c])));
    uint4 *dst = reinterpret_cast<uint4 *>(x0 + (size_t)i * 16);
    dst[0] = *reinterpret_cast<uint4 *>(&v[0]);
    dst[1] = *reinterpret_cast<uint4 *>(&v[8]);
}

// Tangent input: dx0[b][p][16] = s_in ((omega_c - omega0_c) - <omega_c - omega0_c>)
// for c < 3 (the FP64 difference of the two fields, then BF16), 0 for the padding.
__global__ void prep_tangent(const double *omega, const double *omega0, const double *mean, const double *mean0, double s_in,
                             long long n, int nb, __nv_bfloat16 *t0)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * nb) return;
    const long long b = i / n, p = i % n;
    __align__(16) __nv_bfloat16 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(0.f);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const size_t q = (b * 3 + c) * n + p;
        v[c] = __float2bfloat16_rn((float)(s_in * ((omega[q] - omega0[q]) - (mean[b * 3 + c] - mean0[b * 3 + c]))));
    }
    uint4 *dst = reinterpret_cast<uint4 *>(t0 + (size_t)i * 16);
    dst[0] = *reinterpret_cast<uint4 *>(&v[0]);
    dst[1] = *reinterpret_cast<uint4 *>(&v[8]);
}

// Block partials of sum e q over one plane per sample, e = exp(-omega0_S),
// q = expm1(-(omega_S - omega0_S)) (FP32, accurate relative to the change).
__global__ void __launch_bounds__(256) solvent_change_partials(const double *omega, const double *omega0, long long n, double *part,
                                                               double scale, double *out, unsigned *cnt)
{
    __shared__ double red[32];
    const int b = blockIdx.y;
    const long long chunk = (n + kRedBlocks - 1) / kRedBlocks, lo = blockIdx.x * chunk;
    const long long hi = lo + chunk < n ? lo + chunk : n;
    const double *w = omega + ((size_t)b * 3 + 2) * n, *w0 = omega0 + ((size_t)b * 3 + 2) * n;
    float acc = 0.f;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x)
        acc += expf(-(float)w0[i]) * expm1f(-(float)(w[i] - w0[i]));
    const double s = block_sum((double)acc, red);
    if (threadIdx.x == 0) part[(size_t)b * kRedBlocks + blockIdx.x] = s;
    finish_planes(part, gridDim.y, scale, out, cnt);
}

// Densities after a field change: Phi_A, Phi_B = the densities at omega0
// plus s_out (dy4 - <dy4>) (the tangent output); Phi_S of Eq. (11) at omega
// as the densities at omega0 plus the exact change,
//   Phi_S = Phi0_S + Phi0_S (q - m) / (1 + m),  m = <e q> / <e>,
// every term of the size of the change (e, q as in solvent_change_partials).
__global__ void densities_tangent(const float *t4, const double *tmean, const double *phi0, const double *omega,
                                  const double *omega0, const double *e_mean, const double *eq_mean, double s_out, long long n,
                                  int nb, double *phi)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * nb) return;
    const long long b = i / n, p = i % n;
    const float2 y = *reinterpret_cast<const float2 *>(&t4[(size_t)i * 8]);
    phi[(b * 3 + 0) * n + p] = phi0[(b * 3 + 0) * n + p] + s_out * ((double)y.x - tmean[2 * b]);
    phi[(b * 3 + 1) * n + p] = phi0[(b * 3 + 1) * n + p] + s_out * ((double)y.y - tmean[2 * b + 1]);
    const size_t q = (b * 3 + 2) * n + p;
    const double dq = (double)expm1f(-(float)(omega[q] - omega0[q])), m = eq_mean[b] / e_mean[b];
    phi[q] = phi0[q] + phi0[q] * (dq - m) / (1.0 + m);
}

// Densities from the network output: Phi_A, Phi_B with exact means, Phi_S from
// Eq. (11) (exp(-w_S) in FP32, Q_S the per-sample mean of the same values).
__global__ void densities_out(const float *y4, const double *ymean, const double *omega, const double *qs_mean, double s_out,
                              double pa_bar, double pb_bar, double ps_bar, long long n, int nb, double *phi)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * nb) return;
    const long long b = i / n, p = i % n;
    const float2 y = *reinterpret_cast<const float2 *>(&y4[(size_t)i * 8]);
    phi[(b * 3 + 0) * n + p] = pa_bar + s_out * ((double)y.x - ymean[2 * b]);
    phi[(b * 3 + 1) * n + p] = pb_bar + s_out * ((double)y.y - ymean[2 * b + 1]);
    phi[(b * 3 + 2) * n + p] = ps_bar * (double)expf(-(float)omega[(b * 3 + 2) * n + p]) / qs_mean[b];
}

// Loss and output gradient: targets t_c = (Phi_c - <Phi_c>) / s_out for
// c = A, B; loss = mean over samples, channels, pixels of (y - t)^2; dZ4 =
// 2 (y - t) / count in BF16 ([b][p][16], channels >= 2 zero).  Per-block
// partial loss sums to lpart.
__global__ void __launch_bounds__(256) loss_grad(const float *y4, const double *phi_t, const double *tmean, double s_out, long long n,
                                                 int nb, __nv_bfloat16 *dz4, double *lpart)
{
    __shared__ double red[32];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < n * nb) {
        const long long b = i / n, p = i % n;
        const double cnt = 2.0 * (double)n * (double)nb;
        __align__(16) __nv_bfloat16 v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(0.f);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const double tc = (phi_t[(b * 3 + c) * n + p] - tmean[b * 3 + c]) / s_out;
            const double d = (double)y4[(size_t)i * 8 + c] - tc;
            l += d * d;
            v[c] = __float2bfloat16_rn((float)(2.0 * d / cnt));
        }
        uint4 *dst = reinterpret_cast<uint4 *>(dz4 + (size_t)i * 16);
        dst[0] = *reinterpret_cast<uint4 *>(&v[0]);
        dst[1] = *reinterpret_cast<uint4 *>(&v[8]);
    }
    l = block_sum(l, red);
    if (threadIdx.x == 0) lpart[blockIdx.x] = l;
}

// Sum of `cnt` per-block partials (fixed order) -> out[0] / denom.
__global__ void __launch_bounds__(256) sum_parts(const double *part, int cnt, double denom, double *out)
{
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) s += part[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[0] = s / denom;
}

// Reduce dW partials [nblk][9][CO][CI] into the gradient of the packed
// master parameters of one layer ([co][ci][tap]).  A block takes 32
// consecutive entries of a partial (ci fastest: coalesced) and 8 slices of
// the partials; the slices' FP64 sums are added in a fixed order.
constexpr int kDwSlices = 8;
constexpr int kBiasBlocks = 304;  // blocks of the bias-gradient partial sums (2 per SM)
__global__ void __launch_bounds__(256) reduce_dw(const float *part, int nblk, int co_real, int ci_real, int CO, int CI, float *gw)
{
    __shared__ double red[kDwSlices][32];
    const int e = blockIdx.x * 32 + (threadIdx.x & 31), sl = threadIdx.x >> 5;  // e over [tap][CO][CI]
    const int per = 9 * CO * CI;
    double s = 0.0;
    if (e < per)
        for (int b = sl; b < nblk; b += kDwSlices) s += (double)part[(size_t)b * per + e];
    red[sl][threadIdx.x & 31] = s;
    __syncthreads();
    if (sl == 0 && e < per) {
        double t = 0.0;
        for (int k = 0; k < kDwSlices; ++k) t += red[k][threadIdx.x];
        const int tap = e / (CO * CI), co = (e / CI) % CO, ci = e % CI;
        if (co < co_real && ci < ci_real) gw[((size_t)co * ci_real + ci) * 9 + tap] = (float)t;
    }
}

// Bias gradient dB[co] = sum over pixels of dZ[p][co] (CO = 16 or 32): each
// thread reads 8 channels of a pixel per load and keeps FP32 sums over its
// few pixels; FP64 block sums per channel to part[block][co], then
// bias_grad_finish adds the blocks in a fixed order.
__global__ void __launch_bounds__(256) bias_grad_part(const __nv_bfloat16 *dz, long long npix, int CO, double *part)
{
    __shared__ double red[256][8];
    const int c8n = CO / 8, g = threadIdx.x % c8n;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const long long stride = (long long)gridDim.x * (blockDim.x / c8n);
    for (long long p = (long long)blockIdx.x * (blockDim.x / c8n) + threadIdx.x / c8n; p < npix; p += stride) {
        const uint4 v = *reinterpret_cast<const uint4 *>(&dz[(size_t)p * CO + g * 8]);
        const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] += __uint_as_float(j & 1 ? (w4[j >> 1] & 0xFFFF0000u) : (w4[j >> 1] << 16));
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) red[threadIdx.x][j] = (double)acc[j];
    __syncthreads();
    if (threadIdx.x < CO) {
        const int c = threadIdx.x, gc = c / 8, j = c % 8;
        double t = 0.0;
        for (int k = gc; k < (int)blockDim.x; k += c8n) t += red[k][j];
        part[(size_t)blockIdx.x * CO + c] = t;
    }
}
// (one block of 256 threads: 8 slices of the blocks per channel, the
// slices' sums added in a fixed order)
__global__ void __launch_bounds__(256) bias_grad_finish(const double *part, int nblk, int CO, int co_real, float *gb)
{
    __shared__ double red[8][32];
    const int c = threadIdx.x & 31, sl = threadIdx.x >> 5;
    double t = 0.0;
    if (c < CO)
        for (int b = sl; b < nblk; b += 8) t += part[(size_t)b * CO + c];
    red[sl][c] = t;
    __syncthreads();
    if (sl == 0 && c < co_real) {
        double u = 0.0;
        for (int k = 0; k < 8; ++k) u += red[k][c];
        gb[c] = (float)u;
    }
}

// Adam on the FP32 master parameters (Kingma and Ba, 2015).
__global__ void adam(float *w, const float *gw, float *m, float *v, int np, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = gw[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Pack master weights [co][ci][tap] of one layer to the forward layout
// [tap][NP][KP] (BF16) and, if wb is given, the input-gradient layout
// [tap][KP2][NP2] = flipped taps, transposed channels.
__global__ void pack_weights(const float *wm, int co_real, int ci_real, int NP, int KP, __nv_bfloat16 *wf, __nv_bfloat16 *wb, int NPB,
                             int KPB)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int tot_f = 9 * NP * KP;
    if (i < tot_f) {
        const int tap = i / (NP * KP), co = (i / KP) % NP, ci = i % KP;
        const float v = (co < co_real && ci < ci_real) ? wm[((size_t)co * ci_real + ci) * 9 + tap] : 0.f;
        wf[i] = __float2bfloat16_rn(v);
    }
    if (wb && i < 9 * NPB * KPB) {
        // input-gradient conv: output channel = ci (< NPB), input channel = co (< KPB)
        const int tap = i / (NPB * KPB), ci = (i / KPB) % NPB, co = i % KPB;
        const int ftap = 8 - tap;
        const float v = (co < co_real && ci < ci_real) ? wm[((size_t)co * ci_real + ci) * 9 + ftap] : 0.f;
        wb[i] = __float2bfloat16_rn(v);
    }
}

} // namespace sur
} // namespace epdlb

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

namespace epdlb {
namespace sur {

// storage channels (padded) of each layer's input and output; dilations
static const int kKP[kLayers] = {16, 32, 32, 32};
static const int kNP[kLayers] = {32, 32, 32, 8};
constexpr int kD0 = 1, kD1 = 2, kD2 = 2, kD3 = 4;

int num_params()
{
    int s = 0;
    for (int l = 0; l < kLayers; ++l) s += kCout[l] * kCin[l] * 9 + kCout[l];
    return s;
}
int param_offset_w(int layer)
{
    int s = 0;
    for (int l = 0; l < layer; ++l) s += kCout[l] * kCin[l] * 9 + kCout[l];
    return s;
}
int param_offset_b(int layer) { return param_offset_w(layer) + kCout[layer] * kCin[layer] * 9; }

static size_t al(size_t v) { return (v + 255) & ~(size_t)255; }

size_t carve(Work &w, char *base, int nb, int ny, int nx, bool training)
{
    w.nb = nb;
    w.nx = nx;
    w.ny = ny;
    w.n = (long long)nx * ny;
    w.training = training;
    const size_t np = (size_t)nb * w.n;
    size_t off = 0;
    auto take = [&](size_t bytes) -> void * {
        off = al(off);
        void *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    {
        char *hdr = (char *)take(256);
        w.err = (int *)hdr;
        w.cnt = hdr ? (unsigned *)(hdr + 128) : nullptr;
    }
    w.x0 = take(np * 16 * 2);
    for (int l = 0; l < 3; ++l) w.y[l] = take(np * 32 * 2);
    w.y4 = take(np * 8 * 4);
    w.t0 = take(np * 16 * 2);
    w.t[0] = take(np * 32 * 2);
    w.t[1] = take(np * 32 * 2);
    w.t4 = take(np * 8 * 4);
    w.means2 = (double *)take((size_t)nb * 3 * sizeof(double));
    for (int l = 0; l < kLayers; ++l) w.wf[l] = take((size_t)9 * kNP[l] * kKP[l] * 2);
    w.means = (double *)take((size_t)nb * 3 * sizeof(double));
    w.ymean = (double *)take((size_t)nb * 2 * sizeof(double));
    w.qs = (double *)take((size_t)nb * sizeof(double));
    w.red = (double *)take((size_t)nb * 3 * kRedBlocks * sizeof(double));
    if (training) {
        for (int l = 0; l < 3; ++l) w.yf[l] = take(np * 32 * 4);
        w.dz[0] = take(np * 32 * 2);
        w.dz[1] = take(np * 32 * 2);
        w.dz4 = take(np * 16 * 2);
        for (int l = 1; l < kLayers; ++l) w.wb[l] = take((size_t)9 * 32 * kNP[l] * 2 + (size_t)9 * 32 * 16 * 2);
        const long long tiles = (long long)nb * (nx / TW) * (ny / TH);
        w.nblk_dw = (int)std::min<long long>(512, tiles);
        w.dwpart = (float *)take((size_t)w.nblk_dw * 9 * 32 * 32 * sizeof(float));
        w.grad = (float *)take((size_t)num_params() * sizeof(float));
        w.tmean = (double *)take((size_t)nb * 3 * sizeof(double));
        w.lpart = (double *)take((size_t)((np + 255) / 256 + 1) * sizeof(double));
        w.bpart = (double *)take((size_t)kBiasBlocks * 32 * sizeof(double));
    } else {
        for (int l = 0; l < 3; ++l) w.yf[l] = nullptr;
        w.dz[0] = w.dz[1] = w.dz4 = nullptr;
        for (int l = 0; l < kLayers; ++l) w.wb[l] = nullptr;
        w.dwpart = w.grad = nullptr;
        w.tmean = w.lpart = w.bpart = nullptr;
        w.nblk_dw = 0;
    }
    return al(off);
}

static unsigned blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Means over `planes` planes of n values (kind: see plane_partials).
static void plane_means(const Work &w, const void *f, int kind, int planes, double *out, cudaStream_t s)
{
    const dim3 g(kRedBlocks, planes);
    const double sc = 1.0 / (double)w.n;
    if (kind == 0) plane_partials<0><<<g, 256, 0, s>>>(f, w.n, w.red, sc, out, w.cnt);
    else if (kind == 1) plane_partials<1><<<g, 256, 0, s>>>(f, w.n, w.red, sc, out, w.cnt);
    else plane_partials<2><<<g, 256, 0, s>>>(f, w.n, w.red, sc, out, w.cnt);
}

static cudaError_t pack_all(Work &w, const float *params, bool backward, cudaStream_t s)
{
    for (int l = 0; l < kLayers; ++l) {
        const int tot_f = 9 * kNP[l] * kKP[l];
        // input-gradient weights: output channels = this layer's inputs (32),
        // input channels = this layer's outputs as stored (dZ: 32, or 16 for the last layer)
        const int npb = 32, kpb = (l == kLayers - 1) ? 16 : 32;
        const bool bw = backward && l > 0;
        const int tot = bw ? std::max(tot_f, 9 * npb * kpb) : tot_f;
        pack_weights<<<blocks(tot), 256, 0, s>>>(params + param_offset_w(l), kCout[l], kCin[l], kNP[l], kKP[l],
                                                 reinterpret_cast<__nv_bfloat16 *>(w.wf[l]),
                                                 bw ? reinterpret_cast<__nv_bfloat16 *>(w.wb[l]) : nullptr, npb, kpb);
    }
    return cudaGetLastError();
}

// The driver's tensor-map encoder, looked up once through the runtime.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Tensor map of a BF16 activation tensor [nb][ny][nx][kp] with boxes of 8
// channels x hw x hh pixels (one halo plane); false if none can be made
// (the convolution then loads every tile by asynchronous copies).
static bool halo_map(CUtensorMap *m, const void *base, int kp, int nx, int ny, int nb, int hw, int hh)
{
    std::memset(m, 0, sizeof *m);
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || ((uintptr_t)base & 15)) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)kp, (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nb};
    const cuuint64_t strides[3] = {(cuuint64_t)kp * 2, (cuuint64_t)nx * kp * 2, (cuuint64_t)nx * ny * kp * 2};
    const cuuint32_t box[4] = {8, (cuuint32_t)hw, (cuuint32_t)hh, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int KP, int NP, int MODE, int D>
static void conv(Work &w, const void *in, const void *wt, const float *bias, void *out_bf, float *out_f, const float *yprev, int nreal,
                 cudaStream_t s, const void *ycur = nullptr)
{
    constexpr size_t smem = ConvTC<KP, NP, D>::SMEM;
    static std::atomic<bool> conf{false};  // attribute set (idempotent if two threads race)
    if (!conf) {
        cudaFuncSetAttribute(conv3x3_tc<KP, NP, MODE, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        conf = true;
    }
    ConvArgs a;
    CUtensorMap map;
    a.use_tma = halo_map(&map, in, KP, w.nx, w.ny, w.nb, HaloTC<D>::HW, HaloTC<D>::HH) ? 1 : 0;
    a.ycur = reinterpret_cast<const __nv_bfloat16 *>(ycur);
    a.err = w.err;
    a.in = reinterpret_cast<const __nv_bfloat16 *>(in);
    a.w = reinterpret_cast<const __nv_bfloat16 *>(wt);
    a.bias = bias;
    a.out_bf = reinterpret_cast<__nv_bfloat16 *>(out_bf);
    a.out_f = out_f;
    a.yprev = yprev;
    a.nx = w.nx;
    a.ny = w.ny;
    a.logx = ilog2(w.nx);
    a.logy = ilog2(w.ny);
    a.nreal = nreal;
    a.nb = w.nb;
    const int tiles = w.nb * (w.nx / TCW) * (w.ny / TCH);
    // CTAs per SM: by shared memory, and at most 8 (64 TMEM columns each)
    const int per_sm = std::max(1, std::min(8, (int)((220u << 10) / (smem + 1024))));
    conv3x3_tc<KP, NP, MODE, D><<<std::min(tiles, per_sm * 152), 128, smem, s>>>(a, map);
}

static cudaError_t forward_layers(Work &w, const float *params, cudaStream_t s)
{
    const bool tr = w.training;
    conv<16, 32, EP_TANH, kD0>(w, w.x0, w.wf[0], params + param_offset_b(0), w.y[0], tr ? (float *)w.yf[0] : nullptr, nullptr, 32, s);
    conv<32, 32, EP_TANH, kD1>(w, w.y[0], w.wf[1], params + param_offset_b(1), w.y[1], tr ? (float *)w.yf[1] : nullptr, nullptr, 32, s);
    conv<32, 32, EP_TANH, kD2>(w, w.y[1], w.wf[2], params + param_offset_b(2), w.y[2], tr ? (float *)w.yf[2] : nullptr, nullptr, 32, s);
    conv<32, 8, EP_LINEAR, kD3>(w, w.y[2], w.wf[3], params + param_offset_b(3), nullptr, (float *)w.y4, nullptr, 2, s);
    return cudaGetLastError();
}

// zero the one-launch reductions' counter the first time a workspace is used
static cudaError_t ready_counter(Work &w, cudaStream_t s)
{
    if (w.cnt_ready) return cudaSuccess;
    const cudaError_t e = cudaMemsetAsync(w.cnt, 0, sizeof(unsigned), s);
    w.cnt_ready = e == cudaSuccess;
    return e;
}

cudaError_t prepare(Work &w, const float *params, cudaStream_t s)
{
    cudaError_t e;
    w.cnt_ready = false;
    if ((e = ready_counter(w, s))) return e;
    if ((e = pack_all(w, params, false, s))) return e;
    w.prepacked = true;
    return cudaSuccess;
}

cudaError_t forward(Work &w, const float *params, const double *omega, double *phi, double s_in, double s_out, double pa_bar,
                    double pb_bar, double ps_bar, cudaStream_t s)
{
    cudaError_t e;
    if ((e = ready_counter(w, s))) return e;
    if (!w.prepacked && (e = pack_all(w, params, false, s))) return e;
    plane_means(w, omega, 0, w.nb * 3, w.means, s);
    prep_input<<<blocks(w.n * w.nb), 256, 0, s>>>(omega, w.means, s_in, w.n, w.nb, reinterpret_cast<__nv_bfloat16 *>(w.x0));
    if ((e = forward_layers(w, params, s))) return e;
    plane_means(w, w.y4, 2, w.nb * 2, w.ymean, s);
    plane_means(w, omega, 1, w.nb, w.qs, s);
    densities_out<<<blocks(w.n * w.nb), 256, 0, s>>>((const float *)w.y4, w.ymean, omega, w.qs, s_out, pa_bar, pb_bar, ps_bar, w.n, w.nb,
                                                     phi);
    return cudaGetLastError();
}

cudaError_t tangent(Work &w, const float *params, const double *omega, const double *omega0, const double *phi0, double *phi,
                    double s_in, double s_out, double ps_bar, cudaStream_t s)
{
    // the forward pass at omega0 left in w its activations y_l (BF16), the
    // means of omega0 (w.means) and <exp(-omega0_S)> (w.qs)
    cudaError_t e;
    if ((e = ready_counter(w, s))) return e;
    plane_means(w, omega, 0, w.nb * 3, w.means2, s);
    prep_tangent<<<blocks(w.n * w.nb), 256, 0, s>>>(omega, omega0, w.means2, w.means, s_in, w.n, w.nb,
                                                    reinterpret_cast<__nv_bfloat16 *>(w.t0));
    conv<16, 32, EP_JVP, kD0>(w, w.t0, w.wf[0], nullptr, w.t[0], nullptr, nullptr, 32, s, w.y[0]);
    conv<32, 32, EP_JVP, kD1>(w, w.t[0], w.wf[1], nullptr, w.t[1], nullptr, nullptr, 32, s, w.y[1]);
    conv<32, 32, EP_JVP, kD2>(w, w.t[1], w.wf[2], nullptr, w.t[0], nullptr, nullptr, 32, s, w.y[2]);
    conv<32, 8, EP_LINEAR, kD3>(w, w.t[0], w.wf[3], nullptr, nullptr, (float *)w.t4, nullptr, 2, s);
    plane_means(w, w.t4, 2, w.nb * 2, w.ymean, s);
    // <e q> into means2 (free again); <e> at omega0 is in qs
    solvent_change_partials<<<dim3(kRedBlocks, w.nb), 256, 0, s>>>(omega, omega0, w.n, w.red, 1.0 / (double)w.n, w.means2, w.cnt);
    densities_tangent<<<blocks(w.n * w.nb), 256, 0, s>>>((const float *)w.t4, w.ymean, phi0, omega, omega0, w.qs, w.means2, s_out,
                                                         w.n, w.nb, phi);
    (void)ps_bar;
    return cudaGetLastError();
}

template <int CI, int CO, int D>
static void dw(Work &w, const void *x, const void *dzp, cudaStream_t s)
{
    const int tiles_x = w.nx / TW;
    const int ntiles = w.nb * tiles_x * (w.ny / TH);
    const int per = (ntiles + w.nblk_dw - 1) / w.nblk_dw;
    const int nblk = (ntiles + per - 1) / per;
    conv3x3_dw<CI, CO, D><<<nblk, 288, 0, s>>>(reinterpret_cast<const __nv_bfloat16 *>(x), reinterpret_cast<const __nv_bfloat16 *>(dzp),
                                            w.dwpart, w.nx, w.ny, tiles_x, per, ntiles);
    w.nblk_dw = nblk;
}

static void layer_grads(Work &w, int l, const void *x, const void *dzp, int CO, int CI, cudaStream_t s)
{
    const int ntiles_cap = w.nblk_dw;
    if (l == 0) dw<16, 32, kD0>(w, x, dzp, s);
    else if (l == 1) dw<32, 32, kD1>(w, x, dzp, s);
    else if (l == 2) dw<32, 32, kD2>(w, x, dzp, s);
    else dw<32, 16, kD3>(w, x, dzp, s);
    reduce_dw<<<(9 * CO * CI + 31) / 32, 256, 0, s>>>(w.dwpart, w.nblk_dw, kCout[l], kCin[l], CO, CI, w.grad + param_offset_w(l));
    bias_grad_part<<<kBiasBlocks, 256, 0, s>>>(reinterpret_cast<const __nv_bfloat16 *>(dzp), (long long)w.nb * w.n, CO, w.bpart);
    bias_grad_finish<<<1, 256, 0, s>>>(w.bpart, kBiasBlocks, CO, kCout[l], w.grad + param_offset_b(l));
    w.nblk_dw = ntiles_cap;
}

cudaError_t gradients(Work &w, const float *params, const double *omega, const double *phi_t, double s_in, double s_out,
                      double *loss_dev, cudaStream_t s)
{
    cudaError_t e;
    if ((e = ready_counter(w, s))) return e;
    if ((e = pack_all(w, params, true, s))) return e;
    plane_means(w, omega, 0, w.nb * 3, w.means, s);
    prep_input<<<blocks(w.n * w.nb), 256, 0, s>>>(omega, w.means, s_in, w.n, w.nb, reinterpret_cast<__nv_bfloat16 *>(w.x0));
    if ((e = forward_layers(w, params, s))) return e;
    plane_means(w, phi_t, 0, w.nb * 3, w.tmean, s);
    const unsigned lb = blocks(w.n * w.nb);
    loss_grad<<<lb, 256, 0, s>>>((const float *)w.y4, phi_t, w.tmean, s_out, w.n, w.nb, reinterpret_cast<__nv_bfloat16 *>(w.dz4),
                                 w.lpart);
    sum_parts<<<1, 256, 0, s>>>(w.lpart, (int)lb, 2.0 * (double)w.n * w.nb, loss_dev);
    // layer 4: dW from y3 and dZ4; dZ3 = (W4^T dZ4) (1 - y3^2)
    layer_grads(w, 3, w.y[2], w.dz4, 16, 32, s);
    conv<16, 32, EP_DX, kD3>(w, w.dz4, w.wb[3], nullptr, w.dz[0], nullptr, (const float *)w.yf[2], 32, s);
    // layer 3
    layer_grads(w, 2, w.y[1], w.dz[0], 32, 32, s);
    conv<32, 32, EP_DX, kD2>(w, w.dz[0], w.wb[2], nullptr, w.dz[1], nullptr, (const float *)w.yf[1], 32, s);
    // layer 2
    layer_grads(w, 1, w.y[0], w.dz[1], 32, 32, s);
    conv<32, 32, EP_DX, kD1>(w, w.dz[1], w.wb[1], nullptr, w.dz[0], nullptr, (const float *)w.yf[0], 32, s);
    // layer 1
    layer_grads(w, 0, w.x0, w.dz[0], 32, 16, s);
    return cudaGetLastError();
}

cudaError_t adam_step(Work &w, float *params, float *m, float *v, int step, float lr, cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - (float)std::pow((double)b1, (double)step), c2 = 1.f - (float)std::pow((double)b2, (double)step);
    const int np = num_params();
    adam<<<blocks(np), 256, 0, s>>>(params, w.grad, m, v, np, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) rms_diff(const double *a, const double *b, long long n3, double *out)
{
    __shared__ double red[32];
    const double *pa = a + (size_t)blockIdx.x * n3, *pb = b + (size_t)blockIdx.x * n3;
    double s = 0.0;
    for (long long i = threadIdx.x; i < n3; i += blockDim.x) {
        const double d = pa[i] - pb[i];
        s += d * d;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[blockIdx.x] = sqrt(s / (double)n3);
}

__global__ void max_of(const double *v, int cnt, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < cnt; ++i) m = v[i] > m ? v[i] : m;
        out[0] = m;
    }
}

cudaError_t residual_rms(const double *phi_a, const double *phi_b, long long n, int nb, double *tmp, double *out, cudaStream_t s)
{
    rms_diff<<<nb, 256, 0, s>>>(phi_a, phi_b, 3 * n, tmp);
    max_of<<<1, 32, 0, s>>>(tmp, nb, out);
    return cudaGetLastError();
}

// Per run (block): sqrt(sum_{c=A,B} |a_c - b_c|^2 / sum_{c=A,B} |b_c - <b_c>|^2).
__global__ void __launch_bounds__(256) rel_diff(const double *a, const double *b, long long n, double *out)
{
    __shared__ double red[32];
    const double *pa = a + (size_t)blockIdx.x * 3 * n, *pb = b + (size_t)blockIdx.x * 3 * n;
    double num = 0.0, den = 0.0;
    for (int c = 0; c < 2; ++c) {
        double s = 0.0, ss = 0.0, dd = 0.0;
        for (long long i = threadIdx.x; i < n; i += blockDim.x) {
            const double v = pb[c * n + i], d = pa[c * n + i] - v;
            s += v;
            ss += v * v;
            dd += d * d;
        }
        s = block_sum(s, red);
        ss = block_sum(ss, red);
        dd = block_sum(dd, red);
        num += dd;
        den += ss - s * s / (double)n;
    }
    if (threadIdx.x == 0) out[blockIdx.x] = den > 0.0 ? sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0);
}

cudaError_t residual_rel(const double *phi_a, const double *phi_b, long long n, int nb, double *tmp, double *out, cudaStream_t s)
{
    rel_diff<<<nb, 256, 0, s>>>(phi_a, phi_b, n, tmp);
    max_of<<<1, 32, 0, s>>>(tmp, nb, out);
    return cudaGetLastError();
}

} // namespace sur
} // namespace epdlb

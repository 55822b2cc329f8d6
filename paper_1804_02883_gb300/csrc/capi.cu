// capi.cu -- C ABI (include/epd_lb.h) and the engine around the kernels:
// parameter validation, workspace layout, transform tables, CUDA-graph capture
// of the time step, state access and checkpoints.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "engine.h"
#include "fft8.cuh"
#include "surrogate.h"

namespace epdlb {

cudaError_t configure_prop_kernels();
cudaError_t configure_epd_kernels();

cudaError_t configure_kernels()
{
    // once per process (a function-local static is initialised exactly once,
    // also when handles are created on several threads)
    static const cudaError_t status = [] {
        cudaError_t e = configure_prop_kernels();
        if (e == cudaSuccess) e = configure_epd_kernels();
        if (e == cudaSuccess) e = configure_step3d_kernels();
        return e;
    }();
    return status;
}

static size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

// Carve (or size, with base == nullptr) the buffers of one group.
size_t carve_group(Group &G, char *base, size_t off)
{
    const size_t n = (size_t)G.g.n, R = (size_t)G.g.nruns;
    const size_t tb = G.prec == EPD_LB_MIXED_FP32 ? sizeof(float) : sizeof(double);
    auto take = [&](size_t bytes) -> void * {
        off = align_up(off);
        void *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    G.omega = (double *)take(R * 3 * n * sizeof(double));
    G.omega_t = (double *)take(R * 3 * n * sizeof(double));
    G.phi = (double *)take(R * 3 * n * sizeof(double));
    G.phi_t = (double *)take(R * 3 * n * sizeof(double));
    G.q = (double *)take(R * 2 * sizeof(double));
    G.q_t = (double *)take(R * 2 * sizeof(double));
    G.ia = (double *)take(R * n * sizeof(double));
    G.ib = (double *)take(R * n * sizeof(double));
    G.ia2 = (double *)take(R * n * sizeof(double));
    G.ib2 = (double *)take(R * n * sizeof(double));
    G.cz = (double2 *)take(R * 4 * n * sizeof(double2));
    G.part = (double *)take(R * kMaxPart * sizeof(double));
    G.f0_lat = (double *)take(R * sizeof(double));
    G.f0_bulk = take(R * tb);
    G.stage = (double *)take(std::max<size_t>(9 * n, 2 * R + 16) * sizeof(double));
    G.chain = take(R * n * 2 * tb);
    // (decided from the parameters, not from a pointer: the dry run that
    // sizes the workspace carves with null pointers)
    const bool cluster = G.prec == EPD_LB_MIXED_FP32 && G.g.pow2 && cluster_shape_exists(G.g.logx, G.g.logy);
    // MIXED streaming solves keep every node of the reference history for
    // the differential second solve
    const bool stream_diff = G.prec == EPD_LB_MIXED_FP32 && !cluster;
    G.hist_full = G.g.pow2 && stream8_eligible(G.prec, G.g.logx, G.g.logy);
    G.hnodes = stream_diff ? G.g.ns + 1 : G.g.half_lo + 1;
    G.hist = take(R * (size_t)G.hnodes * n * 2 * tb);
    G.efac = take(R * n * 2 * tb);
    G.pop[0] = take(R * 9 * n * tb);
    G.pop[1] = take(R * 9 * n * tb);
    G.vel = take(R * n * 2 * tb);
    G.force = take(R * n * 2 * tb);
    G.twx = take((size_t)G.g.nx * 2 * tb);
    G.twy = take((size_t)G.g.ny * 2 * tb);
    G.kx = take((size_t)G.g.nx * tb);
    G.ky = take((size_t)G.g.ny * tb);
    G.twx_d = (double2 *)take((size_t)G.g.nx * sizeof(double2));
    G.twy_d = (double2 *)take((size_t)G.g.ny * sizeof(double2));
    // radix-8/16 and cluster tables: power-of-two axes only
    G.twx_full = G.twy_full = G.tab8x = G.tab8y = G.tab16x = G.tab16y = nullptr;
    if (G.g.pow2) {
        G.twx_full = (float2 *)take((size_t)G.g.nx * sizeof(float2));
        G.twy_full = (float2 *)take((size_t)G.g.ny * sizeof(float2));
        G.tab8x = (float2 *)take((size_t)tabs_total(G.g.logx) * sizeof(float2));
        G.tab8y = (float2 *)take((size_t)tabs_total(G.g.logy) * sizeof(float2));
        G.tab16x = best_mr(G.g.logx) == 4 ? (float2 *)take((size_t)tabs_total(G.g.logx, 4) * sizeof(float2)) : nullptr;
        G.tab16y = best_mr(G.g.logy) == 4 ? (float2 *)take((size_t)tabs_total(G.g.logy, 4) * sizeof(float2)) : nullptr;
    }
    // cluster solve (MIXED_FP32): stored states of both chains, and the
    // differential second solve's buffers; streaming MIXED solves: the
    // changes at every node and the factor changes
    G.hc = G.hd = G.rho = G.cdiff = nullptr;
    if (cluster) {
        const size_t hs = R * cluster_state_floats2(G.g.nx, G.g.ny, G.g.ns) * sizeof(float2);
        G.hc = take(hs);
        G.hd = take(hs);
        G.rho = take(R * n * sizeof(float2));
        G.cdiff = take(R * 3 * n * sizeof(float));
    } else if (stream_diff) {
        G.hd = take(R * (size_t)(G.g.ns + 1) * n * sizeof(float2));
        G.rho = take(R * n * sizeof(float2));
    }
    // exact step: the inversion's fields and scalars
    G.cg_target = (double *)take(R * 3 * n * sizeof(double));
    G.cg_dir = (double *)take(R * 3 * n * sizeof(double));
    G.cg_trial = (double *)take(R * 3 * n * sizeof(double));
    G.cg_wref = G.cg_pref = nullptr;
    if (cluster || stream_diff) {
        G.cg_wref = (double *)take(R * 3 * n * sizeof(double));
        G.cg_pref = (double *)take(R * 3 * n * sizeof(double));
    }
    G.cg_qref = (double *)take(R * 2 * sizeof(double));
    G.cg_part = (double *)take(R * kCgBlocks * 2 * sizeof(double));
    G.cg = (double *)take(R * kCgSlots * sizeof(double));
    G.diff = false;  // set once the cluster solve is known to launch
    return align_up(off);
}

// View of one run of a group (all per-run buffers offset, nruns = 1).
static Group run_view(const Group &G, int r)
{
    Group V = G;
    const size_t n = (size_t)G.g.n;
    const size_t tb = G.prec == EPD_LB_MIXED_FP32 ? sizeof(float) : sizeof(double);
    V.g.nruns = 1;
    V.omega += (size_t)r * 3 * n;
    V.omega_t += (size_t)r * 3 * n;
    V.phi += (size_t)r * 3 * n;
    V.phi_t += (size_t)r * 3 * n;
    V.q += 2 * r;
    V.q_t += 2 * r;
    V.ia += (size_t)r * n;
    V.ib += (size_t)r * n;
    V.ia2 += (size_t)r * n;
    V.ib2 += (size_t)r * n;
    V.cz += (size_t)r * 4 * n;
    V.part += (size_t)r * kMaxPart;
    V.f0_lat += r;
    V.f0_bulk = (char *)V.f0_bulk + (size_t)r * tb;
    V.chain = (char *)V.chain + (size_t)r * n * 2 * tb;
    V.hist = (char *)V.hist + (size_t)r * G.hnodes * n * 2 * tb;
    V.efac = (char *)V.efac + (size_t)r * n * 2 * tb;
    V.pop[0] = (char *)V.pop[0] + (size_t)r * 9 * n * tb;
    V.pop[1] = (char *)V.pop[1] + (size_t)r * 9 * n * tb;
    V.vel = (char *)V.vel + (size_t)r * n * 2 * tb;
    V.force = (char *)V.force + (size_t)r * n * 2 * tb;
    if (G.hc) {
        const size_t hs = cluster_state_floats2(G.g.nx, G.g.ny, G.g.ns) * sizeof(float2);
        V.hc = (char *)V.hc + (size_t)r * hs;
        V.hd = (char *)V.hd + (size_t)r * hs;
        V.rho = (char *)V.rho + (size_t)r * n * sizeof(float2);
        V.cdiff = (char *)V.cdiff + (size_t)r * 3 * n * sizeof(float);
    } else if (G.hd) {
        V.hd = (char *)V.hd + (size_t)r * (G.g.ns + 1) * n * sizeof(float2);
        V.rho = (char *)V.rho + (size_t)r * n * sizeof(float2);
    }
    if (G.cg_wref) {
        V.cg_wref += (size_t)r * 3 * n;
        V.cg_pref += (size_t)r * 3 * n;
    }
    V.cg_target += (size_t)r * 3 * n;
    V.cg_dir += (size_t)r * 3 * n;
    V.cg_trial += (size_t)r * 3 * n;
    V.cg_qref += 2 * r;
    V.cg_part += (size_t)r * kCgBlocks * 2;
    V.cg += (size_t)r * kCgSlots;
    return V;
}

static bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Radix plan of an axis: radix 4 while it divides, then 2, 3, 5.
static int radix_plan(int n, int *f)
{
    int k = 0;
    for (int p : {4, 2, 3, 5})
        while (n % p == 0 && k < kMaxFactors) {
            f[k++] = p;
            n /= p;
        }
    return k;
}

// Largest divisor of n not above cap (at least 1).
static int divisor_at_most(int n, int cap)
{
    for (int d = std::max(1, std::min(n, cap)); d > 1; --d)
        if (n % d == 0) return d;
    return 1;
}

static double fstar_lattice(const epd_lb_params &p)
{
    const double tau = p.rg * p.rg / p.d_s;
    const double r = p.dt / tau;
    return (p.rg / p.dx) * r * r;
}

static void fill_geom(Group &G)
{
    const epd_lb_params &p = G.p;
    GroupGeom &g = G.g;
    g.nx = p.nx;
    g.ny = p.ny;
    g.pow2 = pow2(p.nx) && pow2(p.ny);
    g.logx = g.pow2 ? ilog2(p.nx) : 0;
    g.logy = g.pow2 ? ilog2(p.ny) : 0;
    g.nfx = radix_plan(p.nx, g.fx);
    g.nfy = radix_plan(p.ny, g.fy);
    g.ns = p.ns;
    g.na = (int)std::lround(p.f_a * (double)p.ns);
    g.jr = p.junction_rule;
    g.half_lo = p.ns / 2;
    g.half_hi = (p.ns + 1) / 2;
    g.nruns = (int)G.run_ids.size();
    g.n = (long long)p.nx * p.ny;
    g.dx = p.dx;
    g.dt = p.dt;
    g.rg = p.rg;
    g.nseg = p.n_seg;
    g.phi_p = p.phi_p;
    g.ds = 1.0 / (double)p.ns;
    g.chi_ab = p.chi_ab;
    g.chi_as = p.chi_as;
    g.chi_bs = p.chi_bs;
    g.kappa_h = p.kappa_h;
    g.d_s = p.d_s;
    g.d_p = p.d_p;
    g.inv_beta_v = p.inv_beta_v;
    g.gamma_s = p.gamma_s;
    g.gamma_b = p.gamma_b;
    g.gamma_g = p.gamma_g;
    g.fstar = fstar_lattice(p);
    g.vscale = p.dx / p.dt;
}

// Launch shapes: about 2048 points per CTA, column tiles at least 32 bytes wide.
static void default_shapes(Group &G)
{
    const int nx = G.g.nx, ny = G.g.ny;
    const bool f32 = G.prec == EPD_LB_MIXED_FP32;
    G.sh.rows_prop = std::max(1, std::min(ny, 2048 / nx));
    G.sh.cols_prop = std::min(nx, std::max(f32 ? 4 : 2, 2048 / ny));
    G.sh.rows_epd = std::max(1, std::min(ny, 2048 / nx));
    G.sh.cols_epd = std::min(nx, std::max(2, 2048 / ny));
    if (!G.g.pow2) {  // tiles must divide the axes
        G.sh.rows_prop = divisor_at_most(ny, G.sh.rows_prop);
        G.sh.cols_prop = divisor_at_most(nx, G.sh.cols_prop);
        G.sh.rows_epd = divisor_at_most(ny, G.sh.rows_epd);
        G.sh.cols_epd = divisor_at_most(nx, G.sh.cols_epd);
    }
}

// Twiddles exp(-2 pi i t / n), t < n (the radix-2 passes read t < n/2), and
// Fourier factors exp(-R_G^2 k^2 ds) / n of the propagator (Eq. (8)), on the
// host in FP64.
template <typename T>
static void host_tables(const Group &G, std::vector<T> &twx, std::vector<T> &twy, std::vector<T> &kx, std::vector<T> &ky,
                        std::vector<double> &twxd, std::vector<double> &twyd)
{
    const double pi = 3.14159265358979323846;
    auto tw = [&](int n, std::vector<T> &out, std::vector<double> &outd) {
        out.resize(2 * (size_t)n);
        outd.resize(2 * (size_t)n);
        for (int t = 0; t < n; ++t) {
            const double a = 2.0 * pi * (double)t / (double)n;
            outd[2 * t] = std::cos(a);
            outd[2 * t + 1] = -std::sin(a);
            out[2 * t] = (T)outd[2 * t];
            out[2 * t + 1] = (T)outd[2 * t + 1];
        }
    };
    tw(G.g.nx, twx, twxd);
    tw(G.g.ny, twy, twyd);
    auto kf = [&](int n, std::vector<T> &out) {
        out.resize(n);
        for (int m = 0; m < n; ++m) {
            const int mm = m <= n / 2 ? m : m - n;
            const double k = 2.0 * pi * (double)mm / ((double)n * G.g.dx);
            out[m] = (T)(std::exp(-G.g.rg * G.g.rg * k * k * G.g.ds) / (double)n);
        }
    };
    kf(G.g.nx, kx);
    kf(G.g.ny, ky);
}

template <typename T>
static cudaError_t upload_tables_t(Group &G, cudaStream_t s)
{
    std::vector<T> twx, twy, kx, ky;
    std::vector<double> twxd, twyd;
    host_tables<T>(G, twx, twy, kx, ky, twxd, twyd);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(G.twx, twx.data(), twx.size() * sizeof(T), cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyAsync(G.twy, twy.data(), twy.size() * sizeof(T), cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyAsync(G.kx, kx.data(), kx.size() * sizeof(T), cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyAsync(G.ky, ky.data(), ky.size() * sizeof(T), cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyAsync(G.twx_d, twxd.data(), twxd.size() * sizeof(double), cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyAsync(G.twy_d, twyd.data(), twyd.size() * sizeof(double), cudaMemcpyHostToDevice, s))) return e;
    if (G.twx_full) {
        const double pi = 3.14159265358979323846;
        auto full = [&](int n) {
            std::vector<float> t(2 * (size_t)n);
            for (int j = 0; j < n; ++j) {
                const double a = 2.0 * pi * (double)j / (double)n;
                t[2 * j] = (float)std::cos(a);
                t[2 * j + 1] = (float)-std::sin(a);
            }
            return t;
        };
        const std::vector<float> fx = full(G.g.nx), fy = full(G.g.ny);
        if ((e = cudaMemcpyAsync(G.twx_full, fx.data(), fx.size() * sizeof(float), cudaMemcpyHostToDevice, s))) return e;
        if ((e = cudaMemcpyAsync(G.twy_full, fy.data(), fy.size() * sizeof(float), cudaMemcpyHostToDevice, s))) return e;
        std::vector<float> tx(2 * (size_t)tabs_total(G.g.logx)), ty(2 * (size_t)tabs_total(G.g.logy));
        build_tables_host(G.g.logx, fx.data(), tx.data());
        build_tables_host(G.g.logy, fy.data(), ty.data());
        if ((e = cudaMemcpyAsync(G.tab8x, tx.data(), tx.size() * sizeof(float), cudaMemcpyHostToDevice, s))) return e;
        if ((e = cudaMemcpyAsync(G.tab8y, ty.data(), ty.size() * sizeof(float), cudaMemcpyHostToDevice, s))) return e;
        std::vector<float> t16x(G.tab16x ? 2 * (size_t)tabs_total(G.g.logx, 4) : 0), t16y(G.tab16y ? 2 * (size_t)tabs_total(G.g.logy, 4) : 0);
        if (G.tab16x) {
            build_tables_host(G.g.logx, fx.data(), t16x.data(), 4);
            if ((e = cudaMemcpyAsync(G.tab16x, t16x.data(), t16x.size() * sizeof(float), cudaMemcpyHostToDevice, s))) return e;
        }
        if (G.tab16y) {
            build_tables_host(G.g.logy, fy.data(), t16y.data(), 4);
            if ((e = cudaMemcpyAsync(G.tab16y, t16y.data(), t16y.size() * sizeof(float), cudaMemcpyHostToDevice, s))) return e;
        }
        if ((e = cudaStreamSynchronize(s))) return e;
    }
    std::vector<double> f0(G.g.nruns);
    for (int r = 0; r < G.g.nruns; ++r) f0[r] = G.run_params[r].f0 * G.g.fstar;
    if ((e = cudaMemcpyAsync(G.f0_lat, f0.data(), f0.size() * sizeof(double), cudaMemcpyHostToDevice, s))) return e;
    std::vector<T> f0b(f0.begin(), f0.end());
    if (G.f0_bulk && (e = cudaMemcpyAsync(G.f0_bulk, f0b.data(), f0b.size() * sizeof(T), cudaMemcpyHostToDevice, s))) return e;
    return cudaStreamSynchronize(s);
}

static cudaError_t upload_tables_e(Group &G, cudaStream_t s)
{
    return G.prec == EPD_LB_MIXED_FP32 ? upload_tables_t<float>(G, s) : upload_tables_t<double>(G, s);
}

void upload_tables(Group &G, cudaStream_t s) { (void)upload_tables_e(G, s); }

// even lengths of the form 2^a 3^b 5^c (the mixed-radix transforms' radices)
static bool smooth_even(int v)
{
    if (v < 2 || (v & 1)) return false;
    for (int p : {2, 3, 5})
        while (v % p == 0) v /= p;
    return v == 1;
}

static std::string validate(const epd_lb_params &p)
{
    char buf[256];
    if (!smooth_even(p.nx) || !smooth_even(p.ny) || p.nx < kMinN || p.ny < kMinN || p.nx > kMaxN || p.ny > kMaxN) {
        std::snprintf(buf, sizeof buf, "nx=%d, ny=%d: each must be even, of the form 2^a 3^b 5^c, in [%d, %d]", p.nx,
                      p.ny, kMinN, kMaxN);
        return buf;
    }
    // the MIXED power-of-two paths (cluster-resident and radix-8 streaming
    // solves) pair contour nodes symmetrically and need N_s even; the radix-2
    // streaming solve (PLAIN_FP64, mixed-radix grids) takes any N_s, such as
    // the paper's N_s = N = 17
    const bool any_ns = p.precision == EPD_LB_PLAIN_FP64 || !(pow2(p.nx) && pow2(p.ny));
    if (p.ns < 2 || p.ns > 512 || ((p.ns & 1) && !any_ns)) {
        std::snprintf(buf, sizeof buf, "ns=%d: must be in [2, 512] (and even for MIXED_FP32 on power-of-two grids)", p.ns);
        return buf;
    }
    if (p.precision != EPD_LB_PLAIN_FP64 && p.precision != EPD_LB_MIXED_FP32) return "precision must be 0 (PLAIN_FP64) or 1 (MIXED_FP32)";
    if (!(p.dx > 0) || !(p.dt > 0) || !(p.rg > 0) || !(p.n_seg > 0) || !(p.d_s > 0) || !(p.d_p > 0))
        return "dx, dt, rg, n_seg, d_s and d_p must be positive";
    if (!(p.f_a >= 0 && p.f_a <= 1)) return "f_a must be in [0, 1]";
    if (!(p.phi_p > 0 && p.phi_p < 1)) return "phi_p must be in (0, 1)";
    if (!(std::fabs(p.gamma_s) < 1) || !(std::fabs(p.gamma_b) < 1) || !(std::fabs(p.gamma_g) < 1))
        return "gamma_s, gamma_b and gamma_g must be in (-1, 1)";
    if (!std::isfinite(p.f0) || !std::isfinite(p.noise_amp) || !std::isfinite(p.inv_beta_v)) return "f0, noise_amp, inv_beta_v must be finite";
    if (p.junction_rule != 0 && p.junction_rule != 1) return "junction_rule must be 0 (literal) or 1 (segment-symmetric)";
    if (p.reserved != 0) return "reserved must be 0";
    return "";
}

// Peak of Eq. (24) in lattice units, f0 L_y^2 / (32 eta): refuse above Mach 0.3.
static bool mach_ok(const epd_lb_params &p, double *vmax)
{
    const double eta = (1.0 / 6.0) * (1.0 + p.gamma_s) / (1.0 - p.gamma_s);
    const double a = std::fabs(p.f0) * fstar_lattice(p);
    *vmax = a * (double)p.ny * p.ny / (32.0 * eta);
    return *vmax <= 0.3 * std::sqrt(1.0 / 3.0);
}

static bool same_group(const epd_lb_params &a, const epd_lb_params &b)
{
    return a.nx == b.nx && a.ny == b.ny && a.ns == b.ns && a.precision == b.precision && a.dx == b.dx && a.dt == b.dt &&
           a.rg == b.rg && a.n_seg == b.n_seg && a.f_a == b.f_a && a.phi_p == b.phi_p && a.chi_ab == b.chi_ab &&
           a.chi_as == b.chi_as && a.chi_bs == b.chi_bs && a.kappa_h == b.kappa_h && a.d_s == b.d_s && a.d_p == b.d_p &&
           a.inv_beta_v == b.inv_beta_v && a.gamma_s == b.gamma_s && a.gamma_b == b.gamma_b && a.gamma_g == b.gamma_g &&
           a.junction_rule == b.junction_rule;
}

static void form_groups(const epd_lb_params *p, int nruns, std::vector<Group> &groups, std::vector<std::pair<int, int>> &where)
{
    groups.clear();
    where.assign(nruns, {-1, -1});
    for (int r = 0; r < nruns; ++r) {
        int gi = -1;
        for (size_t k = 0; k < groups.size(); ++k)
            if (same_group(groups[k].p, p[r])) { gi = (int)k; break; }
        if (gi < 0) {
            Group G = Group();
            G.p = p[r];
            G.prec = p[r].precision;
            groups.push_back(G);
            gi = (int)groups.size() - 1;
        }
        where[r] = {gi, (int)groups[gi].run_ids.size()};
        groups[gi].run_ids.push_back(r);
        groups[gi].run_params.push_back(p[r]);
    }
    for (auto &G : groups) {
        fill_geom(G);
        default_shapes(G);
    }
}

} // namespace epdlb

using namespace epdlb;

// Head of the handle's workspace: the device error word at 0, the observables
// at 256, the partials of the two-stage reductions at 512.
constexpr size_t kHeadBytes = 512 + (size_t)kRedSlots * kRedBlocks * sizeof(double);
static_assert(kHeadBytes % 256 == 0, "workspace head");

struct epd_lb {
    std::vector<Group> groups;
    std::vector<std::pair<int, int>> where;  // run -> (group, member)
    int nruns = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *ws = nullptr;
    bool own_ws = false;
    int *err = nullptr;
    double *obs = nullptr;
    double *part = nullptr;  // partials of the two-stage reductions
    int parity = 0;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    bool timing = false;
    bool timed_cluster = false;  // the timed solve ran as one cluster-resident launch
    // one stream per group beyond the first, forked from and joined to the
    // handle's stream inside the captured step so that groups run concurrently
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> fork_ev, join_ev;
    // learned surrogate (attached with epd_lb_set_surrogate)
    bool sur_on = false;
    int sur_every = 0;
    double sur_tol = 0.0, sur_s_in = 1.0, sur_s_out = 1.0;
    bool sur_hold = false;                     // surrogate steps keep the last exact step's polymer force
    float *sur_params = nullptr;               // device copy
    std::vector<epdlb::sur::Work> sur_work;    // one per group
    double *sur_resid = nullptr;               // [groups + 1] device: per group residual, scratch
    cudaGraphExec_t exec_sur[2] = {nullptr, nullptr}, exec_chk[2] = {nullptr, nullptr};
    long long sur_steps = 0, sur_exact = 0, sur_used = 0, sur_forced = 0;
    double sur_last = 0.0;
    bool sur_fallback = false;
    // exact step (epd_lb_set_inversion): CG iterations per step (0: the
    // inversion truncated to its starting guess) and the residual tolerance
    int cg_max = 0;
    double cg_tol = 1e-8;
    double *cg_host = nullptr;  // pinned copy of one group's per-run scalars
    cudaEvent_t ev[7] = {};
    std::string last_error;
};

static int fail(epd_lb *h, int code, const std::string &msg)
{
    if (h) h->last_error = msg;
    return code;
}

static int cuda_fail(epd_lb *h, cudaError_t e, const char *where)
{
    return fail(h, EPD_LB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                  \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
    } while (0)

extern "C" int epd_lb_workspace_bytes(const epd_lb_params *p, int32_t nruns, size_t *bytes)
{
    if (!p || nruns <= 0 || !bytes) return EPD_LB_EINVAL;
    for (int r = 0; r < nruns; ++r)
        if (!validate(p[r]).empty()) return EPD_LB_EINVAL;
    std::vector<Group> groups;
    std::vector<std::pair<int, int>> where;
    form_groups(p, nruns, groups, where);
    size_t off = kHeadBytes;
    for (auto &G : groups) off = carve_group(G, nullptr, off);
    *bytes = off;
    return EPD_LB_OK;
}

// Record the whole time step of every group (App. C order) on stream s.
enum StepMode { STEP_EXACT = 0, STEP_SURROGATE = 1, STEP_CHECK = 2 };

static void sur_means(const Group &G, double &pa, double &pb, double &ps)
{
    const double fa = (double)G.g.na / (double)G.g.ns;
    pa = G.g.phi_p * fa;
    pb = G.g.phi_p * (1.0 - fa);
    ps = 1.0 - G.g.phi_p;
}

static cudaError_t enqueue_group(epd_lb *h, size_t gi, int parity, cudaStream_t s, int mode = STEP_EXACT)
{
    cudaError_t e;
    Group &G = h->groups[gi];
    if (mode == STEP_SURROGATE) {
        double pa, pb, ps;
        sur_means(G, pa, pb, ps);
        sur::Work &W = h->sur_work[gi];
        if ((e = launch_aux_convection(G, s))) return e;
        if ((e = sur::forward(W, h->sur_params, G.omega_t, G.phi_t, h->sur_s_in, h->sur_s_out, pa, pb, ps, s))) return e;
        if ((e = launch_diffusion(G, s))) return e;
        // Phi(t+dt) = Phi~ + the surrogate's change along omega(t+dt) - omega~
        // (tangent pass), which drives the force unless the force of the last
        // exact step is held
        if ((e = sur::tangent(W, h->sur_params, G.omega, G.omega_t, G.phi_t, G.phi, h->sur_s_in, h->sur_s_out, ps, s))) return e;
        if (!h->sur_hold && (e = launch_force(G, s))) return e;
        return launch_lb(G, parity, s);
    }
    SolveProbe probe;
    const bool timed = h->timing && gi == 0;
    if (timed) {
        for (int k = 0; k < 5; ++k) probe.ev[k] = h->ev[k];
        probe.m_store = std::max(1, G.g.ns / 4);
        probe.m_acc = std::min(G.g.ns, (3 * G.g.ns) / 4 + 1);
    }
    if ((e = launch_aux_convection(G, s))) return e;                      // omega -> omega~
    if ((e = launch_solve(G, G.omega_t, G.phi_t, G.q_t, s))) return e;    // Phi~
    if (mode == STEP_CHECK) {
        // the surrogate at omega~ into the EPD scratch, residual against Phi~
        double pa, pb, ps;
        sur_means(G, pa, pb, ps);
        double *phi_sur = reinterpret_cast<double *>(G.cz);
        if ((e = sur::forward(h->sur_work[gi], h->sur_params, G.omega_t, phi_sur, h->sur_s_in, h->sur_s_out, pa, pb, ps, s))) return e;
        if ((e = sur::residual_rel(phi_sur, G.phi_t, G.g.n, G.g.nruns, G.part, h->sur_resid + gi, s))) return e;
    }
    if ((e = launch_diffusion(G, s))) return e;                           // omega(t+dt)
    if (G.diff) {  // Phi(t+dt) as Phi~ plus the change from the diffusion update
        if ((e = launch_solve_delta(G, s, timed ? &probe : nullptr))) return e;
    } else if ((e = launch_solve(G, G.omega, G.phi, G.q, s, timed ? &probe : nullptr))) {
        return e;  // Phi(t+dt)
    }
    if (timed) h->timed_cluster = probe.cluster;
    if ((e = launch_force(G, s))) return e;                               // polymer force
    if (timed && (e = cudaEventRecordWithFlags(h->ev[5], s, cudaEventRecordExternal))) return e;
    if ((e = launch_lb(G, parity, s))) return e;                          // collide-stream
    if (timed && (e = cudaEventRecordWithFlags(h->ev[6], s, cudaEventRecordExternal))) return e;
    return cudaSuccess;
}

// Record the whole time step of every group (App. C order); group 0 on the
// handle's stream, the others on their own streams forked from it.
static cudaError_t enqueue_step(epd_lb *h, int parity, cudaStream_t s, int mode = STEP_EXACT)
{
    cudaError_t e;
    const size_t ng = h->groups.size();
    for (size_t gi = 1; gi < ng; ++gi) {
        if ((e = cudaEventRecord(h->fork_ev[gi - 1], s))) return e;
        if ((e = cudaStreamWaitEvent(h->side[gi - 1], h->fork_ev[gi - 1], 0))) return e;
        if ((e = enqueue_group(h, gi, parity, h->side[gi - 1], mode))) return e;
        if ((e = cudaEventRecord(h->join_ev[gi - 1], h->side[gi - 1]))) return e;
    }
    if ((e = enqueue_group(h, 0, parity, s, mode))) return e;
    for (size_t gi = 1; gi < ng; ++gi)
        if ((e = cudaStreamWaitEvent(s, h->join_ev[gi - 1], 0))) return e;
    return cudaSuccess;
}

static int capture(epd_lb *h, int par, int mode, cudaGraphExec_t *out)
{
    if (*out) {
        cudaGraphExecDestroy(*out);
        *out = nullptr;
    }
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    cudaError_t e = enqueue_step(h, par, h->stream, mode);
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(h, e, "capturing the time step");
    }
    CK(e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    CK(e, "cudaGraphInstantiate");
    return EPD_LB_OK;
}

static int build_graphs(epd_lb *h)
{
    for (int par = 0; par < 2; ++par) {
        if (int rc = capture(h, par, STEP_EXACT, &h->exec[par])) return rc;
        if (h->sur_on) {
            if (int rc = capture(h, par, STEP_SURROGATE, &h->exec_sur[par])) return rc;
            if (int rc = capture(h, par, STEP_CHECK, &h->exec_chk[par])) return rc;
        }
    }
    return EPD_LB_OK;
}

extern "C" int epd_lb_init(const epd_lb_params *p, int32_t nruns, void *workspace, size_t workspace_bytes,
                           void *cuda_stream, epd_lb **out)
{
    if (!out) return EPD_LB_EINVAL;
    *out = nullptr;
    epd_lb *h = new (std::nothrow) epd_lb();
    if (!h) return EPD_LB_ENOMEM;
    if (!p || nruns <= 0) {
        delete h;
        return EPD_LB_EINVAL;
    }
    for (int r = 0; r < nruns; ++r) {
        std::string msg = validate(p[r]);
        if (!msg.empty()) {
            delete h;
            return EPD_LB_EINVAL;
        }
        double vmax;
        if (!mach_ok(p[r], &vmax)) {
            delete h;
            return EPD_LB_EUNSTABLE;
        }
    }
    h->nruns = nruns;
    form_groups(p, nruns, h->groups, h->where);
    size_t need = kHeadBytes;
    for (auto &G : h->groups) need = carve_group(G, nullptr, need);
    auto bail = [&](int code) {
        epd_lb_destroy(h);
        return code;
    };
    if (cudaError_t e = configure_kernels()) {
        (void)e;
        return bail(EPD_LB_ECUDA);
    }
    if (workspace) {
        if (workspace_bytes < need || ((uintptr_t)workspace & 255)) return bail(EPD_LB_ENOMEM);
        h->ws = workspace;
    } else {
        if (cudaMalloc(&h->ws, need) != cudaSuccess) {
            h->ws = nullptr;
            return bail(EPD_LB_ENOMEM);
        }
        h->own_ws = true;
    }
    if (cuda_stream) {
        h->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(EPD_LB_ECUDA);
        h->own_stream = true;
    }
    char *base = (char *)h->ws;
    h->err = (int *)base;
    h->obs = (double *)(base + 256);
    h->part = (double *)(base + 512);
    size_t off = kHeadBytes;
    for (auto &G : h->groups) {
        off = carve_group(G, base, off);
        G.err = h->err;
    }
    // the carve with real pointers must end where the sizing dry run did
    if (off > need) return bail(EPD_LB_ENOMEM);
    if (cudaMemsetAsync(h->err, 0, sizeof(int), h->stream) != cudaSuccess) return bail(EPD_LB_ECUDA);
    for (auto &G : h->groups) {
        if (upload_tables_e(G, h->stream) != cudaSuccess) return bail(EPD_LB_ECUDA);
        if (launch_init_state(G, h->stream) != cudaSuccess) return bail(EPD_LB_ECUDA);
        if (launch_solve(G, G.omega, G.phi, G.q, h->stream) != cudaSuccess) return bail(EPD_LB_ECUDA);
        if (tune_column_tiles(G, h->stream) != cudaSuccess) return bail(EPD_LB_ECUDA);
        if (tune_stream_tiles(G, h->stream) != cudaSuccess) return bail(EPD_LB_ECUDA);
        // cluster grids: when the cluster solve launches; MIXED streaming
        // grids always
        G.diff = G.hd != nullptr && (G.hc ? G.twx_full != nullptr && cluster_solve_supported(G) : true);
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return bail(EPD_LB_ECUDA);
    for (size_t gi = 1; gi < h->groups.size(); ++gi) {
        cudaStream_t st;
        cudaEvent_t a, b;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return bail(EPD_LB_ECUDA);
        h->side.push_back(st);
        if (cudaEventCreateWithFlags(&a, cudaEventDisableTiming) != cudaSuccess) return bail(EPD_LB_ECUDA);
        h->fork_ev.push_back(a);
        if (cudaEventCreateWithFlags(&b, cudaEventDisableTiming) != cudaSuccess) return bail(EPD_LB_ECUDA);
        h->join_ev.push_back(b);
    }
    h->parity = 0;
    if (int rc = build_graphs(h)) return bail(rc);
    *out = h;
    return EPD_LB_OK;
}

// Whether any run of group G is still iterating (reads the per-run scalars).
static int cg_any_active(epd_lb *h, Group &G, cudaStream_t s, bool *any)
{
    const size_t bytes = (size_t)G.g.nruns * kCgSlots * sizeof(double);
    CK(cudaMemcpyAsync(h->cg_host, G.cg, bytes, cudaMemcpyDeviceToHost, s), "reading the inversion state");
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    *any = false;
    for (int r = 0; r < G.g.nruns; ++r) *any = *any || h->cg_host[(size_t)r * kCgSlots + CG_ACTIVE] != 0.0;
    return EPD_LB_OK;
}

// One exact time step of group gi (App. C with the inversion), enqueued
// eagerly on s: the iteration count depends on the data.
//   Phi~ = Phi(t) - dt div(v Phi(t)); omega~ = Phi^{-1}(Phi~) by CG from the
//   auxiliary convection of omega; then diffusion, second solve, force, LB.
// MIXED groups (cluster solve) evaluate every density of the step as a
// difference from the solve at the starting guess, Phi(t) included, so the
// mismatch carries the FP32 rounding of the changes only.
static int exact_group_step(epd_lb *h, size_t gi, int parity, cudaStream_t s, bool *notconv)
{
    Group &G = h->groups[gi];
    const bool dif = G.diff;
    const size_t m = (size_t)G.g.nruns * 3 * (size_t)G.g.n;
    auto solve_at = [&](const double *om, double *ph, double *q) -> cudaError_t {
        return dif ? launch_solve_delta_at(G, om, G.cg_wref, G.cg_pref, G.cg_qref, ph, q, s) : launch_solve(G, om, ph, q, s);
    };
    if (G.phi_stale && !dif) CK(launch_solve(G, G.omega, G.phi, G.q, s), "Phi(t) of a replaced omega");
    CK(launch_aux_convection(G, s), "auxiliary convection");              // starting guess omega~0
    CK(launch_solve(G, G.omega_t, G.phi_t, G.q_t, s), "solve at the starting guess");
    if (dif) {
        CK(cudaMemcpyAsync(G.cg_wref, G.omega_t, m * sizeof(double), cudaMemcpyDeviceToDevice, s), "reference omega");
        CK(cudaMemcpyAsync(G.cg_pref, G.phi_t, m * sizeof(double), cudaMemcpyDeviceToDevice, s), "reference Phi");
        CK(cudaMemcpyAsync(G.cg_qref, G.q_t, (size_t)G.g.nruns * 2 * sizeof(double), cudaMemcpyDeviceToDevice, s), "reference Q");
        CK(solve_at(G.omega, G.phi, G.q), "Phi(t) against the reference");
    }
    CK(launch_convect_phi(G, G.phi, G.cg_target, s), "convection of Phi");  // target Phi~
    CK(cg_begin(G, G.phi_t, h->cg_tol, s), "inversion start");
    for (int it = 0; it < h->cg_max; ++it) {
        if (h->cg_tol > 0.0) {
            bool any = false;
            if (int rc = cg_any_active(h, G, s, &any)) return rc;
            if (!any) break;
        }
        CK(cg_trial_point(G, G.omega_t, G.cg_trial, s), "trial point");
        CK(solve_at(G.cg_trial, G.phi, G.q), "solve at the trial point");
        CK(cg_line_step(G, G.phi, G.omega_t, s), "line step");
        CK(solve_at(G.omega_t, G.phi_t, G.q_t), "solve at the new iterate");
        CK(cg_direction(G, G.phi_t, h->cg_tol, s), "new direction");
    }
    if (h->cg_tol > 0.0) {
        bool any = false;
        if (int rc = cg_any_active(h, G, s, &any)) return rc;
        *notconv = *notconv || any;
    }
    CK(launch_diffusion(G, s), "diffusion");                              // omega(t+dt)
    CK(solve_at(G.omega, G.phi, G.q), "solve at t + dt");                 // Phi(t+dt)
    CK(launch_force(G, s), "force");
    CK(launch_lb(G, parity, s), "collide-stream");
    return EPD_LB_OK;
}

extern "C" int epd_lb_set_inversion(epd_lb *h, int32_t max_iter, double tol)
{
    if (!h) return EPD_LB_EINVAL;
    if (max_iter < 0 || max_iter > 100000 || !(tol >= 0.0) || !std::isfinite(tol))
        return fail(h, EPD_LB_EINVAL, "max_iter must be in [0, 100000] and tol finite and >= 0");
    if (max_iter > 0) {
        if (h->sur_on) return fail(h, EPD_LB_EINVAL, "the exact step and the surrogate exclude each other");
        for (const Group &G : h->groups)
            if (G.prec != EPD_LB_PLAIN_FP64 && !G.diff)
                return fail(h, EPD_LB_EINVAL,
                            "the exact step needs PLAIN_FP64 or a MIXED_FP32 grid with the differential solve");
        if (!h->cg_host) {
            size_t mr = 1;
            for (const Group &G : h->groups) mr = std::max(mr, (size_t)G.g.nruns);
            CK(cudaMallocHost(&h->cg_host, mr * kCgSlots * sizeof(double)), "cudaMallocHost");
        }
    }
    h->cg_max = max_iter;
    h->cg_tol = tol;
    return EPD_LB_OK;
}

extern "C" int epd_lb_inversion_stats(epd_lb *h, int32_t run, double *out)
{
    Group *G;
    int mb;
    if (!out) return fail(h, EPD_LB_EINVAL, "out is NULL");
    if (!h || run < 0 || run >= h->nruns) return fail(h, EPD_LB_EINVAL, "run index out of range");
    G = &h->groups[h->where[run].first];
    mb = h->where[run].second;
    double c[kCgSlots];
    CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    CK(cudaMemcpy(c, G->cg + (size_t)mb * kCgSlots, sizeof(c), cudaMemcpyDeviceToHost), "reading the inversion state");
    out[0] = c[CG_ITERS];
    out[1] = c[CG_RES0];
    out[2] = c[CG_RES];
    return EPD_LB_OK;
}

extern "C" int epd_lb_step(epd_lb *h, int64_t nsteps)
{
    if (!h || nsteps < 0) return EPD_LB_EINVAL;
    if (h->cg_max > 0) {
        for (int64_t k = 0; k < nsteps; ++k) {
            bool notconv = false;
            for (size_t gi = 0; gi < h->groups.size(); ++gi) {
                if (int rc = exact_group_step(h, gi, h->parity, h->stream, &notconv)) return rc;
                h->groups[gi].phi_stale = false;
            }
            h->parity ^= 1;
            if (notconv)
                return fail(h, EPD_LB_ENOTCONV, "the inversion did not reach the tolerance within max_iter iterations");
        }
        return EPD_LB_OK;
    }
    for (int64_t k = 0; k < nsteps; ++k) {
        if (!h->sur_on) {
            CK(cudaGraphLaunch(h->exec[h->parity], h->stream), "cudaGraphLaunch");
        } else if (h->sur_fallback || h->sur_steps % h->sur_every == 0) {
            // exact step that also checks the surrogate
            CK(cudaGraphLaunch(h->exec_chk[h->parity], h->stream), "cudaGraphLaunch");
            std::vector<double> r(h->groups.size());
            CK(cudaMemcpyAsync(r.data(), h->sur_resid, r.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "reading the residual");
            CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
            double m = 0.0;
            for (double v : r) m = v > m ? v : m;
            if (h->sur_fallback) ++h->sur_forced;
            ++h->sur_exact;
            h->sur_last = m;
            h->sur_fallback = !(m <= h->sur_tol);
            ++h->sur_steps;
        } else {
            CK(cudaGraphLaunch(h->exec_sur[h->parity], h->stream), "cudaGraphLaunch");
            ++h->sur_used;
            ++h->sur_steps;
        }
        for (Group &G : h->groups) G.phi_stale = false;
        h->parity ^= 1;
    }
    return EPD_LB_OK;
}

extern "C" int epd_lb_sync(epd_lb *h)
{
    if (!h) return EPD_LB_EINVAL;
    CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    int err = 0;
    CK(cudaMemcpy(&err, h->err, sizeof(int), cudaMemcpyDeviceToHost), "reading the device error word");
    if (err & 1) return fail(h, EPD_LB_ENONFINITE, "a single-chain solve produced Q <= 0 or a non-finite Q");
    if (err & 4) return fail(h, EPD_LB_ETIMEOUT, "an exchange wait of the cluster solve gave up");
    return EPD_LB_OK;
}

static int locate(epd_lb *h, int run, Group **G, int *m)
{
    if (!h || run < 0 || run >= h->nruns) return fail(h, EPD_LB_EINVAL, "run index out of range");
    *G = &h->groups[h->where[run].first];
    *m = h->where[run].second;
    return EPD_LB_OK;
}

extern "C" int epd_lb_densities_dev(epd_lb *h, int32_t run, double *phi_dev, double *q_dev)
{
    Group *G;
    int m;
    if (int rc = locate(h, run, &G, &m)) return rc;
    const size_t n = (size_t)G->g.n;
    if (phi_dev) CK(cudaMemcpyAsync(phi_dev, G->phi + (size_t)m * 3 * n, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream), "copy phi");
    if (q_dev) CK(cudaMemcpyAsync(q_dev, G->q + 2 * m, 2 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream), "copy q");
    return EPD_LB_OK;
}

extern "C" int epd_lb_fields_dev(epd_lb *h, int32_t run, double *omega_dev, double *phi_dev)
{
    Group *G;
    int m;
    if (int rc = locate(h, run, &G, &m)) return rc;
    const size_t n = (size_t)G->g.n;
    if (omega_dev)
        CK(cudaMemcpyAsync(omega_dev, G->omega + (size_t)m * 3 * n, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream), "copy omega");
    if (phi_dev)
        CK(cudaMemcpyAsync(phi_dev, G->phi + (size_t)m * 3 * n, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream), "copy phi");
    return EPD_LB_OK;
}

extern "C" int epd_lb_step_fields_dev(epd_lb *h, int32_t run, double *omega_tilde_dev, double *phi_tilde_dev)
{
    Group *G;
    int m;
    if (int rc = locate(h, run, &G, &m)) return rc;
    const size_t n = (size_t)G->g.n;
    if (omega_tilde_dev)
        CK(cudaMemcpyAsync(omega_tilde_dev, G->omega_t + (size_t)m * 3 * n, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice,
                           h->stream),
           "copy omega~");
    if (phi_tilde_dev)
        CK(cudaMemcpyAsync(phi_tilde_dev, G->phi_t + (size_t)m * 3 * n, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream),
           "copy Phi~");
    return EPD_LB_OK;
}

extern "C" int epd_lb_densities(epd_lb *h, int32_t run, double *phi, double *q)
{
    Group *G;
    int m;
    if (int rc = locate(h, run, &G, &m)) return rc;
    const size_t n = (size_t)G->g.n;
    if (phi) CK(cudaMemcpyAsync(phi, G->phi + (size_t)m * 3 * n, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy phi");
    if (q) CK(cudaMemcpyAsync(q, G->q + 2 * m, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy q");
    CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return EPD_LB_OK;
}

extern "C" int epd_lb_set_omega_async(epd_lb *h, int32_t run, const double *omega)
{
    Group *G;
    int m;
    if (int rc = locate(h, run, &G, &m)) return rc;
    if (!omega) return fail(h, EPD_LB_EINVAL, "omega is NULL");
    const size_t n = (size_t)G->g.n;
    CK(cudaMemcpyAsync(G->omega + (size_t)m * 3 * n, omega, 3 * n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy omega");
    G->phi_stale = true;  // the exact step recomputes Phi(t) before convecting it
    return EPD_LB_OK;
}

extern "C" int epd_lb_densities_async(epd_lb *h, int32_t run, double *phi, double *q)
{
    Group *G;
    int m;
    if (int rc = locate(h, run, &G, &m)) return rc;
    const size_t n = (size_t)G->g.n;
    if (phi) CK(cudaMemcpyAsync(phi, G->phi + (size_t)m * 3 * n, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy phi");
    if (q) CK(cudaMemcpyAsync(q, G->q + 2 * m, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy q");
    return EPD_LB_OK;
}

extern "C" int epd_lb_velocity_dev(epd_lb *h, int32_t run, double *v_dev)
{
    Group *G;
    int m;
    if (int rc = locate(h, run, &G, &m)) return rc;
    if (!v_dev) return fail(h, EPD_LB_EINVAL, "v_dev is NULL");
    CK(launch_vel_to_f64(*G, m, v_dev, h->stream), "velocity conversion");
    return EPD_LB_OK;
}

extern "C" int epd_lb_velocity(epd_lb *h, int32_t run, double *v)
{
    Group *G;
    int m;
    if (int rc = locate(h, run, &G, &m)) return rc;
    if (!v) return fail(h, EPD_LB_EINVAL, "v is NULL");
    const size_t n = (size_t)G->g.n;
    CK(launch_vel_to_f64(*G, m, G->stage, h->stream), "velocity conversion");
    CK(cudaMemcpyAsync(v, G->stage, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy velocity");
    CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return EPD_LB_OK;
}

extern "C" int epd_lb_get_state(epd_lb *h, int32_t run, double *omega, double *pop, double *vel)
{
    Group *G;
    int m;
    if (int rc = locate(h, run, &G, &m)) return rc;
    const size_t n = (size_t)G->g.n;
    if (omega) CK(cudaMemcpyAsync(omega, G->omega + (size_t)m * 3 * n, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy omega");
    if (pop) {
        CK(launch_gather_pre_collision(*G, m, h->parity, G->stage, h->stream), "gathering populations");
        CK(cudaMemcpyAsync(pop, G->stage, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy populations");
        CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    }
    if (vel) {
        CK(launch_vel_to_f64(*G, m, G->stage, h->stream), "velocity conversion");
        CK(cudaMemcpyAsync(vel, G->stage, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy velocity");
    }
    CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return EPD_LB_OK;
}

extern "C" int epd_lb_set_state(epd_lb *h, int32_t run, const double *omega, const double *pop, const double *vel)
{
    Group *G;
    int m;
    if (int rc = locate(h, run, &G, &m)) return rc;
    const size_t n = (size_t)G->g.n;
    if (omega)
        CK(cudaMemcpyAsync(G->omega + (size_t)m * 3 * n, omega, 3 * n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy omega");
    if (pop) {
        CK(cudaMemcpyAsync(G->stage, pop, 9 * n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy populations");
        CK(launch_scatter_pre_collision(*G, m, h->parity, G->stage, h->stream), "scattering populations");
    }
    if (vel) {
        // the staging buffer is reused: order the velocity upload after the scatter
        CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        CK(cudaMemcpyAsync(G->stage, vel, 2 * n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy velocity");
        CK(launch_vel_from_f64(*G, m, G->stage, h->stream), "velocity conversion");
    }
    if (omega) G->phi_stale = true;  // the exact step recomputes Phi(t) before convecting it
    CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return EPD_LB_OK;
}

extern "C" int epd_lb_solve(epd_lb *h, int32_t run, const double *omega, double *phi, double *q)
{
    Group *G;
    int m;
    if (int rc = locate(h, run, &G, &m)) return rc;
    if (!omega || !phi || !q) return fail(h, EPD_LB_EINVAL, "omega, phi and q are required");
    const size_t n = (size_t)G->g.n;
    Group V = run_view(*G, m);
    // omega~ and Phi~ are scratch between steps
    CK(cudaMemcpyAsync(V.omega_t, omega, 3 * n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy omega");
    CK(launch_solve(V, V.omega_t, V.phi_t, V.q_t, h->stream), "solve");
    CK(cudaMemcpyAsync(phi, V.phi_t, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy phi");
    CK(cudaMemcpyAsync(q, V.q_t, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy q");
    CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return EPD_LB_OK;
}

extern "C" int epd_lb_observables(epd_lb *h, int32_t run, double *out)
{
    Group *G;
    int m;
    if (int rc = locate(h, run, &G, &m)) return rc;
    if (!out) return fail(h, EPD_LB_EINVAL, "out is NULL");
    CK(launch_observables(*G, m, h->parity, h->part, h->obs, h->stream), "observables");
    CK(cudaMemcpyAsync(out, h->obs, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy observables");
    CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return EPD_LB_OK;
}

// Checkpoint format: magic, version, nruns, then per run its parameters and,
// as FP64, omega (3n), the stored post-collision population deviations (9n,
// the library's internal representation, copied exactly) and the velocity
// (2n).
static const uint64_t kMagic = 0x3130444C42445045ULL;  // "EPDLB01" little-endian

// Phi of the current omega for the analysis calls (set_state leaves it stale).
static int refresh_phi(epd_lb *h, Group &G)
{
    if (!G.phi_stale) return EPD_LB_OK;
    CK(launch_solve(G, G.omega, G.phi, G.q, h->stream), "solve");
    G.phi_stale = false;
    return EPD_LB_OK;
}

extern "C" int epd_lb_sigma_delta(epd_lb *h, int32_t run_a, int32_t run_b, double *out)
{
    Group *Ga, *Gb;
    int ma, mb;
    if (!out) return fail(h, EPD_LB_EINVAL, "out is NULL");
    if (int rc = locate(h, run_a, &Ga, &ma)) return rc;
    if (int rc = locate(h, run_b, &Gb, &mb)) return rc;
    if (Ga->g.nx != Gb->g.nx || Ga->g.ny != Gb->g.ny) return fail(h, EPD_LB_EINVAL, "the two runs have different grids");
    if (int rc = refresh_phi(h, *Ga)) return rc;
    if (int rc = refresh_phi(h, *Gb)) return rc;
    const size_t n = (size_t)Ga->g.n;
    CK(launch_sigma_delta(Ga->phi + (size_t)ma * 3 * n, Gb->phi + (size_t)mb * 3 * n, (long long)n, h->part, h->obs, h->stream), "sigma_Delta");
    CK(cudaMemcpyAsync(out, h->obs, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "reading sigma_Delta");
    CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return EPD_LB_OK;
}

extern "C" int epd_lb_width(epd_lb *h, int32_t run, double *out)
{
    Group *G;
    int m;
    if (!out) return fail(h, EPD_LB_EINVAL, "out is NULL");
    if (int rc = locate(h, run, &G, &m)) return rc;
    if (int rc = refresh_phi(h, *G)) return rc;
    CK(launch_width(*G, m, h->part, h->obs, h->stream), "Y_2^P");
    CK(cudaMemcpyAsync(out, h->obs, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "reading Y_2^P");
    CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return EPD_LB_OK;
}

extern "C" int epd_lb_particles(epd_lb *h, int32_t run, double threshold, int32_t max_particles, int32_t *count,
                                double *stats, int32_t *labels)
{
    Group *G;
    int m;
    if (!count) return fail(h, EPD_LB_EINVAL, "count is NULL");
    if (!(threshold > 0.0) || !std::isfinite(threshold)) return fail(h, EPD_LB_EINVAL, "threshold must be positive");
    if (max_particles < 0 || (max_particles > 0 && !stats)) return fail(h, EPD_LB_EINVAL, "bad max_particles or stats");
    if (int rc = locate(h, run, &G, &m)) return rc;
    if (int rc = refresh_phi(h, *G)) return rc;
    const long long n = G->g.n;
    const int maxp = max_particles;
    const size_t sb = particles_scratch_bytes(n, std::max(maxp, 1)) + (labels ? (size_t)n * sizeof(int) : 0);
    void *scratch = nullptr;
    CK(cudaMallocAsync(&scratch, sb, h->stream), "cudaMallocAsync");
    int *labels_dev = labels ? (int *)((char *)scratch + particles_scratch_bytes(n, std::max(maxp, 1))) : nullptr;
    int *total_dev = nullptr;
    double *stats_dev = nullptr;
    cudaError_t e = launch_particles(*G, m, threshold, std::max(maxp, 1), scratch, labels_dev, &total_dev, &stats_dev, h->stream);
    int total = 0, err = 0;
    if (!e) e = cudaMemcpyAsync(&total, total_dev, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (!e) e = cudaMemcpyAsync(&err, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (!e) e = cudaStreamSynchronize(h->stream);
    const int nout = std::min(total, maxp);
    if (!e && nout > 0) e = cudaMemcpy(stats, stats_dev, (size_t)nout * 10 * sizeof(double), cudaMemcpyDeviceToHost);
    if (!e && labels) e = cudaMemcpy(labels, labels_dev, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost);
    cudaFreeAsync(scratch, h->stream);
    cudaStreamSynchronize(h->stream);
    if (e) return cuda_fail(h, e, "particle analysis");
    if (err & 8) return fail(h, EPD_LB_ECUDA, "the cluster labelling did not finish");
    *count = total;
    return EPD_LB_OK;
}

extern "C" int epd_lb_save(epd_lb *h, void *buf, size_t *len)
{
    if (!h || !len) return EPD_LB_EINVAL;
    size_t need = 3 * sizeof(uint64_t);
    for (int r = 0; r < h->nruns; ++r) {
        const Group &G = h->groups[h->where[r].first];
        need += sizeof(epd_lb_params) + 14 * (size_t)G.g.n * sizeof(double);
    }
    if (!buf) {
        *len = need;
        return EPD_LB_OK;
    }
    if (*len < need) return fail(h, EPD_LB_ENOMEM, "checkpoint buffer too small");
    char *c = (char *)buf;
    uint64_t hdr[3] = {kMagic, 2, (uint64_t)h->nruns};
    std::memcpy(c, hdr, sizeof hdr);
    c += sizeof hdr;
    for (int r = 0; r < h->nruns; ++r) {
        Group &G = h->groups[h->where[r].first];
        const int m = h->where[r].second;
        const size_t n = (size_t)G.g.n;
        std::memcpy(c, &G.run_params[m], sizeof(epd_lb_params));
        c += sizeof(epd_lb_params);
        double *om = (double *)c, *pop = om + 3 * n, *vel = pop + 9 * n;
        if (int rc = epd_lb_get_state(h, r, om, nullptr, vel)) return rc;
        CK(launch_pop_raw(G, m, h->parity, G.stage, nullptr, h->stream), "copying populations");
        CK(cudaMemcpyAsync(pop, G.stage, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy populations");
        CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        c += 14 * n * sizeof(double);
    }
    *len = need;
    return EPD_LB_OK;
}

extern "C" int epd_lb_load(epd_lb *h, const void *buf, size_t len)
{
    if (!h || !buf) return EPD_LB_EINVAL;
    const char *c = (const char *)buf;
    uint64_t hdr[3];
    if (len < sizeof hdr) return fail(h, EPD_LB_EINVAL, "checkpoint truncated");
    std::memcpy(hdr, c, sizeof hdr);
    if (hdr[0] != kMagic || hdr[1] != 2 || hdr[2] != (uint64_t)h->nruns) return fail(h, EPD_LB_EINVAL, "checkpoint does not match this handle");
    c += sizeof hdr;
    size_t left = len - sizeof hdr;
    for (int r = 0; r < h->nruns; ++r) {
        Group &G = h->groups[h->where[r].first];
        const int m = h->where[r].second;
        const size_t n = (size_t)G.g.n;
        const size_t need = sizeof(epd_lb_params) + 14 * n * sizeof(double);
        if (left < need) return fail(h, EPD_LB_EINVAL, "checkpoint truncated");
        epd_lb_params p;
        std::memcpy(&p, c, sizeof p);
        if (std::memcmp(&p, &G.run_params[m], sizeof p) != 0)
            return fail(h, EPD_LB_EINVAL, "checkpoint parameters differ from this handle's");
        c += sizeof p;
        const double *om = (const double *)c, *pop = om + 3 * n, *vel = pop + 9 * n;
        if (int rc = epd_lb_set_state(h, r, om, nullptr, vel)) return rc;
        CK(cudaMemcpyAsync(G.stage, pop, 9 * n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy populations");
        CK(launch_pop_raw(G, m, h->parity, nullptr, G.stage, h->stream), "copying populations");
        Group V = run_view(G, m);
        CK(launch_solve(V, V.omega, V.phi, V.q, h->stream), "solve");
        CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        c += 14 * n * sizeof(double);
        left -= need;
    }
    for (Group &G : h->groups) G.phi_stale = false;  // every run was solved above
    return EPD_LB_OK;
}

extern "C" int epd_lb_enable_timing(epd_lb *h, int32_t on)
{
    if (!h) return EPD_LB_EINVAL;
    CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (on && !h->ev[0])
        for (int k = 0; k < 7; ++k) CK(cudaEventCreate(&h->ev[k]), "cudaEventCreate");
    h->timing = on != 0;
    return build_graphs(h);
}

extern "C" int epd_lb_kernel_times(epd_lb *h, double *ms)
{
    if (!h || !ms) return EPD_LB_EINVAL;
    if (!h->timing) return fail(h, EPD_LB_EINVAL, "timing is not enabled");
    CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    const int pairs[4][2] = {{0, 1}, {3, 4}, {2, 3}, {5, 6}};
    for (int k = 0; k < 4; ++k) {
        float t = 0.f;
        if (h->timed_cluster && (k == 1 || k == 2)) {
            ms[k] = 0.0;
            continue;
        }
        CK(cudaEventElapsedTime(&t, h->ev[pairs[k][0]], h->ev[pairs[k][1]]), "cudaEventElapsedTime");
        ms[k] = (double)t;
    }
    ms[4] = h->timed_cluster ? 1.0 : 0.0;
    return EPD_LB_OK;
}

extern "C" int epd_lb_tiles(epd_lb *h, int32_t run, int32_t *out)
{
    Group *G;
    int m;
    if (!out) return EPD_LB_EINVAL;
    if (int rc = locate(h, run, &G, &m)) return rc;
    (void)m;
    const bool cluster = G->hc && G->twx_full && cluster_solve_supported(*G);
    out[0] = cluster ? 2 : (G->hist_full ? 1 : 0);
    out[1] = cluster ? cluster_ctas(*G) : 0;
    out[2] = G->colw;
    out[3] = G->diff ? 1 : 0;
    out[4] = G->colw_prop;
    out[5] = cluster ? cluster_chain_launches(*G, G->diff) : 0;
    return EPD_LB_OK;
}

extern "C" const char *epd_lb_last_error(const epd_lb *h)
{
    if (!h) return "null handle";
    return h->last_error.c_str();
}

extern "C" void epd_lb_destroy(epd_lb *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (int k = 0; k < 2; ++k) {
        if (h->exec[k]) cudaGraphExecDestroy(h->exec[k]);
        if (h->exec_sur[k]) cudaGraphExecDestroy(h->exec_sur[k]);
        if (h->exec_chk[k]) cudaGraphExecDestroy(h->exec_chk[k]);
    }
    for (int k = 0; k < 7; ++k)
        if (h->ev[k]) cudaEventDestroy(h->ev[k]);
    for (auto e : h->fork_ev) cudaEventDestroy(e);
    for (auto e : h->join_ev) cudaEventDestroy(e);
    for (auto st : h->side) cudaStreamDestroy(st);
    if (h->own_ws && h->ws) cudaFree(h->ws);
    if (h->cg_host) cudaFreeHost(h->cg_host);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

// ---------------------------------------------------------------------------
// Stateless single-chain solve on device pointers.
// ---------------------------------------------------------------------------

// Only the buffers a solve touches: chain, history, factors, contour sums,
// partials and tables.
static size_t carve_solve(Group &G, char *base)
{
    const size_t n = (size_t)G.g.n;
    const size_t tb = G.prec == EPD_LB_MIXED_FP32 ? sizeof(float) : sizeof(double);
    size_t off = 0;
    auto take = [&](size_t bytes) -> void * {
        off = align_up(off);
        void *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    G.err = (int *)take(256);
    G.ia = (double *)take(n * sizeof(double));
    G.ib = (double *)take(n * sizeof(double));
    G.part = (double *)take(kMaxPart * sizeof(double));
    G.f0_lat = (double *)take(sizeof(double));
    G.chain = take(n * 2 * tb);
    G.hnodes = G.g.half_lo + 1;
    G.hist = take((size_t)G.hnodes * n * 2 * tb);
    G.efac = take(n * 2 * tb);
    G.twx = take((size_t)G.g.nx * 2 * tb);
    G.twy = take((size_t)G.g.ny * 2 * tb);
    G.kx = take((size_t)G.g.nx * tb);
    G.ky = take((size_t)G.g.ny * tb);
    G.twx_d = (double2 *)take((size_t)G.g.nx * sizeof(double2));
    G.twy_d = (double2 *)take((size_t)G.g.ny * sizeof(double2));
    return align_up(off);
}

// ---------------------------------------------------------------------------
// Stateless single-chain solve on a 3D box (nz x ny x nx).
// ---------------------------------------------------------------------------

constexpr long long kMaxSites3 = 1LL << 22;  // the row pass keeps one Q partial per 2048-site tile

// Geometry, tiles and (with base) the workspace layout; 0 when the box is
// not supported.
static size_t solve3_layout(const epd_lb_params *p, int nz, Solve3 &S, char *base)
{
    if (!p || !validate(*p).empty() || !smooth_even(nz) || nz > kMaxN) return 0;
    Group G = Group();
    G.p = *p;
    G.prec = p->precision;
    fill_geom(G);
    G.g.nruns = 1;
    const int nx = p->nx, ny = p->ny;
    const long long n3 = (long long)nx * ny * nz;
    if (n3 > kMaxSites3) return 0;
    const int nyz = ny * nz, nxy = nx * ny;
    S.vy = G.g;  // y columns: nz planes as runs
    S.vy.nruns = nz;
    S.vy.n = (long long)nxy;
    S.vx = G.g;  // x rows: ny nz rows of nx
    S.vx.ny = nyz;
    S.vx.n = n3;
    S.vx.pow2 = pow2(nx) && pow2(nyz);
    S.vx.logx = S.vx.pow2 ? ilog2(nx) : 0;
    S.vx.logy = S.vx.pow2 ? ilog2(nyz) : 0;
    S.vz = G.g;  // z pillars: nz rows of nx ny
    S.vz.nx = nxy;
    S.vz.ny = nz;
    S.vz.n = n3;
    S.vz.pow2 = pow2(nxy) && pow2(nz);
    S.vz.logx = S.vz.pow2 ? ilog2(nxy) : 0;
    S.vz.logy = S.vz.pow2 ? ilog2(nz) : 0;
    S.vz.nfy = radix_plan(nz, S.vz.fy);
    S.rows_x = divisor_at_most(nyz, std::max(1, 2048 / nx));
    S.cols_y = divisor_at_most(nx, std::max(2, 2048 / ny));
    S.cols_z = divisor_at_most(nxy, std::max(2, 2048 / nz));
    if (nyz / S.rows_x > kMaxPart / 2) return 0;  // Q partials of the row pass
    S.prec = p->precision;
    if (solve3d_smem_max(S) > 200 * 1024) return 0;
    const size_t tb = p->precision == EPD_LB_MIXED_FP32 ? sizeof(float) : sizeof(double);
    size_t off = 0;
    auto take = [&](size_t bytes) -> void * {
        off = align_up(off);
        void *q = base ? base + off : nullptr;
        off += bytes;
        return q;
    };
    S.err = (int *)take(256);
    S.ia = (double *)take((size_t)n3 * sizeof(double));
    S.ib = (double *)take((size_t)n3 * sizeof(double));
    S.part = (double *)take(kMaxPart * sizeof(double));
    S.chain = take((size_t)n3 * 2 * tb);
    S.hist = take((size_t)(G.g.half_lo + 1) * n3 * 2 * tb);
    S.efac = take((size_t)n3 * 2 * tb);
    S.twx = take((size_t)nx * 2 * tb);
    S.twy = take((size_t)ny * 2 * tb);
    S.twz = take((size_t)nz * 2 * tb);
    S.kx = take((size_t)nx * tb);
    S.ky = take((size_t)ny * tb);
    S.kz = take((size_t)nz * tb);
    return align_up(off);
}

// Twiddles exp(-2 pi i t / n), t < n, and (kf not null) factors exp(-R_G^2 k^2 ds) / n of one axis.
template <typename T>
static cudaError_t upload_axis(int n, double dx, double rg, double ds, void *tw, void *kf, cudaStream_t s)
{
    const double pi = 3.14159265358979323846;
    std::vector<T> t(2 * (size_t)n), k((size_t)n);
    for (int j = 0; j < n; ++j) {
        const double a = 2.0 * pi * (double)j / (double)n;
        t[2 * j] = (T)std::cos(a);
        t[2 * j + 1] = (T)-std::sin(a);
        const int mm = j <= n / 2 ? j : j - n;
        const double kk = 2.0 * pi * (double)mm / ((double)n * dx);
        k[j] = (T)(std::exp(-rg * rg * kk * kk * ds) / (double)n);
    }
    cudaError_t e = cudaMemcpyAsync(tw, t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    if (!e && kf) e = cudaMemcpyAsync(kf, k.data(), k.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    if (!e) e = cudaStreamSynchronize(s);  // the host vectors go out of scope
    return e;
}

extern "C" int epd_prop_solve3d_workspace_bytes(const epd_lb_params *p, int32_t nz, size_t *bytes)
{
    Solve3 S;
    if (!bytes) return EPD_LB_EINVAL;
    const size_t b = solve3_layout(p, nz, S, nullptr);
    if (!b) return EPD_LB_EINVAL;
    *bytes = b;
    return EPD_LB_OK;
}

extern "C" int epd_prop_solve3d(const epd_lb_params *p, int32_t nz, const double *omega_dev, double *phi_dev,
                                double *q_dev, void *workspace_dev, size_t workspace_bytes, void *cuda_stream)
{
    Solve3 S;
    if (!omega_dev || !phi_dev || !q_dev || !workspace_dev) return EPD_LB_EINVAL;
    const size_t need = solve3_layout(p, nz, S, nullptr);
    if (!need) return EPD_LB_EINVAL;
    if (workspace_bytes < need || ((uintptr_t)workspace_dev & 255)) return EPD_LB_ENOMEM;
    if (configure_kernels() != cudaSuccess) return EPD_LB_ECUDA;
    solve3_layout(p, nz, S, (char *)workspace_dev);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const double ds = 1.0 / (double)p->ns;
    cudaError_t e = cudaMemsetAsync(S.err, 0, sizeof(int), s);
    auto up = [&](int n, void *tw, void *kf) {
        return p->precision == EPD_LB_MIXED_FP32 ? upload_axis<float>(n, p->dx, p->rg, ds, tw, kf, s)
                                                 : upload_axis<double>(n, p->dx, p->rg, ds, tw, kf, s);
    };
    if (!e) e = up(p->nx, S.twx, S.kx);
    if (!e) e = up(p->ny, S.twy, S.ky);
    if (!e) e = up(nz, S.twz, S.kz);
    if (!e) e = launch_solve3d(S, omega_dev, phi_dev, q_dev, s);
    return e ? EPD_LB_ECUDA : EPD_LB_OK;
}

extern "C" int epd_lb3d_step(const epd_lb_params *p, int32_t nz, const double *pop_in_dev, const double *force_dev,
                             double *pop_out_dev, double *vel_dev, void *cuda_stream)
{
    if (!p || !validate(*p).empty() || !smooth_even(nz) || nz > kMaxN) return EPD_LB_EINVAL;
    if ((long long)p->nx * p->ny * nz > kMaxSites3) return EPD_LB_EINVAL;
    if (!pop_in_dev || !force_dev || !pop_out_dev || !vel_dev || pop_in_dev == pop_out_dev) return EPD_LB_EINVAL;
    const cudaError_t e = launch_lb3d_step(p->nx, p->ny, nz, p->gamma_s, p->gamma_b, p->gamma_g, pop_in_dev, force_dev,
                                           pop_out_dev, vel_dev, (cudaStream_t)cuda_stream);
    return e ? EPD_LB_ECUDA : EPD_LB_OK;
}

// The coupled 3D step: the 3D solve's layout plus the step's fields and the
// FP64 transform buffers and tables.
static Axis3 axis3(int n)
{
    Axis3 a = Axis3();
    a.n = n;
    a.pow2 = pow2(n);
    a.logn = a.pow2 ? ilog2(n) : 0;
    a.nf = radix_plan(n, a.f);
    return a;
}

static size_t step3_layout(const epd_lb_params *p, int nz, Step3 &T, char *base)
{
    const size_t sb = solve3_layout(p, nz, T.S, base);
    if (!sb) return 0;
    const int nx = p->nx, ny = p->ny;
    const long long n = (long long)nx * ny * nz;
    Fft3 &F = T.F;
    F.ax = axis3(nx);
    F.ay = axis3(ny);
    F.az = axis3(nz);
    F.rows_x = divisor_at_most(ny * nz, std::max(1, 2048 / nx));
    F.cols_y = divisor_at_most(nx, std::max(1, 2048 / ny));
    F.cols_z = divisor_at_most(nx * ny, std::max(1, 2048 / nz));
    if (fft3_smem(F) > 200 * 1024) return 0;
    size_t off = sb;
    auto take = [&](size_t bytes) -> void * {
        off = align_up(off);
        void *q = base ? base + off : nullptr;
        off += bytes;
        return q;
    };
    T.wt = (double *)take(3 * n * sizeof(double));
    T.pt = (double *)take(3 * n * sizeof(double));
    T.mu = (double *)take(3 * n * sizeof(double));
    T.qt = (double *)take(2 * sizeof(double));
    T.ftot = (double *)take(3 * n * sizeof(double));
    T.pop2 = (double *)take(19 * n * sizeof(double));
    T.b0 = (double2 *)take(n * sizeof(double2));
    T.b1 = (double2 *)take(n * sizeof(double2));
    F.twx = (const double2 *)take(nx * sizeof(double2));
    F.twy = (const double2 *)take(ny * sizeof(double2));
    F.twz = (const double2 *)take(nz * sizeof(double2));
    T.f0_lat = p->f0 * fstar_lattice(*p);
    return align_up(off);
}

extern "C" int epd_step3d_workspace_bytes(const epd_lb_params *p, int32_t nz, size_t *bytes)
{
    Step3 T;
    if (!bytes) return EPD_LB_EINVAL;
    const size_t b = step3_layout(p, nz, T, nullptr);
    if (!b) return EPD_LB_EINVAL;
    *bytes = b;
    return EPD_LB_OK;
}

extern "C" int epd_step3d(const epd_lb_params *p, int32_t nz, double *omega_dev, double *pop_dev, double *vel_dev,
                          double *phi_dev, double *q_dev, double *force_dev, void *workspace_dev, size_t workspace_bytes,
                          void *cuda_stream)
{
    Step3 T;
    if (!omega_dev || !pop_dev || !vel_dev || !phi_dev || !q_dev || !force_dev || !workspace_dev) return EPD_LB_EINVAL;
    const size_t need = step3_layout(p, nz, T, nullptr);
    if (!need) return EPD_LB_EINVAL;
    if (workspace_bytes < need || ((uintptr_t)workspace_dev & 255)) return EPD_LB_ENOMEM;
    if (configure_kernels() != cudaSuccess) return EPD_LB_ECUDA;
    step3_layout(p, nz, T, (char *)workspace_dev);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const double ds = 1.0 / (double)p->ns;
    cudaError_t e = cudaMemsetAsync(T.S.err, 0, sizeof(int), s);
    auto up = [&](int n, void *tw, void *kf) {
        return p->precision == EPD_LB_MIXED_FP32 ? upload_axis<float>(n, p->dx, p->rg, ds, tw, kf, s)
                                                 : upload_axis<double>(n, p->dx, p->rg, ds, tw, kf, s);
    };
    if (!e) e = up(p->nx, T.S.twx, T.S.kx);
    if (!e) e = up(p->ny, T.S.twy, T.S.ky);
    if (!e) e = up(nz, T.S.twz, T.S.kz);
    // FP64 twiddles of the EPD transforms
    if (!e) e = upload_axis<double>(p->nx, p->dx, p->rg, ds, (void *)T.F.twx, nullptr, s);
    if (!e) e = upload_axis<double>(p->ny, p->dx, p->rg, ds, (void *)T.F.twy, nullptr, s);
    if (!e) e = upload_axis<double>(nz, p->dx, p->rg, ds, (void *)T.F.twz, nullptr, s);
    if (!e) e = launch_step3d(T, omega_dev, pop_dev, vel_dev, phi_dev, q_dev, force_dev, s);
    return e ? EPD_LB_ECUDA : EPD_LB_OK;
}

extern "C" int epd_selftest_bounded_wait(int32_t limit_ms, void *cuda_stream, int32_t *timed_out)
{
    if (!timed_out || limit_ms < 1 || limit_ms > 2000) return EPD_LB_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, khz = 0;
    if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev)) return EPD_LB_ECUDA;
    int *err = nullptr, host = 0;
    if (cudaMallocAsync((void **)&err, sizeof(int), s)) return EPD_LB_ECUDA;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (!e) e = launch_selftest_wait(err, (long long)limit_ms * (long long)(khz > 0 ? khz : 2000000), s);
    if (!e) e = cudaMemcpyAsync(&host, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(err, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return EPD_LB_ECUDA;
    *timed_out = (host & 4) ? 1 : 0;
    return EPD_LB_OK;
}

static bool solve_group(const epd_lb_params *p, Group &G)
{
    if (!p || !validate(*p).empty()) return false;
    std::vector<Group> groups;
    std::vector<std::pair<int, int>> where;
    form_groups(p, 1, groups, where);
    G = groups[0];
    return true;
}

extern "C" int epd_prop_solve_workspace_bytes(const epd_lb_params *p, size_t *bytes)
{
    Group G;
    if (!bytes || !solve_group(p, G)) return EPD_LB_EINVAL;
    *bytes = carve_solve(G, nullptr);
    return EPD_LB_OK;
}

extern "C" int epd_prop_solve(const epd_lb_params *p, const double *omega_dev, double *phi_dev, double *q_dev,
                              void *workspace_dev, size_t workspace_bytes, void *cuda_stream)
{
    Group G;
    if (!solve_group(p, G) || !omega_dev || !phi_dev || !q_dev || !workspace_dev) return EPD_LB_EINVAL;
    if (workspace_bytes < carve_solve(G, nullptr) || ((uintptr_t)workspace_dev & 255)) return EPD_LB_ENOMEM;
    if (configure_kernels() != cudaSuccess) return EPD_LB_ECUDA;
    carve_solve(G, (char *)workspace_dev);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (cudaMemsetAsync(G.err, 0, sizeof(int), s) != cudaSuccess) return EPD_LB_ECUDA;
    if (upload_tables_e(G, s) != cudaSuccess) return EPD_LB_ECUDA;
    if (launch_solve(G, omega_dev, phi_dev, q_dev, s) != cudaSuccess) return EPD_LB_ECUDA;
    return EPD_LB_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free single-chain solve: the scratch of epd_prop_solve lives in a
// fixed array in the device image instead of a caller workspace.
// ---------------------------------------------------------------------------

namespace {

constexpr size_t kNoallocBytes = EPD_PROP_SOLVE_NOALLOC_MAX_BYTES;
constexpr int kNoallocDevices = 64;

// One copy per device that loads this library, held until the process exits.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Device address of g_noalloc_scratch on each device (host code must not use
// the symbol itself as an address).
std::atomic<void *> g_noalloc_addr[kNoallocDevices];

// Twiddles exp(-2 pi i t / n), t < n, and Fourier factors
// exp(-R_G^2 k^2 ds) / n (Eq. (8)), computed on the device in FP64.
template <typename T>
__global__ void noalloc_tables(int nx, int ny, double dx, double rg, double ds, V2<T> *twx, V2<T> *twy, T *kx, T *ky)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    auto twiddle = [](int t, int n, V2<T> *out) {
        double s, c;
        sincospi(2.0 * (double)t / (double)n, &s, &c);
        out[t] = mk<T>((T)c, (T)(-s));
    };
    auto factor = [&](int m, int n, T *out) {
        const double k = 2.0 * 3.14159265358979323846 * (double)signed_bin(m, n) / ((double)n * dx);
        out[m] = (T)(exp(-rg * rg * k * k * ds) / (double)n);
    };
    if (i < nx) twiddle(i, nx, twx);
    if (i < ny) twiddle(i, ny, twy);
    if (i < nx) factor(i, nx, kx);
    if (i < ny) factor(i, ny, ky);
}

template <typename T>
cudaError_t noalloc_launch_tables(Group &G, cudaStream_t s)
{
    const int m = std::max(G.g.nx, G.g.ny);
    noalloc_tables<T><<<(m + kThreads - 1) / kThreads, kThreads, 0, s>>>(
        G.g.nx, G.g.ny, G.g.dx, G.g.rg, G.g.ds, reinterpret_cast<V2<T> *>(G.twx), reinterpret_cast<V2<T> *>(G.twy),
        reinterpret_cast<T *>(G.kx), reinterpret_cast<T *>(G.ky));
    return cudaGetLastError();
}

} // namespace

extern "C" int epd_prop_solve_noalloc(const epd_lb_params *p, const double *omega_dev, double *phi_dev, double *q_dev,
                                      void *cuda_stream)
{
    if (!p || !omega_dev || !phi_dev || !q_dev || !validate(*p).empty()) return EPD_LB_EINVAL;
    Group G = Group();
    G.p = *p;
    G.prec = p->precision;
    fill_geom(G);
    G.g.nruns = 1;
    default_shapes(G);
    if (carve_solve(G, nullptr) > kNoallocBytes) return EPD_LB_ETOOLARGE;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocDevices) return EPD_LB_ECUDA;
    void *base = g_noalloc_addr[dev].load();
    if (!base) {
        if (cudaGetSymbolAddress(&base, g_noalloc_scratch) != cudaSuccess || !base) return EPD_LB_ECUDA;
        g_noalloc_addr[dev].store(base);
    }
    if (configure_kernels() != cudaSuccess) return EPD_LB_ECUDA;
    carve_solve(G, (char *)base);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the error word must start at zero; every other scratch buffer is written
    // before it is read within the call
    if (cudaMemsetAsync(G.err, 0, sizeof(int), s) != cudaSuccess) return EPD_LB_ECUDA;
    const cudaError_t e = G.prec == EPD_LB_MIXED_FP32 ? noalloc_launch_tables<float>(G, s) : noalloc_launch_tables<double>(G, s);
    if (e != cudaSuccess) return EPD_LB_ECUDA;
    if (launch_solve(G, omega_dev, phi_dev, q_dev, s) != cudaSuccess) return EPD_LB_ECUDA;
    return EPD_LB_OK;
}

// ---------------------------------------------------------------------------
// Learned density surrogate
// ---------------------------------------------------------------------------

static bool sur_shape_ok(const epd_lb_params *p, int batch)
{
    return p && validate(*p).empty() && batch > 0 && p->nx % 16 == 0 && p->ny % 16 == 0;
}

extern "C" int32_t epd_sur_num_params(void) { return sur::num_params(); }

extern "C" int epd_sur_workspace_bytes(int32_t ny, int32_t nx, int32_t batch, int32_t training, size_t *bytes)
{
    if (!bytes || batch <= 0 || nx % 16 || ny % 16 || nx <= 0 || ny <= 0) return EPD_LB_EINVAL;
    sur::Work w;
    *bytes = sur::carve(w, nullptr, batch, ny, nx, training != 0);
    return EPD_LB_OK;
}

static int sur_setup(const epd_lb_params *p, int32_t batch, bool training, void *workspace, size_t bytes, sur::Work &w)
{
    if (!sur_shape_ok(p, batch) || !workspace || ((uintptr_t)workspace & 255)) return EPD_LB_EINVAL;
    if (sur::carve(w, nullptr, batch, p->ny, p->nx, training) > bytes) return EPD_LB_ENOMEM;
    sur::carve(w, (char *)workspace, batch, p->ny, p->nx, training);
    return EPD_LB_OK;
}

extern "C" int epd_sur_forward(const epd_lb_params *p, int32_t batch, const float *params_dev, double s_in, double s_out,
                               const double *omega_dev, double *phi_dev, void *workspace, size_t workspace_bytes, void *cuda_stream)
{
    sur::Work w;
    if (!params_dev || !omega_dev || !phi_dev) return EPD_LB_EINVAL;
    if (int rc = sur_setup(p, batch, false, workspace, workspace_bytes, w)) return rc;
    const double na = (double)std::lround(p->f_a * (double)p->ns) / (double)p->ns;
    const cudaError_t e = sur::forward(w, params_dev, omega_dev, phi_dev, s_in, s_out, p->phi_p * na, p->phi_p * (1.0 - na),
                                       1.0 - p->phi_p, (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? EPD_LB_OK : EPD_LB_ECUDA;
}

extern "C" int epd_sur_tangent(const epd_lb_params *p, int32_t batch, const float *params_dev, double s_in, double s_out,
                               const double *omega0_dev, const double *omega_dev, double *phi0_dev, double *phi_dev, void *workspace,
                               size_t workspace_bytes, void *cuda_stream)
{
    sur::Work w;
    if (!params_dev || !omega0_dev || !omega_dev || !phi0_dev || !phi_dev) return EPD_LB_EINVAL;
    if (int rc = sur_setup(p, batch, false, workspace, workspace_bytes, w)) return rc;
    const double na = (double)std::lround(p->f_a * (double)p->ns) / (double)p->ns;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = sur::forward(w, params_dev, omega0_dev, phi0_dev, s_in, s_out, p->phi_p * na, p->phi_p * (1.0 - na),
                                 1.0 - p->phi_p, s);
    if (e == cudaSuccess) e = sur::tangent(w, params_dev, omega_dev, omega0_dev, phi0_dev, phi_dev, s_in, s_out, 1.0 - p->phi_p, s);
    return e == cudaSuccess ? EPD_LB_OK : EPD_LB_ECUDA;
}

extern "C" int epd_sur_gradients(const epd_lb_params *p, int32_t batch, const float *params_dev, double s_in, double s_out,
                                 const double *omega_dev, const double *phi_dev, float *grad_dev, double *loss_dev, void *workspace,
                                 size_t workspace_bytes, void *cuda_stream)
{
    sur::Work w;
    if (!params_dev || !omega_dev || !phi_dev || !grad_dev || !loss_dev) return EPD_LB_EINVAL;
    if (int rc = sur_setup(p, batch, true, workspace, workspace_bytes, w)) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (sur::gradients(w, params_dev, omega_dev, phi_dev, s_in, s_out, loss_dev, s) != cudaSuccess) return EPD_LB_ECUDA;
    if (cudaMemcpyAsync(grad_dev, w.grad, (size_t)sur::num_params() * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return EPD_LB_ECUDA;
    return EPD_LB_OK;
}

extern "C" int epd_sur_train_step(const epd_lb_params *p, int32_t batch, float *params_dev, float *adam_m_dev, float *adam_v_dev,
                                  int32_t step, float lr, double s_in, double s_out, const double *omega_dev, const double *phi_dev,
                                  double *loss_dev, void *workspace, size_t workspace_bytes, void *cuda_stream)
{
    sur::Work w;
    if (!params_dev || !adam_m_dev || !adam_v_dev || !omega_dev || !phi_dev || !loss_dev || step < 1) return EPD_LB_EINVAL;
    if (int rc = sur_setup(p, batch, true, workspace, workspace_bytes, w)) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (sur::gradients(w, params_dev, omega_dev, phi_dev, s_in, s_out, loss_dev, s) != cudaSuccess) return EPD_LB_ECUDA;
    if (sur::adam_step(w, params_dev, adam_m_dev, adam_v_dev, step, lr, s) != cudaSuccess) return EPD_LB_ECUDA;
    return EPD_LB_OK;
}

static size_t handle_sur_bytes(epd_lb *h)
{
    size_t off = 0;
    off = align_up(off + (size_t)sur::num_params() * sizeof(float));
    off = align_up(off + (h->groups.size() + 1) * sizeof(double));
    for (auto &G : h->groups) {
        sur::Work w;
        off = align_up(off + sur::carve(w, nullptr, G.g.nruns, G.g.ny, G.g.nx, false));
    }
    return off;
}

extern "C" int epd_lb_surrogate_workspace_bytes(epd_lb *h, size_t *bytes)
{
    if (!h || !bytes) return EPD_LB_EINVAL;
    for (auto &G : h->groups)
        if (G.g.nx % 16 || G.g.ny % 16) return fail(h, EPD_LB_EINVAL, "the surrogate needs nx % 16 == 0 and ny % 16 == 0");
    *bytes = handle_sur_bytes(h);
    return EPD_LB_OK;
}

extern "C" int epd_lb_set_surrogate(epd_lb *h, const float *params_host, double s_in, double s_out, int32_t exact_every,
                                    double residual_tol, int32_t hold_force, void *workspace, size_t workspace_bytes)
{
    if (!h) return EPD_LB_EINVAL;
    CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (exact_every <= 0) {
        h->sur_on = false;
        return EPD_LB_OK;
    }
    if (h->cg_max > 0) return fail(h, EPD_LB_EINVAL, "the exact step and the surrogate exclude each other");
    size_t need = 0;
    if (int rc = epd_lb_surrogate_workspace_bytes(h, &need)) return rc;
    if (!params_host || !workspace || workspace_bytes < need || ((uintptr_t)workspace & 255))
        return fail(h, EPD_LB_EINVAL, "surrogate parameters or workspace missing or too small");
    char *base = (char *)workspace;
    size_t off = 0;
    h->sur_params = (float *)(base + off);
    off = align_up(off + (size_t)sur::num_params() * sizeof(float));
    h->sur_resid = (double *)(base + off);
    off = align_up(off + (h->groups.size() + 1) * sizeof(double));
    h->sur_work.assign(h->groups.size(), sur::Work());
    for (size_t gi = 0; gi < h->groups.size(); ++gi) {
        Group &G = h->groups[gi];
        const size_t b = sur::carve(h->sur_work[gi], base + off, G.g.nruns, G.g.ny, G.g.nx, false);
        h->sur_work[gi].err = h->err;  // epd_lb_sync reports a convolution that gave up a wait
        off = align_up(off + b);
    }
    CK(cudaMemcpyAsync(h->sur_params, params_host, (size_t)sur::num_params() * sizeof(float), cudaMemcpyHostToDevice, h->stream),
       "copy surrogate parameters");
    // the parameters stay fixed while attached: pack the weights once, outside the step graphs
    for (auto &W : h->sur_work) CK(sur::prepare(W, h->sur_params, h->stream), "packing the surrogate weights");
    CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    h->sur_on = true;
    h->sur_every = exact_every;
    h->sur_tol = residual_tol;
    h->sur_s_in = s_in;
    h->sur_s_out = s_out;
    h->sur_hold = hold_force != 0;
    h->sur_steps = h->sur_exact = h->sur_used = h->sur_forced = 0;
    h->sur_fallback = false;
    h->sur_last = 0.0;
    return build_graphs(h);
}

extern "C" int epd_lb_surrogate_stats(epd_lb *h, double *out)
{
    if (!h || !out) return EPD_LB_EINVAL;
    out[0] = (double)h->sur_steps;
    out[1] = (double)h->sur_exact;
    out[2] = (double)h->sur_used;
    out[3] = (double)h->sur_forced;
    out[4] = h->sur_last;
    out[5] = h->sur_fallback ? 1.0 : 0.0;
    return EPD_LB_OK;
}

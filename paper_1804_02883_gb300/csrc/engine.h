// engine.h -- host-side description of a batch of runs ("group") and the
// launchers of the kernels that make up one hybrid LB/EPD time step.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/epd_lb.h"

namespace epdlb {

// Parameters every kernel of a group needs, by value.
constexpr int kMaxFactors = 16;  // radices of one axis (mixed-radix transforms)

struct GroupGeom {
    int nx, ny, logx, logy;  // logx, logy: 0 unless both axes are powers of two
    int pow2;                // both axes powers of two; else the mixed-radix radix-2-family passes
    int nfx, nfy;            // radix plans (4, 2, 3, 5) of each axis for the mixed-radix transforms
    int fx[kMaxFactors], fy[kMaxFactors];
    int ns, na;          // contour steps, A-block intervals round(f_a ns)
    int jr;              // junction rule: 0 literal, 1 segment-symmetric
    int half_lo, half_hi;  // nodes 0..half_lo are stored; nodes >= half_hi accumulate
    int nruns;
    long long n;         // sites per run
    double dx, dt, rg, nseg, phi_p, ds;
    double chi_ab, chi_as, chi_bs, kappa_h, d_s, d_p, inv_beta_v;
    double gamma_s, gamma_b, gamma_g;
    double fstar;        // f* in lattice units
    double vscale;       // lattice velocity -> R_G/tau
};

// Block (0: A, 1: B) whose field acts in a half-step of the split step of
// Eq. (8) at contour node m of a chain (0: g from the A end; 1: g', which
// sees the field of position 1 - s).  arriving: the half-step that ends the
// interval into node m; otherwise the one that starts the interval out of
// it.  jr = 0 (literal): both take the field of node m, A iff the node of g
// it corresponds to is below N_A (the junction node takes B).  jr = 1
// (segment-symmetric): each takes the block of its own interval (A iff that
// interval of g is below N_A); at the two ends of the chain, which have one
// interval only, both half-steps take that interval's block.
__host__ __device__ inline int half_step_block(int jr, int chain, int m, int ns, int na, bool arriving)
{
    if (jr == 0) return (chain == 0 ? m : ns - m) >= na;
    if (arriving ? m == 0 : m == ns) arriving = !arriving;
    const int j = arriving ? m - 1 : m;  // the interval of this chain
    return (chain == 0 ? j : ns - 1 - j) >= na;
}

// Launch shapes of the transform passes (chosen at init, see tune_shapes).
struct Shapes {
    int rows_prop, cols_prop;  // rows per CTA of the propagator row pass, columns per CTA of its column pass
    int rows_epd, cols_epd;    // the same for the FP64 EPD/force passes
};

// One batch of runs with identical grid, contour and model parameters.
struct Group {
    epd_lb_params p;   // parameters of the first run (f0 and seed may differ per run)
    GroupGeom g;
    Shapes sh;
    int prec;          // EPD_LB_PLAIN_FP64 or EPD_LB_MIXED_FP32
    std::vector<int> run_ids;  // handle-level run index of each member
    std::vector<epd_lb_params> run_params;

    // FP64 fields, [run][species][n]
    double *omega, *omega_t, *phi, *phi_t;
    double *q, *q_t;   // [run][2]
    double *ia, *ib;   // contour sums, [run][n]
    double *ia2, *ib2; // contour sums of the g' chain's terms (cluster solve), [run][n]
    // differential second solve (MIXED_FP32).  Cluster solve: states of both
    // chains at every node, in the padded row layout
    // [run][chain][ns+1][ny/2][nx + nx/8] float2 (hc: plain / reference
    // solve; hd: differential solve).  Streaming solves: hd holds the changes
    // (dg, dg') at every node, [run][ns+1][n] float2, against the reference
    // history in hist.
    void *hc = nullptr;
    void *hd = nullptr;
    void *rho = nullptr;      // (rho_A, rho_B) = expm1(-N d omega ds / 2), [run][n] float2
    void *cdiff = nullptr;    // (1 + rho_d)(1 + rho_a) - 1 for (A,A), (B,B), (A,B), packed rows [run][3][ny/2][nx] float2
    bool diff = false;        // the step uses the reference + differential solve pair
    bool phi_stale = false;   // omega was replaced since phi was last computed
    bool hist_full = false;   // streaming radix-8 solve (hist holds all N_s + 1 nodes)
    int hnodes = 0;           // nodes of hist per run: N_s + 1 (MIXED streaming solves) or half_lo + 1
    int colw = 0;             // radix-8 EPD column tile width chosen by the autotuner (0: default)
    int colw_prop = 0;        // radix-8 streaming propagator column tile width (0: default)
    // exact step (CG inversion of App. C), FP64 [run][3][n] unless noted
    double *cg_target = nullptr;  // Phi~ = Phi(t) - dt div(v Phi(t))
    double *cg_dir = nullptr;     // search direction d
    double *cg_trial = nullptr;   // omega + alpha_t d
    double *cg_wref = nullptr, *cg_pref = nullptr;  // reference omega, Phi of the differential solves (MIXED)
    double *cg_qref = nullptr;    // [run][2]
    double *cg_part = nullptr;    // reduction partials [run][kCgBlocks][2]
    double *cg = nullptr;         // per-run scalars [run][kCgSlots]
    double2 *cz;       // 4 complex FP64 scratch planes per run: [run][4][n]
    double *part;      // reduction partials, [run][kMaxPart]
    double *f0_lat;    // [run]
    void *f0_bulk;     // [run], the same in the bulk type
    double *stage;     // host<->device staging, 9 n doubles (one run)
    // bulk-precision buffers (float or double, by prec)
    void *chain;       // packed (g, g') of the running contour step, [run][n] complex
    void *hist;        // (g, g') at nodes 0..hnodes-1, [run][hnodes][n] complex
    void *efac;        // (E_A, E_B), [run][n] complex
    void *pop[2];      // post-collision populations, [run][9][n]
    void *vel;         // velocity of the last collision, [run][n] complex (x, y)
    void *force;       // polymer force (lattice units), [run][n] complex (x, y)
    // transform tables
    void *twx, *twy, *kx, *ky;     // bulk precision: twiddles, exp(-rg^2 k^2 ds)/N
    double2 *twx_d, *twy_d;        // FP64 twiddles for the EPD/force passes
    float2 *twx_full, *twy_full;   // FP32 twiddles exp(-2 pi i j/N), j < N (cluster solve); may be null
    float2 *tab8x = nullptr, *tab8y = nullptr;  // radix-8 pass tables (fft8.cuh layout); null with twx_full
    float2 *tab16x = nullptr, *tab16y = nullptr;  // radix-16 plan tables of 256-point axes (else null)
    int *err;                      // device error word (shared by the handle)
};

constexpr int kMaxPart = 4096;     // partial sums per run and reduction
constexpr int kCgBlocks = 304;     // blocks per run of the inversion's dot products (2 per SM)
constexpr int kCgSlots = 16;       // per-run scalars of the inversion

// Fletcher-Reeves inversion omega~ = Phi^{-1}(Phi~) (invert.cu).  Slots of G.cg.
enum CgSlot { CG_GG = 0, CG_H0, CG_AT, CG_ALPHA, CG_RES, CG_RES0, CG_ITERS, CG_ACTIVE, CG_BETA };
// g = target - phi; gg, residual, d = -g, h0 = -gg, alpha_t = 1, iterations 0
cudaError_t cg_begin(Group &G, const double *phi, double tol, cudaStream_t s);
// trial point omega + alpha_t d of the active runs (omega itself for the others)
cudaError_t cg_trial_point(Group &G, const double *omega, double *trial, cudaStream_t s);
// slope at the trial densities, the secant step alpha, omega += alpha d
cudaError_t cg_line_step(Group &G, const double *phi_trial, double *omega, cudaStream_t s);
// new mismatch from phi: residual, beta, the new direction, convergence flags
cudaError_t cg_direction(Group &G, const double *phi, double tol, cudaStream_t s);

// Workspace layout: compute (dry run with base == nullptr) or carve.
size_t carve_group(Group &G, char *base, size_t off);

// Tables and initial state.
void upload_tables(Group &G, cudaStream_t s);
cudaError_t launch_init_state(Group &G, cudaStream_t s);

// Optional CUDA events recorded around single launches of a solve (for timing
// inside a captured step): ev[0], ev[1] bracket the row pass of node m_store;
// ev[2], ev[3] the column pass before node m_acc and ev[3], ev[4] its row pass.
// With the cluster-resident solve, ev[0], ev[1] bracket its chain launch (all
// launches of the phased schedule) and `cluster` is set.
struct SolveProbe {
    cudaEvent_t ev[5];
    int m_store, m_acc;
    mutable bool cluster = false;
};

// Single-chain solve, Eqs. (6)-(11): omega (3n per run, FP64) -> phi (3n),
// q (2 per run).  All runs of the group.
cudaError_t launch_solve(Group &G, const double *omega, double *phi, double *q, cudaStream_t s,
                         const SolveProbe *probe = nullptr);
// Second solve of the step as a difference from the reference solve at
// omega~ (phi_t, q_t): Phi(t+dt) = Phi~ + dPhi, Q likewise (G.diff only).
cudaError_t launch_solve_delta(Group &G, cudaStream_t s, const SolveProbe *probe = nullptr);
// The same at any omega against a given reference: omega_ref with its
// densities phi_ref, q_ref, whose chain states the last plain solve stored
// (G.hc, or G.hist on the streaming paths) and whose Boltzmann factors are in
// G.efac.
cudaError_t launch_solve_delta_at(Group &G, const double *omega, const double *omega_ref, const double *phi_ref,
                                  const double *q_ref, double *phi, double *q, cudaStream_t s,
                                  const SolveProbe *probe = nullptr);

// Column tile autotuner of the radix-8 column passes (sets G.colw).
cudaError_t tune_column_tiles(Group &G, cudaStream_t s);
cudaError_t tune_stream_tiles(Group &G, cudaStream_t s);  // sets G.colw_prop

// EPD parts of the step.
cudaError_t launch_aux_convection(Group &G, cudaStream_t s);   // omega, vel -> omega_t
cudaError_t launch_convect_phi(Group &G, const double *phi, double *phi_dst, cudaStream_t s);  // Phi - dt div(v Phi)
cudaError_t launch_diffusion(Group &G, cudaStream_t s);        // phi_t, omega_t -> omega
cudaError_t launch_force(Group &G, cudaStream_t s);            // phi, phi_t -> force
cudaError_t launch_lb(Group &G, int parity, cudaStream_t s);   // pop[parity] -> pop[1-parity], vel

// Analysis of Phi_P (analysis.cu): sigma_Delta of Eq. (22), Y_2^P of
// Eq. (30), particles with their gyration tensors (Eqs. (27)-(29)).
cudaError_t launch_sigma_delta(const double *phi_a, const double *phi_b, long long n, double *part, double *out_dev, cudaStream_t s);
cudaError_t launch_width(const Group &G, int run, double *part, double *out_dev, cudaStream_t s);
size_t particles_scratch_bytes(long long n, int maxp);
// labels_dev (n int, may be null); *total_dev, *stats_dev point into scratch
cudaError_t launch_particles(const Group &G, int run, double thr, int maxp, void *scratch, int *labels_dev,
                             int **total_dev, double **stats_dev, cudaStream_t s);

// State access helpers (one run).
cudaError_t launch_gather_pre_collision(Group &G, int run, int parity, double *dst, cudaStream_t s);
cudaError_t launch_scatter_pre_collision(Group &G, int run, int parity, const double *src, cudaStream_t s);
cudaError_t launch_vel_to_f64(Group &G, int run, double *dst, cudaStream_t s);
cudaError_t launch_vel_from_f64(Group &G, int run, const double *src, cudaStream_t s);
// Two-stage reductions of the observables and the analysis: a fixed grid of
// at most kRedBlocks blocks writes kRedSlots partials per block into part
// (kRedSlots * kRedBlocks doubles), one block sums them in a fixed order, so a
// rerun is bitwise equal.
constexpr int kRedBlocks = 304;
constexpr int kRedSlots = 8;
cudaError_t launch_observables(Group &G, int run, int parity, double *part, double *out_dev, cudaStream_t s);
// Exact copy of a run's stored populations to (dst) or from (src) FP64.
cudaError_t launch_pop_raw(Group &G, int run, int parity, double *dst, const double *src, cudaStream_t s);

// Cluster-resident solve (prop_cluster.cu): availability for the group's
// shape and precision, its launch, and its CTAs per run.
bool cluster_solve_supported(const Group &G);
bool cluster_shape_exists(int logx, int logy);
// Launches of the chain kernel per cluster-resident solve (diff: the
// differential one): 1, or 2 nruns when the chains are one more than the
// clusters that fit at one CTA per SM (the phased schedule); 0 without a shape.
int cluster_chain_launches(const Group &G, bool diff);
// MIXED grids solved by the radix-8 streaming passes with the full history
bool stream8_eligible(int prec, int logx, int logy);
size_t cluster_state_floats2(int nx, int ny, int ns);  // per run, both chains
// Chain launch plus contour sums and normalisation into phi, q (diff: the
// differential solve into G.phi, G.q).  nprep_blocks: solvent partials.
cudaError_t launch_cluster_solve(Group &G, cudaStream_t s, bool diff, int nprep_blocks, double *phi, double *q,
                                 const SolveProbe *probe, const double *phi_ref = nullptr, const double *q_ref = nullptr);
int cluster_ctas(const Group &G);
// The bounded exchange wait of prop_chain on a barrier nothing arrives on:
// sets bit 2 of *err after limit_cycles (test of the failure path).
cudaError_t launch_selftest_wait(int *err, long long limit_cycles, cudaStream_t s);

// Single-chain solve on an nz x ny x nx box (layout [z][y][x]): the
// streaming passes over three views of one array, z pillars (a 2D view with
// nz rows of nx ny sites), y columns (nz planes as runs) and x rows (ny nz
// rows) carrying the node factors, history and contour sums.
struct Solve3 {
    GroupGeom vx, vy, vz;        // the three views (vx holds the chain geometry)
    int rows_x, cols_y, cols_z;  // tiles of the x-row, y-column and z-column passes
    void *chain, *hist, *efac;   // bulk precision: [n3] complex, [half_lo + 1][n3] complex, [n3] complex
    double *ia, *ib, *part;
    void *twx, *twy, *twz, *kx, *ky, *kz;  // bulk precision tables (full twiddle tables)
    int *err;
    int prec;
};
cudaError_t launch_solve3d(const Solve3 &S, const double *omega, double *phi, double *q, cudaStream_t s);
size_t solve3d_smem_max(const Solve3 &S);  // largest dynamic shared memory of the three passes
// One axis of the FP64 3D transforms of the coupled 3D step.
struct Axis3 {
    int n, pow2, logn, nf;
    int f[kMaxFactors];
};
struct Fft3 {
    Axis3 ax, ay, az;
    int rows_x, cols_y, cols_z;    // tiles of the x-row, y-column and z-column transforms
    const double2 *twx, *twy, *twz;  // FP64 twiddles exp(-2 pi i t / n), t < n
};
size_t fft3_smem(const Fft3 &F);
// The coupled step on a 3D box (step3d.cu): state omega (3n), pop (19n,
// pre-collision), vel (3n); outputs phi (3n), q (2), force (3n).
struct Step3 {
    Solve3 S;
    Fft3 F;
    double *wt, *pt, *mu, *qt, *ftot, *pop2;  // omega~, Phi~, mu / dPhi, Q~, total force, populations out
    double2 *b0, *b1;                         // complex FP64 transform buffers [n]
    double f0_lat;                            // body-force amplitude, lattice units
};
cudaError_t launch_step3d(const Step3 &T, double *omega, double *pop, double *vel, double *phi, double *q, double *force,
                          cudaStream_t s);
cudaError_t configure_step3d_kernels();

// D3Q19 collide-stream on an nz x ny x nx box, FP64 ([19][z][y][x] in, out).
cudaError_t launch_lb3d_step(int nx, int ny, int nz, double gs, double gb, double gg, const double *in,
                             const double *force, double *out, double *vel, cudaStream_t s);

// Kernel attributes (dynamic shared memory limits), once per process.
cudaError_t configure_kernels();

// Smallest/largest supported sizes.
constexpr int kMinN = 8, kMaxN = 2048;

} // namespace epdlb

// surrogate.h -- host interface of the learned density surrogate (surrogate.cu).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace epdlb {
namespace sur {

// Architecture: 3 -> 32 -> 32 -> 32 -> 2 channels, 3x3 kernels of dilation
// 1, 2, 2, 4.
constexpr int kLayers = 4;
constexpr int kCin[kLayers] = {3, 32, 32, 32};
constexpr int kCout[kLayers] = {32, 32, 32, 2};
// Master parameters (FP32): per layer W[co][ci][tap] then b[co].
int num_params();
int param_offset_w(int layer);
int param_offset_b(int layer);

// Device buffers of one evaluation / training batch, carved from a workspace.
struct Work {
    int nb, nx, ny;
    long long n;
    bool training;
    void *x0, *y[3], *y4, *yf[3], *dz[2], *dz4;
    void *t0, *t[2], *t4;  // tangent pass: input, hidden tangents (BF16), output (FP32)
    double *means2;
    int *err;              // device error word: bit 2 = a bounded wait of a convolution gave up
    unsigned *cnt;         // arrival counter of the one-launch reductions (0 between launches)
    bool cnt_ready = false;  // cnt zeroed on this workspace
    bool prepacked = false;  // forward weights packed for the parameters in use (prepare)
    void *wf[kLayers], *wb[kLayers];
    float *dwpart, *grad;
    double *means, *ymean, *qs, *tmean, *lpart, *red;
    double *bpart;         // bias-gradient partials [block][32] (training)
    int nblk_dw;
};

size_t carve(Work &w, char *base, int nb, int ny, int nx, bool training);

// For a fixed parameter set used by many forward / tangent calls (the time
// stepper): zero the reduction counter and pack the forward weights once;
// forward then skips the packing.
cudaError_t prepare(Work &w, const float *params, cudaStream_t s);
// Forward pass: omega [nb][3][n] FP64 -> phi [nb][3][n] FP64.
cudaError_t forward(Work &w, const float *params, const double *omega, double *phi, double s_in, double s_out, double pa_bar,
                    double pb_bar, double ps_bar, cudaStream_t s);
// Densities at omega from the surrogate at omega0 to first order in the
// change: phi = phi0 + the tangent pass along omega - omega0 (Phi_A, Phi_B);
// Phi_S from Eq. (11) at omega.  The forward pass at omega0 must have run on
// w last (its activations, the means of omega0 and <exp(-omega0_S)> are
// reused).
cudaError_t tangent(Work &w, const float *params, const double *omega, const double *omega0, const double *phi0, double *phi,
                    double s_in, double s_out, double ps_bar, cudaStream_t s);
// Loss and parameter gradient for targets phi_t; loss to loss_dev[0].
cudaError_t gradients(Work &w, const float *params, const double *omega, const double *phi_t, double s_in, double s_out,
                      double *loss_dev, cudaStream_t s);
// gradients, then one Adam step on params with moments m, v.
cudaError_t adam_step(Work &w, float *params, float *m, float *v, int step, float lr, cudaStream_t s);

// Per run sqrt(sum |phi_a - phi_b|^2 / sum |phi_b - <phi_b>|^2) over the A and
// B densities (the error relative to the fluctuations of phi_b), max over
// runs, to out[0].
cudaError_t residual_rel(const double *phi_a, const double *phi_b, long long n, int nb, double *tmp, double *out, cudaStream_t s);
// RMS of (phi_a - phi_b) per run, max over runs, to out[0].
cudaError_t residual_rms(const double *phi_a, const double *phi_b, long long n, int nb, double *tmp, double *out, cudaStream_t s);

} // namespace sur
} // namespace epdlb

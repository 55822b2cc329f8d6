// surrogate.h -- host interface of the learned density surrogate (surrogate.cu).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace epdlb {
namespace sur {

// Architecture: 3 -> 32 -> 32 -> 32 -> 2 channels, 3x3 kernels.
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
    void *wf[kLayers], *wb[kLayers];
    float *dwpart, *grad;
    double *means, *ymean, *qs, *tmean, *lpart, *red;
    int nblk_dw;
};

size_t carve(Work &w, char *base, int nb, int ny, int nx, bool training);

// Forward pass: omega [nb][3][n] FP64 -> phi [nb][3][n] FP64.
cudaError_t forward(Work &w, const float *params, const double *omega, double *phi, double s_in, double s_out, double pa_bar,
                    double pb_bar, double ps_bar, cudaStream_t s);
// Loss and parameter gradient for targets phi_t; loss to loss_dev[0].
cudaError_t gradients(Work &w, const float *params, const double *omega, const double *phi_t, double s_in, double s_out,
                      double *loss_dev, cudaStream_t s);
// gradients, then one Adam step on params with moments m, v.
cudaError_t adam_step(Work &w, float *params, float *m, float *v, int step, float lr, cudaStream_t s);

// RMS of (phi_a - phi_b) per run, max over runs, to out[0].
cudaError_t residual_rms(const double *phi_a, const double *phi_b, long long n, int nb, double *tmp, double *out, cudaStream_t s);

} // namespace sur
} // namespace epdlb

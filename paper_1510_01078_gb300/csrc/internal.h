// Internal declarations shared by the plan (nedner_api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/nedner.h"
#include "window.h"

namespace nedner {

// Geometry and constants passed by value to every kernel.
struct Geo {
    int M, Nt, nx, ny, nz;
    int Lx, Ly, Lt;        // oversampled lengths sigma*nx, sigma*ny, sigma*Nt
    int w, D;              // window taps, degree of the tap polynomials
    int nxh, nyp;          // nx/2 + 1, ny + 1 (rows of the half lattice)
    float az_hi, az_lo;    // (c Nt dt / Z)^2 as a float-float pair
    float sqrt_az;         // c Nt dt / Z
    float scale;           // s / (nx ny nz) (weighted) or 1 / (nx ny nz)
    int apply_weights;
    int band_mask;
};

// Work-split choices made once per plan.
struct Chunks {
    int c1;   // time samples per CTA in the spread + x-FFT stage
    int c2;   // time samples per CTA in the y-FFT stage
    int c4;   // depth planes per CTA in the y-IFFT stage
    int c5;   // image rows per CTA in the x-c2r stage
    size_t smem1, smem2, smem3, smem4, smem5;
};

// Device-side tables owned by a plan.
struct DevTables {
    float2* tw = nullptr;         // [TW_N] exp(-2 pi i k / TW_N)
    float* deconv_x = nullptr;    // [nx/2+1]   1/phihat(jx / Lx)
    float* deconv_y = nullptr;    // [ny+1]     1/phihat(jy / Ly), jy = -ny/2..ny/2
    float* deconv_t = nullptr;    // [Nt]       1/phihat((n - Nt/2) / Lt)
    float* tapcoef = nullptr;     // [w][D+1]   monomial coefficients of the tap polynomials
    float2* axy = nullptr;        // [nx/2+1][ny+1] (c Nt dt)^2 ((jx/X)^2 + (jy/Y)^2), float-float
    int* sens_bx = nullptr;       // [M] first x tap, mod Lx
    int* sens_by = nullptr;       // [M] first y tap, mod Ly
    float* sens_wx = nullptr;     // [M][w] x taps phi(u_x - (bx + k))
    float* sens_wy = nullptr;     // [M][w] y taps (without the sensor factor)
    float* sens_dwx = nullptr;    // [M][w] d phi / d x_m (per metre)
    float* sens_dwy = nullptr;    // [M][w] d phi / d y_m (per metre)
    float* sens_fac = nullptr;    // [M] w_m = h_m/(dx dy) or 1
    int* row_ptr = nullptr;       // [Ly+1] CSR of (sensor, y tap) entries by grid row
    int* row_m = nullptr;         // [M w] sensor of each entry
    float* row_w = nullptr;       // [M w] y tap times sensor factor
};

}  // namespace nedner

struct nedner_plan_s {
    nedner::Geo geo;
    nedner::Chunks ch;
    nedner::Window win;
    int64_t M = 0;
    int Nt = 0;
    double dt = 0, c = 0, sigma = 2;
    nedner_grid grid{};
    std::vector<double> xy, h;
    nedner::DevTables t;
    void* ws = nullptr;           // device workspace
    size_t ws_bytes = 0;
    size_t region_a = 0;          // bytes of region A (R / V), region B follows (Ghat / Y)
    int device = 0;
};

namespace nedner {

// forward-stage launchers (kernels_fwd.cu); return cudaGetLastError()
cudaError_t launch_ned_spread_xfft(const nedner_plan_s& p, const float* g, float2* R, cudaStream_t s);
cudaError_t launch_ned_yfft(const nedner_plan_s& p, const float2* R, float2* Ghat, cudaStream_t s);
cudaError_t launch_ner_lines(const nedner_plan_s& p, const float2* Ghat, float2* V, cudaStream_t s);
cudaError_t launch_img_yifft(const nedner_plan_s& p, const float2* V, float2* Y, cudaStream_t s);
cudaError_t launch_img_xc2r(const nedner_plan_s& p, const float2* Y, float* p0, cudaStream_t s);
cudaError_t configure_fwd_kernels(const nedner_plan_s& p);

}  // namespace nedner

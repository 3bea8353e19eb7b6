// Internal declarations shared by the plan (nedner_api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/nedner.h"
#include "window.h"

namespace nedner {

// taps per entry of the adjoint's block gather: the 16 + w - 1 columns an
// entry starting anywhere in a 16-column block can reach, rounded up to 4
// entries per staged batch of a warp of the block spread
constexpr int SPREAD_BATCH = 8;    // 16 was measured slower on C3 (0.81 against 0.76 ms): 5 CTAs per SM instead of 6

__host__ __device__ constexpr int gather_aligned_taps(int w) { return (16 + w - 1 + 3) / 4 * 4; }

// bits of the device status word (DevTables::status)
constexpr int NEDNER_FLAG_NONFINITE = 2;

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
    int c2f;  // time samples per CTA in the y-FFT stage and its transpose
    int c4;   // depth planes per CTA in the y-IFFT stage
    int c5;   // image rows per CTA in the x-c2r stage
    int groups1;   // lane groups (column segments) per CTA in the spread stage
    int threads1;  // threads per CTA in the spread stage
    int per1;      // values per thread in the spread stage's in-place x-FFT (16 or 32)
    int tpl1;      // time samples per lane in the spread stage (1 or 2)
    int split1;    // 1: stage (a) runs as block spread + x-FFT + y-FFT over chunks of tq samples
    int tq;        // time samples per chunk of the split stage (a multiple of 64 dividing Nt)
    int wpc_s;     // warps (16-column blocks) per CTA of the block spread
    int nbx;       // complex columns (time-sample pairs) per CTA of the x-FFT kernel
    int thx;       // threads per CTA of the x-FFT kernel
    int perx;      // values per thread of its in-place FFT (16 or 32)
    size_t smem_s, smem_x;
    int gsplit;    // 1: the transposed interpolation runs as transposed x-FFT + block gather per pass of tp_g samples
    int tp_g;      // time samples per pass of the block gather (its grid Q-bar is held in region A after R-bar)
    size_t smem_ga, smem_gg;   // shared memory of the block gather (adjoint, gradient)
    int ca;        // time samples per CTA in the transposed interpolation stage
    int per_adj;   // values per thread in its in-place row FFT (16 or 32)
    int tpl_adj;   // time samples per lane in the transposed gather (1 or 2; 2 means ca = 64)
    int threads_adj;   // threads of the two-sample gather CTA (256, or 512 for 2nx = 512)
    int tp_adj;    // time samples per pass of the transposed gather (its entry buffer holds M w tp_adj floats)
    int lpc;       // line groups per CTA in the NER stage
    int icap3a;    // depth frequencies of one line held at a time by the transposed NER
    int threads3;  // threads per CTA in the NER stage
    size_t smem1, smem2f, smem3, smem3a, smem4, smem5;   // smem3a: the transposed NER
    size_t smem_adj, smem_grad;
};


// Monomial coefficients of the NER interpolation taps, passed by value to the
// NER kernels so that they are read as constant-bank operands.
struct TapPoly {
    float c[16 * 13];   // [k][d], k < w <= 16, d <= D <= 12
};

// Taps stored per spreading entry: w taps placed after up to 3 leading zeros
// (first column aligned to 4), rounded up to a multiple of 4.
inline int spread_taps(int w) { return ((w + 3) + 3) / 4 * 4; }

// Device-side tables owned by a plan.
struct DevTables {
    float2* tw = nullptr;         // [2 TW_N] exp(-2 pi i k / N) at [N + k], N = 1, 2, 4, .., TW_N
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
    float* row_dw = nullptr;      // [M w] y-tap derivative (per metre) times sensor factor
    // spreading: per row, entries sorted by first x column, wrapped ones repeated at bx - Lx
    int* xrow_ptr = nullptr;      // [Ly+1]
    int* xent_m = nullptr;        // [E'] sensor
    float* xent_wx = nullptr;     // [E'][spread_taps(w)] taps from column xent_bx on (x tap times y tap times sensor factor)
    int* xent_bx = nullptr;       // [E'] first x column rounded down to a multiple of 4
    float* xent_gx = nullptr;     // [E'][spread_taps(w)] x-tap derivative times y tap times sensor factor
    float* xent_gy = nullptr;     // [E'][spread_taps(w)] x tap times y-tap derivative times sensor factor
    int* xrow_first = nullptr;    // [Ly] first entry of the row that is not a wrapped entry's second copy
    int* xent_rc = nullptr;       // [E'] the entry's index in the row CSR
    int* sens_ent = nullptr;      // [M][w] row-CSR index of each of the sensor's y taps
    int4* seg = nullptr;          // [Ly][groups1] column range [x, y) and entry range [z, w)
    // the block spread (split1): per (row, 16-column block) the range of
    // entries whose exact taps reach into the block, and per entry its exact
    // first column and its w taps
    int2* bseg = nullptr;         // [Ly][Lx/16] range of the block's entries in bent_m / bent_w
    int* bent_m = nullptr;        // [.] sensor of each (block, entry reaching into it)
    float* bent_w = nullptr;      // [.][16] its taps aligned to the block's columns (block_taps16)
    int* pent_bx = nullptr;       // [E'] first x column (negative for the second copy of a wrapped entry)
    float* pent_w = nullptr;      // [E'][gather_aligned_taps(w)] x tap times y tap times sensor factor, aligned to
                                  // the 32-column window of the entry's 16-column block (the adjoint's block gather)
    float* pent_gx = nullptr;     // [E'][4 ceil(w/4)] the same with the x-tap derivative (position gradient)
    float* pent_gy = nullptr;     // [E'][4 ceil(w/4)] the same with the y-tap derivative
    int2* gseg = nullptr;         // [Ly][Lx/16] entries whose first column lies in the block (block gather)
    int* status = nullptr;        // device flags: NEDNER_FLAG_NONFINITE when an output kernel wrote a non-finite value
    int* lp_kcut = nullptr;       // [M] highest kept frequency bin of the data low-pass (nedner_lowpass)
};

// Stage timer of the profiled entry points (defined in nedner_api.cu): marks
// the stream after a launch, attributing the time since the previous mark to
// the named stage.
struct StageTimer;
void stage_mark(StageTimer* tm, int stage);

// Tensor-product NED state (tcgen05 GEMM path).
struct TPState {
    int enabled = 0;
    int sms = 0;                  // multiprocessors of the device
    void* work = nullptr;         // device: operand matrices of the data, GEMM 1 output, Nyquist line
    size_t work_bytes = 0;
    void* ex = nullptr;           // device BF16: 4 matrices (Re hi, Re lo, Im hi, Im lo), rows jx < nx/2, K = a
    void* ey = nullptr;           // device BF16: 2 tiles x 4 matrices (Re hi/lo, Im hi/lo), rows jy, K = b
    float2* exn = nullptr;        // device FP32: Ex row jx = nx/2
    float2* eyf = nullptr;        // device FP32: Ey [ny+1][nys]
    int* err = nullptr;           // device flag: a bounded wait ran out
    int fp16 = 0;                 // operands FP16 (else BF16)
    int wait_limit = 1 << 26;     // polls of the pipeline waits (nedner_debug_set_wait_limit); drains keep 1 << 26
    unsigned int* absmax = nullptr;   // device word: bits of max |w_m g| (FP16 mode's data scale)
};

}  // namespace nedner

struct nedner_plan_s {
    nedner::Geo geo;
    nedner::Chunks ch;
    nedner::Window win;
    int64_t M = 0;
    int Nt = 0;
    double dt = 0, c = 0, sigma = 2;
    int ner_interp = NEDNER_NER_KB;   // nedner_opts.ner_interp
    nedner_grid grid{};
    std::vector<double> xy, h;
    std::vector<int> lp_kcut;     // host copy of t.lp_kcut
    nedner::DevTables t;
    nedner::TapPoly tap{};
    nedner::TPState tp;
    void* ws = nullptr;           // device workspace
    size_t ws_bytes = 0;
    size_t region_a = 0;          // bytes of region A (R / V), region B follows (Ghat / Y)
    int device = 0;
    // nedner_forward_host: device copies of g and p0, copy streams and their
    // events (created by the first call)
    float* host_g = nullptr;
    float* host_p0 = nullptr;
    cudaStream_t copy_stream[4] = {};
    cudaEvent_t host_ev[16] = {};
};

namespace nedner {

// forward-stage launchers (kernels_fwd.cu); return cudaGetLastError()
// the spread and y-FFT stages for time samples [t0, t0 + nt) (nt < 0: to the
// end; t0 and nt multiples of 64), the x-c2r stage for depth planes [z0, z0 + nzc)
cudaError_t launch_ned_spread_xfft(const nedner_plan_s& p, const float* g, float2* R, cudaStream_t s, int t0 = 0,
                                   int nt = -1);
cudaError_t launch_ned_yfft(const nedner_plan_s& p, const float2* R, float2* Ghat, cudaStream_t s, int t0 = 0,
                            int nt = -1, int rstride = -1, int roff = 0);
// stage (a) in chunks of tq time samples: block spread into Q, x-FFT into R
// (both one chunk), y-FFT into Ghat; Q and R hold tq samples
cudaError_t launch_ned_stage_split(const nedner_plan_s& p, const float* g, float* Q, float2* R, float2* Ghat,
                                   cudaStream_t s, StageTimer* tm = nullptr);
cudaError_t launch_ner_lines(const nedner_plan_s& p, const float2* Ghat, float2* V, cudaStream_t s);
cudaError_t launch_img_yifft(const nedner_plan_s& p, const float2* V, float2* Y, cudaStream_t s);
cudaError_t launch_img_xc2r(const nedner_plan_s& p, const float2* Y, float* p0, cudaStream_t s, int z0 = 0,
                            int nzc = -1);
cudaError_t configure_fwd_kernels(const nedner_plan_s& p);

// transposed-stage launchers (kernels_adj.cu)
cudaError_t launch_img_xr2c_adj(const nedner_plan_s& p, const float* p0, float2* Y, cudaStream_t s);
cudaError_t launch_img_yfft_adj(const nedner_plan_s& p, const float2* Y, float2* V, cudaStream_t s);
cudaError_t launch_ner_lines_adj(const nedner_plan_s& p, const float2* V, float2* Ghat, cudaStream_t s);
cudaError_t launch_ned_yfft_adj(const nedner_plan_s& p, const float2* Ghat, float2* R, cudaStream_t s);
// the gather and its sum run once per pass of time samples; a timer, if
// given, is marked after each (stages 4 and 5 of the transposed path)
cudaError_t launch_adj_gather(const nedner_plan_s& p, const float2* R, float* E, float* g, cudaStream_t s,
                              StageTimer* tm = nullptr);
cudaError_t launch_grad_gather(const nedner_plan_s& p, const float2* R, const float* g, float2* Qe, float* dxy,
                               cudaStream_t s, StageTimer* tm = nullptr);
cudaError_t configure_adj_kernels(const nedner_plan_s& p);

// tensor-product NED (kernels_tp.cu)
cudaError_t configure_tp_kernels();
cudaError_t launch_tp_ned(const nedner_plan_s& p, const float* g, float2* Ghat, cudaStream_t s);
int tp_chunk(int Nt);   // time samples per pass of the tensor-core stage (a)
// data low-pass (kernels_util.cu): each sensor's distance to its nearest
// neighbour (infinite for a lone sensor), and the highest kept DFT bin of
// f_cut = c / (2 dx_m)
std::vector<double> nearest_neighbour_distance(const std::vector<double>& xy, int64_t M, double X, double Y);
std::vector<int> lowpass_bins(const nedner_plan_s& p);
size_t tp_work_bytes(int Nt);
constexpr int TP_SENSORS = 128;   // sensors per axis the tensor-core path is built for
constexpr int TP_WAIT_LIMIT = 1 << 26;   // polls of a bounded mbarrier wait

}  // namespace nedner

// Register-window helpers of the NED spread (Eq. NED_NUFFT, Sec. 3.2), used by
// the spread kernels in kernels_fwd.cu; see the description of the sweep there.
// A lane group sweeps the entries of one column segment [c0, c1) of a grid row
// in first-column order, holding the 2 WT columns [base, base + 2 WT) of its
// time sample(s) in registers.  Also the spread stage's output step.  They
// need only padx and the complex helpers (fft.cuh) and the plan geometry, so
// the same header also builds on the host for tests.
#pragma once

#include <cuda_runtime.h>

#include "fft.cuh"
#include "internal.h"

namespace nedner {

template <int WT>
__device__ __forceinline__ void flush_lower(float (&acc)[2 * WT], float* Zf, int lnb, int hl, int base, int c0,
                                            int c1) {
#pragma unroll
    for (int k = 0; k < WT; ++k) {
        const int col = base + k;
        if (col >= c0 && col < c1) Zf[2 * padx((col << lnb) + (hl >> 1)) + (hl & 1)] = acc[k];
        acc[k] = acc[k + WT];
        acc[k + WT] = 0.f;
    }
}

// taps applied to column pairs with packed FP32x2 FMAs
template <int WT, int D>
__device__ __forceinline__ void add_taps(float (&acc)[2 * WT], const float4 (&wv)[WT / 4], float gval) {
    const float2 g2 = make_float2(gval, gval);
#pragma unroll
    for (int k4 = 0; k4 < WT / 4; ++k4) {
        float2 lo = __ffma2_rn(make_float2(wv[k4].x, wv[k4].y), g2,
                               make_float2(acc[D + 4 * k4 + 0], acc[D + 4 * k4 + 1]));
        float2 hi = __ffma2_rn(make_float2(wv[k4].z, wv[k4].w), g2,
                               make_float2(acc[D + 4 * k4 + 2], acc[D + 4 * k4 + 3]));
        acc[D + 4 * k4 + 0] = lo.x;
        acc[D + 4 * k4 + 1] = lo.y;
        acc[D + 4 * k4 + 2] = hi.x;
        acc[D + 4 * k4 + 3] = hi.y;
    }
}

// one entry: slide the window to bx4, then add its taps at d = bx4 - base
template <int WT>
__device__ __forceinline__ void sweep_entry(float (&acc)[2 * WT], float* Zf, int lnb, int hl, int& base, int c0,
                                            int c1, int bx4, const float4 (&wv)[WT / 4], float gval) {
    while (bx4 - base > WT) {
        flush_lower<WT>(acc, Zf, lnb, hl, base, c0, c1);
        base += WT;
    }
    const int d = (bx4 - base) >> 2;
    if (d == 0) add_taps<WT, 0>(acc, wv, gval);
    else if (d == 1) add_taps<WT, 4>(acc, wv, gval);
    else if (d == 2) add_taps<WT, (WT >= 8 ? 8 : 0)>(acc, wv, gval);
    else if (WT >= 12 && d == 3) add_taps<WT, (WT >= 12 ? 12 : 0)>(acc, wv, gval);
    else if (WT >= 16 && d == 4) add_taps<WT, (WT >= 16 ? 16 : 0)>(acc, wv, gval);
    else if (WT >= 20 && d == 5) add_taps<WT, (WT >= 20 ? 20 : 0)>(acc, wv, gval);
}

// Two time samples per lane (C = 64 per CTA, lane groups of a full warp): the
// lane's samples 2 ln, 2 ln + 1 are exactly complex column ln of the row, so
// the register window holds float2 pairs, every tap is applied to both with
// one packed FMA, and a finished column is one 8-byte store.
template <int WT>
__device__ __forceinline__ void flush_lower2(float2 (&acc)[2 * WT], float2* Z, int ln, int base, int c0, int c1) {
#pragma unroll
    for (int k = 0; k < WT; ++k) {
        const int col = base + k;
        if (col >= c0 && col < c1) Z[padx((col << 5) + ln)] = acc[k];
        acc[k] = acc[k + WT];
        acc[k + WT] = make_float2(0.f, 0.f);
    }
}

template <int WT, int D>
__device__ __forceinline__ void add_taps2(float2 (&acc)[2 * WT], const float4 (&wv)[WT / 4], float2 g2) {
#pragma unroll
    for (int k4 = 0; k4 < WT / 4; ++k4) {
        acc[D + 4 * k4 + 0] = __ffma2_rn(make_float2(wv[k4].x, wv[k4].x), g2, acc[D + 4 * k4 + 0]);
        acc[D + 4 * k4 + 1] = __ffma2_rn(make_float2(wv[k4].y, wv[k4].y), g2, acc[D + 4 * k4 + 1]);
        acc[D + 4 * k4 + 2] = __ffma2_rn(make_float2(wv[k4].z, wv[k4].z), g2, acc[D + 4 * k4 + 2]);
        acc[D + 4 * k4 + 3] = __ffma2_rn(make_float2(wv[k4].w, wv[k4].w), g2, acc[D + 4 * k4 + 3]);
    }
}

template <int WT>
__device__ __forceinline__ void sweep_entry2(float2 (&acc)[2 * WT], float2* Z, int ln, int& base, int c0, int c1,
                                             int bx4, const float4 (&wv)[WT / 4], float2 g2) {
    while (bx4 - base > WT) {
        flush_lower2<WT>(acc, Z, ln, base, c0, c1);
        base += WT;
    }
    const int d = (bx4 - base) >> 2;
    if (d == 0) add_taps2<WT, 0>(acc, wv, g2);
    else if (d == 1) add_taps2<WT, 4>(acc, wv, g2);
    else if (d == 2) add_taps2<WT, (WT >= 8 ? 8 : 0)>(acc, wv, g2);
    else if (WT >= 12 && d == 3) add_taps2<WT, (WT >= 12 ? 12 : 0)>(acc, wv, g2);
    else if (WT >= 16 && d == 4) add_taps2<WT, (WT >= 16 ? 16 : 0)>(acc, wv, g2);
    else if (WT >= 20 && d == 5) add_taps2<WT, (WT >= 20 ? 20 : 0)>(acc, wv, g2);
}

// Block spread (k_ned_spread_blocks): one warp accumulates one block of 16
// columns [c0, c0 + 16) of a grid row for 64 time samples (two per lane)
// over every entry whose w taps reach into the block.  The plan stores, for
// every (grid row, 16-column block) and every entry reaching into the block,
// the entry's taps aligned to the block's columns (block_taps16: column c of
// the block gets tap c0 + c - bx, zero where that is not one of the w taps),
// so that adding an entry is 16 packed FMAs whatever its offset.
__host__ __device__ inline void block_taps16(int bx, int c0, const float* taps, int w, float* out) {
    for (int c = 0; c < 16; ++c) {
        const int k = c0 + c - bx;
        out[c] = (k >= 0 && k < w) ? taps[k] : 0.f;
    }
}

__device__ __forceinline__ void block_entry16(float2 (&acc)[16], const float4 (&t)[4], float2 g2) {
#pragma unroll
    for (int c4 = 0; c4 < 4; ++c4) {
        acc[4 * c4 + 0] = __ffma2_rn(make_float2(t[c4].x, t[c4].x), g2, acc[4 * c4 + 0]);
        acc[4 * c4 + 1] = __ffma2_rn(make_float2(t[c4].y, t[c4].y), g2, acc[4 * c4 + 1]);
        acc[4 * c4 + 2] = __ffma2_rn(make_float2(t[c4].z, t[c4].z), g2, acc[4 * c4 + 2]);
        acc[4 * c4 + 3] = __ffma2_rn(make_float2(t[c4].w, t[c4].w), g2, acc[4 * c4 + 3]);
    }
}

// Output step of the spread stage: jx = 0..nx/2 of the row, divided by
// phihat(jx/Lx), for complex column b (real time samples 2b, 2b+1 packed as
// real and imaginary part), written as the two time samples n0 + 2b, n0 + 2b + 1
// of R.  With fold, the x-FFT's last radix-2 pass is done here (see block_fft_ip).
__device__ __forceinline__ void spread_output(const Geo& G, const float2* Z, int lnb, int b, int jx, bool fold,
                                              const float* __restrict__ deconv_x, const float2* __restrict__ tw,
                                              int gy, int n0, float2* __restrict__ R) {
    const int Lx = G.Lx;
    float2 zk, zm;
    if (fold) {
        const int H = Lx >> 1;
        const float2 a0 = Z[padx((jx << lnb) + b)], a1 = Z[padx(((jx + H) << lnb) + b)];
        if (jx == 0) {
            zk = cadd(a0, a1);
            zm = cconj(zk);
        } else {
            const float2 w = __ldg(&tw[Lx + jx]);                       // exp(-2 pi i jx / Lx)
            const float2 b0 = Z[padx(((H - jx) << lnb) + b)], b1 = Z[padx(((Lx - jx) << lnb) + b)];
            zk = cadd(a0, cmul(w, a1));
            zm = cconj(cadd(b0, cmul(cconj(w), b1)));                     // conj X[Lx - jx]
        }
    } else {
        zk = Z[padx((jx << lnb) + b)];
        zm = cconj(Z[padx((((Lx - jx) & (Lx - 1)) << lnb) + b)]);
    }
    // column 2b = (Z[k] + conj Z[-k]) / 2, column 2b+1 = -i (Z[k] - conj Z[-k]) / 2
    const float d = 0.5f * __ldg(&deconv_x[jx]);
    const float2 x0 = cscale(cadd(zk, zm), d);
    const float2 x1 = cscale(mul_i(csub(zk, zm), -1), d);
    *reinterpret_cast<float4*>(&R[((size_t)jx * G.Ly + gy) * G.Nt + n0 + 2 * b]) = make_float4(x0.x, x0.y, x1.x, x1.y);
}

}  // namespace nedner

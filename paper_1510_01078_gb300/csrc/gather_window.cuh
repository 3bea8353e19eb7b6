// Register-window helpers of the transposed interpolation (the transpose of
// the NED spread, Eq. NED_NUFFT, Sec. 3.2), used by the gather kernels in
// kernels_adj.cu.  A lane group walks the entries of a grid row in
// first-column order, holding the 2 WT columns [base, base + 2 WT) of the
// rebuilt real row (read modulo Lx) for its time sample(s) in registers, and
// forms each entry's tap-weighted sum.  They need only padx (fft.cuh) and
// float2/float4 arithmetic, so the same header also builds on the host for
// tests.
#pragma once

#include <cuda_runtime.h>

#include "fft.cuh"

namespace nedner {

// float offset of real sample (column c, time sample ln) in the padded row:
// 2 padx(c C/2 + ln/2) + ln%2
__device__ __forceinline__ int rpos(int c, int lnb, int ln) { return 2 * padx((c << lnb) + (ln >> 1)) + (ln & 1); }

// Register window of the rebuilt row for one lane: win[k] = r[(base + k) mod Lx],
// k < 2 WT.  A lane group walks entries sorted by first column; an entry
// more than WT columns ahead of base first slides the window by WT.
template <int WT>
__device__ __forceinline__ void win_load(float (&win)[2 * WT], const float* Zf, int lnb, int ln, int Lx, int base,
                                         int k0) {
#pragma unroll
    for (int k = 0; k < WT; ++k) win[k0 + k] = Zf[rpos((base + k0 + k) & (Lx - 1), lnb, ln)];
}

template <int WT>
__device__ __forceinline__ void win_advance(float (&win)[2 * WT], const float* Zf, int lnb, int ln, int Lx, int& base,
                                            int bx4) {
    while (bx4 - base > WT) {
#pragma unroll
        for (int k = 0; k < WT; ++k) win[k] = win[k + WT];
        base += WT;
        win_load<WT>(win, Zf, lnb, ln, Lx, base, WT);
    }
}

// sum_k taps[k] win[D + k] (two tap sets at once when TWO)
template <int WT, int D, bool TWO>
__device__ __forceinline__ float2 win_dot(const float (&win)[2 * WT], const float4* ta, const float4* tb) {
    float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
#pragma unroll
    for (int k4 = 0; k4 < WT / 4; ++k4) {
        const float4 t4 = ta[k4];
        a0 = fmaf(t4.x, win[D + 4 * k4 + 0], a0);
        a1 = fmaf(t4.y, win[D + 4 * k4 + 1], a1);
        a0 = fmaf(t4.z, win[D + 4 * k4 + 2], a0);
        a1 = fmaf(t4.w, win[D + 4 * k4 + 3], a1);
        if (TWO) {
            const float4 u4 = tb[k4];
            b0 = fmaf(u4.x, win[D + 4 * k4 + 0], b0);
            b1 = fmaf(u4.y, win[D + 4 * k4 + 1], b1);
            b0 = fmaf(u4.z, win[D + 4 * k4 + 2], b0);
            b1 = fmaf(u4.w, win[D + 4 * k4 + 3], b1);
        }
    }
    return make_float2(a0 + a1, b0 + b1);
}

// the entry at bx4 = base + 4 d, d = 0 .. WT/4 (uniform across the lane group)
template <int WT, bool TWO>
__device__ __forceinline__ float2 win_entry(const float (&win)[2 * WT], int d, const float4* ta, const float4* tb) {
    if (d == 0) return win_dot<WT, 0, TWO>(win, ta, tb);
    if (d == 1) return win_dot<WT, 4, TWO>(win, ta, tb);
    if (d == 2) return win_dot<WT, (WT >= 8 ? 8 : 0), TWO>(win, ta, tb);
    if (WT >= 12 && d == 3) return win_dot<WT, (WT >= 12 ? 12 : 0), TWO>(win, ta, tb);
    if (WT >= 16 && d == 4) return win_dot<WT, (WT >= 16 ? 16 : 0), TWO>(win, ta, tb);
    return win_dot<WT, (WT >= 20 ? 20 : 0), TWO>(win, ta, tb);
}

// Two time samples per lane (C = 64 per CTA): the lane's samples 2 ln, 2 ln + 1
// are complex column ln of the packed row, so the window holds float2 pairs
// and every tap is one packed FMA.
template <int WT>
__device__ __forceinline__ void win2_load(float2 (&win)[2 * WT], const float2* Z, int ln, int Lx, int base, int k0) {
#pragma unroll
    for (int k = 0; k < WT; ++k) win[k0 + k] = Z[padx((((base + k0 + k) & (Lx - 1)) << 5) + ln)];
}

template <int WT>
__device__ __forceinline__ void win2_advance(float2 (&win)[2 * WT], const float2* Z, int ln, int Lx, int& base,
                                             int bx4) {
    while (bx4 - base > WT) {
#pragma unroll
        for (int k = 0; k < WT; ++k) win[k] = win[k + WT];
        base += WT;
        win2_load<WT>(win, Z, ln, Lx, base, WT);
    }
}

template <int WT, int D, bool TWO>
__device__ __forceinline__ void win2_dot(const float2 (&win)[2 * WT], const float4* ta, const float4* tb, float2& va,
                                         float2& vb) {
    float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
#pragma unroll
    for (int k4 = 0; k4 < WT / 4; ++k4) {
        const float4 t4 = ta[k4];
        a0 = __ffma2_rn(make_float2(t4.x, t4.x), win[D + 4 * k4 + 0], a0);
        a1 = __ffma2_rn(make_float2(t4.y, t4.y), win[D + 4 * k4 + 1], a1);
        a0 = __ffma2_rn(make_float2(t4.z, t4.z), win[D + 4 * k4 + 2], a0);
        a1 = __ffma2_rn(make_float2(t4.w, t4.w), win[D + 4 * k4 + 3], a1);
        if (TWO) {
            const float4 u4 = tb[k4];
            b0 = __ffma2_rn(make_float2(u4.x, u4.x), win[D + 4 * k4 + 0], b0);
            b1 = __ffma2_rn(make_float2(u4.y, u4.y), win[D + 4 * k4 + 1], b1);
            b0 = __ffma2_rn(make_float2(u4.z, u4.z), win[D + 4 * k4 + 2], b0);
            b1 = __ffma2_rn(make_float2(u4.w, u4.w), win[D + 4 * k4 + 3], b1);
        }
    }
    va = __fadd2_rn(a0, a1);
    vb = __fadd2_rn(b0, b1);
}

template <int WT, bool TWO>
__device__ __forceinline__ void win2_entry(const float2 (&win)[2 * WT], int d, const float4* ta, const float4* tb,
                                           float2& va, float2& vb) {
    if (d == 0) win2_dot<WT, 0, TWO>(win, ta, tb, va, vb);
    else if (d == 1) win2_dot<WT, 4, TWO>(win, ta, tb, va, vb);
    else if (d == 2) win2_dot<WT, (WT >= 8 ? 8 : 0), TWO>(win, ta, tb, va, vb);
    else if (WT >= 12 && d == 3) win2_dot<WT, (WT >= 12 ? 12 : 0), TWO>(win, ta, tb, va, vb);
    else if (WT >= 16 && d == 4) win2_dot<WT, (WT >= 16 ? 16 : 0), TWO>(win, ta, tb, va, vb);
    else win2_dot<WT, (WT >= 20 ? 20 : 0), TWO>(win, ta, tb, va, vb);
}

}  // namespace nedner

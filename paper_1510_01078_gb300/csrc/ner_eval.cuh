// Evaluation of one NER value (Eq. NER_NUFFT, Sec. 3.1) from a line's
// oversampled spectrum, used by the NER kernel in kernels_fwd.cu: the
// frequency nu_l in float-float arithmetic, the w-tap interpolation with the
// mirrored tap polynomials, the phase exp(-i pi nu) and the Jacobian
// coefficient.  It needs only the plan's geometry and tap tables and the FFT
// helpers, so the same header also builds on the host for tests.
#pragma once

#include <cuda_runtime.h>

#include "fft.cuh"
#include "internal.h"

namespace nedner {

struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ FF quick_two_sum(float a, float b) {
    float s = a + b;
    return {s, b - (s - a)};
}

// nu^2 = axy + az * l^2 (float-float), then nu = sqrt(.) (float-float)
__device__ __forceinline__ FF nu_abs(const Geo& G, float2 axy, int l) {
    const float L2 = (float)(l * l);              // exact for |l| < 4096
    const float p_hi = G.az_hi * L2;
    const float p_lo = fmaf(G.az_hi, L2, -p_hi) + G.az_lo * L2;
    FF s = two_sum(axy.x, p_hi);
    s = quick_two_sum(s.hi, s.lo + axy.y + p_lo);
    if (s.hi <= 0.f) return {0.f, 0.f};
    const float r = sqrtf(s.hi);
    const float resid = fmaf(-r, r, s.hi) + s.lo;
    return quick_two_sum(r, resid * (0.5f / r));
}

// sum_k P_k(s) B[((mu0 + k) mod Lt) * 2^lld + col] (padded buffer).  The window
// is even, so tap W-1-k is tap k mirrored, P_{W-1-k}(s) = P_k(-s) (the tap
// polynomials interpolate at nodes symmetric in s); with P_k(s) = E_k(s^2) +
// s O_k(s^2) both taps of a pair come from one Horner evaluation of E_k and O_k.
template <int W, int D>
__device__ __forceinline__ float2 ner_gather(const TapPoly& P, const float2* Bf, int mu0, float s, int Lt, int lld,
                                             int col) {
    constexpr int DE = D & ~1;                    // highest even power
    constexpr int DO = (D & 1) ? D : D - 1;       // highest odd power
    const float u = s * s;
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < W / 2; ++k) {
        float e = P.c[k * (D + 1) + DE];
#pragma unroll
        for (int d = DE - 2; d >= 0; d -= 2) e = fmaf(e, u, P.c[k * (D + 1) + d]);
        float o = P.c[k * (D + 1) + DO];
#pragma unroll
        for (int d = DO - 2; d >= 1; d -= 2) o = fmaf(o, u, P.c[k * (D + 1) + d]);
        const float so = s * o;
        const float pk = e + so, pm = e - so;     // taps k and W-1-k
        const float2 bk = Bf[padx((((mu0 + k) & (Lt - 1)) << lld) + col)];
        const float2 bm = Bf[padx((((mu0 + W - 1 - k) & (Lt - 1)) << lld) + col)];
        acc = __ffma2_rn(make_float2(pk, pk), bk, acc);
        acc = __ffma2_rn(make_float2(pm, pm), bm, acc);
    }
    return acc;
}

// nu_l (signed, float-float) and its coefficient: the Jacobian W (2 at j = l = 0,
// 0 at l = 0 otherwise) times the scale, zero outside the band under band_mask
__device__ __forceinline__ float ner_coef(const Geo& G, float2 axy, bool j0, int l, FF& nu) {
    nu = nu_abs(G, axy, l);
    float Wj;
    if (l == 0) {
        Wj = j0 ? 2.f : 0.f;
        nu = {0.f, 0.f};
    } else {
        Wj = 2.f * G.sqrt_az * (float)abs(l) / nu.hi;
        if (l < 0) nu = {-nu.hi, -nu.lo};
    }
    float cl = G.apply_weights ? Wj * G.scale : G.scale;
    if (G.band_mask) {
        const double nd = (double)nu.hi + (double)nu.lo;
        if (!(nd >= -0.5 * G.Nt - 1e-9 && nd < 0.5 * G.Nt - 1e-9)) cl = 0.f;
    }
    return cl;
}

// The comparison method of Sec. 5.1 (FFT with linear interpolation): the
// line's spectrum B, zero-padded at the end to Lt = SIG Nt (SIG = 1: none), is
// interpolated linearly between the grid points around v = SIG nu; no window,
// no deconvolution, no centring.  Column `col` of the padded buffer Bf with
// 2^lld columns.
template <int SIG>
__device__ __forceinline__ float2 ner_value_linear(const Geo& G, float2 axy, bool j0, int l, const float2* Bf,
                                                   int lld, int col) {
    FF nu;
    const float cl = ner_coef(G, axy, j0, l, nu);
    if (cl == 0.f) return make_float2(0.f, 0.f);
    const int Lt = SIG * G.Nt;
    const float vh = SIG * nu.hi, vl = SIG * nu.lo;
    float fl = floorf(vh);
    float t = (vh - fl) + vl;
    if (t < 0.f) { t += 1.f; fl -= 1.f; }
    if (t >= 1.f) { t -= 1.f; fl += 1.f; }
    const int i0 = (int)fl;
    const float2 b0 = Bf[padx(((i0 & (Lt - 1)) << lld) + col)];
    const float2 b1 = Bf[padx((((i0 + 1) & (Lt - 1)) << lld) + col)];
    return cscale(__ffma2_rn(make_float2(t, t), b1, cscale(b0, 1.f - t)), cl);
}

// The direct sum of the NER (the "direct FT" ground truth of Sec. 5.1):
// sum_{n < Nt} Ghat[n] exp(-2 pi i nu n / Nt) over the raw line (column `col`
// of Bf, sample n in row n).  The phase is re-anchored every 16 terms from
// nu n / Nt reduced modulo 1 in FP64 and advanced by one complex rotation in
// between.
__device__ __forceinline__ float2 ner_value_direct(const Geo& G, float2 axy, bool j0, int l, const float2* Bf,
                                                   int lld, int col) {
    FF nu;
    const float cl = ner_coef(G, axy, j0, l, nu);
    if (cl == 0.f) return make_float2(0.f, 0.f);
    const double a = ((double)nu.hi + (double)nu.lo) / G.Nt;      // turns per sample
    float ss, cs;
    const double fa = a - floor(a);
    sincospif(-2.f * (float)fa, &ss, &cs);
    const float2 step = make_float2(cs, ss);
    float2 acc = make_float2(0.f, 0.f);
    for (int n0 = 0; n0 < G.Nt; n0 += 16) {
        const double f = a * n0 - floor(a * n0);
        sincospif(-2.f * (float)f, &ss, &cs);
        float2 w = make_float2(cs, ss);
        const int n1 = n0 + 16 < G.Nt ? n0 + 16 : G.Nt;
        for (int n = n0; n < n1; ++n) {
            acc = cadd(acc, cmul(w, Bf[padx((n << lld) + col)]));
            w = cmul(w, step);
        }
    }
    return cscale(acc, cl);
}

// coefficient(l) * F(nu_l) for one line whose oversampled spectrum is column
// `col` of the padded buffer Bf with 2^lld columns; j0: the line is j = 0
template <int W, int D>
__device__ __forceinline__ float2 ner_value(const Geo& G, const TapPoly& P, float2 axy, bool j0, int l,
                                            const float2* Bf, int lld, int col) {
    FF nu;
    const float cl = ner_coef(G, axy, j0, l, nu);
    if (cl == 0.f) return make_float2(0.f, 0.f);
    // v = sigma nu (sigma = 2): exact scaling of the pair
    const float vh = 2.f * nu.hi, vl = 2.f * nu.lo;
    float fl = floorf(vh);
    float t = (vh - fl) + vl;
    if (t < 0.f) { t += 1.f; fl -= 1.f; }
    if (t >= 1.f) { t -= 1.f; fl += 1.f; }
    const int ifl = (int)fl;
    const float2 acc = ner_gather<W, D>(P, Bf, ifl - W / 2 + 1, 2.f * t - 1.f, G.Lt, lld, col);
    // exp(-i pi nu) = exp(-i pi v/2) = (-i)^floor(v) exp(-i pi t / 2)
    float sn, cs;
    sincospif(0.5f * t, &sn, &cs);
    float2 ph = make_float2(cs, -sn);
    const int q = ifl & 3;
    if (q == 1) ph = make_float2(ph.y, -ph.x);
    else if (q == 2) ph = make_float2(-ph.x, -ph.y);
    else if (q == 3) ph = make_float2(-ph.y, ph.x);
    return cscale(cmul(ph, acc), cl);
}

}  // namespace nedner

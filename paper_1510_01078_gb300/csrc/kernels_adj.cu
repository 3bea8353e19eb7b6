// Transposed NEDNER kernels: g = R^T p (nedner_adjoint) and the
// sensor-position gradient (nedner_grad_positions).
//
// Each kernel is the exact transpose (for real inner products) of one forward
// stage, run in reverse order:
//   p  [nz][ny][nx]
//     -- img_xr2c_adj    -->  Y [nx/2+1][nz][ny]       r2c along x, times 1 or 2
//     -- img_yfft_adj    -->  V [nx/2+1][ny][nz]       forward FFT along y
//     -- ner_lines_adj   -->  Ghat [nx/2+1][ny+1][Nt]  z-FFT, fold^T, W, NER spreading, IFFT
//     -- ned_yfft_adj    -->  R [nx/2+1][Ly][Nt]       pad, deconvolve, IFFT along y
// then, per pass of Tp time samples,
//     -- ned_xfft_adj    -->  Qb [Tp/32][Ly][Lx][32]   real IFFT along x (the forward grid's layout)
//     -- ned_gather_blocks --> E [entry][Tp]          the window taps of every (sensor, row block)
//                                                      entry dotted with the grid
//     -- adj_sum         -->  g [M][Nt]                sum of a sensor's entries
// For records too short for passes (or a plan without room for the pass
// grid) ned_gather_rows does the real IFFT along x and the gather per grid
// row in one kernel.  The position gradient gathers with the derivative taps,
// dots them with g over time (one value per entry and chunk of samples) and
// sums them per sensor (grad_sum).
#include <cuda_runtime.h>

#include <algorithm>

#include "fft.cuh"
#include "async_copy.cuh"
#include "internal.h"
#include "gather_window.cuh"

namespace nedner {


// ---------------------------------------------------------------------------
// Transpose of img_xc2r: Y[kx] = d_kx sum_qx p[qx] exp(-2 pi i kx qx / nx),
// kx = 0..nx/2, d = 1 at kx = 0, nx/2 and 2 otherwise.  Real-to-complex FFT
// through the half-length complex transform of z[p] = x[2p] + i x[2p+1],
// in place in a padded buffer, H * C <= 16 NT.
// ---------------------------------------------------------------------------
template <int NT>
__global__ void __launch_bounds__(NT, 768 / NT) k_img_xr2c_adj(Geo G, int C, const float* __restrict__ p0,
                                                             const float2* __restrict__ tw, float2* __restrict__ Y) {
    extern __shared__ float4 smem4[];
    const int H = G.nx / 2;
    float2* A = reinterpret_cast<float2*>(smem4);   // [H][C], padded
    const int qz = blockIdx.x;
    const int y0 = blockIdx.y * C;
    const int lc = ilog2(C), lh = ilog2(H);
    const float2* src = reinterpret_cast<const float2*>(p0 + ((size_t)qz * G.ny + y0) * G.nx);
#pragma unroll 4
    for (int it = threadIdx.x; it < H * C; it += NT) {
        const int c = it >> lh;
        const int pp = it & (H - 1);
        A[padx(pp * C + c)] = src[it];
    }
    block_fft_ip<16>(A, H, C, -1, tw);
    const size_t kstride = (size_t)G.nz * G.ny;
    float2* dst = Y + (size_t)qz * G.ny + y0;
#pragma unroll 4
    for (int it = threadIdx.x; it < (H + 1) * C; it += NT) {
        const int k = it >> lc;
        const int c = it & (C - 1);
        float2 X = r2c_unpack(A[padx(((k & (H - 1)) << lc) + c)], A[padx((((H - k) & (H - 1)) << lc) + c)], k,
                              G.nx, tw);
        if (k != 0 && k != H) X = cscale(X, 2.f);
        dst[k * kstride + c] = X;
    }
}

// ---------------------------------------------------------------------------
// Transpose of img_yifft: V[kx][ky][qz] = sum_qy exp(-2 pi i ky qy / ny) Y[kx][qz][qy],
// in place in a padded buffer, ny * C <= 16 NT.
// ---------------------------------------------------------------------------
template <int NT>
__global__ void __launch_bounds__(NT, 768 / NT) k_img_yfft_adj(Geo G, int C, const float2* __restrict__ Y,
                                                             const float2* __restrict__ tw, float2* __restrict__ V) {
    extern __shared__ float4 smem4[];
    float2* A = reinterpret_cast<float2*>(smem4);   // [ny][C], padded
    const int kx = blockIdx.x;
    const int z0 = blockIdx.y * C;
    const int lc = ilog2(C), lny = ilog2(G.ny);
    const float2* src = Y + ((size_t)kx * G.nz + z0) * G.ny;
#pragma unroll 4
    for (int it = threadIdx.x; it < G.ny * C; it += NT) {
        const int c = it >> lny;
        const int qy = it & (G.ny - 1);
        A[padx(qy * C + c)] = src[it];
    }
    block_fft_ip<16>(A, G.ny, C, -1, tw);
    float2* dst = V + (size_t)kx * G.ny * G.nz + z0;
#pragma unroll 8
    for (int it = threadIdx.x; it < G.ny * C; it += NT)
        dst[(size_t)(it >> lc) * G.nz + (it & (C - 1))] = A[padx(it)];
}

// ---------------------------------------------------------------------------
// Transpose of ner_lines, one CTA per line group (kx, ky).
//   Ubar = FFT_nz(sign V[line])                       (transpose of the z-IFFT)
//   Tbar_a[l] = ca Ubar[l]          for l = -nz/2..nz/2-1
//   Tbar_b[e] = cb Ubar[slot(e)]    e = l* of some slot l (none for e = -nz/2)
//   Tbar      *= coefficient(e) (Jacobian, scale, band mask)
//   Bbar[mu] = sum_e exp(+i pi nu_e) phi(sigma nu_e - mu) Tbar[e]   (spreading)
//   Ghat-bar[n] = IFFT_Lt(Bbar)[(n - Nt/2) mod Lt] / phihat((n - Nt/2)/Lt)
// The spreading is done as a gather per grid point (ner_adj_line): no atomics
// unless a band is longer than the grid, and a CTA owns its lines, so nothing
// is shared between CTAs.
// ---------------------------------------------------------------------------
struct FF2 {
    float hi, lo;
};

__device__ __forceinline__ FF2 two_sum2(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ FF2 quick_two_sum2(float a, float b) {
    float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ FF2 nu_abs2(const Geo& G, float2 axy, int l) {
    const float L2 = (float)(l * l);
    const float p_hi = G.az_hi * L2;
    const float p_lo = fmaf(G.az_hi, L2, -p_hi) + G.az_lo * L2;
    FF2 s = two_sum2(axy.x, p_hi);
    s = quick_two_sum2(s.hi, s.lo + axy.y + p_lo);
    if (s.hi <= 0.f) return {0.f, 0.f};
    const float r = sqrtf(s.hi);
    const float resid = fmaf(-r, r, s.hi) + s.lo;
    return quick_two_sum2(r, resid * (0.5f / r));
}

// The transposed NER value of one depth frequency l of a line: its weight
// (Jacobian, scale, band mask) times exp(+i pi nu) times tb, and where its w
// taps land on the line's 2Nt grid: the first grid point mu0 and the tap
// argument s (tap k at s, tap w-1-k at -s, as in ner_gather).  mu0 is
// computed whether or not the value is zero, so that it is non-decreasing in
// l (nu is increasing in l).
struct NerAdjItem {
    int mu0;
    float s;
    float2 v;
};

__device__ __forceinline__ NerAdjItem ner_adj_item(const Geo& G, float2 axy, bool j0, int l, float2 tb) {
    FF2 nu = nu_abs2(G, axy, l);
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
    const float vh = 2.f * nu.hi, vl = 2.f * nu.lo;
    float fl = floorf(vh);
    float t = (vh - fl) + vl;
    if (t < 0.f) { t += 1.f; fl -= 1.f; }
    if (t >= 1.f) { t -= 1.f; fl += 1.f; }
    const int ifl = (int)fl;
    NerAdjItem it;
    it.mu0 = ifl - G.w / 2 + 1;
    it.s = 2.f * t - 1.f;
    it.v = make_float2(0.f, 0.f);
    tb = cscale(tb, cl);
    if (tb.x != 0.f || tb.y != 0.f) {
        // exp(+i pi nu) = i^floor(v) exp(+i pi t / 2)
        float sn, cs;
        sincospif(0.5f * t, &sn, &cs);
        float2 ph = make_float2(cs, sn);
        const int q = ifl & 3;
        if (q == 1) ph = make_float2(-ph.y, ph.x);
        else if (q == 2) ph = make_float2(-ph.x, -ph.y);
        else if (q == 3) ph = make_float2(ph.y, -ph.x);
        it.v = cmul(ph, tb);
    }
    return it;
}

// the W tap weights P_k(s), k = 0..W-1 (tap W-1-k is tap k at -s)
template <int W, int D>
__device__ __forceinline__ void ner_taps(const TapPoly& P, float s, float* w) {
    constexpr int DE = D & ~1;
    constexpr int DO = (D & 1) ? D : D - 1;
    const float u = s * s;
#pragma unroll
    for (int k = 0; k < W / 2; ++k) {
        float e = P.c[k * (D + 1) + DE];
#pragma unroll
        for (int d = DE - 2; d >= 0; d -= 2) e = fmaf(e, u, P.c[k * (D + 1) + d]);
        float o = P.c[k * (D + 1) + DO];
#pragma unroll
        for (int d = DO - 2; d >= 1; d -= 2) o = fmaf(o, u, P.c[k * (D + 1) + d]);
        const float so = s * o;
        w[k] = e + so;
        w[W - 1 - k] = e - so;
    }
}

// One line of the transposed NER into column col of the padded line buffer
// LA (2^lld columns, zero on entry): Bbar[mu] = sum_l P_{mu - mu0_l}(s_l) v_l
// over the depth frequencies whose taps reach mu.  The nz + 1 depth
// frequencies are taken in chunks of at most icap: phase 1 stores each
// one's mu0, v and W tap weights (it_mu0, it_v, it_w); phase 2 gives each grid
// point of the chunk's band [mu0_first, mu0_last + W) to one thread, which
// finds the l reaching it by binary search in the non-decreasing mu0 (two
// items of slack either side for rounding in nu) and adds their contributions
// in order of l to the point: no atomics, and the same result on every run.
// A band longer than the grid (nu far beyond the Nyquist band, where grid
// points would be shared modulo 2Nt) is spread with shared-memory atomics
// instead.  Returns true if every band lies within [-Lt/4, Lt/4), i.e. the
// inverse FFT's input is zero on [Lt/4, 3Lt/4).
template <int W, int D, int NT, typename TB>
__device__ bool ner_adj_line(const Geo& G, const TapPoly& P, float2 axy, bool j0, TB tb_of, float2* LA, int lld,
                             int col, int icap, int* it_mu0, float2* it_v, float* it_w) {
    const int nz1 = G.nz + 1, half_nz = G.nz / 2;
    bool zp = true;
    for (int e0 = 0; e0 < nz1; e0 += icap) {
        const int ni = min(icap, nz1 - e0);
        for (int i = threadIdx.x; i < ni; i += NT) {
            const NerAdjItem it = ner_adj_item(G, axy, j0, e0 + i - half_nz, tb_of(e0 + i));
            float w[W];
            ner_taps<W, D>(P, it.s, w);
            it_mu0[i] = it.mu0;
            it_v[i] = it.v;
#pragma unroll
            for (int k = 0; k < W; ++k) it_w[i * (W + 1) + k] = w[k];      // odd stride: no bank conflicts
        }
        __syncthreads();
        const int lo = it_mu0[0] - 2, hi = it_mu0[ni - 1] + W + 2;
        if (hi - lo <= G.Lt) {
            // a warp takes 32 consecutive grid points: lanes 0 and 1 find the
            // items reaching the first and the last (binary search, two items of
            // slack), and every lane walks that range with broadcast loads
            const int lane = threadIdx.x & 31;
            for (int mw = lo + (int)(threadIdx.x & ~31); mw < hi; mw += NT) {
                const int mu = mw + lane;
                int r = 0;
                if (lane < 2) {
                    const int key = lane == 0 ? mw - W + 1 : mw + 32;   // first mu0 >= key
                    int a = 0, b = ni;
                    while (a < b) {
                        const int m = (a + b) >> 1;
                        if (it_mu0[m] < key) a = m + 1;
                        else b = m;
                    }
                    r = lane == 0 ? max(0, a - 2) : min(ni, a + 2);
                }
                const int ia = __shfl_sync(0xffffffffu, r, 0), ib = __shfl_sync(0xffffffffu, r, 1);
                float2 acc = make_float2(0.f, 0.f);
                for (int i = ia; i < ib; ++i) {
                    const int k = mu - it_mu0[i];
                    if (k >= 0 && k < W) {
                        const float wk = it_w[i * (W + 1) + k];
                        const float2 v = it_v[i];
                        acc.x = fmaf(wk, v.x, acc.x);
                        acc.y = fmaf(wk, v.y, acc.y);
                    }
                }
                if (mu < hi) {
                    float2* d = &LA[padx((((mu + G.Lt) & (G.Lt - 1)) << lld) + col)];
                    *d = e0 == 0 ? acc : cadd(*d, acc);
                }
            }
        } else {
            for (int i = threadIdx.x; i < ni; i += NT) {
                const float2 v = it_v[i];
                if (v.x == 0.f && v.y == 0.f) continue;
                for (int k = 0; k < W; ++k) {
                    float2* d = &LA[padx((((it_mu0[i] + k) & (G.Lt - 1)) << lld) + col)];
                    atomicAdd(&d->x, it_w[i * (W + 1) + k] * v.x);
                    atomicAdd(&d->y, it_w[i * (W + 1) + k] * v.y);
                }
            }
        }
        __syncthreads();
        zp = zp && lo >= -(G.Lt / 4) && hi <= G.Lt / 4;
    }
    return zp;
}

// Transpose of ner_lines for the LPC line groups (kx, k0..k0+LPC-1) of the
// forward CTA:
//   Ubar = FFT_nz(sign V[group])                      (transpose of the z-IFFT)
//   line ky of group c:  Tbar[e] = ca Ubar_c[l] (e < nz) + cb Ubar_c[slot(e)] (e > 0)
//   the group ky = -ny/2 feeds line -ny/2 through ca only and line +ny/2
//   through cb (slot(e) = l for e < nz, -nz/2 for e = nz), as the fold reads them;
// each Tbar[e] is weighted (Jacobian, scale, band mask), multiplied by
// exp(+i pi nu) and spread with the w taps onto the line's 2Nt grid
// (ner_adj_line), the grids are inverse-transformed together (the first pass
// skipping the zero half where every band allows), and the centred Nt
// samples, divided by phihat in time and by phihat(jy/Ly) (the transposed
// y-FFT's deconvolution, applied here), are the lines of Ghat.
template <int W, int D, int NT>
__global__ void __launch_bounds__(NT, NT <= 256 ? 4 : 1) k_ner_lines_adj(Geo G, const __grid_constant__ TapPoly P,
                                                                       int LPC, int icap,
                                                                       const float2* __restrict__ V,
                                                                       const float2* __restrict__ axy_tab,
                                                                       const float* __restrict__ deconv_t,
                                                                       const float* __restrict__ deconv_y,
                                                                       const float2* __restrict__ tw,
                                                                       float2* __restrict__ Ghat) {
    constexpr int PER = 16;
    extern __shared__ float4 smem4[];
    const int nz1 = G.nz + 1;
    float2* LA = reinterpret_cast<float2*>(smem4);                 // [Lt][LPC], padded
    float2* UA = LA + padded_len(G.Lt * LPC);                      // [nz][LPC], padded
    float2* it_v = UA + padded_len(G.nz * LPC);                    // [icap] (items of one line)
    int* it_mu0 = reinterpret_cast<int*>(it_v + icap);             // [icap]
    float* it_w = reinterpret_cast<float*>(it_mu0 + icap);         // [icap][W + 1]

    const int llpc = ilog2(LPC), lnz = ilog2(G.nz);
    const int cpk = G.ny >> llpc;
    const int kx = blockIdx.x / cpk;
    const int k0 = (blockIdx.x - kx * cpk) * LPC - G.ny / 2;
    const bool nyq_x = (kx == G.nx / 2);
    const float ca = nyq_x ? 0.f : 0.5f;
    const float cb = nyq_x ? 1.f : 0.5f;
    const int half_nz = G.nz / 2;
    const size_t line0 = (size_t)kx * G.nyp + (k0 + G.ny / 2);

    // Ubar of the LPC groups
    for (int i = threadIdx.x; i < (G.nz << llpc); i += NT) {
        const int c = i >> lnz, q = i & (G.nz - 1);
        const int ky = k0 + c;
        const float sg = ((kx + ky) & 1) ? -1.f : 1.f;
        UA[padx((q << llpc) + c)] = cscale(V[((size_t)kx * G.ny + (ky & (G.ny - 1))) * G.nz + q], sg);
    }
    block_fft_ip<PER>(UA, G.nz, LPC, -1, tw);
    auto slot_of = [&](int e) { return (e == G.nz) ? (-half_nz & (G.nz - 1)) : ((e - half_nz) & (G.nz - 1)); };

    if (k0 == -G.ny / 2) {
        // the line (kx, +ny/2), fed by group 0 through cb, in column 0
        for (int p = threadIdx.x; p < padded_len(G.Lt); p += NT) LA[p] = make_float2(0.f, 0.f);
        __syncthreads();
        const size_t lx = (size_t)kx * G.nyp + G.ny;
        auto tb_of = [&](int e) {
            return e > 0 ? cscale(UA[padx(slot_of(e) << llpc)], cb) : make_float2(0.f, 0.f);
        };
        const bool zp = ner_adj_line<W, D, NT>(G, P, __ldg(&axy_tab[lx]), false, tb_of, LA, 0, 0, icap, it_mu0,
                                              it_v, it_w);
        if (zp) block_fft_ip<PER, true>(LA, G.Lt, 1, +1, tw);
        else block_fft_ip<PER>(LA, G.Lt, 1, +1, tw);
        float2* dst = Ghat + lx * G.Nt;
        const float dy = __ldg(&deconv_y[G.ny]);
        for (int n = threadIdx.x; n < G.Nt; n += NT)
            dst[n] = cscale(LA[padx((n - G.Nt / 2) & (G.Lt - 1))], __ldg(&deconv_t[n]) * dy);
        __syncthreads();
    }
    // the LPC lines (kx, k0 + c), one after another into their columns
    for (int p = threadIdx.x; p < padded_len(G.Lt * LPC); p += NT) LA[p] = make_float2(0.f, 0.f);
    __syncthreads();
    bool zp = true;
    for (int c = 0; c < LPC; ++c) {
        const int ky = k0 + c;
        const bool is_b = (ky != -G.ny / 2);                       // group -ny/2 feeds line +ny/2 instead
        auto tb_of = [&](int e) {
            const int l = e - half_nz;
            float2 tb = make_float2(0.f, 0.f);
            if (e < G.nz) tb = cadd(tb, cscale(UA[padx(((l & (G.nz - 1)) << llpc) + c)], ca));
            if (is_b && e > 0) tb = cadd(tb, cscale(UA[padx((slot_of(e) << llpc) + c)], cb));
            return tb;
        };
        zp &= ner_adj_line<W, D, NT>(G, P, __ldg(&axy_tab[line0 + c]), kx == 0 && ky == 0, tb_of, LA, llpc, c,
                                     icap, it_mu0, it_v, it_w);
    }
    if (zp) block_fft_ip<PER, true>(LA, G.Lt, LPC, +1, tw);
    else block_fft_ip<PER>(LA, G.Lt, LPC, +1, tw);
    for (int i = threadIdx.x; i < (G.Nt << llpc); i += NT) {
        const int c = i >> ilog2(G.Nt), n = i & (G.Nt - 1);
        Ghat[(line0 + c) * G.Nt + n] = cscale(LA[padx((((n - G.Nt / 2) & (G.Lt - 1)) << llpc) + c)],
                                              __ldg(&deconv_t[n]) * __ldg(&deconv_y[k0 + c + G.ny / 2]));
    }
}

// ---------------------------------------------------------------------------
// Transpose of ned_yfft: R[jx][gy][n] = sum_jy exp(+2 pi i jy gy / Ly) Ghat[jx][jy][n] / phihat(jy/Ly)
// (the division by phihat(jy/Ly) is done by k_ner_lines_adj when it writes Ghat).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 4) k_ned_yfft_adj(Geo G, int C, const float2* __restrict__ Ghat,
                                                         const float* __restrict__ deconv_y,
                                                         const float2* __restrict__ tw, float2* __restrict__ R) {
    extern __shared__ float4 smem4[];
    float2* A = reinterpret_cast<float2*>(smem4);   // [Ly][C], padded
    const int jx = blockIdx.y;                      // time chunks on blockIdx.x: neighbouring CTAs
    const int n0 = blockIdx.x * C;                  // read neighbouring pieces of the same rows
    const int lc = ilog2(C);
    // jy = b - ny/2 sits at q = (jy mod Ly); the other Ly - (ny + 1) points are
    // zero.  Ghat arrives already divided by phihat(jy/Ly) (k_ner_lines_adj).
    for (int it = threadIdx.x; it < G.Ly * C; it += 256) {
        const int q = it >> lc;
        const int c = it & (C - 1);
        const int b = (q <= G.ny / 2) ? q + G.ny / 2 : ((q >= G.Ly - G.ny / 2) ? q - G.Ly + G.ny / 2 : -1);
        if (b >= 0) cp_async(&A[padx(it)], &Ghat[((size_t)jx * G.nyp + b) * G.Nt + n0 + c], 8);
        else A[padx(it)] = make_float2(0.f, 0.f);
    }
    cp_async_commit();
    cp_async_wait_all();
    block_fft_ip<16>(A, G.Ly, C, +1, tw);
#pragma unroll 8
    for (int it = threadIdx.x; it < G.Ly * C; it += 256) {
        const int gy = it >> lc;
        const int c = it & (C - 1);
        R[((size_t)jx * G.Ly + gy) * G.Nt + n0 + c] = A[padx(it)];
    }
}

// ---------------------------------------------------------------------------
// Transpose of the x part of the spread stage for one grid row: the real row
//   r[gx][t] = Re sum_{jx=0}^{nx/2} R[jx][t] exp(+2 pi i jx gx / Lx) / phihat(jx/Lx)
// for C time samples, as the inverse FFT of the Hermitian part of the
// zero-extended spectrum, two real samples packed per complex column.  Z is
// the padded [Lx][C/2] complex row (see block_fft_ip); on return the real
// value (gx, t) is at ((float*)Z)[2 padx(gx C/2 + t/2) + t%2].
// ---------------------------------------------------------------------------
constexpr int ADJ_ECH = 128;                     // entries staged at a time by the transposed kernels

template <int PER>
__device__ __forceinline__ void row_rebuild(const Geo& G, int C, const float2* __restrict__ R, int gy, int n0,
                                            const float* __restrict__ deconv_x, const float2* __restrict__ tw,
                                            float2* Z) {
    const int Lx = G.Lx;
    const int nb = C / 2;
    const int lnb = ilog2(nb);
    const int half = G.nx / 2;
    for (int it = threadIdx.x; it < (Lx << lnb); it += blockDim.x) {
        const int k = it >> lnb;
        const int b = it & (nb - 1);
        float2 z = make_float2(0.f, 0.f);
        const int jx = (k <= half) ? k : ((k >= Lx - half) ? Lx - k : -1);
        if (jx >= 0) {
            const float d = __ldg(&deconv_x[jx]);
            const float2* src = R + ((size_t)jx * G.Ly + gy) * G.Nt + n0 + 2 * b;
            const float2 y1 = cscale(src[0], d);
            const float2 y2 = cscale(src[1], d);
            if (k == 0) z = make_float2(y1.x, y2.x);                                   // Re Y1[0] + i Re Y2[0]
            else if (k <= half) z = cscale(cadd(y1, mul_i(y2, +1)), 0.5f);              // H[k] = Y[k] / 2
            else z = cscale(cadd(cconj(y1), mul_i(cconj(y2), +1)), 0.5f);               // H[Lx-k] = conj Y[k] / 2
        }
        Z[padx(it)] = z;
    }
    block_fft_ip<PER>(Z, Lx, nb, +1, tw);
}

// ---------------------------------------------------------------------------
// Transposed interpolation (the transpose of the spread stage's x and y
// parts) and the position gradient, one CTA per (grid row gy, C time
// samples) as in the forward spread.  The CTA rebuilds the real row r
// (row_rebuild), stages the row's entries (sorted by first column, without
// the second copies of wrapped entries) in chunks, and each lane group
// sweeps a contiguous run of a chunk with a register window of the row (the
// forward sweep, transposed): every entry gets
//   v[t] = sum_k tap[k] r[(bx4 + k) mod Lx][t]
// with the forward spread's taps (x tap times y tap times w_m, from a
// 4-aligned column).
//   adjoint:  E[e][t - nb] = v[t], e the entry's index in the row CSR, for the
//             pass of time samples [nb, nb + Tp); adj_sum adds each sensor's
//             w entries (no atomics, fixed order).
//   gradient: the two derivative tap sets give v_x, v_y; the entry's
//             sum_t g[m][t] (v_x[t], v_y[t]) over the C samples goes to
//             Qe[e][time chunk]; grad_sum adds entries and chunks per sensor.
// ---------------------------------------------------------------------------
template <int WT, int PER, bool GRAD>
__global__ void __launch_bounds__(256, 2) k_ned_gather_rows(Geo G, int C, int nb, int Tp,
                                                            const float2* __restrict__ R,
                                                            const float* __restrict__ g,
                                                            const int* __restrict__ xrow_ptr,
                                                            const int* __restrict__ xrow_first,
                                                            const int* __restrict__ xent_m,
                                                            const int* __restrict__ xent_bx,
                                                            const int* __restrict__ xent_rc,
                                                            const float* __restrict__ taps_a,
                                                            const float* __restrict__ taps_b,
                                                            const float* __restrict__ deconv_x,
                                                            const float2* __restrict__ tw, float* __restrict__ E,
                                                            float2* __restrict__ Qe) {
    extern __shared__ float4 smem4[];
    float2* Z = reinterpret_cast<float2*>(smem4);                    // padded [Lx][C/2]
    const float* Zf = reinterpret_cast<const float*>(Z);
    float4* s_ta = reinterpret_cast<float4*>(Z + ((padded_len(G.Lx * (C / 2)) + 1) & ~1));   // [ADJ_ECH][WT/4]
    float4* s_tb = s_ta + ADJ_ECH * (WT / 4);                         // [ADJ_ECH][WT/4] (GRAD)
    int* s_bx = reinterpret_cast<int*>(s_tb + (GRAD ? ADJ_ECH * (WT / 4) : 0));      // [ADJ_ECH]
    int* s_rc = s_bx + ADJ_ECH;                                                        // [ADJ_ECH]
    int* s_m = s_rc + ADJ_ECH;                                                         // [ADJ_ECH] (GRAD)
    const int gy = blockIdx.x;
    const int n0 = nb + blockIdx.y * C;
    const int lc = ilog2(C), lnb = lc - 1;
    const int groups = blockDim.x >> lc;
    const int q = threadIdx.x >> lc;
    const int ln = threadIdx.x & (C - 1);
    const int Lx = G.Lx;
    const unsigned gmask = (C >= 32) ? 0xffffffffu : (((1u << C) - 1u) << ((threadIdx.x & 31) - ln));
    const int nch = G.Nt / C;

    row_rebuild<PER>(G, C, R, gy, n0, deconv_x, tw, Z);
    for (int c0 = xrow_first[gy], e_end = xrow_ptr[gy + 1]; c0 < e_end; c0 += ADJ_ECH) {
        const int ne = min(ADJ_ECH, e_end - c0);
        for (int i = threadIdx.x; i < ne; i += blockDim.x) {
            s_bx[i] = __ldg(&xent_bx[c0 + i]);
            s_rc[i] = __ldg(&xent_rc[c0 + i]);
            if (GRAD) s_m[i] = __ldg(&xent_m[c0 + i]);
        }
        const float4* sa = reinterpret_cast<const float4*>(taps_a + (size_t)c0 * WT);
        const float4* sb = reinterpret_cast<const float4*>(taps_b + (size_t)c0 * WT);
        for (int i = threadIdx.x; i < ne * (WT / 4); i += blockDim.x) {
            s_ta[i] = __ldg(&sa[i]);
            if (GRAD) s_tb[i] = __ldg(&sb[i]);
        }
        __syncthreads();
        const int j0 = (q * ne) / groups, j1 = ((q + 1) * ne) / groups;
        if (j0 < j1) {                                                 // uniform across the lane group
            float win[2 * WT];
            int base = s_bx[j0];
            win_load<WT>(win, Zf, lnb, ln, Lx, base, 0);
            win_load<WT>(win, Zf, lnb, ln, Lx, base, WT);
            float gnext = GRAD ? __ldg(&g[(size_t)s_m[j0] * G.Nt + n0 + ln]) : 0.f;
            for (int j = j0; j < j1; ++j) {
                const int bx4 = s_bx[j];
                const float gv = gnext;                                // the entry's sample of g
                if (GRAD && j + 1 < j1) gnext = __ldg(&g[(size_t)s_m[j + 1] * G.Nt + n0 + ln]);
                win_advance<WT>(win, Zf, lnb, ln, Lx, base, bx4);
                const float2 v = win_entry<WT, GRAD>(win, (bx4 - base) >> 2, s_ta + j * (WT / 4), s_tb + j * (WT / 4));
                if (!GRAD) {
                    E[(size_t)s_rc[j] * Tp + (n0 - nb) + ln] = v.x;
                } else {
                    float sx = gv * v.x, sy = gv * v.y;
                    for (int o = C / 2; o > 0; o >>= 1) {
                        sx += __shfl_xor_sync(gmask, sx, o);
                        sy += __shfl_xor_sync(gmask, sy, o);
                    }
                    if (ln == 0) Qe[(size_t)s_rc[j] * nch + n0 / C] = make_float2(sx, sy);
                }
            }
        }
        __syncthreads();
    }
}

// k_ned_gather_rows with two time samples per lane: C = 64, one lane group
// per warp, the row FFT with 32 values per thread: NT = 256 for 2 nx <= 256,
// NT = 512 (one CTA per SM) for 2 nx = 512.
template <int WT, bool GRAD, int NT>
__global__ void __launch_bounds__(NT, NT <= 256 ? 2 : 1) k_ned_gather_rows2(Geo G, int nb, int Tp, const float2* __restrict__ R,
                                                             const float* __restrict__ g,
                                                             const int* __restrict__ xrow_ptr,
                                                             const int* __restrict__ xrow_first,
                                                             const int* __restrict__ xent_m,
                                                             const int* __restrict__ xent_bx,
                                                             const int* __restrict__ xent_rc,
                                                             const float* __restrict__ taps_a,
                                                             const float* __restrict__ taps_b,
                                                             const float* __restrict__ deconv_x,
                                                             const float2* __restrict__ tw, float* __restrict__ E,
                                                             float2* __restrict__ Qe) {
    constexpr int C = 64;
    extern __shared__ float4 smem4[];
    float2* Z = reinterpret_cast<float2*>(smem4);                    // padded [Lx][32]
    float4* s_ta = reinterpret_cast<float4*>(Z + ((padded_len(G.Lx * (C / 2)) + 1) & ~1));   // [ADJ_ECH][WT/4]
    float4* s_tb = s_ta + ADJ_ECH * (WT / 4);                         // [ADJ_ECH][WT/4] (GRAD)
    int* s_bx = reinterpret_cast<int*>(s_tb + (GRAD ? ADJ_ECH * (WT / 4) : 0));      // [ADJ_ECH]
    int* s_rc = s_bx + ADJ_ECH;                                                        // [ADJ_ECH]
    int* s_m = s_rc + ADJ_ECH;                                                         // [ADJ_ECH] (GRAD)
    const int gy = blockIdx.x;
    const int n0 = nb + blockIdx.y * C;
    const int groups = blockDim.x >> 5;
    const int q = threadIdx.x >> 5;
    const int ln = threadIdx.x & 31;
    const int Lx = G.Lx;
    const int nch = G.Nt / C;

    row_rebuild<32>(G, C, R, gy, n0, deconv_x, tw, Z);
    for (int c0 = xrow_first[gy], e_end = xrow_ptr[gy + 1]; c0 < e_end; c0 += ADJ_ECH) {
        const int ne = min(ADJ_ECH, e_end - c0);
        for (int i = threadIdx.x; i < ne; i += blockDim.x) {
            s_bx[i] = __ldg(&xent_bx[c0 + i]);
            s_rc[i] = __ldg(&xent_rc[c0 + i]);
            if (GRAD) s_m[i] = __ldg(&xent_m[c0 + i]);
        }
        const float4* sa = reinterpret_cast<const float4*>(taps_a + (size_t)c0 * WT);
        const float4* sb = reinterpret_cast<const float4*>(taps_b + (size_t)c0 * WT);
        for (int i = threadIdx.x; i < ne * (WT / 4); i += blockDim.x) {
            s_ta[i] = __ldg(&sa[i]);
            if (GRAD) s_tb[i] = __ldg(&sb[i]);
        }
        __syncthreads();
        const int j0 = (q * ne) / groups, j1 = ((q + 1) * ne) / groups;
        if (j0 < j1) {
            float2 win[2 * WT];
            int base = s_bx[j0];
            win2_load<WT>(win, Z, ln, Lx, base, 0);
            win2_load<WT>(win, Z, ln, Lx, base, WT);
            float2 gnext = GRAD ? __ldg(reinterpret_cast<const float2*>(g + (size_t)s_m[j0] * G.Nt + n0) + ln)
                                : make_float2(0.f, 0.f);
            for (int j = j0; j < j1; ++j) {
                const int bx4 = s_bx[j];
                const float2 gv = gnext;                               // the entry's samples of g
                if (GRAD && j + 1 < j1)
                    gnext = __ldg(reinterpret_cast<const float2*>(g + (size_t)s_m[j + 1] * G.Nt + n0) + ln);
                win2_advance<WT>(win, Z, ln, Lx, base, bx4);
                float2 va, vb;
                win2_entry<WT, GRAD>(win, (bx4 - base) >> 2, s_ta + j * (WT / 4), s_tb + j * (WT / 4), va, vb);
                if (!GRAD) {
                    reinterpret_cast<float2*>(E + (size_t)s_rc[j] * Tp + (n0 - nb))[ln] = va;
                } else {
                    float sx = fmaf(gv.x, va.x, gv.y * va.y), sy = fmaf(gv.x, vb.x, gv.y * vb.y);
                    for (int o = 16; o > 0; o >>= 1) {
                        sx += __shfl_xor_sync(0xffffffffu, sx, o);
                        sy += __shfl_xor_sync(0xffffffffu, sy, o);
                    }
                    if (ln == 0) Qe[(size_t)s_rc[j] * nch + n0 / C] = make_float2(sx, sy);
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// The transposed interpolation as two kernels per pass of Tp time samples
// [nb, nb + Tp) (the transpose of the block spread and the x-FFT):
//
// k_ned_xfft_adj: one CTA per (grid row gy, 2 nbx samples of the pass)
// rebuilds the real row of the pass's grid Qb [Tp/32][Ly][Lx][32] (the layout
// of the forward Q): the inverse x-FFT of the Hermitian half spectrum of
// R-bar divided by phihat, two real samples packed per complex column as in
// row_rebuild.  The packed spectrum H is nonzero only at k <= Lx/4 and
// k >= 3 Lx/4, so the FFT's first pass skips the zero quarter points
// (block_fft_ip's ZP), which also hold the raw R-bar values while they are
// staged (loaded by asynchronous copies, all in flight at once).  The one
// nonzero point there, H[Lx/4] (jx = nx/2), is added after the FFT as
// H[Lx/4] i^gx.  With nbx = 16 each CTA writes one contiguous block.
// ---------------------------------------------------------------------------
// the padded row (the forward x-FFT's buffer) and H[Lx/4] of its nbx <= 16 columns
static size_t xfft_adj_smem(const Chunks& c) { return c.smem_x + 16 * sizeof(float2); }

template <int PER>
__global__ void __launch_bounds__(256, PER <= 16 ? 4 : 2) k_ned_xfft_adj(Geo G, int nb, int nbx,
                                                                        const float2* __restrict__ R,
                                                                        const float* __restrict__ deconv_x,
                                                                        const float2* __restrict__ tw,
                                                                        float* __restrict__ Qb) {
    extern __shared__ float4 smem4[];
    float2* Z = reinterpret_cast<float2*>(smem4);                    // padded [Lx][nbx]
    float2* nyq = Z + ((padded_len(G.Lx * nbx) + 1) & ~1);           // [nbx]: H[Lx/4]
    const int gy = blockIdx.x;
    const int nc = blockIdx.y * 2 * nbx;                             // first sample of the CTA in the pass
    const int lnb = ilog2(nbx);
    const int half = G.nx / 2;                                       // Lx / 4
    const int ys = (half + 1) << lnb;                                // Y2 of jx staged at row half + 1 + jx
    const int nj = (half + 1) << lnb;
    // raw R-bar: Y1 = R[jx][n + 2b] at row jx, Y2 = R[jx][n + 2b + 1] at row half + 1 + jx
    const float2* src = R + (size_t)gy * G.Nt + nb + nc;
    for (int it = threadIdx.x; it < nj; it += blockDim.x) {
        const float2* q = src + (size_t)(it >> lnb) * G.Ly * G.Nt + 2 * (it & (nbx - 1));
        cp_async(&Z[padx(it)], q, 8);
        cp_async(&Z[padx(ys + it)], q + 1, 8);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    // H[0] = Re Y1[0] + i Re Y2[0]; H[jx] = (Y1 + i Y2) / 2 and
    // H[Lx - jx] = (conj Y1 + i conj Y2) / 2 for 0 < jx <= nx/2 (rows written
    // here never overlap the staged Y2 rows of other threads)
    for (int it = threadIdx.x; it < nj; it += blockDim.x) {
        const int jx = it >> lnb, b = it & (nbx - 1);
        const float d = __ldg(&deconv_x[jx]);
        const float2 y1 = cscale(Z[padx(it)], d), y2 = cscale(Z[padx(ys + it)], d);
        if (jx == 0) {
            Z[padx(it)] = make_float2(y1.x, y2.x);
        } else {
            const float2 hk = cscale(cadd(y1, mul_i(y2, +1)), 0.5f);
            if (jx < half) Z[padx(it)] = hk;
            else nyq[b] = hk;
            Z[padx(((G.Lx - jx) << lnb) + b)] = cscale(cadd(cconj(y1), mul_i(cconj(y2), +1)), 0.5f);
        }
    }
    // log2 Lx = 1 mod 4: the last radix-2 pass is done in the output loop
    const bool fold = (ilog2(G.Lx) & 3) == 1;
    block_fft_ip<PER, true>(Z, G.Lx, nbx, +1, tw, fold);
    // samples nc .. nc + 2 nbx: group nc / 32 of 32, offset nc % 32
    float2* dst = reinterpret_cast<float2*>(Qb + ((size_t)(nc >> 5) * G.Ly + gy) * G.Lx * 32 + (nc & 31)) +
                  (threadIdx.x & (nbx - 1));
    // every thread keeps one column b; its points gx step by blockDim / nbx =
    // Lx / PER >= 4, a multiple of 4, so i^gx (the H[Lx/4] term) is fixed
    const int b = threadIdx.x & (nbx - 1);
    const int k0 = threadIdx.x >> lnb, ks = blockDim.x >> lnb;
    const float2 h = nyq[b];
    const float2 hi = (k0 & 1) ? make_float2(-h.y, h.x) : h;
    const float2 add = (k0 & 2) ? make_float2(-hi.x, -hi.y) : hi;
    if (fold) {
        // x[k] = s[k] + w^k s[k + Lx/2], x[k + Lx/2] = s[k] - w^k s[k + Lx/2],
        // w = exp(+2 pi i / Lx); i^(k + Lx/2) = i^k
        const int H = G.Lx >> 1;
        for (int k = k0; k < H; k += ks) {
            const float2 s0 = Z[padx((k << lnb) + b)], s1 = cmul(cconj(__ldg(&tw[G.Lx + k])), Z[padx(((k + H) << lnb) + b)]);
            dst[(size_t)k * 16] = cadd(cadd(s0, s1), add);
            dst[(size_t)(k + H) * 16] = cadd(csub(s0, s1), add);
        }
    } else {
        for (int k = k0; k < G.Lx; k += ks) dst[(size_t)k * 16] = cadd(Z[padx((k << lnb) + b)], add);
    }
}

// k_ned_gather_blocks: one warp per (grid row, block of 16 columns, 64 time
// samples of the pass).  It holds the 32 columns [c0, c0 + 32) (modulo Lx) of
// the row in registers (two samples per lane) and evaluates every entry whose
// first column bx lies in its block, from the exact first column on:
//   v[t] = sum_k tap[k] r[bx + k][t],  k < W
// (W packed FMAs, a branch on d = bx - c0 in [0, 16)).  Each entry is
// evaluated by exactly one warp, so nothing is shared between warps.
//   adjoint:  E[e][t - nb] = v[t] (e the entry's index in the row CSR)
//   gradient: the two derivative tap sets give v_x, v_y, and the entry's
//             sum_t g[m][t] (v_x[t], v_y[t]) over its 64 samples goes to
//             Qe[e][time chunk].
// Entries (first column, row-CSR index, sensor, taps) arrive 32 at a time by
// asynchronous copies, the next batch while the current one is evaluated.
// ---------------------------------------------------------------------------
template <int W, int D>
__device__ __forceinline__ float2 taps_dot(const float2 (&win)[32], const float* t) {
    // four independent accumulators (tap k into k mod 4), taps read as float4
    const float4* t4 = reinterpret_cast<const float4*>(t);
    float2 a[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
    for (int k4 = 0; k4 < (W + 3) / 4; ++k4) {
        const float4 q = t4[k4];
        const float tk[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (4 * k4 + r < W) a[r] = __ffma2_rn(make_float2(tk[r], tk[r]), win[D + 4 * k4 + r], a[r]);
    }
    return __fadd2_rn(__fadd2_rn(a[0], a[1]), __fadd2_rn(a[2], a[3]));
}

// both derivative tap sets of one entry (ta, tb) at the same offset D: one
// branch for the two dot products
template <int W, int D>
__device__ __forceinline__ void taps_dot2(const float2 (&win)[32], const float* ta, const float* tb, float2& va,
                                          float2& vb) {
    va = taps_dot<W, D>(win, ta);
    vb = taps_dot<W, D>(win, tb);
}

template <int W>
__device__ __forceinline__ void block_taps_dot2(const float2 (&win)[32], int d, const float* ta, const float* tb,
                                                float2& va, float2& vb) {
#define NEDNER_DOT2_CASE(I) \
    case I: taps_dot2<W, I>(win, ta, tb, va, vb); break;
    switch (d) {
        NEDNER_DOT2_CASE(0) NEDNER_DOT2_CASE(1) NEDNER_DOT2_CASE(2) NEDNER_DOT2_CASE(3)
        NEDNER_DOT2_CASE(4) NEDNER_DOT2_CASE(5) NEDNER_DOT2_CASE(6) NEDNER_DOT2_CASE(7)
        NEDNER_DOT2_CASE(8) NEDNER_DOT2_CASE(9) NEDNER_DOT2_CASE(10) NEDNER_DOT2_CASE(11)
        NEDNER_DOT2_CASE(12) NEDNER_DOT2_CASE(13) NEDNER_DOT2_CASE(14)
        default: taps_dot2<W, 15>(win, ta, tb, va, vb); break;
    }
#undef NEDNER_DOT2_CASE
}

// sum_c t[c] win[c] over the NA window-aligned taps (zero outside the entry's
// w), in four independent accumulators, taps read as float4
template <int NA>
__device__ __forceinline__ float2 aligned_taps_dot(const float2 (&win)[32], const float* t) {
    const float4* t4 = reinterpret_cast<const float4*>(t);
    float2 a[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
    for (int c4 = 0; c4 < NA / 4; ++c4) {
        const float4 q = t4[c4];
        a[0] = __ffma2_rn(make_float2(q.x, q.x), win[4 * c4 + 0], a[0]);
        a[1] = __ffma2_rn(make_float2(q.y, q.y), win[4 * c4 + 1], a[1]);
        a[2] = __ffma2_rn(make_float2(q.z, q.z), win[4 * c4 + 2], a[2]);
        a[3] = __ffma2_rn(make_float2(q.w, q.w), win[4 * c4 + 3], a[3]);
    }
    return __fadd2_rn(__fadd2_rn(a[0], a[1]), __fadd2_rn(a[2], a[3]));
}

template <int W, bool GRAD>
__global__ void __launch_bounds__(128, GRAD ? 4 : 5) k_ned_gather_blocks(Geo G, int nb, int Tp, const float* __restrict__ Qb,
                                                              const int2* __restrict__ gseg,
                                                              const int* __restrict__ pent_bx,
                                                              const int* __restrict__ xent_rc,
                                                              const int* __restrict__ xent_m,
                                                              const float* __restrict__ taps_a,
                                                              const float* __restrict__ taps_b,
                                                              const float* __restrict__ g, float* __restrict__ E,
                                                              float2* __restrict__ Qe) {
    constexpr int PW = (W + 3) / 4 * 4;
    constexpr int BE = 32;                                           // entries per staged batch
    // adjoint: taps aligned to the window (no branch on the offset); gradient:
    // the two derivative tap sets from the entry's first column
    constexpr int TW = GRAD ? PW : gather_aligned_taps(W);          // taps per set in the table
    constexpr int NTAP = GRAD ? 2 * PW : TW;
    constexpr int BSZ = BE * (3 + NTAP);                             // one batch (4-byte words)
    extern __shared__ float4 smem4[];
    const int q = threadIdx.x >> 5;
    const int ln = threadIdx.x & 31;
    const int nblk = G.Lx >> 4;
    const int gb = blockIdx.x * (blockDim.x >> 5) + q;
    const int gy = gb / nblk;
    const int c0 = (gb - gy * nblk) << 4;
    const int nc = blockIdx.y * 64;                                  // first sample of the warp in the pass
    const int tl = 32 * (ln >> 4) + 2 * (ln & 15);                   // the lane's first sample of the 64

    // the 32 columns of the window, two samples per lane
    float2 win[32];
    {
        const float2* src = reinterpret_cast<const float2*>(Qb + ((size_t)((nc >> 5) + (ln >> 4)) * G.Ly + gy) *
                                                                     G.Lx * 32) + (ln & 15);
#pragma unroll
        for (int c = 0; c < 32; ++c) win[c] = __ldg(src + (size_t)((c0 + c) & (G.Lx - 1)) * 16);
    }
    const int2 rg = gseg[gb];
    const int nent = rg.y - rg.x;
    const int nbt = (nent + BE - 1) / BE;
    int* st = reinterpret_cast<int*>(smem4) + (size_t)q * 2 * BSZ;  // [2][BSZ]: bx, rc, m [BE] each, taps [BE][NTAP]
    auto issue = [&](int b) {
        const int e0 = rg.x + b * BE, n = min(BE, rg.y - e0);
        int* d = st + (b & 1) * BSZ;
        if (ln < n) {
            cp_async(d + ln, pent_bx + e0 + ln, 4);
            cp_async(d + BE + ln, xent_rc + e0 + ln, 4);
            if (GRAD) cp_async(d + 2 * BE + ln, xent_m + e0 + ln, 4);
        }
        float* tp = reinterpret_cast<float*>(d + 3 * BE);
        for (int i = ln; i < n * (TW / 4); i += 32) {
            const int j = i / (TW / 4), k4 = i - j * (TW / 4);
            cp_async(tp + j * NTAP + 4 * k4, taps_a + (size_t)(e0 + j) * TW + 4 * k4, 16);
            if (GRAD) cp_async(tp + j * NTAP + PW + 4 * k4, taps_b + (size_t)(e0 + j) * PW + 4 * k4, 16);
        }
    };
    if (nbt > 0) issue(0);
    cp_async_commit();
    for (int b = 0; b < nbt; ++b) {
        cp_async_wait_all();
        __syncwarp();
        if (b + 1 < nbt) issue(b + 1);
        cp_async_commit();
        const int* d = st + (b & 1) * BSZ;
        const float* tp = reinterpret_cast<const float*>(d + 3 * BE);
        const int n = min(BE, nent - b * BE);
        if (!GRAD) {
#pragma unroll 1
            for (int j = 0; j < n; ++j) {
                const float2 va = aligned_taps_dot<TW>(win, tp + j * NTAP);
                reinterpret_cast<float2*>(E + (size_t)d[BE + j] * Tp + nc)[tl >> 1] = va;
            }
        } else {
            // four entries at a time: their g loads in flight together, the
            // eight sums (x and y per entry) reduced over the warp at once
            // (8 values in 9 shuffles), lane 4 v ends with value v
            for (int j0 = 0; j0 < n; j0 += 4) {
                float2 gv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    gv[u] = (j0 + u < n) ? __ldg(reinterpret_cast<const float2*>(
                                               g + (size_t)d[2 * BE + j0 + u] * G.Nt + nb + nc + tl))
                                         : make_float2(0.f, 0.f);
                float sv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    float sx = 0.f, sy = 0.f;
                    const int j = j0 + u;
                    if (j < n) {
                        const int dd = d[j] - c0;
                        float2 va, vb;
                        block_taps_dot2<W>(win, dd, tp + j * NTAP, tp + j * NTAP + PW, va, vb);
                        sx = fmaf(gv[0].x, va.x, gv[0].y * va.y);
                        sy = fmaf(gv[0].x, vb.x, gv[0].y * vb.y);
                    }
#pragma unroll
                    for (int i = 0; i < 6; ++i) sv[i] = sv[i + 2];
                    sv[6] = sx;
                    sv[7] = sy;
                    gv[0] = gv[1];
                    gv[1] = gv[2];
                    gv[2] = gv[3];
                }
                const bool h16 = ln & 16, h8 = ln & 8, h4 = ln & 4;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    sv[i] = (h16 ? sv[i + 4] : sv[i]) + __shfl_xor_sync(0xffffffffu, h16 ? sv[i] : sv[i + 4], 16);
#pragma unroll
                for (int i = 0; i < 2; ++i)
                    sv[i] = (h8 ? sv[i + 2] : sv[i]) + __shfl_xor_sync(0xffffffffu, h8 ? sv[i] : sv[i + 2], 8);
                float v = (h4 ? sv[1] : sv[0]) + __shfl_xor_sync(0xffffffffu, h4 ? sv[0] : sv[1], 4);
                v += __shfl_xor_sync(0xffffffffu, v, 2);
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                const int vi = (ln >> 2) & 7, j = j0 + (vi >> 1);
                if ((ln & 3) == 0 && j < n)
                    reinterpret_cast<float*>(Qe)[2 * ((size_t)d[BE + j] * (G.Nt >> 6) + ((nb + nc) >> 6)) + (vi & 1)] = v;
            }
        }
        __syncwarp();
    }
}

// g[m][nb + t] = sum_k E[sens_ent[m][k]][t], t < Tp: the sensor's w entries (one per y tap);
// a non-finite result sets NEDNER_FLAG_NONFINITE in *status
__global__ void k_adj_sum(Geo G, int nb, int Tp, const float* __restrict__ E, const int* __restrict__ sens_ent,
                          float* __restrict__ g, int* __restrict__ status) {
    const size_t total = (size_t)G.M * Tp;
    const int ltp = ilog2(Tp);
    bool bad = false;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(i >> ltp), t = (int)(i & (Tp - 1));
        float v = 0.f;
        for (int k = 0; k < G.w; ++k) v += E[(size_t)__ldg(&sens_ent[(size_t)m * G.w + k]) * Tp + t];
        bad |= !isfinite(v);
        g[(size_t)m * G.Nt + nb + t] = v;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, NEDNER_FLAG_NONFINITE);
}

// the same, four consecutive samples per thread (16-byte loads and stores;
// Tp a multiple of 4, g 16-byte aligned); the same sums in the same order
__global__ void k_adj_sum4(Geo G, int nb, int Tp, const float* __restrict__ E, const int* __restrict__ sens_ent,
                           float* __restrict__ g, int* __restrict__ status) {
    const size_t total = (size_t)G.M * Tp / 4;
    const int ltp = ilog2(Tp) - 2;
    bool bad = false;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(i >> ltp), t = 4 * (int)(i & ((Tp >> 2) - 1));
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k = 0; k < G.w; ++k) {
            const float4 e = *reinterpret_cast<const float4*>(
                &E[(size_t)__ldg(&sens_ent[(size_t)m * G.w + k]) * Tp + t]);
            v.x += e.x;
            v.y += e.y;
            v.z += e.z;
            v.w += e.w;
        }
        bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w));
        *reinterpret_cast<float4*>(&g[(size_t)m * G.Nt + nb + t]) = v;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, NEDNER_FLAG_NONFINITE);
}

// entry sum of one pass: the four-sample form where alignment allows
static void launch_adj_sum(const nedner_plan_s& p, int nb, int Tp, const float* E, float* g, cudaStream_t s) {
    const Geo& G = p.geo;
    const bool vec = (Tp % 4) == 0 && (G.Nt % 4) == 0 && ((uintptr_t)g & 15) == 0;
    const size_t total = (size_t)G.M * Tp / (vec ? 4 : 1);
    const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 16);
    if (vec) k_adj_sum4<<<blocks, 256, 0, s>>>(G, nb, Tp, E, p.t.sens_ent, g, p.t.status);
    else k_adj_sum<<<blocks, 256, 0, s>>>(G, nb, Tp, E, p.t.sens_ent, g, p.t.status);
}

// dL/d(x_m, y_m) = sum over the sensor's w entries and the time chunks of Qe
// (one warp per sensor, lanes over (entry, chunk) pairs, fixed order)
__global__ void k_grad_sum(Geo G, int nch, const float2* __restrict__ Qe, const int* __restrict__ sens_ent,
                           float* __restrict__ dxy, int* __restrict__ status) {
    const int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (m >= G.M) return;                       // whole warps: blockDim.x is a multiple of 32
    float sx = 0.f, sy = 0.f;
    for (int i = lane; i < G.w * nch; i += 32) {
        const int k = i / nch, ch = i - k * nch;
        const float2 v = Qe[(size_t)__ldg(&sens_ent[(size_t)m * G.w + k]) * nch + ch];
        sx += v.x;
        sy += v.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) {
        dxy[2 * m] = sx;
        dxy[2 * m + 1] = sy;
        if (!(isfinite(sx) && isfinite(sy))) atomicOr(status, NEDNER_FLAG_NONFINITE);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t configure_adj_kernels(const nedner_plan_s& p) {
    const Chunks& c = p.ch;
    const Geo& G = p.geo;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_img_xr2c_adj<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem5)))
        return e;
    if ((e = cudaFuncSetAttribute(k_img_yfft_adj<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem4)))
        return e;
    const int a = cudaFuncAttributeMaxDynamicSharedMemorySize;
#define NEDNER_ATTR_NER(W, D)                                                                                      \
    if ((e = cudaFuncSetAttribute(k_ner_lines_adj<W, D, 256>, (cudaFuncAttribute)a, (int)c.smem3a))) return e; \
    if ((e = cudaFuncSetAttribute(k_ner_lines_adj<W, D, 512>, (cudaFuncAttribute)a, (int)c.smem3a))) return e;
    NEDNER_ATTR_NER(4, 10) NEDNER_ATTR_NER(6, 10) NEDNER_ATTR_NER(8, 10) NEDNER_ATTR_NER(10, 10)
    NEDNER_ATTR_NER(12, 10) NEDNER_ATTR_NER(14, 12) NEDNER_ATTR_NER(16, 12)
#undef NEDNER_ATTR_NER
    if ((e = cudaFuncSetAttribute(k_ned_yfft_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem2f))) return e;
#define NEDNER_ATTR_GATHER(WT, PER)                                                                         \
    if ((e = cudaFuncSetAttribute(k_ned_gather_rows<WT, PER, false>, (cudaFuncAttribute)a, (int)c.smem_adj))) return e; \
    if ((e = cudaFuncSetAttribute(k_ned_gather_rows<WT, PER, true>, (cudaFuncAttribute)a, (int)c.smem_grad))) return e;
    NEDNER_ATTR_GATHER(8, 16) NEDNER_ATTR_GATHER(12, 16) NEDNER_ATTR_GATHER(16, 16) NEDNER_ATTR_GATHER(20, 16)
#undef NEDNER_ATTR_GATHER
#define NEDNER_ATTR_GATHER2(WT)                                                                             \
    if ((e = cudaFuncSetAttribute(k_ned_gather_rows2<WT, false, 256>, (cudaFuncAttribute)a, (int)c.smem_adj))) return e; \
    if ((e = cudaFuncSetAttribute(k_ned_gather_rows2<WT, true, 256>, (cudaFuncAttribute)a, (int)c.smem_grad))) return e; \
    if ((e = cudaFuncSetAttribute(k_ned_gather_rows2<WT, false, 512>, (cudaFuncAttribute)a, (int)c.smem_adj))) return e; \
    if ((e = cudaFuncSetAttribute(k_ned_gather_rows2<WT, true, 512>, (cudaFuncAttribute)a, (int)c.smem_grad))) return e;
    NEDNER_ATTR_GATHER2(8) NEDNER_ATTR_GATHER2(12) NEDNER_ATTR_GATHER2(16) NEDNER_ATTR_GATHER2(20)
#undef NEDNER_ATTR_GATHER2
    if ((e = cudaFuncSetAttribute(k_ned_xfft_adj<16>, (cudaFuncAttribute)a, (int)xfft_adj_smem(c)))) return e;
    if ((e = cudaFuncSetAttribute(k_ned_xfft_adj<32>, (cudaFuncAttribute)a, (int)xfft_adj_smem(c)))) return e;
#define NEDNER_ATTR_BG(W)                                                                                   \
    if ((e = cudaFuncSetAttribute(k_ned_gather_blocks<W, false>, (cudaFuncAttribute)a, (int)c.smem_ga))) return e; \
    if ((e = cudaFuncSetAttribute(k_ned_gather_blocks<W, true>, (cudaFuncAttribute)a, (int)c.smem_gg))) return e;
    NEDNER_ATTR_BG(4) NEDNER_ATTR_BG(6) NEDNER_ATTR_BG(8) NEDNER_ATTR_BG(10) NEDNER_ATTR_BG(12) NEDNER_ATTR_BG(14)
    NEDNER_ATTR_BG(16)
#undef NEDNER_ATTR_BG
    return cudaSuccess;
}

cudaError_t launch_img_xr2c_adj(const nedner_plan_s& p, const float* p0, float2* Y, cudaStream_t s) {
    const Geo& G = p.geo;
    k_img_xr2c_adj<128><<<dim3(G.nz, G.ny / p.ch.c5), 128, p.ch.smem5, s>>>(G, p.ch.c5, p0, p.t.tw, Y);
    return cudaGetLastError();
}

cudaError_t launch_img_yfft_adj(const nedner_plan_s& p, const float2* Y, float2* V, cudaStream_t s) {
    const Geo& G = p.geo;
    k_img_yfft_adj<128><<<dim3(G.nxh, G.nz / p.ch.c4), 128, p.ch.smem4, s>>>(G, p.ch.c4, Y, p.t.tw, V);
    return cudaGetLastError();
}

cudaError_t launch_ner_lines_adj(const nedner_plan_s& p, const float2* V, float2* Ghat, cudaStream_t s) {
    const Geo& G = p.geo;
    const dim3 grid(G.nxh * (G.ny / p.ch.lpc));
#define NEDNER_NER(W, D)                                                                                        \
    if (p.ch.threads3 <= 256)                                                                                   \
        k_ner_lines_adj<W, D, 256><<<grid, 256, p.ch.smem3a, s>>>(G, p.tap, p.ch.lpc, p.ch.icap3a, V, p.t.axy,   \
                                                                  p.t.deconv_t,                                \
                                                                  p.t.deconv_y, p.t.tw, Ghat);                  \
    else                                                                                                        \
        k_ner_lines_adj<W, D, 512><<<grid, 512, p.ch.smem3a, s>>>(G, p.tap, p.ch.lpc, p.ch.icap3a, V, p.t.axy,   \
                                                                  p.t.deconv_t,                                \
                                                                  p.t.deconv_y, p.t.tw, Ghat)
    switch (G.w) {
        case 4: NEDNER_NER(4, 10); break;
        case 6: NEDNER_NER(6, 10); break;
        case 8: NEDNER_NER(8, 10); break;
        case 10: NEDNER_NER(10, 10); break;
        case 12: NEDNER_NER(12, 10); break;
        case 14: NEDNER_NER(14, 12); break;
        default: NEDNER_NER(16, 12); break;
    }
#undef NEDNER_NER
    return cudaGetLastError();
}

cudaError_t launch_ned_yfft_adj(const nedner_plan_s& p, const float2* Ghat, float2* R, cudaStream_t s) {
    const Geo& G = p.geo;
    k_ned_yfft_adj<<<dim3(G.Nt / p.ch.c2f, G.nxh), 256, p.ch.smem2f, s>>>(G, p.ch.c2f, Ghat, p.t.deconv_y, p.t.tw, R);
    return cudaGetLastError();
}

// the transposed gather kernel, by tap count
#define NEDNER_GATHER_SWITCH(CALL)      \
    switch (spread_taps(G.w)) {         \
        case 8: CALL(8); break;         \
        case 12: CALL(12); break;       \
        case 16: CALL(16); break;       \
        default: CALL(20); break;       \
    }

// block gather of one pass [nb, nb + Tp): transposed x-FFT into Qb, then the
// blocks (adjoint: entry values into E; gradient: per-entry sums into Qe)
static cudaError_t launch_block_gather(const nedner_plan_s& p, const float2* R, float* Qb, int nb, int Tp, bool grad,
                                       const float* g, float* E, float2* Qe, cudaStream_t s, StageTimer* tm) {
    const Geo& G = p.geo;
    const dim3 gx(G.Ly, Tp / (2 * p.ch.nbx));
    if (p.ch.perx <= 16)
        k_ned_xfft_adj<16><<<gx, p.ch.thx, xfft_adj_smem(p.ch), s>>>(G, nb, p.ch.nbx, R, p.t.deconv_x, p.t.tw, Qb);
    else
        k_ned_xfft_adj<32><<<gx, p.ch.thx, xfft_adj_smem(p.ch), s>>>(G, nb, p.ch.nbx, R, p.t.deconv_x, p.t.tw, Qb);
    stage_mark(tm, 4);
    const dim3 grid(G.Ly * (G.Lx / 16) / 4, Tp / 64);
#define NEDNER_BG(W)                                                                                              \
    if (grad)                                                                                                     \
        k_ned_gather_blocks<W, true><<<grid, 128, p.ch.smem_gg, s>>>(G, nb, Tp, Qb, p.t.gseg, p.t.pent_bx,         \
                                                                     p.t.xent_rc, p.t.xent_m, p.t.pent_gx,         \
                                                                     p.t.pent_gy, g, E, Qe);                       \
    else                                                                                                          \
        k_ned_gather_blocks<W, false><<<grid, 128, p.ch.smem_ga, s>>>(G, nb, Tp, Qb, p.t.gseg, p.t.pent_bx,        \
                                                                      p.t.xent_rc, p.t.xent_m, p.t.pent_w,         \
                                                                      p.t.pent_w, g, E, Qe)
    switch (G.w) {
        case 4: NEDNER_BG(4); break;
        case 6: NEDNER_BG(6); break;
        case 8: NEDNER_BG(8); break;
        case 10: NEDNER_BG(10); break;
        case 12: NEDNER_BG(12); break;
        case 14: NEDNER_BG(14); break;
        default: NEDNER_BG(16); break;
    }
#undef NEDNER_BG
    stage_mark(tm, 5);
    return cudaGetLastError();
}

// region A after R-bar: the block gather's pass grid
static float* pass_grid(const nedner_plan_s& p) {
    const size_t rbar = ((size_t)p.geo.nxh * p.geo.Ly * p.geo.Nt * 8 + 255) / 256 * 256;
    return (float*)((char*)p.ws + rbar);
}

cudaError_t launch_adj_gather(const nedner_plan_s& p, const float2* R, float* E, float* g, cudaStream_t s,
                              StageTimer* tm) {
    const Geo& G = p.geo;
    const int C = p.ch.ca, Tp = p.ch.tp_adj;
    if (p.ch.gsplit) {
        cudaError_t e = cudaSuccess;
        for (int nb = 0; nb < G.Nt && !e; nb += Tp) {
            e = launch_block_gather(p, R, pass_grid(p), nb, Tp, false, nullptr, E, nullptr, s, tm);
            if (e) break;
            launch_adj_sum(p, nb, Tp, E, g, s);
            stage_mark(tm, 6);
            e = cudaGetLastError();
        }
        return e;
    }
    for (int nb = 0; nb < G.Nt; nb += Tp) {
        const dim3 grid(G.Ly, Tp / C);
#define NEDNER_ADJ(WT)                                                                                            \
    if (p.ch.tpl_adj == 2 && p.ch.threads_adj == 512)                                                             \
        k_ned_gather_rows2<WT, false, 512><<<grid, 512, p.ch.smem_adj, s>>>(G, nb, Tp, R, nullptr, p.t.xrow_ptr,  \
                                                                            p.t.xrow_first, p.t.xent_m,           \
                                                                            p.t.xent_bx, p.t.xent_rc, p.t.xent_wx, \
                                                                            p.t.xent_wx, p.t.deconv_x, p.t.tw, E, \
                                                                            nullptr);                             \
    else if (p.ch.tpl_adj == 2)                                                                                   \
        k_ned_gather_rows2<WT, false, 256><<<grid, 256, p.ch.smem_adj, s>>>(G, nb, Tp, R, nullptr, p.t.xrow_ptr,  \
                                                                            p.t.xrow_first, p.t.xent_m,           \
                                                                            p.t.xent_bx, p.t.xent_rc, p.t.xent_wx, \
                                                                            p.t.xent_wx, p.t.deconv_x, p.t.tw, E, \
                                                                            nullptr);                             \
    else                                                                                                          \
    k_ned_gather_rows<WT, 16, false><<<grid, 256, p.ch.smem_adj, s>>>(G, C, nb, Tp, R, nullptr, p.t.xrow_ptr,       \
                                                                      p.t.xrow_first, p.t.xent_m, p.t.xent_bx,      \
                                                                      p.t.xent_rc, p.t.xent_wx, p.t.xent_wx,        \
                                                                      p.t.deconv_x, p.t.tw, E, nullptr)
        NEDNER_GATHER_SWITCH(NEDNER_ADJ)
#undef NEDNER_ADJ
        stage_mark(tm, 5);
        launch_adj_sum(p, nb, Tp, E, g, s);
        stage_mark(tm, 6);
    }
    return cudaGetLastError();
}

cudaError_t launch_grad_gather(const nedner_plan_s& p, const float2* R, const float* g, float2* Qe, float* dxy,
                               cudaStream_t s, StageTimer* tm) {
    const Geo& G = p.geo;
    const int C = p.ch.ca;
    const dim3 grid(G.Ly, G.Nt / C);
    if (p.ch.gsplit) {
        cudaError_t e = cudaSuccess;
        for (int nb = 0; nb < G.Nt && !e; nb += p.ch.tp_g)
            e = launch_block_gather(p, R, pass_grid(p), nb, p.ch.tp_g, true, g, nullptr, Qe, s, tm);
        if (e) return e;
        k_grad_sum<<<(G.M + 7) / 8, 256, 0, s>>>(G, G.Nt / 64, Qe, p.t.sens_ent, dxy, p.t.status);
        stage_mark(tm, 6);
        return cudaGetLastError();
    }
#define NEDNER_GRAD(WT)                                                                                          \
    if (p.ch.tpl_adj == 2 && p.ch.threads_adj == 512)                                                             \
        k_ned_gather_rows2<WT, true, 512><<<grid, 512, p.ch.smem_grad, s>>>(G, 0, G.Nt, R, g, p.t.xrow_ptr,       \
                                                                            p.t.xrow_first, p.t.xent_m,           \
                                                                            p.t.xent_bx, p.t.xent_rc, p.t.xent_gx, \
                                                                            p.t.xent_gy, p.t.deconv_x, p.t.tw,    \
                                                                            nullptr, Qe);                         \
    else if (p.ch.tpl_adj == 2)                                                                                   \
        k_ned_gather_rows2<WT, true, 256><<<grid, 256, p.ch.smem_grad, s>>>(G, 0, G.Nt, R, g, p.t.xrow_ptr,       \
                                                                            p.t.xrow_first, p.t.xent_m,           \
                                                                            p.t.xent_bx, p.t.xent_rc, p.t.xent_gx, \
                                                                            p.t.xent_gy, p.t.deconv_x, p.t.tw,    \
                                                                            nullptr, Qe);                         \
    else                                                                                                          \
    k_ned_gather_rows<WT, 16, true><<<grid, 256, p.ch.smem_grad, s>>>(G, C, 0, G.Nt, R, g, p.t.xrow_ptr,           \
                                                                      p.t.xrow_first, p.t.xent_m, p.t.xent_bx,     \
                                                                      p.t.xent_rc, p.t.xent_gx, p.t.xent_gy,       \
                                                                      p.t.deconv_x, p.t.tw, nullptr, Qe)
    NEDNER_GATHER_SWITCH(NEDNER_GRAD)
#undef NEDNER_GRAD
    stage_mark(tm, 5);
    k_grad_sum<<<(G.M + 7) / 8, 256, 0, s>>>(G, G.Nt / C, Qe, p.t.sens_ent, dxy, p.t.status);
    stage_mark(tm, 6);
    return cudaGetLastError();
}

}  // namespace nedner

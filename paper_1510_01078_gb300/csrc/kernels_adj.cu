// Transposed NEDNER kernels: g = R^T p (nedner_adjoint) and the
// sensor-position gradient (nedner_grad_positions).
//
// Each kernel is the exact transpose (for real inner products) of one forward
// stage, run in reverse order:
//   p  [nz][ny][nx]
//     -- img_xr2c_adj    -->  Y [nx/2+1][nz][ny]    r2c along x, times 1 or 2
//     -- img_yfft_adj    -->  V [nx/2+1][ny][nz]    forward FFT along y
//     -- ner_lines_adj   -->  Ghat [nx/2+1][ny+1][Nt]  z-FFT, fold^T, W, NER spreading, IFFT
//     -- ned_yfft_adj    -->  R [nx/2+1][Ly][Nt]    pad, deconvolve, IFFT along y
//     -- ned_interp_adj  -->  P [2][M][Nt]          real IFFT along x, interpolation per row block
//     -- adj_finish      -->  g [M][Nt]             sum of the (at most two) row-block partials
// The position gradient replaces the last two by ned_grad (derivative taps,
// dotted with g over time) and grad_finish.
#include <cuda_runtime.h>

#include <algorithm>

#include "fft.cuh"
#include "internal.h"

namespace nedner {

// ---------------------------------------------------------------------------
// Transpose of img_xc2r: Y[kx] = d_kx sum_qx p[qx] exp(-2 pi i kx qx / nx),
// kx = 0..nx/2, d = 1 at kx = 0, nx/2 and 2 otherwise.  Real-to-complex FFT
// through the half-length complex transform of z[p] = x[2p] + i x[2p+1].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_img_xr2c_adj(Geo G, int C, const float* __restrict__ p0,
                                                      const float2* __restrict__ tw, float2* __restrict__ Y) {
    extern __shared__ float4 smem4[];
    const int H = G.nx / 2;
    const int ld = C + 1;
    float2* A = reinterpret_cast<float2*>(smem4);   // [H][ld]
    float2* B = A + (size_t)H * ld;                 // [H][ld]
    const int qz = blockIdx.x;
    const int y0 = blockIdx.y * C;
    const int lc = ilog2(C), lh = ilog2(H);
#pragma unroll 8
    for (int it = threadIdx.x; it < H * C; it += blockDim.x) {
        const int c = it >> lh;
        const int pp = it & (H - 1);
        A[pp * ld + c] = reinterpret_cast<const float2*>(p0 + ((size_t)qz * G.ny + y0 + c) * G.nx)[pp];
    }
    float2* Z = block_fft(A, B, H, C, ld, -1, tw);
    for (int it = threadIdx.x; it < (H + 1) * C; it += blockDim.x) {
        const int k = it >> lc;
        const int c = it & (C - 1);
        const float2 zk = Z[(k & (H - 1)) * ld + c];
        const float2 zm = cconj(Z[((H - k) & (H - 1)) * ld + c]);
        const float2 E = cscale(cadd(zk, zm), 0.5f);
        const float2 O = cscale(mul_i(csub(zk, zm), -1), 0.5f);     // (zk - zm) / (2i)
        float2 X = cadd(E, cmul(twiddle(tw, k & (G.nx - 1), G.nx, -1), O));
        if (k != 0 && k != H) X = cscale(X, 2.f);
        Y[((size_t)k * G.nz + qz) * G.ny + y0 + c] = X;
    }
}

// ---------------------------------------------------------------------------
// Transpose of img_yifft: V[kx][ky][qz] = sum_qy exp(-2 pi i ky qy / ny) Y[kx][qz][qy].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_img_yfft_adj(Geo G, int C, const float2* __restrict__ Y,
                                                      const float2* __restrict__ tw, float2* __restrict__ V) {
    extern __shared__ float4 smem4[];
    const int ld = C + 1;
    float2* A = reinterpret_cast<float2*>(smem4);
    float2* B = A + (size_t)G.ny * ld;
    const int kx = blockIdx.x;
    const int z0 = blockIdx.y * C;
    const int lc = ilog2(C), lny = ilog2(G.ny);
#pragma unroll 8
    for (int it = threadIdx.x; it < G.ny * C; it += blockDim.x) {
        const int c = it >> lny;
        const int qy = it & (G.ny - 1);
        A[qy * ld + c] = Y[((size_t)kx * G.nz + z0 + c) * G.ny + qy];
    }
    float2* res = block_fft(A, B, G.ny, C, ld, -1, tw);
    for (int it = threadIdx.x; it < G.ny * C; it += blockDim.x) {
        const int ky = it >> lc;
        const int c = it & (C - 1);
        V[((size_t)kx * G.ny + ky) * G.nz + z0 + c] = res[ky * ld + c];
    }
}

// ---------------------------------------------------------------------------
// Transpose of ner_lines, one CTA per line group (kx, ky).
//   Ubar = FFT_nz(sign V[line])                       (transpose of the z-IFFT)
//   Tbar_a[l] = ca Ubar[l]          for l = -nz/2..nz/2-1
//   Tbar_b[e] = cb Ubar[slot(e)]    e = l* of some slot l (none for e = -nz/2)
//   Tbar      *= coefficient(e) (Jacobian, scale, band mask)
//   Bbar[mu] = sum_e exp(+i pi nu_e) phi(sigma nu_e - mu) Tbar[e]   (spreading)
//   Ghat-bar[n] = IFFT_Lt(Bbar)[(n - Nt/2) mod Lt] / phihat((n - Nt/2)/Lt)
// Spreading uses shared-memory atomics: a CTA owns its line, so nothing is
// shared between CTAs.
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

// B[(mu0 + k) mod Lt] += P_k(s) v for the W taps (Horner, unrolled)
template <int W, int D>
__device__ __forceinline__ void ner_scatter(const TapPoly& P, float2* LA, int mu0, float s, int Lt, float2 v) {
#pragma unroll
    for (int k = 0; k < W; ++k) {
        float p = P.c[k * (D + 1) + D];
#pragma unroll
        for (int d = D - 1; d >= 0; --d) p = fmaf(p, s, P.c[k * (D + 1) + d]);
        float2* dst = &LA[(mu0 + k) & (Lt - 1)];
        atomicAdd(&dst->x, p * v.x);
        atomicAdd(&dst->y, p * v.y);
    }
}

template <int W, int D>
__global__ void __launch_bounds__(256) k_ner_lines_adj(Geo G, const __grid_constant__ TapPoly P,
                                                       const float2* __restrict__ V,
                                                       const float2* __restrict__ axy_tab,
                                                       const float* __restrict__ deconv_t,
                                                       const float2* __restrict__ tw, float2* __restrict__ Ghat) {
    extern __shared__ float4 smem4[];
    float2* LA = reinterpret_cast<float2*>(smem4);   // [Lt]
    float2* LB = LA + G.Lt;                          // [Lt]
    float2* T = LB + G.Lt;                           // [nz + 1]
    float2* UA = T + (G.nz + 1);                     // [nz]
    float2* UB = UA + G.nz;                          // [nz]

    const int grp = blockIdx.x;
    const int kx = grp >> ilog2(G.ny);
    const int ky = (grp & (G.ny - 1)) - G.ny / 2;
    const int kyb = (ky == -G.ny / 2) ? G.ny / 2 : ky;
    const bool nyq_x = (kx == G.nx / 2);
    const float ca = nyq_x ? 0.f : 0.5f;
    const float cb = nyq_x ? 1.f : 0.5f;
    const int half_nz = G.nz / 2;
    const float sg = ((kx + ky) & 1) ? -1.f : 1.f;

    const float2* src = V + ((size_t)kx * G.ny + (ky & (G.ny - 1))) * G.nz;
#pragma unroll 4
    for (int q = threadIdx.x; q < G.nz; q += blockDim.x) UA[q] = cscale(src[q], sg);
    float2* Ub = block_fft(UA, UB, G.nz, 1, 1, -1, tw);

    const int nlines = (nyq_x || ky == kyb) ? 1 : 2;
    for (int li = 0; li < nlines; ++li) {
        const int lky = (li == 0 && nlines == 2) ? ky : kyb;
        const size_t line = (size_t)kx * G.nyp + (lky + G.ny / 2);
        const float2 axy = __ldg(&axy_tab[line]);
        const bool is_a = !nyq_x && (lky == ky);
        const bool is_b = (lky == kyb);

        __syncthreads();
        for (int p = threadIdx.x; p < G.Lt; p += blockDim.x) LA[p] = make_float2(0.f, 0.f);
        __syncthreads();
        for (int e = threadIdx.x; e <= G.nz; e += blockDim.x) {
            const int l = e - half_nz;
            float2 tb = make_float2(0.f, 0.f);
            if (is_a && e < G.nz) tb = cadd(tb, cscale(Ub[l & (G.nz - 1)], ca));
            if (is_b && e > 0) {
                // e = +nz/2 feeds slot -nz/2; other e feed slot e
                const int slot = (e == G.nz) ? (-half_nz & (G.nz - 1)) : (l & (G.nz - 1));
                tb = cadd(tb, cscale(Ub[slot], cb));
            }
            FF2 nu = nu_abs2(G, axy, l);
            float Wj;
            if (l == 0) {
                Wj = (kx == 0 && lky == 0) ? 2.f : 0.f;
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
            tb = cscale(tb, cl);
            if (tb.x != 0.f || tb.y != 0.f) {
                const float vh = 2.f * nu.hi, vl = 2.f * nu.lo;
                float fl = floorf(vh);
                float t = (vh - fl) + vl;
                if (t < 0.f) { t += 1.f; fl -= 1.f; }
                if (t >= 1.f) { t -= 1.f; fl += 1.f; }
                const int ifl = (int)fl;
                const int mu0 = ifl - W / 2 + 1;
                // exp(+i pi nu) = i^floor(v) exp(+i pi t / 2)
                float sn, cs;
                sincospif(0.5f * t, &sn, &cs);
                float2 ph = make_float2(cs, sn);
                const int q = ifl & 3;
                if (q == 1) ph = make_float2(-ph.y, ph.x);
                else if (q == 2) ph = make_float2(-ph.x, -ph.y);
                else if (q == 3) ph = make_float2(ph.y, -ph.x);
                ner_scatter<W, D>(P, LA, mu0, 2.f * t - 1.f, G.Lt, cmul(ph, tb));
            }
        }
        float2* z = block_fft(LA, LB, G.Lt, 1, 1, +1, tw);
        float2* dst = Ghat + line * G.Nt;
        for (int n = threadIdx.x; n < G.Nt; n += blockDim.x)
            dst[n] = cscale(z[(n - G.Nt / 2) & (G.Lt - 1)], __ldg(&deconv_t[n]));
    }
    if (nyq_x && ky == -G.ny / 2) {
        // the line (nx/2, -ny/2) is not used by the forward map: its transpose is zero
        float2* dst = Ghat + ((size_t)kx * G.nyp + 0) * G.Nt;
        for (int n = threadIdx.x; n < G.Nt; n += blockDim.x) dst[n] = make_float2(0.f, 0.f);
    }
}

// ---------------------------------------------------------------------------
// Transpose of ned_yfft: R[jx][gy][n] = sum_jy exp(+2 pi i jy gy / Ly) Ghat[jx][jy][n] / phihat(jy/Ly).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_ned_yfft_adj(Geo G, int C, const float2* __restrict__ Ghat,
                                                      const float* __restrict__ deconv_y,
                                                      const float2* __restrict__ tw, float2* __restrict__ R) {
    extern __shared__ float4 smem4[];
    float2* A = reinterpret_cast<float2*>(smem4);
    float2* B = A + (size_t)G.Ly * C;
    const int jx = blockIdx.x;
    const int n0 = blockIdx.y * C;
    const int lc = ilog2(C);
    for (int it = threadIdx.x; it < G.Ly * C; it += blockDim.x) A[it] = make_float2(0.f, 0.f);
    __syncthreads();
#pragma unroll 8
    for (int it = threadIdx.x; it < G.nyp * C; it += blockDim.x) {
        const int b = it >> lc;
        const int c = it & (C - 1);
        const int q = (b - G.ny / 2 + G.Ly) & (G.Ly - 1);
        A[q * C + c] = cscale(Ghat[((size_t)jx * G.nyp + b) * G.Nt + n0 + c], __ldg(&deconv_y[b]));
    }
    float2* res = block_fft(A, B, G.Ly, C, C, +1, tw);
    for (int it = threadIdx.x; it < G.Ly * C; it += blockDim.x) {
        const int gy = it >> lc;
        const int c = it & (C - 1);
        R[((size_t)jx * G.Ly + gy) * G.Nt + n0 + c] = res[it];
    }
}

// ---------------------------------------------------------------------------
// Transpose of the x part of ned_spread_xfft for one grid row: the real row
//   r[gx] = Re sum_{jx=0}^{nx/2} R[jx] exp(+2 pi i jx gx / Lx) / phihat(jx/Lx)
// for C time samples, as the inverse FFT of the Hermitian part of the
// zero-extended spectrum (two real columns packed per complex column).
// Leaves r as floats [Lx][C] in the returned buffer.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float* row_real_ifft(const Geo& G, int C, const float2* __restrict__ R, int gy, int n0,
                                                const float* __restrict__ deconv_x, const float2* __restrict__ tw,
                                                float2* Z, float2* Zs) {
    const int Lx = G.Lx;
    const int nb = C / 2;
    const int lnb = ilog2(nb);
    for (int it = threadIdx.x; it < Lx * nb; it += blockDim.x) Z[it] = make_float2(0.f, 0.f);
    __syncthreads();
#pragma unroll 4
    for (int it = threadIdx.x; it < G.nxh * nb; it += blockDim.x) {
        const int jx = it >> lnb;
        const int b = it & (nb - 1);
        const float d = __ldg(&deconv_x[jx]);
        const float2* src = R + ((size_t)jx * G.Ly + gy) * G.Nt + n0 + 2 * b;
        const float2 y1 = cscale(src[0], d);
        const float2 y2 = cscale(src[1], d);
        if (jx == 0) {
            Z[b] = make_float2(y1.x, y2.x);                       // Re Y1[0] + i Re Y2[0]
        } else {
            // H[k] = Y[k]/2, H[Lx-k] = conj(Y[k])/2; Z = H1 + i H2
            Z[jx * nb + b] = cscale(cadd(y1, mul_i(y2, +1)), 0.5f);
            Z[(Lx - jx) * nb + b] = cscale(cadd(cconj(y1), mul_i(cconj(y2), +1)), 0.5f);
        }
    }
    return reinterpret_cast<float*>(block_fft(Z, Zs, Lx, nb, nb, +1, tw));
}

// ---------------------------------------------------------------------------
// Transposed interpolation: one CTA per (task, C time samples).  A task is a
// block of kRowBlock grid rows and a slice [s0, s1) of the sensors touching
// it.  For each row the CTA rebuilds the real row r (row_real_ifft), then for
// every (sensor, y tap) entry of the row whose sensor is in the slice adds
//   row_w * sum_k wx[m][k] r[(bx_m + k) mod Lx]
// to that sensor's accumulator.  A sensor's rows span at most two blocks; the
// partial of each block goes to P[slot][m][n] (slot 0 = block of its first
// row) and adj_finish adds them.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_ned_interp_adj(Geo G, int C, int smax, const float2* __restrict__ R,
                                                        const int4* __restrict__ tasks,
                                                        const int* __restrict__ row_ptr,
                                                        const int* __restrict__ row_m,
                                                        const float* __restrict__ row_w,
                                                        const int* __restrict__ row_local,
                                                        const int* __restrict__ band_m,
                                                        const int* __restrict__ band_slot,
                                                        const int* __restrict__ sens_bx,
                                                        const float* __restrict__ sens_wx,
                                                        const float* __restrict__ deconv_x,
                                                        const float2* __restrict__ tw, float* __restrict__ P) {
    extern __shared__ float4 smem4[];
    float2* Z = reinterpret_cast<float2*>(smem4);            // [Lx][C/2]
    float2* Zs = Z + (size_t)G.Lx * (C / 2);                 // [Lx][C/2]
    float* acc = reinterpret_cast<float*>(Zs + (size_t)G.Lx * (C / 2));   // [smax][C]
    const int4 tk = tasks[blockIdx.x];                       // block, s0, s1, band start of block
    const int n0 = blockIdx.y * C;
    const int nloc = tk.z - tk.y;
    const int off = tk.y - tk.w;                             // first local index of this slice
    const int lc = ilog2(C);
    const int groups = blockDim.x >> lc;
    const int q = threadIdx.x >> lc;
    const int ln = threadIdx.x & (C - 1);
    const int Lx = G.Lx;

    for (int i = threadIdx.x; i < nloc * C; i += blockDim.x) acc[i] = 0.f;
    for (int rr = 0; rr < kRowBlock; ++rr) {
        const int gy = tk.x * kRowBlock + rr;
        const float* r = row_real_ifft(G, C, R, gy, n0, deconv_x, tw, Z, Zs);
        for (int e = row_ptr[gy] + q; e < row_ptr[gy + 1]; e += groups) {
            const int loc = row_local[e] - off;
            if (loc < 0 || loc >= nloc) continue;
            const int m = row_m[e];
            const int bx = sens_bx[m];
            const float* wx = sens_wx + (size_t)m * G.w;
            float t = 0.f;
            for (int k = 0; k < G.w; ++k) t = fmaf(__ldg(&wx[k]), r[((bx + k) & (Lx - 1)) * C + ln], t);
            acc[loc * C + ln] = fmaf(row_w[e], t, acc[loc * C + ln]);
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < nloc * C; i += blockDim.x) {
        const int loc = i >> lc;
        const int c = i & (C - 1);
        const int b = tk.y + loc;
        P[((size_t)band_slot[b] * G.M + band_m[b]) * G.Nt + n0 + c] = acc[i];
    }
}

__global__ void k_adj_finish(Geo G, const float* __restrict__ P, const unsigned char* __restrict__ two,
                             float* __restrict__ g) {
    const size_t total = (size_t)G.M * G.Nt;
    const int lnt = ilog2(G.Nt);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(i >> lnt);
        float v = P[i];
        if (two[m]) v += P[total + i];
        g[i] = v;
    }
}

// ---------------------------------------------------------------------------
// Position gradient (Eq. disc_rec differentiated in x_m, y_m):
//   dL/dx_m = sum_n g[m][n] sum_rows wy*fac * sum_k dwx[m][k] r[..][n]
//   dL/dy_m = sum_n g[m][n] sum_rows dwy*fac * sum_k wx[m][k]  r[..][n]
// with r the transposed stages applied to dL/dp0.  Same task layout as
// ned_interp_adj; each entry's contribution is reduced over its C time
// samples with shuffles, accumulated per sensor, and written to
// Q[slot][time chunk][m]; grad_finish sums chunks and slots.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_ned_grad(Geo G, int C, int smax, const float2* __restrict__ R,
                                                  const float* __restrict__ g,
                                                  const int4* __restrict__ tasks,
                                                  const int* __restrict__ row_ptr,
                                                  const int* __restrict__ row_m,
                                                  const float* __restrict__ row_w,
                                                  const float* __restrict__ row_dw,
                                                  const int* __restrict__ row_local,
                                                  const int* __restrict__ band_m,
                                                  const int* __restrict__ band_slot,
                                                  const int* __restrict__ sens_bx,
                                                  const float* __restrict__ sens_wx,
                                                  const float* __restrict__ sens_dwx,
                                                  const float* __restrict__ deconv_x,
                                                  const float2* __restrict__ tw, float2* __restrict__ Q) {
    extern __shared__ float4 smem4[];
    float2* Z = reinterpret_cast<float2*>(smem4);
    float2* Zs = Z + (size_t)G.Lx * (C / 2);
    float2* acc = Zs + (size_t)G.Lx * (C / 2);               // [smax] (d/dx, d/dy)
    const int4 tk = tasks[blockIdx.x];
    const int n0 = blockIdx.y * C;
    const int nloc = tk.z - tk.y;
    const int off = tk.y - tk.w;
    const int lc = ilog2(C);
    const int groups = blockDim.x >> lc;
    const int q = threadIdx.x >> lc;
    const int ln = threadIdx.x & (C - 1);
    const int Lx = G.Lx;

    for (int i = threadIdx.x; i < nloc; i += blockDim.x) acc[i] = make_float2(0.f, 0.f);
    for (int rr = 0; rr < kRowBlock; ++rr) {
        const int gy = tk.x * kRowBlock + rr;
        const float* r = row_real_ifft(G, C, R, gy, n0, deconv_x, tw, Z, Zs);
        const int e_beg = row_ptr[gy], e_end = row_ptr[gy + 1];
        // every lane of a group walks the same entries so the shuffles stay converged
        for (int e0 = e_beg; e0 < e_end; e0 += groups) {
            const int e = e0 + q;
            float sx = 0.f, sy = 0.f;
            int loc = -1;
            if (e < e_end) {
                loc = row_local[e] - off;
                if (loc >= 0 && loc < nloc) {
                    const int m = row_m[e];
                    const int bx = sens_bx[m];
                    const float* wx = sens_wx + (size_t)m * G.w;
                    const float* dwx = sens_dwx + (size_t)m * G.w;
                    float tx = 0.f, ty = 0.f;
                    for (int k = 0; k < G.w; ++k) {
                        const float rv = r[((bx + k) & (Lx - 1)) * C + ln];
                        tx = fmaf(__ldg(&dwx[k]), rv, tx);
                        ty = fmaf(__ldg(&wx[k]), rv, ty);
                    }
                    const float gv = __ldg(&g[(size_t)m * G.Nt + n0 + ln]);
                    sx = row_w[e] * tx * gv;
                    sy = row_dw[e] * ty * gv;
                } else {
                    loc = -1;
                }
            }
            for (int o = C / 2; o > 0; o >>= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sy += __shfl_xor_sync(0xffffffffu, sy, o);
            }
            if (ln == 0 && loc >= 0) {
                float2 a = acc[loc];
                acc[loc] = make_float2(a.x + sx, a.y + sy);
            }
        }
        __syncthreads();
    }
    const int nchunk = G.Nt / C;
    for (int i = threadIdx.x; i < nloc; i += blockDim.x) {
        const int b = tk.y + i;
        Q[((size_t)band_slot[b] * nchunk + blockIdx.y) * G.M + band_m[b]] = acc[i];
    }
}

__global__ void k_grad_finish(Geo G, int nchunk, const float2* __restrict__ Q, const unsigned char* __restrict__ two,
                              float* __restrict__ dxy) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= G.M) return;
    float sx = 0.f, sy = 0.f;
    const int nslot = two[m] ? 2 : 1;
    for (int sl = 0; sl < nslot; ++sl)
        for (int ch = 0; ch < nchunk; ++ch) {
            const float2 v = Q[((size_t)sl * nchunk + ch) * G.M + m];
            sx += v.x;
            sy += v.y;
        }
    dxy[2 * m] = sx;
    dxy[2 * m + 1] = sy;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t configure_adj_kernels(const nedner_plan_s& p) {
    const Chunks& c = p.ch;
    const Geo& G = p.geo;
    const size_t s_xr2c = (size_t)2 * (G.nx / 2) * (c.c5 + 1) * 8;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_img_xr2c_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_xr2c))) return e;
    if ((e = cudaFuncSetAttribute(k_img_yfft_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem4))) return e;
    const int a = cudaFuncAttributeMaxDynamicSharedMemorySize;
#define NEDNER_ATTR_NER(W, D) \
    if ((e = cudaFuncSetAttribute(k_ner_lines_adj<W, D>, (cudaFuncAttribute)a, (int)c.smem3a))) return e;
    NEDNER_ATTR_NER(4, 10) NEDNER_ATTR_NER(6, 10) NEDNER_ATTR_NER(8, 10) NEDNER_ATTR_NER(10, 10)
    NEDNER_ATTR_NER(12, 10) NEDNER_ATTR_NER(14, 12) NEDNER_ATTR_NER(16, 12)
#undef NEDNER_ATTR_NER
    if ((e = cudaFuncSetAttribute(k_ned_yfft_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem2))) return e;
    if ((e = cudaFuncSetAttribute(k_ned_interp_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem_interp))) return e;
    if ((e = cudaFuncSetAttribute(k_ned_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem_grad))) return e;
    return cudaSuccess;
}

cudaError_t launch_img_xr2c_adj(const nedner_plan_s& p, const float* p0, float2* Y, cudaStream_t s) {
    const Geo& G = p.geo;
    const size_t smem = (size_t)2 * (G.nx / 2) * (p.ch.c5 + 1) * 8;
    k_img_xr2c_adj<<<dim3(G.nz, G.ny / p.ch.c5), 256, smem, s>>>(G, p.ch.c5, p0, p.t.tw, Y);
    return cudaGetLastError();
}

cudaError_t launch_img_yfft_adj(const nedner_plan_s& p, const float2* Y, float2* V, cudaStream_t s) {
    const Geo& G = p.geo;
    k_img_yfft_adj<<<dim3(G.nxh, G.nz / p.ch.c4), 256, p.ch.smem4, s>>>(G, p.ch.c4, Y, p.t.tw, V);
    return cudaGetLastError();
}

cudaError_t launch_ner_lines_adj(const nedner_plan_s& p, const float2* V, float2* Ghat, cudaStream_t s) {
    const Geo& G = p.geo;
    const dim3 grid(G.nxh * G.ny);
#define NEDNER_NER(W, D) \
    k_ner_lines_adj<W, D><<<grid, 256, p.ch.smem3a, s>>>(G, p.tap, V, p.t.axy, p.t.deconv_t, p.t.tw, Ghat)
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
    k_ned_yfft_adj<<<dim3(G.nxh, G.Nt / p.ch.c2), 256, p.ch.smem2, s>>>(G, p.ch.c2, Ghat, p.t.deconv_y, p.t.tw, R);
    return cudaGetLastError();
}

cudaError_t launch_ned_interp_adj(const nedner_plan_s& p, const float2* R, float* P, cudaStream_t s) {
    const Geo& G = p.geo;
    if (p.t.ntasks == 0) return cudaSuccess;
    k_ned_interp_adj<<<dim3(p.t.ntasks, G.Nt / p.ch.ca), 256, p.ch.smem_interp, s>>>(
        G, p.ch.ca, p.ch.smax, R, p.t.tasks, p.t.row_ptr, p.t.row_m, p.t.row_w, p.t.row_local, p.t.band_m,
        p.t.band_slot, p.t.sens_bx, p.t.sens_wx, p.t.deconv_x, p.t.tw, P);
    return cudaGetLastError();
}

cudaError_t launch_adj_finish(const nedner_plan_s& p, const float* P, float* g, cudaStream_t s) {
    const Geo& G = p.geo;
    if (G.M == 0) return cudaSuccess;
    const size_t total = (size_t)G.M * G.Nt;
    const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 16);
    k_adj_finish<<<blocks, 256, 0, s>>>(G, P, p.t.two_blocks, g);
    return cudaGetLastError();
}

cudaError_t launch_ned_grad(const nedner_plan_s& p, const float2* R, const float* g, float2* Q, cudaStream_t s) {
    const Geo& G = p.geo;
    if (p.t.ntasks == 0) return cudaSuccess;
    k_ned_grad<<<dim3(p.t.ntasks, G.Nt / p.ch.ca), 256, p.ch.smem_grad, s>>>(
        G, p.ch.ca, p.ch.smax, R, g, p.t.tasks, p.t.row_ptr, p.t.row_m, p.t.row_w, p.t.row_dw, p.t.row_local,
        p.t.band_m, p.t.band_slot, p.t.sens_bx, p.t.sens_wx, p.t.sens_dwx, p.t.deconv_x, p.t.tw, Q);
    return cudaGetLastError();
}

cudaError_t launch_grad_finish(const nedner_plan_s& p, const float2* Q, float* dxy, cudaStream_t s) {
    const Geo& G = p.geo;
    if (G.M == 0) return cudaSuccess;
    k_grad_finish<<<(G.M + 255) / 256, 256, 0, s>>>(G, G.Nt / p.ch.ca, Q, p.t.two_blocks, dxy);
    return cudaGetLastError();
}

}  // namespace nedner

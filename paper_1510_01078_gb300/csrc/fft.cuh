// Batched in-shared-memory FFTs used by every stage of the NEDNER path.
//
// Each call transforms nb columns (nb a power of two) of length N (a power of
// two, 2..8192) that sit in shared memory, point p of column b at linear
// index p * nb + b.  The whole thread block cooperates; the call begins and
// ends with __syncthreads().  The algorithm is the self-sorting (Stockham)
// formulation: log2(N) is covered by radix-16 passes (4 x 4 decomposition in
// registers) plus one radix-2, -4 or -8 pass, so no bit-reversal step is
// needed.
//
//   DIR = -1 : X[k] = sum_p x[p] exp(-2 pi i k p / N)
//   DIR = +1 : X[k] = sum_p x[p] exp(+2 pi i k p / N)     (unnormalised)
//
// Twiddles come from a table computed in FP64 on the host that holds, for
// every power of two N <= TW_N, the N values exp(-2 pi i k / N) contiguously
// at tw[N + k] (so a transform of length N touches N consecutive entries).
#pragma once

#include <cuda_runtime.h>

namespace nedner {

constexpr int TW_N = 8192;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// complex add / subtract as packed FP32x2 operations
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (dir = -1) or +i (dir = +1)
__device__ __forceinline__ float2 mul_i(float2 a, int dir) {
    return dir < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// log2 of a power of two
__device__ __forceinline__ int ilog2(int v) { return 31 - __clz(v); }

// exp(dir * 2 pi i * q / N) for 0 <= q < N
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int q, int N, int dir) {
    float2 t = __ldg(&tw[N + q]);
    return dir < 0 ? t : cconj(t);
}

// ---------------------------------------------------------------------------
// small DFTs in registers
// ---------------------------------------------------------------------------
template <int DIR>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
    const float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <int DIR>
__device__ __forceinline__ void dft4(float2& v0, float2& v1, float2& v2, float2& v3) {
    const float2 a0 = cadd(v0, v2), a1 = csub(v0, v2);
    const float2 a2 = cadd(v1, v3), a3 = mul_i(csub(v1, v3), DIR);
    v0 = cadd(a0, a2);
    v2 = csub(a0, a2);
    v1 = cadd(a1, a3);
    v3 = csub(a1, a3);
}

// dft4 with v1 = v2 = 0 on entry (the same sums without the zero terms)
template <int DIR>
__device__ __forceinline__ void dft4_z12(float2& v0, float2& v1, float2& v2, float2& v3) {
    const float2 x0 = v0;
    const float2 a3 = mul_i(make_float2(-v3.x, -v3.y), DIR);
    v0 = cadd(x0, v3);
    v2 = csub(x0, v3);
    v1 = cadd(x0, a3);
    v3 = csub(x0, a3);
}

// exp(DIR 2 pi i q / 16), q = 0..15, from the exact values of cos/sin at multiples of pi/8
template <int DIR>
__device__ __forceinline__ float2 w16(int q) {
    const float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, h = 0.70710678118654752f;
    float cr, si;
    switch (q & 15) {
        case 0: cr = 1.f; si = 0.f; break;
        case 1: cr = c1; si = s1; break;
        case 2: cr = h; si = h; break;
        case 3: cr = s1; si = c1; break;
        case 4: cr = 0.f; si = 1.f; break;
        case 5: cr = -s1; si = c1; break;
        case 6: cr = -h; si = h; break;
        case 7: cr = -c1; si = s1; break;
        case 8: cr = -1.f; si = 0.f; break;
        case 9: cr = -c1; si = -s1; break;
        case 10: cr = -h; si = -h; break;
        case 11: cr = -s1; si = -c1; break;
        case 12: cr = 0.f; si = -1.f; break;
        case 13: cr = s1; si = -c1; break;
        case 14: cr = h; si = -h; break;
        default: cr = c1; si = -s1; break;
    }
    return make_float2(cr, DIR * si);
}

// DFT of R points in registers; X[k] ends up in v[out_index<R>(k)].
// ZP (R = 16): inputs 4..11 are zero
template <int R, int DIR, bool ZP = false>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
    if constexpr (R == 2) {
        dft2<DIR>(v[0], v[1]);
    } else if constexpr (R == 4) {
        dft4<DIR>(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 8) {
        // n = 4 n1 + n2 (n1 < 2, n2 < 4), k = k1 + 2 k2: 4 DFT2 over n1, twiddle W8^(n2 k1), 2 DFT4 over n2
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) dft2<DIR>(v[n2], v[4 + n2]);
#pragma unroll
        for (int n2 = 1; n2 < 4; ++n2) v[4 + n2] = cmul(v[4 + n2], w16<DIR>(2 * n2));
#pragma unroll
        for (int k1 = 0; k1 < 2; ++k1) dft4<DIR>(v[4 * k1 + 0], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    } else {
        // R = 16: n = 4 n1 + n2, k = k1 + 4 k2: 4 DFT4 over n1, twiddle W16^(n2 k1), 4 DFT4 over n2
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            if constexpr (ZP) dft4_z12<DIR>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
            else dft4<DIR>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
        }
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1)
#pragma unroll
            for (int n2 = 1; n2 < 4; ++n2) v[4 * k1 + n2] = cmul(v[4 * k1 + n2], w16<DIR>(n2 * k1));
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) dft4<DIR>(v[4 * k1 + 0], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    }
}

// position in v of output X[k] after dft_reg
template <int R>
__device__ __forceinline__ constexpr int out_index(int k) {
    return R == 8 ? 4 * (k & 1) + (k >> 1) : R == 16 ? 4 * (k & 3) + (k >> 2) : k;
}

// Complex-to-real inverse transform of length N from the half spectrum
// X[0..N/2] through the half-length complex transform (H = N/2): the input of
// the length-H inverse FFT is Z[k] = E[k] + i O[k], E = X[k] + conj X[H-k],
// O = (X[k] - conj X[H-k]) exp(2 pi i k / N); the imaginary parts of X[0] and
// X[H] are dropped (the real part of the full inverse DFT).  For one pair
// (xk = X[k], xm = X[H-k]), 0 <= k <= H/2, returns zk = Z[k] and
// zm = Z[H-k] = conj E[k] + i conj O[k] (zm is Z[H/2] again when k = H/2 and
// unused when k = 0).  Then z = IFFT_H(Z) holds the real samples as
// x[2p] = Re z[p], x[2p+1] = Im z[p].
__device__ __forceinline__ void c2r_pair(float2 xk, float2 xm, int k, int N, const float2* __restrict__ tw,
                                         float2& zk, float2& zm) {
    if (k == 0) {
        xk.y = 0.f;
        xm.y = 0.f;
    }
    const float2 xmc = cconj(xm);
    const float2 E = cadd(xk, xmc);
    const float2 O = cmul(csub(xk, xmc), twiddle(tw, k, N, +1));
    zk = cadd(E, mul_i(O, +1));
    zm = cadd(cconj(E), mul_i(cconj(O), +1));
}

// Real-to-complex transform of length N through the half-length complex
// transform (H = N/2): with z[p] = x[2p] + i x[2p+1] and Z = FFT_H(z),
// X[k] = E + exp(-2 pi i k / N) O, E = (Z[k] + conj Z[H-k]) / 2,
// O = (Z[k] - conj Z[H-k]) / (2i), indices of Z mod H, for k = 0..H.
// zk = Z[k mod H], zh = Z[(H-k) mod H].
__device__ __forceinline__ float2 r2c_unpack(float2 zk, float2 zh, int k, int N, const float2* __restrict__ tw) {
    const float2 zm = cconj(zh);
    const float2 E = cscale(cadd(zk, zm), 0.5f);
    const float2 O = cscale(mul_i(csub(zk, zm), -1), 0.5f);     // (zk - zm) / (2i)
    return cadd(E, cmul(twiddle(tw, k & (N - 1), N, -1), O));
}

// ---------------------------------------------------------------------------
// In place: every thread keeps its share of a pass in registers, so one
// buffer holds the data throughout; the caller guarantees
// N * nb <= PER * blockDim.x (PER a multiple of 16).  The buffer is padded:
// linear index a = p * nb + b (point p, column b) lives at padx(a), one spare
// slot after every 16 values.  With the radix-16 passes first and the
// remaining radix-2/4/8 pass last, the 16 lanes of a half-warp then touch 16
// distinct 8-byte bank pairs on every load and store, for every nb.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int padx(int a) { return a + (a >> 4); }
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> 4); }

// ZP (first radix-16 pass only): points N/4 <= p < 3N/4 are zero and are
// not read, i.e. the input is x zero-padded to twice its length and centred
// (its first half at p < N/4, its second half at p >= 3N/4).
template <int R, int DIR, int PER, bool ZP = false>
__device__ __forceinline__ void fft_pass_ip(float2* buf, int N, int Ns, int nb, const float2* __restrict__ tw) {
    constexpr int IT = PER / R;
    const int stride = N / R;
    const int lnb = ilog2(nb);
    const int items = stride << lnb;
    const int step = N / (Ns * R);
    // Linear distance between the R loads (stride nb) and the R stores (Ns nb)
    // of an item; once it is a multiple of 16 the padded distance is constant,
    // so the addresses advance by one add each.
    const int lld = stride << lnb, lst = Ns << lnb;
    const int dld = lld + (lld >> 4), dst = lst + (lst >> 4);
    float2 v[IT][R];
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int it = threadIdx.x + i * blockDim.x;
        if (it < items) {
            const int j = it >> lnb, b = it & (nb - 1);
            const int a0 = (j << lnb) + b;
            constexpr bool zp = ZP && R == 16;
            if (lld >= 16) {
                const float2* p = buf + padx(a0);
#pragma unroll
                for (int r = 0; r < R; ++r, p += dld) v[i][r] = (zp && r >= 4 && r < 12) ? make_float2(0.f, 0.f) : *p;
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    v[i][r] = (zp && r >= 4 && r < 12) ? make_float2(0.f, 0.f) : buf[padx(a0 + r * lld)];
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int it = threadIdx.x + i * blockDim.x;
        if (it < items) {
            const int j = it >> lnb, b = it & (nb - 1);
            const int k = j & (Ns - 1);
            if (Ns > 1) {
                if (R == 16 && nb < 4) {
                    // few columns: neighbouring lanes need different twiddles, so
                    // the 15 table loads would touch up to 15 x 32 distinct lines;
                    // load w^k and w^4k (w = exp(DIR 2 pi i step / N)) and form
                    // w^(r1 + 4 r2) = (w^k)^r1 (w^4k)^r2 with at most two products
                    // per factor (a few units in the last place)
                    const float2 a1 = twiddle(tw, k * step, N, DIR);
                    const float2 b1 = twiddle(tw, 4 * k * step, N, DIR);
                    const float2 a2 = cmul(a1, a1), a3 = cmul(a2, a1);
                    const float2 b2 = cmul(b1, b1), b3 = cmul(b2, b1);
                    const float2 wa[4] = {make_float2(1.f, 0.f), a1, a2, a3};
                    const float2 wb[4] = {make_float2(1.f, 0.f), b1, b2, b3};
#pragma unroll
                    for (int r = 1; r < R; ++r) {
                        const int r1 = r & 3, r2 = r >> 2;
                        const float2 t = (r1 == 0) ? wb[r2] : (r2 == 0) ? wa[r1] : cmul(wa[r1], wb[r2]);
                        v[i][r] = cmul(v[i][r], t);
                    }
                } else {
                    const float2* tp = tw + N;
                    const int ks = k * step;
                    int q = 0;
#pragma unroll
                    for (int r = 1; r < R; ++r) {
                        q += ks;
                        const float2 t = __ldg(tp + q);
                        v[i][r] = cmul(v[i][r], DIR < 0 ? t : cconj(t));
                    }
                }
            }
            dft_reg<R, DIR, ZP && R == 16>(v[i]);
            const int a0 = (((j - k) * R + k) << lnb) + b;
            if (lst >= 16) {
                float2* p = buf + padx(a0);
#pragma unroll
                for (int r = 0; r < R; ++r, p += dst) *p = v[i][out_index<R>(r)];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) buf[padx(a0 + r * lst)] = v[i][out_index<R>(r)];
            }
        }
    }
    __syncthreads();
}

template <int PER, int DIR, bool ZP>
__device__ __forceinline__ void block_fft_ip_dir(float2* buf, int N, int nb, const float2* __restrict__ tw,
                                                 bool skip_r2) {
    __syncthreads();
    int Ns = 1;
    int rem = ilog2(N);
    if constexpr (ZP) {
        fft_pass_ip<16, DIR, PER, true>(buf, N, Ns, nb, tw);
        rem -= 4;
        Ns <<= 4;
    }
    for (; rem >= 4; rem -= 4, Ns <<= 4) fft_pass_ip<16, DIR, PER>(buf, N, Ns, nb, tw);
    if (rem == 3) fft_pass_ip<8, DIR, PER>(buf, N, Ns, nb, tw);
    else if (rem == 2) fft_pass_ip<4, DIR, PER>(buf, N, Ns, nb, tw);
    else if (rem == 1 && !skip_r2) fft_pass_ip<2, DIR, PER>(buf, N, Ns, nb, tw);
}

// In-place transform of nb columns of length N in a padded buffer.  With
// skip_r2, a final radix-2 pass (log2 N = 1 mod 4) is left to the caller:
// the buffer then holds s with X[k] = s[k] + w^k s[k + N/2] and
// X[k + N/2] = s[k] - w^k s[k + N/2], w = exp(DIR 2 pi i / N).  With ZP
// (N >= 16) the input is zero at N/4 <= p < 3N/4 and those points are never
// read, so the caller need not write them.
template <int PER, bool ZP = false>
__device__ __forceinline__ void block_fft_ip(float2* buf, int N, int nb, int dir, const float2* __restrict__ tw,
                                             bool skip_r2 = false) {
    if (dir < 0) block_fft_ip_dir<PER, -1, ZP>(buf, N, nb, tw, skip_r2);
    else block_fft_ip_dir<PER, +1, ZP>(buf, N, nb, tw, skip_r2);
}

}  // namespace nedner

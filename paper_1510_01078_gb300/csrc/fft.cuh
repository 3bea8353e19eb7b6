// Batched in-shared-memory FFTs used by every stage of the NEDNER path.
//
// Each call transforms nb columns of length N (a power of two, 2..8192) that
// sit in shared memory as buf[p * ld + b] (point p, column b).  The whole
// thread block cooperates; the call begins and ends with __syncthreads().
// The algorithm is the self-sorting (Stockham) formulation: log2(N) is
// covered by radix-4 passes plus at most one radix-2 pass, each pass reading
// one buffer and writing the other, so no bit-reversal step is needed.
//
//   dir = -1 : X[k] = sum_p x[p] exp(-2 pi i k p / N)
//   dir = +1 : X[k] = sum_p x[p] exp(+2 pi i k p / N)     (unnormalised)
//
// Twiddles come from a table tw[i] = exp(-2 pi i i / TW_N) computed in FP64
// on the host (TW_N a power of two >= N).
#pragma once

#include <cuda_runtime.h>

namespace nedner {

constexpr int TW_N = 8192;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (dir = -1) or +i (dir = +1)
__device__ __forceinline__ float2 mul_i(float2 a, int dir) {
    return dir < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// exp(dir * 2 pi i * q / N) for 0 <= q < N
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int q, int N, int dir) {
    float2 t = __ldg(&tw[q * (TW_N / N)]);
    return dir < 0 ? t : cconj(t);
}

// One Stockham pass of radix R over all columns: src -> dst.
template <int R>
__device__ __forceinline__ void fft_pass(const float2* __restrict__ src, float2* __restrict__ dst, int N,
                                         int Ns, int nb, int ld, int dir, const float2* __restrict__ tw) {
    const int stride = N / R;
    const int items = stride * nb;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int j = it / nb;
        const int b = it - j * nb;
        const int k = j & (Ns - 1);
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[(j + r * stride) * ld + b];
        if (Ns > 1) {
            const int step = N / (Ns * R);
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], twiddle(tw, k * r * step, N, dir));
        }
        if (R == 2) {
            float2 a = v[0], c = v[1];
            v[0] = cadd(a, c);
            v[1] = csub(a, c);
        } else {
            float2 a0 = cadd(v[0], v[2]);
            float2 a1 = csub(v[0], v[2]);
            float2 a2 = cadd(v[1], v[3]);
            float2 a3 = mul_i(csub(v[1], v[3]), dir);
            v[0] = cadd(a0, a2);
            v[2] = csub(a0, a2);
            v[1] = cadd(a1, a3);
            v[3] = csub(a1, a3);
        }
        const int i0 = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[(i0 + r * Ns) * ld + b] = v[r];
    }
}

// Transform; returns the buffer (a or b) that holds the result.
__device__ __forceinline__ float2* block_fft(float2* a, float2* b, int N, int nb, int ld, int dir,
                                             const float2* __restrict__ tw) {
    __syncthreads();
    float2* src = a;
    float2* dst = b;
    int Ns = 1;
    int logN = 31 - __clz(N);
    if (logN & 1) {
        fft_pass<2>(src, dst, N, Ns, nb, ld, dir, tw);
        Ns = 2;
        __syncthreads();
        float2* t = src; src = dst; dst = t;
    }
    while (Ns < N) {
        fft_pass<4>(src, dst, N, Ns, nb, ld, dir, tw);
        Ns *= 4;
        __syncthreads();
        float2* t = src; src = dst; dst = t;
    }
    return src;
}

}  // namespace nedner

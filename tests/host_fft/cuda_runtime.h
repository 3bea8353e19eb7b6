// Host stand-in for the few CUDA names that the in-shared-memory FFT header,
// the register-window headers and the NER evaluation header use, so that
// those headers compile with g++ and run on CPU threads (one std::thread per CUDA thread,
// __syncthreads as a std::barrier).  Test infrastructure only.
#pragma once
#include <cmath>

struct float2 {
    float x, y;
};
struct float4 {
    float x, y, z, w;
};
struct int2 {
    int x, y;
};
struct int4 {
    int x, y, z, w;
};
inline float2 make_float2(float x, float y) { return float2{x, y}; }
inline float4 make_float4(float x, float y, float z, float w) { return float4{x, y, z, w}; }

// opaque handles and status of the runtime API (declarations only)
typedef struct HostStream* cudaStream_t;
typedef struct HostEvent* cudaEvent_t;
typedef int cudaError_t;

struct HostDim3 {
    unsigned x = 0, y = 0, z = 0;
};
extern thread_local HostDim3 threadIdx;
extern HostDim3 blockDim;
void __syncthreads();

#define __device__
#define __host__
#define __forceinline__ inline
#define __restrict__ __restrict

template <class T>
inline T __ldg(const T* p) { return *p; }
// one packed FP32x2 add: two independent round-to-nearest adds
inline float2 __fadd2_rn(float2 a, float2 b) { return float2{a.x + b.x, a.y + b.y}; }
// one packed FP32x2 fused multiply-add: two independent fmaf
inline float2 __ffma2_rn(float2 a, float2 b, float2 c) {
    return float2{std::fmaf(a.x, b.x, c.x), std::fmaf(a.y, b.y, c.y)};
}
inline int __clz(int v) { return __builtin_clz((unsigned)v); }
// sin(pi x) and cos(pi x), through double precision
inline void sincospif(float x, float* s, float* c) {
    const double a = 3.14159265358979323846 * (double)x;
    *s = (float)std::sin(a);
    *c = (float)std::cos(a);
}

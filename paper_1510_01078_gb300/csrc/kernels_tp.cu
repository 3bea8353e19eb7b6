// Tensor-product NED stage on the tcgen05 tensor cores.
//
// When the sensors form a tensor product x_m = xs[a], y_m = ys[b]
// (m = b * nxs + a), the NED sum of Eq. disc_rec factorises (Eq. NUDFT2 with a
// separable exponent):
//   G[jx, jy, n] = sum_b Ey[jy, b] sum_a Ex[jx, a] A[b, a, n],
//   Ex[jx, a] = exp(-2 pi i jx xs[a] / X), Ey[jy, b] = exp(-2 pi i jy ys[b] / Y),
//   A[b, a, n] = w_m g[m, n],
// i.e. two dense complex contractions, evaluated exactly (no window, no
// oversampled grid) on the tensor cores:
//   GEMM 1 (per n):       D[jx, b] = sum_a Ex[jx, a] A[b, a, n]     M = jx, N = b, K = a
//   GEMM 2 (per jx):      G[jy, n] = sum_b D[jx, b, n] Ey[jy, b]    M = n, N = jy, K = b
// GEMM 2 takes n as its M dimension so that every output column jy is a run
// of contiguous time samples of Ghat.  Operands are BF16 or FP16 (the two
// precision modes) with a hi + lo split of every real factor (x = hi + lo,
// hi = round(x), lo = round(x - hi)); each real product is formed as
// hi*hi + lo*hi + hi*lo with FP32 accumulation in tensor memory.  FP16 keeps
// 11 significant bits per part against BF16's 8 but has a narrow exponent
// range, so in FP16 mode the data are first scaled by a power of two s (from
// the largest |w_m g[m, n]|, k_tp_absmax) that puts them in [2^7, 2^8) at most,
// which keeps D = sum_a Ex A below 2^15; the epilogues multiply by 1/s.  Shapes handled: nxs = nys = 128 sensors per axis, nx = ny = 256
// output grid: jx = 0..127 as GEMM tiles of 128 rows, jy in two M tiles
// (-128..-1 and 0..127); the row jy = +128 is summed in FP32 in GEMM 1's
// epilogue and the line jx = 128 on the CUDA cores (k_tp_prep, k_tp_nyq_g).
//
// Operand tiles live in global memory already in the tensor cores'
// K-major, unswizzled shared-memory layout, split in K chunks of 64 so that
// every operand block is contiguous and moved by a single bulk copy
// (cp.async.bulk, completion on an mbarrier).  Within a chunk of a matrix
// with `rows` rows, element (row r, k) is at
// ((r/8) * 8 + k/8) * 64 + (r%8) * 8 + k%8 (core matrices of 8 rows x 16
// bytes; 128 bytes between core matrices along K, 1024 bytes between 8-row
// groups).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace nedner {
namespace tp {

constexpr int K = 128;                 // contraction length (sensors per axis)
constexpr int KC = 64;                 // K chunk
constexpr int ROWS = 128;              // M and N of the main tiles
constexpr uint32_t CHUNK = ROWS * KC * 2;          // 16 KB per (128-row matrix, chunk)
constexpr uint32_t MAT = ROWS * K * 2;             // 32 KB per 128-row matrix
constexpr int TM = 128;                             // time samples per GEMM 2 tile (its M)
constexpr int KA = 32;                              // K chunk of the GEMM 2 D tiles
constexpr uint32_t DT_BLK = TM * KA * 2;            // 8 KB: one matrix of a D tile, one K chunk
constexpr uint32_t DT_STAGE = 4 * DT_BLK;           // Re hi, Re lo, Im hi, Im lo of one K chunk
constexpr int STAGES = 3;                           // operand ring of both GEMMs
constexpr int WAIT_LIMIT = TP_WAIT_LIMIT;   // polls of a bounded mbarrier wait (drains; pipeline default)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// element offset of (r, k) inside a chunked K-major matrix with `rows` rows
__device__ __forceinline__ int tile_off(int r, int k, int rows) {
    const int c = k >> 6, kk = k & 63;
    return c * rows * KC + (((r >> 3) * (KC >> 3) + (kk >> 3)) << 6) + ((r & 7) << 3) + (kk & 7);
}

// shared-memory matrix descriptor: K-major, no swizzle, LBO 128 B (along K), SBO between 8-row groups
__device__ __forceinline__ uint64_t sdesc_sbo(uint32_t saddr, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// the same for K chunks of 64 (8-row groups 1024 B apart)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) { return sdesc_sbo(saddr, 1024); }

// instruction descriptor: kind::f16, D = F32, A = B = BF16 (ab = 1) or FP16
// (ab = 0), both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_f16kind(int n, uint32_t ab) {
    return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// the two operand types: the A/B type field of the instruction descriptor and
// the hi + lo split of an FP32 value
template <typename T> struct Op;
template <> struct Op<__nv_bfloat16> {
    static constexpr uint32_t ab = 1;
    static __device__ __forceinline__ void split(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
        hi = __float2bfloat16_rn(x);
        lo = __float2bfloat16_rn(x - __bfloat162float(hi));
    }
};
template <> struct Op<__half> {
    static constexpr uint32_t ab = 0;
    static __device__ __forceinline__ void split(float x, __half& hi, __half& lo) {
        hi = __float2half_rn(x);
        lo = __float2half_rn(x - __half2float(hi));
    }
};

// data scale of the FP16 mode from the largest |w_m g[m, n]| (its bits in
// *absmax): s = 2^(8 - e) with max in [2^(e-1), 2^e), so that s max < 2^8; 1
// when absmax is null (BF16 mode), zero or not finite
__device__ __forceinline__ float data_scale(const unsigned int* absmax) {
    if (!absmax) return 1.f;
    const float mx = __uint_as_float(*absmax);
    if (!(mx > 0.f) || !isfinite(mx)) return 1.f;
    int e = 0;
    frexpf(mx, &e);
    return ldexpf(1.f, min(120, max(-120, 8 - e)));
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void bar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// bounded wait for the phase of parity `parity` (at most `limit` polls);
// false if it did not complete
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, int limit = WAIT_LIMIT) {
    uint32_t done = 0;
    for (int it = 0; it < limit && !done; ++it) {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(smem_u32(bar)), "r"(parity)
                     : "memory");
    }
    return done != 0;
}

// the producer's drain before tensor memory and shared memory are released:
// waits (long limit) for the copies of the last min(STAGES, last + 1) ring
// slots it filled, u = last - STAGES + 1 .. last.  Each of those slots has
// not been refilled since (the producer refills a slot only after the
// consumer frees it), so its barrier completes exactly that phase.
__device__ __forceinline__ void drain_ring(uint64_t* full, int last) {
    for (int u = last; u >= 0 && u > last - STAGES; --u) bar_wait(&full[u % STAGES], (u / STAGES) & 1);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------------------
// FP16 mode: *absmax = bits of max |w_m g[m][n]| (non-negative floats order
// as their bit patterns); *absmax is zeroed before the launch
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tp_absmax(const Geo G, const float* __restrict__ g,
                                                   const float* __restrict__ fac, unsigned int* __restrict__ absmax) {
    const size_t n4 = (size_t)G.M * G.Nt / 4;
    const int lnt4 = __ffs(G.Nt / 4) - 1;                 // Nt / 4 is a power of two
    float mx = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(g) + i);
        const float f = fabsf(__ldg(&fac[i >> lnt4]));
        mx = fmaxf(mx, f * fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(absmax, __float_as_uint(mx));
}

// ---------------------------------------------------------------------------
// prep: A[b][a][n] = s w_m g[m][n] -> per n, matrices (hi, lo) with rows b, K = a
// (256 threads; CTA = 16 time samples x 4 rows b)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_tp_prep(const Geo G, const float* __restrict__ g,
                                                 const float* __restrict__ fac, const float2* __restrict__ exn,
                                                 T* __restrict__ At, float2* __restrict__ t, int nb, int ne,
                                                 const unsigned int* __restrict__ absmax) {
    __shared__ float tile[4 * K][17];
    const float sc = data_scale(absmax);
    const int n0 = nb + blockIdx.x * 16;
    const int b0 = blockIdx.y * 4;
    for (int i = threadIdx.x; i < 4 * K * 16; i += blockDim.x) {
        const int r = i >> 4, c = i & 15;                   // r = (b - b0) * K + a
        const int m = (b0 + (r >> 7)) * K + (r & 127);
        tile[r][c] = (n0 + c < ne) ? fac[m] * g[(size_t)m * G.Nt + n0 + c] : 0.f;
    }
    __syncthreads();
    // items: 16 n x 4 b x 16 groups of 8 a
    for (int it = threadIdx.x; it < 16 * 4 * 16; it += blockDim.x) {
        const int c = it >> 6, rb = (it >> 4) & 3, ag = it & 15;
        const int n = n0 + c;
        if (n >= ne) continue;
        __align__(16) T hi[8], lo[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) Op<T>::split(sc * tile[rb * K + ag * 8 + j][c], hi[j], lo[j]);
        const int off = tile_off(b0 + rb, ag * 8, ROWS);
        T* base = At + (size_t)(n - nb) * 2 * (ROWS * K);
        *reinterpret_cast<uint4*>(base + off) = *reinterpret_cast<uint4*>(hi);
        *reinterpret_cast<uint4*>(base + ROWS * K + off) = *reinterpret_cast<uint4*>(lo);
    }
    // the line jx = nx/2 (CUDA cores, FP32): t[b][n] = sum_a Ex[nx/2, a] A[b, a, n]
    if (threadIdx.x < 64) {
        const int c = threadIdx.x & 15, rb = threadIdx.x >> 4;
        const int n = n0 + c;
        float2 sacc = make_float2(0.f, 0.f);
#pragma unroll 8
        for (int a = 0; a < K; ++a) {
            const float v = tile[rb * K + a][c];
            const float2 e = __ldg(&exn[a]);
            sacc.x = fmaf(e.x, v, sacc.x);
            sacc.y = fmaf(e.y, v, sacc.y);
        }
        if (n < ne) t[(size_t)(b0 + rb) * G.Nt + n] = sacc;
    }
}

// ---------------------------------------------------------------------------
// GEMM 1: persistent and warp-specialised.  Ex (Re hi, Re lo, Im hi, Im lo;
// rows jx = 0..127, K = a; 128 KB) stays in shared memory.  Warp 0 streams
// each time sample's A (hi, lo; rows b) in K chunks of 64 (32 KB) through a
// ring of STAGES buffers; warp 1 issues 6 MMAs (M 128, N 128) per K step of
// 16 into one of two accumulator pairs (D_re, D_im; 256 columns each) in
// tensor memory; warps 2-9 read a pair back (lane quarter = warp % 4, row
// jx; warps 2-5 take b = 0..63, warps 6-9 b = 64..127) and write D as BF16
// hi/lo into the GEMM 2 operand tiles (per jx and tile of 128 time samples:
// rows n, K = b, in K chunks of 32).  Warps 2-5 also sum the row jy = +ny/2 of G in FP32:
//   G[jx, +ny/2, n] = sum_b Ey[+ny/2, b] D[jx, b].
// Waits are bounded as in GEMM 2.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(320, 1) k_tp_gemm1(const Geo G, const T* __restrict__ Ex,
                                                     const T* __restrict__ At,
                                                     const float2* __restrict__ eyf,
                                                     T* __restrict__ Dt, float2* __restrict__ Ghat,
                                                     int* __restrict__ err, int nb, int ne,
                                                     const unsigned int* __restrict__ absmax, int wl) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sEx = smem;                                  // 4 x 32 KB
    unsigned char* sA = smem + 4 * MAT;                         // STAGES x (hi, lo) chunks of 16 KB
    __shared__ __align__(8) uint64_t ex_bar, full[STAGES], empty[STAGES], tfull[2], tempty[2], done_bar;
    __shared__ uint32_t taddr_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        bar_init(&ex_bar, 1);
        for (int s = 0; s < STAGES; ++s) {
            bar_init(&full[s], 1);
            bar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            bar_init(&tfull[a], 1);
            bar_init(&tempty[a], 8);
        }
        bar_init(&done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&taddr_s)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tacc = taddr_s;                              // pair a: Re at 256 a, Im at 256 a + 128

    if (warp == 0) {
        if (lane == 0) {
            expect_tx(&ex_bar, 4 * MAT);
            for (int q = 0; q < 4; ++q) bulk_load(sEx + q * MAT, Ex + (size_t)q * (MAT / 2), MAT, &ex_bar);
            int u = 0, last = -1;
            bool ok = true;
            for (int n = nb + blockIdx.x; n < ne && ok; n += gridDim.x) {
                const T* an = At + (size_t)(n - nb) * 2 * (ROWS * K);
                for (int c = 0; c < 2; ++c, ++u) {
                    const int s = u % STAGES;
                    if (!bar_wait(&empty[s], ((u / STAGES) & 1) ^ 1, wl)) {
                        atomicExch(err, 1);
                        ok = false;
                        break;
                    }
                    expect_tx(&full[s], 2 * CHUNK);
                    bulk_load(sA + s * 2 * CHUNK, an + c * (ROWS * KC), CHUNK, &full[s]);
                    bulk_load(sA + s * 2 * CHUNK + CHUNK, an + ROWS * K + c * (ROWS * KC), CHUNK, &full[s]);
                    last = u;
                }
            }
            drain_ring(full, last);
            bar_wait(&ex_bar, 0);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = bar_wait(&ex_bar, 0, wl);
            const uint32_t id = idesc_f16kind(128, Op<T>::ab);
            const uint64_t x0 = sdesc(smem_u32(sEx)), x1 = x0 + (MAT >> 4), x2 = x0 + 2 * (MAT >> 4),
                           x3 = x0 + 3 * (MAT >> 4);
            const uint64_t abase = sdesc(smem_u32(sA));
            int q = 0, u = 0;
            for (int n = nb + blockIdx.x; n < ne && ok; n += gridDim.x, ++q) {
                const int a = q & 1;
                if (!bar_wait(&tempty[a], ((q >> 1) & 1) ^ 1, wl)) {
                    ok = false;
                    break;
                }
                const uint32_t tre = tacc + 256 * a, tim = tre + 128;
                for (int c = 0; c < 2; ++c, ++u) {
                    const int s = u % STAGES;
                    if (!bar_wait(&full[s], (u / STAGES) & 1, wl)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t ah = abase + (uint64_t)((s * 2 * CHUNK) >> 4), al = ah + (CHUNK >> 4);
#pragma unroll
                    for (int k = 0; k < KC / 16; ++k) {
                        const uint64_t ox = (c * CHUNK + k * 256) >> 4, oa = (k * 256) >> 4;
                        const uint32_t acc = (c | k) ? 1u : 0u;
                        mma(tre, x0 + ox, ah + oa, id, acc);
                        mma(tre, x1 + ox, ah + oa, id, 1u);
                        mma(tre, x0 + ox, al + oa, id, 1u);
                        mma(tim, x2 + ox, ah + oa, id, acc);
                        mma(tim, x3 + ox, ah + oa, id, 1u);
                        mma(tim, x2 + ox, al + oa, id, 1u);
                    }
                    mma_commit(&empty[s]);
                }
                if (!ok) break;
                mma_commit(&tfull[a]);
            }
            if (!ok) atomicExch(err, 1);
            mma_commit(&done_bar);
            bar_wait(&done_bar, 0);
        }
    } else {
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        const int jx = quarter * 32 + lane;
        const int ntn = (ne - nb) / TM;
        const float2* eyp = eyf + (size_t)G.ny * K;             // Ey row jy = +ny/2
        const float inv = 1.f / data_scale(absmax);             // a power of two: exact
        int q = 0;
        for (int n = nb + blockIdx.x; n < ne; n += gridDim.x, ++q) {
            const int a = q & 1;
            if (!__all_sync(0xffffffffu, bar_wait(&tfull[a], (q >> 1) & 1, wl))) {
                if (lane == 0) atomicExch(err, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t trow = tacc + ((uint32_t)(quarter * 32) << 16) + 256 * a;
            const int nr = (n - nb) % TM;
            T* out = Dt + ((size_t)jx * ntn + (n - nb) / TM) * (4 * DT_STAGE / 2);
            float gr = 0.f, gi = 0.f;
            for (int c0 = 0; c0 < 128; c0 += 32) {
                const bool mine = (c0 >> 6) == half;
                if (!mine && half == 1) continue;               // warps 6-9: their own 64 columns only
                uint32_t vr[32], vi[32];
                tmem_ld32(trow + c0, vr);
                tmem_ld32(trow + 128 + c0, vi);
                if (half == 0) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float dr = __uint_as_float(vr[j]), di = __uint_as_float(vi[j]);
                        const float2 e = __ldg(&eyp[c0 + j]);
                        gr = fmaf(e.x, dr, fmaf(-e.y, di, gr));
                        gi = fmaf(e.x, di, fmaf(e.y, dr, gi));
                    }
                }
                if (!mine) continue;
#pragma unroll
                for (int g8 = 0; g8 < 4; ++g8) {
                    __align__(16) T rh[8], rl[8], ih[8], il[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        Op<T>::split(__uint_as_float(vr[g8 * 8 + j]), rh[j], rl[j]);
                        Op<T>::split(__uint_as_float(vi[g8 * 8 + j]), ih[j], il[j]);
                    }
                    {
                        // (row n, b) in K chunk b / 32: ((n / 8) * 4 + (b % 32) / 8) * 64 + (n % 8) * 8 + b % 8
                        const int bb = c0 + g8 * 8;
                        const int off = (bb >> 5) * (DT_STAGE / 2) + (((nr >> 3) * 4 + ((bb & 31) >> 3)) << 6) +
                                        ((nr & 7) << 3);
                        *reinterpret_cast<uint4*>(out + off + 0 * (DT_BLK / 2)) = *reinterpret_cast<uint4*>(rh);
                        *reinterpret_cast<uint4*>(out + off + 1 * (DT_BLK / 2)) = *reinterpret_cast<uint4*>(rl);
                        *reinterpret_cast<uint4*>(out + off + 2 * (DT_BLK / 2)) = *reinterpret_cast<uint4*>(ih);
                        *reinterpret_cast<uint4*>(out + off + 3 * (DT_BLK / 2)) = *reinterpret_cast<uint4*>(il);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) bar_arrive(&tempty[a]);
            if (half == 0) Ghat[((size_t)jx * G.nyp + G.ny) * G.Nt + n] = make_float2(gr * inv, gi * inv);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tacc), "r"(512));
}

// ---------------------------------------------------------------------------
// GEMM 2: persistent and warp-specialised, with the time samples as M:
//   G[jy, n] = sum_b D[jx, b, n] Ey[jy, b]   as   C[n, jy] = sum_b A[n, b] B[jy, b],
// A = the D tile of (jx, 128 time samples), B = Ey, so that each MMA is
// M 128 x N 128 x K 16 (a narrower N spends more shared-memory bandwidth on
// re-reading the operands than on arithmetic) and each output column jy is
// a run of contiguous time samples of Ghat.  A CTA owns one tile of jy
// (blockIdx.x even: jy = -128..-1, odd: 0..127) and keeps that tile of Ey
// (Re hi, Re lo, Im hi, Im lo; rows jy, K = b; 128 KB) in shared memory; it
// loops over work items (jx, n tile) shared out among the CTAs of its tile.
// Warp 0 streams each item's D tile in four K chunks of 32 (32 KB each, the
// four matrices of a chunk contiguous) through a ring of STAGES buffers;
// warp 1 issues 12 MMAs per K step of 16:
//   G_re = D_re Ey_re - D_im Ey_im,  G_im = D_re Ey_im + D_im Ey_re
// (the minus by the instruction's negate-A bit) into one of two accumulator
// pairs in tensor memory (256 columns each); warps 2-5 read a pair back
// (lane quarter = warp % 4 = time sample) and write, for every jy, 32
// consecutive time samples per warp store.  Every wait is bounded: a wait
// that runs out sets *err and the role stops; the others then run out too,
// and the CTA waits for its own copies and MMAs in flight before it frees
// tensor memory.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(192, 1) k_tp_gemm2(const Geo G, const T* __restrict__ Dt,
                                                     const T* __restrict__ Ey,
                                                     float2* __restrict__ Ghat, int* __restrict__ err, int nb,
                                                     int ne, const unsigned int* __restrict__ absmax, int wl) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sEy = smem;                                  // 4 x 32 KB
    unsigned char* sD = smem + 4 * MAT;                         // STAGES x 32 KB
    __shared__ __align__(8) uint64_t ey_bar, full[STAGES], empty[STAGES], tfull[2], tempty[2], done_bar;
    __shared__ uint32_t taddr_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x & 1;
    const int slot = blockIdx.x >> 1, nslots = gridDim.x >> 1;
    const int ntn = (ne - nb) / TM;
    const int items = K * ntn;                                  // jx = 0..127 x n tiles of [nb, ne)

    if (tid == 0) {
        bar_init(&ey_bar, 1);
        for (int s = 0; s < STAGES; ++s) {
            bar_init(&full[s], 1);
            bar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            bar_init(&tfull[a], 1);
            bar_init(&tempty[a], 4);
        }
        bar_init(&done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&taddr_s)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tacc = taddr_s;                              // pair a: Re at 256 a, Im at 256 a + 128

    if (warp == 0) {
        if (lane == 0) {
            expect_tx(&ey_bar, 4 * MAT);
            for (int q = 0; q < 4; ++q)
                bulk_load(sEy + q * MAT, Ey + (size_t)(tile * 4 + q) * (MAT / 2), MAT, &ey_bar);
            int u = 0, last = -1;
            bool ok = true;
            for (int it = slot; it < items && ok; it += nslots) {
                const T* src = Dt + (size_t)it * (4 * DT_STAGE / 2);   // item = jx * ntn + nt
                for (int c = 0; c < 4; ++c, ++u) {
                    const int s = u % STAGES;
                    if (!bar_wait(&empty[s], ((u / STAGES) & 1) ^ 1, wl)) {
                        atomicExch(err, 1);
                        ok = false;
                        break;
                    }
                    expect_tx(&full[s], DT_STAGE);
                    bulk_load(sD + s * DT_STAGE, src + c * (DT_STAGE / 2), DT_STAGE, &full[s]);
                    last = u;
                }
            }
            drain_ring(full, last);
            bar_wait(&ey_bar, 0);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = bar_wait(&ey_bar, 0, wl);
            const uint32_t id = idesc_f16kind(128, Op<T>::ab), idn = id | (1u << 13);    // M = N = 128; negate A
            // descriptors of the operand bases; a K step adds its byte offset / 16
            // to the start-address field (no carry: shared addresses < 2^18)
            const uint64_t e0 = sdesc(smem_u32(sEy)), e1 = e0 + (MAT >> 4), e2 = e0 + 2 * (MAT >> 4),
                           e3 = e0 + 3 * (MAT >> 4);
            const uint64_t dbase = sdesc_sbo(smem_u32(sD), 512);
            int q = 0, u = 0;
            for (int it = slot; it < items && ok; it += nslots, ++q) {
                const int a = q & 1;
                if (!bar_wait(&tempty[a], ((q >> 1) & 1) ^ 1, wl)) {
                    ok = false;
                    break;
                }
                const uint32_t tre = tacc + 256 * a, tim = tre + 128;
                for (int c = 0; c < 4; ++c, ++u) {
                    const int s = u % STAGES;
                    if (!bar_wait(&full[s], (u / STAGES) & 1, wl)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t d0 = dbase + (uint64_t)((s * DT_STAGE) >> 4);
#pragma unroll
                    for (int k = 0; k < KA / 16; ++k) {
                        const int b0 = c * KA + k * 16;                         // first b of the K step
                        const uint64_t oe = (uint64_t)(((b0 >> 6) * CHUNK + (b0 & 63) * 16) >> 4);
                        const uint64_t od = (uint64_t)((k * 256) >> 4);
                        const uint64_t drh = d0 + od, drl = d0 + (DT_BLK >> 4) + od;
                        const uint64_t dih = d0 + 2 * (DT_BLK >> 4) + od, dil = d0 + 3 * (DT_BLK >> 4) + od;
                        const uint64_t erh = e0 + oe, erl = e1 + oe, eih = e2 + oe, eil = e3 + oe;
                        const uint32_t acc = (c | k) ? 1u : 0u;
                        mma(tre, drh, erh, id, acc);
                        mma(tre, drl, erh, id, 1u);
                        mma(tre, drh, erl, id, 1u);
                        mma(tre, dih, eih, idn, 1u);
                        mma(tre, dil, eih, idn, 1u);
                        mma(tre, dih, eil, idn, 1u);
                        mma(tim, drh, eih, id, acc);
                        mma(tim, drl, eih, id, 1u);
                        mma(tim, drh, eil, id, 1u);
                        mma(tim, dih, erh, id, 1u);
                        mma(tim, dil, erh, id, 1u);
                        mma(tim, dih, erl, id, 1u);
                    }
                    mma_commit(&empty[s]);
                }
                if (!ok) break;
                mma_commit(&tfull[a]);
            }
            if (!ok) atomicExch(err, 1);
            // every MMA issued has completed before tensor memory is freed
            mma_commit(&done_bar);
            bar_wait(&done_bar, 0);
        }
    } else {
        const int quarter = warp & 3;                           // TMEM lanes 32 quarter .. + 31
        const int row = quarter * 32 + lane;                    // time sample within the tile
        const float inv = 1.f / data_scale(absmax);             // a power of two: exact
        int q = 0;
        for (int it = slot; it < items; it += nslots, ++q) {
            const int a = q & 1;
            if (!__all_sync(0xffffffffu, bar_wait(&tfull[a], (q >> 1) & 1, wl))) {
                if (lane == 0) atomicExch(err, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int jx = it / ntn, nt = it - jx * ntn;
            float2* o = Ghat + ((size_t)jx * G.nyp + tile * K) * G.Nt + nb + nt * TM + row;   // column jy: + jy * Nt
            const uint32_t ta = tacc + ((uint32_t)(quarter * 32) << 16) + 256 * a;
            for (int j0 = 0; j0 < 128; j0 += 32) {
                uint32_t vr[32], vi[32];
                tmem_ld32(ta + j0, vr);
                tmem_ld32(ta + 128 + j0, vi);
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    o[(size_t)(j0 + j) * G.Nt] = make_float2(__uint_as_float(vr[j]) * inv, __uint_as_float(vi[j]) * inv);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) bar_arrive(&tempty[a]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tacc), "r"(512));
}

// ---------------------------------------------------------------------------
// The line jx = nx/2 for every jy and n, on the CUDA cores in FP32:
//   t[b][n] = sum_a Ex[nx/2, a] A[b, a, n]            (in k_tp_prep, from its tile of A)
//   G[nx/2, jy, n] = sum_b Ey[jy, b] t[b][n]          (k_tp_nyq_g: CTA = 32 n x 8 jy at a time)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tp_nyq_g(const Geo G, const float2* __restrict__ t,
                                                  const float2* __restrict__ eyf, float2* __restrict__ Ghat) {
    __shared__ float2 ts[K][33];                     // t[b][n0 .. n0 + 31]
    const int n0 = blockIdx.x * 32;
    const int ln = threadIdx.x & 31, jr = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < K * 32; i += 256) {
        const int b = i >> 5, c = i & 31;
        ts[b][c] = (n0 + c < G.Nt) ? t[(size_t)b * G.Nt + n0 + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int n = n0 + ln;
    for (int bj = blockIdx.y * 8 + jr; bj < G.nyp; bj += gridDim.y * 8) {   // jy = bj - ny/2
        float2 sacc = make_float2(0.f, 0.f);
#pragma unroll 8
        for (int b = 0; b < K; ++b) {
            const float2 e = __ldg(&eyf[(size_t)bj * K + b]);
            const float2 v = ts[b][ln];
            sacc.x = fmaf(e.x, v.x, fmaf(-e.y, v.y, sacc.x));
            sacc.y = fmaf(e.x, v.y, fmaf(e.y, v.x, sacc.y));
        }
        if (n < G.Nt) Ghat[((size_t)(G.nx / 2) * G.nyp + bj) * G.Nt + n] = sacc;
    }
}

}  // namespace tp

// time samples per pass of the tensor-product stage: the GEMM 2 operand
// tiles of one pass (128 KB per time sample) stay in L2 between the GEMMs
int tp_chunk(int Nt) { return Nt < 512 ? Nt : 512; }

size_t tp_work_bytes(int Nt) {
    // data operands (hi, lo) + GEMM 1 output (4 matrices) per time sample of a
    // pass, plus the Nyquist-line partial sums of all time samples
    return (size_t)tp_chunk(Nt) * (2 + 4) * tp::MAT + (size_t)Nt * tp::K * sizeof(float2);
}

size_t tp_gemm1_smem() { return 4 * tp::MAT + tp::STAGES * 2 * tp::CHUNK; }
size_t tp_gemm2_smem() { return 4 * tp::MAT + tp::STAGES * tp::DT_STAGE; }

cudaError_t configure_tp_kernels() {
    cudaError_t e;
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if ((e = cudaFuncSetAttribute(tp::k_tp_gemm1<__nv_bfloat16>, a, (int)tp_gemm1_smem()))) return e;
    if ((e = cudaFuncSetAttribute(tp::k_tp_gemm2<__nv_bfloat16>, a, (int)tp_gemm2_smem()))) return e;
    if ((e = cudaFuncSetAttribute(tp::k_tp_gemm1<__half>, a, (int)tp_gemm1_smem()))) return e;
    if ((e = cudaFuncSetAttribute(tp::k_tp_gemm2<__half>, a, (int)tp_gemm2_smem()))) return e;
    return cudaSuccess;
}

template <typename T>
static cudaError_t launch_tp_ned_t(const nedner_plan_s& p, const float* g, float2* Ghat, cudaStream_t s,
                                   const unsigned int* absmax) {
    const Geo& G = p.geo;
    T* At = reinterpret_cast<T*>(p.tp.work);
    const int ch = tp_chunk(G.Nt);
    T* Dt = At + (size_t)ch * 2 * (tp::ROWS * tp::K);
    float2* tl = reinterpret_cast<float2*>(Dt + (size_t)ch * 4 * (tp::ROWS * tp::K));
    for (int nb = 0; nb < G.Nt; nb += ch) {
        const int ne = nb + ch;
        tp::k_tp_prep<T><<<dim3(ch / 16, tp::K / 4), 256, 0, s>>>(G, g, p.t.sens_fac, p.tp.exn, At, tl, nb, ne,
                                                                  absmax);
        tp::k_tp_gemm1<T><<<std::min(ch, p.tp.sms), 320, tp_gemm1_smem(), s>>>(
            G, reinterpret_cast<const T*>(p.tp.ex), At, p.tp.eyf, Dt, Ghat, p.tp.err, nb, ne, absmax,
            p.tp.wait_limit);
        tp::k_tp_gemm2<T><<<2 * std::max(1, p.tp.sms / 2), 192, tp_gemm2_smem(), s>>>(
            G, Dt, reinterpret_cast<const T*>(p.tp.ey), Ghat, p.tp.err, nb, ne, absmax, p.tp.wait_limit);
    }
    tp::k_tp_nyq_g<<<dim3((G.Nt + 31) / 32, (G.nyp + 7) / 8), 256, 0, s>>>(G, tl, p.tp.eyf, Ghat);
    return cudaGetLastError();
}

cudaError_t launch_tp_ned(const nedner_plan_s& p, const float* g, float2* Ghat, cudaStream_t s) {
    if (!p.tp.fp16) return launch_tp_ned_t<__nv_bfloat16>(p, g, Ghat, s, nullptr);
    cudaError_t e = cudaMemsetAsync(p.tp.absmax, 0, sizeof(unsigned int), s);
    if (e) return e;
    const size_t n4 = (size_t)p.geo.M * p.geo.Nt / 4;
    const int blocks = (int)std::min<size_t>((n4 + 255) / 256, (size_t)p.tp.sms * 8);
    tp::k_tp_absmax<<<blocks, 256, 0, s>>>(p.geo, g, p.t.sens_fac, p.tp.absmax);
    return launch_tp_ned_t<__half>(p, g, Ghat, s, p.tp.absmax);
}

}  // namespace nedner

// Utilities around the reconstruction that the experiments of Sec. 8 and the
// quality measures of Appendix B use:
//  - the data low-pass of Sec. 8 against spatial aliasing: sensor m's time
//    series keeps the frequencies |f| <= c / (2 dx_m), dx_m the distance from
//    sensor m to its nearest neighbour (the local sensor spacing);
//  - the Tenenbaum sharpness (Appendix B): the sum over an image of the
//    squared responses to the Sobel operator and its transpose, divided by
//    the number of pixels;
//  - maximum intensity projections of a volume (the paper compares
//    reconstructions as MIPs).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "fft.cuh"
#include "internal.h"
#include "nedner.h"

namespace nedner {

// ---------------------------------------------------------------------------
// host: per-sensor cut-off bins of the low-pass
// ---------------------------------------------------------------------------
// Nearest-neighbour distance of every sensor: the sensors are binned into a
// square grid of cells over the aperture; each sensor searches the cells in
// growing square rings around its own until the best distance found is no
// more than the ring's inner distance (all unvisited sensors are at least
// that far away).
std::vector<double> nearest_neighbour_distance(const std::vector<double>& xy, int64_t M, double X, double Y) {
    std::vector<double> d(M, INFINITY);
    if (M < 2) return d;
    const int nc = std::max(1, (int)std::ceil(std::sqrt((double)M)));
    const double cw = X / nc, ch = Y / nc;
    auto cell_of = [&](double v, double lo, double w) {
        return std::min(nc - 1, std::max(0, (int)std::floor((v - lo) / w)));
    };
    std::vector<int> head(nc * nc, -1), next(M, -1);
    std::vector<int> cx(M), cy(M);
    for (int64_t m = 0; m < M; ++m) {
        cx[m] = cell_of(xy[2 * m], -0.5 * X, cw);
        cy[m] = cell_of(xy[2 * m + 1], -0.5 * Y, ch);
        const int c = cy[m] * nc + cx[m];
        next[m] = head[c];
        head[c] = (int)m;
    }
    const double cmin = std::min(cw, ch);
    for (int64_t m = 0; m < M; ++m) {
        double best2 = INFINITY;
        for (int r = 0; r < nc; ++r) {
            for (int y = cy[m] - r; y <= cy[m] + r; ++y) {
                if (y < 0 || y >= nc) continue;
                const bool edge_row = (y == cy[m] - r || y == cy[m] + r);
                for (int x = cx[m] - r; x <= cx[m] + r; x += (edge_row || r == 0) ? 1 : 2 * r) {
                    if (x < 0 || x >= nc) continue;
                    for (int q = head[y * nc + x]; q >= 0; q = next[q]) {
                        if (q == m) continue;
                        const double ex = xy[2 * q] - xy[2 * m], ey = xy[2 * q + 1] - xy[2 * m + 1];
                        best2 = std::min(best2, ex * ex + ey * ey);
                    }
                }
            }
            const double reach = r * cmin;            // every unvisited sensor is at least this far
            if (best2 <= reach * reach) break;
        }
        d[m] = std::sqrt(best2);
    }
    return d;
}

// highest kept bin k (|k| <= k_m of the length-Nt DFT, f_k = k / (Nt dt)) for
// f_cut = c / (2 dx_m); Nt/2 (no filtering) for a lone sensor
std::vector<int> lowpass_bins(const nedner_plan_s& p) {
    const double X = p.grid.nx * p.grid.dx, Y = p.grid.ny * p.grid.dy;
    const std::vector<double> d = nearest_neighbour_distance(p.xy, p.M, X, Y);
    std::vector<int> k(p.M, p.Nt / 2);
    for (int64_t m = 0; m < p.M; ++m) {
        if (!std::isfinite(d[m]) || d[m] <= 0.0) continue;
        const double kf = p.c / (2.0 * d[m]) * p.Nt * p.dt;
        k[m] = (int)std::min<double>(p.Nt / 2, std::floor(kf));
    }
    return k;
}

// ---------------------------------------------------------------------------
// low-pass: one CTA per pair of sensors (m0, m0 + 1), transformed together as
// z = g[m0] + i g[m0 + 1]; the two real spectra are separated through the
// Hermitian pairs (k, Nt - k), each cut at its own bin, recombined and
// transformed back.  Ideal (rectangular) filter.
// ---------------------------------------------------------------------------
template <int PER>
__global__ void __launch_bounds__(256) k_lowpass(int64_t M, int Nt, const float* __restrict__ g,
                                                 const int* __restrict__ kcut, const float2* __restrict__ tw,
                                                 float* __restrict__ out) {
    extern __shared__ float4 smem4[];
    float2* Z = reinterpret_cast<float2*>(smem4);                    // padded [Nt]
    const int64_t m0 = 2 * (int64_t)blockIdx.x, m1 = m0 + 1;
    const bool two = m1 < M;
    const float* a = g + m0 * Nt;
    const float* b = g + m1 * Nt;
    for (int n = threadIdx.x; n < Nt; n += blockDim.x) Z[padx(n)] = make_float2(a[n], two ? b[n] : 0.f);
    block_fft_ip<PER>(Z, Nt, 1, -1, tw);
    const int K0 = __ldg(&kcut[m0]), K1 = two ? __ldg(&kcut[m1]) : 0;
    for (int k = threadIdx.x; k <= Nt / 2; k += blockDim.x) {
        const int km = (Nt - k) & (Nt - 1);
        const float2 zk = Z[padx(k)], zm = cconj(Z[padx(km)]);
        float2 A = cscale(cadd(zk, zm), 0.5f);                         // spectrum of g[m0] at k
        float2 B = cscale(mul_i(csub(zk, zm), -1), 0.5f);              // spectrum of g[m1] at k
        if (k > K0) A = make_float2(0.f, 0.f);
        if (k > K1) B = make_float2(0.f, 0.f);
        Z[padx(k)] = cadd(A, mul_i(B, +1));
        Z[padx(km)] = cadd(cconj(A), mul_i(cconj(B), +1));
    }
    block_fft_ip<PER>(Z, Nt, 1, +1, tw);
    const float s = 1.f / Nt;
    float* oa = out + m0 * Nt;
    float* ob = out + m1 * Nt;
    for (int n = threadIdx.x; n < Nt; n += blockDim.x) {
        const float2 z = Z[padx(n)];
        oa[n] = z.x * s;
        if (two) ob[n] = z.y * s;
    }
}

// ---------------------------------------------------------------------------
// Tenenbaum sharpness: one CTA per image; every thread sums its pixels'
// squared Sobel responses in FP64, then a fixed-order tree over the CTA
// (the result does not depend on scheduling).  Pixels whose 3 x 3
// neighbourhood lies in the image (the valid part of the convolution).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tenenbaum(int ny, int nx, const float* __restrict__ U,
                                                   double* __restrict__ F) {
    __shared__ double part[256];
    const float* u = U + (size_t)blockIdx.x * ny * nx;
    double acc = 0.0;
    const int wx = nx - 2, wy = ny - 2;
    const long npx = (wx > 0 && wy > 0) ? (long)wx * wy : 0;
    for (long i = threadIdx.x; i < npx; i += blockDim.x) {
        const int y = 1 + (int)(i / wx), x = 1 + (int)(i % wx);
        const float* r0 = u + (size_t)(y - 1) * nx + x;
        const float* r1 = r0 + nx;
        const float* r2 = r1 + nx;
        const float gx = (r0[1] + 2.f * r1[1] + r2[1]) - (r0[-1] + 2.f * r1[-1] + r2[-1]);
        const float gy = (r2[-1] + 2.f * r2[0] + r2[1]) - (r0[-1] + 2.f * r0[0] + r0[1]);
        acc += (double)gx * gx + (double)gy * gy;
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) F[blockIdx.x] = part[0] / ((double)nx * ny);
}

// ---------------------------------------------------------------------------
// maximum intensity projections of a (nz, ny, nx) volume along one axis
// ---------------------------------------------------------------------------
// axis 0 -> (ny, nx), axis 1 -> (nz, nx): one thread per output value, the
// threads of a warp on neighbouring x
__global__ void k_mip_zy(int nz, int ny, int nx, int axis, const float* __restrict__ v, float* __restrict__ out) {
    const long n_out = axis == 0 ? (long)ny * nx : (long)nz * nx;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n_out; i += (long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const long o = i / nx;                         // y (axis 0) or z (axis 1)
        float m = -INFINITY;
        if (axis == 0) {
            for (int z = 0; z < nz; ++z) m = fmaxf(m, v[((size_t)z * ny + o) * nx + x]);
        } else {
            for (int y = 0; y < ny; ++y) m = fmaxf(m, v[((size_t)o * ny + y) * nx + x]);
        }
        out[i] = m;
    }
}

// axis 2 -> (nz, ny): one warp per output value, lanes over x
__global__ void k_mip_x(int nz, int ny, int nx, const float* __restrict__ v, float* __restrict__ out) {
    const long n_out = (long)nz * ny;
    const int lane = threadIdx.x & 31;
    for (long i = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n_out;
         i += ((long)gridDim.x * blockDim.x) >> 5) {
        float m = -INFINITY;
        for (int x = lane; x < nx; x += 32) m = fmaxf(m, v[(size_t)i * nx + x]);
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) out[i] = m;
    }
}

}  // namespace nedner

using namespace nedner;

static nedner_status util_status(cudaError_t e) {
    if (e == cudaSuccess) return NEDNER_OK;
    return e == cudaErrorMemoryAllocation ? NEDNER_ENOMEM : NEDNER_ECUDA;
}

extern "C" {

nedner_status nedner_lowpass(nedner_plan_t p, const float* g, float* out, void* stream) {
    if (!p || (p->M > 0 && (!g || !out))) return NEDNER_EINVAL;
    if (((uintptr_t)g & 3) != 0 || ((uintptr_t)out & 3) != 0) return NEDNER_EINVAL;
    if (p->M == 0) return NEDNER_OK;
    const int Nt = p->Nt;
    const int threads = std::max(32, std::min(256, Nt / 16));
    const size_t smem = (size_t)((padded_len(Nt) + 1) & ~1) * sizeof(float2);
    const int per = Nt > 16 * threads ? 32 : 16;
    if ((long)Nt > (long)per * threads) return NEDNER_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned blocks = (unsigned)((p->M + 1) / 2);
    cudaError_t e;
    if (per == 16) {
        if ((e = cudaFuncSetAttribute(k_lowpass<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
            return util_status(e);
        k_lowpass<16><<<blocks, threads, smem, s>>>(p->M, Nt, g, p->t.lp_kcut, p->t.tw, out);
    } else {
        if ((e = cudaFuncSetAttribute(k_lowpass<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
            return util_status(e);
        k_lowpass<32><<<blocks, threads, smem, s>>>(p->M, Nt, g, p->t.lp_kcut, p->t.tw, out);
    }
    return util_status(cudaGetLastError());
}

int nedner_lowpass_bins(nedner_plan_t p, int* out, int64_t nout) {
    if (!p || (nout > 0 && !out)) return -1;
    for (int64_t m = 0; m < p->M && m < nout; ++m) out[m] = p->lp_kcut[m];
    return 0;
}

nedner_status nedner_tenenbaum(const float* U, int64_t B, int ny, int nx, double* F, void* stream) {
    if (B < 0 || ny < 0 || nx < 0) return NEDNER_EINVAL;
    if (B == 0) return NEDNER_OK;
    if (!U || !F || ((uintptr_t)U & 3) != 0 || ((uintptr_t)F & 7) != 0) return NEDNER_EINVAL;
    if (B > 0x7fffffff) return NEDNER_EINVAL;
    k_tenenbaum<<<(unsigned)B, 256, 0, (cudaStream_t)stream>>>(ny, nx, U, F);
    return util_status(cudaGetLastError());
}

nedner_status nedner_mip(const float* vol, int nz, int ny, int nx, int axis, float* out, void* stream) {
    if (nz <= 0 || ny <= 0 || nx <= 0 || axis < 0 || axis > 2) return NEDNER_EINVAL;
    if (!vol || !out || ((uintptr_t)vol & 3) != 0 || ((uintptr_t)out & 3) != 0) return NEDNER_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (axis == 2) {
        const long warps = (long)nz * ny;
        const unsigned blocks = (unsigned)std::min<long>((warps + 7) / 8, 152L * 32);
        k_mip_x<<<blocks, 256, 0, s>>>(nz, ny, nx, vol, out);
    } else {
        const long n = axis == 0 ? (long)ny * nx : (long)nz * nx;
        const unsigned blocks = (unsigned)std::min<long>((n + 255) / 256, 152L * 32);
        k_mip_zy<<<blocks, 256, 0, s>>>(nz, ny, nx, axis, vol, out);
    }
    return util_status(cudaGetLastError());
}

}  // extern "C"

// Forward NEDNER kernels (the reconstruction R of Eq. disc_rec, Sec. 3).
//
// Data flow (all intermediates complex64, n / qz / qy fastest as noted):
//   g [M][Nt]
//     -- ned_spread_blocks -> Q   [tq/32][Ly][Lx][32] spread along y and x, one chunk of tq time samples
//     -- ned_xfft         -->  R    [nx/2+1][Ly][tq]   x-FFT, crop, deconvolve (the chunk)
//     -- ned_yfft         -->  Ghat [nx/2+1][ny+1][Nt] y-FFT, crop, deconvolve (the chunk)
//   (or, fused, ned_spread_xfft --> R [nx/2+1][Ly][Nt] for every time sample at once)
//     -- ner_lines        -->  V    [nx/2+1][ny][nz]   NER, Jacobian, z-IFFT
//     -- img_yifft        -->  Y    [nx/2+1][nz][ny]   y-IFFT
//     -- img_xc2r         -->  p0   [nz][ny][nx]       x complex-to-real IFFT
#include <cuda_runtime.h>


#include "fft.cuh"
#include "async_copy.cuh"
#include "internal.h"
#include "ner_eval.cuh"
#include "spread_window.cuh"

namespace nedner {


// ---------------------------------------------------------------------------
// Stage (a), part 1: NED spreading (Eq. NED_NUFFT) fused with the x-FFT.
// One CTA of 256 threads owns grid row gy and C consecutive time samples.
// Its threads form lane groups of C (lane = time sample); group q owns the
// column segment seg[gy][q] = [c0, c1) of the row.  The row's entries
// (sensor, y tap) are sorted by their first x column; each entry's w taps
// (already multiplied by the y tap and the sensor factor) are stored as WT
// values starting at a column bx4 that is a multiple of 4 (leading zeros
// absorb bx - bx4).  The group sweeps the entries whose taps reach into its
// segment, keeping the 2 WT columns [base, base + 2 WT) in registers: an
// entry with bx4 - base > WT first moves the window up by WT columns (the
// lower WT are final: stored once if inside the segment), then its taps are
// added at offset d = bx4 - base, a multiple of 4 in [0, WT], with WT FMAs
// (a branch on d with WT/4 + 1 cases, uniform across the group).  No atomics,
// no shared-memory read-modify-write; every column is written exactly once.
// Entries are staged eight at a time (indices, taps, samples of g), the next
// batch arriving by asynchronous copies while the current one is swept.
// The row is held as C/2 complex columns (time samples 2b, 2b+1 packed as
// real and imaginary part) in a padded buffer, transformed in place along x
// (PER values per thread), and jx = 0..nx/2 is kept, divided by phihat(jx/Lx).
// ---------------------------------------------------------------------------
template <int WT, int PER>
__global__ void __launch_bounds__(256, PER <= 16 ? 3 : 2) k_ned_spread_xfft(Geo G, int C, int yb, const float* __restrict__ g,
                                                                          const int4* __restrict__ seg,
                                                                          const int* __restrict__ xent_m,
                                                                          const float* __restrict__ xent_wx,
                                                                          const int* __restrict__ xent_bx,
                                                                          const float* __restrict__ deconv_x,
                                                                          const float2* __restrict__ tw,
                                                                          float2* __restrict__ R) {
    constexpr int NT = 256;
    constexpr int B = 8;                                           // entries per staged batch
    extern __shared__ float4 smem4[];
    const int Lx = G.Lx;
    const int nb = C / 2;
    const int lnb = ilog2(nb);
    float2* Z = reinterpret_cast<float2*>(smem4);                  // [Lx][C/2] complex row, padded
    float* Zf = reinterpret_cast<float*>(Z);
    const int zlen = (padded_len(Lx * nb) + 1) & ~1;
    const int gy = blockIdx.x;
    const int n0 = (yb + blockIdx.y) * C;
    const int lc = ilog2(C);
    const int groups = NT >> lc;
    const int q = threadIdx.x >> lc;
    const int ln = threadIdx.x & (C - 1);

    const int4 sg = seg[(size_t)gy * groups + q];      // c0, c1, first entry, end entry
    float acc[2 * WT];
#pragma unroll
    for (int k = 0; k < 2 * WT; ++k) acc[k] = 0.f;
    int base = (sg.x - WT) & ~3;

    // Per-group staging, double-buffered: the entries' sensor indices one batch
    // ahead, and bx4[B], taps[B][WT], g[B][C] of the next batch, arrive by
    // cp.async while the current batch is swept.
    const unsigned gmask = (C >= 32) ? 0xffffffffu : (((1u << C) - 1u) << ((threadIdx.x & 31) - ln));
    constexpr int DB = B + B * WT;                                 // ints + floats before the g block
    const int dsz = DB + B * C;                                    // one data buffer (4-byte words)
    int* st_m = reinterpret_cast<int*>(Z + zlen) + (size_t)q * (2 * B + 2 * dsz);   // [2][B]
    int* st_d = st_m + 2 * B;                                      // [2][dsz]
    const int nent = sg.w - sg.z;
    const int nbt = (nent + B - 1) / B;
    const int cw = C >= 4 ? 4 : C;                                 // floats per copy of g
    auto issue_m = [&](int b) {
        const int e0 = sg.z + b * B, nb_ = min(B, sg.w - e0);
        for (int j = ln; j < nb_; j += C) cp_async(st_m + (b & 1) * B + j, xent_m + e0 + j, 4);
    };
    auto issue_data = [&](int b) {
        const int e0 = sg.z + b * B, nb_ = min(B, sg.w - e0);
        int* d = st_d + (b & 1) * dsz;
        const int* mm = st_m + (b & 1) * B;
        for (int j = ln; j < nb_; j += C) cp_async(d + j, xent_bx + e0 + j, 4);
        const float* wsrc = xent_wx + (size_t)e0 * WT;
        for (int i = ln; i < nb_ * (WT / 4); i += C) cp_async(d + B + 4 * i, wsrc + 4 * i, 16);
        const int per = C / cw;                                    // copies per entry
        for (int i = ln; i < nb_ * per; i += C) {
            const int j = i / per, c = i - j * per;
            cp_async(d + DB + j * C + c * cw, g + (size_t)mm[j] * G.Nt + n0 + c * cw, cw * 4);
        }
    };
    if (nbt > 0) {
        issue_m(0);
        cp_async_commit();
        cp_async_wait_all();
        __syncwarp(gmask);
        issue_data(0);
        if (nbt > 1) issue_m(1);
        cp_async_commit();
    }
    for (int b = 0; b < nbt; ++b) {
        cp_async_wait_all();
        __syncwarp(gmask);
        if (b + 1 < nbt) issue_data(b + 1);
        if (b + 2 < nbt) issue_m(b + 2);
        cp_async_commit();
        const int nbat = min(B, nent - b * B);
        const int* st_bx = st_d + (b & 1) * dsz;
        const float4* wst = reinterpret_cast<const float4*>(st_bx + B);
        const float* st_g = reinterpret_cast<const float*>(st_bx + DB);
#pragma unroll 1
        for (int j = 0; j < nbat; ++j) {
            const int bxa = st_bx[j];
            const float ga = st_g[j * C + ln];
            float4 wa[WT / 4];
#pragma unroll
            for (int k4 = 0; k4 < WT / 4; ++k4) wa[k4] = wst[j * (WT / 4) + k4];
            sweep_entry<WT>(acc, Zf, lnb, ln, base, sg.x, sg.y, bxa, wa, ga);
        }
        __syncwarp(gmask);
    }
    while (base < sg.y) {
        flush_lower<WT>(acc, Zf, lnb, ln, base, sg.x, sg.y);
        base += WT;
    }

    const bool fold = (ilog2(Lx) & 3) == 1;
    block_fft_ip<PER>(Z, Lx, nb, -1, tw, fold);
    for (int it = threadIdx.x; it < (G.nxh << lnb); it += NT)
        spread_output(G, Z, lnb, it & (nb - 1), it >> lnb, fold, deconv_x, tw, gy, n0, R);
}

template <int WT, int NT>
__global__ void __launch_bounds__(NT, NT <= 256 ? 2 : 1) k_ned_spread2_xfft(Geo G, int yb, const float* __restrict__ g,
                                                             const int4* __restrict__ seg,
                                                             const int* __restrict__ xent_m,
                                                             const float* __restrict__ xent_wx,
                                                             const int* __restrict__ xent_bx,
                                                             const float* __restrict__ deconv_x,
                                                             const float2* __restrict__ tw,
                                                             float2* __restrict__ R) {
    constexpr int B = 8, C = 64, NB = 32;
    constexpr int PER = 32;                          // values per thread of the in-place x-FFT, Lx * 32 <= PER * NT
    extern __shared__ float4 smem4[];
    const int Lx = G.Lx;
    float2* Z = reinterpret_cast<float2*>(smem4);                  // [Lx][32] complex row, padded
    const int zlen = (padded_len(Lx * NB) + 1) & ~1;
    const int gy = blockIdx.x;
    const int n0 = (yb + blockIdx.y) * C;
    const int q = threadIdx.x >> 5;                                // lane group = warp
    const int ln = threadIdx.x & 31;

    const int4 sg = seg[(size_t)gy * (NT / 32) + q];   // c0, c1, first entry, end entry
    float2 acc[2 * WT];
#pragma unroll
    for (int k = 0; k < 2 * WT; ++k) acc[k] = make_float2(0.f, 0.f);
    int base = (sg.x - WT) & ~3;

    // double-buffered staging as in k_ned_spread_xfft: m[2][B], then per buffer
    // bx4[B], taps[B][WT], g[B][C]
    constexpr int DB = B + B * WT;
    constexpr int dsz = DB + B * C;
    int* st_m = reinterpret_cast<int*>(Z + zlen) + (size_t)q * (2 * B + 2 * dsz);
    int* st_d = st_m + 2 * B;
    const int nent = sg.w - sg.z;
    const int nbt = (nent + B - 1) / B;
    auto issue_m = [&](int b) {
        const int e0 = sg.z + b * B, nb_ = min(B, sg.w - e0);
        if (ln < nb_) cp_async(st_m + (b & 1) * B + ln, xent_m + e0 + ln, 4);
    };
    auto issue_data = [&](int b) {
        const int e0 = sg.z + b * B, nb_ = min(B, sg.w - e0);
        int* d = st_d + (b & 1) * dsz;
        const int* mm = st_m + (b & 1) * B;
        if (ln < nb_) cp_async(d + ln, xent_bx + e0 + ln, 4);
        const float* wsrc = xent_wx + (size_t)e0 * WT;
        for (int i = ln; i < nb_ * (WT / 4); i += 32) cp_async(d + B + 4 * i, wsrc + 4 * i, 16);
#pragma unroll
        for (int r = 0; r < B * (C / 4) / 32; ++r) {
            const int i = ln + 32 * r;
            const int j = i >> 4, c = i & 15;
            if (j < nb_) cp_async(d + DB + j * C + 4 * c, g + (size_t)mm[j] * G.Nt + n0 + 4 * c, 16);
        }
    };
    if (nbt > 0) {
        issue_m(0);
        cp_async_commit();
        cp_async_wait_all();
        __syncwarp();
        issue_data(0);
        if (nbt > 1) issue_m(1);
        cp_async_commit();
    }
    for (int b = 0; b < nbt; ++b) {
        cp_async_wait_all();
        __syncwarp();
        if (b + 1 < nbt) issue_data(b + 1);
        if (b + 2 < nbt) issue_m(b + 2);
        cp_async_commit();
        const int nbat = min(B, nent - b * B);
        const int* st_bx = st_d + (b & 1) * dsz;
        const float4* wst = reinterpret_cast<const float4*>(st_bx + B);
        const float2* st_g = reinterpret_cast<const float2*>(st_bx + DB);
#pragma unroll 1
        for (int j = 0; j < nbat; ++j) {
            const int bxa = st_bx[j];
            const float2 ga = st_g[j * NB + ln];
            float4 wa[WT / 4];
#pragma unroll
            for (int k4 = 0; k4 < WT / 4; ++k4) wa[k4] = wst[j * (WT / 4) + k4];
            sweep_entry2<WT>(acc, Z, ln, base, sg.x, sg.y, bxa, wa, ga);
        }
        __syncwarp();
    }
    while (base < sg.y) {
        flush_lower2<WT>(acc, Z, ln, base, sg.x, sg.y);
        base += WT;
    }

    const bool fold = (ilog2(Lx) & 3) == 1;
    block_fft_ip<PER>(Z, Lx, NB, -1, tw, fold);
    for (int it = threadIdx.x; it < (G.nxh << 5); it += NT)
        spread_output(G, Z, 5, it & 31, it >> 5, fold, deconv_x, tw, gy, n0, R);
}

// ---------------------------------------------------------------------------
// Stage (a), part 1 as two kernels over a chunk of tq time samples [t0, t0 + tq).
//
// k_ned_spread_blocks: NED spreading (Eq. NED_NUFFT) into the oversampled
// grid Q [tq/32][Ly][Lx][32] (real; groups of 32 time samples, time fastest).
// One warp owns one block of 16 columns of one grid row for 64 time samples
// (two per lane, packed FMAs) and adds every entry (sensor, y tap) of the row
// whose x taps reach into the block.  The plan stores each such entry with
// its taps aligned to the block's 16 columns (block_taps16), so an entry is
// 16 packed FMAs with no branch on its offset (block_entry16); the block's
// entries are one range bseg[row][block] of bent_m / bent_w.  Entries are
// staged SPREAD_BATCH at a time per warp (sensor indices one batch ahead, then taps
// and samples of g by asynchronous copies while the current batch is added).
// The warp then stores its 16 columns (128 contiguous bytes per column and
// 32 samples) and is done: no shared row buffer and no barrier, so warps of
// dense and sparse blocks do not wait for one another, and many small CTAs
// keep every SM busy.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128, 7) k_ned_spread_blocks(Geo G, int t0, int tq, const float* __restrict__ g,
                                                              const int2* __restrict__ bseg,
                                                              const int* __restrict__ bent_m,
                                                              const float* __restrict__ bent_w,
                                                              float* __restrict__ Q) {
    constexpr int B = SPREAD_BATCH, C = 64, NB = 32;
    constexpr int DB = B * 16;                                      // taps before the g block (floats)
    constexpr int dsz = DB + B * C;                                 // one data buffer (4-byte words)
    extern __shared__ float4 smem4[];
    const int wpc = blockDim.x >> 5;
    const int q = threadIdx.x >> 5;
    const int ln = threadIdx.x & 31;
    const int nblk = G.Lx >> 4;
    const int gb = blockIdx.x * wpc + q;                            // (row, block) index
    const int gy = gb / nblk;
    const int c0 = (gb - gy * nblk) << 4;
    const int nc = blockIdx.y * C;                                  // first sample of the warp in the chunk
    const int2 rg = bseg[gb];

    float2 acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = make_float2(0.f, 0.f);

    // sensor indices NM batches deep, data ND batches deep: group k of copies
    // holds the data of batch k and the indices of batch k + 3, so the data of
    // batch b + 2 are issued while batch b is added (their indices arrived two
    // groups earlier)
    constexpr int NM = 4, ND = 3;
    int* st_m = reinterpret_cast<int*>(smem4) + (size_t)q * (NM * B + ND * dsz);  // [NM][B]
    float* st_d = reinterpret_cast<float*>(st_m + NM * B);                          // [ND][dsz]
    const int nent = rg.y - rg.x;
    const int nbt = (nent + B - 1) / B;
    auto issue_m = [&](int b) {
        if (b >= nbt) return;
        const int e0 = rg.x + b * B, nb_ = min(B, rg.y - e0);
        if (ln < nb_) cp_async(st_m + (b % NM) * B + ln, bent_m + e0 + ln, 4);
    };
    auto issue_data = [&](int b) {
        if (b >= nbt) return;
        const int e0 = rg.x + b * B, nb_ = min(B, rg.y - e0);
        float* d = st_d + (b % ND) * dsz;
        const int* mm = st_m + (b % NM) * B;
        // B entries x 16 taps = 4 B copies of 16 bytes
#pragma unroll
        for (int r = 0; r < B / 8; ++r) {
            const int i = ln + 32 * r;
            if ((i >> 2) < nb_) cp_async(d + 4 * i, bent_w + (size_t)e0 * 16 + 4 * i, 16);
        }
#pragma unroll
        for (int r = 0; r < B * (C / 4) / 32; ++r) {
            const int i = ln + 32 * r;
            const int j = i >> 4, c = i & 15;
            if (j < nb_) cp_async(d + DB + j * C + 4 * c, g + (size_t)mm[j] * G.Nt + t0 + nc + 4 * c, 16);
        }
    };
    if (nbt > 0) {
        issue_m(0);
        issue_m(1);
        issue_m(2);
        cp_async_commit();
        cp_async_wait_all();
        __syncwarp();
        issue_data(0);
        issue_m(3);
        cp_async_commit();                                          // group 0
        issue_data(1);
        issue_m(4);
        cp_async_commit();                                          // group 1
    }
    for (int b = 0; b < nbt; ++b) {
        cp_async_wait_group<1>();                                   // groups up to b done
        __syncwarp();
        issue_data(b + 2);                                          // its indices: group b - 1
        issue_m(b + 5);
        cp_async_commit();                                          // group b + 2
        const int nbat = min(B, nent - b * B);
        const float4* wst = reinterpret_cast<const float4*>(st_d + (b % ND) * dsz);
        const float2* st_g = reinterpret_cast<const float2*>(st_d + (b % ND) * dsz + DB);
#pragma unroll 1
        for (int j = 0; j < nbat; ++j) {
            const float4 t[4] = {wst[4 * j], wst[4 * j + 1], wst[4 * j + 2], wst[4 * j + 3]};
            block_entry16(acc, t, st_g[j * NB + ln]);
        }
        __syncwarp();
    }
    cp_async_wait_all();
    // Q is [tq/32][Ly][Lx][32]: lanes 0-15 hold the first 32 samples of the
    // warp's 64, lanes 16-31 the next 32; a column's 32 samples are 128
    // contiguous bytes, and the 16 columns of the block 2 KB
    float2* out = reinterpret_cast<float2*>(Q + ((((size_t)(nc >> 5) + (ln >> 4)) * G.Ly + gy) * G.Lx + c0) * 32) +
                  (ln & 15);
#pragma unroll
    for (int k = 0; k < 16; ++k) out[16 * k] = acc[k];
}

// ---------------------------------------------------------------------------
// k_ned_xfft: the x-FFT of the chunk.  One CTA per (grid row gy, 2 NBX time
// samples of the chunk): the row of Q is loaded as NBX complex columns (time
// samples 2b, 2b+1 packed as real and imaginary part) into a padded buffer by
// asynchronous copies (all in flight at once), transformed in place along x
// (PER values per thread), and jx = 0..nx/2 is written to R (the chunk's
// [nx/2+1][Ly][tq]), divided by phihat(jx/Lx).  With NBX = 16 the CTA's part
// of Q is one contiguous block of Lx x 32 samples.
// ---------------------------------------------------------------------------
template <int PER>
__global__ void __launch_bounds__(256, PER <= 16 ? 4 : 2) k_ned_xfft(Geo G, int tq, int nbx, const float* __restrict__ Q,
                                                                    const float* __restrict__ deconv_x,
                                                                    const float2* __restrict__ tw,
                                                                    float2* __restrict__ R) {
    extern __shared__ float4 smem4[];
    float2* Z = reinterpret_cast<float2*>(smem4);                   // [Lx][nbx], padded
    const int gy = blockIdx.x;
    const int nc = blockIdx.y * 2 * nbx;                             // first sample in the chunk
    const int lnb = ilog2(nbx);
    // samples nc .. nc + 2 nbx of the row: group nc / 32, offset nc % 32
    const float2* src = reinterpret_cast<const float2*>(Q + ((size_t)(nc >> 5) * G.Ly + gy) * G.Lx * 32 + (nc & 31));
    for (int it = threadIdx.x; it < (G.Lx << lnb); it += blockDim.x) {
        const int gx = it >> lnb, b = it & (nbx - 1);
        cp_async(&Z[padx(it)], src + (size_t)gx * 16 + b, 8);
    }
    cp_async_commit();
    cp_async_wait_all();
    const bool fold = (ilog2(G.Lx) & 3) == 1;
    block_fft_ip<PER>(Z, G.Lx, nbx, -1, tw, fold);
    Geo Gc = G;
    Gc.Nt = tq;                                                     // R holds the chunk's tq samples
    for (int it = threadIdx.x; it < (G.nxh << lnb); it += blockDim.x)
        spread_output(Gc, Z, lnb, it & (nbx - 1), it >> lnb, fold, deconv_x, tw, gy, nc, R);
}

// ---------------------------------------------------------------------------
// Stage (a), part 2: y-FFT of length Ly for one jx and C time samples; keeps
// jy = -ny/2..ny/2 (both Nyquist rows) divided by phihat(jy/Ly).  The FFT
// runs in place in a padded buffer, Ly * C <= 256 PER (PER values per thread);
// a last radix-2 pass (log2 Ly = 1 mod 4) is applied to the kept rows only.
// blockIdx.x runs over the time chunks, so consecutive CTAs read neighbouring
// pieces of the same rows.
// ---------------------------------------------------------------------------
// R holds time samples [roff, roff + rstride) (the whole record, or one chunk).
template <int PER>
__global__ void __launch_bounds__(256, PER <= 16 ? 4 : 2) k_ned_yfft(Geo G, int C, int yb, const float2* __restrict__ R,
                                                     int rstride, int roff,
                                                     const float* __restrict__ deconv_y,
                                                     const float2* __restrict__ tw, float2* __restrict__ Ghat) {
    extern __shared__ float4 smem4[];
    float2* A = reinterpret_cast<float2*>(smem4);   // [Ly][C], padded
    const int jx = blockIdx.y;
    const int n0 = (yb + blockIdx.x) * C;
    const int lc = ilog2(C);
    for (int it = threadIdx.x; it < G.Ly * C; it += 256) {
        const int gy = it >> lc;
        const int c = it & (C - 1);
        cp_async(&A[padx(it)], &R[((size_t)jx * G.Ly + gy) * rstride + n0 - roff + c], 8);
    }
    cp_async_commit();
    cp_async_wait_all();
    const bool fold = (ilog2(G.Ly) & 3) == 1;
    block_fft_ip<PER>(A, G.Ly, C, -1, tw, fold);
    const int items = G.nyp * C;
    if (!fold) {
        for (int it = threadIdx.x; it < items; it += 256) {
            const int b = it >> lc;                // jy = b - ny/2
            const int c = it & (C - 1);
            const int q = (b - G.ny / 2 + G.Ly) & (G.Ly - 1);
            Ghat[((size_t)jx * G.nyp + b) * G.Nt + n0 + c] = cscale(A[padx(q * C + c)], __ldg(&deconv_y[b]));
        }
    } else {
        // the last radix-2 pass, applied to the nyp kept rows only
        const int H = G.Ly >> 1;
        for (int it = threadIdx.x; it < items; it += 256) {
            const int b = it >> lc;
            const int c = it & (C - 1);
            const int q = (b - G.ny / 2 + G.Ly) & (G.Ly - 1);
            const int k = q & (H - 1);
            const float2 s0 = A[padx((k << lc) + c)];
            const float2 t = cmul(twiddle(tw, k, G.Ly, -1), A[padx(((k + H) << lc) + c)]);
            Ghat[((size_t)jx * G.nyp + b) * G.Nt + n0 + c] = cscale(q < H ? cadd(s0, t) : csub(s0, t),
                                                                    __ldg(&deconv_y[b]));
        }
    }
}

// ---------------------------------------------------------------------------
// Stage (b)+(c)+(z part of d): one CTA per line group (kx, ky),
// kx = 0..nx/2, ky = -ny/2..ny/2-1.
//
// NER (Eq. NER_NUFFT): the line's samples, divided by phihat((n - Nt/2)/Lt)
// and centred (theta = 2 pi n/N - pi), are zero-padded to Lt and FFT'd; the
// value at nu is exp(-i pi nu) sum_k P_k(t) B[mu0 + k] with v = sigma nu,
// mu0 = floor(v) - w/2 + 1, t = v - floor(v).  nu = sign(l) sqrt(axy + az l^2)
// is formed in float-float arithmetic (FP32 pairs) so that the fractional
// offset t keeps FP32 accuracy for |v| in the thousands.
//
// The real part of the inverse 3-D DFT over G_x x G_Ky is rebuilt from the
// half lattice kx = 0..nx/2 (kx = nx/2 standing for -nx/2):
//   kx < nx/2 : U[l] = (F(kx, ky, l) + F(kx, ky*, l*)) / 2
//   kx = nx/2 : U[l] = F(nx/2, ky*, l*)
// where * maps -n/2 to +n/2 and leaves other indices alone (ky* = ky except
// ky* = +ny/2 for ky = -ny/2, which brings in the extra line jy = +ny/2).
// U is multiplied by the Jacobian W, the scale and the voxel-centring sign
// (-1)^(kx+ky), then inverse-transformed along z.
// ---------------------------------------------------------------------------
// One CTA per LPC consecutive line groups (kx, k0..k0+LPC-1).  The LPC lines
// (kx, ky) are transformed together (a batched FFT, one column per line); the
// CTA whose first group is ky = -ny/2 also needs the line (kx, +ny/2), which
// it transforms and evaluates first in the same buffer.  The FFTs run in
// place in padded buffers (see block_fft_ip), NT threads holding 16 values
// each, so Lt * LPC and nz * LPC are at most 16 NT.
// MODE (nedner_opts.ner_interp): NEDNER_NER_KB the NER-NUFFT above; the
// comparison methods of Sec. 5.1: NEDNER_NER_LINEAR_S2 / _S1 the raw line
// zero-padded at the end to 2 Nt / Nt, FFT'd and interpolated linearly
// (ner_value_linear), NEDNER_NER_DIRECT the direct sum over the raw line
// (ner_value_direct, no FFT).  Everything after the NER values is shared.
template <int W, int D, int NT, int MODE = NEDNER_NER_KB>
__global__ void __launch_bounds__(NT, NT <= 256 ? 4 : 1) k_ner_lines(Geo G, const __grid_constant__ TapPoly P, int LPC,
                                                                   const float2* __restrict__ Ghat,
                                                                   const float2* __restrict__ axy_tab,
                                                                   const float* __restrict__ deconv_t,
                                                                   const float2* __restrict__ tw,
                                                                   float2* __restrict__ V) {
    constexpr int PER = 16;
    constexpr int SIG = MODE == NEDNER_NER_LINEAR_S1 || MODE == NEDNER_NER_DIRECT ? 1 : 2;
    extern __shared__ float4 smem4[];
    const int nz1 = G.nz + 1;
    const int Lt = SIG * G.Nt;
    float2* LA = reinterpret_cast<float2*>(smem4);                 // [Lt][LPC], padded
    float2* T = LA + padded_len(G.Lt * LPC);                       // [LPC + 1][nz + 1] values at l = -nz/2..nz/2
    float2* UA = T + (size_t)(LPC + 1) * nz1;                      // [nz][LPC], padded
    // the NER value of column c of LA at l (e = l + nz/2)
    auto value = [&](float2 axy, bool j0, int l, int lld, int c) {
        if constexpr (MODE == NEDNER_NER_KB) return ner_value<W, D>(G, P, axy, j0, l, LA, lld, c);
        else if constexpr (MODE == NEDNER_NER_DIRECT) return ner_value_direct(G, axy, j0, l, LA, lld, c);
        else return ner_value_linear<SIG>(G, axy, j0, l, LA, lld, c);
    };

    const int llpc = ilog2(LPC), lnz = ilog2(G.nz);
    const int cpk = G.ny >> llpc;                    // CTAs per kx
    const int kx = blockIdx.x / cpk;
    const int k0 = (blockIdx.x - kx * cpk) * LPC - G.ny / 2;
    const bool nyq_x = (kx == G.nx / 2);
    const int half_nz = G.nz / 2;
    const size_t line0 = (size_t)kx * G.nyp + (k0 + G.ny / 2);

    if (k0 == -G.ny / 2) {
        // the line (kx, +ny/2): centred, deconvolved, zero-padded, in column 0
        const size_t lx = (size_t)kx * G.nyp + G.ny;
        const float2* src = Ghat + lx * G.Nt;
        if constexpr (MODE == NEDNER_NER_KB) {
#pragma unroll 4
            for (int n = threadIdx.x; n < G.Nt; n += NT)
                LA[padx((n - G.Nt / 2) & (G.Lt - 1))] = cscale(src[n], __ldg(&deconv_t[n]));
            block_fft_ip<PER, true>(LA, G.Lt, 1, -1, tw);
        } else {
            for (int n = threadIdx.x; n < Lt; n += NT) LA[padx(n)] = n < G.Nt ? src[n] : make_float2(0.f, 0.f);
            if constexpr (MODE == NEDNER_NER_DIRECT) __syncthreads();
            else block_fft_ip<PER>(LA, Lt, 1, -1, tw);
        }
        const float2 axy = __ldg(&axy_tab[lx]);
        for (int e = threadIdx.x; e < nz1; e += NT) T[LPC * nz1 + e] = value(axy, false, e - half_nz, 0, 0);
        __syncthreads();
    }
    // the LPC lines (theta = 2 pi n/N - pi of Sec. 3.1): centred, deconvolved, zero-padded
    if constexpr (MODE == NEDNER_NER_KB) {
        const float2* src = Ghat + line0 * G.Nt;
#pragma unroll 4
        for (int i = threadIdx.x; i < (G.Nt << llpc); i += NT) {
            const int n = i >> llpc, c = i & (LPC - 1);
            const int p = (n - G.Nt / 2) & (G.Lt - 1);
            LA[padx((p << llpc) + c)] = cscale(src[(size_t)c * G.Nt + n], __ldg(&deconv_t[n]));
        }
        // Lt = 2 Nt: the centred samples fill p < Nt/2 and p >= 3Nt/2 only
        block_fft_ip<PER, true>(LA, G.Lt, LPC, -1, tw);
    } else {
        const float2* src = Ghat + line0 * G.Nt;
        for (int i = threadIdx.x; i < (Lt << llpc); i += NT) {
            const int n = i >> llpc, c = i & (LPC - 1);
            LA[padx(i)] = n < G.Nt ? src[(size_t)c * G.Nt + n] : make_float2(0.f, 0.f);
        }
        if constexpr (MODE == NEDNER_NER_DIRECT) __syncthreads();
        else block_fft_ip<PER>(LA, Lt, LPC, -1, tw);
    }

    // NER values of the LPC lines at l = -nz/2..nz/2
    for (int i = threadIdx.x; i < (G.nz << llpc) + LPC; i += NT) {
        int c, e;
        if (i < (G.nz << llpc)) { c = i >> lnz; e = i & (G.nz - 1); }
        else { c = i - (G.nz << llpc); e = G.nz; }
        const float2 axy = __ldg(&axy_tab[line0 + c]);
        T[c * nz1 + e] = value(axy, kx == 0 && k0 + c == 0, e - half_nz, llpc, c);
    }
    __syncthreads();

    // real part over the half lattice (see the comment above FF):
    //   kx < nx/2 : U[l] = (F(kx, ky, l) + F(kx, ky*, l*)) / 2,   kx = nx/2 : U[l] = F(kx, ky*, l*)
    const float ca = nyq_x ? 0.f : 0.5f;
    const float cb = nyq_x ? 1.f : 0.5f;
    for (int i = threadIdx.x; i < (G.nz << llpc); i += NT) {
        const int c = i >> lnz, l0 = i & (G.nz - 1);
        const int l = l0 - half_nz;
        const int ky = k0 + c;
        const int bcol = (ky == -G.ny / 2) ? LPC : c;
        const int estar = (l == -half_nz) ? G.nz : l0;      // l* = +nz/2 for l = -nz/2
        float2 u = cscale(T[bcol * nz1 + estar], cb);
        if (!nyq_x) u = cadd(u, cscale(T[c * nz1 + l0], ca));
        UA[padx(((l & (G.nz - 1)) << llpc) + c)] = u;
    }
    const bool zfold = (lnz & 3) == 1;
    block_fft_ip<PER>(UA, G.nz, LPC, +1, tw, zfold);
    if (!zfold) {
        for (int i = threadIdx.x; i < (G.nz << llpc); i += NT) {
            const int c = i >> lnz, q = i & (G.nz - 1);
            const int ky = k0 + c;
            const float sg = ((kx + ky) & 1) ? -1.f : 1.f;
            V[((size_t)kx * G.ny + (ky & (G.ny - 1))) * G.nz + q] = cscale(UA[padx((q << llpc) + c)], sg);
        }
    } else {
        // the last radix-2 pass of the z-IFFT, applied per output value
        const int hz = G.nz >> 1;
        for (int i = threadIdx.x; i < (G.nz << llpc); i += NT) {
            const int c = i >> lnz, q = i & (G.nz - 1);
            const int ky = k0 + c;
            const float sg = ((kx + ky) & 1) ? -1.f : 1.f;
            const int k = q & (hz - 1);
            const float2 s0 = UA[padx((k << llpc) + c)];
            const float2 t = cmul(twiddle(tw, k, G.nz, +1), UA[padx(((k + hz) << llpc) + c)]);
            V[((size_t)kx * G.ny + (ky & (G.ny - 1))) * G.nz + q] = cscale(q < hz ? cadd(s0, t) : csub(s0, t), sg);
        }
    }
}

// ---------------------------------------------------------------------------
// Stage (d), y part: inverse FFT along ky for one kx and C depth planes,
// written transposed as Y[kx][qz][qy].  In-place padded FFT, ny * C <= 16 NT;
// with C <= 16 both the column loads and the row stores of the padded buffer
// are free of bank conflicts.
// ---------------------------------------------------------------------------
template <int NT>
__global__ void __launch_bounds__(NT, 768 / NT) k_img_yifft(Geo G, int C, const float2* __restrict__ V,
                                                          const float2* __restrict__ tw, float2* __restrict__ Y) {
    extern __shared__ float4 smem4[];
    float2* A = reinterpret_cast<float2*>(smem4);   // [ny][C], padded
    const int kx = blockIdx.x;
    const int z0 = blockIdx.y * C;
    const int lc = ilog2(C), lny = ilog2(G.ny);
    const float2* src = V + (size_t)kx * G.ny * G.nz + z0;
#pragma unroll 8
    for (int it = threadIdx.x; it < G.ny * C; it += NT)
        A[padx(it)] = src[(size_t)(it >> lc) * G.nz + (it & (C - 1))];
    block_fft_ip<16>(A, G.ny, C, +1, tw);
    float2* dst = Y + ((size_t)kx * G.nz + z0) * G.ny;
#pragma unroll 4
    for (int it = threadIdx.x; it < G.ny * C; it += NT) {
        const int c = it >> lny;
        const int qy = it & (G.ny - 1);
        dst[it] = A[padx(qy * C + c)];
    }
}

// ---------------------------------------------------------------------------
// Stage (d), x part: complex-to-real inverse FFT of length nx from the half
// spectrum kx = 0..nx/2 (imaginary parts of kx = 0 and nx/2 dropped, i.e. the
// real part of the full inverse DFT), for one qz and C rows qy.  Uses the
// half-length complex transform: Z[k] = E[k] + i O[k],
// E = X[k] + conj X[H-k], O = (X[k] - conj X[H-k]) exp(2 pi i k / nx),
// z = IFFT_H(Z), p0[2p] = Re z[p], p0[2p+1] = Im z[p].
// The pair (k, H-k) is formed by one thread from one load of each:
// Z[H-k] = conj E[k] + i conj O[k].  In-place padded FFT, H * C <= 16 NT.
// A non-finite output value (from non-finite data, which reaches every voxel
// through the transforms) sets NEDNER_FLAG_NONFINITE in *status.
// ---------------------------------------------------------------------------
template <int NT>
__global__ void __launch_bounds__(NT, 768 / NT) k_img_xc2r(Geo G, int C, int zb, const float2* __restrict__ Y,
                                                         const float2* __restrict__ tw, float* __restrict__ p0,
                                                         int* __restrict__ status) {
    extern __shared__ float4 smem4[];
    const int H = G.nx / 2;
    float2* A = reinterpret_cast<float2*>(smem4);   // [H][C], padded
    const int qz = zb + blockIdx.x;
    const int y0 = blockIdx.y * C;
    const int lc = ilog2(C), lh = ilog2(H);
    const size_t kstride = (size_t)G.nz * G.ny;
    const float2* src = Y + (size_t)qz * G.ny + y0;
#pragma unroll 4
    for (int it = threadIdx.x; it < (H / 2 + 1) * C; it += NT) {
        const int k = it >> lc;
        const int c = it & (C - 1);
        float2 zk, zm;
        c2r_pair(src[k * kstride + c], src[(H - k) * kstride + c], k, G.nx, tw, zk, zm);
        A[padx((k << lc) + c)] = zk;
        if (k > 0 && k < H / 2) A[padx(((H - k) << lc) + c)] = zm;
    }
    block_fft_ip<16>(A, H, C, +1, tw);
    float2* dst = reinterpret_cast<float2*>(p0 + ((size_t)qz * G.ny + y0) * G.nx);
    bool bad = false;
#pragma unroll 4
    for (int it = threadIdx.x; it < H * C; it += NT) {
        const int c = it >> lh;
        const int pp = it & (H - 1);
        const float2 v = A[padx(pp * C + c)];
        bad |= !(isfinite(v.x) && isfinite(v.y));
        dst[it] = v;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, NEDNER_FLAG_NONFINITE);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t configure_fwd_kernels(const nedner_plan_s& p) {
    cudaError_t e;
    const int a = cudaFuncAttributeMaxDynamicSharedMemorySize;
#define NEDNER_ATTR_SPREAD(WT)                                                                              \
    if ((e = cudaFuncSetAttribute(k_ned_spread_xfft<WT, 16>, (cudaFuncAttribute)a, (int)p.ch.smem1))) return e; \
    if ((e = cudaFuncSetAttribute(k_ned_spread_xfft<WT, 32>, (cudaFuncAttribute)a, (int)p.ch.smem1))) return e;
    NEDNER_ATTR_SPREAD(8) NEDNER_ATTR_SPREAD(12) NEDNER_ATTR_SPREAD(16) NEDNER_ATTR_SPREAD(20)
#define NEDNER_ATTR_SPREAD2(WT)                                                                              \
    if ((e = cudaFuncSetAttribute(k_ned_spread2_xfft<WT, 256>, (cudaFuncAttribute)a, (int)p.ch.smem1))) return e; \
    if ((e = cudaFuncSetAttribute(k_ned_spread2_xfft<WT, 512>, (cudaFuncAttribute)a, (int)p.ch.smem1))) return e;
    NEDNER_ATTR_SPREAD2(8) NEDNER_ATTR_SPREAD2(12) NEDNER_ATTR_SPREAD2(16) NEDNER_ATTR_SPREAD2(20)
#undef NEDNER_ATTR_SPREAD2
#undef NEDNER_ATTR_SPREAD
    if ((e = cudaFuncSetAttribute(k_ned_spread_blocks, (cudaFuncAttribute)a, (int)p.ch.smem_s))) return e;
    if ((e = cudaFuncSetAttribute(k_ned_xfft<16>, (cudaFuncAttribute)a, (int)p.ch.smem_x))) return e;
    if ((e = cudaFuncSetAttribute(k_ned_xfft<32>, (cudaFuncAttribute)a, (int)p.ch.smem_x))) return e;
    if ((e = cudaFuncSetAttribute(k_ned_yfft<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.ch.smem2f))) return e;
    if ((e = cudaFuncSetAttribute(k_ned_yfft<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.ch.smem2f))) return e;
#define NEDNER_ATTR_NER(W, D)                                                                                   \
    if ((e = cudaFuncSetAttribute(k_ner_lines<W, D, 256>, (cudaFuncAttribute)a, (int)p.ch.smem3))) return e; \
    if ((e = cudaFuncSetAttribute(k_ner_lines<W, D, 512>, (cudaFuncAttribute)a, (int)p.ch.smem3))) return e;
    NEDNER_ATTR_NER(4, 10) NEDNER_ATTR_NER(6, 10) NEDNER_ATTR_NER(8, 10) NEDNER_ATTR_NER(10, 10)
    NEDNER_ATTR_NER(12, 10) NEDNER_ATTR_NER(14, 12) NEDNER_ATTR_NER(16, 12)
#undef NEDNER_ATTR_NER
#define NEDNER_ATTR_NER_M(MODE)                                                                                   \
    if ((e = cudaFuncSetAttribute(k_ner_lines<4, 10, 256, MODE>, (cudaFuncAttribute)a, (int)p.ch.smem3))) return e; \
    if ((e = cudaFuncSetAttribute(k_ner_lines<4, 10, 512, MODE>, (cudaFuncAttribute)a, (int)p.ch.smem3))) return e;
    NEDNER_ATTR_NER_M(NEDNER_NER_LINEAR_S2) NEDNER_ATTR_NER_M(NEDNER_NER_LINEAR_S1) NEDNER_ATTR_NER_M(NEDNER_NER_DIRECT)
#undef NEDNER_ATTR_NER_M
    if ((e = cudaFuncSetAttribute(k_img_yifft<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.ch.smem4)))
        return e;
    if ((e = cudaFuncSetAttribute(k_img_xc2r<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.ch.smem5)))
        return e;
    return cudaSuccess;
}

cudaError_t launch_ned_spread_xfft(const nedner_plan_s& p, const float* g, float2* R, cudaStream_t s, int t0,
                                   int nt) {
    const Geo& G = p.geo;
    if (nt < 0) nt = G.Nt - t0;
    const int yb = t0 / p.ch.c1;
    dim3 grid(G.Ly, nt / p.ch.c1);
#define NEDNER_SPREAD(WT)                                                                                        \
    if (p.ch.tpl1 == 2 && p.ch.threads1 <= 256)                                                                  \
        k_ned_spread2_xfft<WT, 256><<<grid, 256, p.ch.smem1, s>>>(G, yb, g, p.t.seg, p.t.xent_m, p.t.xent_wx,   \
                                                                  p.t.xent_bx, p.t.deconv_x, p.t.tw, R);         \
    else if (p.ch.tpl1 == 2)                                                                                     \
        k_ned_spread2_xfft<WT, 512><<<grid, 512, p.ch.smem1, s>>>(G, yb, g, p.t.seg, p.t.xent_m, p.t.xent_wx,   \
                                                                  p.t.xent_bx, p.t.deconv_x, p.t.tw, R);         \
    else if (p.ch.per1 <= 16)                                                                                    \
        k_ned_spread_xfft<WT, 16><<<grid, 256, p.ch.smem1, s>>>(G, p.ch.c1, yb, g, p.t.seg, p.t.xent_m,         \
                                                                p.t.xent_wx, p.t.xent_bx, p.t.deconv_x, p.t.tw, R); \
    else                                                                                                         \
        k_ned_spread_xfft<WT, 32><<<grid, 256, p.ch.smem1, s>>>(G, p.ch.c1, yb, g, p.t.seg, p.t.xent_m,         \
                                                                p.t.xent_wx, p.t.xent_bx, p.t.deconv_x, p.t.tw, R)
    switch (spread_taps(G.w)) {
        case 8: NEDNER_SPREAD(8); break;
        case 12: NEDNER_SPREAD(12); break;
        case 16: NEDNER_SPREAD(16); break;
        default: NEDNER_SPREAD(20); break;
    }
#undef NEDNER_SPREAD
    return cudaGetLastError();
}

cudaError_t launch_ned_yfft(const nedner_plan_s& p, const float2* R, float2* Ghat, cudaStream_t s, int t0, int nt,
                            int rstride, int roff) {
    const Geo& G = p.geo;
    if (nt < 0) nt = G.Nt - t0;
    if (rstride < 0) rstride = G.Nt;
    const int yb = t0 / p.ch.c2f;
    dim3 grid(nt / p.ch.c2f, G.nxh);
    if ((long)G.Ly * p.ch.c2f <= 16L * 256)
        k_ned_yfft<16><<<grid, 256, p.ch.smem2f, s>>>(G, p.ch.c2f, yb, R, rstride, roff, p.t.deconv_y, p.t.tw, Ghat);
    else
        k_ned_yfft<32><<<grid, 256, p.ch.smem2f, s>>>(G, p.ch.c2f, yb, R, rstride, roff, p.t.deconv_y, p.t.tw, Ghat);
    return cudaGetLastError();
}

cudaError_t launch_ned_spread_blocks(const nedner_plan_s& p, const float* g, float* Q, int t0, cudaStream_t s) {
    const Geo& G = p.geo;
    const int tq = p.ch.tq, wpc = p.ch.wpc_s;
    const dim3 grid(G.Ly * (G.Lx / 16) / wpc, tq / 64);
    k_ned_spread_blocks<<<grid, 32 * wpc, p.ch.smem_s, s>>>(G, t0, tq, g, p.t.bseg, p.t.bent_m, p.t.bent_w, Q);
    return cudaGetLastError();
}

cudaError_t launch_ned_xfft(const nedner_plan_s& p, const float* Q, float2* R, cudaStream_t s) {
    const Geo& G = p.geo;
    const dim3 grid(G.Ly, p.ch.tq / (2 * p.ch.nbx));
    if (p.ch.perx <= 16)
        k_ned_xfft<16><<<grid, p.ch.thx, p.ch.smem_x, s>>>(G, p.ch.tq, p.ch.nbx, Q, p.t.deconv_x, p.t.tw, R);
    else
        k_ned_xfft<32><<<grid, p.ch.thx, p.ch.smem_x, s>>>(G, p.ch.tq, p.ch.nbx, Q, p.t.deconv_x, p.t.tw, R);
    return cudaGetLastError();
}

// Stage (a) as spread, x-FFT and y-FFT per chunk of tq time samples, Q and R
// holding one chunk; a timer, if given, is marked after each launch (stages 0,
// 1 and 2: spread, x-FFT, y-FFT, summed over the chunks).
cudaError_t launch_ned_stage_split(const nedner_plan_s& p, const float* g, float* Q, float2* R, float2* Ghat,
                                   cudaStream_t s, StageTimer* tm) {
    const Geo& G = p.geo;
    cudaError_t e = cudaSuccess;
    for (int t0 = 0; t0 < G.Nt && !e; t0 += p.ch.tq) {
        if ((e = launch_ned_spread_blocks(p, g, Q, t0, s))) break;
        stage_mark(tm, 0);
        if ((e = launch_ned_xfft(p, Q, R, s))) break;
        stage_mark(tm, 1);
        if ((e = launch_ned_yfft(p, R, Ghat, s, t0, p.ch.tq, p.ch.tq, t0))) break;
        stage_mark(tm, 2);
    }
    return e;
}

cudaError_t launch_ner_lines(const nedner_plan_s& p, const float2* Ghat, float2* V, cudaStream_t s) {
    const Geo& G = p.geo;
    dim3 grid(G.nxh * (G.ny / p.ch.lpc));
#define NEDNER_NER(W, D)                                                                                      \
    if (p.ch.threads3 <= 256)                                                                                 \
        k_ner_lines<W, D, 256><<<grid, 256, p.ch.smem3, s>>>(G, p.tap, p.ch.lpc, Ghat, p.t.axy, p.t.deconv_t, \
                                                             p.t.tw, V);                                      \
    else                                                                                                      \
        k_ner_lines<W, D, 512><<<grid, 512, p.ch.smem3, s>>>(G, p.tap, p.ch.lpc, Ghat, p.t.axy, p.t.deconv_t, \
                                                             p.t.tw, V)
#define NEDNER_NER_M(MODE)                                                                                    \
    if (p.ch.threads3 <= 256)                                                                                 \
        k_ner_lines<4, 10, 256, MODE><<<grid, 256, p.ch.smem3, s>>>(G, p.tap, p.ch.lpc, Ghat, p.t.axy,         \
                                                                    p.t.deconv_t, p.t.tw, V);                 \
    else                                                                                                      \
        k_ner_lines<4, 10, 512, MODE><<<grid, 512, p.ch.smem3, s>>>(G, p.tap, p.ch.lpc, Ghat, p.t.axy,         \
                                                                    p.t.deconv_t, p.t.tw, V)
    if (p.ner_interp == NEDNER_NER_LINEAR_S2) {
        NEDNER_NER_M(NEDNER_NER_LINEAR_S2);
    } else if (p.ner_interp == NEDNER_NER_LINEAR_S1) {
        NEDNER_NER_M(NEDNER_NER_LINEAR_S1);
    } else if (p.ner_interp == NEDNER_NER_DIRECT) {
        NEDNER_NER_M(NEDNER_NER_DIRECT);
    } else {
        switch (G.w) {
            case 4: NEDNER_NER(4, 10); break;
            case 6: NEDNER_NER(6, 10); break;
            case 8: NEDNER_NER(8, 10); break;
            case 10: NEDNER_NER(10, 10); break;
            case 12: NEDNER_NER(12, 10); break;
            case 14: NEDNER_NER(14, 12); break;
            default: NEDNER_NER(16, 12); break;
        }
    }
#undef NEDNER_NER_M
#undef NEDNER_NER
    return cudaGetLastError();
}

cudaError_t launch_img_yifft(const nedner_plan_s& p, const float2* V, float2* Y, cudaStream_t s) {
    const Geo& G = p.geo;
    dim3 grid(G.nxh, G.nz / p.ch.c4);
    k_img_yifft<128><<<grid, 128, p.ch.smem4, s>>>(G, p.ch.c4, V, p.t.tw, Y);
    return cudaGetLastError();
}

cudaError_t launch_img_xc2r(const nedner_plan_s& p, const float2* Y, float* p0, cudaStream_t s, int z0, int nzc) {
    const Geo& G = p.geo;
    if (nzc < 0) nzc = G.nz - z0;
    dim3 grid(nzc, G.ny / p.ch.c5);
    k_img_xc2r<128><<<grid, 128, p.ch.smem5, s>>>(G, p.ch.c5, z0, Y, p.t.tw, p0, p.t.status);
    return cudaGetLastError();
}

}  // namespace nedner

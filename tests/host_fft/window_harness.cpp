// Runs the register-window helpers of the spread (spread_window.cuh) and of
// the transposed gather (gather_window.cuh) on the host for tests.
//  - host_sweep: every lane of one lane group sweeps the entries of a column
//    segment [c0, c1) exactly as the spread kernels do (window base,
//    retirement of the lower WT columns, taps added at offset bx4 - base),
//    writing finished columns into the padded row buffer, returned in linear
//    layout (NaN where the sweep wrote nothing).
//  - host_gather: every lane walks a run of entries exactly as the gather
//    kernels do and returns each entry's two tap-weighted sums of the row
//    (read modulo Lx).
// Test infrastructure only.
#include <cmath>
#include <cstring>
#include <vector>

#include "gather_window.cuh"
#include "spread_window.cuh"

thread_local HostDim3 threadIdx;
HostDim3 blockDim;
void __syncthreads() {}

using namespace nedner;

// Two time samples per lane (32 lanes, 64 samples): g is [nent][64].
template <int WT>
static void sweep2(int Lx, int c0, int c1, int nent, const int* bx4, const float* taps, const float* g,
                   float* out) {
    std::vector<float2> Z((size_t)padded_len(Lx * 32) + 16, make_float2(NAN, NAN));
    for (int ln = 0; ln < 32; ++ln) {
        float2 acc[2 * WT];
        for (int k = 0; k < 2 * WT; ++k) acc[k] = make_float2(0.f, 0.f);
        int base = (c0 - WT) & ~3;
        for (int e = 0; e < nent; ++e) {
            float4 wv[WT / 4];
            for (int k4 = 0; k4 < WT / 4; ++k4)
                wv[k4] = float4{taps[e * WT + 4 * k4], taps[e * WT + 4 * k4 + 1], taps[e * WT + 4 * k4 + 2],
                                taps[e * WT + 4 * k4 + 3]};
            const float2 g2 = make_float2(g[e * 64 + 2 * ln], g[e * 64 + 2 * ln + 1]);
            sweep_entry2<WT>(acc, Z.data(), ln, base, c0, c1, bx4[e], wv, g2);
        }
        while (base < c1) {
            flush_lower2<WT>(acc, Z.data(), ln, base, c0, c1);
            base += WT;
        }
    }
    for (int col = 0; col < Lx; ++col)
        for (int ln = 0; ln < 32; ++ln) {
            const float2 v = Z[padx(col * 32 + ln)];
            out[(col * 32 + ln) * 2] = v.x;
            out[(col * 32 + ln) * 2 + 1] = v.y;
        }
}

// One time sample per lane (C lanes, C a power of two >= 2): g is [nent][C].
template <int WT>
static void sweep1(int Lx, int C, int c0, int c1, int nent, const int* bx4, const float* taps, const float* g,
                   float* out) {
    const int nb = C / 2, lnb = ilog2(nb);
    std::vector<float2> Z((size_t)padded_len(Lx * nb) + 16, make_float2(NAN, NAN));
    float* Zf = reinterpret_cast<float*>(Z.data());
    for (int hl = 0; hl < C; ++hl) {
        float acc[2 * WT];
        for (int k = 0; k < 2 * WT; ++k) acc[k] = 0.f;
        int base = (c0 - WT) & ~3;
        for (int e = 0; e < nent; ++e) {
            float4 wv[WT / 4];
            for (int k4 = 0; k4 < WT / 4; ++k4)
                wv[k4] = float4{taps[e * WT + 4 * k4], taps[e * WT + 4 * k4 + 1], taps[e * WT + 4 * k4 + 2],
                                taps[e * WT + 4 * k4 + 3]};
            sweep_entry<WT>(acc, Zf, lnb, hl, base, c0, c1, bx4[e], wv, g[e * C + hl]);
        }
        while (base < c1) {
            flush_lower<WT>(acc, Zf, lnb, hl, base, c0, c1);
            base += WT;
        }
    }
    for (int col = 0; col < Lx; ++col)
        for (int hl = 0; hl < C; ++hl) out[col * C + hl] = Zf[2 * padx((col << lnb) + (hl >> 1)) + (hl & 1)];
}

extern "C" int host_sweep(int two, int WT, int Lx, int C, int c0, int c1, int nent, const int* bx4,
                          const float* taps, const float* g, float* out) {
    if (c0 < 0 || c1 > Lx || c0 > c1) return -1;
    if (two) {
        switch (WT) {
            case 8: sweep2<8>(Lx, c0, c1, nent, bx4, taps, g, out); return 0;
            case 12: sweep2<12>(Lx, c0, c1, nent, bx4, taps, g, out); return 0;
            case 16: sweep2<16>(Lx, c0, c1, nent, bx4, taps, g, out); return 0;
            case 20: sweep2<20>(Lx, c0, c1, nent, bx4, taps, g, out); return 0;
        }
        return -1;
    }
    if (C < 2 || (C & (C - 1))) return -1;
    switch (WT) {
        case 8: sweep1<8>(Lx, C, c0, c1, nent, bx4, taps, g, out); return 0;
        case 12: sweep1<12>(Lx, C, c0, c1, nent, bx4, taps, g, out); return 0;
        case 16: sweep1<16>(Lx, C, c0, c1, nent, bx4, taps, g, out); return 0;
        case 20: sweep1<20>(Lx, C, c0, c1, nent, bx4, taps, g, out); return 0;
    }
    return -1;
}

// row: [Lx][lanes] real samples (lanes = 64 with two per lane, else C);
// out_a, out_b: [nent][lanes].
template <int WT>
static void gather2(int Lx, int nent, const int* bx4, const float* ta, const float* tb, const float* row,
                    float* out_a, float* out_b) {
    std::vector<float2> Z((size_t)padded_len(Lx * 32) + 16, make_float2(NAN, NAN));
    for (int col = 0; col < Lx; ++col)
        for (int ln = 0; ln < 32; ++ln) Z[padx(col * 32 + ln)] = make_float2(row[col * 64 + 2 * ln], row[col * 64 + 2 * ln + 1]);
    for (int ln = 0; ln < 32; ++ln) {
        float2 win[2 * WT];
        int base = bx4[0];
        win2_load<WT>(win, Z.data(), ln, Lx, base, 0);
        win2_load<WT>(win, Z.data(), ln, Lx, base, WT);
        for (int j = 0; j < nent; ++j) {
            win2_advance<WT>(win, Z.data(), ln, Lx, base, bx4[j]);
            float2 va, vb;
            win2_entry<WT, true>(win, (bx4[j] - base) >> 2, reinterpret_cast<const float4*>(ta + j * WT),
                                 reinterpret_cast<const float4*>(tb + j * WT), va, vb);
            out_a[j * 64 + 2 * ln] = va.x;
            out_a[j * 64 + 2 * ln + 1] = va.y;
            out_b[j * 64 + 2 * ln] = vb.x;
            out_b[j * 64 + 2 * ln + 1] = vb.y;
        }
    }
}

template <int WT>
static void gather1(int Lx, int C, int nent, const int* bx4, const float* ta, const float* tb, const float* row,
                    float* out_a, float* out_b) {
    const int nb = C / 2, lnb = ilog2(nb);
    std::vector<float2> Z((size_t)padded_len(Lx * nb) + 16, make_float2(NAN, NAN));
    float* Zf = reinterpret_cast<float*>(Z.data());
    for (int col = 0; col < Lx; ++col)
        for (int ln = 0; ln < C; ++ln) Zf[rpos(col, lnb, ln)] = row[col * C + ln];
    for (int ln = 0; ln < C; ++ln) {
        float win[2 * WT];
        int base = bx4[0];
        win_load<WT>(win, Zf, lnb, ln, Lx, base, 0);
        win_load<WT>(win, Zf, lnb, ln, Lx, base, WT);
        for (int j = 0; j < nent; ++j) {
            win_advance<WT>(win, Zf, lnb, ln, Lx, base, bx4[j]);
            const float2 v = win_entry<WT, true>(win, (bx4[j] - base) >> 2, reinterpret_cast<const float4*>(ta + j * WT),
                                                 reinterpret_cast<const float4*>(tb + j * WT));
            out_a[j * C + ln] = v.x;
            out_b[j * C + ln] = v.y;
        }
    }
}

extern "C" int host_gather(int two, int WT, int Lx, int C, int nent, const int* bx4, const float* ta, const float* tb,
                           const float* row, float* out_a, float* out_b) {
    if (nent < 1 || Lx < 8 || (Lx & (Lx - 1))) return -1;
    if (!two && (C < 2 || (C & (C - 1)))) return -1;
#define NEDNER_HOST_GATHER(W)                                                   \
    if (two) gather2<W>(Lx, nent, bx4, ta, tb, row, out_a, out_b);             \
    else gather1<W>(Lx, C, nent, bx4, ta, tb, row, out_a, out_b);              \
    return 0;
    switch (WT) {
        case 8: NEDNER_HOST_GATHER(8)
        case 12: NEDNER_HOST_GATHER(12)
        case 16: NEDNER_HOST_GATHER(16)
        case 20: NEDNER_HOST_GATHER(20)
    }
#undef NEDNER_HOST_GATHER
    return -1;
}

// The spread stage's output step for one row: Zin is the row after the x-FFT
// (with fold, before its last radix-2 pass), linear [Lx][nb] interleaved
// complex; out is R for that row, [nxh][2 nb] complex (time samples 2b, 2b+1).
extern "C" int host_spread_output(int Lx, int nb, int fold, const float* Zin, const float* deconv_x, float* out) {
    if (Lx < 8 || (Lx & (Lx - 1)) || nb < 1 || (nb & (nb - 1)) || Lx > TW_N) return -1;
    std::vector<float2> tw(2 * TW_N);
    tw[0] = make_float2(1.f, 0.f);
    for (int N = 1; N <= TW_N; N *= 2)
        for (int k = 0; k < N; ++k) {
            const double a = -2.0 * 3.14159265358979323846 * (double)k / N;
            tw[N + k] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
    Geo G;
    std::memset(&G, 0, sizeof(G));
    G.Lx = Lx;
    G.nx = Lx / 2;
    G.nxh = Lx / 4 + 1;
    G.Ly = 1;
    G.Nt = 2 * nb;
    std::vector<float2> Z((size_t)padded_len(Lx * nb) + 16);
    for (int a = 0; a < Lx * nb; ++a) Z[padx(a)] = make_float2(Zin[2 * a], Zin[2 * a + 1]);
    std::vector<float2> R((size_t)G.nxh * G.Nt);
    const int lnb = ilog2(nb);
    for (int jx = 0; jx < G.nxh; ++jx)
        for (int b = 0; b < nb; ++b) spread_output(G, Z.data(), lnb, b, jx, fold != 0, deconv_x, tw.data(), 0, 0, R.data());
    for (size_t i = 0; i < R.size(); ++i) {
        out[2 * i] = R[i].x;
        out[2 * i + 1] = R[i].y;
    }
    return 0;
}

// The block spread (block_taps16 + block_entry16): the 32 lanes of a warp accumulate the
// 16-column block [c0, c0 + 16) over the entries whose W taps (from their
// exact first column bx, taps [nent][4 ceil(W/4)]) reach into it; g is
// [nent][64].  out: [16][64] (column, time sample).
template <int W>
static void block_sweep(int c0, int nent, const int* bx, const float* taps, const float* g, float* out) {
    constexpr int WQ = (W + 3) / 4;
    for (int ln = 0; ln < 32; ++ln) {
        float2 acc[16];
        for (int k = 0; k < 16; ++k) acc[k] = make_float2(0.f, 0.f);
        for (int e = 0; e < nent; ++e) {
            // the plan's table entry: the taps aligned to the block's columns
            float t16[16];
            block_taps16(bx[e], c0, taps + e * 4 * WQ, W, t16);
            float4 t[4];
            for (int c4 = 0; c4 < 4; ++c4) t[c4] = float4{t16[4 * c4], t16[4 * c4 + 1], t16[4 * c4 + 2], t16[4 * c4 + 3]};
            block_entry16(acc, t, make_float2(g[e * 64 + 2 * ln], g[e * 64 + 2 * ln + 1]));
        }
        for (int k = 0; k < 16; ++k) {
            out[k * 64 + 2 * ln] = acc[k].x;
            out[k * 64 + 2 * ln + 1] = acc[k].y;
        }
    }
}

extern "C" int host_block_sweep(int W, int c0, int nent, const int* bx, const float* taps, const float* g,
                                float* out) {
    switch (W) {
        case 4: block_sweep<4>(c0, nent, bx, taps, g, out); return 0;
        case 6: block_sweep<6>(c0, nent, bx, taps, g, out); return 0;
        case 8: block_sweep<8>(c0, nent, bx, taps, g, out); return 0;
        case 10: block_sweep<10>(c0, nent, bx, taps, g, out); return 0;
        case 12: block_sweep<12>(c0, nent, bx, taps, g, out); return 0;
        case 14: block_sweep<14>(c0, nent, bx, taps, g, out); return 0;
        case 16: block_sweep<16>(c0, nent, bx, taps, g, out); return 0;
    }
    return -1;
}

// Plan construction and the C-ABI entry points of include/nedner.h.
//
// The plan precomputes, once per geometry (the "precomputed Psi" of Sec. 5,
// Table 2: reusing the window tables across reconstructions), in FP64 on the
// host: the per-sensor window taps and grid offsets of the NED-NUFFT
// (Eq. NED_NUFFT), the row lists that let each CTA gather the sensors of its
// grid row, the deconvolution tables 1/phihat of both NUFFTs (Eq. PSI), the
// tap polynomials of the NER interpolation, and the lateral part of nu^2 for
// every line.  It then allocates the device workspace.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "fft.cuh"
#include "spread_window.cuh"
#include "internal.h"

// Stage timer for the profiled entry points: records a CUDA event on the
// stream after each launch and adds the time since the previous mark to the
// stage it names (a stage launched several times, e.g. once per pass, sums).
namespace nedner {

struct StageTimer {
    cudaStream_t s;
    std::vector<std::pair<int, cudaEvent_t>> marks;
    cudaError_t err = cudaSuccess;
    explicit StageTimer(cudaStream_t st) : s(st) {}
    void mark(int stage) {
        cudaEvent_t ev = nullptr;
        if (err == cudaSuccess) err = cudaEventCreate(&ev);
        if (err == cudaSuccess) err = cudaEventRecord(ev, s);
        if (ev) marks.emplace_back(stage, ev);
    }
    // waits for the last mark; ms[stage] += elapsed since the previous mark
    cudaError_t finish(float* ms, int nstages) {
        for (int k = 0; k < nstages; ++k) ms[k] = 0.f;
        if (err == cudaSuccess && !marks.empty()) err = cudaEventSynchronize(marks.back().second);
        for (size_t i = 1; i < marks.size() && err == cudaSuccess; ++i) {
            float t = 0.f;
            err = cudaEventElapsedTime(&t, marks[i - 1].second, marks[i].second);
            if (marks[i].first >= 0 && marks[i].first < nstages) ms[marks[i].first] += t;
        }
        for (auto& m : marks) cudaEventDestroy(m.second);
        marks.clear();
        return err;
    }
};

void stage_mark(StageTimer* tm, int stage) {
    if (tm) tm->mark(stage);
}

}  // namespace nedner

using namespace nedner;

namespace {

const double kPi = 3.14159265358979323846264338327950288;

bool is_pow2(long v) { return v > 0 && (v & (v - 1)) == 0; }

template <typename T>
cudaError_t upload(T** dptr, const std::vector<T>& h, cudaStream_t s) {
    if (h.empty()) {
        *dptr = nullptr;
        return cudaSuccess;
    }
    cudaError_t e = cudaMalloc((void**)dptr, h.size() * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(*dptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

void free_sensor_tables(DevTables& t) {
    cudaFree(t.sens_bx); cudaFree(t.sens_by); cudaFree(t.sens_wx); cudaFree(t.sens_wy);
    cudaFree(t.sens_dwx); cudaFree(t.sens_dwy); cudaFree(t.sens_fac);
    cudaFree(t.row_ptr); cudaFree(t.row_m); cudaFree(t.row_w); cudaFree(t.row_dw);
    cudaFree(t.xrow_ptr); cudaFree(t.xent_m); cudaFree(t.xent_wx); cudaFree(t.xent_bx); cudaFree(t.seg);
    cudaFree(t.xent_gx); cudaFree(t.xent_gy); cudaFree(t.xrow_first);
    cudaFree(t.xent_rc); cudaFree(t.sens_ent);
    cudaFree(t.bseg); cudaFree(t.bent_m); cudaFree(t.bent_w); cudaFree(t.pent_bx); cudaFree(t.pent_w);
    cudaFree(t.pent_gx); cudaFree(t.pent_gy); cudaFree(t.gseg); cudaFree(t.lp_kcut);
    t.bseg = nullptr; t.bent_m = nullptr; t.bent_w = nullptr; t.pent_bx = nullptr; t.pent_w = nullptr;
    t.pent_gx = nullptr; t.pent_gy = nullptr; t.gseg = nullptr; t.lp_kcut = nullptr;
    t.sens_bx = t.sens_by = nullptr;
    t.sens_wx = t.sens_wy = t.sens_dwx = t.sens_dwy = t.sens_fac = nullptr;
    t.row_ptr = t.row_m = nullptr;
    t.row_w = t.row_dw = nullptr;
    t.xrow_ptr = t.xent_m = t.xent_bx = nullptr;
    t.xent_wx = nullptr;
    t.xent_gx = t.xent_gy = nullptr;
    t.xrow_first = t.xent_rc = t.sens_ent = nullptr;
    t.seg = nullptr;
}

void free_tp(TPState& tp) {
    cudaFree(tp.work); cudaFree(tp.ex); cudaFree(tp.ey); cudaFree(tp.exn); cudaFree(tp.eyf); cudaFree(tp.err);
    cudaFree(tp.absmax);
    tp = TPState();
}

// host BF16 (round to nearest even) and the hi + lo split of a float
uint16_t f2bf(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float bf2f(uint16_t h) {
    uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// host FP16 (round to nearest even, subnormals kept) through the CUDA header's conversion
uint16_t f2h(float f) {
    const __half h = __float2half_rn(f);
    uint16_t u;
    std::memcpy(&u, &h, 2);
    return u;
}
float h2f(uint16_t u) {
    __half h;
    std::memcpy(&h, &u, 2);
    return __half2float(h);
}

// the hi + lo split of an exponent factor in the plan's operand type
void split16(float x, bool fp16, uint16_t& hi, uint16_t& lo) {
    if (fp16) {
        hi = f2h(x);
        lo = f2h(x - h2f(hi));
    } else {
        hi = f2bf(x);
        lo = f2bf(x - bf2f(hi));
    }
}

// element offset of (r, k) in a chunked K-major operand matrix (K chunks of 64)
size_t tp_off(int r, int k, int rows) {
    const int c = k >> 6, kk = k & 63;
    return (size_t)c * rows * 64 + (size_t)(((r >> 3) * 8 + (kk >> 3)) << 6) + ((r & 7) << 3) + (kk & 7);
}

// Tensor-product path: check the layout and build the exponent operands.
nedner_status build_tp(nedner_plan_s& p, cudaStream_t s, bool fp16) {
    const int NS = TP_SENSORS;
    const Geo& G = p.geo;
    if (p.M != (int64_t)NS * NS || G.nx != 2 * NS || G.ny != 2 * NS) return NEDNER_EINVAL;
    const double X = p.grid.nx * p.grid.dx, Y = p.grid.ny * p.grid.dy;
    std::vector<double> xs(NS), ys(NS);
    for (int a = 0; a < NS; ++a) xs[a] = p.xy[2 * a];
    for (int b = 0; b < NS; ++b) ys[b] = p.xy[2 * (size_t)b * NS + 1];
    for (int b = 0; b < NS; ++b)
        for (int a = 0; a < NS; ++a) {
            const size_t m = (size_t)b * NS + a;
            if (std::fabs(p.xy[2 * m] - xs[a]) > 1e-12 * X || std::fabs(p.xy[2 * m + 1] - ys[b]) > 1e-12 * Y)
                return NEDNER_EINVAL;
        }
    const size_t MATE = (size_t)NS * NS;               // elements of a 128-row matrix
    if (G.Nt < 128) return NEDNER_EINVAL;               // GEMM 2 tiles hold 128 time samples
    std::vector<uint16_t> ex(4 * MATE), ey(2 * 4 * MATE, 0);
    for (int jx = 0; jx < NS; ++jx)
        for (int a = 0; a < NS; ++a) {
            const double ph = -2.0 * kPi * (double)jx * xs[a] / X;
            const float re = (float)std::cos(ph), im = (float)std::sin(ph);
            const size_t o = tp_off(jx, a, NS);
            split16(re, fp16, ex[0 * MATE + o], ex[1 * MATE + o]);
            split16(im, fp16, ex[2 * MATE + o], ex[3 * MATE + o]);
        }
    // Ey as GEMM 2's A operand: two M tiles (jy = -128..-1, 0..127), 4 matrices each
    for (int t = 0; t < 2; ++t)
        for (int r = 0; r < NS; ++r) {
            const int jy = (t == 0) ? r - NS : r;
            for (int b = 0; b < NS; ++b) {
                const double ph = -2.0 * kPi * (double)jy * ys[b] / Y;
                const float re = (float)std::cos(ph), im = (float)std::sin(ph);
                const size_t o = (size_t)t * 4 * MATE + tp_off(r, b, NS);
                split16(re, fp16, ey[o + 0 * MATE], ey[o + 1 * MATE]);
                split16(im, fp16, ey[o + 2 * MATE], ey[o + 3 * MATE]);
            }
        }
    std::vector<float2> exn(NS), eyf((size_t)G.nyp * NS);
    for (int a = 0; a < NS; ++a) {
        const double ph = -2.0 * kPi * (double)(G.nx / 2) * xs[a] / X;
        exn[a] = make_float2((float)std::cos(ph), (float)std::sin(ph));
    }
    for (int bj = 0; bj < G.nyp; ++bj)
        for (int b = 0; b < NS; ++b) {
            const double ph = -2.0 * kPi * (double)(bj - G.ny / 2) * ys[b] / Y;
            eyf[(size_t)bj * NS + b] = make_float2((float)std::cos(ph), (float)std::sin(ph));
        }
    TPState& tp = p.tp;
    cudaError_t e = cudaSuccess;
    int dev = 0;
    if (!e) e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&tp.sms, cudaDevAttrMultiProcessorCount, dev);
    uint16_t* dex = nullptr;
    uint16_t* dey = nullptr;
    if (!e) e = upload(&dex, ex, s);
    if (!e) e = upload(&dey, ey, s);
    tp.ex = dex;
    tp.ey = dey;
    if (!e) e = upload(&tp.exn, exn, s);
    if (!e) e = upload(&tp.eyf, eyf, s);
    tp.work_bytes = tp_work_bytes(G.Nt);
    if (!e) e = cudaMalloc(&tp.work, tp.work_bytes);
    if (!e) e = cudaMalloc((void**)&tp.err, sizeof(int));
    if (!e) e = cudaMemsetAsync(tp.err, 0, sizeof(int), s);
    if (!e && fp16) e = cudaMalloc((void**)&tp.absmax, sizeof(unsigned int));
    if (!e) e = configure_tp_kernels();
    if (!e) e = cudaStreamSynchronize(s);
    if (e) {
        cudaGetLastError();
        free_tp(tp);
        return e == cudaErrorMemoryAllocation ? NEDNER_ENOMEM : NEDNER_ECUDA;
    }
    tp.enabled = 1;
    tp.fp16 = fp16 ? 1 : 0;
    return NEDNER_OK;
}

void free_tables(DevTables& t) {
    cudaFree(t.tw); cudaFree(t.deconv_x); cudaFree(t.deconv_y); cudaFree(t.deconv_t);
    cudaFree(t.tapcoef); cudaFree(t.axy); cudaFree(t.status);
    t.tw = nullptr; t.deconv_x = t.deconv_y = t.deconv_t = t.tapcoef = nullptr; t.axy = nullptr;
    t.status = nullptr;
    free_sensor_tables(t);
}

nedner_status check_positions(const nedner_plan_s& p, const double* xy) {
    const double X = p.grid.nx * p.grid.dx, Y = p.grid.ny * p.grid.dy;
    for (int64_t m = 0; m < p.M; ++m) {
        double x = xy[2 * m], y = xy[2 * m + 1];
        if (!std::isfinite(x) || !std::isfinite(y)) return NEDNER_EINVAL;
        if (!(x > -0.5 * X && x < 0.5 * X && y > -0.5 * Y && y < 0.5 * Y)) return NEDNER_ERANGE;
    }
    return NEDNER_OK;
}

// Per-sensor taps and the row lists (Sec. 3.2: mu_{m,k} are the w grid
// points nearest u_m = x_m Lx / X, the weights phi(u_m - mu)).
//
// Three views of the (sensor, y tap) entries are built:
//  - row CSR: the entries of each grid row (transposed interpolation);
//  - per row, the entries sorted by their first x column, entries that wrap
//    around x = Lx repeated at bx - Lx, and each row cut into groups1 column
//    segments of about equal entry count (spreading: every lane group of a CTA
//    owns one segment and writes it without atomics);
//  - per sensor, the row-CSR indices of its w entries (the transposed kernels
//    write one value per entry and then sum each sensor's entries).
nedner_status build_sensor_tables(nedner_plan_s& p, cudaStream_t s) {
    const Geo& G = p.geo;
    const Chunks& C = p.ch;
    const int64_t M = p.M;
    const int w = G.w;
    const double X = p.grid.nx * p.grid.dx, Y = p.grid.ny * p.grid.dy;
    std::vector<int> bx(M), by(M);
    std::vector<float> wx(M * w), wy(M * w), dwx(M * w), dwy(M * w), fac(M);
    for (int64_t m = 0; m < M; ++m) {
        double ux = p.xy[2 * m] / X * G.Lx, uy = p.xy[2 * m + 1] / Y * G.Ly;
        double fx = std::floor(ux), fy = std::floor(uy);
        long b0x = (long)fx - w / 2 + 1, b0y = (long)fy - w / 2 + 1;
        bx[m] = (int)(((b0x % G.Lx) + G.Lx) % G.Lx);
        by[m] = (int)(((b0y % G.Ly) + G.Ly) % G.Ly);
        for (int k = 0; k < w; ++k) {
            double ax = ux - (double)(b0x + k), ay = uy - (double)(b0y + k);
            wx[m * w + k] = (float)win_phi(p.win, ax);
            wy[m * w + k] = (float)win_phi(p.win, ay);
            dwx[m * w + k] = (float)(win_dphi(p.win, ax) * G.Lx / X);
            dwy[m * w + k] = (float)(win_dphi(p.win, ay) * G.Ly / Y);
        }
        fac[m] = (float)(G.apply_weights ? p.h[m] / (p.grid.dx * p.grid.dy) : 1.0);
    }
    // row CSR: entry (m, k) lands in row (by_m + k) mod Ly
    std::vector<int> row_ptr(G.Ly + 1, 0);
    for (int64_t m = 0; m < M; ++m)
        for (int k = 0; k < w; ++k) row_ptr[((by[m] + k) & (G.Ly - 1)) + 1]++;
    for (int r = 0; r < G.Ly; ++r) row_ptr[r + 1] += row_ptr[r];
    std::vector<int> fill(row_ptr.begin(), row_ptr.end() - 1);
    const size_t E = (size_t)M * w;
    std::vector<int> row_m(E), sens_ent(E);
    std::vector<float> row_w(E), row_dw(E);
    for (int64_t m = 0; m < M; ++m)
        for (int k = 0; k < w; ++k) {
            int r = (by[m] + k) & (G.Ly - 1);
            int e = fill[r]++;
            sens_ent[m * w + k] = e;
            row_m[e] = (int)m;
            row_w[e] = wy[m * w + k] * fac[m];
            row_dw[e] = dwy[m * w + k] * fac[m];
        }

    // spreading view: sorted by first x column, wrapped entries repeated
    struct XE { int bx, m; float w, dw; int e; };
    std::vector<int> xrow_ptr(G.Ly + 1, 0);
    std::vector<int> xent_m, xent_bx, xent_e;
    std::vector<float> xent_wx, xent_gx, xent_gy;
    std::vector<int4> seg((size_t)G.Ly * C.groups1);
    // block spread (split1): exact first column and w taps per entry, and per
    // (row, 16-column block) the range of entries reaching into the block
    const int PW = (w + 3) / 4 * 4;
    const int nblk = G.Lx / 16;
    std::vector<int> pent_bx;
    std::vector<float> pent_w, pent_gx, pent_gy;
    std::vector<int2> bseg(C.split1 ? (size_t)G.Ly * nblk : 0);
    std::vector<int> bent_m;           // per (row, block): the sensors of the entries reaching into it
    std::vector<float> bent_w;         // and their taps aligned to the block's columns, [.][16]
    std::vector<int2> gseg(C.split1 ? (size_t)G.Ly * nblk : 0);
    std::vector<XE> tmp;
    for (int r = 0; r < G.Ly; ++r) {
        tmp.clear();
        for (int e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
            int m = row_m[e];
            tmp.push_back({bx[m], m, row_w[e], row_dw[e], e});
            if (bx[m] > G.Lx - w) tmp.push_back({bx[m] - G.Lx, m, row_w[e], row_dw[e], e});
        }
        std::stable_sort(tmp.begin(), tmp.end(), [](const XE& a, const XE& b) { return a.bx < b.bx; });
        const int base = (int)xent_m.size();
        const int WT = spread_taps(w);
        for (const XE& x : tmp) {
            const int bx4 = x.bx & ~3;                  // floor to a multiple of 4 (also for negative bx)
            const int off = x.bx - bx4;
            xent_m.push_back(x.m);
            xent_bx.push_back(bx4);
            xent_e.push_back(x.e);
            if (C.split1) {
                pent_bx.push_back(x.bx);
                // the adjoint's block gather: taps aligned to the 32-column
                // window of the entry's 16-column block (offset bx mod 16)
                const int d16 = ((x.bx % 16) + 16) % 16;
                for (int c = 0; c < gather_aligned_taps(w); ++c) {
                    const int k = c - d16;
                    pent_w.push_back(k >= 0 && k < w ? x.w * wx[(size_t)x.m * w + k] : 0.f);
                }
                for (int k = 0; k < PW; ++k) {
                    pent_gx.push_back(k < w ? x.w * dwx[(size_t)x.m * w + k] : 0.f);
                    pent_gy.push_back(k < w ? x.dw * wx[(size_t)x.m * w + k] : 0.f);
                }
            }
            for (int k = 0; k < WT; ++k) {
                const int t = k - off;
                const bool in = t >= 0 && t < w;
                xent_wx.push_back(in ? x.w * wx[(size_t)x.m * w + t] : 0.f);
                // position gradient: d/dx_m (x-tap derivative) and d/dy_m (y-tap derivative)
                xent_gx.push_back(in ? x.w * dwx[(size_t)x.m * w + t] : 0.f);
                xent_gy.push_back(in ? x.dw * wx[(size_t)x.m * w + t] : 0.f);
            }
        }
        xrow_ptr[r + 1] = (int)xent_m.size();
        const int Er = (int)tmp.size();
        if (C.split1) {
            // entries of block b: first column in [16 b - w + 1, 16 b + 16)
            int lo = 0, hi = 0;
            for (int b = 0; b < nblk; ++b) {
                while (lo < Er && tmp[lo].bx < 16 * b - w + 1) ++lo;
                if (hi < lo) hi = lo;
                while (hi < Er && tmp[hi].bx < 16 * b + 16) ++hi;
                // the block's entries with their taps aligned to its 16 columns
                const int start = (int)bent_m.size();
                for (int i = lo; i < hi; ++i) {
                    float taps[16], t16[16];
                    for (int k = 0; k < w; ++k) taps[k] = tmp[i].w * wx[(size_t)tmp[i].m * w + k];
                    block_taps16(tmp[i].bx, 16 * b, taps, w, t16);
                    bent_m.push_back(tmp[i].m);
                    bent_w.insert(bent_w.end(), t16, t16 + 16);
                }
                bseg[(size_t)r * nblk + b] = make_int2(start, (int)bent_m.size());
            }
            // the block gather: entries whose first column is in block b
            // (second copies of wrapped entries, at bx < 0, belong to none)
            int a = 0;
            for (int b = 0; b < nblk; ++b) {
                while (a < Er && tmp[a].bx < 16 * b) ++a;
                int z = a;
                while (z < Er && tmp[z].bx < 16 * b + 16) ++z;
                gseg[(size_t)r * nblk + b] = make_int2(base + a, base + z);
            }
        }
        // cut the columns so that each lane group's sweep costs about the same:
        // an entry costs about as much as 1.5 columns of window sliding
        std::vector<int> cut(C.groups1 + 1);
        cut[0] = 0;
        cut[C.groups1] = G.Lx;
        {
            std::vector<double> cum(G.Lx + 1, 0.0);     // cost of columns < c
            size_t i = 0;
            for (int c = 0; c < G.Lx; ++c) {
                double add = 1.0;
                while (i < tmp.size() && tmp[i].bx <= c) { add += 1.5; ++i; }
                cum[c + 1] = cum[c] + add;
            }
            int c = 0;
            for (int q = 1; q < C.groups1; ++q) {
                const double target = cum[G.Lx] * q / C.groups1;
                while (c < G.Lx && cum[c] < target) ++c;
                cut[q] = std::max(cut[q - 1], c);
            }
        }
        for (int q = 0; q < C.groups1; ++q) {
            const int c0 = cut[q], c1 = cut[q + 1];
            int lo = 0, hi = 0;
            while (lo < Er && tmp[lo].bx < c0 - w + 1) ++lo;
            hi = lo;
            while (hi < Er && tmp[hi].bx < c1) ++hi;
            seg[(size_t)r * C.groups1 + q] = make_int4(c0, c1, base + lo, base + hi);
        }
    }

    // per row the first sorted entry that is not the second copy of a wrapped
    // one (the transposed kernels read wrapped entries modulo Lx instead)
    std::vector<int> xrow_first(G.Ly);
    for (int r = 0; r < G.Ly; ++r) {
        int i = xrow_ptr[r];
        while (i < xrow_ptr[r + 1] && xent_bx[i] < 0) ++i;
        xrow_first[r] = i;
    }

    free_sensor_tables(p.t);
    cudaError_t e = cudaSuccess;
    if (!e) e = upload(&p.t.sens_bx, bx, s);
    if (!e) e = upload(&p.t.sens_by, by, s);
    if (!e) e = upload(&p.t.sens_wx, wx, s);
    if (!e) e = upload(&p.t.sens_wy, wy, s);
    if (!e) e = upload(&p.t.sens_dwx, dwx, s);
    if (!e) e = upload(&p.t.sens_dwy, dwy, s);
    if (!e) e = upload(&p.t.sens_fac, fac, s);
    if (!e) e = upload(&p.t.row_ptr, row_ptr, s);
    if (!e) e = upload(&p.t.row_m, row_m, s);
    if (!e) e = upload(&p.t.row_w, row_w, s);
    if (!e) e = upload(&p.t.row_dw, row_dw, s);
    if (!e) e = upload(&p.t.xrow_ptr, xrow_ptr, s);
    if (!e) e = upload(&p.t.xent_m, xent_m, s);
    if (!e) e = upload(&p.t.xent_wx, xent_wx, s);
    if (!e) e = upload(&p.t.xent_bx, xent_bx, s);
    if (!e) e = upload(&p.t.xent_gx, xent_gx, s);
    if (!e) e = upload(&p.t.xent_gy, xent_gy, s);
    if (!e) e = upload(&p.t.xrow_first, xrow_first, s);
    if (!e) e = upload(&p.t.xent_rc, xent_e, s);
    if (!e) e = upload(&p.t.sens_ent, sens_ent, s);
    if (!e) e = upload(&p.t.seg, seg, s);
    if (!e) e = upload(&p.t.bseg, bseg, s);
    if (!e) e = upload(&p.t.bent_m, bent_m, s);
    if (!e) e = upload(&p.t.bent_w, bent_w, s);
    if (!e) e = upload(&p.t.pent_bx, pent_bx, s);
    if (!e) e = upload(&p.t.pent_w, pent_w, s);
    if (!e) e = upload(&p.t.pent_gx, pent_gx, s);
    if (!e) e = upload(&p.t.pent_gy, pent_gy, s);
    if (!e) e = upload(&p.t.gseg, gseg, s);
    p.lp_kcut = lowpass_bins(p);
    if (!e) e = upload(&p.t.lp_kcut, p.lp_kcut, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e == cudaErrorMemoryAllocation) return NEDNER_ENOMEM;
    return e ? NEDNER_ECUDA : NEDNER_OK;
}

nedner_status build_static_tables(nedner_plan_s& p, cudaStream_t s) {
    const Geo& G = p.geo;
    // twiddles exp(-2 pi i k / N) for every power of two N <= TW_N, at [N + k]
    std::vector<float2> tw(2 * TW_N, make_float2(0.f, 0.f));
    for (int N = 1; N <= TW_N; N *= 2)
        for (int k = 0; k < N; ++k) {
            double a = 2.0 * kPi * (double)k / (double)N;
            tw[N + k] = make_float2((float)std::cos(a), (float)-std::sin(a));
        }
    std::vector<float> dx(G.nxh), dy(G.nyp), dt(G.Nt);
    for (int j = 0; j < G.nxh; ++j) dx[j] = (float)(1.0 / win_phihat(p.win, (double)j / G.Lx));
    for (int b = 0; b < G.nyp; ++b) dy[b] = (float)(1.0 / win_phihat(p.win, (double)(b - G.ny / 2) / G.Ly));
    for (int n = 0; n < G.Nt; ++n) dt[n] = (float)(1.0 / win_phihat(p.win, (double)(n - G.Nt / 2) / G.Lt));
    std::vector<double> cd;
    win_tap_polys(p.win, G.D, cd);
    std::vector<float> cf(cd.begin(), cd.end());
    for (size_t i = 0; i < cf.size() && i < sizeof(p.tap.c) / sizeof(float); ++i) p.tap.c[i] = cf[i];
    // lateral part of nu^2: (c Nt dt)^2 ((jx/X)^2 + (jy/Y)^2), jx = 0..nx/2, jy = -ny/2..ny/2
    const double X = p.grid.nx * p.grid.dx, Y = p.grid.ny * p.grid.dy;
    const double T = p.c * p.Nt * p.dt;
    std::vector<float2> axy((size_t)G.nxh * G.nyp);
    for (int a = 0; a < G.nxh; ++a)
        for (int b = 0; b < G.nyp; ++b) {
            double jx = a, jy = b - G.ny / 2;
            double v = T * T * ((jx / X) * (jx / X) + (jy / Y) * (jy / Y));
            float hi = (float)v;
            axy[(size_t)a * G.nyp + b] = make_float2(hi, (float)(v - (double)hi));
        }
    cudaError_t e = cudaSuccess;
    if (!e) e = upload(&p.t.tw, tw, s);
    if (!e) e = upload(&p.t.deconv_x, dx, s);
    if (!e) e = upload(&p.t.deconv_y, dy, s);
    if (!e) e = upload(&p.t.deconv_t, dt, s);
    if (!e) e = upload(&p.t.tapcoef, cf, s);
    if (!e) e = upload(&p.t.axy, axy, s);
    if (!e) e = cudaMalloc((void**)&p.t.status, sizeof(int));
    if (!e) e = cudaMemsetAsync(p.t.status, 0, sizeof(int), s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e == cudaErrorMemoryAllocation) return NEDNER_ENOMEM;
    return e ? NEDNER_ECUDA : NEDNER_OK;
}

// length of a padded FFT buffer (one spare slot after every 16 values)
long padded(long n) { return n + (n >> 4); }

int pow2_floor(long v) {
    int r = 1;
    while ((long)r * 2 <= v) r *= 2;
    return r;
}

// preferred time samples per chunk of the split stage (a): the whole record
// where the workspace allows (fewer, fuller launches); a limit on the
// workspace makes the chunks shorter
constexpr int kChunkPref = 4096;

// bytes of the split stage's per-chunk buffers (Q, then R) for tq samples
size_t split_chunk_bytes(const Geo& G, int tq) {
    const size_t q = ((size_t)G.Ly * G.Lx * tq * 4 + 255) / 256 * 256;
    return q + (size_t)G.nxh * G.Ly * tq * 8;
}

void choose_chunks(nedner_plan_s& p) {
    Geo& G = p.geo;
    Chunks& c = p.ch;
    // split stage (a): block spread (4 warps of 16 columns per CTA), x-FFT of
    // nbx complex columns per CTA with Lx nbx <= 4096 (16 values per thread:
    // three CTAs of 8 warps fit an SM where 32 values per thread left two)
    c.split1 = (G.Nt >= 64 && G.Lx >= 64) ? 1 : 0;
    c.wpc_s = 4;
    {
        // per warp, batches of SPREAD_BATCH entries: sensor indices (four
        // buffers), and block-aligned taps (16) and 64 samples of g (three)
        constexpr long B = SPREAD_BATCH;
        c.smem_s = (size_t)c.wpc_s * (4 * B + 3 * (B * 16 + B * 64)) * 4;
    }
    c.nbx = (int)std::min<long>(16, std::max<long>(1, 4096 / G.Lx));
    c.perx = ((long)G.Lx * c.nbx >= 8192) ? 32 : 16;
    c.thx = (int)((long)G.Lx * c.nbx / c.perx);
    c.smem_x = (size_t)((padded((long)G.Lx * c.nbx) + 1) & ~1L) * 8;
    c.tq = std::min(G.Nt, kChunkPref);
    {
        // block gather, per warp: two batches of 32 entries (first column,
        // row-CSR index, sensor; taps; for the gradient a second tap set)
        const long pw = (G.w + 3) / 4 * 4;
        c.smem_ga = (size_t)4 * 2 * 32 * (3 + gather_aligned_taps(G.w)) * 4;
        c.smem_gg = (size_t)4 * 2 * 32 * (3 + 2 * pw) * 4;
    }
    c.gsplit = 0;
    c.tp_g = 0;
    // spread + x-FFT: lane groups of a full warp (32 time samples) while the
    // row fits in 128 KB of shared memory, smaller groups beyond
    c.c1 = std::min<long>(32, std::max<long>(2, pow2_floor((128L * 1024) / (8L * G.Lx))));
    c.c1 = std::min(c.c1, G.Nt);
    // transposed gather: two time samples per lane (64 per CTA) where the row
    // FFT has 32 values per thread (256 threads up to 2nx = 256, one CTA of 512
    // threads per SM at 2nx = 512), else time samples per CTA such that it has 16
    c.tpl_adj = (G.Lx <= 512 && G.Nt >= 64) ? 2 : 1;
    c.threads_adj = G.Lx > 256 ? 512 : 256;
    c.ca = c.tpl_adj == 2 ? 64 : (int)std::min<long>(c.c1, std::max<long>(2, 8192 / G.Lx));
    c.threads1 = 256;
    c.tpl1 = 1;
    {
        // Complex row [Lx][c1/2], padded and rounded to 16 bytes, then the
        // sweep's double-buffered batch staging (8 entries per lane group).
        // Two samples per lane (c1 = 64, warp-wide groups) when that fits two
        // CTAs per SM; else one sample per lane.
        const int wt = spread_taps(G.w);
        auto smem_for = [&](long cc, long groups) {
            const long zlen = (padded((long)G.Lx * cc / 2) + 1) & ~1L;
            return (size_t)zlen * 8 + (size_t)groups * (2 * 8 + 2 * 8 * (1 + wt + cc)) * 4;
        };
        if (G.Nt >= 64 && smem_for(64, 8) <= 115200) {
            c.tpl1 = 2;
            c.c1 = 64;
            c.groups1 = 8;
            c.smem1 = smem_for(64, 8);
            c.per1 = 32;
        } else if (G.Nt >= 64 && (long)G.Lx * 32 <= 32L * 512 && smem_for(64, 16) <= 227 * 1024) {
            // one CTA of 512 threads per SM
            c.tpl1 = 2;
            c.c1 = 64;
            c.threads1 = 512;
            c.groups1 = 16;
            c.smem1 = smem_for(64, 16);
            c.per1 = 32;
        } else {
            c.groups1 = c.threads1 / c.c1;
            c.smem1 = smem_for(c.c1, c.groups1);
            c.per1 = (long)G.Lx * c.c1 / 2 <= 16L * c.threads1 ? 16 : 32;
        }
    }
    {
        // transposed gather: padded complex row [Lx][ca/2] (16-byte rounded), then the
        // staged entries (128 at a time): taps, first column, row-CSR index (and the
        // second tap set and the samples of g for the gradient)
        const size_t zb = (size_t)((padded((long)G.Lx * c.ca / 2) + 1) & ~1L) * 8;
        const size_t wt = (size_t)spread_taps(G.w);
        c.smem_adj = zb + 128 * (wt + 2) * 4;
        c.smem_grad = zb + 128 * (2 * wt + 3) * 4;
        c.per_adj = 16;
    }
    c.c2f = (int)std::min<long>(std::min<long>(16, G.Nt), std::max<long>(1, 4096 / G.Ly));
    c.smem2f = (size_t)padded((long)G.Ly * c.c2f) * 8;
    // NER: lines per CTA such that the batched line FFT has Lt * lpc = 4096 points
    // (16 per thread of 256; 512 threads for Lt = 8192), within nz * lpc <= 4096
    c.threads3 = G.Lt > 4096 ? 512 : 256;
    c.lpc = 1;
    while (c.lpc * 2 <= G.ny && (long)G.Lt * c.lpc * 2 <= 16L * c.threads3 &&
           (long)G.nz * c.lpc * 2 <= 16L * c.threads3)
        c.lpc *= 2;
    c.smem3 = (size_t)(padded(G.Lt * c.lpc) + (c.lpc + 1) * (G.nz + 1) + padded(G.nz * c.lpc)) * 8;
    // transposed NER: line buffers, Ubar, then the items (value, first grid
    // point, w tap weights) of icap3a depth frequencies of one line at a time:
    // all nz + 1 (at most 1025), or half of them where that lets a fourth CTA
    // of 256 threads share an SM
    {
        const size_t base = (size_t)(padded(G.Lt * c.lpc) + padded(G.nz * c.lpc)) * 8;
        const size_t per_item = 8 + 4 + 4 * (size_t)(G.w + 1);
        const size_t four = 228 * 1024 / 4 - 1024;       // per CTA for four CTAs per SM
        const int all = std::min(G.nz + 1, 1025), half = (G.nz + 2) / 2;
        c.icap3a = (c.threads3 <= 256 && base + all * per_item > four && base + half * per_item <= four) ? half
                                                                                                       : all;
        c.smem3a = base + (size_t)c.icap3a * per_item;
    }
    // inverse y- and x-FFTs: C <= 16 columns (conflict-free padded loads and
    // stores), N * C <= 2048 (16 values per thread of 128)
    c.c4 = (int)std::min<long>(std::min<long>(16, G.nz), 2048 / G.ny);
    c.smem4 = (size_t)padded((long)G.ny * c.c4) * 8;
    const long H = G.nx / 2;
    c.c5 = (int)std::min<long>(std::min<long>(16, G.ny), 2048 / H);
    c.smem5 = (size_t)padded(H * c.c5) * 8;
}

}  // namespace

static nedner_status run(cudaError_t e) {
    return e == cudaSuccess ? NEDNER_OK : NEDNER_ECUDA;
}

// Stage (a) of the forward path into Ghat (region B), with the plan's
// workspace region A as scratch: the tensor-core stage, the split stage (block
// spread, x-FFT and y-FFT per chunk of time samples, the chunk's Q and R in
// region A) or the fused spread + x-FFT followed by the y-FFT.  A timer, if
// given, gets stages 0 (spread), 1 (x-FFT) and 2 (y-FFT); the tensor-core
// stage and the fused spread count as stage 0.
static cudaError_t launch_stage_a(const nedner_plan_s& p, const float* g, float2* Ghat, cudaStream_t s,
                                  StageTimer* tm = nullptr) {
    cudaError_t e;
    if (p.tp.enabled) {
        e = launch_tp_ned(p, g, Ghat, s);
        stage_mark(tm, 0);
        return e;
    }
    if (p.ch.split1) {
        float* Q = (float*)p.ws;
        float2* R = (float2*)((char*)p.ws + ((size_t)p.geo.Ly * p.geo.Lx * p.ch.tq * 4 + 255) / 256 * 256);
        return launch_ned_stage_split(p, g, Q, R, Ghat, s, tm);
    }
    float2* A = (float2*)p.ws;
    if ((e = launch_ned_spread_xfft(p, g, A, s))) return e;
    stage_mark(tm, 0);
    e = launch_ned_yfft(p, A, Ghat, s);
    stage_mark(tm, 2);
    return e;
}

extern "C" {

const char* nedner_strerror(nedner_status st) {
    switch (st) {
        case NEDNER_OK: return "ok";
        case NEDNER_EINVAL: return "invalid argument";
        case NEDNER_ERANGE: return "sensor outside the aperture (-X/2, X/2) x (-Y/2, Y/2)";
        case NEDNER_ENOMEM: return "out of memory or workspace above the limit";
        case NEDNER_ECUDA: return "CUDA error";
        case NEDNER_ENAN: return "non-finite input";
    }
    return "unknown status";
}

nedner_status nedner_plan(const double* sensor_xy, int64_t M, int Nt, double dt, double c,
                          const nedner_grid* og, nedner_window window, double sigma,
                          const nedner_opts* opts, void* stream, nedner_plan_t* out) {
    if (!out || !og || M < 0 || (M > 0 && !sensor_xy)) return NEDNER_EINVAL;
    if (M > (int64_t)1 << 26) return NEDNER_EINVAL;
    if (!is_pow2(Nt) || Nt < 8 || Nt > 4096) return NEDNER_EINVAL;
    if (!is_pow2(og->nx) || !is_pow2(og->ny) || !is_pow2(og->nz)) return NEDNER_EINVAL;
    if (og->nx < 8 || og->ny < 8 || og->nz < 8 || og->nx > 2048 || og->ny > 2048 || og->nz > 2048)
        return NEDNER_EINVAL;
    if (!(og->dx > 0) || !(og->dy > 0) || !(og->dz > 0) || !(dt > 0) || !(c > 0)) return NEDNER_EINVAL;
    if (!std::isfinite(og->dx) || !std::isfinite(og->dy) || !std::isfinite(og->dz) || !std::isfinite(dt) ||
        !std::isfinite(c))
        return NEDNER_EINVAL;
    if (sigma != 2.0) return NEDNER_EINVAL;
    if (window.kind != NEDNER_WINDOW_KB && window.kind != NEDNER_WINDOW_GAUSS) return NEDNER_EINVAL;
    if (window.width < 4 || window.width > 16 || (window.width & 1)) return NEDNER_EINVAL;
    nedner_opts o = {1, 0, 0, nullptr, NEDNER_PRECISION_FP32_NUFFT, NEDNER_NER_KB};
    if (opts) o = *opts;
    if (o.ner_interp < NEDNER_NER_KB || o.ner_interp > NEDNER_NER_DIRECT) return NEDNER_EINVAL;
    if (o.precision != NEDNER_PRECISION_FP32_NUFFT && o.precision != NEDNER_PRECISION_BF16_GEMM &&
        o.precision != NEDNER_PRECISION_FP16_GEMM)
        return NEDNER_EINVAL;

    nedner_plan_s* p = new (std::nothrow) nedner_plan_s();
    if (!p) return NEDNER_ENOMEM;
    p->M = M;
    p->Nt = Nt;
    p->dt = dt;
    p->c = c;
    p->sigma = sigma;
    p->ner_interp = o.ner_interp;
    p->grid = *og;
    p->win = make_window(window.kind, window.width, sigma);
    p->xy.assign(sensor_xy, sensor_xy + 2 * M);
    const double X = og->nx * og->dx, Y = og->ny * og->dy, Z = og->nz * og->dz;
    if (o.sensor_w) {
        p->h.assign(o.sensor_w, o.sensor_w + M);
        for (double v : p->h)
            if (!std::isfinite(v)) { delete p; return NEDNER_EINVAL; }
    } else {
        p->h.assign(M, X * Y / (double)std::max<int64_t>(M, 1));
    }
    nedner_status st = check_positions(*p, sensor_xy);
    if (st != NEDNER_OK) { delete p; return st; }

    Geo& G = p->geo;
    G.M = (int)M;
    G.Nt = Nt;
    G.nx = og->nx; G.ny = og->ny; G.nz = og->nz;
    G.Lx = 2 * og->nx; G.Ly = 2 * og->ny; G.Lt = 2 * Nt;
    G.w = window.width;
    G.D = window.width <= 12 ? 10 : 12;
    G.nxh = og->nx / 2 + 1;
    G.nyp = og->ny + 1;
    const double T = c * Nt * dt;
    const double az = (T / Z) * (T / Z);
    G.az_hi = (float)az;
    G.az_lo = (float)(az - (double)G.az_hi);
    G.sqrt_az = (float)(T / Z);
    const double N = (double)og->nx * og->ny * og->nz;
    G.apply_weights = o.apply_weights ? 1 : 0;
    G.band_mask = o.band_mask ? 1 : 0;
    G.scale = (float)((G.apply_weights ? c * dt / og->dz : 1.0) / N);
    choose_chunks(*p);

    cudaStream_t s = (cudaStream_t)stream;
    if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return NEDNER_ECUDA; }
    // workspace: region A holds R (forward) / V, region B holds Ghat / Y
    size_t r_bytes = (size_t)G.nxh * G.Ly * Nt * 8;
    size_t v_bytes = (size_t)G.nxh * G.ny * G.nz * 8;
    size_t gh_bytes = (size_t)G.nxh * G.nyp * Nt * 8;
    // Region B also holds the transposed gather's entry buffer (M w floats per
    // time sample of a pass) and the gradient's per-entry sums.  Passes are as
    // long as fit in max(Ghat / Y, 4 GB), or, under a workspace limit, in what
    // the limit leaves beside region A (256 MB at most).
    // The split stage (a) keeps one chunk of tq time samples of the oversampled
    // grid Q and of R in region A: the whole record by default; under a
    // workspace limit the chunks shrink (to 64 samples at least) until the
    // plan fits, so the forward streams over time instead of failing.
    const size_t base_a = (std::max(r_bytes, v_bytes) + 255) / 256 * 256;
    auto region_a_for = [&](int tq) {
        return p->ch.split1 ? std::max(base_a, (split_chunk_bytes(G, tq) + 255) / 256 * 256) : base_a;
    };
    const size_t base_b = std::max(gh_bytes, v_bytes);
    if (p->ch.split1 && o.max_workspace_bytes)
        while (p->ch.tq > 64 && region_a_for(p->ch.tq) + base_b > o.max_workspace_bytes) p->ch.tq /= 2;
    p->region_a = region_a_for(p->ch.tq);
    const size_t ents = (size_t)M * G.w;
    size_t cap = std::max(gh_bytes, v_bytes);
    // the entry buffer: without a limit up to 4 GB (one pass over the whole
    // record where that fits: C3's 1.6 GB, about 2 % faster than passes of
    // 512 samples); under a limit what it leaves beside region A, 256 MB at most
    size_t extra = o.max_workspace_bytes ? ((size_t)256 << 20) : ((size_t)4 << 30);
    if (o.max_workspace_bytes)
        extra = std::min(extra, o.max_workspace_bytes > p->region_a ? o.max_workspace_bytes - p->region_a : 0);
    cap = std::max(cap, extra);
    p->ch.tp_adj = Nt;
    while (p->ch.tp_adj > p->ch.ca && ents * p->ch.tp_adj * 4 > cap) p->ch.tp_adj /= 2;
    // block gather: its pass grid Q-bar (Ly Lx tp_g floats) sits in region A
    // after R-bar; passes no longer than the entry buffer's
    {
        const size_t rbar = (r_bytes + 255) / 256 * 256;
        int tp = p->ch.tp_adj;
        while (tp > 64 && rbar + (size_t)G.Ly * G.Lx * tp * 4 > p->region_a) tp /= 2;
        p->ch.gsplit = (p->ch.split1 && tp >= 64 && rbar + (size_t)G.Ly * G.Lx * tp * 4 <= p->region_a) ? 1 : 0;
        p->ch.tp_g = p->ch.gsplit ? tp : 0;
        if (p->ch.gsplit) p->ch.tp_adj = tp;
    }
    size_t pa_bytes = ents * p->ch.tp_adj * 4;
    size_t q_bytes = ents * (Nt / p->ch.ca) * 8;
    p->ws_bytes = p->region_a + std::max(std::max(gh_bytes, v_bytes), std::max(pa_bytes, q_bytes));
    if (o.max_workspace_bytes && p->ws_bytes > o.max_workspace_bytes) { delete p; return NEDNER_ENOMEM; }
    cudaError_t e = cudaMalloc(&p->ws, p->ws_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return e == cudaErrorMemoryAllocation ? NEDNER_ENOMEM : NEDNER_ECUDA;
    }
    st = build_static_tables(*p, s);
    if (st == NEDNER_OK) st = build_sensor_tables(*p, s);
    if (st == NEDNER_OK && configure_fwd_kernels(*p) != cudaSuccess) st = NEDNER_ECUDA;
    if (st == NEDNER_OK && configure_adj_kernels(*p) != cudaSuccess) st = NEDNER_ECUDA;
    if (st == NEDNER_OK && o.precision != NEDNER_PRECISION_FP32_NUFFT)
        st = build_tp(*p, s, o.precision == NEDNER_PRECISION_FP16_GEMM);
    if (st != NEDNER_OK) {
        cudaGetLastError();
        free_tables(p->t);
        free_tp(p->tp);
        cudaFree(p->ws);
        delete p;
        return st;
    }
    *out = p;
    return NEDNER_OK;
}

nedner_status nedner_set_positions(nedner_plan_t p, const double* sensor_xy) {
    if (!p || (p->M > 0 && !sensor_xy)) return NEDNER_EINVAL;
    nedner_status st = check_positions(*p, sensor_xy);
    if (st != NEDNER_OK) return st;
    p->xy.assign(sensor_xy, sensor_xy + 2 * p->M);
    if (cudaSetDevice(p->device) != cudaSuccess) return NEDNER_ECUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return NEDNER_ECUDA;
    return build_sensor_tables(*p, 0);
}

nedner_status nedner_forward(nedner_plan_t p, const float* g, float* p0, void* stream) {
    if (!p || !p0 || (p->M > 0 && !g)) return NEDNER_EINVAL;
    if (((uintptr_t)p0 & 7) != 0 || ((uintptr_t)g & 15) != 0) return NEDNER_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    float2* A = (float2*)p->ws;
    float2* B = (float2*)((char*)p->ws + p->region_a);
    cudaError_t e;
    if ((e = launch_stage_a(*p, g, B, s))) return run(e);
    if ((e = launch_ner_lines(*p, B, A, s))) return run(e);
    if ((e = launch_img_yifft(*p, A, B, s))) return run(e);
    return run(launch_img_xc2r(*p, B, p0, s));
}

nedner_status nedner_forward_profiled(nedner_plan_t p, const float* g, float* p0, void* stream,
                                      float* stage_ms) {
    if (!p || !p0 || !stage_ms || (p->M > 0 && !g)) return NEDNER_EINVAL;
    if (((uintptr_t)p0 & 7) != 0 || ((uintptr_t)g & 15) != 0) return NEDNER_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    float2* A = (float2*)p->ws;
    float2* B = (float2*)((char*)p->ws + p->region_a);
    StageTimer tm(s);
    tm.mark(-1);
    cudaError_t e = launch_stage_a(*p, g, B, s, &tm);
    if (!e) e = launch_ner_lines(*p, B, A, s);
    tm.mark(3);
    if (!e) e = launch_img_yifft(*p, A, B, s);
    tm.mark(4);
    if (!e) e = launch_img_xc2r(*p, B, p0, s);
    tm.mark(5);
    cudaError_t f = tm.finish(stage_ms, NEDNER_FORWARD_KERNELS);
    return run(e ? e : f);
}

nedner_status nedner_ned_stage(nedner_plan_t p, const float* g, void* Ghat, void* stream) {
    if (!p || !Ghat || (p->M > 0 && !g)) return NEDNER_EINVAL;
    if (((uintptr_t)g & 15) != 0 || ((uintptr_t)Ghat & 15) != 0) return NEDNER_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return run(launch_stage_a(*p, g, (float2*)Ghat, s));
}

// Transposed stages shared by the adjoint and the position gradient:
// p0-shaped input -> R-bar in region A.
static cudaError_t transposed_to_R(nedner_plan_t p, const float* p0, cudaStream_t s) {
    float2* A = (float2*)p->ws;
    float2* B = (float2*)((char*)p->ws + p->region_a);
    cudaError_t e;
    if ((e = launch_img_xr2c_adj(*p, p0, B, s))) return e;
    if ((e = launch_img_yfft_adj(*p, B, A, s))) return e;
    if ((e = launch_ner_lines_adj(*p, A, B, s))) return e;
    return launch_ned_yfft_adj(*p, B, A, s);
}

nedner_status nedner_adjoint(nedner_plan_t p, const float* p0, float* g, void* stream) {
    if (!p || !p0 || (p->M > 0 && !g)) return NEDNER_EINVAL;
    if (p->ner_interp != NEDNER_NER_KB) return NEDNER_EINVAL;
    if (((uintptr_t)p0 & 7) != 0) return NEDNER_EINVAL;
    if (p->M == 0) return NEDNER_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = transposed_to_R(p, p0, s))) return run(e);
    float2* A = (float2*)p->ws;
    float* Eb = (float*)((char*)p->ws + p->region_a);
    return run(launch_adj_gather(*p, A, Eb, g, s));
}

// the transposed path with a stage timer: stages 0-3 are the inverse image
// transposes, the transposed NER and the transposed y-FFT, 4 the gather and 5
// its per-sensor sum (both summed over the passes of time samples)
static cudaError_t transposed_to_R_timed(nedner_plan_t p, const float* p0, cudaStream_t s, StageTimer& tm) {
    float2* A = (float2*)p->ws;
    float2* B = (float2*)((char*)p->ws + p->region_a);
    cudaError_t e;
    tm.mark(-1);
    if ((e = launch_img_xr2c_adj(*p, p0, B, s))) return e;
    tm.mark(0);
    if ((e = launch_img_yfft_adj(*p, B, A, s))) return e;
    tm.mark(1);
    if ((e = launch_ner_lines_adj(*p, A, B, s))) return e;
    tm.mark(2);
    if ((e = launch_ned_yfft_adj(*p, B, A, s))) return e;
    tm.mark(3);
    return tm.err;
}

nedner_status nedner_adjoint_profiled(nedner_plan_t p, const float* p0, float* g, void* stream, float* stage_ms) {
    if (!p || !p0 || !stage_ms || (p->M > 0 && !g)) return NEDNER_EINVAL;
    if (p->ner_interp != NEDNER_NER_KB) return NEDNER_EINVAL;
    if (((uintptr_t)p0 & 7) != 0) return NEDNER_EINVAL;
    for (int k = 0; k < NEDNER_TRANSPOSED_KERNELS; ++k) stage_ms[k] = 0.f;
    if (p->M == 0) return NEDNER_OK;
    cudaStream_t s = (cudaStream_t)stream;
    StageTimer tm(s);
    cudaError_t e = transposed_to_R_timed(p, p0, s, tm);
    float2* A = (float2*)p->ws;
    float* Eb = (float*)((char*)p->ws + p->region_a);
    if (!e) e = launch_adj_gather(*p, A, Eb, g, s, &tm);
    cudaError_t f = tm.finish(stage_ms, NEDNER_TRANSPOSED_KERNELS);
    return run(e ? e : f);
}

nedner_status nedner_grad_positions_profiled(nedner_plan_t p, const float* g, const float* dL_dp0, float* dL_dxy,
                                             void* stream, float* stage_ms) {
    if (!p || !dL_dp0 || !stage_ms || (p->M > 0 && (!g || !dL_dxy))) return NEDNER_EINVAL;
    if (p->ner_interp != NEDNER_NER_KB) return NEDNER_EINVAL;
    if (((uintptr_t)dL_dp0 & 7) != 0) return NEDNER_EINVAL;
    for (int k = 0; k < NEDNER_TRANSPOSED_KERNELS; ++k) stage_ms[k] = 0.f;
    if (p->M == 0) return NEDNER_OK;
    cudaStream_t s = (cudaStream_t)stream;
    StageTimer tm(s);
    cudaError_t e = transposed_to_R_timed(p, dL_dp0, s, tm);
    float2* A = (float2*)p->ws;
    float2* Q = (float2*)((char*)p->ws + p->region_a);
    if (!e) e = launch_grad_gather(*p, A, g, Q, dL_dxy, s, &tm);
    cudaError_t f = tm.finish(stage_ms, NEDNER_TRANSPOSED_KERNELS);
    return run(e ? e : f);
}

nedner_status nedner_grad_positions(nedner_plan_t p, const float* g, const float* dL_dp0, float* dL_dxy,
                                    void* stream) {
    if (!p || !dL_dp0 || (p->M > 0 && (!g || !dL_dxy))) return NEDNER_EINVAL;
    if (p->ner_interp != NEDNER_NER_KB) return NEDNER_EINVAL;
    if (((uintptr_t)dL_dp0 & 7) != 0) return NEDNER_EINVAL;
    if (p->M == 0) return NEDNER_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = transposed_to_R(p, dL_dp0, s))) return run(e);
    float2* A = (float2*)p->ws;
    float2* Q = (float2*)((char*)p->ws + p->region_a);
    return run(launch_grad_gather(*p, A, g, Q, dL_dxy, s));
}

nedner_status nedner_device_status(nedner_plan_t p, int* flags) {
    if (!p || !flags) return NEDNER_EINVAL;
    *flags = 0;
    if (cudaSetDevice(p->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return NEDNER_ECUDA;
    const int zero = 0;
    int f = 0, st = 0;
    if (p->tp.err) {
        if (cudaMemcpy(&f, p->tp.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return NEDNER_ECUDA;
        if (cudaMemcpy(p->tp.err, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return NEDNER_ECUDA;
    }
    if (p->t.status) {
        if (cudaMemcpy(&st, p->t.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return NEDNER_ECUDA;
        if (cudaMemcpy(p->t.status, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return NEDNER_ECUDA;
    }
    *flags = (f ? NEDNER_STATUS_WAIT_TIMEOUT : 0) | ((st & NEDNER_FLAG_NONFINITE) ? NEDNER_STATUS_NONFINITE : 0);
    return (*flags & NEDNER_STATUS_NONFINITE) ? NEDNER_ENAN : NEDNER_OK;
}

nedner_status nedner_debug_set_wait_limit(nedner_plan_t p, int polls) {
    if (!p || polls < 0) return NEDNER_EINVAL;
    p->tp.wait_limit = std::min(polls, TP_WAIT_LIMIT);
    return NEDNER_OK;
}

size_t nedner_workspace_bytes(nedner_plan_t p) { return p ? p->ws_bytes : 0; }

int nedner_plan_info(nedner_plan_t p, int64_t* out, int nout) {
    if (!p || !out || nout < 0) return -1;
    const Geo& G = p->geo;
    const Chunks& c = p->ch;
    int64_t fwd;
    if (p->tp.enabled) fwd = 3 * (G.Nt / tp_chunk(G.Nt)) + 1 + (p->tp.fp16 ? 1 : 0) + 3;   // passes, Nyquist line, scale; NER, images
    else if (c.split1) fwd = 3 * (G.Nt / c.tq) + 3;                                     // spread, x-FFT, y-FFT per chunk
    else fwd = 5;
    const int64_t adj = p->M == 0 ? 0 : 4 + (int64_t)(c.gsplit ? 3 : 2) * (G.Nt / c.tp_adj);
    const int64_t grad = p->M == 0 ? 0 : 4 + (c.gsplit ? 2 * (int64_t)(G.Nt / c.tp_g) + 1 : 2);
    const int64_t v[] = {c.split1, c.tq, c.tp_adj, c.gsplit, c.tp_g, fwd, adj, grad};
    const int n = (int)(sizeof(v) / sizeof(v[0]));
    for (int i = 0; i < n && i < nout; ++i) out[i] = v[i];
    return n;
}

int nedner_work_split(int nx, int ny, int nz, int Nt, int w, int64_t* out, int nout) {
    if (!out || nout < 0) return -1;
    if (!is_pow2(Nt) || Nt < 8 || Nt > 4096) return -1;
    if (!is_pow2(nx) || !is_pow2(ny) || !is_pow2(nz)) return -1;
    if (nx < 8 || ny < 8 || nz < 8 || nx > 2048 || ny > 2048 || nz > 2048) return -1;
    if (w < 4 || w > 16 || (w & 1)) return -1;
    nedner_plan_s p;
    Geo& G = p.geo;
    G.Nt = Nt;
    G.nx = nx; G.ny = ny; G.nz = nz;
    G.Lx = 2 * nx; G.Ly = 2 * ny; G.Lt = 2 * Nt;
    G.nxh = nx / 2 + 1; G.nyp = ny + 1;
    G.w = w;
    choose_chunks(p);
    const Chunks& c = p.ch;
    const int64_t v[] = {c.c1, c.c2f, c.c4, c.c5, c.groups1, c.threads1, c.per1, c.tpl1, c.ca, c.per_adj,
                         c.tpl_adj, c.threads_adj, c.lpc, c.threads3, (int64_t)c.smem1, (int64_t)c.smem2f,
                         (int64_t)c.smem3, (int64_t)c.smem4, (int64_t)c.smem5, (int64_t)c.smem_adj,
                         (int64_t)c.smem_grad, c.split1, c.tq, c.wpc_s, c.nbx, c.thx, c.perx, (int64_t)c.smem_s,
                         (int64_t)c.smem_x, (int64_t)c.smem3a, c.icap3a};
    const int n = (int)(sizeof(v) / sizeof(v[0]));
    for (int i = 0; i < n && i < nout; ++i) out[i] = v[i];
    return n;
}

nedner_status nedner_forward_host(nedner_plan_t p, const float* g_host, float* p0_host, void* stream) {
    if (!p || !p0_host || (p->M > 0 && !g_host)) return NEDNER_EINVAL;
    const Geo& G = p->geo;
    constexpr int NCS = 4;                               // copy streams (several copy engines at once)
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    const size_t gbytes = (size_t)p->M * G.Nt * sizeof(float);
    const size_t pbytes = (size_t)G.nx * G.ny * G.nz * sizeof(float);
    if (!p->host_p0 || !p->host_ev[15]) {
        // first call: device copies of g and p0, the copy streams and their
        // events; after a failure, a later call creates only what is missing
        if (!e && gbytes && !p->host_g) e = cudaMalloc((void**)&p->host_g, gbytes);
        if (!e && !p->host_p0) e = cudaMalloc((void**)&p->host_p0, pbytes);
        for (int i = 0; i < NCS && !e; ++i)
            if (!p->copy_stream[i]) e = cudaStreamCreateWithFlags(&p->copy_stream[i], cudaStreamNonBlocking);
        for (int i = 0; i < 16 && !e; ++i)
            if (!p->host_ev[i]) e = cudaEventCreateWithFlags(&p->host_ev[i], cudaEventDisableTiming);
        if (e) return e == cudaErrorMemoryAllocation ? NEDNER_ENOMEM : NEDNER_ECUDA;
    }
    cudaStream_t* cs = p->copy_stream;
    cudaEvent_t* ev = p->host_ev;
    float2* A = (float2*)p->ws;
    float2* B = (float2*)((char*)p->ws + p->region_a);
    // upload g in NCS contiguous parts (whole sensor rows), one per copy stream,
    // after the work already queued on the caller's stream
    if ((e = cudaEventRecord(ev[0], s))) return run(e);
    const int64_t mp = (p->M + NCS - 1) / NCS;
    for (int i = 0; i < NCS; ++i) {
        const int64_t m0 = std::min<int64_t>(p->M, i * mp), m1 = std::min<int64_t>(p->M, m0 + mp);
        if ((e = cudaStreamWaitEvent(cs[i], ev[0], 0))) return run(e);
        if (m1 > m0 && (e = cudaMemcpyAsync(p->host_g + m0 * G.Nt, g_host + m0 * G.Nt,
                                            (size_t)(m1 - m0) * G.Nt * sizeof(float), cudaMemcpyHostToDevice, cs[i])))
            return run(e);
        if ((e = cudaEventRecord(ev[1 + i], cs[i])) || (e = cudaStreamWaitEvent(s, ev[1 + i], 0))) return run(e);
    }
    if ((e = launch_stage_a(*p, p->host_g, B, s))) return run(e);
    if ((e = launch_ner_lines(*p, B, A, s))) return run(e);
    if ((e = launch_img_yifft(*p, A, B, s))) return run(e);
    // p0 in NCS blocks of depth planes, each downloaded as soon as it is written
    const int zc = (G.nz + NCS - 1) / NCS;
    for (int i = 0; i * zc < G.nz; ++i) {
        const int z0 = i * zc, nzc = std::min(zc, G.nz - z0);
        if ((e = launch_img_xc2r(*p, B, p->host_p0, s, z0, nzc))) return run(e);
        if ((e = cudaEventRecord(ev[5 + i], s)) || (e = cudaStreamWaitEvent(cs[i], ev[5 + i], 0))) return run(e);
        const size_t off = (size_t)z0 * G.ny * G.nx, cnt = (size_t)nzc * G.ny * G.nx * sizeof(float);
        if ((e = cudaMemcpyAsync(p0_host + off, p->host_p0 + off, cnt, cudaMemcpyDeviceToHost, cs[i]))) return run(e);
        if ((e = cudaEventRecord(ev[9 + i], cs[i]))) return run(e);
    }
    // the caller's stream completes when p0 has arrived
    for (int i = 0; i * zc < G.nz; ++i)
        if ((e = cudaStreamWaitEvent(s, ev[9 + i], 0))) return run(e);
    return NEDNER_OK;
}

nedner_status nedner_destroy(nedner_plan_t p) {
    if (!p) return NEDNER_OK;
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    free_tables(p->t);
    free_tp(p->tp);
    cudaFree(p->ws);
    cudaFree(p->host_g);
    cudaFree(p->host_p0);
    for (cudaEvent_t& ev : p->host_ev)
        if (ev) cudaEventDestroy(ev);
    for (cudaStream_t& cs : p->copy_stream)
        if (cs) cudaStreamDestroy(cs);
    delete p;
    return NEDNER_OK;
}

}  // extern "C"

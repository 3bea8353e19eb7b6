// Plan construction and the C-ABI entry points of include/nedner.h.
//
// The plan precomputes, once per geometry (the "precomputed Psi" of Sec. 5,
// Table 2: reusing the window tables across reconstructions), in FP64 on the
// host: the per-sensor window taps and grid offsets of the NED-NUFFT
// (Eq. NED_NUFFT), the row lists that let each CTA gather the sensors of its
// grid row, the deconvolution tables 1/phihat of both NUFFTs (Eq. PSI), the
// tap polynomials of the NER interpolation, and the lateral part of nu^2 for
// every line.  It then allocates the device workspace.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "fft.cuh"
#include "internal.h"

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
    cudaFree(t.row_ptr); cudaFree(t.row_m); cudaFree(t.row_w);
    t.sens_bx = t.sens_by = nullptr;
    t.sens_wx = t.sens_wy = t.sens_dwx = t.sens_dwy = t.sens_fac = nullptr;
    t.row_ptr = t.row_m = nullptr;
    t.row_w = nullptr;
}

void free_tables(DevTables& t) {
    cudaFree(t.tw); cudaFree(t.deconv_x); cudaFree(t.deconv_y); cudaFree(t.deconv_t);
    cudaFree(t.tapcoef); cudaFree(t.axy);
    t.tw = nullptr; t.deconv_x = t.deconv_y = t.deconv_t = t.tapcoef = nullptr; t.axy = nullptr;
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
nedner_status build_sensor_tables(nedner_plan_s& p, cudaStream_t s) {
    const Geo& G = p.geo;
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
    // CSR by grid row: entry (m, ky) lands in row (by_m + ky) mod Ly
    std::vector<int> row_ptr(G.Ly + 1, 0);
    for (int64_t m = 0; m < M; ++m)
        for (int k = 0; k < w; ++k) row_ptr[((by[m] + k) & (G.Ly - 1)) + 1]++;
    for (int r = 0; r < G.Ly; ++r) row_ptr[r + 1] += row_ptr[r];
    std::vector<int> fill(row_ptr.begin(), row_ptr.end() - 1);
    std::vector<int> row_m((size_t)M * w);
    std::vector<float> row_w((size_t)M * w);
    for (int64_t m = 0; m < M; ++m)
        for (int k = 0; k < w; ++k) {
            int r = (by[m] + k) & (G.Ly - 1);
            int e = fill[r]++;
            row_m[e] = (int)m;
            row_w[e] = wy[m * w + k] * fac[m];
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
    if (!e) e = cudaStreamSynchronize(s);
    if (e == cudaErrorMemoryAllocation) return NEDNER_ENOMEM;
    return e ? NEDNER_ECUDA : NEDNER_OK;
}

nedner_status build_static_tables(nedner_plan_s& p, cudaStream_t s) {
    const Geo& G = p.geo;
    std::vector<float2> tw(TW_N);
    for (int k = 0; k < TW_N; ++k) {
        double a = 2.0 * kPi * (double)k / (double)TW_N;
        tw[k] = make_float2((float)std::cos(a), (float)-std::sin(a));
    }
    std::vector<float> dx(G.nxh), dy(G.nyp), dt(G.Nt);
    for (int j = 0; j < G.nxh; ++j) dx[j] = (float)(1.0 / win_phihat(p.win, (double)j / G.Lx));
    for (int b = 0; b < G.nyp; ++b) dy[b] = (float)(1.0 / win_phihat(p.win, (double)(b - G.ny / 2) / G.Ly));
    for (int n = 0; n < G.Nt; ++n) dt[n] = (float)(1.0 / win_phihat(p.win, (double)(n - G.Nt / 2) / G.Lt));
    std::vector<double> cd;
    win_tap_polys(p.win, G.D, cd);
    std::vector<float> cf(cd.begin(), cd.end());
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
    if (!e) e = cudaStreamSynchronize(s);
    if (e == cudaErrorMemoryAllocation) return NEDNER_ENOMEM;
    return e ? NEDNER_ECUDA : NEDNER_OK;
}

int pow2_floor(long v) {
    int r = 1;
    while ((long)r * 2 <= v) r *= 2;
    return r;
}

void choose_chunks(nedner_plan_s& p) {
    Geo& G = p.geo;
    Chunks& c = p.ch;
    const long budget = 64 * 1024;                     // bytes of shared memory per CTA
    c.c1 = std::min<long>(32, std::max<long>(2, pow2_floor(budget / (8L * G.Lx))));
    c.c1 = std::min(c.c1, G.Nt);
    c.smem1 = (size_t)G.Lx * c.c1 * 8;                 // real row + complex scratch
    c.c2 = std::min<long>(16, std::max<long>(1, pow2_floor(budget / (16L * G.Ly))));
    c.c2 = std::min(c.c2, G.Nt);
    c.smem2 = (size_t)G.Ly * c.c2 * 16;
    c.smem3 = (size_t)(2 * G.Lt + (G.nz + 1) + 2 * G.nz) * 8 + (size_t)G.w * (G.D + 1) * 4;
    c.c4 = 1;
    while (c.c4 * 2 <= 16 && c.c4 * 2 <= G.nz && 2L * G.ny * (c.c4 * 2 + 1) * 8 <= 96 * 1024) c.c4 *= 2;
    c.smem4 = (size_t)2 * G.ny * (c.c4 + 1) * 8;
    const long H = G.nx / 2;
    c.c5 = 1;
    while (c.c5 * 2 <= 16 && c.c5 * 2 <= G.ny && (3 * H + 1) * (c.c5 * 2 + 1) * 8 <= 96 * 1024) c.c5 *= 2;
    c.smem5 = (size_t)(3 * H + 1) * (c.c5 + 1) * 8;
}

}  // namespace

static nedner_status run(cudaError_t e) {
    return e == cudaSuccess ? NEDNER_OK : NEDNER_ECUDA;
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
    nedner_opts o = {1, 0, 0, nullptr};
    if (opts) o = *opts;

    nedner_plan_s* p = new (std::nothrow) nedner_plan_s();
    if (!p) return NEDNER_ENOMEM;
    p->M = M;
    p->Nt = Nt;
    p->dt = dt;
    p->c = c;
    p->sigma = sigma;
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
    p->region_a = (std::max(r_bytes, v_bytes) + 255) / 256 * 256;
    p->ws_bytes = p->region_a + std::max(gh_bytes, v_bytes);
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
    if (st != NEDNER_OK) {
        cudaGetLastError();
        free_tables(p->t);
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
    if (((uintptr_t)p0 & 7) != 0) return NEDNER_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    float2* A = (float2*)p->ws;
    float2* B = (float2*)((char*)p->ws + p->region_a);
    cudaError_t e;
    if ((e = launch_ned_spread_xfft(*p, g, A, s))) return run(e);
    if ((e = launch_ned_yfft(*p, A, B, s))) return run(e);
    if ((e = launch_ner_lines(*p, B, A, s))) return run(e);
    if ((e = launch_img_yifft(*p, A, B, s))) return run(e);
    return run(launch_img_xc2r(*p, B, p0, s));
}

nedner_status nedner_forward_profiled(nedner_plan_t p, const float* g, float* p0, void* stream,
                                      float* stage_ms) {
    if (!p || !p0 || !stage_ms || (p->M > 0 && !g)) return NEDNER_EINVAL;
    if (((uintptr_t)p0 & 7) != 0) return NEDNER_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    float2* A = (float2*)p->ws;
    float2* B = (float2*)((char*)p->ws + p->region_a);
    cudaEvent_t ev[NEDNER_FORWARD_KERNELS + 1];
    int made = 0;
    cudaError_t e = cudaSuccess;
    for (; made <= NEDNER_FORWARD_KERNELS && !e; ++made) e = cudaEventCreate(&ev[made]);
    if (!e) e = cudaEventRecord(ev[0], s);
    if (!e) e = launch_ned_spread_xfft(*p, g, A, s);
    if (!e) e = cudaEventRecord(ev[1], s);
    if (!e) e = launch_ned_yfft(*p, A, B, s);
    if (!e) e = cudaEventRecord(ev[2], s);
    if (!e) e = launch_ner_lines(*p, B, A, s);
    if (!e) e = cudaEventRecord(ev[3], s);
    if (!e) e = launch_img_yifft(*p, A, B, s);
    if (!e) e = cudaEventRecord(ev[4], s);
    if (!e) e = launch_img_xc2r(*p, B, p0, s);
    if (!e) e = cudaEventRecord(ev[5], s);
    if (!e) e = cudaEventSynchronize(ev[5]);
    for (int k = 0; k < NEDNER_FORWARD_KERNELS && !e; ++k) e = cudaEventElapsedTime(&stage_ms[k], ev[k], ev[k + 1]);
    for (int k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
    return run(e);
}

nedner_status nedner_ned_stage(nedner_plan_t p, const float* g, void* Ghat, void* stream) {
    if (!p || !Ghat || (p->M > 0 && !g)) return NEDNER_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    float2* A = (float2*)p->ws;
    cudaError_t e;
    if ((e = launch_ned_spread_xfft(*p, g, A, s))) return run(e);
    return run(launch_ned_yfft(*p, A, (float2*)Ghat, s));
}

nedner_status nedner_adjoint(nedner_plan_t p, const float* p0, float* g, void* stream) {
    (void)p; (void)p0; (void)g; (void)stream;
    return NEDNER_EINVAL;
}

nedner_status nedner_grad_positions(nedner_plan_t p, const float* g, const float* dL_dp0, float* dL_dxy,
                                    void* stream) {
    (void)p; (void)g; (void)dL_dp0; (void)dL_dxy; (void)stream;
    return NEDNER_EINVAL;
}

size_t nedner_workspace_bytes(nedner_plan_t p) { return p ? p->ws_bytes : 0; }

nedner_status nedner_destroy(nedner_plan_t p) {
    if (!p) return NEDNER_OK;
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    free_tables(p->t);
    cudaFree(p->ws);
    delete p;
    return NEDNER_OK;
}

}  // extern "C"

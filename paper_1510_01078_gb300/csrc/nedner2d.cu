// The two-dimensional variant (Sec. 7): sensors on a line z = 0, an output
// image (nz, nx).  The 2-D reconstruction is Eq. disc_rec with one lateral
// axis:
//   G[jx, n] = sum_m (h_m / dx) g[m, n] exp(-2 pi i jx x_m / X)
//   nu = sign(l) c Nt dt sqrt((jx/X)^2 + (l/Z)^2),  F = W s sum_n G exp(-2 pi i nu n / Nt)
//   p2[qz, qx] = Re (1/(nx nz)) sum_{jx, l} F exp(2 pi i (jx (qx - nx/2)/nx + l qz/nz)).
// It is evaluated by the 3-D path on a grid of ny = NY2D rows with every
// sensor at y = 0 and area h_m dy: the 3-D NED sum then does not depend on
// jy, the jy = 0 lines carry exactly the 2-D nu, W and F, and summing the 3-D
// image over its rows keeps only jy = 0 (sum_qy exp(2 pi i jy (qy - ny/2)/ny)
// = ny [jy = 0]), which cancels the 3-D scale's extra 1/ny:
//   p2 = sum_qy p3,        R2 = S R3,        R2^T = R3^T S^T,
// S the sum over rows and S^T the copy of an image to every row.  The cost is
// the 3-D path's on NY2D rows.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "internal.h"
#include "nedner.h"

namespace nedner {

constexpr int NY2D = 8;   // the smallest grid the 3-D plan accepts

// p2[qz][qx] = sum_qy p3[qz][qy][qx]
__global__ void k_sum_rows(int nz, int ny, int nx, const float* __restrict__ p3, float* __restrict__ p2) {
    const long n = (long)nz * nx;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const long qz = i / nx, qx = i - qz * nx;
        float s = 0.f;
        for (int qy = 0; qy < ny; ++qy) s += p3[((size_t)qz * ny + qy) * nx + qx];
        p2[i] = s;
    }
}

// p3[qz][qy][qx] = p2[qz][qx] for every qy
__global__ void k_copy_rows(int nz, int ny, int nx, const float* __restrict__ p2, float* __restrict__ p3) {
    const long n = (long)nz * ny * nx;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const long qx = i % nx, qz = i / ((long)ny * nx);
        p3[i] = p2[qz * nx + qx];
    }
}

}  // namespace nedner

struct nedner2d_plan_s {
    nedner_plan_t p3 = nullptr;
    int64_t M = 0;
    int Nt = 0, nx = 0, nz = 0;
    double dx = 0, dz = 0;
    float* img3 = nullptr;          // [nz][NY2D][nx] f32, the 3-D image
    std::vector<double> xy;         // the embedded positions (x_m, 0)
};

using namespace nedner;

static nedner_status st2d(cudaError_t e) {
    if (e == cudaSuccess) return NEDNER_OK;
    return e == cudaErrorMemoryAllocation ? NEDNER_ENOMEM : NEDNER_ECUDA;
}

static unsigned grid_for(long n) { return (unsigned)std::min<long>((n + 255) / 256, 152L * 16); }

extern "C" {

nedner_status nedner2d_plan(const double* sensor_x, int64_t M, int Nt, double dt, double c, int nx, int nz,
                            double dx, double dz, nedner_window window, double sigma, const nedner_opts* opts,
                            void* stream, nedner2d_plan_t* out) {
    if (!out || M < 0 || (M > 0 && !sensor_x) || !(dx > 0) || !(dz > 0)) return NEDNER_EINVAL;
    nedner2d_plan_s* q = new (std::nothrow) nedner2d_plan_s();
    if (!q) return NEDNER_ENOMEM;
    q->M = M; q->Nt = Nt; q->nx = nx; q->nz = nz; q->dx = dx; q->dz = dz;
    q->xy.assign(2 * M, 0.0);
    for (int64_t m = 0; m < M; ++m) q->xy[2 * m] = sensor_x[m];
    // lengths h_m (default X / M) become areas h_m dy with dy = dx
    nedner_opts o = {1, 0, 0, nullptr, NEDNER_PRECISION_FP32_NUFFT, NEDNER_NER_KB};
    if (opts) o = *opts;
    if (o.precision != NEDNER_PRECISION_FP32_NUFFT) { delete q; return NEDNER_EINVAL; }
    std::vector<double> area(M, nx * dx * dx / (double)std::max<int64_t>(M, 1));
    if (o.sensor_w)
        for (int64_t m = 0; m < M; ++m) area[m] = o.sensor_w[m] * dx;
    o.sensor_w = M > 0 ? area.data() : nullptr;
    const nedner_grid g3 = {nx, NY2D, nz, dx, dx, dz};
    nedner_status st = nedner_plan(q->xy.data(), M, Nt, dt, c, &g3, window, sigma, &o, stream, &q->p3);
    if (st != NEDNER_OK) { delete q; return st; }
    if (cudaMalloc(&q->img3, (size_t)nz * NY2D * nx * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        nedner_destroy(q->p3);
        delete q;
        return NEDNER_ENOMEM;
    }
    *out = q;
    return NEDNER_OK;
}

nedner_status nedner2d_set_positions(nedner2d_plan_t q, const double* sensor_x) {
    if (!q || (q->M > 0 && !sensor_x)) return NEDNER_EINVAL;
    std::vector<double> xy(2 * q->M, 0.0);
    for (int64_t m = 0; m < q->M; ++m) xy[2 * m] = sensor_x[m];
    nedner_status st = nedner_set_positions(q->p3, xy.data());
    if (st == NEDNER_OK) q->xy.swap(xy);
    return st;
}

nedner_status nedner2d_forward(nedner2d_plan_t q, const float* g, float* p2, void* stream) {
    if (!q || !p2 || (q->M > 0 && !g)) return NEDNER_EINVAL;
    if (((uintptr_t)p2 & 3) != 0) return NEDNER_EINVAL;
    nedner_status st = nedner_forward(q->p3, g, q->img3, stream);
    if (st != NEDNER_OK) return st;
    const long n = (long)q->nz * q->nx;
    k_sum_rows<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(q->nz, NY2D, q->nx, q->img3, p2);
    return st2d(cudaGetLastError());
}

nedner_status nedner2d_adjoint(nedner2d_plan_t q, const float* p2, float* g, void* stream) {
    if (!q || !p2 || (q->M > 0 && !g)) return NEDNER_EINVAL;
    if (((uintptr_t)p2 & 3) != 0) return NEDNER_EINVAL;
    const long n = (long)q->nz * NY2D * q->nx;
    k_copy_rows<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(q->nz, NY2D, q->nx, p2, q->img3);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return st2d(e);
    return nedner_adjoint(q->p3, q->img3, g, stream);
}

nedner_status nedner2d_destroy(nedner2d_plan_t q) {
    if (!q) return NEDNER_OK;
    nedner_status st = nedner_destroy(q->p3);
    cudaFree(q->img3);
    delete q;
    return st;
}

}  // extern "C"

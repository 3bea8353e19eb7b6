// Runs the NER value evaluation (ner_eval.cuh) on the host for tests: the
// float-float frequency nu_l and the coefficient times F(nu_l) interpolated
// from one line's oversampled spectrum, with the tap polynomials the plan
// builds (window.cpp).  Test infrastructure only.
#include <cstring>
#include <vector>

#include "ner_eval.cuh"
#include "window.h"

thread_local HostDim3 threadIdx;
HostDim3 blockDim;
void __syncthreads() {}

using namespace nedner;

static Geo geo(int Nt, double az, int w) {
    Geo G;
    std::memset(&G, 0, sizeof(G));
    G.Nt = Nt;
    G.Lt = 2 * Nt;
    G.w = w;
    G.D = w <= 12 ? 10 : 12;
    G.az_hi = (float)az;
    G.az_lo = (float)(az - (double)G.az_hi);
    G.sqrt_az = (float)std::sqrt(az);
    G.scale = 1.f;
    G.apply_weights = 0;
    G.band_mask = 0;
    return G;
}

extern "C" {
// nu_l = sign(l) sqrt(axy + az l^2) as hi + lo (axy given as a float pair)
void host_nu_abs(double az, float axy_hi, float axy_lo, int l, float* hi, float* lo) {
    const Geo G = geo(64, az, 12);
    const FF v = nu_abs(G, make_float2(axy_hi, axy_lo), l);
    *hi = v.hi;
    *lo = v.lo;
}

// B: the line's oversampled spectrum, Lt = 2 Nt complex values (interleaved);
// out: the NER values at l = l0 .. l0 + nl - 1 (interleaved complex)
int host_ner_values(int kind, int w, int Nt, double az, float axy_hi, float axy_lo, int j0, int l0, int nl,
                    const float* B, float* out) {
    if (w < 4 || w > 16 || (w & 1)) return -1;
    const Geo G = geo(Nt, az, w);
    const Window W = make_window(kind, w, 2.0);
    std::vector<double> cd;
    win_tap_polys(W, G.D, cd);
    TapPoly P;
    std::memset(&P, 0, sizeof(P));
    for (int k = 0; k < w; ++k)
        for (int d = 0; d <= G.D; ++d) P.c[k * (G.D + 1) + d] = (float)cd[(size_t)k * (G.D + 1) + d];
    const int Lt = G.Lt;
    std::vector<float2> Bf((size_t)padded_len(Lt) + 16);
    for (int p = 0; p < Lt; ++p) Bf[padx(p)] = make_float2(B[2 * p], B[2 * p + 1]);
    for (int i = 0; i < nl; ++i) {
        float2 v;
        const float2 axy = make_float2(axy_hi, axy_lo);
#define NEDNER_HOST_NER(WW, DD) v = ner_value<WW, DD>(G, P, axy, j0 != 0, l0 + i, Bf.data(), 0, 0);
        switch (w) {
            case 4: NEDNER_HOST_NER(4, 10) break;
            case 6: NEDNER_HOST_NER(6, 10) break;
            case 8: NEDNER_HOST_NER(8, 10) break;
            case 10: NEDNER_HOST_NER(10, 10) break;
            case 12: NEDNER_HOST_NER(12, 10) break;
            case 14: NEDNER_HOST_NER(14, 12) break;
            default: NEDNER_HOST_NER(16, 12) break;
        }
#undef NEDNER_HOST_NER
        out[2 * i] = v.x;
        out[2 * i + 1] = v.y;
    }
    return 0;
}
}

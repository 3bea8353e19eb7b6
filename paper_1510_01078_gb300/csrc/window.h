// Interpolation windows of the NED- and NER-NUFFT (Sec. 3.1-3.2), host side.
//
// The paper requires a window Psi, positive on [-pi, pi] with compact support,
// whose transform is concentrated in [-K, K], and names the Kaiser-Bessel pair
// as the usual choice without giving its parameters.  Here the window lives on
// the oversampled grid (unit spacing) with support |u| <= w/2, w = 2K taps:
//
//   Kaiser-Bessel  phi(u) = I0(beta sqrt(1 - (2u/w)^2)) / I0(beta),
//                  beta = pi sqrt((w/sigma)^2 (sigma - 1/2)^2 - 0.8)
//                  (the shape parameter of Beatty, Nishimura and Pauly,
//                  IEEE TMI 24(6), 2005, for oversampling sigma);
//   Gaussian       phi(u) = exp(-u^2 / (2 tau^2)),
//                  tau^2 = w / (4 pi sqrt(1 - 1/sigma))
//                  (truncation and aliasing errors balanced).
//
// Deconvolution uses the continuous transform phihat(f) = int phi(u)
// exp(-2 pi i f u) du, computed by Gauss-Legendre quadrature in FP64 (the
// analytic KB transform is not needed).
#pragma once

#include <vector>

namespace nedner {

struct Window {
    int kind = 0;        // 0 KB, 1 Gauss
    int w = 12;          // taps
    double sigma = 2.0;  // oversampling
    double beta = 0.0;   // KB shape
    double tau2 = 0.0;   // Gauss variance (grid units^2)
};

Window make_window(int kind, int w, double sigma);
double win_phi(const Window& W, double u);     // window value
double win_dphi(const Window& W, double u);    // d phi / du
double win_phihat(const Window& W, double f);  // continuous transform at f (cycles per grid step)

// Monomial coefficients, in s = 2 t - 1, of degree-D polynomials P_k with
// P_k(s) ~ phi(t + w/2 - 1 - k), t in [0, 1), for each tap k = 0..w-1
// (Chebyshev interpolation in FP64).  Layout coef[k * (D + 1) + d].
// Returns the largest deviation seen on a fine sample of t in (0, 1),
// relative to max |phi|.
double win_tap_polys(const Window& W, int D, std::vector<double>& coef);

}  // namespace nedner

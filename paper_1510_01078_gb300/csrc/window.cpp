// Window functions of the NUFFT stages (Sec. 3.1-3.2), host side, FP64.
#include "window.h"

#include <cmath>

namespace nedner {

namespace {

const double kPi = 3.14159265358979323846264338327950288;

// I0(z) = sum_k (z^2/4)^k / (k!)^2 (power series of the definition).
double bessel_i0(double z) {
    double q = 0.25 * z * z, term = 1.0, sum = 1.0;
    for (int k = 1; k < 200; ++k) {
        term *= q / ((double)k * (double)k);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

// I1(z) / z = (1/2) sum_k (z^2/4)^k / (k! (k+1)!).
double bessel_i1_over_z(double z) {
    double q = 0.25 * z * z, term = 0.5, sum = 0.5;
    for (int k = 1; k < 200; ++k) {
        term *= q / ((double)k * (double)(k + 1));
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& wt) {
    x.assign(n, 0.0);
    wt.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            // p1 = P_n(z), p0 = P_{n-1}(z)
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = -z;
        x[n - 1 - i] = z;
        wt[i] = wt[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

struct Quad {
    std::vector<double> x, w;
    Quad() { gauss_legendre(256, x, w); }
};

const Quad& quad() {
    static Quad q;
    return q;
}

}  // namespace

Window make_window(int kind, int w, double sigma) {
    Window W;
    W.kind = kind;
    W.w = w;
    W.sigma = sigma;
    double a = (double)w / sigma * (sigma - 0.5);
    W.beta = kPi * std::sqrt(std::fmax(a * a - 0.8, 1e-6));
    W.tau2 = (double)w / (4.0 * kPi * std::sqrt(1.0 - 1.0 / sigma));
    return W;
}

double win_phi(const Window& W, double u) {
    double h = 0.5 * W.w;
    if (std::fabs(u) >= h) return 0.0;
    if (W.kind == 0) {
        double x = u / h;
        return bessel_i0(W.beta * std::sqrt(1.0 - x * x)) / bessel_i0(W.beta);
    }
    return std::exp(-u * u / (2.0 * W.tau2));
}

double win_dphi(const Window& W, double u) {
    double h = 0.5 * W.w;
    if (std::fabs(u) >= h) return 0.0;
    if (W.kind == 0) {
        double x = u / h;
        double z = W.beta * std::sqrt(1.0 - x * x);
        // d/du I0(z) = I1(z) dz/du, dz/du = -beta^2 x / (z h)
        return -bessel_i1_over_z(z) * W.beta * W.beta * x / h / bessel_i0(W.beta);
    }
    return -u / W.tau2 * std::exp(-u * u / (2.0 * W.tau2));
}

double win_phihat(const Window& W, double f) {
    // phi is even: phihat(f) = 2 int_0^{w/2} phi(u) cos(2 pi f u) du
    const Quad& q = quad();
    double h = 0.5 * W.w, s = 0.0;
    for (size_t i = 0; i < q.x.size(); ++i) {
        double u = 0.5 * h * (q.x[i] + 1.0);
        s += q.w[i] * win_phi(W, u) * std::cos(2.0 * kPi * f * u);
    }
    return 2.0 * 0.5 * h * s;
}

double win_tap_polys(const Window& W, int D, std::vector<double>& coef) {
    const int w = W.w, n = D + 1;
    coef.assign((size_t)w * n, 0.0);
    // monomial coefficients of T_0..T_D
    std::vector<std::vector<double>> T(n, std::vector<double>(n, 0.0));
    T[0][0] = 1.0;
    if (n > 1) T[1][1] = 1.0;
    for (int d = 2; d < n; ++d) {
        for (int i = 0; i < n; ++i) {
            double v = -T[d - 2][i];
            if (i > 0) v += 2.0 * T[d - 1][i - 1];
            T[d][i] = v;
        }
    }
    double fmax = 0.0, errmax = 0.0;
    for (int k = 0; k < w; ++k) {
        // values at Chebyshev nodes s_i = cos(pi (i + 1/2) / n)
        std::vector<double> f(n), c(n, 0.0);
        for (int i = 0; i < n; ++i) {
            double s = std::cos(kPi * (i + 0.5) / n);
            double t = 0.5 * (s + 1.0);
            f[i] = win_phi(W, t + 0.5 * w - 1.0 - k);
        }
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int i = 0; i < n; ++i) acc += f[i] * std::cos(kPi * j * (i + 0.5) / n);
            c[j] = acc * (j == 0 ? 1.0 : 2.0) / n;
        }
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) coef[(size_t)k * n + i] += c[j] * T[j][i];
        // t in the open interval (0, 1): at t = 0 the last tap sits on the
        // support edge, where phi is 0 by convention and the polynomial gives
        // the one-sided limit 1/I0(beta), the window's own truncation step
        for (int i = 0; i <= 400; ++i) {
            double t = (i + 0.5) / 401.0;
            double s = 2.0 * t - 1.0, p = 0.0;
            for (int d = D; d >= 0; --d) p = p * s + coef[(size_t)k * n + d];
            double ref = win_phi(W, t + 0.5 * w - 1.0 - k);
            fmax = std::fmax(fmax, std::fabs(ref));
            errmax = std::fmax(errmax, std::fabs(p - ref));
        }
    }
    return fmax > 0 ? errmax / fmax : errmax;
}

}  // namespace nedner

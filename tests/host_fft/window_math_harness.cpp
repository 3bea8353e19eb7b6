// C entry points over the plan's window code (csrc/window.cpp, plain C++) for
// host tests of the window, its derivative, its continuous transform and the
// NER tap polynomials.  Test infrastructure only.
#include <vector>

#include "window.h"

using namespace nedner;

extern "C" {
double hw_phi(int kind, int w, double sigma, double u) { return win_phi(make_window(kind, w, sigma), u); }
double hw_dphi(int kind, int w, double sigma, double u) { return win_dphi(make_window(kind, w, sigma), u); }
double hw_phihat(int kind, int w, double sigma, double f) { return win_phihat(make_window(kind, w, sigma), f); }
double hw_beta(int w, double sigma) { return make_window(0, w, sigma).beta; }
double hw_tau2(int w, double sigma) { return make_window(1, w, sigma).tau2; }
// coef: [w][D + 1]; returns the fit's largest deviation relative to max |phi|
double hw_tap_polys(int kind, int w, double sigma, int D, double* coef) {
    std::vector<double> c;
    const double err = win_tap_polys(make_window(kind, w, sigma), D, c);
    for (size_t i = 0; i < c.size(); ++i) coef[i] = c[i];
    return err;
}
}

/*
 * FP64 reference ("oracle") for the NEDNER reconstruction of Schmid et al.,
 * "Non-Equispaced Grid Sampling in Photoacoustics with a Non-Uniform FFT"
 * (arXiv:1510.01078).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; it is used by the test-suite, by the smoke check and by the
 * CPU-baseline leg of the benchmark.  It shares no code with the CUDA library.
 *
 * Every routine is a direct, unblocked evaluation of one sum of the
 * discretised inversion formula (Sec. 2, Eq. disc_rec) or of its transpose.
 * No window, no oversampling and no FFT appear here: the non-uniform sums are
 * written out term by term in double precision.  The only rewriting used is
 * exp(a+b) = exp(a) exp(b) to evaluate the separable lateral exponent from two
 * one-dimensional tables.
 *
 * Layouts (all row-major, complex numbers interleaved re,im):
 *   xy   [M][2]            sensor positions x_m, y_m (metres)
 *   w    [M]               per-sensor factor (h_m / (dx dy) in Eq. disc_rec)
 *   g    [M][Nt]           sensor time series, n fastest
 *   G    [njx][njy][Nt][2] lateral spectrum of the data
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double TWO_PI = 6.283185307179586476925286766559;

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* exp(-2 pi i k u) for k in ks[], u in us[]:  E[a][m] */
static double* exp_table(int nk, const int* ks, int64_t M, const double* xy,
                         int comp, double extent, double sign) {
    double* E = (double*)malloc(sizeof(double) * 2 * (size_t)nk * (size_t)M);
    if (!E) return NULL;
#pragma omp parallel for schedule(static)
    for (int a = 0; a < nk; ++a) {
        for (int64_t m = 0; m < M; ++m) {
            double ph = sign * TWO_PI * ((double)ks[a] * xy[2 * m + comp] / extent);
            E[2 * ((size_t)a * M + m) + 0] = cos(ph);
            E[2 * ((size_t)a * M + m) + 1] = sin(ph);
        }
    }
    return E;
}

/*
 * NED sum of Eq. disc_rec (Sec. 2; Eq. NUDFT2 of Sec. 3.2):
 *   G[a][b][n] = sum_m w[m] g[m][n] exp(-2 pi i (jx[a] x_m / X + jy[b] y_m / Y))
 * The paper writes the phase as j.x_m / M; read as j.x_m / X with x_m in
 * metres (the discrete Fourier exponent of the grid Delta_x G_x).
 * Returns 0 on success, -1 on allocation failure.
 */
int orc_ned(int64_t M, const double* xy, const double* w, int Nt, const double* g,
            double X, double Y, int njx, const int* jx, int njy, const int* jy,
            double* G, int nthreads) {
    set_threads(nthreads);
    double* Ex = exp_table(njx, jx, M, xy, 0, X, -1.0);
    double* Ey = exp_table(njy, jy, M, xy, 1, Y, -1.0);
    if (!Ex || !Ey) { free(Ex); free(Ey); return -1; }
    int failed = 0;
#pragma omp parallel
    {
        double* acc = (double*)malloc(sizeof(double) * 2 * (size_t)Nt);
        if (!acc) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for collapse(2) schedule(dynamic, 1)
        for (int a = 0; a < njx; ++a) {
            for (int b = 0; b < njy; ++b) {
                if (!acc) continue;
                for (int n = 0; n < 2 * Nt; ++n) acc[n] = 0.0;
                for (int64_t m = 0; m < M; ++m) {
                    double er = Ex[2 * ((size_t)a * M + m)], ei = Ex[2 * ((size_t)a * M + m) + 1];
                    double fr = Ey[2 * ((size_t)b * M + m)], fi = Ey[2 * ((size_t)b * M + m) + 1];
                    /* exp(-2 pi i (jx x + jy y)) = exp(-2 pi i jx x) exp(-2 pi i jy y) */
                    double pr = (er * fr - ei * fi) * w[m];
                    double pi = (er * fi + ei * fr) * w[m];
                    const double* gm = g + (size_t)m * Nt;
                    for (int n = 0; n < Nt; ++n) {
                        acc[2 * n + 0] += pr * gm[n];
                        acc[2 * n + 1] += pi * gm[n];
                    }
                }
                double* out = G + 2 * (((size_t)a * njy + b) * (size_t)Nt);
                for (int n = 0; n < 2 * Nt; ++n) out[n] = acc[n];
            }
        }
        free(acc);
    }
    free(Ex);
    free(Ey);
    return failed ? -1 : 0;
}

/*
 * NER sum of Eq. disc_rec (Sec. 2; Eq. NUDFT1 of Sec. 3.1), one line at a time:
 *   F[j][l] = sum_{n=0}^{Nt-1} G[j][n] exp(-2 pi i nu[j][l] n / Nt)
 * with nu the non-equispaced temporal frequency of the kappa mapping.
 * G holds nn columns per line, column i being time sample ns[i] (ns = NULL:
 * all Nt samples in order); samples not listed are zero and add nothing.
 */
void orc_ner(int64_t nlines, int Nt, int nn, const int* ns, const double* G, int nl,
             const double* nu, double* F, int nthreads) {
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < nlines; ++j) {
        const double* Gj = G + 2 * (size_t)j * nn;
        for (int l = 0; l < nl; ++l) {
            double v = nu[(size_t)j * nl + l];
            double sr = 0.0, si = 0.0;
            for (int i = 0; i < nn; ++i) {
                int n = ns ? ns[i] : i;
                double ph = -TWO_PI * (v * (double)n / (double)Nt);
                double c = cos(ph), s = sin(ph);
                sr += Gj[2 * i] * c - Gj[2 * i + 1] * s;
                si += Gj[2 * i] * s + Gj[2 * i + 1] * c;
            }
            F[2 * ((size_t)j * nl + l) + 0] = sr;
            F[2 * ((size_t)j * nl + l) + 1] = si;
        }
    }
}

/*
 * Transpose (conjugate transpose) of orc_ner:
 *   T[j][n] = sum_l exp(+2 pi i nu[j][l] n / Nt) P[j][l]
 */
void orc_ner_adj(int64_t nlines, int Nt, const double* P, int nl, const double* nu,
                 double* T, int nthreads) {
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < nlines; ++j) {
        for (int n = 0; n < Nt; ++n) {
            double sr = 0.0, si = 0.0;
            for (int l = 0; l < nl; ++l) {
                double v = nu[(size_t)j * nl + l];
                double ph = TWO_PI * (v * (double)n / (double)Nt);
                double c = cos(ph), s = sin(ph);
                double pr = P[2 * ((size_t)j * nl + l)], pi = P[2 * ((size_t)j * nl + l) + 1];
                sr += pr * c - pi * s;
                si += pr * s + pi * c;
            }
            T[2 * ((size_t)j * Nt + n) + 0] = sr;
            T[2 * ((size_t)j * Nt + n) + 1] = si;
        }
    }
}

/*
 * Transpose of orc_ned restricted to a real output (the data are real):
 *   out[m][n] = w[m] * Re sum_{a,b} exp(+2 pi i (jx[a] x_m/X + jy[b] y_m/Y)) T[a][b][n]
 */
int orc_ned_adj(int64_t M, const double* xy, const double* w, int Nt,
                double X, double Y, int njx, const int* jx, int njy, const int* jy,
                const double* T, double* out, int nthreads) {
    set_threads(nthreads);
    double* Ex = exp_table(njx, jx, M, xy, 0, X, +1.0);
    double* Ey = exp_table(njy, jy, M, xy, 1, Y, +1.0);
    if (!Ex || !Ey) { free(Ex); free(Ey); return -1; }
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t m = 0; m < M; ++m) {
        double* om = out + (size_t)m * Nt;
        for (int n = 0; n < Nt; ++n) om[n] = 0.0;
        for (int a = 0; a < njx; ++a) {
            double er = Ex[2 * ((size_t)a * M + m)], ei = Ex[2 * ((size_t)a * M + m) + 1];
            for (int b = 0; b < njy; ++b) {
                double fr = Ey[2 * ((size_t)b * M + m)], fi = Ey[2 * ((size_t)b * M + m) + 1];
                double pr = er * fr - ei * fi;
                double pi = er * fi + ei * fr;
                const double* Tab = T + 2 * (((size_t)a * njy + b) * (size_t)Nt);
                for (int n = 0; n < Nt; ++n)
                    om[n] += pr * Tab[2 * n] - pi * Tab[2 * n + 1];
            }
        }
        for (int n = 0; n < Nt; ++n) om[n] *= w[m];
    }
    free(Ex);
    free(Ey);
    return 0;
}

/*
 * Derivative of the NED exponent with respect to the sensor position, paired
 * with the data (the sensor-position gradient of a loss):
 *   out[m][0] = w[m] sum_n g[m][n] Re sum_{a,b} (-2 pi i jx[a]/X) e_{ab}(x_m) S[a][b][n]
 *   out[m][1] = w[m] sum_n g[m][n] Re sum_{a,b} (-2 pi i jy[b]/Y) e_{ab}(x_m) S[a][b][n]
 * with e_{ab}(x_m) = exp(-2 pi i (jx[a] x_m/X + jy[b] y_m/Y)).
 */
int orc_ned_grad(int64_t M, const double* xy, const double* w, int Nt, const double* g,
                 double X, double Y, int njx, const int* jx, int njy, const int* jy,
                 const double* S, double* out, int nthreads) {
    set_threads(nthreads);
    double* Ex = exp_table(njx, jx, M, xy, 0, X, -1.0);
    double* Ey = exp_table(njy, jy, M, xy, 1, Y, -1.0);
    if (!Ex || !Ey) { free(Ex); free(Ey); return -1; }
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t m = 0; m < M; ++m) {
        const double* gm = g + (size_t)m * Nt;
        double dx_acc = 0.0, dy_acc = 0.0;
        for (int a = 0; a < njx; ++a) {
            double er = Ex[2 * ((size_t)a * M + m)], ei = Ex[2 * ((size_t)a * M + m) + 1];
            for (int b = 0; b < njy; ++b) {
                double fr = Ey[2 * ((size_t)b * M + m)], fi = Ey[2 * ((size_t)b * M + m) + 1];
                double pr = er * fr - ei * fi;
                double pi = er * fi + ei * fr;
                const double* Sab = S + 2 * (((size_t)a * njy + b) * (size_t)Nt);
                /* q = sum_n g[m][n] S[a][b][n] */
                double qr = 0.0, qi = 0.0;
                for (int n = 0; n < Nt; ++n) {
                    qr += gm[n] * Sab[2 * n];
                    qi += gm[n] * Sab[2 * n + 1];
                }
                /* e * q */
                double zr = pr * qr - pi * qi;
                double zi = pr * qi + pi * qr;
                /* Re((-2 pi i k / X) z) = 2 pi k / X * Im(z) */
                dx_acc += TWO_PI * (double)jx[a] / X * zi;
                dy_acc += TWO_PI * (double)jy[b] / Y * zi;
            }
        }
        out[2 * m + 0] = w[m] * dx_acc;
        out[2 * m + 1] = w[m] * dy_acc;
    }
    free(Ex);
    free(Ey);
    return 0;
}

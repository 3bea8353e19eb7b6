// Runs the device FFT header (block_fft_ip) on CPU threads for tests: one
// std::thread per CUDA thread of a block, __syncthreads as a barrier.  The
// twiddle table follows the header's contract, tw[N + k] = exp(-2 pi i k / N)
// for every power of two N <= TW_N, computed here in double.  Test
// infrastructure only; nothing in the library uses it.
#include <barrier>
#include <cmath>
#include <memory>
#include <thread>
#include <vector>

#include "fft.cuh"

thread_local HostDim3 threadIdx;
HostDim3 blockDim;
static std::barrier<>* g_bar = nullptr;
void __syncthreads() { g_bar->arrive_and_wait(); }

using namespace nedner;

static std::vector<float2> twiddles() {
    std::vector<float2> tw(2 * TW_N);
    tw[0] = make_float2(1.f, 0.f);
    for (int N = 1; N <= TW_N; N *= 2)
        for (int k = 0; k < N; ++k) {
            const double a = -2.0 * 3.14159265358979323846 * (double)k / N;
            tw[N + k] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
    return tw;
}

template <int PER, bool ZP>
static void run(float2* buf, int N, int nb, int dir, const float2* tw, bool skip_r2, int nt) {
    std::barrier<> bar(nt);
    g_bar = &bar;
    blockDim.x = (unsigned)nt;
    std::vector<std::thread> th;
    th.reserve(nt);
    for (int t = 0; t < nt; ++t)
        th.emplace_back([=] {
            threadIdx.x = (unsigned)t;
            block_fft_ip<PER, ZP>(buf, N, nb, dir, tw, skip_r2);
        });
    for (auto& x : th) x.join();
    g_bar = nullptr;
}

// in/out: interleaved complex, point p of column b at 2 (p nb + b).  With zp,
// points N/4 <= p < 3N/4 of the buffer are filled with NaN (the pass must not
// read them; the input there is zero by contract).  Returns 0, or -1 for a
// configuration the header does not support.
extern "C" int host_block_fft(int N, int nb, int dir, int per, int nt, int skip_r2, int zp, const float* in,
                              float* out) {
    if (N < 2 || N > TW_N || (N & (N - 1)) || nb < 1 || (nb & (nb - 1))) return -1;
    if ((long)N * nb > (long)per * nt || (zp && N < 16)) return -1;
    static const std::vector<float2> tw = twiddles();
    std::vector<float2> buf((size_t)padded_len(N * nb) + 16, make_float2(NAN, NAN));
    for (int p = 0; p < N; ++p)
        for (int b = 0; b < nb; ++b) {
            if (zp && p >= N / 4 && p < 3 * N / 4) continue;
            const int a = p * nb + b;
            buf[padx(a)] = make_float2(in[2 * a], in[2 * a + 1]);
        }
    if (per == 16 && !zp) run<16, false>(buf.data(), N, nb, dir, tw.data(), skip_r2, nt);
    else if (per == 16) run<16, true>(buf.data(), N, nb, dir, tw.data(), skip_r2, nt);
    else if (per == 32 && !zp) run<32, false>(buf.data(), N, nb, dir, tw.data(), skip_r2, nt);
    else if (per == 32) run<32, true>(buf.data(), N, nb, dir, tw.data(), skip_r2, nt);
    else return -1;
    for (int a = 0; a < N * nb; ++a) {
        out[2 * a] = buf[padx(a)].x;
        out[2 * a + 1] = buf[padx(a)].y;
    }
    return 0;
}

// The complex-to-real pair formation (c2r_pair) for a half spectrum X[0..N/2]
// (interleaved complex): out is Z[0..N/2-1] (interleaved), formed pair by pair
// for k = 0..N/4 as the x complex-to-real kernel does.
extern "C" int host_c2r_pairs(int N, const float* X, float* out) {
    if (N < 4 || N > TW_N || (N & (N - 1))) return -1;
    static const std::vector<float2> tw = twiddles();
    const int H = N / 2;
    for (int k = 0; k <= H / 2; ++k) {
        float2 zk, zm;
        c2r_pair(make_float2(X[2 * k], X[2 * k + 1]), make_float2(X[2 * (H - k)], X[2 * (H - k) + 1]), k, N,
                 tw.data(), zk, zm);
        out[2 * k] = zk.x;
        out[2 * k + 1] = zk.y;
        if (k > 0 && k < H / 2) {
            out[2 * (H - k)] = zm.x;
            out[2 * (H - k) + 1] = zm.y;
        }
    }
    return 0;
}

// The real-to-complex unpack (r2c_unpack): Z is FFT_{N/2} of the packed real
// samples (interleaved complex); out is X[0..N/2] (interleaved).
extern "C" int host_r2c_unpack(int N, const float* Z, float* out) {
    if (N < 4 || N > TW_N || (N & (N - 1))) return -1;
    static const std::vector<float2> tw = twiddles();
    const int H = N / 2;
    for (int k = 0; k <= H; ++k) {
        const int a = k & (H - 1), b = (H - k) & (H - 1);
        const float2 X = r2c_unpack(make_float2(Z[2 * a], Z[2 * a + 1]), make_float2(Z[2 * b], Z[2 * b + 1]), k, N,
                                    tw.data());
        out[2 * k] = X.x;
        out[2 * k + 1] = X.y;
    }
    return 0;
}

// Host check of the arithmetic the CUDA kernels use (csrc/hostdev.h): the
// in-place FFT passes (decimation in frequency / time) with their position
// maps, the real-FFT packing pair on digit-reversed data, the column
// kernel's transform pair around a pointwise product, the shared-memory
// swizzles and the B-spline weights.
// Compiled with g++ by tests/test_hostdev.py; prints "name value"
// lines (errors) that the test compares with thresholds.
#include <cmath>
#include <complex>
#include <cstdio>
#include <random>
#include <vector>

#include "hostdev.h"

using namespace hr;
typedef std::complex<double> cd;

// The kernels' in-place passes (dif_plan order), run sequentially on a
// sequence in natural order: forward passes leave digit-reversed order,
// inverse passes take it.
template <int R>
static void dif_pass(std::vector<cf>& a, int S, const cf* T, int b, bool inverse) {
    const int base = dif_base(R, S, b);
    const int m = b % S;
    cf x[R];
    for (int r = 0; r < R; ++r) x[r] = a[base + r * S];
    if (!inverse) {
        dft_small<R>(x, -1);
        if (S > 1)
            for (int k = 1; k < R; ++k) x[k] = cmul(x[k], T[(k - 1) * S + m]);
    } else {
        if (S > 1)
            for (int k = 1; k < R; ++k) x[k] = cmulc(x[k], T[(k - 1) * S + m]);
        dft_small<R>(x, +1);
    }
    for (int r = 0; r < R; ++r) a[base + r * S] = x[r];
}

static void dif_pass_any(int R, std::vector<cf>& a, int S, const cf* T, int b, bool inv) {
    switch (R) {
        case 16: dif_pass<16>(a, S, T, b, inv); break;
        case 12: dif_pass<12>(a, S, T, b, inv); break;
        case 10: dif_pass<10>(a, S, T, b, inv); break;
        case 9: dif_pass<9>(a, S, T, b, inv); break;
        case 8: dif_pass<8>(a, S, T, b, inv); break;
        case 6: dif_pass<6>(a, S, T, b, inv); break;
        case 5: dif_pass<5>(a, S, T, b, inv); break;
        case 4: dif_pass<4>(a, S, T, b, inv); break;
        case 3: dif_pass<3>(a, S, T, b, inv); break;
        default: dif_pass<2>(a, S, T, b, inv); break;
    }
}

struct DifRun {
    int s, R[kMaxDifPasses], S[kMaxDifPasses];
    std::vector<cf> T;
    std::vector<int> off;
    explicit DifRun(int n) {
        s = dif_plan(n, R, S);
        T.resize(fft_dif_tables(n, nullptr) + 1);
        fft_dif_tables(n, T.data());
        int ofs = 0;
        for (int p = 0; p < s; ++p) {
            off.push_back(ofs);
            ofs += stage_table_len(S[p], R[p]);
        }
    }
    void forward(std::vector<cf>& a) const {
        for (int p = 0; p < s; ++p)
            for (int b = 0; b < (int)a.size() / R[p]; ++b) dif_pass_any(R[p], a, S[p], T.data() + off[p], b, false);
    }
    void inverse(std::vector<cf>& a) const {
        for (int p = s - 1; p >= 0; --p)
            for (int b = 0; b < (int)a.size() / R[p]; ++b) dif_pass_any(R[p], a, S[p], T.data() + off[p], b, true);
    }
};

// Forward passes read back in natural order through dif_pos, and inverse
// passes on a digit-reversed input, against a direct DFT.
static double fft_error(int n, int dir, std::mt19937& rng) {
    std::normal_distribution<double> N(0, 1);
    DifRun D(n);
    std::vector<cf> x(n);
    std::vector<cd> xd(n);
    for (int i = 0; i < n; ++i) {
        x[i] = {(float)N(rng), (float)N(rng)};
        xd[i] = cd(x[i].x, x[i].y);
    }
    std::vector<cf> y(n);
    if (dir < 0) {
        std::vector<cf> a = x;
        D.forward(a);
        for (int k = 0; k < n; ++k) y[k] = a[dif_pos(D.s, D.R, D.S, k)];
    } else {
        std::vector<cf> a(n);
        for (int k = 0; k < n; ++k) a[dif_pos(D.s, D.R, D.S, k)] = x[k];
        D.inverse(a);
        y = a;
    }
    double num = 0, den = 0;
    for (int k = 0; k < n; ++k) {
        cd acc = 0;
        for (int i = 0; i < n; ++i) acc += xd[i] * std::polar(1.0, dir * 2 * M_PI * (double)((long)k * i % n) / n);
        num += std::norm(acc - cd(y[k].x, y[k].y));
        den += std::norm(acc);
    }
    return std::sqrt(num / den);
}

// The row kernels' real FFT: the packed pairs through the forward passes,
// then r2c_post_at at the positions of k and M - k; returns the error of
// X_mine against 2 X_true (the kernels omit the factors 1/2).
static double rfft_error(int P, std::mt19937& rng) {
    std::normal_distribution<double> N(0, 1);
    const int M = P / 2;
    DifRun D(M);
    std::vector<double> x(P);
    for (auto& v : x) v = N(rng);
    std::vector<cf> z(M);
    for (int n = 0; n < M; ++n) z[n] = {(float)x[2 * n], (float)x[2 * n + 1]};
    D.forward(z);
    std::vector<cf> twP(M + 1);
    for (int k = 0; k <= M; ++k) twP[k] = {(float)std::cos(-2 * M_PI * k / P), (float)std::sin(-2 * M_PI * k / P)};
    double num = 0, den = 0;
    for (int k = 0; k < M; ++k) {
        cd acc = 0;
        for (int n = 0; n < P; ++n) acc += x[n] * std::polar(1.0, -2 * M_PI * (double)((long)k * n % P) / P);
        const int pk = dif_pos(D.s, D.R, D.S, k), pmk = dif_pos(D.s, D.R, D.S, k == 0 ? 0 : M - k);
        cf X = r2c_post_at(z.data(), pk, pmk, k, twP.data());
        num += std::norm(cd(X.x, X.y) - 2.0 * acc);
        den += std::norm(2.0 * acc);
    }
    return std::sqrt(num / den);
}

// Inverse: half spectrum with bins 0..kmax (X0 real), c2r_pre_vals on the
// pairs (k, M - k), k <= M/2, written at their positions, inverse passes;
// returns the error of x_mine against P * irfft(X).
static double irfft_error(int P, int kmax, std::mt19937& rng) {
    std::normal_distribution<double> N(0, 1);
    const int M = P / 2;
    DifRun D(M);
    std::vector<cd> Xd(M + 1, 0.0);
    for (int k = 0; k <= kmax; ++k) Xd[k] = cd(N(rng), k ? N(rng) : 0.0);
    auto X = [&](int k) { return cf{(float)Xd[k].real(), (float)Xd[k].imag()}; };
    std::vector<cf> twP(M + 1);
    for (int k = 0; k <= M; ++k) twP[k] = {(float)std::cos(-2 * M_PI * k / P), (float)std::sin(-2 * M_PI * k / P)};
    std::vector<cf> z(M, cf{0.f, 0.f});
    for (int k = 0; k <= M / 2; ++k) {
        if (k == 0) {
            z[dif_pos(D.s, D.R, D.S, 0)] = c2r_pre_dc(X(0));
            continue;
        }
        cf zk, zmk;
        c2r_pre_vals(X(k), X(M - k), twP[k], zk, zmk);
        z[dif_pos(D.s, D.R, D.S, k)] = zk;
        z[dif_pos(D.s, D.R, D.S, M - k)] = zmk;
    }
    D.inverse(z);
    double num = 0, den = 0;
    for (int n = 0; n < P; ++n) {
        double acc = Xd[0].real();
        for (int k = 1; k < M; ++k) acc += 2.0 * (Xd[k] * std::polar(1.0, 2 * M_PI * (double)((long)k * n % P) / P)).real();
        const double mine = (n & 1) ? z[n >> 1].y : z[n >> 1].x;
        num += (mine - acc) * (mine - acc);
        den += acc * acc;
    }
    return std::sqrt(num / den);
}

// The column kernel's transform pair: forward passes, product with a
// spectrum K at each position's frequency, inverse passes; returns the
// relative L2 error against n * IDFT(K .* DFT(x)) in FP64, and counts
// positions whose frequency map is not a permutation or not inverted by
// dif_pos.
static double dif_conv_error(int n, std::mt19937& rng, int& bad_freq) {
    std::normal_distribution<double> N(0, 1);
    DifRun D(n);
    std::vector<cf> a(n), K(n);
    std::vector<cd> xd(n), Kd(n);
    for (int i = 0; i < n; ++i) {
        a[i] = {(float)N(rng), (float)N(rng)};
        xd[i] = cd(a[i].x, a[i].y);
        K[i] = {(float)N(rng), (float)N(rng)};
        Kd[i] = cd(K[i].x, K[i].y);
    }
    D.forward(a);
    std::vector<int> seen(n, 0);
    for (int pos = 0; pos < n; ++pos) {
        const int f = dif_freq(D.s, D.R, D.S, pos);
        if (f < 0 || f >= n || seen[f]++ || dif_pos(D.s, D.R, D.S, f) != pos) ++bad_freq;
        else a[pos] = cmul(a[pos], K[f]);
    }
    D.inverse(a);
    std::vector<cd> X(n);
    for (int k = 0; k < n; ++k) {
        cd acc = 0;
        for (int i = 0; i < n; ++i) acc += xd[i] * std::polar(1.0, -2 * M_PI * (double)((long)k * i % n) / n);
        X[k] = acc * Kd[k];
    }
    double num = 0, den = 0;
    for (int i = 0; i < n; ++i) {
        cd acc = 0;
        for (int k = 0; k < n; ++k) acc += X[k] * std::polar(1.0, 2 * M_PI * (double)((long)k * i % n) / n);
        num += std::norm(acc - cd(a[i].x, a[i].y));
        den += std::norm(acc);
    }
    return std::sqrt(num / den);
}

static double b3_error() {
    double e = 0;
    for (int i = 0; i <= 1000; ++i) {
        const float f = i / 1000.0f;
        float w[4];
        b3_weights(f, w);
        auto B3 = [](double x) {
            x = std::fabs(x);
            return x < 1 ? 2.0 / 3 - x * x + 0.5 * x * x * x : (x < 2 ? (2 - x) * (2 - x) * (2 - x) / 6 : 0.0);
        };
        for (int a = 0; a < 4; ++a) e = std::max(e, std::fabs(w[a] - B3(f + 1 - a)));
        e = std::max(e, std::fabs((double)w[0] + w[1] + w[2] + w[3] - 1.0));
    }
    return e;
}

// The quintic weights against the truncated-power definition of B5.
static double b5_error() {
    auto B5 = [](double x) {
        const double a = std::fabs(x);
        auto tp = [](double u) { return u > 0 ? u * u * u * u * u : 0.0; };
        return (tp(3 - a) - 6 * tp(2 - a) + 15 * tp(1 - a)) / 120.0;
    };
    double e = 0;
    for (int i = 0; i <= 1000; ++i) {
        const float f = i / 1000.0f;
        float w[6];
        b5_weights(f, w);
        double sum = 0;
        for (int d = 0; d < 6; ++d) {
            e = std::max(e, std::fabs(w[d] - B5(f + 2 - d)));
            sum += w[d];
        }
        e = std::max(e, std::fabs(sum - 1.0));
    }
    return e;
}

int main() {
    std::mt19937 rng(1604);
    double e = 0;
    for (int n : {2, 3, 4, 5, 6, 8, 9, 10, 12, 16, 18, 20, 24, 32, 36, 40, 48, 64, 72, 80, 96, 128, 144, 160, 192,
                  256, 288, 320, 384, 512, 576, 640, 768, 1024, 1152, 1280, 1536, 2048, 2304, 2560, 3072, 4096, 5120,
                  6144})
        e = std::max(e, std::max(fft_error(n, -1, rng), fft_error(n, +1, rng)));
    std::printf("fft_rel_l2 %.3e\n", e);
    e = 0;
    for (int P : {8, 12, 18, 20, 48, 64, 80, 96, 144, 768, 1024, 2304, 2560, 3072}) e = std::max(e, rfft_error(P, rng));
    std::printf("rfft_rel_l2 %.3e\n", e);
    e = 0;
    for (int P : {8, 12, 18, 20, 48, 64, 80, 96, 144, 768, 1024, 2304, 2560, 3072})
        e = std::max(e, irfft_error(P, P / 2 - 1, rng));
    for (int P : {64, 768}) e = std::max(e, irfft_error(P, P / 5, rng));
    std::printf("irfft_rel_l2 %.3e\n", e);
    std::printf("b3_weights %.3e\n", b3_error());
    std::printf("b5_weights %.3e\n", b5_error());
    e = 0;
    int bad_freq = 0;
    for (int n : {2, 3, 4, 5, 6, 8, 9, 10, 12, 16, 18, 20, 24, 32, 36, 40, 48, 64, 72, 80, 96, 128, 144, 160, 192,
                  256, 288, 320, 384, 512, 576, 640, 768, 1024, 1152, 1280, 1536, 2048, 2304, 2560, 3072, 4096, 5120,
                  6144})
        e = std::max(e, dif_conv_error(n, rng, bad_freq));
    std::printf("dif_conv_rel_l2 %.3e\n", e);
    std::printf("dif_freq_violations %d\n", bad_freq);
    // the layout swizzle is a permutation of [0, n) for every FFT length used
    int bad = 0, nlen = 0;
    for (int n = 1; n <= 6144; ++n) {
        int rad[32];
        if (fft_radices(n, rad) < 0 || (n % 3 == 0 ? n > 6144 : n % 5 == 0 ? n > 5120 : n > 4096)) continue;
        ++nlen;
        std::vector<int> seen(n, 0), seen2(n, 0);
        for (int i = 0; i < n; ++i) {
            const int p = sw(i), q = swc(i);
            if (p < 0 || p >= n || seen[p]++) ++bad;
            if (q < 0 || q >= n || seen2[q]++) ++bad;
        }
    }
    std::printf("swizzle_violations %d\n", bad);
    std::printf("fft_lengths %d\n", nlen);
    return 0;
}

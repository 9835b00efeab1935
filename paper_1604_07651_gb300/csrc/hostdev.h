// Pure arithmetic shared by the device kernels and by the host unit tests of
// those kernels (compiled with g++ for the tests, nvcc for the library):
// * cubic B-spline tap weights (the B3 of Eq. (14)-(17));
// * the in-register DFTs and the in-place FFT passes, with their position
//   maps (the FFTs of Eq. (7), (16)-(17));
// * the packing of a real FFT into a complex FFT of half the length.
#pragma once

#include <math.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define HD __host__ __device__ __forceinline__
#define HD_UNROLL _Pragma("unroll")
#else
#define HD inline
#define HD_UNROLL
#endif

namespace hr {

struct cf { float x, y; };             // complex float

// Cubic B-spline weights of the four taps i0 .. i0+3, i0 = floor(x) - 1,
// at fractional part f = x - floor(x): B3(f+1), B3(f), B3(f-1), B3(f-2).
HD void b3_weights(float f, float w[4]) {
    float g = 1.0f - f;
    float f2 = f * f, f3 = f2 * f;
    w[0] = g * g * g * (1.0f / 6.0f);
    w[1] = (4.0f - 6.0f * f2 + 3.0f * f3) * (1.0f / 6.0f);
    w[2] = (1.0f + 3.0f * f + 3.0f * f2 - 3.0f * f3) * (1.0f / 6.0f);
    w[3] = f3 * (1.0f / 6.0f);
}

// Quintic B-spline weights of the six taps i0 .. i0+5, i0 = floor(x) - 2, at
// fractional part t: B5(t+2), B5(t+1), B5(t), B5(t-1), B5(t-2), B5(t-3), the
// pieces of (3-|x|)^5 - 6 (2-|x|)^5 + 15 (1-|x|)^5 over 120 (terms with a
// positive base only), expanded in t; weights d and 5-d are mirror images
// (t -> 1 - t).
HD void b5_weights(float t, float w[6]) {
    const float s = 1.0f - t;
    const float t2 = t * t, s2 = s * s;
    const float k = 1.0f / 120.0f;
    w[0] = s2 * s2 * s * k;
    w[5] = t2 * t2 * t * k;
    // 5 t^5 - 20 t^4 + 20 t^3 + 20 t^2 - 50 t + 26 and its mirror
    w[1] = ((((5.0f * t - 20.0f) * t + 20.0f) * t + 20.0f) * t - 50.0f) * t * k + 26.0f * k;
    w[4] = ((((5.0f * s - 20.0f) * s + 20.0f) * s + 20.0f) * s - 50.0f) * s * k + 26.0f * k;
    // -10 t^5 + 30 t^4 - 60 t^2 + 66 and its mirror
    w[2] = (((-10.0f * t + 30.0f) * t2 - 60.0f) * t2 + 66.0f) * k;
    w[3] = (((-10.0f * s + 30.0f) * s2 - 60.0f) * s2 + 66.0f) * k;
}

// B-spline weights of NT = order + 1 taps: cubic (4) or quintic (6).
template <int NT>
HD void bspline_weights(float f, float w[NT]);
template <>
HD void bspline_weights<4>(float f, float w[4]) { b3_weights(f, w); }
template <>
HD void bspline_weights<6>(float f, float w[6]) { b5_weights(f, w); }

// Shared-memory layout of every FFT buffer: element i of a sequence lives at
// sw(i). XOR-ing the low four bits with the next four spreads the strided
// stores of the first radix-16 stage (stride 16 elements) over all banks and
// keeps contiguous accesses conflict-free. A permutation within each block of
// 16 (and the identity below 16), so sw(i) < n for every length the FFT uses.
HD int sw(int i) { return i ^ ((i >> 4) & 15); }

HD cf cmul(cf a, cf b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
HD cf cmulc(cf a, cf b) { return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y}; }  // a * conj(b)
HD cf cadd(cf a, cf b) { return {a.x + b.x, a.y + b.y}; }
HD cf csub(cf a, cf b) { return {a.x - b.x, a.y - b.y}; }
HD cf cconj(cf a) { return {a.x, -a.y}; }

// In-register DFT of size R (2, 3 or 4) with sign dir (-1 forward, +1 inverse).
template <int R>
HD void dft_small(cf v[R], int dir);

template <>
HD void dft_small<2>(cf v[2], int) {
    cf a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <>
HD void dft_small<4>(cf v[4], int dir) {
    cf a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    cf b0 = cadd(v[1], v[3]), b1 = csub(v[1], v[3]);
    // b1 * (dir * i)
    cf jb1 = dir < 0 ? cf{b1.y, -b1.x} : cf{-b1.y, b1.x};
    v[0] = cadd(a0, b0);
    v[2] = csub(a0, b0);
    v[1] = cadd(a1, jb1);
    v[3] = csub(a1, jb1);
}

template <>
HD void dft_small<3>(cf v[3], int dir) {
    const float c = -0.5f;
    const float s = 0.86602540378443864676f * (float)dir;  // sin(2 pi/3) * dir
    cf t = cadd(v[1], v[2]);
    cf d = csub(v[1], v[2]);
    cf m = {v[0].x + c * t.x, v[0].y + c * t.y};
    cf id = {-s * d.y, s * d.x};  // i * s * d
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, id);
    v[2] = csub(m, id);
}

// cos(2 pi i / 16); with i a compile-time constant after unrolling, the
// switch folds to a literal (no table in local memory).
HD float cos16(int i) {
    switch (i & 15) {
        case 0: return 1.0f;
        case 1: case 15: return 0.92387953251128674f;
        case 2: case 14: return 0.70710678118654752f;
        case 3: case 13: return 0.38268343236508977f;
        case 4: case 12: return 0.0f;
        case 5: case 11: return -0.38268343236508977f;
        case 6: case 10: return -0.70710678118654752f;
        case 7: case 9: return -0.92387953251128674f;
        default: return -1.0f;
    }
}

// exp(dir * 2 pi i k / N) for the in-register DFTs of size 8 and 16.
template <int N>
HD cf unit_root(int k, int dir) {
    const int i = k * (16 / N);
    return {cos16(i), dir * cos16(i - 4)};   // sin(x) = cos(x - pi/2)
}

// exp(dir * 2 pi i m / 12) for the in-register DFTs of size 6 and 12; m is
// a compile-time constant after unrolling.
HD float cos12(int i) {
    switch (((i % 12) + 12) % 12) {
        case 0: return 1.0f;
        case 1: case 11: return 0.86602540378443864676f;   // sqrt(3)/2
        case 2: case 10: return 0.5f;
        case 3: case 9: return 0.0f;
        case 4: case 8: return -0.5f;
        case 5: case 7: return -0.86602540378443864676f;
        default: return -1.0f;
    }
}
HD cf root12(int m, int dir) { return {cos12(m), dir * cos12(m - 3)}; }

// Size 6 as 3 x 2 and size 12 as 3 x 4 (Cooley-Tukey with n = F n1 + n2,
// k = k1 + 3 k2): Y[n2][k1] = DFT3 over n1 of x[F n1 + n2], times
// W^(n2 k1), then X[k1 + 3 k2] = DFT-F over n2.
template <int F>
HD void dft_3xF(cf v[3 * F], int dir) {
    cf y[F][3];
HD_UNROLL
    for (int n2 = 0; n2 < F; ++n2) {
HD_UNROLL
        for (int n1 = 0; n1 < 3; ++n1) y[n2][n1] = v[F * n1 + n2];
        dft_small<3>(y[n2], dir);
    }
HD_UNROLL
    for (int k1 = 0; k1 < 3; ++k1) {
        cf z[F];
HD_UNROLL
        for (int n2 = 0; n2 < F; ++n2)
            z[n2] = (n2 * k1 != 0) ? cmul(y[n2][k1], root12(n2 * k1 * (12 / (3 * F)), dir)) : y[n2][k1];
        dft_small<F>(z, dir);
HD_UNROLL
        for (int k2 = 0; k2 < F; ++k2) v[k1 + 3 * k2] = z[k2];
    }
}

template <>
HD void dft_small<6>(cf v[6], int dir) { dft_3xF<2>(v, dir); }

template <>
HD void dft_small<12>(cf v[12], int dir) { dft_3xF<4>(v, dir); }

// exp(dir * 2 pi i m / 9) for m = 1, 2, 4, the twiddles of the 3 x 3 split
// (cos and sin of 40, 80 and 160 degrees).
HD cf root9(int m, int dir) {
    switch (m) {
        case 1: return {0.76604444311897803520f, dir * 0.64278760968653932632f};
        case 2: return {0.17364817766693034885f, dir * 0.98480775301220805936f};
        default: return {-0.93969262078590838405f, dir * 0.34202014332566873304f};
    }
}

// Size 9 as 3 x 3 (Cooley-Tukey with n = 3 n1 + n2, k = k1 + 3 k2):
// Y[n2][k1] = DFT3 over n1 of x[3 n1 + n2], times W9^(n2 k1), then
// X[k1 + 3 k2] = DFT3 over n2.
template <>
HD void dft_small<9>(cf v[9], int dir) {
    cf y[3][3];
HD_UNROLL
    for (int n2 = 0; n2 < 3; ++n2) {
HD_UNROLL
        for (int n1 = 0; n1 < 3; ++n1) y[n2][n1] = v[3 * n1 + n2];
        dft_small<3>(y[n2], dir);
    }
HD_UNROLL
    for (int k1 = 0; k1 < 3; ++k1) {
        cf z[3];
HD_UNROLL
        for (int n2 = 0; n2 < 3; ++n2) z[n2] = (n2 * k1 != 0) ? cmul(y[n2][k1], root9(n2 * k1, dir)) : y[n2][k1];
        dft_small<3>(z, dir);
HD_UNROLL
        for (int k2 = 0; k2 < 3; ++k2) v[k1 + 3 * k2] = z[k2];
    }
}

// Size 5 directly: with t1 = x1 + x4, t2 = x2 + x3, t3 = x1 - x4,
// t4 = x2 - x3 and c_m = cos(2 pi m / 5), s_m = sin(2 pi m / 5):
// X1,4 = x0 + c1 t1 + c2 t2 +- i dir (s1 t3 + s2 t4),
// X2,3 = x0 + c2 t1 + c1 t2 +- i dir (s2 t3 - s1 t4).
template <>
HD void dft_small<5>(cf v[5], int dir) {
    const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;   // (sqrt5 - 1)/4, -(sqrt5 + 1)/4
    const float s1 = 0.95105651629515357212f * (float)dir, s2 = 0.58778525229247312917f * (float)dir;
    const cf t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    const cf t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    const cf a1 = {v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y};
    const cf a2 = {v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y};
    const cf b1 = {s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y};
    const cf b2 = {s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y};
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = {a1.x - b1.y, a1.y + b1.x};   // a1 + i b1
    v[4] = {a1.x + b1.y, a1.y - b1.x};   // a1 - i b1
    v[2] = {a2.x - b2.y, a2.y + b2.x};
    v[3] = {a2.x + b2.y, a2.y - b2.x};
}

// cos(2 pi m / 10) and exp(dir * 2 pi i m / 10), m a compile-time constant
// after unrolling.
HD float cos10(int i) {
    switch (((i % 10) + 10) % 10) {
        case 0: return 1.0f;
        case 1: case 9: return 0.80901699437494742410f;    // (sqrt5 + 1)/4
        case 2: case 8: return 0.30901699437494742410f;    // (sqrt5 - 1)/4
        case 3: case 7: return -0.30901699437494742410f;
        case 4: case 6: return -0.80901699437494742410f;
        default: return -1.0f;
    }
}
HD float sin10(int i) {
    switch (((i % 10) + 10) % 10) {
        case 1: case 4: return 0.58778525229247312917f;    // sin 36 deg = sin 144 deg
        case 2: case 3: return 0.95105651629515357212f;    // sin 72 deg = sin 108 deg
        case 6: case 9: return -0.58778525229247312917f;
        case 7: case 8: return -0.95105651629515357212f;
        default: return 0.0f;
    }
}

// Size 10 as 5 x 2: Y[n2][k1] = DFT5 over n1 of x[2 n1 + n2], times
// W10^(n2 k1), then X[k1 + 5 k2] = DFT2 over n2.
template <>
HD void dft_small<10>(cf v[10], int dir) {
    cf y0[5], y1[5];
HD_UNROLL
    for (int n1 = 0; n1 < 5; ++n1) {
        y0[n1] = v[2 * n1];
        y1[n1] = v[2 * n1 + 1];
    }
    dft_small<5>(y0, dir);
    dft_small<5>(y1, dir);
HD_UNROLL
    for (int k1 = 0; k1 < 5; ++k1) {
        const cf t = k1 ? cmul(y1[k1], cf{cos10(k1), dir * sin10(k1)}) : y1[k1];
        v[k1] = cadd(y0[k1], t);
        v[k1 + 5] = csub(y0[k1], t);
    }
}

// Size 8 as 2 x 4: inputs x[2 n1 + n2], X[k1 + 4 k2].
template <>
HD void dft_small<8>(cf v[8], int dir) {
    cf e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft_small<4>(e, dir);
    dft_small<4>(o, dir);
HD_UNROLL
    for (int k = 0; k < 4; ++k) {
        const cf t = k ? cmul(o[k], unit_root<8>(k, dir)) : o[k];
        v[k] = cadd(e[k], t);
        v[k + 4] = csub(e[k], t);
    }
}

// Size 16 as 4 x 4: Y[n2][k1] = DFT4 over n1 of x[4 n1 + n2], times
// W16^(n2 k1), then X[k1 + 4 k2] = DFT4 over n2.
template <>
HD void dft_small<16>(cf v[16], int dir) {
    cf y[4][4];
HD_UNROLL
    for (int n2 = 0; n2 < 4; ++n2) {
HD_UNROLL
        for (int n1 = 0; n1 < 4; ++n1) y[n2][n1] = v[4 * n1 + n2];
        dft_small<4>(y[n2], dir);
    }
HD_UNROLL
    for (int k1 = 0; k1 < 4; ++k1) {
        cf z[4];
HD_UNROLL
        for (int n2 = 0; n2 < 4; ++n2) z[n2] = (n2 * k1 != 0) ? cmul(y[n2][k1], unit_root<16>(n2 * k1, dir)) : y[n2][k1];
        dft_small<4>(z, dir);
HD_UNROLL
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = z[k2];
    }
}

// Twiddle table of one FFT pass with Ns butterflies per block and radix R:
// entry (r - 1) Ns + jm is exp(-2 pi i r jm / (Ns R)), r = 1 .. R-1,
// jm < Ns; computed in FP64 and rounded once. A pass with Ns = 1 has none.
HD int stage_table_len(int Ns, int R) { return Ns > 1 ? Ns * (R - 1) : 0; }

inline void stage_twiddles(int Ns, int R, cf* T) {
    if (Ns <= 1) return;
    for (int r = 1; r < R; ++r)
        for (int jm = 0; jm < Ns; ++jm) {
            const double a = -2.0 * 3.14159265358979323846 * (double)((r * jm) % (Ns * R)) / (double)(Ns * R);
            T[(r - 1) * Ns + jm] = {(float)cos(a), (float)sin(a)};
        }
}

// Radix plan of n = 2^a, 3 * 2^a, 5 * 2^a or 9 * 2^a (n <= 2304): radix 16
// while possible, then the rest r = n / 16^k in one stage when r is 2, 3, 4,
// 5, 6, 8, 9, 10 or 12, else radix 4 then 6 (r = 24), radix 4 then 5
// (r = 20), radix 8 then 5 (r = 40) or radix 2, 4, 8 then 9 (r = 18, 36,
// 72); the factor 3, 5 or 9 is always in the last stage, so every stage sees
// a power-of-two Ns. Returns the number of stages, or -1 for any other n.
HD int fft_radices(int n, int rad[32]) {
    int m = n;
    if (m % 9 == 0) {
        if (n > 2304) return -1;   // 9 * 2^a up to 2304 (a larger one would need radix 18)
        m /= 9;
    } else if (m % 3 == 0) m /= 3;
    else if (m % 5 == 0) m /= 5;
    if (m < 1 || (m & (m - 1)) != 0) return -1;
    int k = 0;
    while (n % 16 == 0) {
        rad[k++] = 16;
        n /= 16;
    }
    if (n == 24) {
        rad[k++] = 4;
        rad[k++] = 6;
    } else if (n == 20) {
        rad[k++] = 4;
        rad[k++] = 5;
    } else if (n == 40) {
        rad[k++] = 8;
        rad[k++] = 5;
    } else if (n == 18 || n == 36 || n == 72) {
        rad[k++] = n / 9;
        rad[k++] = 9;
    } else if (n != 1) {
        rad[k++] = n;   // 2, 3, 4, 5, 6, 8, 9, 10 or 12
    }
    return k;
}

// ---------------------------------------------------------------------------
// In-place mixed-radix FFT by decimation in frequency (forward) and in time
// (inverse). The forward transform leaves its output in digit-reversed order
// and the inverse takes digit-reversed input back to natural order, so a
// pointwise product between them needs no reordering, and every pass reads
// and writes the same positions (one barrier between passes in shared
// memory).
//
// Passes p = 0 .. s-1 take the radices of fft_radices in order, with strides
// S_p = n / (R_0 ... R_p) and blocks of L_p = R_p S_p consecutive elements.
// Forward pass p, butterfly b in [0, n / R_p): block q = b div S_p,
// m = b mod S_p; inputs x_r at q L_p + m + r S_p (r < R_p); outputs
//     y_k = W_{L_p}^(m k) sum_r x_r W_{R_p}^(r k),   W_N = exp(-2 pi i / N),
// at the same positions (k in place of r). After the last pass position
// sum_p k_p S_p holds frequency sum_p k_p R_0 ... R_(p-1). Inverse pass p
// (p = s-1 down to 0) undoes forward pass p up to the factor R_p:
//     x_r = sum_k conj(W_{L_p}^(m k)) y_k W_{R_p}^(-r k).
// The twiddles W_{L_p}^(m k) of pass p are stage_twiddles(S_p, R_p); the last
// pass has S = 1 and none.
// ---------------------------------------------------------------------------
constexpr int kMaxDifPasses = 8;

// Radices and strides of the passes of length n: the radices of fft_radices
// in reverse order (the factor 3, 5 or 9 first, radix 16 last, so that the
// last pass, stride 1, is a radix-16 pass whenever 16 divides n); returns s
// (-1 if n is not a supported length).
HD int dif_plan(int n, int R[kMaxDifPasses], int S[kMaxDifPasses]) {
    int rad[32];
    const int s = fft_radices(n, rad);
    if (s < 0 || s > kMaxDifPasses) return -1;
    int L = n;
    for (int p = 0; p < s; ++p) {
        R[p] = rad[s - 1 - p];
        S[p] = L / R[p];
        L = S[p];
    }
    return s;
}

// Shared-memory layout of the 16-byte elements (two spectrum columns) of the
// column kernel: the low three bits of the index are XOR-ed with bits 4..6,
// so that the 8 elements of a quarter warp land in 8 different 16-byte bank
// groups both for consecutive indices and for the stride-16 accesses of a
// radix-16 pass. Changes only the low three bits: a permutation of every
// aligned group of 8 (and the identity below 16).
HD int swc(int i) { return i ^ ((i >> 4) & 7); }

// First position of butterfly b's elements in pass (R, S): q L + m.
HD int dif_base(int R, int S, int b) {
    const int q = b / S;
    return q * S * R + (b - q * S);
}

// Frequency held at position pos after the forward passes.
HD int dif_freq(int s, const int R[kMaxDifPasses], const int S[kMaxDifPasses], int pos) {
    int f = 0, w = 1;
    for (int p = 0; p < s; ++p) {
        const int k = pos / S[p];
        pos -= k * S[p];
        f += k * w;
        w *= R[p];
    }
    return f;
}

// Position holding frequency f after the forward passes (inverse of
// dif_freq): the digits of f in the mixed radix R_0, R_1, ... (least
// significant first) weighted by the strides.
HD int dif_pos(int s, const int R[kMaxDifPasses], const int S[kMaxDifPasses], int f) {
    int pos = 0;
    for (int p = 0; p < s; ++p) {
        const int q = f / R[p];
        pos += (f - q * R[p]) * S[p];
        f = q;
    }
    return pos;
}

// Every pass's twiddle table back to back in pass order (the last pass has
// none); returns the number of entries (T may be null to query it).
inline int fft_dif_tables(int n, cf* T) {
    int R[kMaxDifPasses], S[kMaxDifPasses];
    const int s = dif_plan(n, R, S);
    int len = 0;
    for (int p = 0; p < s; ++p) {
        if (T) stage_twiddles(S[p], R[p], T + len);
        len += stage_table_len(S[p], R[p]);
    }
    return len;
}

// Real FFT of length P = 2M through a complex FFT of length M of the packed
// pairs z[n] = x[2n] + i x[2n+1] with transform Z. Unnormalised, without the
// factors 1/2 (they are folded into the kernel spectrum):
//   X[k] = (Z[k] + conj Z[M-k]) - i W^k (Z[k] - conj Z[M-k]),  W = exp(-2 pi i / P),
// Z[M] = Z[0], twP[k] = W^k. The inverse builds, for the pair (k, M-k),
// 0 < k < M, from the half spectrum X (X[M] = 0), Z[k] = E + i O with
//   E = X[k] + conj X[M-k],  O = W^-k (X[k] - conj X[M-k]),
// and W^-(M-k) = -W^k gives Z[M-k] from the same two values.
// k = 0 of the inverse: X[0] real part only (its imaginary part and X[M]
// are zero for a real signal), Z[0] = X0 + i X0.
HD cf c2r_pre_dc(cf X0) { return {X0.x, X0.x}; }

// The row kernels hold Z in digit-reversed order: the forward step reads
// Z[k] and Z[M-k] from buffer positions pk and pmk;
HD cf r2c_post_at(const cf* Z, int pk, int pmk, int k, const cf* twP) {
    cf a = Z[pk];
    cf b = cconj(Z[pmk]);
    cf e = cadd(a, b);
    cf o = cmul(twP[k], csub(a, b));
    return {e.x + o.y, e.y - o.x};
}
// the inverse step takes a = X[k], b = X[M-k] and w = W^k and gives the
// packed inputs Z[k] (zk) and Z[M-k] (zmk), 0 < k < M.
HD void c2r_pre_vals(cf a, cf b, cf w, cf& zk, cf& zmk) {
    cf e1 = cadd(a, cconj(b));
    cf o1 = cmulc(csub(a, cconj(b)), w);
    cf e2 = cadd(b, cconj(a));
    cf o2 = cmul(csub(b, cconj(a)), w);
    zk = {e1.x - o1.y, e1.y + o1.x};
    zmk = {e2.x + o2.y, e2.y - o2.x};
}

}  // namespace hr

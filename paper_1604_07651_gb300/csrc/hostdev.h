// Pure arithmetic shared by the device kernels and by the host unit tests of
// those kernels (compiled with g++ for the tests, nvcc for the library):
// * cubic B-spline tap weights (the B3 of Eq. (14)-(17));
// * one radix-r Stockham butterfly (the FFT of Eq. (7), (16)-(17));
// * the packing of a real FFT into a complex FFT of half the length.
#pragma once

#include <math.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define HD __host__ __device__ __forceinline__
#else
#define HD inline
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

// One Stockham autosort butterfly (Govindaraju et al., SC'08 formulation):
// stage of radix R with Ns = product of the radices already applied, for the
// butterfly index j in [0, n/R). tw[k] = exp(-2 pi i k / n), k < n (the
// forward twiddles; the inverse, dir = +1, uses their conjugates).
template <int R>
HD void stockham_butterfly(const cf* in, cf* out, int n, int Ns, int j, const cf* tw, int dir) {
    cf v[R];
    int jm = j % Ns;
    int step = n / (Ns * R);                 // twiddle index stride: k/(Ns R) = k*step/n
    for (int r = 0; r < R; ++r) {
        cf x = in[j + r * (n / R)];
        int t = r * jm * step;               // < n
        v[r] = r ? (dir < 0 ? cmul(x, tw[t]) : cmulc(x, tw[t])) : x;
    }
    dft_small<R>(v, dir);
    int dst = (j / Ns) * Ns * R + jm;
    for (int r = 0; r < R; ++r) out[dst + r * Ns] = v[r];
}

// Radix plan of n = 2^a 3^b: radices 4, then 2, then 3. Returns the number
// of stages, or -1 if n has another prime factor.
HD int fft_radices(int n, int rad[32]) {
    int k = 0;
    while (n % 4 == 0) { rad[k++] = 4; n /= 4; }
    while (n % 2 == 0) { rad[k++] = 2; n /= 2; }
    while (n % 3 == 0) { rad[k++] = 3; n /= 3; }
    return n == 1 ? k : -1;
}

// Real FFT of length P = 2M through a complex FFT of length M of the packed
// pairs z[n] = x[2n] + i x[2n+1] with transform Z. Unnormalised, without the
// factors 1/2 (they are folded into the kernel spectrum):
//   X[k] = (Z[k] + conj Z[M-k]) - i W^k (Z[k] - conj Z[M-k]),  W = exp(-2 pi i / P),
// Z[M] = Z[0]. twP[k] = W^k.
HD cf r2c_post(const cf* Z, int M, int k, const cf* twP) {
    cf a = Z[k];
    cf b = cconj(Z[k == 0 ? 0 : M - k]);
    cf e = cadd(a, b);
    cf o = cmul(twP[k], csub(a, b));
    return {e.x + o.y, e.y - o.x};          // e - i o
}

// Inverse of r2c_post for the pair (k, M-k), 0 < k < M, in place: from the
// half spectrum X (X[M] = 0) build Z[k] = E + i O with
//   E = X[k] + conj X[M-k],  O = W^-k (X[k] - conj X[M-k]).
// W^-(M-k) = -W^k gives Z[M-k] from the same two values.
HD void c2r_pre_pair(cf* X, int M, int k, const cf* twP) {
    cf a = X[k], b = X[M - k];
    cf w = twP[k];
    cf e1 = cadd(a, cconj(b));
    cf o1 = cmulc(csub(a, cconj(b)), w);     // (a - conj b) * conj(W^k)
    cf e2 = cadd(b, cconj(a));
    cf o2 = cmul(csub(b, cconj(a)), w);      // (b - conj a) * W^k, times -1 below
    X[k] = {e1.x - o1.y, e1.y + o1.x};       // e1 + i o1
    X[M - k] = {e2.x + o2.y, e2.y - o2.x};   // e2 + i (-o2)
}

// k = 0 of the inverse: X[0] real part only (its imaginary part and X[M]
// are zero for a real signal), Z[0] = X0 + i X0.
HD cf c2r_pre_dc(cf X0) { return {X0.x, X0.x}; }

}  // namespace hr

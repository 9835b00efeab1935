// sm_103a kernels of the log-polar hyperbolic Radon transform and of the
// direct-summation comparator.
//
// Forward, per sub-problem (Sections 2-4):
//   k_grid_tiles       gridding of the gather samples onto the log-polar
//                      lattice with cubic B-splines (Eq. (14)-(15)), one tile
//                      of lattice cells per CTA in shared memory;
//   k_rows_r2c         real FFT of the lattice rows (first half of Eq. (7)/(16));
//   k_colconv          FFT along theta, product with the kernel spectrum
//                      chi_L zeta_hat / B3_hat^2 (Eq. (16)-(17)), inverse FFT;
//   k_rows_c2r         inverse real FFT of the rows -> B-spline coefficients;
//   k_interp_columns   cubic B-spline interpolation at (phi, eta) = P2 S(tau^2,
//                      q^2) (Eq. (17)), summed over the time pieces.
// Adjoint (Eq. (16), Section 3): the same kernels with the roles exchanged:
//   k_col_profiles_cols -> k_band_rows -> k_colconv (conjugate kernel) -> k_rows_c2r ->
//   k_gather_samples.
//
// Lattice positions do not depend on the data: the plan computes them once in
// FP64 (k_sample_table, k_radon_table) and stores first tap and fractional
// part, so the transforms themselves are FP32 loads, B-spline weights and
// sums. Shared-memory accumulation is fixed point (integer atomics, order
// independent); a lattice tile cut into several gridding work units is
// summed from their partial tiles in a fixed order by the last unit to
// finish. No kernel uses floating-point atomics: the forward and the adjoint
// are bitwise reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "internal.h"

namespace hr {

__device__ __forceinline__ cf ldcf(const cf* p) {
    float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
}
// --------------------------------------------------------------------------
// Row kernels: scatter into a band of lattice rows, then real FFT of the rows.
// Shared memory: [R][Prho] floats (rows, viewed as [R][M] complex); the FFT
// works in place.
// --------------------------------------------------------------------------

extern __shared__ __align__(16) float smem_f[];

// Piece of this block in a batched launch, and the block's index within it:
// from the descriptors passed as a kernel parameter (up to kMaxBatch pieces)
// or from a device-resident batch (any number of pieces of many gathers).
__device__ __forceinline__ int batch_piece(const PieceBatch& B, int& bx) {
    int pi = 0;
#pragma unroll
    for (int k = 1; k < kMaxBatch; ++k)
        if (k < B.n && (int)blockIdx.x >= B.first[k]) pi = k;
    bx = (int)blockIdx.x - B.first[pi];
    return pi;
}
__device__ __forceinline__ const PieceDev& piece_of(const PieceBatch& B, int& bx) { return B.p[batch_piece(B, bx)]; }
__device__ __forceinline__ const PieceDev& piece_of(const DevBatch& B, int& bx) {
    const int2 m = __ldg(B.map + blockIdx.x);
    bx = m.y;
    return B.p[m.x];
}

// Dynamic shared memory of the launch: the row and column kernels check it
// against what their piece needs and leave the block untouched (never write
// past it) if a launch gave too little.
__device__ __forceinline__ unsigned dyn_smem_bytes() {
    unsigned r;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

__device__ __forceinline__ float load_in(const float* p) { return __ldg(p); }
__device__ __forceinline__ float load_in(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }

// Real sample n of a row buffer (stored as complex pairs in the sw layout).
__device__ __forceinline__ int swr(int n) { return 2 * sw(n >> 1) + (n & 1); }

// Row transforms: the real FFT of a lattice row of length Prho (first half
// of Eq. (7)/(16)) as a complex FFT of the M = Prho / 2 packed pairs
// z[n] = x[2n] + i x[2n+1], and its inverse, by the in-place decimation in
// frequency / time of the column pass (dif_plan of M: P.fftM, twiddles
// P.twM). The forward leaves Z in digit-reversed order; the real-FFT
// post-processing reads Z[k] and Z[M - k] at their positions (P.rpos), and
// the inverse's pre-processing writes the packed pairs straight to theirs.
// One row butterfly per thread, the band's rows back to back in shared
// memory ([R][M] complex, element i of a row at sw(i)), one barrier per pass.
// Stride between the band's rows in shared memory, in complex elements: one
// element of padding, so that the same position of the band's rows falls in
// different banks (M is a multiple of 16).
__host__ __device__ __forceinline__ int row_stride(int M) { return M + 1; }
// Shared memory of the row kernels: R rows of row_stride(Prho / 2) complex.
__host__ __device__ __forceinline__ size_t rows_smem(const PieceDev& P) {
    return (size_t)P.R * row_stride(P.Prho / 2) * sizeof(cf);
}

template <int R>
__device__ __forceinline__ void row_fwd(cf x[R], const cf* __restrict__ T, int S, int m) {
    dft_small<R>(x, -1);
    if (S > 1) {
#pragma unroll
        for (int k = 1; k < R; ++k) x[k] = cmul(x[k], ldcf(T + (k - 1) * S + m));
    }
}
template <int R>
__device__ __forceinline__ void row_inv(cf x[R], const cf* __restrict__ T, int S, int m) {
    if (S > 1) {
#pragma unroll
        for (int k = 1; k < R; ++k) x[k] = cmulc(x[k], ldcf(T + (k - 1) * S + m));
    }
    dft_small<R>(x, +1);
}

// One pass over every row of the band, in place in shared memory.
template <int R, bool INV>
__device__ __forceinline__ void rows_pass(cf* X, int M, int nrows, int S, const cf* __restrict__ T) {
    const int nb = M / R, tot = nb * nrows;
    const float inv_nb = 1.0f / (float)nb, invS = 1.0f / (float)S;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
        const int row = (int)(((float)idx + 0.5f) * inv_nb);   // exact for idx < 2^22
        const int b = idx - row * nb;
        const int q = (int)(((float)b + 0.5f) * invS);
        const int m = b - q * S;
        const int base = q * S * R + m;
        cf* Z = X + row * row_stride(M);
        cf x[R];
#pragma unroll
        for (int r = 0; r < R; ++r) x[r] = Z[sw(base + r * S)];
        if (INV) row_inv<R>(x, T, S, m);
        else row_fwd<R>(x, T, S, m);
#pragma unroll
        for (int r = 0; r < R; ++r) Z[sw(base + r * S)] = x[r];
    }
}

// Forward pass 0 reading the band's lattice rows (Nr reals each, zero padded)
// from global memory.
template <int R>
__device__ __forceinline__ void rows_first_lat(cf* X, const float* __restrict__ lat, int Nr, int M, int nrows, int S,
                                               const cf* __restrict__ T) {
    const int tot = S * nrows;
    const float invS = 1.0f / (float)S;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
        const int row = (int)(((float)idx + 0.5f) * invS);
        const int m = idx - row * S;
        const float* src = lat + (size_t)row * Nr;
        cf x[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int n2 = 2 * (m + r * S);
            x[r].x = n2 < Nr ? __ldg(src + n2) : 0.f;
            x[r].y = n2 + 1 < Nr ? __ldg(src + n2 + 1) : 0.f;
        }
        row_fwd<R>(x, T, S, m);
        cf* Z = X + row * row_stride(M);
#pragma unroll
        for (int r = 0; r < R; ++r) Z[sw(m + r * S)] = x[r];
    }
}

// Inverse pass 0 writing the band's lattice rows (first Nr reals) to global
// memory.
template <int R>
__device__ __forceinline__ void rows_last_lat(const cf* X, float* lat, int Nr, int M, int nrows, int S,
                                              const cf* __restrict__ T) {
    const int tot = S * nrows;
    const float invS = 1.0f / (float)S;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
        const int row = (int)(((float)idx + 0.5f) * invS);
        const int m = idx - row * S;
        const cf* Z = X + row * row_stride(M);
        cf x[R];
#pragma unroll
        for (int r = 0; r < R; ++r) x[r] = Z[sw(m + r * S)];
        row_inv<R>(x, T, S, m);
        float* dst = lat + (size_t)row * Nr;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int n2 = 2 * (m + r * S);
            if (n2 < Nr) dst[n2] = x[r].x;
            if (n2 + 1 < Nr) dst[n2 + 1] = x[r].y;
        }
    }
}

#define HR_RADIX_CASES(CALL) \
    case 16: CALL(16); break; \
    case 12: CALL(12); break; \
    case 10: CALL(10); break; \
    case 9: CALL(9); break;   \
    case 8: CALL(8); break;   \
    case 6: CALL(6); break;   \
    case 5: CALL(5); break;   \
    case 4: CALL(4); break;   \
    case 3: CALL(3); break;   \
    default: CALL(2); break;

// The same passes for the row lengths M = R0 * 256 with radices R0, 16, 16
// (the plans of the 2048^2 and 4096^2 workloads), every length, stride and
// count a compile-time constant (the index arithmetic folds to shifts and
// constant divisions). Same arithmetic as the general passes.
template <int R, int S, int M, bool INV>
__device__ __forceinline__ void rows_pass_c(cf* X, int nrows, const cf* __restrict__ T) {
    constexpr int nb = M / R;
    const int tot = nb * nrows;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
        const int row = idx / nb;
        const int b = idx - row * nb;
        const int q = b / S, m = b - q * S;
        const int base = q * S * R + m;
        cf* Z = X + row * row_stride(M);
        cf x[R];
#pragma unroll
        for (int r = 0; r < R; ++r) x[r] = Z[sw(base + r * S)];
        if (INV) row_inv<R>(x, T, S, m);
        else row_fwd<R>(x, T, S, m);
#pragma unroll
        for (int r = 0; r < R; ++r) Z[sw(base + r * S)] = x[r];
    }
}
template <int R0>
__device__ __forceinline__ void rows_first_lat_c(cf* X, const float* __restrict__ lat, int Nr, int nrows,
                                                 const cf* __restrict__ T) {
    constexpr int S = 256, M = R0 * 256;
    const int tot = S * nrows;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
        const int row = idx / S, m = idx % S;
        const float* src = lat + (size_t)row * Nr;
        cf x[R0];
#pragma unroll
        for (int r = 0; r < R0; ++r) {
            const int n2 = 2 * (m + r * S);
            x[r].x = n2 < Nr ? __ldg(src + n2) : 0.f;
            x[r].y = n2 + 1 < Nr ? __ldg(src + n2 + 1) : 0.f;
        }
        row_fwd<R0>(x, T, S, m);
        cf* Z = X + row * row_stride(M);
#pragma unroll
        for (int r = 0; r < R0; ++r) Z[sw(m + r * S)] = x[r];
    }
}
template <int R0>
__device__ __forceinline__ void rows_last_lat_c(const cf* X, float* lat, int Nr, int nrows, const cf* __restrict__ T) {
    constexpr int S = 256, M = R0 * 256;
    const int tot = S * nrows;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
        const int row = idx / S, m = idx % S;
        const cf* Z = X + row * row_stride(M);
        cf x[R0];
#pragma unroll
        for (int r = 0; r < R0; ++r) x[r] = Z[sw(m + r * S)];
        row_inv<R0>(x, T, S, m);
        float* dst = lat + (size_t)row * Nr;
#pragma unroll
        for (int r = 0; r < R0; ++r) {
            const int n2 = 2 * (m + r * S);
            if (n2 < Nr) dst[n2] = x[r].x;
            if (n2 + 1 < Nr) dst[n2 + 1] = x[r].y;
        }
    }
}
// R0 of a plan of length R0 * 256 with radices R0, 16, 16, else 0.
__device__ __forceinline__ int plan_x256(const FftPlan& fp) {
    return (fp.nst == 3 && fp.st[0] == 256 && fp.rad[1] == 16 && fp.rad[2] == 16) ? fp.rad[0] : 0;
}
#define HR_X256_CASES(CALL) \
    case 2: CALL(2); break;  \
    case 3: CALL(3); break;  \
    case 4: CALL(4); break;  \
    case 5: CALL(5); break;  \
    case 6: CALL(6); break;  \
    case 8: CALL(8); break;  \
    case 9: CALL(9); break;  \
    case 10: CALL(10); break; \
    case 12: CALL(12); break;

// Forward passes p0 .. s-1 in shared memory (p0 = 1 after rows_first_lat).
__device__ __forceinline__ void rows_fwd_passes(cf* X, int M, int nrows, const FftPlan& fp, const cf* T, int p0) {
    switch (plan_x256(fp)) {
#define HR_RX(R0)                                                                    \
    if (p0 == 0) {                                                                   \
        rows_pass_c<R0, 256, R0 * 256, false>(X, nrows, T);                          \
        __syncthreads();                                                             \
    }                                                                                \
    rows_pass_c<16, 16, R0 * 256, false>(X, nrows, T + fp.tw[1]);                    \
    __syncthreads();                                                                 \
    rows_pass_c<16, 1, R0 * 256, false>(X, nrows, T);                                \
    __syncthreads();                                                                 \
    return;
        HR_X256_CASES(HR_RX)
#undef HR_RX
        default: break;
    }
    for (int p = p0; p < fp.nst; ++p) {
#define HR_RF(RR) rows_pass<RR, false>(X, M, nrows, fp.st[p], T + fp.tw[p])
        switch (fp.rad[p]) { HR_RADIX_CASES(HR_RF) }
#undef HR_RF
        __syncthreads();
    }
}

// Real-FFT post-processing of the band's transformed rows (digit-reversed in
// shared memory) into the half spectrum, bins k <= k2max, blocked layout.
__device__ __forceinline__ void rows_post(const PieceDev& P, const cf* Z0, int mb, int nrows) {
    cf* __restrict__ spec = P.spec;
    const int M = P.Prho / 2;
    const int nk = P.k2max + 1;
    const int per_kb = nrows * 2;                 // (row, c) of a column block (CB = 2), c fastest
    const int total = P.nkb * per_kb;
    const float inv_per_kb = 1.0f / (float)per_kb;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int kb = (int)(((float)idx + 0.5f) * inv_per_kb);   // exact for idx < 2^22
        const int rem = idx - kb * per_kb;
        const int m = rem >> 1;
        const int c = rem & 1;
        const int k = kb * 2 + c;
        cf X = {0.f, 0.f};
        if (k < nk)
            X = r2c_post_at(Z0 + m * row_stride(M), sw(__ldg(P.rpos + k)), sw(__ldg(P.rpos + (k == 0 ? 0 : M - k))), k,
                            P.twP);
        spec[((size_t)kb * P.Ntheta + (mb + m)) * 2 + c] = X;
    }
}

// Inverse: the real-FFT pre-processing of the band's half-spectrum rows
// (bins above k2max are zero), pairs (k, M - k) for 0 <= k <= M/2, written to
// their digit-reversed positions in shared memory.
__device__ __forceinline__ void rows_pre(const PieceDev& P, cf* X, int mb, int nrows) {
    const cf* __restrict__ spec = P.spec;
    const int M = P.Prho / 2, half = M / 2;
    const int nk = P.k2max + 1;
    const int per_kb = nrows * 2;                 // (row, c) of a column block, c fastest
    const int total = (half / 2 + 1) * per_kb;    // k = 2 kb + c <= half
    constexpr int U = 4;                          // pairs per thread whose spectrum loads go out together
    const float inv_per_kb = 1.0f / (float)per_kb;
    for (int i0 = threadIdx.x; i0 < total; i0 += U * blockDim.x) {
        cf a[U], b[U];
        int kk[U], mm[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = i0 + u * (int)blockDim.x;
            const int kb = (int)(((float)idx + 0.5f) * inv_per_kb);   // exact for idx < 2^22
            const int rem = idx - kb * per_kb;
            const int m = rem >> 1;
            const int k = 2 * kb + (rem & 1);
            kk[u] = idx < total && k <= half ? k : -1;
            mm[u] = m;
            a[u] = b[u] = cf{0.f, 0.f};
            if (kk[u] < 0) continue;
            const size_t rowoff = (size_t)(mb + m) * 2;
            const int k2 = M - k;
            if (k < nk) a[u] = ldcf(spec + (size_t)(k >> 1) * P.Ntheta * 2 + rowoff + (k & 1));
            if (k > 0 && k2 < nk) b[u] = ldcf(spec + (size_t)(k2 >> 1) * P.Ntheta * 2 + rowoff + (k2 & 1));
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = kk[u];
            if (k < 0) continue;
            cf* Z = X + mm[u] * row_stride(M);
            if (k == 0) {
                Z[sw(__ldg(P.rpos))] = c2r_pre_dc(a[u]);
                continue;
            }
            cf zk, zmk;
            c2r_pre_vals(a[u], b[u], ldcf(P.twP + k), zk, zmk);
            Z[sw(__ldg(P.rpos + k))] = zk;
            Z[sw(__ldg(P.rpos + M - k))] = zmk;
        }
    }
}

// Shared gridding tile: the kTileRows x kTileCols cells plus a halo of
// NT - 1 cells on every side (NT taps per axis: 4 cubic, 6 quintic), so that
// every tap of a sample whose footprint meets the tile lands in it without a
// bounds check (the halo is dropped at the end: the neighbouring tiles'
// units add those cells). The odd pitch puts the rows on different banks.
template <int NT>
struct GridTile {
    static constexpr int halo = NT - 1;
    static constexpr int pitch = kTileCols + 2 * halo + 1;
    static constexpr int rows = kTileRows + 2 * halo;
};

// Fixed-point accumulation in shared memory. Integer adds to shared memory
// are single fire-and-forget instructions, float adds are compare-and-swap
// loops (measured 3.7x apart on conflict-free addresses), and integer sums do
// not depend on the order in which warps arrive. A block accumulating into a
// region whose cells provably stay below vmax * C in magnitude (vmax the
// largest |input| it adds, C a plan-time bound on the total weight any cell
// collects, C < 2^(ec+1)) scales its inputs by 2^sh with
// sh = 28 - ec - ilogb(vmax): every cell stays below 2^30, and every
// contribution is rounded to 2^-31 of at most four times the bound. The
// power of two is applied as two factors so that it spans the whole float
// range. The plan stores 28 - ec.
__device__ __forceinline__ float pow2i(int k) { return __int_as_float((127 + k) << 23); }   // |k| <= 126

struct Pow2Scale {
    float up1, up2, down1, down2;
    __device__ __forceinline__ Pow2Scale(int sh) {
        const int h1 = sh / 2, h2 = sh - h1;
        up1 = pow2i(h1);
        up2 = pow2i(h2);
        down1 = pow2i(-h1);
        down2 = pow2i(-h2);
    }
    __device__ __forceinline__ float up(float v) const { return v * up1 * up2; }
    __device__ __forceinline__ float down(int t) const { return (float)t * down1 * down2; }
};

__device__ __forceinline__ void red_fixed(int* p, float v) { atomicAdd(p, __float2int_rn(v)); }

// Maximum of a non-negative float over the block (all threads get it); NaN
// wins, so a non-finite input shows as a non-finite maximum.
__device__ __forceinline__ float block_max_abs(float v, float* red) {
    v = fabsf(v);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const float o = __shfl_xor_sync(0xffffffffu, v, d);
        v = (o > v || o != o) ? o : v;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float m = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        const float o = red[w];
        m = (o > m || o != o) ? o : m;
    }
    return m;
}

// Forward gridding (Eq. (15)) of the gather f[Nx][Nt] onto the lattice
// P.lat (zeroed before). The plan lists, per tile of kTileRows x kTileCols
// cells, chunks of at most 8 consecutive samples of one trace whose NT x NT
// footprint meets the tile, and cuts every tile's list into work units of at
// most kUnitChunks chunks (sample density varies by two orders of magnitude
// over the lattice, so units, not tiles, balance the CTAs), each with the
// largest total B-spline weight one of its cells can collect. A CTA takes one
// unit, each thread one chunk: neighbouring threads are 8 samples apart, so
// their footprints rarely meet, and a thread sums its samples in registers
// in an NT x NT register window over the cells of its current footprint. When the
// first tap (m0, n0) moves by one cell along either axis (consecutive samples
// of a trace mostly do), only the row or column that leaves the window goes
// to the fixed-point shared tile and the window slides; a longer jump flushes
// the whole window. The tile's touched cells are then added to P.lat. A
// non-finite sample makes the unit's tile NaN (the FFTs that follow would
// spread it over the whole piece in any case).
// The window acc[NT a + c] holds cells (wm + a, wn + c); t points at
// (wm, wn) in the shared tile.
template <int NT>
__device__ __forceinline__ void flush_window(int* t, const float (&acc)[NT * NT]) {
#pragma unroll
    for (int a = 0; a < NT; ++a)
#pragma unroll
        for (int c = 0; c < NT; ++c) red_fixed(t + a * GridTile<NT>::pitch + c, acc[NT * a + c]);
}
// window one row down (row wm leaves) / up (row wm + NT - 1 leaves)
template <int NT>
__device__ __forceinline__ void slide_rows_down(int* t, float (&acc)[NT * NT]) {
#pragma unroll
    for (int c = 0; c < NT; ++c) {
        red_fixed(t + c, acc[c]);
#pragma unroll
        for (int a = 0; a + 1 < NT; ++a) acc[NT * a + c] = acc[NT * (a + 1) + c];
        acc[NT * (NT - 1) + c] = 0.f;
    }
}
template <int NT>
__device__ __forceinline__ void slide_rows_up(int* t, float (&acc)[NT * NT]) {
#pragma unroll
    for (int c = 0; c < NT; ++c) {
        red_fixed(t + (NT - 1) * GridTile<NT>::pitch + c, acc[NT * (NT - 1) + c]);
#pragma unroll
        for (int a = NT - 1; a > 0; --a) acc[NT * a + c] = acc[NT * (a - 1) + c];
        acc[c] = 0.f;
    }
}
// window one column right (column wn leaves) / left (column wn + NT - 1 leaves)
template <int NT>
__device__ __forceinline__ void slide_cols_right(int* t, float (&acc)[NT * NT]) {
#pragma unroll
    for (int a = 0; a < NT; ++a) {
        red_fixed(t + a * GridTile<NT>::pitch, acc[NT * a]);
#pragma unroll
        for (int c = 0; c + 1 < NT; ++c) acc[NT * a + c] = acc[NT * a + c + 1];
        acc[NT * a + NT - 1] = 0.f;
    }
}
template <int NT>
__device__ __forceinline__ void slide_cols_left(int* t, float (&acc)[NT * NT]) {
#pragma unroll
    for (int a = 0; a < NT; ++a) {
        red_fixed(t + a * GridTile<NT>::pitch + NT - 1, acc[NT * a + NT - 1]);
#pragma unroll
        for (int c = NT - 1; c > 0; --c) acc[NT * a + c] = acc[NT * a + c - 1];
        acc[NT * a] = 0.f;
    }
}

// Split tiles: the unit's partial tile (value(i) of cell i, row-major over
// the kTileRows x kTileCols cells) goes to its slot; the unit that finds it
// is the tile's last to arrive (the others' slots are then complete and
// visible) sums every slot of the tile in slot order into the lattice and
// clears the counter. The result does not depend on which unit runs first.
// Ordering: the block's slot stores, a barrier, then one thread's fence and
// count (release, cumulative over the block through the barrier); on the
// reading side that thread's fence after the count, a barrier, and L2 loads.
template <class F>
__device__ __forceinline__ void grid_merge_split(const PieceDev& P, int4 us, int m_lo, int n_lo, int nr, int nc,
                                                 F&& value) {
    __shared__ int s_last;
    constexpr int kCells = kTileRows * kTileCols;
    float* slot0 = P.slots + (size_t)us.x * kCells;
    for (int i = threadIdx.x; i < kCells; i += blockDim.x) slot0[(size_t)us.z * kCells + i] = value(i);
    __syncthreads();
    int* counter = reinterpret_cast<int*>(P.lat + (size_t)P.Ntheta * P.Nrho) + us.w;
    if (threadIdx.x == 0) {
        __threadfence();
        const int last = atomicAdd(counter, 1) == us.y - 1;
        if (last) __threadfence();
        s_last = last;
    }
    __syncthreads();
    if (!s_last) return;
    // each thread sums its kCells / kUnitChunks cells over the slots in slot
    // order, all its cells' loads of two slots in flight together
    constexpr int kPer = kCells / kUnitChunks;
    static_assert(kCells % kUnitChunks == 0, "cells per thread");
    float acc[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) acc[j] = 0.f;
    const float* src = slot0 + threadIdx.x;
#pragma unroll 2
    for (int u = 0; u < us.y; ++u) {
        float v[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) v[j] = __ldcg(src + (size_t)u * kCells + j * kUnitChunks);
#pragma unroll
        for (int j = 0; j < kPer; ++j) acc[j] += v[j];
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int i = threadIdx.x + j * kUnitChunks;
        const int m = i / kTileCols, n = i - m * kTileCols;
        if (m < nr && n < nc) P.lat[(size_t)(m_lo + m) * P.Nrho + n_lo + n] = acc[j];
    }
    if (threadIdx.x == 0) *counter = 0;
}

template <class Src, class T, int NT>
__global__ void __launch_bounds__(kUnitChunks, NT == 4 ? 4 : 2) k_grid_tiles(const __grid_constant__ Src B,
                                                                             const T* __restrict__ f) {
    using Tile = GridTile<NT>;
    __shared__ int tile[Tile::rows * Tile::pitch];
    __shared__ float red[kUnitChunks / 32];
    int bx;
    const PieceDev& P = piece_of(B, bx);
    const int4 u = __ldg(P.units + bx);           // (tile, first chunk, end chunk, 28 - ec)
    const int ti = u.x / P.ntc, tj = u.x - ti * P.ntc;
    const int m_lo = ti * kTileRows, n_lo = tj * kTileCols;
    for (int i = threadIdx.x; i < Tile::rows * Tile::pitch; i += blockDim.x) tile[i] = 0;
    // one chunk per thread: issue every load of the chunk before the first is used
    const int c = u.y + threadIdx.x;
    int4 ent[8];
    float v[8];
    float vmax = 0.f;
    {
        int4 ch = make_int4(0, 0, 0, 0);                // (trace, first sample, count)
        if (c < u.z) ch = __ldg(P.chunks + c);
        const int4* st = reinterpret_cast<const int4*>(P.stab + (size_t)ch.x * P.nj - P.jt_lo) + ch.y;
        const T* fk = f + P.f_off + (size_t)ch.x * P.Nt + ch.y;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            if (s < ch.z) {
                ent[s] = __ldg(st + s);
                v[s] = load_in(fk + s);
            } else {
                ent[s] = make_int4(0, 0, 0, 0);
                v[s] = 0.f;
            }
        }
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const float w = __int_as_float(ent[s].w);
            v[s] = w != 0.f ? v[s] * w : 0.f;   // muted samples add nothing, whatever f holds
            const float a = fabsf(v[s]);
            vmax = (a > vmax || a != a) ? a : vmax;
        }
    }
    vmax = block_max_abs(vmax, red);   // also orders the tile's zeroing before the adds
    const int4 us = __ldg(P.uslot + bx);  // (first slot, units of the tile, index, counter)
    const int nr = min(kTileRows, P.Ntheta - m_lo), nc = min(kTileCols, P.Nrho - n_lo);
    if (!(vmax > 0.f && vmax <= 3.402823466e38f)) {   // all zero (nothing to add) or not finite (NaN tile)
        const float fill = vmax == 0.f ? 0.f : __int_as_float(0x7fc00000);
        if (us.y > 1) {
            grid_merge_split(P, us, m_lo, n_lo, nr, nc, [&](int) { return fill; });
        } else if (fill != 0.f) {
            for (int i = threadIdx.x; i < kTileRows * kTileCols; i += blockDim.x) {
                const int m = i / kTileCols, n = i - m * kTileCols;
                if (m < nr && n < nc) P.lat[(size_t)(m_lo + m) * P.Nrho + n_lo + n] = fill;
            }
        }
        return;
    }
    const Pow2Scale sc(u.w - ilogbf(vmax));
#pragma unroll
    for (int s = 0; s < 8; ++s) v[s] = sc.up(v[s]);
    float acc[NT * NT];
#pragma unroll
    for (int q = 0; q < NT * NT; ++q) acc[q] = 0.f;
    int* win = nullptr;                                  // shared-tile address of the window's (wm, wn)
    int wm = 0, wn = 0;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        const int4 e = ent[s];
        if (v[s] == 0.f) continue;
        const int m0 = e.x >> 16, n0 = e.x & 0xffff;
        const int dm = m0 - wm, dn = n0 - wn;
        if (win == nullptr || dm < -1 || dm > 1 || dn < -1 || dn > 1) {
            if (win != nullptr) {
                flush_window<NT>(win, acc);
#pragma unroll
                for (int q = 0; q < NT * NT; ++q) acc[q] = 0.f;
            }
        } else {
            if (dm == 1) slide_rows_down<NT>(win, acc);
            else if (dm == -1) slide_rows_up<NT>(win, acc);
            win += dm * Tile::pitch;
            if (dn == 1) slide_cols_right<NT>(win, acc);
            else if (dn == -1) slide_cols_left<NT>(win, acc);
        }
        wm = m0;
        wn = n0;
        win = tile + (m0 - m_lo + Tile::halo) * Tile::pitch + n0 - n_lo + Tile::halo;
        float wt[NT], wr[NT];
        bspline_weights<NT>(__int_as_float(e.y), wt);
        bspline_weights<NT>(__int_as_float(e.z), wr);
#pragma unroll
        for (int a = 0; a < NT; ++a) {
            const float va = v[s] * wt[a];
#pragma unroll
            for (int q = 0; q < NT; ++q) acc[NT * a + q] = fmaf(va, wr[q], acc[NT * a + q]);
        }
    }
    if (win != nullptr) flush_window<NT>(win, acc);
    __syncthreads();
    if (us.y > 1) {
        grid_merge_split(P, us, m_lo, n_lo, nr, nc,
                         [&](int i) {
                             return sc.down(tile[(i / kTileCols + Tile::halo) * Tile::pitch + i % kTileCols + Tile::halo]);
                         });
        return;
    }
    for (int i = threadIdx.x; i < kTileRows * kTileCols; i += blockDim.x) {   // the tile's only unit
        const int m = i / kTileCols, n = i - m * kTileCols;
        const int t = tile[(m + Tile::halo) * Tile::pitch + n + Tile::halo];
        if (t != 0 && m < nr && n < nc) P.lat[(size_t)(m_lo + m) * P.Nrho + n_lo + n] = sc.down(t);
    }
}

// Real FFT of a band of lattice rows (P.lat, zero-padded to Prho) into the
// half spectrum (first half of Eq. (7)/(16)): pass 0 reads the rows from
// global memory.
template <class Src>
__global__ void __launch_bounds__(512, 2) k_rows_r2c(const __grid_constant__ Src B) {
    int bx;
    const PieceDev& P = piece_of(B, bx);
    if (P.CB != 2 || rows_smem(P) > dyn_smem_bytes()) return;
    const int mb = bx * P.R;
    const int nrows = min(P.R, P.Ntheta - mb);
    const int M = P.Prho / 2;
    cf* X = reinterpret_cast<cf*>(smem_f);
    const FftPlan& fp = P.fftM;
    switch (plan_x256(fp)) {
#define HR_RL(R0) rows_first_lat_c<R0>(X, P.lat + (size_t)mb * P.Nrho, P.Nrho, nrows, P.twM); break;
        HR_X256_CASES(HR_RL)
#undef HR_RL
        default:
#define HR_RL(RR) rows_first_lat<RR>(X, P.lat + (size_t)mb * P.Nrho, P.Nrho, M, nrows, fp.st[0], P.twM)
            switch (fp.rad[0]) { HR_RADIX_CASES(HR_RL) }
#undef HR_RL
    }
    __syncthreads();
    rows_fwd_passes(X, M, nrows, fp, P.twM, 1);
    rows_post(P, X, mb, nrows);
}

// Adjoint of the output interpolation (transpose of Eq. (17)), separated
// along the two axes. Every output of a slowness column has the same theta
// taps (the column's angle), so the transpose is a 1-D scatter along rho per
// column followed by an NT-tap spread of the column profiles over theta
// (B the cubic or quintic B-spline, NT = 4 or 6 taps):
//   h_l[n]   = s_l sum_i g[l][i] B(rho_il - rho_n)           (k_col_profiles_cols)
//   G'[m][n] = sum_l B(theta_l - theta_m) h_l[n]             (k_band_rows)
// The profiles are summed in fixed point (order-independent), the spread is a
// plain per-thread sum over the band's columns in a fixed order: the adjoint
// interpolation has no floating-point atomics and is deterministic.

// The profiles P.prof[lc][0..Nrho) (pitch hpitch) of every time piece of
// one output column, from the column's outputs g[l][*] scaled by each
// piece's output scale: one CTA per column (cmap[b] = (first piece, number
// of pieces, column l), or, when np_all > 0, column b of pieces[0..np_all)
// with ntau_all outputs), so that the column's outputs are read once for the
// scale and once for all its pieces ([np][nrho_max] in shared memory). Fixed
// point with the bound max|g| of the column times each piece's plan-time
// weight bound for the column; a non-finite g makes the profiles NaN.
template <int NT>
__global__ void __launch_bounds__(256) k_col_profiles_cols(const PieceDev* __restrict__ pieces,
                                                           const int4* __restrict__ cmap, int nrho_max, int ntau_all,
                                                           int np_all, const float* __restrict__ g) {
    const int4 c = np_all > 0 ? make_int4(0, np_all, (int)blockIdx.x, 0) : __ldg(cmap + blockIdx.x);
    const int l = c.z, np = c.y;
    const int Ntau = np_all > 0 ? ntau_all : pieces[c.x].Ntau;
    if (np > kMaxColPieces || (size_t)np * nrho_max * sizeof(int) > dyn_smem_bytes()) return;
    int* prof = reinterpret_cast<int*>(smem_f);
    __shared__ float red[8];
    __shared__ const int2* s_rt[kMaxColPieces];
    __shared__ float* s_hl[kMaxColPieces];
    __shared__ float s_sc[kMaxColPieces];
    __shared__ int s_sh[kMaxColPieces];
    __shared__ int2 s_rg[kMaxColPieces];
    __shared__ int s_nr[kMaxColPieces], s_hp[kMaxColPieces];
    if ((int)threadIdx.x < np) {
        const PieceDev& P = pieces[c.x + threadIdx.x];
        const int lc = l - P.l_lo;
        s_rt[threadIdx.x] = reinterpret_cast<const int2*>(P.rtab + (size_t)lc * Ntau);
        s_hl[threadIdx.x] = P.prof + (size_t)lc * P.hpitch;
        s_sc[threadIdx.x] = __ldg(P.colscale + lc);
        s_sh[threadIdx.x] = __ldg(P.colsh + lc);
        s_rg[threadIdx.x] = __ldg(P.rrange + lc);
        s_nr[threadIdx.x] = P.Nrho;
        s_hp[threadIdx.x] = P.hpitch;
    }
    for (int i = threadIdx.x; i < np * nrho_max; i += blockDim.x) prof[i] = 0;
    const float* gl = g + (np_all > 0 ? 0 : pieces[c.x].g_off) + (size_t)l * Ntau;
    constexpr int Q = 8;                        // outputs per thread
    const int chunk = Q * (int)blockDim.x;
    float mx = 0.f;
    for (int i0 = 0; i0 < Ntau; i0 += chunk) {
        float v[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int i = i0 + q * (int)blockDim.x + threadIdx.x;
            v[q] = i < Ntau ? __ldg(gl + i) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const float a = fabsf(v[q]);
            mx = (a > mx || a != a) ? a : mx;
        }
    }
    const float vmax = block_max_abs(mx, red);   // also orders the zeroing and the column data before use
    if (!(vmax > 0.f && vmax <= 3.402823466e38f)) {
        const float fill = vmax == 0.f ? 0.f : __int_as_float(0x7fc00000);
        for (int p = 0; p < np; ++p)
            for (int n = threadIdx.x; n < s_hp[p]; n += blockDim.x) s_hl[p][n] = fill;
        return;
    }
    const int ev = ilogbf(vmax);
    int lo = Ntau, hi = -1;                     // outputs valid in some piece
    for (int p = 0; p < np; ++p) {
        lo = min(lo, s_rg[p].x);
        hi = max(hi, s_rg[p].y);
    }
    // every thread takes Q consecutive outputs: their first rho tap is
    // nondecreasing, so each piece's contributions collect in an NT-cell
    // register window that slides one cell as the tap advances (the
    // departing cell goes to the shared profile) and is flushed whole on a
    // longer jump; dozens of outputs that share a cell at small intercept
    // times cost one add
    for (int i0 = lo & ~7; i0 <= hi; i0 += chunk) {
        const int ib = i0 + Q * (int)threadIdx.x;
        float v[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) v[q] = (ib + q >= lo && ib + q <= hi) ? __ldg(gl + ib + q) : 0.f;
        for (int p = 0; p < np; ++p) {
            const int2 rg = s_rg[p];
            const int2* rt = s_rt[p];
            int2 e[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int i = ib + q;
                e[q] = (i >= rg.x && i <= rg.y) ? __ldg(rt + i) : make_int2(-1, 0);
            }
            const Pow2Scale scl(s_sh[p] - ev);
            const float sc = s_sc[p];
            int* pr = prof + p * nrho_max;
            float w[NT];
#pragma unroll
            for (int k = 0; k < NT; ++k) w[k] = 0.f;
            int wn = -1;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int n0 = e[q].x;
                if (n0 < 0) continue;
                if (wn < 0) {
                    wn = n0;
                } else if (n0 != wn) {
                    if (n0 == wn + 1) {
                        red_fixed(pr + wn, w[0]);
#pragma unroll
                        for (int k = 0; k + 1 < NT; ++k) w[k] = w[k + 1];
                        w[NT - 1] = 0.f;
                    } else {
#pragma unroll
                        for (int k = 0; k < NT; ++k) {
                            red_fixed(pr + wn + k, w[k]);
                            w[k] = 0.f;
                        }
                    }
                    wn = n0;
                }
                float wr[NT];
                bspline_weights<NT>(__int_as_float(e[q].y), wr);
                const float x = scl.up(v[q] * sc);
#pragma unroll
                for (int k = 0; k < NT; ++k) w[k] = fmaf(x, wr[k], w[k]);
            }
            if (wn >= 0) {
#pragma unroll
                for (int k = 0; k < NT; ++k) red_fixed(pr + wn + k, w[k]);
            }
        }
    }
    __syncthreads();
    for (int p = 0; p < np; ++p) {
        const Pow2Scale scl(s_sh[p] - ev);
        const int* pr = prof + p * nrho_max;
        const int nr = s_nr[p];
        float* hl = s_hl[p];
        for (int n = threadIdx.x; n < s_hp[p]; n += blockDim.x) hl[n] = n < nr ? scl.down(pr[n]) : 0.f;
    }
}

// One band of R <= kMaxBandRows lattice rows: G' rows from the profiles of
// the band's candidate columns (NT theta taps of each column from the plan),
// then the row FFT into the half spectrum. Each thread owns four rho cells
// of every row of the band and sums the columns in order in registers.
template <class Src, int NT>
__global__ void __launch_bounds__(512, 2) k_band_rows(const __grid_constant__ Src B) {
    int band;
    const PieceDev& P = piece_of(B, band);
    if (P.CB != 2 || rows_smem(P) > dyn_smem_bytes()) return;
    const float* __restrict__ h = P.prof;
    const int hp = P.hpitch;
    const int mb = band * P.R;
    const int nrows = min(P.R, P.Ntheta - mb);
    const int2 lr = __ldg(P.lband + band);
    const int Pr = P.Prho;
    for (int n4 = threadIdx.x; n4 < Pr / 4; n4 += blockDim.x) {
        float4 acc[kMaxBandRows];
#pragma unroll
        for (int r = 0; r < kMaxBandRows; ++r) acc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (4 * n4 < hp) {
#pragma unroll 4
            for (int l = lr.x; l <= lr.y; ++l) {
                const int lc = l - P.l_lo;
                const int a0 = mb - __ldg(P.colm0 + lc);     // tap of the band's first row
                const float4 w4 = __ldg(P.colw + lc);
                const float2 w2 = NT > 4 ? __ldg(P.colw2 + lc) : make_float2(0.f, 0.f);
                const float4 hv = __ldg(reinterpret_cast<const float4*>(h + (size_t)lc * hp) + n4);
#pragma unroll
                for (int r = 0; r < kMaxBandRows; ++r) {
                    const int a = a0 + r;
                    if (r < nrows && a >= 0 && a < NT) {
                        const float w = a == 0 ? w4.x : a == 1 ? w4.y : a == 2 ? w4.z : a == 3 ? w4.w
                                      : a == 4 ? w2.x : w2.y;
                        acc[r].x = fmaf(w, hv.x, acc[r].x);
                        acc[r].y = fmaf(w, hv.y, acc[r].y);
                        acc[r].z = fmaf(w, hv.z, acc[r].z);
                        acc[r].w = fmaf(w, hv.w, acc[r].w);
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kMaxBandRows; ++r) {
            if (r < nrows) {
                float* row = smem_f + r * 2 * row_stride(Pr / 2);
                const int n = 4 * n4;
                row[swr(n)] = acc[r].x;
                row[swr(n + 1)] = acc[r].y;
                row[swr(n + 2)] = acc[r].z;
                row[swr(n + 3)] = acc[r].w;
            }
        }
    }
    __syncthreads();
    rows_fwd_passes(reinterpret_cast<cf*>(smem_f), P.Prho / 2, nrows, P.fftM, P.twM, 0);
    rows_post(P, reinterpret_cast<const cf*>(smem_f), mb, nrows);
}

// --------------------------------------------------------------------------
// Column pass: FFT along theta, product with K (or conj K), inverse FFT
// (Eq. (16)-(17)). One CTA of kColThreads threads per block of two spectrum
// columns, which the blocked layout [kb][m][2] stores as one 16-byte row per
// lattice row; thread pairs (2 t, 2 t + 1) take the same butterfly of the two
// columns, so every shared and global access of a pair is one 16-byte word
// (shared buffer [Ptheta] of 16-byte elements, swizzled by swc). One column
// per thread keeps a radix-16 butterfly in 64 registers; three CTAs (30
// warps) per SM hide the pass latencies (measured at 2048^2: 49.5 us against
// 54.7 us at 512 threads and two CTAs per SM, 59 us at 384 threads; earlier,
// both columns per thread at 256 threads 90 us, that at one CTA per SM 112).
// The column block's slice of K and the pass twiddle tables are copied into
// shared memory (cp.async) while pass 0 runs.
//
// The pair runs in place by decimation in frequency / time (dif_plan):
//   pass 0        reads the column block's Ntheta rows straight from global
//                 memory (the zero padding is never loaded) and writes
//                 shared memory;
//   passes 1..    forward passes in shared memory, one barrier each;
//   last pass     (stride 1) forward butterfly, product with K at each
//                 element's frequency (digit-reversed order: no reordering),
//                 inverse butterfly, all in registers;
//   back down     inverse passes, the last one writing only the Ntheta rows
//                 back to global memory.
// --------------------------------------------------------------------------
// Threads of a column-pass CTA: two per butterfly of the two columns. 320
// keeps the radix-16 passes of the R0 * 256 lengths (144 or 160 butterflies
// per column) 90-100 % busy, with three CTAs per SM; launches with a piece of
// another length (the general passes, all twiddle tables in shared memory)
// take 512 threads and two CTAs per SM.
constexpr int kColThreads = 320;
constexpr int kColThreadsGeneral = 512;
// 16-byte asynchronous copies global -> shared (cp.async; the completion
// wait is the hardware's, no spin loop).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

template <int R>
__device__ __forceinline__ void c1_fwd(cf x[R], const cf* T, int S, int m) {
    dft_small<R>(x, -1);
    if (S > 1) {
#pragma unroll
        for (int k = 1; k < R; ++k) x[k] = cmul(x[k], T[(k - 1) * S + m]);
    }
}
template <int R>
__device__ __forceinline__ void c1_inv(cf x[R], const cf* T, int S, int m) {
    if (S > 1) {
#pragma unroll
        for (int k = 1; k < R; ++k) x[k] = cmulc(x[k], T[(k - 1) * S + m]);
    }
    dft_small<R>(x, +1);
}
template <int R>
__device__ __forceinline__ void c1_ld(const cf* A, int base, int S, int c, cf x[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = A[2 * swc(base + r * S) + c];
}
template <int R>
__device__ __forceinline__ void c1_st(cf* A, int base, int S, int c, const cf x[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) A[2 * swc(base + r * S) + c] = x[r];
}
template <int R>
__device__ __forceinline__ void c1_first(cf* A, const cf* __restrict__ col, int Nth, int S, const cf* T, int t, int nt, int c) {
    for (int m = t; m < S; m += nt) {
        cf x[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = m + r * S;
            x[r] = row < Nth ? ldcf(col + 2 * row + c) : cf{0.f, 0.f};
        }
        c1_fwd<R>(x, T, S, m);
        c1_st<R>(A, m, S, c, x);
    }
}
template <int R>
__device__ __forceinline__ void c1_last(const cf* A, cf* col, int Nth, int S, const cf* T, int t, int nt, int c) {
    for (int m = t; m < S; m += nt) {
        cf x[R];
        c1_ld<R>(A, m, S, c, x);
        c1_inv<R>(x, T, S, m);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = m + r * S;
            if (row < Nth) col[2 * row + c] = x[r];
        }
    }
}
template <int R, bool INV>
__device__ __forceinline__ void c1_mid(cf* A, int n, int S, const cf* T, int t, int nt, int c) {
    const int nb = n / R;
    const float invS = 1.0f / (float)S;
    for (int b = t; b < nb; b += nt) {
        const int q = (int)(((float)b + 0.5f) * invS);
        const int m = b - q * S;
        const int base = q * S * R + m;
        cf x[R];
        c1_ld<R>(A, base, S, c, x);
        if (INV) c1_inv<R>(x, T, S, m);
        else c1_fwd<R>(x, T, S, m);
        c1_st<R>(A, base, S, c, x);
    }
}
template <int R>
__device__ __forceinline__ void c1_kernel(cf* A, const FftPlan& fp, const cf* K, int k1n, int adjoint, int t, int nt, int c) {
    const int n = fp.n, s = fp.nst;
    const int nb = n / R;
    for (int b = t; b < nb; b += nt) {
        int fb = 0, w = 1, rem = b;
        for (int p = 0; p + 1 < s; ++p) {
            const int d = fp.st[p] / R;
            const int k = (int)(((float)rem + 0.5f) / (float)d);
            rem -= k * d;
            fb += k * w;
            w *= fp.rad[p];
        }
        cf x[R];
        c1_ld<R>(A, b * R, 1, c, x);
        dft_small<R>(x, -1);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int f = fb + nb * k;
            const int kk = f <= n - f ? f : n - f;
            if (kk < k1n) {
                const cf kv = K[2 * kk + c];
                x[k] = adjoint ? cmulc(x[k], kv) : cmul(x[k], kv);
            } else {
                x[k] = cf{0.f, 0.f};
            }
        }
        dft_small<R>(x, +1);
        c1_st<R>(A, b * R, 1, c, x);
    }
}

// The pair for Ptheta = R0 * 256 (radices R0, 16, 16: the plans of the
// 2048^2 workload) with every stride and count a compile-time constant: one
// butterfly per thread and pass (256 threads per column), the stride-1
// pass's first frequency b / 16 + R0 (b mod 16) without the general digit
// loop. Same arithmetic as the general passes.
template <int R0>
__device__ __forceinline__ void c1_x256(cf* A, cf* col, int Nth, const cf* Tg, const cf* T1, const cf* K, int k1n,
                                        int adjoint, int t, int nt, int c) {
    constexpr int n = R0 * 256, nb = R0 * 16;
    c1_first<R0>(A, col, Nth, 256, Tg, t, nt, c);
    cp_async_wait_all();
    __syncthreads();
    for (int b = t; b < nb; b += nt) {
        const int q = b >> 4, m = b & 15;
        cf x[16];
        c1_ld<16>(A, q * 256 + m, 16, c, x);
        c1_fwd<16>(x, T1, 16, m);
        c1_st<16>(A, q * 256 + m, 16, c, x);
    }
    __syncthreads();
    for (int b = t; b < nb; b += nt) {
        const int q = b >> 4, m = b & 15;
        const int fb = q + R0 * m;
        cf x[16];
        c1_ld<16>(A, b * 16, 1, c, x);
        // forward DFT, product with K, inverse DFT as conj(DFT(conj(.))):
        // one DFT body run twice (half the code of the pass)
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            dft_small<16>(x, -1);
            if (h == 0) {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int f = fb + nb * k;
                    const int kk = f <= n - f ? f : n - f;
                    if (kk < k1n) {
                        const cf kv = K[2 * kk + c];
                        x[k] = cconj(adjoint ? cmulc(x[k], kv) : cmul(x[k], kv));
                    } else {
                        x[k] = cf{0.f, 0.f};
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < 16; ++k) x[k] = cconj(x[k]);
            }
        }
        c1_st<16>(A, b * 16, 1, c, x);
    }
    __syncthreads();
    for (int b = t; b < nb; b += nt) {
        const int q = b >> 4, m = b & 15;
        cf x[16];
        c1_ld<16>(A, q * 256 + m, 16, c, x);
        c1_inv<16>(x, T1, 16, m);
        c1_st<16>(A, q * 256 + m, 16, c, x);
    }
    __syncthreads();
    c1_last<R0>(A, col, Nth, 256, Tg, t, nt, c);
}

// R0 of a column plan that the compile-time pair c1_x256 serves, else 0.
__host__ __device__ __forceinline__ int colconv_x256(const FftPlan& fp) {
    if (fp.nst != 3 || fp.st[0] != 256 || fp.rad[1] != 16 || fp.rad[2] != 16) return 0;
    const int r = fp.rad[0];
    return (r == 5 || r == 6 || r == 8 || r == 9 || r == 10 || r == 12) ? r : 0;
}

// Shared memory of the column kernel: the column block [Ptheta] (16-byte
// elements), its slice of K [k1max + 1] (16 bytes each), the twiddle tables
// (twlen complex, a multiple of 2): all passes' tables, or for the
// compile-time pair only the stride-16 pass's 240 (the first pass reads its
// own from global memory), which lets three CTAs share an SM.
constexpr int kX256Twiddles = 16 * 15;
__host__ __device__ __forceinline__ size_t colconv_smem(int Pt, int k1n, int twlen) {
    return ((size_t)Pt + k1n) * 16 + (size_t)twlen * 8;
}
__host__ __device__ __forceinline__ size_t colconv_smem(const PieceDev& P) {
    return colconv_smem(P.Ptheta, P.k1max + 1, colconv_x256(P.fftT) ? kX256Twiddles : P.twT_len);
}

template <class Src, int TPB>
__global__ void __launch_bounds__(TPB, TPB == kColThreads ? 3 : 2) k_colconv(const __grid_constant__ Src B, int adjoint) {
    int kb;
    const PieceDev& P = piece_of(B, kb);
    const int Pt = P.Ptheta, Nth = P.Ntheta, k1n = P.k1max + 1;
    if (P.CB != 2 || (P.twT_len & 1) || colconv_smem(P) > dyn_smem_bytes()) return;
    const int x256 = colconv_x256(P.fftT);
    float4* A4 = reinterpret_cast<float4*>(smem_f);
    float4* Ks4 = A4 + Pt;
    cf* Ts = reinterpret_cast<cf*>(Ks4 + k1n);
    cf* A = reinterpret_cast<cf*>(A4);
    const cf* K = reinterpret_cast<const cf*>(Ks4);
    cf* col = P.spec + (size_t)kb * Nth * 2;
    {
        const float4* Kg = reinterpret_cast<const float4*>(P.K) + (size_t)kb * k1n;
        for (int i = threadIdx.x; i < k1n; i += blockDim.x) cp_async16(Ks4 + i, Kg + i);
        const float4* Tg = reinterpret_cast<const float4*>(P.twT + (x256 ? P.fftT.tw[1] : 0));
        float4* T4 = reinterpret_cast<float4*>(Ts);
        const int n4 = (x256 ? kX256Twiddles : P.twT_len) / 2;
        for (int i = threadIdx.x; i < n4; i += blockDim.x) cp_async16(T4 + i, Tg + i);
    }
    const int c = threadIdx.x & 1, t = threadIdx.x >> 1, nt = blockDim.x >> 1;
    const FftPlan& fp = P.fftT;
    const int s = fp.nst;
    const cf* T = Ts;
    const int R0 = fp.rad[0], S0 = fp.st[0];
    if (s == 1) {
        for (int m = threadIdx.x; m < Pt; m += blockDim.x)
            A4[swc(m)] = m < Nth ? __ldg(reinterpret_cast<const float4*>(col) + m) : make_float4(0.f, 0.f, 0.f, 0.f);
        cp_async_wait_all();
        __syncthreads();
#define HR_K(RR) c1_kernel<RR>(A, fp, K, k1n, adjoint, t, nt, c)
        switch (R0) { HR_RADIX_CASES(HR_K) }
        __syncthreads();
        for (int m = threadIdx.x; m < Nth; m += blockDim.x) reinterpret_cast<float4*>(col)[m] = A4[swc(m)];
        return;
    }
    switch (x256) {
        case 5: c1_x256<5>(A, col, Nth, P.twT, T, K, k1n, adjoint, t, nt, c); return;
        case 6: c1_x256<6>(A, col, Nth, P.twT, T, K, k1n, adjoint, t, nt, c); return;
        case 8: c1_x256<8>(A, col, Nth, P.twT, T, K, k1n, adjoint, t, nt, c); return;
        case 9: c1_x256<9>(A, col, Nth, P.twT, T, K, k1n, adjoint, t, nt, c); return;
        case 10: c1_x256<10>(A, col, Nth, P.twT, T, K, k1n, adjoint, t, nt, c); return;
        case 12: c1_x256<12>(A, col, Nth, P.twT, T, K, k1n, adjoint, t, nt, c); return;
        default: break;
    }
#define HR_FIRST(RR) c1_first<RR>(A, col, Nth, S0, P.twT, t, nt, c)
    switch (R0) { HR_RADIX_CASES(HR_FIRST) }
    cp_async_wait_all();
    __syncthreads();
    for (int p = 1; p + 1 < s; ++p) {
#define HR_FWD(RR) c1_mid<RR, false>(A, Pt, fp.st[p], T + fp.tw[p], t, nt, c)
        switch (fp.rad[p]) { HR_RADIX_CASES(HR_FWD) }
        __syncthreads();
    }
    switch (fp.rad[s - 1]) { HR_RADIX_CASES(HR_K) }
    __syncthreads();
    for (int p = s - 2; p >= 1; --p) {
#define HR_INV(RR) c1_mid<RR, true>(A, Pt, fp.st[p], T + fp.tw[p], t, nt, c)
        switch (fp.rad[p]) { HR_RADIX_CASES(HR_INV) }
        __syncthreads();
    }
#define HR_LAST(RR) c1_last<RR>(A, col, Nth, S0, T, t, nt, c)
    switch (R0) { HR_RADIX_CASES(HR_LAST) }
#undef HR_K
#undef HR_FIRST
#undef HR_FWD
#undef HR_INV
#undef HR_LAST
}

// --------------------------------------------------------------------------
// Inverse real FFT of a band of rows from the half spectrum (bins <= k2max,
// the rest zero) into the real lattice P.lat[Ntheta][Nrho]: the
// pre-processing reads the spectrum from global memory, the last pass writes
// the lattice rows.
// --------------------------------------------------------------------------
template <class Src>
__global__ void __launch_bounds__(512, 2) k_rows_c2r(const __grid_constant__ Src B) {
    int bx;
    const PieceDev& P = piece_of(B, bx);
    if (P.CB != 2 || rows_smem(P) > dyn_smem_bytes()) return;
    const int mb = bx * P.R;
    const int nrows = min(P.R, P.Ntheta - mb);
    const int M = P.Prho / 2;
    cf* X = reinterpret_cast<cf*>(smem_f);
    const FftPlan& fp = P.fftM;
    rows_pre(P, X, mb, nrows);
    __syncthreads();
    switch (plan_x256(fp)) {
#define HR_CX(R0)                                                                    \
    rows_pass_c<16, 1, R0 * 256, true>(X, nrows, P.twM);                             \
    __syncthreads();                                                                 \
    rows_pass_c<16, 16, R0 * 256, true>(X, nrows, P.twM + fp.tw[1]);                 \
    __syncthreads();                                                                 \
    rows_last_lat_c<R0>(X, P.lat + (size_t)mb * P.Nrho, P.Nrho, nrows, P.twM);       \
    return;
        HR_X256_CASES(HR_CX)
#undef HR_CX
        default: break;
    }
    for (int p = fp.nst - 1; p >= 1; --p) {
#define HR_RI(RR) rows_pass<RR, true>(X, M, nrows, fp.st[p], P.twM + fp.tw[p])
        switch (fp.rad[p]) { HR_RADIX_CASES(HR_RI) }
#undef HR_RI
        __syncthreads();
    }
#define HR_RW(RR) rows_last_lat<RR>(X, P.lat + (size_t)mb * P.Nrho, P.Nrho, M, nrows, fp.st[0], P.twM)
    switch (fp.rad[0]) { HR_RADIX_CASES(HR_RW) }
#undef HR_RW
}

// --------------------------------------------------------------------------
// Gathers.
// --------------------------------------------------------------------------

// NT x NT taps of the lattice at first tap (m0, n0).
template <int NT>
__device__ __forceinline__ float taps_nt(const float* __restrict__ lat, int Nr, int m0, int n0,
                                         const float (&wt)[NT], const float (&wr)[NT]) {
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < NT; ++a) {
        const float* row = lat + (size_t)(m0 + a) * Nr + n0;
        float r = __ldg(row) * wr[0];
#pragma unroll
        for (int c = 1; c < NT; ++c) r += __ldg(row + c) * wr[c];
        s += wt[a] * r;
    }
    return s;
}

// Forward output interpolation (Eq. (17)): one CTA per output column, summed
// over the time pieces of its slowness piece; cmap[b] = (first piece, number
// of pieces, column l). As in the adjoint, the column's outputs share its
// theta taps, so the NT x NT taps separate: the CTA first spreads the NT
// lattice rows of the column's angle into a rho profile in shared memory,
//   r[n] = sum_a B(theta_l - theta_{m0+a}) H[m0 + a][n],
// for every time piece at once (shared memory: [np][nrho_max] profiles),
// then every output takes NT taps of each piece's profile and sums the
// pieces in a fixed order. Outputs outside a piece's valid range skip its
// table.
template <int NT>
__global__ void __launch_bounds__(256) k_interp_columns(const PieceDev* __restrict__ pieces,
                                                        const int4* __restrict__ cmap, int nrho_max,
                                                        int ntau_all, int np_all, float* __restrict__ g) {
    // np_all > 0: one gather with one slowness piece of np_all time pieces and
    // ntau_all outputs per column, column = block (no map load before the work)
    const int4 c = np_all > 0 ? make_int4(0, np_all, (int)blockIdx.x, 0) : __ldg(cmap + blockIdx.x);
    const int l = c.z, np = c.y;
    const int Ntau = np_all > 0 ? ntau_all : pieces[c.x].Ntau;
    if (np > kMaxColPieces || (size_t)np * nrho_max * sizeof(float) > dyn_smem_bytes()) return;
    // per-piece column data, loaded for all pieces at once
    __shared__ float4 s_w4[kMaxColPieces];
    __shared__ float2 s_w2[NT > 4 ? kMaxColPieces : 1];
    __shared__ const float* s_r0[kMaxColPieces];
    __shared__ const int2* s_rt[kMaxColPieces];
    __shared__ float s_sc[kMaxColPieces];
    __shared__ int2 s_rg[kMaxColPieces];
    __shared__ int s_nr[kMaxColPieces];
    if ((int)threadIdx.x < np) {
        const PieceDev& P = pieces[c.x + threadIdx.x];
        const int lc = l - P.l_lo;
        s_w4[threadIdx.x] = __ldg(P.colw + lc);
        if (NT > 4) s_w2[threadIdx.x] = __ldg(P.colw2 + lc);
        s_sc[threadIdx.x] = __ldg(P.colscale + lc);
        s_r0[threadIdx.x] = P.lat + (size_t)__ldg(P.colm0 + lc) * P.Nrho;
        s_rt[threadIdx.x] = reinterpret_cast<const int2*>(P.rtab + (size_t)lc * Ntau);
        s_rg[threadIdx.x] = __ldg(P.rrange + lc);
        s_nr[threadIdx.x] = P.Nrho;
    }
    __syncthreads();
    // theta taps (the column's NT lattice rows) of every piece: the rho
    // profiles, np * nrho_max floats; all pieces' loads in flight together
    for (int p = 0; p < np; ++p) {
        const int Nr = s_nr[p];
        const float4 w4 = s_w4[p];
        const float* r0 = s_r0[p];
        float* prof = smem_f + p * nrho_max;
#pragma unroll 2
        for (int n = threadIdx.x; n < Nr; n += blockDim.x) {
            const float a0 = __ldg(r0 + n), a1 = __ldg(r0 + Nr + n);
            const float a2 = __ldg(r0 + 2 * Nr + n), a3 = __ldg(r0 + 3 * Nr + n);
            if (NT > 4) {
                const float2 w2 = s_w2[p];
                const float a4 = __ldg(r0 + 4 * Nr + n), a5 = __ldg(r0 + 5 * Nr + n);
                prof[n] = w4.x * a0 + w4.y * a1 + w4.z * a2 + w4.w * a3 + w2.x * a4 + w2.y * a5;
            } else {
                prof[n] = w4.x * a0 + w4.y * a1 + w4.z * a2 + w4.w * a3;
            }
        }
    }
    __syncthreads();
    // rho taps: every output sums its pieces in piece order
    float* gl = g + (np_all > 0 ? 0 : pieces[c.x].g_off) + (size_t)l * Ntau;
    // each thread takes U outputs at once and loads their table entries of a
    // piece together before using any (the entries come from DRAM and each
    // output's taps wait on its entry: U chains in flight instead of one)
    constexpr int U = 4;
    for (int i0 = threadIdx.x; i0 < Ntau; i0 += U * blockDim.x) {
        float acc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) acc[u] = 0.f;
        for (int p = 0; p < np; ++p) {
            const int2 rg = s_rg[p];
            int2 e[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 + u * (int)blockDim.x;
                e[u] = (i >= rg.x && i <= rg.y) ? __ldg(s_rt[p] + i) : make_int2(-1, 0);
            }
            const float scp = s_sc[p];
            const float* rp = smem_f + p * nrho_max;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (e[u].x < 0) continue;
                float wr[NT];
                bspline_weights<NT>(__int_as_float(e[u].y), wr);
                const float* r = rp + e[u].x;
                float t = wr[0] * r[0];
#pragma unroll
                for (int c = 1; c < NT; ++c) t += wr[c] * r[c];
                acc[u] += scp * t;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * (int)blockDim.x;
            if (i < Ntau) gl[i] = acc[u];
        }
    }
}

// Adjoint of the gridding (transpose of Eq. (15)): every gather sample reads
// the NT x NT taps of each sub-problem that holds it. One CTA per kSampleBlock
// samples of one gather: smap[b] = (first piece, number of pieces, first
// sample of the block within the gather).
template <int NT>
__global__ void __launch_bounds__(kSampleBlock, NT == 4 ? 8 : 4) k_gather_samples(const PieceDev* __restrict__ pieces,
                                                                    const int4* __restrict__ smap,
                                                                    float* __restrict__ f, int np_all, int Nt_all,
                                                                    int Nx_all) {
    // np_all > 0: one gather of Nt_all x Nx_all samples in np_all pieces,
    // samples = blocks in order (no map load before the work)
    const int4 m = np_all > 0 ? make_int4(0, np_all, (int)blockIdx.x * kSampleBlock, 0) : __ldg(smap + blockIdx.x);
    const int Nt = np_all > 0 ? Nt_all : pieces[m.x].Nt;
    const int Nx = np_all > 0 ? Nx_all : pieces[m.x].Nx;
    const long idx = (long)m.z + threadIdx.x;
    if (idx >= (long)Nt * Nx) return;
    const int k = (int)(idx / Nt);
    const int j = (int)(idx - (long)k * Nt);
    float acc = 0.f;
    for (int p = m.x; p < m.x + m.y; ++p) {
        const PieceDev& P = pieces[p];
        if (j < P.jt_lo || j > P.jt_hi) continue;
        const int4 e = __ldg(reinterpret_cast<const int4*>(P.stab + (size_t)k * P.nj + (j - P.jt_lo)));
        const float w = __int_as_float(e.w);
        if (w == 0.f) continue;
        float wt[NT], wr[NT];
        bspline_weights<NT>(__int_as_float(e.y), wt);
        bspline_weights<NT>(__int_as_float(e.z), wr);
        acc += w * taps_nt<NT>(P.lat, P.Nrho, e.x >> 16, e.x & 0xffff, wt, wr);
    }
    f[(np_all > 0 ? 0 : pieces[m.x].f_off) + idx] = acc;
}

// --------------------------------------------------------------------------
// Plan time, FP64: lattice positions of every gather sample and of every
// output (the maps P1 T of Eq. (10)/(14) and P2 S of Eq. (9)/(17)).
// --------------------------------------------------------------------------
__global__ void k_sample_table(TableArgs A, const double* __restrict__ cj, const double* __restrict__ wk,
                               const int* __restrict__ jfirst, SampleEnt* __restrict__ out) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)A.nj * A.Nx) return;
    const int k = (int)(idx / A.nj);
    const int jl = (int)(idx - (long)k * A.nj);
    const int j = A.jt_lo + jl;
    const double tb = j / A.n_t, xb = A.xb[k];
    const double ds = tb * tb - 0.5, dy = xb * xb - 0.5;
    const double u1 = A.a * (A.ca * ds - A.sa * dy) + A.O1;
    const double u2 = A.a * (A.sa * ds + A.ca * dy) + A.O2;
    const double r2 = u1 * u1 + u2 * u2;
    const double xth = (atan2(u2, u1) - A.theta0) / A.dtheta;
    const double xrh = (0.5 * log(r2) - A.rho0) / A.drho;
    const double fm = floor(xth), fn = floor(xrh);
    const int back = A.ntaps / 2 - 1;            // first tap: floor - (order - 1) / 2
    int m0 = (int)fm - back, n0 = (int)fn - back;
    double w = (j >= jfirst[k]) ? cj[jl] * wk[k] / sqrt(r2) : 0.0;
    if (m0 < 0 || m0 + A.ntaps - 1 >= A.Ntheta || n0 < 0 || n0 + A.ntaps - 1 >= A.Nrho) {
        w = 0.0;
        m0 = 0;
        n0 = 0;
    }
    SampleEnt e;
    e.mn = (m0 << 16) | n0;
    e.ft = (float)(xth - fm);
    e.fr = (float)(xrh - fn);
    e.w = (float)w;
    out[idx] = e;
}

__global__ void k_radon_table(TableArgs A, const double* __restrict__ qb2, RadonEnt* __restrict__ out) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)A.ncol * A.Ntau) return;
    const int lc = (int)(idx / A.Ntau);
    const int i = (int)(idx - (long)lc * A.Ntau);
    const double m = qb2[lc];
    const double psi = atan(m);
    const double theta = A.alpha - psi;
    const double tb = (A.tau0 + i * A.dtau) / A.T;
    const double e = A.a * cos(psi) * (tb * tb - 0.5 + 0.5 * m) + A.O1 * cos(theta) + A.O2 * sin(theta);
    RadonEnt r;
    r.n0 = -1;
    r.fr = 0.f;
    if (e >= A.a_r && e <= A.r_max) {
        const double xrh = (log(e) - A.rho0) / A.drho;
        const double fn = floor(xrh);
        const int n0 = (int)fn - (A.ntaps / 2 - 1);
        if (n0 >= 0 && n0 + A.ntaps - 1 < A.Nrho) {
            r.n0 = n0;
            r.fr = (float)(xrh - fn);
        }
    }
    out[idx] = r;
}

// --------------------------------------------------------------------------
// Plan time, FP64: zeta_hat as a quadrature written as a matrix product,
// Z = A B with A[k1][n] = cos(2 pi theta_n w1) and B[n][k2] the complex
// weights (real and imaginary parts as two matrices). 16x16 tiles.
// --------------------------------------------------------------------------
__global__ void k_zeta_gemm(const double* __restrict__ A, const double* __restrict__ Bre,
                            const double* __restrict__ Bim, int n1, int nn, int n2,
                            double* __restrict__ Zre, double* __restrict__ Zim) {
    __shared__ double sA[16][17];
    __shared__ double sR[16][17];
    __shared__ double sI[16][17];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int row = blockIdx.y * 16 + ty;   // k1
    const int col = blockIdx.x * 16 + tx;   // k2
    double accr = 0.0, acci = 0.0;
    for (int t0 = 0; t0 < nn; t0 += 16) {
        const int ta = t0 + tx, tb = t0 + ty;
        sA[ty][tx] = (row < n1 && ta < nn) ? A[(size_t)row * nn + ta] : 0.0;
        sR[ty][tx] = (tb < nn && col < n2) ? Bre[(size_t)tb * n2 + col] : 0.0;
        sI[ty][tx] = (tb < nn && col < n2) ? Bim[(size_t)tb * n2 + col] : 0.0;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            accr = fma(sA[ty][q], sR[q][tx], accr);
            acci = fma(sA[ty][q], sI[q][tx], acci);
        }
        __syncthreads();
    }
    if (row < n1 && col < n2) {
        Zre[(size_t)row * n2 + col] = accr;
        Zim[(size_t)row * n2 + col] = acci;
    }
}

// --------------------------------------------------------------------------
// Direct summation over hyperbolas on the GPU (FP32): the plain O(N^3)
// comparator, Eq. (3) with the same discretisation as the paper's reference
// (Keys cubic in t, trapezoid in x).
// --------------------------------------------------------------------------
__device__ __forceinline__ float keys_w(float s) {
    s = fabsf(s);
    if (s <= 1.f) return (1.5f * s - 2.5f) * s * s + 1.f;
    if (s < 2.f) return ((-0.5f * s + 2.5f) * s - 4.f) * s + 2.f;
    return 0.f;
}

__global__ void __launch_bounds__(256) k_direct_fwd(const float* __restrict__ f, float* __restrict__ g,
                                                    int Nt, int Nx, int Ntau, float tau0_dt,
                                                    float dtau_dt, float qmin_dx_dt, float dq_dx_dt,
                                                    float two_dx) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int l = blockIdx.y;
    if (i >= Ntau) return;
    const float tt = tau0_dt + dtau_dt * (float)i;      // tau / dt
    const float qq = qmin_dx_dt + dq_dx_dt * (float)l;  // q dx / dt
    const float tt2 = tt * tt, qq2 = qq * qq;
    float acc = 0.f;
    for (int k = 0; k < Nx; ++k) {
        const float p = sqrtf(tt2 + qq2 * (float)k * (float)k);  // t / dt
        const float fl = floorf(p);
        const int j0 = (int)fl;
        const float s = p - fl;
        const float* tr = f + (size_t)k * Nt;
        float v = 0.f;
        if (j0 - 1 >= 0 && j0 + 2 < Nt) {
            v = __ldg(tr + j0 - 1) * keys_w(s + 1.f) + __ldg(tr + j0) * keys_w(s) +
                __ldg(tr + j0 + 1) * keys_w(s - 1.f) + __ldg(tr + j0 + 2) * keys_w(s - 2.f);
        } else {
#pragma unroll
            for (int d = -1; d <= 2; ++d) {
                const int jj = j0 + d;
                if (jj >= 0 && jj < Nt) v += __ldg(tr + jj) * keys_w(s - (float)d);
            }
        }
        acc += (k == 0 || k == Nx - 1) ? 0.5f * v : v;
    }
    g[(size_t)l * Ntau + i] = two_dx * acc;
}

__global__ void __launch_bounds__(256) k_direct_adj(const float* __restrict__ g, float* __restrict__ f,
                                                    int Nt, int Nx, int Ntau, int Nq, float tau0_dt,
                                                    float dtau_dt, float qmin_dx_dt, float dq_dx_dt,
                                                    float two_dx) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (j >= Nt) return;
    const float kk = (float)k;
    const float lo = fmaxf((float)(j - 2), 0.f), hi = (float)(j + 2);
    float acc = 0.f;
    for (int l = 0; l < Nq; ++l) {
        const float qq = (qmin_dx_dt + dq_dx_dt * (float)l) * kk;   // q x / dt
        const float qq2 = qq * qq;
        const float hi2 = hi * hi - qq2;
        if (hi2 < 0.f) continue;
        const float lo2 = lo * lo - qq2;
        const float tlo = lo2 > 0.f ? sqrtf(lo2) : 0.f;
        const float thi = sqrtf(hi2);
        int i0 = (int)floorf((tlo - tau0_dt) / dtau_dt) - 1;
        int i1 = (int)ceilf((thi - tau0_dt) / dtau_dt) + 1;
        i0 = max(i0, 0);
        i1 = min(i1, Ntau - 1);
        const float* gl = g + (size_t)l * Ntau;
        for (int i = i0; i <= i1; ++i) {
            const float tt = tau0_dt + dtau_dt * (float)i;
            const float p = sqrtf(tt * tt + qq2);
            acc += __ldg(gl + i) * keys_w(p - (float)j);
        }
    }
    f[(size_t)k * Nt + j] = ((k == 0 || k == Nx - 1) ? 0.5f : 1.f) * two_dx * acc;
}

// --------------------------------------------------------------------------
// Launchers
// --------------------------------------------------------------------------
static int check_launch() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 0 : (int)e;
}

size_t scatter_smem_bytes(const PieceDev& P) { return rows_smem(P); }

size_t colconv_smem_bytes(const PieceDev& P) { return colconv_smem(P); }

int max_smem_optin() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

// Dynamic shared-memory limit of a kernel: raised only when a launch needs
// more than the largest value already set on this device (the attribute call
// costs host time on every launch otherwise).
static int set_smem(const void* fn, size_t bytes) {
    struct Entry { const void* fn; int dev; size_t bytes; };
    static std::mutex mu;
    static std::vector<Entry> set;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    for (const Entry& e : set)
        if (e.fn == fn && e.dev == dev && e.bytes >= bytes) return 0;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return (int)e;
    for (Entry& en : set)
        if (en.fn == fn && en.dev == dev) {
            en.bytes = bytes;
            return 0;
        }
    set.push_back(Entry{fn, dev, bytes});
    return 0;
}

// Batch descriptor of n pieces with count(piece) blocks each; returns the
// total number of blocks.
template <class F>
static int make_batch(const PieceDev* P, int n, PieceBatch& B, F&& count) {
    B.n = n;
    int total = 0;
    for (int k = 0; k < kMaxBatch; ++k) {
        B.first[k] = total;
        if (k < n) {
            B.p[k] = P[k];
            total += count(P[k]);
        }
    }
    B.first[kMaxBatch] = total;
    return total;
}

// Kernels with B-spline taps exist for 4 (cubic) and 6 (quintic) taps per
// axis; every piece of one launch has the same number.
#define HR_TAPS(NTAPS, ...)                                           \
    do {                                                              \
        if ((NTAPS) == 6) {                                           \
            constexpr int NT = 6;                                     \
            __VA_ARGS__;                                              \
        } else if ((NTAPS) == 4) {                                    \
            constexpr int NT = 4;                                     \
            __VA_ARGS__;                                              \
        } else {                                                      \
            return (int)cudaErrorInvalidValue;                        \
        }                                                             \
    } while (0)

int launch_grid_tiles(const PieceDev* P, int n, const float* f, void* stream) {
    PieceBatch B;
    const int nb = make_batch(P, n, B, [](const PieceDev& q) { return q.nunits; });
    if (nb > 0)
        HR_TAPS(P[0].ntaps, (k_grid_tiles<PieceBatch, float, NT><<<nb, kUnitChunks, 0, (cudaStream_t)stream>>>(B, f)));
    return check_launch();
}

static size_t max_over(const PieceDev* P, int n, size_t (*fn)(const PieceDev&)) {
    size_t m = 0;
    for (int k = 0; k < n; ++k) m = std::max(m, fn(P[k]));
    return m;
}

size_t rows_smem_bytes(const PieceDev& P) { return scatter_smem_bytes(P); }

// One stage over n <= kMaxBatch pieces (descriptors as a parameter) or over
// a device-resident batch (descriptors and block map in device memory).
template <class Src>
static int set_and_launch(void (*kern)(Src), int nb, size_t sm, const Src& B, void* stream) {
    if (int e = set_smem((const void*)kern, sm)) return e;
    if (nb > 0) kern<<<nb, 512, sm, (cudaStream_t)stream>>>(B);
    return check_launch();
}

int launch_rows_r2c(const PieceDev* P, int n, void* stream) {
    PieceBatch B;
    const int nb = make_batch(P, n, B, [](const PieceDev& q) { return q.nbands; });
    return set_and_launch(k_rows_r2c<PieceBatch>, nb, max_over(P, n, rows_smem_bytes), B, stream);
}

int launch_band_rows(const PieceDev* P, int n, void* stream) {
    PieceBatch B;
    const int nb = make_batch(P, n, B, [](const PieceDev& q) { return q.nbands; });
    const size_t sm = max_over(P, n, rows_smem_bytes);
    if (P[0].ntaps == 6) return set_and_launch(k_band_rows<PieceBatch, 6>, nb, sm, B, stream);
    if (P[0].ntaps == 4) return set_and_launch(k_band_rows<PieceBatch, 4>, nb, sm, B, stream);
    return (int)cudaErrorInvalidValue;
}

bool colconv_all_x256(const PieceDev* P, int n) {
    for (int k = 0; k < n; ++k)
        if (!colconv_x256(P[k].fftT)) return false;
    return true;
}

template <class Src>
static int launch_colconv_as(const Src& B, int nb, size_t sm, bool x256, int adjoint, void* stream) {
    if (x256) {
        if (int e = set_smem((const void*)k_colconv<Src, kColThreads>, sm)) return e;
        if (nb > 0) k_colconv<Src, kColThreads><<<nb, kColThreads, sm, (cudaStream_t)stream>>>(B, adjoint);
    } else {
        if (int e = set_smem((const void*)k_colconv<Src, kColThreadsGeneral>, sm)) return e;
        if (nb > 0)
            k_colconv<Src, kColThreadsGeneral><<<nb, kColThreadsGeneral, sm, (cudaStream_t)stream>>>(B, adjoint);
    }
    return check_launch();
}

int launch_colconv(const PieceDev* P, int n, int adjoint, void* stream) {
    const size_t sm = max_over(P, n, colconv_smem_bytes);
    PieceBatch B;
    const int nb = make_batch(P, n, B, [](const PieceDev& q) { return q.nkb; });
    return launch_colconv_as(B, nb, sm, colconv_all_x256(P, n), adjoint, stream);
}

int launch_rows_c2r(const PieceDev* P, int n, void* stream) {
    PieceBatch B;
    const int nb = make_batch(P, n, B, [](const PieceDev& q) { return q.nbands; });
    return set_and_launch(k_rows_c2r<PieceBatch>, nb, max_over(P, n, rows_smem_bytes), B, stream);
}

int launch_grid_tiles_dev(const DevBatch& S, int nblocks, int ntaps, const void* f, int in_type, void* stream) {
    if (nblocks <= 0) return 0;
    HR_TAPS(ntaps, {
        if (in_type == kInBF16)
            k_grid_tiles<DevBatch, __nv_bfloat16, NT><<<nblocks, kUnitChunks, 0, (cudaStream_t)stream>>>(
                S, (const __nv_bfloat16*)f);
        else
            k_grid_tiles<DevBatch, float, NT><<<nblocks, kUnitChunks, 0, (cudaStream_t)stream>>>(S, (const float*)f);
    });
    return check_launch();
}

int launch_rows_r2c_dev(const DevBatch& S, int nblocks, size_t smem, void* stream) {
    return set_and_launch(k_rows_r2c<DevBatch>, nblocks, smem, S, stream);
}

int launch_band_rows_dev(const DevBatch& S, int nblocks, int ntaps, size_t smem, void* stream) {
    if (ntaps == 6) return set_and_launch(k_band_rows<DevBatch, 6>, nblocks, smem, S, stream);
    if (ntaps == 4) return set_and_launch(k_band_rows<DevBatch, 4>, nblocks, smem, S, stream);
    return (int)cudaErrorInvalidValue;
}

int launch_colconv_dev(const DevBatch& S, int nblocks, size_t smem, bool x256, int adjoint, void* stream) {
    return launch_colconv_as(S, nblocks, smem, x256, adjoint, stream);
}

int launch_rows_c2r_dev(const DevBatch& S, int nblocks, size_t smem, void* stream) {
    return set_and_launch(k_rows_c2r<DevBatch>, nblocks, smem, S, stream);
}

// Dynamic shared memory the per-column profile kernels (the output
// interpolation and its adjoint's profiles) may take on the current device:
// the opt-in limit less the larger of the two kernels' static shared arrays.
size_t interp_smem_limit(int ntaps) {
    size_t stat = 0;
    const void* fns[2] = {ntaps == 6 ? (const void*)k_interp_columns<6> : (const void*)k_interp_columns<4>,
                          ntaps == 6 ? (const void*)k_col_profiles_cols<6> : (const void*)k_col_profiles_cols<4>};
    for (const void* fn : fns) {
        cudaFuncAttributes fa{};
        if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        stat = std::max(stat, (size_t)fa.sharedSizeBytes);
    }
    const size_t lim = (size_t)max_smem_optin();
    return lim > stat ? lim - stat : 0;
}

int launch_col_profiles_cols(const PieceDev* pieces, const int4* cmap, int ncols, int nrho_max, int np_max,
                             int ntau_all, int np_all, int ntaps, const float* g, void* stream) {
    if (np_max > kMaxColPieces) return (int)cudaErrorInvalidValue;
    const size_t sm = (size_t)np_max * nrho_max * sizeof(int);
    HR_TAPS(ntaps, {
        if (int e = set_smem((const void*)k_col_profiles_cols<NT>, sm)) return e;
        if (ncols > 0)
            k_col_profiles_cols<NT><<<ncols, 256, sm, (cudaStream_t)stream>>>(pieces, cmap, nrho_max, ntau_all, np_all,
                                                                              g);
    });
    return check_launch();
}

int launch_interp_columns(const PieceDev* pieces, const int4* cmap, int ncols, int nrho_max, int np_max,
                          int ntau_all, int np_all, int ntaps, float* g, void* stream) {
    if (np_max > kMaxColPieces) return (int)cudaErrorInvalidValue;
    const size_t sm = (size_t)np_max * nrho_max * sizeof(float);
    HR_TAPS(ntaps, {
        if (int e = set_smem((const void*)k_interp_columns<NT>, sm)) return e;
        if (ncols > 0)
            k_interp_columns<NT><<<ncols, 256, sm, (cudaStream_t)stream>>>(pieces, cmap, nrho_max, ntau_all, np_all, g);
    });
    return check_launch();
}

int launch_gather_samples(const PieceDev* pieces, const int4* smap, int nblocks, float* f, int np_all, int Nt_all,
                          int Nx_all, int ntaps, void* stream) {
    if (nblocks > 0)
        HR_TAPS(ntaps, (k_gather_samples<NT><<<nblocks, kSampleBlock, 0, (cudaStream_t)stream>>>(pieces, smap, f, np_all,
                                                                                                Nt_all, Nx_all)));
    return check_launch();
}

int launch_sample_table(const TableArgs& A, const double* cj, const double* wk, const int* jfirst,
                        SampleEnt* out) {
    const long total = (long)A.nj * A.Nx;
    k_sample_table<<<(unsigned)((total + 255) / 256), 256>>>(A, cj, wk, jfirst, out);
    return check_launch();
}

int launch_radon_table(const TableArgs& A, const double* qb2, RadonEnt* out) {
    const long total = (long)A.ncol * A.Ntau;
    k_radon_table<<<(unsigned)((total + 255) / 256), 256>>>(A, qb2, out);
    return check_launch();
}

int launch_zeta_gemm(const double* A, const double* Bre, const double* Bim, int n1, int nn, int n2,
                     double* Zre, double* Zim, void* stream) {
    dim3 bs(16, 16);
    dim3 gs((n2 + 15) / 16, (n1 + 15) / 16);
    k_zeta_gemm<<<gs, bs, 0, (cudaStream_t)stream>>>(A, Bre, Bim, n1, nn, n2, Zre, Zim);
    return check_launch();
}

int launch_direct_fwd(const float* f, float* g, int Nt, int Nx, int Ntau, int Nq, double dt,
                      double dx, double tau0, double dtau, double qmin, double dq, void* stream) {
    dim3 bs(256);
    dim3 gs((Ntau + 255) / 256, Nq);
    k_direct_fwd<<<gs, bs, 0, (cudaStream_t)stream>>>(
        f, g, Nt, Nx, Ntau, (float)(tau0 / dt), (float)(dtau / dt), (float)(qmin * dx / dt),
        (float)(dq * dx / dt), (float)(2.0 * dx));
    return check_launch();
}

int launch_direct_adj(const float* g, float* f, int Nt, int Nx, int Ntau, int Nq, double dt,
                      double dx, double tau0, double dtau, double qmin, double dq, void* stream) {
    dim3 bs(256);
    dim3 gs((Nt + 255) / 256, Nx);
    k_direct_adj<<<gs, bs, 0, (cudaStream_t)stream>>>(
        g, f, Nt, Nx, Ntau, Nq, (float)(tau0 / dt), (float)(dtau / dt), (float)(qmin * dx / dt),
        (float)(dq * dx / dt), (float)(2.0 * dx));
    return check_launch();
}

}  // namespace hr

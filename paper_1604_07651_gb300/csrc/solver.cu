// Sparse Radon inversion by iterative soft thresholding (Section 3, the
// iterations (iters) and (itersmd) after Daubechies, Defrise and De Mol) and
// the power iteration that bounds its step, on top of radon_fwd / radon_adj.
//
// The paper's iteration for min_g ||chi_S R_h* g - f||^2 + mu ||g||_1 is
//   g^n = S_{c^2 mu}( g^{n-1} + c^2 R_h (f - chi_S R_h* g^{n-1}) ),
// S_mu(v) = sign(v) max(|v| - mu/2, 0), c ||R_h|| < 1 -- the proximal gradient
// method of that objective with step c^2 / 2. With `accelerate` the gradient
// step is taken at the extrapolated point y^{n-1} instead of g^{n-1}
// (Beck and Teboulle's FISTA):
//   y^n = g^n + ((t_{n-1} - 1) / t_n) (g^n - g^{n-1}),
//   t_n = (1 + sqrt(1 + 4 t_{n-1}^2)) / 2,  t_0 = 1,  y^0 = g^0.
// Each iteration is radon_adj, one fused residual kernel, radon_fwd and one
// fused threshold/extrapolation kernel, all on the caller's stream; the host
// only computes the scalar momentum sequence.
//
// Multiple attenuation (Section 6, "Multiple attenuation"): primaries and
// multiples separate by moveout in the sparse Radon image; the part of the
// image beyond a border line in the (tau, q) plane (larger slowness: the
// multiples) is taken back to (t, x) with R_h* and subtracted from the
// gather.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>

#include "hradon.h"
#include "internal.h"

namespace hr {
namespace {

constexpr int kThreads = 256;
constexpr int kNormBlocks = 512;   // partial sums of the norm reduction

// r = f - mask[k] * a  (a = R_h* y), over [Nx][Nt]; mask NULL means all ones.
__global__ void __launch_bounds__(kThreads) k_residual(const float* __restrict__ f, const float* __restrict__ mask,
                                                      float* __restrict__ r, int Nt, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float m = mask ? __ldg(mask + i / Nt) : 1.f;
        r[i] = __ldg(f + i) - m * r[i];
    }
}

// g_new = S(y + c2 u), threshold c2 mu / 2; y <- g_new + beta (g_new - g);
// g <- g_new. With y == g (ISTA, beta = 0) the update is in place.
__global__ void __launch_bounds__(kThreads) k_threshold(float* g, float* y, const float* __restrict__ u,
                                                       float c2, float thr, float beta, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float v = y[i] + c2 * __ldg(u + i);
        const float a = fabsf(v) - thr;
        const float gn = a > 0.f ? copysignf(a, v) : 0.f;
        const float go = g[i];
        g[i] = gn;
        y[i] = gn + beta * (gn - go);
    }
}

// Partial sums of squares (FP64) over a grid-stride partition: block b
// writes part[b]. Fixed grid, fixed order: the sum is deterministic.
__global__ void __launch_bounds__(kThreads) k_sumsq_partial(const float* __restrict__ x, long n,
                                                           double* __restrict__ part) {
    __shared__ double red[kThreads / 32];
    double s = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double v = __ldg(x + i);
        s += v * v;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// Sum of the partials, in the same order in every block.
__device__ __forceinline__ double sum_partials(const double* __restrict__ part, int np) {
    __shared__ double tot;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < np; ++b) t += part[b];
        tot = t;
    }
    __syncthreads();
    return tot;
}

// y = x / ||x|| (||x|| from the partials); norm_out (if set) = ||x||.
__global__ void __launch_bounds__(kThreads) k_normalize(const float* __restrict__ x, float* __restrict__ y, long n,
                                                       const double* __restrict__ part, int np,
                                                       float* __restrict__ norm_out) {
    const double nrm = sqrt(sum_partials(part, np));
    const float inv = nrm > 0.0 ? (float)(1.0 / nrm) : 0.f;
    if (norm_out && blockIdx.x == 0 && threadIdx.x == 0) *norm_out = (float)nrm;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        y[i] = x[i] * inv;
}

// Zero g[l][i] on one side of the line q = q0 + slope * tau in the (tau, q)
// plane: side 0 zeroes q > q0 + slope tau (keeps the primaries), side 1
// zeroes q <= q0 + slope tau (keeps the multiples). src may alias dst.
__global__ void __launch_bounds__(kThreads) k_mute(const float* src, float* dst, int Ntau, long n, double tau0,
                                                  double dtau, double qmin, double dq, const double* qv,
                                                  double q0, double slope, int side) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const long l = i / Ntau;
        const double tau = tau0 + dtau * (double)(i - l * Ntau);
        const double q = qv ? qv[l] : qmin + dq * (double)l;
        const bool above = q > q0 + slope * tau;
        dst[i] = (above == (side == 0)) ? 0.f : src[i];
    }
}

// out = a - b, elementwise.
__global__ void __launch_bounds__(kThreads) k_subtract(const float* __restrict__ a, const float* __restrict__ b,
                                                      float* __restrict__ out, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        out[i] = __ldg(a + i) - __ldg(b + i);
}

int grid_for(long n) {
    const long b = (n + kThreads - 1) / kThreads;
    return (int)(b < 1184 ? (b > 0 ? b : 1) : 1184);   // 152 SMs x 8 resident blocks: grid-stride beyond
}

int last_cuda() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 0 : (int)e;
}

radon_status cuda_fail(int e, const char* what) {
    return (radon_status)set_error(RADON_ERR_CUDA, (std::string(what) + ": " + cudaGetErrorString((cudaError_t)e)).c_str());
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace
}  // namespace hr

using namespace hr;

extern "C" radon_status radon_ista_work_bytes(radon_plan p, size_t* bytes) {
    if (!p || !bytes) return (radon_status)set_error(RADON_ERR_INVALID_ARG, "NULL argument");
    radon_desc d;
    if (radon_status s = radon_plan_desc(p, &d)) return s;
    const size_t data = (size_t)d.Nt * d.Nx * sizeof(float), image = (size_t)d.Nq * d.Ntau * sizeof(float);
    *bytes = align256(data) + 2 * align256(image) + align256(kNormBlocks * sizeof(double));
    return RADON_OK;
}

extern "C" radon_status radon_ista(radon_plan p, const float* f, const float* mask, float* g, int iters,
                                   float c2, float mu, int accelerate, void* work, size_t work_bytes,
                                   void* stream) {
    if (!p) return (radon_status)set_error(RADON_ERR_INVALID_ARG, "plan is NULL");
    if (!f || !g || !work) return (radon_status)set_error(RADON_ERR_INVALID_ARG, "NULL data pointer");
    if (iters < 0 || !(c2 > 0.f) || !(mu >= 0.f) || !std::isfinite(c2) || !std::isfinite(mu))
        return (radon_status)set_error(RADON_ERR_INVALID_ARG, "iters >= 0, c2 > 0 and mu >= 0 (finite) required");
    size_t need = 0;
    radon_ista_work_bytes(p, &need);
    if (work_bytes < need || ((uintptr_t)work & 255))
        return (radon_status)set_error(RADON_ERR_INVALID_ARG, "work area too small or not 256-byte aligned");
    radon_desc d;
    radon_plan_desc(p, &d);
    const long nd = (long)d.Nt * d.Nx, ni = (long)d.Nq * d.Ntau;
    char* w = (char*)work;
    float* r = (float*)w;                                     // residual, [Nx][Nt]
    float* u = (float*)(w + align256(nd * sizeof(float)));    // R_h r, [Nq][Ntau]
    float* y = (float*)((char*)u + align256(ni * sizeof(float)));   // extrapolated point, [Nq][Ntau]
    cudaStream_t s = (cudaStream_t)stream;
    if (!accelerate) y = g;
    else if (cudaMemcpyAsync(y, g, ni * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return cuda_fail(last_cuda(), "copy of the initial iterate");
    const float thr = 0.5f * c2 * mu;
    double t = 1.0;
    for (int it = 0; it < iters; ++it) {
        if (radon_status st = radon_adj(p, y, r, stream)) return st;
        k_residual<<<grid_for(nd), kThreads, 0, s>>>(f, mask, r, d.Nt, nd);
        if (int e = last_cuda()) return cuda_fail(e, "residual");
        if (radon_status st = radon_fwd(p, r, u, stream)) return st;
        double beta = 0.0;
        if (accelerate) {
            const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
            beta = (t - 1.0) / tn;
            t = tn;
        }
        k_threshold<<<grid_for(ni), kThreads, 0, s>>>(g, y, u, c2, thr, (float)beta, ni);
        if (int e = last_cuda()) return cuda_fail(e, "threshold");
    }
    return RADON_OK;
}

extern "C" radon_status radon_opnorm_work_bytes(radon_plan p, size_t* bytes) {
    if (!p || !bytes) return (radon_status)set_error(RADON_ERR_INVALID_ARG, "NULL argument");
    radon_desc d;
    if (radon_status s = radon_plan_desc(p, &d)) return s;
    const size_t data = (size_t)d.Nt * d.Nx * sizeof(float), image = (size_t)d.Nq * d.Ntau * sizeof(float);
    *bytes = align256(data) + 2 * align256(image) + align256(kNormBlocks * sizeof(double));
    return RADON_OK;
}

extern "C" radon_status radon_opnorm(radon_plan p, const float* v0, int iters, float* norm2, void* work,
                                     size_t work_bytes, void* stream) {
    if (!p) return (radon_status)set_error(RADON_ERR_INVALID_ARG, "plan is NULL");
    if (!v0 || !norm2 || !work) return (radon_status)set_error(RADON_ERR_INVALID_ARG, "NULL data pointer");
    if (iters < 1) return (radon_status)set_error(RADON_ERR_INVALID_ARG, "iters >= 1 required");
    size_t need = 0;
    radon_opnorm_work_bytes(p, &need);
    if (work_bytes < need || ((uintptr_t)work & 255))
        return (radon_status)set_error(RADON_ERR_INVALID_ARG, "work area too small or not 256-byte aligned");
    radon_desc d;
    radon_plan_desc(p, &d);
    const long nd = (long)d.Nt * d.Nx, ni = (long)d.Nq * d.Ntau;
    char* w = (char*)work;
    float* a = (float*)w;                                                  // R_h* v, [Nx][Nt]
    float* v = (float*)(w + align256(nd * sizeof(float)));                 // unit vector, [Nq][Ntau]
    float* z = (float*)((char*)v + align256(ni * sizeof(float)));          // R_h R_h* v
    double* part = (double*)((char*)z + align256(ni * sizeof(float)));
    cudaStream_t s = (cudaStream_t)stream;
    k_sumsq_partial<<<kNormBlocks, kThreads, 0, s>>>(v0, ni, part);
    k_normalize<<<grid_for(ni), kThreads, 0, s>>>(v0, v, ni, part, kNormBlocks, nullptr);
    if (int e = last_cuda()) return cuda_fail(e, "power iteration start");
    for (int it = 0; it < iters; ++it) {
        if (radon_status st = radon_adj(p, v, a, stream)) return st;
        if (radon_status st = radon_fwd(p, a, z, stream)) return st;
        // ||R R* v|| with ||v|| = 1 tends to the largest eigenvalue of R R*, ||R_h||^2
        k_sumsq_partial<<<kNormBlocks, kThreads, 0, s>>>(z, ni, part);
        k_normalize<<<grid_for(ni), kThreads, 0, s>>>(z, v, ni, part, kNormBlocks, norm2);
        if (int e = last_cuda()) return cuda_fail(e, "power iteration");
    }
    return RADON_OK;
}

static double q_step(const radon_desc& d) { return d.Nq > 1 ? (d.qmax - d.qmin) / (d.Nq - 1) : 0.0; }

extern "C" radon_status radon_mute(radon_plan p, const float* g, float* out, double q0, double slope, int side,
                                   void* stream) {
    if (!p) return (radon_status)set_error(RADON_ERR_INVALID_ARG, "plan is NULL");
    if (!g || !out) return (radon_status)set_error(RADON_ERR_INVALID_ARG, "NULL data pointer");
    if (side != RADON_KEEP_BELOW && side != RADON_KEEP_ABOVE)
        return (radon_status)set_error(RADON_ERR_INVALID_ARG, "side must be RADON_KEEP_BELOW or RADON_KEEP_ABOVE");
    radon_desc d;
    radon_plan_desc(p, &d);
    const long ni = (long)d.Nq * d.Ntau;
    k_mute<<<grid_for(ni), kThreads, 0, (cudaStream_t)stream>>>(g, out, d.Ntau, ni, d.tau0, d.dtau, d.qmin, q_step(d),
                                                                 plan_q_values(p), q0, slope, side);
    if (int e = last_cuda()) return cuda_fail(e, "mute");
    return RADON_OK;
}

extern "C" radon_status radon_demultiple_work_bytes(radon_plan p, size_t* bytes) {
    if (radon_status s = radon_ista_work_bytes(p, bytes)) return s;
    radon_desc d;
    radon_plan_desc(p, &d);
    *bytes += align256((size_t)d.Nq * d.Ntau * sizeof(float)) + align256((size_t)d.Nt * d.Nx * sizeof(float));
    return RADON_OK;
}

extern "C" radon_status radon_demultiple(radon_plan p, const float* f, double q0, double slope, int iters,
                                         float c2, float mu, int accelerate, float* g, float* f_out, void* work,
                                         size_t work_bytes, void* stream) {
    if (!p) return (radon_status)set_error(RADON_ERR_INVALID_ARG, "plan is NULL");
    if (!f || !g || !f_out || !work) return (radon_status)set_error(RADON_ERR_INVALID_ARG, "NULL data pointer");
    size_t need = 0, ista_b = 0;
    radon_demultiple_work_bytes(p, &need);
    radon_ista_work_bytes(p, &ista_b);
    if (work_bytes < need || ((uintptr_t)work & 255))
        return (radon_status)set_error(RADON_ERR_INVALID_ARG, "work area too small or not 256-byte aligned");
    radon_desc d;
    radon_plan_desc(p, &d);
    const long nd = (long)d.Nt * d.Nx, ni = (long)d.Nq * d.Ntau;
    float* gm = (float*)((char*)work + ista_b);                                   // multiples' image
    float* fm = (float*)((char*)gm + align256((size_t)ni * sizeof(float)));       // multiples' gather
    if (radon_status st = radon_ista(p, f, nullptr, g, iters, c2, mu, accelerate, work, ista_b, stream)) return st;
    if (radon_status st = radon_mute(p, g, gm, q0, slope, RADON_KEEP_ABOVE, stream)) return st;
    if (radon_status st = radon_adj(p, gm, fm, stream)) return st;
    k_subtract<<<grid_for(nd), kThreads, 0, (cudaStream_t)stream>>>(f, fm, f_out, nd);
    if (int e = last_cuda()) return cuda_fail(e, "subtraction of the multiples");
    return RADON_OK;
}

// Host side of hradon: descriptor checks, the FP64 geometry of every
// sub-problem (Sections 2.1, 2.2 and 4 of the paper), the plan-time tables,
// the kernel spectra and the C ABI of include/hradon.h.
//
// Built with -ffp-contract=off so that the FP64 geometry rounds the same way
// on every host architecture.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "hradon.h"
#include "internal.h"

using namespace hr;

namespace {

thread_local std::string g_err;

radon_status fail(radon_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

// Allocation-failure hook for tests of the out-of-memory path: when the
// environment variable RADON_FAIL_ALLOC_AT holds n > 0 at the start of a
// plan or batch creation, the n-th device allocation of that creation fails
// as if cudaMalloc had run out of memory (counted over every thread of the
// creation; nothing is asked of the device). Unset, 0 or not a number: off.
std::atomic<long> g_alloc_countdown{0};

void arm_alloc_hook() {
    const char* v = std::getenv("RADON_FAIL_ALLOC_AT");
    long n = 0;
    if (v) {
        char* end = nullptr;
        n = std::strtol(v, &end, 10);
        if (end == v || n < 0) n = 0;
    }
    g_alloc_countdown.store(n);
}

// True when the hook makes this allocation fail.
bool alloc_hook_fails() {
    if (g_alloc_countdown.load(std::memory_order_relaxed) <= 0) return false;
    return g_alloc_countdown.fetch_sub(1) == 1;
}

// cudaMalloc behind the hook.
cudaError_t hooked_malloc(void** ptr, size_t bytes) {
    if (alloc_hook_fails()) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(ptr, bytes);
}

const double kPi = 3.14159265358979323846;
const double kTOverlap = 1.25;   // half-width ratio of the time-partition transition bands
const double kBetaMin = 1e-3;    // smallest angular opening of a sub-problem

// Smallest FFT length >= n of the form 2^a, 3 * 2^a, 5 * 2^a or 9 * 2^a
// (18 <= 9 * 2^a <= 2304, the range the FFT passes and the real-FFT half
// length handle).
int fft_size(int n) {
    long best = -1;
    for (long p = 1; p < 2L * n + 2; p *= 2) {
        for (long c : {p, 3 * p, 5 * p, (p >= 2 && p <= 256) ? 9 * p : 0})
            if (c >= n && (best < 0 || c < best)) best = c;
    }
    return (int)best;
}

// Pass schedule of an FFT pair by decimation in frequency / time
// (dif_plan): radices, strides and twiddle-table offsets.
FftPlan make_dif_fft_plan(int n) {
    FftPlan fp{};
    fp.n = n;
    int R[kMaxDifPasses], S[kMaxDifPasses];
    fp.nst = dif_plan(n, R, S);
    int ofs = 0;
    for (int p = 0; p < fp.nst && p < 8; ++p) {
        fp.rad[p] = R[p];
        fp.st[p] = S[p];
        fp.tw[p] = ofs;
        ofs += stage_table_len(S[p], R[p]);
    }
    return fp;
}

// Rising edge of the time partition at split b (raised cosine in log t).
double t_edge(double tb, double b, double r) {
    double u = std::log(std::max(tb, 1e-300) / b) / std::log(r);
    u = std::min(1.0, std::max(-1.0, u));
    return 0.5 * (1.0 + std::sin(0.5 * kPi * u));
}

// Accepted time split points (sorted, separated by the overlap bands).
std::vector<double> accepted_splits(const radon_desc& d) {
    std::vector<double> in(d.tsplit, d.tsplit + std::max(0, std::min(d.n_tsplit, RADON_MAX_TSPLIT)));
    std::sort(in.begin(), in.end());
    std::vector<double> bs;
    const double r = kTOverlap;
    for (double b : in) {
        if (!(b > 0.0 && b < 1.0)) continue;
        if (b * r >= 1.0) continue;
        if (!bs.empty() && b / r < bs.back() * r) continue;
        bs.push_back(b);
    }
    return bs;
}

struct TPiece { int lo, hi, idx; };

std::vector<TPiece> time_pieces(const radon_desc& d, const std::vector<double>& bs) {
    const double n = (double)(d.Nt - 1);
    const double r = kTOverlap;
    std::vector<TPiece> out;
    const int np = (int)bs.size() + 1;
    for (int p = 0; p < np; ++p) {
        int lo = p == 0 ? 0 : (int)std::ceil(bs[p - 1] / r * n - 1e-9);
        int hi = p == np - 1 ? d.Nt - 1 : (int)std::floor(bs[p] * r * n + 1e-9);
        out.push_back({lo, hi, p});
    }
    return out;
}

double t_window(const std::vector<double>& bs, int p, double tb) {
    const double r = kTOverlap;
    double lo = p == 0 ? 1.0 : t_edge(tb, bs[p - 1], r);
    double hi = p == (int)bs.size() ? 0.0 : t_edge(tb, bs[p], r);
    return lo - hi;
}

// Offsets of the gather and slownesses of the output: the descriptor's
// regular grids (empty vectors) or given lists (unequally spaced grids,
// Section 4); time and intercept time stay regular.
struct Grid {
    std::vector<double> x;   // [Nx] offsets, km, strictly increasing, x[0] >= 0
    std::vector<double> q;   // [Nq] slownesses, s/km, strictly increasing, q[0] >= 0
};

// X of the rescaling Eq. (12): the largest offset.
double offset_X(const radon_desc& d, const Grid& g) { return g.x.empty() ? (d.Nx - 1) * d.dx : g.x.back(); }

// Rescaled offsets x_k / X.
std::vector<double> offsets_bar(const radon_desc& d, const Grid& g) {
    std::vector<double> xb(d.Nx);
    const double n_x = d.Nx - 1;
    for (int k = 0; k < d.Nx; ++k) xb[k] = g.x.empty() ? k / n_x : g.x[k] / g.x.back();
    return xb;
}

// Rescaled offsets the lattice spacing of Eq. (18) is taken over: on given
// offsets, equally spaced ones over the same range [x_0, X] (the gridding
// treats the samples as a quadrature, so the lattice resolves the band of
// the data, which the mean spacing sets; the largest gap would coarsen it).
std::vector<double> spacing_offsets_bar(const radon_desc& d, const Grid& g) {
    if (g.x.empty()) return offsets_bar(d, g);
    std::vector<double> xb(d.Nx);
    const double X = g.x.back(), x0 = g.x[0];
    for (int k = 0; k < d.Nx; ++k) xb[k] = (x0 + k * ((X - x0) / (d.Nx - 1))) / X;
    return xb;
}

// Trapezoid weights of the offsets in units of 1/(Nx - 1) of the rescaled
// range: 1/2 at the ends and 1 inside on the regular grid.
std::vector<double> offset_weights(const radon_desc& d, const Grid& g) {
    std::vector<double> w(d.Nx);
    if (g.x.empty()) {
        for (int k = 0; k < d.Nx; ++k) w[k] = (k == 0 || k == d.Nx - 1) ? 0.5 : 1.0;
        return w;
    }
    const std::vector<double> xb = offsets_bar(d, g);
    const double n_x = d.Nx - 1;
    for (int k = 0; k < d.Nx; ++k) {
        const double lo = xb[k > 0 ? k - 1 : 0], hi = xb[k < d.Nx - 1 ? k + 1 : d.Nx - 1];
        w[k] = 0.5 * (hi - lo) * n_x;
    }
    return w;
}

std::vector<double> q_grid(const radon_desc& d, const Grid& g) {
    if (!g.q.empty()) return g.q;
    std::vector<double> q(d.Nq);
    if (d.Nq == 1) {
        q[0] = d.qmin;
        return q;
    }
    const double dq = (d.qmax - d.qmin) / (d.Nq - 1);
    for (int l = 0; l < d.Nq; ++l) q[l] = d.qmin + l * dq;
    return q;
}

std::vector<std::pair<int, int>> slowness_pieces(const radon_desc& d, const Grid& g) {
    const double T = (d.Nt - 1) * d.dt, X = offset_X(d, g);
    std::vector<double> q = q_grid(d, g);
    int n = std::max(1, d.n_qsplit);
    if (n == 1 || d.Nq < 2) return {{0, d.Nq - 1}};
    std::vector<double> psi(d.Nq);
    for (int l = 0; l < d.Nq; ++l) {
        double qb = q[l] * X / T;
        psi[l] = std::atan(qb * qb);
    }
    const double lo = psi[0], hi = psi[d.Nq - 1];
    std::vector<int> piece(d.Nq, 0);
    for (int p = 1; p < n; ++p) {
        double bnd = lo + (hi - lo) * p / n;
        for (int l = 0; l < d.Nq; ++l)
            if (psi[l] >= bnd) piece[l] += 1;
    }
    std::vector<std::pair<int, int>> out;
    for (int p = 0; p < n; ++p) {
        int a = -1, b = -1;
        for (int l = 0; l < d.Nq; ++l)
            if (piece[l] == p) {
                if (a < 0) a = l;
                b = l;
            }
        if (a >= 0) out.push_back({a, b});
    }
    return out;
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double pp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; ++j) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
    std::sort(x.begin(), x.end());
}

// Fourier transform of the centred B-spline of degree `order` (3 or 5) at
// frequency w in cycles per cell: sinc^(order + 1).
double bspline_symbol(double w, int order) {
    if (w == 0.0) return 1.0;
    const double s = std::sin(kPi * w) / (kPi * w);
    double r = 1.0;
    for (int i = 0; i <= order; ++i) r *= s;
    return r;
}

double b3(double x) {
    double ax = std::fabs(x);
    if (ax < 1.0) return 2.0 / 3.0 - ax * ax + 0.5 * ax * ax * ax;
    if (ax < 2.0) return (2.0 - ax) * (2.0 - ax) * (2.0 - ax) / 6.0;
    return 0.0;
}

// Centred quintic B-spline: truncated powers (3-|x|)^5 - 6 (2-|x|)^5 +
// 15 (1-|x|)^5 over 120, each term only where its base is positive.
double b5(double x) {
    const double a = std::fabs(x);
    auto tp = [](double u) { return u > 0 ? u * u * u * u * u : 0.0; };
    return (tp(3 - a) - 6 * tp(2 - a) + 15 * tp(1 - a)) / 120.0;
}

double bspline(double x, int order) { return order == 5 ? b5(x) : b3(x); }

// Taps per axis (order + 1) and guard cells per lattice side ((order + 1) / 2).
int spline_taps(int order) { return order + 1; }
int guard_cells(int order) { return (order + 1) / 2; }

// The kernels' float tap weights (4 or 6 taps) at fractional part f.
void spline_weights(int ntaps, float f, float* w) {
    if (ntaps == 6) bspline_weights<6>(f, w);
    else bspline_weights<4>(f, w);
}

}  // namespace

// ---------------------------------------------------------------------------

struct HostPiece {
    int tpiece = 0, jt_lo = 0, jt_hi = 0, l_lo = 0, l_hi = 0;
    double s0 = 0, s1 = 0, m_lo = 0, m_hi = 0, alpha = 0, beta = 0, a = 0, O1 = 0, O2 = 0;
    double c_min = 0, k2 = 0, a_r = 0, r_max = 0, dphi_rule = 0, deta_rule = 0;
    int n_theta = 0, n_rho = 0, Ntheta = 0, Nrho = 0, Ptheta = 0, Prho = 0, k1max = 0, k2max = 0;
    double dtheta = 0, drho = 0, theta0 = 0, rho0 = 0, theta_m = 0;
    std::vector<int> jfirst;
    int Rmax = 1;                                  // most rows per band shared memory allows
    int max_tile_chunks = 0;                       // most gridding chunks of one tile
    int order = 3;                                 // B-spline degree
    const int2* lband_R[kMaxBandRows + 1] = {};    // band column ranges for each rows-per-band
    PieceDev dev{};
};

// Rows per band of a piece: the band count and column ranges follow.
static void set_rows(HostPiece& h, int R) {
    h.dev.R = R;
    h.dev.nbands = (h.Ntheta + R - 1) / R;
    h.dev.lband = h.lband_R[R];
}

struct radon_plan_s {
    radon_desc d{};
    Grid grid;                                   // given offsets / slownesses (empty: regular)
    const double* q_dev = nullptr;               // [Nq] given slownesses on the device (mute)
    int device = 0;
    std::vector<HostPiece> pieces;               // slowness-piece major
    std::vector<std::pair<int, int>> qpieces;    // columns of each slowness piece
    std::vector<int> qfirst, qcount;             // pieces of each slowness piece
    PieceDev* dev_pieces = nullptr;
    float* lat_all = nullptr;                    // every piece's lattice, back to back
    size_t lat_bytes = 0;
    std::vector<PieceDev> host_devs;             // host copies of the descriptors (launch parameters)
    const int4* cmap = nullptr;                  // output columns: (first piece, count, l, 0)
    int ncols = 0;
    int col_pieces = 0;                          // largest count of cmap
    const int4* smap = nullptr;                  // sample blocks: (first piece, count, first sample, 0)
    int nsblocks = 0;
    int nrho_max = 0;
    std::vector<void*> allocs;
    size_t bytes = 0;
    // per-stage timing
    bool profiling = false;
    struct Rec { int stage; cudaEvent_t a, b; double bytes; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> event_pool;
    size_t pool_next = 0;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = cudaSetDevice(dev) == cudaSuccess;
        }
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

template <class T>
radon_status dev_upload(radon_plan_s* p, const std::vector<T>& v, const T** out) {
    void* ptr = nullptr;
    size_t bytes = std::max<size_t>(v.size(), 1) * sizeof(T);
    if (hooked_malloc(&ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(RADON_ERR_OOM, "cudaMalloc of a plan table failed");
    }
    p->allocs.push_back(ptr);
    p->bytes += bytes;
    if (!v.empty() && cudaMemcpy(ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(RADON_ERR_CUDA, "cudaMemcpy of a plan table failed");
    *out = (const T*)ptr;
    return RADON_OK;
}

radon_status dev_alloc(radon_plan_s* p, size_t bytes, void** out) {
    void* ptr = nullptr;
    if (hooked_malloc(&ptr, std::max<size_t>(bytes, 16)) != cudaSuccess) {
        cudaGetLastError();
        return fail(RADON_ERR_OOM, "cudaMalloc of a plan buffer failed");
    }
    p->allocs.push_back(ptr);
    p->bytes += bytes;
    *out = ptr;
    return RADON_OK;
}

radon_status check_desc(const radon_desc* d) {
    if (!d) return fail(RADON_ERR_INVALID_ARG, "descriptor is NULL");
    if (d->Nt < 2 || d->Nx < 2 || d->Ntau < 2 || d->Nq < 1)
        return fail(RADON_ERR_INVALID_ARG, "need Nt, Nx, Ntau >= 2 and Nq >= 1");
    if ((long)d->Nt * d->Nx > (1L << 30) || (long)d->Ntau * d->Nq > (1L << 30) || d->Nt > (1 << 20) ||
        d->Ntau > (1 << 20))
        return fail(RADON_ERR_UNSUPPORTED, "gather or image larger than 2^30 samples");
    if (!(d->dt > 0) || !(d->dx > 0) || !std::isfinite(d->dt) || !std::isfinite(d->dx))
        return fail(RADON_ERR_INVALID_ARG, "dt and dx must be positive and finite");
    if (!(d->qmin >= 0) || !(d->qmax >= d->qmin) || !std::isfinite(d->qmax))
        return fail(RADON_ERR_INVALID_ARG, "need 0 <= qmin <= qmax");
    if (d->Nq > 1 && !(d->qmax > d->qmin))
        return fail(RADON_ERR_INVALID_ARG, "need qmin < qmax when Nq > 1");
    if (d->Nq == 1 && !(d->qmin > 0) && !(d->qmax > 0))
        return fail(RADON_ERR_INVALID_ARG, "a single slowness column needs q > 0");
    if (!(d->tau0 >= 0) || !std::isfinite(d->tau0) || !(d->dtau >= 0) || !std::isfinite(d->dtau))
        return fail(RADON_ERR_INVALID_ARG, "need tau0 >= 0 and dtau >= 0");
    if (!(d->sigma > 0) || !(d->sigma <= 16))
        return fail(RADON_ERR_INVALID_ARG, "need 0 < sigma <= 16");
    if (!(d->omega_c > 0) || !(d->omega_c < 0.5))
        return fail(RADON_ERR_INVALID_ARG, "need 0 < omega_c < 0.5");
    if (d->n_tsplit < 0 || d->n_tsplit > RADON_MAX_TSPLIT)
        return fail(RADON_ERR_INVALID_ARG, "n_tsplit out of range");
    if (d->n_qsplit < 1 || d->n_qsplit > 64)
        return fail(RADON_ERR_INVALID_ARG, "need 1 <= n_qsplit <= 64");
    if (d->rows_per_band < 0 || d->rows_per_band > kMaxBandRows)
        return fail(RADON_ERR_INVALID_ARG, "need 0 <= rows_per_band <= 6");
    if (d->spline_order != 3 && d->spline_order != 5)
        return fail(RADON_ERR_INVALID_ARG, "spline_order must be 3 (cubic) or 5 (quintic)");
    return RADON_OK;
}

void map_T(const HostPiece& h, double s, double y, double& u1, double& u2) {
    const double ca = std::cos(h.alpha), sa = std::sin(h.alpha);
    const double ds = s - 0.5, dy = y - 0.5;
    u1 = h.a * (ca * ds - sa * dy) + h.O1;
    u2 = h.a * (sa * ds + ca * dy) + h.O2;
}

// Vertices of {(s,y) in [s0,s1]x[0,1] : s >= c + m y}.
std::vector<std::pair<double, double>> clip_region(double s0, double s1, double c, double m) {
    const double rect[4][2] = {{s0, 0.0}, {s1, 0.0}, {s1, 1.0}, {s0, 1.0}};
    std::vector<std::pair<double, double>> out;
    for (int i = 0; i < 4; ++i) {
        const double* p = rect[i];
        const double* r = rect[(i + 1) % 4];
        double vp = p[0] - c - m * p[1], vr = r[0] - c - m * r[1];
        if (vp >= 0) out.push_back({p[0], p[1]});
        if ((vp >= 0) != (vr >= 0)) {
            double t = vp / (vp - vr);
            out.push_back({p[0] + t * (r[0] - p[0]), p[1] + t * (r[1] - p[1])});
        }
    }
    return out;
}

// FP64 geometry of one sub-problem (same definitions as the paper's
// Sections 2.1, 2.2 and 4; readings documented with the descriptor).
radon_status make_geometry(const radon_desc& d, const Grid& g, const TPiece& tp, std::pair<int, int> lq,
                           HostPiece& h, std::vector<double>& phi_all) {
    const double n_t = d.Nt - 1;
    const double T = n_t * d.dt, X = offset_X(d, g);
    const std::vector<double> q = q_grid(d, g);
    const std::vector<double> xbar = offsets_bar(d, g);
    h.order = d.spline_order;
    h.tpiece = tp.idx;
    h.jt_lo = tp.lo;
    h.jt_hi = tp.hi;
    h.l_lo = lq.first;
    h.l_hi = lq.second;
    h.s0 = (tp.lo / n_t) * (tp.lo / n_t);
    h.s1 = (tp.hi / n_t) * (tp.hi / n_t);
    double qb_lo = q[lq.first] * X / T, qb_hi = q[lq.second] * X / T;
    h.m_lo = qb_lo * qb_lo;
    h.m_hi = qb_hi * qb_hi;
    double psi_lo = std::atan(h.m_lo), psi_hi = std::atan(h.m_hi);
    if (psi_hi - psi_lo < kBetaMin) {
        double mid = std::max(0.5 * (psi_lo + psi_hi), 0.5 * kBetaMin);
        psi_lo = mid - 0.5 * kBetaMin;
        psi_hi = mid + 0.5 * kBetaMin;
    }
    h.beta = psi_hi - psi_lo;
    h.alpha = 0.5 * (psi_hi + psi_lo);
    {
        const double s2a = std::sin(2 * h.alpha), sb = std::sin(h.beta), cb = std::cos(h.beta);
        h.a = sb / std::sqrt(s2a * sb + cb * (s2a + sb) + 1.0);
        const double th = std::tan(h.beta / 2);
        h.O1 = h.a * std::sin(h.alpha + kPi / 4) / (std::sqrt(2.0) * th);
        h.O2 = h.a * std::cos(h.alpha + kPi / 4) * th / std::sqrt(2.0);
    }
    // Mute with the smallest slowness of the whole problem.
    const double taub_min = d.tau0 / T;
    h.c_min = taub_min * taub_min;
    const double qb0 = q[0] * X / T;
    h.k2 = qb0 * qb0;
    h.jfirst.assign(d.Nx, tp.hi + 1);
    for (int k = 0; k < d.Nx; ++k) {
        const double xb = xbar[k];
        const double lim = h.c_min + h.k2 * (xb * xb);
        for (int j = tp.lo; j <= tp.hi; ++j) {
            const double tb = j / n_t;
            if (tb * tb >= lim) {
                h.jfirst[k] = j;
                break;
            }
        }
    }
    // Inner and outer radius over the data region.
    auto poly = clip_region(h.s0, h.s1, h.c_min, h.k2);
    if (poly.empty()) return fail(RADON_ERR_INVALID_ARG, "a time piece lies entirely in the muted region");
    double ar = 1e300, rmax = 0.0;
    for (double th : {-h.beta / 2, h.beta / 2})
        for (auto& v : poly) {
            double u1, u2;
            map_T(h, v.first, v.second, u1, u2);
            ar = std::min(ar, u1 * std::cos(th) + u2 * std::sin(th));
        }
    for (auto& v : poly) {
        double u1, u2;
        map_T(h, v.first, v.second, u1, u2);
        rmax = std::max(rmax, std::sqrt(u1 * u1 + u2 * u2));
    }
    if (!(ar > 0)) return fail(RADON_ERR_INVALID_ARG, "degenerate log-polar setup (inner radius <= 0)");
    h.a_r = ar;
    h.r_max = rmax;
    // Spacing of Eq. (18) over every sample of the time piece (given offsets:
    // over equally spaced offsets of the same range).
    const std::vector<double> xsp = spacing_offsets_bar(d, g);
    const int nj = tp.hi - tp.lo + 1;
    phi_all.assign((size_t)nj * d.Nx, 0.0);
    std::vector<double> eta_prev(nj), eta_cur(nj);
    double dphi = 0.0, deta = 0.0;
    for (int k = 0; k < d.Nx; ++k) {
        const double xb = xsp[k];
        const double y = xb * xb;
        double* ph = &phi_all[(size_t)k * nj];
        for (int jj = 0; jj < nj; ++jj) {
            const double tb = (tp.lo + jj) / n_t;
            double u1, u2;
            map_T(h, tb * tb, y, u1, u2);
            ph[jj] = std::atan2(u2, u1);
            eta_cur[jj] = 0.5 * std::log(u1 * u1 + u2 * u2);
            if (jj > 0) {
                dphi = std::max(dphi, std::fabs(ph[jj] - ph[jj - 1]));
                deta = std::max(deta, std::fabs(eta_cur[jj] - eta_cur[jj - 1]));
            }
            if (k > 0) {
                dphi = std::max(dphi, std::fabs(ph[jj] - phi_all[(size_t)(k - 1) * nj + jj]));
                deta = std::max(deta, std::fabs(eta_cur[jj] - eta_prev[jj]));
            }
        }
        std::swap(eta_prev, eta_cur);
    }
    if (!(dphi > 0) || !(deta > 0)) return fail(RADON_ERR_INVALID_ARG, "degenerate sample spacing");
    h.dphi_rule = dphi;
    h.deta_rule = deta;
    h.n_theta = std::max(1, (int)std::ceil(d.sigma * h.beta / dphi - 1e-9));
    const double L_rho = std::log(h.r_max) - std::log(h.a_r);
    h.n_rho = std::max(1, (int)std::ceil(d.sigma * L_rho / deta - 1e-9));
    h.dtheta = h.beta / h.n_theta;
    h.drho = L_rho / h.n_rho;
    const int guard = guard_cells(h.order);
    h.theta0 = -h.beta / 2 - guard * h.dtheta;
    h.rho0 = std::log(h.a_r) - guard * h.drho;
    h.Ntheta = h.n_theta + 2 * guard + 1;
    h.Nrho = h.n_rho + 2 * guard + 1;
    h.theta_m = std::min((h.Ntheta - 1) * h.dtheta, std::acos(std::exp(-(h.Nrho - 1) * h.drho)));
    const int Ka = (int)std::ceil(h.theta_m / h.dtheta - 1e-9);
    const int Kr = (int)std::ceil(-std::log(std::cos(h.theta_m)) / h.drho - 1e-9);
    h.Ptheta = fft_size(h.Ntheta + Ka);
    h.Prho = fft_size(h.Nrho + Kr);
    h.k1max = std::min((int)std::floor(d.omega_c * h.Ptheta), h.Ptheta / 2 - 1);
    h.k2max = std::min((int)std::floor(d.omega_c * h.Prho), h.Prho / 2 - 1);
    return RADON_OK;
}

// zeta_hat on the lattice's frequency grid (FP64 quadrature on the device),
// divided twice by the B-spline symbol and normalised for the kernels' FFT
// conventions; stored in the blocked layout [nkb][k1max+1][CB].
radon_status kernel_spectrum(radon_plan_s* p, const HostPiece& h, int CB, int nkb,
                             std::vector<cf>& Kout) {
    const int n1 = h.k1max + 1, n2 = h.k2max + 1;
    const double dw1 = 1.0 / (h.Ptheta * h.dtheta), dw2 = 1.0 / (h.Prho * h.drho);
    const double lc_m = std::log(std::cos(h.theta_m));
    const double cycles = h.k1max * dw1 * h.theta_m + h.k2max * dw2 * std::fabs(lc_m);
    const int npan = (int)std::ceil(cycles) + 4;
    std::vector<double> gx, gw;
    gauss_legendre(20, gx, gw);
    const int nn = npan * 20;
    std::vector<double> th(nn), wt(nn);
    for (int pn = 0; pn < npan; ++pn) {
        const double e0 = h.theta_m * pn / npan, e1 = h.theta_m * (pn + 1) / npan;
        const double hh = 0.5 * (e1 - e0), c = 0.5 * (e1 + e0);
        for (int i = 0; i < 20; ++i) {
            th[pn * 20 + i] = c + hh * gx[i];
            wt[pn * 20 + i] = hh * gw[i];
        }
    }
    std::vector<double> A((size_t)n1 * nn), Bre((size_t)nn * n2), Bim((size_t)nn * n2);
    for (int k1 = 0; k1 < n1; ++k1)
        for (int t = 0; t < nn; ++t) A[(size_t)k1 * nn + t] = std::cos(2 * kPi * th[t] * (k1 * dw1));
    for (int t = 0; t < nn; ++t) {
        const double ct = std::cos(th[t]);
        const double l = std::log(ct);
        const double base = wt[t] / ct;
        for (int k2 = 0; k2 < n2; ++k2) {
            const double ph = -2 * kPi * (k2 * dw2) * l;
            Bre[(size_t)t * n2 + k2] = base * std::cos(ph);
            Bim[(size_t)t * n2 + k2] = base * std::sin(ph);
        }
    }
    double *dA = nullptr, *dR = nullptr, *dI = nullptr, *dZr = nullptr, *dZi = nullptr;
    const size_t bA = A.size() * 8, bB = Bre.size() * 8, bZ = (size_t)n1 * n2 * 8;
    if (hooked_malloc((void**)&dA, bA) != cudaSuccess || hooked_malloc((void**)&dR, bB) != cudaSuccess ||
        hooked_malloc((void**)&dI, bB) != cudaSuccess || hooked_malloc((void**)&dZr, bZ) != cudaSuccess ||
        hooked_malloc((void**)&dZi, bZ) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dA); cudaFree(dR); cudaFree(dI); cudaFree(dZr); cudaFree(dZi);
        return fail(RADON_ERR_OOM, "cudaMalloc of the kernel-spectrum work arrays failed");
    }
    radon_status st = RADON_OK;
    std::vector<double> Zr((size_t)n1 * n2), Zi((size_t)n1 * n2);
    if (cudaMemcpy(dA, A.data(), bA, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dR, Bre.data(), bB, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dI, Bim.data(), bB, cudaMemcpyHostToDevice) != cudaSuccess) {
        st = fail(RADON_ERR_CUDA, "upload of the kernel-spectrum tables failed");
    } else if (int e = launch_zeta_gemm(dA, dR, dI, n1, nn, n2, dZr, dZi, nullptr)) {
        st = fail(RADON_ERR_CUDA, std::string("zeta quadrature launch failed: ") +
                                      cudaGetErrorString((cudaError_t)e));
    } else if (cudaMemcpy(Zr.data(), dZr, bZ, cudaMemcpyDeviceToHost) != cudaSuccess ||
               cudaMemcpy(Zi.data(), dZi, bZ, cudaMemcpyDeviceToHost) != cudaSuccess) {
        st = fail(RADON_ERR_CUDA, "zeta quadrature failed");
    }
    cudaFree(dA); cudaFree(dR); cudaFree(dI); cudaFree(dZr); cudaFree(dZi);
    if (st != RADON_OK) return st;
    (void)p;
    // Normalisation of the kernels' transforms: the row real FFT pair without
    // its 1/2 factors gives 2 Prho, the unnormalised column pair Ptheta.
    const double norm = 1.0 / (2.0 * h.Ptheta * h.Prho);
    Kout.assign((size_t)nkb * n1 * CB, cf{0.f, 0.f});
    for (int k1 = 0; k1 < n1; ++k1) {
        const double s1 = bspline_symbol((double)k1 / h.Ptheta, h.order);
        for (int k2 = 0; k2 < n2; ++k2) {
            const double s2 = bspline_symbol((double)k2 / h.Prho, h.order);
            const double den = (s1 * s2) * (s1 * s2);
            const double zr = 2.0 * Zr[(size_t)k1 * n2 + k2], zi = 2.0 * Zi[(size_t)k1 * n2 + k2];
            const int kb = k2 / CB, c = k2 % CB;
            Kout[((size_t)kb * n1 + k1) * CB + c] = {(float)(zr / den * norm), (float)(zi / den * norm)};
        }
    }
    return RADON_OK;
}

// Tile lists of the forward gridding, built from the device's own position
// table (copied back once) so that membership matches the kernel exactly:
// for every tile, the chunks of at most 8 consecutive samples of one trace
// whose NT x NT footprint meets it (along a trace the footprint moves
// monotonically, so each trace meets a tile in one run of samples).
radon_status build_tile_lists(radon_plan_s* p, HostPiece& h, PieceDev& P) {
    const int TR = kTileRows, TC = kTileCols;
    const int NT = P.ntaps;
    P.ntr = (h.Ntheta + TR - 1) / TR;
    P.ntc = (h.Nrho + TC - 1) / TC;
    const int ntiles = P.ntr * P.ntc;
    std::vector<SampleEnt> tab((size_t)P.nj * P.Nx);
    if (cudaMemcpy(tab.data(), P.stab, tab.size() * sizeof(SampleEnt), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(RADON_ERR_CUDA, "reading back the position table failed");
    std::vector<std::vector<int4>> runs(ntiles);
    std::vector<int> last_k(ntiles, -1), last_j(ntiles, -2);
    for (int k = 0; k < P.Nx; ++k) {
        for (int jl = 0; jl < P.nj; ++jl) {
            const SampleEnt& e = tab[(size_t)k * P.nj + jl];
            if (e.w == 0.f) continue;
            const int m0 = e.mn >> 16, n0 = e.mn & 0xffff;
            const int j = P.jt_lo + jl;
            for (int ti = m0 / TR; ti <= (m0 + NT - 1) / TR && ti < P.ntr; ++ti)
                for (int tj = n0 / TC; tj <= (n0 + NT - 1) / TC && tj < P.ntc; ++tj) {
                    const int t = ti * P.ntc + tj;
                    if (last_k[t] == k && last_j[t] == j - 1 && runs[t].back().z < 8) {
                        runs[t].back().z += 1;
                    } else {
                        runs[t].push_back(int4{k, j, 1, 0});
                    }
                    last_k[t] = k;
                    last_j[t] = j;
                }
        }
    }
    // work units: every tile's chunks cut into pieces of at most kUnitChunks
    // chunks, each with the exponent of the largest B-spline weight sum a
    // cell of the tile collects from the unit's samples (the fixed-point
    // bound of the kernel, computed with the kernel's own weights)
    std::vector<int4> flat, units;
    std::vector<long> uwork;
    std::vector<double> cell((size_t)TR * TC);
    for (int t = 0; t < ntiles; ++t) {
        const int base = (int)flat.size();
        const int m_lo = (t / P.ntc) * TR, n_lo = (t % P.ntc) * TC;
        flat.insert(flat.end(), runs[t].begin(), runs[t].end());
        for (int c = 0; c < (int)runs[t].size(); c += kUnitChunks) {
            const int e = std::min((int)runs[t].size(), c + kUnitChunks);
            long w = 0;
            std::fill(cell.begin(), cell.end(), 0.0);
            for (int q = c; q < e; ++q) {
                const int4 ch = runs[t][q];
                w += ch.z;
                for (int sidx = 0; sidx < ch.z; ++sidx) {
                    const SampleEnt& se = tab[(size_t)ch.x * P.nj + (ch.y - P.jt_lo) + sidx];
                    float wt[6], wr[6];
                    spline_weights(NT, se.ft, wt);
                    spline_weights(NT, se.fr, wr);
                    const int m0 = (se.mn >> 16) - m_lo, n0 = (se.mn & 0xffff) - n_lo;
                    for (int a = 0; a < NT; ++a)
                        for (int b = 0; b < NT; ++b) {
                            const int m = m0 + a, n = n0 + b;
                            if (m >= 0 && m < TR && n >= 0 && n < TC) cell[(size_t)m * TC + n] += (double)wt[a] * wr[b];
                        }
                }
            }
            const double cmax = *std::max_element(cell.begin(), cell.end());
            units.push_back(int4{t, base + c, base + e, 28 - std::ilogb(cmax > 0 ? cmax : 1.0)});
            uwork.push_back(w);
        }
    }
    // tiles cut into several units: one partial-tile slot per unit (in chunk
    // order) and one arrival counter per tile; the last unit to finish sums
    // the slots in slot order, so the lattice does not depend on the order in
    // which units run
    for (int t = 0; t < ntiles; ++t) h.max_tile_chunks = std::max(h.max_tile_chunks, (int)runs[t].size());
    std::vector<int> nper(ntiles, 0), slot0(ntiles, 0), cidx(ntiles, -1), seen(ntiles, 0);
    for (const int4& u : units) nper[u.x]++;
    int nslots = 0, ncount = 0;
    for (int t = 0; t < ntiles; ++t)
        if (nper[t] > 1) {
            slot0[t] = nslots;
            nslots += nper[t];
            cidx[t] = ncount++;
        }
    std::vector<int4> uslot(units.size());
    for (size_t i = 0; i < units.size(); ++i) {
        const int t = units[i].x;
        uslot[i] = nper[t] > 1 ? int4{slot0[t], nper[t], seen[t]++, cidx[t]} : int4{0, 1, 0, -1};
    }
    std::vector<int> order(units.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return uwork[x] > uwork[y]; });
    std::vector<int4> sorted(units.size()), sorted_slot(units.size());
    for (size_t i = 0; i < order.size(); ++i) {
        sorted[i] = units[order[i]];
        sorted_slot[i] = uslot[order[i]];
    }
    P.nunits = (int)sorted.size();
    P.nslots = nslots;
    P.ncount = ncount;
    radon_status s = RADON_OK;
    if ((s = dev_upload(p, flat, &P.chunks)) || (s = dev_upload(p, sorted, &P.units)) ||
        (s = dev_upload(p, sorted_slot, &P.uslot)))
        return s;
    void* slots = nullptr;
    if ((s = dev_alloc(p, (size_t)std::max(nslots, 1) * TR * TC * sizeof(float), &slots))) return s;
    P.slots = (float*)slots;
    return RADON_OK;
}

radon_status build_piece_tables(radon_plan_s* p, HostPiece& h, const std::vector<double>& bs,
                                const std::vector<double>& phi_all, int smem_max) {
    const radon_desc& d = p->d;
    const double n_t = d.Nt - 1, n_x = d.Nx - 1;
    const double T = n_t * d.dt, X = offset_X(d, p->grid);
    PieceDev& P = h.dev;
    P.Ntheta = h.Ntheta;
    P.Nrho = h.Nrho;
    P.ntaps = spline_taps(h.order);
    P.Ptheta = h.Ptheta;
    P.Prho = h.Prho;
    P.k1max = h.k1max;
    P.k2max = h.k2max;
    // FFT lengths the in-place passes handle: 2^a <= 4096,
    // 3 * 2^a <= 6144, 5 * 2^a <= 5120, 9 * 2^a <= 2304
    auto fft_ok = [](int n) {
        int R[kMaxDifPasses], S[kMaxDifPasses];
        return ((n % 3 == 0) ? n <= 6144 : (n % 5 == 0) ? n <= 5120 : n <= 4096) && dif_plan(n, R, S) > 0;
    };
    if (!fft_ok(h.Prho / 2) || !fft_ok(h.Ptheta))
        return fail(RADON_ERR_UNSUPPORTED,
                    "FFT length " + std::to_string(std::max(h.Prho / 2, h.Ptheta)) +
                        " above the FFT passes' limit (4096, 6144 = 3*2048 or 5120 = 5*1024)");
    // rows per band: any value up to what shared memory allows gives the same
    // results; the descriptor's choice, else 3 until the plan times them
    // (the row kernels pad each row of their band by one complex element)
    const int Rmax = (int)std::min<size_t>(kMaxBandRows, (size_t)smem_max / ((h.Prho + 2) * sizeof(float)));
    if (Rmax < 1) return fail(RADON_ERR_UNSUPPORTED, "row FFT length too large for shared memory");
    h.Rmax = Rmax;
    const int R = std::min(Rmax, d.rows_per_band > 0 ? d.rows_per_band : 3);
    const int CB = 2;   // spectrum columns per column block (the column kernel holds both)
    // the column kernel holds the column block, its slice of K and the twiddle tables
    const size_t col_smem = ((size_t)h.Ptheta + h.k1max + 1) * 2 * sizeof(cf) +
                            (size_t)((fft_dif_tables(h.Ptheta, nullptr) + 2) & ~1) * sizeof(cf);
    if (col_smem > (size_t)smem_max)
        return fail(RADON_ERR_UNSUPPORTED, "column FFT length too large for shared memory");
    P.R = R;
    P.CB = CB;
    P.nkb = (h.k2max + 1 + CB - 1) / CB;
    P.nbands = (h.Ntheta + R - 1) / R;
    P.Nt = d.Nt;
    P.Nx = d.Nx;
    P.jt_lo = h.jt_lo;
    P.jt_hi = h.jt_hi;
    P.nj = h.jt_hi - h.jt_lo + 1;
    P.Ntau = d.Ntau;
    P.l_lo = h.l_lo;
    P.l_hi = h.l_hi;
    P.fftM = make_dif_fft_plan(h.Prho / 2);
    P.fftT = make_dif_fft_plan(h.Ptheta);

    // per-time weight (window, 2 a^2 tb, quadrature and B-spline normalisation)
    // and trapezoid weights in x, both FP64 for the position-table kernel
    std::vector<double> cj(P.nj), wk(d.Nx);
    for (int jl = 0; jl < P.nj; ++jl) {
        const double tb = (h.jt_lo + jl) / n_t;
        const double w = t_window(bs, h.tpiece, tb);
        cj[jl] = w * 2.0 * h.a * h.a * tb / (n_t * n_x * h.dtheta * h.drho);
    }
    wk = offset_weights(d, p->grid);
    // output columns: theta taps, scale, e^rho polynomial; band column ranges
    const std::vector<double> q = q_grid(d, p->grid);
    const int ncol = h.l_hi - h.l_lo + 1;
    const int NT = P.ntaps;
    std::vector<float4> colw(ncol);
    std::vector<float2> colw2(NT > 4 ? ncol : 0);
    std::vector<int> colm0(ncol);
    std::vector<float> colscale(ncol);
    std::vector<double> qb2(ncol);
    const double dtau = d.dtau > 0 ? d.dtau : T / (d.Ntau - 1);
    for (int lc = 0; lc < ncol; ++lc) {
        const double qb = q[h.l_lo + lc] * X / T;
        const double m = qb * qb;
        const double psi = std::atan(m);
        const double theta = h.alpha - psi;
        const double xth = (theta - h.theta0) / h.dtheta;
        const double fl = std::floor(xth);
        int m0 = (int)fl - (NT / 2 - 1);              // first tap: floor - (order - 1) / 2
        m0 = std::min(std::max(m0, 0), h.Ntheta - NT);
        double w[6];
        for (int a = 0; a < NT; ++a) w[a] = bspline(xth - (m0 + a), h.order);
        colm0[lc] = m0;
        colw[lc] = make_float4((float)w[0], (float)w[1], (float)w[2], (float)w[3]);
        if (NT > 4) colw2[lc] = make_float2((float)w[4], (float)w[5]);
        colscale[lc] = (float)(2.0 * X * std::cos(psi) / h.a);
        qb2[lc] = m;
    }
    // candidate output columns of every band of rb rows: those whose NT
    // theta taps m0 .. m0+NT-1 meet the band
    for (int rb = 1; rb <= Rmax; ++rb) {
        const int nbands = (h.Ntheta + rb - 1) / rb;
        std::vector<int2> lband(nbands, int2{1, 0});
        for (int lc = 0; lc < ncol; ++lc) {
            const int m0 = colm0[lc];                        // >= 0
            const int first = (m0 + rb) / rb - 1;             // ceil((m0 + 1) / rb) - 1
            const int last = std::min(nbands - 1, (m0 + NT - 1) / rb);
            for (int b = first; b <= last; ++b) {
                int2& r = lband[b];
                const int l = h.l_lo + lc;
                if (r.x > r.y) r = int2{l, l};
                else {
                    r.x = std::min(r.x, l);
                    r.y = std::max(r.y, l);
                }
            }
        }
        if (radon_status s = dev_upload(p, lband, &h.lband_R[rb])) return s;
    }
    set_rows(h, R);
    // twiddles
    const int M = h.Prho / 2;
    std::vector<cf> twM(fft_dif_tables(M, nullptr) + 1), twP(M + 1), twT((fft_dif_tables(h.Ptheta, nullptr) + 2) & ~1);
    fft_dif_tables(M, twM.data());
    fft_dif_tables(h.Ptheta, twT.data());
    std::vector<int> rpos(M);
    {
        int R[kMaxDifPasses], S[kMaxDifPasses];
        const int s = dif_plan(M, R, S);
        for (int k = 0; k < M; ++k) rpos[k] = dif_pos(s, R, S, k);
    }
    P.twT_len = (int)twT.size();
    for (int k = 0; k <= M; ++k)
        twP[k] = {(float)std::cos(-2 * kPi * k / h.Prho), (float)std::sin(-2 * kPi * k / h.Prho)};
    std::vector<cf> K;
    if (radon_status s = kernel_spectrum(p, h, CB, P.nkb, K)) return s;

    radon_status s = RADON_OK;
    if (NT > 4 && (s = dev_upload(p, colw2, &P.colw2))) return s;
    if ((s = dev_upload(p, colw, &P.colw)) || (s = dev_upload(p, colm0, &P.colm0)) ||
        (s = dev_upload(p, colscale, &P.colscale)) || (s = dev_upload(p, K, &P.K)) ||
        (s = dev_upload(p, twM, &P.twM)) || (s = dev_upload(p, twP, &P.twP)) || (s = dev_upload(p, rpos, &P.rpos)) ||
        (s = dev_upload(p, twT, &P.twT)))
        return s;
    // position tables, FP64 on the device
    TableArgs A;
    A.a = h.a;
    A.ca = std::cos(h.alpha);
    A.sa = std::sin(h.alpha);
    A.O1 = h.O1;
    A.O2 = h.O2;
    A.alpha = h.alpha;
    A.theta0 = h.theta0;
    A.dtheta = h.dtheta;
    A.rho0 = h.rho0;
    A.drho = h.drho;
    A.a_r = h.a_r;
    A.r_max = h.r_max;
    A.n_t = n_t;
    A.T = T;
    A.tau0 = d.tau0;
    A.dtau = dtau;
    A.jt_lo = h.jt_lo;
    A.nj = P.nj;
    A.Nx = d.Nx;
    A.Ntheta = h.Ntheta;
    A.Nrho = h.Nrho;
    A.Ntau = d.Ntau;
    A.ncol = ncol;
    A.ntaps = NT;
    const double *dcj = nullptr, *dwk = nullptr, *dqb2 = nullptr, *dxb = nullptr;
    const int* djf = nullptr;
    void* tab = nullptr;
    if ((s = dev_upload(p, cj, &dcj)) || (s = dev_upload(p, wk, &dwk)) ||
        (s = dev_upload(p, h.jfirst, &djf)) || (s = dev_upload(p, qb2, &dqb2)) ||
        (s = dev_upload(p, offsets_bar(d, p->grid), &dxb)))
        return s;
    A.xb = dxb;
    if ((s = dev_alloc(p, (size_t)P.nj * d.Nx * sizeof(SampleEnt), &tab))) return s;
    P.stab = (const SampleEnt*)tab;
    if (int e = launch_sample_table(A, dcj, dwk, djf, (SampleEnt*)tab))
        return fail(RADON_ERR_CUDA, std::string("position table: ") + cudaGetErrorString((cudaError_t)e));
    if ((s = build_tile_lists(p, h, P))) return s;
    if ((s = dev_alloc(p, (size_t)ncol * d.Ntau * sizeof(RadonEnt), &tab))) return s;
    P.rtab = (const RadonEnt*)tab;
    if (int e = launch_radon_table(A, dqb2, (RadonEnt*)tab))
        return fail(RADON_ERR_CUDA, std::string("position table: ") + cudaGetErrorString((cudaError_t)e));
    // fixed-point bound of the adjoint column profiles: per column, the
    // exponent of the largest total weight scale * wr one of its rho cells
    // collects from the column's outputs (the kernel's own float weights)
    {
        std::vector<RadonEnt> rt((size_t)ncol * d.Ntau);
        if (cudaMemcpy(rt.data(), tab, rt.size() * sizeof(RadonEnt), cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(RADON_ERR_CUDA, "reading back the output position table failed");
        std::vector<double> prof(h.Nrho);
        std::vector<int> colsh(ncol);
        std::vector<int2> rrange(ncol);
        for (int lc = 0; lc < ncol; ++lc) {
            std::fill(prof.begin(), prof.end(), 0.0);
            rrange[lc] = int2{d.Ntau, -1};
            for (int i = 0; i < d.Ntau; ++i) {
                const RadonEnt e = rt[(size_t)lc * d.Ntau + i];
                if (e.n0 < 0) continue;
                rrange[lc].x = std::min(rrange[lc].x, i);
                rrange[lc].y = std::max(rrange[lc].y, i);
                float wr[6];
                spline_weights(NT, e.fr, wr);
                for (int c = 0; c < NT; ++c) prof[e.n0 + c] += (double)colscale[lc] * wr[c];
            }
            const double cmax = *std::max_element(prof.begin(), prof.end());
            colsh[lc] = 28 - std::ilogb(cmax > 0 ? cmax : 1.0);
        }
        if ((s = dev_upload(p, colsh, &P.colsh)) || (s = dev_upload(p, rrange, &P.rrange))) return s;
    }
    P.hpitch = (h.Nrho + 3) & ~3;
    return RADON_OK;
}

size_t round256b(size_t v) { return (v + 255) & ~(size_t)255; }
// The lattice of a piece followed by the arrival counters of its split
// gridding tiles (cleared together before every forward gridding).
size_t piece_lattice_bytes(const PieceDev& P) {
    return round256b((size_t)P.Ntheta * P.Nrho * sizeof(float) + (size_t)P.ncount * sizeof(int));
}
size_t piece_slot_bytes(const PieceDev& P) { return round256b((size_t)P.nslots * kTileRows * kTileCols * sizeof(float)); }
size_t piece_spectrum_bytes(const PieceDev& P) { return round256b((size_t)P.nkb * P.CB * P.Ntheta * sizeof(cf)); }
size_t piece_profile_bytes(const PieceDev& P) {
    return round256b((size_t)(P.l_hi - P.l_lo + 1) * P.hpitch * sizeof(float));
}

// Output columns of a plan for the interpolation kernel: every column of
// every slowness piece with the range of its time pieces (piece indices
// offset by `base`, the plan's first piece in a larger descriptor array).
void column_map(const radon_plan_s* p, int base, std::vector<int4>& out) {
    for (size_t qi = 0; qi < p->qpieces.size(); ++qi)
        for (int l = p->qpieces[qi].first; l <= p->qpieces[qi].second; ++l)
            out.push_back(int4{base + p->qfirst[qi], p->qcount[qi], l, 0});
}

// Sample blocks of a plan's gather for the adjoint gather kernel.
void sample_map(const radon_plan_s* p, int base, int, std::vector<int4>& out) {
    const long n = (long)p->d.Nt * p->d.Nx;
    for (long b = 0; b < n; b += kSampleBlock)
        out.push_back(int4{base, (int)p->pieces.size(), (int)b, 0});
}

void destroy_plan(radon_plan_s* p) {
    if (!p) return;
    for (void* a : p->allocs) cudaFree(a);
    for (cudaEvent_t e : p->event_pool) cudaEventDestroy(e);
    delete p;
}

cudaEvent_t pool_event(radon_plan_s* p) {
    if (p->pool_next == p->event_pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        p->event_pool.push_back(e);
    }
    return p->event_pool[p->pool_next++];
}

// Runs one launch, bracketed by events when profiling is on.
template <class F>
int timed(radon_plan_s* p, int stage, double bytes, void* stream, F&& launch) {
    if (!p->profiling) return launch();
    cudaEvent_t a = pool_event(p), b = pool_event(p);
    if (!a || !b) return launch();
    cudaEventRecord(a, (cudaStream_t)stream);
    int e = launch();
    cudaEventRecord(b, (cudaStream_t)stream);
    p->recs.push_back({stage, a, b, bytes});
    return e;
}

// Algorithmic bytes of each stage of one sub-problem.
double bytes_spectrum(const PieceDev& P) { return 8.0 * P.Ntheta * (P.k2max + 1); }
double bytes_lattice(const PieceDev& P) { return 4.0 * P.Ntheta * P.Nrho; }
double bytes_samples(const PieceDev& P) { return 4.0 * P.Nx * (P.jt_hi - P.jt_lo + 1); }
double bytes_kernel(const PieceDev& P) { return 8.0 * (P.k1max + 1) * (P.k2max + 1); }

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" radon_status radon_desc_init(radon_desc* d, int Nt, int Nx, int Ntau, int Nq, double dt,
                                        double dx, double qmin, double qmax) {
    if (!d) return fail(RADON_ERR_INVALID_ARG, "descriptor is NULL");
    std::memset(d, 0, sizeof(*d));
    d->Nt = Nt;
    d->Nx = Nx;
    d->Ntau = Ntau;
    d->Nq = Nq;
    d->dt = dt;
    d->dx = dx;
    d->qmin = qmin;
    d->qmax = qmax;
    d->tau0 = 0.0;
    d->dtau = 0.0;
    d->sigma = 1.1;
    d->omega_c = 0.4;
    d->n_tsplit = 2;
    d->tsplit[0] = 0.25;
    d->tsplit[1] = 0.5;
    d->n_qsplit = 1;
    d->device = -1;
    d->rows_per_band = 3;
    d->spline_order = 3;
    return RADON_OK;
}

extern "C" radon_status radon_plan_create(radon_plan* out, int Nt, int Nx, int Ntau, int Nq, double dt,
                                          double dx, double qmax) {
    radon_desc d;
    radon_desc_init(&d, Nt, Nx, Ntau, Nq, dt, dx, 0.0, qmax);
    return radon_plan_create_ex(out, &d);
}

// Geometry, tables and kernel spectra of every piece of a plan; no work
// buffers and no gather maps (a single plan and a batch lay those out
// differently).
// Given offsets / slownesses (NULL: the regular grid): finite, strictly
// increasing, non-negative; copied into g.
static radon_status check_grid(const radon_desc& d, const double* x, const double* q, Grid& g) {
    g = Grid{};
    if (x) {
        if (d.Nx < 2) return fail(RADON_ERR_INVALID_ARG, "given offsets need Nx >= 2");
        for (int k = 0; k < d.Nx; ++k)
            if (!std::isfinite(x[k]) || (k == 0 ? !(x[0] >= 0) : !(x[k] > x[k - 1])))
                return fail(RADON_ERR_INVALID_ARG, "offsets must be finite, >= 0 and strictly increasing");
        g.x.assign(x, x + d.Nx);
    }
    if (q) {
        for (int l = 0; l < d.Nq; ++l)
            if (!std::isfinite(q[l]) || (l == 0 ? !(q[0] >= 0) : !(q[l] > q[l - 1])))
                return fail(RADON_ERR_INVALID_ARG, "slownesses must be finite, >= 0 and strictly increasing");
        if (d.Nq == 1 && !(q[0] > 0)) return fail(RADON_ERR_INVALID_ARG, "a single slowness must be > 0");
        g.q.assign(q, q + d.Nq);
    }
    return RADON_OK;
}

static radon_status plan_core(const radon_desc* din, const double* x, const double* q, radon_plan_s** out) {
    *out = nullptr;
    if (radon_status s = check_desc(din)) return s;
    Grid grid;
    if (radon_status s = check_grid(*din, x, q, grid)) return s;
    radon_plan_s* p = new (std::nothrow) radon_plan_s();
    if (!p) return fail(RADON_ERR_OOM, "host allocation failed");
    p->d = *din;
    p->grid = std::move(grid);
    radon_desc& d = p->d;
    if (!p->grid.q.empty()) {            // the descriptor reports the given range
        d.qmin = p->grid.q.front();
        d.qmax = p->grid.q.back();
    }
    if (d.dtau <= 0) d.dtau = (d.Nt - 1) * d.dt / (d.Ntau - 1);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        delete p;
        return fail(RADON_ERR_CUDA, "no CUDA device");
    }
    if (d.device < 0) {
        cudaGetDevice(&p->device);
        d.device = p->device;
    } else if (d.device >= ndev) {
        delete p;
        return fail(RADON_ERR_INVALID_ARG, "device ordinal out of range");
    } else {
        p->device = d.device;
    }
    DeviceGuard guard(p->device);
    const int smem_max = max_smem_optin();
    const std::vector<double> bs = accepted_splits(d);
    const std::vector<TPiece> tps = time_pieces(d, bs);
    p->qpieces = slowness_pieces(d, p->grid);
    std::vector<double> phi_all;
    for (auto& lq : p->qpieces) {
        p->qfirst.push_back((int)p->pieces.size());
        for (auto& tp : tps) {
            HostPiece h;
            radon_status s = make_geometry(d, p->grid, tp, lq, h, phi_all);
            if (s == RADON_OK) s = build_piece_tables(p, h, bs, phi_all, smem_max);
            if (s != RADON_OK) {
                destroy_plan(p);
                return s;
            }
            p->pieces.push_back(std::move(h));
        }
        p->qcount.push_back((int)tps.size());
    }
    for (auto& h : p->pieces) p->nrho_max = std::max(p->nrho_max, h.dev.Nrho);
    if (!p->grid.q.empty()) {
        if (radon_status s = dev_upload(p, p->grid.q, &p->q_dev)) {
            destroy_plan(p);
            return s;
        }
    }
    *out = p;
    return RADON_OK;
}

// Rows-per-band tuner: every feasible value is timed on the plan's own
// (cleared) work buffers with the three row-FFT kernels, and the fastest
// kept. The value changes the work split only, not the results.
template <class Run>
static int tune_rows(int rmax, Run&& run, void* stream) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int best = 0;
    float best_ms = 0.f;
    for (int R = 1; R <= rmax; ++R) {
        if (run(R) != 0) break;                     // warm-up (shared-memory attributes, caches)
        cudaEventRecord(a, (cudaStream_t)stream);
        for (int rep = 0; rep < 3; ++rep)
            if (run(R) != 0) break;
        cudaEventRecord(b, (cudaStream_t)stream);
        if (cudaEventSynchronize(b) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (best == 0 || ms < best_ms) {
            best = R;
            best_ms = ms;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaGetLastError();
    return best;
}

extern "C" radon_status radon_plan_create_ex(radon_plan* out, const radon_desc* din) {
    return radon_plan_create_grid(out, din, nullptr, nullptr);
}

extern "C" radon_status radon_plan_create_grid(radon_plan* out, const radon_desc* din, const double* x,
                                               const double* q) {
    if (!out) return fail(RADON_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    arm_alloc_hook();
    radon_plan_s* p = nullptr;
    if (radon_status s = plan_core(din, x, q, &p)) return s;
    DeviceGuard guard(p->device);
    // per-piece work buffers: lattices back to back (one clear per forward),
    // spectra (the column pass works in place), adjoint column profiles
    size_t lat_b = 0, spec_b = 0, prof_b = 0;
    for (auto& h : p->pieces) {
        lat_b += piece_lattice_bytes(h.dev);
        spec_b += piece_spectrum_bytes(h.dev);
        prof_b += piece_profile_bytes(h.dev);
    }
    void *lat = nullptr, *spec = nullptr, *prof = nullptr;
    radon_status s = RADON_OK;
    if ((s = dev_alloc(p, lat_b, &lat)) || (s = dev_alloc(p, spec_b, &spec)) || (s = dev_alloc(p, prof_b, &prof))) {
        destroy_plan(p);
        return s;
    }
    p->lat_all = (float*)lat;
    p->lat_bytes = lat_b;
    void* const spec_base = spec;
    void* const prof_base = prof;
    for (auto& h : p->pieces) {
        h.dev.lat = (float*)lat;
        h.dev.spec = (cf*)spec;
        h.dev.prof = (float*)prof;
        lat = (char*)lat + piece_lattice_bytes(h.dev);
        spec = (char*)spec + piece_spectrum_bytes(h.dev);
        prof = (char*)prof + piece_profile_bytes(h.dev);
    }
    if (p->d.rows_per_band == 0) {
        int rmax = kMaxBandRows;
        for (auto& h : p->pieces) rmax = std::min(rmax, h.Rmax);
        cudaMemset(p->lat_all, 0, lat_b);
        cudaMemset(spec_base, 0, spec_b);
        cudaMemset(prof_base, 0, prof_b);
        const int np = (int)p->pieces.size();
        const int best = tune_rows(
            rmax,
            [&](int R) {
                std::vector<PieceDev> P;
                for (auto& h : p->pieces) {
                    set_rows(h, R);
                    P.push_back(h.dev);
                }
                for (int i = 0; i < np; i += kMaxBatch) {
                    const int n = std::min(kMaxBatch, np - i);
                    if (int e = launch_rows_r2c(P.data() + i, n, nullptr)) return e;
                    if (int e = launch_band_rows(P.data() + i, n, nullptr)) return e;
                    if (int e = launch_rows_c2r(P.data() + i, n, nullptr)) return e;
                }
                return 0;
            },
            nullptr);
        const int R = best > 0 ? best : std::min(3, rmax);
        for (auto& h : p->pieces) set_rows(h, R);
        p->d.rows_per_band = R;
    }
    std::vector<PieceDev> devs;
    for (auto& h : p->pieces) devs.push_back(h.dev);
    p->host_devs = devs;
    const PieceDev* dp = nullptr;
    if ((s = dev_upload(p, devs, &dp))) { destroy_plan(p); return s; }
    p->dev_pieces = const_cast<PieceDev*>(dp);
    // column and sample maps of the two gathers
    std::vector<int4> cmap, smap;
    column_map(p, 0, cmap);
    sample_map(p, 0, 0, smap);
    if ((s = dev_upload(p, cmap, &p->cmap)) || (s = dev_upload(p, smap, &p->smap))) {
        destroy_plan(p);
        return s;
    }
    p->ncols = (int)cmap.size();
    for (const int4& c : cmap) p->col_pieces = std::max(p->col_pieces, c.y);
    p->nsblocks = (int)smap.size();
    // the output interpolation holds one rho profile per time piece of a column
    if ((size_t)p->col_pieces * p->nrho_max * sizeof(float) > interp_smem_limit(spline_taps(p->d.spline_order))) {
        destroy_plan(p);
        return fail(RADON_ERR_UNSUPPORTED, "too many time pieces for the lattice length along rho "
                                           "(the output interpolation's profiles exceed shared memory)");
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        destroy_plan(p);
        return fail(RADON_ERR_CUDA, "plan creation failed on the device");
    }
    *out = p;
    return RADON_OK;
}

extern "C" radon_status radon_plan_destroy(radon_plan p) {
    if (!p) return RADON_OK;
    DeviceGuard guard(p->device);
    cudaDeviceSynchronize();
    destroy_plan(p);
    return RADON_OK;
}

static radon_status cuda_status(int e, const char* what) {
    if (e == 0) return RADON_OK;
    return fail(RADON_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString((cudaError_t)e));
}

// The forward chain over the pieces `P` (host copies; `dP` the same on the
// device), lattices in [lat, lat + lat_bytes). Every stage is one launch per
// group of at most kMaxBatch pieces; the output interpolation is one launch
// over every output column.
static radon_status run_forward(radon_plan_s* p, const PieceDev* P, const PieceDev* dP, float* lat,
                                size_t lat_bytes, const float* f, float* g, void* stream) {
    const int np = (int)p->pieces.size();
    double b_samp = 0, b_lat = 0, b_spec = 0, b_ker = 0;
    for (int i = 0; i < np; ++i) {
        b_samp += bytes_samples(P[i]);
        b_lat += bytes_lattice(P[i]);
        b_spec += bytes_spectrum(P[i]);
        b_ker += bytes_kernel(P[i]);
    }
    auto groups = [&](auto&& launch) {
        for (int i = 0; i < np; i += kMaxBatch)
            if (int e = launch(P + i, std::min(kMaxBatch, np - i))) return e;
        return 0;
    };
    if (radon_status s = cuda_status(
            timed(p, 0, b_samp + b_lat, stream,
                  [&] {
                      if (cudaError_t e = cudaMemsetAsync(lat, 0, lat_bytes, (cudaStream_t)stream)) return (int)e;
                      return groups([&](const PieceDev* q, int n) { return launch_grid_tiles(q, n, f, stream); });
                  }),
            "gridding"))
        return s;
    if (radon_status s = cuda_status(
            timed(p, 1, b_lat + b_spec, stream,
                  [&] { return groups([&](const PieceDev* q, int n) { return launch_rows_r2c(q, n, stream); }); }),
            "row FFT"))
        return s;
    if (radon_status s = cuda_status(
            timed(p, 2, 2 * b_spec + b_ker, stream,
                  [&] { return groups([&](const PieceDev* q, int n) { return launch_colconv(q, n, 0, stream); }); }),
            "convolution"))
        return s;
    if (radon_status s = cuda_status(
            timed(p, 3, b_spec + b_lat, stream,
                  [&] { return groups([&](const PieceDev* q, int n) { return launch_rows_c2r(q, n, stream); }); }),
            "inverse row FFT"))
        return s;
    const double gb = 4.0 * p->d.Ntau * p->d.Nq;
    if (radon_status s = cuda_status(
            timed(p, 4, b_lat + gb, stream,
                  [&] { return launch_interp_columns(dP, p->cmap, p->ncols, p->nrho_max, p->col_pieces, p->d.Ntau,
                                               p->qpieces.size() == 1 ? np : 0, spline_taps(p->d.spline_order), g,
                                               stream); }),
            "interpolation"))
        return s;
    return RADON_OK;
}

static const std::vector<PieceDev>& host_pieces(const radon_plan_s* p) { return p->host_devs; }

extern "C" radon_status radon_fwd(radon_plan p, const float* f, float* g, void* stream) {
    if (!p) return fail(RADON_ERR_INVALID_ARG, "plan is NULL");
    if (!f || !g) return fail(RADON_ERR_INVALID_ARG, "NULL data pointer");
    DeviceGuard guard(p->device);
    const std::vector<PieceDev>& P = host_pieces(p);
    return run_forward(p, P.data(), p->dev_pieces, p->lat_all, p->lat_bytes, f, g, stream);
}

extern "C" radon_status radon_adj(radon_plan p, const float* g, float* f, void* stream) {
    if (!p) return fail(RADON_ERR_INVALID_ARG, "plan is NULL");
    if (!f || !g) return fail(RADON_ERR_INVALID_ARG, "NULL data pointer");
    DeviceGuard guard(p->device);
    const std::vector<PieceDev>& P = host_pieces(p);
    const int np = (int)P.size();
    // the image is read once: every output column's CTA serves all its pieces
    const double b_g = 4.0 * p->d.Ntau * p->d.Nq;
    double b_lat = 0, b_spec = 0, b_ker = 0, b_h = 0;
    for (const PieceDev& q : P) {
        b_lat += bytes_lattice(q);
        b_spec += bytes_spectrum(q);
        b_ker += bytes_kernel(q);
        b_h += 4.0 * (q.l_hi - q.l_lo + 1) * q.Nrho;
    }
    auto groups = [&](auto&& launch) {
        for (int i = 0; i < np; i += kMaxBatch)
            if (int e = launch(P.data() + i, std::min(kMaxBatch, np - i))) return e;
        return 0;
    };
    if (radon_status s = cuda_status(
            timed(p, 9, b_g + b_h, stream,
                  [&] {
                      return launch_col_profiles_cols(p->dev_pieces, p->cmap, p->ncols, p->nrho_max, p->col_pieces,
                                                      p->d.Ntau, p->qpieces.size() == 1 ? np : 0,
                                                      spline_taps(p->d.spline_order), g, stream);
                  }),
            "adjoint interpolation (profiles)"))
        return s;
    if (radon_status s = cuda_status(
            timed(p, 5, b_h + b_spec, stream,
                  [&] { return groups([&](const PieceDev* q, int n) { return launch_band_rows(q, n, stream); }); }),
            "adjoint interpolation (bands)"))
        return s;
    if (radon_status s = cuda_status(
            timed(p, 6, 2 * b_spec + b_ker, stream,
                  [&] { return groups([&](const PieceDev* q, int n) { return launch_colconv(q, n, 1, stream); }); }),
            "adjoint convolution"))
        return s;
    if (radon_status s = cuda_status(
            timed(p, 7, b_spec + b_lat, stream,
                  [&] { return groups([&](const PieceDev* q, int n) { return launch_rows_c2r(q, n, stream); }); }),
            "inverse row FFT"))
        return s;
    return cuda_status(timed(p, 8, b_lat + 4.0 * p->d.Nt * p->d.Nx, stream,
                             [&] {
                                 return launch_gather_samples(p->dev_pieces, p->smap, p->nsblocks, f, np, p->d.Nt,
                                                              p->d.Nx, spline_taps(p->d.spline_order), stream);
                             }),
                       "adjoint gridding");
}

extern "C" radon_status radon_plan_num_pieces(radon_plan p, int* n) {
    if (!p || !n) return fail(RADON_ERR_INVALID_ARG, "NULL argument");
    *n = (int)p->pieces.size();
    return RADON_OK;
}

static void fill_info(const HostPiece& h, radon_piece_info* info) {
    info->jt_lo = h.jt_lo;
    info->jt_hi = h.jt_hi;
    info->l_lo = h.l_lo;
    info->l_hi = h.l_hi;
    info->alpha = h.alpha;
    info->beta = h.beta;
    info->a = h.a;
    info->O1 = h.O1;
    info->O2 = h.O2;
    info->a_r = h.a_r;
    info->r_max = h.r_max;
    info->dphi_rule = h.dphi_rule;
    info->deta_rule = h.deta_rule;
    info->dtheta = h.dtheta;
    info->drho = h.drho;
    info->theta0 = h.theta0;
    info->rho0 = h.rho0;
    info->Ntheta = h.Ntheta;
    info->Nrho = h.Nrho;
    info->Ptheta = h.Ptheta;
    info->Prho = h.Prho;
    info->k1max = h.k1max;
    info->k2max = h.k2max;
    info->theta_m = h.theta_m;
    info->grid_tiles = h.dev.ntr * h.dev.ntc;
    info->grid_units = h.dev.nunits;
    info->grid_split_tiles = h.dev.ncount;
    info->grid_max_tile_chunks = h.max_tile_chunks;
}

extern "C" radon_status radon_plan_piece_info(radon_plan p, int piece, radon_piece_info* info) {
    if (!p || !info) return fail(RADON_ERR_INVALID_ARG, "NULL argument");
    if (piece < 0 || piece >= (int)p->pieces.size()) return fail(RADON_ERR_INVALID_ARG, "piece out of range");
    fill_info(p->pieces[piece], info);
    return RADON_OK;
}

extern "C" radon_status radon_plan_piece_lattice(radon_plan p, int piece, float* out, size_t count) {
    if (!p || !out) return fail(RADON_ERR_INVALID_ARG, "NULL argument");
    if (piece < 0 || piece >= (int)p->pieces.size()) return fail(RADON_ERR_INVALID_ARG, "piece out of range");
    const PieceDev& P = p->pieces[piece].dev;
    const size_t n = (size_t)P.Ntheta * P.Nrho;
    if (count < n)
        return fail(RADON_ERR_INVALID_ARG,
                    "out holds " + std::to_string(count) + " floats, the lattice has " + std::to_string(n));
    DeviceGuard guard(p->device);
    if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(out, P.lat, n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(RADON_ERR_CUDA, std::string("lattice copy failed: ") + cudaGetErrorString(cudaGetLastError()));
    return RADON_OK;
}

extern "C" radon_status radon_plan_piece_samples(radon_plan p, int piece, double* theta, double* rho, float* weight,
                                                 size_t count) {
    if (!p) return fail(RADON_ERR_INVALID_ARG, "plan is NULL");
    if (piece < 0 || piece >= (int)p->pieces.size()) return fail(RADON_ERR_INVALID_ARG, "piece out of range");
    const PieceDev& P = p->pieces[piece].dev;
    const size_t n = (size_t)P.nj * P.Nx;
    if (count < n)
        return fail(RADON_ERR_INVALID_ARG,
                    "the outputs hold " + std::to_string(count) + " entries, the piece has " + std::to_string(n));
    std::vector<SampleEnt> tab(n);
    DeviceGuard guard(p->device);
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(tab.data(), P.stab, n * sizeof(SampleEnt), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(RADON_ERR_CUDA, std::string("table copy failed: ") + cudaGetErrorString(cudaGetLastError()));
    const int back = P.ntaps / 2 - 1;       // first tap = floor(position) - back
    for (size_t e = 0; e < n; ++e) {
        if (theta) theta[e] = (double)((tab[e].mn >> 16) + back) + (double)tab[e].ft;
        if (rho) rho[e] = (double)((tab[e].mn & 0xffff) + back) + (double)tab[e].fr;
        if (weight) weight[e] = tab[e].w;
    }
    return RADON_OK;
}

extern "C" radon_status radon_geometry(const radon_desc* din, int* npieces, radon_piece_info* infos,
                                       int max_infos) {
    return radon_geometry_grid(din, nullptr, nullptr, npieces, infos, max_infos);
}

extern "C" radon_status radon_geometry_grid(const radon_desc* din, const double* x, const double* q,
                                            int* npieces, radon_piece_info* infos, int max_infos) {
    if (!npieces) return fail(RADON_ERR_INVALID_ARG, "npieces is NULL");
    if (radon_status s = check_desc(din)) return s;
    Grid g;
    if (radon_status s = check_grid(*din, x, q, g)) return s;
    radon_desc d = *din;
    if (d.dtau <= 0) d.dtau = (d.Nt - 1) * d.dt / (d.Ntau - 1);
    const std::vector<double> bs = accepted_splits(d);
    const std::vector<TPiece> tps = time_pieces(d, bs);
    std::vector<double> phi_all;
    int n = 0;
    for (auto& lq : slowness_pieces(d, g))
        for (auto& tp : tps) {
            HostPiece h;
            if (radon_status s = make_geometry(d, g, tp, lq, h, phi_all)) return s;
            if (infos && n < max_infos) fill_info(h, infos + n);
            ++n;
        }
    *npieces = n;
    return RADON_OK;
}

const double* plan_q_values(const radon_plan_s* p) { return p ? p->q_dev : nullptr; }

extern "C" radon_status radon_plan_desc(radon_plan p, radon_desc* d) {
    if (!p || !d) return fail(RADON_ERR_INVALID_ARG, "NULL argument");
    *d = p->d;
    return RADON_OK;
}

extern "C" radon_status radon_plan_device_bytes(radon_plan p, size_t* bytes) {
    if (!p || !bytes) return fail(RADON_ERR_INVALID_ARG, "NULL argument");
    *bytes = p->bytes;
    return RADON_OK;
}

static radon_status check_direct(const void* a, const void* b, int Nt, int Nx, int Ntau, int Nq, double dt,
                                 double dx, double tau0, double dtau) {
    if (!a || !b) return fail(RADON_ERR_INVALID_ARG, "NULL data pointer");
    if (Nt < 2 || Nx < 2 || Ntau < 1 || Nq < 1) return fail(RADON_ERR_INVALID_ARG, "bad sizes");
    if (!(dt > 0) || !(dx > 0) || !(dtau > 0) || !(tau0 >= 0))
        return fail(RADON_ERR_INVALID_ARG, "need dt, dx, dtau > 0 and tau0 >= 0");
    if (Nq > 65535 || Nx > 65535) return fail(RADON_ERR_UNSUPPORTED, "Nq and Nx must be below 65536");
    return RADON_OK;
}

extern "C" radon_status radon_direct_fwd(const float* f, float* g, int Nt, int Nx, int Ntau, int Nq,
                                         double dt, double dx, double tau0, double dtau, double qmin,
                                         double dq, void* stream) {
    if (radon_status s = check_direct(f, g, Nt, Nx, Ntau, Nq, dt, dx, tau0, dtau)) return s;
    return cuda_status(launch_direct_fwd(f, g, Nt, Nx, Ntau, Nq, dt, dx, tau0, dtau, qmin, dq, stream),
                       "direct summation");
}

extern "C" radon_status radon_direct_adj(const float* g, float* f, int Nt, int Nx, int Ntau, int Nq,
                                         double dt, double dx, double tau0, double dtau, double qmin,
                                         double dq, void* stream) {
    if (radon_status s = check_direct(g, f, Nt, Nx, Ntau, Nq, dt, dx, tau0, dtau)) return s;
    return cuda_status(launch_direct_adj(g, f, Nt, Nx, Ntau, Nq, dt, dx, tau0, dtau, qmin, dq, stream),
                       "direct summation adjoint");
}

extern "C" radon_status radon_plan_set_profiling(radon_plan p, int enable) {
    if (!p) return fail(RADON_ERR_INVALID_ARG, "plan is NULL");
    p->profiling = enable != 0;
    return RADON_OK;
}

extern "C" radon_status radon_plan_profile_read(radon_plan p, double ms[RADON_NSTAGES],
                                                long long launches[RADON_NSTAGES],
                                                double bytes[RADON_NSTAGES]) {
    if (!p) return fail(RADON_ERR_INVALID_ARG, "plan is NULL");
    DeviceGuard guard(p->device);
    double t[RADON_NSTAGES] = {0}, b[RADON_NSTAGES] = {0};
    long long n[RADON_NSTAGES] = {0};
    radon_status st = RADON_OK;
    for (auto& r : p->recs) {
        float v = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&v, r.a, r.b) != cudaSuccess) {
            st = fail(RADON_ERR_CUDA, "reading a profiling event failed");
            continue;
        }
        t[r.stage] += v;
        b[r.stage] += r.bytes;
        n[r.stage] += 1;
    }
    p->recs.clear();
    p->pool_next = 0;
    for (int i = 0; i < RADON_NSTAGES; ++i) {
        if (ms) ms[i] = t[i];
        if (launches) launches[i] = n[i];
        if (bytes) bytes[i] = b[i];
    }
    return st;
}

extern "C" const char* radon_last_error(void) { return g_err.c_str(); }

extern "C" const char* radon_version(void) { return "hradon 0.1 (sm_103a)"; }

// ---------------------------------------------------------------------------
// Batches of gathers of different sizes: every stage one launch over all
// sub-problems of all gathers, descriptors and block maps in device memory.
// ---------------------------------------------------------------------------
struct radon_batch_s {
    int device = 0;
    std::vector<radon_plan_s*> plans;
    radon_plan_s* store = nullptr;             // owns the batch's own device allocations
    std::vector<long long> f_off, g_off;       // n + 1 prefix offsets (elements)
    const PieceDev* pieces = nullptr;          // every piece of every gather
    const int2 *map_units = nullptr, *map_bands = nullptr, *map_kb = nullptr;
    int n_units = 0, n_bands = 0, n_kb = 0;
    const int4* cmap = nullptr;
    const int4* smap = nullptr;
    int ncols = 0, nsblocks = 0, col_pieces = 0;
    size_t smem_rows = 0, smem_cols = 0;
    int nrho_max = 0;
    int ntaps = 4;                             // B-spline taps per axis of every gather
    bool col_x256 = false;                     // every piece takes the compile-time column pass
    float* lat_all = nullptr;
    size_t lat_bytes = 0;
};

static void destroy_batch(radon_batch_s* b) {
    if (!b) return;
    for (radon_plan_s* p : b->plans)
        if (p) destroy_plan(p);
    destroy_plan(b->store);
    delete b;
}

extern "C" radon_status radon_batch_create(radon_batch* out, int n, const radon_desc* descs) {
    return radon_batch_create_grid(out, n, descs, nullptr, nullptr);
}

extern "C" radon_status radon_batch_create_grid(radon_batch* out, int n, const radon_desc* descs,
                                                const double* const* x, const double* const* q) {
    if (!out) return fail(RADON_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || !descs) return fail(RADON_ERR_INVALID_ARG, "a batch needs n >= 1 descriptors");
    for (int i = 1; i < n; ++i)
        if (descs[i].spline_order != descs[0].spline_order)
            return fail(RADON_ERR_UNSUPPORTED, "the gathers of a batch must share the B-spline order");
    arm_alloc_hook();
    radon_batch_s* b = new (std::nothrow) radon_batch_s();
    if (!b) return fail(RADON_ERR_OOM, "host allocation failed");
    b->store = new (std::nothrow) radon_plan_s();
    if (!b->store) {
        delete b;
        return fail(RADON_ERR_OOM, "host allocation failed");
    }
    // every gather on the first descriptor's device (the calling thread's
    // current device when it names none)
    b->device = descs[0].device;
    if (b->device < 0 && cudaGetDevice(&b->device) != cudaSuccess) {
        destroy_batch(b);
        return fail(RADON_ERR_CUDA, "no CUDA device");
    }
    // the plans are independent: build them on several host threads (their
    // host-side table work dominates), keeping the first failure
    b->plans.assign(n, nullptr);
    std::atomic<int> next{0};
    std::mutex err_mutex;
    radon_status first_err = RADON_OK;
    std::string first_msg;
    auto worker = [&]() {
        for (int i = next++; i < n; i = next++) {
            radon_desc d = descs[i];
            d.device = b->device;
            radon_plan_s* p = nullptr;
            if (radon_status s = plan_core(&d, x ? x[i] : nullptr, q ? q[i] : nullptr, &p)) {
                std::lock_guard<std::mutex> lock(err_mutex);
                if (first_err == RADON_OK) {
                    first_err = s;
                    first_msg = "gather " + std::to_string(i) + ": " + g_err;
                }
                next = n;
                return;
            }
            b->plans[i] = p;
        }
    };
    const int nthreads = std::max(1, std::min<int>(n, std::min(16u, std::max(1u, std::thread::hardware_concurrency()))));
    std::vector<std::thread> pool;
    for (int t = 1; t < nthreads; ++t) pool.emplace_back(worker);
    worker();
    for (auto& t : pool) t.join();
    if (first_err != RADON_OK) {
        destroy_batch(b);
        return fail(first_err, first_msg);
    }
    b->ntaps = spline_taps(descs[0].spline_order);
    b->f_off.push_back(0);
    b->g_off.push_back(0);
    for (radon_plan_s* p : b->plans) {
        b->f_off.push_back(b->f_off.back() + (long long)p->d.Nt * p->d.Nx);
        b->g_off.push_back(b->g_off.back() + (long long)p->d.Ntau * p->d.Nq);
    }
    DeviceGuard guard(b->device);
    b->store->device = b->device;
    // work buffers of every piece, lattices back to back (one clear per forward)
    std::vector<PieceDev> host;
    for (int i = 0; i < n; ++i)
        for (auto& h : b->plans[i]->pieces) {
            PieceDev P = h.dev;
            P.f_off = b->f_off[i];
            P.g_off = b->g_off[i];
            host.push_back(P);
        }
    size_t lat_b = 0, spec_b = 0, prof_b = 0;
    for (auto& P : host) {
        lat_b += piece_lattice_bytes(P);
        spec_b += piece_spectrum_bytes(P);
        prof_b += piece_profile_bytes(P);
    }
    void *lat = nullptr, *spec = nullptr, *prof = nullptr;
    radon_status s = RADON_OK;
    if ((s = dev_alloc(b->store, lat_b, &lat)) || (s = dev_alloc(b->store, spec_b, &spec)) ||
        (s = dev_alloc(b->store, prof_b, &prof))) {
        destroy_batch(b);
        return s;
    }
    b->lat_all = (float*)lat;
    b->lat_bytes = lat_b;
    void* const spec_base = spec;
    void* const prof_base = prof;
    for (auto& P : host) {
        P.lat = (float*)lat;
        P.spec = (cf*)spec;
        P.prof = (float*)prof;
        lat = (char*)lat + piece_lattice_bytes(P);
        spec = (char*)spec + piece_spectrum_bytes(P);
        prof = (char*)prof + piece_profile_bytes(P);
        b->smem_rows = std::max(b->smem_rows, rows_smem_bytes(P));
        b->smem_cols = std::max(b->smem_cols, colconv_smem_bytes(P));
        b->nrho_max = std::max(b->nrho_max, P.Nrho);
    }
    b->col_x256 = colconv_all_x256(host.data(), (int)host.size());
    // block maps of the stage launches and the maps of the two gathers
    std::vector<int2> mu, mb, mk;
    for (int gi = 0; gi < (int)host.size(); ++gi) {
        const PieceDev& P = host[gi];
        for (int u = 0; u < P.nunits; ++u) mu.push_back(int2{gi, u});
        for (int u = 0; u < P.nbands; ++u) mb.push_back(int2{gi, u});
        for (int u = 0; u < P.nkb; ++u) mk.push_back(int2{gi, u});
    }
    std::vector<int4> cmap, smap;
    int base = 0;
    for (radon_plan_s* p : b->plans) {
        column_map(p, base, cmap);
        sample_map(p, base, 0, smap);
        base += (int)p->pieces.size();
    }
    if ((s = dev_upload(b->store, host, &b->pieces)) || (s = dev_upload(b->store, mu, &b->map_units)) ||
        (s = dev_upload(b->store, mb, &b->map_bands)) || (s = dev_upload(b->store, mk, &b->map_kb)) ||
        (s = dev_upload(b->store, cmap, &b->cmap)) ||
        (s = dev_upload(b->store, smap, &b->smap))) {
        destroy_batch(b);
        return s;
    }
    b->n_units = (int)mu.size();
    b->n_bands = (int)mb.size();
    b->n_kb = (int)mk.size();
    b->ncols = (int)cmap.size();
    for (const int4& c : cmap) b->col_pieces = std::max(b->col_pieces, c.y);
    b->nsblocks = (int)smap.size();
    if ((size_t)b->col_pieces * b->nrho_max * sizeof(float) > interp_smem_limit(b->ntaps)) {
        destroy_batch(b);
        return fail(RADON_ERR_UNSUPPORTED, "too many time pieces for the lattice length along rho "
                                           "(the output interpolation's profiles exceed shared memory)");
    }
    // rows per band tuned over the whole batch when every descriptor asks
    bool tune = true;
    int rmax = kMaxBandRows;
    for (int i = 0; i < n; ++i) tune = tune && descs[i].rows_per_band == 0;
    for (radon_plan_s* p : b->plans)
        for (auto& h : p->pieces) rmax = std::min(rmax, h.Rmax);
    if (tune) {
        cudaMemset(b->lat_all, 0, b->lat_bytes);
        cudaMemset(spec_base, 0, spec_b);
        cudaMemset(prof_base, 0, prof_b);
        // descriptors and band map for R rows per band (new device copies)
        auto apply = [&](int R) -> radon_status {
            int gi = 0;
            mb.clear();
            b->smem_rows = 0;
            for (radon_plan_s* p : b->plans)
                for (auto& h : p->pieces) {
                    set_rows(h, R);
                    host[gi].R = h.dev.R;
                    host[gi].nbands = h.dev.nbands;
                    host[gi].lband = h.dev.lband;
                    // the row kernels' shared memory grows with R
                    b->smem_rows = std::max(b->smem_rows, rows_smem_bytes(host[gi]));
                    for (int u = 0; u < host[gi].nbands; ++u) mb.push_back(int2{gi, u});
                    ++gi;
                }
            radon_status st = RADON_OK;
            if ((st = dev_upload(b->store, host, &b->pieces)) || (st = dev_upload(b->store, mb, &b->map_bands)))
                return st;
            b->n_bands = (int)mb.size();
            return RADON_OK;
        };
        radon_status st = RADON_OK;
        const int best = tune_rows(
            rmax,
            [&](int R) {
                if ((st = apply(R))) return 1;
                const DevBatch Bd{b->pieces, b->map_bands};
                if (int e = launch_rows_r2c_dev(Bd, b->n_bands, b->smem_rows, nullptr)) return e;
                if (int e = launch_band_rows_dev(Bd, b->n_bands, b->ntaps, b->smem_rows, nullptr)) return e;
                if (int e = launch_rows_c2r_dev(Bd, b->n_bands, b->smem_rows, nullptr)) return e;
                return 0;
            },
            nullptr);
        if (st || (st = apply(best > 0 ? best : std::min(3, rmax)))) {
            destroy_batch(b);
            return st;
        }
        for (radon_plan_s* p : b->plans) p->d.rows_per_band = host.empty() ? 3 : host[0].R;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        destroy_batch(b);
        return fail(RADON_ERR_CUDA, "batch creation failed on the device");
    }
    *out = b;
    return RADON_OK;
}

extern "C" radon_status radon_batch_destroy(radon_batch b) {
    if (!b) return RADON_OK;
    DeviceGuard guard(b->device);
    cudaDeviceSynchronize();
    destroy_batch(b);
    return RADON_OK;
}

extern "C" radon_status radon_batch_layout(radon_batch b, int* n, long long* f_offsets, long long* g_offsets) {
    if (!b) return fail(RADON_ERR_INVALID_ARG, "batch is NULL");
    if (n) *n = (int)b->plans.size();
    for (size_t i = 0; i < b->f_off.size(); ++i) {
        if (f_offsets) f_offsets[i] = b->f_off[i];
        if (g_offsets) g_offsets[i] = b->g_off[i];
    }
    return RADON_OK;
}

extern "C" radon_status radon_batch_plan(radon_batch b, int i, radon_desc* d) {
    if (!b || !d) return fail(RADON_ERR_INVALID_ARG, "NULL argument");
    if (i < 0 || i >= (int)b->plans.size()) return fail(RADON_ERR_INVALID_ARG, "gather index out of range");
    *d = b->plans[i]->d;
    return RADON_OK;
}

extern "C" radon_status radon_batch_fwd(radon_batch b, const void* f, int in_type, float* g, void* stream) {
    if (!b) return fail(RADON_ERR_INVALID_ARG, "batch is NULL");
    if (!f || !g) return fail(RADON_ERR_INVALID_ARG, "NULL data pointer");
    if (in_type != RADON_IN_F32 && in_type != RADON_IN_BF16) return fail(RADON_ERR_INVALID_ARG, "unknown input type");
    DeviceGuard guard(b->device);
    const DevBatch U{b->pieces, b->map_units}, Bd{b->pieces, b->map_bands}, K{b->pieces, b->map_kb};
    if (cudaError_t e = cudaMemsetAsync(b->lat_all, 0, b->lat_bytes, (cudaStream_t)stream))
        return cuda_status((int)e, "clearing the lattices");
    if (radon_status s = cuda_status(launch_grid_tiles_dev(U, b->n_units, b->ntaps, f, in_type, stream), "gridding")) return s;
    if (radon_status s = cuda_status(launch_rows_r2c_dev(Bd, b->n_bands, b->smem_rows, stream), "row FFT")) return s;
    if (radon_status s = cuda_status(launch_colconv_dev(K, b->n_kb, b->smem_cols, b->col_x256, 0, stream), "convolution"))
        return s;
    if (radon_status s = cuda_status(launch_rows_c2r_dev(Bd, b->n_bands, b->smem_rows, stream), "inverse row FFT"))
        return s;
    return cuda_status(launch_interp_columns(b->pieces, b->cmap, b->ncols, b->nrho_max, b->col_pieces, 0, 0, b->ntaps, g, stream),
                       "interpolation");
}

extern "C" radon_status radon_batch_adj(radon_batch b, const float* g, float* f, void* stream) {
    if (!b) return fail(RADON_ERR_INVALID_ARG, "batch is NULL");
    if (!f || !g) return fail(RADON_ERR_INVALID_ARG, "NULL data pointer");
    DeviceGuard guard(b->device);
    const DevBatch Bd{b->pieces, b->map_bands}, K{b->pieces, b->map_kb};
    if (radon_status s = cuda_status(launch_col_profiles_cols(b->pieces, b->cmap, b->ncols, b->nrho_max, b->col_pieces,
                                                              0, 0, b->ntaps, g, stream),
                                     "adjoint interpolation (profiles)"))
        return s;
    if (radon_status s = cuda_status(launch_band_rows_dev(Bd, b->n_bands, b->ntaps, b->smem_rows, stream),
                                     "adjoint interpolation (bands)"))
        return s;
    if (radon_status s = cuda_status(launch_colconv_dev(K, b->n_kb, b->smem_cols, b->col_x256, 1, stream), "adjoint convolution"))
        return s;
    if (radon_status s = cuda_status(launch_rows_c2r_dev(Bd, b->n_bands, b->smem_rows, stream), "inverse row FFT"))
        return s;
    return cuda_status(launch_gather_samples(b->pieces, b->smap, b->nsblocks, f, 0, 0, 0, b->ntaps, stream), "adjoint gridding");
}

// ---------------------------------------------------------------------------
// Forward transform on caller-given work memory (used by radon_fwd_noalloc in
// noalloc.cu). Layout of the area: the device copies of the piece
// descriptors, every piece's lattice (with its gridding counters) back to
// back, then every piece's spectrum, then every piece's gridding slots, each
// 256-byte aligned. Every byte the kernels read there is
// written earlier in the same call, so nothing has to be cleared beforehand.
// ---------------------------------------------------------------------------
namespace hr {

int set_error(int status, const char* msg) { return fail((radon_status)status, msg); }

int plan_device(const radon_plan_s* p) { return p->device; }

int plan_forward_work_bytes(const radon_plan_s* p, size_t* bytes) {
    if (!p || !bytes) return fail(RADON_ERR_INVALID_ARG, "NULL argument");
    size_t b = round256b(p->pieces.size() * sizeof(PieceDev));
    for (auto& h : p->pieces) b += piece_lattice_bytes(h.dev) + piece_spectrum_bytes(h.dev) + piece_slot_bytes(h.dev);
    *bytes = b;
    return RADON_OK;
}

int plan_forward_in_work(radon_plan_s* p, const float* f, float* g, void* work, size_t bytes,
                         void* stream) {
    if (!p) return fail(RADON_ERR_INVALID_ARG, "plan is NULL");
    if (!f || !g || !work) return fail(RADON_ERR_INVALID_ARG, "NULL data pointer");
    const int np = (int)p->pieces.size();
    if (np > kWorkMaxPieces)
        return fail(RADON_ERR_UNSUPPORTED, "the static-work forward handles plans of at most 32 pieces");
    size_t need = 0;
    plan_forward_work_bytes(p, &need);
    if (need > bytes)
        return fail(RADON_ERR_UNSUPPORTED,
                    "plan needs " + std::to_string(need) + " bytes of work memory, the area holds " +
                        std::to_string(bytes));
    char* base = (char*)work;
    PieceDev* dpieces = (PieceDev*)base;
    size_t off = round256b(np * sizeof(PieceDev));
    float* lat = (float*)(base + off);
    size_t lat_bytes = 0;
    PieceDev local[kWorkMaxPieces];
    for (int i = 0; i < np; ++i) {
        local[i] = p->pieces[i].dev;
        local[i].lat = (float*)(base + off);
        local[i].prof = nullptr;
        off += piece_lattice_bytes(local[i]);
        lat_bytes += piece_lattice_bytes(local[i]);
    }
    for (int i = 0; i < np; ++i) {
        local[i].spec = (cf*)(base + off);
        off += piece_spectrum_bytes(local[i]);
    }
    for (int i = 0; i < np; ++i) {
        local[i].slots = (float*)(base + off);
        off += piece_slot_bytes(local[i]);
    }
    DeviceGuard guard(p->device);
    if (radon_status s = cuda_status(launch_write_pieces(local, np, dpieces, stream), "piece descriptors"))
        return s;
    return run_forward(p, local, dpieces, lat, lat_bytes, f, g, stream);
}

}  // namespace hr

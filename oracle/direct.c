/*
 * Oracle (test infrastructure only): FP64 direct summation over hyperbolas.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg use
 * this file; the library never links it.
 *
 * Forward, the definition of Eq. (1) folded as in Eq. (3) (Section 2), with
 * the paper's reference discretisation of Section 5: "direct summation ...
 * cubic interpolation in time":
 *
 *   g(tau_i, q_l) = 2 * sum_k w_k dx * I_t[f(., x_k)]( sqrt(tau_i^2 + q_l^2 x_k^2) )
 *
 *   w_0 = w_{Nx-1} = 1/2, else 1                       (trapezoid in x)
 *   I_t = Keys cubic convolution, a = -1/2, 4 taps      (interpolation in t)
 *   samples outside 0..Nt-1 are zero (f = 0 outside the rectangle, Eq. (11))
 *
 * Adjoint, defined by the inner-product identity Eq. (16) with the plain
 * sample-sum inner product:
 *
 *   f*(t_j, x_k) = 2 w_k dx * sum_{i,l} g(tau_i, q_l) * c( sqrt(tau_i^2+q_l^2 x_k^2)/dt - j )
 *
 * where c is the Keys kernel. Sampled variants evaluate single outputs in
 * O(Nx) (forward) or O(Nq) (adjoint, using the closed-form tau-range whose
 * hyperbolas pass within two samples of t_j).
 */
#include <math.h>
#include <stddef.h>

/* Keys (1981) cubic convolution kernel with a = -1/2. */
static double keys(double s)
{
    const double a = -0.5;
    s = fabs(s);
    if (s <= 1.0) return ((a + 2.0) * s - (a + 3.0)) * s * s + 1.0;
    if (s < 2.0) return ((a * s - 5.0 * a) * s + 8.0 * a) * s - 4.0 * a;
    return 0.0;
}

/* Keys interpolation of one trace at fractional sample position p. */
static double interp_trace(const double *tr, int Nt, double p)
{
    double fl = floor(p);
    long j0 = (long)fl;
    double acc = 0.0;
    for (long j = j0 - 1; j <= j0 + 2; ++j) {
        if (j < 0 || j >= Nt) continue;
        acc += tr[j] * keys(p - (double)j);
    }
    return acc;
}

static double wx(int k, int Nx)
{
    return (k == 0 || k == Nx - 1) ? 0.5 : 1.0;
}

/* One forward output g(tau, q). */
static double fwd_point(const double *f, int Nt, int Nx, double dt, double dx,
                        double tau, double q)
{
    double acc = 0.0;
    for (int k = 0; k < Nx; ++k) {
        double x = k * dx;
        double t = sqrt(tau * tau + q * q * x * x);
        acc += wx(k, Nx) * interp_trace(f + (size_t)k * Nt, Nt, t / dt);
    }
    return 2.0 * dx * acc;
}

/* g[l*Ntau + i] for all outputs. tau[], q[] are the output grids. */
void oracle_direct_fwd(const double *f, int Nt, int Nx, double dt, double dx,
                       const double *tau, int Ntau, const double *q, int Nq,
                       double *g)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int l = 0; l < Nq; ++l)
        for (int i = 0; i < Ntau; ++i)
            g[(size_t)l * Ntau + i] = fwd_point(f, Nt, Nx, dt, dx, tau[i], q[l]);
}

/* Forward at npts sampled outputs (li[p], ii[p]). */
void oracle_direct_fwd_points(const double *f, int Nt, int Nx, double dt, double dx,
                              const double *tau, const double *q,
                              const int *ii, const int *li, int npts, double *out)
{
    #pragma omp parallel for schedule(static)
    for (int p = 0; p < npts; ++p)
        out[p] = fwd_point(f, Nt, Nx, dt, dx, tau[ii[p]], q[li[p]]);
}

/*
 * One adjoint output f*(t_j, x_k). For each q_l, only intercepts tau_i whose
 * hyperbola time t = sqrt(tau_i^2 + q_l^2 x_k^2) lies in (t_j - 2dt, t_j + 2dt)
 * have a non-zero Keys weight; that tau-range is taken from the inequality,
 * widened by one sample on each side, and every term is still weighted by
 * keys(), which is exactly zero outside the support.
 * The tau grid is tau_i = tau0 + i * dtau.
 */
static double adj_point(const double *g, int Nt, int Nx, double dt, double dx,
                        double tau0, double dtau, int Ntau, const double *q, int Nq,
                        int j, int k)
{
    (void)Nt;
    double x = k * dx;
    double tlo = (j - 2) * dt, thi = (j + 2) * dt;
    double acc = 0.0;
    for (int l = 0; l < Nq; ++l) {
        double qx2 = q[l] * q[l] * x * x;
        double lo2 = tlo > 0.0 ? tlo * tlo - qx2 : -qx2;
        double hi2 = thi * thi - qx2;
        if (hi2 < 0.0) continue;
        double taulo = lo2 > 0.0 ? sqrt(lo2) : 0.0;
        double tauhi = sqrt(hi2);
        long i0 = (long)floor((taulo - tau0) / dtau) - 1;
        long i1 = (long)ceil((tauhi - tau0) / dtau) + 1;
        if (i0 < 0) i0 = 0;
        if (i1 > Ntau - 1) i1 = Ntau - 1;
        for (long i = i0; i <= i1; ++i) {
            double tau = tau0 + i * dtau;
            double t = sqrt(tau * tau + qx2);
            double w = keys(t / dt - (double)j);
            if (w != 0.0) acc += g[(size_t)l * Ntau + i] * w;
        }
    }
    return 2.0 * wx(k, Nx) * dx * acc;
}

void oracle_direct_adj(const double *g, int Nt, int Nx, double dt, double dx,
                       double tau0, double dtau, int Ntau, const double *q, int Nq,
                       double *f)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < Nx; ++k)
        for (int j = 0; j < Nt; ++j)
            f[(size_t)k * Nt + j] = adj_point(g, Nt, Nx, dt, dx, tau0, dtau, Ntau,
                                              q, Nq, j, k);
}

void oracle_direct_adj_points(const double *g, int Nt, int Nx, double dt, double dx,
                              double tau0, double dtau, int Ntau,
                              const double *q, int Nq,
                              const int *jj, const int *kk, int npts, double *out)
{
    #pragma omp parallel for schedule(static)
    for (int p = 0; p < npts; ++p)
        out[p] = adj_point(g, Nt, Nx, dt, dx, tau0, dtau, Ntau, q, Nq, jj[p], kk[p]);
}

/*
 * Brute-force adjoint: every (i, l) pair, no range shortcut. Used on tiny
 * grids to check the shortcut above.
 */
void oracle_direct_adj_brute(const double *g, int Nt, int Nx, double dt, double dx,
                             const double *tau, int Ntau, const double *q, int Nq,
                             double *f)
{
    for (int k = 0; k < Nx; ++k) {
        double x = k * dx;
        for (int j = 0; j < Nt; ++j) {
            double acc = 0.0;
            for (int l = 0; l < Nq; ++l)
                for (int i = 0; i < Ntau; ++i) {
                    double t = sqrt(tau[i] * tau[i] + q[l] * q[l] * x * x);
                    acc += g[(size_t)l * Ntau + i] * keys(t / dt - (double)j);
                }
            f[(size_t)k * Nt + j] = 2.0 * wx(k, Nx) * dx * acc;
        }
    }
}

/*
 * Unequally spaced offsets. Section 4 states that the method carries over to
 * unequally spaced (t, x) and (tau, q) grids; the reference sum then takes
 * the trapezoid rule on the given offsets x_0 < x_1 < ... < x_{Nx-1}:
 *
 *   g(tau_i, q_l) = 2 * sum_k om_k * I_t[f(., x_k)]( sqrt(tau_i^2 + q_l^2 x_k^2) )
 *   om_0 = (x_1 - x_0) / 2,  om_k = (x_{k+1} - x_{k-1}) / 2,
 *   om_{Nx-1} = (x_{Nx-1} - x_{Nx-2}) / 2
 *
 * (om_k = w_k dx on a regular grid), the slownesses q_l being any list; the
 * adjoint is again the transpose under the plain sample-sum inner product:
 *
 *   f*(t_j, x_k) = 2 om_k * sum_{i,l} g(tau_i, q_l) * c( sqrt(tau_i^2+q_l^2 x_k^2)/dt - j )
 *
 * Needs Nx >= 2.
 */
static double trap_weight(const double *x, int Nx, int k)
{
    if (k == 0) return 0.5 * (x[1] - x[0]);
    if (k == Nx - 1) return 0.5 * (x[Nx - 1] - x[Nx - 2]);
    return 0.5 * (x[k + 1] - x[k - 1]);
}

static double fwd_point_x(const double *f, int Nt, int Nx, double dt, const double *x,
                          double tau, double q)
{
    double acc = 0.0;
    for (int k = 0; k < Nx; ++k) {
        double t = sqrt(tau * tau + q * q * x[k] * x[k]);
        acc += trap_weight(x, Nx, k) * interp_trace(f + (size_t)k * Nt, Nt, t / dt);
    }
    return 2.0 * acc;
}

void oracle_direct_fwd_x(const double *f, int Nt, int Nx, double dt, const double *x,
                         const double *tau, int Ntau, const double *q, int Nq, double *g)
{
    #pragma omp parallel for schedule(static)
    for (int l = 0; l < Nq; ++l)
        for (int i = 0; i < Ntau; ++i)
            g[(size_t)l * Ntau + i] = fwd_point_x(f, Nt, Nx, dt, x, tau[i], q[l]);
}

void oracle_direct_fwd_x_points(const double *f, int Nt, int Nx, double dt, const double *x,
                                const double *tau, const double *q,
                                const int *ii, const int *li, int npts, double *out)
{
    #pragma omp parallel for schedule(static)
    for (int p = 0; p < npts; ++p)
        out[p] = fwd_point_x(f, Nt, Nx, dt, x, tau[ii[p]], q[li[p]]);
}

/* One adjoint output on unequal offsets; the same tau-range shortcut as
 * adj_point (every term still weighted by keys()). */
static double adj_point_x(const double *g, int Nx, double dt, const double *x,
                          double tau0, double dtau, int Ntau, const double *q, int Nq,
                          int j, int k)
{
    double tlo = (j - 2) * dt, thi = (j + 2) * dt;
    double acc = 0.0;
    for (int l = 0; l < Nq; ++l) {
        double qx2 = q[l] * q[l] * x[k] * x[k];
        double lo2 = tlo > 0.0 ? tlo * tlo - qx2 : -qx2;
        double hi2 = thi * thi - qx2;
        if (hi2 < 0.0) continue;
        double taulo = lo2 > 0.0 ? sqrt(lo2) : 0.0;
        double tauhi = sqrt(hi2);
        long i0 = (long)floor((taulo - tau0) / dtau) - 1;
        long i1 = (long)ceil((tauhi - tau0) / dtau) + 1;
        if (i0 < 0) i0 = 0;
        if (i1 > Ntau - 1) i1 = Ntau - 1;
        for (long i = i0; i <= i1; ++i) {
            double tau = tau0 + i * dtau;
            double t = sqrt(tau * tau + qx2);
            double w = keys(t / dt - (double)j);
            if (w != 0.0) acc += g[(size_t)l * Ntau + i] * w;
        }
    }
    return 2.0 * trap_weight(x, Nx, k) * acc;
}

void oracle_direct_adj_x(const double *g, int Nt, int Nx, double dt, const double *x,
                         double tau0, double dtau, int Ntau, const double *q, int Nq,
                         double *f)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < Nx; ++k)
        for (int j = 0; j < Nt; ++j)
            f[(size_t)k * Nt + j] = adj_point_x(g, Nx, dt, x, tau0, dtau, Ntau, q, Nq, j, k);
}

void oracle_direct_adj_x_points(const double *g, int Nx, double dt, const double *x,
                                double tau0, double dtau, int Ntau, const double *q, int Nq,
                                const int *jj, const int *kk, int npts, double *out)
{
    #pragma omp parallel for schedule(static)
    for (int p = 0; p < npts; ++p)
        out[p] = adj_point_x(g, Nx, dt, x, tau0, dtau, Ntau, q, Nq, jj[p], kk[p]);
}

/* Threads the following calls use (OpenMP; no effect without it). */
void oracle_set_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

/* Number of OpenMP threads the oracle runs with (1 without OpenMP). */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

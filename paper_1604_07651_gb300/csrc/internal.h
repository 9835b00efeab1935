// Internal structures shared by the host plan (plan.cpp) and the kernels
// (kernels.cu). Not part of the public ABI.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "hostdev.h"

struct radon_plan_s;  // defined in plan.cpp

namespace hr {

struct FftPlan {            // radix schedule of one FFT length
    int n;
    int nst;
    int rad[24];
};

// Device-visible description of one sub-problem (one time piece of one
// slowness piece). Passed to kernels by value.
struct PieceDev {
    // lattice
    int Ntheta, Nrho, Ptheta, Prho;
    int k1max, k2max;
    int CB;                 // spectrum columns per block of the blocked layout
    int nkb;                // number of column blocks: ceil((k2max+1)/CB)
    int R;                  // lattice rows per band of the row kernels
    int nbands;
    float theta0, rho0;     // lattice origin (approximate, for picking references)
    float inv_dtheta, inv_drho;
    float alpha;
    // samples of the gather
    int Nt, Nx;
    int jt_lo, jt_hi;
    // output columns of the slowness piece
    int Ntau, l_lo, l_hi;
    float a_r, r_max;       // lines with e^rho outside [a_r, r_max] miss the data
    // tables (device pointers)
    const ff* lam;          // [Nt]   rotated-frame coordinate along e_alpha, per sample time
    const float* cj;        // [Nt]   per-time weight: window * 2 a^2 tb / (n_t n_x dtheta drho)
    const int* jfirst;      // [Nx]   first sample of each trace kept by the mute
    const ff* hk;           // [Nx]   rotated-frame coordinate along e_perp, per trace
    const float* wk;        // [Nx]   trapezoid weight in x
    const int2* jband;      // [nbands][Nx] candidate sample range of each band
    const int2* lband;      // [nbands] candidate output-column range of each band
    const ff* rowc;         // [Ntheta] cos(theta_m - alpha)
    const ff* rows;         // [Ntheta] sin(theta_m - alpha)
    const ff* R1;           // [Nrho] e^{rho_n}
    const ff* R2;           // [Nrho] e^{2 rho_n}
    const ff* E;            // [3 * ncol] e^rho(i) = E0 + E1 i + E2 i^2 per column
    const float4* colw;     // [ncol] theta tap weights of each column
    const int* colm0;       // [ncol] first theta tap of each column
    const float* colscale;  // [ncol] output scale 2 X cos(psi) / a
    const cf* K;            // [nkb][k1max+1][CB] kernel spectrum (normalised)
    const cf* twM;          // [Prho/2]  exp(-2 pi i k / (Prho/2))
    const cf* twP;          // [Prho/2+1] exp(-2 pi i k / Prho)
    const cf* twT;          // [Ptheta]  exp(-2 pi i k / Ptheta)
    FftPlan fftM;           // row FFT (length Prho/2)
    FftPlan fftT;           // column FFT (length Ptheta)
    float* lat;             // [Ntheta][Nrho] real lattice (Q forward, G' adjoint)
};

// Launchers (kernels.cu)
int launch_scatter_gather_rows(const PieceDev& P, const float* f, cf* spec, void* stream);
int launch_scatter_radon_rows(const PieceDev& P, const float* g, cf* spec, void* stream);
int launch_colconv(const PieceDev& P, const cf* in, cf* out, int adjoint, void* stream);
int launch_rows_c2r(const PieceDev& P, const cf* spec, void* stream);
int launch_gather_radon(const PieceDev* pieces, int npieces, const PieceDev* dev_pieces,
                        int l_lo, int l_hi, float* g, void* stream);
int launch_gather_samples(const PieceDev* dev_pieces, int npieces, int Nt, int Nx,
                          float* f, void* stream);
int launch_zeta_gemm(const double* A, const double* Bre, const double* Bim, int n1, int nn,
                     int n2, double* Zre, double* Zim, void* stream);
int launch_direct_fwd(const float* f, float* g, int Nt, int Nx, int Ntau, int Nq, double dt,
                      double dx, double tau0, double dtau, double qmin, double dq, void* stream);
int launch_direct_adj(const float* g, float* f, int Nt, int Nx, int Ntau, int Nq, double dt,
                      double dx, double tau0, double dtau, double qmin, double dq, void* stream);
size_t scatter_smem_bytes(const PieceDev& P);

// Forward transform of a plan with every work buffer carved out of the
// caller-given device area `work` (256-byte aligned, `bytes` long) instead of
// the plan's own buffers; allocates nothing (plan.cpp). Return radon_status.
int set_error(int status, const char* msg);   // records the thread's last error, returns status
int plan_device(const radon_plan_s* p);
int plan_forward_work_bytes(const radon_plan_s* p, size_t* bytes);
int plan_forward_in_work(radon_plan_s* p, const float* f, float* g, void* work, size_t bytes,
                         void* stream);
size_t colconv_smem_bytes(const PieceDev& P);
int max_smem_optin();

}  // namespace hr

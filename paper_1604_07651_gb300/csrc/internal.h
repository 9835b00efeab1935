// Internal structures shared by the host plan (plan.cpp) and the kernels
// (kernels.cu). Not part of the public ABI.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "hostdev.h"

struct radon_plan_s;  // defined in plan.cpp
// The plan's given slownesses on its device ([Nq], s/km), or NULL when it
// samples the regular slowness grid of its descriptor.
const double* plan_q_values(const radon_plan_s* p);

namespace hr {

struct FftPlan {            // radix schedule of one FFT length
    int n;
    int nst;
    int rad[8];             // radix of each stage / pass
    int st[8];              // column plans (decimation in frequency): stride of each pass
    int tw[8];              // column plans: offset of each pass's twiddles in the table
};

// Lattice position of one gather sample, computed once per plan in FP64:
// first taps (m0, n0) packed as (m0 << 16) | n0, fractional parts (ft, fr)
// of the position in cells, and the sample weight w (zero when the sample is
// muted or outside the sub-problem).
struct __align__(16) SampleEnt { int mn; float ft, fr, w; };
// Rho position of one output of a slowness column: first tap n0 (-1 when the
// line misses the sub-problem's data) and fractional part fr.
struct __align__(8) RadonEnt { int n0; float fr; };

// FP64 geometry the plan-time table kernels need (by value).
struct TableArgs {
    double a, ca, sa, O1, O2, alpha;
    double theta0, dtheta, rho0, drho, a_r, r_max;
    double n_t, T, tau0, dtau;
    const double* xb;       // [Nx] rescaled offsets x_k / X (device)
    int jt_lo, nj, Nx, Ntheta, Nrho, Ntau, ncol;
    int ntaps;              // B-spline taps per axis: 4 (cubic) or 6 (quintic)
};

// Device-visible description of one sub-problem (one time piece of one
// slowness piece). Passed to kernels by value.
struct PieceDev {
    // lattice
    int Ntheta, Nrho, Ptheta, Prho;
    int ntaps;              // B-spline taps per axis: 4 (cubic) or 6 (quintic)
    int k1max, k2max;
    int CB;                 // spectrum columns per block of the blocked layout
    int nkb;                // number of column blocks: ceil((k2max+1)/CB)
    int R;                  // lattice rows per band of the row kernels
    int nbands;
    // samples of the gather
    int Nt, Nx;
    int jt_lo, jt_hi, nj;   // nj = jt_hi - jt_lo + 1
    // output columns of the slowness piece
    int Ntau, l_lo, l_hi;
    // tables (device pointers)
    const SampleEnt* stab;  // [Nx][nj] position and weight of every sample of the piece
    const RadonEnt* rtab;   // [ncol][Ntau] rho position of every output of the piece
    const int2* rrange;     // [ncol] first and last output of the column with a valid rtab entry
                            // (x > y: none); every valid entry lies inside
    int ntr, ntc;           // lattice tiles of the forward gridding: rows, columns
    int nunits;             // work units of the forward gridding
    const int4* units;      // (tile, first chunk, end chunk, 28 - ilogb(cell weight bound)), heaviest first
    const int4* uslot;      // per unit: (first slot of its tile, units of the tile, its index among them,
                            // counter of the tile); tiles of one unit: (0, 1, 0, -1)
    float* slots;           // [nslots][kTileRows * kTileCols] partial tiles of the split tiles
    int nslots;             // units of split tiles (tiles cut into several units)
    int ncount;             // split tiles: their counters follow the lattice, [ncount] ints
    const int4* chunks;     // (trace k, first sample j, count <= 8, 0), grouped by tile
    const int2* lband;      // [nbands] candidate output-column range of each band
    const int* colsh;       // [ncol] 28 - ilogb(cell weight bound) of the adjoint column profiles
    const float4* colw;     // [ncol] theta tap weights of each column (taps 0 .. 3)
    const float2* colw2;    // [ncol] theta tap weights 4 and 5 (six taps only; else null)
    const int* colm0;       // [ncol] first theta tap of each column
    const float* colscale;  // [ncol] output scale 2 X cos(psi) / a
    const cf* K;            // [nkb][k1max+1][CB] kernel spectrum (normalised)
    const cf* twM;          // pass twiddle tables of the row FFT pair (length Prho/2)
    const int* rpos;        // [Prho/2] position of each frequency after the forward row passes
    const cf* twP;          // [Prho/2+1] exp(-2 pi i k / Prho)
    const cf* twT;          // pass twiddle tables of the column FFT pair (length Ptheta), twT_len entries
    int twT_len;            // entries of twT, a multiple of 2 (16-byte copies)
    FftPlan fftM;           // row FFT (length Prho/2)
    FftPlan fftT;           // column FFT (length Ptheta)
    float* lat;             // [Ntheta][Nrho] real lattice (Q forward, G' adjoint)
    cf* spec;               // [nkb][Ntheta][CB] half spectrum of the lattice rows (in-place column pass)
    float* prof;            // [ncol][hpitch] rho profiles of the output columns (adjoint)
    int hpitch;             // row pitch of prof, floats, multiple of 4
    long long f_off;        // element offset of this gather in packed gather buffers (0: single plan)
    long long g_off;        // element offset of this gather's image in packed image buffers
};

// Up to kMaxBatch sub-problems launched as one grid: the blocks of piece k
// are [first[k], first[k+1]); passed by value (about 3.3 KB of parameters).
constexpr int kMaxBatch = 8;
// Time pieces of one output column at most (RADON_MAX_TSPLIT + 1).
constexpr int kMaxColPieces = 9;
struct PieceBatch {
    int n;
    int first[kMaxBatch + 1];
    PieceDev p[kMaxBatch];
};

// Any number of sub-problems (of many gathers) launched as one grid: the
// descriptors live in device memory and map[b] = (piece, block within the
// piece) for every block b of the launch.
struct DevBatch {
    const PieceDev* p;
    const int2* map;
};

// Input element types of the gridding.
enum { kInF32 = 0, kInBF16 = 1 };

// Lattice tile of the forward gridding (rows x columns of cells) and the
// largest work unit (chunks of <= 8 samples; one thread per chunk).
constexpr int kTileRows = 32;
constexpr int kTileCols = 64;
constexpr int kUnitChunks = 256;
// Most lattice rows one band of the row kernels holds.
constexpr int kMaxBandRows = 6;

// Launchers (kernels.cu). The batched ones take n <= kMaxBatch pieces (host
// copies of the descriptors) and launch one grid over all of them. Every
// piece of one launch has the same number of B-spline taps (`ntaps`, or the
// first descriptor's); another number than 4 or 6 returns
// cudaErrorInvalidValue.
int launch_grid_tiles(const PieceDev* P, int n, const float* f, void* stream);
int launch_rows_r2c(const PieceDev* P, int n, void* stream);
int launch_band_rows(const PieceDev* P, int n, void* stream);
int launch_colconv(const PieceDev* P, int n, int adjoint, void* stream);
int launch_rows_c2r(const PieceDev* P, int n, void* stream);
// The same stages over a device-resident batch: `nblocks` blocks, map in S,
// `smem` the largest dynamic shared memory any piece of the launch needs.
int launch_grid_tiles_dev(const DevBatch& S, int nblocks, int ntaps, const void* f, int in_type, void* stream);
int launch_rows_r2c_dev(const DevBatch& S, int nblocks, size_t smem, void* stream);
int launch_band_rows_dev(const DevBatch& S, int nblocks, int ntaps, size_t smem, void* stream);
// x256: every piece of the launch takes the compile-time column pass
// (colconv_all_x256), which runs at fewer threads per CTA.
int launch_colconv_dev(const DevBatch& S, int nblocks, size_t smem, bool x256, int adjoint, void* stream);
bool colconv_all_x256(const PieceDev* P, int n);
int launch_rows_c2r_dev(const DevBatch& S, int nblocks, size_t smem, void* stream);
// Output interpolation: one CTA per output column; cmap[b] = (first piece,
// number of time pieces, column l, 0) in `pieces` (device), or, when
// np_all > 0 (one gather, one slowness piece of np_all time pieces, ntau_all
// outputs per column), column b of pieces[0..np_all). np_max: the largest
// number of time pieces of a column (<= kMaxColPieces); shared memory
// np_max * nrho_max floats.
int launch_interp_columns(const PieceDev* pieces, const int4* cmap, int ncols, int nrho_max, int np_max,
                          int ntau_all, int np_all, int ntaps, float* g, void* stream);
// Adjoint column profiles of every time piece of a column at once, one CTA
// per output column (cmap / np_all / shared memory as the interpolation's).
int launch_col_profiles_cols(const PieceDev* pieces, const int4* cmap, int ncols, int nrho_max, int np_max,
                             int ntau_all, int np_all, int ntaps, const float* g, void* stream);
// Adjoint gather: one CTA per kSampleBlock samples of one gather;
// smap[b] = (first piece, number of pieces, first sample, 0), or, when
// np_all > 0 (one gather of Nt_all x Nx_all samples in np_all pieces),
// samples [b kSampleBlock, (b + 1) kSampleBlock).
constexpr int kSampleBlock = 256;
int launch_gather_samples(const PieceDev* pieces, const int4* smap, int nblocks, float* f, int np_all, int Nt_all,
                          int Nx_all, int ntaps, void* stream);
size_t rows_smem_bytes(const PieceDev& P);
int launch_sample_table(const TableArgs& A, const double* cj, const double* wk, const int* jfirst,
                        SampleEnt* out);
int launch_radon_table(const TableArgs& A, const double* qb2, RadonEnt* out);
int launch_zeta_gemm(const double* A, const double* Bre, const double* Bim, int n1, int nn,
                     int n2, double* Zre, double* Zim, void* stream);
int launch_direct_fwd(const float* f, float* g, int Nt, int Nx, int Ntau, int Nq, double dt,
                      double dx, double tau0, double dtau, double qmin, double dq, void* stream);
int launch_direct_adj(const float* g, float* f, int Nt, int Nx, int Ntau, int Nq, double dt,
                      double dx, double tau0, double dtau, double qmin, double dq, void* stream);
size_t scatter_smem_bytes(const PieceDev& P);   // = rows_smem_bytes

// Forward transform of a plan with every work buffer carved out of the
// caller-given device area `work` (256-byte aligned, `bytes` long) instead of
// the plan's own buffers; allocates nothing (plan.cpp). Return radon_status.
int set_error(int status, const char* msg);   // records the thread's last error, returns status
int plan_device(const radon_plan_s* p);
int plan_forward_work_bytes(const radon_plan_s* p, size_t* bytes);
int plan_forward_in_work(radon_plan_s* p, const float* f, float* g, void* work, size_t bytes,
                         void* stream);
// Most pieces a plan may have for plan_forward_in_work; launch_write_pieces
// writes n <= kWorkMaxPieces descriptors to device memory `dst` with one
// kernel launch on `stream` (the descriptors travel as its parameter).
constexpr int kWorkMaxPieces = 32;
int launch_write_pieces(const PieceDev* pieces, int n, PieceDev* dst, void* stream);
size_t colconv_smem_bytes(const PieceDev& P);
int max_smem_optin();
// Dynamic shared memory available to the output interpolation's profiles
// (the opt-in limit less the kernel's static shared memory); 0 on error.
size_t interp_smem_limit(int ntaps);

}  // namespace hr

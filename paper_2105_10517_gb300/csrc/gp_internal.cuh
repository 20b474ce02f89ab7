// gp_internal.cuh -- data layout and launch arguments shared by the CUDA
// translation units of libgpspin (not part of the public C ABI).
//
// One split-step Crank-Nicolson time step (arXiv 2105.10517, program summary
// "Solution method"; Supplementary Material Eqs. S.1-S.5) is two line passes:
//
//   x-pass  psi[c][j][i] --(pending scale s, pointwise substep P, U_y^dagger)-->
//           Sigma_y eigen-channels --(CN solve along x per row and channel)-->
//           --(U_x^dagger U_y)--> Sigma_x eigen-channels, stored TRANSPOSED as
//           t[mu][i][j] so that the y-pass reads whole columns contiguously;
//   y-pass  t[mu][i][j] --(CN solve along y per column and channel)--(U_x)-->
//           psi[c][j][i] plus per-CTA partial norms (FP64).
//
// In imaginary time a one-CTA kernel turns the partial norms into the scale
// s = 1/sqrt(N) that the next x-pass applies on load ("pending" scale).
//
// The SO term gamma(eta p_y Sigma_x - p_x Sigma_y) is diagonalised by the
// constant unitaries U_y (eigenvectors of Sigma_y) in the x-pass and U_x
// (eigenvectors of Sigma_x) in the y-pass, so each line system is a scalar
// tridiagonal per channel lambda in {+1, 0, -1}:
//   A = -1/2 D2 + kappa D1,  kappa = i(gamma lambda - Omega y_j)      (x-pass)
//                            kappa = i(Omega x_i - eta gamma mu)       (y-pass)
//
// Both passes exist for complex128 (double2, the FP64 path) and complex64
// (float2, the FP32-storage path); coefficient tables are always computed in
// FP64 and stored in the pass's precision; norms are always summed in FP64.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "../../include/gpspin.h"

namespace gpspin {

// Head length of the tabulated Thomas factorisation and of the fixup powers.
constexpr int kHead = 32;
constexpr int kFix = 64;

// Thomas factorisation of (I + tau A) for one line and one eigen-channel.
// Row k of the elimination: inv_k = 1/(beta - alpha c'_{k-1}), c'_k = gamma' inv_k,
// g_k = alpha inv_k.  Entries k >= kHead equal entry kHead-1 to rounding (the
// recurrence contracts by |c'|^2 per row), so kernels index min(k, kHead-1).
// pf[t] = (-g_inf)^(t+1) and pb[t] = (-c'_inf)^(t+1) are the influence of a
// chunk's carry on the t-th element after (forward) or before (backward) it.
template <typename C>
struct LineCoefT {
    C inv[kHead];
    C g[kHead];
    C cp[kHead];
    C pf[kFix];
    C pb[kFix];
};
using LineCoef = LineCoefT<double2>;
using LineCoefF = LineCoefT<float2>;

// Tiling of one line pass (chosen on the host).
struct LineTiling {
    int L;      // line length
    int nlines; // number of lines
    int R;      // lines per CTA
    int m;      // chunk length of the parallel Thomas solve
    int Q;      // chunks per line = ceil(L / m)
    int F;      // fixup length (|c'_inf|^F below the precision's rounding), F < m
    int cs;     // smem stride of one chunk (>= m; the padding spreads the chunk-parallel
                // accesses of the solve over the banks)
    int Lp;     // smem stride of one line-channel in a CTA (>= Qc cs)
    int S;      // CTAs per line group (a thread-block cluster when S > 1)
    int Qc;     // chunks per CTA = ceil(Q / S); CTA rank r holds chunks r*Qc ..
    int threads;
    size_t smem;
    size_t off_b;  // byte offsets in dynamic smem of the second line array (also the
    size_t off_cf; // staging area of the bulk row copies) and of the carry arrays
    size_t off_cb;
    int bulk;      // rows are 16-byte aligned: stage them with cp.async.bulk
    int single;    // one line array: rows are staged in place (register-resident solve: complex64
                   // m = 16/24/32, complex128 m = 32)
};

// Kinds of tiling: complex128; complex64 with the shared-memory solve (two line
// arrays, any chunk length); complex64 with the register-resident solve;
// complex128 with the register-resident solve (one line array, m = 32).
enum TileKind { TILE_C128 = 0, TILE_C64 = 1, TILE_C64_REG = 2, TILE_C128_REG = 3 };

template <typename C>
struct PassArgsT {
    const C* in;
    C* out;
    const LineCoefT<C>* coef;  // [nlines][3]
    LineTiling t;
    int nx, ny;
    int do_p;                  // x-pass: apply the pointwise substep
    int do_solve;              // apply the CN solve (0: channels pass through)
    const double* scale;       // device scalar: pending normalisation (x-pass)
    double* partials;          // y-pass: per-CTA sum |psi|^2 (per component when mcomp)
    int mcomp;                 // y-pass: three partials per CTA, one per component
    int* err;                  // status bits set by the kernel (8: bulk-copy wait timed out)
    // pointwise substep constants (x-pass)
    const C* ex;               // [nx] exp(-tau' wx^2 x^2 / 2)
    const C* ey;               // [ny] exp(-tau' wy^2 y^2 / 2)
    double dt, c0, c2, rabi;
    // grid and trap (the complex64 pass evaluates the trap factor inline)
    double x0, dx, y0, dy, wx, wy;
    // the same constants rounded once to FP32 on the host (complex64 x-pass):
    // dt c0, dt c2, dt R / sqrt2, dt, x0, dx, y0, dy, dt wx^2 / 2, dt wy^2 / 2
    float kf[10];
};
using PassArgs = PassArgsT<double2>;
using PassArgsF = PassArgsT<float2>;

int report_cuda(cudaError_t e, const char* what);
// parameter checks and tiling (gp_capi.cu)
int validate(const gp_params* p);
int eta_of(const gp_params& p);
double gamma_of(const gp_params& p);
double max_cp(const gp_params& p, int dir, int mode);
// fp32 = 1: tiling for complex64 lines (fixups to 2^-26 instead of 2^-60)
// split = 1 allows a line group to span a 2-CTA cluster (not for batched launches).
int choose_tiling(int L, int nlines, double cpmax, LineTiling* t, int kind = TILE_C128, int split = 1);
// A specific tiling (autotuner candidates): S CTAs per line group, R lines per
// CTA, chunk length m (raised to the minimum the precision needs).
// compact = 1: chunk stride = chunk length (no chunk padding), the line-channel
// stride padded for the fewest bank conflicts: less shared memory per CTA, which
// can buy one more resident CTA per SM at the price of a few conflicts.
int make_tiling(int L, int nlines, double cpmax, int kind, int S, int R, int m, LineTiling* t, int compact = 0);

// launchers (gp_sweeps.cu)
int launch_coef(LineCoef* coef, int nlines, int dir, int mode, double h, double line_len, double line_h,
                double dt, double omeg, double gamma, int eta, int* status, cudaStream_t st);
int launch_coef(LineCoefF* coef, int nlines, int dir, int mode, double h, double line_len, double line_h,
                double dt, double omeg, double gamma, int eta, int* status, cudaStream_t st);
int launch_trap_table(double2* out, int n, double len, double w, double dt, int mode, cudaStream_t st);
int launch_trap_table(float2* out, int n, double len, double w, double dt, int mode, cudaStream_t st);
int launch_xpass(const PassArgs& a, int mode, cudaStream_t st);
// closing x-pass of a second-order step (solve, U_y, pointwise substep, natural store, partial norms)
int launch_xtail(const PassArgs& a, int mode, cudaStream_t st);
int launch_ypass(const PassArgs& a, int mode, cudaStream_t st);
int launch_xpass(const PassArgsF& a, int mode, cudaStream_t st);
int launch_ypass(const PassArgsF& a, int mode, cudaStream_t st);
// Batched passes over (instance, CTA) work items; m_reg = 16/24/32 selects the
// register-resident solve (every item's tiling one-array with that m), 0 the
// shared-memory solve.  work: null for one CTA per item; else two device ints,
// zero before the launch and zero again after it, that make the launch
// persistent (one CTA per resident slot, items taken from a counter), with at
// most max_ctas CTAs if max_ctas > 0.
int launch_xpass_batched(const PassArgs* args, const int2* items, const int* n_items, int capacity, int threads,
                         size_t smem, int mode, cudaStream_t st, int m_reg = 0, int* work = nullptr,
                         int max_ctas = 0);
int launch_ypass_batched(const PassArgs* args, const int2* items, const int* n_items, int capacity, int threads,
                         size_t smem, int mode, cudaStream_t st, int m_reg = 0, int* work = nullptr,
                         int max_ctas = 0);
int launch_xpass_batched(const PassArgsF* args, const int2* items, const int* n_items, int capacity, int threads,
                         size_t smem, int mode, cudaStream_t st, int m_reg = 0, int* work = nullptr,
                         int max_ctas = 0);
int launch_ypass_batched(const PassArgsF* args, const int2* items, const int* n_items, int capacity, int threads,
                         size_t smem, int mode, cudaStream_t st, int m_reg = 0, int* work = nullptr,
                         int max_ctas = 0);
// the bounded mbarrier wait of the passes on a barrier nothing arrives on
int launch_wait_probe(int tries, int* err, cudaStream_t st);
// launchers (gp_reduce.cu)
int launch_norm(const double2* psi, size_t n, double* partials, int nblk, double da, double* scale, int* flag,
                cudaStream_t st);
int launch_finalize_norm(const double* partials, int n, double da, double* scale, int* flag, cudaStream_t st);
// One CTA per instance: fin[b] = {partials, n_partials, da, scale} of instance b.
struct FinArgs {
    const double* partials;
    int n;
    double da;
    double* scale;
};
int launch_finalize_norm_batched(const FinArgs* fin, const int* n_inst, int capacity, int* flag, cudaStream_t st);
int launch_finalize_m(const double* partials, int n, double da, double m, double* sigma, int* flag, cudaStream_t st);
int launch_apply_comp_scale(double2* psi, size_t plane, const double* sigma, cudaStream_t st);
int launch_apply_comp_scale(float2* psi, size_t plane, const double* sigma, cudaStream_t st);
int launch_apply_scale(double2* psi, size_t n, double* scale, cudaStream_t st);
int launch_apply_scale(float2* psi, size_t n, double* scale, cudaStream_t st);
int launch_set_scalar(double* p, double v, cudaStream_t st);
int launch_scaled_copy(double2* dst, const double2* src, size_t n, const double* scale, cudaStream_t st);
int launch_scaled_copy(double2* dst, const float2* src, size_t n, const double* scale, cudaStream_t st);
int launch_narrow(float2* dst, const double2* src, size_t n, cudaStream_t st);
int launch_init_gaussian(double2* psi, int nx, int ny, double xlen, double ylen, const double frac[3],
                         const int winding[3], unsigned long long seed, double noise, cudaStream_t st);
int obs_blocks(int nx, int ny);
int obs_slots();
int launch_observables(const double2* psi, const double* scale, int nx, int ny, double xlen, double ylen, double wx,
                       double wy, double c0, double c2, double rabi, double omeg, double gamma, int eta,
                       double* partials, double* out, int* flag, cudaStream_t st);

}  // namespace gpspin

// gp_capi.cu -- the C ABI of libgpspin (include/gpspin.h): handle, device
// state, Thomas coefficient cache, tiling choice and the step sequence of the
// split-step Crank-Nicolson method (arXiv 2105.10517, program summary "Solution
// method"; Supplementary Material Eqs. S.1-S.6).
//
// A handle created with precision GP_FP32_MIXED propagates a complex64 copy of
// psi (float2 storage and sweeps; coefficient tables computed in FP64, norms
// summed in FP64) until gp_refine_fp64 widens it to complex128 and continues in
// FP64.  State input/output and observables always go through the complex128
// buffer (widening float -> double is exact).
#include "../../include/gpspin.h"
#include "gp_internal.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>

using namespace gpspin;

#include "gp_handle.cuh"

namespace gpspin {

static bool is_finite(double v) { return std::isfinite(v); }

// Failure injection for the allocator: while armed with n >= 0, the n-th device
// allocation from then on (0: the next one) fails as if the device were full,
// once; -1 is disarmed.
static std::atomic<long long> g_fail_after{-1};

int dev_alloc(void** p, size_t bytes)
{
    *p = nullptr;
    long long n = g_fail_after.load();
    while (n >= 0 && !g_fail_after.compare_exchange_weak(n, n - 1)) {
    }
    if (n == 0) return GP_ERR_OOM;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();  // an out-of-memory error is not sticky: clear it
        *p = nullptr;
        return GP_ERR_OOM;
    }
    return GP_OK;
}

int validate(const gp_params* p)
{
    if (!p) return GP_ERR_ARG;
    if (p->nx < 4 || p->ny < 4) return GP_ERR_ARG;
    if (!(p->xlen > 0) || !(p->ylen > 0) || !(p->dt > 0) || !is_finite(p->xlen) || !is_finite(p->ylen) ||
        !is_finite(p->dt))
        return GP_ERR_ARG;
    const double v[] = {p->wx, p->wy, p->c0, p->c2, p->omeg, p->gamma, p->rabi};
    for (double x : v)
        if (!is_finite(x)) return GP_ERR_ARG;
    if (p->so_type < 0 || p->so_type > 2) return GP_ERR_ARG;
    if (p->precision != GP_FP64 && p->precision != GP_FP32_MIXED) return GP_ERR_ARG;
    return GP_OK;
}

int eta_of(const gp_params& p) { return p.so_type == GP_SO_RASHBA ? 1 : (p.so_type == GP_SO_DRESSELHAUS ? -1 : 0); }
double gamma_of(const gp_params& p) { return p.so_type == GP_SO_NONE ? 0.0 : p.gamma; }

// Largest |c'_inf| over the lines and channels of one direction: the modulus of
// the smaller root of alpha z^2 - beta z + gamma' = 0 (the fixed point of the
// Thomas recurrence c'_k = gamma' / (beta - alpha c'_{k-1})).  It fixes how many
// elements a chunk carry influences above rounding.
double max_cp(const gp_params& p, int dir, int mode)
{
    typedef std::complex<double> cd;
    const int nlines = dir == 0 ? p.ny : p.nx;
    const double h = dir == 0 ? p.xlen / p.nx : p.ylen / p.ny;
    const double len = dir == 0 ? p.ylen : p.xlen, lh = dir == 0 ? p.ylen / p.ny : p.xlen / p.nx;
    const cd tau = mode == GP_REAL ? cd(0, 0.5 * p.dt) : cd(0.5 * p.dt, 0);
    double best = 0;
    for (int line = 0; line < nlines; ++line) {
        double pos = -0.5 * len + (line + 0.5) * lh;
        for (int ch = 0; ch < 3; ++ch) {
            double lam = 1.0 - ch;
            double kb = dir == 0 ? gamma_of(p) * lam - p.omeg * pos : p.omeg * pos - eta_of(p) * gamma_of(p) * lam;
            cd a(-0.5 / (h * h), -kb / (2 * h)), c(-0.5 / (h * h), kb / (2 * h));
            cd alpha = tau * a, gam = tau * c, beta = 1.0 + tau / (h * h);
            cd disc = std::sqrt(beta * beta - 4.0 * alpha * gam);
            cd z1 = (beta - disc) / (2.0 * alpha), z2 = (beta + disc) / (2.0 * alpha);
            double r = std::min(std::abs(z1), std::abs(z2));
            if (r > best) best = r;
        }
    }
    return best;
}

// Chunk length m, fixup length F and lines per CTA for lines of length L:
// F makes |c'_inf|^F <= 2^-60 (complex128) or 2^-26 (complex64); m >= H + F
// with H the rows until the factorisation has converged (contraction |c'|^2
// per row); R lines per CTA within ~100 KB of shared memory (two CTAs per SM)
// and 512 threads.
// Bank conflicts of the solve's chunk-parallel shared-memory accesses: thread
// tid = ql * nl3 + lc accesses element lc * Lp + ql * cs + t in units of `unit`
// elements (one access), and the threads of each group of G accesses served by
// one 128-byte wavefront should fall on distinct banks, i.e. their offsets in
// units differ modulo G.  Returns the extra wavefronts.
static int solve_conflicts(int cs, int Lp, int nl3, int Qc, int G, int unit)
{
    const int n = nl3 * Qc;
    int extra = 0;
    for (int g0 = 0; g0 < n; g0 += G) {
        int cnt[16] = {0}, mx = 0;
        for (int tid = g0; tid < std::min(n, g0 + G); ++tid) {
            const int ql = tid / nl3, lc = tid - ql * nl3;
            mx = std::max(mx, ++cnt[((lc * Lp + ql * cs) / unit) % G]);
        }
        extra += mx - 1;
    }
    return extra;
}

int make_tiling(int L, int nlines, double cpmax, int kind, int S, int R, int m_req, LineTiling* t, int compact)
{
    if (!(cpmax < 0.5)) return GP_ERR_UNSUPPORTED;
    if (S < 1 || S > 8 || (S & (S - 1)) || R < 1) return GP_ERR_ARG;  // portable cluster sizes
    if (kind < TILE_C128 || kind > TILE_C128_REG) return GP_ERR_ARG;
    const bool c64 = kind == TILE_C64 || kind == TILE_C64_REG;
    const double bits = c64 ? 26.0 : 60.0;
    const size_t elem = c64 ? sizeof(float2) : sizeof(double2);
    int F = cpmax > 0 ? (int)std::ceil(bits * std::log(2.0) / -std::log(cpmax)) + 1 : 1;
    int H = (F + 1) / 2 + 2;
    if (F > kFix || H > kHead) return GP_ERR_UNSUPPORTED;
    int m = std::max(std::max(16, H + F), m_req);
    m = (m + 3) / 4 * 4;
    if (kind == TILE_C64_REG && m <= 32) m = m <= 16 ? 16 : (m <= 24 ? 24 : 32);
    if (kind == TILE_C128_REG) {
        if (m > 32) return GP_ERR_UNSUPPORTED;  // compiled for m = 32 only
        m = 32;
    }
    const bool single = (kind == TILE_C64_REG && m <= 32) || kind == TILE_C128_REG;
    int Q = (L + m - 1) / m;
    if (S > 1 && Q < 2 * S) return GP_ERR_ARG;  // at least two chunks per CTA
    const int Qc = (Q + S - 1) / S;
    if (3 * R * Qc > 512 || R > nlines) return GP_ERR_ARG;
    // strides: fewest bank conflicts, then least shared memory.  With one line
    // array the chunks are staged in place by 16-byte bulk copies and the solve
    // moves two complex64 per access: even strides, conflicts counted per
    // 16-byte access (8 per wavefront).
    const int unit = single && c64 ? 2 : 1;
    const int G = single ? 8 : (c64 ? 16 : 8);
    int cs = m, Lp = Qc * m, best = -1;
    for (int dc = 0; dc < (compact ? 1 : G * unit); dc += unit)
        for (int dl = 0; dl < G * unit; dl += unit) {
            const int c = m + dc, l = Qc * c + dl;
            const int k = solve_conflicts(c, l, 3 * R, Qc, G, unit);
            if (best < 0 || k < best || (k == best && l < Lp)) {
                best = k;
                cs = c;
                Lp = l;
            }
        }
    auto up = [](size_t b) { return (b + 127) / 128 * 128; };
    const size_t line_bytes = up(3 * R * Lp * elem);
    // carries: cf, cb (3R Qc each) and, after cb, the two 3R-slot halos that
    // the cluster neighbours push into (register-resident solve)
    const size_t smem = line_bytes * (single ? 1 : 2) + 2 * up(3 * R * Qc * elem) + up(2 * 3 * R * elem);
    if (smem > 227 * 1024) return GP_ERR_UNSUPPORTED;
    // the complex128 register-resident kernels are compiled for at most 384 threads
    if (kind == TILE_C128_REG && 3 * R * Qc > 384) return GP_ERR_ARG;
    t->L = L;
    t->nlines = nlines;
    t->R = R;
    t->m = m;
    t->Q = Q;
    t->S = S;
    t->Qc = Qc;
    t->F = std::min(F, m - 1);
    t->cs = cs;
    t->Lp = Lp;
    t->threads = std::min(512, (std::max(32, 3 * R * Qc) + 31) / 32 * 32);
    t->smem = smem;
    t->off_b = single ? 0 : line_bytes;
    t->off_cf = line_bytes * (single ? 1 : 2);
    t->off_cb = t->off_cf + up(3 * R * Qc * elem);
    t->bulk = 0;  // set per pass by the caller (needs 16-byte aligned rows)
    t->single = single ? 1 : 0;
    return GP_OK;
}

// Default tiling: the minimum chunk length, lines per CTA within ~100 KB of
// shared memory and 256 threads, and long lines (>= 256 points) split over a
// 2-CTA cluster (twice the work units for the SMs, half the shared memory per CTA).
int choose_tiling(int L, int nlines, double cpmax, LineTiling* t, int kind, int split)
{
    LineTiling base;
    int st = make_tiling(L, nlines, cpmax, kind, 1, 1, 0, &base);
    if (st) return st;
    int m = base.m, Q = base.Q;
    while (3 * Q > 512) {  // keep one thread per chunk within a CTA
        m += 4;
        Q = (L + m - 1) / m;
    }
    const int S = (split && L >= 256 && Q >= 8) ? 2 : 1;
    const int Qc = (Q + S - 1) / S;
    int R = std::max(1, 256 / (3 * Qc));
    if (kind != TILE_C128 && S == 1) R = std::max(R, 4);  // >= 32-byte segments in the transposed store
    if (S > 1) R = 1;
    R = std::min(R, nlines);
    for (; R >= 1; --R) {
        if (make_tiling(L, nlines, cpmax, kind, S, R, m, t) == GP_OK && (R == 1 || t->smem <= 100 * 1024)) return GP_OK;
    }
    return GP_ERR_UNSUPPORTED;
}

#define CK(x)                                                  \
    do {                                                       \
        if (report_cuda((x), #x) != 0) return GP_ERR_CUDA;     \
    } while (0)
#define LK(x)                                                  \
    do {                                                       \
        if ((x) != 0) return GP_ERR_CUDA;                      \
    } while (0)

void drop_graphs(gp_handle* h)
{
    for (auto& row : h->graph)
        for (auto& g : row)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
}

void free_coef(CoefSet& c)
{
    cudaFree(c.cx);
    cudaFree(c.cy);
    cudaFree(c.ex);
    cudaFree(c.ey);
    cudaFree(c.fx);
    cudaFree(c.fy);
    cudaFree(c.fex);
    cudaFree(c.fey);
    cudaFree(c.cxh);
    cudaFree(c.exh);
    cudaFree(c.eyh);
    c = CoefSet{};
}

bool wants_fp32(const gp_handle* h) { return h->p.precision == GP_FP32_MIXED; }

bool same_physics(const gp_params& a, const gp_params& b)
{
    return a.dt == b.dt && a.wx == b.wx && a.wy == b.wy && a.omeg == b.omeg && a.so_type == b.so_type &&
           a.gamma == b.gamma && a.nx == b.nx && a.ny == b.ny && a.xlen == b.xlen && a.ylen == b.ylen;
}

int ensure_coef(gp_handle* h, int mode)
{
    CoefSet& cs = h->coef[mode];
    if (cs.valid && same_physics(cs.key, h->p)) return GP_OK;
    const gp_params& p = h->p;
    const bool f32 = wants_fp32(h);
    LineTiling tx, ty, ftx{}, fty{}, ux, uy, fux{}, fuy{};
    const double cx = max_cp(p, 0, mode), cy = max_cp(p, 1, mode);
    int st = choose_tiling(p.nx, p.ny, cx, &tx);
    if (st) return st;
    if ((st = choose_tiling(p.ny, p.nx, cy, &ty))) return st;
    if ((st = choose_tiling(p.nx, p.ny, cx, &ux, TILE_C128, 0))) return st;
    if ((st = choose_tiling(p.ny, p.nx, cy, &uy, TILE_C128, 0))) return st;
    if (f32) {
        if ((st = choose_tiling(p.nx, p.ny, cx, &ftx, TILE_C64_REG))) return st;
        if ((st = choose_tiling(p.ny, p.nx, cy, &fty, TILE_C64_REG))) return st;
        if ((st = choose_tiling(p.nx, p.ny, cx, &fux, TILE_C64_REG, 0))) return st;  // batched launches
        if ((st = choose_tiling(p.ny, p.nx, cy, &fuy, TILE_C64_REG, 0))) return st;
    }
    if (!cs.cx) {
        bool ok = dalloc(&cs.cx, sizeof(LineCoef) * 3 * (size_t)p.ny) &&
                  dalloc(&cs.cy, sizeof(LineCoef) * 3 * (size_t)p.nx) &&
                  dalloc(&cs.ex, sizeof(double2) * p.nx) &&
                  dalloc(&cs.ey, sizeof(double2) * p.ny);
        if (ok && f32)
            ok = dalloc(&cs.fx, sizeof(LineCoefF) * 3 * (size_t)p.ny) &&
                 dalloc(&cs.fy, sizeof(LineCoefF) * 3 * (size_t)p.nx) &&
                 dalloc(&cs.fex, sizeof(float2) * p.nx) &&
                 dalloc(&cs.fey, sizeof(float2) * p.ny);
        if (!ok) {
            free_coef(cs);
            return GP_ERR_OOM;
        }
    }
    drop_graphs(h);
    cs.half_valid = false;
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
    const double dx = p.xlen / p.nx, dy = p.ylen / p.ny;
    const double g = gamma_of(p);
    const int eta = eta_of(p);
    LK(launch_coef(cs.cx, p.ny, 0, mode, dx, p.ylen, dy, p.dt, p.omeg, g, eta, h->flag, h->stream));
    LK(launch_coef(cs.cy, p.nx, 1, mode, dy, p.xlen, dx, p.dt, p.omeg, g, eta, h->flag, h->stream));
    LK(launch_trap_table(cs.ex, p.nx, p.xlen, p.wx, p.dt, mode, h->stream));
    LK(launch_trap_table(cs.ey, p.ny, p.ylen, p.wy, p.dt, mode, h->stream));
    if (f32) {
        LK(launch_coef(cs.fx, p.ny, 0, mode, dx, p.ylen, dy, p.dt, p.omeg, g, eta, h->flag, h->stream));
        LK(launch_coef(cs.fy, p.nx, 1, mode, dy, p.xlen, dx, p.dt, p.omeg, g, eta, h->flag, h->stream));
        LK(launch_trap_table(cs.fex, p.nx, p.xlen, p.wx, p.dt, mode, h->stream));
        LK(launch_trap_table(cs.fey, p.ny, p.ylen, p.wy, p.dt, mode, h->stream));
    }
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (flag & 1) return GP_ERR_UNSUPPORTED;
    cs.tx = tx;
    cs.ty = ty;
    cs.ftx = ftx;
    cs.fty = fty;
    cs.ux = ux;
    cs.uy = uy;
    cs.fux = fux;
    cs.fuy = fuy;
    cs.key = p;
    cs.valid = true;
    return GP_OK;
}

template <typename C>
void fill_common(gp_handle* h, PassArgsT<C>& a)
{
    a.nx = h->p.nx;
    a.ny = h->p.ny;
    a.scale = h->scal;
    a.dt = h->p.dt;
    a.c0 = h->p.c0;
    a.c2 = h->p.c2;
    a.rabi = h->p.rabi;
    a.do_p = 1;
    a.do_solve = 1;
    a.err = h->flag;
    a.dx = h->p.xlen / h->p.nx;
    a.dy = h->p.ylen / h->p.ny;
    a.x0 = -0.5 * h->p.xlen + 0.5 * a.dx;
    a.y0 = -0.5 * h->p.ylen + 0.5 * a.dy;
    a.wx = h->p.wx;
    a.wy = h->p.wy;
    const double kf[10] = {a.dt * a.c0, a.dt * a.c2, a.dt * a.rabi * 0.70710678118654752440, a.dt, a.x0, a.dx, a.y0,
                           a.dy, 0.5 * a.dt * a.wx * a.wx, 0.5 * a.dt * a.wy * a.wy};
    for (int i = 0; i < 10; ++i) a.kf[i] = (float)kf[i];
}

// Rows can be staged with cp.async.bulk when every row starts on a 16-byte
// boundary and its size is a multiple of 16 bytes.
template <typename C>
void set_bulk(PassArgsT<C>& a, int dir, int nx, int ny)
{
    const int L = dir == 0 ? nx : ny;
    a.t.bulk = ((size_t)L * sizeof(C)) % 16 == 0 ? 1 : 0;
}

PassArgs pass_args(gp_handle* h, const CoefSet& cs, int dir)
{
    PassArgs a{};
    fill_common(h, a);
    a.ex = cs.ex;
    a.ey = cs.ey;
    if (dir == 0) {
        a.in = h->psi;
        a.out = h->work;
        a.coef = cs.cx;
        a.t = cs.tx;
    } else {
        a.in = h->work;
        a.out = h->psi;
        a.coef = cs.cy;
        a.t = cs.ty;
    }
    set_bulk(a, dir, h->p.nx, h->p.ny);
    return a;
}

PassArgsF pass_args_f32(gp_handle* h, const CoefSet& cs, int dir)
{
    PassArgsF a{};
    fill_common(h, a);
    a.ex = cs.fex;
    a.ey = cs.fey;
    if (dir == 0) {
        a.in = h->psi32;
        a.out = h->work32;
        a.coef = cs.fx;
        a.t = cs.ftx;
    } else {
        a.in = h->work32;
        a.out = h->psi32;
        a.coef = cs.fy;
        a.t = cs.fty;
    }
    set_bulk(a, dir, h->p.nx, h->p.ny);
    return a;
}

size_t n_elems(const gp_handle* h) { return 3 * (size_t)h->p.nx * h->p.ny; }
double cell(const gp_handle* h) { return (h->p.xlen / h->p.nx) * (h->p.ylen / h->p.ny); }

int norm_blocks(const gp_handle* h)
{
    size_t n = n_elems(h);
    size_t b = (n + 255) / 256;
    return (int)std::min<size_t>(std::max<size_t>(b, 1), 608);
}

// Makes the stored (active) state the true state (no pending normalisation).
int flush_scale(gp_handle* h)
{
    if (!h->scale_pending) return GP_OK;
    if (h->active == GP_FP32_MIXED) {
        LK(launch_apply_scale(h->psi32, n_elems(h), h->scal, h->stream));
    } else {
        LK(launch_apply_scale(h->psi, n_elems(h), h->scal, h->stream));
    }
    h->scale_pending = false;
    return GP_OK;
}

// The complex128 buffer psi mirrors the complex64 state (exact widening); the
// pending scale stays pending.
int widen_into_psi(gp_handle* h)
{
    if (h->active != GP_FP32_MIXED) return GP_OK;
    LK(launch_scaled_copy(h->psi, h->psi32, n_elems(h), h->scal + 2, h->stream));
    return GP_OK;
}

// After psi (complex128) was written from outside: refresh the complex64 copy.
int narrow_from_psi(gp_handle* h)
{
    if (h->active != GP_FP32_MIXED) return GP_OK;
    LK(launch_narrow(h->psi32, h->psi, n_elems(h), h->stream));
    return GP_OK;
}

int sync_status(gp_handle* h)
{
    CK(cudaStreamSynchronize(h->stream));
    return GP_OK;
}

int y_blocks(const LineTiling& t) { return (t.nlines + t.R - 1) / t.R * t.S; }

size_t handle_bytes(const gp_params& p)
{
    const size_t n = 3 * (size_t)p.nx * p.ny, lines = (size_t)p.nx + p.ny;
    size_t b = n * 2 * sizeof(double2);  // psi, work
    b += kNormBlocksMax * sizeof(double) + (size_t)obs_blocks(p.nx, p.ny) * obs_slots() * sizeof(double);
    b += 3 * lines * sizeof(LineCoef) + lines * sizeof(double2);  // tables of one mode
    if (p.precision == GP_FP32_MIXED) b += n * 2 * sizeof(float2) + 3 * lines * sizeof(LineCoefF) + lines * sizeof(float2);
    return b + 4096;  // scalars, flag and allocation rounding
}

// Launch sequence of n steps (x-pass, y-pass and, in imaginary time, the
// normalisation) on the handle's stream.
template <typename C>
int apply_sigma(gp_handle* h, const PassArgsT<C>& ay)
{
    return launch_apply_comp_scale(ay.out, (size_t)h->p.nx * h->p.ny, h->scal + 3, h->stream);
}

template <typename A>
int enqueue_steps(gp_handle* h, int mode, const A& ax, const A& ay, int gy, long long n)
{
    // debug: every byte a pass must write is first set to 0xFF (a NaN in both
    // precisions), so an element a pass skipped reaches the state as a NaN
    const bool poison = h->debug & GP_DEBUG_POISON;
    const size_t bytes = n_elems(h) * sizeof(*ax.out);
    for (long long s = 0; s < n; ++s) {
        if (poison) CK(cudaMemsetAsync(ax.out, 0xFF, bytes, h->stream));
        LK(launch_xpass(ax, mode, h->stream));
        if (poison) CK(cudaMemsetAsync(ay.out, 0xFF, bytes, h->stream));  // psi: read by the x-pass, not yet rewritten
        LK(launch_ypass(ay, mode, h->stream));
        if (mode == GP_IMAG && h->mcon) {
            // magnetisation-constrained normalisation, applied at once
            LK(launch_finalize_m(h->partials, gy, cell(h), h->m_target, h->scal + 3, h->flag, h->stream));
            LK(apply_sigma(h, ay));
        } else if (mode == GP_IMAG) {
            LK(launch_finalize_norm(h->partials, gy, cell(h), h->scal, h->flag, h->stream));
        }
    }
    return GP_OK;
}

// Runs n steps: whole blocks of kGraphSteps steps replay one captured CUDA
// graph (captured on first use, dropped when parameters or tables change); the
// remainder is launched directly.  If capture is not possible on this stream the
// steps are launched directly.
constexpr int kGraphSteps = 16;

template <typename A>
int run_steps(gp_handle* h, int mode, const A& ax, const A& ay, int gy, long long n)
{
    cudaGraphExec_t& ge = h->graph[h->active == GP_FP32_MIXED ? 1 : 0][mode];
    if (n >= kGraphSteps && !ge) {
        // one direct step first: it sets the kernels' shared-memory attributes
        int st = enqueue_steps(h, mode, ax, ay, gy, 1);
        if (st) return st;
        --n;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            int cst = enqueue_steps(h, mode, ax, ay, gy, kGraphSteps);
            cudaError_t e = cudaStreamEndCapture(h->stream, &g);
            if (cst == GP_OK && e == cudaSuccess && g) {
                if (cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) ge = nullptr;
            }
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();  // a failed capture only means direct launches
    }
    if (ge) {
        for (; n >= kGraphSteps; n -= kGraphSteps) CK(cudaGraphLaunch(ge, h->stream));
    }
    return enqueue_steps(h, mode, ax, ay, gy, n);
}

}  // namespace gpspin

namespace {

// Second-order (Strang) steps, complex128: per step
//   x-pass    P(dt/2) then X(dt/2), with the pending normalisation  (dt/2 tables)
//   y-pass    Y(dt)                                                 (dt tables)
//   tail      X(dt/2), then P(dt/2), natural-layout store, partial norms
//   [imaginary time: norm finalize; the scale is applied by the next x-pass]
// The x tables of dt/2 are tabulated beside the dt ones; the tiling of the dt
// tables serves them (their fixups reach fewer rows).
int ensure_half(gp_handle* h, int mode)
{
    CoefSet& cs = h->coef[mode];
    if (cs.half_valid) return GP_OK;
    const gp_params& p = h->p;
    if (!cs.cxh) {
        bool ok = dalloc(&cs.cxh, sizeof(LineCoef) * 3 * (size_t)p.ny) &&
                  dalloc(&cs.exh, sizeof(double2) * p.nx) &&
                  dalloc(&cs.eyh, sizeof(double2) * p.ny);
        if (!ok) return GP_ERR_OOM;
    }
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
    const double dx = p.xlen / p.nx, dy = p.ylen / p.ny, hdt = 0.5 * p.dt;
    LK(launch_coef(cs.cxh, p.ny, 0, mode, dx, p.ylen, dy, hdt, p.omeg, gamma_of(p), eta_of(p), h->flag, h->stream));
    LK(launch_trap_table(cs.exh, p.nx, p.xlen, p.wx, hdt, mode, h->stream));
    LK(launch_trap_table(cs.eyh, p.ny, p.ylen, p.wy, hdt, mode, h->stream));
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (flag & 1) return GP_ERR_UNSUPPORTED;
    cs.half_valid = true;
    return GP_OK;
}

// Pass arguments of a second-order step: x-pass with the dt/2 tables, y-pass
// (no partials), tail in place on psi with nothing pending (partials in
// imaginary time).  Returns the tail's CTA count through gx.
int strang_args(gp_handle* h, int mode, PassArgs* ax, PassArgs* ay, PassArgs* at, int* gx)
{
    if (h->active != GP_FP64 || h->mcon) return GP_ERR_UNSUPPORTED;
    int st = ensure_coef(h, mode);
    if (st || (st = ensure_half(h, mode))) return st;
    const CoefSet& cs = h->coef[mode];
    *gx = y_blocks(cs.tx);
    if (*gx > kNormBlocksMax) return GP_ERR_UNSUPPORTED;
    if (mode == GP_REAL && (st = flush_scale(h))) return st;
    *ax = pass_args(h, cs, 0);
    *ay = pass_args(h, cs, 1);
    ax->coef = cs.cxh;
    ax->ex = cs.exh;
    ax->ey = cs.eyh;
    ax->dt = 0.5 * h->p.dt;
    *at = *ax;
    at->in = h->psi;
    at->out = h->psi;
    at->do_p = 0;
    at->scale = h->scal + 2;
    at->partials = mode == GP_IMAG ? h->partials : nullptr;
    ay->partials = nullptr;
    return GP_OK;
}

int propagate_strang(gp_handle* h, long long nsteps, int mode)
{
    PassArgs ax, ay, at;
    int gx = 0;
    int st = strang_args(h, mode, &ax, &ay, &at, &gx);
    if (st) return st;
    for (long long k = 0; k < nsteps; ++k) {
        LK(launch_xpass(ax, mode, h->stream));
        LK(launch_ypass(ay, mode, h->stream));
        LK(launch_xtail(at, mode, h->stream));
        if (mode == GP_IMAG) LK(launch_finalize_norm(h->partials, gx, cell(h), h->scal, h->flag, h->stream));
    }
    if (mode == GP_IMAG) h->scale_pending = true;
    h->steps += nsteps;
    return GP_OK;
}

int propagate_active(gp_handle* h, long long nsteps, int mode)
{
    if (h->split == GP_SPLIT_STRANG) return propagate_strang(h, nsteps, mode);
    int st = ensure_coef(h, mode);
    if (st) return st;
    const CoefSet& cs = h->coef[mode];
    if (mode == GP_REAL && (st = flush_scale(h))) return st;
    const bool f32 = h->active == GP_FP32_MIXED;
    const int gy = y_blocks(f32 ? cs.fty : cs.ty);
    const bool mc = mode == GP_IMAG && h->mcon;
    if (gy * (mc ? 3 : 1) > kNormBlocksMax) return GP_ERR_UNSUPPORTED;
    if (mc) {
        if (gamma_of(h->p) != 0.0 || h->p.rabi != 0.0) return GP_ERR_ARG;  // m is not conserved there
        if ((st = flush_scale(h))) return st;
    }
    if (f32) {
        PassArgsF ax = pass_args_f32(h, cs, 0), ay = pass_args_f32(h, cs, 1);
        if (mode == GP_IMAG) ay.partials = h->partials;
        ay.mcomp = mc;
        st = run_steps(h, mode, ax, ay, gy, nsteps);
    } else {
        PassArgs ax = pass_args(h, cs, 0), ay = pass_args(h, cs, 1);
        if (mode == GP_IMAG) ay.partials = h->partials;
        ay.mcomp = mc;
        st = run_steps(h, mode, ax, ay, gy, nsteps);
    }
    if (st) return st;
    if (mode == GP_IMAG && !mc) h->scale_pending = true;
    h->steps += nsteps;
    return GP_OK;
}

}  // namespace

extern "C" {

const char* gp_strerror(int s)
{
    switch (s) {
    case GP_OK: return "ok";
    case GP_ERR_ARG: return "invalid argument";
    case GP_ERR_OOM: return "device allocation failed";
    case GP_ERR_CUDA: return "CUDA runtime error";
    case GP_ERR_NONFINITE: return "non-finite values in the wave function";
    case GP_ERR_UNSUPPORTED: return "parameters outside the supported range of the tabulated line solver";
    case GP_ERR_TOO_LARGE: return "grid larger than the fixed scratch of gp_propagate_noalloc (nx, ny <= 256)";
    case GP_ERR_TIMEOUT: return "a device-side wait gave up (bulk copy did not complete)";
    case GP_ERR_QUEUE_FULL: return "the batch's queue limit is reached";
    default: return "unknown status";
    }
}

int gp_create(const gp_params* params, void* cuda_stream, gp_handle** out)
{
    if (!out) return GP_ERR_ARG;
    *out = nullptr;
    int st = validate(params);
    if (st) return st;
    gp_handle* h = new (std::nothrow) gp_handle();
    if (!h) return GP_ERR_OOM;
    h->p = *params;
    h->active = params->precision;
    cudaGetDevice(&h->device);
    if (cuda_stream) {
        h->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return GP_ERR_CUDA;
        }
        h->own_stream = true;
    }
    size_t n = n_elems(h);
    bool ok = dalloc(&h->psi, n * sizeof(double2)) &&
              dalloc(&h->work, n * sizeof(double2)) &&
              dalloc(&h->partials, kNormBlocksMax * sizeof(double)) &&
              dalloc(&h->obs_part, (size_t)obs_blocks(h->p.nx, h->p.ny) * obs_slots() * sizeof(double)) &&
              dalloc(&h->scal, 6 * sizeof(double)) &&
              dalloc(&h->obs_out, 8 * sizeof(double)) &&
              dalloc(&h->flag, sizeof(int));
    if (ok && wants_fp32(h))
        ok = dalloc(&h->psi32, n * sizeof(float2)) &&
             dalloc(&h->work32, n * sizeof(float2));
    if (!ok) {
        gp_destroy(h);
        return GP_ERR_OOM;
    }
    if (cudaMemsetAsync(h->psi, 0, n * sizeof(double2), h->stream) != cudaSuccess ||
        (h->psi32 && cudaMemsetAsync(h->psi32, 0, n * sizeof(float2), h->stream) != cudaSuccess) ||
        launch_set_scalar(h->scal, 1.0, h->stream) != 0 || launch_set_scalar(h->scal + 2, 1.0, h->stream) != 0 ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        gp_destroy(h);
        return GP_ERR_CUDA;
    }
    *out = h;
    return GP_OK;
}

void gp_destroy(gp_handle* h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto& c : h->coef) free_coef(c);
    drop_graphs(h);
    cudaFree(h->psi);
    cudaFree(h->work);
    cudaFree(h->psi32);
    cudaFree(h->work32);
    cudaFree(h->partials);
    cudaFree(h->obs_part);
    cudaFree(h->scal);
    cudaFree(h->obs_out);
    cudaFree(h->flag);
    for (auto& e : h->ev)
        if (e) cudaEventDestroy(e);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
}

int gp_set_params(gp_handle* h, const gp_params* params)
{
    if (!h) return GP_ERR_ARG;
    int st = validate(params);
    if (st) return st;
    if (params->nx != h->p.nx || params->ny != h->p.ny || params->xlen != h->p.xlen || params->ylen != h->p.ylen ||
        params->precision != h->p.precision)
        return GP_ERR_ARG;
    h->p = *params;
    drop_graphs(h);  // the captured launches hold c0, c2, R and dt by value
    return GP_OK;
}

int gp_set_splitting(gp_handle* h, int split)
{
    if (!h || (split != GP_SPLIT_LIE && split != GP_SPLIT_STRANG)) return GP_ERR_ARG;
    if (split == GP_SPLIT_STRANG && (h->p.precision != GP_FP64 || h->mcon)) return GP_ERR_UNSUPPORTED;
    h->split = split;
    drop_graphs(h);
    return GP_OK;
}

int gp_set_magnetization(gp_handle* h, int enable, double m)
{
    if (!h || !(std::isfinite(m)) || !(m > -1.0 && m < 1.0)) return GP_ERR_ARG;
    if (enable && (gamma_of(h->p) != 0.0 || h->p.rabi != 0.0)) return GP_ERR_ARG;
    h->mcon = enable ? 1 : 0;
    h->m_target = m;
    drop_graphs(h);  // the captured step sequence depends on the normalisation
    return GP_OK;
}

int gp_set_state(gp_handle* h, const double* psi_host, int normalize)
{
    if (!h || !psi_host) return GP_ERR_ARG;
    CK(cudaMemcpyAsync(h->psi, psi_host, n_elems(h) * sizeof(double2), cudaMemcpyHostToDevice, h->stream));
    LK(launch_set_scalar(h->scal, 1.0, h->stream));
    LK(narrow_from_psi(h));
    h->scale_pending = false;
    if (normalize) {
        CK(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
        LK(launch_norm(h->psi, n_elems(h), h->partials, norm_blocks(h), cell(h), h->scal, h->flag, h->stream));
        h->scale_pending = true;
        int flag = 0;
        CK(cudaMemcpyAsync(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        if (flag & 2) return GP_ERR_NONFINITE;
    }
    return sync_status(h);
}

int gp_get_state(gp_handle* h, double* psi_out)
{
    if (!h || !psi_out) return GP_ERR_ARG;
    if (h->active == GP_FP32_MIXED) {
        LK(launch_scaled_copy(h->work, h->psi32, n_elems(h), h->scal, h->stream));
    } else {
        LK(launch_scaled_copy(h->work, h->psi, n_elems(h), h->scal, h->stream));
    }
    CK(cudaMemcpyAsync(psi_out, h->work, n_elems(h) * sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
    return sync_status(h);
}

int gp_init_winding(gp_handle* h, const double frac[3], const int winding[3], unsigned long long seed,
                    double phase_noise)
{
    if (!h || !frac || !winding || !is_finite(phase_noise)) return GP_ERR_ARG;
    for (int c = 0; c < 3; ++c) {
        if (!(frac[c] >= 0) || !is_finite(frac[c])) return GP_ERR_ARG;
        if (winding[c] < -8 || winding[c] > 8) return GP_ERR_ARG;
    }
    LK(launch_init_gaussian(h->psi, h->p.nx, h->p.ny, h->p.xlen, h->p.ylen, frac, winding, seed, phase_noise,
                            h->stream));
    LK(narrow_from_psi(h));
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
    LK(launch_norm(h->psi, n_elems(h), h->partials, norm_blocks(h), cell(h), h->scal, h->flag, h->stream));
    h->scale_pending = true;
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return (flag & 2) ? GP_ERR_NONFINITE : GP_OK;
}

int gp_init_gaussian(gp_handle* h, const double frac[3], unsigned long long seed, double phase_noise)
{
    const int none[3] = {0, 0, 0};
    return gp_init_winding(h, frac, none, seed, phase_noise);
}

// Status bits the kernels of a propagation set: a bulk-copy wait that gave up
// (bit 8) or a non-finite norm (bit 2).
static int check_flags(gp_handle* h)
{
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (flag & 8) return GP_ERR_TIMEOUT;
    if (flag & 2) return GP_ERR_NONFINITE;
    return GP_OK;
}

int gp_propagate(gp_handle* h, long long nsteps, int mode)
{
    gpspin::TraceRange trace("gp_propagate");
    if (!h || nsteps < 0 || (mode != GP_IMAG && mode != GP_REAL)) return GP_ERR_ARG;
    if (nsteps == 0) return GP_OK;
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
    int st = propagate_active(h, nsteps, mode);
    if (st) return st;
    return check_flags(h);
}

int gp_refine_fp64(gp_handle* h, long long nsteps, int mode)
{
    gpspin::TraceRange trace("gp_refine_fp64");
    if (!h || nsteps < 0 || (mode != GP_IMAG && mode != GP_REAL)) return GP_ERR_ARG;
    if (h->active == GP_FP32_MIXED) {
        // widen the complex64 state (the pending scale stays pending)
        LK(widen_into_psi(h));
        h->active = GP_FP64;
    }
    if (nsteps == 0) return sync_status(h);
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
    int st = propagate_active(h, nsteps, mode);
    if (st) return st;
    return check_flags(h);
}

// Device address through which kernels can read or write the host buffer p
// (16-byte aligned, complex128): pinned memory through its mapping, pageable
// memory where the device reaches it through the host page tables.  nullptr if
// neither holds: the caller then copies with cudaMemcpyAsync.
static double2* device_view(const double* p)
{
    if (reinterpret_cast<uintptr_t>(p) % 16) return nullptr;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type == cudaMemoryTypeHost) return static_cast<double2*>(at.devicePointer);
    if (at.type != cudaMemoryTypeUnregistered) return nullptr;
    int dev = 0, pageable = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return pageable ? reinterpret_cast<double2*>(const_cast<double*>(p)) : nullptr;
}

int gp_propagate_host(gp_handle* h, const double* psi_in, long long nsteps, int mode, double* psi_out)
{
    gpspin::TraceRange trace("gp_propagate_host");
    if (!h || !psi_in || !psi_out || nsteps < 0 || (mode != GP_IMAG && mode != GP_REAL)) return GP_ERR_ARG;
    const double2* din = device_view(psi_in);
    double2* dout = device_view(psi_out);
    const bool mc = mode == GP_IMAG && h->mcon;
    if (!din || h->active != GP_FP64 || nsteps == 0 || h->split != GP_SPLIT_LIE) {
        int st = gp_set_state(h, psi_in, 0);
        if (st == GP_OK) st = gp_propagate(h, nsteps, mode);
        return st == GP_OK ? gp_get_state(h, psi_out) : st;
    }
    // the state of gp_set_state(h, psi_in, 0): nothing pending
    LK(launch_set_scalar(h->scal, 1.0, h->stream));
    h->scale_pending = false;
    int st = ensure_coef(h, mode);
    if (st) return st;
    const CoefSet& cs = h->coef[mode];
    const int gy = y_blocks(cs.ty);
    if (gy * (mc ? 3 : 1) > kNormBlocksMax) return GP_ERR_UNSUPPORTED;
    if (mc && (gamma_of(h->p) != 0.0 || h->p.rabi != 0.0)) return GP_ERR_ARG;
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
    // first step: the x-pass loads the host state directly (plain loads; bulk
    // copies are kept for device memory), overlapping the transfer with its work
    PassArgs ax = pass_args(h, cs, 0), ay = pass_args(h, cs, 1);
    ax.in = din;
    ax.t.bulk = 0;
    if (mode == GP_IMAG) ay.partials = h->partials;
    ay.mcomp = mc;
    if ((st = enqueue_steps(h, mode, ax, ay, gy, 1))) return st;
    if (mode == GP_IMAG && !mc) h->scale_pending = true;
    h->steps += 1;
    if (nsteps > 1 && (st = propagate_active(h, nsteps - 1, mode))) return st;
    if ((st = check_flags(h))) return st;
    if (!dout) return gp_get_state(h, psi_out);
    // the normalised result is written straight into the caller's buffer
    LK(launch_scaled_copy(dout, h->psi, n_elems(h), h->scal, h->stream));
    return sync_status(h);
}

int gp_profile_step(gp_handle* h, int mode, float* ms_out)
{
    if (!h || !ms_out || (mode != GP_IMAG && mode != GP_REAL)) return GP_ERR_ARG;
    for (auto& e : h->ev)
        if (!e) CK(cudaEventCreate(&e));
    float t[4] = {0, 0, 0, 0};
    if (h->split == GP_SPLIT_STRANG) {
        // x-pass (dt/2), y-pass, closing x-pass, normalisation
        PassArgs ax, ay, at;
        int gx = 0;
        int st = strang_args(h, mode, &ax, &ay, &at, &gx);
        if (st) return st;
        CK(cudaEventRecord(h->ev[0], h->stream));
        LK(launch_xpass(ax, mode, h->stream));
        CK(cudaEventRecord(h->ev[1], h->stream));
        LK(launch_ypass(ay, mode, h->stream));
        CK(cudaEventRecord(h->ev[2], h->stream));
        LK(launch_xtail(at, mode, h->stream));
        CK(cudaEventRecord(h->ev[3], h->stream));
        if (mode == GP_IMAG) {
            LK(launch_finalize_norm(h->partials, gx, cell(h), h->scal, h->flag, h->stream));
            h->scale_pending = true;
        }
    } else {
        int st = ensure_coef(h, mode);
        if (st) return st;
        const CoefSet& cs = h->coef[mode];
        const bool mc = mode == GP_IMAG && h->mcon;
        if (mc && (gamma_of(h->p) != 0.0 || h->p.rabi != 0.0)) return GP_ERR_ARG;
        if ((mode == GP_REAL || mc) && (st = flush_scale(h))) return st;
        const bool f32 = h->active == GP_FP32_MIXED;
        const int gy = y_blocks(f32 ? cs.fty : cs.ty);
        if (gy * (mc ? 3 : 1) > kNormBlocksMax) return GP_ERR_UNSUPPORTED;
        CK(cudaEventRecord(h->ev[0], h->stream));
        if (f32) {
            PassArgsF ax = pass_args_f32(h, cs, 0), ay = pass_args_f32(h, cs, 1);
            if (mode == GP_IMAG) ay.partials = h->partials;
            ay.mcomp = mc;
            LK(launch_xpass(ax, mode, h->stream));
            CK(cudaEventRecord(h->ev[1], h->stream));
            LK(launch_ypass(ay, mode, h->stream));
            CK(cudaEventRecord(h->ev[2], h->stream));
            CK(cudaEventRecord(h->ev[3], h->stream));
            if (mc) {
                LK(launch_finalize_m(h->partials, gy, cell(h), h->m_target, h->scal + 3, h->flag, h->stream));
                LK(apply_sigma(h, ay));
            }
        } else {
            PassArgs ax = pass_args(h, cs, 0), ay = pass_args(h, cs, 1);
            if (mode == GP_IMAG) ay.partials = h->partials;
            ay.mcomp = mc;
            LK(launch_xpass(ax, mode, h->stream));
            CK(cudaEventRecord(h->ev[1], h->stream));
            LK(launch_ypass(ay, mode, h->stream));
            CK(cudaEventRecord(h->ev[2], h->stream));
            CK(cudaEventRecord(h->ev[3], h->stream));
            if (mc) {
                LK(launch_finalize_m(h->partials, gy, cell(h), h->m_target, h->scal + 3, h->flag, h->stream));
                LK(apply_sigma(h, ay));
            }
        }
        if (mode == GP_IMAG && !mc) {
            LK(launch_finalize_norm(h->partials, gy, cell(h), h->scal, h->flag, h->stream));
            h->scale_pending = true;
        }
    }
    CK(cudaEventRecord(h->ev[4], h->stream));
    CK(cudaEventSynchronize(h->ev[4]));
    CK(cudaEventElapsedTime(&t[0], h->ev[0], h->ev[1]));
    CK(cudaEventElapsedTime(&t[1], h->ev[1], h->ev[2]));
    CK(cudaEventElapsedTime(&t[2], h->ev[2], h->ev[3]));
    CK(cudaEventElapsedTime(&t[3], h->ev[3], h->ev[4]));
    ms_out[0] = t[0] + t[2];  // x-passes (the closing one of a second-order step included)
    ms_out[1] = t[1];
    ms_out[2] = t[3];
    CK(cudaEventElapsedTime(&ms_out[3], h->ev[0], h->ev[4]));
    h->steps += 1;
    return GP_OK;
}

extern "C++" {
// Times one pass (x: dir 0, y: dir 1) with the given tiling: the median of five
// launches after one warm-up, on the handle's stream, in ms (negative if a
// launch fails).  The median, not the minimum: candidates within a few percent
// of each other would otherwise be ranked by their luckiest launch.  With a
// flush buffer each timed launch starts from a cold L2 (the buffer, larger than
// L2, is written first), as in a step whose input has left the cache.
template <typename A>
float time_pass(gp_handle* h, A a, int dir, int mode, void* flush, size_t flush_bytes)
{
    a.partials = nullptr;
    constexpr int kTimed = 5;
    float t[kTimed];
    for (int rep = 0; rep <= kTimed; ++rep) {
        if (flush && cudaMemsetAsync(flush, rep, flush_bytes, h->stream) != cudaSuccess) return -1.0f;
        if (cudaEventRecord(h->ev[0], h->stream) != cudaSuccess) return -1.0f;
        int rc = dir == 0 ? launch_xpass(a, mode, h->stream) : launch_ypass(a, mode, h->stream);
        if (rc || cudaEventRecord(h->ev[1], h->stream) != cudaSuccess || cudaEventSynchronize(h->ev[1]) != cudaSuccess)
            return -1.0f;
        float ms = 0;
        cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
        if (rep > 0) t[rep - 1] = ms;  // the first launch warms up
    }
    std::sort(t, t + kTimed);
    return t[kTimed / 2];
}

}  // extern "C++"

int gp_autotune(gp_handle* h, int mode, double* ms_out)
{
    gpspin::TraceRange trace("gp_autotune");
    if (!h || (mode != GP_IMAG && mode != GP_REAL)) return GP_ERR_ARG;
    int st = ensure_coef(h, mode);
    if (st) return st;
    for (auto& e : h->ev)
        if (!e) CK(cudaEventCreate(&e));
    CoefSet& cs = h->coef[mode];
    const gp_params& p = h->p;
    const bool f32 = h->active == GP_FP32_MIXED;
    const size_t bytes = n_elems(h) * (f32 ? sizeof(float2) : sizeof(double2));
    // the y-pass overwrites psi: keep a copy and restore it afterwards
    void* keep = nullptr;
    if (!dalloc(&keep, bytes)) return GP_ERR_OOM;
    void* state = f32 ? (void*)h->psi32 : (void*)h->psi;
    if (cudaMemcpyAsync(keep, state, bytes, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess) {
        cudaFree(keep);
        return GP_ERR_CUDA;
    }
    // scratch larger than L2 for cold-cache timings (warm timings if it does not fit)
    void* flush = nullptr;
    size_t flush_bytes = 0;
    {
        int dev = 0, l2 = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess &&
            l2 > 0) {
            flush_bytes = (size_t)l2 * 3 / 2;
            if (!dalloc(&flush, flush_bytes)) {
                flush = nullptr;
                cudaGetLastError();
            }
        }
    }
    double best_total = 0;
    for (int dir = 0; dir < 2 && st == GP_OK; ++dir) {
        const int L = dir == 0 ? p.nx : p.ny, nl = dir == 0 ? p.ny : p.nx;
        const double cp = max_cp(p, dir, mode);
        LineTiling& cur = f32 ? (dir == 0 ? cs.ftx : cs.fty) : (dir == 0 ? cs.tx : cs.ty);
        LineTiling best = cur;
        float best_ms = -1.0f;
        const int ms_add[] = {0, 4, 8, 16, 32};
        // complex128: the shared-memory solve and the register-resident one (m = 32)
        const int kinds[2] = {f32 ? TILE_C64_REG : TILE_C128, TILE_C128_REG};
        for (int kind : kinds)
        for (int compact : {0, 1})
        for (int S : {1, 2, 4, 8})
            for (int R : {1, 2, 4, 8})
                for (int add : ms_add) {
                    if (f32 && kind == TILE_C128_REG) continue;
                    LineTiling t;
                    if (make_tiling(L, nl, cp, kind, S, R, cur.m - (cur.m % 4) + add, &t, compact) != GP_OK)
                        continue;
                    if (S > 1 && L < 64) continue;
                    float ms;
                    if (f32) {
                        PassArgsF a = pass_args_f32(h, cs, dir);
                        t.bulk = a.t.bulk;
                        a.t = t;
                        ms = time_pass(h, a, dir, mode, flush, flush_bytes);
                    } else {
                        PassArgs a = pass_args(h, cs, dir);
                        t.bulk = a.t.bulk;
                        a.t = t;
                        ms = time_pass(h, a, dir, mode, flush, flush_bytes);
                    }
                    if (ms > 0 && (best_ms < 0 || ms < best_ms)) {
                        best_ms = ms;
                        best = t;
                    }
                }
        if (best_ms < 0) st = GP_ERR_CUDA;
        cur = best;
        cur.bulk = 0;
        best_total += best_ms;
    }
    cudaGetLastError();
    if (cudaMemcpyAsync(state, keep, bytes, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess) st = GP_ERR_CUDA;
    cudaStreamSynchronize(h->stream);
    cudaFree(keep);
    cudaFree(flush);
    drop_graphs(h);
    if (ms_out) *ms_out = best_total;
    return st;
}

int gp_plan_tiling(const gp_params* p, int mode, int dir, int* out)
{
    if (!out || (mode != GP_IMAG && mode != GP_REAL) || dir < 0 || dir > 1) return GP_ERR_ARG;
    int st = validate(p);
    if (st) return st;
    const int L = dir == 0 ? p->nx : p->ny, nl = dir == 0 ? p->ny : p->nx;
    const int kind = p->precision == GP_FP32_MIXED ? TILE_C64_REG : TILE_C128;
    LineTiling t;
    if ((st = choose_tiling(L, nl, max_cp(*p, dir, mode), &t, kind))) return st;
    const int unit = t.single ? 2 : 1, G = t.single ? 8 : (kind == TILE_C128 ? 8 : 16);
    out[0] = t.S;
    out[1] = t.R;
    out[2] = t.m;
    out[3] = t.Q;
    out[4] = t.threads;
    out[5] = (int)t.smem;
    out[6] = y_blocks(t);
    out[7] = t.single;
    out[8] = t.F;
    out[9] = t.cs;
    out[10] = t.Lp;
    out[11] = solve_conflicts(t.cs, t.Lp, 3 * t.R, t.Qc, G, unit);
    return GP_OK;
}

int gp_set_debug(gp_handle* h, int flags)
{
    if (!h || (flags & ~GP_DEBUG_POISON)) return GP_ERR_ARG;
    if (h->debug != flags) drop_graphs(h);  // the captured steps hold the other form
    h->debug = flags;
    return GP_OK;
}

int gp_set_tiling(gp_handle* h, int mode, int dir, int cluster, int lines_per_cta, int chunk, int register_solve)
{
    if (!h || (mode != GP_IMAG && mode != GP_REAL) || dir < 0 || dir > 1) return GP_ERR_ARG;
    if (register_solve < -1 || register_solve > 1) return GP_ERR_ARG;
    int st = ensure_coef(h, mode);
    if (st) return st;
    CoefSet& cs = h->coef[mode];
    const gp_params& p = h->p;
    const bool f32 = h->active == GP_FP32_MIXED;
    const int kind = f32 ? (register_solve == 0 ? TILE_C64 : TILE_C64_REG)
                         : (register_solve == 1 ? TILE_C128_REG : TILE_C128);
    LineTiling t;
    st = make_tiling(dir == 0 ? p.nx : p.ny, dir == 0 ? p.ny : p.nx, max_cp(p, dir, mode), kind, cluster,
                     lines_per_cta, chunk, &t);
    if (st) return st;
    if (register_solve == 1 && !t.single) return GP_ERR_UNSUPPORTED;  // chunk longer than the compiled ones
    (f32 ? (dir == 0 ? cs.ftx : cs.fty) : (dir == 0 ? cs.tx : cs.ty)) = t;
    drop_graphs(h);
    return GP_OK;
}

int gp_tiling_info(gp_handle* h, int mode, int dir, int* out)
{
    if (!h || !out || (mode != GP_IMAG && mode != GP_REAL) || dir < 0 || dir > 1) return GP_ERR_ARG;
    int st = ensure_coef(h, mode);
    if (st) return st;
    const CoefSet& cs = h->coef[mode];
    const bool f32 = h->active == GP_FP32_MIXED;
    const LineTiling& t = f32 ? (dir == 0 ? cs.ftx : cs.fty) : (dir == 0 ? cs.tx : cs.ty);
    out[0] = t.S;
    out[1] = t.R;
    out[2] = t.m;
    out[3] = t.Q;
    out[4] = t.threads;
    out[5] = (int)t.smem;
    out[6] = y_blocks(t);
    out[7] = t.single;
    return GP_OK;
}

int gp_apply_substep(gp_handle* h, int which, int mode)
{
    if (!h || which < 0 || which > 2 || (mode != GP_IMAG && mode != GP_REAL)) return GP_ERR_ARG;
    int st = ensure_coef(h, mode);
    if (st) return st;
    if ((st = flush_scale(h))) return st;
    const CoefSet& cs = h->coef[mode];
    if (h->active == GP_FP32_MIXED) {
        PassArgsF ax = pass_args_f32(h, cs, 0), ay = pass_args_f32(h, cs, 1);
        ax.do_p = which == 0;
        ax.do_solve = which == 1;
        ay.do_solve = which == 2;
        LK(launch_xpass(ax, mode, h->stream));
        LK(launch_ypass(ay, mode, h->stream));
    } else {
        PassArgs ax = pass_args(h, cs, 0), ay = pass_args(h, cs, 1);
        ax.do_p = which == 0;
        ax.do_solve = which == 1;
        ay.do_solve = which == 2;
        LK(launch_xpass(ax, mode, h->stream));
        LK(launch_ypass(ay, mode, h->stream));
    }
    return sync_status(h);
}

void gp_inject_alloc_failure(long long after) { g_fail_after.store(after < 0 ? -1 : after); }

// ---- checkpoints -------------------------------------------------------------
// A checkpoint is the handle's exact device state: parameters, step count,
// storage precision, the pending imaginary-time scale and the stored state in
// that precision (complex128 or complex64), in host byte order.  Restoring it
// and propagating gives bitwise the results of the uninterrupted run (same
// library build, same tilings).
namespace {
struct CkptHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    gp_params p;
    long long steps;
    int32_t active;
    int32_t scale_pending;
    double scale;
    int32_t split;
    int32_t mcon;
    double m_target;
    uint64_t state_bytes;
};
constexpr char kCkptMagic[8] = {'G', 'P', 'S', 'P', 'C', 'K', 'P', '1'};

size_t state_bytes(const gp_handle* h)
{
    return n_elems(h) * (h->active == GP_FP32_MIXED ? sizeof(float2) : sizeof(double2));
}
}  // namespace

size_t gp_checkpoint_bytes(gp_handle* h) { return h ? sizeof(CkptHeader) + state_bytes(h) : 0; }

int gp_checkpoint_save(gp_handle* h, void* buf, size_t size)
{
    if (!h || !buf || size < gp_checkpoint_bytes(h)) return GP_ERR_ARG;
    CkptHeader hd{};
    std::memcpy(hd.magic, kCkptMagic, sizeof hd.magic);
    hd.version = 1;
    hd.header_bytes = sizeof(CkptHeader);
    hd.p = h->p;
    hd.steps = h->steps;
    hd.active = h->active;
    hd.scale_pending = h->scale_pending ? 1 : 0;
    hd.split = h->split;
    hd.mcon = h->mcon;
    hd.m_target = h->m_target;
    hd.state_bytes = state_bytes(h);
    double scale = 1.0;
    const void* src = h->active == GP_FP32_MIXED ? (const void*)h->psi32 : (const void*)h->psi;
    unsigned char* out = static_cast<unsigned char*>(buf);
    CK(cudaMemcpyAsync(&scale, h->scal, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(out + sizeof(CkptHeader), src, hd.state_bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    hd.scale = scale;
    std::memcpy(out, &hd, sizeof hd);
    return GP_OK;
}

int gp_checkpoint_load(gp_handle* h, const void* buf, size_t size)
{
    if (!h || !buf || size < sizeof(CkptHeader)) return GP_ERR_ARG;
    CkptHeader hd;
    std::memcpy(&hd, buf, sizeof hd);
    if (std::memcmp(hd.magic, kCkptMagic, sizeof hd.magic) != 0 || hd.version != 1 ||
        hd.header_bytes != sizeof(CkptHeader))
        return GP_ERR_ARG;
    const gp_params& p = hd.p;
    if (validate(&p) != GP_OK || p.nx != h->p.nx || p.ny != h->p.ny || p.xlen != h->p.xlen ||
        p.ylen != h->p.ylen || p.precision != h->p.precision)
        return GP_ERR_ARG;
    if (hd.active != GP_FP64 && hd.active != GP_FP32_MIXED) return GP_ERR_ARG;
    if (hd.active == GP_FP32_MIXED && !h->psi32) return GP_ERR_ARG;
    const size_t want = n_elems(h) * (hd.active == GP_FP32_MIXED ? sizeof(float2) : sizeof(double2));
    if (hd.state_bytes != want || size < sizeof(CkptHeader) + want || !std::isfinite(hd.scale) ||
        (hd.split != GP_SPLIT_LIE && hd.split != GP_SPLIT_STRANG))
        return GP_ERR_ARG;
    const unsigned char* in = static_cast<const unsigned char*>(buf) + sizeof(CkptHeader);
    void* dst = hd.active == GP_FP32_MIXED ? (void*)h->psi32 : (void*)h->psi;
    CK(cudaMemcpyAsync(dst, in, want, cudaMemcpyHostToDevice, h->stream));
    LK(launch_set_scalar(h->scal, hd.scale, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->p = p;
    h->active = hd.active;
    h->steps = hd.steps;
    h->scale_pending = hd.scale_pending != 0;
    h->split = hd.split;
    h->mcon = hd.mcon;
    h->m_target = hd.m_target;
    drop_graphs(h);  // the captured launches hold the previous parameters
    return GP_OK;
}

int gp_check_wait_timeout(gp_handle* h, int polls)
{
    if (!h || polls < 1 || polls > (1 << 16)) return GP_ERR_ARG;
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
    LK(launch_wait_probe(polls, h->flag, h->stream));
    return check_flags(h);
}

int gp_observables(gp_handle* h, gp_obs* out)
{
    if (!h || !out) return GP_ERR_ARG;
    const gp_params& p = h->p;
    LK(widen_into_psi(h));
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
    LK(launch_observables(h->psi, h->scal, p.nx, p.ny, p.xlen, p.ylen, p.wx, p.wy, p.c0, p.c2, p.rabi, p.omeg,
                          gamma_of(p), eta_of(p), h->obs_part, h->obs_out, h->flag, h->stream));
    double v[8];
    int flag = 0;
    CK(cudaMemcpyAsync(v, h->obs_out, 7 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    out->norm[0] = v[0];
    out->norm[1] = v[1];
    out->norm[2] = v[2];
    out->norm_total = v[3];
    out->magnetization = v[4];
    out->energy = v[5];
    out->mu = v[6];
    out->steps = h->steps;
    return (flag & 4) ? GP_ERR_NONFINITE : GP_OK;
}

}  // extern "C"

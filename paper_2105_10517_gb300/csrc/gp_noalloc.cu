// gp_noalloc.cu -- gp_propagate_noalloc: the time step of gp_propagate for
// callers that must not allocate device memory.
//
// Who needs this: code that runs inside a host application which owns the
// device memory budget (a plugin that gets its buffers from the host's pool,
// a real-time loop with a no-allocation rule, a process sharing a GPU under a
// fixed memory quota).  Such a caller already holds the wave function in device
// memory but may not call cudaMalloc/cudaFree, so it cannot create a gp_handle.
//
// Everything the step needs besides the caller's psi -- the transposed
// intermediate between the two line passes, the Thomas coefficient tables, the
// trap factors, the per-CTA partial norms, the normalisation scalar and a status
// flag -- lives in the file-scope __device__ arrays below.  Their size is fixed
// for grids up to kMaxLine x kMaxLine points (about 8.6 MB); every GPU that loads
// the library keeps them until the process exits.
#include "gp_internal.cuh"

#include <mutex>

namespace gpspin {
namespace {

constexpr int kMaxLine = 256;                       // nx, ny <= 256
constexpr size_t kMaxSites = (size_t)kMaxLine * kMaxLine;

static __device__ __align__(256) double2 g_work[3 * kMaxSites];
static __device__ __align__(256) LineCoef g_coef_x[3 * kMaxLine];
static __device__ __align__(256) LineCoef g_coef_y[3 * kMaxLine];
static __device__ __align__(256) double2 g_ex[kMaxLine];
static __device__ __align__(256) double2 g_ey[kMaxLine];
static __device__ __align__(256) double g_partials[kMaxLine];
static __device__ __align__(256) double g_scale[2];
static __device__ __align__(256) int g_flag;

// Device addresses of the arrays above.  In host code the array names are
// host-side stand-ins, not device addresses, so each device looks them up once
// with cudaGetSymbolAddress while it is current.
struct Scratch {
    double2* work;
    LineCoef* cx;
    LineCoef* cy;
    double2* ex;
    double2* ey;
    double* partials;
    double* scale;
    int* flag;
};

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
Scratch g_scratch[kMaxDevices];
bool g_ready[kMaxDevices];

int lookup(void** p, const void* sym, const char* what)
{
    return report_cuda(cudaGetSymbolAddress(p, sym), what);
}

// Looks the addresses up for the current device.  A failed lookup is not
// remembered: the next call on that device tries again.
int setup(int dev)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_ready[dev]) return GP_OK;
    Scratch s{};
    int bad = 0;
    bad |= lookup((void**)&s.work, g_work, "cudaGetSymbolAddress(g_work)");
    bad |= lookup((void**)&s.cx, g_coef_x, "cudaGetSymbolAddress(g_coef_x)");
    bad |= lookup((void**)&s.cy, g_coef_y, "cudaGetSymbolAddress(g_coef_y)");
    bad |= lookup((void**)&s.ex, g_ex, "cudaGetSymbolAddress(g_ex)");
    bad |= lookup((void**)&s.ey, g_ey, "cudaGetSymbolAddress(g_ey)");
    bad |= lookup((void**)&s.partials, g_partials, "cudaGetSymbolAddress(g_partials)");
    bad |= lookup((void**)&s.scale, g_scale, "cudaGetSymbolAddress(g_scale)");
    bad |= lookup((void**)&s.flag, &g_flag, "cudaGetSymbolAddress(g_flag)");
    if (bad) return GP_ERR_CUDA;
    g_scratch[dev] = s;
    g_ready[dev] = true;
    return GP_OK;
}

#define NK(x)                                                  \
    do {                                                       \
        if (report_cuda((x), #x) != 0) return GP_ERR_CUDA;     \
    } while (0)
#define NL(x)                                                  \
    do {                                                       \
        if ((x) != 0) return GP_ERR_CUDA;                      \
    } while (0)

}  // namespace
}  // namespace gpspin

using namespace gpspin;

extern "C" int gp_propagate_noalloc(const gp_params* params, double* psi_dev, long long nsteps, int mode,
                                    void* cuda_stream)
{
    int st = validate(params);
    if (st) return st;
    if (!psi_dev || nsteps < 0 || (mode != GP_IMAG && mode != GP_REAL)) return GP_ERR_ARG;
    // the passes move psi as 16-byte complex128 values
    if (reinterpret_cast<uintptr_t>(psi_dev) % 16 != 0) return GP_ERR_ARG;
    const gp_params& p = *params;
    if (p.nx > kMaxLine || p.ny > kMaxLine) return GP_ERR_TOO_LARGE;
    if (nsteps == 0) return GP_OK;
    int dev = 0;
    NK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return GP_ERR_CUDA;
    if ((st = setup(dev))) return st;
    const Scratch& S = g_scratch[dev];
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    // unsplit tilings: one CTA per line group, so the y-pass writes at most
    // kMaxLine partial norms into g_partials
    LineTiling tx, ty;
    if ((st = choose_tiling(p.nx, p.ny, max_cp(p, 0, mode), &tx, TILE_C128, 0))) return st;
    if ((st = choose_tiling(p.ny, p.nx, max_cp(p, 1, mode), &ty, TILE_C128, 0))) return st;
    if ((ty.nlines + ty.R - 1) / ty.R * ty.S > kMaxLine) return GP_ERR_TOO_LARGE;

    // The arrays keep the previous call's contents: the flag must start at zero
    // and the scale at one; every other array is fully rewritten below.
    const double dx = p.xlen / p.nx, dy = p.ylen / p.ny;
    NK(cudaMemsetAsync(S.flag, 0, sizeof(int), stream));
    NL(launch_set_scalar(S.scale, 1.0, stream));
    NL(launch_coef(S.cx, p.ny, 0, mode, dx, p.ylen, dy, p.dt, p.omeg, gamma_of(p), eta_of(p), S.flag, stream));
    NL(launch_coef(S.cy, p.nx, 1, mode, dy, p.xlen, dx, p.dt, p.omeg, gamma_of(p), eta_of(p), S.flag, stream));
    NL(launch_trap_table(S.ex, p.nx, p.xlen, p.wx, p.dt, mode, stream));
    NL(launch_trap_table(S.ey, p.ny, p.ylen, p.wy, p.dt, mode, stream));
    int flag = 0;
    NK(cudaMemcpyAsync(&flag, S.flag, sizeof(int), cudaMemcpyDeviceToHost, stream));
    NK(cudaStreamSynchronize(stream));
    if (flag & 1) return GP_ERR_UNSUPPORTED;

    PassArgs ax{}, ay{};
    ax.nx = ay.nx = p.nx;
    ax.ny = ay.ny = p.ny;
    ax.scale = ay.scale = S.scale;
    ax.dt = ay.dt = p.dt;
    ax.c0 = ay.c0 = p.c0;
    ax.c2 = ay.c2 = p.c2;
    ax.rabi = ay.rabi = p.rabi;
    ax.ex = ay.ex = S.ex;
    ax.ey = ay.ey = S.ey;
    ax.do_p = ay.do_p = 1;
    ax.do_solve = ay.do_solve = 1;
    ax.in = reinterpret_cast<const double2*>(psi_dev);
    ax.out = S.work;
    ax.coef = S.cx;
    ax.t = tx;
    ay.in = S.work;
    ay.out = reinterpret_cast<double2*>(psi_dev);
    ay.coef = S.cy;
    ay.t = ty;
    ax.err = ay.err = S.flag;
    ax.dx = ay.dx = dx;
    ax.dy = ay.dy = dy;
    ax.x0 = ay.x0 = -0.5 * p.xlen + 0.5 * dx;
    ax.y0 = ay.y0 = -0.5 * p.ylen + 0.5 * dy;
    ax.wx = ay.wx = p.wx;
    ax.wy = ay.wy = p.wy;
    ax.t.bulk = ((size_t)p.nx * sizeof(double2)) % 16 == 0;
    ay.t.bulk = ((size_t)p.ny * sizeof(double2)) % 16 == 0;
    const double da = dx * dy;
    const int gy = (ty.nlines + ty.R - 1) / ty.R * ty.S;
    if (mode == GP_IMAG) ay.partials = S.partials;
    for (long long s = 0; s < nsteps; ++s) {
        NL(launch_xpass(ax, mode, stream));
        NL(launch_ypass(ay, mode, stream));
        if (mode == GP_IMAG) NL(launch_finalize_norm(S.partials, gy, da, S.scale, S.flag, stream));
    }
    // leave the caller's psi normalised (imaginary time) and the scale at one
    if (mode == GP_IMAG) NL(launch_apply_scale(reinterpret_cast<double2*>(psi_dev), 3 * (size_t)p.nx * p.ny,
                                               S.scale, stream));
    NK(cudaMemcpyAsync(&flag, S.flag, sizeof(int), cudaMemcpyDeviceToHost, stream));
    NK(cudaStreamSynchronize(stream));
    // the same order as gp_propagate: a bulk-copy wait that gave up (bit 8)
    // makes psi unreliable, then a non-finite norm (bit 2)
    if (flag & 8) return GP_ERR_TIMEOUT;
    if (flag & 2) return GP_ERR_NONFINITE;
    return GP_OK;
}

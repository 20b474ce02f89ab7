// gp_reduce.cu -- FP64 reductions (normalisation, observables of Eq. S.6), the
// seeded initial state and small state kernels of libgpspin.
//
// Every reduction is deterministic: each CTA sums a fixed set of sites in a
// fixed order, warps combine by shuffles in a fixed pattern, and one CTA adds
// the per-CTA partials in index order.  No floating-point atomics.
#include "gp_internal.cuh"
#include <cmath>
#include <cstdio>
#include <cstdlib>

namespace gpspin {

constexpr int kRedThreads = 256;
constexpr double kRs2r = 0.70710678118654752440;

__device__ __forceinline__ double warp_sum(double v)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Block sum in a fixed order; valid in thread 0.  blockDim.x == kRedThreads.
__device__ __forceinline__ double block_sum(double v, double* sh)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kRedThreads / 32; ++w) t += sh[w];
    return t;
}

// ---------------------------------------------------------------- norms ----
__global__ void __launch_bounds__(kRedThreads) norm_partials_kernel(const double2* psi, size_t n, double* partials)
{
    __shared__ double sh[32];
    double acc = 0.0;
    for (size_t k = blockIdx.x * (size_t)kRedThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kRedThreads) {
        double2 v = psi[k];
        acc += fma(v.x, v.x, v.y * v.y);
    }
    double t = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// N = dA * sum(partials) in index order (per thread strided, then fixed tree);
// scale[0] = 1/sqrt(N) (the pending normalisation), scale[1] = N.
// A non-finite or non-positive N leaves scale[0] = 1 and raises flag bit 1.
__global__ void __launch_bounds__(kRedThreads) finalize_norm_kernel(const double* partials, int n, double da,
                                                                    double* scale, int* flag)
{
    __shared__ double sh[32];
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += kRedThreads) acc += partials[k];
    double t = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        double nrm = t * da;
        scale[1] = nrm;
        if (nrm > 0.0 && isfinite(nrm)) {
            scale[0] = 1.0 / sqrt(nrm);
        } else {
            scale[0] = 1.0;
            atomicOr(flag, 2);
        }
    }
}

template <typename C>
__global__ void apply_scale_kernel(C* psi, size_t n, double* scale)
{
    const double s = scale[0];
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        C v = psi[k];
        v.x = s * v.x;
        v.y = s * v.y;
        psi[k] = v;
    }
}

// dst = s * src in FP64 (the source is either precision; widening is exact).
template <typename C>
__global__ void scaled_copy_kernel(double2* dst, const C* src, size_t n, const double* scale)
{
    const double s = scale[0];
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        C v = src[k];
        dst[k] = make_double2(s * (double)v.x, s * (double)v.y);
    }
}

// complex128 -> complex64 (round to nearest).
__global__ void narrow_kernel(float2* dst, const double2* src, size_t n)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        double2 v = src[k];
        dst[k] = make_float2((float)v.x, (float)v.y);
    }
}

__global__ void set_scalar_kernel(double* p, double v) { *p = v; }

// Magnetisation-constrained normalisation: N_c = dA * sum of the per-component
// partials (index order); sigma_c makes N = 1 and N+ - N- = m with
// sigma+ sigma- = sigma0^2:  sigma0^2 = (1 - m^2) / (N0 + sqrt(N0^2 m^2 + 4 (1 - m^2) N+ N-)),
// sigma+-^2 = (1 +- m - sigma0^2 N0) / (2 N+-); an empty +-1 component keeps 1.
__global__ void __launch_bounds__(kRedThreads) finalize_m_kernel(const double* partials, int n, double da, double m,
                                                                 double* sigma, int* flag)
{
    __shared__ double sh[32];
    __shared__ double nc[3];
    for (int c = 0; c < 3; ++c) {
        double acc = 0.0;
        for (int k = threadIdx.x; k < n; k += kRedThreads) acc += partials[3 * k + c];
        double t = block_sum(acc, sh);
        if (threadIdx.x == 0) nc[c] = t * da;
    }
    if (threadIdx.x == 0) {
        const double np_ = nc[0], n0 = nc[1], nm = nc[2];
        const double a = (1.0 - m * m) / (n0 + sqrt(n0 * n0 * m * m + 4.0 * (1.0 - m * m) * np_ * nm));
        double s0 = sqrt(a);
        double sp = np_ > 0 ? sqrt((1.0 + m - a * n0) / (2.0 * np_)) : 1.0;
        double sm = nm > 0 ? sqrt((1.0 - m - a * n0) / (2.0 * nm)) : 1.0;
        if (!(isfinite(s0) && isfinite(sp) && isfinite(sm))) {
            s0 = sp = sm = 1.0;
            atomicOr(flag, 2);
        }
        sigma[0] = sp;
        sigma[1] = s0;
        sigma[2] = sm;
    }
}

template <typename C>
__global__ void apply_comp_scale_kernel(C* psi, size_t plane, const double* sigma)
{
    const double s[3] = {sigma[0], sigma[1], sigma[2]};
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < 3 * plane; k += (size_t)gridDim.x * blockDim.x) {
        const double f = s[k / plane];
        C v = psi[k];
        v.x = f * v.x;
        v.y = f * v.y;
        psi[k] = v;
    }
}

// Batched normalisation: CTA b finalises instance b (same arithmetic and order
// as finalize_norm_kernel, so an instance gets the same scale alone or batched).
__global__ void __launch_bounds__(kRedThreads) finalize_norm_batched_kernel(const FinArgs* fin, const int* n_inst,
                                                                            int* flag)
{
    __shared__ double sh[32];
    if ((int)blockIdx.x >= *n_inst) return;
    const FinArgs f = fin[blockIdx.x];
    double acc = 0.0;
    for (int k = threadIdx.x; k < f.n; k += kRedThreads) acc += f.partials[k];
    double t = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        double nrm = t * f.da;
        f.scale[1] = nrm;
        if (nrm > 0.0 && isfinite(nrm)) {
            f.scale[0] = 1.0 / sqrt(nrm);
        } else {
            f.scale[0] = 1.0;
            atomicOr(flag, 2);
        }
    }
}

// --------------------------------------------------------- initial state ---
// splitmix64 (Steele, Lea and Flood, OOPSLA 2014) on the counter seed ^ index.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x)
{
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// psi_c = sqrt(f_c) pi^-1/2 (x + i sgn(l_c) y)^|l_c| exp(-(x^2+y^2)/2) exp(i phi),
// phi = noise (2u - 1), u from splitmix64(seed ^ ((c ny + j) nx + i)).
__global__ void init_gaussian_kernel(double2* psi, int nx, int ny, double xlen, double ylen, double f0, double f1,
                                     double f2, int l0, int l1, int l2, unsigned long long seed, double noise)
{
    const size_t plane = (size_t)nx * ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < 3 * plane; k += (size_t)gridDim.x * blockDim.x) {
        int c = (int)(k / plane);
        size_t rem = k - c * plane;
        int j = (int)(rem / nx), i = (int)(rem - (size_t)j * nx);
        double x = -0.5 * xlen + (i + 0.5) * (xlen / nx);
        double y = -0.5 * ylen + (j + 0.5) * (ylen / ny);
        double u = (double)(splitmix64(seed ^ (unsigned long long)k) >> 11) * 0x1.0p-53;
        double ph = noise * (2.0 * u - 1.0);
        double fr = c == 0 ? f0 : (c == 1 ? f1 : f2);
        int l = c == 0 ? l0 : (c == 1 ? l1 : l2);
        double amp = sqrt(fr) * exp(-0.5 * (x * x + y * y)) / sqrt(3.14159265358979323846);
        double sn, cs;
        sincos(ph, &sn, &cs);
        double2 v = make_double2(amp * cs, amp * sn);
        // centre vortex of charge l: multiply by (x + i sgn(l) y)^|l|
        const double zy = l > 0 ? y : -y;
        for (int q = 0; q < (l < 0 ? -l : l); ++q) v = make_double2(v.x * x - v.y * zy, v.x * zy + v.y * x);
        psi[k] = v;
    }
}

// ----------------------------------------------------------- observables ---
// Per-site terms of E (Eq. S.6) in operator form, discretised consistently with
// the sweeps: kinetic 1/2 sum over every forward link (including the links to
// the zero exterior) of |psi_b - psi_a|^2 / h^2; V rho; c0 rho^2 / 2;
// c2 |F|^2 / 2 (equal to the c2 bracket of S.6); R F_x (the Rabi bracket);
// -Omega Re psi^dagger L_z psi with L_z = -i (x D_y - y D_x); and
// gamma Re psi^dagger (eta p_y Sigma_x - p_x Sigma_y) psi, D central differences.
// Partial slots: 0 kinetic, 1 V rho, 2 rho^2, 3 |F|^2, 4 F_x, 5 Im psi^* (x D_y - y D_x) psi,
// 6 Im psi^dag Sigma_x D_y psi, 7 Im psi^dag Sigma_y D_x psi, 8-10 |psi_c|^2.
constexpr int kObs = 11;

struct ObsArgs {
    const double2* psi;
    const double* scale;
    int nx, ny;
    double xlen, ylen, wx, wy;
};

__device__ __forceinline__ double2 ld(const ObsArgs& A, int c, int j, int i, double s)
{
    if (i < 0 || i >= A.nx || j < 0 || j >= A.ny) return make_double2(0.0, 0.0);
    double2 v = A.psi[((size_t)c * A.ny + j) * A.nx + i];
    return make_double2(s * v.x, s * v.y);
}

__device__ __forceinline__ double im_conj_mul(double2 a, double2 b) { return a.x * b.y - a.y * b.x; }

__global__ void __launch_bounds__(kRedThreads) obs_partials_kernel(ObsArgs A, double* partials)
{
    __shared__ double sh[32];
    const double s = A.scale[0];
    const double dx = A.xlen / A.nx, dy = A.ylen / A.ny;
    double acc[kObs];
    for (int q = 0; q < kObs; ++q) acc[q] = 0.0;
    const size_t n = (size_t)A.nx * A.ny;
    for (size_t k = blockIdx.x * (size_t)kRedThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kRedThreads) {
        int j = (int)(k / A.nx), i = (int)(k - (size_t)j * A.nx);
        double x = -0.5 * A.xlen + (i + 0.5) * dx, y = -0.5 * A.ylen + (j + 0.5) * dy;
        double2 v[3], dxv[3], dyv[3];
        for (int c = 0; c < 3; ++c) {
            v[c] = ld(A, c, j, i, s);
            double2 xr = ld(A, c, j, i + 1, s), xl = ld(A, c, j, i - 1, s);
            double2 yu = ld(A, c, j + 1, i, s), yd = ld(A, c, j - 1, i, s);
            double kx = (xr.x - v[c].x) * (xr.x - v[c].x) + (xr.y - v[c].y) * (xr.y - v[c].y);
            double ky = (yu.x - v[c].x) * (yu.x - v[c].x) + (yu.y - v[c].y) * (yu.y - v[c].y);
            double r = v[c].x * v[c].x + v[c].y * v[c].y;
            acc[0] += kx / (dx * dx) + ky / (dy * dy) + (i == 0 ? r / (dx * dx) : 0.0) + (j == 0 ? r / (dy * dy) : 0.0);
            dxv[c] = make_double2((xr.x - xl.x) / (2 * dx), (xr.y - xl.y) / (2 * dx));
            dyv[c] = make_double2((yu.x - yd.x) / (2 * dy), (yu.y - yd.y) / (2 * dy));
            acc[8 + c] += r;
            // Im conj(psi) (x D_y psi - y D_x psi)
            acc[5] += x * im_conj_mul(v[c], dyv[c]) - y * im_conj_mul(v[c], dxv[c]);
        }
        double rp = v[0].x * v[0].x + v[0].y * v[0].y;
        double r0 = v[1].x * v[1].x + v[1].y * v[1].y;
        double rm = v[2].x * v[2].x + v[2].y * v[2].y;
        double rho = rp + r0 + rm;
        double vtr = 0.5 * (A.wx * A.wx * x * x + A.wy * A.wy * y * y);
        acc[1] += vtr * rho;
        acc[2] += rho * rho;
        double fr = v[0].x * v[1].x + v[0].y * v[1].y + v[1].x * v[2].x + v[1].y * v[2].y;
        double fi = v[0].x * v[1].y - v[0].y * v[1].x + v[1].x * v[2].y - v[1].y * v[2].x;
        acc[3] += 2.0 * (fr * fr + fi * fi) + (rp - rm) * (rp - rm);
        acc[4] += 1.4142135623730950488 * fr;
        // Im psi^dag Sigma_x u, u = D_y psi: Sigma_x u = (u0, u+ + u-, u0)/sqrt2
        double2 sxu0 = dyv[1];
        double2 sxu1 = make_double2(dyv[0].x + dyv[2].x, dyv[0].y + dyv[2].y);
        acc[6] += kRs2r * (im_conj_mul(v[0], sxu0) + im_conj_mul(v[1], sxu1) + im_conj_mul(v[2], sxu0));
        // Im psi^dag Sigma_y u, u = D_x psi: Sigma_y u = (-i u0, i (u+ - u-), i u0)/sqrt2;
        // Im conj(a) (i b) = Re conj(a) b
        double2 u0 = dxv[1], ud = make_double2(dxv[0].x - dxv[2].x, dxv[0].y - dxv[2].y);
        double re_p = v[0].x * u0.x + v[0].y * u0.y;
        double re_0 = v[1].x * ud.x + v[1].y * ud.y;
        double re_m = v[2].x * u0.x + v[2].y * u0.y;
        acc[7] += kRs2r * (-re_p + re_0 + re_m);
    }
    for (int q = 0; q < kObs; ++q) {
        double t = block_sum(acc[q], sh);
        if (threadIdx.x == 0) partials[(size_t)blockIdx.x * kObs + q] = t;
    }
}

struct ObsConsts {
    double da, c0, c2, rabi, omeg, gamma, eta;
};

// out: norm[3], N, m, E, mu, then the raw sums; flag bit 4 if anything is non-finite.
__global__ void __launch_bounds__(kRedThreads) finalize_obs_kernel(const double* partials, int nblk, ObsConsts k,
                                                                   double* out, int* flag)
{
    __shared__ double sh[32];
    __shared__ double tot[kObs];
    for (int q = 0; q < kObs; ++q) {
        double acc = 0.0;
        for (int b = threadIdx.x; b < nblk; b += kRedThreads) acc += partials[(size_t)b * kObs + q];
        double t = block_sum(acc, sh);
        if (threadIdx.x == 0) tot[q] = t;
    }
    if (threadIdx.x == 0) {
        double da = k.da;
        double n0 = tot[8] * da, n1 = tot[9] * da, n2 = tot[10] * da;
        double ntot = n0 + n1 + n2;
        double nl = 0.5 * k.c0 * tot[2] + 0.5 * k.c2 * tot[3];
        double e = da * (0.5 * tot[0] + tot[1] + nl + k.rabi * tot[4] - k.omeg * tot[5] +
                         k.gamma * (k.eta * tot[6] - tot[7]));
        double mu = (e + da * nl) / ntot;
        out[0] = n0; out[1] = n1; out[2] = n2; out[3] = ntot; out[4] = n0 - n2; out[5] = e; out[6] = mu;
        bool bad = false;
        for (int q = 0; q < 7; ++q) bad |= !isfinite(out[q]);
        if (bad) atomicOr(flag, 4);
    }
}

// ------------------------------------------------------------- launchers ---
// Returns 0 for cudaSuccess; otherwise 1, and with GPSPIN_DEBUG set in the
// environment prints the failing call to stderr.
int report_cuda(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return 0;
    static const bool dbg = std::getenv("GPSPIN_DEBUG") != nullptr;
    if (dbg) std::fprintf(stderr, "libgpspin: %s failed: %s\n", what, cudaGetErrorString(e));
    return 1;
}

static int grid_for(size_t n, int threads, int cap)
{
    size_t g = (n + threads - 1) / threads;
    return (int)(g < (size_t)cap ? (g > 0 ? g : 1) : cap);
}

int launch_norm(const double2* psi, size_t n, double* partials, int nblk, double da, double* scale, int* flag,
                cudaStream_t st)
{
    norm_partials_kernel<<<nblk, kRedThreads, 0, st>>>(psi, n, partials);
    finalize_norm_kernel<<<1, kRedThreads, 0, st>>>(partials, nblk, da, scale, flag);
    return report_cuda(cudaGetLastError(), __func__);
}

int launch_finalize_norm(const double* partials, int n, double da, double* scale, int* flag, cudaStream_t st)
{
    finalize_norm_kernel<<<1, kRedThreads, 0, st>>>(partials, n, da, scale, flag);
    return report_cuda(cudaGetLastError(), __func__);
}

int launch_finalize_norm_batched(const FinArgs* fin, const int* n_inst, int capacity, int* flag, cudaStream_t st)
{
    if (capacity <= 0) return 0;
    finalize_norm_batched_kernel<<<capacity, kRedThreads, 0, st>>>(fin, n_inst, flag);
    return report_cuda(cudaGetLastError(), __func__);
}

int launch_finalize_m(const double* partials, int n, double da, double m, double* sigma, int* flag, cudaStream_t st)
{
    finalize_m_kernel<<<1, kRedThreads, 0, st>>>(partials, n, da, m, sigma, flag);
    return report_cuda(cudaGetLastError(), __func__);
}

int launch_apply_comp_scale(double2* psi, size_t plane, const double* sigma, cudaStream_t st)
{
    apply_comp_scale_kernel<<<grid_for(3 * plane, 256, 1216), 256, 0, st>>>(psi, plane, sigma);
    return report_cuda(cudaGetLastError(), __func__);
}

int launch_apply_comp_scale(float2* psi, size_t plane, const double* sigma, cudaStream_t st)
{
    apply_comp_scale_kernel<<<grid_for(3 * plane, 256, 1216), 256, 0, st>>>(psi, plane, sigma);
    return report_cuda(cudaGetLastError(), __func__);
}

int launch_apply_scale(double2* psi, size_t n, double* scale, cudaStream_t st)
{
    apply_scale_kernel<<<grid_for(n, 256, 1216), 256, 0, st>>>(psi, n, scale);
    set_scalar_kernel<<<1, 1, 0, st>>>(scale, 1.0);
    return report_cuda(cudaGetLastError(), __func__);
}

int launch_apply_scale(float2* psi, size_t n, double* scale, cudaStream_t st)
{
    apply_scale_kernel<<<grid_for(n, 256, 1216), 256, 0, st>>>(psi, n, scale);
    set_scalar_kernel<<<1, 1, 0, st>>>(scale, 1.0);
    return report_cuda(cudaGetLastError(), __func__);
}

int launch_set_scalar(double* p, double v, cudaStream_t st)
{
    set_scalar_kernel<<<1, 1, 0, st>>>(p, v);
    return report_cuda(cudaGetLastError(), __func__);
}

int launch_scaled_copy(double2* dst, const double2* src, size_t n, const double* scale, cudaStream_t st)
{
    scaled_copy_kernel<<<grid_for(n, 256, 1216), 256, 0, st>>>(dst, src, n, scale);
    return report_cuda(cudaGetLastError(), __func__);
}

int launch_scaled_copy(double2* dst, const float2* src, size_t n, const double* scale, cudaStream_t st)
{
    scaled_copy_kernel<<<grid_for(n, 256, 1216), 256, 0, st>>>(dst, src, n, scale);
    return report_cuda(cudaGetLastError(), __func__);
}

int launch_narrow(float2* dst, const double2* src, size_t n, cudaStream_t st)
{
    narrow_kernel<<<grid_for(n, 256, 1216), 256, 0, st>>>(dst, src, n);
    return report_cuda(cudaGetLastError(), __func__);
}

int launch_init_gaussian(double2* psi, int nx, int ny, double xlen, double ylen, const double frac[3],
                         const int winding[3], unsigned long long seed, double noise, cudaStream_t st)
{
    size_t n = 3 * (size_t)nx * ny;
    init_gaussian_kernel<<<grid_for(n, 256, 1216), 256, 0, st>>>(psi, nx, ny, xlen, ylen, frac[0], frac[1], frac[2],
                                                                 winding[0], winding[1], winding[2], seed, noise);
    return report_cuda(cudaGetLastError(), __func__);
}

int obs_blocks(int nx, int ny) { return grid_for((size_t)nx * ny, kRedThreads, 608); }
int obs_slots() { return kObs; }

int launch_observables(const double2* psi, const double* scale, int nx, int ny, double xlen, double ylen, double wx,
                       double wy, double c0, double c2, double rabi, double omeg, double gamma, int eta,
                       double* partials, double* out, int* flag, cudaStream_t st)
{
    int nblk = obs_blocks(nx, ny);
    ObsArgs a{psi, scale, nx, ny, xlen, ylen, wx, wy};
    obs_partials_kernel<<<nblk, kRedThreads, 0, st>>>(a, partials);
    ObsConsts k{(xlen / nx) * (ylen / ny), c0, c2, rabi, omeg, gamma, (double)eta};
    finalize_obs_kernel<<<1, kRedThreads, 0, st>>>(partials, nblk, k, out, flag);
    return report_cuda(cudaGetLastError(), __func__);
}

}  // namespace gpspin

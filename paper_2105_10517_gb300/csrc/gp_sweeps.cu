// gp_sweeps.cu -- coefficient precompute and the two fused line passes of one
// split-step Crank-Nicolson step (arXiv 2105.10517, program summary "Solution
// method"; Supplementary Material Eqs. S.1-S.5), for complex128 (FP64 path) and
// complex64 (FP32-storage path) wave functions.
//
// FP64 on GB300 is issue-bound: one warp-wide DFMA/DMUL/DADD occupies a
// sub-partition's FP64 unit for ~64 clocks whether 1 or 32 lanes are active,
// and a dependent chain runs at that same rate.  So every FP64 instruction
// here is issued by full warps, transcendentals of small arguments are short
// Taylor polynomials, and the tridiagonal solves are split into chunks that
// many threads run at once (the chunked Thomas solve below).
#include "gp_internal.cuh"
#include <cmath>
#include <cooperative_groups.h>
#include <mutex>
#include <vector>

namespace cg = cooperative_groups;

namespace gpspin {

// ---------------------------------------------------------------- complex --
template <typename C> struct RealOf;
template <> struct RealOf<double2> { typedef double type; };
template <> struct RealOf<float2> { typedef float type; };

template <typename C> __device__ __forceinline__ C mkc(typename RealOf<C>::type x, typename RealOf<C>::type y);
template <> __device__ __forceinline__ double2 mkc<double2>(double x, double y) { return make_double2(x, y); }
template <> __device__ __forceinline__ float2 mkc<float2>(float x, float y) { return make_float2(x, y); }

template <typename C> __device__ __forceinline__ C cmul(C a, C b)
{
    return mkc<C>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a*b + c
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C c)
{
    return mkc<C>(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// c - a*b
template <typename C> __device__ __forceinline__ C cfnma(C a, C b, C c)
{
    return mkc<C>(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 dsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 drecip(double2 z)
{
    double d = z.x * z.x + z.y * z.y;
    return make_double2(z.x / d, -z.y / d);
}

template <typename C> __device__ __forceinline__ C store_as(double2 v);
template <> __device__ __forceinline__ double2 store_as<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 store_as<float2>(double2 v)
{
    return make_float2((float)v.x, (float)v.y);
}

// ------------------------------------------------- bulk row copies (TMA) ---
// Whole input rows are staged into shared memory with cp.async.bulk (the
// Blackwell bulk-copy engine), completing on an mbarrier, so every row of the
// CTA is in flight at once instead of one global load per loop iteration.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* m)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(m))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(m)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on the phase of the barrier with the given parity (phase 0 for a
// barrier used once).  Returns true (for the whole CTA) once the copies have
// landed; if any thread gives up after `tries` polls, the CTA sets bit 8 of
// *err, waits once more (again bounded) so that no copy is still writing its
// shared memory, and returns false.
constexpr int kWaitTries = 1 << 22;

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* m, int* err, int tries = kWaitTries, uint32_t parity = 0)
{
    bool ok = false;
    for (int it = 0; it < tries && !ok; ++it) ok = mbar_try_wait(m, parity);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0 && err) atomicOr(err, 8);
        for (int it = 0; it < tries && !ok; ++it) ok = mbar_try_wait(m, parity);
        __syncthreads();
        return false;
    }
    return true;
}

// Check of the give-up path above: the same bounded wait on an mbarrier that no
// copy targets and no thread arrives on, so its phase never completes and
// nothing is in flight when the CTA gives up after `tries` polls (bit 8 set).
__global__ void wait_probe_kernel(int tries, int* err)
{
    __shared__ uint64_t mbar;
    if (threadIdx.x == 0) mbar_init(&mbar, 1);
    __syncthreads();
    mbar_wait_bounded(&mbar, err, tries);
}

int launch_wait_probe(int tries, int* err, cudaStream_t st)
{
    wait_probe_kernel<<<1, 32, 0, st>>>(tries, err);
    return report_cuda(cudaGetLastError(), "wait_probe_kernel launch");
}

// Cluster barrier in two halves: an arrive that does not wait and a later wait
// for every thread of the cluster to have arrived.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire;" ::: "memory"); }
// Arrive without release ordering: for the start of a pass, whose only job is
// to publish mbarrier initialisations that their own fence.mbarrier_init
// (release, cluster scope) already orders.
__device__ __forceinline__ void cluster_arrive_relaxed()
{
    asm volatile("barrier.cluster.arrive.relaxed;" ::: "memory");
}

// Point-to-point carries between neighbouring CTAs of a cluster: the producer
// stores the value into the neighbour's shared memory and arrives on the
// neighbour's mbarrier (release, cluster scope); the consumer waits on its own
// mbarrier (acquire, cluster scope).  The wait is bounded: a time-out sets status
// bit 8 and goes on.
__device__ __forceinline__ uint32_t cluster_map(const void* p, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}

__device__ __forceinline__ void push_carry(float2 v, float2* slot, uint64_t* bar, uint32_t rank)
{
    const uint32_t a = cluster_map(slot, rank), b = cluster_map(bar, rank);
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(b) : "memory");
}

__device__ __forceinline__ void push_carry(double2 v, double2* slot, uint64_t* bar, uint32_t rank)
{
    const uint32_t a = cluster_map(slot, rank), b = cluster_map(bar, rank);
    asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v.x), "d"(v.y) : "memory");
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(b) : "memory");
}

__device__ __forceinline__ void wait_carry(uint64_t* bar, int* err)
{
    uint32_t ok = 0;
    for (int it = 0; it < kWaitTries && !ok; ++it)
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], 0;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar))
            : "memory");
    if (!ok && err) atomicOr(err, 8);
}

// Stages row segments base + c * plane + (line0 + r) * L + k0 .. + len for
// r < nl, c < 3 into dst[(r * 3 + c) * stride].  Segments and destination rows
// must be 16-byte aligned and a multiple of 16 bytes long.
// phase < 0: the barrier is initialised here and used once; phase >= 0: it was
// initialised by the caller and has completed `phase` earlier stagings.
template <typename C>
__device__ __forceinline__ bool stage_rows(C* dst, const C* base, size_t plane, int line0, int nl, int L, int k0,
                                           int len, int stride, uint64_t* mbar, int* err, int phase = -1)
{
    if (threadIdx.x == 0 && phase < 0) mbar_init(mbar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t seg_bytes = (uint32_t)(len * sizeof(C));
        mbar_expect_tx(mbar, seg_bytes * 3u * (uint32_t)nl);
        for (int r = 0; r < nl; ++r)
            for (int c = 0; c < 3; ++c)
                bulk_g2s(dst + (size_t)(r * 3 + c) * stride, base + c * plane + (size_t)(line0 + r) * L + k0, seg_bytes,
                         mbar);
    }
    return mbar_wait_bounded(mbar, err, kWaitTries, phase < 0 ? 0u : (uint32_t)(phase & 1));
}

// Stages the chunks of the CTA's line segments into their slots of the line
// array, one bulk copy per chunk issued by the thread that solves it
// (u = ql * 3 nl + lc): chunk (lc, ql) of line point k0 + ql m .. to
// dst[lc * Lp + ql * cs].  Every copy must start on a 16-byte boundary and move a
// multiple of 16 bytes: complex128 always; complex64 with even L, m, cs and Lp.
// `phase` as for stage_rows.
template <typename C>
__device__ __forceinline__ bool stage_chunks(C* dst, const C* base, size_t plane, int line0, int nl, int L, int k0,
                                             int len, int m, int cs, int Lp, uint64_t* mbar, int* err, int phase = -1)
{
    if (threadIdx.x == 0) {
        if (phase < 0) mbar_init(mbar, 1);
        mbar_expect_tx(mbar, (uint32_t)(3 * nl * len * sizeof(C)));
    }
    __syncthreads();
    const int nl3 = 3 * nl, nq = (len + m - 1) / m;
    for (int u = threadIdx.x; u < nl3 * nq; u += blockDim.x) {
        const int ql = u / nl3, lc = u - ql * nl3, r = lc / 3, c = lc - 3 * r;
        const int k = ql * m, n = min(m, len - k);
        bulk_g2s(dst + lc * Lp + ql * cs, base + c * plane + (size_t)(line0 + r) * L + k0 + k,
                 (uint32_t)(n * sizeof(C)), mbar);
    }
    return mbar_wait_bounded(mbar, err, kWaitTries, phase < 0 ? 0u : (uint32_t)(phase & 1));
}

// The part of a line group one CTA works on: lines line0 .. line0 + nl - 1,
// chunks q0 .. q0 + nq - 1, positions k0 .. k0 + len - 1.  With S > 1 the S CTAs
// of a cluster share the line group (cluster rank = part index).
struct Part {
    int rank, line0, nl, q0, nq, k0, len;
};

__device__ __forceinline__ Part make_part(const LineTiling& T, int cta)
{
    Part P;
    P.rank = T.S > 1 ? (int)cg::this_cluster().block_rank() : 0;
    P.line0 = (cta / T.S) * T.R;
    P.nl = min(T.R, T.nlines - P.line0);
    P.q0 = P.rank * T.Qc;
    P.nq = max(0, min(T.Qc, T.Q - P.q0));
    P.k0 = P.q0 * T.m;
    P.len = max(0, min(T.L, P.k0 + T.Qc * T.m) - P.k0);
    return P;
}

// Barrier over the CTAs that share a line group.
__device__ __forceinline__ void group_sync(const LineTiling& T)
{
    if (T.S > 1)
        cg::this_cluster().sync();
    else
        __syncthreads();
}

// ------------------------------------------------------------------ K1 ----
// One thread per (line, channel), always in FP64 (stored in the pass's
// precision).  The line operator is A = -1/2 D2 + kappa D1 with kappa = i kb;
// the CN system matrix is I + tau A with tau = dt/2 (imaginary time) or i dt/2
// (real time): constant sub-diagonal alpha, diagonal beta, super-diagonal gamma'.
// In imaginary time beta and alpha gamma' = tau^2 (1/(4h^4) + kb^2/(4h^2)) are
// real, so every pivot is real: the recurrence is run in real arithmetic and the
// stored inv has a zero imaginary part, which the sweeps use (a real scaling).
template <typename C>
__global__ void coef_kernel(LineCoefT<C>* coef, int nlines, int dir, int mode, double h, double line_len,
                            double line_h, double dt, double omeg, double gamma, int eta, int* status)
{
    int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= nlines * 3) return;
    int line = id / 3, ch = id - 3 * (id / 3);
    double lam = 1.0 - ch;                                   // channel eigenvalue +1, 0, -1
    double pos = -0.5 * line_len + (line + 0.5) * line_h;    // y_j (x-pass) or x_i (y-pass)
    double kb = dir == 0 ? gamma * lam - omeg * pos : omeg * pos - eta * gamma * lam;
    double2 a = make_double2(-0.5 / (h * h), -kb / (2 * h));
    double2 c = make_double2(-0.5 / (h * h), kb / (2 * h));
    double b = 1.0 / (h * h);
    double2 tau = mode == 1 ? make_double2(0.0, 0.5 * dt) : make_double2(0.5 * dt, 0.0);
    double2 alpha = cmul(tau, a), gam = cmul(tau, c);
    double2 beta = make_double2(1.0 + tau.x * b, tau.y * b);
    LineCoefT<C>& Co = coef[id];
    double2 cprev = make_double2(0.0, 0.0), glast = cprev;
    const double ag = alpha.x * gam.x - alpha.y * gam.y;  // real alpha gamma' (imaginary time)
    double rinv = 0.0;
    for (int k = 0; k < kHead; ++k) {
        double2 inv;
        if (mode == 1) {
            inv = drecip(dsub(beta, cmul(alpha, cprev)));
        } else {
            rinv = 1.0 / (beta.x - ag * rinv);
            inv = make_double2(rinv, 0.0);
        }
        double2 cp = cmul(gam, inv);
        double2 g = cmul(alpha, inv);
        Co.inv[k] = store_as<C>(inv);
        Co.g[k] = store_as<C>(g);
        Co.cp[k] = store_as<C>(cp);
        if (k == kHead - 1) {
            double dlt = hypot(cp.x - cprev.x, cp.y - cprev.y);
            if (!(dlt <= 1e-15 * hypot(cp.x, cp.y) + 1e-300)) atomicOr(status, 1);  // a few ulps
        }
        cprev = cp;
        glast = g;
    }
    double2 mg = make_double2(-glast.x, -glast.y);
    double2 mc = make_double2(-cprev.x, -cprev.y);
    double2 pf = mg, pb = mc;
    for (int t = 0; t < kFix; ++t) {
        Co.pf[t] = store_as<C>(pf);
        Co.pb[t] = store_as<C>(pb);
        pf = cmul(pf, mg);
        pb = cmul(pb, mc);
    }
}

// exp(-tau' w^2 q^2 / 2) on the cell-centred axis q (the separable trap factor
// of the pointwise substep), evaluated in FP64.
template <typename C>
__global__ void trap_table_kernel(C* out, int n, double len, double w, double dt, int mode)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double h = len / n;
    double q = -0.5 * len + (i + 0.5) * h;
    double arg = dt * 0.5 * w * w * q * q;
    if (mode == 1) {
        double s, c;
        sincos(arg, &s, &c);
        out[i] = store_as<C>(make_double2(c, -s));
    } else {
        out[i] = store_as<C>(make_double2(exp(-arg), 0.0));
    }
}

// ------------------------------------------------------- pointwise substep --
// psi <- exp(-tau' H_loc) psi with H_loc = (V + c0 rho) I + B.Sigma,
// B = c2 F + R e_x, F = psi^dagger Sigma psi, frozen at the start of the substep
// (the c2 and Rabi terms of Eqs. S.1-S.2), tau' = dt or i dt.
// Spin-1: (n.Sigma)^3 = n.Sigma, so with M = dt B.Sigma and u = dt^2 |B|^2
//   imaginary: exp(-M) = I - s1(u) M + s2(u) M^2,  s1 = sinh(t)/t, s2 = (cosh t - 1)/t^2
//   real:      exp(-iM) = I - i s1(u) M - s2(u) M^2, s1 = sin(t)/t,  s2 = (1 - cos t)/t^2
// with t = sqrt(u); both are power series in u, used directly: three terms for
// u <= 1e-4 and five for u <= 1/100 (first omitted term <= 2.5e-18 relative).
// The scalar factor exp(-tau' c0 rho) is a Taylor series: eight terms (imaginary
// time) or four plus four (cos, sin in real time) for |dt c0 rho| <= 1/64, and
// eleven/twelve terms up to 1/8 (<= 3e-18); larger arguments take the library
// exp / sincos.  The tiers test |x|: an attractive contact interaction (c0 < 0)
// makes the argument negative, and the truncation bounds depend on |x| only.
// The trap factor comes from the per-axis tables.  The complex64 version evaluates the same formulas in
// FP32 (three-term series for u <= 1/100, library expf / sincosf otherwise).
template <typename R>
struct PConstT {
    R dtc0;  // dt c0 s^2
    R dtc2;  // dt c2 s^2
    R dtr;   // dt R / sqrt(2)
    R s;     // pending normalisation
    R dt;
};

// v = M psi for M = dt B.Sigma, with bx = dt B_x/sqrt2, by = dt B_y/sqrt2, bz = dt B_z.
template <typename C, typename R>
__device__ __forceinline__ void spin_mv(R bx, R by, R bz, C a, C b, C c, C& va, C& vb, C& vc)
{
    // row +1: bz a + (bx - i by) b
    va.x = fma(bz, a.x, fma(bx, b.x, by * b.y));
    va.y = fma(bz, a.y, fma(bx, b.y, -by * b.x));
    // row 0: (bx + i by) a + (bx - i by) c
    vb.x = fma(bx, a.x, fma(-by, a.y, fma(bx, c.x, by * c.y)));
    vb.y = fma(bx, a.y, fma(by, a.x, fma(bx, c.y, -by * c.x)));
    // row -1: (bx + i by) b - bz c
    vc.x = fma(bx, b.x, fma(-by, b.y, -bz * c.x));
    vc.y = fma(bx, b.y, fma(by, b.x, -bz * c.y));
}

// s1, s2 of the spin exponential (see above).
template <int MODE>
__device__ __forceinline__ void spin_series(double u, double& s1, double& s2)
{
    if (u <= 1e-4) {
        // three terms: the first omitted term of s1 is u^3/7! <= 2e-16 and it multiplies
        // M psi, |M psi| <= sqrt(u) |psi| <= 1e-2 |psi|, so psi' changes by <= 2e-18 |psi|
        const double su = MODE == 1 ? -u : u;
        s1 = fma(fma(su, 1.0 / 120.0, 1.0 / 6.0), su, 1.0);
        s2 = fma(fma(su, 1.0 / 720.0, 1.0 / 24.0), su, 0.5);
    } else if (u <= 0.01) {
        const double su = MODE == 1 ? -u : u;
        s1 = fma(fma(fma(fma(su, 1.0 / 362880.0, 1.0 / 5040.0), su, 1.0 / 120.0), su, 1.0 / 6.0), su, 1.0);
        s2 = fma(fma(fma(fma(su, 1.0 / 3628800.0, 1.0 / 40320.0), su, 1.0 / 720.0), su, 1.0 / 24.0), su, 0.5);
    } else {
        double t = sqrt(u);
        if (MODE == 1) {
            double sh = sin(0.5 * t);
            s1 = sin(t) / t;
            s2 = 2.0 * sh * sh / u;
        } else {
            double sh = sinh(0.5 * t);
            s1 = sinh(t) / t;
            s2 = 2.0 * sh * sh / u;
        }
    }
}

template <int MODE>
__device__ __forceinline__ void spin_series(float u, float& s1, float& s2)
{
    if (u <= 0.01f) {
        // first omitted term u^3/7! <= 2e-10 (FP32 rounding is 6e-8)
        const float su = MODE == 1 ? -u : u;
        s1 = fmaf(fmaf(su, 1.0f / 120.0f, 1.0f / 6.0f), su, 1.0f);
        s2 = fmaf(fmaf(su, 1.0f / 720.0f, 1.0f / 24.0f), su, 0.5f);
    } else {
        float t = sqrtf(u);
        if (MODE == 1) {
            float sh = sinf(0.5f * t);
            s1 = sinf(t) / t;
            s2 = 2.0f * sh * sh / u;
        } else {
            float sh = sinhf(0.5f * t);
            s1 = sinhf(t) / t;
            s2 = 2.0f * sh * sh / u;
        }
    }
}

// e^{-x} (imaginary time) and cos x, sin x (real time) of x = dt c0 rho, of
// either sign (c0 < 0 is an attractive interaction).
__device__ __forceinline__ double scalar_exp(double x)
{
    const double mx = -x, ax = fabs(x);
    if (ax <= 0.015625) {
        // eight terms for |x| <= 1/64: the first omitted one is |x|^8/8! <= 1.7e-19
        return fma(fma(fma(fma(fma(fma(fma(mx, 1.0 / 5040.0, 1.0 / 720.0), mx, 1.0 / 120.0), mx, 1.0 / 24.0), mx,
                                1.0 / 6.0), mx, 0.5), mx, 1.0), mx, 1.0);
    } else if (ax <= 0.125) {
        double e = fma(fma(fma(fma(fma(fma(fma(fma(fma(fma(mx, 1.0 / 39916800.0, 1.0 / 3628800.0), mx, 1.0 / 362880.0),
                                                   mx, 1.0 / 40320.0), mx, 1.0 / 5040.0), mx, 1.0 / 720.0),
                                       mx, 1.0 / 120.0), mx, 1.0 / 24.0), mx, 1.0 / 6.0), mx, 0.5), mx, 1.0);
        return fma(e, mx, 1.0);
    }
    return exp(-x);
}
__device__ __forceinline__ float scalar_exp(float x) { return expf(-x); }

__device__ __forceinline__ void scalar_cis(double x, double& cs, double& sn)
{
    const double ax = fabs(x);
    if (ax <= 0.015625) {
        // |x| <= 1/64: the first omitted terms |x|^8/8! and |x|^9/9! are <= 1e-19
        double x2 = x * x;
        cs = fma(fma(fma(x2, -1.0 / 720.0, 1.0 / 24.0), x2, -0.5), x2, 1.0);
        sn = x * fma(fma(fma(x2, -1.0 / 5040.0, 1.0 / 120.0), x2, -1.0 / 6.0), x2, 1.0);
    } else if (ax <= 0.125) {
        double x2 = x * x;
        cs = fma(fma(fma(fma(fma(x2, -1.0 / 3628800.0, 1.0 / 40320.0), x2, -1.0 / 720.0), x2, 1.0 / 24.0), x2, -0.5),
                 x2, 1.0);
        sn = x * fma(fma(fma(fma(fma(x2, -1.0 / 39916800.0, 1.0 / 362880.0), x2, -1.0 / 5040.0), x2, 1.0 / 120.0), x2,
                         -1.0 / 6.0), x2, 1.0);
    } else {
        sincos(x, &sn, &cs);
    }
}
__device__ __forceinline__ void scalar_cis(float x, float& cs, float& sn) { sincosf(x, &sn, &cs); }

// ev: trap factor from the tables (complex128 pass); tv: dt V added to the
// scalar exponent instead (complex64 pass, ev = 1, one expf/sincosf per site).
// In imaginary time the scalar factor s ev exp(-x) is real and is returned in ps,
// not applied: the basis rotation that follows takes it in its two constants.
// In real time it is applied here and ps = 1.
template <int MODE, typename C>
__device__ __forceinline__ void pointwise(C& a, C& b, C& c, C ev, typename RealOf<C>::type tv,
                                          const PConstT<typename RealOf<C>::type>& k, typename RealOf<C>::type& ps)
{
    typedef typename RealOf<C>::type R;
    R rp = fma(a.x, a.x, a.y * a.y);
    R r0 = fma(b.x, b.x, b.y * b.y);
    R rm = fma(c.x, c.x, c.y * c.y);
    R rho = rp + r0 + rm;
    // F_+ / sqrt2 = conj(a) b + conj(b) c
    R fr = fma(a.x, b.x, fma(a.y, b.y, fma(b.x, c.x, b.y * c.y)));
    R fi = fma(a.x, b.y, fma(-a.y, b.x, fma(b.x, c.y, -b.y * c.x)));
    R bx = fma(k.dtc2, fr, k.dtr);
    R by = k.dtc2 * fi;
    R bz = k.dtc2 * (rp - rm);
    R u = fma(R(2), fma(bx, bx, by * by), bz * bz);
    R s1, s2;
    spin_series<MODE>(u, s1, s2);
    C va, vb, vc, wa, wb, wc;
    spin_mv(bx, by, bz, a, b, c, va, vb, vc);
    spin_mv(bx, by, bz, va, vb, vc, wa, wb, wc);
    const R x = fma(k.dtc0, rho, tv);
    if (MODE == 1) {
        // t = psi - i s1 v - s2 w
        C ta = mkc<C>(fma(s1, va.y, fma(-s2, wa.x, a.x)), fma(-s1, va.x, fma(-s2, wa.y, a.y)));
        C tb = mkc<C>(fma(s1, vb.y, fma(-s2, wb.x, b.x)), fma(-s1, vb.x, fma(-s2, wb.y, b.y)));
        C tc = mkc<C>(fma(s1, vc.y, fma(-s2, wc.x, c.x)), fma(-s1, vc.x, fma(-s2, wc.y, c.y)));
        R cs, sn;
        scalar_cis(x, cs, sn);
        // ph = ev exp(-i x): nothing is pending in real time (every real-time
        // step starts from an applied normalisation, s = 1 exactly)
        C ph = mkc<C>(fma(ev.x, cs, ev.y * sn), fma(ev.y, cs, -ev.x * sn));
        a = cmul(ph, ta);
        b = cmul(ph, tb);
        c = cmul(ph, tc);
        ps = R(1);
    } else {
        ps = k.s * ev.x * scalar_exp(x);
        a = mkc<C>(fma(-s1, va.x, fma(s2, wa.x, a.x)), fma(-s1, va.y, fma(s2, wa.y, a.y)));
        b = mkc<C>(fma(-s1, vb.x, fma(s2, wb.x, b.x)), fma(-s1, vb.y, fma(s2, wb.y, b.y)));
        c = mkc<C>(fma(-s1, vc.x, fma(s2, wc.x, c.x)), fma(-s1, vc.y, fma(s2, wc.y, c.y)));
    }
}

// --------------------------------------------------------- basis rotations --
// phi = U_y^dagger (ps psi): Sigma_y eigen-channels lambda = +1, 0, -1 with
// eigenvectors (1, i sqrt2, -1)/2, (1, 0, 1)/sqrt2, (1, -i sqrt2, -1)/2, and a
// real scale ps folded into the constants.
template <typename C>
__device__ __forceinline__ void to_sigma_y(C a, C b, C c, typename RealOf<C>::type ps, C& p, C& z, C& m)
{
    typedef typename RealOf<C>::type R;
    const R rs2 = R(0.70710678118654752440) * ps, half = R(0.5) * ps;
    R dx = half * (a.x - c.x), dy = half * (a.y - c.y);
    p = mkc<C>(fma(rs2, b.y, dx), fma(-rs2, b.x, dy));
    m = mkc<C>(fma(-rs2, b.y, dx), fma(rs2, b.x, dy));
    z = mkc<C>(rs2 * (a.x + c.x), rs2 * (a.y + c.y));
}

// psi = U_y phi (the inverse of to_sigma_y without scale):
//   a = phi_0/sqrt2 + (phi_+ + phi_-)/2,  c = phi_0/sqrt2 - (phi_+ + phi_-)/2,
//   b = i (phi_+ - phi_-)/sqrt2.
template <typename C>
__device__ __forceinline__ void from_sigma_y(C p, C z, C m, C& a, C& b, C& c)
{
    typedef typename RealOf<C>::type R;
    const R rs2 = R(0.70710678118654752440);
    R sx = R(0.5) * (p.x + m.x), sy = R(0.5) * (p.y + m.y);
    R zx = rs2 * z.x, zy = rs2 * z.y;
    a = mkc<C>(zx + sx, zy + sy);
    c = mkc<C>(zx - sx, zy - sy);
    b = mkc<C>(-rs2 * (p.y - m.y), rs2 * (p.x - m.x));
}

// chi = U_x^dagger U_y phi: from Sigma_y channels to Sigma_x channels
// (Sigma_x eigenvectors (1, sqrt2, 1)/2, (1, 0, -1)/sqrt2, (1, -sqrt2, 1)/2):
//   chi_{+-} = phi_0/sqrt2 +- (i/2)(phi_+ - phi_-),  chi_0 = (phi_+ + phi_-)/sqrt2.
template <typename C>
__device__ __forceinline__ void sigma_y_to_x(C p, C z, C m, C& xp, C& x0, C& xm)
{
    typedef typename RealOf<C>::type R;
    const R rs2 = R(0.70710678118654752440);
    R hx = R(0.5) * (p.x - m.x), hy = R(0.5) * (p.y - m.y);
    R zx = rs2 * z.x, zy = rs2 * z.y;
    xp = mkc<C>(zx - hy, zy + hx);
    xm = mkc<C>(zx + hy, zy - hx);
    x0 = mkc<C>(rs2 * (p.x + m.x), rs2 * (p.y + m.y));
}

// psi = U_x chi.
template <typename C>
__device__ __forceinline__ void from_sigma_x(C xp, C x0, C xm, C& a, C& b, C& c)
{
    typedef typename RealOf<C>::type R;
    const R rs2 = R(0.70710678118654752440);
    R sx = R(0.5) * (xp.x + xm.x), sy = R(0.5) * (xp.y + xm.y);
    a = mkc<C>(fma(rs2, x0.x, sx), fma(rs2, x0.y, sy));
    c = mkc<C>(fma(-rs2, x0.x, sx), fma(-rs2, x0.y, sy));
    b = mkc<C>(rs2 * (xp.x - xm.x), rs2 * (xp.y - xm.y));
}

// ------------------------------------------------------- chunked Thomas ----
// Solves (I + tau A) w = phi for every (line, channel) of the CTA and replaces
// phi by psi' = 2 w - phi = (I + tau A)^{-1} (I - tau A) phi.
// Each line is cut into Q chunks of m points, one thread per chunk:
//  1. forward elimination inside the chunk from a zero carry -> y^, chunk end;
//  2. the true y differs by pf[t] * (true end value of the previous chunk) on
//     the chunk's first F points (|pf[t]| below rounding beyond), then back
//     substitution inside the chunk from a zero carry -> w^, chunk start;
//  3. the true w differs by pb[m-1-t] * (true start value of the next chunk) on
//     the chunk's last F points.
// Because m > F, a chunk's local end/start value equals the true one to
// rounding, so no carry has to be propagated sequentially across chunks.
// Smem: line-channel arrays of stride Lp, chunk q at offset q cs (the strides
// keep chunk-parallel accesses on distinct banks).
// In imaginary time (MODE 0) the pivots are real and inv scales phi as a real.
template <int MODE, typename C>
__device__ __forceinline__ C scale_inv(const C& inv, const C& v)
{
    if constexpr (MODE == 0)
        return mkc<C>(inv.x * v.x, inv.x * v.y);
    else
        return cmul(inv, v);
}

template <int MODE, typename C>
__device__ __forceinline__ void chunked_thomas(C* sa, C* sb, C* cf, C* cb, const LineCoefT<C>* coef,
                                               const LineTiling& T, const Part& P)
{
    typedef typename RealOf<C>::type R;
    const int m = T.m, Q = T.Q, F = T.F, L = T.L, Lp = T.Lp, Qc = T.Qc;
    const int nl3 = 3 * max(P.nl, 1);
    const int tid = threadIdx.x;
    const int ql = tid / nl3;              // chunk within the CTA (chunk-major: the
    const int lc = tid - ql * nl3;         // line-start chunks sit in the first warp); r * 3 + ch
    const bool active = ql < P.nq;
    const int q = P.q0 + ql;               // chunk within the line
    const int start = q * m;
    const int len = max(0, min(m, L - start));
    const LineCoefT<C>* Co = coef + lc;    // coef already offset to the CTA's first line
    C* __restrict__ pa = sa + lc * Lp + ql * T.cs;
    C* __restrict__ pbf = sb + lc * Lp + ql * T.cs;
    // carries of the neighbouring CTAs of the cluster (distributed shared memory)
    const C* cf_prev = cf;
    const C* cb_next = cb;
    if (T.S > 1) {
        cg::cluster_group cl = cg::this_cluster();
        if (P.rank > 0) cf_prev = cl.map_shared_rank(cf, P.rank - 1);
        if (P.rank < T.S - 1) cb_next = cl.map_shared_rank(cb, P.rank + 1);
    }

    // Converged factorisation (rows >= kHead - 1) in registers; rows inside the
    // table head are fetched with a predicated load (no divergent branch).
    const C inv_c = Co->inv[kHead - 1], g_c = Co->g[kHead - 1], cp_c = Co->cp[kHead - 1];
    if (active) {
        C y = mkc<C>(R(0), R(0));
#pragma unroll 4
        for (int t = 0; t < len; ++t) {
            const int k = start + t;
            const bool head = k < kHead - 1;
            C inv = inv_c, g = g_c;
            if (head) {
                inv = Co->inv[k];
                g = Co->g[k];
            }
            y = cfnma(g, y, scale_inv<MODE>(inv, pa[t]));
            pbf[t] = y;
        }
        cf[lc * Qc + ql] = y;
    }
    group_sync(T);
    if (active) {
        if (q > 0) {
            C yc = ql > 0 ? cf[lc * Qc + ql - 1] : cf_prev[lc * Qc + Qc - 1];
            int nf = min(F, len);
            if constexpr (sizeof(R) == 4) {
                // complex64: powers (-g_inf)^(t+1) by a running product (no table loads)
                const C mg = mkc<C>(-g_c.x, -g_c.y);
                C pw = mg;
                for (int t = 0; t < nf; ++t) {
                    pbf[t] = cfma(pw, yc, pbf[t]);
                    pw = cmul(pw, mg);
                }
            } else {
                for (int t = 0; t < nf; ++t) pbf[t] = cfma(Co->pf[t], yc, pbf[t]);
            }
        }
        C w = mkc<C>(R(0), R(0));
#pragma unroll 4
        for (int t = len - 1; t >= 0; --t) {
            const int k = start + t;
            C cp = cp_c;
            if (k < kHead - 1) cp = Co->cp[k];
            w = cfnma(cp, w, pbf[t]);
            pbf[t] = w;
        }
        cb[lc * Qc + ql] = w;
    }
    group_sync(T);
    if (active) {
        const bool fix = q < Q - 1;
        C wc = !fix ? mkc<C>(R(0), R(0)) : (ql < P.nq - 1 ? cb[lc * Qc + ql + 1] : cb_next[lc * Qc + 0]);
        const int tf = fix ? len - F : len;  // points t >= tf get the backward fixup
        if constexpr (sizeof(R) == 4) {
            // complex64: powers (-c'_inf)^(len - t) by a running product, applied first
            const C mc = mkc<C>(-cp_c.x, -cp_c.y);
            C pw = mc;
            for (int t = len - 1; t >= tf; --t) {
                pbf[t] = cfma(pw, wc, pbf[t]);
                pw = cmul(pw, mc);
            }
#pragma unroll 4
            for (int t = 0; t < len; ++t) {
                C w = pbf[t];
                C ph = pa[t];
                pa[t] = mkc<C>(fma(R(2), w.x, -ph.x), fma(R(2), w.y, -ph.y));
            }
        } else {
#pragma unroll 4
            for (int t = 0; t < len; ++t) {
                C w = pbf[t];
                if (t >= tf) w = cfma(Co->pb[len - t - 1], wc, w);
                C ph = pa[t];
                pa[t] = mkc<C>(fma(R(2), w.x, -ph.x), fma(R(2), w.y, -ph.y));
            }
        }
    }
    // no CTA of the cluster may leave while its carries can still be read
    group_sync(T);
}

// Converged factorisation of the thread's line-channel (chunk-major mapping:
// lc = tid mod 3 nl), loaded at the start of a pass so that the global-memory
// latency overlaps the staging and pointwise work.
template <typename C>
struct ConvCoef {
    C inv, g, cp;
};

template <typename C>
__device__ __forceinline__ ConvCoef<C> load_conv(const LineCoefT<C>* coef, const Part& P)
{
    const LineCoefT<C>* Co = coef + (int)(threadIdx.x % (unsigned)(3 * max(P.nl, 1)));
    return ConvCoef<C>{Co->inv[kHead - 1], Co->g[kHead - 1], Co->cp[kHead - 1]};
}

// The same solve with the chunk length M fixed at compile time and each
// thread's chunk of y / w held in registers: shared memory is read for phi in
// the forward sweep and in the final step and written once with psi'.
// Chunks q >= 1 start at row m >= H + F, past the rows where the factorisation
// still differs from its limit (H rows) and where the fixup powers matter, so
// they use the converged coefficients throughout; chunk 0 takes the table rows.
// Complex64 moves two points per 16-byte shared-memory access, complex128 one.
template <int MODE, typename C, int M>
__device__ __forceinline__ void chunked_thomas_reg(C* sa, C* cf, C* cb, const LineCoefT<C>* coef,
                                                   const ConvCoef<C>& cc, const LineTiling& T, const Part& P,
                                                   C* hf, C* hb, uint64_t* cbar, int* err)
{
    typedef typename RealOf<C>::type R;
    static_assert(sizeof(C) == 16 || M % 2 == 0, "pairs of complex64 per 16-byte shared-memory access");
    const int Q = T.Q, F = T.F, L = T.L, Lp = T.Lp, Qc = T.Qc;
    const int nl3 = 3 * max(P.nl, 1);
    const int tid = threadIdx.x;
    const int ql = tid / nl3;
    const int lc = tid - ql * nl3;
    const bool active = ql < P.nq;
    const int q = P.q0 + ql;
    const int len = max(0, min(M, L - q * M));
    const LineCoefT<C>* Co = coef + lc;
    C* __restrict__ pa = sa + lc * Lp + ql * T.cs;
    // In a cluster the first chunk of a CTA takes its forward carry from the
    // left neighbour's last chunk (pushed into hf, counted on cbar[0]) and the
    // last chunk its backward carry from the right neighbour's first (hb, cbar[1]).
    const C zero = mkc<C>(R(0), R(0));
    const C inv_c = cc.inv, g_c = cc.g, cp_c = cc.cp;
    C y[M];
    if (active && sizeof(C) == 16) {
        // complex128: forward elimination from a zero carry, one point per access
        C v = zero;
        if (q == 0) {
#pragma unroll
            for (int t = 0; t < M; ++t) {
                const int k = t < kHead - 1 ? t : kHead - 1;
                v = cfnma(Co->g[k], v, scale_inv<MODE>(Co->inv[k], pa[t]));
                y[t] = t < len ? v : zero;
            }
        } else if (len == M) {
#pragma unroll
            for (int t = 0; t < M; ++t) {
                v = cfnma(g_c, v, scale_inv<MODE>(inv_c, pa[t]));
                y[t] = v;
            }
        } else {
#pragma unroll
            for (int t = 0; t < M; ++t) {
                v = cfnma(g_c, v, scale_inv<MODE>(inv_c, pa[t]));
                y[t] = t < len ? v : zero;
            }
        }
        cf[lc * Qc + ql] = y[M - 1];
    } else if (active) {
        // forward elimination from a zero carry; rows past the line end stay zero
        C v = zero;
        // phi two points per 16-byte load (chunk starts are 16-byte aligned)
        const float4* p4 = reinterpret_cast<const float4*>(pa);
        if (q == 0) {
#pragma unroll
            for (int t = 0; t < M; t += 2) {
                const float4 d = p4[t / 2];
                const int k0 = t < kHead - 1 ? t : kHead - 1, k1 = t + 1 < kHead - 1 ? t + 1 : kHead - 1;
                v = cfnma(Co->g[k0], v, scale_inv<MODE>(Co->inv[k0], mkc<C>(d.x, d.y)));
                y[t] = t < len ? v : zero;
                v = cfnma(Co->g[k1], v, scale_inv<MODE>(Co->inv[k1], mkc<C>(d.z, d.w)));
                y[t + 1] = t + 1 < len ? v : zero;
            }
        } else if (len == M) {  // every chunk but a line's last
#pragma unroll
            for (int t = 0; t < M; t += 2) {
                const float4 d = p4[t / 2];
                v = cfnma(g_c, v, scale_inv<MODE>(inv_c, mkc<C>(d.x, d.y)));
                y[t] = v;
                v = cfnma(g_c, v, scale_inv<MODE>(inv_c, mkc<C>(d.z, d.w)));
                y[t + 1] = v;
            }
        } else {
#pragma unroll
            for (int t = 0; t < M; t += 2) {
                const float4 d = p4[t / 2];
                v = cfnma(g_c, v, scale_inv<MODE>(inv_c, mkc<C>(d.x, d.y)));
                y[t] = t < len ? v : zero;
                v = cfnma(g_c, v, scale_inv<MODE>(inv_c, mkc<C>(d.z, d.w)));
                y[t + 1] = t + 1 < len ? v : zero;
            }
        }
        cf[lc * Qc + ql] = y[M - 1];
    }
    if (T.S > 1) {
        cluster_wait();  // start barrier: the neighbours' mbarriers are initialised
        if (active && ql == P.nq - 1 && P.rank < T.S - 1) push_carry(y[M - 1], hf + lc, cbar, P.rank + 1);
    }
    __syncthreads();
    if (active) {
        if (q > 0) {
            C yc;
            if (ql > 0) {
                yc = cf[lc * Qc + ql - 1];
            } else {  // q > 0 with ql == 0: a cluster rank > 0
                wait_carry(cbar, err);
                yc = hf[lc];
            }
            const int nf = min(F, len);
            if constexpr (sizeof(R) == 4) {
                const C mg = mkc<C>(-g_c.x, -g_c.y);
                C pw = mg;
#pragma unroll
                for (int t = 0; t < M; ++t) {
                    if (t >= nf) break;  // one exit branch instead of a predicate per row
                    y[t] = cfma(pw, yc, y[t]);
                    pw = cmul(pw, mg);
                }
            } else {
#pragma unroll
                for (int t = 0; t < M; ++t)
                    if (t < nf) y[t] = cfma(Co->pf[t], yc, y[t]);
            }
        }
        // back substitution from a zero carry
        C w = zero;
        if (q == 0) {
#pragma unroll
            for (int t = M - 1; t >= 0; --t) {
                const int k = t < kHead - 1 ? t : kHead - 1;
                w = cfnma(Co->cp[k], w, y[t]);
                y[t] = w;
            }
        } else {
#pragma unroll
            for (int t = M - 1; t >= 0; --t) {
                w = cfnma(cp_c, w, y[t]);
                y[t] = w;
            }
        }
        cb[lc * Qc + ql] = y[0];
        if (T.S > 1 && ql == 0 && P.rank > 0) push_carry(y[0], hb + lc, cbar + 1, P.rank - 1);
    }
    // No CTA of the cluster may leave while a neighbour's store into its shared
    // memory can be in flight: this CTA's stores are done here (arrive), and the
    // matching cluster_wait() closes the pass, overlapping the store phase.
    if (T.S > 1) cluster_arrive();
    __syncthreads();
    if (active) {
        if (q < Q - 1) {  // full chunk (len == M): the last F points take the backward fixup
            C wc;
            if (ql < P.nq - 1) {
                wc = cb[lc * Qc + ql + 1];
            } else {  // the last chunk of a CTA that is not the line's last: rank < S - 1
                wait_carry(cbar + 1, err);
                wc = hb[lc];
            }
            if constexpr (sizeof(R) == 4) {
                const C mc = mkc<C>(-cp_c.x, -cp_c.y);
                C pw = mc;
#pragma unroll
                for (int t = M - 1; t >= 0; --t) {
                    if (t < M - F) break;
                    y[t] = cfma(pw, wc, y[t]);
                    pw = cmul(pw, mc);
                }
            } else {
#pragma unroll
                for (int t = M - 1; t >= 0; --t)
                    if (t >= M - F) y[t] = cfma(Co->pb[M - 1 - t], wc, y[t]);
            }
        }
        if constexpr (sizeof(C) == 16) {
#pragma unroll
            for (int t = 0; t < M; ++t) {
                if (t >= len) break;
                const C d = pa[t];
                pa[t] = mkc<C>(fma(R(2), y[t].x, -d.x), fma(R(2), y[t].y, -d.y));
            }
        } else {
            // psi' = 2 w - phi, two points per 16-byte access (len is even)
#pragma unroll
            for (int t = 0; t < M; t += 2) {
                if (t >= len) break;
                float4* p4 = reinterpret_cast<float4*>(pa) + t / 2;
                const float4 d = *p4;
                *p4 = make_float4(fma(R(2), y[t].x, -d.x), fma(R(2), y[t].y, -d.y), fma(R(2), y[t + 1].x, -d.z),
                                  fma(R(2), y[t + 1].y, -d.w));
            }
        }
    }
    __syncthreads();  // psi' visible to the whole CTA
}

// Solve of the CTA's lines: the register-resident form when the kernel is
// compiled for the tiling's chunk length M, the shared-memory form for M = 0.
template <int MODE, typename C, int M>
__device__ __forceinline__ void solve_lines(C* sa, C* sb, C* cf, C* cb, const LineCoefT<C>* coef,
                                            const ConvCoef<C>& cc, const LineTiling& T, const Part& P,
                                            uint64_t* cbar, int* err)
{
    if constexpr (M > 0)
        chunked_thomas_reg<MODE, C, M>(sa, cf, cb, coef, cc, T, P, cb + 3 * T.R * T.Qc, cb + 3 * T.R * (T.Qc + 1),
                                       cbar, err);
    else
        chunked_thomas<MODE>(sa, sb, cf, cb, coef, T, P);
}

// Division by a per-CTA constant d as a multiply-high: q = floor(k * ceil(2^32 / d) / 2^32)
// is exact for 0 <= k < 2^32 / d (the rounding-up error of the multiplier adds
// less than k / 2^32 < 1/d to k/d).  A CTA's shared memory holds fewer than
// 2^13 line points, so every index k and divisor d of a pass satisfies k d < 2^26.
struct FastDiv {
    uint32_t mul;  // ceil(2^32 / d); 0 encodes d == 1
    __device__ __forceinline__ explicit FastDiv(int d) : mul(d > 1 ? 0xffffffffu / (uint32_t)d + 1u : 0u) {}
    __device__ __forceinline__ int operator()(int k) const
    {
        return mul ? (int)__umulhi((uint32_t)k, mul) : k;
    }
};

// shared-memory position of line point k: chunk k / m at offset (k / m) cs
struct SPos {
    FastDiv dm;
    int pad;  // cs - m
    __device__ __forceinline__ explicit SPos(const LineTiling& T) : dm(T.m), pad(T.cs - T.m) {}
    __device__ __forceinline__ int operator()(int k) const { return k + dm(k) * pad; }
};

// --------------------------------------------------------------- x-pass ----
// One CTA of the x-pass: lines cta*R .. cta*R + R - 1 of instance A.
// TAIL (second-order splitting, complex128): the solve comes first and the pass
// ends with psi = U_y phi', the pointwise substep, a natural-layout store and the
// per-CTA partial norms (wsum: warp sums).
// phase: null for a CTA that runs one item (the staging barrier is initialised
// here); in a persistent CTA the count of stagings its barrier has completed,
// advanced here, or negative after a staging wait gave up.
template <int MODE, typename C, int M, bool TAIL = false>
__device__ __forceinline__ void xpass_body(const PassArgsT<C>& A, int cta, unsigned char* smem_raw, uint64_t& mbar,
                                           uint64_t* cbar, double* wsum = nullptr, int* phase = nullptr)
{
    typedef typename RealOf<C>::type R;
    const LineTiling& T = A.t;
    C* sa = reinterpret_cast<C*>(smem_raw);
    C* sb = reinterpret_cast<C*>(smem_raw + T.off_b);
    C* cf = reinterpret_cast<C*>(smem_raw + T.off_cf);
    C* cb = reinterpret_cast<C*>(smem_raw + T.off_cb);
    const Part P = make_part(T, cta);
    const int line0 = P.line0, nl = P.nl, Ll = P.len, k0 = P.k0;
    const int nx = A.nx, ny = A.ny, L = T.L;
    const size_t plane = (size_t)nx * ny;
    // stage the CTA's row segments psi[c][j][k0 .. k0 + Ll) into sb ([r][c][k] contiguous).
    // If the bounded wait gives up (status bit set), the CTA still runs every
    // barrier -- the other CTA of its cluster waits on them -- but writes nothing.
    ConvCoef<C> cc{};
    if (M > 0 && A.do_solve) cc = load_conv(A.coef + (size_t)line0 * 3, P);
    if constexpr (M > 0) {
        if (T.S > 1) {  // carry mbarriers, then the start half of the cluster barrier
            if (threadIdx.x == 0) {
                mbar_init(&cbar[0], 3 * nl);
                mbar_init(&cbar[1], 3 * nl);
            }
            cluster_arrive_relaxed();
        }
    }
    // pending normalisation, loaded before the staging wait (complex64 pass)
    double sd = 0.0;
    if constexpr (sizeof(R) == 4) sd = *A.scale;
    // with one line array (M > 0) the chunks are staged in place
    bool ok = true;
    if (T.bulk && Ll > 0) {
        const int ph = phase ? *phase : -1;
        if constexpr (M > 0)
            ok = stage_chunks(sa, A.in, plane, line0, nl, L, k0, Ll, T.m, T.cs, T.Lp, &mbar, A.err, ph);
        else
            ok = stage_rows(sb, A.in, plane, line0, nl, L, k0, Ll, Ll, &mbar, A.err, ph);
        if (phase) *phase = ok ? ph + 1 : -1;
    }

    // Pointwise constants.  The complex64 pass takes them rounded to FP32 on the
    // host and converts only the pending normalisation in each thread (FP64
    // instructions are costly on this part even inside the complex64 pass); the
    // complex128 pass computes them once in thread 0 and broadcasts them.
    struct KC {
        PConstT<R> k;
        R fx0, fdx, fy0, fdy, hx, hy;  // grid and trap constants (complex64 pass)
    };
    KC kk;
    if constexpr (sizeof(R) == 4) {
        const float s = (float)sd;
        kk.k.dtc0 = A.kf[0] * s * s;
        kk.k.dtc2 = A.kf[1] * s * s;
        kk.k.dtr = A.kf[2];
        kk.k.s = s;
        kk.k.dt = A.kf[3];
        kk.fx0 = A.kf[4];
        kk.fdx = A.kf[5];
        kk.fy0 = A.kf[6];
        kk.fdy = A.kf[7];
        kk.hx = A.kf[8];
        kk.hy = A.kf[9];
    } else {
        __shared__ KC kc;
        if (threadIdx.x == 0) {
            sd = *A.scale;
            kc.k.dtc0 = A.dt * A.c0 * sd * sd;
            kc.k.dtc2 = A.dt * A.c2 * sd * sd;
            kc.k.dtr = A.dt * A.rabi * 0.70710678118654752440;
            kc.k.s = sd;
            kc.k.dt = A.dt;
        }
        __syncthreads();
        kk = kc;
    }
    const PConstT<R> k = kk.k;
    const KC& tk = kk;
    const FastDiv div_len(Ll), div_nl(nl);
    const SPos spos(T);
    const int Lp = T.Lp;
    // P (when asked) and U_y^dagger of the site (i, j)
    auto site = [&](C a, C b, C c, int i, int j, C& p, C& z, C& m) {
        R ps;
        if (A.do_p) {
            if constexpr (sizeof(R) == 8) {
                // trap factor from the per-axis tables (real in imaginary time)
                C ev = MODE == 1 ? cmul(A.ex[i], A.ey[j]) : mkc<C>(A.ex[i].x * A.ey[j].x, R(0));
                pointwise<MODE>(a, b, c, ev, R(0), k, ps);
            } else {
                // complex64: dt V joins the scalar exponent (no table loads)
                const R xx = fma(R(i), tk.fdx, tk.fx0), yy = fma(R(j), tk.fdy, tk.fy0);
                const R tv = fma(tk.hx * xx, xx, tk.hy * yy * yy);
                pointwise<MODE>(a, b, c, mkc<C>(R(1), R(0)), tv, k, ps);
            }
        } else {
            ps = k.s;  // channels pass through, with the pending normalisation
        }
        to_sigma_y(a, b, c, ps, p, z, m);
    };
    bool paired = false;
    if constexpr (M > 0 && sizeof(C) == 8) {
        if (T.bulk) {
            // Pairs of neighbouring sites (kl even): a chunk holds an even number of
            // points and starts on a 16-byte boundary, so each component of the
            // pair moves as one 16-byte access; the chunk index is a division by
            // the compile-time chunk length.
            paired = true;
            const int Lh = Ll >> 1, pad = T.cs - M, q4 = Lp >> 1;
            const FastDiv div_lh(Lh);
            for (int q = threadIdx.x; threadIdx.x < T.threads && q < nl * Lh; q += T.threads) {
                const int r = div_lh(q), kl = 2 * (q - r * Lh), i = k0 + kl, j = line0 + r;
                float4* row = reinterpret_cast<float4*>(sa + r * 3 * Lp + kl + (kl / M) * pad);
                const float4 va = row[0], vb = row[q4], vc = row[2 * q4];
                C p0, z0, m0, p1, z1, m1;
                site(mkc<C>(va.x, va.y), mkc<C>(vb.x, vb.y), mkc<C>(vc.x, vc.y), i, j, p0, z0, m0);
                site(mkc<C>(va.z, va.w), mkc<C>(vb.z, vb.w), mkc<C>(vc.z, vc.w), i + 1, j, p1, z1, m1);
                row[0] = make_float4(p0.x, p0.y, p1.x, p1.y);
                row[q4] = make_float4(z0.x, z0.y, z1.x, z1.y);
                row[2 * q4] = make_float4(m0.x, m0.y, m1.x, m1.y);
            }
        }
    }
    for (int e = threadIdx.x; !paired && threadIdx.x < T.threads && e < nl * Ll; e += T.threads) {
        int r = div_len(e), kl = e - r * Ll, i = k0 + kl, j = line0 + r;
        C a, b, c;
        if (T.bulk) {
            const int ss = M > 0 ? Lp : Ll;
            const C* row = M > 0 ? sa + r * 3 * Lp + spos(kl) : sb + (size_t)r * 3 * Ll + kl;
            a = row[0];
            b = row[ss];
            c = row[2 * ss];
        } else {
            size_t o = (size_t)j * nx + i;
            a = A.in[o];
            b = A.in[plane + o];
            c = A.in[2 * plane + o];
        }
        C p, z, m;
        site(a, b, c, i, j, p, z, m);
        C* dst = sa + r * 3 * Lp + spos(kl);
        dst[0] = p;
        dst[Lp] = z;
        dst[2 * Lp] = m;
    }
    __syncthreads();
    if (A.do_solve) solve_lines<MODE, C, M>(sa, sb, cf, cb, A.coef + (size_t)line0 * 3, cc, T, P, cbar, A.err);
    if constexpr (TAIL) {
        // psi = U_y phi', then the pointwise substep (constants of this pass),
        // stored in natural layout; consecutive threads -> consecutive i
        R acc = R(0);
        for (int e = threadIdx.x; threadIdx.x < T.threads && e < nl * Ll; e += T.threads) {
            int r = div_len(e), kl = e - r * Ll, i = k0 + kl, j = line0 + r;
            const C* src = sa + r * 3 * Lp + spos(kl);
            C a, b, c;
            from_sigma_y(src[0], src[Lp], src[2 * Lp], a, b, c);
            C ev = MODE == 1 ? cmul(A.ex[i], A.ey[j]) : mkc<C>(A.ex[i].x * A.ey[j].x, R(0));
            R ps;
            pointwise<MODE>(a, b, c, ev, R(0), k, ps);
            a = mkc<C>(ps * a.x, ps * a.y);
            b = mkc<C>(ps * b.x, ps * b.y);
            c = mkc<C>(ps * c.x, ps * c.y);
            if (!ok) continue;
            size_t o = (size_t)j * nx + i;
            A.out[o] = a;
            A.out[plane + o] = b;
            A.out[2 * plane + o] = c;
            acc += fma(a.x, a.x, a.y * a.y) + fma(b.x, b.x, b.y * b.y) + fma(c.x, c.x, c.y * c.y);
        }
        if (A.partials) {
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
            if (lane == 0) wsum[warp] = acc;
            __syncthreads();
            if (threadIdx.x == 0) {
                double t = 0.0;
                for (int w = 0; w < nw; ++w) t += wsum[w];
                A.partials[cta] = t;
            }
        }
        return;
    }
    // transposed store t[mu][i][j], consecutive threads -> consecutive j
    bool pstore = false;
    if constexpr (M > 0 && sizeof(C) == 8) {
        if (((nl | ny | line0) & 1) == 0) {
            // lines j, j + 1 (j even) at the same i: one 16-byte store per channel
            pstore = true;
            const int nh = nl >> 1, pad = T.cs - M;
            const size_t ph = plane >> 1;
            const FastDiv div_nh(nh);
            for (int q = threadIdx.x; threadIdx.x < T.threads && q < nh * Ll; q += T.threads) {
                const int kl = div_nh(q), r = 2 * (q - kl * nh), i = k0 + kl, j = line0 + r;
                const C* s0 = sa + r * 3 * Lp + kl + (kl / M) * pad;
                const C* s1 = s0 + 3 * Lp;
                C xp0, x00, xm0, xp1, x01, xm1;
                sigma_y_to_x(s0[0], s0[Lp], s0[2 * Lp], xp0, x00, xm0);
                sigma_y_to_x(s1[0], s1[Lp], s1[2 * Lp], xp1, x01, xm1);
                if (!ok) continue;
                float4* o = reinterpret_cast<float4*>(A.out + (size_t)i * ny + j);
                o[0] = make_float4(xp0.x, xp0.y, xp1.x, xp1.y);
                o[ph] = make_float4(x00.x, x00.y, x01.x, x01.y);
                o[2 * ph] = make_float4(xm0.x, xm0.y, xm1.x, xm1.y);
            }
        }
    }
    for (int e = threadIdx.x; !pstore && threadIdx.x < T.threads && e < nl * Ll; e += T.threads) {
        int kl = div_nl(e), r = e - kl * nl, i = k0 + kl, j = line0 + r;
        C xp, x0, xm;
        const C* src = sa + r * 3 * Lp + spos(kl);
        sigma_y_to_x(src[0], src[Lp], src[2 * Lp], xp, x0, xm);
        if (!ok) continue;
        size_t o = (size_t)i * ny + j;
        A.out[o] = xp;
        A.out[plane + o] = x0;
        A.out[2 * plane + o] = xm;
    }
    if constexpr (M > 0) {
        if (T.S > 1) cluster_wait();  // no neighbour store into this CTA is still in flight
    }
}

// Single-instance passes with the shared-memory solve.
template <int MODE, typename C>
__global__ void __launch_bounds__(512) xpass_kernel(PassArgsT<C> A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t mbar;
    __shared__ uint64_t cbar[2];
    xpass_body<MODE, C, 0>(A, blockIdx.x, smem_raw, mbar, cbar);
}

// The closing x-pass of a second-order step (complex128): solve, U_y, pointwise
// substep, natural-layout store, partial norms.
template <int MODE>
__global__ void __launch_bounds__(512) xtail_kernel(PassArgs A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t mbar;
    __shared__ uint64_t cbar[2];
    __shared__ double wsum[32];
    xpass_body<MODE, double2, 0, true>(A, blockIdx.x, smem_raw, mbar, cbar, wsum);
}

// With the register-resident solve of chunk length M (one-array tilings).  The
// complex64 register caps (a few dozen bytes of spill at most) keep five to ten
// CTAs per SM; complex128 (M = 32, 128 registers of chunk) takes 168 registers,
// four CTAs of 96 threads, so its CTAs have at most 384 threads.
template <typename C>
constexpr int reg_cap(int M)
{
    return sizeof(C) == 16 ? 168 : (M == 16 ? 64 : (M == 24 ? 80 : 96));
}
template <typename C>
constexpr int reg_threads()
{
    return sizeof(C) == 16 ? 384 : 512;
}

template <int MODE, typename C, int M>
__global__ void __launch_bounds__(reg_threads<C>()) __maxnreg__(reg_cap<C>(M)) xpass_kernel_reg(PassArgsT<C> A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t mbar;
    __shared__ uint64_t cbar[2];
    xpass_body<MODE, C, M>(A, blockIdx.x, smem_raw, mbar, cbar);
}

// --------------------------------------------------------------- y-pass ----
// Partial norms: each thread sums its sites' |psi|^2 in the pass's precision
// (a few dozen sites), the CTA then adds the threads' sums in FP64.
// phase: as for the x-pass.
template <int MODE, typename C, int M>
__device__ __forceinline__ void ypass_body(const PassArgsT<C>& A, int cta, unsigned char* smem_raw, uint64_t& mbar,
                                           double* wsum, uint64_t* cbar, int* phase = nullptr)
{
    typedef typename RealOf<C>::type R;
    const LineTiling& T = A.t;
    C* sa = reinterpret_cast<C*>(smem_raw);
    C* sb = reinterpret_cast<C*>(smem_raw + T.off_b);
    C* cf = reinterpret_cast<C*>(smem_raw + T.off_cf);
    C* cb = reinterpret_cast<C*>(smem_raw + T.off_cb);
    const Part P = make_part(T, cta);
    const int line0 = P.line0, nl = P.nl, Ll = P.len, k0 = P.k0;
    const int nx = A.nx, ny = A.ny, L = T.L;
    const size_t plane = (size_t)nx * ny;
    // stage the CTA's row segments t[mu][i][k0 .. k0 + Ll) into sb ([r][mu][k] contiguous);
    // on a timeout the CTA runs every barrier but writes nothing (see the x-pass)
    ConvCoef<C> cc{};
    if (M > 0 && A.do_solve) cc = load_conv(A.coef + (size_t)line0 * 3, P);
    if constexpr (M > 0) {
        if (T.S > 1) {  // carry mbarriers, then the start half of the cluster barrier
            if (threadIdx.x == 0) {
                mbar_init(&cbar[0], 3 * nl);
                mbar_init(&cbar[1], 3 * nl);
            }
            cluster_arrive_relaxed();
        }
    }
    // The chunks are staged straight into their slots of the line array, one
    // bulk copy per chunk, and need no copy: with one line array (M > 0), and for
    // complex128, whose 16-byte elements keep every chunk copy 16-byte aligned.
    // Complex64 with the shared-memory solve stages whole rows and copies them in.
    constexpr bool in_place = M > 0 || sizeof(C) == 16;
    bool ok = true;
    if (T.bulk && Ll > 0) {
        const int ph = phase ? *phase : -1;
        if constexpr (in_place)
            ok = stage_chunks(sa, A.in, plane, line0, nl, L, k0, Ll, T.m, T.cs, T.Lp, &mbar, A.err, ph);
        else
            ok = stage_rows(sb, A.in, plane, line0, nl, L, k0, Ll, Ll, &mbar, A.err, ph);
        if (phase) *phase = ok ? ph + 1 : -1;
    }

    const FastDiv div_len(Ll), div_nl(nl);
    const SPos spos(T);
    const int Lp = T.Lp;
    const bool copy_in = !(in_place && T.bulk);
    for (int e = threadIdx.x; copy_in && threadIdx.x < T.threads && e < nl * Ll; e += T.threads) {
        int r = div_len(e), kl = e - r * Ll, j = k0 + kl, i = line0 + r;
        C* dst = sa + r * 3 * Lp + spos(kl);
        if (T.bulk) {
            const C* row = sb + (size_t)r * 3 * Ll + kl;
            dst[0] = row[0];
            dst[Lp] = row[Ll];
            dst[2 * Lp] = row[2 * Ll];
        } else {
            size_t o = (size_t)i * ny + j;
            dst[0] = A.in[o];
            dst[Lp] = A.in[plane + o];
            dst[2 * Lp] = A.in[2 * plane + o];
        }
    }
    __syncthreads();
    if (A.do_solve) solve_lines<MODE, C, M>(sa, sb, cf, cb, A.coef + (size_t)line0 * 3, cc, T, P, cbar, A.err);
    R acc = R(0), acc3[3] = {R(0), R(0), R(0)};
    auto tally = [&](C a, C b, C c) {
        if (A.mcomp) {
            acc3[0] += fma(a.x, a.x, a.y * a.y);
            acc3[1] += fma(b.x, b.x, b.y * b.y);
            acc3[2] += fma(c.x, c.x, c.y * c.y);
        } else {
            acc += fma(a.x, a.x, a.y * a.y) + fma(b.x, b.x, b.y * b.y) + fma(c.x, c.x, c.y * c.y);
        }
    };
    bool pstore = false;
    if constexpr (M > 0 && sizeof(C) == 8) {
        if (((nl | nx | line0) & 1) == 0) {
            // columns i, i + 1 (i even) at the same j: one 16-byte store per component
            pstore = true;
            const int nh = nl >> 1, pad = T.cs - M;
            const size_t ph = plane >> 1;
            const FastDiv div_nh(nh);
            for (int q = threadIdx.x; threadIdx.x < T.threads && q < nh * Ll; q += T.threads) {
                const int kl = div_nh(q), r = 2 * (q - kl * nh), j = k0 + kl, i = line0 + r;
                const C* s0 = sa + r * 3 * Lp + kl + (kl / M) * pad;
                const C* s1 = s0 + 3 * Lp;
                C a0, b0, c0, a1, b1, c1;
                from_sigma_x(s0[0], s0[Lp], s0[2 * Lp], a0, b0, c0);
                from_sigma_x(s1[0], s1[Lp], s1[2 * Lp], a1, b1, c1);
                if (!ok) continue;
                float4* o = reinterpret_cast<float4*>(A.out + (size_t)j * nx + i);
                o[0] = make_float4(a0.x, a0.y, a1.x, a1.y);
                o[ph] = make_float4(b0.x, b0.y, b1.x, b1.y);
                o[2 * ph] = make_float4(c0.x, c0.y, c1.x, c1.y);
                tally(a0, b0, c0);
                tally(a1, b1, c1);
            }
        }
    }
    for (int e = threadIdx.x; !pstore && threadIdx.x < T.threads && e < nl * Ll; e += T.threads) {
        int kl = div_nl(e), r = e - kl * nl, j = k0 + kl, i = line0 + r;
        C a, b, c;
        const C* src = sa + r * 3 * Lp + spos(kl);
        from_sigma_x(src[0], src[Lp], src[2 * Lp], a, b, c);
        if (!ok) continue;
        size_t o = (size_t)j * nx + i;
        A.out[o] = a;
        A.out[plane + o] = b;
        A.out[2 * plane + o] = c;
        tally(a, b, c);
    }
    if (A.partials && A.mcomp) {
        // per-component partials (magnetisation-constrained normalisation)
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
        for (int cc = 0; cc < 3; ++cc) {
            R racc = acc3[cc];
            for (int off = 16; off > 0; off >>= 1) racc += __shfl_xor_sync(0xffffffffu, racc, off);
            if (lane == 0) wsum[warp] = (double)racc;
            __syncthreads();
            if (threadIdx.x == 0) {
                double t = 0.0;
                for (int w = 0; w < nw; ++w) t += wsum[w];
                A.partials[3 * cta + cc] = t;
            }
            __syncthreads();
        }
    } else if (A.partials) {
        // warp sums in the pass precision, widened once per warp, CTA sum in FP64
        R racc = acc;
        for (int off = 16; off > 0; off >>= 1) racc += __shfl_xor_sync(0xffffffffu, racc, off);
        double dacc = (double)racc;
        // threads past T.threads (batched launches) hold acc = 0: the sum is the
        // same as in a launch of exactly T.threads threads
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
        if (lane == 0) wsum[warp] = dacc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += wsum[w];
            A.partials[cta] = t;
        }
    }
    if constexpr (M > 0) {
        if (T.S > 1) cluster_wait();  // no neighbour store into this CTA is still in flight
    }
}

template <int MODE, typename C>
__global__ void __launch_bounds__(512) ypass_kernel(PassArgsT<C> A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t mbar;
    __shared__ uint64_t cbar[2];
    __shared__ double wsum[32];
    ypass_body<MODE, C, 0>(A, blockIdx.x, smem_raw, mbar, wsum, cbar);
}

template <int MODE, typename C, int M>
__global__ void __launch_bounds__(reg_threads<C>()) __maxnreg__(reg_cap<C>(M)) ypass_kernel_reg(PassArgsT<C> A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t mbar;
    __shared__ uint64_t cbar[2];
    __shared__ double wsum[32];
    ypass_body<MODE, C, M>(A, blockIdx.x, smem_raw, mbar, wsum, cbar);
}

// ------------------------------------------------------- batched passes ----
// Many instances in one launch, over work items (instance, cta) of the pass.
// work == null: CTA b runs item b (the grid is the list's capacity; CTAs past
// *n_items exit at once).  Otherwise the launch is persistent: at most one CTA
// per resident slot, each taking the next item from the counter work[0] until
// the list is exhausted; the last CTA to finish resets work[0..1] to zero for
// the next launch.  Either way an item runs the single-instance pass body with
// its instance's tiling, so its results do not depend on the launch form.
template <bool X, int MODE, typename C, int M>
__device__ __forceinline__ void batched_item(const PassArgsT<C>& A, int cta, unsigned char* smem_raw, uint64_t& mbar,
                                             uint64_t* cbar, double* wsum, int* phase)
{
    if constexpr (X)
        xpass_body<MODE, C, M>(A, cta, smem_raw, mbar, cbar, nullptr, phase);
    else
        ypass_body<MODE, C, M>(A, cta, smem_raw, mbar, wsum, cbar, phase);
}

// One CTA per work item (the grid is the list's capacity; CTAs past *n_items exit at once).
template <bool X, int MODE, typename C, int M>
__device__ __forceinline__ void batched_one(const PassArgsT<C>* args, const int2* items, const int* n_items)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t mbar;
    __shared__ uint64_t cbar[2];
    __shared__ double wsum[32];
    if ((int)blockIdx.x >= *n_items) return;
    const int2 it = items[blockIdx.x];
    const PassArgsT<C> A = args[it.x];
    batched_item<X, MODE, C, M>(A, it.y, smem_raw, mbar, cbar, wsum, nullptr);
}

// Persistent: each CTA takes items from the counter work[0] until the list is
// exhausted; the last CTA to finish resets work[0..1] to zero for the next launch.
template <bool X, int MODE, typename C, int M>
__device__ __forceinline__ void batched_loop(const PassArgsT<C>* args, const int2* items, const int* n_items,
                                             int* work)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t mbar;
    __shared__ uint64_t cbar[2];
    __shared__ double wsum[32];
    __shared__ int next;
    const int n = *n_items;
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        next = atomicAdd(work, 1);
    }
    int phase = 0;
    __syncthreads();  // publishes the first item and the barrier initialisation
    int b = next;
    while (b < n) {
        // the next item is taken now and read after this one: the counter's
        // round trip overlaps the item's work
        int take = 0;
        if (threadIdx.x == 0) take = atomicAdd(work, 1);
        const int2 it = items[b];
        const PassArgsT<C> A = args[it.x];
        batched_item<X, MODE, C, M>(A, it.y, smem_raw, mbar, cbar, wsum, &phase);
        // this item's shared-memory writes come before the next item's bulk copies
        // into the same bytes (generic proxy before async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (threadIdx.x == 0) next = take;
        __syncthreads();
        // a staging wait gave up (status bit 8): leave the barrier unused (the item
        // taken last is not run; the instance's status reports the failure)
        if (phase < 0) break;
        b = next;
    }
    if (threadIdx.x == 0) {
        __threadfence();  // this CTA's last take from work[0] comes before its count below
        if (atomicAdd(work + 1, 1) == (int)gridDim.x - 1) {
            work[0] = 0;
            work[1] = 0;
        }
    }
}

// shared-memory solve (complex128; complex64 tilings with two line arrays)
template <bool X, int MODE, typename C>
__global__ void __launch_bounds__(512) pass_batched(const PassArgsT<C>* args, const int2* items, const int* n_items)
{
    batched_one<X, MODE, C, 0>(args, items, n_items);
}

template <bool X, int MODE, typename C>
__global__ void __launch_bounds__(512) pass_persistent(const PassArgsT<C>* args, const int2* items,
                                                       const int* n_items, int* work)
{
    batched_loop<X, MODE, C, 0>(args, items, n_items, work);
}

// register-resident solve: every item's tiling is a one-array tiling of chunk length M
template <bool X, int MODE, typename C, int M>
__global__ void __launch_bounds__(512) __maxnreg__(reg_cap<C>(M))
    pass_batched_reg(const PassArgsT<C>* args, const int2* items, const int* n_items)
{
    batched_one<X, MODE, C, M>(args, items, n_items);
}

template <bool X, int MODE, typename C, int M>
__global__ void __launch_bounds__(512) __maxnreg__(reg_cap<C>(M))
    pass_persistent_reg(const PassArgsT<C>* args, const int2* items, const int* n_items, int* work)
{
    batched_loop<X, MODE, C, M>(args, items, n_items, work);
}

// ------------------------------------------------------------- launchers ---
template <typename C>
static int launch_coef_t(LineCoefT<C>* coef, int nlines, int dir, int mode, double h, double line_len,
                         double line_h, double dt, double omeg, double gamma, int eta, int* status, cudaStream_t st)
{
    int n = nlines * 3;
    coef_kernel<C><<<(n + 127) / 128, 128, 0, st>>>(coef, nlines, dir, mode, h, line_len, line_h, dt, omeg, gamma,
                                                     eta, status);
    return report_cuda(cudaGetLastError(), "coef_kernel launch");
}

int launch_coef(LineCoef* coef, int nlines, int dir, int mode, double h, double line_len, double line_h, double dt,
                double omeg, double gamma, int eta, int* status, cudaStream_t st)
{
    return launch_coef_t(coef, nlines, dir, mode, h, line_len, line_h, dt, omeg, gamma, eta, status, st);
}

int launch_coef(LineCoefF* coef, int nlines, int dir, int mode, double h, double line_len, double line_h, double dt,
                double omeg, double gamma, int eta, int* status, cudaStream_t st)
{
    return launch_coef_t(coef, nlines, dir, mode, h, line_len, line_h, dt, omeg, gamma, eta, status, st);
}

int launch_trap_table(double2* out, int n, double len, double w, double dt, int mode, cudaStream_t st)
{
    trap_table_kernel<<<(n + 127) / 128, 128, 0, st>>>(out, n, len, w, dt, mode);
    return report_cuda(cudaGetLastError(), "trap_table_kernel launch");
}

int launch_trap_table(float2* out, int n, double len, double w, double dt, int mode, cudaStream_t st)
{
    trap_table_kernel<<<(n + 127) / 128, 128, 0, st>>>(out, n, len, w, dt, mode);
    return report_cuda(cudaGetLastError(), "trap_table_kernel launch");
}

// Opt in to the dynamic shared memory a launch needs (static shared memory of
// the kernel counts against the same per-block limit).
template <typename K, typename A>
static int launch_pass(K kernel, const A& a, cudaStream_t st)
{
    if (a.t.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a.t.smem);
        if (e != cudaSuccess) return report_cuda(e, "cudaFuncSetAttribute(line pass)");
    }
    const int grid = (a.t.nlines + a.t.R - 1) / a.t.R * a.t.S;
    if (a.t.S == 1) {
        kernel<<<grid, a.t.threads, a.t.smem, st>>>(a);
        return report_cuda(cudaGetLastError(), "line pass launch");
    }
    // a line group spans a cluster of S CTAs
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(a.t.threads);
    cfg.dynamicSmemBytes = a.t.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = a.t.S;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return report_cuda(cudaLaunchKernelEx(&cfg, kernel, a), "line pass cluster launch");
}

// Kernel for the tiling: a one-array complex64 tiling (m = 16, 24, 32) runs the
// register-resident solve compiled for its m, every other tiling the
// shared-memory solve.
template <bool X, int MODE, typename C>
static int launch_line_pass(const PassArgsT<C>& a, cudaStream_t st)
{
    if (a.t.single) {
        if constexpr (sizeof(C) == sizeof(double2)) {
            if (a.t.m == 32)
                return X ? launch_pass(xpass_kernel_reg<MODE, C, 32>, a, st)
                         : launch_pass(ypass_kernel_reg<MODE, C, 32>, a, st);
        }
        if constexpr (sizeof(C) == sizeof(float2)) {
            switch (a.t.m) {
            case 16: return X ? launch_pass(xpass_kernel_reg<MODE, C, 16>, a, st) : launch_pass(ypass_kernel_reg<MODE, C, 16>, a, st);
            case 24: return X ? launch_pass(xpass_kernel_reg<MODE, C, 24>, a, st) : launch_pass(ypass_kernel_reg<MODE, C, 24>, a, st);
            case 32: return X ? launch_pass(xpass_kernel_reg<MODE, C, 32>, a, st) : launch_pass(ypass_kernel_reg<MODE, C, 32>, a, st);
            default: break;
            }
        }
        return GP_ERR_ARG;  // one line array only with a register-resident solve (complex64 m = 16/24/32,
                            // complex128 m = 32)
    }
    return X ? launch_pass(xpass_kernel<MODE, C>, a, st) : launch_pass(ypass_kernel<MODE, C>, a, st);
}

int launch_xtail(const PassArgs& a, int mode, cudaStream_t st)
{
    return mode == 1 ? launch_pass(xtail_kernel<1>, a, st) : launch_pass(xtail_kernel<0>, a, st);
}

int launch_xpass(const PassArgs& a, int mode, cudaStream_t st)
{
    return mode == 1 ? launch_line_pass<true, 1>(a, st) : launch_line_pass<true, 0>(a, st);
}

int launch_ypass(const PassArgs& a, int mode, cudaStream_t st)
{
    return mode == 1 ? launch_line_pass<false, 1>(a, st) : launch_line_pass<false, 0>(a, st);
}

int launch_xpass(const PassArgsF& a, int mode, cudaStream_t st)
{
    return mode == 1 ? launch_line_pass<true, 1>(a, st) : launch_line_pass<true, 0>(a, st);
}

int launch_ypass(const PassArgsF& a, int mode, cudaStream_t st)
{
    return mode == 1 ? launch_line_pass<false, 1>(a, st) : launch_line_pass<false, 0>(a, st);
}

// Resident CTAs per SM of a batched kernel at the launch's threads and dynamic
// shared memory (cached: a tick issues the same few launch shapes many times).
template <typename K>
static int resident_slots(K kernel, int threads, size_t smem)
{
    struct Entry {
        const void* k;
        int threads;
        size_t smem;
        int slots;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    std::lock_guard<std::mutex> lock(mu);
    for (const Entry& e : cache)
        if (e.k == (const void*)kernel && e.threads == threads && e.smem == smem) return e.slots;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess)
        return -1;
    const int slots = std::max(1, per_sm) * sms;
    cache.push_back(Entry{(const void*)kernel, threads, smem, slots});
    return slots;
}

// Batched launches: threads and dynamic shared memory the maximum over the
// batch's instances.  work == null: kernel `one`, grid = capacity items (CTAs
// past *n_items exit at once); otherwise kernel `loop`, persistent, grid =
// min(capacity, resident slots, max_ctas if > 0).
template <typename C, typename K1, typename KP>
static int launch_batched_t(K1 one, KP loop, const PassArgsT<C>* args, const int2* items, const int* n_items,
                            int capacity, int threads, size_t smem, int* work, int max_ctas, cudaStream_t st)
{
    if (capacity <= 0) return 0;
    if (smem > 48 * 1024) {
        cudaError_t e = work ? cudaFuncSetAttribute(loop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                             : cudaFuncSetAttribute(one, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return report_cuda(e, "cudaFuncSetAttribute(batched pass)");
    }
    if (!work) {
        one<<<capacity, threads, smem, st>>>(args, items, n_items);
        return report_cuda(cudaGetLastError(), "batched pass launch");
    }
    const int slots = resident_slots(loop, threads, smem);
    if (slots < 0) return report_cuda(cudaGetLastError(), "occupancy of a batched pass");
    int grid = std::min(capacity, slots);
    if (max_ctas > 0) grid = std::min(grid, max_ctas);
    loop<<<grid, threads, smem, st>>>(args, items, n_items, work);
    return report_cuda(cudaGetLastError(), "persistent batched pass launch");
}

template <bool X, int MODE, typename C>
static int launch_batched_m(const PassArgsT<C>* args, const int2* items, const int* n_items, int capacity,
                            int threads, size_t smem, int* work, int max_ctas, cudaStream_t st, int m_reg)
{
#define GP_BATCHED(M)                                                                                          \
    launch_batched_t(pass_batched_reg<X, MODE, C, M>, pass_persistent_reg<X, MODE, C, M>, args, items, n_items, \
                     capacity, threads, smem, work, max_ctas, st)
    if (m_reg == 0)
        return launch_batched_t(pass_batched<X, MODE, C>, pass_persistent<X, MODE, C>, args, items, n_items,
                                capacity, threads, smem, work, max_ctas, st);
    if constexpr (sizeof(C) == sizeof(float2)) {  // the register-resident solve is complex64 only
        switch (m_reg) {
        case 16: return GP_BATCHED(16);
        case 24: return GP_BATCHED(24);
        case 32: return GP_BATCHED(32);
        default: break;
        }
    }
    return GP_ERR_ARG;
#undef GP_BATCHED
}

int launch_xpass_batched(const PassArgs* args, const int2* items, const int* n_items, int capacity, int threads,
                         size_t smem, int mode, cudaStream_t st, int m_reg, int* work, int max_ctas)
{
    if (m_reg) return GP_ERR_ARG;  // complex128 tilings use the shared-memory solve
    return mode == 1
               ? launch_batched_m<true, 1>(args, items, n_items, capacity, threads, smem, work, max_ctas, st, 0)
               : launch_batched_m<true, 0>(args, items, n_items, capacity, threads, smem, work, max_ctas, st, 0);
}

int launch_ypass_batched(const PassArgs* args, const int2* items, const int* n_items, int capacity, int threads,
                         size_t smem, int mode, cudaStream_t st, int m_reg, int* work, int max_ctas)
{
    if (m_reg) return GP_ERR_ARG;
    return mode == 1
               ? launch_batched_m<false, 1>(args, items, n_items, capacity, threads, smem, work, max_ctas, st, 0)
               : launch_batched_m<false, 0>(args, items, n_items, capacity, threads, smem, work, max_ctas, st, 0);
}

int launch_xpass_batched(const PassArgsF* args, const int2* items, const int* n_items, int capacity, int threads,
                         size_t smem, int mode, cudaStream_t st, int m_reg, int* work, int max_ctas)
{
    return mode == 1
               ? launch_batched_m<true, 1>(args, items, n_items, capacity, threads, smem, work, max_ctas, st, m_reg)
               : launch_batched_m<true, 0>(args, items, n_items, capacity, threads, smem, work, max_ctas, st, m_reg);
}

int launch_ypass_batched(const PassArgsF* args, const int2* items, const int* n_items, int capacity, int threads,
                         size_t smem, int mode, cudaStream_t st, int m_reg, int* work, int max_ctas)
{
    return mode == 1
               ? launch_batched_m<false, 1>(args, items, n_items, capacity, threads, smem, work, max_ctas, st, m_reg)
               : launch_batched_m<false, 0>(args, items, n_items, capacity, threads, smem, work, max_ctas, st, m_reg);
}

}  // namespace gpspin

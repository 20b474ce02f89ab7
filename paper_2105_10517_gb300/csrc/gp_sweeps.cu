// gp_sweeps.cu -- coefficient precompute and the two fused line passes of one
// split-step Crank-Nicolson step (arXiv 2105.10517, program summary "Solution
// method"; Supplementary Material Eqs. S.1-S.5).
//
// FP64 on GB300 is issue-bound: one warp-wide DFMA/DMUL/DADD occupies a
// sub-partition's FP64 unit for ~64 clocks whether 1 or 32 lanes are active,
// and a dependent chain runs at that same rate.  So every FP64 instruction
// here is issued by full warps, transcendentals of small arguments are short
// Taylor polynomials, and the tridiagonal solves are split into chunks that
// many threads run at once (the chunked Thomas solve below).
#include "gp_internal.cuh"
#include <cmath>

namespace gpspin {

// ---------------------------------------------------------------- complex --
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a*b + c
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c)
{
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// c - a*b
__device__ __forceinline__ double2 cfnma(double2 a, double2 b, double2 c)
{
    return make_double2(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 crecip(double2 z)
{
    double d = z.x * z.x + z.y * z.y;
    return make_double2(z.x / d, -z.y / d);
}

// ------------------------------------------------------------------ K1 ----
// One thread per (line, channel).  The line operator is A = -1/2 D2 + kappa D1
// with kappa = i kb; the CN system matrix is I + tau A with tau = dt/2
// (imaginary time) or i dt/2 (real time), i.e. constant sub-diagonal alpha,
// diagonal beta and super-diagonal gamma' along the line.
__global__ void coef_kernel(LineCoef* coef, int nlines, int dir, int mode, double h, double line_len,
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
    LineCoef& C = coef[id];
    double2 cprev = make_double2(0.0, 0.0);
    for (int k = 0; k < kHead; ++k) {
        double2 inv = crecip(csub(beta, cmul(alpha, cprev)));
        double2 cp = cmul(gam, inv);
        C.inv[k] = inv;
        C.g[k] = cmul(alpha, inv);
        C.cp[k] = cp;
        if (k == kHead - 1) {
            double dlt = hypot(cp.x - cprev.x, cp.y - cprev.y);
            if (!(dlt <= 1e-15 * hypot(cp.x, cp.y) + 1e-300)) atomicOr(status, 1);  // a few ulps
        }
        cprev = cp;
    }
    double2 mg = make_double2(-C.g[kHead - 1].x, -C.g[kHead - 1].y);
    double2 mc = make_double2(-C.cp[kHead - 1].x, -C.cp[kHead - 1].y);
    double2 pf = mg, pb = mc;
    for (int t = 0; t < kFix; ++t) {
        C.pf[t] = pf;
        C.pb[t] = pb;
        pf = cmul(pf, mg);
        pb = cmul(pb, mc);
    }
}

// exp(-tau' w^2 q^2 / 2) on the cell-centred axis q (the separable trap factor
// of the pointwise substep).
__global__ void trap_table_kernel(double2* out, int n, double len, double w, double dt, int mode)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double h = len / n;
    double q = -0.5 * len + (i + 0.5) * h;
    double arg = dt * 0.5 * w * w * q * q;
    if (mode == 1) {
        double s, c;
        sincos(arg, &s, &c);
        out[i] = make_double2(c, -s);
    } else {
        out[i] = make_double2(exp(-arg), 0.0);
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
// The scalar factor exp(-tau' c0 rho) is a Taylor series: eight terms for
// dt c0 rho <= 1/64 (imaginary time) and eleven/twelve terms up to 1/8 (<= 3e-18);
// larger arguments take the library exp / sincos.  The trap factor comes from
// the per-axis tables.
struct PConst {
    double dtc0;  // dt c0 s^2
    double dtc2;  // dt c2 s^2
    double dtr;   // dt R / sqrt(2)
    double s;     // pending normalisation
};

// v = M psi for M = dt B.Sigma, with bx = dt B_x/sqrt2, by = dt B_y/sqrt2, bz = dt B_z.
__device__ __forceinline__ void spin_mv(double bx, double by, double bz, double2 a, double2 b, double2 c,
                                        double2& va, double2& vb, double2& vc)
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

template <int MODE>
__device__ __forceinline__ void pointwise(double2& a, double2& b, double2& c, double2 ev, const PConst& k)
{
    double rp = fma(a.x, a.x, a.y * a.y);
    double r0 = fma(b.x, b.x, b.y * b.y);
    double rm = fma(c.x, c.x, c.y * c.y);
    double rho = rp + r0 + rm;
    // F_+ / sqrt2 = conj(a) b + conj(b) c
    double fr = fma(a.x, b.x, fma(a.y, b.y, fma(b.x, c.x, b.y * c.y)));
    double fi = fma(a.x, b.y, fma(-a.y, b.x, fma(b.x, c.y, -b.y * c.x)));
    double bx = fma(k.dtc2, fr, k.dtr);
    double by = k.dtc2 * fi;
    double bz = k.dtc2 * (rp - rm);
    double u = fma(2.0, fma(bx, bx, by * by), bz * bz);
    double s1, s2;
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
    double2 va, vb, vc, wa, wb, wc;
    spin_mv(bx, by, bz, a, b, c, va, vb, vc);
    spin_mv(bx, by, bz, va, vb, vc, wa, wb, wc);
    const double x = k.dtc0 * rho;
    if (MODE == 1) {
        // t = psi - i s1 v - s2 w
        double2 ta = make_double2(fma(s1, va.y, fma(-s2, wa.x, a.x)), fma(-s1, va.x, fma(-s2, wa.y, a.y)));
        double2 tb = make_double2(fma(s1, vb.y, fma(-s2, wb.x, b.x)), fma(-s1, vb.x, fma(-s2, wb.y, b.y)));
        double2 tc = make_double2(fma(s1, vc.y, fma(-s2, wc.x, c.x)), fma(-s1, vc.x, fma(-s2, wc.y, c.y)));
        double cs, sn;
        if (x <= 0.125) {
            double x2 = x * x;
            cs = fma(fma(fma(fma(fma(x2, -1.0 / 3628800.0, 1.0 / 40320.0), x2, -1.0 / 720.0), x2, 1.0 / 24.0), x2,
                         -0.5), x2, 1.0);
            sn = x * fma(fma(fma(fma(fma(x2, -1.0 / 39916800.0, 1.0 / 362880.0), x2, -1.0 / 5040.0), x2, 1.0 / 120.0),
                             x2, -1.0 / 6.0), x2, 1.0);
        } else {
            sincos(x, &sn, &cs);
        }
        // ph = s ev exp(-i x)
        double2 ph = make_double2(k.s * fma(ev.x, cs, ev.y * sn), k.s * fma(ev.y, cs, -ev.x * sn));
        a = cmul(ph, ta);
        b = cmul(ph, tb);
        c = cmul(ph, tc);
    } else {
        double e;
        if (x <= 0.015625) {
            // eight terms for x <= 1/64: the first omitted one is x^8/8! <= 1.7e-19
            const double mx = -x;
            e = fma(fma(fma(fma(fma(fma(fma(mx, 1.0 / 5040.0, 1.0 / 720.0), mx, 1.0 / 120.0), mx, 1.0 / 24.0), mx,
                                1.0 / 6.0), mx, 0.5), mx, 1.0), mx, 1.0);
        } else if (x <= 0.125) {
            const double mx = -x;
            e = fma(fma(fma(fma(fma(fma(fma(fma(fma(fma(mx, 1.0 / 39916800.0, 1.0 / 3628800.0), mx, 1.0 / 362880.0),
                                                    mx, 1.0 / 40320.0), mx, 1.0 / 5040.0), mx, 1.0 / 720.0),
                                        mx, 1.0 / 120.0), mx, 1.0 / 24.0), mx, 1.0 / 6.0), mx, 0.5), mx, 1.0);
            e = fma(e, mx, 1.0);
        } else {
            e = exp(-x);
        }
        double ph = k.s * ev.x * e;
        a = make_double2(ph * fma(-s1, va.x, fma(s2, wa.x, a.x)), ph * fma(-s1, va.y, fma(s2, wa.y, a.y)));
        b = make_double2(ph * fma(-s1, vb.x, fma(s2, wb.x, b.x)), ph * fma(-s1, vb.y, fma(s2, wb.y, b.y)));
        c = make_double2(ph * fma(-s1, vc.x, fma(s2, wc.x, c.x)), ph * fma(-s1, vc.y, fma(s2, wc.y, c.y)));
    }
}

// --------------------------------------------------------- basis rotations --
constexpr double kRs2 = 0.70710678118654752440;  // 1/sqrt(2)

// phi = U_y^dagger psi: Sigma_y eigen-channels lambda = +1, 0, -1 with
// eigenvectors (1, i sqrt2, -1)/2, (1, 0, 1)/sqrt2, (1, -i sqrt2, -1)/2.
__device__ __forceinline__ void to_sigma_y(double2 a, double2 b, double2 c, double2& p, double2& z, double2& m)
{
    double dx = 0.5 * (a.x - c.x), dy = 0.5 * (a.y - c.y);
    p = make_double2(fma(kRs2, b.y, dx), fma(-kRs2, b.x, dy));
    m = make_double2(fma(-kRs2, b.y, dx), fma(kRs2, b.x, dy));
    z = make_double2(kRs2 * (a.x + c.x), kRs2 * (a.y + c.y));
}

// chi = U_x^dagger U_y phi: from Sigma_y channels to Sigma_x channels
// (Sigma_x eigenvectors (1, sqrt2, 1)/2, (1, 0, -1)/sqrt2, (1, -sqrt2, 1)/2):
//   chi_{+-} = phi_0/sqrt2 +- (i/2)(phi_+ - phi_-),  chi_0 = (phi_+ + phi_-)/sqrt2.
__device__ __forceinline__ void sigma_y_to_x(double2 p, double2 z, double2 m, double2& xp, double2& x0, double2& xm)
{
    double hx = 0.5 * (p.x - m.x), hy = 0.5 * (p.y - m.y);
    double zx = kRs2 * z.x, zy = kRs2 * z.y;
    xp = make_double2(zx - hy, zy + hx);
    xm = make_double2(zx + hy, zy - hx);
    x0 = make_double2(kRs2 * (p.x + m.x), kRs2 * (p.y + m.y));
}

// psi = U_x chi.
__device__ __forceinline__ void from_sigma_x(double2 xp, double2 x0, double2 xm, double2& a, double2& b, double2& c)
{
    double sx = 0.5 * (xp.x + xm.x), sy = 0.5 * (xp.y + xm.y);
    a = make_double2(fma(kRs2, x0.x, sx), fma(kRs2, x0.y, sy));
    c = make_double2(fma(-kRs2, x0.x, sx), fma(-kRs2, x0.y, sy));
    b = make_double2(kRs2 * (xp.x - xm.x), kRs2 * (xp.y - xm.y));
}

// ------------------------------------------------------- chunked Thomas ----
// Solves (I + tau A) w = phi for every (line, channel) of the CTA and replaces
// phi by psi' = 2 w - phi = (I + tau A)^{-1} (I - tau A) phi.
// Each line is cut into Q chunks of m points, one thread per chunk:
//  1. forward elimination inside the chunk from a zero carry -> y^, chunk end;
//  2. the true y differs by pf[t] * (true end value of the previous chunk) on
//     the chunk's first F points (|pf[t]| <= 2^-60 beyond), then back
//     substitution inside the chunk from a zero carry -> w^, chunk start;
//  3. the true w differs by pb[m-1-t] * (true start value of the next chunk) on
//     the chunk's last F points.
// Because m > F, a chunk's local end/start value equals the true one to FP64
// rounding, so no carry has to be propagated sequentially across chunks.
// Smem: line-channel arrays of stride Lp, chunk q at offset q (m + 1) (the pad
// keeps chunk-parallel accesses on distinct banks).
__device__ __forceinline__ void chunked_thomas(double2* sa, double2* sb, double2* cf, double2* cb,
                                               const LineCoef* coef, const LineTiling& T, int nl)
{
    const int m = T.m, Q = T.Q, F = T.F, L = T.L, Lp = T.Lp;
    const int nthr = 3 * nl * Q;
    const int tid = threadIdx.x;
    const bool active = tid < nthr;
    const int q = active ? tid % Q : 0;
    const int lc = active ? tid / Q : 0;  // r * 3 + ch
    const int start = q * m;
    const int len = min(m, L - start);
    const LineCoef* C = coef + lc;        // coef already offset to the CTA's first line
    double2* pa = sa + lc * Lp + q * (m + 1);
    double2* pbf = sb + lc * Lp + q * (m + 1);

    if (active) {
        double2 y = make_double2(0.0, 0.0);
        for (int t = 0; t < len; ++t) {
            int kk = min(start + t, kHead - 1);
            y = cfnma(C->g[kk], y, cmul(C->inv[kk], pa[t]));
            pbf[t] = y;
        }
        cf[lc * Q + q] = y;
    }
    __syncthreads();
    if (active) {
        if (q > 0) {
            double2 yc = cf[lc * Q + q - 1];
            int nf = min(F, len);
            for (int t = 0; t < nf; ++t) pbf[t] = cfma(C->pf[t], yc, pbf[t]);
        }
        double2 w = make_double2(0.0, 0.0);
        for (int t = len - 1; t >= 0; --t) {
            int kk = min(start + t, kHead - 1);
            w = cfnma(C->cp[kk], w, pbf[t]);
            pbf[t] = w;
        }
        cb[lc * Q + q] = w;
    }
    __syncthreads();
    if (active) {
        const bool fix = q < Q - 1;
        double2 wc = fix ? cb[lc * Q + q + 1] : make_double2(0.0, 0.0);
        for (int t = 0; t < len; ++t) {
            double2 w = pbf[t];
            int d = len - t;
            if (fix && d <= F) w = cfma(C->pb[d - 1], wc, w);
            double2 ph = pa[t];
            pa[t] = make_double2(fma(2.0, w.x, -ph.x), fma(2.0, w.y, -ph.y));
        }
    }
    __syncthreads();
}

__device__ __forceinline__ int sidx(const LineTiling& T, int lc, int k) { return lc * T.Lp + k + k / T.m; }

// --------------------------------------------------------------- x-pass ----
template <int MODE>
__global__ void __launch_bounds__(512) xpass_kernel(PassArgs A)
{
    extern __shared__ double2 smem[];
    const LineTiling& T = A.t;
    double2* sa = smem;
    double2* sb = sa + 3 * T.R * T.Lp;
    double2* cf = sb + 3 * T.R * T.Lp;
    double2* cb = cf + 3 * T.R * T.Q;
    const int line0 = blockIdx.x * T.R;
    const int nl = min(T.R, T.nlines - line0);
    const int nx = A.nx, ny = A.ny, L = T.L;
    const size_t plane = (size_t)nx * ny;

    const double s = *A.scale;
    PConst k;
    k.dtc0 = A.dt * A.c0 * s * s;
    k.dtc2 = A.dt * A.c2 * s * s;
    k.dtr = A.dt * A.rabi * kRs2;
    k.s = s;
    for (int e = threadIdx.x; e < nl * L; e += blockDim.x) {
        int r = e / L, i = e - r * L, j = line0 + r;
        size_t o = (size_t)j * nx + i;
        double2 a = A.in[o], b = A.in[plane + o], c = A.in[2 * plane + o];
        if (A.do_p) {
            // the trap factor is real in imaginary time
            double2 ev = MODE == 1 ? cmul(A.ex[i], A.ey[j]) : make_double2(A.ex[i].x * A.ey[j].x, 0.0);
            pointwise<MODE>(a, b, c, ev, k);
        } else {
            a = make_double2(s * a.x, s * a.y);
            b = make_double2(s * b.x, s * b.y);
            c = make_double2(s * c.x, s * c.y);
        }
        double2 p, z, m;
        to_sigma_y(a, b, c, p, z, m);
        sa[sidx(T, r * 3 + 0, i)] = p;
        sa[sidx(T, r * 3 + 1, i)] = z;
        sa[sidx(T, r * 3 + 2, i)] = m;
    }
    __syncthreads();
    if (A.do_solve) chunked_thomas(sa, sb, cf, cb, A.coef + (size_t)line0 * 3, T, nl);
    // transposed store t[mu][i][j], consecutive threads -> consecutive j
    for (int e = threadIdx.x; e < nl * L; e += blockDim.x) {
        int i = e / nl, r = e - i * nl, j = line0 + r;
        double2 xp, x0, xm;
        sigma_y_to_x(sa[sidx(T, r * 3 + 0, i)], sa[sidx(T, r * 3 + 1, i)], sa[sidx(T, r * 3 + 2, i)], xp, x0, xm);
        size_t o = (size_t)i * ny + j;
        A.out[o] = xp;
        A.out[plane + o] = x0;
        A.out[2 * plane + o] = xm;
    }
}

// --------------------------------------------------------------- y-pass ----
template <int MODE>
__global__ void __launch_bounds__(512) ypass_kernel(PassArgs A)
{
    extern __shared__ double2 smem[];
    __shared__ double wsum[32];
    const LineTiling& T = A.t;
    double2* sa = smem;
    double2* sb = sa + 3 * T.R * T.Lp;
    double2* cf = sb + 3 * T.R * T.Lp;
    double2* cb = cf + 3 * T.R * T.Q;
    const int line0 = blockIdx.x * T.R;
    const int nl = min(T.R, T.nlines - line0);
    const int nx = A.nx, ny = A.ny, L = T.L;
    const size_t plane = (size_t)nx * ny;

    for (int e = threadIdx.x; e < nl * L; e += blockDim.x) {
        int r = e / L, j = e - r * L, i = line0 + r;
        size_t o = (size_t)i * ny + j;
        sa[sidx(T, r * 3 + 0, j)] = A.in[o];
        sa[sidx(T, r * 3 + 1, j)] = A.in[plane + o];
        sa[sidx(T, r * 3 + 2, j)] = A.in[2 * plane + o];
    }
    __syncthreads();
    if (A.do_solve) chunked_thomas(sa, sb, cf, cb, A.coef + (size_t)line0 * 3, T, nl);
    double acc = 0.0;
    for (int e = threadIdx.x; e < nl * L; e += blockDim.x) {
        int j = e / nl, r = e - j * nl, i = line0 + r;
        double2 a, b, c;
        from_sigma_x(sa[sidx(T, r * 3 + 0, j)], sa[sidx(T, r * 3 + 1, j)], sa[sidx(T, r * 3 + 2, j)], a, b, c);
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
            A.partials[blockIdx.x] = t;
        }
    }
}

// ------------------------------------------------------------- launchers ---
int launch_coef(LineCoef* coef, int nlines, int dir, int mode, double h, double line_len, double line_h,
                double dt, double omeg, double gamma, int eta, int* status, cudaStream_t st)
{
    int n = nlines * 3;
    coef_kernel<<<(n + 127) / 128, 128, 0, st>>>(coef, nlines, dir, mode, h, line_len, line_h, dt, omeg, gamma, eta,
                                                  status);
    return report_cuda(cudaGetLastError(), "coef_kernel launch");
}

int launch_trap_table(double2* out, int n, double len, double w, double dt, int mode, cudaStream_t st)
{
    trap_table_kernel<<<(n + 127) / 128, 128, 0, st>>>(out, n, len, w, dt, mode);
    return report_cuda(cudaGetLastError(), "trap_table_kernel launch");
}

// Opt in to the dynamic shared memory a launch needs (static shared memory of
// the kernel counts against the same per-block limit).
template <typename K>
static int launch_pass(K kernel, const PassArgs& a, cudaStream_t st)
{
    if (a.t.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a.t.smem);
        if (e != cudaSuccess) return report_cuda(e, "cudaFuncSetAttribute(line pass)");
    }
    int grid = (a.t.nlines + a.t.R - 1) / a.t.R;
    kernel<<<grid, a.t.threads, a.t.smem, st>>>(a);
    return report_cuda(cudaGetLastError(), "line pass launch");
}

int launch_xpass(const PassArgs& a, int mode, cudaStream_t st)
{
    return mode == 1 ? launch_pass(xpass_kernel<1>, a, st) : launch_pass(xpass_kernel<0>, a, st);
}

int launch_ypass(const PassArgs& a, int mode, cudaStream_t st)
{
    return mode == 1 ? launch_pass(ypass_kernel<1>, a, st) : launch_pass(ypass_kernel<0>, a, st);
}

}  // namespace gpspin

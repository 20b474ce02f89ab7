/*
 * gp_oracle.c -- plain, slow FP64 CPU oracle for one split-step Crank-Nicolson
 * time step of the 2D rotating spin-1 Gross-Pitaevskii equation with Rashba or
 * Dresselhaus spin-orbit (SO) coupling and Rabi coupling
 * (arXiv 2105.10517, Supplementary Material, Eqs. S.1-S.6).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker the GPU path is compared
 * against.  Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  The product path never calls it, and it shares no code,
 * header, table or constant with the CUDA library.
 *
 * Everything is written from the continuum equations in the most direct form:
 *   - the pointwise substep is the 3x3 matrix exponential of the local
 *     Hamiltonian, evaluated by a scaled Taylor series applied to the spinor
 *     (no closed form, no spin eigenbasis);
 *   - each directional substep is the Crank-Nicolson system of that direction
 *     solved line by line in the ORIGINAL spin basis as a block-tridiagonal
 *     system with 3x3 blocks (textbook block Thomas, re-derived every call);
 *   - observables evaluate the energy functional (S.6) term by term with the
 *     explicit SO terms f_{+1}, f_0, f_{-1} printed below Eq. (S.5).
 *
 * Readings of what the paper leaves open (each is listed in the design notes):
 *   grid      cell-centred, x_i = -xlen/2 + (i+1/2) dx, psi = 0 outside the box;
 *   splitting Lie order P(dt) -> X(dt) -> Y(dt) -> [imag: renormalise to 1];
 *             the second-order (Strang) composition is an extension;
 *   P         psi <- exp(-tau' H_loc) psi with H_loc = V + c0 rho + c2 F.Sigma
 *             + R Sigma_x frozen at the start of the substep (c2 and Rabi terms
 *             of Eqs. S.1-S.2), tau' = dt (imaginary time) or i dt (real time);
 *   X, Y      CN of the directional operators
 *             A_x = -1/2 d_xx + (-i Omega y + i gamma Sigma_y) d_x
 *             A_y = -1/2 d_yy + ( i Omega x - i eta gamma Sigma_x) d_y
 *             (L_z = -i(x d_y - y d_x); SO term gamma(eta p_y Sigma_x - p_x Sigma_y))
 *             with second-order central differences;
 *   norm      rectangle rule, rescale all components by 1/sqrt(N) after every
 *             imaginary-time step; magnetisation is reported, not enforced.
 *
 * psi layout: psi[c][j][i] complex128 (re, im interleaved), c = 0,1,2 for the
 * components m_F = +1, 0, -1; j = y index (ny lines); i = x index (fastest).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* Parameters of the problem statement (grid, trap, nonlinearities, rotation,
 * SO type and strength, Rabi strength).  so_type: 0 none, 1 Rashba (eta=+1),
 * 2 Dresselhaus (eta=-1). */
typedef struct {
    int nx, ny;
    double xlen, ylen;
    double dt;
    double wx, wy;
    double c0, c2, omeg;
    int so_type;
    double gamma, rabi;
} orc_params;

enum { ORC_OK = 0, ORC_EARG = 1, ORC_ENOTDOM = 2, ORC_ESINGULAR = 3, ORC_ENOMEM = 4 };
enum { ORC_IMAG = 0, ORC_REAL = 1 };

/* ---- grid ---------------------------------------------------------------- */
static double grid_dx(const orc_params* p) { return p->xlen / p->nx; }
static double grid_dy(const orc_params* p) { return p->ylen / p->ny; }
static double grid_x(const orc_params* p, int i) { return -0.5 * p->xlen + (i + 0.5) * grid_dx(p); }
static double grid_y(const orc_params* p, int j) { return -0.5 * p->ylen + (j + 0.5) * grid_dy(p); }
static double trap_v(const orc_params* p, double x, double y)
{
    return 0.5 * (p->wx * p->wx * x * x + p->wy * p->wy * y * y);
}
static int so_eta(const orc_params* p) { return p->so_type == 1 ? 1 : (p->so_type == 2 ? -1 : 0); }
static double so_gamma(const orc_params* p) { return p->so_type == 0 ? 0.0 : p->gamma; }

/* ---- threads ---------------------------------------------------------------
 * The substeps work on independent grid lines (rows for P and X, columns for Y),
 * the way the paper's program spreads them over OpenMP threads.  Each line's
 * arithmetic is the same whichever thread runs it, so every thread count gives
 * bitwise identical results; the sums (norms, observables) stay sequential. */
static int g_threads = 1;

/* Sets the number of threads the substeps use (n >= 1; n <= 0 only queries);
 * returns the number in effect (1 when the library was built without OpenMP). */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) g_threads = n;
#else
    (void)n;
    g_threads = 1;
#endif
    return g_threads;
}

static int check_params(const orc_params* p)
{
    if (!p || p->nx < 2 || p->ny < 2) return ORC_EARG;
    if (!(p->xlen > 0) || !(p->ylen > 0) || !(p->dt > 0)) return ORC_EARG;
    if (p->so_type < 0 || p->so_type > 2) return ORC_EARG;
    return ORC_OK;
}

#define PSI(psi, p, c, j, i) (psi)[((size_t)(c) * (p)->ny + (j)) * (p)->nx + (i)]

/* ---- spin-1 matrices, Eq. (S.5); Sigma_z = diag(1, 0, -1) ------------------ */
static void spin_matrices(cplx sx[9], cplx sy[9], cplx sz[9])
{
    const double r = 1.0 / sqrt(2.0);
    for (int k = 0; k < 9; ++k) sx[k] = sy[k] = sz[k] = 0;
    sx[0 * 3 + 1] = r;  sx[1 * 3 + 0] = r;  sx[1 * 3 + 2] = r;  sx[2 * 3 + 1] = r;
    sy[0 * 3 + 1] = -I * r; sy[1 * 3 + 0] = I * r; sy[1 * 3 + 2] = -I * r; sy[2 * 3 + 1] = I * r;
    sz[0] = 1; sz[8] = -1;
}

/* ---- small dense complex 3x3 helpers -------------------------------------- */
static void m3_vec(const cplx a[9], const cplx v[3], cplx out[3])
{
    for (int r = 0; r < 3; ++r) out[r] = a[r * 3] * v[0] + a[r * 3 + 1] * v[1] + a[r * 3 + 2] * v[2];
}
static void m3_mul(const cplx a[9], const cplx b[9], cplx out[9])
{
    cplx t[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) t[r * 3 + c] = a[r * 3] * b[c] + a[r * 3 + 1] * b[3 + c] + a[r * 3 + 2] * b[6 + c];
    memcpy(out, t, sizeof t);
}
/* Gauss-Jordan inverse with partial pivoting. */
static int m3_inv(const cplx a[9], cplx out[9])
{
    cplx m[3][6];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 6; ++c) m[r][c] = c < 3 ? a[r * 3 + c] : (c - 3 == r ? 1.0 : 0.0);
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int r = col + 1; r < 3; ++r)
            if (cabs(m[r][col]) > cabs(m[piv][col])) piv = r;
        if (cabs(m[piv][col]) == 0.0) return ORC_ESINGULAR;
        if (piv != col)
            for (int c = 0; c < 6; ++c) { cplx t = m[col][c]; m[col][c] = m[piv][c]; m[piv][c] = t; }
        cplx d = m[col][col];
        for (int c = 0; c < 6; ++c) m[col][c] /= d;
        for (int r = 0; r < 3; ++r) {
            if (r == col) continue;
            cplx f = m[r][col];
            for (int c = 0; c < 6; ++c) m[r][c] -= f * m[col][c];
        }
    }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) out[r * 3 + c] = m[r][c + 3];
    return ORC_OK;
}
static double m3_norm_inf(const cplx a[9])
{
    double best = 0;
    for (int r = 0; r < 3; ++r) {
        double s = cabs(a[r * 3]) + cabs(a[r * 3 + 1]) + cabs(a[r * 3 + 2]);
        if (s > best) best = s;
    }
    return best;
}

/* ---- local spin density ---------------------------------------------------- */
/* F = psi^dagger Sigma psi at one site (the vector whose contraction with Sigma
 * reproduces the c2 terms of Eqs. S.1-S.2). */
static void spin_density(const cplx v[3], double f[3])
{
    cplx sx[9], sy[9], sz[9], t[3];
    spin_matrices(sx, sy, sz);
    const cplx* s[3] = { sx, sy, sz };
    for (int k = 0; k < 3; ++k) {
        m3_vec(s[k], v, t);
        f[k] = creal(conj(v[0]) * t[0] + conj(v[1]) * t[1] + conj(v[2]) * t[2]);
    }
}

/* ---- substep P: psi <- exp(-tau' H_loc) psi at every site ------------------ */
/* exp(G) v by scaling and squaring of the Taylor series, applied to the vector:
 * choose s with ||G||_inf / 2^s <= 1/2, then apply sum_k (G/2^s)^k / k! 2^s times. */
static void expm_apply(const cplx g[9], cplx v[3])
{
    double nrm = m3_norm_inf(g);
    int s = 0;
    while (nrm / ldexp(1.0, s) > 0.5) ++s;
    cplx gs[9];
    for (int k = 0; k < 9; ++k) gs[k] = g[k] / ldexp(1.0, s);
    for (long rep = 0; rep < (1L << s); ++rep) {
        cplx sum[3] = { v[0], v[1], v[2] }, term[3] = { v[0], v[1], v[2] }, nxt[3];
        for (int k = 1; k <= 60; ++k) {
            m3_vec(gs, term, nxt);
            for (int r = 0; r < 3; ++r) term[r] = nxt[r] / k;
            double tn = cabs(term[0]) + cabs(term[1]) + cabs(term[2]);
            double sn = cabs(sum[0]) + cabs(sum[1]) + cabs(sum[2]);
            for (int r = 0; r < 3; ++r) sum[r] += term[r];
            if (tn <= 1e-20 * sn || tn == 0.0) break;
        }
        v[0] = sum[0]; v[1] = sum[1]; v[2] = sum[2];
    }
}

/* Local Hamiltonian at one site: (V + c0 rho) I + c2 F.Sigma + R Sigma_x.
 * This is the non-derivative part of Eqs. (S.1)-(S.3). */
static void local_hamiltonian(const orc_params* p, double x, double y, const cplx v[3], cplx h[9])
{
    cplx sx[9], sy[9], sz[9];
    spin_matrices(sx, sy, sz);
    double rho = creal(v[0] * conj(v[0])) + creal(v[1] * conj(v[1])) + creal(v[2] * conj(v[2]));
    double f[3];
    spin_density(v, f);
    double diag = trap_v(p, x, y) + p->c0 * rho;
    for (int k = 0; k < 9; ++k) h[k] = p->c2 * (f[0] * sx[k] + f[1] * sy[k] + f[2] * sz[k]) + p->rabi * sx[k];
    h[0] += diag; h[4] += diag; h[8] += diag;
}

int orc_substep_p(const orc_params* p, cplx* psi, int mode)
{
    int st = check_params(p);
    if (st) return st;
    cplx tau = mode == ORC_REAL ? I * p->dt : p->dt;
#ifdef _OPENMP
#pragma omp parallel for num_threads(g_threads) schedule(static)
#endif
    for (int j = 0; j < p->ny; ++j)
        for (int i = 0; i < p->nx; ++i) {
            cplx v[3] = { PSI(psi, p, 0, j, i), PSI(psi, p, 1, j, i), PSI(psi, p, 2, j, i) };
            cplx h[9], g[9];
            local_hamiltonian(p, grid_x(p, i), grid_y(p, j), v, h);
            for (int k = 0; k < 9; ++k) g[k] = -tau * h[k];
            expm_apply(g, v);
            for (int c = 0; c < 3; ++c) PSI(psi, p, c, j, i) = v[c];
        }
    return ORC_OK;
}

/* ---- directional CN substeps (block tridiagonal, original spin basis) ----- */
/* One line of n spinors u[k] (stride between consecutive points = `stride`
 * complex elements inside each component plane, planes `plane` apart).
 * The line operator is A = -1/2 D2 (x) I + D1 (x) K with D1, D2 the central
 * first/second differences of spacing h and K the 3x3 first-derivative
 * coefficient.  Solves (I + tau A) u' = (I - tau A) u with zero Dirichlet data. */
static int cn_line(cplx* base, size_t stride, size_t plane, int n, double h, const cplx kmat[9], cplx tau,
                   cplx* work)
{
    cplx sub[9], dia[9], sup[9];
    for (int k = 0; k < 9; ++k) {
        double id = (k % 4 == 0) ? 1.0 : 0.0;
        sub[k] = -0.5 / (h * h) * id - kmat[k] / (2 * h);
        dia[k] = 1.0 / (h * h) * id;
        sup[k] = -0.5 / (h * h) * id + kmat[k] / (2 * h);
    }
    /* System matrix blocks. */
    cplx ms[9], md[9], mu[9];
    for (int k = 0; k < 9; ++k) {
        double id = (k % 4 == 0) ? 1.0 : 0.0;
        ms[k] = tau * sub[k];
        md[k] = id + tau * dia[k];
        mu[k] = tau * sup[k];
    }
    /* Pivot-free block elimination is safe under strict block diagonal dominance. */
    cplx mdi[9];
    if (m3_inv(md, mdi)) return ORC_ESINGULAR;
    if (!(m3_norm_inf(mdi) * (m3_norm_inf(ms) + m3_norm_inf(mu)) < 1.0)) return ORC_ENOTDOM;

    cplx* u = work;            /* n x 3 : the line, then the solution        */
    cplx* rhs = work + 3 * n;  /* n x 3 : right-hand side, then d'          */
    cplx* cp = work + 6 * n;   /* n x 9 : C' blocks                         */
    for (int k = 0; k < n; ++k)
        for (int c = 0; c < 3; ++c) u[3 * k + c] = base[c * plane + k * stride];
    /* rhs = (I - tau A) u */
    for (int k = 0; k < n; ++k) {
        cplx au[3] = { 0, 0, 0 }, t[3];
        m3_vec(dia, &u[3 * k], t);
        for (int c = 0; c < 3; ++c) au[c] += t[c];
        if (k > 0) { m3_vec(sub, &u[3 * (k - 1)], t); for (int c = 0; c < 3; ++c) au[c] += t[c]; }
        if (k < n - 1) { m3_vec(sup, &u[3 * (k + 1)], t); for (int c = 0; c < 3; ++c) au[c] += t[c]; }
        for (int c = 0; c < 3; ++c) rhs[3 * k + c] = u[3 * k + c] - tau * au[c];
    }
    /* Forward elimination: S_k = Md - Ms C'_{k-1}; C'_k = S_k^-1 Mu;
     * d'_k = S_k^-1 (rhs_k - Ms d'_{k-1}). */
    for (int k = 0; k < n; ++k) {
        cplx s[9], si[9], t9[9], r[3], t3[3];
        memcpy(s, md, sizeof s);
        memcpy(r, &rhs[3 * k], sizeof r);
        if (k > 0) {
            m3_mul(ms, &cp[9 * (k - 1)], t9);
            for (int q = 0; q < 9; ++q) s[q] -= t9[q];
            m3_vec(ms, &rhs[3 * (k - 1)], t3);
            for (int c = 0; c < 3; ++c) r[c] -= t3[c];
        }
        if (m3_inv(s, si)) return ORC_ESINGULAR;
        m3_mul(si, mu, &cp[9 * k]);
        m3_vec(si, r, &rhs[3 * k]);
    }
    /* Back substitution: u_{n-1} = d'_{n-1}; u_k = d'_k - C'_k u_{k+1}. */
    for (int c = 0; c < 3; ++c) u[3 * (n - 1) + c] = rhs[3 * (n - 1) + c];
    for (int k = n - 2; k >= 0; --k) {
        cplx t3[3];
        m3_vec(&cp[9 * k], &u[3 * (k + 1)], t3);
        for (int c = 0; c < 3; ++c) u[3 * k + c] = rhs[3 * k + c] - t3[c];
    }
    for (int k = 0; k < n; ++k)
        for (int c = 0; c < 3; ++c) base[c * plane + k * stride] = u[3 * k + c];
    return ORC_OK;
}

/* X substep: along every row y_j, K_x = -i Omega y_j I + i gamma Sigma_y. */
int orc_substep_x(const orc_params* p, cplx* psi, int mode)
{
    int st = check_params(p);
    if (st) return st;
    cplx sx[9], sy[9], sz[9];
    spin_matrices(sx, sy, sz);
    cplx tau = mode == ORC_REAL ? I * 0.5 * p->dt : 0.5 * p->dt;
    size_t plane = (size_t)p->nx * p->ny;
#ifdef _OPENMP
#pragma omp parallel num_threads(g_threads)
#endif
    {
        int lst = ORC_OK;
        cplx* work = malloc(sizeof(cplx) * 15 * (size_t)p->nx);
        if (!work) lst = ORC_ENOMEM;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int j = 0; j < p->ny; ++j) {
            if (lst) continue;
            double y = grid_y(p, j);
            cplx k[9];
            for (int q = 0; q < 9; ++q) k[q] = (q % 4 == 0 ? -I * p->omeg * y : 0.0) + I * so_gamma(p) * sy[q];
            lst = cn_line(&PSI(psi, p, 0, j, 0), 1, plane, p->nx, grid_dx(p), k, tau, work);
        }
        free(work);
#ifdef _OPENMP
#pragma omp critical
#endif
        if (lst && !st) st = lst;
    }
    return st;
}

/* Y substep: along every column x_i, K_y = i Omega x_i I - i eta gamma Sigma_x. */
int orc_substep_y(const orc_params* p, cplx* psi, int mode)
{
    int st = check_params(p);
    if (st) return st;
    cplx sx[9], sy[9], sz[9];
    spin_matrices(sx, sy, sz);
    cplx tau = mode == ORC_REAL ? I * 0.5 * p->dt : 0.5 * p->dt;
    size_t plane = (size_t)p->nx * p->ny;
#ifdef _OPENMP
#pragma omp parallel num_threads(g_threads)
#endif
    {
        int lst = ORC_OK;
        cplx* work = malloc(sizeof(cplx) * 15 * (size_t)p->ny);
        if (!work) lst = ORC_ENOMEM;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int i = 0; i < p->nx; ++i) {
            if (lst) continue;
            double x = grid_x(p, i);
            cplx k[9];
            for (int q = 0; q < 9; ++q)
                k[q] = (q % 4 == 0 ? I * p->omeg * x : 0.0) - I * so_eta(p) * so_gamma(p) * sx[q];
            lst = cn_line(&PSI(psi, p, 0, 0, i), (size_t)p->nx, plane, p->ny, grid_dy(p), k, tau, work);
        }
        free(work);
#ifdef _OPENMP
#pragma omp critical
#endif
        if (lst && !st) st = lst;
    }
    return st;
}

/* ---- normalisation ∫rho = 1 (rectangle rule) ------------------------------- */
double orc_norm(const orc_params* p, const cplx* psi)
{
    double s = 0;
    size_t n = 3 * (size_t)p->nx * p->ny;
    for (size_t k = 0; k < n; ++k) s += creal(psi[k] * conj(psi[k]));
    return s * grid_dx(p) * grid_dy(p);
}

int orc_normalize(const orc_params* p, cplx* psi)
{
    double nrm = orc_norm(p, psi);
    if (!(nrm > 0) || !isfinite(nrm)) return ORC_EARG;
    double s = 1.0 / sqrt(nrm);
    size_t n = 3 * (size_t)p->nx * p->ny;
    for (size_t k = 0; k < n; ++k) psi[k] *= s;
    return ORC_OK;
}

/* ---- magnetisation-constrained normalisation (gamma = R = 0) ---------------- */
/* Enforces both conditions printed below Eq. (S.5), N = 1 and N_{+1} - N_{-1} = m,
 * with one factor per component, psi_c <- sigma_c psi_c, and the extra condition
 * sigma_{+1} sigma_{-1} = sigma_0^2 of the normalised gradient flow for spin-1
 * condensates (Bao and Lim, SIAM J. Sci. Comput. 30 (2008) 1925).  With
 * a = sigma_0^2 the conditions give sigma_{+-}^2 = (1 +- m - a N0) / (2 N_{+-}) and
 * the quadratic (N0^2 - 4 N+ N-) a^2 - 2 N0 a + (1 - m^2) = 0, whose root in
 * (0, 1/N0] is taken.  An empty +-1 component keeps sigma = 1. */
int orc_normalize_m(const orc_params* p, cplx* psi, double m)
{
    if (!(m > -1.0 && m < 1.0)) return ORC_EARG;
    const double dA = grid_dx(p) * grid_dy(p);
    const size_t plane = (size_t)p->nx * p->ny;
    double nc[3] = { 0, 0, 0 };
    for (int c = 0; c < 3; ++c)
        for (size_t k = 0; k < plane; ++k) nc[c] += creal(psi[c * plane + k] * conj(psi[c * plane + k]));
    for (int c = 0; c < 3; ++c) nc[c] *= dA;
    double qa = nc[1] * nc[1] - 4.0 * nc[0] * nc[2];
    double a;
    if (fabs(qa) < 1e-14 * (nc[1] * nc[1] + 1e-300)) {
        a = (1.0 - m * m) / (2.0 * nc[1]);
    } else {
        double disc = nc[1] * nc[1] - qa * (1.0 - m * m);
        if (disc < 0) return ORC_EARG;
        a = (nc[1] - sqrt(disc)) / qa;
    }
    if (!(a > 0) || !isfinite(a)) return ORC_EARG;
    double sig[3];
    sig[1] = sqrt(a);
    for (int s = 0; s < 2; ++s) {
        int c = s == 0 ? 0 : 2;
        double num = 1.0 + (s == 0 ? m : -m) - a * nc[1];
        sig[c] = nc[c] > 0 ? sqrt(num / (2.0 * nc[c])) : 1.0;
        if (!isfinite(sig[c])) return ORC_EARG;
    }
    for (int c = 0; c < 3; ++c)
        for (size_t k = 0; k < plane; ++k) psi[c * plane + k] *= sig[c];
    return ORC_OK;
}

/* ---- one full step and propagation ----------------------------------------- */
int orc_step(const orc_params* p, cplx* psi, int mode)
{
    int st;
    if ((st = orc_substep_p(p, psi, mode))) return st;
    if ((st = orc_substep_x(p, psi, mode))) return st;
    if ((st = orc_substep_y(p, psi, mode))) return st;
    if (mode == ORC_IMAG) return orc_normalize(p, psi);
    return ORC_OK;
}

/* Imaginary-time step with the magnetisation-constrained normalisation. */
int orc_step_m(const orc_params* p, cplx* psi, double m)
{
    int st;
    if (so_gamma(p) != 0.0 || p->rabi != 0.0) return ORC_EARG;
    if ((st = orc_substep_p(p, psi, ORC_IMAG))) return st;
    if ((st = orc_substep_x(p, psi, ORC_IMAG))) return st;
    if ((st = orc_substep_y(p, psi, ORC_IMAG))) return st;
    return orc_normalize_m(p, psi, m);
}

int orc_propagate(const orc_params* p, cplx* psi, long long nsteps, int mode)
{
    for (long long s = 0; s < nsteps; ++s) {
        int st = orc_step(p, psi, mode);
        if (st) return st;
    }
    return ORC_OK;
}

/* ---- observables: norms, magnetisation, energy (S.6), chemical potential --- */
/* Central difference of component c at (j,i) along x (dir 0) or y (dir 1),
 * zero outside the box. */
/* ---- second-order (Strang) splitting: an extension ----------------------------
 * The paper names the split-step scheme but not its order; the step above is the
 * first-order (Lie) reading.  The symmetric composition
 *   P(dt/2) -> X(dt/2) -> Y(dt) -> X(dt/2) -> P(dt/2) -> [imag: renormalise]
 * is second order.  Each substep is the one above with its own time step. */
int orc_step_strang(const orc_params* p, cplx* psi, int mode)
{
    orc_params half = *p;
    half.dt = 0.5 * p->dt;
    int st;
    if ((st = orc_substep_p(&half, psi, mode))) return st;
    if ((st = orc_substep_x(&half, psi, mode))) return st;
    if ((st = orc_substep_y(p, psi, mode))) return st;
    if ((st = orc_substep_x(&half, psi, mode))) return st;
    if ((st = orc_substep_p(&half, psi, mode))) return st;
    if (mode == ORC_IMAG) return orc_normalize(p, psi);
    return ORC_OK;
}

int orc_propagate_strang(const orc_params* p, cplx* psi, long long nsteps, int mode)
{
    for (long long s = 0; s < nsteps; ++s) {
        int st = orc_step_strang(p, psi, mode);
        if (st) return st;
    }
    return ORC_OK;
}

static cplx dcen(const orc_params* p, const cplx* psi, int c, int j, int i, int dir)
{
    if (dir == 0) {
        cplx a = i + 1 < p->nx ? PSI(psi, p, c, j, i + 1) : 0;
        cplx b = i > 0 ? PSI(psi, p, c, j, i - 1) : 0;
        return (a - b) / (2 * grid_dx(p));
    }
    cplx a = j + 1 < p->ny ? PSI(psi, p, c, j + 1, i) : 0;
    cplx b = j > 0 ? PSI(psi, p, c, j - 1, i) : 0;
    return (a - b) / (2 * grid_dy(p));
}

/* out[0..2] = N_{+1}, N_0, N_{-1}; out[3] = N; out[4] = m; out[5] = E; out[6] = mu.
 * E is Eq. (S.6) with: |grad psi|^2 as forward differences over every link,
 * including the links to the zero exterior; L_z psi = -i (x d_y - y d_x) psi and
 * the explicit SO terms f_{+-1}, f_0 with central differences. */
int orc_observables(const orc_params* p, const cplx* psi, double out[7])
{
    int st = check_params(p);
    if (st) return st;
    const double dx = grid_dx(p), dy = grid_dy(p), dA = dx * dy;
    const double eta = so_eta(p), gt = so_gamma(p) / sqrt(2.0);
    double nc[3] = { 0, 0, 0 };
    double e_kin = 0, e_trap = 0, e_c0 = 0, e_c2 = 0, e_rabi = 0, e_rot = 0, e_so = 0;
    for (int j = 0; j < p->ny; ++j)
        for (int i = 0; i < p->nx; ++i) {
            double x = grid_x(p, i), y = grid_y(p, j);
            cplx ps = PSI(psi, p, 0, j, i), p0 = PSI(psi, p, 1, j, i), pm = PSI(psi, p, 2, j, i);
            double rp = creal(ps * conj(ps)), r0 = creal(p0 * conj(p0)), rm = creal(pm * conj(pm));
            double rho = rp + r0 + rm;
            nc[0] += rp; nc[1] += r0; nc[2] += rm;
            /* kinetic: forward links (i,i+1) and (j,j+1), plus the link from the
             * exterior zero into the first point of each line */
            for (int c = 0; c < 3; ++c) {
                cplx v = PSI(psi, p, c, j, i);
                cplx vx = i + 1 < p->nx ? PSI(psi, p, c, j, i + 1) : 0;
                cplx vy = j + 1 < p->ny ? PSI(psi, p, c, j + 1, i) : 0;
                e_kin += creal((vx - v) * conj(vx - v)) / (dx * dx) + creal((vy - v) * conj(vy - v)) / (dy * dy);
                if (i == 0) e_kin += creal(v * conj(v)) / (dx * dx);
                if (j == 0) e_kin += creal(v * conj(v)) / (dy * dy);
            }
            e_trap += 2 * trap_v(p, x, y) * rho;
            e_c0 += p->c0 * rho * rho;
            /* c2 bracket of (S.6) */
            cplx cross = conj(pm) * p0 * p0 * conj(ps) + pm * conj(p0) * conj(p0) * ps;
            e_c2 += p->c2 * creal(rp * rp + rm * rm + 2 * (rp * r0 + rm * r0 - rp * rm + cross));
            /* Rabi bracket of (S.6) */
            e_rabi += sqrt(2.0) * p->rabi * creal((conj(ps) + conj(pm)) * p0 + conj(p0) * (ps + pm));
            /* rotation: -2 Omega sum_j psi_j^* L_z psi_j */
            for (int c = 0; c < 3; ++c) {
                cplx lz = -I * (x * dcen(p, psi, c, j, i, 1) - y * dcen(p, psi, c, j, i, 0));
                e_rot += -2 * p->omeg * creal(conj(PSI(psi, p, c, j, i)) * lz);
            }
            /* SO: 2 gamma [psi+^* f+ + psi-^* f- + psi0^* f0], explicit component form */
            if (gt != 0) {
                cplx dx0 = dcen(p, psi, 1, j, i, 0), dy0 = dcen(p, psi, 1, j, i, 1);
                cplx dxp = dcen(p, psi, 0, j, i, 0), dyp = dcen(p, psi, 0, j, i, 1);
                cplx dxm = dcen(p, psi, 2, j, i, 0), dym = dcen(p, psi, 2, j, i, 1);
                cplx fp = -I * gt * (eta * dy0 + I * dx0);
                cplx fm = -I * gt * (eta * dy0 - I * dx0);
                cplx f0 = -I * gt * (-I * dxp + I * dxm + eta * dyp + eta * dym);
                e_so += 2 * creal(conj(ps) * fp + conj(pm) * fm + conj(p0) * f0);
            }
        }
    double ntot = (nc[0] + nc[1] + nc[2]) * dA;
    out[0] = nc[0] * dA; out[1] = nc[1] * dA; out[2] = nc[2] * dA;
    out[3] = ntot;
    out[4] = (nc[0] - nc[2]) * dA;
    double e = 0.5 * dA * (e_kin + e_trap + e_c0 + e_c2 + e_rabi + e_rot + e_so);
    out[5] = e;
    /* mu = <H_GP> / N: the c0 and c2 terms enter the GP operator with twice
     * their weight in E. */
    out[6] = ntot > 0 ? (e + 0.5 * dA * (e_c0 + e_c2)) / ntot : NAN;
    return ORC_OK;
}

/* ---- interaction constants of Eq. (S.4) ------------------------------------ */
/* c0 = 2 N sqrt(2 pi kappa)(a0 + 2 a2)/(3 l0), c2 = 2 N sqrt(2 pi kappa)(a2 - a0)/(3 l0);
 * lengths in one common unit; l0_over_sqrt_kappa = l0/sqrt(kappa). */
void orc_interaction_constants(double natoms, double a0, double a2, double l0_over_sqrt_kappa, double out[2])
{
    double pref = 2 * natoms * sqrt(2 * 3.14159265358979323846) / (3 * l0_over_sqrt_kappa);
    out[0] = pref * (a0 + 2 * a2);
    out[1] = pref * (a2 - a0);
}

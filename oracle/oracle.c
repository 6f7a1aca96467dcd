/*
 * oracle.c -- plain FP64 CPU oracle for the staggered even/odd Dirac operator,
 * the multi-shift CG and the fermion force.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file; the product path never
 * does.  It shares no code, header or table with the CUDA library.
 *
 * Everything here is the plain definition written out: loops over sites and
 * directions in natural order, full 3x3 complex matrices (no compression),
 * C99 double complex arithmetic, no blocking or fusion.
 *
 * Conventions (the paper fixes none of them; these are the readings used):
 *   site   i = x + Lx*(y + Ly*(z + Lz*t)), mu = 0..3 = x, y, z, t
 *   parity (x+y+z+t) mod 2; a site of either parity sits at half index i>>1
 *   links  U[mu][i][a][b]  (row a, column b), complex128
 *   fields psi[h][c] on one parity (Vh = V/2 sites), complex128
 *   eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1})           (staggered phases)
 *   u_mu(x)   = eta_mu(x) * (-1 if mu = t, x_t = Lt-1 and antiperiodic)
 *   (D psi)(x) = 1/2 sum_mu [ u_mu(x) U_mu(x) psi(x+mu)
 *                              - u_mu(x-mu) U_mu(x-mu)^dag psi(x-mu) ]
 * The phase is attached to the link, as the paper multiplies pseudofermions
 * by u_mu(x) U_mu(x) (Sec. 4.1).  D is then anti-Hermitian for any links,
 * which gives D_oe^dag = -D_eo (Sec. 2).  D_eo is the block with even rows and
 * odd columns (odd -> even), D_oe the block with odd rows and even columns.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* geometry                                                             */
/* ------------------------------------------------------------------ */

static long volume_of(const int L[4]) { return (long)L[0] * L[1] * L[2] * L[3]; }

static void coords_of(const int L[4], long i, int c[4])
{
    c[0] = (int)(i % L[0]); i /= L[0];
    c[1] = (int)(i % L[1]); i /= L[1];
    c[2] = (int)(i % L[2]); i /= L[2];
    c[3] = (int)i;
}

static long index_of(const int L[4], const int c[4])
{
    return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3]));
}

/* neighbour of site i one step along +mu (dir = +1) or -mu (dir = -1), periodic */
static long neighbour(const int L[4], long i, int mu, int dir)
{
    int c[4];
    coords_of(L, i, c);
    c[mu] = (c[mu] + dir + L[mu]) % L[mu];
    return index_of(L, c);
}

static int parity_of(const int L[4], long i)
{
    int c[4];
    coords_of(L, i, c);
    return (c[0] + c[1] + c[2] + c[3]) & 1;
}

/* u_mu(x): staggered phase times the antiperiodic-time sign of the link (x, mu) */
static double link_phase(const int L[4], int antiperiodic, long i, int mu)
{
    int c[4], s = 0;
    coords_of(L, i, c);
    for (int nu = 0; nu < mu; ++nu) s += c[nu];
    double eta = (s & 1) ? -1.0 : 1.0;
    if (mu == 3 && antiperiodic && c[3] == L[3] - 1) eta = -eta;
    return eta;
}

static const cplx *link_at(const cplx *U, long V, int mu, long i) { return U + ((long)mu * V + i) * 9; }

/* ------------------------------------------------------------------ */
/* the staggered operator                                                */
/* ------------------------------------------------------------------ */

/* out = D in on the full lattice (both parities), fields [V][3]. */
int oracle_dslash_full(const int L[4], int antiperiodic, const cplx *U, const cplx *in, cplx *out)
{
    long V = volume_of(L);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; ++i) {
        cplx acc[3] = {0, 0, 0};
        for (int mu = 0; mu < 4; ++mu) {
            /* forward hop: u_mu(x) U_mu(x) psi(x + mu) */
            long f = neighbour(L, i, mu, +1);
            const cplx *Uf = link_at(U, V, mu, i);
            double pf = link_phase(L, antiperiodic, i, mu);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    acc[a] += pf * Uf[a * 3 + b] * in[f * 3 + b];
            /* backward hop: - u_mu(x - mu) U_mu(x - mu)^dag psi(x - mu) */
            long g = neighbour(L, i, mu, -1);
            const cplx *Ub = link_at(U, V, mu, g);
            double pb = link_phase(L, antiperiodic, g, mu);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    acc[a] -= pb * conj(Ub[b * 3 + a]) * in[g * 3 + b];
        }
        for (int a = 0; a < 3; ++a) out[i * 3 + a] = 0.5 * acc[a];
    }
    return 0;
}

/* One off-diagonal block of D (Sec. 2): out_parity = 0 gives D_eo (odd -> even),
 * out_parity = 1 gives D_oe (even -> odd).  in/out are [Vh][3] half fields.
 * Written as "embed the input on its parity of the full lattice, apply D,
 * restrict to the output parity", which is the block definition itself. */
int oracle_dslash_eo(const int L[4], int antiperiodic, const cplx *U, int out_parity,
                     const cplx *in_half, cplx *out_half)
{
    long V = volume_of(L);
    cplx *full_in = calloc((size_t)V * 3, sizeof(cplx));
    cplx *full_out = malloc((size_t)V * 3 * sizeof(cplx));
    if (!full_in || !full_out) { free(full_in); free(full_out); return -1; }
    for (long i = 0; i < V; ++i)
        if (parity_of(L, i) != out_parity)
            for (int a = 0; a < 3; ++a) full_in[i * 3 + a] = in_half[(i >> 1) * 3 + a];
    oracle_dslash_full(L, antiperiodic, U, full_in, full_out);
    for (long i = 0; i < V; ++i)
        if (parity_of(L, i) == out_parity)
            for (int a = 0; a < 3; ++a) out_half[(i >> 1) * 3 + a] = full_out[i * 3 + a];
    free(full_in);
    free(full_out);
    return 0;
}

/* A_sigma psi = (m^2 + sigma) psi - D_eo D_oe psi on even sites (Eq. shift_eo). */
int oracle_normal_op(const int L[4], int antiperiodic, const cplx *U, double mass, double sigma,
                     const cplx *in_even, cplx *out_even)
{
    long Vh = volume_of(L) / 2;
    cplx *tmp_odd = malloc((size_t)Vh * 3 * sizeof(cplx));
    cplx *dd = malloc((size_t)Vh * 3 * sizeof(cplx));
    if (!tmp_odd || !dd) { free(tmp_odd); free(dd); return -1; }
    oracle_dslash_eo(L, antiperiodic, U, 1, in_even, tmp_odd); /* D_oe psi   */
    oracle_dslash_eo(L, antiperiodic, U, 0, tmp_odd, dd);      /* D_eo D_oe psi */
    for (long k = 0; k < Vh * 3; ++k) out_even[k] = (mass * mass + sigma) * in_even[k] - dd[k];
    free(tmp_odd);
    free(dd);
    return 0;
}

/* ------------------------------------------------------------------ */
/* vector linear algebra (plain serial loops: fixed summation order)     */
/* ------------------------------------------------------------------ */

static cplx vdot(long n, const cplx *a, const cplx *b)
{
    cplx s = 0;
    for (long k = 0; k < n; ++k) s += conj(a[k]) * b[k];
    return s;
}

static double vnorm2(long n, const cplx *a)
{
    double s = 0;
    for (long k = 0; k < n; ++k) s += creal(a[k]) * creal(a[k]) + cimag(a[k]) * cimag(a[k]);
    return s;
}

/* |b - A_sigma x| / |b| */
double oracle_true_residual(const int L[4], int antiperiodic, const cplx *U, double mass, double sigma,
                            const cplx *b, const cplx *x)
{
    long n = volume_of(L) / 2 * 3;
    cplx *ax = malloc((size_t)n * sizeof(cplx));
    if (!ax) return -1.0;
    oracle_normal_op(L, antiperiodic, U, mass, sigma, x, ax);
    double rr = 0;
    for (long k = 0; k < n; ++k) {
        cplx d = b[k] - ax[k];
        rr += creal(d) * creal(d) + cimag(d) * cimag(d);
    }
    free(ax);
    return sqrt(rr / vnorm2(n, b));
}

/* ------------------------------------------------------------------ */
/* plain CG on A_sigma x = b, starting from the x passed in              */
/* ------------------------------------------------------------------ */

/* Stops when the recursively updated residual satisfies |r| <= tol |b|.
 * Returns the iteration count, or -1 on allocation failure. */
int oracle_cg(const int L[4], int antiperiodic, const cplx *U, double mass, double sigma,
              double tol, int max_iter, const cplx *b, cplx *x)
{
    long n = volume_of(L) / 2 * 3;
    cplx *r = malloc((size_t)n * sizeof(cplx));
    cplx *p = malloc((size_t)n * sizeof(cplx));
    cplx *q = malloc((size_t)n * sizeof(cplx));
    if (!r || !p || !q) { free(r); free(p); free(q); return -1; }
    oracle_normal_op(L, antiperiodic, U, mass, sigma, x, q);
    for (long k = 0; k < n; ++k) { r[k] = b[k] - q[k]; p[k] = r[k]; }
    double bnorm = sqrt(vnorm2(n, b));
    double rr = vnorm2(n, r);
    int it = 0;
    while (it < max_iter && sqrt(rr) > tol * bnorm) {
        oracle_normal_op(L, antiperiodic, U, mass, sigma, p, q);
        double alpha = rr / creal(vdot(n, p, q));
        for (long k = 0; k < n; ++k) { x[k] += alpha * p[k]; r[k] -= alpha * q[k]; }
        double rr_new = vnorm2(n, r);
        double beta = rr_new / rr;
        for (long k = 0; k < n; ++k) p[k] = r[k] + beta * p[k];
        rr = rr_new;
        ++it;
    }
    free(r); free(p); free(q);
    return it;
}

/* ------------------------------------------------------------------ */
/* multi-shift CG (Sec. 2, Eq. shift_eo; shifted CG of Jegerlehner)     */
/* ------------------------------------------------------------------ */

/*
 * Solves (m^2 - D_eo D_oe + sigma_i) x_i = b for all i with one Krylov space.
 * Base shift sigma_0 = min_i sigma_i, relative shifts s_i = sigma_i - sigma_0.
 *   x_i = 0, r = p = p_i = b, zeta_i = zeta_i_old = 1, alpha_old = 1, beta_old = 0
 *   repeat:  q = A_{sigma_0} p ;  alpha = <r,r> / Re<p,q>
 *            zeta_i' = zeta_i zeta_i_old alpha_old
 *                      / (alpha beta_old (zeta_i_old - zeta_i) + zeta_i_old alpha_old (1 + s_i alpha))
 *            alpha_i = alpha zeta_i' / zeta_i ;  x_i += alpha_i p_i
 *            r -= alpha q ;  beta = <r,r>_new / <r,r>_old ;  beta_i = beta (zeta_i' / zeta_i)^2
 *            p_i = zeta_i' r + beta_i p_i ;  p = r + beta p ;  rotate histories
 *            shift i stops once zeta_i |r| <= tol |b|
 * After the loop each shift's true residual |b - A_{sigma_i} x_i| / |b| is
 * computed in FP64; any shift above tol is finished with plain CG from x_i.
 *
 * x: [nshift][Vh][3] output.  true_resid[nshift], shift_iters[nshift] outputs.
 * scalar_log (optional, may be NULL): row k = (alpha_k, beta_k, zeta_0^{k+1}, ...,
 * zeta_{n-1}^{k+1}) for the first log_rows iterations.
 * finish == 0 skips the true residuals and the refinement (true_resid = -1).
 * Returns the number of multi-shift iterations, or -1 on allocation failure.
 */
int oracle_mscg(const int L[4], int antiperiodic, const cplx *U, double mass,
                int nshift, const double *sigma, double tol, int max_iter,
                const cplx *b, cplx *x, double *true_resid, int *shift_iters,
                int *refine_iters, double *scalar_log, int log_rows, int finish)
{
    long n = volume_of(L) / 2 * 3;
    double sigma0 = sigma[0];
    for (int i = 1; i < nshift; ++i) if (sigma[i] < sigma0) sigma0 = sigma[i];

    cplx *r = malloc((size_t)n * sizeof(cplx));
    cplx *p = malloc((size_t)n * sizeof(cplx));
    cplx *q = malloc((size_t)n * sizeof(cplx));
    cplx *ps = malloc((size_t)n * nshift * sizeof(cplx));
    double *zeta = malloc(sizeof(double) * nshift), *zeta_old = malloc(sizeof(double) * nshift);
    double *zeta_new = malloc(sizeof(double) * nshift), *s = malloc(sizeof(double) * nshift);
    int *active = malloc(sizeof(int) * nshift);
    if (!r || !p || !q || !ps || !zeta || !zeta_old || !zeta_new || !s || !active) return -1;

    for (int i = 0; i < nshift; ++i) {
        s[i] = sigma[i] - sigma0;
        zeta[i] = zeta_old[i] = 1.0;
        active[i] = 1;
        shift_iters[i] = 0;
    }
    memset(x, 0, (size_t)n * nshift * sizeof(cplx));
    for (long k = 0; k < n; ++k) { r[k] = b[k]; p[k] = b[k]; }
    for (int i = 0; i < nshift; ++i) memcpy(ps + (long)i * n, b, (size_t)n * sizeof(cplx));

    double bnorm = sqrt(vnorm2(n, b));
    double rr = vnorm2(n, r);
    double alpha_old = 1.0, beta_old = 0.0;
    int it = 0, nactive = nshift;

    while (nactive > 0 && it < max_iter) {
        oracle_normal_op(L, antiperiodic, U, mass, sigma0, p, q);
        double alpha = rr / creal(vdot(n, p, q));

        for (int i = 0; i < nshift; ++i) {
            if (!active[i]) continue;
            zeta_new[i] = zeta[i] * zeta_old[i] * alpha_old /
                          (alpha * beta_old * (zeta_old[i] - zeta[i]) +
                           zeta_old[i] * alpha_old * (1.0 + s[i] * alpha));
            double alpha_i = alpha * zeta_new[i] / zeta[i];
            cplx *xi = x + (long)i * n, *pi = ps + (long)i * n;
            for (long k = 0; k < n; ++k) xi[k] += alpha_i * pi[k];
        }

        for (long k = 0; k < n; ++k) r[k] -= alpha * q[k];
        double rr_new = vnorm2(n, r);
        double beta = rr_new / rr;

        for (int i = 0; i < nshift; ++i) {
            if (!active[i]) continue;
            double ratio = zeta_new[i] / zeta[i];
            double beta_i = beta * ratio * ratio;
            cplx *pi = ps + (long)i * n;
            for (long k = 0; k < n; ++k) pi[k] = zeta_new[i] * r[k] + beta_i * pi[k];
        }
        for (long k = 0; k < n; ++k) p[k] = r[k] + beta * p[k];

        if (scalar_log && it < log_rows) {
            double *row = scalar_log + (long)it * (2 + nshift);
            row[0] = alpha;
            row[1] = beta;
            for (int i = 0; i < nshift; ++i) row[2 + i] = active[i] ? zeta_new[i] : 0.0;
        }

        for (int i = 0; i < nshift; ++i) {
            if (!active[i]) continue;
            zeta_old[i] = zeta[i];
            zeta[i] = zeta_new[i];
        }
        alpha_old = alpha;
        beta_old = beta;
        rr = rr_new;
        ++it;

        for (int i = 0; i < nshift; ++i) {
            if (active[i] && zeta[i] * sqrt(rr) <= tol * bnorm) {
                active[i] = 0;
                shift_iters[i] = it;
                --nactive;
            }
        }
    }
    for (int i = 0; i < nshift; ++i) if (active[i]) shift_iters[i] = it;

    /* true residuals; finish any shift above tol with plain CG from x_i (finish == 0 skips both
       and leaves true_resid at -1: timing of the multi-shift iterations alone) */
    if (refine_iters) *refine_iters = 0;
    for (int i = 0; i < nshift && !finish; ++i) true_resid[i] = -1.0;
    for (int i = 0; i < nshift && finish; ++i) {
        cplx *xi = x + (long)i * n;
        true_resid[i] = oracle_true_residual(L, antiperiodic, U, mass, sigma[i], b, xi);
        if (true_resid[i] > tol) {
            int ri = oracle_cg(L, antiperiodic, U, mass, sigma[i], 0.5 * tol, max_iter, b, xi);
            if (refine_iters && ri > 0) *refine_iters += ri;
            true_resid[i] = oracle_true_residual(L, antiperiodic, U, mass, sigma[i], b, xi);
        }
    }

    free(r); free(p); free(q); free(ps);
    free(zeta); free(zeta_old); free(zeta_new); free(s); free(active);
    return it;
}

/* ------------------------------------------------------------------ */
/* fermion force                                                         */
/* ------------------------------------------------------------------ */

/*
 * Pseudofermion action S = sum_i r_i Re(b^dag x_i), x_i = A_{sigma_i}^{-1} b.
 * Its variation under a change dU of one link is dS = Re tr(dU W) with, for
 * the link (z, mu), y_i = D_oe x_i and u = u_mu(z):
 *   z even:  W = + sum_i r_i u  y_i(z+mu) x_i(z)^dag
 *   z odd :  W = - sum_i r_i u  x_i(z+mu) y_i(z)^dag
 * (dS = -sum_i r_i x_i^dag dA_i x_i, dA_i = -(dD_eo D_oe + D_eo dD_oe), and
 * D_eo = -D_oe^dag.)  Along dU = eps X U with X in su(3),
 * dS/deps = tr(X F), F = TA(U W), TA(Z) = (Z - Z^dag)/2 - tr(Z - Z^dag)/6 * 1.
 *
 * x: [nshift][Vh][3] even-site solutions.  out: [4][V][3][3].
 * kind 0 writes F = TA(U W); kind 1 writes W^dag, the gradient of S with
 * respect to the link entries in the (dS/dRe U + i dS/dIm U) convention.
 */
int oracle_force(const int L[4], int antiperiodic, const cplx *U, int nshift, const double *residues,
                 const cplx *x, cplx *out, int kind)
{
    long V = volume_of(L), Vh = V / 2, n = Vh * 3;
    cplx *y = malloc((size_t)n * nshift * sizeof(cplx));
    if (!y) return -1;
    for (int i = 0; i < nshift; ++i)
        oracle_dslash_eo(L, antiperiodic, U, 1, x + (long)i * n, y + (long)i * n);

#pragma omp parallel for schedule(static)
    for (long zz = 0; zz < 4 * V; ++zz) {
        int mu = (int)(zz / V);
        long z = zz % V;
        long zf = neighbour(L, z, mu, +1);
        double u = link_phase(L, antiperiodic, z, mu);
        int even = parity_of(L, z) == 0;
        cplx W[9] = {0};
        for (int i = 0; i < nshift; ++i) {
            const cplx *xi = x + (long)i * n, *yi = y + (long)i * n;
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) {
                    if (even)
                        W[a * 3 + c] += residues[i] * u * yi[(zf >> 1) * 3 + a] * conj(xi[(z >> 1) * 3 + c]);
                    else
                        W[a * 3 + c] -= residues[i] * u * xi[(zf >> 1) * 3 + a] * conj(yi[(z >> 1) * 3 + c]);
                }
        }
        cplx *o = out + zz * 9;
        if (kind == 1) {
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) o[a * 3 + c] = conj(W[c * 3 + a]);
            continue;
        }
        const cplx *Uz = link_at(U, V, mu, z);
        cplx Z[9] = {0};
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c)
                for (int b = 0; b < 3; ++b) Z[a * 3 + c] += Uz[a * 3 + b] * W[b * 3 + c];
        cplx tr = 0;
        for (int a = 0; a < 3; ++a) tr += Z[a * 4] - conj(Z[a * 4]);
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c)
                o[a * 3 + c] = 0.5 * (Z[a * 3 + c] - conj(Z[c * 3 + a])) - (a == c ? tr / 6.0 : 0.0);
    }
    free(y);
    return 0;
}

/* number of OpenMP threads the site loops use */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* sets the number of OpenMP threads of the following calls (n >= 1) */
void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/*
 * lqcd_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for the
 * even/odd staggered Dirac operator and the multi-shift conjugate gradient of
 * Bonati et al., "Design and optimization of a portable LQCD Monte Carlo code
 * using OpenACC" (arXiv:1701.00426).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or helper with the CUDA
 * path: it is written directly from the paper's definitions with
 * full-lattice coordinate loops and C99 `double complex` arithmetic.
 *
 * Definitions followed (paper sections / equations):
 *   - Eq. (lexicographic_eo), Sec. 4.1: half-lattice index
 *       idxh = (x0 + N0 (x1 + N1 (x2 + N2 x3))) / 2  for sites of one parity;
 *     all sides even.
 *   - Eq. (diracblock), Sec. 2.2: M = m I + [[0, D_oe], [D_eo, 0]],
 *     D_oe^dag = -D_eo; D_eo maps odd-site vectors to even sites.
 *   - Eq. (lineqeo), Sec. 2.2: (m^2 I - D_eo D_oe) phi_e = b_e, positive
 *     definite, solved by CG.
 *   - Eq. (shlineq), Sec. 2.2: shifted systems (A + sigma_i) x_i = b solved
 *     together using one matrix-vector product per iteration thanks to the
 *     shift invariance of the Krylov space.
 *
 * Readings where the paper is silent:
 *   - D carries the factor 1/2:  (D psi)(n) = 1/2 sum_mu [ s_mu(n) U_mu(n)
 *     psi(n+mu) - s_mu(n-mu) U_mu(n-mu)^dag psi(n-mu) ].
 *   - Staggered phases eta_0 = 1, eta_mu = (-1)^(x_0+...+x_{mu-1}); time is
 *     x3; the antiperiodic boundary is a factor -1 on U_3(n) with x3 = N3-1.
 *     s_mu(n) = eta_mu(n) * (that boundary factor).
 *   - Multi-shift CG: base system = smallest shift; recurrences for the
 *     shifted coefficients derived from the collinearity of shifted residuals
 *     (written out at oracle_mscg below); a shift stops when
 *     |zeta_i| ||r|| <= tol ||b||; the FP64 true residual is then checked and
 *     a shift whose true residual exceeds tol is finished by plain CG started
 *     from its current solution.
 *
 * Parity of every function here is pinned by tests/test_oracle_*.py against
 * invariants and closed forms (anti-hermiticity, gauge covariance, the free
 * field spectrum, brute-force geometry, dense LAPACK solves).
 *
 * Mutation hooks: compiling with -DORACLE_MUTANT=k plants one deliberate
 * mistake (listed at each #if); the test suite builds those variants on the
 * CPU and checks that the pins catch every one.  The default build has none.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------------ */
/* Geometry: Eq. (lexicographic_eo)                                          */
/* ------------------------------------------------------------------------ */

static long volume(const int N[4]) { return (long)N[0] * N[1] * N[2] * N[3]; }

static long lex_index(const int N[4], const int x[4])
{
    return x[0] + (long)N[0] * (x[1] + (long)N[1] * (x[2] + (long)N[2] * x[3]));
}

long oracle_lex(const int N[4], const int x[4]) { return lex_index(N, x); }

long oracle_idxh(const int N[4], const int x[4]) { return lex_index(N, x) / 2; }

int oracle_parity(const int x[4]) { return (x[0] + x[1] + x[2] + x[3]) & 1; }

/* Staggered sign of the link U_mu(x): eta_mu(x) times the antiperiodic
 * time-boundary factor (reading stated in the header). */
double oracle_link_sign(const int N[4], const int x[4], int mu)
{
    int s = 0;
    for (int nu = 0; nu < mu; ++nu) s += x[nu];
#if ORACLE_MUTANT == 5
    /* planted: eta_2 depends on x1 only (no longer anticommuting) */
    if (mu == 2) s = x[1];
#endif
    double eta = (s & 1) ? -1.0 : 1.0;
#if ORACLE_MUTANT != 4 /* mutant 4 planted: periodic instead of antiperiodic time */
    if (mu == 3 && x[3] == N[3] - 1) eta = -eta;
#endif
    return eta;
}

/* ------------------------------------------------------------------------ */
/* D_eo / D_oe: Eq. (diracblock) with the 1/2 normalisation                  */
/* ------------------------------------------------------------------------ */

/* out (sites of parity out_parity, [Vh][3]) = D restricted to that parity,
 * acting on in (sites of the other parity, [Vh][3]).
 * links: [4][V][3][3], U_mu(x)[row][col] at lexicographic index of x.      */
void oracle_deo(const int N[4], int out_parity, const cplx *links,
                const cplx *in, cplx *out)
{
    const long V = volume(N);
#pragma omp parallel for schedule(static)
    for (int x3 = 0; x3 < N[3]; ++x3)
        for (int x2 = 0; x2 < N[2]; ++x2)
            for (int x1 = 0; x1 < N[1]; ++x1)
                for (int x0 = 0; x0 < N[0]; ++x0) {
                    const int x[4] = {x0, x1, x2, x3};
                    if (oracle_parity(x) != out_parity) continue;
                    cplx acc[3] = {0, 0, 0};
                    for (int mu = 0; mu < 4; ++mu) {
                        int xp[4] = {x0, x1, x2, x3}, xm[4] = {x0, x1, x2, x3};
                        xp[mu] = (x[mu] + 1) % N[mu];
                        xm[mu] = (x[mu] - 1 + N[mu]) % N[mu];
#if ORACLE_MUTANT == 10
                        /* planted: forward and backward neighbours swapped in direction 1 */
                        if (mu == 1) { int t = xp[1]; xp[1] = xm[1]; xm[1] = t; }
#endif
                        const cplx *Uf = links + ((long)mu * V + lex_index(N, x)) * 9;
#if ORACLE_MUTANT == 2
                        /* planted: backward hop uses the link at n, not n - mu */
                        const cplx *Ub = links + ((long)mu * V + lex_index(N, x)) * 9;
#else
                        const cplx *Ub = links + ((long)mu * V + lex_index(N, xm)) * 9;
#endif
                        const double sf = oracle_link_sign(N, x, mu);
                        const double sb = oracle_link_sign(N, xm, mu);
                        const cplx *vf = in + oracle_idxh(N, xp) * 3;
                        const cplx *vb = in + oracle_idxh(N, xm) * 3;
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b) {
#if ORACLE_MUTANT == 7
                                /* planted: forward link transposed */
                                acc[a] += sf * Uf[b * 3 + a] * vf[b];
#else
                                acc[a] += sf * Uf[a * 3 + b] * vf[b];
#endif
#if ORACLE_MUTANT == 1
                                /* planted: dagger dropped on the backward hop */
                                acc[a] -= sb * Ub[a * 3 + b] * vb[b];
#elif ORACLE_MUTANT == 3
                                /* planted: backward hop added instead of subtracted */
                                acc[a] += sb * conj(Ub[b * 3 + a]) * vb[b];
#else
                                acc[a] -= sb * conj(Ub[b * 3 + a]) * vb[b];
#endif
                            }
                    }
                    cplx *o = out + oracle_idxh(N, x) * 3;
#if ORACLE_MUTANT == 6
                    /* planted: the 1/2 normalisation is missing */
                    for (int a = 0; a < 3; ++a) o[a] = acc[a];
#else
                    for (int a = 0; a < 3; ++a) o[a] = 0.5 * acc[a];
#endif
                }
}

/* ------------------------------------------------------------------------ */
/* Vector helpers on half-lattice fields (n = 3 * Vh complex numbers)        */
/* ------------------------------------------------------------------------ */

/* <a, b> = sum conj(a) b, accumulated serially in index order. */
cplx oracle_dot(long n, const cplx *a, const cplx *b)
{
    cplx s = 0;
    for (long i = 0; i < n; ++i) s += conj(a[i]) * b[i];
    return s;
}

double oracle_norm2(long n, const cplx *a)
{
    double s = 0;
    for (long i = 0; i < n; ++i) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return s;
}

/* ------------------------------------------------------------------------ */
/* Normal operator: Eq. (lineqeo) plus a shift                               */
/* ------------------------------------------------------------------------ */

/* out = (m^2 + sigma) in - D_eo D_oe in, in/out on even sites;
 * tmp is an odd-site scratch field of the same size. */
void oracle_apply_A(const int N[4], const cplx *links, double mass, double sigma,
                    const cplx *in, cplx *out, cplx *tmp)
{
    const long n = volume(N) / 2 * 3;
    oracle_deo(N, 1, links, in, tmp);   /* D_oe: even -> odd */
    oracle_deo(N, 0, links, tmp, out);  /* D_eo: odd -> even */
    const double a = mass * mass + sigma;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) out[i] = a * in[i] - out[i];
}

/* ||(A + sigma) x - b|| / ||b|| in FP64. */
double oracle_true_residual(const int N[4], const cplx *links, double mass,
                            double sigma, const cplx *b, const cplx *x)
{
    const long n = volume(N) / 2 * 3;
    cplx *ax = malloc(sizeof(cplx) * n), *tmp = malloc(sizeof(cplx) * n);
#if ORACLE_MUTANT == 21
    /* planted: the shift is left out of the residual's operator */
    oracle_apply_A(N, links, mass, 0.0, x, ax, tmp);
#else
    oracle_apply_A(N, links, mass, sigma, x, ax, tmp);
#endif
    double rr = 0;
    for (long i = 0; i < n; ++i) {
        cplx d = ax[i] - b[i];
        rr += creal(d) * creal(d) + cimag(d) * cimag(d);
    }
    double bb = oracle_norm2(n, b);
    free(ax);
    free(tmp);
#if ORACLE_MUTANT == 20
    /* planted: divided by ||b||^2 instead of ||b|| */
    return bb > 0 ? sqrt(rr) / bb : sqrt(rr);
#else
    return bb > 0 ? sqrt(rr / bb) : sqrt(rr);
#endif
}

/* ------------------------------------------------------------------------ */
/* Single-shift CG on (A + sigma) x = b, started from the given x            */
/* ------------------------------------------------------------------------ */

/* Plain conjugate gradient (the SPD solver named after Eq. (lineqeo)).
 * Stops when ||r|| <= tol ||b|| with r the recursively updated residual.
 * Returns the number of iterations, or -1 if max_iter was reached. */
int oracle_cg(const int N[4], const cplx *links, double mass, double sigma,
              const cplx *b, cplx *x, double tol, int max_iter)
{
    const long n = volume(N) / 2 * 3;
    cplx *r = malloc(sizeof(cplx) * n), *p = malloc(sizeof(cplx) * n);
    cplx *q = malloc(sizeof(cplx) * n), *tmp = malloc(sizeof(cplx) * n);
    oracle_apply_A(N, links, mass, sigma, x, q, tmp);
    for (long i = 0; i < n; ++i) { r[i] = b[i] - q[i]; p[i] = r[i]; }
    const double bnorm = sqrt(oracle_norm2(n, b));
    double rho = oracle_norm2(n, r);
    int k = 0;
    while (sqrt(rho) > tol * bnorm) {
        if (k >= max_iter) { k = -1; break; }
        oracle_apply_A(N, links, mass, sigma, p, q, tmp);
        const double alpha = rho / creal(oracle_dot(n, p, q));
        for (long i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        const double rho_new = oracle_norm2(n, r);
        const double beta = rho_new / rho;
        for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        rho = rho_new;
        ++k;
    }
    free(r); free(p); free(q); free(tmp);
    return k;
}

/* ------------------------------------------------------------------------ */
/* Multi-shift CG: Eq. (shlineq) on top of Eq. (lineqeo)                     */
/* ------------------------------------------------------------------------ */

/*
 * Solves (A + sigma_i) x_i = b for i = 0..n_shift-1, with A = m^2 - D_eo D_oe.
 *
 * Base system: A0 = A + sigma_b with sigma_b = min_i sigma_i; relative shifts
 * s_i = sigma_i - sigma_b >= 0.  Plain CG on A0 generates residuals r_k and
 * search directions p_k with step alpha_k and beta_k.  Because the Krylov
 * spaces of A0 and A0 + s_i coincide and both start from r_0 = b, the
 * residual of shift i after k steps is collinear with r_k:
 * r_k^i = zeta_k^i r_k.  Writing the CG three-term recurrence for both
 * systems and matching coefficients gives (zeta_{-1} = zeta_0 = 1,
 * alpha_{-1} = 1, beta_{-1} = 0)
 *
 *   zeta_{k+1} = zeta_k zeta_{k-1} alpha_{k-1} /
 *                [ alpha_k beta_{k-1} (zeta_{k-1} - zeta_k)
 *                  + zeta_{k-1} alpha_{k-1} (1 + s alpha_k) ]
 *   alpha_k^i = alpha_k zeta_{k+1} / zeta_k
 *   beta_k^i  = beta_k (zeta_{k+1} / zeta_k)^2
 *   x^i_{k+1} = x^i_k + alpha_k^i p^i_k
 *   p^i_{k+1} = zeta_{k+1} r_{k+1} + beta_k^i p^i_k
 *
 * For s = 0 these reduce to plain CG (zeta = 1).  Shift i stops updating
 * once |zeta^i| ||r|| <= tol ||b||; the loop ends when every shift stopped.
 * Afterwards the FP64 true residual of every shift is computed and a shift
 * above tol is finished by oracle_cg from its current x_i.
 *
 * x: [n_shift][Vh][3].  iters_out[0] = base iterations, iters_out[1] =
 * total refinement iterations; shift_iters[i] = iteration at which shift i
 * stopped; true_resid[i] = final true residual.  Returns 0, -1 when
 * max_iter was hit before all shifts stopped, -2 for n_shift outside 1..64.
 */
int oracle_mscg(const int N[4], const cplx *links, double mass,
                const double *shifts, int n_shift, const cplx *b, cplx *x,
                double tol, int max_iter, int *iters_out, int *shift_iters,
                double *true_resid)
{
    const long n = volume(N) / 2 * 3;
    if (n_shift < 1 || n_shift > 64) return -2;
    int ib = 0;
    for (int i = 1; i < n_shift; ++i)
        if (shifts[i] < shifts[ib]) ib = i;
    const double sigma_b = shifts[ib];

    cplx *r = malloc(sizeof(cplx) * n), *p = malloc(sizeof(cplx) * n);
    cplx *q = malloc(sizeof(cplx) * n), *tmp = malloc(sizeof(cplx) * n);
    cplx *ps = malloc(sizeof(cplx) * n * n_shift);
    double *zeta = malloc(sizeof(double) * n_shift);
    double *zeta_prev = malloc(sizeof(double) * n_shift);
    int *active = malloc(sizeof(int) * n_shift);

    for (long i = 0; i < n; ++i) { r[i] = b[i]; p[i] = b[i]; }
    for (int s = 0; s < n_shift; ++s) {
        for (long i = 0; i < n; ++i) { ps[s * n + i] = b[i]; x[s * n + i] = 0; }
        zeta[s] = zeta_prev[s] = 1.0;
        active[s] = 1;
        shift_iters[s] = 0;
    }
    const double bnorm = sqrt(oracle_norm2(n, b));
    double rho = oracle_norm2(n, r);
    double alpha_prev = 1.0, beta_prev = 0.0;
    int k = 0, status = 0;
    for (int s = 0; s < n_shift; ++s)
        if (fabs(zeta[s]) * sqrt(rho) <= tol * bnorm) active[s] = 0;

    for (;;) {
        int n_active = 0;
        for (int s = 0; s < n_shift; ++s) n_active += active[s];
        if (n_active == 0) break;
        if (k >= max_iter) { status = -1; break; }

        /* q = A0 p, alpha = rho / <p, q> */
        oracle_apply_A(N, links, mass, sigma_b, p, q, tmp);
        const double alpha = rho / creal(oracle_dot(n, p, q));

        /* shifted step lengths and solution updates (old p_i) */
        double zeta_new[64], alpha_s[64];
        for (int s = 0; s < n_shift; ++s) {
            if (!active[s]) continue;
            const double sh = shifts[s] - sigma_b;
#if ORACLE_MUTANT == 8
            /* planted: the beta term of the zeta recurrence is dropped */
            const double den = zeta_prev[s] * alpha_prev * (1.0 + sh * alpha);
#else
            const double den = alpha * beta_prev * (zeta_prev[s] - zeta[s])
                             + zeta_prev[s] * alpha_prev * (1.0 + sh * alpha);
#endif
            zeta_new[s] = zeta[s] * zeta_prev[s] * alpha_prev / den;
#if ORACLE_MUTANT == 9
            /* planted: ratio of zetas inverted in the shifted step */
            alpha_s[s] = alpha * zeta[s] / zeta_new[s];
#else
            alpha_s[s] = alpha * zeta_new[s] / zeta[s];
#endif
            for (long i = 0; i < n; ++i) x[s * n + i] += alpha_s[s] * ps[s * n + i];
        }

        /* base residual and new direction */
        for (long i = 0; i < n; ++i) r[i] -= alpha * q[i];
        const double rho_new = oracle_norm2(n, r);
        const double beta = rho_new / rho;
        for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];

        /* shifted directions */
        for (int s = 0; s < n_shift; ++s) {
            if (!active[s]) continue;
            const double ratio = zeta_new[s] / zeta[s];
            const double beta_s = beta * ratio * ratio;
            for (long i = 0; i < n; ++i)
                ps[s * n + i] = zeta_new[s] * r[i] + beta_s * ps[s * n + i];
            zeta_prev[s] = zeta[s];
            zeta[s] = zeta_new[s];
        }
        alpha_prev = alpha;
        beta_prev = beta;
        rho = rho_new;
        ++k;
        for (int s = 0; s < n_shift; ++s)
            if (active[s] && fabs(zeta[s]) * sqrt(rho) <= tol * bnorm) {
                active[s] = 0;
                shift_iters[s] = k;
            }
    }
    iters_out[0] = k;
    iters_out[1] = 0;

    /* true residual per shift; finish any shift above tol with plain CG
     * (only after the shifted iteration converged: a run stopped by
     * max_iter reports its residuals as they are) */
    for (int s = 0; s < n_shift; ++s) {
        true_resid[s] = oracle_true_residual(N, links, mass, shifts[s], b, x + s * n);
        if (status == 0 && true_resid[s] > tol) {
            int it = oracle_cg(N, links, mass, shifts[s], b, x + s * n, tol, max_iter);
            if (it < 0) status = -1; else iters_out[1] += it;
            true_resid[s] = oracle_true_residual(N, links, mass, shifts[s], b, x + s * n);
        }
    }
    free(r); free(p); free(q); free(tmp); free(ps);
    free(zeta); free(zeta_prev); free(active);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Rational function of A applied to a source (Sec. 2.2, RHMC)              */
/* ------------------------------------------------------------------------ */

/* The RHMC replaces the root of the fermion matrix in Eq. (rooting) by a
 * rational function with real poles sigma_i (Sec. 2.2, Eq. shlineq):
 *
 *   r(A) b = a0 b + sum_i a_i (A + sigma_i)^{-1} b ,   A = m^2 - D_eo D_oe,
 *
 * and the pseudofermion action is phi^dag r(A) phi (Eq. rooting); the
 * heatbath, the initial and the final action (Algorithm 1, steps 3, 4, 6) are
 * each one such application.  Written out: the shifted solutions x_i come
 * from oracle_mscg with tolerance tol, then y = a0 b + sum_i a_i x_i site by
 * site, and *action = Re <b, y>.  Returns the status of oracle_mscg. */
int oracle_rational_apply(const int N[4], const cplx *links, double mass, double a0,
                          const double *a, const double *shifts, int n_shift,
                          const cplx *b, cplx *y, double tol, int max_iter,
                          double *action)
{
    const long n = volume(N) / 2 * 3;
    if (n_shift < 1 || n_shift > 64) return -2;
    cplx *x = malloc(sizeof(cplx) * n * n_shift);
    int iters[2], shift_iters[64];
    double resid[64];
    const int status = oracle_mscg(N, links, mass, shifts, n_shift, b, x, tol, max_iter,
                                   iters, shift_iters, resid);
    for (long i = 0; i < n; ++i) {
        cplx v = a0 * b[i];
#if ORACLE_MUTANT == 11
        /* planted: each coefficient applied to the next pole's solution */
        for (int s = 0; s < n_shift; ++s) v += a[(s + 1) % n_shift] * x[s * n + i];
#else
        for (int s = 0; s < n_shift; ++s) v += a[s] * x[s * n + i];
#endif
        y[i] = v;
    }
#if ORACLE_MUTANT == 12
    /* planted: the action takes the imaginary part */
    *action = cimag(oracle_dot(n, b, y));
#else
    *action = creal(oracle_dot(n, b, y));
#endif
    free(x);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Fermion force of the rational pseudofermion action (Sec. 2.2)            */
/* ------------------------------------------------------------------------ */

/* S_f = phi^dag r(A) phi with r(A) = a0 + sum_i a_i (A + sigma_i)^{-1}
 * (Eq. rooting with the rational approximation of Eq. shlineq).  Written
 * out from the derivative: with x_i = (A + sigma_i)^{-1} phi (even sites),
 * y_i = D_oe x_i (odd sites) and D_oe^dag = -D_eo (Eq. diracblock),
 *   dS_f = sum_i a_i [ x_i^dag (dD) y_i - y_i^dag (dD) x_i ],
 * and a link U_mu(n) enters D through (1/2) s_mu(n) U_mu(n) psi(n+mu) at n
 * and -(1/2) s_mu(n) U_mu(n)^dag psi(n) at n+mu.  Along
 * U_mu(n) -> exp(i e X) U_mu(n) this gives d/de S_f = Tr(X F_mu(n)) with
 *   F_mu(n) = traceless part of (i s_mu(n) / 2) c sum_i a_i (W_i - W_i^dag),
 *   n even:  W_i = U_mu(n) y_i(n+mu) x_i(n)^dag,   c = +1,
 *   n odd:   W_i = U_mu(n) x_i(n+mu) y_i(n)^dag,   c = -1.
 * F: [4][V][3][3]; *action = Re <phi, r(A) phi>.  Returns the status of the
 * multi-shift solve (tolerance tol on every pole). */
static void m_mul(const cplx *a, const cplx *b, cplx *c);

int oracle_fermion_force(const int N[4], const cplx *links, double mass, double a0, const double *a,
                         const double *shifts, int n_shift, const cplx *phi, double tol, int max_iter,
                         cplx *F, double *action)
{
    const long V = volume(N), Vh = V / 2, n3 = Vh * 3;
    if (n_shift < 1 || n_shift > 64) return -2;
    cplx *x = malloc(sizeof(cplx) * n3 * n_shift), *y = malloc(sizeof(cplx) * n3 * n_shift);
    int iters[2], shift_iters[64];
    double resid[64];
    const int status = oracle_mscg(N, links, mass, shifts, n_shift, phi, x, tol, max_iter, iters, shift_iters,
                                   resid);
    for (int i = 0; i < n_shift; ++i) oracle_deo(N, 1, links, x + i * n3, y + i * n3);
    double act = 0.0;
    for (long k = 0; k < n3; ++k) {
        cplx v = a0 * phi[k];
        for (int i = 0; i < n_shift; ++i) v += a[i] * x[i * n3 + k];
        act += creal(conj(phi[k]) * v);
    }
    *action = act;
#pragma omp parallel for schedule(static)
    for (long lex = 0; lex < V; ++lex) {
        int xn[4];
        long r = lex;
        for (int m = 0; m < 4; ++m) { xn[m] = (int)(r % N[m]); r /= N[m]; }
        const int par = oracle_parity(xn);
        for (int mu = 0; mu < 4; ++mu) {
            int xp[4] = {xn[0], xn[1], xn[2], xn[3]};
            xp[mu] = (xp[mu] + 1) % N[mu];
            const long hn = oracle_idxh(N, xn), hp = oracle_idxh(N, xp);
            /* O = sum_i a_i (left)(right)^dag: left at n + mu, right at n */
            cplx O[9];
            for (int q = 0; q < 9; ++q) O[q] = 0;
            for (int i = 0; i < n_shift; ++i) {
                const cplx *left = (par == 0 ? y : x) + i * n3 + hp * 3;
                const cplx *right = (par == 0 ? x : y) + i * n3 + hn * 3;
                for (int p = 0; p < 3; ++p)
                    for (int q = 0; q < 3; ++q) O[p * 3 + q] += a[i] * left[p] * conj(right[q]);
            }
            cplx W[9];
            m_mul(links + ((long)mu * V + lex) * 9, O, W);
#if ORACLE_MUTANT == 17
            /* planted: the staggered sign of the link is dropped from the force */
            const double s = 1.0;
#else
            const double s = oracle_link_sign(N, xn, mu);
#endif
#if ORACLE_MUTANT == 16
            /* planted: the odd-site terms keep the even-site sign */
            const double c = 1.0;
#else
            const double c = (par == 0) ? 1.0 : -1.0;
#endif
            cplx *f = F + ((long)mu * V + lex) * 9;
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q)
                    f[p * 3 + q] = I * 0.5 * s * c * (W[p * 3 + q] - conj(W[q * 3 + p]));
            const cplx tr = (f[0] + f[4] + f[8]) / 3.0;
            f[0] -= tr; f[4] -= tr; f[8] -= tr;
        }
    }
    free(x);
    free(y);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Gauge part of the molecular dynamics step (Sec. 2.1, Sec. 4.2)           */
/* ------------------------------------------------------------------------ */

/* The gauge action is the tree-level Symanzik improved action (Sec. 2.1).
 * Reading (the paper cites it and prints no formula):
 *
 *   S_g = -(beta/3) sum_x [ c0 sum_{mu<nu} Re Tr P_{mu nu}(x)
 *                         + c1 sum_{mu!=nu} Re Tr R_{mu nu}(x) ],
 *   c0 = 5/3, c1 = -1/12  (c0 + 8 c1 = 1),
 *
 * P_{mu nu}(x) the 1x1 plaquette and R_{mu nu}(x) the rectangle with two
 * links along mu and one along nu, both starting at x, every loop counted
 * once.  The momenta H_mu(x) are Hermitian and traceless (Sec. 2.2); the
 * links move as U -> exp(i eps H) U, the kinetic term is (1/2) sum Tr H^2,
 * so energy conservation fixes the force: F_mu(x) is the Hermitian traceless
 * matrix with d/de S(exp(i e X) U)|_{e=0} = sum Tr(X_mu(x) F_mu(x)) for every
 * Hermitian traceless X, and the momenta move as H -> H - eps F.  The gauge
 * cycle of Algorithm 2 is built from these two updates; its most expensive
 * part is the sum of the C-shaped 3- and 5-link paths around each link
 * (Listing lst:rect_staples). */

static const double SYM_C0 = 5.0 / 3.0;
static const double SYM_C1 = -1.0 / 12.0;

static void m_mul(const cplx *a, const cplx *b, cplx *c)
{
    cplx t[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx s = 0;
            for (int k = 0; k < 3; ++k) s += a[i * 3 + k] * b[k * 3 + j];
            t[i * 3 + j] = s;
        }
    memcpy(c, t, sizeof t);
}

static void m_dag(const cplx *a, cplx *c)
{
    cplx t[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) t[i * 3 + j] = conj(a[j * 3 + i]);
    memcpy(c, t, sizeof t);
}

static void m_unit(cplx *a)
{
    for (int i = 0; i < 9; ++i) a[i] = (i % 4 == 0) ? 1.0 : 0.0;
}

/* coordinates x + d (periodic) */
static void shifted(const int N[4], const int x[4], const int d[4], int y[4])
{
    for (int m = 0; m < 4; ++m) y[m] = ((x[m] + d[m]) % N[m] + N[m]) % N[m];
}

/* the link leaving site x + d in direction mu: U_mu(x + d) */
static const cplx *link(const int N[4], const cplx *links, const int x[4], const int d[4], int mu)
{
    int y[4];
    shifted(N, x, d, y);
    return links + ((long)mu * volume(N) + lex_index(N, y)) * 9;
}

/* product of a path: start at x, take steps (dir, sign), multiply the link
 * of each step: U_dir(y) for a step forward, U_dir(y - dir)^dag backward. */
static void path_product(const int N[4], const cplx *links, const int x[4], int nsteps, const int *dir,
                         const int *sgn, cplx *out)
{
    int d[4] = {0, 0, 0, 0};
    cplx acc[9], t[9];
    m_unit(acc);
    for (int k = 0; k < nsteps; ++k) {
        if (sgn[k] > 0) {
            memcpy(t, link(N, links, x, d, dir[k]), sizeof t);
            d[dir[k]] += 1;
        } else {
            d[dir[k]] -= 1;
            m_dag(link(N, links, x, d, dir[k]), t);
        }
        m_mul(acc, t, acc);
    }
    memcpy(out, acc, sizeof acc);
}

static double re_trace(const cplx *a) { return creal(a[0] + a[4] + a[8]); }

/* S_g by enumeration of every plaquette and rectangle (closed paths). */
double oracle_gauge_action(const int N[4], const cplx *links, double beta)
{
    const long V = volume(N);
    double sp = 0.0, sr = 0.0;
    for (long n = 0; n < V; ++n) {
        int x[4];
        long r = n;
        for (int m = 0; m < 4; ++m) { x[m] = (int)(r % N[m]); r /= N[m]; }
        cplx W[9];
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = 0; nu < 4; ++nu) {
                if (nu == mu) continue;
                if (mu < nu) {
                    const int dir[4] = {mu, nu, mu, nu}, sg[4] = {1, 1, -1, -1};
                    path_product(N, links, x, 4, dir, sg, W);
                    sp += re_trace(W);
                }
                const int dir[6] = {mu, mu, nu, mu, mu, nu}, sg[6] = {1, 1, 1, -1, -1, -1};
                path_product(N, links, x, 6, dir, sg, W);
                sr += re_trace(W);
            }
    }
    return -(beta / 3.0) * (SYM_C0 * sp + SYM_C1 * sr);
}

/* Sum of the staples of U_mu(x): A with S_g = -(beta/3) Re Tr(U_mu(x) A) +
 * (terms without U_mu(x)), written as the open paths from x + mu back to x
 * that close each loop through U_mu(x), for nu != mu and both signs of nu:
 *   plaquette:      nu, -mu, -nu
 *   rectangle (a):  mu, nu, -mu, -mu, -nu        (U_mu(x) first of two)
 *   rectangle (b):  nu, -mu, -mu, -nu, mu        (U_mu(x) second of two)
 *   rectangle (c):  nu, nu, -mu, -nu, -nu        (two steps along nu)
 * (with nu replaced by -nu for the other sign). */
static void staple_sum(const int N[4], const cplx *links, const int x[4], int mu, cplx *A)
{
    int xp[4];
    const int dmu[4] = {mu == 0, mu == 1, mu == 2, mu == 3};
    shifted(N, x, dmu, xp);
    for (int i = 0; i < 9; ++i) A[i] = 0;
    cplx P[9];
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        for (int s = -1; s <= 1; s += 2) {
            {
                const int dir[3] = {nu, mu, nu}, sg[3] = {s, -1, -s};
                path_product(N, links, xp, 3, dir, sg, P);
                for (int i = 0; i < 9; ++i) A[i] += SYM_C0 * P[i];
            }
            {
                const int dir[5] = {mu, nu, mu, mu, nu}, sg[5] = {1, s, -1, -1, -s};
                path_product(N, links, xp, 5, dir, sg, P);
                for (int i = 0; i < 9; ++i) A[i] += SYM_C1 * P[i];
            }
#if ORACLE_MUTANT != 13 /* mutant 13 planted: rectangle staple (b) left out */
            {
                const int dir[5] = {nu, mu, mu, nu, mu}, sg[5] = {s, -1, -1, -s, 1};
                path_product(N, links, xp, 5, dir, sg, P);
                for (int i = 0; i < 9; ++i) A[i] += SYM_C1 * P[i];
            }
#endif
            {
                const int dir[5] = {nu, nu, mu, nu, nu}, sg[5] = {s, s, -1, -s, -s};
                path_product(N, links, xp, 5, dir, sg, P);
                for (int i = 0; i < 9; ++i) A[i] += SYM_C1 * P[i];
            }
        }
    }
}

/* F_mu(x) = traceless part of -(i beta / 6) (M - M^dag), M = U_mu(x) A_mu(x):
 * from d/de Re Tr(exp(i e X) M) = (i/2) Tr(X (M - M^dag)).  F: [4][V][3][3]. */
void oracle_gauge_force(const int N[4], const cplx *links, double beta, cplx *F)
{
    const long V = volume(N);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < V; ++n) {
        int x[4];
        long r = n;
        for (int m = 0; m < 4; ++m) { x[m] = (int)(r % N[m]); r /= N[m]; }
        for (int mu = 0; mu < 4; ++mu) {
            cplx A[9], M[9];
            staple_sum(N, links, x, mu, A);
            m_mul(links + ((long)mu * V + n) * 9, A, M);
            cplx *f = F + ((long)mu * V + n) * 9;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    f[i * 3 + j] = -I * (beta / 6.0) * (M[i * 3 + j] - conj(M[j * 3 + i]));
#if ORACLE_MUTANT != 15 /* mutant 15 planted: the trace of the force is kept */
            const cplx tr = (f[0] + f[4] + f[8]) / 3.0;
            f[0] -= tr; f[4] -= tr; f[8] -= tr;
#endif
        }
    }
}

/* E = exp(i t H) from the power series of the exponential: scale Z = i t H
 * by 2^-k until its 1-norm is below 1/4, sum the series until the terms
 * vanish against the partial sum, square k times. */
void oracle_exp_iH(const cplx *H, double t, cplx *E)
{
    cplx Z[9], term[9], sum[9];
    double nrm = 0.0;
    for (int j = 0; j < 3; ++j) {
        double c = 0.0;
        for (int i = 0; i < 3; ++i) c += cabs(H[i * 3 + j]);
        if (c > nrm) nrm = c;
    }
    nrm *= fabs(t);
    int k = 0;
    while (nrm > 0.25 && k < 60) { nrm *= 0.5; ++k; }
    const double scale = ldexp(t, -k);
    for (int i = 0; i < 9; ++i) Z[i] = I * scale * H[i];
    m_unit(sum);
    m_unit(term);
    for (int n = 1; n < 40; ++n) {
        m_mul(term, Z, term);
        for (int i = 0; i < 9; ++i) term[i] /= n;
        double tn = 0.0;
        for (int i = 0; i < 9; ++i) { sum[i] += term[i]; tn += cabs(term[i]); }
        if (tn < 1e-18) break;
    }
    for (int q = 0; q < k; ++q) m_mul(sum, sum, sum);
    memcpy(E, sum, sizeof sum);
}

/* H_mu(x) -= eps F_mu(x) for every link (momenta [4][V][3][3]). */
void oracle_mom_update(const int N[4], const cplx *links, cplx *mom, double beta, double eps)
{
    const long n9 = 4 * volume(N) * 9;
    cplx *F = malloc(sizeof(cplx) * n9);
    oracle_gauge_force(N, links, beta, F);
    for (long i = 0; i < n9; ++i) mom[i] -= eps * F[i];
    free(F);
}

/* U_mu(x) <- exp(i eps H_mu(x)) U_mu(x) for every link. */
void oracle_link_update(const int N[4], cplx *links, const cplx *mom, double eps)
{
    const long nl = 4 * volume(N);
#pragma omp parallel for schedule(static)
    for (long l = 0; l < nl; ++l) {
        cplx E[9];
#if ORACLE_MUTANT == 14
        /* planted: links move with exp(-i eps H) */
        oracle_exp_iH(mom + l * 9, -eps, E);
#else
        oracle_exp_iH(mom + l * 9, eps, E);
#endif
        m_mul(E, links + l * 9, links + l * 9);
    }
}

/* (1/2) sum Tr H^2 over all links. */
double oracle_mom_energy(const int N[4], const cplx *mom)
{
    const long nl = 4 * volume(N);
    double k = 0.0;
    for (long l = 0; l < nl; ++l) {
        const cplx *h = mom + l * 9;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) k += creal(h[i * 3 + j] * h[j * 3 + i]);
    }
    return 0.5 * k;
}

/* ------------------------------------------------------------------------ */
/* Stout smearing of the fermion links (Sec. 2.1: stout-improved staggered  */
/* action, Ref. Morningstar:2003gk; Sec. 2.2: up to a few stout levels)      */
/* ------------------------------------------------------------------------ */

/* Reading (the paper cites the method and prints no formula): isotropic
 * smearing with one weight rho per level,
 *   C_mu(x) = rho sum_{nu != mu} [ U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
 *                                 + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) ],
 *   Omega = C U^dag,  Q = (i/2)(Omega^dag - Omega) - (i/6) Tr(Omega^dag - Omega),
 *   U'_mu(x) = exp(i Q_mu(x)) U_mu(x);
 * n levels apply the map n times.  Q is Hermitian and traceless, so U' stays
 * in SU(3). */
static void stout_C(const int N[4], const cplx *links, const int x[4], int mu, double rho, cplx *C)
{
    cplx P[9];
    for (int i = 0; i < 9; ++i) C[i] = 0;
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        const int dir[3] = {nu, mu, nu};
        const int up[3] = {1, 1, -1}, dn[3] = {-1, 1, 1};
        path_product(N, links, x, 3, dir, up, P);
        for (int i = 0; i < 9; ++i) C[i] += rho * P[i];
#if ORACLE_MUTANT == 22
        /* planted: the lower staples are left out */
        (void)dn;
#else
        path_product(N, links, x, 3, dir, dn, P);
#if ORACLE_MUTANT == 23
        /* planted: the lower staples are added without the weight rho */
        for (int i = 0; i < 9; ++i) C[i] += P[i];
#else
        for (int i = 0; i < 9; ++i) C[i] += rho * P[i];
#endif
#endif
    }
}

static void stout_Q(const cplx *C, const cplx *U, cplx *Q)
{
    cplx Ud[9], Om[9];
    m_dag(U, Ud);
    m_mul(C, Ud, Om);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Q[i * 3 + j] = 0.5 * I * (conj(Om[j * 3 + i]) - Om[i * 3 + j]);
    const cplx tr = (Q[0] + Q[4] + Q[8]) / 3.0;
    Q[0] -= tr; Q[4] -= tr; Q[8] -= tr;
}

/* out = one stout level of in (both [4][V][3][3]). */
void oracle_stout_smear(const int N[4], const cplx *in, double rho, cplx *out)
{
    const long V = volume(N);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < V; ++n) {
        int x[4];
        long r = n;
        for (int m = 0; m < 4; ++m) { x[m] = (int)(r % N[m]); r /= N[m]; }
        for (int mu = 0; mu < 4; ++mu) {
            cplx C[9], Q[9], E[9];
            stout_C(N, in, x, mu, rho, C);
            const cplx *U = in + ((long)mu * V + n) * 9;
#if ORACLE_MUTANT == 18
            /* planted: the links move with exp(-iQ) */
            stout_Q(C, U, Q);
            oracle_exp_iH(Q, -1.0, E);
#else
            stout_Q(C, U, Q);
            oracle_exp_iH(Q, 1.0, E);
#endif
            m_mul(E, U, out + ((long)mu * V + n) * 9);
        }
    }
}

/* exp of an n x n complex matrix Z (n <= 6): power series after scaling by
 * 2^-k until the 1-norm is below 1/4, then k squarings. */
static void expm_n(int n, const cplx *Z, cplx *E)
{
    cplx S[36], T[36], W[36], Zs[36];
    double nrm = 0.0;
    for (int j = 0; j < n; ++j) {
        double c = 0.0;
        for (int i = 0; i < n; ++i) c += cabs(Z[i * n + j]);
        if (c > nrm) nrm = c;
    }
    int k = 0;
    while (nrm > 0.25 && k < 60) { nrm *= 0.5; ++k; }
    for (int i = 0; i < n * n; ++i) {
        Zs[i] = ldexp(1.0, -k) * Z[i];
        S[i] = T[i] = (i / n == i % n) ? 1.0 : 0.0;
    }
    for (int m = 1; m < 40; ++m) {
        double tn = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                cplx a = 0;
                for (int l = 0; l < n; ++l) a += T[i * n + l] * Zs[l * n + j];
                W[i * n + j] = a / m;
            }
        for (int i = 0; i < n * n; ++i) { T[i] = W[i]; S[i] += T[i]; tn += cabs(T[i]); }
        if (tn < 1e-18) break;
    }
    for (int q = 0; q < k; ++q) {
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                cplx a = 0;
                for (int l = 0; l < n; ++l) a += S[i * n + l] * S[l * n + j];
                W[i * n + j] = a;
            }
        memcpy(S, W, sizeof(cplx) * n * n);
    }
    memcpy(E, S, sizeof(cplx) * n * n);
}

/* D = d/dt exp(X + t A) at t = 0 (the Frechet derivative of exp at X in
 * the direction A) = the upper-right 3x3 block of exp([[X, A], [0, X]]). */
static void frechet_exp(const cplx *X, const cplx *A, cplx *D)
{
    cplx Z[36], E[36];
    for (int i = 0; i < 36; ++i) Z[i] = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            Z[i * 6 + j] = X[i * 3 + j];
            Z[(i + 3) * 6 + j + 3] = X[i * 3 + j];
            Z[i * 6 + j + 3] = A[i * 3 + j];
        }
    expm_n(6, Z, E);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) D[i * 3 + j] = E[i * 6 + j + 3];
}

static void m_add_scaled(cplx *G, double a, const cplx *B)
{
    for (int i = 0; i < 9; ++i) G[i] += a * B[i];
}

/* Force on the links of one stout level from the force on the smeared links
 * (Ref. Morningstar:2003gk, restated from the definitions).  Fp: Hermitian
 * traceless, d/de S(exp(i e X) U') = sum Tr(X Fp) for U' = smear(U); output
 * F, the same for U.  With Sigma' = -i U'^dag Fp, dS = Re Tr(Sigma' dU')
 * summed over the links for every variation that keeps U' in SU(3), and
 *   dU' = exp(iQ) dU + Dexp_{iQ}[i dQ] U,
 *   Re Tr(Sigma' Dexp_{iQ}[i dQ] U) = Re Tr(i Gamma dQ),  Gamma = Dexp_{iQ}[U Sigma']
 *     (the derivative of exp is self-adjoint under Tr(A B)),
 *   Re Tr(i Gamma dQ) = Re Tr(L dOmega),  L = traceless anti-Hermitian part of Gamma,
 *   dOmega = dC U^dag + C dU^dag.
 * The gradient G_mu(x) of S (dS = Re Tr(G dU) over the links) collects
 *   Sigma' exp(iQ) - C^dag L         at the link itself, and
 *   for each staple product P1 P2 P3 of C_mu(x), with M = U_mu(x)^dag L_mu(x)
 *   (times rho): Re Tr(M A dX B) -> G_X += B M A, Re Tr(M A dX^dag B) ->
 *   G_X += A^dag M^dag B^dag.
 * Then F = traceless part of (i/2)(U G - G^dag U^dag). */
void oracle_stout_force(const int N[4], const cplx *links, double rho, const cplx *Fp, cplx *F)
{
    const long V = volume(N), nl = 4 * V;
    cplx *G = calloc((size_t)nl * 9, sizeof(cplx));
    cplx *Mall = malloc(sizeof(cplx) * nl * 9);
    /* local terms and M per link */
    for (long n = 0; n < V; ++n) {
        int x[4];
        long r = n;
        for (int m = 0; m < 4; ++m) { x[m] = (int)(r % N[m]); r /= N[m]; }
        for (int mu = 0; mu < 4; ++mu) {
            const long l = (long)mu * V + n;
            const cplx *U = links + l * 9;
            cplx C[9], Q[9], E[9], Up[9], Upd[9], Sp[9], iQ[9], USp[9], Gam[9], L[9], Cd[9], t[9];
            stout_C(N, links, x, mu, rho, C);
            stout_Q(C, U, Q);
            oracle_exp_iH(Q, 1.0, E);
            m_mul(E, U, Up);
            m_dag(Up, Upd);
            m_mul(Upd, Fp + l * 9, Sp);
            for (int i = 0; i < 9; ++i) { Sp[i] *= -I; iQ[i] = I * Q[i]; }
            m_mul(U, Sp, USp);
            frechet_exp(iQ, USp, Gam);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) L[i * 3 + j] = 0.5 * (Gam[i * 3 + j] - conj(Gam[j * 3 + i]));
            const cplx tr = (L[0] + L[4] + L[8]) / 3.0;
            L[0] -= tr; L[4] -= tr; L[8] -= tr;
            m_mul(Sp, E, t);
            m_add_scaled(G + l * 9, 1.0, t);
            m_dag(C, Cd);
            m_mul(Cd, L, t);
#if ORACLE_MUTANT == 19
            /* planted: the C^dag L term enters with the wrong sign */
            m_add_scaled(G + l * 9, 1.0, t);
#else
            m_add_scaled(G + l * 9, -1.0, t);
#endif
            cplx Ud[9];
            m_dag(U, Ud);
            m_mul(Ud, L, Mall + l * 9);
        }
    }
    /* staple terms, scattered to the links of each staple */
    for (long n = 0; n < V; ++n) {
        int x[4];
        long r = n;
        for (int m = 0; m < 4; ++m) { x[m] = (int)(r % N[m]); r /= N[m]; }
        for (int mu = 0; mu < 4; ++mu) {
            const cplx *M = Mall + ((long)mu * V + n) * 9;
            cplx Md[9];
            m_dag(M, Md);
            for (int nu = 0; nu < 4; ++nu) {
                if (nu == mu) continue;
                int dm[4] = {0, 0, 0, 0}, dn[4] = {0, 0, 0, 0}, dmn[4] = {0, 0, 0, 0}, dnm[4] = {0, 0, 0, 0};
                const int z[4] = {0, 0, 0, 0};
                dm[mu] = 1;
                dn[nu] = 1;
                dmn[mu] = 1; dmn[nu] = -1;
                dnm[nu] = -1;
                int y[4];
                /* upper: U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag */
                const cplx *a1 = link(N, links, x, z, nu), *a2 = link(N, links, x, dn, mu),
                           *a3 = link(N, links, x, dm, nu);
                cplx a3d[9], B[9], T1[9], T2[9], a1d[9], a2d[9];
                m_dag(a3, a3d);
                m_mul(a2, a3d, B);                 /* X = a1, A = 1, B = a2 a3^dag: G += B M */
                m_mul(B, M, T1);
                shifted(N, x, z, y);
                m_add_scaled(G + ((long)nu * V + lex_index(N, y)) * 9, rho, T1);
                m_mul(a3d, M, T1);                 /* X = a2, A = a1, B = a3^dag: G += B M A */
                m_mul(T1, a1, T2);
                shifted(N, x, dn, y);
                m_add_scaled(G + ((long)mu * V + lex_index(N, y)) * 9, rho, T2);
                m_dag(a1, a1d);                    /* X = a3 (dag), A = a1 a2, B = 1: G += A^dag M^dag */
                m_dag(a2, a2d);
                m_mul(a2d, a1d, T1);
                m_mul(T1, Md, T2);
                shifted(N, x, dm, y);
                m_add_scaled(G + ((long)nu * V + lex_index(N, y)) * 9, rho, T2);
                /* lower: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) */
                const cplx *b1 = link(N, links, x, dnm, nu), *b2 = link(N, links, x, dnm, mu),
                           *b3 = link(N, links, x, dmn, nu);
                cplx b1d[9], Bd[9];
                m_mul(b2, b3, B);                  /* X = b1 (dag), A = 1, B = b2 b3: G += M^dag B^dag */
                m_dag(B, Bd);
                m_mul(Md, Bd, T1);
                shifted(N, x, dnm, y);
                m_add_scaled(G + ((long)nu * V + lex_index(N, y)) * 9, rho, T1);
                m_dag(b1, b1d);                    /* X = b2, A = b1^dag, B = b3: G += B M A */
                m_mul(b3, M, T1);
                m_mul(T1, b1d, T2);
                m_add_scaled(G + ((long)mu * V + lex_index(N, y)) * 9, rho, T2);
                m_mul(M, b1d, T1);                 /* X = b3, A = b1^dag b2, B = 1: G += M A */
                m_mul(T1, b2, T2);
                shifted(N, x, dmn, y);
                m_add_scaled(G + ((long)nu * V + lex_index(N, y)) * 9, rho, T2);
            }
        }
    }
    for (long l = 0; l < nl; ++l) {
        cplx UG[9];
        m_mul(links + l * 9, G + l * 9, UG);
        cplx *f = F + l * 9;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) f[i * 3 + j] = 0.5 * I * (UG[i * 3 + j] - conj(UG[j * 3 + i]));
        const cplx tr = (f[0] + f[4] + f[8]) / 3.0;
        f[0] -= tr; f[4] -= tr; f[8] -= tr;
    }
    free(G);
    free(Mall);
}

/* ------------------------------------------------------------------------ */
/* Timing support                                                            */
/* ------------------------------------------------------------------------ */

/* Set the threads of the parallel loops (n <= 0: one per processor); returns
 * the number in use (1 when built without OpenMP). */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int oracle_mutant(void) { return ORACLE_MUTANT; }

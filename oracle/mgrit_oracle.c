/*
 * Oracle: plain, slow FP64 CPU implementation of the MGRIT method of
 * Danieli & MacLachlan, "Multigrid Reduction in Time for non-linear hyperbolic
 * equations" (arXiv:2104.09404), for scalar 1D periodic conservation laws.
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it.  It shares no code, header,
 * table or helper with the CUDA library; the two only agree through the
 * mathematics written in the paper.
 *
 * Every routine follows the paper's equations in the paper's order, with
 * plain loops, no blocking and no fusion:
 *   flux f and its eigenvalue ..................... Sec. 2, Eq. (burgers)
 *   cell-average finite volumes, periodic ......... Sec. 2.1, Eq. (spaceDisc)
 *   WENO reconstruction, k = 2 tables ............. Sec. 2.1.1, Eqs. (C),(B),(omega),(D)
 *   k = 0 reconstruction .......................... Sec. 2.1.1 (closing remark)
 *   Lax-Friedrichs flux, global alpha ............. Sec. 2.1.2, Eq. (LFflux)
 *   Roe flux, Harten-Hyman entropy fix ............ Sec. 2.1.2, Eq. (roeflux)
 *   SSPRK3 / forward Euler ........................ Sec. 2.2, Eqs. (SSPRK3),(SSPRK1)
 *   F-/FCF-relaxation ............................. Sec. 3.2, Eq. (relaxation)
 *   injection + FAS restriction, coarse guess ..... Sec. 3.2, Eqs. (restriction::rhs),(restriction::u)
 *   coarsest sequential solve ..................... Sec. 3.2, Eq. (coarseCorr)
 *   ideal interpolation ........................... Sec. 3.2, Eq. (interpolation)
 *   V-cycle ....................................... Algorithm 1
 *   F-cycle ....................................... Sec. 3.2 (Fig. MGcycles)
 *   classical LF + FE fine scheme ................. Sec. 3.3, Eq. (fineLF)
 *   matched coarse integrators Psi0, Psi1 ......... Sec. 3.3, Eqs. (coarseLFord0),
 *                                                   (coarseLFord1), (fineLFxM)
 *
 * Readings of the paper taken where it is silent or inconsistent:
 *   - the WENO tables' row r acts on cells {i-r, i-r+1, i-r+2} (the printed
 *     rows, weights and smoothness matrices only agree with each other in
 *     that order);
 *   - the Lax-Friedrichs dissipation term enters with a minus sign
 *     (F = (f(u+)+f(u-))/2 - alpha (u+ - u-)/2), the dissipative choice;
 *   - alpha is global over the domain and recomputed at every RK stage;
 *   - the default numerical flux is the global Lax-Friedrichs *splitting*
 *     f^(+/-) = (f(u) +/- alpha u)/2 with WENO applied to f^+ (left-biased)
 *     and f^- (right-biased); the state-reconstruction form of Eq. (LFflux)
 *     is the variant NUMFLUX_LF_STATE;
 *   - nt counts time *steps*: nt+1 time points, dt = T/nt, nt/m chunks;
 *   - the residual is the Euclidean norm over all level-0 C-points i >= 1
 *     of Phi_0(u^{mi-1}) + g^{mi} - u^{mi}, taken right after the level-0
 *     relaxation of each cycle; the cycle stops there when it is < tol;
 *   - divergence: a non-finite residual or one above 1e8 times the first.
 *
 * Pinned by tests/test_oracle_*.py against closed forms (polynomial cell
 * averages, the smoothness-indicator integral of Eq. (B), the SSPRK3 Taylor
 * polynomial for a linear operator, exact shift of first-order upwind at
 * CFL 1, conservation, 5th-order accuracy, the exact entropy solution of
 * Burgers Riemann problems), against the k = 2 tables as printed
 * (tests/golden/, tests/test_golden_tables.py) and against the MGRIT
 * structure (fixed point = serial stepping, two-level exactness,
 * brute-force monolithic residual).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* identifiers passed in from Python; values chosen independently of the
 * CUDA library, which documents the same integers in its own header */
enum { ORC_SCHEME_WENO5_SSPRK3 = 0, ORC_SCHEME_FO_FE = 1, ORC_SCHEME_LF_FE = 2 };
enum { ORC_FLUX_BURGERS = 0, ORC_FLUX_ADVECTION = 1 };
enum { ORC_NUMFLUX_LF_SPLIT = 0, ORC_NUMFLUX_LF_STATE = 1, ORC_NUMFLUX_ROE = 2 };
enum { ORC_RELAX_F = 0, ORC_RELAX_FCF = 1 };
enum { ORC_GUESS_EQ17 = 0, ORC_GUESS_INJECT = 1 };
enum { ORC_CYCLE_V = 0, ORC_CYCLE_F = 1 };
enum { ORC_COARSE_REDISC = 0, ORC_COARSE_PSI0 = 1, ORC_COARSE_PSI1 = 2 };
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -3, ORC_EDIVERGED = -4,
       ORC_ENOTCONV = -5 };

#define WENO_EPS 1e-6

/* ---------------------------------------------------------------------- */
/* Physical flux, Sec. 2 Eq. (burgers); linear advection with speed 1.    */
/* ---------------------------------------------------------------------- */
static double phys_flux(int flux, double u)
{
    return flux == ORC_FLUX_BURGERS ? 0.5 * u * u : u;
}

/* eigenvalue of the flux Jacobian (Sec. 2.1.3: lambda = u for Burgers) */
static double phys_speed(int flux, double u)
{
    return flux == ORC_FLUX_BURGERS ? u : 1.0;
}

/* ---------------------------------------------------------------------- */
/* WENO reconstruction for k = 2, Sec. 2.1.1.                             */
/* The tables below are the paper's c_{r,j} (x 1/6), d_r (x 1/10) and     */
/* B_r (x 1/6), printed for k = 2.                                        */
/* ---------------------------------------------------------------------- */
static const double TAB_C[3][3] = {
    {  2.0,  5.0, -1.0 },
    { -1.0,  5.0,  2.0 },
    {  2.0, -7.0, 11.0 },
};
static const double TAB_D[3] = { 3.0, 6.0, 1.0 };
static const double TAB_B[3][3][3] = {
    { {  20.0, -31.0,  11.0 }, { -31.0,  50.0, -19.0 }, {  11.0, -19.0,   8.0 } },
    { {   8.0, -13.0,   5.0 }, { -13.0,  26.0, -13.0 }, {   5.0, -13.0,   8.0 } },
    { {   8.0, -19.0,  11.0 }, { -19.0,  50.0, -31.0 }, {  11.0, -31.0,  20.0 } },
};

/*
 * Left-of-interface value q^-_{i+1/2} from q[0..4] = q_{i-2..i+2}.
 * Row r of the tables uses the stencil {i-r, i-r+1, i-r+2}, i.e. the three
 * consecutive entries starting at q[2-r].  Outputs the candidate values
 * (Eq. C), smoothness indicators (Eq. B) and weights (Eq. omega) if the
 * pointers are non-NULL.
 */
static double weno5_left(const double q[5], double p_out[3], double beta_out[3],
                         double omega_out[3])
{
    double p[3], beta[3], alpha[3], asum = 0.0, w = 0.0;
    for (int r = 0; r < 3; ++r) {
        const double *s = &q[2 - r];
        /* Eq. (C): candidate reconstruction on stencil r */
        p[r] = (TAB_C[r][0] * s[0] + TAB_C[r][1] * s[1] + TAB_C[r][2] * s[2]) / 6.0;
        /* Eq. (B): beta_r = s^T B_r s.  Every row and column of the printed
         * B_r sums to zero, so beta_r(s) = beta_r(s - s_1 (1,1,1)); the form
         * is evaluated on the stencil minus its middle value, which avoids
         * cancelling O(|q|^2) terms when the data are smooth. */
        const double t[3] = { s[0] - s[1], 0.0, s[2] - s[1] };
        double qf = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                qf += t[a] * TAB_B[r][a][b] * t[b];
        beta[r] = qf / 6.0;
        /* Eq. (omega): alpha_r = d_r / (eps + beta_r)^2 */
        double den = WENO_EPS + beta[r];
        alpha[r] = (TAB_D[r] / 10.0) / (den * den);
        asum += alpha[r];
    }
    for (int r = 0; r < 3; ++r) {
        double om = alpha[r] / asum;
        if (omega_out) omega_out[r] = om;
        w += om * p[r];
    }
    if (p_out) memcpy(p_out, p, sizeof p);
    if (beta_out) memcpy(beta_out, beta, sizeof beta);
    return w;
}

static int wrap(int i, int nx)
{
    i %= nx;
    return i < 0 ? i + nx : i;
}

/* q^-_{i+1/2}: k = 2 WENO on q_{i-2..i+2}; k = 0 gives q_i */
static double recon_minus(int k, const double *q, int nx, int i)
{
    if (k == 0) return q[wrap(i, nx)];
    double s[5];
    for (int j = 0; j < 5; ++j) s[j] = q[wrap(i - 2 + j, nx)];
    return weno5_left(s, NULL, NULL, NULL);
}

/* q^+_{i+1/2}: the mirrored procedure on q_{i+3..i-1}; k = 0 gives q_{i+1} */
static double recon_plus(int k, const double *q, int nx, int i)
{
    if (k == 0) return q[wrap(i + 1, nx)];
    double s[5];
    for (int j = 0; j < 5; ++j) s[j] = q[wrap(i + 3 - j, nx)];
    return weno5_left(s, NULL, NULL, NULL);
}

static int scheme_k(int scheme) { return scheme == ORC_SCHEME_FO_FE ? 0 : 2; }

/* ---------------------------------------------------------------------- */
/* Semi-discrete operator A(u), Sec. 2.1 Eq. (spaceDisc):                 */
/*   A_i = -(F_{i+1/2} - F_{i-1/2}) / dx, periodic indices.               */
/* F[i] holds F_{i+1/2}.                                                  */
/* ---------------------------------------------------------------------- */
static void spatial_op(int nx, double dx, int scheme, int flux, int numflux,
                       const double *u, double *A, double *work /* 3*nx */)
{
    int k = scheme_k(scheme);
    double *F = work, *t1 = work + nx, *t2 = work + 2 * nx;
    double alpha = 0.0;
    if (numflux == ORC_NUMFLUX_LF_SPLIT) {
        /* global alpha over the cell values of this stage */
        for (int j = 0; j < nx; ++j) {
            double s = fabs(phys_speed(flux, u[j]));
            if (s > alpha) alpha = s;
        }
        for (int j = 0; j < nx; ++j) {
            t1[j] = 0.5 * (phys_flux(flux, u[j]) + alpha * u[j]);  /* f^+ */
            t2[j] = 0.5 * (phys_flux(flux, u[j]) - alpha * u[j]);  /* f^- */
        }
        for (int i = 0; i < nx; ++i)
            F[i] = recon_minus(k, t1, nx, i) + recon_plus(k, t2, nx, i);
    } else if (numflux == ORC_NUMFLUX_ROE) {
        /* Eq. (roeflux) for a scalar law on reconstructed states: Roe speed
         * lam = (f(u+) - f(u-)) / (u+ - u-), i.e. the Roe average (u+ + u-)/2
         * for Burgers and 1 for advection; eigenvalues at the states
         * lam-/+ = f'(u-/+); Harten-Hyman entropy fix
         *   delta = max(0, lam - lam-, lam+ - lam),
         *   q = (lam^2/delta + delta)/2 if |lam| < delta, else |lam|;
         *   F = (f(u-) + f(u+))/2 - q (u+ - u-)/2. */
        for (int i = 0; i < nx; ++i) {
            double um = recon_minus(k, u, nx, i), up = recon_plus(k, u, nx, i);
            double lam = flux == ORC_FLUX_BURGERS ? 0.5 * (up + um) : 1.0;
            double lm = flux == ORC_FLUX_BURGERS ? um : 1.0;
            double lp = flux == ORC_FLUX_BURGERS ? up : 1.0;
            double delta = 0.0;
            if (lam - lm > delta) delta = lam - lm;
            if (lp - lam > delta) delta = lp - lam;
            double q = fabs(lam) < delta ? 0.5 * (lam * lam / delta + delta) : fabs(lam);
            F[i] = 0.5 * (phys_flux(flux, um) + phys_flux(flux, up)) - 0.5 * q * (up - um);
        }
    } else {
        /* Eq. (LFflux) on reconstructed states, alpha over all u^{+/-} */
        for (int i = 0; i < nx; ++i) {
            t1[i] = recon_minus(k, u, nx, i);   /* u^-_{i+1/2} */
            t2[i] = recon_plus(k, u, nx, i);    /* u^+_{i+1/2} */
        }
        for (int i = 0; i < nx; ++i) {
            double a = fabs(phys_speed(flux, t1[i]));
            double b = fabs(phys_speed(flux, t2[i]));
            if (a > alpha) alpha = a;
            if (b > alpha) alpha = b;
        }
        for (int i = 0; i < nx; ++i)
            F[i] = 0.5 * (phys_flux(flux, t2[i]) + phys_flux(flux, t1[i]))
                 - 0.5 * alpha * (t2[i] - t1[i]);
    }
    for (int i = 0; i < nx; ++i)
        A[i] = -(F[i] - F[wrap(i - 1, nx)]) / dx;
}

/* ---------------------------------------------------------------------- */
/* Classical Lax-Friedrichs + forward Euler, Sec. 3.3 Eq. (fineLF):       */
/*   u_i^{n+1} = (E u)_i - dt (D f(u))_i,                                 */
/*   (E v)_i = (v_{i+1} + v_{i-1}) / 2,  (D v)_i = (v_{i+1} - v_{i-1})/2dx */
/* ---------------------------------------------------------------------- */
static void op_E(int nx, const double *v, double *out)
{
    for (int i = 0; i < nx; ++i) out[i] = 0.5 * (v[wrap(i + 1, nx)] + v[wrap(i - 1, nx)]);
}

static void op_D(int nx, double dx, const double *v, double *out)
{
    for (int i = 0; i < nx; ++i) out[i] = (v[wrap(i + 1, nx)] - v[wrap(i - 1, nx)]) / (2.0 * dx);
}

static void op_f(int nx, int flux, const double *v, double *out)
{
    for (int i = 0; i < nx; ++i) out[i] = phys_flux(flux, v[i]);
}

/* v <- E^k v (work: nx) */
static void op_E_pow(int nx, int k, double *v, double *work)
{
    for (int j = 0; j < k; ++j) {
        op_E(nx, v, work);
        memcpy(v, work, sizeof(double) * (size_t)nx);
    }
}

/* ---------------------------------------------------------------------- */
/* Time stepper Phi with step dt, Sec. 2.2: SSPRK3 (Eq. SSPRK3) or        */
/* forward Euler (Eq. SSPRK1); or Eq. (fineLF).  out may not alias u.     */
/* ---------------------------------------------------------------------- */
static void phi_step(int nx, double dx, double dt, int scheme, int flux, int numflux,
                     const double *u, double *out, double *work /* 6*nx */)
{
    double *A = work, *u1 = work + nx, *u2 = work + 2 * nx, *w3 = work + 3 * nx;
    if (scheme == ORC_SCHEME_LF_FE) {
        op_E(nx, u, u1);
        op_f(nx, flux, u, u2);
        op_D(nx, dx, u2, A);
        for (int i = 0; i < nx; ++i) out[i] = u1[i] - dt * A[i];
        return;
    }
    if (scheme == ORC_SCHEME_FO_FE) {
        spatial_op(nx, dx, scheme, flux, numflux, u, A, w3);
        for (int i = 0; i < nx; ++i) out[i] = u[i] + dt * A[i];
        return;
    }
    spatial_op(nx, dx, scheme, flux, numflux, u, A, w3);
    for (int i = 0; i < nx; ++i) u1[i] = u[i] + dt * A[i];
    spatial_op(nx, dx, scheme, flux, numflux, u1, A, w3);
    for (int i = 0; i < nx; ++i)
        u2[i] = 3.0 / 4.0 * u[i] + 1.0 / 4.0 * u1[i] + 1.0 / 4.0 * dt * A[i];
    spatial_op(nx, dx, scheme, flux, numflux, u2, A, w3);
    for (int i = 0; i < nx; ++i)
        out[i] = 1.0 / 3.0 * u[i] + 2.0 / 3.0 * u2[i] + 2.0 / 3.0 * dt * A[i];
}

/* ---------------------------------------------------------------------- */
/* Coarse integrators matched to M steps of Eq. (fineLF), Sec. 3.3        */
/* (Eqs. coarseLFord0, coarseLFord1, fineLFxM), dt the fine step:         */
/*   Psi0(u) = E^M u - M dt D f(u)                                        */
/*   Psi1(u) = E^M u - dt sum_{i=1..M} E^{i-1} D f(E^{M-i} u)             */
/* work: 4*nx                                                             */
/* ---------------------------------------------------------------------- */
static void psi_step(int nx, double dx, double dt, int M, int order, int flux,
                     const double *u, double *out, double *work)
{
    double *a = work, *b = work + nx, *c = work + 2 * nx, *t = work + 3 * nx;
    /* E^M u */
    memcpy(out, u, sizeof(double) * (size_t)nx);
    op_E_pow(nx, M, out, t);
    if (order == 0) {
        op_f(nx, flux, u, a);
        op_D(nx, dx, a, b);
        for (int i = 0; i < nx; ++i) out[i] -= M * dt * b[i];
        return;
    }
    for (int i = 1; i <= M; ++i) {
        memcpy(a, u, sizeof(double) * (size_t)nx);
        op_E_pow(nx, M - i, a, t);          /* E^{M-i} u */
        op_f(nx, flux, a, b);               /* f(E^{M-i} u) */
        op_D(nx, dx, b, c);                 /* D f(...) */
        op_E_pow(nx, i - 1, c, t);          /* E^{i-1} D f(...) */
        for (int x = 0; x < nx; ++x) out[x] -= dt * c[x];
    }
}

/* ====================================================================== */
/* Discrete adjoint of the stepper (vector-Jacobian products), by the     */
/* chain rule through Eq. (SSPRK3)/(SSPRK1), Eq. (spaceDisc), the global  */
/* Lax-Friedrichs splitting and the WENO weights of Eqs. (C),(B),(omega).  */
/* The paper has no adjoint; this is the gradient of J(u^{nt}) with       */
/* respect to u^0 for the discrete scheme above (split numerical flux).   */
/* ====================================================================== */

/* d q^-_{i+1/2} / d q[k], k = 0..4, for the reconstruction weno5_left:
 *   W = sum_r w_r p_r, w_r = a_r / sum a, a_r = d_r/(eps + beta_r)^2
 *   dW = sum_r w_r dp_r + (1/sum a) sum_r (p_r - W) da_r,
 *   da_r = -2 d_r/(eps + beta_r)^3 dbeta_r, dbeta_r = (B_r + B_r^T) s / 6 */
static void weno5_left_grad(const double q[5], double grad[5])
{
    double p[3], beta[3], alpha[3], dadb[3], asum = 0.0, w = 0.0;
    double dp[3][5], db[3][5];
    memset(dp, 0, sizeof dp);
    memset(db, 0, sizeof db);
    for (int r = 0; r < 3; ++r) {
        const double *s = &q[2 - r];
        p[r] = (TAB_C[r][0] * s[0] + TAB_C[r][1] * s[1] + TAB_C[r][2] * s[2]) / 6.0;
        /* beta_r and its gradient on the stencil minus its middle value, as in
         * weno5_left (both are invariant under adding a constant) */
        const double t[3] = { s[0] - s[1], 0.0, s[2] - s[1] };
        double qf = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                qf += t[a] * TAB_B[r][a][b] * t[b];
        beta[r] = qf / 6.0;
        for (int a = 0; a < 3; ++a) {
            dp[r][2 - r + a] = TAB_C[r][a] / 6.0;
            double g = 0.0;
            for (int b = 0; b < 3; ++b) g += (TAB_B[r][a][b] + TAB_B[r][b][a]) * t[b];
            db[r][2 - r + a] = g / 6.0;
        }
        double den = WENO_EPS + beta[r];
        alpha[r] = (TAB_D[r] / 10.0) / (den * den);
        dadb[r] = -2.0 * (TAB_D[r] / 10.0) / (den * den * den);
        asum += alpha[r];
    }
    for (int r = 0; r < 3; ++r) w += alpha[r] / asum * p[r];
    for (int k = 0; k < 5; ++k) {
        double g = 0.0;
        for (int r = 0; r < 3; ++r)
            g += alpha[r] / asum * dp[r][k] + (p[r] - w) * dadb[r] * db[r][k] / asum;
        grad[k] = g;
    }
}

/* out += A'(w)^T mu for the split numerical flux (alpha = max|f'(w_j)|,
 * differentiated at its first maximiser) */
static void spatial_op_vjp(int nx, double dx, int scheme, int flux, const double *w,
                           const double *mu, double *out, double *work /* 5*nx */)
{
    int k = scheme_k(scheme);
    double *fp = work, *fm = work + nx, *muF = work + 2 * nx, *mufp = work + 3 * nx,
           *mufm = work + 4 * nx;
    double alpha = 0.0;
    int kstar = -1;
    for (int j = 0; j < nx; ++j) {
        double sp = fabs(phys_speed(flux, w[j]));
        if (sp > alpha) { alpha = sp; kstar = j; }
    }
    for (int j = 0; j < nx; ++j) {
        fp[j] = 0.5 * (phys_flux(flux, w[j]) + alpha * w[j]);
        fm[j] = 0.5 * (phys_flux(flux, w[j]) - alpha * w[j]);
        mufp[j] = mufm[j] = 0.0;
    }
    /* A_i = -(F_i - F_{i-1})/dx with F_i = F_{i+1/2} */
    for (int i = 0; i < nx; ++i) muF[i] = (mu[wrap(i + 1, nx)] - mu[i]) / dx;
    for (int i = 0; i < nx; ++i) {
        if (k == 0) {
            mufp[i] += muF[i];
            mufm[wrap(i + 1, nx)] += muF[i];
            continue;
        }
        double s[5], g[5];
        for (int j = 0; j < 5; ++j) s[j] = fp[wrap(i - 2 + j, nx)];
        weno5_left_grad(s, g);
        for (int j = 0; j < 5; ++j) mufp[wrap(i - 2 + j, nx)] += muF[i] * g[j];
        for (int j = 0; j < 5; ++j) s[j] = fm[wrap(i + 3 - j, nx)];
        weno5_left_grad(s, g);
        for (int j = 0; j < 5; ++j) mufm[wrap(i + 3 - j, nx)] += muF[i] * g[j];
    }
    double mualpha = 0.0;
    for (int j = 0; j < nx; ++j) {
        double fprime = flux == ORC_FLUX_BURGERS ? w[j] : 1.0;
        out[j] += mufp[j] * 0.5 * (fprime + alpha) + mufm[j] * 0.5 * (fprime - alpha);
        mualpha += 0.5 * w[j] * (mufp[j] - mufm[j]);
    }
    if (flux == ORC_FLUX_BURGERS && kstar >= 0 && w[kstar] != 0.0)
        out[kstar] += mualpha * (w[kstar] > 0.0 ? 1.0 : -1.0);
}

/* lam_out = Phi'(u)^T lam (step dt) */
static void phi_step_vjp(int nx, double dx, double dt, int scheme, int flux, const double *u,
                         const double *lam, double *lam_out, double *work /* 12*nx */)
{
    double *A = work, *u1 = work + nx, *u2 = work + 2 * nx, *t = work + 3 * nx,
           *l2 = work + 4 * nx, *l1 = work + 5 * nx, *w5 = work + 6 * nx, *w3 = work + 11 * nx;
    (void)w3;
    if (scheme == ORC_SCHEME_FO_FE) {
        for (int i = 0; i < nx; ++i) { lam_out[i] = lam[i]; t[i] = dt * lam[i]; }
        spatial_op_vjp(nx, dx, scheme, flux, u, t, lam_out, w5);
        return;
    }
    /* forward stages (Eq. SSPRK3) */
    spatial_op(nx, dx, scheme, flux, ORC_NUMFLUX_LF_SPLIT, u, A, w5);
    for (int i = 0; i < nx; ++i) u1[i] = u[i] + dt * A[i];
    spatial_op(nx, dx, scheme, flux, ORC_NUMFLUX_LF_SPLIT, u1, A, w5);
    for (int i = 0; i < nx; ++i)
        u2[i] = 3.0 / 4.0 * u[i] + 1.0 / 4.0 * u1[i] + 1.0 / 4.0 * dt * A[i];
    /* stage 3: out = u/3 + 2/3 u2 + 2/3 dt A(u2) */
    for (int i = 0; i < nx; ++i) {
        lam_out[i] = 1.0 / 3.0 * lam[i];
        l2[i] = 2.0 / 3.0 * lam[i];
        t[i] = 2.0 / 3.0 * dt * lam[i];
    }
    spatial_op_vjp(nx, dx, scheme, flux, u2, t, l2, w5);
    /* stage 2: u2 = 3/4 u + 1/4 u1 + 1/4 dt A(u1) */
    for (int i = 0; i < nx; ++i) {
        lam_out[i] += 3.0 / 4.0 * l2[i];
        l1[i] = 1.0 / 4.0 * l2[i];
        t[i] = 1.0 / 4.0 * dt * l2[i];
    }
    spatial_op_vjp(nx, dx, scheme, flux, u1, t, l1, w5);
    /* stage 1: u1 = u + dt A(u) */
    for (int i = 0; i < nx; ++i) {
        lam_out[i] += l1[i];
        t[i] = dt * l1[i];
    }
    spatial_op_vjp(nx, dx, scheme, flux, u, t, lam_out, w5);
}

void orc_weno5_left_grad(const double *q5, double *grad5) { weno5_left_grad(q5, grad5); }

void orc_step_vjp(int nx, double Lx, double dt, int scheme, int flux, const double *u,
                  const double *lam, double *lam_out)
{
    double *work = malloc(sizeof(double) * 12 * (size_t)nx);
    phi_step_vjp(nx, Lx / nx, dt, scheme, flux, u, lam, lam_out, work);
    free(work);
}

/* dJ/du^0 for J = J(u^{nsteps}) given lamT = dJ/du^{nsteps}: forward serial
 * stepping stores every state, then lam^n = Phi'(u^n)^T lam^{n+1}. */
void orc_adjoint_serial(int nx, double Lx, double dt, int nsteps, int scheme, int flux,
                        const double *u0, const double *lamT, double *lam0)
{
    double *traj = malloc(sizeof(double) * (size_t)(nsteps + 1) * nx);
    double *work = malloc(sizeof(double) * 12 * (size_t)nx);
    double *a = malloc(sizeof(double) * (size_t)nx), *b = malloc(sizeof(double) * (size_t)nx);
    memcpy(traj, u0, sizeof(double) * (size_t)nx);
    for (int n = 0; n < nsteps; ++n)
        phi_step(nx, Lx / nx, dt, scheme, flux, ORC_NUMFLUX_LF_SPLIT, traj + (size_t)n * nx,
                 traj + (size_t)(n + 1) * nx, work);
    memcpy(a, lamT, sizeof(double) * (size_t)nx);
    for (int n = nsteps - 1; n >= 0; --n) {
        phi_step_vjp(nx, Lx / nx, dt, scheme, flux, traj + (size_t)n * nx, a, b, work);
        double *t = a; a = b; b = t;
    }
    memcpy(lam0, a, sizeof(double) * (size_t)nx);
    free(traj); free(work); free(a); free(b);
}

/* ====================================================================== */
/* Exported single-step pieces (pinned individually by the tests).        */
/* ====================================================================== */

double orc_weno5_left(const double *q5, double *p3, double *beta3, double *omega3)
{
    return weno5_left(q5, p3, beta3, omega3);
}

void orc_spatial_op(int nx, double Lx, int scheme, int flux, int numflux,
                    const double *u, double *A)
{
    double *work = malloc(sizeof(double) * 3 * (size_t)nx);
    spatial_op(nx, Lx / nx, scheme, flux, numflux, u, A, work);
    free(work);
}

void orc_step(int nx, double Lx, double dt, int scheme, int flux, int numflux,
              const double *u, double *out)
{
    double *work = malloc(sizeof(double) * 6 * (size_t)nx);
    phi_step(nx, Lx / nx, dt, scheme, flux, numflux, u, out, work);
    free(work);
}

void orc_psi_step(int nx, double Lx, double dt, int M, int order, int flux, const double *u,
                  double *out)
{
    double *work = malloc(sizeof(double) * 4 * (size_t)nx);
    psi_step(nx, Lx / nx, dt, M, order, flux, u, out, work);
    free(work);
}

/* Serial fine time-stepping u^{n+1} = Phi(u^n) (forward substitution of
 * Eq. monolithicSystem).  traj is (nsteps+1)*nx if store_all, else nx. */
void orc_serial(int nx, double Lx, double dt, int nsteps, int scheme, int flux,
                int numflux, const double *u0, double *traj, int store_all)
{
    double *work = malloc(sizeof(double) * 6 * (size_t)nx);
    double *a = malloc(sizeof(double) * (size_t)nx);
    double *b = malloc(sizeof(double) * (size_t)nx);
    memcpy(a, u0, sizeof(double) * (size_t)nx);
    if (store_all) memcpy(traj, u0, sizeof(double) * (size_t)nx);
    for (int n = 0; n < nsteps; ++n) {
        phi_step(nx, Lx / nx, dt, scheme, flux, numflux, a, b, work);
        double *t = a; a = b; b = t;
        if (store_all) memcpy(traj + (size_t)(n + 1) * nx, a, sizeof(double) * (size_t)nx);
    }
    if (!store_all) memcpy(traj, a, sizeof(double) * (size_t)nx);
    free(work); free(a); free(b);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ====================================================================== */
/* MGRIT, Sec. 3 and Algorithm 1, with full storage of every time point   */
/* on every level.                                                        */
/* ====================================================================== */

typedef struct {
    int nx, m, L, scheme, flux, numflux, relax, guess, cycle, coarse;
    double dx, dt0;
    int nt[32];            /* steps on level l: nt / m^l */
    double *u[32];         /* (nt_l + 1) * nx */
    double *g[32];         /* (nt_l + 1) * nx */
    /* adjoint mode: the propagator of step i on level l is the transposed
     * linearisation Phi_l'(U)^T at the forward state U of fine index
     * nt - i m^l (rows 0..nt-1 of traj), i.e. the same Algorithm 1 run
     * backward in time on lam^n = Phi'(u^n)^T lam^{n+1} */
    int adjoint;
    const double *traj;
} orc_mg;

static double *row(double *base, int nx, int i) { return base + (size_t)i * nx; }

static double level_dt(const orc_mg *M, int l)
{
    double dt = M->dt0;
    for (int i = 0; i < l; ++i) dt *= M->m;
    return dt;
}

/* the level-l propagator of the step that ends at point i, applied to x:
 * Phi_l(x), or in adjoint mode Phi_l'(U)^T x (work: 12*nx) */
static void propagate(const orc_mg *M, int l, int i, const double *x, double *y, double *work)
{
    if (!M->adjoint) {
        if (l > 0 && M->coarse != ORC_COARSE_REDISC) {
            /* matched coarse integrator: M_l = m^l fine steps of Eq. (fineLF) */
            int Ml = 1;
            for (int k = 0; k < l; ++k) Ml *= M->m;
            psi_step(M->nx, M->dx, M->dt0, Ml, M->coarse == ORC_COARSE_PSI1, M->flux, x, y, work);
            return;
        }
        phi_step(M->nx, M->dx, level_dt(M, l), M->scheme, M->flux, M->numflux, x, y, work);
        return;
    }
    long long s = 1;
    for (int k = 0; k < l; ++k) s *= M->m;
    const double *U = M->traj + (size_t)((long long)M->nt[0] - (long long)i * s) * M->nx;
    phi_step_vjp(M->nx, M->dx, level_dt(M, l), M->scheme, M->flux, U, x, y, work);
}

/* Phi_l(x) + g_l^{i} into y */
static void step_plus_g(const orc_mg *M, int l, const double *x, int gi, double *y,
                        double *work)
{
    propagate(M, l, gi, x, y, work);
    const double *g = row(M->g[l], M->nx, gi);
    for (int c = 0; c < M->nx; ++c) y[c] += g[c];
}

/* F-relaxation on level l, Eq. (relaxation): inside every chunk j,
 * u^{mj+r} = Phi_l(u^{mj+r-1}) + g^{mj+r}, r = 1..m-1.  Chunks are
 * independent (block-diagonal A_FF, Eq. AFF). */
static void f_relax(orc_mg *M, int l)
{
    int nx = M->nx, m = M->m, nc = M->nt[l] / m;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int j = 0; j < nc; ++j) {
        double *work = malloc(sizeof(double) * 12 * (size_t)nx);
        for (int r = 1; r < m; ++r)
            step_plus_g(M, l, row(M->u[l], nx, m * j + r - 1), m * j + r,
                        row(M->u[l], nx, m * j + r), work);
        free(work);
    }
}

/* C-relaxation: u^{mj} = Phi_l(u^{mj-1}) + g^{mj}, j = 1..nc */
static void c_relax(orc_mg *M, int l)
{
    int nx = M->nx, m = M->m, nc = M->nt[l] / m;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int j = 1; j <= nc; ++j) {
        double *work = malloc(sizeof(double) * 12 * (size_t)nx);
        step_plus_g(M, l, row(M->u[l], nx, m * j - 1), m * j, row(M->u[l], nx, m * j), work);
        free(work);
    }
}

static void relax(orc_mg *M, int l)
{
    f_relax(M, l);
    if (M->relax == ORC_RELAX_FCF) {
        c_relax(M, l);
        f_relax(M, l);
    }
}

/*
 * Residual at the C-points of level l and FAS restriction to level l+1,
 * Eqs. (restriction::rhs) and (restriction::u):
 *   phi_i      = Phi_l(u_l^{mi-1})
 *   r^i        = phi_i + g_l^{mi} - u_l^{mi}                 (returned ||r||^2)
 *   g_{l+1}^i  = g_l^{mi} + phi_i - Phi_{l+1}(u_l^{m(i-1)})
 *   u_{l+1}^i  = phi_i + g_l^{mi}  (Eq. restriction::u)  or  u_l^{mi} (injection)
 * for i = 1..nt_l/m, and g_{l+1}^0 = g_l^0, u_{l+1}^0 = u_l^0.
 * If do_restrict is 0 only the residual is formed.
 */
static double residual_restrict(orc_mg *M, int l, int do_restrict)
{
    int nx = M->nx, m = M->m, nc = M->nt[l] / m;
    double *rsq = calloc((size_t)nc + 1, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int i = 1; i <= nc; ++i) {
        double *work = malloc(sizeof(double) * 12 * (size_t)nx);
        double *phi = malloc(sizeof(double) * (size_t)nx);
        double *psi = malloc(sizeof(double) * (size_t)nx);
        const double *gl = row(M->g[l], nx, m * i);
        const double *ul = row(M->u[l], nx, m * i);
        propagate(M, l, m * i, row(M->u[l], nx, m * i - 1), phi, work);
        double s = 0.0;
        for (int c = 0; c < nx; ++c) {
            double r = phi[c] + gl[c] - ul[c];
            s += r * r;
        }
        rsq[i] = s;
        if (do_restrict) {
            propagate(M, l + 1, i, row(M->u[l], nx, m * (i - 1)), psi, work);
            double *gc = row(M->g[l + 1], nx, i);
            double *uc = row(M->u[l + 1], nx, i);
            for (int c = 0; c < nx; ++c) {
                gc[c] = gl[c] + phi[c] - psi[c];
                uc[c] = (M->guess == ORC_GUESS_EQ17) ? phi[c] + gl[c] : ul[c];
            }
        }
        free(work); free(phi); free(psi);
    }
    if (do_restrict) {
        memcpy(row(M->g[l + 1], nx, 0), row(M->g[l], nx, 0), sizeof(double) * (size_t)nx);
        memcpy(row(M->u[l + 1], nx, 0), row(M->u[l], nx, 0), sizeof(double) * (size_t)nx);
    }
    double tot = 0.0;
    for (int i = 1; i <= nc; ++i) tot += rsq[i];
    free(rsq);
    return tot;
}

/* coarsest level, Eq. (coarseCorr): forward substitution with S_Phi */
static void coarse_solve(orc_mg *M, int l)
{
    int nx = M->nx;
    double *work = malloc(sizeof(double) * 12 * (size_t)nx);
    memcpy(row(M->u[l], nx, 0), row(M->g[l], nx, 0), sizeof(double) * (size_t)nx);
    for (int i = 1; i <= M->nt[l]; ++i)
        step_plus_g(M, l, row(M->u[l], nx, i - 1), i, row(M->u[l], nx, i), work);
    free(work);
}

/* Interpolation, Eq. (interpolation): inject level-(l+1) values into the
 * C-points of level l, then F-relax level l (skipped when do_frelax = 0). */
static void interpolate(orc_mg *M, int l, int do_frelax)
{
    int nx = M->nx, m = M->m, nc = M->nt[l] / m;
    for (int i = 0; i <= nc; ++i)
        memcpy(row(M->u[l], nx, m * i), row(M->u[l + 1], nx, i), sizeof(double) * (size_t)nx);
    if (do_frelax) f_relax(M, l);
}

/* Algorithm 1, entered below level 0 (level 0's relaxation and residual
 * are driven by orc_mgrit so that the stopping test sits between them). */
static void vcycle_from(orc_mg *M, int l)
{
    if (l < M->L - 1) {
        relax(M, l);
        residual_restrict(M, l, 1);
        vcycle_from(M, l + 1);
        interpolate(M, l, 1);
    } else {
        coarse_solve(M, l);
    }
}

/* F-cycle (Sec. 3.2, the cycle sketch of Fig. MGcycles; the standard
 * multigrid F-cycle): below a level, first an F-cycle, then one V-cycle,
 * each with the level's relaxation, restriction and interpolation around it. */
static void fcycle_from(orc_mg *M, int l)
{
    if (l < M->L - 1) {
        relax(M, l);
        residual_restrict(M, l, 1);
        fcycle_from(M, l + 1);
        interpolate(M, l, 1);
        relax(M, l);
        residual_restrict(M, l, 1);
        vcycle_from(M, l + 1);
        interpolate(M, l, 1);
    } else {
        coarse_solve(M, l);
    }
}

static void cycle_from(orc_mg *M, int l)
{
    if (M->cycle == ORC_CYCLE_F)
        fcycle_from(M, l);
    else
        vcycle_from(M, l);
}

static void mg_free(orc_mg *M)
{
    for (int l = 0; l < M->L; ++l) { free(M->u[l]); free(M->g[l]); }
}

static int mg_init(orc_mg *M, int nx, int nt, int m, int levels, int scheme, int flux,
                   int numflux, double Lx, double T, int relax_kind, int guess, int cycle,
                   int coarse)
{
    if (nx < 1 || nt < 1 || m < 2 || levels < 2 || levels > 31) return ORC_EINVAL;
    if (cycle != ORC_CYCLE_V && cycle != ORC_CYCLE_F) return ORC_EINVAL;
    if (coarse < ORC_COARSE_REDISC || coarse > ORC_COARSE_PSI1) return ORC_EINVAL;
    if (coarse != ORC_COARSE_REDISC && scheme != ORC_SCHEME_LF_FE) return ORC_EINVAL;
    if (scheme == ORC_SCHEME_LF_FE && nx < 3) return ORC_EINVAL;
    if (scheme == ORC_SCHEME_WENO5_SSPRK3 && nx < 5) return ORC_EINVAL;
    memset(M, 0, sizeof *M);
    M->nx = nx; M->m = m; M->L = levels; M->scheme = scheme; M->flux = flux;
    M->numflux = numflux; M->relax = relax_kind; M->guess = guess; M->cycle = cycle;
    M->coarse = coarse;
    M->dx = Lx / nx; M->dt0 = T / nt;
    long long div = 1;
    for (int l = 0; l < levels; ++l) {
        if (nt % div) return ORC_EINVAL;
        M->nt[l] = (int)(nt / div);
        if (l < levels - 1 && M->nt[l] % m) return ORC_EINVAL;
        div *= m;
    }
    for (int l = 0; l < levels; ++l) {
        size_t n = (size_t)(M->nt[l] + 1) * nx;
        M->u[l] = calloc(n, sizeof(double));
        M->g[l] = calloc(n, sizeof(double));
        if (!M->u[l] || !M->g[l]) { mg_free(M); return ORC_ENOMEM; }
    }
    return ORC_OK;
}

/* Cycle k: relax level 0, r_k = ||residual||; stop if r_k < tol; divergence
 * if r_k is not finite or r_k > 1e8 r_0; give up after max_iter cycles;
 * otherwise restrict, recurse, inject. */
static int mg_loop(orc_mg *M, double tol, int max_iter, int *iters_out, double *res_hist)
{
    double r0 = 0.0;
    int k = 0, st;
    for (;; ++k) {
        relax(M, 0);
        double rk = sqrt(residual_restrict(M, 0, 0));
        if (res_hist) res_hist[k] = rk;
        if (k == 0) r0 = rk;
        if (rk < tol) { st = ORC_OK; break; }
        if (!isfinite(rk) || rk > 1e8 * r0) { st = ORC_EDIVERGED; break; }
        if (k >= max_iter) { st = ORC_ENOTCONV; break; }
        residual_restrict(M, 0, 1);
        cycle_from(M, 1);
        interpolate(M, 0, 0);
    }
    if (iters_out) *iters_out = k;
    return st;
}

/*
 * Full FAS MGRIT V-cycle solve.  Level-0 initial iterate: every C-point is
 * uC_init (if given, (nt/m+1)*nx) else u0; g_0 = [u0, 0, ..., 0].
 * Cycle k: relax level 0, r_k = ||residual||; stop if r_k < tol; divergence
 * if r_k is not finite or r_k > 1e8 r_0; give up after max_iter cycles;
 * otherwise restrict, recurse, inject.  On exit the level-0 C-points are
 * those after the last relaxation and the F-points are consistent with them.
 * Returns ORC_OK / ORC_EDIVERGED / ORC_ENOTCONV / ORC_EINVAL.
 */
int orc_mgrit(int nx, int nt, int m, int levels, int scheme, int flux, int numflux,
              double Lx, double T, int relax_kind, int guess, int cycle, int coarse,
              double tol, int max_iter,
              const double *u0, const double *uC_init, double *uC_out, double *u_full_out,
              double *uT_out, int *iters_out, double *res_hist)
{
    orc_mg M;
    int st = mg_init(&M, nx, nt, m, levels, scheme, flux, numflux, Lx, T, relax_kind, guess,
                     cycle, coarse);
    if (st) return st;
    size_t rowb = sizeof(double) * (size_t)nx;
    memcpy(row(M.g[0], nx, 0), u0, rowb);
    for (int i = 0; i <= M.nt[0]; ++i) {
        const double *src = u0;
        if (uC_init && i % m == 0) src = uC_init + (size_t)(i / m) * nx;
        memcpy(row(M.u[0], nx, i), src, rowb);
    }
    memcpy(row(M.u[0], nx, 0), u0, rowb);
    st = mg_loop(&M, tol, max_iter, iters_out, res_hist);
    if (uC_out)
        for (int i = 0; i <= M.nt[0] / m; ++i)
            memcpy(uC_out + (size_t)i * nx, row(M.u[0], nx, m * i), rowb);
    if (u_full_out) memcpy(u_full_out, M.u[0], rowb * (size_t)(M.nt[0] + 1));
    if (uT_out) memcpy(uT_out, row(M.u[0], nx, M.nt[0]), rowb);
    mg_free(&M);
    return st;
}

/*
 * Exactly ncycles V-cycles from the initial iterate (all C-points = u0), each
 * recording the level-0 residual after its relaxation; no stopping test.
 * Used to time the oracle on the same work as one GPU V-cycle.  The final
 * level-0 C-points (after the last cycle's relaxation) go to uC_out if given.
 */
int orc_vcycles(int nx, int nt, int m, int levels, int scheme, int flux, int numflux,
                double Lx, double T, int relax_kind, int guess, int cycle, int coarse,
                int ncycles,
                const double *u0, double *uC_out, double *res_hist)
{
    orc_mg M;
    int st = mg_init(&M, nx, nt, m, levels, scheme, flux, numflux, Lx, T, relax_kind, guess,
                     cycle, coarse);
    if (st) return st;
    size_t rowb = sizeof(double) * (size_t)nx;
    memcpy(row(M.g[0], nx, 0), u0, rowb);
    for (int i = 0; i <= M.nt[0]; ++i) memcpy(row(M.u[0], nx, i), u0, rowb);
    for (int k = 0; k < ncycles; ++k) {
        relax(&M, 0);
        double rk = sqrt(residual_restrict(&M, 0, 1));
        if (res_hist) res_hist[k] = rk;
        cycle_from(&M, 1);
        interpolate(&M, 0, 0);
    }
    if (uC_out)
        for (int i = 0; i <= M.nt[0] / m; ++i)
            memcpy(uC_out + (size_t)i * nx, row(M.u[0], nx, m * i), rowb);
    mg_free(&M);
    return ORC_OK;
}

/*
 * Adjoint MGRIT: dJ/du^0 = lam^0 of lam^n = Phi'(u^n)^T lam^{n+1}, lam^nt =
 * lamT, solved by the V-cycle above backward in time.  In reversed time
 * k = nt - n the system is v^k = Phi'(u^{nt-k})^T v^{k-1}, v^0 = lamT: a
 * linear forward-substitution system of the same block-bidiagonal form as
 * Eq. (monolithicSystem), so Algorithm 1 applies unchanged with the
 * propagator of step k on level l = Phi_l'(U)^T at the forward state of fine
 * index nt - k m^l (the coarse operator linearised at the injected forward
 * C-state).  The paper has no adjoint; this is its method applied to the
 * adjoint system.
 * The forward fine states are regenerated chunk by chunk from the forward
 * C-point checkpoints uC ((nt/m+1)*nx): u^{mj+r} = Phi^r(uC_j), r < m.
 * Split numerical flux only.  Outputs: lam0_out (nx) and, if given,
 * lamC_out with row i = lam at forward point m*i, i = 0..nt/m.
 */
int orc_adjoint_mgrit(int nx, int nt, int m, int levels, int scheme, int flux, double Lx,
                      double T, int relax_kind, int guess, int cycle, double tol, int max_iter,
                      const double *uC, const double *lamT, double *lam0_out,
                      double *lamC_out, int *iters_out, double *res_hist)
{
    orc_mg M;
    if (scheme == ORC_SCHEME_LF_FE) return ORC_EINVAL;   /* no adjoint of Eq. (fineLF) */
    int st = mg_init(&M, nx, nt, m, levels, scheme, flux, ORC_NUMFLUX_LF_SPLIT, Lx, T,
                     relax_kind, guess, cycle, ORC_COARSE_REDISC);
    if (st) return st;
    size_t rowb = sizeof(double) * (size_t)nx;
    double *traj = malloc(rowb * (size_t)nt);
    if (!traj) { mg_free(&M); return ORC_ENOMEM; }
    int nc = nt / m;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int j = 0; j < nc; ++j) {
        double *work = malloc(sizeof(double) * 6 * (size_t)nx);
        memcpy(row(traj, nx, m * j), uC + (size_t)j * nx, rowb);
        for (int r = 1; r < m; ++r)
            phi_step(nx, M.dx, M.dt0, scheme, flux, ORC_NUMFLUX_LF_SPLIT,
                     row(traj, nx, m * j + r - 1), row(traj, nx, m * j + r), work);
        free(work);
    }
    M.adjoint = 1;
    M.traj = traj;
    memcpy(row(M.g[0], nx, 0), lamT, rowb);
    for (int i = 0; i <= M.nt[0]; ++i) memcpy(row(M.u[0], nx, i), lamT, rowb);
    st = mg_loop(&M, tol, max_iter, iters_out, res_hist);
    if (lam0_out) memcpy(lam0_out, row(M.u[0], nx, nt), rowb);
    if (lamC_out)
        for (int i = 0; i <= nc; ++i)
            memcpy(lamC_out + (size_t)i * nx, row(M.u[0], nx, nt - m * i), rowb);
    free(traj);
    mg_free(&M);
    return st;
}

/* ||r|| for given level-0 C-points uC ((nt/m+1)*nx): each chunk is stepped
 * m times from its C-point and compared with the next C-point. */
int orc_residual(int nx, int nt, int m, int scheme, int flux, int numflux, double Lx,
                 double T, const double *uC, double *norm_out)
{
    if (nx < 1 || m < 2 || nt % m) return ORC_EINVAL;
    int nc = nt / m;
    double dx = Lx / nx, dt = T / nt;
    double *rsq = calloc((size_t)nc + 1, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int i = 1; i <= nc; ++i) {
        double *work = malloc(sizeof(double) * 6 * (size_t)nx);
        double *a = malloc(sizeof(double) * (size_t)nx);
        double *b = malloc(sizeof(double) * (size_t)nx);
        memcpy(a, uC + (size_t)(i - 1) * nx, sizeof(double) * (size_t)nx);
        for (int r = 0; r < m; ++r) {
            phi_step(nx, dx, dt, scheme, flux, numflux, a, b, work);
            double *t = a; a = b; b = t;
        }
        double s = 0.0;
        const double *c = uC + (size_t)i * nx;
        for (int x = 0; x < nx; ++x) { double r = a[x] - c[x]; s += r * r; }
        rsq[i] = s;
        free(work); free(a); free(b);
    }
    double tot = 0.0;
    for (int i = 1; i <= nc; ++i) tot += rsq[i];
    free(rsq);
    *norm_out = sqrt(tot);
    return ORC_OK;
}

/*
 * FP64 CPU oracle for the hybrid-QMC hot path of "Scalable hybrid quantum
 * Monte Carlo simulation of U(1) gauge field coupled to fermions on GPU"
 * (arXiv 2508.16298).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the GPU library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no code, header, table or helper with the CUDA library.
 *
 * Everything is double precision and follows the paper's definitions in
 * their printed order, with no fusion, blocking or reordering:
 *   - 2x2 bond exponential exp(a T_ij) = cosh(a) 1 + sinh(a) T_ij,
 *     T_ij = [[0, e^{i phi_ij}], [e^{-i phi_ij}, 0]]      (Methods, "Matrix-free
 *     representation of M^dagger M v", the family exponential after Eq. (eq24))
 *   - symmetric checkerboard B = e^{V4/2} e^{V3/2} e^{V2/2} e^{V1/2} e^{V1/2}
 *     e^{V2/2} e^{V3/2} e^{V4/2}, V_fam = dtau*t * (+) T_ij            (Eq. (eq24))
 *   - block-cyclic fermion matrix M: identity diagonal, -B_tau below the
 *     diagonal, +B_Ntau in the top-right corner              (Eq. (M_alpha))
 *   - CG recurrence for (M^dagger M) X = v with the identity preconditioner
 *                                                              (Eq. (pCG))
 *   - fermion force -d/dphi [eta^dagger (M^dagger M)^{-1} eta]
 *                          (Supplement SI, Eqs. (force&CG), (fermion_force))
 *   - bosonic actions L_B^c and L_B^nc                  (Results, Eq. (eq3))
 *   - H = S_B + sum p^2 + eta^dagger (M^dagger M)^{-1} eta       (Eq. (H_hmc))
 *   - leapfrog with dphi/dt = 2p                   (Eqs. (H_diff), (leapfrog))
 *   - Metropolis accept with probability min(1, e^{H0 - H1})
 *                                          (Methods, HQMC step (iii))
 *
 * Conventions (the paper leaves these to the reader):
 *   tau = 0..Ntau-1 (0-based: slice tau carries the paper's B_{tau+1});
 *   site s = x + L*y; theta[((tau*L + y)*L + x)*2 + c], c = 0 the bond
 *   (x,y)->(x+1,y), c = 1 the bond (x,y)->(x,y+1), periodic in space;
 *   vectors are complex double v[(tau*L + y)*L + x].
 *   Bond families: 1 = x-bonds with even tail x, 2 = x-bonds with odd tail x
 *   (includes the wrap L-1 -> 0), 3 = y-bonds with even tail y, 4 = y-bonds
 *   with odd tail y.  L must be even so that every family pairs every site.
 *
 * Parity status: every function here is pinned by tests that do not call it
 * back (dense matrices built with matrix exponentials, closed-form spectra,
 * gauge covariance, finite differences, integrator invariants).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
    int L;          /* spatial extent (even) */
    int Ntau;       /* number of imaginary-time slices */
    double dtau;    /* Trotter step Delta tau */
    double t;       /* hopping amplitude */
    double J;       /* gauge coupling */
    double K;       /* plaquette coupling */
    int noncompact; /* 0: compact action L_B^c, 1: non-compact L_B^nc */
} orc_lattice;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int wrap(int a, int L) { return ((a % L) + L) % L; }
static long vol(const orc_lattice* lat) { return (long)lat->L * lat->L; }

/* ------------------------------------------------------------------------ */
/* Checkerboard factors                                                     */
/* ------------------------------------------------------------------------ */

/* The seven factors of B in matrix-product order (leftmost first), Eq. (eq24)
 * with the two middle e^{V1/2} written as one e^{V1}.  Each entry is the
 * family and the multiple of dtau*t in the exponent. */
static const int FACTOR_FAMILY[7] = {4, 3, 2, 1, 2, 3, 4};
static const double FACTOR_WEIGHT[7] = {0.5, 0.5, 0.5, 1.0, 0.5, 0.5, 0.5};

/* Bond number b (0 .. L*L/2 - 1) of family fam: tail site i and head site j,
 * and the index of its angle inside one slice of theta. */
static void family_bond(int L, int fam, int b, int* i, int* j, int* th) {
    int half = L / 2;
    if (fam == 1 || fam == 2) {
        int y = b / half, k = b % half;
        int x = 2 * k + (fam == 2 ? 1 : 0);
        *i = x + L * y;
        *j = wrap(x + 1, L) + L * y;
        *th = 2 * (*i) + 0;
    } else {
        int x = b % L, k = b / L;
        int y = 2 * k + (fam == 4 ? 1 : 0);
        *i = x + L * y;
        *j = x + L * wrap(y + 1, L);
        *th = 2 * (*i) + 1;
    }
}

/* v <- exp(alpha * (+)_{ij in fam} T_ij) v, or its conjugate transpose.
 * On every bond (i,j) the 2x2 block is [[cosh a, e^{i phi} sinh a],
 * [e^{-i phi} sinh a, cosh a]] acting on (v_i, v_j). */
static void apply_family(int L, int fam, double alpha, const double* th_slice,
                         cplx* v, int adjoint) {
    int nb = L * L / 2;
    double ch = cosh(alpha), sh = sinh(alpha);
    for (int b = 0; b < nb; ++b) {
        int i, j, k;
        family_bond(L, fam, b, &i, &j, &k);
        cplx e = cexp(I * th_slice[k]);
        cplx m00 = ch, m01 = sh * e, m10 = sh * conj(e), m11 = ch;
        if (adjoint) {
            cplx t01 = conj(m10), t10 = conj(m01);
            m00 = conj(m00); m11 = conj(m11); m01 = t01; m10 = t10;
        }
        cplx vi = v[i], vj = v[j];
        v[i] = m00 * vi + m01 * vj;
        v[j] = m10 * vi + m11 * vj;
    }
}

/* out = B v (adjoint = 0) or B^dagger v (adjoint = 1) for one slice. */
void orc_apply_B(const orc_lattice* lat, const double* th_slice, const cplx* in,
                 cplx* out, int adjoint) {
    long V = vol(lat);
    double a = lat->dtau * lat->t;
    memcpy(out, in, sizeof(cplx) * V);
    if (!adjoint) {
        /* B v: the rightmost factor acts first. */
        for (int k = 6; k >= 0; --k)
            apply_family(lat->L, FACTOR_FAMILY[k], FACTOR_WEIGHT[k] * a, th_slice, out, 0);
    } else {
        /* B^dagger = F_7^dagger ... F_1^dagger: F_1^dagger acts first. */
        for (int k = 0; k <= 6; ++k)
            apply_family(lat->L, FACTOR_FAMILY[k], FACTOR_WEIGHT[k] * a, th_slice, out, 1);
    }
}

/* ------------------------------------------------------------------------ */
/* Fermion matrix, Eq. (M_alpha)                                            */
/* ------------------------------------------------------------------------ */

/* y = M x (dagger = 0) or y = M^dagger x (dagger = 1).
 * Row tau of M (0-based): (M x)_tau = x_tau - B_{tau-1} x_{tau-1} for tau >= 1
 * and (M x)_0 = x_0 + B_{Ntau-1} x_{Ntau-1}.  Its adjoint reads
 * (M^dagger x)_tau = x_tau - B_tau^dagger x_{tau+1} for tau < Ntau-1 and
 * (M^dagger x)_{Ntau-1} = x_{Ntau-1} + B_{Ntau-1}^dagger x_0. */
void orc_apply_M(const orc_lattice* lat, const double* theta, const cplx* x,
                 cplx* y, int dagger) {
    long V = vol(lat);
    int N = lat->Ntau;
#pragma omp parallel
    {
        cplx* tmp = (cplx*)malloc(sizeof(cplx) * V);
#pragma omp for schedule(static)
        for (int tau = 0; tau < N; ++tau) {
            if (!dagger) {
                int src = (tau == 0) ? N - 1 : tau - 1;
                double sign = (tau == 0) ? +1.0 : -1.0;
                orc_apply_B(lat, theta + (long)src * V * 2, x + (long)src * V, tmp, 0);
                for (long s = 0; s < V; ++s)
                    y[(long)tau * V + s] = x[(long)tau * V + s] + sign * tmp[s];
            } else {
                int src = (tau == N - 1) ? 0 : tau + 1;
                double sign = (tau == N - 1) ? +1.0 : -1.0;
                orc_apply_B(lat, theta + (long)tau * V * 2, x + (long)src * V, tmp, 1);
                for (long s = 0; s < V; ++s)
                    y[(long)tau * V + s] = x[(long)tau * V + s] + sign * tmp[s];
            }
        }
        free(tmp);
    }
}

/* y = M^dagger (M x), two plain applications. */
void orc_apply_MdagM(const orc_lattice* lat, const double* theta, const cplx* x, cplx* y) {
    long n = vol(lat) * lat->Ntau;
    cplx* t = (cplx*)malloc(sizeof(cplx) * n);
    orc_apply_M(lat, theta, x, t, 0);
    orc_apply_M(lat, theta, t, y, 1);
    free(t);
}

/* <a, b> = sum conj(a_i) b_i, summed in index order. */
void orc_dot(long n, const cplx* a, const cplx* b, double* re, double* im) {
    cplx s = 0;
    for (long i = 0; i < n; ++i) s += conj(a[i]) * b[i];
    *re = creal(s);
    *im = cimag(s);
}

static double norm2(long n, const cplx* a) {
    double s = 0;
    for (long i = 0; i < n; ++i) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return s;
}

/* ------------------------------------------------------------------------ */
/* Conjugate gradient, Eq. (pCG) with the identity preconditioner           */
/* ------------------------------------------------------------------------ */

/* Solves (M^dagger M) X = v.  X holds the initial guess on entry (zero for
 * the paper's X_0 = 0) and the solution on exit.  Stops when the recursive
 * residual satisfies ||r|| <= tol ||v||; then the true residual
 * ||v - O X|| / ||v|| is recomputed, and if it exceeds tol the recurrence is
 * restarted from the true residual (same iteration budget).
 * Returns 0 on convergence, 1 if maxit applications of O were used up. */
int orc_cg(const orc_lattice* lat, const double* theta, const cplx* v, cplx* X,
           double tol, int maxit, int* iters_out, double* true_res_out) {
    long n = vol(lat) * lat->Ntau;
    cplx* r = (cplx*)malloc(sizeof(cplx) * n);
    cplx* d = (cplx*)malloc(sizeof(cplx) * n);
    cplx* Od = (cplx*)malloc(sizeof(cplx) * n);
    double vv = norm2(n, v);
    int iters = 0, status = 1;
    double true_res = 0.0;
    if (vv == 0.0) {
        memset(X, 0, sizeof(cplx) * n);
        *iters_out = 0;
        *true_res_out = 0.0;
        free(r); free(d); free(Od);
        return 0;
    }
    for (;;) {
        /* r_0 = v - O X_0, d_0 = r_0 */
        orc_apply_MdagM(lat, theta, X, Od);
        for (long i = 0; i < n; ++i) { r[i] = v[i] - Od[i]; d[i] = r[i]; }
        double rr = norm2(n, r);
        while (rr > tol * tol * vv && iters < maxit) {
            orc_apply_MdagM(lat, theta, d, Od);
            ++iters;
            double dOd_re, dOd_im;
            orc_dot(n, d, Od, &dOd_re, &dOd_im);
            double zeta = rr / dOd_re;
            for (long i = 0; i < n; ++i) X[i] += zeta * d[i];
            for (long i = 0; i < n; ++i) r[i] -= zeta * Od[i];
            double rr_new = norm2(n, r);
            double rho = rr_new / rr;
            for (long i = 0; i < n; ++i) d[i] = r[i] + rho * d[i];
            rr = rr_new;
        }
        orc_apply_MdagM(lat, theta, X, Od);
        double res = 0;
        for (long i = 0; i < n; ++i) {
            cplx e = v[i] - Od[i];
            res += creal(e) * creal(e) + cimag(e) * cimag(e);
        }
        true_res = sqrt(res / vv);
        if (true_res <= tol) { status = 0; break; }
        if (iters >= maxit) { status = 1; break; }
    }
    *iters_out = iters;
    *true_res_out = true_res;
    free(r); free(d); free(Od);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Fermion force, Supplement SI                                             */
/* ------------------------------------------------------------------------ */

/* dS[b] = d/dtheta_b [ eta^dagger (M^dagger M)^{-1} eta ] given
 * X = (M^dagger M)^{-1} eta.  With Y = M X this is -2 Re[Y^dagger (dM/dtheta) X].
 * The block of M that depends on theta_tau is -B_tau at (tau+1, tau) for
 * tau < Ntau-1 and +B_{Ntau-1} at (0, Ntau-1), so
 *   dS = +2 Re[Y_{tau+1}^dagger dB_tau X_tau]   (tau < Ntau-1)
 *   dS = -2 Re[Y_0^dagger dB_{Ntau-1} X_{Ntau-1}] (tau = Ntau-1),
 * and dB_tau follows the product rule over the factors of Eq. (eq24) that
 * contain the bond. */
void orc_fermion_dS(const orc_lattice* lat, const double* theta, const cplx* X, double* dS) {
    long V = vol(lat);
    int L = lat->L, N = lat->Ntau;
    long n = V * N;
    double a = lat->dtau * lat->t;
    cplx* Y = (cplx*)malloc(sizeof(cplx) * n);
    orc_apply_M(lat, theta, X, Y, 0);
    memset(dS, 0, sizeof(double) * 2 * n);
#pragma omp parallel
    {
        cplx* u = (cplx*)malloc(sizeof(cplx) * V);
        cplx* w = (cplx*)malloc(sizeof(cplx) * V);
#pragma omp for schedule(static)
        for (int tau = 0; tau < N; ++tau) {
            const double* th = theta + (long)tau * V * 2;
            const cplx* Wv = (tau < N - 1) ? Y + (long)(tau + 1) * V : Y;
            double sign = (tau < N - 1) ? +1.0 : -1.0;
            for (int k = 0; k < 7; ++k) {
                /* u = F_{k+1} ... F_6 X_tau (factors right of position k) */
                memcpy(u, X + (long)tau * V, sizeof(cplx) * V);
                for (int m = 6; m > k; --m)
                    apply_family(L, FACTOR_FAMILY[m], FACTOR_WEIGHT[m] * a, th, u, 0);
                /* w = F_{k-1}^dagger ... F_0^dagger W (factors left of position k) */
                memcpy(w, Wv, sizeof(cplx) * V);
                for (int m = 0; m < k; ++m)
                    apply_family(L, FACTOR_FAMILY[m], FACTOR_WEIGHT[m] * a, th, w, 1);
                int fam = FACTOR_FAMILY[k];
                double sh = sinh(FACTOR_WEIGHT[k] * a);
                for (int b = 0; b < L * L / 2; ++b) {
                    int i, j, kk;
                    family_bond(L, fam, b, &i, &j, &kk);
                    cplx e = cexp(I * th[kk]);
                    /* d/dphi of [[c, s e^{i phi}], [s e^{-i phi}, c]] */
                    cplx d01 = I * sh * e, d10 = -I * sh * conj(e);
                    cplx val = conj(w[i]) * d01 * u[j] + conj(w[j]) * d10 * u[i];
                    dS[(long)tau * V * 2 + kk] += sign * 2.0 * creal(val);
                }
            }
        }
        free(u);
        free(w);
    }
    free(Y);
}

/* ------------------------------------------------------------------------ */
/* Bosonic action (Results, Eq. (eq3) and the compact form beside it)       */
/* ------------------------------------------------------------------------ */

/* Lattice curl of the spatial plaquette with lower-left corner (x, y) in
 * slice tau, edges taken along the positive (counter-clockwise) direction. */
static double curl(int L, const double* th, int x, int y) {
    int xp = wrap(x + 1, L), yp = wrap(y + 1, L);
    return th[2 * (x + L * y) + 0] + th[2 * (xp + L * y) + 1]
         - th[2 * (x + L * yp) + 0] - th[2 * (x + L * y) + 1];
}

/* S_B = dtau * sum_tau L_B with the imaginary-time integral written as
 * dtau * sum over slices (periodic in tau for the gauge field):
 *   compact:     (1/(J dtau)) sum [1 - cos(theta_{tau+1} - theta_tau)]
 *   non-compact: (1/(J dtau)) sum (theta_{tau+1} - theta_tau)^2
 * plus K dtau sum_{tau, plaquettes} cos(curl theta). */
double orc_bosonic_action(const orc_lattice* lat, const double* theta) {
    long V = vol(lat);
    int L = lat->L, N = lat->Ntau;
    double kin = 0, pot = 0;
    for (int tau = 0; tau < N; ++tau) {
        const double* th = theta + (long)tau * V * 2;
        const double* thn = theta + (long)((tau + 1) % N) * V * 2;
        for (long b = 0; b < 2 * V; ++b) {
            double d = thn[b] - th[b];
            kin += lat->noncompact ? d * d : 1.0 - cos(d);
        }
        if (lat->K != 0.0)
            for (int y = 0; y < L; ++y)
                for (int x = 0; x < L; ++x) pot += cos(curl(L, th, x, y));
    }
    return kin / (lat->J * lat->dtau) + lat->K * lat->dtau * pot;
}

/* dS[b] = d S_B / d theta_b. */
void orc_bosonic_dS(const orc_lattice* lat, const double* theta, double* dS) {
    long V = vol(lat);
    int L = lat->L, N = lat->Ntau;
    double cB = 1.0 / (lat->J * lat->dtau);
    memset(dS, 0, sizeof(double) * 2 * V * N);
    for (int tau = 0; tau < N; ++tau) {
        const double* th = theta + (long)tau * V * 2;
        const double* thn = theta + (long)((tau + 1) % N) * V * 2;
        double* g = dS + (long)tau * V * 2;
        double* gn = dS + (long)((tau + 1) % N) * V * 2;
        /* term f(theta_{tau+1} - theta_tau) with f = 1 - cos or f = d^2 */
        for (long b = 0; b < 2 * V; ++b) {
            double d = thn[b] - th[b];
            double fp = lat->noncompact ? 2.0 * d : sin(d);
            gn[b] += cB * fp;
            g[b] -= cB * fp;
        }
        if (lat->K != 0.0) {
            for (int y = 0; y < L; ++y)
                for (int x = 0; x < L; ++x) {
                    double dc = -lat->K * lat->dtau * sin(curl(L, th, x, y));
                    int xp = wrap(x + 1, L), yp = wrap(y + 1, L);
                    g[2 * (x + L * y) + 0] += dc;
                    g[2 * (xp + L * y) + 1] += dc;
                    g[2 * (x + L * yp) + 0] -= dc;
                    g[2 * (x + L * y) + 1] -= dc;
                }
        }
    }
}

/* eta^dagger X (real part; the imaginary part vanishes for Hermitian O). */
double orc_fermion_action(const orc_lattice* lat, const cplx* eta, const cplx* X) {
    double re, im;
    orc_dot(vol(lat) * lat->Ntau, eta, X, &re, &im);
    return re;
}

/* ------------------------------------------------------------------------ */
/* Hamiltonian dynamics, Eqs. (H_diff) and (leapfrog)                       */
/* ------------------------------------------------------------------------ */

/* F = -dS_B/dtheta - dS_f/dtheta at theta, with X solved from guess X. */
static int total_force(const orc_lattice* lat, const double* theta, const cplx* eta,
                       cplx* X, double* F, double* scratch, double tol, int maxit,
                       int* iters) {
    long nb = 2 * vol(lat) * lat->Ntau;
    int it = 0;
    double res = 0;
    int st = orc_cg(lat, theta, eta, X, tol, maxit, &it, &res);
    *iters += it;
    orc_fermion_dS(lat, theta, X, F);
    orc_bosonic_dS(lat, theta, scratch);
    for (long b = 0; b < nb; ++b) F[b] = -F[b] - scratch[b];
    return st;
}

/* nsteps leapfrog steps of size dt on (theta, p).  X holds the CG guess for
 * the first solve on entry and (M^dagger M)^{-1} eta at the final theta on
 * exit; every solve starts from the previous solution.  Returns the number
 * of CG solves that did not converge. */
int orc_leapfrog(const orc_lattice* lat, double* theta, double* p, const cplx* eta, cplx* X,
                 int nsteps, double dt, double tol, int maxit, int* cg_iters) {
    long nb = 2 * vol(lat) * lat->Ntau;
    double* F = (double*)malloc(sizeof(double) * nb);
    double* scratch = (double*)malloc(sizeof(double) * nb);
    int bad = 0;
    *cg_iters = 0;
    bad += total_force(lat, theta, eta, X, F, scratch, tol, maxit, cg_iters);
    for (int n = 0; n < nsteps; ++n) {
        for (long b = 0; b < nb; ++b) p[b] += F[b] * dt / 2;
        for (long b = 0; b < nb; ++b) theta[b] += 2.0 * p[b] * dt;
        bad += total_force(lat, theta, eta, X, F, scratch, tol, maxit, cg_iters);
        for (long b = 0; b < nb; ++b) p[b] += F[b] * dt / 2;
    }
    free(F);
    free(scratch);
    return bad;
}

/* One HQMC update (Methods, steps (i)-(iv)) with the Gaussian draws supplied:
 * p0 ~ N(0, 1/2) per bond and R ~ CN(0, 1) per site.  eta = M^dagger R;
 * H0 = S_B + sum p^2 + R^dagger R (= eta^dagger (M^dagger M)^{-1} eta exactly);
 * H1 = S_B + sum p^2 + eta^dagger X at the end point.  Accepts iff
 * u < exp(H0 - H1); on rejection theta is restored.  Returns the number of
 * unconverged CG solves. */
int orc_trajectory(const orc_lattice* lat, double* theta, const double* p0, const cplx* R,
                   double u, int nsteps, double dt, double tol, int maxit,
                   double* H0_out, double* H1_out, int* accepted, int* cg_iters) {
    long n = vol(lat) * lat->Ntau, nb = 2 * n;
    cplx* eta = (cplx*)malloc(sizeof(cplx) * n);
    cplx* X = (cplx*)calloc(n, sizeof(cplx));
    double* p = (double*)malloc(sizeof(double) * nb);
    double* th0 = (double*)malloc(sizeof(double) * nb);
    memcpy(p, p0, sizeof(double) * nb);
    memcpy(th0, theta, sizeof(double) * nb);
    orc_apply_M(lat, theta, R, eta, 1);
    double pp = 0;
    for (long b = 0; b < nb; ++b) pp += p[b] * p[b];
    double H0 = orc_bosonic_action(lat, theta) + pp + norm2(n, R);
    int bad = orc_leapfrog(lat, theta, p, eta, X, nsteps, dt, tol, maxit, cg_iters);
    pp = 0;
    for (long b = 0; b < nb; ++b) pp += p[b] * p[b];
    double H1 = orc_bosonic_action(lat, theta) + pp + orc_fermion_action(lat, eta, X);
    *accepted = (u < exp(H0 - H1)) ? 1 : 0;
    if (!*accepted) memcpy(theta, th0, sizeof(double) * nb);
    *H0_out = H0;
    *H1_out = H1;
    free(eta); free(X); free(p); free(th0);
    return bad;
}

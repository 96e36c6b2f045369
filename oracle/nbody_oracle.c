/*
 * nbody_oracle.c -- plain, slow, FP64 CPU oracle for the direct-sum Hermite
 * block-timestep N-body method (Groen, Portegies Zwart, McMillan & Makino,
 * "Distributed N-body Simulation on the Grid Using Dedicated Hardware").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA library is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the product path never
 * does.  It shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (all in IEEE FP64, G = 1, N-body units):
 *   - orc_forces:      Sec. 4.1 step 4 / Eq. 3 (t_force = tau_force n N):
 *                      for every active i, the Plummer-softened acceleration,
 *                      its time derivative (jerk) and the potential, summed
 *                      over all j != i in ascending j order.  The softening
 *                      length is the "softening parameter" of Sec. 2.
 *   - orc_predict:     Sec. 4.1 step 3: Taylor prediction of x, v of all N.
 *   - orc_correct:     Sec. 4.1 step 5: 4th-order Hermite corrector (the
 *                      scheme Sec. 2 cites, Makino & Aarseth 1992; the paper
 *                      does not print its formulas).
 *   - orc_aarseth_dt / orc_block_dt / orc_initial_dt:
 *                      Sec. 2: block time-steps in powers of two between
 *                      2^-22 and 2^-3; the step criterion itself is not
 *                      printed in the paper (standard Aarseth form used).
 *   - orc_hermite_run: Sec. 4.1 steps 2-6, the whole block-step loop.
 *   - orc_energy:      kinetic + softened potential energy (the paper is
 *                      silent; used for drift checks).
 *
 * Parity pins (tests/test_oracle_*.py): brute-force symbolic differentiation
 * of the potential for N<=6, Newton's third law, finite-difference jerk,
 * polynomial exactness of the corrector, circular-orbit time step, Kepler
 * two-body closed form, 4th-order convergence, Plummer virial ratio and energy
 * drift.
 *
 * Vectors are row-major [n][3].  No -ffast-math: every operation is IEEE FP64
 * (compiled with -ffp-contract=off so no FMA is formed behind our back).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Summation: plain left-to-right, or Neumaier-compensated (Neumaier 1974).  */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } orc_acc;

static inline void acc_add(orc_acc* a, double x, int compensated) {
    if (!compensated) { a->s += x; return; }
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else                       a->c += (x - t) + a->s;
    a->s = t;
}
static inline double acc_val(const orc_acc* a) { return a->s + a->c; }

static int set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) return nthreads;
    return omp_get_max_threads();
#else
    (void)nthreads; return 1;
#endif
}

int orc_max_threads(void) { return set_threads(0); }

/*
 * Direct-sum force on one i-particle at position xi, velocity vi, index self.
 * For every j != self (ascending j):
 *   r   = x_j - x_i,  w = v_j - v_i,  s^2 = r.r + eps^2
 *   acc  += m_j r / s^3
 *   jerk += m_j ( w / s^3 - 3 (r.w) r / s^5 )
 *   pot  -= m_j / s
 * Sec. 4.1 step 4 (forces and their time derivatives between the active
 * particle and all N particles), softening of Sec. 2 taken as Plummer form.
 */
static void force_one(int64_t N, const double* m, const double* x, const double* v,
                      double eps2, int64_t self, const double xi[3], const double vi[3],
                      int compensated, double acc[3], double jerk[3], double* pot)
{
    orc_acc A[3] = {{0, 0}, {0, 0}, {0, 0}}, J[3] = {{0, 0}, {0, 0}, {0, 0}}, P = {0, 0};
    for (int64_t j = 0; j < N; ++j) {
        if (j == self) continue;
        const double r0 = x[3 * j + 0] - xi[0];
        const double r1 = x[3 * j + 1] - xi[1];
        const double r2 = x[3 * j + 2] - xi[2];
        const double w0 = v[3 * j + 0] - vi[0];
        const double w1 = v[3 * j + 1] - vi[1];
        const double w2 = v[3 * j + 2] - vi[2];
        const double s2 = r0 * r0 + r1 * r1 + r2 * r2 + eps2;
        const double s = sqrt(s2);
        const double inv_s = 1.0 / s;
        const double inv_s3 = inv_s / s2;             /* 1/s^3 */
        const double rw = r0 * w0 + r1 * w1 + r2 * w2;
        const double mj = m[j];
        const double c_acc = mj * inv_s3;
        const double c_jrk = 3.0 * rw / s2;           /* 3 (r.w) / s^2 */
        acc_add(&A[0], c_acc * r0, compensated);
        acc_add(&A[1], c_acc * r1, compensated);
        acc_add(&A[2], c_acc * r2, compensated);
        acc_add(&J[0], c_acc * (w0 - c_jrk * r0), compensated);
        acc_add(&J[1], c_acc * (w1 - c_jrk * r1), compensated);
        acc_add(&J[2], c_acc * (w2 - c_jrk * r2), compensated);
        acc_add(&P, -mj * inv_s, compensated);
    }
    for (int k = 0; k < 3; ++k) { acc[k] = acc_val(&A[k]); jerk[k] = acc_val(&J[k]); }
    *pot = acc_val(&P);
}

/*
 * Forces on the n active particles idx[0..n) (all N if idx == NULL), from all
 * N particles at positions x and velocities v (both taken as already predicted
 * to the common time).  Outputs acc[n][3], jerk[n][3], pot[n].
 */
void orc_forces(int64_t N, const double* m, const double* x, const double* v, double eps,
                int64_t n, const int64_t* idx, double* acc, double* jerk, double* pot,
                int compensated, int nthreads)
{
    const double eps2 = eps * eps;
    const int nt = set_threads(nthreads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t k = 0; k < n; ++k) {
        const int64_t i = idx ? idx[k] : k;
        force_one(N, m, x, v, eps2, i, &x[3 * i], &v[3 * i], compensated,
                  &acc[3 * k], &jerk[3 * k], &pot[k]);
    }
}

/*
 * Predictor, Sec. 4.1 step 3: for every particle, with h = t - t_i,
 *   xp = x + v h + a h^2/2 + j h^3/6,   vp = v + a h + j h^2/2.
 */
void orc_predict(int64_t N, const double* x, const double* v, const double* a, const double* jk,
                 const double* t_i, double t, double* xp, double* vp)
{
    for (int64_t i = 0; i < N; ++i) {
        const double h = t - t_i[i];
        for (int k = 0; k < 3; ++k) {
            const int64_t q = 3 * i + k;
            xp[q] = x[q] + v[q] * h + a[q] * (h * h / 2.0) + jk[q] * (h * h * h / 6.0);
            vp[q] = v[q] + a[q] * h + jk[q] * (h * h / 2.0);
        }
    }
}

/*
 * Hermite corrector, Sec. 4.1 step 5 (scheme of Makino & Aarseth 1992, cited
 * in Sec. 2).  The acceleration over the step is the cubic Hermite
 * interpolant through (a0, j0) at the start and (a1, j1) at the end; its 2nd
 * and 3rd derivatives at the start are
 *   a2 = [-6 (a0 - a1) - h (4 j0 + 2 j1)] / h^2
 *   a3 = [12 (a0 - a1) + 6 h (j0 + j1)] / h^3
 * and the predicted orbit is corrected by the two missing Taylor terms
 *   x1 = xp + a2 h^4/24 + a3 h^5/120,   v1 = vp + a2 h^3/6 + a3 h^4/24.
 * Also returns the 2nd derivative at the END of the step, a2 + a3 h, and a3,
 * which feed the time-step criterion.
 */
void orc_correct(int64_t n, const double* x0, const double* v0, const double* a0, const double* j0,
                 const double* xp, const double* vp, const double* a1, const double* j1,
                 const double* h_arr, double* x1, double* v1, double* a2_end, double* a3_out)
{
    (void)x0; (void)v0;
    for (int64_t i = 0; i < n; ++i) {
        const double h = h_arr[i];
        const double h2 = h * h, h3 = h2 * h, h4 = h3 * h, h5 = h4 * h;
        for (int k = 0; k < 3; ++k) {
            const int64_t q = 3 * i + k;
            const double da = a0[q] - a1[q];
            const double a2 = (-6.0 * da - h * (4.0 * j0[q] + 2.0 * j1[q])) / h2;
            const double a3 = (12.0 * da + 6.0 * h * (j0[q] + j1[q])) / h3;
            x1[q] = xp[q] + a2 * h4 / 24.0 + a3 * h5 / 120.0;
            v1[q] = vp[q] + a2 * h3 / 6.0 + a3 * h4 / 24.0;
            if (a2_end) a2_end[q] = a2 + a3 * h;
            if (a3_out) a3_out[q] = a3;
        }
    }
}

static double norm3(const double* u) { return sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]); }

/*
 * Aarseth time-step criterion (standard form; the paper only fixes the power-
 * of-two block and its bounds, Sec. 2):
 *   dt = sqrt( eta (|a||a2| + |j|^2) / (|j||a3| + |a2|^2) ).
 */
double orc_aarseth_dt(const double* a, const double* j, const double* a2, const double* a3, double eta)
{
    const double na = norm3(a), nj = norm3(j), n2 = norm3(a2), n3 = norm3(a3);
    const double num = na * n2 + nj * nj;
    const double den = nj * n3 + n2 * n2;
    if (den == 0.0) return INFINITY;
    return sqrt(eta * num / den);
}

/* largest power of two <= x, for x > 0 (by repeated halving/doubling). */
static double pow2_floor(double x)
{
    if (!(x > 0.0)) return 0.0;
    if (isinf(x)) return INFINITY;
    double p = 1.0;
    while (p > x) p *= 0.5;
    while (p * 2.0 <= x) p *= 2.0;
    return p;
}

double orc_pow2_floor(double x) { return pow2_floor(x); }

/*
 * Block rule (Sec. 2: powers of two between dt_min and dt_max):
 *   c = largest power of two <= dt_crit, clamped to [dt_min, dt_max];
 *   shrink freely (c < dt_old -> c);  grow only by a factor 2 and only when t
 *   is a multiple of 2 dt_old (keeps t_i a multiple of dt_i); else keep.
 * Sets *underflow = 1 when dt_crit < dt_min.
 */
double orc_block_dt(double dt_crit, double dt_old, double t, double dt_min, double dt_max, int* underflow)
{
    if (underflow) *underflow = (dt_crit < dt_min) ? 1 : 0;
    double c = pow2_floor(dt_crit);
    if (c > dt_max) c = dt_max;
    if (c < dt_min) c = dt_min;
    if (c < dt_old) return c;
    if (c >= 2.0 * dt_old && 2.0 * dt_old <= dt_max && fmod(t, 2.0 * dt_old) == 0.0) return 2.0 * dt_old;
    return dt_old;
}

/* initial step: largest power of two <= eta |a|/|j|, clamped to [dt_min, dt_max]. */
double orc_initial_dt(const double* a, const double* j, double eta, double dt_min, double dt_max)
{
    const double na = norm3(a), nj = norm3(j);
    double d = (nj > 0.0) ? eta * na / nj : INFINITY;
    double c = pow2_floor(d);
    if (c > dt_max) c = dt_max;
    if (c < dt_min) c = dt_min;
    return c;
}

/*
 * Kinetic and potential energy: K = sum m v^2 / 2, W = (1/2) sum_i m_i phi_i,
 * with phi_i the softened potential of orc_forces (j != i).  Compensated sums.
 */
void orc_energy(int64_t N, const double* m, const double* x, const double* v, double eps,
                int nthreads, double* ekin, double* epot)
{
    double* acc = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* jrk = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* pot = (double*)malloc(sizeof(double) * (size_t)N);
    orc_forces(N, m, x, v, eps, N, NULL, acc, jrk, pot, 1, nthreads);
    orc_acc K = {0, 0}, W = {0, 0};
    for (int64_t i = 0; i < N; ++i) {
        const double v2 = v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2];
        acc_add(&K, 0.5 * m[i] * v2, 1);
        acc_add(&W, 0.5 * m[i] * pot[i], 1);
    }
    *ekin = acc_val(&K);
    *epot = acc_val(&W);
    free(acc); free(jrk); free(pot);
}

typedef struct {
    int64_t block_steps;      /* number of block steps taken          */
    int64_t particle_steps;   /* sum over block steps of n_active     */
    double  interactions;     /* sum over block steps of n_active * N */
    int64_t dt_underflows;    /* criterion below dt_min (clamped)     */
} orc_stats;

/*
 * The whole single-node loop of Sec. 4.1:
 *   (1) initialise (if `initialize`): forces of all N at t = 0 and initial
 *       steps; t_i = 0;
 *   (2) t = min_i (t_i + dt_i); active block = { i : t_i + dt_i == t },
 *       ascending index;
 *   (3) predict all N to t;
 *   (4) forces on the active block from all N predicted particles;
 *   (5) correct the active block, store new a, j, pot, t_i = t, new dt_i;
 *   (6) repeat until the next block time would exceed t_end.
 * t_end must be a multiple of dt_max so that every particle lands on it.
 * Arrays (row-major [N][3] for vectors) are updated in place.  Returns the
 * number of block steps, or -1 on bad arguments.
 */
int64_t orc_hermite_run(int64_t N, const double* m, double* x, double* v, double* a, double* jk,
                        double* pot, double* t_i, double* dt, double eps, double eta,
                        double dt_min, double dt_max, double t_end, int initialize,
                        int compensated, int nthreads, int64_t max_block_steps, orc_stats* st)
{
    if (N <= 0 || !(dt_min > 0) || !(dt_max >= dt_min) || !(eps >= 0)) return -1;
    if (fmod(t_end, dt_max) != 0.0) return -1;
    orc_stats s = {0, 0, 0.0, 0};
    const size_t n3 = 3 * (size_t)N;
    double* xp = (double*)malloc(sizeof(double) * n3);
    double* vp = (double*)malloc(sizeof(double) * n3);
    double* a1 = (double*)malloc(sizeof(double) * n3);
    double* j1 = (double*)malloc(sizeof(double) * n3);
    double* p1 = (double*)malloc(sizeof(double) * (size_t)N);
    int64_t* act = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    double* bx0 = (double*)malloc(sizeof(double) * n3);   /* per-block gathers */
    double* bv0 = (double*)malloc(sizeof(double) * n3);
    double* ba0 = (double*)malloc(sizeof(double) * n3);
    double* bj0 = (double*)malloc(sizeof(double) * n3);
    double* bxp = (double*)malloc(sizeof(double) * n3);
    double* bvp = (double*)malloc(sizeof(double) * n3);
    double* bx1 = (double*)malloc(sizeof(double) * n3);
    double* bv1 = (double*)malloc(sizeof(double) * n3);
    double* ba2 = (double*)malloc(sizeof(double) * n3);
    double* ba3 = (double*)malloc(sizeof(double) * n3);
    double* bh  = (double*)malloc(sizeof(double) * (size_t)N);

    if (initialize) {
        orc_forces(N, m, x, v, eps, N, NULL, a, jk, pot, compensated, nthreads);
        for (int64_t i = 0; i < N; ++i) {
            t_i[i] = 0.0;
            dt[i] = orc_initial_dt(&a[3 * i], &jk[3 * i], eta, dt_min, dt_max);
        }
    }

    while (max_block_steps < 0 || s.block_steps < max_block_steps) {
        /* (2) next system time and active block */
        double t = INFINITY;
        for (int64_t i = 0; i < N; ++i) { const double ti = t_i[i] + dt[i]; if (ti < t) t = ti; }
        if (t > t_end) break;
        int64_t n = 0;
        for (int64_t i = 0; i < N; ++i) if (t_i[i] + dt[i] == t) act[n++] = i;
        /* (3) predict all N */
        orc_predict(N, x, v, a, jk, t_i, t, xp, vp);
        /* (4) forces on the active block at predicted positions */
        orc_forces(N, m, xp, vp, eps, n, act, a1, j1, p1, compensated, nthreads);
        /* (5) correct the active block */
        for (int64_t k = 0; k < n; ++k) {
            const int64_t i = act[k];
            memcpy(&bx0[3 * k], &x[3 * i], 3 * sizeof(double));
            memcpy(&bv0[3 * k], &v[3 * i], 3 * sizeof(double));
            memcpy(&ba0[3 * k], &a[3 * i], 3 * sizeof(double));
            memcpy(&bj0[3 * k], &jk[3 * i], 3 * sizeof(double));
            memcpy(&bxp[3 * k], &xp[3 * i], 3 * sizeof(double));
            memcpy(&bvp[3 * k], &vp[3 * i], 3 * sizeof(double));
            bh[k] = t - t_i[i];
        }
        orc_correct(n, bx0, bv0, ba0, bj0, bxp, bvp, a1, j1, bh, bx1, bv1, ba2, ba3);
        for (int64_t k = 0; k < n; ++k) {
            const int64_t i = act[k];
            memcpy(&x[3 * i], &bx1[3 * k], 3 * sizeof(double));
            memcpy(&v[3 * i], &bv1[3 * k], 3 * sizeof(double));
            memcpy(&a[3 * i], &a1[3 * k], 3 * sizeof(double));
            memcpy(&jk[3 * i], &j1[3 * k], 3 * sizeof(double));
            pot[i] = p1[k];
            const double crit = orc_aarseth_dt(&a1[3 * k], &j1[3 * k], &ba2[3 * k], &ba3[3 * k], eta);
            int uf = 0;
            dt[i] = orc_block_dt(crit, dt[i], t, dt_min, dt_max, &uf);
            s.dt_underflows += uf;
            t_i[i] = t;
        }
        s.block_steps += 1;
        s.particle_steps += n;
        s.interactions += (double)n * (double)N;
    }
    free(xp); free(vp); free(a1); free(j1); free(p1); free(act);
    free(bx0); free(bv0); free(ba0); free(bj0); free(bxp); free(bvp);
    free(bx1); free(bv1); free(ba2); free(ba3); free(bh);
    if (st) *st = s;
    return s.block_steps;
}

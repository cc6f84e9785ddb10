/*
 * FP64 CPU oracle for N coupled spin-torque oscillators (arXiv 2312.01121).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test suite, the package's smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, constant or helper with the CUDA library.
 *
 * What it computes, in the paper's order and notation:
 *   Sec. 3.1, Eq. (gov): for every oscillator k
 *       dm_k/dt = -gamma/(1+alpha^2) m_k x b_k
 *                 - alpha gamma/(1+alpha^2) m_k x (m_k x b_k)
 *   with b_k = H_total_k + H_s(m_k) p x m_k,
 *        H_s(m_k) = hbar eta I / (2 e (1 + lambda m_k.p) M V),
 *        H_total_k = H(m_k) + H_cp_k + H_in_k,
 *        H(m_k)    = [H_appl + (H_K - 4 pi M) m_k^z] e_z,
 *        H_cp_k    = A_cp sum_i w_cp[k,i] m_i^x e_x      (Eq. coup, read with
 *                    the source index i, see below),
 *        H_in_k    = A_in sum_i w_in[k,i] u_i e_x         (Eq. in).
 *   Sec. 3.2: classic fourth-order Runge-Kutta with a fixed step dt.
 *
 * Readings where the paper is silent or garbled (each is listed with its
 * justification in the design notes of the repository):
 *   - Eq. (coup) prints m_k^x inside the sum over i.  Sec. 3.3 states that the
 *     coupling is the matrix product W^cp x with x in R^N and Sec. 3.1 that the
 *     field costs O(N^2), so the summand is read as w_cp[k,i] m_i^x.
 *   - Units of H_s: hbar, e in SI, I in A, M in emu/cm^3, V in cm^3; the
 *     J -> erg factor 1e7 turns hbar I /(e M V) into Oe.  At the Table values
 *     this gives H_s0 = 134.87 Oe, the only reading under which a single
 *     oscillator at I = 2.5 mA oscillates, as Sec. 3.1 says the parameters are
 *     chosen to make it do.
 *   - The input u is a discrete series (Sec. 3.1); sample t is held constant
 *     over `substeps` RK4 steps (zero-order hold) and the reservoir state is
 *     sampled after the last of them.  An optional gain g multiplies A_in.
 *   - No renormalisation of |m| is ever applied: |m_k| - 1 is the error
 *     measure the paper uses (Sec. 3.2, Sec. 3.3).
 *
 * Layout: a state is three arrays of N doubles (m^x, m^y, m^z), W is N x N
 * row-major with row k = target oscillator and column i = source, w_in is
 * N x n_in row-major, u is T x n_in row-major, states is T x N row-major.
 *
 * Parity pins (which closed forms and invariants check each function) live
 * in the test suite; nothing here is checked against the CUDA path.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Parameters, defaults = Table "Summary of parameters" (Sec. 3.1). */
typedef struct orc_params {
  double gamma;      /* gyromagnetic ratio, rad/(Oe s) */
  double alpha;      /* Gilbert damping */
  double M;          /* saturation magnetisation, emu/cm^3 */
  double H_K;        /* anisotropy field, Oe */
  double H_appl;     /* applied field, Oe */
  double eta;        /* spin polarisation */
  double lambda;     /* spin-transfer torque asymmetry */
  double I;          /* current, A */
  double V;          /* free-layer volume, cm^3 */
  double e;          /* elementary charge, C */
  double hbar;       /* reduced Planck constant, J s */
  double p[3];       /* pinned-layer direction */
  double A_cp;       /* coupling amplitude, Oe */
  double A_in;       /* input amplitude, Oe */
  double g;          /* input gain (1 = the plain method) */
  double dt;         /* RK4 step, s */
  int substeps;      /* RK4 steps per input sample */
  int n_in;          /* number of input channels */
  int component;     /* sampled component: 0 = x, 1 = y, 2 = z */
  int pad;
} orc_params;

/* Derived constants of Eq. (gov): gamma' = gamma/(1+alpha^2),
 * H_K' = H_K - 4 pi M and H_s0 = hbar eta I 1e7 / (2 e M V), the spin-torque
 * strength before the (1 + lambda m.p) factor.  out = {gamma', H_K', H_s0}. */
void orc_derived(const orc_params* P, double out[3]) {
  out[0] = P->gamma / (1.0 + P->alpha * P->alpha);
  out[1] = P->H_K - 4.0 * M_PI * P->M;
  out[2] = P->hbar * P->eta * P->I * 1.0e7 / (2.0 * P->e * P->M * P->V);
}

/* Coupling field magnitude h_k = A_cp sum_i W[k,i] x_i (Eq. coup), summed
 * sequentially over ascending i, rows split over `nthreads` threads. */
void orc_coupling(int N, const orc_params* P, const double* W, const double* x,
                  double* h, int nthreads) {
  long long n = N;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(static)
#endif
  for (long long k = 0; k < n; ++k) {
    double s = 0.0;
    const double* row = W + k * n;
    for (long long i = 0; i < n; ++i) s += row[i] * x[i];
    h[k] = P->A_cp * s;
  }
  (void)nthreads;
}

/* Right-hand side of Eq. (gov) for one oscillator, given its magnetisation m,
 * the x-directed field from coupling plus input (hx = h_cp + h_in) and the
 * derived constants.  Writes dm/dt to f. */
static void orc_node_rhs(const orc_params* P, const double d[3], const double m[3],
                         double hx, double f[3]) {
  const double gp = d[0], HKp = d[1], Hs0 = d[2];
  const double* p = P->p;
  /* H_s(m) = H_s0 / (1 + lambda m.p) */
  double mp = m[0] * p[0] + m[1] * p[1] + m[2] * p[2];
  double Hs = Hs0 / (1.0 + P->lambda * mp);
  /* p x m */
  double c[3] = {p[1] * m[2] - p[2] * m[1], p[2] * m[0] - p[0] * m[2],
                 p[0] * m[1] - p[1] * m[0]};
  /* b = H(m) + H_cp + H_in + H_s p x m */
  double b[3] = {hx + Hs * c[0], Hs * c[1], P->H_appl + HKp * m[2] + Hs * c[2]};
  /* t = m x b */
  double t[3] = {m[1] * b[2] - m[2] * b[1], m[2] * b[0] - m[0] * b[2],
                 m[0] * b[1] - m[1] * b[0]};
  /* m x t = m x (m x b) */
  double mt[3] = {m[1] * t[2] - m[2] * t[1], m[2] * t[0] - m[0] * t[2],
                  m[0] * t[1] - m[1] * t[0]};
  for (int a = 0; a < 3; ++a) f[a] = -gp * t[a] - P->alpha * gp * mt[a];
}

/* The full vector field of Eq. (gov) for all N oscillators.
 * m = {mx[N], my[N], mz[N]}; hin[k] = H_in_k (may be NULL = 0);
 * f receives dm/dt in the same layout; h (may be NULL) receives h_cp. */
void orc_field(int N, const orc_params* P, const double* W, const double* m,
               const double* hin, double* f, double* h_out, int nthreads) {
  double d[3];
  orc_derived(P, d);
  double* h = h_out ? h_out : (double*)malloc(sizeof(double) * (size_t)N);
  orc_coupling(N, P, W, m /* m^x is the first block */, h, nthreads);
  for (int k = 0; k < N; ++k) {
    double mk[3] = {m[k], m[N + k], m[2 * N + k]};
    double fk[3];
    orc_node_rhs(P, d, mk, h[k] + (hin ? hin[k] : 0.0), fk);
    f[k] = fk[0];
    f[N + k] = fk[1];
    f[2 * N + k] = fk[2];
  }
  if (!h_out) free(h);
}

/* Input field magnitude H_in_k = g A_in sum_j w_in[k,j] u_j (Eq. in). */
void orc_input_field(int N, const orc_params* P, const double* w_in,
                     const double* u_t, double* hin) {
  for (int k = 0; k < N; ++k) {
    double s = 0.0;
    for (int j = 0; j < P->n_in; ++j) s += w_in[(size_t)k * P->n_in + j] * u_t[j];
    hin[k] = P->g * P->A_in * s;
  }
}

/* One classic RK4 step of size dt (Sec. 3.2) with the input field held. */
void orc_rk4_step(int N, const orc_params* P, const double* W, const double* hin,
                  double* m, int nthreads) {
  size_t n3 = 3 * (size_t)N;
  double* k1 = (double*)malloc(sizeof(double) * n3);
  double* k2 = (double*)malloc(sizeof(double) * n3);
  double* k3 = (double*)malloc(sizeof(double) * n3);
  double* k4 = (double*)malloc(sizeof(double) * n3);
  double* y = (double*)malloc(sizeof(double) * n3);
  double* h = (double*)malloc(sizeof(double) * (size_t)N);
  const double dt = P->dt;
  orc_field(N, P, W, m, hin, k1, h, nthreads);
  for (size_t a = 0; a < n3; ++a) y[a] = m[a] + 0.5 * dt * k1[a];
  orc_field(N, P, W, y, hin, k2, h, nthreads);
  for (size_t a = 0; a < n3; ++a) y[a] = m[a] + 0.5 * dt * k2[a];
  orc_field(N, P, W, y, hin, k3, h, nthreads);
  for (size_t a = 0; a < n3; ++a) y[a] = m[a] + dt * k3[a];
  orc_field(N, P, W, y, hin, k4, h, nthreads);
  for (size_t a = 0; a < n3; ++a)
    m[a] = m[a] + dt / 6.0 * (k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a]);
  free(k1); free(k2); free(k3); free(k4); free(y); free(h);
}

/* Run T input samples: for each t, hold H_in from u[t], take `substeps` RK4
 * steps, then record states[t*N + k] = m_k^(component).  m is advanced in
 * place; states may be NULL.  Returns 0, or -1 on bad arguments. */
int orc_run(int N, const orc_params* P, const double* W, const double* w_in,
            double* m, const double* u, int T, double* states, int nthreads) {
  if (N < 1 || T < 0 || !P || !W || !m || (T > 0 && (!u || !w_in)) ||
      P->substeps < 1 || P->n_in < 1 || P->component < 0 || P->component > 2)
    return -1;
  double* hin = (double*)malloc(sizeof(double) * (size_t)N);
  for (int t = 0; t < T; ++t) {
    orc_input_field(N, P, w_in, u + (size_t)t * P->n_in, hin);
    for (int s = 0; s < P->substeps; ++s) orc_rk4_step(N, P, W, hin, m, nthreads);
    if (states)
      for (int k = 0; k < N; ++k)
        states[(size_t)t * N + k] = m[(size_t)P->component * N + k];
  }
  free(hin);
  return 0;
}

/* Default initial condition, Eq. (initial): every oscillator starts at
 * (sin phi0 cos phi0, sin phi0 sin phi0, cos phi0) with phi0 = 2 pi / 360. */
void orc_initial_state(int N, double* m) {
  const double phi0 = 2.0 * M_PI / 360.0;
  for (int k = 0; k < N; ++k) {
    m[k] = sin(phi0) * cos(phi0);
    m[N + k] = sin(phi0) * sin(phi0);
    m[2 * N + k] = cos(phi0);
  }
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Discrete adjoint of the RK4 stepper (gradients of a scalar loss that
 * depends on the sampled states).  Not part of the paper's method: it is the
 * reference for the gradient-based parameter search built on top of it
 * (Sec. 1 and Sec. 2 call the parameter exploration time-consuming).
 *
 * Given dL/dstates (T x N), computes the exact derivatives of
 *     L = sum_t sum_k dL_dstates[t,k] * states[t,k]
 * (a vector-Jacobian product of the whole run) with respect to
 *     A_cp, the current I, w_in (N x n_in) and the initial state m0 (3N).
 * RK4 step m' = m + dt/6 (k1 + 2 k2 + 2 k3 + k4), k_s = f(y_s):
 *     kb4 = dt/6 lam;           yb4 = J(y4)^T kb4
 *     kb3 = dt/3 lam + dt yb4;  yb3 = J(y3)^T kb3
 *     kb2 = dt/3 lam + dt/2 yb3; yb2 = J(y2)^T kb2
 *     kb1 = dt/6 lam + dt/2 yb2; yb1 = J(y1)^T kb1
 *     lam <- lam + yb1 + yb2 + yb3 + yb4,
 * and each J^T kb also yields the parameter terms (kb . df/dtheta at y_s).
 * J^T v for one oscillator, with b the full field at m:
 *     bbar = gamma' (m x v) - alpha gamma' m x (m x v)          (d/db)
 *     mbar = -gamma' [b x v + alpha ((m.b) v + (m.v) b - 2 (b.v) m)]
 *            + H_K' bbar_z e_z + H_s (bbar x p) - (bbar.c) lambda H_s/(1+lambda s) p
 *     coupling: xbar_i += A_cp sum_k W[k,i] bbar_x,k
 * ------------------------------------------------------------------------ */

/* J^T v for all oscillators at state y (3N) with input field hin; adds the
 * state cotangent into ybar (3N) and the parameter terms into g. */
static void orc_field_vjp(int N, const orc_params* P, const double d[3], const double* W,
                          const double* w_in, const double* u_t, const double* y,
                          const double* hin, const double* v, double* ybar, double* gA,
                          double* gI, double* gwin, int nthreads) {
  const double gp = d[0], HKp = d[1], Hs0 = d[2];
  const double dHs0_dI = P->hbar * P->eta * 1.0e7 / (2.0 * P->e * P->M * P->V);
  const double* p = P->p;
  double* hraw = (double*)malloc(sizeof(double) * (size_t)N);
  double* gbar = (double*)malloc(sizeof(double) * (size_t)N);
  orc_params Pone = *P;
  Pone.A_cp = 1.0;
  orc_coupling(N, &Pone, W, y, hraw, nthreads); /* raw W x */
  for (int k = 0; k < N; ++k) {
    double m[3] = {y[k], y[N + k], y[2 * N + k]};
    double vv[3] = {v[k], v[N + k], v[2 * N + k]};
    double s = m[0] * p[0] + m[1] * p[1] + m[2] * p[2];
    double D = 1.0 + P->lambda * s;
    double Hs = Hs0 / D;
    double c[3] = {p[1] * m[2] - p[2] * m[1], p[2] * m[0] - p[0] * m[2],
                   p[0] * m[1] - p[1] * m[0]};
    double b[3] = {P->A_cp * hraw[k] + hin[k] + Hs * c[0], Hs * c[1],
                   P->H_appl + HKp * m[2] + Hs * c[2]};
    /* bbar = gamma' (m x v) - alpha gamma' m x (m x v) */
    double mv[3] = {m[1] * vv[2] - m[2] * vv[1], m[2] * vv[0] - m[0] * vv[2],
                    m[0] * vv[1] - m[1] * vv[0]};
    double mmv[3] = {m[1] * mv[2] - m[2] * mv[1], m[2] * mv[0] - m[0] * mv[2],
                     m[0] * mv[1] - m[1] * mv[0]};
    double bb[3];
    for (int a = 0; a < 3; ++a) bb[a] = gp * mv[a] - P->alpha * gp * mmv[a];
    /* explicit m dependence at fixed b */
    double bxv[3] = {b[1] * vv[2] - b[2] * vv[1], b[2] * vv[0] - b[0] * vv[2],
                     b[0] * vv[1] - b[1] * vv[0]};
    double mb = m[0] * b[0] + m[1] * b[1] + m[2] * b[2];
    double mvd = m[0] * vv[0] + m[1] * vv[1] + m[2] * vv[2];
    double bv = b[0] * vv[0] + b[1] * vv[1] + b[2] * vv[2];
    double mbar[3];
    for (int a = 0; a < 3; ++a)
      mbar[a] = -gp * (bxv[a] + P->alpha * (mb * vv[a] + mvd * b[a] - 2.0 * bv * m[a]));
    /* through b(m): anisotropy and spin torque */
    mbar[2] += HKp * bb[2];
    double bbxp[3] = {bb[1] * p[2] - bb[2] * p[1], bb[2] * p[0] - bb[0] * p[2],
                      bb[0] * p[1] - bb[1] * p[0]};
    double bc = bb[0] * c[0] + bb[1] * c[1] + bb[2] * c[2];
    for (int a = 0; a < 3; ++a) mbar[a] += Hs * bbxp[a] - bc * P->lambda * Hs / D * p[a];
    ybar[k] += mbar[0];
    ybar[N + k] += mbar[1];
    ybar[2 * N + k] += mbar[2];
    gbar[k] = bb[0];
    /* parameters */
    *gA += bb[0] * hraw[k];
    *gI += bc * dHs0_dI / D;
    for (int j = 0; j < P->n_in; ++j)
      gwin[(size_t)k * P->n_in + j] += bb[0] * P->g * P->A_in * u_t[j];
  }
  /* coupling: xbar_i += A_cp sum_k W[k,i] gbar_k (column sums, ascending k) */
  for (int i = 0; i < N; ++i) {
    double sacc = 0.0;
    for (int k = 0; k < N; ++k) sacc += W[(size_t)k * N + i] * gbar[k];
    ybar[i] += P->A_cp * sacc;
  }
  free(hraw);
  free(gbar);
}

/* grads layout: [0] dL/dA_cp, [1] dL/dI, [2 .. 2 + N n_in) dL/dw_in,
 * then 3N entries dL/dm0.  Returns 0, or -1 on bad arguments. */
int orc_adjoint(int N, const orc_params* P, const double* W, const double* w_in,
                const double* m0, const double* u, int T, const double* dL_dstates,
                double* grads, int nthreads) {
  if (N < 1 || T < 1 || !P || !W || !w_in || !m0 || !u || !dL_dstates || !grads ||
      P->substeps < 1 || P->n_in < 1 || P->component < 0 || P->component > 2)
    return -1;
  const int S = P->substeps;
  const size_t n3 = 3 * (size_t)N;
  const long long steps = (long long)T * S;
  double d[3];
  orc_derived(P, d);
  /* forward, keeping the state before every RK4 step */
  double* traj = (double*)malloc(sizeof(double) * n3 * (size_t)(steps + 1));
  double* hin = (double*)malloc(sizeof(double) * (size_t)N);
  memcpy(traj, m0, sizeof(double) * n3);
  for (int t = 0; t < T; ++t) {
    orc_input_field(N, P, w_in, u + (size_t)t * P->n_in, hin);
    for (int s = 0; s < S; ++s) {
      long long n = (long long)t * S + s;
      memcpy(traj + n3 * (size_t)(n + 1), traj + n3 * (size_t)n, sizeof(double) * n3);
      orc_rk4_step(N, P, W, hin, traj + n3 * (size_t)(n + 1), nthreads);
    }
  }
  /* reverse sweep */
  const size_t nwin = (size_t)N * P->n_in;
  double gA = 0.0, gI = 0.0;
  double* gwin = (double*)calloc(nwin, sizeof(double));
  double* lam = (double*)calloc(n3, sizeof(double));
  double* y = (double*)malloc(sizeof(double) * n3);
  double* k1 = (double*)malloc(sizeof(double) * n3);
  double* k2 = (double*)malloc(sizeof(double) * n3);
  double* k3 = (double*)malloc(sizeof(double) * n3);
  double* y2 = (double*)malloc(sizeof(double) * n3);
  double* y3 = (double*)malloc(sizeof(double) * n3);
  double* y4 = (double*)malloc(sizeof(double) * n3);
  double* kb = (double*)malloc(sizeof(double) * n3);
  double* yb[4];
  for (int q = 0; q < 4; ++q) yb[q] = (double*)malloc(sizeof(double) * n3);
  const double dt = P->dt;
  for (long long n = steps - 1; n >= 0; --n) {
    const int t = (int)(n / S);
    if (n % S == S - 1)  /* the state after this step is sample t */
      for (int k = 0; k < N; ++k)
        lam[(size_t)P->component * N + k] += dL_dstates[(size_t)t * N + k];
    const double* u_t = u + (size_t)t * P->n_in;
    orc_input_field(N, P, w_in, u_t, hin);
    const double* m = traj + n3 * (size_t)n;
    /* stage points */
    orc_field(N, P, W, m, hin, k1, NULL, nthreads);
    for (size_t a = 0; a < n3; ++a) y2[a] = m[a] + 0.5 * dt * k1[a];
    orc_field(N, P, W, y2, hin, k2, NULL, nthreads);
    for (size_t a = 0; a < n3; ++a) y3[a] = m[a] + 0.5 * dt * k2[a];
    orc_field(N, P, W, y3, hin, k3, NULL, nthreads);
    for (size_t a = 0; a < n3; ++a) y4[a] = m[a] + dt * k3[a];
    /* stage 4 */
    for (size_t a = 0; a < n3; ++a) { kb[a] = dt / 6.0 * lam[a]; yb[3][a] = 0.0; }
    orc_field_vjp(N, P, d, W, w_in, u_t, y4, hin, kb, yb[3], &gA, &gI, gwin, nthreads);
    /* stage 3 */
    for (size_t a = 0; a < n3; ++a) { kb[a] = dt / 3.0 * lam[a] + dt * yb[3][a]; yb[2][a] = 0.0; }
    orc_field_vjp(N, P, d, W, w_in, u_t, y3, hin, kb, yb[2], &gA, &gI, gwin, nthreads);
    /* stage 2 */
    for (size_t a = 0; a < n3; ++a) { kb[a] = dt / 3.0 * lam[a] + 0.5 * dt * yb[2][a]; yb[1][a] = 0.0; }
    orc_field_vjp(N, P, d, W, w_in, u_t, y2, hin, kb, yb[1], &gA, &gI, gwin, nthreads);
    /* stage 1 */
    for (size_t a = 0; a < n3; ++a) { kb[a] = dt / 6.0 * lam[a] + 0.5 * dt * yb[1][a]; yb[0][a] = 0.0; }
    orc_field_vjp(N, P, d, W, w_in, u_t, m, hin, kb, yb[0], &gA, &gI, gwin, nthreads);
    for (size_t a = 0; a < n3; ++a) lam[a] += yb[0][a] + yb[1][a] + yb[2][a] + yb[3][a];
  }
  grads[0] = gA;
  grads[1] = gI;
  memcpy(grads + 2, gwin, sizeof(double) * nwin);
  memcpy(grads + 2 + nwin, lam, sizeof(double) * n3);
  free(traj); free(hin); free(gwin); free(lam); free(y); free(k1); free(k2); free(k3);
  free(y2); free(y3); free(y4); free(kb);
  for (int q = 0; q < 4; ++q) free(yb[q]);
  return 0;
}

/* ------------------------------------------------------------------------
 * General explicit Runge-Kutta stepping (the paper's closing claim: the
 * approach applies to any reservoir evolved by an explicit method).  An
 * s-stage explicit tableau (a strictly lower triangular, weights b):
 *     k_i = f(m + dt sum_{j<i} a[i][j] k_j),   m' = m + dt sum_i b[i] k_i.
 * The input field is held over the step, as for RK4.
 * ------------------------------------------------------------------------ */
void orc_erk_step(int N, const orc_params* P, const double* W, const double* hin, double* m,
                  int s, const double* a, const double* b, int nthreads) {
  size_t n3 = 3 * (size_t)N;
  double* k = (double*)malloc(sizeof(double) * n3 * (size_t)s);
  double* y = (double*)malloc(sizeof(double) * n3);
  for (int i = 0; i < s; ++i) {
    for (size_t q = 0; q < n3; ++q) {
      double acc = 0.0;
      for (int j = 0; j < i; ++j) acc += a[i * s + j] * k[(size_t)j * n3 + q];
      y[q] = m[q] + P->dt * acc;
    }
    orc_field(N, P, W, y, hin, k + (size_t)i * n3, NULL, nthreads);
  }
  for (size_t q = 0; q < n3; ++q) {
    double acc = 0.0;
    for (int i = 0; i < s; ++i) acc += b[i] * k[(size_t)i * n3 + q];
    m[q] += P->dt * acc;
  }
  free(k);
  free(y);
}

/* orc_run with an explicit tableau in place of classic RK4. */
int orc_run_erk(int N, const orc_params* P, const double* W, const double* w_in, double* m,
                const double* u, int T, double* states, int s, const double* a, const double* b,
                int nthreads) {
  if (N < 1 || T < 0 || !P || !W || !m || (T > 0 && (!u || !w_in)) || s < 1 || s > 8 ||
      !a || !b || P->substeps < 1 || P->n_in < 1 || P->component < 0 || P->component > 2)
    return -1;
  double* hin = (double*)malloc(sizeof(double) * (size_t)N);
  for (int t = 0; t < T; ++t) {
    orc_input_field(N, P, w_in, u + (size_t)t * P->n_in, hin);
    for (int q = 0; q < P->substeps; ++q) orc_erk_step(N, P, W, hin, m, s, a, b, nthreads);
    if (states)
      for (int k = 0; k < N; ++k) states[(size_t)t * N + k] = m[(size_t)P->component * N + k];
  }
  free(hin);
  return 0;
}

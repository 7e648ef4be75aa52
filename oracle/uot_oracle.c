/*
 * FP64 CPU oracle for entropic unbalanced optimal transport (UOT) and MMD
 * (Lakshmanan & Pichler, "Unbalanced Optimal Transport and Maximum Mean
 * Discrepancies: Interconnections and Rapid Evaluation", arXiv 2306.13618).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU library computes.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no code, header, table or constant with the CUDA library, and the CUDA
 * library never calls it.
 *
 * Conventions (paper notation, Sec. 3):
 *   measures mu = sum_i mu_i delta_{x_i} (n atoms), nu = sum_j nu_j delta_{y_j}
 *   (m atoms) in R^d; cost d_ij^r with r = 2, d_ij = ||x_i - y_j||;
 *   Gibbs kernel k_ij = exp(-lambda d_ij^2)  (lambda = 1/eps);
 *   marginal penalties eta1, eta2; dual potentials beta (n), gamma (m).
 * Every sum is an FP64 Neumaier-compensated sum.  No -ffast-math.
 * Arrays are row-major: point i of a cloud is p[i*d .. i*d+d-1].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------- compensated summation (Neumaier's variant of Kahan) ---------- */
typedef struct { double s, c; } nsum;
static inline void nsum_add(nsum* a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}
static inline double nsum_get(const nsum* a) { return a->s + a->c; }

static inline double sqdist(int d, const double* a, const double* b) {
  double r = 0.0;
  for (int t = 0; t < d; ++t) { double u = a[t] - b[t]; r += u * u; }
  return r;
}

/* The cost d(x, y)^r of Eq. (W4): r = 2 the squared Euclidean distance (the
 * Gaussian Gibbs kernel), r = 1 the distance itself (the Laplacian kernel
 * e^{-lambda |x - y|} of the complexity paragraph of Sec. 4.4). */
static inline double cost_r(int d, const double* a, const double* b, double r) {
  const double s = sqdist(d, a, b);
  return r == 2.0 ? s : (r == 1.0 ? sqrt(s) : pow(sqrt(s), r));
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int k) {
#ifdef _OPENMP
  if (k > 0) omp_set_num_threads(k);
#else
  (void)k;
#endif
}

/* Radial Gaussian kernel summation, Eq. (fast_sum) with K(v) = exp(-||v||^2/eps):
 *   out_j = sum_i w_i exp(-||src_i - tgt_j||^2 / eps),  j = 0..m-1.
 * This is the matrix-vector product k.w of Alg. 1 written out. */
void orc_ksum(int d, const double* src, int64_t n, const double* w,
              const double* tgt, int64_t m, double eps, double* out) {
  const double inv = 1.0 / eps;
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < m; ++j) {
    nsum acc = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i)
      nsum_add(&acc, w[i] * exp(-sqdist(d, src + i * d, tgt + j * d) * inv));
    out[j] = nsum_get(&acc);
  }
}

/* One half-step of Alg. 1, written for the beta side: for every i,
 *   beta_i = -q * log( sum_j k_ij * exp(lambda*gamma_j) * nu_j )           (ref 0)
 *   beta_i =  q * ( log mu_i - log( sum_j k_ij * exp(lambda*gamma_j) ) )   (ref 1)
 * with q = eta/(1+eta*lambda) (Eq. Sinkhorn_uot_iteration).  Ref 0 is the
 * paper's product reference measure D(pi || mu (x) nu); ref 1 is the counting
 * reference, where the scaling update reads u = (a/(K v))^{rho/(rho+eps)}.
 * logdomain != 0 evaluates the same logarithm as a row-wise log-sum-exp. */
static void half_step(int d, const double* x, int64_t n, const double* mu,
                      const double* y, int64_t m, const double* nu,
                      double lambda, double eta, int ref, int logdomain,
                      const double* gamma, double* beta, double r) {
  const double q = eta / (1.0 + eta * lambda);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double lg;
    if (!logdomain) {
      nsum acc = {0.0, 0.0};
      for (int64_t j = 0; j < m; ++j) {
        double kij = exp(-lambda * cost_r(d, x + i * d, y + j * d, r));
        double wj = exp(lambda * gamma[j]) * (ref == 0 ? nu[j] : 1.0);
        nsum_add(&acc, kij * wj);
      }
      lg = log(nsum_get(&acc));
    } else {
      double mx = -INFINITY;
      for (int64_t j = 0; j < m; ++j) {
        double a = -lambda * cost_r(d, x + i * d, y + j * d, r) + lambda * gamma[j] +
                   (ref == 0 ? log(nu[j]) : 0.0);
        if (a > mx) mx = a;
      }
      nsum acc = {0.0, 0.0};
      for (int64_t j = 0; j < m; ++j) {
        double a = -lambda * cost_r(d, x + i * d, y + j * d, r) + lambda * gamma[j] +
                   (ref == 0 ? log(nu[j]) : 0.0);
        nsum_add(&acc, exp(a - mx));
      }
      lg = mx + log(nsum_get(&acc));
    }
    beta[i] = (ref == 0) ? -q * lg : q * (log(mu[i]) - lg);
  }
}

/* Alg. 1 (Sinkhorn algorithm UOT), fixed number of sweeps.  One sweep is the
 * beta half-step (odd Delta) followed by the gamma half-step (even Delta).
 * gamma holds the starting value gamma^0 on entry (the paper sets 0) and
 * gamma^S on exit; beta receives beta^S. */
void orc_uot_sinkhorn(int d, const double* x, int64_t n, const double* mu,
                      const double* y, int64_t m, const double* nu,
                      double lambda, double eta1, double eta2, int sweeps,
                      int ref, int logdomain, double* beta, double* gamma, double r) {
  for (int s = 0; s < sweeps; ++s) {
    half_step(d, x, n, mu, y, m, nu, lambda, eta1, ref, logdomain, gamma, beta, r);
    half_step(d, y, m, nu, x, n, mu, lambda, eta2, ref, logdomain, beta, gamma, r);
  }
}

/* Dual objective D(beta, gamma) of Theorem thm:dual_EUOT, Eq. (dual_euot):
 *   - eta1 sum_i mu_i e^{-beta_i/eta1} - eta2 sum_j nu_j e^{-gamma_j/eta2}
 *   + eta1 sum_i mu_i + eta2 sum_j nu_j
 *   - (1/lambda) sum_ij mu_i (e^{lambda beta_i} k_ij e^{lambda gamma_j} - 1) nu_j.
 * For the counting reference (ref 1) the coupling term reads
 *   - (1/lambda) sum_ij e^{lambda beta_i} k_ij e^{lambda gamma_j}
 * (the reference-mass constant n*m/lambda is dropped). */
double orc_dual_value(int d, const double* x, int64_t n, const double* mu,
                      const double* y, int64_t m, const double* nu,
                      double lambda, double eta1, double eta2,
                      const double* beta, const double* gamma, int ref, double r) {
  nsum a = {0, 0}, b = {0, 0}, sm = {0, 0}, sn = {0, 0};
  for (int64_t i = 0; i < n; ++i) {
    nsum_add(&a, mu[i] * exp(-beta[i] / eta1));
    nsum_add(&sm, mu[i]);
  }
  for (int64_t j = 0; j < m; ++j) {
    nsum_add(&b, nu[j] * exp(-gamma[j] / eta2));
    nsum_add(&sn, nu[j]);
  }
  double* row = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    nsum rs = {0, 0};
    for (int64_t j = 0; j < m; ++j) {
      /* e^{lambda beta_i} k_ij e^{lambda gamma_j} as one exponential, which
         stays finite where the factors alone would overflow or underflow */
      double v = exp(lambda * (beta[i] + gamma[j]) - lambda * cost_r(d, x + i * d, y + j * d, r));
      nsum_add(&rs, ref == 0 ? mu[i] * v * nu[j] : v);
    }
    row[i] = nsum_get(&rs);
  }
  nsum c = {0, 0};
  for (int64_t i = 0; i < n; ++i) nsum_add(&c, row[i]);
  free(row);
  double coupling = nsum_get(&c);
  if (ref == 0) coupling -= nsum_get(&sm) * nsum_get(&sn);
  return -eta1 * nsum_get(&a) - eta2 * nsum_get(&b) + eta1 * nsum_get(&sm) +
         eta2 * nsum_get(&sn) - coupling / lambda;
}

/* Transport plan recovered from the duals (Sec. 3.1, below Alg. 1):
 *   pi_ij = mu_i nu_j e^{lambda beta_i} k_ij e^{lambda gamma_j}   (ref 0)
 *   pi_ij =           e^{lambda beta_i} k_ij e^{lambda gamma_j}   (ref 1). */
void orc_plan(int d, const double* x, int64_t n, const double* mu,
              const double* y, int64_t m, const double* nu, double lambda,
              const double* beta, const double* gamma, int ref, double* pi, double r) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < m; ++j) {
      double v = exp(lambda * (beta[i] + gamma[j]) -
                     lambda * cost_r(d, x + i * d, y + j * d, r));
      pi[i * m + j] = ref == 0 ? mu[i] * nu[j] * v : v;
    }
}

/* Discrete primal objective of Eq. (W4), Sec. 3.1 (product reference):
 *   sum_ij d_ij^2 pi_ij + (1/lambda) (sum pi log(pi/(mu_i nu_j)) + sum mu_i nu_j - sum pi)
 *   + eta1 (sum_i r_i log(r_i/mu_i) + sum mu - sum pi)
 *   + eta2 (sum_j c_j log(c_j/nu_j) + sum nu - sum pi),
 * r, c the row and column sums of pi.  Evaluated at the plan of the duals. */
double orc_primal_value(int d, const double* x, int64_t n, const double* mu,
                        const double* y, int64_t m, const double* nu,
                        double lambda, double eta1, double eta2,
                        const double* beta, const double* gamma, double r) {
  nsum cost = {0, 0}, ent = {0, 0}, tot = {0, 0}, sm = {0, 0}, sn = {0, 0};
  double* col = (double*)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
  nsum marg1 = {0, 0}, marg2 = {0, 0};
  for (int64_t i = 0; i < n; ++i) {
    nsum rs = {0, 0};
    for (int64_t j = 0; j < m; ++j) {
      double dij = cost_r(d, x + i * d, y + j * d, r);
      double lv = lambda * (beta[i] + gamma[j]) - lambda * dij; /* log(pi/(mu nu)) */
      double p = mu[i] * nu[j] * exp(lv);
      nsum_add(&cost, dij * p);
      nsum_add(&ent, p * lv);
      nsum_add(&ent, mu[i] * nu[j]);
      nsum_add(&ent, -p);
      nsum_add(&tot, p);
      nsum_add(&rs, p);
      col[j] += p;
    }
    double ri = nsum_get(&rs);
    if (ri > 0) nsum_add(&marg1, ri * log(ri / mu[i]));
    nsum_add(&sm, mu[i]);
  }
  for (int64_t j = 0; j < m; ++j) {
    if (col[j] > 0) nsum_add(&marg2, col[j] * log(col[j] / nu[j]));
    nsum_add(&sn, nu[j]);
  }
  free(col);
  double T = nsum_get(&tot);
  return nsum_get(&cost) + nsum_get(&ent) / lambda +
         eta1 * (nsum_get(&marg1) + nsum_get(&sm) - T) +
         eta2 * (nsum_get(&marg2) + nsum_get(&sn) - T);
}

/* MMD^2 of Eq. (1205) with the Gaussian kernel of Table tab:0,
 * k(x, x~) = exp(-||x - x~||^2 / ell^2):
 *   sum_ij mu_i mu_j k(x_i,x_j) - 2 sum_ij mu_i nu_j k(x_i,y_j) + sum_ij nu_i nu_j k(y_i,y_j).
 * parts (may be NULL) receives the three double sums A, B, C (MMD^2 = A - 2B + C). */
double orc_mmd2(int d, const double* x, int64_t n, const double* mu,
                const double* y, int64_t m, const double* nu, double ell,
                double* parts) {
  const double eps = ell * ell;
  double* kx = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* ky = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  nsum A = {0, 0}, B = {0, 0}, C = {0, 0};
  orc_ksum(d, x, n, mu, x, n, eps, kx); /* (K_xx mu)_i */
  for (int64_t i = 0; i < n; ++i) nsum_add(&A, mu[i] * kx[i]);
  orc_ksum(d, y, m, nu, x, n, eps, kx); /* (K_xy nu)_i */
  for (int64_t i = 0; i < n; ++i) nsum_add(&B, mu[i] * kx[i]);
  orc_ksum(d, y, m, nu, y, m, eps, ky); /* (K_yy nu)_j */
  for (int64_t j = 0; j < m; ++j) nsum_add(&C, nu[j] * ky[j]);
  free(kx);
  free(ky);
  if (parts) { parts[0] = nsum_get(&A); parts[1] = nsum_get(&B); parts[2] = nsum_get(&C); }
  return nsum_get(&A) - 2.0 * nsum_get(&B) + nsum_get(&C);
}

/* Unbalanced Sinkhorn divergence, Eq. (586):
 *   sd = UOT(mu,nu) - UOT(mu,mu)/2 - UOT(nu,nu)/2 + (mu(X) - nu(X))^2 / (2 lambda),
 * each UOT value taken as D(beta, gamma) at the duals after `sweeps` sweeps of
 * Alg. 1 from gamma^0 = 0 (product reference, eta1 = eta2 = eta).
 * parts (may be NULL) receives the three UOT values. */
double orc_sinkhorn_divergence(int d, const double* x, int64_t n, const double* mu,
                               const double* y, int64_t m, const double* nu,
                               double lambda, double eta, int sweeps, double* parts, double r) {
  int64_t nmax = n > m ? n : m;
  double* b = (double*)malloc(sizeof(double) * (size_t)(nmax > 0 ? nmax : 1));
  double* g = (double*)malloc(sizeof(double) * (size_t)(nmax > 0 ? nmax : 1));
  double v[3];
  memset(g, 0, sizeof(double) * (size_t)m);
  orc_uot_sinkhorn(d, x, n, mu, y, m, nu, lambda, eta, eta, sweeps, 0, 0, b, g, r);
  v[0] = orc_dual_value(d, x, n, mu, y, m, nu, lambda, eta, eta, b, g, 0, r);
  memset(g, 0, sizeof(double) * (size_t)n);
  orc_uot_sinkhorn(d, x, n, mu, x, n, mu, lambda, eta, eta, sweeps, 0, 0, b, g, r);
  v[1] = orc_dual_value(d, x, n, mu, x, n, mu, lambda, eta, eta, b, g, 0, r);
  memset(g, 0, sizeof(double) * (size_t)m);
  orc_uot_sinkhorn(d, y, m, nu, y, m, nu, lambda, eta, eta, sweeps, 0, 0, b, g, r);
  v[2] = orc_dual_value(d, y, m, nu, y, m, nu, lambda, eta, eta, b, g, 0, r);
  free(b);
  free(g);
  nsum sm = {0, 0}, sn = {0, 0};
  for (int64_t i = 0; i < n; ++i) nsum_add(&sm, mu[i]);
  for (int64_t j = 0; j < m; ++j) nsum_add(&sn, nu[j]);
  double dm = nsum_get(&sm) - nsum_get(&sn);
  if (parts) { parts[0] = v[0]; parts[1] = v[1]; parts[2] = v[2]; }
  return v[0] - 0.5 * v[1] - 0.5 * v[2] + dm * dm / (2.0 * lambda);
}

/* Balanced entropic OT (the eta -> infinity limit of Rem. rem:813), textbook
 * Sinkhorn with reference measure P (x) Q: alternately
 *   f_i = -(1/lambda) log sum_j k_ij Q_j e^{lambda g_j},
 *   g_j = -(1/lambda) log sum_i k_ij P_i e^{lambda f_i},
 * plan pi_ij = P_i Q_j e^{lambda (f_i + g_j)} k_ij.  Requires sum P = sum Q. */
void orc_balanced_sinkhorn(int d, const double* x, int64_t n, const double* P,
                           const double* y, int64_t m, const double* Q,
                           double lambda, int iters, double* f, double* g) {
  for (int64_t j = 0; j < m; ++j) g[j] = 0.0;
  for (int it = 0; it < iters; ++it) {
    /* q -> 1/lambda is the eta -> infinity limit of eta/(1+eta*lambda) */
    for (int side = 0; side < 2; ++side) {
      const double* a = side ? y : x; int64_t na = side ? m : n;
      const double* b = side ? x : y; int64_t nb = side ? n : m;
      const double* wb = side ? P : Q;
      const double* pb = side ? f : g;
      double* pa = side ? g : f;
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < na; ++i) {
        nsum acc = {0, 0};
        for (int64_t j = 0; j < nb; ++j)
          nsum_add(&acc, exp(-lambda * sqdist(d, a + i * d, b + j * d) + lambda * pb[j]) * wb[j]);
        pa[i] = -log(nsum_get(&acc)) / lambda;
      }
    }
  }
}

/* ---------------------------- gradients ------------------------------------
 * Partial derivatives of the quantities above with respect to the weights and
 * the support points, written directly from the definitions with
 *   d/du k(u, v) = -(2/eps) (u - v) k(u, v),  k(u, v) = exp(-||u - v||^2/eps),
 * every pairwise difference (u - v) formed explicitly.  Points are row-major
 * (gx[i*d + c] = d/dx_ic). */

/* Derivatives of MMD^2 (Eq. 1205), eps = ell^2:
 *   d/dmu_i = 2 sum_j mu_j k(x_i,x_j) - 2 sum_j nu_j k(x_i,y_j)
 *   d/dx_i  = 2 mu_i sum_j mu_j d/dx_i k(x_i,x_j) - 2 mu_i sum_j nu_j d/dx_i k(x_i,y_j)
 * (each pair of the symmetric double sum counted from both ends), and the same
 * for (nu, y) with the roles exchanged. */
static void mmd2_grad_side(int d, const double* x, int64_t n, const double* mu,
                           const double* y, int64_t m, const double* nu, double eps,
                           const int64_t* rows, int64_t nrows, double* gw, double* gp) {
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < nrows; ++r) {
    const int64_t i = rows ? rows[r] : r;
    nsum t = {0, 0};
    nsum* g = (nsum*)calloc((size_t)d, sizeof(nsum));
    for (int64_t j = 0; j < n; ++j) {
      double k = exp(-sqdist(d, x + i * d, x + j * d) / eps);
      nsum_add(&t, 2.0 * mu[j] * k);
      for (int c = 0; c < d; ++c)
        nsum_add(&g[c], 2.0 * mu[i] * mu[j] * (-2.0 / eps) * (x[i * d + c] - x[j * d + c]) * k);
    }
    for (int64_t j = 0; j < m; ++j) {
      double k = exp(-sqdist(d, x + i * d, y + j * d) / eps);
      nsum_add(&t, -2.0 * nu[j] * k);
      for (int c = 0; c < d; ++c)
        nsum_add(&g[c], -2.0 * mu[i] * nu[j] * (-2.0 / eps) * (x[i * d + c] - y[j * d + c]) * k);
    }
    if (gw) gw[r] = nsum_get(&t);
    if (gp)
      for (int c = 0; c < d; ++c) gp[r * d + c] = nsum_get(&g[c]);
    free(g);
  }
}

void orc_mmd2_grad(int d, const double* x, int64_t n, const double* mu,
                   const double* y, int64_t m, const double* nu, double ell,
                   double* gmu, double* gx, double* gnu, double* gy) {
  const double eps = ell * ell;
  mmd2_grad_side(d, x, n, mu, y, m, nu, eps, NULL, n, gmu, gx);
  mmd2_grad_side(d, y, m, nu, x, n, mu, eps, NULL, m, gnu, gy);
}

/* The same derivatives at selected rows only: side 0 gives d/dmu and d/dx at
 * the points x[rows[r]], side 1 d/dnu and d/dy at y[rows[r]]; output row r. */
void orc_mmd2_grad_rows(int d, const double* x, int64_t n, const double* mu,
                        const double* y, int64_t m, const double* nu, double ell, int side,
                        const int64_t* rows, int64_t nrows, double* gw, double* gp) {
  const double eps = ell * ell;
  if (side == 0) mmd2_grad_side(d, x, n, mu, y, m, nu, eps, rows, nrows, gw, gp);
  else mmd2_grad_side(d, y, m, nu, x, n, mu, eps, rows, nrows, gw, gp);
}

/* Partial derivatives of D(beta, gamma) of Eq. (dual_euot) (product
 * reference) in mu, x, nu, y at FIXED duals:
 *   dD/dmu_i = -eta1 e^{-beta_i/eta1} + eta1
 *              - (1/lambda) (sum_j e^{lambda beta_i} k_ij e^{lambda gamma_j} nu_j - sum_j nu_j)
 *   dD/dx_i  = -(1/lambda) sum_j mu_i nu_j e^{lambda (beta_i + gamma_j)} d/dx_i k_ij
 * with lambda = 1/eps in k, and the same for nu, y with eta2. */
static void dual_grad_side(int d, const double* x, int64_t n, const double* mu,
                           const double* y, int64_t m, const double* nu, double lambda,
                           double eta, const double* beta, const double* gamma,
                           double* gw, double* gp) {
  nsum sn = {0, 0};
  for (int64_t j = 0; j < m; ++j) nsum_add(&sn, nu[j]);
  const double mass = nsum_get(&sn);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    nsum t = {0, 0};
    nsum* g = (nsum*)calloc((size_t)d, sizeof(nsum));
    for (int64_t j = 0; j < m; ++j) {
      /* ek = e^{lambda (beta_i + gamma_j)} k_ij as one exponential */
      double ek = exp(lambda * (beta[i] + gamma[j]) - lambda * sqdist(d, x + i * d, y + j * d));
      nsum_add(&t, ek * nu[j]);
      for (int c = 0; c < d; ++c) {
        double dk = -2.0 * lambda * (x[i * d + c] - y[j * d + c]);  /* d/dx_ic k_ij / k_ij */
        nsum_add(&g[c], -(1.0 / lambda) * mu[i] * nu[j] * ek * dk);
      }
    }
    if (gw) gw[i] = -eta * exp(-beta[i] / eta) + eta - (nsum_get(&t) - mass) / lambda;
    if (gp)
      for (int c = 0; c < d; ++c) gp[i * d + c] = nsum_get(&g[c]);
    free(g);
  }
}

void orc_dual_grad(int d, const double* x, int64_t n, const double* mu,
                   const double* y, int64_t m, const double* nu, double lambda,
                   double eta1, double eta2, const double* beta, const double* gamma,
                   double* gmu, double* gx, double* gnu, double* gy) {
  dual_grad_side(d, x, n, mu, y, m, nu, lambda, eta1, beta, gamma, gmu, gx);
  dual_grad_side(d, y, m, nu, x, n, mu, lambda, eta2, gamma, beta, gnu, gy);
}

/* Gradient of the Sinkhorn divergence of Eq. (586) by the envelope theorem:
 * each UOT value is max D(beta, gamma), so its derivative is the partial
 * derivative of D at the maximising duals, here the duals after `sweeps`
 * sweeps of Alg. 1 from gamma^0 = 0.  In UOT(mu, mu) and UOT(nu, nu) the
 * measure fills both arguments and both partial derivatives count.  The
 * mass term adds (mu(X) - nu(X))/lambda to d/dmu and subtracts it from d/dnu.
 * Returns the divergence (as orc_sinkhorn_divergence). */
double orc_sinkhorn_divergence_grad(int d, const double* x, int64_t n, const double* mu,
                                    const double* y, int64_t m, const double* nu,
                                    double lambda, double eta, int sweeps,
                                    double* gmu, double* gx, double* gnu, double* gy) {
  int64_t nmax = n > m ? n : m;
  size_t sz = (size_t)(nmax > 0 ? nmax : 1);
  double* b = (double*)malloc(sizeof(double) * sz);
  double* g = (double*)malloc(sizeof(double) * sz);
  double* w1 = (double*)malloc(sizeof(double) * sz);
  double* w2 = (double*)malloc(sizeof(double) * sz);
  double* p1 = (double*)malloc(sizeof(double) * sz * (size_t)d);
  double* p2 = (double*)malloc(sizeof(double) * sz * (size_t)d);
  double v[3];
  /* UOT(mu, nu) */
  memset(g, 0, sizeof(double) * (size_t)m);
  orc_uot_sinkhorn(d, x, n, mu, y, m, nu, lambda, eta, eta, sweeps, 0, 0, b, g, 2.0);
  v[0] = orc_dual_value(d, x, n, mu, y, m, nu, lambda, eta, eta, b, g, 0, 2.0);
  orc_dual_grad(d, x, n, mu, y, m, nu, lambda, eta, eta, b, g, gmu, gx, gnu, gy);
  /* UOT(mu, mu) */
  memset(g, 0, sizeof(double) * (size_t)n);
  orc_uot_sinkhorn(d, x, n, mu, x, n, mu, lambda, eta, eta, sweeps, 0, 0, b, g, 2.0);
  v[1] = orc_dual_value(d, x, n, mu, x, n, mu, lambda, eta, eta, b, g, 0, 2.0);
  orc_dual_grad(d, x, n, mu, x, n, mu, lambda, eta, eta, b, g, w1, p1, w2, p2);
  for (int64_t i = 0; i < n; ++i) {
    gmu[i] -= 0.5 * (w1[i] + w2[i]);
    for (int c = 0; c < d; ++c) gx[i * d + c] -= 0.5 * (p1[i * d + c] + p2[i * d + c]);
  }
  /* UOT(nu, nu) */
  memset(g, 0, sizeof(double) * (size_t)m);
  orc_uot_sinkhorn(d, y, m, nu, y, m, nu, lambda, eta, eta, sweeps, 0, 0, b, g, 2.0);
  v[2] = orc_dual_value(d, y, m, nu, y, m, nu, lambda, eta, eta, b, g, 0, 2.0);
  orc_dual_grad(d, y, m, nu, y, m, nu, lambda, eta, eta, b, g, w1, p1, w2, p2);
  for (int64_t j = 0; j < m; ++j) {
    gnu[j] -= 0.5 * (w1[j] + w2[j]);
    for (int c = 0; c < d; ++c) gy[j * d + c] -= 0.5 * (p1[j * d + c] + p2[j * d + c]);
  }
  free(b); free(g); free(w1); free(w2); free(p1); free(p2);
  nsum sm = {0, 0}, sn = {0, 0};
  for (int64_t i = 0; i < n; ++i) nsum_add(&sm, mu[i]);
  for (int64_t j = 0; j < m; ++j) nsum_add(&sn, nu[j]);
  double dm = nsum_get(&sm) - nsum_get(&sn);
  for (int64_t i = 0; i < n; ++i) gmu[i] += dm / lambda;
  for (int64_t j = 0; j < m; ++j) gnu[j] -= dm / lambda;
  return v[0] - 0.5 * v[1] - 0.5 * v[2] + dm * dm / (2.0 * lambda);
}

/* ------------------- the other kernels of Table tab:0 -----------------------
 * kind 0 Gauss   k = exp(-r^2 / p^2)
 * kind 1 Laplace k = exp(-r / p)
 * kind 2 IMQ     k = 1 / sqrt(r^2 + p^2)       (p = the constant c of the table)
 * kind 3 energy  k = -r
 * with r = ||x - x~||. */
static inline double kern(int kind, double r2, double p) {
  switch (kind) {
    case 0: return exp(-r2 / (p * p));
    case 1: return exp(-sqrt(r2) / p);
    case 2: return 1.0 / sqrt(r2 + p * p);
    default: return -sqrt(r2);
  }
}

/* out_j = sum_i w_i k(src_i, tgt_j) for the kernel `kind` with parameter p. */
void orc_ksum_kernel(int kind, double p, int d, const double* src, int64_t n, const double* w,
                     const double* tgt, int64_t m, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < m; ++j) {
    nsum acc = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i)
      nsum_add(&acc, w[i] * kern(kind, sqdist(d, src + i * d, tgt + j * d), p));
    out[j] = nsum_get(&acc);
  }
}

/* MMD^2 of Eq. (1205) with the kernel `kind` (parameter p); parts as orc_mmd2. */
double orc_mmd2_kernel(int kind, double p, int d, const double* x, int64_t n, const double* mu,
                       const double* y, int64_t m, const double* nu, double* parts) {
  double* kx = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* ky = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  nsum A = {0, 0}, B = {0, 0}, C = {0, 0};
  orc_ksum_kernel(kind, p, d, x, n, mu, x, n, kx);
  for (int64_t i = 0; i < n; ++i) nsum_add(&A, mu[i] * kx[i]);
  orc_ksum_kernel(kind, p, d, y, m, nu, x, n, kx);
  for (int64_t i = 0; i < n; ++i) nsum_add(&B, mu[i] * kx[i]);
  orc_ksum_kernel(kind, p, d, y, m, nu, y, m, ky);
  for (int64_t j = 0; j < m; ++j) nsum_add(&C, nu[j] * ky[j]);
  free(kx);
  free(ky);
  if (parts) { parts[0] = nsum_get(&A); parts[1] = nsum_get(&B); parts[2] = nsum_get(&C); }
  return nsum_get(&A) - 2.0 * nsum_get(&B) + nsum_get(&C);
}

/* <mu (x) nu | d^r> = sum_i sum_j mu_i nu_j ||x_i - y_j||^r, the plain double sum
 * (r = 2: the mean-cost numerator of Eq. (561); r = 1: the inner product of the
 * complexity paragraph of Sec. 4.4, d = -k_e). */
double orc_mean_cost(int d, const double* x, int64_t n, const double* mu, const double* y,
                     int64_t m, const double* nu, double r) {
  nsum acc = {0.0, 0.0};
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < m; ++j) {
      double s = sqdist(d, x + i * d, y + j * d);
      nsum_add(&acc, mu[i] * nu[j] * (r == 2.0 ? s : pow(sqrt(s), r)));
    }
  return nsum_get(&acc);
}

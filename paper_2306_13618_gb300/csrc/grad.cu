// Gradients of MMD^2 (Eq. 1205) and of the unbalanced Sinkhorn divergence
// (Eq. 586) with respect to the weights and the support points of both
// measures.
//
// Both reduce to kernel summations on the engine that computes the value:
//   grad_x k(x, y) = -(2/eps) (x - y) k(x, y),
// so every gradient row needs, besides t_i = sum_j w_j k_ij, the sums
//   s_ic = sum_j w_j y'_jc k_ij   (c = 1..d),   y' = y - o,
// and reads sum_j w_j (x_i - y_j)_c k_ij = x'_ic t_i - s_ic.  The origin o is
// the first support point of x: the difference is translation invariant, and
// a common point of the clouds keeps |x'|, |y'| within their joint diameter.
//
// Sinkhorn divergence: each UOT value is the dual maximum D(beta*, gamma*) of
// Eq. (dual_euot), so by the envelope theorem its derivative in any parameter
// is the partial derivative of D at the maximising duals.  We evaluate it at
// the duals of the last sweep (exact at convergence).  For one problem
// UOT(mu, nu) (product reference, eta1 = eta2 = eta, lambda = 1/eps):
//   dD/dmu_i = -eta e^{-beta_i/eta} + eta - (e^{lambda beta_i} T_i - nu(X))/lambda,
//   dD/dx_i  = 2 mu_i e^{lambda beta_i} sum_j nu_j e^{lambda gamma_j} (x_i - y_j) k_ij,
//   T_i = sum_j k_ij nu_j e^{lambda gamma_j},
// and the same with the roles of (mu, x, beta) and (nu, y, gamma) exchanged.
// The symmetric problems UOT(mu, mu), UOT(nu, nu) contribute through both roles.
#include <math.h>

#include <memory>

#include "solver.cuh"

namespace uotk {

namespace {

// out[i] = base[i] * (p[q(i)*d + c] - org[c]) for i < count (base NULL: 1),
// q = perm (NULL: identity); out[count .. count+4) = 0.
__global__ void k_coord_weights(const int* __restrict__ perm, const float* __restrict__ pts,
                                long long count, int d, int c, const float* __restrict__ org,
                                const float* __restrict__ base, float* __restrict__ out) {
  const float o = org[c];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count + 4;
       i += (long long)gridDim.x * blockDim.x) {
    if (i >= count) {
      out[i] = 0.f;
      continue;
    }
    const long long q = perm ? perm[i] : i;
    const float v = __fsub_rn(pts[q * d + c], o);
    out[i] = base ? __fmul_rn(base[i], v) : v;
  }
}

// One role of one UOT problem, internal index i of the side with potential pot:
//   e_i = exp(lambda pot_i + M),  M = shift of the other side's weights,
//   g_w[q(i)]   += coef * (-eta e^{-pot_i/eta} + eta - (e_i t_i - mass_other)/lambda)
//   g_p[q(i),c] += coef * 2 w_i e_i (p'_ic t_i - s[c*count + i])
// Either output may be NULL; each caller index is owned by one thread.
__global__ void k_uot_role_grad(long long count, int d, const int* __restrict__ perm,
                                const float* __restrict__ pts, const float* __restrict__ org,
                                const float* __restrict__ w, const double* __restrict__ pot,
                                const float* __restrict__ t, const float* __restrict__ s,
                                double lam, double eta, double mass_other,
                                const long long* __restrict__ shift_slot, double coef,
                                double* __restrict__ g_w, double* __restrict__ g_p) {
  const double M = ordered_to_dbl(*shift_slot);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const long long q = perm ? perm[i] : i;
    const double e = exp(lam * pot[i] + M);
    const double ti = (double)t[i];
    if (g_w) g_w[q] += coef * (-eta * exp(-pot[i] / eta) + eta - (e * ti - mass_other) / lam);
    if (g_p) {
      const double f = coef * 2.0 * (double)w[i] * e;
      for (int c = 0; c < d; ++c) {
        const double pc = (double)__fsub_rn(pts[q * d + c], org[c]);
        g_p[q * d + c] += f * (pc * ti - (double)s[c * count + i]);
      }
    }
  }
}

// MMD^2 rows of one side, internal index i:
//   g_w[q(i)]   = 2 (t1_i - t2_i)
//   g_p[q(i),c] = -(4 w_i/eps) (p'_ic (t1_i - t2_i) - (s1 - s2)[c*count + i])
__global__ void k_mmd_grad(long long count, int d, const int* __restrict__ perm,
                           const float* __restrict__ pts, const float* __restrict__ org,
                           const float* __restrict__ w, const float* __restrict__ t1,
                           const float* __restrict__ t2, const float* __restrict__ s1,
                           const float* __restrict__ s2, double eps, double* __restrict__ g_w,
                           double* __restrict__ g_p) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const long long q = perm ? perm[i] : i;
    const double dt = (double)t1[i] - (double)t2[i];
    if (g_w) g_w[q] = 2.0 * dt;
    if (g_p) {
      const double f = -4.0 * (double)w[i] / eps;
      for (int c = 0; c < d; ++c) {
        const double pc = (double)__fsub_rn(pts[q * d + c], org[c]);
        const long long k = c * count + i;
        g_p[q * d + c] = f * (pc * dt - ((double)s1[k] - (double)s2[k]));
      }
    }
  }
}

uotk_status coord_weights(uotk_ctx* ctx, cudaStream_t s, const Engine* E, int side,
                          const float* pts, int64_t count, int d, int c, const float* org,
                          const float* base, float* out) {
  k_coord_weights<<<grid_for(ctx, count + 4, 256), 256, 0, s>>>(E->perm(side), pts, count, d, c,
                                                                org, base, out);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

int64_t at_least1(int64_t v) { return v > 0 ? v : 1; }

__global__ void k_add_constant(double* __restrict__ g, long long count, double v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    g[i] += v;
}

uotk_status add_constant(uotk_ctx* ctx, cudaStream_t s, double* g, int64_t count, double v) {
  if (!g || count == 0) return UOTK_OK;
  k_add_constant<<<grid_for(ctx, count, 256), 256, 0, s>>>(g, count, v);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// MMD^2 and its gradient.
// ---------------------------------------------------------------------------
uotk_status op_mmd2_grad(uotk_ctx* ctx, cudaStream_t s, int d, const float* x, int64_t n,
                         const float* a, const float* y, int64_t m, const float* b, double ell,
                         double* mmd2, double* grad_a, double* grad_x, double* grad_b,
                         double* grad_y, const uotk_sum_opts* opts) {
  const double eps = ell * ell;
  EngineSpec sp{opts ? opts->method : UOTK_DIRECT, d, x, n, a, y, m, b, eps, opts};
  const bool px = grad_x != nullptr, py = grad_y != nullptr;
  const bool coords = px || py;
  const int64_t n1 = at_least1(n), m1 = at_least1(m);
  // d <= 3: every coordinate's weights at once, so that each (source, target)
  // pair of clouds takes one multi-sum of 1 + d right-hand sides
  const bool fused = coords && d <= 3;
  auto carve = [&](Carver& cv, float** t, float** sx, float** sy, float** wbuf, Reducer& R) {
    for (int k = 0; k < 2; ++k) t[k] = cv.take<float>(n1);
    for (int k = 2; k < 4; ++k) t[k] = cv.take<float>(m1);
    for (int k = 0; k < 2; ++k) sx[k] = cv.take<float>(coords ? (size_t)d * n1 : 1);
    for (int k = 0; k < 2; ++k) sy[k] = cv.take<float>(coords ? (size_t)d * m1 : 1);
    *wbuf = cv.take<float>((size_t)(fused ? 2 * d : 1) * ((n > m ? n : m) + 4));
    carve_reducer(ctx, cv, R);
  };
  float *t[4], *sx[2], *sy[2], *wbuf;
  Reducer R;
  const size_t eb = engine_bytes(ctx, sp);
  Carver size(nullptr);
  size.off = eb;
  carve(size, t, sx, sy, &wbuf, R);
  UOTK_TRY(ws_reserve(ctx, size.off));
  UOTK_TRY(flags_reset(ctx, s));
  Carver cv(ctx->ws);
  Engine* raw = nullptr;
  UOTK_TRY(engine_create(ctx, s, sp, cv, &raw));
  std::unique_ptr<Engine> E(raw);
  cv.off = eb;
  carve(cv, t, sx, sy, &wbuf, R);
  const float* ai = E->weights(0);
  const float* bi = E->weights(1);
  if (fused) {
    // right-hand sides {w, w (p_1 - o_1), .., w (p_d - o_d)} of each cloud
    const size_t stride = (size_t)((n > m ? n : m) + 4);
    const float* W[2][4] = {{ai}, {bi}};
    for (int c = 0; c < d; ++c) {
      float* wx = wbuf + (size_t)c * stride;
      float* wy = wbuf + (size_t)(d + c) * stride;
      UOTK_TRY(coord_weights(ctx, s, E.get(), 0, x, n, d, c, x, ai, wx));
      UOTK_TRY(coord_weights(ctx, s, E.get(), 1, y, m, d, c, x, bi, wy));
      W[0][1 + c] = wx;
      W[1][1 + c] = wy;
    }
    // (src, tgt, t output, coordinate-sum output): K_xx a, K_xy b, K_yy b, K_yx a
    struct Job { int src, tgt; float* t; float* sc; int64_t len; bool want; };
    const Job jobs[4] = {{0, 0, t[0], sx[0], n1, px}, {1, 0, t[1], sx[1], n1, px},
                         {1, 1, t[2], sy[0], m1, py}, {0, 1, t[3], sy[1], m1, py}};
    for (const Job& j : jobs) {
      float* outs[4] = {j.t};
      for (int c = 0; c < d; ++c) outs[1 + c] = j.sc + c * j.len;
      UOTK_TRY(E->sums_multi(s, j.src, j.tgt, j.want ? 1 + d : 1, W[j.src], nullptr, 0.0,
                             nullptr, outs));
    }
  } else {
    UOTK_TRY(E->plain(s, 0, 0, ai, t[0]));  // (K_xx a)_i
    UOTK_TRY(E->plain(s, 1, 0, bi, t[1]));  // (K_xy b)_i
    UOTK_TRY(E->plain(s, 1, 1, bi, t[2]));  // (K_yy b)_j
    UOTK_TRY(E->plain(s, 0, 1, ai, t[3]));  // (K_yx a)_j
  }
  if (coords && !fused) {
    for (int c = 0; c < d; ++c) {
      UOTK_TRY(coord_weights(ctx, s, E.get(), 0, x, n, d, c, x, ai, wbuf));
      if (px) UOTK_TRY(E->plain(s, 0, 0, wbuf, sx[0] + c * n1));
      if (py) UOTK_TRY(E->plain(s, 0, 1, wbuf, sy[1] + c * m1));
      UOTK_TRY(coord_weights(ctx, s, E.get(), 1, y, m, d, c, x, bi, wbuf));
      if (px) UOTK_TRY(E->plain(s, 1, 0, wbuf, sx[1] + c * n1));
      if (py) UOTK_TRY(E->plain(s, 1, 1, wbuf, sy[0] + c * m1));
    }
  }
  if (grad_a || px) {
    k_mmd_grad<<<grid_for(ctx, n, 256), 256, 0, s>>>(n, d, E->perm(0), x, x, ai, t[0], t[1],
                                                     sx[0], sx[1], eps, grad_a, grad_x);
    UOTK_LAUNCHED(ctx);
  }
  if (grad_b || py) {
    k_mmd_grad<<<grid_for(ctx, m, 256), 256, 0, s>>>(m, d, E->perm(1), y, x, bi, t[2], t[3],
                                                     sy[0], sy[1], eps, grad_b, grad_y);
    UOTK_LAUNCHED(ctx);
  }
  SumTerms T{};
  T.count = 3;
  T.k[0] = SumTerm{2, n, ai, nullptr, t[0], 1.0, 1.0, 0};
  T.k[1] = SumTerm{2, n, ai, nullptr, t[1], 1.0, 1.0, 0};
  T.k[2] = SumTerm{2, m, bi, nullptr, t[2], 1.0, 1.0, 0};
  UOTK_TRY(run_sums(ctx, s, R, T, ctx->host + 16));
  UOTK_TRY(flags_check(ctx, s, "mmd2_grad"));
  const double* h = ctx->host + 16;
  if (mmd2) *mmd2 = h[0] - 2.0 * h[1] + h[2];
  return UOTK_OK;
}

// ---------------------------------------------------------------------------
// Sinkhorn divergence and its gradient.
// ---------------------------------------------------------------------------
uotk_status op_sinkhorn_divergence_grad(uotk_ctx* ctx, cudaStream_t s, int d, const float* x,
                                        int64_t n, const float* a, const float* y, int64_t m,
                                        const float* b, double eps, double rho, int max_sweeps,
                                        double tol, double* sd, double* parts, double* grad_a,
                                        double* grad_x, double* grad_b, double* grad_y,
                                        const uotk_sum_opts* opts) {
  const int method = opts ? opts->method : UOTK_DIRECT;
  const EngineSpec specs[3] = {
      {method, d, x, n, a, y, m, b, eps, opts},
      {method, d, x, n, a, x, n, a, eps, opts},
      {method, d, y, m, b, y, m, b, eps, opts}};
  // Outputs of each problem's two roles: (weights, points) gradients and
  // their coefficients in Eq. (586).
  double* gw[3][2] = {{grad_a, grad_b}, {grad_a, grad_a}, {grad_b, grad_b}};
  double* gp[3][2] = {{grad_x, grad_y}, {grad_x, grad_x}, {grad_y, grad_y}};
  const double coef[3] = {1.0, -0.5, -0.5};
  const double lam = 1.0 / eps;
  // d <= 3: all coordinate weights of a role at once (one multi-sum per role)
  const bool fused = d <= 3;
  auto carve = [&](Carver& cv, const EngineSpec& sp, SolveBufs& B, Reducer& R, float** tx,
                   float** sxy, float** wbuf) {
    carve_solve(cv, sp.n, sp.m, true, B);
    carve_reducer(ctx, cv, R);
    *tx = cv.take<float>(at_least1(sp.n));
    sxy[0] = cv.take<float>((size_t)d * at_least1(sp.n));
    sxy[1] = cv.take<float>((size_t)d * at_least1(sp.m));
    *wbuf = cv.take<float>((size_t)(fused ? d : 1) * ((sp.n > sp.m ? sp.n : sp.m) + 4));
  };
  size_t need = 0;
  for (const EngineSpec& sp : specs) {
    Carver c(nullptr);
    c.off = engine_bytes(ctx, sp);
    SolveBufs B;
    Reducer R;
    float *tx, *sxy[2], *wbuf;
    carve(c, sp, B, R, &tx, sxy, &wbuf);
    need = c.off > need ? c.off : need;
  }
  UOTK_TRY(ws_reserve(ctx, need));
  if (grad_a) UOTK_CUDA(ctx, cudaMemsetAsync(grad_a, 0, sizeof(double) * n, s));
  if (grad_b) UOTK_CUDA(ctx, cudaMemsetAsync(grad_b, 0, sizeof(double) * m, s));
  if (grad_x) UOTK_CUDA(ctx, cudaMemsetAsync(grad_x, 0, sizeof(double) * n * d, s));
  if (grad_y) UOTK_CUDA(ctx, cudaMemsetAsync(grad_y, 0, sizeof(double) * m * d, s));
  double v[3];
  double masses[2] = {0, 0};
  bool all_converged = true;
  for (int k = 0; k < 3; ++k) {
    const EngineSpec& sp = specs[k];
    const bool pts_role[2] = {gp[k][0] != nullptr, gp[k][1] != nullptr};
    const bool any_role[2] = {pts_role[0] || gw[k][0], pts_role[1] || gw[k][1]};
    UOTK_TRY(flags_reset(ctx, s));
    Carver cv(ctx->ws);
    Engine* raw = nullptr;
    UOTK_TRY(engine_create(ctx, s, sp, cv, &raw));
    std::unique_ptr<Engine> E(raw);
    cv.off = engine_bytes(ctx, sp);
    SolveBufs B;
    Reducer R;
    float *tx, *sxy[2], *wbuf;
    carve(cv, sp, B, R, &tx, sxy, &wbuf);
    SolveResult res;
    UOTK_TRY(solve(ctx, s, E.get(), sp.n, sp.m, eps, rho, rho, max_sweeps, tol, 0, false, B, R,
                   &res));
    all_converged = all_converged && res.converged;
    v[k] = res.value;
    const double mass[2] = {ctx->host[8 + 2], ctx->host[8 + 3]};
    if (k == 0) { masses[0] = mass[0]; masses[1] = mass[1]; }
    // Shift slots of the final duals (see solve()).
    const int last = (res.sweeps - 1) & 1;
    const long long* shift_g = ctx->dflags + FLAG_MAX_G0 + (last ^ 1);
    const long long* shift_b = ctx->dflags + FLAG_MAX_B0 + last;
    const float* wx = E->weights(0);
    const float* wy = E->weights(1);
    // Role 0 (first cloud, potential beta): T_i at the final gamma, and the
    // coordinate sums over the second cloud with the final-gamma weights.
    const size_t stride = (size_t)((sp.n > sp.m ? sp.n : sp.m) + 4);
    if (fused) {
      // one multi-sum per role: {T_i, s_i1, .., s_id} over the other cloud
      const float* W[4] = {wy};
      float* outs[4] = {tx};
      if (any_role[0]) {
        const int K = pts_role[0] ? 1 + d : 1;
        for (int c = 0; pts_role[0] && c < d; ++c) {
          UOTK_TRY(coord_weights(ctx, s, E.get(), 1, sp.y, sp.m, d, c, x, wy,
                                 wbuf + (size_t)c * stride));
          W[1 + c] = wbuf + (size_t)c * stride;
          outs[1 + c] = sxy[0] + c * at_least1(sp.n);
        }
        UOTK_TRY(E->sums_multi(s, 1, 0, K, W, B.gamma, lam, shift_g, outs));
      }
      // Role 1 (second cloud, potential gamma): B.ty already holds the sum at
      // the final beta (the last half-step); coordinate sums over the first cloud.
      if (pts_role[1]) {
        for (int c = 0; c < d; ++c) {
          UOTK_TRY(coord_weights(ctx, s, E.get(), 0, sp.x, sp.n, d, c, x, wx,
                                 wbuf + (size_t)c * stride));
          W[c] = wbuf + (size_t)c * stride;
          outs[c] = sxy[1] + c * at_least1(sp.m);
        }
        UOTK_TRY(E->sums_multi(s, 0, 1, d, W, B.beta, lam, shift_b, outs));
      }
    } else {
      if (any_role[0]) UOTK_TRY(E->half(s, 0, wy, B.gamma, lam, shift_g, tx));
      if (pts_role[0]) {
        for (int c = 0; c < d; ++c) {
          UOTK_TRY(coord_weights(ctx, s, E.get(), 1, sp.y, sp.m, d, c, x, wy, wbuf));
          UOTK_TRY(E->half(s, 0, wbuf, B.gamma, lam, shift_g, sxy[0] + c * at_least1(sp.n)));
        }
      }
      // Role 1 (second cloud, potential gamma): B.ty already holds the sum at the
      // final beta (the last half-step); coordinate sums over the first cloud.
      if (pts_role[1]) {
        for (int c = 0; c < d; ++c) {
          UOTK_TRY(coord_weights(ctx, s, E.get(), 0, sp.x, sp.n, d, c, x, wx, wbuf));
          UOTK_TRY(E->half(s, 1, wbuf, B.beta, lam, shift_b, sxy[1] + c * at_least1(sp.m)));
        }
      }
    }
    if (any_role[0]) {
      k_uot_role_grad<<<grid_for(ctx, sp.n, 256), 256, 0, s>>>(
          sp.n, d, E->perm(0), sp.x, x, wx, B.beta, tx, sxy[0], lam, rho, mass[1], shift_g,
          coef[k], gw[k][0], gp[k][0]);
      UOTK_LAUNCHED(ctx);
    }
    if (any_role[1]) {
      k_uot_role_grad<<<grid_for(ctx, sp.m, 256), 256, 0, s>>>(
          sp.m, d, E->perm(1), sp.y, x, wy, B.gamma, B.ty, sxy[1], lam, rho, mass[0], shift_b,
          coef[k], gw[k][1], gp[k][1]);
      UOTK_LAUNCHED(ctx);
    }
    // The engine's workspace is reused by the next problem: finish first.
    UOTK_TRY(flags_check(ctx, s, "sinkhorn_divergence_grad"));
  }
  const double dm = masses[0] - masses[1];
  if (sd) *sd = v[0] - 0.5 * v[1] - 0.5 * v[2] + 0.5 * eps * dm * dm;
  if (parts) { parts[0] = v[0]; parts[1] = v[1]; parts[2] = v[2]; }
  // d/dmu_i and d/dnu_j of the mass term (mu(X) - nu(X))^2 / (2 lambda).
  if (grad_a || grad_b) {
    UOTK_TRY(add_constant(ctx, s, grad_a, n, eps * dm));
    UOTK_TRY(add_constant(ctx, s, grad_b, m, -eps * dm));
  }
  UOTK_CUDA(ctx, cudaStreamSynchronize(s));
  if (tol > 0.0 && !all_converged)
    return set_error(ctx, UOTK_ERR_NOT_CONVERGED,
                     "sinkhorn_divergence_grad: tol %g not reached", tol);
  return UOTK_OK;
}

}  // namespace uotk

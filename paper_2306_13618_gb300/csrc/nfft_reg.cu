// NFFT fast summation for the non-smooth kernels of Table tab:0 (Laplace
// exp(-r/p), inverse multiquadric 1/sqrt(r^2 + p^2), energy -r), Sec. 4.2.
//
// In torus units rbar = r/h the kernel is replaced by the regularised kernel
//   K_R(rbar) = T_I(rbar)   rbar < eps_I
//             = K(h rbar)   eps_I <= rbar <= 1/2 - eps_B
//             = T_B(rbar)   1/2 - eps_B < rbar <= 1/2
//             = K_B         rbar > 1/2,
// T_I and T_B two-point Taylor interpolants of degree 2p - 1: T_I matches the
// first p derivatives (orders 0..p-1) of K at +-eps_I (K_R is even); T_B
// matches them at 1/2 - eps_B and is flat at 1/2 with the value K_B, the
// midpoint value of the interpolant that matches K at 1/2 - eps_B and its
// mirror image at 1/2 + eps_B.  K_R is then C^{p-1} on the torus and its
// Fourier coefficients b_k, the DFT of its samples on I_N^d, decay fast; the
// fast summation of Eq. (1724) uses them in place of the Gaussian's, and the
// near field sum_{|x - y| < eps_I h} w (K - T_I) restores the exact kernel.
// The plan keeps every difference below (1/2 - eps_B) h, so K_R = K there
// otherwise.
#include <math.h>

#include <vector>

#include "nfft.cuh"

namespace uotk {

namespace {

constexpr int REG_MAXP = 12;
constexpr int NEAR_THREADS = 256;

// Monomial coefficients (in a scaled variable t) of the regularised pieces.
struct RegPoly {
  double ti[REG_MAXP];       // T_I = sum_q ti[q] u^q,  u = (rbar / eps_I)^2
  double tb[2 * REG_MAXP];   // T_B = sum_q tb[q] t^q,  t = (rbar - 1/2 + eps_B/2) / (eps_B/2)
  double kb;                 // K_B
  double eps_i, eps_b, h, par;
  int kind, P;
};

// c_j = K^{(j)}(r0) / j!, j < order, for the kernel `kind` with parameter par.
void kernel_taylor(int kind, double par, double r0, int order, double* c) {
  for (int j = 0; j < order; ++j) c[j] = 0.0;
  if (kind == UOTK_KERNEL_LAPLACE) {
    double f = exp(-r0 / par);
    for (int j = 0; j < order; ++j) {
      c[j] = f;
      f *= -1.0 / (par * (j + 1));
    }
  } else if (kind == UOTK_KERNEL_IMQ) {
    // (r^2 + par^2) K' + r K = 0, expanded about r0 in powers of (r - r0)
    const double g0 = r0 * r0 + par * par;
    c[0] = 1.0 / sqrt(g0);
    for (int n = 0; n + 1 < order; ++n) {
      const double prev = n >= 1 ? c[n - 1] : 0.0;
      c[n + 1] = -((2.0 * n + 1.0) * r0 * c[n] + n * prev) / ((n + 1.0) * g0);
    }
  } else {  // energy
    c[0] = -r0;
    if (order > 1) c[1] = -1.0;
  }
}

// a * b for polynomials given by their coefficient vectors.
std::vector<double> pmul(const std::vector<double>& a, const std::vector<double>& b) {
  std::vector<double> r(a.size() + b.size() - 1, 0.0);
  for (size_t i = 0; i < a.size(); ++i)
    for (size_t j = 0; j < b.size(); ++j) r[i + j] += a[i] * b[j];
  return r;
}
void padd(std::vector<double>& acc, const std::vector<double>& a, double f) {
  if (acc.size() < a.size()) acc.resize(a.size(), 0.0);
  for (size_t i = 0; i < a.size(); ++i) acc[i] += f * a[i];
}
std::vector<double> ppow(const std::vector<double>& a, int e) {
  std::vector<double> r{1.0};
  for (int i = 0; i < e; ++i) r = pmul(r, a);
  return r;
}
double binom(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// Monomial coefficients on t in [-1, 1] of the polynomial T of degree 2P - 1
// with T^{(j)}(-1)/j! = ca[j] and T^{(j)}(1)/j! = cb[j], j < P.  With
// s = (t + 1)/2 the Hermite form is
//   T = (1-s)^P sum_j ca_j (t+1)^j sum_{k<P-j} C(P-1+k, k) s^k
//     + s^P     sum_j cb_j (t-1)^j sum_{k<P-j} C(P-1+k, k) (1-s)^k,
// each sum over k being the series of (1-s)^{-P} (resp. s^{-P}) cut where it
// stops affecting the derivatives of order < P at its end point.
std::vector<double> two_point(const double* ca, const double* cb, int P) {
  const std::vector<double> s{0.5, 0.5}, oms{0.5, -0.5}, tp1{1.0, 1.0}, tm1{-1.0, 1.0};
  const std::vector<double> sP = ppow(s, P), omsP = ppow(oms, P);
  std::vector<double> T(2 * P, 0.0);
  for (int j = 0; j < P; ++j) {
    std::vector<double> sa{0.0}, sb{0.0};
    for (int k = 0; k < P - j; ++k) {
      padd(sa, ppow(s, k), binom(P - 1 + k, k));
      padd(sb, ppow(oms, k), binom(P - 1 + k, k));
    }
    padd(T, pmul(omsP, pmul(ppow(tp1, j), sa)), ca[j]);
    padd(T, pmul(sP, pmul(ppow(tm1, j), sb)), cb[j]);
  }
  T.resize(2 * P);
  return T;
}

RegPoly make_reg_poly(const NfftParams& Pm) {
  RegPoly R{};
  const int P = Pm.reg_p;
  R.P = P;
  R.kind = Pm.kernel;
  R.par = Pm.eps;
  R.h = Pm.h;
  R.eps_i = R.eps_b = Pm.eps_i;
  double c[REG_MAXP], ca[REG_MAXP], cb[REG_MAXP];
  // T_I on rbar in [-eps_I, eps_I], t = rbar / eps_I: derivatives of K at r = h eps_I
  kernel_taylor(R.kind, R.par, R.h * R.eps_i, P, c);
  double sc = 1.0;
  for (int j = 0; j < P; ++j) {
    cb[j] = c[j] * sc;
    ca[j] = (j & 1) ? -cb[j] : cb[j];
    sc *= R.h * R.eps_i;
  }
  const std::vector<double> ti = two_point(ca, cb, P);
  for (int q = 0; q < P; ++q) R.ti[q] = ti[2 * q];  // even: odd coefficients vanish
  // K_B: the mirror-symmetric interpolant about 1/2 on [1/2 - eps_B, 1/2 + eps_B],
  // t = (rbar - 1/2)/eps_B, at t = 0
  kernel_taylor(R.kind, R.par, R.h * (0.5 - R.eps_b), P, c);
  sc = 1.0;
  for (int j = 0; j < P; ++j) {
    ca[j] = c[j] * sc;
    cb[j] = (j & 1) ? -ca[j] : ca[j];
    sc *= R.h * R.eps_b;
  }
  R.kb = two_point(ca, cb, P)[0];
  // T_B on [1/2 - eps_B, 1/2], t = (rbar - 1/2 + eps_B/2) / (eps_B/2): K's
  // derivatives at t = -1, the constant K_B (flat) at t = 1
  sc = 1.0;
  for (int j = 0; j < P; ++j) {
    ca[j] = c[j] * sc;
    cb[j] = j == 0 ? R.kb : 0.0;
    sc *= 0.5 * R.h * R.eps_b;
  }
  const std::vector<double> tb = two_point(ca, cb, P);
  for (int q = 0; q < 2 * P; ++q) R.tb[q] = tb[q];
  return R;
}

__host__ __device__ double reg_kernel(const RegPoly& R, double rb) {
  if (rb < R.eps_i) {
    const double u = (rb / R.eps_i) * (rb / R.eps_i);
    double v = R.ti[R.P - 1];
    for (int q = R.P - 2; q >= 0; --q) v = fma(v, u, R.ti[q]);
    return v;
  }
  if (rb <= 0.5 - R.eps_b) {
    const double r = R.h * rb;
    if (R.kind == UOTK_KERNEL_LAPLACE) return exp(-r / R.par);
    if (R.kind == UOTK_KERNEL_IMQ) return 1.0 / sqrt(r * r + R.par * R.par);
    return -r;
  }
  if (rb <= 0.5) {
    const double t = (rb - 0.5 + 0.5 * R.eps_b) / (0.5 * R.eps_b);
    double v = R.tb[2 * R.P - 1];
    for (int q = 2 * R.P - 2; q >= 0; --q) v = fma(v, t, R.tb[q]);
    return v;
  }
  return R.kb;
}

// K_R(|l|/N) for l in I_N^d, index i0 + N (i1 + N i2), l_t = i_t - N/2.
__global__ void k_reg_samples(RegPoly R, int N, int d, double* __restrict__ out) {
  long long total = N;
  for (int t = 1; t < d; ++t) total *= N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long q = i;
    double r2 = 0.0;
    for (int t = 0; t < d; ++t) {
      const double l = (double)(q % N - N / 2) / N;
      r2 += l * l;
      q /= N;
    }
    out[i] = reg_kernel(R, sqrt(r2));
  }
}

// One axis of the real, even DFT: out[.., j, ..] = sum_i in[.., i, ..] ctab[j N + i],
// ctab[j N + i] = cos(2 pi (j - N/2)(i - N/2) / N).
__global__ void k_dct_axis(const double* __restrict__ in, double* __restrict__ out, int N, int d,
                           int axis, const double* __restrict__ ctab) {
  long long total = N, stride = 1;
  for (int t = 1; t < d; ++t) total *= N;
  for (int t = 0; t < axis; ++t) stride *= N;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < total;
       o += (long long)gridDim.x * blockDim.x) {
    const int j = (int)((o / stride) % N);
    const long long base = o - (long long)j * stride;
    const double* c = ctab + (long long)j * N;
    double acc = 0.0;
    for (int i = 0; i < N; ++i) acc = fma(in[base + i * stride], c[i], acc);
    out[o] = acc;
  }
}

// full[(kz' N + ky') N + kx'] = B[k restricted to d dims] / N^d * prod_t dec_t(k_t').
__global__ void k_reg_full(const double* __restrict__ B, int N, int d,
                           const double* __restrict__ dec, double scale, float* __restrict__ full) {
  const long long total = (long long)N * N * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(i % N), ky = (int)((i / N) % N), kz = (int)(i / ((long long)N * N));
    const double f = dec[kx] * dec[N + ky] * dec[2 * N + kz];
    long long bi = kx;
    if (d >= 2) bi += (long long)N * ky;
    if (d >= 3) bi += (long long)N * N * kz;
    full[i] = f == 0.0 ? 0.f : (float)(B[bi] * scale * f);
  }
}

// m[kx'] = scale * sum over the other indices of B: the coefficients of the
// trigonometric polynomial restricted to the first axis (its values there).
__global__ void k_reg_marginal(const double* __restrict__ B, int N, int d, double scale,
                               double* __restrict__ out) {
  __shared__ double sh[256];
  long long others = 1;
  for (int t = 1; t < d; ++t) others *= N;
  const int kx = blockIdx.x;
  double acc = 0.0;
  for (long long o = threadIdx.x; o < others; o += blockDim.x) acc += B[kx + (long long)N * o];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[kx] = sh[0] * scale;
}

struct NearArgs {
  float e[REG_MAXP];   // T_I = sum_q e[q] u^q, u = r2 / r2i (grid units)
  int P;
  float r2i;           // (eps_I n)^2: the near-field radius squared in grid units
  float inv_r2i;
  float c1, c2;        // kernel constants for r2 in grid units (see k_near)
  int tiles1, R;
};

// Decoded grid-unit position of a binned point (cell + fraction).
__device__ __forceinline__ void grid_pos(const int4 c, float& x, float& y, float& z) {
  x = (float)(c.x & 1023) + __int_as_float(c.y);
  y = (float)((c.x >> 10) & 1023) + __int_as_float(c.z);
  z = (float)((c.x >> 20) & 1023) + __int_as_float(c.w);
}

// K at squared grid distance r2 (r = sqrt(r2) h/n):
//   laplace exp2(c1 sqrt(r2)), c1 = -(h/n) log2(e) / p;  imq rsqrt(c1 r2 + c2),
//   c1 = (h/n)^2, c2 = p^2;  energy -c1 sqrt(r2), c1 = h/n.
template <int KIND>
__device__ __forceinline__ float near_kernel(float r2, float c1, float c2) {
  if (KIND == UOTK_KERNEL_LAPLACE) return ex2_approx(c1 * sqrtf(r2));
  if (KIND == UOTK_KERNEL_IMQ) return rsqrtf(fmaf(c1, r2, c2));
  return -c1 * sqrtf(r2);
}

// Work items of the near field: (target tile, first target) for every chunk of
// NFFT_NEAR_CHUNK targets of a non-empty tile, in any order.
__global__ void k_near_items(const int* __restrict__ ttile, int tiles, int2* __restrict__ items,
                             int* __restrict__ ctr) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tiles; t += gridDim.x * blockDim.x) {
    const int b = ttile[t], e = ttile[t + 1];
    if (b == e) continue;
    const int k = (e - b + NFFT_NEAR_CHUNK - 1) / NFFT_NEAR_CHUNK;
    const int base = atomicAdd(&ctr[0], k);
    for (int i = 0; i < k; ++i) items[base + i] = make_int2(t, b + i * NFFT_NEAR_CHUNK);
  }
}

// Persistent CTAs take work items from a counter: each item is up to
// NFFT_NEAR_CHUNK targets of one tile, NEAR_TPT per thread; the sources of the
// (2R+1)^3 neighbouring tiles, contiguous per (z, y) row of tiles in sorted
// order, are staged through shared memory.  T_I has P coefficients held in
// registers (P = 12 serves any p <= 12, the unused coefficients being zero).
constexpr int NEAR_TPT = 4;
static_assert(NEAR_TPT * NEAR_THREADS == NFFT_NEAR_CHUNK, "one pass per work item");
template <int KIND, int P>
__global__ void __launch_bounds__(NEAR_THREADS)
    k_near(const int4* __restrict__ tcell, const int* __restrict__ ttile,
           const int4* __restrict__ scell, const int* __restrict__ stile,
           const float* __restrict__ w, const int2* __restrict__ items,
           int* __restrict__ ctr, NearArgs a, float* __restrict__ out) {
  __shared__ float4 sh[NEAR_THREADS];
  __shared__ int item;
  float e[P];
#pragma unroll
  for (int q = 0; q < P; ++q) e[q] = a.e[q];
  const float r2i = a.r2i, inv_r2i = a.inv_r2i, c1 = a.c1, c2 = a.c2;
  const int T = a.tiles1, R = a.R;
  const int nitems = ctr[0];
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(&ctr[1], 1);
    __syncthreads();
    const int li = item;
    __syncthreads();
    if (li >= nitems) break;
    const int2 it = items[li];
    const int tile = it.x;
    const int te = min(it.y + NFFT_NEAR_CHUNK, ttile[tile + 1]);
    const int tx = tile % T, ty = (tile / T) % T, tz = tile / (T * T);
    {
      const int t0 = it.y;
      float px[NEAR_TPT], py[NEAR_TPT], pz[NEAR_TPT], acc[NEAR_TPT];
#pragma unroll
      for (int q = 0; q < NEAR_TPT; ++q) {
        const int i = t0 + threadIdx.x + q * NEAR_THREADS;
        px[q] = py[q] = pz[q] = 1e18f;   // far from every source
        acc[q] = 0.f;
        if (i < te) grid_pos(tcell[i], px[q], py[q], pz[q]);
      }
      for (int dz = -R; dz <= R; ++dz) {
        const int z = tz + dz;
        if (z < 0 || z >= T) continue;
        for (int dy = -R; dy <= R; ++dy) {
          const int y = ty + dy;
          if (y < 0 || y >= T) continue;
          const int x0 = max(tx - R, 0), x1 = min(tx + R, T - 1);
          const int row = (z * T + y) * T;
          const int sb = stile[row + x0], se = stile[row + x1 + 1];
          for (int s0 = sb; s0 < se; s0 += NEAR_THREADS) {
            __syncthreads();
            const int j = s0 + threadIdx.x;
            if (j < se) {
              float x, yy, zz;
              grid_pos(scell[j], x, yy, zz);
              sh[threadIdx.x] = make_float4(x, yy, zz, w[j]);
            }
            __syncthreads();
            const int cnt = min(NEAR_THREADS, se - s0);
            for (int k = 0; k < cnt; ++k) {
              const float4 s = sh[k];
#pragma unroll
              for (int q = 0; q < NEAR_TPT; ++q) {
                const float dx = px[q] - s.x, dy2 = py[q] - s.y, dz2 = pz[q] - s.z;
                const float r2 = fmaf(dx, dx, fmaf(dy2, dy2, dz2 * dz2));
                if (r2 < r2i) {
                  const float u = r2 * inv_r2i;
                  float ti = e[P - 1];
#pragma unroll
                  for (int j2 = P - 2; j2 >= 0; --j2) ti = fmaf(ti, u, e[j2]);
                  acc[q] = fmaf(s.w, near_kernel<KIND>(r2, c1, c2) - ti, acc[q]);
                }
              }
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < NEAR_TPT; ++q) {
        const int i = t0 + threadIdx.x + q * NEAR_THREADS;
        if (i < te) out[i] += acc[q];
      }
    }
  }
}

template <int KIND>
void launch_near(int P, int blocks, cudaStream_t s, const NfftPoints& src, const float* w,
                 const NfftPoints& tgt, const NfftWork& W, const NearArgs& a, float* out) {
#define UOTK_NEAR_ARGS tgt.cell, tgt.tile_start, src.cell, src.tile_start, w, W.near_items, \
                       W.near_ctr, a, out
  switch (P) {
    case 4: k_near<KIND, 4><<<blocks, NEAR_THREADS, 0, s>>>(UOTK_NEAR_ARGS); break;
    case 6: k_near<KIND, 6><<<blocks, NEAR_THREADS, 0, s>>>(UOTK_NEAR_ARGS); break;
    case 8: k_near<KIND, 8><<<blocks, NEAR_THREADS, 0, s>>>(UOTK_NEAR_ARGS); break;
    default: k_near<KIND, REG_MAXP><<<blocks, NEAR_THREADS, 0, s>>>(UOTK_NEAR_ARGS); break;
  }
#undef UOTK_NEAR_ARGS
}

}  // namespace

uotk_status nfft_reg_table(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P, NfftWork& W) {
  const RegPoly R = make_reg_poly(P);
  const int N = P.N, d = P.d;
  long long nd = N;
  for (int t = 1; t < d; ++t) nd *= N;
  // FP64 scratch inside the complex work grid (>= 6 N^3 floats2 > 2 N^d + N^2 + 3N doubles)
  double* A = reinterpret_cast<double*>(W.cgrid);
  double* B = A + nd;
  double* ctab = B + nd;
  double* dec = ctab + (size_t)N * N;
  std::vector<double> h(N * N + 3 * N);
  for (int j = 0; j < N; ++j)
    for (int i = 0; i < N; ++i)
      h[(size_t)j * N + i] = cos(2.0 * M_PI * (double)(j - N / 2) * (double)(i - N / 2) / N);
  nfft_deconv_rows(P, h.data() + (size_t)N * N);
  UOTK_PROF(ctx, s, "reg_table");
  UOTK_CUDA(ctx, cudaMemcpyAsync(ctab, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice,
                                 s));
  k_reg_samples<<<grid_for(ctx, nd, 256), 256, 0, s>>>(R, N, d, A);
  UOTK_LAUNCHED(ctx);
  double* cur = A;
  double* nxt = B;
  for (int axis = 0; axis < d; ++axis) {
    k_dct_axis<<<grid_for(ctx, nd, 256), 256, 0, s>>>(cur, nxt, N, d, axis, ctab);
    UOTK_LAUNCHED(ctx);
    double* t = cur;
    cur = nxt;
    nxt = t;
  }
  k_reg_full<<<grid_for(ctx, (long long)N * N * N, 256), 256, 0, s>>>(cur, N, d, dec,
                                                                      1.0 / (double)nd, W.full);
  UOTK_LAUNCHED(ctx);
  // Self-check of the Fourier approximation: on the first axis the series is
  // sum_k m_k cos(2 pi k t); it interpolates K_R at the grid points t = l/N, so
  // compare it with K_R halfway between them, over the radii pairs can have.
  k_reg_marginal<<<N, 256, 0, s>>>(cur, N, d, 1.0 / (double)nd, nxt);
  UOTK_LAUNCHED(ctx);
  std::vector<double> mk(N);
  UOTK_CUDA(ctx, cudaMemcpyAsync(mk.data(), nxt, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  // the pageable vectors must outlive the copies
  UOTK_CUDA(ctx, cudaStreamSynchronize(s));
  // Error bound per unit weight, relative to max |K| over the radii pairs can
  // have (K itself, not K_R: the near field restores K there).
  double err = 0.0, kmax = 0.0;
  for (int l = 0; l < N / 2; ++l) {
    const double t = (l + 0.5) / N;
    if (t > 0.5 - R.eps_b) break;
    double f = 0.0;
    for (int i = 0; i < N; ++i) f += mk[i] * cos(2.0 * M_PI * (double)(i - N / 2) * t);
    err = fmax(err, fabs(f - reg_kernel(R, t)));
  }
  for (int l = 0; l <= 256; ++l) {
    const double r = R.h * (0.5 - R.eps_b) * l / 256.0;
    double c[1];
    kernel_taylor(R.kind, R.par, r, 1, c);
    kmax = fmax(kmax, fabs(c[0]));
  }
  const double rel = kmax > 0.0 ? err / kmax : err;
  if (!(rel <= P.reg_target))
    return set_error(ctx, UOTK_ERR_UNSUPPORTED,
                     "NFFT: the regularised kernel (p = %d, bandwidth %d, period %g, parameter %g) "
                     "misses the accuracy goal: estimated error %.1e > %.1e; raise the grid or "
                     "the regularisation degree, or use the direct form",
                     P.reg_p, N, P.h, P.eps, rel, P.reg_target);
  return UOTK_OK;
}

uotk_status nfft_near(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P, const NfftPoints& src,
                      const float* w, const NfftPoints& tgt, NfftWork& W, float* out) {
  if (src.n == 0 || tgt.n == 0) return UOTK_OK;
  const RegPoly R = make_reg_poly(P);
  NearArgs a{};
  a.P = R.P;
  for (int q = 0; q < R.P; ++q) a.e[q] = (float)R.ti[q];
  const double rad = P.eps_i * P.n;  // grid units
  a.r2i = (float)(rad * rad);
  a.inv_r2i = (float)(1.0 / (rad * rad));
  const double hn = P.h / P.n;
  if (P.kernel == UOTK_KERNEL_LAPLACE) {
    a.c1 = (float)(-hn * 1.4426950408889634 / P.eps);
  } else if (P.kernel == UOTK_KERNEL_IMQ) {
    a.c1 = (float)(hn * hn);
    a.c2 = (float)(P.eps * P.eps);
  } else {
    a.c1 = (float)hn;
  }
  a.tiles1 = P.tiles1;
  a.R = (int)ceil(rad / NFFT_TILE);
  const int tiles = P.tiles1 * P.tiles1 * P.tiles1;
  const int blocks = 5 * ctx->num_sms;   // resident CTAs (43 registers x 256 threads)
  UOTK_PROF(ctx, s, "near");
  UOTK_CUDA(ctx, cudaMemsetAsync(W.near_ctr, 0, 2 * sizeof(int), s));
  k_near_items<<<grid_for(ctx, tiles, 256), 256, 0, s>>>(tgt.tile_start, tiles, W.near_items,
                                                         W.near_ctr);
  UOTK_LAUNCHED(ctx);
  switch (P.kernel) {
    case UOTK_KERNEL_LAPLACE:
      launch_near<UOTK_KERNEL_LAPLACE>(a.P, blocks, s, src, w, tgt, W, a, out);
      break;
    case UOTK_KERNEL_IMQ:
      launch_near<UOTK_KERNEL_IMQ>(a.P, blocks, s, src, w, tgt, W, a, out);
      break;
    default:
      launch_near<UOTK_KERNEL_ENERGY>(a.P, blocks, s, src, w, tgt, W, a, out);
      break;
  }
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

}  // namespace uotk

// C ABI, plan lifecycle, set-up pipeline, the V-cycle (Algorithm 7) and the
// outer PCG (Algorithm 8, FP64) or its mixed-precision flexible variant.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "sps_internal.h"

namespace sps {

static thread_local std::string g_last_error = "no error";
static std::atomic<unsigned long long> g_launches{0};

void count_launches(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
  return SPS_ECUDA;
}

namespace {

// scalar slots in plan->scal
constexpr int S_RZ_A = 0, S_PV = 2, S_RR = 3, S_W = 4, S_FLAG = 6, S_RZ_B = 8, S_TMP = 10, S_TMP2 = 12;
constexpr int NSCAL = 96;   // slots 16..31 belong to the inner coarse CG (grid_ops.cu)
constexpr int LZ_MAX = 32, LZ_A = 32, LZ_B = 64;   // Lanczos coefficients alpha_j, beta_j^2 (estimate_omega)

// ---- exact 1-D Gram matrices of the cubic B-splines --------------------------
// Piece m of the uniform cubic B-spline on one cell, as monomial coefficients
// in the local coordinate t: basis function (cell + m) restricted to the cell.
const double kPiece[4][4] = {{1.0 / 6, -3.0 / 6, 3.0 / 6, -1.0 / 6},
                             {4.0 / 6, 0.0, -6.0 / 6, 3.0 / 6},
                             {1.0 / 6, 3.0 / 6, 3.0 / 6, -3.0 / 6},
                             {0.0, 0.0, 0.0, 1.0 / 6}};

// E_r[a][b] = int_0^1 d^r piece_a * d^r piece_b dt, exact (monomial integrals).
void element_matrix(int r, double E[4][4]) {
  double d[4][4];
  for (int m = 0; m < 4; ++m) {
    double c[4];
    for (int k = 0; k < 4; ++k) c[k] = kPiece[m][k];
    for (int s = 0; s < r; ++s) {
      for (int k = 0; k < 3; ++k) c[k] = (k + 1) * c[k + 1];
      c[3] = 0.0;
    }
    for (int k = 0; k < 4; ++k) d[m][k] = c[k];
  }
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      double s = 0.0;
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) s += d[a][i] * d[b][j] / (double)(i + j + 1);
      E[a][b] = s;
    }
}

// Band of Psi_r on [lo, hi] with N cells: band[j][o + q] = Psi_r[j, j + o].
// The Gram matrix is the sum over the cells of the domain of the element
// matrix (Section 2.4, Gramian of the r-th derivatives), scaled by h^(1-2r).
void gram_band(int N, double h, int r, double* band) {
  double E[4][4];
  element_matrix(r, E);
  const double sc = std::pow(h, 1.0 - 2.0 * r);
  const int J = N + Q;
  for (int j = 0; j < J; ++j)
    for (int o = -Q; o <= Q; ++o) {
      const int l = j + o;
      double s = 0.0;
      if (l >= 0 && l < J) {
        const int c0 = std::max(0, std::max(j - Q, l - Q));
        const int c1 = std::min(N - 1, std::min(j, l));
        for (int c = c0; c <= c1; ++c) s += E[j - c][l - c];
      }
      band[(long long)j * BAND + o + Q] = s * sc;
    }
}

void free_points(sps_plan* pl) {
  if (pl->x32_sorted != pl->x_sorted) pfree(pl, pl->x32_sorted);
  pl->x32_sorted = nullptr;
  pfree(pl, pl->x_sorted);
  pfree(pl, pl->y_sorted);
  pfree(pl, pl->keys);
  pfree(pl, pl->keys_tmp);
  pfree(pl, pl->perm);
  pfree(pl, pl->perm_tmp);
  pl->n_cap = 0;
}


__global__ void k_hash_fill(double* x, long long n, unsigned long long seed) {
  // SplitMix64 (Steele, Lea, Flood 2014) in counter mode, mapped to [-1, 1).
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

__global__ void k_sqrt_copy(double* out, const double* in, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = sqrt(in[i]);
}

// x = y / sqrt(scal[slot])
__global__ void k_normalize(double* x, const double* y, long long n, const double* scal, int slot) {
  const double s = 1.0 / sqrt(scal[slot]);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = y[i] * s;
}

// Lanczos step: w -= alpha_j q + beta_{j-1} qp (beta_{j-1} = sqrt(scal[bslot]), none when bslot < 0)
__global__ void k_lanczos_orth(double* w, const double* q, const double* qp, long long n, const double* scal,
                               int aslot, int bslot) {
  const double a = scal[aslot];
  const double b = bslot >= 0 ? sqrt(fmax(scal[bslot], 0.0)) : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    w[i] = w[i] - a * q[i] - b * qp[i];
}

// qp <- q; q <- w / beta_j (q <- 0 when beta_j vanishes: the Krylov space is invariant)
__global__ void k_lanczos_next(double* qp, double* q, const double* w, long long n, const double* scal, int bslot) {
  const double b2 = scal[bslot];
  const double inv = b2 > 1e-300 ? 1.0 / sqrt(b2) : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    qp[i] = q[i];
    q[i] = w[i] * inv;
  }
}

__global__ void k_mul(double* out, const double* a, const double* b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = a[i] * b[i];
}

template <typename T>
__global__ void k_fma_probe(T* out, int iters, T seed) {
  T a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = seed + T(k) * T(1e-3) + T(threadIdx.x) * T(1e-7);
  const T m = T(0.999999), c = T(1e-6);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == T(-12345)) out[0] = s;   // keeps the loop alive
}

cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

long long max_K(const sps_plan* pl) {
  long long m = 0;
  for (int g = 0; g < pl->G; ++g) m = std::max(m, pl->lev[g].geom.K);
  return m;
}

int read_scalars(sps_plan* pl, cudaStream_t st) {
  SPS_CUDA(cudaMemcpyAsync(pl->host_scal, pl->scal, sizeof(double) * NSCAL, cudaMemcpyDeviceToHost, st));
  SPS_CUDA(cudaStreamSynchronize(st));
  return SPS_OK;
}

int copy_in(double* dst, const double* src, long long n, int mem, cudaStream_t st) {
  SPS_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * n,
                           mem == SPS_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
  return SPS_OK;
}

int copy_out(double* dst, const double* src, long long n, int mem, cudaStream_t st) {
  SPS_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * n,
                           mem == SPS_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
  if (mem == SPS_MEM_HOST) SPS_CUDA(cudaStreamSynchronize(st));
  return SPS_OK;
}

}  // namespace

// ---- device memory of a plan ----------------------------------------------------
int plan_alloc(sps_plan* pl, void** p, size_t bytes) {
  *p = nullptr;
  if (pl->opt.max_device_bytes > 0 && pl->dev_bytes + (long long)bytes > (long long)pl->opt.max_device_bytes) {
    set_error("the plan's device memory limit (sps_options.max_device_bytes) would be exceeded");
    return SPS_ENOMEM;
  }
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error("device allocation failed");
    return SPS_ENOMEM;
  }
  pl->dev_sizes[*p] = bytes;
  pl->dev_bytes += (long long)bytes;
  return SPS_OK;
}

void plan_free(sps_plan* pl, void* p) {
  if (!p) return;
  auto it = pl->dev_sizes.find(p);
  if (it != pl->dev_sizes.end()) {
    pl->dev_bytes -= (long long)it->second;
    pl->dev_sizes.erase(it);
  }
  cudaFree(p);
}

int check_device_errors(sps_plan* pl, cudaStream_t st) {
  int flags = 0;
  SPS_CUDA(cudaMemcpyAsync(&flags, pl->err_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  SPS_CUDA(cudaStreamSynchronize(st));
  if (flags & ERR_SMEM) {
    SPS_CUDA(cudaMemsetAsync(pl->err_flag, 0, sizeof(int), st));
    set_error("internal error: the point operator's staged points exceeded its shared memory (work skipped)");
    return SPS_EINTERNAL;
  }
  if (flags & ERR_WAIT) {
    SPS_CUDA(cudaMemsetAsync(pl->err_flag, 0, sizeof(int), st));
    set_error("internal error: the point operator's asynchronous copies did not complete in time (work skipped)");
    return SPS_EINTERNAL;
  }
  return SPS_OK;
}

// ---- operator on one level: u = (Phi_g'Phi_g + lambda Lambda_g) v --------------
template <typename T>
int apply_level(sps_plan* pl, int g, const T* v, T* u, cudaStream_t st) {
  const Level& L = pl->lev[g - 1];
  if ((sizeof(T) == 8 && L.st_d) || (sizeof(T) == 4 && L.st_f))
    return stencil_apply<T>(pl, g, v, u, st);             // assembled coarse level
  SPS_TRY(penalty_apply<T>(pl, g, v, u, pl->lam, st));    // u = lambda Lambda v
  return point_op<T>(pl, g, PT_APPLY, v, u, st);          // u += Phi'Phi v
}
template int apply_level<double>(sps_plan*, int, const double*, double*, cudaStream_t);
template int apply_level<float>(sps_plan*, int, const float*, float*, cudaStream_t);

// ---- Algorithm 7 from alpha = 0: xG = V(bG) -------------------------------------
template <typename T>
int vcycle_into(sps_plan* pl, const T* bG, T* xG, cudaStream_t st) {
  const int G = pl->G;
  const int nu1 = pl->opt.nu1, nu2 = pl->opt.nu2;
  auto B = [&](int g) -> T* { return g == G ? const_cast<T*>(bG) : vecs<T>(pl->lev[g - 1]).b; };
  auto X = [&](int g) -> T* { return g == G ? xG : vecs<T>(pl->lev[g - 1]).alpha; };
  for (int g = G; g >= 2; --g) {
    Level& L = pl->lev[g - 1];
    LevelVecs<T>& V = vecs<T>(L);
    const long long K = L.geom.K;
    const T om = T(L.omega);
    if (nu1 >= 1) {
      SPS_TRY(vec_scale_mul<T>(X(g), V.dinv, B(g), om, K, st));        // first sweep from alpha = 0
      for (int s = 1; s < nu1; ++s) {
        SPS_TRY(apply_level<T>(pl, g, X(g), V.u, st));
        SPS_TRY(vec_jacobi<T>(X(g), V.dinv, B(g), V.u, om, K, st));
      }
      SPS_TRY(apply_level<T>(pl, g, X(g), V.u, st));                  // r = A alpha - b
    } else {
      SPS_CUDA(cudaMemsetAsync(X(g), 0, sizeof(T) * K, st));
      SPS_CUDA(cudaMemsetAsync(V.u, 0, sizeof(T) * K, st));
    }
    SPS_TRY(restrict_res<T>(pl, g, V.u, B(g), B(g - 1), st));         // b_{g-1} = I'(A alpha - b)
  }
  if (pl->opt.coarse_cg) {                                            // e ~ A_1^{-1} r by inner CG
    T* t6 = sizeof(T) == 8 ? (T*)pl->dtmp[6] : (T*)pl->ftmp[6];
    T* t7 = sizeof(T) == 8 ? (T*)pl->dtmp[7] : (T*)pl->ftmp[7];
    SPS_TRY(coarse_cg<T>(pl, B(1), X(1), t6, t7, st));
  } else {
    SPS_TRY(coarse_solve<T>(pl, B(1), X(1), st));                     // e = A_1^{-1} r
  }
  for (int g = 2; g <= G; ++g) {
    Level& L = pl->lev[g - 1];
    LevelVecs<T>& V = vecs<T>(L);
    const long long K = L.geom.K;
    const T om = T(L.omega);
    SPS_TRY(prolong_sub<T>(pl, g, X(g - 1), X(g), 1, st));            // alpha <- alpha - I e
    for (int s = 0; s < nu2; ++s) {
      SPS_TRY(apply_level<T>(pl, g, X(g), V.u, st));
      SPS_TRY(vec_jacobi<T>(X(g), V.dinv, B(g), V.u, om, K, st));
    }
  }
  return SPS_OK;
}

namespace {

// Largest eigenvalue of the symmetric tridiagonal matrix with diagonal a and
// off-diagonal b (b[j] couples j and j + 1), by bisection on the Sturm count,
// and the last component of its unit eigenvector by inverse iteration.
void tridiag_top(const std::vector<double>& a, const std::vector<double>& b, double* theta, double* s_last) {
  const int m = (int)a.size();
  double lo = a[0], hi = a[0];
  for (int j = 0; j < m; ++j) {
    const double r = (j > 0 ? std::fabs(b[j - 1]) : 0.0) + (j + 1 < m ? std::fabs(b[j]) : 0.0);
    lo = std::min(lo, a[j] - r);
    hi = std::max(hi, a[j] + r);
  }
  const double tiny = 1e-300;
  auto below = [&](double x) {   // number of eigenvalues < x (LDL' pivots of T - x I)
    int c = 0;
    double d = 1.0;
    for (int j = 0; j < m; ++j) {
      d = a[j] - x - (j > 0 ? b[j - 1] * b[j - 1] / d : 0.0);
      if (d == 0.0) d = -tiny;
      if (d < 0.0) ++c;
    }
    return c;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(std::fabs(hi), std::fabs(lo)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (below(mid) == m) hi = mid;   // every eigenvalue below mid
    else lo = mid;
  }
  *theta = hi;
  // inverse iteration: (T - sigma I) x = x_prev with sigma just above theta
  const double sigma = hi + 1e-10 * std::max(std::fabs(hi), 1e-30);
  std::vector<double> x(m, 1.0), c(m), d(m);
  for (int rep = 0; rep < 3; ++rep) {
    // Thomas algorithm on the tridiagonal system
    double piv = a[0] - sigma;
    if (std::fabs(piv) < tiny) piv = -tiny;
    c[0] = m > 1 ? b[0] / piv : 0.0;
    d[0] = x[0] / piv;
    for (int j = 1; j < m; ++j) {
      piv = a[j] - sigma - b[j - 1] * c[j - 1];
      if (std::fabs(piv) < tiny) piv = -tiny;
      c[j] = j + 1 < m ? b[j] / piv : 0.0;
      d[j] = (x[j] - b[j - 1] * d[j - 1]) / piv;
    }
    x[m - 1] = d[m - 1];
    for (int j = m - 2; j >= 0; --j) x[j] = d[j] - c[j] * x[j + 1];
    double nrm = 0.0;
    for (int j = 0; j < m; ++j) nrm += x[j] * x[j];
    nrm = std::sqrt(nrm);
    if (!(nrm > 0.0) || !std::isfinite(nrm)) break;
    for (int j = 0; j < m; ++j) x[j] /= nrm;
  }
  *s_last = std::isfinite(x[m - 1]) ? std::fabs(x[m - 1]) : 1.0;
}

// From m Lanczos coefficients alpha_j and beta_j^2: theta, the top Ritz value
// (top eigenvalue of the tridiagonal T_m), and lambda_hat = theta +
// beta_{m-1} |s_m| with s the unit eigenvector of T_m for theta.  False when a
// coefficient is not finite or theta is not positive.
bool lanczos_lambda_hat(const double* alpha, const double* beta2, int m, double* theta, double* lambda_hat) {
  std::vector<double> a(m), b(m);
  bool finite = true;
  for (int j = 0; j < m; ++j) {
    a[j] = alpha[j];
    b[j] = std::sqrt(std::max(beta2[j], 0.0));
    finite = finite && std::isfinite(a[j]) && std::isfinite(beta2[j]);
  }
  if (!finite) return false;
  double s_last = 1.0;
  tridiag_top(a, b, theta, &s_last);
  *lambda_hat = *theta + b[m - 1] * s_last;
  return *theta > 0.0 && std::isfinite(*lambda_hat);
}

// omega_g lambda_hat: the damping of the Jacobi smoother relative to the
// estimate of lambda_max(D_g^-1 A_g).  Below 2 the damped Jacobi sweep, and
// with nu1 = nu2 the V-cycle, stay symmetric positive definite.
constexpr double OMEGA_LMAX = 1.8;

// Largest eigenvalue of D_g^-1 A_g, i.e. of S = D^-1/2 A D^-1/2, by m
// Lanczos steps (FP32 operator on matrix-free levels, FP64 vectors and
// recurrences, no reorthogonalisation: the largest Ritz value converges
// first).  lambda_hat = theta + beta_m |s_m|, the top Ritz value of the
// tridiagonal T_m plus its residual bound, so that lambda_hat bounds
// lambda_max once the top Ritz value has settled on it; omega_g =
// OMEGA_LMAX / lambda_hat.
int estimate_omega(sps_plan* pl, int g, cudaStream_t st) {
  Level& L = pl->lev[g - 1];
  const long long K = L.geom.K;
  const int blocks = grid_blocks(K, 256);
  double* q = L.d.alpha;      // q_j
  double* w = L.d.u;          // S q_j, then the next Lanczos direction
  double* s = L.d.b;          // D^-1/2
  double* qp = pl->dtmp[7];   // q_{j-1}
  const int m = std::min(std::max(pl->opt.power_iters, 1), LZ_MAX);
  k_sqrt_copy<<<blocks, 256, 0, st>>>(s, L.d.dinv, K);
  k_hash_fill<<<blocks, 256, 0, st>>>(q, K, 0x5EEDull + (unsigned long long)g);
  SPS_CHECK_LAUNCH("Lanczos init");
  SPS_TRY(dot(pl, q, q, K, S_TMP, st));
  k_normalize<<<blocks, 256, 0, st>>>(q, q, K, pl->scal, S_TMP);
  SPS_CUDA(cudaMemsetAsync(qp, 0, sizeof(double) * K, st));
  for (int j = 0; j < m; ++j) {
    k_mul<<<blocks, 256, 0, st>>>(w, s, q, K);
    if (L.st_d) {   // assembled FP64 level: its stencil product is the cheapest apply
      SPS_TRY(apply_level<double>(pl, g, w, pl->dtmp[6], st));
      k_mul<<<blocks, 256, 0, st>>>(w, s, pl->dtmp[6], K);
    } else {
      SPS_TRY(vec_cast_d2f(L.f.alpha, w, K, st));
      SPS_TRY(apply_level<float>(pl, g, L.f.alpha, L.f.u, st));
      SPS_TRY(vec_cast_f2d(w, L.f.u, K, st));
      k_mul<<<blocks, 256, 0, st>>>(w, s, w, K);
    }
    SPS_TRY(dot(pl, q, w, K, LZ_A + j, st));   // alpha_j = q_j' S q_j
    k_lanczos_orth<<<blocks, 256, 0, st>>>(w, q, qp, K, pl->scal, LZ_A + j, j > 0 ? LZ_B + j - 1 : -1);
    SPS_TRY(dot(pl, w, w, K, LZ_B + j, st));   // beta_j^2
    k_lanczos_next<<<blocks, 256, 0, st>>>(qp, q, w, K, pl->scal, LZ_B + j);
    SPS_CHECK_LAUNCH("Lanczos step");
  }
  SPS_TRY(read_scalars(pl, st));
  double theta = 0.0, lmax = 0.0;
  if (!lanczos_lambda_hat(pl->host_scal + LZ_A, pl->host_scal + LZ_B, m, &theta, &lmax)) {
    set_error("Lanczos estimate of lambda_max for the Jacobi damping failed");
    return SPS_EBREAKDOWN;
  }
  L.omega = OMEGA_LMAX / lmax;
  return SPS_OK;
}

// Levels strictly between the coarsest and the finest are assembled in
// stencil form when one sparse matrix-vector product over the (2q+1)^P
// stencil moves fewer bytes than the point sweep costs in arithmetic:
//   S K_g sizeof(T) / (0.6 * 6.8 TB/s)  <  n * 2 (q+1)^P / (0.3 * FMA rate of T),
// with a budget of 8 GB per level.  The assembled matrix is exactly A_g
// (same sums, another order), so the method is unchanged; the finest level
// always stays matrix free.
int assemble_coarse_levels(sps_plan* pl, cudaStream_t st) {
  if (!pl->opt.hybrid) return SPS_OK;
  const int P = pl->P;
  long long S = 1, loc = 1;
  for (int p = 0; p < P; ++p) {
    S *= BAND;
    loc *= Q + 1;
  }
  const bool mixed = pl->opt.precision == SPS_PREC_MIXED;
  const double tsize = mixed ? 4.0 : 8.0;
  const double rate = mixed ? 38.7e12 : 0.53e12;
  for (int g = 2; g < pl->G; ++g) {
    Level& L = pl->lev[g - 1];
    const long long K = L.geom.K;
    const double spmv_s = (double)S * K * tsize / (0.6 * 6.8e12);
    const double sweep_s = (double)pl->n * 2.0 * loc / (0.3 * rate);
    const bool want = spmv_s < sweep_s && (double)S * K * 8.0 <= 8e9;
    if (!want) {
      pfree(pl, L.st_d);
      pfree(pl, L.st_f);
      continue;
    }
    L.S = (int)S;
    if (!L.st_d) SPS_TRY(palloc(pl, &L.st_d, S * K));
    if (mixed && !L.st_f) SPS_TRY(palloc(pl, &L.st_f, S * K));
    SPS_TRY(stencil_assemble(pl, g, st));
    if (mixed) {   // the FP32 V-cycle reads the FP32 copy only
      pfree(pl, L.st_d);
    }
  }
  return SPS_OK;
}

int check_plan_points(const sps_plan* pl) {
  if (!pl) {
    set_error("null plan");
    return SPS_EINVAL;
  }
  if (!pl->have_points) {
    set_error("sps_set_points has not been called");
    return SPS_ESTATE;
  }
  return SPS_OK;
}

// ---- one PCG iteration as a CUDA graph -------------------------------------
// The body of an iteration after the first -- V-cycle, the dot products and
// direction update of Algorithm 8, then the next operator apply and vector
// updates, and the copy of the scalars to pinned host memory -- is captured
// once per set-up and replayed; the host only checks the residual between
// replays.  Scalar slots are fixed (r'z of the new iteration is copied over the
// old one inside the body).
template <typename Body>
int run_iteration(sps_plan* pl, int which, Body&& body, cudaStream_t st) {
  sps_plan::IterGraph& gr = pl->graph[which];
  if (!pl->opt.graphs) {
    SPS_TRY(body(st));
    SPS_CUDA(cudaStreamSynchronize(st));
    return SPS_OK;
  }
  const bool prof = profile_active();
  if (!gr.exec || gr.gen != pl->gen || gr.profiled != prof) {
    if (gr.exec) cudaGraphExecDestroy(gr.exec);
    gr.exec = nullptr;
    if (!pl->cap_stream) SPS_CUDA(cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking));
    SPS_CUDA(cudaStreamSynchronize(st));
    const int first = profile_mark();
    cudaGraph_t g;
    const unsigned long long l0 = g_launches.load();
    SPS_CUDA(cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = body(pl->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(pl->cap_stream, &g);
    // captured kernels run at each replay, not now: count them per replay
    gr.nlaunch = g_launches.load() - l0;
    g_launches.fetch_sub(gr.nlaunch);
    if (rc != SPS_OK) return rc;
    if (ce != cudaSuccess) return cuda_fail(ce, "graph capture");
    ce = cudaGraphInstantiate(&gr.exec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return cuda_fail(ce, "graph instantiate");
    gr.prof_first = first;
    gr.prof_last = profile_mark();
    profile_capture_end(gr.prof_first, gr.prof_last);
    gr.gen = pl->gen;
    gr.profiled = prof;
  }
  SPS_CUDA(cudaGraphLaunch(gr.exec, st));
  count_launches(gr.nlaunch);
  SPS_CUDA(cudaStreamSynchronize(st));
  if (prof) SPS_TRY(profile_harvest(gr.prof_first, gr.prof_last));
  return SPS_OK;
}

int solve_fp64(sps_plan* pl, double tol, sps_result* res, bool warm, cudaStream_t st) {
  const int G = pl->G;
  const long long K = pl->lev[G - 1].geom.K;
  const double nb = pl->rhs_norm;
  int it = 0;
  int status = SPS_OK;
  double rel = 1.0;
  // z = V(r) (Algorithm 7), or z = r for plain CG (the paper's comparison method)
  auto precondition64 = [&](cudaStream_t s) -> int {
    if (pl->opt.precondition) return vcycle_into<double>(pl, pl->r, pl->z, s);
    SPS_CUDA(cudaMemcpyAsync(pl->z, pl->r, sizeof(double) * K, cudaMemcpyDeviceToDevice, s));
    return SPS_OK;
  };
  auto restart = [&](bool have_x) -> int {
    if (have_x) {
      SPS_TRY(apply_level<double>(pl, G, pl->x, pl->v, st));
      SPS_TRY(vec_residual(pl->r, pl->rhs, pl->v, K, pl->scal, S_RR, pl, st));
      res->fp64_applies++;
    } else {
      SPS_CUDA(cudaMemsetAsync(pl->x, 0, sizeof(double) * K, st));
      SPS_CUDA(cudaMemcpyAsync(pl->r, pl->rhs, sizeof(double) * K, cudaMemcpyDeviceToDevice, st));
      SPS_TRY(dot(pl, pl->r, pl->r, K, S_RR, st));
    }
    SPS_TRY(precondition64(st));
    SPS_CUDA(cudaMemcpyAsync(pl->p, pl->z, sizeof(double) * K, cudaMemcpyDeviceToDevice, st));
    SPS_TRY(dot(pl, pl->r, pl->z, K, S_RZ_A, st));
    SPS_TRY(read_scalars(pl, st));
    rel = std::sqrt(pl->host_scal[S_RR]) / nb;
    return SPS_OK;
  };
  // v = A p; w = r'z / p'v; alpha += w p; r -= w v (Algorithm 8)
  auto half_apply = [&](cudaStream_t s) -> int {
    SPS_TRY(apply_level<double>(pl, G, pl->p, pl->v, s));
    SPS_TRY(dot(pl, pl->p, pl->v, K, S_PV, s));
    if (pl->opt.precondition && pl->opt.coarse_cg)   // r_prev for the flexible beta
      SPS_CUDA(cudaMemcpyAsync(pl->rprev, pl->r, sizeof(double) * K, cudaMemcpyDeviceToDevice, s));
    SPS_TRY(pcg_update_xr(pl, K, S_RZ_A, s));
    SPS_CUDA(cudaMemcpyAsync(pl->host_scal, pl->scal, sizeof(double) * NSCAL, cudaMemcpyDeviceToHost, s));
    return SPS_OK;
  };
  // z = V(r); beta = r'z / r~'z~ (Algorithm 8), or z'(r - r~) / r~'z~ (flexible,
  // when the inner coarse CG makes the V-cycle nonlinear); p = z + beta p;
  // then the next half_apply
  const bool flexible = pl->opt.precondition && pl->opt.coarse_cg;
  auto body = [&](cudaStream_t s) -> int {
    SPS_TRY(precondition64(s));
    if (flexible) SPS_TRY(dot2(pl, pl->z, pl->r, pl->rprev, K, S_RZ_B, s));   // z'r, z'r_prev
    else SPS_TRY(dot(pl, pl->r, pl->z, K, S_RZ_B, s));
    SPS_TRY(pcg_update_p(pl, K, S_RZ_B, S_RZ_A, flexible ? 1 : 0, s));
    SPS_CUDA(cudaMemcpyAsync(pl->scal + S_RZ_A, pl->scal + S_RZ_B, sizeof(double), cudaMemcpyDeviceToDevice, s));
    return half_apply(s);
  };
  SPS_CUDA(cudaMemsetAsync(pl->scal, 0, sizeof(double) * NSCAL, st));
  SPS_TRY(restart(warm));
  for (int round = 0; round < 4; ++round) {
    bool first = true;
    // !(rel <= tol): a non-finite residual does not count as converged
    while (!(rel <= tol) && std::isfinite(rel) && it < pl->opt.max_iter) {
      if (first) {
        SPS_TRY(half_apply(st));
        SPS_CUDA(cudaStreamSynchronize(st));
        first = false;
      } else {
        SPS_TRY(run_iteration(pl, 0, body, st));
      }
      res->fp64_applies++;
      ++it;
      if (pl->host_scal[S_FLAG] != 0.0) {
        status = SPS_EBREAKDOWN;
        break;
      }
      rel = std::sqrt(pl->host_scal[S_RR]) / nb;
    }
    if (status != SPS_OK) break;
    // true residual in FP64; iterate on if the recursion drifted
    SPS_TRY(apply_level<double>(pl, G, pl->x, pl->v, st));
    SPS_TRY(vec_residual(pl->z, pl->rhs, pl->v, K, pl->scal, S_TMP, pl, st));
    SPS_TRY(read_scalars(pl, st));
    res->rel_res_true = std::sqrt(pl->host_scal[S_TMP]) / nb;
    if (res->rel_res_true <= tol || it >= pl->opt.max_iter || !std::isfinite(res->rel_res_true)) break;
    SPS_TRY(restart(true));
  }
  res->iterations = it;
  res->rel_res = rel;
  if (status == SPS_OK && !(res->rel_res_true <= tol)) status = SPS_ENOCONV;
  res->status = status;
  return status;
}

// Flexible PCG (Polak-Ribiere beta, Notay 2000) in FP64 with the FP32 V-cycle
// and FP32 point operator; the FP64 residual b - A alpha is recomputed when
// the recursive residual has dropped by replace_ratio (reliable updates).
// When the FP32 outer operator breaks the iteration down (p'A p <= 0 or a
// non-finite step: the system is too ill-conditioned for FP32 to resolve), the
// solve restarts from the current iterate with the FP64 residual and goes on
// with the FP64 outer operator (the V-cycle stays FP32); a breakdown after
// that is reported.
int solve_mixed(sps_plan* pl, double tol, sps_result* res, bool warm, cudaStream_t st) {
  const int G = pl->G;
  Level& LG = pl->lev[G - 1];
  const long long K = LG.geom.K;
  const double nb = pl->rhs_norm;
  float* a32 = LG.f.alpha;
  float* v32 = pl->ftmp[7];      // the apply does not use ftmp[6..7]
  int it = 0, status = SPS_OK;
  double rel = 1.0, rlast = 0.0;
  const double ratio = pl->opt.replace_ratio > 0 ? pl->opt.replace_ratio : 1e-2;
  bool outer64 = false;   // FP64 outer operator after an FP32 breakdown
  SPS_CUDA(cudaMemsetAsync(pl->scal, 0, sizeof(double) * NSCAL, st));
  if (warm) {
    SPS_TRY(apply_level<double>(pl, G, pl->x, pl->v, st));
    SPS_TRY(vec_residual(pl->r, pl->rhs, pl->v, K, pl->scal, S_RR, pl, st));
    res->fp64_applies++;
  } else {
    SPS_CUDA(cudaMemsetAsync(pl->x, 0, sizeof(double) * K, st));
    SPS_CUDA(cudaMemcpyAsync(pl->r, pl->rhs, sizeof(double) * K, cudaMemcpyDeviceToDevice, st));
    SPS_TRY(dot(pl, pl->r, pl->r, K, S_RR, st));
  }
  auto precondition = [&](cudaStream_t s) -> int {          // z = V32(r)
    if (!pl->opt.precondition) {
      SPS_CUDA(cudaMemcpyAsync(pl->z, pl->r, sizeof(double) * K, cudaMemcpyDeviceToDevice, s));
      return SPS_OK;
    }
    SPS_TRY(vec_cast_d2f(LG.f.b, pl->r, K, s));
    SPS_TRY(vcycle_into<float>(pl, LG.f.b, a32, s));
    return vec_cast_f2d(pl->z, a32, K, s);
  };
  // v = A32 p (A64 p after a breakdown); w = r'z / p'v; alpha += w p; r -= w v
  auto half_apply = [&](cudaStream_t s) -> int {
    if (outer64) {
      SPS_TRY(apply_level<double>(pl, G, pl->p, pl->v, s));
    } else {
      SPS_TRY(vec_cast_d2f(pl->p32, pl->p, K, s));
      SPS_TRY(apply_level<float>(pl, G, pl->p32, v32, s));          // FP32 operator
      SPS_TRY(vec_cast_f2d(pl->v, v32, K, s));
    }
    SPS_TRY(dot(pl, pl->p, pl->v, K, S_PV, s));
    SPS_CUDA(cudaMemcpyAsync(pl->rprev, pl->r, sizeof(double) * K, cudaMemcpyDeviceToDevice, s));
    SPS_TRY(pcg_update_xr(pl, K, S_RZ_A, s));
    SPS_CUDA(cudaMemcpyAsync(pl->host_scal, pl->scal, sizeof(double) * NSCAL, cudaMemcpyDeviceToHost, s));
    return SPS_OK;
  };
  // z = V32(r); beta = z'(r - r_prev) / r~'z~; p = z + beta p; then half_apply
  auto body = [&](cudaStream_t s) -> int {
    SPS_TRY(precondition(s));
    SPS_TRY(dot2(pl, pl->z, pl->r, pl->rprev, K, S_RZ_B, s));      // z'r, z'r_prev
    SPS_TRY(pcg_update_p(pl, K, S_RZ_B, S_RZ_A, 1, s));
    SPS_CUDA(cudaMemcpyAsync(pl->scal + S_RZ_A, pl->scal + S_RZ_B, sizeof(double), cudaMemcpyDeviceToDevice, s));
    return half_apply(s);
  };
  SPS_TRY(precondition(st));
  SPS_CUDA(cudaMemcpyAsync(pl->p, pl->z, sizeof(double) * K, cudaMemcpyDeviceToDevice, st));
  SPS_TRY(dot(pl, pl->r, pl->z, K, S_RZ_A, st));
  SPS_TRY(read_scalars(pl, st));
  rel = std::sqrt(pl->host_scal[S_RR]) / nb;
  rlast = std::sqrt(pl->host_scal[S_RR]);
  bool restarted = true;   // the next step is a half_apply (after the first V-cycle or a replacement)
  while (!(rel <= tol) && std::isfinite(rel) && it < pl->opt.max_iter) {
    if (restarted) {
      SPS_TRY(half_apply(st));
      SPS_CUDA(cudaStreamSynchronize(st));
      restarted = false;
    } else {
      SPS_TRY(run_iteration(pl, outer64 ? 2 : 1, body, st));
    }
    ++it;
    if (outer64) res->fp64_applies++;
    if (pl->host_scal[S_FLAG] != 0.0) {
      if (outer64) {
        status = SPS_EBREAKDOWN;
        break;
      }
      // the step was not taken (x, r unchanged): FP64 residual, V-cycle, new direction
      outer64 = true;
      SPS_CUDA(cudaMemsetAsync(pl->scal, 0, sizeof(double) * NSCAL, st));
      SPS_TRY(apply_level<double>(pl, G, pl->x, pl->v, st));
      SPS_TRY(vec_residual(pl->r, pl->rhs, pl->v, K, pl->scal, S_RR, pl, st));
      res->fp64_applies++;
      SPS_TRY(precondition(st));
      SPS_CUDA(cudaMemcpyAsync(pl->p, pl->z, sizeof(double) * K, cudaMemcpyDeviceToDevice, st));
      SPS_TRY(dot(pl, pl->r, pl->z, K, S_RZ_A, st));
      SPS_TRY(read_scalars(pl, st));
      rlast = std::sqrt(pl->host_scal[S_RR]);
      rel = rlast / nb;
      restarted = true;
      continue;
    }
    double rn = std::sqrt(pl->host_scal[S_RR]);
    rel = rn / nb;
    if (rel <= tol || rn <= ratio * rlast) {                         // FP64 residual replacement
      SPS_TRY(apply_level<double>(pl, G, pl->x, pl->v, st));
      SPS_TRY(vec_residual(pl->r, pl->rhs, pl->v, K, pl->scal, S_RR, pl, st));
      SPS_TRY(read_scalars(pl, st));
      res->fp64_applies++;
      rn = std::sqrt(pl->host_scal[S_RR]);
      rel = rn / nb;
      rlast = rn;
      if (rel <= tol) break;
      // continue with the replaced residual: next V-cycle, beta, direction, apply
      SPS_TRY(body(st));
      SPS_CUDA(cudaStreamSynchronize(st));
      ++it;
      if (pl->host_scal[S_FLAG] != 0.0) {
        if (outer64) {
          status = SPS_EBREAKDOWN;
          break;
        }
        outer64 = true;   // handled at the top of the loop on the next breakdown check
        SPS_CUDA(cudaMemsetAsync(pl->scal + S_FLAG, 0, sizeof(double), st));
        SPS_CUDA(cudaStreamSynchronize(st));
        pl->host_scal[S_FLAG] = 0.0;
        restarted = false;
        // restart as above: FP64 residual from the (unchanged) iterate
        SPS_CUDA(cudaMemsetAsync(pl->scal, 0, sizeof(double) * NSCAL, st));
        SPS_TRY(apply_level<double>(pl, G, pl->x, pl->v, st));
        SPS_TRY(vec_residual(pl->r, pl->rhs, pl->v, K, pl->scal, S_RR, pl, st));
        res->fp64_applies++;
        SPS_TRY(precondition(st));
        SPS_CUDA(cudaMemcpyAsync(pl->p, pl->z, sizeof(double) * K, cudaMemcpyDeviceToDevice, st));
        SPS_TRY(dot(pl, pl->r, pl->z, K, S_RZ_A, st));
        SPS_TRY(read_scalars(pl, st));
        rlast = std::sqrt(pl->host_scal[S_RR]);
        rel = rlast / nb;
        restarted = true;
        continue;
      }
      rn = std::sqrt(pl->host_scal[S_RR]);
      rel = rn / nb;
    }
  }
  res->iterations = it;
  res->rel_res = rel;
  // final FP64 check (the loop exits right after a replacement when converged)
  SPS_TRY(apply_level<double>(pl, G, pl->x, pl->v, st));
  SPS_TRY(vec_residual(pl->z, pl->rhs, pl->v, K, pl->scal, S_TMP, pl, st));
  SPS_TRY(read_scalars(pl, st));
  res->rel_res_true = std::sqrt(pl->host_scal[S_TMP]) / nb;
  if (status == SPS_OK && !(res->rel_res_true <= tol)) status = SPS_ENOCONV;
  res->status = status;
  return status;
}

// Temporary device buffers of a call (counted against the plan's limit while held).
struct DevBuf {
  sps_plan* pl;
  void* p = nullptr;
  explicit DevBuf(sps_plan* plan) : pl(plan) {}
  ~DevBuf() { plan_free(pl, p); }
};

int stage_in(const double* src, long long n, int mem, DevBuf& buf, const double** dev, cudaStream_t st) {
  if (mem == SPS_MEM_DEVICE) {
    *dev = src;
    return SPS_OK;
  }
  SPS_TRY(palloc(buf.pl, (double**)&buf.p, n));
  SPS_CUDA(cudaMemcpyAsync(buf.p, src, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  *dev = (const double*)buf.p;
  return SPS_OK;
}

int stage_out_ptr(double* dst, long long n, int mem, DevBuf& buf, double** dev) {
  if (mem == SPS_MEM_DEVICE) {
    *dev = dst;
    return SPS_OK;
  }
  SPS_TRY(palloc(buf.pl, (double**)&buf.p, n));
  *dev = (double*)buf.p;
  return SPS_OK;
}

int finish_out(double* dst, const double* dev, long long n, int mem, cudaStream_t st) {
  if (mem == SPS_MEM_DEVICE) return SPS_OK;
  return copy_out(dst, dev, n, SPS_MEM_HOST, st);
}

int check_level(const sps_plan* pl, int level, int lowest) {
  if (level < lowest || level > pl->G) {
    set_error("level out of range");
    return SPS_EINVAL;
  }
  return SPS_OK;
}

// Run a float kernel on double inputs: widen/narrow through temporaries.
template <typename F>
int run_f32(sps_plan* pl, long long nin, long long nout, const double* in, double* out, F&& fn, cudaStream_t st) {
  DevBuf a(pl), b(pl);
  SPS_TRY(palloc(pl, (float**)&a.p, nin));
  SPS_TRY(palloc(pl, (float**)&b.p, nout));
  SPS_TRY(vec_cast_d2f((float*)a.p, in, nin, st));
  SPS_TRY(fn((const float*)a.p, (float*)b.p));
  SPS_TRY(vec_cast_f2d(out, (const float*)b.p, nout, st));
  SPS_CUDA(cudaStreamSynchronize(st));
  return SPS_OK;
}

}  // namespace
}  // namespace sps

using namespace sps;

namespace sps {
void level_tile(LevelGeom& G, int ts) {
  G.ts = ts;
  for (int p = 0; p < G.P; ++p) {
    G.E[p] = std::min(ts, G.N[p]) + Q;
    G.invE[p] = 1.0f / (float)G.E[p];
  }
  int es = 1;
  for (int p = G.P - 1; p >= 0; --p) {
    G.Es[p] = es;
    es *= G.E[p];
  }
  G.patch = es;
}
}  // namespace sps

extern "C" {

void sps_default_options(sps_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = SPS_PREC_FP64;
  opt->nu1 = 1;
  opt->nu2 = 1;
  opt->omega = 0.0;
  opt->power_iters = 20;
  opt->max_iter = 20000;
  opt->warm_start = 0;
  opt->tile = 0;
  opt->replace_ratio = 1e-2;
  opt->hybrid = 1;
  opt->graphs = 1;
  opt->precondition = 1;
  opt->autotune = 0;
  opt->lanes_r = 0;
  opt->coarse_cg = 0;
  opt->coarse_iters = 32;
  opt->max_device_bytes = 0;
}

const char* sps_last_error(void) { return g_last_error.c_str(); }

int sps_plan_create(sps_plan** out, int P, int q, const int* intervals, const double* lo, const double* hi,
                    int levels, double lambda, const sps_options* opt) {
  if (!out || !intervals) {
    set_error("null argument");
    return SPS_EINVAL;
  }
  *out = nullptr;
  if (P < 1 || P > MAXP) {
    set_error("P must be in 1..5");
    return SPS_EINVAL;
  }
  if (q != Q) {
    set_error("only cubic splines (q = 3) are built");
    return SPS_EINVAL;
  }
  if (levels < 1 || levels > MAXL) {
    set_error("levels must be in 1..12");
    return SPS_EINVAL;
  }
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) {
    set_error("lambda must be finite and >= 0");
    return SPS_EINVAL;
  }
  sps_options o;
  sps_default_options(&o);
  if (opt) o = *opt;
  if (o.nu1 < 0 || o.nu2 < 0 || o.max_iter < 1 || (o.precision != SPS_PREC_FP64 && o.precision != SPS_PREC_MIXED) ||
      o.tile < 0 || (o.tile & (o.tile - 1)) != 0 || (o.autotune != 0 && o.autotune != 1) ||
      (o.lanes_r != 0 && o.lanes_r != 2 && o.lanes_r != 3) || (o.coarse_cg != 0 && o.coarse_cg != 1) ||
      o.coarse_iters < 1 || o.coarse_iters > 100000 || o.max_device_bytes < 0 || !(o.omega >= 0.0 || o.omega <= 0.0) ||
      (o.replace_ratio != 0.0 && !(o.replace_ratio > 0.0 && o.replace_ratio < 1.0))) {
    set_error("invalid options");
    return SPS_EINVAL;
  }
  int Lbits = 1;
  for (int p = 0; p < P; ++p) {
    const int N = intervals[p];
    if (N < 1 || (N & (N - 1)) != 0 || N > 4096) {
      set_error("intervals must be powers of two <= 4096");
      return SPS_EINVAL;
    }
    if ((N >> (levels - 1)) < 1) {
      set_error("too many levels for the grid: the coarsest level needs >= 1 interval");
      return SPS_EINVAL;
    }
    int b = 0;
    while ((1 << b) < N) ++b;
    Lbits = std::max(Lbits, b);
    const double l = lo ? lo[p] : 0.0, h = hi ? hi[p] : 1.0;
    if (!std::isfinite(l) || !std::isfinite(h) || !(h > l)) {
      set_error("domain bounds must be finite with lo < hi");
      return SPS_EINVAL;
    }
  }
  if (P * Lbits > 26) {
    set_error("grid too fine for the cell index (P * log2(max N) must be <= 26)");
    return SPS_EINVAL;
  }
  sps_plan* pl = new (std::nothrow) sps_plan();
  if (!pl) {
    set_error("host allocation failed");
    return SPS_ENOMEM;
  }
  pl->P = P;
  pl->q = q;
  pl->G = levels;
  pl->lam = lambda;
  pl->opt = o;
  pl->Lbits = Lbits;
  cudaGetDevice(&pl->device);
  for (int p = 0; p < P; ++p) {
    pl->N[p] = intervals[p];
    pl->lo[p] = lo ? lo[p] : 0.0;
    pl->hi[p] = hi ? hi[p] : 1.0;
  }
  const int ts_default[6] = {0, 256, 32, 8, 4, 2};
  int rc = SPS_OK;
  for (int g = 1; g <= levels && rc == SPS_OK; ++g) {
    LevelGeom& G = pl->lev[g - 1].geom;
    G = LevelGeom();
    G.P = P;
    G.shift = levels - g;
    G.ts = o.tile > 0 ? o.tile : ts_default[P];
    G.K = 1;
    for (int p = P - 1; p >= 0; --p) {
      G.N[p] = intervals[p] >> (levels - g);
      G.J[p] = G.N[p] + Q;
      G.stride[p] = G.K;
      G.K *= G.J[p];
      G.lo[p] = pl->lo[p];
      G.inv_h[p] = (double)G.N[p] / (pl->hi[p] - pl->lo[p]);
    }
    level_tile(G, G.ts);
    pl->lev[g - 1].lanes_r = (P == 3 || P == 4) ? o.lanes_r : 0;
    if (g == 1 && G.K > COARSE_MAX && !o.coarse_cg) {
      set_error("coarsest level too large for the dense coarse solve (K_1 > 4096): add levels or use coarse_cg");
      rc = SPS_EINVAL;
    }
    if ((long long)G.patch * 8 * 2 > 200 * 1024) {
      set_error("tile too large for shared memory");
      rc = SPS_EINVAL;
    }
  }
  if (rc != SPS_OK) {
    delete pl;
    return rc;
  }
  // per-level vectors and Gram bands
  std::vector<double> hb;
  for (int g = 1; g <= levels && rc == SPS_OK; ++g) {
    Level& L = pl->lev[g - 1];
    const LevelGeom& G = L.geom;
    long long nb = 0;
    for (int p = 0; p < P; ++p) nb += 3LL * G.J[p] * BAND;
    hb.assign(nb, 0.0);
    long long off = 0;
    for (int p = 0; p < P; ++p) {
      const double h = (pl->hi[p] - pl->lo[p]) / G.N[p];
      for (int r = 0; r < 3; ++r) gram_band(G.N[p], h, r, hb.data() + off + (long long)r * G.J[p] * BAND);
      off += 3LL * G.J[p] * BAND;
    }
    std::vector<float> hf(hb.begin(), hb.end());
    if ((rc = palloc(pl, &L.d.alpha, G.K)) || (rc = palloc(pl, &L.d.b, G.K)) || (rc = palloc(pl, &L.d.u, G.K)) ||
        (rc = palloc(pl, &L.d.dinv, G.K)) || (rc = palloc(pl, &L.d.band, nb)) || (rc = palloc(pl, &L.f.alpha, G.K)) ||
        (rc = palloc(pl, &L.f.b, G.K)) || (rc = palloc(pl, &L.f.u, G.K)) || (rc = palloc(pl, &L.f.dinv, G.K)) ||
        (rc = palloc(pl, &L.f.band, nb)) || (rc = palloc(pl, &L.diag, G.K)))
      break;
    if (cudaMemcpy(L.d.band, hb.data(), sizeof(double) * nb, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(L.f.band, hf.data(), sizeof(float) * nb, cudaMemcpyHostToDevice) != cudaSuccess) {
      set_error("copy of Gram bands failed");
      rc = SPS_ECUDA;
    }
  }
  const long long KG = pl->lev[levels - 1].geom.K;
  const long long K1 = pl->lev[0].geom.K;
  const long long Km = max_K(pl);
  for (int i = 0; i < 8 && rc == SPS_OK; ++i) {
    rc = palloc(pl, &pl->dtmp[i], Km);
    if (rc == SPS_OK) rc = palloc(pl, &pl->ftmp[i], Km);
  }
  if (rc == SPS_OK)
    if ((rc = palloc(pl, &pl->x, KG)) || (rc = palloc(pl, &pl->r, KG)) || (rc = palloc(pl, &pl->z, KG)) ||
        (rc = palloc(pl, &pl->p, KG)) || (rc = palloc(pl, &pl->v, KG)) || (rc = palloc(pl, &pl->rprev, KG)) ||
        (rc = palloc(pl, &pl->p32, KG)) || (rc = palloc(pl, &pl->rhs, KG)) ||
        (rc = palloc(pl, &pl->scal, NSCAL)) || (rc = palloc(pl, &pl->red_part, 4 * 304)) ||
        (rc = palloc(pl, &pl->red_count, 1)) || (rc = palloc(pl, &pl->err_flag, 1))) {
    }
  if (rc == SPS_OK && !o.coarse_cg)
    if ((rc = palloc(pl, &pl->coarse_A, K1 * K1)) || (rc = palloc(pl, &pl->coarse_inv, K1 * K1)) ||
        (rc = palloc(pl, &pl->coarse_invt, K1 * K1)) || (rc = palloc(pl, &pl->coarse_tmp, 6 * K1 + K1 * K1))) {
    }
  if (rc == SPS_OK) {
    if (cudaMemset(pl->red_count, 0, sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(pl->err_flag, 0, sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&pl->host_scal, sizeof(double) * NSCAL) != cudaSuccess) {
      set_error("initialisation failed");
      rc = SPS_ECUDA;
    }
  }
  if (rc != SPS_OK) {
    sps_destroy(pl);
    return rc;
  }
  *out = pl;
  return SPS_OK;
}

int sps_set_lambda(sps_plan* pl, double lambda) {
  if (!pl || !(lambda >= 0.0) || !std::isfinite(lambda)) {
    set_error("invalid plan or lambda");
    return SPS_EINVAL;
  }
  pl->lam = lambda;
  pl->have_points = false;   // the diagonals and the coarse matrix depend on lambda
  ++pl->gen;
  return SPS_OK;
}

int sps_destroy(sps_plan* pl) {
  if (!pl) return SPS_OK;
  // every device buffer of the plan was allocated by plan_alloc
  for (auto& kv : pl->dev_sizes) cudaFree(kv.first);
  pl->dev_sizes.clear();
  pl->dev_bytes = 0;
  if (pl->host_scal) cudaFreeHost(pl->host_scal);
  for (auto& gr : pl->graph)
    if (gr.exec) cudaGraphExecDestroy(gr.exec);
  if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
  delete pl;
  return SPS_OK;
}

int sps_set_points(sps_plan* pl, int64_t n, const void* x, const void* y, int dtype, int mem, void* stream) {
  if (!pl || !x || !y) {
    set_error("null argument");
    return SPS_EINVAL;
  }
  if (n == 0) {
    set_error("no data points");
    return SPS_EEMPTY;
  }
  if (n < 0 || n >= (1LL << 31) - 1 || (dtype != SPS_F32 && dtype != SPS_F64) ||
      (mem != SPS_MEM_HOST && mem != SPS_MEM_DEVICE)) {
    set_error("invalid n, dtype or mem");
    return SPS_EINVAL;
  }
  cudaStream_t st = as_stream(stream);
  pl->have_points = false;
  const int P = pl->P;
  const size_t es = dtype == SPS_F64 ? 8 : 4;
  if (n > pl->n_cap || dtype != pl->dtype) {
    free_points(pl);
    int rc;
    if ((rc = palloc(pl, (char**)&pl->x_sorted, (long long)es * P * n)) || (rc = palloc(pl, &pl->y_sorted, n)) ||
        (rc = palloc(pl, &pl->keys, n)) || (rc = palloc(pl, &pl->keys_tmp, n)) || (rc = palloc(pl, &pl->perm, n)) ||
        (rc = palloc(pl, &pl->perm_tmp, n)) ||
        (dtype == SPS_F64 && (rc = palloc(pl, &pl->x32_sorted, (long long)P * n)))) {
      free_points(pl);
      return rc;
    }
    if (dtype == SPS_F32) pl->x32_sorted = (float*)pl->x_sorted;
    pl->n_cap = n;
  }
  pl->n = n;
  pl->dtype = dtype;
  // device copies of host inputs
  DevBuf hx(pl), hy(pl);
  const void* xd = x;
  const void* yd = y;
  if (mem == SPS_MEM_HOST) {
    SPS_TRY(palloc(pl, (char**)&hx.p, (long long)es * P * n));
    SPS_TRY(palloc(pl, (char**)&hy.p, (long long)es * n));
    SPS_CUDA(cudaMemcpyAsync(hx.p, x, es * P * n, cudaMemcpyHostToDevice, st));
    SPS_CUDA(cudaMemcpyAsync(hy.p, y, es * n, cudaMemcpyHostToDevice, st));
    xd = hx.p;
    yd = hy.p;
  }
  SPS_TRY(compute_keys(pl, xd, yd, dtype, st));
  int bad = 0;
  SPS_CUDA(cudaMemcpyAsync(&bad, pl->err_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  SPS_CUDA(cudaStreamSynchronize(st));
  if (bad & ERR_DOMAIN) {
    SPS_CUDA(cudaMemsetAsync(pl->err_flag, 0, sizeof(int), st));
    set_error("a point lies outside [lo, hi], or a coordinate or response is not finite");
    return SPS_EDOM;
  }
  SPS_TRY(radix_sort(pl, P * pl->Lbits, st));
  SPS_TRY(gather_points(pl, xd, yd, dtype, st));
  for (int g = 1; g <= pl->G; ++g) SPS_TRY(build_level_work(pl, g, st));
  // right-hand side Phi'y (Algorithm 3 with the responses)
  const int G = pl->G;
  const long long KG = pl->lev[G - 1].geom.K;
  SPS_CUDA(cudaMemsetAsync(pl->rhs, 0, sizeof(double) * KG, st));
  SPS_TRY(point_op<double>(pl, G, PT_RHS, nullptr, pl->rhs, st));
  SPS_TRY(dot(pl, pl->rhs, pl->rhs, KG, S_TMP, st));
  // diag(A_g) = diag(Phi_g'Phi_g) (Algorithm 5) + lambda diag(Lambda_g)
  for (int g = 1; g <= G; ++g) {
    Level& L = pl->lev[g - 1];
    SPS_CUDA(cudaMemsetAsync(L.diag, 0, sizeof(double) * L.geom.K, st));
    SPS_TRY(point_op<double>(pl, g, PT_DIAG, nullptr, L.diag, st));
    SPS_TRY(penalty_diag(pl, g, L.diag, st));
    SPS_TRY(vec_recip(L.d.dinv, L.f.dinv, L.diag, L.geom.K, st));
  }
  SPS_TRY(read_scalars(pl, st));
  pl->rhs_norm = std::sqrt(pl->host_scal[S_TMP]);
  if (!std::isfinite(pl->rhs_norm)) {
    set_error("the right-hand side Phi'y is not finite");
    return SPS_EDOM;
  }
  if (!pl->opt.coarse_cg) SPS_TRY(coarse_assemble(pl, st));
  SPS_TRY(assemble_coarse_levels(pl, st));
  // FP64 mode: basis values of the points on every matrix-free level (>= 2)
  if (pl->opt.precision == SPS_PREC_FP64) {
    for (int g = 2; g <= G; ++g) {
      Level& L = pl->lev[g - 1];
      if (L.st_d) continue;
      const long long need = pl->n * 4LL * P;
      if (L.pre_cap < need) {
        pfree(pl, L.pre);
        L.pre_cap = 0;
        SPS_TRY(palloc(pl, &L.pre, need));
        L.pre_cap = need;
      }
      if (P == 3) {   // products for the four-lane layout
        const long long need2 = pl->n * (long long)PRE2_STRIDE;
        if (L.pre2_cap < need2) {
          pfree(pl, L.pre2);
          L.pre2_cap = 0;
          SPS_TRY(palloc(pl, &L.pre2, need2));
          L.pre2_cap = need2;
        }
      }
      SPS_TRY(basis_precompute(pl, g, st));
    }
  }
  if (pl->opt.autotune && !pl->tuned) {
    SPS_TRY(autotune(pl, st));
    pl->tuned = true;
  }
  for (int g = 2; g <= G; ++g) {
    if (pl->opt.omega > 0.0) pl->lev[g - 1].omega = pl->opt.omega;
    else SPS_TRY(estimate_omega(pl, g, st));
  }
  pl->lev[0].omega = pl->opt.omega > 0.0 ? pl->opt.omega : 0.0;
  SPS_CUDA(cudaStreamSynchronize(st));
  SPS_CUDA(cudaGetLastError());
  SPS_TRY(check_device_errors(pl, st));
  pl->have_points = true;
  ++pl->gen;
  return SPS_OK;
}

int sps_solve(sps_plan* pl, double* coef, int mem, double tol, sps_result* res_out, void* stream) {
  SPS_TRY(check_plan_points(pl));
  if (!coef || !(tol > 0.0) || (mem != SPS_MEM_HOST && mem != SPS_MEM_DEVICE)) {
    set_error("invalid coef, tol or mem");
    return SPS_EINVAL;
  }
  cudaStream_t st = as_stream(stream);
  auto t0 = std::chrono::steady_clock::now();
  sps_result res;
  std::memset(&res, 0, sizeof(res));
  const long long KG = pl->lev[pl->G - 1].geom.K;
  if (pl->rhs_norm == 0.0) {   // y = 0: alpha = 0
    SPS_CUDA(cudaMemsetAsync(pl->x, 0, sizeof(double) * KG, st));
    res.status = SPS_OK;
  } else {
    const bool warm = pl->opt.warm_start != 0;
    if (warm) SPS_TRY(copy_in(pl->x, coef, KG, mem, st));
    int rc = pl->opt.precision == SPS_PREC_MIXED ? solve_mixed(pl, tol, &res, warm, st)
                                                 : solve_fp64(pl, tol, &res, warm, st);
    if (rc != SPS_OK && rc != SPS_ENOCONV && rc != SPS_EBREAKDOWN) return rc;
    if (rc == SPS_EBREAKDOWN) set_error("CG breakdown (p'Ap <= 0 or non-finite)");
    if (rc == SPS_ENOCONV) set_error("max_iter reached before the tolerance");
  }
  SPS_TRY(copy_out(coef, pl->x, KG, mem, st));
  SPS_CUDA(cudaStreamSynchronize(st));
  SPS_TRY(check_device_errors(pl, st));
  res.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (res_out) *res_out = res;
  return res.status;
}

namespace {
int check_batch(sps_plan* const* plans, int count, double* const* coefs, int mem, double tol) {
  if (!plans || !coefs || count < 1 || !(tol > 0.0) || (mem != SPS_MEM_HOST && mem != SPS_MEM_DEVICE)) {
    set_error("invalid batch arguments");
    return SPS_EINVAL;
  }
  for (int i = 0; i < count; ++i) {
    SPS_TRY(check_plan_points(plans[i]));
    if (plans[i]->P > 3 || !coefs[i] || plans[i]->lev[plans[i]->G - 1].geom.K >= (1LL << 31) ||
        plans[i]->opt.coarse_cg) {
      set_error("batched solves take P <= 3, fewer than 2^31 coefficients, the dense coarse solver and a "
                "coefficient buffer per problem");
      return SPS_EINVAL;
    }
    if (plans[i]->rhs_norm == 0.0) {
      set_error("a problem of the batch has a zero right-hand side");
      return SPS_EINVAL;
    }
  }
  return SPS_OK;
}
}  // namespace

int sps_solve_batch(sps_plan* const* plans, int count, double* const* coefs, int mem, double tol,
                    sps_result* results, void* stream) {
  SPS_TRY(check_batch(plans, count, coefs, mem, tol));
  return solve_batch(plans, count, coefs, mem, tol, nullptr, results, nullptr, as_stream(stream));
}

int sps_solve_batch_shape(sps_plan* const* plans, int count, double* const* coefs, int mem, double tol,
                          const sps_batch_shape* shape, sps_result* results, sps_batch_shape* used, void* stream) {
  SPS_TRY(check_batch(plans, count, coefs, mem, tol));
  if (shape && ((shape->cluster != 1 && shape->cluster != 2 && shape->cluster != 4 && shape->cluster != 8) ||
                shape->big < -1)) {
    set_error("batch shape: cluster must be 1, 2, 4 or 8 and big >= -1");
    return SPS_EINVAL;
  }
  return solve_batch(plans, count, coefs, mem, tol, shape, results, used, as_stream(stream));
}

int sps_tune_batch(sps_plan* const* plans, int count, double* const* coefs, int mem, double tol,
                   sps_batch_shape* best, void* stream) {
  SPS_TRY(check_batch(plans, count, coefs, mem, tol));
  return tune_batch(plans, count, coefs, mem, tol, best, as_stream(stream));
}

int sps_coef_count(const sps_plan* pl, int level, int64_t* K) {
  if (!pl || !K) {
    set_error("null argument");
    return SPS_EINVAL;
  }
  SPS_TRY(check_level(pl, level, 1));
  *K = pl->lev[level - 1].geom.K;
  return SPS_OK;
}

int sps_apply(sps_plan* pl, int level, int prec, const double* v, double* u, int mem, void* stream) {
  SPS_TRY(check_plan_points(pl));
  SPS_TRY(check_level(pl, level, 1));
  cudaStream_t st = as_stream(stream);
  const long long K = pl->lev[level - 1].geom.K;
  DevBuf bi(pl), bo(pl);
  const double* vd;
  double* ud;
  SPS_TRY(stage_in(v, K, mem, bi, &vd, st));
  SPS_TRY(stage_out_ptr(u, K, mem, bo, &ud));
  if (prec == SPS_PREC_MIXED) {
    SPS_TRY(run_f32(pl, K, K, vd, ud, [&](const float* a, float* b) { return apply_level<float>(pl, level, a, b, st); },
                    st));
  } else {
    SPS_TRY(apply_level<double>(pl, level, vd, ud, st));
  }
  SPS_TRY(check_device_errors(pl, st));
  return finish_out(u, ud, K, mem, st);
}

int sps_point_apply(sps_plan* pl, int level, int prec, const double* v, double* u, int mem, void* stream) {
  SPS_TRY(check_plan_points(pl));
  SPS_TRY(check_level(pl, level, 1));
  cudaStream_t st = as_stream(stream);
  const long long K = pl->lev[level - 1].geom.K;
  DevBuf bi(pl), bo(pl);
  const double* vd;
  double* ud;
  SPS_TRY(stage_in(v, K, mem, bi, &vd, st));
  SPS_TRY(stage_out_ptr(u, K, mem, bo, &ud));
  if (prec == SPS_PREC_MIXED) {
    SPS_TRY(run_f32(pl, K, K, vd, ud,
                    [&](const float* a, float* b) {
                      SPS_CUDA(cudaMemsetAsync(b, 0, sizeof(float) * K, st));
                      return point_op<float>(pl, level, PT_APPLY, a, b, st);
                    },
                    st));
  } else {
    SPS_CUDA(cudaMemsetAsync(ud, 0, sizeof(double) * K, st));
    SPS_TRY(point_op<double>(pl, level, PT_APPLY, vd, ud, st));
  }
  SPS_TRY(check_device_errors(pl, st));
  return finish_out(u, ud, K, mem, st);
}

int sps_profile_begin(void) { return profile_begin(); }

int sps_profile_end(double* point_apply_ms, uint64_t* point_apply_launches) {
  if (!point_apply_ms || !point_apply_launches) {
    set_error("null argument");
    return SPS_EINVAL;
  }
  unsigned long long l = 0;
  SPS_TRY(profile_end(point_apply_ms, &l));
  *point_apply_launches = l;
  return SPS_OK;
}

int sps_launch_count(uint64_t* count) {
  if (!count) {
    set_error("null argument");
    return SPS_EINVAL;
  }
  *count = g_launches.load();
  return SPS_OK;
}

int sps_penalty_apply(sps_plan* pl, int level, int prec, const double* v, double* u, int mem, void* stream) {
  SPS_TRY(check_plan_points(pl));
  SPS_TRY(check_level(pl, level, 1));
  cudaStream_t st = as_stream(stream);
  const long long K = pl->lev[level - 1].geom.K;
  DevBuf bi(pl), bo(pl);
  const double* vd;
  double* ud;
  SPS_TRY(stage_in(v, K, mem, bi, &vd, st));
  SPS_TRY(stage_out_ptr(u, K, mem, bo, &ud));
  if (prec == SPS_PREC_MIXED) {
    SPS_TRY(run_f32(pl, K, K, vd, ud,
                    [&](const float* a, float* b) { return penalty_apply<float>(pl, level, a, b, 1.0, st); }, st));
  } else {
    SPS_TRY(penalty_apply<double>(pl, level, vd, ud, 1.0, st));
  }
  return finish_out(u, ud, K, mem, st);
}

int sps_diag(sps_plan* pl, int level, double* d, int mem, void* stream) {
  SPS_TRY(check_plan_points(pl));
  SPS_TRY(check_level(pl, level, 1));
  cudaStream_t st = as_stream(stream);
  return copy_out(d, pl->lev[level - 1].diag, pl->lev[level - 1].geom.K, mem, st);
}

int sps_rhs(sps_plan* pl, double* b, int mem, void* stream) {
  SPS_TRY(check_plan_points(pl));
  return copy_out(b, pl->rhs, pl->lev[pl->G - 1].geom.K, mem, as_stream(stream));
}

int sps_prolong(sps_plan* pl, int level, int prec, const double* c, double* f, int mem, void* stream) {
  SPS_TRY(check_plan_points(pl));
  SPS_TRY(check_level(pl, level, 2));
  cudaStream_t st = as_stream(stream);
  const long long Kc = pl->lev[level - 2].geom.K, Kf = pl->lev[level - 1].geom.K;
  DevBuf bi(pl), bo(pl);
  const double* cd;
  double* fd;
  SPS_TRY(stage_in(c, Kc, mem, bi, &cd, st));
  SPS_TRY(stage_out_ptr(f, Kf, mem, bo, &fd));
  if (prec == SPS_PREC_MIXED) {
    SPS_TRY(run_f32(pl, Kc, Kf, cd, fd, [&](const float* a, float* b) { return prolong_sub<float>(pl, level, a, b, 0, st); },
                    st));
  } else {
    SPS_TRY(prolong_sub<double>(pl, level, cd, fd, 0, st));
  }
  return finish_out(f, fd, Kf, mem, st);
}

int sps_restrict(sps_plan* pl, int level, int prec, const double* f, double* c, int mem, void* stream) {
  SPS_TRY(check_plan_points(pl));
  SPS_TRY(check_level(pl, level, 2));
  cudaStream_t st = as_stream(stream);
  const long long Kc = pl->lev[level - 2].geom.K, Kf = pl->lev[level - 1].geom.K;
  DevBuf bi(pl), bo(pl);
  const double* fd;
  double* cd;
  SPS_TRY(stage_in(f, Kf, mem, bi, &fd, st));
  SPS_TRY(stage_out_ptr(c, Kc, mem, bo, &cd));
  if (prec == SPS_PREC_MIXED) {
    SPS_TRY(run_f32(pl, Kf, Kc, fd, cd,
                    [&](const float* a, float* b) { return restrict_res<float>(pl, level, a, nullptr, b, st); }, st));
  } else {
    SPS_TRY(restrict_res<double>(pl, level, fd, nullptr, cd, st));
  }
  return finish_out(c, cd, Kc, mem, st);
}

int sps_coarse_solve(sps_plan* pl, const double* r, double* e, int mem, void* stream) {
  SPS_TRY(check_plan_points(pl));
  cudaStream_t st = as_stream(stream);
  const long long K = pl->lev[0].geom.K;
  DevBuf bi(pl), bo(pl);
  const double* rd;
  double* ed;
  SPS_TRY(stage_in(r, K, mem, bi, &rd, st));
  SPS_TRY(stage_out_ptr(e, K, mem, bo, &ed));
  if (pl->opt.coarse_cg) {   // level-1 vectors other than the penalty temporaries
    SPS_CUDA(cudaMemcpyAsync(pl->lev[0].d.b, rd, sizeof(double) * K, cudaMemcpyDeviceToDevice, st));
    SPS_TRY(coarse_cg<double>(pl, pl->lev[0].d.b, ed, pl->dtmp[6], pl->dtmp[7], st));
    SPS_TRY(check_device_errors(pl, st));
  } else {
    SPS_TRY(coarse_solve<double>(pl, rd, ed, st));
  }
  return finish_out(e, ed, K, mem, st);
}

int sps_vcycle(sps_plan* pl, int prec, const double* r, double* z, int mem, void* stream) {
  SPS_TRY(check_plan_points(pl));
  cudaStream_t st = as_stream(stream);
  const int G = pl->G;
  const long long K = pl->lev[G - 1].geom.K;
  DevBuf bi(pl), bo(pl);
  const double* rd;
  double* zd;
  SPS_TRY(stage_in(r, K, mem, bi, &rd, st));
  SPS_TRY(stage_out_ptr(z, K, mem, bo, &zd));
  if (prec == SPS_PREC_MIXED) {
    Level& LG = pl->lev[G - 1];
    SPS_TRY(vec_cast_d2f(LG.f.b, rd, K, st));
    SPS_TRY(vcycle_into<float>(pl, LG.f.b, LG.f.alpha, st));
    SPS_TRY(vec_cast_f2d(zd, LG.f.alpha, K, st));
  } else {
    SPS_CUDA(cudaMemcpyAsync(pl->r, rd, sizeof(double) * K, cudaMemcpyDeviceToDevice, st));
    SPS_TRY(vcycle_into<double>(pl, pl->r, zd, st));
  }
  SPS_CUDA(cudaStreamSynchronize(st));
  SPS_TRY(check_device_errors(pl, st));
  return finish_out(z, zd, K, mem, st);
}

int sps_get_sort(sps_plan* pl, int64_t* perm, uint64_t* key, int mem, void* stream) {
  SPS_TRY(check_plan_points(pl));
  cudaStream_t st = as_stream(stream);
  const long long n = pl->n;
  if (key) {
    SPS_CUDA(cudaMemcpyAsync(key, pl->keys, sizeof(uint64_t) * n,
                             mem == SPS_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
  }
  if (perm) {
    // widen the 32-bit permutation on the host side of the copy
    std::vector<unsigned int> h(n);
    SPS_CUDA(cudaMemcpyAsync(h.data(), pl->perm, sizeof(unsigned int) * n, cudaMemcpyDeviceToHost, st));
    SPS_CUDA(cudaStreamSynchronize(st));
    std::vector<int64_t> w(h.begin(), h.end());
    SPS_CUDA(cudaMemcpyAsync(perm, w.data(), sizeof(int64_t) * n,
                             mem == SPS_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice, st));
  }
  SPS_CUDA(cudaStreamSynchronize(st));
  return SPS_OK;
}

int sps_get_tuning(const sps_plan* pl, int level, int* tile, int* lanes_r) {
  if (!pl || level < 1 || level > pl->G) {
    set_error("invalid plan or level");
    return SPS_EINVAL;
  }
  if (tile) *tile = pl->lev[level - 1].geom.ts;
  if (lanes_r) *lanes_r = pl->lev[level - 1].lanes_r;
  return SPS_OK;
}

int sps_plan_device_bytes(const sps_plan* pl, int64_t* bytes) {
  if (!pl || !bytes) {
    set_error("null argument");
    return SPS_EINVAL;
  }
  *bytes = pl->dev_bytes;
  return SPS_OK;
}

int sps_level_matrix(sps_plan* pl, int level, double* out, int64_t* entries, int mem, void* stream) {
  SPS_TRY(check_plan_points(pl));
  SPS_TRY(check_level(pl, level, 1));
  if (!entries || (mem != SPS_MEM_HOST && mem != SPS_MEM_DEVICE)) {
    set_error("invalid entries pointer or mem");
    return SPS_EINVAL;
  }
  cudaStream_t st = as_stream(stream);
  const Level& L = pl->lev[level - 1];
  const long long K = L.geom.K;
  long long count = 0;
  if (level == 1 && pl->coarse_A) count = K * K;
  else if (L.st_d || L.st_f) count = (long long)L.S * K;
  *entries = count;
  if (!out || count == 0) return SPS_OK;
  if (level == 1 && pl->coarse_A) return copy_out(out, pl->coarse_A, count, mem, st);
  if (L.st_d) return copy_out(out, L.st_d, count, mem, st);
  DevBuf bo(pl);   // mixed plans hold the FP32 stencil only: widen it
  double* od;
  SPS_TRY(stage_out_ptr(out, count, mem, bo, &od));
  SPS_TRY(vec_cast_f2d(od, L.st_f, count, st));
  SPS_CUDA(cudaStreamSynchronize(st));
  return finish_out(out, od, count, mem, st);
}

int sps_simulate_batch(const int* order, const double* t1, const double* tc, int n, int cluster, int big, int grid,
                       double* makespan_ms) {
  if (!order || !t1 || !tc || !makespan_ms || n < 1 ||
      (cluster != 1 && cluster != 2 && cluster != 4 && cluster != 8) || grid < cluster || big < 0 || big > n) {
    set_error("sps_simulate_batch: null pointer or bad sizes");
    return SPS_EINVAL;
  }
  std::vector<char> seen(n, 0);
  for (int i = 0; i < n; ++i) {
    if (order[i] < 0 || order[i] >= n || seen[order[i]]) {
      set_error("sps_simulate_batch: order is not a permutation of 0 .. n-1");
      return SPS_EINVAL;
    }
    seen[order[i]] = 1;
    if (!(t1[i] >= 0.0) || !(tc[i] >= 0.0) || !std::isfinite(t1[i]) || !std::isfinite(tc[i])) {
      set_error("sps_simulate_batch: times must be finite and >= 0");
      return SPS_EINVAL;
    }
  }
  *makespan_ms = batch_makespan(order, t1, tc, n, cluster, cluster == 1 ? 0 : big, grid);
  return SPS_OK;
}

int sps_lanczos_estimate(const double* alpha, const double* beta2, int m, double* theta, double* lambda_hat) {
  if (!alpha || !beta2 || !theta || !lambda_hat || m < 1 || m > LZ_MAX) {
    set_error("sps_lanczos_estimate: null pointer or m outside 1..32");
    return SPS_EINVAL;
  }
  if (!lanczos_lambda_hat(alpha, beta2, m, theta, lambda_hat)) {
    set_error("sps_lanczos_estimate: non-finite coefficients or no positive Ritz value");
    return SPS_EBREAKDOWN;
  }
  return SPS_OK;
}

int sps_get_omega(const sps_plan* pl, double* omega) {
  if (!pl || !omega) {
    set_error("null argument");
    return SPS_EINVAL;
  }
  for (int g = 0; g < pl->G; ++g) omega[g] = pl->lev[g].omega;
  return SPS_OK;
}

int sps_set_omega(sps_plan* pl, const double* omega) {
  if (!pl || !omega) {
    set_error("null argument");
    return SPS_EINVAL;
  }
  for (int g = 0; g < pl->G; ++g)
    if (!(omega[g] > 0.0) || !std::isfinite(omega[g])) {
      set_error("omega must be positive");
      return SPS_EINVAL;
    }
  for (int g = 0; g < pl->G; ++g) pl->lev[g].omega = omega[g];
  ++pl->gen;
  return SPS_OK;
}

int sps_probe_fma_rate(int fp, double* fma_per_s, void* stream) {
  if (!fma_per_s) {
    set_error("null argument");
    return SPS_EINVAL;
  }
  cudaStream_t st = as_stream(stream);
  int dev = 0, sms = 0;
  SPS_CUDA(cudaGetDevice(&dev));
  SPS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  struct Out {
    void* p = nullptr;
    ~Out() { if (p) cudaFree(p); }
  } out;
  SPS_CUDA(cudaMalloc(&out.p, sizeof(double)));
  const int threads = 256, blocks = sms * 8;
  const int iters = fp ? 4000 : 100000;
  cudaEvent_t e0, e1;
  SPS_CUDA(cudaEventCreate(&e0));
  SPS_CUDA(cudaEventCreate(&e1));
  float ms = 0.0f;
  for (int rep = 0; rep < 2; ++rep) {   // first launch warms up
    SPS_CUDA(cudaEventRecord(e0, st));
    if (fp) k_fma_probe<double><<<blocks, threads, 0, st>>>((double*)out.p, iters, 1.0);
    else k_fma_probe<float><<<blocks, threads, 0, st>>>((float*)out.p, iters, 1.0f);
    SPS_CUDA(cudaEventRecord(e1, st));
    SPS_CUDA(cudaEventSynchronize(e1));
    SPS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *fma_per_s = (double)blocks * threads * iters * 8.0 / (ms * 1e-3);
  return SPS_OK;
}

}  // extern "C"

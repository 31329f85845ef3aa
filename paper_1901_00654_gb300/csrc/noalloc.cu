// sps_penalty_apply_noalloc: u = scale * Lambda v on one grid, with no
// device allocation at all.
//
// Who needs it: callers that must not call cudaMalloc/cudaFree -- for
// example code running inside another framework whose caching allocator has
// reserved the device memory, or latency-critical loops where cudaFree's
// implicit device-wide synchronisation is not acceptable.  A plan
// (sps_plan_create) allocates its buffers, so this entry point takes the grid
// directly and keeps its temporaries in a fixed device array instead.
//
// The scratch is one file-scope __device__ array of SPS_NOALLOC_MAX_COEF
// coefficients times 6 doubles (12 MiB).  It belongs to this file's module:
// with CUDA's default lazy module loading the module -- and so the 12 MiB --
// is loaded on a device at the first call there (the cudaGetSymbolAddress
// of the set-up), and stays until the process exits; with
// CUDA_MODULE_LOADING=EAGER it is loaded with the library.  A caller whose
// memory is about to be handed to another allocator should therefore make
// one call first.  Every call shares the array, so calls that overlap on the
// GPU (different streams, different host threads) race on it.  Each sweep
// writes all K entries of its outputs before the next sweep reads them, so
// nothing in the scratch has to start at zero.
//
// The first call on a device does the set-up (cudaGetSymbolAddress of the
// scratch, upload of the cubic element matrices to constant memory); make
// that first call before any stream capture.  The cached set-up is not
// redone after cudaDeviceReset: the entry point must not be used on a device
// after a reset in the same process.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "sps_internal.h"

namespace sps {
namespace {

constexpr long long NOALLOC_MAX = SPS_NOALLOC_MAX_COEF;

static __device__ __align__(256) double g_noalloc_scratch[6 * NOALLOC_MAX];
__constant__ double c_elem[3][4][4];     // element matrices of the cubic pieces, r = 0, 1, 2

struct DeviceSetup {
  std::mutex mu;
  bool ready[64] = {false};
  double* scratch[64] = {nullptr};
};
DeviceSetup g_setup;

// Element matrix E_r[a][b] = int_0^1 d^r p_a(t) d^r p_b(t) dt of the four
// uniform cubic B-spline pieces p_m (m = basis index minus cell index), by
// exact integration of polynomial products.
void cubic_element(int r, double E[4][4]) {
  static const double pc[4][4] = {{1.0 / 6, -0.5, 0.5, -1.0 / 6},     // (1-t)^3/6
                                  {2.0 / 3, 0.0, -1.0, 0.5},          // (3t^3-6t^2+4)/6
                                  {1.0 / 6, 0.5, 0.5, -0.5},          // (-3t^3+3t^2+3t+1)/6
                                  {0.0, 0.0, 0.0, 1.0 / 6}};          // t^3/6
  double d[4][4];
  for (int m = 0; m < 4; ++m) {
    for (int k = 0; k < 4; ++k) d[m][k] = pc[m][k];
    for (int s = 0; s < r; ++s) {
      for (int k = 0; k < 3; ++k) d[m][k] = (k + 1) * d[m][k + 1];
      d[m][3] = 0.0;
    }
  }
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      double acc = 0.0;
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) acc += d[a][i] * d[b][j] / (i + j + 1);
      E[a][b] = acc;
    }
}

struct NoallocGeom {
  int P;
  int N[MAXP], J[MAXP];
  long long stride[MAXP];
  long long K;
  double hs[MAXP][3];   // h^(1 - 2r) per dimension and derivative order
};

// Psi_r[j, j + o] on N cells: sum over the cells carrying both functions.
__device__ __forceinline__ double gram(int r, int j, int o, int N, double hs) {
  const int l = j + o;
  const int c0 = max(0, max(j - Q, l - Q)), c1 = min(N - 1, min(j, l));
  double s = 0.0;
  for (int c = c0; c <= c1; ++c) s += c_elem[r][j - c][l - c];
  return s * hs;
}

// One dimension of the three-term Kronecker-sum recursion (stage 0 first, 1
// middle, 2 last, 3 only dimension); w*/o* are consecutive K-blocks.
__global__ void k_noalloc_sweep(NoallocGeom g, int p, int stage, const double* __restrict__ w0,
                                const double* __restrict__ w1, const double* __restrict__ w2,
                                double* __restrict__ o0, double* __restrict__ o1, double* __restrict__ o2,
                                double scale) {
  const int Jp = g.J[p], Np = g.N[p];
  const long long strd = g.stride[p];
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < g.K; k += (long long)gridDim.x * blockDim.x) {
    const int j = (int)((k / strd) % Jp);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int o = -Q; o <= Q; ++o) {
      if (j + o < 0 || j + o >= Jp) continue;
      const long long kk = k + (long long)o * strd;
      const double m = gram(0, j, o, Np, g.hs[p][0]);
      const double d1 = gram(1, j, o, Np, g.hs[p][1]);
      const double d2 = gram(2, j, o, Np, g.hs[p][2]);
      if (stage == 0) {
        const double x = w0[kk];
        a0 = fma(m, x, a0);
        a1 = fma(d1, x, a1);
        a2 = fma(d2, x, a2);
      } else if (stage == 3) {
        a2 = fma(d2, w0[kk], a2);
      } else {
        const double x0 = w0[kk], x1 = w1[kk], x2 = w2[kk];
        a0 = fma(m, x0, a0);
        a1 = fma(m, x1, fma(d1, x0, a1));
        a2 = fma(m, x2, fma(2.0 * d1, x1, fma(d2, x0, a2)));
      }
    }
    if (stage <= 1) {
      o0[k] = a0;
      o1[k] = a1;
      o2[k] = a2;
    } else {
      o2[k] = scale * a2;
    }
  }
}

int setup_device(int dev, double** scratch) {
  std::lock_guard<std::mutex> lock(g_setup.mu);
  if (dev < 0 || dev >= 64) {
    set_error("device index out of range for the no-allocation scratch");
    return SPS_EINVAL;
  }
  if (!g_setup.ready[dev]) {
    void* ptr = nullptr;
    SPS_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    double E[3][4][4];
    for (int r = 0; r < 3; ++r) cubic_element(r, E[r]);
    SPS_CUDA(cudaMemcpyToSymbol(c_elem, E, sizeof(E)));
    g_setup.scratch[dev] = (double*)ptr;
    g_setup.ready[dev] = true;
  }
  *scratch = g_setup.scratch[dev];
  return SPS_OK;
}

}  // namespace
}  // namespace sps

using namespace sps;

extern "C" int sps_penalty_apply_noalloc(int P, const int* intervals, const double* lo, const double* hi,
                                         double scale, const double* v, double* u, void* stream) {
  if (P < 1 || P > MAXP || !intervals || !v || !u || !std::isfinite(scale)) {
    set_error("invalid argument");
    return SPS_EINVAL;
  }
  NoallocGeom g;
  g.P = P;
  g.K = 1;
  for (int p = P - 1; p >= 0; --p) {
    const int N = intervals[p];
    const double l = lo ? lo[p] : 0.0, h = hi ? hi[p] : 1.0;
    if (N < 1 || N > 4096 || !std::isfinite(l) || !std::isfinite(h) || !(h > l)) {
      set_error("invalid grid: intervals in 1..4096 and finite lo < hi required");
      return SPS_EINVAL;
    }
    g.N[p] = N;
    g.J[p] = N + Q;
    g.stride[p] = g.K;
    g.K *= g.J[p];
    const double hh = (h - l) / N;
    for (int r = 0; r < 3; ++r) g.hs[p][r] = std::pow(hh, 1.0 - 2.0 * r);
  }
  if (g.K > NOALLOC_MAX) {
    set_error("grid has more than SPS_NOALLOC_MAX_COEF (262144) coefficients; use sps_penalty_apply with a plan");
    return SPS_EINVAL;
  }
  // u is written while v is still read (for P = 1 the single sweep reads v[k +- 3]
  // while writing u[k]): the two must not overlap
  {
    const char* vb = (const char*)v;
    const char* ub = (const char*)u;
    const size_t bytes = sizeof(double) * (size_t)g.K;
    if (ub < vb + bytes && vb < ub + bytes) {
      set_error("u and v must not overlap");
      return SPS_EINVAL;
    }
  }
  int dev = 0;
  SPS_CUDA(cudaGetDevice(&dev));
  double* scr = nullptr;
  int rc = setup_device(dev, &scr);
  if (rc != SPS_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const long long K = g.K;
  double* A[3] = {scr, scr + NOALLOC_MAX, scr + 2 * NOALLOC_MAX};
  double* Bv[3] = {scr + 3 * NOALLOC_MAX, scr + 4 * NOALLOC_MAX, scr + 5 * NOALLOC_MAX};
  const int blocks = grid_blocks(K, 256);
  if (P == 1) {
    k_noalloc_sweep<<<blocks, 256, 0, st>>>(g, 0, 3, v, nullptr, nullptr, nullptr, nullptr, u, scale);
    SPS_CHECK_LAUNCH("penalty (no allocation)");
    return SPS_OK;
  }
  for (int p = 0; p < P; ++p) {
    if (p == 0) {
      k_noalloc_sweep<<<blocks, 256, 0, st>>>(g, p, 0, v, nullptr, nullptr, A[0], A[1], A[2], 1.0);
    } else if (p < P - 1) {
      k_noalloc_sweep<<<blocks, 256, 0, st>>>(g, p, 1, A[0], A[1], A[2], Bv[0], Bv[1], Bv[2], 1.0);
      for (int i = 0; i < 3; ++i) std::swap(A[i], Bv[i]);
    } else {
      k_noalloc_sweep<<<blocks, 256, 0, st>>>(g, p, 2, A[0], A[1], A[2], nullptr, nullptr, u, scale);
    }
    SPS_CHECK_LAUNCH("penalty sweep (no allocation)");
  }
  return SPS_OK;
}

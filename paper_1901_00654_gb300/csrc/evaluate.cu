// sps_evaluate: values of the fitted spline s(x) = sum_k alpha_k phi_k(x) at
// query points -- the transposed Khatri-Rao product of Algorithm 4 with the
// query points in place of the data, on the finest grid (Sections 2.1, 2.2).
//
// One thread per query point: the cell and local coordinate of every
// dimension, the q+1 = 4 cubic pieces per dimension, and the (q+1)^P-term sum
// over the cell's coefficients, sum-factorised dimension by dimension
// (4 + 4^2 + ... + 4^P multiply-adds); the last dimension's four
// coefficients are contiguous.  FP64 throughout.
#include <cuda_runtime.h>

#include <cmath>

#include "sps_internal.h"

namespace sps {
namespace {

struct EvalGeom {
  int N[MAXP];
  long long stride[MAXP];
  double lo[MAXP], hi[MAXP], inv_h[MAXP];
};

__device__ __forceinline__ void cubic_pieces(double t, double* b) {
  const double omt = 1.0 - t;
  const double t2 = t * t;
  b[0] = omt * omt * omt * (1.0 / 6.0);
  b[1] = fma(t2, fma(t, 0.5, -1.0), 2.0 / 3.0);
  b[2] = fma(fma(fma(t, -0.5, 0.5), t, 0.5), t, 1.0 / 6.0);
  b[3] = t2 * t * (1.0 / 6.0);
}

// sum over dimensions D..P-1 of the cell's coefficients weighted by the pieces
template <int P, int D>
__device__ __forceinline__ double gather(const double* __restrict__ coef, long long base, const EvalGeom& g,
                                         const double (*b)[4]) {
  if constexpr (D == P - 1) {
    const double* c = coef + base;
    return fma(b[D][0], c[0], fma(b[D][1], c[1], fma(b[D][2], c[2], b[D][3] * c[3])));
  } else {
    double s = 0.0;
#pragma unroll
    for (int m = 0; m < 4; ++m) s = fma(b[D][m], gather<P, D + 1>(coef, base + m * g.stride[D], g, b), s);
    return s;
  }
}

template <int P, typename CT>
__global__ void k_evaluate(const CT* __restrict__ xq, long long m, EvalGeom g, const double* __restrict__ coef,
                           double* __restrict__ out, int* __restrict__ err) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x) {
    double b[P][4];
    long long base = 0;
    bool bad = false;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      double x = (double)xq[i * P + p];
      if (!(x >= g.lo[p] && x <= g.hi[p])) {   // also rejects NaN
        bad = true;
        x = g.lo[p];
      }
      const double u = (x - g.lo[p]) * g.inv_h[p];
      long long c = (long long)floor(u);
      if (c > g.N[p] - 1) c = g.N[p] - 1;   // x = hi belongs to the last cell
      if (c < 0) c = 0;
      cubic_pieces(u - (double)c, b[p]);
      base += c * g.stride[p];
    }
    if (bad) {
      atomicOr(err, 1);
      out[i] = nan("");
      continue;
    }
    out[i] = gather<P, 0>(coef, base, g, b);
  }
}

template <int P>
void launch_eval(const void* xq, int dtype, long long m, const EvalGeom& g, const double* coef, double* out, int* err,
                 cudaStream_t st) {
  const int blocks = grid_blocks(m, 128);
  if (dtype == SPS_F64)
    k_evaluate<P, double><<<blocks, 128, 0, st>>>((const double*)xq, m, g, coef, out, err);
  else
    k_evaluate<P, float><<<blocks, 128, 0, st>>>((const float*)xq, m, g, coef, out, err);
}

struct Tmp {
  void* p = nullptr;
  ~Tmp() { if (p) cudaFree(p); }
};

}  // namespace
}  // namespace sps

using namespace sps;

extern "C" int sps_evaluate(sps_plan* pl, const double* coef, int64_t m, const void* xq, int dtype, double* out,
                            int mem, void* stream) {
  if (!pl || m < 0 || (m > 0 && (!coef || !xq || !out)) || (dtype != SPS_F32 && dtype != SPS_F64) ||
      (mem != SPS_MEM_HOST && mem != SPS_MEM_DEVICE)) {
    set_error("invalid plan, m, buffers, dtype or mem");
    return SPS_EINVAL;
  }
  if (m == 0) return SPS_OK;
  const int P = pl->P;
  const LevelGeom& G = pl->lev[pl->G - 1].geom;
  EvalGeom g;
  for (int p = 0; p < P; ++p) {
    g.N[p] = G.N[p];
    g.stride[p] = G.stride[p];
    g.lo[p] = pl->lo[p];
    g.hi[p] = pl->hi[p];
    g.inv_h[p] = G.inv_h[p];
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t es = dtype == SPS_F64 ? 8 : 4;
  const long long K = G.K;
  Tmp tc, tx, to, terr;
  const double* cd = coef;
  const void* xd = xq;
  double* od = out;
  SPS_CUDA(cudaMalloc(&terr.p, sizeof(int)));
  if (mem == SPS_MEM_HOST) {
    SPS_CUDA(cudaMalloc(&tc.p, sizeof(double) * K));
    SPS_CUDA(cudaMalloc(&tx.p, es * P * m));
    SPS_CUDA(cudaMalloc(&to.p, sizeof(double) * m));
    SPS_CUDA(cudaMemcpyAsync(tc.p, coef, sizeof(double) * K, cudaMemcpyHostToDevice, st));
    SPS_CUDA(cudaMemcpyAsync(tx.p, xq, es * P * m, cudaMemcpyHostToDevice, st));
    cd = (const double*)tc.p;
    xd = tx.p;
    od = (double*)to.p;
  }
  int* err = (int*)terr.p;
  SPS_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  switch (P) {
    case 1: launch_eval<1>(xd, dtype, m, g, cd, od, err, st); break;
    case 2: launch_eval<2>(xd, dtype, m, g, cd, od, err, st); break;
    case 3: launch_eval<3>(xd, dtype, m, g, cd, od, err, st); break;
    case 4: launch_eval<4>(xd, dtype, m, g, cd, od, err, st); break;
    default: launch_eval<5>(xd, dtype, m, g, cd, od, err, st); break;
  }
  SPS_CHECK_LAUNCH("spline evaluation");
  int bad = 0;
  SPS_CUDA(cudaMemcpyAsync(&bad, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (mem == SPS_MEM_HOST) SPS_CUDA(cudaMemcpyAsync(out, od, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
  SPS_CUDA(cudaStreamSynchronize(st));
  if (bad) {
    set_error("a query point lies outside [lo, hi] or is not finite");
    return SPS_EDOM;
  }
  return SPS_OK;
}

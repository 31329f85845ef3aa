// Autotuner of the point operator's launch shape (sps_options.autotune).
//
// The point operator's speed depends on two choices that the data decide: the
// tile side ts (cells per CTA along each dimension: a larger tile amortises
// the staging and flush of its (ts+q)^P coefficient patch over more points,
// a smaller one gives more CTAs and less shared memory per CTA), and, for
// P = 3, 4 (FP32, or FP64 from precomputed basis values), how many lanes
// share one run of points (4^(P-2) lanes holding 16 accumulators each, or
// 4^(P-3) lanes holding 64).  On the first
// sps_set_points of a plan with autotune = 1, every matrix-free level that
// the solve applies is timed with each candidate (CUDA events, the solve's
// own precision) and keeps the fastest; later set-ups of the plan reuse the
// choice.  The operator is the same matrix for every candidate (only the
// order of the floating-point sums changes).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "sps_internal.h"

namespace sps {

namespace {

struct Candidate {
  int ts, lanes_r;
};

// Mean time of `reps` applies of level g after one untimed apply.
int time_apply(sps_plan* pl, int g, bool fp32, int reps, cudaEvent_t e0, cudaEvent_t e1, cudaStream_t st,
               float* ms) {
  Level& L = pl->lev[g - 1];
  const double* vd = L.diag;   // any nonzero vector: a zero input would skip the flush
  double* ud = L.d.u;
  const float* vf = L.f.dinv;
  float* uf = L.f.u;
  auto one = [&]() -> int {
    return fp32 ? point_op<float>(pl, g, PT_APPLY, vf, uf, st) : point_op<double>(pl, g, PT_APPLY, vd, ud, st);
  };
  SPS_TRY(one());
  SPS_CUDA(cudaEventRecord(e0, st));
  for (int r = 0; r < reps; ++r) SPS_TRY(one());
  SPS_CUDA(cudaEventRecord(e1, st));
  SPS_CUDA(cudaEventSynchronize(e1));
  float t = 0.f;
  SPS_CUDA(cudaEventElapsedTime(&t, e0, e1));
  *ms = t / reps;
  return SPS_OK;
}

int tune_level(sps_plan* pl, int g, bool fp32, cudaEvent_t e0, cudaEvent_t e1, cudaStream_t st) {
  Level& L = pl->lev[g - 1];
  const int P = pl->P;
  const int ts0 = L.geom.ts;
  int nmax = 0;
  for (int p = 0; p < P; ++p) nmax = std::max(nmax, L.geom.N[p]);
  std::vector<Candidate> cand;
  for (int ts : {ts0 / 2, ts0, ts0 * 2}) {
    if (ts < 1 || (ts > nmax && ts != ts0)) continue;
    LevelGeom G = L.geom;
    level_tile(G, ts);
    if (point_apply_smem(pl, G, fp32) > POINT_SMEM_MAX - 2048) continue;
    const bool pre = !fp32 && L.pre != nullptr;   // FP64 apply from precomputed basis values
    if ((fp32 || pre) && (P == 3 || P == 4)) {
      cand.push_back({ts, 2});
      cand.push_back({ts, 3});
    } else {
      cand.push_back({ts, 0});
    }
  }
  float best = 3.4e38f;
  Candidate pick = {ts0, L.lanes_r};
  for (const Candidate& c : cand) {
    if (c.ts != L.geom.ts) {
      level_tile(L.geom, c.ts);
      SPS_TRY(build_level_work(pl, g, st));
    }
    L.lanes_r = c.lanes_r;
    float ms = 0.f;
    SPS_TRY(time_apply(pl, g, fp32, 3, e0, e1, st, &ms));
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  if (pick.ts != L.geom.ts) {
    level_tile(L.geom, pick.ts);
    SPS_TRY(build_level_work(pl, g, st));
  }
  L.lanes_r = pick.lanes_r;
  return SPS_OK;
}

}  // namespace

int autotune(sps_plan* pl, cudaStream_t st) {
  const bool fp32 = pl->opt.precision == SPS_PREC_MIXED;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SPS_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    set_error("event creation failed");
    return SPS_ENOMEM;
  }
  int rc = SPS_OK;
  for (int g = 2; g <= pl->G && rc == SPS_OK; ++g) {
    const Level& L = pl->lev[g - 1];
    if (L.st_d || L.st_f) continue;   // assembled: applied as a stencil, no point sweep
    rc = tune_level(pl, g, fp32, e0, e1, st);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace sps

// Batched solves: many independent smoothing problems in one persistent
// kernel launch, captured in a CUDA graph.
//
// A team of CTAs takes whole problems from a device-side queue (largest
// first) and runs the complete mixed-precision flexible PCG of one problem --
// FP32 V-cycle (Algorithm 7 with Algorithm 6) and FP32 point operator, FP64
// outer vectors, dot products, residual replacement and coarse solve -- with
// a barrier between the phases.  A team is a thread-block cluster for the
// largest problems (loops split across its CTAs, cluster barriers, dot
// products through distributed shared memory) and a single CTA for the rest.  Small problems (K <= 40k, n <= 1e5)
// are launch-latency bound when each step is its own kernel; here a
// problem's whole solve costs one queue pop.  Problems with P <= 3 only (one
// lane per run).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <queue>
#include <vector>

#include "sps_internal.h"

namespace sps {

namespace {

constexpr int BT = 256;   // threads per CTA

struct BatchLevel {
  LevelGeom geom;
  const int* run_begin;
  const unsigned long long* run_cell;
  int nruns;
  float *alpha, *b, *u;
  const float* dinv;
  const float* band;
  const double* band_d;
  const float* st_f;
  int S;
  float omega;
};

struct BatchProblem {
  int P, G, x_f64, nu1, nu2, max_iter;
  long long n;
  const void* xs;        // sorted coordinates in the input precision (FP64 path)
  const float* xs32;     // the same rounded to FP32 (FP32 path)
  double lam, tol, ratio, rhs_norm;
  float* ftmp[8];
  double* dtmp[6];
  double *x, *r, *z, *p, *v, *rprev;
  float* p32;
  const double* rhs;
  const double* coarse_z;    // A_1^-1 = Z'Z: Z and Z' (K_1 x K_1 each)
  const double* coarse_zt;
  BatchLevel lev[MAXL];
};

struct BatchOut {
  int iterations, status, fp64_applies, pad;
  double rel_res, rel_res_true;
  double ms;               // time the CTA spent on this problem (globaltimer)
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

namespace cg = cooperative_groups;

// The CTAs that solve one problem together: one CTA, or a thread-block
// cluster whose CTAs split every loop and meet at cluster barriers.
struct Team {
  int rank, size, phase;
  __device__ long long start() const { return (long long)rank * BT + threadIdx.x; }
  __device__ long long stride() const { return (long long)size * BT; }
};

__device__ __forceinline__ void team_sync(const Team& tm) {
  if (tm.size == 1) __syncthreads();
  else cg::this_cluster().sync();
}

// Sum over every thread of the team, the same value in every thread (fixed
// order: every CTA of a cluster gets bitwise the same total, so all of them
// take the same branches).
__device__ __forceinline__ double team_sum(double v, double* sh, Team& tm) {
  __shared__ double slot[2];
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < BT / 32; ++w) t += sh[w];
  if (tm.size == 1) return t;
  cg::cluster_group cl = cg::this_cluster();
  if (threadIdx.x == 0) slot[tm.phase] = t;
  cl.sync();
  double tot = 0.0;
  for (int r = 0; r < tm.size; ++r) tot += *cl.map_shared_rank(&slot[tm.phase], r);
  tm.phase ^= 1;   // the other slot next time: readers of this one pass the next barrier first
  return tot;
}

template <typename T>
__device__ __forceinline__ void cubic(T t, T* b) {
  const T omt = T(1) - t;
  const T t2 = t * t;
  b[0] = omt * omt * (omt * T(1.0 / 6.0));
  b[1] = fma(t2, fma(t, T(0.5), T(-1.0)), T(2.0 / 3.0));
  b[2] = fma(fma(fma(t, T(-0.5), T(0.5)), t, T(0.5)), t, T(1.0 / 6.0));
  b[3] = t2 * (t * T(1.0 / 6.0));
}

// u += Phi_g'(Phi_g v): one thread per run (points of one cell), partial
// sums of the cell's (q+1)^P coefficients in registers, one global atomic per
// coefficient per run.
template <int P, typename T>
__device__ void cta_point(const BatchProblem& pb, const BatchLevel& L, const T* v, T* u, const Team& tm) {
  constexpr int NR = 1 << (2 * P);
  const LevelGeom& g = L.geom;
  for (long long r = tm.start(); r < L.nruns; r += tm.stride()) {
    const int i0 = L.run_begin[r], i1 = L.run_begin[r + 1];
    const unsigned long long pc = L.run_cell[r];
    long long base = 0;
    T tsh[P], inv[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const int c = (int)((pc >> (12 * p)) & 0xFFFull);
      base += (long long)c * g.stride[p];
      inv[p] = T(g.inv_h[p]);
      tsh[p] = T(g.lo[p] * g.inv_h[p] + (double)c);
    }
    auto gidx = [&](int k) -> long long {
      if (P == 3) return base + (k >> 4) * g.stride[0] + ((k >> 2) & 3) * g.stride[1] + (k & 3);
      if (P == 2) return base + (k >> 2) * g.stride[0] + (k & 3);
      return base + k;
    };
    constexpr bool VR = sizeof(T) == 4;   // FP32: the cell's v in registers; FP64: re-read (rare path)
    T vr[VR ? NR : 1], acc[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      if (VR) vr[VR ? k : 0] = v[gidx(k)];
      acc[k] = T(0);
    }
    auto V = [&](int k) -> T { return VR ? vr[VR ? k : 0] : v[gidx(k)]; };
    for (int i = i0; i < i1; ++i) {
      T bv[P][4];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const T xp = (sizeof(T) == 4 || !pb.x_f64) ? T(pb.xs32[(long long)p * pb.n + i])
                                                    : T(((const double*)pb.xs)[(long long)p * pb.n + i]);
        cubic(fma(xp, inv[p], -tsh[p]), bv[p]);
      }
      T s = T(0);
      if (P == 3) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          T s2 = T(0);
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            T s1 = T(0);
#pragma unroll
            for (int d = 0; d < 4; ++d) s1 = fma(bv[P - 1][d], V((a * 4 + b) * 4 + d), s1);
            s2 = fma(bv[P - 2][b], s1, s2);
          }
          s = fma(bv[0][a], s2, s);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const T t1 = s * bv[0][a];
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const T t2 = t1 * bv[1][b];
#pragma unroll
            for (int d = 0; d < 4; ++d) acc[(a * 4 + b) * 4 + d] = fma(t2, bv[2][d], acc[(a * 4 + b) * 4 + d]);
          }
        }
      } else if (P == 2) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          T s1 = T(0);
#pragma unroll
          for (int d = 0; d < 4; ++d) s1 = fma(bv[P - 1][d], V(a * 4 + d), s1);
          s = fma(bv[0][a], s1, s);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const T t1 = s * bv[0][a];
#pragma unroll
          for (int d = 0; d < 4; ++d) acc[a * 4 + d] = fma(t1, bv[1][d], acc[a * 4 + d]);
        }
      } else {
#pragma unroll
        for (int d = 0; d < 4; ++d) s = fma(bv[0][d], V(d), s);
#pragma unroll
        for (int d = 0; d < 4; ++d) acc[d] = fma(s, bv[0][d], acc[d]);
      }
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) atomicAdd(&u[gidx(k)], acc[k]);
  }
}

// u = scale * Lambda_g v by the three-term Kronecker recursion (one sweep per
// dimension, temporaries t[0..5]).
template <typename T>
__device__ void cta_penalty(const LevelGeom& g, const T* band, const T* v, T* out, T scale, T* const* t,
                            const Team& tm) {
  const int P = g.P;
  const long long K = g.K;
  const T* in0 = v;
  const T* in1 = nullptr;
  const T* in2 = nullptr;
  long long boff = 0;
  int ping = 0;
  for (int p = 0; p < P; ++p) {
    const int Jp = g.J[p];
    const long long strd = g.stride[p];
    const T* M = band + boff;
    const T* D1 = M + (long long)Jp * BAND;
    const T* D2 = M + 2LL * Jp * BAND;
    const bool first = p == 0, last = p == P - 1;
    T* o0 = t[3 * ping];
    T* o1 = t[3 * ping + 1];
    T* o2 = t[3 * ping + 2];
    for (long long k = tm.start(); k < K; k += tm.stride()) {
      const int j = (int)(((unsigned)k / (unsigned)strd) % (unsigned)Jp);   // K < 2^31 (checked by the host)
      T a0 = T(0), a1 = T(0), a2 = T(0);
      for (int o = -Q; o <= Q; ++o) {
        const int jj = j + o;
        if (jj < 0 || jj >= Jp) continue;
        const long long kk = k + (long long)o * strd;
        const T m = M[(long long)j * BAND + o + Q], d1 = D1[(long long)j * BAND + o + Q],
                d2 = D2[(long long)j * BAND + o + Q];
        if (first) {
          const T x = in0[kk];
          a0 = fma(m, x, a0);
          a1 = fma(d1, x, a1);
          a2 = fma(d2, x, a2);
        } else {
          const T x0 = in0[kk], x1 = in1[kk], x2 = in2[kk];
          a0 = fma(m, x0, a0);
          a1 = fma(m, x1, fma(d1, x0, a1));
          a2 = fma(m, x2, fma(T(2) * d1, x1, fma(d2, x0, a2)));
        }
      }
      if (last) out[k] = scale * a2;
      else {
        o0[k] = a0;
        o1[k] = a1;
        o2[k] = a2;
      }
    }
    team_sync(tm);
    in0 = o0;
    in1 = o1;
    in2 = o2;
    ping ^= 1;
    boff += 3LL * Jp * BAND;
  }
}

template <int P, typename T>
__device__ void cta_apply(const BatchProblem& pb, int lev, const T* v, T* u, T* const* t, const T* band,
                          const Team& tm) {
  const BatchLevel& L = pb.lev[lev - 1];
  if (sizeof(T) == 4 && L.st_f) {
    const LevelGeom& g = L.geom;
    for (long long k = tm.start(); k < g.K; k += tm.stride()) {
      int j[P];
      for (int p = 0; p < P; ++p) j[p] = (int)(((unsigned)k / (unsigned)g.stride[p]) % (unsigned)g.J[p]);
      T acc = T(0);
      for (int s = 0; s < L.S; ++s) {
        int ss = s;
        long long off = 0;
        bool ok = true;
        for (int p = P - 1; p >= 0; --p) {
          const int o = ss % BAND - Q;
          ss /= BAND;
          ok = ok && j[p] + o >= 0 && j[p] + o < g.J[p];
          off += (long long)o * g.stride[p];
        }
        if (ok) acc = fma(T(L.st_f[(long long)s * g.K + k]), v[k + off], acc);
      }
      u[k] = acc;
    }
    team_sync(tm);
    return;
  }
  cta_penalty<T>(L.geom, band, v, u, T(pb.lam), t, tm);
  cta_point<P, T>(pb, L, v, u, tm);
  team_sync(tm);
}

// c = I'(f - fb) (fb may be null); P sweeps through t6/t7.
__device__ void cta_restrict(const BatchProblem& pb, int g, const float* f, const float* fb, float* c,
                             const Team& tm) {
  const LevelGeom& Gf = pb.lev[g - 1].geom;
  const LevelGeom& Gc = pb.lev[g - 2].geom;
  const float* in = f;
  const float* inb = fb;
  for (int p = 0; p < pb.P; ++p) {
    long long inner = 1, outer = 1;
    for (int q = p + 1; q < pb.P; ++q) inner *= Gf.J[q];
    for (int q = 0; q < p; ++q) outer *= Gc.J[q];
    const int Jin = Gf.J[p], Jout = Gc.J[p];
    const long long Kout = outer * Jout * inner;
    float* out = p == pb.P - 1 ? c : pb.ftmp[6 + (p & 1)];
    for (long long k = tm.start(); k < Kout; k += tm.stride()) {
      const unsigned blk = (unsigned)Jout * (unsigned)inner, ku = (unsigned)k;
      const long long o = ku / blk;
      const unsigned rem = ku - (unsigned)o * blk;
      const int j = (int)(rem / (unsigned)inner);
      const long long ii = rem - (unsigned)j * (unsigned)inner;
      float s = 0.0f;
      for (int kk = 0; kk <= Q + 1; ++kk) {
        const int i = 2 * j - Q + kk;
        if (i < 0 || i >= Jin) continue;
        const long long src = (o * Jin + i) * inner + ii;
        const float val = inb ? in[src] - inb[src] : in[src];
        const float w = kk == 2 ? 0.75f : (kk == 0 || kk == 4) ? 0.125f : 0.5f;   // 2^-q binom(q+1, kk)
        s = fmaf(w, val, s);
      }
      out[k] = s;
    }
    team_sync(tm);
    in = out;
    inb = nullptr;
  }
}

// f -= I c.
__device__ void cta_prolong_sub(const BatchProblem& pb, int g, const float* c, float* f, const Team& tm) {
  const LevelGeom& Gf = pb.lev[g - 1].geom;
  const LevelGeom& Gc = pb.lev[g - 2].geom;
  const float* in = c;
  for (int p = 0; p < pb.P; ++p) {
    long long inner = 1, outer = 1;
    for (int q = p + 1; q < pb.P; ++q) inner *= Gc.J[q];
    for (int q = 0; q < p; ++q) outer *= Gf.J[q];
    const int Jin = Gc.J[p], Jout = Gf.J[p];
    const long long Kout = outer * Jout * inner;
    const bool last = p == pb.P - 1;
    float* out = last ? f : pb.ftmp[6 + (p & 1)];
    for (long long k = tm.start(); k < Kout; k += tm.stride()) {
      const unsigned blk = (unsigned)Jout * (unsigned)inner, ku = (unsigned)k;
      const long long o = ku / blk;
      const unsigned rem = ku - (unsigned)o * blk;
      const int i = (int)(rem / (unsigned)inner);
      const long long ii = rem - (unsigned)i * (unsigned)inner;
      float s = 0.0f;
      for (int kk = 0; kk <= Q + 1; ++kk) {
        const int num = i + Q - kk;
        if (num & 1) continue;
        const int j = num >> 1;
        if (j < 0 || j >= Jin) continue;
        const float w = kk == 2 ? 0.75f : (kk == 0 || kk == 4) ? 0.125f : 0.5f;
        s = fmaf(w, in[(o * Jin + j) * inner + ii], s);
      }
      if (last) out[k] -= s; else out[k] = s;
    }
    team_sync(tm);
    in = out;
  }
}

// alpha_G = V(b_G), FP32 (Algorithm 7 from zero).
template <int P>
__device__ void cta_vcycle(const BatchProblem& pb, const float* bG, float* xG, const Team& tm) {
  const int G = pb.G;
  float* const* t = pb.ftmp;
  auto B = [&](int g) -> float* { return g == G ? const_cast<float*>(bG) : pb.lev[g - 1].b; };
  auto X = [&](int g) -> float* { return g == G ? xG : pb.lev[g - 1].alpha; };
  for (int g = G; g >= 2; --g) {
    const BatchLevel& L = pb.lev[g - 1];
    const long long K = L.geom.K;
    float* x = X(g);
    const float* b = B(g);
    for (long long k = tm.start(); k < K; k += tm.stride()) x[k] = pb.nu1 >= 1 ? L.omega * L.dinv[k] * b[k] : 0.0f;
    team_sync(tm);
    for (int s = 1; s < pb.nu1; ++s) {
      cta_apply<P, float>(pb, g, x, L.u, t, L.band, tm);
      for (long long k = tm.start(); k < K; k += tm.stride()) x[k] = fmaf(L.omega * L.dinv[k], b[k] - L.u[k], x[k]);
      team_sync(tm);
    }
    if (pb.nu1 >= 1) cta_apply<P, float>(pb, g, x, L.u, t, L.band, tm);
    else {
      for (long long k = tm.start(); k < K; k += tm.stride()) L.u[k] = 0.0f;
      team_sync(tm);
    }
    cta_restrict(pb, g, L.u, b, B(g - 1), tm);
  }
  {
    // e = Z'(Z b) through an FP64 intermediate (a penalty temporary, unused here)
    const long long K1 = pb.lev[0].geom.K;
    const float* b1 = B(1);
    float* x1 = X(1);
    double* y1 = pb.dtmp[0];
    for (long long row = tm.start(); row < K1; row += tm.stride()) {
      double s = 0.0;
      for (long long c = 0; c < K1; ++c) s = fma(pb.coarse_z[row * K1 + c], (double)b1[c], s);
      y1[row] = s;
    }
    team_sync(tm);
    for (long long row = tm.start(); row < K1; row += tm.stride()) {
      double s = 0.0;
      for (long long c = 0; c < K1; ++c) s = fma(pb.coarse_zt[row * K1 + c], y1[c], s);
      x1[row] = (float)s;
    }
    team_sync(tm);
  }
  for (int g = 2; g <= G; ++g) {
    const BatchLevel& L = pb.lev[g - 1];
    const long long K = L.geom.K;
    float* x = X(g);
    const float* b = B(g);
    cta_prolong_sub(pb, g, X(g - 1), x, tm);
    for (int s = 0; s < pb.nu2; ++s) {
      cta_apply<P, float>(pb, g, x, L.u, t, L.band, tm);
      for (long long k = tm.start(); k < K; k += tm.stride()) x[k] = fmaf(L.omega * L.dinv[k], b[k] - L.u[k], x[k]);
      team_sync(tm);
    }
  }
}

template <int P>
__device__ void cta_solve(const BatchProblem& pb, BatchOut* out, double* sh, Team& tm) {
  double* const* dt = pb.dtmp;
  const int G = pb.G;
  const BatchLevel& LG = pb.lev[G - 1];
  const long long K = LG.geom.K;
  const double nb = pb.rhs_norm;
  double* x = pb.x;
  double* r = pb.r;
  double* z = pb.z;
  double* p = pb.p;
  double* v = pb.v;
  double* rp = pb.rprev;
  float* b32 = LG.b;
  float* a32 = LG.alpha;
  float* v32 = pb.ftmp[7];
  auto fp64_residual = [&]() -> double {   // r = rhs - A x in FP64 (Alg. 8 residual, recomputed)
    cta_penalty<double>(LG.geom, LG.band_d, x, v, pb.lam, dt, tm);
    cta_point<P, double>(pb, LG, x, v, tm);
    team_sync(tm);
    double s = 0.0;
    for (long long k = tm.start(); k < K; k += tm.stride()) {
      const double rk = pb.rhs[k] - v[k];
      r[k] = rk;
      s = fma(rk, rk, s);
    }
    return team_sum(s, sh, tm);
  };
  auto precondition = [&]() {
    for (long long k = tm.start(); k < K; k += tm.stride()) b32[k] = (float)r[k];
    team_sync(tm);
    cta_vcycle<P>(pb, b32, a32, tm);
    for (long long k = tm.start(); k < K; k += tm.stride()) z[k] = (double)a32[k];
    team_sync(tm);
  };
  double s = 0.0;
  for (long long k = tm.start(); k < K; k += tm.stride()) {
    x[k] = 0.0;
    r[k] = pb.rhs[k];
    s = fma(r[k], r[k], s);
  }
  double rr = team_sum(s, sh, tm);
  double rlast = sqrt(rr);
  double rel = rlast / nb;
  int it = 0, status = SPS_OK, f64 = 0;
  precondition();
  s = 0.0;
  for (long long k = tm.start(); k < K; k += tm.stride()) {
    p[k] = z[k];
    s = fma(r[k], z[k], s);
  }
  double rz = team_sum(s, sh, tm);
  while (rel > pb.tol && it < pb.max_iter) {
    for (long long k = tm.start(); k < K; k += tm.stride()) pb.p32[k] = (float)p[k];
    team_sync(tm);
    cta_apply<P, float>(pb, G, pb.p32, v32, pb.ftmp, LG.band, tm);
    s = 0.0;
    for (long long k = tm.start(); k < K; k += tm.stride()) {
      v[k] = (double)v32[k];
      s = fma(p[k], v[k], s);
    }
    const double pv = team_sum(s, sh, tm);
    const double w = rz / pv;
    if (!(pv > 0.0) || !isfinite(w)) {
      status = SPS_EBREAKDOWN;
      break;
    }
    s = 0.0;
    for (long long k = tm.start(); k < K; k += tm.stride()) {
      rp[k] = r[k];
      x[k] = fma(w, p[k], x[k]);
      const double rk = fma(-w, v[k], r[k]);
      r[k] = rk;
      s = fma(rk, rk, s);
    }
    rr = team_sum(s, sh, tm);
    ++it;
    double rn = sqrt(rr);
    rel = rn / nb;
    if (rel <= pb.tol || rn <= pb.ratio * rlast) {
      rr = fp64_residual();
      ++f64;
      rn = sqrt(rr);
      rel = rn / nb;
      rlast = rn;
      if (rel <= pb.tol) break;
    }
    precondition();
    double s1 = 0.0, s2 = 0.0;
    for (long long k = tm.start(); k < K; k += tm.stride()) {
      s1 = fma(z[k], r[k], s1);
      s2 = fma(z[k], rp[k], s2);
    }
    const double zr = team_sum(s1, sh, tm);
    const double zrp = team_sum(s2, sh, tm);
    const double beta = (zr - zrp) / rz;
    for (long long k = tm.start(); k < K; k += tm.stride()) p[k] = fma(beta, p[k], z[k]);
    team_sync(tm);
    rz = zr;
  }
  const double rt = sqrt(fp64_residual()) / nb;
  ++f64;
  if (threadIdx.x == 0 && tm.rank == 0) {
    out->iterations = it;
    out->rel_res = rel;
    out->rel_res_true = rt;
    out->fp64_applies = f64;
    out->status = status != SPS_OK ? status : (rt <= pb.tol ? SPS_OK : SPS_ENOCONV);
  }
  team_sync(tm);
}

// Persistent batched solver.  Phase 1 (C > 1): each cluster takes the next
// of the nbig largest problems from queue[0] and solves it with all C CTAs.
// Phase 2: every CTA takes the next remaining problem from queue[1] and
// solves it alone.  Problems arrive in decreasing cost order.
// C is the cluster size of the launch (1: no cluster); one instantiation
// serves every C, since the team's size is a run-time value anyway.
__global__ void __launch_bounds__(BT, 1) k_batch_solve(const BatchProblem* __restrict__ probs,
                                                       const int* __restrict__ order, int count, int nbig,
                                                       int* queue, BatchOut* __restrict__ outs, int C) {
  __shared__ double sh[BT / 32];
  __shared__ int cur;
  Team tm;
  tm.size = C;
  tm.rank = C > 1 ? (int)cg::this_cluster().block_rank() : 0;
  tm.phase = 0;
  for (;;) {
    int q;
    if (tm.size > 1) {
      cg::cluster_group cl = cg::this_cluster();
      if (threadIdx.x == 0 && tm.rank == 0) cur = atomicAdd(&queue[0], 1);
      cl.sync();
      q = *cl.map_shared_rank(&cur, 0);
      cl.sync();   // every CTA has read rank 0's slot before it is written again or the CTAs part
      if (q >= nbig) {
        tm.size = 1;   // phase 2: this CTA alone
        tm.rank = 0;
        continue;
      }
    } else {
      if (threadIdx.x == 0) cur = atomicAdd(&queue[1], 1);
      __syncthreads();
      q = nbig + cur;
      __syncthreads();
      if (q >= count) return;
    }
    const int i = order[q];
    const BatchProblem& pb = probs[i];
    const unsigned long long t0 = globaltimer_ns();
    if (pb.P == 1) cta_solve<1>(pb, outs + i, sh, tm);
    else if (pb.P == 2) cta_solve<2>(pb, outs + i, sh, tm);
    else cta_solve<3>(pb, outs + i, sh, tm);
    if (threadIdx.x == 0 && tm.rank == 0) outs[i].ms = (double)(globaltimer_ns() - t0) * 1e-6;
  }
}

}  // namespace

// ---------------------------------------------------------------- host side

namespace {

// Batch signature (count and every problem's P, K, n) -> the autotuner's shape.
std::mutex g_tune_mu;
std::map<unsigned long long, sps_batch_shape> g_tuned;

unsigned long long batch_signature(sps_plan* const* plans, int count) {
  unsigned long long h = 1469598103934665603ull ^ (unsigned long long)count;
  for (int i = 0; i < count; ++i) {
    const unsigned long long v[3] = {(unsigned long long)plans[i]->P,
                                     (unsigned long long)plans[i]->lev[plans[i]->G - 1].geom.K,
                                     (unsigned long long)plans[i]->n};
    for (unsigned long long x : v) {
      h ^= x + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
      h *= 1099511628211ull;
    }
  }
  return h;
}

// CTAs of the persistent launch for cluster size C (C = 1: no cluster), or 0
// when such clusters cannot be resident.
int batch_grid(int C, int count, int sms) {
  if (C == 1) return std::min(count, sms);
  cudaLaunchConfig_t oc = {};
  oc.gridDim = dim3(((sms + C - 1) / C) * C);
  oc.blockDim = dim3(BT);
  cudaLaunchAttribute oa;
  oa.id = cudaLaunchAttributeClusterDimension;
  oa.val.clusterDim.x = C;
  oa.val.clusterDim.y = 1;
  oa.val.clusterDim.z = 1;
  oc.attrs = &oa;
  oc.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, k_batch_solve, &oc) != cudaSuccess || clusters < 1) {
    cudaGetLastError();
    return 0;
  }
  return clusters * C;
}

struct BatchHost {
  std::vector<BatchProblem> hp;
  std::vector<double> cost;
  std::vector<int> order;   // problems by decreasing cost
};

void build_descriptors(sps_plan* const* plans, int count, double tol, BatchHost& bh) {
  bh.hp.assign(count, BatchProblem());
  bh.cost.assign(count, 0.0);
  for (int i = 0; i < count; ++i) {
    sps_plan* pl = plans[i];
    BatchProblem& b = bh.hp[i];
    std::memset(&b, 0, sizeof(b));
    b.P = pl->P;
    b.G = pl->G;
    b.x_f64 = pl->dtype == SPS_F64;
    b.nu1 = pl->opt.nu1;
    b.nu2 = pl->opt.nu2;
    b.max_iter = pl->opt.max_iter;
    b.n = pl->n;
    b.xs = pl->x_sorted;
    b.xs32 = pl->x32_sorted;
    b.lam = pl->lam;
    b.tol = tol;
    b.ratio = pl->opt.replace_ratio > 0 ? pl->opt.replace_ratio : 1e-2;
    b.rhs_norm = pl->rhs_norm;
    for (int k = 0; k < 8; ++k) b.ftmp[k] = pl->ftmp[k];
    for (int k = 0; k < 6; ++k) b.dtmp[k] = pl->dtmp[k];
    b.x = pl->x;
    b.r = pl->r;
    b.z = pl->z;
    b.p = pl->p;
    b.v = pl->v;
    b.rprev = pl->rprev;
    b.p32 = pl->p32;
    b.rhs = pl->rhs;
    b.coarse_z = pl->coarse_inv;
    b.coarse_zt = pl->coarse_invt;
    for (int g = 0; g < pl->G; ++g) {
      const Level& L = pl->lev[g];
      BatchLevel& bl = b.lev[g];
      bl.geom = L.geom;
      bl.run_begin = L.run_begin;
      bl.run_cell = L.run_cell;
      bl.nruns = L.nruns;
      bl.alpha = L.f.alpha;
      bl.b = L.f.b;
      bl.u = L.f.u;
      bl.dinv = L.f.dinv;
      bl.band = L.f.band;
      bl.band_d = L.d.band;
      bl.st_f = L.st_f;
      bl.S = L.S;
      bl.omega = (float)L.omega;
    }
    bh.cost[i] = (double)pl->n * pl->G * (double)(1 << (2 * pl->P)) + (double)pl->lev[pl->G - 1].geom.K * 50.0;
  }
  bh.order.resize(count);
  for (int i = 0; i < count; ++i) bh.order[i] = i;
  std::stable_sort(bh.order.begin(), bh.order.end(), [&](int a, int b) { return bh.cost[a] > bh.cost[b]; });
}

// The default split: problems whose cost exceeds a balanced share of the
// batch per CTA would bound the batch's time if one CTA solved them.
int default_big(const BatchHost& bh, int grid) {
  double total = 0.0;
  for (double c : bh.cost) total += c;
  const double share = total / std::max(grid, 1);
  int big = 0;
  while (big < (int)bh.order.size() && bh.cost[bh.order[big]] > share) ++big;
  return big;
}

// One persistent launch of the whole batch with cluster size C and `big`
// problems solved by clusters; per-problem outputs (status, times) in out.
int run_batch(sps_plan* const* plans, int count, const BatchHost& bh, int C, int big, int grid,
              std::vector<BatchOut>& out, cudaStream_t st) {
  const size_t sz_p = sizeof(BatchProblem) * count, sz_o = sizeof(int) * count, sz_r = sizeof(BatchOut) * count;
  const size_t off_o = (sz_p + 255) & ~(size_t)255, off_q = (off_o + sz_o + 255) & ~(size_t)255,
               off_r = off_q + 256, total = off_r + sz_r;
  char* dev = nullptr;
  if (cudaMalloc(&dev, total) != cudaSuccess) {
    cudaGetLastError();
    set_error("allocation of batch descriptors failed");
    return SPS_ENOMEM;
  }
  struct Free {
    char* p;
    ~Free() { cudaFree(p); }
  } guard{dev};
  SPS_CUDA(cudaMemcpyAsync(dev, bh.hp.data(), sz_p, cudaMemcpyHostToDevice, st));
  SPS_CUDA(cudaMemcpyAsync(dev + off_o, bh.order.data(), sz_o, cudaMemcpyHostToDevice, st));
  // capture: reset the queue, then the persistent kernel
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  cudaStream_t cs;
  SPS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  SPS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaMemsetAsync(dev + off_q, 0, 2 * sizeof(int), cs);
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(BT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = cs;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const BatchProblem* a0 = (const BatchProblem*)dev;
    const int* a1 = (const int*)(dev + off_o);
    int* a3 = (int*)(dev + off_q);
    BatchOut* a4 = (BatchOut*)(dev + off_r);
    const cudaError_t le = cudaLaunchKernelEx(&cfg, k_batch_solve, a0, a1, count, C > 1 ? big : 0, a3, a4, C);
    if (le != cudaSuccess) {
      cudaGraph_t dummy;
      cudaStreamEndCapture(cs, &dummy);
      cudaStreamDestroy(cs);
      return cuda_fail(le, "batched launch");
    }
  }
  SPS_CUDA(cudaStreamEndCapture(cs, &graph));
  SPS_CUDA(cudaGraphInstantiate(&exec, graph, 0));
  count_launches(1);
  SPS_CUDA(cudaStreamSynchronize(st));   // descriptors are in place before the graph runs on cs
  SPS_CUDA(cudaGraphLaunch(exec, cs));
  SPS_CUDA(cudaStreamSynchronize(cs));
  SPS_CUDA(cudaGetLastError());
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  out.resize(count);
  SPS_CUDA(cudaMemcpy(out.data(), dev + off_r, sz_r, cudaMemcpyDeviceToHost));
  return SPS_OK;
}

// Makespan of the persistent queues with measured per-problem times: `grid`
// CTAs as grid / C teams take the `big` costliest problems (times tc); a team
// that finds that queue empty splits into C single CTAs, which take the rest
// in cost order (times t1).  C = 1: single CTAs throughout.
double simulate_batch(const std::vector<int>& order, const std::vector<double>& t1, const std::vector<double>& tc,
                      int C, int big, int grid) {
  using Ev = std::pair<double, int>;   // (time free, team size)
  std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> q;
  const int teams = C > 1 ? grid / C : grid;
  for (int t = 0; t < teams; ++t) q.push({0.0, C > 1 ? C : 1});
  int next_big = 0, next = C > 1 ? big : 0;
  const int n = (int)order.size();
  double makespan = 0.0;
  while (!q.empty()) {
    const Ev e = q.top();
    q.pop();
    if (e.second > 1) {
      if (next_big < big) {
        const double f = e.first + tc[order[next_big++]];
        makespan = std::max(makespan, f);
        q.push({f, e.second});
      } else {
        for (int k = 0; k < e.second; ++k) q.push({e.first, 1});
      }
    } else if (next < n) {
      const double f = e.first + t1[order[next++]];
      makespan = std::max(makespan, f);
      q.push({f, 1});
    }
  }
  return makespan;
}

void fill_results(sps_plan* const* plans, int count, double* const* coefs, int mem, const std::vector<BatchOut>& out,
                  sps_result* res, int* worst, cudaStream_t st, int* rc) {
  *worst = SPS_OK;
  for (int i = 0; i < count; ++i) {
    sps_plan* pl = plans[i];
    const long long K = pl->lev[pl->G - 1].geom.K;
    const cudaError_t e = cudaMemcpyAsync(coefs[i], pl->x, sizeof(double) * K,
                                          mem == SPS_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
      *rc = cuda_fail(e, "copy of batch coefficients");
      return;
    }
    if (res) {
      sps_result& r = res[i];
      std::memset(&r, 0, sizeof(r));
      r.status = out[i].status;
      r.iterations = out[i].iterations;
      r.rel_res = out[i].rel_res;
      r.rel_res_true = out[i].rel_res_true;
      r.fp64_applies = out[i].fp64_applies;
      r.solve_ms = out[i].ms;
    }
    if (out[i].status != SPS_OK && *worst == SPS_OK) *worst = out[i].status;
  }
}

}  // namespace

// Host side of sps_solve_batch: descriptors, cost order, shape, graph launch.
int solve_batch(sps_plan* const* plans, int count, double* const* coefs, int mem, double tol,
                const sps_batch_shape* shape, sps_result* res, sps_batch_shape* used, cudaStream_t st) {
  BatchHost bh;
  build_descriptors(plans, count, tol, bh);
  int sms = 0, devid = 0;
  SPS_CUDA(cudaGetDevice(&devid));
  SPS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, devid));
  sps_batch_shape sh = {2, -1, 0.0};   // clusters of two CTAs for the costliest problems
  if (shape) {
    sh = *shape;
  } else {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(batch_signature(plans, count));
    if (it != g_tuned.end()) sh = it->second;
  }
  int C = sh.cluster;
  int grid = batch_grid(C, count, sms);
  if (grid == 0) {   // such clusters cannot be resident: one CTA per problem
    C = 1;
    grid = batch_grid(1, count, sms);
  }
  const int big = C == 1 ? 0 : (sh.big < 0 ? default_big(bh, grid) : std::min(sh.big, count));
  std::vector<BatchOut> out;
  SPS_TRY(run_batch(plans, count, bh, C, big, grid, out, st));
  if (used) {
    used->cluster = C;
    used->big = big;
    used->predicted_ms = sh.predicted_ms;
  }
  int worst = SPS_OK, rc = SPS_OK;
  fill_results(plans, count, coefs, mem, out, res, &worst, st, &rc);
  if (rc != SPS_OK) return rc;
  SPS_CUDA(cudaStreamSynchronize(st));
  if (worst != SPS_OK) set_error("at least one problem of the batch did not converge");
  return worst;
}

double batch_makespan(const int* order, const double* t1, const double* tc, int n, int C, int big, int grid) {
  return simulate_batch(std::vector<int>(order, order + n), std::vector<double>(t1, t1 + n),
                        std::vector<double>(tc, tc + n), C, big, grid);
}

// The autotuner: solve the batch once per cluster size C in {1, 2, 4, 8} with
// every problem on a team of C CTAs, keep the measured time of every problem
// for every C, then choose the cluster size and the number of problems solved
// by clusters whose simulated batch time is the shortest.
int tune_batch(sps_plan* const* plans, int count, double* const* coefs, int mem, double tol, sps_batch_shape* best,
               cudaStream_t st) {
  BatchHost bh;
  build_descriptors(plans, count, tol, bh);
  int sms = 0, devid = 0;
  SPS_CUDA(cudaGetDevice(&devid));
  SPS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, devid));
  const int cands[4] = {1, 2, 4, 8};
  std::vector<double> times[4];
  int grids[4] = {0, 0, 0, 0};
  std::vector<BatchOut> out;
  for (int c = 0; c < 4; ++c) {
    const int C = cands[c];
    grids[c] = batch_grid(C, count, sms);
    if (grids[c] == 0) continue;
    SPS_TRY(run_batch(plans, count, bh, C, count, grids[c], out, st));
    times[c].resize(count);
    for (int i = 0; i < count; ++i) times[c][i] = out[i].ms;
  }
  sps_batch_shape pick = {1, 0, simulate_batch(bh.order, times[0], times[0], 1, 0, grids[0])};
  for (int c = 1; c < 4; ++c) {
    if (grids[c] == 0) continue;
    for (int big = 1; big <= count; ++big) {
      const double m = simulate_batch(bh.order, times[0], times[c], cands[c], big, grids[c]);
      if (m < pick.predicted_ms) pick = {cands[c], big, m};
    }
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[batch_signature(plans, count)] = pick;
  }
  if (best) *best = pick;
  // leave the coefficients of the last tuning run in coefs (a valid solve)
  int worst = SPS_OK, rc = SPS_OK;
  fill_results(plans, count, coefs, mem, out, nullptr, &worst, st, &rc);
  if (rc != SPS_OK) return rc;
  SPS_CUDA(cudaStreamSynchronize(st));
  return SPS_OK;
}

}  // namespace sps

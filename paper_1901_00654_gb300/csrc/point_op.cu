// The point operator u += Phi_g'(Phi_g v) on one grid level (Section 3.2,
// hierarchy: all n points on every level), fused from the transposed
// Khatri-Rao product s_i = (kron_p Phi_p[i,.])' v (Algorithm 4) and the
// Khatri-Rao product u = sum_i s_i kron_p Phi_p[i,.] (Algorithm 3), with the
// (q+1)^P tensor-product basis values of each point formed on the fly from
// its coordinates.  The same kernel with s_i = 1 and squared basis values
// gives diag(Phi_g'Phi_g) (Algorithm 5), and with s_i = y_i the right-hand
// side Phi'y (first line of Algorithm 8).
//
// Work decomposition (GB300 design, not the paper's loop order):
//  * The points are sorted by cell, so the points of one level cell form a
//    contiguous "run" (at most RUN_MAX points).  A CTA owns the runs of one
//    tile of ts^P cells; the (ts+q)^P coefficients its points can touch are
//    staged in shared memory.
//  * The item's point coordinates and run table are contiguous after the
//    sort and are staged in shared memory before the run loop, all copies in
//    flight at once: TMA bulk copies for the coordinates, cp.async for the
//    run table and the coefficient patch (FP64 levels read precomputed basis
//    values instead of coordinates).
//  * A group of TPP = 4^(P-R) lanes takes one run at a time, R = 2 or 3 being
//    the number of trailing dimensions a lane holds: each lane owns 4^R of the
//    cell's (q+1)^P coefficients (16 or 64) and keeps their partial sums in
//    registers while it walks the run, so the scatter costs one shared-memory
//    atomic per coefficient per run instead of one per point.  The gather is
//    sum-factorised over the lane's R dimensions and reduced across the group
//    with shuffles.  The layout per level is chosen by the autotuner.
//  * The shared accumulator is flushed to global memory with atomics, since
//    neighbouring tiles overlap in q layers of coefficients.  For P >= 3 the
//    patch is staged and flushed by rows along the last dimension (one
//    multi-index decode per row).
//  * On coordinate-based levels the groups of a warp walk their runs in step
//    (the warp loops to its longest run, finished groups carry weight 0), and
//    the FP32 16-sum layout does its multiply-adds on packed float pairs.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "sps_internal.h"

namespace sps {

namespace {

__host__ __device__ constexpr int ipow4(int e) { return e <= 0 ? 1 : 4 * ipow4(e - 1); }

// ---- asynchronous copies into shared memory (sm_90+ PTX) ----
// A CTA's prologue issues every copy of its work item at once -- the run table
// and the coefficient patch with cp.async, the contiguous coordinate ranges
// with one TMA bulk copy per dimension, completed on an mbarrier -- so that it
// waits for one memory round trip instead of one per dependent load chain.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Copy BYTES (4, 8 or 16) from global to shared memory; zero-fill when !valid
// (src is then not read).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_addr(dst)), "l"(src), "n"(BYTES),
               "r"(valid ? BYTES : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// One arrival that also announces `bytes` of bulk copies to come.
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
// TMA bulk copy global -> shared: both addresses 16-byte aligned, bytes a
// multiple of 16; completes `bytes` on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// Wait for phase `parity` of the mbarrier, giving up after about a second of
// SM clocks (returns false then).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity) {
  const long long t0 = clock64();
  for (;;) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > (1LL << 31)) return false;
  }
}

// Values of the q+1 = 4 cubic B-splines that are nonzero on a cell, at local
// coordinate t in [0, 1]: b[m] belongs to basis function (cell + m).  They are
// the four polynomial pieces of the uniform cubic B-spline (de Boor 1978).
template <typename T>
__device__ __forceinline__ void cubic_basis(T t, T* b) {
  const T omt = T(1) - t;
  const T t2 = t * t;
  b[0] = omt * omt * (omt * T(1.0 / 6.0));
  b[1] = fma(t2, fma(t, T(0.5), T(-1.0)), T(2.0 / 3.0));
  b[2] = fma(fma(fma(t, T(-0.5), T(0.5)), t, T(0.5)), t, T(1.0 / 6.0));
  b[3] = t2 * (t * T(1.0 / 6.0));
}

// PRE (FP64 only): 1 -- the 4P basis values of every point on this level were
// computed once at set-up and are read from `pre` ([point][dimension][m])
// instead of being re-evaluated from the coordinates in every sweep.  On
// GB300 an FP64 operation costs about as much as moving 40 bytes from HBM, so
// streaming 8*4P bytes per point is cheaper than the 12P FP64 operations.
// 2 (P = 3, four-lane layout) -- per point the 4 pieces of the first dimension
// and the 16 products of the other two, so each lane's gather and scatter are
// 16 multiply-adds each with no product formation (160 bytes per point).
// RR: dimensions held in a lane's registers (0 = min(P, 3)); the FP32
// kernel for P = 3 uses RR = 2, i.e. four lanes per run with 16 coefficients
// each, for four times the resident warps of the one-lane layout.
template <int P, typename T, typename CT, int MODE, int PRE = 0, int RR = 0>
__global__ void __launch_bounds__(POINT_THREADS, PRE == 2 ? 5 : 2)
k_point(const WorkItem* __restrict__ items, const unsigned* __restrict__ item_span,
        const unsigned* __restrict__ item_cell, const CT* __restrict__ xs, long long n,
        const double* __restrict__ ys, const T* __restrict__ v, T* __restrict__ u, LevelGeom geom,
        int* __restrict__ err, const double* __restrict__ pre = nullptr) {
  constexpr int R = RR > 0 ? RR : (P < 3 ? P : 3);   // dimensions held in a lane's registers
  constexpr int NR = ipow4(R);
  constexpr int F = P - R;                    // leading dimensions fixed per lane
  constexpr int TPP = ipow4(F);               // lanes per run
  constexpr bool VREG = sizeof(T) == 4;       // FP32: cache the cell's v in registers
  // FP32 apply with 16 sums per lane: packed two-wide multiply-adds
  constexpr bool FF2 = VREG && R == 2 && PRE == 0 && MODE == PT_APPLY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* acc = reinterpret_cast<T*>(smem_raw);
  T* vp = acc + geom.patch;
  // the item's points (contiguous after the sort) are staged here, one array per dimension
  const size_t xoff = ((size_t)(MODE == PT_APPLY ? 2 : 1) * geom.patch * sizeof(T) + 15) & ~(size_t)15;
  CT* xsh = reinterpret_cast<CT*>(smem_raw + xoff);

  const WorkItem it = items[blockIdx.x];
  const int pbeg = it.pbeg;
  const int npts = it.npts;
  // The item's run table (in processing order, built at set-up) is staged in
  // shared memory with the coordinates, so the run loop reads no global memory
  // before its points.  Items hold at most MAXR runs (the item builder's cap).
  constexpr int MAXR = 128;
  constexpr int CB = 32 / P;                        // bits per dimension of a packed cell offset
  constexpr unsigned CMASK = CB >= 32 ? 0xffffffffu : (1u << CB) - 1u;
  __shared__ unsigned int s_span[MAXR];             // first | end << 16, relative to pbeg
  __shared__ unsigned int s_cell[MAXR];             // cell - tile origin, CB bits per dimension
  const int nr = min(it.run_hi - it.run_lo, MAXR);
  // Coordinates: dimension p of the item's points is the contiguous range
  // [p n + pbeg, p n + pbeg + npts) of xs.  Its 16-byte-aligned middle is
  // fetched by one TMA bulk copy, the at most 2 (E16 - 1) elements at its ends
  // by cp.async; in shared memory the range starts at offset sh_p = (p n +
  // pbeg) mod E16 of a 16-byte-aligned array of XS elements, so the middle
  // lands 16-byte aligned too.  xo[p] + i indexes coordinate p of point i.
  constexpr int E16 = 16 / (int)sizeof(CT);
  const int XS = (npts + 2 * E16 - 1) / E16 * E16;
  int xo[P];
#pragma unroll
  for (int p = 0; p < P; ++p) xo[p] = 0;
  __shared__ __align__(8) unsigned long long s_bar;   // completion of the bulk copies
  __shared__ int s_fail;
  if (!PRE) {
    // The host sizes the shared memory by the largest item.  Never stage past
    // it: if an item ever exceeded it, its contribution is skipped and the
    // error flag makes the calling sps_* return SPS_EINTERNAL.
    unsigned dsm;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsm));
    if (xoff + (size_t)P * XS * sizeof(CT) > dsm || (smem_addr(xsh) & 15u) != 0) {
      if (threadIdx.x == 0) atomicOr(err, ERR_SMEM);
      return;
    }
    const unsigned bar = smem_addr(&s_bar);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const long long g0 = (long long)p * n + pbeg, g1 = g0 + npts;
      const int sh = (int)(g0 % E16);
      xo[p] = p * XS + sh - pbeg;
      CT* dst = xsh + p * XS + sh;                       // element g0 goes to dst[0]
      const long long a0 = (g0 + E16 - 1) / E16 * E16;   // aligned middle [a0, a1)
      const long long a1 = g1 / E16 * E16;
      const long long h1 = a0 < g1 ? a0 : g1, t0 = a1 > a0 ? a1 : a0;
      // ends: lanes 0 .. E16-2 the head [g0, h1), lanes E16-1 .. 2E16-3 the tail [t0, g1)
      const int k = threadIdx.x;
      if (k < E16 - 1) {
        if (g0 + k < h1) cp_async<sizeof(CT)>(dst + k, xs + g0 + k, true);
      } else if (k < 2 * (E16 - 1)) {
        const long long e = t0 + (k - (E16 - 1));
        if (e < g1) cp_async<sizeof(CT)>(dst + (e - g0), xs + e, true);
      }
    }
    if (threadIdx.x == 0) {
      s_fail = 0;
      mbar_init(bar, 1);
      unsigned bytes = 0;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const long long g0 = (long long)p * n + pbeg, g1 = g0 + npts;
        const long long a0 = (g0 + E16 - 1) / E16 * E16, a1 = g1 / E16 * E16;
        if (a1 > a0) bytes += (unsigned)((a1 - a0) * sizeof(CT));
      }
      mbar_arrive_expect_tx(bar, bytes);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const long long g0 = (long long)p * n + pbeg, g1 = g0 + npts;
        const long long a0 = (g0 + E16 - 1) / E16 * E16, a1 = g1 / E16 * E16;
        if (a1 > a0)
          bulk_g2s(xsh + p * XS + (int)(g0 % E16) + (int)(a0 - g0), xs + a0, (unsigned)((a1 - a0) * sizeof(CT)), bar);
      }
    }
  }
  for (int e = threadIdx.x; e < nr; e += blockDim.x) {
    cp_async<4>(&s_span[e], item_span + it.run_lo + e, true);
    cp_async<4>(&s_cell[e], item_cell + it.run_lo + e, true);
  }
  // ROWS (P >= 3): the patch is staged and flushed by rows along the last
  // dimension (stride 1 in the coefficient array), so a thread decodes one
  // row's multi-index for its E_{P-1} elements instead of one per element.
  constexpr bool ROWS = P >= 3;
  const int EL = geom.E[P - 1];
  const int nrows = geom.patch / EL;
  const int nl = min(EL, geom.J[P - 1] - it.c0[P - 1]);   // in-range elements of a row
  auto row_start = [&](int r, bool& inb) -> long long {
    int rem = r;
    long long gi = it.c0[P - 1];
    inb = true;
#pragma unroll
    for (int p = P - 2; p >= 0; --p) {
      const int qd = (int)(((float)rem + 0.5f) * geom.invE[p]);   // rem / E, as below
      const int m = rem - qd * geom.E[p];
      rem = qd;
      const int j = it.c0[p] + m;
      inb = inb && j < geom.J[p];
      gi += (long long)j * geom.stride[p];
    }
    return gi;
  };
  if (ROWS) {
    uint4* a4 = reinterpret_cast<uint4*>(acc);
    const int n4 = (int)((size_t)geom.patch * sizeof(T) / 16);
    for (int e = threadIdx.x; e < n4; e += blockDim.x) a4[e] = make_uint4(0u, 0u, 0u, 0u);
    for (int e = n4 * (int)(16 / sizeof(T)) + threadIdx.x; e < geom.patch; e += blockDim.x) acc[e] = T(0);
    if (MODE == PT_APPLY) {
      for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
        bool inb;
        const long long gi = row_start(r, inb);
        T* dst = vp + r * EL;
        for (int m = 0; m < EL; ++m) {
          const bool ok = inb && m < nl;
          cp_async<sizeof(T)>(dst + m, ok ? v + gi + m : v, ok);
        }
      }
    }
  }
  for (int e = threadIdx.x; !ROWS && e < geom.patch; e += blockDim.x) {
    acc[e] = T(0);
    if (MODE == PT_APPLY) {
      int rem = e;
      long long gi = 0;
      bool inb = true;
#pragma unroll
      for (int p = P - 1; p >= 0; --p) {
        // rem / E by a float product: (rem + 0.5) / E is at least 1/(2E) away
        // from an integer, far more than the rounding error for rem < 2^16
        const int qd = (int)(((float)rem + 0.5f) * geom.invE[p]);
        const int m = rem - qd * geom.E[p];
        rem = qd;
        const int j = it.c0[p] + m;
        inb = inb && j < geom.J[p];
        gi += (long long)j * geom.stride[p];
      }
      cp_async<sizeof(T)>(&vp[e], inb ? v + gi : v, inb);
    }
  }
  if (!PRE && threadIdx.x == 0) {
    // bounded wait: on time-out the item is skipped and reported, after a
    // second bounded wait so that no copy is still landing when the CTA exits
    if (!mbar_wait_bounded(smem_addr(&s_bar), 0)) {
      atomicOr(err, ERR_WAIT);
      s_fail = 1;
      mbar_wait_bounded(smem_addr(&s_bar), 0);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  if (!PRE && s_fail) return;

  const int group = threadIdx.x / TPP;
  const int glane = threadIdx.x % TPP;
  const int ngroups = blockDim.x / TPP;
  unsigned gmask = 0xffffffffu;
  if (TPP < 32) gmask = ((1u << TPP) - 1u) << ((threadIdx.x & 31) & ~(TPP - 1));
  int mfix[F > 0 ? F : 1];
  {
    int l = glane;
#pragma unroll
    for (int p = F - 1; p >= 0; --p) {
      mfix[p] = l & 3;
      l >>= 2;
    }
  }
  T inv[P], loinv[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    inv[p] = T(geom.inv_h[p]);
    loinv[p] = T(geom.lo[p] * geom.inv_h[p]);
  }
  // A lane needs only piece mfix[p] of the cubic in each fixed dimension: its
  // power-basis coefficients c0 + c1 t + c2 t^2 + c3 t^3, from the four pieces
  // (1-t)^3/6, (3t^3-6t^2+4)/6, (-3t^3+3t^2+3t+1)/6 and t^3/6.  Used by the
  // register-light layouts (RR > 0); elsewhere the 4F extra registers would
  // cost occupancy, and the lane evaluates all four pieces and selects.
  // P = 4, FP32, 16 lanes per run: the 16 (dimension, piece) values of a
  // point are computed once each -- lane l evaluates piece l & 3 of dimension
  // l >> 2 -- and shared with shuffles, instead of every lane evaluating the
  // pieces of all four dimensions.
  constexpr bool SHARED_BASIS = P == 4 && R == 2 && !PRE && sizeof(T) == 4 && MODE == PT_APPLY;
  const int sdim = SHARED_BASIS ? (glane >> 2) : 0;
  const int spc = glane & 3;
  const T sinv = sdim == 0 ? inv[0] : sdim == 1 ? inv[P > 1 ? 1 : 0] : sdim == 2 ? inv[P > 2 ? 2 : 0]
                                                                                 : inv[P > 3 ? 3 : 0];
  const int xos = sdim == 0 ? xo[0] : sdim == 1 ? xo[P > 1 ? 1 : 0] : sdim == 2 ? xo[P > 2 ? 2 : 0]
                                                                              : xo[P > 3 ? 3 : 0];
  const T sc0 = spc == 0 ? T(1.0 / 6.0) : spc == 1 ? T(2.0 / 3.0) : spc == 2 ? T(1.0 / 6.0) : T(0);
  const T sc1 = spc == 0 ? T(-0.5) : spc == 1 ? T(0) : spc == 2 ? T(0.5) : T(0);
  const T sc2 = spc == 0 ? T(0.5) : spc == 1 ? T(-1) : spc == 2 ? T(0.5) : T(0);
  const T sc3 = spc == 0 ? T(-1.0 / 6.0) : spc == 1 ? T(0.5) : spc == 2 ? T(-0.5) : T(1.0 / 6.0);
  constexpr bool ONEPIECE = RR > 0 && F > 0 && !SHARED_BASIS;
  constexpr int NF = ONEPIECE ? F : 1;
  T pc0[NF], pc1[NF], pc2[NF], pc3[NF];
#pragma unroll
  for (int p = 0; p < (ONEPIECE ? F : 0); ++p) {
    const int m = mfix[p];
    pc0[p] = m == 0 ? T(1.0 / 6.0) : m == 1 ? T(2.0 / 3.0) : m == 2 ? T(1.0 / 6.0) : T(0);
    pc1[p] = m == 0 ? T(-0.5) : m == 1 ? T(0) : m == 2 ? T(0.5) : T(0);
    pc2[p] = m == 0 ? T(0.5) : m == 1 ? T(-1) : m == 2 ? T(0.5) : T(0);
    pc3[p] = m == 0 ? T(-1.0 / 6.0) : m == 1 ? T(0.5) : m == 2 ? T(-0.5) : T(1.0 / 6.0);
  }

  // one run per thread when TPP == 1 (runs_per_item == ngroups): which lanes hold one
  const unsigned has_run_mask = __ballot_sync(0xffffffffu, group < nr);
  // UNIFORM (coordinate-based levels): the groups of a warp take consecutive
  // runs and walk them in step.  The warp loops to its longest run; a group
  // past the end of its own run, or without a run, repeats its first point
  // with weight 0.  The point loop then never diverges, and the shuffles
  // inside it run on the converged warp.
  constexpr bool UNIFORM = !PRE;
  if (UNIFORM) gmask = 0xffffffffu;
  const int wfirst = (threadIdx.x & ~31) / TPP;   // this warp's first group
  for (int e = group; UNIFORM ? e - group + wfirst < nr : e < nr; e += ngroups) {
    const bool act = !UNIFORM || e < nr;
    const int er = act ? e : e - group + wfirst;   // a run of this warp's round (< nr)
    const unsigned span = s_span[er], pc = s_cell[er];
    const int i0 = pbeg + (int)(span & 0xFFFFu), i1 = pbeg + (int)(span >> 16);
    const int len = act ? i1 - i0 : 0;
    const int nsteps = UNIFORM ? (int)__reduce_max_sync(0xffffffffu, (unsigned)len) : len;
    T tsh[P];
    int base = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      int o = (int)((pc >> (CB * p)) & CMASK);
      const int c = it.c0[p] + o;
      if (p < F) o += mfix[p];
      base += o * geom.Es[p];
      tsh[p] = loinv[p] + T(c);   // t = x * inv - (lo * inv + c)
    }
    const T stsh = sdim == 0 ? tsh[0] : sdim == 1 ? tsh[P > 1 ? 1 : 0] : sdim == 2 ? tsh[P > 2 ? 2 : 0]
                                                                                : tsh[P > 3 ? 3 : 0];
    const int e0 = R >= 3 ? geom.Es[P - 3] : 0;
    const int e1 = R >= 2 ? geom.Es[P - 2] : 0;
    auto vidx = [&](int k) -> int {
      if (R == 3) return base + (k >> 4) * e0 + ((k >> 2) & 3) * e1 + (k & 3);
      if (R == 2) return base + (k >> 2) * e1 + (k & 3);
      return base + k;
    };
    T vr[VREG ? NR : 1];
    if (VREG && MODE == PT_APPLY) {
#pragma unroll
      for (int k = 0; k < NR; ++k) vr[VREG ? k : 0] = vp[vidx(k)];
    }
    T accr[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) accr[k] = T(0);

    for (int k = 0; k < nsteps; ++k) {
      const bool live = k < len;
      const int i = live ? i0 + k : i0;
      if constexpr (PRE == 2 && P == 3 && R == 2 && MODE == PT_APPLY) {
        // products b2[b] b3[d] precomputed: 16 multiply-adds each way per lane
        const double* q = pre + (long long)i * PRE2_STRIDE;
        const T ba = T(q[mfix[0]]);
        const double2* q2 = reinterpret_cast<const double2*>(q + 4);
        T pr[16];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const double2 t = __ldg(q2 + k);
          pr[2 * k] = T(t.x);
          pr[2 * k + 1] = T(t.y);
        }
        T g = T(0);
#pragma unroll
        for (int k = 0; k < 16; ++k) g = fma(pr[k], VREG ? vr[VREG ? k : 0] : vp[vidx(k)], g);
        g *= ba;
#pragma unroll
        for (int o = TPP / 2; o >= 1; o >>= 1) g += __shfl_xor_sync(gmask, g, o, TPP);
        const T w = g * ba;
#pragma unroll
        for (int k = 0; k < 16; ++k) accr[k] = fma(w, pr[k], accr[k]);
        continue;
      }
      T bv[P][4];
      T fixw = live ? T(1) : T(0);
      if (PRE) {
        const double2* q = reinterpret_cast<const double2*>(pre + (long long)i * (4 * P));
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const double2 a = __ldg(q + 2 * p), b = __ldg(q + 2 * p + 1);
          bv[p][0] = T(a.x);
          bv[p][1] = T(a.y);
          bv[p][2] = T(b.x);
          bv[p][3] = T(b.y);
        }
#pragma unroll
        for (int p = 0; p < F; ++p) {   // select without dynamic register indexing
          const int m = mfix[p];
          fixw *= m == 0 ? bv[p][0] : m == 1 ? bv[p][1] : m == 2 ? bv[p][2] : bv[p][3];
        }
      } else if (SHARED_BASIS) {
        const T t = fma(T(xsh[xos + i]), sinv, -stsh);
        const T val = fma(fma(fma(sc3, t, sc2), t, sc1), t, sc0);
        fixw *= __shfl_sync(gmask, val, mfix[0], TPP) * __shfl_sync(gmask, val, 4 + mfix[F > 1 ? 1 : 0], TPP);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          bv[P - 2][m] = __shfl_sync(gmask, val, 8 + m, TPP);
          bv[P - 1][m] = __shfl_sync(gmask, val, 12 + m, TPP);
        }
      } else {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const T xp = T(xsh[xo[p] + i]);
          const T t = fma(xp, inv[p], -tsh[p]);
          if (ONEPIECE && p < F) {
            const int q = ONEPIECE ? p : 0;
            T b = fma(fma(fma(pc3[q], t, pc2[q]), t, pc1[q]), t, pc0[q]);
            if (MODE == PT_DIAG) b *= b;
            fixw *= b;
          } else {
            cubic_basis(t, bv[p]);
            if (MODE == PT_DIAG) {
#pragma unroll
              for (int m = 0; m < 4; ++m) bv[p][m] *= bv[p][m];
            }
            if (!ONEPIECE && p < F) {   // select without dynamic register indexing
              const int m = mfix[p];
              fixw *= m == 0 ? bv[p][0] : m == 1 ? bv[p][1] : m == 2 ? bv[p][2] : bv[p][3];
            }
          }
        }
      }
      if constexpr (FF2) {
        // Packed FP32 pairs (two multiply-adds per instruction): the 16
        // products z[a][d] = b_{P-2,a} b_{P-1,d} are formed once and used by
        // the gather and by the scatter.
        const float2 b3a = make_float2(bv[P - 1][0], bv[P - 1][1]);
        const float2 b3b = make_float2(bv[P - 1][2], bv[P - 1][3]);
        float2 z[4][2];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const float2 ba = make_float2(bv[P - 2][a], bv[P - 2][a]);
          z[a][0] = __fmul2_rn(ba, b3a);
          z[a][1] = __fmul2_rn(ba, b3b);
        }
        float2 ga = __fmul2_rn(z[0][0], make_float2(vr[0], vr[1]));
        float2 gb = __fmul2_rn(z[0][1], make_float2(vr[2], vr[3]));
#pragma unroll
        for (int a = 1; a < 4; ++a) {
          ga = __ffma2_rn(z[a][0], make_float2(vr[4 * a], vr[4 * a + 1]), ga);
          gb = __ffma2_rn(z[a][1], make_float2(vr[4 * a + 2], vr[4 * a + 3]), gb);
        }
        T g = ((ga.x + ga.y) + (gb.x + gb.y)) * fixw;
#pragma unroll
        for (int o = TPP / 2; o >= 1; o >>= 1) g += __shfl_xor_sync(gmask, g, o, TPP);
        const T w = g * fixw;
        const float2 w2 = make_float2(w, w);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float2 c = make_float2(accr[4 * a + 2 * h], accr[4 * a + 2 * h + 1]);
            c = __ffma2_rn(w2, z[a][h], c);
            accr[4 * a + 2 * h] = c.x;
            accr[4 * a + 2 * h + 1] = c.y;
          }
        }
        continue;
      }
      T s;
      if (MODE == PT_APPLY) {
        T g = T(0);
        if (R == 3) {
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            T s2 = T(0);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              T s1 = T(0);
#pragma unroll
              for (int d = 0; d < 4; ++d) {
                const int k = (a * 4 + b) * 4 + d;
                const T vv = VREG ? vr[VREG ? k : 0] : vp[vidx(k)];
                s1 = fma(bv[P - 1][d], vv, s1);
              }
              s2 = fma(bv[P - 2][b], s1, s2);
            }
            g = fma(bv[P - 3][a], s2, g);
          }
        } else if (R == 2) {
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            T s1 = T(0);
#pragma unroll
            for (int d = 0; d < 4; ++d) {
              const int k = a * 4 + d;
              const T vv = VREG ? vr[VREG ? k : 0] : vp[vidx(k)];
              s1 = fma(bv[P - 1][d], vv, s1);
            }
            g = fma(bv[P - 2][a], s1, g);
          }
        } else {
#pragma unroll
          for (int d = 0; d < 4; ++d) {
            const T vv = VREG ? vr[VREG ? d : 0] : vp[vidx(d)];
            g = fma(bv[P - 1][d], vv, g);
          }
        }
        g *= fixw;
#pragma unroll
        for (int o = TPP / 2; o >= 1; o >>= 1) g += __shfl_xor_sync(gmask, g, o, TPP);
        s = g;
      } else if (MODE == PT_RHS) {
        s = T(ys[i]);
      } else {
        s = T(1);
      }
      const T w = s * fixw;
      if (R == 3) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const T t1 = w * bv[P - 3][a];
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const T t2 = t1 * bv[P - 2][b];
#pragma unroll
            for (int d = 0; d < 4; ++d) accr[(a * 4 + b) * 4 + d] = fma(t2, bv[P - 1][d], accr[(a * 4 + b) * 4 + d]);
          }
        }
      } else if (R == 2) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const T t1 = w * bv[P - 2][a];
#pragma unroll
          for (int d = 0; d < 4; ++d) accr[a * 4 + d] = fma(t1, bv[P - 1][d], accr[a * 4 + d]);
        }
      } else {
#pragma unroll
        for (int d = 0; d < 4; ++d) accr[d] = fma(w, bv[P - 1][d], accr[d]);
      }
    }
    bool flushed = false;
    if (TPP == 1 && NR == 64 && has_run_mask == 0xffffffffu) {
      // Coarse levels put a whole warp's runs in one cell: reduce the 64 sums
      // across the warp first (reduce-scatter; lane l ends with the totals of
      // coefficients 2l and 2l+1) instead of 32-way conflicting atomics.
      const unsigned pc0 = __shfl_sync(0xffffffffu, pc, 0);
      if (__all_sync(0xffffffffu, pc == pc0)) {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int step = 0; step < 5; ++step) {
          const int o = 16 >> step, h = 32 >> step;
          const bool up = (lane & o) != 0;
#pragma unroll
          for (int i = 0; i < h; ++i) {
            const T send = up ? accr[i] : accr[i + h];
            const T keep = up ? accr[i + h] : accr[i];
            accr[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
          }
        }
        atomicAdd(&acc[vidx(2 * lane)], accr[0]);
        atomicAdd(&acc[vidx(2 * lane + 1)], accr[1]);
        flushed = true;
      }
    }
    if (!flushed && act) {
#pragma unroll
      for (int k = 0; k < NR; ++k) atomicAdd(&acc[vidx(k)], accr[k]);
    }
  }
  __syncthreads();

  if constexpr (ROWS) {
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
      bool inb;
      const long long gi = row_start(r, inb);
      if (!inb) continue;
      const T* src = acc + r * EL;
      for (int m = 0; m < nl; ++m) {
        const T a = src[m];
        if (a != T(0)) atomicAdd(&u[gi + m], a);
      }
    }
  } else {
    for (int e = threadIdx.x; e < geom.patch; e += blockDim.x) {
      const T a = acc[e];
      if (a == T(0)) continue;
      int rem = e;
      long long gi = 0;
      bool inb = true;
#pragma unroll
      for (int p = P - 1; p >= 0; --p) {
        const int qd = (int)(((float)rem + 0.5f) * geom.invE[p]);
        const int m = rem - qd * geom.E[p];
        rem = qd;
        const int j = it.c0[p] + m;
        inb = inb && j < geom.J[p];
        gi += (long long)j * geom.stride[p];
      }
      if (inb) atomicAdd(&u[gi], a);
    }
  }
}

// Event records of the profile: inside a stream capture an ordinary
// cudaEventRecord only marks a dependency, so the record is captured as an
// external event-record node, which replays of the graph then record.
inline cudaError_t record_event(cudaEvent_t e, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  if (cs == cudaStreamCaptureStatusActive) return cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
  return cudaEventRecord(e, st);
}

// Event pool for sps_profile_begin / sps_profile_end.
struct ProfileState {
  bool active = false;
  int used = 0;
  std::vector<cudaEvent_t> ev;   // pairs
  std::vector<char> in_graph;    // pair recorded by a graph node (harvested per replay)
  double harvest_ms = 0.0;
  long long harvest_cnt = 0;
};
ProfileState g_prof;
constexpr int PROFILE_MAX = 8192;

// cudaFuncSetAttribute applies to the current device only: each kernel
// instantiation records the devices (bit per ordinal) it was raised on.
template <typename Kern>
int raise_smem(Kern kern, std::atomic<unsigned long long>& done) {
  int dev = 0;
  SPS_CUDA(cudaGetDevice(&dev));
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(done.load(std::memory_order_acquire) & bit)) {
    SPS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)POINT_SMEM_MAX));
    done.fetch_or(bit, std::memory_order_release);
  }
  return SPS_OK;
}

template <typename Kern, typename... Args>
int launch_k(Kern kern, std::atomic<unsigned long long>& attr, int grid, size_t smem, cudaStream_t st,
             Args... args) {
  SPS_TRY(raise_smem(kern, attr));
  kern<<<grid, POINT_THREADS, smem, st>>>(args...);
  SPS_CHECK_LAUNCH("point operator");
  return SPS_OK;
}

template <int P, typename T, typename CT, int MODE>
int launch_point(sps_plan* pl, const Level& L, const T* v, T* u, cudaStream_t st) {
  if (L.nitems == 0) return SPS_OK;
  // patch accumulator (+ patch of v) + staged coordinates of the largest item's points
  // (each dimension's staged range is shifted by up to 16 bytes and rounded up)
  const size_t pts = (size_t)L.max_item_pts;
  const size_t smem = (size_t)(MODE == PT_APPLY ? 2 : 1) * L.geom.patch * sizeof(T) + pts * P * sizeof(CT) +
                      48 * P + 16;
  if (smem > POINT_SMEM_MAX) {
    set_error("tile too large for the point operator's shared memory");
    return SPS_EINVAL;
  }
  const bool timed = MODE == PT_APPLY && g_prof.active && g_prof.used < PROFILE_MAX;
  if (timed) SPS_CUDA(record_event(g_prof.ev[2 * g_prof.used], st));
  const CT* xs = sizeof(CT) == 4 ? (const CT*)pl->x32_sorted : (const CT*)pl->x_sorted;
  if ((reinterpret_cast<uintptr_t>(xs) & 15) != 0) {   // the bulk copies need 16-byte alignment
    set_error("sorted coordinates not 16-byte aligned");
    return SPS_EINTERNAL;
  }
  int rc = SPS_OK;
  bool done = false;
  if constexpr (sizeof(T) == 8 && MODE == PT_APPLY) {
    if (L.pre) {
      const size_t smem_pre = (size_t)2 * L.geom.patch * sizeof(T) + 16;
      // P = 3, 4: the 4^(P-2)-lane layout (16 sums per lane) when chosen: about
      // 10 % more FP64 operations per point, but four times the resident warps
      // and runs of more similar length within a warp
      if constexpr (P == 3) {
        if (L.lanes_r == 2 && L.pre2) {   // products of the last two dimensions precomputed
          static std::atomic<unsigned long long> a22{0};
          rc = launch_k(k_point<P, T, CT, MODE, 2, 2>, a22, L.nitems, smem_pre, st, L.items, L.item_span, L.item_cell,
                        xs, pl->n, (const double*)pl->y_sorted, v, u, L.geom, pl->err_flag,
                        (const double*)L.pre2);
          done = true;
        }
      }
      if constexpr (P == 3 || P == 4) {
        if (!done && L.lanes_r == 2) {
          static std::atomic<unsigned long long> a12{0};
          rc = launch_k(k_point<P, T, CT, MODE, 1, 2>, a12, L.nitems, smem_pre, st, L.items, L.item_span, L.item_cell,
                        xs, pl->n, (const double*)pl->y_sorted, v, u, L.geom, pl->err_flag,
                        (const double*)L.pre);
          done = true;
        }
      }
      if (!done) {
        static std::atomic<unsigned long long> a1{0};
        rc = launch_k(k_point<P, T, CT, MODE, 1>, a1, L.nitems, smem_pre, st, L.items, L.item_span, L.item_cell,
                      xs, pl->n, (const double*)pl->y_sorted, v, u, L.geom, pl->err_flag,
                      (const double*)L.pre);
        done = true;
      }
    }
  }
  if (!done) {
    // FP32: two register layouts per run -- R = 2 dimensions in a lane's
    // registers (4^(P-2) lanes per run, 16 accumulators each) or R = 3
    // (4^(P-3) lanes, 64 accumulators).  P = 3 defaults to R = 2 (more resident
    // warps); the autotuner may pick either for the apply of P = 3 and P = 4.
    constexpr bool TWO_LAYOUTS = sizeof(T) == 4 && (P == 3 || (P == 4 && MODE == PT_APPLY));
    const int rsel = L.lanes_r ? L.lanes_r : (P == 3 ? 2 : 3);
    bool launched = false;
    if constexpr (TWO_LAYOUTS) {
      if (!launched && (rsel == 2 || (P == 3 && MODE != PT_APPLY))) {
        static std::atomic<unsigned long long> ar2{0};
        rc = launch_k(k_point<P, T, CT, MODE, 0, 2>, ar2, L.nitems, smem, st, L.items, L.item_span, L.item_cell,
                      xs, pl->n, (const double*)pl->y_sorted, v, u, L.geom, pl->err_flag,
                      (const double*)nullptr);
        launched = true;
      }
      if constexpr (P == 4 && MODE == PT_APPLY) {
        if (!launched && rsel == 3) {   // 4 lanes per run, each evaluating one piece of dimension 1
          static std::atomic<unsigned long long> ar3{0};
          rc = launch_k(k_point<P, T, CT, MODE, 0, 3>, ar3, L.nitems, smem, st, L.items, L.item_span,
                        L.item_cell, xs, pl->n, (const double*)pl->y_sorted, v, u, L.geom, pl->err_flag,
                        (const double*)nullptr);
          launched = true;
        }
      }
    }
    if (!launched) {
      static std::atomic<unsigned long long> a0{0};
      rc = launch_k(k_point<P, T, CT, MODE>, a0, L.nitems, smem, st, L.items, L.item_span, L.item_cell,
                    xs, pl->n, (const double*)pl->y_sorted, v, u, L.geom, pl->err_flag, (const double*)nullptr);
    }
  }
  if (rc != SPS_OK) return rc;
  if (timed) SPS_CUDA(record_event(g_prof.ev[2 * g_prof.used++ + 1], st));
  return SPS_OK;
}

template <int P, typename T>
int dispatch_mode(sps_plan* pl, const Level& L, int mode, const T* v, T* u, cudaStream_t st) {
  if (pl->dtype == SPS_F64 && sizeof(T) == 8) {
    if (mode == PT_APPLY) return launch_point<P, T, double, PT_APPLY>(pl, L, v, u, st);
    if (mode == PT_DIAG) return launch_point<P, T, double, PT_DIAG>(pl, L, v, u, st);
    return launch_point<P, T, double, PT_RHS>(pl, L, v, u, st);
  }
  if (mode == PT_APPLY) return launch_point<P, T, float, PT_APPLY>(pl, L, v, u, st);
  if (mode == PT_DIAG) return launch_point<P, T, float, PT_DIAG>(pl, L, v, u, st);
  return launch_point<P, T, float, PT_RHS>(pl, L, v, u, st);
}

}  // namespace

size_t point_apply_smem(const sps_plan* pl, const LevelGeom& G, bool fp32) {
  const size_t t = fp32 ? 4 : 8;
  const size_t ct = (fp32 || pl->dtype == SPS_F32) ? 4 : 8;
  const size_t pts = (size_t)runs_per_item(pl->P) * RUN_MAX;
  return 2 * (size_t)G.patch * t + pts * pl->P * ct + 48 * pl->P + 16;   // the FP64 basis-value path needs less
}

template <typename T>
int point_op(sps_plan* pl, int g, int mode, const T* v, T* u, cudaStream_t st) {
  const Level& L = pl->lev[g - 1];
  switch (pl->P) {
    case 1: return dispatch_mode<1, T>(pl, L, mode, v, u, st);
    case 2: return dispatch_mode<2, T>(pl, L, mode, v, u, st);
    case 3: return dispatch_mode<3, T>(pl, L, mode, v, u, st);
    case 4: return dispatch_mode<4, T>(pl, L, mode, v, u, st);
    case 5: return dispatch_mode<5, T>(pl, L, mode, v, u, st);
  }
  set_error("unsupported dimension");
  return SPS_EINVAL;
}

namespace {

// The 4P basis values of every point on level g (one thread per run).
template <int P, typename CT>
__global__ void k_basis_pre(const int* __restrict__ run_begin, const unsigned long long* __restrict__ run_cell,
                            int nruns, const CT* __restrict__ xs, long long n, LevelGeom geom,
                            double* __restrict__ pre) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nruns; r += gridDim.x * blockDim.x) {
    const unsigned long long pc = run_cell[r];
    double tsh[P], inv[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const int c = (int)((pc >> (12 * p)) & 0xFFFull);
      inv[p] = geom.inv_h[p];
      tsh[p] = geom.lo[p] * geom.inv_h[p] + (double)c;
    }
    for (int i = run_begin[r]; i < run_begin[r + 1]; ++i) {
#pragma unroll
      for (int p = 0; p < P; ++p) {
        double b[4];
        cubic_basis(fma((double)xs[(long long)p * n + i], inv[p], -tsh[p]), b);
#pragma unroll
        for (int m = 0; m < 4; ++m) pre[(long long)i * (4 * P) + 4 * p + m] = b[m];
      }
    }
  }
}

// P = 3: the 4 pieces of dimension 1 and the 16 products of the pieces of
// dimensions 2 and 3 of every point (one thread per run), [point][20].
template <typename CT>
__global__ void k_basis_pre2(const int* __restrict__ run_begin, const unsigned long long* __restrict__ run_cell,
                             int nruns, const CT* __restrict__ xs, long long n, LevelGeom geom,
                             double* __restrict__ pre2) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nruns; r += gridDim.x * blockDim.x) {
    const unsigned long long pc = run_cell[r];
    double tsh[3], inv[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      const int c = (int)((pc >> (12 * p)) & 0xFFFull);
      inv[p] = geom.inv_h[p];
      tsh[p] = geom.lo[p] * geom.inv_h[p] + (double)c;
    }
    for (int i = run_begin[r]; i < run_begin[r + 1]; ++i) {
      double b[3][4];
#pragma unroll
      for (int p = 0; p < 3; ++p) cubic_basis(fma((double)xs[(long long)p * n + i], inv[p], -tsh[p]), b[p]);
      double* o = pre2 + (long long)i * PRE2_STRIDE;
#pragma unroll
      for (int m = 0; m < 4; ++m) o[m] = b[0][m];
#pragma unroll
      for (int k = 0; k < 16; ++k) o[4 + k] = b[1][k >> 2] * b[2][k & 3];
    }
  }
}

template <int P>
int basis_pre_launch(sps_plan* pl, const Level& L, cudaStream_t st) {
  const int blocks = grid_blocks(L.nruns, 128);
  if (pl->dtype == SPS_F64)
    k_basis_pre<P, double><<<blocks, 128, 0, st>>>(L.run_begin, L.run_cell, L.nruns, (const double*)pl->x_sorted,
                                                   pl->n, L.geom, L.pre);
  else
    k_basis_pre<P, float><<<blocks, 128, 0, st>>>(L.run_begin, L.run_cell, L.nruns, pl->x32_sorted, pl->n,
                                                  L.geom, L.pre);
  SPS_CHECK_LAUNCH("basis precompute");
  if constexpr (P == 3) {
    if (L.pre2) {
      if (pl->dtype == SPS_F64)
        k_basis_pre2<double><<<blocks, 128, 0, st>>>(L.run_begin, L.run_cell, L.nruns, (const double*)pl->x_sorted,
                                                     pl->n, L.geom, L.pre2);
      else
        k_basis_pre2<float><<<blocks, 128, 0, st>>>(L.run_begin, L.run_cell, L.nruns, pl->x32_sorted, pl->n,
                                                    L.geom, L.pre2);
      SPS_CHECK_LAUNCH("basis product precompute");
    }
  }
  return SPS_OK;
}

}  // namespace

int basis_precompute(sps_plan* pl, int g, cudaStream_t st) {
  const Level& L = pl->lev[g - 1];
  switch (pl->P) {
    case 1: return basis_pre_launch<1>(pl, L, st);
    case 2: return basis_pre_launch<2>(pl, L, st);
    case 3: return basis_pre_launch<3>(pl, L, st);
    case 4: return basis_pre_launch<4>(pl, L, st);
    case 5: return basis_pre_launch<5>(pl, L, st);
  }
  set_error("unsupported dimension");
  return SPS_EINVAL;
}

template int point_op<double>(sps_plan*, int, int, const double*, double*, cudaStream_t);
template int point_op<float>(sps_plan*, int, int, const float*, float*, cudaStream_t);

int profile_begin() {
  if (g_prof.ev.empty()) {
    g_prof.ev.resize(2 * PROFILE_MAX);
    for (auto& e : g_prof.ev) SPS_CUDA(cudaEventCreate(&e));
    g_prof.in_graph.assign(PROFILE_MAX, 0);
  }
  g_prof.used = 0;
  std::fill(g_prof.in_graph.begin(), g_prof.in_graph.end(), 0);
  g_prof.harvest_ms = 0.0;
  g_prof.harvest_cnt = 0;
  g_prof.active = true;
  return SPS_OK;
}

bool profile_active() { return g_prof.active; }
int profile_mark() { return g_prof.used; }

// Pairs [first, last) were recorded into a graph being captured: they are
// timed per replay by profile_harvest, not at profile_end.
void profile_capture_end(int first, int last) {
  for (int i = first; i < last && i < PROFILE_MAX; ++i) g_prof.in_graph[i] = 1;
}

// After a replay of a graph holding pairs [first, last) has completed.
int profile_harvest(int first, int last) {
  if (!g_prof.active) return SPS_OK;
  for (int i = first; i < last; ++i) {
    float t = 0.0f;
    SPS_CUDA(cudaEventElapsedTime(&t, g_prof.ev[2 * i], g_prof.ev[2 * i + 1]));
    g_prof.harvest_ms += t;
    ++g_prof.harvest_cnt;
  }
  return SPS_OK;
}

int profile_end(double* ms, unsigned long long* launches) {
  g_prof.active = false;
  double tot = g_prof.harvest_ms;
  unsigned long long cnt = (unsigned long long)g_prof.harvest_cnt;
  for (int i = 0; i < g_prof.used; ++i) {
    if (g_prof.in_graph[i]) continue;
    SPS_CUDA(cudaEventSynchronize(g_prof.ev[2 * i + 1]));
    float t = 0.0f;
    SPS_CUDA(cudaEventElapsedTime(&t, g_prof.ev[2 * i], g_prof.ev[2 * i + 1]));
    tot += t;
    ++cnt;
  }
  *ms = tot;
  *launches = cnt;
  return SPS_OK;
}

}  // namespace sps

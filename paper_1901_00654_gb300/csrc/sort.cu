// Cell index, Morton key, stable LSD radix sort and the per-level work lists.
//
// The cell of a coordinate is c = min(floor((x - lo) * (N / (hi - lo))), N - 1)
// in the precision of the input (a point at hi belongs to the last cell); it
// is the knot interval that carries the q+1 nonzero B-splines of the point
// (support of the B-splines, Section 2.1).  The key interleaves the bits of
// the finest-level cell multi-index from the most significant bit down, so
// that after one stable sort the points of every cell and of every aligned
// power-of-two block of cells, on every grid level, are contiguous.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>
#include <cmath>

#include "sps_internal.h"

namespace sps {

namespace {

struct KeyParams {
  int P, L;
  int N[MAXP];
  double lo[MAXP], hi[MAXP], inv[MAXP];
};

template <typename CT>
__global__ void k_keys(const CT* __restrict__ x, const CT* __restrict__ y, long long n, KeyParams kp,
                       unsigned long long* __restrict__ keys, unsigned int* __restrict__ perm,
                       int* __restrict__ err) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    unsigned int c[MAXP];
    bool bad = !isfinite((double)y[i]);   // a non-finite response would make Phi'y non-finite
    for (int p = 0; p < kp.P; ++p) {
      CT xv = x[i * kp.P + p];
      double xd = (double)xv;
      if (!(xd >= kp.lo[p] && xd <= kp.hi[p])) bad = true;   // also rejects NaN
      CT u = (CT)(xv - (CT)kp.lo[p]);
      u = (CT)(u * (CT)kp.inv[p]);
      long long ci = bad ? 0 : (long long)floor((double)u);
      if (ci > kp.N[p] - 1) ci = kp.N[p] - 1;
      if (ci < 0) ci = 0;
      c[p] = (unsigned int)ci;
    }
    if (bad) atomicOr(err, ERR_DOMAIN);
    unsigned long long key = 0;
    for (int b = kp.L - 1; b >= 0; --b)
      for (int p = 0; p < kp.P; ++p) key = (key << 1) | (unsigned long long)((c[p] >> b) & 1u);
    keys[i] = key;
    perm[i] = (unsigned int)i;
  }
}

// ---------------------------------------------------------------- radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_BINS = 256;

__global__ void k_rs_hist(const unsigned long long* __restrict__ keys, long long n, int shift,
                          int ntiles, unsigned int* __restrict__ hist) {
  __shared__ unsigned int h[RS_BINS];
  for (int b = threadIdx.x; b < RS_BINS; b += blockDim.x) h[b] = 0;
  __syncthreads();
  long long base = (long long)blockIdx.x * RS_TILE;
  for (int k = 0; k < RS_ITEMS; ++k) {
    long long i = base + k * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xFF], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < RS_BINS; b += blockDim.x) hist[(long long)b * ntiles + blockIdx.x] = h[b];
}

// Exclusive scan of a uint array in place, one block of 1024 threads.
__global__ void k_scan_u32_single(unsigned int* __restrict__ a, long long n) {
  __shared__ unsigned int warp_sums[32];
  __shared__ unsigned int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (long long base = 0; base < n; base += blockDim.x) {
    long long i = base + threadIdx.x;
    unsigned int v = i < n ? a[i] : 0u;
    unsigned int s = v;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned int t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    if (lane == 31) warp_sums[wid] = s;
    __syncthreads();
    if (wid == 0) {
      unsigned int w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0u;
      for (int o = 1; o < 32; o <<= 1) {
        unsigned int t = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += t;
      }
      warp_sums[lane] = w;
    }
    __syncthreads();
    unsigned int excl = carry + (wid > 0 ? warp_sums[wid - 1] : 0u) + s - v;
    if (i < n) a[i] = excl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + v;
    __syncthreads();
  }
}

__global__ void k_rs_scatter(const unsigned long long* __restrict__ kin, const unsigned int* __restrict__ vin,
                             unsigned long long* __restrict__ kout, unsigned int* __restrict__ vout,
                             long long n, int shift, int ntiles, const unsigned int* __restrict__ offs) {
  __shared__ unsigned int base[RS_BINS];
  __shared__ unsigned int wcnt[RS_THREADS / 32][RS_BINS];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int b = threadIdx.x; b < RS_BINS; b += blockDim.x)
    base[b] = offs[(long long)b * ntiles + blockIdx.x];
  const long long tile0 = (long long)blockIdx.x * RS_TILE;
  for (int k = 0; k < RS_ITEMS; ++k) {
    for (int e = threadIdx.x; e < (RS_THREADS / 32) * RS_BINS; e += blockDim.x) (&wcnt[0][0])[e] = 0;
    __syncthreads();
    long long i = tile0 + k * RS_THREADS + threadIdx.x;
    bool valid = i < n;
    unsigned long long key = valid ? kin[i] : 0ull;
    unsigned int d = valid ? (unsigned int)((key >> shift) & 0xFF) : RS_BINS;   // sentinel for the tail
    unsigned int peers = __match_any_sync(0xffffffffu, d);
    unsigned int rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[wid][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      unsigned int off = base[d] + rank;
      for (int w = 0; w < wid; ++w) off += wcnt[w][d];
      kout[off] = key;
      vout[off] = vin[i];
    }
    __syncthreads();
    for (int b = threadIdx.x; b < RS_BINS; b += blockDim.x) {
      unsigned int t = 0;
      for (int w = 0; w < RS_THREADS / 32; ++w) t += wcnt[w][b];
      base[b] += t;
    }
    __syncthreads();
  }
}

template <typename CT>
__global__ void k_gather(const CT* __restrict__ x, const CT* __restrict__ y,
                         const unsigned int* __restrict__ perm, long long n, int P,
                         CT* __restrict__ xs, float* __restrict__ xs32, double* __restrict__ ys) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    long long s = perm[i];
    for (int p = 0; p < P; ++p) {
      const CT xv = x[s * P + p];
      xs[(long long)p * n + i] = xv;
      if (xs32) xs32[(long long)p * n + i] = (float)xv;   // FP32 copy for the FP32 kernels
    }
    ys[i] = (double)y[s];
  }
}

// ---------------------------------------------------------------- segments
__device__ __forceinline__ long long lower_bound_key(const unsigned long long* keys, long long n,
                                                     unsigned long long v) {
  long long lo = 0, hi = n;
  while (lo < hi) {
    long long mid = (lo + hi) >> 1;
    if (keys[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void deinterleave(unsigned long long id, int P, int bits, int* c) {
  for (int p = 0; p < P; ++p) c[p] = 0;
  for (int b = 0; b < bits; ++b)
    for (int p = P - 1; p >= 0; --p) {
      c[p] |= (int)(id & 1ull) << b;
      id >>= 1;
    }
}

// Runs per level cell: ceil(points / RUN_MAX), of balanced lengths (a cell
// of 17 points gives runs of 9 and 8, not 16 and 1), so that the lanes of a
// warp, which walk runs of similar rank, finish together.  cnt has ncell + 1
// entries.
__global__ void k_cell_runs(const unsigned long long* __restrict__ keys, long long n, long long ncell,
                            int sh, unsigned int* __restrict__ cnt, unsigned int* __restrict__ pts) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c <= ncell;
       c += (long long)gridDim.x * blockDim.x) {
    if (c == ncell) { cnt[c] = 0; continue; }
    long long a = lower_bound_key(keys, n, (unsigned long long)c << sh);
    long long b = lower_bound_key(keys, n, (unsigned long long)(c + 1) << sh);
    cnt[c] = (unsigned int)((b - a + RUN_MAX - 1) / RUN_MAX);
    pts[c] = (unsigned int)(b - a);
  }
}

__global__ void k_fill_runs(const unsigned long long* __restrict__ keys, long long n, long long ncell,
                            int sh, int P, int cbits, const unsigned int* __restrict__ off,
                            const unsigned int* __restrict__ pts,
                            int* __restrict__ run_begin, unsigned long long* __restrict__ run_cell,
                            long long nruns) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    unsigned int o0 = off[c], o1 = off[c + 1];
    if (o0 == o1) continue;
    long long a = lower_bound_key(keys, n, (unsigned long long)c << sh);
    const long long m = pts[c];
    const long long k = o1 - o0;   // ceil(m / RUN_MAX) runs of floor(m/k) or ceil(m/k) points
    const long long len = m / k, extra = m - len * k;   // the first `extra` runs hold one more
    int cc[MAXP];
    deinterleave((unsigned long long)c, P, cbits, cc);
    unsigned long long packed = 0;
    for (int p = 0; p < P; ++p) packed |= (unsigned long long)cc[p] << (12 * p);
    for (unsigned int r = o0; r < o1; ++r) {
      const long long j = r - o0;
      run_begin[r] = (int)(a + j * len + (j < extra ? j : extra));
      run_cell[r] = packed;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) run_begin[nruns] = (int)n;
}

// Items per tile: runs of the tile split into chunks of at most `cap`.
__global__ void k_tile_items(const unsigned int* __restrict__ run_off, long long ntile, int cells_per_tile_log,
                             int cap, unsigned int* __restrict__ cnt) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t <= ntile;
       t += (long long)gridDim.x * blockDim.x) {
    if (t == ntile) { cnt[t] = 0; continue; }
    unsigned int r0 = run_off[t << cells_per_tile_log], r1 = run_off[(t + 1) << cells_per_tile_log];
    cnt[t] = (r1 - r0 + cap - 1) / cap;
  }
}

__global__ void k_fill_items(const unsigned int* __restrict__ run_off, const unsigned int* __restrict__ ioff,
                             long long ntile, int cells_per_tile_log, int cap, int P, int tbits, int tb,
                             const int* __restrict__ run_begin, WorkItem* __restrict__ items) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ntile;
       t += (long long)gridDim.x * blockDim.x) {
    unsigned int i0 = ioff[t], i1 = ioff[t + 1];
    if (i0 == i1) continue;
    unsigned int r0 = run_off[t << cells_per_tile_log], r1 = run_off[(t + 1) << cells_per_tile_log];
    int tc[MAXP];
    deinterleave((unsigned long long)t, P, tbits, tc);
    for (unsigned int k = i0; k < i1; ++k) {
      WorkItem it;
      it.run_lo = (int)(r0 + (k - i0) * cap);
      it.run_hi = (int)min((unsigned int)(r0 + (k - i0 + 1) * cap), r1);
      it.pbeg = run_begin[it.run_lo];
      it.npts = run_begin[it.run_hi] - it.pbeg;
      for (int p = 0; p < MAXP; ++p) it.c0[p] = p < P ? (tc[p] << tb) : 0;
      for (int p = 0; p < (int)(sizeof(it.pad) / sizeof(int)); ++p) it.pad[p] = 0;
      items[k] = it;
    }
  }
}

// Order the runs of each work item by length, longest first (bitonic sort of
// at most 128 runs in shared memory, ties by run index), so that the lanes of
// a warp walk runs of similar length; write the order and, per run slot, the
// run's span relative to the item's first point and its cell relative to the
// tile origin (32/P bits per dimension).
__global__ void k_sort_item_runs(const WorkItem* __restrict__ items, const int* __restrict__ run_begin,
                                 const unsigned long long* __restrict__ run_cell, int P,
                                 int* __restrict__ run_order, unsigned* __restrict__ item_span,
                                 unsigned* __restrict__ item_cell) {
  __shared__ long long key[128];
  const WorkItem it = items[blockIdx.x];
  const int nr = it.run_hi - it.run_lo;
  const int t = threadIdx.x;
  if (t < 128) {
    if (t < nr) {
      const int r = it.run_lo + t;
      const long long len = run_begin[r + 1] - run_begin[r];
      key[t] = ((128 - len) << 20) | (long long)t;    // ascending key = longest first, then index
    } else {
      key[t] = 0x7fffffffffffffffLL;
    }
  }
  __syncthreads();
  for (int k = 2; k <= 128; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int l = t ^ j;
      if (t < 128 && l > t) {
        const bool asc = (t & k) == 0;
        const long long a = key[t], b = key[l];
        if ((a > b) == asc) {
          key[t] = b;
          key[l] = a;
        }
      }
      __syncthreads();
    }
  if (t < nr) {
    const int r = it.run_lo + (int)(key[t] & 0xFFFFF);
    run_order[it.run_lo + t] = r;
    const int cb = 32 / P;
    const unsigned long long pc = run_cell[r];
    unsigned cl = 0;
    for (int p = 0; p < P; ++p) cl |= (unsigned)((int)((pc >> (12 * p)) & 0xFFFull) - it.c0[p]) << (cb * p);
    item_span[it.run_lo + t] = (unsigned)(run_begin[r] - it.pbeg) | ((unsigned)(run_begin[r + 1] - it.pbeg) << 16);
    item_cell[it.run_lo + t] = cl;
  }
}

// Point count of every work item.
__global__ void k_item_npts(const WorkItem* __restrict__ items, const int* __restrict__ run_begin, int nitems,
                            unsigned int* __restrict__ npts) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nitems; k += gridDim.x * blockDim.x)
    npts[k] = (unsigned)items[k].npts;
}

__global__ void k_permute_items(const WorkItem* __restrict__ in, const unsigned int* __restrict__ perm, int nitems,
                                WorkItem* __restrict__ out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nitems; k += gridDim.x * blockDim.x) out[k] = in[perm[k]];
}

int ensure_seg(sps_plan* pl, long long need) {
  if (pl->seg_cap >= need) return SPS_OK;
  pfree(pl, pl->seg_tmp);
  pl->seg_cap = 0;
  SPS_TRY(palloc(pl, &pl->seg_tmp, need));
  pl->seg_cap = need;
  return SPS_OK;
}

int scan_u32(unsigned int* a, long long n, cudaStream_t st) {
  k_scan_u32_single<<<1, 1024, 0, st>>>(a, n);
  SPS_CHECK_LAUNCH("scan");
  return SPS_OK;
}

}  // namespace

int grid_blocks(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152LL * 32) b = 152LL * 32;
  return (int)b;
}

int compute_keys(sps_plan* pl, const void* x_dev, const void* y_dev, int dtype, cudaStream_t st) {
  KeyParams kp;
  kp.P = pl->P;
  kp.L = pl->Lbits;
  for (int p = 0; p < pl->P; ++p) {
    kp.N[p] = pl->N[p];
    kp.lo[p] = pl->lo[p];
    kp.hi[p] = pl->hi[p];
    kp.inv[p] = (double)pl->N[p] / (pl->hi[p] - pl->lo[p]);
  }
  SPS_CUDA(cudaMemsetAsync(pl->err_flag, 0, sizeof(int), st));
  int blocks = grid_blocks(pl->n, 256);
  if (dtype == SPS_F64)
    k_keys<double><<<blocks, 256, 0, st>>>((const double*)x_dev, (const double*)y_dev, pl->n, kp, pl->keys,
                                           pl->perm, pl->err_flag);
  else
    k_keys<float><<<blocks, 256, 0, st>>>((const float*)x_dev, (const float*)y_dev, pl->n, kp, pl->keys, pl->perm,
                                          pl->err_flag);
  SPS_CHECK_LAUNCH("keys");
  return SPS_OK;
}

int radix_sort(sps_plan* pl, int nbits, cudaStream_t st) {
  const long long n = pl->n;
  const int ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
  const long long hsize = (long long)RS_BINS * ntiles;
  if (pl->sort_hist_cap < hsize) {
    pfree(pl, pl->sort_hist);
    pl->sort_hist_cap = 0;
    SPS_TRY(palloc(pl, &pl->sort_hist, hsize));
    pl->sort_hist_cap = hsize;
  }
  unsigned long long *kin = pl->keys, *kout = pl->keys_tmp;
  unsigned int *vin = pl->perm, *vout = pl->perm_tmp;
  int passes = 0;
  for (int shift = 0; shift < nbits; shift += 8, ++passes) {
    k_rs_hist<<<ntiles, RS_THREADS, 0, st>>>(kin, n, shift, ntiles, pl->sort_hist);
    SPS_CHECK_LAUNCH("radix hist");
    int e = scan_u32(pl->sort_hist, hsize, st);
    if (e) return e;
    k_rs_scatter<<<ntiles, RS_THREADS, 0, st>>>(kin, vin, kout, vout, n, shift, ntiles, pl->sort_hist);
    SPS_CHECK_LAUNCH("radix scatter");
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  if (passes & 1) {   // result lives in the scratch buffers: swap ownership
    std::swap(pl->keys, pl->keys_tmp);
    std::swap(pl->perm, pl->perm_tmp);
  }
  return SPS_OK;
}

int gather_points(sps_plan* pl, const void* x_dev, const void* y_dev, int dtype, cudaStream_t st) {
  int blocks = grid_blocks(pl->n, 256);
  if (dtype == SPS_F64)
    k_gather<double><<<blocks, 256, 0, st>>>((const double*)x_dev, (const double*)y_dev, pl->perm, pl->n, pl->P,
                                             (double*)pl->x_sorted, pl->x32_sorted, pl->y_sorted);
  else
    k_gather<float><<<blocks, 256, 0, st>>>((const float*)x_dev, (const float*)y_dev, pl->perm, pl->n, pl->P,
                                            (float*)pl->x_sorted, nullptr, pl->y_sorted);
  SPS_CHECK_LAUNCH("gather");
  return SPS_OK;
}

// Build runs (points of one level cell, at most RUN_MAX) and work items (runs
// of one tile, at most a CTA's worth) for level g.
int build_level_work(sps_plan* pl, int g, cudaStream_t st) {
  Level& L = pl->lev[g - 1];
  const LevelGeom& G = L.geom;
  const int P = pl->P;
  const int cbits = std::max(pl->Lbits - G.shift, 0);       // bits per dim of a level-cell id
  const long long ncell = 1LL << (P * cbits);
  const int sh = P * G.shift;                                 // key bits below the level cell
  int e = ensure_seg(pl, 2 * (ncell + 1) + 2);
  if (e) return e;
  unsigned int* run_off = (unsigned int*)pl->seg_tmp;
  unsigned int* item_off = run_off + (ncell + 1);
  // item_off holds the cells' point counts until the items are built
  k_cell_runs<<<grid_blocks(ncell + 1, 256), 256, 0, st>>>(pl->keys, pl->n, ncell, sh, run_off, item_off);
  SPS_CHECK_LAUNCH("cell runs");
  if ((e = scan_u32(run_off, ncell + 1, st))) return e;
  unsigned int nruns = 0;
  SPS_CUDA(cudaMemcpyAsync(&nruns, run_off + ncell, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
  SPS_CUDA(cudaStreamSynchronize(st));
  if ((int)nruns > L.run_cap) {   // grow only: cudaFree would synchronise the whole device
    pfree(pl, L.run_begin);
    pfree(pl, L.run_cell);
    pfree(pl, L.run_order);
    pfree(pl, L.item_span);
    pfree(pl, L.item_cell);
    L.run_cap = 0;
    const unsigned int cap = nruns + nruns / 4 + 16;
    SPS_TRY(palloc(pl, &L.run_begin, (long long)cap + 1));
    SPS_TRY(palloc(pl, &L.run_cell, (long long)cap));
    SPS_TRY(palloc(pl, &L.run_order, (long long)cap));
    SPS_TRY(palloc(pl, &L.item_span, (long long)cap));
    SPS_TRY(palloc(pl, &L.item_cell, (long long)cap));
    L.run_cap = (int)cap;
  }
  L.nruns = (int)nruns;
  k_fill_runs<<<grid_blocks(ncell, 256), 256, 0, st>>>(pl->keys, pl->n, ncell, sh, P, cbits, run_off, item_off,
                                                       L.run_begin, L.run_cell, nruns);
  SPS_CHECK_LAUNCH("fill runs");
  // tiles of ts^P level cells
  int tb = 0;
  while ((1 << tb) < G.ts) ++tb;
  tb = std::min(tb, cbits);
  const int tbits = cbits - tb;
  const long long ntile = 1LL << (P * tbits);
  const int cap = runs_per_item(P);
  k_tile_items<<<grid_blocks(ntile + 1, 256), 256, 0, st>>>(run_off, ntile, P * tb, cap, item_off);
  SPS_CHECK_LAUNCH("tile items");
  if ((e = scan_u32(item_off, ntile + 1, st))) return e;
  unsigned int nitems = 0;
  SPS_CUDA(cudaMemcpyAsync(&nitems, item_off + ntile, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
  SPS_CUDA(cudaStreamSynchronize(st));
  if ((int)nitems > L.item_cap) {
    pfree(pl, L.items);
    L.item_cap = 0;
    const unsigned int cap = nitems + nitems / 4 + 16;
    SPS_TRY(palloc(pl, &L.items, (long long)cap));
    L.item_cap = (int)cap;
  }
  L.nitems = (int)nitems;
  k_fill_items<<<grid_blocks(ntile, 256), 256, 0, st>>>(run_off, item_off, ntile, P * tb, cap, P, tbits, tb,
                                                        L.run_begin, L.items);
  SPS_CHECK_LAUNCH("fill items");
  if (nitems > 0) {
    k_sort_item_runs<<<nitems, 128, 0, st>>>(L.items, L.run_begin, L.run_cell, P, L.run_order, L.item_span,
                                             L.item_cell);
    SPS_CHECK_LAUNCH("sort item runs");
  }
  L.max_item_pts = 0;
  if (nitems > 0) {
    // Point counts of the items: the largest sizes the point operator's shared
    // memory.  Then the items in decreasing order of their point counts: CTAs
    // start roughly in block order, so the large items run in the first wave
    // and the small ones fill the tail (longest-processing-time-first).
    const long long item_words = (long long)((sizeof(WorkItem) + 3) / 4) * nitems;
    if ((e = ensure_seg(pl, 2LL * nitems + item_words))) return e;
    unsigned int* npts = (unsigned int*)pl->seg_tmp;
    unsigned int* perm = npts + nitems;
    WorkItem* tmp = reinterpret_cast<WorkItem*>(perm + nitems);
    k_item_npts<<<grid_blocks(nitems, 256), 256, 0, st>>>(L.items, L.run_begin, (int)nitems, npts);
    SPS_CHECK_LAUNCH("item sizes");
    std::vector<unsigned int> h(nitems), order(nitems);
    SPS_CUDA(cudaMemcpyAsync(h.data(), npts, sizeof(unsigned int) * nitems, cudaMemcpyDeviceToHost, st));
    SPS_CUDA(cudaStreamSynchronize(st));
    for (unsigned int k = 0; k < nitems; ++k) {
      order[k] = k;
      L.max_item_pts = std::max(L.max_item_pts, (int)h[k]);
    }
    std::stable_sort(order.begin(), order.end(), [&](unsigned a, unsigned b) { return h[a] > h[b]; });
    SPS_CUDA(cudaMemcpyAsync(perm, order.data(), sizeof(unsigned int) * nitems, cudaMemcpyHostToDevice, st));
    k_permute_items<<<grid_blocks(nitems, 256), 256, 0, st>>>(L.items, perm, (int)nitems, tmp);
    SPS_CHECK_LAUNCH("item order");
    SPS_CUDA(cudaMemcpyAsync(L.items, tmp, sizeof(WorkItem) * nitems, cudaMemcpyDeviceToDevice, st));
    SPS_CUDA(cudaStreamSynchronize(st));   // `order` is a host buffer of this frame
  }
  return SPS_OK;
}

}  // namespace sps

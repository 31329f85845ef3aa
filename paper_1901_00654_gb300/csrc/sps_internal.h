// Internal declarations of the spline smoothing library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/sps.h"

namespace sps {

constexpr int Q = 3;                 // cubic B-splines
constexpr int BAND = 2 * Q + 1;      // diagonals of the 1-D Gram matrices
constexpr int MAXP = SPS_MAX_DIM;
constexpr int MAXL = SPS_MAX_LEVELS;
constexpr int RUN_MAX = 16;          // points per run (one thread group, one cell)
constexpr int POINT_THREADS = 128;   // threads per CTA of the point operator

// Lanes that share one run: 4^(P-3) for P > 3, else 1.
inline int lanes_per_run(int P) { return P <= 3 ? 1 : (P == 4 ? 4 : 16); }
// Runs per work item: 128 for P <= 4 (one tile of 4^4 cells in one item), 32 for
// P = 5.  The point operator's shared memory is sized by the largest item's
// actual point count (Level::max_item_pts), at most 128 * RUN_MAX = 2048.
inline int runs_per_item(int P) { return P <= 4 ? 128 : 32; }
constexpr int COARSE_MAX = 4096;     // K_1 limit of the dense coarse inverse

// Geometry of one grid level, passed by value to kernels.
struct LevelGeom {
  int P;
  int N[MAXP];          // knot intervals per dimension
  int J[MAXP];          // N + q coefficients per dimension
  long long stride[MAXP];
  long long K;
  int shift;            // level cell = finest cell >> shift
  double inv_h[MAXP];   // N_p / (hi_p - lo_p) at this level
  double lo[MAXP];
  int ts;               // tile side in level cells (power of two)
  int E[MAXP];          // patch extent per dimension: min(ts, N_p) + q
  float invE[MAXP];     // 1 / E (patch index division, exact for the sizes used)
  int Es[MAXP];         // patch strides (last dimension fastest)
  int patch;            // prod E
};

// One CTA of the point operator: runs [run_lo, run_hi) of one tile, whose
// points are [pbeg, pbeg + npts) (contiguous after the sort).
struct WorkItem {
  int run_lo, run_hi;
  int pbeg, npts;
  int c0[MAXP];         // tile origin in level cells
  int pad[3];
};

template <typename T>
struct LevelVecs {
  T* alpha = nullptr;   // smoother iterate / correction on this level
  T* b = nullptr;       // right-hand side on this level
  T* u = nullptr;       // operator output
  T* dinv = nullptr;    // 1 / diag(A_g)
  T* band = nullptr;    // Gram bands [p][r][J_p][BAND]
};

struct Level {
  LevelGeom geom;
  // runs: points [run_begin[r], run_begin[r+1]) share one level cell run_cell[r]
  int* run_begin = nullptr;
  unsigned long long* run_cell = nullptr;   // 12 bits per dimension
  int* run_order = nullptr;                 // runs of each item sorted by length (longest first)
  // the same order as a ready table per run slot: first | end << 16 relative to
  // the item's first point, and the cell relative to the tile origin (32/P bits
  // per dimension), so the point operator stages an item's runs with one read
  unsigned* item_span = nullptr;
  unsigned* item_cell = nullptr;
  int nruns = 0, run_cap = 0;
  WorkItem* items = nullptr;
  int nitems = 0, item_cap = 0;
  double omega = 0.0;
  double* diag = nullptr;                   // FP64 diag(A_g)
  // assembled operator of a coarse level, offset-major stencil form
  // A_st[s * K + k] = A_g(k, k + offset_s), s < S = (2q+1)^P; null when the
  // level is applied matrix free
  int S = 0;
  double* st_d = nullptr;
  float* st_f = nullptr;
  // FP64 matrix-free levels: basis values of every point, [point][dim][m]
  double* pre = nullptr;
  long long pre_cap = 0;
  // P = 3 FP64 matrix-free levels, four-lane layout: per point the 4 pieces of
  // dimension 1 and the 16 products of dimensions 2 and 3, [point][20]
  double* pre2 = nullptr;
  long long pre2_cap = 0;
  // FP32 apply of the point operator: dimensions held in a lane's registers
  // (2: 4^(P-2) lanes per run; 3: 4^(P-3) lanes per run; 0: the default for P)
  int lanes_r = 0;
  int max_item_pts = 0;   // points of the largest work item (sizes the staged coordinates)
  LevelVecs<double> d;
  LevelVecs<float> f;
};

}  // namespace sps

struct sps_plan {
  int P = 0, q = 3, G = 0;
  double lam = 0.0;
  int N[sps::MAXP] = {0};
  double lo[sps::MAXP] = {0}, hi[sps::MAXP] = {0};
  sps_options opt;
  int device = 0;
  int Lbits = 1;            // bits per dimension of the Morton key
  bool tuned = false;       // the autotuner has chosen the levels' launch shapes
  sps::Level lev[sps::MAXL];
  // points (sorted)
  long long n = 0, n_cap = 0;
  int dtype = SPS_F64;
  void* x_sorted = nullptr;   // P x n SoA in the input dtype
  float* x32_sorted = nullptr; // P x n SoA rounded to FP32 (aliases x_sorted for FP32 input)
  double* y_sorted = nullptr;
  unsigned long long* keys = nullptr;
  unsigned int* perm = nullptr;
  // scratch for the sort (n entries each) and segment building
  unsigned long long* keys_tmp = nullptr;
  unsigned int* perm_tmp = nullptr;
  unsigned int* sort_hist = nullptr;
  long long sort_hist_cap = 0;
  int* seg_tmp = nullptr;       // per-segment counts / offsets
  long long seg_cap = 0;
  int* err_flag = nullptr;      // device error flags (ERR_* bits)
  // right-hand side Phi'y (FP64) and its norm
  double* rhs = nullptr;
  double rhs_norm = 0.0;
  // dense coarse solver: the assembled A_1, the inverse Cholesky factor Z of
  // its Jacobi-scaled form with the scale folded in (A_1^-1 = Z'Z) and Z',
  // each K_1 x K_1 FP64; null with the inner coarse CG (opt.coarse_cg)
  double* coarse_A = nullptr;
  double* coarse_inv = nullptr;
  double* coarse_invt = nullptr;
  double* coarse_tmp = nullptr;   // scale, pivots, work vectors (6 K_1) + scaled copy (K_1^2)
  double coarse_shift = 0.0;      // diagonal shift the factorisation needed (0 when A_1 was definite)
  // penalty and transfer temporaries (max K over levels)
  double* dtmp[8] = {nullptr};
  float* ftmp[8] = {nullptr};
  // outer PCG vectors (FP64, K_G)
  double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *v = nullptr, *rprev = nullptr;
  float* p32 = nullptr;
  double* scal = nullptr;         // device scalars
  double* red_part = nullptr;     // reduction partials
  unsigned int* red_count = nullptr;
  double* host_scal = nullptr;    // pinned mirror of scal
  bool have_points = false;
  // CUDA graph of one PCG iteration (V-cycle, vector updates, apply), per
  // precision; rebuilt when `gen` (bumped by set_points/set_omega/set_lambda)
  // or the profiling state changes
  struct IterGraph {
    cudaGraphExec_t exec = nullptr;
    unsigned gen = ~0u;
    bool profiled = false;
    int prof_first = 0, prof_last = 0;
    unsigned long long nlaunch = 0;   // kernels per replay
  } graph[3];   // FP64 PCG, mixed PCG, mixed PCG with the FP64 outer operator
  unsigned gen = 0;
  cudaStream_t cap_stream = nullptr;
  // device memory held by the plan (every cudaMalloc goes through plan_alloc)
  std::unordered_map<void*, size_t> dev_sizes;
  long long dev_bytes = 0;
};

namespace sps {

// ---- error handling ----
void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
#define SPS_CUDA(call)                                   \
  do {                                                   \
    cudaError_t _e = (call);                             \
    if (_e != cudaSuccess) return sps::cuda_fail(_e, #call); \
  } while (0)
// device error flags (plan->err_flag)
constexpr int ERR_DOMAIN = 1;     // a coordinate outside [lo, hi] or a non-finite coordinate/response
constexpr int ERR_SMEM = 2;       // the point operator's staged points exceeded its shared memory
constexpr int ERR_WAIT = 4;       // the point operator's wait for its asynchronous copies ran out of time
// propagate a non-OK status code
#define SPS_TRY(x)                   \
  do {                               \
    int _r = (x);                    \
    if (_r != SPS_OK) return _r;     \
  } while (0)
// every kernel launch is followed by this check, which also counts the launch
void count_launches(unsigned long long k);
#define SPS_CHECK_LAUNCH(what)  \
  do {                          \
    sps::count_launches(1);     \
    SPS_CUDA(cudaGetLastError()); \
  } while (0)

// ---- device memory of a plan (api.cu) ----
// Every allocation of plan memory goes through plan_alloc, which enforces
// sps_options.max_device_bytes and tracks the bytes held.
int plan_alloc(sps_plan* pl, void** p, size_t bytes);
void plan_free(sps_plan* pl, void* p);
template <typename T>
int palloc(sps_plan* pl, T** p, long long count) {
  if (count < 1) count = 1;
  return plan_alloc(pl, (void**)p, sizeof(T) * (size_t)count);
}
template <typename T>
void pfree(sps_plan* pl, T*& p) {
  plan_free(pl, (void*)p);
  p = nullptr;
}
// Reads and clears the device error flags; SPS_EINTERNAL if the point
// operator reported an inconsistent launch.
int check_device_errors(sps_plan* pl, cudaStream_t st);

// ---- sort.cu ----
int compute_keys(sps_plan* pl, const void* x_dev, const void* y_dev, int dtype, cudaStream_t st);
int radix_sort(sps_plan* pl, int nbits, cudaStream_t st);
int gather_points(sps_plan* pl, const void* x_dev, const void* y_dev, int dtype, cudaStream_t st);   // also fills x32_sorted
int build_level_work(sps_plan* pl, int g, cudaStream_t st);

// ---- point_op.cu ----
enum PointMode { PT_APPLY = 0, PT_DIAG = 1, PT_RHS = 2 };
// dynamic shared memory of one apply launch on a level with this geometry
size_t point_apply_smem(const sps_plan* pl, const LevelGeom& G, bool fp32);
constexpr size_t POINT_SMEM_MAX = 160 * 1024;   // opt-in dynamic shared memory of k_point
template <typename T>
int point_op(sps_plan* pl, int g, int mode, const T* v, T* u, cudaStream_t st);
int basis_precompute(sps_plan* pl, int g, cudaStream_t st);
constexpr int PRE2_STRIDE = 20;   // doubles per point of Level::pre2
int profile_begin();
int profile_end(double* ms, unsigned long long* launches);
bool profile_active();
int profile_mark();
void profile_capture_end(int first, int last);
int profile_harvest(int first, int last);

// ---- api.cu ----
void level_tile(LevelGeom& G, int ts);   // tile side ts: patch extents, strides and size

// ---- tune.cu ----
int autotune(sps_plan* pl, cudaStream_t st);

// ---- grid_ops.cu ----
template <typename T>
int penalty_apply(sps_plan* pl, int g, const T* v, T* out, double scale, cudaStream_t st);
int penalty_diag(sps_plan* pl, int g, double* d, cudaStream_t st);
template <typename T>
int prolong_sub(sps_plan* pl, int g, const T* c, T* f, int mode, cudaStream_t st);  // mode 0: f = Ic; 1: f -= Ic
template <typename T>
int restrict_res(sps_plan* pl, int g, const T* f, const T* fb, T* c, cudaStream_t st);  // c = I'(f - fb) (fb may be null)
int coarse_assemble(sps_plan* pl, cudaStream_t st);
int stencil_assemble(sps_plan* pl, int g, cudaStream_t st);
template <typename T>
int stencil_apply(sps_plan* pl, int g, const T* v, T* u, cudaStream_t st);
template <typename T>
int coarse_solve(sps_plan* pl, const T* r, T* e, cudaStream_t st);   // dense inverse (+ refinement in FP64)
// Inner Jacobi-preconditioned CG on level 1 from e = 0, opt.coarse_iters
// iterations; r1, p1 are level-1 work vectors distinct from the penalty temporaries.
template <typename T>
int coarse_cg(sps_plan* pl, const T* b, T* e, T* r1, T* p1, cudaStream_t st);

// elementwise / reductions
template <typename T>
int vec_scale_mul(T* out, const T* a, const T* b, T s, long long n, cudaStream_t st);     // out = s*a*b
template <typename T>
int vec_jacobi(T* alpha, const T* dinv, const T* b, const T* u, T omega, long long n, cudaStream_t st);
int vec_cast_d2f(float* out, const double* in, long long n, cudaStream_t st);
int vec_cast_f2d(double* out, const float* in, long long n, cudaStream_t st);
int vec_set_d(double* out, double v, long long n, cudaStream_t st);
int vec_set_f(float* out, float v, long long n, cudaStream_t st);
int vec_recip(double* dinv, float* dinv_f, const double* d, long long n, cudaStream_t st);
int vec_residual(double* r, const double* b, const double* u, long long n, double* scal, int slot,
                 sps_plan* pl, cudaStream_t st);  // r = b - u; scal[slot] = r.r
int dot(sps_plan* pl, const double* a, const double* b, long long n, int slot, cudaStream_t st);
int dot2(sps_plan* pl, const double* a, const double* b, const double* c, long long n, int slot,
         cudaStream_t st);   // scal[slot] = a.b, scal[slot+1] = a.c
int pcg_update_xr(sps_plan* pl, long long n, int rz_slot, cudaStream_t st);
int pcg_update_p(sps_plan* pl, long long n, int num_slot, int den_slot, int flexible, cudaStream_t st);

// ---- batch.cu ----
int solve_batch(sps_plan* const* plans, int count, double* const* coefs, int mem, double tol,
                const sps_batch_shape* shape, sps_result* res, sps_batch_shape* used, cudaStream_t st);
int tune_batch(sps_plan* const* plans, int count, double* const* coefs, int mem, double tol, sps_batch_shape* best,
               cudaStream_t st);
// Makespan (ms) of the batched solver's persistent queues for per-problem
// times t1 (single CTA) and tc (team of C CTAs), problems taken in `order`:
// the model the batch autotuner minimises (host only).
double batch_makespan(const int* order, const double* t1, const double* tc, int n, int C, int big, int grid);

// ---- solver (api.cu) ----
template <typename T>
int apply_level(sps_plan* pl, int g, const T* v, T* u, cudaStream_t st);
template <typename T>
int vcycle_into(sps_plan* pl, const T* bG, T* xG, cudaStream_t st);   // xG = V(bG) on level G

template <typename T>
LevelVecs<T>& vecs(Level& L);
template <>
inline LevelVecs<double>& vecs<double>(Level& L) { return L.d; }
template <>
inline LevelVecs<float>& vecs<float>(Level& L) { return L.f; }

int grid_blocks(long long n, int threads);

}  // namespace sps

// Coefficient-space kernels: the penalty Lambda v through its Kronecker-sum
// structure, the subdivision prolongation and its transpose, the coarse
// matrix and its inverse, the elementwise smoother updates and the fused PCG
// vector updates with their dot products.
#include <cuda_runtime.h>

#include <algorithm>

#include "sps_internal.h"

namespace sps {

namespace {

constexpr int EW_THREADS = 256;
constexpr int RED_BLOCKS = 304;      // 2 per SM; fixed so reductions are deterministic

// ------------------------------------------------------------------ penalty
// Lambda = sum_{|r|=2} (2/r!) kron_p Psi^p_{r_p} (Section 2.2, Section 2.4).
// Dimension by dimension (Algorithm 2 applies one Kronecker factor per mode)
// three partial sums are carried: W0 (all factors Psi_0 so far), W1 (exactly
// one Psi_1), W2 (derivative order two, weighted by 2/r!):
//   W0' = M W0,  W1' = M W1 + D1 W0,  W2' = M W2 + 2 D1 W1 + D2 W0,
// with M = Psi^p_0, D1 = Psi^p_1, D2 = Psi^p_2 banded (2q+1 diagonals).
// stage: 0 first dimension, 1 middle, 2 last, 3 only dimension.
// IT: index type -- 32-bit unsigned when every index fits (one integer
// division instead of a 64-bit division routine per element), else 64-bit.
template <typename T, typename IT>
__global__ void k_pen_sweep(int stage, IT K, IT strd, int Jp, const T* __restrict__ band,
                            const T* __restrict__ w0, const T* __restrict__ w1, const T* __restrict__ w2,
                            T* __restrict__ o0, T* __restrict__ o1, T* __restrict__ o2, T scale) {
  for (IT k = (IT)blockIdx.x * blockDim.x + threadIdx.x; k < K; k += (IT)gridDim.x * blockDim.x) {
    const int j = (int)((k / strd) % (IT)Jp);
    const T* M = band + (long long)j * BAND;
    const T* D1 = band + ((long long)Jp + j) * BAND;
    const T* D2 = band + (2LL * Jp + j) * BAND;
    T a0 = T(0), a1 = T(0), a2 = T(0), h = T(0);   // h = D1 x1: a2 gets 2h after the taps
#pragma unroll
    for (int o = -Q; o <= Q; ++o) {
      const int jj = j + o;
      if (jj < 0 || jj >= Jp) continue;
      const IT kk = k + (IT)((long long)o * (long long)strd);
      const T m = M[o + Q], d1 = D1[o + Q], d2 = D2[o + Q];
      if (stage == 0) {
        const T x = w0[kk];
        a0 = fma(m, x, a0);
        a1 = fma(d1, x, a1);
        a2 = fma(d2, x, a2);
      } else if (stage == 3) {
        a2 = fma(d2, w0[kk], a2);
      } else {
        const T x0 = w0[kk], x1 = w1[kk], x2 = w2[kk];
        if (stage == 1) {
          a0 = fma(m, x0, a0);
          a1 = fma(m, x1, fma(d1, x0, a1));
        }
        a2 = fma(m, x2, fma(d2, x0, a2));
        h = fma(d1, x1, h);
      }
    }
    if (stage == 1 || stage == 2) a2 = fma(T(2), h, a2);
    if (stage <= 1) {
      o0[k] = a0;
      o1[k] = a1;
      o2[k] = a2;
    } else {
      o2[k] = scale * a2;
    }
  }
}

// diag(Lambda) by the same recursion on the central band entries.
__global__ void k_pen_diag(long long K, LevelGeom geom, const double* __restrict__ band, double lam,
                           double* __restrict__ d, int accumulate) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < K;
       k += (long long)gridDim.x * blockDim.x) {
    double d0 = 1.0, d1 = 0.0, d2 = 0.0;
    long long boff = 0;
    for (int p = 0; p < geom.P; ++p) {
      const int Jp = geom.J[p];
      const int j = (int)((k / geom.stride[p]) % Jp);
      const double m = band[boff + (long long)j * BAND + Q];
      const double e1 = band[boff + ((long long)Jp + j) * BAND + Q];
      const double e2 = band[boff + (2LL * Jp + j) * BAND + Q];
      d2 = m * d2 + 2.0 * e1 * d1 + e2 * d0;
      d1 = m * d1 + e1 * d0;
      d0 = m * d0;
      boff += 3LL * Jp * BAND;
    }
    d[k] = (accumulate ? d[k] : 0.0) + lam * d2;
  }
}

// ------------------------------------------------------------------ transfers
// 1-D subdivision weights 2^-q binom(q+1, k), k = i - 2j + q (Section 2.4).
__constant__ double c_subdiv[Q + 2] = {1.0 / 8, 4.0 / 8, 6.0 / 8, 4.0 / 8, 1.0 / 8};

// out (fine along the swept mode) = I_1d * in (coarse along it).
template <typename T, typename IT>
__global__ void k_prolong_sweep(IT Kout, IT inner, int Jin, int Jout, const T* __restrict__ in,
                                T* __restrict__ out, int subtract) {
  const IT blk = (IT)Jout * inner;
  for (IT k = (IT)blockIdx.x * blockDim.x + threadIdx.x; k < Kout; k += (IT)gridDim.x * blockDim.x) {
    const IT outer = k / blk;
    const IT rem = k - outer * blk;
    const int i = (int)(rem / inner);
    const IT ii = rem - (IT)i * inner;
    T s = T(0);
#pragma unroll
    for (int kk = 0; kk <= Q + 1; ++kk) {
      const int num = i + Q - kk;
      if (num & 1) continue;
      const int j = num >> 1;
      if (j < 0 || j >= Jin) continue;
      s = fma(T(c_subdiv[kk]), in[(outer * (IT)Jin + (IT)j) * inner + ii], s);
    }
    if (subtract) out[k] -= s; else out[k] = s;
  }
}

// out (coarse along the mode) = I_1d' * (in - inb) (fine along it).
template <typename T, typename IT>
__global__ void k_restrict_sweep(IT Kout, IT inner, int Jin, int Jout, const T* __restrict__ in,
                                 const T* __restrict__ inb, T* __restrict__ out) {
  const IT blk = (IT)Jout * inner;
  for (IT k = (IT)blockIdx.x * blockDim.x + threadIdx.x; k < Kout; k += (IT)gridDim.x * blockDim.x) {
    const IT outer = k / blk;
    const IT rem = k - outer * blk;
    const int j = (int)(rem / inner);
    const IT ii = rem - (IT)j * inner;
    T s = T(0);
#pragma unroll
    for (int kk = 0; kk <= Q + 1; ++kk) {
      const int i = 2 * j - Q + kk;
      if (i < 0 || i >= Jin) continue;
      const IT src = (outer * (IT)Jin + (IT)i) * inner + ii;
      const T val = inb ? in[src] - inb[src] : in[src];
      s = fma(T(c_subdiv[kk]), val, s);
    }
    out[k] = s;
  }
}

// ------------------------------------------------------------------ coarse matrix
// A_1 = Phi_1'Phi_1 + lambda Lambda_1, assembled densely (Section 3.2, coarse
// grid solver).  One CTA takes a contiguous range of runs (points of one cell)
// and a block of CB local columns; each thread owns 16 entries of the local
// (q+1)^P x CB block of sum_i b_i b_i' in FP64 registers.  Products use TP.
// STENCIL = true writes the same sums into the offset-major stencil form
// A_st[s * K + k] (s = the (2q+1)^P offset of column l from row k) used for
// the assembled coarse levels.
template <int P, typename TP, bool STENCIL>
__global__ void __launch_bounds__(256) k_coarse_phi(const int* __restrict__ run_begin,
                                                    const unsigned long long* __restrict__ run_cell, int nruns,
                                                    int runs_per_cta, const void* __restrict__ xs_raw, int x_f64,
                                                    long long n, LevelGeom geom, double* __restrict__ A1) {
  constexpr int LOC = 1 << (2 * P);
  constexpr int CB = P <= 3 ? LOC : (P == 4 ? 16 : 4);
  constexpr int PER = (LOC * CB + 255) / 256;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TP* B = reinterpret_cast<TP*>(smem_raw);                 // [RUN_MAX][LOC]
  TP* bas = B + RUN_MAX * LOC;                              // [RUN_MAX][P][4]
  const int cb0 = blockIdx.y * CB;
  double acc[PER];
  TP part[PER];
#pragma unroll
  for (int e = 0; e < PER; ++e) acc[e] = 0.0;
  const int r0 = blockIdx.x * runs_per_cta;
  const int r1 = min(r0 + runs_per_cta, nruns);
  unsigned long long cur = ~0ull;
  auto flush = [&](unsigned long long cell) {
    int c[MAXP];
    for (int p = 0; p < P; ++p) c[p] = (int)((cell >> (12 * p)) & 0xFFF);
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const int le = threadIdx.x + 256 * e;
      if (le >= LOC * CB) break;
      const int row = le / CB, col = le % CB + cb0;
      long long gr = 0, gc = 0;
      int rr = row, cc = col, so = 0, sw = 1;
      for (int p = P - 1; p >= 0; --p) {
        gr += (long long)(c[p] + (rr & 3)) * geom.stride[p];
        gc += (long long)(c[p] + (cc & 3)) * geom.stride[p];
        so += ((cc & 3) - (rr & 3) + Q) * sw;
        sw *= BAND;
        rr >>= 2;
        cc >>= 2;
      }
      if (acc[e] != 0.0) {
        if (STENCIL) atomicAdd(&A1[(long long)so * geom.K + gr], acc[e]);
        else atomicAdd(&A1[gr * geom.K + gc], acc[e]);
      }
      acc[e] = 0.0;
    }
  };
  for (int r = r0; r < r1; ++r) {
    const unsigned long long cell = run_cell[r];
    if (cell != cur) {
      if (cur != ~0ull) flush(cur);
      cur = cell;
    }
    const int i0 = run_begin[r], i1 = run_begin[r + 1];
    const int np = i1 - i0;
    __syncthreads();
    for (int e = threadIdx.x; e < np * P; e += blockDim.x) {
      const int i = e / P, p = e % P;
      const double xv = x_f64 ? ((const double*)xs_raw)[(long long)p * n + i0 + i]
                              : (double)((const float*)xs_raw)[(long long)p * n + i0 + i];
      const int c = (int)((cell >> (12 * p)) & 0xFFF);
      const double t = xv * geom.inv_h[p] - (geom.lo[p] * geom.inv_h[p] + (double)c);
      const double om = 1.0 - t, t2 = t * t;
      TP* b = bas + (i * P + p) * 4;
      b[0] = TP(om * om * om / 6.0);
      b[1] = TP(t2 * (0.5 * t - 1.0) + 2.0 / 3.0);
      b[2] = TP(((-0.5 * t + 0.5) * t + 0.5) * t + 1.0 / 6.0);
      b[3] = TP(t2 * t / 6.0);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < np * LOC; e += blockDim.x) {
      const int i = e / LOC, l = e % LOC;
      TP v = TP(1);
      int ll = l;
      for (int p = P - 1; p >= 0; --p) {
        v *= bas[(i * P + p) * 4 + (ll & 3)];
        ll >>= 2;
      }
      B[i * LOC + l] = v;
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < PER; ++e) part[e] = TP(0);
    for (int i = 0; i < np; ++i) {
#pragma unroll
      for (int e = 0; e < PER; ++e) {
        const int le = threadIdx.x + 256 * e;
        if (le >= LOC * CB) break;
        const int row = le / CB, col = le % CB + cb0;
        part[e] = fma(B[i * LOC + row], B[i * LOC + col], part[e]);
      }
    }
#pragma unroll
    for (int e = 0; e < PER; ++e) acc[e] += (double)part[e];
  }
  if (cur != ~0ull) flush(cur);
}

// + lambda Lambda_1 on the stencil neighbourhood of every row.
__global__ void k_coarse_penalty(LevelGeom geom, const double* __restrict__ band, double lam,
                                 double* __restrict__ A1) {
  const long long K = geom.K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < K * K;
       e += (long long)gridDim.x * blockDim.x) {
    const long long k = e / K, l = e % K;
    double d0 = 1.0, d1 = 0.0, d2 = 0.0;
    long long boff = 0;
    bool nz = true;
    for (int p = 0; p < geom.P && nz; ++p) {
      const int Jp = geom.J[p];
      const int j = (int)((k / geom.stride[p]) % Jp);
      const int jl = (int)((l / geom.stride[p]) % Jp);
      const int o = jl - j;
      if (o < -Q || o > Q) { nz = false; break; }
      const double m = band[boff + (long long)j * BAND + o + Q];
      const double e1 = band[boff + ((long long)Jp + j) * BAND + o + Q];
      const double e2 = band[boff + (2LL * Jp + j) * BAND + o + Q];
      d2 = m * d2 + 2.0 * e1 * d1 + e2 * d0;
      d1 = m * d1 + e1 * d0;
      d0 = m * d0;
      boff += 3LL * Jp * BAND;
    }
    if (nz) A1[e] += lam * d2;
  }
}

// + lambda Lambda_g in stencil form: entry (k, k + offset s).
__global__ void k_stencil_penalty(LevelGeom geom, const double* __restrict__ band, double lam,
                                  double* __restrict__ A, int S) {
  const long long K = geom.K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)S * K;
       e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e / K);
    const long long k = e - (long long)s * K;
    double d0 = 1.0, d1 = 0.0, d2 = 0.0;
    long long boff = 0;
    int ss = s;
    int o[MAXP];
    for (int p = geom.P - 1; p >= 0; --p) {
      o[p] = ss % BAND - Q;
      ss /= BAND;
    }
    bool ok = true;
    for (int p = 0; p < geom.P; ++p) {
      const int Jp = geom.J[p];
      const int j = (int)((k / geom.stride[p]) % Jp);
      if (j + o[p] < 0 || j + o[p] >= Jp) { ok = false; break; }
      const double m = band[boff + (long long)j * BAND + o[p] + Q];
      const double e1 = band[boff + ((long long)Jp + j) * BAND + o[p] + Q];
      const double e2 = band[boff + (2LL * Jp + j) * BAND + o[p] + Q];
      d2 = m * d2 + 2.0 * e1 * d1 + e2 * d0;
      d1 = m * d1 + e1 * d0;
      d0 = m * d0;
      boff += 3LL * Jp * BAND;
    }
    if (ok) A[e] += lam * d2;
  }
}

__global__ void k_d2f_scaled(const double* __restrict__ a, float* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// u = A_st v for an assembled level.  A block is 32 consecutive rows x
// SPMV_Y offset groups: lane x owns row k (so the offset-major matrix and v
// are read coalesced), row y of the block takes every SPMV_Y-th combination of
// the leading P-1 offsets and walks the last offset as a straight loop; the
// SPMV_Y partial sums of a row are added in shared memory.  Offsets outside the
// grid are skipped by range, not by division.

template <int P, typename T, int SPMV_Y>
__global__ void __launch_bounds__(32 * SPMV_Y) k_stencil_spmv(const T* __restrict__ A, LevelGeom geom,
                                                              const T* __restrict__ v, T* __restrict__ u) {
  __shared__ T part[SPMV_Y][33];
  const long long K = geom.K;
  const long long k = (long long)blockIdx.x * 32 + threadIdx.x;
  T acc = T(0);
  if (k < K) {
    int lo[P], hi[P];
    long long rem = k;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const int j = (int)(rem / geom.stride[p]);
      rem -= (long long)j * geom.stride[p];
      lo[p] = max(-Q, -j);
      hi[p] = min(Q, geom.J[p] - 1 - j);
    }
    constexpr int NOUT = P == 1 ? 1 : (P == 2 ? BAND : (P == 3 ? BAND * BAND : (P == 4 ? BAND * BAND * BAND
                                                                                      : BAND * BAND * BAND * BAND)));
    for (int c = threadIdx.y; c < NOUT; c += SPMV_Y) {
      // decode the leading offsets of combination c (division by the constant 7)
      int cc = c;
      long long s = 0, off = 0;
      bool ok = true;
#pragma unroll
      for (int p = P - 2; p >= 0; --p) {
        const int o = cc % BAND - Q;
        cc /= BAND;
        ok = ok && o >= lo[p] && o <= hi[p];
        off += (long long)o * geom.stride[p];
      }
      if (!ok) continue;
      long long sw = BAND;
      s = 0;
      {
        int c2 = c;
#pragma unroll
        for (int p = P - 2; p >= 0; --p) {
          s += (long long)(c2 % BAND) * sw;
          c2 /= BAND;
          sw *= BAND;
        }
      }
      // s: index of (leading offsets, last offset = -q); walk the last offset
      for (int oi = lo[P - 1]; oi <= hi[P - 1]; ++oi)
        acc = fma(A[(s + oi + Q) * K + k], v[k + off + oi], acc);
    }
  }
  part[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && k < K) {
    T t = T(0);
#pragma unroll
    for (int y = 0; y < SPMV_Y; ++y) t += part[y][threadIdx.x];
    u[k] = t;
  }
}

// Inverse Cholesky factor of the SPD coarse matrix: Z = L^-1 with A = L L'.
// Step k of the Cholesky elimination is applied to [A | I]: the trailing part
// of A (lower triangle) is updated, a_ij -= a_ik a_jk / a_kk, and the same row
// operations, row_i -= (a_ik / a_kk) row_k, turn I into L^-1; row k is scaled
// by 1 / sqrt(a_kk) one launch later (when nothing reads it any more).  The
// coarse solve is then e = Z' (Z r): Z'Z is symmetric positive definite for
// any nonsingular Z, so the coarse correction keeps the V-cycle an SPD
// preconditioner however ill-conditioned A_1 is, and Z's rounding errors grow
// like sqrt(cond(A_1)) instead of cond(A_1) for an explicit inverse.
// Launch k covers rows k-1 .. K-1 (launch K only scales row K-1).
// A pivot that is not positive and finite (the assembled matrix is not
// definite to working accuracy) is counted in *bad and replaced by 1 so that
// the sweep ends with finite values; coarse_assemble then refactors with a
// diagonal shift.
__global__ void k_chol_inv_step(double* __restrict__ A, double* __restrict__ Z, double* __restrict__ piv, long long K,
                                int k, int* __restrict__ bad) {
  const long long r0 = k > 0 ? k - 1 : 0;
  double p = k < K ? A[(long long)k * K + k] : 1.0;
  if (!(p > 0.0) || !isfinite(p)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(bad, 1);
    p = 1.0;
  }
  const double ip = 1.0 / p;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (K - r0) * K;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = r0 + e / K, j = e - (e / K) * K;
    if (i == k - 1) {
      if (j <= i) Z[i * K + j] /= sqrt(piv[i]);
    } else if (i == k) {
      if (j == 0) piv[k] = p;
    } else {
      const double l = A[i * K + k] * ip;
      if (j > k && j <= i) A[i * K + j] -= l * A[j * K + k];
      else if (j <= k) Z[i * K + j] -= l * Z[(long long)k * K + j];
    }
  }
}

__global__ void k_identity(double* __restrict__ Z, long long K) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < K * K;
       e += (long long)gridDim.x * blockDim.x)
    Z[e] = (e / K == e - (e / K) * K) ? 1.0 : 0.0;
}

// Z <- Z S (columns scaled: (S A S)^-1 = Z_s' Z_s gives A^-1 = (Z_s S)' (Z_s S)), and Zt = Z'.
__global__ void k_unscale_transpose(double* __restrict__ Z, double* __restrict__ Zt, const double* __restrict__ sc,
                                    long long K) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < K * K;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / K, j = e - (e / K) * K;
    const double z = Z[e] * sc[j];
    Z[e] = z;
    Zt[j * K + i] = z;
  }
}

// Symmetric Jacobi scaling of the coarse matrix: s_i = 1 / sqrt(A_ii), and
// out = S A S.  The inverse is formed from the scaled matrix (unit diagonal;
// for the workloads' A_1 its condition number is 4-6 orders of magnitude
// below that of A_1) and scaled back, A^-1 = S (S A S)^-1 S.
__global__ void k_coarse_scale(const double* __restrict__ A, long long K, double* __restrict__ sc) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < K; i += (long long)gridDim.x * blockDim.x) {
    const double d = A[i * K + i];
    sc[i] = d > 0.0 ? 1.0 / sqrt(d) : 1.0;
  }
}

// `shift` is added to the diagonal of the scaled matrix.
__global__ void k_scale_sym(const double* __restrict__ A, long long K, const double* __restrict__ sc,
                            double* __restrict__ out, double shift) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < K * K;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / K, j = e - (e / K) * K;
    out[e] = sc[i] * A[e] * sc[j] + (i == j ? shift : 0.0);
  }
}

// One warp per row, FP64 arithmetic: mode 0: y = M x; 1: y = b - M x; 2: y += M x.
template <typename TX, typename T>
__global__ void k_gemv(const double* __restrict__ M, long long K, const TX* __restrict__ x, T* __restrict__ y,
                       const T* __restrict__ b, int mode) {
  const int lane = threadIdx.x & 31;
  for (long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; row < K;
       row += ((long long)gridDim.x * blockDim.x) >> 5) {
    double s = 0.0;
    for (long long c = lane; c < K; c += 32) s = fma(M[row * K + c], (double)x[c], s);
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      if (mode == 0) y[row] = T(s);
      else if (mode == 1) y[row] = T((double)b[row] - s);
      else y[row] = T((double)y[row] + s);
    }
  }
}

// ------------------------------------------------------------------ elementwise
template <typename T>
__global__ void k_scale_mul(T* __restrict__ out, const T* __restrict__ a, const T* __restrict__ b, T s, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = s * a[i] * b[i];
}

// Algorithm 6: alpha <- alpha + omega D^-1 (b - A alpha), with u = A alpha.
template <typename T>
__global__ void k_jacobi(T* __restrict__ alpha, const T* __restrict__ dinv, const T* __restrict__ b,
                         const T* __restrict__ u, T omega, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    alpha[i] = fma(omega * dinv[i], b[i] - u[i], alpha[i]);
}

__global__ void k_cast_d2f(float* __restrict__ o, const double* __restrict__ a, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    o[i] = (float)a[i];
}
__global__ void k_cast_f2d(double* __restrict__ o, const float* __restrict__ a, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    o[i] = (double)a[i];
}
template <typename T>
__global__ void k_set(T* __restrict__ o, T v, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    o[i] = v;
}
__global__ void k_recip(double* __restrict__ dinv, float* __restrict__ dinv_f, const double* __restrict__ d,
                        long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = 1.0 / d[i];
    dinv[i] = v;
    if (dinv_f) dinv_f[i] = (float)v;
  }
}

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;   // valid in thread 0
}

// Last-block reduction of NV per-block partials (fixed order: deterministic).
template <int NV>
__device__ __forceinline__ bool finish_reduction(const double* vals, double* part, unsigned int* count,
                                                 double* out, double* sh) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    for (int q = 0; q < NV; ++q) part[q * gridDim.x + blockIdx.x] = vals[q];
    __threadfence();
    const unsigned int t = atomicAdd(count, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  for (int q = 0; q < NV; ++q) {
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += *((volatile double*)&part[q * gridDim.x + b]);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) out[q] = s;
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = 0;
  return true;
}

__global__ void k_dot(const double* __restrict__ a, const double* __restrict__ b, const double* __restrict__ c,
                      long long n, double* part, unsigned int* count, double* out) {
  __shared__ double sh[32];
  double s0 = 0.0, s1 = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double av = a[i];
    s0 = fma(av, b[i], s0);
    if (c) s1 = fma(av, c[i], s1);
  }
  double v[2];
  v[0] = block_sum(s0, sh);
  __syncthreads();
  v[1] = c ? block_sum(s1, sh) : 0.0;
  finish_reduction<2>(v, part, count, out, sh);
}

// Algorithm 8: w = rz / p'v; alpha += w p; r -= w v; and |r|^2.
// scal layout: [rz_slot] r'z, [2] p'v, [3] r'r (out), [4] w (out), [6] flag.
__global__ void k_update_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                            const double* __restrict__ v, long long n, double* scal, int rz_slot, double* part,
                            unsigned int* count) {
  __shared__ double sh[32];
  const double pv = scal[2];
  const double w = scal[rz_slot] / pv;
  const bool bad = !(pv > 0.0) || !isfinite(w);
  double s = 0.0;
  if (!bad) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
      x[i] = fma(w, p[i], x[i]);
      const double ri = fma(-w, v[i], r[i]);
      r[i] = ri;
      s = fma(ri, ri, s);
    }
  }
  double vals[1];
  vals[0] = block_sum(s, sh);
  if (finish_reduction<1>(vals, part, count, scal + 3, sh) && threadIdx.x == 0) {
    scal[4] = w;
    if (bad) scal[6] = 1.0;
  }
}

// p = z + beta p with beta = num / den (flexible: (num - num2) / den).
__global__ void k_update_p(double* __restrict__ p, const double* __restrict__ z, long long n, const double* scal,
                           int num_slot, int den_slot, int flexible) {
  double beta = scal[num_slot];
  if (flexible) beta -= scal[num_slot + 1];
  beta /= scal[den_slot];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

__global__ void k_residual(double* __restrict__ r, const double* __restrict__ b, const double* __restrict__ u,
                           long long n, double* part, unsigned int* count, double* out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double ri = b[i] - u[i];
    r[i] = ri;
    s = fma(ri, ri, s);
  }
  double vals[1];
  vals[0] = block_sum(s, sh);
  finish_reduction<1>(vals, part, count, out, sh);
}

// ---- inner Jacobi-preconditioned CG on the coarse level (Section 3.2, coarse
// grid solver: a matrix-free CG instead of a factorisation).  Vectors in T,
// reductions and scalars in FP64; scalar slots in plan->scal:
constexpr int C_PQ = 16, C_RZ0 = 18, C_RZ1 = 20;

// e = 0; r = b; p = D^-1 b; scal[C_RZ0] = b' D^-1 b
template <typename T>
__global__ void k_ccg_init(const T* __restrict__ b, const T* __restrict__ dinv, T* __restrict__ e,
                           T* __restrict__ r, T* __restrict__ p, long long n, double* scal, double* part,
                           unsigned int* count) {
  __shared__ double sh[32];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const T bi = b[i];
    const T zi = dinv[i] * bi;
    e[i] = T(0);
    r[i] = bi;
    p[i] = zi;
    s = fma((double)bi, (double)zi, s);
  }
  double v[1];
  v[0] = block_sum(s, sh);
  finish_reduction<1>(v, part, count, scal + C_RZ0, sh);
}

// scal[C_PQ] = p'q
template <typename T>
__global__ void k_ccg_pq(const T* __restrict__ p, const T* __restrict__ q, long long n, double* scal, double* part,
                         unsigned int* count) {
  __shared__ double sh[32];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s = fma((double)p[i], (double)q[i], s);
  double v[1];
  v[0] = block_sum(s, sh);
  finish_reduction<1>(v, part, count, scal + C_PQ, sh);
}

// a = rz / p'q (0 once the iteration has converged or broken down);
// e += a p; r -= a q; scal[rz_new] = r' D^-1 r
template <typename T>
__global__ void k_ccg_update(T* __restrict__ e, T* __restrict__ r, const T* __restrict__ p, const T* __restrict__ q,
                             const T* __restrict__ dinv, long long n, double* scal, int rz_old, int rz_new,
                             double* part, unsigned int* count) {
  __shared__ double sh[32];
  const double pq = scal[C_PQ], rz = scal[rz_old];
  double a = rz / pq;
  if (!(pq > 0.0) || !isfinite(a)) a = 0.0;
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    e[i] = T(fma(a, (double)p[i], (double)e[i]));
    const T ri = T(fma(-a, (double)q[i], (double)r[i]));
    r[i] = ri;
    s = fma((double)ri, (double)(dinv[i] * ri), s);
  }
  double v[1];
  v[0] = block_sum(s, sh);
  finish_reduction<1>(v, part, count, scal + rz_new, sh);
}

// p = D^-1 r + beta p, beta = rz_new / rz_old (0 once converged)
template <typename T>
__global__ void k_ccg_dir(T* __restrict__ p, const T* __restrict__ r, const T* __restrict__ dinv, long long n,
                          const double* scal, int rz_old, int rz_new) {
  double beta = scal[rz_new] / scal[rz_old];
  if (!(scal[rz_old] > 0.0) || !isfinite(beta)) beta = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = T(fma(beta, (double)p[i], (double)(dinv[i] * r[i])));
}

template <typename T>
T* tmp_of(sps_plan* pl, int i);
template <>
double* tmp_of<double>(sps_plan* pl, int i) { return pl->dtmp[i]; }
template <>
float* tmp_of<float>(sps_plan* pl, int i) { return pl->ftmp[i]; }

}  // namespace

// ------------------------------------------------------------------ host wrappers
template <typename T>
int penalty_apply(sps_plan* pl, int g, const T* v, T* out, double scale, cudaStream_t st) {
  Level& L = pl->lev[g - 1];
  const LevelGeom& G = L.geom;
  const int P = pl->P;
  const T* band = vecs<T>(L).band;
  const int blocks = grid_blocks(G.K, EW_THREADS);
  const bool i32 = G.K < (1LL << 31);
  auto sweep = [&](int stage, int p, const T* bp, const T* w0, const T* w1, const T* w2, T* o0, T* o1, T* o2,
                   T sc) {
    if (i32)
      k_pen_sweep<T, unsigned><<<blocks, EW_THREADS, 0, st>>>(stage, (unsigned)G.K, (unsigned)G.stride[p], G.J[p],
                                                              bp, w0, w1, w2, o0, o1, o2, sc);
    else
      k_pen_sweep<T, long long><<<blocks, EW_THREADS, 0, st>>>(stage, G.K, G.stride[p], G.J[p], bp, w0, w1, w2, o0,
                                                               o1, o2, sc);
  };
  if (P == 1) {
    sweep(3, 0, band, v, nullptr, nullptr, nullptr, nullptr, out, T(scale));
    SPS_CHECK_LAUNCH("penalty");
    return SPS_OK;
  }
  T* A[3] = {tmp_of<T>(pl, 0), tmp_of<T>(pl, 1), tmp_of<T>(pl, 2)};
  T* B[3] = {tmp_of<T>(pl, 3), tmp_of<T>(pl, 4), tmp_of<T>(pl, 5)};
  long long boff = 0;
  for (int p = 0; p < P; ++p) {
    const T* bp = band + boff;
    if (p == 0) {
      sweep(0, p, bp, v, nullptr, nullptr, A[0], A[1], A[2], T(1));
    } else if (p < P - 1) {
      sweep(1, p, bp, A[0], A[1], A[2], B[0], B[1], B[2], T(1));
      std::swap(A, B);
    } else {
      sweep(2, p, bp, A[0], A[1], A[2], nullptr, nullptr, out, T(scale));
    }
    SPS_CHECK_LAUNCH("penalty sweep");
    boff += 3LL * G.J[p] * BAND;
  }
  return SPS_OK;
}
template int penalty_apply<double>(sps_plan*, int, const double*, double*, double, cudaStream_t);
template int penalty_apply<float>(sps_plan*, int, const float*, float*, double, cudaStream_t);

int penalty_diag(sps_plan* pl, int g, double* d, cudaStream_t st) {
  Level& L = pl->lev[g - 1];
  k_pen_diag<<<grid_blocks(L.geom.K, EW_THREADS), EW_THREADS, 0, st>>>(L.geom.K, L.geom, L.d.band, pl->lam, d, 1);
  SPS_CHECK_LAUNCH("penalty diag");
  return SPS_OK;
}

// f = I c (mode 0) or f -= I c (mode 1); c on level g-1, f on level g.
template <typename T>
int prolong_sub(sps_plan* pl, int g, const T* c, T* f, int mode, cudaStream_t st) {
  const LevelGeom& Gf = pl->lev[g - 1].geom;
  const LevelGeom& Gc = pl->lev[g - 2].geom;
  const int P = pl->P;
  T* tmp[2] = {tmp_of<T>(pl, 6), tmp_of<T>(pl, 7)};
  const T* in = c;
  for (int p = 0; p < P; ++p) {
    long long inner = 1, outer = 1;
    for (int q = p + 1; q < P; ++q) inner *= Gc.J[q];
    for (int q = 0; q < p; ++q) outer *= Gf.J[q];
    const long long Kout = outer * Gf.J[p] * inner;
    const bool last = p == P - 1;
    T* out = last ? f : tmp[p & 1];
    if (Gf.K < (1LL << 31))
      k_prolong_sweep<T, unsigned><<<grid_blocks(Kout, EW_THREADS), EW_THREADS, 0, st>>>(
          (unsigned)Kout, (unsigned)inner, Gc.J[p], Gf.J[p], in, out, last ? mode : 0);
    else
      k_prolong_sweep<T, long long><<<grid_blocks(Kout, EW_THREADS), EW_THREADS, 0, st>>>(
          Kout, inner, Gc.J[p], Gf.J[p], in, out, last ? mode : 0);
    SPS_CHECK_LAUNCH("prolong");
    in = out;
  }
  return SPS_OK;
}
template int prolong_sub<double>(sps_plan*, int, const double*, double*, int, cudaStream_t);
template int prolong_sub<float>(sps_plan*, int, const float*, float*, int, cudaStream_t);

// c = I' (f - fb) with f, fb on level g and c on level g-1.
template <typename T>
int restrict_res(sps_plan* pl, int g, const T* f, const T* fb, T* c, cudaStream_t st) {
  const LevelGeom& Gf = pl->lev[g - 1].geom;
  const LevelGeom& Gc = pl->lev[g - 2].geom;
  const int P = pl->P;
  T* tmp[2] = {tmp_of<T>(pl, 6), tmp_of<T>(pl, 7)};
  const T* in = f;
  const T* inb = fb;
  for (int p = 0; p < P; ++p) {
    long long inner = 1, outer = 1;
    for (int q = p + 1; q < P; ++q) inner *= Gf.J[q];
    for (int q = 0; q < p; ++q) outer *= Gc.J[q];
    const long long Kout = outer * Gc.J[p] * inner;
    T* out = p == P - 1 ? c : tmp[p & 1];
    if (Gf.K < (1LL << 31))
      k_restrict_sweep<T, unsigned><<<grid_blocks(Kout, EW_THREADS), EW_THREADS, 0, st>>>(
          (unsigned)Kout, (unsigned)inner, Gf.J[p], Gc.J[p], in, inb, out);
    else
      k_restrict_sweep<T, long long><<<grid_blocks(Kout, EW_THREADS), EW_THREADS, 0, st>>>(
          Kout, inner, Gf.J[p], Gc.J[p], in, inb, out);
    SPS_CHECK_LAUNCH("restrict");
    in = out;
    inb = nullptr;
  }
  return SPS_OK;
}
template int restrict_res<double>(sps_plan*, int, const double*, const double*, double*, cudaStream_t);
template int restrict_res<float>(sps_plan*, int, const float*, const float*, float*, cudaStream_t);

template <int P, typename TP, bool STENCIL>
int phi_assembly_launch(sps_plan* pl, const Level& L, double* out, cudaStream_t st) {
  constexpr int LOC = 1 << (2 * P);
  constexpr int CB = P <= 3 ? LOC : (P == 4 ? 16 : 4);
  const int rpc = 8;
  if (L.nruns == 0) return SPS_OK;
  dim3 grid((L.nruns + rpc - 1) / rpc, LOC / CB);
  const size_t smem = sizeof(TP) * (RUN_MAX * LOC + RUN_MAX * P * 4);
  SPS_CUDA(cudaFuncSetAttribute(k_coarse_phi<P, TP, STENCIL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                200 * 1024));
  k_coarse_phi<P, TP, STENCIL><<<grid, 256, smem, st>>>(L.run_begin, L.run_cell, L.nruns, rpc, pl->x_sorted,
                                                        pl->dtype == SPS_F64, pl->n, L.geom, out);
  SPS_CHECK_LAUNCH("Phi'Phi assembly");
  return SPS_OK;
}

// Phi_g'Phi_g assembled into `out` (dense K x K, or stencil form): FP64
// basis values and products in FP64 plans; FP32 products with FP64
// accumulation in mixed plans, whose V-cycle runs in FP32.
template <int P>
int coarse_phi_launch(sps_plan* pl, const Level& L, double* out, bool stencil, cudaStream_t st) {
  const bool fp32 = pl->opt.precision == SPS_PREC_MIXED;
  if (fp32) return stencil ? phi_assembly_launch<P, float, true>(pl, L, out, st)
                           : phi_assembly_launch<P, float, false>(pl, L, out, st);
  return stencil ? phi_assembly_launch<P, double, true>(pl, L, out, st)
                 : phi_assembly_launch<P, double, false>(pl, L, out, st);
}

int phi_assembly(sps_plan* pl, const Level& L, double* out, bool stencil, cudaStream_t st) {
  switch (pl->P) {
    case 1: return coarse_phi_launch<1>(pl, L, out, stencil, st);
    case 2: return coarse_phi_launch<2>(pl, L, out, stencil, st);
    case 3: return coarse_phi_launch<3>(pl, L, out, stencil, st);
    case 4: return coarse_phi_launch<4>(pl, L, out, stencil, st);
    case 5: return coarse_phi_launch<5>(pl, L, out, stencil, st);
  }
  set_error("unsupported dimension");
  return SPS_EINVAL;
}

// Assemble A_1 into coarse_A; the inverse Cholesky factor of its Jacobi-scaled
// form, scaled back, into coarse_inv (Z) and its transpose into coarse_invt.
int coarse_assemble(sps_plan* pl, cudaStream_t st) {
  Level& L = pl->lev[0];
  const long long K = L.geom.K;
  SPS_CUDA(cudaMemsetAsync(pl->coarse_A, 0, sizeof(double) * K * K, st));
  int e = phi_assembly(pl, L, pl->coarse_A, false, st);
  if (e) return e;
  k_coarse_penalty<<<grid_blocks(K * K, EW_THREADS), EW_THREADS, 0, st>>>(L.geom, L.d.band, pl->lam,
                                                                          pl->coarse_A);
  SPS_CHECK_LAUNCH("coarse penalty");
  double* sc = pl->coarse_tmp;          // Jacobi scale
  double* piv = sc + K;                  // pivots of the elimination
  double* As = pl->coarse_tmp + 6 * K;   // scaled working copy of A_1 (K x K)
  const int blocks = grid_blocks(K * K, EW_THREADS);
  k_coarse_scale<<<grid_blocks(K, EW_THREADS), EW_THREADS, 0, st>>>(pl->coarse_A, K, sc);
  SPS_CHECK_LAUNCH("coarse scale");
  // The scaled matrix (unit diagonal) is factored as it is.  If a pivot is not
  // positive -- mixed plans assemble A_1 from FP32 products, accurate to about
  // 1e-7 relative, so beyond a scaled condition number near 1e7 the assembled
  // matrix need not be positive definite -- it is refactored with the diagonal
  // shifted by 1e-8, 1e-6, 1e-4 in turn: Z'Z then inverts the nearest definite
  // matrix, as good a coarse correction as those products define.
  int* bad = reinterpret_cast<int*>(pl->coarse_tmp + 4 * K);
  const double shifts[4] = {0.0, 1e-8, 1e-6, 1e-4};
  for (int attempt = 0; attempt < 4; ++attempt) {
    SPS_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
    k_scale_sym<<<blocks, EW_THREADS, 0, st>>>(pl->coarse_A, K, sc, As, shifts[attempt]);
    SPS_CHECK_LAUNCH("coarse scale");
    k_identity<<<blocks, EW_THREADS, 0, st>>>(pl->coarse_inv, K);
    SPS_CHECK_LAUNCH("coarse identity");
    for (int k = 0; k <= K; ++k) k_chol_inv_step<<<blocks, EW_THREADS, 0, st>>>(As, pl->coarse_inv, piv, K, k, bad);
    count_launches(K);
    SPS_CHECK_LAUNCH("coarse elimination");
    int nbad = 0;
    SPS_CUDA(cudaMemcpyAsync(&nbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    SPS_CUDA(cudaStreamSynchronize(st));
    pl->coarse_shift = shifts[attempt];
    if (nbad == 0) break;
    if (attempt == 3) {
      set_error("coarse matrix not positive definite even with a diagonal shift of 1e-4");
      return SPS_EBREAKDOWN;
    }
  }
  k_unscale_transpose<<<blocks, EW_THREADS, 0, st>>>(pl->coarse_inv, pl->coarse_invt, sc, K);
  SPS_CHECK_LAUNCH("coarse unscale");
  return SPS_OK;
}

// Assemble A_g = Phi_g'Phi_g + lambda Lambda_g of level g in stencil form
// (FP64 accumulation; FP32 copy for the mixed V-cycle).
int stencil_assemble(sps_plan* pl, int g, cudaStream_t st) {
  Level& L = pl->lev[g - 1];
  const long long K = L.geom.K;
  const int S = L.S;
  SPS_CUDA(cudaMemsetAsync(L.st_d, 0, sizeof(double) * S * K, st));
  int e = phi_assembly(pl, L, L.st_d, true, st);
  if (e) return e;
  k_stencil_penalty<<<grid_blocks((long long)S * K, EW_THREADS), EW_THREADS, 0, st>>>(L.geom, L.d.band, pl->lam,
                                                                                     L.st_d, S);
  SPS_CHECK_LAUNCH("stencil penalty");
  if (L.st_f) {
    k_d2f_scaled<<<grid_blocks((long long)S * K, EW_THREADS), EW_THREADS, 0, st>>>(L.st_d, L.st_f, (long long)S * K);
    SPS_CHECK_LAUNCH("stencil cast");
  }
  return SPS_OK;
}

template <typename T>
int stencil_apply(sps_plan* pl, int g, const T* v, T* u, cudaStream_t st) {
  Level& L = pl->lev[g - 1];
  const T* A = nullptr;
  if constexpr (sizeof(T) == 8) A = (const T*)L.st_d; else A = (const T*)L.st_f;
  const int blocks = (int)((L.geom.K + 31) / 32);
  // 8 offset groups per row; 32 on small levels, where a few dozen CTAs
  // cannot fill the GPU and each thread's chain of offsets sets the time
  if (L.geom.K <= 16384) {
    const dim3 tb(32, 32);
    switch (pl->P) {
      case 1: k_stencil_spmv<1, T, 32><<<blocks, tb, 0, st>>>(A, L.geom, v, u); break;
      case 2: k_stencil_spmv<2, T, 32><<<blocks, tb, 0, st>>>(A, L.geom, v, u); break;
      case 3: k_stencil_spmv<3, T, 32><<<blocks, tb, 0, st>>>(A, L.geom, v, u); break;
      case 4: k_stencil_spmv<4, T, 32><<<blocks, tb, 0, st>>>(A, L.geom, v, u); break;
      default: k_stencil_spmv<5, T, 32><<<blocks, tb, 0, st>>>(A, L.geom, v, u); break;
    }
  } else {
    const dim3 tb(32, 8);
    switch (pl->P) {
      case 1: k_stencil_spmv<1, T, 8><<<blocks, tb, 0, st>>>(A, L.geom, v, u); break;
      case 2: k_stencil_spmv<2, T, 8><<<blocks, tb, 0, st>>>(A, L.geom, v, u); break;
      case 3: k_stencil_spmv<3, T, 8><<<blocks, tb, 0, st>>>(A, L.geom, v, u); break;
      case 4: k_stencil_spmv<4, T, 8><<<blocks, tb, 0, st>>>(A, L.geom, v, u); break;
      default: k_stencil_spmv<5, T, 8><<<blocks, tb, 0, st>>>(A, L.geom, v, u); break;
    }
  }
  SPS_CHECK_LAUNCH("stencil apply");
  return SPS_OK;
}
template int stencil_apply<double>(sps_plan*, int, const double*, double*, cudaStream_t);
template int stencil_apply<float>(sps_plan*, int, const float*, float*, cudaStream_t);

// e = A_1^-1 r as e = Z'(Z r); in FP64 one step of iterative refinement
// follows: e += Z'Z (r - A_1 e), with the residual from the assembled A_1
// (the refined operator 2M - MAM, M = Z'Z, is symmetric positive definite).
// (the intermediate y = Z r is FP64 in both precisions: Z's entries grow
// like sqrt(cond(A_1)) / sqrt(min diag A_1), beyond what FP32 keeps exactly)
template <typename T>
int coarse_solve(sps_plan* pl, const T* r, T* e, cudaStream_t st) {
  const long long K = pl->lev[0].geom.K;
  const int blocks = (int)std::min<long long>((K * 32 + EW_THREADS - 1) / EW_THREADS, 152LL * 16);
  double* y = pl->coarse_tmp + 2 * K;
  k_gemv<T, double><<<blocks, EW_THREADS, 0, st>>>(pl->coarse_inv, K, r, y, nullptr, 0);
  k_gemv<double, T><<<blocks, EW_THREADS, 0, st>>>(pl->coarse_invt, K, y, e, nullptr, 0);
  count_launches(1);
  SPS_CHECK_LAUNCH("coarse solve");
  if constexpr (sizeof(T) == 8) {
    T* res = (T*)(pl->coarse_tmp + 3 * K);
    k_gemv<T, T><<<blocks, EW_THREADS, 0, st>>>(pl->coarse_A, K, e, res, r, 1);
    k_gemv<T, double><<<blocks, EW_THREADS, 0, st>>>(pl->coarse_inv, K, res, y, nullptr, 0);
    k_gemv<double, T><<<blocks, EW_THREADS, 0, st>>>(pl->coarse_invt, K, y, e, nullptr, 2);
    count_launches(2);
    SPS_CHECK_LAUNCH("coarse refinement");
  }
  return SPS_OK;
}

template <typename T>
int coarse_cg(sps_plan* pl, const T* b, T* e, T* r1, T* p1, cudaStream_t st) {
  Level& L = pl->lev[0];
  LevelVecs<T>& V = vecs<T>(L);
  const long long K = L.geom.K;
  T* q = V.u;
  k_ccg_init<T><<<RED_BLOCKS, EW_THREADS, 0, st>>>(b, V.dinv, e, r1, p1, K, pl->scal, pl->red_part, pl->red_count);
  SPS_CHECK_LAUNCH("coarse CG init");
  int rz_old = C_RZ0, rz_new = C_RZ1;
  for (int it = 0; it < pl->opt.coarse_iters; ++it) {
    SPS_TRY(apply_level<T>(pl, 1, p1, q, st));
    k_ccg_pq<T><<<RED_BLOCKS, EW_THREADS, 0, st>>>(p1, q, K, pl->scal, pl->red_part, pl->red_count);
    k_ccg_update<T><<<RED_BLOCKS, EW_THREADS, 0, st>>>(e, r1, p1, q, V.dinv, K, pl->scal, rz_old, rz_new,
                                                       pl->red_part, pl->red_count);
    k_ccg_dir<T><<<grid_blocks(K, EW_THREADS), EW_THREADS, 0, st>>>(p1, r1, V.dinv, K, pl->scal, rz_old, rz_new);
    count_launches(2);
    SPS_CHECK_LAUNCH("coarse CG step");
    std::swap(rz_old, rz_new);
  }
  return SPS_OK;
}
template int coarse_cg<double>(sps_plan*, const double*, double*, double*, double*, cudaStream_t);
template int coarse_cg<float>(sps_plan*, const float*, float*, float*, float*, cudaStream_t);
template int coarse_solve<double>(sps_plan*, const double*, double*, cudaStream_t);
template int coarse_solve<float>(sps_plan*, const float*, float*, cudaStream_t);

template <typename T>
int vec_scale_mul(T* out, const T* a, const T* b, T s, long long n, cudaStream_t st) {
  k_scale_mul<T><<<grid_blocks(n, EW_THREADS), EW_THREADS, 0, st>>>(out, a, b, s, n);
  SPS_CHECK_LAUNCH("scale mul");
  return SPS_OK;
}
template int vec_scale_mul<double>(double*, const double*, const double*, double, long long, cudaStream_t);
template int vec_scale_mul<float>(float*, const float*, const float*, float, long long, cudaStream_t);

template <typename T>
int vec_jacobi(T* alpha, const T* dinv, const T* b, const T* u, T omega, long long n, cudaStream_t st) {
  k_jacobi<T><<<grid_blocks(n, EW_THREADS), EW_THREADS, 0, st>>>(alpha, dinv, b, u, omega, n);
  SPS_CHECK_LAUNCH("jacobi");
  return SPS_OK;
}
template int vec_jacobi<double>(double*, const double*, const double*, const double*, double, long long, cudaStream_t);
template int vec_jacobi<float>(float*, const float*, const float*, const float*, float, long long, cudaStream_t);

int vec_cast_d2f(float* out, const double* in, long long n, cudaStream_t st) {
  k_cast_d2f<<<grid_blocks(n, EW_THREADS), EW_THREADS, 0, st>>>(out, in, n);
  SPS_CHECK_LAUNCH("cast");
  return SPS_OK;
}
int vec_cast_f2d(double* out, const float* in, long long n, cudaStream_t st) {
  k_cast_f2d<<<grid_blocks(n, EW_THREADS), EW_THREADS, 0, st>>>(out, in, n);
  SPS_CHECK_LAUNCH("cast");
  return SPS_OK;
}
int vec_set_d(double* out, double v, long long n, cudaStream_t st) {
  k_set<double><<<grid_blocks(n, EW_THREADS), EW_THREADS, 0, st>>>(out, v, n);
  SPS_CHECK_LAUNCH("set");
  return SPS_OK;
}
int vec_set_f(float* out, float v, long long n, cudaStream_t st) {
  k_set<float><<<grid_blocks(n, EW_THREADS), EW_THREADS, 0, st>>>(out, v, n);
  SPS_CHECK_LAUNCH("set");
  return SPS_OK;
}
int vec_recip(double* dinv, float* dinv_f, const double* d, long long n, cudaStream_t st) {
  k_recip<<<grid_blocks(n, EW_THREADS), EW_THREADS, 0, st>>>(dinv, dinv_f, d, n);
  SPS_CHECK_LAUNCH("recip");
  return SPS_OK;
}

int vec_residual(double* r, const double* b, const double* u, long long n, double* scal, int slot, sps_plan* pl,
                 cudaStream_t st) {
  k_residual<<<RED_BLOCKS, EW_THREADS, 0, st>>>(r, b, u, n, pl->red_part, pl->red_count, scal + slot);
  SPS_CHECK_LAUNCH("residual");
  return SPS_OK;
}

int dot(sps_plan* pl, const double* a, const double* b, long long n, int slot, cudaStream_t st) {
  k_dot<<<RED_BLOCKS, EW_THREADS, 0, st>>>(a, b, nullptr, n, pl->red_part, pl->red_count, pl->scal + slot);
  SPS_CHECK_LAUNCH("dot");
  return SPS_OK;
}

int dot2(sps_plan* pl, const double* a, const double* b, const double* c, long long n, int slot, cudaStream_t st) {
  k_dot<<<RED_BLOCKS, EW_THREADS, 0, st>>>(a, b, c, n, pl->red_part, pl->red_count, pl->scal + slot);
  SPS_CHECK_LAUNCH("dot2");
  return SPS_OK;
}

int pcg_update_xr(sps_plan* pl, long long n, int rz_slot, cudaStream_t st) {
  k_update_xr<<<RED_BLOCKS, EW_THREADS, 0, st>>>(pl->x, pl->r, pl->p, pl->v, n, pl->scal, rz_slot, pl->red_part,
                                                 pl->red_count);
  SPS_CHECK_LAUNCH("update x r");
  return SPS_OK;
}

int pcg_update_p(sps_plan* pl, long long n, int num_slot, int den_slot, int flexible, cudaStream_t st) {
  k_update_p<<<grid_blocks(n, EW_THREADS), EW_THREADS, 0, st>>>(pl->p, pl->z, n, pl->scal, num_slot, den_slot,
                                                                flexible);
  SPS_CHECK_LAUNCH("update p");
  return SPS_OK;
}

}  // namespace sps

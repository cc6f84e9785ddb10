// Linear readout of the reservoir states (Sec. 1: the readout is the only
// trained part of a reservoir computer).  Ridge regression with a bias
// column, solved on the GPU in FP64:
//
//   Phi = [states[t, 0..N-1], 1]        rows t in [t0, t1)      (m x n, n = N + 1)
//   A   = Phi^T Phi + beta D,  D = diag(1, ..., 1, 0)  (the bias is not penalised)
//   beta = beta_rel * trace(Phi^T Phi) / n
//   w   = A^{-1} Phi^T y                                  (n weights, bias last)
//
// Steps (each a kernel below):
//   1. gram_kernel: the lower triangle of the Gram matrix of the augmented
//      rows [states[t], 1, y_t] (n + 1 columns), column-major, FP64 sums of
//      exact FP64 products of the FP32 states.  Its last row holds Phi^T y.
//   2. ridge_shift_kernel: beta from the trace, added to the state diagonal.
//   3. Blocked right-looking Cholesky A = L L^T over the first n columns, in
//      place (chol_diag_kernel, chol_panel_kernel, chol_update_kernel per
//      block column of kCholB).  The panel solves and trailing updates also
//      run over the augmented row, so that row ends as z = L^{-1} Phi^T y:
//      the forward substitution comes out of the factorisation.
//   4. back_solve_kernel: L^T w = z.
//   predict_kernel: y_hat[t] = states[t] . w[0..N-1] + w[N].
//   nmse_kernel: mean((y_hat - y)^2) and the variance of y over [t0, t1).
//
// No kernel waits on another CTA: the steps are ordered by the stream.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sto {
namespace readout {

constexpr int kGramTile = 64;   // Gram tile edge (outputs per CTA: 64 x 64)
constexpr int kGramKt = 16;     // rows of Phi staged per step
constexpr int kCholB = 32;      // Cholesky block column width
constexpr int kUpdTile = 64;    // trailing-update tile edge

// Element c of augmented row t: the FP32 state, 1 for the bias, y_t last.
__device__ __forceinline__ double aug_elem(const float* __restrict__ states, int64_t ld,
                                           const double* __restrict__ y, int N, int64_t t, int c) {
  if (c < N) return static_cast<double>(states[t * ld + c]);
  if (c == N) return 1.0;
  return y[t];
}

// Lower triangle of G = Phi_aug^T Phi_aug over rows [t0, t1); nr = N + 2
// columns; G column-major with leading dimension nr.  Grid (tiles, tiles),
// blockIdx.x = tile row, blockIdx.y = tile column; 256 threads, 4 x 4
// outputs each (rows ty + 16 a, columns tx + 16 b of the tile).
__global__ void __launch_bounds__(256) gram_kernel(const float* __restrict__ states, int64_t ld,
                                                   const double* __restrict__ y, int N, int64_t t0,
                                                   int64_t t1, double* __restrict__ G) {
  const int I = blockIdx.x, J = blockIdx.y;
  if (J > I) return;
  const int nr = N + 2;
  const int i0 = I * kGramTile, j0 = J * kGramTile;
  __shared__ double Pi[kGramKt][kGramTile];
  __shared__ double Pj[kGramKt][kGramTile];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int64_t tb = t0; tb < t1; tb += kGramKt) {
    // stage kGramKt rows: 16 x 64 elements per tile side, 4 per thread
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = tid + 256 * e;
      const int r = idx >> 6, c = idx & 63;
      const int64_t t = tb + r;
      const bool row_ok = t < t1;
      Pi[r][c] = (row_ok && i0 + c < nr) ? aug_elem(states, ld, y, N, t, i0 + c) : 0.0;
      Pj[r][c] = (row_ok && j0 + c < nr) ? aug_elem(states, ld, y, N, t, j0 + c) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kGramKt; ++k) {
      double pi[4], pj[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) pi[a] = Pi[k][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) pj[b] = Pj[k][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(pi[a], pj[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty + 16 * a;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + tx + 16 * b;
      if (i < nr && j <= i) G[static_cast<int64_t>(j) * nr + i] = acc[a][b];
    }
  }
}

// beta = beta_rel * trace(G[0..n-1]) / n, added to the first n - 1 diagonal
// entries (the states; not the bias at n - 1).  One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) ridge_shift_kernel(double* __restrict__ G, int nr, int n,
                                                           double beta_rel, double* __restrict__ beta_out) {
  __shared__ double part[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += G[static_cast<int64_t>(i) * nr + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) part[0] = v;
  }
  __syncthreads();
  const double beta = beta_rel * part[0] / static_cast<double>(n);
  for (int i = threadIdx.x; i < n - 1; i += blockDim.x) G[static_cast<int64_t>(i) * nr + i] += beta;
  if (threadIdx.x == 0) *beta_out = beta;
}

// Unblocked Cholesky of the kb x kb diagonal block at (k0, k0), in place
// (lower triangle).  One CTA of kCholB x kCholB threads.  A pivot that is not
// positive (or not finite) sets *status and the factor is abandoned.
__global__ void __launch_bounds__(kCholB* kCholB) chol_diag_kernel(double* __restrict__ A, int lda, int k0,
                                                                   int kb, int* __restrict__ status) {
  __shared__ double S[kCholB][kCholB + 1];
  __shared__ int bad;
  const int r = threadIdx.x / kCholB, c = threadIdx.x % kCholB;  // S[r][c]
  if (threadIdx.x == 0) bad = 0;
  if (r < kb && c <= r) S[r][c] = A[static_cast<int64_t>(k0 + c) * lda + k0 + r];
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (threadIdx.x == 0) {
      const double d = S[j][j];
      if (!(d > 0.0) || !isfinite(d)) {
        bad = 1;
        *status = 1;
      } else {
        S[j][j] = sqrt(d);
      }
    }
    __syncthreads();
    if (bad) return;
    if (c == j && r > j && r < kb) S[r][j] /= S[j][j];
    __syncthreads();
    if (r > j && r < kb && c > j && c <= r) S[r][c] -= S[r][j] * S[c][j];
    __syncthreads();
  }
  if (r < kb && c <= r) A[static_cast<int64_t>(k0 + c) * lda + k0 + r] = S[r][c];
}

// Rows i in [k0 + kb, nr) of the block column: x L11^T = a_i, i.e.
// x_j = (a_ij - sum_{l<j} x_l L11[j][l]) / L11[j][j]; one thread per row.
__global__ void __launch_bounds__(256) chol_panel_kernel(double* __restrict__ A, int lda, int nr, int k0,
                                                         int kb, const int* __restrict__ status) {
  __shared__ double L[kCholB][kCholB + 1];
  if (*status) return;
  for (int e = threadIdx.x; e < kCholB * kCholB; e += blockDim.x) {
    const int r = e / kCholB, c = e % kCholB;
    L[r][c] = (r < kb && c <= r) ? A[static_cast<int64_t>(k0 + c) * lda + k0 + r] : 0.0;
  }
  __syncthreads();
  const int64_t i = static_cast<int64_t>(k0) + kb + blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= nr) return;
  double x[kCholB];
#pragma unroll
  for (int j = 0; j < kCholB; ++j) {
    if (j < kb) {
      double v = A[static_cast<int64_t>(k0 + j) * lda + i];
#pragma unroll
      for (int l = 0; l < j; ++l) v -= x[l] * L[j][l];
      x[j] = v / L[j][j];
      A[static_cast<int64_t>(k0 + j) * lda + i] = x[j];
    } else {
      x[j] = 0.0;
    }
  }
}

// Trailing update A[i][j] -= sum_l A[i][k0 + l] A[j][k0 + l] for
// k0 + kb <= j <= i < nr.  Grid (tiles, tiles) over the trailing block,
// blockIdx.x = tile row, blockIdx.y = tile column; 256 threads, 4 x 4 each.
__global__ void __launch_bounds__(256) chol_update_kernel(double* __restrict__ A, int lda, int nr, int k0,
                                                          int kb, const int* __restrict__ status) {
  const int I = blockIdx.x, J = blockIdx.y;
  if (J > I || *status) return;
  const int base = k0 + kb;
  const int i0 = base + I * kUpdTile, j0 = base + J * kUpdTile;
  __shared__ double Li[kCholB][kUpdTile];
  __shared__ double Lj[kCholB][kUpdTile];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int e = tid; e < kCholB * kUpdTile; e += 256) {
    const int l = e / kUpdTile, c = e % kUpdTile;
    const bool lok = l < kb;
    Li[l][c] = (lok && i0 + c < nr) ? A[static_cast<int64_t>(k0 + l) * lda + i0 + c] : 0.0;
    Lj[l][c] = (lok && j0 + c < nr) ? A[static_cast<int64_t>(k0 + l) * lda + j0 + c] : 0.0;
  }
  __syncthreads();
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
#pragma unroll 8
  for (int l = 0; l < kCholB; ++l) {
    double pi[4], pj[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) pi[a] = Li[l][ty + 16 * a];
#pragma unroll
    for (int b = 0; b < 4; ++b) pj[b] = Lj[l][tx + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(pi[a], pj[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty + 16 * a;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + tx + 16 * b;
      if (i < nr && j <= i) A[static_cast<int64_t>(j) * lda + i] -= acc[a][b];
    }
  }
}

// Block-wide sum of one double per thread (1024 threads); every thread gets it.
__device__ __forceinline__ double block_sum_1024(double v, double* part) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = part[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) part[32] = s;
  }
  __syncthreads();
  s = part[32];
  __syncthreads();
  return s;
}

// L^T w = z, z = row nr - 1 of A (columns 0 .. n-1), L the factor in the
// first n columns: w_j = (z_j - sum_{i>j} L[i][j] w_i) / L[j][j] for
// j = n-1 .. 0.  One CTA of 1024 threads; w in global memory.
__global__ void __launch_bounds__(1024) back_solve_kernel(const double* __restrict__ A, int lda, int nr, int n,
                                                          double* __restrict__ w, const int* __restrict__ status) {
  __shared__ double part[33];
  if (*status) return;
  for (int j = threadIdx.x; j < n; j += blockDim.x) w[j] = A[static_cast<int64_t>(j) * lda + (nr - 1)];
  __syncthreads();
  for (int j = n - 1; j >= 0; --j) {
    const double* col = A + static_cast<int64_t>(j) * lda;
    double s = 0.0;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) s = fma(col[i], w[i], s);
    s = block_sum_1024(s, part);
    if (threadIdx.x == 0) w[j] = (w[j] - s) / col[j];
    __syncthreads();
  }
}

// y_hat[t] = sum_k states[t][k] w[k] + w[N], t in [0, T); one warp per row,
// FP64 sums.
__global__ void __launch_bounds__(256) predict_kernel(const float* __restrict__ states, int64_t ld, int N,
                                                      int64_t T, const double* __restrict__ w,
                                                      double* __restrict__ y_hat) {
  const int64_t t = blockIdx.x * 8LL + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= T) return;
  const float* row = states + t * ld;
  double s = 0.0;
  for (int k = lane; k < N; k += 32) s = fma(static_cast<double>(row[k]), w[k], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y_hat[t] = s + w[N];
}

// out[0] = mean over [t0, t1) of (y_hat - y)^2, out[1] = the (population)
// variance of y over the same samples.  One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) nmse_kernel(const double* __restrict__ y_hat, const double* __restrict__ y,
                                                    int64_t t0, int64_t t1, double* __restrict__ out) {
  __shared__ double part[33];
  const double m = static_cast<double>(t1 - t0);
  double s = 0.0;
  for (int64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) s += y[t];
  const double mean = block_sum_1024(s, part) / m;
  double se = 0.0, sv = 0.0;
  for (int64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
    const double e = y_hat[t] - y[t], d = y[t] - mean;
    se = fma(e, e, se);
    sv = fma(d, d, sv);
  }
  se = block_sum_1024(se, part);
  sv = block_sum_1024(sv, part);
  if (threadIdx.x == 0) {
    out[0] = se / m;
    out[1] = sv / m;
  }
}

}  // namespace readout
}  // namespace sto

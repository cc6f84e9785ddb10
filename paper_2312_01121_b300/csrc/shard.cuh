// One row block of a reservoir split across GPUs.  The coupling of Eq. (coup)
// is the matrix-vector product W m^x (Sec. 3.3), so the rows of W and the
// oscillators they drive can live on different GPUs: a GPU that owns the
// rows [row0, row0 + rows) needs, per RK4 stage, only the stage values m^x
// of all N oscillators, which the GPUs exchange (an all-gather of N floats)
// between stages.  One launch of shard_stage_kernel finishes one stage for
// the block:
//
//   h_k   = sum_i W[k, i] x_i                (FP32 products, FP32 sums)
//   d     = dt f(stage state, A_cp h_k + H_in,k)   (double-float, Eq. (gov))
//   RK4 combination of Sec. 3.2, next stage value x'_k = its m^x (FP32)
//
// with the same double-float arithmetic as the single-GPU stepper's owner
// program; only the order of the FP32 row sum differs.  The block's state
// (m_n, the stage state and the RK4 sum as double-float triples, and the
// input field of the current sample) stays in this GPU's memory between
// launches.  Nothing in this file waits on another CTA or another GPU: the
// exchange is the caller's, between launches, ordered by the stream.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "sto_kernel.cuh"

namespace sto {

struct ShardArgs {
  const float* W;     // rows x ld, row-major (ld >= N, a multiple of 4; zero padded)
  const float* w_in;  // rows x n_in
  float2* mn;         // [3][rows] double-float state m_n
  float2* ms;         // [3][rows] stage state
  float2* ks;         // [3][rows] RK4 sum of the increments so far
  float2* hin;        // [rows] input field H_in of the current sample
  int N, ld, rows, n_in, comp;
  KArgs c;            // constants of Eq. (gov) (gdt, alpha, happl, hkp, hs0, lambda, p, acp, sixth, ain_g)
};

enum ShardFlags { kShardSampleStart = 1, kShardSampleEnd = 2 };

__device__ __forceinline__ df ld_df(const float2* p, int i) {
  const float2 v = p[i];
  return df{v.x, v.y};
}
__device__ __forceinline__ void st_df(float2* p, int i, df v) { p[i] = make_float2(v.hi, v.lo); }

// Stage `st` (0..3 of an RK4 step) for the block's oscillators: one warp per
// oscillator k; x = the gathered stage values (N floats, 16-byte aligned).
// flags: kShardSampleStart forms H_in from u_t first (stage 0 of the first
// RK4 step of an input sample); kShardSampleEnd writes the sampled component
// to states_row[k] after stage 3 (the last RK4 step of the sample).
__global__ void __launch_bounds__(256) shard_stage_kernel(const __grid_constant__ ShardArgs a,
                                                          const float* __restrict__ x, int st,
                                                          const float* __restrict__ u_t, int flags,
                                                          float* __restrict__ x_next,
                                                          float* __restrict__ states_row) {
  const int k = static_cast<int>((blockIdx.x * static_cast<unsigned>(blockDim.x) + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= a.rows) return;
  const float* wr = a.W + static_cast<size_t>(k) * a.ld;
  const int n4 = a.N >> 2;
  const float4* w4 = reinterpret_cast<const float4*>(wr);
  const float4* x4 = reinterpret_cast<const float4*>(x);
  float s = 0.f;
  for (int j = lane; j < n4; j += 32) {
    const float4 w = w4[j], v = x4[j];
    s = fmaf(w.x, v.x, s);
    s = fmaf(w.y, v.y, s);
    s = fmaf(w.z, v.z, s);
    s = fmaf(w.w, v.w, s);
  }
  if (lane < (a.N & 3)) s = fmaf(wr[4 * n4 + lane], x[4 * n4 + lane], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane != 0) return;

  const int R = a.rows;
  df mn[3], ms[3], ksum[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    mn[i] = ld_df(a.mn, i * R + k);
    ms[i] = st == 0 ? mn[i] : ld_df(a.ms, i * R + k);
    ksum[i] = st == 0 ? df{0.f, 0.f} : ld_df(a.ks, i * R + k);
  }
  df hin;
  if (flags & kShardSampleStart) {
    double su = 0.0;
    for (int jj = 0; jj < a.n_in; ++jj)
      su += static_cast<double>(a.w_in[static_cast<size_t>(k) * a.n_in + jj]) * static_cast<double>(u_t[jj]);
    hin = df_from_double(a.c.ain_g * su);
    st_df(a.hin, k, hin);
  } else {
    hin = ld_df(a.hin, k);
  }
  df fa[3], fb[3];
  llg_affine(a.c, ms, fa, fb);
  const df hx = df_add(df_mul_f(a.c.acp, s), hin);
  df d[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) d[i] = df_fma(hx, fb[i], fa[i]);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (st == 0) {
      ksum[i] = d[i];
      ms[i] = df_add(mn[i], df_scale2(d[i], 0.5f));
    } else if (st == 1) {
      ksum[i] = df_add(ksum[i], df_scale2(d[i], 2.0f));
      ms[i] = df_add(mn[i], df_scale2(d[i], 0.5f));
    } else if (st == 2) {
      ksum[i] = df_add(ksum[i], df_scale2(d[i], 2.0f));
      ms[i] = df_add(mn[i], d[i]);
    } else {
      ksum[i] = df_add(ksum[i], d[i]);
      mn[i] = df_fma(ksum[i], a.c.sixth, mn[i]);
      ms[i] = mn[i];
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (st == 3) {
      st_df(a.mn, i * R + k, mn[i]);
    } else {
      st_df(a.ms, i * R + k, ms[i]);
      st_df(a.ks, i * R + k, ksum[i]);
    }
  }
  x_next[k] = ms[0].hi;
  if (st == 3 && (flags & kShardSampleEnd) && states_row) states_row[k] = mn[a.comp].hi;
}

// The block's stage values at the start of a run (the first stage is at m_n).
__global__ void shard_publish_kernel(const float2* __restrict__ mn, int rows, float* __restrict__ x_rows) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < rows) x_rows[k] = mn[k].x;
}

// m_n (3 x rows doubles) <-> double-float pairs.
__global__ void shard_state_in_kernel(const double* __restrict__ m, int n, float2* __restrict__ mn) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const df v = df_from_double(m[i]);
    mn[i] = make_float2(v.hi, v.lo);
  }
}
__global__ void shard_state_out_kernel(const float2* __restrict__ mn, int n, double* __restrict__ m) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) m[i] = df_to_double(df{mn[i].x, mn[i].y});
}

// W rows (rows x N, row-major, any alignment) -> rows x ld, zero padded.
__global__ void shard_pad_w_kernel(const float* __restrict__ W, int rows, int N, int ld, float* __restrict__ Wp) {
  const long long total = static_cast<long long>(rows) * ld;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long r = i / ld, c = i % ld;
    Wp[i] = c < N ? W[r * N + c] : 0.f;
  }
}

}  // namespace sto

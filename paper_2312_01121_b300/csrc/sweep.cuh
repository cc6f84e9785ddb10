// Batched parameter sweep: R reservoirs that share one coupling matrix W
// (N x N) but differ in their current I_r and input gain g_r, all driven by
// the same input series.  Per RK4 stage the coupling of every reservoir is
// one dense product
//     D = W X,   X = [m^x of reservoir 0 | ... | m^x of reservoir R-1]
// (N x R), which runs on the 5th-generation tensor cores (tcgen05.mma,
// BF16 operands, FP32 accumulation in tensor memory).  The stage value X is
// split into two BF16 terms, X = X_hi + X_lo, and both are multiplied by the
// BF16-rounded W in one K-concatenated product, so the only rounding the
// product adds to FP32 accumulation is that of W itself.  The per-element
// torque, RK4 combination and state (double-float, as in the single
// reservoir stepper) run in a second kernel over all R x N pairs.
//
// Layouts.  Both product operands are kept in global memory in the order
// the tensor cores read them from shared memory, so one K slice of one tile
// is a single contiguous block fetched with one bulk copy (TMA):
//   Wt   tile (i, j) = rows [128 i, 128 i + 128) x columns [64 j, 64 j + 64)
//        of W (BF16, zero padded), 16 KB at ((i * Kpad/64) + j) * 16 KB;
//   Xt   tile (n, j) = reservoirs [64 n, 64 n + 64) x columns [64 j, 64 j + 64)
//        of [X_hi | X_lo] (K = 2 Kpad), 8 KB at ((n * 2Kpad/64) + j) * 8 KB;
//   inside a tile: 8-row x 16-byte core matrices, column chunk c (8 values)
//   at c * (rows/8) * 128 B, row group g at g * 128 B, row r % 8 at 16 B steps
//   (the no-swizzle K-major layout: LBO = (rows/8) * 128 B, SBO = 128 B).
//   Dt   [R][N] float (D transposed: reservoir-major)
//   state: mn, ms, ksum as df pairs, [3][R][N] each
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "sto_kernel.cuh"

namespace sto {

constexpr int kSwM = 128;          // tile rows (oscillators)
constexpr int kSwN = 64;           // tile columns (reservoirs)
constexpr int kSwK = 64;           // K slice per pipeline stage
constexpr int kSwSlots = 3;        // pipeline depth (96 KB: two CTAs per SM, one wave of tiles)
constexpr int kSwThreads = 128;    // 4 warps: TMEM lanes 0..127
constexpr int kSwSliceA = kSwM * kSwK * 2;        // 16 KB of W
constexpr int kSwSliceB = kSwN * kSwK * 2;        // 8 KB of X_hi, 8 KB of X_lo
constexpr int kSwSlot = kSwSliceA + 2 * kSwSliceB;
constexpr int kSwSmem = kSwSlots * kSwSlot + 128;

struct GemmArgs {
  const __nv_bfloat16* Wb;   // Wt tiles
  const __nv_bfloat16* Xs;   // Xt tiles
  float* Dt;                 // [R][N]
  int* err;                  // int32[4], as the stepper's
  int N, R, Kpad;
  unsigned long long timeout_ns;
};

// Shared-memory matrix descriptor of tcgen05.mma for a K-major operand in the
// no-swizzle layout: 8-row x 16-byte core matrices, `lbo` bytes between
// core matrices adjacent in K, `sbo` bytes between core matrices adjacent in
// rows; bits 46-47 hold the descriptor version (1).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) |
         (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator, BF16
// A and B, both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(m >> 4) << 24);
}

// Element offsets (in BF16 values) of the tiled layouts described above.
__host__ __device__ __forceinline__ size_t wt_offset(int row, int col, int Kpad) {
  const size_t tile = static_cast<size_t>(row / kSwM) * (Kpad / kSwK) + col / kSwK;
  const int r = row % kSwM, c = col % kSwK;
  return tile * (kSwM * kSwK) + ((c / 8) * (kSwM / 8) * 128 + (r / 8) * 128 + (r % 8) * 16 + (c % 8) * 2) / 2;
}
__host__ __device__ __forceinline__ size_t xt_offset(int res, int kcol, int Kpad) {
  const size_t tile = static_cast<size_t>(res / kSwN) * (2 * Kpad / kSwK) + kcol / kSwK;
  const int r = res % kSwN, c = kcol % kSwK;
  return tile * (kSwN * kSwK) + ((c / 8) * (kSwN / 8) * 128 + (r / 8) * 128 + (r % 8) * 16 + (c % 8) * 2) / 2;
}

// One 128 x 64 tile of D = W X_hi + W X_lo per CTA; writes D^T.
// Thread 0 streams K slices (one W tile and the matching X_hi and X_lo
// tiles) with bulk copies into a ring (full / empty mbarriers) and issues the
// MMAs, each W slice serving both halves; all four warps then read the
// accumulator from tensor memory.
__global__ void __launch_bounds__(kSwThreads) sweep_gemm_kernel(const __grid_constant__ GemmArgs g) {
  extern __shared__ __align__(128) unsigned char sw_smem[];
  unsigned char* smem = sw_smem;
  __shared__ uint64_t full[kSwSlots], empty[kSwSlots], done;
  __shared__ uint32_t tmem_base;
  __shared__ int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kSwM, n0 = blockIdx.y * kSwN;
  const int nk = g.Kpad / kSwK;       // K slices of W
  auto slotA = [&](int s) { return smem + s * kSwSlot; };
  auto slotB = [&](int s) { return smem + s * kSwSlot + kSwSliceA; };  // X_hi, then X_lo

  if (tid == 0) {
    for (int s = 0; s < kSwSlots; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    s_ok = 1;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "n"(kSwN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (tid == 0) {
    constexpr uint32_t idesc = umma_idesc_bf16(kSwM, kSwN);
    const __nv_bfloat16* wtile = g.Wb + static_cast<size_t>(blockIdx.x) * nk * (kSwM * kSwK);
    const __nv_bfloat16* xtile = g.Xs + static_cast<size_t>(blockIdx.y) * 2 * nk * (kSwN * kSwK);
    const uint64_t pol = policy_evict_last();
    bool ok = true;
    int p = 0;  // next slice to load
    int c = 0;  // next slice to multiply
    for (; c < nk && ok; ++c) {
      while (p < nk && p < c + kSwSlots) {
        const int s = p % kSwSlots;
        if (p >= kSwSlots && !mbar_wait_bounded(&empty[s], ((p / kSwSlots) - 1) & 1, g.timeout_ns, nullptr)) {
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(&full[s], kSwSlot);
        bulk_g2s(slotA(s), wtile + static_cast<size_t>(p) * (kSwM * kSwK), kSwSliceA, &full[s], pol);
        bulk_g2s(slotB(s), xtile + static_cast<size_t>(p) * (kSwN * kSwK), kSwSliceB, &full[s], pol);
        bulk_g2s(slotB(s) + kSwSliceB, xtile + static_cast<size_t>(nk + p) * (kSwN * kSwK), kSwSliceB,
                 &full[s], pol);
        ++p;
      }
      if (!ok) break;
      const int s = c % kSwSlots;
      if (!mbar_wait_bounded(&full[s], (c / kSwSlots) & 1, g.timeout_ns, nullptr)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(slotA(s)), b0 = smem_u32(slotB(s));
#pragma unroll
      for (int j = 0; j < 2 * (kSwK / 16); ++j) {
        const int jk = j % (kSwK / 16), half = j / (kSwK / 16);  // X_hi, then X_lo
        const uint64_t ad = umma_desc(a0 + jk * 2 * (kSwM / 8) * 128, (kSwM / 8) * 128, 128);
        const uint64_t bd = umma_desc(b0 + half * kSwSliceB + jk * 2 * (kSwN / 8) * 128,
                                      (kSwN / 8) * 128, 128);
        const uint32_t acc = (c > 0 || j > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&empty[s]))
          : "memory");
    }
    if (!ok) {
      report_error(g.err, kErrTimeout, blockIdx.x, 0u, kSiteFull);
      s_ok = 0;
      // copies still in flight land before the CTA leaves
      for (int q = c; q < p; ++q)
        mbar_wait_bounded(&full[q % kSwSlots], (q / kSwSlots) & 1, g.timeout_ns, nullptr);
    }
    // completion of every MMA issued above
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&done))
        : "memory");
  }
  const bool fin = mbar_wait_bounded(&done, 0u, g.timeout_ns, nullptr);
  const bool ok = __syncthreads_and(fin) && s_ok;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    // warp w owns TMEM lanes (tile rows) 32w .. 32w + 31
    const int k = m0 + 32 * warp + lane;
#pragma unroll
    for (int c0 = 0; c0 < kSwN; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + (static_cast<uint32_t>(32 * warp) << 16) + static_cast<uint32_t>(c0);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
            "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (k < g.N) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int r = n0 + c0 + j;
          if (r < g.R) g.Dt[static_cast<size_t>(r) * g.N + k] = __uint_as_float(v[j]);
        }
      }
    }
  } else if (!fin && tid == 0) {
    report_error(g.err, kErrTimeout, blockIdx.x, 0u, kSiteDrain);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kSwN) : "memory");
}

struct EpiArgs {
  const float* Dt;          // [R][N]
  const float* w_in;        // N x n_in (shared)
  const float* u;           // T x n_in
  const int* t_dev;         // current input sample (device counter)
  float2* mn;               // [3][R][N] df
  float2* ms;
  float2* ksum;
  __nv_bfloat16* Xs;        // Xt tiles
  float* states_out;        // [T][R][N] or nullptr
  const df* hs0_r;          // per reservoir H_s0
  const df* ain_g_r;        // per reservoir g A_in
  int N, R, Kpad, n_in, comp, st, last_sub;
  KArgs c;                  // shared constants (gdt, alpha, happl, hkp, lambda, p, acp, sixth)
};

// dt * dm/dt of Eq. (gov) for one oscillator in double-float, with the
// reservoir's own H_s0 and the full x-field hx (coupling + input).
__device__ __forceinline__ void sweep_increment(const KArgs& c, df hs0, const df m[3], df hx,
                                                df d[3]) {
  const df s = df_add(df_add(df_mul(m[0], c.px), df_mul(m[1], c.py)), df_mul(m[2], c.pz));
  const df hs = df_mul(hs0, df_rcp(df_add_f(df_mul(c.lambda, s), 1.0f)));
  const df cx = df_cross1(c.py, m[2], c.pz, m[1]);
  const df cy = df_cross1(c.pz, m[0], c.px, m[2]);
  const df cz = df_cross1(c.px, m[1], c.py, m[0]);
  const df b[3] = {df_add(hx, df_mul(hs, cx)), df_mul(hs, cy),
                   df_add(df_add(c.happl, df_mul(c.hkp, m[2])), df_mul(hs, cz))};
  const df t[3] = {df_cross1(m[1], b[2], m[2], b[1]), df_cross1(m[2], b[0], m[0], b[2]),
                   df_cross1(m[0], b[1], m[1], b[0])};
  const df u[3] = {df_cross1(m[1], t[2], m[2], t[1]), df_cross1(m[2], t[0], m[0], t[2]),
                   df_cross1(m[0], t[1], m[1], t[0])};
#pragma unroll
  for (int i = 0; i < 3; ++i) d[i] = df_mul(c.gdt, df_add(t[i], df_mul(c.alpha, u[i])));
}

// One (reservoir, oscillator) pair per thread: finish stage st with the
// coupling sum from the product, combine RK4, publish the next stage value
// into X (hi and lo BF16 parts) and sample at the end of an input sample.
// Each stage reads and writes only the state it needs: stage 0 evaluates at
// m_n and writes (sum, stage state); stages 1-2 update both; stage 3 writes
// m_{n+1} only (the next stage 0 starts from it).
__global__ void __launch_bounds__(256) sweep_epilogue_kernel(const __grid_constant__ EpiArgs e) {
  // R N <= 2^31 (checked at create): 32-bit index arithmetic
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= static_cast<unsigned>(e.R) * static_cast<unsigned>(e.N)) return;
  const unsigned r = idx / static_cast<unsigned>(e.N), k = idx - r * static_cast<unsigned>(e.N);
  const size_t RN = static_cast<size_t>(e.R) * e.N;
  const int t = *e.t_dev;
  const int st = e.st;
  df mn[3], ms[3], ks[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float2 a = e.mn[i * RN + idx];
    mn[i] = df{a.x, a.y};
    if (st > 0) {
      const float2 b = e.ms[i * RN + idx], c = e.ksum[i * RN + idx];
      ms[i] = df{b.x, b.y};
      ks[i] = df{c.x, c.y};
    } else {
      ms[i] = mn[i];
    }
  }
  // input drive w_in . u_t in double-float (each product exact), no FP64:
  // that pipe runs at 1/64 of the FP32 rate here
  df s = two_prod(e.w_in[static_cast<size_t>(k) * e.n_in], e.u[static_cast<size_t>(t) * e.n_in]);
  for (int j = 1; j < e.n_in; ++j)
    s = df_add(s, two_prod(e.w_in[static_cast<size_t>(k) * e.n_in + j],
                           e.u[static_cast<size_t>(t) * e.n_in + j]));
  const df hx = df_add(df_mul_f(e.c.acp, e.Dt[idx]), df_mul(e.ain_g_r[r], s));
  df d[3];
  sweep_increment(e.c, e.hs0_r[r], ms, hx, d);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (st == 0) {
      ks[i] = d[i];
      ms[i] = df_add(mn[i], df_scale2(d[i], 0.5f));
    } else if (st == 1) {
      ks[i] = df_add(ks[i], df_scale2(d[i], 2.0f));
      ms[i] = df_add(mn[i], df_scale2(d[i], 0.5f));
    } else if (st == 2) {
      ks[i] = df_add(ks[i], df_scale2(d[i], 2.0f));
      ms[i] = df_add(mn[i], d[i]);
    } else {
      ks[i] = df_add(ks[i], d[i]);
      mn[i] = df_add(mn[i], df_mul(ks[i], e.c.sixth));
      ms[i] = mn[i];
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (st == 3) {
      e.mn[i * RN + idx] = make_float2(mn[i].hi, mn[i].lo);
    } else {
      e.ms[i * RN + idx] = make_float2(ms[i].hi, ms[i].lo);
      e.ksum[i * RN + idx] = make_float2(ks[i].hi, ks[i].lo);
    }
  }
  // next stage value, split into two BF16 terms
  const float x = ms[0].hi;
  const __nv_bfloat16 xh = __float2bfloat16_rn(x);
  const __nv_bfloat16 xl = __float2bfloat16_rn(x - __bfloat162float(xh));
  e.Xs[xt_offset(r, k, e.Kpad)] = xh;
  e.Xs[xt_offset(r, e.Kpad + k, e.Kpad)] = xl;
  if (st == 3 && e.last_sub && e.states_out)
    e.states_out[static_cast<size_t>(t) * RN + idx] = mn[e.comp].hi;
}

// Initial X from the stage state (ms) of every pair.
__global__ void sweep_publish_kernel(const float2* ms, __nv_bfloat16* Xs, int N, int R, int Kpad) {
  const long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (idx >= static_cast<long long>(R) * N) return;
  const int r = static_cast<int>(idx / N), k = static_cast<int>(idx % N);
  const float x = ms[idx].x;
  const __nv_bfloat16 xh = __float2bfloat16_rn(x);
  const __nv_bfloat16 xl = __float2bfloat16_rn(x - __bfloat162float(xh));
  Xs[xt_offset(r, k, Kpad)] = xh;
  Xs[xt_offset(r, Kpad + k, Kpad)] = xl;
}

__global__ void sweep_advance_kernel(int* t_dev) { *t_dev += 1; }

// W (float, N x N row-major) -> BF16 Wt tiles (zeroed beforehand).
__global__ void sweep_pack_w_kernel(const float* W, __nv_bfloat16* Wb, int N, int Kpad) {
  const long long total = static_cast<long long>(N) * N;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int k = static_cast<int>(i / N), j = static_cast<int>(i % N);
    Wb[wt_offset(k, j, Kpad)] = __float2bfloat16_rn(W[i]);
  }
}

}  // namespace sto

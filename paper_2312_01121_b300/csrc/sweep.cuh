// Batched parameter sweep: R reservoirs that share one coupling matrix W
// (N x N) but differ in their current I_r and input gain g_r, all driven by
// the same input series.  Per RK4 stage the coupling of every reservoir is
// one dense product
//     D = W X,   X = [m^x of reservoir 0 | ... | m^x of reservoir R-1]
// (N x R), which runs on the 5th-generation tensor cores (tcgen05.mma,
// BF16 operands, FP32 accumulation in tensor memory).  The stage value X is
// split into two BF16 terms, X = X_hi + X_lo, and both are multiplied by the
// BF16-rounded W, so the only rounding the product adds to FP32 accumulation
// is that of W itself.  The two terms are stacked along N (one MMA of width
// 2 BN per K step reads each W slice once; the tensor cores are bound by
// shared-memory bandwidth at these widths) and summed in the epilogue.
//
// One persistent cooperative launch runs a whole sto_run_batched call.  The
// product is cut into tiles of 128 oscillators x BN reservoirs.  Warp 0
// issues the MMAs of a tile into one of two tensor-memory accumulators while
// warps 1-3 stream its K slices (kSlotK W slices and the matching X_hi and
// X_lo slices per ring slot, two 1-D bulk copies) through a shared-memory
// ring; the other 28 warps
// read a finished accumulator with tcgen05.ld and run the per-pair epilogue
// (double-float torque, RK4 combination, BF16 split of the next X, sampling)
// while the next tile's MMAs fill the other accumulator.
//
// Reservoir groups.  Reservoirs are independent: the next stage of a
// reservoir needs only its own column of D.  The tile columns are split into
// `groups` (1 or 2) sets, each with its own grid barrier, and the work runs
// as units (stage g, group q) in the order (0,0), (0,1), (1,0), (1,1), ...
// Unit (g, q) waits only for every CTA's epilogue of (g-1, q), so with two
// groups the MMAs of one group run while the epilogue warps finish the
// other: the tensor-core product and the double-float update overlap
// instead of following each other across a grid-wide barrier.  CTA c takes
// tiles c, c + G, ... of each group.
//
// Layouts.  Both product operands are kept in global memory in the order
// the tensor cores read them from shared memory, so one K slice of one tile
// is a single contiguous block:
//   Wt   tile (i, j) = rows [128 i, 128 i + 128) x columns [64 j, 64 j + 64)
//        of W (BF16, zero padded), 16 KB at ((i * Kpad/64) + j) * 16 KB;
//   Xt   tile (n, j) = columns [64 j, 64 j + 64) of X_hi (rows 0 .. BN-1)
//        and of X_lo (rows BN .. 2BN-1) for reservoirs [BN n, BN n + BN),
//        2 BN * 128 B at ((n * Kpad/64) + j) * 2 BN * 128 B, so one copy
//        brings both terms of a K slice;
//   inside a tile: the 128-byte-swizzled K-major layout the tensor cores read
//   at full shared-memory bandwidth: row r (64 K values = 128 B) at r * 128 B,
//   its 16-byte chunk c (8 values) stored at chunk position c ^ (r % 8); 8-row
//   groups are 1024 B apart (SBO), and slots start on 1024-byte boundaries.
//   state: mn, ms, ksum as df pairs, [3][R][N] each.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "sto_kernel.cuh"

namespace sto {

constexpr int kSwM = 128;          // tile rows (oscillators) = TMEM lanes
constexpr int kSwK = 64;           // K slice per copy
constexpr int kSwSliceA = kSwM * kSwK * 2;             // 16 KB of W per slice
// K slices per ring slot: one wait, 8 MMAs and one commit per slot (the
// MMA thread's fixed cost per slot is about that of 4 MMAs); Kpad is a
// multiple of kSlotK * kSwK
constexpr int kSlotK = 2;
// Three warps issue the copies, warp p owning the ring slots s = p (mod 3);
// the ring holds 2 to 9 slots (with 2 the third copy warp idles).
constexpr int kSpProducers = 3;
constexpr int kSpEpiFirst = 1 + kSpProducers;          // warp 0 multiplies, 1..3 copy
constexpr int kSpMaxSlots = 9;
constexpr unsigned kSpPollSleepNs = 100;  // copy warps' pause between polls of a unit release
// Epilogue warps per TMEM lane quarter (EPQ, a template parameter of the
// kernel): 7 (1024 threads of 64 registers) or 3 (512 threads of 128
// registers, room to hold the next pair's state while the current one is
// computed, and the block shape of the single-reservoir stepper).
template <int EPQ>
constexpr int sp_threads() {
  return 32 * (kSpEpiFirst + 4 * EPQ);
}

struct SweepArgs {
  const __nv_bfloat16* Wb;   // Wt tiles
  __nv_bfloat16* X0;         // Xt tiles read by even stages (written by odd ones)
  __nv_bfloat16* X1;         // Xt tiles read by odd stages
  float2* mn;                // [3][R][N] df
  float2* ms;
  float2* ksum;
  float* states_out;         // [T][R][N] or nullptr
  const float* w_in;         // N x n_in (shared)
  const float* u;            // T x n_in
  const df* hs0_r;           // per reservoir H_s0
  const df* ain_g_r;         // per reservoir g A_in
  int* err;                  // int32[4], as the stepper's
  unsigned long long* gbar;  // one grid barrier counter per group, zero at launch
  int N, R, Kpad, n_in, comp, S, T;
  int bn, slots, tiles_m, tiles_n, acc_cols;  // plan: tile width, ring depth, tiles, TMEM columns per accumulator
  int groups, tn_split;      // reservoir groups (1 or 2); group 0 = tile columns [0, tn_split)
  int staged;                // 1: the next pair's state is loaded into registers ahead
  unsigned long long timeout_ns;
  KArgs c;                   // shared constants (gdt, alpha, happl, hkp, lambda, p, acp, sixth)
};

// Shared-memory matrix descriptor of tcgen05.mma for a K-major operand in the
// 128-byte swizzle layout: start address >> 4 (bits 0-13), the unused
// leading-dimension offset (1), 1024 B between 8-row groups (bits 32-45),
// descriptor version 1 (bits 46-47), layout type 2 = 128-byte swizzle (bits
// 61-63).  The K steps of 16 values inside a 128-byte row advance the start
// address by 32 B; the swizzle is applied to the final address bits.
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) | (1ull << 16) | (static_cast<uint64_t>(1024 >> 4) << 32) |
         (1ull << 46) | (2ull << 61);
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator, BF16
// A and B, both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(m >> 4) << 24);
}

// Element offset (in BF16 values) of (row r, K value c) inside one swizzled
// 64-wide K slice, and of the tiled layouts described above.
__host__ __device__ __forceinline__ int sw128_offset(int r, int c) {
  return r * 64 + (((c >> 3) ^ (r & 7)) << 3) + (c & 7);
}
__host__ __device__ __forceinline__ size_t wt_offset(int row, int col, int Kpad) {
  const size_t tile = static_cast<size_t>(row / kSwM) * (Kpad / kSwK) + col / kSwK;
  return tile * (kSwM * kSwK) + sw128_offset(row % kSwM, col % kSwK);
}
// kcol in [0, 2 Kpad): columns [0, Kpad) are X_hi, [Kpad, 2 Kpad) X_lo.
__host__ __device__ __forceinline__ size_t xt_offset(int res, int kcol, int Kpad, int bn) {
  const int term = kcol >= Kpad ? 1 : 0, kk = kcol - term * Kpad;
  const size_t tile = static_cast<size_t>(res / bn) * (Kpad / kSwK) + kk / kSwK;
  return tile * (2 * static_cast<size_t>(bn) * kSwK) + sw128_offset(term * bn + res % bn, kk % kSwK);
}

// dt * dm/dt of Eq. (gov) for one oscillator in double-float (the damping
// term's inner cross product in FP32), with the reservoir's own H_s0 and the
// full x-field hx (coupling + input).
__device__ __forceinline__ void sweep_increment(const KArgs& c, df hs0, const df m[3], df hx,
                                                df d[3]) {
  df s, pm[3];
  df_p_terms(c.px, c.py, c.pz, m, &s, pm);
  const df hs = df_mul(hs0, df_rcp(df_add_f(df_mul(c.lambda, s), 1.0f)));
  const df b[3] = {df_fma(hs, pm[0], hx), df_mul(hs, pm[1]),
                   df_fma(hs, pm[2], df_fma(c.hkp, m[2], c.happl))};
  const df t[3] = {df_cross1(m[1], b[2], m[2], b[1]), df_cross1(m[2], b[0], m[0], b[2]),
                   df_cross1(m[0], b[1], m[1], b[0])};
  // the damping term m x (m x b) enters scaled by alpha = 0.005: formed in
  // FP32 from the hi words, its rounding is ~3e-10 of the increment
  const float uf[3] = {__fmaf_rn(m[1].hi, t[2].hi, -__fmul_rn(m[2].hi, t[1].hi)),
                       __fmaf_rn(m[2].hi, t[0].hi, -__fmul_rn(m[0].hi, t[2].hi)),
                       __fmaf_rn(m[0].hi, t[1].hi, -__fmul_rn(m[1].hi, t[0].hi))};
#pragma unroll
  for (int i = 0; i < 3; ++i) d[i] = df_mul(c.gdt, df_add_f(t[i], __fmul_rn(c.alpha.hi, uf[i])));
}

// Finish stage ST of pair (reservoir r, oscillator k; element idx = r N + k
// of the [3][R][N] state arrays) with the coupling sum hraw, given the
// pair's state (mn; ms and ks when ST > 0) and the input drive w_in . u_t of
// oscillator k: the RK4 combination, the next stage's X (hi and lo BF16
// terms, at element offsets xo and xo + lo_off of Xn) and the sample at the
// end of an input sample.  Each stage writes only the state the next one
// reads: stages 0-2 write (sum, stage state); stage 3 writes m_{n+1} only
// (the next stage 0 starts from it).  Offsets are 32-bit: the batch keeps
// R N <= 2^29, so 3 R N and the X extent stay below 2^31.
template <int ST>
__device__ __forceinline__ void sweep_pair(const SweepArgs& a, df hs0, df ain_g, unsigned idx, unsigned RN,
                                           float hraw, int t, bool sample, df drive, df mn[3], df ms[3],
                                           df ks[3], __nv_bfloat16* Xn, unsigned xo, unsigned lo_off) {
  if constexpr (ST == 0) {
#pragma unroll
    for (int i = 0; i < 3; ++i) ms[i] = mn[i];
  }
  const df hx = df_fma(ain_g, drive, df_mul_f(a.c.acp, hraw));
  df d[3];
  sweep_increment(a.c, hs0, ms, hx, d);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if constexpr (ST == 0) {
      ks[i] = d[i];
      ms[i] = df_add(mn[i], df_scale2(d[i], 0.5f));
    } else if constexpr (ST == 1) {
      ks[i] = df_add(ks[i], df_scale2(d[i], 2.0f));
      ms[i] = df_add(mn[i], df_scale2(d[i], 0.5f));
    } else if constexpr (ST == 2) {
      ks[i] = df_add(ks[i], df_scale2(d[i], 2.0f));
      ms[i] = df_add(mn[i], d[i]);
    } else {
      ks[i] = df_add(ks[i], d[i]);
      mn[i] = df_fma(ks[i], a.c.sixth, mn[i]);
      ms[i] = mn[i];
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if constexpr (ST == 3) {
      a.mn[i * RN + idx] = make_float2(mn[i].hi, mn[i].lo);
    } else {
      a.ms[i * RN + idx] = make_float2(ms[i].hi, ms[i].lo);
      a.ksum[i * RN + idx] = make_float2(ks[i].hi, ks[i].lo);
    }
  }
  const float x = ms[0].hi;
  const __nv_bfloat16 xh = __float2bfloat16_rn(x);
  const __nv_bfloat16 xl = __float2bfloat16_rn(x - __bfloat162float(xh));
  Xn[xo] = xh;
  Xn[xo + lo_off] = xl;
  if constexpr (ST == 3) {
    if (sample && a.states_out) a.states_out[static_cast<size_t>(t) * RN + idx] = mn[a.comp].hi;
  }
}

constexpr int kSpAlignSlack = 1024;                        // room to align the ring

__device__ __forceinline__ void red_release_add(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Unit release from the MMA thread to the copy warps: a monotonic counter in
// shared memory (units released so far).  A counter, not an mbarrier phase:
// with empty units the MMA thread can release two units before a copy warp
// looks, which a phase parity cannot tell apart.
__device__ __forceinline__ void st_release_cta_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.cta.shared::cta.u64 [%0], %1;" ::"r"(smem_u32(p)), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_cta_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.cta.shared::cta.u64 %0, [%1];" : "=l"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// Tiles of group q: count, and the (tm, tn) of the group's tile `idx`.
__device__ __forceinline__ int sweep_group_tiles(const SweepArgs& a, int q) {
  return a.tiles_m * (q == 0 ? a.tn_split : a.tiles_n - a.tn_split);
}
__device__ __forceinline__ void sweep_tile(const SweepArgs& a, int q, int idx, int* tm, int* tn) {
  *tm = idx % a.tiles_m;
  *tn = idx / a.tiles_m + (q == 0 ? 0 : a.tn_split);
}

// The state of one pair (mn; ms and ks when ST > 0) read from the [3][R][N]
// arrays at element idx, and its reservoir r's H_s0 and g A_in, or zeros for
// a pair outside the batch.  The reservoir constants are read here, with the
// state, rather than where the update first needs them: with the ring in
// shared memory little L1 is left, and a load issued there sat on the
// update's dependency chain.
struct PairState {
  df m[3], s[3], k[3];
  df hs0, ain_g;
};
template <int ST>
__device__ __forceinline__ PairState load_pair(const SweepArgs& a, unsigned RN, unsigned r, unsigned idx,
                                               bool ok) {
  PairState p;
  if (ok) {
    p.hs0 = a.hs0_r[r];
    p.ain_g = a.ain_g_r[r];
#pragma unroll
    for (int qq = 0; qq < 3; ++qq) {
      const float2 x0 = a.mn[qq * RN + idx];
      p.m[qq] = df{x0.x, x0.y};
      if constexpr (ST > 0) {
        const float2 x1 = a.ms[qq * RN + idx], x2 = a.ksum[qq * RN + idx];
        p.s[qq] = df{x1.x, x1.y};
        p.k[qq] = df{x2.x, x2.y};
      }
    }
  } else {
    p = PairState{};
  }
  return p;
}

// The epilogue of one tile for one epilogue warp: the pairs (reservoir
// tn * bn + jc, oscillator k = this lane's TMEM row) for jc = wi, wi + EPQ,
// ...  With PREF the state of the next column's pair is loaded into
// registers while the current one is computed, and the first pair's before
// the accumulator is waited for (the loads overlap the tile's MMAs).  tacc
// addresses this warp's TMEM lanes of the accumulator; xk is the X offset of
// (jc = 0, k).  Returns false when the accumulator never filled (timeout or
// abort).
template <int ST, bool PREF, int EPQ>
__device__ __forceinline__ bool sweep_tile_update(const SweepArgs& a, uint32_t tacc, int tn, unsigned k,
                                                  bool row_ok, unsigned xk, unsigned kchunk, df drive, int t,
                                                  bool sample, __nv_bfloat16* Xn, unsigned lo_off, int wi,
                                                  uint64_t* acc_bar, uint32_t acc_parity,
                                                  const volatile int* abort_flag) {
  const unsigned R = static_cast<unsigned>(a.R), N = static_cast<unsigned>(a.N), RN = R * N;
  constexpr unsigned kStep = EPQ;
  const unsigned istep = kStep * N;
  unsigned r = static_cast<unsigned>(tn * a.bn + wi), idx = r * N + k;
  PairState cur, nxt;
  if constexpr (PREF) nxt = load_pair<ST>(a, RN, r, idx, row_ok && r < R);
  const bool landed = mbar_wait_bounded(acc_bar, acc_parity, a.timeout_ns, abort_flag);
  if (!__all_sync(0xffffffffu, landed)) return false;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  for (int jc = wi; jc < a.bn; jc += kStep, r += kStep, idx += istep) {
    uint32_t vh, vl;  // W X_hi and W X_lo of this pair
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(vh) : "r"(tacc + jc));
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(vl) : "r"(tacc + a.bn + jc));
    const bool pair_ok = row_ok && r < R;
    if constexpr (PREF) {
      cur = nxt;
      if (jc + static_cast<int>(kStep) < a.bn)
        nxt = load_pair<ST>(a, RN, r + kStep, idx + istep, row_ok && r + kStep < R);
    } else {
      cur = load_pair<ST>(a, RN, r, idx, pair_ok);
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const float hraw = __fadd_rn(__uint_as_float(vh), __uint_as_float(vl));
    if (pair_ok) {
      const unsigned xo = xk + static_cast<unsigned>(jc) * 64u + ((kchunk ^ (static_cast<unsigned>(jc) & 7u)) << 3);
      sweep_pair<ST>(a, cur.hs0, cur.ain_g, idx, RN, hraw, t, sample, drive, cur.m, cur.s, cur.k, Xn, xo,
                     lo_off);
    }
  }
  return true;
}

// The whole sweep call for CTA `cta` of the G CTAs that run it: 4 S T
// stages of every group.  Warp 0 (one thread) passes each unit's group
// barrier, releases the unit to the copy warps and issues the MMAs; warps
// 1-3 (one thread each) fill their ring slots; the other 4 EPQ warps run the
// epilogue.  smem_raw: the CTA's dynamic shared memory (the ring).
template <int EPQ>
__device__ __forceinline__ void sweep_cta(const SweepArgs& a, const int cta, const int G,
                                          unsigned char* smem_raw) {
  constexpr int kSpEpiWarps = 4 * EPQ;
  // the swizzle pattern repeats every 1024 B: the ring starts on such a boundary
  unsigned char* sp_smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ uint64_t full[kSpMaxSlots], empty[kSpMaxSlots], acc_full[2], acc_empty[2];
  __shared__ uint64_t stage_done[2], drain;
  __shared__ unsigned long long s_go;  // units released to the copy warps
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_grp = a.groups;
  // this CTA's tiles of each group, and the CTAs with tiles in each group
  const int T0 = sweep_group_tiles(a, 0), T1 = n_grp > 1 ? sweep_group_tiles(a, 1) : 0;
  const int my0 = cta < T0 ? (T0 - 1 - cta) / G + 1 : 0, my1 = cta < T1 ? (T1 - 1 - cta) / G + 1 : 0;
  const int G0 = T0 < G ? T0 : G, G1 = T1 < G ? T1 : G;
  auto n_my = [&](int q) { return q == 0 ? my0 : my1; };
  const int nk = a.Kpad / kSwK;
  const uint32_t sliceB = static_cast<uint32_t>(a.bn) * kSwK * 2;  // one X slice (hi or lo)
  // slot: kSlotK W slices, then the kSlotK matching [X_hi | X_lo] slices
  const uint32_t slot_bytes = kSlotK * (kSwSliceA + 2 * sliceB);
  const int nkk = nk / kSlotK;  // slots per tile
  const long long n_stages = 4LL * a.S * a.T;
  const long long n_units = n_stages * n_grp;
  const volatile int* abort_flag = &s_abort;

  if (tid == 0) {
    for (int s = 0; s < a.slots; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kSpEpiWarps);
      mbar_init(&stage_done[b], kSpEpiWarps);
    }
    mbar_init(&drain, 1);
    s_go = 0;
    s_abort = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(2u * a.acc_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      // ----------------------------------------- group barriers and MMAs
      const uint32_t idesc = umma_idesc_bf16(kSwM, 2 * a.bn);  // [X_hi | X_lo] rows
      long long seq = 0;  // accumulator sequence number of the unit's first tile
      // ring slot and phase parity of the next position: positions run
      // contiguously through all units, so both advance by counting (a 64-bit
      // division by the ring depth per K slice cost more than its MMAs)
      int s = 0;
      uint32_t ph = 0;
      // shared-memory descriptors of the slot's operands (umma_desc_sw128) as
      // two 32-bit words: the start address advances by 32 B (2 in the
      // address field) per K step of 16; the high word is the same for all
      const uint32_t slot0 = smem_u32(sp_smem);
      const uint32_t d_hi = static_cast<uint32_t>(umma_desc_sw128(slot0) >> 32);
      uint32_t a_addr = slot0;  // slot s
      bool ok = true;
      for (long long u = 0; u < n_units && ok; ++u) {
        const long long g = u / n_grp;
        const int q = static_cast<int>(u % n_grp);
        const int nm = n_my(q);
        if (g > 0 && nm > 0) {
          // group barrier: this CTA's epilogue of (g-1, q) is done (its X of
          // the group for stage g written), then every CTA's of the group
          if (!mbar_wait_bounded(&stage_done[q], static_cast<uint32_t>((g - 1) & 1), a.timeout_ns, abort_flag)) {
            ok = false;
            break;
          }
          red_release_add(a.gbar + q, 1ull);
          const unsigned long long target =
              static_cast<unsigned long long>(q == 0 ? G0 : G1) * static_cast<unsigned long long>(g);
          const unsigned long long t0 = gtimer();
          for (uint32_t n = 1; ld_acquire_u64(a.gbar + q) < target; ++n) {
            if ((n & 31u) == 0) {
              if (ld_relaxed_i32(a.err) != 0 || gtimer() - t0 > a.timeout_ns) {
                ok = false;
                break;
              }
            }
          }
          if (!ok) break;
          fence_proxy_async_global();
        }
        st_release_cta_u64(&s_go, static_cast<unsigned long long>(u + 1));  // the copy warps may read this unit's X
        for (int i = 0; i < nm && ok; ++i) {
          const long long sq = seq + i;
          for (int j = 0; j < nkk; ++j) {
            const int b = static_cast<int>(sq & 1);
            if (j == 0 && sq >= 2) {
              // the epilogue has read this accumulator's previous tile
              if (!mbar_wait_bounded(&acc_empty[b], static_cast<uint32_t>(((sq >> 1) - 1) & 1), a.timeout_ns,
                                     abort_flag)) {
                ok = false;
                break;
              }
            }
            if (!mbar_wait_bounded(&full[s], ph, a.timeout_ns, abort_flag)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t dt = tmem + static_cast<uint32_t>(b * a.acc_cols);
#pragma unroll
            for (int h = 0; h < kSlotK; ++h) {
              const uint32_t a_lo = static_cast<uint32_t>(umma_desc_sw128(a_addr + h * kSwSliceA));
              const uint32_t b_lo =
                  static_cast<uint32_t>(umma_desc_sw128(a_addr + kSlotK * kSwSliceA + h * 2 * sliceB));
#pragma unroll
              for (int jk = 0; jk < kSwK / 16; ++jk) {
                // B: the X_hi slice and the X_lo slice behind it, 2 bn rows
                const uint32_t accum = (j > 0 || h > 0 || jk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t.reg .b64 ad, bd;\n\t"
                    "setp.ne.u32 p, %4, 0;\n\t"
                    "mov.b64 ad, {%1, %5};\n\t"
                    "mov.b64 bd, {%2, %5};\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], ad, bd, %3, p;\n\t}" ::"r"(dt),
                    "r"(a_lo + 2u * jk), "r"(b_lo + 2u * jk), "r"(idesc), "r"(accum), "r"(d_hi)
                    : "memory");
              }
            }
            umma_commit(&empty[s]);
            if (j == nkk - 1) umma_commit(&acc_full[b]);
            a_addr += slot_bytes;
            if (++s == a.slots) {
              s = 0;
              ph ^= 1u;
              a_addr = slot0;
            }
          }
        }
        seq += nm;
      }
      if (!ok) {
        if (!*abort_flag) report_error(a.err, kErrTimeout, cta, 0u, kSiteFull);
        s_abort = 1;
        // never leave with MMAs in flight
        umma_commit(&drain);
        mbar_wait_bounded(&drain, 0u, a.timeout_ns, nullptr);
      }
    }
  } else if (warp < kSpEpiFirst) {
    if (lane == 0) {
      // ------------------------------------------------------------ copies
      // this warp owns the ring slots s = pid (mod kSpProducers) and issues
      // every position P that lands in one of them (s = P % slots)
      const int pid = warp - 1;
      const uint64_t pol = policy_evict_last();
      long long last = -1;  // last position issued
      // position, its ring slot and that slot's phase parity, by counting
      // (no 64-bit division by the ring depth per position)
      long long P = 0;
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (long long u = 0; u < n_units && ok; ++u) {
        if (ld_acquire_cta_u64(&s_go) <= static_cast<unsigned long long>(u)) {
          // the next unit is released when the group's barrier passes, most
          // of a stage away: poll gently (a tight loop of shared-memory loads
          // took issue slots from the update warps of the same SM)
          const unsigned long long t0 = gtimer();
          for (uint32_t n = 1; ld_acquire_cta_u64(&s_go) <= static_cast<unsigned long long>(u); ++n) {
            if (n > 8) __nanosleep(kSpPollSleepNs);
            if ((n & 15u) == 0 && (*abort_flag || gtimer() - t0 > a.timeout_ns)) {
              ok = false;
              break;
            }
          }
          if (!ok) break;
        }
        fence_proxy_async_global();  // the released X writes, before this warp's bulk copies read them
        const long long g = u / n_grp;
        const int q = static_cast<int>(u % n_grp);
        const __nv_bfloat16* X = (g & 1) ? a.X1 : a.X0;
        const int nm = n_my(q);
        for (int i = 0; i < nm && ok; ++i) {
          int tm, tn;
          sweep_tile(a, q, cta + i * G, &tm, &tn);
          const __nv_bfloat16* Wt = a.Wb + static_cast<size_t>(tm) * nk * (kSwM * kSwK);
          const __nv_bfloat16* xt = X + static_cast<size_t>(tn) * nk * (2 * a.bn * kSwK);
          for (int j = 0; j < nkk; ++j, ++P) {
            if (s % kSpProducers == pid) {
              // the slot's previous use (lap - 1, parity ph ^ 1) has been consumed
              if (P >= a.slots && !mbar_wait_bounded(&empty[s], ph ^ 1u, a.timeout_ns, abort_flag)) {
                ok = false;
                break;
              }
              unsigned char* slot = sp_smem + static_cast<size_t>(s) * slot_bytes;
              mbar_arrive_expect_tx(&full[s], slot_bytes);
              // K slices kSlotK j .. kSlotK j + kSlotK - 1 are adjacent tiles of both operands
              bulk_g2s(slot, Wt + static_cast<size_t>(kSlotK * j) * (kSwM * kSwK), kSlotK * kSwSliceA, &full[s],
                       pol);
              bulk_g2s(slot + kSlotK * kSwSliceA, xt + static_cast<size_t>(kSlotK * j) * (2 * a.bn * kSwK),
                       kSlotK * 2 * sliceB, &full[s], pol);  // X_hi and X_lo rows
              last = P;
            }
            if (++s == a.slots) {
              s = 0;
              ph ^= 1u;
            }
          }
        }
      }
      if (!ok) {
        if (!*abort_flag) report_error(a.err, kErrTimeout, cta, 0u, kSiteEmpty);
        s_abort = 1;
      }
      // never leave with copies in flight: the latest use of each own slot
      // (every own position up to `last` was issued, so it lies in (last - slots, last])
      for (long long P = last; P >= 0 && P > last - a.slots; --P)
        if (static_cast<int>(P % a.slots) % kSpProducers == pid &&
            !mbar_wait_bounded(&full[P % a.slots], static_cast<uint32_t>((P / a.slots) & 1), a.timeout_ns, nullptr)) {
          report_error(a.err, kErrTimeout, cta, 0u, kSiteDrain);
          break;
        }
    }
  } else {
    // ---------------------------------------------------------- epilogue
    const int q4 = warp & 3;                      // TMEM lanes 32 q4 .. 32 q4 + 31
    const int wi = (warp - kSpEpiFirst) >> 2;     // 0 .. EPQ - 1
    const uint32_t lane_base = static_cast<uint32_t>(32 * q4) << 16;
    // row jc + BN of a slice holds X_lo; BN % 8 == 0 keeps its swizzle phase
    const unsigned lo_off = static_cast<unsigned>(a.bn) * kSwK;
    long long seq = 0;
    bool ok = true;
    for (long long u = 0; u < n_units && ok; ++u) {
      const long long g = u / n_grp;
      const int q = static_cast<int>(u % n_grp);
      const int nm = n_my(q);
      if (nm == 0) continue;  // no tiles of this group here (and no barrier arrival)
      const int st = static_cast<int>(g & 3);
      const long long step = g >> 2;
      const int t = static_cast<int>(step / a.S);
      const bool sample = (step % a.S) == a.S - 1;
      __nv_bfloat16* Xn = (g & 1) ? a.X0 : a.X1;  // the next stage's operand
      for (int i = 0; i < nm; ++i, ++seq) {
        int tm, tn;
        sweep_tile(a, q, cta + i * G, &tm, &tn);
        const int b = static_cast<int>(seq & 1);
        const unsigned k = static_cast<unsigned>(tm * kSwM + 32 * q4 + lane);
        const bool row_ok = k < static_cast<unsigned>(a.N);
        // X offset of (reservoir tn*bn + jcol, oscillator k), hi term: slice
        // base + sw128_offset(jcol, k % 64)
        const unsigned xk = (static_cast<unsigned>(tn) * nk + (k >> 6)) * (2u * a.bn * kSwK) + (k & 7u);
        const unsigned kchunk = (k & 63u) >> 3;
        // input drive of oscillator k for this sample (the same for every reservoir)
        df drive{0.f, 0.f};
        if (row_ok) {
          drive = two_prod(a.w_in[static_cast<size_t>(k) * a.n_in], a.u[static_cast<size_t>(t) * a.n_in]);
          for (int jj = 1; jj < a.n_in; ++jj)
            drive = df_add(drive, two_prod(a.w_in[static_cast<size_t>(k) * a.n_in + jj],
                                           a.u[static_cast<size_t>(t) * a.n_in + jj]));
        }
        const uint32_t tacc = tmem + lane_base + static_cast<uint32_t>(b * a.acc_cols);
        const uint32_t par = static_cast<uint32_t>((seq >> 1) & 1);
        bool landed = false;
#define STO_SWEEP_TILE(ST_, STAGED_)                                                                 \
  landed = sweep_tile_update<ST_, (STAGED_) && EPQ == 3, EPQ>(a, tacc, tn, k, row_ok, xk, kchunk, drive, t, sample, Xn, \
                                                lo_off, wi, &acc_full[b], par, abort_flag)
        if (EPQ == 3 && a.staged) {
          switch (st) {
            case 0: STO_SWEEP_TILE(0, true); break;
            case 1: STO_SWEEP_TILE(1, true); break;
            case 2: STO_SWEEP_TILE(2, true); break;
            default: STO_SWEEP_TILE(3, true); break;
          }
        } else {
          switch (st) {
            case 0: STO_SWEEP_TILE(0, false); break;
            case 1: STO_SWEEP_TILE(1, false); break;
            case 2: STO_SWEEP_TILE(2, false); break;
            default: STO_SWEEP_TILE(3, false); break;
          }
        }
#undef STO_SWEEP_TILE
        if (!landed) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[b]);
      }
      if (!ok) break;
      fence_proxy_async_global();  // this unit's X writes, before the copies of the next
      __syncwarp();
      if (lane == 0) mbar_arrive(&stage_done[q]);
    }
    if (!ok && lane == 0) {
      if (!*abort_flag) report_error(a.err, kErrTimeout, cta, 0u, kSiteFull);
      s_abort = 1;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2u * a.acc_cols)
                 : "memory");
  }
}

template <int EPQ>
__global__ void __launch_bounds__(sp_threads<EPQ>(), 1) sweep_persistent_kernel(const __grid_constant__ SweepArgs a) {
  extern __shared__ __align__(1024) unsigned char sp_smem_raw[];
  sweep_cta<EPQ>(a, blockIdx.x, gridDim.x, sp_smem_raw);
}

// A whole parameter sweep in one cooperative launch: CTAs [0, sweep_ctas)
// run the shared-W reservoirs (sweep_cta, tensor-core product and update),
// the CTAs after them the own-W group's lanes (group_cta, the stepper
// engine).  Both roles run 512 threads; no CTA of one role waits for one of
// the other, and each role's waits are the ones of its lone launch.
struct SweepGroupArgs {
  SweepArgs sw;
  GroupArgs grp;
  int sweep_ctas;
};
static_assert(sp_threads<3>() == kThreads, "the sweep's 512-thread form has the stepper's block shape");

__global__ void __launch_bounds__(kThreads, 1) sweep_group_kernel(const __grid_constant__ SweepGroupArgs f) {
  // 128-byte alignment, as the stepper engine's: sweep_cta aligns its ring to
  // 1024 B inside the region (the plan's slack), so the static part stays small
  extern __shared__ __align__(128) unsigned char sg_smem_raw[];
  const int c = static_cast<int>(blockIdx.x);
  if (c < f.sweep_ctas)
    sweep_cta<3>(f.sw, c, f.sweep_ctas, sg_smem_raw);
  else
    group_cta(f.grp, c - f.sweep_ctas);
}

// The batch's initial state in the [3][R][N] double-float layout: mn = ms =
// m0, ksum = 0.  m0 is [R][3][N] float (nullptr: the initial condition
// (ic0, ic1, ic2) of Eq. (initial) for every oscillator).  A non-finite m0
// value sets bad[0].
__global__ void sweep_state_init_kernel(const float* __restrict__ m0, long long R, long long N, double ic0,
                                        double ic1, double ic2, float2* __restrict__ st, int* __restrict__ bad) {
  const long long RN = R * N, total = 3 * RN;
  for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long i = idx / RN, rem = idx - i * RN, r = rem / N, k = rem - r * N;
    const double v = m0 ? static_cast<double>(m0[(r * 3 + i) * N + k]) : (i == 0 ? ic0 : (i == 1 ? ic1 : ic2));
    if (!isfinite(v)) atomicOr(bad, 1);
    const df d = df_from_double(v);
    st[idx] = make_float2(d.hi, d.lo);           // mn
    st[3 * RN + idx] = make_float2(d.hi, d.lo);  // ms
    st[6 * RN + idx] = make_float2(0.f, 0.f);    // ksum
  }
}

// X of stage 0 of the next RK4 step from m_n (mn, component x) of every pair.
__global__ void sweep_publish_kernel(const float2* mn, __nv_bfloat16* Xs, int N, int R, int Kpad, int bn) {
  const long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (idx >= static_cast<long long>(R) * N) return;
  const int r = static_cast<int>(idx / N), k = static_cast<int>(idx % N);
  const float x = mn[idx].x;
  const __nv_bfloat16 xh = __float2bfloat16_rn(x);
  const __nv_bfloat16 xl = __float2bfloat16_rn(x - __bfloat162float(xh));
  Xs[xt_offset(r, k, Kpad, bn)] = xh;
  Xs[xt_offset(r, Kpad + k, Kpad, bn)] = xl;
}

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

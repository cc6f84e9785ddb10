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
// Layouts (row-major, reservoir-major):
//   Wb   [Mpad][Kpad] bf16, zero padded (Mpad = 128-multiple >= N,
//        Kpad = 64-multiple >= N)
//   Xs   [Rpad][2 Kpad] bf16: row r = [X_hi(r, 0..Kpad) | X_lo(r, 0..Kpad)]
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
constexpr int kSwSlots = 4;        // pipeline depth
constexpr int kSwThreads = 128;    // 4 warps: TMEM lanes 0..127
constexpr int kSwSliceA = kSwM * kSwK * 2;        // 16 KB
constexpr int kSwSliceB = kSwN * kSwK * 2;        // 8 KB
constexpr int kSwSmem = kSwSlots * (kSwSliceA + kSwSliceB) + 128;

struct GemmArgs {
  const __nv_bfloat16* Wb;   // [Mpad][Kpad]
  const __nv_bfloat16* Xs;   // [Rpad][2 Kpad]
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

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int Npend>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(Npend) : "memory");
}

// Load K slice `kk` of the tile into a pipeline slot in the core-matrix
// layout (A: LBO = 2048, B: LBO = 1024, SBO = 128 for both).
__device__ __forceinline__ void sweep_load_slice(const GemmArgs& g, int m0, int n0, int kk,
                                                 unsigned char* sA, unsigned char* sB) {
  const int k2 = kk * kSwK;                       // column in the K-concatenated operand
  const int kw = k2 % g.Kpad;                     // column of W
  const size_t xw = static_cast<size_t>(2) * g.Kpad;
  for (int c = threadIdx.x; c < kSwM * (kSwK / 8); c += kSwThreads) {
    const int kc = c & 7, r = c >> 3;
    cp_async16(sA + kc * (kSwM / 8) * 128 + (r >> 3) * 128 + (r & 7) * 16,
               g.Wb + static_cast<size_t>(m0 + r) * g.Kpad + kw + kc * 8);
  }
  for (int c = threadIdx.x; c < kSwN * (kSwK / 8); c += kSwThreads) {
    const int kc = c & 7, r = c >> 3;
    cp_async16(sB + kc * (kSwN / 8) * 128 + (r >> 3) * 128 + (r & 7) * 16,
               g.Xs + static_cast<size_t>(n0 + r) * xw + k2 + kc * 8);
  }
}

// One 128 x 64 tile of D = [W | W] [X_hi ; X_lo] per CTA; writes D^T.
__global__ void __launch_bounds__(kSwThreads) sweep_gemm_kernel(const __grid_constant__ GemmArgs g) {
  extern __shared__ __align__(128) unsigned char sw_smem[];
  unsigned char* smem = sw_smem;
  __shared__ uint64_t mbar[kSwSlots + 1];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kSwM, n0 = blockIdx.y * kSwN;
  const int nk = 2 * g.Kpad / kSwK;
  auto slotA = [&](int s) { return smem + s * (kSwSliceA + kSwSliceB); };
  auto slotB = [&](int s) { return smem + s * (kSwSliceA + kSwSliceB) + kSwSliceA; };

  if (tid == 0) {
    for (int s = 0; s <= kSwSlots; ++s) mbar_init(&mbar[s], 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "n"(kSwN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // prologue: three slices in flight
  for (int s = 0; s < kSwSlots - 1 && s < nk; ++s) {
    sweep_load_slice(g, m0, n0, s, slotA(s), slotB(s));
    cp_async_commit();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = umma_idesc_bf16(kSwM, kSwN);
  bool ok = true;

  for (int kk = 0; kk < nk && ok; ++kk) {
    const int s = kk % kSwSlots;
    const int pending = min(kSwSlots - 2, nk - 1 - kk);  // later slices already issued
    if (pending >= 2) cp_async_wait<2>();
    else if (pending == 1) cp_async_wait<1>();
    else cp_async_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(slotA(s)), b0 = smem_u32(slotB(s));
#pragma unroll
      for (int j = 0; j < kSwK / 16; ++j) {
        const uint64_t ad = umma_desc(a0 + j * 2 * (kSwM / 8) * 128, (kSwM / 8) * 128, 128);
        const uint64_t bd = umma_desc(b0 + j * 2 * (kSwN / 8) * 128, (kSwN / 8) * 128, 128);
        const uint32_t acc = (kk > 0 || j > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&mbar[s]))
          : "memory");
    }
    // refill the slot of slice kk - 1 once its MMAs are done
    const int nxt = kk + kSwSlots - 1;
    if (nxt < nk) {
      const int t = nxt % kSwSlots;
      if (kk >= 1) {
        const uint32_t par = static_cast<uint32_t>(((kk - 1) / kSwSlots) & 1);
        ok = mbar_wait_bounded(&mbar[t], par, g.timeout_ns, nullptr);
      }
      if (ok) sweep_load_slice(g, m0, n0, nxt, slotA(t), slotB(t));
      cp_async_commit();
    }
    ok = __syncthreads_and(ok);
  }
  cp_async_wait<0>();
  if (tid == 0 && ok) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&mbar[kSwSlots]))
        : "memory");
  }
  if (ok) ok = mbar_wait_bounded(&mbar[kSwSlots], 0u, g.timeout_ns, nullptr);
  ok = __syncthreads_and(ok);
  if (!ok) {
    if (tid == 0) report_error(g.err, kErrTimeout, blockIdx.x, 0u, kSiteFull);
    // let every issued MMA finish before the tensor memory is released
    if (tid == 0) {
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&mbar[kSwSlots]))
          : "memory");
    }
    mbar_wait_bounded(&mbar[kSwSlots], 0u, g.timeout_ns, nullptr);
  }
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
  __nv_bfloat16* Xs;        // [Rpad][2 Kpad]
  float* states_out;        // [T][R][N] or nullptr
  const df* hs0_r;          // per reservoir H_s0
  const double* ain_g_r;    // per reservoir g A_in
  int N, R, Kpad, n_in, comp, st, last_sub;
  KArgs c;                  // shared constants (gdt, alpha, happl, hkp, lambda, p, acp, sixth)
};

// One (reservoir, oscillator) pair per thread: finish stage st with the
// coupling sum from the product, combine RK4, publish the next stage value
// into X (hi and lo BF16 parts) and sample at the end of an input sample.
__global__ void __launch_bounds__(256) sweep_epilogue_kernel(const __grid_constant__ EpiArgs e) {
  const long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (idx >= static_cast<long long>(e.R) * e.N) return;
  const int r = static_cast<int>(idx / e.N), k = static_cast<int>(idx % e.N);
  const size_t RN = static_cast<size_t>(e.R) * e.N;
  const int t = *e.t_dev;
  df mn[3], ms[3], ks[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float2 a = e.mn[i * RN + idx], b = e.ms[i * RN + idx], c = e.ksum[i * RN + idx];
    mn[i] = df{a.x, a.y};
    ms[i] = df{b.x, b.y};
    ks[i] = df{c.x, c.y};
  }
  double s = 0.0;
  for (int j = 0; j < e.n_in; ++j)
    s += static_cast<double>(e.w_in[static_cast<size_t>(k) * e.n_in + j]) *
         static_cast<double>(e.u[static_cast<size_t>(t) * e.n_in + j]);
  const df hx = df_add(df_mul_f(e.c.acp, e.Dt[idx]), df_from_double(e.ain_g_r[r] * s));
  KArgs kc = e.c;
  kc.hs0 = e.hs0_r[r];
  df A[3], B[3];
  llg_affine(kc, ms, A, B);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const df d = df_add(A[i], df_mul(hx, B[i]));
    if (e.st == 0) {
      ks[i] = d;
      ms[i] = df_add(mn[i], df_scale2(d, 0.5f));
    } else if (e.st == 1) {
      ks[i] = df_add(ks[i], df_scale2(d, 2.0f));
      ms[i] = df_add(mn[i], df_scale2(d, 0.5f));
    } else if (e.st == 2) {
      ks[i] = df_add(ks[i], df_scale2(d, 2.0f));
      ms[i] = df_add(mn[i], d);
    } else {
      ks[i] = df_add(ks[i], d);
      mn[i] = df_add(mn[i], df_mul(ks[i], e.c.sixth));
      ms[i] = mn[i];
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    e.mn[i * RN + idx] = make_float2(mn[i].hi, mn[i].lo);
    e.ms[i * RN + idx] = make_float2(ms[i].hi, ms[i].lo);
    e.ksum[i * RN + idx] = make_float2(ks[i].hi, ks[i].lo);
  }
  // next stage value, split into two BF16 terms
  const float x = ms[0].hi;
  const __nv_bfloat16 xh = __float2bfloat16_rn(x);
  const __nv_bfloat16 xl = __float2bfloat16_rn(x - __bfloat162float(xh));
  const size_t row = static_cast<size_t>(r) * 2 * e.Kpad;
  e.Xs[row + k] = xh;
  e.Xs[row + e.Kpad + k] = xl;
  if (e.st == 3 && e.last_sub && e.states_out)
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
  Xs[static_cast<size_t>(r) * 2 * Kpad + k] = xh;
  Xs[static_cast<size_t>(r) * 2 * Kpad + Kpad + k] = xl;
}

__global__ void sweep_advance_kernel(int* t_dev) { *t_dev += 1; }

// W (float, N x N row-major) -> zero-padded BF16 [Mpad][Kpad].
__global__ void sweep_pack_w_kernel(const float* W, __nv_bfloat16* Wb, int N, int Kpad) {
  const long long total = static_cast<long long>(N) * N;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int k = static_cast<int>(i / N), j = static_cast<int>(i % N);
    Wb[static_cast<size_t>(k) * Kpad + j] = __float2bfloat16_rn(W[i]);
  }
}

}  // namespace sto

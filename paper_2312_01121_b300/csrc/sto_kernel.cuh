// Device code of libsto: the persistent RK4 stepper for N coupled
// spin-torque oscillators (arXiv 2312.01121, Sec. 3.1 Eq. (gov), Sec. 3.2).
//
// One cooperative launch runs a whole sto_run call.  CTA c owns oscillators
// [r0, r0 + R) and the matching rows of W.  Per RK4 stage every CTA
//   1. gathers the stage's m^x of all N oscillators into shared memory
//      (tagged 8-byte words published by their owners, see below),
//   2. computes h_k = sum_i W[k,i] m^x_i for its rows while a producer warp
//      streams its W rows through a shared-memory ring with TMA bulk copies,
//   3. evaluates the LLG + spin-transfer torque of its oscillators in
//      double-float (about 48 significand bits on the FP32 pipes), combines
//      the RK4 stage and publishes the next stage's m^x.
// The W stream never waits for step 1: W is constant, so the producer runs
// ahead across stage boundaries and HBM stays busy while CTAs synchronise.
//
// Inter-CTA exchange: the m^x of oscillator k for stage tag g is the 64-bit
// word (tag << 32 | float bits) at xbuf[(g & 1) * N + k], written with one
// st.relaxed.gpu and read with ld.relaxed.gpu.  A reader accepts a word only
// when its tag equals g, so no grid barrier and no fence is needed; the two
// parity buffers are safe because a CTA can only publish tag g + 1 after it
// has read every tag-g word, which every owner wrote after reading all of
// its tag g - 1 words.
//
// Coupling precision (template parameter kW).  kWf32: W and the product in
// FP32 (the words above).  The two FP64 modes replicate the paper's own FP64
// benchmark (Sec. 3.3): the published value is the full double-float stage
// value, two tagged words per oscillator (low 32 bits of each word: hi and lo
// floats for kWdf, low and high halves of the FP64 value for kWf64) at
// xbuf[(g & 1) * 2N + 2k + {0, 1}]; a reader takes the pair once both words
// carry tag g.  kWdf stores W as an exact pair of floats per element (FP64
// rounded to 48 significand bits) and forms the products and row sums in
// double-float on the FP32 pipes; kWf64 stores W in FP64 and uses FP64 fused
// multiply-adds.  A W row panel is 512 bytes in every mode (128 FP32 or 64
// wide elements), so the producer and the ring are the same.
//
// Every wait is bounded by a_.timeout_ns of %globaltimer; on expiry the kernel
// records STO_ETIMEOUT in the error word; the consumer warps of a CTA agree
// on leaving through an OR-reducing barrier (bar.red.or), and the producer
// warp waits for its copies in flight before it leaves.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "dfloat.cuh"

namespace sto {

constexpr int kPanelCols = 128;                 // W columns per panel: 1 float4 per lane
constexpr int kConsWarps = 15;                  // warps that consume panels (16 warps in all: 128 registers each)
constexpr int kCons = kConsWarps * 32;          // consumer threads
constexpr int kThreads = kCons + 32;            // + one producer warp
constexpr int kMaxRowsPerWarp = 16;             // rows of a CTA <= 240
constexpr int kColSplitRows = 16;               // W on chip and at most this many rows: column split
constexpr int kRegUnits = 3;                    // register-resident W: 32-column units per consumer warp
constexpr int kRegWarps = kConsWarps - 1;       // consumer warps holding W (warp 0 owns the oscillators)
constexpr int kRegMaxN = 32 * kRegUnits * kRegWarps;  // 1344

// Error word layout (int32[4]): code, CTA, stage tag, site.
enum ErrSite { kSiteGather = 1, kSiteFull = 2, kSiteEmpty = 3, kSiteDrain = 4 };
constexpr int kErrTimeout = -4;  // == STO_ETIMEOUT

struct KArgs {
  const float* W;            // tiled row blocks (see host planner)
  const float* w_in;         // N x n_in
  const float* u;            // T x n_in
  double* state;             // 3 x N: m^x | m^y | m^z
  float* states_out;         // T x N or nullptr
  unsigned long long* xbuf;  // 2 x N tagged words
  int* err;                  // int32[4]
  int N, n_in, T, S, P, ns, resident, comp, inject_cta;
  int l2_keep;               // W small enough to stay in L2 between stages
  int zigzag;                // streamed W: panels in reverse order on odd stages
  int keep_panels;           // otherwise: leading panels of each row block kept in L2
  unsigned int tag_base;
  unsigned long long timeout_ns;
  // constants of Eq. (gov) as double-float pairs
  df gdt;        // -gamma' * dt
  df alpha, happl, hkp, hs0, lambda, px, py, pz, acp, sixth;
  double ain_g;  // g * A_in (input field formed once per sample in FP64)
  // forward recording for the adjoint (nullptr: off): per RK4 step n the
  // state before the step (rec_m[(n*3 + i)*N + k], df pairs) and the raw
  // coupling sums of its four stages (rec_h[(n*4 + s)*N + k])
  float2* rec_m;
  float* rec_h;
  // adjoint pass (kAdjoint kernels only)
  const float* dLds;         // T x N: dL/dstates of the segment
  double* lam;               // 3 x N: dL/dm at the segment end (in), at its start (out)
  double* g_win;             // N x n_in accumulated dL/dw_in
  double* g_acp;             // N partial sums of dL/dA_cp
  double* g_cur;             // N partial sums of dL/dI
  float dhs0_di_f;           // dH_s0/dI (the adjoint's dL/dI term)
  // explicit Runge-Kutta tableau (TableauProgram; classic RK4 otherwise)
  int rk_stages;             // stages per step (4 for classic RK4)
  df rk_a[4][4];             // a[i][j], j < i
  df rk_b[4];                // weights
};

enum ProgramKind { kProgForward = 0, kProgAdjoint = 1, kProgTableau = 2 };
enum CouplingMode { kWf32 = 0, kWdf = 1, kWf64 = 2 };

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// 1-D TMA bulk copy global -> shared, completion counted on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Barrier over the consumer warps that also ORs `flag` across them, so every
// consumer takes the same abort decision.
__device__ __forceinline__ bool consumer_sync_or(bool flag) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, 1, %2, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"(static_cast<uint32_t>(flag)), "n"(kCons)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ unsigned long long pack_x(float x, unsigned tag) {
  return (static_cast<unsigned long long>(tag) << 32) | __float_as_uint(x);
}

__device__ __noinline__ void report_error(int* err, int code, int cta, unsigned tag, int site) {
  if (atomicCAS(err, 0, code) == 0) {
    err[1] = cta;
    err[2] = static_cast<int>(tag);
    err[3] = site;
  }
}

// Wait for an mbarrier phase; false after timeout or when the CTA aborts.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned long long timeout_ns,
                                                  const volatile int* s_abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  for (uint32_t n = 1;; ++n) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((n & 15u) == 0) {
      if (s_abort && *s_abort) return false;
      if (gtimer() - t0 > timeout_ns) return false;
    }
  }
}

// Spin on one tagged word until it carries `tag`.  Returns the word, or 0
// (tag 0 is never used) after a timeout or when any CTA has recorded an error.
__device__ __noinline__ unsigned long long poll_word(const unsigned long long* p, unsigned tag,
                                                     int* err, unsigned long long timeout_ns) {
  const unsigned long long t0 = gtimer();
  for (uint32_t n = 1;; ++n) {
    const unsigned long long w = ld_relaxed_u64(p);
    if (static_cast<unsigned>(w >> 32) == tag) return w;
    if ((n & 31u) == 0) {
      if (ld_relaxed_i32(err) != 0) return 0ull;
      if (gtimer() - t0 > timeout_ns) {
        report_error(err, kErrTimeout, blockIdx.x, tag, kSiteGather);
        return 0ull;
      }
    }
  }
}

// Copy the stage's m^x (tag) of all N oscillators into xs; thread `g` of
// `ng` gatherers takes words g, g + ng, ...
__device__ __forceinline__ bool gather_x(const KArgs& a, float* xs, unsigned tag, int g, int ng) {
  const unsigned long long* xb = a.xbuf + static_cast<size_t>(tag & 1u) * a.N;
  for (int base = g; base < a.N; base += 4 * ng) {
    unsigned long long w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = base + q * ng;
      w[q] = (i < a.N) ? ld_relaxed_u64(xb + i) : 0ull;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = base + q * ng;
      if (i < a.N) {
        unsigned long long v = w[q];
        if (static_cast<unsigned>(v >> 32) != tag) {
          v = poll_word(xb + i, tag, a.err, a.timeout_ns);
          if (v == 0ull) return false;
        }
        xs[i] = __uint_as_float(static_cast<unsigned>(v));
      }
    }
  }
  return true;
}

// The FP64 modes: the pair of tagged words of every oscillator, stored as
// two 32-bit halves in xs2 (hi, lo floats or the FP64 value's bits).
__device__ __forceinline__ bool gather_x2(const KArgs& a, uint2* xs2, unsigned tag, int g, int ng) {
  const unsigned long long* xb = a.xbuf + static_cast<size_t>(tag & 1u) * 2 * a.N;
  for (int base = g; base < a.N; base += 2 * ng) {
    unsigned long long w[4];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = base + q * ng;
      w[2 * q] = (i < a.N) ? ld_relaxed_u64(xb + 2 * static_cast<size_t>(i)) : 0ull;
      w[2 * q + 1] = (i < a.N) ? ld_relaxed_u64(xb + 2 * static_cast<size_t>(i) + 1) : 0ull;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = base + q * ng;
      if (i < a.N) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (static_cast<unsigned>(w[2 * q + h] >> 32) != tag) {
            w[2 * q + h] = poll_word(xb + 2 * static_cast<size_t>(i) + h, tag, a.err, a.timeout_ns);
            if (w[2 * q + h] == 0ull) return false;
          }
        }
        xs2[i] = make_uint2(static_cast<unsigned>(w[2 * q]), static_cast<unsigned>(w[2 * q + 1]));
      }
    }
  }
  return true;
}

// Eq. (gov) is affine in the x-field that coupling and input add to b:
// with b = b0 + h e_x,
//   dt dm/dt = -gamma' dt [m x b + alpha m x (m x b)] = A(m) + h B(m),
//   A = -gamma' dt [m x b0 + alpha m x (m x b0)],
//   B = -gamma' dt [m x e_x + alpha m x (m x e_x)]
//     = -gamma' dt [(0, m_z, -m_y) + alpha (-(m_y^2 + m_z^2), m_x m_y, m_x m_z)],
// where b0 = H(m) + H_s(m) p x m holds the anisotropy, applied and
// spin-torque fields.  A and B depend only on the stage state, so they are
// formed while the CTA waits for the other oscillators' m^x; once the
// coupling field is known the increment costs three df multiply-adds.
__device__ __forceinline__ void llg_affine(const KArgs& a, const df m[3], df A[3], df B[3]) {
  df s, c[3];                                                                               // m.p, p x m
  df_p_terms(a.px, a.py, a.pz, m, &s, c);
  const df hs = df_mul(a.hs0, df_rcp(df_add_f(df_mul(a.lambda, s), 1.0f)));              // H_s(m)
  const df b[3] = {df_mul(hs, c[0]), df_mul(hs, c[1]),                                      // b0
                   df_fma(hs, c[2], df_fma(a.hkp, m[2], a.happl))};
  const df t[3] = {df_cross1(m[1], b[2], m[2], b[1]),                                       // m x b0
                   df_cross1(m[2], b[0], m[0], b[2]),
                   df_cross1(m[0], b[1], m[1], b[0])};
  const df u[3] = {df_cross1(m[1], t[2], m[2], t[1]),                                       // m x (m x b0)
                   df_cross1(m[2], t[0], m[0], t[2]),
                   df_cross1(m[0], t[1], m[1], t[0])};
  const df e[3] = {df{0.f, 0.f}, m[2], df_neg(m[1])};                                       // m x e_x
  const df v[3] = {df_neg(df_add(df_mul_raw(m[1], m[1]), df_mul_raw(m[2], m[2]))),         // m x (m x e_x)
                   df_mul(m[0], m[1]), df_mul(m[0], m[2])};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    A[i] = df_mul(a.gdt, df_fma(a.alpha, u[i], t[i]));
    B[i] = df_mul(a.gdt, df_fma(a.alpha, v[i], e[i]));
  }
}

// ------------------------------------------------------- owner programs
//
// The engine below exchanges one float per oscillator per stage and reduces
// W z for the published z.  What an oscillator's owner thread does with the
// reduced sum, and what it publishes next, is its "program".

// Publishes oscillator `node`'s stage value under tag `tg`: its FP32
// rounding (kWf32), or the full double-float value (kWdf as two floats,
// kWf64 as an FP64 value).
struct Publisher {
  unsigned long long* xbuf;
  float* xs;
  int N;
  int mode;      // CouplingMode of the launch
  bool single;   // one CTA: write shared memory directly
  bool enabled;  // false only for the CTA a test stalls on purpose
  __device__ __forceinline__ void operator()(int node, df v, unsigned tg) const {
    if (mode == kWf32) {
      if (single)
        xs[node] = v.hi;
      else if (enabled)
        st_relaxed_u64(xbuf + static_cast<size_t>(tg & 1u) * N + node, pack_x(v.hi, tg));
      return;
    }
    uint32_t w0, w1;
    if (mode == kWdf) {
      w0 = __float_as_uint(v.hi);
      w1 = __float_as_uint(v.lo);
    } else {
      const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(df_to_double(v)));
      w0 = static_cast<uint32_t>(b);
      w1 = static_cast<uint32_t>(b >> 32);
    }
    if (single) {
      reinterpret_cast<uint2*>(xs)[node] = make_uint2(w0, w1);
    } else if (enabled) {
      unsigned long long* p = xbuf + static_cast<size_t>(tg & 1u) * 2 * N + 2 * static_cast<size_t>(node);
      const unsigned long long t = static_cast<unsigned long long>(tg) << 32;
      st_relaxed_u64(p, t | w0);
      st_relaxed_u64(p + 1, t | w1);
    }
  }
};

// A_cp times the reduced coupling sum, as a double-float field.
__device__ __forceinline__ df acp_times(const KArgs& a, float h) { return df_mul_f(a.acp, h); }
__device__ __forceinline__ df acp_times(const KArgs& a, df h) { return df_mul(a.acp, h); }

// Forward RK4 (Sec. 3.2) of Eq. (gov): publishes m^x of every stage state.
struct ForwardProgram {
  df mn[3], ms[3], ksum[3], fa[3], fb[3], hin;
  int t, sub;

  __device__ __forceinline__ void load_hin(const KArgs& a, int node) {
    double s = 0.0;
    for (int jj = 0; jj < a.n_in; ++jj)
      s += static_cast<double>(a.w_in[static_cast<size_t>(node) * a.n_in + jj]) *
           static_cast<double>(a.u[static_cast<size_t>(t) * a.n_in + jj]);
    hin = df_from_double(a.ain_g * s);
  }

  __device__ __forceinline__ void init(const KArgs& a, int node, const Publisher& pub, unsigned tag) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      mn[i] = df_from_double(a.state[static_cast<size_t>(i) * a.N + node]);
      ms[i] = mn[i];
      ksum[i] = df{0.f, 0.f};
    }
    t = 0;
    sub = 0;
    load_hin(a, node);
    pub(node, ms[0], tag);
    llg_affine(a, ms, fa, fb);
  }

  // Finish stage g with the raw coupling sum hraw = (W x)_node (a float, or
  // a double-float in the FP64 modes), then publish the next stage's m^x
  // under next_tag.
  template <class HS>
  __device__ __forceinline__ void stage(const KArgs& a, int node, long long g, HS hraw,
                                        const Publisher& pub, unsigned next_tag) {
    const int st = static_cast<int>(g & 3);
    if constexpr (std::is_same<HS, float>::value) {  // recording (FP32 coupling only)
      if (a.rec_h) {
        const size_t n = static_cast<size_t>(g >> 2);
        a.rec_h[(n * 4 + st) * a.N + node] = hraw;
        if (st == 0) {
#pragma unroll
          for (int i = 0; i < 3; ++i) a.rec_m[(n * 3 + i) * a.N + node] = make_float2(mn[i].hi, mn[i].lo);
        }
      }
    }
    const df hx = df_add(acp_times(a, hraw), hin);
    df d[3];
    d[0] = df_fma(hx, fb[0], fa[0]);
    // the next stage's m^x goes out first (the other CTAs wait for it); the
    // same operations are repeated below for the stored state
    {
      df x;
      if (st == 0 || st == 1)
        x = df_add(mn[0], df_scale2(d[0], 0.5f));
      else if (st == 2)
        x = df_add(mn[0], d[0]);
      else
        x = df_fma(df_add(ksum[0], d[0]), a.sixth, mn[0]);
      pub(node, x, next_tag);
    }
#pragma unroll
    for (int i = 1; i < 3; ++i) d[i] = df_fma(hx, fb[i], fa[i]);
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
        mn[i] = df_fma(ksum[i], a.sixth, mn[i]);
        ms[i] = mn[i];
      }
    }
    if (st == 3 && ++sub == a.S) {  // end of input sample t: sample the state
      sub = 0;
      if (a.states_out) {
        const df v = a.comp == 0 ? mn[0] : (a.comp == 1 ? mn[1] : mn[2]);
        a.states_out[static_cast<size_t>(t) * a.N + node] = v.hi;
      }
      if (++t < a.T) load_hin(a, node);
    }
    llg_affine(a, ms, fa, fb);  // for the next stage, overlapping the exchange
  }

  __device__ __forceinline__ void finish(const KArgs& a, int node) {
#pragma unroll
    for (int i = 0; i < 3; ++i) a.state[static_cast<size_t>(i) * a.N + node] = df_to_double(mn[i]);
  }
};

// Any explicit Runge-Kutta method with up to four stages (Butcher tableau
// a strictly lower triangular, weights b): with increments d_i = dt f(y_i),
//   y_1 = m_n,  y_{i+1} = m_n + sum_{j<=i} a[i+1][j] d_j,  m_{n+1} = m_n + sum b_i d_i.
// The paper closes by noting that its approach carries over to any
// reservoir evolved by an explicit method; the engine is the same, only
// the per-oscillator combination differs.
struct TableauProgram {
  df mn[3], ms[3], d0[3], d1[3], d2[3], acc[3], fa[3], fb[3], hin;
  int t, sub, st;

  __device__ __forceinline__ void load_hin(const KArgs& a, int node) {
    double s = 0.0;
    for (int jj = 0; jj < a.n_in; ++jj)
      s += static_cast<double>(a.w_in[static_cast<size_t>(node) * a.n_in + jj]) *
           static_cast<double>(a.u[static_cast<size_t>(t) * a.n_in + jj]);
    hin = df_from_double(a.ain_g * s);
  }

  __device__ __forceinline__ void init(const KArgs& a, int node, const Publisher& pub, unsigned tag) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      mn[i] = df_from_double(a.state[static_cast<size_t>(i) * a.N + node]);
      ms[i] = mn[i];
    }
    t = sub = st = 0;
    load_hin(a, node);
    pub(node, ms[0], tag);
    llg_affine(a, ms, fa, fb);
  }

  template <class HS>
  __device__ __forceinline__ void stage(const KArgs& a, int node, long long /*g*/, HS hraw,
                                        const Publisher& pub, unsigned next_tag) {
    const df hx = df_add(acp_times(a, hraw), hin);
    df d[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      d[i] = df_add(fa[i], df_mul(hx, fb[i]));
      const df bd = df_mul(a.rk_b[st], d[i]);
      acc[i] = st == 0 ? bd : df_add(acc[i], bd);
    }
    if (st + 1 < a.rk_stages) {
      const int nx = st + 1;  // next stage: y = m_n + sum_{j<nx} a[nx][j] d_j
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (st == 0) d0[i] = d[i];
        else if (st == 1) d1[i] = d[i];
        else d2[i] = d[i];
        df y = df_add(mn[i], df_mul(a.rk_a[nx][0], d0[i]));
        if (nx > 1) y = df_add(y, df_mul(a.rk_a[nx][1], d1[i]));
        if (nx > 2) y = df_add(y, df_mul(a.rk_a[nx][2], d2[i]));
        ms[i] = y;
      }
      st = nx;
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        mn[i] = df_add(mn[i], acc[i]);
        ms[i] = mn[i];
      }
      st = 0;
      if (++sub == a.S) {  // end of input sample t: sample the state
        sub = 0;
        if (a.states_out) {
          const df v = a.comp == 0 ? mn[0] : (a.comp == 1 ? mn[1] : mn[2]);
          a.states_out[static_cast<size_t>(t) * a.N + node] = v.hi;
        }
        if (++t < a.T) load_hin(a, node);
      }
    }
    pub(node, ms[0], next_tag);
    llg_affine(a, ms, fa, fb);
  }

  __device__ __forceinline__ void finish(const KArgs& a, int node) {
#pragma unroll
    for (int i = 0; i < 3; ++i) a.state[static_cast<size_t>(i) * a.N + node] = df_to_double(mn[i]);
  }
};

// Discrete adjoint of the RK4 step, run backwards over a recorded segment.
// For step m' = m + dt/6 (k1 + 2 k2 + 2 k3 + k4), k_s = f(y_s), and the
// cotangent lam = dL/dm':
//   kb4 = dt/6 lam,            yb4 = J(y4)^T kb4
//   kb3 = dt/3 lam + dt yb4,   yb3 = J(y3)^T kb3
//   kb2 = dt/3 lam + dt/2 yb3, yb2 = J(y2)^T kb2
//   kb1 = dt/6 lam + dt/2 yb2, yb1 = J(y1)^T kb1,   lam <- lam + sum yb_s.
// J^T v splits into a local part and the coupling part A_cp W^T gbar, where
// gbar_k = bbar_x,k is what the engine exchanges and reduces (with W^T).
// With b the full field at m (derivation in the design notes):
//   bbar = gamma' (m x v) - alpha gamma' m x (m x v)            (so gbar is a
//          fixed linear form of v: cheap once v is known),
//   mbar = -gamma' [b x v + alpha ((m.b) v + (m.v) b - 2 (b.v) m)]
//          + H_K' bbar_z e_z + H_s (bbar x p) - (bbar.c) lambda H_s / (1 + lambda m.p) p.
// Only gbar sits on the critical path; mbar and the parameter terms are
// formed after publishing, while the exchange is in flight.  Double-float
// throughout: the A_cp gradient is a strongly cancelling sum over stages.
struct AdjointProgram {
  df lam[3], lacc[3], mbar[3];
  df y[4][3], hx[4];
  float hraw[4];
  df gacp, gcur, sumg, hin;
  long long n;        // current RK4 step (counting down)
  int nt, nsb;        // n = nt S + nsb: its input sample and substep (counted, not divided)
  int si;             // current stage index 0..3 (stage 1..4)

  __device__ __forceinline__ static void cross(const df a[3], const df b[3], df r[3]) {
    r[0] = df_cross1(a[1], b[2], a[2], b[1]);
    r[1] = df_cross1(a[2], b[0], a[0], b[2]);
    r[2] = df_cross1(a[0], b[1], a[1], b[0]);
  }
  __device__ __forceinline__ static df dot(const df a[3], const df b[3]) {
    return df_add(df_add(df_mul(a[0], b[0]), df_mul(a[1], b[1])), df_mul(a[2], b[2]));
  }

  __device__ __forceinline__ void setup_step(const KArgs& a, int node) {
    const int S = a.S;
    const int t = nt, sb = nsb;
    if (sb == S - 1) {  // the state after this step is sample t; its input field
      lam[a.comp] = df_add_f(lam[a.comp], a.dLds[static_cast<size_t>(t) * a.N + node]);
      double s = 0.0;
      for (int jj = 0; jj < a.n_in; ++jj)
        s += static_cast<double>(a.w_in[static_cast<size_t>(node) * a.n_in + jj]) *
             static_cast<double>(a.u[static_cast<size_t>(t) * a.n_in + jj]);
      hin = df_from_double(a.ain_g * s);
    }
    df m[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float2 v = a.rec_m[(static_cast<size_t>(n) * 3 + i) * a.N + node];
      m[i] = df{v.x, v.y};
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      hraw[q] = a.rec_h[(static_cast<size_t>(n) * 4 + q) * a.N + node];
      hx[q] = df_add(df_mul_f(a.acp, hraw[q]), hin);
    }
    // stage points, with dt dm/dt = A + h B exactly as the forward formed them
    df A[3], B[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) y[0][i] = m[i];
    llg_affine(a, y[0], A, B);
#pragma unroll
    for (int i = 0; i < 3; ++i) y[1][i] = df_add(m[i], df_scale2(df_add(A[i], df_mul(hx[0], B[i])), 0.5f));
    llg_affine(a, y[1], A, B);
#pragma unroll
    for (int i = 0; i < 3; ++i) y[2][i] = df_add(m[i], df_scale2(df_add(A[i], df_mul(hx[1], B[i])), 0.5f));
    llg_affine(a, y[2], A, B);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      y[3][i] = df_add(m[i], df_add(A[i], df_mul(hx[2], B[i])));
      lacc[i] = df{0.f, 0.f};
    }
  }

  // gbar = bbar_x at stage point q for cotangent v (in units of 1/dt: the
  // dt of kbar is applied here, gamma' dt = -gdt)
  __device__ __forceinline__ df gbar_of(const KArgs& a, int q, const df v[3]) const {
    const df* m = y[q];
    // (m x v)_x - alpha (m x (m x v))_x,  m x (m x v) = (m.v) m - |m|^2 v
    const df mxv_x = df_cross1(m[1], v[2], m[2], v[1]);
    const df mv = dot(m, v);
    const df mm = dot(m, m);
    const df mmv_x = df_sub(df_mul(mv, m[0]), df_mul(mm, v[0]));
    return df_mul(df_neg(a.gdt), df_sub(mxv_x, df_mul(a.alpha, mmv_x)));
  }

  // the rest of J(y_q)^T v: mbar (local part) and the parameter terms
  __device__ __forceinline__ void local_vjp(const KArgs& a, int q, const df v[3], df gb) {
    const df* m = y[q];
    const df p[3] = {a.px, a.py, a.pz};
    const df gpd = df_neg(a.gdt);  // gamma' dt (the dt of v)
    const df s = dot(m, p);
    const df rD = df_rcp(df_add_f(df_mul(a.lambda, s), 1.0f));
    const df hs = df_mul(a.hs0, rD);
    df c[3], b[3];
    cross(p, m, c);
    b[0] = df_add(hx[q], df_mul(hs, c[0]));
    b[1] = df_mul(hs, c[1]);
    b[2] = df_add(df_add(a.happl, df_mul(a.hkp, m[2])), df_mul(hs, c[2]));
    df mv[3], mmv[3], bb[3], bxv[3], bbxp[3];
    cross(m, v, mv);
    cross(m, mv, mmv);
#pragma unroll
    for (int i = 0; i < 3; ++i) bb[i] = df_mul(gpd, df_sub(mv[i], df_mul(a.alpha, mmv[i])));
    cross(b, v, bxv);
    const df mb = dot(m, b), mvd = dot(m, v), bv = dot(b, v);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const df inner = df_add(df_add(df_mul(mb, v[i]), df_mul(mvd, b[i])), df_scale2(df_mul(bv, m[i]), -2.0f));
      mbar[i] = df_neg(df_mul(gpd, df_add(bxv[i], df_mul(a.alpha, inner))));
    }
    mbar[2] = df_add(mbar[2], df_mul(a.hkp, bb[2]));
    cross(bb, p, bbxp);
    const df bc = dot(bb, c);
    const df lam_term = df_mul(df_mul(bc, a.lambda), df_mul(hs, rD));
#pragma unroll
    for (int i = 0; i < 3; ++i) mbar[i] = df_sub(df_add(mbar[i], df_mul(hs, bbxp[i])), df_mul(lam_term, p[i]));
    gacp = df_add(gacp, df_mul_f(gb, hraw[q]));
    gcur = df_add(gcur, df_mul(df_mul_f(bc, a.dhs0_di_f), rD));
    sumg = df_add(sumg, gb);
  }

  // kbar / dt for stage index q from lam and yb (the ybar of stage q + 1)
  __device__ __forceinline__ void kbar(int q, const df yb[3], df v[3]) const {
    // dt/6, dt/3, dt/3, dt/6 on lam; 0, dt, dt/2, dt/2 on yb; the common dt
    // is folded into gamma' dt in gbar_of / local_vjp
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const df l = (q == 3 || q == 0) ? df_mul(lam[i], df{0.16666667f, -4.967054e-09f})
                                      : df_mul(lam[i], df{0.33333334f, -9.934108e-09f});
      v[i] = q == 3 ? l : df_add(l, q == 2 ? yb[i] : df_scale2(yb[i], 0.5f));
    }
  }

  __device__ __forceinline__ void publish_stage(const KArgs& a, int node, int q, const df v[3],
                                                const Publisher& pub, unsigned tag) {
    const df gb = gbar_of(a, q, v);
    pub(node, gb, tag);
    local_vjp(a, q, v, gb);  // overlaps the exchange
  }

  __device__ __forceinline__ void init(const KArgs& a, int node, const Publisher& pub, unsigned tag) {
#pragma unroll
    for (int i = 0; i < 3; ++i) lam[i] = df_from_double(a.lam[static_cast<size_t>(i) * a.N + node]);
    gacp = gcur = sumg = hin = df{0.f, 0.f};
    n = static_cast<long long>(a.T) * a.S - 1;
    nt = a.T - 1;
    nsb = a.S - 1;
    setup_step(a, node);
    si = 3;
    const df zero[3] = {df{0.f, 0.f}, df{0.f, 0.f}, df{0.f, 0.f}};
    df v[3];
    kbar(3, zero, v);
    publish_stage(a, node, 3, v, pub, tag);
  }

  // q = (W^T gbar)_node for the current stage
  __device__ __forceinline__ void stage(const KArgs& a, int node, long long /*g*/, float q,
                                        const Publisher& pub, unsigned next_tag) {
    // ybar of this stage; the coupling part carries the dt folded into gbar
    df yb[3] = {df_add(mbar[0], df_mul_f(a.acp, q)), mbar[1], mbar[2]};
#pragma unroll
    for (int i = 0; i < 3; ++i) lacc[i] = df_add(lacc[i], yb[i]);
    if (si > 0) {
      --si;
      df v[3];
      kbar(si, yb, v);
      publish_stage(a, node, si, v, pub, next_tag);
      return;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) lam[i] = df_add(lam[i], lacc[i]);
    if (nsb == 0) {  // first RK4 step of its sample: flush dL/dw_in
      const int t = nt;
      const double sg = df_to_double(sumg);
      for (int jj = 0; jj < a.n_in; ++jj)
        a.g_win[static_cast<size_t>(node) * a.n_in + jj] +=
            a.ain_g * static_cast<double>(a.u[static_cast<size_t>(t) * a.n_in + jj]) * sg;
      sumg = df{0.f, 0.f};
    }
    if (--n >= 0) {
      if (nsb == 0) {
        nsb = a.S - 1;
        --nt;
      } else {
        --nsb;
      }
      setup_step(a, node);
      si = 3;
      const df zero[3] = {df{0.f, 0.f}, df{0.f, 0.f}, df{0.f, 0.f}};
      df v[3];
      kbar(3, zero, v);
      publish_stage(a, node, 3, v, pub, next_tag);
    }
  }

  __device__ __forceinline__ void finish(const KArgs& a, int node) {
#pragma unroll
    for (int i = 0; i < 3; ++i) a.lam[static_cast<size_t>(i) * a.N + node] = df_to_double(lam[i]);
    a.g_acp[node] += df_to_double(gacp);
    a.g_cur[node] += df_to_double(gcur);
  }
};

// Row block and offset of row k in the tiled layout of a plan with G CTAs.
__device__ __forceinline__ void tiled_row(int N, int G, int k, int* r0, int* R) {
  const int q = N / G, rem = N % G;
  if (k < rem * (q + 1)) {
    *r0 = (k / (q + 1)) * (q + 1);
    *R = q + 1;
  } else {
    *r0 = ((k - rem * (q + 1)) / q) * q + rem * (q + 1);
    *R = q;
  }
}

// ------------------------------------------------------------ the stepper

// Per-row partial sums of W x for the rows a consumer warp owns (rows warp,
// warp + 15, ...), one specialisation per coupling mode.  panel() adds one
// 512-byte panel row per owned row; store() reduces across the warp and
// writes the row sums to shared memory (float, float2 hi/lo, or double).
template <int kW, int RPW>
struct RowSums;

template <int RPW>
struct RowSums<kWf32, RPW> {
  float s[RPW];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int q = 0; q < RPW; ++q) s[q] = 0.f;
  }
  __device__ __forceinline__ void panel(const float* slot, const float* xs, int j, int warp, int lane, int R) {
    const float4* p4 = reinterpret_cast<const float4*>(slot);
    const float4 xv = reinterpret_cast<const float4*>(xs)[j * (kPanelCols / 4) + lane];
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      const int r = warp + q * kConsWarps;
      if (r < R) {
        const float4 w = p4[r * (kPanelCols / 4) + lane];
        float v = s[q];
        v = fmaf(w.x, xv.x, v);
        v = fmaf(w.y, xv.y, v);
        v = fmaf(w.z, xv.z, v);
        v = fmaf(w.w, xv.w, v);
        s[q] = v;
      }
    }
  }
  // The same panel with this thread's W values read from tensor memory
  // (kTmemW): row q's four at columns taddr + 4 q of its lane.  The FMAs
  // are those of panel(), in the same order.
  __device__ __forceinline__ void panel_tmem(uint32_t taddr, const float* xs, int j, int warp, int lane, int R) {
    const float4 xv = reinterpret_cast<const float4*>(xs)[j * (kPanelCols / 4) + lane];
    uint32_t w[RPW][4];
    __syncwarp();  // the loads below are warp-aligned
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      w[q][0] = w[q][1] = w[q][2] = w[q][3] = 0u;
      if (warp + q * kConsWarps < R)  // the same for every lane of the warp
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(w[q][0]), "=r"(w[q][1]), "=r"(w[q][2]), "=r"(w[q][3])
                     : "r"(taddr + 4u * q));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      if (warp + q * kConsWarps < R) {
        float v = s[q];
        v = fmaf(__uint_as_float(w[q][0]), xv.x, v);
        v = fmaf(__uint_as_float(w[q][1]), xv.y, v);
        v = fmaf(__uint_as_float(w[q][2]), xv.z, v);
        v = fmaf(__uint_as_float(w[q][3]), xv.w, v);
        s[q] = v;
      }
    }
  }
  __device__ __forceinline__ void store(float* hs, int warp, int lane, int R) {
    // butterfly sums of all rows at once (rows past R hold 0), so the
    // shuffle chains of different rows overlap
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int q = 0; q < RPW; ++q) s[q] += __shfl_xor_sync(0xffffffffu, s[q], off);
    }
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        const int r = warp + q * kConsWarps;
        if (r < R) hs[r] = s[q];
      }
    }
  }
};

// Double-float: per element (wh + wl)(xh + xl) = p + e with p = fl(wh xh)
// and e = its exact error + wh xl + wl xh (wl xl, below 2^-48 relative, is
// dropped); p enters the running sum through Knuth's TwoSum, e and the sum's
// rounding errors collect in the lo word.
template <int RPW>
struct RowSums<kWdf, RPW> {
  float hi[RPW], lo[RPW];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int q = 0; q < RPW; ++q) hi[q] = lo[q] = 0.f;
  }
  __device__ __forceinline__ static void acc(float& sh, float& sl, float wh, float wl, float xh, float xl) {
    const float p = __fmul_rn(wh, xh);
    float e = __fmaf_rn(wh, xh, -p);
    e = __fmaf_rn(wh, xl, e);
    e = __fmaf_rn(wl, xh, e);
    const df t = two_sum(sh, p);
    sh = t.hi;
    sl = __fadd_rn(sl, __fadd_rn(t.lo, e));
  }
  __device__ __forceinline__ void panel(const float* slot, const float* xs, int j, int warp, int lane, int R) {
    const float4* p4 = reinterpret_cast<const float4*>(slot);
    // (xh, xl) of elements 64 j + 2 lane and 64 j + 2 lane + 1
    const float4 xv = reinterpret_cast<const float4*>(xs)[j * (kPanelCols / 4) + lane];
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      const int r = warp + q * kConsWarps;
      if (r < R) {
        const float4 w = p4[r * (kPanelCols / 4) + lane];
        acc(hi[q], lo[q], w.x, w.y, xv.x, xv.y);
        acc(hi[q], lo[q], w.z, w.w, xv.z, xv.w);
      }
    }
  }
  __device__ __forceinline__ void store(float* hs, int warp, int lane, int R) {
    df v[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) v[q] = two_sum(hi[q], lo[q]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        const df o{__shfl_xor_sync(0xffffffffu, v[q].hi, off), __shfl_xor_sync(0xffffffffu, v[q].lo, off)};
        v[q] = df_add(v[q], o);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        const int r = warp + q * kConsWarps;
        if (r < R) reinterpret_cast<float2*>(hs)[r] = make_float2(v[q].hi, v[q].lo);
      }
    }
  }
};

template <int RPW>
struct RowSums<kWf64, RPW> {
  double s[RPW];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int q = 0; q < RPW; ++q) s[q] = 0.0;
  }
  __device__ __forceinline__ void panel(const float* slot, const float* xs, int j, int warp, int lane, int R) {
    const double2* p2 = reinterpret_cast<const double2*>(slot);
    const double2 xv = reinterpret_cast<const double2*>(xs)[j * (kPanelCols / 4) + lane];
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
      const int r = warp + q * kConsWarps;
      if (r < R) {
        const double2 w = p2[r * (kPanelCols / 4) + lane];
        s[q] = fma(w.y, xv.y, fma(w.x, xv.x, s[q]));
      }
    }
  }
  __device__ __forceinline__ void store(float* hs, int warp, int lane, int R) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int q = 0; q < RPW; ++q) s[q] += __shfl_xor_sync(0xffffffffu, s[q], off);
    }
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        const int r = warp + q * kConsWarps;
        if (r < R) reinterpret_cast<double*>(hs)[r] = s[q];
      }
    }
  }
};

// kRowMajorW = false: a.W is the tiled copy made by sto_create (one bulk copy
// per panel).  kRowMajorW = true: a.W is the caller's row-major N x N matrix
// (N a multiple of 4); each panel arrives as one bulk copy per row, issued by
// the 32 lanes of the producer warp.  Consumers are identical in both.
//
// stepper_engine is the whole launch as seen by CTA c of the G CTAs that
// run reservoir `a`: sto_persistent_kernel runs one reservoir on the whole
// grid, sto_group_kernel runs several, each on its own range of CTAs.
//
// kRegW (W on chip, at most 16 rows per CTA, N <= 1344, several CTAs): W is
// moved from shared memory into registers once.  Lane l of consumer warp w
// (1..14) holds the CTA's rows of W for columns 32 u + l, u = w - 1 + 14 k,
// k < 3, polls exactly those columns' x words into registers, multiplies and
// reduces its 16 row partials across the warp as in the column split.  One
// barrier per stage remains (before the owners add the warps' partials);
// warp 0 holds no columns, so its owners' work after publishing never
// delays a poll.
// W panels held in tensor memory (kTmemW: FP32 coupling, W streamed).  The
// engine has no use for the SM's 256 KB of tensor memory otherwise, so each
// consumer thread keeps its rows' four columns of a few streamed panels of
// its row block there for the whole launch.  Those panels are never copied
// again, and DRAM moves that many fewer bytes per stage.  They are taken
// from the middle of the streamed panels [keep_panels, P): the panels next
// to either end are the ones the alternating panel order already finds in
// L2 at a stage boundary.
// Tensor memory is 128 lanes x 512 columns of 32 bits; a warp reaches only
// the 32 lanes of its quarter (warp % 4), so the four warps of a quarter
// take 128 columns each (warp / 4).  A panel costs a thread 4 RPW columns.
constexpr int kTmemAllocCols = 512;
constexpr int kTmemWarpCols = 128;
template <int RPW>
__device__ __host__ __forceinline__ int tmem_panel_count(int P, int keep_panels) {
  const int fit = kTmemWarpCols / (4 * RPW), streamed = P - keep_panels;
  return fit < streamed ? fit : (streamed > 0 ? streamed : 0);
}

template <int RPW, bool kRowMajorW, int kProg, int kW, bool kRegW = false, bool kTmemW = false>
__device__ __forceinline__ void stepper_engine(const KArgs& a, const int c, const int G) {
  static_assert(!kTmemW || (kW == kWf32 && !kRowMajorW && !kRegW && kTmemWarpCols / (4 * RPW) >= 1),
                "tensor-memory panels: FP32 coupling, tiled W, streamed");
  extern __shared__ __align__(128) unsigned char smem[];
  const int q = a.N / G, rem = a.N % G;
  const int R = q + (c < rem ? 1 : 0);
  const int r0 = c * q + (c < rem ? c : rem);
  const int R_max = q + (rem > 0 ? 1 : 0);
  const size_t slot_floats = static_cast<size_t>(R_max) * kPanelCols;

  float* ring = reinterpret_cast<float*>(smem);
  float* xs = ring + slot_floats * a.ns;
  float* hs = xs + static_cast<size_t>(a.P) * kPanelCols;
  // row sums: one float per row, two in the FP64 modes (8-byte aligned:
  // every region before them is a multiple of 512 bytes); then, for the
  // column split (FP32, W on chip, <= 16 rows), 16 row partials per warp
  const bool colsplit = kW == kWf32 && a.resident && R_max <= kColSplitRows;
  float* part = hs + (kW == kWf32 ? 1 : 2) * ((R_max + 3) & ~3);
  uint64_t* full = reinterpret_cast<uint64_t*>(part + (colsplit ? kConsWarps * kColSplitRows : 0));
  uint64_t* empty = full + a.ns;
  volatile int* s_abort = reinterpret_cast<volatile int*>(empty + a.ns);
  // beside the abort flag, in the 16 bytes the plan keeps after the barriers
  [[maybe_unused]] uint32_t* s_tmem = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(empty + a.ns) + 4);
  // panels [t0, t0 + Pt) of the row block live in tensor memory (kTmemW);
  // the other Ps panels are streamed
  const int Pt = kTmemW ? tmem_panel_count<RPW>(a.P, a.keep_panels) : 0;
  const int Ps = a.P - Pt;
  const int t0 = kTmemW ? a.keep_panels + (a.P - a.keep_panels - Pt) / 2 : a.P;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < a.ns; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsWarps);
    }
    *s_abort = 0;
    fence_mbar_init();
  }
  for (int i = tid; i < a.P * kPanelCols; i += kThreads) xs[i] = 0.f;
  if constexpr (kRowMajorW) {
    // columns past N of the last panel are never written by a copy: keep
    // them finite (they meet x = 0)
    for (size_t i = tid; i < slot_floats * a.ns; i += kThreads) ring[i] = 0.f;
  }
  if constexpr (kTmemW) {
    if (warp == 0) {
      __syncwarp();  // thread 0 initialised the barriers alone
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                   "r"(static_cast<uint32_t>(kTmemAllocCols))
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();

  const float* Wc = a.W + static_cast<size_t>(r0) * a.P * kPanelCols;
  const uint32_t panel_bytes = static_cast<uint32_t>(R) * kPanelCols * 4u;
  // this thread's columns of tensor memory: its warp's lane quarter and
  // column block; panel t0 + t starts at column 4 RPW t of the block
  [[maybe_unused]] uint32_t tmem_w = 0;
  if constexpr (kTmemW) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tmem_w = *s_tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16) +
             static_cast<uint32_t>(kTmemWarpCols * (warp >> 2));
    if (warp < kConsWarps) {
      // fill once: this thread's four columns of each of its rows
      for (int t = 0; t < Pt; ++t) {
        const float4* src = reinterpret_cast<const float4*>(Wc + static_cast<size_t>(t0 + t) * R * kPanelCols);
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
          const int r = warp + q * kConsWarps;
          if (r < R) {  // the same for every lane of the warp
            const float4 v = src[r * (kPanelCols / 4) + lane];
            __syncwarp();
            asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(
                             tmem_w + static_cast<uint32_t>(4 * (RPW * t + q))),
                         "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(__float_as_uint(v.z)),
                         "r"(__float_as_uint(v.w))
                         : "memory");
          }
        }
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
  }

  // ------------------------------------------------------------ producer
  if constexpr (kRowMajorW) {
    if (warp == kConsWarps) {
      const uint64_t pol = (a.resident || a.l2_keep) ? policy_evict_last() : policy_evict_first();
      const long long total =
          a.resident ? a.P : static_cast<long long>(a.P) * a.rk_stages * a.S * a.T;
      const float* Wrows = a.W + static_cast<size_t>(r0) * a.N;
      long long it = 0;
      int slot = 0, j = 0;
      uint32_t lap = 0;
      bool ok = true;
      for (; it < total; ++it) {
        if (!a.resident && lap > 0) {
          bool freed = true;
          if (lane == 0)
            freed = mbar_wait_bounded(&empty[slot], (lap - 1u) & 1u, a.timeout_ns, s_abort);
          if (!__shfl_sync(0xffffffffu, freed, 0)) {
            ok = false;
            break;
          }
        }
        const int cols = min(kPanelCols, a.N - j * kPanelCols);
        const uint32_t row_bytes = static_cast<uint32_t>(cols) * 4u;
        if (lane == 0) mbar_arrive_expect_tx(&full[slot], row_bytes * static_cast<uint32_t>(R));
        __syncwarp();
        for (int r = lane; r < R; r += 32)
          bulk_g2s(ring + static_cast<size_t>(slot) * slot_floats + static_cast<size_t>(r) * kPanelCols,
                   Wrows + static_cast<size_t>(r) * a.N + static_cast<size_t>(j) * kPanelCols,
                   row_bytes, &full[slot], pol);
        if (++j == a.P) j = 0;
        if (++slot == a.ns) {
          slot = 0;
          ++lap;
        }
      }
      if (lane == 0) {
        if (!ok) {
          if (!*s_abort) report_error(a.err, kErrTimeout, c, a.tag_base, kSiteEmpty);
          *s_abort = 1;
        }
        const long long first = it > a.ns ? it - a.ns : 0;
        for (long long d = first; d < it; ++d) {
          const int s = static_cast<int>(d % a.ns);
          const uint32_t par = static_cast<uint32_t>((d / a.ns) & 1);
          if (!mbar_wait_bounded(&full[s], par, a.timeout_ns, nullptr)) {
            report_error(a.err, kErrTimeout, c, a.tag_base, kSiteDrain);
            break;
          }
        }
      }
      return;
    }
  }
  if (warp == kConsWarps) {
    if (lane == 0) {
      // W that fits in L2 stays there (evict_last); larger W keeps its
      // leading keep_panels panels of every row block in L2 and streams the
      // rest from HBM (evict_first), so that part is not re-read from DRAM
      const uint64_t keep = policy_evict_last(), stream = policy_evict_first();
      const bool all_keep = a.resident || a.l2_keep;
      // streamed panels only: [t0, t0 + Pt) are in tensor memory (kTmemW)
      const long long total =
          a.resident ? a.P : static_cast<long long>(Ps) * a.rk_stages * a.S * a.T;
      long long it = 0;
      int slot = 0, j = 0;
      uint32_t lap = 0;  // it / ns
      uint32_t odd = 0;  // (it / Ps) & 1: the stage walks its row block backwards
      bool ok = true;
      for (; it < total; ++it) {
        if (!a.resident && lap > 0) {
          if (!mbar_wait_bounded(&empty[slot], (lap - 1u) & 1u, a.timeout_ns, s_abort)) {
            ok = false;
            break;
          }
        }
        mbar_arrive_expect_tx(&full[slot], panel_bytes);
        // odd stages walk the row block backwards: the panels read last in
        // one stage, still in L2, are the first the next stage needs
        int jp = (a.zigzag && !a.resident && odd) ? Ps - 1 - j : j;
        if constexpr (kTmemW) jp += jp >= t0 ? Pt : 0;  // step over the held panels
        bulk_g2s(ring + static_cast<size_t>(slot) * slot_floats,
                 Wc + static_cast<size_t>(jp) * R * kPanelCols, panel_bytes, &full[slot],
                 (all_keep || jp < a.keep_panels) ? keep : stream);
        if (++j == Ps) {
          j = 0;
          odd ^= 1u;
        }
        if (++slot == a.ns) {
          slot = 0;
          ++lap;
        }
      }
      if (!ok) {
        if (!*s_abort) report_error(a.err, kErrTimeout, c, a.tag_base, kSiteEmpty);
        *s_abort = 1;
      }
      // Never leave with copies in flight: wait for the last ns issued.
      const long long first = it > a.ns ? it - a.ns : 0;
      for (long long d = first; d < it; ++d) {
        const int s = static_cast<int>(d % a.ns);
        const uint32_t par = static_cast<uint32_t>((d / a.ns) & 1);
        if (!mbar_wait_bounded(&full[s], par, a.timeout_ns, nullptr)) {
          report_error(a.err, kErrTimeout, c, a.tag_base, kSiteDrain);
          break;
        }
      }
    }
    return;
  }

  // ------------------------------------------------------------ consumers
  const int ctid = tid;
  const int node = r0 + ctid;
  const bool owner = ctid < R;
  const Publisher pub{a.xbuf, xs, a.N, kW, G == 1, c != a.inject_cta};
  // owners sit in the first warps; the others gather while owners work
  const int owner_warps = (R_max + 31) / 32;
  const int gather_first = owner_warps < kConsWarps ? owner_warps * 32 : 0;
  using Program = typename std::conditional<
      kProg == kProgAdjoint, AdjointProgram,
      typename std::conditional<kProg == kProgTableau, TableauProgram, ForwardProgram>::type>::type;
  Program prog;
  unsigned tag = a.tag_base;
  if (owner) prog.init(a, node, pub, tag);

  int cslot = 0;
  uint32_t cphase = 0;
  bool aborted = false;
  if (a.resident) {
    // The row block is loaded once: wait for every panel here, not per stage.
    bool landed = true;
    for (int j = 0; j < a.P && landed; ++j)
      landed = mbar_wait_bounded(&full[j], 0u, a.timeout_ns, s_abort);
    landed = __all_sync(0xffffffffu, landed);
    if (!landed && lane == 0) {
      if (!*s_abort) report_error(a.err, kErrTimeout, c, tag, kSiteFull);
      *s_abort = 1;
    }
    aborted = consumer_sync_or(!landed);
  }
  // register-resident W (kRegW): this lane's columns, all rows
  [[maybe_unused]] float wr[kRegUnits][kColSplitRows];
  [[maybe_unused]] const int n_units = (a.N + 31) / 32;
  if constexpr (kRegW) {
#pragma unroll
    for (int k = 0; k < kRegUnits; ++k) {
      const int u = warp - 1 + kRegWarps * k, col = 32 * u + lane;
      const bool ok = warp >= 1 && u < n_units && col < a.N;
      const float* pj = ring + static_cast<size_t>(col / kPanelCols) * slot_floats + (col % kPanelCols);
#pragma unroll
      for (int r = 0; r < kColSplitRows; ++r) wr[k][r] = (ok && r < R) ? pj[r * kPanelCols] : 0.f;
    }
  }
  const long long n_stages = static_cast<long long>(a.rk_stages) * a.S * a.T;
  for (long long g = 0; g < n_stages && !aborted; ++g) {
    if constexpr (kRegW) {
      bool fail = false;
      if (warp >= 1 && warp - 1 < n_units) {
        const unsigned long long* xb = a.xbuf + static_cast<size_t>(tag & 1u) * a.N;
        float xr[kRegUnits];
        unsigned long long wv[kRegUnits];
        bool pend[kRegUnits];
#pragma unroll
        for (int k = 0; k < kRegUnits; ++k) {
          const int u = warp - 1 + kRegWarps * k, col = 32 * u + lane;
          pend[k] = u < n_units && col < a.N;
          xr[k] = 0.f;
          wv[k] = pend[k] ? ld_relaxed_u64(xb + col) : 0ull;
        }
        bool waiting = false;
#pragma unroll
        for (int k = 0; k < kRegUnits; ++k) {
          if (pend[k] && static_cast<unsigned>(wv[k] >> 32) == tag) {
            xr[k] = __uint_as_float(static_cast<unsigned>(wv[k]));
            pend[k] = false;
          }
          waiting = waiting || pend[k];
        }
        if (waiting) {
          const unsigned long long t0 = gtimer();
          for (uint32_t n = 1; waiting; ++n) {
            waiting = false;
#pragma unroll
            for (int k = 0; k < kRegUnits; ++k) {
              if (pend[k]) {
                const unsigned long long v = ld_relaxed_u64(xb + 32 * (warp - 1 + kRegWarps * k) + lane);
                if (static_cast<unsigned>(v >> 32) == tag) {
                  xr[k] = __uint_as_float(static_cast<unsigned>(v));
                  pend[k] = false;
                }
              }
              waiting = waiting || pend[k];
            }
            if (waiting && (n & 31u) == 0) {
              if (ld_relaxed_i32(a.err) != 0) {
                fail = true;
                break;
              }
              if (gtimer() - t0 > a.timeout_ns) {
                report_error(a.err, kErrTimeout, c, tag, kSiteGather);
                fail = true;
                break;
              }
            }
          }
        }
        if (fail) *s_abort = 1;
        float p[kColSplitRows];
#pragma unroll
        for (int r = 0; r < kColSplitRows; ++r) {
          float v = 0.f;
#pragma unroll
          for (int k = 0; k < kRegUnits; ++k) v = fmaf(wr[k][r], xr[k], v);
          p[r] = v;
        }
#pragma unroll
        for (int half = kColSplitRows / 2, off = 16; half >= 1; half >>= 1, off >>= 1) {
          const bool up = (lane & off) != 0;
#pragma unroll
          for (int i = 0; i < half; ++i) {
            const float keep = up ? p[half + i] : p[i];
            const float send = up ? p[i] : p[half + i];
            p[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
          }
        }
        p[0] += __shfl_xor_sync(0xffffffffu, p[0], 1);
        if ((lane & 1) == 0) part[(warp - 1) * kColSplitRows + (lane >> 1)] = p[0];
      }
      if (consumer_sync_or(fail)) { aborted = true; break; }
      if (owner) {
        const int nw = n_units < kRegWarps ? n_units : kRegWarps;  // warps holding columns
        float pv[kRegWarps];
#pragma unroll
        for (int w = 0; w < kRegWarps; ++w) pv[w] = w < nw ? part[w * kColSplitRows + ctid] : 0.f;
        float hraw = pv[0];
#pragma unroll
        for (int w = 1; w < kRegWarps; ++w)
          if (w < nw) hraw += pv[w];
        prog.stage(a, node, g, hraw, pub, tag + 1u);
      }
      ++tag;
      continue;
    }
    // 1. the stage's published value of every oscillator
    bool fail = false;
    if (G > 1 && ctid >= gather_first) {
      bool got;
      if constexpr (kW == kWf32)
        got = gather_x(a, xs, tag, ctid - gather_first, kCons - gather_first);
      else
        got = gather_x2(a, reinterpret_cast<uint2*>(xs), tag, ctid - gather_first, kCons - gather_first);
      if (!got) {
        fail = true;
        *s_abort = 1;
      }
    }
    if (consumer_sync_or(fail)) { aborted = true; break; }
    // 2. h = W x over this CTA's rows, panel by panel
    RowSums<kW, RPW> sums;
    sums.zero();
    if (a.resident && colsplit) {
      if constexpr (kW == kWf32) {
        // Column split: warp w multiplies panels w, w + 15, ... for every
        // row (each x value is read from shared memory once per CTA, not once
        // per warp), then reduces its 16 row partials across the lanes by
        // recursive halving: after the steps at lane offsets 16, 8, 4, 2 and 1
        // lanes 2r and 2r + 1 hold the warp's sum for row r.  The owner of
        // row r adds the warps' partials in warp order.
        float p[kColSplitRows];
#pragma unroll
        for (int r = 0; r < kColSplitRows; ++r) p[r] = 0.f;
        const float4* x4 = reinterpret_cast<const float4*>(xs) + lane;
        const float4* w4 = reinterpret_cast<const float4*>(ring) + lane;
        const int pstride = static_cast<int>(slot_floats / 4);
        for (int j = warp; j < a.P; j += kConsWarps) {
          const float4 xv = x4[j * (kPanelCols / 4)];
          const float4* pj = w4 + j * pstride;
#pragma unroll
          for (int r = 0; r < kColSplitRows; ++r) {
            if (r < R) {
              const float4 w = pj[r * (kPanelCols / 4)];
              float v = p[r];
              v = fmaf(w.x, xv.x, v);
              v = fmaf(w.y, xv.y, v);
              v = fmaf(w.z, xv.z, v);
              v = fmaf(w.w, xv.w, v);
              p[r] = v;
            }
          }
        }
#pragma unroll
        for (int half = kColSplitRows / 2, off = 16; half >= 1; half >>= 1, off >>= 1) {
          const bool up = (lane & off) != 0;  // keep the upper half of the rows
#pragma unroll
          for (int i = 0; i < half; ++i) {
            const float keep = up ? p[half + i] : p[i];
            const float send = up ? p[i] : p[half + i];
            p[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
          }
        }
        p[0] += __shfl_xor_sync(0xffffffffu, p[0], 1);
        if ((lane & 1) == 0) part[warp * kColSplitRows + (lane >> 1)] = p[0];
      }
    } else if (a.resident) {
      if constexpr (kW == kWf32) {
        // all panels on chip: plain unrolled loop, loads run ahead of FMAs;
        // with few rows per warp, four partial sums per row shorten the
        // dependent FMA chain
        const float4* x4 = reinterpret_cast<const float4*>(xs) + lane;
        constexpr int kPart = RPW <= 2 ? 4 : 1;
        float part[RPW][kPart];
#pragma unroll
        for (int qq = 0; qq < RPW; ++qq)
#pragma unroll
          for (int k = 0; k < kPart; ++k) part[qq][k] = 0.f;
        const float4* w4 = reinterpret_cast<const float4*>(ring) + lane;
        const int pstride = static_cast<int>(slot_floats / 4);
#pragma unroll 4
        for (int j = 0; j < a.P; ++j) {
          const float4 xv = x4[j * (kPanelCols / 4)];
          const float4* pj = w4 + j * pstride;
#pragma unroll
          for (int qq = 0; qq < RPW; ++qq) {
            const int r = warp + qq * kConsWarps;
            if (r < R) {
              const float4 w = pj[r * (kPanelCols / 4)];
              if constexpr (kPart == 4) {
                part[qq][0] = fmaf(w.x, xv.x, part[qq][0]);
                part[qq][1] = fmaf(w.y, xv.y, part[qq][1]);
                part[qq][2] = fmaf(w.z, xv.z, part[qq][2]);
                part[qq][3] = fmaf(w.w, xv.w, part[qq][3]);
              } else {
                float v = part[qq][0];
                v = fmaf(w.x, xv.x, v);
                v = fmaf(w.y, xv.y, v);
                v = fmaf(w.z, xv.z, v);
                v = fmaf(w.w, xv.w, v);
                part[qq][0] = v;
              }
            }
          }
        }
#pragma unroll
        for (int qq = 0; qq < RPW; ++qq) {
          if constexpr (kPart == 4)
            sums.s[qq] = (part[qq][0] + part[qq][1]) + (part[qq][2] + part[qq][3]);
          else
            sums.s[qq] = part[qq][0];
        }
      } else {
#pragma unroll 2
        for (int j = 0; j < a.P; ++j) sums.panel(ring + static_cast<size_t>(j) * slot_floats, xs, j, warp, lane, R);
      }
    } else {
      for (int j = 0; j < a.P; ++j) {
        if constexpr (kTmemW) {
          // the order of the panels is the same; those past Ps come from tensor memory
          const int jp = (a.zigzag && (g & 1)) ? a.P - 1 - j : j;
          if (jp >= t0 && jp < t0 + Pt) {
            sums.panel_tmem(tmem_w + static_cast<uint32_t>(4 * RPW * (jp - t0)), xs, jp, warp, lane, R);
            continue;
          }
        }
        const int slot = cslot;
        // every lane waits; the vote keeps the warp's decision uniform
        const bool landed = mbar_wait_bounded(&full[slot], cphase, a.timeout_ns, s_abort);
        if (!__all_sync(0xffffffffu, landed)) {
          if (lane == 0) {
            if (!*s_abort) report_error(a.err, kErrTimeout, c, tag, kSiteFull);
            *s_abort = 1;
          }
          fail = true;
          break;
        }
        sums.panel(ring + static_cast<size_t>(slot) * slot_floats, xs, (a.zigzag && (g & 1)) ? a.P - 1 - j : j,
                   warp, lane, R);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
        if (++cslot == a.ns) {
          cslot = 0;
          cphase ^= 1u;
        }
      }
    }
    if (!colsplit) sums.store(hs, warp, lane, R);
    if (consumer_sync_or(fail)) { aborted = true; break; }

    // 3. the owner's program finishes the stage and publishes the next
    if (owner) {
      if constexpr (kW == kWf32) {
        float hraw;
        if (colsplit) {
          const int nw = a.P < kConsWarps ? a.P : kConsWarps;  // warps that had panels
          float pv[kConsWarps];
#pragma unroll
          for (int w = 0; w < kConsWarps; ++w) pv[w] = w < nw ? part[w * kColSplitRows + ctid] : 0.f;
          hraw = pv[0];
#pragma unroll
          for (int w = 1; w < kConsWarps; ++w)
            if (w < nw) hraw += pv[w];
        } else {
          hraw = hs[ctid];
        }
        prog.stage(a, node, g, hraw, pub, tag + 1u);
      } else if constexpr (kW == kWdf) {
        const float2 v = reinterpret_cast<const float2*>(hs)[ctid];
        prog.stage(a, node, g, df{v.x, v.y}, pub, tag + 1u);
      } else {
        prog.stage(a, node, g, df_from_double(reinterpret_cast<const double*>(hs)[ctid]), pub, tag + 1u);
      }
    }
    ++tag;
  }
  if (!aborted && owner) prog.finish(a, node);
  if constexpr (kTmemW) {
    // every consumer's tensor-memory loads are done before the columns go back
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncwarp();
    consumer_sync_or(false);
    if (warp == 0) {
      __syncwarp();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*s_tmem),
                   "r"(static_cast<uint32_t>(kTmemAllocCols))
                   : "memory");
    }
  }
}

template <int RPW, bool kRowMajorW, int kProg = kProgForward, int kW = kWf32, bool kRegW = false,
          bool kTmemW = false>
__global__ void __launch_bounds__(kThreads, 1) sto_persistent_kernel(const __grid_constant__ KArgs a) {
  stepper_engine<RPW, kRowMajorW, kProg, kW, kRegW, kTmemW>(a, static_cast<int>(blockIdx.x),
                                                            static_cast<int>(gridDim.x));
}

// Several reservoirs with their own W in one cooperative launch.  The grid
// is cut into n_lanes lanes of lane_width CTAs; lane l runs the reservoirs
// order[lane_begin[l] .. lane_begin[l+1]) one after another, each on all of
// the lane's CTAs (its record jobs[j] planned for that CTA count), so
// reservoirs on different lanes run at the same time.  A lane's CTAs leave a
// reservoir within one stage of each other and start the next together, so
// every wait of the engine stays as short as in a lone launch; no CTA ever
// waits for a CTA of another lane.
struct GroupArgs {
  const KArgs* jobs;      // per reservoir: the arguments of its stepper launch
  const int* lane_begin;  // n_lanes + 1 offsets into order
  const int* order;       // reservoir indices, lane by lane, in running order
  const int* rpw;         // per reservoir: rows per consumer warp of its plan (1, 2, 4 or 8)
  int n_lanes, lane_width;
};

// CTA `cta` of the group's n_lanes * lane_width CTAs.
__device__ __forceinline__ void group_cta(const GroupArgs& g, const int cta) {
  const int lane = cta / g.lane_width;
  if (lane >= g.n_lanes) return;
  const int c = cta - lane * g.lane_width;
  for (int i = g.lane_begin[lane]; i < g.lane_begin[lane + 1]; ++i) {
    const int j = g.order[i];
    const KArgs& a = g.jobs[j];
    switch (g.rpw[j]) {
      case 1: stepper_engine<1, false, kProgForward, kWf32>(a, c, g.lane_width); break;
      case 2: stepper_engine<2, false, kProgForward, kWf32>(a, c, g.lane_width); break;
      case 4: stepper_engine<4, false, kProgForward, kWf32>(a, c, g.lane_width); break;
      default: stepper_engine<8, false, kProgForward, kWf32>(a, c, g.lane_width); break;
    }
    // every warp has left the reservoir (the producer after draining its
    // copies) before the next one re-initialises shared memory
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads, 1) sto_group_kernel(const __grid_constant__ GroupArgs g) {
  group_cta(g, static_cast<int>(blockIdx.x));
}

// Re-tile W from the layout of a plan with G_old CTAs to one with G_new
// (same panel count P).  The destination must be zeroed beforehand.
__global__ void retile_w_kernel(const float* __restrict__ Wt_old, float* __restrict__ Wt_new, int N, int P,
                                int G_old, int G_new) {
  const long long total = static_cast<long long>(N) * P * kPanelCols;
  for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int k = static_cast<int>(idx / (static_cast<long long>(P) * kPanelCols));
    const int i = static_cast<int>(idx % (static_cast<long long>(P) * kPanelCols));  // padded column
    int r0, R, s0, S0;
    tiled_row(N, G_old, k, &r0, &R);
    tiled_row(N, G_new, k, &s0, &S0);
    const int j = i / kPanelCols, col = i % kPanelCols;
    Wt_new[static_cast<size_t>(s0) * P * kPanelCols + static_cast<size_t>(j) * S0 * kPanelCols +
           static_cast<size_t>(k - s0) * kPanelCols + col] =
        Wt_old[static_cast<size_t>(r0) * P * kPanelCols + static_cast<size_t>(j) * R * kPanelCols +
               static_cast<size_t>(k - r0) * kPanelCols + col];
  }
}

// Scatter a row-major N x N matrix into the tiled layout: CTA c's rows
// [r0, r0 + R) become P panels of R x kPanelCols floats, panel j holding
// columns [j*kPanelCols, (j+1)*kPanelCols) (zero beyond N).  The destination
// must be zeroed beforehand.
__global__ void tile_w_kernel(const float* __restrict__ W, float* __restrict__ Wt, int N, int G,
                              int P) {
  const int q = N / G, rem = N % G;
  const long long total = static_cast<long long>(N) * N;
  for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int k = static_cast<int>(idx / N), i = static_cast<int>(idx % N);
    int r0, R;
    if (k < rem * (q + 1)) {
      const int cc = k / (q + 1);
      r0 = cc * (q + 1);
      R = q + 1;
    } else {
      const int cc = rem + (k - rem * (q + 1)) / q;
      r0 = cc * q + rem;
      R = q;
    }
    const int r = k - r0, j = i / kPanelCols, col = i % kPanelCols;
    Wt[static_cast<size_t>(r0) * P * kPanelCols + static_cast<size_t>(j) * R * kPanelCols +
       static_cast<size_t>(r) * kPanelCols + col] = W[idx];
  }
}

// The FP64 modes: a row-major N x N FP64 matrix into the same tiled layout
// with 64 elements (512 bytes) per panel row; element (k, i) takes the two
// floats at row offset 2 (i mod 64): its hi/lo split (kWdf: hi = fl32(w),
// lo = fl32(w - hi), so hi + lo is w to 48 significand bits) or the FP64
// value itself (kWf64).  The destination must be zeroed beforehand.
__global__ void tile_w_wide_kernel(const double* __restrict__ W, float* __restrict__ Wt, int N, int G,
                                   int P, int mode) {
  constexpr int kCols = kPanelCols / 2;
  const int q = N / G, rem = N % G;
  const long long total = static_cast<long long>(N) * N;
  for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int k = static_cast<int>(idx / N), i = static_cast<int>(idx % N);
    int r0, R;
    if (k < rem * (q + 1)) {
      r0 = (k / (q + 1)) * (q + 1);
      R = q + 1;
    } else {
      r0 = ((k - rem * (q + 1)) / q) * q + rem * (q + 1);
      R = q;
    }
    const int r = k - r0, j = i / kCols, col = i % kCols;
    float* dst = Wt + static_cast<size_t>(r0) * P * kPanelCols + static_cast<size_t>(j) * R * kPanelCols +
                 static_cast<size_t>(r) * kPanelCols + 2 * col;
    const double w = W[idx];
    if (mode == kWdf) {
      const float hi = __double2float_rn(w);
      reinterpret_cast<float2*>(dst)[0] = make_float2(hi, __double2float_rn(w - static_cast<double>(hi)));
    } else {
      reinterpret_cast<double*>(dst)[0] = w;
    }
  }
}

// W^T in the tiled layout, read from W in the same layout.  The destination
// must be zeroed beforehand (its padding columns stay zero).
__global__ void transpose_tiled_kernel(const float* __restrict__ Wt, float* __restrict__ WTt, int N,
                                       int G, int P) {
  const long long total = static_cast<long long>(N) * N;
  for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int k = static_cast<int>(idx / N), i = static_cast<int>(idx % N);  // W[k][i]
    int r0, R;
    tiled_row(N, G, k, &r0, &R);
    const float v = Wt[static_cast<size_t>(r0) * P * kPanelCols +
                       static_cast<size_t>(i / kPanelCols) * R * kPanelCols +
                       static_cast<size_t>(k - r0) * kPanelCols + i % kPanelCols];
    int s0, S0;
    tiled_row(N, G, i, &s0, &S0);  // W^T[i][k]
    WTt[static_cast<size_t>(s0) * P * kPanelCols + static_cast<size_t>(k / kPanelCols) * S0 * kPanelCols +
        static_cast<size_t>(i - s0) * kPanelCols + k % kPanelCols] = v;
  }
}

// flag = 1 if any of the n floats is NaN or Inf.
__global__ void nonfinite_kernel(const float* __restrict__ p, long long n, int* flag) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    if (!isfinite(p[i])) *flag = 1;
  }
}

// flag = 1 if any of the n doubles is NaN or Inf.
__global__ void nonfinite_f64_kernel(const double* __restrict__ p, long long n, int* flag) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    if (!isfinite(p[i])) *flag = 1;
  }
}

}  // namespace sto

// libsto host side: the C ABI declared in include/sto.h.
//
// The handle owns, in device memory of the device current at creation:
//   W in the tiled layout of the plan (N x P*128 floats, zero padded; P
//   panels of 128 FP32 or, for the FP64 coupling modes, 64 eight-byte
//   elements), w_in (N x n_in floats), the FP64 state (3 x N doubles),
//   the tagged m^x exchange buffer (2 x N 64-bit words, twice that in the
//   FP64 modes), the error word, and staging buffers for calls made with
//   host pointers.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "sto.h"
#include "readout.cuh"
#include "shard.cuh"
#include "sto_kernel.cuh"
#include "stepper_plan.h"
#include "sweep.cuh"

namespace {

thread_local char g_errbuf[512];
thread_local cudaError_t g_last_cuda = cudaSuccess;

constexpr int kDefaultTimeoutMs = 2000;

int cuda_fail(cudaError_t e) {
  g_last_cuda = e;
  return STO_ECUDA;
}

// STO_OK, or STO_ECUDA with the error recorded.
int cuda_rc(cudaError_t e) { return e == cudaSuccess ? STO_OK : cuda_fail(e); }

#define STO_CUDA(call)                         \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void default_params(sto_params* p) {
  std::memset(p, 0, sizeof(*p));
  p->gamma = 1.764e7;
  p->alpha = 0.005;
  p->Ms = 1448.3;
  p->Hk = 18616.0;
  p->Happl = 200.0;
  p->eta = 0.537;
  p->lambda = 0.288;
  p->current = 2.5e-3;
  p->volume = M_PI * 60.0 * 60.0 * 2.0 * 1e-21;  // pi 60^2 2 nm^3 in cm^3
  p->e_charge = 1.60217733e-19;
  p->hbar = 1.05457266e-34;
  p->p[0] = 1.0;
  p->p[1] = 0.0;
  p->p[2] = 6.123234e-17;
  p->A_cp = 1.0;
  p->A_in = 1.0;
  p->input_gain = 1.0;
  p->dt = 1e-11;
  p->substeps = 100;
  p->n_in = 1;
  p->sample_component = 0;
}

int check_params(const sto_params* p) {
  if (!p) return STO_EINVAL;
  const double v[] = {p->gamma, p->alpha, p->Ms, p->Hk, p->Happl, p->eta, p->lambda,
                      p->current, p->volume, p->e_charge, p->hbar, p->p[0], p->p[1],
                      p->p[2], p->A_cp, p->A_in, p->input_gain, p->dt};
  for (double x : v)
    if (!std::isfinite(x)) return STO_EINVAL;
  if (p->Ms <= 0 || p->volume <= 0 || p->e_charge <= 0 || p->dt <= 0) return STO_EINVAL;
  if (p->substeps < 1 || p->n_in < 1 || p->n_in > 4096) return STO_EINVAL;
  if (p->sample_component < 0 || p->sample_component > 2 || p->reserved != 0) return STO_EINVAL;
  return STO_OK;
}

}  // namespace

struct sto_handle {
  int device = 0;
  int sm_count = 0;
  cudaStream_t stream = nullptr;
  int64_t N = 0;
  sto_params params{};
  Plan plan;
  int timeout_ms = kDefaultTimeoutMs;
  int l2_keep_mb = 0;
  int rk_stages = 4;           // explicit tableau; classic RK4 unless set
  bool rk_classic = true;
  double rk_a[16] = {};
  double rk_b[4] = {};
  int inject_cta = -1;
  int wmode = sto::kWf32;      // coupling precision (sto_create_f64: kWdf or kWf64)
  uint64_t stage_counter = 0;
  float* d_W = nullptr;
  float* d_win = nullptr;
  double* d_state = nullptr;
  unsigned long long* d_xbuf = nullptr;       // the exchange buffer in use, inside the pool
  unsigned long long* d_xbuf_pool = nullptr;  // xbuf_n candidate placements, xbuf_stride bytes apart
  int xbuf_n = 1;
  size_t xbuf_stride = 0;
  int xbuf_slot = 0;
  int xbuf_timed = 0;         // placements timed (0: not tuned)
  bool xbuf_pending = false;  // placements still to time, at the first run or adjoint
  int* d_err = nullptr;
  int* h_err = nullptr;  // pinned, 4 ints
  float* d_u = nullptr;
  size_t d_u_cap = 0;
  float* d_states = nullptr;
  size_t d_states_cap = 0;
  // adjoint working set (allocated on the first sto_adjoint)
  float* d_WT = nullptr;       // W^T in the tiled layout of the plan
  float* d_rec = nullptr;      // recording of one segment (rec_m then rec_h)
  size_t d_rec_cap = 0;        // floats
  double* d_ckpt = nullptr;    // checkpoints, (segments + 1) x 3N
  size_t d_ckpt_cap = 0;       // doubles
  double* d_lam = nullptr;     // 3N
  double* d_gacc = nullptr;    // g_acp (N) | g_cur (N) | g_win (N n_in)
  float* d_dl = nullptr;       // staged dL/dstates
  size_t d_dl_cap = 0;
  // the recomputation that overlaps the reverse pass (adjoint_overlap_ready)
  float* d_rec2 = nullptr;     // a second segment recording
  size_t d_rec2_cap = 0;
  double* d_state2 = nullptr;  // 3N: its state
  int* d_err2 = nullptr;       // its error word
  int* h_err2 = nullptr;       // pinned
  cudaStream_t s_aux = nullptr;
  cudaEvent_t ev_aux[5] = {};  // start, recorded[2], reversed[2]
};

namespace {

void free_handle(sto_handle* h) {
  if (!h) return;
  cudaFree(h->d_W);
  cudaFree(h->d_win);
  cudaFree(h->d_state);
  cudaFree(h->d_xbuf_pool);
  cudaFree(h->d_err);
  cudaFree(h->d_u);
  cudaFree(h->d_states);
  cudaFree(h->d_WT);
  cudaFree(h->d_rec);
  cudaFree(h->d_ckpt);
  cudaFree(h->d_lam);
  cudaFree(h->d_gacc);
  cudaFree(h->d_dl);
  cudaFree(h->d_rec2);
  cudaFree(h->d_state2);
  cudaFree(h->d_err2);
  if (h->h_err2) cudaFreeHost(h->h_err2);
  for (cudaEvent_t e : h->ev_aux)
    if (e) cudaEventDestroy(e);
  if (h->s_aux) cudaStreamDestroy(h->s_aux);
  if (h->h_err) cudaFreeHost(h->h_err);
  delete h;
}

// The device's opt-in shared-memory limit per block.  The kernels' dynamic
// shared-memory cap is set to it, not to one plan's size: handles of
// different N share the function, and a captured graph (sto_run_group) holds
// launches of several sizes, so a per-launch cap would leave the last one set
// below what an earlier launch in the graph asks for.
int smem_optin_limit() {
  static int cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (cached[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess)
      cached[dev] = v;
  }
  return cached[dev];
}

// Raise a kernel's dynamic shared-memory cap to what the device allows next
// to its static shared memory; the room left, or -1.
template <typename F>
int raise_dyn_smem_cap(F* func) {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, func) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  const int room = smem_optin_limit() - static_cast<int>(fa.sharedSizeBytes);
  if (room <= 0 || cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, room) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return room;
}

template <int RPW, bool kRowMajorW = false, int kProg = sto::kProgForward, int kW = sto::kWf32,
          bool kRegW = false, bool kTmemW = false>
cudaError_t launch_rpw(const Plan& pl, const sto::KArgs& a, cudaStream_t s) {
  const int room = raise_dyn_smem_cap(sto::sto_persistent_kernel<RPW, kRowMajorW, kProg, kW, kRegW, kTmemW>);
  if (room < static_cast<int>(pl.smem)) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(pl.G);
  cfg.blockDim = dim3(sto::kThreads);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs co-resident, or the launch fails
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, sto::sto_persistent_kernel<RPW, kRowMajorW, kProg, kW, kRegW, kTmemW>, a);
}

cudaError_t launch_stepper_rowmajor(const Plan& pl, const sto::KArgs& a, cudaStream_t s) {
  if (pl.rpw <= 1) return launch_rpw<1, true>(pl, a, s);
  if (pl.rpw <= 2) return launch_rpw<2, true>(pl, a, s);
  if (pl.rpw <= 4) return launch_rpw<4, true>(pl, a, s);
  if (pl.rpw <= 8) return launch_rpw<8, true>(pl, a, s);
  return launch_rpw<16, true>(pl, a, s);
}

cudaError_t launch_adjoint(const Plan& pl, const sto::KArgs& a, cudaStream_t s) {
  constexpr int A = sto::kProgAdjoint;
  // W^T is tiled like W, so a register-resident plan holds W^T the same way
  if (pl.regw) return pl.rpw <= 1 ? launch_rpw<1, false, A, sto::kWf32, true>(pl, a, s)
                                  : launch_rpw<2, false, A, sto::kWf32, true>(pl, a, s);
  if (pl.rpw <= 1) return launch_rpw<1, false, A>(pl, a, s);
  if (pl.rpw <= 2) return launch_rpw<2, false, A>(pl, a, s);
  if (pl.rpw <= 4) return launch_rpw<4, false, A>(pl, a, s);
  if (pl.rpw <= 8) return launch_rpw<8, false, A>(pl, a, s);
  return launch_rpw<16, false, A>(pl, a, s);
}

cudaError_t launch_tableau(const Plan& pl, const sto::KArgs& a, cudaStream_t s) {
  constexpr int B = sto::kProgTableau;
  if (pl.rpw <= 1) return launch_rpw<1, false, B>(pl, a, s);
  if (pl.rpw <= 2) return launch_rpw<2, false, B>(pl, a, s);
  if (pl.rpw <= 4) return launch_rpw<4, false, B>(pl, a, s);
  if (pl.rpw <= 8) return launch_rpw<8, false, B>(pl, a, s);
  return launch_rpw<16, false, B>(pl, a, s);
}

// Whether a forward FP32 launch holds panels in tensor memory: W streamed
// (not on chip, not all L2-resident), at least 3 rows per warp.
bool tmem_used(const Plan& pl, int l2_keep, int keep) {
  return pl.tmem && !pl.resident && !l2_keep && keep < pl.P && pl.rpw > 2;
}
int tmem_panels_of(const Plan& pl, int l2_keep, int keep) {
  if (!tmem_used(pl, l2_keep, keep)) return 0;
  if (pl.rpw <= 4) return sto::tmem_panel_count<4>(pl.P, keep);
  if (pl.rpw == 5) return sto::tmem_panel_count<5>(pl.P, keep);
  if (pl.rpw <= 8) return sto::tmem_panel_count<8>(pl.P, keep);
  return sto::tmem_panel_count<16>(pl.P, keep);
}

template <int kW>
cudaError_t launch_stepper_mode(const Plan& pl, const sto::KArgs& a, cudaStream_t s) {
  constexpr int F = sto::kProgForward;
  if constexpr (kW == sto::kWf32) {
    if (pl.regw) return pl.rpw <= 1 ? launch_rpw<1, false, F, kW, true>(pl, a, s)
                                    : launch_rpw<2, false, F, kW, true>(pl, a, s);
    // W streamed from HBM (not all of it L2-resident): the last panels of
    // each row block stay in tensor memory
    if (tmem_used(pl, a.l2_keep, a.keep_panels)) {
      if (pl.rpw <= 4) return launch_rpw<4, false, F, kW, false, true>(pl, a, s);
      if (pl.rpw == 5) return launch_rpw<5, false, F, kW, false, true>(pl, a, s);
      if (pl.rpw <= 8) return launch_rpw<8, false, F, kW, false, true>(pl, a, s);
      return launch_rpw<16, false, F, kW, false, true>(pl, a, s);
    }
  }
  if (pl.rpw <= 1) return launch_rpw<1, false, F, kW>(pl, a, s);
  if (pl.rpw <= 2) return launch_rpw<2, false, F, kW>(pl, a, s);
  if (pl.rpw <= 4) return launch_rpw<4, false, F, kW>(pl, a, s);
  // rows a warp does not own still cost issue slots (the FP64 FMA coupling is
  // bound by the FP64 pipe), so N = 10^4 on 148 CTAs (68 rows, 5 per warp)
  // gets its own width instead of 8
  if (pl.rpw == 5) return launch_rpw<5, false, F, kW>(pl, a, s);
  if (pl.rpw <= 8) return launch_rpw<8, false, F, kW>(pl, a, s);
  return launch_rpw<16, false, F, kW>(pl, a, s);
}

cudaError_t launch_stepper(const Plan& pl, const sto::KArgs& a, cudaStream_t s, int wmode = sto::kWf32) {
  if (wmode == sto::kWdf) return launch_stepper_mode<sto::kWdf>(pl, a, s);
  if (wmode == sto::kWf64) return launch_stepper_mode<sto::kWf64>(pl, a, s);
  return launch_stepper_mode<sto::kWf32>(pl, a, s);
}

// Device copy of n floats from a host or device pointer into dst.
int upload_floats(float* dst, const float* src, size_t n, cudaStream_t s) {
  STO_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(float),
                           is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  return STO_OK;
}

// n floats from host or device into a host vector.
int fetch_floats(std::vector<float>* out, const float* src, size_t n, cudaStream_t s) {
  out->resize(n);
  STO_CUDA(cudaMemcpyAsync(out->data(), src, n * sizeof(float), cudaMemcpyDefault, s));
  STO_CUDA(cudaStreamSynchronize(s));
  return STO_OK;
}

int any_nonfinite(const float* d_p, long long n, cudaStream_t s, int* d_flag, int* h_flag,
                  bool* result) {
  STO_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), s));
  if (n > 0) {
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    sto::nonfinite_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(d_p, n, d_flag);
    STO_CUDA(cudaGetLastError());
  }
  STO_CUDA(cudaMemcpyAsync(h_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  STO_CUDA(cudaStreamSynchronize(s));
  *result = (*h_flag != 0);
  return STO_OK;
}

int any_nonfinite_f64(const double* d_p, long long n, cudaStream_t s, int* d_flag, int* h_flag,
                      bool* result) {
  STO_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), s));
  if (n > 0) {
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    sto::nonfinite_f64_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(d_p, n, d_flag);
    STO_CUDA(cudaGetLastError());
  }
  STO_CUDA(cudaMemcpyAsync(h_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  STO_CUDA(cudaStreamSynchronize(s));
  *result = (*h_flag != 0);
  return STO_OK;
}

int set_state_host_f64(sto_handle* h, const double* m) {
  const size_t n = 3 * static_cast<size_t>(h->N);
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(m[i])) return STO_ENONFINITE;
  STO_CUDA(cudaMemcpyAsync(h->d_state, m, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  STO_CUDA(cudaStreamSynchronize(h->stream));
  return STO_OK;
}

int grow(float** buf, size_t* cap, size_t n) {
  if (*cap >= n) return STO_OK;
  cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  if (cudaMalloc(buf, n * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    *buf = nullptr;
    return STO_ENOMEM;
  }
  *cap = n;
  return STO_OK;
}

// Constants of Eq. (gov) in the form the stepper uses.
void set_constants(const sto_params& P, sto::KArgs* a) {
  using sto::df_split_host;
  const double gp = P.gamma / (1.0 + P.alpha * P.alpha);
  a->gdt = df_split_host(-gp * P.dt);
  a->alpha = df_split_host(P.alpha);
  a->happl = df_split_host(P.Happl);
  a->hkp = df_split_host(P.Hk - 4.0 * M_PI * P.Ms);
  a->hs0 = df_split_host(P.hbar * P.eta * P.current * 1.0e7 / (2.0 * P.e_charge * P.Ms * P.volume));
  a->lambda = df_split_host(P.lambda);
  a->px = df_split_host(P.p[0]);
  a->py = df_split_host(P.p[1]);
  a->pz = df_split_host(P.p[2]);
  a->acp = df_split_host(P.A_cp);
  a->sixth = df_split_host(1.0 / 6.0);
  a->ain_g = P.A_in * P.input_gain;
  a->dhs0_di_f = static_cast<float>(P.hbar * P.eta * 1.0e7 / (2.0 * P.e_charge * P.Ms * P.volume));
}

// ------------------------------------------------- allocation-free entry point
//
// Scratch of sto_run_noalloc: a file-scope device array, present on every
// device that loads the library until the process exits.  Layout: bytes
// [0, 16) error word, [16, 20) non-finite flag, [256, 256 + 16 N) the two
// parity buffers of tagged m^x words.  In host code the name is only a
// stand-in; the device address comes from cudaGetSymbolAddress.
constexpr int64_t kNoAllocMaxN = 16384;
constexpr size_t kNoAllocHeader = 256;
constexpr size_t kNoAllocBytes = kNoAllocHeader + 2 * static_cast<size_t>(kNoAllocMaxN) * 8;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_dev[kMaxDevices] = {};

// Device address of the scratch on device `dev` (current), looked up once.
int noalloc_scratch(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (dev < 0 || dev >= kMaxDevices) return STO_ENOTSUP;
  if (!g_noalloc_dev[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e);
    g_noalloc_dev[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_noalloc_dev[dev];
  return STO_OK;
}

int grow_d(double** buf, size_t* cap, size_t n) {
  if (*cap >= n) return STO_OK;
  cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  if (cudaMalloc(buf, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    *buf = nullptr;
    return STO_ENOMEM;
  }
  *cap = n;
  return STO_OK;
}

// Exchange buffer: two parity buffers of one tagged word per oscillator, or
// of two in the FP64 modes.
size_t xbuf_bytes(int64_t N, int wmode) {
  return 2 * static_cast<size_t>(N) * 8 * (wmode == sto::kWf32 ? 1 : 2);
}

// Candidate placements of the exchange buffer for plans with W on chip (see
// tune_xbuf), each on its own 4 KB-aligned block.
constexpr int kXbufCandidates = 8;
size_t xbuf_stride_bytes(int64_t N, int wmode) { return (xbuf_bytes(N, wmode) + 4095) / 4096 * 4096; }

// Kernel arguments shared by the forward and adjoint launches of a handle.
sto::KArgs base_args(sto_handle* h, const float* d_u, int64_t T) {
  const sto_params& P = h->params;
  sto::KArgs a{};
  a.W = h->d_W;
  a.w_in = h->d_win;
  a.u = d_u;
  a.state = h->d_state;
  a.xbuf = h->d_xbuf;
  a.err = h->d_err;
  a.N = static_cast<int>(h->N);
  a.n_in = P.n_in;
  a.T = static_cast<int>(T);
  a.S = P.substeps;
  a.P = h->plan.P;
  a.ns = h->plan.ns;
  a.resident = h->plan.resident;
  a.comp = P.sample_component;
  a.inject_cta = h->inject_cta;
  a.timeout_ns = static_cast<unsigned long long>(h->timeout_ms) * 1000000ULL;
  a.l2_keep = l2_keeps(h->N, w_elem_bytes(h->wmode));
  a.keep_panels = keep_panels(h->N, h->plan.P, h->l2_keep_mb, w_elem_bytes(h->wmode));
  a.zigzag = h->plan.resident ? 0 : 1;
  set_constants(P, &a);
  a.rk_stages = h->rk_stages;
  for (int i = 0; i < 4; ++i) {
    a.rk_b[i] = sto::df_split_host(i < h->rk_stages ? h->rk_b[i] : 0.0);
    for (int j = 0; j < 4; ++j)
      a.rk_a[i][j] = sto::df_split_host(i < h->rk_stages && j < i ? h->rk_a[i * 4 + j] : 0.0);
  }
  // tags [base, base + stages] are fresh: none was written before
  const uint64_t stages = static_cast<uint64_t>(h->rk_stages) * static_cast<uint64_t>(P.substeps) *
                          static_cast<uint64_t>(T);
  if (h->stage_counter + stages + 2 >= 0xfffffff0ULL) {
    cudaMemsetAsync(h->d_xbuf_pool, 0xff, h->xbuf_n * h->xbuf_stride, h->stream);
    h->stage_counter = 0;
  }
  const uint64_t base = h->stage_counter + 1;
  h->stage_counter = base + stages;
  a.tag_base = static_cast<unsigned>(base);
  return a;
}

// Enqueue one forward launch (optionally recording the trajectory) on
// stream s (the handle's own stream unless a group capture passes another).
int engine_launch_on(sto_handle* h, cudaStream_t s, const float* d_u, int64_t T, float* d_states,
                     float2* rec_m, float* rec_h) {
  sto::KArgs a = base_args(h, d_u, T);
  a.states_out = d_states;
  a.rec_m = rec_m;
  a.rec_h = rec_h;
  STO_CUDA(cudaMemsetAsync(h->d_err, 0, 16, s));
  if (h->rk_classic)
    STO_CUDA(launch_stepper(h->plan, a, s, h->wmode));
  else
    STO_CUDA(launch_tableau(h->plan, a, s));
  STO_CUDA(cudaMemcpyAsync(h->h_err, h->d_err, 16, cudaMemcpyDeviceToHost, s));
  return STO_OK;
}

int engine_launch(sto_handle* h, const float* d_u, int64_t T, float* d_states, float2* rec_m,
                  float* rec_h) {
  return engine_launch_on(h, h->stream, d_u, T, d_states, rec_m, rec_h);
}

// Enqueue one adjoint launch over a recorded segment of T samples.
int engine_launch_adjoint(sto_handle* h, const float* d_u, int64_t T, const float* d_dl,
                          const float2* rec_m, const float* rec_h) {
  sto::KArgs a = base_args(h, d_u, T);
  a.W = h->d_WT;
  a.rec_m = const_cast<float2*>(rec_m);
  a.rec_h = const_cast<float*>(rec_h);
  a.dLds = d_dl;
  a.lam = h->d_lam;
  a.g_acp = h->d_gacc;
  a.g_cur = h->d_gacc + h->N;
  a.g_win = h->d_gacc + 2 * h->N;
  a.inject_cta = -1;
  STO_CUDA(cudaMemsetAsync(h->d_err, 0, 16, h->stream));
  STO_CUDA(launch_adjoint(h->plan, a, h->stream));
  STO_CUDA(cudaMemcpyAsync(h->h_err, h->d_err, 16, cudaMemcpyDeviceToHost, h->stream));
  return STO_OK;
}

// Wait for the enqueued launch and turn its error word into a status.
int finish_launch(sto_handle* h) {
  STO_CUDA(cudaStreamSynchronize(h->stream));
  h->inject_cta = -1;
  if (h->h_err[0] != 0) return h->h_err[0] == sto::kErrTimeout ? STO_ETIMEOUT : STO_ECUDA;
  return STO_OK;
}

// Placement of the exchange buffer.  With W on chip a stage is one exchange
// round trip: every CTA polls the lines of the tagged words, one line per
// owning CTA, and how those lines fall on the L2 slices sets how long the
// slowest poll takes (measured at N = 10^3 on one device: 1.62-1.72 us per
// stage for some buffers, 1.9-2.4 us for others, the same plan and data).
// At the handle's first sto_run or sto_adjoint (a member run only through a
// group never pays for it), time a short launch (zero input, at most 50 RK4
// steps) in each candidate block of the pool, the best of three, keep the
// fastest, and restore the state.  Placement changes no arithmetic: the
// results are the same bits.  Placement only changes speed, so a trial that
// cannot run (no memory for the saved state, a trial launch that fails or
// times out on a busy device) leaves the first placement in use, untimed,
// and the caller's run goes ahead; only a failure to restore the state
// fails the call.
int tune_xbuf(sto_handle* h) {
  if (!h->xbuf_pending) return STO_OK;
  h->xbuf_pending = false;
  const size_t sbytes = 3 * static_cast<size_t>(h->N) * sizeof(double);
  double* saved = nullptr;
  float* u0 = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    cudaFree(saved);
    cudaFree(u0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaMalloc(reinterpret_cast<void**>(&saved), sbytes) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&u0), static_cast<size_t>(h->params.n_in) * sizeof(float)) !=
          cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return STO_OK;  // no trials: the first placement stays
  }
  cudaError_t e;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess ||
      (e = cudaMemsetAsync(u0, 0, static_cast<size_t>(h->params.n_in) * sizeof(float), h->stream)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(saved, h->d_state, sbytes, cudaMemcpyDeviceToDevice, h->stream)) != cudaSuccess) {
    cleanup();
    return cuda_fail(e);
  }
  const int substeps = h->params.substeps;
  h->params.substeps = substeps < 50 ? substeps : 50;
  const int inject = h->inject_cta;  // a stall injected for the next run is kept for that run
  h->inject_cta = -1;
  int rc = STO_OK, best = 0;
  float best_ms = 0.f;
  for (int c = 0; c < h->xbuf_n && rc == STO_OK; ++c) {
    h->d_xbuf = h->d_xbuf_pool + c * (h->xbuf_stride / sizeof(unsigned long long));
    float ms_c = 0.f;
    for (int rep = 0; rep < 3 && rc == STO_OK; ++rep) {
      if ((e = cudaEventRecord(e0, h->stream)) != cudaSuccess) {
        rc = cuda_fail(e);
        break;
      }
      rc = engine_launch(h, u0, 1, nullptr, nullptr, nullptr);
      if (rc) break;
      if ((e = cudaEventRecord(e1, h->stream)) != cudaSuccess) {
        rc = cuda_fail(e);
        break;
      }
      rc = finish_launch(h);
      float ms = 0.f;
      if (!rc && (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) rc = cuda_fail(e);
      if (!rc && (rep == 0 || ms < ms_c)) ms_c = ms;
    }
    if (!rc && (c == 0 || ms_c < best_ms)) {
      best_ms = ms_c;
      best = c;
    }
  }
  h->params.substeps = substeps;
  h->inject_cta = inject;
  if (rc == STO_OK) {
    h->xbuf_slot = best;
    h->xbuf_timed = h->xbuf_n;
  } else {
    // a failed trial decides nothing: first placement, not timed
    best = 0;
    h->xbuf_slot = 0;
    h->xbuf_timed = 0;
    cudaGetLastError();
  }
  h->d_xbuf = h->d_xbuf_pool + best * (h->xbuf_stride / sizeof(unsigned long long));
  // back to the state before the trial launches
  rc = STO_OK;
  if ((e = cudaMemcpyAsync(h->d_state, saved, sbytes, cudaMemcpyDeviceToDevice, h->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(h->stream)) != cudaSuccess)
    rc = cuda_fail(e);
  cleanup();
  return rc;
}

// W^T in the tiled layout of the plan, derived from the tiled W.
int ensure_transpose(sto_handle* h) {
  if (h->d_WT) return STO_OK;
  const size_t elems = static_cast<size_t>(h->N) * h->plan.P * sto::kPanelCols;
  if (cudaMalloc(&h->d_WT, elems * 4) != cudaSuccess) {
    cudaGetLastError();
    h->d_WT = nullptr;
    return STO_ENOMEM;
  }
  STO_CUDA(cudaMemsetAsync(h->d_WT, 0, elems * 4, h->stream));
  long long blocks = (h->N * h->N + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  sto::transpose_tiled_kernel<<<static_cast<unsigned>(blocks), 256, 0, h->stream>>>(
      h->d_W, h->d_WT, static_cast<int>(h->N), h->plan.G, h->plan.P);
  STO_CUDA(cudaGetLastError());
  STO_CUDA(cudaStreamSynchronize(h->stream));
  return STO_OK;
}

// sto_create_ex and sto_create_f64: W is N x N float (wmode kWf32) or double
// (the FP64 modes), m0 3 x N float or double (m0_f64) or NULL.
int create_impl(int64_t N, const sto_params* params, const void* W, int wmode, const float* w_in,
                const void* m0, bool m0_f64, void* stream, const sto_config* cfg, sto_handle** out) {
  if (!out) return STO_EINVAL;
  *out = nullptr;
  if (N < 1 || !W || !w_in) return STO_EINVAL;
  int rc = check_params(params);
  if (rc) return rc;
  if (cfg) {
    if (cfg->grid < 0 || cfg->timeout_ms < 0 || cfg->l2_keep_mb < -1 || cfg->tmem_w < -1 || cfg->tmem_w > 0)
      return STO_EINVAL;
    for (int i = 0; i < 4; ++i)
      if (cfg->reserved[i] != 0) return STO_EINVAL;
  }
  if (N > (1LL << 20)) return STO_ENOTSUP;

  sto_handle* h = new (std::nothrow) sto_handle();
  if (!h) return STO_ENOMEM;
  h->N = N;
  h->wmode = wmode;
  h->params = *params;
  h->stream = static_cast<cudaStream_t>(stream);
  if (cfg && cfg->timeout_ms > 0) h->timeout_ms = cfg->timeout_ms;
  if (cfg) h->l2_keep_mb = cfg->l2_keep_mb;

  auto fail = [&](int code) {
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_handle(h);
    return code;
  };
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) return fail(cuda_fail(e));
  int smem_optin = 0;
  if ((e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device)) !=
          cudaSuccess ||
      (e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                  h->device)) != cudaSuccess)
    return fail(cuda_fail(e));
  rc = make_plan(N, cfg ? cfg->grid : 0, h->sm_count, static_cast<size_t>(smem_optin), &h->plan, wmode);
  if (rc) return fail(rc);
  // streamed FP32 W keeps its last panels in tensor memory (launch_stepper_mode)
  h->plan.tmem = (wmode == sto::kWf32 && !h->plan.resident && !(cfg && cfg->tmem_w < 0)) ? 1 : 0;

  const int n_in = params->n_in;
  const size_t wt_elems = static_cast<size_t>(N) * h->plan.P * sto::kPanelCols;
  h->xbuf_n = (h->plan.resident && h->plan.G > 1) ? kXbufCandidates : 1;
  h->xbuf_stride = xbuf_stride_bytes(N, wmode);
  auto alloc = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return false;
    }
    return true;
  };
  if (!alloc(reinterpret_cast<void**>(&h->d_W), wt_elems * 4) ||
      !alloc(reinterpret_cast<void**>(&h->d_win), static_cast<size_t>(N) * n_in * 4) ||
      !alloc(reinterpret_cast<void**>(&h->d_state), 3 * static_cast<size_t>(N) * 8) ||
      !alloc(reinterpret_cast<void**>(&h->d_xbuf_pool), h->xbuf_n * h->xbuf_stride) ||
      !alloc(reinterpret_cast<void**>(&h->d_err), 16))
    return fail(STO_ENOMEM);
  if (cudaMallocHost(reinterpret_cast<void**>(&h->h_err), 16) != cudaSuccess) {
    cudaGetLastError();
    h->h_err = nullptr;
    return fail(STO_ENOMEM);
  }
  cudaStream_t s = h->stream;

  // W: stage row-major on the device, check, tile.
  const size_t ebytes = static_cast<size_t>(w_elem_bytes(wmode));
  const void* d_src = W;
  void* d_tmp = nullptr;
  if (!is_device_ptr(W)) {
    if (!alloc(&d_tmp, static_cast<size_t>(N) * N * ebytes)) return fail(STO_ENOMEM);
    e = cudaMemcpyAsync(d_tmp, W, static_cast<size_t>(N) * N * ebytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { cudaFree(d_tmp); return fail(cuda_fail(e)); }
    d_src = d_tmp;
  }
  bool bad = false;
  if (wmode == sto::kWf32)
    rc = any_nonfinite(static_cast<const float*>(d_src), N * N, s, h->d_err, h->h_err, &bad);
  else
    rc = any_nonfinite_f64(static_cast<const double*>(d_src), N * N, s, h->d_err, h->h_err, &bad);
  if (!rc && bad) rc = STO_ENONFINITE;
  if (!rc) {
    e = cudaMemsetAsync(h->d_W, 0, wt_elems * 4, s);
    if (e == cudaSuccess) {
      long long blocks = (N * N + 255) / 256;
      if (blocks > 8192) blocks = 8192;
      if (wmode == sto::kWf32)
        sto::tile_w_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(
            static_cast<const float*>(d_src), h->d_W, static_cast<int>(N), h->plan.G, h->plan.P);
      else
        sto::tile_w_wide_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(
            static_cast<const double*>(d_src), h->d_W, static_cast<int>(N), h->plan.G, h->plan.P, wmode);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e);
  }
  if (d_tmp) cudaFree(d_tmp);
  if (rc) return fail(rc);

  // w_in
  rc = upload_floats(h->d_win, w_in, static_cast<size_t>(N) * n_in, s);
  if (!rc) {
    rc = any_nonfinite(h->d_win, N * n_in, s, h->d_err, h->h_err, &bad);
    if (!rc && bad) rc = STO_ENONFINITE;
  }
  if (rc) return fail(rc);

  // exchange buffer: tag 0xffffffff is never used by a launch
  h->d_xbuf = h->d_xbuf_pool;
  e = cudaMemsetAsync(h->d_xbuf_pool, 0xff, h->xbuf_n * h->xbuf_stride, s);
  if (e != cudaSuccess) return fail(cuda_fail(e));

  // state
  std::vector<double> m(3 * static_cast<size_t>(N));
  if (m0 && m0_f64) {
    e = cudaMemcpyAsync(m.data(), m0, m.size() * sizeof(double), cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(cuda_fail(e));
  } else if (m0) {
    std::vector<float> mf;
    rc = fetch_floats(&mf, static_cast<const float*>(m0), m.size(), s);
    if (rc) return fail(rc);
    for (size_t i = 0; i < m.size(); ++i) m[i] = mf[i];
  } else {
    const double phi0 = 2.0 * M_PI / 360.0;  // Eq. (initial)
    for (int64_t k = 0; k < N; ++k) {
      m[k] = std::sin(phi0) * std::cos(phi0);
      m[N + k] = std::sin(phi0) * std::sin(phi0);
      m[2 * N + k] = std::cos(phi0);
    }
  }
  rc = set_state_host_f64(h, m.data());
  if (rc) return fail(rc);
  h->xbuf_pending = h->xbuf_n > 1;
  *out = h;
  return STO_OK;
}

// Re-plan a handle for G CTAs (a lane of a group launch): new plan, W
// re-tiled on the device.  A lane of a warp sums the same columns of a row
// in the same order under any plan, except that a plan holding W on chip
// with at most two rows per warp keeps four partial sums per row: the new
// plan can change the last bits of the coupling sums.
// Re-plan for G CTAs with at most smem_optin - reserve bytes of dynamic
// shared memory per CTA (reserve: static shared memory of the kernel that
// will run the plan beside its own).
int replan_handle(sto_handle* h, int G, size_t reserve = 0) {
  int smem_optin = 0;
  STO_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
  const size_t smem_max = static_cast<size_t>(smem_optin) - reserve;
  if (h->plan.G == G && h->plan.smem <= smem_max) return STO_OK;
  Plan p;
  int rc = make_plan(h->N, G, h->sm_count, smem_max, &p, h->wmode);
  if (rc) return rc;
  if (p.P != h->plan.P) return STO_ENOTSUP;
  const size_t elems = static_cast<size_t>(h->N) * p.P * sto::kPanelCols;
  float* d_new = nullptr;
  if (cudaMalloc(&d_new, elems * 4) != cudaSuccess) {
    cudaGetLastError();
    return STO_ENOMEM;
  }
  cudaError_t e = cudaMemsetAsync(d_new, 0, elems * 4, h->stream);
  if (e == cudaSuccess) {
    long long blocks = static_cast<long long>((elems + 255) / 256);
    if (blocks > 8192) blocks = 8192;
    sto::retile_w_kernel<<<static_cast<unsigned>(blocks), 256, 0, h->stream>>>(
        h->d_W, d_new, static_cast<int>(h->N), p.P, h->plan.G, G);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    cudaFree(d_new);
    return cuda_fail(e);
  }
  cudaFree(h->d_W);
  h->d_W = d_new;
  h->plan = p;
  cudaFree(h->d_WT);  // the adjoint's W^T follows the plan; rebuilt on demand
  h->d_WT = nullptr;
  return STO_OK;
}

}  // namespace

// A fixed set of reservoirs run by one cooperative launch per call (see
// sto_group_kernel): lanes of CTAs, each running its reservoirs in turn.
struct sto_group {
  std::vector<sto_handle*> hs;
  int n = 0, lanes = 1, width = 1;
  size_t smem = 0;
  std::vector<int> lane_begin, order, rpw;
  sto::KArgs* d_jobs = nullptr;
  sto::KArgs* h_jobs = nullptr;  // pinned staging of the job records
  int* d_tab = nullptr;          // lane_begin | order | rpw
  int* d_errs = nullptr;         // 4 ints per reservoir
  int* h_errs = nullptr;         // pinned
  float* d_u = nullptr;
  size_t d_u_cap = 0;
};

namespace {
void free_group(sto_group* g) {
  if (!g) return;
  cudaFree(g->d_jobs);
  cudaFree(g->d_tab);
  cudaFree(g->d_errs);
  cudaFree(g->d_u);
  if (g->h_jobs) cudaFreeHost(g->h_jobs);
  if (g->h_errs) cudaFreeHost(g->h_errs);
  delete g;
}
}  // namespace

extern "C" {

void sto_default_params(sto_params* out) {
  if (out) default_params(out);
}

int sto_abi_version(void) { return STO_ABI_VERSION; }

const char* sto_strerror(int code) {
  const char* base = "unknown status";
  switch (code) {
    case STO_OK: base = "ok"; break;
    case STO_EINVAL: base = "invalid argument"; break;
    case STO_ENOMEM: base = "out of memory"; break;
    case STO_ECUDA: base = "CUDA error"; break;
    case STO_ETIMEOUT: base = "device wait timed out"; break;
    case STO_ENONFINITE: base = "non-finite input"; break;
    case STO_ENOTSUP: base = "size or option not supported by the library"; break;
    case STO_ETOOBIG: base = "size exceeds the static scratch of sto_run_noalloc (N <= 16384)"; break;
    case STO_ESINGULAR: base = "the ridge system is not positive definite"; break;
    default: break;
  }
  if (code == STO_ECUDA && g_last_cuda != cudaSuccess)
    std::snprintf(g_errbuf, sizeof(g_errbuf), "%s: %s (%s)", base, cudaGetErrorName(g_last_cuda),
                  cudaGetErrorString(g_last_cuda));
  else
    std::snprintf(g_errbuf, sizeof(g_errbuf), "%s", base);
  return g_errbuf;
}

int sto_create(int64_t N, const sto_params* params, const float* W, const float* w_in,
               const float* m0, void* stream, sto_handle** out) {
  return sto_create_ex(N, params, W, w_in, m0, stream, nullptr, out);
}

int sto_create_ex(int64_t N, const sto_params* params, const float* W, const float* w_in,
                  const float* m0, void* stream, const sto_config* cfg, sto_handle** out) {
  return create_impl(N, params, W, sto::kWf32, w_in, m0, false, stream, cfg, out);
}

int sto_create_f64(int64_t N, const sto_params* params, const double* W, const float* w_in,
                   const double* m0, void* stream, const sto_config* cfg, int32_t product,
                   sto_handle** out) {
  if (out) *out = nullptr;
  if (product != STO_PRODUCT_DF && product != STO_PRODUCT_F64) return STO_EINVAL;
  return create_impl(N, params, W, product == STO_PRODUCT_DF ? sto::kWdf : sto::kWf64, w_in, m0, true,
                     stream, cfg, out);
}

void sto_destroy(sto_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  free_handle(h);
}

int sto_set_params(sto_handle* h, const sto_params* params) {
  if (!h) return STO_EINVAL;
  int rc = check_params(params);
  if (rc) return rc;
  if (params->n_in != h->params.n_in) return STO_EINVAL;
  h->params = *params;
  return STO_OK;
}

int sto_get_info(const sto_handle* h, sto_info* out) {
  if (!h || !out) return STO_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->N = h->N;
  out->grid = h->plan.G;
  out->rows_max = h->plan.R_max;
  out->panel_cols = panel_cols(h->wmode);
  out->panels = h->plan.P;
  out->ring_slots = h->plan.ns;
  out->resident = h->plan.resident;
  out->smem_bytes = static_cast<int32_t>(h->plan.smem);
  out->sm_count = h->sm_count;
  out->w_bytes = w_elem_bytes(h->wmode) * h->N * h->N;
  out->xbuf_timed = h->xbuf_timed;
  out->xbuf_slot = h->xbuf_slot;
  if (h->wmode == sto::kWf32)
    out->tmem_panels = tmem_panels_of(h->plan, l2_keeps(h->N),
                                      keep_panels(h->N, h->plan.P, h->l2_keep_mb));
  return STO_OK;
}

int sto_set_state(sto_handle* h, const float* m) {
  if (!h || !m) return STO_EINVAL;
  std::vector<float> mf;
  int rc = fetch_floats(&mf, m, 3 * static_cast<size_t>(h->N), h->stream);
  if (rc) return rc;
  std::vector<double> md(mf.begin(), mf.end());
  return set_state_host_f64(h, md.data());
}

int sto_set_state_f64(sto_handle* h, const double* m) {
  if (!h || !m) return STO_EINVAL;
  const size_t n = 3 * static_cast<size_t>(h->N);
  std::vector<double> md(n);
  STO_CUDA(cudaMemcpyAsync(md.data(), m, n * sizeof(double), cudaMemcpyDefault, h->stream));
  STO_CUDA(cudaStreamSynchronize(h->stream));
  return set_state_host_f64(h, md.data());
}

int sto_get_state_f64(const sto_handle* h, double* m) {
  if (!h || !m) return STO_EINVAL;
  STO_CUDA(cudaMemcpyAsync(m, h->d_state, 3 * static_cast<size_t>(h->N) * sizeof(double),
                           cudaMemcpyDefault, h->stream));
  STO_CUDA(cudaStreamSynchronize(h->stream));
  return STO_OK;
}

int sto_get_state(const sto_handle* h, float* m) {
  if (!h || !m) return STO_EINVAL;
  const size_t n = 3 * static_cast<size_t>(h->N);
  std::vector<double> md(n);
  STO_CUDA(cudaMemcpyAsync(md.data(), h->d_state, n * sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream));
  STO_CUDA(cudaStreamSynchronize(h->stream));
  std::vector<float> mf(n);
  for (size_t i = 0; i < n; ++i) mf[i] = static_cast<float>(md[i]);
  STO_CUDA(cudaMemcpyAsync(m, mf.data(), n * sizeof(float), cudaMemcpyDefault, h->stream));
  STO_CUDA(cudaStreamSynchronize(h->stream));
  return STO_OK;
}

int sto_debug_inject_stall(sto_handle* h, int32_t cta) {
  if (!h) return STO_EINVAL;
  h->inject_cta = cta < 0 ? -1 : cta;
  return STO_OK;
}

int sto_run(sto_handle* h, const float* u, int64_t T, float* states_out) {
  if (!h || T < 0) return STO_EINVAL;
  if (T == 0) return STO_OK;
  if (!u) return STO_EINVAL;
  const sto_params& P = h->params;
  const uint64_t stages = static_cast<uint64_t>(h->rk_stages) * static_cast<uint64_t>(P.substeps) *
                          static_cast<uint64_t>(T);
  if (T > (1LL << 31) - 1 || stages > 0x40000000ULL) return STO_ENOTSUP;
  const int64_t N = h->N;
  cudaStream_t s = h->stream;
  const size_t n_u = static_cast<size_t>(T) * P.n_in;
  const size_t n_states = static_cast<size_t>(T) * N;

  if (const int rc = tune_xbuf(h)) return rc;
  const float* d_u = u;
  if (!is_device_ptr(u)) {
    int rc = grow(&h->d_u, &h->d_u_cap, n_u);
    if (rc) return rc;
    STO_CUDA(cudaMemcpyAsync(h->d_u, u, n_u * 4, cudaMemcpyHostToDevice, s));
    d_u = h->d_u;
  }
  float* d_states = states_out;
  const bool host_states = states_out && !is_device_ptr(states_out);
  if (host_states) {
    int rc = grow(&h->d_states, &h->d_states_cap, n_states);
    if (rc) return rc;
    d_states = h->d_states;
  }
  const int rc = engine_launch(h, d_u, T, d_states, nullptr, nullptr);
  if (rc) return rc;
  if (host_states)
    STO_CUDA(cudaMemcpyAsync(states_out, d_states, n_states * 4, cudaMemcpyDeviceToHost, s));
  return finish_launch(h);
}

// The working set of the overlapped reverse sweep: a second recording, a
// state copy, an error word, a stream and events.  It needs a second
// exchange buffer, which only plans with W on chip have (the placement
// pool); otherwise, or without the memory, the sweep runs in sequence.
int adjoint_overlap_ready(sto_handle* h, size_t rec_floats) {
  if (h->xbuf_n < 2) return STO_ENOTSUP;
  if (const int rc = grow(&h->d_rec2, &h->d_rec2_cap, rec_floats)) return rc;
  const size_t n3 = 3 * static_cast<size_t>(h->N);
  auto fail = [&]() {
    cudaGetLastError();
    return STO_ENOMEM;
  };
  if (!h->d_state2 && cudaMalloc(&h->d_state2, n3 * 8) != cudaSuccess) return fail();
  if (!h->d_err2 && cudaMalloc(&h->d_err2, 16) != cudaSuccess) return fail();
  if (!h->h_err2 && cudaMallocHost(&h->h_err2, 16) != cudaSuccess) return fail();
  if (!h->s_aux && cudaStreamCreateWithFlags(&h->s_aux, cudaStreamNonBlocking) != cudaSuccess) return fail();
  for (cudaEvent_t& e : h->ev_aux)
    if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail();
  return STO_OK;
}

// Step 2 of sto_adjoint with the recomputation of segment g - 1 running
// beside the reverse pass of segment g: the recomputation on the auxiliary
// stream (its own state copy, exchange buffer and error word, the two
// recordings alternating), the reverse passes in order on the handle's
// stream.  Each reverse pass waits for its segment's recording; each
// recomputation waits for the reverse pass that last read its buffer.  The
// launches, their inputs and their order per buffer are those of the plain
// sweep, so the gradients are the same bits.  Both streams are idle on
// return.
int adjoint_reverse_overlapped(sto_handle* h, const float* d_u, const float* d_dl, int64_t K, int64_t nseg,
                               int64_t T) {
  cudaStream_t s = h->stream, s2 = h->s_aux;
  const int64_t N = h->N;
  const int n_in = h->params.n_in;
  const size_t n3 = 3 * static_cast<size_t>(N);
  const size_t rec_m_floats = static_cast<size_t>(K) * h->params.substeps * static_cast<size_t>(N) * 6;
  float* recs[2] = {h->d_rec, h->d_rec2};
  unsigned long long* xbuf2 =
      h->d_xbuf_pool + static_cast<size_t>((h->xbuf_slot + 1) % h->xbuf_n) * (h->xbuf_stride / sizeof(unsigned long long));
  cudaEvent_t ev_start = h->ev_aux[0];
  cudaEvent_t* ev_rec = h->ev_aux + 1;  // recording of buffer b done
  cudaEvent_t* ev_rev = h->ev_aux + 3;  // reverse pass over buffer b done
  // the error words collect the first error of any launch (read at the end)
  STO_CUDA(cudaMemsetAsync(h->d_err, 0, 16, s));
  STO_CUDA(cudaEventRecord(ev_start, s));  // checkpoints and accumulator resets are in place
  STO_CUDA(cudaStreamWaitEvent(s2, ev_start, 0));
  STO_CUDA(cudaMemsetAsync(h->d_err2, 0, 16, s2));
  auto recompute = [&](int64_t g) -> int {
    const int b = static_cast<int>(g & 1);
    const int64_t t0 = g * K, Tg = (T - t0) < K ? (T - t0) : K;
    STO_CUDA(cudaMemcpyAsync(h->d_state2, h->d_ckpt + g * n3, n3 * 8, cudaMemcpyDeviceToDevice, s2));
    sto::KArgs a = base_args(h, d_u + t0 * n_in, Tg);
    a.state = h->d_state2;
    a.xbuf = xbuf2;
    a.err = h->d_err2;
    a.inject_cta = -1;
    a.rec_m = reinterpret_cast<float2*>(recs[b]);
    a.rec_h = recs[b] + rec_m_floats;
    STO_CUDA(launch_stepper(h->plan, a, s2, h->wmode));
    STO_CUDA(cudaEventRecord(ev_rec[b], s2));
    return STO_OK;
  };
  auto reverse = [&](int64_t g) -> int {
    const int b = static_cast<int>(g & 1);
    const int64_t t0 = g * K, Tg = (T - t0) < K ? (T - t0) : K;
    STO_CUDA(cudaStreamWaitEvent(s, ev_rec[b], 0));
    sto::KArgs a = base_args(h, d_u + t0 * n_in, Tg);
    a.W = h->d_WT;
    a.rec_m = reinterpret_cast<float2*>(recs[b]);
    a.rec_h = recs[b] + rec_m_floats;
    a.dLds = d_dl + t0 * N;
    a.lam = h->d_lam;
    a.g_acp = h->d_gacc;
    a.g_cur = h->d_gacc + N;
    a.g_win = h->d_gacc + 2 * N;
    a.inject_cta = -1;
    STO_CUDA(launch_adjoint(h->plan, a, s));
    STO_CUDA(cudaEventRecord(ev_rev[b], s));
    return STO_OK;
  };
  int rc = recompute(nseg - 1);
  for (int64_t g = nseg - 1; g >= 0 && rc == STO_OK; --g) {
    rc = reverse(g);
    if (rc == STO_OK && g > 0) {
      // buffer (g - 1) & 1 was last read by the reverse pass of g + 1
      if (g + 1 <= nseg - 1) {
        const cudaError_t e = cudaStreamWaitEvent(s2, ev_rev[(g - 1) & 1], 0);
        if (e != cudaSuccess) rc = cuda_fail(e);
      }
      if (rc == STO_OK) rc = recompute(g - 1);
    }
  }
  // never return with work in flight on either stream
  const cudaError_t e1 = cudaMemcpyAsync(h->h_err2, h->d_err2, 16, cudaMemcpyDeviceToHost, s2);
  const cudaError_t e2 = cudaMemcpyAsync(h->h_err, h->d_err, 16, cudaMemcpyDeviceToHost, s);
  const cudaError_t e3 = cudaStreamSynchronize(s2);
  const cudaError_t e4 = cudaStreamSynchronize(s);
  if (rc) return rc;
  for (cudaError_t e : {e1, e2, e3, e4})
    if (e != cudaSuccess) return cuda_fail(e);
  for (const int* w : {h->h_err, h->h_err2})
    if (w[0] != 0) return w[0] == sto::kErrTimeout ? STO_ETIMEOUT : STO_ECUDA;
  return STO_OK;
}

int sto_adjoint(sto_handle* h, const float* u, int64_t T, const float* dL_dstates,
                int32_t ckpt_every, sto_grads* out) {
  if (!h || T < 1 || !u || !dL_dstates || !out || ckpt_every < 1) return STO_EINVAL;
  if (!h->rk_classic) return STO_ENOTSUP;  // the adjoint is that of classic RK4
  if (h->wmode != sto::kWf32) return STO_ENOTSUP;  // and of the FP32 coupling
  const sto_params& P = h->params;
  const uint64_t stages = 4ULL * static_cast<uint64_t>(P.substeps) * static_cast<uint64_t>(T);
  if (T > (1LL << 31) - 1 || stages > 0x40000000ULL) return STO_ENOTSUP;
  const int64_t N = h->N;
  const int n_in = P.n_in;
  cudaStream_t s = h->stream;
  if (const int rc = tune_xbuf(h)) return rc;
  const int64_t K = ckpt_every < T ? ckpt_every : T;
  const int64_t nseg = (T + K - 1) / K;
  const size_t n3 = 3 * static_cast<size_t>(N);
  const size_t rec_floats = static_cast<size_t>(K) * P.substeps * static_cast<size_t>(N) * 10;
  int rc;

  // inputs on the device
  const float* d_u = u;
  if (!is_device_ptr(u)) {
    rc = grow(&h->d_u, &h->d_u_cap, static_cast<size_t>(T) * n_in);
    if (rc) return rc;
    STO_CUDA(cudaMemcpyAsync(h->d_u, u, static_cast<size_t>(T) * n_in * 4, cudaMemcpyHostToDevice, s));
    d_u = h->d_u;
  }
  const float* d_dl = dL_dstates;
  if (!is_device_ptr(dL_dstates)) {
    rc = grow(&h->d_dl, &h->d_dl_cap, static_cast<size_t>(T) * N);
    if (rc) return rc;
    STO_CUDA(cudaMemcpyAsync(h->d_dl, dL_dstates, static_cast<size_t>(T) * N * 4,
                             cudaMemcpyHostToDevice, s));
    d_dl = h->d_dl;
  }
  // working set
  rc = ensure_transpose(h);
  if (rc) return rc;
  rc = grow(&h->d_rec, &h->d_rec_cap, rec_floats);
  if (rc) return rc;
  rc = grow_d(&h->d_ckpt, &h->d_ckpt_cap, static_cast<size_t>(nseg + 1) * n3);
  if (rc) return rc;
  if (!h->d_lam) {
    if (cudaMalloc(&h->d_lam, n3 * 8) != cudaSuccess ||
        cudaMalloc(&h->d_gacc, (2 + static_cast<size_t>(n_in)) * N * 8) != cudaSuccess) {
      cudaGetLastError();
      return STO_ENOMEM;
    }
  }
  float2* rec_m = reinterpret_cast<float2*>(h->d_rec);
  float* rec_h = h->d_rec + static_cast<size_t>(K) * P.substeps * N * 6;

  // the tags of the whole call (three sweeps) fit before the counter wraps:
  // a wrap resets the whole pool, which must not happen while the
  // overlapped sweep's second exchange buffer is in use
  if (h->stage_counter + 3 * stages + 8 * static_cast<uint64_t>(nseg) + 16 >= 0xfffffff0ULL) {
    STO_CUDA(cudaMemsetAsync(h->d_xbuf_pool, 0xff, h->xbuf_n * h->xbuf_stride, s));
    h->stage_counter = 0;
  }
  // 1. checkpoints every K samples
  STO_CUDA(cudaMemcpyAsync(h->d_ckpt, h->d_state, n3 * 8, cudaMemcpyDeviceToDevice, s));
  for (int64_t g = 0; g < nseg; ++g) {
    const int64_t t0 = g * K, Tg = (T - t0) < K ? (T - t0) : K;
    rc = engine_launch(h, d_u + t0 * n_in, Tg, nullptr, nullptr, nullptr);
    if (!rc) rc = finish_launch(h);
    if (rc) return rc;
    STO_CUDA(cudaMemcpyAsync(h->d_ckpt + (g + 1) * n3, h->d_state, n3 * 8,
                             cudaMemcpyDeviceToDevice, s));
  }
  // 2. segments in reverse: recompute with recording, then the adjoint pass
  STO_CUDA(cudaMemsetAsync(h->d_lam, 0, n3 * 8, s));
  STO_CUDA(cudaMemsetAsync(h->d_gacc, 0, (2 + static_cast<size_t>(n_in)) * N * 8, s));
  if (nseg > 1 && adjoint_overlap_ready(h, rec_floats) == STO_OK) {
    // the recomputation of segment g - 1 overlaps the reverse pass of g
    rc = adjoint_reverse_overlapped(h, d_u, d_dl, K, nseg, T);
    if (rc) return rc;
  } else {
  for (int64_t g = nseg - 1; g >= 0; --g) {
    const int64_t t0 = g * K, Tg = (T - t0) < K ? (T - t0) : K;
    STO_CUDA(cudaMemcpyAsync(h->d_state, h->d_ckpt + g * n3, n3 * 8, cudaMemcpyDeviceToDevice, s));
    rc = engine_launch(h, d_u + t0 * n_in, Tg, nullptr, rec_m, rec_h);
    if (!rc) rc = finish_launch(h);
    if (!rc) rc = engine_launch_adjoint(h, d_u + t0 * n_in, Tg, d_dl + t0 * N, rec_m, rec_h);
    if (!rc) rc = finish_launch(h);
    if (rc) return rc;
  }
  }
  // 3. results; the state ends where sto_run would leave it
  STO_CUDA(cudaMemcpyAsync(h->d_state, h->d_ckpt + nseg * n3, n3 * 8, cudaMemcpyDeviceToDevice, s));
  std::vector<double> gacc((2 + static_cast<size_t>(n_in)) * N);
  std::vector<double> lam(n3);
  STO_CUDA(cudaMemcpyAsync(gacc.data(), h->d_gacc, gacc.size() * 8, cudaMemcpyDeviceToHost, s));
  STO_CUDA(cudaMemcpyAsync(lam.data(), h->d_lam, n3 * 8, cudaMemcpyDeviceToHost, s));
  STO_CUDA(cudaStreamSynchronize(s));
  double ga = 0.0, gc = 0.0;
  for (int64_t k = 0; k < N; ++k) {
    ga += gacc[k];
    gc += gacc[N + k];
  }
  out->dA_cp = ga;
  out->dcurrent = gc;
  if (out->dw_in) {
    STO_CUDA(cudaMemcpyAsync(out->dw_in, gacc.data() + 2 * N, static_cast<size_t>(N) * n_in * 8,
                             cudaMemcpyDefault, s));
  }
  if (out->dm0) STO_CUDA(cudaMemcpyAsync(out->dm0, lam.data(), n3 * 8, cudaMemcpyDefault, s));
  STO_CUDA(cudaStreamSynchronize(s));
  return STO_OK;
}

int sto_run_group(sto_handle* const* hs, int32_t n, const float* u, int64_t T,
                  float* const* states_out) {
  if (!hs || n < 1 || T < 0) return STO_EINVAL;
  if (T == 0) return STO_OK;
  if (!u) return STO_EINVAL;
  sto_handle* h0 = hs[0];
  if (!h0) return STO_EINVAL;
  const int n_in = h0->params.n_in;
  for (int i = 0; i < n; ++i) {
    if (!hs[i] || hs[i]->params.n_in != n_in || hs[i]->device != h0->device) return STO_EINVAL;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return STO_EINVAL;
    const uint64_t stages = static_cast<uint64_t>(hs[i]->rk_stages) *
                            static_cast<uint64_t>(hs[i]->params.substeps) * static_cast<uint64_t>(T);
    if (stages > 0x40000000ULL) return STO_ENOTSUP;
  }
  if (T > (1LL << 31) - 1) return STO_ENOTSUP;
  cudaStream_t s0 = h0->stream;
  // the shared input, staged once
  const size_t n_u = static_cast<size_t>(T) * n_in;
  const float* d_u = u;
  if (!is_device_ptr(u)) {
    int rc = grow(&h0->d_u, &h0->d_u_cap, n_u);
    if (rc) return rc;
    STO_CUDA(cudaMemcpyAsync(h0->d_u, u, n_u * 4, cudaMemcpyHostToDevice, s0));
    d_u = h0->d_u;
  }
  std::vector<float*> d_states(n, nullptr);
  for (int i = 0; i < n; ++i) {
    float* so = states_out ? states_out[i] : nullptr;
    d_states[i] = so;
    if (so && !is_device_ptr(so)) {
      int rc = grow(&hs[i]->d_states, &hs[i]->d_states_cap, static_cast<size_t>(T) * hs[i]->N);
      if (rc) return rc;
      d_states[i] = hs[i]->d_states;
    }
  }
  // every reservoir's persistent launch, in order, as one CUDA graph
  cudaStream_t cs = nullptr;
  cudaEvent_t ev = nullptr;
  STO_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    e = cudaEventRecord(ev, hs[i]->stream);  // after each handle's earlier work
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev, 0);
  }
  if (e == cudaSuccess) e = cudaEventRecord(ev, s0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev, 0);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int rc = STO_OK;
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int i = 0; i < n && !rc; ++i) rc = engine_launch_on(hs[i], cs, d_u, T, d_states[i], nullptr, nullptr);
    const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (!rc && ce != cudaSuccess) rc = cuda_fail(ce);
  } else {
    rc = cuda_fail(e);
  }
  if (!rc) {
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, cs);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
      float* so = states_out ? states_out[i] : nullptr;
      if (so && so != d_states[i])
        e = cudaMemcpyAsync(so, d_states[i], static_cast<size_t>(T) * hs[i]->N * 4,
                            cudaMemcpyDeviceToHost, cs);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) rc = cuda_fail(e);
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaEventDestroy(ev);
  cudaStreamDestroy(cs);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    hs[i]->inject_cta = -1;
    if (hs[i]->h_err[0] != 0) return hs[i]->h_err[0] == sto::kErrTimeout ? STO_ETIMEOUT : STO_ECUDA;
  }
  return STO_OK;
}

int sto_group_create(sto_handle* const* hs, int32_t n, int32_t lanes, sto_group** out) {
  return sto_group_create_ex(hs, n, lanes, 0, out);
}

int sto_group_create_ex(sto_handle* const* hs, int32_t n, int32_t lanes, int32_t ctas, sto_group** out) {
  if (!out) return STO_EINVAL;
  *out = nullptr;
  if (!hs || n < 1 || lanes < 0 || ctas < 0) return STO_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!hs[i] || hs[i]->params.n_in != hs[0]->params.n_in || hs[i]->device != hs[0]->device) return STO_EINVAL;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return STO_EINVAL;
    if (hs[i]->wmode != sto::kWf32) return STO_ENOTSUP;  // the group kernel runs the FP32 coupling
  }
  if (ctas > hs[0]->sm_count) return STO_EINVAL;
  const int sms = ctas > 0 ? ctas : hs[0]->sm_count;  // the CTAs the group's lanes share
  int64_t n_min = hs[0]->N, n_max = hs[0]->N;
  for (int i = 0; i < n; ++i) {
    n_min = hs[i]->N < n_min ? hs[i]->N : n_min;
    n_max = hs[i]->N > n_max ? hs[i]->N : n_max;
  }
  // lanes of `width` CTAs: every reservoir needs at least one oscillator per
  // CTA and at most 8 rows per consumer warp (120 per CTA)
  auto fits = [&](int L) {
    const int w = sms / L;
    return L >= 1 && w >= 1 && n_min >= w && (n_max + w - 1) / w <= 8 * sto::kConsWarps;
  };
  int L = lanes;
  if (L == 0) {
    for (L = n < 8 ? n : 8; L > 1 && !fits(L); --L) {
    }
  }
  if (L > sms || !fits(L)) return STO_ENOTSUP;
  sto_group* g = new (std::nothrow) sto_group();
  if (!g) return STO_ENOMEM;
  g->hs.assign(hs, hs + n);
  g->n = n;
  g->lanes = L;
  g->width = sms / L;
  // a group that shares its launch with a sweep (ctas > 0) runs inside
  // sweep_group_kernel, whose static shared memory its plans leave room for
  size_t reserve = 0;
  if (ctas > 0) {
    cudaFuncAttributes fa{};
    if (const cudaError_t e = cudaFuncGetAttributes(&fa, sto::sweep_group_kernel)) {
      free_group(g);
      return cuda_fail(e);
    }
    reserve = fa.sharedSizeBytes;
  }
  for (int i = 0; i < n; ++i) {
    const int rc = replan_handle(hs[i], g->width, reserve);
    if (rc) {
      free_group(g);
      return rc;
    }
    // members keep W in shared memory (the group kernel inlines no
    // register-W engine: its register budget goes to the streaming members)
    hs[i]->plan.regw = 0;
    const int rpw = hs[i]->plan.rpw <= 1 ? 1 : (hs[i]->plan.rpw <= 2 ? 2 : (hs[i]->plan.rpw <= 4 ? 4 : 8));
    g->rpw.push_back(rpw);
    g->smem = hs[i]->plan.smem > g->smem ? hs[i]->plan.smem : g->smem;
  }
  // longest processing time first onto the least loaded lane; a reservoir's
  // time is its stage count times the larger of the exchange latency (about
  // 2.5 us per stage) and streaming its W at ~90 GB/s per CTA
  std::vector<double> cost(n), load(L, 0.0);
  std::vector<std::vector<int>> lane_jobs(L);
  for (int i = 0; i < n; ++i) {
    const double w_s = 4.0 * static_cast<double>(hs[i]->N) * hs[i]->N / (g->width * 90e9);
    cost[i] = (w_s > 2.5e-6 ? w_s : 2.5e-6) * hs[i]->rk_stages * hs[i]->params.substeps;
  }
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  for (int i : idx) {
    int best = 0;
    for (int l = 1; l < L; ++l)
      if (load[l] < load[best]) best = l;
    load[best] += cost[i];
    lane_jobs[best].push_back(i);
  }
  // odd lanes run their jobs shortest first, so that while some lanes
  // stream large W from HBM the others run small, latency-bound members
  // (largest first everywhere puts every lane on HBM at the start and every
  // lane on latency-bound members at the end)
  for (int l = 1; l < L; l += 2) std::reverse(lane_jobs[l].begin(), lane_jobs[l].end());
  g->lane_begin.push_back(0);
  for (int l = 0; l < L; ++l) {
    for (int j : lane_jobs[l]) g->order.push_back(j);
    g->lane_begin.push_back(static_cast<int>(g->order.size()));
  }
  // device tables
  const size_t tab_n = g->lane_begin.size() + g->order.size() + g->rpw.size();
  std::vector<int> tab;
  tab.insert(tab.end(), g->lane_begin.begin(), g->lane_begin.end());
  tab.insert(tab.end(), g->order.begin(), g->order.end());
  tab.insert(tab.end(), g->rpw.begin(), g->rpw.end());
  cudaStream_t s = hs[0]->stream;
  cudaError_t e = cudaMalloc(&g->d_jobs, sizeof(sto::KArgs) * n);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_tab, sizeof(int) * tab_n);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_errs, sizeof(int) * 4 * n);
  if (e == cudaSuccess) e = cudaMallocHost(&g->h_jobs, sizeof(sto::KArgs) * n);
  if (e == cudaSuccess) e = cudaMallocHost(&g->h_errs, sizeof(int) * 4 * n);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->d_tab, tab.data(), sizeof(int) * tab_n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_group(g);
    return e == cudaErrorMemoryAllocation ? STO_ENOMEM : cuda_fail(e);
  }
  *out = g;
  return STO_OK;
}

int sto_group_run(sto_group* g, const float* u, int64_t T, float* const* states_out) {
  if (!g || T < 0) return STO_EINVAL;
  if (T == 0) return STO_OK;
  if (!u || T > (1LL << 31) - 1) return u ? STO_ENOTSUP : STO_EINVAL;
  const int n = g->n;
  sto_handle* h0 = g->hs[0];
  cudaStream_t s0 = h0->stream;
  for (int i = 0; i < n; ++i) {
    sto_handle* h = g->hs[i];
    // planned for the lane, classic RK4, FP32 coupling (a tableau set since
    // creation or a re-planned handle cannot run here)
    if (!h->rk_classic || h->wmode != sto::kWf32 || h->plan.G != g->width || h->plan.regw) return STO_ENOTSUP;
    const uint64_t stages = 4ULL * static_cast<uint64_t>(h->params.substeps) * static_cast<uint64_t>(T);
    if (stages > 0x40000000ULL) return STO_ENOTSUP;
    if (h->params.n_in != h0->params.n_in) return STO_EINVAL;
  }
  const size_t n_u = static_cast<size_t>(T) * h0->params.n_in;
  const float* d_u = u;
  if (!is_device_ptr(u)) {
    int rc = grow(&g->d_u, &g->d_u_cap, n_u);
    if (rc) return rc;
    STO_CUDA(cudaMemcpyAsync(g->d_u, u, n_u * 4, cudaMemcpyHostToDevice, s0));
    d_u = g->d_u;
  }
  std::vector<float*> d_states(n, nullptr);
  for (int i = 0; i < n; ++i) {
    float* so = states_out ? states_out[i] : nullptr;
    d_states[i] = so;
    if (so && !is_device_ptr(so)) {
      int rc = grow(&g->hs[i]->d_states, &g->hs[i]->d_states_cap, static_cast<size_t>(T) * g->hs[i]->N);
      if (rc) return rc;
      d_states[i] = g->hs[i]->d_states;
    }
  }
  STO_CUDA(cudaStreamSynchronize(s0));  // the pinned job records are free to rewrite
  for (int i = 0; i < n; ++i) {
    sto::KArgs a = base_args(g->hs[i], d_u, T);  // may reset the exchange buffer on the member's stream
    a.states_out = d_states[i];
    a.err = g->d_errs + 4 * i;
    g->h_jobs[i] = a;
  }
  // the launch follows every member's earlier work
  cudaEvent_t ev = nullptr;
  STO_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t e = cudaSuccess;
  for (int i = 1; i < n && e == cudaSuccess; ++i) {
    if (g->hs[i]->stream == s0) continue;
    e = cudaEventRecord(ev, g->hs[i]->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s0, ev, 0);
  }
  cudaEventDestroy(ev);
  if (e != cudaSuccess) return cuda_fail(e);
  STO_CUDA(cudaMemcpyAsync(g->d_jobs, g->h_jobs, sizeof(sto::KArgs) * n, cudaMemcpyHostToDevice, s0));
  STO_CUDA(cudaMemsetAsync(g->d_errs, 0, sizeof(int) * 4 * n, s0));
  sto::GroupArgs ga{};
  ga.jobs = g->d_jobs;
  ga.lane_begin = g->d_tab;
  ga.order = g->d_tab + g->lane_begin.size();
  ga.rpw = g->d_tab + g->lane_begin.size() + g->order.size();
  ga.n_lanes = g->lanes;
  ga.lane_width = g->width;
  const int room = raise_dyn_smem_cap(sto::sto_group_kernel);
  if (room < static_cast<int>(g->smem)) return STO_ENOTSUP;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(g->lanes * g->width);
  cfg.blockDim = dim3(sto::kThreads);
  cfg.dynamicSmemBytes = g->smem;
  cfg.stream = s0;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every lane's CTAs resident together
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  STO_CUDA(cudaLaunchKernelEx(&cfg, sto::sto_group_kernel, ga));
  STO_CUDA(cudaMemcpyAsync(g->h_errs, g->d_errs, sizeof(int) * 4 * n, cudaMemcpyDeviceToHost, s0));
  for (int i = 0; i < n; ++i) {
    float* so = states_out ? states_out[i] : nullptr;
    if (so && so != d_states[i])
      STO_CUDA(cudaMemcpyAsync(so, d_states[i], static_cast<size_t>(T) * g->hs[i]->N * 4, cudaMemcpyDeviceToHost,
                               s0));
  }
  STO_CUDA(cudaStreamSynchronize(s0));
  int rc = STO_OK;
  for (int i = 0; i < n; ++i) {
    g->hs[i]->inject_cta = -1;
    if (g->h_errs[4 * i] != 0 && rc == STO_OK) rc = g->h_errs[4 * i] == sto::kErrTimeout ? STO_ETIMEOUT : STO_ECUDA;
  }
  return rc;
}

int sto_group_get_info(const sto_group* g, int32_t* lanes, int32_t* lane_width, int32_t* lane_of) {
  if (!g) return STO_EINVAL;
  if (lanes) *lanes = g->lanes;
  if (lane_width) *lane_width = g->width;
  if (lane_of)
    for (int l = 0; l < g->lanes; ++l)
      for (int k = g->lane_begin[l]; k < g->lane_begin[l + 1]; ++k) lane_of[g->order[k]] = l;
  return STO_OK;
}

void sto_group_destroy(sto_group* g) {
  if (!g) return;
  cudaStreamSynchronize(g->hs[0]->stream);
  free_group(g);
}

int sto_set_tableau(sto_handle* h, int32_t stages, const double* a, const double* b) {
  if (!h) return STO_EINVAL;
  if (stages == 0) {  // back to classic RK4
    h->rk_stages = 4;
    h->rk_classic = true;
    return STO_OK;
  }
  if (stages < 1 || stages > 4 || !a || !b) return STO_EINVAL;
  if (h->wmode != sto::kWf32) return STO_ENOTSUP;  // tableaus run with the FP32 coupling
  for (int i = 0; i < stages; ++i) {
    if (!std::isfinite(b[i])) return STO_EINVAL;
    for (int j = 0; j < stages; ++j) {
      const double v = a[i * stages + j];
      if (!std::isfinite(v) || (j >= i && v != 0.0)) return STO_EINVAL;  // explicit only
    }
  }
  h->rk_stages = stages;
  for (int i = 0; i < 4; ++i) {
    h->rk_b[i] = i < stages ? b[i] : 0.0;
    for (int j = 0; j < 4; ++j) h->rk_a[i * 4 + j] = (i < stages && j < stages) ? a[i * stages + j] : 0.0;
  }
  h->rk_classic = false;
  return STO_OK;
}

int sto_set_input_weights(sto_handle* h, const float* w_in) {
  if (!h || !w_in) return STO_EINVAL;
  const size_t n = static_cast<size_t>(h->N) * h->params.n_in;
  int rc = upload_floats(h->d_win, w_in, n, h->stream);
  if (rc) return rc;
  bool bad = false;
  rc = any_nonfinite(h->d_win, static_cast<long long>(n), h->stream, h->d_err, h->h_err, &bad);
  if (rc) return rc;
  return bad ? STO_ENONFINITE : STO_OK;
}

int sto_run_noalloc(int64_t N, const sto_params* params, const float* W, const float* w_in,
                    double* state, const float* u, int64_t T, float* states_out, void* stream) {
  int rc = check_params(params);
  if (rc) return rc;
  if (N < 1 || T < 0 || !W || !w_in || !state || (T > 0 && !u)) return STO_EINVAL;
  if (N > kNoAllocMaxN) return STO_ETOOBIG;
  if (N % 4 != 0 || (reinterpret_cast<uintptr_t>(W) & 15u) != 0) return STO_EINVAL;
  if (T == 0) return STO_OK;
  const sto_params& P = *params;
  const uint64_t stages = 4ULL * static_cast<uint64_t>(P.substeps) * static_cast<uint64_t>(T);
  if (T > (1LL << 31) - 1 || stages > 0x40000000ULL) return STO_ENOTSUP;
  if (!is_device_ptr(W) || !is_device_ptr(w_in) || !is_device_ptr(state) || !is_device_ptr(u) ||
      (states_out && !is_device_ptr(states_out)))
    return STO_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sm_count = 0, smem_optin = 0;
  STO_CUDA(cudaGetDevice(&dev));
  STO_CUDA(cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev));
  STO_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  Plan plan;
  rc = make_plan(N, 0, sm_count, static_cast<size_t>(smem_optin), &plan);
  if (rc) return rc;
  unsigned char* scratch = nullptr;
  rc = noalloc_scratch(dev, &scratch);
  if (rc) return rc;
  int* d_err = reinterpret_cast<int*>(scratch);
  int* d_flag = reinterpret_cast<int*>(scratch + 16);
  auto* d_xbuf = reinterpret_cast<unsigned long long*>(scratch + kNoAllocHeader);

  // The scratch keeps the previous call's contents: clear the error word and
  // flag, and mark every exchange word with tag 0xffffffff (never used).
  STO_CUDA(cudaMemsetAsync(scratch, 0, kNoAllocHeader, s));
  STO_CUDA(cudaMemsetAsync(d_xbuf, 0xff, 2 * static_cast<size_t>(N) * 8, s));
  const long long nw = N * N, nwin = N * static_cast<long long>(P.n_in);
  sto::nonfinite_kernel<<<4096, 256, 0, s>>>(W, nw, d_flag);
  STO_CUDA(cudaGetLastError());
  sto::nonfinite_kernel<<<static_cast<unsigned>((nwin + 255) / 256 < 4096 ? (nwin + 255) / 256 : 4096),
                          256, 0, s>>>(w_in, nwin, d_flag);
  STO_CUDA(cudaGetLastError());
  int h_flag = 0;
  STO_CUDA(cudaMemcpyAsync(&h_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  STO_CUDA(cudaStreamSynchronize(s));
  if (h_flag) return STO_ENONFINITE;

  sto::KArgs a{};
  a.W = W;
  a.w_in = w_in;
  a.u = u;
  a.state = state;
  a.states_out = states_out;
  a.xbuf = d_xbuf;
  a.err = d_err;
  a.N = static_cast<int>(N);
  a.n_in = P.n_in;
  a.T = static_cast<int>(T);
  a.S = P.substeps;
  a.P = plan.P;
  a.ns = plan.ns;
  a.resident = plan.resident;
  a.comp = P.sample_component;
  a.inject_cta = -1;
  a.tag_base = 1u;
  a.timeout_ns = static_cast<unsigned long long>(kDefaultTimeoutMs) * 1000000ULL;
  a.l2_keep = l2_keeps(N);
  a.rk_stages = 4;
  set_constants(P, &a);
  STO_CUDA(launch_stepper_rowmajor(plan, a, s));
  int h_err[4] = {0, 0, 0, 0};
  STO_CUDA(cudaMemcpyAsync(h_err, d_err, sizeof(h_err), cudaMemcpyDeviceToHost, s));
  STO_CUDA(cudaStreamSynchronize(s));
  if (h_err[0] != 0) return h_err[0] == sto::kErrTimeout ? STO_ETIMEOUT : STO_ECUDA;
  return STO_OK;
}

// ---------------------------------------------------------------- sweep

// Launch plan of the persistent sweep kernel: tile width (reservoirs per
// tile), copy-ring depth, CTAs.
struct SweepPlan {
  int bn = 0, slots = 0, G = 0, tiles_m = 0, tiles_n = 0, acc_cols = 0, staged = 0;
  int groups = 1, tn_split = 0;  // reservoir groups with their own barriers (see sweep.cuh)
  int epq = 3;                   // epilogue warps per TMEM lane quarter: 3 (512 threads) or 7 (1024)
  size_t smem = 0;
};

// Threads per CTA of the sweep kernel with epq epilogue warps per quarter.
int sweep_threads(int epq) { return epq == 7 ? sto::sp_threads<7>() : sto::sp_threads<3>(); }

}  // namespace

struct sto_batch {
  cudaStream_t stream = nullptr;      // the caller's stream
  cudaStream_t own = nullptr;         // capturable stream the sweep runs on
  cudaEvent_t ev = nullptr;
  int64_t N = 0;
  int32_t R = 0;
  int Mpad = 0, Kpad = 0;
  sto_params params{};
  __nv_bfloat16* Wb = nullptr;
  __nv_bfloat16* X[2] = {nullptr, nullptr};  // stage operands in the plan's tile layout
  size_t x_cap = 0;                   // BF16 values per X buffer
  float* win = nullptr;
  float2* st = nullptr;       // mn | ms | ksum, each [3][R][N]
  sto::df* hs0 = nullptr;     // [R]
  sto::df* aing = nullptr;    // [R] g A_in as double-float
  unsigned long long* gbar = nullptr;  // grid barrier counter
  int* d_err = nullptr;
  int* h_err = nullptr;
  float* d_u = nullptr;
  size_t d_u_cap = 0;
  float* d_states = nullptr;
  size_t d_states_cap = 0;
  SweepPlan plan;
  bool planned = false;
  int tuned = 0, candidates = 0;
  float tuned_us = 0.f;
};

namespace {

void free_batch(sto_batch* b) {
  if (!b) return;
  cudaFree(b->Wb);
  cudaFree(b->X[0]);
  cudaFree(b->X[1]);
  cudaFree(b->win);
  cudaFree(b->st);
  cudaFree(b->hs0);
  cudaFree(b->aing);
  cudaFree(b->gbar);
  cudaFree(b->d_err);
  cudaFree(b->d_u);
  cudaFree(b->d_states);
  if (b->h_err) cudaFreeHost(b->h_err);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->own) cudaStreamDestroy(b->own);
  delete b;
}

// Plan for tile width bn, ring depth slots and 1 or 2 reservoir groups, or
// false when it cannot run: bn a multiple of 8 in [16, 128] (the MMA N = 2 bn
// of the hi/lo stack is a multiple of 16, a tcgen05 M = 128 shape), shared
// memory within the device limit, every CTA resident (one per SM), and with
// two groups at least two tile columns.
bool sweep_plan(const sto_batch* b, int bn, int slots, int staged, int groups, int epq, SweepPlan* out,
                int max_ctas = 0) {
  if (bn < 16 || bn > 128 || bn % 8 != 0 || slots < 2 || slots > sto::kSpMaxSlots || groups < 1 || groups > 2 ||
      (epq != 3 && epq != 7) || (staged && epq != 3))  // 64 registers leave no room to load ahead
    return false;
  SweepPlan p;
  p.bn = bn;
  p.slots = slots;
  p.tiles_m = b->Mpad / sto::kSwM;
  p.tiles_n = (b->R + bn - 1) / bn;
  if (groups == 2 && p.tiles_n < 2) return false;
  p.groups = groups;
  p.tn_split = groups == 2 ? (p.tiles_n + 1) / 2 : p.tiles_n;
  p.acc_cols = 2 * bn <= 32 ? 32 : (2 * bn <= 64 ? 64 : (2 * bn <= 128 ? 128 : 256));  // [hi | lo] columns
  p.staged = staged ? 1 : 0;
  p.epq = epq;
  p.smem = static_cast<size_t>(slots) * sto::kSlotK * (sto::kSwSliceA + 2u * bn * sto::kSwK * 2u) +
           sto::kSpAlignSlack;
  const int room = epq == 7 ? raise_dyn_smem_cap(sto::sweep_persistent_kernel<7>)
                            : raise_dyn_smem_cap(sto::sweep_persistent_kernel<3>);
  if (room < 0 || p.smem > static_cast<size_t>(room)) return false;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return false;
  const cudaError_t occ =
      epq == 7 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sto::sweep_persistent_kernel<7>,
                                                               sweep_threads(7), p.smem)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sto::sweep_persistent_kernel<3>,
                                                               sweep_threads(3), p.smem);
  if (occ != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return false;
  }
  // balanced grid: the fewest CTAs that keep the most loaded one at the
  // minimum number of tiles (of the larger group)
  const long long n_tiles = static_cast<long long>(p.tiles_m) * p.tn_split;
  // one CTA per SM, on at most max_ctas SMs when given
  const long long slots_avail = static_cast<long long>(max_ctas > 0 && max_ctas < sms ? max_ctas : sms);
  const long long per = (n_tiles + slots_avail - 1) / slots_avail;
  p.G = static_cast<int>((n_tiles + per - 1) / per);
  *out = p;
  return true;
}

// Make X buffers for the plan and publish the current stage state into X[0].
int sweep_apply_plan(sto_batch* b, const SweepPlan& p) {
  cudaStream_t s = b->own;
  const size_t need = static_cast<size_t>(p.tiles_n) * p.bn * 2 * b->Kpad;
  if (need > b->x_cap) {
    cudaStreamSynchronize(s);
    for (int i = 0; i < 2; ++i) {
      cudaFree(b->X[i]);
      b->X[i] = nullptr;
      if (cudaMalloc(reinterpret_cast<void**>(&b->X[i]), need * 2) != cudaSuccess) {
        cudaGetLastError();
        b->x_cap = 0;
        return STO_ENOMEM;
      }
    }
    b->x_cap = need;
  }
  const size_t RN = static_cast<size_t>(b->R) * b->N;
  STO_CUDA(cudaMemsetAsync(b->X[0], 0, need * 2, s));
  STO_CUDA(cudaMemsetAsync(b->X[1], 0, need * 2, s));
  // between calls the next stage is stage 0, evaluated at m_n (the stage
  // state array is not rewritten by stage 3)
  sto::sweep_publish_kernel<<<static_cast<unsigned>((RN + 255) / 256), 256, 0, s>>>(
      b->st, b->X[0], static_cast<int>(b->N), b->R, b->Kpad, p.bn);
  STO_CUDA(cudaGetLastError());
  b->plan = p;
  b->planned = true;
  return STO_OK;
}

// Kernel arguments of a sweep launch over T input samples with plan p.
sto::SweepArgs sweep_args(const sto_batch* b, const SweepPlan& p, const float* d_u, int64_t T, int substeps,
                          float* d_states) {
  const sto_params& P = b->params;
  sto::SweepArgs a{};
  const size_t RN = static_cast<size_t>(b->R) * b->N;
  a.Wb = b->Wb;
  a.X0 = b->X[0];
  a.X1 = b->X[1];
  a.mn = b->st;
  a.ms = b->st + 3 * RN;
  a.ksum = b->st + 6 * RN;
  a.states_out = d_states;
  a.w_in = b->win;
  a.u = d_u;
  a.hs0_r = b->hs0;
  a.ain_g_r = b->aing;
  a.err = b->d_err;
  a.gbar = b->gbar;
  a.N = static_cast<int>(b->N);
  a.R = b->R;
  a.Kpad = b->Kpad;
  a.n_in = P.n_in;
  a.comp = P.sample_component;
  a.S = substeps;
  a.T = static_cast<int>(T);
  a.bn = p.bn;
  a.slots = p.slots;
  a.tiles_m = p.tiles_m;
  a.tiles_n = p.tiles_n;
  a.acc_cols = p.acc_cols;
  a.groups = p.groups;
  a.tn_split = p.tn_split;
  a.staged = p.staged;
  a.timeout_ns = static_cast<unsigned long long>(kDefaultTimeoutMs) * 1000000ULL;
  set_constants(P, &a.c);
  return a;
}

// Enqueue one persistent launch over T input samples on the sweep's stream.
int sweep_enqueue(sto_batch* b, const float* d_u, int64_t T, int substeps, float* d_states) {
  const SweepPlan& p = b->plan;
  cudaStream_t s = b->own;
  const sto::SweepArgs a = sweep_args(b, p, d_u, T, substeps, d_states);
  STO_CUDA(cudaMemsetAsync(b->gbar, 0, 16, s));  // one counter per group
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.G);
  cfg.blockDim = dim3(sweep_threads(p.epq));
  cfg.dynamicSmemBytes = p.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: they meet at the grid barrier
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (p.epq == 7)
    STO_CUDA(cudaLaunchKernelEx(&cfg, sto::sweep_persistent_kernel<7>, a));
  else
    STO_CUDA(cudaLaunchKernelEx(&cfg, sto::sweep_persistent_kernel<3>, a));
  return STO_OK;
}

// Tile widths, ring depths and group counts the autotuner times.
constexpr int kTuneBn[] = {16, 32, 40, 48, 64, 80, 96, 112, 128};
constexpr int kTuneSlots[] = {2, 3, 4, 5};
constexpr int kTuneGroups[] = {1, 2};
constexpr int kTuneEpq[] = {3, 7};

struct TuneKey {
  int dev;
  int64_t N;
  int32_t R;
  bool operator<(const TuneKey& o) const {
    return dev != o.dev ? dev < o.dev : (N != o.N ? N < o.N : R < o.R);
  }
};

// Process-wide cache of tuned plans (bn, slots * 2 + staged, groups,
// measured us per stage, epilogue warps per quarter).
std::map<TuneKey, std::array<float, 5>>& tune_cache() {
  static std::map<TuneKey, std::array<float, 5>> m;
  return m;
}
std::mutex& tune_mutex() {
  static std::mutex m;
  return m;
}

// Time every valid (bn, slots) on a short run (2 RK4 steps of one sample of
// zero input) from the batch's own state, restore the state, keep the
// fastest.  Results are cached per (device, N, R) for the process.
int sweep_autotune(sto_batch* b) {
  int dev = 0;
  STO_CUDA(cudaGetDevice(&dev));
  const TuneKey key{dev, b->N, b->R};
  {
    std::lock_guard<std::mutex> lk(tune_mutex());
    auto it = tune_cache().find(key);
    if (it != tune_cache().end()) {
      SweepPlan p;
      const int code = static_cast<int>(it->second[1]);
      if (sweep_plan(b, static_cast<int>(it->second[0]), code / 2, code % 2, static_cast<int>(it->second[2]),
                     static_cast<int>(it->second[4]), &p)) {
        const int rc = sweep_apply_plan(b, p);
        if (rc) return rc;
        b->tuned = 1;
        b->tuned_us = it->second[3];
        return STO_OK;
      }
    }
  }
  cudaStream_t s = b->own;
  const size_t RN = static_cast<size_t>(b->R) * b->N;
  float2* saved = nullptr;
  float* u0 = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    cudaFree(saved);
    cudaFree(u0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaMalloc(reinterpret_cast<void**>(&saved), 9 * RN * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&u0), 64 * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return STO_ENOMEM;
  }
  cudaError_t e;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess ||
      (e = cudaMemsetAsync(u0, 0, 64 * sizeof(float), s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(saved, b->st, 9 * RN * sizeof(float2), cudaMemcpyDeviceToDevice, s)) != cudaSuccess) {
    cleanup();
    return cuda_fail(e);
  }
  float best = 0.f;
  SweepPlan best_p;
  int n = 0;
  int rc = STO_OK;
  for (int bn : kTuneBn) {
    if (bn > ((b->R + 15) / 16) * 16) break;  // tiles wider than R only add padding
    constexpr int kSlotsN = static_cast<int>(sizeof(kTuneSlots) / sizeof(kTuneSlots[0]));
    for (int cand = 0; cand < 8 * kSlotsN; ++cand) {
      const int slots = kTuneSlots[(cand / 2) % kSlotsN], staged = cand % 2,
                groups = kTuneGroups[(cand / (2 * kSlotsN)) % 2], epq = kTuneEpq[cand / (4 * kSlotsN)];
      SweepPlan p;
      if (!sweep_plan(b, bn, slots, staged, groups, epq, &p)) continue;
      if ((rc = sweep_apply_plan(b, p)) != STO_OK) break;
      float ms = 0.f;
      for (int rep = 0; rep < 3 && rc == STO_OK; ++rep) {
        if ((e = cudaMemsetAsync(b->d_err, 0, 16, s)) != cudaSuccess || (e = cudaEventRecord(e0, s)) != cudaSuccess) {
          rc = cuda_fail(e);
          break;
        }
        if ((rc = sweep_enqueue(b, u0, 1, 2, nullptr)) != STO_OK) break;
        if ((e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
            (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess ||
            (e = cudaMemcpyAsync(b->h_err, b->d_err, 16, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess) {
          rc = cuda_fail(e);
          break;
        }
        if (b->h_err[0] != 0) {
          rc = b->h_err[0] == sto::kErrTimeout ? STO_ETIMEOUT : STO_ECUDA;
          break;
        }
      }
      if (rc) break;
      const float us = ms * 1000.f / 8.f;  // the last of three runs, per stage
      ++n;
      if (n == 1 || us < best) {
        best = us;
        best_p = p;
      }
      // back to the state before the trial
      if ((e = cudaMemcpyAsync(b->st, saved, 9 * RN * sizeof(float2), cudaMemcpyDeviceToDevice, s)) != cudaSuccess) {
        rc = cuda_fail(e);
        break;
      }
    }
    if (rc) break;
  }
  if (rc == STO_OK && n == 0) rc = STO_ENOTSUP;
  if (rc == STO_OK) {
    rc = cuda_rc(cudaMemcpyAsync(b->st, saved, 9 * RN * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    if (rc == STO_OK) rc = sweep_apply_plan(b, best_p);
    if (rc == STO_OK) rc = cuda_rc(cudaStreamSynchronize(s));
  } else {
    cudaMemcpyAsync(b->st, saved, 9 * RN * sizeof(float2), cudaMemcpyDeviceToDevice, s);
    cudaStreamSynchronize(s);
    b->planned = false;
  }
  cleanup();
  if (rc) return rc;
  b->tuned = 1;
  b->candidates = n;
  b->tuned_us = best;
  std::lock_guard<std::mutex> lk(tune_mutex());
  tune_cache()[key] = {static_cast<float>(best_p.bn), static_cast<float>(best_p.slots * 2 + best_p.staged),
                       static_cast<float>(best_p.groups), best, static_cast<float>(best_p.epq)};
  return STO_OK;
}

}  // namespace

extern "C" {

int sto_batch_create(int64_t N, int32_t R, const sto_params* params, const double* current,
                     const double* input_gain, const float* W, const float* w_in,
                     const float* m0, void* stream, sto_batch** out) {
  if (!out) return STO_EINVAL;
  *out = nullptr;
  if (N < 1 || R < 1 || !W || !w_in) return STO_EINVAL;
  int rc = check_params(params);
  if (rc) return rc;
  // the update indexes the [3][R][N] state with 32-bit offsets
  if (N > 32768 || R > 65536 || static_cast<long long>(N) * R > (1LL << 29)) return STO_ENOTSUP;
  sto_batch* b = new (std::nothrow) sto_batch();
  if (!b) return STO_ENOMEM;
  b->stream = static_cast<cudaStream_t>(stream);
  b->N = N;
  b->R = R;
  b->params = *params;
  b->Mpad = static_cast<int>((N + sto::kSwM - 1) / sto::kSwM * sto::kSwM);
  constexpr int kKStep = sto::kSlotK * sto::kSwK;  // whole ring slots of K
  b->Kpad = static_cast<int>((N + kKStep - 1) / kKStep * kKStep);
  cudaStream_t s = b->stream;
  auto fail = [&](int code) {
    if (b->stream) cudaStreamSynchronize(b->stream);
    free_batch(b);
    return code;
  };
  const size_t RN = static_cast<size_t>(R) * N;
  const int n_in = params->n_in;
  auto alloc = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return false;
    }
    return true;
  };
  if (!alloc(reinterpret_cast<void**>(&b->Wb), static_cast<size_t>(b->Mpad) * b->Kpad * 2) ||
      !alloc(reinterpret_cast<void**>(&b->win), static_cast<size_t>(N) * n_in * 4) ||
      !alloc(reinterpret_cast<void**>(&b->st), 9 * RN * sizeof(float2)) ||
      !alloc(reinterpret_cast<void**>(&b->hs0), R * sizeof(sto::df)) ||
      !alloc(reinterpret_cast<void**>(&b->aing), R * sizeof(sto::df)) ||
      !alloc(reinterpret_cast<void**>(&b->gbar), 16) ||
      !alloc(reinterpret_cast<void**>(&b->d_err), 16))
    return fail(STO_ENOMEM);
  if (cudaMallocHost(reinterpret_cast<void**>(&b->h_err), 16) != cudaSuccess) {
    cudaGetLastError();
    b->h_err = nullptr;
    return fail(STO_ENOMEM);
  }
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming)) != cudaSuccess)
    return fail(cuda_fail(e));
  // W -> BF16, zero padded
  const float* d_src = W;
  float* d_tmp = nullptr;
  if (!is_device_ptr(W)) {
    if (!alloc(reinterpret_cast<void**>(&d_tmp), static_cast<size_t>(N) * N * 4)) return fail(STO_ENOMEM);
    e = cudaMemcpyAsync(d_tmp, W, static_cast<size_t>(N) * N * 4, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { cudaFree(d_tmp); return fail(cuda_fail(e)); }
    d_src = d_tmp;
  }
  bool bad = false;
  rc = any_nonfinite(d_src, N * N, s, b->d_err, b->h_err, &bad);
  if (!rc && bad) rc = STO_ENONFINITE;
  if (!rc) {
    e = cudaMemsetAsync(b->Wb, 0, static_cast<size_t>(b->Mpad) * b->Kpad * 2, s);
    if (e == cudaSuccess) {
      sto::sweep_pack_w_kernel<<<2048, 256, 0, s>>>(d_src, b->Wb, static_cast<int>(N), b->Kpad);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e);
  }
  if (d_tmp) cudaFree(d_tmp);
  if (rc) return fail(rc);
  rc = upload_floats(b->win, w_in, static_cast<size_t>(N) * n_in, s);
  if (!rc) {
    rc = any_nonfinite(b->win, N * n_in, s, b->d_err, b->h_err, &bad);
    if (!rc && bad) rc = STO_ENONFINITE;
  }
  if (rc) return fail(rc);
  // per-reservoir constants
  std::vector<sto::df> hs0(R);
  std::vector<sto::df> aing(R);
  const double hs0_per_amp = params->hbar * params->eta * 1.0e7 /
                             (2.0 * params->e_charge * params->Ms * params->volume);
  for (int r = 0; r < R; ++r) {
    const double I = current ? current[r] : params->current;
    const double gn = input_gain ? input_gain[r] : params->input_gain;
    if (!std::isfinite(I) || !std::isfinite(gn)) return fail(STO_EINVAL);
    hs0[r] = sto::df_split_host(hs0_per_amp * I);
    aing[r] = sto::df_split_host(params->A_in * gn);
  }
  if ((e = cudaMemcpyAsync(b->hs0, hs0.data(), R * sizeof(sto::df), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(b->aing, aing.data(), R * sizeof(sto::df), cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return fail(cuda_fail(e));
  // states: mn = ms = m0, ksum = 0 (device layout [3][R][N] df), formed on
  // the device: at R N = 2^29 the state is 38.6 GB, more than a host copy
  // should ever hold
  const double phi0 = 2.0 * M_PI / 360.0;
  const double ic[3] = {std::sin(phi0) * std::cos(phi0), std::sin(phi0) * std::sin(phi0), std::cos(phi0)};
  const float* d_m0 = nullptr;
  float* m0_tmp = nullptr;
  if (m0) {
    if (is_device_ptr(m0)) {
      d_m0 = m0;
    } else {
      if (cudaMalloc(reinterpret_cast<void**>(&m0_tmp), 3 * RN * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return fail(STO_ENOMEM);
      }
      if ((e = cudaMemcpyAsync(m0_tmp, m0, 3 * RN * sizeof(float), cudaMemcpyHostToDevice, s)) != cudaSuccess) {
        cudaFree(m0_tmp);
        return fail(cuda_fail(e));
      }
      d_m0 = m0_tmp;
    }
  }
  e = cudaMemsetAsync(b->d_err, 0, 16, s);
  if (e == cudaSuccess) {
    const long long total = 3LL * static_cast<long long>(RN);
    const unsigned blocks = static_cast<unsigned>(total / 256 + 1 < 65536 ? total / 256 + 1 : 65536);
    sto::sweep_state_init_kernel<<<blocks, 256, 0, s>>>(d_m0, R, N, ic[0], ic[1], ic[2], b->st, b->d_err);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_err, b->d_err, 16, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(m0_tmp);
  if (e != cudaSuccess) return fail(cuda_fail(e));
  if (b->h_err[0] != 0) return fail(STO_ENONFINITE);
  // the launch plan (tile width, ring depth) is chosen by the first run
  // (autotuner) or by sto_batch_set_plan
  *out = b;
  return STO_OK;
}

int sto_batch_set_plan(sto_batch* b, int32_t tile_n, int32_t slots) {
  return sto_batch_set_plan_ex(b, tile_n, slots, 1);
}

int sto_batch_set_plan_ex(sto_batch* b, int32_t tile_n, int32_t slots, int32_t groups) {
  return sto_batch_set_plan_staged(b, tile_n, slots, groups, -1);
}

int sto_batch_set_plan_staged(sto_batch* b, int32_t tile_n, int32_t slots, int32_t groups, int32_t staged) {
  return sto_batch_set_plan_threads(b, tile_n, slots, groups, staged, 512);
}

int sto_batch_set_plan_threads(sto_batch* b, int32_t tile_n, int32_t slots, int32_t groups, int32_t staged,
                               int32_t threads) {
  if (!b) return STO_EINVAL;
  if (groups < 1 || groups > 2 || staged < -1 || staged > 1) return STO_EINVAL;
  if (threads != sweep_threads(3) && threads != sweep_threads(7)) return STO_EINVAL;
  cudaStreamSynchronize(b->stream);
  if (tile_n == 0 && slots == 0) return sweep_autotune(b);
  SweepPlan p;
  const int epq = threads == sweep_threads(7) ? 7 : 3;
  // staged = -1: hold the next pair's state in registers where the threads have room (512 threads)
  const bool found = sweep_plan(b, tile_n, slots, staged == -1 ? (epq == 3 ? 1 : 0) : staged, groups, epq, &p);
  if (!found) return STO_ENOTSUP;
  int rc = sweep_apply_plan(b, p);
  if (rc) return rc;
  b->tuned = 0;
  b->candidates = 0;
  b->tuned_us = 0.f;
  return cuda_rc(cudaStreamSynchronize(b->own));
}

int sto_batch_get_plan(const sto_batch* b, sto_batch_plan* out) {
  if (!b || !out) return STO_EINVAL;
  std::memset(out, 0, sizeof(*out));
  if (!b->planned) return STO_OK;
  out->tile_n = b->plan.bn;
  out->slots = b->plan.slots;
  out->grid = b->plan.G;
  out->tiles = b->plan.tiles_m * b->plan.tiles_n;
  out->smem_bytes = static_cast<int32_t>(b->plan.smem);
  out->tuned = b->tuned;
  out->candidates = b->candidates;
  out->tuned_us_per_stage = b->tuned_us;
  out->staged = b->plan.staged;
  out->groups = b->plan.groups;
  out->threads = sweep_threads(b->plan.epq);
  return STO_OK;
}

int sto_run_batched(sto_batch* b, const float* u, int64_t T, float* states_out) {
  if (!b || T < 0) return STO_EINVAL;
  if (T == 0) return STO_OK;
  if (!u) return STO_EINVAL;
  const sto_params& P = b->params;
  if (T > (1LL << 31) - 1 || 4ULL * static_cast<uint64_t>(P.substeps) * static_cast<uint64_t>(T) > 0x40000000ULL)
    return STO_ENOTSUP;
  cudaStream_t s = b->stream;
  if (!b->planned) {
    cudaStreamSynchronize(s);
    const int rc = sweep_autotune(b);
    if (rc) return rc;
  }
  const size_t n_u = static_cast<size_t>(T) * P.n_in;
  const size_t n_states = static_cast<size_t>(T) * b->R * b->N;
  int rc = grow(&b->d_u, &b->d_u_cap, n_u);
  if (rc) return rc;
  STO_CUDA(cudaMemcpyAsync(b->d_u, u, n_u * 4, cudaMemcpyDefault, s));
  float* d_states = states_out;
  const bool host_states = states_out && !is_device_ptr(states_out);
  if (host_states) {
    rc = grow(&b->d_states, &b->d_states_cap, n_states);
    if (rc) return rc;
    d_states = b->d_states;
  }
  STO_CUDA(cudaMemsetAsync(b->d_err, 0, 16, s));
  // the sweep runs on its own stream, ordered after the caller's work
  STO_CUDA(cudaEventRecord(b->ev, s));
  STO_CUDA(cudaStreamWaitEvent(b->own, b->ev, 0));
  // the call (barrier reset + one persistent launch) as a CUDA graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  STO_CUDA(cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal));
  rc = sweep_enqueue(b, b->d_u, T, P.substeps, d_states);
  const cudaError_t ce = cudaStreamEndCapture(b->own, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (ce != cudaSuccess) return cuda_fail(ce);
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, b->own);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev, b->own);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_err, b->d_err, 16, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && host_states)
    e = cudaMemcpyAsync(states_out, d_states, n_states * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (exec) cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e);
  if (b->h_err[0] != 0) return b->h_err[0] == sto::kErrTimeout ? STO_ETIMEOUT : STO_ECUDA;
  return STO_OK;
}

int sto_batch_get_state(const sto_batch* b, double* m) {
  if (!b || !m) return STO_EINVAL;
  const size_t RN = static_cast<size_t>(b->R) * b->N;
  std::vector<float2> mn(3 * RN);
  STO_CUDA(cudaMemcpyAsync(mn.data(), b->st, 3 * RN * sizeof(float2), cudaMemcpyDeviceToHost, b->stream));
  STO_CUDA(cudaStreamSynchronize(b->stream));
  std::vector<double> out(3 * RN);
  for (int r = 0; r < b->R; ++r)
    for (int i = 0; i < 3; ++i)
      for (int64_t k = 0; k < b->N; ++k) {
        const float2 v = mn[i * RN + static_cast<size_t>(r) * b->N + k];
        out[(static_cast<size_t>(r) * 3 + i) * b->N + k] = static_cast<double>(v.x) + v.y;
      }
  STO_CUDA(cudaMemcpyAsync(m, out.data(), out.size() * 8, cudaMemcpyDefault, b->stream));
  STO_CUDA(cudaStreamSynchronize(b->stream));
  return STO_OK;
}

void sto_batch_destroy(sto_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  free_batch(b);
}

}  // extern "C"

// ------------------------------------------------- sweep and group in one launch

extern "C" int sto_run_sweep_group(sto_batch* b, sto_group* g, const float* u, int64_t T, float* sweep_states_out,
                                   float* const* group_states_out) {
  if (!b || !g || T < 0) return STO_EINVAL;
  if (T == 0) return STO_OK;
  if (!u) return STO_EINVAL;
  const int n = g->n;
  sto_handle* h0 = g->hs[0];
  const sto_params& P = b->params;
  if (h0->params.n_in != P.n_in) return STO_EINVAL;
  int dev = 0;
  STO_CUDA(cudaGetDevice(&dev));
  if (dev != h0->device) return STO_EINVAL;
  if (T > (1LL << 31) - 1 || 4ULL * static_cast<uint64_t>(P.substeps) * static_cast<uint64_t>(T) > 0x40000000ULL)
    return STO_ENOTSUP;
  for (int i = 0; i < n; ++i) {
    sto_handle* h = g->hs[i];
    if (!h->rk_classic || h->wmode != sto::kWf32 || h->plan.G != g->width || h->plan.regw) return STO_ENOTSUP;
    if (4ULL * static_cast<uint64_t>(h->params.substeps) * static_cast<uint64_t>(T) > 0x40000000ULL)
      return STO_ENOTSUP;
  }
  const int ctas_g = g->lanes * g->width;
  const int sweep_ctas = h0->sm_count - ctas_g;  // the SMs the group leaves to the sweep
  if (sweep_ctas < 1) return STO_ENOTSUP;
  cudaStream_t s = b->stream;
  int rc;
  if (!b->planned) {
    cudaStreamSynchronize(s);
    if ((rc = sweep_autotune(b))) return rc;
  }
  // the batch's tile width on the sweep's SMs, 512 threads; the X layout
  // depends only on the tile width, so the batch's buffers and plan stay
  SweepPlan pf;
  if (!sweep_plan(b, b->plan.bn, b->plan.slots, 1, b->plan.groups, 3, &pf, sweep_ctas) &&
      !sweep_plan(b, b->plan.bn, b->plan.slots, 1, 1, 3, &pf, sweep_ctas))
    return STO_ENOTSUP;
  const size_t smem = pf.smem > g->smem ? pf.smem : g->smem;
  const int room = raise_dyn_smem_cap(sto::sweep_group_kernel);
  if (room < 0 || smem > static_cast<size_t>(room)) return STO_ENOTSUP;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sto::sweep_group_kernel, sto::kThreads, smem) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return STO_ENOTSUP;
  }
  // inputs and outputs on the device
  const size_t n_u = static_cast<size_t>(T) * P.n_in;
  if ((rc = grow(&b->d_u, &b->d_u_cap, n_u))) return rc;
  STO_CUDA(cudaMemcpyAsync(b->d_u, u, n_u * 4, cudaMemcpyDefault, s));
  const size_t n_sw = static_cast<size_t>(T) * b->R * b->N;
  float* d_sw = sweep_states_out;
  const bool host_sw = sweep_states_out && !is_device_ptr(sweep_states_out);
  if (host_sw) {
    if ((rc = grow(&b->d_states, &b->d_states_cap, n_sw))) return rc;
    d_sw = b->d_states;
  }
  std::vector<float*> d_gs(n, nullptr);
  for (int i = 0; i < n; ++i) {
    float* so = group_states_out ? group_states_out[i] : nullptr;
    d_gs[i] = so;
    if (so && !is_device_ptr(so)) {
      if ((rc = grow(&g->hs[i]->d_states, &g->hs[i]->d_states_cap, static_cast<size_t>(T) * g->hs[i]->N)))
        return rc;
      d_gs[i] = g->hs[i]->d_states;
    }
  }
  STO_CUDA(cudaStreamSynchronize(h0->stream));  // the pinned job records are free to rewrite
  for (int i = 0; i < n; ++i) {
    sto::KArgs a = base_args(g->hs[i], b->d_u, T);
    a.states_out = d_gs[i];
    a.err = g->d_errs + 4 * i;
    g->h_jobs[i] = a;
  }
  // the launch follows the caller's and every member's earlier work
  STO_CUDA(cudaEventRecord(b->ev, s));
  STO_CUDA(cudaStreamWaitEvent(b->own, b->ev, 0));
  for (int i = 0; i < n; ++i) {
    STO_CUDA(cudaEventRecord(b->ev, g->hs[i]->stream));
    STO_CUDA(cudaStreamWaitEvent(b->own, b->ev, 0));
  }
  sto::SweepGroupArgs f{};
  f.sw = sweep_args(b, pf, b->d_u, T, P.substeps, d_sw);
  f.grp.jobs = g->d_jobs;
  f.grp.lane_begin = g->d_tab;
  f.grp.order = g->d_tab + g->lane_begin.size();
  f.grp.rpw = g->d_tab + g->lane_begin.size() + g->order.size();
  f.grp.n_lanes = g->lanes;
  f.grp.lane_width = g->width;
  f.sweep_ctas = pf.G;
  // the call (counters and error words reset, job records, one persistent
  // launch) as a CUDA graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  STO_CUDA(cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaMemsetAsync(b->gbar, 0, 16, b->own);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, 16, b->own);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->d_errs, 0, sizeof(int) * 4 * n, b->own);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->d_jobs, g->h_jobs, sizeof(sto::KArgs) * n, cudaMemcpyHostToDevice, b->own);
  if (e == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(pf.G + ctas_g);
    cfg.blockDim = dim3(sto::kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = b->own;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // every CTA of both roles resident
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, sto::sweep_group_kernel, f);
  }
  const cudaError_t ce = cudaStreamEndCapture(b->own, &graph);
  if (e != cudaSuccess || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(e != cudaSuccess ? e : ce);
  }
  e = cudaGraphInstantiate(&exec, graph, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, b->own);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev, b->own);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_err, b->d_err, 16, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->h_errs, g->d_errs, sizeof(int) * 4 * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && host_sw) e = cudaMemcpyAsync(sweep_states_out, d_sw, n_sw * 4, cudaMemcpyDeviceToHost, s);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    float* so = group_states_out ? group_states_out[i] : nullptr;
    if (so && so != d_gs[i])
      e = cudaMemcpyAsync(so, d_gs[i], static_cast<size_t>(T) * g->hs[i]->N * 4, cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (exec) cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e);
  rc = STO_OK;
  if (b->h_err[0] != 0) rc = b->h_err[0] == sto::kErrTimeout ? STO_ETIMEOUT : STO_ECUDA;
  for (int i = 0; i < n; ++i) {
    g->hs[i]->inject_cta = -1;
    if (g->h_errs[4 * i] != 0 && rc == STO_OK) rc = g->h_errs[4 * i] == sto::kErrTimeout ? STO_ETIMEOUT : STO_ECUDA;
  }
  return rc;
}

// ---------------------------------------------------------------- readout
//
// Ridge readout on the GPU (readout.cuh): Gram matrix, ridge shift, blocked
// Cholesky with the forward substitution folded in, back substitution.  The
// scratch (the (N + 2)^2 FP64 Gram matrix, copies of host inputs) is
// allocated per call and freed before it returns.

namespace {

// Device memory freed when it goes out of scope.
struct ScopedDev {
  void* p = nullptr;
  ScopedDev() = default;
  ScopedDev(const ScopedDev&) = delete;
  ScopedDev& operator=(const ScopedDev&) = delete;
  ~ScopedDev() {
    if (p) cudaFree(p);
  }
  int alloc(size_t bytes) {
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return STO_ENOMEM;
    }
    return STO_OK;
  }
};

// A device pointer to `bytes` of src (host or device): device memory is used
// in place, host memory is copied into tmp on stream s.
int device_input(const void* src, size_t bytes, cudaStream_t s, ScopedDev* tmp, const void** out) {
  if (is_device_ptr(src)) {
    *out = src;
    return STO_OK;
  }
  if (const int rc = tmp->alloc(bytes)) return rc;
  STO_CUDA(cudaMemcpyAsync(tmp->p, src, bytes, cudaMemcpyHostToDevice, s));
  *out = tmp->p;
  return STO_OK;
}

constexpr int64_t kReadoutMaxN = 32768;  // the Gram matrix is (N + 2)^2 doubles (8.6 GB here)

int readout_check(const float* states, int64_t T, int64_t N, int64_t t0, int64_t t1) {
  if (!states || T < 1 || N < 1 || t0 < 0 || t1 > T || t1 <= t0) return STO_EINVAL;
  if (N > kReadoutMaxN) return STO_ENOTSUP;
  return STO_OK;
}

// flag: any non-finite value among n floats (device) or nd doubles (device).
int readout_nonfinite(const float* d_f, long long n, const double* d_d, long long nd, cudaStream_t s,
                      int* d_flag, bool* bad) {
  STO_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), s));
  if (n > 0) {
    const long long b = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    sto::nonfinite_kernel<<<static_cast<unsigned>(b), 256, 0, s>>>(d_f, n, d_flag);
    STO_CUDA(cudaGetLastError());
  }
  if (nd > 0) {
    const long long b = (nd + 255) / 256 < 4096 ? (nd + 255) / 256 : 4096;
    sto::nonfinite_f64_kernel<<<static_cast<unsigned>(b), 256, 0, s>>>(d_d, nd, d_flag);
    STO_CUDA(cudaGetLastError());
  }
  int h = 0;
  STO_CUDA(cudaMemcpyAsync(&h, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  STO_CUDA(cudaStreamSynchronize(s));
  *bad = h != 0;
  return STO_OK;
}

// y_hat (m doubles, device) of the m state rows at d_rows (device).
int readout_predict_dev(const float* d_rows, int64_t m, int64_t N, const double* d_w, double* d_yhat,
                        cudaStream_t s) {
  const int64_t blocks = (m + 7) / 8;
  sto::readout::predict_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(d_rows, N, static_cast<int>(N), m,
                                                                             d_w, d_yhat);
  STO_CUDA(cudaGetLastError());
  return STO_OK;
}

}  // namespace

extern "C" {

int sto_readout_fit(const float* states, int64_t T, int64_t N, const double* y, int64_t t0, int64_t t1,
                    double beta_rel, double* w_out, void* stream) {
  if (int rc = readout_check(states, T, N, t0, t1)) return rc;
  if (!y || !w_out || !std::isfinite(beta_rel) || beta_rel < 0.0) return STO_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t m = t1 - t0, n = N + 1, nr = N + 2;
  int rc;
  // rows [t0, t1) of the states and the target, on the device
  ScopedDev t_states, t_y, t_gram, t_misc, t_w;
  const void* pv = nullptr;
  if ((rc = device_input(states + t0 * N, static_cast<size_t>(m * N) * 4, s, &t_states, &pv))) return rc;
  const float* d_rows = static_cast<const float*>(pv);
  if ((rc = device_input(y + t0, static_cast<size_t>(m) * 8, s, &t_y, &pv))) return rc;
  const double* d_y = static_cast<const double*>(pv);
  if ((rc = t_gram.alloc(static_cast<size_t>(nr) * nr * 8))) return rc;
  if ((rc = t_misc.alloc(64))) return rc;
  double* d_G = static_cast<double*>(t_gram.p);
  int* d_status = static_cast<int*>(t_misc.p);
  int* d_flag = d_status + 1;
  double* d_beta = static_cast<double*>(t_misc.p) + 1;
  double* d_w = w_out;
  if (!is_device_ptr(w_out)) {
    if ((rc = t_w.alloc(static_cast<size_t>(n) * 8))) return rc;
    d_w = static_cast<double*>(t_w.p);
  }
  bool bad = false;
  if ((rc = readout_nonfinite(d_rows, m * N, d_y, m, s, d_flag, &bad))) return rc;
  if (bad) return STO_ENONFINITE;

  using namespace sto::readout;
  const int nri = static_cast<int>(nr), ni = static_cast<int>(n);
  const unsigned gt = static_cast<unsigned>((nr + kGramTile - 1) / kGramTile);
  gram_kernel<<<dim3(gt, gt), 256, 0, s>>>(d_rows, N, d_y, static_cast<int>(N), 0, m, d_G);
  STO_CUDA(cudaGetLastError());
  ridge_shift_kernel<<<1, 1024, 0, s>>>(d_G, nri, ni, beta_rel, d_beta);
  STO_CUDA(cudaGetLastError());
  STO_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), s));
  for (int k0 = 0; k0 < ni; k0 += kCholB) {
    const int kb = ni - k0 < kCholB ? ni - k0 : kCholB;
    chol_diag_kernel<<<1, kCholB * kCholB, 0, s>>>(d_G, nri, k0, kb, d_status);
    STO_CUDA(cudaGetLastError());
    const int below = nri - k0 - kb;  // rows under the diagonal block, the target row included
    if (below > 0) {
      chol_panel_kernel<<<static_cast<unsigned>((below + 255) / 256), 256, 0, s>>>(d_G, nri, nri, k0, kb,
                                                                                   d_status);
      STO_CUDA(cudaGetLastError());
      const unsigned ut = static_cast<unsigned>((below + kUpdTile - 1) / kUpdTile);
      chol_update_kernel<<<dim3(ut, ut), 256, 0, s>>>(d_G, nri, nri, k0, kb, d_status);
      STO_CUDA(cudaGetLastError());
    }
  }
  back_solve_kernel<<<1, 1024, 0, s>>>(d_G, nri, nri, ni, d_w, d_status);
  STO_CUDA(cudaGetLastError());
  int status = 0;
  STO_CUDA(cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (d_w != w_out) STO_CUDA(cudaMemcpyAsync(w_out, d_w, static_cast<size_t>(n) * 8, cudaMemcpyDeviceToHost, s));
  STO_CUDA(cudaStreamSynchronize(s));
  return status ? STO_ESINGULAR : STO_OK;
}

int sto_readout_predict(const float* states, int64_t T, int64_t N, const double* w, double* y_hat,
                        void* stream) {
  if (int rc = readout_check(states, T, N, 0, T)) return rc;
  if (!w || !y_hat) return STO_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc;
  ScopedDev t_states, t_w, t_out;
  const void* pv = nullptr;
  if ((rc = device_input(states, static_cast<size_t>(T * N) * 4, s, &t_states, &pv))) return rc;
  const float* d_rows = static_cast<const float*>(pv);
  if ((rc = device_input(w, static_cast<size_t>(N + 1) * 8, s, &t_w, &pv))) return rc;
  const double* d_w = static_cast<const double*>(pv);
  double* d_out = y_hat;
  if (!is_device_ptr(y_hat)) {
    if ((rc = t_out.alloc(static_cast<size_t>(T) * 8))) return rc;
    d_out = static_cast<double*>(t_out.p);
  }
  if ((rc = readout_predict_dev(d_rows, T, N, d_w, d_out, s))) return rc;
  if (d_out != y_hat) STO_CUDA(cudaMemcpyAsync(y_hat, d_out, static_cast<size_t>(T) * 8, cudaMemcpyDeviceToHost, s));
  STO_CUDA(cudaStreamSynchronize(s));
  return STO_OK;
}

int sto_readout_nmse(const float* states, int64_t T, int64_t N, const double* w, const double* y, int64_t t0,
                     int64_t t1, double* nmse, void* stream) {
  if (int rc = readout_check(states, T, N, t0, t1)) return rc;
  if (!w || !y || !nmse) return STO_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t m = t1 - t0;
  int rc;
  ScopedDev t_states, t_w, t_y, t_yhat, t_out;
  const void* pv = nullptr;
  if ((rc = device_input(states + t0 * N, static_cast<size_t>(m * N) * 4, s, &t_states, &pv))) return rc;
  const float* d_rows = static_cast<const float*>(pv);
  if ((rc = device_input(w, static_cast<size_t>(N + 1) * 8, s, &t_w, &pv))) return rc;
  const double* d_w = static_cast<const double*>(pv);
  if ((rc = device_input(y + t0, static_cast<size_t>(m) * 8, s, &t_y, &pv))) return rc;
  const double* d_y = static_cast<const double*>(pv);
  if ((rc = t_yhat.alloc(static_cast<size_t>(m) * 8)) || (rc = t_out.alloc(16))) return rc;
  double* d_yhat = static_cast<double*>(t_yhat.p);
  double* d_out = static_cast<double*>(t_out.p);
  if ((rc = readout_predict_dev(d_rows, m, N, d_w, d_yhat, s))) return rc;
  sto::readout::nmse_kernel<<<1, 1024, 0, s>>>(d_yhat, d_y, 0, m, d_out);
  STO_CUDA(cudaGetLastError());
  double h[2] = {0.0, 0.0};
  STO_CUDA(cudaMemcpyAsync(h, d_out, sizeof(h), cudaMemcpyDeviceToHost, s));
  STO_CUDA(cudaStreamSynchronize(s));
  if (!(h[1] > 0.0)) return STO_EINVAL;  // a constant target has no normalised error
  *nmse = h[0] / h[1];
  return STO_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- row shards
//
// One row block of a reservoir split across GPUs (shard.cuh).  The handle
// owns, on the device current at creation, the block's rows of W (padded to
// a multiple of 4 columns), its input weights, its double-float state and
// input field.  Stages are launched one at a time by the caller, who
// exchanges the stage values between launches.

struct sto_shard {
  int device = 0;
  cudaStream_t stream = nullptr;
  int64_t N = 0, row0 = 0, rows = 0, ld = 0;
  sto_params params{};
  float* d_W = nullptr;
  float* d_win = nullptr;
  float2* d_st = nullptr;  // mn | ms | ks ([3][rows] each), hin [rows]
  int* d_flag = nullptr;
  sto::ShardArgs args{};
};

namespace {

void free_shard(sto_shard* h) {
  if (!h) return;
  cudaFree(h->d_W);
  cudaFree(h->d_win);
  cudaFree(h->d_st);
  cudaFree(h->d_flag);
  delete h;
}

int shard_set_state_host(sto_shard* h, const double* m) {
  const int n = static_cast<int>(3 * h->rows);
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(m[i])) return STO_ENONFINITE;
  ScopedDev tmp;
  if (const int rc = tmp.alloc(static_cast<size_t>(n) * 8)) return rc;
  STO_CUDA(cudaMemcpyAsync(tmp.p, m, static_cast<size_t>(n) * 8, cudaMemcpyHostToDevice, h->stream));
  sto::shard_state_in_kernel<<<(n + 255) / 256, 256, 0, h->stream>>>(static_cast<const double*>(tmp.p), n,
                                                                      h->d_st);
  STO_CUDA(cudaGetLastError());
  STO_CUDA(cudaStreamSynchronize(h->stream));
  return STO_OK;
}

}  // namespace

extern "C" {

int sto_shard_create(int64_t N, int64_t row0, int64_t rows, const sto_params* params, const float* W_rows,
                     const float* w_in_rows, const float* m0_rows, void* stream, sto_shard** out) {
  if (!out) return STO_EINVAL;
  *out = nullptr;
  if (N < 1 || row0 < 0 || rows < 1 || row0 + rows > N || !W_rows || !w_in_rows) return STO_EINVAL;
  if (int rc = check_params(params)) return rc;
  if (N > (1LL << 24) || rows * N > (1LL << 34)) return STO_ENOTSUP;
  sto_shard* h = new (std::nothrow) sto_shard();
  if (!h) return STO_ENOMEM;
  h->N = N;
  h->row0 = row0;
  h->rows = rows;
  h->ld = (N + 3) / 4 * 4;
  h->params = *params;
  h->stream = static_cast<cudaStream_t>(stream);
  auto fail = [&](int code) {
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_shard(h);
    return code;
  };
  if (const cudaError_t e = cudaGetDevice(&h->device)) return fail(cuda_fail(e));
  const int n_in = params->n_in;
  const size_t w_elems = static_cast<size_t>(rows) * N, win_elems = static_cast<size_t>(rows) * n_in;
  if (cudaMalloc(&h->d_W, static_cast<size_t>(rows) * h->ld * 4) != cudaSuccess ||
      cudaMalloc(&h->d_win, win_elems * 4) != cudaSuccess ||
      cudaMalloc(&h->d_st, static_cast<size_t>(10) * rows * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&h->d_flag, 16) != cudaSuccess) {
    cudaGetLastError();
    return fail(STO_ENOMEM);
  }
  int rc;
  {
    ScopedDev tw;
    const void* pv = nullptr;
    if ((rc = device_input(W_rows, w_elems * 4, h->stream, &tw, &pv))) return fail(rc);
    const float* dW = static_cast<const float*>(pv);
    bool bad = false;
    if ((rc = readout_nonfinite(dW, static_cast<long long>(w_elems), nullptr, 0, h->stream, h->d_flag, &bad)))
      return fail(rc);
    if (bad) return fail(STO_ENONFINITE);
    const long long total = rows * h->ld;
    const unsigned blocks = static_cast<unsigned>((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192);
    sto::shard_pad_w_kernel<<<blocks, 256, 0, h->stream>>>(dW, static_cast<int>(rows), static_cast<int>(N),
                                                           static_cast<int>(h->ld), h->d_W);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e));
  }
  if (const cudaError_t e = cudaMemcpyAsync(h->d_win, w_in_rows, win_elems * 4, cudaMemcpyDefault, h->stream))
    return fail(cuda_fail(e));
  {
    bool bad = false;
    if ((rc = readout_nonfinite(h->d_win, static_cast<long long>(win_elems), nullptr, 0, h->stream, h->d_flag,
                                &bad)))
      return fail(rc);
    if (bad) return fail(STO_ENONFINITE);
  }
  std::vector<double> m(3 * static_cast<size_t>(rows));
  if (m0_rows) {
    std::vector<float> mf;
    if ((rc = fetch_floats(&mf, m0_rows, m.size(), h->stream))) return fail(rc);
    for (size_t i = 0; i < m.size(); ++i) m[i] = mf[i];
  } else {
    const double phi0 = 2.0 * M_PI / 360.0;  // Eq. (initial)
    for (int64_t k = 0; k < rows; ++k) {
      m[k] = std::sin(phi0) * std::cos(phi0);
      m[rows + k] = std::sin(phi0) * std::sin(phi0);
      m[2 * rows + k] = std::cos(phi0);
    }
  }
  if (const cudaError_t e = cudaMemsetAsync(h->d_st, 0, static_cast<size_t>(10) * rows * sizeof(float2), h->stream))
    return fail(cuda_fail(e));
  if ((rc = shard_set_state_host(h, m.data()))) return fail(rc);
  sto::ShardArgs& a = h->args;
  a.W = h->d_W;
  a.w_in = h->d_win;
  a.mn = h->d_st;
  a.ms = h->d_st + 3 * rows;
  a.ks = h->d_st + 6 * rows;
  a.hin = h->d_st + 9 * rows;
  a.N = static_cast<int>(N);
  a.ld = static_cast<int>(h->ld);
  a.rows = static_cast<int>(rows);
  a.n_in = n_in;
  a.comp = params->sample_component;
  set_constants(*params, &a.c);
  *out = h;
  return STO_OK;
}

int sto_shard_publish(sto_shard* h, float* x_rows) {
  if (!h || !x_rows || !is_device_ptr(x_rows)) return STO_EINVAL;
  const int rows = static_cast<int>(h->rows);
  sto::shard_publish_kernel<<<(rows + 255) / 256, 256, 0, h->stream>>>(h->d_st, rows, x_rows);
  return cuda_rc(cudaGetLastError());
}

int sto_shard_stage(sto_shard* h, const float* x, int32_t stage, const float* u_t, int32_t flags, float* x_next,
                    float* states_row) {
  if (!h || !x || !x_next || stage < 0 || stage > 3 || (flags & ~3) != 0) return STO_EINVAL;
  if ((flags & sto::kShardSampleStart) && (!u_t || stage != 0)) return STO_EINVAL;
  if ((flags & sto::kShardSampleEnd) && stage != 3) return STO_EINVAL;
  if ((reinterpret_cast<uintptr_t>(x) & 15u) != 0) return STO_EINVAL;
  if (!is_device_ptr(x) || !is_device_ptr(x_next) || (u_t && !is_device_ptr(u_t)) ||
      (states_row && !is_device_ptr(states_row)))
    return STO_EINVAL;
  const unsigned blocks = static_cast<unsigned>((h->rows + 7) / 8);
  sto::shard_stage_kernel<<<blocks, 256, 0, h->stream>>>(h->args, x, stage, u_t, flags, x_next, states_row);
  return cuda_rc(cudaGetLastError());
}

int sto_shard_set_state_f64(sto_shard* h, const double* m) {
  if (!h || !m) return STO_EINVAL;
  std::vector<double> md(3 * static_cast<size_t>(h->rows));
  STO_CUDA(cudaMemcpyAsync(md.data(), m, md.size() * 8, cudaMemcpyDefault, h->stream));
  STO_CUDA(cudaStreamSynchronize(h->stream));
  return shard_set_state_host(h, md.data());
}

int sto_shard_get_state_f64(const sto_shard* h, double* m) {
  if (!h || !m) return STO_EINVAL;
  const int n = static_cast<int>(3 * h->rows);
  ScopedDev tmp;
  if (const int rc = tmp.alloc(static_cast<size_t>(n) * 8)) return rc;
  sto::shard_state_out_kernel<<<(n + 255) / 256, 256, 0, h->stream>>>(h->d_st, n, static_cast<double*>(tmp.p));
  STO_CUDA(cudaGetLastError());
  STO_CUDA(cudaMemcpyAsync(m, tmp.p, static_cast<size_t>(n) * 8, cudaMemcpyDefault, h->stream));
  STO_CUDA(cudaStreamSynchronize(h->stream));
  return STO_OK;
}

void sto_shard_destroy(sto_shard* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  free_shard(h);
}

}  // extern "C"

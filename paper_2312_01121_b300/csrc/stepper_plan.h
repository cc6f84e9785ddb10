// Launch plan of the stepper (sto_persistent_kernel, sto_group_kernel): how
// many CTAs, how the W panels ring through shared memory, and which part of
// W the L2 keeps.  Together with sto_kernel.cuh this decides the kernel's
// memory traffic; the benchmark's recorded DRAM bytes are tied to these files.
#pragma once

#include <cstddef>
#include <cstdint>

#include "sto.h"
#include "sto_kernel.cuh"

namespace {

struct Plan {
  int G = 1, R_max = 1, P = 1, ns = 1, resident = 1, rpw = 1;
  int regw = 0;  // W in registers (FP32 coupling, on chip, <= 16 rows, several CTAs, N <= 1344)
  int tmem = 0;  // streamed FP32 W: the last panels of each row block held in tensor memory
  size_t smem = 0;
};

// W elements per 512-byte panel row and bytes per element of a coupling mode.
int panel_cols(int wmode) { return wmode == sto::kWf32 ? sto::kPanelCols : sto::kPanelCols / 2; }
int w_elem_bytes(int wmode) { return wmode == sto::kWf32 ? 4 : 8; }

// Dynamic shared memory of the stepper for a plan with `ns` ring slots
// (ns == P: W held on chip).
size_t smem_bytes(int R_max, int P, int ns, int wmode = sto::kWf32) {
  size_t b = static_cast<size_t>(ns) * R_max * sto::kPanelCols * 4;  // ring
  b += static_cast<size_t>(P) * sto::kPanelCols * 4;                 // xs
  b += static_cast<size_t>((R_max + 3) & ~3) * (wmode == sto::kWf32 ? 4 : 8);  // hs
  if (wmode == sto::kWf32 && ns == P && R_max <= sto::kColSplitRows)
    b += static_cast<size_t>(sto::kConsWarps) * sto::kColSplitRows * 4;  // column-split partials
  b += static_cast<size_t>(2 * ns) * 8 + 16;                         // barriers, abort flag
  return b;
}

// Choose the CTA count, panel ring and residency for N oscillators.
int make_plan(int64_t N, int grid_req, int sm_count, size_t smem_max, Plan* out,
              int wmode = sto::kWf32) {
  Plan p;
  const int cols = panel_cols(wmode);
  p.P = static_cast<int>((N + cols - 1) / cols);
  auto fill = [&](int G) -> bool {
    p.G = G;
    p.R_max = static_cast<int>((N + G - 1) / G);
    if (p.R_max > sto::kConsWarps * sto::kMaxRowsPerWarp) return false;
    p.rpw = (p.R_max + sto::kConsWarps - 1) / sto::kConsWarps;
    if (smem_bytes(p.R_max, p.P, p.P, wmode) <= smem_max) {
      p.resident = 1;
      p.ns = p.P;
    } else {
      p.resident = 0;
      const size_t fixed = smem_bytes(p.R_max, p.P, 0, wmode);
      const size_t per = static_cast<size_t>(p.R_max) * sto::kPanelCols * 4 + 16;
      if (fixed >= smem_max) return false;
      p.ns = static_cast<int>((smem_max - fixed) / per);
      if (p.ns > 8) p.ns = 8;
      if (p.ns < 2) return false;
    }
    p.smem = smem_bytes(p.R_max, p.P, p.ns, wmode);
    p.regw = (wmode == sto::kWf32 && p.resident && G > 1 && p.R_max <= sto::kColSplitRows &&
              N <= sto::kRegMaxN) ? 1 : 0;
    return p.smem <= smem_max;
  };
  if (grid_req > 0) {
    if (grid_req > sm_count || grid_req > N) return STO_EINVAL;
    if (!fill(grid_req)) return STO_ENOTSUP;
  } else if (fill(1) && p.resident) {
    // the whole W fits in one CTA: no inter-CTA exchange at all
  } else {
    // W on chip: latency-bound, and fewer CTAs mean less skew in the m^x
    // exchange; about 16 rows per CTA measured best at N = 10^3 (2.75 vs
    // 3.46 us per stage with 148 CTAs).  Otherwise stream with every SM.
    const int Gmax = static_cast<int>(N < sm_count ? N : sm_count);
    int G = static_cast<int>((N + 15) / 16);
    if (G > Gmax) G = Gmax;
    while (G < Gmax && !(fill(G) && p.resident)) ++G;
    if (!fill(G)) return STO_ENOTSUP;
  }
  *out = p;
  return STO_OK;
}

// W of at most 96 MB (three quarters of the 126 MB L2) is streamed with an
// evict_last hint so that it is re-read from L2 every stage; larger W is
// streamed from HBM with evict_first so that it does not flush the rest.
int l2_keeps(int64_t N, int ebytes = 4) {
  return static_cast<double>(ebytes) * static_cast<double>(N) * N <= 96.0 * (1 << 20) ? 1 : 0;
}

// Leading panels of every row block to keep L2-resident when W is larger
// than L2: a `mb` megabyte slice of W (default 110 MB of the 126 MB L2; with
// the panel order reversed on odd stages, measured best among 0-110 MB at
// N = 10^4).
int keep_panels(int64_t N, int P, int mb, int ebytes = 4) {
  if (mb < 0 || l2_keeps(N, ebytes)) return 0;
  const double budget = (mb == 0 ? 110.0 : static_cast<double>(mb)) * (1 << 20);
  const double wbytes = static_cast<double>(ebytes) * static_cast<double>(N) * N;
  const int k = static_cast<int>(P * budget / wbytes);
  return k < P ? k : P;
}

}  // namespace

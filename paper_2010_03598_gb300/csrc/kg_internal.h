// Internal structures shared by the host library and the device kernels.
#pragma once

#include <cstddef>
#include <cstdint>

namespace kg {

constexpr int kMaxM = 32;          // largest Krylov basis (one warp holds T and c)
constexpr int kMaxL = 30;
constexpr int kNRed = 4;           // values per reduction slot
constexpr int kMaxCtas = 2048;     // reduction slots per group
constexpr size_t kAlign = 256;
constexpr int kIRing = 4;          // slots of the fixed-point sum ring (4 words each)
constexpr size_t kCtrlBytes = 256; // control block cleared before each launch: status words (0),
                                   // barrier counter (32), fixed-point sum ring (64)

// Scalars kept in the workspace (float64 unless stated).
enum ScalarIdx {
  kScBetaRe = 0, kScBetaIm = 1, kScErrMax = 2, kScNormFinal = 3, kScBreakdowns = 4,
  kScCount = 8
};

// Status words in the control block.
enum CtrlIdx { kCtrlStatus = 0, kCtrlAbort = 1 };

// Everything one evaluation kernel needs; passed by value as the kernel parameter.
struct EvalParams {
  // problem
  int L, N, m, t_bits;
  int grad_mode, hc_kind, hc_site, ckpt;
  unsigned long long hc_mask;
  double Jxy, Jz, hc_amp, dt, bd_tol;
  const double* u;          // [N]
  const double* psi0;       // [2D] complex128 interleaved
  const double* target;     // [2D] complex128 interleaved
  double* fid;              // [1]
  double* grad;             // [N] or null
  // workspace (vectors are complex64 or complex128 depending on the kernel)
  void* basis;              // m-1 vectors: Lanczos slots 1..m-1
  void* traj;               // psi storage: N+1 vectors, or checkpoints (see ckpt layout)
  void* seg;                // ckpt > 0: C+1 vectors (segment recompute + 2 forward temps)
  void* chi;                // 2 vectors (co-state ping-pong)
  void* wbuf;               // 2 vectors: W_k of the Lanczos recurrence (ping-pong)
  void* xbuf;               // 1 vector: tile-leaving part of H v_k (streaming variant)
  double* G;                // [N+1] overlaps
  double* nrm;              // [N+1] ||psi_j|| of the forward sweep
  double* Gi;               // [2N] G at the interior Gauss-Lobatto nodes (KG_GRAD_EXACT), or null
  void* tint;               // [2N] psi at the interior nodes of every slice (KG_GRAD_EXACT), or null
  double* scal;             // [kScCount]
  unsigned long long* bar;  // group barrier counter
  double* red;              // [2][red_stride][kNRed] reduction slots
  int red_stride;           // slots per parity (>= CTAs of the group)
  int* ctrl;                // [kCtrlStatus, kCtrlAbort]
  unsigned long long* iring;  // [kIRing][4] fixed-point group sums (zeroed before each launch), or null
  long long wait_limit_ns;
  int debug_fault;          // 1: CTA 0 skips its arrival at the first group barrier; 2: at the first Lanczos step's
  int reorth;               // full CGS2 re-orthogonalisation of every Lanczos step
  long long* prof;          // [8] phase cycles of CTA 0, or null
};

// Batched launch: CTA c runs items [item_off[c], item_off[c+1]) in order; item i evaluates
// problem `problem` as rank `rank` of a group of `size` CTAs with barrier counter bars[group]
// and reduction slots reds + group * kBatchRedPerGroup.
constexpr int kBatchMaxGroup = 64;
constexpr size_t kBatchRedPerGroup = (size_t)2 * kBatchMaxGroup * kNRed;

struct BatchItem {
  int problem, rank, size, group;
};

struct BatchParams {
  const EvalParams* probs;  // [B]
  const int* item_off;      // [ctas + 1]
  const BatchItem* items;
  unsigned long long* bars;  // [groups]
  double* reds;              // [groups][kBatchRedPerGroup]
  int* ctrl;                 // shared status word and abort flag
};

}  // namespace kg

// K-GRAPE evaluation kernel: forward Krylov sweep, target overlap, backward co-state
// sweep with per-slice gradient overlaps, all in one cooperative persistent launch.
//
// Work split.  The 2^L amplitudes are cut into tiles of 2^t contiguous amplitudes; CTA r
// of the group owns tiles r, r + G, r + 2G, ...  A thread owns amplitudes li = tid + j*NT
// (j < APT) of each of its CTA's tiles, so index bits >= log2(NT) are thread-local.
//
// Lanczos step k of a slice (App. A, Algorithm "Lanczos", in Paige's order), one group
// barrier per step:
//   v_k      = (W_k - alpha_{k-1} v_{k-1}) / b_k           own amplitudes, stored as basis slot k
//   H v_k    = diag v_k + (Jxy/2) sum_{bonds inside the tile} v_k[partner]   (shared memory)
//            + X_k                                                            (bonds leaving the tile)
//   X_k      = (sum_{bonds leaving the tile} wgt W_k[partner] - alpha_{k-1} X_{k-1}) / b_k
//   W_{k+1}  = H v_k - b_k v_{k-1}                          stored for the other tiles' partners
//   alpha_k  = <v_k|W_{k+1}>,  b_{k+1}^2 = ||W_{k+1}||^2 - 2 alpha_k <v_k|W_{k+1}> + alpha_k^2 ||v_k||^2
// X_k is the part of H v_k that couples to amplitudes of other tiles; the partner set of an
// amplitude is the same in every step, so X obeys the same two-term recurrence as v and
// only W's partners are read.  alpha and b come out of one reduction.  After m steps every
// CTA forms c = exp(-i sigma dt T) e_1 (one warp, FP64) and recombines
// psi' = ||psi|| sum_k c_k v_k for its own tiles (App. A).
//
// Resident variant (RES): every CTA owns at most TPC tiles; W and X of its amplitudes stay on
// chip (registers and shared memory; tensor memory in the complex64 full-tile loop) and v_k,
// v_{k-1} of its tiles in shared memory for the whole slice.  Streaming variant: one tile at
// a time, W from the global W buffer, X from a global scratch vector, v_{k-1} from the basis.
#include <cuda_runtime.h>

#include "kg_device.cuh"
#include "kg_launch.h"

namespace kg {

enum ExtraKind { kExtraNone = 0, kExtraOverlapTarget = 1, kExtraGradOverlap = 2 };

constexpr int kLogNT = 9;  // log2(kThreads)
// Lanczos loop of a kernel: generic (any tile, complex64 or complex128), complex64 resident
// (4096-amplitude tiles, two per CTA, on chip), complex64 streaming (4096-amplitude tiles
// that do not stay on chip).
enum { kModeGeneric = 0, kModeResident64 = 1, kModeStream64 = 2, kModeResident64b = 3 };
static_assert((1 << kLogNT) == kThreads, "kLogNT must match kThreads");

constexpr int kSlotRanks = 256;  // groups up to this size prefetch their reduction slots
constexpr int kLzStages = 4;
// complex64 streaming path: per-thread copy ring of kStrDepth blocks (4 granules of 16 B per
// thread each) behind two tiles of v_k for the stencil
constexpr int kStrDepth = 4;
constexpr int kStrSvBufs = 2;  // tiles of v_k for the stencil (1: one more barrier per tile)
constexpr size_t kStrSmemBytes = (size_t)kStrSvBufs * 4096 * 8 + (size_t)kStrDepth * 4 * 512 * 16;    // Lanczos partner ring: 4 x 32 KB behind the 64 KB of v_k
constexpr int kLzMaxChunks = 2 * (1 + (kMaxL - 13) + 1);  // two tiles: bond 11, outer bonds, Sx site
// Headline loop (lanczos_res64b): partner blocks stream through a per-thread ring of kPrRing units
// in the shared memory behind W_k (64 KB) and the diagonal (32 KB); a unit is two 16-byte granules
// per thread, 16 KB per CTA.  A whole-tile table entry is two units, a half entry one.
constexpr int kPrRing = 5;
constexpr int kLzMaxUnits = 2 * kLzMaxChunks;
// Dynamic shared memory of the headline kernel: the Lanczos loop's W_k, diagonal and partner ring,
// or the recombination's kRecombDepth (3) basis vectors of 64 KB, whichever is larger.
constexpr size_t kRes64bSmemBytes = ((size_t)96 + (size_t)kPrRing * 16 > (size_t)3 * 64)
                                        ? ((size_t)96 + (size_t)kPrRing * 16) * 1024
                                        : (size_t)3 * 64 * 1024;
constexpr uint32_t kTmemCols = 512;  // 128 columns per warp, 4 warps per lane quarter
// Headline loop (lanczos_res64b): 16 worker warps and the control warp (warp 16), which meet at
// named barriers -- kBarPost (workers arrive with a step's partial sums, the control warp waits),
// kBarGroup (the control warp arrives once the group barrier has passed) and kBarScal (it
// arrives once the next step's scalars are formed).  Barrier 1 is the workers' own (wsync).
constexpr int kCtlThreads = kThreads + 32;
enum { kBarPost = 2, kBarGroup = 3, kBarScal = 4 };
constexpr int kCtlLast = 1 << 16;  // ctl_cmd flag: the slice's last step
constexpr int kCtlExit = -1;       // ctl_cmd: the evaluation is over
static_assert(kThreads == kWorkMax, "worker threads of a block");

// What the complex64 resident loop reads in its steps, per CTA (shared memory).
struct ResCtx {
  size_t tbase[2];   // own tiles' first amplitude
  float2* basis;     // basis slot 1 (slot k at basis + (k - 1) D)
  size_t D;
  float2* sw;        // W_k of the own tiles (shared memory)
  float2* ring;      // partner-block ring (shared memory); the headline loop: the diagonal of H_j
  float4* pring;     // the headline loop's partner ring (shared memory)
  unsigned maskL1, mk;
  int L1, hs, hcsx, n_own, m;
  float hxy, qz, cusx, cusz, amax, bmax, bdtol;
  float fscale, finv;  // fixed-point scale 2^S of the slice's group sums, and 2^-S
};

struct SmemSlice {
  SmemRed red;
  double alpha[kMaxM];
  double beta[kMaxM + 1];
  double coef_re[kMaxM];
  double coef_im[kMaxM];
  float coef_re_f[kMaxM];
  float coef_im_f[kMaxM];
  float alpha_f[kMaxM];
  float beta_f[kMaxM + 1];
  double err;
  // scalars of the Lanczos recurrence, formed once per CTA by thread 0 and broadcast
  double s_ap, s_ib, s_bk, s_alpha, s_b2, beta_m, nrm_out, s_ib0;
  float f_ap, f_ib, f_bk, f_alpha, f_ib0, f_bk0, f_beta_m;
  int code1, stop, meff, broke;
  double rco_re[kMaxM], rco_im[kMaxM];  // re-orthogonalisation coefficients <v_i|r>
  // resident complex64 path: the Lanczos step's ring of partner-tile copies, its chunk table,
  // the float-float sums of every step (for the FP64 tridiagonal), the TMEM address
  unsigned long long lmbar[kLzStages];
  unsigned ctab[kLzMaxChunks];
  unsigned utab[kLzMaxUnits];  // headline loop: units of the partner ring (build_unit_table)
  int n_units, n_units0;  // units of both own tiles, and of tile 0 (they come first)
  int ct_start[3];
  int first;  // the own tile computed first (more partner blocks)
  long long prof_last, prof_acc[8];  // phase timing (thread 0 of CTA 0)
  ResCtx r;   // the resident loop's per-slice constants
  Group grp;  // the group's barrier state while the resident loop runs (written by thread 0)
  float2 ff_a[kMaxM], ff_n[kMaxM], ff_q[kMaxM], ff_e[kMaxM];
  float4 slotbuf[2 * kSlotRanks];  // the group's reduction slots, prefetched by warp 0
  int recomb_pre;  // the Lanczos loop has issued the recombination's first copies (complex64)
  int ctl_cmd;  // control warp: the step whose sums were handed over (| kCtlLast), or kCtlExit
  int ctl_ok;   // control warp: the group barrier passed (0: aborted or timed out)
  unsigned ff_e_set;
  uint32_t tmem_base;
};

template <class R> __device__ __forceinline__ R pick_r(double d, float f);
template <> __device__ __forceinline__ float pick_r<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double pick_r<double>(double d, float) { return d; }

// Thread 0: start of a slice's Lanczos loop with ||psi|| = nrm (alpha_{-1} = 0, b_0 = nrm).
__device__ __forceinline__ void lz_init(SmemSlice& ss, double nrm, int m) {
  const double inv = (nrm > 0.0) ? 1.0 / nrm : 0.0;
  ss.s_ap = 0.0;
  ss.s_ib = inv;
  ss.s_bk = nrm;
  ss.f_ap = 0.f;
  ss.f_ib = (float)inv;
  ss.f_bk = (float)nrm;
  ss.s_ib0 = inv;
  ss.f_ib0 = (float)inv;
  ss.f_bk0 = ss.f_bk;
  ss.f_beta_m = 0.f;
  ss.meff = (nrm > 0.0) ? m : 0;
  ss.broke = 0;
  ss.beta_m = 0.0;
}

// Thread 0, after the reduction of step k (out = <v|W>, ||W||^2, ||v||^2): alpha_k and
// b_{k+1}^2 = ||W||^2 - 2 alpha <v|W> + alpha^2 ||v||^2.  code1: 0 go on, 1 the identity
// cancels (near an invariant subspace: form ||W - alpha v||^2 explicitly), 2 non-finite.
__device__ __forceinline__ void lz_after_reduce(SmemSlice& ss, int k, bool last, const double (&out)[3]) {
  const double alpha = out[0];
  ss.alpha[k] = alpha;
  ss.s_alpha = alpha;
  ss.f_alpha = (float)alpha;
  ss.alpha_f[k] = ss.f_alpha;
  ss.s_b2 = out[1] - 2.0 * alpha * alpha + alpha * alpha * out[2];
  int code = 0;
  if (!isfinite(alpha) || !isfinite(out[1])) code = 2;
  else if (!last && ss.s_b2 < 1e-3 * out[1]) code = 1;
  ss.code1 = code;
}

// Thread 0: b_{k+1}, the breakdown test of Alg. "Lanczos" (b_j > 0, with a tolerance), and
// the scalars of step k+1.  stop = 1 after the last step or a breakdown.
__device__ __forceinline__ void lz_finish_step(SmemSlice& ss, int k, bool last, double bd_tol, double& amax,
                                               double& bmax) {
  const double b2 = fmax(ss.s_b2, 0.0);
  const double rb = (b2 > 0.0) ? rsqrt(b2) : 0.0;  // 1 / b_{k+1}
  const double beta = b2 * rb;
  const double alpha = ss.s_alpha;
  int stop = 0;
  if (last) {
    ss.beta_m = beta;
    ss.f_beta_m = (float)beta;
    stop = 1;
  } else {
    amax = fmax(amax, fabs(alpha));
    if (beta <= bd_tol * fmax(1.0, amax + bmax)) {
      ss.meff = k + 1;
      ss.broke = 1;
      stop = 1;
    } else {
      bmax = fmax(bmax, beta);
      ss.beta[k + 1] = beta;
      const double inv = rb;
      ss.s_ap = alpha;
      ss.s_ib = inv;
      ss.s_bk = beta;
      ss.f_ap = (float)alpha;
      ss.f_ib = (float)inv;
      ss.f_bk = (float)beta;
      ss.beta_f[k + 1] = ss.f_bk;
    }
  }
  ss.stop = stop;
}

__device__ __forceinline__ void flag_nonfinite(const EvalParams& p) {
  atomicCAS(p.ctrl + kCtrlStatus, 0, (int)KG_ERR_NONFINITE);
  atomicExch(p.ctrl + kCtrlAbort, 1);
}

// Wait for phase `parity` of a bulk-copy barrier, at most `limit_ns`; false on time-out (the
// status word then holds KG_ERR_TIMEOUT and the group is told to stop).
__device__ __forceinline__ bool mbar_wait_bounded(const EvalParams& p, unsigned long long* bar, uint32_t parity) {
  unsigned long long t0 = 0;
  for (unsigned it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u) {
      const unsigned long long now = globaltimer_ns();
      if (t0 == 0) {
        t0 = now;
      } else if ((long long)(now - t0) > p.wait_limit_ns) {
        atomicCAS(p.ctrl + kCtrlStatus, 0, (int)KG_ERR_TIMEOUT);
        atomicExch(p.ctrl + kCtrlAbort, 1);
        return false;
      }
    }
  }
}

// Phase timing (thread 0 of CTA 0): cycles since the previous mark go to counter `phase`.
__device__ __forceinline__ void prof_mark(SmemSlice& ss, int phase) {
  const long long now = clock64();
  ss.prof_acc[phase] += now - ss.prof_last;
  ss.prof_last = now;
}

template <class V>
struct Ctx {
  using R = typename VecTraits<V>::R;
  const EvalParams* p;
  Group g;
  SmemSlice* ss;
  V* sv[2];         // shared memory: v_k and v_{k-1} of the own tiles ([TPC][tile] each)
  V* sx;            // shared memory (resident variant): X of the own tiles ([TPC][tile])
  int t, tile, ntiles, n_own;
  bool paired;      // tiles go to CTAs in pairs (2p, 2p ^ alt), pair p to CTA p mod size (equal cross-tile work)
  unsigned alt;     // alternating bits 0, 2, 4, ... of the tile index
  size_t D;
  unsigned maskL1;  // bonds 0..L-2 in (i ^ i>>1)
  double err_max;
  int breakdowns;
  unsigned lz_count;     // Lanczos partner bulk copies consumed so far (complex64 resident path)
  uint32_t tm;           // this warp's TMEM address: its lane quarter, its 128-column group
  bool prof_on;          // phase timing (CTA 0, thread 0; the counters are in shared memory)

  __device__ __forceinline__ void mark(int phase) {
    if (prof_on && threadIdx.x == 0) prof_mark(*ss, phase);
  }
  __device__ V* basis_slot(int k) const { return (V*)p->basis + (size_t)(k - 1) * D; }
  __device__ V* wbuf(int k) const { return (V*)p->wbuf + (size_t)(k & 1) * D; }
  // Tile owned as number c.  Paired: flipping every other tile-index bit toggles whether
  // each adjacent pair of tile bits differs, so the two tiles of a CTA together have the
  // same number of tile-uniform antiparallel bonds (cross-tile partner tiles) as any other pair.
  __device__ size_t tile_base(int c) const {
    if (paired) {
      const unsigned T0 = 2u * (unsigned)(g.rank + (c >> 1) * g.size);
      return (size_t)((c & 1) ? (T0 ^ alt) : T0) << t;
    }
    return (size_t)(g.rank + c * g.size) << t;
  }
};

template <class V>
__device__ __forceinline__ V vzero() { return vmake<V>(0, 0); }

// Bonds (and the Sx control) that leave the tile: acc[j] += wgt * src[partner] for the own
// amplitudes of the tile at `base`.  The partner set depends only on the amplitude index.
template <class V, int APT>
__device__ __forceinline__ void add_cross(const Ctx<V>& c, size_t base, const V* __restrict__ src,
                                          typename VecTraits<V>::R hxy, typename VecTraits<V>::R cu_sx,
                                          V (&acc)[APT]) {
  using R = typename VecTraits<V>::R;
  const EvalParams& p = *c.p;
  const int tid = threadIdx.x;
  const int L1 = p.L - 1;
  const int t = c.t;
  if (t - 1 >= 0 && t - 1 < L1) {  // bond t-1: bit t-1 inside the tile, bit t outside
    const int b = t - 1;
    const unsigned bt = (unsigned)((base >> t) & 1u);
#pragma unroll
    for (int j = 0; j < APT; ++j) {
      const int li = tid + j * kThreads;
      if (li < c.tile && ((unsigned)(li >> b) & 1u) != bt) {
        const V q = ldv(src + ((base + li) ^ ((size_t)3 << b)));
        acc[j].x += hxy * q.x;
        acc[j].y += hxy * q.y;
      }
    }
  }
  for (int b = t; b < L1; ++b) {  // bits b, b+1 both outside the tile: same for the whole tile
    if (((base >> b) ^ (base >> (b + 1))) & 1u) {
      const V* q0 = src + (base ^ ((size_t)3 << b));
      V q[APT];
#pragma unroll
      for (int j = 0; j < APT; ++j) {
        const int li = tid + j * kThreads;
        q[j] = (li < c.tile) ? ldv(q0 + li) : vzero<V>();
      }
#pragma unroll
      for (int j = 0; j < APT; ++j) {
        acc[j].x += hxy * q[j].x;
        acc[j].y += hxy * q[j].y;
      }
    }
  }
  if (p.hc_kind == KG_HC_SX_SITE && p.hc_site >= t) {
    const V* q0 = src + (base ^ ((size_t)1 << p.hc_site));
#pragma unroll
    for (int j = 0; j < APT; ++j) {
      const int li = tid + j * kThreads;
      if (li < c.tile) {
        const V q = ldv(q0 + li);
        acc[j].x += cu_sx * q.x;
        acc[j].y += cu_sx * q.y;
      }
    }
  }
}

// The part of H v that stays inside the tile, for the own amplitudes of one tile whose v is
// in shared memory `sv`:  hv = diag v + (Jxy/2) sum_{bonds inside the tile} v[partner] + Hc-term.  Bonds are the outer (runtime) loop and the thread's APT amplitudes the inner
// (unrolled) one, so every bond issues APT independent shared-memory loads.
template <class V, int APT>
__device__ __forceinline__ void apply_H_tile(const Ctx<V>& c, size_t base, const V* sv,
                                             typename VecTraits<V>::R hxy, typename VecTraits<V>::R qz,
                                             typename VecTraits<V>::R cu_sx, typename VecTraits<V>::R cu_sz,
                                             V (&hv)[APT]) {
  using R = typename VecTraits<V>::R;
  const EvalParams& p = *c.p;
  const int tid = threadIdx.x;
  const int tin = c.t - 1;  // bonds b < tin have both bits inside the tile
  const int T = c.tile;
#pragma unroll
  for (int j = 0; j < APT; ++j) hv[j] = vzero<V>();
  for (int b = 0; b < tin; ++b) {
#pragma unroll
    for (int j = 0; j < APT; ++j) {
      const int li = tid + j * kThreads;
      if (li < T && (((li >> b) ^ (li >> (b + 1))) & 1)) {
        const V q = sv[li ^ (3 << b)];
        hv[j].x += q.x;
        hv[j].y += q.y;
      }
    }
  }
  const unsigned mk = (unsigned)p.hc_mask;
#pragma unroll
  for (int j = 0; j < APT; ++j) {
    const int li = tid + j * kThreads;
    if (li >= T) continue;
    const unsigned gi = (unsigned)(base + li);
    const unsigned x = (gi ^ (gi >> 1)) & c.maskL1;  // bit b set <=> bits b, b+1 antiparallel
    R d = qz * (R)((p.L - 1) - 2 * __popc(x));
    if (p.hc_kind == KG_HC_SZ_SITES) d += cu_sz * (R)0.5 * (R)(__popc(mk) - 2 * __popc(gi & mk));
    const V v = sv[li];
    R wr = d * v.x + hxy * hv[j].x;
    R wi = d * v.y + hxy * hv[j].y;
    if (p.hc_kind == KG_HC_SX_SITE && p.hc_site < c.t) {
      const V q = sv[li ^ (1 << p.hc_site)];
      wr += cu_sx * q.x;
      wi += cu_sx * q.y;
    }
    hv[j] = vmake<V>(wr, wi);
  }
}

// Full re-orthogonalisation of step k (KG_FLAG_FULL_REORTH; App. A's remedy for the loss of
// orthogonality): the residual r, held in r_g for the own tiles (W_{k+1} on entry), loses its
// components on every basis vector v_0..v_k by classical Gram-Schmidt applied twice,
//   c_i = <v_i|r>,  r <- r - sum_i c_i v_i,
// then thread 0 records b_{k+1}^2 = ||r||^2.  v_0 is psi / ||psi|| (slot 0 holds psi itself),
// v_i (i >= 1) are the normalised basis slots.  Coefficients are reduced two vectors at a time.
template <class V, class A, int APT>
__device__ __noinline__ bool reorth_cgs2(Ctx<V>& c, int k, const V* src, V* r_g) {
  using R = typename VecTraits<V>::R;
  SmemSlice& ss = *c.ss;
  const int tid = threadIdx.x;
  const int T = c.tile;
  const R ib0 = pick_r<R>(ss.s_ib0, ss.f_ib0);
  for (int pass = 0; pass < 2; ++pass) {
    for (int i0 = 0; i0 <= k; i0 += 2) {
      A part[4] = {0, 0, 0, 0};
      for (int ct = 0; ct < c.n_own; ++ct) {
        const size_t base = c.tile_base(ct);
#pragma unroll
        for (int j = 0; j < APT; ++j) {
          const int li = tid + j * kThreads;
          if (li >= T) continue;
          const V rv = ldv(r_g + base + li);
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int i = i0 + u;
            if (i > k) break;
            V v = ldv(((i == 0) ? src : c.basis_slot(i)) + base + li);
            if (i == 0) v = vmake<V>(v.x * ib0, v.y * ib0);
            part[2 * u] += (A)(v.x * rv.x + v.y * rv.y);
            part[2 * u + 1] += (A)(v.x * rv.y - v.y * rv.x);
          }
        }
      }
      double out[4];
      if (!group_reduce<4>(c.g, ss.red, part, out)) return false;
      if (tid == 0) {
        ss.rco_re[i0] = out[0];
        ss.rco_im[i0] = out[1];
        if (i0 + 1 <= k) {
          ss.rco_re[i0 + 1] = out[2];
          ss.rco_im[i0 + 1] = out[3];
        }
      }
    }
    wsync();
    for (int ct = 0; ct < c.n_own; ++ct) {
      const size_t base = c.tile_base(ct);
#pragma unroll
      for (int j = 0; j < APT; ++j) {
        const int li = tid + j * kThreads;
        if (li >= T) continue;
        V rv = ldv(r_g + base + li);
        for (int i = 0; i <= k; ++i) {
          V v = ldv(((i == 0) ? src : c.basis_slot(i)) + base + li);
          if (i == 0) v = vmake<V>(v.x * ib0, v.y * ib0);
          const R a = (R)ss.rco_re[i], b = (R)ss.rco_im[i];
          rv.x -= a * v.x - b * v.y;
          rv.y -= a * v.y + b * v.x;
        }
        stv(r_g + base + li, rv);
      }
    }
  }
  A n2[1] = {0};
  for (int ct = 0; ct < c.n_own; ++ct) {
    const size_t base = c.tile_base(ct);
#pragma unroll
    for (int j = 0; j < APT; ++j) {
      const int li = tid + j * kThreads;
      if (li >= T) continue;
      const V rv = ldv(r_g + base + li);
      n2[0] += (A)(rv.x * rv.x + rv.y * rv.y);
    }
  }
  double o1[1];
  if (!group_reduce<1>(c.g, ss.red, n2, o1)) return false;
  if (tid == 0) ss.s_b2 = o1[0];
  return true;
}

template <class V, class A, int APT, int TPC, bool RES>
__device__ __forceinline__ bool lanczos_generic(Ctx<V>& c, const V* src, double nrm_src, double uj) {
  using R = typename VecTraits<V>::R;
  const EvalParams& p = *c.p;
  SmemSlice& ss = *c.ss;
  const int m = p.m;
  const int tid = threadIdx.x;
  const R hxy = (R)(0.5 * p.Jxy), qz = (R)(0.25 * p.Jz);
  const R cu_sx = (R)(0.5 * uj * p.hc_amp), cu_sz = (R)(uj * p.hc_amp);
  const int T = c.tile;
  constexpr int NB = RES ? TPC : 1;  // tiles held at once

  V W[NB][APT];                    // W_k of the own amplitudes (k = 0: the source vector psi)
  V X[RES ? 1 : NB][RES ? 1 : APT];  // streaming: part of H v_k leaving the tile (resident: in c.sx)
  double amax = 0.0, bmax = 0.0;     // thread 0: running maxima for the breakdown test
  if (tid == 0) lz_init(ss, nrm_src, m);
  wsync();
  if (ss.meff > 0) {
    for (int k = 0; k < m; ++k) {
      const bool last = (k == m - 1);
      const V* wsrc = (k == 0) ? src : c.wbuf(k);       // W_k (global, all tiles)
      V* wdst = last ? nullptr : c.wbuf(k + 1);          // W_{k+1}
      V* vslot = (k == 0) ? nullptr : c.basis_slot(k);  // v_k (normalised)
      const V* vprev_g = (k == 0) ? nullptr : ((k == 1) ? src : c.basis_slot(k - 1));
      const R ap = pick_r<R>(ss.s_ap, ss.f_ap);
      const R ib = pick_r<R>(ss.s_ib, ss.f_ib);
      const R bk = pick_r<R>(ss.s_bk, ss.f_bk);
      // slot 0 is psi itself (unnormalised): v_0 = psi * (1 / b_0); ib of step 1 is 1 / b_1
      const R vprev_scale = (k == 1) ? pick_r<R>(ss.s_ib0, ss.f_ib0) : (R)1;
      V* s_cur = c.sv[k & 1];
      V* s_prev = c.sv[(k & 1) ^ 1];
      A acc[3] = {0, 0, 0};
      for (int c0 = 0; c0 < c.n_own; c0 += NB) {
        // ---- stage 1: v_k of the own amplitudes, partners leaving the tile
#pragma unroll
        for (int cc = 0; cc < NB; ++cc) {
          const int ct = c0 + cc;
          if (ct >= c.n_own) break;
          const size_t base = c.tile_base(ct);
          V* sc = s_cur + (RES ? cc * T : 0);
          const V* sp = s_prev + (RES ? cc * T : 0);
          if (!RES || k == 0) {
#pragma unroll
            for (int j = 0; j < APT; ++j) {
              const int li = tid + j * kThreads;
              W[cc][j] = (li < T) ? ldv(wsrc + base + li) : vzero<V>();
            }
          }
          V xt[APT];  // X_{k-1}, then X_k
#pragma unroll
          for (int j = 0; j < APT; ++j) {
            const int li = tid + j * kThreads;
            if (k == 0 || li >= T) xt[j] = vzero<V>();
            else if (RES) xt[j] = c.sx[cc * T + li];
            else xt[j] = ldv((const V*)p.xbuf + base + li);
          }
#pragma unroll
          for (int j = 0; j < APT; ++j) {
            const int li = tid + j * kThreads;
            if (li >= T) continue;
            V v;
            if (k == 0) {
              v = vmake<V>(W[cc][j].x * ib, W[cc][j].y * ib);
            } else {
              V q;
              if (RES) {
                q = sp[li];  // normalised v_{k-1}
              } else {
                q = ldv(vprev_g + base + li);
                q.x *= vprev_scale;
                q.y *= vprev_scale;
              }
              v = vmake<V>((W[cc][j].x - ap * q.x) * ib, (W[cc][j].y - ap * q.y) * ib);
              stv(vslot + base + li, v);
            }
            sc[li] = v;
          }
          // X_k = (sum wgt W_k[partner] - alpha_{k-1} X_{k-1}) / b_k
#pragma unroll
          for (int j = 0; j < APT; ++j) xt[j] = vmake<V>(-ap * xt[j].x, -ap * xt[j].y);
          add_cross<V, APT>(c, base, wsrc, hxy, cu_sx, xt);
#pragma unroll
          for (int j = 0; j < APT; ++j) {
            const int li = tid + j * kThreads;
            const V x = vmake<V>(xt[j].x * ib, xt[j].y * ib);
            if constexpr (RES) {
              if (li < T) c.sx[cc * T + li] = x;
            } else {
              X[0][j] = x;
            }
          }
        }
        wsync();
        c.mark(0);
        // ---- stage 2: H v_k, W_{k+1} = H v_k - b_k v_{k-1}, partial sums
#pragma unroll
        for (int cc = 0; cc < NB; ++cc) {
          const int ct = c0 + cc;
          if (ct >= c.n_own) break;
          const size_t base = c.tile_base(ct);
          const V* sc = s_cur + (RES ? cc * T : 0);
          const V* sp = s_prev + (RES ? cc * T : 0);
          apply_H_tile<V, APT>(c, base, sc, hxy, qz, cu_sx, cu_sz, W[cc]);  // W <- (H v_k) inside the tile
#pragma unroll
          for (int j = 0; j < APT; ++j) {
            const int li = tid + j * kThreads;
            if (li >= T) continue;
            V w = W[cc][j];
            V x;
            if constexpr (RES) x = c.sx[cc * T + li];
            else x = X[0][j];
            w.x += x.x;
            w.y += x.y;
            if (k > 0) {
              V q;
              if (RES) {
                q = sp[li];
              } else {
                q = ldv(vprev_g + base + li);
                q.x *= vprev_scale;
                q.y *= vprev_scale;
              }
              w.x -= bk * q.x;
              w.y -= bk * q.y;
            }
            const V v = sc[li];
            acc[0] += (A)(v.x * w.x + v.y * w.y);
            acc[1] += (A)(w.x * w.x + w.y * w.y);
            acc[2] += (A)(v.x * v.x + v.y * v.y);
            W[cc][j] = w;
            if (!last) stv(wdst + base + li, w);
            if constexpr (!RES) stv((V*)p.xbuf + base + li, X[0][j]);
          }
        }
        if (!RES) wsync();
      }
      c.mark(1);
      double out[3];
      if (!group_reduce<3>(c.g, ss.red, acc, out)) return false;
      c.mark(2);
      if (tid == 0) lz_after_reduce(ss, k, last, out);
      wsync();
      const int code = ss.code1;
      if (code == 2) {
        if (tid == 0) flag_nonfinite(p);
        return false;
      }
      const bool reorth = !RES && p.reorth && !last;
      if (reorth) {  // the residual, orthogonalised against the whole basis, replaces W_{k+1}
        if constexpr (!RES)
          if (!reorth_cgs2<V, A, APT>(c, k, src, wdst)) return false;
      } else if (code == 1) {
        // Near an invariant subspace the identity loses the small b_{k+1} to cancellation:
        // form ||W_{k+1} - alpha_k v_k||^2 explicitly (one more reduction, rare).
        A n1[1] = {0};
        const R ra = pick_r<R>(ss.s_alpha, ss.f_alpha);
        for (int ct = 0; ct < c.n_own; ++ct) {
          const size_t base = c.tile_base(ct);
#pragma unroll
          for (int j = 0; j < APT; ++j) {
            const int li = tid + j * kThreads;
            if (li >= T) continue;
            const V w = ldv(wdst + base + li);
            V v;
            if (k == 0) v = vmake<V>(ldv(src + base + li).x * ib, ldv(src + base + li).y * ib);
            else v = ldv(vslot + base + li);
            const R rx = w.x - ra * v.x, ry = w.y - ra * v.y;
            n1[0] += (A)(rx * rx + ry * ry);
          }
        }
        double o1[1];
        if (!group_reduce<1>(c.g, ss.red, n1, o1)) return false;
        if (tid == 0) ss.s_b2 = o1[0];
      }
      if (tid == 0) {
        lz_finish_step(ss, k, last, p.bd_tol, amax, bmax);
        if (reorth) {  // W_{k+1} is the orthogonalised residual: v_{k+1} = W_{k+1} / b_{k+1}
          ss.s_ap = 0.0;
          ss.f_ap = 0.f;
        }
      }
      wsync();
      c.mark(3);
      if (ss.stop) break;
    }
  }
  return true;
}

// Store the recombined amplitudes y of one tile and add their contributions to ||dst||^2 and
// to the fused overlap (see finish_slice).
template <class V, class A, int APT>
__device__ __forceinline__ void recomb_finalize(const Ctx<V>& c, size_t base, const V (&y)[APT], V* dst, int extra,
                                                const V* psi_other, A& nacc, A& gacc, double& ex0, double& ex1) {
  using R = typename VecTraits<V>::R;
  const EvalParams& p = *c.p;
  const int tid = threadIdx.x;
#pragma unroll
  for (int j = 0; j < APT; ++j) {
    const int li = tid + j * kThreads;
    if (li >= c.tile) continue;
    const size_t gi = base + li;
    const R yr = y[j].x, yi = y[j].y;
    stv(dst + gi, y[j]);
    nacc += (A)(yr * yr + yi * yi);
    if (extra == kExtraOverlapTarget) {
      const double2 f = reinterpret_cast<const double2*>(p.target)[gi];
      ex0 += f.x * (double)yr + f.y * (double)yi;
      ex1 += f.x * (double)yi - f.y * (double)yr;
    } else if (extra == kExtraGradOverlap) {
      V q;
      if (p.hc_kind == KG_HC_SX_SITE) {
        q = ldv(psi_other + (gi ^ ((size_t)1 << p.hc_site)));
        const R h = pick_r<R>(0.5 * p.hc_amp, 0.5f * (float)p.hc_amp);
        q.x *= h;
        q.y *= h;
      } else {
        const unsigned mk = (unsigned)p.hc_mask;
        const int nz = __popc(mk) - 2 * __popc((unsigned)gi & mk);
        const R dz = pick_r<R>(p.hc_amp * 0.5 * (double)nz, (float)p.hc_amp * 0.5f * (float)nz);
        q = ldv(psi_other + gi);
        q.x *= dz;
        q.y *= dz;
      }
      gacc += (A)(yr * q.y - yi * q.x);  // Im(conj(y) q)
    }
  }
}

// Small exponential c = exp(-i tau T) e_1 and recombination dst = ||src|| sum_k c_k v_k of the
// own tiles (App. A), with fused ||dst||^2 and the optional overlap:
// extra == kExtraOverlapTarget: e = <f|dst> (f = target, complex128, FP64 sums);
// extra == kExtraGradOverlap:   e.x = Im <dst|Hc|psi_other>.
// Reads meff, broke and b_m of the Lanczos loop from shared memory.
// Recombination of the complex64 resident path: basis vectors in flight per thread.
constexpr int kRecombDepth = 3;  // 3 x 64 KB: all of the resident path's shared memory

// This thread's asynchronous copies of basis vector vk for the own tiles at rb[0..n_own):
// amplitude pairs 2 (tid + 512 g) + {0, 1}, g < 4, into stage st[(ct * 4 + g) * kThreads + tid].
// The basis is read once here: the copies carry an evict_first L2 policy (see l2_policy_first).
__device__ __forceinline__ void recomb_issue(const float2* vk, const size_t (&rb)[2], int n_own, float4* st) {
  const int tid = threadIdx.x;
  const unsigned long long pol = l2_policy_first();
#pragma unroll
  for (int ct = 0; ct < 2; ++ct) {
    if (ct < n_own) {
#pragma unroll
      for (int g = 0; g < 4; ++g)
        cp_async16_hint(st + (ct * 4 + g) * kThreads + tid, vk + rb[ct] + 2 * (size_t)(tid + g * kThreads), pol);
    }
  }
}

// What the recombination's fused overlaps need, read once per slice.
struct RecombConsts {
  const double2* target;
  unsigned mk;
  int sx_site;  // Sx control site, or -1 for an Sz-sites control
  float h_amp;
};

// One recombined amplitude y at global index gi: store it and add its contributions to
// ||dst||^2 and to the fused overlap (see recomb_finalize).
template <class A>
__device__ __forceinline__ void recomb_amp(const RecombConsts& rc, size_t gi, float2 y, float2* dst, int extra,
                                           const float2* psi_other, A& nacc, A& gacc, double& ex0, double& ex1) {
  stv_hint(dst + gi, y, l2_policy_first());
  nacc += (A)(y.x * y.x + y.y * y.y);
  if (extra == kExtraOverlapTarget) {
    const double2 f = rc.target[gi];
    ex0 += f.x * (double)y.x + f.y * (double)y.y;
    ex1 += f.x * (double)y.y - f.y * (double)y.x;
  } else if (extra == kExtraGradOverlap) {
    float2 q;
    if (rc.sx_site >= 0) {
      q = ldv(psi_other + (gi ^ ((size_t)1 << rc.sx_site)));
      const float h = 0.5f * rc.h_amp;
      q.x *= h;
      q.y *= h;
    } else {
      const int nz = __popc(rc.mk) - 2 * __popc((unsigned)gi & rc.mk);
      const float dz = rc.h_amp * 0.5f * (float)nz;
      q = ldv(psi_other + gi);
      q.x *= dz;
      q.y *= dz;
    }
    gacc += (A)(y.x * q.y - y.y * q.x);  // Im(conj(y) q)
  }
}

template <class V, class A, int APT, bool WBASIS>
__device__ __forceinline__ bool finish_slice(Ctx<V>& c, const V* src, double nrm_src, double tau, V* dst, int extra,
                                             const V* psi_other, double& nrm_dst, double2& e, bool interior = false) {
  using R = typename VecTraits<V>::R;
  const EvalParams& p = *c.p;
  SmemSlice& ss = *c.ss;
  const int tid = threadIdx.x;
  const int T = c.tile;
  const int meff = ss.meff;
  // Complex64 resident path: the recombination streams the own tiles' share of the basis
  // through the shared memory the Lanczos loop no longer needs, by per-thread asynchronous
  // copies (cp.async) kRecombDepth basis vectors deep.  Thread tid copies and combines the
  // amplitude pairs 2 (tid + 512 g) + {0, 1}, g < 4, of each own tile, so it waits only for
  // its own copies.  The first copies do not depend on c: they go out before the exponential.
  float4* stg = reinterpret_cast<float4*>(c.sv[0]);  // [kRecombDepth][2 tiles x 4][kThreads]
  size_t rb[2] = {0, 0};
  bool pre = false;
  if constexpr (WBASIS) {
    rb[0] = (c.n_own > 0) ? c.tile_base(0) : 0;
    rb[1] = (c.n_own > 1) ? c.tile_base(1) : 0;
    wsync();  // every thread is done with the Lanczos loop's shared memory
    pre = ss.recomb_pre != 0;  // the Lanczos loop has issued the first copies already
    if (tid >= 32 && !pre) {  // warp 0 issues its copies after the exponential
      for (int s = 0; s < kRecombDepth; ++s) {
        if (s < meff) {  // newest basis vector first (see the loop below)
          const int ks = meff - 1 - s;
          recomb_issue(ks == 0 ? src : c.basis_slot(ks), rb, c.n_own, stg + (size_t)s * 8 * kThreads);
        }
        cp_async_commit();
      }
    }
  }
  // ---- small exponential and recombination coefficients (warp 0, FP64)
  if (tid < 32) {
    const bool broke = ss.broke != 0;
    double cr = 0.0, ci = 0.0;
    float tnorm = 0.f;
    const double tol = (sizeof(R) == 4) ? 1e-13 : 1e-18;
    if (meff > 0) {
      if constexpr (sizeof(R) == 4)
        tridiag_expv_e1_ff(ss.alpha, ss.beta, ss.alpha_f, ss.beta_f, meff, tau, (float)tau, tol, cr, ci, tnorm);
      else
        tridiag_expv_e1(ss.alpha, ss.beta, ss.alpha_f, ss.beta_f, meff, tau, (float)tau, tol, cr, ci, tnorm);
    }
    if (tid < meff) {
      // basis slot 0 is psi itself (unnormalised); slots k >= 1 hold normalised v_k
      const double f = (tid == 0) ? 1.0 : nrm_src;
      ss.coef_re[tid] = cr * f;
      ss.coef_im[tid] = ci * f;
      ss.coef_re_f[tid] = (float)(cr * f);
      ss.coef_im_f[tid] = (float)(ci * f);
    }
    if (tid == meff - 1) {
      // a-posteriori indicator ||psi|| b_m |c_{m-1}| (= b_m |coef_{m-1}| for m > 1), in FP32;
      // where the Taylor series stopped before index m-1, ||psi|| b_m ||tau T||^(m-1)/(m-1)!
      // bounds it instead
      float cm = sqrtf(ss.coef_re_f[tid] * ss.coef_re_f[tid] + ss.coef_im_f[tid] * ss.coef_im_f[tid]);
      if (tid == 0) cm *= ss.f_bk0;
      if (cm == 0.f && !broke) {
        cm = ss.f_bk0;
        for (int i = 1; i < meff; ++i) cm *= tnorm * kInvFF[i].x;  // / i
      }
      const float err = broke ? 0.f : ss.f_beta_m * cm;
      if (!interior) c.err_max = fmax(c.err_max, (double)err);  // lane meff-1 of warp 0 keeps the maximum
    }
    if constexpr (WBASIS) {
      // Slots k >= 1 hold W_k with v_k = (W_k - alpha_{k-1} v_{k-1}) / b_k, v_0 = psi/||psi||:
      // ||psi|| sum_k c_k v_k = sum_k e_k W_k + (s_0/||psi||) psi, where, from the top,
      // s_{m-1} = ||psi|| c_{m-1}, e_k = s_k / b_k, s_{k-1} = ||psi|| c_{k-1} - e_k alpha_{k-1}.
      // FP32 suffices: the coefficients only combine complex64 vectors.
      // Lane k holds ||psi|| c_k (s_k once the lanes above have passed e_{k+1} down); the
      // recurrence runs down the lanes, one shuffle per step.
      __syncwarp();
      if (meff > 1) {
        const bool own = tid < meff;
        float sr = own ? ss.coef_re_f[tid] : 0.f, si = own ? ss.coef_im_f[tid] : 0.f;
        const float ib = (own && tid >= 1) ? 1.f / ss.beta_f[tid] : 0.f;
        const float al = own ? ss.alpha_f[tid] : 0.f;  // alpha_k on lane k
        for (int k = meff - 1; k >= 1; --k) {
          const float er = sr * ib, ei = si * ib;  // e_k on lane k
          const float erb = __shfl_sync(0xffffffffu, er, k), eib = __shfl_sync(0xffffffffu, ei, k);
          if (tid == k) {
            ss.coef_re_f[k] = er;
            ss.coef_im_f[k] = ei;
          } else if (tid == k - 1) {
            if (k >= 2) {
              sr = sr - erb * al;  // ||psi|| c_{k-1} - e_k alpha_{k-1}
              si = si - eib * al;
            } else {
              // psi coefficient s_0 / ||psi|| = c_0 - e_1 alpha_0 / ||psi|| (slot 0 held c_0)
              ss.coef_re_f[0] = sr - erb * al * ss.f_ib0;
              ss.coef_im_f[0] = si - eib * al * ss.f_ib0;
            }
          }
        }
      }
      for (int s = 0; s < kRecombDepth && !pre; ++s) {
        if (s < meff) {  // newest basis vector first (see the loop below)
          const int ks = meff - 1 - s;
          recomb_issue(ks == 0 ? src : c.basis_slot(ks), rb, c.n_own, stg + (size_t)s * 8 * kThreads);
        }
        cp_async_commit();
      }
    }
  }
  wsync();
  if (WBASIS && tid == 0) ss.recomb_pre = 0;  // every thread has read it
  c.mark(4);
  if (tid == 0 && meff > 0 && !interior) c.breakdowns += ss.broke ? 1 : 0;
  // ---- recombination dst = sum_k coef_k (basis slot k) (+ fused norms / overlaps)
  A nacc = 0, gacc = 0;
  double ex0 = 0.0, ex1 = 0.0;
  if constexpr (WBASIS) {
    float4 y[2][4];
#pragma unroll
    for (int ct = 0; ct < 2; ++ct)
#pragma unroll
      for (int g = 0; g < 4; ++g) y[ct][g] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int n_own = c.n_own;
    const size_t D = c.D;
    const float2* slot1 = (const float2*)p.basis;  // basis slot k at slot1 + (k - 1) D
    // The basis vectors are read newest first: the slice has just written all m of them (8 MB
    // each at L=20) and L2 still holds the latest ones, while in order of age every read would
    // evict the next vector needed before it is reached.
    for (int i = 0; i < meff; ++i) {
      cp_async_wait<kRecombDepth - 1>();  // this thread's copies of basis vector k have landed
      const int k = meff - 1 - i;
      const float a = ss.coef_re_f[k], b = ss.coef_im_f[k];
      const float4* q = stg + (size_t)(i % kRecombDepth) * 8 * kThreads + tid;
#pragma unroll
      for (int ct = 0; ct < 2; ++ct) {
        if (ct < n_own) {
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            const float4 w = q[(ct * 4 + g) * kThreads];
            y[ct][g].x += a * w.x - b * w.y;
            y[ct][g].y += a * w.y + b * w.x;
            y[ct][g].z += a * w.z - b * w.w;
            y[ct][g].w += a * w.w + b * w.z;
          }
        }
      }
      if (i + kRecombDepth < meff) {
        const int kn = meff - 1 - (i + kRecombDepth);
        recomb_issue(kn == 0 ? (const float2*)src : slot1 + (size_t)(kn - 1) * D, rb, n_own,
                     stg + (size_t)(i % kRecombDepth) * 8 * kThreads);
      }
      cp_async_commit();
    }
    cp_async_wait<0>();
    RecombConsts rc;
    rc.target = reinterpret_cast<const double2*>(p.target);
    rc.mk = (unsigned)p.hc_mask;
    rc.sx_site = (p.hc_kind == KG_HC_SX_SITE) ? p.hc_site : -1;
    rc.h_amp = (float)p.hc_amp;
    for (int ct = 0; ct < n_own; ++ct) {
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const size_t gi = rb[ct] + 2 * (size_t)(tid + g * kThreads);
        recomb_amp<A>(rc, gi, make_float2(y[ct][g].x, y[ct][g].y), dst, extra, psi_other, nacc, gacc, ex0, ex1);
        recomb_amp<A>(rc, gi + 1, make_float2(y[ct][g].z, y[ct][g].w), dst, extra, psi_other, nacc, gacc, ex0, ex1);
      }
    }
  } else {
    for (int ct = 0; ct < c.n_own; ++ct) {
      const size_t base = c.tile_base(ct);
      V y[APT];
#pragma unroll
      for (int j = 0; j < APT; ++j) y[j] = vzero<V>();
      int k = 0;
      for (; k + 2 <= meff; k += 2) {  // two basis vectors in flight
        V q[2][APT];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const V* s = (k + u == 0) ? src : c.basis_slot(k + u);
#pragma unroll
          for (int j = 0; j < APT; ++j) {
            const int li = tid + j * kThreads;
            q[u][j] = (li < T) ? ldv(s + base + li) : vzero<V>();
          }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const R a = pick_r<R>(ss.coef_re[k + u], ss.coef_re_f[k + u]);
          const R b = pick_r<R>(ss.coef_im[k + u], ss.coef_im_f[k + u]);
#pragma unroll
          for (int j = 0; j < APT; ++j) {
            y[j].x += a * q[u][j].x - b * q[u][j].y;
            y[j].y += a * q[u][j].y + b * q[u][j].x;
          }
        }
      }
      for (; k < meff; ++k) {
        const V* s = (k == 0) ? src : c.basis_slot(k);
        const R a = pick_r<R>(ss.coef_re[k], ss.coef_re_f[k]), b = pick_r<R>(ss.coef_im[k], ss.coef_im_f[k]);
        V q[APT];
#pragma unroll
        for (int j = 0; j < APT; ++j) {
          const int li = tid + j * kThreads;
          q[j] = (li < T) ? ldv(s + base + li) : vzero<V>();
        }
#pragma unroll
        for (int j = 0; j < APT; ++j) {
          y[j].x += a * q[j].x - b * q[j].y;
          y[j].y += a * q[j].y + b * q[j].x;
        }
      }
      recomb_finalize<V, A, APT>(c, base, y, dst, extra, psi_other, nacc, gacc, ex0, ex1);
    }
  }
  double out[3] = {0.0, 0.0, 0.0};
  if (extra == kExtraOverlapTarget) {
    double vals[3] = {(double)nacc, ex0, ex1};
    if (!group_reduce<3>(c.g, ss.red, vals, out)) return false;
  } else {
    A vals[2] = {nacc, gacc};
    double o2[2];
    if (!group_reduce<2>(c.g, ss.red, vals, o2)) return false;
    out[0] = o2[0];
    out[1] = o2[1];
  }
  if (tid == 0) {
    ss.nrm_out = sqrt(fmax(out[0], 0.0));
    ss.code1 = isfinite(out[0]) ? 0 : 2;
  }
  wsync();
  if (ss.code1 == 2) {
    if (tid == 0) flag_nonfinite(p);
    return false;
  }
  nrm_dst = ss.nrm_out;
  e = make_double2(out[1], out[2]);
  c.mark(5);
  return true;
}

// Packed FP32x2 helpers (Blackwell FADD2/FMUL2/FFMA2) for complex64 arithmetic.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Chunk table of the complex64 resident path.  The partner amplitudes of the bonds that
// leave a 4096-amplitude tile come from other tiles as whole contiguous blocks:
//   bond 11 (bit 11 = the top in-tile bit, bit 12 = the lowest tile bit): the own half
//     h = 1 - bt (bt = bit 12 of the tile) pairs with half bt of tile base ^ 2^12, element
//     for element;
//   bond b >= 12, antiparallel for the whole tile: tile base ^ (3 << b), element for element;
//   an Sx control on site s >= 12: tile base ^ (1 << s), element for element.
// Entry: bits 3.. = source offset in units of 2048 amplitudes (16 KB), bit 2 = whole tile
// (32 KB, feeds every own amplitude) rather than one half, bit 1 = the own half h fed by a
// half block, bit 0 = weight of the Sx control instead of Jxy/2.  ct_start[cc] .. ct_start[cc+1]
// are tile cc's entries.  `first` is the tile with more blocks: the CTA computes it first,
// from plain loads issued right after the barrier, while the other tile's blocks stream
// into the bulk-copy ring.
__device__ __forceinline__ void build_chunk_table(const Ctx<float2>& c, const EvalParams& p, SmemSlice& ss) {
  const int L1 = p.L - 1;
  int n = 0;
  ss.ct_start[0] = 0;
  for (int cc = 0; cc < 2; ++cc) {
    if (cc < c.n_own) {
      const size_t base = c.tile_base(cc);
      if (L1 > 11) {
        const unsigned bt = (unsigned)((base >> 12) & 1u);
        const size_t off = ((base ^ ((size_t)1 << 12)) >> 11) + bt;
        ss.ctab[n++] = ((unsigned)off << 3) | ((1u - bt) << 1);
      }
      for (int b = 12; b < L1; ++b)
        if (((base >> b) ^ (base >> (b + 1))) & 1u)
          ss.ctab[n++] = ((unsigned)((base ^ ((size_t)3 << b)) >> 11) << 3) | 4u;
      if (p.hc_kind == KG_HC_SX_SITE && p.hc_site >= 12)
        ss.ctab[n++] = ((unsigned)((base ^ ((size_t)1 << p.hc_site)) >> 11) << 3) | 5u;
    }
    ss.ct_start[cc + 1] = n;
  }
  ss.first = (c.n_own == 2 && ss.ct_start[2] - ss.ct_start[1] > ss.ct_start[1]) ? 1 : 0;
}

// First table entry and number of blocks of the tile whose blocks go through the ring.
__device__ __forceinline__ int ring_i0(const SmemSlice& ss) { return ss.ct_start[ss.first ^ 1]; }
__device__ __forceinline__ int ring_n(const SmemSlice& ss) {
  return (ss.r.n_own == 2) ? ss.ct_start[(ss.first ^ 1) + 1] - ss.ct_start[ss.first ^ 1] : 0;
}

// Thread 0: bulk copy of chunk i of the table from vector `vec` into ring stage g % stages
// (g = the copy's running number), completing on that stage's barrier.
__device__ __forceinline__ void lz_issue(SmemSlice& ss, const float2* vec, int i, unsigned g) {
  const unsigned e = ss.ctab[i];
  const unsigned st = g % kLzStages;
  const uint32_t bytes = (e & 4u) ? 32768u : 16384u;
  mbar_arrive_expect_tx(&ss.lmbar[st], bytes);
  tma_load_1d(ss.r.ring + (size_t)st * 4096, vec + ((size_t)(e >> 3) << 11), bytes, &ss.lmbar[st]);
}

// Thread 0: the first ring copies of the second tile's blocks of vector vec (written by the
// group before the barrier this thread has just passed).
__device__ __forceinline__ void ring_start(SmemSlice& ss, const float2* vec, unsigned gbase) {
  fence_proxy_async_global();
  const int i0 = ring_i0(ss), n = ring_n(ss);
  for (int r = 0; r < n && r < kLzStages; ++r) lz_issue(ss, vec, i0 + r, gbase + (unsigned)r);
}

// Every thread: wait for ring copies that were started but will not be consumed (the loop
// ends early); true if they all arrived in time.
__device__ __forceinline__ bool ring_drain(const EvalParams& p, SmemSlice& ss, unsigned gbase) {
  bool ok = true;
  const int n = ring_n(ss);
  for (int r = 0; r < n && r < kLzStages; ++r) {
    const unsigned g = gbase + (unsigned)r;
    ok = ok && mbar_wait_bounded(p, &ss.lmbar[g % kLzStages], (g / kLzStages) & 1u);
  }
  return ok;
}

// Thread 0, complex64 resident path: alpha_k and b_{k+1}^2 = ||W||^2 + alpha^2 (||v||^2 - 2)
// from the float-float sums o = (<v|W>, ||W||^2, ||v||^2) of step k (about 44 bits; the FP64
// tridiagonal is formed from the same sums once the slice's steps are done).  code1 as in
// lz_after_reduce.
__device__ __forceinline__ FF lzf_after_reduce(SmemSlice& ss, int k, bool last, const FF (&o)[3]) {
  ss.ff_a[k] = make_float2(o[0].hi, o[0].lo);
  ss.ff_n[k] = make_float2(o[1].hi, o[1].lo);
  ss.ff_q[k] = make_float2(o[2].hi, o[2].lo);
  const float alpha = __fadd_rn(o[0].hi, o[0].lo);
  ss.f_alpha = alpha;
  ss.alpha_f[k] = alpha;
  const FF b2 = ff_add(o[1], ff_mul(ff_mul(o[0], o[0]), ff_add(o[2], FF{-2.f, 0.f})));
  int code = 0;
  if (!isfinite(alpha) || !isfinite(o[1].hi)) code = 2;
  else if (!last && b2.hi < 1e-3f * o[1].hi) code = 1;
  ss.code1 = code;
  return b2;
}

// Thread 0: b_{k+1} in FP32 (it only scales complex64 vectors), the breakdown test and the
// scalars of step k+1, as lz_finish_step.
__device__ __forceinline__ void lzf_finish_step(SmemSlice& ss, int k, bool last, FF b2, float bd_tol, float& amax,
                                                float& bmax) {
  const float beta = __fsqrt_rn(fmaxf(__fadd_rn(b2.hi, b2.lo), 0.f));
  const float alpha = ss.f_alpha;
  int stop = 0;
  if (last) {
    ss.f_beta_m = beta;
    stop = 1;
  } else {
    amax = fmaxf(amax, fabsf(alpha));
    if (beta <= bd_tol * fmaxf(1.f, amax + bmax)) {
      ss.meff = k + 1;
      ss.broke = 1;
      stop = 1;
    } else {
      bmax = fmaxf(bmax, beta);
      ss.f_ap = alpha;
      ss.f_ib = __frcp_rn(beta);
      ss.f_bk = beta;
      ss.beta_f[k + 1] = beta;
    }
  }
  ss.stop = stop;
}

// Warp 0 after the last step: the FP64 tridiagonal T (alpha_k, b_{k+1}) from the stored
// float-float sums, lane k for step k: b_{k+1}^2 from the same identity as lz_after_reduce,
// or from the explicit ||W - alpha v||^2 where that was formed.
__device__ __forceinline__ void lzf_build_T(SmemSlice& ss, int m) {
  const int k = threadIdx.x & 31;
  const int meff = ss.meff;
  if (k < meff) {
    const double al = ff_to_double(FF{ss.ff_a[k].x, ss.ff_a[k].y});
    double b2;
    if ((ss.ff_e_set >> k) & 1u) {
      b2 = ff_to_double(FF{ss.ff_e[k].x, ss.ff_e[k].y});
    } else {
      const double nn = ff_to_double(FF{ss.ff_n[k].x, ss.ff_n[k].y});
      const double q = ff_to_double(FF{ss.ff_q[k].x, ss.ff_q[k].y});
      b2 = nn - 2.0 * al * al + al * al * q;
    }
    const double be = sqrt(fmax(b2, 0.0));
    ss.alpha[k] = al;
    if (k + 1 < meff) ss.beta[k + 1] = be;
    if (k == m - 1) ss.beta_m = be;
  }
  __syncwarp();
}

// Warp 0, right after the barrier that closed a step: asynchronous copies of the group's
// reduction slots (this step's CTA partials) into shared memory, so that their L2 latency
// passes while the warp loads partner blocks and runs its stencil.
__device__ __forceinline__ void slot_prefetch(SmemSlice& ss) {
  const Group& g = ss.grp;
  const int size = g.size;
  if (size <= 1 || size > kSlotRanks) return;
  const float4* slots = reinterpret_cast<const float4*>(g.red + (size_t)((g.phase - 1) & 1) * g.stride * kNRed);
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < kSlotRanks / 32; ++i) {
    const int r = lane + 32 * i;
    if (r < size) {
      cp_async16(&ss.slotbuf[2 * r], slots + (size_t)r * (kNRed / 2));
      cp_async16(&ss.slotbuf[2 * r + 1], slots + (size_t)r * (kNRed / 2) + 1);
    }
  }
  cp_async_commit();
}

// Warp 0 after the barrier that closed step k: float-float totals of the step's sums, then
// thread 0 sets alpha_k, b_{k+1} and the scalars of step k+1.
__device__ __forceinline__ void warp0_scalars(SmemSlice& ss, int k, bool last) {
  FF o[3];
  if (ss.grp.size > 1 && ss.grp.size <= kSlotRanks) {
    // the slots were prefetched into shared memory (slot_prefetch); same summation order as
    // reduce_ff_collect
    cp_async_wait<0>();
    __syncwarp();
    const int lane = threadIdx.x & 31;
    FF t[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    for (int r = lane; r < ss.grp.size; r += 32) {
      const float4 a = ss.slotbuf[2 * r], b = ss.slotbuf[2 * r + 1];
      t[0] = ff_add(t[0], FF{a.x, a.y});
      t[1] = ff_add(t[1], FF{a.z, a.w});
      t[2] = ff_add(t[2], FF{b.x, b.y});
    }
#pragma unroll
    for (int v = 0; v < 3; ++v) o[v] = ff_warp_sum(t[v]);
  } else {
    reduce_ff_collect<3>(ss.grp, ss.red, o);
  }
  if (threadIdx.x == 0) {
    const FF b2 = lzf_after_reduce(ss, k, last, o);
    if (ss.code1 == 0) lzf_finish_step(ss, k, last, b2, ss.r.bdtol, ss.r.amax, ss.r.bmax);
  }
}

// Partner sums xs += sum wgt W[partner] of one tile from vector pv (table entries i0 .. i1),
// three blocks in flight in registers.
__device__ __forceinline__ void partner_regs(const SmemSlice& ss, const float2* pv, int i0, int i1, float2 (&xs)[8]) {
  constexpr int APT = 8, NT = kThreads, G = 3;
  const int tid = threadIdx.x;
  const float hxy = ss.r.hxy, cu_sx = ss.r.cusx;
  for (int ib = i0; ib < i1; ib += G) {
    float2 q[G][APT];
    float wq[G];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int i = ib + u;
      const unsigned e = (i < i1) ? ss.ctab[i] : 0u;
      // own amplitude j reads sb[j * NT]: the block itself, or for a half block feeding own
      // half h, the block shifted down by h * 2048 (only j in [4h, 4h + 4) are read)
      const unsigned hm = (i >= i1) ? 0u : ((e & 4u) ? 0xffu : (((e >> 1) & 1u) ? 0xf0u : 0x0fu));
      wq[u] = (e & 1u) ? cu_sx : hxy;
      const long long off = ((long long)(e >> 3) << 11) + tid - (((e & 6u) == 2u) ? 4 * NT : 0);
      const float2* sb = pv + off;
#pragma unroll
      for (int j = 0; j < APT; ++j) q[u][j] = ((hm >> j) & 1u) ? ldv(sb + j * NT) : f2(0.f);
    }
#pragma unroll
    for (int u = 0; u < G; ++u)
#pragma unroll
      for (int j = 0; j < APT; ++j) xs[j] = f2fma(f2(wq[u]), q[u][j], xs[j]);
  }
}

// Lanczos loop of one slice for complex64 tiles of 4096 amplitudes (512 threads x 8), every
// CTA holding its (at most 2) tiles resident.  Same recurrence as lanczos_generic, in
// another arrangement of the same arithmetic: the stencil acts on the raw vector W_k, which
// needs none of the step's scalars,
//   H W_k     = diag W_k + (Jxy/2) sum_{bonds} W_k[partner]   (+ control)
//   v_k       = (W_k - alpha_{k-1} v_{k-1}) / b_k
//   H v_k     = (H W_k - alpha_{k-1} H v_{k-1}) / b_k
//   W_{k+1}   = H v_k - b_k v_{k-1}
//   alpha_k   = <v_k|W_{k+1}>,  b_{k+1}^2 = ||W_{k+1}||^2 - 2 alpha_k <v_k|W_{k+1}> + alpha_k^2 ||v_k||^2,
// so the stencil of a step runs while warp 0 is still collecting the previous step's sums.
// The basis slots hold the raw vectors W_k (slot 0: psi): they are written anyway for the
// other tiles' partners, and the recombination sum_k c_k v_k is a sum over the W_k with
// transformed coefficients.  The amplitude of thread tid in register j is li = tid + 512 j:
//   bonds 0..7  (bits inside tid):  antiparallel test shared by all j, partner (tid ^ 3<<b) + 512 j
//   bond 8      (bit 8 of tid, bit 0 of j): partner (tid ^ 256) + 512 (j ^ 1)
//   bonds 9, 10 (bits of j):        partner in registers, test known at compile time
//   bond 11 and up:                 other tiles' blocks of W_k (global memory)
// Where the data lives: W_k of the own tiles in shared memory (the stencil reads the
// neighbours' amplitudes); v_{k-1} and H v_{k-1}, which only their thread reads, in tensor
// memory; the slice's constants and the group's barrier state in shared memory (the L1 left
// beside 200 KB of shared memory is too small for per-thread stack frames).  Partner
// blocks: for the tile with more blocks, plain L2 loads into registers, three blocks in
// flight, right after the barrier; for the other tile, a ring of 32 KB bulk copies (TMA)
// that thread 0 starts at the barrier and that fills while the first tile is computed.  The
// step's three sums are reduced in float-float; the FP32 scalars that scale the vectors come
// from them at once, the FP64 tridiagonal after the last step.
__device__ __noinline__ bool lanczos_res64(Ctx<float2>& c, const float2* src, double nrm_src, double uj) {
  const EvalParams& p = *c.p;
  SmemSlice& ss = *c.ss;
  constexpr int APT = 8, NB = 2, T = 4096, NT = kThreads;
  const int tid = threadIdx.x;
  const unsigned xt = (unsigned)(tid ^ (tid >> 1));
  const int t8 = (tid >> 8) & 1;
  const bool prof = c.prof_on && tid == 0;
  // TMEM columns: v_{k-1} of tile cc at tV + 16 cc, H v_{k-1} at tH + 16 cc, and H W_k of the
  // tile in hand at tP while the step's scalars are formed
  const uint32_t tV = c.tm, tH = c.tm + 32u, tP = c.tm + 64u, tW = c.tm + 96u;
  if (tid == 0) {
    ResCtx& r = ss.r;
    r.tbase[0] = c.tile_base(0);
    r.tbase[1] = (c.n_own > 1) ? c.tile_base(1) : 0;
    r.basis = (float2*)p.basis;
    r.D = c.D;
    r.sw = c.sv[0];
    r.ring = c.sv[1];
    r.maskL1 = c.maskL1;
    r.mk = (unsigned)p.hc_mask;
    r.L1 = p.L - 1;
    r.hs = p.hc_site;
    r.hcsx = (p.hc_kind == KG_HC_SX_SITE) ? 1 : 0;
    r.n_own = c.n_own;
    r.m = p.m;
    r.hxy = (float)(0.5 * p.Jxy);
    r.qz = (float)(0.25 * p.Jz);
    r.cusx = (float)(0.5 * uj * p.hc_amp);
    r.cusz = (float)(uj * p.hc_amp);
    r.amax = 0.f;  // running maxima for the breakdown test
    r.bmax = 0.f;
    r.bdtol = (float)p.bd_tol;
    ss.grp = c.g;
    lz_init(ss, nrm_src, p.m);
    ss.ff_e_set = 0u;
    build_chunk_table(c, p, ss);
  }
  // W_0 = psi: the own amplitudes into shared memory
  {
    float2* sw = c.sv[0];
#pragma unroll
    for (int cc = 0; cc < NB; ++cc) {
      if (cc >= c.n_own) break;
      const size_t base = c.tile_base(cc);
#pragma unroll
      for (int j = 0; j < APT; ++j) sw[cc * T + tid + j * NT] = ldv(src + base + tid + j * NT);
    }
  }
  wsync();
  if (ss.meff == 0) return true;
  const int m = ss.r.m;
  unsigned gbase = c.lz_count;  // running number of the step's first ring copy
  if (tid == 0 && ring_n(ss) > 0) ring_start(ss, src, gbase);
  const float2* vec = src;  // W_k: the vector whose partner blocks are read in step k
  bool done = false;        // the loop ran all m steps (the last step's sums still to collect)
  for (int k = 0; k < m; ++k) {
    const bool last = (k == m - 1);
    float2* wdst = last ? nullptr : ss.r.basis + (size_t)k * ss.r.D;  // W_{k+1}: basis slot k+1
    float2 acc_a = f2(0.f), acc_n = f2(0.f), acc_q = f2(0.f);
    bool stopped = false;
#pragma unroll 1
    for (int qq = 0; qq < NB; ++qq) {
      if (qq >= ss.r.n_own) break;
      const int cc = ss.first ^ qq;
      // ---- partner sums of W_k for this tile
      float2 xs[APT];
#pragma unroll
      for (int j = 0; j < APT; ++j) xs[j] = f2(0.f);
      if (qq == 0) {
        partner_regs(ss, vec, ss.ct_start[cc], ss.ct_start[cc + 1], xs);
      } else {
        const int iB0 = ss.ct_start[cc], nB = ss.ct_start[cc + 1] - iB0;
        const float2* ring = ss.r.ring;
        for (int r = 0; r < nB; ++r) {
          const unsigned g = gbase + (unsigned)r;
          const unsigned st = g % kLzStages;
          const bool ok = mbar_wait_bounded(p, &ss.lmbar[st], (g / kLzStages) & 1u);
          if (ok) {
            const unsigned e = ss.ctab[iB0 + r];
            const float2 wg = f2((e & 1u) ? ss.r.cusx : ss.r.hxy);
            const float2* buf = ring + (size_t)st * T;
            if (e & 4u) {
#pragma unroll
              for (int j = 0; j < APT; ++j) xs[j] = f2fma(wg, buf[tid + j * NT], xs[j]);
            } else if (e & 2u) {
#pragma unroll
              for (int j = 0; j < 4; ++j) xs[4 + j] = f2fma(wg, buf[tid + j * NT], xs[4 + j]);
            } else {
#pragma unroll
              for (int j = 0; j < 4; ++j) xs[j] = f2fma(wg, buf[tid + j * NT], xs[j]);
            }
          }
          // Every thread is done with stage st: its reads have returned, so the next copy may
          // overwrite it (no proxy fence: a fence here would wait for the copies in flight).
          if (wsync_or(!ok)) return false;
          if (tid == 0 && r + kLzStages < nB) lz_issue(ss, vec, iB0 + r + kLzStages, g + kLzStages);
        }
      }
      if (prof) prof_mark(ss, 0);
      // ---- stencil: hw = H W_k on the own amplitudes (parked in TMEM across the barrier)
      {
        const size_t base = ss.r.tbase[cc];
        const float2* sc = ss.r.sw + cc * T;
        float2 h[APT], wo[APT], hw[APT];
#pragma unroll
        for (int j = 0; j < APT; ++j) h[j] = f2(0.f);
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          if ((xt >> b) & 1u) {
            const float2* ps = sc + (tid ^ (3 << b));
#pragma unroll
            for (int j = 0; j < APT; ++j) h[j] = f2add(h[j], ps[j * NT]);
          }
        }
        {
          const float2* ps = sc + (tid ^ 256);
#pragma unroll
          for (int j = 0; j < APT; ++j)
            if (t8 != (j & 1)) h[j] = f2add(h[j], ps[(j ^ 1) * NT]);
        }
#pragma unroll
        for (int j = 0; j < APT; ++j) wo[j] = sc[tid + j * NT];
#pragma unroll
        for (int j = 0; j < APT; ++j) {
          if ((j ^ (j >> 1)) & 1) h[j] = f2add(h[j], wo[j ^ 3]);         // bond 9
          if (((j >> 1) ^ (j >> 2)) & 1) h[j] = f2add(h[j], wo[j ^ 6]);  // bond 10
        }
        const float hxy = ss.r.hxy, qz = ss.r.qz, cu_sx = ss.r.cusx, cu_sz = ss.r.cusz;
        const unsigned mk = ss.r.mk, maskL1 = ss.r.maskL1;
        const bool hc_sx = ss.r.hcsx != 0;
        const int hs = ss.r.hs, L1 = ss.r.L1;
#pragma unroll
        for (int j = 0; j < APT; ++j) {
          const int li = tid + j * NT;
          const unsigned gi = (unsigned)(base + li);
          const unsigned xg = (gi ^ (gi >> 1)) & maskL1;
          float d = qz * (float)(L1 - 2 * __popc(xg));
          if (!hc_sx) d += cu_sz * 0.5f * (float)(__popc(mk) - 2 * __popc(gi & mk));
          float2 hv = f2fma(f2(d), wo[j], f2fma(f2(hxy), h[j], xs[j]));
          if (hc_sx && hs < 12) hv = f2fma(f2(cu_sx), sc[li ^ (1 << hs)], hv);
          hw[j] = hv;
        }
        tmem_st8c(tP, hw);
      }
      if (qq == 0 && k > 0 && tid < 32) warp0_scalars(ss, k - 1, false);
      wsync();  // the scalars of step k; every neighbour read of W_k in this tile done
      if (qq == 0 && k > 0) {
        const int code = ss.code1;
        if (code == 2) {
          if (tid == 0) flag_nonfinite(p);
          ring_drain(p, ss, gbase);
          return false;
        }
        if (code == 1) {  // near an invariant subspace: explicit ||W_k - alpha_{k-1} v_{k-1}||^2
          float n1[1] = {0.f};
          const float ra = ss.f_alpha;
          for (int c2 = 0; c2 < ss.r.n_own; ++c2) {
            float2 vp[APT];
            tmem_ld8c(tV + 16u * c2, vp);
#pragma unroll
            for (int j = 0; j < APT; ++j) {
              const float2 rr = f2fma(f2(-ra), vp[j], ss.r.sw[c2 * T + tid + j * NT]);
              n1[0] += rr.x * rr.x + rr.y * rr.y;
            }
          }
          if (!reduce_ff_arrive_shared<1>(ss.grp, ss.red, n1)) {
            ring_drain(p, ss, gbase);
            return false;
          }
          if (tid < 32) {
            FF o1[1];
            reduce_ff_collect<1>(ss.grp, ss.red, o1);
            if (tid == 0) {
              ss.ff_e[k - 1] = make_float2(o1[0].hi, o1[0].lo);
              ss.ff_e_set |= 1u << (k - 1);
              lzf_finish_step(ss, k - 1, false, o1[0], ss.r.bdtol, ss.r.amax, ss.r.bmax);
            }
          }
          wsync();
        }
        if (ss.stop) {  // breakdown: v_k does not exist; the copies started for step k are not used
          if (wsync_or(!ring_drain(p, ss, gbase))) return false;
          gbase += (unsigned)min(ring_n(ss), kLzStages);
          stopped = true;
          break;
        }
      }
      if (prof) prof_mark(ss, 3);
      // ---- v_k, H v_k, W_{k+1} = H v_k - b_k v_{k-1} for the own amplitudes; partial sums
      {
        const float ap = ss.f_ap, ib = ss.f_ib, bk = ss.f_bk;
        float2* sw = ss.r.sw + cc * T;
        float2 vp[APT], hp[APT], wo[APT], hw[APT];
        tmem_ld8c(tP, hw);
#pragma unroll
        for (int j = 0; j < APT; ++j) wo[j] = sw[tid + j * NT];  // W_k, own amplitudes
        if (k > 0) {
          tmem_ld8c(tV + 16u * cc, vp);
          tmem_ld8c(tH + 16u * cc, hp);
        }
#pragma unroll
        for (int j = 0; j < APT; ++j) {
          float2 v, hv, w;
          if (k == 0) {
            v = f2mul(wo[j], f2(ib));
            hv = f2mul(hw[j], f2(ib));
            w = hv;
          } else {
            v = f2mul(f2fma(f2(-ap), vp[j], wo[j]), f2(ib));
            hv = f2mul(f2fma(f2(-ap), hp[j], hw[j]), f2(ib));
            w = f2fma(f2(-bk), vp[j], hv);
          }
          acc_a = f2fma(v, w, acc_a);
          acc_n = f2fma(w, w, acc_n);
          acc_q = f2fma(v, v, acc_q);
          vp[j] = v;
          hp[j] = hv;
          wo[j] = w;
        }
        if (!last) {
          tmem_st8c(tV + 16u * cc, vp);
          tmem_st8c(tH + 16u * cc, hp);
          const size_t base = ss.r.tbase[cc];
#pragma unroll
          for (int j = 0; j < APT; ++j) {
            const int li = tid + j * NT;
            sw[li] = wo[j];
            stv(wdst + base + li, wo[j]);
          }
        }
      }
      if (prof) prof_mark(ss, 1);
    }
    if (stopped) break;
    float acc[3] = {acc_a.x + acc_a.y, acc_n.x + acc_n.y, acc_q.x + acc_q.y};
    if (!reduce_ff_arrive_shared<3>(ss.grp, ss.red, acc)) return false;
    if (prof) prof_mark(ss, 2);
    gbase += (unsigned)ring_n(ss);  // every ring copy of step k has been consumed
    if (!last && tid < 32) {
      if (tid == 0 && ring_n(ss) > 0) ring_start(ss, wdst, gbase);
      slot_prefetch(ss);  // step k's partials, summed by warp 0 during step k+1
    }
    vec = wdst;
    if (last) done = true;
  }
  if (done) {  // the sums of the last step: alpha_{m-1}, b_m (error indicator)
    if (tid < 32) {
      slot_prefetch(ss);  // (the last step did not prefetch)
      warp0_scalars(ss, m - 1, true);
    }
    wsync();
    if (ss.code1 == 2) {
      if (tid == 0) flag_nonfinite(p);
      return false;
    }
  }
  c.lz_count = gbase;
  c.g.phase = ss.grp.phase;  // the group state goes back to every thread's context
  c.g.epoch = ss.grp.epoch;
  c.g.skip_arrival = ss.grp.skip_arrival;
  if (tid < 32) lzf_build_T(ss, m);
  return true;
}

// Complex64 helpers of the pair layout: a float4 holds the amplitude pair (2P, 2P + 1).
__device__ __forceinline__ float2 lo2(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi2(float4 a) { return make_float2(a.z, a.w); }
__device__ __forceinline__ float4 pair4(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
__device__ __forceinline__ float4 ldv4(const float4* p) { return __ldcg(p); }
__device__ __forceinline__ void stv4(float4* p, float4 v) { __stcg(p, v); }
// Stores with an L2 eviction priority.  Within a slice the L2 (about 126 MB) cannot hold the whole
// Krylov basis at L = 20 (19 vectors of 8 MiB): the basis vectors are stored with evict_last, so
// that as many as possible are still there when the recombination reads them; the recombination's
// reads of the basis and the state it writes go with evict_first (l2_policy_first).
__device__ __forceinline__ unsigned long long l2_evict_last() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void stv4_hint(float4* p, float4 v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w), "l"(pol)
               : "memory");
}

// Units of the partner ring (thread 0, once per slice, from the chunk table): a whole-tile entry
// gives two units -- own pairs g = 0, 1 from granules 0, 1 of the block, g = 2, 3 from granules
// 2, 3 -- and a half entry (bond 11) one: own half h, pairs g = 2h, 2h + 1, from granules 0, 1 of
// the half block.  Granule g of a block is the float4 at 512 g + tid.  Unit word: bits 2.. = the
// unit's first granule in float4 from the vector's start, bit 1 = the own half d (pairs 2d,
// 2d + 1), bit 0 = weight of the Sx control instead of Jxy/2.  Tile 0's units (n_units0 of them)
// come first, then tile 1's.
__device__ __forceinline__ void build_unit_table(SmemSlice& ss, int n_own) {
  int n = 0;
  for (int cc = 0; cc < n_own; ++cc) {
    for (int i = ss.ct_start[cc]; i < ss.ct_start[cc + 1]; ++i) {
      const unsigned e = ss.ctab[i];
      const unsigned off4 = (e >> 3) << 10;  // 2048 amplitudes = 1024 float4
      if (e & 4u) {
        ss.utab[n++] = (off4 << 2) | (e & 1u);
        ss.utab[n++] = ((off4 + 1024u) << 2) | 2u | (e & 1u);
      } else {
        ss.utab[n++] = (off4 << 2) | (((e >> 1) & 1u) << 1) | (e & 1u);
      }
    }
    if (cc == 0) ss.n_units0 = n;
  }
  ss.n_units = n;
}

// h[4d .. 4d + 3] += wt (a, b): one unit's two granules added to own pairs 2d, 2d + 1.
__device__ __forceinline__ void unit_acc(float2 (&h)[8], unsigned d, float wt, float4 a, float4 b) {
  if (d == 0) {
    h[0] = f2fma(f2(wt), lo2(a), h[0]);
    h[1] = f2fma(f2(wt), hi2(a), h[1]);
    h[2] = f2fma(f2(wt), lo2(b), h[2]);
    h[3] = f2fma(f2(wt), hi2(b), h[3]);
  } else {
    h[4] = f2fma(f2(wt), lo2(a), h[4]);
    h[5] = f2fma(f2(wt), hi2(a), h[5]);
    h[6] = f2fma(f2(wt), lo2(b), h[6]);
    h[7] = f2fma(f2(wt), hi2(b), h[7]);
  }
}

// Partner ring of the headline loop.  The partner granules of W_k stream through this thread's
// slots of a ring of kPrRing units in shared memory by 16-byte asynchronous copies (cp.async.cg:
// L2 only; the blocks were written by other CTAs before the group barrier).  pring_start puts the
// first kPrRing units in flight; pring_take adds units [u0, u1) to h in table order (h holds the
// in-tile part of H W_k of the tile they feed), each unit taken freeing its slot for the unit
// kPrRing further on.  A thread reads back only the granules it copied, so no block barrier is
// needed, and no register holds a load in flight.
__device__ __forceinline__ void pring_start(const SmemSlice& ss, const float2* pv) {
  const int tid = threadIdx.x;
  const int nU = ss.n_units;
  const float4* v4 = reinterpret_cast<const float4*>(pv) + tid;
  float4* slot0 = ss.r.pring + tid;
#pragma unroll
  for (int s = 0; s < kPrRing; ++s) {
    if (s < nU) {
      const float4* src = v4 + (ss.utab[s] >> 2);
      cp_async16(slot0 + s * (2 * kThreads), src);
      cp_async16(slot0 + s * (2 * kThreads) + kThreads, src + kThreads);
    }
    cp_async_commit();
  }
}
__device__ __forceinline__ void pring_take(const SmemSlice& ss, const float2* pv, int u0, int u1, float2 (&h)[8]) {
  constexpr int R = kPrRing;
  const int tid = threadIdx.x;
  const int nU = ss.n_units;
  const float4* v4 = reinterpret_cast<const float4*>(pv) + tid;
  float4* slot0 = ss.r.pring + tid;
  const float hxy = ss.r.hxy, cu_sx = ss.r.cusx;
  int s = u0 % R;  // unit u sits in slot u % R
#pragma unroll 1
  for (int u = u0; u < u1; ++u) {
    cp_async_wait<R - 1>();  // this thread's granules of unit u have landed
    const unsigned w = ss.utab[u];
    float4* q = slot0 + s * (2 * kThreads);
    const float4 a = q[0], b = q[kThreads];
    unit_acc(h, (w >> 1) & 1u, (w & 1u) ? cu_sx : hxy, a, b);
    if (u + R < nU) {
      const float4* src = v4 + (ss.utab[u + R] >> 2);
      cp_async16(q, src);
      cp_async16(q + kThreads, src + kThreads);
    }
    cp_async_commit();
    s = (s + 1 == R) ? 0 : s + 1;
  }
}

// Step k's update of own tile cc from the complete H W_k parked in tensor memory (tP + 16 cc) and
// the own W_k (tW + 16 cc): v_k, H v_k and W_{k+1} (tensor memory, not waited for), W_{k+1} = H v_k - b_k v_{k-1} (shared memory and basis slot k+1,
// unless this is the slice's last step) and the tile's share of the step's partial sums.
// It runs pair by pair (pair g: TMEM columns 4 g .. 4 g + 3 of each quantity).
__device__ __forceinline__ void update_tile(const SmemSlice& ss, int cc, int k, uint32_t tP, uint32_t tV, uint32_t tH,
                                            uint32_t tW, float2& acc_a, float2& acc_n, float2& acc_q) {
  constexpr int T = 4096;
  const int tid = threadIdx.x;
  const bool last = (k == ss.r.m - 1);
  const float ap = ss.f_ap, ib = ss.f_ib, bk = ss.f_bk;
  float4* sw4 = reinterpret_cast<float4*>(ss.r.sw + cc * T);
  float4* d4 = reinterpret_cast<float4*>(ss.r.basis + (size_t)k * ss.r.D + ss.r.tbase[cc]);  // W_{k+1}: slot k+1
  const unsigned long long keep = l2_evict_last();
#pragma unroll
  for (int g = 0; g < 4; ++g) {  // pair g: TMEM columns 4 g .. 4 g + 3
    const uint32_t co = 16u * cc + 4u * g;
    float2 hw[2], vp[2], hp[2], wo[2];
    tmem_ld2c_x4(tP + co, tV + co, tH + co, tW + co, hw, vp, hp, wo);  // vp, hp unused at k = 0
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      float2 v, hv, w;
      if (k == 0) {
        v = f2mul(wo[a], f2(ib));
        hv = f2mul(hw[a], f2(ib));
        w = hv;
      } else {
        v = f2mul(f2fma(f2(-ap), vp[a], wo[a]), f2(ib));
        hv = f2mul(f2fma(f2(-ap), hp[a], hw[a]), f2(ib));
        w = f2fma(f2(-bk), vp[a], hv);
      }
      acc_a = f2fma(v, w, acc_a);
      acc_n = f2fma(w, w, acc_n);
      acc_q = f2fma(v, v, acc_q);
      vp[a] = v;
      hp[a] = hv;
      wo[a] = w;
    }
    if (!last) {
      tmem_st2c_x3_nowait(tV + co, tH + co, tW + co, vp, hp, wo);
      const float4 w4 = pair4(wo[0], wo[1]);
      sw4[tid + 512 * g] = w4;
      stv4_hint(d4 + tid + 512 * g, w4, keep);
    }
  }
}

// In-tile part of H_j W for the own pairs of tile cc, from shared memory only: the bonds inside
// the tile (times Jxy/2), the diagonal (formed once per slice) and an Sx control inside the tile;
// parked in tensor memory at tP + 16 cc (the store is not waited for here).  The thread's own pairs
// come from tensor memory (tW + 16 cc), their neighbours' from shared memory.  Index bits of an
// own amplitude: bit 0 = x, bits 1..9 = tid, bits 10, 11 = g.  Bonds:
//   bond 0 (bits 0, 1): the element x = 1 - (tid & 1) of each pair, partner element tid & 1 of
//     pair tid ^ 1;
//   bonds 1..8 (tid bits b-1, b): pair tid ^ (3 << (b-1)), both elements;
//   bond 9 (tid bit 8, g bit 0): pair (tid ^ 256) + 512 (g ^ 1) where they differ;
//   bond 10 (g bits 0, 1): own pair g ^ 3 for g = 1, 2 (registers).
// An Sx control on site 1 (bit 0) couples the two elements of an own pair (registers).
__device__ __forceinline__ void stencil_park(const SmemSlice& ss, int cc, uint32_t tP, uint32_t tW) {
  constexpr int T = 4096;
  const int tid = threadIdx.x;
  const float4* sw4 = reinterpret_cast<const float4*>(ss.r.sw + cc * T);
  const float2* sw2 = ss.r.sw + cc * T;
  float2 h[8];
  {
    const unsigned xt = (unsigned)(tid ^ (tid >> 1));
    const float ma = (float)(tid & 1), mb = 1.f - ma;  // bond 0 feeds element 0 <=> tid odd
    float2 b0[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) b0[g] = sw2[2 * ((tid ^ 1) + 512 * g) + (tid & 1)];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      h[2 * g] = f2mul(f2(ma), b0[g]);
      h[2 * g + 1] = f2mul(f2(mb), b0[g]);
    }
#pragma unroll
    for (int b = 1; b <= 8; ++b) {
      if ((xt >> (b - 1)) & 1u) {
        const float4* ps = sw4 + (tid ^ (3 << (b - 1)));
        float4 pv4[4];
#pragma unroll
        for (int g = 0; g < 4; ++g) pv4[g] = ps[512 * g];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          h[2 * g] = f2add(h[2 * g], lo2(pv4[g]));
          h[2 * g + 1] = f2add(h[2 * g + 1], hi2(pv4[g]));
        }
      }
    }
    const int t8 = (tid >> 8) & 1;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      if (t8 != (g & 1)) {
        const float4 pv4 = sw4[(tid ^ 256) + 512 * (g ^ 1)];
        h[2 * g] = f2add(h[2 * g], lo2(pv4));
        h[2 * g + 1] = f2add(h[2 * g + 1], hi2(pv4));
      }
    }
  }
  const float cu_sx = ss.r.cusx, hxy = ss.r.hxy;
  const bool hc_sx = ss.r.hcsx != 0;
  const int hs = ss.r.hs;
  const float2* dg = reinterpret_cast<const float2*>(ss.r.ring) + cc * (T / 2);
  float4 wp[4];
  {  // the own pairs, from tensor memory (the caller has waited for their stores)
    float2 w8[8];
    tmem_ld8c(tW + 16u * cc, w8);
#pragma unroll
    for (int g = 0; g < 4; ++g) wp[g] = pair4(w8[2 * g], w8[2 * g + 1]);
  }
  // bond 10 (g bits 0, 1): g = 1 <-> g = 2
  h[2] = f2add(h[2], lo2(wp[2]));
  h[3] = f2add(h[3], hi2(wp[2]));
  h[4] = f2add(h[4], lo2(wp[1]));
  h[5] = f2add(h[5], hi2(wp[1]));
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const float2 d = dg[tid + 512 * g];
    h[2 * g] = f2fma(f2(d.x), lo2(wp[g]), f2mul(f2(hxy), h[2 * g]));
    h[2 * g + 1] = f2fma(f2(d.y), hi2(wp[g]), f2mul(f2(hxy), h[2 * g + 1]));
  }
  if (hc_sx && hs < 12) {  // the Sx control inside the tile
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      float4 q;
      if (hs == 0) q = make_float4(wp[g].z, wp[g].w, wp[g].x, wp[g].y);
      else if (hs <= 9) q = sw4[(tid ^ (1 << (hs - 1))) + 512 * g];
      else q = (hs == 10) ? wp[g ^ 1] : wp[g ^ 2];
      h[2 * g] = f2fma(f2(cu_sx), lo2(q), h[2 * g]);
      h[2 * g + 1] = f2fma(f2(cu_sx), hi2(q), h[2 * g + 1]);
    }
  }
  tmem_st8c_nowait(tP + 16u * cc, h);
}

// Near an invariant subspace (the identity for b_k^2 cancels): ||W_k - alpha_{k-1} v_{k-1}||^2
// over the group, explicitly, then b_k and the scalars of step k (lanczos_res64b, pair layout).
// Out of line: it runs rarely and keeps its registers out of the step loop.
__device__ __noinline__ bool res64b_explicit_norm(SmemSlice& ss, uint32_t tV, int k) {
  constexpr int T = 4096;
  const int tid = threadIdx.x;
  float n1[1] = {0.f};
  const float ra = ss.f_alpha;
  for (int c2 = 0; c2 < ss.r.n_own; ++c2) {
    float2 vp[8];
    tmem_ld8c(tV + 16u * c2, vp);
    const float4* s4 = reinterpret_cast<const float4*>(ss.r.sw + c2 * T);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const float4 wq4 = s4[tid + 512 * g];
      const float2 r0 = f2fma(f2(-ra), vp[2 * g], lo2(wq4));
      const float2 r1 = f2fma(f2(-ra), vp[2 * g + 1], hi2(wq4));
      n1[0] += r0.x * r0.x + r0.y * r0.y + r1.x * r1.x + r1.y * r1.y;
    }
  }
  if (!reduce_ff_arrive_shared<1>(ss.grp, ss.red, n1)) return false;
  if (tid < 32) {
    FF o1[1];
    reduce_ff_collect<1>(ss.grp, ss.red, o1);
    if (tid == 0) {
      ss.ff_e[k - 1] = make_float2(o1[0].hi, o1[0].lo);
      ss.ff_e_set |= 1u << (k - 1);
      lzf_finish_step(ss, k - 1, false, o1[0], ss.r.bdtol, ss.r.amax, ss.r.bmax);
    }
  }
  wsync();
  return true;
}

// Lanczos loop of one slice for complex64 tiles of 4096 amplitudes, two per CTA, resident: the
// algebra and storage of lanczos_res64 (stencil on the raw vector W_k, H v_k by its two-term
// recurrence, basis slots holding W_k, v_{k-1} and H v_{k-1} in tensor memory, W_k of the own
// tiles in shared memory for the neighbours and in tensor memory for the owning thread), in the
// pair layout -- thread tid owns the amplitude pairs
// P = tid + 512 g (g < 4) of each own tile, amplitudes 2P and 2P + 1, so that every vector access
// moves 16 bytes -- with group sums in fixed point, served by the block's control warp
// (res64b_control).  Step k, for the 16 worker warps:
//   1. (the in-tile part of H W_k is parked in tensor memory) wait until W_k is visible to the
//      group (named barrier kBarGroup; nothing to wait for at k = 0);
//   2. both tiles: H W_k = the parked in-tile part + the partner blocks of W_k from other tiles
//      (16-byte asynchronous copies through a per-thread ring in shared memory, kPrRing units
//      of 16 KB per CTA in flight);
//   3. take alpha_{k-1}, b_k and the scalars of step k, which the control warp formed from the
//      group totals during stage 2 (named barrier kBarScal); b_k explicitly near an invariant
//      subspace;
//   4. both tiles: v_k, H v_k, W_{k+1} (tensor memory, shared memory and basis slot k+1), partial
//      sums;
//   5. hand the warps' partial sums to the control warp (named barrier kBarPost; no wait): it
//      adds the CTA's share to the group sums and arrives at the group barrier, which waits
//      for the W_{k+1} stores to drain;
//   6. meanwhile, after a workers' barrier: the in-tile part of H W_{k+1} (shared memory only;
//      the diagonal was formed once per slice), parked in tensor memory.
// No worker waits for a store to drain, polls the group barrier or forms a scalar.  Tensor-memory
// stores are not waited for where they are issued; one wait comes before the next loads.
__device__ __noinline__ bool lanczos_res64b(Ctx<float2>& c, const float2* src, double nrm_src, double uj) {
  const EvalParams& p = *c.p;
  SmemSlice& ss = *c.ss;
  constexpr int NB = 2, T = 4096;
  const int tid = threadIdx.x;
  const bool prof = c.prof_on && tid == 0;
  // TMEM columns: v_{k-1} of tile cc at tV + 16 cc, H v_{k-1} at tH + 16 cc, the in-tile part
  // of H W_k at tP + 16 cc, the thread's own pairs of W_k at tW + 16 cc (all 128 columns)
  const uint32_t tV = c.tm, tH = c.tm + 32u, tP = c.tm + 64u, tW = c.tm + 96u;
  if (tid == 0) {
    ResCtx& r = ss.r;
    r.tbase[0] = c.tile_base(0);
    r.tbase[1] = (c.n_own > 1) ? c.tile_base(1) : 0;
    r.basis = (float2*)p.basis;
    r.D = c.D;
    r.sw = c.sv[0];
    r.ring = c.sv[1];  // here: the diagonal of H_j, [2 tiles][2048 pairs] float2
    r.pring = reinterpret_cast<float4*>(c.sv[1] + NB * (T / 2));  // partner ring behind it
    r.maskL1 = c.maskL1;
    r.mk = (unsigned)p.hc_mask;
    r.L1 = p.L - 1;
    r.hs = p.hc_site;
    r.hcsx = (p.hc_kind == KG_HC_SX_SITE) ? 1 : 0;
    r.n_own = c.n_own;
    r.m = p.m;
    r.hxy = (float)(0.5 * p.Jxy);
    r.qz = (float)(0.25 * p.Jz);
    r.cusx = (float)(0.5 * uj * p.hc_amp);
    r.cusz = (float)(uj * p.hc_amp);
    r.amax = 0.f;
    r.bmax = 0.f;
    r.bdtol = (float)p.bd_tol;
    // Fixed-point scale of the step sums <v|W>, ||W||^2, ||v||^2: with ||v|| = 1 and
    // ||W_{k+1}|| = ||H v_k - b_k v_{k-1}|| <= 2 ||H_j||, every total and every CTA's share is
    // below B = 1.5 max(1, 4 hb^2), hb a row-sum bound of ||H_j||; 2^S B stays below 2^61.
    const float hcw = (p.hc_kind == KG_HC_SX_SITE) ? 0.5f : 0.5f * (float)__popcll(p.hc_mask);
    const float hb = (float)(p.L - 1) * (0.5f * fabsf((float)p.Jxy) + 0.25f * fabsf((float)p.Jz)) +
                     fabsf((float)uj) * fabsf((float)p.hc_amp) * hcw;
    int e2 = 0;
    frexpf(1.5f * fmaxf(1.f, 4.f * hb * hb), &e2);  // B < 2^e2
    const int S = min(max(61 - e2, 0), 100);
    r.fscale = ldexpf(1.f, S);
    r.finv = ldexpf(1.f, -S);
    ss.grp = c.g;
    lz_init(ss, nrm_src, p.m);
    ss.ff_e_set = 0u;
    build_chunk_table(c, p, ss);
    build_unit_table(ss, c.n_own);
  }
  // W_0 = psi: the own pairs into shared memory; the diagonal of H_j (pair order) beside it
  {
    const float qz = (float)(0.25 * p.Jz), cu_sz = (float)(uj * p.hc_amp);
    const unsigned mk = (unsigned)p.hc_mask, maskL1 = c.maskL1;
    const bool hc_sx = (p.hc_kind == KG_HC_SX_SITE);
    const int L1 = p.L - 1;
    float4* sw4 = reinterpret_cast<float4*>(c.sv[0]);
    float2* dg = reinterpret_cast<float2*>(c.sv[1]);
#pragma unroll
    for (int cc = 0; cc < NB; ++cc) {
      if (cc >= c.n_own) break;
      const size_t base = c.tile_base(cc);
      const float4* s4 = reinterpret_cast<const float4*>(src + base);
      float2 w4[4];
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const float4 q = ldv4(s4 + tid + 512 * g);
        sw4[cc * (T / 2) + tid + 512 * g] = q;
        w4[2 * (g & 1)] = lo2(q);
        w4[2 * (g & 1) + 1] = hi2(q);
        if (g & 1) tmem_st4c_nowait(tW + 16u * cc + 8u * (g >> 1), w4);  // own pairs of W_0 (update, stencil)
        float dd[2];
#pragma unroll
        for (int x = 0; x < 2; ++x) {
          const unsigned gi = (unsigned)(base + 2 * (tid + 512 * g) + x);
          const unsigned xg = (gi ^ (gi >> 1)) & maskL1;
          dd[x] = qz * (float)(L1 - 2 * __popc(xg));
          if (!hc_sx) dd[x] += cu_sz * 0.5f * (float)(__popc(mk) - 2 * __popc(gi & mk));
        }
        dg[cc * (T / 2) + tid + 512 * g] = make_float2(dd[0], dd[1]);
      }
    }
  }
  wsync();
  if (ss.meff == 0) return true;
  const int m = ss.r.m;
  const int n_own = ss.r.n_own;
  tmem_st_wait();  // W_0's own pairs
  for (int cc = 0; cc < n_own; ++cc) stencil_park(ss, cc, tP, tW);  // in-tile part of H W_0
  const float2* vec = src;  // W_k: the vector whose partner blocks are read in step k
  bool done = false;
  for (int k = 0; k < m; ++k) {
    const bool last = (k == m - 1);
    // ---- 1. W_k is visible to the group (the barrier of step k - 1)
    if (k > 0) {
      nbar_sync(kBarGroup, kCtlThreads);
      if (!ss.ctl_ok) {
        nbar_sync(kBarScal, kCtlThreads);
        tmem_st_wait();
        return false;
      }
      if (prof) prof_mark(ss, 2);
    }
    // ---- 2. H W_k of both tiles: the parked in-tile parts plus the partner blocks, which stream
    // through the ring (tile 0's units first), parked again
    {
      pring_start(ss, vec);
      float2 h[8];
      tmem_st_wait();  // the in-tile parts were parked without a wait
      tmem_ld8c(tP, h);
      pring_take(ss, vec, 0, ss.n_units0, h);
      if (n_own > 1) {
        tmem_st8c_nowait(tP, h);
        tmem_ld8c(tP + 16u, h);
        pring_take(ss, vec, ss.n_units0, ss.n_units, h);
        tmem_st8c_nowait(tP + 16u, h);
      } else {
        tmem_st8c_nowait(tP, h);
      }
    }
    if (prof) prof_mark(ss, 0);
    // ---- 3. alpha_{k-1}, b_k and the scalars of step k (formed by the control warp)
    if (k > 0) {
      nbar_sync(kBarScal, kCtlThreads);
      const int code = ss.code1;
      if (code == 2) {
        tmem_st_wait();
        if (tid == 0) flag_nonfinite(p);
        return false;
      }
      if (code == 1) {  // near an invariant subspace: b_k from ||W_k - alpha_{k-1} v_{k-1}||^2
        tmem_st_wait();
        if (!res64b_explicit_norm(ss, tV, k)) return false;
      }
      if (ss.stop) break;  // breakdown: v_k does not exist
    }
    if (prof) prof_mark(ss, 3);
    // ---- 4. v_k, H v_k, W_{k+1} = H v_k - b_k v_{k-1} for the own amplitudes; partial sums
    float2 acc_a = f2(0.f), acc_n = f2(0.f), acc_q = f2(0.f);
    tmem_st_wait();  // H W_k parked above
#pragma unroll 1
    for (int cc = 0; cc < n_own; ++cc) update_tile(ss, cc, k, tP, tV, tH, tW, acc_a, acc_n, acc_q);
    if (prof) prof_mark(ss, 1);
    // ---- 5. the warps' partial sums of step k to the control warp (it arrives for the CTA)
    {
      float acc[3] = {warp_sum(acc_a.x + acc_a.y), warp_sum(acc_n.x + acc_n.y), warp_sum(acc_q.x + acc_q.y)};
      if ((tid & 31) == 0) {
#pragma unroll
        for (int v = 0; v < 3; ++v) ss.red.warp_part_f[(tid >> 5) * kNRed + v] = acc[v];
      }
      if (tid == 0) ss.ctl_cmd = k | (last ? kCtlLast : 0);
      nbar_arrive(kBarPost, kCtlThreads);
    }
    // ---- 6. the in-tile part of H W_{k+1} while the group arrives (it reads other threads'
    // amplitudes of W_{k+1} in shared memory: one workers' barrier first)
    if (!last) {
      wsync();
      tmem_st_wait();  // W_{k+1}'s own pairs
      for (int cc = 0; cc < n_own; ++cc) stencil_park(ss, cc, tP, tW);
    }
    vec = ss.r.basis + (size_t)k * ss.r.D;  // W_{k+1}: basis slot k+1
    if (last) done = true;
  }
  tmem_st_wait();  // every store of v_k, H v_k has completed
  if (done) {  // the last step's sums: alpha_{m-1}, b_m (error indicator), formed by the control warp
    // Meanwhile the recombination's first copies go out (the own tiles of the newest basis
    // vectors, which this CTA stored itself; they do not depend on the last sums), into the
    // shared memory the loop no longer needs.
    wsync();
    {
      const size_t rb[2] = {ss.r.tbase[0], ss.r.tbase[1]};
      float4* stg = reinterpret_cast<float4*>(c.sv[0]);
      for (int s = 0; s < kRecombDepth; ++s) {
        if (s < m) {
          const int ks = m - 1 - s;
          recomb_issue(ks == 0 ? src : ss.r.basis + (size_t)(ks - 1) * ss.r.D, rb, n_own,
                       stg + (size_t)s * 8 * kThreads);
        }
        cp_async_commit();
      }
      if (tid == 0) ss.recomb_pre = 1;
    }
    nbar_sync(kBarGroup, kCtlThreads);
    nbar_sync(kBarScal, kCtlThreads);
    if (!ss.ctl_ok || ss.code1 == 2) {
      cp_async_wait<0>();
      if (ss.ctl_ok && tid == 0) flag_nonfinite(p);
      return false;
    }
  }
  c.g.phase = ss.grp.phase;  // the group state goes back to every thread's context
  c.g.epoch = ss.grp.epoch;
  c.g.skip_arrival = ss.grp.skip_arrival;
  c.g.iseq = ss.grp.iseq;
  if (tid < 32) lzf_build_T(ss, m);
  return true;
}

// The control warp of the headline kernel (threads kThreads .. kThreads + 31): serves the group
// sums of lanczos_res64b until the workers send kCtlExit.  For Lanczos step k it takes the
// workers' warp partials (kBarPost), adds the CTA's share to the group's fixed-point sums,
// arrives at the group barrier -- the release waits for the block's W_{k+1} stores to drain --
// and waits for the group (kBarGroup); then, while the workers read the partner blocks of
// W_{k+1}, it reads the totals and forms alpha_k, b_{k+1} and the scalars of step k + 1
// (kBarScal).  Every step handed over is answered at both barriers, also when the group aborts.
__device__ __noinline__ void res64b_control(SmemSlice& ss) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    nbar_sync(kBarPost, kCtlThreads);
    const int cmd = ss.ctl_cmd;
    if (cmd == kCtlExit) return;
    const int k = cmd & (kCtlLast - 1);
    const bool last = (cmd & kCtlLast) != 0;
    Group& g = ss.grp;
    ctl_add_partials<3>(g, ss.red, kThreads / 32, ss.r.fscale);
    bool ok = true;
    if (lane == 0) {
      ctl_arrive(g);
      ok = ctl_wait(g);
      ss.ctl_ok = ok ? 1 : 0;
    }
    __syncwarp();
    nbar_arrive(kBarGroup, kCtlThreads);
    if (lane == 0 && ok) {
      FF tot[3];
      if (!fix_totals<3>(g, ss.red, fix_load(g), ss.r.finv, tot)) {
        ss.code1 = 2;
      } else {
        const FF b2 = lzf_after_reduce(ss, k, last, tot);
        if (ss.code1 == 0) lzf_finish_step(ss, k, last, b2, ss.r.bdtol, ss.r.amax, ss.r.bmax);
      }
    }
    __syncwarp();
    nbar_arrive(kBarScal, kCtlThreads);
  }
}

// ---------------------------------------------------------------- complex64 streaming path
// For chains whose tiles do not stay on chip (more than two 4096-amplitude tiles per CTA), every
// Lanczos step streams each own tile through the SM.  Same recurrence and global layout as
// lanczos_generic (basis of normalised v_k, W ping-pong, X scratch), but a thread owns amplitude
// PAIRS 2q, 2q+1 with q = tid + 512 g, g < 4, so that every block it needs -- its own W_k, X_{k-1},
// v_{k-1} and, element for element, the partner blocks of W_k -- arrives by 16-byte asynchronous
// copies (cp.async.cg) of exactly the granules it will read.  The copies run kStrDepth blocks
// ahead through a per-thread ring in shared memory: no block barrier, no registers held, and no
// single copy engine to queue behind.  Only the stencil's neighbour reads need one barrier per tile.

// One block of a tile's stream: granule g of the own tile (bit g of gmask) reads granule g ^ gx
// of the source tile starting at `src`.
struct StrBlk {
  const float2* src;
  unsigned gmask;
  int gx;
};

// Partner blocks of the tile at `base` (for W = vector w): bond 11 (own half h = 1 - bt against
// half bt of tile base ^ 2^12: granules g with bit 1 = h, source granule g ^ 2), the antiparallel
// bonds b >= 12 (tile base ^ (3 << b)), an Sx control on a site >= 12 (tile base ^ (1 << s),
// weight of the control).  str_partners returns their number; str_partner the n-th of them.
__device__ __forceinline__ unsigned str_outer(size_t base, int L1) {
  unsigned act = 0;
  for (int b = 12; b < L1; ++b)
    if (((base >> b) ^ (base >> (b + 1))) & 1u) act |= 1u << (b - 12);
  return act;
}
__device__ __forceinline__ int str_partners(size_t base, int L1, bool sx12) {
  return ((L1 > 11) ? 1 : 0) + __popc(str_outer(base, L1)) + (sx12 ? 1 : 0);
}
__device__ __forceinline__ StrBlk str_partner(size_t base, const float2* w, int L1, int hs, bool sx12, int n,
                                              bool& is_ctrl) {
  is_ctrl = false;
  if (L1 > 11) {
    if (n == 0) {
      const unsigned h = 1u - (unsigned)((base >> 12) & 1u);
      return {w + (base ^ ((size_t)1 << 12)), h ? 0xcu : 0x3u, 2};
    }
    --n;
  }
  unsigned act = str_outer(base, L1);
  const int na = __popc(act);
  if (n < na) {
    for (int i = 0; i < n; ++i) act &= act - 1;
    const int b = 12 + __ffs(act) - 1;
    return {w + (base ^ ((size_t)3 << b)), 0xfu, 0};
  }
  is_ctrl = sx12;
  return {w + (base ^ ((size_t)1 << hs)), 0xfu, 0};
}

// This thread's copies of block `bk` into ring stage st: stage layout [kStrDepth][4][512] float4.
__device__ __forceinline__ void str_issue(float4* ring, int st, const StrBlk& bk) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int g = 0; g < 4; ++g)
    if ((bk.gmask >> g) & 1u)
      cp_async16(ring + (st * 4 + g) * kThreads + tid, bk.src + 2 * (size_t)(tid + ((g ^ bk.gx) << 9)));
}

// The stream of one step: for every own tile c (in order) its partner blocks, then X_{k-1}
// and v_{k-1} (k > 0), then W_k.  StrCursor walks it; both the issuer (kStrDepth blocks ahead)
// and the consumer use one, all threads identically.
struct StrStep {
  const float2* w;      // W_k (all tiles)
  const float2* x;      // X_{k-1}
  const float2* vprev;  // v_{k-1} (k = 1: psi, scaled on use)
  int k, L1, hs, n_own;
  bool sx12;
};
struct StrCursor {
  int c, b, nb;  // tile, block within the tile, blocks of the tile
  size_t base;
};
__device__ __forceinline__ int str_nblk(const StrStep& S, size_t base) {
  return str_partners(base, S.L1, S.sx12) + (S.k > 0 ? 3 : 1);
}
__device__ __forceinline__ void str_cursor_tile(const Ctx<float2>& c, const StrStep& S, StrCursor& u) {
  if (u.c < S.n_own) {
    u.base = c.tile_base(u.c);
    u.nb = str_nblk(S, u.base);
  }
}
// Block b of the tile at `base`: partners first, then (k > 0) X and V, then W.
__device__ __forceinline__ StrBlk str_block(const StrStep& S, size_t base, int b) {
  const int np = str_partners(base, S.L1, S.sx12);
  if (b < np) {
    bool ctrl;
    return str_partner(base, S.w, S.L1, S.hs, S.sx12, b, ctrl);
  }
  b -= np;
  if (S.k == 0) return {S.w + base, 0xfu, 0};
  if (b == 0) return {S.x + base, 0xfu, 0};
  if (b == 1) return {S.vprev + base, 0xfu, 0};
  return {S.w + base, 0xfu, 0};
}
// Issuer: copy the block under the cursor (if the step has one left) and advance; one commit
// group per call, empty past the end, so that every consumed block is exactly kStrDepth - 1
// groups behind the newest.
__device__ __forceinline__ void str_issue_next(const Ctx<float2>& c, const StrStep& S, StrCursor& u, float4* ring,
                                               int& slot) {
  if (u.c < S.n_own) {
    str_issue(ring, slot, str_block(S, u.base, u.b));
    if (++u.b == u.nb) {
      ++u.c;
      u.b = 0;
      str_cursor_tile(c, S, u);
    }
  }
  cp_async_commit();
  slot = (slot + 1 == kStrDepth) ? 0 : slot + 1;
}

__device__ __forceinline__ float4 f4fma(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float4 f4add(float4 x, float4 y) {
  return make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w);
}
__device__ __forceinline__ float4 f4scale(float a, float4 x) { return make_float4(a * x.x, a * x.y, a * x.z, a * x.w); }
__device__ __forceinline__ float4 f4zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// Consume the next ring stage: wait until this thread's copies of it have landed.
__device__ __forceinline__ const float4* str_wait(const float4* ring, int slot) {
  cp_async_wait<kStrDepth - 1>();
  return ring + slot * 4 * kThreads + threadIdx.x;
}

// Complex64 streaming Lanczos loop of one slice (see above).  Scalars, reductions and the
// breakdown handling are those of lanczos_generic.
__device__ __noinline__ bool lanczos_str64(Ctx<float2>& c, const float2* src, double nrm_src, double uj) {
  const EvalParams& p = *c.p;
  SmemSlice& ss = *c.ss;
  constexpr int NT = kThreads;
  const int m = p.m;
  const int tid = threadIdx.x;
  const float hxy = (float)(0.5 * p.Jxy), qz = (float)(0.25 * p.Jz);
  const float cu_sx = (float)(0.5 * uj * p.hc_amp), cu_sz = (float)(uj * p.hc_amp);
  const unsigned mk = (unsigned)p.hc_mask;
  const bool hc_sx = (p.hc_kind == KG_HC_SX_SITE);
  const int hs = p.hc_site, L1 = p.L - 1;
  const unsigned maskL1 = c.maskL1;
  const size_t D = c.D;
  float4* sv4 = reinterpret_cast<float4*>(c.sv[0]);  // [kStrSvBufs][2048] pairs: v_k of the tile in hand
  float4* ring = sv4 + kStrSvBufs * 2048;            // [kStrDepth][4][512] per-thread copy ring
  float2* basis = (float2*)p.basis;                  // slot k at basis + (k - 1) D
  float2* wb = (float2*)p.wbuf;
  float2* xb = (float2*)p.xbuf;
  double amax = 0.0, bmax = 0.0;  // thread 0: running maxima for the breakdown test
  if (tid == 0) lz_init(ss, nrm_src, m);
  wsync();
  if (ss.meff == 0) return true;
  StrStep S;
  S.L1 = L1;
  S.hs = hs;
  S.n_own = c.n_own;
  S.sx12 = hc_sx && hs >= 12;
  for (int k = 0; k < m; ++k) {
    const bool last = (k == m - 1);
    S.k = k;
    S.w = (k == 0) ? src : wb + (size_t)(k & 1) * D;
    S.x = xb;
    S.vprev = (k <= 1) ? src : basis + (size_t)(k - 2) * D;
    float2* vslot = (k == 0) ? nullptr : basis + (size_t)(k - 1) * D;  // v_k
    float2* wdst = last ? nullptr : wb + (size_t)((k + 1) & 1) * D;    // W_{k+1}
    const float ap = ss.f_ap, ib = ss.f_ib, bk = ss.f_bk;
    const float vsc = (k == 1) ? ss.f_ib0 : 1.f;  // slot 0 is psi itself: v_0 = psi / b_0
    StrCursor iu{0, 0, 0, 0};
    str_cursor_tile(c, S, iu);
    int islot = 0, cslot = 0;
    for (int d = 0; d < kStrDepth; ++d) str_issue_next(c, S, iu, ring, islot);
    float acc_a = 0.f, acc_n = 0.f, acc_q = 0.f;
    for (int ct = 0; ct < S.n_own; ++ct) {
      const size_t base = c.tile_base(ct);
      const int np = str_partners(base, L1, S.sx12);
      // ---- partner sums of W_k, block by block
      float4 xs[4];
#pragma unroll
      for (int g = 0; g < 4; ++g) xs[g] = f4zero();
      for (int b = 0; b < np; ++b) {
        bool ctrl;
        const StrBlk blk = str_partner(base, S.w, L1, hs, S.sx12, b, ctrl);
        const float wg = ctrl ? cu_sx : hxy;
        const float4* q = str_wait(ring, cslot);
#pragma unroll
        for (int g = 0; g < 4; ++g)
          if ((blk.gmask >> g) & 1u) xs[g] = f4fma(wg, q[g * NT], xs[g]);
        str_issue_next(c, S, iu, ring, islot);
        cslot = (cslot + 1 == kStrDepth) ? 0 : cslot + 1;
      }
      // ---- own blocks, each folded in as it arrives: X_{k-1} (X_k = (XS_k - alpha X_{k-1}) / b_k),
      //      v_{k-1}, W_k (v_k = (W_k - alpha v_{k-1}) / b_k; x <- X_k - b_k v_{k-1}, the part of
      //      W_{k+1} that needs no neighbour)
      float4* sv = sv4 + (ct % kStrSvBufs) * 2048;
      float4 x[4], vp[4];
      if (k > 0) {
        const float4* q = str_wait(ring, cslot);
#pragma unroll
        for (int g = 0; g < 4; ++g) x[g] = f4scale(ib, f4fma(-ap, q[g * NT], xs[g]));
        str_issue_next(c, S, iu, ring, islot);
        cslot = (cslot + 1 == kStrDepth) ? 0 : cslot + 1;
        q = str_wait(ring, cslot);
#pragma unroll
        for (int g = 0; g < 4; ++g) vp[g] = f4scale(vsc, q[g * NT]);
        str_issue_next(c, S, iu, ring, islot);
        cslot = (cslot + 1 == kStrDepth) ? 0 : cslot + 1;
      } else {
#pragma unroll
        for (int g = 0; g < 4; ++g) x[g] = f4scale(ib, xs[g]);
      }
      if (kStrSvBufs == 1) wsync();  // the previous tile's stencil is done with sv
      {
        const float4* q = str_wait(ring, cslot);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const int qi = tid + g * NT;
          const float4 w = q[g * NT];
          float4 v;
          if (k == 0) {
            v = f4scale(ib, w);
          } else {
            v = f4scale(ib, f4fma(-ap, vp[g], w));
            __stcg(reinterpret_cast<float4*>(vslot + base) + qi, v);
          }
          sv[qi] = v;
          if (!last) __stcg(reinterpret_cast<float4*>(xb + base) + qi, x[g]);
          if (k > 0) x[g] = f4fma(-bk, vp[g], x[g]);
        }
        str_issue_next(c, S, iu, ring, islot);
        cslot = (cslot + 1 == kStrDepth) ? 0 : cslot + 1;
      }
      wsync();  // the tile's v_k is complete in shared memory
      float4 vv[4];
#pragma unroll
      for (int g = 0; g < 4; ++g) vv[g] = sv[tid + g * NT];
      // ---- stage 2: W_{k+1} = H v_k - b_k v_{k-1} (the latter already in x), partial sums
      float4 h[4];
#pragma unroll
      for (int g = 0; g < 4; ++g) h[g] = f4zero();
      {  // bond 0: bits 0 (pair element) and 1 (bit 0 of tid); partner pair of tid ^ 1, swapped
        const bool q0 = (tid & 1) != 0;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const float4 Q = sv[(tid ^ 1) + g * NT];
          if (!q0) {
            h[g].z += Q.x;
            h[g].w += Q.y;
          } else {
            h[g].x += Q.z;
            h[g].y += Q.w;
          }
        }
      }
#pragma unroll
      for (int b = 1; b <= 8; ++b) {  // bonds 1..8: bits b-1, b of tid
        if (((tid >> (b - 1)) ^ (tid >> b)) & 1) {
#pragma unroll
          for (int g = 0; g < 4; ++g) h[g] = f4add(h[g], sv[(tid ^ (3 << (b - 1))) + g * NT]);
        }
      }
      {  // bond 9: bit 8 of tid, bit 0 of g
        const int t8 = (tid >> 8) & 1;
#pragma unroll
        for (int g = 0; g < 4; ++g)
          if (t8 != (g & 1)) h[g] = f4add(h[g], sv[(tid ^ 256) + (g ^ 1) * NT]);
      }
#pragma unroll
      for (int g = 0; g < 4; ++g)  // bond 10: bits 0, 1 of g
        if ((g ^ (g >> 1)) & 1) h[g] = f4add(h[g], vv[g ^ 3]);
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const int q = tid + g * NT;
        float4 cx = f4zero();  // in-tile Sx control partner of each element
        if (hc_sx && hs < 12) {
          if (hs == 0) {
            cx = make_float4(vv[g].z, vv[g].w, vv[g].x, vv[g].y);
          } else {
            cx = sv[q ^ (1 << (hs - 1))];
          }
        }
        float d[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const unsigned gi = (unsigned)(base + 2 * (size_t)q + e);
          const unsigned xg = (gi ^ (gi >> 1)) & maskL1;
          d[e] = qz * (float)(L1 - 2 * __popc(xg));
          if (!hc_sx) d[e] += cu_sz * 0.5f * (float)(__popc(mk) - 2 * __popc(gi & mk));
        }
        float4 wn;
        wn.x = d[0] * vv[g].x + hxy * h[g].x + x[g].x + cu_sx * cx.x;
        wn.y = d[0] * vv[g].y + hxy * h[g].y + x[g].y + cu_sx * cx.y;
        wn.z = d[1] * vv[g].z + hxy * h[g].z + x[g].z + cu_sx * cx.z;
        wn.w = d[1] * vv[g].w + hxy * h[g].w + x[g].w + cu_sx * cx.w;
        acc_a += vv[g].x * wn.x + vv[g].y * wn.y + vv[g].z * wn.z + vv[g].w * wn.w;
        acc_n += wn.x * wn.x + wn.y * wn.y + wn.z * wn.z + wn.w * wn.w;
        acc_q += vv[g].x * vv[g].x + vv[g].y * vv[g].y + vv[g].z * vv[g].z + vv[g].w * vv[g].w;
        if (!last) __stcg(reinterpret_cast<float4*>(wdst + base) + q, wn);
      }
    }
    c.mark(0);
    float acc[3] = {acc_a, acc_n, acc_q};
    double out[3];
    if (!group_reduce<3>(c.g, ss.red, acc, out)) return false;
    c.mark(2);
    if (tid == 0) lz_after_reduce(ss, k, last, out);
    wsync();
    const int code = ss.code1;
    if (code == 2) {
      if (tid == 0) flag_nonfinite(p);
      return false;
    }
    if (code == 1) {
      // near an invariant subspace: ||W_{k+1} - alpha_k v_k||^2 explicitly (one more reduction)
      float n1[1] = {0.f};
      const float ra = ss.f_alpha;
      for (int ct = 0; ct < S.n_own; ++ct) {
        const size_t base = c.tile_base(ct);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const int q = tid + g * NT;
          const float4 wn = __ldcg(reinterpret_cast<const float4*>(wdst + base) + q);
          const float4 v = (k == 0) ? f4scale(ib, __ldcg(reinterpret_cast<const float4*>(src + base) + q))
                                    : __ldcg(reinterpret_cast<const float4*>(vslot + base) + q);
          const float4 r = f4fma(-ra, v, wn);
          n1[0] += r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w;
        }
      }
      double o1[1];
      if (!group_reduce<1>(c.g, ss.red, n1, o1)) return false;
      if (tid == 0) ss.s_b2 = o1[0];
    }
    if (tid == 0) lz_finish_step(ss, k, last, p.bd_tol, amax, bmax);
    wsync();
    c.mark(3);
    if (ss.stop) break;
  }
  return true;
}

// One Krylov step src -> dst (App. A): Lanczos basis, small exponential, recombination.
// tau = sigma * dt.  Returns false on abort.
template <class V, class A, int APT, int TPC, bool RES, int MODE>
__device__ __noinline__ bool krylov_slice(Ctx<V>& c, const V* src, double nrm_src, double uj, double tau, V* dst,
                                          int extra, const V* psi_other, double& nrm_dst, double2& e) {
  bool ok;
  if constexpr (MODE == kModeResident64) ok = lanczos_res64(c, src, nrm_src, uj);
  else if constexpr (MODE == kModeResident64b) ok = lanczos_res64b(c, src, nrm_src, uj);
  else if constexpr (MODE == kModeStream64) ok = lanczos_str64(c, src, nrm_src, uj);
  else ok = lanczos_generic<V, A, APT, TPC, RES>(c, src, nrm_src, uj);
  if (!ok) return false;
  return finish_slice<V, A, APT, MODE == kModeResident64 || MODE == kModeResident64b>(c, src, nrm_src, tau, dst, extra,
                                                                                     psi_other, nrm_dst, e);
}

// Another step of length tau from the Krylov basis the last krylov_slice built (the basis
// slots and T are still in place): psi(tau) at an interior quadrature node of the slice
// (KG_GRAD_EXACT), with the same fused overlaps.
template <class V, class A, int APT, int TPC, bool RES, int MODE>
__device__ __noinline__ bool interior_step(Ctx<V>& c, const V* src, double nrm_src, double tau, V* dst, int extra,
                                           const V* psi_other, double2& e) {
  double nrm_dst;
  return finish_slice<V, A, APT, MODE == kModeResident64 || MODE == kModeResident64b>(c, src, nrm_src, tau, dst, extra,
                                                                                     psi_other, nrm_dst, e, true);
}

// chi_N = beta f, ||chi_N||, and G_N = 2 dt Im <chi_N|Hc|psi_N>.
template <class V>
__device__ bool init_costate(Ctx<V>& c, double2 beta, V* chi, const V* psiN, double& nrm, double& gim) {
  using R = typename VecTraits<V>::R;
  const EvalParams& p = *c.p;
  double acc[2] = {0.0, 0.0};
  for (int ct = 0; ct < c.n_own; ++ct) {
    const size_t base = c.tile_base(ct);
    for (int li = threadIdx.x; li < c.tile; li += nwork()) {
      const size_t gi = base + li;
      const double2 f = reinterpret_cast<const double2*>(p.target)[gi];
      const double yr = beta.x * f.x - beta.y * f.y, yi = beta.x * f.y + beta.y * f.x;
      const V y = vmake<V>((R)yr, (R)yi);
      stv(chi + gi, y);
      acc[0] += (double)y.x * y.x + (double)y.y * y.y;
      V q;
      if (p.hc_kind == KG_HC_SX_SITE) {
        q = ldv(psiN + (gi ^ ((size_t)1 << p.hc_site)));
        q.x *= (R)(0.5 * p.hc_amp);
        q.y *= (R)(0.5 * p.hc_amp);
      } else {
        const unsigned mk = (unsigned)p.hc_mask;
        const R dz = (R)(p.hc_amp * 0.5 * (double)(__popc(mk) - 2 * __popc((unsigned)gi & mk)));
        q = ldv(psiN + gi);
        q.x *= dz;
        q.y *= dz;
      }
      acc[1] += (double)(y.x * q.y - y.y * q.x);
    }
  }
  double out[2];
  if (!group_reduce<2>(c.g, c.ss->red, acc, out)) return false;
  nrm = sqrt(fmax(out[0], 0.0));
  gim = out[1];
  return true;
}

// psi_0 <- psi0 (rounded to V), ||psi_0||.
template <class V>
__device__ bool init_state(Ctx<V>& c, V* dst, double& nrm) {
  using R = typename VecTraits<V>::R;
  const EvalParams& p = *c.p;
  double acc[1] = {0.0};
  for (int ct = 0; ct < c.n_own; ++ct) {
    const size_t base = c.tile_base(ct);
    for (int li = threadIdx.x; li < c.tile; li += nwork()) {
      const size_t gi = base + li;
      const double2 a = reinterpret_cast<const double2*>(p.psi0)[gi];
      const V y = vmake<V>((R)a.x, (R)a.y);
      stv(dst + gi, y);
      acc[0] += (double)y.x * y.x + (double)y.y * y.y;
    }
  }
  double out[1];
  if (!group_reduce<1>(c.g, c.ss->red, acc, out)) return false;
  nrm = sqrt(fmax(out[0], 0.0));
  return true;
}

// Storage of psi_j.  ckpt == 0: traj[j].  ckpt == C: checkpoints traj[j/C] for j % C == 0,
// psi_N in traj[N/C + 1] when N % C != 0, everything else in two forward temporaries
// seg[C-1], seg[C] (alternating) or, during the backward sweep, in seg[j - a - 1] for the
// segment (a, b] being recomputed.
template <class V>
__device__ __forceinline__ V* fwd_slot(const Ctx<V>& c, int j) {
  const EvalParams& p = *c.p;
  V* traj = (V*)p.traj;
  if (p.ckpt == 0) return traj + (size_t)j * c.D;
  const int C = p.ckpt;
  if (j % C == 0) return traj + (size_t)(j / C) * c.D;
  if (j == p.N) return traj + (size_t)(p.N / C + 1) * c.D;
  return (V*)p.seg + (size_t)(C - 1 + (j & 1)) * c.D;
}

// Interior node a (0, 1) of the 4-point Gauss-Lobatto rule on [0, dt]: (1 -+ 1/sqrt 5) dt / 2.
__device__ __forceinline__ double lobatto_node(double dt, int a) {
  const double s1 = 0.5 * dt * (1.0 - 0.4472135954999579);  // 1/sqrt(5)
  return (a == 0) ? s1 : dt - s1;
}

// One whole evaluation (forward sweep, overlap, co-state sweep, gradient) of problem p by the
// group of `size` CTAs in which this CTA has rank `rank`.  Returns false if the group aborted.
template <class V, class A, int APT, int TPC, bool RES, int MODE>
__device__ __noinline__ bool run_eval(const EvalParams& p, int rank, int size, SmemSlice& ss,
                                      unsigned char* smem_dyn, unsigned& lz_count) {
  Ctx<V> c;
  c.p = &p;
  c.g.rank = rank;
  c.g.size = size;
  c.g.bar = p.bar;
  c.g.red = p.red;
  c.g.ctrl = p.ctrl;
  c.g.wait_limit_ns = p.wait_limit_ns;
  c.g.phase = 0;
  c.g.epoch = 0;
  c.g.skip_arrival = (p.debug_fault == 1 && rank == 0) ? 1 : 0;
  c.g.stride = p.red_stride;
  c.g.iring = p.iring;
  c.g.iseq = 0u;
  c.ss = &ss;
  c.t = p.t_bits;
  c.tile = 1 << p.t_bits;
  constexpr int NB = RES ? TPC : 1;
  c.sv[0] = reinterpret_cast<V*>(smem_dyn);
  c.sv[1] = c.sv[0] + (size_t)NB * c.tile;
  c.sx = c.sv[1] + (size_t)NB * c.tile;
  c.D = (size_t)1 << p.L;
  c.ntiles = (int)(c.D >> p.t_bits);
  // Pairs (resident paths with two tiles per CTA, and the complex64 streaming path): every pair
  // has the same number of cross-tile partner blocks, so dealing pairs balances the CTAs.
  c.paired = (c.ntiles >= 2 && (2 * c.g.size == c.ntiles || MODE == kModeStream64));
  if (c.paired) {
    const int npairs = c.ntiles / 2;
    c.n_own = (c.g.rank < npairs) ? 2 * ((npairs - c.g.rank + c.g.size - 1) / c.g.size) : 0;
  } else {
    c.n_own = (c.ntiles - c.g.rank + c.g.size - 1) / c.g.size;
  }
  c.alt = 0x55555555u & (unsigned)(c.ntiles - 1);
  c.maskL1 = (p.L >= 2) ? ((1u << (p.L - 1)) - 1u) : 0u;
  c.err_max = 0.0;
  c.breakdowns = 0;
  c.lz_count = lz_count;
  c.tm = ss.tmem_base + ((((unsigned)threadIdx.x >> 5) & 3u) << 21) + 128u * ((unsigned)threadIdx.x >> 7);
  c.prof_on = (p.prof != nullptr && rank == 0);
  const long long prof_t0 = clock64();
  if (c.prof_on && threadIdx.x == 0) ss.prof_last = prof_t0;
#pragma unroll
  for (int i = 0; i < 8; ++i)
    if (c.prof_on && threadIdx.x == 0) ss.prof_acc[i] = 0;
  const bool lead = (rank == 0 && threadIdx.x == 0);
  if (threadIdx.x == 0) ss.recomb_pre = 0;

  // ---- forward sweep (Alg. "Basic GRAPE", step 4)
  double nrm_prev;
  if (!init_state<V>(c, fwd_slot<V>(c, 0), nrm_prev)) return false;
  if (p.debug_fault == 2 && rank == 0) c.g.skip_arrival = 1;  // at the first Lanczos step's barrier
  if (lead) p.nrm[0] = nrm_prev;
  c.mark(6);
  double2 beta = make_double2(0.0, 0.0);
  for (int j = 1; j <= p.N; ++j) {
    double nrm_new;
    double2 e;
    const int extra = (j == p.N) ? kExtraOverlapTarget : kExtraNone;
    if (!krylov_slice<V, A, APT, TPC, RES, MODE>(c, fwd_slot<V>(c, j - 1), nrm_prev, p.u[j - 1], p.dt, fwd_slot<V>(c, j),
                                           extra, nullptr, nrm_new, e))
      return false;
    if (p.grad_mode == KG_GRAD_EXACT) {  // psi at the slice's interior quadrature nodes (ckpt == 0)
      for (int a = 0; a < 2; ++a) {
        double2 ei;
        V* d = (V*)p.tint + (size_t)(2 * (j - 1) + a) * c.D;
        if (!interior_step<V, A, APT, TPC, RES, MODE>(c, fwd_slot<V>(c, j - 1), nrm_prev, lobatto_node(p.dt, a), d,
                                                      kExtraNone, nullptr, ei))
          return false;
      }
    }
    if (lead) p.nrm[j] = nrm_new;
    nrm_prev = nrm_new;
    if (j == p.N) beta = e;
  }
  if (lead) {
    p.scal[kScBetaRe] = beta.x;
    p.scal[kScBetaIm] = beta.y;
    p.scal[kScNormFinal] = nrm_prev;
    p.fid[0] = beta.x * beta.x + beta.y * beta.y;
  }

  if (p.grad_mode != KG_GRAD_NONE) {
    // ---- backward sweep (Alg. "Basic GRAPE", steps 5-7)
    V* chi[2] = {(V*)p.chi, (V*)p.chi + c.D};
    const V* psiN = fwd_slot<V>(c, p.N);
    double nchi, gim;
    if (!init_costate<V>(c, beta, chi[0], psiN, nchi, gim)) return false;
    if (lead) p.G[p.N] = 2.0 * p.dt * gim;
    c.mark(6);
    int cur = 0;
    const int C = p.ckpt;
    const int nseg = (C > 0) ? (p.N + C - 1) / C : 1;
    for (int sgi = nseg - 1; sgi >= 0; --sgi) {
      const int a = (C > 0) ? sgi * C : 0;
      const int b = (C > 0) ? min(a + C, p.N) : p.N;
      if (C > 0) {
        // recompute psi_{a+1..b-1} of this segment from its checkpoint
        const V* prev = (V*)p.traj + (size_t)(a / C) * c.D;
        double np = p.nrm[a];
        for (int i = a + 1; i < b; ++i) {
          V* d = (V*)p.seg + (size_t)(i - a - 1) * c.D;
          double nn;
          double2 e;
          if (!krylov_slice<V, A, APT, TPC, RES, MODE>(c, prev, np, p.u[i - 1], p.dt, d, kExtraNone, nullptr, nn, e))
            return false;
          prev = d;
          np = nn;
        }
      }
      for (int j = b; j > a; --j) {
        const V* psi_jm1;
        if (C == 0) psi_jm1 = (V*)p.traj + (size_t)(j - 1) * c.D;
        else if (j - 1 == a) psi_jm1 = (V*)p.traj + (size_t)(a / C) * c.D;
        else psi_jm1 = (V*)p.seg + (size_t)(j - 1 - a - 1) * c.D;
        double nn;
        double2 e;
        if (!krylov_slice<V, A, APT, TPC, RES, MODE>(c, chi[cur], nchi, p.u[j - 1], -p.dt, chi[cur ^ 1],
                                               kExtraGradOverlap, psi_jm1, nn, e))
          return false;
        if (lead) p.G[j - 1] = 2.0 * p.dt * e.x;
        if (p.grad_mode == KG_GRAD_EXACT) {
          // chi at t_{j-1} + s = exp(+i (dt - s) H_j) chi_j, overlapped with the stored psi there
          for (int a = 0; a < 2; ++a) {
            double2 ei;
            const V* psi_s = (const V*)p.tint + (size_t)(2 * (j - 1) + a) * c.D;
            if (!interior_step<V, A, APT, TPC, RES, MODE>(c, chi[cur], nchi, -(p.dt - lobatto_node(p.dt, a)),
                                                          (V*)p.wbuf, kExtraGradOverlap, psi_s, ei))
              return false;
            if (lead) p.Gi[2 * (j - 1) + a] = 2.0 * p.dt * ei.x;
          }
        }
        cur ^= 1;
        nchi = nn;
      }
    }
  }
  // ---- outputs (rank 0)
  if (rank == 0) {
    wsync();
    if (p.grad_mode != KG_GRAD_NONE) {
      for (int j = threadIdx.x; j < p.N; j += nwork()) {
        const double gl = p.G[j], gr = p.G[j + 1];
        if (p.grad_mode == KG_GRAD_EXACT)  // Gauss-Lobatto weights 1/12, 5/12, 5/12, 1/12
          p.grad[j] = (gl + gr) / 12.0 + 5.0 * (p.Gi[2 * j] + p.Gi[2 * j + 1]) / 12.0;
        else
          p.grad[j] = (p.grad_mode == KG_GRAD_ZEROTH) ? gr : 0.5 * (gl + gr);
      }
    }
    double em = (threadIdx.x < 32) ? warp_max(c.err_max) : 0.0;
    if (threadIdx.x == 0) {
      p.scal[kScErrMax] = em;
      p.scal[kScBreakdowns] = (double)c.breakdowns;
      if (c.prof_on) {
        c.mark(6);
        for (int i = 0; i < 7; ++i) p.prof[i] = ss.prof_acc[i];
        p.prof[7] = clock64() - prof_t0;
      }
    }
  }
  lz_count = c.lz_count;
  return true;
}

// Shared prologue/epilogue of the kernels: bulk-copy barriers, and (complex64 resident path)
// the tensor memory of the CTA, allocated by warp 0 and freed by it on every way out.
__device__ __forceinline__ void cta_setup(SmemSlice& ss, bool tmem) {
  if (threadIdx.x == 0) {
    for (int i = 0; i < kLzStages; ++i) mbar_init(&ss.lmbar[i], 1);
    fence_mbar_init();
  }
  if (tmem) {
    if (threadIdx.x < 32) tmem_alloc(&ss.tmem_base, kTmemCols);
    tmem_fence_before_sync();
  }
  __syncthreads();
  if (tmem) tmem_fence_after_sync();
}
__device__ __forceinline__ void cta_teardown(SmemSlice& ss, bool tmem) {
  if (!tmem) return;
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (threadIdx.x < 32) tmem_dealloc(ss.tmem_base, kTmemCols);
}

// Threads per CTA of an evaluation kernel: the headline loop's blocks carry the control warp.
constexpr int eval_threads(int mode) { return mode == kModeResident64b ? kCtlThreads : kThreads; }

template <class V, class A, int APT, int TPC, bool RES, int MODE>
__global__ void __launch_bounds__(eval_threads(MODE), 1) kg_eval_kernel(const __grid_constant__ EvalParams p) {
  extern __shared__ __align__(16) unsigned char smem_dyn[];
  __shared__ SmemSlice ss;
  constexpr bool kTmem = (MODE == kModeResident64 || MODE == kModeResident64b);
  cta_setup(ss, kTmem);
  unsigned lz_count = 0u;  // Lanczos ring copies consumed (stage and phase parity of the ring)
  if constexpr (MODE == kModeResident64b) {
    if (threadIdx.x >= kThreads) {
      res64b_control(ss);
    } else {
      run_eval<V, A, APT, TPC, RES, MODE>(p, blockIdx.x, gridDim.x, ss, smem_dyn, lz_count);
      if (threadIdx.x == 0) ss.ctl_cmd = kCtlExit;  // no step is in flight: every one was answered
      nbar_arrive(kBarPost, kCtlThreads);
    }
  } else {
    run_eval<V, A, APT, TPC, RES, MODE>(p, blockIdx.x, gridDim.x, ss, smem_dyn, lz_count);
  }
  cta_teardown(ss, kTmem);
}

// Many independent problems (complex64) in one cooperative launch.  Every CTA walks its own
// list of items in the order the host scheduled them; a group of CTAs forms for one problem
// and uses its own barrier counter.  Lists are ordered consistently (a global sequence), so a
// CTA waiting in a group only waits for members that will reach that item.
__global__ void __launch_bounds__(kThreads, 1) kg_batch_kernel(const __grid_constant__ BatchParams bp) {
  extern __shared__ __align__(16) unsigned char smem_dyn[];
  __shared__ SmemSlice ss;
  cta_setup(ss, true);
  unsigned lz_count = 0u;  // Lanczos ring copies consumed (stage and phase parity of the ring)
  const int i0 = bp.item_off[blockIdx.x], i1 = bp.item_off[blockIdx.x + 1];
  for (int it = i0; it < i1; ++it) {
    const BatchItem item = bp.items[it];
    EvalParams p = bp.probs[item.problem];
    p.bar = bp.bars + item.group;
    p.red = bp.reds + (size_t)item.group * kBatchRedPerGroup;
    p.red_stride = kBatchMaxGroup;
    p.ctrl = bp.ctrl;
    const int ntiles = 1 << (p.L - p.t_bits);
    bool ok;
    if (ntiles <= 2 * item.size && p.t_bits == 12)
      ok = run_eval<float2, float, 8, 2, true, kModeResident64>(p, item.rank, item.size, ss, smem_dyn, lz_count);
    else if (ntiles <= 2 * item.size)
      ok = run_eval<float2, float, 8, 2, true, kModeGeneric>(p, item.rank, item.size, ss, smem_dyn, lz_count);
    else
      ok = run_eval<float2, float, 8, 1, false, kModeGeneric>(p, item.rank, item.size, ss, smem_dyn, lz_count);
    if (!ok) break;
    wsync();
  }
  cta_teardown(ss, true);
}

size_t batch_smem_bytes() { return (size_t)3 * 2 * 4096 * sizeof(float2); }

cudaError_t launch_batch_kernel(const BatchParams& bp, int ctas, cudaStream_t stream) {
  const size_t smem = batch_smem_bytes();
  cudaError_t err = cudaFuncSetAttribute(kg_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kg_batch_kernel, bp);
}

cudaError_t batch_kernel_max_ctas(int* out) {
  const size_t smem = batch_smem_bytes();
  cudaError_t err = cudaFuncSetAttribute(kg_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kg_batch_kernel, kThreads, smem);
  if (err != cudaSuccess) return err;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *out = per_sm * sms;
  return cudaSuccess;
}

// ---------------------------------------------------------------- host-side launch helpers
struct KernelChoice {
  const void* fn;
  size_t smem;
  int threads;
};

template <class V, class A, int APT, int TPC, bool RES, int MODE>
static KernelChoice choice(int t_bits) {
  constexpr int NB = RES ? TPC : 1;
  // complex64 streaming: two v_k tiles for the stencil plus the per-thread copy ring
  const size_t smem = (MODE == kModeStream64)      ? kStrSmemBytes
                      : (MODE == kModeResident64b) ? kRes64bSmemBytes
                                                   : (size_t)(RES ? 3 : 2) * NB * ((size_t)1 << t_bits) * sizeof(V);
  return {(const void*)kg_eval_kernel<V, A, APT, TPC, RES, MODE>, smem, eval_threads(MODE)};
}

// Variants: complex64 resident with full 4096-amplitude tiles (specialised loop), complex64
// resident (<= 2 tiles of <= 4096 amplitudes per CTA), complex64 streaming (specialised loop
// for 4096-amplitude tiles, generic otherwise), complex128 streaming (tiles of <= 2048
// amplitudes).
static KernelChoice pick(int prec, int variant, int t_bits) {
  if (prec == KG_PREC_C128) return choice<double2, double, 4, 1, false, kModeGeneric>(t_bits);
  if (variant == kVariantGenericStream) return choice<float2, float, 8, 1, false, kModeGeneric>(t_bits);
  if (variant == kVariantResidentFull) return choice<float2, float, 8, 2, true, kModeResident64b>(t_bits);
  if (variant == kVariantResident) return choice<float2, float, 8, 2, true, kModeGeneric>(t_bits);
  if (t_bits == 12) return choice<float2, float, 8, 1, false, kModeStream64>(t_bits);
  return choice<float2, float, 8, 1, false, kModeGeneric>(t_bits);
}

int eval_kernel_threads(int prec, int variant, int t_bits) { return pick(prec, variant, t_bits).threads; }

int max_tile_bits(int prec) { return prec == KG_PREC_C128 ? kLogNT + 2 : kLogNT + 3; }
int resident_tiles_per_cta(int prec) { return prec == KG_PREC_C128 ? 0 : 2; }

cudaError_t launch_eval_kernel(int prec, int variant, const EvalParams& p, int ctas, cudaStream_t stream) {
  KernelChoice k = pick(prec, variant, p.t_bits);
  cudaError_t err = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
  if (err != cudaSuccess) return err;
  EvalParams pc = p;
  void* args[] = {&pc};
  return cudaLaunchCooperativeKernel(k.fn, dim3(ctas), dim3(k.threads), args, k.smem, stream);
}

cudaError_t eval_kernel_max_ctas(int prec, int variant, int t_bits, int* out) {
  KernelChoice k = pick(prec, variant, t_bits);
  cudaError_t err = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fn, k.threads, k.smem);
  if (err != cudaSuccess) return err;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *out = per_sm * sms;
  return cudaSuccess;
}

}  // namespace kg

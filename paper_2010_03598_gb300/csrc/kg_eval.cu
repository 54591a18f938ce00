// K-GRAPE evaluation kernel: forward Krylov sweep, target overlap, backward co-state
// sweep with per-slice gradient overlaps, all in one cooperative persistent launch.
//
// Work split.  The 2^L amplitudes are cut into tiles of 2^t contiguous amplitudes; the
// CTAs of the group own tiles round robin (tile T -> CTA T mod size).  Each Lanczos step
// of each slice is:
//   phase A (per own tile): stage v_k's tile in shared memory, form
//            w = H_j v_k - b_k v_{k-1} with the matrix-free XXZ stencil (bonds inside the
//            tile from shared memory, bonds that cross into another tile from L2), write w,
//            accumulate <v_k|w>;                                   -> reduce alpha_k
//   phase B (per own tile): w <- w - alpha_k v_k, accumulate ||w||^2 -> reduce b_{k+1}
// (the order of Paige's Lanczos, App. A's Algorithm "Lanczos" with the coefficients
// taken against the updated vector), with v_{k+1} = w / b_{k+1} kept implicit as a
// scale.  After m steps every CTA forms c = exp(-i sigma dt T) e_1 (one warp, FP64) and
// recombines psi' = ||psi|| sum_k c_k v_k for its own tiles (App. A).
#include <cuda_runtime.h>

#include "kg_device.cuh"
#include "kg_launch.h"

namespace kg {

enum ExtraKind { kExtraNone = 0, kExtraOverlapTarget = 1, kExtraGradOverlap = 2 };

struct SmemSlice {
  SmemRed red;
  double alpha[kMaxM];
  double beta[kMaxM + 1];
  double scale[kMaxM];
  double coef_re[kMaxM];
  double coef_im[kMaxM];
  double err;
};

template <class V>
struct Ctx {
  using R = typename VecTraits<V>::R;
  const EvalParams* p;
  Group g;
  SmemSlice* ss;
  V* s_v;          // one tile of the current Lanczos vector
  int t, tile, ntiles;
  size_t D;
  unsigned maskL1;  // bonds 0..L-2 in (i ^ i>>1)
  double err_max;
  int breakdowns;

  __device__ V* basis_slot(int k) const { return (V*)p->basis + (size_t)(k - 1) * D; }
};

template <class V>
__device__ __forceinline__ V vscale(V a, typename VecTraits<V>::R s) { return vmake<V>(a.x * s, a.y * s); }

// (H0 + u Hc) applied to amplitude gi of v, where v's tile is in shared memory.
// Partners outside the tile come from `src` (global, scaled by sk).
template <class V>
__device__ __forceinline__ V apply_H_amp(const Ctx<V>& c, const V* __restrict__ src,
                                         typename VecTraits<V>::R sk, unsigned gi, int li,
                                         typename VecTraits<V>::R hxy, typename VecTraits<V>::R qz,
                                         typename VecTraits<V>::R cu_sx, typename VecTraits<V>::R cu_sz) {
  using R = typename VecTraits<V>::R;
  const EvalParams& p = *c.p;
  const V v = c.s_v[li];
  const unsigned x = (gi ^ (gi >> 1)) & c.maskL1;   // bit b set <=> bits b, b+1 antiparallel
  const int anti = __popc(x);
  // diagonal: Jz/4 per parallel bond, -Jz/4 per antiparallel bond
  R d = qz * (R)((p.L - 1) - 2 * anti);
  R hr = 0, hi = 0;
  const int L1 = p.L - 1;
  const int tin = c.t - 1;  // bonds b < tin stay inside the tile
  for (int b = 0; b < L1; ++b) {
    if ((x >> b) & 1u) {
      V q;
      if (b < tin) q = c.s_v[li ^ (3 << b)];
      else q = vscale(ldv(src + (gi ^ (3u << b))), sk);
      hr += q.x;
      hi += q.y;
    }
  }
  R wr = d * v.x + hxy * hr;
  R wi = d * v.y + hxy * hi;
  if (p.hc_kind == KG_HC_SX_SITE) {
    const int s = p.hc_site;
    V q;
    if (s < c.t) q = c.s_v[li ^ (1 << s)];
    else q = vscale(ldv(src + (gi ^ (1u << s))), sk);
    wr += cu_sx * q.x;
    wi += cu_sx * q.y;
  } else {
    const unsigned mk = (unsigned)p.hc_mask;
    const R dz = (R)0.5 * (R)(__popc(mk) - 2 * __popc(gi & mk));
    wr += cu_sz * dz * v.x;
    wi += cu_sz * dz * v.y;
  }
  return vmake<V>(wr, wi);
}

// One Krylov step src -> dst (App. A).  tau = sigma * dt.  Returns false on abort.
// extra == kExtraOverlapTarget: also e = <f|dst> (f = target, complex128).
// extra == kExtraGradOverlap:   also e.x = Im <dst|Hc|psi_other>.
template <class V, class A>
__device__ bool krylov_slice(Ctx<V>& c, const V* src, double nrm_src, double uj, double tau, V* dst,
                             int extra, const V* psi_other, double& nrm_dst, double2& e) {
  using R = typename VecTraits<V>::R;
  const EvalParams& p = *c.p;
  SmemSlice& ss = *c.ss;
  const int m = p.m;
  const int tid = threadIdx.x, nt = blockDim.x;
  int meff = 0;
  bool broke = false;
  double beta_m = 0.0;
  const R hxy = (R)(0.5 * p.Jxy), qz = (R)(0.25 * p.Jz);
  const R cu_sx = (R)(0.5 * uj * p.hc_amp), cu_sz = (R)(uj * p.hc_amp);

  if (nrm_src > 0.0) {
    if (tid == 0) ss.scale[0] = 1.0 / nrm_src;
    __syncthreads();
    double amax = 0.0, bmax = 0.0;
    meff = m;
    for (int k = 0; k < m; ++k) {
      const bool last = (k == m - 1);
      const V* vk = (k == 0) ? src : c.basis_slot(k);
      const V* vkm1 = (k == 0) ? nullptr : ((k == 1) ? src : c.basis_slot(k - 1));
      V* w_out = last ? nullptr : c.basis_slot(k + 1);
      const R sk = (R)ss.scale[k];
      const R skm1 = (k == 0) ? (R)0 : (R)ss.scale[k - 1];
      const R bk = (k == 0) ? (R)0 : (R)ss.beta[k];
      A acc[3] = {0, 0, 0};
      // ---- phase A: w = H v_k - b_k v_{k-1}
      for (int T = c.g.rank; T < c.ntiles; T += c.g.size) {
        const size_t base = (size_t)T << c.t;
        for (int li = tid; li < c.tile; li += nt) c.s_v[li] = vscale(ldv(vk + base + li), sk);
        __syncthreads();
        for (int li = tid; li < c.tile; li += nt) {
          const unsigned gi = (unsigned)(base + li);
          V w = apply_H_amp<V>(c, vk, sk, gi, li, hxy, qz, cu_sx, cu_sz);
          if (k > 0) {
            const V q = ldv(vkm1 + gi);
            w.x -= bk * (q.x * skm1);
            w.y -= bk * (q.y * skm1);
          }
          const V v = c.s_v[li];
          acc[0] += (A)(v.x * w.x + v.y * w.y);
          if (last) {
            acc[1] += (A)(w.x * w.x + w.y * w.y);
            acc[2] += (A)(v.x * v.x + v.y * v.y);
          } else {
            stv(w_out + gi, w);
          }
        }
        __syncthreads();
      }
      if (!last) {
        double out[1];
        A a1[1] = {acc[0]};
        if (!group_reduce<1>(c.g, ss.red, a1, out)) return false;
        const double alpha = out[0];
        // ---- phase B: w <- w - alpha v_k, ||w||^2
        A n1[1] = {0};
        const R ra = (R)alpha;
        for (int T = c.g.rank; T < c.ntiles; T += c.g.size) {
          const size_t base = (size_t)T << c.t;
          for (int li = tid; li < c.tile; li += nt) {
            const size_t gi = base + li;
            V w = ldv(w_out + gi);
            const V v = ldv(vk + gi);
            w.x -= ra * (v.x * sk);
            w.y -= ra * (v.y * sk);
            stv(w_out + gi, w);
            n1[0] += (A)(w.x * w.x + w.y * w.y);
          }
        }
        double out2[1];
        if (!group_reduce<1>(c.g, ss.red, n1, out2)) return false;
        const double beta = sqrt(fmax(out2[0], 0.0));
        if (!isfinite(alpha) || !isfinite(beta)) {
          if (tid == 0) { atomicCAS(p.ctrl + kCtrlStatus, 0, (int)KG_ERR_NONFINITE); atomicExch(p.ctrl + kCtrlAbort, 1); }
          return false;
        }
        if (tid == 0) ss.alpha[k] = alpha;
        amax = fmax(amax, fabs(alpha));
        if (beta <= p.bd_tol * fmax(1.0, amax + bmax)) {
          meff = k + 1;
          broke = true;
          break;
        }
        bmax = fmax(bmax, beta);
        if (tid == 0) { ss.beta[k + 1] = beta; ss.scale[k + 1] = 1.0 / beta; }
        __syncthreads();
      } else {
        double out[3];
        if (!group_reduce<3>(c.g, ss.red, acc, out)) return false;
        const double alpha = out[0];
        if (!isfinite(alpha) || !isfinite(out[1])) {
          if (tid == 0) { atomicCAS(p.ctrl + kCtrlStatus, 0, (int)KG_ERR_NONFINITE); atomicExch(p.ctrl + kCtrlAbort, 1); }
          return false;
        }
        if (tid == 0) ss.alpha[k] = alpha;
        // ||w - alpha v||^2 = ||w||^2 - 2 alpha <v|w> + alpha^2 ||v||^2, with <v|w> = alpha
        beta_m = sqrt(fmax(out[1] - 2.0 * alpha * alpha + alpha * alpha * out[2], 0.0));
      }
    }
  }
  __syncthreads();
  // ---- small exponential and recombination coefficients (warp 0)
  if (tid < 32) {
    double cr = 0.0, ci = 0.0;
    if (meff > 0) tridiag_expv_e1(ss.alpha, ss.beta, meff, tau, cr, ci);
    if (tid < meff) {
      const double f = nrm_src * ss.scale[tid];
      ss.coef_re[tid] = cr * f;
      ss.coef_im[tid] = ci * f;
    }
    if (tid == meff - 1 && meff > 0) ss.err = (broke ? 0.0 : nrm_src * beta_m * sqrt(cr * cr + ci * ci));
  }
  __syncthreads();
  if (meff > 0) {
    if (tid == 0) { c.err_max = fmax(c.err_max, ss.err); c.breakdowns += broke ? 1 : 0; }
  }
  // ---- recombination dst = sum_k coef_k v_k (+ fused norms / overlaps)
  A nacc[1] = {0};
  double ex[2] = {0.0, 0.0};
  for (int T = c.g.rank; T < c.ntiles; T += c.g.size) {
    const size_t base = (size_t)T << c.t;
    for (int li = tid; li < c.tile; li += nt) {
      const size_t gi = base + li;
      R yr = 0, yi = 0;
      for (int k = 0; k < meff; ++k) {
        const V q = ldv(((k == 0) ? src : c.basis_slot(k)) + gi);
        const R a = (R)ss.coef_re[k], b = (R)ss.coef_im[k];
        yr += a * q.x - b * q.y;
        yi += a * q.y + b * q.x;
      }
      const V y = vmake<V>(yr, yi);
      stv(dst + gi, y);
      nacc[0] += (A)(yr * yr + yi * yi);
      if (extra == kExtraOverlapTarget) {
        const double2 f = reinterpret_cast<const double2*>(p.target)[gi];
        ex[0] += f.x * (double)yr + f.y * (double)yi;
        ex[1] += f.x * (double)yi - f.y * (double)yr;
      } else if (extra == kExtraGradOverlap) {
        V q;
        if (p.hc_kind == KG_HC_SX_SITE) {
          q = ldv(psi_other + (gi ^ ((size_t)1 << p.hc_site)));
          q.x *= (R)(0.5 * p.hc_amp);
          q.y *= (R)(0.5 * p.hc_amp);
        } else {
          const unsigned mk = (unsigned)p.hc_mask;
          const R dz = (R)(p.hc_amp * 0.5 * (double)(__popc(mk) - 2 * __popc((unsigned)gi & mk)));
          q = ldv(psi_other + gi);
          q.x *= dz;
          q.y *= dz;
        }
        // Im(conj(y) q)
        ex[0] += (double)(yr * q.y - yi * q.x);
      }
    }
  }
  double out[3];
  double vals[3] = {(double)nacc[0], ex[0], ex[1]};
  if (!group_reduce<3>(c.g, ss.red, vals, out)) return false;
  nrm_dst = sqrt(fmax(out[0], 0.0));
  e = make_double2(out[1], out[2]);
  if (!isfinite(out[0])) {
    if (tid == 0) { atomicCAS(p.ctrl + kCtrlStatus, 0, (int)KG_ERR_NONFINITE); atomicExch(p.ctrl + kCtrlAbort, 1); }
    return false;
  }
  return true;
}

// chi_N = beta f, ||chi_N||, and G_N = 2 dt Im <chi_N|Hc|psi_N>.
template <class V>
__device__ bool init_costate(Ctx<V>& c, double2 beta, V* chi, const V* psiN, double& nrm, double& gim) {
  using R = typename VecTraits<V>::R;
  const EvalParams& p = *c.p;
  double acc[2] = {0.0, 0.0};
  for (int T = c.g.rank; T < c.ntiles; T += c.g.size) {
    const size_t base = (size_t)T << c.t;
    for (int li = threadIdx.x; li < c.tile; li += blockDim.x) {
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
  for (int T = c.g.rank; T < c.ntiles; T += c.g.size) {
    const size_t base = (size_t)T << c.t;
    for (int li = threadIdx.x; li < c.tile; li += blockDim.x) {
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

template <class V, class A>
__global__ void __launch_bounds__(kThreads, 1) kg_eval_kernel(const __grid_constant__ EvalParams p) {
  extern __shared__ __align__(16) unsigned char smem_dyn[];
  __shared__ SmemSlice ss;
  Ctx<V> c;
  c.p = &p;
  c.g.rank = blockIdx.x;
  c.g.size = gridDim.x;
  c.g.bar = p.bar;
  c.g.red = p.red;
  c.g.ctrl = p.ctrl;
  c.g.wait_limit_ns = p.wait_limit_ns;
  c.g.phase = 0;
  c.g.skip_arrival = (p.debug_fault == 1 && blockIdx.x == 0) ? 1 : 0;
  c.ss = &ss;
  c.s_v = reinterpret_cast<V*>(smem_dyn);
  c.t = p.t_bits;
  c.tile = 1 << p.t_bits;
  c.D = (size_t)1 << p.L;
  c.ntiles = (int)(c.D >> p.t_bits);
  c.maskL1 = (p.L >= 2) ? ((1u << (p.L - 1)) - 1u) : 0u;
  c.err_max = 0.0;
  c.breakdowns = 0;
  const bool lead = (blockIdx.x == 0 && threadIdx.x == 0);

  // ---- forward sweep (Alg. "Basic GRAPE", step 4)
  double nrm_prev;
  if (!init_state<V>(c, fwd_slot<V>(c, 0), nrm_prev)) return;
  if (lead) p.nrm[0] = nrm_prev;
  double2 beta = make_double2(0.0, 0.0);
  for (int j = 1; j <= p.N; ++j) {
    const double uj = p.u[j - 1];
    double nrm_new;
    double2 e;
    const int extra = (j == p.N) ? kExtraOverlapTarget : kExtraNone;
    if (!krylov_slice<V, A>(c, fwd_slot<V>(c, j - 1), nrm_prev, uj, p.dt, fwd_slot<V>(c, j), extra, nullptr,
                            nrm_new, e))
      return;
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
    if (!init_costate<V>(c, beta, chi[0], psiN, nchi, gim)) return;
    if (lead) p.G[p.N] = 2.0 * p.dt * gim;
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
          if (!krylov_slice<V, A>(c, prev, np, p.u[i - 1], p.dt, d, kExtraNone, nullptr, nn, e)) return;
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
        if (!krylov_slice<V, A>(c, chi[cur], nchi, p.u[j - 1], -p.dt, chi[cur ^ 1], kExtraGradOverlap, psi_jm1,
                                nn, e))
          return;
        if (lead) p.G[j - 1] = 2.0 * p.dt * e.x;
        cur ^= 1;
        nchi = nn;
      }
    }
  }
  // ---- outputs (CTA 0)
  if (blockIdx.x == 0) {
    __syncthreads();
    if (p.grad_mode != KG_GRAD_NONE) {
      for (int j = threadIdx.x; j < p.N; j += blockDim.x) {
        const double gl = p.G[j], gr = p.G[j + 1];
        p.grad[j] = (p.grad_mode == KG_GRAD_ZEROTH) ? gr : 0.5 * (gl + gr);
      }
    }
    if (threadIdx.x == 0) {
      p.scal[kScErrMax] = c.err_max;
      p.scal[kScBreakdowns] = (double)c.breakdowns;
    }
  }
}

// ---------------------------------------------------------------- host-side launch helpers
template <class V, class A>
static cudaError_t launch_eval(const EvalParams& p, int ctas, cudaStream_t stream) {
  const size_t smem = ((size_t)1 << p.t_bits) * sizeof(V);
  auto kern = kg_eval_kernel<V, A>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  EvalParams pc = p;
  void* args[] = {&pc};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(ctas), dim3(kThreads), args, smem, stream);
}

template <class V, class A>
static cudaError_t max_ctas(int t_bits, int* out) {
  const size_t smem = ((size_t)1 << t_bits) * sizeof(V);
  auto kern = kg_eval_kernel<V, A>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  if (err != cudaSuccess) return err;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *out = per_sm * sms;
  return cudaSuccess;
}

cudaError_t launch_eval_kernel(int prec, const EvalParams& p, int ctas, cudaStream_t stream) {
  if (prec == KG_PREC_C128) return launch_eval<double2, double>(p, ctas, stream);
  return launch_eval<float2, float>(p, ctas, stream);
}

cudaError_t eval_kernel_max_ctas(int prec, int t_bits, int* out) {
  if (prec == KG_PREC_C128) return max_ctas<double2, double>(t_bits, out);
  return max_ctas<float2, float>(t_bits, out);
}

}  // namespace kg

// K-GRAPE evaluation in a parity-excitation (PE) subspace of the XXZ chain (Sec. 3.1), one CTA
// per control pulse, and the host side of the kg_sector_* entry points.
//
// The subspaces of Sec. 3.1 are small (D of a few hundred to a few thousand) and the pulses long
// (M = 4D slices), so a pulse is a long chain of short Krylov steps whose cost is latency.  A CTA
// keeps the whole state in shared memory and runs the forward sweep, the target overlap, the
// co-state sweep with the gradient overlaps and the gradient assembly of one pulse with nothing
// but block barriers; the CTAs of a launch take independent pulses (a batch: line-search
// candidates, restarts, scans).
//
// H0 in the reduced basis.  Basis vector r is |r> = (|s_r> + p |Pi s_r>)/sqrt(n_r) over the orbit
// {s_r, Pi s_r} (n_r = 1 for a palindrome).  Since H0 commutes with Pi,
//   <r'|H0|r> = sqrt(n_r'/n_r) sum_{t in orbit r} phi(t) <t|H0|s_r'>,
// phi(t) = +1 for the smaller member of its orbit, p for the mirrored one (parity 0: one state per
// orbit).  Row r' therefore needs H0 applied to the single state s_r': its diagonal
// (Jz/4)(L-1 - 2 popcount((s ^ s>>1) & mask)), computed on the fly, and one term Jxy/2 per
// antiparallel bond, landing in orbit r(t) with the factor sqrt(n_r'/n_r(t)) phi(t).  The host
// tabulates those terms per row as 16-bit entries (13 bits: column r(t); 3 bits: one of the
// factor classes 1, sqrt 2, 1/sqrt 2, -1, 0) in an ELL layout [entry][row], which the CTA keeps in
// shared memory.  Hc is diagonal (mirror-symmetric Sz mask): hc_amp (popcount(mask) -
// 2 popcount(s & mask))/2.
//
// One Lanczos step (App. A, Alg. "Lanczos", Paige's order), thread t owning rows t + NT i:
//   w       = H v_k - b_k v_{k-1}                      (gather from shared memory)
//   alpha_k = <v_k|w>,  b_{k+1}^2 = ||w||^2 - 2 alpha_k <v_k|w> + alpha_k^2 ||v_k||^2   (one block reduction)
//   v_{k+1} = (w - alpha_k v_k) / b_{k+1}               (into shared memory and the basis)
// Complex64 path: vectors and partial sums in FP32, cross-warp sums in float-float, the
// tridiagonal T in FP64 (warp 0, once per slice).  Complex128 path: FP64 throughout.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <unordered_map>
#include <type_traits>
#include <vector>

#include "kg_device.cuh"
#include "kg_launch.h"

namespace kg {

// ---------------------------------------------------------------- float-float vectors (KG_PREC_FF)
// Every amplitude is the unevaluated sum hi + lo of two FP32 numbers (about 44 significant bits),
// and the arithmetic on it is FP32 with error-free transformations (Knuth's TwoSum, the FMA
// TwoProduct: ff_add, ff_mul), so that the rounding of the Krylov vectors -- what limits the
// complex64 path over the 2 x 4D slices of Sec. 3.2's pulses -- shrinks by about 2^20 without one
// FP64 instruction (1/64 of the FP32 rate on this GPU) per amplitude.  The scalars that steer the
// recurrence (alpha, b, norms, overlaps) come from FP64 block sums of the float-float partials,
// as on the complex128 path.
struct FFR {
  float hi, lo;
  FFR() = default;
  __device__ __forceinline__ FFR(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ FFR(int a) : hi((float)a), lo(0.f) {}
  __device__ __forceinline__ explicit FFR(double a) : hi((float)a), lo((float)(a - (double)(float)a)) {}
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
  __device__ __forceinline__ explicit operator float() const { return __fadd_rn(hi, lo); }
};
struct __align__(16) FFC {
  FFR x, y;
};
__device__ __forceinline__ FFR operator+(FFR a, FFR b) {
  const FF s = ff_add(FF{a.hi, a.lo}, FF{b.hi, b.lo});
  return FFR(s.hi, s.lo);
}
__device__ __forceinline__ FFR operator-(FFR a) { return FFR(-a.hi, -a.lo); }
__device__ __forceinline__ FFR operator-(FFR a, FFR b) { return a + (-b); }
__device__ __forceinline__ FFR operator*(FFR a, FFR b) {
  const FF p = ff_mul(FF{a.hi, a.lo}, FF{b.hi, b.lo});
  return FFR(p.hi, p.lo);
}
__device__ __forceinline__ FFR fma(FFR a, FFR b, FFR c) { return a * b + c; }
// Square root and reciprocal: the FP32 estimate refined by one Newton step carried out in
// float-float (the residual a - s^2, or 1 - b y, formed exactly with an FMA), about 44 bits.
__device__ __forceinline__ FF ff_sqrt(FF a) {
  if (!(a.hi > 0.f)) return FF{0.f, 0.f};
  const float s = sqrtf(a.hi);
  const float p = __fmul_rn(s, s);
  const float e = __fmaf_rn(s, s, -p);                                      // s^2 = p + e exactly
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), e), a.lo);       // a - s^2
  return ff_two_sum(s, __fdiv_rn(r, __fmul_rn(2.f, s)));
}
__device__ __forceinline__ FF ff_rcp(FF b) {
  const float y = __frcp_rn(b.hi);
  const float p = __fmul_rn(b.hi, y);
  const float pe = __fmaf_rn(b.hi, y, -p);                                  // b.hi y = p + pe exactly
  const float r = __fsub_rn(__fsub_rn(__fsub_rn(1.f, p), pe), __fmul_rn(b.lo, y));  // 1 - b y
  return ff_two_sum(y, __fmul_rn(y, r));
}
// Scalar operations, once per Lanczos step: comparisons on (hi, lo) in order.
__device__ __forceinline__ bool ffr_less(FFR a, FFR b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ FFR operator/(FFR a, FFR b) {
  const FF q = ff_rcp(FF{b.hi, b.lo});
  return a * FFR(q.hi, q.lo);
}
__device__ __forceinline__ bool operator<=(FFR a, FFR b) { return !ffr_less(b, a); }
__device__ __forceinline__ FFR fmax(FFR a, FFR b) { return ffr_less(a, b) ? b : a; }
__device__ __forceinline__ FFR fabs(FFR a) { return (a.hi < 0.f) ? -a : a; }
__device__ __forceinline__ FFR sqrt(FFR a) {
  const FF s = ff_sqrt(FF{a.hi, a.lo});
  return FFR(s.hi, s.lo);
}
// the float and double functions stay visible beside these overloads inside namespace kg
using ::fma;
using ::fmax;
using ::fabs;
using ::sqrt;
template <> struct VecTraits<FFC> { using R = FFR; };
template <> __device__ __forceinline__ FFC vmake<FFC>(FFR a, FFR b) { return FFC{a, b}; }

constexpr int kSecColBits = 13;
constexpr int kSecMaxD = 1 << kSecColBits;  // columns fit the entry's 13 bits
constexpr int kSecClasses = 8;
enum SecClass { kSecW1 = 0, kSecWSqrt2 = 1, kSecWInvSqrt2 = 2, kSecWMinus1 = 3, kSecWZero = 7 };

struct SectorParams {
  int D, N, m, ell, B, L1, grad_mode;
  unsigned maskL1, hc_mask;
  double qz, hc_amp, dt, bd_tol;
  double wcls[kSecClasses];      // weight of each entry class: (Jxy/2) x factor
  const unsigned short* ell_g;   // [ell][D] entries
  const unsigned* states;        // [D] s_r
  const double* u;               // [B][N]
  const double* psi0;            // [2D] complex128
  const double* target;          // [2D] complex128
  double* fid;                   // [B]
  double* grad;                  // [B][N] or null
  void* traj;                    // [grid][N+1][D] psi_0..psi_N of the pulse in hand
  void* basis;                   // [grid][m][D] Lanczos vectors of the slice in hand
  void* tint;                    // [grid][2N][D] interior Gauss-Lobatto states (KG_GRAD_EXACT), or null
  double* G;                     // [grid][N+1]
  double* scal;                  // [B][kScCount]
  int* ctrl;                     // status word
  long long time_limit_ns;       // per pulse
  long long* prof;               // [8] phase cycles of CTA 0 (KG_FLAG_PHASE_TIMING), or null
};

// Block barrier of this kernel.  Several barriers follow work that only thread 0 does (FP64
// square roots and divisions, the failure record, the time check), so lanes of warp 0 may reach
// them apart.  __syncthreads() is PTX's .aligned barrier, whose behaviour is undefined unless every
// warp arrives converged at the same barrier instruction; with it, CTAs that evaluated a second
// pulse came out of step by a barrier.  The barrier without .aligned waits per thread and is
// defined for diverged arrival.
__device__ __forceinline__ void sec_sync() { asm volatile("barrier.sync 0;" ::: "memory"); }

struct SecSmem {
  float red_f[2][32 * 4];   // warp partials (complex64), by reduction parity
  double red_d[2][32 * 4];  // warp partials (complex128)
  float2 tot_f[2][4];       // float-float totals
  double tot_d[2][4];
  float wcls_f[kSecClasses];
  double wcls_d[kSecClasses];
  float2 wcls_ff[kSecClasses];  // float-float (hi, lo)
  double alpha[kMaxM], beta[kMaxM + 1];
  float alpha_f[kMaxM], beta_f[kMaxM + 1];
  float2 ff_a[kMaxM], ff_n[kMaxM], ff_q[kMaxM], ff_e[kMaxM];
  float coef_f[3][2][kMaxM];   // [slice end, interior node a, b][re, im][k]
  double coef_d[3][2][kMaxM];
  double nrm_d, ex_d, tay_d, err_max;
  float beta_m_f, inv_f;
  unsigned ff_e_set;
  int breakdowns;
  int abort;                    // the pulse in hand is abandoned (status set)
  int fail_step, fail_check;    // where it was abandoned (sec_record)
  long long prof_last, prof_acc[8];  // phase timing (thread 0 of CTA 0)
  unsigned long long t_start;   // globaltimer at the pulse's start
};

// Phase timing (KG_FLAG_PHASE_TIMING, thread 0 of CTA 0): cycles since the last mark go to
// counter `ph`: 0 Lanczos gathers and updates, 1 block reductions, 4 tridiagonal T and small
// exponential, 5 recombination, 6 pulse setup and overlaps.
__device__ __forceinline__ void sec_mark(const SectorParams& p, SecSmem& sm, int ph) {
  if (p.prof && blockIdx.x == 0 && threadIdx.x == 0) {
    const long long now = clock64();
    sm.prof_acc[ph] += now - sm.prof_last;
    sm.prof_last = now;
  }
}

// ---------------------------------------------------------------- block reductions
// Every thread receives the totals.  Two barriers: warp partials, then warp v sums value v.
template <int NT, int NV>
__device__ __forceinline__ void sec_reduce(SecSmem& sm, int& par, const float (&vals)[NV], FF (&out)[NV]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* red = sm.red_f[par];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const float x = warp_sum(vals[v]);
    if (lane == 0) red[warp * 4 + v] = x;
  }
  sec_sync();
  if (warp < NV) {
    FF s{(lane < NT / 32) ? red[lane * 4 + warp] : 0.f, 0.f};
    s = ff_warp_sum(s);
    if (lane == 0) sm.tot_f[par][warp] = make_float2(s.hi, s.lo);
  }
  sec_sync();
#pragma unroll
  for (int v = 0; v < NV; ++v) out[v] = FF{sm.tot_f[par][v].x, sm.tot_f[par][v].y};
  par ^= 1;
}
template <int NT, int NV>
__device__ __forceinline__ void sec_reduce(SecSmem& sm, int& par, const double (&vals)[NV], double (&out)[NV]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* red = sm.red_d[par];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double x = warp_sum(vals[v]);
    if (lane == 0) red[warp * 4 + v] = x;
  }
  sec_sync();
  if (warp < NV) {
    double s = (lane < NT / 32) ? red[lane * 4 + warp] : 0.0;
    s = warp_sum(s);
    if (lane == 0) sm.tot_d[par][warp] = s;
  }
  sec_sync();
#pragma unroll
  for (int v = 0; v < NV; ++v) out[v] = sm.tot_d[par][v];
  par ^= 1;
}

// Float-float partial sums (KG_PREC_FF): the same two stages, warp sums by ff_add (the warp partials
// are kept in the complex128 path's slots, two floats in each).
template <int NT, int NV>
__device__ __forceinline__ void sec_reduce(SecSmem& sm, int& par, const FF (&vals)[NV], FF (&out)[NV]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2* red = reinterpret_cast<float2*>(sm.red_d[par]);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const FF x = ff_warp_sum(vals[v]);
    if (lane == 0) red[warp * 4 + v] = make_float2(x.hi, x.lo);
  }
  sec_sync();
  if (warp < NV) {
    FF s{0.f, 0.f};
    if (lane < NT / 32) s = FF{red[lane * 4 + warp].x, red[lane * 4 + warp].y};
    s = ff_warp_sum(s);
    if (lane == 0) sm.tot_f[par][warp] = make_float2(s.hi, s.lo);
  }
  sec_sync();
#pragma unroll
  for (int v = 0; v < NV; ++v) out[v] = FF{sm.tot_f[par][v].x, sm.tot_f[par][v].y};
  par ^= 1;
}

__device__ __forceinline__ void sec_flag(const SectorParams& p, int code) { atomicCAS(p.ctrl, 0, code); }

// Where a pulse was abandoned, kept in the pulse's scalar block for diagnosis: scal[5] = slice
// (+j forward, -j backward), scal[6] = Lanczos step (-1: after the loop), scal[7] = check
// (1 non-finite step sums, 2 non-finite norm, 3 tridiagonal bound, 4 time limit).  Thread 0 only.
__device__ __forceinline__ void sec_record(SecSmem& sm, int k, int check) {
  if (sm.fail_check == 0) {
    sm.fail_step = k;
    sm.fail_check = check;
  }
}

template <class V> __device__ __forceinline__ V vscale(typename VecTraits<V>::R a, V x) {
  return vmake<V>(a * x.x, a * x.y);
}
template <class V> __device__ __forceinline__ V vaxpy(typename VecTraits<V>::R a, V x, V y) {
  return vmake<V>(fma(a, x.x, y.x), fma(a, x.y, y.y));
}

// Scalars of step k from the reduced sums o = (<v|w>, ||w||^2, ||v||^2), computed by every thread
// alike.  code: 0 go on, 1 the identity cancels (form ||w - alpha v||^2 explicitly), 2 non-finite.
struct SecStep {
  float alpha, b2;
  int code;
};
__device__ __forceinline__ SecStep sec_scalars(const FF (&o)[3], bool last, FF& b2ff) {
  SecStep s;
  s.alpha = __fadd_rn(o[0].hi, o[0].lo);
  b2ff = ff_add(o[1], ff_mul(ff_mul(o[0], o[0]), ff_add(o[2], FF{-2.f, 0.f})));
  s.b2 = __fadd_rn(b2ff.hi, b2ff.lo);
  s.code = 0;
  if (!isfinite(s.alpha) || !isfinite(o[1].hi)) s.code = 2;
  else if (!last && b2ff.hi < 1e-3f * o[1].hi) s.code = 1;
  return s;
}

// Taylor-hierarchy terms of backward slice j (App. B, Eq. gradp), this thread's partial sum:
// x was chi_j, psi_end is psi_j, H = H_j, and Im <chi| Hbar_c^[P] |psi> with a_m = H^m chi,
// b_n = H^n psi and Hc diagonal is
//   P = 1: Im M00 - (dt/2) Re(M10 - M01);  P = 2: also - (dt^2/6) Im(M20 - 2 M11 + M02),
// M_mn = <a_m|Hc|b_n>.  The a_m come from the slice's Lanczos vectors (H v_0 = alpha_0 v_0 +
// b_1 v_1, H v_1 = b_1 v_0 + alpha_1 v_1 + b_2 v_2), the b_n from the slice's gather applied to
// psi_j once or twice.  Nothing reads the shared vectors after the Lanczos loop.  Kept out of
// line: it runs once per backward slice and its arrays would crowd the Lanczos loop's registers.
template <class V, int NT, int RPT>
__device__ __noinline__ typename VecTraits<V>::R sec_taylor(const SectorParams& p, SecSmem& sm, V* Sa, V* Sb,
                                                          const unsigned short* ell, const V* basis, double uj,
                                                          int meff, typename VecTraits<V>::R nin, int taylor,
                                                          const V* psi_end) {
  using R = typename VecTraits<V>::R;
  constexpr bool F32 = sizeof(R) == 4;
  const int tid = threadIdx.x, D = p.D, ne = p.ell;
  const R* wcls = F32 ? (const R*)sm.wcls_f : (const R*)sm.wcls_d;
  // the diagonals of H0 and Hc, formed again here from the rows' states (as in sec_eval)
  R dj[RPT], hh[RPT];
  const int npc = __popc(p.hc_mask);
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int r = tid + NT * i;
    dj[i] = 0;
    hh[i] = 0;
    if (r < D) {
      const unsigned st = p.states[r];
      const R d0 = (R)(p.qz * (double)(p.L1 - 2 * __popc((st ^ (st >> 1)) & p.maskL1)));
      hh[i] = (R)(0.5 * p.hc_amp * (double)(npc - 2 * __popc(st & p.hc_mask)));
      dj[i] = fma((R)uj, hh[i], d0);
    }
  }
  R pt = 0;
  V b0[RPT], b1[RPT], b2[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int r = tid + NT * i;
    b0[i] = (r < D) ? psi_end[r] : vmake<V>(0, 0);
    b2[i] = vmake<V>(0, 0);
    if (r < D) Sa[r] = b0[i];
  }
  sec_sync();
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int r = tid + NT * i;
    V h = vmake<V>(0, 0);
    if (r < D) {
      h = vscale<V>(dj[i], b0[i]);
#pragma unroll 4
      for (int e = 0; e < ne; ++e) {
        const unsigned en = ell[e * D + r];
        h = vaxpy<V>(wcls[en >> kSecColBits], Sa[en & (kSecMaxD - 1)], h);
      }
      if (taylor >= 2) Sb[r] = h;
    }
    b1[i] = h;
  }
  if (taylor >= 2) {
    sec_sync();
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int r = tid + NT * i;
      if (r < D) {
        V h = vscale<V>(dj[i], b1[i]);
#pragma unroll 4
        for (int e = 0; e < ne; ++e) {
          const unsigned en = ell[e * D + r];
          h = vaxpy<V>(wcls[en >> kSecColBits], Sb[en & (kSecMaxD - 1)], h);
        }
        b2[i] = h;
      }
    }
  }
  const R al0 = (meff > 0) ? (F32 ? (R)sm.alpha_f[0] : (R)sm.alpha[0]) : (R)0;
  const R al1 = (meff > 1) ? (F32 ? (R)sm.alpha_f[1] : (R)sm.alpha[1]) : (R)0;
  const R be1 = (meff > 1) ? (F32 ? (R)sm.beta_f[1] : (R)sm.beta[1]) : (R)0;
  const R be2 = (meff > 2) ? (F32 ? (R)sm.beta_f[2] : (R)sm.beta[2]) : (R)0;
  const R c0 = al0 * al0 + be1 * be1, c1 = be1 * (al0 + al1), c2 = be1 * be2;
  const R h1 = (R)(0.5 * p.dt), h2 = (R)(p.dt * p.dt / 6.0);
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int r = tid + NT * i;
    if (r < D && meff > 0) {
      const V v0 = basis[r];
      const V v1 = (meff > 1) ? basis[(size_t)D + r] : vmake<V>(0, 0);
      const V v2 = (taylor >= 2 && meff > 2) ? basis[(size_t)2 * D + r] : vmake<V>(0, 0);
      const V a0 = vscale<V>(nin, v0);
      const V a1 = vscale<V>(nin, vaxpy<V>(be1, v1, vscale<V>(al0, v0)));
      // conj(a) b = (a.x b.x + a.y b.y) + i (a.x b.y - a.y b.x)
      R t = a0.x * b0[i].y - a0.y * b0[i].x;                                                   // Im M00
      t -= h1 * ((a1.x * b0[i].x + a1.y * b0[i].y) - (a0.x * b1[i].x + a0.y * b1[i].y));     // Re(M10 - M01)
      if (taylor >= 2) {
        const V a2 = vscale<V>(nin, vaxpy<V>(c2, v2, vaxpy<V>(c1, v1, vscale<V>(c0, v0))));
        const R i20 = a2.x * b0[i].y - a2.y * b0[i].x, i11 = a1.x * b1[i].y - a1.y * b1[i].x;
        const R i02 = a0.x * b2[i].y - a0.y * b2[i].x;
        t -= h2 * (i20 - (R)2 * i11 + i02);
      }
      pt = fma(hh[i], t, pt);
    }
  }
  return pt;
}

// Interior Gauss-Lobatto states of a slice (KG_GRAD_EXACT), from the slice's basis and the
// coefficients warps 1 and 2 formed: forward (lob = 1) psi(t_{j-1} + s) for s = s_a, s_b, stored
// to io[0..D), io[D..2D); backward (lob = 2) chi(t_{j-1} + s), overlapped with those stored states:
// the return value is this thread's share of Im <chi_a|Hc|psi_a> + Im <chi_b|Hc|psi_b>.  Out of line,
// so that its arrays stay out of the Lanczos loop's registers.
template <class V, int NT, int RPT>
__device__ __noinline__ typename VecTraits<V>::R sec_interior(const SectorParams& p, SecSmem& sm, const V* basis,
                                                            int meff, int lob, V* io) {
  using R = typename VecTraits<V>::R;
  constexpr bool F32 = sizeof(R) == 4;
  const int tid = threadIdx.x, D = p.D;
  const int npc = __popc(p.hc_mask);
  R pg = 0;
  for (int w = 1; w <= 2; ++w) {
    V y[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) y[i] = vmake<V>(0, 0);
    for (int k = 0; k < meff; ++k) {
      const R a = F32 ? (R)sm.coef_f[w][0][k] : (R)sm.coef_d[w][0][k];
      const R b = F32 ? (R)sm.coef_f[w][1][k] : (R)sm.coef_d[w][1][k];
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int r = tid + NT * i;
        if (r < D) {
          const V q = basis[(size_t)k * D + r];
          y[i].x = fma(a, q.x, fma(-b, q.y, y[i].x));
          y[i].y = fma(a, q.y, fma(b, q.x, y[i].y));
        }
      }
    }
    V* slot = io + (size_t)(w - 1) * D;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int r = tid + NT * i;
      if (r >= D) continue;
      if (lob == 1) {
        slot[r] = y[i];
      } else {
        const unsigned st = p.states[r];
        const R hc = (R)(0.5 * p.hc_amp * (double)(npc - 2 * __popc(st & p.hc_mask)));
        const V o = slot[r];
        pg = fma(hc, y[i].x * o.y - y[i].y * o.x, pg);  // Im(conj(chi_s) Hc psi_s), Hc diagonal
      }
    }
  }
  return pg;
}

// One slice: x (own rows, norm nrm) -> x = ||x|| V exp(-i tau T) e_1 (App. A), written to dst
// (if not null), then ||x||^2 and, for extra = 1, G = Im <x| Hc |other> over the own rows are
// reduced.  Returns false after a non-finite coefficient (status set).
template <class V, int NT, int RPT>
__device__ __forceinline__ bool sec_slice(const SectorParams& p, SecSmem& sm, int& par, V* Sa, V* Sb,
                                          const unsigned short* ell, V* basis,
                                          const typename VecTraits<V>::R (&dd)[RPT],
                                          const typename VecTraits<V>::R (&hh)[RPT], double uj, double tau,
                                          V (&x)[RPT], double& nrm, typename VecTraits<V>::R& inv, int extra,
                                          const V* other, V* dst, double& ex, int taylor = 0,
                                          const V* psi_end = nullptr, double* tay = nullptr, int lob = 0,
                                          V* tint_io = nullptr) {
  using R = typename VecTraits<V>::R;
  constexpr bool F32 = sizeof(R) == 4;
  constexpr bool FFM = std::is_same<R, FFR>::value;  // float-float vectors (KG_PREC_FF)
  const int tid = threadIdx.x, D = p.D, m = p.m, ne = p.ell;
  const R* wcls = F32 ? (const R*)sm.wcls_f : FFM ? (const R*)sm.wcls_ff : (const R*)sm.wcls_d;
  R dj[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) dj[i] = fma((R)uj, hh[i], dd[i]);
  // ---- v_0 = x / ||x||
  const R inv0 = inv;
  const R nin = (R)nrm;  // ||x||: the Taylor terms rebuild H x, H^2 x from the basis
  V* Sc = Sa;
  V* Sn = Sb;
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int r = tid + NT * i;
    if (r < D) {
      const V v = vscale<V>(inv0, x[i]);
      Sc[r] = v;
      basis[r] = v;
    }
  }
  sec_sync();
  int meff = (nrm > 0.0) ? m : 0;
  bool broke = false;
  R bk = 0, amax = 0, bmax = 0;
  const R tol = (R)p.bd_tol;
  V w[RPT], vv[RPT];
  for (int k = 0; k < meff; ++k) {
    const bool last = (k == m - 1);
    R pa = 0, pn = 0, pq = 0;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int r = tid + NT * i;
      V h = vmake<V>(0, 0), v = vmake<V>(0, 0);
      if (r < D) {
        v = Sc[r];
        h = vscale<V>(dj[i], v);
#pragma unroll 4
        for (int e = 0; e < ne; ++e) {
          const unsigned en = ell[e * D + r];
          h = vaxpy<V>(wcls[en >> kSecColBits], Sc[en & (kSecMaxD - 1)], h);
        }
        if (k > 0) h = vaxpy<V>(-bk, Sn[r], h);
        pa = fma(v.x, h.x, fma(v.y, h.y, pa));
        pn = fma(h.x, h.x, fma(h.y, h.y, pn));
        pq = fma(v.x, v.x, fma(v.y, v.y, pq));
      }
      w[i] = h;
      vv[i] = v;
    }
    R alpha, beta;
    R b2;
    if constexpr (F32) {
      const float vals[3] = {pa, pn, pq};
      FF o[3], b2ff;
      sec_mark(p, sm, 0);
      sec_reduce<NT, 3>(sm, par, vals, o);
      sec_mark(p, sm, 1);
      SecStep st = sec_scalars(o, last, b2ff);
      if (st.code == 2) {
        if (tid == 0) {
          sec_flag(p, KG_ERR_NONFINITE);
          sec_record(sm, k, 1);
        }
        return false;
      }
      if (tid == 0) {
        sm.ff_a[k] = make_float2(o[0].hi, o[0].lo);
        sm.ff_n[k] = make_float2(o[1].hi, o[1].lo);
        sm.ff_q[k] = make_float2(o[2].hi, o[2].lo);
      }
      if (st.code == 1) {  // near an invariant subspace: ||w - alpha v||^2 explicitly
        float e1[1] = {0.f};
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const V d = vaxpy<V>(-st.alpha, vv[i], w[i]);
          e1[0] = fmaf(d.x, d.x, fmaf(d.y, d.y, e1[0]));
        }
        FF o1[1];
        sec_reduce<NT, 1>(sm, par, e1, o1);
        if (tid == 0) {
          sm.ff_e[k] = make_float2(o1[0].hi, o1[0].lo);
          sm.ff_e_set |= 1u << k;
        }
        st.b2 = __fadd_rn(o1[0].hi, o1[0].lo);
      }
      alpha = st.alpha;
      b2 = st.b2;
    } else if constexpr (FFM) {
      // float-float sums and scalars: alpha_k and b_{k+1}^2 = ||w||^2 + alpha^2 (||v||^2 - 2) in
      // float-float, as the complex64 path forms them, but kept at float-float for the vectors
      const FF vals[3] = {FF{pa.hi, pa.lo}, FF{pn.hi, pn.lo}, FF{pq.hi, pq.lo}};
      FF o[3];
      sec_mark(p, sm, 0);
      sec_reduce<NT, 3>(sm, par, vals, o);
      sec_mark(p, sm, 1);
      if (!isfinite(o[0].hi) || !isfinite(o[1].hi)) {
        if (tid == 0) {
          sec_flag(p, KG_ERR_NONFINITE);
          sec_record(sm, k, 1);
        }
        return false;
      }
      FF b2ff = ff_add(o[1], ff_mul(ff_mul(o[0], o[0]), ff_add(o[2], FF{-2.f, 0.f})));
      if (tid == 0) {
        sm.ff_a[k] = make_float2(o[0].hi, o[0].lo);
        sm.ff_n[k] = make_float2(o[1].hi, o[1].lo);
        sm.ff_q[k] = make_float2(o[2].hi, o[2].lo);
      }
      if (!last && b2ff.hi < 1e-3f * o[1].hi) {  // near an invariant subspace: ||w - alpha v||^2 explicitly
        const R ra = R(o[0].hi, o[0].lo);
        R e = 0;
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const V d = vaxpy<V>(-ra, vv[i], w[i]);
          e = fma(d.x, d.x, fma(d.y, d.y, e));
        }
        const FF e1[1] = {FF{e.hi, e.lo}};
        FF o1[1];
        sec_reduce<NT, 1>(sm, par, e1, o1);
        if (tid == 0) {
          sm.ff_e[k] = make_float2(o1[0].hi, o1[0].lo);
          sm.ff_e_set |= 1u << k;
        }
        b2ff = o1[0];
      }
      alpha = R(o[0].hi, o[0].lo);
      b2 = R(b2ff.hi, b2ff.lo);
    } else {
      const double vals[3] = {(double)pa, (double)pn, (double)pq};
      double o[3];
      sec_mark(p, sm, 0);
      sec_reduce<NT, 3>(sm, par, vals, o);
      sec_mark(p, sm, 1);
      double bd = o[1] - 2.0 * o[0] * o[0] + o[0] * o[0] * o[2];
      if (!isfinite(o[0]) || !isfinite(o[1])) {
        if (tid == 0) {
          sec_flag(p, KG_ERR_NONFINITE);
          sec_record(sm, k, 1);
        }
        return false;
      }
      if (!last && bd < 1e-3 * o[1]) {
        double e1[1] = {0.0};
        const R ra = (R)o[0];
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const V d = vaxpy<V>(-ra, vv[i], w[i]);
          const double dx = (double)d.x, dy = (double)d.y;
          e1[0] = fma(dx, dx, fma(dy, dy, e1[0]));
        }
        double o1[1];
        sec_reduce<NT, 1>(sm, par, e1, o1);
        bd = o1[0];
      }
      alpha = (R)o[0];
      b2 = (R)bd;
      if (tid == 0) sm.alpha[k] = o[0];
    }
    beta = sqrt(fmax(b2, (R)0));
    if (tid == 0) {
      sm.alpha_f[k] = (float)alpha;
      if (last) sm.beta_m_f = (float)beta;  // b_m of the error indicator
    }
    if (last) break;
    amax = fmax(amax, fabs(alpha));
    if (beta <= tol * fmax((R)1, amax + bmax)) {  // Alg. "Lanczos": b_j > 0, with a tolerance
      meff = k + 1;
      broke = true;
      break;
    }
    bmax = fmax(bmax, beta);
    if (tid == 0) {
      sm.beta_f[k + 1] = (float)beta;
      if (!F32) sm.beta[k + 1] = (double)beta;
    }
    const R ib = (R)1 / beta;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int r = tid + NT * i;
      if (r < D) {
        const V vn = vscale<V>(ib, vaxpy<V>(-alpha, vv[i], w[i]));
        Sn[r] = vn;
        basis[(size_t)(k + 1) * D + r] = vn;
      }
    }
    bk = beta;
    V* t = Sc;
    Sc = Sn;
    Sn = t;
    sec_sync();
  }
  sec_mark(p, sm, 0);
  // ---- T (FP64), exp(-i tau T) e_1 and the recombination coefficients (warp 0; with lob, warps 1
  // and 2 form the coefficients of the two interior Gauss-Lobatto nodes at the same time)
  if (tid < 32) {
    __syncwarp();  // thread 0's stores of the step sums are visible to the warp
    const int k = tid;
    if constexpr (F32 || FFM) {
      if (k < meff) {
        const double al = ff_to_double(FF{sm.ff_a[k].x, sm.ff_a[k].y});
        double b2;
        if ((sm.ff_e_set >> k) & 1u) {
          b2 = ff_to_double(FF{sm.ff_e[k].x, sm.ff_e[k].y});
        } else {
          const double nn = ff_to_double(FF{sm.ff_n[k].x, sm.ff_n[k].y});
          const double q = ff_to_double(FF{sm.ff_q[k].x, sm.ff_q[k].y});
          b2 = nn - 2.0 * al * al + al * al * q;
        }
        sm.alpha[k] = al;
        if (k + 1 < meff) sm.beta[k + 1] = sqrt(fmax(b2, 0.0));
      }
      __syncwarp();
    }
  }
  if (lob) sec_sync();  // T is read by warps 1 and 2 as well
  if (tid < (lob ? 96 : 32)) {
    const int w = tid >> 5, k = tid & 31;
    // slice end, or the interior nodes s_a, s_b = (1 -+ 1/sqrt 5) dt/2: forward exp(-i s H) psi_{j-1},
    // backward exp(+i (dt - s) H) chi_j
    double tw = tau;
    if (w > 0) {
      const double sn = 0.5 * p.dt * (1.0 + (w == 1 ? -1.0 : 1.0) / sqrt(5.0));
      tw = (lob == 1) ? sn : -(p.dt - sn);
    }
    double cr = 0.0, ci = 0.0;
    float tnorm = 0.f;
    const double etol = F32 ? 1e-13 : 1e-18;
    // The exponential takes ceil(||tau T|| / 4) sub-steps: refuse a T whose Gershgorin bound is not a
    // finite, sane number (it would come from corrupted coefficients) instead of looping on it.
    float row = 0.f;
    if (k < meff)
      row = fabsf((float)tw) * (fabsf(sm.alpha_f[k]) + (k >= 1 ? sm.beta_f[k] : 0.f) +
                                (k + 1 < meff ? sm.beta_f[k + 1] : 0.f));
    row = (row == row) ? row : 3.0e38f;  // NaN -> refused
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) row = fmaxf(row, __shfl_xor_sync(0xffffffffu, row, o));
    const bool sane = row <= 1.0e5f;
    if (tid == 0 && !sane) {
      sec_flag(p, KG_ERR_NONFINITE);
      sec_record(sm, -1, 3);
      sm.abort = 1;
    }
    if (meff > 0 && sane) {
      if constexpr (F32)  // float-float: FP64 instructions are slow on this GPU (see tridiag_expv_e1_ff)
        tridiag_expv_e1_ff(sm.alpha, sm.beta, sm.alpha_f, sm.beta_f, meff, tw, (float)tw, etol, cr, ci, tnorm);
      else
        tridiag_expv_e1(sm.alpha, sm.beta, sm.alpha_f, sm.beta_f, meff, tw, (float)tw, etol, cr, ci, tnorm);
    }
    if (k < meff) {
      sm.coef_d[w][0][k] = cr * nrm;
      sm.coef_d[w][1][k] = ci * nrm;
      sm.coef_f[w][0][k] = (float)(cr * nrm);
      sm.coef_f[w][1][k] = (float)(ci * nrm);
    }
    if (w == 0 && k == meff - 1) {  // a-posteriori indicator ||x|| b_m |c_{m-1}| (0 after a breakdown)
      double cm = nrm * sqrt(cr * cr + ci * ci);
      if (cm == 0.0 && !broke) {
        cm = nrm;
        for (int i = 1; i < meff; ++i) cm *= (double)tnorm / (double)i;
      }
      const double err = broke ? 0.0 : (double)sm.beta_m_f * cm;
      sm.err_max = fmax(sm.err_max, err);
      if (broke) sm.breakdowns += 1;
    }
    __syncwarp();
    if (tid == 0) {
      sm.ff_e_set = 0u;
      // time limit of one pulse: a pulse that runs past it ends with KG_ERR_TIMEOUT
      if (sm.abort == 0 && (long long)(globaltimer_ns() - sm.t_start) > p.time_limit_ns) {
        sec_flag(p, KG_ERR_TIMEOUT);
        sec_record(sm, -1, 4);
        sm.abort = 1;
      }
    }
  }
  sec_sync();
  if (sm.abort) return false;
  sec_mark(p, sm, 4);
  // ---- recombination x = sum_k coef_k v_k (own rows), fused ||x||^2 and the overlap
  // the own rows' basis values come from L2: KB basis vectors' loads are issued together
  constexpr int KB = F32 ? 4 : 2;
  V y[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) y[i] = vmake<V>(0, 0);
  for (int k0 = 0; k0 < meff; k0 += KB) {
    V q[KB][RPT];
#pragma unroll
    for (int u = 0; u < KB; ++u)
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int r = tid + NT * i;
        q[u][i] = (k0 + u < meff && r < D) ? basis[(size_t)(k0 + u) * D + r] : vmake<V>(0, 0);
      }
#pragma unroll
    for (int u = 0; u < KB; ++u) {
      const int k = k0 + u;
      const R a = (k < meff) ? (F32 ? (R)sm.coef_f[0][0][k] : (R)sm.coef_d[0][0][k]) : (R)0;
      const R b = (k < meff) ? (F32 ? (R)sm.coef_f[0][1][k] : (R)sm.coef_d[0][1][k]) : (R)0;
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        y[i].x = fma(a, q[u][i].x, fma(-b, q[u][i].y, y[i].x));
        y[i].y = fma(a, q[u][i].y, fma(b, q[u][i].x, y[i].y));
      }
    }
  }
  R pn = 0, pg = 0;
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int r = tid + NT * i;
    if (r < D) {
      if (dst) dst[r] = y[i];
      pn = fma(y[i].x, y[i].x, fma(y[i].y, y[i].y, pn));
      if (extra == 1) {
        const V o = other[r];
        pg = fma(hh[i], y[i].x * o.y - y[i].y * o.x, pg);  // Im(conj(y) Hc o), Hc diagonal
      }
    }
    x[i] = y[i];
  }
  // ---- Taylor hierarchy (App. B, Eq. gradp), backward slice j (sec_taylor)
  R pt = 0;
  if constexpr (!FFM) {  // the float-float path offers the centred and zeroth-order gradients
    if (taylor > 0) pt = sec_taylor<V, NT, RPT>(p, sm, Sa, Sb, ell, basis, uj, meff, nin, taylor, psi_end);
    if (lob > 0) pt = sec_interior<V, NT, RPT>(p, sm, basis, meff, lob, tint_io);
  }
  if constexpr (F32) {
    const float vals[3] = {pn, pg, pt};
    FF o[3];
    sec_mark(p, sm, 5);
    sec_reduce<NT, 3>(sm, par, vals, o);
    if (!isfinite(o[0].hi)) {
      if (tid == 0) {
        sec_flag(p, KG_ERR_NONFINITE);
        sec_record(sm, -1, 2);
      }
      return false;
    }
    // FP64 is slow on this GPU: thread 0 forms ||x|| and 1/||x|| for everyone (the next write of
    // these fields comes a whole slice later, after many barriers)
    if (tid == 0) {
      const double n = sqrt(fmax(ff_to_double(o[0]), 0.0));
      sm.nrm_d = n;
      sm.inv_f = (n > 0.0) ? (float)(1.0 / n) : 0.f;
      sm.ex_d = (extra == 1) ? ff_to_double(o[1]) : 0.0;
      sm.tay_d = (taylor > 0 || lob == 2) ? ff_to_double(o[2]) : 0.0;  // Taylor or interior overlaps
    }
    sec_sync();
    nrm = sm.nrm_d;
    inv = (R)sm.inv_f;
    ex = sm.ex_d;
    if (tay) *tay = sm.tay_d;
  } else {
    const double vals[3] = {(double)pn, (double)pg, (double)pt};
    double o[3];
    sec_mark(p, sm, 5);
    sec_reduce<NT, 3>(sm, par, vals, o);
    if (!isfinite(o[0])) {
      if (tid == 0) {
        sec_flag(p, KG_ERR_NONFINITE);
        sec_record(sm, -1, 2);
      }
      return false;
    }
    nrm = sqrt(fmax(o[0], 0.0));
    inv = (nrm > 0.0) ? (R)(1.0 / nrm) : (R)0;
    ex = o[1];
    if (tay) *tay = o[2];
  }
  sec_mark(p, sm, 1);
  return true;
}

// FP64 sums of the own rows of the pulse's first and last states (once per evaluation).
template <int NT, int NV>
__device__ __forceinline__ void sec_reduce_fp64(SecSmem& sm, int& par, const double (&vals)[NV], double (&out)[NV]) {
  sec_reduce<NT, NV>(sm, par, vals, out);
}

// Thread 0: F = NaN and the failure record of pulse b, abandoned in slice j (negative: backward).
__device__ __forceinline__ void sec_abandon(const SectorParams& p, const SecSmem& sm, int b, int j) {
  p.fid[b] = __longlong_as_double(0x7ff8000000000000LL);
  double* sc = p.scal + (size_t)b * kScCount;
  sc[5] = (double)j;
  sc[6] = (double)sm.fail_step;
  sc[7] = (double)sm.fail_check;
}

template <class V, int NT, int RPT>
__device__ __forceinline__ void sec_eval(const SectorParams& p, int b, SecSmem& sm, V* S0, V* S1,
                                      const unsigned short* ell) {
  using R = typename VecTraits<V>::R;
  const int tid = threadIdx.x, D = p.D, N = p.N;
  V* traj = (V*)p.traj + (size_t)blockIdx.x * (size_t)(N + 1) * D;
  V* basis = (V*)p.basis + (size_t)blockIdx.x * (size_t)p.m * D;
  double* G = p.G + (size_t)blockIdx.x * (N + 1);
  const double* u = p.u + (size_t)b * N;
  const double2* psi0 = reinterpret_cast<const double2*>(p.psi0);
  const double2* tgt = reinterpret_cast<const double2*>(p.target);
  R dd[RPT], hh[RPT];
  const int npc = __popc(p.hc_mask);
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int r = tid + NT * i;
    dd[i] = 0;
    hh[i] = 0;
    if (r < D) {
      const unsigned s = p.states[r];
      dd[i] = (R)(p.qz * (double)(p.L1 - 2 * __popc((s ^ (s >> 1)) & p.maskL1)));
      hh[i] = (R)(0.5 * p.hc_amp * (double)(npc - 2 * __popc(s & p.hc_mask)));
    }
  }
  sec_sync();  // the previous pulse (possibly abandoned after a non-finite value) is done with shared memory
  if (tid == 0) {
    sm.err_max = 0.0;
    sm.breakdowns = 0;
    sm.ff_e_set = 0u;
    sm.abort = 0;
    sm.prof_last = clock64();
    sm.fail_step = 0;
    sm.fail_check = 0;
    sm.t_start = globaltimer_ns();
  }
  int par = 0;
  V x[RPT];
  double nrm;
  {  // psi_0 into the trajectory and its norm (FP64)
    double acc[1] = {0.0};
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int r = tid + NT * i;
      x[i] = vmake<V>(0, 0);
      if (r < D) {
        const double2 q = psi0[r];
        x[i] = vmake<V>((R)q.x, (R)q.y);
        traj[r] = x[i];
        acc[0] = fma((double)x[i].x, (double)x[i].x, fma((double)x[i].y, (double)x[i].y, acc[0]));
      }
    }
    double o[1];
    sec_reduce_fp64<NT, 1>(sm, par, acc, o);
    nrm = sqrt(o[0]);
  }
  R inv = (nrm > 0.0) ? (R)(1.0 / nrm) : (R)0;
  double ex = 0.0;
  sec_mark(p, sm, 6);
  const bool exact = (p.grad_mode == KG_GRAD_EXACT);
  V* tint = exact ? (V*)p.tint + (size_t)blockIdx.x * 2 * (size_t)N * D : nullptr;
  for (int j = 1; j <= N; ++j) {
    if (!sec_slice<V, NT, RPT>(p, sm, par, S0, S1, ell, basis, dd, hh, u[j - 1], p.dt, x, nrm, inv, 0, nullptr,
                               traj + (size_t)j * D, ex, 0, nullptr, nullptr, exact ? 1 : 0,
                               exact ? tint + (size_t)2 * (j - 1) * D : nullptr)) {
      if (tid == 0) sec_abandon(p, sm, b, j);
      return;
    }
  }
  // beta = <f|psi_N> (FP64), F = |beta|^2
  double br, bi, nfin = nrm;
  {
    double acc[2] = {0.0, 0.0};
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int r = tid + NT * i;
      if (r < D) {
        const double2 f = tgt[r];
        const double xr = (double)x[i].x, xi = (double)x[i].y;
        acc[0] = fma(f.x, xr, fma(f.y, xi, acc[0]));   // Re(conj(f) x)
        acc[1] = fma(f.x, xi, fma(-f.y, xr, acc[1]));  // Im(conj(f) x)
      }
    }
    double o[2];
    sec_reduce_fp64<NT, 2>(sm, par, acc, o);
    br = o[0];
    bi = o[1];
  }
  if (p.grad_mode != KG_GRAD_NONE) {
    const int taylor = (p.grad_mode == KG_GRAD_TAYLOR1) ? 1 : (p.grad_mode == KG_GRAD_TAYLOR2) ? 2 : 0;
    // chi_N = beta f; G_N = 2 dt Im <chi_N|Hc|psi_N>
    double acc[2] = {0.0, 0.0};
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int r = tid + NT * i;
      V c = vmake<V>(0, 0);
      if (r < D) {
        const double2 f = tgt[r];
        c = vmake<V>((R)(br * f.x - bi * f.y), (R)(br * f.y + bi * f.x));
        const double cr = (double)c.x, ci = (double)c.y;
        acc[0] = fma(cr, cr, fma(ci, ci, acc[0]));
        acc[1] = fma((double)hh[i], cr * (double)x[i].y - ci * (double)x[i].x, acc[1]);
      }
      x[i] = c;
    }
    double o[2];
    sec_reduce_fp64<NT, 2>(sm, par, acc, o);
    nrm = sqrt(o[0]);
    inv = (nrm > 0.0) ? (R)(1.0 / nrm) : (R)0;
    if (tid == 0) G[N] = 2.0 * p.dt * o[1];
    sec_mark(p, sm, 6);
    for (int j = N; j >= 1; --j) {
      // chi_{j-1} = exp(+i dt H_j) chi_j, fused G_{j-1} = 2 dt Im <chi_{j-1}|Hc|psi_{j-1}>
      double tay = 0.0;
      if (!sec_slice<V, NT, RPT>(p, sm, par, S0, S1, ell, basis, dd, hh, u[j - 1], -p.dt, x, nrm, inv, 1,
                                 traj + (size_t)(j - 1) * D, nullptr, ex, taylor, traj + (size_t)j * D, &tay,
                                 exact ? 2 : 0, exact ? tint + (size_t)2 * (j - 1) * D : nullptr)) {
        if (tid == 0) sec_abandon(p, sm, b, -j);
        return;
      }
      if (tid == 0) {
        G[j - 1] = 2.0 * p.dt * ex;
        if (taylor) G[j] = 2.0 * p.dt * tay;  // slice j's Taylor-hierarchy value replaces G_j
        if (exact)  // 4-point Gauss-Lobatto over slice j: weights 1/12, 5/12, 5/12, 1/12
          p.grad[(size_t)b * N + (j - 1)] = (G[j - 1] + G[j]) / 12.0 + (5.0 / 12.0) * 2.0 * p.dt * tay;
      }
    }
    sec_sync();  // G complete (written by thread 0)
    double* gb = p.grad + (size_t)b * N;
    for (int j = tid; j < N && !exact; j += NT)
      gb[j] = (p.grad_mode == KG_GRAD_CENTERED) ? 0.5 * (G[j] + G[j + 1]) : G[j + 1];  // zeroth, Taylor
  }
  if (tid == 0) {
    p.fid[b] = br * br + bi * bi;
    double* sc = p.scal + (size_t)b * kScCount;
    sc[kScBetaRe] = br;
    sc[kScBetaIm] = bi;
    sc[kScErrMax] = sm.err_max;
    sc[kScNormFinal] = nfin;
    sc[kScBreakdowns] = (double)sm.breakdowns;
    sc[5] = sc[6] = sc[7] = 0.0;
  }
  sec_sync();
}

// CTAs (pulses) per SM the register allocation is sized for.  A pulse is a chain of latencies
// (block barriers, FP64 on warp 0), so pulses sharing an SM hide each other's: complex64 blocks of
// 128 threads are held to 64 registers a thread, eight pulses per SM (a few spills; measured 1.9x the
// pulses/s of three per SM at D = 511); float-float blocks of 128 threads to 128 registers, four per
// SM (no spills; 732 against 626 pulses/s at three per SM, D = 511); other blocks of up to 256
// threads to 128 registers, two per SM.
template <class V, int NT>
constexpr int sec_min_blocks() {
  return (NT == 128 && sizeof(V) == sizeof(float2)) ? 8 : (NT == 128 && std::is_same<V, FFC>::value) ? 4
                                                    : (NT <= 256) ? 2 : 1;
}

template <class V, int NT, int RPT>
__global__ void __launch_bounds__(NT, (sec_min_blocks<V, NT>())) kg_sector_kernel(const __grid_constant__ SectorParams p) {
  extern __shared__ __align__(16) unsigned char sec_dyn[];
  __shared__ SecSmem sm;
  const int Dp = (p.D + 15) & ~15;
  V* S0 = reinterpret_cast<V*>(sec_dyn);
  V* S1 = S0 + Dp;
  unsigned short* ell = reinterpret_cast<unsigned short*>(S1 + Dp);
  for (int i = threadIdx.x; i < p.ell * p.D; i += NT) ell[i] = p.ell_g[i];
  if (threadIdx.x < kSecClasses) {
    sm.wcls_f[threadIdx.x] = (float)p.wcls[threadIdx.x];
    sm.wcls_d[threadIdx.x] = p.wcls[threadIdx.x];
    const float wh = (float)p.wcls[threadIdx.x];
    sm.wcls_ff[threadIdx.x] = make_float2(wh, (float)(p.wcls[threadIdx.x] - (double)wh));
  }
  if (threadIdx.x < 8) sm.prof_acc[threadIdx.x] = 0;
  const long long t0 = clock64();
  sec_sync();
  for (int b = blockIdx.x; b < p.B; b += gridDim.x) sec_eval<V, NT, RPT>(p, b, sm, S0, S1, ell);
  if (p.prof && blockIdx.x == 0 && threadIdx.x == 0) {
    for (int i = 0; i < 7; ++i) p.prof[i] = sm.prof_acc[i];
    p.prof[7] = clock64() - t0;
  }
}

// ---------------------------------------------------------------- launch selection
struct SecKernel {
  const void* fn;
  int threads;
};

template <class V, int NT, int RPT>
static SecKernel sec_choice() {
  return {reinterpret_cast<const void*>(&kg_sector_kernel<V, NT, RPT>), NT};
}

// Threads and rows per thread by dimension: the smallest block that covers D with <= 8 rows per
// thread (10 for complex64 up to 2560, which keeps two CTAs on an SM); or, with nt = 128, 256 or
// 512 threads, that block with the fewest rows per thread that covers D (nt.threads == 0: none).
static SecKernel sec_pick(int prec, int D, int nt = 0) {
  if (prec == KG_PREC_FF) {  // the complex128 path's shapes (16-byte amplitudes); 512 x 5 up to
                             // D = 2560 holds its arrays in registers (512 x 8 spills)
    if (nt == 128) return (D <= 512) ? sec_choice<FFC, 128, 4>() : SecKernel{nullptr, 0};
    if (nt == 256) return (D <= 1024) ? sec_choice<FFC, 256, 4>()
                                      : (D <= 2048) ? sec_choice<FFC, 256, 8>() : SecKernel{nullptr, 0};
    if (nt == 512)
      return (D <= 2560) ? sec_choice<FFC, 512, 5>() : (D <= 4096) ? sec_choice<FFC, 512, 8>() : SecKernel{nullptr, 0};
    if (D <= 512) return sec_choice<FFC, 128, 4>();
    if (D <= 1024) return sec_choice<FFC, 256, 4>();
    if (D <= 2048) return sec_choice<FFC, 256, 8>();
    if (D <= 2560) return sec_choice<FFC, 512, 5>();
    return sec_choice<FFC, 512, 8>();
  }
  if (prec == KG_PREC_C128) {  // 512 x 5 up to D = 2560 spills less than 512 x 8
    if (nt == 128) return (D <= 512) ? sec_choice<double2, 128, 4>() : SecKernel{nullptr, 0};
    if (nt == 256) return (D <= 1024) ? sec_choice<double2, 256, 4>()
                                      : (D <= 2048) ? sec_choice<double2, 256, 8>() : SecKernel{nullptr, 0};
    if (nt == 512)
      return (D <= 2560) ? sec_choice<double2, 512, 5>()
                         : (D <= 4096) ? sec_choice<double2, 512, 8>() : SecKernel{nullptr, 0};
    if (D <= 512) return sec_choice<double2, 128, 4>();
    if (D <= 1024) return sec_choice<double2, 256, 4>();
    if (D <= 2048) return sec_choice<double2, 256, 8>();
    if (D <= 2560) return sec_choice<double2, 512, 5>();
    return sec_choice<double2, 512, 8>();
  }
  if (nt == 128) return (D <= 512) ? sec_choice<float2, 128, 4>() : SecKernel{nullptr, 0};
  if (nt == 256)
    return (D <= 1024) ? sec_choice<float2, 256, 4>()
                       : (D <= 2048) ? sec_choice<float2, 256, 8>()
                                     : (D <= 2560) ? sec_choice<float2, 256, 10>() : SecKernel{nullptr, 0};
  if (nt == 512) return (D <= 4096) ? sec_choice<float2, 512, 8>() : SecKernel{nullptr, 0};
  if (D <= 512) return sec_choice<float2, 128, 4>();
  if (D <= 1024) return sec_choice<float2, 256, 4>();
  if (D <= 2048) return sec_choice<float2, 256, 8>();
  if (D <= 2560) return sec_choice<float2, 256, 10>();  // two CTAs per SM (registers)
  return sec_choice<float2, 512, 8>();
}

constexpr int kSecMaxRows = 4096;  // 512 threads x 8 rows

size_t sector_smem_bytes(int prec, int D, int ell) {
  const size_t vb = (prec == KG_PREC_C64_F64REC) ? 8 : 16;
  const size_t Dp = ((size_t)D + 15) & ~(size_t)15;
  return 2 * Dp * vb + (size_t)ell * D * 2;
}

cudaError_t sector_kernel_max_ctas(int prec, int D, int ell, int nt, int* out) {
  const SecKernel k = sec_pick(prec, D, nt);
  if (!k.fn) return cudaErrorInvalidValue;
  const size_t smem = sector_smem_bytes(prec, D, ell);
  cudaError_t e = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k.fn, k.threads, smem)) != cudaSuccess) return e;
  *out = per * sms;
  return cudaSuccess;
}

int sector_threads(int prec, int D, int nt) { return sec_pick(prec, D, nt).threads; }
bool sector_shape_ok(int prec, int D, int nt) { return sec_pick(prec, D, nt).fn != nullptr; }

cudaError_t launch_sector_kernel(int prec, const SectorParams& p, int ctas, int nt, cudaStream_t stream) {
  const SecKernel k = sec_pick(prec, p.D, nt);
  if (!k.fn) return cudaErrorInvalidValue;
  const size_t smem = sector_smem_bytes(prec, p.D, p.ell);
  cudaError_t e = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<SectorParams*>(&p)};
  return cudaLaunchKernel(k.fn, dim3(ctas), dim3(k.threads), args, smem, stream);
}

}  // namespace kg

// ================================================================ host side of the ABI
namespace {

using kg::host_fail;

struct SectorBasis {
  std::vector<uint64_t> states;       // s_r, ascending
  std::vector<unsigned short> ell;    // [ell][D]
  int D = 0, ell_width = 0;
};

uint64_t mirror_bits(uint64_t s, int L) {
  uint64_t r = 0;
  for (int b = 0; b < L; ++b) r |= ((s >> b) & 1ull) << (L - 1 - b);
  return r;
}

kg_status check_sector(const kg_sector* s) {
  if (!s) return host_fail(KG_ERR_INVALID_ARG, "sector must not be NULL");
  if (s->L < 2 || s->L > kg::kMaxL) return host_fail(KG_ERR_INVALID_ARG, "L must satisfy 2 <= L <= 30");
  if (s->K < 0 || s->K > s->L) return host_fail(KG_ERR_INVALID_ARG, "K must satisfy 0 <= K <= L");
  if (s->parity < -1 || s->parity > 1) return host_fail(KG_ERR_INVALID_ARG, "parity must be -1, 0 or +1");
  if (s->block_threads != 0 && s->block_threads != 128 && s->block_threads != 256 && s->block_threads != 512)
    return host_fail(KG_ERR_INVALID_ARG, "block_threads must be 0, 128, 256 or 512");
  if ((s->hc_site_mask >> s->L) != 0) return host_fail(KG_ERR_INVALID_ARG, "hc_site_mask has bits at or above L");
  if (s->parity != 0 && mirror_bits(s->hc_site_mask, s->L) != s->hc_site_mask)
    return host_fail(KG_ERR_INVALID_ARG, "a parity subspace needs a mirror-symmetric hc_site_mask");
  if (!std::isfinite(s->Jxy) || !std::isfinite(s->Jz) || !std::isfinite(s->hc_amp))
    return host_fail(KG_ERR_INVALID_ARG, "Jxy, Jz and hc_amp must be finite");
  return KG_OK;
}

// Orbits of the K-excitation states under the mirror, in the order of their smaller member.
// orbit[s] for every state s of the sector (via its position in `all`): the row, the member's
// sign phi, and whether the orbit is a palindrome.  Returns false if D would exceed `limit`.
struct OrbitInfo {
  int row;     // -1: no basis vector (a palindrome in the odd subspace)
  int phi;     // +1 smaller member, parity for the mirrored one
  int n;       // orbit size
};

bool build_basis(const kg_sector* s, size_t limit, bool want_ell, SectorBasis& out, std::string& why) {
  const int L = s->L, K = s->K, P = s->parity;
  // the dimension in closed form, to refuse large subspaces before enumerating them: C(L,K) states,
  // pal of them mirror-symmetric (fixed by the first floor(L/2) bits and, for odd L, the middle one);
  // D = C (parity 0), (C + pal)/2 (even), (C - pal)/2 (odd)
  {
    auto binom = [](int n, int k) {
      double c = 1.0;
      for (int i = 0; i < k; ++i) c = c * (double)(n - i) / (double)(i + 1);
      return c;
    };
    const int h = L / 2;
    const double C = binom(L, K);
    const double pal = (L % 2 == 0) ? ((K % 2 == 0) ? binom(h, K / 2) : 0.0) : binom(h, K / 2);
    const double Dd = (P == 0) ? C : 0.5 * (C + (double)P * pal);
    if (Dd > (double)limit + 0.5) {
      why = "subspace dimension " + std::to_string((long long)(Dd + 0.5)) + " exceeds " + std::to_string(limit);
      return false;
    }
  }
  std::vector<uint64_t> all;  // the K-excitation states, ascending (Gosper's next-combination step)
  if (K == 0) {
    all.push_back(0);
  } else {
    uint64_t v = (1ull << K) - 1;
    const uint64_t end = 1ull << L;
    while (v < end) {
      all.push_back(v);
      if (all.size() > 64ull * 1024 * 1024) {
        why = "the K-excitation sector is too large";
        return false;
      }
      const uint64_t c = v & (~v + 1);
      const uint64_t r = v + c;
      v = (((r ^ v) >> 2) / c) | r;
    }
  }
  std::unordered_map<uint64_t, OrbitInfo> orb;
  orb.reserve(all.size() * 2);
  out.states.clear();
  for (const uint64_t st : all) {
    const uint64_t t = (P == 0) ? st : mirror_bits(st, L);
    if (t < st) continue;  // met at its smaller member already
    OrbitInfo oi{-1, 1, (t == st) ? 1 : 2};
    if (!(P == -1 && t == st)) {
      oi.row = (int)out.states.size();
      out.states.push_back(st);
    }
    orb[st] = oi;
    if (t != st) orb[t] = OrbitInfo{oi.row, P, 2};
  }
  out.D = (int)out.states.size();
  if ((size_t)out.D > limit) {
    why = "subspace dimension " + std::to_string(out.D) + " exceeds " + std::to_string(limit);
    return false;
  }
  if (!want_ell) return true;
  // per row: one entry per antiparallel bond of s_r whose image has a basis vector
  std::vector<std::vector<unsigned short>> rows(out.D);
  int width = 0;
  for (int r = 0; r < out.D; ++r) {
    const uint64_t st = out.states[r];
    const int nr = orb[st].n;
    for (int b = 0; b + 1 < L; ++b) {
      if (((st >> b) & 1ull) == ((st >> (b + 1)) & 1ull)) continue;
      const OrbitInfo& o = orb.at(st ^ (3ull << b));
      if (o.row < 0) continue;
      int cls;
      if (P == 1) cls = (nr == o.n) ? kg::kSecW1 : (nr == 2 ? kg::kSecWSqrt2 : kg::kSecWInvSqrt2);
      else if (P == -1) cls = (o.phi > 0) ? kg::kSecW1 : kg::kSecWMinus1;
      else cls = kg::kSecW1;
      rows[r].push_back((unsigned short)((cls << kg::kSecColBits) | o.row));
    }
    width = std::max(width, (int)rows[r].size());
  }
  out.ell_width = width;
  out.ell.assign((size_t)width * out.D, 0);
  for (int r = 0; r < out.D; ++r)
    for (int e = 0; e < width; ++e)
      out.ell[(size_t)e * out.D + r] = (e < (int)rows[r].size())
                                           ? rows[r][e]
                                           : (unsigned short)((kg::kSecWZero << kg::kSecColBits) | r);
  return true;
}

struct SectorLayout {
  size_t ctrl = 0, scal = 0, prof = 0, G = 0, basis = 0, traj = 0, tint = 0, ell = 0, states = 0, total = 0;
};

size_t align_up(size_t x) { return (x + kg::kAlign - 1) / kg::kAlign * kg::kAlign; }

SectorLayout sector_layout(int D, int ell, const kg_options* o, int B, int grid) {
  SectorLayout l;
  const size_t vb = (size_t)D * (o->prec == KG_PREC_C64_F64REC ? 8 : 16);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  l.ctrl = take(64);
  l.scal = take(sizeof(double) * kg::kScCount * (size_t)B);
  l.prof = take(sizeof(long long) * 8);
  l.G = take(sizeof(double) * (size_t)(o->N + 1) * grid);
  l.basis = take(vb * (size_t)o->m * grid);
  l.traj = take(vb * (size_t)(o->N + 1) * grid);
  l.tint = take(o->grad == KG_GRAD_EXACT ? vb * 2 * (size_t)o->N * grid : 0);
  l.ell = take((size_t)ell * D * 2);
  l.states = take(sizeof(unsigned) * (size_t)D);
  l.total = off;
  return l;
}

kg_status check_sector_opts(const kg_options* o, int B) {
  if (!o) return host_fail(KG_ERR_INVALID_ARG, "options must not be NULL");
  if (B < 1) return host_fail(KG_ERR_INVALID_ARG, "B must be >= 1");
  if (o->N < 1) return host_fail(KG_ERR_INVALID_ARG, "N must be >= 1");
  if (o->m < 1 || o->m > kg::kMaxM) return host_fail(KG_ERR_INVALID_ARG, "m must satisfy 1 <= m <= 32");
  if (o->prec != KG_PREC_C128 && o->prec != KG_PREC_C64_F64REC && o->prec != KG_PREC_FF)
    return host_fail(KG_ERR_INVALID_ARG, "prec must be KG_PREC_C128, KG_PREC_C64_F64REC or KG_PREC_FF");
  if (o->grad != KG_GRAD_NONE && o->grad != KG_GRAD_CENTERED && o->grad != KG_GRAD_ZEROTH &&
      o->grad != KG_GRAD_EXACT && o->grad != KG_GRAD_TAYLOR1 && o->grad != KG_GRAD_TAYLOR2)
    return host_fail(KG_ERR_INVALID_ARG, "grad must be KG_GRAD_NONE, _CENTERED, _ZEROTH, _EXACT, _TAYLOR1 or _TAYLOR2");
  if (o->prec == KG_PREC_FF && o->grad != KG_GRAD_NONE && o->grad != KG_GRAD_CENTERED &&
      o->grad != KG_GRAD_ZEROTH)
    return host_fail(KG_ERR_UNSUPPORTED, "KG_PREC_FF offers KG_GRAD_NONE, _CENTERED and _ZEROTH");
  if (o->ckpt_every != 0) return host_fail(KG_ERR_UNSUPPORTED, "subspace evaluations keep every state: ckpt_every must be 0");
  if (o->tile_bits != 0) return host_fail(KG_ERR_INVALID_ARG, "tile_bits must be 0 for subspaces");
  if ((o->flags & ~KG_FLAG_PHASE_TIMING) != 0)
    return host_fail(KG_ERR_INVALID_ARG, "only KG_FLAG_PHASE_TIMING is accepted for subspaces");
  if (o->ctas < 0) return host_fail(KG_ERR_INVALID_ARG, "ctas must be >= 0");
  if (!(o->dt > 0.0) || !std::isfinite(o->dt)) return host_fail(KG_ERR_INVALID_ARG, "dt must be finite and > 0");
  if (std::isnan(o->breakdown_tol)) return host_fail(KG_ERR_INVALID_ARG, "breakdown_tol must not be NaN");
  return KG_OK;
}

// Grid for B pulses: every CTA that fits co-resident, at most B, at most opts->ctas.
kg_status sector_grid(const kg_options* o, int D, int ell, int nt, int B, int* grid) {
  const size_t smem = kg::sector_smem_bytes(o->prec, D, ell);
  if (smem > 200 * 1024)
    return host_fail(KG_ERR_UNSUPPORTED, "the subspace's state and tables exceed one CTA's shared memory");
  int maxc = 0;
  cudaError_t e = kg::sector_kernel_max_ctas(o->prec, D, ell, nt, &maxc);
  if (e != cudaSuccess) {
    return host_fail(KG_ERR_CUDA, std::string("occupancy query: ") + cudaGetErrorName(e));
  }
  if (maxc < 1) return host_fail(KG_ERR_UNSUPPORTED, "the subspace kernel does not fit on this device");
  int g = std::min(B, maxc);
  if (o->ctas > 0) g = std::min(g, o->ctas);
  *grid = g;
  return KG_OK;
}

}  // namespace

struct kg_sector_handle {
  kg_sector sector;
  kg_options opts;
  SectorLayout lay;
  SectorBasis basis;
  char* ws = nullptr;
  cudaStream_t stream = nullptr;
  int device = 0, B = 1, grid = 1;
};

extern "C" {

kg_status kg_sector_dim(const kg_sector* s, int32_t* D) {
  if (!D) return host_fail(KG_ERR_INVALID_ARG, "D must not be NULL");
  kg_status st = check_sector(s);
  if (st != KG_OK) return st;
  SectorBasis b;
  std::string why;
  if (!build_basis(s, (size_t)kg::kSecMaxRows, false, b, why)) return host_fail(KG_ERR_UNSUPPORTED, why);
  *D = b.D;
  return KG_OK;
}

kg_status kg_sector_states(const kg_sector* s, uint64_t* states, int32_t D) {
  if (!states) return host_fail(KG_ERR_INVALID_ARG, "states must not be NULL");
  kg_status st = check_sector(s);
  if (st != KG_OK) return st;
  SectorBasis b;
  std::string why;
  if (!build_basis(s, (size_t)kg::kSecMaxRows, false, b, why)) return host_fail(KG_ERR_UNSUPPORTED, why);
  if (D != b.D) return host_fail(KG_ERR_INVALID_ARG, "D must equal the subspace dimension " + std::to_string(b.D));
  std::copy(b.states.begin(), b.states.end(), states);
  return KG_OK;
}

kg_status kg_sector_apply_h0(const kg_sector* s, const double* v, double* w, int32_t D) {
  if (!v || !w) return host_fail(KG_ERR_INVALID_ARG, "v and w must not be NULL");
  kg_status st = check_sector(s);
  if (st != KG_OK) return st;
  SectorBasis b;
  std::string why;
  if (!build_basis(s, (size_t)kg::kSecMaxRows, true, b, why)) return host_fail(KG_ERR_UNSUPPORTED, why);
  if (D != b.D) return host_fail(KG_ERR_INVALID_ARG, "D must equal the subspace dimension " + std::to_string(b.D));
  double wc[kg::kSecClasses] = {0, 0, 0, 0, 0, 0, 0, 0};
  const double hxy = 0.5 * s->Jxy;
  wc[kg::kSecW1] = hxy;
  wc[kg::kSecWSqrt2] = hxy * std::sqrt(2.0);
  wc[kg::kSecWInvSqrt2] = hxy / std::sqrt(2.0);
  wc[kg::kSecWMinus1] = -hxy;
  const uint64_t maskL1 = (1ull << (s->L - 1)) - 1ull;
  for (int r = 0; r < b.D; ++r) {  // the kernel's row: diagonal from s_r, then the table's entries
    const uint64_t x = b.states[r];
    const double d = 0.25 * s->Jz * (double)(s->L - 1 - 2 * __builtin_popcountll((x ^ (x >> 1)) & maskL1));
    double re = d * v[2 * r], im = d * v[2 * r + 1];
    for (int e = 0; e < b.ell_width; ++e) {
      const unsigned en = b.ell[(size_t)e * b.D + r];
      const int c = (int)(en & (kg::kSecMaxD - 1));
      re += wc[en >> kg::kSecColBits] * v[2 * c];
      im += wc[en >> kg::kSecColBits] * v[2 * c + 1];
    }
    w[2 * r] = re;
    w[2 * r + 1] = im;
  }
  return KG_OK;
}

kg_status kg_sector_workspace_bytes(const kg_sector* s, const kg_options* o, int32_t B, size_t* bytes) {
  if (!bytes) return host_fail(KG_ERR_INVALID_ARG, "bytes must not be NULL");
  kg_status st = check_sector(s);
  if (st != KG_OK) return st;
  if ((st = check_sector_opts(o, B)) != KG_OK) return st;
  SectorBasis b;
  std::string why;
  if (!build_basis(s, (size_t)kg::kSecMaxRows, true, b, why)) return host_fail(KG_ERR_UNSUPPORTED, why);
  if (!kg::sector_shape_ok(o->prec, b.D, s->block_threads))
    return host_fail(KG_ERR_INVALID_ARG, "block_threads too few for the subspace's dimension");
  // one trajectory per CTA: size for the grid kg_sector_create will choose on the current device
  // (B CTAs if no device can be queried)
  int grid = B;
  int dev = 0, maxc = 0;
  if (cudaGetDevice(&dev) == cudaSuccess &&
      kg::sector_smem_bytes(o->prec, b.D, b.ell_width) <= 200 * 1024 &&
      kg::sector_kernel_max_ctas(o->prec, b.D, b.ell_width, s->block_threads, &maxc) == cudaSuccess && maxc > 0) {
    grid = std::min(B, maxc);
    if (o->ctas > 0) grid = std::min(grid, o->ctas);
  } else {
    cudaGetLastError();  // no device here: clear the error the query left
  }
  *bytes = sector_layout(b.D, b.ell_width, o, B, grid).total;
  return KG_OK;
}

kg_status kg_sector_create(kg_sector_handle** handle, const kg_sector* s, const kg_options* o, int32_t B,
                           void* workspace, size_t bytes, void* cuda_stream) {
  if (!handle) return host_fail(KG_ERR_INVALID_ARG, "handle must not be NULL");
  *handle = nullptr;
  kg_status st = check_sector(s);
  if (st != KG_OK) return st;
  if ((st = check_sector_opts(o, B)) != KG_OK) return st;
  kg_sector_handle* h = new kg_sector_handle();
  std::string why;
  if (!build_basis(s, (size_t)kg::kSecMaxRows, true, h->basis, why)) {
    delete h;
    return host_fail(KG_ERR_UNSUPPORTED, why);
  }
  if (h->basis.D < 1) {
    delete h;
    return host_fail(KG_ERR_INVALID_ARG, "the subspace is empty");
  }
  if (!kg::sector_shape_ok(o->prec, h->basis.D, s->block_threads)) {
    delete h;
    return host_fail(KG_ERR_INVALID_ARG, "block_threads too few for the subspace's dimension");
  }
  const size_t need1 = sector_layout(h->basis.D, h->basis.ell_width, o, B, 1).total;  // one CTA
  if (!workspace || ((uintptr_t)workspace % kg::kAlign) != 0 || bytes < need1) {
    delete h;
    return host_fail(KG_ERR_WORKSPACE, "workspace must be 256-byte aligned and hold at least " +
                                           std::to_string(need1) + " bytes");
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    delete h;
    return host_fail(KG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorName(e));
  }
  int grid = 1;
  if ((st = sector_grid(o, h->basis.D, h->basis.ell_width, s->block_threads, B, &grid)) != KG_OK) {
    delete h;
    return st;
  }
  const size_t need = sector_layout(h->basis.D, h->basis.ell_width, o, B, grid).total;
  if (bytes < need) {
    delete h;
    return host_fail(KG_ERR_WORKSPACE, "workspace too small: need " + std::to_string(need) + " bytes, got " +
                                           std::to_string(bytes));
  }
  h->sector = *s;
  h->opts = *o;
  if (!(h->opts.breakdown_tol > 0.0))
    h->opts.breakdown_tol = (o->prec == KG_PREC_C128) ? 1e-12 : (o->prec == KG_PREC_FF) ? 1e-10 : 1e-5;
  h->lay = sector_layout(h->basis.D, h->basis.ell_width, o, B, grid);
  h->ws = (char*)workspace;
  h->stream = (cudaStream_t)cuda_stream;
  h->device = dev;
  h->B = B;
  h->grid = grid;
  // tables into the workspace (32-bit states: L <= 30)
  std::vector<unsigned> st32(h->basis.states.begin(), h->basis.states.end());
  e = cudaMemcpyAsync(h->ws + h->lay.states, st32.data(), st32.size() * sizeof(unsigned), cudaMemcpyHostToDevice,
                      h->stream);
  if (e == cudaSuccess && !h->basis.ell.empty())
    e = cudaMemcpyAsync(h->ws + h->lay.ell, h->basis.ell.data(), h->basis.ell.size() * 2, cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    delete h;
    return host_fail(KG_ERR_CUDA, std::string("upload of the subspace tables: ") + cudaGetErrorName(e));
  }
  *handle = h;
  return KG_OK;
}

kg_status kg_sector_evaluate(kg_sector_handle* h, const double* u, const void* psi0, const void* target, double* fid,
                             double* grad) {
  if (!h) return host_fail(KG_ERR_INVALID_ARG, "handle must not be NULL");
  if (!u || !psi0 || !target || !fid) return host_fail(KG_ERR_INVALID_ARG, "u, psi0, target and fid must not be NULL");
  if (h->opts.grad != KG_GRAD_NONE && !grad) return host_fail(KG_ERR_INVALID_ARG, "grad must not be NULL");
  if (((uintptr_t)psi0 % 16) || ((uintptr_t)target % 16) || ((uintptr_t)u % 8) || ((uintptr_t)fid % 8) ||
      (grad && ((uintptr_t)grad % 8)))
    return host_fail(KG_ERR_INVALID_ARG, "psi0/target must be 16-byte aligned, u/fid/grad 8-byte aligned");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->device) return host_fail(KG_ERR_INVALID_ARG, "current device differs from the handle's device");
  const kg_sector& s = h->sector;
  const kg_options& o = h->opts;
  kg::SectorParams p{};
  p.D = h->basis.D;
  p.N = o.N;
  p.m = o.m;
  p.ell = h->basis.ell_width;
  p.B = h->B;
  p.L1 = s.L - 1;
  p.grad_mode = o.grad;
  p.maskL1 = (unsigned)((1ull << (s.L - 1)) - 1ull);
  p.hc_mask = (unsigned)s.hc_site_mask;
  p.qz = 0.25 * s.Jz;
  p.hc_amp = s.hc_amp;
  p.dt = o.dt;
  p.bd_tol = o.breakdown_tol;
  for (int c = 0; c < kg::kSecClasses; ++c) p.wcls[c] = 0.0;
  const double hxy = 0.5 * s.Jxy;
  p.wcls[kg::kSecW1] = hxy;
  p.wcls[kg::kSecWSqrt2] = hxy * std::sqrt(2.0);
  p.wcls[kg::kSecWInvSqrt2] = hxy / std::sqrt(2.0);
  p.wcls[kg::kSecWMinus1] = -hxy;
  char* ws = h->ws;
  p.ell_g = (const unsigned short*)(ws + h->lay.ell);
  p.states = (const unsigned*)(ws + h->lay.states);
  p.u = u;
  p.psi0 = (const double*)psi0;
  p.target = (const double*)target;
  p.fid = fid;
  p.grad = grad;
  p.traj = ws + h->lay.traj;
  p.basis = ws + h->lay.basis;
  p.tint = (o.grad == KG_GRAD_EXACT) ? (void*)(ws + h->lay.tint) : nullptr;
  p.G = (double*)(ws + h->lay.G);
  p.scal = (double*)(ws + h->lay.scal);
  p.ctrl = (int*)(ws + h->lay.ctrl);
  p.time_limit_ns = kg::sector_time_limit_ns();
  p.prof = (o.flags & KG_FLAG_PHASE_TIMING) ? (long long*)(ws + h->lay.prof) : nullptr;
  cudaError_t e = cudaMemsetAsync(ws + h->lay.ctrl, 0, 64, h->stream);
  if (e != cudaSuccess) return host_fail(KG_ERR_CUDA, std::string("cudaMemsetAsync(control block): ") + cudaGetErrorName(e));
  e = kg::launch_sector_kernel(o.prec, p, h->grid, h->sector.block_threads, h->stream);
  if (e != cudaSuccess) return host_fail(KG_ERR_CUDA, std::string("launch of the subspace kernel: ") + cudaGetErrorName(e));
  return KG_OK;
}

kg_status kg_sector_sync(kg_sector_handle* h, kg_report* rep) {
  if (!h) return host_fail(KG_ERR_INVALID_ARG, "handle must not be NULL");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return host_fail(KG_ERR_CUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorName(e));
  int ctrl[2] = {0, 0};
  e = cudaMemcpy(ctrl, h->ws + h->lay.ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return host_fail(KG_ERR_CUDA, std::string("cudaMemcpy(status): ") + cudaGetErrorName(e));
  if (rep) {
    std::vector<double> sc((size_t)h->B * kg::kScCount);
    e = cudaMemcpy(sc.data(), h->ws + h->lay.scal, sc.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return host_fail(KG_ERR_CUDA, std::string("cudaMemcpy(report): ") + cudaGetErrorName(e));
    std::memset(rep, 0, sizeof(*rep));
    rep->beta_re = sc[kg::kScBetaRe];
    rep->beta_im = sc[kg::kScBetaIm];
    rep->norm_final = sc[kg::kScNormFinal];
    double emax = 0.0, bd = 0.0;
    for (int b = 0; b < h->B; ++b) {
      emax = std::max(emax, sc[(size_t)b * kg::kScCount + kg::kScErrMax]);
      bd += sc[(size_t)b * kg::kScCount + kg::kScBreakdowns];
    }
    rep->krylov_err_max = emax;
    rep->breakdowns = (int32_t)bd;
    rep->status = ctrl[kg::kCtrlStatus];
    rep->launches = 1;
    rep->ctas = h->grid;
    rep->threads = kg::sector_threads(h->opts.prec, h->basis.D, h->sector.block_threads);
    rep->ckpt_every = 0;
    rep->reserved0 = 0;
    if (h->opts.flags & KG_FLAG_PHASE_TIMING) {
      long long pc[8];
      e = cudaMemcpy(pc, h->ws + h->lay.prof, sizeof(pc), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return host_fail(KG_ERR_CUDA, std::string("cudaMemcpy(phase timing): ") + cudaGetErrorName(e));
      for (int i = 0; i < 8; ++i) rep->phase_cycles[i] = pc[i];
    }
  }
  const int stv = ctrl[kg::kCtrlStatus];
  if (stv == KG_ERR_TIMEOUT) return host_fail(KG_ERR_TIMEOUT, "a pulse ran past the per-pulse time limit");
  if (stv == KG_ERR_NONFINITE) return host_fail(KG_ERR_NONFINITE, "non-finite Lanczos coefficient or norm");
  if (stv != 0) return host_fail(KG_ERR_CUDA, "device status " + std::to_string(stv));
  return KG_OK;
}

kg_status kg_sector_destroy(kg_sector_handle* h) {
  delete h;
  return KG_OK;
}

}  // extern "C"

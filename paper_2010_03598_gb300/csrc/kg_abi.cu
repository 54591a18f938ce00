// Host side of the C ABI declared in include/kgrape.h: argument checks, workspace layout,
// launch configuration, and the synchronous host-buffer entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <vector>
#include <cstdio>
#include <cstring>
#include <string>

#include "kg_internal.h"
#include "kg_launch.h"
#include "kgrape.h"

namespace {

thread_local std::string g_last_error;
std::atomic<long long> g_wait_limit_ns{2000000000LL};
std::atomic<int> g_debug_fault{0};

kg_status fail(kg_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

kg_status cuda_fail(cudaError_t e, const char* what) {
  return fail(KG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

size_t align_up(size_t x) { return (x + kg::kAlign - 1) / kg::kAlign * kg::kAlign; }

struct Layout {
  size_t ctrl = 0, bar = 0, iring = 0, red = 0, scal = 0, G = 0, nrm = 0, prof = 0, Gi = 0, tint = 0;
  size_t basis = 0, traj = 0, seg = 0, chi = 0, wbuf = 0, xbuf = 0;
  size_t st_u = 0, st_psi0 = 0, st_target = 0, st_fid = 0, st_grad = 0;
  size_t total = 0;
  size_t vec_bytes = 0;
};

kg_status check_args(const kg_chain* ch, const kg_options* o) {
  if (!ch || !o) return fail(KG_ERR_INVALID_ARG, "chain and options must not be NULL");
  if (ch->L < 1) return fail(KG_ERR_INVALID_ARG, "L must be >= 1");
  if (ch->L > kg::kMaxL) return fail(KG_ERR_UNSUPPORTED, "L > 30 is not supported");
  if (ch->hc_kind != KG_HC_SX_SITE && ch->hc_kind != KG_HC_SZ_SITES)
    return fail(KG_ERR_INVALID_ARG, "hc_kind must be KG_HC_SX_SITE or KG_HC_SZ_SITES");
  if (ch->hc_kind == KG_HC_SX_SITE && (ch->hc_site < 0 || ch->hc_site >= ch->L))
    return fail(KG_ERR_INVALID_ARG, "hc_site must satisfy 0 <= hc_site < L");
  if (ch->hc_kind == KG_HC_SZ_SITES && (ch->hc_site_mask >> ch->L) != 0)
    return fail(KG_ERR_INVALID_ARG, "hc_site_mask has bits at or above L");
  if (ch->reserved0 != 0) return fail(KG_ERR_INVALID_ARG, "reserved0 must be 0");
  if (!std::isfinite(ch->Jxy) || !std::isfinite(ch->Jz) || !std::isfinite(ch->hc_amp))
    return fail(KG_ERR_INVALID_ARG, "Jxy, Jz and hc_amp must be finite");
  if (o->N < 1) return fail(KG_ERR_INVALID_ARG, "N must be >= 1");
  if (o->m < 1 || o->m > kg::kMaxM) return fail(KG_ERR_INVALID_ARG, "m must satisfy 1 <= m <= 32");
  if (o->prec == KG_PREC_FF)
    return fail(KG_ERR_UNSUPPORTED, "float-float vectors (KG_PREC_FF) are available for subspaces (kg_sector_*)");
  if (o->prec != KG_PREC_C128 && o->prec != KG_PREC_C64_F64REC)
    return fail(KG_ERR_INVALID_ARG, "prec must be KG_PREC_C128 or KG_PREC_C64_F64REC");
  if (o->grad == KG_GRAD_TAYLOR1 || o->grad == KG_GRAD_TAYLOR2)
    return fail(KG_ERR_UNSUPPORTED, "Taylor-hierarchy gradients are available for subspaces (kg_sector_*)");
  if (o->grad != KG_GRAD_NONE && o->grad != KG_GRAD_CENTERED && o->grad != KG_GRAD_ZEROTH &&
      o->grad != KG_GRAD_EXACT)
    return fail(KG_ERR_INVALID_ARG, "grad must be KG_GRAD_NONE, _CENTERED, _ZEROTH or _EXACT");
  if (o->ckpt_every < 0 && o->ckpt_every != KG_CKPT_AUTO)
    return fail(KG_ERR_INVALID_ARG, "ckpt_every must be >= 0 or KG_CKPT_AUTO");
  if (o->mem_budget < 0) return fail(KG_ERR_INVALID_ARG, "mem_budget must be >= 0");
  if (o->grad == KG_GRAD_EXACT && o->ckpt_every > 0)
    return fail(KG_ERR_UNSUPPORTED, "KG_GRAD_EXACT keeps every slice's interior states: no checkpointing");
  if (o->tile_bits != 0 && (o->tile_bits < 1 || o->tile_bits > 13))
    return fail(KG_ERR_INVALID_ARG, "tile_bits must be 0 (auto) or 1..13");
  if (o->ctas < 0 || o->ctas > kg::kMaxCtas) return fail(KG_ERR_INVALID_ARG, "ctas must be 0 (auto) or 1..2048");
  if ((o->flags & ~(KG_FLAG_HOST_STAGING | KG_FLAG_PHASE_TIMING | KG_FLAG_FULL_REORTH)) != 0)
    return fail(KG_ERR_INVALID_ARG, "unknown flag bits");
  if (!(o->dt > 0.0) || !std::isfinite(o->dt)) return fail(KG_ERR_INVALID_ARG, "dt must be finite and > 0");
  if (std::isnan(o->breakdown_tol)) return fail(KG_ERR_INVALID_ARG, "breakdown_tol must not be NaN");
  return KG_OK;
}

Layout make_layout(const kg_chain* ch, const kg_options* o) {
  Layout l;
  const size_t D = (size_t)1 << ch->L;
  const size_t vb = D * (o->prec == KG_PREC_C128 ? 16 : 8);
  l.vec_bytes = vb;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  l.ctrl = take(kg::kCtrlBytes);  // status words, barrier counter and sum ring share one memset block
  l.bar = l.ctrl + 32;
  l.iring = l.ctrl + 64;
  l.red = take(sizeof(double) * 2 * kg::kMaxCtas * kg::kNRed);
  l.scal = take(sizeof(double) * kg::kScCount);
  l.prof = take(sizeof(long long) * 8);
  l.G = take(sizeof(double) * (size_t)(o->N + 1));
  l.nrm = take(sizeof(double) * (size_t)(o->N + 1));
  l.basis = take(vb * (size_t)(o->m > 1 ? o->m - 1 : 1));
  const int C = o->ckpt_every;
  size_t ntraj = (C == 0) ? (size_t)o->N + 1 : (size_t)(o->N / C + 1 + (o->N % C != 0 ? 1 : 0));
  l.traj = take(vb * ntraj);
  l.seg = take(C == 0 ? 0 : vb * (size_t)(C + 1));
  l.chi = take(o->grad == KG_GRAD_NONE ? 0 : 2 * vb);
  l.wbuf = take(2 * vb);
  l.xbuf = take(vb);
  if (o->grad == KG_GRAD_EXACT) {  // G and psi at the two interior quadrature nodes of every slice
    l.Gi = take(sizeof(double) * 2 * (size_t)o->N);
    l.tint = take(vb * 2 * (size_t)o->N);
  }
  if (o->flags & KG_FLAG_HOST_STAGING) {
    l.st_u = take(sizeof(double) * (size_t)o->N);
    l.st_psi0 = take(16 * D);
    l.st_target = take(16 * D);
    l.st_fid = take(sizeof(double));
    l.st_grad = take(sizeof(double) * (size_t)o->N);
  }
  l.total = off;
  return l;
}

// KG_CKPT_AUTO: every psi_j kept when that workspace fits the budget, else a checkpoint every
// ceil(sqrt(N)) slices.  `budget` 0 asks the current device for its free memory (90 % of it); with
// no device to ask, every psi_j is kept.  Other values of ckpt_every are returned unchanged.
int resolve_ckpt(const kg_chain* ch, const kg_options* o, size_t budget) {
  if (o->ckpt_every != KG_CKPT_AUTO) return o->ckpt_every;
  if (o->grad == KG_GRAD_EXACT) return 0;  // the exact gradient keeps every slice's interior states
  kg_options full = *o;
  full.ckpt_every = 0;
  const size_t need = make_layout(ch, &full).total;
  if (budget == 0) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    budget = free_b / 10 * 9;
  }
  if (need <= budget) return 0;
  int C = (int)std::ceil(std::sqrt((double)o->N));
  if (C < 1) C = 1;
  return (C >= o->N) ? 0 : C;
}

// The options with KG_CKPT_AUTO resolved.
kg_options resolved(const kg_chain* ch, const kg_options* o, size_t budget_override = 0) {
  kg_options r = *o;
  r.ckpt_every = resolve_ckpt(ch, o, budget_override ? budget_override : (size_t)o->mem_budget);
  return r;
}

int default_tile_bits(const kg_chain* ch, const kg_options* o) {
  const int tmax = kg::max_tile_bits(o->prec);
  int t = (o->tile_bits > 0) ? o->tile_bits : tmax;
  if (t > tmax) t = tmax;
  if (t > ch->L) t = ch->L;
  return t;
}

}  // namespace

namespace kg {
// Failures of the other host translation units go through the same thread-local message.
kg_status host_fail(kg_status st, const std::string& msg) { return fail(st, msg); }
// Time limit of one pulse of a subspace launch: 60 device-side wait limits (2 minutes by default).
long long sector_time_limit_ns() { return 60LL * g_wait_limit_ns.load(); }
}  // namespace kg

struct kg_handle {
  kg_chain chain;
  kg_options opts;
  Layout lay;
  char* ws = nullptr;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int ctas = 1;
  int t_bits = 1;
  int variant = 0;
  int launches = 0;
};

namespace {

// Launch configuration of one evaluation on device dev (shared by kg_create and
// kg_evaluate_static): tile size, kernel variant, CTA count, default breakdown tolerance.
kg_status configure_handle(const kg_chain* chain, const kg_options* opts, const Layout& lay, int dev, kg_handle* h) {
  const int t = default_tile_bits(chain, opts);
  const int ntiles = 1 << (chain->L - t);
  cudaError_t e;
  // Resident variant when every CTA can keep its tiles in registers/shared memory.
  int variant = kg::kVariantStreaming;
  int ctas = 0;
  const int tpc = kg::resident_tiles_per_cta(opts->prec);
  if (tpc > 0 && !(opts->flags & KG_FLAG_FULL_REORTH)) {
    int maxr = 0;
    e = kg::eval_kernel_max_ctas(opts->prec, kg::kVariantResident, t, &maxr);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    // default: two tiles per CTA (paired so that every CTA has the same cross-tile work)
    int c = (opts->ctas > 0) ? opts->ctas : (ntiles >= 2 ? ntiles / 2 : 1);
    if (c > ntiles) c = ntiles;
    if (c > maxr) c = maxr;
    if (c > kg::kMaxCtas) c = kg::kMaxCtas;
    if (c >= 1 && (long long)c * tpc >= ntiles) {
      variant = (t == kg::max_tile_bits(opts->prec)) ? kg::kVariantResidentFull : kg::kVariantResident;
      ctas = c;
    }
  }
  if (variant == kg::kVariantStreaming && (opts->flags & KG_FLAG_FULL_REORTH)) variant = kg::kVariantGenericStream;
  if (variant == kg::kVariantStreaming || variant == kg::kVariantGenericStream) {
    int maxc = 0;
    e = kg::eval_kernel_max_ctas(opts->prec, variant, t, &maxc);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (maxc < 1) return fail(KG_ERR_UNSUPPORTED, "evaluation kernel does not fit on this device");
    ctas = (opts->ctas > 0) ? opts->ctas : ntiles;
    if (ctas > ntiles) ctas = ntiles;
    if (ctas > maxc) ctas = maxc;
    if (ctas > kg::kMaxCtas) ctas = kg::kMaxCtas;
  }
  h->chain = *chain;
  h->opts = *opts;
  if (!(h->opts.breakdown_tol > 0.0)) h->opts.breakdown_tol = (opts->prec == KG_PREC_C128) ? 1e-12 : 1e-5;
  h->lay = lay;
  h->device = dev;
  h->ctas = ctas;
  h->t_bits = t;
  h->variant = variant;
  return KG_OK;
}

}  // namespace

extern "C" {

int kg_version(void) { return 100; }

const char* kg_last_error(void) { return g_last_error.c_str(); }

kg_status kg_set_wait_limit_ns(int64_t ns) {
  if (ns < 1) return fail(KG_ERR_INVALID_ARG, "wait limit must be >= 1 ns");
  g_wait_limit_ns.store(ns);
  return KG_OK;
}

kg_status kg_debug_set_fault(int32_t kind) {
  if (kind < 0 || kind > 2) return fail(KG_ERR_INVALID_ARG, "fault kind must be 0, 1 or 2");
  g_debug_fault.store(kind);
  return KG_OK;
}

kg_status kg_workspace_bytes(const kg_chain* chain, const kg_options* opts, size_t* bytes) {
  kg_status st = check_args(chain, opts);
  if (st != KG_OK) return st;
  if (!bytes) return fail(KG_ERR_INVALID_ARG, "bytes must not be NULL");
  const kg_options r = resolved(chain, opts);
  *bytes = make_layout(chain, &r).total;
  return KG_OK;
}

kg_status kg_create(kg_handle** handle, const kg_chain* chain, const kg_options* opts_in, void* workspace,
                    size_t bytes, void* cuda_stream) {
  if (!handle) return fail(KG_ERR_INVALID_ARG, "handle must not be NULL");
  *handle = nullptr;
  kg_status st = check_args(chain, opts_in);
  if (st != KG_OK) return st;
  const kg_options ropts = resolved(chain, opts_in);
  const kg_options* opts = &ropts;
  const Layout lay = make_layout(chain, opts);
  if (!workspace) return fail(KG_ERR_WORKSPACE, "workspace must not be NULL");
  if (((uintptr_t)workspace % kg::kAlign) != 0) return fail(KG_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (bytes < lay.total)
    return fail(KG_ERR_WORKSPACE, "workspace too small: need " + std::to_string(lay.total) + " bytes, got " +
                                      std::to_string(bytes));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  kg_handle* h = new kg_handle();
  st = configure_handle(chain, opts, lay, dev, h);
  if (st != KG_OK) {
    delete h;
    return st;
  }
  h->ws = (char*)workspace;
  h->bytes = bytes;
  h->stream = (cudaStream_t)cuda_stream;
  *handle = h;
  return KG_OK;
}

static kg_status enqueue(kg_handle* h, const double* u, const void* psi0, const void* target, double* fid,
                         double* grad) {
  const kg_chain& ch = h->chain;
  const kg_options& o = h->opts;
  kg::EvalParams p{};
  p.L = ch.L;
  p.N = o.N;
  p.m = o.m;
  p.t_bits = h->t_bits;
  p.grad_mode = o.grad;
  p.hc_kind = ch.hc_kind;
  p.hc_site = ch.hc_site;
  p.ckpt = o.ckpt_every;
  p.hc_mask = ch.hc_site_mask;
  p.Jxy = ch.Jxy;
  p.Jz = ch.Jz;
  p.hc_amp = ch.hc_amp;
  p.dt = o.dt;
  p.bd_tol = o.breakdown_tol;
  p.reorth = (o.flags & KG_FLAG_FULL_REORTH) ? 1 : 0;
  p.u = u;
  p.psi0 = (const double*)psi0;
  p.target = (const double*)target;
  p.fid = fid;
  p.grad = grad;
  char* ws = h->ws;
  p.basis = ws + h->lay.basis;
  p.traj = ws + h->lay.traj;
  p.seg = ws + h->lay.seg;
  p.chi = ws + h->lay.chi;
  p.wbuf = ws + h->lay.wbuf;
  p.xbuf = ws + h->lay.xbuf;
  p.G = (double*)(ws + h->lay.G);
  p.nrm = (double*)(ws + h->lay.nrm);
  p.Gi = (o.grad == KG_GRAD_EXACT) ? (double*)(ws + h->lay.Gi) : nullptr;
  p.tint = (o.grad == KG_GRAD_EXACT) ? (void*)(ws + h->lay.tint) : nullptr;
  p.scal = (double*)(ws + h->lay.scal);
  p.bar = (unsigned long long*)(ws + h->lay.bar);
  p.red = (double*)(ws + h->lay.red);
  p.red_stride = kg::kMaxCtas;
  p.ctrl = (int*)(ws + h->lay.ctrl);
  p.iring = (unsigned long long*)(ws + h->lay.iring);
  p.wait_limit_ns = g_wait_limit_ns.load();
  p.debug_fault = g_debug_fault.exchange(0);
  p.prof = (o.flags & KG_FLAG_PHASE_TIMING) ? (long long*)(ws + h->lay.prof) : nullptr;
  cudaError_t e = cudaMemsetAsync(ws + h->lay.ctrl, 0, kg::kCtrlBytes, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(control block)");
  e = kg::launch_eval_kernel(o.prec, h->variant, p, h->ctas, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cooperative launch of the evaluation kernel");
  h->launches = 1;
  return KG_OK;
}

kg_status kg_evaluate(kg_handle* h, const double* u, const void* psi0, const void* target, double* fid,
                      double* grad) {
  if (!h) return fail(KG_ERR_INVALID_ARG, "handle must not be NULL");
  if (!u || !psi0 || !target || !fid) return fail(KG_ERR_INVALID_ARG, "u, psi0, target and fid must not be NULL");
  if (h->opts.grad != KG_GRAD_NONE && !grad) return fail(KG_ERR_INVALID_ARG, "grad must not be NULL");
  if (((uintptr_t)psi0 % 16) || ((uintptr_t)target % 16) || ((uintptr_t)u % 8) || ((uintptr_t)fid % 8) ||
      (grad && ((uintptr_t)grad % 8)))
    return fail(KG_ERR_INVALID_ARG, "psi0/target must be 16-byte aligned, u/fid/grad 8-byte aligned");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->device) return fail(KG_ERR_INVALID_ARG, "current device differs from the handle's device");
  return enqueue(h, u, psi0, target, fid, grad);
}

kg_status kg_sync(kg_handle* h, kg_report* rep) {
  if (!h) return fail(KG_ERR_INVALID_ARG, "handle must not be NULL");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  int ctrl[2] = {0, 0};
  e = cudaMemcpy(ctrl, h->ws + h->lay.ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(status)");
  if (rep) {
    double sc[kg::kScCount];
    e = cudaMemcpy(sc, h->ws + h->lay.scal, sizeof(sc), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(report)");
    rep->krylov_err_max = sc[kg::kScErrMax];
    rep->norm_final = sc[kg::kScNormFinal];
    rep->beta_re = sc[kg::kScBetaRe];
    rep->beta_im = sc[kg::kScBetaIm];
    rep->breakdowns = (int32_t)sc[kg::kScBreakdowns];
    rep->status = ctrl[kg::kCtrlStatus];
    rep->launches = h->launches;
    rep->ctas = h->ctas;
    rep->tile_bits = h->t_bits;
    rep->threads = kg::eval_kernel_threads(h->opts.prec, h->variant, h->t_bits);
    rep->ckpt_every = h->opts.ckpt_every;
    rep->reserved0 = 0;
    long long pc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (h->opts.flags & KG_FLAG_PHASE_TIMING) {
      e = cudaMemcpy(pc, h->ws + h->lay.prof, sizeof(pc), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(phase timing)");
    }
    for (int i = 0; i < 8; ++i) rep->phase_cycles[i] = pc[i];
  }
  const int st = ctrl[kg::kCtrlStatus];
  if (st == KG_ERR_TIMEOUT) return fail(KG_ERR_TIMEOUT, "a device-side wait ran past its time limit");
  if (st == KG_ERR_NONFINITE) return fail(KG_ERR_NONFINITE, "non-finite Lanczos coefficient or norm");
  if (st != 0) return fail(KG_ERR_CUDA, "device status " + std::to_string(st));
  return KG_OK;
}

kg_status kg_evaluate_host(kg_handle* h, const double* u, const void* psi0, const void* target, double* fid,
                           double* grad) {
  if (!h) return fail(KG_ERR_INVALID_ARG, "handle must not be NULL");
  if (!(h->opts.flags & KG_FLAG_HOST_STAGING))
    return fail(KG_ERR_INVALID_ARG, "handle was created without KG_FLAG_HOST_STAGING");
  if (!u || !psi0 || !target || !fid) return fail(KG_ERR_INVALID_ARG, "u, psi0, target and fid must not be NULL");
  if (h->opts.grad != KG_GRAD_NONE && !grad) return fail(KG_ERR_INVALID_ARG, "grad must not be NULL");
  const size_t D = (size_t)1 << h->chain.L;
  const int N = h->opts.N;
  char* ws = h->ws;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(ws + h->lay.st_u, u, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream)) ||
      (e = cudaMemcpyAsync(ws + h->lay.st_psi0, psi0, 16 * D, cudaMemcpyHostToDevice, h->stream)) ||
      (e = cudaMemcpyAsync(ws + h->lay.st_target, target, 16 * D, cudaMemcpyHostToDevice, h->stream)))
    return cuda_fail(e, "cudaMemcpyAsync(host inputs)");
  kg_status st = enqueue(h, (const double*)(ws + h->lay.st_u), ws + h->lay.st_psi0, ws + h->lay.st_target,
                         (double*)(ws + h->lay.st_fid), (double*)(ws + h->lay.st_grad));
  if (st != KG_OK) return st;
  if ((e = cudaMemcpyAsync(fid, ws + h->lay.st_fid, sizeof(double), cudaMemcpyDeviceToHost, h->stream)))
    return cuda_fail(e, "cudaMemcpyAsync(fid)");
  if (h->opts.grad != KG_GRAD_NONE &&
      (e = cudaMemcpyAsync(grad, ws + h->lay.st_grad, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream)))
    return cuda_fail(e, "cudaMemcpyAsync(grad)");
  return kg_sync(h, nullptr);
}

kg_status kg_destroy(kg_handle* h) {
  delete h;
  return KG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- evaluation without allocation
// Scratch for kg_evaluate_static: a fixed device array in place of a caller workspace (see the
// header for who needs this).  In host code the name g_static_ws is only a host-side handle of
// the symbol, not a device address; the device address is resolved once per device below.
static __device__ __align__(256) unsigned char g_static_ws[KG_STATIC_WORKSPACE_BYTES];

namespace {

constexpr int kStaticMaxDevices = 64;
// Device address of g_static_ws per device, and the context it was resolved in.  A symbol's
// address belongs to one context: after cudaDeviceReset, or when the caller makes another
// context current on the device, the address is resolved again.
struct StaticAddr {
  void* ctx = nullptr;
  void* addr = nullptr;
};
StaticAddr g_static_addr[kStaticMaxDevices];
std::mutex g_static_mu;  // guards the set-up only; calls themselves must not overlap

using CtxGetCurrentFn = int (*)(void**);  // the driver's cuCtxGetCurrent (CUresult, CUcontext*)

// The current context of the calling thread (through the driver entry point the runtime hands
// out, so that the library does not link the driver library itself).
kg_status current_context(void** ctx) {
  static CtxGetCurrentFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDriverEntryPointByVersion(cuCtxGetCurrent)");
    if (q != cudaDriverEntryPointSuccess || !p) return fail(KG_ERR_CUDA, "cuCtxGetCurrent is not available");
    fn = (CtxGetCurrentFn)p;
  }
  *ctx = nullptr;
  if (fn(ctx) != 0 || !*ctx) return fail(KG_ERR_CUDA, "no current CUDA context on the calling thread");
  return KG_OK;
}

// Set-up, once per device and context, with that device current: the device address of the
// scratch array.
kg_status static_scratch_address(int dev, void** out) {
  void* ctx = nullptr;
  kg_status st = current_context(&ctx);
  if (st != KG_OK) return st;
  std::lock_guard<std::mutex> lock(g_static_mu);
  StaticAddr& a = g_static_addr[dev];
  if (!a.addr || a.ctx != ctx) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_ws);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    a.ctx = ctx;
    a.addr = p;
  }
  *out = a.addr;
  return KG_OK;
}

}  // namespace

extern "C" kg_status kg_evaluate_static(const kg_chain* chain, const kg_options* opts_in, const double* u,
                                        const void* psi0, const void* target, double* fid, double* grad,
                                        void* cuda_stream) {
  kg_status st = check_args(chain, opts_in);
  if (st != KG_OK) return st;
  // KG_CKPT_AUTO chooses against the size of the static scratch
  const kg_options ropts = resolved(chain, opts_in, KG_STATIC_WORKSPACE_BYTES);
  const kg_options* opts = &ropts;
  if (opts->flags & KG_FLAG_HOST_STAGING)
    return fail(KG_ERR_INVALID_ARG, "kg_evaluate_static does not take KG_FLAG_HOST_STAGING");
  const Layout lay = make_layout(chain, opts);
  if (lay.total > KG_STATIC_WORKSPACE_BYTES)
    return fail(KG_ERR_WORKSPACE, "kg_evaluate_static: the problem needs " + std::to_string(lay.total) +
                                      " bytes of workspace; the static scratch holds " +
                                      std::to_string(KG_STATIC_WORKSPACE_BYTES) +
                                      " (use kg_create with a caller workspace)");
  if (!u || !psi0 || !target || !fid) return fail(KG_ERR_INVALID_ARG, "u, psi0, target and fid must not be NULL");
  if (opts->grad != KG_GRAD_NONE && !grad) return fail(KG_ERR_INVALID_ARG, "grad must not be NULL");
  if (((uintptr_t)psi0 % 16) || ((uintptr_t)target % 16) || ((uintptr_t)u % 8) || ((uintptr_t)fid % 8) ||
      (grad && ((uintptr_t)grad % 8)))
    return fail(KG_ERR_INVALID_ARG, "psi0/target must be 16-byte aligned, u/fid/grad 8-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kStaticMaxDevices) return fail(KG_ERR_UNSUPPORTED, "device index above 63");
  // The call waits for its stream and reads the status back, which a stream capture forbids.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing((cudaStream_t)cuda_stream, &cap);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
  if (cap != cudaStreamCaptureStatusNone)
    return fail(KG_ERR_INVALID_ARG, "kg_evaluate_static is synchronous and cannot be called during stream capture");
  void* ws = nullptr;
  st = static_scratch_address(dev, &ws);
  if (st != KG_OK) return st;
  kg_handle h;  // on the stack: nothing is allocated
  st = configure_handle(chain, opts, lay, dev, &h);
  if (st != KG_OK) return st;
  h.ws = (char*)ws;
  h.bytes = KG_STATIC_WORKSPACE_BYTES;
  h.stream = (cudaStream_t)cuda_stream;
  st = enqueue(&h, u, psi0, target, fid, grad);
  if (st != KG_OK) return st;
  return kg_sync(&h, nullptr);
}

// ---------------------------------------------------------------- batched evaluation
struct kg_batch {
  int B = 0;
  kg_options opts{};
  char* ws = nullptr;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int ctas = 0;
  size_t clear_off = 0, clear_bytes = 0;  // control block + barrier counters, zeroed per launch
  kg::BatchParams bp{};
};

namespace {

struct BatchLayout {
  size_t ctrl = 0, bars = 0, reds = 0, probs = 0, item_off = 0, items = 0, total = 0;
  std::vector<size_t> prob;  // start of each problem's own workspace
  size_t max_items = 0;
};

int batch_tile_bits(const kg_chain& ch) { return ch.L < 12 ? ch.L : 12; }

BatchLayout make_batch_layout(int B, const kg_chain* chains, const kg_options* o) {
  BatchLayout l;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  l.ctrl = take(64 + sizeof(unsigned long long) * (size_t)B);  // ctrl words, then barrier counters
  l.bars = l.ctrl + 64;
  l.reds = take(sizeof(double) * kg::kBatchRedPerGroup * (size_t)B);
  l.probs = take(sizeof(kg::EvalParams) * (size_t)B);
  l.item_off = take(sizeof(int) * (size_t)(kg::kMaxCtas + 1));
  for (int b = 0; b < B; ++b) l.max_items += (size_t)1 << (chains[b].L - batch_tile_bits(chains[b]));
  l.items = take(sizeof(kg::BatchItem) * l.max_items);
  l.prob.resize(B);
  for (int b = 0; b < B; ++b) l.prob[b] = take(make_layout(&chains[b], o).total);
  l.total = off;
  return l;
}

kg_status check_batch(int B, const kg_chain* chains, const kg_options* o) {
  if (B < 1) return fail(KG_ERR_INVALID_ARG, "batch size must be >= 1");
  if (!chains || !o) return fail(KG_ERR_INVALID_ARG, "chains and options must not be NULL");
  if (o->prec != KG_PREC_C64_F64REC) return fail(KG_ERR_UNSUPPORTED, "batched evaluation runs the complex64 path only");
  if (o->flags != 0) return fail(KG_ERR_INVALID_ARG, "batched evaluation takes no flags");
  if (o->grad == KG_GRAD_EXACT) return fail(KG_ERR_UNSUPPORTED, "batched evaluation has no KG_GRAD_EXACT");
  if (o->ckpt_every == KG_CKPT_AUTO)
    return fail(KG_ERR_INVALID_ARG, "batched evaluation takes an explicit ckpt_every (not KG_CKPT_AUTO)");
  if (o->tile_bits != 0 || o->ctas != 0)
    return fail(KG_ERR_INVALID_ARG, "tile_bits and ctas are set by the batch schedule, not the options");
  for (int b = 0; b < B; ++b) {
    kg_status st = check_args(&chains[b], o);
    if (st != KG_OK) return fail(st, "problem " + std::to_string(b) + ": " + g_last_error);
  }
  return KG_OK;
}

}  // namespace

extern "C" {

kg_status kg_batch_workspace_bytes(int32_t B, const kg_chain* chains, const kg_options* opts, size_t* bytes) {
  kg_status st = check_batch(B, chains, opts);
  if (st != KG_OK) return st;
  if (!bytes) return fail(KG_ERR_INVALID_ARG, "bytes must not be NULL");
  *bytes = make_batch_layout(B, chains, opts).total;
  return KG_OK;
}

kg_status kg_batch_create(kg_batch** batch, int32_t B, const kg_chain* chains, const kg_options* opts,
                          const kg_batch_schedule* sched, const double* const* u, const void* const* psi0,
                          const void* const* target, double* fid, double* const* grad, void* workspace,
                          size_t bytes, void* cuda_stream) {
  if (!batch) return fail(KG_ERR_INVALID_ARG, "batch must not be NULL");
  *batch = nullptr;
  kg_status st = check_batch(B, chains, opts);
  if (st != KG_OK) return st;
  if (!u || !psi0 || !target || !fid || (opts->grad != KG_GRAD_NONE && !grad))
    return fail(KG_ERR_INVALID_ARG, "u, psi0, target, fid (and grad) must not be NULL");
  kg_batch_schedule sc{0, 0, 0, 0};
  if (sched) sc = *sched;
  if (sc.reserved0 || sc.reserved1) return fail(KG_ERR_INVALID_ARG, "schedule reserved fields must be 0");
  if (sc.tiles_per_cta == 0) sc.tiles_per_cta = 2;
  if (sc.tiles_per_cta != 1 && sc.tiles_per_cta != 2) return fail(KG_ERR_INVALID_ARG, "tiles_per_cta must be 1 or 2");
  if (sc.ctas < 0 || sc.ctas > kg::kMaxCtas) return fail(KG_ERR_INVALID_ARG, "ctas must be 0..2048");
  const BatchLayout lay = make_batch_layout(B, chains, opts);
  if (!workspace || ((uintptr_t)workspace % kg::kAlign)) return fail(KG_ERR_WORKSPACE, "workspace NULL or not 256-byte aligned");
  if (bytes < lay.total)
    return fail(KG_ERR_WORKSPACE, "workspace too small: need " + std::to_string(lay.total) + " bytes");
  for (int b = 0; b < B; ++b) {
    if (!u[b] || !psi0[b] || !target[b] || (opts->grad != KG_GRAD_NONE && !grad[b]))
      return fail(KG_ERR_INVALID_ARG, "problem " + std::to_string(b) + ": NULL input or output pointer");
    if (((uintptr_t)psi0[b] % 16) || ((uintptr_t)target[b] % 16) || ((uintptr_t)u[b] % 8))
      return fail(KG_ERR_INVALID_ARG, "problem " + std::to_string(b) + ": misaligned pointer");
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  int maxc = 0;
  e = kg::batch_kernel_max_ctas(&maxc);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  int ctas = sc.ctas > 0 ? std::min(sc.ctas, maxc) : maxc;
  if (ctas < 1) return fail(KG_ERR_UNSUPPORTED, "batch kernel does not fit on this device");

  // ---- schedule: largest problems first, each onto the least loaded CTAs it needs
  struct Job {
    int b, g;
    double cost;
  };
  std::vector<Job> jobs(B);
  const double steps_per_slice = (double)opts->m;
  for (int b = 0; b < B; ++b) {
    const int t = batch_tile_bits(chains[b]);
    const int ntiles = 1 << (chains[b].L - t);
    int g = (ntiles + sc.tiles_per_cta - 1) / sc.tiles_per_cta;
    g = std::min(g, std::min(kg::kBatchMaxGroup, ctas));
    const double slices = (double)opts->N * (opts->grad != KG_GRAD_NONE ? 2.0 : 1.0) *
                          (opts->ckpt_every > 0 ? 1.5 : 1.0);
    const double amps_per_cta = (double)((size_t)1 << chains[b].L) / g;
    const double step_us = (g > 1 ? 4.5 : 1.5) + 2.5 * amps_per_cta / 4096.0;
    jobs[b] = {b, g, slices * steps_per_slice * step_us};
  }
  std::stable_sort(jobs.begin(), jobs.end(), [](const Job& a, const Job& c) { return a.cost > c.cost; });
  std::vector<double> busy(ctas, 0.0);
  std::vector<std::vector<kg::BatchItem>> lists(ctas);
  std::vector<int> order(ctas);
  for (const Job& jb : jobs) {
    for (int i = 0; i < ctas; ++i) order[i] = i;
    std::partial_sort(order.begin(), order.begin() + jb.g, order.end(),
                      [&](int a, int c) { return busy[a] < busy[c] || (busy[a] == busy[c] && a < c); });
    double start = 0.0;
    for (int r = 0; r < jb.g; ++r) start = std::max(start, busy[order[r]]);
    for (int r = 0; r < jb.g; ++r) {
      busy[order[r]] = start + jb.cost;
      lists[order[r]].push_back(kg::BatchItem{jb.b, r, jb.g, jb.b});
    }
  }
  std::vector<int> item_off(ctas + 1, 0);
  std::vector<kg::BatchItem> items;
  for (int c = 0; c < ctas; ++c) {
    item_off[c] = (int)items.size();
    items.insert(items.end(), lists[c].begin(), lists[c].end());
  }
  item_off[ctas] = (int)items.size();

  // ---- problem table
  char* ws = (char*)workspace;
  std::vector<kg::EvalParams> probs(B);
  for (int b = 0; b < B; ++b) {
    const kg_chain& ch = chains[b];
    const Layout pl = make_layout(&ch, opts);
    char* w = ws + lay.prob[b];
    kg::EvalParams& p = probs[b];
    p = kg::EvalParams{};
    p.L = ch.L;
    p.N = opts->N;
    p.m = opts->m;
    p.t_bits = batch_tile_bits(ch);
    p.grad_mode = opts->grad;
    p.hc_kind = ch.hc_kind;
    p.hc_site = ch.hc_site;
    p.ckpt = opts->ckpt_every;
    p.hc_mask = ch.hc_site_mask;
    p.Jxy = ch.Jxy;
    p.Jz = ch.Jz;
    p.hc_amp = ch.hc_amp;
    p.dt = opts->dt;
    p.bd_tol = (opts->breakdown_tol > 0.0) ? opts->breakdown_tol : 1e-5;
    p.u = u[b];
    p.psi0 = (const double*)psi0[b];
    p.target = (const double*)target[b];
    p.fid = fid + b;
    p.grad = (opts->grad != KG_GRAD_NONE) ? grad[b] : nullptr;
    p.basis = w + pl.basis;
    p.traj = w + pl.traj;
    p.seg = w + pl.seg;
    p.chi = w + pl.chi;
    p.wbuf = w + pl.wbuf;
    p.xbuf = w + pl.xbuf;
    p.G = (double*)(w + pl.G);
    p.nrm = (double*)(w + pl.nrm);
    p.scal = (double*)(w + pl.scal);
    p.wait_limit_ns = g_wait_limit_ns.load();
    p.debug_fault = 0;
    p.reorth = 0;
    p.Gi = nullptr;
    p.tint = nullptr;
    p.prof = nullptr;
  }
  if ((e = cudaMemcpy(ws + lay.probs, probs.data(), sizeof(kg::EvalParams) * B, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(ws + lay.item_off, item_off.data(), sizeof(int) * (ctas + 1), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(ws + lay.items, items.data(), sizeof(kg::BatchItem) * items.size(), cudaMemcpyHostToDevice)))
    return cuda_fail(e, "cudaMemcpy(batch tables)");

  kg_batch* h = new kg_batch();
  h->B = B;
  h->opts = *opts;
  h->ws = ws;
  h->bytes = bytes;
  h->stream = (cudaStream_t)cuda_stream;
  h->device = dev;
  h->ctas = ctas;
  h->clear_off = lay.ctrl;
  h->clear_bytes = 64 + sizeof(unsigned long long) * (size_t)B;
  h->bp.probs = (const kg::EvalParams*)(ws + lay.probs);
  h->bp.item_off = (const int*)(ws + lay.item_off);
  h->bp.items = (const kg::BatchItem*)(ws + lay.items);
  h->bp.bars = (unsigned long long*)(ws + lay.bars);
  h->bp.reds = (double*)(ws + lay.reds);
  h->bp.ctrl = (int*)(ws + lay.ctrl);
  *batch = h;
  return KG_OK;
}

kg_status kg_batch_launch(kg_batch* b) {
  if (!b) return fail(KG_ERR_INVALID_ARG, "batch must not be NULL");
  cudaError_t e = cudaMemsetAsync(b->ws + b->clear_off, 0, b->clear_bytes, b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(batch control block)");
  e = kg::launch_batch_kernel(b->bp, b->ctas, b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cooperative launch of the batch kernel");
  return KG_OK;
}

kg_status kg_batch_sync(kg_batch* b, int32_t* ctas_used) {
  if (!b) return fail(KG_ERR_INVALID_ARG, "batch must not be NULL");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  int ctrl[2] = {0, 0};
  e = cudaMemcpy(ctrl, b->ws + b->clear_off, sizeof(ctrl), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(status)");
  if (ctas_used) *ctas_used = b->ctas;
  const int st = ctrl[kg::kCtrlStatus];
  if (st == KG_ERR_TIMEOUT) return fail(KG_ERR_TIMEOUT, "a device-side wait ran past its time limit");
  if (st == KG_ERR_NONFINITE) return fail(KG_ERR_NONFINITE, "non-finite Lanczos coefficient or norm");
  if (st != 0) return fail(KG_ERR_CUDA, "device status " + std::to_string(st));
  return KG_OK;
}

kg_status kg_batch_destroy(kg_batch* b) {
  delete b;
  return KG_OK;
}

}  // extern "C"

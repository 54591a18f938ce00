/*
 * kgrape.h - C ABI of the GB300 K-GRAPE hot path (fidelity and gradient of a
 * piecewise-constant control pulse on an open XXZ chain).
 *
 * What is computed (Larocca & Wisniacki, "K-GRAPE", arXiv:2010.03598):
 *   H_j = H0 + u_{j-1} Hc                       (Eq. htot with the PWC ansatz, Eq. PWC)
 *   H0  = sum_{b=0}^{L-2} Jxy (Sx_b Sx_{b+1} + Sy_b Sy_{b+1}) + Jz Sz_b Sz_{b+1}   (Eq. H01)
 *   psi_j = exp(-i dt H_j) psi_{j-1}, j = 1..N, each step by a Lanczos/Krylov
 *           approximation with an m-vector basis                                   (Appendix A)
 *   beta = <f|psi_N>, F = |beta|^2 = 1 - I                                         (Eq. objective)
 *   chi_N = beta f, chi_{j-1} = exp(+i dt H_j) chi_j                                (Alg. "Basic GRAPE", step 6)
 *   G_j = 2 dt Im <chi_j|Hc|psi_j>, j = 0..N                                        (Eq. gradI)
 *   dF/du_{j-1} = G_j                (KG_GRAD_ZEROTH: Hc at the end of slice j, Eq. gradI)
 *   dF/du_{j-1} = (G_{j-1} + G_j)/2  (KG_GRAD_CENTERED: trapezoid over slice j, App. B last paragraph)
 *   dF/du_{j-1} = average of G(t) over slice j by the 4-point Gauss-Lobatto rule
 *                 (KG_GRAD_EXACT: App. B, Eqs. natu_integr and natgrad; see kg_grad_mode)
 * Gradients are of the fidelity F (the paper's are of the infidelity I = 1 - F).
 *
 * Basis convention: amplitude index i in [0, 2^L); site k (1-based) is bit k-1 of i;
 * bit value 0 = spin up (Sz = +1/2), as in the spin-up-is-zero encoding of Sec. 3.1.
 * Complex vectors are interleaved (re, im) pairs: complex128 = two doubles per amplitude.
 *
 * Conventions for every entry point:
 *   - status codes are returned, never thrown; kg_last_error() gives a message for the
 *     calling thread's last failure;
 *   - device pointers belong to the caller; the library allocates no device memory:
 *     every buffer it needs lives in the caller's workspace (size from kg_workspace_bytes);
 *   - work is enqueued on the caller's CUDA stream and is asynchronous unless stated;
 *     errors detected on the device (KG_ERR_TIMEOUT, KG_ERR_NONFINITE) are reported by
 *     kg_sync() after the stream has drained;
 *   - a handle (and its workspace) serves one evaluation at a time: calls that share a
 *     handle must be ordered on one stream.
 */
#ifndef KGRAPE_H
#define KGRAPE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum kg_status {
  KG_OK = 0,
  KG_ERR_INVALID_ARG = 1,  /* a pointer, size or option is out of range */
  KG_ERR_UNSUPPORTED = 2,  /* valid request the library does not implement (e.g. L > 30) */
  KG_ERR_CUDA = 3,         /* a CUDA runtime call failed (message has the CUDA error) */
  KG_ERR_NONFINITE = 4,    /* a Lanczos coefficient or norm became NaN/Inf on the device */
  KG_ERR_TIMEOUT = 5,      /* a device-side wait (group barrier) ran past its time limit */
  KG_ERR_WORKSPACE = 6     /* workspace too small or misaligned (256-byte alignment) */
} kg_status;

typedef enum kg_precision {
  KG_PREC_C128 = 0,        /* complex128 vectors, FP64 arithmetic throughout */
  KG_PREC_C64_F64REC = 1,  /* complex64 vectors and H*v in FP32; alpha/beta recurrences,
                              norms, the m x m exponential and <f|psi_N> in FP64 */
  KG_PREC_FF = 2           /* float-float vectors: each real part and imaginary part is the
                              unevaluated sum hi + lo of two FP32 numbers (about 44 significant
                              bits), H*v, the Lanczos updates, the recombination and the Lanczos
                              sums and scalars in FP32 with error-free transformations (TwoSum,
                              FMA TwoProduct); the tridiagonal, the m x m exponential, the per-slice
                              norms and the overlaps in FP64.  16 bytes per
                              amplitude, like complex128.  Subspace engines (kg_sector_*) only,
                              with KG_GRAD_NONE, _CENTERED or _ZEROTH: it carries the paper's
                              subspace task (Sec. 3.2: 2 x 4D slices of dt = 0.5) to 1e-5 of the
                              complex128 oracle, where the rounding of complex64 Krylov vectors
                              accumulates past it.  The full-chain entry points answer
                              KG_ERR_UNSUPPORTED. */
} kg_precision;

typedef enum kg_grad_mode {
  KG_GRAD_NONE = 0,        /* fidelity only (no backward sweep) */
  KG_GRAD_CENTERED = 1,    /* (G_{j-1} + G_j) / 2, the gradient fed to L-BFGS in Sec. 2 */
  KG_GRAD_ZEROTH = 2,      /* G_j (Eq. gradI) */
  KG_GRAD_EXACT = 3,       /* the natural gradient G(t) = 2 dt Im <chi(t)|Hc|psi(t)> averaged over
                              slice j (App. B, Eqs. natu_integr, natgrad) with the 4-point
                              Gauss-Lobatto rule: nodes t_{j-1} + s, s = 0, (1 -+ 1/sqrt 5) dt/2, dt,
                              weights 1/12, 5/12, 5/12, 1/12; exact up to O(dt^7) per component.
                              The interior states come from the slices' own Krylov bases (two more
                              recombinations per slice and direction); the workspace keeps 2N more
                              vectors.  Not combined with checkpointing (KG_ERR_UNSUPPORTED). */
  KG_GRAD_TAYLOR1 = 4,     /* 2 dt Im <chi_j| Hbar_c^[P] |psi_j> with the slice average of Hc expanded in
                              the Liouvillian L = [H_j, .] (App. B, Eq. gradp):
                              Hbar_c^[P] = sum_{p<=P} (-i dt)^p/(p+1)! L^p Hc, here P = 1 (error
                              O(dt^3) per component; P = 0 would be KG_GRAD_ZEROTH) */
  KG_GRAD_TAYLOR2 = 5      /* the same with P = 2 (error O(dt^4)).  Both Taylor modes are available for
                              parity-excitation subspaces (kg_sector_*), where H_j chi_j and H_j^2 chi_j
                              come from the slice's Lanczos vectors and H_j psi_j, H_j^2 psi_j from one or
                              two extra applications of H_j; kg_create answers KG_ERR_UNSUPPORTED */
} kg_grad_mode;

typedef enum kg_hc_kind {
  KG_HC_SX_SITE = 0,       /* Hc = hc_amp * Sx on site hc_site+1 (bit hc_site) */
  KG_HC_SZ_SITES = 1       /* Hc = hc_amp * sum over set bits s of hc_site_mask of Sz_s;
                              Sec. 3.1's (J/2)(sigma^z_1 + sigma^z_L) is hc_amp = J,
                              mask = 1 | 1 << (L-1) */
} kg_hc_kind;

/* The chain and its control operator (Eq. H01, Eq. htot). */
typedef struct kg_chain {
  int32_t L;               /* number of spins, 1 <= L <= 30; state dimension D = 2^L */
  int32_t hc_kind;         /* kg_hc_kind */
  int32_t hc_site;         /* KG_HC_SX_SITE: 0-based site, 0 <= hc_site < L */
  int32_t reserved0;       /* must be 0 */
  uint64_t hc_site_mask;   /* KG_HC_SZ_SITES: sites the Sz terms act on (bits < L) */
  double Jxy;              /* flip-flop coupling: Jxy (SxSx + SySy) per bond */
  double Jz;               /* Ising coupling: Jz SzSz per bond */
  double hc_amp;           /* amplitude of Hc */
} kg_chain;

/* Pulse, Krylov and execution options. */
typedef struct kg_options {
  int32_t N;               /* number of PWC slices (controls), N >= 1 */
  int32_t m;               /* Krylov basis size (vectors), 1 <= m <= 32 */
  int32_t prec;            /* kg_precision */
  int32_t grad;            /* kg_grad_mode */
  int32_t ckpt_every;      /* 0: keep every psi_j for the backward sweep;
                              C > 0: keep psi_0, psi_C, psi_2C, ... and psi_N, and recompute
                              each segment forward during the backward sweep;
                              KG_CKPT_AUTO: keep every psi_j if that workspace fits mem_budget,
                              else checkpoint every ceil(sqrt(N)) slices (the C that minimises
                              the N/C + C vectors held); the choice is reported in
                              kg_report.ckpt_every */
  int32_t tile_bits;       /* 0 = automatic; else amplitudes per tile = 2^tile_bits (6..13) */
  int32_t ctas;            /* 0 = automatic; else CTAs cooperating on the problem */
  int32_t flags;           /* KG_FLAG_* */
  double dt;               /* slice length, dt > 0 */
  double breakdown_tol;    /* <= 0: 1e-12 (C128) or 1e-5 (C64); Lanczos stops when
                              b_{k+1} <= tol * max(1, max|alpha| + max b) (Alg. "Lanczos",
                              the b_j > 0 test) */
  int64_t mem_budget;      /* with KG_CKPT_AUTO: workspace bytes the caller can give; 0 = 90 % of
                              the memory cudaMemGetInfo reports free on the current device when
                              kg_workspace_bytes / kg_create runs.  Ignored otherwise. */
} kg_options;

/* ckpt_every value that lets the library choose the checkpoint interval (App. B: the trajectory
 * psi_0..psi_N is what limits the memory of the gradient).  Not combined with KG_GRAD_EXACT (the
 * choice is then 0) nor accepted by the batched and subspace entry points. */
#define KG_CKPT_AUTO (-1)

#define KG_FLAG_HOST_STAGING 1u  /* reserve workspace for kg_evaluate_host's input/output copies */
#define KG_FLAG_PHASE_TIMING 2u  /* record per-phase SM cycles of CTA 0 into kg_report.phase_cycles */
/* Full re-orthogonalisation (App. A names it as the remedy for the loss of orthogonality of the
 * Lanczos vectors): after each step, classical Gram-Schmidt of the residual against every basis
 * vector, applied twice; b_{k+1} is the norm of what remains.  Without the flag the recurrence
 * removes only the last two directions, as in Alg. "Lanczos".  Runs the generic streaming
 * kernel (two more passes over the basis per step), for any precision. */
#define KG_FLAG_FULL_REORTH 4u

/* Diagnostics of the last evaluation, filled by kg_sync. */
typedef struct kg_report {
  double krylov_err_max;   /* max over all slices of ||psi|| b_m |[exp(-i dt T) e_1]_{m-1}| */
  double norm_final;       /* ||psi_N|| (1 up to rounding and Krylov error) */
  double beta_re, beta_im; /* <f|psi_N> */
  int32_t breakdowns;      /* slices whose Lanczos basis ended early (invariant subspace) */
  int32_t status;          /* device status word (a kg_status) */
  int32_t launches;        /* kernels launched by the last evaluate call */
  int32_t ctas;            /* CTAs that cooperated on the problem */
  int32_t tile_bits;       /* tile size used */
  int32_t threads;         /* threads per CTA */
  int32_t ckpt_every;      /* checkpoint interval used (0: every psi_j kept), KG_CKPT_AUTO resolved */
  int32_t reserved0;
  int64_t phase_cycles[8]; /* with KG_FLAG_PHASE_TIMING: SM clock cycles CTA 0 spent in
                              [0] Lanczos stage 1 (v_k, partners from other tiles),
                              [1] stage 2 (stencil inside the tile), [2] group reductions
                              incl. the barrier wait, [3] recurrence scalars and broadcast,
                              [4] small exponential, [5] recombination, [6] sweep setup,
                              [7] total; zeros otherwise */
} kg_report;

typedef struct kg_handle kg_handle;   /* opaque host object; owns no device memory */

/* Library version (major*10000 + minor*100 + patch). Never fails. */
int kg_version(void);

/* Message for the calling thread's most recent failure ("" if none). Never fails. */
const char* kg_last_error(void);

/* Workspace bytes needed for (chain, opts) on the current device.
 * Returns KG_ERR_INVALID_ARG / KG_ERR_UNSUPPORTED for bad options. */
kg_status kg_workspace_bytes(const kg_chain* chain, const kg_options* opts, size_t* bytes);

/* Create a handle bound to the current device, a caller-owned device workspace
 * (>= kg_workspace_bytes, 256-byte aligned) and a CUDA stream (cudaStream_t; NULL = legacy
 * default stream).  Chooses the launch configuration.  The workspace must stay valid until
 * kg_destroy; it holds the Krylov basis, the trajectory psi_0..psi_N (or its checkpoints),
 * the co-state, barrier counters and reduction slots. */
kg_status kg_create(kg_handle** handle, const kg_chain* chain, const kg_options* opts,
                    void* workspace, size_t bytes, void* cuda_stream);

/* One fidelity(+gradient) evaluation, asynchronous on the handle's stream.
 *   u      [N]        float64, device: controls, u[j-1] acts in slice j
 *   psi0   [2^L]      complex128, device: initial state
 *   target [2^L]      complex128, device: target f (the caller normalises it)
 *   fid    [1]        float64, device: F = |<f|psi_N>|^2
 *   grad   [N]        float64, device: dF/du (ignored, may be NULL, if opts.grad == NONE)
 * Inputs are read and outputs written by the device after the call returns; they must stay
 * valid until the stream reaches this work. */
kg_status kg_evaluate(kg_handle* handle, const double* u, const void* psi0, const void* target,
                      double* fid, double* grad);

/* Same evaluation with HOST buffers (same shapes and types as kg_evaluate).  Copies the
 * inputs into the workspace (the handle must be created with KG_FLAG_HOST_STAGING), runs,
 * copies F and the gradient back, and waits for the stream.  Pinned host memory makes the
 * copies asynchronous DMA; pageable memory works but is slower.  Returns device-side errors
 * directly (it calls kg_sync). */
kg_status kg_evaluate_host(kg_handle* handle, const double* u, const void* psi0,
                           const void* target, double* fid, double* grad);

/* Wait for the handle's stream, read the device status word and, if rep != NULL, fill it.
 * Returns the device status (KG_OK, KG_ERR_TIMEOUT, KG_ERR_NONFINITE) or KG_ERR_CUDA. */
kg_status kg_sync(kg_handle* handle, kg_report* rep);

/* Destroy the handle (host memory only; the workspace stays the caller's). NULL is a no-op. */
kg_status kg_destroy(kg_handle* handle);

/* Time limit, in nanoseconds, of every device-side wait of later launches in this process
 * (default 2e9).  After a wait runs out the kernel sets KG_ERR_TIMEOUT, every CTA leaves at
 * its next wait, and the launch ends; the context stays usable.  ns must be >= 1. */
kg_status kg_set_wait_limit_ns(int64_t ns);

/* ---------------------------------------------------------------- batched evaluation
 * Many independent pulses (each its own chain, controls, initial state and target; shared
 * kg_options) evaluated by ONE cooperative persistent launch: the host schedules every problem
 * onto a group of CTAs (largest first, onto the least loaded CTAs); each group synchronises
 * on its own barrier, so small problems run on single CTAs without any grid-wide wait.
 * Complex64 path only (KG_PREC_C64_F64REC).  The launch is CUDA-graph capturable: all
 * pointers are fixed when the batch is created. */
typedef struct kg_batch kg_batch;  /* opaque host object; owns no device memory */

typedef struct kg_batch_schedule {
  int32_t ctas;           /* CTAs of the launch; 0 = every CTA that fits co-resident */
  int32_t tiles_per_cta;  /* 1 or 2 (0 = 2): a problem of T tiles gets ceil(T/tiles_per_cta) CTAs */
  int32_t reserved0;      /* must be 0 */
  int32_t reserved1;      /* must be 0 */
} kg_batch_schedule;

/* Workspace bytes for B problems (independent of the schedule). */
kg_status kg_batch_workspace_bytes(int32_t B, const kg_chain* chains, const kg_options* opts, size_t* bytes);

/* Create a batch.  chains[B] (host), opts (host, shared), sched (host, nullable = defaults).
 * u[B], psi0[B], target[B], grad[B]: HOST arrays of DEVICE pointers with the shapes of
 * kg_evaluate (u[b] has opts->N doubles, psi0[b]/target[b] 2^L_b complex128); fid: device
 * array of B doubles.  The pointers are copied; the buffers they point to must stay valid for
 * every launch.  Uploads the problem table into the workspace (synchronously). */
kg_status kg_batch_create(kg_batch** batch, int32_t B, const kg_chain* chains, const kg_options* opts,
                          const kg_batch_schedule* sched, const double* const* u, const void* const* psi0,
                          const void* const* target, double* fid, double* const* grad, void* workspace,
                          size_t bytes, void* cuda_stream);

/* Enqueue one evaluation of every problem of the batch on the batch's stream (a 64-byte
 * memset of the control block plus one cooperative kernel; capturable in a CUDA graph). */
kg_status kg_batch_launch(kg_batch* batch);

/* Wait for the stream and return the device status (as kg_sync). ctas_used (nullable) receives
 * the grid size of the launch. */
kg_status kg_batch_sync(kg_batch* batch, int32_t* ctas_used);

/* Destroy (host memory only). NULL is a no-op. */
kg_status kg_batch_destroy(kg_batch* batch);

/* Size of the library's fixed device scratch array used by kg_evaluate_static. */
#define KG_STATIC_WORKSPACE_BYTES (64ull * 1024ull * 1024ull)

/* One fidelity(+gradient) evaluation that allocates nothing.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory themselves — a host
 * application or runtime that owns the whole device memory budget and forbids further
 * cudaMalloc after start-up, code without a device allocator at hand (plain C callers that
 * have no torch or workspace allocator), or latency-critical loops that must not pay
 * cudaMalloc's implicit device synchronisation.  Instead of a caller workspace it uses a
 * fixed scratch array of KG_STATIC_WORKSPACE_BYTES (64 MiB) compiled into the library
 * (a static __device__ array: every GPU that loads the library holds it until the process
 * exits).  Arguments are those of kg_create + kg_evaluate (device pointers, caller-owned);
 * KG_FLAG_HOST_STAGING is not accepted.  Requests whose workspace (kg_workspace_bytes) exceeds
 * the array are rejected with KG_ERR_WORKSPACE before any device work.
 * The call is synchronous: it enqueues on cuda_stream (NULL = legacy default stream), waits
 * for it and returns the device status like kg_sync.  It must never be called while
 * cuda_stream is being captured into a CUDA graph (the wait and the status read are illegal
 * there): such calls are rejected with KG_ERR_INVALID_ARG before any device work.  Every call
 * on a device shares the one array, which keeps the last call's contents (the control block is
 * cleared at each call): calls that overlap on the GPU — from several host threads or streams —
 * race and give wrong results.  The first call on a device, and the first after the device's
 * context changed (cudaDeviceReset, or another context made current), resolves the array's
 * device address in that context (cudaGetSymbolAddress, which may load the library's device
 * code).  Without a current CUDA context the call returns KG_ERR_CUDA and launches nothing.
 * No device or host memory is allocated on the success path. */
kg_status kg_evaluate_static(const kg_chain* chain, const kg_options* opts, const double* u, const void* psi0,
                             const void* target, double* fid, double* grad, void* cuda_stream);

/* ---------------------------------------------------------------- parity-excitation subspaces
 * Sec. 3.1's own setting.  H0 and a diagonal control Hc = hc_amp * sum_{s in mask} Sz_s keep the
 * number of excitations fixed (set bits of the basis index, i.e. spins down) and, when the mask is
 * mirror-symmetric, commute with the parity Pi that mirrors the chain (bit b <-> bit L-1-b).  An
 * evaluation can then run in one parity-excitation (PE) subspace, which Sec. 3.1 builds by
 * diagonalising Pi on the K-excitation sector and reducing H0 and Hc to the eigenvectors of the
 * wanted parity.  Basis of the subspace (K excitations, parity p):
 *   p = +1: (|s> + |Pi s>)/sqrt 2 for every orbit {s, Pi s} with s < Pi s, and |s> for s = Pi s;
 *   p = -1: (|s> - |Pi s>)/sqrt 2 for every orbit with s < Pi s (palindromes have even parity);
 *   p =  0: |s> for every s with K set bits (no parity reduction);
 * ordered by s ascending (Sec. 3.1 orders the reduced basis by the binary number of the bit string;
 * the smaller member of an orbit is the same whichever end the number starts from).  For states in
 * the subspace, F and the gradient equal those of the full 2^L chain.  Vectors (psi0, target) are
 * complex128 in this basis; the Krylov sweeps, gradient modes and precisions are those of
 * kg_evaluate, plus KG_PREC_FF (float-float vectors, subspaces only).  Each problem of a batch (one control pulse each) runs on one CTA, with the whole
 * state in shared memory; CTAs take problems b, b + grid, b + 2 grid, ...  No device-side wait. */
typedef struct kg_sector {
  int32_t L;               /* number of spins, 2 <= L <= 30 */
  int32_t K;               /* excitations (set bits), 0 <= K <= L */
  int32_t parity;          /* +1 even, -1 odd, 0 the whole K-excitation sector */
  int32_t block_threads;   /* threads per CTA (one pulse per CTA): 0 = chosen from D, or 128, 256,
                              512; with rows per thread of 4 (128), 10 (256, complex64) or 8 (256,
                              complex128 and float-float; 512, where these two take 5 rows up to
                              D = 2560) the block must cover D, else KG_ERR_INVALID_ARG.  The
                              block shape changes only the speed (kg_sector_* results are the same to
                              rounding); tune.py times the shapes */
  uint64_t hc_site_mask;   /* sites of the Sz terms of Hc (bits < L); mirror-symmetric if parity != 0 */
  double Jxy;              /* as kg_chain: flip-flop coupling per bond */
  double Jz;               /* as kg_chain: Ising coupling per bond */
  double hc_amp;           /* amplitude of Hc.  Sec. 3.1's drift (J/2) sum sigma.sigma with alpha_z, and
                              control (J/2)(sigma^z_1 + sigma^z_L), are Jxy = 2J, Jz = 2J alpha_z,
                              hc_amp = J, mask = sites 1 and L */
} kg_sector;

typedef struct kg_sector_handle kg_sector_handle;  /* opaque host object; owns no device memory */

/* Dimension D of the subspace (host only).  KG_ERR_INVALID_ARG for bad fields; KG_ERR_UNSUPPORTED
 * when D exceeds what one CTA holds (the limit depends on prec; see kg_sector_workspace_bytes). */
kg_status kg_sector_dim(const kg_sector* sector, int32_t* D);

/* The smaller member s of every basis vector's orbit, in basis order (host array of D entries;
 * host only).  Use it to place states of the full chain in the subspace and back. */
kg_status kg_sector_states(const kg_sector* sector, uint64_t* states, int32_t D);

/* H0 v on the host, from the same basis and tables the kernel uses (a check of the reduction
 * that needs no GPU): v, w host arrays of D complex128.  Hc is diagonal: hc_amp/2 (popcount(mask)
 * - 2 popcount(s_r & mask)) on row r. */
kg_status kg_sector_apply_h0(const kg_sector* sector, const double* v, double* w, int32_t D);

/* Workspace bytes for B pulses with options opts (N, m <= 32, prec, grad NONE / CENTERED / ZEROTH /
 * EXACT / TAYLOR1 / TAYLOR2 (EXACT keeps 2N interior states per CTA; KG_PREC_FF takes NONE, CENTERED
 * and ZEROTH only, else KG_ERR_UNSUPPORTED; its vectors take 16 bytes per amplitude),
 * dt, breakdown_tol, ctas = most CTAs to use (0 = every one that fits); ckpt_every and tile_bits
 * must be 0; flags: KG_FLAG_PHASE_TIMING only, recording CTA 0's cycles in kg_report.phase_cycles as
 * [0] Lanczos gathers and updates, [1] block reductions, [4] tridiagonal T and small exponential,
 * [5] recombination, [6] pulse setup and overlaps, [7] total).  The workspace holds one trajectory psi_0..psi_N per CTA of the launch, so it
 * is sized for the grid kg_sector_create will choose on the current device (min(B, resident CTAs,
 * ctas); B CTAs if no device is visible).  KG_ERR_UNSUPPORTED for checkpoints or a subspace too large
 * for one CTA's shared memory. */
kg_status kg_sector_workspace_bytes(const kg_sector* sector, const kg_options* opts, int32_t B, size_t* bytes);

/* Create a handle for B pulses on the current device, a caller-owned 256-byte aligned workspace of
 * at least kg_sector_workspace_bytes and a CUDA stream (NULL = legacy default stream).  Builds the
 * subspace's tables on the host and copies them into the workspace (synchronously). */
kg_status kg_sector_create(kg_sector_handle** handle, const kg_sector* sector, const kg_options* opts,
                           int32_t B, void* workspace, size_t bytes, void* cuda_stream);

/* Evaluate B pulses, asynchronous on the handle's stream (one kernel launch).  Device pointers:
 *   u      [B][N] float64: pulse b's controls, u[b][j-1] acts in slice j
 *   psi0   [D] complex128: initial state (shared by all pulses)
 *   target [D] complex128: target state f (shared; normalised by the caller)
 *   fid    [B] float64: F_b = |<f|psi_N>|^2
 *   grad   [B][N] float64: dF_b/du_b (NULL only with KG_GRAD_NONE)
 * psi0/target 16-byte aligned, the others 8-byte aligned. */
kg_status kg_sector_evaluate(kg_sector_handle* handle, const double* u, const void* psi0, const void* target,
                             double* fid, double* grad);

/* Wait for the stream; return the device status (KG_ERR_NONFINITE if a Lanczos coefficient or a
 * norm was not finite; KG_ERR_TIMEOUT if a pulse ran longer than 60 times the kg_set_wait_limit_ns
 * limit, i.e. 2 minutes by default, checked at every slice).  rep (nullable): beta and norm_final of pulse 0, the largest Krylov error
 * indicator and the total breakdowns over all pulses, the grid (ctas) and threads per CTA. */
kg_status kg_sector_sync(kg_sector_handle* handle, kg_report* rep);

kg_status kg_sector_destroy(kg_sector_handle* handle);

/* Test hook for failure detection.  kind 1: in the next launch, CTA 0 does not arrive at
 * the first group barrier (a member that never joins); the other CTAs' waits, and its own,
 * run out after the wait limit and the launch ends with KG_ERR_TIMEOUT (read by kg_sync).
 * kind 2: the same at the barrier of the first Lanczos step instead (in the resident complex64
 * loop of 4096-amplitude tiles, the barrier its control warp arrives at and waits on).  Only
 * multi-CTA launches have a group barrier.  The hook applies to one launch and then clears
 * itself; kind 0 clears it.  Nothing faults, traps or hangs.  Returns KG_ERR_INVALID_ARG for
 * another kind. */
kg_status kg_debug_set_fault(int32_t kind);

#ifdef __cplusplus
}
#endif

#endif /* KGRAPE_H */

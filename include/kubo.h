/*
 * kubo.h -- C ABI of the GB300 Kubo-formula anomalous Hall conductivity library.
 *
 * The library evaluates, for every k-point of a uniform Brillouin-zone mesh, the four
 * steps of the paper's baseline algorithm (Sec. 2.2, List 1; batched form Sec. 2.3,
 * List 2 and Eq. 4) and the k-sum of Eq. 2:
 *
 *   (1) H(k) = sum_R e^{i k.R} H(R),  d_a H(k) = sum_R i R_a e^{i k.R} H(R), a = x, y
 *   (2) H(k) = U diag(E) U^dagger                     (Hermitian eigendecomposition)
 *   (3) v^a  = U^dagger d_a H U                       ("convert" to the eigenbasis)
 *   (4) Omega_n = -2 sum_{m != n} Im(v^x_nm v^y_mn) / ((E_n - E_m)^2 + eta^2)   (Eq. 3)
 *   S(E_F) = (1/N_k) sum_k sum_n occ(E_n(k); E_F) Omega_n(k)                      (Eq. 2)
 *
 * occ is theta(E_F - E_n) (occupied iff E_n < E_F) for kT = 0, else the Fermi-Dirac
 * factor 1/(1 + exp((E_n - E_F)/kT)).  S is dimensionless (lattice units, integer R);
 * for one 2-D layer the Chern number is 2 pi S, and the 3-D conductivity is
 * sigma_xy = -(e^2/hbar) S / V_cell (conversion left to the caller).  The paper's
 * Eq. 3 omits eta; eta > 0 regularises near-degenerate pairs.  With eta = 0, pairs with
 * |E_n - E_m| <= 1e-12 max|E| are skipped.
 *
 * Memory conventions.
 *   - complex128 arrays are interleaved (re, im) doubles, row-major.
 *   - H_R: [N_R][W][W] complex128 with H(-R) = H(R)^dagger; R_vecs: [N_R][3] int32,
 *     closed under R -> -R and containing R = 0.
 *   - k-point linear index: (j1*N2 + j2)*N3 + j3 for k = 2 pi (j1/N1, j2/N2, j3/N3).
 *   - "packed Hermitian" (W*W doubles) P of a Hermitian A: P[i][j] = Re A_ij for i <= j
 *     and P[i][j] = Im A_ji for i > j.
 *   - The caller owns every buffer; the library never frees caller memory.
 *
 * Errors.  Every entry point validates its arguments on the host before any launch and
 * returns a kubo_status; no C++ exception crosses the ABI.  Entry points that take H_R
 * also check Hermitian pairing on the device (max |H(-R) - H(R)^dagger| <= 1e-12 max|H|,
 * all entries finite).  Calls are stream-ordered on opt->stream and return after that
 * stream has completed the call's work (the device status word is read back), so the
 * returned status covers device-detected errors too.  Outputs are written only when the
 * call returns KUBO_OK.
 */
#ifndef KUBO_H
#define KUBO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KUBO_OK = 0,
  KUBO_ERR_INVALID_ARG = 1,     /* bad size, null pointer, non-finite eta/kT/E_F, ... */
  KUBO_ERR_NOT_HERMITIAN = 2,   /* H(-R) != H(R)^dagger beyond 1e-12 max|H|, or non-finite H */
  KUBO_ERR_R_NOT_CLOSED = 3,    /* some -R missing, R = 0 missing, or duplicate R */
  KUBO_ERR_UNSUPPORTED = 4,     /* W or precision outside what this build supports */
  KUBO_ERR_OOM = 5,             /* device allocation failed */
  KUBO_ERR_CUDA = 6,            /* a CUDA runtime call failed */
  KUBO_ERR_NO_CONVERGENCE = 7,  /* eigensolver hit its iteration cap at some k-point */
  KUBO_ERR_WORKSPACE = 8,       /* caller workspace smaller than kubo_workspace_size() */
  KUBO_ERR_TIMEOUT = 9          /* a bounded device-side wait (tensor-core pipeline) gave up */
} kubo_status;

typedef enum {
  KUBO_FP64 = 0,            /* every step in FP64 */
  KUBO_MIXED = 1,           /* the mixed-precision form: step (1) on the tensor cores (fixed-point
                               BF16 slices with exact FP32 block accumulation: H(k) to ~2^-31
                               relative, the velocity columns, which feed only step (3), to
                               ~2^-23, stored in FP32 for W <= 64); the eigensolver in FP64:
                               Householder reduction, inverse iteration for the eigenvectors,
                               and as eigenvalues the FP64 Rayleigh quotients of those vectors
                               (the QL iteration, which only supplies the inverse iteration's
                               shifts, runs in double-float); step (3) in FP32, with U = Q D Z
                               formed in FP32 from the FP64 factors; energy differences and the
                               k-sum in FP64; curvature quotient in FP32 (FP64 below a 2^-86
                               denominator) */
  KUBO_MIXED_FOURIER = 2,   /* error-budget mode: only step (1) mixed, step (3) in FP64 */
  KUBO_MIXED_ROTATION = 3,  /* error-budget mode: only step (3) mixed (FP32), step (1) in FP64 */
  KUBO_MIXED_DF = 4         /* KUBO_MIXED with the eigensolver in double-float instead of FP64:
                               pairs of FP32 (~2^-46 per operation) on the FP32 pipe, FP64 in and
                               out; eigenvalues to ~1e-12 relative at W = 64.  Not an FP64
                               eigensolver: a faster variant at the same 1e-5 target on S. */
} kubo_precision;
/* Magnitude range.  S(E_F) is unchanged when H(R), E_F, eta and kT are scaled by one factor
 * (Omega is homogeneous of degree zero in them).  In the modes whose step (3) runs in FP32
 * (KUBO_MIXED, KUBO_MIXED_ROTATION, KUBO_MIXED_DF) an H(R) whose largest entry lies outside
 * [2^-20, 2^20] is therefore scaled inside the call by the power of two that brings that entry
 * into [1, 2), with eta scaled alike and the eigenvalues scaled back: exact, and it leaves the
 * FP32 products and the FP32 pairs no magnitude range of their own.  The separable Fourier sum
 * (kubo_options.fourier_separable) does not scale: with it keep max |H(R)| within [2^-40, 2^40]
 * in KUBO_MIXED_ROTATION. */

/* Pipeline stages, for the optional per-stage timing in kubo_profile. */
enum {
  KUBO_STAGE_PREP = 0,          /* Hermitian check, twiddles, packed Fourier basis */
  KUBO_STAGE_FOURIER = 1,       /* step (1) */
  KUBO_STAGE_TRIDIAG = 2,       /* step (2): Householder tridiagonalisation */
  KUBO_STAGE_QL = 3,            /* step (2): implicit QL on the tridiagonals */
  KUBO_STAGE_BACKTRANSFORM = 4, /* step (2): eigenvectors U = Q D Z */
  KUBO_STAGE_BERRY = 5,         /* steps (3)-(4) */
  KUBO_STAGE_KSUM = 6,          /* k-sum of Eq. 2 */
  KUBO_STAGE_FIXUP = 7,         /* mixed precision: FP64 redo of k-points with a level near E_F */
  KUBO_STAGE_ADJOINT = 8,       /* kubo_ahc_grad: reverse mode of steps (1)-(4) */
  KUBO_N_STAGES = 9
};

/* Per-stage kernel launch counts and summed device time (CUDA events recorded on the call's
 * stream around each launch).  The library adds to the fields; the caller zeroes them. */
typedef struct kubo_profile {
  int64_t launches[KUBO_N_STAGES];
  double ms[KUBO_N_STAGES];
  int64_t fixup_k;          /* k-points re-evaluated in FP64 by the mixed-precision fix-up */
} kubo_profile;

typedef struct kubo_options {
  int precision;            /* kubo_precision; default KUBO_FP64 */
  int n_eta;                /* > 0: evaluate every broadening in etas (host array) */
  const double* etas;       /*       and write out as [n_eta][n_EF]; 0: use the eta arg */
  double kT;                /* 0: step occupation; > 0: Fermi-Dirac temperature (energy units) */
  int64_t k_begin, k_end;   /* sub-range [k_begin, k_end) of linear mesh indices; both 0 =
                               whole mesh.  The weight stays 1/N_k, so results over a
                               partition of the mesh add up to the full-mesh result. */
  void* stream;             /* cudaStream_t; NULL = legacy default stream */
  void* workspace;          /* device scratch of workspace_bytes; NULL = the library
                               allocates it (cudaMallocAsync from the current device's DEFAULT
                               memory pool) and frees it inside the call.  Process-wide side
                               effect of a library allocation: so that the freed workspace stays
                               mapped for the next call (re-mapping GBs costs ~30 ms per call),
                               the library raises that default pool's release threshold
                               (cudaMemPoolAttrReleaseThreshold) to the largest workspace it
                               has used, and never lowers it; other cudaMallocAsync users of the
                               same pool in the process see that threshold too.  A caller that
                               must keep its own threshold passes a workspace here. */
  size_t workspace_bytes;
  int chunk_k;              /* k-points per internal batch; 0 = automatic (a fixed 24 GiB of
                               batch buffers, at most 65,536 k-points) */
  kubo_profile* profile;    /* non-NULL: accumulate per-stage launch counts and times */
  double mixed_fixup_rel;   /* KUBO_MIXED / KUBO_MIXED_FOURIER, k-summed entry points; > 0
                               enables an FP64 redo of every k-point with some
                               |E_n - E_F| < rel * max_n |E_n| (occupations that a reduced-
                               precision energy could flip) and of the 0.5 % of each batch with
                               the largest ||Omega(k)||_inf (near-degenerate pairs).  <= 0 (the
                               default) = no fix-up. */
  double grad_eps;          /* kubo_ahc_grad: broadening eps of the eigenvector-derivative
                               kernel (E_j - E_i) / ((E_j - E_i)^2 + eps^2) (energy units);
                               <= 0 (the default) = 1e-12 max_n |E_n(k)| at each k. */
  int layout_unpadded;      /* 1: shared-memory matrices of the eigenvector and rotation
                               kernels with leading dimension W instead of the padded one
                               (W + 1 for FP64 matrices, the W + P = 4 mod 16 of the FP32
                               rotation) -- the padding ablation (Sec. 2.3 pads against
                               memory-bank conflicts); slower, same results.  0 (default):
                               padded. */
  int fourier_separable;    /* 1: step (1) as three one-axis sums over the bounding box of the
                               R set instead of the dense contraction (FP64; precision
                               KUBO_FP64 or KUBO_MIXED_ROTATION; kubo_ahc / kubo_ahc_host with a
                               k-range of whole k1-planes; bounding box at most 8 N_R vectors;
                               otherwise KUBO_ERR_UNSUPPORTED).  Same result up to rounding
                               order.  0 (default): dense contraction. */
  int rotation_tc;          /* kernel of the FP32-grade step (3) in KUBO_MIXED /
                               KUBO_MIXED_ROTATION / KUBO_MIXED_DF for W <= 64 (larger W: batched
                               FP32 GEMMs), one accuracy class:
                               3 = tensor cores in 3xTF32: tcgen05 kind::tf32 with every FP32
                                 operand split into two TF32 parts (hi lo + lo hi + hi hi per
                                 product, a fresh FP32 accumulator per K-quarter of 32, the
                                 quarters summed with round-to-nearest), k-points padded to 64;
                               1 = tensor cores with exact fixed-point BF16-slice products;
                               2 = FP32 on the FMA pipe (SIMT);
                               0 (default) = automatic: 3 for 40 < W <= 64, where it is at least
                                 as fast as 2 (and at W = 64 the more accurate), else 2.
                               Other values: KUBO_ERR_INVALID_ARG.  layout_unpadded = 1 implies
                               2 (the ablation concerns the SIMT kernel's shared-memory
                               layout). */
  int ql_max_sweeps;        /* cap on the implicit-QL sweeps spent on one eigenvalue; 0 = the
                               default (60, far above the 2-3 that Wilkinson shifts need).  A
                               k-point that reaches the cap makes the call return
                               KUBO_ERR_NO_CONVERGENCE with its outputs untouched; a cap of 1
                               forces that path on any matrix that needs a second sweep.
                               < 0: KUBO_ERR_INVALID_ARG. */
  int ql_fp64;              /* KUBO_MIXED: 1 = its QL iteration in FP64 as well and the QL
                               eigenvalues reported (every operation of the eigensolver in
                               FP64); 0 (default) = the QL iteration in double-float, used only
                               for the inverse iteration's shifts, and the eigenvalues reported
                               as the FP64 Rayleigh quotients of the FP64 eigenvectors (equal to
                               the FP64 QL ones within a few W eps max|E|).  Ignored by the other
                               modes.  Other values: KUBO_ERR_INVALID_ARG. */
} kubo_options;

/* Fill *opt with the defaults (FP64, single eta, kT = 0, whole mesh, default stream,
 * library-managed workspace, automatic batch size). */
void kubo_options_init(kubo_options* opt);

/* Human-readable name of a status code (static storage). */
const char* kubo_status_string(kubo_status s);

/* Largest orbital count W supported by this build for the given precision (128 for every
 * precision).  Up to W = 64 the eigenvectors and the rotations of a k-point are formed inside
 * one thread block each; for 64 < W <= 128 they run as batched multi-pass kernels whose
 * scratch is part of the workspace. */
int kubo_max_orbitals(int precision);

/*
 * Anomalous Hall sum S(E_F) over the k-mesh (Eq. 2 with the integrand of Eq. 3; the
 * steps of List 1 / List 2 evaluated for every mesh point).
 *   H_R    device, complex128 [N_R][W][W]
 *   R_vecs host,   int32 [N_R][3]
 *   kmesh  host,   int32 [3], each >= 1
 *   E_F    device, double [n_EF]  (any order)
 *   out    device, double [n_eta][n_EF]  (n_eta = opt->n_eta if > 0, else 1 with eta)
 * Returns KUBO_OK or an error; on error out is untouched.
 */
kubo_status kubo_ahc(const double* H_R, const int32_t* R_vecs, int W, int N_R,
                     const int32_t* kmesh, const double* E_F, int n_EF, double eta,
                     double* out, const kubo_options* opt);

/*
 * Same computation as kubo_ahc with HOST buffers for H_R, E_F and out: the library copies
 * H_R and E_F to the device and out back to the host inside the call.
 */
kubo_status kubo_ahc_host(const double* H_R, const int32_t* R_vecs, int W, int N_R,
                          const int32_t* kmesh, const double* E_F, int n_EF, double eta,
                          double* out, const kubo_options* opt);

/*
 * Per-k results for a list of mesh points (steps (1)-(4) of List 1 without the k-sum):
 *   kidx   device, int64 [n_k] linear mesh indices (each in [0, N_k), checked on the device
 *          before anything is computed: KUBO_ERR_INVALID_ARG otherwise; any order, repeats
 *          allowed)
 *   E      device, double [n_k][W]            eigenvalues, ascending
 *   Omega  device, double [n_eta][n_k][W]     band Berry curvatures
 * opt->k_begin/k_end are ignored.
 */
kubo_status kubo_ahc_k(const double* H_R, const int32_t* R_vecs, int W, int N_R,
                       const int32_t* kmesh, const int64_t* kidx, int64_t n_k, double eta,
                       double* E, double* Omega, const kubo_options* opt);

/*
 * Step (1) alone ("define_matrices" of List 1/2): packed Hermitian H(k), d_x H(k), d_y H(k)
 * for the listed mesh points.
 *   Hk, dHx, dHy  device, double [n_k][W*W] each (packed Hermitian)
 */
kubo_status kubo_bloch(const double* H_R, const int32_t* R_vecs, int W, int N_R,
                       const int32_t* kmesh, const int64_t* kidx, int64_t n_k,
                       double* Hk, double* dHx, double* dHy, const kubo_options* opt);

/*
 * Step (2) alone: batched Hermitian eigendecomposition ("diagonalize" of List 2, the
 * batched EISPACK-style solver of Sec. 2.3) in FP64.
 *   A  device, double [n][W*W] packed Hermitian matrices
 *   E  device, double [n][W] ascending eigenvalues
 *   U  device, complex128 [n][W][W]; column j is the eigenvector of E[j] (U may be NULL
 *      to compute eigenvalues only)
 */
kubo_status kubo_eigh_batched(const double* A, int W, int64_t n, double* E, double* U,
                              const kubo_options* opt);

/*
 * Steps (3)-(4) alone ("convert" + "evaluate" of List 1/2): band Berry curvatures from
 * eigenpairs and velocity matrices.
 *   E        device, double [n][W]
 *   U        device, complex128 [n][W][W] (columns = eigenvectors)
 *   dHx, dHy device, double [n][W*W] packed Hermitian
 *   Omega    device, double [n_eta][n][W]
 */
kubo_status kubo_berry_batched(const double* E, const double* U, const double* dHx,
                               const double* dHy, int W, int64_t n, double eta,
                               double* Omega, const kubo_options* opt);

/*
 * Allocation-free batched eigensolver: the same computation and output layout as
 * kubo_eigh_batched, for callers that cannot let a library allocate device memory during
 * a call -- for example applications whose own allocator has reserved (nearly) all of the
 * GPU's memory up front, where a cudaMalloc from inside the library would fail, and
 * latency-critical loops in which cudaMalloc/cudaFree would synchronise the device.  The
 * paper has no counterpart to this entry point.
 *
 * It calls no cudaMalloc, cudaFree or allocating library routine.  Its intermediates live
 * in one fixed 32 MiB block of device memory compiled into the library (every GPU that
 * loads the library holds that block until the process exits).  Limits:
 *   - W <= 64; a larger W returns KUBO_ERR_UNSUPPORTED without launching anything.
 *   - any n >= 1: the matrices are processed in passes of as many as fit in the block
 *     (about 480 per pass at W = 64, about 6900 at W = 16).
 * Every call looks up the block's device address on the current device (a symbol lookup,
 * which allocates nothing), so an address never outlives a device reset.  The first call on a
 * device also loads the library's device code there; make that first call before any stream
 * capture.  Every call
 * shares the block and it keeps the previous call's contents (the call clears what must
 * start at zero), so calls that overlap on the GPU -- on different streams or from
 * different host threads on the same device -- race and corrupt each other's results:
 * serialise them.  The call returns after `stream` (a cudaStream_t; NULL = legacy default
 * stream) has finished its work.
 *   A  device, double [n][W*W] packed Hermitian;  E  device, double [n][W] ascending;
 *   U  device, complex128 [n][W][W] (columns = eigenvectors), or NULL for eigenvalues only.
 */
kubo_status kubo_eigh_batched_noalloc(const double* A, int W, int64_t n, double* E, double* U,
                                      void* stream);

/*
 * Gradient of the anomalous Hall sum with respect to H(R) (reverse mode of Eq. 2-3 and of
 * steps (1)-(4); the paper evaluates sigma only, this is its adjoint).  FP64 only: any other
 * opt->precision returns KUBO_ERR_UNSUPPORTED.
 *   dL_dout   device, double [n_eta][n_EF]: weights g of L = sum g[e][j] S_e(E_F_j) (the
 *             incoming gradient of the outputs of kubo_ahc)
 *   grad_H_R  device, complex128 [N_R][W][W]: G(R) = dL/dRe H(R) + i dL/dIm H(R), the
 *             Hermitian part of H(k), d_x H(k), d_y H(k) being what L depends on; hence
 *             G(-R) = G(R)^dagger.  A Hermitian-paired real step d of H(R)_ij and H(-R)_ji
 *             changes L by 2 d Re G(R)_ij (d Re G(0)_ii for a diagonal entry of H(0)); an
 *             imaginary step i d by 2 d Im G(R)_ij.  This is also PyTorch's convention for the
 *             gradient of a real loss with respect to a complex tensor.
 *   out       device, double [n_eta][n_EF] or NULL: S(E_F) of the same call (as kubo_ahc)
 * Other arguments and options as kubo_ahc (etas, kT: Fermi-Dirac occupation derivative
 * included; kT = 0 differentiates the step almost everywhere, i.e. without the Fermi-surface
 * term; k_begin/k_end; opt->grad_eps).  The eigenvectors are recomputed batch by batch inside
 * the call (never stored for the whole mesh).  Deterministic.  grad_H_R and out are written
 * only on KUBO_OK.
 */
kubo_status kubo_ahc_grad(const double* H_R, const int32_t* R_vecs, int W, int N_R,
                          const int32_t* kmesh, const double* E_F, int n_EF, double eta,
                          const double* dL_dout, double* grad_H_R, double* out,
                          const kubo_options* opt);

/*
 * Many models in one call (the paper's high-throughput setting: one sigma per material, many
 * materials).  Each problem carries the arguments kubo_ahc takes for one model; every model
 * is summed over its whole mesh.
 */
typedef struct kubo_problem {
  const double* H_R;        /* device, complex128 [N_R][W][W] */
  const int32_t* R_vecs;    /* host, int32 [N_R][3] */
  int W, N_R;
  int32_t kmesh[3];
  const double* E_F;        /* device, double [n_EF] */
  int n_EF;
  double eta;               /* broadening when opt->n_eta == 0 */
  double* out;              /* device, double [n_eta][n_EF]; written only if status == KUBO_OK */
  kubo_status status;       /* written by the call: this model's result */
} kubo_problem;

/* Schedule of a kubo_ahc_batched call.  In: 0 fields are chosen by the library; tune = 1 runs
 * the autotuner (candidate schedules timed on a probe of every model's first k-points; the
 * winner is cached per batch signature).  Out: the schedule that ran. */
typedef struct kubo_batch_schedule {
  int tune;                 /* in: 1 = autotune the fields below that are 0 */
  int streams;              /* concurrent CUDA streams the models are spread over */
  int chunk_k;              /* upper bound on the k-points per internal batch of a model */
  int graph;                /* in: 0 = capture the batch in a CUDA graph (default), -1 = no */
  double probe_ms;          /* out: the tuner's time for the chosen schedule (0 if not tuned) */
  int tuned_candidates;     /* out: configurations the tuner timed (0 if cached or not tuned) */
  /* Kernel parameters, applied to every model (in: 0 = the default, or tuned when tune = 1;
   * out: the values used).  The tuner first picks streams and chunk_k on the default kernel
   * parameters, then tries each parameter's alternatives in turn on that schedule. */
  int fourier_group_m;      /* tensor-core Fourier sum: 128-k tiles rasterised together per
                               column tile of the H columns (L2 reuse of the basis tiles; the
                               velocity columns use min(64, 4 x this)); default 8, tuned over
                               {4, 8, 16}; 1..64 */
  int symv_parts;           /* Householder reduction: cap on the column partitions per row of
                               its symv (W <= 64: the count up to the cap with the fewest FP64
                               instructions for each trailing order; W > 64: the cap where
                               the threads allow); default 4, tuned over {2, 4, 8}; 1..8 */
  int rotation;             /* step (3) kernel as kubo_options.rotation_tc (1..3 fix it);
                               0 = opt->rotation_tc, tuned over {automatic, 2, 3} when that is
                               0 and the precision has an FP32-grade step (3) */
} kubo_batch_schedule;

/*
 * sigma for n_probs models of uneven W, N_R and k-mesh in one call.  Models are ordered by
 * estimated cost (longest first) and spread over `streams` concurrent streams; the whole batch
 * (basis preparation, every k-batch of every model, the k-sums) is captured in one CUDA
 * graph and launched once.  Shared settings come from opt (precision, etas, kT, stream);
 * opt->k_begin/k_end must be 0, opt->workspace NULL (the library allocates), and the mixed-
 * precision fix-up and per-stage profile are not available in this entry point.  Hermitian
 * pairing of every model is checked before any model runs.  Returns KUBO_OK when every model
 * succeeded, else the first failing model's status (every problem's status field is set).
 * sched may be NULL (library defaults).  Deterministic for a given schedule.
 */
kubo_status kubo_ahc_batched(kubo_problem* probs, int n_probs, const kubo_options* opt,
                             kubo_batch_schedule* sched);

/*
 * Failure-detection check (no counterpart in the paper): runs, on one thread, the bounded
 * mbarrier wait that every pipeline wait of the tensor-core kernel uses, on a barrier that
 * nothing completes, giving up after `spins` tries.  Returns KUBO_ERR_TIMEOUT -- the status a
 * stalled tensor-core pipeline reports -- and leaves the context usable; no fault, trap or
 * hang is involved.  spins < 1: KUBO_ERR_INVALID_ARG.  stream: cudaStream_t (NULL = legacy).
 */
kubo_status kubo_check_bounded_wait(uint32_t spins, void* stream);

/*
 * Test hook (no counterpart in the paper): the next `n` device allocations that the library
 * itself attempts (the workspace of kubo_ahc, kubo_ahc_host, kubo_ahc_k, kubo_ahc_grad,
 * kubo_bloch, kubo_eigh_batched, kubo_berry_batched and the batch buffer of kubo_ahc_batched)
 * fail as if the device were out of memory, so that callers can exercise their handling of
 * KUBO_ERR_OOM without exhausting a shared GPU.  Nothing is launched or allocated by this call;
 * n <= 0 clears a pending count.  Process-wide; thread-safe.
 */
void kubo_debug_fail_allocations(int n);

/* Device bytes of scratch a kubo_ahc / kubo_ahc_k call with these sizes needs. */
size_t kubo_workspace_size(int W, int N_R, const int32_t* kmesh, int n_EF,
                           const kubo_options* opt);

/* Device bytes of scratch a kubo_ahc_grad call with these sizes needs (0 for invalid sizes
 * or a precision other than KUBO_FP64). */
size_t kubo_grad_workspace_size(int W, int N_R, const int32_t* kmesh, int n_EF,
                                const kubo_options* opt);

#ifdef __cplusplus
}
#endif

#endif /* KUBO_H */

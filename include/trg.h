/*
 * trg.h — C ABI of libtrg: the triad-ATRG coarse-graining step for 4D lattice spin
 * models on one NVIDIA B300 (sm_103a).
 *
 * Method: Y. Sugimoto, S. Sasaki, "Triad representation for the anisotropic tensor
 * renormalization group in four dimensions", arXiv:2507.21909.
 *
 * Conventions shared by every entry point
 *   - One library-global context (not thread-safe).  All device memory is allocated and
 *     owned by the library; callers pass scalars and HOST pointers only.
 *   - The coarse tensor is held on the device as T = sum_g Phi[i1,i2,i3,i4,g]
 *     Psi[j1,j2,j3,j4,g] (forward legs x backward legs, rank-factorised), FP64,
 *     row-major with g fastest, and an optional impurity factor Psi_imp.
 *   - Return value: TRG_OK (0) or a negative TRG_ERR_* code; trg_last_error() gives a
 *     one-line message.  No entry point aborts or exits the process.
 *   - Results written to host pointers are valid when the call returns (the library
 *     synchronises its own stream before returning host scalars).
 */
#ifndef TRG_H
#define TRG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef int trg_status;

#define TRG_OK             0
#define TRG_ERR_ARG       -1   /* bad argument (range, NULL pointer, unsupported d)   */
#define TRG_ERR_OOM       -2   /* device allocation failed                            */
#define TRG_ERR_CUDA      -3   /* a CUDA runtime call or kernel launch failed         */
#define TRG_ERR_NONFINITE -4   /* NaN/Inf in the norm c_n or a spectrum               */
#define TRG_ERR_TIMEOUT   -5   /* a bounded device-side iteration did not converge    */
#define TRG_ERR_NOINIT    -6   /* no model initialised                                */

/* Precision of the contractions (trg_set_params): */
#define TRG_PREC_FP64      0   /* every GEMM in FP64 on CUDA cores (parity form)       */
#define TRG_PREC_BF16X3    1   /* bulk GEMMs as 3-term BF16-split tcgen05, FP32 accum */
#define TRG_PREC_BF16X6    2   /* bulk GEMMs as 6-term BF16-split tcgen05, FP32 accum */
#define TRG_PREC_BF16X10   3   /* bulk GEMMs as 10-term BF16-split tcgen05, FP32 accum */
#define TRG_PREC_OZ4       4   /* bulk GEMMs with 4 exact 7-bit digits per row (10
                                  tcgen05 products), exact FP32 chunks + int64 sums      */
#define TRG_PREC_OZ5       5   /* 5 digits (15 products)                               */
#define TRG_PREC_OZ6       6   /* 6 digits (21 products)                               */
#define TRG_PREC_TF32X3    7   /* bulk GEMMs as 3xTF32 tcgen05 (kind::tf32: a_hi b_hi +
                                  a_hi b_lo + a_lo b_hi), FP32 accum                     */
#define TRG_PREC_OZ7       8   /* 7 digits (28 products), levels 0..3 exact: the FP64-
                                  equivalent digit GEMM, for every bulk GEMM             */
/* In the mixed forms (1..8) the first three steps run in FP64, later steps put their bulk
 * GEMMs on the tensor cores.  In the digit forms (4..6, 8) the products that the bulk
 * rule keeps off the tensor cores (Grams and R^-1 products of the orthonormalisations,
 * squeezer Gram roots, thin products) run as the seven-digit FP64-equivalent GEMM. */

/* Initial tensor of the d-dimensional Ising model, Sec. III (CP form
 * T = sum_a prod_legs W[a, leg], W = [[sqrt(cosh b), sqrt(sinh b)],
 * [sqrt(cosh b), -sqrt(sinh b)]]) with an added site field e^{h s}.
 * d: 4 (the paper's case) or 3 (the three-dimensional triad step whose cost the paper
 * gives at the end of Sec. II B).  beta >= 0.  The impurity factor (one site carrying
 * s) is created as well.  Resets the log-norm sum to ln c_0, c_0 = ||T_0||_F, and the
 * step counter to 0.  Errors: TRG_ERR_ARG (d not 3 or 4, beta < 0 or not finite, h not
 * finite), TRG_ERR_OOM, TRG_ERR_CUDA. */
trg_status trg_init_ising(int d, double beta, double h);

/* Z_q clock model (extension, not in the paper): bond weight e^{beta cos(th-th')},
 * th = 2 pi k / q, factorised in the real Fourier basis; site weight e^{h cos th};
 * impurity observable cos th.  d = 3 or 4, q in [2, 8], beta >= 0.  Errors:
 * TRG_ERR_ARG, TRG_ERR_OOM, TRG_ERR_CUDA. */
trg_status trg_init_clock(int d, int q, double beta, double h);

/* One triad-ATRG coarse-graining step along physical axis `axis` (0..d-1):
 * re-split T = A s D (eq. ABCD), bond swap by randomized SVD (Appendix A, eqs.
 * bond1/bond2, XY), triad isometries from the canonical-form Grams (eq. HOSVD), triads
 * E..L (eqs. E-L), squeezers from the Gram matrices O, P (Sec. II B), coarse
 * contraction Phi / Psi (eqs. makeMG, makeMH), then T <- T / c_n with
 * c_n = ||T||_F and lnZ bookkeeping sum += ln(c_n) / 2^n.
 * D >= 1: bond dimension kept.  sketch_oversample p >= 0: the overspanned internal
 * lines have width chi = min(D + p, natural dimension) (r = eta = (D+p)/D).
 * Errors: TRG_ERR_NOINIT, TRG_ERR_ARG, TRG_ERR_OOM, TRG_ERR_CUDA, TRG_ERR_NONFINITE. */
trg_status trg_step(int axis, int D, int sketch_oversample);

/* Free energy per site of the current 2^N-site periodic lattice (N = steps taken):
 * lnZ/V = sum_n ln(c_n)/2^n + 2^-N ln Tr T_N (legs mu paired with mu),
 * f = -(lnZ/V)/beta (Sec. III A).  f is NaN when beta = 0.  Either pointer may be
 * NULL.  Errors: TRG_ERR_NOINIT, TRG_ERR_CUDA. */
trg_status trg_free_energy(double *f_per_site, double *lnZ_per_site);

/* One-site impurity expectation <s> (Ising) or <cos th> (clock):
 * Tr(Phi Psi_imp^T) / Tr(Phi Psi^T).  The impurity is coarse-grained with the pure
 * tensor's frozen projectors, averaged over its two slots in each step (the impurity
 * tensors of Sec. III D, one site).  After trg_set_impurity_pair and a step it returns
 * the pair's <o_x o_(x+e)>.  Errors: TRG_ERR_NOINIT (no model or no impurity factor),
 * TRG_ERR_ARG (m NULL), TRG_ERR_CUDA. */
trg_status trg_magnetisation_impurity(double *m);

/* Parameters of the randomized SVDs and the precision mode (defaults: 4, 4, 0x5EED,
 * TRG_PREC_FP64).  q_swap >= 1 rounds of the bond-swap loop (q of eqs. bond1/bond2,
 * Appendix A); q_rho >= 0 extra power rounds of the triad / squeezer range finders;
 * seed of the counter-based Gaussian sketches; precision TRG_PREC_* (an extension: the
 * paper runs FP64).  Take effect from the next trg_step or trg_atrg_step.
 * Errors: TRG_ERR_ARG (q_swap < 1, q_rho < 0, precision outside 0..8). */
trg_status trg_set_params(int q_swap, int q_rho, unsigned long long seed, int precision);

/* Internal-line overspanning of the bond swap, the ILO form (Sec. II C; Appendix A with
 * r_bond > 1): from the next trg_step on, the re-split bonds alpha, beta and the swapped
 * bond gamma keep r_bond D singular values instead of D, and the bond-swap sketch has
 * r_bond D + p columns (p = sketch_oversample; p = D gives the appendix's (r_bond + 1) D).
 * The triad isometries and squeezers, and so the coarse tensor's pair legs, are as in
 * the plain form; the coarse tensor's bond (last index of Phi and Psi) has r_bond D
 * values.  r_bond = 1 (default) is the plain method.  Applies to the single-instance
 * path (trg_init_* / trg_step); batched lanes use r_bond = 1.
 * Errors: TRG_ERR_ARG (r_bond outside 1..8). */
trg_status trg_set_bond_overspan(int r_bond);

/* Two-impurity network (Sec. III D; the internal energy from two impurity tensors).  Called
 * after trg_init_* and before the first trg_step: the impurity (s, resp. cos theta) is
 * placed on both sites of the first step's unit cell, i.e. on nearest neighbours along
 * that step's axis; the first step contracts them into one coarse impurity tensor with
 * the pure tensor's projectors, and later steps carry it like the one-site impurity.
 * trg_magnetisation_impurity then returns <o_x o_(x+e)>.  A new trg_init_* or
 * trg_set_state returns to the one-site impurity.
 * Errors: TRG_ERR_NOINIT (no model), TRG_ERR_ARG (a step was already taken). */
trg_status trg_set_impurity_pair(void);

/* Ising coupling energy per site (Sec. III D) U = -(1/V) d lnZ/d beta = -d <s_x s_(x+e)>, from the
 * merged pair of trg_set_impurity_pair (the pair's axis stands for every axis; the
 * field term -h <s> is not included).  Errors: TRG_ERR_ARG (u NULL, not the Ising
 * model), TRG_ERR_NOINIT (no merged pair: trg_set_impurity_pair and one step first). */
trg_status trg_internal_energy(double *u);

/* Plain ATRG (eqs. makeG / makeH), the paper's comparison method, for the Ising model
 * in d = 2, 3 or 4 dimensions, with its own state (independent of trg_init_* /
 * trg_step).  Same re-split, Gaussian sketches (trg_set_params: q_swap, q_rho, seed,
 * precision), squeezer rule and normalisation as the triad step; the bond swap and the
 * blocks A X sigma, Y D are formed as tensors of D^(2d) values, so d = 4 is limited to
 * small D (about 12 on one GPU).  For d = 2 the triad form coincides with this method
 * (Sec. II B), and the free energy compares with Onsager's solution.
 * trg_atrg_init_ising: T0 of Sec. III in d dimensions with field h.  Errors:
 * TRG_ERR_ARG (d outside 2..4, beta < 0 or not finite), TRG_ERR_OOM, TRG_ERR_CUDA. */
trg_status trg_atrg_init_ising(int d, double beta, double h);
/* One plain-ATRG step (eqs. makeG / makeH) along physical axis 0 <= axis < d, bond
 * dimension D, sketch oversampling p (bond-swap sketch width D + p, squeezer ranges
 * min(D + p, pair dimension)).  On an error the ATRG state keeps its factors.
 * Errors: TRG_ERR_NOINIT, TRG_ERR_ARG, TRG_ERR_OOM, TRG_ERR_CUDA, TRG_ERR_NONFINITE. */
trg_status trg_atrg_step(int axis, int D, int sketch_oversample);
/* f and lnZ/V of the ATRG state, as trg_free_energy (Sec. III A).  Either pointer may be
 * NULL.  Errors: TRG_ERR_NOINIT, TRG_ERR_CUDA. */
trg_status trg_atrg_free_energy(double *f_per_site, double *lnZ_per_site);
/* Diagnostics of the ATRG state (not in the paper): ln c_n of the last step, the
 * smallest relative gap at its bond-swap and squeezer cuts, steps taken.  Any pointer
 * may be NULL.  Reads host-side values only; always TRG_OK. */
trg_status trg_atrg_diag(double *log_c, double *min_gap, int *nsteps);

/* Run all device work on this cudaStream_t (NULL = the library's own stream); the
 * previous stream is synchronised first.  A service of the library (no counterpart in
 * the paper).  Errors: TRG_ERR_CUDA. */
trg_status trg_set_stream(void *cuda_stream);


/* Diagnostics of the last step (not in the paper): ln c_n, the smallest relative
 * singular-value gap at the bond-swap and squeezer truncations (a gap near 0 marks a
 * near-degenerate cut, where two implementations may keep different subspaces), and the
 * number of steps taken.  Any pointer may be NULL; always TRG_OK. */
trg_status trg_diag(double *log_c, double *min_gap, int *nsteps);

/* Device time (ms, CUDA events on the library stream) of the phases of the last step:
 * [0] leg rotation + re-split, [1] bond swap, [2] triad isometries, [3] triads, Grams O, P
 * and environments, [4] squeezers, [5] coarse contraction Phi, Psi, [6] impurity,
 * [7] normalisation and state update.  Writes min(n, 8) values.  Measurement service
 * (not in the paper).  Errors: TRG_ERR_ARG (ms NULL or n < 0), TRG_ERR_CUDA. */
trg_status trg_step_timings(double *ms, int n);

/* Counters of the tensor-core GEMM launches inside trg_step / trg_atrg_step since the
 * last reset, written to out[0..min(n, 13)):
 *   [0] exact-digit GEMM (3..6 digits, TRG_PREC_OZ4..6) device ms (CUDA events on the
 *   launching stream), [1] its algorithmic flop, 2 M N K per product asked for (the
 *   FP64-equivalent work), [2] its tensor-pipe flop (every BF16 digit product counted,
 *   a TF32 product as two), [3] its launches, [4..7] the same for the split GEMM
 *   (TRG_PREC_BF16X*, TRG_PREC_TF32X3, and the impurity-only products of the digit forms),
 *   [8..11] the same for the seven-digit FP64-equivalent digit GEMM (TRG_PREC_OZ7, and the
 *   decomposition products of the digit forms), [12] all kernel launches of the library.
 * reset != 0 zeroes them after reading.  Measurement service (not in the paper).
 * Errors: TRG_ERR_ARG (out NULL with n > 0, n < 0). */
trg_status trg_kernel_stats(double *out, int n, int reset);

/* Device scratch of the step engine in bytes: in use now, high-water mark, reserved.
 * Any pointer may be NULL; always TRG_OK. */
trg_status trg_mem_stats(long long *in_use, long long *high_water, long long *reserved);

/* Gu-Wen ratio of the current coarse tensor (Sec. III D, eq. X):
 * X = (Tr A)^2 / Tr(A^2) with A_kl = sum T[i1 i2 i3 k, i1 i2 i3 l], the open leg being the
 * slot of the last physical axis (t) and the other three traced pairwise.  X counts the
 * ground-state degeneracy: -> 1 in the disordered phase, -> 2 in the Z2-ordered phase;
 * for the initial Ising tensor at h = 0, X = 2 / (1 + exp(-4 beta)).  Synchronises.
 * Errors: TRG_ERR_NOINIT, TRG_ERR_ARG (X NULL). */
trg_status trg_gu_wen_ratio(double *X);

/* Copy a state factor to the host.  which: 0 = Phi, 1 = Psi, 2 = Psi_imp.
 * dims_out[0..4] receives (d1, d2, d3, d4, r); host may be NULL (query only), else it
 * must hold `capacity` doubles >= d1 d2 d3 d4 r.  axes_out[0..3] (may be NULL) gets
 * the physical axis of each leg slot.  A three-dimensional state (d1, d2, d3, r) is
 * reported as (d1, d2, d3, 1, r), the same row-major layout, with axes_out[3] = -1.
 * Errors: TRG_ERR_NOINIT, TRG_ERR_ARG. */
trg_status trg_get_state(int which, int *dims_out, int *axes_out, double *host,
                         long long capacity);

/* beta, the running sum ln Z/V so far without the final trace (sum_n ln c_n / 2^n) and
 * the step count of the current state: with trg_get_state, everything trg_set_state
 * needs to resume a run.  Any pointer may be NULL.  Errors: TRG_ERR_NOINIT,
 * TRG_ERR_CUDA. */
trg_status trg_get_scalars(double *beta, double *logsum, int *nsteps);

/* Load a state (e.g. an oracle state at step n, for per-step parity):
 * dims[0..4] = (d1, d2, d3, d4, r), phi/psi[/psi_imp (may be NULL)] row-major host
 * arrays, axes[0..3] the physical axis of each slot, nsteps taken so far and the
 * log-norm sum so far.  dims[3] = 1 with axes[3] = -1 loads a three-dimensional state
 * (d1, d2, d3, r) (axes[0..2] a permutation of 0..2).  Errors: TRG_ERR_ARG (NULL pointers, a dim < 1, axes not a
 * permutation of 0..3, negative nsteps, beta or logsum not finite), TRG_ERR_NONFINITE
 * (a NaN or Inf in phi, psi or psi_imp), TRG_ERR_OOM.  Arguments and buffers are checked
 * on the host before the current state is touched, so a rejected call leaves it as it
 * was. */
trg_status trg_set_state(double beta, const int *dims, const double *phi,
                         const double *psi, const double *psi_imp, const int *axes,
                         int nsteps, double logsum);

/* C = alpha op(A) op(B) + beta C for host row-major FP64 buffers (op = transpose when
 * ta / tb != 0), computed on the device in `precision` (TRG_PREC_*): the FP64 CUDA-core
 * GEMM or the split-BF16 tcgen05 GEMM that the step uses.  For verification and
 * benchmarking of the contraction engine.  Errors: TRG_ERR_ARG, TRG_ERR_OOM,
 * TRG_ERR_CUDA, TRG_ERR_TIMEOUT. */
trg_status trg_gemm(int precision, int ta, int tb, long long M, long long N, long long K,
                    double alpha, const double *A, long long lda, const double *B,
                    long long ldb, double beta, double *C, long long ldc);

/* C = alpha op(A) op(B) + beta C like trg_gemm, but on the caller's DEVICE buffers
 * (row-major FP64, leading dimensions lda, ldb, ldc) and without allocating anything.
 * The paper has no counterpart; this is a service of the library's contraction engine,
 * for callers that cannot call cudaMalloc where they need a product: host frameworks
 * that own all device memory through their own pool and forbid foreign allocations,
 * real-time loops that must not risk an allocation stall or an out-of-memory failure
 * after start-up, and code that must not let cudaMalloc synchronise the device in the
 * middle of its own asynchronous work.
 * precision: TRG_PREC_BF16X3, _BF16X6 or _BF16X10 (the split-BF16 tcgen05 GEMM; the
 * FP64 CUDA-core GEMM needs a workspace and is not offered here).  lda >= K (ta = 0) or
 * M (ta != 0), ldb >= N (tb = 0) or K (tb != 0), ldc >= N.  The only scratch is a fixed
 * 64 MiB __device__ array in the library (every GPU that loads the library holds it
 * until the process exits); problems that need more (BF16 slices of A and B plus
 * split-K partial tiles) are rejected with TRG_ERR_ARG and a message.  The work is
 * queued on `stream` (a cudaStream_t, NULL = legacy default stream); the call then
 * waits for it (cudaStreamSynchronize) and returns TRG_ERR_TIMEOUT if a bounded wait
 * inside the tensor-core kernel gave up, in which case C is not valid.  If `stream` is
 * capturing work when the call is made, it is not waited on and no kernel status is
 * returned.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream capture.  Every
 * call shares the array and leaves its contents behind; all scratch is overwritten
 * before it is read, so nothing carries over between calls, but calls whose work
 * overlaps on the GPU (different streams, or different host threads) race on it:
 * serialise them.
 * Errors: TRG_ERR_ARG (before any work is queued), TRG_ERR_CUDA, TRG_ERR_TIMEOUT; see
 * trg_last_error(). */
trg_status trg_gemm_noalloc(int precision, int ta, int tb, long long M, long long N,
                            long long K, double alpha, const double *A, long long lda,
                            const double *B, long long ldb, double beta, double *C,
                            long long ldc, void *stream);

/* ---------------------------------------------------------------------------------
 * Batched coupling sweep: many independent instances of the step (each its own model,
 * beta, h, D, p and sketch seed), e.g. the sweep over couplings and bond dimensions that
 * locates a transition.  The paper runs one lattice at a time; the instances share
 * nothing but the GPU.  `lanes` engine contexts (each its own CUDA stream and scratch
 * arena, driven by its own host thread) run concurrently; every instance is bound to one
 * lane, which steps its instances in index order.  Lanes hold one bond dimension each
 * (a lane's arena grows to its largest instance): the largest D gets a quarter of the
 * lanes, the smaller (latency-bound) sizes share the rest by cost D^7 + 24^7; with fewer
 * lanes than distinct sizes, longest-processing-time assignment over all instances.  Results do not depend on the lane count or schedule: each
 * instance goes through exactly the kernels of trg_step.  The batch is independent of
 * the single-instance context of trg_init_* / trg_step.
 * ------------------------------------------------------------------------------- */

/* Create n instances: model[i] = 0 (Ising) or q in 2..8 (Z_q clock), beta[i] >= 0, h[i],
 * D[i] >= 1, p[i] >= 0 (NULL: 2 D[i]), seed[i] (NULL: 0x5EED); all in d = 4, with the
 * common q_swap, q_rho and precision (TRG_PREC_*).  Replaces any earlier batch.  Host
 * arrays of length n, read during the call.  Errors: TRG_ERR_ARG, TRG_ERR_OOM,
 * TRG_ERR_CUDA. */
trg_status trg_batch_create(int n, const int *model, const double *beta, const double *h,
                            const int *D, const int *p, const unsigned long long *seed,
                            int lanes, int q_swap, int q_rho, int precision);

/* Every instance takes nsteps steps, each along the axis after its previous one
 * (instance step k is along axis k mod 4).  *wall_ms (may be NULL) = host wall time of
 * the call, all lanes synchronised.  Errors name the first failing lane. */
trg_status trg_batch_step(int nsteps, double *wall_ms);

/* Per instance (host arrays of length n, any may be NULL): f per site, ln Z/V, the
 * one-site impurity observable (Ising: <s>, clock: <cos theta>), steps taken, as
 * trg_free_energy / trg_magnetisation_impurity per instance.  Errors: TRG_ERR_NOINIT (no
 * batch), TRG_ERR_CUDA. */
trg_status trg_batch_results(double *f, double *lnz, double *m, int *nsteps);

/* lane_of[i] (length n) and the scratch bytes each lane has reserved (length lanes);
 * either may be NULL.  Errors: TRG_ERR_NOINIT (no batch). */
trg_status trg_batch_lanes(int *lane_of, long long *scratch_bytes);

/* Release every instance and lane (no batch: nothing to do).  Always TRG_OK. */
trg_status trg_batch_free(void);

/* Gu-Wen ratio of every instance (host array of length n); see trg_gu_wen_ratio
 * (Sec. III D, eq. X).  Errors: TRG_ERR_NOINIT (no batch), TRG_ERR_ARG (X NULL),
 * TRG_ERR_CUDA. */
trg_status trg_batch_gu_wen(double *X);

/* ---------------------------------------------------------------------------------
 * Learned sketch of the triad-isometry range finders (Sec. II B, eq. HOSVD: U^A, U^X,
 * U^Y, U^D are ranges of the Grams rho over a leg pair (a, b), n = d_a d_b).  The paper
 * draws a Gaussian sketch G (n x chi); the learned form keeps the same G and rescales
 * its rows, Omega[(a b), m] = w1[a] w2[b] G[(a b), m], w_l[i] = 2^(round(16 u_l[i])/16)
 * (clamped to 2^-8..2^8), with u_l[i] the output of a 3-layer MLP (5 -> 256 -> 256 -> 1,
 * ReLU, FP32 weights, BF16 inference) on five statistics of index i of leg l: (i+0.5)/d_l,
 * log2(max(m_i d_l, 2^-40))/8 with m_i the share of tr(rho) on index i's diagonal entries,
 * log2(d_l)/8, log2(d_other)/8 and chi/n.  The learned range is kept unless its probe
 * residual ||rho P - Q Q^T rho P||_F (8 Gaussian probe columns) exceeds 1.5x that of the
 * plain range, which is then used instead.  Training targets are 0.5 log2(leverage d_l)
 * of each leg index in the plain method's range.
 *
 * Parameters: one flat FP32 array of TRG_SKETCH_PARAMS values, in the order W1 (256 x 5,
 * row-major), b1 (256), W2 (256 x 256), b2 (256), W3 (256), b3 (1).
 * ------------------------------------------------------------------------------- */
#define TRG_SKETCH_IN 5
#define TRG_SKETCH_PARAMS 67585

/* Load the network (host FP32 array of n = TRG_SKETCH_PARAMS values; copied). Resets
 * the Adam moments.  Errors: TRG_ERR_ARG (wrong n or NULL), TRG_ERR_CUDA. */
trg_status trg_sketch_set_net(const float *params, long long n);

/* Copy the current network to the host (n = TRG_SKETCH_PARAMS).  Errors: TRG_ERR_ARG
 * (wrong n or NULL), TRG_ERR_NOINIT (none loaded), TRG_ERR_CUDA. */
trg_status trg_sketch_get_net(float *params, long long n);

/* u[r] for rows x TRG_SKETCH_IN host inputs X (row-major); bf16 != 0: the inference
 * kernel used inside trg_step (BF16 inputs, weights and activations, FP32 sums),
 * bf16 == 0: the FP32 training forward pass.  Host buffers; synchronous.  Errors:
 * TRG_ERR_ARG (NULL buffers, rows < 1), TRG_ERR_NOINIT (no network), TRG_ERR_CUDA. */
trg_status trg_sketch_forward(const float *X, long long rows, float *u, int bf16);

/* Loss L = mean (u - t)^2 of the FP32 network over rows (X rows x 5, t rows; host) and
 * its gradient (host, TRG_SKETCH_PARAMS floats, parameter order as above).  Errors:
 * TRG_ERR_ARG (NULL buffers, rows < 1), TRG_ERR_NOINIT (no network), TRG_ERR_CUDA. */
trg_status trg_sketch_grad(const float *X, const float *t, long long rows, double *loss,
                           float *grad);

/* Adam (beta 0.9, 0.999, eps 1e-8, rate lr) over `epochs` passes of shuffled minibatches
 * of `batch` rows (host std::mt19937_64(seed) permutation; a ragged last batch is
 * skipped); *loss = mean loss of the last epoch.  The network must be loaded.
 * Errors: TRG_ERR_ARG (NULL buffers, rows, epochs or batch < 1), TRG_ERR_NOINIT,
 * TRG_ERR_OOM, TRG_ERR_CUDA. */
trg_status trg_sketch_train(const float *X, const float *t, long long rows, int epochs,
                            int batch, float lr, unsigned long long seed, double *loss);

/* 0: Gaussian sketches (the paper's form, default); 1: learned sketch with the plain
 * range as fallback.  Errors: TRG_ERR_ARG (other modes), TRG_ERR_NOINIT (1 without a
 * loaded network). */
trg_status trg_set_sketch_mode(int mode);

/* Collect training rows during trg_step: every triad range finder (with chi < n) appends
 * d_a + d_b rows (inputs, target) computed from its plain range, up to `capacity` rows
 * (later rows are counted as dropped).  capacity 0 stops collecting and frees the
 * buffer; a new call discards earlier rows.  Errors: TRG_ERR_ARG (capacity < 0),
 * TRG_ERR_OOM, TRG_ERR_CUDA. */
trg_status trg_sketch_collect(long long capacity);

/* Copy the collected rows to the host: X (capacity x 5 floats), t (capacity floats);
 * either may be NULL (then only *rows / *dropped are written).  TRG_ERR_ARG if
 * capacity < the number of collected rows; TRG_ERR_CUDA. */
trg_status trg_sketch_fetch(float *X, float *t, long long capacity, long long *rows,
                            long long *dropped);

/* Range finders that kept the learned range / fell back to the plain one since the last
 * reset (reset != 0 zeroes the counters after reading).  Either pointer may be NULL.
 * Errors: TRG_ERR_CUDA. */
trg_status trg_sketch_stats(long long *learned, long long *fallback, int reset);

/* Release every device buffer of the library: the single-instance and ATRG states, the
 * batch, the sketch network and collection buffers, the scratch arena.  Always TRG_OK
 * (release errors are ignored). */
trg_status trg_finalize(void);

/* Message of the last error (static storage, never NULL). */
const char *trg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TRG_H */

/*
 * syk.h -- C ABI of the GB300 (sm_103a) matrix-free Krylov engine for the
 * Sachdev-Ye-Kitaev model (Kobrin et al., "Many-Body Chaos in the SYK Model").
 *
 * Conventions shared by every call
 * --------------------------------
 * Model.  H = sum_{i<j<k<l} J_ijkl chi_i chi_j chi_k chi_l (Eq. 1), N even,
 *   4 <= N <= 64, Majoranas normalised by {chi_i, chi_j} = delta_ij and mapped
 *   to n = N/2 spins by the Jordan-Wigner map of Supp. Sec. I.A (spin k = bit k
 *   of the basis index; sigma^y = i sigma^x sigma^z).  Indices are 0-based.
 * Parity sectors.  H conserves the parity of popcount(x) (Supp. Sec. I.A).
 *   Sector p in {0 = even, 1 = odd} has dimension D = 2^(n-1); its compact
 *   index c is the low n-1 bits of x, and x = c | ((popcount(c)+p) & 1) << (n-1).
 * Vectors.  A batch of B states is stored state-interleaved: element (c, b)
 *   of a D x B array is at offset c*B + b.  dtype SYK_C64 stores each element
 *   as two floats (re, im), SYK_C128 as two doubles.  Every scalar reduction
 *   (Lanczos alpha/beta, dots, norms) and the tridiagonal exponential are FP64
 *   for both dtypes.
 * Memory.  Vector arguments are DEVICE pointers owned by the caller unless a
 *   parameter says "host".  The library owns the term tables (device copies
 *   are uploaded on first use, on the current device) and its internal
 *   scratch.  Calls taking `stream` (a cudaStream_t, NULL = legacy default
 *   stream) are asynchronous unless they return host arrays, which
 *   synchronise the stream before returning.
 * Errors.  Every int-returning call returns SYK_OK (0) or a negative code and
 *   never throws; syk_last_error() gives a message for the calling thread.
 */
#ifndef SYK_H
#define SYK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SYK_OK 0
#define SYK_EINVAL (-1)   /* bad argument (size, index, dtype, null pointer) */
#define SYK_ENOMEM (-2)   /* host or device allocation failed, or workspace too small */
#define SYK_ECUDA (-3)    /* CUDA runtime error (message in syk_last_error) */
#define SYK_ENUMERIC (-4) /* NaN/Inf in a Lanczos scalar or a non-positive norm where one is needed */
#define SYK_ETIMEOUT (-5) /* a bounded device-side wait gave up */

#define SYK_C64 1
#define SYK_C128 2

typedef struct syk_terms syk_terms;

/* ---------------------------------------------------------------- Hamiltonian
 * syk_build_terms -- Eq. 1 and Supp. Sec. I.A/I.B ("symbolic representation of
 * H, which contains only O(N^4) terms").  J: host array of C(N,4) real
 * couplings for i<j<k<l in lexicographic order.  Builds, on the host, the
 * Pauli string of every term (chi_i chi_j chi_k chi_l = (1/4) i^p X^m Z^z with
 * X^m Z^z|x> = (-1)^popcount(z&x) |x^m>) and the per-X-mask coefficient
 * tables the kernels evaluate.  *out is library-owned: free it with
 * syk_free_terms.  No GPU is touched.  Errors: SYK_EINVAL (N odd, <4, >64,
 * NULL), SYK_ENOMEM.
 */
int syk_build_terms(int N, const double* J, syk_terms** out);
void syk_free_terms(syk_terms* terms);

/* syk_terms_info -- sizes of a term set (any pointer may be NULL):
 * N, C(N,4) terms, number of distinct X-masks, sector dimension D. */
int syk_terms_info(const syk_terms* terms, int* N, int64_t* nterms, int64_t* nmasks, int64_t* dim);

/* syk_term_table -- host copy of the Pauli form of every term, in
 * lexicographic term order (Supp. Sec. I.A): xmask, zmask (bit k = spin k) and
 * phase p in 0..3 such that 4 chi_i chi_j chi_k chi_l = i^p X^xmask Z^zmask.
 * Each output is a caller-owned host array of C(N,4) entries (NULL skips it). */
int syk_term_table(const syk_terms* terms, uint64_t* xmask, uint64_t* zmask, uint8_t* phase);

/* --------------------------------------------------------------- matvec (K1)
 * syk_apply_H -- y = H psi in parity sector `parity` (Supp. Sec. I.B: the
 * matrix-free "core computational component", O(N^4 2^{N/2}) work).
 * psi, y: device D x batch arrays of `dtype`; must not overlap.  Errors:
 * SYK_EINVAL, SYK_ECUDA. */
int syk_apply_H(const syk_terms* terms, int parity, int dtype, const void* psi, void* y,
                int64_t batch, void* stream);

/* syk_status -- synchronises `stream` and reads the status word that the matvec kernels
 * launched with this term set (on the current device) write when a bounded device-side wait
 * gives up: SYK_ETIMEOUT if a wait for a staged tile ran out since the last reset (those
 * results are incomplete; the kernel still let every copy it had started land before it
 * exited, so the context stays usable), else SYK_OK.  syk_apply_H itself is asynchronous
 * and cannot report it; syk_expmv and the correlators check the word at every convergence
 * check and return SYK_ETIMEOUT.  The word is sticky: reset != 0 clears it. */
int syk_status(const syk_terms* terms, int reset, void* stream);

/* syk_c128_arith -- arithmetic of the complex128 matvec: mode 0 (the default) does the
 * multiply-adds in double-float form, each double carried as an unevaluated sum of two
 * floats and every product and sum made exact with FP32 error-free transformations (Knuth's
 * TwoSum, Dekker's TwoProduct by FMA), because GB300 runs FP64 FMA at 1/64 of the FP32 rate;
 * mode 1 uses native FP64.  Double-float keeps 48 significand bits, so a matvec differs from
 * the FP64 one by about 1e-13 relative (FP64 rounding: 1e-16).  Vectors stay complex128 in
 * memory in both modes; the double-float kernel covers batches of 1, 2, 4, 8 and 16 on the
 * tiled path (other launches use FP64).  mode < 0 only queries.  Returns the mode in effect
 * before the call, or SYK_EINVAL.  The paper computes in complex128 throughout; the mode
 * changes the arithmetic, not the stored precision. */
int syk_c128_arith(int mode);

/* syk_apply_chi -- y = chi_i psi (Supp. Sec. I.A map, with the 1/sqrt(2) that
 * {chi_i, chi_i} = 1 requires).  psi is in sector parity_in; y is in sector
 * 1 - parity_in.  Device D x batch arrays; must not overlap. */
int syk_apply_chi(int N, int i, int parity_in, int dtype, const void* psi, void* y, int64_t batch,
                  void* stream);

/* --------------------------------------------------------- Krylov (K2 - K4)
 * syk_tridiag_expm -- the m x m step of the Krylov method (Supp. Sec. I.B:
 * "exponentiating the projection of H within the subspace"): for each of
 * `batch` real symmetric tridiagonal matrices T_b (alpha[k*batch+b] on the
 * diagonal, beta[k*batch+b] for k < m-1 off it) returns
 * out[k*batch+b] = beta0[b] * (e^{z T_b} e_1)_k as (re, im) doubles.
 * All pointers are device pointers; 1 <= m <= SYK_MAX_KRYLOV. */
#define SYK_MAX_KRYLOV 64
int syk_tridiag_expm(int m, int64_t batch, const double* alpha, const double* beta,
                     const double* beta0, double z_re, double z_im, double* out, void* stream);

/* syk_workspace_bytes -- device scratch syk_expmv needs for (N, dtype,
 * krylov_dim, batch): the Krylov basis of krylov_dim+1 vectors, one work
 * vector and the FP64 scalars, plus for SYK_C128 one more vector (the
 * double-float copy of the matvec input, see syk_c128_arith).  `kind` is
 * reserved (pass 0). */
size_t syk_workspace_bytes(int N, int dtype, int krylov_dim, int64_t batch, int kind);

/* syk_expmv -- out = e^{z H} psi in sector `parity` by Lanczos with full
 * classical Gram-Schmidt reorthogonalisation against the whole basis (two
 * passes for SYK_C128, one for SYK_C64) (Supp. Sec. I.B;
 * Saad 1992 a-posteriori error estimate).  z = z_re + i z_im: z = -i t for
 * real time, z = -tau for imaginary time.  Each Krylov basis of dimension
 * <= krylov_dim (2..SYK_MAX_KRYLOV) advances all states of the batch by a
 * common sub-step chosen so that the estimated relative error of the step is
 * <= tol; steps repeat until z is covered ("dividing the time evolution into
 * a series of small time steps").  A happy breakdown (invariant subspace)
 * shortens the basis.  workspace: device scratch of ws_bytes >=
 * syk_workspace_bytes(...), or NULL to let the library allocate it.  psi and
 * out may be the same array.  *nsteps (may be NULL) receives the number of
 * Krylov bases used.  Synchronises `stream` once per Krylov basis.
 * Errors: SYK_EINVAL, SYK_ENOMEM, SYK_ECUDA, SYK_ENUMERIC. */
int syk_expmv(const syk_terms* terms, int parity, int dtype, double z_re, double z_im,
              const void* psi, void* out, int64_t batch, int krylov_dim, double tol,
              void* workspace, size_t ws_bytes, void* stream, int* nsteps);

/* syk_lanczos_orth -- orthogonalisation of syk_expmv's Lanczos basis for `dtype` (used by
 * every call that evolves a state: the correlators, the batch and the gradients; the
 * eigenvalue Lanczos always uses two full passes).  mode 0: classical Gram-Schmidt of each
 * new vector against the whole basis (the default for SYK_C128: one pass for SYK_C64, two
 * for SYK_C128); mode 1: the three-term recurrence alone (each vector orthogonalised against
 * the two before it; the default for SYK_C64).  In finite precision the
 * three-term recurrence loses global orthogonality as Ritz values converge, but the Krylov
 * approximation of a matrix function is known to stay accurate to about the rounding level
 * of the vectors (Druskin, Greenbaum & Knizhnerman 1998), and it reads 2 basis vectors per
 * step instead of 2(j+1).  mode < 0 only queries.  Returns the previous mode or SYK_EINVAL.
 * Supp. Sec. I.B does not specify the Krylov variant. */
int syk_lanczos_orth(int dtype, int mode);

/* syk_expmv_static -- syk_expmv with its workspace in a fixed array of device
 * memory inside the library, so the call itself allocates nothing.  The paper
 * has no counterpart; this entry point is for callers that cannot allocate
 * device memory when they call: services whose device memory is budgeted up
 * front and must not fail with out-of-memory mid-run, hosts that route every
 * device allocation through their own pool, and latency-critical loops where
 * cudaMalloc/cudaFree would stall or synchronise the device.  It calls no
 * cudaMalloc, cudaFree or other allocating routine, and unlike syk_expmv it
 * never records or instantiates CUDA graphs of its Lanczos iterations (an
 * instantiated graph takes device memory): every kernel is launched directly.
 * Limit: the scratch array is SYK_STATIC_SCRATCH_BYTES (16 MiB) of static
 * device memory, held by every GPU that loads the library until the process
 * exits; a call whose syk_workspace_bytes(N, dtype, krylov_dim, batch, 0)
 * exceeds it fails with SYK_ENOMEM.  The term set must already be on the
 * current device (any earlier call with it on this device uploads it), else
 * SYK_EINVAL.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any stream
 * capture.  Every call uses the same array, which keeps the previous call's
 * contents (the call zeroes what must start at zero); calls that overlap on the
 * GPU (other streams or host threads) race on it, so the caller must
 * serialise them.  Arguments, results and other errors as syk_expmv. */
#define SYK_STATIC_SCRATCH_BYTES (16u << 20)
int syk_expmv_static(const syk_terms* terms, int parity, int dtype, double z_re, double z_im,
                     const void* psi, void* out, int64_t batch, int krylov_dim, double tol,
                     void* stream, int* nsteps);

/* ------------------------------------------------------------- correlators
 * syk_correlator_G -- real-time two-point function, Eq. G with Eq.
 * q_typicality: for each of `nstates` states psi~ (in the EVEN sector),
 * phi = e^{-beta H/2} psi~,
 * G(t) = <phi| e^{iHt} chi_i e^{-iHt} chi_i |phi> / <phi|phi>  (G_R = 2 Re G).
 * t: host array of nt >= 1 non-negative, non-decreasing times.  psi0: D x
 * nstates array, device or host memory (host memory is copied in).  Outputs
 * are host arrays: G_re_im[(k*nstates + s)*2 + {0,1}] and Z[s] = <phi|phi>.
 * Synchronises `stream`. */
int syk_correlator_G(const syk_terms* terms, double beta, int i, const double* t, int nt,
                     const void* psi0, int64_t nstates, int dtype, int krylov_dim, double tol,
                     double* G_re_im, double* Z, void* stream);

/* syk_otoc -- regularized OTOC, Eq. F_reg with rho = e^{-beta H} split in four
 * quarters, estimated with random states (Eq. q_typicality) by the chain
 *   phi = rho^{1/8} psi~,  a0 = rho^{1/4} chi_j phi,
 *   p = chi_i U(t) phi,  q = chi_i U(t) a0,  U(t) = e^{-iHt},
 *   F(t) = < rho^{1/4} U(t)^dag p | chi_j | rho^{1/4} U(t)^dag q >,
 * which equals <psi~| rho^{1/8} chi_i(t) rho^{1/4} chi_j rho^{1/4} chi_i(t)
 * rho^{1/4} chi_j rho^{1/8} |psi~> by cyclicity.  i != j.  Unnormalised:
 * F~(t) = F(t)/F(0).  Same argument conventions as syk_correlator_G;
 * F_re_im[(k*nstates + s)*2 + {0,1}] (host).  Synchronises `stream`. */
int syk_otoc(const syk_terms* terms, double beta, int i, int j, const double* t, int nt,
             const void* psi0, int64_t nstates, int dtype, int krylov_dim, double tol,
             double* F_re_im, void* stream);

/* syk_otoc_split -- the OTOC family with a general split of rho = e^{-beta H}
 * between the four operators (Supp. Sec. on unregularized OTOCs and on
 * regularizations: reducing the imaginary-time separation of the operators):
 *   F(t) = Tr[chi_i(t) rho^{x1} chi_j rho^{x2} chi_i(t) rho^{x3} chi_j rho^{x4}],
 * x[0..3] >= 0 summing to 1; x = 1/4 each is syk_otoc (Eq. F_reg), x = (0,0,0,1)
 * the unregularized OTOC <chi_i(t) chi_j chi_i(t) chi_j rho>.  One-state estimate
 * (Eq. q_typicality) by the chain phi = rho^{x4/2} psi~, a0 = rho^{x3} chi_j phi,
 * F = < rho^{x1} U^dag chi_i U phi | chi_j | rho^{x2} U^dag chi_i U a0 >.  Other
 * conventions as syk_otoc. */
int syk_otoc_split(const syk_terms* terms, double beta, const double* x, int i, int j, const double* t,
                   int nt, const void* psi0, int64_t nstates, int dtype, int krylov_dim, double tol,
                   double* F_re_im, void* stream);

/* syk_correlator_G_imag -- imaginary-time two-point function, Eq. G:
 * G(tau) = <chi_i(tau) chi_i(0)>_beta with chi(tau) = e^{tau H} chi e^{-tau H}, estimated
 * (Eq. q_typicality) as <psi~|e^{-beta H/2} chi_i(tau) chi_i e^{-beta H/2}|psi~> / Z,
 * Z = <psi~|e^{-beta H}|psi~>, for 0 <= tau (non-decreasing).  The factor
 * e^{(tau - beta/2) H} grows for tau > beta/2, so the estimate loses digits like
 * e^{(tau - beta/2) |E|}.  Conventions as syk_correlator_G. */
int syk_correlator_G_imag(const syk_terms* terms, double beta, int i, const double* tau, int ntau,
                          const void* psi0, int64_t nstates, int dtype, int krylov_dim, double tol,
                          double* G_re_im, double* Z, void* stream);

/* syk_otoc_batch -- the batched workload: many independent OTOC evaluations
 * (coupling draws of any N, each with its beta and its D x nstates random
 * states, device or host memory) at the common times t, Majoranas i, j, dtype
 * and Krylov settings.  complex64 items (three-term Lanczos recurrence) run
 * as ONE persistent kernel launch (a CUDA graph of the queue reset and the
 * kernel) when their states split into sub-items of Bs in {16, 8, 4, 2}
 * states (or one state for one-state items), Bs a divisor of nstates, whose
 * sector vectors of D x Bs values fit one CTA's shared memory (N <= 24 at 8
 * states per CTA, N = 28 at 2, N = 30 for one-state items; items split over
 * several CTAs only when the batch's split sub-items fill at least half the
 * SMs): each CTA takes sub-items from a device-side queue and evaluates their
 * entire chain -- Lanczos evolutions with FP64 scalars, tridiagonal
 * eigendecompositions, step control, Majoranas, dots -- with no host round
 * trip (syk_batch_persistent(0) turns this off).  The other items are taken,
 * largest first, by `nworkers` host threads, each with its own CUDA stream,
 * concurrently with that launch; every distinct (N, nstates) of theirs is
 * autotuned first.  Each item's F_re_im (host, nt x nstates x 2) is filled as
 * by syk_otoc; item_status (may be NULL) receives each item's return code.
 * Returns the first failure.  The paper averages over hundreds of such draws
 * (Supp. Sec. I.C). */
typedef struct {
  const syk_terms* terms;
  double beta;
  const void* psi0;
  int64_t nstates;
  double* F_re_im;
} syk_otoc_item;
int syk_otoc_batch(const syk_otoc_item* items, int nitems, int i, int j, const double* t, int nt,
                   int dtype, int krylov_dim, double tol, int nworkers, int* item_status);
/* syk_batch_persistent -- 1 (default): syk_otoc_batch runs the items that fit
 * its persistent launch there (items split over several CTAs only when there
 * are enough of them, see syk_otoc_batch); 2: split items always go there too;
 * 0: every item takes the per-item path.  Returns the previous mode.
 * Plumbing; no counterpart in the paper. */
int syk_batch_persistent(int on);
/* syk_batch_plan -- how syk_otoc_batch's persistent launch would take a complex64
 * item of N Majoranas with nstates states at Krylov dimension krylov_dim, given
 * smem_limit bytes of shared memory per CTA (<= 0: the current device's opt-in
 * limit): *states_per_cta = the states one CTA takes (a power of two <= 16 that
 * divides nstates; 1 only for one-state items), 0 when the item takes the
 * per-item path; *smem_per_cta (may be NULL) = that launch's shared memory per
 * CTA.  Host arithmetic only (no device needed when smem_limit > 0); whether a
 * split item actually goes to the persistent launch also depends on the batch
 * (see syk_otoc_batch).  Plumbing; no counterpart in the paper. */
int syk_batch_plan(int N, int64_t nstates, int krylov_dim, int smem_limit, int* states_per_cta,
                   int* smem_per_cta);
/* syk_batch_report -- counters of the last syk_otoc_batch call (host array of
 * n <= 12 words): items in the persistent launch, items on the per-item path,
 * CTAs of the persistent launch; summed over its sub-items (one CTA's share of
 * an item's states): SM clock cycles spent in matvecs, in convergence checks
 * (tridiagonal eigendecompositions and step selection), in the combination
 * coefficients of accepted bases (with their full eigendecomposition when no
 * check computed it) and in whole sub-items; H applications (states x
 * matvecs), convergence checks, separate full eigendecompositions; the
 * number of sub-items; and the matvecs' algorithmic flops (8 per nonzero of the
 * sector Hamiltonian per state).  Measurement; no counterpart in the paper. */
int syk_batch_report(long long* out, int n);

/* --------------------------------------------------------------- gradients
 * syk_otoc_grad -- F~(t) = F(t)/F(0) of syk_otoc at one time t for each state,
 * with its derivatives with respect to every coupling J_ijkl (Eq. 1) and beta.
 * The correlators are sesquilinear forms of chains of exponentials e^{zH} and
 * Majoranas; each exponential is differentiated with Duhamel's formula
 *   d e^{zH}/dJ_T = z int_0^1 e^{(1-v)zH} P_T e^{vzH} dv,  P_T = chi_i chi_j chi_k chi_l,
 * integrated with 4-point Gauss-Legendre on sub-intervals of |z| rho <= quad_dz
 * (rho = 3 sqrt(sum J^2/16), a scale of the spectral radius), with the forward
 * states checkpointed every ceil(sqrt(#sub-intervals)) and recomputed per segment;
 * <lam|P_T|psi> for all terms is one pass over the state per quadrature node.
 * d e^{-c beta H}/dbeta = -c H e^{-c beta H}.  The paper computes no gradients;
 * the correlators differentiated are its Eq. F_reg and Eq. G.
 * psi0: D x nstates, device or host memory (even sector).  Host outputs:
 * Ft_re_im[2*s..], dFt_dJ[(T*nstates + s)*2 + {0,1}] (C(N,4) x nstates complex),
 * dFt_dbeta[2*s..].  Synchronises `stream`. */
int syk_otoc_grad(const syk_terms* terms, double beta, int i, int j, double t, const void* psi0,
                  int64_t nstates, int dtype, int krylov_dim, double tol, double quad_dz,
                  double* Ft_re_im, double* dFt_dJ, double* dFt_dbeta, void* stream);
/* syk_correlator_G_grad -- G(t) of syk_correlator_G at one time t (normalised by
 * Z = <phi|phi>) per state, with dG/dJ_T and dG/dbeta; conventions as syk_otoc_grad. */
int syk_correlator_G_grad(const syk_terms* terms, double beta, int i, double t, const void* psi0,
                          int64_t nstates, int dtype, int krylov_dim, double tol, double quad_dz,
                          double* G_re_im, double* dG_dJ, double* dG_dbeta, void* stream);

/* syk_lowest_eigenvalues -- the k lowest eigenvalues of H in sector `parity`, for the
 * finite-size rescaling (Supp. Sec. "Finite-size rescaling method": only sizes whose lowest
 * 20 eigenstates lie within the thermal window of the ground state enter the extrapolation).
 * Lanczos from the start vector psi0 (D complex amplitudes of `dtype`, device or host
 * memory; a random state reaches every eigenvector with probability 1) with full two-pass
 * Gram-Schmidt reorthogonalisation, up to max_steps (<= SYK_MAX_EIG_STEPS) steps; every 16
 * steps the Ritz values of the tridiagonal projection are computed on the host (FP64) and
 * the run stops once the k lowest have residual bounds beta_j |y_i(j)| <= tol * max(1, |T|)
 * (|T|: the largest Ritz value in magnitude, at least 1).  Outputs (host): evals[k], the k
 * lowest DISTINCT levels ascending (Ritz values closer than 10 tol |T| are one level: SYK
 * levels are doubly degenerate within a sector for N = 4 mod 8, and rounding lets a single
 * start vector find both members of a pair), resid[k] (may be NULL) their residual bounds,
 * *nsteps (may be NULL) the Lanczos steps taken.  Returns SYK_ENUMERIC if the k levels have
 * not converged within max_steps (outputs filled as far as known) or the Krylov space of
 * psi0 holds fewer than k levels; synchronises `stream`.
 * Device scratch: (min(max_steps, D) + 2) vectors. */
#define SYK_MAX_EIG_STEPS 4096
int syk_lowest_eigenvalues(const syk_terms* terms, int parity, int dtype, const void* psi0, int k, int max_steps,
                           double tol, double* evals, double* resid, int* nsteps, void* stream);

/* ------------------------------------------------------------- autotuner
 * syk_autotune_apply -- times every tile configuration of the tiled matvec
 * (CTA width 64/128/256 threads x thread-block cluster of 1/2/4/8 CTAs sharing a
 * tile) for this term set's N, `dtype` and `batch` (1, 2, 4, 8 or 16) on
 * scratch vectors it allocates, with `reps` timed applies each, and records
 * the fastest; later syk_apply_H / syk_expmv calls with the same (N, dtype,
 * batch) use it.  *best_ms (may be NULL) receives its time per apply.
 * Synchronises `stream`.  The work of the batched workload has no counterpart
 * in the paper; this only picks launch shapes. */
int syk_autotune_apply(const syk_terms* terms, int parity, int dtype, int64_t batch, int reps,
                       void* stream, double* best_ms);
/* syk_autotune_export / _import -- the tuned table as JSON
 * ({"apply_tiles": [{"N":..,"dtype":..,"batch":..,"ntb":..,"cluster":..,"variant":..,"ms":..}]};
 * variant 0 is the plain tiled kernel, 1..3 the complex64 coset kernel with 2^variant rows
 * per thread; a missing variant reads as 0),
 * so a tuning run can be cached in a file and reloaded. */
int syk_autotune_export(char* buf, size_t len);
int syk_autotune_import(const char* json);
/* syk_autotune_reset -- forgets every tuned entry, so later launches use the built-in
 * launch-shape heuristic again.  Host only; returns 0. */
int syk_autotune_reset(void);

/* ------------------------------------------------------------- diagnostics
 * syk_last_error -- message of the last failed call on this thread ("" if none). */
const char* syk_last_error(void);

/* syk_fma_peak -- measured FMA throughput of the current device, the roofline of the
 * matvec (one complex multiply-add, 4 real FMA, per nonzero of H and state: FP32 for
 * SYK_C64, FP64 for SYK_C128).  The paper has no counterpart; this is measurement.  Runs
 * `iters` x 128 dependent FMA (8 independent chains) in each of 4 x 256 threads per SM,
 * timed with CUDA events on `stream` after one short warm-up launch.  bits: 32 or 64.
 * Outputs (host, any may be NULL): *tflops = 2 x FMA / time, *sms = the device's SM count
 * (cudaDevAttrMultiProcessorCount), *ms = the timed launch.  Synchronises `stream`. */
int syk_fma_peak(int bits, int iters, double* tflops, int* sms, double* ms, void* stream);

/* syk_counters -- counters since the last reset (any pointer may be NULL):
 * H applications per state (a batch of B states counts B), Krylov bases, and
 * kernel launches made by the library.  reset != 0 zeroes them after reading. */
int syk_counters(int64_t* h_applies, int64_t* krylov_bases, int64_t* launches, int reset);

/* syk_matvec_launches -- matvec launches since the last reset by kernel family (any
 * pointer may be NULL): the row kernel (small sectors, other batch sizes, unaligned
 * vectors), the tiled kernel and the complex64 coset kernel.  A Lanczos segment replayed
 * from a captured graph adds the launches it recorded.  reset != 0 zeroes them. */
int syk_matvec_launches(int64_t* rows, int64_t* tiled, int64_t* coset, int reset);

/* syk_profile_enable / syk_profile_read -- CUDA-event timing of every apply_H
 * launch the library makes (on the stream it is launched on).  While enabled,
 * each launch is bracketed by two events; elapsed times are accumulated when
 * the library next synchronises (or in syk_profile_read, which synchronises
 * the device).  Reading returns launches and total milliseconds; reset != 0
 * zeroes them. */
int syk_profile_enable(int on);
/* syk_use_graphs -- how the Krylov evolutions are launched.  0: every kernel directly, with
 * one host read per convergence check.  1 (default): the same, but the Lanczos iterations
 * between two convergence checks are replayed as captured CUDA graphs (per host thread, per
 * workspace; rebuilt after term sets are freed or tile shapes retuned).  2: each evolution of a
 * correlator chain (syk_correlator_G, syk_otoc, syk_otoc_split, syk_correlator_G_imag, the
 * batch) is one launch of a graph that runs the whole Krylov loop with its step control on the
 * device (conditional WHILE and IF nodes): the chain is enqueued without host
 * synchronisation, with bit-identical results; the graph is built once per workspace, term
 * set and sector, which costs more than it saves for a chain run only once (syk_expmv and
 * the gradients stay host-driven).  Graphs are not used while profiling is enabled. */
int syk_use_graphs(int on);
int syk_profile_read(int64_t* launches, double* total_ms, int reset);

#ifdef __cplusplus
}
#endif
#endif /* SYK_H */

/*
 * ppl_cpd.h -- matrix-free CP-ALS of the DF particle-particle-ladder (PPL) tensor
 * on one NVIDIA GB300 (sm_103a).  C ABI of libpplcpd.so.
 *
 * The method (Pierce, "Towards Using Matrix-Free Tensor Decompositions to
 * Systematically Improve Approximate Tensor-Networks"):
 *
 *   R[a,b,i,j] = sum_{Q,c,d} B[Q,a,c] B[Q,b,d] tau[i,j,c,d]          Eq. (dfB), D-bar = D
 *   R~[a,b,i,j] = sum_r lam[r] Ua[a,r] Ub[b,r] Ui[i,r] Uj[j,r]        Eq. (cp-ppl)
 *
 * R is never formed.  Each ALS sweep updates Ua, Ub, Ui, Uj in that order
 * (Optimizing the CP-PPL tensor-network section): a matrix-free MTTKRP
 * (Eqs. full_der, distribute, foreachr), the Hadamard product V of the other
 * three Gram matrices, a Cholesky solve U~ = M V^-1, and a column
 * normalisation into lam.  The fit follows Eq. (cpfit) with the residual
 * expansion and Eq. (cp_norm2).
 *
 * Conventions for every call below:
 *  - Tensor arguments are DEVICE pointers, allocated and owned by the caller;
 *    the library never frees them and keeps using B and tau until
 *    ppl_cpd_destroy (or ppl_cpd_set_tau for tau).  All arrays are dense,
 *    row-major, FP64.
 *  - `stream` is a cudaStream_t passed as void*; all device work of a handle
 *    is issued on it.  Calls that return host scalars synchronise that stream.
 *  - Every call returns a PPL_* status; on error, ppl_last_error(h) (or
 *    ppl_last_error(NULL) before a handle exists) gives a message.  No call
 *    aborts the process.  A non-positive-definite V is not an error: its
 *    clamped pivots are counted (ppl_cpd_stats).
 *  - The library allocates no device memory: everything it needs lives in
 *    the caller's workspace (ppl_cpd_workspace_size, then ppl_cpd_init).
 */
#ifndef PPL_CPD_H
#define PPL_CPD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PPL_OK        0
#define PPL_EINVAL    1   /* bad argument (NULL pointer, size out of range)          */
#define PPL_ENOMEM    2   /* workspace smaller than ppl_cpd_workspace_size          */
#define PPL_ECUDA     3   /* a CUDA runtime call failed                             */
#define PPL_ETIMEOUT  4   /* a bounded device wait expired; the kernel returned     */
#define PPL_ENOTREADY 5   /* fit asked for before ||R||^2 or before any sweep       */

/* arithmetic of the MTTKRP contractions; Gram, solve, fit and energy are FP64 always */
#define PPL_PREC_FP64   0  /* plain FP64 on the CUDA cores                                 */
#define PPL_PREC_BF16X3 1  /* tcgen05 BF16 hi/lo split, hi*hi + hi*lo + lo*hi, FP32 accum. */
#define PPL_PREC_TF32   2  /* tcgen05 TF32 (round-to-nearest operands), FP32 accumulate    */
#define PPL_PREC_TF32X3 3  /* tcgen05 TF32 hi/lo split (22 bits), three products, FP32
                              accumulate restarted every acc_chunk K blocks and summed
                              with round-to-nearest                                        */

/* initial guess of ppl_cpd_init (the Role of the Initial Guess section: a random start) */
#define PPL_INIT_USER    0  /* the factors buffer holds the caller's guess                     */
#define PPL_INIT_NORMAL  1  /* U_a, U_b, U_i, U_j filled on the device with N(0, 1) numbers     */
#define PPL_INIT_UNIFORM 2  /* the same with uniform numbers in [0, 1)                          */

#define PPL_MODE_A 0  /* alpha, first virtual index  */
#define PPL_MODE_B 1  /* beta, second virtual index  */
#define PPL_MODE_I 2  /* gamma, first occupied index  */
#define PPL_MODE_J 3  /* rho, second occupied index   */

typedef struct ppl_cpd ppl_cpd;   /* opaque handle, host memory owned by the library */

typedef struct {
    int precision;   /* PPL_PREC_*                                                       */
    int r_chunk;     /* columns of r per pass of the chain (workspace grows with it), at most
                        1024; 0 = automatic: equal chunks of at most 256 columns in FP64,
                        on the tensor cores as wide as keeps one [rc][X][v] operand
                        buffer within 8 GiB                                              */
    int use_graph;   /* 1: capture one sweep in a CUDA graph on first use and replay it  */
    int want_eta;    /* 1: also compute eta, Eqs. (N3_stopping)/(new_conv), each sweep    */
    int profile;     /* 1: record CUDA events between the phases of every sweep           */
    int dressed;     /* 1: reserve room for the t1-dressed D-bar (ppl_cpd_set_t1)         */
    int acc_chunk;   /* K blocks (64 bf16 / 32 tf32 columns) summed in one tensor-core
                        accumulator before the epilogue adds it to FP32 registers with
                        round-to-nearest; 0 = the precision's default (TF32X3: 1,
                        otherwise no restart), -1 = never restart                       */
    int acc_steps;   /* > 0 (1..3): restart it every acc_steps MMA K steps (16 bf16 / 8
                        tf32 columns) inside each K block instead: less round-toward-
                        zero bias, more round-to-nearest additions, slower; 0 or -1 =
                        off (the default)                                                */
    int wait_limit_us; /* > 0: every bounded device wait of this handle's kernels (grid
                        barriers of the solve, tensor-core pipeline barriers) gives up
                        after this many microseconds; 0 = 1 s for the solve, 0.5 s for
                        the pipeline.  On expiry the kernel records the error, drains
                        what it issued and returns; the call reports PPL_ETIMEOUT.     */
    int acc_steps_p; /* as acc_steps, for the contractions of the S-build (W_b, S, P, and
                        W_a, which it then forms itself instead of taking the mode-b
                        chain's), whose result M_j sets lam and so the energy; 0 = as
                        acc_steps                                                       */
    int init;        /* PPL_INIT_*: with NORMAL or UNIFORM, ppl_cpd_init overwrites the
                        factors buffer: element e of U_a, U_b, U_i, U_j (in that order,
                        each [dim][R] row-major, e counted over all four) is, from the
                        counter-based splitmix64 generator (Steele, Lea & Flood 2014) with
                        key = mix(init_seed ^ 4 * 0xD1B54A32D192ED03) and uniforms
                        u_k = (mix(key + (k + 1) * 0x9E3779B97F4A7C15) >> 11) * 2^-53,
                        NORMAL: sqrt(-2 log1p(-u_2e)) cos(2 pi u_2e+1) (Box-Muller),
                        UNIFORM: u_e.  The same numbers as the seeded synthetic inputs'
                        initial factors (up to the last bits of log1p and cos).         */
    int init_seed;   /* seed of the NORMAL / UNIFORM guess (taken as unsigned)          */
    int reserved[4];
} ppl_cpd_opts;

typedef struct {
    long long sweeps;          /* sweeps run since init                                   */
    long long clamped_pivots;  /* Cholesky pivots replaced by the tolerance, all solves   */
    long long timeouts;        /* bounded device waits that expired                       */
    double    last_fit;        /* fit after the last sweep (NaN if ||R||^2 unknown)       */
    double    last_eta;        /* eta after the last sweep (NaN unless want_eta)          */
    double    last_inner;      /* <R, R~> after the last sweep                            */
    double    last_norm2;      /* ||R~||^2 after the last sweep, Eq. (cp_norm2)           */
    double    flops_per_sweep; /* algorithmic MTTKRP flops per sweep, 4 o^2 v^2 R + 16 X v^2 R */
    long long kernels_per_sweep; /* kernel nodes in the captured sweep graph (0 before capture) */
} ppl_cpd_stats;

/* Fill *opts with defaults: TF32X3, automatic r_chunk, graphs on, eta off. */
void ppl_cpd_default_opts(ppl_cpd_opts* opts);

/* Bytes of device workspace a handle with these sizes and options needs.
 * o, v, X, R >= 1.  Pure host arithmetic (no CUDA call).  EINVAL on bad sizes. */
int ppl_cpd_workspace_size(int o, int v, int X, int R, const ppl_cpd_opts* opts, size_t* bytes);

/* Create a handle.
 *   B        [X][o+v][o+v]  DF factor D^{pX}_q (Eq. SQG), occupied orbitals first,
 *                           symmetric in p, q (only the symmetric problem is defined).
 *   tau      [o][o][v][v]   tau[i,j,c,d] = t2 + t1 t1 (Eq. B); pair symmetry is not required.
 *   factors  Ua[v*R] | Ub[v*R] | Ui[o*R] | Uj[o*R] | lam[R], each [dim][R] row-major.
 *            In: the initial guess (lam is ignored and set to 1).  The handle
 *            updates this buffer in place; after a call returns it holds the
 *            current model with unit-norm columns and the scales in lam.
 *   workspace, ws_bytes: device memory of at least ppl_cpd_workspace_size bytes,
 *            256-byte aligned; owned by the caller, used until ppl_cpd_destroy.
 *   opts     NULL for defaults.
 * The tensor-core operand copies of tau and B (BF16X3, TF32 or TF32X3) are
 * made here (device work on `stream`). */
int ppl_cpd_init(ppl_cpd** h, int o, int v, int X, int R,
                 const double* B, const double* tau, double* factors,
                 void* workspace, size_t ws_bytes, const ppl_cpd_opts* opts, void* stream);

/* MTTKRP of the current factors for one mode, M_out [dim][R] FP64 device
 * (dim = v for modes a, b and o for i, j).  Eq. (full_der) numerator:
 *   M_a[a,r] = sum_{b,i,j} R[a,b,i,j] Ub[b,r] Ui[i,r] Uj[j,r], and likewise.
 * The factors are not changed. */
int ppl_cpd_mttkrp(ppl_cpd* h, int mode, double* M_out);

/* Run nsweeps ALS sweeps (a, b, i, j).  fit_hist (HOST, may be NULL) receives
 * the fit after each sweep, or NaN where ||R||^2 is not known. */
int ppl_cpd_sweep(ppl_cpd* h, int nsweeps, double* fit_hist);

/* Supply ||R||^2 for the fit (Eq. cpfit) without ppl_exact_contract. */
int ppl_cpd_set_normR2(ppl_cpd* h, double normR2);

/* Fit after the last sweep: 1 - sqrt(max(0, ||R||^2 - 2<R,R~> + ||R~||^2)) / ||R||.
 * ENOTREADY if ||R||^2 is unknown or no sweep has run. */
int ppl_cpd_fit(ppl_cpd* h, double* fit);

/* CP estimate of the PPL energy, E = sum R~[a,b,i,j] (2 g[iajb] - g[ibja]) with
 * g[iajb] = sum_Q B[Q,i,a] B[Q,j,b], computed without forming R~:
 *   E = sum_r lam_r sum_Q [2 A_Q(Ui,Ua) A_Q(Uj,Ub) - A_Q(Ui,Ub) A_Q(Uj,Ua)],
 *   A_Q(x,y)_r = sum_{i,a} B[Q,i,a] x[i,r] y[a,r].                    (FP64) */
int ppl_cpd_energy(ppl_cpd* h, double* E_cp);

/* Exact contraction of Eq. (dfB), blocked over a: returns ||R||^2 and
 * E_exact = sum R[a,b,i,j] (2 g[iajb] - g[ibja]) (host scalars, either may be
 * NULL) and, if R_out != NULL, R itself as [v][v][o][o] (device).  Stores
 * ||R||^2 in the handle for ppl_cpd_fit.  Cost 2 X v^4 + 2 o^2 v^4 flops, FP64. */
int ppl_exact_contract(ppl_cpd* h, double* normR2, double* E_exact, double* R_out);

/* The same exact contraction on the tensor cores, in the handle's precision
 * (BF16X3, TF32 or TF32X3; EINVAL for FP64 handles): per a, G_a[b][(c,d)] =
 * sum_Q B[Q,a,c] D-bar[Q,b,d] and R[a] = G_a tau^T with FP32 accumulation,
 * split-K sums and the ||R||^2 / energy reductions in FP64.  Relative error of
 * the order of the precision's unit roundoff (1e-5 for BF16X3); use
 * ppl_exact_contract where FP64 accuracy matters and the size allows it. */
int ppl_exact_contract_mixed(ppl_cpd* h, double* normR2, double* E_exact, double* R_out);

/* The CP model in canonical form, R~[a,b,i,j] = sum_r lam_r Ua[a,r] Ub[b,r] Ui[i,r] Uj[j,r],
 * written to R_out [v][v][o][o] (FP64, device); with symmetrise != 0 it is
 * replaced by 0.5 (R~[a,b,i,j] + R~[b,a,j,i]), the post-reconstruction
 * symmetrisation of the CPD-PPL section.  2 v^2 o^2 R flops, FP64. */
int ppl_cpd_reconstruct(ppl_cpd* h, double* R_out, int symmetrise);

/* Use the t1-dressed D-bar of Eq. fulldfB on the b side of the PPL tensor,
 *   D-bar[Q,b,d] = B[Q,b,d] - 2 sum_k B[Q,b,k] t1[k,d]  (k occupied, b, d virtual),
 *   R[a,b,i,j]  = sum_{Q,c,d} B[Q,a,c] D-bar[Q,b,d] tau[i,j,c,d].
 * t1 [o][v] FP64 device (t1[i][a] = t^a_i); NULL restores D-bar = B.  Needs
 * opts.dressed = 1 at ppl_cpd_init (EINVAL otherwise).  The stored ||R||^2 is
 * forgotten.  Energies keep g from the undressed B. */
int ppl_cpd_set_t1(ppl_cpd* h, const double* t1);

/* Point the handle at a new tau (same shape, device) for the next CC-like
 * step; the factors in the caller's buffer are kept as the warm start
 * (the paper's "Optimal guess", Role of the Initial Guess section).  The
 * stored ||R||^2 is forgotten. */
int ppl_cpd_set_tau(ppl_cpd* h, const double* tau);

/* Device time of the phases of the last sweep, in ms (needs opts.profile = 1):
 *   ms[0] tau^{cd}_r (Khatri-Rao build + T contraction)   ms[1] MTTKRP chain, mode a
 *   ms[2] solve a    ms[3] MTTKRP chain, mode b    ms[4] solve b
 *   ms[5] S and P contractions (modes i, j)    ms[6] solves i and j    ms[7] fit terms
 * ENOTREADY if profiling is off or no sweep has run. */
int ppl_cpd_phase_ms(ppl_cpd* h, double* ms);

/* ---- stopping rules and initial guesses (Low cost CPD stopping condition and
 *      Role of the Initial Guess sections) ------------------------------------------- */
#define PPL_STOP_FIXED 0   /* exactly max_sweeps sweeps                                          */
#define PPL_STOP_DFIT  1   /* after sweep n >= 2: |fit_n - fit_{n-1}| < eps (Eq. canon); needs ||R||^2 */
#define PPL_STOP_ETA   2   /* after sweep n >= 1: eta_n < eps (Eq. N3_stopping); needs want_eta    */

#define PPL_GUESS_OPTIMAL      0  /* start each solve from the current factors (default)          */
#define PPL_GUESS_NEAR_OPTIMAL 1  /* cache the iterate n-5 of a solve that needed n > 5 sweeps and
                                     start every later solve from the cache                       */
#define PPL_GUESS_RANDOM       2  /* start every solve from the guess given to ppl_cpd_init       */

/* Choose how ppl_cpd_solve starts its second and later solves.  The first
 * solve always starts from the factors in the caller's buffer.  While no
 * Near-Optimal cache exists yet, the guess given to ppl_cpd_init is used. */
int ppl_cpd_set_guess_policy(ppl_cpd* h, int policy);

/* One CPD: ALS sweeps until stop_rule fires or max_sweeps is reached.
 * sweeps_done (host, may be NULL) receives n; fit_hist / eta_hist (host,
 * [max_sweeps] each, may be NULL) the per-sweep fit (NaN if ||R||^2 unknown)
 * and eta (NaN unless want_eta).  EINVAL for PPL_STOP_ETA without want_eta,
 * ENOTREADY for PPL_STOP_DFIT without ||R||^2. */
int ppl_cpd_solve(ppl_cpd* h, int max_sweeps, int stop_rule, double eps, int* sweeps_done,
                  double* fit_hist, double* eta_hist);

/* The caller has written a new guess into its factor buffer (the layout of
 * ppl_cpd_init): recompute the Gram matrices the solves use and reset lam to 1. */
int ppl_cpd_factors_changed(ppl_cpd* h);

/* ---- autotuning and batches of uneven instances ----------------------------------- */

/* Time the MTTKRP chain of this handle for candidate r-chunk sizes (multiples of
 * 16 up to the size its workspace was planned for) and keep the fastest for all
 * later sweeps.  r_chunk_out (host, may be NULL) receives the choice.  Call it
 * before the first sweep (a captured sweep graph is discarded). */
int ppl_cpd_autotune(ppl_cpd* h, int* r_chunk_out);

typedef struct ppl_cpd_batch ppl_cpd_batch;   /* opaque, host memory owned by the library */

/* Group n handles (each from ppl_cpd_init with its own workspace; sizes and
 * options may differ, and only contractions of the same kernel are grouped) so that one sweep of
 * every instance runs from a single CUDA graph, forked from and joined back to
 * `stream`: every instance is captured on its own internal stream, then the
 * instances' tensor-core contractions of equal depth in their chains run as
 * grouped persistent launches (up to 40 contractions each), and each mode's
 * solves of all instances (at most 64 per launch) as one cooperative launch
 * whose blocks form lanes that solve their instances in turn (the Role of the
 * Initial Guess section motivates many CPDs per CC iteration; the grouping has
 * no counterpart in the paper).  nstreams >= 1 sets the share of the SMs, about
 * 4/nstreams, that a contraction left out of a group may use (reset by
 * ppl_cpd_batch_destroy).  The handles stay owned by the caller and must
 * outlive the batch. */
int ppl_cpd_batch_create(ppl_cpd_batch** b, int n, ppl_cpd* const* handles, int nstreams, void* stream);

/* nsweeps sweeps of every instance; fits (HOST, may be NULL) receives
 * [nsweeps][n] fit values (NaN where ||R||^2 is unknown). */
int ppl_cpd_batch_sweep(ppl_cpd_batch* b, int nsweeps, double* fits);

/* Kernel nodes in the batch's captured sweep graph (0 before the first sweep). */
int ppl_cpd_batch_kernels(ppl_cpd_batch* b, long long* kernels_per_sweep);

int ppl_cpd_batch_destroy(ppl_cpd_batch* b);

/* Counters and the last sweep's scalars. */
int ppl_cpd_stats_get(ppl_cpd* h, ppl_cpd_stats* stats);

/* Message for the last failed call on h (h may be NULL: errors of init / size
 * queries).  The string belongs to the library. */
const char* ppl_last_error(const ppl_cpd* h);

/* Release the handle (host memory and any captured graph).  The caller then
 * frees its workspace, B, tau and factors.  h may be NULL. */
int ppl_cpd_destroy(ppl_cpd* h);

/* ---- allocation-free variant ----------------------------------------------------
 * ppl_cp_energy_static: the CP energy of ppl_cpd_energy (same formula, FP64)
 * for callers that cannot allocate device memory at the point of the call:
 * code running inside a framework whose device memory is owned by its own
 * pooling allocator and that has no way to hand a workspace through, or
 * latency-bound code that must not call cudaMalloc / cudaFree (both can
 * synchronise the whole device) in the middle of a solve.  The paper has no
 * counterpart; this is a convenience of the library.
 *
 * Inputs are the same device arrays as ppl_cpd_init takes: B [X][o+v][o+v]
 * and the factor buffer Ua | Ub | Ui | Uj | lam.  E_cp is a HOST double;
 * the call synchronises `stream`.  Scratch is one array of
 * PPL_STATIC_SCRATCH_BYTES in the library's device image, which every GPU
 * that loads the library holds until the process exits; it requires
 * 2 * o * R * 8 + 8448 <= PPL_STATIC_SCRATCH_BYTES (o * R <= 523760) and
 * returns PPL_EINVAL otherwise.  The first call on a device (and the first
 * call in a new context of it, e.g. after cudaDeviceReset) looks up the
 * array's device address (cudaGetSymbolAddress), so make that first call
 * before any stream capture; a failed call forgets the address.  A launch
 * error left pending by earlier work is cleared on entry, not reported.  All calls share the one array and it keeps the
 * previous call's contents (the call clears what it accumulates into): calls
 * that overlap on the GPU, from several streams or threads, race. */
#define PPL_STATIC_SCRATCH_BYTES (8u << 20)
int ppl_cp_energy_static(int o, int v, int X, int R, const double* B, const double* factors,
                         double* E_cp, void* stream);

/* Test of the bounded device waits (no counterpart in the paper): arms a one-
 * shot flag in the handle's device memory so that, in the next mode update,
 * one block of the cooperative solve does not arrive at its first grid
 * barrier.  The other blocks' wait then runs out (after opts.wait_limit_us,
 * or 1 s), every block returns, and the sweep reports PPL_ETIMEOUT and counts
 * it in ppl_cpd_stats.timeouts.  Nothing faults or hangs and the handle stays
 * usable; the factors are left mid-update, so reset them
 * (ppl_cpd_factors_changed) before further sweeps.  Works under graph replay. */
int ppl_cpd_inject_wait_timeout(ppl_cpd* h);

/* Measured FP64 FMA throughput of the current device (no counterpart in the
 * paper; the peak of the FP64 roofline the benchmark reports the solves
 * against): independent FMA chains on every SM, eight blocks of 256 threads
 * per SM, best of three launches of about 50 ms timed with CUDA events on
 * `stream`.  Writes TFLOP/s (2 flops per FMA) to the host double *tflops.
 * Allocates nothing (its sink is a static device variable). */
int ppl_probe_fp64_peak(double* tflops, void* stream);

/* Self-test of the reciprocal the Cholesky uses for its pivots (no counterpart
 * in the paper): out[i] = the solve kernel's 1/d[i] for n positive normal
 * doubles d (device arrays), computed with the same device function.  The call
 * synchronises `stream`.  PPL_EINVAL for NULL arrays or n < 0. */
int ppl_test_reciprocal(const double* d, double* out, int n, void* stream);

/* Building-block check of the tensor-core contraction used by the MTTKRP:
 * C[M][N] = A[M][K] . B[N][K]^T for FP32 device inputs, computed with the
 * given PPL_PREC_BF16X3, PPL_PREC_TF32 or PPL_PREC_TF32X3 tcgen05 kernel
 * (operands split or rounded on the device, FP32 accumulate; TF32X3 restarts
 * the accumulator every K block as a handle does by default) and written to
 * C (FP32 device, [M][N]).  workspace must hold ppl_tc_gemm_workspace_size bytes. */
int ppl_tc_gemm_workspace_size(int M, int N, int K, int precision, size_t* bytes);
int ppl_tc_gemm(int precision, int M, int N, int K, const float* A, const float* B, float* C,
                void* workspace, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PPL_CPD_H */

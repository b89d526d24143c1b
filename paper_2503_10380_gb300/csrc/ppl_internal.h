// Internal interfaces shared by the translation units of libpplcpd.so.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

// Index map i -> (i / div) * hi + (i % div) * lo.  With div >= 2^30 it is a
// plain stride.  Lets one strided kernel read the flattened compound indices
// of the method ((Q,c), (c,d), (i,j), ...) straight out of B and tau.
struct Idx2 {
    long long hi, lo;
    int div;
};
static inline Idx2 ix1(long long stride) { return Idx2{0, stride, 1 << 30}; }
static inline Idx2 ix2(int div, long long hi, long long lo) { return Idx2{hi, lo, div}; }

// C[b][m][n] = alpha * sum_k A[b][m][k] * B[b][n][k] (+ beta * C), FP64.
struct G64 {
    const double* A; Idx2 am, ak; long long ab;
    const double* B; Idx2 bn, bk; long long bb;
    double* C; Idx2 cm, cn; long long cb;
    int M, N, K, batch, ksplit;
    double alpha, beta;
    int atomic;   // 1: atomicAdd(alpha * acc) into C (split-K); beta ignored
    int lower;    // 1: skip tiles whose columns all lie above the diagonal (n > m)
};
void gemm64(const G64& g, cudaStream_t s);

// ---- small FP64 kernels (ppl_fp64.cu) -------------------------------------
// KR[r][i*o+j] = Ui[i][r] * Uj[j][r]   (FP64, [R][ld])
void kr_build_f64(const double* Ui, const double* Uj, int o, int R, double* KR, int ld, cudaStream_t s);
// V = G1 .* G2 .* G3 (R x R); tol[0] = max(2^-52 R max_k V_kk, 1e-300)
void hadamard3(const double* G1, const double* G2, const double* G3, int R, double* V, double* tol, cudaStream_t s);
// One mode update in one cooperative launch (ppl_solve.cu): V = G1.G2.G3, clamped
// Cholesky, U~ = M V^-1, U = U~ / lam, G = U^T U.  Workspace: V [R][R], Linv
// [ceil(R/32)][32][32] (per diagonal block L[i][j] / L[j][j] below the diagonal and
// 1 / L[i][i] on it), Z [dim][R]; sync (4 words) and maxdiag are reset here.
// grid_cap > 0 limits the cooperative grid (so that several solves can share the GPU).
// wait_ns > 0 bounds every barrier wait (default 1 s); *withhold != 0 makes one
// block skip its first barrier arrival once (the test of the bounded waits).
int solve_mode_coop(const double* G1, const double* G2, const double* G3, const double* M, int dim, int R,
                    double* V, double* Linv, double* Z, double* U, double* lam, double* G,
                    unsigned int* sync, unsigned long long* maxdiag, unsigned long long* nclamp, unsigned int* err,
                    int grid_cap, unsigned long long wait_ns, unsigned int* withhold, cudaStream_t s);
// The same mode update for several instances in one cooperative launch (at most
// 64 per launch; more are launched in turn on s): instance k gets its own blocks
// and barrier words (a[k].sync); the blocks are shared out by FP64 work.
struct SolveArgs {
    const double *G1, *G2, *G3, *M;
    int dim, R;
    double *V, *Linv, *Z, *U, *lam, *G;
    unsigned int* sync;
    unsigned long long *maxdiag, *nclamp;
    unsigned int* err;
    unsigned long long wait_ns;
    unsigned int* withhold;
};
int solve_modes_batched(const SolveArgs* a, int n, cudaStream_t s);
// U = Ut / lam (column 2-norms); zero column keeps lam = 0
void normalise_cols(const double* Ut, int dim, int R, double* U, double* lam, cudaStream_t s);
// out[0] = sum_{x,r} M[x][r] * Ut[x][r] (Ut = U * lam),  out[1] = lam^T (Ga.Gb.Gi.Gj) lam
void fit_terms(const double* M, const double* U, const double* lam, int dim, int R,
               const double* Ga, const double* Gb, const double* Gi, const double* Gj,
               double* partial, double* out, cudaStream_t s);
// hist[0..3] = {fit, inner, norm2, eta}; fit from terms[0], terms[1], *normR2 (NaN if *normR2 <= 0)
void finish_fit(const double* terms, const double* normR2, double* hist, cudaStream_t s);
// eta from norm2_new, norm2_old and the cross term lam1^T (prod_m X_m) lam0
void eta_terms(const double* X0, const double* X1, const double* X2, const double* X3,
               const double* lam1, const double* lam0, int R, double* partial, double* out, cudaStream_t s);
void finish_eta(const double* cross, const double* norm2_new, const double* norm2_old, double* hist, cudaStream_t s);
// M_i[i][r] = sum_j P[r][i*o+j] Uj[j][r]  (which = 0);  M_j[j][r] = sum_i P[r][i*o+j] Ui[i][r] (which = 1)
void occ_mttkrp(const double* P, int ldP, const double* U, int o, int R, int which, double* M, cudaStream_t s);
// energy: out = sum_r lam_r sum_Q [2 A(i,a) A(j,b) - A(i,b) A(j,a)], A from Z_a/Z_b [X][o][R]
void energy_reduce(const double* Za, const double* Zb, const double* Ui, const double* Uj,
                   const double* lam, int X, int o, int R, double* partial, double* out, cudaStream_t s);
// g[i][a][j][b] buffer is built with gemm64; this reduces R-block [ab][v][o][o] against it
void exact_reduce(const double* Rblk, int a0, int na, int v, int o, const double* g,
                  double* partial, double* acc, cudaStream_t s);
void sum_partials(const double* partial, int n, double* out, int accumulate, cudaStream_t s);
// out[(p*d2 + q)][r'] = U1[p][r0+r'] U2[q][r0+r'] (lam[r0+r'] if lam), r' < rc; out row stride rc
void kr_pair(const double* U1, const double* U2, const double* lam, int d1, int d2, int R, int r0, int rc,
             double* out, cudaStream_t s);
// X[a][b][i][j] <- 0.5 (X[a][b][i][j] + X[b][a][j][i]) in place
void symmetrise_pairs(double* X, int v, int o, cudaStream_t s);
void fill_f64(double* p, size_t n, double val, cudaStream_t s);
// f[e], e < n: N(0,1) (normal = 1, Box-Muller) or U[0,1) numbers of the counter-
// based splitmix64 stream (seed, stream_id); see ppl_cpd_opts.init
void fill_random(double* f, long long n, int normal, unsigned int seed, int stream_id, cudaStream_t s);
// out[Q][b][d] = B[Q][o+b][o+d]
void extract_vv(const double* B, int o, int v, int X, double* out, cudaStream_t s);

// ---- tensor-core path (ppl_tc.cu) ------------------------------------------
// Operands of the tcgen05 GEMM are K-major: rows of K contiguous elements.
// BF16X3 keeps two planes (hi, lo) of bf16, TF32X3 two planes of fp32 holding
// tf32 values, TF32 one plane of fp32 (already rounded to tf32).  A "plane"
// below is the hi plane; lo = hi + plane_elems.
struct TcMat {
    void* ptr;              // hi plane (bf16) or fp32 plane
    long long plane_elems;  // distance to the lo plane in elements (BF16X3)
    int rows, cols;         // cols = K extent; rows = M or N extent
    int batch;              // 3rd dimension
    long long ld;           // row stride in elements (multiple of 8); panel layout: rows allocated per panel
    long long bstride;      // batch stride in elements (multiple of 8)
    int panel;              // 1: K-panel layout, element (b, row, k) at
                            //    b*bstride + (k / KE)*(ld*KE) + row*KE + k % KE, KE = one 128-byte row
                            //    (32 fp32 or 64 bf16); a panel's elements past K must be zero
};
// Epilogue: element (m, n) of batch b, split-K slice ks goes to
//   out + b*sb + ks*sk + rowoff(m) + coloff(n), where with PW the elements of one
//   128-byte row of the operand precision (32 fp32 or 64 bf16; the K-panel width)
//   rowoff(m) = (q1 / PW)*q1p + (q1 % PW)*q1s + (q0 / PW)*q0p + (q0 % PW)*q0s,
//               q1 = m / mdiv, q0 = m % mdiv (mdiv <= 0: q1 = 0, q0 = m)
//   coloff(n) = (n / PW)*np + (n % PW)*ns
// so that a plain stride s is (PW*s, s) and a K-panel index is (panel stride, 1).
enum TcEpi { EPI_SPLIT = 0, EPI_F32 = 1, EPI_ATOMIC_F64 = 2, EPI_ATOMIC_F32 = 3 };
struct TcOut {
    int kind;               // TcEpi; EPI_SPLIT writes operand planes of the same precision
    void* out; long long plane_elems;
    long long sb, sk;       // batch stride; split-K slice stride (EPI_F32 partials)
    int mdiv;
    long long q1p, q1s, q0p, q0s, np, ns;
    float alpha;
};
struct TcGemm {
    int prec;               // PPL_PREC_BF16X3 or PPL_PREC_TF32
    TcMat A, B;             // A: [batch][M][K], B: [batch][N][K]
    int M, N, K, batch;
    int a_row0, b_row0;     // row offsets into A and B
    int a_b0, b_b0;         // batch offsets; a_bstep / b_bstep: 0 broadcasts one batch entry
    int a_bstep, b_bstep;
    int ksplit;             // split-K factor (atomic epilogues only)
    int bn;                 // N tile (multiple of 16, <= 256); 0 = automatic
    int kchunk;             // > 0: restart the accumulator every kchunk K blocks, sum chunks in registers
    int ksub;               // > 0: restart it every ksub MMA K steps inside each K block instead
    int nfast;              // 1: tile order N-fastest, so that the N tiles of one A row block run together
    int grid_cap;           // > 0: at most this many persistent CTAs (several contractions can share the GPU)
    unsigned long long wait_ns;   // > 0: bound of every pipeline barrier wait (default 0.5 s)
    TcOut out;
};
int tc_gemm(const TcGemm& g, unsigned int* err_flag, cudaStream_t s);
// out[m * ldo + n] = sum_k part[k][n][m] (FP64 sum of FP32 split-K partials, deterministic)
void reduce_partials(const float* part, int ksplit, int M, int N, double* out, long long ldo, cudaStream_t s);
// dst[b][j][i] = src[b][i][j], i, j < n, operand planes of the given precision
void transpose_operand(int prec, const void* src, void* dst, long long plane_elems, int n, long long ld,
                       long long bstride, int batch, cudaStream_t s);
int tc_init_driver();   // resolves cuTensorMapEncodeTiled; returns 0 on success
// Several independent contractions in one persistent launch.  A captured launch
// of tc_gemm is a kernel node whose kernelParams[0] is its argument block; the
// grouped kernel walks the tiles of up to tc_group_capacity() such contractions.
// tc_group_kernel: the grouped counterpart of a single-contraction kernel (nullptr
// if f is not one).  tc_group_node_params: the kernel-node parameters of one
// grouped launch of the n argument blocks args (all of kernel f); *storage holds
// them until tc_group_release, after the node is created.  Returns 0 on success.
const void* tc_group_kernel(const void* f);
int tc_group_capacity();
int tc_group_node_params(const void* f, const void* const* args, int n, cudaKernelNodeParams* out, void** storage);
void tc_group_release(void* storage);
// FP64 -> operand planes: dst[b][r][c] from src with generic index maps, rows x cols per batch
struct SplitSrc {
    const double* src; Idx2 rmap, cmap; long long bstride;
    const float* src32;    // alternative FP32 source (for ppl_tc_gemm)
};
void split_to_operand(int prec, const SplitSrc& s, int rows, int cols, int batch,
                      void* dst, long long plane_elems, long long ld, long long bstride, cudaStream_t st);
// The same into the K-panel layout dst[b][c / KE][r][c % KE] (prow rows allocated
// per panel, npan = ceil(cols / KE) panels per batch entry, bstride = npan*prow*KE);
// every element of the panels that is not a valid (r < rows, c < cols, and
// c % kdiv < kmod when kdiv > 0) source element is written as zero.
void split_to_panels(int prec, const SplitSrc& s, int rows, int prow, int cols, int kdiv, int kmod, int batch,
                     void* dst, long long plane_elems, cudaStream_t st);
// Per-batch transpose between K-panel layouts: src[b][k / KE][a][k % KE] = X_b[a][k]
// (A rows, B columns, A rows per panel) to dst[b][a / KE][k][a % KE] (B rows per
// panel); plane_* elements from the hi to the lo plane, bstride_* elements per b.
void transpose_panels(int prec, const void* src, void* dst, long long plane_s, long long plane_d, int A, int B,
                      long long bstride_s, long long bstride_d, int batch, cudaStream_t s);
// elements of one 128-byte operand row (the K-panel width) of a precision
int panel_width(int prec);
void zero_bytes(void* p, size_t n, cudaStream_t s);

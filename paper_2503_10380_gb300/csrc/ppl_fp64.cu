// FP64 kernels of the CP-ALS sweep: the strided GEMM used by the plain FP64
// form, and the Gram / Hadamard / Cholesky / triangular-solve / normalise /
// fit / energy steps that run in FP64 in every precision mode.
#include "ppl_internal.h"

#include "../../include/ppl_cpd.h"

#include <cmath>
#include <cstdio>

namespace {

constexpr int GBM = 64, GBN = 64, GBK = 16;

__device__ __forceinline__ long long ixd(const Idx2& x, int i) {
    return (long long)(i / x.div) * x.hi + (long long)(i % x.div) * x.lo;
}

// 64x64 output tile per CTA, 256 threads, 4x4 outputs per thread at
// (ty + 16 i, tx + 16 j).  Operands are read through Idx2 maps, so every
// layout of the method is served without copies; the FP64 pipe (not the
// loads) bounds this kernel on GB300.
__global__ void __launch_bounds__(256) k_gemm64(G64 g) {
    const int b = blockIdx.z / g.ksplit, ks = blockIdx.z % g.ksplit;
    const int m0 = blockIdx.x * GBM, n0 = blockIdx.y * GBN;
    if (g.lower && n0 > m0 + GBM - 1) return;
    const int per = (((g.K + g.ksplit - 1) / g.ksplit) + GBK - 1) / GBK * GBK;
    const int kbeg = ks * per, kend = min(g.K, kbeg + per);
    if (kbeg >= kend && g.atomic) return;

    __shared__ double As[GBK][GBM];
    __shared__ double Bs[GBK][GBN];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const double* A = g.A + (long long)b * g.ab;
    const double* B = g.B + (long long)b * g.bb;
    const bool a_kfast = (g.ak.lo == 1 && g.ak.div >= (1 << 30));
    const bool b_kfast = (g.bk.lo == 1 && g.bk.div >= (1 << 30));

    // per-thread load coordinates: 4 elements of each 64x16 tile
    int a_ml[4], a_kl[4], b_nl[4], b_kl[4];
    long long a_row[4], b_row[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int e = tid + 256 * q;
        a_ml[q] = a_kfast ? e / GBK : e % GBM;
        a_kl[q] = a_kfast ? e % GBK : e / GBM;
        b_nl[q] = b_kfast ? e / GBK : e % GBN;
        b_kl[q] = b_kfast ? e % GBK : e / GBN;
        const int m = m0 + a_ml[q], n = n0 + b_nl[q];
        a_row[q] = (m < g.M) ? ixd(g.am, m) : -1;
        b_row[q] = (n < g.N) ? ixd(g.bn, n) : -1;
    }

    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    for (int k0 = kbeg; k0 < kend; k0 += GBK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int ka = k0 + a_kl[q], kb = k0 + b_kl[q];
            As[a_kl[q]][a_ml[q]] = (a_row[q] >= 0 && ka < kend) ? A[a_row[q] + ixd(g.ak, ka)] : 0.0;
            Bs[b_kl[q]][b_nl[q]] = (b_row[q] >= 0 && kb < kend) ? B[b_row[q] + ixd(g.bk, kb)] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }

    double* C = g.C + (long long)b * g.cb;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= g.M) continue;
        const long long cr = ixd(g.cm, m);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n >= g.N) continue;
            double* p = C + cr + ixd(g.cn, n);
            if (g.atomic) {
                atomicAdd(p, g.alpha * acc[i][j]);
            } else {
                const double old = (g.beta != 0.0) ? g.beta * *p : 0.0;
                *p = fma(g.alpha, acc[i][j], old);
            }
        }
    }
}

__global__ void k_kr(const double* Ui, const double* Uj, int o, int R, double* KR, int ld) {
    const long long total = (long long)R * o * o;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int ij = (int)(e % (o * o));
        const int r = (int)(e / (o * o));
        const int i = ij / o, j = ij % o;
        KR[(long long)r * ld + ij] = Ui[(long long)i * R + r] * Uj[(long long)j * R + r];
    }
}

__global__ void k_hadamard3(const double* G1, const double* G2, const double* G3, int R, double* V) {
    const long long total = (long long)R * R;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x)
        V[e] = G1[e] * G2[e] * G3[e];
}

__global__ void k_diag_tol(const double* V, int R, double* tol) {
    __shared__ double red[256];
    double m = 0.0;
    for (int i = threadIdx.x; i < R; i += blockDim.x) m = fmax(m, V[(long long)i * R + i]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) tol[0] = fmax(ldexp(1.0, -52) * (double)R * red[0], 1e-300);
}

__global__ void k_normalise(const double* Ut, int dim, int R, double* U, double* lam) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double s = 0.0;
    for (int x = 0; x < dim; ++x) {
        const double u = Ut[(long long)x * R + r];
        s = fma(u, u, s);
    }
    const double l = sqrt(s);
    const double inv = (l > 0.0) ? 1.0 / l : 1.0;
    for (int x = 0; x < dim; ++x) U[(long long)x * R + r] = Ut[(long long)x * R + r] * inv;
    lam[r] = l;
}

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x / 32, l = threadIdx.x % 32;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    v = (threadIdx.x < NT / 32) ? red[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;  // valid in thread 0
}

constexpr int RB = 256;      // threads per reduction block
// Blocks of the two-stage FP64 reductions (fit, eta, energy, exact contraction):
// a fixed width, 2 x the 152 SMs of GB300, not a device query, so that the sums
// are formed in the same order on every device (deterministic results) and the
// workspace's partial-sum buffer (2 values per block) is sized by the host-side
// planner, which runs without a device.
constexpr int RGRID = 304;

__global__ void __launch_bounds__(RB) k_fit_terms(const double* M, const double* U, const double* lam, int dim, int R,
                                                  const double* Ga, const double* Gb, const double* Gi,
                                                  const double* Gj, double* partial) {
    __shared__ double red[32];
    double s_in = 0.0, s_n2 = 0.0;
    const long long nIn = (long long)dim * R, nN2 = (long long)R * R;
    for (long long e = blockIdx.x * (long long)RB + threadIdx.x; e < nIn; e += (long long)gridDim.x * RB) {
        const int r = (int)(e % R);
        s_in = fma(M[e] * U[e], lam[r], s_in);
    }
    for (long long e = blockIdx.x * (long long)RB + threadIdx.x; e < nN2; e += (long long)gridDim.x * RB) {
        const int r = (int)(e / R), q = (int)(e % R);
        s_n2 = fma(lam[r] * lam[q], Ga[e] * Gb[e] * Gi[e] * Gj[e], s_n2);
    }
    s_in = block_sum<RB>(s_in, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s_in;
    s_n2 = block_sum<RB>(s_n2, red);
    if (threadIdx.x == 0) partial[gridDim.x + blockIdx.x] = s_n2;
}

__global__ void __launch_bounds__(RB) k_sum_partials(const double* partial, int n, int nvec, double* out, int accumulate) {
    __shared__ double red[32];
    for (int q = 0; q < nvec; ++q) {
        double s = 0.0;
        for (int e = threadIdx.x; e < n; e += RB) s += partial[q * n + e];
        s = block_sum<RB>(s, red);
        if (threadIdx.x == 0) out[q] = accumulate ? out[q] + s : s;
        __syncthreads();
    }
}

__global__ void k_finish_fit(const double* terms, const double* normR2p, double* hist) {
    const double inner = terms[0], norm2 = terms[1], normR2 = normR2p[0];
    double fit = nan("");
    if (normR2 > 0.0) fit = 1.0 - sqrt(fmax(normR2 - 2.0 * inner + norm2, 0.0)) / sqrt(normR2);
    hist[0] = fit;
    hist[1] = inner;
    hist[2] = norm2;
    hist[3] = nan("");
}

__global__ void __launch_bounds__(RB) k_eta_terms(const double* X0, const double* X1, const double* X2, const double* X3,
                                                  const double* lam1, const double* lam0, int R, double* partial) {
    __shared__ double red[32];
    double s = 0.0;
    const long long n = (long long)R * R;
    for (long long e = blockIdx.x * (long long)RB + threadIdx.x; e < n; e += (long long)gridDim.x * RB) {
        const int r = (int)(e / R), q = (int)(e % R);
        s = fma(lam1[r] * lam0[q], X0[e] * X1[e] * X2[e] * X3[e], s);
    }
    s = block_sum<RB>(s, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_finish_eta(const double* cross, const double* n_new, const double* n_old, double* hist) {
    const double num2 = n_new[0] - 2.0 * cross[0] + n_old[0];
    hist[3] = sqrt(fmax(num2, 0.0)) / sqrt(n_old[0]);
}

__global__ void k_occ_mttkrp(const double* P, int ldP, const double* U, int o, int R, int which, double* M) {
    const long long total = (long long)o * R;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(e / R), r = (int)(e % R);
        double s = 0.0;
        for (int y = 0; y < o; ++y) {
            const int ij = which == 0 ? x * o + y : y * o + x;
            s = fma(P[(long long)ij * ldP + r], U[(long long)y * R + r], s);
        }
        M[e] = s;
    }
}

__global__ void __launch_bounds__(RB) k_energy(const double* Za, const double* Zb, const double* Ui, const double* Uj,
                                               const double* lam, int X, int o, int R, double* partial) {
    __shared__ double red[32];
    double s = 0.0;
    const long long total = (long long)X * R;
    for (long long e = blockIdx.x * (long long)RB + threadIdx.x; e < total; e += (long long)gridDim.x * RB) {
        const int Q = (int)(e / R), r = (int)(e % R);
        const double* za = Za + (long long)Q * o * R + r;
        const double* zb = Zb + (long long)Q * o * R + r;
        double ia = 0, jb = 0, ib = 0, ja = 0;
        for (int x = 0; x < o; ++x) {
            const double ui = Ui[(long long)x * R + r], uj = Uj[(long long)x * R + r];
            const double a = za[(long long)x * R], bb = zb[(long long)x * R];
            ia = fma(ui, a, ia);
            jb = fma(uj, bb, jb);
            ib = fma(ui, bb, ib);
            ja = fma(uj, a, ja);
        }
        s = fma(lam[r], 2.0 * ia * jb - ib * ja, s);
    }
    s = block_sum<RB>(s, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// R block rows a in [a0, a0+na): Rblk[al][b][i][j]; g[i][a][j][b]
__global__ void __launch_bounds__(RB) k_exact_reduce(const double* Rblk, int a0, int na, int v, int o, const double* g,
                                                     double* partial) {
    __shared__ double red[32];
    double s2 = 0.0, sE = 0.0;
    const long long total = (long long)na * v * o * o;
    const long long ov = (long long)o * v;
    for (long long e = blockIdx.x * (long long)RB + threadIdx.x; e < total; e += (long long)gridDim.x * RB) {
        const int j = (int)(e % o);
        const int i = (int)((e / o) % o);
        const int b = (int)((e / ((long long)o * o)) % v);
        const int a = a0 + (int)(e / ((long long)o * o * v));
        const double r = Rblk[e];
        const double giajb = g[((long long)i * v + a) * ov + (long long)j * v + b];
        const double gibja = g[((long long)i * v + b) * ov + (long long)j * v + a];
        s2 = fma(r, r, s2);
        sE = fma(r, 2.0 * giajb - gibja, sE);
    }
    s2 = block_sum<RB>(s2, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s2;
    sE = block_sum<RB>(sE, red);
    if (threadIdx.x == 0) partial[gridDim.x + blockIdx.x] = sE;
}

__global__ void k_kr_pair(const double* U1, const double* U2, const double* lam, int d1, int d2, int R, int r0,
                          int rc, double* out) {
    const long long total = (long long)d1 * d2 * rc;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e % rc);
        const long long pq = e / rc;
        const int p = (int)(pq / d2), q = (int)(pq % d2);
        double x = U1[(long long)p * R + r0 + r] * U2[(long long)q * R + r0 + r];
        if (lam) x *= lam[r0 + r];
        out[e] = x;
    }
}

__global__ void k_symmetrise(double* X, int v, int o) {
    const long long oo = (long long)o * o, total = (long long)v * v * oo;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e % o), i = (int)((e / o) % o);
        const int b = (int)((e / oo) % v), a = (int)(e / (oo * v));
        const long long f = (((long long)b * v + a) * o + j) * o + i;
        if (e < f) {
            const double m = 0.5 * (X[e] + X[f]);
            X[e] = m;
            X[f] = m;
        }
    }
}

__global__ void k_extract_vv(const double* B, int o, int v, int X, double* out) {
    const int n = o + v;
    const long long total = (long long)X * v * v;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int d = (int)(e % v), b = (int)((e / v) % v);
        const long long Q = e / ((long long)v * v);
        out[e] = B[Q * n * n + (long long)(o + b) * n + o + d];
    }
}

__global__ void k_fill(double* p, size_t n, double val) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        p[e] = val;
}

inline int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

void gemm64(const G64& g, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
    dim3 grid((g.M + GBM - 1) / GBM, (g.N + GBN - 1) / GBN, g.batch * g.ksplit);
    if (g.K <= 0) {
        if (!g.atomic) {
            G64 z = g;  // C = beta * C: run with an empty K range
            k_gemm64<<<grid, 256, 0, s>>>(z);
        }
        return;
    }
    k_gemm64<<<grid, 256, 0, s>>>(g);
}

void kr_build_f64(const double* Ui, const double* Uj, int o, int R, double* KR, int ld, cudaStream_t s) {
    k_kr<<<grid_for((long long)R * o * o, 256), 256, 0, s>>>(Ui, Uj, o, R, KR, ld);
}

void hadamard3(const double* G1, const double* G2, const double* G3, int R, double* V, double* tol, cudaStream_t s) {
    k_hadamard3<<<grid_for((long long)R * R, 256), 256, 0, s>>>(G1, G2, G3, R, V);
    k_diag_tol<<<1, 256, 0, s>>>(V, R, tol);
}

void normalise_cols(const double* Ut, int dim, int R, double* U, double* lam, cudaStream_t s) {
    k_normalise<<<(R + 127) / 128, 128, 0, s>>>(Ut, dim, R, U, lam);
}

void fit_terms(const double* M, const double* U, const double* lam, int dim, int R,
               const double* Ga, const double* Gb, const double* Gi, const double* Gj,
               double* partial, double* out, cudaStream_t s) {
    k_fit_terms<<<RGRID, RB, 0, s>>>(M, U, lam, dim, R, Ga, Gb, Gi, Gj, partial);
    k_sum_partials<<<1, RB, 0, s>>>(partial, RGRID, 2, out, 0);
}

void finish_fit(const double* terms, const double* normR2, double* hist, cudaStream_t s) {
    k_finish_fit<<<1, 1, 0, s>>>(terms, normR2, hist);
}

void eta_terms(const double* X0, const double* X1, const double* X2, const double* X3,
               const double* lam1, const double* lam0, int R, double* partial, double* out, cudaStream_t s) {
    k_eta_terms<<<RGRID, RB, 0, s>>>(X0, X1, X2, X3, lam1, lam0, R, partial);
    k_sum_partials<<<1, RB, 0, s>>>(partial, RGRID, 1, out, 0);
}

void finish_eta(const double* cross, const double* n_new, const double* n_old, double* hist, cudaStream_t s) {
    k_finish_eta<<<1, 1, 0, s>>>(cross, n_new, n_old, hist);
}

void occ_mttkrp(const double* P, int ldP, const double* U, int o, int R, int which, double* M, cudaStream_t s) {
    k_occ_mttkrp<<<grid_for((long long)o * R, 256), 256, 0, s>>>(P, ldP, U, o, R, which, M);
}

void energy_reduce(const double* Za, const double* Zb, const double* Ui, const double* Uj,
                   const double* lam, int X, int o, int R, double* partial, double* out, cudaStream_t s) {
    k_energy<<<RGRID, RB, 0, s>>>(Za, Zb, Ui, Uj, lam, X, o, R, partial);
    k_sum_partials<<<1, RB, 0, s>>>(partial, RGRID, 1, out, 0);
}

void exact_reduce(const double* Rblk, int a0, int na, int v, int o, const double* g,
                  double* partial, double* acc, cudaStream_t s) {
    k_exact_reduce<<<RGRID, RB, 0, s>>>(Rblk, a0, na, v, o, g, partial);
    k_sum_partials<<<1, RB, 0, s>>>(partial, RGRID, 2, acc, 1);
}

void sum_partials(const double* partial, int n, double* out, int accumulate, cudaStream_t s) {
    k_sum_partials<<<1, RB, 0, s>>>(partial, n, 1, out, accumulate);
}

void kr_pair(const double* U1, const double* U2, const double* lam, int d1, int d2, int R, int r0, int rc,
             double* out, cudaStream_t s) {
    k_kr_pair<<<grid_for((long long)d1 * d2 * rc, 256), 256, 0, s>>>(U1, U2, lam, d1, d2, R, r0, rc, out);
}

void symmetrise_pairs(double* X, int v, int o, cudaStream_t s) {
    k_symmetrise<<<grid_for((long long)v * v * o * o, 256), 256, 0, s>>>(X, v, o);
}

void extract_vv(const double* B, int o, int v, int X, double* out, cudaStream_t s) {
    k_extract_vv<<<grid_for((long long)X * v * v, 256), 256, 0, s>>>(B, o, v, X, out);
}

void fill_f64(double* p, size_t n, double val, cudaStream_t s) {
    k_fill<<<grid_for((long long)n, 256), 256, 0, s>>>(p, n, val);
}

// ---- FP64 FMA throughput probe (measurement of the FP64 roofline's peak) ----

namespace {

constexpr int PROBE_CHAINS = 8;       // independent FMA chains per thread (covers the FMA latency)
constexpr int PROBE_ITERS = 12000;

__device__ double g_probe_sink;

__global__ void k_dfma_probe(double a, double b, int iters) {
    double x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
    if (s == 1234.5678) g_probe_sink = s;   // keeps the chains live; practically never taken
}

}  // namespace

extern "C" int ppl_probe_fp64_peak(double* tflops, void* stream) {
    if (!tflops) return PPL_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0) {
        cudaGetLastError();
        return PPL_ECUDA;
    }
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return PPL_ECUDA;
    }
    // a contraction factor below 1 keeps the chains finite and away from denormals
    const double a = 0.999999, b = 1e-6;
    k_dfma_probe<<<blocks, threads, 0, s>>>(a, b, PROBE_ITERS);   // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, s);
        k_dfma_probe<<<blocks, threads, 0, s>>>(a, b, PROBE_ITERS);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms > 0.0f && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return PPL_ECUDA;
    const double flops = 2.0 * PROBE_CHAINS * (double)PROBE_ITERS * blocks * threads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return PPL_OK;
}

// ---- seeded initial guess -----------------------------------------------------

namespace {

// splitmix64 finaliser (Steele, Lea & Flood, "Fast splittable pseudorandom
// number generators", OOPSLA 2014)
__host__ __device__ __forceinline__ unsigned long long sm64_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// uniform number i (0-based) of the counter stream with this key, in [0, 1)
__device__ __forceinline__ double sm64_u01(unsigned long long key, unsigned long long i) {
    const unsigned long long x = sm64_mix(key + (i + 1ull) * 0x9E3779B97F4A7C15ull);
    return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

__global__ void k_fill_random(double* f, long long n, int normal, unsigned long long key) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        if (normal) {
            // Box-Muller, cosine branch: normal e from uniforms 2e and 2e + 1
            const double u1 = sm64_u01(key, 2ull * (unsigned long long)e);
            const double u2 = sm64_u01(key, 2ull * (unsigned long long)e + 1ull);
            f[e] = sqrt(-2.0 * log1p(-u1)) * cos(6.283185307179586 * u2);
        } else {
            f[e] = sm64_u01(key, (unsigned long long)e);
        }
    }
}

}  // namespace

void fill_random(double* f, long long n, int normal, unsigned int seed, int stream_id, cudaStream_t s) {
    if (n <= 0) return;
    const unsigned long long key = sm64_mix((unsigned long long)seed ^ ((unsigned long long)stream_id * 0xD1B54A32D192ED03ull));
    long long g = (n + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    k_fill_random<<<(int)g, 256, 0, s>>>(f, n, normal, key);
}

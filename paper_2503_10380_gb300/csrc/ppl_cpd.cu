// libpplcpd: C ABI and the ALS sweep orchestration (host side).
//
// One sweep (Optimizing the CP-PPL tensor-network section; Gauss-Seidel
// order a, b, i, j, each update using the newest factors):
//   phase A  KR[ij,r] = Ui[i,r] Uj[j,r];  T[r,c,d] = sum_ij tau[ij,cd] KR[ij,r]   (tau^{cd}_r)
//            mode a:  per r-chunk  W = B.Ub  ->  Y_r = W_r T_r^T  ->  M_a += B . Y   (Eq. foreachr)
//                     solve: V = Gb.Gi.Gj, Cholesky, U~ = M V^-1, normalise, Ga = Ua^T Ua
//            mode b:  the same with Ua (new) and T transposed
//   phase B  per r-chunk  Wa = B.Ua, Wb = B.Ub, S_r = Wa_r^T Wb_r, P[ij,r] += sum_cd tau[ij,cd] S_r[cd]
//            modes i, j: M_i = sum_j P Uj, solve; M_j = sum_i P Ui (new), solve
//            fit terms: <R,R~> from M_j, ||R~||^2 from the four Gram matrices (Eq. cp_norm2)
// Only r-chunks of the X*v*R intermediates exist at any time.
#include "ppl_internal.h"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <algorithm>
#include <map>
#include <unordered_map>
#include <utility>
#include <vector>

#include "../../include/ppl_cpd.h"

namespace {

thread_local std::string g_err;

long long rup(long long x, long long m) { return (x + m - 1) / m * m; }

struct Layout {
    // offsets (bytes) into the workspace; -1 = absent
    size_t G[4], V, Linv, Z, M, P, scal, partial, hist, flags, KR64, Uold[4], lamold, Xc[4];
    size_t T64, W64, Y64, S64;                       // FP64 form
    size_t tauT, tauN, Bn, Bp, BpW, UopA, UopB, KRT, T, Tt, W, Y, WTa, WTb, S, PART;   // tensor-core form
    size_t Bbar, BbN, BbP, BbT;   // t1-dressed D-bar: FP64 [X][v][v] and its operand layouts
    size_t Bq, BbQ, Gop;          // tensor-core exact contraction: B and D-bar as [(p,q)][Q], G_a
    size_t Za, Zb, gov, Gblk, Rblk;
    size_t ring, cache, guess0;   // 6 iterates, the Near-Optimal cache, the initial guess
    size_t recon;                 // Khatri-Rao chunks for the reconstruction
    int rcr;
    size_t total;
    int rc, na;
    long long ldv, ldX, ldo2, ldvv;
    long long ldk;   // tensor-core form: v padded to the K-panel width (a K extent of v per block of a compound index)
    int ke;          // the K-panel width: elements of one 128-byte operand row
};

constexpr int NPART = 2 * 304 + 8;
constexpr int KSMAX = 80;   // most split-K slices of one tensor-core contraction
constexpr int RC_MAX = 1024; // most rank columns per pass of the chain
#ifndef TF32X3_ACC_STEPS
#define TF32X3_ACC_STEPS 0      // default MMA K steps per TF32X3 accumulation chunk (0: a K block)
#endif
#ifndef BATCH_TC_SHARE
#define BATCH_TC_SHARE 4        // a batched tensor-core contraction takes about SHARE / nstreams of the SMs (0: all)
#endif
#ifndef BATCH_GROUP_SETS
#define BATCH_GROUP_SETS 4      // grouped contraction launches per depth of a batch graph
#endif
#ifndef BATCH_SOLVE_SHARE
#define BATCH_SOLVE_SHARE 4     // a batched solve takes about SHARE / nstreams of the SMs
#endif
constexpr int NSCAL = 64;
// scalar slots
constexpr int SC_TERMS = 2, SC_NORMR2 = 8, SC_NORM2_PREV = 9, SC_CROSS = 10, SC_ENERGY = 12,
              SC_EXACT = 14;

bool plan(int o, int v, int X, int R, const ppl_cpd_opts& op, Layout& L) {
    if (o < 1 || v < 1 || X < 1 || R < 1) return false;
    if ((long long)o * o > (1 << 28) || (long long)v * v > (1 << 29) || (long long)X * v > (1 << 29) || R > (1 << 20))
        return false;
    const bool tc = op.precision != PPL_PREC_FP64;
    L.ldv = rup(v, 8);
    L.ldX = rup(X, 8);
    L.ldo2 = rup((long long)o * o, 8);
    L.ldvv = rup((long long)v * v, 8);
    // r-chunk: an explicit r_chunk up to RC_MAX; automatic = chunks of equal
    // size, each at most 256 columns in FP64 and, on the tensor cores, as many
    // as keep one chunk buffer ([rc][X][v] operand planes) within 8 GiB (each
    // pass of the chain reads the B operand copies once, so fewer passes move
    // fewer bytes)
    int rc;
    if (op.r_chunk > 0) {
        rc = op.r_chunk > RC_MAX ? RC_MAX : op.r_chunk;
    } else {
        long long cap = 256;
        if (tc) {
            const long long per_r = (long long)X * L.ldv * (op.precision == PPL_PREC_TF32X3 ? 8 : 4);
            cap = (8ll << 30) / per_r;
            if (cap > RC_MAX) cap = RC_MAX;
            if (cap < 16) cap = 16;
        }
        const long long nch = (R + cap - 1) / cap;
        rc = (int)((R + nch - 1) / nch);
    }
    if (tc) rc = (int)rup(rc, 16) > RC_MAX ? RC_MAX : (int)rup(rc, 16);
    if (rc > R) rc = R;
    L.rc = rc;
    const long long dim = v > o ? v : o;
    const long long v3 = (long long)v * v * v;
    long long na = 32ll * 1024 * 1024 / (v3 + (long long)v * o * o);
    if (na < 1) na = 1;
    if (na > v) na = v;
    L.na = (int)na;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off += (size_t)rup((long long)bytes, 256);
        return at;
    };
    const size_t d = sizeof(double);
    const size_t RR = (size_t)R * R;
    for (int m = 0; m < 4; ++m) L.G[m] = take(RR * d);
    L.V = take(RR * d);
    L.Linv = take((size_t)((R + 31) / 32) * 32 * 32 * d);
    L.Z = take((size_t)dim * R * d);
    L.M = take((size_t)dim * R * d);
    L.P = take((size_t)o * o * R * d);
    L.scal = take(NSCAL * d);
    L.partial = take(NPART * d);
    L.hist = take(4 * d);
    L.flags = take(64);
    L.KR64 = take((size_t)R * o * o * d);
    for (int m = 0; m < 4; ++m) L.Uold[m] = take((size_t)dim * R * d);
    L.lamold = take((size_t)R * d);
    for (int m = 0; m < 4; ++m) L.Xc[m] = take(RR * d);
    L.Za = take((size_t)X * o * R * d);
    L.Zb = take((size_t)X * o * R * d);
    L.gov = take((size_t)o * v * o * v * d);
    L.Gblk = take((size_t)na * v3 * d);
    L.Rblk = take((size_t)na * v * o * o * d);
    const size_t fsz = (size_t)(2 * v + 2 * o + 1) * R * d;
    L.ring = take(6 * fsz);
    L.cache = take(fsz);
    L.guess0 = take(fsz);
    L.rcr = R < 64 ? R : 64;
    L.recon = take((size_t)((long long)v * v + (long long)o * o) * L.rcr * d);
    const size_t none = (size_t)-1;
    L.T64 = L.W64 = L.Y64 = L.S64 = none;
    L.tauT = L.tauN = L.Bn = L.Bp = L.BpW = L.UopA = L.UopB = L.KRT = L.T = L.Tt = L.W = L.Y = L.WTa = L.WTb = L.S = none;
    L.ldk = 0;
    L.ke = 0;
    L.PART = none;
    L.Bbar = L.BbN = L.BbP = L.BbT = none;
    L.Bq = L.BbQ = L.Gop = none;
    if (op.dressed) L.Bbar = take((size_t)X * v * v * d);
    if (!tc) {
        L.T64 = take((size_t)R * v * v * d);
        L.W64 = take((size_t)rc * X * v * d);
        L.Y64 = take((size_t)rc * X * v * d);
        L.S64 = take((size_t)rc * v * v * d);
    } else {
        // operands in the K-panel layout (rows x K, K padded to the panel width ke)
        const size_t e = op.precision == PPL_PREC_TF32X3 ? 8 : 4;   // bf16 hi + lo, fp32 hi + lo, or one fp32
        const long long ke = op.precision == PPL_PREC_BF16X3 ? 64 : 32;
        L.ke = (int)ke;
        L.ldk = rup(v, ke);
        const long long ko2 = rup((long long)o * o, ke), kX = rup(X, ke), kvv = (long long)v * L.ldk;
        const size_t vv = (size_t)v * v, Xv = (size_t)X * v;
        L.tauT = take(vv * ko2 * e);                       // rows (c,d), K = (i,j)
        L.tauN = take((size_t)o * o * kvv * e);            // rows (i,j), K = (c, d) with d padded
        L.Bn = take(Xv * L.ldk * e);                       // rows (Q,d), K = b
        L.Bp = take((size_t)v * X * L.ldk * e);            // rows a, K = (Q, c) with c padded
        L.BpW = take(Xv * L.ldk * e);                      // rows (c,Q), K = a
        L.UopA = take((size_t)R * L.ldk * e);              // rows r, K = b
        L.UopB = take((size_t)R * L.ldk * e);
        L.KRT = take((size_t)R * ko2 * e);                 // rows r, K = (i,j)
        L.T = take((size_t)R * v * L.ldk * e);             // per r: rows c, K = d
        L.Tt = take((size_t)R * v * L.ldk * e);            // per r: rows d, K = c
        L.W = take((size_t)rc * X * L.ldk * e);            // per r: rows Q, K = d
        L.Y = take((size_t)rc * X * L.ldk * e);            // rows r, K = (Q, c)
        L.WTa = take((size_t)R * v * kX * e);              // per r: rows c, K = Q (every r: chain b fills it)
        L.WTb = take((size_t)rc * v * kX * e);
        L.S = take((size_t)rc * kvv * e);                  // rows r, K = (c, d)
        {
            const size_t chain_part = (size_t)KSMAX * (size_t)(v > o * o ? v : o * o) * rc;
            const size_t exact_part = (size_t)KSMAX * (size_t)v * o * o;
            L.PART = take((chain_part > exact_part ? chain_part : exact_part) * sizeof(float));
        }
        L.Bq = take(vv * kX * e);                          // rows (p,q), K = Q
        L.Gop = take((size_t)v * kvv * e);                 // rows b, K = (c, d)
        if (op.dressed) L.BbQ = take(vv * kX * e);
        if (op.dressed) {
            L.BbN = take(Xv * L.ldk * e);
            L.BbP = take((size_t)v * X * L.ldk * e);
            L.BbT = take(Xv * L.ldk * e);
        }
    }
    L.total = off;
    return true;
}

}  // namespace

struct ppl_cpd {
    int o, v, X, R, n;
    ppl_cpd_opts opts;
    cudaStream_t user;   // caller's stream
    cudaStream_t st;     // internal stream (capturable)
    cudaEvent_t ev_in, ev_out;
    const double* B;
    const double* tau;
    double* fac;
    double* U[4];
    double* lam;
    char* ws;
    size_t ws_bytes;
    Layout L;
    double normR2;
    bool have_normR2;
    long long sweeps;
    cudaGraph_t graph;
    cudaGraphExec_t gexec;
    bool graph_ready;
    double last_hist[4];
    std::string err;
    cudaEvent_t pev[9];
    bool have_pev;
    long long kernels_per_sweep;
    int guess_policy;
    int solve_cap;       // > 0: at most this many blocks per cooperative solve (set inside a batch)
    int tc_cap;          // > 0: at most this many CTAs per tensor-core contraction (set inside a batch)
    bool cache_valid;
    long long nsolves;
    long long ntimeouts;           // bounded device waits that expired (calls that returned PPL_ETIMEOUT)
    unsigned long long wait_ns;    // opts.wait_limit_us in ns (0: each kernel's default)
    size_t fac_bytes() const { return (size_t)(2 * v + 2 * o + 1) * R * sizeof(double); }

    template <class T>
    T* at(size_t off) const { return off == (size_t)-1 ? nullptr : reinterpret_cast<T*>(ws + off); }
    double* G(int m) const { return at<double>(L.G[m]); }
    double* scal() const { return at<double>(L.scal); }
    unsigned long long* nclamp() const { return at<unsigned long long>(L.flags); }
    unsigned int* errflag() const { return reinterpret_cast<unsigned int*>(ws + L.flags + 8); }
    unsigned int* withhold() const { return reinterpret_cast<unsigned int*>(ws + L.flags + 48); }
    int dim(int m) const { return m < 2 ? v : o; }
    bool tc() const { return opts.precision != PPL_PREC_FP64; }
    // bytes of one operand element over all its planes
    size_t opbytes() const { return opts.precision == PPL_PREC_TF32X3 ? 8 : 4; }
    // MMA K steps per accumulation chunk inside a K block (0: whole K blocks)
    int ksub() const {
        if (opts.acc_steps > 0) return opts.acc_steps;
        if (opts.acc_steps < 0) return 0;
        return opts.precision == PPL_PREC_TF32X3 ? TF32X3_ACC_STEPS : 0;
    }
    // the same for the S-build contractions (WT, S, P), whose result sets lam
    int ksub_p() const {
        if (opts.acc_steps_p > 0) return opts.acc_steps_p;
        if (opts.acc_steps_p < 0) return 0;
        return ksub();
    }
    bool in_p = false;   // run_tc: the contraction belongs to the S-build
    // K blocks per tensor-core accumulation chunk (0: one chunk per tile)
    int kchunk() const {
        if (opts.acc_chunk > 0) return opts.acc_chunk;
        if (opts.acc_chunk < 0) return 0;
        return opts.precision == PPL_PREC_TF32X3 ? 1 : 0;
    }
    bool dressed() const { return opts.dressed != 0; }
    // bytes of one element of one operand plane
    size_t plane_es() const { return opts.precision == PPL_PREC_BF16X3 ? 2 : 4; }
    // the S-build takes W_a from the mode-b chain of the same sweep, unless the
    // two are set to different accumulation restarts
    bool reuse_wa() const { return ksub_p() == ksub(); }
};

namespace {

int fail(ppl_cpd* h, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h)
        h->err = buf;
    else
        g_err = buf;
    return code;
}

int check_cuda(ppl_cpd* h, const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(h, PPL_ECUDA, "%s: %s", where, cudaGetErrorString(e));
    return PPL_OK;
}

// ---- tensor-core helpers ------------------------------------------------------

TcMat mat(void* p, long long plane, int rows, int cols, int batch, long long ld, long long bstride) {
    TcMat t{};
    t.ptr = p;
    t.plane_elems = plane;
    t.rows = rows;
    t.cols = cols;
    t.batch = batch;
    t.ld = ld;
    t.bstride = bstride;
    return t;
}

// an operand in the K-panel layout: rows x K, prow rows allocated per panel,
// batch entries bstride elements apart
TcMat pmat(void* p, long long plane, int rows, int cols, int batch, long long prow, long long bstride) {
    TcMat t = mat(p, plane, rows, cols, batch, prow, bstride);
    t.panel = 1;
    return t;
}

// one index of an output map: (panel stride, in-panel stride)
struct Ix {
    long long p, s;
};
// a plain stride s (the index is not the consumer's K)
Ix plain(long long s, int ke) { return Ix{ke * s, s}; }
// the consumer's K index inside its K panels, panels pstride elements apart
Ix kpan(long long pstride) { return Ix{pstride, 1}; }

// EPI_SPLIT output: element (m, n) of batch b at b*sb + map(m / mdiv, m % mdiv) + map(n)
TcOut out_map(void* p, long long plane, long long sb, int mdiv, Ix q1, Ix q0, Ix n) {
    TcOut o{};
    o.kind = EPI_SPLIT;
    o.out = p;
    o.plane_elems = plane;
    o.sb = sb;
    o.mdiv = mdiv;
    o.q1p = q1.p; o.q1s = q1.s;
    o.q0p = q0.p; o.q0s = q0.s;
    o.np = n.p; o.ns = n.s;
    o.alpha = 1.0f;
    return o;
}

int sm_count() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            sms <= 0) {
            cudaGetLastError();
            sms = 152;
        }
    }
    return sms;
}

// Split-K slices of a long contraction.  Each slice sums its K blocks in FP32
// registers (one restarted chunk per K block) and the slices are reduced in
// FP64, so a slice holds at most KB_PER_SLICE K blocks (the FP32 sum of a few
// hundred chunks, not thousands); among the counts that satisfy this, the
// smallest one whose work items (tiles x slices) fill whole waves of the SMs
// to >= 95% is taken.
constexpr int KB_PER_SLICE = 512;
int auto_ksplit(int M, int N, int bn, int K, int prec) {
    const int ke = prec == PPL_PREC_BF16X3 ? 64 : 32;
    const long long sms = sm_count();
    const long long tiles = (long long)((M + 127) / 128) * ((N + bn - 1) / bn);
    const long long nkb = (K + ke - 1) / ke;
    long long lo = (nkb + KB_PER_SLICE - 1) / KB_PER_SLICE;
    if (lo < 1) lo = 1;
    if (lo > KSMAX) lo = KSMAX;
    long long best = lo;
    if (tiles * lo < sms) {
        best = sms / tiles;                       // one wave, as many slices as fit
        if (best > KSMAX) best = KSMAX;
    } else {
        for (long long ks = lo; ks <= KSMAX; ++ks) {
            const long long items = tiles * ks, waves = (items + sms - 1) / sms;
            if ((double)items / (double)(waves * sms) >= 0.95) {
                best = ks;
                break;
            }
        }
    }
    if (best > nkb) best = nkb;
    if (best < 1) best = 1;
    return (int)best;
}

int bn_for(int N) {
    int tiles = (N + 255) / 256;
    int bn = (N + tiles - 1) / tiles;
    return (bn + 15) / 16 * 16;
}

int run_tc(ppl_cpd* h, TcGemm& g, const char* what) {
    g.prec = h->opts.precision;
    g.kchunk = h->kchunk();
    g.ksub = h->in_p ? h->ksub_p() : h->ksub();
    g.grid_cap = h->tc_cap;
    g.wait_ns = h->wait_ns;
    if (g.bn == 0) g.bn = bn_for(g.N);
    const int r = tc_gemm(g, h->errflag(), h->st);
    if (r != 0)
        return fail(h, PPL_ECUDA, "tensor-core GEMM (%s) failed to launch (%d%s%s)", what, r, r <= -1000 ? ": " : "",
                    r <= -1000 ? cudaGetErrorString((cudaError_t)(-r - 1000)) : "");
    return PPL_OK;
}

// ---- FP64 pieces shared by both precisions ------------------------------------

void gram(ppl_cpd* h, int m) {
    G64 g{};
    const int R = h->R;
    g.A = h->U[m]; g.am = ix1(1); g.ak = ix1(R);
    g.B = h->U[m]; g.bn = ix1(1); g.bk = ix1(R);
    g.C = h->G(m); g.cm = ix1(R); g.cn = ix1(1);
    g.M = R; g.N = R; g.K = h->dim(m); g.batch = 1; g.ksplit = 1; g.alpha = 1.0;
    gemm64(g, h->st);
}

// the arguments of mode m's update: V from the other three Gram matrices, M from L.M
SolveArgs solve_args(ppl_cpd* h, int m) {
    int oth[3], k = 0;
    for (int q = 0; q < 4; ++q)
        if (q != m) oth[k++] = q;
    char* f = h->ws + h->L.flags;
    SolveArgs a;
    a.G1 = h->G(oth[0]); a.G2 = h->G(oth[1]); a.G3 = h->G(oth[2]);
    a.M = h->at<double>(h->L.M);
    a.dim = h->dim(m); a.R = h->R;
    a.V = h->at<double>(h->L.V); a.Linv = h->at<double>(h->L.Linv); a.Z = h->at<double>(h->L.Z);
    a.U = h->U[m]; a.lam = h->lam; a.G = h->G(m);
    a.sync = reinterpret_cast<unsigned int*>(f + 16);
    a.maxdiag = reinterpret_cast<unsigned long long*>(f + 32);
    a.nclamp = h->nclamp(); a.err = h->errflag();
    a.wait_ns = h->wait_ns; a.withhold = h->withhold();
    return a;
}

// solve the normal equations of mode m from M (in L.M), update U[m], lam, G[m]
int solve_mode(ppl_cpd* h, int m) {
    const SolveArgs a = solve_args(h, m);
    const int r = solve_mode_coop(a.G1, a.G2, a.G3, a.M, a.dim, a.R, a.V, a.Linv, a.Z, a.U, a.lam, a.G, a.sync,
                                  a.maxdiag, a.nclamp, a.err, h->solve_cap, a.wait_ns, a.withhold, h->st);
    if (r != 0)
        return fail(h, PPL_ECUDA, "cooperative solve launch failed (%d%s%s)", r, r <= -1000 ? ": " : "",
                    r <= -1000 ? cudaGetErrorString((cudaError_t)(-r - 1000)) : "");
    return PPL_OK;
}

// ---- MTTKRP, FP64 form --------------------------------------------------------

void t_fp64(ppl_cpd* h) {
    const int o = h->o, v = h->v, R = h->R;
    double* KR = h->at<double>(h->L.KR64);
    kr_build_f64(h->U[2], h->U[3], o, R, KR, o * o, h->st);
    G64 g{};
    g.A = KR; g.am = ix1((long long)o * o); g.ak = ix1(1);
    g.B = h->tau; g.bn = ix1(1); g.bk = ix1((long long)v * v);
    g.C = h->at<double>(h->L.T64); g.cm = ix1((long long)v * v); g.cn = ix1(1);
    g.M = R; g.N = v * v; g.K = o * o; g.batch = 1; g.ksplit = 1; g.alpha = 1.0;
    gemm64(g, h->st);
}

// W[r][Q][d] = sum_b B[Q][o+b][o+d] U[b][r0+r]; bside: the dressed D-bar[Q][b][d]
void w_fp64(ppl_cpd* h, const double* U, int r0, int rcur, double* W, bool bside = false) {
    const int o = h->o, v = h->v, X = h->X, R = h->R, n = h->n;
    G64 g{};
    if (bside && h->dressed()) {
        g.A = h->at<double>(h->L.Bbar); g.am = ix2(v, (long long)v * v, 1); g.ak = ix1(v);
    } else {
        g.A = h->B + (long long)o * n + o; g.am = ix2(v, (long long)n * n, n); g.ak = ix1(1);
    }
    g.B = U + r0; g.bn = ix1(1); g.bk = ix1(R);
    g.C = W; g.cm = ix1(1); g.cn = ix1((long long)X * v);
    g.M = X * v; g.N = rcur; g.K = v; g.batch = 1; g.ksplit = 1; g.alpha = 1.0;
    gemm64(g, h->st);
}

void mttkrp_ab_fp64(ppl_cpd* h, int mode, double* Mout) {
    const int o = h->o, v = h->v, X = h->X, R = h->R, n = h->n, rc = h->L.rc;
    double* T = h->at<double>(h->L.T64);
    double* W = h->at<double>(h->L.W64);
    double* Y = h->at<double>(h->L.Y64);
    cudaMemsetAsync(Mout, 0, (size_t)v * R * sizeof(double), h->st);
    for (int r0 = 0; r0 < R; r0 += rc) {
        const int rcur = (R - r0 < rc) ? R - r0 : rc;
        w_fp64(h, mode == 0 ? h->U[1] : h->U[0], r0, rcur, W, mode == 0);
        G64 y{};
        y.A = W; y.ab = (long long)X * v; y.am = ix1(v); y.ak = ix1(1);
        y.B = T + (long long)r0 * v * v; y.bb = (long long)v * v;
        if (mode == 0) { y.bn = ix1(v); y.bk = ix1(1); }   // T[r][c][d], contract d
        else           { y.bn = ix1(1); y.bk = ix1(v); }   // T[r][c][d], contract c
        y.C = Y; y.cb = (long long)X * v; y.cm = ix1(v); y.cn = ix1(1);
        y.M = X; y.N = v; y.K = v; y.batch = rcur; y.ksplit = 1; y.alpha = 1.0;
        gemm64(y, h->st);
        G64 m{};
        if (mode == 1 && h->dressed()) {
            m.A = h->at<double>(h->L.Bbar); m.am = ix1(v); m.ak = ix2(v, (long long)v * v, 1);
        } else {
            m.A = h->B + (long long)o * n + o; m.am = ix1(n); m.ak = ix2(v, (long long)n * n, 1);
        }
        m.B = Y; m.bn = ix1((long long)X * v); m.bk = ix1(1);
        m.C = Mout + r0; m.cm = ix1(R); m.cn = ix1(1);
        m.M = v; m.N = rcur; m.K = X * v; m.batch = 1; m.alpha = 1.0; m.atomic = 1;
        const long long tiles = (long long)((v + 63) / 64) * ((rcur + 63) / 64);
        long long ks = (608 + tiles - 1) / tiles;
        if (ks > (X * (long long)v) / 64) ks = (X * (long long)v) / 64;
        m.ksplit = ks < 1 ? 1 : (int)ks;
        gemm64(m, h->st);
    }
}

void p_fp64(ppl_cpd* h) {
    const int o = h->o, v = h->v, X = h->X, R = h->R, rc = h->L.rc;
    double* Wa = h->at<double>(h->L.W64);
    double* Wb = h->at<double>(h->L.Y64);
    double* S = h->at<double>(h->L.S64);
    double* P = h->at<double>(h->L.P);
    cudaMemsetAsync(P, 0, (size_t)o * o * R * sizeof(double), h->st);
    for (int r0 = 0; r0 < R; r0 += rc) {
        const int rcur = (R - r0 < rc) ? R - r0 : rc;
        w_fp64(h, h->U[0], r0, rcur, Wa);
        w_fp64(h, h->U[1], r0, rcur, Wb, true);
        G64 s{};
        s.A = Wa; s.ab = (long long)X * v; s.am = ix1(1); s.ak = ix1(v);
        s.B = Wb; s.bb = (long long)X * v; s.bn = ix1(1); s.bk = ix1(v);
        s.C = S; s.cb = (long long)v * v; s.cm = ix1(v); s.cn = ix1(1);
        s.M = v; s.N = v; s.K = X; s.batch = rcur; s.ksplit = 1; s.alpha = 1.0;
        gemm64(s, h->st);
        G64 p{};
        p.A = h->tau; p.am = ix1((long long)v * v); p.ak = ix1(1);
        p.B = S; p.bn = ix1((long long)v * v); p.bk = ix1(1);
        p.C = P + r0; p.cm = ix1(R); p.cn = ix1(1);
        p.M = o * o; p.N = rcur; p.K = v * v; p.batch = 1; p.alpha = 1.0; p.atomic = 1;
        const long long tiles = (long long)((o * o + 63) / 64) * ((rcur + 63) / 64);
        long long ks = (608 + tiles - 1) / tiles;
        if (ks > (long long)v * v / 64) ks = (long long)v * v / 64;
        p.ksplit = ks < 1 ? 1 : (int)ks;
        gemm64(p, h->st);
    }
}

// ---- MTTKRP, tensor-core form ---------------------------------------------------

void* opb(ppl_cpd* h, size_t off) { return h->ws + off; }

// Operand layouts of the tensor-core form (elements per plane; ke = K-panel
// width, ldk = v padded to ke; a compound K index (Q, c) or (c, d) is
// Q * ldk + c, so that no panel straddles two blocks and the padding is zero):
//   tauT   rows (c,d)  K (i,j)         tauN  rows (i,j)  K (c, d)
//   Bn     rows (Q,d)  K b             Bp    rows a      K (Q, c)      BpW  rows (c,Q)  K a
//   Uop    rows r      K b             KRT   rows r      K (i,j)
//   T      per r: rows c, K d          Tt    per r: rows d, K c
//   W      per r: rows Q, K d          Y     rows r (rc per panel), K (Q, c)
//   WT     per r: rows c, K Q          S     rows r (rc per panel), K (c, d)
//   Bq     rows (p,q)  K Q             Gop   rows b      K (c, d)
struct Pan {
    long long ke, ldk, kX, ko2, kvv;
};
Pan pan_of(const ppl_cpd* h) {
    Pan q;
    q.ke = h->L.ke;
    q.ldk = h->L.ldk;
    q.kX = rup(h->X, q.ke);
    q.ko2 = rup((long long)h->o * h->o, q.ke);
    q.kvv = (long long)h->v * q.ldk;
    return q;
}

int uop(ppl_cpd* h, int m, size_t dst) {
    SplitSrc s{};
    s.src = h->U[m];
    s.rmap = ix1(1);
    s.cmap = ix1(h->R);
    const long long plane = (long long)h->R * h->L.ldk;
    split_to_panels(h->opts.precision, s, h->R, h->R, h->dim(m), 0, 0, 1, opb(h, dst), plane, h->st);
    return PPL_OK;
}

int t_tc(ppl_cpd* h) {
    const int o = h->o, v = h->v, R = h->R;
    const Pan q = pan_of(h);
    double* KR = h->at<double>(h->L.KR64);
    kr_build_f64(h->U[2], h->U[3], o, R, KR, o * o, h->st);
    SplitSrc s{};
    s.src = KR;
    s.rmap = ix1((long long)o * o);
    s.cmap = ix1(1);
    const long long pKRT = (long long)R * q.ko2;
    split_to_panels(h->opts.precision, s, R, R, o * o, 0, 0, 1, opb(h, h->L.KRT), pKRT, h->st);
    const long long bT = (long long)v * q.ldk;     // one r of T
    const long long pT = (long long)R * bT;
    TcGemm g{};
    g.A = pmat(opb(h, h->L.tauT), (long long)v * v * q.ko2, v * v, o * o, 1, (long long)v * v, 0);
    g.B = pmat(opb(h, h->L.KRT), pKRT, R, o * o, 1, R, 0);
    g.M = v * v; g.N = R; g.K = o * o; g.batch = 1; g.ksplit = 1;
    // T[r]: rows c, K d; m = c*v + d, n = r
    g.out = out_map(opb(h, h->L.T), pT, 0, v, plain(q.ke, q.ke), kpan((long long)v * q.ke), plain(bT, q.ke));
    int rc = run_tc(h, g, "T");
    if (rc) return rc;
    // T transposed per r: Tt[r] rows d, K c.  (A second copy written by the T
    // epilogue itself would be uncoalesced: consecutive rows d of a tile are a
    // panel row apart in Tt, and each 128-byte line of Tt takes one element
    // from each of 32 tiles; the transpose goes through shared memory instead.)
    transpose_panels(h->opts.precision, opb(h, h->L.T), opb(h, h->L.Tt), pT, pT, v, v, bT, bT, R, h->st);
    return PPL_OK;
}

// split-K contraction through FP32 partials [ks][n][m] in L.PART, then an FP64
// reduction into out[m * ldo + n]
int run_tc_partial(ppl_cpd* h, TcGemm& g, double* out, long long ldo, const char* what) {
    g.prec = h->opts.precision;
    if (g.bn == 0) g.bn = bn_for(g.N);
    g.ksplit = auto_ksplit(g.M, g.N, g.bn, g.K, g.prec);
    const int ke = g.prec == PPL_PREC_BF16X3 ? 64 : 32;
    const int nkb = (g.K + ke - 1) / ke;
    const int per = (nkb + g.ksplit - 1) / g.ksplit;
    const int ks = (nkb + per - 1) / per;      // the split count the kernel will use
    float* part = h->at<float>(h->L.PART);
    g.out = TcOut{};
    g.out.kind = EPI_F32;
    g.out.out = part;
    g.out.sk = (long long)g.M * g.N;
    g.out.q0p = ke; g.out.q0s = 1;
    g.out.np = (long long)ke * g.M; g.out.ns = g.M;
    g.out.alpha = 1.0f;
    int e = run_tc(h, g, what);
    if (e) return e;
    reduce_partials(part, ks, g.M, g.N, out, ldo, h->st);
    return PPL_OK;
}

// keep_wa (mode b only): also store W = B U_a of every r-chunk, transposed per r
// to rows c, K = Q, in L.WTa, where the S-build of the same sweep reads it
int chain_tc(ppl_cpd* h, int mode, double* Mout, bool keep_wa) {
    const int v = h->v, X = h->X, R = h->R, rc = h->L.rc;
    const Pan q = pan_of(h);
    const long long pBn = (long long)X * v * q.ldk;       // Bn / Bp plane
    const long long pU = (long long)R * q.ldk;
    const long long bT = (long long)v * q.ldk;
    const long long pT = (long long)R * bT;
    const long long bW = (long long)X * q.ldk;            // one r of W
    const long long pW = (long long)rc * bW;
    const int KY = (int)(X * q.ldk);                      // K of M = B . Y: (Q, c)
    uop(h, mode == 0 ? 1 : 0, h->L.UopA);
    for (int r0 = 0; r0 < R; r0 += rc) {
        const int rcur = (R - r0 < rc) ? R - r0 : rc;
        // W[r] rows Q, K d: W[r][Q][d] = sum_b B[Q][d][b] U[b][r0+r]
        TcGemm g1{};
        g1.A = pmat(opb(h, (mode == 0 && h->dressed()) ? h->L.BbN : h->L.Bn), pBn, X * v, v, 1, (long long)X * v, 0);
        g1.B = pmat(opb(h, h->L.UopA), pU, R, v, 1, R, 0);
        g1.M = X * v; g1.N = rcur; g1.K = v; g1.batch = 1; g1.ksplit = 1; g1.b_row0 = r0; g1.nfast = 1;
        g1.out = out_map(opb(h, h->L.W), pW, 0, v, plain(q.ke, q.ke), kpan((long long)X * q.ke), plain(bW, q.ke));
        int e = run_tc(h, g1, "W");
        if (e) return e;
        if (keep_wa) {
            // W[r][Q][c] (X rows per panel, K = c) -> WTa[r0 + r][c][Q] (v rows per panel, K = Q)
            const long long bWT = (long long)v * q.kX;
            transpose_panels(h->opts.precision, opb(h, h->L.W), opb(h, h->L.WTa + (size_t)r0 * bWT * h->plane_es()),
                             pW, (long long)R * bWT, X, v, bW, bWT, rcur, h->st);
        }
        // Y[r][Q][c] = sum_d T[r][c][d] W[r][Q][d]   (mode b: Tt, contracting c);
        // stored rows r, K (Q, c): m = c, n = Q, batch r
        TcGemm g2{};
        g2.A = pmat(opb(h, mode == 0 ? h->L.T : h->L.Tt), pT, v, v, R, v, bT);
        g2.a_b0 = r0; g2.a_bstep = 1;
        g2.B = pmat(opb(h, h->L.W), pW, X, v, rc, X, bW);
        g2.b_b0 = 0; g2.b_bstep = 1;
        g2.M = v; g2.N = X; g2.K = v; g2.batch = rcur; g2.ksplit = 1;
        g2.out = out_map(opb(h, h->L.Y), pW, q.ke, 0, Ix{0, 0}, kpan((long long)rc * q.ke),
                         plain(q.ldk * rc, q.ke));
        e = run_tc(h, g2, "Y");
        if (e) return e;
        // M[a][r0+r] += sum_{Q,c} B[Q][a][c] Y[r][Q][c]
        TcGemm g3{};
        g3.A = pmat(opb(h, (mode == 1 && h->dressed()) ? h->L.BbP : h->L.Bp), pBn, v, KY, 1, v, 0);
        g3.B = pmat(opb(h, h->L.Y), pW, rcur, KY, 1, rc, 0);
        g3.M = v; g3.N = rcur; g3.K = KY; g3.batch = 1;
        e = run_tc_partial(h, g3, Mout + r0, R, "M");
        if (e) return e;
    }
    return PPL_OK;
}

int p_tc_body(ppl_cpd* h, bool wa_ready);
int p_tc(ppl_cpd* h, bool wa_ready) {
    h->in_p = true;
    const int e = p_tc_body(h, wa_ready);
    h->in_p = false;
    return e;
}
// W_b = D-bar U_b is formed here per r-chunk.  W_a = B U_a is the W of the
// mode-b chain: with wa_ready the chain of the same sweep (same U_a) has left
// it in L.WTa, transposed to rows c, K = Q by a shared-memory transpose (a
// second layout written by the chain's own epilogue would be uncoalesced, one
// 4-byte L2 request per element); otherwise it is formed here too.
int p_tc_body(ppl_cpd* h, bool wa_ready) {
    const int o = h->o, v = h->v, X = h->X, R = h->R, rc = h->L.rc;
    const Pan q = pan_of(h);
    const long long pBn = (long long)X * v * q.ldk;
    const long long pU = (long long)R * q.ldk;
    const long long bWT = (long long)v * q.kX;            // one r of WT
    const long long pWT = (long long)rc * bWT;            // one chunk of WT
    const long long pWTa = (long long)R * bWT;            // WTa holds every r
    const long long pS = (long long)rc * q.kvv;
    double* P = h->at<double>(h->L.P);
    uop(h, 0, h->L.UopA);
    uop(h, 1, h->L.UopB);
    for (int r0 = 0; r0 < R; r0 += rc) {
        const int rcur = (R - r0 < rc) ? R - r0 : rc;
        for (int w = wa_ready ? 1 : 0; w < 2; ++w) {
            // WT[r] rows c, K Q: WT[r][c][Q] = sum_a B[Q][c][a] U[a][r0+r]; m = c*X + Q, n = r
            TcGemm g1{};
            g1.A = pmat(opb(h, (w == 1 && h->dressed()) ? h->L.BbT : h->L.BpW), pBn, v * X, v, 1, (long long)v * X, 0);
            g1.B = pmat(opb(h, w == 0 ? h->L.UopA : h->L.UopB), pU, R, v, 1, R, 0);
            g1.M = v * X; g1.N = rcur; g1.K = v; g1.batch = 1; g1.ksplit = 1; g1.b_row0 = r0; g1.nfast = 1;
            g1.out = out_map(w == 0 ? opb(h, h->L.WTa + (size_t)r0 * bWT * h->plane_es()) : opb(h, h->L.WTb),
                             w == 0 ? pWTa : pWT, 0, X, plain(q.ke, q.ke),
                             kpan((long long)v * q.ke), plain(bWT, q.ke));
            int e = run_tc(h, g1, "WT");
            if (e) return e;
        }
        // S[r][c][d] = sum_Q WTa[r][c][Q] WTb[r][d][Q]; stored rows r, K (c, d): m = d, n = c, batch r
        TcGemm gs{};
        gs.A = pmat(opb(h, h->L.WTb), pWT, v, X, rc, v, bWT);
        gs.B = pmat(opb(h, h->L.WTa), pWTa, v, X, R, v, bWT);
        gs.b_b0 = r0;
        gs.a_bstep = 1; gs.b_bstep = 1;
        gs.M = v; gs.N = v; gs.K = X; gs.batch = rcur; gs.ksplit = 1;
        gs.out = out_map(opb(h, h->L.S), pS, q.ke, 0, Ix{0, 0}, kpan((long long)rc * q.ke), plain(q.ldk * rc, q.ke));
        int e = run_tc(h, gs, "S");
        if (e) return e;
        // P[ij][r0+r] += sum_cd tau[ij][cd] S[r][cd]
        TcGemm gp{};
        gp.A = pmat(opb(h, h->L.tauN), (long long)o * o * q.kvv, o * o, (int)q.kvv, 1, (long long)o * o, 0);
        gp.B = pmat(opb(h, h->L.S), pS, rcur, (int)q.kvv, 1, rc, 0);
        gp.M = o * o; gp.N = rcur; gp.K = (int)q.kvv; gp.batch = 1;
        e = run_tc_partial(h, gp, P + r0, R, "P");
        if (e) return e;
    }
    return PPL_OK;
}

// the operand copies of a [X][v][v] source (B_vv or D-bar): Bn, Bp, BpW, Bq
// layouts (see the table above); src is B[Q][p][q] at Q*sQ + p*sp + q
void split_b_family(ppl_cpd* h, const double* src, long long sQ, long long sp, size_t offN, size_t offP, size_t offW,
                    size_t offQ) {
    const int v = h->v, X = h->X, prec = h->opts.precision;
    const Pan q = pan_of(h);
    const long long pBn = (long long)X * v * q.ldk;
    SplitSrc s{};
    s.src = src;
    if (offN != (size_t)-1) {   // rows (Q,d), K = b: B[Q][b][d]
        s.rmap = ix2(v, sQ, 1); s.cmap = ix1(sp);
        split_to_panels(prec, s, X * v, X * v, v, 0, 0, 1, opb(h, offN), pBn, h->st);
    }
    if (offP != (size_t)-1) {   // rows a, K = (Q, c): B[Q][a][c]
        s.rmap = ix1(sp); s.cmap = ix2((int)q.ldk, sQ, 1);
        split_to_panels(prec, s, v, v, (int)(X * q.ldk), (int)q.ldk, v, 1, opb(h, offP), pBn, h->st);
    }
    if (offW != (size_t)-1) {   // rows (c,Q), K = a: B[Q][c][a]
        s.rmap = ix2(X, sp, sQ); s.cmap = ix1(1);
        split_to_panels(prec, s, v * X, v * X, v, 0, 0, 1, opb(h, offW), pBn, h->st);
    }
    if (offQ != (size_t)-1) {   // rows (p,q), K = Q: B[Q][p][q]
        s.rmap = ix2(v, sp, 1); s.cmap = ix1(sQ);
        split_to_panels(prec, s, v * v, v * v, X, 0, 0, 1, opb(h, offQ), (long long)v * v * q.kX, h->st);
    }
}

// D-bar = B_vv - 2 B_vo t1 (t1 == nullptr: D-bar = B_vv), then its operand copies
void build_dbar(ppl_cpd* h, const double* t1) {
    const int o = h->o, v = h->v, X = h->X, n = h->n;
    double* Bb = h->at<double>(h->L.Bbar);
    extract_vv(h->B, o, v, X, Bb, h->st);
    if (t1) {
        G64 g{};
        g.A = h->B + (long long)o * n; g.ab = (long long)n * n; g.am = ix1(n); g.ak = ix1(1);   // B[Q][o+b][k]
        g.B = t1; g.bn = ix1(1); g.bk = ix1(v);                                            // t1[k][d]
        g.C = Bb; g.cb = (long long)v * v; g.cm = ix1(v); g.cn = ix1(1);
        g.M = v; g.N = v; g.K = o; g.batch = X; g.ksplit = 1; g.alpha = -2.0; g.beta = 1.0;
        gemm64(g, h->st);
    }
    if (!h->tc()) return;
    // D-bar[Q][b][d] is not symmetric in (b, d): the b side of every contraction reads it with b as the row index
    split_b_family(h, Bb, (long long)v * v, v, h->L.BbN, (size_t)-1, (size_t)-1, (size_t)-1);
    {
        // rows b, K = (Q, d): D-bar[Q][b][d]
        const Pan q = pan_of(h);
        SplitSrc s{};
        s.src = Bb; s.rmap = ix1(v); s.cmap = ix2((int)q.ldk, (long long)v * v, 1);
        split_to_panels(h->opts.precision, s, v, v, (int)(X * q.ldk), (int)q.ldk, v, 1, opb(h, h->L.BbP),
                        (long long)X * v * q.ldk, h->st);
        // rows (d,Q), K = b: D-bar[Q][b][d]
        s.rmap = ix2(X, 1, (long long)v * v); s.cmap = ix1(v);
        split_to_panels(h->opts.precision, s, v * X, v * X, v, 0, 0, 1, opb(h, h->L.BbT), (long long)X * v * q.ldk,
                        h->st);
        // rows (b,d), K = Q: D-bar[Q][b][d]
        s.rmap = ix1(1); s.cmap = ix1((long long)v * v);
        split_to_panels(h->opts.precision, s, v * v, v * v, X, 0, 0, 1, opb(h, h->L.BbQ), (long long)v * v * q.kX,
                        h->st);
    }
}

// operand copies of tau and B (once per tau / B)
int prepare_operands(ppl_cpd* h, bool tau_only) {
    if (!h->tc()) return PPL_OK;
    const int o = h->o, v = h->v, X = h->X, n = h->n, prec = h->opts.precision;
    const Pan q = pan_of(h);
    SplitSrc s{};
    // tauT rows (c,d), K = (i,j)
    s.src = h->tau; s.rmap = ix1(1); s.cmap = ix1((long long)v * v);
    split_to_panels(prec, s, v * v, v * v, o * o, 0, 0, 1, opb(h, h->L.tauT), (long long)v * v * q.ko2, h->st);
    // tauN rows (i,j), K = (c, d), d padded to ldk
    s.rmap = ix1((long long)v * v); s.cmap = ix2((int)q.ldk, v, 1);
    split_to_panels(prec, s, o * o, o * o, (int)q.kvv, (int)q.ldk, v, 1, opb(h, h->L.tauN), (long long)o * o * q.kvv,
                    h->st);
    if (tau_only) return PPL_OK;
    split_b_family(h, h->B + (long long)o * n + o, (long long)n * n, n, h->L.Bn, h->L.Bp, h->L.BpW, h->L.Bq);
    // intermediates whose K padding (never written by the epilogues) must read as zero
    const size_t eb = h->opbytes();
    zero_bytes(opb(h, h->L.T), (size_t)h->R * v * q.ldk * eb, h->st);
    zero_bytes(opb(h, h->L.Tt), (size_t)h->R * v * q.ldk * eb, h->st);
    zero_bytes(opb(h, h->L.W), (size_t)h->L.rc * X * q.ldk * eb, h->st);
    zero_bytes(opb(h, h->L.Y), (size_t)h->L.rc * X * q.ldk * eb, h->st);
    zero_bytes(opb(h, h->L.WTa), (size_t)h->R * v * q.kX * eb, h->st);
    zero_bytes(opb(h, h->L.WTb), (size_t)h->L.rc * v * q.kX * eb, h->st);
    zero_bytes(opb(h, h->L.S), (size_t)h->L.rc * q.kvv * eb, h->st);
    zero_bytes(opb(h, h->L.Gop), (size_t)v * q.kvv * eb, h->st);
    return PPL_OK;
}

int mttkrp_into(ppl_cpd* h, int mode, double* Mout) {
    const int o = h->o, R = h->R;
    if (mode < 2) {
        if (h->tc()) {
            int e = t_tc(h);
            if (e) return e;
            return chain_tc(h, mode, Mout, false);
        }
        t_fp64(h);
        mttkrp_ab_fp64(h, mode, Mout);
        return PPL_OK;
    }
    if (h->tc()) {
        int e = p_tc(h, false);
        if (e) return e;
    } else {
        p_fp64(h);
    }
    occ_mttkrp(h->at<double>(h->L.P), R, mode == 2 ? h->U[3] : h->U[2], o, R, mode == 2 ? 0 : 1, Mout, h->st);
    return PPL_OK;
}

// cross Gram X_m = U_m^T Uold_m
void cross_gram(ppl_cpd* h, int m) {
    G64 g{};
    const int R = h->R;
    g.A = h->U[m]; g.am = ix1(1); g.ak = ix1(R);
    g.B = h->at<double>(h->L.Uold[m]); g.bn = ix1(1); g.bk = ix1(R);
    g.C = h->at<double>(h->L.Xc[m]); g.cm = ix1(R); g.cn = ix1(1);
    g.M = R; g.N = R; g.K = h->dim(m); g.batch = 1; g.ksplit = 1; g.alpha = 1.0;
    gemm64(g, h->st);
}

// phase boundary; External makes the record a real event node when the
// sweep is being captured into a graph
void mark(ppl_cpd* h, int k) {
    if (h->opts.profile) cudaEventRecordWithFlags(h->pev[k], h->st, cudaEventRecordExternal);
}

// One sweep in five phases; phase q = 0..3 leaves mode q's MTTKRP in L.M and is
// followed by mode q's solve, phase 4 forms the fit terms (and eta).
int sweep_phase(ppl_cpd* h, int q) {
    const int o = h->o, R = h->R;
    double* M = h->at<double>(h->L.M);
    double* P = h->at<double>(h->L.P);
    int e = PPL_OK;
    switch (q) {
    case 0:
        if (h->opts.want_eta) {
            for (int m = 0; m < 4; ++m)
                cudaMemcpyAsync(h->at<double>(h->L.Uold[m]), h->U[m], (size_t)h->dim(m) * R * sizeof(double),
                                cudaMemcpyDeviceToDevice, h->st);
            cudaMemcpyAsync(h->at<double>(h->L.lamold), h->lam, (size_t)R * sizeof(double),
                            cudaMemcpyDeviceToDevice, h->st);
        }
        mark(h, 0);
        if (h->tc()) {
            if ((e = t_tc(h))) return e;
            mark(h, 1);
            if ((e = chain_tc(h, 0, M, false))) return e;
        } else {
            t_fp64(h);
            mark(h, 1);
            mttkrp_ab_fp64(h, 0, M);
        }
        mark(h, 2);
        break;
    case 1:
        mark(h, 3);
        if (h->tc()) {
            if ((e = chain_tc(h, 1, M, h->reuse_wa()))) return e;
        } else {
            mttkrp_ab_fp64(h, 1, M);
        }
        mark(h, 4);
        break;
    case 2:
        mark(h, 5);
        if (h->tc()) {
            if ((e = p_tc(h, h->reuse_wa()))) return e;
        } else {
            p_fp64(h);
        }
        mark(h, 6);
        occ_mttkrp(P, R, h->U[3], o, R, 0, M, h->st);
        break;
    case 3:
        occ_mttkrp(P, R, h->U[2], o, R, 1, M, h->st);
        break;
    default: {
        mark(h, 7);
        double* sc = h->scal();
        double* hist = h->at<double>(h->L.hist);
        fit_terms(M, h->U[3], h->lam, o, R, h->G(0), h->G(1), h->G(2), h->G(3), h->at<double>(h->L.partial),
                  sc + SC_TERMS, h->st);
        finish_fit(sc + SC_TERMS, sc + SC_NORMR2, hist, h->st);
        if (h->opts.want_eta) {
            for (int m = 0; m < 4; ++m) cross_gram(h, m);
            eta_terms(h->at<double>(h->L.Xc[0]), h->at<double>(h->L.Xc[1]), h->at<double>(h->L.Xc[2]),
                      h->at<double>(h->L.Xc[3]), h->lam, h->at<double>(h->L.lamold), R,
                      h->at<double>(h->L.partial), sc + SC_CROSS, h->st);
            finish_eta(sc + SC_CROSS, sc + SC_TERMS + 1, sc + SC_NORM2_PREV, hist, h->st);
            cudaMemcpyAsync(sc + SC_NORM2_PREV, sc + SC_TERMS + 1, sizeof(double), cudaMemcpyDeviceToDevice, h->st);
        }
        mark(h, 8);
    }
    }
    return PPL_OK;
}

int sweep_body(ppl_cpd* h) {
    int e;
    for (int q = 0; q < 4; ++q) {
        if ((e = sweep_phase(h, q))) return e;
        if ((e = solve_mode(h, q))) return e;
    }
    if ((e = sweep_phase(h, 4))) return e;
    return check_cuda(h, "sweep");
}

// the factor buffer holds a new guess: lam = 1, Gram matrices, ||R~_0||^2 (on h->st)
void refresh_factors(ppl_cpd* h) {
    fill_f64(h->lam, (size_t)h->R, 1.0, h->st);
    for (int m = 0; m < 4; ++m) gram(h, m);
    fit_terms(h->at<double>(h->L.M), h->U[0], h->lam, 0, h->R, h->G(0), h->G(1), h->G(2), h->G(3),
              h->at<double>(h->L.partial), h->scal() + SC_TERMS, h->st);
    cudaMemcpyAsync(h->scal() + SC_NORM2_PREV, h->scal() + SC_TERMS + 1, sizeof(double), cudaMemcpyDeviceToDevice,
                    h->st);
}

int enter(ppl_cpd* h) {
    cudaEventRecord(h->ev_in, h->user);
    cudaStreamWaitEvent(h->st, h->ev_in, 0);
    return check_cuda(h, "stream order");
}

int leave(ppl_cpd* h) {
    cudaEventRecord(h->ev_out, h->st);
    cudaStreamWaitEvent(h->user, h->ev_out, 0);
    return check_cuda(h, "stream order");
}

int sync_and_check(ppl_cpd* h) {
    cudaError_t e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return fail(h, PPL_ECUDA, "stream synchronise: %s", cudaGetErrorString(e));
    unsigned int flag = 0;
    cudaMemcpy(&flag, h->errflag(), sizeof flag, cudaMemcpyDeviceToHost);
    if (flag) {
        cudaMemset(h->errflag(), 0, sizeof flag);
        h->ntimeouts++;
        return fail(h, PPL_ETIMEOUT, "a bounded device wait expired (flags 0x%x)", flag);
    }
    return PPL_OK;
}

}  // namespace

// message for ppl_last_error(NULL) from other translation units
void ppl_set_global_error(const char* msg) { g_err = msg; }

// ============================================================================
// C ABI
// ============================================================================

extern "C" {

void ppl_cpd_default_opts(ppl_cpd_opts* opts) {
    if (!opts) return;
    memset(opts, 0, sizeof *opts);
    opts->precision = PPL_PREC_TF32X3;
    opts->r_chunk = 0;
    opts->use_graph = 1;
    opts->want_eta = 0;
}

int ppl_cpd_workspace_size(int o, int v, int X, int R, const ppl_cpd_opts* opts, size_t* bytes) {
    ppl_cpd_opts op;
    ppl_cpd_default_opts(&op);
    if (opts) op = *opts;
    if (!bytes) return fail(nullptr, PPL_EINVAL, "bytes is NULL");
    if (op.precision < 0 || op.precision > 3) return fail(nullptr, PPL_EINVAL, "unknown precision %d", op.precision);
    Layout L;
    if (!plan(o, v, X, R, op, L)) return fail(nullptr, PPL_EINVAL, "sizes out of range (o=%d v=%d X=%d R=%d)", o, v, X, R);
    *bytes = L.total;
    return PPL_OK;
}

int ppl_cpd_init(ppl_cpd** hp, int o, int v, int X, int R, const double* B, const double* tau, double* factors,
                 void* workspace, size_t ws_bytes, const ppl_cpd_opts* opts, void* stream) {
    if (!hp) return fail(nullptr, PPL_EINVAL, "handle pointer is NULL");
    *hp = nullptr;
    ppl_cpd_opts op;
    ppl_cpd_default_opts(&op);
    if (opts) op = *opts;
    if (op.precision < 0 || op.precision > 3) return fail(nullptr, PPL_EINVAL, "unknown precision %d", op.precision);
    if (op.init < PPL_INIT_USER || op.init > PPL_INIT_UNIFORM)
        return fail(nullptr, PPL_EINVAL, "unknown initial guess %d", op.init);
    if (!B || !tau || !factors || !workspace) return fail(nullptr, PPL_EINVAL, "NULL device pointer");
    if (((uintptr_t)workspace) % 256) return fail(nullptr, PPL_EINVAL, "workspace not 256-byte aligned");
    Layout L;
    if (!plan(o, v, X, R, op, L)) return fail(nullptr, PPL_EINVAL, "sizes out of range (o=%d v=%d X=%d R=%d)", o, v, X, R);
    if (ws_bytes < L.total)
        return fail(nullptr, PPL_ENOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, L.total);
    if (op.precision != PPL_PREC_FP64 && tc_init_driver() != 0)
        return fail(nullptr, PPL_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    ppl_cpd* h = new (std::nothrow) ppl_cpd();
    if (!h) return fail(nullptr, PPL_EINVAL, "out of host memory");
    h->o = o; h->v = v; h->X = X; h->R = R; h->n = o + v;
    h->opts = op;
    h->user = (cudaStream_t)stream;
    h->B = B; h->tau = tau; h->fac = factors;
    h->U[0] = factors;
    h->U[1] = factors + (size_t)v * R;
    h->U[2] = factors + (size_t)2 * v * R;
    h->U[3] = factors + (size_t)2 * v * R + (size_t)o * R;
    h->lam = factors + (size_t)2 * v * R + (size_t)2 * o * R;
    h->ws = (char*)workspace; h->ws_bytes = ws_bytes;
    h->L = L;
    h->normR2 = 0.0; h->have_normR2 = false; h->sweeps = 0;
    h->graph = nullptr; h->gexec = nullptr; h->graph_ready = false;
    for (double& x : h->last_hist) x = nan("");
    h->have_pev = false;
    h->kernels_per_sweep = 0;
    h->guess_policy = PPL_GUESS_OPTIMAL;
    h->solve_cap = 0;
    h->tc_cap = 0;
    h->cache_valid = false;
    h->nsolves = 0;
    h->ntimeouts = 0;
    h->wait_ns = op.wait_limit_us > 0 ? (unsigned long long)op.wait_limit_us * 1000ull : 0ull;
    if (op.profile) {
        for (int k = 0; k < 9; ++k)
            if (cudaEventCreate(&h->pev[k]) != cudaSuccess) {
                cudaGetLastError();
                delete h;
                return fail(nullptr, PPL_ECUDA, "could not create profiling events");
            }
        h->have_pev = true;
    }
    if (cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(nullptr, PPL_ECUDA, "could not create the internal stream/events");
    }
    int e = enter(h);
    if (!e) {
        cudaMemsetAsync(h->ws + L.scal, 0, NSCAL * sizeof(double), h->st);
        cudaMemsetAsync(h->ws + L.flags, 0, 64, h->st);
        // the stream of the seeded synthetic inputs' initial factors (id 4)
        if (op.init != PPL_INIT_USER)
            fill_random(h->fac, (long long)(2 * v + 2 * o) * R, op.init == PPL_INIT_NORMAL, (unsigned int)op.init_seed, 4,
                        h->st);
        fill_f64(h->lam, (size_t)R, 1.0, h->st);
        cudaMemcpyAsync(h->ws + L.guess0, h->fac, h->fac_bytes(), cudaMemcpyDeviceToDevice, h->st);
        for (int m = 0; m < 4; ++m) gram(h, m);
        // ||R~_0||^2 of the initial guess (eta's first denominator)
        fit_terms(h->at<double>(h->L.M), h->U[0], h->lam, 0, R, h->G(0), h->G(1), h->G(2), h->G(3),
                  h->at<double>(h->L.partial), h->scal() + SC_TERMS, h->st);
        cudaMemcpyAsync(h->scal() + SC_NORM2_PREV, h->scal() + SC_TERMS + 1, sizeof(double),
                        cudaMemcpyDeviceToDevice, h->st);
        e = prepare_operands(h, false);
        if (!e && h->dressed()) build_dbar(h, nullptr);
    }
    if (!e) e = check_cuda(h, "init");
    if (!e) e = leave(h);
    if (e) {
        g_err = h->err;
        cudaStreamDestroy(h->st);
        cudaEventDestroy(h->ev_in);
        cudaEventDestroy(h->ev_out);
        delete h;
        return e;
    }
    *hp = h;
    return PPL_OK;
}

int ppl_cpd_mttkrp(ppl_cpd* h, int mode, double* M_out) {
    if (!h) return fail(nullptr, PPL_EINVAL, "NULL handle");
    if (mode < 0 || mode > 3) return fail(h, PPL_EINVAL, "mode %d out of range", mode);
    if (!M_out) return fail(h, PPL_EINVAL, "M_out is NULL");
    int e = enter(h);
    if (!e) e = mttkrp_into(h, mode, M_out);
    if (!e) e = check_cuda(h, "mttkrp");
    if (!e) e = sync_and_check(h);
    leave(h);
    return e;
}

int ppl_cpd_sweep(ppl_cpd* h, int nsweeps, double* fit_hist) {
    if (!h) return fail(nullptr, PPL_EINVAL, "NULL handle");
    if (nsweeps < 0) return fail(h, PPL_EINVAL, "nsweeps < 0");
    if (nsweeps == 0) return PPL_OK;
    int e = enter(h);
    if (e) return e;
    double* hist = h->at<double>(h->L.hist);
    double host_hist[4];
    for (int k = 0; k < nsweeps; ++k) {
        if (h->opts.use_graph) {
            if (!h->graph_ready) {
                cudaError_t ce = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal);
                if (ce != cudaSuccess) return fail(h, PPL_ECUDA, "begin capture: %s", cudaGetErrorString(ce));
                int be = sweep_body(h);
                cudaGraph_t gr = nullptr;
                ce = cudaStreamEndCapture(h->st, &gr);
                if (be) {
                    if (gr) cudaGraphDestroy(gr);
                    return be;
                }
                if (ce != cudaSuccess) return fail(h, PPL_ECUDA, "end capture: %s", cudaGetErrorString(ce));
                ce = cudaGraphInstantiate(&h->gexec, gr, 0);
                if (ce != cudaSuccess) {
                    cudaGraphDestroy(gr);
                    return fail(h, PPL_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));
                }
                h->graph = gr;
                h->graph_ready = true;
                size_t nn = 0;
                cudaGraphGetNodes(gr, nullptr, &nn);
                if (nn) {
                    cudaGraphNode_t* nodes = new cudaGraphNode_t[nn];
                    cudaGraphGetNodes(gr, nodes, &nn);
                    long long kc = 0;
                    for (size_t q = 0; q < nn; ++q) {
                        cudaGraphNodeType t;
                        cudaGraphNodeGetType(nodes[q], &t);
                        if (t == cudaGraphNodeTypeKernel) ++kc;
                    }
                    delete[] nodes;
                    h->kernels_per_sweep = kc;
                }
            }
            cudaGraphLaunch(h->gexec, h->st);
        } else {
            e = sweep_body(h);
            if (e) return e;
        }
        if (fit_hist || k == nsweeps - 1) {
            e = sync_and_check(h);
            if (e) { leave(h); return e; }
            cudaMemcpy(host_hist, hist, sizeof host_hist, cudaMemcpyDeviceToHost);
            if (fit_hist) fit_hist[k] = host_hist[0];
            for (int q = 0; q < 4; ++q) h->last_hist[q] = host_hist[q];
        }
        h->sweeps++;
    }
    e = check_cuda(h, "sweep");
    leave(h);
    return e;
}

int ppl_cpd_set_normR2(ppl_cpd* h, double normR2) {
    if (!h) return fail(nullptr, PPL_EINVAL, "NULL handle");
    if (!(normR2 > 0.0)) return fail(h, PPL_EINVAL, "normR2 must be positive");
    h->normR2 = normR2;
    h->have_normR2 = true;
    int e = enter(h);
    if (e) return e;
    cudaMemcpyAsync(h->scal() + SC_NORMR2, &h->normR2, sizeof(double), cudaMemcpyHostToDevice, h->st);
    e = sync_and_check(h);
    leave(h);
    return e;
}

int ppl_cpd_fit(ppl_cpd* h, double* fit) {
    if (!h || !fit) return fail(h, PPL_EINVAL, "NULL argument");
    if (!h->have_normR2) return fail(h, PPL_ENOTREADY, "||R||^2 unknown: call ppl_exact_contract or ppl_cpd_set_normR2");
    if (h->sweeps == 0) return fail(h, PPL_ENOTREADY, "no sweep has run");
    const double inner = h->last_hist[1], norm2 = h->last_hist[2];
    *fit = 1.0 - sqrt(fmax(h->normR2 - 2.0 * inner + norm2, 0.0)) / sqrt(h->normR2);
    return PPL_OK;
}

int ppl_cpd_energy(ppl_cpd* h, double* E_cp) {
    if (!h || !E_cp) return fail(h, PPL_EINVAL, "NULL argument");
    const int o = h->o, v = h->v, X = h->X, R = h->R, n = h->n;
    int e = enter(h);
    if (e) return e;
    double* Z[2] = {h->at<double>(h->L.Za), h->at<double>(h->L.Zb)};
    for (int w = 0; w < 2; ++w) {
        G64 g{};
        g.A = h->B + o; g.ab = (long long)n * n; g.am = ix1(n); g.ak = ix1(1);
        g.B = h->U[w]; g.bn = ix1(1); g.bk = ix1(R);
        g.C = Z[w]; g.cb = (long long)o * R; g.cm = ix1(R); g.cn = ix1(1);
        g.M = o; g.N = R; g.K = v; g.batch = X; g.ksplit = 1; g.alpha = 1.0;
        gemm64(g, h->st);
    }
    energy_reduce(Z[0], Z[1], h->U[2], h->U[3], h->lam, X, o, R, h->at<double>(h->L.partial),
                  h->scal() + SC_ENERGY, h->st);
    e = check_cuda(h, "energy");
    if (!e) e = sync_and_check(h);
    if (!e) cudaMemcpy(E_cp, h->scal() + SC_ENERGY, sizeof(double), cudaMemcpyDeviceToHost);
    leave(h);
    return e ? e : check_cuda(h, "energy");
}

int ppl_exact_contract(ppl_cpd* h, double* normR2, double* E_exact, double* R_out) {
    if (!h) return fail(nullptr, PPL_EINVAL, "NULL handle");
    const int o = h->o, v = h->v, X = h->X, n = h->n, na = h->L.na;
    int e = enter(h);
    if (e) return e;
    double* gov = h->at<double>(h->L.gov);
    double* Gb = h->at<double>(h->L.Gblk);
    double* Rb = h->at<double>(h->L.Rblk);
    double* acc = h->scal() + SC_EXACT;
    cudaMemsetAsync(acc, 0, 2 * sizeof(double), h->st);
    // g[i][a][j][b] = sum_Q B[Q][i][o+a] B[Q][j][o+b]
    G64 g{};
    g.A = h->B + o; g.am = ix2(v, n, 1); g.ak = ix1((long long)n * n);
    g.B = h->B + o; g.bn = ix2(v, n, 1); g.bk = ix1((long long)n * n);
    g.C = gov; g.cm = ix1((long long)o * v); g.cn = ix1(1);
    g.M = o * v; g.N = o * v; g.K = X; g.batch = 1; g.ksplit = 1; g.alpha = 1.0;
    gemm64(g, h->st);
    const long long v3 = (long long)v * v * v, vo2 = (long long)v * o * o;
    for (int a0 = 0; a0 < v; a0 += na) {
        const int nb = (v - a0 < na) ? v - a0 : na;
        // G_a[c][b*v+d] = sum_Q B[Q][o+a][o+c] B[Q][o+b][o+d]
        G64 q{};
        q.A = h->B + (long long)(o + a0) * n + o; q.ab = n; q.am = ix1(1); q.ak = ix1((long long)n * n);
        if (h->dressed()) {
            q.B = h->at<double>(h->L.Bbar); q.bb = 0; q.bn = ix1(1); q.bk = ix1((long long)v * v);
        } else {
            q.B = h->B + (long long)o * n + o; q.bb = 0; q.bn = ix2(v, n, 1); q.bk = ix1((long long)n * n);
        }
        q.C = Gb; q.cb = v3; q.cm = ix1((long long)v * v); q.cn = ix1(1);
        q.M = v; q.N = v * v; q.K = X; q.batch = nb; q.ksplit = 1; q.alpha = 1.0;
        gemm64(q, h->st);
        // R[a][b][ij] = sum_{c,d} G_a[c][b][d] tau[ij][c][d]
        double* Rdst = R_out ? R_out + (long long)a0 * vo2 : Rb;
        G64 r{};
        r.A = Gb; r.ab = v3; r.am = ix1(v); r.ak = ix2(v, (long long)v * v, 1);
        r.B = h->tau; r.bb = 0; r.bn = ix1((long long)v * v); r.bk = ix1(1);
        r.C = Rdst; r.cb = vo2; r.cm = ix1((long long)o * o); r.cn = ix1(1);
        r.M = v; r.N = o * o; r.K = v * v; r.batch = nb; r.ksplit = 1; r.alpha = 1.0;
        gemm64(r, h->st);
        exact_reduce(Rdst, a0, nb, v, o, gov, h->at<double>(h->L.partial), acc, h->st);
    }
    e = check_cuda(h, "exact_contract");
    if (!e) e = sync_and_check(h);
    double res[2] = {0, 0};
    if (!e) cudaMemcpy(res, acc, sizeof res, cudaMemcpyDeviceToHost);
    leave(h);
    if (e) return e;
    if (normR2) *normR2 = res[0];
    if (E_exact) *E_exact = res[1];
    if (res[0] > 0.0) return ppl_cpd_set_normR2(h, res[0]);
    return PPL_OK;
}

int ppl_cpd_reconstruct(ppl_cpd* h, double* R_out, int symmetrise) {
    if (!h || !R_out) return fail(h, PPL_EINVAL, "NULL argument");
    const int o = h->o, v = h->v, R = h->R, rcr = h->L.rcr;
    int e = enter(h);
    if (e) return e;
    double* Kab = h->at<double>(h->L.recon);
    double* Kij = Kab + (size_t)v * v * rcr;
    for (int r0 = 0; r0 < R; r0 += rcr) {
        const int rc = (R - r0 < rcr) ? R - r0 : rcr;
        kr_pair(h->U[0], h->U[1], h->lam, v, v, R, r0, rc, Kab, h->st);
        kr_pair(h->U[2], h->U[3], nullptr, o, o, R, r0, rc, Kij, h->st);
        G64 g{};
        g.A = Kab; g.am = ix1(rc); g.ak = ix1(1);
        g.B = Kij; g.bn = ix1(rc); g.bk = ix1(1);
        g.C = R_out; g.cm = ix1((long long)o * o); g.cn = ix1(1);
        g.M = v * v; g.N = o * o; g.K = rc; g.batch = 1; g.ksplit = 1;
        g.alpha = 1.0; g.beta = (r0 == 0) ? 0.0 : 1.0;
        gemm64(g, h->st);
    }
    if (symmetrise) symmetrise_pairs(R_out, v, o, h->st);
    e = check_cuda(h, "reconstruct");
    if (!e) e = sync_and_check(h);
    leave(h);
    return e;
}

int ppl_exact_contract_mixed(ppl_cpd* h, double* normR2, double* E_exact, double* R_out) {
    if (!h) return fail(nullptr, PPL_EINVAL, "NULL handle");
    if (!h->tc()) return fail(h, PPL_EINVAL, "ppl_exact_contract_mixed needs a tensor-core (BF16X3, TF32 or TF32X3) handle");
    const int o = h->o, v = h->v, X = h->X, n = h->n;
    const long long vo2 = (long long)v * o * o;
    int e = enter(h);
    if (e) return e;
    double* gov = h->at<double>(h->L.gov);
    double* acc = h->scal() + SC_EXACT;
    cudaMemsetAsync(acc, 0, 2 * sizeof(double), h->st);
    G64 g{};
    g.A = h->B + o; g.am = ix2(v, n, 1); g.ak = ix1((long long)n * n);
    g.B = h->B + o; g.bn = ix2(v, n, 1); g.bk = ix1((long long)n * n);
    g.C = gov; g.cm = ix1((long long)o * v); g.cn = ix1(1);
    g.M = o * v; g.N = o * v; g.K = X; g.batch = 1; g.ksplit = 1; g.alpha = 1.0;
    gemm64(g, h->st);
    const Pan pq = pan_of(h);
    const long long pQ = (long long)v * v * pq.kX, pG = (long long)v * pq.kvv;
    for (int a = 0; a < v && !e; ++a) {
        // G_a[b][c][d] = sum_Q D-bar[Q][b][d] B[Q][a][c]; stored rows b, K (c, d): m = b*v + d, n = c
        TcGemm g1{};
        g1.A = pmat(opb(h, h->dressed() ? h->L.BbQ : h->L.Bq), pQ, v * v, X, 1, (long long)v * v, 0);
        g1.B = pmat(opb(h, h->L.Bq), pQ, v * v, X, 1, (long long)v * v, 0);
        g1.b_row0 = a * v;
        g1.M = v * v; g1.N = v; g1.K = X; g1.batch = 1; g1.ksplit = 1;
        g1.out = out_map(opb(h, h->L.Gop), pG, 0, v, plain(pq.ke, pq.ke), kpan((long long)v * pq.ke),
                         plain(pq.ldk * v, pq.ke));
        e = run_tc(h, g1, "exact G");
        if (e) break;
        // R[a][b][ij] = sum_{cd} G_a[b][cd] tau[ij][cd], split-K summed in FP64
        double* Rdst = R_out ? R_out + (long long)a * vo2 : h->at<double>(h->L.Rblk);
        TcGemm g2{};
        g2.A = pmat(opb(h, h->L.Gop), pG, v, (int)pq.kvv, 1, v, 0);
        g2.B = pmat(opb(h, h->L.tauN), (long long)o * o * pq.kvv, o * o, (int)pq.kvv, 1, (long long)o * o, 0);
        g2.M = v; g2.N = o * o; g2.K = (int)pq.kvv; g2.batch = 1;
        e = run_tc_partial(h, g2, Rdst, (long long)o * o, "exact R");
        if (e) break;
        exact_reduce(Rdst, a, 1, v, o, gov, h->at<double>(h->L.partial), acc, h->st);
    }
    if (!e) e = check_cuda(h, "exact_contract_mixed");
    if (!e) e = sync_and_check(h);
    double res[2] = {0, 0};
    if (!e) cudaMemcpy(res, acc, sizeof res, cudaMemcpyDeviceToHost);
    leave(h);
    if (e) return e;
    if (normR2) *normR2 = res[0];
    if (E_exact) *E_exact = res[1];
    if (res[0] > 0.0) return ppl_cpd_set_normR2(h, res[0]);
    return PPL_OK;
}

int ppl_cpd_set_t1(ppl_cpd* h, const double* t1) {
    if (!h) return fail(nullptr, PPL_EINVAL, "NULL handle");
    if (!h->dressed()) return fail(h, PPL_EINVAL, "the handle was created without opts.dressed");
    h->have_normR2 = false;
    h->normR2 = 0.0;
    int e = enter(h);
    if (e) return e;
    cudaMemsetAsync(h->scal() + SC_NORMR2, 0, sizeof(double), h->st);
    build_dbar(h, t1);
    e = check_cuda(h, "set_t1");
    if (!e) e = sync_and_check(h);
    leave(h);
    return e;
}

int ppl_cpd_set_tau(ppl_cpd* h, const double* tau) {
    if (!h || !tau) return fail(h, PPL_EINVAL, "NULL argument");
    const bool same = (tau == h->tau);
    h->tau = tau;
    h->have_normR2 = false;
    h->normR2 = 0.0;
    int e = enter(h);
    if (e) return e;
    cudaMemsetAsync(h->scal() + SC_NORMR2, 0, sizeof(double), h->st);
    e = prepare_operands(h, true);
    if (!e) e = check_cuda(h, "set_tau");
    if (!e) e = sync_and_check(h);
    leave(h);
    // the FP64 form reads tau through its pointer, which a captured graph has baked in
    if (h->graph_ready && !same) {
        cudaGraphExecDestroy(h->gexec);
        cudaGraphDestroy(h->graph);
        h->gexec = nullptr;
        h->graph = nullptr;
        h->graph_ready = false;
    }
    return e;
}

int ppl_cpd_factors_changed(ppl_cpd* h) {
    if (!h) return fail(nullptr, PPL_EINVAL, "NULL handle");
    int e = enter(h);
    if (e) return e;
    refresh_factors(h);
    e = check_cuda(h, "factors_changed");
    if (!e) e = sync_and_check(h);
    leave(h);
    return e;
}

int ppl_cpd_set_guess_policy(ppl_cpd* h, int policy) {
    if (!h) return fail(nullptr, PPL_EINVAL, "NULL handle");
    if (policy < PPL_GUESS_OPTIMAL || policy > PPL_GUESS_RANDOM) return fail(h, PPL_EINVAL, "unknown policy %d", policy);
    h->guess_policy = policy;
    return PPL_OK;
}

int ppl_cpd_solve(ppl_cpd* h, int max_sweeps, int stop_rule, double eps, int* sweeps_done, double* fit_hist,
                  double* eta_hist) {
    if (!h) return fail(nullptr, PPL_EINVAL, "NULL handle");
    if (max_sweeps < 1) return fail(h, PPL_EINVAL, "max_sweeps < 1");
    if (stop_rule < PPL_STOP_FIXED || stop_rule > PPL_STOP_ETA) return fail(h, PPL_EINVAL, "unknown stop rule");
    if (stop_rule == PPL_STOP_ETA && !h->opts.want_eta) return fail(h, PPL_EINVAL, "PPL_STOP_ETA needs want_eta");
    if (stop_rule == PPL_STOP_DFIT && !h->have_normR2) return fail(h, PPL_ENOTREADY, "PPL_STOP_DFIT needs ||R||^2");
    int e = enter(h);
    if (e) return e;
    const size_t fb = h->fac_bytes();
    if (h->nsolves > 0 && h->guess_policy != PPL_GUESS_OPTIMAL) {
        const size_t src = (h->guess_policy == PPL_GUESS_NEAR_OPTIMAL && h->cache_valid) ? h->L.cache : h->L.guess0;
        cudaMemcpyAsync(h->fac, h->ws + src, fb, cudaMemcpyDeviceToDevice, h->st);
        refresh_factors(h);
    }
    cudaMemcpyAsync(h->ws + h->L.ring, h->fac, fb, cudaMemcpyDeviceToDevice, h->st);   // iterate 0
    e = leave(h);
    if (e) return e;
    double prev_fit = nan("");
    int n = 0;
    for (n = 1; n <= max_sweeps; ++n) {
        double fit = 0.0;
        e = ppl_cpd_sweep(h, 1, &fit);
        if (e) return e;
        if (fit_hist) fit_hist[n - 1] = fit;
        if (eta_hist) eta_hist[n - 1] = h->last_hist[3];
        if ((e = enter(h))) return e;
        cudaMemcpyAsync(h->ws + h->L.ring + (size_t)(n % 6) * fb, h->fac, fb, cudaMemcpyDeviceToDevice, h->st);
        if ((e = leave(h))) return e;
        bool stop = false;
        if (stop_rule == PPL_STOP_DFIT && n >= 2 && fabs(fit - prev_fit) < eps) stop = true;
        if (stop_rule == PPL_STOP_ETA && h->last_hist[3] < eps) stop = true;
        prev_fit = fit;
        if (stop) break;
    }
    if (n > max_sweeps) n = max_sweeps;
    if (h->guess_policy == PPL_GUESS_NEAR_OPTIMAL && n > 5) {
        if ((e = enter(h))) return e;
        cudaMemcpyAsync(h->ws + h->L.cache, h->ws + h->L.ring + (size_t)((n - 5) % 6) * fb, fb,
                        cudaMemcpyDeviceToDevice, h->st);
        e = check_cuda(h, "solve");
        if (!e) e = sync_and_check(h);
        leave(h);
        if (e) return e;
        h->cache_valid = true;
    }
    h->nsolves++;
    if (sweeps_done) *sweeps_done = n;
    return PPL_OK;
}

int ppl_cpd_autotune(ppl_cpd* h, int* r_chunk_out) {
    if (!h) return fail(nullptr, PPL_EINVAL, "NULL handle");
    const int planned = h->L.rc;
    const int step = h->tc() ? 16 : 1;
    // candidates up to the planned (allocated) chunk: fixed widths and the
    // balanced splits of R into 1..16 passes
    std::vector<int> cand;
    const int base[] = {48, 64, 96, 128, 160, 208, 256};
    for (int c : base) {
        const int cc = (c / step) * step;
        if (cc >= step && cc < planned) cand.push_back(cc);
    }
    for (int n = 1; n <= 16; ++n) {
        int cc = (h->R + n - 1) / n;
        cc = (cc + step - 1) / step * step;
        if (cc < planned) cand.push_back(cc);
    }
    cand.push_back(planned);
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    int e = enter(h);
    if (e) return e;
    double* M = h->at<double>(h->L.M);
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    if (h->tc()) e = t_tc(h);
    else t_fp64(h);
    float best_ms = 1e30f;
    int best = planned;
    for (int c : cand) {
        h->L.rc = c;
        for (int rep = 0; rep < 2 && !e; ++rep) {   // the first pass warms up
            cudaEventRecord(t0, h->st);
            if (h->tc()) e = chain_tc(h, 0, M, false);
            else mttkrp_ab_fp64(h, 0, M);
            cudaEventRecord(t1, h->st);
        }
        if (e) break;
        if (cudaEventSynchronize(t1) != cudaSuccess) { e = check_cuda(h, "autotune"); break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, t0, t1);
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    h->L.rc = e ? planned : best;
    if (!e) e = check_cuda(h, "autotune");
    if (!e) e = sync_and_check(h);
    leave(h);
    if (h->graph_ready) {
        cudaGraphExecDestroy(h->gexec);
        cudaGraphDestroy(h->graph);
        h->gexec = nullptr;
        h->graph = nullptr;
        h->graph_ready = false;
    }
    if (!e && r_chunk_out) *r_chunk_out = h->L.rc;
    return e;
}

int ppl_cpd_stats_get(ppl_cpd* h, ppl_cpd_stats* s) {
    if (!h || !s) return fail(h, PPL_EINVAL, "NULL argument");
    unsigned long long nc = 0;
    cudaStreamSynchronize(h->st);
    cudaMemcpy(&nc, h->nclamp(), sizeof nc, cudaMemcpyDeviceToHost);
    s->sweeps = h->sweeps;
    s->clamped_pivots = (long long)nc;
    s->timeouts = h->ntimeouts;
    s->last_fit = h->have_normR2 ? h->last_hist[0] : nan("");
    s->last_inner = h->last_hist[1];
    s->last_norm2 = h->last_hist[2];
    s->last_eta = h->opts.want_eta ? h->last_hist[3] : nan("");
    const double o = h->o, v = h->v, X = h->X, R = h->R;
    s->flops_per_sweep = 4.0 * o * o * v * v * R + 16.0 * X * v * v * R;
    s->kernels_per_sweep = h->kernels_per_sweep;
    return check_cuda(h, "stats");
}

const char* ppl_last_error(const ppl_cpd* h) { return h ? h->err.c_str() : g_err.c_str(); }

int ppl_cpd_inject_wait_timeout(ppl_cpd* h) {
    if (!h) return fail(nullptr, PPL_EINVAL, "NULL handle");
    int e = enter(h);
    if (e) return e;
    const unsigned int one = 1u;
    cudaMemcpyAsync(h->withhold(), &one, sizeof one, cudaMemcpyHostToDevice, h->st);
    e = check_cuda(h, "inject_wait_timeout");
    if (!e) {
        const cudaError_t ce = cudaStreamSynchronize(h->st);
        if (ce != cudaSuccess) e = fail(h, PPL_ECUDA, "inject_wait_timeout: %s", cudaGetErrorString(ce));
    }
    leave(h);
    return e;
}

}  // extern "C"

namespace {

// Merge the tensor-core contractions of a captured batch graph into grouped
// launches.  Every instance's work is a chain of nodes; a contraction's depth is
// the number of contractions on the longest path that ends in it.  Contractions
// of equal depth (and kernel) lie on no common path, so each such set becomes one
// persistent launch (at most tc_group_capacity() contractions each) that depends
// on all of the members' predecessors and precedes all of their successors.
// Returns 0, or a CUDA error code; *removed counts the launches saved.
int group_contractions(cudaGraph_t g, long long* removed) {
    *removed = 0;
    size_t nn = 0, ne = 0;
    if (cudaGraphGetNodes(g, nullptr, &nn) != cudaSuccess) return -1;
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn && cudaGraphGetNodes(g, nodes.data(), &nn) != cudaSuccess) return -1;
    if (cudaGraphGetEdges(g, nullptr, nullptr, nullptr, &ne) != cudaSuccess) return -1;
    std::vector<cudaGraphNode_t> from(ne), to(ne);
    if (ne && cudaGraphGetEdges(g, from.data(), to.data(), nullptr, &ne) != cudaSuccess) return -1;
    std::unordered_map<cudaGraphNode_t, int> id;
    for (size_t i = 0; i < nn; ++i) id[nodes[i]] = (int)i;
    std::vector<std::vector<int>> succ(nn), pred(nn);
    for (size_t e = 0; e < ne; ++e) {
        succ[id[from[e]]].push_back(id[to[e]]);
        pred[id[to[e]]].push_back(id[from[e]]);
    }
    std::vector<const void*> func(nn, nullptr), arg0(nn, nullptr);
    for (size_t i = 0; i < nn; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess) return -1;
        if (t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp{};
        if (cudaGraphKernelNodeGetParams(nodes[i], &kp) != cudaSuccess) return -1;
        if (tc_group_kernel(kp.func) && kp.kernelParams) {
            func[i] = kp.func;
            arg0[i] = kp.kernelParams[0];
        }
    }
    // depths in topological order
    std::vector<int> indeg(nn), depth(nn, 0), order;
    order.reserve(nn);
    for (size_t i = 0; i < nn; ++i) {
        indeg[i] = (int)pred[i].size();
        if (!indeg[i]) order.push_back((int)i);
    }
    for (size_t q = 0; q < order.size(); ++q) {
        const int v = order[q];
        if (func[v]) depth[v] += 1;
        for (int w : succ[v]) {
            depth[w] = std::max(depth[w], depth[v]);
            if (--indeg[w] == 0) order.push_back(w);
        }
    }
    if (order.size() != nn) return -2;   // not a DAG: leave the graph as it is
    std::map<std::pair<int, const void*>, std::vector<int>> sets;
    for (size_t i = 0; i < nn; ++i)
        if (func[i]) sets[{depth[i], func[i]}].push_back((int)i);
    const int cap = tc_group_capacity();
    // replaced node -> its group node (sets are visited by increasing depth, so a
    // member's predecessors may be contractions replaced earlier)
    std::unordered_map<cudaGraphNode_t, cudaGraphNode_t> repl;
    for (auto& kv : sets) {
        const std::vector<int>& all = kv.second;
        if (all.size() < 2) continue;
        // a few groups per depth rather than one: each holds a run of instances in
        // capture order, so the groups' chains stay largely independent and the
        // small kernels of one overlap the contractions of another
        int nparts = (int)((all.size() + cap - 1) / cap);
        const int sets = std::min<int>(BATCH_GROUP_SETS, (int)all.size() / 2);
        if (nparts < sets) nparts = sets;
        for (int part = 0; part < nparts; ++part) {
            const size_t b0 = all.size() * part / nparts, b1 = all.size() * (part + 1) / nparts;
            if (b1 - b0 < 2) continue;
            std::vector<const void*> args;
            std::vector<cudaGraphNode_t> deps, outs;
            for (size_t k = b0; k < b1; ++k) {
                const int m = all[k];
                args.push_back(arg0[m]);
                for (int u : pred[m]) {
                    cudaGraphNode_t d = nodes[u];
                    const auto r = repl.find(d);
                    if (r != repl.end()) d = r->second;
                    if (std::find(deps.begin(), deps.end(), d) == deps.end()) deps.push_back(d);
                }
                for (int w : succ[m])
                    if (std::find(outs.begin(), outs.end(), nodes[w]) == outs.end()) outs.push_back(nodes[w]);
            }
            cudaKernelNodeParams kp{};
            void* storage = nullptr;
            if (tc_group_node_params(kv.first.second, args.data(), (int)args.size(), &kp, &storage) != 0) continue;
            cudaGraphNode_t gn;
            cudaError_t ce = cudaGraphAddKernelNode(&gn, g, deps.data(), deps.size(), &kp);
            tc_group_release(storage);
            if (ce != cudaSuccess) return (int)ce;
            for (cudaGraphNode_t w : outs) {
                ce = cudaGraphAddDependencies(g, &gn, &w, nullptr, 1);
                if (ce != cudaSuccess) return (int)ce;
            }
            for (size_t k = b0; k < b1; ++k) {
                ce = cudaGraphDestroyNode(nodes[all[k]]);
                if (ce != cudaSuccess) return (int)ce;
                repl[nodes[all[k]]] = gn;
            }
            *removed += (long long)(b1 - b0) - 1;
        }
    }
    return 0;
}

}  // namespace

struct ppl_cpd_batch {
    std::vector<ppl_cpd*> hs;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaStream_t user, origin;
    cudaEvent_t fork, ev_in, ev_out;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    bool ready;
    long long kernels;
};

extern "C" {

int ppl_cpd_batch_create(ppl_cpd_batch** bp, int n, ppl_cpd* const* handles, int nstreams, void* stream) {
    if (!bp || n < 1 || !handles || nstreams < 1) return fail(nullptr, PPL_EINVAL, "bad batch arguments");
    for (int k = 0; k < n; ++k)
        if (!handles[k]) return fail(nullptr, PPL_EINVAL, "handle %d is NULL", k);
    ppl_cpd_batch* b = new (std::nothrow) ppl_cpd_batch();
    if (!b) return fail(nullptr, PPL_EINVAL, "out of host memory");
    b->hs.assign(handles, handles + n);
    b->user = (cudaStream_t)stream;
    b->graph = nullptr;
    b->exec = nullptr;
    b->ready = false;
    bool ok = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) == cudaSuccess;
    const int ns = nstreams < n ? nstreams : n;
    // solves are latency-bound chains of small FP64 steps: inside a batch each
    // takes a share of the SMs so that the solves of several instances overlap
    if (ns > 1) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int cap = sms > 0 ? (sms * BATCH_SOLVE_SHARE + ns - 1) / ns : 0;
        const int tcap = sms > 0 ? (sms * BATCH_TC_SHARE + ns - 1) / ns : 0;
        for (int k = 0; k < n; ++k) {
            handles[k]->solve_cap = cap;
            handles[k]->tc_cap = tcap;
        }
    }
    // one capture stream per instance: every instance's work is its own chain in the
    // graph, so that contractions of equal depth can be grouped (group_contractions)
    for (int i = 0; ok && i < n; ++i) {
        cudaStream_t s;
        cudaEvent_t e;
        ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        if (ok) {
            b->streams.push_back(s);
            b->joins.push_back(e);
        }
    }
    if (!ok) {
        cudaGetLastError();
        ppl_cpd_batch_destroy(b);
        return fail(nullptr, PPL_ECUDA, "could not create the batch streams/events");
    }
    *bp = b;
    return PPL_OK;
}

int ppl_cpd_batch_sweep(ppl_cpd_batch* b, int nsweeps, double* fits) {
    if (!b || nsweeps < 0) return fail(nullptr, PPL_EINVAL, "bad batch arguments");
    const int n = (int)b->hs.size();
    cudaEventRecord(b->ev_in, b->user);
    cudaStreamWaitEvent(b->origin, b->ev_in, 0);
    if (!b->ready) {
        cudaError_t ce = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) return fail(nullptr, PPL_ECUDA, "batch capture: %s", cudaGetErrorString(ce));
        // Phase by phase: every instance's contractions of a phase on the forked
        // streams, then one cooperative launch that solves that mode for all
        // instances at once (each on its share of the SMs, with its own barriers).
        int err = PPL_OK;
        auto fork = [&]() {
            cudaEventRecord(b->fork, b->origin);
            for (size_t i = 0; i < b->streams.size(); ++i) cudaStreamWaitEvent(b->streams[i], b->fork, 0);
        };
        auto join = [&]() {
            for (size_t i = 0; i < b->streams.size(); ++i) {
                cudaEventRecord(b->joins[i], b->streams[i]);
                cudaStreamWaitEvent(b->origin, b->joins[i], 0);
            }
        };
        std::vector<SolveArgs> args(n);
        fork();
        for (int q = 0; q < 5 && !err; ++q) {
            for (int k = 0; k < n && !err; ++k) {
                ppl_cpd* h = b->hs[k];
                cudaStream_t keep = h->st;
                h->st = b->streams[k % b->streams.size()];
                err = sweep_phase(h, q);
                h->st = keep;
                if (err) g_err = h->err;
            }
            if (q == 4 || err) break;
            join();
            for (int k = 0; k < n; ++k) args[k] = solve_args(b->hs[k], q);
            const int r = solve_modes_batched(args.data(), n, b->origin);
            if (r != 0) {
                err = fail(nullptr, PPL_ECUDA, "batched solve launch failed (%d%s%s)", r, r <= -1000 ? ": " : "",
                           r <= -1000 ? cudaGetErrorString((cudaError_t)(-r - 1000)) : "");
                break;
            }
            fork();
        }
        join();
        cudaGraph_t gr = nullptr;
        ce = cudaStreamEndCapture(b->origin, &gr);
        if (err) {
            if (gr) cudaGraphDestroy(gr);
            return err;
        }
        if (ce != cudaSuccess) return fail(nullptr, PPL_ECUDA, "batch end capture: %s", cudaGetErrorString(ce));
        long long saved = 0;
        const int ge = group_contractions(gr, &saved);
        if (ge != 0) {
            cudaGraphDestroy(gr);
            cudaGetLastError();
            return fail(nullptr, PPL_ECUDA, "batch: grouping the contractions failed (%d)", ge);
        }
        ce = cudaGraphInstantiate(&b->exec, gr, 0);
        if (ce != cudaSuccess) {
            cudaGraphDestroy(gr);
            return fail(nullptr, PPL_ECUDA, "batch instantiate: %s", cudaGetErrorString(ce));
        }
        b->graph = gr;
        b->ready = true;
        size_t nn = 0;
        cudaGraphGetNodes(gr, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn) cudaGraphGetNodes(gr, nodes.data(), &nn);
        b->kernels = 0;
        for (size_t q = 0; q < nn; ++q) {
            cudaGraphNodeType t;
            cudaGraphNodeGetType(nodes[q], &t);
            if (t == cudaGraphNodeTypeKernel) ++b->kernels;
        }
    }
    for (int s = 0; s < nsweeps; ++s) {
        if (cudaGraphLaunch(b->exec, b->origin) != cudaSuccess)
            return fail(nullptr, PPL_ECUDA, "batch launch: %s", cudaGetErrorString(cudaGetLastError()));
        if (fits || s == nsweeps - 1) {
            if (cudaStreamSynchronize(b->origin) != cudaSuccess)
                return fail(nullptr, PPL_ECUDA, "batch sync: %s", cudaGetErrorString(cudaGetLastError()));
            for (int k = 0; k < n; ++k) {
                ppl_cpd* h = b->hs[k];
                unsigned int flag = 0;
                cudaMemcpy(&flag, h->errflag(), sizeof flag, cudaMemcpyDeviceToHost);
                if (flag) {
                    cudaMemset(h->errflag(), 0, sizeof flag);
                    h->ntimeouts++;
                    return fail(nullptr, PPL_ETIMEOUT, "instance %d: a bounded device wait expired (0x%x)", k, flag);
                }
                double hist[4];
                cudaMemcpy(hist, h->at<double>(h->L.hist), sizeof hist, cudaMemcpyDeviceToHost);
                for (int q = 0; q < 4; ++q) h->last_hist[q] = hist[q];
                if (fits) fits[(size_t)s * n + k] = hist[0];
            }
        }
        for (int k = 0; k < n; ++k) b->hs[k]->sweeps++;
    }
    cudaEventRecord(b->ev_out, b->origin);
    cudaStreamWaitEvent(b->user, b->ev_out, 0);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, PPL_ECUDA, "batch: %s", cudaGetErrorString(e));
    return PPL_OK;
}

int ppl_cpd_batch_kernels(ppl_cpd_batch* b, long long* kernels_per_sweep) {
    if (!b || !kernels_per_sweep) return fail(nullptr, PPL_EINVAL, "NULL argument");
    *kernels_per_sweep = b->ready ? b->kernels : 0;
    return PPL_OK;
}

int ppl_cpd_batch_destroy(ppl_cpd_batch* b) {
    if (b)
        for (ppl_cpd* h : b->hs)
            if (h) {
                h->solve_cap = 0;
                h->tc_cap = 0;
            }
    if (!b) return PPL_OK;
    if (b->origin) cudaStreamSynchronize(b->origin);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
    if (b->origin) cudaStreamDestroy(b->origin);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    delete b;
    return PPL_OK;
}

int ppl_cpd_destroy(ppl_cpd* h) {
    if (!h) return PPL_OK;
    cudaStreamSynchronize(h->st);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    cudaStreamDestroy(h->st);
    cudaEventDestroy(h->ev_in);
    cudaEventDestroy(h->ev_out);
    if (h->have_pev)
        for (int k = 0; k < 9; ++k) cudaEventDestroy(h->pev[k]);
    delete h;
    return PPL_OK;
}

int ppl_cpd_phase_ms(ppl_cpd* h, double* ms) {
    if (!h || !ms) return fail(h, PPL_EINVAL, "NULL argument");
    if (!h->have_pev || h->sweeps == 0) return fail(h, PPL_ENOTREADY, "profiling off or no sweep has run");
    cudaStreamSynchronize(h->st);
    for (int k = 0; k < 8; ++k) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, h->pev[k], h->pev[k + 1]) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, PPL_ECUDA, "event timing failed");
        }
        ms[k] = t;
    }
    return PPL_OK;
}

int ppl_tc_gemm_workspace_size(int M, int N, int K, int precision, size_t* bytes) {
    if (!bytes || M < 1 || N < 1 || K < 1 ||
        (precision != PPL_PREC_BF16X3 && precision != PPL_PREC_TF32 && precision != PPL_PREC_TF32X3))
        return fail(nullptr, PPL_EINVAL, "bad arguments");
    const long long ld = rup(K, 8);
    const long long eb = precision == PPL_PREC_TF32X3 ? 8 : 4;
    *bytes = (size_t)rup((long long)M * ld * eb, 256) + (size_t)rup((long long)N * ld * eb, 256) + 256;
    return PPL_OK;
}

int ppl_tc_gemm(int precision, int M, int N, int K, const float* A, const float* B, float* C, void* workspace,
                size_t ws_bytes, void* stream) {
    size_t need = 0;
    int e = ppl_tc_gemm_workspace_size(M, N, K, precision, &need);
    if (e) return e;
    if (!A || !B || !C || !workspace) return fail(nullptr, PPL_EINVAL, "NULL device pointer");
    if (ws_bytes < need) return fail(nullptr, PPL_ENOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, need);
    if (((uintptr_t)workspace) % 256) return fail(nullptr, PPL_EINVAL, "workspace not 256-byte aligned");
    if (tc_init_driver() != 0) return fail(nullptr, PPL_ECUDA, "cuTensorMapEncodeTiled unavailable");
    cudaStream_t s = (cudaStream_t)stream;
    const long long ld = rup(K, 8);
    const long long eb = precision == PPL_PREC_TF32X3 ? 8 : 4;
    char* w = (char*)workspace;
    void* Aop = w;
    void* Bop = w + rup((long long)M * ld * eb, 256);
    unsigned int* flag = (unsigned int*)(w + rup((long long)M * ld * eb, 256) + rup((long long)N * ld * eb, 256));
    cudaMemsetAsync(flag, 0, sizeof(unsigned int), s);
    SplitSrc sa{};
    sa.src32 = A; sa.rmap = ix1(K); sa.cmap = ix1(1);
    split_to_operand(precision, sa, M, K, 1, Aop, (long long)M * ld, ld, 0, s);
    SplitSrc sb{};
    sb.src32 = B; sb.rmap = ix1(K); sb.cmap = ix1(1);
    split_to_operand(precision, sb, N, K, 1, Bop, (long long)N * ld, ld, 0, s);
    TcGemm g{};
    g.prec = precision;
    g.A = mat(Aop, (long long)M * ld, M, K, 1, ld, 0);
    g.B = mat(Bop, (long long)N * ld, N, K, 1, ld, 0);
    g.M = M; g.N = N; g.K = K; g.batch = 1; g.ksplit = 1;
    g.kchunk = precision == PPL_PREC_TF32X3 ? 1 : 0;
    g.out = TcOut{};
    {
        const int ke = panel_width(precision);
        g.out.kind = EPI_F32; g.out.out = C; g.out.alpha = 1.0f;
        g.out.q0p = (long long)ke * N; g.out.q0s = N;    // row m at m * N
        g.out.np = ke; g.out.ns = 1;                       // column n at n
    }
    g.bn = bn_for(N);
    int r = tc_gemm(g, flag, s);
    if (r)
        return fail(nullptr, PPL_ECUDA, "tensor-core GEMM launch failed (%d%s%s)", r, r <= -1000 ? ": " : "",
                    r <= -1000 ? cudaGetErrorString((cudaError_t)(-r - 1000)) : "");
    cudaError_t ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return fail(nullptr, PPL_ECUDA, "%s", cudaGetErrorString(ce));
    unsigned int f = 0;
    cudaMemcpy(&f, flag, sizeof f, cudaMemcpyDeviceToHost);
    if (f) return fail(nullptr, PPL_ETIMEOUT, "a bounded device wait expired (flags 0x%x)", f);
    return PPL_OK;
}

}  // extern "C"

// One ALS mode update in a single cooperative FP64 kernel (Optimizing the
// CP-PPL tensor-network section: W as the Hadamard product of the other
// three Gram matrices, a Cholesky solve of the normal equations, column
// normalisation; then the new factor's Gram matrix for the next updates).
//
//   P0  V = G1 .* G2 .* G3 (lower triangle), Z = M, tol = max(2^-52 R max V_kk, 1e-300)
//   P1  right-looking blocked Cholesky of V (32-wide blocks, pivots clamped at tol;
//       panels by warp-per-row triangular solves with the column-scaled diagonal block)
//       with the rows of Z appended below V, so the same panel and trailing updates
//       carry out the forward substitution Z <- M L^-T; the next diagonal block is
//       updated by three blocks (one lower quarter each) and factored by block 0
//       while the others update the rest
//   P2  back substitution U~ L = Z: the rows are independent, so every block solves
//       its own rows over all column blocks with no grid barrier (one warp per
//       column block in turn, all eight warps for the updates left of it)
//   P3  lam_r = ||U~[:, r]||, U = U~ / lam (a zero column keeps lam = 0)
//   P4  G = U^T U
//
// GB300 executes about two FP64 FMAs per clock per SM, so every phase is
// spread over all SMs in 32 x 32 tiles and 8-row panels; phases are separated
// by grid barriers (a cooperative launch guarantees co-residency).  Every
// barrier wait is bounded: on expiry the kernel raises an abort flag that
// all blocks observe, records the error and returns.
#include "ppl_internal.h"

#include <algorithm>

#include <cmath>

namespace {

constexpr int NB = 32;
constexpr int NT = 256;
constexpr unsigned long long BAR_NS = 1000ull * 1000ull * 1000ull;   // 1 s per barrier wait

struct SolveP {
    const double* G1;
    const double* G2;
    const double* G3;
    double* V;
    double* Linv;
    const double* M;
    double* Z;
    double* U;
    double* lam;
    double* G;
    unsigned int* sync;              // [0] arrivals, [1] generation, [2] abort
    unsigned long long* maxdiag;
    unsigned long long* nclamp;
    unsigned int* err;
    unsigned int* withhold;          // != 0: block 1 skips its first barrier arrival (once)
    unsigned long long wait_ns;      // bound of every barrier wait
    int R, dim;
};

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_vol(const unsigned int* p) { return *(volatile const unsigned int*)p; }

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned int atom_add_release(unsigned int* p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// grid-wide barrier; false when the wait expired or another block aborted.
// The block's writes are ordered before its arrival by __syncthreads and the
// release of the arrival; the waiters' acquire loads order what follows.
__device__ bool gsync(const SolveP& p, unsigned int& gen, int* s_flag, int bid, int G) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        // the test of the bounded waits: block 1 withholds its first arrival, so
        // the other blocks' wait runs out; it waits (bounded) for their abort
        const bool withhold =
            bid == 1 && p.withhold && ld_vol(p.withhold) != 0u && atomicExch(p.withhold, 0u) != 0u;
        if (withhold) {
            const unsigned long long t0 = gtimer();
            while (!ld_vol(&p.sync[2]) && gtimer() - t0 < 4 * p.wait_ns) {
            }
            ok = 0;
        } else {
            const unsigned int arrived = atom_add_release(&p.sync[0], 1u) + 1u;
            if (arrived == (unsigned int)G) {
                atomicExch(&p.sync[0], 0u);
                atom_add_release(&p.sync[1], 1u);
            } else {
                const unsigned long long t0 = gtimer();
                while (ld_acquire(&p.sync[1]) == gen) {
                    if (ld_vol(&p.sync[2])) {
                        ok = 0;
                        break;
                    }
                    if (gtimer() - t0 > p.wait_ns) {
                        atomicExch(&p.sync[2], 1u);
                        atomicOr(p.err, 16u);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        gen += 1;
        if (ld_vol(&p.sync[2])) ok = 0;
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

__device__ __forceinline__ void tri_index(int t, int& I, int& J) {
    // t -> (I, J), I >= J, row-major over the lower triangle (an FP32 estimate,
    // corrected exactly below: the FP64 pipe is the solve's bottleneck)
    int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    while (i * (i + 1) / 2 > t) --i;
    I = i;
    J = t - i * (i + 1) / 2;
}

// Factor the kb x kb diagonal block held in Ls (lower) in place, clamping
// pivots at tol, and leave in Li the column-scaled factor the panel solves
// with.  All NT threads.
//
// GB300 issues an FP64 warp instruction at the same cost whether or not its
// lanes are masked, so the factorisation keeps the FP64 instruction count close
// to the useful work: right-looking on unscaled columns (with d_j the clamped
// pivot, A[i][c] -= A[i][j] A[c][j] / d_j, one reciprocal per column); at step
// j only the n(n+1)/2 active elements of the trailing triangle are enumerated,
// packed onto consecutive threads through the (row, col) table tri; square
// roots and column scalings follow in one parallel pass.

// 1/d for a positive normal d: the PTX approximate reciprocal refined by two
// Newton-Raphson steps x <- x + x (1 - d x), each squaring the relative error
// (within an ulp or two of the correctly rounded quotient).  Four FP64 FMAs
// instead of the longer IEEE division sequence on the factorisation's
// critical path.
__device__ __forceinline__ double recip_nr(double d) {
    double x;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(d));
    double e = fma(-d, x, 1.0);
    x = fma(x, e, x);
    e = fma(-d, x, 1.0);
    return fma(x, e, x);
}
__device__ void diag_factor(double (*Ls)[NB + 1], double (*Li)[NB + 1], double* rd, const unsigned short* tri,
                            int kb, double tol, unsigned long long* nclamp) {
    const int t = threadIdx.x;
    // the pivot of column j is clamped and inverted by thread 0 right after its
    // own update of that element in step j - 1 (the table puts the next diagonal
    // element on thread 0), so each step needs one barrier
    if (t == 0 && kb > 0) {
        double d = Ls[0][0];
        if (!(d > tol)) {
            d = tol;
            atomicAdd(nclamp, 1ull);
        }
        Ls[0][0] = d;
        rd[0] = recip_nr(d);
    }
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
        const int n = kb - j - 1;
        const int nel = n * (n + 1) / 2;
        if (t < nel) {
            const unsigned short ic = tri[t];
            const int ii = j + 1 + (ic >> 8), cc = j + 1 + (ic & 0xff);
            const double x = fma(-(Ls[ii][j] * rd[j]), Ls[cc][j], Ls[ii][cc]);
            if (t == 0) {
                double d = x;
                if (!(d > tol)) {
                    d = tol;
                    atomicAdd(nclamp, 1ull);
                }
                Ls[ii][cc] = d;
                rd[j + 1] = recip_nr(d);
            } else {
                Ls[ii][cc] = x;
            }
        }
        if (t + NT < nel) {
            const unsigned short ic = tri[t + NT];
            const int ii = j + 1 + (ic >> 8), cc = j + 1 + (ic & 0xff);
            Ls[ii][cc] = fma(-(Ls[ii][j] * rd[j]), Ls[cc][j], Ls[ii][cc]);
        }
        __syncthreads();
    }
    // L = A_unscaled * diag(1/sqrt(d)), L_jj = sqrt(d_j); rd <- 1 / L_jj
    if (t < kb) {
        const double sd = sqrt(Ls[t][t]);
        rd[t] = recip_nr(sd);
        Ls[t][t] = sd;
    }
    __syncthreads();
    {
        const int nl = kb * (kb - 1) / 2;    // strictly lower elements, row-major
        for (int e = t; e < nl; e += NT) {
            const unsigned short ic = tri[e];
            const int i = (ic >> 8) + 1, j = ic & 0xff;   // (i, j) with j < i
            Ls[i][j] *= rd[j];
        }
    }
    __syncthreads();
    // Li <- the column-scaled factor used by the panel's triangular solves:
    // Li[i][j] = L[i][j] / L[j][j] below the diagonal, Li[i][i] = 1 / L[i][i]
    for (int e = t; e < NB * NB; e += NT) {
        const int i = e / NB, j = e % NB;
        Li[i][j] = (i < kb && j < i) ? Ls[i][j] * rd[j] : ((i < kb && j == i) ? rd[i] : 0.0);
    }
    __syncthreads();
}

// load the lower kb x kb block of V at (k0, k0) into Ls, factor it, write L
// back to V and the column-scaled factor the panels solve with to Linv[k]
__device__ void factor_block(const SolveP& p, int k, double tol, double (*Ls)[NB + 1], double (*Li)[NB + 1],
                             double* rd, const unsigned short* tri, double (*Tw)[NB + 1]) {
    const int R = p.R, tid = threadIdx.x;
    const int k0 = k * NB, kb = min(NB, R - k0);
    for (int e = tid; e < NB * NB; e += NT) {
        const int i = e / NB, j = e % NB;
        Ls[i][j] = (i < kb && j <= i) ? __ldcg(p.V + (long long)(k0 + i) * R + k0 + j) : 0.0;
    }
    __syncthreads();
    diag_factor(Ls, Li, rd, tri, kb, tol, p.nclamp);
    for (int e = tid; e < kb * kb; e += NT) {
        const int i = e / kb, j = e % kb;
        if (j <= i) p.V[(long long)(k0 + i) * R + k0 + j] = Ls[i][j];
    }
    for (int e = tid; e < NB * NB; e += NT) p.Linv[(long long)k * NB * NB + e] = Li[e / NB][e % NB];
    __syncthreads();
}

constexpr int RB = 4;   // rows of U~ per back-substitution pass

// asynchronous global -> shared copies (cp.async), waited for by the issuing thread
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// one warp copies an NB x NB block (row-major, NB doubles per row) into dst
__device__ __forceinline__ void stage_block(const double* src, double (*dst)[NB + 1], int lane) {
#pragma unroll 8
    for (int q = 0; q < NB; ++q) cp_async8(&dst[q][lane], src + q * NB + lane);
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Zl[r][c + bs b] -= sum_q x[r][q] L[j0 + q][lane + c + bs b] for the NR rows and
// CB column blocks b of one warp (Zl and Ll point at the lane's column: Zl at
// Z[r0][lane], Ll at L[j0][lane]).  KEEP: one block, the result returned in acc
// instead of stored.
template <int NR, int CB, bool KEEP = false>
__device__ __forceinline__ void back_update(double* Zl, int R, const double* Ll, const double (*x)[NB], int c, int kb,
                                            int bs, double (*acc)[NR]) {
#pragma unroll
    for (int b = 0; b < CB; ++b)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[b][r] = __ldcg(Zl + (long long)r * R + c + b * bs);
#pragma unroll 4
    for (int q = 0; q < kb; ++q) {
        double l[CB];
#pragma unroll
        for (int b = 0; b < CB; ++b) l[b] = __ldcg(Ll + (long long)q * R + c + b * bs);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const double xv = x[r][q];
#pragma unroll
            for (int b = 0; b < CB; ++b) acc[b][r] = fma(-xv, l[b], acc[b][r]);
        }
    }
    if (!KEEP) {
#pragma unroll
        for (int b = 0; b < CB; ++b)
#pragma unroll
            for (int r = 0; r < NR; ++r) Zl[(long long)r * R + c + b * bs] = acc[b][r];
    }
}

// The kb unknowns of one column block for NR rows (one warp, lane = column):
// w holds the block of Z with every block to its right already subtracted; with
// the column-scaled diagonal block Ld (L_qt / L_tt below the diagonal, 1 / L_tt
// on it), x_q is final once the columns right of q are subtracted, then
// w_t -= x_q L_qt / L_tt for t < q.
template <int NR>
__device__ __forceinline__ void back_diag(const double (*Ld)[NB + 1], int kb, int lane, double* w) {
    const double dinv = (lane < kb) ? Ld[lane][lane] : 0.0;
#pragma unroll
    for (int r = 0; r < NR; ++r) w[r] = (lane < kb) ? w[r] * dinv : 0.0;
    for (int q = kb - 1; q > 0; --q) {
        const double lq = (lane < q) ? Ld[q][lane] : 0.0;
#pragma unroll
        for (int r = 0; r < NR; ++r) w[r] = fma(-__shfl_sync(0xffffffffu, w[r], q), lq, w[r]);
    }
}

// Rows r0 .. r0+NR-1 of the back substitution U~ L = Z, all NT threads of the
// block, column blocks from the last one down.  At step J the unknowns x_J are
// published in shared memory; warp (J-1) mod 8 subtracts x_J L[rows of J][block
// J-1] from block J-1, keeps the result in registers and solves it at once
// (x_{J-1}), while the seven other warps subtract x_J from blocks 0 .. J-2; one
// block barrier per step.  The diagonal block of J-1 was copied to shared memory
// (cp.async) by the same warp one step earlier; the published values and the
// staged blocks alternate between two buffers.
template <int NR>
__device__ void back_rows(const SolveP& p, int r0, double (*xs)[RB][NB], double (*lb0)[NB + 1], double (*lb1)[NB + 1]) {
    constexpr int NW = NT / 32, NO = NW - 1;
    // CB blocks per pass, so that a pass keeps 4 sums and CB loads per step of q
    // in flight also when NR is small
    constexpr int CB = (NR == 1) ? 4 : (NR == 2 ? 2 : 1);
    const int R = p.R;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int nt = (R + NB - 1) / NB;
    double* Zr = p.Z + (long long)r0 * R;
    auto publish = [&](int J, const double* w) {
        const int j0 = J * NB, kb = min(NB, R - j0);
        if (lane < kb) {
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                xs[J & 1][r][lane] = w[r];
                p.U[(long long)(r0 + r) * R + j0 + lane] = w[r];
            }
        }
    };
    {   // the last block has nothing to its right
        const int J = nt - 1, j0 = J * NB, kb = min(NB, R - j0);
        if (warp == J % NW) {
            stage_block(p.Linv + (long long)J * NB * NB, (J & 1) ? lb1 : lb0, lane);
            cp_async_wait_all();
            __syncwarp();
            double w[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) w[r] = (lane < kb) ? __ldcg(Zr + (long long)r * R + j0 + lane) : 0.0;
            back_diag<NR>((J & 1) ? lb1 : lb0, kb, lane, w);
            publish(J, w);
        }
        if (J >= 1 && warp == (J - 1) % NW) stage_block(p.Linv + (long long)(J - 1) * NB * NB, ((J - 1) & 1) ? lb1 : lb0, lane);
        __syncthreads();
    }
    for (int J = nt - 1; J >= 1; --J) {
        const int j0 = J * NB, kb = min(NB, R - j0);
        const double (*x)[NB] = xs[J & 1];
        const double* Ll = p.V + (long long)j0 * R + lane;     // L[j0 + q][lane + c] at q * R + c
        const int ow = (J - 1) % NW;
        if (J >= 2 && warp == (J - 2) % NW) stage_block(p.Linv + (long long)(J - 2) * NB * NB, (J & 1) ? lb1 : lb0, lane);
        if (warp == ow) {
            double w[1][NR];
            back_update<NR, 1, true>(Zr + lane, R, Ll, x, (J - 1) * NB, kb, 0, w);
            cp_async_wait_all();
            __syncwarp();
            back_diag<NR>(((J - 1) & 1) ? lb1 : lb0, NB, lane, w[0]);
            publish(J - 1, w[0]);
        } else {
            const int w7 = (warp - ow - 1 + NW) % NW;
            int Jc = w7;
            double acc[CB][NR];
            for (; Jc + NO * (CB - 1) < J - 1; Jc += NO * CB) back_update<NR, CB>(Zr + lane, R, Ll, x, Jc * NB, kb, NO * NB, acc);
            for (; Jc < J - 1; Jc += NO) back_update<NR, 1>(Zr + lane, R, Ll, x, Jc * NB, kb, NO * NB, acc);
        }
        __syncthreads();
    }
}

// One 32 x 32 tile of a block step's trailing update: C -= Pa Pb^T over the kb
// columns of the panel, C in the lower triangle of V (tiles below the next
// diagonal) or in Z (the appended rows).
struct TrailTile {
    const double* Pa;
    const double* Pb;
    double* C;
    int arows, brows;
    bool diag;      // a diagonal tile of V: only j <= i is updated
};

__device__ __forceinline__ TrailTile trail_tile(const SolveP& p, int tile, int k0, int kb, int ntri, int Tk, int dim) {
    const int R = p.R;
    TrailTile t;
    int i0, j0;
    if (tile < ntri) {
        int I, J;
        tri_index(tile, I, J);
        i0 = k0 + kb + I * NB;
        j0 = k0 + kb + J * NB;
        t.Pa = p.V + (long long)i0 * R + k0;
        t.arows = R - i0;
        t.C = p.V + (long long)i0 * R + j0;
        t.diag = (I == J);
    } else {
        const int tz = tile - ntri;
        const int Mb = tz / Tk, J = tz % Tk;
        i0 = Mb * NB;
        j0 = k0 + kb + J * NB;
        t.Pa = p.Z + (long long)i0 * R + k0;
        t.arows = dim - i0;
        t.C = p.Z + (long long)i0 * R + j0;
        t.diag = false;
    }
    t.brows = R - j0;
    t.Pb = p.V + (long long)j0 * R + k0;
    return t;
}

__device__ __forceinline__ bool trail_owns(const TrailTile& t, int i, int j) {
    return i < t.arows && j < t.brows && (!t.diag || j <= i);
}

// this thread's four elements of each operand tile and its four C values
__device__ __forceinline__ void trail_fetch(const TrailTile& t, int R, int kb, int tid, int tx, int ty, double* pa,
                                            double* pb, double* pc) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int e = tid + u * NT;
        const int i = e / NB, s2 = e % NB;
        pa[u] = (i < t.arows && s2 < kb) ? __ldcg(t.Pa + (long long)i * R + s2) : 0.0;
        pb[u] = (i < t.brows && s2 < kb) ? __ldcg(t.Pb + (long long)i * R + s2) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = ty + 16 * (u >> 1), j = tx + 16 * (u & 1);
        pc[u] = trail_owns(t, i, j) ? __ldcg(t.C + (long long)i * R + j) : 0.0;
    }
}

// this thread's two elements of each 32 x 16 operand of the Gram tile at (i0, j0)
// (16 x 16 tiles of the lower triangle), rows x0 .. x0+31 of U
__device__ __forceinline__ void gram_fetch(const SolveP& p, int i0, int j0, int x0, int tid, double* qa, double* qb) {
    constexpr int T16 = 16;
    const int R = p.R, dim = p.dim;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int e = tid + u * NT;
        const int x = e / T16, c = e % T16;
        const bool okx = (x0 + x < dim);
        qa[u] = (okx && i0 + c < R) ? __ldcg(p.U + (long long)(x0 + x) * R + i0 + c) : 0.0;
        qb[u] = (okx && j0 + c < R) ? __ldcg(p.U + (long long)(x0 + x) * R + j0 + c) : 0.0;
    }
}

// One mode update of one instance, run by blocks bid = 0 .. G-1 (of one launch,
// or of one instance's share of a batched launch); the barriers count G blocks.
__device__ __forceinline__ void solve_body(const SolveP& p, const int bid, const int G) {
    __shared__ double Ls[NB][NB + 1];
    __shared__ double Li[NB][NB + 1];
    __shared__ double Ta[NB][NB + 1];
    __shared__ double Tb[NB][NB + 1];
    __shared__ double rd[NB];
    __shared__ double red[NT / 32];
    __shared__ unsigned short tri[NB * (NB + 1) / 2];   // (row << 8) | col of the lower triangle, row-major
    __shared__ int s_flag;
    __shared__ unsigned int s_gen;

    const int R = p.R, dim = p.dim;
    const int tid = threadIdx.x;
    const long long gtid = (long long)bid * NT + tid;
    const long long gthreads = (long long)G * NT;
    if (tid == 0) s_gen = ld_vol(&p.sync[1]);
    for (int i = 0, e = 0; i < NB; ++i)
        for (int c = 0; c <= i; ++c, ++e)
            if (e % NT == tid) tri[e] = (unsigned short)((i << 8) | c);
    __syncthreads();
    unsigned int gen = s_gen;   // meaningful in thread 0 only
    const int kb0 = min(NB, R);

    // ---- P0 --------------------------------------------------------------------
    // every block forms the pivot tolerance from the diagonal of V itself
    double mx = 0.0;
    for (int i = tid; i < R; i += NT) {
        const long long d = (long long)i * R + i;
        mx = fmax(mx, p.G1[d] * p.G2[d] * p.G3[d]);
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (tid % 32 == 0) red[tid / 32] = mx;
    __syncthreads();
    mx = red[0];
    for (int w = 1; w < NT / 32; ++w) mx = fmax(mx, red[w]);
    const double tol = fmax(ldexp(1.0, -52) * (double)R * mx, 1e-300);
    __syncthreads();
    for (long long e = gtid; e < (long long)R * R; e += gthreads) {
        const int r = (int)(e / R), q = (int)(e % R);
        if (q <= r && !(r < kb0 && q < kb0)) p.V[e] = p.G1[e] * p.G2[e] * p.G3[e];
    }
    for (long long e = gtid; e < (long long)dim * R; e += gthreads) p.Z[e] = p.M[e];
    if (bid == 0) {
        // the first diagonal block straight from the Gram matrices
        for (int e = tid; e < kb0 * kb0; e += NT) {
            const int i = e / kb0, j = e % kb0;
            if (j <= i) {
                const long long d = (long long)i * R + j;
                p.V[d] = p.G1[d] * p.G2[d] * p.G3[d];
            }
        }
        __syncthreads();
        factor_block(p, 0, tol, Ls, Li, rd, tri, Tb);
    }
    if (!gsync(p, gen, &s_flag, bid, G)) return;

    const int nt = (R + NB - 1) / NB;
    const int D = (dim + NB - 1) / NB;
    const int tx = tid % 16, ty = tid / 16;

    // ---- P1: Cholesky with the forward substitution fused, one block of look-ahead
    for (int k = 0; k < nt; ++k) {
        const int k0 = k * NB, kb = min(NB, R - k0);
        for (int e = tid; e < NB * NB; e += NT) Li[e / NB][e % NB] = __ldcg(p.Linv + (long long)k * NB * NB + e);
        __syncthreads();
        // panel: rows below the block (V) and all rows of Z, 8 rows per task
        const int vrows = R - k0 - kb;
        const int prow = vrows + dim;                // V rows below the block, then the rows of Z
        // one warp per row solves x L^T = a: with val_q final, x_q = val_q / L_qq
        // and val_t -= val_q (L_tq / L_qq), so each column costs one FMA
        const int ntask = (prow + 7) / 8;
        for (int task = bid; task < ntask; task += G) {
            const int rr = task * 8 + tid / NB, t = tid % NB;
            double* row = nullptr;
            if (rr < vrows)
                row = p.V + (long long)(k0 + kb + rr) * R + k0;
            else if (rr < prow)
                row = p.Z + (long long)(rr - vrows) * R + k0;
            if (row) {   // warp-uniform: rr is the same for the 32 lanes
                double val = (t < kb) ? __ldcg(row + t) : 0.0;
                for (int q = 0; q < kb; ++q) {
                    const double yq = __shfl_sync(0xffffffffu, val, q);
                    if (t > q) val = fma(-yq, Li[t][q], val);
                }
                if (t < kb) row[t] = val * Li[t][t];
            }
        }
        if (!gsync(p, gen, &s_flag, bid, G)) return;
        // trailing update of V (lower tiles) and of Z.  Tile 0 is the next
        // diagonal block: block 0 updates it and factors it while the other
        // blocks take the remaining tiles.
        const int Tk = (vrows + NB - 1) / NB;
        const int ntri = Tk * (Tk + 1) / 2;
        const int ntile = ntri + D * Tk;
        // With three or more blocks, tile 0 (the next diagonal block) is split:
        // blocks 0, 1, 2 each update one of its three lower 16 x 16 quarters,
        // blocks 1 and 2 then signal block 0, which factors the block once both
        // quarters have landed.  Block 0 takes no other tile.
        const bool split0 = (G >= 3 && k + 1 < nt && ntile > 0);
        if (split0 && bid < 3) {
            const int q = bid;
            const int d0 = k0 + kb, nb1 = min(NB, R - d0);
            const int r0 = (q == 0) ? 0 : 16, c0 = (q == 2) ? 16 : 0;
            const double* Pd = p.V + (long long)d0 * R + k0;     // rows of the panel at the next block
            for (int e = tid; e < 16 * NB; e += NT) {
                const int i = e / NB, s2 = e % NB;
                Ta[i][s2] = (r0 + i < nb1 && s2 < kb) ? __ldcg(Pd + (long long)(r0 + i) * R + s2) : 0.0;
                Tb[i][s2] = (c0 + i < nb1 && s2 < kb) ? __ldcg(Pd + (long long)(c0 + i) * R + s2) : 0.0;
            }
            __syncthreads();
            const int ti = tid / 16, tj = tid % 16;
            double acc = 0.0;
            for (int s2 = 0; s2 < kb; ++s2) acc = fma(Ta[ti][s2], Tb[tj][s2], acc);
            const int i = r0 + ti, j = c0 + tj;
            if (i < nb1 && j <= i) {
                double* c = p.V + (long long)(d0 + i) * R + d0 + j;
                *c = __ldcg(c) - acc;
            }
            __syncthreads();
            if (q > 0) {
                if (tid == 0) atom_add_release(&p.sync[3], 1u);
            } else {
                if (tid == 0) {
                    int ok = 1;
                    const unsigned int target = 2u * (unsigned int)(k + 1);
                    const unsigned long long t0 = gtimer();
                    while (ld_acquire(&p.sync[3]) < target) {
                        if (ld_vol(&p.sync[2])) {
                            ok = 0;
                            break;
                        }
                        if (gtimer() - t0 > p.wait_ns) {
                            atomicExch(&p.sync[2], 1u);
                            atomicOr(p.err, 64u);
                            ok = 0;
                            break;
                        }
                    }
                    s_flag = ok;
                }
                __syncthreads();
                if (s_flag) factor_block(p, k + 1, tol, Ls, Li, rd, tri, Tb);
            }
        }
        int first, stride;
        if (G == 1) {
            first = 0;
            stride = 1;
        } else if (bid == 0) {
            first = split0 ? ntile : 0;   // tile 0 only, unless split above
            stride = ntile + 1;
        } else {
            first = bid;
            stride = G - 1;
        }
        // each block's tiles in turn; the operands and the C values of the next
        // tile are loaded into registers while the current one is multiplied
        TrailTile cur{}, nxt{};
        double pa[4], pb[4], pc[4];
        int tile = first;
        if (tile < ntile) {
            cur = trail_tile(p, tile, k0, kb, ntri, Tk, dim);
            trail_fetch(cur, R, kb, tid, tx, ty, pa, pb, pc);
        }
        for (; tile < ntile; tile += stride) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = tid + u * NT;
                Ta[e / NB][e % NB] = pa[u];
                Tb[e / NB][e % NB] = pb[u];
            }
            double c4[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) c4[u] = pc[u];
            __syncthreads();
            if (tile + stride < ntile) {
                nxt = trail_tile(p, tile + stride, k0, kb, ntri, Tk, dim);
                trail_fetch(nxt, R, kb, tid, tx, ty, pa, pb, pc);
            }
            double a00 = 0, a01 = 0, a10 = 0, a11 = 0;
            for (int s2 = 0; s2 < kb; ++s2) {
                const double x0 = Ta[ty][s2], x1 = Ta[ty + 16][s2];
                const double y0 = Tb[tx][s2], y1 = Tb[tx + 16][s2];
                a00 = fma(x0, y0, a00);
                a01 = fma(x0, y1, a01);
                a10 = fma(x1, y0, a10);
                a11 = fma(x1, y1, a11);
            }
            const double acc[4] = {a00, a01, a10, a11};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = ty + 16 * (u >> 1), j = tx + 16 * (u & 1);
                if (trail_owns(cur, i, j)) cur.C[(long long)i * R + j] = c4[u] - acc[u];
            }
            __syncthreads();
            if (tile == 0 && k + 1 < nt && !split0) factor_block(p, k + 1, tol, Ls, Li, rd, tri, Tb);
            cur = nxt;
        }
        if (!gsync(p, gen, &s_flag, bid, G)) return;
    }

    // ---- P2: back substitution U~ L = Z, RB rows at a time ------------------------
    {
        __shared__ double xs[2][RB][NB];
        const int rpc = (dim + G - 1) / G;
        const int rbeg = bid * rpc, rend = min(dim, rbeg + rpc);
        for (int r0 = rbeg; r0 < rend; r0 += RB) {
            switch (min(RB, rend - r0)) {
                case 4: back_rows<4>(p, r0, xs, Ls, Li); break;
                case 3: back_rows<3>(p, r0, xs, Ls, Li); break;
                case 2: back_rows<2>(p, r0, xs, Ls, Li); break;
                default: back_rows<1>(p, r0, xs, Ls, Li); break;
            }
        }
    }
    constexpr int T16 = 16;
    const int ty16 = tid / T16, tx16 = tid % T16;
    if (!gsync(p, gen, &s_flag, bid, G)) return;

    // ---- P3: normalise: 32 columns per block, 8 row groups, a zero column keeps lam = 0
    {
        const int c = tid % 32, rg = tid / 32;
        for (int cb = bid; cb * 32 < R; cb += G) {
            const int r = cb * 32 + c;
            double s = 0.0;
            if (r < R)
                for (int x = rg; x < dim; x += NT / 32) {
                    const double u = __ldcg(p.U + (long long)x * R + r);
                    s = fma(u, u, s);
                }
            Ta[rg][c] = s;
            __syncthreads();
            if (rg == 0) {
                double t = 0.0;
                for (int q = 0; q < NT / 32; ++q) t += Ta[q][c];
                Tb[0][c] = t;
            }
            __syncthreads();
            if (r < R) {
                const double l = sqrt(Tb[0][c]);
                const double inv = (l > 0.0) ? 1.0 / l : 1.0;
                for (int x = rg; x < dim; x += NT / 32) p.U[(long long)x * R + r] = __ldcg(p.U + (long long)x * R + r) * inv;
                if (rg == 0) p.lam[r] = l;
            }
            __syncthreads();
        }
    }
    if (!gsync(p, gen, &s_flag, bid, G)) return;

    // ---- P4: Gram of the new factor, 16 x 16 tiles of the lower triangle ------------
    const int TR = (R + T16 - 1) / T16;
    const int ntri = TR * (TR + 1) / 2;
    // each block's (tile, 32-row step) pairs in turn, the next pair's operands
    // loaded into registers while the current one is multiplied
    {
        const int nx = (dim + NB - 1) / NB;
        int tile = bid, xs = 0;
        int ti0 = 0, tj0 = 0;              // the current tile's corner
        if (tile < ntri) {
            int I, J;
            tri_index(tile, I, J);
            ti0 = I * T16;
            tj0 = J * T16;
        }
        int ni0 = ti0, nj0 = tj0;          // the next pair's tile corner
        double qa[2], qb[2];
        if (tile < ntri) gram_fetch(p, ti0, tj0, 0, tid, qa, qb);
        double acc = 0.0;
        while (tile < ntri) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int e = tid + u * NT;
                Ta[e / T16][e % T16] = qa[u];
                Tb[e / T16][e % T16] = qb[u];
            }
            __syncthreads();
            int ntl = tile, nxs = xs + 1;
            if (nxs == nx) {
                ntl += G;
                nxs = 0;
                if (ntl < ntri) {
                    int I, J;
                    tri_index(ntl, I, J);
                    ni0 = I * T16;
                    nj0 = J * T16;
                }
            }
            if (ntl < ntri) gram_fetch(p, ni0, nj0, nxs * NB, tid, qa, qb);
#pragma unroll 8
            for (int x = 0; x < NB; ++x) acc = fma(Ta[x][ty16], Tb[x][tx16], acc);
            __syncthreads();
            if (nxs == 0) {
                const int i = ti0 + ty16, j = tj0 + tx16;
                if (i < R && j < R) {
                    p.G[(long long)i * R + j] = acc;
                    p.G[(long long)j * R + i] = acc;
                }
                acc = 0.0;
            }
            tile = ntl;
            xs = nxs;
            ti0 = ni0;
            tj0 = nj0;
        }
    }
}

__global__ void __launch_bounds__(NT, 1) k_solve(const __grid_constant__ SolveP p) { solve_body(p, blockIdx.x, gridDim.x); }

// Several instances' mode updates in one cooperative launch.  The blocks form
// lanes: lane l is blocks lane_blk0[l] .. lane_blk0[l+1]-1 and solves the
// instances order[lane_inst0[l]] .. order[lane_inst0[l+1]-1] one after the
// other, each with its own barrier words, so the lanes proceed independently
// and only share the SMs.
constexpr int MAX_BATCH = 64;
struct SolveBatch {
    int n, nl;
    int lane_blk0[MAX_BATCH + 1];
    int lane_inst0[MAX_BATCH + 1];
    int order[MAX_BATCH];
    SolveP p[MAX_BATCH];
};

__global__ void __launch_bounds__(NT, 3) k_solve_batch(const __grid_constant__ SolveBatch b) {
    int l = 0;
    while (l + 1 < b.nl && b.lane_blk0[l + 1] <= (int)blockIdx.x) ++l;
    const int bid = (int)blockIdx.x - b.lane_blk0[l], G = b.lane_blk0[l + 1] - b.lane_blk0[l];
    for (int i = b.lane_inst0[l]; i < b.lane_inst0[l + 1]; ++i) {
        solve_body(b.p[b.order[i]], bid, G);
        __syncthreads();   // the block's shared memory is reused by the next instance
    }
}

// the barrier words and the diagonal maximum of every instance start at zero
__global__ void k_solve_batch_prep(const __grid_constant__ SolveBatch b) {
    const int k = threadIdx.x;
    if (k < b.n) {
        for (int w = 0; w < 4; ++w) b.p[k].sync[w] = 0u;
        *b.p[k].maxdiag = 0ull;
    }
}

int g_solve_grid = 0;

}  // namespace

namespace {

SolveP to_params(const SolveArgs& a) {
    SolveP p;
    p.G1 = a.G1; p.G2 = a.G2; p.G3 = a.G3; p.V = a.V; p.Linv = a.Linv; p.M = a.M; p.Z = a.Z;
    p.U = a.U; p.lam = a.lam; p.G = a.G;
    p.sync = a.sync; p.maxdiag = a.maxdiag; p.nclamp = a.nclamp; p.err = a.err; p.R = a.R; p.dim = a.dim;
    p.withhold = a.withhold;
    p.wait_ns = a.wait_ns > 0 ? a.wait_ns : BAR_NS;
    return p;
}

int sm_total() {
    if (g_solve_grid == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) return -1;
        g_solve_grid = sms;   // one block per SM: the look-ahead block keeps its SM's FP64 pipe
    }
    return g_solve_grid;
}

// blocks one instance can use: enough for the first block step's tiles and panel
// rows, at least 8, at most one per SM
int solve_want(int dim, int R, int sms) {
    const int t0 = (R > NB) ? (R - NB + NB - 1) / NB : 0;
    const int d = (dim + NB - 1) / NB;
    int want = t0 * (t0 + 1) / 2 + d * t0;
    const int ptask = (R + dim + 7) / 8;
    if (ptask > want) want = ptask;
    if (want < 8) want = 8;
    return want < sms ? want : sms;
}

int g_batch_per_sm = 0;

}  // namespace

int solve_mode_coop(const double* G1, const double* G2, const double* G3, const double* M, int dim, int R,
                    double* V, double* Linv, double* Z, double* U, double* lam, double* G,
                    unsigned int* sync, unsigned long long* maxdiag, unsigned long long* nclamp, unsigned int* err,
                    int grid_cap, unsigned long long wait_ns, unsigned int* withhold, cudaStream_t s) {
    const int sms = sm_total();
    if (sms <= 0) return -1;
    // small problems take fewer blocks, so that several instances' solves can share the GPU
    int grid = solve_want(dim, R, sms);
    if (grid_cap > 0 && grid > grid_cap) grid = grid_cap < 8 ? 8 : grid_cap;
    cudaMemsetAsync(sync, 0, 4 * sizeof(unsigned int), s);
    cudaMemsetAsync(maxdiag, 0, sizeof(unsigned long long), s);
    SolveArgs a{G1, G2, G3, M, dim, R, V, Linv, Z, U, lam, G, sync, maxdiag, nclamp, err, wait_ns, withhold};
    const SolveP p = to_params(a);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_solve, p);
    return e == cudaSuccess ? 0 : -(1000 + (int)e);
}

int solve_modes_batched(const SolveArgs* a, int n, cudaStream_t s) {
    const int sms = sm_total();
    if (sms <= 0) return -1;
    if (g_batch_per_sm == 0) {
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_solve_batch, NT, 0) != cudaSuccess || per <= 0) {
            cudaGetLastError();
            return -2;
        }
        g_batch_per_sm = per;
    }
    const int cap = g_batch_per_sm * sms;   // blocks that are co-resident in one cooperative launch
    for (int k0 = 0; k0 < n; k0 += MAX_BATCH) {
        const int nb = (n - k0 < MAX_BATCH) ? n - k0 : MAX_BATCH;
        if (2 * nb > cap) return -3;
        SolveBatch b;
        b.n = nb;
        int want[MAX_BATCH];
        double work[MAX_BATCH], steps[MAX_BATCH];
        for (int k = 0; k < nb; ++k) {
            const SolveArgs& x = a[k0 + k];
            want[k] = solve_want(x.dim, x.R, sms);
            work[k] = (double)x.R * x.R * x.R / 3.0 + 4.0 * x.dim * (double)x.R * x.R;
            steps[k] = (double)((x.R + NB - 1) / NB);
            b.p[k] = to_params(x);
        }
        // Lanes: L lanes of cap / L blocks; each instance goes to one lane, longest
        // first to the least loaded.  Modelled time of an instance on G blocks: its
        // FP64 work at G blocks' share of the FP64 rate (2 FMA per clock per SM at
        // about 2 GHz, shared by the blocks of an SM) plus a latency per 32-wide
        // block step; L is the one with the shortest modelled makespan.
        const double rate_blk = 8.0e9 / g_batch_per_sm, step_s = 20e-6;
        auto est = [&](int k, int G) { return work[k] / ((double)(G < want[k] ? G : want[k]) * rate_blk) + steps[k] * step_s; };
        int best_L = 0, best_lane[MAX_BATCH] = {};
        double best_span = 0.0;
        for (int L = 1; L <= nb; ++L) {
            const int W = cap / L;
            if (W < 2) break;
            int idx[MAX_BATCH], lane[MAX_BATCH];
            double t[MAX_BATCH], load[MAX_BATCH];
            for (int k = 0; k < nb; ++k) {
                idx[k] = k;
                t[k] = est(k, W);
            }
            std::sort(idx, idx + nb, [&](int x, int y) { return t[x] > t[y]; });
            for (int l = 0; l < L; ++l) load[l] = 0.0;
            for (int q = 0; q < nb; ++q) {
                int lmin = 0;
                for (int l = 1; l < L; ++l)
                    if (load[l] < load[lmin]) lmin = l;
                lane[idx[q]] = lmin;
                load[lmin] += t[idx[q]];
            }
            double span = 0.0;
            for (int l = 0; l < L; ++l) span = load[l] > span ? load[l] : span;
            if (best_L == 0 || span < best_span) {
                best_L = L;
                best_span = span;
                for (int k = 0; k < nb; ++k) best_lane[k] = lane[k];
            }
        }
        if (best_L == 0) return -3;
        b.nl = best_L;
        int blk = 0, q = 0;
        for (int l = 0; l < best_L; ++l) {
            b.lane_blk0[l] = blk;
            blk += cap / best_L + (l < cap % best_L ? 1 : 0);
            b.lane_inst0[l] = q;
            for (int k = 0; k < nb; ++k)
                if (best_lane[k] == l) b.order[q++] = k;
        }
        b.lane_blk0[best_L] = blk;
        b.lane_inst0[best_L] = q;
        k_solve_batch_prep<<<1, MAX_BATCH, 0, s>>>(b);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(blk);
        cfg.blockDim = dim3(NT);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const cudaError_t e = cudaLaunchKernelEx(&cfg, k_solve_batch, b);
        if (e != cudaSuccess) return -(1000 + (int)e);
    }
    return 0;
}

// ---- self-test of the pivot reciprocal --------------------------------------

namespace {

__global__ void k_recip_check(const double* d, double* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = recip_nr(d[i]);
}

}  // namespace

extern "C" int ppl_test_reciprocal(const double* d, double* out, int n, void* stream) {
    if (!d || !out || n < 0) return 1;   // PPL_EINVAL
    if (n == 0) return 0;
    k_recip_check<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(d, out, n);
    const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return 3;   // PPL_ECUDA
    return 0;
}

// Tensor-core contraction for the MTTKRP steps of the CP-ALS sweep on sm_103a.
//
// C[b][m][n] = sum_k A[b][m][k] B[b][n][k], both operands K-major in global
// memory, staged by TMA (128-byte swizzle, no multicast) into a ring of
// shared-memory stages and multiplied by tcgen05.mma with the FP32
// accumulator in tensor memory.  Two operand precisions:
//   BF16X3: x = hi + lo with hi = bf16(x), lo = bf16(x - hi); the product is
//           hi*hi + hi*lo + lo*hi (three MMAs into one accumulator), after
//           Henry, Tang & Heinecke, "Leveraging the bfloat16 artificial
//           intelligence datatype for higher-precision computations" (2019);
//           within each K block the cross products are issued before hi*hi;
//   TF32:   operands rounded to tf32 (round to nearest) when written, one MMA;
//   TF32X3: x = hi + lo with hi = tf32(x), lo = tf32(x - hi) (22 significant
//           bits, the FP32 exponent range), three kind::tf32 MMAs as above.
// The FP32 accumulator of tcgen05.mma rounds toward zero at every MMA, so a
// long sum drifts toward zero by about half an ulp per instruction.  With a
// positive kchunk the mainloop restarts the accumulator every kchunk K blocks
// (ping-ponging the two TMEM buffers) and the epilogue warps add the chunks in
// FP32 registers with round-to-nearest, which removes that bias.
// Persistent: one CTA per SM walks the 128 x bn output tiles.  Lane 0 of warp
// 0 issues TMA into a ring of shared-memory stages, lane 0 of warp 1 issues the
// MMAs into one of two TMEM accumulators, and warps 2..9 drain the other
// accumulator to global memory, so a tile's epilogue overlaps the next tile's
// mainloop.  Warp 2 owns the TMEM allocation.
// Every mbarrier wait is bounded; on expiry the kernel records the error,
// drains what it issued, frees TMEM and returns.
#include "ppl_internal.h"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/ppl_cpd.h"

namespace {

constexpr int TM = 128;               // rows of the accumulator tile (TMEM lanes)
constexpr int KROW_BYTES = 128;       // one swizzle row: 64 bf16 or 32 fp32
constexpr int SMEM_BUDGET = 200 * 1024;      // operand stages
constexpr int SMEM_ATTR = 220 * 1024;        // dynamic smem opt-in (stages + alignment + barriers)
constexpr unsigned long long WAIT_NS = 500ull * 1000ull * 1000ull;   // 0.5 s per wait
// Block layout: one control warpgroup (warp 0 issues TMA, warp 1 issues the
// MMAs, warp 2 owns the TMEM allocation, warp 3 idles) and two epilogue
// warpgroups, warps 4..11: two warps per TMEM lane quarter (a warp reads the 32
// lanes of its quarter, warp % 4), each draining one 128-column half of the tile
// as two 64-column slices.  With the accumulator restarted every K block an
// epilogue thread holds 128 running sums and loads 64 columns per TMEM round
// trip, more registers than a 384-thread block gives every thread, so the
// control warpgroup hands registers to the epilogue (setmaxnreg): 56 for it and
// 224 for each epilogue thread, 128*56 + 256*224 = 384*168, exactly the launch's
// allocation (checked on the host before every launch: a split above the
// allocation would wait forever).
constexpr int NCTRL = 4;                      // warps of the control warpgroup
constexpr int NEPI = 8;                       // epilogue warps
constexpr int NTHREADS = 32 * (NCTRL + NEPI);
constexpr int REG_LAUNCH = 168;               // registers per thread at launch (65536 / 384, rounded to 8)
constexpr int REG_CTRL = 56, REG_EPI = 224;
static_assert(32 * NCTRL * REG_CTRL + 32 * NEPI * REG_EPI == NTHREADS * REG_LAUNCH, "register split");
constexpr int SLW = 64;                       // columns per slice
constexpr int NSL = 2;                        // slices per epilogue warp (a 128-column half)

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

struct KParams {
    int M, N, K, bn, acc_cols, ksplit, nkb_total, per_split, stages;
    int a_row0, b_row0, a_b0, b_b0, a_bstep, b_bstep;
    int batch;
    int kind;
    void* out;
    long long plane, sb, sk, q1p, q1s, q0p, q0s, np, ns;
    int mdiv;
    float alpha;
    int kchunk;             // K blocks per accumulation chunk (drained kernels)
    int ksub;               // > 0: MMA K steps per accumulation chunk, splitting each K block
    int nfast;              // 1: consecutive tiles walk N first (one A tile shared by neighbours)
    int a_panel, b_panel;   // 1: the operand is in the K-panel layout (4-D tensor map)
    unsigned long long wait_ns;   // bound of every barrier wait
    unsigned int* err;
};

// One contraction: the tensor maps of A hi, A lo, B hi, B lo and its parameters.
struct TcArgs {
    CUtensorMap m[4];
    KParams p;
};
// Several independent contractions in one persistent launch (one CUDA graph
// node): the CTAs walk the concatenated tile lists; tile0[i] is the first tile
// of contraction i.  The shared-memory stages and the TMEM accumulators are laid
// out for the widest N tile of the group.
constexpr int TC_GROUP_MAX = 40;
struct TcGroupArgs {
    int n, bn_max, stages, acc_cols;
    unsigned long long wait_ns;
    int tile0[TC_GROUP_MAX + 1];
    CUtensorMap m[TC_GROUP_MAX][4];
    KParams p[TC_GROUP_MAX];
};
static_assert(sizeof(TcGroupArgs) <= 32000, "kernel parameter space");

// operand traits of the precisions
template <int PREC> struct Prec {
    static constexpr int PLANES = (PREC == PPL_PREC_BF16X3 || PREC == PPL_PREC_TF32X3) ? 2 : 1;
    static constexpr bool HALF = (PREC == PPL_PREC_BF16X3);   // 2-byte elements
    static constexpr int KE = HALF ? 64 : 32;                  // elements per 128-byte row
    static constexpr int KSTEP = HALF ? 16 : 8;                // K per MMA instruction
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: true when the phase completed, false after limit_ns
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, unsigned long long limit_ns) {
    if (mbar_try(a, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (true) {
        if (mbar_try(a, parity)) return true;
        if (gtimer() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
        : "memory");
}

// one operand tile: K block kb of rows row.. of batch entry b
__device__ __forceinline__ void load_op(uint32_t dst, const CUtensorMap* map, bool panel, int kb, int ke, int row, int b,
                                        uint32_t mbar) {
    if (panel)
        tma_load_4d(dst, map, 0, row, kb, b, mbar);
    else
        tma_load_3d(dst, map, kb * ke, row, b, mbar);
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ unsigned long long make_desc(uint32_t saddr) {
    unsigned long long d = 0;
    d |= (unsigned long long)((saddr & 0x3FFFFu) >> 4);
    d |= 1ull << 16;                       // leading byte offset (unused for swizzled K-major)
    d |= (unsigned long long)(1024 >> 4) << 32;   // stride byte offset
    d |= 1ull << 46;                       // descriptor version
    d |= 2ull << 61;                       // SWIZZLE_128B
    return d;
}

template <int PREC>
__device__ __forceinline__ void mma(uint32_t tmem, unsigned long long ad, unsigned long long bd, uint32_t idesc,
                                    uint32_t acc) {
    if constexpr (Prec<PREC>::HALF) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
}

// two FP32 values in one 64-bit register pair, added with one packed
// round-to-nearest instruction (the same rounding as two scalar adds)
__device__ __forceinline__ unsigned long long pack2(uint32_t a, uint32_t b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ void unpack2(unsigned long long x, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x));
}

// 64 accumulator columns as two 32-column loads (each into 32 consecutive
// registers, which the allocator finds more easily than one block of 64) and
// one wait
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&v)[64]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%64];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, "
        "%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%65];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]),
          "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]), "=r"(v[38]), "=r"(v[39]),
          "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]), "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]),
          "=r"(v[48]), "=r"(v[49]), "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]),
          "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]), "=r"(v[62]), "=r"(v[63])
        : "r"(taddr), "r"(taddr + 32u)
        : "memory");
}

__device__ __forceinline__ float round_tf32(float x) {
    uint32_t y;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
    return __uint_as_float(y);
}

// Column offsets of the 32 consecutive columns n0 .. n0 + 31 in the output:
// (n / PW) * np + (n % PW) * ns.  They span at most two panels (PW >= 32), so
// column j is at base + j * ns, plus jump once j reaches the next panel.
struct ColOff {
    long long base, ns, jump;
    int split;
};
template <int PREC>
__device__ __forceinline__ ColOff coloffs(const KParams& p, int n0) {
    constexpr int PW = Prec<PREC>::KE;
    ColOff c;
    c.base = (long long)(n0 / PW) * p.np + (long long)(n0 % PW) * p.ns;
    c.ns = p.ns;
    c.jump = p.np - (long long)PW * p.ns;
    c.split = PW - n0 % PW;
    return c;
}
__device__ __forceinline__ long long col_at(const ColOff& c, int j) {
    return c.base + (long long)j * c.ns + (j >= c.split ? c.jump : 0ll);
}

// the epilogue's store of 32 consecutive columns n0 .. n0 + 31 of one row
template <int PREC>
__device__ __forceinline__ void emit32(const KParams& p, long long mo, int n0, int nvalid, const float (&x)[32]) {
    const ColOff co = coloffs<PREC>(p, n0);
    if (p.kind == EPI_SPLIT) {
        if constexpr (PREC == PPL_PREC_BF16X3) {
            __nv_bfloat16* o = (__nv_bfloat16*)p.out + mo;
            __nv_bfloat16* ol = o + p.plane;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (j < nvalid) {
                    const long long c = col_at(co, j);
                    const __nv_bfloat16 hi = __float2bfloat16_rn(x[j]);
                    o[c] = hi;
                    ol[c] = __float2bfloat16_rn(x[j] - __bfloat162float(hi));
                }
            }
        } else if constexpr (PREC == PPL_PREC_TF32X3) {
            float* o = (float*)p.out + mo;
            float* ol = o + p.plane;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (j < nvalid) {
                    const long long c = col_at(co, j);
                    const float hi = round_tf32(x[j]);
                    o[c] = hi;
                    ol[c] = round_tf32(x[j] - hi);
                }
            }
        } else {
            float* o = (float*)p.out + mo;
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (j < nvalid) o[col_at(co, j)] = round_tf32(x[j]);
        }
    } else if (p.kind == EPI_F32) {
        float* o = (float*)p.out + mo;
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (j < nvalid) o[col_at(co, j)] = x[j];
    } else {
        double* o = (double*)p.out + mo;
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (j < nvalid) atomicAdd(o + col_at(co, j), (double)x[j]);
    }
}

// tiles of one contraction
__host__ __device__ __forceinline__ int tc_tiles(const KParams& p) {
    return ((p.M + TM - 1) / TM) * ((p.N + p.bn - 1) / p.bn) * p.batch * p.ksplit;
}

// The kernel body for nprob contractions: P[i] and the four maps M4[4 i .. 4 i + 3]
// of contraction i, whose tiles are tile0[i] .. tile0[i + 1] - 1 of the walk
// (tile0 == nullptr: one contraction).  Stages of bn_max-wide B tiles, S of them,
// and two TMEM accumulators of acc_cols_u columns serve every contraction.
template <int PREC, bool DRAIN>
__device__ __forceinline__ void tc_body(const KParams* P, const CUtensorMap* M4, const int* tile0, int nprob,
                                        int bn_max, int S, int acc_cols_u, unsigned long long wait_ns) {
    constexpr bool SPLIT = (Prec<PREC>::PLANES == 2);
    constexpr int KE = Prec<PREC>::KE;
    constexpr int KSTEP = Prec<PREC>::KSTEP;
    constexpr int ASTEP_BYTES = 32;           // one MMA's K slice of a 128-byte row

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int total = tile0 ? tile0[nprob] : tc_tiles(P[0]);
    // contraction of walk tile t and the tile's index inside it
    auto locate = [&](int t, int& lt) -> int {
        int pi = 0;
        if (tile0)
            while (pi + 1 < nprob && tile0[pi + 1] <= t) ++pi;
        lt = tile0 ? t - tile0[pi] : t;
        return pi;
    };

    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* gbase = smem_raw + (base - raw);

    const uint32_t a_bytes = TM * KROW_BYTES;
    const uint32_t b_bytes = (uint32_t)bn_max * KROW_BYTES;          // stage layout: the widest B tile
    const uint32_t stage_bytes = (SPLIT ? 2u : 1u) * (a_bytes + b_bytes);
    const uint32_t bar_off = stage_bytes * S;
    const uint32_t full0 = base + bar_off;
    const uint32_t empty0 = full0 + 8u * S;
    const uint32_t tfull0 = empty0 + 8u * S;     // 2 accumulators
    const uint32_t tempty0 = tfull0 + 16u;
    const uint32_t drain_bar = tempty0 + 16u;
    const uint32_t slot = drain_bar + 8u;
    volatile uint32_t* slot_ptr = (volatile uint32_t*)(gbase + (slot - base));
    __shared__ int s_fail;
    __shared__ int s_issued, s_consumed;

    const uint32_t acc_cols = (uint32_t)acc_cols_u;
    const uint32_t ncols = 2u * acc_cols;

    if (threadIdx.x == 0) {
        s_fail = 0;
        s_issued = 0;
        s_consumed = 0;
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8u * s, 1);
            mbar_init(empty0 + 8u * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull0 + 8u * b, 1);
            mbar_init(tempty0 + 8u * b, NEPI);
        }
        mbar_init(drain_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&M4[0]) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&M4[2]) : "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *slot_ptr;
    volatile int* vfail = &s_fail;
    // the control warpgroup gives registers to the two epilogue warpgroups (each
    // role's code is dominated by its own register count)
    if (warp < NCTRL) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(REG_CTRL) : "memory");
        if (warp == 0) {
            if (lane == 0) {
                // TMA producer: one ring of S stages shared by all tiles of this block
                int it = 0;
                for (int t = blockIdx.x; t < total && !*vfail; t += gridDim.x) {
                    int lt;
                    const int pi = locate(t, lt);
                    const KParams& p = P[pi];
                    const CUtensorMap* mp = M4 + 4 * pi;
                    const int ntm = (p.M + TM - 1) / TM, ntn = (p.N + p.bn - 1) / p.bn, tiles_mn = ntm * ntn;
                    const uint32_t tx_bytes = (SPLIT ? 2u : 1u) * (a_bytes + (uint32_t)p.bn * KROW_BYTES);
                    const int z = lt / tiles_mn, rem = lt % tiles_mn;
                    const int m0 = (p.nfast ? rem / ntn : rem % ntm) * TM, n0 = (p.nfast ? rem % ntn : rem / ntm) * p.bn;
                    const int bz = z / p.ksplit, ks = z % p.ksplit;
                    const int kb0 = ks * p.per_split;
                    const int nk = min(p.per_split, p.nkb_total - kb0);
                    const int a_b = p.a_b0 + bz * p.a_bstep, b_b = p.b_b0 + bz * p.b_bstep;
                    for (int kbi = 0; kbi < nk; ++kbi, ++it) {
                        const int s = it % S;
                        if (it >= S && !mbar_wait(empty0 + 8u * s, (uint32_t)((it / S - 1) & 1), wait_ns)) {
                            atomicOr(p.err, 1u);
                            *vfail = 1;
                            break;
                        }
                        const uint32_t sa = base + stage_bytes * s;
                        const uint32_t fb = full0 + 8u * s;
                        mbar_expect_tx(fb, tx_bytes);
                        const int kb = kb0 + kbi;
                        load_op(sa, &mp[0], p.a_panel, kb, KE, p.a_row0 + m0, a_b, fb);
                        load_op(sa + (SPLIT ? 2u : 1u) * a_bytes, &mp[2], p.b_panel, kb, KE, p.b_row0 + n0, b_b, fb);
                        if constexpr (SPLIT) {
                            load_op(sa + a_bytes, &mp[1], p.a_panel, kb, KE, p.a_row0 + m0, a_b, fb);
                            load_op(sa + 2u * a_bytes + b_bytes, &mp[3], p.b_panel, kb, KE, p.b_row0 + n0, b_b, fb);
                        }
                        s_issued = it + 1;
                    }
                }
            }
        } else if (warp == 1) {
            if (lane == 0) {
                // MMA issuer
                int it = 0, li = 0;   // li counts accumulation chunks (one per tile unless DRAIN)
                bool ok = true;
                for (int t = blockIdx.x; t < total && ok && !*vfail; t += gridDim.x) {
                    int lt;
                    const KParams& p = P[locate(t, lt)];
                    uint32_t idesc = (1u << 4) | ((uint32_t)p.bn >> 3 << 17) | ((uint32_t)(TM >> 4) << 24);
                    idesc |= Prec<PREC>::HALF ? ((1u << 7) | (1u << 10)) : ((2u << 7) | (2u << 10));
                    const int tiles_mn = ((p.M + TM - 1) / TM) * ((p.N + p.bn - 1) / p.bn);
                    const int z = lt / tiles_mn;
                    const int ks = z % p.ksplit;
                    const int kb0 = ks * p.per_split;
                    const int nk = min(p.per_split, p.nkb_total - kb0);
                    const int kch = DRAIN ? p.kchunk : nk;
                    if (DRAIN && p.ksub > 0) {
                        // each K block in chunks of ksub MMA K steps, one accumulator each
                        for (int kbi = 0; kbi < nk && ok; ++kbi, ++it) {
                            const int s = it % S;
                            if (!mbar_wait(full0 + 8u * s, (uint32_t)((it / S) & 1), wait_ns)) {
                                atomicOr(p.err, 2u);
                                *vfail = 1;
                                ok = false;
                                break;
                            }
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            const uint32_t sa = base + stage_bytes * s;
                            const uint32_t sah = sa, sal = sa + a_bytes;
                            const uint32_t sbh = sa + (SPLIT ? 2u : 1u) * a_bytes, sbl = sbh + b_bytes;
                            const int kc = (kb0 + kbi) * KE;
                            int ksteps = KE / KSTEP;
                            if (p.K - kc < KE) ksteps = (p.K - kc + KSTEP - 1) / KSTEP;
                            const unsigned long long dah = make_desc(sah), dbh = make_desc(sbh);
                            const unsigned long long dal = make_desc(sal), dbl = make_desc(sbl);
                            for (int kk0 = 0; kk0 < ksteps; kk0 += p.ksub, ++li) {
                                const int kk1 = min(ksteps, kk0 + p.ksub);
                                const int buf = li & 1;
                                if (li >= 2 && !mbar_wait(tempty0 + 8u * buf, (uint32_t)(((li >> 1) - 1) & 1), wait_ns)) {
                                    atomicOr(p.err, 8u);
                                    *vfail = 1;
                                    ok = false;
                                    break;
                                }
                                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                                const uint32_t d = tmem + (uint32_t)buf * acc_cols;
                                if constexpr (SPLIT) {
                                    for (int kk = kk0; kk < kk1; ++kk) {
                                        const unsigned long long off = (unsigned long long)((kk * ASTEP_BYTES) >> 4);
                                        mma<PREC>(d, dah + off, dbl + off, idesc, kk > kk0 ? 1u : 0u);
                                        mma<PREC>(d, dal + off, dbh + off, idesc, 1u);
                                    }
                                    for (int kk = kk0; kk < kk1; ++kk) {
                                        const unsigned long long off = (unsigned long long)((kk * ASTEP_BYTES) >> 4);
                                        mma<PREC>(d, dah + off, dbh + off, idesc, 1u);
                                    }
                                } else {
                                    for (int kk = kk0; kk < kk1; ++kk) {
                                        const unsigned long long off = (unsigned long long)((kk * ASTEP_BYTES) >> 4);
                                        mma<PREC>(d, dah + off, dbh + off, idesc, kk > kk0 ? 1u : 0u);
                                    }
                                }
                                mma_commit(tfull0 + 8u * buf);
                            }
                            if (!ok) break;
                            mma_commit(empty0 + 8u * s);
                            s_consumed = it + 1;
                        }
                        continue;
                    }
                    for (int kc0 = 0; kc0 < nk && ok; kc0 += kch, ++li) {
                        const int kc1 = min(nk, kc0 + kch);
                        const int buf = li & 1;
                        if (li >= 2 && !mbar_wait(tempty0 + 8u * buf, (uint32_t)(((li >> 1) - 1) & 1), wait_ns)) {
                            atomicOr(p.err, 8u);
                            *vfail = 1;
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t d = tmem + (uint32_t)buf * acc_cols;
                        for (int kbi = kc0; kbi < kc1; ++kbi, ++it) {
                            const int s = it % S;
                            if (!mbar_wait(full0 + 8u * s, (uint32_t)((it / S) & 1), wait_ns)) {
                                atomicOr(p.err, 2u);
                                *vfail = 1;
                                ok = false;
                                break;
                            }
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            const uint32_t sa = base + stage_bytes * s;
                            const uint32_t sah = sa, sal = sa + a_bytes;
                            const uint32_t sbh = sa + (SPLIT ? 2u : 1u) * a_bytes, sbl = sbh + b_bytes;
                            const int kc = (kb0 + kbi) * KE;
                            int ksteps = KE / KSTEP;
                            if (p.K - kc < KE) ksteps = (p.K - kc + KSTEP - 1) / KSTEP;
                            const unsigned long long dah = make_desc(sah), dbh = make_desc(sbh);
                            const unsigned long long dal = make_desc(sal), dbl = make_desc(sbl);
                            if constexpr (SPLIT) {
                                // the small cross products first, while the accumulator is small,
                                // then hi*hi: fewer round-toward-zero additions at full magnitude
                                for (int kk = 0; kk < ksteps; ++kk) {
                                    const unsigned long long off = (unsigned long long)((kk * ASTEP_BYTES) >> 4);
                                    mma<PREC>(d, dah + off, dbl + off, idesc, (kbi > kc0 || kk > 0) ? 1u : 0u);
                                    mma<PREC>(d, dal + off, dbh + off, idesc, 1u);
                                }
                                for (int kk = 0; kk < ksteps; ++kk) {
                                    const unsigned long long off = (unsigned long long)((kk * ASTEP_BYTES) >> 4);
                                    mma<PREC>(d, dah + off, dbh + off, idesc, 1u);
                                }
                            } else {
                                for (int kk = 0; kk < ksteps; ++kk) {
                                    const unsigned long long off = (unsigned long long)((kk * ASTEP_BYTES) >> 4);
                                    mma<PREC>(d, dah + off, dbh + off, idesc, (kbi > kc0 || kk > 0) ? 1u : 0u);
                                }
                            }
                            mma_commit(empty0 + 8u * s);
                            s_consumed = it + 1;
                        }
                        if (!ok) break;
                        mma_commit(tfull0 + 8u * buf);
                    }
                }
                mma_commit(drain_bar);   // completes once every MMA issued here has finished
            }
        }
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(REG_EPI) : "memory");
        // epilogue: warps 4..11; warp w reads TMEM lanes 32*(w%4) .. +31 and
        // columns cg*128 .. cg*128 + 127 of the accumulator
        const int q = warp & 3, cg = (warp - NCTRL) >> 2;
        int li = 0;
        float racc[DRAIN ? NSL : 1][SLW];   // running sums of the chunks (DRAIN only)
        bool ok = true;
        for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
            int lt;
            const KParams& p = P[locate(t, lt)];
            const int ntm = (p.M + TM - 1) / TM, ntn = (p.N + p.bn - 1) / p.bn, tiles_mn = ntm * ntn;
            const int z = lt / tiles_mn, rem = lt % tiles_mn;
            const int m0 = (p.nfast ? rem / ntn : rem % ntm) * TM, n0 = (p.nfast ? rem % ntn : rem / ntm) * p.bn;
            const int bz = z / p.ksplit, ks = z % p.ksplit;
            const int nk = min(p.per_split, p.nkb_total - ks * p.per_split);
            int nch = DRAIN ? (nk + p.kchunk - 1) / p.kchunk : 1;
            if (DRAIN && p.ksub > 0) {
                // the same chunking as the MMA warp: ceil(steps / ksub) per K block
                const int full_st = KE / KSTEP, per_full = (full_st + p.ksub - 1) / p.ksub;
                const bool tail = (ks * p.per_split + nk == p.nkb_total) && (p.K % KE != 0);
                nch = (nk - (tail ? 1 : 0)) * per_full;
                if (tail) nch += (((p.K % KE) + KSTEP - 1) / KSTEP + p.ksub - 1) / p.ksub;
            }
            const int m = m0 + q * 32 + lane;
            const bool mrow = (m < p.M);
            long long mo = 0;
            if (mrow) {
                constexpr int PW = Prec<PREC>::KE;
                const int q1 = m / p.mdiv, q0 = m % p.mdiv;
                mo = (long long)bz * p.sb + (long long)ks * p.sk + (long long)(q1 / PW) * p.q1p +
                     (long long)(q1 % PW) * p.q1s + (long long)(q0 / PW) * p.q0p + (long long)(q0 % PW) * p.q0s;
            }
            if constexpr (DRAIN) {
#pragma unroll
                for (int sl = 0; sl < NSL; ++sl)
#pragma unroll
                    for (int j = 0; j < SLW; ++j) racc[sl][j] = 0.0f;
            }
            for (int c = 0; c < nch; ++c, ++li) {
                const int buf = li & 1;
                if (!mbar_wait(tfull0 + 8u * buf, (uint32_t)((li >> 1) & 1), wait_ns)) {
                    if (lane == 0) atomicOr(p.err, 4u);
                    *vfail = 1;
                    ok = false;
                    break;
                }
                if (*vfail) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t tb = tmem + (uint32_t)buf * acc_cols + ((uint32_t)(q * 32) << 16);
                const bool last = (c == nch - 1);
                if constexpr (DRAIN) {
#pragma unroll
                    for (int sl = 0; sl < NSL; ++sl) {
                        const int c0 = cg * (NSL * SLW) + sl * SLW;
                        if (c0 < p.bn) {
                            uint32_t v[SLW];
                            tmem_ld64(tb + (uint32_t)c0, v);
#pragma unroll
                            for (int j = 0; j < SLW; ++j) racc[sl][j] += __uint_as_float(v[j]);
                        }
                    }
                    if (last) {
                        // the sums are in registers: give the accumulator back to the
                        // MMA warp before the (long) stores of the tile.  (Releasing it
                        // between the second slice's load and its adds measured slower:
                        // the loads then serialise behind the first slice's adds.)
                        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                        __syncwarp();
                        if (lane == 0)
                            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tempty0 + 8u * buf) : "memory");
#pragma unroll
                        for (int sl = 0; sl < NSL; ++sl) {
#pragma unroll
                            for (int hh = 0; hh < SLW / 32; ++hh) {
                                const int c0 = cg * (NSL * SLW) + sl * SLW + hh * 32;
                                const int nvalid = min(min(32, p.bn - c0), p.N - (n0 + c0));
                                if (c0 < p.bn && mrow && nvalid > 0) {
                                    float x[32];
#pragma unroll
                                    for (int j = 0; j < 32; ++j) x[j] = racc[sl][hh * 32 + j];
                                    emit32<PREC>(p, mo, n0 + c0, nvalid, x);
                                }
                            }
                        }
                        continue;
                    }
                } else {
                    for (int c0 = cg * (NSL * SLW); c0 < min(p.bn, (cg + 1) * NSL * SLW); c0 += SLW) {
                        uint32_t v[SLW];
                        tmem_ld64(tb + (uint32_t)c0, v);
#pragma unroll
                        for (int hh = 0; hh < SLW / 32; ++hh) {
                            const int c1 = c0 + hh * 32;
                            const int nvalid = min(min(32, p.bn - c1), p.N - (n0 + c1));   // this tile's columns only
                            if (mrow && nvalid > 0) {
                                float x[32];
#pragma unroll
                                for (int j = 0; j < 32; ++j) x[j] = __uint_as_float(v[hh * 32 + j]);
                                emit32<PREC>(p, mo, n0 + c1, nvalid, x);
                            }
                        }
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tempty0 + 8u * buf) : "memory");
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // every MMA of this block has completed before TMEM is released
        if (!mbar_wait(drain_bar, 0, wait_ns))
            for (int q = 0; q < nprob; ++q) atomicOr(P[q].err, 32u);
        if (*vfail) {
            // loads issued but never consumed must land before the block exits
            for (int it = s_consumed; it < s_issued; ++it)
                if (!mbar_wait(full0 + 8u * (it % S), (uint32_t)((it / S) & 1), wait_ns)) break;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 2) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

template <int PREC, bool DRAIN>
__global__ void __launch_bounds__(NTHREADS, 1) k_tc_gemm(const __grid_constant__ TcArgs a) {
    tc_body<PREC, DRAIN>(&a.p, a.m, nullptr, 1, a.p.bn, a.p.stages, a.p.acc_cols, a.p.wait_ns);
}

template <int PREC, bool DRAIN>
__global__ void __launch_bounds__(NTHREADS, 1) k_tc_gemm_group(const __grid_constant__ TcGroupArgs g) {
    tc_body<PREC, DRAIN>(g.p, &g.m[0][0], g.tile0, g.n, g.bn_max, g.stages, g.acc_cols, g.wait_ns);
}

// the single-contraction kernels and their grouped counterparts
const void* const k_single[6] = {(const void*)k_tc_gemm<PPL_PREC_BF16X3, false>, (const void*)k_tc_gemm<PPL_PREC_BF16X3, true>,
                                 (const void*)k_tc_gemm<PPL_PREC_TF32, false>,   (const void*)k_tc_gemm<PPL_PREC_TF32, true>,
                                 (const void*)k_tc_gemm<PPL_PREC_TF32X3, false>, (const void*)k_tc_gemm<PPL_PREC_TF32X3, true>};
const void* const k_grouped[6] = {
    (const void*)k_tc_gemm_group<PPL_PREC_BF16X3, false>, (const void*)k_tc_gemm_group<PPL_PREC_BF16X3, true>,
    (const void*)k_tc_gemm_group<PPL_PREC_TF32, false>,   (const void*)k_tc_gemm_group<PPL_PREC_TF32, true>,
    (const void*)k_tc_gemm_group<PPL_PREC_TF32X3, false>, (const void*)k_tc_gemm_group<PPL_PREC_TF32X3, true>};

// Sum split-K partials part[ks][n][m] (fp32) in FP64 into out[m * ldo + n].
__global__ void k_reduce_partials(const float* part, int ksplit, int M, int N, double* out, long long ldo) {
    const long long total = (long long)M * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(e % M), n = (int)(e / M);
        double s = 0.0;
        for (int k = 0; k < ksplit; ++k) s += (double)part[(long long)k * total + e];
        out[(long long)m * ldo + n] = s;
    }
}

// Batched transpose of operand planes: dst[b][j][i] = src[b][i][j] for i, j < n
// (row stride ld); 2-byte elements in two planes (BF16X3) or 4-byte in one (TF32).
template <typename T, int PLANES>
__global__ void k_transpose(const T* src, T* dst, long long plane, int n, long long ld, long long bstride) {
    __shared__ T tile[PLANES][32][33];
    const int tiles = (n + 31) / 32;
    const int b = blockIdx.z;
    const int ti = blockIdx.y, tj = blockIdx.x;
    if (ti >= tiles || tj >= tiles) return;
    const int i0 = ti * 32, j0 = tj * 32;
    const long long off = (long long)b * bstride;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = i0 + r, j = j0 + threadIdx.x;
        for (int pl = 0; pl < PLANES; ++pl)
            tile[pl][r][threadIdx.x] = (i < n && j < n) ? src[pl * plane + off + (long long)i * ld + j] : T(0);
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = j0 + r, i = i0 + threadIdx.x;
        if (i < n && j < n)
            for (int pl = 0; pl < PLANES; ++pl) dst[pl * plane + off + (long long)j * ld + i] = tile[pl][threadIdx.x][r];
    }
}

// ---- operand preparation -----------------------------------------------------

__device__ __forceinline__ long long ixd(const Idx2& x, int i) {
    return (long long)(i / x.div) * x.hi + (long long)(i % x.div) * x.lo;
}

template <int PREC>
__global__ void k_split(SplitSrc s, int rows, int cols, int batch, void* dst, long long plane, long long ld,
                        long long bstride) {
    const long long per = (long long)rows * ld;
    const long long total = per * batch;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / per);
        const long long rc = e % per;
        const int r = (int)(rc / ld), c = (int)(rc % ld);
        float x = 0.0f;
        double xd = 0.0;
        if (c < cols) {
            if (s.src32)
                xd = (double)s.src32[(long long)b * s.bstride + ixd(s.rmap, r) + ixd(s.cmap, c)];
            else
                xd = s.src[(long long)b * s.bstride + ixd(s.rmap, r) + ixd(s.cmap, c)];
        }
        const long long di = (long long)b * bstride + (long long)r * ld + c;
        if constexpr (PREC == PPL_PREC_BF16X3) {
            const __nv_bfloat16 hi = __double2bfloat16(xd);
            const __nv_bfloat16 lo = __double2bfloat16(xd - (double)__bfloat162float(hi));
            ((__nv_bfloat16*)dst)[di] = hi;
            ((__nv_bfloat16*)dst)[di + plane] = lo;
        } else if constexpr (PREC == PPL_PREC_TF32X3) {
            const float hi = round_tf32((float)xd);
            ((float*)dst)[di] = hi;
            ((float*)dst)[di + plane] = round_tf32((float)(xd - (double)hi));
        } else {
            x = (float)xd;
            ((float*)dst)[di] = round_tf32(x);
        }
    }
}

// FP64 (or FP32) source -> operand planes in the K-panel layout; one thread per
// destination element, so the writes are contiguous.
template <int PREC>
__global__ void k_split_panels(SplitSrc s, int rows, int prow, int cols, int kdiv, int kmod, int npan, int batch,
                               void* dst, long long plane) {
    constexpr int KE = Prec<PREC>::KE;
    const long long per_pan = (long long)prow * KE;
    const long long per = per_pan * npan;
    const long long total = per * batch;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / per);
        const long long rem = e % per;
        const int pan = (int)(rem / per_pan);
        const int rk = (int)(rem % per_pan);
        const int r = rk / KE, c = pan * KE + rk % KE;
        double xd = 0.0;
        if (r < rows && c < cols && (kdiv <= 0 || c % kdiv < kmod)) {
            const long long si = (long long)b * s.bstride + ixd(s.rmap, r) + ixd(s.cmap, c);
            xd = s.src32 ? (double)s.src32[si] : s.src[si];
        }
        if constexpr (PREC == PPL_PREC_BF16X3) {
            const __nv_bfloat16 hi = __double2bfloat16(xd);
            ((__nv_bfloat16*)dst)[e] = hi;
            ((__nv_bfloat16*)dst)[e + plane] = __double2bfloat16(xd - (double)__bfloat162float(hi));
        } else if constexpr (PREC == PPL_PREC_TF32X3) {
            const float hi = round_tf32((float)xd);
            ((float*)dst)[e] = hi;
            ((float*)dst)[e + plane] = round_tf32((float)(xd - (double)hi));
        } else {
            ((float*)dst)[e] = round_tf32((float)xd);
        }
    }
}

// X_b[a][k] in [b][k / KE][a][k % KE] (A rows per panel, k < B) ->
// [b][a / KE][k][a % KE] (B rows per panel), through a KE x KE tile in shared
// memory: both sides read and write whole contiguous KE-element rows.
// 4-byte elements (KE = 32) with 16-byte accesses: thread t reads
// row a0 + t / 8, elements 4 (t % 8) .. + 3 of a tile's 128-byte source row and
// writes row k0 + t / 8, elements 4 (t % 8) .. + 3 of a destination row; the
// padded shared tile makes both sides conflict-free.  vec = 0 (offsets that are
// not multiples of 4 elements) and the ragged edge tiles go element by element.
template <int PLANES>
__global__ void __launch_bounds__(256) k_transpose_panels4(const float* src, float* dst, long long plane_s,
                                                           long long plane_d, int A, int B, long long bstride_s,
                                                           long long bstride_d, int vec) {
    constexpr int KE = 32;
    __shared__ float tile[PLANES][KE][KE + 1];
    const int b = blockIdx.z;
    const int a0 = blockIdx.y * KE, k0 = blockIdx.x * KE;
    if (a0 >= A || k0 >= B) return;
    const long long os = (long long)b * bstride_s, od = (long long)b * bstride_d;
    const long long pan_s = (long long)A * KE, pan_d = (long long)B * KE;
    if (vec && a0 + KE <= A && k0 + KE <= B) {
        const int r = threadIdx.x >> 3, q = (threadIdx.x & 7) * 4;
        const float* sp = src + os + (long long)blockIdx.x * pan_s + (long long)(a0 + r) * KE + q;
        float4 v[PLANES];
#pragma unroll
        for (int pl = 0; pl < PLANES; ++pl) v[pl] = *(const float4*)(sp + pl * plane_s);
#pragma unroll
        for (int pl = 0; pl < PLANES; ++pl) {
            tile[pl][r][q] = v[pl].x;
            tile[pl][r][q + 1] = v[pl].y;
            tile[pl][r][q + 2] = v[pl].z;
            tile[pl][r][q + 3] = v[pl].w;
        }
        __syncthreads();
        float* dp = dst + od + (long long)blockIdx.y * pan_d + (long long)(k0 + r) * KE + q;
#pragma unroll
        for (int pl = 0; pl < PLANES; ++pl)
            *(float4*)(dp + pl * plane_d) =
                make_float4(tile[pl][q][r], tile[pl][q + 1][r], tile[pl][q + 2][r], tile[pl][q + 3][r]);
        return;
    }
    for (int e = threadIdx.x; e < KE * KE; e += blockDim.x) {
        const int ai = e / KE, ki = e % KE;
        const int a = a0 + ai, k = k0 + ki;
        for (int pl = 0; pl < PLANES; ++pl)
            tile[pl][ai][ki] = (a < A && k < B) ? src[pl * plane_s + os + (long long)blockIdx.x * pan_s + (long long)a * KE + ki]
                                                : 0.0f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < KE * KE; e += blockDim.x) {
        const int ki = e / KE, ai = e % KE;
        const int a = a0 + ai, k = k0 + ki;
        if (a < A && k < B)
            for (int pl = 0; pl < PLANES; ++pl)
                dst[pl * plane_d + od + (long long)blockIdx.y * pan_d + (long long)k * KE + ai] = tile[pl][ai][ki];
    }
}

// The same for 2-byte elements (bf16, KE = 64): 64 x 64 tiles, thread t moves
// elements 8 (t % 8) .. + 7 of rows t / 8 and 32 + t / 8 as 16-byte accesses;
// the shared tile's rows are 33 words, so both sides are nearly conflict-free.
template <int PLANES>
__global__ void __launch_bounds__(256) k_transpose_panels_h(const unsigned short* src, unsigned short* dst,
                                                            long long plane_s, long long plane_d, int A, int B,
                                                            long long bstride_s, long long bstride_d, int vec) {
    constexpr int KE = 64;
    __shared__ unsigned short tile[PLANES][KE][KE + 2];
    const int b = blockIdx.z;
    const int a0 = blockIdx.y * KE, k0 = blockIdx.x * KE;
    if (a0 >= A || k0 >= B) return;
    const long long os = (long long)b * bstride_s, od = (long long)b * bstride_d;
    const long long pan_s = (long long)A * KE, pan_d = (long long)B * KE;
    if (vec && a0 + KE <= A && k0 + KE <= B) {
        const int r = threadIdx.x >> 3, q = (threadIdx.x & 7) * 8;
        uint4 v[PLANES][2];
#pragma unroll
        for (int pl = 0; pl < PLANES; ++pl)
#pragma unroll
            for (int h = 0; h < 2; ++h)
                v[pl][h] = *(const uint4*)(src + pl * plane_s + os + (long long)blockIdx.x * pan_s +
                                           (long long)(a0 + r + 32 * h) * KE + q);
#pragma unroll
        for (int pl = 0; pl < PLANES; ++pl)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t w[4] = {v[pl][h].x, v[pl][h].y, v[pl][h].z, v[pl][h].w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    tile[pl][r + 32 * h][q + 2 * j] = (unsigned short)(w[j] & 0xffffu);
                    tile[pl][r + 32 * h][q + 2 * j + 1] = (unsigned short)(w[j] >> 16);
                }
            }
        __syncthreads();
#pragma unroll
        for (int pl = 0; pl < PLANES; ++pl)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int kr = r + 32 * h;   // destination row k0 + kr, elements a0 + q .. + 7
                uint32_t w[4];
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    w[j] = (uint32_t)tile[pl][q + 2 * j][kr] | ((uint32_t)tile[pl][q + 2 * j + 1][kr] << 16);
                *(uint4*)(dst + pl * plane_d + od + (long long)blockIdx.y * pan_d + (long long)(k0 + kr) * KE + q) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
        return;
    }
    for (int e = threadIdx.x; e < KE * KE; e += blockDim.x) {
        const int ai = e / KE, ki = e % KE;
        const int a = a0 + ai, k = k0 + ki;
        for (int pl = 0; pl < PLANES; ++pl)
            tile[pl][ai][ki] = (a < A && k < B)
                                   ? src[pl * plane_s + os + (long long)blockIdx.x * pan_s + (long long)a * KE + ki]
                                   : (unsigned short)0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < KE * KE; e += blockDim.x) {
        const int ki = e / KE, ai = e % KE;
        const int a = a0 + ai, k = k0 + ki;
        if (a < A && k < B)
            for (int pl = 0; pl < PLANES; ++pl)
                dst[pl * plane_d + od + (long long)blockIdx.y * pan_d + (long long)k * KE + ai] = tile[pl][ai][ki];
    }
}

bool make_map(CUtensorMap* m, int prec, const void* ptr, const TcMat& t, int box_rows) {
    const bool split = (prec == PPL_PREC_BF16X3);   // 2-byte elements
    const size_t es = split ? 2 : 4;
    const cuuint64_t ke = KROW_BYTES / es;
    const CUtensorMapDataType dt = split ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint64_t nb = (cuuint64_t)(t.batch > 0 ? t.batch : 1);
    CUresult r;
    if (t.panel) {
        // K panels of ke elements: {k in panel, row, panel, batch}
        const cuuint64_t npan = ((cuuint64_t)t.cols + ke - 1) / ke;
        cuuint64_t dims[4] = {ke, (cuuint64_t)t.rows, npan, nb};
        const cuuint64_t bs = (cuuint64_t)(t.bstride > 0 ? t.bstride : (long long)npan * t.ld * (long long)ke);
        cuuint64_t strides[3] = {ke * es, (cuuint64_t)t.ld * ke * es, bs * es};
        cuuint32_t box[4] = {(cuuint32_t)ke, (cuuint32_t)box_rows, 1, 1};
        cuuint32_t estr[4] = {1, 1, 1, 1};
        r = g_encode(m, dt, 4, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        cuuint64_t dims[3] = {(cuuint64_t)t.cols, (cuuint64_t)t.rows, nb};
        cuuint64_t strides[2] = {(cuuint64_t)(t.ld * es), (cuuint64_t)((t.bstride > 0 ? t.bstride : t.ld * t.rows) * es)};
        cuuint32_t box[3] = {(cuuint32_t)ke, (cuuint32_t)box_rows, 1};
        cuuint32_t estr[3] = {1, 1, 1};
        r = g_encode(m, dt, 3, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    return r == CUDA_SUCCESS;
}

int choose_bn(int N) {
    int tiles = (N + 255) / 256;
    int bn = (N + tiles - 1) / tiles;
    bn = (bn + 15) / 16 * 16;
    if (bn < 16) bn = 16;
    if (bn > 256) bn = 256;
    return bn;
}

inline int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

int tc_init_driver() {
    if (g_encode) return 0;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return -1;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    static bool attr_done = false;
    if (!attr_done) {
        const void* fns[12];
        for (int i = 0; i < 6; ++i) {
            fns[i] = k_single[i];
            fns[6 + i] = k_grouped[i];
        }
        for (const void* f : fns) {
            if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_ATTR) != cudaSuccess) {
                cudaGetLastError();
                return -2;
            }
            // the setmaxnreg split assumes exactly REG_LAUNCH registers per thread at
            // launch; with fewer, the epilogue's increase would wait forever
            cudaFuncAttributes fa;
            if (cudaFuncGetAttributes(&fa, f) != cudaSuccess) {
                cudaGetLastError();
                return -2;
            }
            if (fa.numRegs != REG_LAUNCH || fa.maxThreadsPerBlock < NTHREADS) return -12;
        }
        attr_done = true;
    }
    return 0;
}

namespace {

template <int PREC>
void launch_tc(bool drain, int grid, size_t smem, cudaStream_t s, const TcArgs& a) {
    if (drain)
        k_tc_gemm<PREC, true><<<grid, NTHREADS, smem, s>>>(a);
    else
        k_tc_gemm<PREC, false><<<grid, NTHREADS, smem, s>>>(a);
}


}  // namespace

int tc_gemm(const TcGemm& g, unsigned int* err_flag, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0 || g.K <= 0) return 0;
    if (tc_init_driver() != 0) return -1;
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) return -7;
    }
    if (g.prec != PPL_PREC_BF16X3 && g.prec != PPL_PREC_TF32 && g.prec != PPL_PREC_TF32X3) return -10;
    const bool split = (g.prec == PPL_PREC_BF16X3 || g.prec == PPL_PREC_TF32X3);   // hi and lo planes
    const bool half = (g.prec == PPL_PREC_BF16X3);
    const int KE = half ? 64 : 32;
    KParams p{};
    p.M = g.M; p.N = g.N; p.K = g.K;
    p.bn = g.bn > 0 ? g.bn : choose_bn(g.N);
    if (p.bn % 16 || p.bn > 256) return -8;
    p.acc_cols = SLW;      // at least one 64-column slice per accumulator, so no TMEM load leaves its buffer
    while (p.acc_cols < p.bn) p.acc_cols <<= 1;
    p.nkb_total = (g.K + KE - 1) / KE;
    p.ksplit = g.ksplit > 0 ? g.ksplit : 1;
    if (p.ksplit > p.nkb_total) p.ksplit = p.nkb_total;
    p.per_split = (p.nkb_total + p.ksplit - 1) / p.ksplit;
    p.ksplit = (p.nkb_total + p.per_split - 1) / p.per_split;   // every split slice is non-empty
    const int stage_bytes = (split ? 2 : 1) * (TM + p.bn) * KROW_BYTES;
    p.stages = SMEM_BUDGET / stage_bytes;
    if (p.stages > 8) p.stages = 8;
    if (p.stages < 2) return -2;
    p.a_row0 = g.a_row0; p.b_row0 = g.b_row0; p.a_b0 = g.a_b0; p.b_b0 = g.b_b0;
    p.a_bstep = g.a_bstep; p.b_bstep = g.b_bstep;
    p.batch = g.batch;
    p.kind = g.out.kind; p.out = g.out.out; p.plane = g.out.plane_elems;
    p.sb = g.out.sb; p.sk = g.out.sk;
    p.q1p = g.out.q1p; p.q1s = g.out.q1s; p.q0p = g.out.q0p; p.q0s = g.out.q0s; p.np = g.out.np; p.ns = g.out.ns;
    p.mdiv = g.out.mdiv > 0 ? g.out.mdiv : (1 << 30);
    if (g.out.alpha != 1.0f) return -9;
    p.alpha = 1.0f;
    p.kchunk = g.kchunk;
    p.ksub = (g.ksub > 0 && g.ksub < KE / (half ? 16 : 8)) ? g.ksub : 0;
    if (p.ksub > 0) p.kchunk = 1;
    p.nfast = g.nfast;
    p.a_panel = g.A.panel ? 1 : 0;
    p.b_panel = g.B.panel ? 1 : 0;
    const bool drain = p.ksub > 0 || (g.kchunk > 0 && g.kchunk < p.per_split);
    if (drain && p.bn > 256) return -8;
    p.err = err_flag;
    p.wait_ns = g.wait_ns > 0 ? g.wait_ns : WAIT_NS;

    TcArgs a;
    CUtensorMap &mAh = a.m[0], &mAl = a.m[1], &mBh = a.m[2], &mBl = a.m[3];
    const size_t es = half ? 2 : 4;
    if (!make_map(&mAh, g.prec, g.A.ptr, g.A, TM) || !make_map(&mBh, g.prec, g.B.ptr, g.B, p.bn)) return -3;
    if (split) {
        if (!make_map(&mAl, g.prec, (const char*)g.A.ptr + g.A.plane_elems * es, g.A, TM) ||
            !make_map(&mBl, g.prec, (const char*)g.B.ptr + g.B.plane_elems * es, g.B, p.bn))
            return -3;
    } else {
        mAl = mAh;
        mBl = mBh;
    }
    a.p = p;
    const size_t smem = (size_t)stage_bytes * p.stages + 1024 + 16 * p.stages + 64;
    if (smem > (size_t)SMEM_ATTR) return -6;
    const long long tiles = (long long)((g.M + TM - 1) / TM) * ((g.N + p.bn - 1) / p.bn) * g.batch * p.ksplit;
    if (tiles > (1ll << 30)) return -4;
    int grid = (int)(tiles < sms ? tiles : sms);
    if (g.grid_cap > 0 && grid > g.grid_cap) grid = g.grid_cap;
    if (g.prec == PPL_PREC_BF16X3)
        launch_tc<PPL_PREC_BF16X3>(drain, grid, smem, s, a);
    else if (g.prec == PPL_PREC_TF32X3)
        launch_tc<PPL_PREC_TF32X3>(drain, grid, smem, s, a);
    else
        launch_tc<PPL_PREC_TF32>(drain, grid, smem, s, a);
    const cudaError_t le = cudaGetLastError();
    return le == cudaSuccess ? 0 : -(1000 + (int)le);
}

void reduce_partials(const float* part, int ksplit, int M, int N, double* out, long long ldo, cudaStream_t s) {
    const long long total = (long long)M * N;
    if (total <= 0) return;
    k_reduce_partials<<<grid_for(total, 256), 256, 0, s>>>(part, ksplit, M, N, out, ldo);
}

void transpose_operand(int prec, const void* src, void* dst, long long plane_elems, int n, long long ld,
                       long long bstride, int batch, cudaStream_t s) {
    if (n <= 0 || batch <= 0) return;
    const int tiles = (n + 31) / 32;
    dim3 grid(tiles, tiles, batch), block(32, 8);
    if (prec == PPL_PREC_BF16X3)
        k_transpose<unsigned short, 2><<<grid, block, 0, s>>>((const unsigned short*)src, (unsigned short*)dst,
                                                              plane_elems, n, ld, bstride);
    else if (prec == PPL_PREC_TF32X3)
        k_transpose<float, 2><<<grid, block, 0, s>>>((const float*)src, (float*)dst, plane_elems, n, ld, bstride);
    else
        k_transpose<float, 1><<<grid, block, 0, s>>>((const float*)src, (float*)dst, plane_elems, n, ld, bstride);
}

void split_to_operand(int prec, const SplitSrc& s, int rows, int cols, int batch, void* dst, long long plane_elems,
                      long long ld, long long bstride, cudaStream_t st) {
    const long long total = (long long)rows * ld * batch;
    if (total <= 0) return;
    if (prec == PPL_PREC_BF16X3)
        k_split<PPL_PREC_BF16X3><<<grid_for(total, 256), 256, 0, st>>>(s, rows, cols, batch, dst, plane_elems, ld,
                                                                       bstride);
    else if (prec == PPL_PREC_TF32X3)
        k_split<PPL_PREC_TF32X3><<<grid_for(total, 256), 256, 0, st>>>(s, rows, cols, batch, dst, plane_elems, ld,
                                                                       bstride);
    else
        k_split<PPL_PREC_TF32><<<grid_for(total, 256), 256, 0, st>>>(s, rows, cols, batch, dst, plane_elems, ld,
                                                                     bstride);
}

int panel_width(int prec) { return prec == PPL_PREC_BF16X3 ? 64 : 32; }

void split_to_panels(int prec, const SplitSrc& s, int rows, int prow, int cols, int kdiv, int kmod, int batch,
                     void* dst, long long plane_elems, cudaStream_t st) {
    const int ke = panel_width(prec);
    const int npan = (cols + ke - 1) / ke;
    const long long total = (long long)prow * ke * npan * batch;
    if (total <= 0) return;
    if (prec == PPL_PREC_BF16X3)
        k_split_panels<PPL_PREC_BF16X3><<<grid_for(total, 256), 256, 0, st>>>(s, rows, prow, cols, kdiv, kmod, npan,
                                                                              batch, dst, plane_elems);
    else if (prec == PPL_PREC_TF32X3)
        k_split_panels<PPL_PREC_TF32X3><<<grid_for(total, 256), 256, 0, st>>>(s, rows, prow, cols, kdiv, kmod, npan,
                                                                              batch, dst, plane_elems);
    else
        k_split_panels<PPL_PREC_TF32><<<grid_for(total, 256), 256, 0, st>>>(s, rows, prow, cols, kdiv, kmod, npan,
                                                                            batch, dst, plane_elems);
}

void transpose_panels(int prec, const void* src, void* dst, long long plane_s, long long plane_d, int A, int B,
                      long long bstride_s, long long bstride_d, int batch, cudaStream_t s) {
    if (A <= 0 || B <= 0 || batch <= 0) return;
    if (prec == PPL_PREC_BF16X3) {
        auto m8 = [](long long x) { return x % 8 == 0; };
        const int vec = m8(plane_s) && m8(plane_d) && m8(bstride_s) && m8(bstride_d) &&
                        (uintptr_t)src % 16 == 0 && (uintptr_t)dst % 16 == 0;
        k_transpose_panels_h<2><<<dim3((B + 63) / 64, (A + 63) / 64, batch), 256, 0, s>>>(
            (const unsigned short*)src, (unsigned short*)dst, plane_s, plane_d, A, B, bstride_s, bstride_d, vec);
    } else {
        auto m4 = [](long long x) { return x % 4 == 0; };
        const int vec = m4(plane_s) && m4(plane_d) && m4(bstride_s) && m4(bstride_d) &&
                        (uintptr_t)src % 16 == 0 && (uintptr_t)dst % 16 == 0;
        const dim3 grid((B + 31) / 32, (A + 31) / 32, batch);
        if (prec == PPL_PREC_TF32X3)
            k_transpose_panels4<2><<<grid, 256, 0, s>>>((const float*)src, (float*)dst, plane_s, plane_d, A, B,
                                                       bstride_s, bstride_d, vec);
        else
            k_transpose_panels4<1><<<grid, 256, 0, s>>>((const float*)src, (float*)dst, plane_s, plane_d, A, B,
                                                       bstride_s, bstride_d, vec);
    }
}

void zero_bytes(void* p, size_t n, cudaStream_t s) {
    if (n) cudaMemsetAsync(p, 0, n, s);
}

// ---- several captured contractions as one persistent launch ------------------

namespace {
struct GroupNode {
    TcGroupArgs a;
    void* params[1];
};
}  // namespace

const void* tc_group_kernel(const void* f) {
    for (int i = 0; i < 6; ++i)
        if (k_single[i] == f) return k_grouped[i];
    return nullptr;
}

int tc_group_capacity() { return TC_GROUP_MAX; }

int tc_group_node_params(const void* f, const void* const* args, int n, cudaKernelNodeParams* out, void** storage) {
    *storage = nullptr;
    int ki = -1;
    for (int i = 0; i < 6; ++i)
        if (k_single[i] == f) ki = i;
    if (ki < 0 || n < 1 || n > TC_GROUP_MAX || !args || !out) return -1;
    if (tc_init_driver() != 0) return -1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) return -7;
    GroupNode* g = new (std::nothrow) GroupNode();
    if (!g) return -2;
    TcGroupArgs& a = g->a;
    a.n = n;
    a.bn_max = 0;
    a.acc_cols = 0;
    a.wait_ns = 0;
    long long tot = 0;
    for (int i = 0; i < n; ++i) {
        const TcArgs* x = (const TcArgs*)args[i];
        for (int j = 0; j < 4; ++j) a.m[i][j] = x->m[j];
        a.p[i] = x->p;
        if (x->p.bn > a.bn_max) a.bn_max = x->p.bn;
        if (x->p.acc_cols > a.acc_cols) a.acc_cols = x->p.acc_cols;
        if (x->p.wait_ns > a.wait_ns) a.wait_ns = x->p.wait_ns;
        a.tile0[i] = (int)tot;
        tot += tc_tiles(x->p);
    }
    if (tot > (1ll << 30)) {
        delete g;
        return -4;
    }
    a.tile0[n] = (int)tot;
    const int planes = (ki / 2 == 1) ? 1 : 2;   // TF32 one plane; BF16X3 and TF32X3 hi and lo
    const int stage_bytes = planes * (TM + a.bn_max) * KROW_BYTES;
    a.stages = SMEM_BUDGET / stage_bytes;
    if (a.stages > 8) a.stages = 8;
    const size_t smem = (size_t)stage_bytes * a.stages + 1024 + 16 * a.stages + 64;
    if (a.stages < 2 || smem > (size_t)SMEM_ATTR) {
        delete g;
        return -6;
    }
    g->params[0] = &g->a;
    *out = cudaKernelNodeParams{};
    out->func = const_cast<void*>(k_grouped[ki]);
    out->gridDim = dim3((unsigned)(tot < sms ? tot : sms));
    out->blockDim = dim3(NTHREADS);
    out->sharedMemBytes = (unsigned)smem;
    out->kernelParams = g->params;
    out->extra = nullptr;
    *storage = g;
    return 0;
}

void tc_group_release(void* storage) { delete (GroupNode*)storage; }

// Allocation-free CP energy: ppl_cp_energy_static (include/ppl_cpd.h).
//
// Same arithmetic as ppl_cpd_energy (the strided FP64 GEMM for
// Z_y[Q][i][r] = sum_a B[Q][i][o+a] y[a][r], then the per-(Q, r) reduction),
// but its scratch lives in one file-scope device array instead of a
// caller-provided workspace, and the auxiliary index Q is processed in
// chunks that fit that array.  No call here allocates memory.
#include "ppl_internal.h"

#include <cstdio>
#include <mutex>

#include "../../include/ppl_cpd.h"

void ppl_set_global_error(const char* msg);   // ppl_cpd.cu

namespace {

constexpr size_t SCALAR_BYTES = 256;          // running total and the chunk's sum
constexpr size_t PARTIAL_BYTES = 8192;        // per-block partial sums of the reduction
constexpr size_t Z_OFFSET = SCALAR_BYTES + PARTIAL_BYTES;

// Held by every GPU that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_scratch[PPL_STATIC_SCRATCH_BYTES];

std::mutex g_mu;
struct Entry {
    void* ctx;    // the context the address belongs to
    void* ptr;
};
Entry g_dev_ptr[64] = {};

typedef int (*CtxGetCurrentFn)(void**);
CtxGetCurrentFn g_ctx_current = nullptr;

// The current context (the driver's cuCtxGetCurrent, resolved once through the
// runtime so that the library keeps no link dependency on libcuda); nullptr if
// it cannot be resolved.
void* current_context() {
    if (!g_ctx_current) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return nullptr;
        }
        g_ctx_current = (CtxGetCurrentFn)fn;
    }
    void* c = nullptr;
    return g_ctx_current(&c) == 0 ? c : nullptr;
}

// Device address of g_scratch on the current device, looked up once per
// device and context (the name g_scratch in host code is only a stand-in for
// the symbol).  A context created after a device reset looks it up again.
int scratch_address(void** out, int* dev_out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return -1;
    }
    *dev_out = dev;
    void* ctx = current_context();
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev].ptr || g_dev_ptr[dev].ctx != ctx || !ctx) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            g_dev_ptr[dev] = Entry{nullptr, nullptr};
            return -2;
        }
        g_dev_ptr[dev] = Entry{ctx, p};
    }
    *out = g_dev_ptr[dev].ptr;
    return 0;
}

// forget the cached address of a device after a failed call
void drop_address(int dev) {
    if (dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lock(g_mu);
    g_dev_ptr[dev] = Entry{nullptr, nullptr};
}

int fail_static(int code, const char* msg) {
    ppl_set_global_error(msg);
    return code;
}

}  // namespace

extern "C" int ppl_cp_energy_static(int o, int v, int X, int R, const double* B, const double* factors,
                                    double* E_cp, void* stream) {
    if (!B || !factors || !E_cp) return fail_static(PPL_EINVAL, "ppl_cp_energy_static: NULL argument");
    if (o < 1 || v < 1 || X < 1 || R < 1) return fail_static(PPL_EINVAL, "ppl_cp_energy_static: sizes must be >= 1");
    const size_t per_q = 2 * (size_t)o * (size_t)R * sizeof(double);
    const size_t room = PPL_STATIC_SCRATCH_BYTES - Z_OFFSET;
    if (per_q > room) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "ppl_cp_energy_static: o*R = %lld exceeds the static scratch limit o*R <= %lld (%zu bytes)",
                 (long long)o * R, (long long)(room / (2 * sizeof(double))), (size_t)PPL_STATIC_SCRATCH_BYTES);
        return fail_static(PPL_EINVAL, buf);
    }
    cudaGetLastError();   // a launch error left behind by earlier work is not this call's
    void* base = nullptr;
    int dev = -1;
    if (scratch_address(&base, &dev) != 0)
        return fail_static(PPL_ECUDA, "ppl_cp_energy_static: cudaGetSymbolAddress of the scratch array failed");
    cudaStream_t s = (cudaStream_t)stream;
    char* w = (char*)base;
    double* total = (double*)w;
    double* chunk = total + 1;
    double* partial = (double*)(w + SCALAR_BYTES);
    double* Za = (double*)(w + Z_OFFSET);
    const int qc = (int)((room / per_q) < (size_t)X ? room / per_q : (size_t)X);
    double* Zb = Za + (size_t)qc * o * R;
    const int n = o + v;
    const double* U[2] = {factors, factors + (size_t)v * R};
    const double* Ui = factors + (size_t)2 * v * R;
    const double* Uj = Ui + (size_t)o * R;
    const double* lam = Uj + (size_t)o * R;
    double* Z[2] = {Za, Zb};

    cudaMemsetAsync(total, 0, sizeof(double), s);   // the array keeps the previous call's contents
    for (int q0 = 0; q0 < X; q0 += qc) {
        const int xc = (X - q0 < qc) ? X - q0 : qc;
        for (int w2 = 0; w2 < 2; ++w2) {
            G64 g{};
            g.A = B + (long long)q0 * n * n + o; g.ab = (long long)n * n; g.am = ix1(n); g.ak = ix1(1);
            g.B = U[w2]; g.bn = ix1(1); g.bk = ix1(R);
            g.C = Z[w2]; g.cb = (long long)o * R; g.cm = ix1(R); g.cn = ix1(1);
            g.M = o; g.N = R; g.K = v; g.batch = xc; g.ksplit = 1; g.alpha = 1.0;
            gemm64(g, s);
        }
        energy_reduce(Za, Zb, Ui, Uj, lam, xc, o, R, partial, chunk, s);
        sum_partials(chunk, 1, total, 1, s);
    }
    cudaMemcpyAsync(E_cp, total, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    const cudaError_t le = cudaGetLastError();
    if (e == cudaSuccess) e = le;
    if (e != cudaSuccess) {
        drop_address(dev);
        char buf[256];
        snprintf(buf, sizeof buf, "ppl_cp_energy_static: %s", cudaGetErrorString(e));
        return fail_static(PPL_ECUDA, buf);
    }
    return PPL_OK;
}

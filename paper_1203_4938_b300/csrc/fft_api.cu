// fft_api.cu -- plans and the C ABI declared in include/fft.h.
//
// A plan is the analogue of the paper's cached program (Sec. II-D, the run
// protocol's program ID): everything that depends only on the shape -- the
// factorisation, the FP64-evaluated twiddle tables, the workspace, the kernel
// configuration -- is built once by fft_plan_create, and fft_exec only
// enqueues kernels on the caller's stream.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <string>

#include "../../include/fft.h"
#include "launch.h"
#include "plan.h"

using namespace b300fft;

namespace {

thread_local fft_status g_last_error = FFT_OK;
std::mutex g_registry_mu;
std::set<const void*> g_registry;  // live plan handles

bool is_registered(const fft_plan_s* p) {
    std::lock_guard<std::mutex> lk(g_registry_mu);
    return p && g_registry.count(p) && p->magic == kPlanMagic;
}

int ilog2_exact(int64_t v) {
    if (v <= 0 || (v & (v - 1))) return -1;
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return l;
}

fft_plan fail(fft_status s, fft_plan_s* p) {
    g_last_error = s;
    if (p) {
        destroy_plan_resources(p);
        delete p;
    }
    return nullptr;
}

}  // namespace

namespace b300fft {

void destroy_plan_resources(fft_plan_s* p) {
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->d_tables) cudaFree(p->d_tables);
    if (p->d_work) cudaFree(p->d_work);
    if (p->d_status) cudaFree(p->d_status);
    if (p->d_aux) cudaFree(p->d_aux);
    p->graph_exec = nullptr;
    p->graph = nullptr;
    p->d_tables = nullptr;
    p->d_work = nullptr;
    p->d_status = nullptr;
    p->d_aux = nullptr;
}

}  // namespace b300fft

// --------------------------------------------------------------------------
// plan construction
// --------------------------------------------------------------------------
namespace {

fft_status alloc_tables(fft_plan_s* p, size_t entries) {
    if (entries == 0) entries = 1;
    if (cudaMalloc(&p->d_tables, entries * sizeof(float2)) != cudaSuccess) return FFT_ERR_ALLOC;
    return FFT_OK;
}

fft_status build_pow2_1d(fft_plan_s* p, int logn) {
    const int single_max = p->single_max_log;
    if (logn <= single_max) {
        p->kind = PlanKind::Rows;
        p->logn_a = logn;
        p->off_a = 0;
        size_t ent = (size_t)pow2_table_entries(logn);
        fft_status s = alloc_tables(p, ent);
        if (s != FFT_OK) return s;
        if (gen_pow2_table(p->d_tables + p->off_a, logn, 0) != cudaSuccess) return FFT_ERR_CUDA;
        if (rows_prepare(logn, false) != cudaSuccess) return FFT_ERR_CUDA;
        p->kernels = 1;
        std::snprintf(p->desc, sizeof p->desc, "rows N=2^%d tpc=%d threads=%d smem=%d", logn,
                      rows_tpc(logn, false), rows_threads(logn, false), rows_smem(logn, false));
        return FFT_OK;
    }
    // four-step: N = N1 * N2, pass A = columns of length N1 (stride N2) with
    // the W_N^{n2 k1} twiddle, pass B = rows of length N2, transposed store.
    int l2 = (logn + 1) / 2, l1 = logn - l2;
    if (l2 > kColsMaxLog || l1 > kColsMaxLog || l2 < 5 || l1 < 1) return FFT_ERR_UNSUPPORTED;
    if ((int64_t(1) << l2) % cols_width(l1) != 0) return FFT_ERR_UNSUPPORTED;
    p->kind = PlanKind::FourStep;
    p->cols_c = cols_width(l1);
    p->logn_a = l1;
    p->logn_b = l2;
    p->sh = (logn + 1) / 2;
    const size_t ea = (size_t)pow2_table_entries(l1), eb = (size_t)pow2_table_entries(l2);
    const size_t elo = size_t(1) << p->sh, ehi = size_t(1) << (logn - p->sh);
    p->off_a = 0;
    p->off_b = p->off_a + ea;
    p->off_lo = p->off_b + eb;
    p->off_hi = p->off_lo + elo;
    fft_status s = alloc_tables(p, p->off_hi + ehi);
    if (s != FFT_OK) return s;
    const int64_t n = int64_t(1) << logn;
    if (gen_pow2_table(p->d_tables + p->off_a, l1, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (gen_pow2_table(p->d_tables + p->off_b, l2, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (gen_root_table(p->d_tables + p->off_lo, (int64_t)elo, 1, n, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (gen_root_table(p->d_tables + p->off_hi, (int64_t)ehi, (int64_t)elo, n, 0) != cudaSuccess)
        return FFT_ERR_CUDA;
    p->work_bytes = (size_t)n * (size_t)p->batch * sizeof(float2);
    if (cudaMalloc(&p->d_work, p->work_bytes) != cudaSuccess) return FFT_ERR_ALLOC;
    if (cols_prepare(l1, p->cols_c) != cudaSuccess || rows_prepare(l2, true) != cudaSuccess) return FFT_ERR_CUDA;
    p->kernels = 2;
    std::snprintf(p->desc, sizeof p->desc,
                  "fourstep N=2^%d = 2^%d (cols C=%d threads=%d) x 2^%d (rows-T tpc=%d threads=%d) work=%zuB",
                  logn, l1, p->cols_c, cols_threads(l1, p->cols_c), l2, rows_tpc(l2, true), rows_threads(l2, true),
                  p->work_bytes);
    return FFT_OK;
}

fft_status build_pow2_2d(fft_plan_s* p, int logh, int logw) {
    if (logw > kRowsMaxLog || logh > kColsMaxLog || logh < 1) return FFT_ERR_UNSUPPORTED;
    p->kind = PlanKind::TwoD;
    p->cols_c = cols_width_for(logh, int64_t(1) << logw);
    p->logn_a = logw;  // rows pass
    p->logn_b = logh;  // columns pass
    const size_t ea = (size_t)pow2_table_entries(logw), eb = (size_t)pow2_table_entries(logh);
    p->off_a = 0;
    p->off_b = ea;
    fft_status s = alloc_tables(p, ea + eb);
    if (s != FFT_OK) return s;
    if (gen_pow2_table(p->d_tables + p->off_a, logw, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (gen_pow2_table(p->d_tables + p->off_b, logh, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (rows_prepare(logw, false) != cudaSuccess || cols_prepare(logh, p->cols_c) != cudaSuccess) return FFT_ERR_CUDA;
    p->kernels = 2;
    std::snprintf(p->desc, sizeof p->desc, "2d H=2^%d W=2^%d: rows(tpc=%d) then cols(C=%d threads=%d)", logh,
                  logw, rows_tpc(logw, false), p->cols_c, cols_threads(logh, p->cols_c));
    return FFT_OK;
}

}  // namespace

extern "C" {

fft_plan fft_plan_create(int dims, const int64_t* lengths, int64_t batch, int precision) {
    g_last_error = FFT_OK;
    if ((dims != 1 && dims != 2) || !lengths || batch < 1) return fail(FFT_ERR_INVALID_ARG, nullptr);
    for (int d = 0; d < dims; ++d)
        if (lengths[d] < 1 || lengths[d] > (int64_t(1) << 30)) return fail(FFT_ERR_INVALID_ARG, nullptr);
    if (precision < FFT_FP32 || precision > FFT_TC_BF16_PLAIN) return fail(FFT_ERR_INVALID_ARG, nullptr);
    int64_t total = batch;
    for (int d = 0; d < dims; ++d) {
        if (total > (int64_t(1) << 40) / lengths[d]) return fail(FFT_ERR_INVALID_ARG, nullptr);
        total *= lengths[d];
    }
    fft_plan_s* p = new (std::nothrow) fft_plan_s();
    if (!p) return fail(FFT_ERR_ALLOC, nullptr);
    p->dims = dims;
    p->len[0] = lengths[0];
    p->len[1] = dims == 2 ? lengths[1] : 1;
    p->batch = batch;
    p->precision = precision;
    p->elements = total;
    if (cudaMalloc(&p->d_status, sizeof(int)) != cudaSuccess) return fail(FFT_ERR_ALLOC, p);
    if (cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess) return fail(FFT_ERR_CUDA, p);

    fft_status s = FFT_ERR_UNSUPPORTED;
    if (precision != FFT_FP32) {
        s = build_tc_plan(p);
    } else if (dims == 1) {
        const int l = ilog2_exact(lengths[0]);
        if (l >= 0) s = build_pow2_1d(p, l);
        else s = build_generic_1d(p);
    } else {
        const int lh = ilog2_exact(lengths[0]), lw = ilog2_exact(lengths[1]);
        if (lh >= 0 && lw >= 0) s = build_pow2_2d(p, lh, lw);
        else s = FFT_ERR_UNSUPPORTED;
    }
    if (s != FFT_OK) return fail(s, p);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(FFT_ERR_CUDA, p);
    p->magic = kPlanMagic;
    {
        std::lock_guard<std::mutex> lk(g_registry_mu);
        g_registry.insert(p);
    }
    return p;
}

fft_status fft_last_error(void) { return g_last_error; }

fft_status fft_exec(fft_plan plan, const void* in, void* out, int direction, void* stream) {
    if (!is_registered(plan)) return FFT_ERR_BAD_HANDLE;
    if (!in || !out) return FFT_ERR_INVALID_ARG;
    if (direction != FFT_FORWARD && direction != FFT_INVERSE) return FFT_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
        return FFT_ERR_MISALIGNED;
    return exec_plan(plan, static_cast<const float2*>(in), static_cast<float2*>(out), direction == FFT_INVERSE,
                     static_cast<cudaStream_t>(stream));
}

fft_status fft_exec_kernel(fft_plan plan, int k, const void* in, void* out, int direction, void* stream) {
    if (!is_registered(plan)) return FFT_ERR_BAD_HANDLE;
    if (k < 0 || k >= plan->kernels) return FFT_ERR_INVALID_ARG;
    if (!in || !out) return FFT_ERR_INVALID_ARG;
    if (direction != FFT_FORWARD && direction != FFT_INVERSE) return FFT_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
        return FFT_ERR_MISALIGNED;
    return exec_plan(plan, static_cast<const float2*>(in), static_cast<float2*>(out), direction == FFT_INVERSE,
                     static_cast<cudaStream_t>(stream), k);
}

fft_status fft_plan_check(fft_plan plan) {
    if (!is_registered(plan)) return FFT_ERR_BAD_HANDLE;
    int h = 0;
    if (cudaMemcpy(&h, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return FFT_ERR_CUDA;
    if (h != 0) {
        int z = 0;
        cudaMemcpy(plan->d_status, &z, sizeof(int), cudaMemcpyHostToDevice);
        return (fft_status)h;
    }
    return FFT_OK;
}

fft_status fft_plan_destroy(fft_plan plan) {
    {
        std::lock_guard<std::mutex> lk(g_registry_mu);
        if (!plan || !g_registry.count(plan) || plan->magic != kPlanMagic) return FFT_ERR_BAD_HANDLE;
        g_registry.erase(plan);
    }
    cudaDeviceSynchronize();
    plan->magic = 0;
    destroy_plan_resources(plan);
    delete plan;
    return FFT_OK;
}

size_t fft_plan_workspace_bytes(fft_plan plan) {
    if (!is_registered(plan)) return 0;
    return plan->work_bytes;
}

const char* fft_status_string(fft_status s) {
    switch (s) {
        case FFT_OK: return "ok";
        case FFT_ERR_INVALID_ARG: return "invalid argument";
        case FFT_ERR_UNSUPPORTED: return "unsupported shape or precision";
        case FFT_ERR_ALLOC: return "allocation failed";
        case FFT_ERR_MISALIGNED: return "pointer not 16-byte aligned";
        case FFT_ERR_CUDA: return "CUDA runtime error";
        case FFT_ERR_TIMEOUT: return "device wait timed out";
        case FFT_ERR_BAD_HANDLE: return "invalid plan handle";
    }
    return "unknown status";
}

int fft_plan_kernel_count(fft_plan plan) {
    if (!is_registered(plan)) return 0;
    return plan->kernels;
}

int fft_plan_describe(fft_plan plan, char* buf, size_t cap) {
    if (!is_registered(plan)) return -1;
    const size_t n = std::strlen(plan->desc);
    if (buf && cap) {
        const size_t c = n < cap - 1 ? n : cap - 1;
        std::memcpy(buf, plan->desc, c);
        buf[c] = 0;
    }
    return (int)n;
}

}  // extern "C"

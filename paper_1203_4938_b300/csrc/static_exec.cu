// static_exec.cu -- fft_exec_pow2_static: the two-launch four-step transform
// with its workspace and twiddle tables in file-scope device arrays, for
// callers that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or forbidden
// -- inside a memory-pool-less real-time loop, a plugin whose host forbids
// allocation after start-up, or a caller that budgets every device byte up
// front -- can still run a large 1-D transform.  The arrays below are part
// of the library image: every GPU on which the library's device code is
// loaded holds them (about 32.1 MiB) until the process exits.  Under CUDA's
// default lazy module loading this file's module is loaded, and the 32.1 MiB
// committed, at the first call on each device (the cudaGetSymbolAddress of
// the set-up), so a caller should make one call per device before it fixes
// its device-memory budget, and before any stream capture.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/fft.h"
#include "launch.h"

namespace b300fft {

// Largest n * batch the static entry point accepts (complex elements).
constexpr int64_t kStaticMaxElements = int64_t(1) << 22;  // 32 MiB of workspace
constexpr int kStaticTableEntries = 16384;                 // twiddle tables of n <= 2^22

static __device__ __align__(256) float2 g_static_work[kStaticMaxElements];
static __device__ __align__(256) float2 g_static_tables[kStaticTableEntries];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
bool g_static_ready[kMaxDevices] = {};
float2* g_static_work_ptr[kMaxDevices] = {};
float2* g_static_tab_ptr[kMaxDevices] = {};
int64_t g_static_tab_n[kMaxDevices] = {};  // n whose tables the device's array holds (0: none)

// Once per device, with that device current: device addresses of the static
// arrays (the host-side symbols are not device addresses) and the
// shared-memory limits of the kernels used below.
fft_status setup_device(int dev) {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (g_static_ready[dev]) return FFT_OK;
    void* w = nullptr;
    void* t = nullptr;
    if (cudaGetSymbolAddress(&w, g_static_work) != cudaSuccess) return FFT_ERR_CUDA;
    if (cudaGetSymbolAddress(&t, g_static_tables) != cudaSuccess) return FFT_ERR_CUDA;
    for (int l = 1; l <= 11; ++l) {
        for (int c = 1; c <= 64; c *= 2)
            if (cols_width_valid(l, c) && cols_prepare(l, c) != cudaSuccess) return FFT_ERR_CUDA;
        if (l >= 5)
            for (int tpc = 2; tpc <= 64; tpc *= 2)
                if (rowsT_threads(l, tpc) <= 1024 && rowsT_prepare(l, tpc) != cudaSuccess) return FFT_ERR_CUDA;
    }
    g_static_work_ptr[dev] = static_cast<float2*>(w);
    g_static_tab_ptr[dev] = static_cast<float2*>(t);
    g_static_ready[dev] = true;
    return FFT_OK;
}

int ilog2_pow2(int64_t v) {
    if (v <= 0 || (v & (v - 1))) return -1;
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return l;
}

}  // namespace
}  // namespace b300fft

using namespace b300fft;

extern "C" fft_status fft_exec_pow2_static(const void* in, void* out, int64_t n, int64_t batch, int direction,
                                           void* stream) {
    const int logn = ilog2_pow2(n);
    if (logn < 13 || logn > 22 || batch < 1) return FFT_ERR_INVALID_ARG;
    if (batch > kStaticMaxElements / n) return FFT_ERR_INVALID_ARG;
    if (!in || !out) return FFT_ERR_INVALID_ARG;
    if (direction != FFT_FORWARD && direction != FFT_INVERSE) return FFT_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15)) return FFT_ERR_MISALIGNED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FFT_ERR_CUDA;
    fft_status s = setup_device(dev);
    if (s != FFT_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool inv = direction == FFT_INVERSE;

    // N = N1 * N2: columns of length N1 with the W_N^{n2 k1} twiddle into the
    // static workspace, then rows of length N2 stored transposed into out.
    const int l1 = logn / 2, l2 = logn - l1;
    const int64_t n1 = int64_t(1) << l1, n2 = int64_t(1) << l2;
    const int c = cols_width_for(l1, n2);
    int tpc = c < 2 ? 2 : c;
    while (tpc > 2 && (rowsT_threads(l2, tpc) > 1024 || n1 % tpc != 0)) tpc /= 2;
    if (c == 0 || rowsT_threads(l2, tpc) > 1024 || n1 % tpc != 0) return FFT_ERR_UNSUPPORTED;

    // twiddle tables of this n, built on the caller's stream when the
    // device's array holds another length's (calls are ordered on the GPU, so
    // a later call with the same n reads what an earlier one wrote)
    float2* tab = g_static_tab_ptr[dev];
    const int sh = (logn + 1) / 2;
    const int64_t ea = pow2_table_entries(l1), eb = pow2_table_entries(l2);
    const int64_t elo = int64_t(1) << sh, ehi = int64_t(1) << (logn - sh);
    const int64_t off_b = ea, off_lo = ea + eb, off_hi = off_lo + elo;
    if (off_hi + ehi > kStaticTableEntries) return FFT_ERR_UNSUPPORTED;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (g_static_tab_n[dev] != n) {
            g_static_tab_n[dev] = 0;
            if (gen_pow2_table(tab, l1, st) != cudaSuccess) return FFT_ERR_CUDA;
            if (gen_pow2_table(tab + off_b, l2, st) != cudaSuccess) return FFT_ERR_CUDA;
            if (gen_root_table(tab + off_lo, elo, 1, n, st) != cudaSuccess) return FFT_ERR_CUDA;
            if (gen_root_table(tab + off_hi, ehi, elo, n, st) != cudaSuccess) return FFT_ERR_CUDA;
            g_static_tab_n[dev] = n;
        }
    }

    float2* work = g_static_work_ptr[dev];
    const float2* x = static_cast<const float2*>(in);
    if (launch_cols(l1, c, inv, true, x, work, n2, n2, n, batch, tab, tab + off_lo, tab + off_hi, sh, st) !=
        cudaSuccess)
        return FFT_ERR_CUDA;
    if (launch_rowsT(l2, tpc, inv, work, static_cast<float2*>(out), batch * n1, tab + off_b, n1, st) != cudaSuccess)
        return FFT_ERR_CUDA;
    return FFT_OK;
}

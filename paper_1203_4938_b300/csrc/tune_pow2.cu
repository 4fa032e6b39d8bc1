// tune_pow2.cu -- autotuner of the batched power-of-two planner.
//
// For one length 2^logn and batch, every kernel family and shape the library
// has compiled for that length is a candidate: the single-pass rows kernel
// (logn <= 14; at 2^13 / 2^14 also its persistent form with staged input),
// each persistent four-step split and tile width, with plain or
// asynchronous (tensor-memory-accelerator ring) loads and two chunk sizes,
// and each three-stage split with 4096- or 16384-point tiles, with plain or
// asynchronous loads.  A candidate
// is built as a real plan (the planner honours the forced choice), run twice
// to warm up and then timed over five forward executions with CUDA events on
// a scratch batch of the same size; the fastest wins.  Picks are cached per
// process and, when FFT_TUNE_CACHE names a file, appended to that file, so a
// later process (or a later plan of the same shape) reuses them.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fft.h"
#include "launch.h"
#include "plan.h"

namespace b300fft {

namespace {

thread_local const Pow2Choice* t_force = nullptr;
std::mutex g_mu;
bool g_loaded = false;
std::map<std::string, Pow2Choice> g_cache;

std::string device_key() {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp pr{};
    cudaGetDeviceProperties(&pr, dev);
    std::string s = pr.name;
    for (auto& c : s)
        if (c == ' ') c = '_';
    return s;
}

void cache_load() {
    if (g_loaded) return;
    g_loaded = true;
    const char* path = std::getenv("FFT_TUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    char line[512], key[256];
    while (std::fgets(line, sizeof line, f)) {
        if (std::strncmp(line, "pow2:", 5) != 0) continue;
        Pow2Choice c;
        if (std::sscanf(line, "%255s %d %d %d %d %d %d %d %d", key, &c.family, &c.a, &c.b, &c.c, &c.d, &c.chunk_mb,
                        &c.pipe, &c.lookahead) == 9)
            g_cache[key] = c;
    }
    std::fclose(f);
}

void cache_store(const std::string& key, const Pow2Choice& c, double us) {
    g_cache[key] = c;
    const char* path = std::getenv("FFT_TUNE_CACHE");
    if (!path) return;
    if (FILE* f = std::fopen(path, "a")) {
        std::fprintf(f, "%s %d %d %d %d %d %d %d %d %.2f\n", key.c_str(), c.family, c.a, c.b, c.c, c.d, c.chunk_mb,
                     c.pipe, c.lookahead, us);
        std::fclose(f);
    }
}

std::vector<Pow2Choice> candidates(int logn) {
    std::vector<Pow2Choice> out;
    if (logn <= kRowsMaxLog) {
        Pow2Choice c;
        c.family = 1;
        out.push_back(c);
        if (rows_staged_available(logn)) {
            c.pipe = 1;  // persistent, bulk-copied input staging
            out.push_back(c);
        }
    }
    for (int l1 = 6; l1 <= 12; ++l1) {
        const int l2 = logn - l1;
        if (l2 < 6 || l2 > 12) continue;
        for (int cw = 2; cw <= 64; cw *= 2)
            for (int tpc = 2; tpc <= 64; tpc *= 2) {
                const PersistConfig pc{l1, cw, l2, tpc};
                if (!persist_config_available(pc)) continue;
                for (int mb : {16, 32}) {
                    Pow2Choice c;
                    c.family = 2;
                    c.a = l1;
                    c.b = cw;
                    c.c = l2;
                    c.d = tpc;
                    c.chunk_mb = mb;
                    out.push_back(c);
                }
                for (int ns : {2, 3})
                    if (pipe_config_available(pc, ns)) {
                        Pow2Choice c;
                        c.family = 2;
                        c.a = l1;
                        c.b = cw;
                        c.c = l2;
                        c.d = tpc;
                        c.chunk_mb = 32;
                        c.pipe = ns;
                        out.push_back(c);
                    }
            }
    }
    for (int la = 6; la <= 8; ++la)
        for (int lb1 = 6; lb1 <= 8; ++lb1) {
            const int lb2 = logn - la - lb1;
            if (lb2 < 6 || lb2 > 8) continue;
            for (int tile : {4096, 16384}) {
                const ThreeConfig tc{la, lb1, lb2, tile};
                if (!three_config_available(tc)) continue;
                Pow2Choice c;
                c.family = 3;
                c.a = la;
                c.b = lb1;
                c.c = lb2;
                c.d = tile;
                c.chunk_mb = 32;
                out.push_back(c);
                for (int ns : {2, 3})
                    if (three_pipe_available(tc, ns)) {
                        Pow2Choice q = c;
                        q.pipe = ns;
                        out.push_back(q);
                    }
            }
        }
    return out;
}

}  // namespace

const Pow2Choice* pow2_forced() { return t_force; }
void pow2_force(const Pow2Choice* c) { t_force = c; }

bool tune_pow2(int logn, int64_t batch, Pow2Choice* best) {
    std::lock_guard<std::mutex> lk(g_mu);
    cache_load();
    const std::string key =
        "pow2:" + device_key() + ":" + std::to_string(logn) + ":" + std::to_string((long long)batch);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
        *best = it->second;
        return true;
    }
    const std::vector<Pow2Choice> cand = candidates(logn);
    if (cand.size() < 2) return false;
    const int64_t n = int64_t(1) << logn;
    const size_t bytes = sizeof(float2) * (size_t)n * (size_t)batch;
    float2 *x = nullptr, *y = nullptr;
    if (cudaMalloc(&x, bytes) != cudaSuccess || cudaMalloc(&y, bytes) != cudaSuccess) {
        cudaFree(x);
        cudaFree(y);
        cudaGetLastError();
        return false;
    }
    cudaMemset(x, 0x3c, bytes);  // finite, non-zero values
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    bool found = false;
    constexpr int kReps = 5;
    for (const Pow2Choice& c : cand) {
        pow2_force(&c);
        fft_plan p = fft_plan_create(1, &n, batch, FFT_FP32);
        pow2_force(nullptr);
        if (!p) continue;
        bool ok = fft_exec(p, x, y, FFT_FORWARD, nullptr) == FFT_OK && fft_exec(p, x, y, FFT_FORWARD, nullptr) == FFT_OK;
        cudaEventRecord(e0);
        for (int r = 0; ok && r < kReps; ++r) ok = fft_exec(p, x, y, FFT_FORWARD, nullptr) == FFT_OK;
        cudaEventRecord(e1);
        ok = ok && cudaEventSynchronize(e1) == cudaSuccess && fft_plan_check(p) == FFT_OK;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        fft_plan_destroy(p);
        if (ok && ms < best_ms) {
            best_ms = ms;
            *best = c;
            found = true;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(x);
    cudaFree(y);
    if (found) cache_store(key, *best, best_ms * 1e3 / kReps);
    return found;
}

}  // namespace b300fft

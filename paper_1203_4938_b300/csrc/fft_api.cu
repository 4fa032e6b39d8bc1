// fft_api.cu -- plans and the C ABI declared in include/fft.h.
//
// A plan is the analogue of the paper's cached program (Sec. II-D, the run
// protocol's program ID): everything that depends only on the shape -- the
// factorisation, the FP64-evaluated twiddle tables, the workspace, the kernel
// configuration -- is built once by fft_plan_create, and fft_exec only
// enqueues kernels on the caller's stream.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <string>

#include "../../include/fft.h"
#include "gplan.h"
#include "launch.h"
#include "persist.cuh"
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
    if (p->inner) {
        fft_plan_destroy(p->inner);
        p->inner = nullptr;
    }
    if (p->inner2) {
        fft_plan_destroy(p->inner2);
        p->inner2 = nullptr;
    }
    if (p->gplan) {
        graph_plan_free(p->gplan);
        delete p->gplan;
        p->gplan = nullptr;
    }
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

int env_int(const char* name, int dflt) {
    const char* v = std::getenv(name);
    return (v && *v) ? std::atoi(v) : dflt;
}

// Persistent four-step: both passes in one launch with L2-resident chunks.
fft_status build_fourstep_persist(fft_plan_s* p, int logn) {
    // Measured best (l1, c, l2, tpc, chunk MiB) per log2 N on a B300 with 2^26
    // elements per exec (2^13 and 2^14 are faster as one single-CTA pass).
    static const int kCfg[25][5] = {
        {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0},
        {7, 32, 8, 16, 32}, {8, 16, 8, 16, 16}, {8, 16, 9, 8, 32}, {8, 16, 10, 4, 32}, {9, 16, 10, 8, 16},
        {10, 8, 10, 8, 16}, {10, 16, 11, 8, 16}, {11, 4, 11, 4, 32}, {12, 4, 11, 8, 48}, {12, 4, 12, 4, 8}};
    const Pow2Choice* force = pow2_forced();
    if (force && force->family != 2) force = nullptr;
    const bool forced = force || std::getenv("B300FFT_PERSIST_CFG") != nullptr;
    if (logn > 24 || (kCfg[logn][0] == 0 && !forced)) return FFT_ERR_UNSUPPORTED;
    PersistConfig cfg{kCfg[logn][0], kCfg[logn][1], kCfg[logn][2], kCfg[logn][3]};
    if (const char* v = std::getenv("B300FFT_PERSIST_CFG")) {
        PersistConfig o{};
        if (std::sscanf(v, "%d,%d,%d,%d", &o.l1, &o.c, &o.l2, &o.tpc) == 4 && o.l1 + o.l2 == logn) cfg = o;
    }
    if (force) cfg = PersistConfig{force->a, force->b, force->c, force->d};
    if (cfg.l1 + cfg.l2 != logn) return FFT_ERR_UNSUPPORTED;
    // Asynchronous-load form (k_pipe.cu): slots in its shared-memory ring per
    // log2 N, 0 = the plain persistent kernel (measured slower at every size
    // of the sweep, so off by default; B300FFT_PIPE=2 or 3 selects it).
    const int pipe_ns = force ? force->pipe : env_int("B300FFT_PIPE", 0);
    PersistInfo info;
    p->ppipe = 0;
    if (pipe_ns && pipe_config_available(cfg, pipe_ns) && pipe_prepare(cfg, pipe_ns, &info) == cudaSuccess &&
        info.blocks_per_sm >= 1) {
        p->ppipe = pipe_ns;
    } else {
        if (!persist_config_available(cfg)) return FFT_ERR_UNSUPPORTED;
        if (persist_prepare(cfg, &info) != cudaSuccess || info.blocks_per_sm < 1) return FFT_ERR_CUDA;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t n = int64_t(1) << logn, n1 = int64_t(1) << cfg.l1, n2 = int64_t(1) << cfg.l2;
    const int64_t chunk_bytes =
        int64_t(force && force->chunk_mb ? force->chunk_mb
                                         : env_int("B300FFT_CHUNK_MB", kCfg[logn][4] ? kCfg[logn][4] : 32))
        << 20;
    int64_t cb = chunk_bytes / (n * 8);
    if (cb < 1) cb = 1;
    if (cb > p->batch) cb = p->batch;
    const int64_t nch = (p->batch + cb - 1) / cb;
    const int64_t na = cb * (n2 / cfg.c), nb = cb * (n1 / cfg.tpc);
    if (nch * (na + nb) > 0x7fffffffLL) return FFT_ERR_UNSUPPORTED;
    p->kind = PlanKind::FourStepPersist;
    p->pl1 = cfg.l1;
    p->pc = cfg.c;
    p->pl2 = cfg.l2;
    p->ptpc = cfg.tpc;
    p->pcb = cb;
    p->pnch = (int)nch;
    p->pna = (int)na;
    p->pnb = (int)nb;
    const int64_t items = nch * (na + nb);
    const int64_t slots = (int64_t)sms * info.blocks_per_sm;
    p->pgrid = (int)(items < slots ? items : slots);
    p->spin_limit = env_int("B300FFT_SPIN_LIMIT", 1 << 23);
    p->withhold_chunk = env_int("B300FFT_DEBUG_WITHHOLD_CHUNK", -1);
    p->sh = (logn + 1) / 2;
    const size_t ea = (size_t)pow2_table_entries(cfg.l1), eb = (size_t)pow2_table_entries(cfg.l2);
    const size_t elo = size_t(1) << p->sh, ehi = size_t(1) << (logn - p->sh);
    p->off_a = 0;
    p->off_b = ea;
    p->off_lo = ea + eb;
    p->off_hi = p->off_lo + elo;
    fft_status s = alloc_tables(p, p->off_hi + ehi);
    if (s != FFT_OK) return s;
    if (gen_pow2_table(p->d_tables + p->off_a, cfg.l1, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (gen_pow2_table(p->d_tables + p->off_b, cfg.l2, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (gen_root_table(p->d_tables + p->off_lo, (int64_t)elo, 1, n, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (gen_root_table(p->d_tables + p->off_hi, (int64_t)ehi, (int64_t)elo, n, 0) != cudaSuccess)
        return FFT_ERR_CUDA;
    p->work_bytes = (size_t)n * (size_t)p->batch * sizeof(float2);
    if (cudaMalloc(&p->d_work, p->work_bytes) != cudaSuccess) return FFT_ERR_ALLOC;
    if (cudaMalloc(&p->d_aux, sizeof(int) * (size_t)(1 + nch)) != cudaSuccess) return FFT_ERR_ALLOC;
    p->kernels = 1;
    std::snprintf(p->desc, sizeof p->desc,
                  "fourstep-persist N=2^%d = 2^%d (C=%d) x 2^%d (tpc=%d) threads=%d grid=%d chunk=%lld x %lld%s",
                  logn, cfg.l1, cfg.c, cfg.l2, cfg.tpc, info.threads, p->pgrid, (long long)cb, (long long)nch,
                  p->ppipe == 3 ? " tma-ring=3" : (p->ppipe == 2 ? " tma-ring=2" : ""));
    return FFT_OK;
}

// Persistent three-stage: N = N1 * M1 * M2 with 2^6 .. 2^8-point stages.
// kThree[log2 N] = {log2 N1, log2 M1, log2 M2, chunk MiB, default on, tile points}.
// Measured on a B300 with 2^26 elements per exec: faster than the two-pass
// persistent four-step from 2^22 on (2^19 and 2^20 are slower, and at 2^21
// the two-pass kernel with 16384-point tiles on 1024 threads wins: 473 vs
// 501 us).  Chunks of
// 32 MiB (one or two transforms): 2^21 494 us vs 503 us with 128 MiB chunks;
// letting the A stage run more than one chunk ahead was slower at every size.
static const int kThree[25][6] = {
    {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0},
    {6, 6, 7, 128, 0, 4096}, {6, 7, 7, 128, 0, 4096}, {7, 7, 7, 32, 0, 4096}, {7, 7, 8, 32, 1, 4096},
    {8, 7, 8, 32, 1, 4096}, {8, 8, 8, 32, 1, 4096}};

bool three_preferred(int logn) { return logn >= 0 && logn <= 24 && kThree[logn][4] != 0; }

fft_status build_threestep(fft_plan_s* p, int logn) {
    const Pow2Choice* force = pow2_forced();
    if (force && force->family != 3) force = nullptr;
    const char* forced = std::getenv("B300FFT_THREE_CFG");
    if (logn > 24 || (kThree[logn][0] == 0 && !forced && !force)) return FFT_ERR_UNSUPPORTED;
    ThreeConfig cfg{kThree[logn][0], kThree[logn][1], kThree[logn][2], kThree[logn][5]};
    if (forced) {
        ThreeConfig o{};
        if (std::sscanf(forced, "%d,%d,%d", &o.la, &o.lb1, &o.lb2) == 3 && o.la + o.lb1 + o.lb2 == logn) cfg = o;
    }
    cfg.tile = env_int("B300FFT_THREE_TILE", cfg.tile);
    if (force) cfg = ThreeConfig{force->a, force->b, force->c, force->d};
    if (cfg.la + cfg.lb1 + cfg.lb2 != logn) return FFT_ERR_UNSUPPORTED;
    // asynchronous-load form (k_three_pipe.cu): ring slots, 0 = plain kernel
    // (measured slower at every size, so off by default)
    const int pipe_ns = force ? force->pipe : env_int("B300FFT_PIPE", 0);
    PersistInfo info;
    p->ppipe = 0;
    if (pipe_ns && three_pipe_available(cfg, pipe_ns) && three_pipe_prepare(cfg, pipe_ns, &info) == cudaSuccess &&
        info.blocks_per_sm >= 1) {
        p->ppipe = pipe_ns;
    } else {
        if (!three_config_available(cfg)) return FFT_ERR_UNSUPPORTED;
        if (three_prepare(cfg, &info) != cudaSuccess || info.blocks_per_sm < 1) return FFT_ERR_CUDA;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t n = int64_t(1) << logn;
    const int64_t n1 = int64_t(1) << cfg.la, m1 = int64_t(1) << cfg.lb1, m2 = int64_t(1) << cfg.lb2;
    const int64_t n2 = m1 * m2;
    const int64_t ca = cfg.tile >> cfg.la, cb_cols = cfg.tile >> cfg.lb1, tpc = cfg.tile >> cfg.lb2;
    const int64_t chunk_bytes =
        int64_t(force && force->chunk_mb ? force->chunk_mb
                                         : env_int("B300FFT_CHUNK_MB", kThree[logn][3] ? kThree[logn][3] : 32))
        << 20;
    int64_t cb = chunk_bytes / (n * 8);
    if (cb < 1) cb = 1;
    if (cb > p->batch) cb = p->batch;
    const int64_t nch = (p->batch + cb - 1) / cb;
    const int64_t na = cb * (n2 / ca);
    const int64_t G = cb * (n1 / tpc), nb1g = tpc * (m2 / cb_cols), nb2g = m1;
    const int64_t nb = G * (nb1g + nb2g);
    if (nch * (na + nb) > 0x7fffffffLL || nch * G > (1 << 26)) return FFT_ERR_UNSUPPORTED;
    p->kind = PlanKind::ThreeStep;
    p->pl1 = cfg.la;
    p->pc = cfg.lb1;
    p->pl2 = cfg.lb2;
    p->ptpc = cfg.tile;
    p->pcb = cb;
    p->pnch = (int)nch;
    p->pna = (int)na;
    p->pnb = (int)nb;
    p->pG = (int)G;
    p->pnb1g = (int)nb1g;
    p->pnb2g = (int)nb2g;
    const int64_t items = nch * (na + nb);
    const int64_t slots = (int64_t)sms * info.blocks_per_sm;
    p->pgrid = (int)(items < slots ? items : slots);
    // B1 lookahead: at least twice the CTAs in flight between a B1 tile and its first consumer
    int64_t D = (2 * (int64_t)p->pgrid + nb1g - 1) / nb1g;
    D = force && force->lookahead > 0 ? force->lookahead : env_int("B300FFT_THREE_LOOKAHEAD", (int)D);
    if (D < 1) D = 1;
    if (D > G) D = G;
    p->pD = (int)D;
    p->spin_limit = env_int("B300FFT_SPIN_LIMIT", 1 << 23);
    p->withhold_chunk = env_int("B300FFT_DEBUG_WITHHOLD_CHUNK", -1);
    // L2 tensor prefetch of the next A / B1 tile's box: measured 0.4-0.8 %
    // faster at 2^23 and 2^24 (whose workspace spills to DRAM) and 2 % slower
    // at 2^21 and 2^22 (2^26 elements per exec), so on from 2^23
    p->pprefetch = env_int("B300FFT_PREFETCH", logn >= 23 ? 1 : 0) != 0 && tensor_maps_available() ? 1 : 0;
    p->sh = (logn + 1) / 2;
    const size_t ea = (size_t)pow2_table_entries(cfg.la), eb = (size_t)pow2_table_entries(cfg.lb1),
                 ec = (size_t)pow2_table_entries(cfg.lb2);
    const size_t elo = size_t(1) << p->sh, ehi = size_t(1) << (logn - p->sh);
    p->off_a = 0;
    p->off_b = ea;
    p->off_c = ea + eb;
    p->off_lo = ea + eb + ec;
    p->off_hi = p->off_lo + elo;
    fft_status s = alloc_tables(p, p->off_hi + ehi);
    if (s != FFT_OK) return s;
    if (gen_pow2_table(p->d_tables + p->off_a, cfg.la, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (gen_pow2_table(p->d_tables + p->off_b, cfg.lb1, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (gen_pow2_table(p->d_tables + p->off_c, cfg.lb2, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (gen_root_table(p->d_tables + p->off_lo, (int64_t)elo, 1, n, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (gen_root_table(p->d_tables + p->off_hi, (int64_t)ehi, (int64_t)elo, n, 0) != cudaSuccess)
        return FFT_ERR_CUDA;
    p->work_bytes = (size_t)n * (size_t)p->batch * sizeof(float2);
    if (cudaMalloc(&p->d_work, p->work_bytes) != cudaSuccess) return FFT_ERR_ALLOC;
    if (cudaMalloc(&p->d_aux, sizeof(int) * (size_t)(1 + nch + nch * G)) != cudaSuccess) return FFT_ERR_ALLOC;
    p->kernels = 1;
    std::snprintf(p->desc, sizeof p->desc,
                  "threestep N=2^%d = 2^%d x (2^%d x 2^%d) threads=%d grid=%d chunk=%lld x %lld groups=%lld ahead=%lld%s",
                  logn, cfg.la, cfg.lb1, cfg.lb2, info.threads, p->pgrid, (long long)cb, (long long)nch, (long long)G,
                  (long long)D, p->ppipe == 3 ? " tma-ring=3" : (p->ppipe == 2 ? " tma-ring=2" : ""));
    return FFT_OK;
}

// Thread-block-cluster single pass: N = K * 2^lm, one transform per cluster.
// kCluster[log2 N] = {lm, K, default on}.
static const int kCluster[18][3] = {{0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0},
                                    {12, 8, 0}, {13, 8, 0}, {14, 8, 0}};

fft_status build_cluster(fft_plan_s* p, int logn, bool forced) {
    if (logn < 15 || logn > 17) return FFT_ERR_UNSUPPORTED;
    int lm = kCluster[logn][0], k = kCluster[logn][1];
    if (!forced && !kCluster[logn][2]) return FFT_ERR_UNSUPPORTED;
    if (const char* v = std::getenv("B300FFT_CLUSTER_CFG")) {
        int a = 0, b = 0;
        if (std::sscanf(v, "%d,%d", &a, &b) == 2 && (int64_t(b) << a) == (int64_t(1) << logn)) {
            lm = a;
            k = b;
        }
    }
    if (!cluster_config_available(lm, k) || (int64_t(k) << lm) != (int64_t(1) << logn)) return FFT_ERR_UNSUPPORTED;
    if ((int64_t)k * p->batch > 0x7fffffffLL) return FFT_ERR_UNSUPPORTED;
    int clusters = 0;
    if (cluster_prepare(lm, k, &clusters) != cudaSuccess) {
        cudaGetLastError();
        return FFT_ERR_UNSUPPORTED;
    }
    if (clusters < 1) return FFT_ERR_UNSUPPORTED;
    p->kind = PlanKind::Cluster;
    p->cl_lm = lm;
    p->cl_k = k;
    p->sh = (logn + 1) / 2;
    const int64_t n = int64_t(1) << logn;
    const size_t ea = (size_t)pow2_table_entries(lm);
    const size_t elo = size_t(1) << p->sh, ehi = size_t(1) << (logn - p->sh);
    p->off_a = 0;
    p->off_lo = ea;
    p->off_hi = ea + elo;
    fft_status s = alloc_tables(p, p->off_hi + ehi);
    if (s != FFT_OK) return s;
    if (gen_pow2_table(p->d_tables + p->off_a, lm, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (gen_root_table(p->d_tables + p->off_lo, (int64_t)elo, 1, n, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (gen_root_table(p->d_tables + p->off_hi, (int64_t)ehi, (int64_t)elo, n, 0) != cudaSuccess)
        return FFT_ERR_CUDA;
    p->kernels = 1;
    std::snprintf(p->desc, sizeof p->desc,
                  "cluster N=2^%d = %d CTAs x 2^%d (DSMEM exchange) threads=%d co-resident clusters=%d", logn, k, lm,
                  (1 << lm) / 16, clusters);
    return FFT_OK;
}

fft_status build_pow2_1d(fft_plan_s* p, int logn) {
    // FFT_AUTOTUNE=1: time the candidate kernels and shapes for this length and
    // batch (tune_pow2.cu) and build the fastest
    Pow2Choice pick;
    if (!pow2_forced() && env_int("FFT_AUTOTUNE", 0) != 0 && tune_pow2(logn, p->batch, &pick)) {
        pow2_force(&pick);
        fft_status s = build_pow2_1d(p, logn);
        pow2_force(nullptr);
        return s;
    }
    const Pow2Choice* force = pow2_forced();
    if (force) {  // exactly the forced family, or unsupported
        if (force->family == 1) {
            if (logn > kRowsMaxLog) return FFT_ERR_UNSUPPORTED;
        } else if (force->family == 2) {
            return build_fourstep_persist(p, logn);
        } else if (force->family == 3) {
            return build_threestep(p, logn);
        } else {
            return FFT_ERR_UNSUPPORTED;
        }
    }
    p->single_max_log = env_int("B300FFT_SINGLE_MAX_LOG", p->single_max_log);
    if (force || (logn <= p->single_max_log && logn <= kRowsMaxLog)) {
        p->kind = PlanKind::Rows;
        p->logn_a = logn;
        p->off_a = 0;
        size_t ent = (size_t)pow2_table_entries(logn);
        fft_status s = alloc_tables(p, ent);
        if (s != FFT_OK) return s;
        if (gen_pow2_table(p->d_tables + p->off_a, logn, 0) != cudaSuccess) return FFT_ERR_CUDA;
        if (rows_prepare(logn) != cudaSuccess) return FFT_ERR_CUDA;
        p->kernels = 1;
        // 2^14: the persistent form with bulk-copied input staging
        // (B300FFT_ROWS_STAGED=0|1 overrides)
        p->rows_staged = 0;
        const int staged = force ? force->pipe : env_int("B300FFT_ROWS_STAGED", rows_staged_default(logn));
        PersistInfo info;
        if (staged && rows_staged_available(logn) && rows_staged_prepare(logn, &info) == cudaSuccess &&
            info.blocks_per_sm >= 1) {
            int dev = 0, sms = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const int64_t slots = (int64_t)sms * info.blocks_per_sm;
            p->rows_staged = 1;
            p->pgrid = (int)(p->batch < slots ? p->batch : slots);
            p->spin_limit = env_int("B300FFT_SPIN_LIMIT", 1 << 23);
            std::snprintf(p->desc, sizeof p->desc, "rows N=2^%d staged threads=%d grid=%d", logn, info.threads,
                          p->pgrid);
            return FFT_OK;
        }
        if (force && force->pipe) return FFT_ERR_UNSUPPORTED;
        std::snprintf(p->desc, sizeof p->desc, "rows N=2^%d tpc=%d threads=%d", logn, rows_tpc(logn),
                      rows_threads(logn));
        return FFT_OK;
    }
    // cluster single pass where it is measured faster; B300FFT_CLUSTER=1 forces it, 0 disables it
    {
        const int cl = env_int("B300FFT_CLUSTER", -1);
        if (cl != 0) {
            fft_status cs = build_cluster(p, logn, cl == 1);
            if (cs != FFT_ERR_UNSUPPORTED) return cs;
        }
    }
    // three-stage form where it is measured faster; B300FFT_THREE=1 forces it, 0 disables it
    const int three = env_int("B300FFT_THREE", -1);
    if (three == 1 || (three < 0 && three_preferred(logn))) {
        fft_status ts = build_threestep(p, logn);
        if (ts != FFT_ERR_UNSUPPORTED) return ts;
    }
    if (env_int("B300FFT_PERSIST", 1)) {
        fft_status ps = build_fourstep_persist(p, logn);
        if (ps != FFT_ERR_UNSUPPORTED) return ps;
    }
    // four-step: N = N1 * N2, pass A = columns of length N1 (stride N2) with
    // the W_N^{n2 k1} twiddle, pass B = rows of length N2, transposed store.
    // Measured best (split log2 N1, column width, transposed rows per CTA)
    // for each log2 N on a B300 with 2^26 elements per exec.
    static const int kTuned[25][3] = {
        {0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0},
        {0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {7, 16, 32}, {7, 16, 32}, {7, 16, 8}, {8, 16, 8},
        {8, 16, 8}, {8, 16, 8}, {8, 8, 4}, {9, 4, 4}, {10, 4, 4}, {11, 4, 4}, {12, 4, 4}, {12, 4, 4}};
    const bool tuned = logn <= 24 && kTuned[logn][0] > 0;
    int l1 = env_int("B300FFT_SPLIT_L1", tuned ? kTuned[logn][0] : logn / 2);
    if (l1 < 1 || l1 >= logn) l1 = logn / 2;
    const int l2 = logn - l1;
    if (l2 > kColsMaxLog || l1 > kColsMaxLog || l2 < 5) return FFT_ERR_UNSUPPORTED;
    const int64_t n1 = int64_t(1) << l1, n2 = int64_t(1) << l2;
    int c = env_int("B300FFT_COLS_C", tuned ? kTuned[logn][1] : cols_width(l1));
    if (!cols_width_valid(l1, c) || n2 % c != 0) c = cols_width_for(l1, n2);
    if (c == 0) return FFT_ERR_UNSUPPORTED;
    int tpc = env_int("B300FFT_ROWST_TPC", tuned ? kTuned[logn][2] : (c < 2 ? 2 : c));
    while (tpc > 2 && (rowsT_threads(l2, tpc) > 1024 || n1 % tpc != 0)) tpc /= 2;
    if (tpc < 2 || n1 % tpc != 0 || rowsT_threads(l2, tpc) > 1024) return FFT_ERR_UNSUPPORTED;
    p->kind = PlanKind::FourStep;
    p->cols_c = c;
    p->rowsT_tpc = tpc;
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
    if (cols_prepare(l1, c) != cudaSuccess || rowsT_prepare(l2, tpc) != cudaSuccess) return FFT_ERR_CUDA;
    p->kernels = 2;
    std::snprintf(p->desc, sizeof p->desc,
                  "fourstep N=2^%d = 2^%d (cols C=%d threads=%d) x 2^%d (rowsT tpc=%d threads=%d) work=%zuB", logn,
                  l1, c, cols_threads(l1, c), l2, tpc, rowsT_threads(l2, tpc), p->work_bytes);
    return FFT_OK;
}

// Persistent 2-D with L2-resident chunks of images (square sizes with a
// tiling below; images of more than 48 MiB keep the two-launch form).
// kTwoD[log2 side] = {rows per row tile, columns per column tile, chunk MiB}.
fft_status build_2d_persist(fft_plan_s* p, int logh, int logw) {
    static const int kTwoD[12][3] = {{0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {8, 8, 32}, {8, 8, 32}, {4, 4, 32}};
    if (logh != logw || logw < 9 || logw > 11) return FFT_ERR_UNSUPPORTED;
    const int64_t hw = int64_t(1) << (logh + logw);
    if (hw * 8 > (int64_t(48) << 20)) return FFT_ERR_UNSUPPORTED;
    PersistConfig cfg{logw, kTwoD[logw][0], logh, kTwoD[logw][1]};
    if (const char* v = std::getenv("B300FFT_2D_CFG")) {
        int tpc = 0, c = 0;
        if (std::sscanf(v, "%d,%d", &tpc, &c) == 2) {
            cfg.c = tpc;
            cfg.tpc = c;
        }
    }
    if (!persist2d_config_available(cfg)) return FFT_ERR_UNSUPPORTED;
    PersistInfo info;
    if (persist2d_prepare(cfg, &info) != cudaSuccess || info.blocks_per_sm < 1) return FFT_ERR_CUDA;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t chunk_bytes = int64_t(env_int("B300FFT_CHUNK_MB", kTwoD[logw][2])) << 20;
    int64_t cb = chunk_bytes / (hw * 8);
    if (cb < 1) cb = 1;
    if (cb > p->batch) cb = p->batch;
    const int64_t nch = (p->batch + cb - 1) / cb;
    const int64_t na = cb * ((int64_t(1) << logh) / cfg.c), nb = cb * ((int64_t(1) << logw) / cfg.tpc);
    if (nch * (na + nb) > 0x7fffffffLL) return FFT_ERR_UNSUPPORTED;
    p->kind = PlanKind::TwoDPersist;
    p->logn_a = logw;
    p->logn_b = logh;
    p->pl1 = cfg.l1;
    p->pc = cfg.c;
    p->pl2 = cfg.l2;
    p->ptpc = cfg.tpc;
    p->pcb = cb;
    p->pnch = (int)nch;
    p->pna = (int)na;
    p->pnb = (int)nb;
    const int64_t items = nch * (na + nb), slots = (int64_t)sms * info.blocks_per_sm;
    p->pgrid = (int)(items < slots ? items : slots);
    p->spin_limit = env_int("B300FFT_SPIN_LIMIT", 1 << 23);
    p->withhold_chunk = env_int("B300FFT_DEBUG_WITHHOLD_CHUNK", -1);
    const size_t ea = (size_t)pow2_table_entries(logw), eb = (size_t)pow2_table_entries(logh);
    p->off_a = 0;
    p->off_b = ea;
    fft_status s = alloc_tables(p, ea + eb);
    if (s != FFT_OK) return s;
    if (gen_pow2_table(p->d_tables + p->off_a, logw, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (gen_pow2_table(p->d_tables + p->off_b, logh, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (cudaMalloc(&p->d_aux, sizeof(int) * (size_t)(1 + nch)) != cudaSuccess) return FFT_ERR_ALLOC;
    p->kernels = 1;
    std::snprintf(p->desc, sizeof p->desc,
                  "2d-persist H=2^%d W=2^%d: rows(tpc=%d) then cols(C=%d) threads=%d grid=%d chunk=%lld x %lld", logh,
                  logw, cfg.c, cfg.tpc, info.threads, p->pgrid, (long long)cb, (long long)nch);
    return FFT_OK;
}

fft_status build_pow2_2d(fft_plan_s* p, int logh, int logw) {
    if (env_int("B300FFT_PERSIST", 1)) {
        fft_status ps = build_2d_persist(p, logh, logw);
        if (ps != FFT_ERR_UNSUPPORTED) return ps;
    }
    if (logw > kRowsMaxLog || logh > kColsMaxLog || logh < 1) return FFT_ERR_UNSUPPORTED;
    p->kind = PlanKind::TwoD;
    p->logn_a = logw;  // rows pass
    p->logn_b = logh;  // columns pass
    int c = env_int("B300FFT_COLS_C", cols_width_for(logh, int64_t(1) << logw));
    if (!cols_width_valid(logh, c) || ((int64_t(1) << logw) % c) != 0) c = cols_width_for(logh, int64_t(1) << logw);
    if (c == 0) return FFT_ERR_UNSUPPORTED;
    p->cols_c = c;
    const size_t ea = (size_t)pow2_table_entries(logw), eb = (size_t)pow2_table_entries(logh);
    p->off_a = 0;
    p->off_b = ea;
    fft_status s = alloc_tables(p, ea + eb);
    if (s != FFT_OK) return s;
    if (gen_pow2_table(p->d_tables + p->off_a, logw, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (gen_pow2_table(p->d_tables + p->off_b, logh, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (rows_prepare(logw) != cudaSuccess || cols_prepare(logh, c) != cudaSuccess) return FFT_ERR_CUDA;
    p->kernels = 2;
    std::snprintf(p->desc, sizeof p->desc, "2d H=2^%d W=2^%d: rows(tpc=%d) then cols(C=%d threads=%d)", logh, logw,
                  rows_tpc(logw), c, cols_threads(logh, c));
    return FFT_OK;
}

fft_plan finish(fft_plan_s* p) {
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(FFT_ERR_CUDA, p);
    p->magic = kPlanMagic;
    {
        std::lock_guard<std::mutex> lk(g_registry_mu);
        g_registry.insert(p);
    }
    return p;
}

}  // namespace

namespace b300fft {

// N = M * 2^k > 4096 with M = 3, 5, 7.
bool mixed_fourstep_length(int64_t n, int* m, int* k) {
    if (n <= 4096) return false;
    for (int mm : {3, 5, 7}) {
        if (n % mm) continue;
        const int64_t q = n / mm;
        if (q & (q - 1)) continue;
        int kk = 0;
        while ((int64_t(1) << kk) < q) ++kk;
        *m = mm;
        *k = kk;
        return true;
    }
    return false;
}

// L = M * 2^K <= 4096 (M = 3, 5, 7): the compile-time single-pass kernel.
fft_status build_mixed_1d(fft_plan_s* p, int m, int k) {
    const int entries = mixed_table_entries(m, k);
    if (entries < 0) return FFT_ERR_UNSUPPORTED;
    fft_status s = alloc_tables(p, (size_t)entries);
    if (s != FFT_OK) return s;
    if (entries > 0 && gen_mixed_table(p->d_tables, m, k, 0) != cudaSuccess) return FFT_ERR_CUDA;
    p->kind = PlanKind::RowsMixed;
    p->mix_m = m;
    p->logn_a = k;
    p->kernels = 1;
    std::snprintf(p->desc, sizeof p->desc, "rows-mixed N=%lld = %d x 2^%d lines/CTA=%d threads=256",
                  (long long)p->len[0], m, k, mixed_lines_per_cta(m, k));
    return FFT_OK;
}

// N = M * 2^k > 4096 (M = 3, 5, 7): four-step N = N1 * N2 with N1 = M * 2^a
// columns by the compile-time mixed kernel, then N2 = 2^b rows by the
// power-of-two transposed-row kernel.  Measured on 2^24 elements per exec
// (sweep over b = 7..12 and 4..32 rows per CTA): b = 8 with 16 rows per CTA
// (128-byte store runs) from k = 12, N1 at most M * 2^6, then b grows to 12
// with 8 (b <= 11) or 4 rows per CTA; k < 12: a = 2.  Against b = min(12, k-2)
// with 4 rows: 49152 112.0 -> 103.9 us, 57344 109.2 -> 101.9 us.
// Returns FFT_ERR_UNSUPPORTED where no column kernel fits.
fft_status build_mixed_fourstep(fft_plan_s* p, int m, int k) {
    int a = k >= 12 ? k - 8 : 2;
    if (a > 6) a = 6;
    if (k - a > 12) a = k - 12;
    int b = env_int("B300FFT_MIXED_B", k - a);
    if (b < 6 || b > 12 || b > k) return FFT_ERR_UNSUPPORTED;
    a = k - b;
    const int c = mixed_cols_width(m, a);
    if (b < 6 || c == 0 || c > (1 << b)) return FFT_ERR_UNSUPPORTED;
    const int64_t n1 = int64_t(m) << a, n2 = int64_t(1) << b, n = n1 * n2;
    int tpc = env_int("B300FFT_MIXED_TPC", b <= 8 ? 16 : (b <= 11 ? 8 : 4));
    if (tpc < 2 || tpc > 64 || (tpc & (tpc - 1))) tpc = 16;
    while (tpc > 2 && (rowsT_threads(b, tpc) > 1024 || n1 % tpc != 0)) tpc /= 2;
    if (n1 % tpc != 0 || rowsT_threads(b, tpc) > 1024) return FFT_ERR_UNSUPPORTED;
    int lg = 0;
    while ((int64_t(1) << lg) < n) ++lg;
    p->sh = (lg + 1) / 2;
    const int ea = mixed_table_entries(m, a), eb = pow2_table_entries(b);
    if (ea < 0) return FFT_ERR_UNSUPPORTED;
    const int64_t elo = int64_t(1) << p->sh, ehi = (n + elo - 1) / elo;
    p->off_a = 0;
    p->off_b = (size_t)ea;
    p->off_lo = p->off_b + (size_t)eb;
    p->off_hi = p->off_lo + (size_t)elo;
    fft_status s = alloc_tables(p, p->off_hi + (size_t)ehi);
    if (s != FFT_OK) return s;
    if (ea > 0 && gen_mixed_table(p->d_tables + p->off_a, m, a, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (gen_pow2_table(p->d_tables + p->off_b, b, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (gen_root_table(p->d_tables + p->off_lo, elo, 1, n, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (gen_root_table(p->d_tables + p->off_hi, ehi, elo, n, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (rowsT_prepare(b, tpc) != cudaSuccess) return FFT_ERR_CUDA;
    p->work_bytes = (size_t)n * (size_t)p->batch * sizeof(float2);
    if (cudaMalloc(&p->d_work, p->work_bytes) != cudaSuccess) return FFT_ERR_ALLOC;
    p->kind = PlanKind::FourStepMixed;
    p->mix_m = m;
    p->logn_a = a;
    p->logn_b = b;
    p->cols_c = c;
    p->rowsT_tpc = tpc;
    p->kernels = 2;
    std::snprintf(p->desc, sizeof p->desc,
                  "fourstep-mixed N=%lld = (%d x 2^%d, %d columns/CTA) x 2^%d (tpc=%d)", (long long)n, m, a, c, b,
                  tpc);
    return FFT_OK;
}

// 2-D [H][W] where each side is a power of two (rows <= 2^14, columns
// <= 2^12 points) or M * 2^K <= 4096 (M = 3, 5, 7) and at least one side is
// the latter: the rows kernel of W, then the in-place column pass over H.
fft_status build_mixed_2d(fft_plan_s* p, int64_t h, int64_t w) {
    int mh = 0, kh = 0, mw = 0, kw = 0;
    const int lh = ilog2_exact(h), lw = ilog2_exact(w);
    const bool mix_h = lh < 0 && mixed_supported(h, &mh, &kh), mix_w = lw < 0 && mixed_supported(w, &mw, &kw);
    if ((lh < 0 && !mix_h) || (lw < 0 && !mix_w)) return FFT_ERR_UNSUPPORTED;
    if ((!mix_w && lw > kRowsMaxLog) || (!mix_h && (lh > kColsMaxLog || lh < 1))) return FFT_ERR_UNSUPPORTED;
    int c = 0;
    if (mix_h) {
        c = mixed_cols2d_width(mh, kh);
        if (c == 0 || w % c != 0) return FFT_ERR_UNSUPPORTED;
    } else {
        c = cols_width_for(lh, w);
        if (c == 0) return FFT_ERR_UNSUPPORTED;
    }
    const int ea = mix_w ? mixed_table_entries(mw, kw) : pow2_table_entries(lw);
    const int eb = mix_h ? mixed_table_entries(mh, kh) : pow2_table_entries(lh);
    if (ea < 0 || eb < 0) return FFT_ERR_UNSUPPORTED;
    p->off_a = 0;
    p->off_b = (size_t)ea;
    fft_status s = alloc_tables(p, (size_t)ea + (size_t)eb);
    if (s != FFT_OK) return s;
    cudaError_t e = cudaSuccess;
    if (ea > 0) e = mix_w ? gen_mixed_table(p->d_tables, mw, kw, 0) : gen_pow2_table(p->d_tables, lw, 0);
    if (e == cudaSuccess && eb > 0)
        e = mix_h ? gen_mixed_table(p->d_tables + p->off_b, mh, kh, 0) : gen_pow2_table(p->d_tables + p->off_b, lh, 0);
    if (e == cudaSuccess && !mix_w) e = rows_prepare(lw);
    if (e == cudaSuccess && !mix_h) e = cols_prepare(lh, c);
    if (e != cudaSuccess) return FFT_ERR_CUDA;
    p->kind = PlanKind::TwoDMixed;
    p->mix_mw = mix_w ? mw : 0;
    p->mix_mh = mix_h ? mh : 0;
    p->logn_a = mix_w ? kw : lw;
    p->logn_b = mix_h ? kh : lh;
    p->cols_c = c;
    p->kernels = 2;
    std::snprintf(p->desc, sizeof p->desc, "2d-mixed H=%lld W=%lld: rows (%s) then cols (%s, %d per CTA)",
                  (long long)h, (long long)w, mix_w ? "mixed" : "power of two", mix_h ? "mixed" : "power of two", c);
    return FFT_OK;
}

// Any other H x W: the 2-D DFT as 1-D DFTs along the rows, then along the
// columns, with the column pass done on transposed data: a 1-D plan over the
// batch * H rows of length W (in -> out), a transpose (out -> workspace), a
// 1-D plan over the batch * W rows of length H (in place in the workspace) and
// a transpose back (workspace -> out).  Each 1-D plan is whatever
// fft_plan_create picks for its length (power of two, mixed radix,
// Bluestein), so every pair of supported 1-D lengths works in 2-D.
fft_status build_2d_transpose(fft_plan_s* p, int64_t h, int64_t w) {
    if (env_int("B300FFT_2D_TRANSPOSE", 1) == 0) return FFT_ERR_UNSUPPORTED;
    if (p->d_tables || p->d_work || p->d_aux || p->gplan) return FFT_ERR_UNSUPPORTED;  // a partly built plan
    // A pass over rows of length L = 2^5..2^12 runs as the four-step's
    // transposed-row kernel, which writes its output transposed straight away
    // (tpc rows of one image per CTA, tpc*8-byte store runs), so the transpose
    // after it disappears: the rows pass writes [batch][W][H] into the
    // workspace, the columns pass writes [batch][H][W] into `out`.  Measured
    // on a B300 (forward) against the plan + transpose form: rows pass
    // 8192 x 4096 344 vs 386 us, 8192 x 512 x 8 303 vs 379 us, 16384 x 64 x 64
    // 648 vs 835 us, 1000 x 1024 x 32 620 vs 705 us; columns pass 1024 x 1000
    // x 32 621 vs 706 us, 4096 x 1000 x 8 658 vs 711 us.
    const bool use = env_int("B300FFT_2D_ROWST", 1) != 0;
    auto pick = [use](int64_t len, int64_t rows_per_image) {
        const int l = ilog2_exact(len);
        if (!use || l < 5 || l > 12) return 0;
        for (int c = 16; c >= 4; c /= 2)
            if (rows_per_image % c == 0 && rowsT_threads(l, c) <= 1024 && rowsT_prepare(l, c) == cudaSuccess) return c;
        return 0;
    };
    const int tr = pick(w, h), tc = pick(h, w);  // rows pass: rows of W, H per image; columns: rows of H, W
    const size_t ea = tr ? (size_t)pow2_table_entries(ilog2_exact(w)) : 0;
    const size_t eb = tc ? (size_t)pow2_table_entries(ilog2_exact(h)) : 0;
    if (ea + eb > 0) {
        fft_status s = alloc_tables(p, ea + eb);
        if (s != FFT_OK) return s;
        p->off_a = 0;
        p->off_b = ea;
        if (tr && gen_pow2_table(p->d_tables + p->off_a, ilog2_exact(w), 0) != cudaSuccess) return FFT_ERR_CUDA;
        if (tc && gen_pow2_table(p->d_tables + p->off_b, ilog2_exact(h), 0) != cudaSuccess) return FFT_ERR_CUDA;
    }
    p->rowsT_tpc = tr;
    p->colsT_tpc = tc;
    p->logn_a = tr ? ilog2_exact(w) : 0;
    p->logn_b = tc ? ilog2_exact(h) : 0;
    const int64_t lw = w, lh = h;
    if (!tr) {
        p->inner = fft_plan_create(1, &lw, p->batch * h, FFT_FP32);
        if (!p->inner) return fft_last_error();
    }
    if (!tc) {
        p->inner2 = fft_plan_create(1, &lh, p->batch * w, FFT_FP32);
        if (!p->inner2) return fft_last_error();
    }
    p->work_bytes = (size_t)h * (size_t)w * (size_t)p->batch * sizeof(float2);
    if (cudaMalloc(&p->d_work, p->work_bytes) != cudaSuccess) return FFT_ERR_ALLOC;
    p->kind = PlanKind::TwoDTranspose;
    p->kernels = (tr ? 1 : fft_plan_kernel_count(p->inner) + 1) + (tc ? 1 : fft_plan_kernel_count(p->inner2) + 1);
    char a[110] = "", b[110] = "";
    if (tr) std::snprintf(a, sizeof a, "rows with transposed store (tpc=%d)", tr);
    else {
        std::snprintf(a, sizeof a, "rows [");
        fft_plan_describe(p->inner, a + 6, sizeof a - 8);
        std::strncat(a, "], transpose", sizeof a - std::strlen(a) - 1);
    }
    if (tc) std::snprintf(b, sizeof b, "columns with transposed store (tpc=%d)", tc);
    else {
        std::snprintf(b, sizeof b, "columns [");
        fft_plan_describe(p->inner2, b + 9, sizeof b - 11);
        std::strncat(b, "], transpose", sizeof b - std::strlen(b) - 1);
    }
    std::snprintf(p->desc, sizeof p->desc, "2d-transpose H=%lld W=%lld: %s, %s", (long long)h, (long long)w, a, b);
    return FFT_OK;
}

// 1-D lengths above what one plan covers (2^24 points): the six-step form of
// N = N1 * N2 (Sec. III-A's split into DFTs of the factors) with N1 <= N2
// the divisor nearest sqrt(N) whose two lengths both have 1-D plans:
// transpose [N1][N2] -> [N2][N1], N1-point plan over batch * N2 rows, multiply
// by W_N^(n2*k1) while transposing back to [N1][N2], N2-point plan over
// batch * N1 rows, transpose to [N2][N1], which is X[k1 + N1 * k2] in natural
// order.  Every pass is a batched plan of its own (power of two, mixed radix,
// Bluestein); the twiddle comes from two FP64-generated tables of W_N.
fft_status build_sixstep(fft_plan_s* p, int64_t n) {
    if (env_int("B300FFT_SIXSTEP", 1) == 0 || n <= (int64_t(1) << 24) || n >= (int64_t(1) << 31))
        return FFT_ERR_UNSUPPORTED;
    if (p->gplan) {  // a stage-graph plan that did not take the length
        graph_plan_free(p->gplan);
        delete p->gplan;
        p->gplan = nullptr;
    }
    if (p->d_tables || p->d_work || p->d_aux) return FFT_ERR_UNSUPPORTED;
    // Column form where 2^8 divides N: the 256-point transforms run straight
    // on the strided columns of [256][N2] (16 columns per tile, 128-byte row
    // segments) with the W_N twiddle on their store, so the first transpose
    // and the twiddle pass fold into one HBM round trip; then the N2-point
    // plan over the 256 * batch rows and one transpose.  Measured on a B300
    // (forward): 2^25 x 2 1007 -> 754 us, 2^30 20.3 -> 13.9 ms, 3 * 2^25
    // 1.86 -> 1.38 ms against the transposing form below.
    if (env_int("B300FFT_SIXSTEP_COLS", 1) != 0 && n % 256 == 0 && (n / 256) % 16 == 0 &&
        n / 256 <= (int64_t(1) << 24)) {
        const int64_t n1 = 256, n2 = n / 256;
        fft_plan b = fft_plan_create(1, &n2, p->batch * n1, FFT_FP32);
        if (b) {
            p->inner2 = b;
            p->six_n1 = n1;
            p->six_n2 = n2;
            p->six_cols = true;
            int lg = 0;
            while ((int64_t(1) << lg) < n) ++lg;
            p->sh = (lg + 1) / 2;
            const int64_t elo = int64_t(1) << p->sh, ehi = (n + elo - 1) / elo;
            const size_t ea = (size_t)pow2_table_entries(8);
            p->off_a = 0;
            p->off_lo = ea;
            p->off_hi = ea + (size_t)elo;
            fft_status s = alloc_tables(p, p->off_hi + (size_t)ehi);
            if (s != FFT_OK) return s;
            if (gen_pow2_table(p->d_tables + p->off_a, 8, 0) != cudaSuccess) return FFT_ERR_CUDA;
            if (gen_root_table(p->d_tables + p->off_lo, elo, 1, n, 0) != cudaSuccess) return FFT_ERR_CUDA;
            if (gen_root_table(p->d_tables + p->off_hi, ehi, elo, n, 0) != cudaSuccess) return FFT_ERR_CUDA;
            if (cols_prepare(8, 16) != cudaSuccess) return FFT_ERR_CUDA;
            p->work_bytes = (size_t)n * (size_t)p->batch * sizeof(float2);
            if (cudaMalloc(&p->d_work, p->work_bytes) != cudaSuccess) return FFT_ERR_ALLOC;
            p->kind = PlanKind::SixStep;
            p->kernels = 1 + fft_plan_kernel_count(b) + 1;
            char db[160];
            fft_plan_describe(b, db, sizeof db);
            std::snprintf(p->desc, sizeof p->desc, "sixstep N=%lld = 256 (columns, C=16, twiddle) x %lld: [%s], transpose",
                          (long long)n, (long long)n2, db);
            return FFT_OK;
        }
    }
    int64_t root = 1;
    while ((root + 1) * (root + 1) <= n) ++root;
    int tries = 0;
    for (int64_t d = root; d >= 2 && tries < 8; --d) {
        if (n % d != 0 || n / d > (int64_t(1) << 24)) continue;
        ++tries;
        const int64_t n1 = d, n2 = n / d;
        fft_plan a = fft_plan_create(1, &n1, p->batch * n2, FFT_FP32);
        if (!a) continue;
        fft_plan b = fft_plan_create(1, &n2, p->batch * n1, FFT_FP32);
        if (!b) {
            fft_plan_destroy(a);
            continue;
        }
        p->inner = a;
        p->inner2 = b;
        p->six_n1 = n1;
        p->six_n2 = n2;
        int lg = 0;
        while ((int64_t(1) << lg) < n) ++lg;
        p->sh = (lg + 1) / 2;
        const int64_t elo = int64_t(1) << p->sh, ehi = (n + elo - 1) / elo;
        p->off_lo = 0;
        p->off_hi = (size_t)elo;
        fft_status s = alloc_tables(p, (size_t)(elo + ehi));
        if (s != FFT_OK) return s;
        if (gen_root_table(p->d_tables + p->off_lo, elo, 1, n, 0) != cudaSuccess) return FFT_ERR_CUDA;
        if (gen_root_table(p->d_tables + p->off_hi, ehi, elo, n, 0) != cudaSuccess) return FFT_ERR_CUDA;
        p->work_bytes = (size_t)n * (size_t)p->batch * sizeof(float2);
        if (cudaMalloc(&p->d_work, p->work_bytes) != cudaSuccess) return FFT_ERR_ALLOC;
        p->kind = PlanKind::SixStep;
        p->kernels = fft_plan_kernel_count(a) + fft_plan_kernel_count(b) + 3;
        char da[100], db[100];
        fft_plan_describe(a, da, sizeof da);
        fft_plan_describe(b, db, sizeof db);
        std::snprintf(p->desc, sizeof p->desc, "sixstep N=%lld = %lld x %lld: [%s], twiddle-transpose, [%s]",
                      (long long)n, (long long)n1, (long long)n2, da, db);
        return FFT_OK;
    }
    return FFT_ERR_UNSUPPORTED;
}

// Non-power-of-two 1-D lengths: mixed radix 2/3/4/5/7/8/16 (single tile or
// four-step) or Bluestein, through the stage-graph executor.
fft_status build_generic_1d(fft_plan_s* p) {
    p->gplan = new (std::nothrow) GraphPlan();
    if (!p->gplan) return FFT_ERR_ALLOC;
    fft_status s = graph_plan_build(p->gplan, std::vector<int64_t>{p->len[0]}, p->batch, false);
    if (s != FFT_OK) return s;
    p->kind = PlanKind::Generic;
    p->kernels = 1;
    p->work_bytes = p->gplan->work_bytes;
    std::snprintf(p->desc, sizeof p->desc, "generic N=%lld: %s", (long long)p->len[0], p->gplan->desc.c_str());
    return FFT_OK;
}

fft_status build_ragged(fft_plan_s* p, const int64_t* lengths, int64_t count) {
    p->gplan = new (std::nothrow) GraphPlan();
    if (!p->gplan) return FFT_ERR_ALLOC;
    fft_status s = graph_plan_build(p->gplan, std::vector<int64_t>(lengths, lengths + count), count, true);
    if (s != FFT_OK) return s;
    p->kind = PlanKind::Ragged;
    p->kernels = 1;
    p->work_bytes = p->gplan->work_bytes;
    std::snprintf(p->desc, sizeof p->desc, "ragged count=%lld: %s", (long long)count, p->gplan->desc.c_str());
    return FFT_OK;
}

}  // namespace b300fft

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
        int mm = 0, kk = 0;
        if (l >= 0) s = build_pow2_1d(p, l);
        else if (mixed_supported(lengths[0], &mm, &kk) && env_int("B300FFT_MIXED", 1) != 0)
            s = build_mixed_1d(p, mm, kk);
        else if (mixed_fourstep_length(lengths[0], &mm, &kk) && env_int("B300FFT_MIXED", 1) != 0) {
            s = build_mixed_fourstep(p, mm, kk);  // unsupported splits return before allocating
            if (s == FFT_ERR_UNSUPPORTED) s = build_generic_1d(p);
        } else {
            s = build_generic_1d(p);
        }
        if (s == FFT_ERR_UNSUPPORTED) s = build_sixstep(p, lengths[0]);
    } else {
        const int lh = ilog2_exact(lengths[0]), lw = ilog2_exact(lengths[1]);
        if (env_int("B300FFT_2D_TRANSPOSE", 1) == 2) s = build_2d_transpose(p, lengths[0], lengths[1]);  // forced
        else if (lh >= 0 && lw >= 0) s = build_pow2_2d(p, lh, lw);
        else if (env_int("B300FFT_MIXED", 1) != 0) s = build_mixed_2d(p, lengths[0], lengths[1]);
        else s = FFT_ERR_UNSUPPORTED;
        if (s == FFT_ERR_UNSUPPORTED) s = build_2d_transpose(p, lengths[0], lengths[1]);
    }
    if (s != FFT_OK) return fail(s, p);
    return finish(p);
}

fft_plan fft_plan_create_real(int64_t n, int64_t batch) {
    g_last_error = FFT_OK;
    if (n < 2 || batch < 1 || n > (int64_t(1) << 31) || batch > (int64_t(1) << 40) / n)
        return fail(FFT_ERR_INVALID_ARG, nullptr);
    if (n & 1) return fail(FFT_ERR_UNSUPPORTED, nullptr);
    fft_plan_s* p = new (std::nothrow) fft_plan_s();
    if (!p) return fail(FFT_ERR_ALLOC, nullptr);
    p->dims = 1;
    p->len[0] = n;
    p->batch = batch;
    p->elements = n * batch;
    if (cudaMalloc(&p->d_status, sizeof(int)) != cudaSuccess) return fail(FFT_ERR_ALLOC, p);
    if (cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess) return fail(FFT_ERR_CUDA, p);
    fft_status s = build_real_plan(p, n, batch);
    if (s != FFT_OK) return fail(s, p);
    return finish(p);
}

fft_plan fft_plan_create_ragged(const int64_t* lengths, int64_t count, int precision) {
    g_last_error = FFT_OK;
    if (!lengths || count < 1 || count > (int64_t(1) << 24)) return fail(FFT_ERR_INVALID_ARG, nullptr);
    if (precision < FFT_FP32 || precision > FFT_TC_BF16_PLAIN) return fail(FFT_ERR_INVALID_ARG, nullptr);
    int64_t total = 0;
    for (int64_t i = 0; i < count; ++i) {
        if (lengths[i] < 1 || lengths[i] > (int64_t(1) << 20)) return fail(FFT_ERR_INVALID_ARG, nullptr);
        total += lengths[i];
    }
    if (precision != FFT_FP32) return fail(FFT_ERR_UNSUPPORTED, nullptr);
    fft_plan_s* p = new (std::nothrow) fft_plan_s();
    if (!p) return fail(FFT_ERR_ALLOC, nullptr);
    p->dims = 1;
    p->batch = count;
    p->precision = precision;
    p->elements = total;
    if (cudaMalloc(&p->d_status, sizeof(int)) != cudaSuccess) return fail(FFT_ERR_ALLOC, p);
    if (cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess) return fail(FFT_ERR_CUDA, p);
    fft_status s = build_ragged(p, lengths, count);
    if (s != FFT_OK) return fail(s, p);
    return finish(p);
}

fft_status fft_last_error(void) { return g_last_error; }

fft_status fft_exec_per_size(fft_plan plan, const void* in, void* out, int direction, void* stream) {
    if (!is_registered(plan)) return FFT_ERR_BAD_HANDLE;
    if (!in || !out) return FFT_ERR_INVALID_ARG;
    if (direction != FFT_FORWARD && direction != FFT_INVERSE) return FFT_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
        return FFT_ERR_MISALIGNED;
    return exec_plan(plan, static_cast<const float2*>(in), static_cast<float2*>(out), direction == FFT_INVERSE,
                     static_cast<cudaStream_t>(stream), -1, true);
}

fft_status fft_exec(fft_plan plan, const void* in, void* out, int direction, void* stream) {
    if (!is_registered(plan)) return FFT_ERR_BAD_HANDLE;
    if (!in || !out) return FFT_ERR_INVALID_ARG;
    if (direction != FFT_FORWARD && direction != FFT_INVERSE) return FFT_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
        return FFT_ERR_MISALIGNED;
    return exec_plan(plan, static_cast<const float2*>(in), static_cast<float2*>(out), direction == FFT_INVERSE,
                     static_cast<cudaStream_t>(stream));
}

fft_status fft_convolve(fft_plan plan, const void* x, const void* hspec, void* out, float scale, int conj_h,
                        void* stream) {
    if (!is_registered(plan)) return FFT_ERR_BAD_HANDLE;
    if (!x || !hspec || !out) return FFT_ERR_INVALID_ARG;
    if (plan->precision != FFT_FP32 || plan->kind == PlanKind::Ragged || plan->kind == PlanKind::Real)
        return FFT_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(hspec) & 15) ||
        (reinterpret_cast<uintptr_t>(out) & 15))
        return FFT_ERR_MISALIGNED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float2* in = static_cast<const float2*>(x);
    float2* o = static_cast<float2*>(out);
    const float2* hs = static_cast<const float2*>(hspec);
    if (plan->kind == PlanKind::Rows)  // one fused pass
        return launch_conv_rows(plan->logn_a, conj_h != 0, in, o, plan->batch, plan->d_tables + plan->off_a, hs,
                                scale, st) == cudaSuccess
                   ? FFT_OK
                   : FFT_ERR_CUDA;
    const int64_t n = plan->len[0] * (plan->dims == 2 ? plan->len[1] : 1);  // points per transform
    fft_status s = exec_plan(plan, in, o, false, st);
    if (s == FFT_OK) s = fft_spectrum_product(o, hs, o, n, plan->batch, scale, conj_h, stream);
    if (s == FFT_OK) s = exec_plan(plan, o, o, true, st);
    return s;
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
    }
    // the plans a Real or TwoDTranspose plan runs (their words are read and cleared too)
    fft_status r = (fft_status)h;
    for (fft_plan q : {plan->inner, plan->inner2}) {
        if (!q) continue;
        const fft_status s = fft_plan_check(q);
        if (r == FFT_OK) r = s;
    }
    return r;
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
    size_t b = plan->work_bytes;
    for (fft_plan q : {plan->inner, plan->inner2})
        if (q) b += fft_plan_workspace_bytes(q);
    return b;
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

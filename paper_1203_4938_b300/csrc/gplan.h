// gplan.h -- host-side stage-graph plans (generic lengths, Bluestein, ragged).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/fft.h"

namespace b300fft {

struct GShape;
struct GStage;
struct GTransform;

// Tunables of one length (chosen by the planner, or by the autotuner).
struct GLenConfig {
    int tile_max = 4096;  // largest length done in one tile
    int split_n2 = 0;     // four-step second-pass length (0: planner's choice)
    int lpt_a = 0;        // lines per tile, first / only stage (0: planner's choice)
    int lpt_b = 0;        // lines per tile, second four-step stage
};

struct GraphPlan {
    // device arrays
    float2* pool = nullptr;
    GShape* shapes = nullptr;
    GStage* stages[2] = {nullptr, nullptr};  // forward, inverse
    GTransform* xf = nullptr;
    uint64_t* items = nullptr;      // queue in stage rounds (per-stage launch groups)
    uint64_t* items_lag = nullptr;  // queue of the persistent launch (stages lagged per transform)
    int* ctl = nullptr;
    float2* work = nullptr;
    size_t work_bytes = 0;
    // sizes
    int nitems = 0, ncounters = 0, ntransforms = 0;
    int grid = 0;
    // per-stage launch groups: [item0, item1) share stage index and kind
    std::vector<std::pair<int, int>> groups;
    // graphs of the persistent launch, one per direction
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    cudaGraphNode_t knode[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [direction][launch]
    bool use_graph = true;
    // Executor instantiations (generic.cuh): transforms whose stages are all
    // compile-time tiles run in a lean executor without the runtime tiles
    // (4 CTAs per SM), the others in the full one; either kind includes the
    // mixed-radix tiles only when its transforms need them.  A plan with both
    // kinds runs two persistent launches: the first nrest queue items in the
    // full executor (kfull, grid CTAs), then the rest in the lean one (klean,
    // grid_lean CTAs).
    bool mix = false;   // some stage uses the compile-time mixed-radix tiles
    bool lean = false;  // every transform runs in the lean executor
    int kfull = 0, klean = 0;
    int nrest = 0, grid_lean = 0;
    int64_t spin_limit = int64_t(1) << 23;
    int withhold_xf = -1;  // test-only fault injection (B300FFT_DEBUG_WITHHOLD_XF)
    std::string desc;
    int64_t* line_off = nullptr;              // grouped-line offsets (device)
    bool no_tune = false;                     // candidate plans built by the autotuner
    std::map<int64_t, GLenConfig> configs;    // tile configuration used per length
};

// Measured tile configuration of one length (the autotuner): candidates are
// timed as ragged plans of ~2^22 elements of that length; results are cached
// per process and, when FFT_TUNE_CACHE names a file, in that file.
GLenConfig tune_length(int64_t n, int64_t count, const GLenConfig& base);

// Build a plan for transforms of the given lengths, packed back to back
// (offsets = exclusive prefix sum), or for `batch` copies of one length when
// lengths.size() == 1 and batch > 1 (uniform batch).
fft_status graph_plan_build(GraphPlan* gp, const std::vector<int64_t>& lengths, int64_t batch, bool ragged);
void graph_plan_free(GraphPlan* gp);
// Enqueue: persistent launch (graph when possible) or per-stage launches.
fft_status graph_plan_exec(GraphPlan* gp, const float2* in, float2* out, bool inv, cudaStream_t st, int* d_status,
                           bool per_stage);
// Lengths the stage graph can transform (any N >= 1 up to 2^24 smooth, primes via Bluestein).
bool graph_length_supported(int64_t n);

}  // namespace b300fft

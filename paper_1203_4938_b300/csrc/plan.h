// plan.h -- the plan object behind the opaque fft_plan handle.  Internal.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fft.h"

namespace b300fft {

constexpr uint64_t kPlanMagic = 0xB300FF7A5EEDULL;

enum class PlanKind : int {
    None = 0,
    Rows,      // single-pass power-of-two rows kernel
    FourStep,  // columns + transposed rows, through the workspace
    FourStepPersist,  // both four-step passes in one persistent launch, L2-resident chunks
    ThreeStep,        // three short-transform stages in one persistent launch (N = N1 * M1 * M2)
    Cluster,          // one transform per thread-block cluster, DSMEM exchanges, one HBM round trip
    TwoD,      // rows pass then in-place columns pass
    TwoDPersist,  // both 2-D passes in one persistent launch, L2-resident chunks of images
    RowsMixed, // single-pass mixed-radix rows kernel, L = M * 2^K <= 4096 (M = 3, 5, 7)
    FourStepMixed, // N = (M * 2^a) * 2^b: mixed columns kernel + power-of-two transposed rows
    TwoDMixed, // 2-D with a side of M * 2^K: rows kernel (power of two or mixed), then in-place column pass
    TwoDTranspose,  // any other 2-D: 1-D plan over the rows, transpose, 1-D plan over the columns, transpose
    SixStep,   // 1-D N = N1 * N2 beyond one plan: transpose, N1-point plan, twiddle + transpose, N2-point plan, transpose
    Generic,   // runtime mixed-radix (2,3,4,5,7,8,16) single CTA / multi-pass
    Bluestein, // chirp-z through a power-of-two convolution
    Ragged,    // persistent work-queue kernel over uneven lengths
    TensorCore, // radix-16 stages as tensor-core GEMMs
    Real        // real-to-complex / complex-to-real around a complex plan of N/2
};

struct GraphPlan;  // gplan.h
struct TcPlan;     // tc.cu

}  // namespace b300fft

struct fft_plan_s {
    uint64_t magic = 0;
    int dims = 1;
    int64_t len[2] = {1, 1};
    int64_t batch = 1;
    int64_t elements = 0;  // complex elements per exec (in and out)
    int precision = 0;
    b300fft::PlanKind kind = b300fft::PlanKind::None;
    int single_max_log = 14;  // largest power-of-two length done in one pass

    // power-of-two kernels
    int logn_a = 0, logn_b = 0, sh = 0;
    int mix_m = 0;  // RowsMixed: L = mix_m * 2^logn_a
    int mix_mh = 0, mix_mw = 0;  // TwoDMixed: odd factor of H / W (0: power of two, logn_b / logn_a = log2)
    bool real_fused = false;     // Real: one-pass fused rows + split kernel (h = 2^5 .. 2^12)
    int rows_staged = 0;  // Rows: persistent form with bulk-copied input staging (grid pgrid)
    int cols_c = 0;     // columns kernel width
    int rowsT_tpc = 0;  // transposed-rows kernel rows per CTA (TwoDTranspose: of the rows pass, 0: plan + transpose)
    int colsT_tpc = 0;  // TwoDTranspose: transposed-rows kernel rows per CTA of the columns pass (0: plan + transpose)

    // persistent four-step
    int pl1 = 0, pc = 0, pl2 = 0, ptpc = 0;
    int ppipe = 0;  // > 0: the persistent four-step runs with asynchronous loads into a ring of ppipe slots
    int pprefetch = 0;  // three-stage: L2 tensor prefetch of the next tile's box
    int pgrid = 0, pnch = 0, pna = 0, pnb = 0;
    int64_t pcb = 0;
    int64_t spin_limit = int64_t(1) << 23;
    int withhold_chunk = -1;
    int cl_lm = 0, cl_k = 0;  // cluster: N = cl_k * 2^cl_lm
    int pG = 0, pnb1g = 0, pnb2g = 0, pD = 1;  // three-stage: groups per chunk, B1 / B2 tiles per group, lookahead
    size_t off_a = 0, off_b = 0, off_c = 0, off_lo = 0, off_hi = 0;  // into d_tables (float2 units)

    float2* d_tables = nullptr;
    float2* d_work = nullptr;
    size_t work_bytes = 0;
    int* d_status = nullptr;
    void* d_aux = nullptr;  // kind-specific device block (descriptors, queues)

    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;

    b300fft::GraphPlan* gplan = nullptr;  // Generic / Ragged kinds
    fft_plan inner = nullptr;             // Real: the complex plan of N/2; TwoDTranspose: the rows plan
    fft_plan inner2 = nullptr;            // TwoDTranspose: the plan over the transposed columns; SixStep: N2
    int64_t six_n1 = 0, six_n2 = 0;       // SixStep: N = six_n1 * six_n2 (inner: N1 points, inner2: N2 points)
    bool six_cols = false;                // SixStep: N1 = 2^8 by the columns kernel (no inner, no first transpose)
    b300fft::TcPlan* tc = nullptr;
    int tc_grid[2] = {0, 0};  // TensorCore: persistent CTAs of its (first, second) kernel
    int tc_per_sm = 0;        // TensorCore: persistent CTAs per SM of its last kernel

    int kernels = 0;
    char desc[256] = {0};
};

namespace b300fft {

// An explicit choice for the batched power-of-two planner: what the
// autotuner times as a candidate and returns as its pick.
struct Pow2Choice {
    int family = 0;     // 1 single-pass rows, 2 persistent four-step, 3 persistent three-stage
    int a = 0, b = 0, c = 0, d = 0;  // four-step: l1, columns, l2, rows per tile; three-stage: la, lb1, lb2, tile
    int chunk_mb = 0;   // transforms per dependency chunk, in MiB (0: table)
    int pipe = 0;       // ring slots of the asynchronous-load form (0: plain loads); rows: 1 = staged input
    int lookahead = 0;  // three-stage B1 lookahead in row groups (0: planner's rule)
};
// The calling thread's forced choice (null: tables and environment decide).
const Pow2Choice* pow2_forced();
void pow2_force(const Pow2Choice* c);
// Time the candidates for transforms of 2^logn x batch on the current device
// and return the fastest in *best (false when there is nothing to choose).
// Results are cached per process and, when FFT_TUNE_CACHE names a file, in
// that file (lines "pow2:<device>:<logn>:<batch> family a b c d chunk pipe
// lookahead us").
bool tune_pow2(int logn, int64_t batch, Pow2Choice* best);

void destroy_plan_resources(fft_plan_s* p);
// only < 0: every kernel; else only kernel `only` of the sequence
fft_status exec_plan(fft_plan_s* p, const float2* in, float2* out, bool inv, cudaStream_t st, int only = -1,
                     bool per_size = false);

// Builders of the other kernel families (return FFT_ERR_UNSUPPORTED when the
// shape is outside what they implement).
fft_status build_generic_1d(fft_plan_s* p);
fft_status build_ragged(fft_plan_s* p, const int64_t* lengths, int64_t count);
fft_status build_tc_plan(fft_plan_s* p);
fft_status exec_tc(fft_plan_s* p, const float2* in, float2* out, bool inv, cudaStream_t st, int only);
fft_status build_real_plan(fft_plan_s* p, int64_t n, int64_t batch);
fft_status exec_real(fft_plan_s* p, const void* in, void* out, bool inv, cudaStream_t st);

}  // namespace b300fft

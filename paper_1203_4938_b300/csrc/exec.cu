// exec.cu -- fft_exec dispatch: enqueue the kernels of a plan on a stream.
#include "gplan.h"
#include "launch.h"
#include "persist.cuh"
#include "persist2d.cuh"
#include "threestep.cuh"
#include "plan.h"

namespace b300fft {

fft_status exec_plan(fft_plan_s* p, const float2* in, float2* out, bool inv, cudaStream_t st, int only,
                     bool per_size) {
    cudaError_t e = cudaSuccess;
    auto want = [only](int k) { return only < 0 || only == k; };
    switch (p->kind) {
        case PlanKind::Rows:
            if (!want(0)) break;
            // (fft_exec admits only 16-byte aligned buffers, as the row copies need)
            if (p->rows_staged && (reinterpret_cast<uintptr_t>(in) & 15) == 0)
                // the waits are for this CTA's own copies: never shorter than ~1 s,
                // whatever spin limit the plan was given, so a CTA never leaves
                // with a copy into its shared memory still running
                e = launch_rows_staged(p->logn_a, inv, in, out, p->batch, p->d_tables + p->off_a, p->d_status,
                                       p->spin_limit > (1 << 20) ? p->spin_limit : (1 << 20), p->pgrid, st);
            else
                e = launch_rows(p->logn_a, inv, in, out, p->batch, p->d_tables + p->off_a, st);
            break;
        case PlanKind::FourStepMixed: {
            const int64_t n1 = int64_t(p->mix_m) << p->logn_a, n2 = int64_t(1) << p->logn_b;
            if (want(0))
                e = launch_cols_mixed(p->mix_m, p->logn_a, inv, in, p->d_work, n2, p->batch, p->d_tables + p->off_a,
                                      p->d_tables + p->off_lo, p->d_tables + p->off_hi, p->sh, st);
            if (e == cudaSuccess && want(1))
                e = launch_rowsT(p->logn_b, p->rowsT_tpc, inv, p->d_work, out, p->batch * n1, p->d_tables + p->off_b,
                                 n1, st);
            break;
        }
        case PlanKind::RowsMixed:
            if (want(0)) e = launch_rows_mixed(p->mix_m, p->logn_a, inv, in, out, p->batch, p->d_tables, st);
            break;
        case PlanKind::FourStep: {
            const int64_t n1 = int64_t(1) << p->logn_a, n2 = int64_t(1) << p->logn_b;
            if (want(0))
                e = launch_cols(p->logn_a, p->cols_c, inv, true, in, p->d_work, n2, n2, n1 * n2, p->batch,
                                p->d_tables + p->off_a, p->d_tables + p->off_lo, p->d_tables + p->off_hi, p->sh, st);
            if (e == cudaSuccess && want(1))
                e = launch_rowsT(p->logn_b, p->rowsT_tpc, inv, p->d_work, out, p->batch * n1, p->d_tables + p->off_b, n1,
                                 st);
            break;
        }
        case PlanKind::FourStepPersist: {
            if (!want(0)) break;
            PersistArgs a{};
            a.in = in;
            a.out = out;
            a.work = p->d_work;
            a.ctl = static_cast<int*>(p->d_aux);
            a.status = p->d_status;
            a.batch = p->batch;
            a.cb = p->pcb;
            a.nch = p->pnch;
            a.na = p->pna;
            a.nb = p->pnb;
            a.tw_a = p->d_tables + p->off_a;
            a.tw_b = p->d_tables + p->off_b;
            a.lo = p->d_tables + p->off_lo;
            a.hi = p->d_tables + p->off_hi;
            a.sh = p->sh;
            a.spin_limit = p->spin_limit;
            a.withhold_chunk = p->withhold_chunk;
            e = cudaMemsetAsync(p->d_aux, 0, sizeof(int) * (size_t)(1 + p->pnch), st);
            if (e == cudaSuccess)
                e = p->ppipe ? launch_fourstep_pipe(PersistConfig{p->pl1, p->pc, p->pl2, p->ptpc}, p->ppipe, inv, a,
                                                    p->pgrid, st)
                             : launch_fourstep_persist(PersistConfig{p->pl1, p->pc, p->pl2, p->ptpc}, inv, a, p->pgrid,
                                                       st);
            break;
        }
        case PlanKind::ThreeStep: {
            if (!want(0)) break;
            ThreeArgs a{};
            a.in = in;
            a.out = out;
            a.work = p->d_work;
            a.ctl = static_cast<int*>(p->d_aux);
            a.status = p->d_status;
            a.batch = p->batch;
            a.cb = p->pcb;
            a.nch = p->pnch;
            a.na = p->pna;
            a.nb = p->pnb;
            a.G = p->pG;
            a.nb1g = p->pnb1g;
            a.nb2g = p->pnb2g;
            a.D = p->pD;
            a.tw_a = p->d_tables + p->off_a;
            a.tw_b1 = p->d_tables + p->off_b;
            a.tw_b2 = p->d_tables + p->off_c;
            a.lo = p->d_tables + p->off_lo;
            a.hi = p->d_tables + p->off_hi;
            a.sh = p->sh;
            a.spin_limit = p->spin_limit;
            a.withhold_chunk = p->withhold_chunk;
            a.prefetch = p->pprefetch;
            e = cudaMemsetAsync(p->d_aux, 0, sizeof(int) * (size_t)(1 + p->pnch + (int64_t)p->pnch * p->pG), st);
            if (e == cudaSuccess)
                e = p->ppipe ? launch_threestep_pipe(ThreeConfig{p->pl1, p->pc, p->pl2, p->ptpc}, p->ppipe, inv, a,
                                                     p->pgrid, st)
                             : launch_threestep(ThreeConfig{p->pl1, p->pc, p->pl2, p->ptpc}, inv, a, p->pgrid, st);
            break;
        }
        case PlanKind::TwoDPersist: {
            if (!want(0)) break;
            PersistArgs a{};
            a.in = in;
            a.out = out;
            a.work = out;
            a.ctl = static_cast<int*>(p->d_aux);
            a.status = p->d_status;
            a.batch = p->batch;
            a.cb = p->pcb;
            a.nch = p->pnch;
            a.na = p->pna;
            a.nb = p->pnb;
            a.tw_a = p->d_tables + p->off_a;
            a.tw_b = p->d_tables + p->off_b;
            a.lo = nullptr;
            a.hi = nullptr;
            a.sh = 0;
            a.spin_limit = p->spin_limit;
            a.withhold_chunk = p->withhold_chunk;
            e = cudaMemsetAsync(p->d_aux, 0, sizeof(int) * (size_t)(1 + p->pnch), st);
            if (e == cudaSuccess)
                e = launch_2d_persist(PersistConfig{p->pl1, p->pc, p->pl2, p->ptpc}, inv, a, p->pgrid, st);
            break;
        }
        case PlanKind::Cluster:
            if (want(0))
                e = launch_cluster_fft(p->cl_lm, p->cl_k, inv, in, out, p->batch, p->d_tables + p->off_a,
                                       p->d_tables + p->off_lo, p->d_tables + p->off_hi, p->sh, st);
            break;
        case PlanKind::TwoD: {
            const int64_t h = p->len[0], w = p->len[1];
            if (want(0)) e = launch_rows(p->logn_a, inv, in, out, p->batch * h, p->d_tables + p->off_a, st);
            if (e == cudaSuccess && want(1))
                e = launch_cols(p->logn_b, p->cols_c, inv, false, out, out, w, w, h * w, p->batch, p->d_tables + p->off_b,
                                nullptr, nullptr, 0, st);
            break;
        }
        case PlanKind::TwoDMixed: {
            const int64_t h = p->len[0], w = p->len[1];
            const float2* tb = p->d_tables + p->off_b;
            if (want(0))
                e = p->mix_mw ? launch_rows_mixed(p->mix_mw, p->logn_a, inv, in, out, p->batch * h, p->d_tables, st)
                              : launch_rows(p->logn_a, inv, in, out, p->batch * h, p->d_tables, st);
            if (e == cudaSuccess && want(1))
                e = p->mix_mh ? launch_cols2d_mixed(p->mix_mh, p->logn_b, inv, out, out, w, p->batch, tb, st)
                              : launch_cols(p->logn_b, p->cols_c, inv, false, out, out, w, w, h * w, p->batch, tb,
                                            nullptr, nullptr, 0, st);
            break;
        }
        case PlanKind::Real:
            if (!want(0)) return FFT_OK;
            return exec_real(p, in, out, inv, st);
        case PlanKind::SixStep: {
            const int64_t n1 = p->six_n1, n2 = p->six_n2, n = n1 * n2;
            if (p->six_cols) {
                // kernel sequence: columns (in -> workspace, with the twiddle), the N2 plan's
                // (in place), transpose (workspace -> out); in == out is fine
                const int kb = p->inner2->kernels;
                fft_status s = FFT_OK;
                if (want(0))
                    e = launch_cols(8, 16, inv, true, in, p->d_work, n2, n2, n, p->batch, p->d_tables + p->off_a,
                                    p->d_tables + p->off_lo, p->d_tables + p->off_hi, p->sh, st);
                if (e == cudaSuccess && (only < 0 || (only >= 1 && only <= kb)))
                    s = exec_plan(p->inner2, p->d_work, p->d_work, inv, st, only < 0 ? -1 : only - 1, per_size);
                if (s == FFT_OK && e == cudaSuccess && want(kb + 1))
                    e = launch_transpose(p->d_work, out, n1, n2, p->batch, st);
                if (s != FFT_OK) return s;
                break;
            }
            // kernel sequence: transpose, the N1 plan's, twiddle-transpose, the N2 plan's, transpose
            const int ka = p->inner->kernels, kb = p->inner2->kernels;
            const bool inplace = in == out;
            float2* t = inplace ? p->d_work : out;  // [N2][N1] between the first two steps
            float2* z = inplace ? out : p->d_work;  // [N1][N2] between the last two
            fft_status s = FFT_OK;
            if (want(0)) e = launch_transpose(in, t, n1, n2, p->batch, st);
            if (e == cudaSuccess && (only < 0 || (only >= 1 && only <= ka)))
                s = exec_plan(p->inner, t, t, inv, st, only < 0 ? -1 : only - 1, per_size);
            if (s == FFT_OK && e == cudaSuccess && want(ka + 1))
                e = launch_twiddle_transpose(t, z, n2, n1, p->batch, n, p->d_tables + p->off_lo,
                                             p->d_tables + p->off_hi, p->sh, inv, st);
            if (s == FFT_OK && e == cudaSuccess && (only < 0 || (only >= ka + 2 && only <= ka + 1 + kb)))
                s = exec_plan(p->inner2, z, z, inv, st, only < 0 ? -1 : only - ka - 2, per_size);
            if (s == FFT_OK && e == cudaSuccess && want(ka + kb + 2)) {
                if (inplace) {
                    e = launch_transpose(z, p->d_work, n1, n2, p->batch, st);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(out, p->d_work, (size_t)n * (size_t)p->batch * sizeof(float2),
                                            cudaMemcpyDeviceToDevice, st);
                } else {
                    e = launch_transpose(z, out, n1, n2, p->batch, st);
                }
            }
            if (s != FFT_OK) return s;
            break;
        }
        case PlanKind::TwoDTranspose: {
            // kernel sequence: rows pass (transposed-store kernel, or the rows plan's kernels then a
            // transpose) into the workspace [W][H]; columns pass (transposed-store kernel, or the
            // columns plan's kernels in place then a transpose) into `out`.  in == out is fine.
            const int64_t h = p->len[0], w = p->len[1];
            const int k1 = p->rowsT_tpc ? 1 : p->inner->kernels + 1;
            const int k2 = p->colsT_tpc ? 1 : p->inner2->kernels + 1;
            fft_status s = FFT_OK;
            if (p->rowsT_tpc) {
                if (want(0))
                    e = launch_rowsT(p->logn_a, p->rowsT_tpc, inv, in, p->d_work, p->batch * h,
                                     p->d_tables + p->off_a, h, st);
            } else {
                if (only < 0 || only < k1 - 1) s = exec_plan(p->inner, in, out, inv, st, only, per_size);
                if (s == FFT_OK && want(k1 - 1)) e = launch_transpose(out, p->d_work, h, w, p->batch, st);
            }
            if (s == FFT_OK && e == cudaSuccess) {
                if (p->colsT_tpc) {
                    if (want(k1))
                        e = launch_rowsT(p->logn_b, p->colsT_tpc, inv, p->d_work, out, p->batch * w,
                                         p->d_tables + p->off_b, w, st);
                } else {
                    if (only < 0 || (only >= k1 && only < k1 + k2 - 1))
                        s = exec_plan(p->inner2, p->d_work, p->d_work, inv, st, only < 0 ? -1 : only - k1, per_size);
                    if (s == FFT_OK && want(k1 + k2 - 1)) e = launch_transpose(p->d_work, out, w, h, p->batch, st);
                }
            }
            if (s != FFT_OK) return s;
            break;
        }
        case PlanKind::TensorCore:
            return exec_tc(p, in, out, inv, st, only);
        case PlanKind::Generic:
        case PlanKind::Ragged:
            if (!want(0)) return FFT_OK;
            return graph_plan_exec(p->gplan, in, out, inv, st, p->d_status, per_size);
        default:
            return FFT_ERR_UNSUPPORTED;
    }
    return e == cudaSuccess ? FFT_OK : FFT_ERR_CUDA;
}


}  // namespace b300fft

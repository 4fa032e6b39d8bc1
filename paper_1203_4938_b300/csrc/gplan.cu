// gplan.cu -- host side of the stage-graph engine (generic.cuh): radix
// plans, stage chains, the table pool, the work queue and its execution as
// one persistent launch (captured in a CUDA graph) or as per-stage launches.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "generic.cuh"
#include "gplan.h"
#include "launch.h"

namespace b300fft {

namespace {

int env_i(const char* name, int dflt) {
    const char* v = std::getenv(name);
    return (v && *v) ? std::atoi(v) : dflt;
}

// The executor instantiations: full or lean (no runtime tiles, 4 CTAs per
// SM), each with or without the compile-time mixed tiles.
enum GKind : int { GK_BASE = 0, GK_MIX = 1, GK_LEAN = 2, GK_LEANMIX = 3 };
const void* gexec_fn(int k) {
    switch (k) {
        case GK_MIX: return (const void*)k_gexec<true, false>;
        case GK_LEAN: return (const void*)k_gexec<false, true>;
        case GK_LEANMIX: return (const void*)k_gexec<true, true>;
        default: return (const void*)k_gexec<false, false>;
    }
}
int gexec_smem(int k) { return k == GK_LEAN ? kGSmemLean : (k == GK_LEANMIX ? kGSmemLeanMix : kGSmem); }
void launch_gexec(int k, int grid, const GExecArgs& a, cudaStream_t st) {
    const int sm = gexec_smem(k);
    switch (k) {
        case GK_MIX: k_gexec<true, false><<<grid, kGThreads, sm, st>>>(a); break;
        case GK_LEAN: k_gexec<false, true><<<grid, kGThreads, sm, st>>>(a); break;
        case GK_LEANMIX: k_gexec<true, true><<<grid, kGThreads, sm, st>>>(a); break;
        default: k_gexec<false, false><<<grid, kGThreads, sm, st>>>(a); break;
    }
}

// The persistent launches of a plan (see GraphPlan::nrest).
struct GPart {
    int kind, item0, nitems, grid, head;
};
int gexec_parts(const GraphPlan* gp, GPart* parts) {
    if (gp->nrest > 0 && gp->nrest < gp->nitems) {
        parts[0] = {gp->kfull, 0, gp->nrest, gp->grid, 0};
        parts[1] = {gp->klean, gp->nrest, gp->nitems - gp->nrest, gp->grid_lean, 1 + gp->ncounters};
        return 2;
    }
    parts[0] = {gp->lean ? gp->klean : gp->kfull, 0, gp->nitems, gp->grid, 0};
    return 1;
}

bool is_smooth(int64_t n) {
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) n /= p;
    return n == 1;
}

int64_t next_pow2(int64_t v) {
    int64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Radix sequence of a smooth length <= kGTileMax: 16s first, then the rest
// of the power of two, then 3, 5, 7 factors.
bool radix_plan(int L, std::vector<int>* r) {
    r->clear();
    if (L == 1) {
        r->push_back(1);
        return true;
    }
    int m = L, p2 = 0;
    while (m % 2 == 0) {
        m /= 2;
        ++p2;
    }
    while (p2 >= 4) {
        r->push_back(16);
        p2 -= 4;
    }
    if (p2) r->push_back(1 << p2);
    for (int p : {3, 5, 7})
        while (m % p == 0) {
            r->push_back(p);
            m /= p;
        }
    return m == 1 && (int)r->size() <= kGMaxPass;
}

struct Builder {
    std::vector<GShape> shapes;
    std::map<int, int> shape_of;  // L -> index
    std::vector<GStage> st_f, st_i;
    std::map<int64_t, std::pair<int64_t, int64_t>> fourstep_tabs;  // N -> (lo, hi)
    std::map<int64_t, std::array<int64_t, 3>> blue_tabs;           // N -> (chirp, Bf fwd, Bf inv)
    int64_t pool_size = 0;
    // deferred table generation
    struct PassTab {
        int64_t off;
        int ns, r;
    };
    struct RootTab {
        int64_t off, count, mult, n;
    };
    struct BlueTab {
        int64_t n, M, chirp, ff, fi;
    };
    std::vector<PassTab> pass_tabs;
    std::vector<RootTab> root_tabs;
    std::vector<BlueTab> blue_list;
    std::map<int, int64_t> pow2_tabs;  // log2 L -> offset of the templated tiles' Stockham table
    std::map<int, int64_t> mixed_tabs;  // 64 M + K -> offset of the compile-time mixed tiles' table

    int64_t mixed_table(int m, int k) {
        auto it = mixed_tabs.find(64 * m + k);
        if (it != mixed_tabs.end()) return it->second;
        const int64_t o = alloc(std::max(1, mixed_table_entries(m, k)));
        mixed_tabs[64 * m + k] = o;
        return o;
    }

    int64_t pow2_table(int logn) {
        auto it = pow2_tabs.find(logn);
        if (it != pow2_tabs.end()) return it->second;
        const int64_t o = alloc(pow2_table_entries(logn));
        pow2_tabs[logn] = o;
        return o;
    }

    int64_t alloc(int64_t n) {
        int64_t o = pool_size;
        pool_size += (n + 1) & ~int64_t(1);  // keep 16-byte alignment
        return o;
    }
    int shape(int L) {
        auto it = shape_of.find(L);
        if (it != shape_of.end()) return it->second;
        std::vector<int> r;
        if (!radix_plan(L, &r)) return -1;
        GShape s{};
        s.L = L;
        s.npass = (int)r.size();
        int ns = 1;
        for (int p = 0; p < s.npass; ++p) {
            s.radix[p] = r[p];
            s.ns[p] = ns;
            if (p > 0 && r[p] > 1) {
                s.tw[p] = alloc((int64_t)(r[p] - 1) * ns);
                pass_tabs.push_back({s.tw[p], ns, r[p]});
            }
            ns *= r[p];
        }
        shapes.push_back(s);
        shape_of[L] = (int)shapes.size() - 1;
        return (int)shapes.size() - 1;
    }
    std::pair<int64_t, int64_t> tw4(int64_t n, int* sh) {
        int lg = 0;
        while ((int64_t(1) << lg) < n) ++lg;
        *sh = (lg + 1) / 2;
        auto it = fourstep_tabs.find(n);
        if (it != fourstep_tabs.end()) return it->second;
        const int64_t nlo = int64_t(1) << *sh, nhi = (n + nlo - 1) / nlo;
        const int64_t lo = alloc(nlo), hi = alloc(nhi);
        root_tabs.push_back({lo, nlo, 1, n});
        root_tabs.push_back({hi, nhi, nlo, n});
        fourstep_tabs[n] = {lo, hi};
        return {lo, hi};
    }
    std::array<int64_t, 3> blue(int64_t n, int64_t M) {
        auto it = blue_tabs.find(n);
        if (it != blue_tabs.end()) return it->second;
        std::array<int64_t, 3> t{alloc(n), alloc(M), alloc(M)};
        blue_list.push_back({n, M, t[0], t[1], t[2]});
        blue_tabs[n] = t;
        return t;
    }
};

// Compile-time mixed tiles (B300FFT_G_MIXT=0 turns them off): lines of
// L = M * 2^K <= 4096, and four-step columns of M * 2^A with a column width.
bool mixed_rows_templated(int64_t n, int* m, int* k) {
    if (env_i("B300FFT_G_MIXT", 1) == 0) return false;
    if (n >= 16 && n <= 4096 && (n & (n - 1)) == 0) {  // power-of-two lines: M = 1
        *m = 1;
        *k = 0;
        while ((int64_t(1) << *k) < n) ++*k;
        return true;
    }
    return mixed_supported(n, m, k);
}
bool mixed_cols_templated(int64_t n1, int64_t n2, int* m, int* a, int* width) {
    if (env_i("B300FFT_G_MIXT", 1) == 0 || !mixed_supported(n1, m, a)) return false;
    *width = mixed_cols_width(*m, *a);
    return *width > 0 && n2 % *width == 0;
}

// Power-of-two lengths the stage graph runs with the templated tiles.
bool pow2_templated(int64_t n) {
    return n >= (int64_t(1) << 13) && n <= (int64_t(1) << 16) && (n & (n - 1)) == 0 && env_i("B300FFT_G_POW2T", 1) != 0;
}

GStage base_stage(int shape, int nlines, int lpt, int inv) {
    GStage s{};
    s.line_tab = -1;
    s.shape = shape;
    s.nlines = nlines;
    s.lpt = std::max(1, std::min(lpt, nlines));
    s.ntiles = (nlines + s.lpt - 1) / s.lpt;
    s.inv = inv;
    s.pre = G_PRE_NONE;
    s.post = G_POST_NONE;
    return s;
}

int lines_per_tile(int L, int want) {
    int cap = std::max(1, std::min(kGMaxLines, kGTileMax / L));
    return want > 0 ? std::min(want, cap) : cap;
}

// Second-pass length of N = M * 2^k > 4096 (M = 3, 5, 7) as the batched
// mixed four-step chooses it (build_mixed_fourstep): short mixed columns of
// M * 2^a (a = 2 below 2^12, else k - 8, at most 6) by the compile-time
// column tile, then rows of 2^b = 2^(k-a) <= 4096.  Measured against the
// balanced split in this executor: uniform batches of 6144 and 12288 points
// (1.7e7 elements) 8-11 % faster, 40960 unchanged (the same split).  0 when
// N is not such a length.
int64_t mixed_split_n2(int64_t n) {
    for (int m : {3, 5, 7}) {
        if (n % m) continue;
        const int64_t q = n / m;
        if (q & (q - 1)) continue;
        int k = 0;
        while ((int64_t(1) << k) < q) ++k;
        if (n <= 4096) return 0;
        int a = k >= 12 ? k - 8 : 2;
        if (a > 6) a = 6;
        if (k - a > 12) a = k - 12;
        const int b = k - a;
        return b >= 6 && b <= 12 ? int64_t(1) << b : 0;
    }
    return 0;
}

// Choose N = N1 * N2 (both <= tile max) for a smooth N; N2 a power of two
// when possible (radix-16 rows, long transposed-store runs).
bool split_four(int64_t n, int tile_max, int want_n2, int64_t* n1, int64_t* n2) {
    int64_t best = -1;
    double bestd = 1e30;
    auto consider = [&](int64_t b) {
        if (b < 2 || n % b) return;
        const int64_t a = n / b;
        if (a > tile_max || b > tile_max || a < 2) return;
        if (!is_smooth(a) || !is_smooth(b)) return;
        const double d = std::fabs(std::log((double)a) - std::log((double)b)) + ((b & (b - 1)) ? 1.0 : 0.0);
        if (d < bestd) {
            bestd = d;
            best = b;
        }
    };
    if (want_n2 > 0) consider(want_n2);
    if (best < 0)
        for (int64_t b = 2; b <= tile_max; ++b) consider(b);
    if (best < 0) return false;
    *n2 = best;
    *n1 = n / best;
    return true;
}

// Stages of one transform kind (length n); `lines` > 1 only for single-tile
// uniform batches (every batch row is a line of one stage).
bool build_kind(Builder& B, int64_t n, int64_t lines, const GLenConfig& cfg, int* nstages, int64_t* w1,
                int64_t* w2, int64_t line_tab) {
    *w1 = *w2 = 0;
    std::vector<GStage> f, i;
    if (is_smooth(n) && n <= cfg.tile_max) {
        const int sh = B.shape((int)n);
        if (sh < 0) return false;
        for (int d = 0; d < 2; ++d) {
            GStage s = base_stage(sh, (int)lines, lines_per_tile((int)n, cfg.lpt_a), d);
            s.in_buf = G_BUF_IN;
            s.out_buf = G_BUF_OUT;
            s.in_ls = s.out_ls = n;
            s.in_es = s.out_es = 1;
            s.in_valid = s.out_valid = lines * n;
            if (line_tab >= 0) {  // lines are separate transforms at line_off[line_tab + l]
                s.line_tab = line_tab;
                s.in_valid = s.out_valid = INT64_MAX;
            }
            int mm = 0, kk = 0;
            if (mixed_rows_templated(n, &mm, &kk)) {
                s.tmpl = 1000 + 16 * mm + kk;
                s.lpt = std::min(kGMixLines((int)n), std::max(1, (int)lines));
                s.ntiles = (int)((lines + kGMixLines((int)n) - 1) / kGMixLines((int)n));
                s.mtab = B.mixed_table(mm, kk);
            }
            (d ? i : f).push_back(s);
        }
    } else if (pow2_templated(n)) {
        // 2^13 .. 2^16: the batched path's register-staged tiles, (log2 N1, C, log2 N2, TPC) as below
        int lg = 0;
        while ((int64_t(1) << lg) < n) ++lg;
        static const int kT[17][4] = {{0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0}, {0},
                                      {6, 64, 7, 32}, {7, 32, 7, 32}, {7, 32, 8, 16}, {8, 16, 8, 16}};
        const int l1 = kT[lg][0], c = kT[lg][1], l2 = kT[lg][2], tpc = kT[lg][3];
        const int sa = B.shape(1 << l1);
        if (sa < 0) return false;
        int shs;
        auto tabs = B.tw4(n, &shs);
        const int64_t ta = B.pow2_table(l1), tb = B.pow2_table(l2);
        for (int d = 0; d < 2; ++d) {
            GStage a = base_stage(sa, 1, 1, d);
            a.ntiles = (1 << l2) / c;
            a.tmpl = 2 * lg;
            a.in_buf = G_BUF_IN;
            a.out_buf = G_BUF_W1;
            a.pre_tab = ta;
            a.lo = tabs.first;
            a.hi = tabs.second;
            a.sh = shs;
            GStage b = base_stage(sa, 1, 1, d);
            b.ntiles = (1 << l1) / tpc;
            b.tmpl = 2 * lg + 1;
            b.in_buf = G_BUF_W1;
            b.out_buf = G_BUF_OUT;
            b.post_tab = tb;
            (d ? i : f).push_back(a);
            (d ? i : f).push_back(b);
        }
        *w1 = n;
    } else if (is_smooth(n)) {
        int64_t n1, n2;
        const int64_t want = cfg.split_n2 ? cfg.split_n2 : (env_i("B300FFT_G_MIXSPLIT", 1) ? mixed_split_n2(n) : 0);
        if (!split_four(n, cfg.tile_max, (int)want, &n1, &n2)) return false;
        const int sa = B.shape((int)n1), sb = B.shape((int)n2);
        if (sa < 0 || sb < 0) return false;
        int shs;
        auto tabs = B.tw4(n, &shs);
        for (int d = 0; d < 2; ++d) {
            GStage a = base_stage(sa, (int)n2, lines_per_tile((int)n1, cfg.lpt_a), d);
            a.in_buf = G_BUF_IN;
            a.out_buf = G_BUF_W1;
            a.in_line_fast = a.out_line_fast = 1;
            a.in_ls = a.out_ls = 1;
            a.in_es = a.out_es = n2;
            a.in_valid = a.out_valid = n;
            a.post = G_POST_TW4;
            a.lo = tabs.first;
            a.hi = tabs.second;
            a.sh = shs;
            int mm = 0, aa = 0, width = 0;
            if (mixed_cols_templated(n1, n2, &mm, &aa, &width)) {
                a.tmpl = 2000 + 16 * mm + aa;
                a.lpt = width;
                a.ntiles = (int)(n2 / width);
                a.mtab = B.mixed_table(mm, aa);
            }
            GStage b = base_stage(sb, (int)n1, lines_per_tile((int)n2, cfg.lpt_b), d);
            b.in_buf = G_BUF_W1;
            b.out_buf = G_BUF_OUT;
            b.out_line_fast = 1;
            b.in_ls = n2;
            b.in_es = 1;
            b.out_ls = 1;
            b.out_es = n1;
            b.in_valid = b.out_valid = n;
            // rows of 128 or 256 points and a line count the rows-per-tile divide:
            // the templated transposed-row tile (32 or 16 rows, 256 threads)
            const int tpc2 = n2 == 128 ? 32 : (n2 == 256 ? 16 : 0);
            int l2 = 0;
            while ((int64_t(1) << l2) < n2) ++l2;
            if (tpc2 && n1 % tpc2 == 0 && env_i("B300FFT_G_POW2T", 1) != 0) {
                b.tmpl = 100 + (n2 == 128 ? 7 : 8);
                b.ntiles = (int)(n1 / tpc2);
                b.post_tab = B.pow2_table(n2 == 128 ? 7 : 8);
            } else if ((int64_t(1) << l2) == n2 && l2 >= 5 && l2 <= 12 && env_i("B300FFT_G_MIXT", 1) != 0) {
                // other power-of-two rows: the compile-time transposed-row tile
                // (any line count; the last tile may hold fewer lines)
                b.tmpl = 3000 + l2;
                b.ntiles = (int)((n1 + kGMixLines((int)n2) - 1) / kGMixLines((int)n2));
                b.mtab = B.mixed_table(1, l2);
            }
            (d ? i : f).push_back(a);
            (d ? i : f).push_back(b);
        }
        *w1 = n;
    } else {
        // Bluestein: M = 2^k >= 2n - 1
        const int64_t M = next_pow2(2 * n - 1);
        auto bt = B.blue(n, M);
        if (M <= cfg.tile_max) {
            const int sm = B.shape((int)M);
            for (int d = 0; d < 2; ++d) {
                GStage a = base_stage(sm, 1, 1, 0);
                a.in_buf = G_BUF_IN;
                a.out_buf = G_BUF_W1;
                a.in_ls = a.out_ls = M;
                a.in_es = a.out_es = 1;
                a.in_valid = n;
                a.out_valid = M;
                a.pre = d ? G_PRE_TABLE_CONJ : G_PRE_TABLE;
                a.pre_tab = bt[0];
                a.post = G_POST_TABLE;
                a.post_tab = d ? bt[2] : bt[1];
                GStage b = base_stage(sm, 1, 1, 1);
                b.in_buf = G_BUF_W1;
                b.out_buf = G_BUF_OUT;
                b.in_ls = b.out_ls = M;
                b.in_es = b.out_es = 1;
                b.in_valid = M;
                b.out_valid = n;
                b.post = d ? G_POST_TABLE_CONJ : G_POST_TABLE;
                b.post_tab = bt[0];
                int lm = 0;
                while ((int64_t(1) << lm) < M) ++lm;
                if (lm >= 7 && lm <= 12 && env_i("B300FFT_G_MIXT", 1) != 0) {  // compile-time tiles
                    a.tmpl = b.tmpl = 4000 + lm;
                    a.mtab = b.mtab = B.mixed_table(1, lm);
                }
                (d ? i : f).push_back(a);
                (d ? i : f).push_back(b);
            }
            *w1 = M;
        } else {
            int64_t m1, m2;
            if (!split_four(M, cfg.tile_max, 0, &m1, &m2)) return false;
            const int sa = B.shape((int)m1), sb = B.shape((int)m2);
            int shs;
            auto tabs = B.tw4(M, &shs);
            for (int d = 0; d < 2; ++d) {
                for (int k = 0; k < 2; ++k) {  // k = 0: FFT_M of x*w; k = 1: IFFT_M
                    GStage a = base_stage(sa, (int)m2, lines_per_tile((int)m1, cfg.lpt_a), k);
                    a.in_buf = k ? G_BUF_W2 : G_BUF_IN;
                    a.out_buf = G_BUF_W1;
                    a.in_line_fast = a.out_line_fast = 1;
                    a.in_ls = a.out_ls = 1;
                    a.in_es = a.out_es = m2;
                    a.in_valid = k ? M : n;
                    a.out_valid = M;
                    if (!k) {
                        a.pre = d ? G_PRE_TABLE_CONJ : G_PRE_TABLE;
                        a.pre_tab = bt[0];
                    }
                    a.post = G_POST_TW4;
                    a.lo = tabs.first;
                    a.hi = tabs.second;
                    a.sh = shs;
                    GStage b = base_stage(sb, (int)m1, lines_per_tile((int)m2, cfg.lpt_b), k);
                    b.in_buf = G_BUF_W1;
                    b.out_buf = k ? G_BUF_OUT : G_BUF_W2;
                    b.out_line_fast = 1;
                    b.in_ls = m2;
                    b.in_es = 1;
                    b.out_ls = 1;
                    b.out_es = m1;
                    b.in_valid = M;
                    b.out_valid = k ? n : M;
                    if (!k) {
                        b.post = G_POST_TABLE;
                        b.post_tab = d ? bt[2] : bt[1];
                    } else {
                        b.post = d ? G_POST_TABLE_CONJ : G_POST_TABLE;
                        b.post_tab = bt[0];
                    }
                    // compile-time tiles: columns of 2^la (pre multiply, W_M twiddle),
                    // then rows of 2^lb with the transposed store (post multiply)
                    int la = 0, lb = 0;
                    while ((int64_t(1) << la) < m1) ++la;
                    while ((int64_t(1) << lb) < m2) ++lb;
                    const int cw = la >= 6 && la <= 9 ? (4096 >> la < 64 ? 4096 >> la : 64) : 0;
                    if (cw && m2 % cw == 0 && lb >= 5 && lb <= 12 && env_i("B300FFT_G_MIXT", 1) != 0) {
                        a.tmpl = 5000 + la;
                        a.mtab = B.mixed_table(1, la);
                        a.lpt = cw;
                        a.ntiles = (int)(m2 / cw);
                        b.tmpl = 3000 + lb;
                        b.mtab = B.mixed_table(1, lb);
                        b.ntiles = (int)((m1 + kGMixLines((int)m2) - 1) / kGMixLines((int)m2));
                    }
                    (d ? i : f).push_back(a);
                    (d ? i : f).push_back(b);
                }
            }
            *w1 = M;
            *w2 = M;
        }
    }
    *nstages = (int)f.size();
    B.st_f.insert(B.st_f.end(), f.begin(), f.end());
    B.st_i.insert(B.st_i.end(), i.begin(), i.end());
    return true;
}

template <class T>
cudaError_t upload(T** d, const std::vector<T>& h) {
    if (h.empty()) {
        *d = nullptr;
        return cudaSuccess;
    }
    cudaError_t e = cudaMalloc(d, sizeof(T) * h.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
}

GExecArgs make_args(const GraphPlan* gp, const float2* in, float2* out, bool inv, int* d_status, int single,
                    int item0) {
    GExecArgs a{};
    a.in = in;
    a.out = out;
    a.work = gp->work;
    a.pool = gp->pool;
    a.shapes = gp->shapes;
    a.stages = gp->stages[inv ? 1 : 0];
    a.xf = gp->xf;
    a.items = single ? gp->items : gp->items_lag;
    a.nitems = gp->nitems;
    a.ctl = gp->ctl;
    a.qhead = gp->ctl;
    a.status = d_status;
    a.spin_limit = gp->spin_limit;
    a.single = single;
    a.item0 = item0;
    a.line_off = gp->line_off;
    a.withhold_xf = gp->withhold_xf;
    return a;
}

}  // namespace

bool graph_length_supported(int64_t n) {
    if (n < 1) return false;
    if (is_smooth(n)) return n <= (int64_t)kGTileMax * kGTileMax;
    return next_pow2(2 * n - 1) <= (int64_t)kGTileMax * kGTileMax;
}

namespace {
fft_status build_impl(GraphPlan* gp, const std::vector<int64_t>& lengths, int64_t batch, bool ragged,
                      const GLenConfig* force);
}

fft_status graph_plan_build(GraphPlan* gp, const std::vector<int64_t>& lengths, int64_t batch, bool ragged) {
    return build_impl(gp, lengths, batch, ragged, nullptr);
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
namespace {
std::mutex g_tune_mu;
std::map<std::string, GLenConfig> g_tune_cache;
bool g_tune_loaded = false;

std::string device_name() {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp pr{};
    cudaGetDeviceProperties(&pr, dev);
    std::string s = pr.name;
    for (auto& c : s)
        if (c == ' ') c = '_';
    return s;
}

void tune_cache_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = std::getenv("FFT_TUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    char line[512], key[256];
    while (std::fgets(line, sizeof line, f)) {
        if (std::strncmp(line, "pow2:", 5) == 0) continue;  // the batched power-of-two tuner's lines
        GLenConfig c;
        if (std::sscanf(line, "%255s %d %d %d %d", key, &c.tile_max, &c.split_n2, &c.lpt_a, &c.lpt_b) == 5)
            g_tune_cache[key] = c;
    }
    std::fclose(f);
}

void tune_cache_store(const std::string& key, const GLenConfig& c, double us) {
    g_tune_cache[key] = c;
    const char* path = std::getenv("FFT_TUNE_CACHE");
    if (!path) return;
    if (FILE* f = std::fopen(path, "a")) {
        std::fprintf(f, "%s %d %d %d %d %.2f\n", key.c_str(), c.tile_max, c.split_n2, c.lpt_a, c.lpt_b, us);
        std::fclose(f);
    }
}

std::vector<GLenConfig> tune_candidates(int64_t n, const GLenConfig& base) {
    std::vector<GLenConfig> out;
    auto halves = [](int cap) {
        std::vector<int> v;
        for (int l = cap; l >= 1 && (int)v.size() < 3; l /= 2) v.push_back(l);
        return v;
    };
    if (is_smooth(n) && n <= base.tile_max) {
        for (int l : halves(lines_per_tile((int)n, 0))) {
            GLenConfig c = base;
            c.lpt_a = l;
            out.push_back(c);
        }
    } else if (is_smooth(n)) {
        std::vector<std::pair<double, int64_t>> splits;
        for (int64_t b = 2; b <= base.tile_max; ++b) {
            if (n % b || n / b > base.tile_max || n / b < 2 || !is_smooth(b) || !is_smooth(n / b)) continue;
            splits.push_back({std::fabs(std::log((double)(n / b)) - std::log((double)b)), b});
        }
        std::sort(splits.begin(), splits.end());
        if (splits.size() > 3) splits.resize(3);
        // and the batched mixed four-step's split for M * 2^k
        const int64_t ms = mixed_split_n2(n);
        if (ms && std::none_of(splits.begin(), splits.end(), [&](const std::pair<double, int64_t>& v) {
                return v.second == ms;
            }))
            splits.insert(splits.begin(), {0.0, ms});  // first: the candidate list is capped
        for (size_t si = 0; si < splits.size(); ++si) {
            const int64_t n2 = splits[si].second, n1 = n / n2;
            for (int la : halves(lines_per_tile((int)n1, 0)))
                for (int lb : halves(lines_per_tile((int)n2, 0))) {
                    if (out.size() >= 24) break;
                    GLenConfig c = base;
                    c.split_n2 = (int)n2;
                    c.lpt_a = la;
                    c.lpt_b = lb;
                    out.push_back(c);
                }
        }
    }
    if (out.empty()) out.push_back(base);
    return out;
}
}  // namespace

GLenConfig tune_length(int64_t n, int64_t count, const GLenConfig& base) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_cache_load();
    const std::string key = device_name() + ":" + std::to_string(n);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) return it->second;
    std::vector<GLenConfig> cand = tune_candidates(n, base);
    if (cand.size() == 1) return cand[0];
    const int64_t reps = std::max<int64_t>(1, (int64_t(1) << 22) / n);
    (void)count;
    std::vector<int64_t> L((size_t)reps, n);
    float2 *x = nullptr, *y = nullptr;
    int* st = nullptr;
    if (cudaMalloc(&x, sizeof(float2) * reps * n) != cudaSuccess || cudaMalloc(&y, sizeof(float2) * reps * n) != cudaSuccess ||
        cudaMalloc(&st, sizeof(int)) != cudaSuccess) {
        cudaFree(x);
        cudaFree(y);
        return base;
    }
    cudaMemset(x, 0x3c, sizeof(float2) * reps * n);  // finite, non-zero values
    cudaMemset(st, 0, sizeof(int));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    GLenConfig best = base;
    float best_ms = 1e30f;
    for (const GLenConfig& c : cand) {
        GraphPlan tp;
        tp.no_tune = true;
        tp.use_graph = false;
        if (build_impl(&tp, L, reps, true, &c) != FFT_OK) {
            graph_plan_free(&tp);
            continue;
        }
        graph_plan_exec(&tp, x, y, false, 0, st, false);
        cudaEventRecord(e0);
        for (int it2 = 0; it2 < 5; ++it2) graph_plan_exec(&tp, x, y, false, 0, st, false);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        graph_plan_free(&tp);
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(x);
    cudaFree(y);
    cudaFree(st);
    tune_cache_store(key, best, best_ms * 1e3 / 5);
    return best;
}

namespace {
fft_status build_impl(GraphPlan* gp, const std::vector<int64_t>& lengths, int64_t batch, bool ragged,
                      const GLenConfig* force) {
    Builder B;
    GLenConfig cfg;
    cfg.tile_max = env_i("B300FFT_G_TILE_MAX", kGTileMax);
    if (cfg.tile_max > kGTileMax || cfg.tile_max < 16) cfg.tile_max = kGTileMax;
    cfg.lpt_a = env_i("B300FFT_G_LPT_A", 0);
    cfg.lpt_b = env_i("B300FFT_G_LPT_B", 0);
    for (int64_t n : lengths)
        if (!graph_length_supported(n)) return FFT_ERR_UNSUPPORTED;

    // kinds: distinct lengths, largest first (big work dequeued early)
    std::vector<int64_t> uniq(lengths.begin(), lengths.end());
    std::sort(uniq.begin(), uniq.end(), std::greater<int64_t>());
    uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
    struct Kind {
        int first, nstages;
        int64_t w1, w2;
        int64_t lines;
        bool group;  // ragged single-tile length: all its transforms are lines of one stage
    };
    std::map<int64_t, Kind> kinds;
    std::map<int64_t, int64_t> count_of;
    for (int64_t n : lengths) ++count_of[n];
    // per-length tile configuration: planner defaults or measured (autotuner)
    std::map<int64_t, GLenConfig> lcfg;
    const bool tune = env_i("FFT_AUTOTUNE", 0) != 0 && !gp->no_tune;
    for (int64_t n : uniq) lcfg[n] = force ? *force : (tune ? tune_length(n, ragged ? count_of[n] : batch, cfg) : cfg);
    std::vector<int64_t> line_off;  // element offsets of grouped lines
    {
        // packed offset of every transform, for the grouped lengths
        std::map<int64_t, std::vector<int64_t>> offs;
        if (ragged) {
            int64_t o = 0;
            for (int64_t n : lengths) {
                offs[n].push_back(o);
                o += n;
            }
        }
        const bool uniform = !ragged;
        for (int64_t n : uniq) {
            Kind k{};
            k.first = (int)B.st_f.size();
            const bool single_tile = is_smooth(n) && n <= lcfg[n].tile_max;
            k.group = ragged && single_tile;
            k.lines = single_tile ? (uniform ? batch : count_of[n]) : 1;
            if (k.lines > 0x7fffffffLL) return FFT_ERR_UNSUPPORTED;
            int64_t ltab = -1;
            if (k.group) {
                ltab = (int64_t)line_off.size();
                line_off.insert(line_off.end(), offs[n].begin(), offs[n].end());
            }
            if (!build_kind(B, n, k.lines, lcfg[n], &k.nstages, &k.w1, &k.w2, ltab)) return FFT_ERR_UNSUPPORTED;
            kinds[n] = k;
        }
    }
    gp->configs = lcfg;

    // transforms (packed offsets), workspace, counters
    std::vector<GTransform> xf;
    int64_t off = 0, woff = 0;
    int ctr = 0;
    auto add_xf = [&](int64_t n, int64_t at) {
        const Kind& k = kinds[n];
        GTransform x{};
        x.kind = k.first;
        x.nstages = k.nstages;
        x.ctr = ctr;
        ctr += k.nstages - 1;
        x.in_off = x.out_off = at;
        x.w1_off = woff;
        woff += (k.w1 + 1) & ~int64_t(1);
        x.w2_off = woff;
        woff += (k.w2 + 1) & ~int64_t(1);
        xf.push_back(x);
    };
    // test-only fault injection: the caller's transform number `wh` (its
    // record, when it has one of its own) never signals its first stage
    const int64_t wh = env_i("B300FFT_DEBUG_WITHHOLD_XF", -1);
    gp->withhold_xf = -1;
    if (ragged) {
        for (auto& kv : kinds)
            if (kv.second.group) add_xf(kv.first, 0);  // one transform holds every line of the length
        for (size_t i = 0; i < lengths.size(); ++i) {
            const int64_t n = lengths[i];
            if (!kinds[n].group) {
                if ((int64_t)i == wh) gp->withhold_xf = (int)xf.size();
                add_xf(n, off);
            }
            off += n;
        }
    } else {
        const int64_t n = lengths[0];
        if (kinds[n].lines > 1) add_xf(n, 0);
        else
            for (int64_t b = 0; b < batch; ++b) {
                if (b == wh) gp->withhold_xf = (int)xf.size();
                add_xf(n, b * n);
            }
    }
    if ((int64_t)xf.size() >= (int64_t(1) << 31)) return FFT_ERR_UNSUPPORTED;

    // queue: stage rounds; within a round, kinds largest first
    std::vector<uint64_t> items;
    int maxst = 0;
    for (auto& kv : kinds) maxst = std::max(maxst, kv.second.nstages);
    std::vector<std::vector<int>> by_kind;  // transform indices per kind, kinds in uniq order
    for (int64_t n : uniq) {
        std::vector<int> v;
        for (int t = 0; t < (int)xf.size(); ++t)
            if (xf[t].kind == kinds[n].first) v.push_back(t);
        by_kind.push_back(v);
    }
    gp->groups.clear();
    for (int s = 0; s < maxst; ++s) {
        for (size_t ki = 0; ki < uniq.size(); ++ki) {
            const Kind& k = kinds[uniq[ki]];
            if (s >= k.nstages) continue;
            const GStage& st = B.st_f[k.first + s];
            const int g0 = (int)items.size();
            for (int t : by_kind[ki])
                for (int tile = 0; tile < st.ntiles; ++tile)
                    items.push_back(((uint64_t)t << 32) | ((uint64_t)s << 24) | (uint64_t)tile);
            if ((int)items.size() > g0) gp->groups.push_back({g0, (int)items.size()});
        }
    }
    if (items.size() >= (size_t)0x7fffffff) return FFT_ERR_UNSUPPORTED;

    // Persistent-launch order: transforms in the same (largest kind first)
    // order, stage s of a transform placed `lag` items after its stage s-1,
    // so every dependency precedes its consumers in the queue.  A four-step
    // transform's second stage follows its first 5 x SMs items later (about
    // the CTAs in flight: the intermediate is read back from L2, and the
    // first stage is done by then): ragged mix 0.910 -> 0.845 ms against an
    // unlimited lag (1 x SMs: 1.24 ms, 2 x SMs: 0.93, 8 x SMs: 0.875).  Other
    // multi-stage transforms (Bluestein's chains) run every first stage before
    // any second one (an unlimited lag): Bluestein 1009 1025 vs 1116 us with
    // a short lag.
    std::vector<uint64_t> items_lag;
    {
        int dev0 = 0, sms0 = 148;
        cudaGetDevice(&dev0);
        cudaDeviceGetAttribute(&sms0, cudaDevAttrMultiProcessorCount, dev0);
        const int64_t lag_fs = env_i("B300FFT_G_LAG", 5 * sms0);
        struct Grp {
            int64_t key;
            int s, t, ntiles;
        };
        std::vector<Grp> grps;
        int64_t k0 = 0;
        for (size_t ki = 0; ki < uniq.size(); ++ki) {
            const Kind& k = kinds[uniq[ki]];
            const GStage& a0 = B.st_f[k.first];
            const bool fourstep = k.nstages == 2 && (a0.post == G_POST_TW4 || (a0.tmpl >= 2000 && a0.tmpl < 3000) ||
                                                     (a0.tmpl > 0 && a0.tmpl < 100 && (a0.tmpl & 1) == 0));
            const int64_t lag = fourstep ? lag_fs : (int64_t(1) << 30);
            for (int t : by_kind[ki]) {
                int64_t key = k0;
                for (int s2 = 0; s2 < k.nstages; ++s2) {
                    const int nt = B.st_f[k.first + s2].ntiles;
                    grps.push_back({key, s2, t, nt});
                    if (s2 == 0) k0 += nt;
                    key += std::max<int64_t>(lag, nt);
                }
            }
        }
        std::stable_sort(grps.begin(), grps.end(), [](const Grp& x, const Grp& y) {
            return x.key != y.key ? x.key < y.key : x.s < y.s;
        });
        items_lag.reserve(items.size());
        for (const Grp& g : grps)
            for (int tile = 0; tile < g.ntiles; ++tile)
                items_lag.push_back(((uint64_t)g.t << 32) | ((uint64_t)g.s << 24) | (uint64_t)tile);
        if (items_lag.size() != items.size()) return FFT_ERR_UNSUPPORTED;
    }
    // transforms whose stages are all compile-time tiles run in the lean
    // executor; with other transforms present they go last, in a launch of
    // their own (queue order kept within each part)
    gp->mix = false;
    gp->nrest = 0;
    {
        const bool allow = env_i("B300FFT_G_LEAN", 1) != 0;
        std::vector<char> xlean(xf.size(), 1);
        bool any_lean = false, all_lean = true, mix_full = false, mix_lean = false;
        for (size_t t = 0; t < xf.size(); ++t) {
            bool mx = false;
            for (int s2 = 0; s2 < xf[t].nstages; ++s2) {
                const int tm = B.st_f[xf[t].kind + s2].tmpl;
                xlean[t] &= allow && tm > 0;
                mx = mx || tm >= 1000;
            }
            gp->mix = gp->mix || mx;
            (xlean[t] ? mix_lean : mix_full) |= mx;
            any_lean = any_lean || xlean[t];
            all_lean = all_lean && xlean[t];
        }
        const bool split = any_lean && !all_lean && env_i("B300FFT_G_SPLIT", 1) != 0;
        if (any_lean && !all_lean && !split) mix_full = gp->mix;  // everything in the full executor
        gp->lean = all_lean;
        gp->kfull = mix_full ? GK_MIX : GK_BASE;
        gp->klean = mix_lean ? GK_LEANMIX : GK_LEAN;
        if (split) {
            std::vector<uint64_t> rest, lean;
            for (uint64_t it : items_lag) (xlean[it >> 32] ? lean : rest).push_back(it);
            gp->nrest = (int)rest.size();
            rest.insert(rest.end(), lean.begin(), lean.end());
            items_lag.swap(rest);
        }
    }

    // device data
    cudaStream_t st = 0;
    if (cudaMalloc(&gp->pool, sizeof(float2) * (size_t)std::max<int64_t>(B.pool_size, 2)) != cudaSuccess)
        return FFT_ERR_ALLOC;
    for (auto& t : B.pass_tabs)
        if (gen_pass_table(gp->pool + t.off, t.ns, t.r, st) != cudaSuccess) return FFT_ERR_CUDA;
    for (auto& t : B.root_tabs)
        if (gen_root_table(gp->pool + t.off, t.count, t.mult, t.n, st) != cudaSuccess) return FFT_ERR_CUDA;
    for (auto& t : B.pow2_tabs)
        if (gen_pow2_table(gp->pool + t.second, t.first, st) != cudaSuccess) return FFT_ERR_CUDA;
    for (auto& t : B.mixed_tabs)
        if (mixed_table_entries(t.first / 64, t.first % 64) > 0 &&
            gen_mixed_table(gp->pool + t.second, t.first / 64, t.first % 64, st) != cudaSuccess)
            return FFT_ERR_CUDA;
    if (!B.blue_list.empty()) {
        int64_t maxM = 0;
        for (auto& b : B.blue_list) maxM = std::max(maxM, b.M);
        double2* scratch = nullptr;
        if (cudaMalloc(&scratch, sizeof(double2) * 2 * (size_t)maxM) != cudaSuccess) return FFT_ERR_ALLOC;
        cudaError_t e = cudaSuccess;
        for (auto& b : B.blue_list) {
            if (e == cudaSuccess) e = gen_chirp(gp->pool + b.chirp, b.n, st);
            if (e == cudaSuccess) e = gen_bluestein_filter(gp->pool + b.ff, b.n, b.M, false, scratch, st);
            if (e == cudaSuccess) e = gen_bluestein_filter(gp->pool + b.fi, b.n, b.M, true, scratch, st);
        }
        cudaDeviceSynchronize();
        cudaFree(scratch);
        if (e != cudaSuccess) return FFT_ERR_CUDA;
    }
    if (upload(&gp->shapes, B.shapes) != cudaSuccess) return FFT_ERR_ALLOC;
    if (upload(&gp->stages[0], B.st_f) != cudaSuccess) return FFT_ERR_ALLOC;
    if (upload(&gp->stages[1], B.st_i) != cudaSuccess) return FFT_ERR_ALLOC;
    if (upload(&gp->xf, xf) != cudaSuccess) return FFT_ERR_ALLOC;
    if (upload(&gp->items, items) != cudaSuccess) return FFT_ERR_ALLOC;
    if (upload(&gp->items_lag, items_lag) != cudaSuccess) return FFT_ERR_ALLOC;
    if (upload(&gp->line_off, line_off) != cudaSuccess) return FFT_ERR_ALLOC;
    gp->nitems = (int)items.size();
    gp->ncounters = ctr;
    gp->ntransforms = (int)xf.size();
    if (cudaMalloc(&gp->ctl, sizeof(int) * (size_t)(2 + ctr)) != cudaSuccess) return FFT_ERR_ALLOC;
    gp->work_bytes = (size_t)woff * sizeof(float2);
    if (woff > 0 && cudaMalloc(&gp->work, gp->work_bytes) != cudaSuccess) return FFT_ERR_ALLOC;
    int bps[4] = {0, 0, 0, 0}, dev = 0, sms = 0;
    for (int k = 0; k < 4; ++k) {
        const void* kfn = gexec_fn(k);
        if (cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, gexec_smem(k)) != cudaSuccess)
            return FFT_ERR_CUDA;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps[k], kfn, kGThreads, gexec_smem(k)) != cudaSuccess ||
            bps[k] < 1)
            return FFT_ERR_CUDA;
    }
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    {
        GPart parts[2];
        gp->grid = gp->nitems;  // placeholders for gexec_parts
        const int np = gexec_parts(gp, parts);
        // beside a lean launch the full one takes two thirds of its CTA slots,
        // so the lean one starts on every SM at once (measured on the ragged
        // mix: 942 us vs 960 us with every slot, 948 us with half)
        const int pct = np > 1 ? env_i("B300FFT_G_FULL_PCT", 66) : 100;
        gp->grid = std::max(1, std::min(parts[0].nitems, sms * bps[parts[0].kind] * pct / 100));
        gp->grid_lean = np > 1 ? std::max(1, std::min(parts[1].nitems, sms * bps[gp->klean])) : 0;
    }
    gp->spin_limit = env_i("B300FFT_SPIN_LIMIT", 1 << 23);
    gp->use_graph = env_i("B300FFT_GRAPH", 1) != 0;
    char buf[256];
    std::snprintf(buf, sizeof buf,
                  "graph kinds=%zu transforms=%d items=%d stages<=%d grid=%d%s work=%zuB pool=%lldB",
                  uniq.size(), gp->ntransforms, gp->nitems, maxst, gp->grid,
                  gp->lean ? " lean" : (gp->nrest > 0 && gp->nrest < gp->nitems ? " +lean launch" : ""),
                  gp->work_bytes, (long long)(B.pool_size * 8));
    gp->desc = buf;
    if (cudaDeviceSynchronize() != cudaSuccess) return FFT_ERR_CUDA;
    return FFT_OK;
}
}  // namespace

void graph_plan_free(GraphPlan* gp) {
    cudaFree(gp->line_off);
    gp->line_off = nullptr;
    for (int d = 0; d < 2; ++d) {
        if (gp->gexec[d]) cudaGraphExecDestroy(gp->gexec[d]);
        if (gp->graph[d]) cudaGraphDestroy(gp->graph[d]);
        if (gp->stages[d]) cudaFree(gp->stages[d]);
        gp->gexec[d] = nullptr;
        gp->graph[d] = nullptr;
        gp->stages[d] = nullptr;
    }
    cudaFree(gp->pool);
    cudaFree(gp->shapes);
    cudaFree(gp->xf);
    cudaFree(gp->items);
    cudaFree(gp->items_lag);
    cudaFree(gp->ctl);
    cudaFree(gp->work);
    gp->pool = nullptr;
    gp->shapes = nullptr;
    gp->xf = nullptr;
    gp->items = nullptr;
    gp->items_lag = nullptr;
    gp->ctl = nullptr;
    gp->work = nullptr;
}

namespace {
// Capture memset(ctl) + the persistent launch(es) once per direction; later
// execs only patch the arguments of the kernel nodes.
cudaError_t ensure_graph(GraphPlan* gp, bool inv, const GExecArgs& a) {
    const int d = inv ? 1 : 0;
    if (gp->gexec[d]) return cudaSuccess;
    GPart parts[2];
    const int np = gexec_parts(gp, parts);
    // two launches sit on parallel branches of the graph (their transforms do
    // not depend on each other): the lean one takes the SMs the full one
    // leaves idle while its last dependency chains finish
    const bool par = np == 2 && env_i("B300FFT_G_PARALLEL", 1) != 0;
    cudaStream_t cs, cs2 = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    if (par) {
        if (cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev1, cudaEventDisableTiming) != cudaSuccess)
            e = cudaErrorMemoryAllocation;
    }
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(gp->ctl, 0, sizeof(int) * (size_t)(2 + gp->ncounters), cs);
        if (par) {
            cudaEventRecord(ev0, cs);
            cudaStreamWaitEvent(cs2, ev0, 0);
        }
        for (int i = 0; i < np; ++i) {
            GExecArgs b = a;
            b.items += parts[i].item0;
            b.nitems = parts[i].nitems;
            b.qhead = gp->ctl + parts[i].head;
            launch_gexec(parts[i].kind, parts[i].grid, b, par && i == 1 ? cs2 : cs);
        }
        if (par) {
            cudaEventRecord(ev1, cs2);
            cudaStreamWaitEvent(cs, ev1, 0);
        }
        const cudaError_t e2 = cudaStreamEndCapture(cs, &gp->graph[d]);
        e = cudaGetLastError() != cudaSuccess ? cudaErrorUnknown : e2;
    }
    cudaStreamDestroy(cs);
    if (cs2) cudaStreamDestroy(cs2);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (e != cudaSuccess) return e;
    size_t nn = 0;
    cudaGraphGetNodes(gp->graph[d], nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(gp->graph[d], nodes.data(), &nn);
    for (auto n : nodes) {
        cudaGraphNodeType t;
        cudaGraphNodeGetType(n, &t);
        if (t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp{};
        if (cudaGraphKernelNodeGetParams(n, &kp) != cudaSuccess) return cudaErrorUnknown;
        for (int i = 0; i < np; ++i)
            if (kp.func == gexec_fn(parts[i].kind)) gp->knode[d][i] = n;
    }
    for (int i = 0; i < np; ++i)
        if (!gp->knode[d][i]) return cudaErrorUnknown;
    return cudaGraphInstantiate(&gp->gexec[d], gp->graph[d], 0);
}
}  // namespace

fft_status graph_plan_exec(GraphPlan* gp, const float2* in, float2* out, bool inv, cudaStream_t st, int* d_status,
                           bool per_stage) {
    cudaError_t e = cudaSuccess;
    if (per_stage) {
        // one kernel for every group: the lean one only when it covers every transform
        const int k = gp->lean ? gp->klean : (gp->mix ? GK_MIX : GK_BASE);
        for (auto& g : gp->groups) {
            GExecArgs a = make_args(gp, in, out, inv, d_status, 1, g.first);
            launch_gexec(k, g.second - g.first, a, st);
            e = cudaGetLastError();
            if (e != cudaSuccess) return FFT_ERR_CUDA;
        }
        return FFT_OK;
    }
    GExecArgs a = make_args(gp, in, out, inv, d_status, 0, 0);
    GPart parts[2];
    const int np = gexec_parts(gp, parts);
    GExecArgs pa[2];
    for (int i = 0; i < np; ++i) {
        pa[i] = a;
        pa[i].items += parts[i].item0;
        pa[i].nitems = parts[i].nitems;
        pa[i].qhead = gp->ctl + parts[i].head;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cap);
    if (gp->use_graph && cap == cudaStreamCaptureStatusNone) {
        const int d = inv ? 1 : 0;
        if (ensure_graph(gp, inv, a) != cudaSuccess) return FFT_ERR_CUDA;
        for (int i = 0; i < np && e == cudaSuccess; ++i) {
            cudaKernelNodeParams kp{};
            void* params[1] = {&pa[i]};
            kp.func = const_cast<void*>(gexec_fn(parts[i].kind));
            kp.gridDim = dim3(parts[i].grid);
            kp.blockDim = dim3(kGThreads);
            kp.sharedMemBytes = gexec_smem(parts[i].kind);
            kp.kernelParams = params;
            e = cudaGraphExecKernelNodeSetParams(gp->gexec[d], gp->knode[d][i], &kp);
        }
        if (e == cudaSuccess) e = cudaGraphLaunch(gp->gexec[d], st);
        return e == cudaSuccess ? FFT_OK : FFT_ERR_CUDA;
    }
    e = cudaMemsetAsync(gp->ctl, 0, sizeof(int) * (size_t)(2 + gp->ncounters), st);
    for (int i = 0; i < np && e == cudaSuccess; ++i) {
        launch_gexec(parts[i].kind, parts[i].grid, pa[i], st);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? FFT_OK : FFT_ERR_CUDA;
}

}  // namespace b300fft

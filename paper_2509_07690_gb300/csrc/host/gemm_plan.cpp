// Tables of the precision form's tensor-core sup-sup update (HYLU Sec. 2.2,
// Fig. 1c: a supernode destination takes the updates of its source
// supernodes as dense products), built once per plan on the host.  See
// GemmPlan in plan.hpp.
#include <algorithm>
#include <vector>

#include "plan.hpp"

namespace hylu {

namespace {

int32_t round_up(int64_t x, int32_t m) { return (int32_t)((x + m - 1) / m * m); }

}  // namespace

int build_gemm_plan(const Plan& P, int32_t min_rows, GemmPlan& G) {
    G = GemmPlan();
    const int32_t n = P.n, nn = P.nnodes;
    G.gd_of_node.assign(nn, -1);
    if (min_rows <= 0 || nn == 0) return 0;
    G.min_src = std::min(16, std::max(2, min_rows));
    auto seg_len = [&](int32_t S) { return P.sn_start[S + 1] - P.sn_start[S]; };
    auto ntask = [&](int32_t S) { return P.node_ntask.empty() ? 0 : P.node_ntask[S]; };

    // ---- destinations: the supernodes of at least min_rows rows
    std::vector<char> is(nn, 0);
    for (int32_t D = 0; D < nn; ++D) is[D] = seg_len(D) >= min_rows;
    for (int32_t D = 0; D < nn; ++D)
        if (is[D]) {
            G.gd_of_node[D] = G.ngd++;
            G.gd_node.push_back(D);
        }
    if (G.ngd == 0) return 0;

    // ---- pairs (destination, large source supernode with tail entries at
    //      or past the destination's first row), their A columns and maps
    G.gd_slot.assign(P.lcols.size(), -1);
    std::vector<int32_t> colx(n, -1);          // global column -> U-column index of the destination
    std::vector<int32_t> pair_of(nn, -1);      // source -> pair of the current destination
    std::vector<int32_t> srcs;
    for (int32_t g = 0; g < G.ngd; ++g) {
        const int32_t D = G.gd_node[g];
        const int32_t r = P.sn_start[D], e = P.sn_start[D + 1] - 1, s = e - r + 1;
        const int64_t t0 = P.node_tail_off[D];
        const int32_t nT = (int32_t)(P.node_tail_off[D + 1] - t0);
        for (int32_t x = 0; x < s; ++x) colx[r + x] = x;
        for (int32_t j = 0; j < nT; ++j) colx[P.tcols[t0 + j]] = s + j;
        srcs.clear();
        for (int32_t i = r; i <= e; ++i)
            for (int64_t t = P.row_lptr[i]; t < P.row_lptr[i + 1];) {
                const int32_t S = P.node_of[P.lcols[t]];
                srcs.push_back(S);
                t += seg_len(S);
            }
        std::sort(srcs.begin(), srcs.end());
        srcs.erase(std::unique(srcs.begin(), srcs.end()), srcs.end());
        int32_t kp = 0;
        for (int32_t S : srcs) {
            if (seg_len(S) < G.min_src) continue;
            const int64_t a = P.node_tail_off[S], b = P.node_tail_off[S + 1];
            const int64_t jr = std::lower_bound(P.tcols.begin() + a, P.tcols.begin() + b, r) - P.tcols.begin();
            if (jr == b) continue;
            const int32_t p = (int32_t)G.pair_gd.size();
            pair_of[S] = p;
            G.pair_gd.push_back(g);
            G.pair_src.push_back(S);
            G.pair_u0.push_back(kp);
            G.pair_len.push_back(seg_len(S));
            G.pair_jr.push_back((int32_t)(jr - a));
            G.pair_nj.push_back((int32_t)(b - jr));
            G.pair_need.push_back(0);
            G.pair_x_off.push_back((int64_t)G.xmap.size());
            for (int64_t j = jr; j < b; ++j) {
                const int32_t x = colx[P.tcols[j]];
                if (x < 0) return -1;            // a tail column outside D's U columns: not closed
                G.xmap.push_back(x);
            }
            kp += round_up(seg_len(S), GemmPlan::TK);
        }
        for (int32_t i = r; i <= e; ++i)
            for (int64_t t = P.row_lptr[i]; t < P.row_lptr[i + 1];) {
                const int32_t S = P.node_of[P.lcols[t]];
                if (pair_of[S] >= 0) {
                    G.gd_slot[t] = pair_of[S];
                    G.pair_need[pair_of[S]]++;
                }
                t += seg_len(S);
            }
        for (int32_t S : srcs) pair_of[S] = -1;
        for (int32_t x = 0; x < s; ++x) colx[r + x] = -1;
        for (int32_t j = 0; j < nT; ++j) colx[P.tcols[t0 + j]] = -1;
        G.gd_Kp.push_back(kp);
        G.gd_Mp.push_back(round_up(s, GemmPlan::TM));
        G.gd_a_off.push_back(G.a_elems);
        G.a_elems += (int64_t)G.gd_Mp.back() * kp;
    }

    // ---- levels (Sec. 2.2.1): a row of another node as in the plan (after
    //      its sources complete and after the previous row of its node); a
    //      destination row walks after its sources complete, the
    //      destination's GEMM tasks come after every walk, the diagonal-block
    //      steps after the tasks, one row per level; tail tasks after the
    //      node's last row or step
    G.walk_level.assign(n, -1);
    G.diag_level.assign(n, -1);
    std::vector<int32_t> gemm_level(G.ngd, 0);
    auto done_level = [&](int32_t S) {
        const int32_t e = P.sn_start[S + 1] - 1;
        const int32_t last = is[S] ? G.diag_level[e] : G.walk_level[e];
        return last + (ntask(S) > 0 ? 1 : 0);
    };
    int32_t maxl = 0;
    for (int32_t D = 0; D < nn; ++D) {
        const int32_t r = P.sn_start[D], e = P.sn_start[D + 1] - 1;
        int32_t lg = 0;
        for (int32_t i = r; i <= e; ++i) {
            int32_t l = (!is[D] && i > r) ? G.walk_level[i - 1] + 1 : 0;
            for (int64_t t = P.row_lptr[i]; t < P.row_lptr[i + 1];) {
                const int32_t S = P.node_of[P.lcols[t]];
                l = std::max(l, done_level(S) + 1);
                t += seg_len(S);
            }
            G.walk_level[i] = l;
            lg = std::max(lg, l + 1);
        }
        if (is[D]) {
            gemm_level[G.gd_of_node[D]] = lg;
            for (int32_t i = r; i <= e; ++i) G.diag_level[i] = (i == r) ? lg + 1 : G.diag_level[i - 1] + 1;
        }
        maxl = std::max(maxl, done_level(D));
        maxl = std::max(maxl, is[D] ? G.diag_level[e] : G.walk_level[e]);
    }
    for (int32_t i = 0; i < n; ++i)
        if (G.diag_level[i] >= 0) G.diag_row.push_back(i);
    // rows' queue: tail tasks first inside a level, then diag tasks, then rows
    const int32_t nd = (int32_t)G.diag_row.size();
    std::vector<int32_t> task_lev(P.n_tasks);
    for (int32_t t = 0; t < P.n_tasks; ++t) task_lev[t] = done_level(P.task_node[t]);
    std::vector<int32_t> cnt(maxl + 2, 0);
    for (int32_t t = 0; t < P.n_tasks; ++t) cnt[task_lev[t] + 1]++;
    for (int32_t d = 0; d < nd; ++d) cnt[G.diag_level[G.diag_row[d]] + 1]++;
    for (int32_t i = 0; i < n; ++i) cnt[G.walk_level[i] + 1]++;
    for (int32_t l = 0; l <= maxl; ++l) cnt[l + 1] += cnt[l];
    G.row_order.assign((size_t)n + P.n_tasks + nd, 0);
    for (int32_t t = 0; t < P.n_tasks; ++t) G.row_order[cnt[task_lev[t]]++] = n + t;
    for (int32_t d = 0; d < nd; ++d) G.row_order[cnt[G.diag_level[G.diag_row[d]]]++] = n + P.n_tasks + d;
    for (int32_t i = 0; i < n; ++i) G.row_order[cnt[G.walk_level[i]]++] = i;
    G.levels = maxl + 1;
    // GEMM tasks by level, then pair, M tile, tail tile
    std::vector<int32_t> order(G.pair_gd.size());
    for (size_t p = 0; p < order.size(); ++p) order[p] = (int32_t)p;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return gemm_level[G.pair_gd[a]] < gemm_level[G.pair_gd[b]]; });
    G.gd_ntask.assign(G.ngd, 0);
    for (int32_t p : order) {
        const int32_t g = G.pair_gd[p];
        for (int32_t mt = 0; mt < G.gd_Mp[g] / GemmPlan::TM; ++mt)
            for (int32_t jt = 0; jt * GemmPlan::TN < G.pair_nj[p]; ++jt) {
                G.task_pair.push_back(p);
                G.task_mt.push_back(mt);
                G.task_jt.push_back(jt);
                G.task_level.push_back(gemm_level[g]);
                G.gd_ntask[g]++;
            }
    }
    return 0;
}

}  // namespace hylu

// Tables of the precision form's tensor-core sup-sup update (HYLU Sec. 2.2,
// Fig. 1c: a supernode destination takes the updates of its sources as dense
// products), built once per plan on the host.  See GemmPlan in plan.hpp.
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
    auto seg_len = [&](int32_t S) { return P.sn_start[S + 1] - P.sn_start[S]; };
    auto ntask = [&](int32_t S) { return P.node_ntask.empty() ? 0 : P.node_ntask[S]; };

    // ---- destinations: large supernodes and every node downstream of one
    std::vector<char> is(nn, 0);
    for (int32_t D = 0; D < nn; ++D) {
        const int32_t r = P.sn_start[D], e = P.sn_start[D + 1] - 1;
        bool g = (e - r + 1) >= min_rows;
        for (int32_t i = r; i <= e && !g; ++i)
            for (int64_t t = P.row_lptr[i]; t < P.row_lptr[i + 1];) {
                const int32_t S = P.node_of[P.lcols[t]];
                if (is[S]) { g = true; break; }
                t += seg_len(S);
            }
        is[D] = g;
    }
    for (int32_t D = 0; D < nn; ++D)
        if (is[D]) {
            G.gd_of_node[D] = G.ngd++;
            G.gd_node.push_back(D);
        }
    if (G.ngd == 0) return 0;

    // ---- per destination: union L columns, A block, union position of
    //      every L slot, and the (N tile, source segment) triples
    G.lu_pos.assign(P.lcols.size(), -1);
    G.gd_lc_off.push_back(0);
    G.gd_tile_base.push_back(0);
    G.pr_tri_off.push_back(0);
    G.pr_ck_off.push_back(0);
    std::vector<int32_t> colx(n, -1);        // global column -> U-column index of the destination
    std::vector<int32_t> lc;
    for (int32_t g = 0; g < G.ngd; ++g) {
        const int32_t D = G.gd_node[g];
        const int32_t r = P.sn_start[D], e = P.sn_start[D + 1] - 1, s = e - r + 1;
        const int64_t t0 = P.node_tail_off[D];
        const int32_t nT = (int32_t)(P.node_tail_off[D + 1] - t0);
        const int32_t w = s + nT;
        lc.clear();
        for (int32_t i = r; i <= e; ++i)
            lc.insert(lc.end(), P.lcols.begin() + P.row_lptr[i], P.lcols.begin() + P.row_lptr[i + 1]);
        std::sort(lc.begin(), lc.end());
        lc.erase(std::unique(lc.begin(), lc.end()), lc.end());
        const int32_t K = (int32_t)lc.size();
        G.gd_K.push_back(K);
        G.gd_Kp.push_back(round_up(K, GemmPlan::TK));
        G.gd_Mp.push_back(round_up(s, GemmPlan::TM));
        G.gd_a_off.push_back(G.a_elems);
        G.a_elems += (int64_t)G.gd_Mp.back() * G.gd_Kp.back();
        G.lc_cols.insert(G.lc_cols.end(), lc.begin(), lc.end());
        G.gd_lc_off.push_back((int64_t)G.lc_cols.size());
        for (int32_t i = r; i <= e; ++i)
            for (int64_t t = P.row_lptr[i]; t < P.row_lptr[i + 1]; ++t)
                G.lu_pos[t] = (int32_t)(std::lower_bound(lc.begin(), lc.end(), P.lcols[t]) - lc.begin());
        const int32_t ntiles = (w + GemmPlan::TN - 1) / GemmPlan::TN;
        G.gd_ntiles.push_back(ntiles);
        G.gd_tile_base.push_back(G.gd_tile_base.back() + ntiles);
        for (int32_t x = 0; x < s; ++x) colx[r + x] = x;
        for (int32_t j = 0; j < nT; ++j) colx[P.tcols[t0 + j]] = s + j;
        struct Tri { int32_t u0, len, S, jlo, jhi; };
        std::vector<std::vector<Tri>> per(ntiles);
        for (int32_t u = 0; u < K;) {
            const int32_t S = P.node_of[lc[u]], len = seg_len(S);
            if (lc[u] != P.sn_start[S] || u + len > K || lc[u + len - 1] != P.sn_start[S + 1] - 1) return -1;
            const int64_t a = P.node_tail_off[S], b = P.node_tail_off[S + 1];
            int64_t j = std::lower_bound(P.tcols.begin() + a, P.tcols.begin() + b, r) - P.tcols.begin();
            while (j < b) {
                const int32_t x = colx[P.tcols[j]];
                if (x < 0) return -1;                 // a tail column outside D's U columns: not closed
                const int32_t nt = x / GemmPlan::TN;
                int64_t j2 = j + 1;
                while (j2 < b && colx[P.tcols[j2]] >= 0 && colx[P.tcols[j2]] / GemmPlan::TN == nt) ++j2;
                per[nt].push_back({u, len, S, (int32_t)(j - a), (int32_t)(j2 - a)});
                j = j2;
            }
            u += len;
        }
        for (int32_t x = 0; x < s; ++x) colx[r + x] = -1;
        for (int32_t j = 0; j < nT; ++j) colx[P.tcols[t0 + j]] = -1;
        for (int32_t nt = 0; nt < ntiles; ++nt) {
            const int32_t base = (int32_t)G.tri_u0.size();
            for (const Tri& q : per[nt]) {
                const int32_t idx = (int32_t)G.tri_u0.size();
                G.tri_u0.push_back(q.u0);
                G.tri_len.push_back(q.len);
                G.tri_node.push_back(q.S);
                G.tri_jlo.push_back(q.jlo);
                G.tri_jhi.push_back(q.jhi);
                const int32_t k0 = q.u0 / GemmPlan::TK, k1 = (q.u0 + q.len - 1) / GemmPlan::TK;
                for (int32_t kc = k0; kc <= k1; ++kc) {
                    const size_t nc = G.ck_kc.size();
                    if (nc > (size_t)G.pr_ck_off.back() && G.ck_kc[nc - 1] == kc) {
                        G.ck_t1[nc - 1] = idx + 1;
                    } else {
                        G.ck_kc.push_back(kc);
                        G.ck_t0.push_back(idx);
                        G.ck_t1.push_back(idx + 1);
                    }
                }
            }
            (void)base;
            G.pr_tri_off.push_back((int32_t)G.tri_u0.size());
            G.pr_ck_off.push_back((int32_t)G.ck_kc.size());
        }
    }

    // ---- levels: nodes before any destination keep theirs; a destination
    //      row walks after its sources complete, the node's GEMM tiles after
    //      every walk, the diagonal-block steps after the tiles, one row per
    //      level, and its tail tasks after the last step
    G.walk_level.assign(n, -1);
    G.diag_level.assign(n, -1);
    std::vector<int32_t> gemm_level(G.ngd, 0);
    auto done_level = [&](int32_t S) {
        const int32_t e = P.sn_start[S + 1] - 1;
        const int32_t last = is[S] ? G.diag_level[e] : P.row_level[e];
        return last + (ntask(S) > 0 ? 1 : 0);
    };
    int32_t maxl = P.row_levels - 1;
    for (int32_t g = 0; g < G.ngd; ++g) {
        const int32_t D = G.gd_node[g];
        const int32_t r = P.sn_start[D], e = P.sn_start[D + 1] - 1;
        int32_t lg = 0;
        for (int32_t i = r; i <= e; ++i) {
            int32_t l = 0;
            for (int64_t t = P.row_lptr[i]; t < P.row_lptr[i + 1];) {
                const int32_t S = P.node_of[P.lcols[t]];
                l = std::max(l, done_level(S) + 1);
                t += seg_len(S);
            }
            G.walk_level[i] = l;
            lg = std::max(lg, l + 1);
        }
        gemm_level[g] = lg;
        for (int32_t i = r; i <= e; ++i) G.diag_level[i] = (i == r) ? lg + 1 : G.diag_level[i - 1] + 1;
        maxl = std::max(maxl, done_level(D));
    }
    for (int32_t i = 0; i < n; ++i)
        if (!is[P.node_of[i]]) G.walk_level[i] = P.row_level[i];
    for (int32_t i = 0; i < n; ++i)
        if (G.diag_level[i] >= 0) G.diag_row.push_back(i);
    // rows' queue: tail tasks first inside a level, then diag tasks, then rows
    const int32_t nd = (int32_t)G.diag_row.size();
    std::vector<int32_t> task_lev(P.n_tasks);
    for (int32_t t = 0; t < P.n_tasks; ++t) {
        const int32_t S = P.task_node[t];
        task_lev[t] = is[S] ? G.diag_level[P.sn_start[S + 1] - 1] + 1 : P.task_level[t];
    }
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
    // GEMM tasks by level, then destination, M tile, N tile
    std::vector<int32_t> order(G.ngd);
    for (int32_t g = 0; g < G.ngd; ++g) order[g] = g;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return gemm_level[a] < gemm_level[b]; });
    for (int32_t g : order)
        for (int32_t mt = 0; mt < G.gd_Mp[g] / GemmPlan::TM; ++mt)
            for (int32_t nt = 0; nt < G.gd_ntiles[g]; ++nt) {
                G.task_gd.push_back(g);
                G.task_mt.push_back(mt);
                G.task_nt.push_back(nt);
                G.task_level.push_back(gemm_level[g]);
            }
    return 0;
}

}  // namespace hylu

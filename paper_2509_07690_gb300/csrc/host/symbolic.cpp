// Symbolic factorization, supernode detection, padded storage pattern and
// the node/task tables of the numeric phase (HYLU Sec. 2.1 and Sec. 2.2).
//
// Row structure (up-looking): row i holds Ahat(i,:), i, and for every k < i it
// holds, U(k, >k).  Rows are found by depth-first search over the graph of U
// from the lower entries of Ahat(i,:).  The search follows a pruned adjacency
// (Eisenstat and Liu): once a row p with L(p,k) != 0 and U(k,p) != 0 has been
// built, U(k, >p) is contained in U(p,:), so the search from k may stop at p.
// This gives the same sets as the plain closure in far less time.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "plan.hpp"

namespace hylu {

void symbolic_rows(const CsrPattern& ahat, std::vector<int64_t>& frp, std::vector<int32_t>& fci,
                   std::vector<int64_t>& fdiag) {
    const int32_t n = ahat.n;
    frp.assign(n + 1, 0);
    fci.clear();
    fci.reserve((size_t)ahat.rp[n] * 4 + n);
    fdiag.assign(n, 0);
    std::vector<int64_t> prune_end(n, -1);     // end (exclusive) of the traversed part of U(k,:)
    std::vector<int32_t> mark(n, -1);
    std::vector<int32_t> lset, uset;
    std::vector<std::pair<int32_t, int64_t>> stack;
    for (int32_t i = 0; i < n; ++i) {
        lset.clear(); uset.clear();
        mark[i] = i; uset.push_back(i);
        for (int64_t q = ahat.rp[i]; q < ahat.rp[i + 1]; ++q) {
            int32_t c = ahat.ci[q];
            if (mark[c] == i) continue;
            mark[c] = i;
            if (c > i) { uset.push_back(c); continue; }
            // DFS from c over the pruned U graph, collecting nodes < i
            lset.push_back(c);
            stack.clear();
            stack.push_back({c, fdiag[c] + 1});
            while (!stack.empty()) {
                int32_t k = stack.back().first;
                int64_t& it = stack.back().second;
                int64_t end = prune_end[k] >= 0 ? prune_end[k] : frp[k + 1];
                bool pushed = false;
                while (it < end) {
                    int32_t j = fci[it++];
                    if (mark[j] == i) continue;
                    mark[j] = i;
                    if (j < i) { lset.push_back(j); stack.push_back({j, fdiag[j] + 1}); pushed = true; break; }
                    uset.push_back(j);
                }
                if (!pushed) stack.pop_back();
            }
        }
        std::sort(lset.begin(), lset.end());
        std::sort(uset.begin(), uset.end());
        fci.insert(fci.end(), lset.begin(), lset.end());
        fdiag[i] = (int64_t)fci.size();
        fci.insert(fci.end(), uset.begin(), uset.end());
        frp[i + 1] = (int64_t)fci.size();
        // symmetric pruning of the sources of row i
        for (int32_t k : lset) {
            if (prune_end[k] >= 0) continue;
            const int32_t* b = fci.data() + fdiag[k] + 1;
            const int32_t* e = fci.data() + frp[k + 1];
            const int32_t* f = std::lower_bound(b, e, i);
            if (f != e && *f == i) prune_end[k] = (int64_t)(f - fci.data()) + 1;
        }
    }
}

void supernode_partition(int32_t n, const std::vector<int64_t>& frp, const std::vector<int32_t>& fci,
                         const std::vector<int64_t>& fdiag, int32_t sn_max, std::vector<int32_t>& start) {
    start.clear();
    start.push_back(0);
    int32_t cur = 0;
    for (int32_t r = 0; r + 1 < n; ++r) {
        int64_t lr = frp[r + 1] - fdiag[r], ln = frp[r + 2] - fdiag[r + 1];
        bool same = (lr - 1 == ln) &&
                    std::memcmp(fci.data() + fdiag[r] + 1, fci.data() + fdiag[r + 1], sizeof(int32_t) * ln) == 0;
        if (!same || (r + 1 - cur) >= sn_max) { cur = r + 1; start.push_back(r + 1); }
    }
    start.push_back(n);
}

// Padded pattern (Sec. 2.2 storage, read as): each row keeps its own L
// columns, widened to whole source supernodes; every node stores its rows'
// diagonal block densely together with the shared U tail.
void build_nodes(Plan& P, const std::vector<int64_t>& frp, const std::vector<int32_t>& fci,
                 const std::vector<int64_t>& fdiag) {
    const int32_t n = P.n;
    const int32_t nn = (int32_t)P.sn_start.size() - 1;
    P.nnodes = nn;
    P.node_of.assign(n, 0);
    for (int32_t s = 0; s < nn; ++s)
        for (int32_t i = P.sn_start[s]; i < P.sn_start[s + 1]; ++i) P.node_of[i] = s;
    P.row_lptr.assign(n + 1, 0);
    P.lcols.clear();
    P.node_tail_off.assign(nn + 1, 0);
    P.node_panel_off.assign(nn + 1, 0);
    P.tcols.clear();
    std::vector<char> in(n, 0);
    std::vector<int32_t> lst;
    int64_t poff = 0;
    P.max_row = 0;
    for (int32_t s = 0; s < nn; ++s) {
        int32_t r = P.sn_start[s], e = P.sn_start[s + 1] - 1, sz = e - r + 1;
        for (int64_t q = fdiag[e] + 1; q < frp[e + 1]; ++q) P.tcols.push_back(fci[q]);
        P.node_tail_off[s + 1] = (int64_t)P.tcols.size();
        int64_t w = sz + (P.node_tail_off[s + 1] - P.node_tail_off[s]);
        P.node_panel_off[s] = poff;
        poff += w * sz;
        P.node_panel_off[s + 1] = poff;
        for (int32_t i = r; i <= e; ++i) {
            lst.clear();
            for (int64_t q = frp[i]; q < fdiag[i]; ++q) {
                int32_t k = fci[q];
                if (k >= r) break;
                if (in[k]) continue;
                int32_t S = P.node_of[k];
                for (int32_t t = P.sn_start[S]; t < P.sn_start[S + 1]; ++t)
                    if (!in[t]) { in[t] = 1; lst.push_back(t); }
            }
            std::sort(lst.begin(), lst.end());
            for (int32_t t : lst) in[t] = 0;
            P.lcols.insert(P.lcols.end(), lst.begin(), lst.end());
            P.row_lptr[i + 1] = (int64_t)P.lcols.size();
            P.max_row = std::max<int32_t>(P.max_row, (int32_t)(lst.size() + w));
        }
    }
    P.nnz_l = (int64_t)P.lcols.size();
    P.nnz_panel = poff;
    P.nnz_store = P.nnz_l + P.nnz_panel;
    // flop counts (Sec. 2.1): one division per L(i,k) plus two per U(k, >k) entry
    double fu = 0.0, fp = 0.0;
    std::vector<int64_t> ulen(n);
    for (int32_t i = 0; i < n; ++i) ulen[i] = frp[i + 1] - fdiag[i];
    for (int32_t i = 0; i < n; ++i)
        for (int64_t q = frp[i]; q < fdiag[i]; ++q) fu += 1.0 + 2.0 * (double)(ulen[fci[q]] - 1);
    P.row_flops.assign(n, 0.0);
    for (int32_t i = 0; i < n; ++i) {
        double f = 0.0;
        for (int64_t t = P.row_lptr[i]; t < P.row_lptr[i + 1]; ++t) f += 1.0 + 2.0 * (double)(ulen[P.lcols[t]] - 1);
        for (int32_t k = P.sn_start[P.node_of[i]]; k < i; ++k) f += 1.0 + 2.0 * (double)(ulen[k] - 1);
        P.row_flops[i] = f;
        fp += f;
    }
    P.flops_unpadded = fu;
    P.flops_padded = fp;
    P.nnz_f = frp[n];
    // tail tasks: a 32-column group costs s^2 / 2 multiply-adds per lane; a
    // task takes about 512 of them (one group from s = 32 up), at most one
    // task per group.  A node whose whole tail is about one task's work (or
    // less) gets none: its last row solves the tail after its own
    // diagonal-block step, saving a claim and a hand-off.
    P.node_ntask.assign(nn, 0);
    for (int32_t D = 0; D < nn; ++D) {
        const int64_t sz = P.sn_start[D + 1] - P.sn_start[D];
        const int64_t nT = P.node_tail_off[D + 1] - P.node_tail_off[D];
        if (sz < 2 || nT == 0) continue;
        const int64_t ng = (nT + 31) / 32;
        if (sz * sz * ng <= 1024) continue;
        const int64_t want = (sz * sz * ng + 1023) / 1024;
        P.node_ntask[D] = (int32_t)std::max<int64_t>(1, std::min<int64_t>(want, ng));
    }
    // dependency levels (Sec. 2.2.1: the task graph is levelized so that tasks
    // of one level are independent); claiming level by level keeps the claimed
    // tasks close to ready
    std::vector<int32_t> lev(n, 0);
    auto done_level = [&](int32_t S) {
        return lev[P.sn_start[S + 1] - 1] + (P.node_ntask[S] > 0 ? 1 : 0);
    };
    int32_t maxl = 0;
    for (int32_t i = 0; i < n; ++i) {
        const int32_t D = P.node_of[i], r = P.sn_start[D];
        int32_t l = (i > r) ? lev[i - 1] + 1 : 0;
        for (int64_t t = P.row_lptr[i]; t < P.row_lptr[i + 1];) {
            const int32_t S = P.node_of[P.lcols[t]];
            l = std::max(l, done_level(S) + 1);
            t += P.sn_start[S + 1] - P.sn_start[S];   // whole segment of S
        }
        lev[i] = l;
        maxl = std::max(maxl, l);
    }
    P.task_node.clear();
    P.task_chunk.clear();
    P.task_level.clear();
    for (int32_t D = 0; D < nn; ++D)
        for (int32_t c = 0; c < P.node_ntask[D]; ++c) {
            P.task_node.push_back(D);
            P.task_chunk.push_back(c);
            P.task_level.push_back(done_level(D));
            maxl = std::max(maxl, done_level(D));
        }
    P.n_tasks = (int32_t)P.task_node.size();
    P.row_levels = maxl + 1;
    P.row_level = lev;
    // tasks first inside a level: they complete nodes and never wait long
    std::vector<int32_t> cnt(maxl + 2, 0);
    for (int32_t i = 0; i < n; ++i) cnt[lev[i] + 1]++;
    for (int32_t t = 0; t < P.n_tasks; ++t) cnt[P.task_level[t] + 1]++;
    for (int32_t l = 0; l <= maxl; ++l) cnt[l + 1] += cnt[l];
    P.row_order.assign((size_t)n + P.n_tasks, 0);
    for (int32_t t = 0; t < P.n_tasks; ++t) P.row_order[cnt[P.task_level[t]]++] = n + t;
    for (int32_t i = 0; i < n; ++i) P.row_order[cnt[lev[i]]++] = i;

    // ---- substitution schedules
    const int32_t nn2 = P.nnodes;
    P.fwd_level.assign(nn2, 0);
    P.bwd_level.assign(nn2, 0);
    for (int32_t D = 0; D < nn2; ++D) {          // forward: sources are earlier nodes
        int32_t l = 0;
        for (int32_t i = P.sn_start[D]; i < P.sn_start[D + 1]; ++i)
            for (int64_t t = P.row_lptr[i]; t < P.row_lptr[i + 1];) {
                const int32_t S = P.node_of[P.lcols[t]];
                l = std::max(l, P.fwd_level[S] + 1);
                t += P.sn_start[S + 1] - P.sn_start[S];
            }
        P.fwd_level[D] = l;
    }
    for (int32_t D = nn2 - 1; D >= 0; --D) {     // backward: tail columns are later nodes
        int32_t l = 0;
        for (int64_t t = P.node_tail_off[D]; t < P.node_tail_off[D + 1]; ++t)
            l = std::max(l, P.bwd_level[P.node_of[P.tcols[t]]] + 1);
        P.bwd_level[D] = l;
    }
    auto schedule = [&](const std::vector<int32_t>& nl, bool descending, std::vector<int32_t>& order,
                        std::vector<int32_t>& count) {
        int32_t ml = 0;
        for (int32_t D = 0; D < nn2; ++D) ml = std::max(ml, nl[D]);
        count.assign(ml + 1, 0);
        for (int32_t D = 0; D < nn2; ++D) count[nl[D]]++;
        std::vector<int64_t> start(ml + 2, 0);
        for (int32_t D = 0; D < nn2; ++D) start[nl[D] + 1] += P.sn_start[D + 1] - P.sn_start[D];
        for (int32_t l = 0; l <= ml; ++l) start[l + 1] += start[l];
        order.assign(n, 0);
        if (!descending) {
            for (int32_t i = 0; i < n; ++i) order[start[nl[P.node_of[i]]]++] = i;
        } else {
            for (int32_t i = n - 1; i >= 0; --i) order[start[nl[P.node_of[i]]]++] = i;
        }
    };
    schedule(P.fwd_level, false, P.fwd_order, P.fwd_count);
    schedule(P.bwd_level, true, P.bwd_order, P.bwd_count);

    // ---- transpose substitution.  U^T v = h: node D needs every earlier node
    //      whose U tail reaches a column of D.  L^T u = v: node D needs every
    //      later node with an L entry in a column of D.  Rows are counted per
    //      level (each row task pushes its own contributions).
    P.ut_level.assign(nn2, 0);
    P.lt_level.assign(nn2, 0);
    for (int32_t S = 0; S < nn2; ++S)
        for (int64_t t = P.node_tail_off[S]; t < P.node_tail_off[S + 1]; ++t) {
            const int32_t D = P.node_of[P.tcols[t]];
            P.ut_level[D] = std::max(P.ut_level[D], P.ut_level[S] + 1);
        }
    for (int32_t J = nn2 - 1; J >= 0; --J)
        for (int32_t i = P.sn_start[J]; i < P.sn_start[J + 1]; ++i)
            for (int64_t t = P.row_lptr[i]; t < P.row_lptr[i + 1];) {
                const int32_t D = P.node_of[P.lcols[t]];
                P.lt_level[D] = std::max(P.lt_level[D], P.lt_level[J] + 1);
                t += P.sn_start[D + 1] - P.sn_start[D];
            }
    auto row_schedule = [&](const std::vector<int32_t>& nl, bool descending, std::vector<int32_t>& order,
                            std::vector<int32_t>& count) {
        int32_t ml = 0;
        for (int32_t D = 0; D < nn2; ++D) ml = std::max(ml, nl[D]);
        count.assign(ml + 1, 0);
        std::vector<int64_t> start(ml + 2, 0);
        for (int32_t D = 0; D < nn2; ++D) {
            const int32_t rows = P.sn_start[D + 1] - P.sn_start[D];
            count[nl[D]] += rows;
            start[nl[D] + 1] += rows;
        }
        for (int32_t l = 0; l <= ml; ++l) start[l + 1] += start[l];
        order.assign(n, 0);
        if (!descending) {
            for (int32_t i = 0; i < n; ++i) order[start[nl[P.node_of[i]]]++] = i;
        } else {
            for (int32_t i = n - 1; i >= 0; --i) order[start[nl[P.node_of[i]]]++] = i;
        }
    };
    row_schedule(P.ut_level, false, P.ut_order, P.ut_count);   // first row of a node first
    row_schedule(P.lt_level, true, P.lt_order, P.lt_count);    // last row of a node first
}

// Rows whose own update work dwarfs the rest (the dense rows that AMD puts
// last in circuit matrices) sit at the deepest levels, so level order would
// claim them last although most of their sources finish early.  Claimed at
// once, they consume those sources while the rest of the task graph is still
// running (Sec. 2.2.1 pipeline mode).  A row qualifies only if it has that
// early work: the prefix of its L list (taken in order, as the kernel does)
// whose sources lie at no more than half its level carries at least half of
// its flops.  Top separators of nested dissection fail the test: their
// sources finish late, and claiming them early would only idle warps.
void split_heavy_rows(Plan& P, double heavy_ratio) {
    const int32_t n = P.n;
    P.heavy_order.clear();
    P.heavy_rank.assign(n, INT32_MAX);
    if (!(heavy_ratio > 0.0) || n == 0) return;
    double tot = 0.0;
    for (double f : P.row_flops) tot += f;
    const double cut = std::max(1e6, heavy_ratio * tot / (double)n);
    std::vector<int32_t> ulen(n);
    for (int32_t D = 0; D < P.nnodes; ++D) {
        const int32_t nT = (int32_t)(P.node_tail_off[D + 1] - P.node_tail_off[D]);
        for (int32_t i = P.sn_start[D]; i < P.sn_start[D + 1]; ++i) ulen[i] = (P.sn_start[D + 1] - i) + nT;
    }
    for (size_t q = 0; q < P.row_order.size(); ++q) {
        const int32_t i = P.row_order[q];
        if (i >= n || P.row_flops[i] < cut) continue;
        const int32_t lam = P.row_level[i] / 2;
        double early = 0.0;
        for (int64_t t = P.row_lptr[i]; t < P.row_lptr[i + 1]; ++t) {
            const int32_t k = P.lcols[t];
            const int32_t eS = P.sn_start[P.node_of[k] + 1] - 1;
            if (P.row_level[eS] > lam) break;
            early += 1.0 + 2.0 * (double)(ulen[k] - 1);
        }
        if (early >= 0.5 * P.row_flops[i]) {
            P.heavy_rank[i] = (int32_t)P.heavy_order.size();
            P.heavy_order.push_back(i);
        }
    }
}

}  // namespace hylu

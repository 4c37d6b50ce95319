// Symbolic factorization, supernode detection, padded storage pattern and
// the node/task tables of the numeric phase (HYLU Sec. 2.1 and Sec. 2.2).
//
// Row structure (up-looking): row i holds Ahat(i,:), i, and for every k < i it
// holds, U(k, >k).  Rows are found by a search over the graph of U from the
// lower entries of Ahat(i,:), with two reductions that leave the sets as they
// are:
//   - symmetric pruning (Eisenstat and Liu): once a row p with L(p,k) != 0 and
//     U(k,p) != 0 has been built, U(k, >p) is contained in U(p,:), so the
//     search through k may stop at p;
//   - chains: when U(k+1,:) = U(k,:) \ {k} for k = a..e-1, every U(k, >k) in
//     the chain is {k+1..e} plus U(e, >e).  Reaching any k of it puts k..e
//     into L(i,:) at once, and only U(e, >e) is searched.
// L(i,:) is kept as runs of consecutive columns; U(i,:) is the union of the
// sorted lists searched, merged.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "plan.hpp"

namespace hylu {

void symbolic_rows(const CsrPattern& ahat, SymbolicRows& F) {
    const int32_t n = ahat.n;
    F.urp.assign(n + 1, 0);
    F.uci.clear();
    F.uci.reserve((size_t)ahat.rp[n] * 2 + n);
    F.lrp.assign(n + 1, 0);
    F.lrun_first.clear();
    F.lrun_len.clear();
    F.nnz_l = 0;
    std::vector<int64_t>& urp = F.urp;
    std::vector<int32_t>& uci = F.uci;
    std::vector<int64_t> prune_end(n, -1);      // end (exclusive) of the searched part of U(k,:)
    std::vector<int32_t> mark(n, -1);
    std::vector<int32_t> chain_first(n), chain_end(n);
    std::vector<int32_t> uset, ubuf, ends, work, merged;
    std::vector<std::pair<int32_t, int32_t>> runs;   // L runs: (first column, count)
    std::vector<size_t> ucut, ncut;                  // boundaries of the sorted runs of uset
    for (int32_t i = 0; i < n; ++i) {
        uset.clear(); runs.clear(); ends.clear(); work.clear(); ucut.clear();
        mark[i] = i;
        uset.push_back(i);
        auto visit = [&](int32_t k) {                // k < i, not yet in row i
            const int32_t e = chain_end[chain_first[k]];
            int32_t j = k;
            while (j <= e && mark[j] != i) mark[j++] = i;
            runs.push_back({k, j - k});
            if (j > e) { work.push_back(e); ends.push_back(e); }
        };
        for (int64_t q = ahat.rp[i]; q < ahat.rp[i + 1]; ++q) {
            const int32_t c = ahat.ci[q];
            if (mark[c] == i) continue;
            if (c > i) { mark[c] = i; uset.push_back(c); continue; }
            visit(c);
        }
        ucut.push_back(0);
        if (work.size() > 1) {                       // the longest list first: one long sorted run
            size_t best = 0;
            int64_t bl = -1;
            for (size_t t = 0; t < work.size(); ++t) {
                const int32_t e = work[t];
                const int64_t len = (prune_end[e] >= 0 ? prune_end[e] : urp[e + 1]) - urp[e];
                if (len > bl) { bl = len; best = t; }
            }
            std::swap(work[best], work.back());
        }
        while (!work.empty()) {
            const int32_t e = work.back();
            work.pop_back();
            if (uset.size() != ucut.back()) ucut.push_back(uset.size());
            const int64_t end = prune_end[e] >= 0 ? prune_end[e] : urp[e + 1];
            for (int64_t it = urp[e] + 1; it < end; ++it) {
                const int32_t j = uci[it];
                if (mark[j] == i) continue;
                if (j < i) { visit(j); continue; }
                mark[j] = i;
                uset.push_back(j);
            }
        }
        if (uset.size() != ucut.back()) ucut.push_back(uset.size());
        // ---- L: disjoint runs, sorted by their first column (or read off the
        //      marks when the row is dense in its range)
        if (!runs.empty()) {
            int32_t lo = i;
            int64_t nl = 0;
            for (auto& r : runs) { lo = std::min(lo, r.first); nl += r.second; }
            const double rs = (double)runs.size();
            if (rs * (std::log2(rs) + 1.0) * 4.0 > (double)(i - lo)) {
                runs.clear();
                for (int32_t j = lo; j < i; ++j) {
                    if (mark[j] != i) continue;
                    int32_t t = j;
                    while (t < i && mark[t] == i) ++t;
                    runs.push_back({j, t - j});
                    j = t;
                }
            } else {
                std::sort(runs.begin(), runs.end());
            }
            for (auto& r : runs) { F.lrun_first.push_back(r.first); F.lrun_len.push_back(r.second); }
            F.nnz_l += nl;
        }
        F.lrp[i + 1] = (int64_t)F.lrun_first.size();
        // ---- U: one long run plus short ones, pairwise merges, or the marks
        if (ucut.size() > 2) {
            const size_t R = ucut.size() - 1;
            const double m = (double)uset.size();
            size_t big = 0, bsz = 0;
            int32_t hi = i;
            for (size_t r = 0; r < R; ++r) {
                if (ucut[r + 1] - ucut[r] > bsz) { bsz = ucut[r + 1] - ucut[r]; big = r; }
                hi = std::max(hi, uset[ucut[r + 1] - 1]);
            }
            const double rest = m - (double)bsz;
            const double c_pair = m * std::log2((double)R), c_big = m + rest * std::log2(rest + 2.0);
            if (R > 2 && c_pair * 4.0 > (double)(hi - i)) {
                int32_t* o = uset.data();
                for (int32_t j = i; j <= hi; ++j) if (mark[j] == i) *o++ = j;
            } else if (c_big < c_pair) {
                ubuf.clear();
                for (size_t r = 0; r < R; ++r)
                    if (r != big) ubuf.insert(ubuf.end(), uset.begin() + ucut[r], uset.begin() + ucut[r + 1]);
                std::sort(ubuf.begin(), ubuf.end());
                merged.resize(uset.size());
                std::merge(uset.begin() + ucut[big], uset.begin() + ucut[big + 1], ubuf.begin(), ubuf.end(),
                           merged.begin());
                uset.swap(merged);
            } else {
                while (ucut.size() > 2) {
                    ubuf.resize(uset.size());
                    ncut.assign(1, 0);
                    size_t r = 0;
                    for (; r + 2 < ucut.size(); r += 2) {
                        std::merge(uset.begin() + ucut[r], uset.begin() + ucut[r + 1], uset.begin() + ucut[r + 1],
                                   uset.begin() + ucut[r + 2], ubuf.begin() + ucut[r]);
                        ncut.push_back(ucut[r + 2]);
                    }
                    if (r + 1 < ucut.size()) {
                        std::copy(uset.begin() + ucut[r], uset.begin() + ucut[r + 1], ubuf.begin() + ucut[r]);
                        ncut.push_back(ucut[r + 1]);
                    }
                    uset.swap(ubuf);
                    ucut.swap(ncut);
                }
            }
        }
        uci.insert(uci.end(), uset.begin(), uset.end());
        urp[i + 1] = (int64_t)uci.size();
        // ---- symmetric pruning of the searched chain ends
        for (int32_t k : ends) {
            if (prune_end[k] >= 0) continue;
            const int32_t* b = uci.data() + urp[k] + 1;
            const int32_t* e = uci.data() + urp[k + 1];
            const int32_t* f = std::lower_bound(b, e, i);
            if (f != e && *f == i) prune_end[k] = (int64_t)(f - uci.data()) + 1;
        }
        // ---- chains: row i continues row i-1 when U(i,:) = U(i-1,:) \ {i-1}
        bool cont = false;
        if (i > 0) {
            const int64_t lp = urp[i] - urp[i - 1], li = urp[i + 1] - urp[i];
            cont = (lp - 1 == li) &&
                   std::memcmp(uci.data() + urp[i - 1] + 1, uci.data() + urp[i], sizeof(int32_t) * li) == 0;
        }
        if (cont) { chain_first[i] = chain_first[i - 1]; chain_end[chain_first[i]] = i; }
        else { chain_first[i] = i; chain_end[i] = i; }
    }
}

void supernode_partition(int32_t n, const SymbolicRows& F, int32_t sn_max, std::vector<int32_t>& start) {
    start.clear();
    start.push_back(0);
    int32_t cur = 0;
    for (int32_t r = 0; r + 1 < n; ++r) {
        const int64_t lr = F.urp[r + 1] - F.urp[r], ln = F.urp[r + 2] - F.urp[r + 1];
        const bool same = (lr - 1 == ln) &&
                          std::memcmp(F.uci.data() + F.urp[r] + 1, F.uci.data() + F.urp[r + 1],
                                      sizeof(int32_t) * ln) == 0;
        if (!same || (r + 1 - cur) >= sn_max) { cur = r + 1; start.push_back(r + 1); }
    }
    if (n > 0) start.push_back(n);     // an empty matrix has no supernode
}

// Padded pattern (Sec. 2.2 storage, read as): each row keeps its own L
// columns, widened to whole source supernodes; every node stores its rows'
// diagonal block densely together with the shared U tail.
void build_nodes(Plan& P, const SymbolicRows& F) {
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
    // L columns of row i, ascending: every source node below the row's own
    // node contributes its whole segment once (the L runs are ascending, so a
    // node already taken is the last one taken).  Called once to count, once
    // to fill.
    auto row_segments = [&](int32_t i, int32_t r, auto&& take) {
        int32_t last = -1;
        for (int64_t q = F.lrp[i]; q < F.lrp[i + 1]; ++q) {
            const int32_t a = F.lrun_first[q], b = std::min(a + F.lrun_len[q], r);
            for (int32_t k = a; k < b;) {
                const int32_t S = P.node_of[k];
                if (S != last) { take(P.sn_start[S], P.sn_start[S + 1]); last = S; }
                k = P.sn_start[S + 1];
            }
            if (b < a + F.lrun_len[q]) break;
        }
    };
    int64_t poff = 0;
    P.max_row = 0;
    for (int32_t s = 0; s < nn; ++s) {
        const int32_t r = P.sn_start[s], e = P.sn_start[s + 1] - 1, sz = e - r + 1;
        for (int64_t q = F.urp[e] + 1; q < F.urp[e + 1]; ++q) P.tcols.push_back(F.uci[q]);
        P.node_tail_off[s + 1] = (int64_t)P.tcols.size();
        const int64_t w = sz + (P.node_tail_off[s + 1] - P.node_tail_off[s]);
        P.node_panel_off[s] = poff;
        poff += w * sz;
        P.node_panel_off[s + 1] = poff;
        for (int32_t i = r; i <= e; ++i) {
            int64_t cnt = 0;
            row_segments(i, r, [&](int32_t s0, int32_t s1) { cnt += s1 - s0; });
            P.row_lptr[i + 1] = P.row_lptr[i] + cnt;
            P.max_row = std::max<int32_t>(P.max_row, (int32_t)(cnt + w));
        }
    }
    P.lcols.resize(P.row_lptr[n]);
    for (int32_t s = 0; s < nn; ++s)
        for (int32_t i = P.sn_start[s]; i < P.sn_start[s + 1]; ++i) {
            int32_t* o = P.lcols.data() + P.row_lptr[i];
            row_segments(i, P.sn_start[s], [&](int32_t s0, int32_t s1) {
                for (int32_t t = s0; t < s1; ++t) *o++ = t;
            });
        }
    P.nnz_l = (int64_t)P.lcols.size();
    P.nnz_panel = poff;
    P.nnz_store = P.nnz_l + P.nnz_panel;
    // flop counts (Sec. 2.1): one division per L(i,k) plus two per U(k, >k) entry
    // (integer terms: the unpadded total is exact, summed over L runs by prefix sums)
    double fp = 0.0;
    std::vector<int64_t> ulen(n), upre(n + 1, 0);
    for (int32_t i = 0; i < n; ++i) {
        ulen[i] = F.urp[i + 1] - F.urp[i];
        upre[i + 1] = upre[i] + 2 * ulen[i] - 1;
    }
    int64_t fu = 0;
    for (size_t q = 0; q < F.lrun_first.size(); ++q)
        fu += upre[F.lrun_first[q] + F.lrun_len[q]] - upre[F.lrun_first[q]];
    P.row_flops.assign(n, 0.0);
    P.flops_row_row = P.flops_sup_row = P.flops_sup_sup = P.flops_in_sn = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        const int32_t D = P.node_of[i];
        const bool dest_sn = P.sn_start[D + 1] - P.sn_start[D] > 1;
        double f = 0.0;
        for (int64_t t = P.row_lptr[i]; t < P.row_lptr[i + 1]; ++t) {
            const double g = 1.0 + 2.0 * (double)(ulen[P.lcols[t]] - 1);
            const int32_t S = P.node_of[P.lcols[t]];
            if (P.sn_start[S + 1] - P.sn_start[S] == 1) P.flops_row_row += g;
            else if (dest_sn) P.flops_sup_sup += g;
            else P.flops_sup_row += g;
            f += g;
        }
        for (int32_t k = P.sn_start[D]; k < i; ++k) {
            const double g = 1.0 + 2.0 * (double)(ulen[k] - 1);
            P.flops_in_sn += g;
            f += g;
        }
        P.row_flops[i] = f;
        fp += f;
    }
    P.flops_unpadded = (double)fu;
    P.flops_padded = fp;
    P.nnz_f = F.nnz_l + F.urp[n];
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
// Share of a heavy row's work that must come from sources at no more than
// half its level.  0: every row past the work cut is heavy.
constexpr double kHeavyEarlyFrac = 0.0;

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
        if (early >= kHeavyEarlyFrac * P.row_flops[i]) {
            P.heavy_rank[i] = (int32_t)P.heavy_order.size();
            P.heavy_order.push_back(i);
        }
    }
}

}  // namespace hylu

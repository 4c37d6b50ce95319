// Sequential part of the bulk-sequential substitution (HYLU Sec. 2.3,
// Fig. 3): the levels of a triangular solve that hold many rows are solved in
// bulk, one warp per row, with a level watermark between levels; a chain of
// consecutive light levels (few rows, little work) is one segment, solved
// level after level by a single thread block, with a block barrier instead of
// the watermark's hand-off between its levels.  See SeqSegments in plan.hpp.
#include <algorithm>
#include <array>
#include <vector>

#include "plan.hpp"

namespace hylu {

void build_seq_segments(const Plan& P, bool backward, int32_t max_rows, SeqSegments& S, int32_t long_min,
                        int32_t chunk_len) {
    S = SeqSegments();
    const std::vector<int32_t>& order = backward ? P.bwd_order : P.fwd_order;
    const std::vector<int32_t>& level = backward ? P.bwd_level : P.fwd_level;
    const std::vector<int32_t>& count = backward ? P.bwd_count : P.fwd_count;
    const std::vector<int32_t>& offv = backward ? P.bwd_off : P.fwd_off;
    const int32_t nn = P.nnodes;
    std::vector<int32_t> off = offv;
    if (off.empty()) off = {0, (int32_t)count.size()};
    const int32_t ni = (int32_t)off.size() - 1;
    auto inst = [&](int32_t D) { return P.node_inst.empty() ? 0 : P.node_inst[D]; };
    S.seg_off.push_back(0);
    S.lvl_row.push_back(0);
    S.lvl_node.push_back(0);
    std::vector<char> in_seg(nn, 0);
    if (max_rows > 0 && nn > 0) {
        // per level of every instance: rows, largest node, work in entries
        // (the rows' L lists or U tails, and the dense diagonal blocks)
        const size_t nl = count.size();
        std::vector<int64_t> rows(nl, 0), work(nl, 0);
        std::vector<int32_t> big(nl, 0);
        std::vector<std::vector<int32_t>> nodes_at(nl);
        for (int32_t D = 0; D < nn; ++D) {
            const size_t g = (size_t)off[inst(D)] + level[D];
            const int32_t r = P.sn_start[D], s = P.sn_start[D + 1] - r;
            rows[g] += s;
            big[g] = std::max(big[g], s);
            int64_t w = (int64_t)s * s;
            if (backward) w += (int64_t)s * (P.node_tail_off[D + 1] - P.node_tail_off[D]);
            else w += P.row_lptr[r + s] - P.row_lptr[r];
            work[g] += w;
            nodes_at[g].push_back(D);
        }
        const int64_t max_work = 1024 * (int64_t)max_rows;
        auto light = [&](size_t g) { return rows[g] <= max_rows && big[g] <= max_rows && work[g] <= max_work; };
        // maximal chains of two or more consecutive light levels, ordered by
        // first level (instances are independent): a block that claims a
        // segment then waits only on bulk rows and on segments claimed before
        std::vector<std::array<int32_t, 3>> segs;   // first level, instance, last level
        for (int32_t q = 0; q < ni; ++q) {
            const int32_t L = off[q + 1] - off[q];
            for (int32_t l0 = 0; l0 < L;) {
                if (!light((size_t)off[q] + l0)) { ++l0; continue; }
                int32_t l1 = l0;
                while (l1 + 1 < L && light((size_t)off[q] + l1 + 1)) ++l1;
                if (l1 > l0) segs.push_back({l0, q, l1});
                l0 = l1 + 1;
            }
        }
        std::sort(segs.begin(), segs.end());
        for (const auto& sg : segs) {
            const int32_t l0 = sg[0], q = sg[1], l1 = sg[2];
            S.meta.insert(S.meta.end(), {q, l0, l1});
            for (int32_t l = l0; l <= l1; ++l) {
                std::vector<int32_t>& at = nodes_at[(size_t)off[q] + l];
                std::sort(at.begin(), at.end());
                for (int32_t D : at) {
                    in_seg[D] = 1;
                    for (int32_t i = P.sn_start[D]; i < P.sn_start[D + 1]; ++i) S.rows.push_back(i);
                    if (P.sn_start[D + 1] - P.sn_start[D] > 1) S.snodes.push_back(D);
                }
                S.lvl_row.push_back((int32_t)S.rows.size());
                S.lvl_node.push_back((int32_t)S.snodes.size());
            }
            S.seg_off.push_back((int32_t)S.lvl_row.size() - 1);
        }
    }
    std::vector<int32_t> rows;
    rows.reserve(order.size());
    for (int32_t i : order)
        if (!in_seg[P.node_of[i]]) rows.push_back(i);
    // the forward solve's long rows: their L lists split into chunks of about
    // chunk_len entries (the rectangular blocks of Sec. 2.3, nonzeros spread
    // evenly over workers), each a claim entry n + c of its own that waits
    // only for the levels its entries come from; the row then adds the
    // chunks' sums in chunk order
    S.row_chunk_off.assign((size_t)P.n + 1, 0);
    if (!backward && long_min > 0) {
        // by row index, so that row_chunk_off lists every row's chunks
        std::vector<char> bulk(P.n, 0);
        for (int32_t i : rows) bulk[i] = 1;
        for (int32_t i = 0; i < P.n; ++i) {
            const int64_t l0 = P.row_lptr[i], nl = P.row_lptr[i + 1] - l0;
            if (!bulk[i] || nl < long_min) continue;
            const int64_t nc = (nl + chunk_len - 1) / chunk_len;
            for (int64_t c = 0; c < nc; ++c) {
                const int32_t a = (int32_t)(c * nl / nc), b = (int32_t)((c + 1) * nl / nc);
                int32_t lv = 0;
                for (int64_t t = l0 + a; t < l0 + b; ++t) lv = std::max(lv, level[P.node_of[P.lcols[t]]] + 1);
                S.chunk_row.push_back(i);
                S.chunk_a.push_back(a);
                S.chunk_b.push_back(b);
                S.chunk_level.push_back(lv);
            }
            S.row_chunk_off[i + 1] = (int32_t)nc;
        }
        for (int32_t i = 0; i < P.n; ++i) S.row_chunk_off[i + 1] += S.row_chunk_off[i];
    }
    // claim list: at each level, the chunks waiting for it, then the rows
    // of that level in their order (the rows' order is by level); a chunk's
    // level is at most its row's, so it comes before its row
    const int32_t nch = (int32_t)S.chunk_row.size();
    std::vector<int32_t> corder(nch);
    for (int32_t c = 0; c < nch; ++c) corder[c] = c;
    std::stable_sort(corder.begin(), corder.end(),
                     [&](int32_t x, int32_t y) { return S.chunk_level[x] < S.chunk_level[y]; });
    S.task.reserve(rows.size() + nch);
    size_t k = 0;
    for (int32_t i : rows) {
        const int32_t li = level[P.node_of[i]];
        while (k < corder.size() && S.chunk_level[corder[k]] <= li) S.task.push_back(P.n + corder[k++]);
        S.task.push_back(i);
    }
    while (k < corder.size()) S.task.push_back(P.n + corder[k++]);
}

}  // namespace hylu

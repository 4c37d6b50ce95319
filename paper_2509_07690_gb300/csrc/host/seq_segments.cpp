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

void build_seq_segments(const Plan& P, bool backward, int32_t max_rows, SeqSegments& S) {
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
    S.task.reserve(order.size());
    for (int32_t i : order)
        if (!in_seg[P.node_of[i]]) S.task.push_back(i);
}

}  // namespace hylu

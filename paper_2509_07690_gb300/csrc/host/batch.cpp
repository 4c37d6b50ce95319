// Combined plan of a batch of independent systems and value sets: the block
// diagonal of all instances, so that one persistent launch factors (and one
// solve launch sequence solves) every instance; the claim orders merge the
// instances level by level, which interleaves them and keeps every SM busy.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "plan.hpp"

namespace hylu {

namespace {

template <class T>
void append_shifted(std::vector<T>& dst, const std::vector<T>& src, size_t from, size_t to, T shift) {
    for (size_t q = from; q < to; ++q) dst.push_back(src[q] + shift);
}

// rows of all instances sorted by (level, instance, row); descending rows
// inside an instance's level when `desc`
void merge_by_level(const std::vector<const Plan*>& inst_plan, const std::vector<int32_t>& row_base,
                    const std::vector<int32_t>& node_base_of_inst,
                    const std::vector<const std::vector<int32_t>*>& node_levels, bool desc,
                    std::vector<int32_t>& order, std::vector<int32_t>& count_nodes, std::vector<int32_t>& count_rows) {
    int32_t ml = 0;
    for (size_t q = 0; q < inst_plan.size(); ++q)
        for (int32_t l : *node_levels[q]) ml = std::max(ml, l);
    count_nodes.assign(ml + 1, 0);
    count_rows.assign(ml + 1, 0);
    std::vector<int64_t> start(ml + 2, 0);
    for (size_t q = 0; q < inst_plan.size(); ++q) {
        const Plan& P = *inst_plan[q];
        for (int32_t D = 0; D < P.nnodes; ++D) {
            const int32_t l = (*node_levels[q])[D];
            count_nodes[l]++;
            const int32_t rows = P.sn_start[D + 1] - P.sn_start[D];
            count_rows[l] += rows;
            start[l + 1] += rows;
        }
    }
    for (int32_t l = 0; l <= ml; ++l) start[l + 1] += start[l];
    int64_t total = start[ml + 1];
    order.assign(total, 0);
    for (size_t q = 0; q < inst_plan.size(); ++q) {
        const Plan& P = *inst_plan[q];
        if (!desc) {
            for (int32_t i = 0; i < P.n; ++i) order[start[(*node_levels[q])[P.node_of[i]]]++] = i + row_base[q];
        } else {
            for (int32_t i = P.n - 1; i >= 0; --i) order[start[(*node_levels[q])[P.node_of[i]]]++] = i + row_base[q];
        }
    }
    (void)node_base_of_inst;
}

}  // namespace

int combine(const std::vector<const Plan*>& sys, int32_t nsets, Plan& C, BatchLayout& B) {
    const int32_t k = (int32_t)sys.size();
    B.k = k;
    B.nsets = nsets;
    std::vector<const Plan*> inst;
    for (int32_t v = 0; v < nsets; ++v)
        for (int32_t s = 0; s < k; ++s) inst.push_back(sys[s]);
    const size_t Q = inst.size();
    B.row_base.assign(Q, 0);
    B.val_base.assign(Q, 0);
    std::vector<int32_t> nbase(Q, 0);
    int64_t rows = 0, vals = 0, nodes = 0;
    B.pos_n = 0;
    for (size_t q = 0; q < Q; ++q) {
        B.row_base[q] = (int32_t)rows;
        B.val_base[q] = vals;
        nbase[q] = (int32_t)nodes;
        rows += inst[q]->n;
        vals += inst[q]->nnz_a;
        nodes += inst[q]->nnodes;
        B.pos_n = std::max(B.pos_n, inst[q]->n);
    }
    if (rows > INT32_MAX - 1) return -4;
    C = Plan();
    C.n = (int32_t)rows;
    C.nnz_a = vals;
    C.nnodes = (int32_t)nodes;
    C.a_rp.push_back(0);
    C.ah_rp.push_back(0);
    C.sn_start.clear();
    C.row_lptr.push_back(0);
    C.node_tail_off.push_back(0);
    C.node_panel_off.clear();
    B.node_base.clear();
    int64_t l_off = 0, t_off = 0, p_off = 0, ah_off = 0, a_off = 0;
    for (size_t q = 0; q < Q; ++q) {
        const Plan& P = *inst[q];
        const int32_t rb = B.row_base[q];
        const int64_t vb = B.val_base[q];
        append_shifted<int64_t>(C.a_rp, P.a_rp, 1, P.a_rp.size(), a_off);
        append_shifted<int32_t>(C.a_ci, P.a_ci, 0, P.a_ci.size(), rb);
        append_shifted<int32_t>(C.rowperm, P.rowperm, 0, P.rowperm.size(), rb);
        append_shifted<int32_t>(C.colperm, P.colperm, 0, P.colperm.size(), rb);
        C.dr.insert(C.dr.end(), P.dr.begin(), P.dr.end());
        C.dc.insert(C.dc.end(), P.dc.begin(), P.dc.end());
        append_shifted<int64_t>(C.ah_rp, P.ah_rp, 1, P.ah_rp.size(), ah_off);
        C.ah_slot.insert(C.ah_slot.end(), P.ah_slot.begin(), P.ah_slot.end());
        append_shifted<int64_t>(C.ah_src, P.ah_src, 0, P.ah_src.size(), vb);
        C.ah_scale.insert(C.ah_scale.end(), P.ah_scale.begin(), P.ah_scale.end());
        append_shifted<int32_t>(C.sn_start, P.sn_start, 0, P.sn_start.size() - 1, rb);
        append_shifted<int32_t>(C.node_of, P.node_of, 0, P.node_of.size(), nbase[q]);
        for (int32_t D = 0; D < P.nnodes; ++D) B.node_base.push_back(rb);
        append_shifted<int64_t>(C.row_lptr, P.row_lptr, 1, P.row_lptr.size(), l_off);
        append_shifted<int32_t>(C.lcols, P.lcols, 0, P.lcols.size(), rb);
        append_shifted<int64_t>(C.node_tail_off, P.node_tail_off, 1, P.node_tail_off.size(), t_off);
        append_shifted<int32_t>(C.tcols, P.tcols, 0, P.tcols.size(), rb);
        append_shifted<int64_t>(C.node_panel_off, P.node_panel_off, 0, P.node_panel_off.size() - 1, p_off);
        C.row_flops.insert(C.row_flops.end(), P.row_flops.begin(), P.row_flops.end());
        a_off += P.a_rp.back();
        ah_off += P.ah_rp.back();
        l_off += P.row_lptr.back();
        t_off += P.node_tail_off.back();
        p_off += P.node_panel_off.back();
        C.nnz_l += P.nnz_l;
        C.nnz_panel += P.nnz_panel;
        C.nnz_store += P.nnz_store;
        C.nnz_f += P.nnz_f;
        C.flops_unpadded += P.flops_unpadded;
        C.flops_padded += P.flops_padded;
        C.flops_row_row += P.flops_row_row;
        C.flops_sup_row += P.flops_sup_row;
        C.flops_sup_sup += P.flops_sup_sup;
        C.flops_in_sn += P.flops_in_sn;
        C.ordering = (q == 0 || C.ordering == P.ordering) ? P.ordering : HYLU_ORDER_AUTO;   // AUTO: mixed
        C.max_sn = std::max(C.max_sn, P.max_sn);
        C.max_row = std::max(C.max_row, P.max_row);
        C.analyze_ms += P.analyze_ms;
        for (int ph = 0; ph < 4; ++ph) C.analyze_phase_ms[ph] += P.analyze_phase_ms[ph];
    }
    C.sn_start.push_back(C.n);
    C.node_panel_off.push_back(p_off);
    // claim orders, merged level by level across instances: rows keep their
    // instance's levels; tail tasks (entry C.n + t) come first inside a level
    {
        int32_t ml = 0;
        for (size_t q = 0; q < Q; ++q) ml = std::max(ml, inst[q]->row_levels);
        C.node_ntask.clear();
        C.task_node.clear();
        C.task_chunk.clear();
        C.task_level.clear();
        for (size_t q = 0; q < Q; ++q) {
            const Plan& P = *inst[q];
            C.node_ntask.insert(C.node_ntask.end(), P.node_ntask.begin(), P.node_ntask.end());
            append_shifted<int32_t>(C.task_node, P.task_node, 0, P.task_node.size(), nbase[q]);
            C.task_chunk.insert(C.task_chunk.end(), P.task_chunk.begin(), P.task_chunk.end());
            C.task_level.insert(C.task_level.end(), P.task_level.begin(), P.task_level.end());
        }
        C.n_tasks = (int32_t)C.task_node.size();
        std::vector<int64_t> start(ml + 2, 0);
        for (int32_t t = 0; t < C.n_tasks; ++t) start[C.task_level[t] + 1]++;
        for (size_t q = 0; q < Q; ++q)
            for (int32_t i = 0; i < inst[q]->n; ++i) start[inst[q]->row_level[i] + 1]++;
        for (int32_t l = 0; l <= ml; ++l) start[l + 1] += start[l];
        C.row_order.assign((size_t)C.n + C.n_tasks, 0);
        C.row_level.assign(C.n, 0);
        for (int32_t t = 0; t < C.n_tasks; ++t) C.row_order[start[C.task_level[t]]++] = C.n + t;
        for (size_t q = 0; q < Q; ++q)
            for (int32_t i = 0; i < inst[q]->n; ++i) {
                const int32_t l = inst[q]->row_level[i];
                C.row_order[start[l]++] = i + B.row_base[q];
                C.row_level[i + B.row_base[q]] = l;
            }
        C.row_levels = ml;
    }
    std::vector<int32_t> rows_per_level;
    std::vector<const std::vector<int32_t>*> lv(Q);
    for (size_t q = 0; q < Q; ++q) lv[q] = &inst[q]->fwd_level;
    merge_by_level(inst, B.row_base, nbase, lv, false, C.fwd_order, C.fwd_count, rows_per_level);
    for (size_t q = 0; q < Q; ++q) lv[q] = &inst[q]->bwd_level;
    merge_by_level(inst, B.row_base, nbase, lv, true, C.bwd_order, C.bwd_count, rows_per_level);
    std::vector<int32_t> nodes_per_level;
    for (size_t q = 0; q < Q; ++q) lv[q] = &inst[q]->ut_level;
    merge_by_level(inst, B.row_base, nbase, lv, false, C.ut_order, nodes_per_level, C.ut_count);
    for (size_t q = 0; q < Q; ++q) lv[q] = &inst[q]->lt_level;
    merge_by_level(inst, B.row_base, nbase, lv, true, C.lt_order, nodes_per_level, C.lt_count);
    // per-instance level counts (each instance has its own watermark)
    auto slices = [&](std::vector<int32_t> Plan::*cnt, std::vector<int32_t>& out, std::vector<int32_t>& off) {
        out.clear();
        off.assign(1, 0);
        for (size_t q = 0; q < Q; ++q) {
            const std::vector<int32_t>& c = inst[q]->*cnt;
            out.insert(out.end(), c.begin(), c.end());
            off.push_back((int32_t)out.size());
        }
    };
    slices(&Plan::fwd_count, C.fwd_count, C.fwd_off);
    slices(&Plan::bwd_count, C.bwd_count, C.bwd_off);
    slices(&Plan::ut_count, C.ut_count, C.ut_off);
    slices(&Plan::lt_count, C.lt_count, C.lt_off);
    C.node_inst.clear();
    for (size_t q = 0; q < Q; ++q) C.node_inst.insert(C.node_inst.end(), inst[q]->nnodes, (int32_t)q);
    for (size_t q = 0; q < Q; ++q) {
        C.fwd_level.insert(C.fwd_level.end(), inst[q]->fwd_level.begin(), inst[q]->fwd_level.end());
        C.bwd_level.insert(C.bwd_level.end(), inst[q]->bwd_level.begin(), inst[q]->bwd_level.end());
        C.ut_level.insert(C.ut_level.end(), inst[q]->ut_level.begin(), inst[q]->ut_level.end());
        C.lt_level.insert(C.lt_level.end(), inst[q]->lt_level.begin(), inst[q]->lt_level.end());
    }
    return 0;
}

}  // namespace hylu

// analyze(): the preprocessing phase of HYLU (Sec. 2.1) end to end.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <exception>
#include <numeric>
#include <thread>

#include "plan.hpp"
#include "../../../include/hylu.h"

namespace hylu {

static int validate(int32_t n, const int64_t* rp, const int32_t* ci) {
    if (n < 0 || rp[0] != 0) return HYLU_ERR_PATTERN;
    for (int32_t i = 0; i < n; ++i) {
        if (rp[i + 1] < rp[i]) return HYLU_ERR_PATTERN;
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
            if (ci[q] < 0 || ci[q] >= n) return HYLU_ERR_PATTERN;
            if (q > rp[i] && ci[q] <= ci[q - 1]) return HYLU_ERR_PATTERN;
        }
    }
    return 0;
}

// Estimated factorization time of a plan on one GB300, for choosing between
// orderings (Sec. 2.1: the kernels and, here, the ordering are chosen from the
// flop count and the structure the symbolic factorization yields): the larger
// of the flops at the measured FP64 rate (1.06e12 flop/s) and the dependency
// chain at the measured cost of one level along it (about 21 us: 182 ms for
// the 8,676-level chain of the circuit workload under AMD).
static double estimated_seconds(const Plan& P) {
    return std::max(P.flops_unpadded / 1.06e12, (double)P.row_levels * 21e-6);
}

int analyze(int32_t n, const int64_t* rp, const int32_t* ci, const double* v,
            const int32_t* user_perm, const AnalyzeOptions& opt, Plan& P) {
    if (opt.ordering == HYLU_ORDER_AUTO) {
        // both fill-reducing orderings, then the plan with the lower estimate
        // (AMD on a tie)
        const auto w0 = std::chrono::steady_clock::now();
        AnalyzeOptions oa = opt, ob = opt;
        oa.ordering = HYLU_ORDER_AMD;
        ob.ordering = HYLU_ORDER_ND;
        Plan pa, pb;
        // the two analyses share no state: nested dissection on a second thread
        int rb = 0;
        std::exception_ptr eb;
        std::thread t([&] {
            try { rb = analyze(n, rp, ci, v, user_perm, ob, pb); } catch (...) { eb = std::current_exception(); }
        });
        int rc = 0;
        try { rc = analyze(n, rp, ci, v, user_perm, oa, pa); } catch (...) { t.join(); throw; }
        t.join();
        if (eb) std::rethrow_exception(eb);
        if (rc) return rc;
        if (rb) return rb;
        P = estimated_seconds(pb) < estimated_seconds(pa) ? std::move(pb) : std::move(pa);
        P.analyze_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
        return 0;
    }
    auto t0 = std::chrono::steady_clock::now();
    auto since = [](std::chrono::steady_clock::time_point a) {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - a).count();
    };
    int st = validate(n, rp, ci);
    if (st) return st;
    P.n = n;
    P.nnz_a = rp[n];
    P.a_rp.assign(rp, rp + n + 1);
    P.a_ci.assign(ci, ci + rp[n]);
    // ---- static pivoting and scaling (maximum-product matching)
    std::vector<int32_t> match(n);
    std::vector<double> dr(n, 1.0), dc(n, 1.0);
    if (opt.static_pivot) {
        if (!v) return HYLU_ERR_ARG;
        for (int64_t q = 0; q < rp[n]; ++q)          // the matching weighs finite magnitudes only
            if (!std::isfinite(v[q])) return HYLU_ERR_ARG;
        if (!max_product_matching(n, rp, ci, v, match, dr, dc)) return HYLU_ERR_STRUCT_SINGULAR;
        if (!opt.scale) { std::fill(dr.begin(), dr.end(), 1.0); std::fill(dc.begin(), dc.end(), 1.0); }
    } else {
        std::iota(match.begin(), match.end(), 0);
    }
    // row of A that lands on row j of M*A: the row matched to column j
    std::vector<int32_t> mrow(n);
    for (int32_t i = 0; i < n; ++i) mrow[match[i]] = i;
    P.analyze_phase_ms[0] = since(t0);
    const auto t_order = std::chrono::steady_clock::now();
    // pattern of B = M*A (rows permuted), for the ordering
    std::vector<int64_t> brp(n + 1, 0);
    std::vector<int32_t> bci(rp[n]);
    for (int32_t j = 0; j < n; ++j) brp[j + 1] = brp[j] + (rp[mrow[j] + 1] - rp[mrow[j]]);
    for (int32_t j = 0; j < n; ++j)
        std::copy(ci + rp[mrow[j]], ci + rp[mrow[j] + 1], bci.begin() + brp[j]);
    // ---- fill-reducing ordering on B + B^T
    std::vector<int32_t> q(n);
    if (opt.ordering == 3) {
        if (!user_perm) return HYLU_ERR_ARG;
        std::vector<char> seen(n, 0);
        for (int32_t k = 0; k < n; ++k) {
            if (user_perm[k] < 0 || user_perm[k] >= n || seen[user_perm[k]]) return HYLU_ERR_ARG;
            seen[user_perm[k]] = 1;
            q[k] = user_perm[k];
        }
    } else if (opt.ordering == 2) {
        std::iota(q.begin(), q.end(), 0);
    } else {
        CsrPattern g = symmetrize(n, brp.data(), bci.data());
        if (opt.ordering == 1) nd_order(g, q, opt.nd_leaf, opt.amd_dense); else amd_order(g, q, opt.amd_dense);
    }
    P.analyze_phase_ms[1] = since(t_order);
    const auto t_sym = std::chrono::steady_clock::now();
    P.ordering = (opt.ordering >= 0 && opt.ordering <= 3) ? opt.ordering : HYLU_ORDER_AMD;
    P.rowperm.resize(n); P.colperm.resize(n);
    for (int32_t k = 0; k < n; ++k) { P.colperm[k] = q[k]; P.rowperm[k] = mrow[q[k]]; }
    P.dr = dr; P.dc = dc;
    std::vector<int32_t> qinv(n);
    for (int32_t k = 0; k < n; ++k) qinv[q[k]] = k;
    // ---- Ahat pattern (sorted rows) with source indices
    CsrPattern ah;
    ah.n = n;
    ah.rp.assign(n + 1, 0);
    ah.ci.resize(rp[n]);
    std::vector<int64_t> src(rp[n]);
    {
        std::vector<std::pair<int32_t, int64_t>> row;
        int64_t pos = 0;
        for (int32_t i = 0; i < n; ++i) {
            int32_t r = P.rowperm[i];
            row.clear();
            for (int64_t t = rp[r]; t < rp[r + 1]; ++t) row.push_back({qinv[ci[t]], t});
            std::sort(row.begin(), row.end());
            for (auto& pr : row) { ah.ci[pos] = pr.first; src[pos] = pr.second; ++pos; }
            ah.rp[i + 1] = pos;
        }
    }
    // ---- symbolic factorization, supernodes, padded nodes
    SymbolicRows F;
    symbolic_rows(ah, F);
    supernode_partition(n, F, std::max(1, opt.sn_max), P.sn_start);
    build_nodes(P, F);
    split_heavy_rows(P, opt.heavy_ratio);
    P.analyze_phase_ms[2] = since(t_sym);
    const auto t_map = std::chrono::steady_clock::now();
    // ---- Ahat entries -> slots of their row: [0, nL) the L list, then the
    //      node's block (s slots) and tail
    P.ah_rp = ah.rp;
    P.ah_slot.resize(rp[n]);
    P.ah_src = src;
    P.ah_scale.resize(rp[n]);
    for (int32_t i = 0; i < n; ++i) {
        int32_t nd = P.node_of[i];
        int32_t r = P.sn_start[nd], e = P.sn_start[nd + 1] - 1;
        const int32_t* l0 = P.lcols.data() + P.row_lptr[i];
        const int32_t* l1 = P.lcols.data() + P.row_lptr[i + 1];
        const int32_t* t0 = P.tcols.data() + P.node_tail_off[nd];
        const int32_t* t1 = P.tcols.data() + P.node_tail_off[nd + 1];
        int32_t nl = (int32_t)(l1 - l0), sz = e - r + 1;
        int32_t orow = P.rowperm[i];
        for (int64_t t = ah.rp[i]; t < ah.rp[i + 1]; ++t) {
            int32_t c = ah.ci[t], slot;
            if (c < r) {
                const int32_t* f = std::lower_bound(l0, l1, c);
                if (f == l1 || *f != c) return HYLU_ERR_INTERNAL;
                slot = (int32_t)(f - l0);
            } else if (c <= e) {
                slot = nl + (c - r);
            } else {
                const int32_t* f = std::lower_bound(t0, t1, c);
                if (f == t1 || *f != c) return HYLU_ERR_INTERNAL;
                slot = nl + sz + (int32_t)(f - t0);
            }
            P.ah_slot[t] = slot;
            P.ah_scale[t] = dr[orow] * dc[ci[src[t]]];
        }
    }
    P.max_sn = 1;
    for (int32_t s = 0; s < P.nnodes; ++s) P.max_sn = std::max(P.max_sn, P.sn_start[s + 1] - P.sn_start[s]);
    P.analyze_phase_ms[3] = since(t_map);
    P.analyze_ms = since(t0);
    return 0;
}

}  // namespace hylu

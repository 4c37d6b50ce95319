// Checkpoint of an analysis: the Plan of a handle (preprocessing outputs,
// symbolic pattern, supernodes, task and substitution schedules), its batch
// layout and its options, written to and read from a flat byte image.
//
// Layout (native little-endian, which both supported hosts use):
//   "HYLUPLAN" | u32 version | u32 byte-order marker 0x01020304 |
//   fields in the order of visit() below: a scalar as its raw bytes, a vector
//   as u64 element count then the elements |
//   u64 FNV-1a 64 checksum of every byte before it.
// Save and load run the same visit(), so every field written is read back in
// the same place.  A loaded plan is checked for consistent sizes and index
// ranges before it can reach the device.
#include <cstring>
#include <type_traits>

#include "plan.hpp"
#include "../../../include/hylu.h"

namespace hylu {

namespace {

constexpr char kMagic[8] = {'H', 'Y', 'L', 'U', 'P', 'L', 'A', 'N'};
constexpr uint32_t kVersion = 3;
constexpr uint32_t kOrder = 0x01020304u;

uint64_t fnv1a(const uint8_t* p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) { h ^= p[i]; h *= 1099511628211ull; }
    return h;
}

struct Writer {
    std::vector<uint8_t>& out;
    void raw(const void* p, size_t n) {
        const uint8_t* b = static_cast<const uint8_t*>(p);
        out.insert(out.end(), b, b + n);
    }
    template <class T> bool operator()(T& x) {
        static_assert(std::is_trivially_copyable<T>::value, "scalar fields only");
        raw(&x, sizeof(T));
        return true;
    }
    template <class T> bool operator()(std::vector<T>& v) {
        uint64_t c = v.size();
        raw(&c, sizeof(c));
        if (c) raw(v.data(), sizeof(T) * c);
        return true;
    }
};

struct Reader {
    const uint8_t* p;
    size_t left;
    bool take(void* dst, size_t n) {
        if (n > left) return false;
        std::memcpy(dst, p, n);
        p += n;
        left -= n;
        return true;
    }
    template <class T> bool operator()(T& x) { return take(&x, sizeof(T)); }
    template <class T> bool operator()(std::vector<T>& v) {
        uint64_t c = 0;
        if (!take(&c, sizeof(c)) || c > left / sizeof(T)) return false;
        v.resize(c);
        return c == 0 || take(v.data(), sizeof(T) * c);
    }
};

// Every field of the image, in order.  Returns false when a read runs past
// the end of the buffer.
template <class V>
bool visit(V& f, Plan& P, BatchLayout& B, int32_t& batch, hylu_options& o) {
    bool ok = true;
    // options the handle was analysed with (field by field: no padding bytes)
    ok = ok && f(o.ordering) && f(o.static_pivot) && f(o.scale) && f(o.sn_max) && f(o.nd_leaf);
    ok = ok && f(o.pivot_tau) && f(o.refine_tol) && f(o.refine_maxit) && f(o.refine) && f(o.spin_limit);
    ok = ok && f(o.rows_per_task) && f(o.debug) && f(o.amd_dense) && f(o.timing) && f(o.precision);
    ok = ok && f(o.heavy_ratio) && f(o.gemm_min_rows) && f(o.solve_seq_rows);
    // plan scalars
    ok = ok && f(P.n) && f(P.nnz_a) && f(P.nnodes) && f(P.nnz_l) && f(P.nnz_panel) && f(P.nnz_store);
    ok = ok && f(P.nnz_f) && f(P.flops_unpadded) && f(P.flops_padded) && f(P.n_tasks) && f(P.row_levels);
    ok = ok && f(P.flops_row_row) && f(P.flops_sup_row) && f(P.flops_sup_sup) && f(P.flops_in_sn);
    ok = ok && f(P.ordering) && f(P.max_row) && f(P.max_sn) && f(P.analyze_ms) && f(P.analyze_phase_ms);
    // pattern of A, preprocessing, Ahat scatter
    ok = ok && f(P.a_rp) && f(P.a_ci) && f(P.rowperm) && f(P.colperm) && f(P.dr) && f(P.dc);
    ok = ok && f(P.ah_rp) && f(P.ah_slot) && f(P.ah_src) && f(P.ah_scale);
    // nodes and factor storage
    ok = ok && f(P.sn_start) && f(P.node_of) && f(P.row_lptr) && f(P.lcols) && f(P.node_tail_off);
    ok = ok && f(P.tcols) && f(P.node_panel_off) && f(P.row_flops);
    // factor kernel schedule
    ok = ok && f(P.node_ntask) && f(P.task_node) && f(P.task_chunk) && f(P.task_level) && f(P.row_order);
    ok = ok && f(P.heavy_order) && f(P.heavy_rank) && f(P.row_level);
    // substitution schedules
    ok = ok && f(P.fwd_order) && f(P.bwd_order) && f(P.fwd_level) && f(P.bwd_level) && f(P.fwd_count);
    ok = ok && f(P.bwd_count) && f(P.ut_order) && f(P.lt_order) && f(P.ut_level) && f(P.lt_level);
    ok = ok && f(P.ut_count) && f(P.lt_count);
    ok = ok && f(P.node_inst) && f(P.fwd_off) && f(P.bwd_off) && f(P.ut_off) && f(P.lt_off);
    // batch layout
    ok = ok && f(batch) && f(B.k) && f(B.nsets) && f(B.pos_n) && f(B.row_base) && f(B.node_base);
    ok = ok && f(B.val_base);
    return ok;
}

template <class T>
bool in_range(const std::vector<T>& v, int64_t lo, int64_t hi) {   // every entry in [lo, hi)
    for (const T& x : v)
        if ((int64_t)x < lo || (int64_t)x >= hi) return false;
    return true;
}

template <class T>
bool ascending_from_zero(const std::vector<T>& v, size_t size) {    // offsets: v[0] = 0, nondecreasing
    if (v.size() != size || v.empty() || v[0] != 0) return false;
    for (size_t i = 1; i < v.size(); ++i)
        if (v[i] < v[i - 1]) return false;
    return true;
}

// Sizes and index ranges the kernels rely on.
bool consistent(const Plan& P, const BatchLayout& B, int32_t batch) {
    const int64_t n = P.n, nn = P.nnodes, nt = P.n_tasks;
    if (n < 0 || nn < 0 || nt < 0 || nn > n) return false;
    if (!ascending_from_zero(P.a_rp, n + 1) || P.a_rp[n] != P.nnz_a) return false;
    if ((int64_t)P.a_ci.size() != P.nnz_a || !in_range(P.a_ci, 0, n)) return false;
    if ((int64_t)P.rowperm.size() != n || (int64_t)P.colperm.size() != n) return false;
    if (!in_range(P.rowperm, 0, n) || !in_range(P.colperm, 0, n)) return false;
    if ((int64_t)P.dr.size() != n || (int64_t)P.dc.size() != n) return false;
    if (!ascending_from_zero(P.ah_rp, n + 1) || P.ah_rp[n] != P.nnz_a) return false;
    if ((int64_t)P.ah_slot.size() != P.nnz_a || (int64_t)P.ah_src.size() != P.nnz_a) return false;
    if ((int64_t)P.ah_scale.size() != P.nnz_a || !in_range(P.ah_src, 0, INT64_MAX)) return false;
    if (!in_range(P.ah_slot, 0, (int64_t)P.max_row)) return false;
    if (!ascending_from_zero(P.sn_start, nn + 1) || P.sn_start[nn] != n) return false;
    if ((int64_t)P.node_of.size() != n || !in_range(P.node_of, 0, nn)) return false;
    if (!ascending_from_zero(P.row_lptr, n + 1) || P.row_lptr[n] != P.nnz_l) return false;
    if ((int64_t)P.lcols.size() != P.nnz_l || !in_range(P.lcols, 0, n)) return false;
    if (!ascending_from_zero(P.node_tail_off, nn + 1)) return false;
    if ((int64_t)P.tcols.size() != P.node_tail_off[nn] || !in_range(P.tcols, 0, n)) return false;
    if (!ascending_from_zero(P.node_panel_off, nn + 1) || P.node_panel_off[nn] != P.nnz_panel) return false;
    if ((int64_t)P.node_ntask.size() != nn) return false;
    if ((int64_t)P.task_node.size() != nt || !in_range(P.task_node, 0, nn)) return false;
    if ((int64_t)P.task_chunk.size() != nt || (int64_t)P.task_level.size() != nt) return false;
    if ((int64_t)P.row_order.size() != n + nt || !in_range(P.row_order, 0, n + nt)) return false;
    if (!in_range(P.heavy_order, 0, n) || (int64_t)P.row_level.size() != n) return false;
    if (!P.heavy_rank.empty() && (int64_t)P.heavy_rank.size() != n) return false;
    for (const std::vector<int32_t>* o : {&P.fwd_order, &P.bwd_order, &P.ut_order, &P.lt_order})
        if ((int64_t)o->size() != n || !in_range(*o, 0, n)) return false;
    for (const std::vector<int32_t>* l : {&P.fwd_level, &P.bwd_level, &P.ut_level, &P.lt_level})
        if ((int64_t)l->size() != nn || !in_range(*l, 0, n + 1)) return false;
    if (!P.node_inst.empty() && (int64_t)P.node_inst.size() != nn) return false;
    if (batch) {
        const int64_t q = (int64_t)B.k * B.nsets;
        if (B.k < 1 || B.nsets < 1 || (int64_t)B.row_base.size() != q || (int64_t)B.val_base.size() != q)
            return false;
        if ((int64_t)B.node_base.size() != nn || !in_range(B.row_base, 0, n) || !in_range(B.node_base, 0, n))
            return false;
        if (B.pos_n < 1 || B.pos_n > n) return false;
    }
    return true;
}

}  // namespace

int save_plan(const Plan& P, const BatchLayout& B, bool batch, const hylu_options& opt,
              std::vector<uint8_t>& out) {
    out.clear();
    out.insert(out.end(), kMagic, kMagic + sizeof(kMagic));
    Writer w{out};
    uint32_t ver = kVersion, ord = kOrder;
    w(ver);
    w(ord);
    // visit() takes mutable references for the reader's sake; the writer only reads them
    Plan& p = const_cast<Plan&>(P);
    BatchLayout& b = const_cast<BatchLayout&>(B);
    int32_t bt = batch ? 1 : 0;
    hylu_options o = opt;
    visit(w, p, b, bt, o);
    uint64_t h = fnv1a(out.data(), out.size());
    w(h);
    return HYLU_OK;
}

int load_plan(const uint8_t* buf, size_t bytes, Plan& P, BatchLayout& B, bool& batch, hylu_options& opt) {
    if (bytes < sizeof(kMagic) + 8 + 8 || std::memcmp(buf, kMagic, sizeof(kMagic)) != 0) return HYLU_ERR_PATTERN;
    uint64_t stored;
    std::memcpy(&stored, buf + bytes - 8, 8);
    if (fnv1a(buf, bytes - 8) != stored) return HYLU_ERR_PATTERN;
    Reader r{buf + sizeof(kMagic), bytes - sizeof(kMagic) - 8};
    uint32_t ver = 0, ord = 0;
    if (!r(ver) || !r(ord) || ver != kVersion || ord != kOrder) return HYLU_ERR_PATTERN;
    int32_t bt = 0;
    if (!visit(r, P, B, bt, opt) || r.left != 0) return HYLU_ERR_PATTERN;
    batch = bt != 0;
    if (!consistent(P, B, bt)) return HYLU_ERR_PATTERN;
    return HYLU_OK;
}

}  // namespace hylu

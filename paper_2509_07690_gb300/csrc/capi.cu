// C ABI of the library (declared in include/hylu.h): handle lifetime, plan
// upload, the factorization / substitution / refinement drivers.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <map>
#include <vector>

#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define HYLU_HAVE_NVTX 1
#endif
#endif

#include "../../include/hylu.h"
#include "host/plan.hpp"
#include "kernels.cuh"

struct hylu_handle {
    hylu::Plan P;
    hylu_options opt;
    int device = -1;
    bool uploaded = false;
    bool factored = false;
    hylu::DevPlan dp{};
    std::vector<void*> allocs;
    // original A (for the residual) and preprocessing outputs on the device
    double* d_avals = nullptr;
    int64_t* d_arp = nullptr;
    int32_t* d_aci = nullptr;
    int32_t *d_rowperm = nullptr, *d_colperm = nullptr;
    double *d_dr = nullptr, *d_dc = nullptr;
    // solve workspace (n * cap_rhs each)
    int cap_rhs = 0;
    size_t cap_elems = 0;
    double *d_z = nullptr, *d_xh = nullptr, *d_r = nullptr, *d_d = nullptr, *d_norms = nullptr;
    double* d_colsum = nullptr;
    double* h_norms = nullptr;   // pinned
    int32_t* h_status = nullptr; // pinned
    int grid = 0;                        // blocks of the factor launch
    int solve_grid = 0;                  // blocks of the substitution launches
    int tuned = 0;                       // hylu_tune ran: tuned_* below are its choice
    bool heavy_off = false;              // the tuner found the heavy-row queue slower
    cudaStream_t last = nullptr;
    int32_t nperturb = 0, refine_iters = 0, device_status = 0, failed_node = -1;
    double backward_error = -1.0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // batched form
    bool batch = false;
    hylu::BatchLayout layout;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int64_t graph_launches = 0;          // kernel launches recorded into the graph
    int graph_corrections = 0;           // refinement steps recorded after the graph's solve
    double gemm_flops = 0.0;             // useful flops of the tensor-core sup-sup tasks
    int graph_nrhs = 0;
    bool graph_norms_pending = false;    // a replay wrote residual norms not yet read
    int grid_max = 0;
    bool timed_factor = false, timed_solve = false;
    // device tables of the bulk-sequential substitution, per solve_seq_rows
    // value built so far (the tuner tries several)
    struct SeqTables {
        const int32_t *fwd_task, *bwd_task;
        int32_t n_fwd_tasks, n_bwd_tasks, seq_blocks;
        hylu::SegTable fseg, bseg;
        const int32_t *fch_row, *fch_a, *fch_b, *fch_level, *frow_chunk_off;
        double* fch_part;
        int32_t* fch_flag;
    };
    std::map<int, SeqTables> seq_tables;
};

namespace {

template <class T>
int dalloc(hylu_handle* h, T** p, size_t count) {
    void* q = nullptr;
    if (cudaMalloc(&q, sizeof(T) * (count ? count : 1)) != cudaSuccess) return HYLU_ERR_NOMEM;
    h->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return HYLU_OK;
}

template <class T>
int upload(hylu_handle* h, T** p, const std::vector<T>& v, cudaStream_t st) {
    int rc = dalloc(h, p, v.size());
    if (rc) return rc;
    if (!v.empty() && cudaMemcpyAsync(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return HYLU_ERR_CUDA;
    return HYLU_OK;
}

#define TRY(x) do { int rc_ = (x); if (rc_ < 0) return rc_; } while (0)

// NVTX range around an entry point or a refinement step, for timeline tools
// (nsys, ncu --nvtx); without an attached tool the calls do nothing, and a
// toolkit without the NVTX headers builds the ranges as no-ops.
struct Range {
#ifdef HYLU_HAVE_NVTX
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
#else
    explicit Range(const char*) {}
#endif
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

// No C++ exception crosses the C ABI: host allocation failures become
// HYLU_ERR_NOMEM, anything else HYLU_ERR_INTERNAL.
template <class F>
int guarded(F&& f) {
    try {
        return f();
    } catch (const std::bad_alloc&) {
        return HYLU_ERR_NOMEM;
    } catch (...) {
        return HYLU_ERR_INTERNAL;
    }
}

// Precision form: the tables of the tensor-core sup-sup update (GemmPlan),
// the split multiplier blocks and their TMA tensor maps.  Off (n_gd = 0) for
// FP64 factors, gemm_min_rows = 0, when no pair qualifies, or without the
// driver's tensor-map encoder.
int upload_gemm(hylu_handle* h, cudaStream_t st) {
    hylu::DevPlan& d = h->dp;
    d.n_gd = d.n_gtask = d.n_diag = d.gemm_blocks = d.n_pair = 0;
    d.a_elems = 0;
    d.a_term[0] = d.a_term[1] = d.a_term[2] = nullptr;
    d.tmaps = nullptr;
    if (h->opt.precision != 1 || h->opt.gemm_min_rows <= 0) return HYLU_OK;
    if (!hylu::tensor_maps_available() || !hylu::gemm_smem_fits()) return HYLU_OK;
    const int tc_blocks = hylu::tc_grid(h->device);
    if (tc_blocks < 1) return HYLU_OK;
    hylu::GemmPlan G;
    if (hylu::build_gemm_plan(h->P, h->opt.gemm_min_rows, G) != 0) return HYLU_ERR_INTERNAL;
    if (G.ngd == 0 || G.task_pair.empty()) return HYLU_OK;
    int32_t *gon, *gn, *gkp, *gnt, *pg, *ps, *pu, *pj, *pn, *pnd, *xm, *gs, *tp, *tm, *tj, *dr, *ro;
    int64_t *gao, *pxo;
    TRY(upload(h, &gon, G.gd_of_node, st));
    TRY(upload(h, &gn, G.gd_node, st));
    TRY(upload(h, &gkp, G.gd_Kp, st));
    TRY(upload(h, &gao, G.gd_a_off, st));
    TRY(upload(h, &gnt, G.gd_ntask, st));
    TRY(upload(h, &pg, G.pair_gd, st));
    TRY(upload(h, &ps, G.pair_src, st));
    TRY(upload(h, &pu, G.pair_u0, st));
    TRY(upload(h, &pj, G.pair_jr, st));
    TRY(upload(h, &pn, G.pair_nj, st));
    TRY(upload(h, &pnd, G.pair_need, st));
    TRY(upload(h, &pxo, G.pair_x_off, st));
    TRY(upload(h, &xm, G.xmap, st));
    TRY(upload(h, &gs, G.gd_slot, st));
    TRY(upload(h, &tp, G.task_pair, st));
    TRY(upload(h, &tm, G.task_mt, st));
    TRY(upload(h, &tj, G.task_jt, st));
    TRY(upload(h, &dr, G.diag_row, st));
    TRY(upload(h, &ro, G.row_order, st));
    d.gd_of_node = gon; d.gd_node = gn; d.gd_Kp = gkp; d.gd_a_off = gao; d.gd_ntask = gnt;
    d.pair_gd = pg; d.pair_src = ps; d.pair_u0 = pu; d.pair_jr = pj; d.pair_nj = pn; d.pair_need = pnd;
    d.pair_x_off = pxo; d.xmap = xm; d.gd_slot = gs; d.gt_pair = tp; d.gt_mt = tm; d.gt_jt = tj;
    d.diag_row = dr;
    d.row_order = ro;
    d.gemm_prog = nullptr;
    if (h->opt.debug & 2) {
        TRY(dalloc(h, &d.gemm_prog, 4 * (size_t)std::max(1, h->grid)));
        if (cudaMemsetAsync(d.gemm_prog, 0xff, sizeof(int32_t) * 4 * (size_t)std::max(1, h->grid), st) != cudaSuccess)
            return HYLU_ERR_CUDA;
    }
    TRY(dalloc(h, &d.pair_cnt, G.pair_gd.size()));
    TRY(dalloc(h, &d.gd_done, G.ngd));
    TRY(dalloc(h, &d.walk_done, h->P.n));
    if (cudaMemsetAsync(d.walk_done, 0, sizeof(int32_t) * h->P.n, st) != cudaSuccess) return HYLU_ERR_CUDA;
    for (int s = 0; s < 3; ++s) TRY(dalloc(h, &d.a_term[s], (size_t)G.a_elems));
    std::vector<unsigned char> maps(hylu::tensor_map_bytes() * 3 * (size_t)G.ngd);
    TRY(hylu::encode_a_maps(G.ngd, G.gd_Mp.data(), G.gd_Kp.data(), G.gd_a_off.data(), d.a_term, maps.data()));
    unsigned char* dm = nullptr;
    TRY(upload(h, &dm, maps, st));
    d.tmaps = dm;
    d.n_gd = G.ngd;
    d.gemm_blocks = tc_blocks;
    d.n_pair = (int32_t)G.pair_gd.size();
    d.n_gtask = (int32_t)G.task_pair.size();
    d.n_diag = (int32_t)G.diag_row.size();
    d.a_elems = G.a_elems;
    h->gemm_flops = 0.0;
    for (size_t p = 0; p < G.pair_gd.size(); ++p) {
        h->gemm_flops += 2.0 * (double)G.pair_need[p] * G.pair_len[p] * G.pair_nj[p];
    }
    // the host copies above must outlive the asynchronous uploads
    if (cudaStreamSynchronize(st) != cudaSuccess) return HYLU_ERR_CUDA;
    return HYLU_OK;
}

// Bulk-sequential substitution (Sec. 2.3, Fig. 3): the bulk claim lists and
// the segments of light levels for solve_seq_rows = max_rows, both
// directions, built and uploaded once per value and made current.  One block
// takes the segments of a single system (they form one chain of levels); a
// batch gets one block per 8 segments (capped at launch), since its
// instances' segments are independent.
static int use_seq_segments(hylu_handle* h, int max_rows, cudaStream_t st) {
    hylu::DevPlan& d = h->dp;
    max_rows = std::max(0, max_rows);
    auto it = h->seq_tables.find(max_rows);
    if (it == h->seq_tables.end()) {
        hylu_handle::SeqTables Q{};
        int32_t nseg_max = 0;
        for (int dir = 0; dir < 2; ++dir) {
            hylu::SeqSegments S;
            hylu::build_seq_segments(h->P, dir == 1, max_rows, S);
            hylu::SegTable T{};
            T.nseg = (int32_t)(S.seg_off.size() - 1);
            nseg_max = std::max(nseg_max, T.nseg);
            for (std::vector<int32_t>* v : {&S.meta, &S.rows, &S.snodes})
                if (v->empty()) v->push_back(0);   // keep every array non-empty
            int32_t *task, *meta, *so, *lr, *ln, *rows, *sn;
            TRY(upload(h, &task, S.task, st));
            TRY(upload(h, &meta, S.meta, st));
            TRY(upload(h, &so, S.seg_off, st));
            TRY(upload(h, &lr, S.lvl_row, st));
            TRY(upload(h, &ln, S.lvl_node, st));
            TRY(upload(h, &rows, S.rows, st));
            TRY(upload(h, &sn, S.snodes, st));
            if (cudaStreamSynchronize(st) != cudaSuccess) return HYLU_ERR_CUDA;   // S goes out of scope
            T.meta = meta; T.seg_off = so; T.lvl_row = lr; T.lvl_node = ln; T.rows = rows; T.snodes = sn;
            if (dir == 0) {
                Q.fwd_task = task; Q.n_fwd_tasks = (int32_t)S.task.size(); Q.fseg = T;
                // long rows' chunks (forward only)
                const size_t nch = S.chunk_row.size();
                for (std::vector<int32_t>* v : {&S.chunk_row, &S.chunk_a, &S.chunk_b, &S.chunk_level})
                    if (v->empty()) v->push_back(0);
                int32_t *cr, *ca, *cb, *cl, *rco, *cf;
                double* cp;
                TRY(upload(h, &cr, S.chunk_row, st));
                TRY(upload(h, &ca, S.chunk_a, st));
                TRY(upload(h, &cb, S.chunk_b, st));
                TRY(upload(h, &cl, S.chunk_level, st));
                TRY(upload(h, &rco, S.row_chunk_off, st));
                TRY(dalloc(h, &cp, std::max<size_t>(1, nch)));
                TRY(dalloc(h, &cf, std::max<size_t>(1, nch)));
                if (cudaMemsetAsync(cf, 0, sizeof(int32_t) * std::max<size_t>(1, nch), st) != cudaSuccess)
                    return HYLU_ERR_CUDA;
                if (cudaStreamSynchronize(st) != cudaSuccess) return HYLU_ERR_CUDA;
                Q.fch_row = cr; Q.fch_a = ca; Q.fch_b = cb; Q.fch_level = cl; Q.frow_chunk_off = rco;
                Q.fch_part = cp; Q.fch_flag = cf;
            } else {
                Q.bwd_task = task; Q.n_bwd_tasks = (int32_t)S.task.size(); Q.bseg = T;
            }
        }
        const bool batch = !h->P.node_inst.empty();
        Q.seq_blocks = nseg_max == 0 ? 0 : batch ? std::max(1, (nseg_max + 7) / 8) : 1;
        it = h->seq_tables.emplace(max_rows, Q).first;
    }
    const hylu_handle::SeqTables& Q = it->second;
    d.fwd_task = Q.fwd_task; d.n_fwd_tasks = Q.n_fwd_tasks; d.fseg = Q.fseg;
    d.bwd_task = Q.bwd_task; d.n_bwd_tasks = Q.n_bwd_tasks; d.bseg = Q.bseg;
    d.seq_blocks = Q.seq_blocks;
    d.fch_row = Q.fch_row; d.fch_a = Q.fch_a; d.fch_b = Q.fch_b; d.fch_level = Q.fch_level;
    d.frow_chunk_off = Q.frow_chunk_off; d.fch_part = Q.fch_part; d.fch_flag = Q.fch_flag;
    h->opt.solve_seq_rows = max_rows;
    return HYLU_OK;
}

int ensure_uploaded(hylu_handle* h, cudaStream_t st) {
    if (h->uploaded) return HYLU_OK;
    if (cudaGetDevice(&h->device) != cudaSuccess) return HYLU_ERR_CUDA;
    hylu::Plan& P = h->P;
    hylu::DevPlan& d = h->dp;
    d.n = P.n;
    d.nnodes = P.nnodes;
    int32_t *sn, *nof, *lc, *tc, *ahs;
    int64_t *rl, *nto, *npo, *ahr, *ahsrc;
    double* ahsc;
    TRY(upload(h, &sn, P.sn_start, st));
    TRY(upload(h, &nof, P.node_of, st));
    TRY(upload(h, &rl, P.row_lptr, st));
    TRY(upload(h, &lc, P.lcols, st));
    TRY(upload(h, &nto, P.node_tail_off, st));
    TRY(upload(h, &tc, P.tcols, st));
    TRY(upload(h, &npo, P.node_panel_off, st));
    TRY(upload(h, &ahr, P.ah_rp, st));
    TRY(upload(h, &ahs, P.ah_slot, st));
    TRY(upload(h, &ahsrc, P.ah_src, st));
    TRY(upload(h, &ahsc, P.ah_scale, st));
    d.sn_start = sn; d.node_of = nof; d.row_lptr = rl; d.lcols = lc; d.node_tail_off = nto;
    d.tcols = tc; d.node_panel_off = npo; d.ah_rp = ahr; d.ah_slot = ahs; d.ah_src = ahsrc;
    d.ah_scale = ahsc;
    int32_t* ro;
    TRY(upload(h, &ro, P.row_order, st));
    d.row_order = ro;
    d.n_heavy = (int32_t)P.heavy_order.size();
    d.heavy_order = nullptr;
    d.heavy_rank = nullptr;
    if (d.n_heavy > 0) {
        int32_t *ho, *hr;
        TRY(upload(h, &ho, P.heavy_order, st));
        TRY(upload(h, &hr, P.heavy_rank, st));
        d.heavy_order = ho;
        d.heavy_rank = hr;
    }
    d.trace = nullptr;
    if (h->opt.debug & 2) TRY(dalloc(h, &d.trace, 4 * (size_t)P.n));
    d.strace = nullptr;
    if (h->opt.debug & 4) {
        TRY(dalloc(h, &d.strace, 2 * (size_t)std::max(1, P.nnodes)));
        if (cudaMemsetAsync(d.strace, 0, sizeof(unsigned long long) * 2 * std::max(1, P.nnodes), st) != cudaSuccess)
            return HYLU_ERR_CUDA;
    }
    d.lval = nullptr; d.pval = nullptr; d.lval32 = nullptr; d.pval32 = nullptr; d.dinv32 = nullptr;
    if (h->opt.precision == 1) {
        TRY(dalloc(h, &d.lval32, P.nnz_l));
        TRY(dalloc(h, &d.pval32, P.nnz_panel));
        TRY(dalloc(h, &d.dinv32, P.n));
    } else {
        TRY(dalloc(h, &d.lval, P.nnz_l));
        TRY(dalloc(h, &d.pval, P.nnz_panel));
    }
    TRY(dalloc(h, &d.piv, P.n));
    TRY(dalloc(h, &d.pinv, P.n));
    TRY(dalloc(h, &d.ready, P.n));
    TRY(dalloc(h, &d.dready, P.n));
    TRY(dalloc(h, &d.gens, 2));
    if (cudaMemsetAsync(d.gens, 0, sizeof(int32_t) * 2, st) != cudaSuccess) return HYLU_ERR_CUDA;
    TRY(dalloc(h, &d.node_done, std::max<int32_t>(1, P.nnodes)));
    d.n_tasks = P.n_tasks;
    {
        int32_t *tn, *tch, *nnt;
        TRY(upload(h, &nnt, P.node_ntask, st));
        TRY(upload(h, &tn, P.task_node, st));
        TRY(upload(h, &tch, P.task_chunk, st));
        d.node_ntask = nnt; d.task_node = tn; d.task_chunk = tch;
    }
    {
        int32_t *fo, *bo, *fl, *bl, *fc, *bc;
        TRY(upload(h, &fo, P.fwd_order, st));
        TRY(upload(h, &bo, P.bwd_order, st));
        TRY(upload(h, &fl, P.fwd_level, st));
        TRY(upload(h, &bl, P.bwd_level, st));
        TRY(upload(h, &fc, P.fwd_count, st));
        TRY(upload(h, &bc, P.bwd_count, st));
        d.fwd_order = fo; d.bwd_order = bo; d.fwd_level = fl; d.bwd_level = bl;
        d.fwd_count = fc; d.bwd_count = bc;
        d.n_fwd_levels = (int32_t)P.fwd_count.size();
        d.n_bwd_levels = (int32_t)P.bwd_count.size();
        TRY(dalloc(h, &d.fwd_done, P.fwd_count.size()));
        TRY(dalloc(h, &d.bwd_done, P.bwd_count.size()));
        // split points of the substitution's dot products: the entries whose
        // sources lie two or more levels below the row's own
        {
            std::vector<int32_t> fs(P.n, 0), bs(P.nnodes, 0);
            for (int32_t D = 0; D < P.nnodes; ++D) {
                const int32_t L = P.fwd_level[D];
                for (int32_t i = P.sn_start[D]; i < P.sn_start[D + 1]; ++i) {
                    int64_t t = P.row_lptr[i];
                    while (t < P.row_lptr[i + 1] && P.fwd_level[P.node_of[P.lcols[t]]] <= L - 2) ++t;
                    fs[i] = (int32_t)(t - P.row_lptr[i]);
                }
                const int32_t Lb = P.bwd_level[D];
                const int64_t a = P.node_tail_off[D];
                int64_t sp = P.node_tail_off[D + 1];
                while (sp > a && P.bwd_level[P.node_of[P.tcols[sp - 1]]] <= Lb - 2) --sp;
                bs[D] = (int32_t)(sp - a);
            }
            int32_t *dfs, *dbs;
            TRY(upload(h, &dfs, fs, st));
            TRY(upload(h, &dbs, bs, st));
            if (cudaStreamSynchronize(st) != cudaSuccess) return HYLU_ERR_CUDA;   // fs, bs go out of scope
            d.fwd_split = dfs;
            d.bwd_split = dbs;
        }
        TRY(use_seq_segments(h, h->opt.solve_seq_rows, st));
        int32_t *uo, *lo, *ul, *ll, *uc, *lcn;
        TRY(upload(h, &uo, P.ut_order, st));
        TRY(upload(h, &lo, P.lt_order, st));
        TRY(upload(h, &ul, P.ut_level, st));
        TRY(upload(h, &ll, P.lt_level, st));
        TRY(upload(h, &uc, P.ut_count, st));
        TRY(upload(h, &lcn, P.lt_count, st));
        d.ut_order = uo; d.lt_order = lo; d.ut_level = ul; d.lt_level = ll; d.ut_count = uc; d.lt_count = lcn;
        d.n_ut_levels = (int32_t)P.ut_count.size();
        d.n_lt_levels = (int32_t)P.lt_count.size();
        TRY(dalloc(h, &d.ut_done, P.ut_count.size()));
        TRY(dalloc(h, &d.lt_done, P.lt_count.size()));
        // instances and their slices of the level counts (one for a single system)
        const int32_t ni = P.node_inst.empty() ? 1 : (int32_t)P.fwd_off.size() - 1;
        d.n_inst = ni;
        d.node_inst = nullptr;
        if (!P.node_inst.empty()) {
            int32_t* nin;
            TRY(upload(h, &nin, P.node_inst, st));
            d.node_inst = nin;
        }
        auto slice = [&](const std::vector<int32_t>& off, const std::vector<int32_t>& cnt, const int32_t** out) {
            std::vector<int32_t> o = off.empty() ? std::vector<int32_t>{0, (int32_t)cnt.size()} : off;
            int32_t* dp = nullptr;
            int rc = upload(h, &dp, o, st);
            *out = dp;
            return rc;
        };
        TRY(slice(P.fwd_off, P.fwd_count, &d.fwd_off));
        TRY(slice(P.bwd_off, P.bwd_count, &d.bwd_off));
        TRY(slice(P.ut_off, P.ut_count, &d.ut_off));
        TRY(slice(P.lt_off, P.lt_count, &d.lt_off));
        TRY(dalloc(h, &d.wm_f, ni));
        TRY(dalloc(h, &d.wm_b, ni));
    }
    TRY(dalloc(h, &d.fwd_row, P.n));
    TRY(dalloc(h, &d.bwd_row, P.n));
    TRY(dalloc(h, &d.tile_f, P.n));
    TRY(dalloc(h, &d.tile_b, P.n));
    TRY(dalloc(h, &d.dinv, P.n));
    TRY(dalloc(h, &d.status, hylu::ST_WORDS));
    h->grid = hylu::factor_grid(h->device, h->opt.precision == 1);
    h->solve_grid = h->grid;
    TRY(upload_gemm(h, st));
    {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        h->grid_max = std::max(h->grid, sms * 4);
    }
    d.pos_n = h->batch ? h->layout.pos_n : P.n;
    d.node_base = nullptr;
    if (h->batch) {
        int32_t* nb;
        TRY(upload(h, &nb, h->layout.node_base, st));
        d.node_base = nb;
    }
    TRY(dalloc(h, &d.pos, (size_t)h->grid_max * hylu::warps_per_block() * (size_t)d.pos_n));
    d.spa64 = nullptr;
    d.spa32 = nullptr;
    {
        int64_t max_nl = 0;
        for (int32_t i = 0; i < P.n; ++i) max_nl = std::max<int64_t>(max_nl, P.row_lptr[i + 1] - P.row_lptr[i]);
        if (max_nl > hylu::dense_l_min()) {
            const size_t cnt = (size_t)h->grid_max * hylu::warps_per_block() * (size_t)d.pos_n;
            if (h->opt.precision == 1) TRY(dalloc(h, &d.spa32, cnt));
            else TRY(dalloc(h, &d.spa64, cnt));
        }
    }
    if (cudaMemsetAsync(d.ready, 0, sizeof(int32_t) * P.n, st) != cudaSuccess) return HYLU_ERR_CUDA;
    if (cudaMemsetAsync(d.dready, 0, sizeof(int32_t) * P.n, st) != cudaSuccess) return HYLU_ERR_CUDA;
    if (cudaMemsetAsync(d.fwd_row, 0, sizeof(int32_t) * P.n, st) != cudaSuccess) return HYLU_ERR_CUDA;
    if (cudaMemsetAsync(d.bwd_row, 0, sizeof(int32_t) * P.n, st) != cudaSuccess) return HYLU_ERR_CUDA;
    if (cudaMemsetAsync(d.tile_f, 0, sizeof(int32_t) * P.n, st) != cudaSuccess) return HYLU_ERR_CUDA;
    if (cudaMemsetAsync(d.tile_b, 0, sizeof(int32_t) * P.n, st) != cudaSuccess) return HYLU_ERR_CUDA;
    TRY(dalloc(h, &h->d_avals, P.nnz_a));
    TRY(upload(h, &h->d_arp, P.a_rp, st));
    TRY(upload(h, &h->d_aci, P.a_ci, st));
    TRY(upload(h, &h->d_rowperm, P.rowperm, st));
    TRY(upload(h, &h->d_colperm, P.colperm, st));
    TRY(upload(h, &h->d_dr, P.dr, st));
    TRY(upload(h, &h->d_dc, P.dc, st));
    if (cudaMallocHost(&h->h_status, sizeof(int32_t) * hylu::ST_WORDS) != cudaSuccess) return HYLU_ERR_NOMEM;
    for (int q = 0; q < 4; ++q)
        if (cudaEventCreate(&h->ev[q]) != cudaSuccess) return HYLU_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HYLU_ERR_CUDA;   // host vectors stay alive anyway
    h->uploaded = true;
    return HYLU_OK;
}

int ensure_rhs(hylu_handle* h, int nrhs, int ld) {
    const size_t need = (size_t)ld * (size_t)nrhs;
    if (nrhs <= h->cap_rhs && need <= h->cap_elems) return HYLU_OK;
    const size_t n = (size_t)h->P.n;
    TRY(dalloc(h, &h->d_z, n * nrhs));
    TRY(dalloc(h, &h->d_xh, n * nrhs));
    TRY(dalloc(h, &h->d_r, need));
    TRY(dalloc(h, &h->d_d, need));
    if (!h->d_colsum) TRY(dalloc(h, &h->d_colsum, n));
    h->cap_elems = need;
    TRY(dalloc(h, &h->d_norms, 3 * (size_t)nrhs + 1));
    if (h->h_norms) cudaFreeHost(h->h_norms);
    if (cudaMallocHost(&h->h_norms, sizeof(double) * (3 * (size_t)nrhs + 1)) != cudaSuccess) return HYLU_ERR_NOMEM;
    h->cap_rhs = nrhs;
    return HYLU_OK;
}

int read_status(hylu_handle* h, cudaStream_t st) {
    if (cudaMemcpyAsync(h->h_status, h->dp.status, sizeof(int32_t) * hylu::ST_WORDS, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return HYLU_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HYLU_ERR_CUDA;
    h->nperturb = h->h_status[hylu::ST_NPERT];
    h->device_status = h->h_status[hylu::ST_ERR];
    h->failed_node = h->device_status ? h->h_status[hylu::ST_FAILED] : -1;
    return h->device_status ? h->device_status : HYLU_OK;
}

int do_factor(hylu_handle* h, const double* d_vals, cudaStream_t st) {
    if (h->P.n == 0) {                 // empty system: nothing to factor, no device work
        h->factored = true;
        return HYLU_OK;
    }
    if (!d_vals) return HYLU_ERR_ARG;
    TRY(ensure_uploaded(h, st));
    if (cudaMemcpyAsync(h->d_avals, d_vals, sizeof(double) * h->P.nnz_a, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return HYLU_ERR_CUDA;
    TRY(hylu::launch_reset(h->dp.status, h->dp.piv, h->dp.pinv, h->dp.gens, h->P.n, st));
    TRY(hylu::launch_factor(h->dp, h->d_avals, h->P.nnz_a, h->opt.pivot_tau,
                            h->opt.spin_limit, h->grid, st, h->opt.timing ? h->ev[0] : nullptr,
                            h->opt.timing ? h->ev[1] : nullptr));
    if (h->opt.timing) h->timed_factor = true;
    h->factored = true;
    h->last = st;
    return HYLU_OK;
}

double max_be(const hylu_handle* h, int nrhs) {
    double anorm;
    std::memcpy(&anorm, &h->h_norms[3 * nrhs], sizeof(double));
    double be = 0.0;
    for (int r = 0; r < nrhs; ++r) {
        double rn = h->h_norms[3 * r], xn = h->h_norms[3 * r + 1], bn = h->h_norms[3 * r + 2];
        double den = anorm * xn + bn;
        double b = den > 0 ? rn / den : rn;
        if (!(b <= be)) be = b;   // NaN propagates
    }
    return be;
}

int do_solve(hylu_handle* h, const double* d_b, double* d_x, int nrhs, int ld, cudaStream_t st) {
    if (!h->factored) return HYLU_ERR_STATE;
    if (h->P.n == 0) return nrhs < 1 || ld < 0 ? HYLU_ERR_ARG : HYLU_OK;
    if (!d_b || !d_x || nrhs < 1 || ld < h->P.n) return HYLU_ERR_ARG;
    TRY(ensure_rhs(h, nrhs, ld));
    // the perturbation count decides whether to refine (Sec. 2.3); this also
    // surfaces a device-side failure of the factorization.  opt.refine < 0:
    // no refinement and no synchronization (the call stays asynchronous).
    if (h->opt.refine >= 0) TRY(read_status(h, st));
    hylu::DevPlan& P = h->dp;
    TRY(hylu::launch_solve(P, d_b, d_x, h->d_z, h->d_xh, h->d_rowperm, h->d_colperm, h->d_dr, h->d_dc,
                           nrhs, ld, h->opt.spin_limit, h->solve_grid, st,
                           h->opt.timing ? h->ev[2] : nullptr, h->opt.timing ? h->ev[3] : nullptr));
    if (h->opt.timing) h->timed_solve = true;
    h->refine_iters = 0;
    h->backward_error = -1.0;
    h->last = st;
    h->graph_norms_pending = false;
    if (h->opt.refine < 0 || !(h->nperturb > 0 || h->opt.refine)) return HYLU_OK;
    // iterative refinement in FP64 on the original A (Sec. 2.3)
    double be_prev = INFINITY;
    for (;;) {
        TRY(hylu::launch_residual(h->P.n, h->d_arp, h->d_aci, h->d_avals, d_x, d_b, h->d_r, h->d_norms,
                                  nrhs, ld, st));
        if (cudaMemcpyAsync(h->h_norms, h->d_norms, sizeof(double) * (3 * nrhs + 1), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return HYLU_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return HYLU_ERR_CUDA;
        double be = max_be(h, nrhs);
        h->backward_error = be;
        if (be <= h->opt.refine_tol) return HYLU_OK;
        if (h->refine_iters >= h->opt.refine_maxit || !(be <= 0.5 * be_prev)) return HYLU_WARN_REFINE_STALLED;
        be_prev = be;
        Range step("hylu_refine_step");
        TRY(hylu::launch_solve(P, h->d_r, h->d_d, h->d_z, h->d_xh, h->d_rowperm, h->d_colperm, h->d_dr,
                               h->d_dc, nrhs, ld, h->opt.spin_limit, h->solve_grid, st));
        TRY(hylu::launch_axpy(h->P.n, d_x, h->d_d, nrhs, ld, st));
        ++h->refine_iters;
    }
}

// Transpose solve A^T x = b with the same refinement rule as do_solve.
int do_solve_transpose(hylu_handle* h, const double* d_b, double* d_x, int nrhs, int ld, cudaStream_t st) {
    if (!h->factored) return HYLU_ERR_STATE;
    if (h->P.n == 0) return nrhs < 1 || ld < 0 ? HYLU_ERR_ARG : HYLU_OK;
    if (!d_b || !d_x || nrhs < 1 || ld < h->P.n) return HYLU_ERR_ARG;
    TRY(ensure_rhs(h, nrhs, ld));
    TRY(read_status(h, st));
    hylu::DevPlan& P = h->dp;
    TRY(hylu::launch_solve_transpose(P, d_b, d_x, h->d_z, h->d_rowperm, h->d_colperm, h->d_dr, h->d_dc, nrhs, ld,
                                     h->opt.spin_limit, h->solve_grid, st));
    h->refine_iters = 0;
    h->backward_error = -1.0;
    h->last = st;
    if (!(h->nperturb > 0 || h->opt.refine)) return HYLU_OK;
    double be_prev = INFINITY;
    for (;;) {
        TRY(hylu::launch_residual_transpose(h->P.n, h->d_arp, h->d_aci, h->d_avals, d_x, d_b, h->d_r, h->d_colsum,
                                            h->d_norms, nrhs, ld, st));
        if (cudaMemcpyAsync(h->h_norms, h->d_norms, sizeof(double) * (3 * nrhs + 1), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return HYLU_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return HYLU_ERR_CUDA;
        double be = max_be(h, nrhs);
        h->backward_error = be;
        if (be <= h->opt.refine_tol) return HYLU_OK;
        if (h->refine_iters >= h->opt.refine_maxit || !(be <= 0.5 * be_prev)) return HYLU_WARN_REFINE_STALLED;
        be_prev = be;
        Range step("hylu_refine_step");
        TRY(hylu::launch_solve_transpose(P, h->d_r, h->d_d, h->d_z, h->d_rowperm, h->d_colperm, h->d_dr, h->d_dc,
                                         nrhs, ld, h->opt.spin_limit, h->solve_grid, st));
        TRY(hylu::launch_axpy(h->P.n, d_x, h->d_d, nrhs, ld, st));
        ++h->refine_iters;
    }
}

}  // namespace

// Substitution into caller-provided work vectors z and xh (n doubles each):
// no allocation, no synchronization, no refinement.  Used by the
// allocation-free entry point in static_solve.cu.
namespace hylu {
int32_t handle_n(const hylu_handle* h) { return h->P.n; }

// HYLU_OK when the allocation-free substitution can run on h now, 1 when
// there is nothing to do (a factored empty system), else an error: not
// factored, FP32 factors (they need the refinement of hylu_solve to reach
// the FP64 backward error), or a current device other than the handle's.
int static_solve_ready(const hylu_handle* h) {
    if (!h->factored) return HYLU_ERR_STATE;
    if (h->P.n == 0) return 1;
    if (!h->uploaded || h->opt.precision != 0) return HYLU_ERR_STATE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return HYLU_ERR_CUDA;
    return dev == h->device ? HYLU_OK : HYLU_ERR_ARG;
}

int solve_into(hylu_handle* h, const double* d_b, double* d_x, double* z, double* xh, cudaStream_t st) {
    const int ready = static_solve_ready(h);
    if (ready != HYLU_OK) return ready < 0 ? ready : HYLU_OK;
    h->last = st;
    return launch_solve(h->dp, d_b, d_x, z, xh, h->d_rowperm, h->d_colperm, h->d_dr, h->d_dc, 1, h->P.n,
                        h->opt.spin_limit, h->solve_grid, st);
}
}  // namespace hylu

extern "C" {

int hylu_default_options(hylu_options* o) {
    if (!o) return HYLU_ERR_ARG;
    std::memset(o, 0, sizeof(*o));
    o->ordering = HYLU_ORDER_AMD;
    o->static_pivot = 1;
    o->scale = 1;
    o->sn_max = 256;
    o->nd_leaf = 256;
    o->pivot_tau = 1.4901161193847656e-08;
    o->refine_tol = 1e-12;
    o->refine_maxit = 10;
    o->refine = 0;
    o->spin_limit = 1LL << 26;
    o->rows_per_task = 1;
    o->debug = 0;
    o->amd_dense = 2.0;
    o->timing = 0;
    o->precision = 0;
    o->heavy_ratio = 32.0;
    o->gemm_min_rows = 64;
    o->solve_seq_rows = 8;
    return HYLU_OK;
}

int hylu_analyze(int32_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col, const double* vals,
                 const int32_t* user_perm, const hylu_options* opt, hylu_handle** out) {
    Range range_("hylu_analyze");
    if (!out || n < 0 || !rowptr || (nnz > 0 && !col)) return HYLU_ERR_ARG;
    *out = nullptr;
    if (rowptr[n] != nnz) return HYLU_ERR_PATTERN;
    hylu_options o;
    if (opt) o = *opt; else hylu_default_options(&o);
    if (o.sn_max < 1 || o.sn_max > 256) return HYLU_ERR_ARG;
    if (o.ordering < HYLU_ORDER_AMD || o.ordering > HYLU_ORDER_AUTO) return HYLU_ERR_ARG;
    if (o.precision != 0 && o.precision != 1) return HYLU_ERR_ARG;
    if (!(o.heavy_ratio >= 0.0)) return HYLU_ERR_ARG;
    if (o.precision == 1 && o.refine == 0) o.refine = 1;   // FP32 factors: always refine in FP64
    hylu_handle* h = new (std::nothrow) hylu_handle();
    if (!h) return HYLU_ERR_NOMEM;
    h->opt = o;
    hylu::AnalyzeOptions ao;
    ao.ordering = o.ordering;
    ao.static_pivot = o.static_pivot;
    ao.scale = o.scale;
    ao.sn_max = o.sn_max;
    ao.nd_leaf = o.nd_leaf > 0 ? o.nd_leaf : 256;
    ao.amd_dense = o.amd_dense > 0 ? o.amd_dense : 2.0;
    ao.heavy_ratio = o.heavy_ratio;
    const int rc = guarded([&] { return hylu::analyze(n, rowptr, col, vals, user_perm, ao, h->P); });
    if (rc) { delete h; return rc; }
    *out = h;
    return HYLU_OK;
}

int hylu_factor(hylu_handle* h, const double* d_vals, void* stream) {
    Range range_("hylu_factor");
    if (!h) return HYLU_ERR_ARG;
    return guarded([&] { return do_factor(h, d_vals, static_cast<cudaStream_t>(stream)); });
}

int hylu_refactor(hylu_handle* h, const double* d_vals, void* stream) {
    Range range_("hylu_refactor");
    if (!h) return HYLU_ERR_ARG;
    if (!h->factored) return HYLU_ERR_STATE;
    return guarded([&] { return do_factor(h, d_vals, static_cast<cudaStream_t>(stream)); });
}

int hylu_solve(hylu_handle* h, const double* d_b, double* d_x, int nrhs, int ld, void* stream) {
    Range range_("hylu_solve");
    if (!h) return HYLU_ERR_ARG;
    return guarded([&] { return do_solve(h, d_b, d_x, nrhs, ld, static_cast<cudaStream_t>(stream)); });
}

int hylu_solve_transpose(hylu_handle* h, const double* d_b, double* d_x, int nrhs, int ld, void* stream) {
    Range range_("hylu_solve_transpose");
    if (!h) return HYLU_ERR_ARG;
    return guarded([&] { return do_solve_transpose(h, d_b, d_x, nrhs, ld, static_cast<cudaStream_t>(stream)); });
}

int hylu_grad_values(hylu_handle* h, const double* d_lam, const double* d_x, double* d_dvals, int nrhs, int ld,
                     void* stream) {
    Range range_("hylu_grad_values");
    if (!h || nrhs < 1 || ld < h->P.n) return HYLU_ERR_ARG;
    if (h->P.n == 0) return h->factored ? HYLU_OK : HYLU_ERR_STATE;
    if (!d_lam || !d_x || !d_dvals) return HYLU_ERR_ARG;
    if (!h->uploaded) return HYLU_ERR_STATE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    h->last = st;
    return hylu::launch_grad_values(h->P.n, h->d_arp, h->d_aci, d_lam, d_x, d_dvals, nrhs, ld, st);
}

int hylu_get_info(hylu_handle* h, hylu_info* info) {
    if (!h || !info) return HYLU_ERR_ARG;
    std::memset(info, 0, sizeof(*info));
    const hylu::Plan& P = h->P;
    info->n = P.n;
    info->nnz_a = P.nnz_a;
    info->nnz_lu = P.nnz_f;
    info->nnz_store = P.nnz_l + P.nnz_panel;
    info->nnodes = P.nnodes;
    int ns = 0, rs = 0, mx = 0;
    for (int32_t s = 0; s < P.nnodes; ++s) {
        int sz = P.sn_start[s + 1] - P.sn_start[s];
        if (sz > 1) { ++ns; rs += sz; }
        if (sz > mx) mx = sz;
    }
    info->nsupernodes = ns;
    info->rows_in_supernodes = rs;
    info->max_supernode = mx;
    info->ntasks = P.n + P.n_tasks;
    info->nheavy = (int32_t)P.heavy_order.size();
    info->factor_levels = P.row_levels;
    auto levels = [](const std::vector<int32_t>& off, const std::vector<int32_t>& cnt) {
        if (off.size() < 2) return (int32_t)cnt.size();
        int32_t m = 0;
        for (size_t q = 0; q + 1 < off.size(); ++q) m = std::max(m, off[q + 1] - off[q]);
        return m;
    };
    info->fwd_levels = levels(P.fwd_off, P.fwd_count);
    info->bwd_levels = levels(P.bwd_off, P.bwd_count);
    info->flops = P.flops_unpadded;
    info->flops_padded = P.flops_padded;
    info->flops_row_row = P.flops_row_row;
    info->flops_sup_row = P.flops_sup_row;
    info->flops_sup_sup = P.flops_sup_sup;
    info->flops_in_supernode = P.flops_in_sn;
    info->ordering = P.ordering;
    for (int ph = 0; ph < 4; ++ph) info->analyze_phase_ms[ph] = P.analyze_phase_ms[ph];
    info->tuned = h->tuned;
    {
        int sms = 1;
        if (h->uploaded) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        sms = std::max(1, sms);
        info->factor_blocks_per_sm = h->uploaded ? h->grid / sms : 0;
        info->solve_blocks_per_sm = h->uploaded ? h->solve_grid / sms : 0;
    }
    info->heavy_queue = (h->dp.n_heavy > 0) ? 1 : 0;
    info->solve_seq_rows = h->opt.solve_seq_rows;
    info->solve_segments[0] = h->uploaded ? h->dp.fseg.nseg : 0;
    info->solve_segments[1] = h->uploaded ? h->dp.bseg.nseg : 0;
    info->gemm_destinations = h->dp.n_gd;
    info->gemm_tasks = h->dp.n_gtask;
    info->gemm_flops = h->gemm_flops;
    info->analyze_ms = P.analyze_ms;
    int rc = HYLU_OK;
    if (h->factored && h->uploaded) rc = read_status(h, h->last);
    if (rc == HYLU_OK && h->graph_norms_pending) {
        // the last replay's final residual: its backward error (read_status
        // above synchronized the stream the graph ran on)
        const int nr = h->graph_nrhs;
        if (cudaMemcpy(h->h_norms, h->d_norms, sizeof(double) * (3 * nr + 1), cudaMemcpyDeviceToHost) != cudaSuccess)
            return HYLU_ERR_CUDA;
        h->backward_error = max_be(h, nr);
        h->refine_iters = h->graph_corrections;
        h->graph_norms_pending = false;
    }
    info->nperturb = h->nperturb;
    info->refine_iters = h->refine_iters;
    info->backward_error = h->backward_error;
    info->device_status = h->device_status;
    info->failed_node = h->failed_node;
    info->factor_kernel_ms = -1.0;
    info->solve_kernel_ms = -1.0;
    float ms = 0.f;
    if (h->timed_factor && cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]) == cudaSuccess) info->factor_kernel_ms = ms;
    if (h->timed_solve && cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]) == cudaSuccess) info->solve_kernel_ms = ms;
    return rc < 0 ? rc : HYLU_OK;
}

int hylu_export_perm(hylu_handle* h, int32_t* rowperm, int32_t* colperm, double* dr, double* dc,
                     int32_t* sn_start) {
    if (!h) return HYLU_ERR_ARG;
    const hylu::Plan& P = h->P;
    if (rowperm) std::memcpy(rowperm, P.rowperm.data(), sizeof(int32_t) * P.n);
    if (colperm) std::memcpy(colperm, P.colperm.data(), sizeof(int32_t) * P.n);
    if (dr) std::memcpy(dr, P.dr.data(), sizeof(double) * P.n);
    if (dc) std::memcpy(dc, P.dc.data(), sizeof(double) * P.n);
    if (sn_start) std::memcpy(sn_start, P.sn_start.data(), sizeof(int32_t) * P.sn_start.size());
    return HYLU_OK;
}

int hylu_export_schedule(hylu_handle* h, int32_t* order, int32_t* heavy, int32_t* task_node) {
    if (!h) return HYLU_ERR_ARG;
    const hylu::Plan& P = h->P;
    if (order) std::memcpy(order, P.row_order.data(), sizeof(int32_t) * P.row_order.size());
    if (heavy) std::memcpy(heavy, P.heavy_order.data(), sizeof(int32_t) * P.heavy_order.size());
    if (task_node) std::memcpy(task_node, P.task_node.data(), sizeof(int32_t) * P.task_node.size());
    return HYLU_OK;
}

int hylu_export_gemm_plan(hylu_handle* h, int min_rows, int64_t* buf, int64_t* len) {
    if (!h || !len) return HYLU_ERR_ARG;
    return guarded([&] {
        hylu::GemmPlan G;
        if (hylu::build_gemm_plan(h->P, min_rows, G) != 0) return HYLU_ERR_INTERNAL;
        std::vector<int64_t> out;
        const int64_t head[10] = {G.ngd, (int64_t)G.pair_gd.size(), (int64_t)G.xmap.size(),
                                  (int64_t)G.task_pair.size(), (int64_t)G.diag_row.size(),
                                  (int64_t)G.row_order.size(), G.levels, (int64_t)h->P.lcols.size(), G.min_src,
                                  G.a_elems};
        out.insert(out.end(), head, head + 10);
        if (G.ngd) {
            auto put = [&](const auto& v) { for (auto x : v) out.push_back((int64_t)x); };
            put(G.gd_node); put(G.gd_Kp); put(G.gd_Mp); put(G.gd_a_off); put(G.gd_ntask);
            put(G.pair_gd); put(G.pair_src); put(G.pair_u0); put(G.pair_len); put(G.pair_jr); put(G.pair_nj);
            put(G.pair_need); put(G.pair_x_off); put(G.xmap); put(G.gd_slot);
            put(G.task_pair); put(G.task_mt); put(G.task_jt); put(G.task_level);
            put(G.row_order); put(G.diag_row); put(G.walk_level); put(G.diag_level);
        }
        const int64_t need = (int64_t)out.size();
        if (!buf) { *len = need; return HYLU_OK; }
        if (*len < need) { *len = need; return HYLU_ERR_ARG; }
        std::memcpy(buf, out.data(), sizeof(int64_t) * out.size());
        *len = need;
        return HYLU_OK;
    });
}

int hylu_export_solve_segments(hylu_handle* h, int backward, int max_rows, int32_t* buf, int64_t* len) {
    if (!h || !len) return HYLU_ERR_ARG;
    return guarded([&] {
        hylu::SeqSegments S;
        hylu::build_seq_segments(h->P, backward != 0, max_rows, S);
        std::vector<int32_t> out = {(int32_t)S.task.size(), (int32_t)(S.seg_off.size() - 1),
                                    (int32_t)(S.lvl_row.size() - 1), (int32_t)S.rows.size(), (int32_t)S.snodes.size(),
                                    (int32_t)S.chunk_row.size()};
        for (const std::vector<int32_t>* v : {&S.task, &S.meta, &S.seg_off, &S.lvl_row, &S.lvl_node, &S.rows, &S.snodes,
                                              &S.chunk_row, &S.chunk_a, &S.chunk_b, &S.chunk_level, &S.row_chunk_off})
            out.insert(out.end(), v->begin(), v->end());
        const int64_t need = (int64_t)out.size();
        if (!buf) { *len = need; return HYLU_OK; }
        if (*len < need) { *len = need; return HYLU_ERR_ARG; }
        std::memcpy(buf, out.data(), sizeof(int32_t) * out.size());
        *len = need;
        return HYLU_OK;
    });
}

int hylu_export_pattern(hylu_handle* h, int64_t* rowptr, int32_t* col) {
    if (!h) return HYLU_ERR_ARG;
    const hylu::Plan& P = h->P;
    int64_t pos = 0;
    if (rowptr) rowptr[0] = 0;
    for (int32_t i = 0; i < P.n; ++i) {
        const int32_t D = P.node_of[i], r = P.sn_start[D], e = P.sn_start[D + 1] - 1;
        for (int64_t t = P.row_lptr[i]; t < P.row_lptr[i + 1]; ++t) { if (col) col[pos] = P.lcols[t]; ++pos; }
        for (int32_t c = r; c <= e; ++c) { if (col) col[pos] = c; ++pos; }
        for (int64_t t = P.node_tail_off[D]; t < P.node_tail_off[D + 1]; ++t) { if (col) col[pos] = P.tcols[t]; ++pos; }
        if (rowptr) rowptr[i + 1] = pos;
    }
    return HYLU_OK;
}

static int export_factors_impl(hylu_handle* h, double* vals, int32_t* piv) {
    if (!h) return HYLU_ERR_ARG;
    if (!h->factored) return HYLU_ERR_STATE;
    const hylu::Plan& P = h->P;
    if (P.n == 0) return HYLU_OK;
    if (cudaStreamSynchronize(h->last) != cudaSuccess) return HYLU_ERR_CUDA;
    std::vector<double> lv(P.nnz_l), pv(P.nnz_panel);
    std::vector<int32_t> pv_piv(P.n);
    if (h->dp.lval32) {
        std::vector<float> lf(P.nnz_l), pf(P.nnz_panel);
        if (cudaMemcpy(lf.data(), h->dp.lval32, sizeof(float) * P.nnz_l, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(pf.data(), h->dp.pval32, sizeof(float) * P.nnz_panel, cudaMemcpyDeviceToHost) != cudaSuccess)
            return HYLU_ERR_CUDA;
        for (int64_t q = 0; q < P.nnz_l; ++q) lv[q] = lf[q];
        for (int64_t q = 0; q < P.nnz_panel; ++q) pv[q] = pf[q];
    } else if (cudaMemcpy(lv.data(), h->dp.lval, sizeof(double) * P.nnz_l, cudaMemcpyDeviceToHost) != cudaSuccess ||
               cudaMemcpy(pv.data(), h->dp.pval, sizeof(double) * P.nnz_panel, cudaMemcpyDeviceToHost) != cudaSuccess) {
        return HYLU_ERR_CUDA;
    }
    if (cudaMemcpy(pv_piv.data(), h->dp.piv, sizeof(int32_t) * P.n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return HYLU_ERR_CUDA;
    if (piv) std::memcpy(piv, pv_piv.data(), sizeof(int32_t) * P.n);
    if (!vals) return HYLU_OK;
    int64_t pos = 0;
    for (int32_t i = 0; i < P.n; ++i) {
        const int32_t D = P.node_of[i], r = P.sn_start[D], e = P.sn_start[D + 1] - 1, s = e - r + 1;
        const int64_t nT = P.node_tail_off[D + 1] - P.node_tail_off[D];
        const double* row = pv.data() + P.node_panel_off[D] + (int64_t)(i - r) * (s + nT);
        for (int64_t t = P.row_lptr[i]; t < P.row_lptr[i + 1]; ++t) vals[pos++] = lv[t];
        for (int32_t p = r; p <= e; ++p) vals[pos++] = row[pv_piv[p] - r];   // block: label -> position
        for (int64_t t = 0; t < nT; ++t) vals[pos++] = row[s + t];
    }
    return HYLU_OK;
}

int hylu_export_factors(hylu_handle* h, double* vals, int32_t* piv) {
    return guarded([&] { return export_factors_impl(h, vals, piv); });
}

int hylu_destroy(hylu_handle* h) {
    if (!h) return HYLU_OK;
    if (h->uploaded) cudaDeviceSynchronize();
    for (void* p : h->allocs) cudaFree(p);
    for (int q = 0; q < 4; ++q) if (h->ev[q]) cudaEventDestroy(h->ev[q]);
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->h_norms) cudaFreeHost(h->h_norms);
    if (h->h_status) cudaFreeHost(h->h_status);
    delete h;
    return HYLU_OK;
}

int64_t hylu_launch_count(void) { return hylu::launches(); }

int hylu_analyze_batch(int32_t k, const int32_t* n, const int64_t* const* rowptr, const int32_t* const* col,
                       const double* const* vals, int32_t nsets, const hylu_options* opt, hylu_handle** out) {
    Range range_("hylu_analyze_batch");
    if (!out || k < 1 || nsets < 1 || !n || !rowptr || !col) return HYLU_ERR_ARG;
    *out = nullptr;
    for (int32_t s = 0; s < k; ++s)
        if (n[s] < 1) return HYLU_ERR_ARG;   // every instance holds at least one row
    hylu_options o;
    if (opt) o = *opt; else hylu_default_options(&o);
    if (o.sn_max < 1 || o.sn_max > 256) return HYLU_ERR_ARG;
    if (o.ordering < HYLU_ORDER_AMD || o.ordering > HYLU_ORDER_AUTO) return HYLU_ERR_ARG;
    if (o.precision != 0 && o.precision != 1) return HYLU_ERR_ARG;
    if (!(o.heavy_ratio >= 0.0)) return HYLU_ERR_ARG;
    if (o.precision == 1 && o.refine == 0) o.refine = 1;
    hylu::AnalyzeOptions ao;
    ao.ordering = o.ordering == HYLU_ORDER_USER ? HYLU_ORDER_AMD : o.ordering;
    ao.static_pivot = o.static_pivot;
    ao.scale = o.scale;
    ao.sn_max = o.sn_max;
    ao.nd_leaf = o.nd_leaf > 0 ? o.nd_leaf : 256;
    ao.amd_dense = o.amd_dense > 0 ? o.amd_dense : 2.0;
    ao.heavy_ratio = o.heavy_ratio;
    std::vector<hylu::Plan> plans(k);
    std::vector<int> rcs(k, 0);
    unsigned nt = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), (unsigned)k));
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([&, t]() {
            for (int32_t s = (int32_t)t; s < k; s += (int32_t)nt) {
                rcs[s] = guarded([&] {
                    return hylu::analyze(n[s], rowptr[s], col[s], vals ? vals[s] : nullptr, nullptr, ao, plans[s]);
                });
            }
        });
    for (auto& t : th) t.join();
    for (int32_t s = 0; s < k; ++s) if (rcs[s]) return rcs[s];
    hylu_handle* h = new (std::nothrow) hylu_handle();
    if (!h) return HYLU_ERR_NOMEM;
    h->opt = o;
    h->batch = true;
    std::vector<const hylu::Plan*> ps;
    for (auto& p : plans) ps.push_back(&p);
    const int rc = guarded([&] {
        const int r = hylu::combine(ps, nsets, h->P, h->layout);
        if (r == 0) hylu::split_heavy_rows(h->P, ao.heavy_ratio);
        return r;
    });
    if (rc) { delete h; return rc < 0 ? rc : HYLU_ERR_INTERNAL; }
    *out = h;
    return HYLU_OK;
}

int hylu_batch_layout(hylu_handle* h, int32_t* row_base, int64_t* val_base, int32_t* total_n) {
    if (!h) return HYLU_ERR_ARG;
    if (!h->batch) return HYLU_ERR_STATE;
    if (row_base) std::memcpy(row_base, h->layout.row_base.data(), sizeof(int32_t) * h->layout.row_base.size());
    if (val_base) std::memcpy(val_base, h->layout.val_base.data(), sizeof(int64_t) * h->layout.val_base.size());
    if (total_n) *total_n = h->P.n;
    return HYLU_OK;
}

static int graph_capture_impl(hylu_handle* h, const double* d_vals, const double* d_b, double* d_x, int nrhs,
                              int ld, int corrections, void* stream) {
    if (!h || !d_vals || !d_b || !d_x || nrhs < 1 || ld < h->P.n) return HYLU_ERR_ARG;
    if (corrections < 0 || corrections > 16) return HYLU_ERR_ARG;
    if (!h->factored || nrhs > h->cap_rhs || (size_t)ld * nrhs > h->cap_elems) return HYLU_ERR_STATE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!st) return HYLU_ERR_ARG;   // the legacy default stream cannot be captured
    if (cudaStreamSynchronize(st) != cudaSuccess) return HYLU_ERR_CUDA;
    if (h->graph_exec) { cudaGraphExecDestroy(h->graph_exec); h->graph_exec = nullptr; }
    if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
    const int saved_refine = h->opt.refine;
    const int saved_timing = h->opt.timing;
    h->opt.refine = -1;
    h->opt.timing = 0;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        h->opt.refine = saved_refine; h->opt.timing = saved_timing;
        return HYLU_ERR_CUDA;
    }
    const int64_t l0 = hylu::launches();
    int rc = do_factor(h, d_vals, st);
    if (rc >= 0) rc = do_solve(h, d_b, d_x, nrhs, ld, st);
    // fixed refinement steps (Sec. 2.3) and the residual of the final x,
    // whose norms hylu_get_info reads after a replay
    for (int c = 0; rc >= 0 && c <= corrections; ++c) {
        rc = hylu::launch_residual(h->P.n, h->d_arp, h->d_aci, h->d_avals, d_x, d_b, h->d_r, h->d_norms, nrhs,
                                   ld, st);
        if (rc >= 0 && c < corrections)
            rc = hylu::launch_solve(h->dp, h->d_r, h->d_d, h->d_z, h->d_xh, h->d_rowperm, h->d_colperm, h->d_dr,
                                    h->d_dc, nrhs, ld, h->opt.spin_limit, h->solve_grid, st);
        if (rc >= 0 && c < corrections) rc = hylu::launch_axpy(h->P.n, d_x, h->d_d, nrhs, ld, st);
    }
    h->graph_launches = hylu::launches() - l0;
    hylu::add_launches(-h->graph_launches);  // recorded, not issued: replays count them
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(st, &g);
    h->opt.refine = saved_refine;
    h->opt.timing = saved_timing;
    if (rc < 0) { if (g) cudaGraphDestroy(g); return rc; }
    if (ce != cudaSuccess || !g) return HYLU_ERR_CUDA;
    h->graph = g;
    if (cudaGraphInstantiate(&h->graph_exec, g, 0) != cudaSuccess) return HYLU_ERR_CUDA;
    h->graph_corrections = corrections;
    h->graph_nrhs = nrhs;
    h->graph_norms_pending = false;
    return HYLU_OK;
}

int hylu_graph_capture(hylu_handle* h, const double* d_vals, const double* d_b, double* d_x, int nrhs, int ld,
                       int corrections, void* stream) {
    Range range_("hylu_graph_capture");
    return guarded([&] { return graph_capture_impl(h, d_vals, d_b, d_x, nrhs, ld, corrections, stream); });
}

int hylu_graph_launch(hylu_handle* h, void* stream) {
    Range range_("hylu_graph_launch");
    if (!h) return HYLU_ERR_ARG;
    if (!h->graph_exec) return HYLU_ERR_STATE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    h->last = st;
    // the captured launches count as the library's own launches
    hylu::add_launches(h->graph_launches);
    if (cudaGraphLaunch(h->graph_exec, st) != cudaSuccess) return HYLU_ERR_CUDA;
    h->graph_norms_pending = true;
    return HYLU_OK;
}

// Short timed trials on the handle's own values (Sec. 3.2's repeated mode
// makes them pay: the chosen point serves every later refactorization):
// blocks per SM of the factor launch, the heavy-row queue on or off at that
// grid, and blocks per SM of the substitution launches (right-hand sides of
// ones, as many as the handle's solves used, 1 to 8).  Each point is timed
// twice after a first untimed run.
static int tune_impl(hylu_handle* h, const double* d_vals, int* blocks_per_sm, void* stream) {
    if (!h || !d_vals) return HYLU_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TRY(do_factor(h, d_vals, st));   // uploads and allocates on first use
    if (h->P.n == 0) {               // empty system: no launch to tune
        if (blocks_per_sm) *blocks_per_sm = 1;
        return HYLU_OK;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    sms = std::max(1, sms);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto timed = [&](auto&& run, float* out) -> int {
        float tot = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, st);
            const int rc = run();
            cudaEventRecord(e1, st);
            if (rc < 0) return rc;
            if (cudaEventSynchronize(e1) != cudaSuccess) return HYLU_ERR_CUDA;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep) tot += ms;
        }
        *out = tot;
        return HYLU_OK;
    };
    int rc = HYLU_OK;
    // 1. factor grid (the tensor-core variant runs one block per SM: fixed)
    int best = h->grid / sms;
    if (h->dp.n_gd == 0) {
        const int maxper = std::max(1, h->grid_max / sms);
        float best_ms = 1e30f;
        for (int per = 1; per <= maxper && rc == HYLU_OK; ++per) {
            h->grid = sms * per;
            float ms = 0.f;
            rc = timed([&] { return do_factor(h, d_vals, st); }, &ms);
            if (ms < best_ms) { best_ms = ms; best = per; }
        }
        h->grid = sms * best;
    }
    // 2. heavy-row queue on or off
    const int32_t nheavy = (int32_t)h->P.heavy_order.size();
    if (rc == HYLU_OK && nheavy > 0) {
        float on = 0.f, off = 0.f;
        h->dp.n_heavy = nheavy;
        rc = timed([&] { return do_factor(h, d_vals, st); }, &on);
        if (rc == HYLU_OK) {
            h->dp.n_heavy = 0;
            rc = timed([&] { return do_factor(h, d_vals, st); }, &off);
        }
        h->heavy_off = (rc == HYLU_OK && off < on);
        h->dp.n_heavy = h->heavy_off ? 0 : nheavy;
    }
    // 3. substitution grid, with as many right-hand sides as the handle's
    //    solves have used so far (at least one, at most eight)
    const int nr = std::max(1, std::min(8, h->cap_rhs));
    const size_t nv = (size_t)h->P.n * nr;
    if (rc == HYLU_OK) rc = ensure_rhs(h, nr, h->P.n);
    double *b = nullptr, *x = nullptr;
    if (rc == HYLU_OK && (cudaMalloc(&b, sizeof(double) * nv) != cudaSuccess ||
                          cudaMalloc(&x, sizeof(double) * nv) != cudaSuccess))
        rc = HYLU_ERR_NOMEM;
    if (rc == HYLU_OK) {
        std::vector<double> ones(nv, 1.0);
        if (cudaMemcpy(b, ones.data(), sizeof(double) * nv, cudaMemcpyHostToDevice) != cudaSuccess)
            rc = HYLU_ERR_CUDA;
        // with the bulk-sequential segments of the handle's own solve_seq_rows,
        // and with every level in bulk (Sec. 2.3, Fig. 3)
        const int maxper = std::max(1, h->grid_max / sms);
        int sbest = h->solve_grid / sms;
        const int seq0 = h->opt.solve_seq_rows;
        int seq_best = seq0;
        float best_ms = 1e30f;
        std::vector<int> seqs = {seq0};
        if (seq0 > 0) seqs.push_back(0);
        for (int seq : seqs) {
            if (rc != HYLU_OK) break;
            rc = use_seq_segments(h, seq, st);
            for (int per = 1; per <= maxper && rc == HYLU_OK; ++per) {
                h->solve_grid = sms * per;
                float ms = 0.f;
                rc = timed([&] {
                    return hylu::launch_solve(h->dp, b, x, h->d_z, h->d_xh, h->d_rowperm, h->d_colperm, h->d_dr,
                                              h->d_dc, nr, h->P.n, h->opt.spin_limit, h->solve_grid, st);
                }, &ms);
                if (ms < best_ms) { best_ms = ms; sbest = per; seq_best = seq; }
            }
        }
        if (rc == HYLU_OK) rc = use_seq_segments(h, seq_best, st);
        h->solve_grid = sms * sbest;
    }
    if (b) cudaFree(b);
    if (x) cudaFree(x);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc < 0) return rc;
    h->tuned = 1;
    if (blocks_per_sm) *blocks_per_sm = best;
    TRY(do_factor(h, d_vals, st));   // leave the factors of d_vals at the chosen point
    return read_status(h, st);
}

int hylu_tune(hylu_handle* h, const double* d_vals, int* blocks_per_sm, void* stream) {
    Range range_("hylu_tune");
    return guarded([&] { return tune_impl(h, d_vals, blocks_per_sm, stream); });
}

int hylu_debug_trace(hylu_handle* h, unsigned long long* out) {
    if (!h || !out) return HYLU_ERR_ARG;
    if (!h->dp.trace) return HYLU_ERR_STATE;
    if (cudaStreamSynchronize(h->last) != cudaSuccess) return HYLU_ERR_CUDA;
    if (cudaMemcpy(out, h->dp.trace, sizeof(unsigned long long) * 4 * (size_t)h->P.n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return HYLU_ERR_CUDA;
    return HYLU_OK;
}

int hylu_debug_solve_trace(hylu_handle* h, unsigned long long* out) {
    if (!h || !out) return HYLU_ERR_ARG;
    if (!h->dp.strace) return HYLU_ERR_STATE;
    if (cudaStreamSynchronize(h->last) != cudaSuccess) return HYLU_ERR_CUDA;
    if (cudaMemcpy(out, h->dp.strace, sizeof(unsigned long long) * 2 * (size_t)h->P.nnodes, cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return HYLU_ERR_CUDA;
    return HYLU_OK;
}

int hylu_debug_occupancy(int* out4) {
    if (!out4) return HYLU_ERR_ARG;
    hylu::factor_occupancy(out4, out4 + 1, out4 + 2, out4 + 3);
    return HYLU_OK;
}

int hylu_debug_gemm(hylu_handle* h, int32_t* pair_cnt, int32_t* gd_done, int32_t* walk_done, int32_t* status,
                    int32_t* block_prog, int32_t* nblocks) {
    if (!h) return HYLU_ERR_ARG;
    const hylu::DevPlan& d = h->dp;
    if (!h->uploaded || d.n_gd == 0) return HYLU_ERR_STATE;
    if (cudaStreamSynchronize(h->last) != cudaSuccess) return HYLU_ERR_CUDA;
    auto get = [](int32_t* dst, const int32_t* src, size_t n) {
        return !dst || cudaMemcpy(dst, src, sizeof(int32_t) * n, cudaMemcpyDeviceToHost) == cudaSuccess;
    };
    if (!get(pair_cnt, d.pair_cnt, d.n_pair) || !get(gd_done, d.gd_done, d.n_gd) ||
        !get(walk_done, d.walk_done, h->P.n) || !get(status, d.status, hylu::ST_WORDS))
        return HYLU_ERR_CUDA;
    if (nblocks) *nblocks = d.gemm_prog ? d.gemm_blocks : 0;
    if (block_prog && d.gemm_prog && !get(block_prog, d.gemm_prog, 4 * (size_t)d.gemm_blocks)) return HYLU_ERR_CUDA;
    return HYLU_OK;
}

int hylu_plan_save(hylu_handle* h, void* buf, int64_t* bytes) {
    Range range_("hylu_plan_save");
    if (!h || !bytes) return HYLU_ERR_ARG;
    return guarded([&] {
        std::vector<uint8_t> img;
        TRY(hylu::save_plan(h->P, h->layout, h->batch, h->opt, img));
        const int64_t need = (int64_t)img.size();
        if (!buf) { *bytes = need; return HYLU_OK; }
        if (*bytes < need) { *bytes = need; return HYLU_ERR_ARG; }
        std::memcpy(buf, img.data(), img.size());
        *bytes = need;
        return HYLU_OK;
    });
}

int hylu_plan_load(const void* buf, int64_t bytes, const hylu_options* opt, hylu_handle** out) {
    Range range_("hylu_plan_load");
    if (!out || !buf || bytes <= 0) return HYLU_ERR_ARG;
    *out = nullptr;
    if (opt && opt->precision != 0 && opt->precision != 1) return HYLU_ERR_ARG;
    hylu_handle* h = new (std::nothrow) hylu_handle();
    if (!h) return HYLU_ERR_NOMEM;
    hylu_options saved;
    hylu_default_options(&saved);
    bool batch = false;
    const int rc = guarded([&] {
        return hylu::load_plan(static_cast<const uint8_t*>(buf), (size_t)bytes, h->P, h->layout, batch, saved);
    });
    if (rc) { delete h; return rc; }
    hylu_options o = saved;
    if (opt) {
        // numeric options from the caller; the analysis is the saved one
        o = *opt;
        if (o.precision == 1 && o.refine == 0) o.refine = 1;   // FP32 factors: always refine in FP64
        o.ordering = saved.ordering;
        o.static_pivot = saved.static_pivot;
        o.scale = saved.scale;
        o.sn_max = saved.sn_max;
        o.nd_leaf = saved.nd_leaf;
        o.amd_dense = saved.amd_dense;
        o.heavy_ratio = saved.heavy_ratio;
    }
    h->opt = o;
    h->batch = batch;
    *out = h;
    return HYLU_OK;
}

int hylu_measure_fp64_peak(double* gflops, void* stream) {
    if (!gflops) return HYLU_ERR_ARG;
    return hylu::measure_fp64_peak(gflops, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

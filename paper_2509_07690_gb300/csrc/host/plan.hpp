// Host-side plan of one sparsity pattern: preprocessing outputs (Sec. 2.1) and
// the node/task tables that drive the numeric kernels (Sec. 2.2, 2.2.1).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "preprocess.hpp"
#include "../../../include/hylu.h"

namespace hylu {

struct Plan {
    int32_t n = 0;
    int64_t nnz_a = 0;
    std::vector<int64_t> a_rp;          // original pattern (kept for the residual)
    std::vector<int32_t> a_ci;
    // static pivoting + scaling + ordering: Ahat(i,k) = dr[rowperm[i]] A(rowperm[i], colperm[k]) dc[colperm[k]]
    std::vector<int32_t> rowperm, colperm;
    std::vector<double> dr, dc;
    // Ahat, row by row: for each entry its slot in the node column list, the
    // index of its value in the caller's CSR array and its scale dr * dc
    std::vector<int64_t> ah_rp;
    std::vector<int32_t> ah_slot;
    std::vector<int64_t> ah_src;
    std::vector<double> ah_scale;
    // supernode partition; a node is a supernode or a standalone row
    std::vector<int32_t> sn_start;      // nnodes + 1, first row of each node
    int32_t nnodes = 0;
    std::vector<int32_t> node_of;       // row -> node
    // L part: each row's own sorted columns below its node (full supernode segments)
    std::vector<int64_t> row_lptr;      // n + 1 into lcols / the L values
    std::vector<int32_t> lcols;
    // U part: per node a dense panel of s rows x (s + |tail|) columns,
    // the diagonal block (columns r..e) then the shared U tail
    std::vector<int64_t> node_tail_off; // nnodes + 1 into tcols
    std::vector<int32_t> tcols;
    std::vector<int64_t> node_panel_off;// nnodes + 1 into the panel values
    int64_t nnz_l = 0, nnz_panel = 0, nnz_store = 0, nnz_f = 0;
    double flops_unpadded = 0.0, flops_padded = 0.0;
    // the padded flops by kernel (Sec. 2.2, Fig. 1): updates from standalone
    // source rows (row-row), from source supernodes into standalone rows
    // (sup-row) and into supernode rows (sup-sup), and each supernode row's
    // elimination against the earlier rows of its own diagonal block
    double flops_row_row = 0.0, flops_sup_row = 0.0, flops_sup_sup = 0.0, flops_in_sn = 0.0;
    std::vector<double> row_flops;      // padded flops of each row
    // tail tasks of the in-supernode step (Sec. 2.2, the triangular solve of
    // a supernode's U tail by its unit lower diagonal block): a supernode with
    // s > 1 rows and a tail gets node_ntask[D] tasks; task t solves the 32-column
    // groups task_chunk[t], + node_ntask, ... of node task_node[t]
    std::vector<int32_t> node_ntask, task_node, task_chunk, task_level;
    int32_t n_tasks = 0;
    // claim order of the factor kernel: rows (entries < n) and tail tasks
    // (entry n + t) sorted by dependency level.  A row depends on its source
    // nodes being complete (last row, or the node's tail tasks) and on the
    // diagonal-block step of the earlier rows of its own supernode; a tail
    // task on the diagonal-block step of its node's last row.
    std::vector<int32_t> row_order;
    // heavy rows (see split_heavy_rows), by level, and each row's rank there
    // (INT32_MAX for the others); the factor kernel claims the first ones from
    // a queue of their own
    std::vector<int32_t> heavy_order, heavy_rank;
    std::vector<int32_t> row_level;     // dependency level of every row
    int32_t row_levels = 0;
    // substitution schedules (bulk mode of Sec. 2.2.1 / 2.3): node levels of
    // the forward (L) and backward (U) dependency graphs, the rows in claim
    // order (level by level; backward descending inside a level) and the
    // number of nodes of every level
    std::vector<int32_t> fwd_order, bwd_order, fwd_level, bwd_level, fwd_count, bwd_count;
    // transpose substitution (U^T forward, then L^T backward), push form:
    // node levels, rows in claim order, rows per level
    std::vector<int32_t> ut_order, lt_order, ut_level, lt_level, ut_count, lt_count;
    // independent instances (a batch): every instance has its own level
    // watermark; node_inst maps a node to its instance (empty: one instance)
    // and the *_off arrays give each instance's slice of the per-level
    // count arrays above (empty: one slice, the whole array)
    std::vector<int32_t> node_inst, fwd_off, bwd_off, ut_off, lt_off;
    int32_t ordering = 0;               // HYLU_ORDER_* the plan was built with (AUTO: mixed batch)
    int32_t max_row = 0;                // longest row pattern (L + block + tail)
    int32_t max_sn = 1;
    double analyze_ms = 0.0;
    // analysis wall time by phase: matching and scaling, ordering, symbolic
    // factorization with the node tables and schedules, value map
    double analyze_phase_ms[4] = {0.0, 0.0, 0.0, 0.0};
    std::string error;
};

struct AnalyzeOptions {
    int ordering = 0;        // 0 AMD, 1 ND, 2 natural, 3 user, 4 the better of AMD and ND
    int static_pivot = 1;    // maximum-product matching
    int scale = 1;           // apply the matching's scalings
    int sn_max = 256;
    int nd_leaf = 256;
    double amd_dense = 2.0;
    double heavy_ratio = 32.0; // rows with this many times the mean row work are claimed first (0: off)
};

// Batch of independent systems (Sec. 3.2 repeated solves, extended to many
// patterns): instance q = v * k + s (value set v of system s) occupies rows
// [row_base[q], row_base[q] + n_s) of one block-diagonal plan; its values are
// read from the concatenated input at val_base[q].  node_base gives every
// node the first row of its instance; pos_n is the largest system.
struct BatchLayout {
    int32_t k = 0, nsets = 0, pos_n = 0;
    std::vector<int32_t> row_base, node_base;
    std::vector<int64_t> val_base;
};
int combine(const std::vector<const Plan*>& sys, int32_t nsets, Plan& C, BatchLayout& B);

// Returns 0 or a negative hylu status code; fills P.
int analyze(int32_t n, const int64_t* rp, const int32_t* ci, const double* v,
            const int32_t* user_perm, const AnalyzeOptions& opt, Plan& P);

// Picks the heavy rows: update work >= heavy_ratio x the mean row (and >= 1e6
// flops), of which at least half comes from sources at no more than half the
// row's own dependency level.  Fills heavy_order / heavy_rank from the
// level-ordered row_order.
void split_heavy_rows(Plan& P, double heavy_ratio);

// Unpadded structure of L and U (row i of the up-looking factorization):
// U(i, >=i) sorted, starting with i itself, and L(i, <i) as sorted, disjoint
// runs of consecutive columns [lrun_first, lrun_first + lrun_len).
struct SymbolicRows {
    std::vector<int64_t> urp;            // n + 1 into uci
    std::vector<int32_t> uci;
    std::vector<int64_t> lrp;            // n + 1 into the run arrays
    std::vector<int32_t> lrun_first, lrun_len;
    int64_t nnz_l = 0;                   // unpadded entries of L (strictly lower)
};

// Sequential part of the bulk-sequential substitution (Sec. 2.3, Fig. 3;
// seq_segments.cpp).  A level of one instance is light when it holds at most
// max_rows rows, no node larger than that, and at most 1024 max_rows entries
// of work (its rows' L lists or U tails plus its dense diagonal blocks);
// every maximal chain of two or more consecutive light levels is a segment,
// solved level after level by one thread block (0: no segments).
//   task      the bulk claim list: the rows outside the segments, in claim order
//   meta      per segment: instance, first level, last level (segments sorted
//             by first level)
//   seg_off   segments + 1, into the level table
//   lvl_row   level table + 1, into rows (a level's rows, node by node)
//   lvl_node  level table + 1, into snodes (a level's nodes of more than one row)
//   forward only: rows outside the segments with at least long_min L entries
//   have their lists split into chunks of about chunk_len entries (entries
//   [chunk_a, chunk_b) of row chunk_row); a chunk waits for level
//   chunk_level (one past its entries' highest source level); row_chunk_off
//   (n + 1) gives every row's chunks; the claim list holds chunk c as entry
//   n + c, before the rows of its level
struct SeqSegments {
    std::vector<int32_t> task, meta, seg_off, lvl_row, lvl_node, rows, snodes;
    std::vector<int32_t> chunk_row, chunk_a, chunk_b, chunk_level, row_chunk_off;
};
constexpr int32_t LONG_ROW_MIN = 2048;   // default long_min
constexpr int32_t LONG_ROW_CHUNK = 1024; // default chunk_len
void build_seq_segments(const Plan& P, bool backward, int32_t max_rows, SeqSegments& S,
                        int32_t long_min = LONG_ROW_MIN, int32_t chunk_len = LONG_ROW_CHUNK);

// Checkpoint of an analysis (serialize.cpp): the plan, the batch layout and
// the options as one flat byte image with a checksum, and back.  load_plan
// returns HYLU_ERR_PATTERN for an image that is not one (wrong magic,
// version or byte order, bad checksum, truncated, or sizes and index ranges
// that do not fit together).
int save_plan(const Plan& P, const BatchLayout& B, bool batch, const hylu_options& opt,
              std::vector<uint8_t>& out);
int load_plan(const uint8_t* buf, size_t bytes, Plan& P, BatchLayout& B, bool& batch, hylu_options& opt);

// Tensor-core tables of the precision form (gemm_plan.cpp).  A supernode of
// at least min_rows rows is a GEMM destination D.  Its rows
// walk their sources as other rows do, but for a large source supernode S
// (at least min_src = min(16, max(2, min_rows)) rows) a row only computes
// its multipliers L(i, S) (the triangular solve with S's diagonal block)
// and the updates that land in its own L part; the updates of D's diagonal
// block and U tail from S are the dense product
//     X_D[:, T_S >= r_D] -= L_{D,S} * U_{S, T_S >= r_D}
// computed by GEMM tasks on the tensor cores, one per (pair (D, S), 128-row
// M tile of D, 64-entry tile of S's tail) and added into D's panel.  Each
// row of D then takes its diagonal-block step in a task of its own (a
// "diag task") once its walk and D's GEMM tasks are done.
struct GemmPlan {
    static constexpr int TM = 128, TN = 64, TK = 32;
    int32_t ngd = 0, min_src = 0;
    std::vector<int32_t> gd_of_node;    // node -> destination, or -1
    std::vector<int32_t> gd_node;       // destination -> node
    std::vector<int32_t> gd_Kp, gd_Mp;  // A block of the destination: Mp rows x Kp columns
    std::vector<int64_t> gd_a_off;      // its start in each term array
    std::vector<int32_t> gd_ntask;      // GEMM tasks of the destination
    int64_t a_elems = 0;                // elements of one term array
    // pairs (destination, large source): A columns [u0, u0 + len) hold
    // L_{D,S} (u0 a multiple of TK), the source's tail entries jr .. jr + nj
    // are the ones at or past r_D, need = rows of D that hold S, and xmap
    // [x_off, x_off + nj) gives each of them its U-column index in D
    std::vector<int32_t> pair_gd, pair_src, pair_u0, pair_len, pair_jr, pair_nj, pair_need;
    std::vector<int64_t> pair_x_off;
    std::vector<int32_t> xmap;
    std::vector<int32_t> gd_slot;       // per L slot: the pair at the first slot of a large source
                                        // segment in a destination row, else -1
    // GEMM tasks in claim order (by level): pair, M tile, tail tile
    std::vector<int32_t> task_pair, task_mt, task_jt, task_level;
    // claim order of the rows' queue: rows (< n), tail tasks (n + t) and diag
    // tasks (n + n_tasks + d, the diagonal-block step of row diag_row[d])
    std::vector<int32_t> row_order, diag_row;
    std::vector<int32_t> walk_level, diag_level;   // per row (diag: destination rows only, else -1)
    int32_t levels = 0;
};
int build_gemm_plan(const Plan& P, int32_t min_rows, GemmPlan& G);

void symbolic_rows(const CsrPattern& ahat, SymbolicRows& F);
void supernode_partition(int32_t n, const SymbolicRows& F, int32_t sn_max, std::vector<int32_t>& start);
void build_nodes(Plan& P, const SymbolicRows& F);

}  // namespace hylu

// Device-side view of one factorization plan and the kernel entry points of
// the numeric phase (HYLU Sec. 2.2) and the substitution (Sec. 2.3).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hylu {


// Status words in device memory (int32):
//   [0] error code (0 or HYLU_ERR_DEVICE_TIMEOUT), [1] row/node where a wait
//   expired, [2] perturbed pivots, [3] task counter of the factor kernel,
//   [4] task counter of the forward solve, [5] of the backward solve,
//   [6..7] max |Ahat| as the bit pattern of a non-negative double.
//   [8..9] substitution: forward / backward claim counters ([10..11] unused).
//   [12] task counter of the factor kernel's heavy-row queue, [13] of its
//   tensor-core GEMM queue ([14..15] unused).
enum { ST_ERR = 0, ST_FAILED = 1, ST_NPERT = 2, ST_CNT_F = 3, ST_AMAX = 6, ST_CNT_FWD = 8,
       ST_CNT_BWD = 9, ST_ROLE_F = 10, ST_ROLE_B = 11, ST_CNT_H = 12, ST_CNT_G = 13, ST_SEG_F = 14,
       ST_SEG_B = 15, ST_WORDS = 16 };

// Segments of light levels of one substitution direction (the sequential
// mode of Sec. 2.3's bulk-sequential solve): per segment its instance, first
// and last level (meta), its levels (seg_off, into the level table), and per
// level its rows (lvl_row into rows) and its nodes of more than one row
// (lvl_node into snodes).
struct SegTable {
    const int32_t* meta;
    const int32_t* seg_off;
    const int32_t* lvl_row;
    const int32_t* lvl_node;
    const int32_t* rows;
    const int32_t* snodes;
    int32_t nseg;
};

struct DevPlan {
    int32_t n, nnodes;
    const int32_t* sn_start;       // nnodes + 1
    const int32_t* node_of;        // n
    const int64_t* row_lptr;       // n + 1
    const int32_t* lcols;          // nnz_l
    const int64_t* node_tail_off;  // nnodes + 1
    const int32_t* tcols;
    const int64_t* node_panel_off; // nnodes + 1
    double* lval;                  // nnz_l   : L(i, position) values
    double* pval;                  // nnz_panel: per node s x (s + tail), block by label
    float* lval32;                 // the same in FP32 (precision form), else null
    float* pval32;
    float* dinv32;
    const int64_t* ah_rp;          // n + 1 (rows of Ahat)
    const int32_t* ah_slot;
    const int64_t* ah_src;
    const double* ah_scale;
    int32_t* piv;                  // position -> label
    int32_t* pinv;                 // label -> position
    int32_t* ready;                // per row, factor generation: the row (for a supernode, the whole node) is final
    int32_t* dready;               // per supernode row: its diagonal-block step is done (pivot, multipliers)
    int32_t* node_done;            // per node: tail tasks finished (zeroed before each factor)
    const int32_t* node_ntask;     // per node: tail tasks (0: the rows publish themselves)
    const int32_t* task_node;      // per tail task: node
    const int32_t* task_chunk;     // per tail task: first 32-column group
    int32_t n_tasks;
    // substitution schedules (rows in level order, node levels, nodes per
    // level) and per-level completion counters (reset by every solve)
    const int32_t* fwd_order;
    const int32_t* bwd_order;
    const int32_t* fwd_level;
    const int32_t* bwd_level;
    const int32_t* fwd_count;
    const int32_t* bwd_count;
    int32_t* fwd_done;
    int32_t* bwd_done;
    int32_t n_fwd_levels, n_bwd_levels;
    const int32_t* ut_order;
    const int32_t* lt_order;
    const int32_t* ut_level;
    const int32_t* lt_level;
    const int32_t* ut_count;       // rows per level
    const int32_t* lt_count;
    int32_t* ut_done;
    int32_t* lt_done;
    int32_t n_ut_levels, n_lt_levels;     // lengths of the count / done arrays
    // instances with their own level watermarks (a batch; one otherwise):
    // node -> instance (null: all 0), each instance's slice of the count and
    // done arrays, and the forward / backward watermarks per instance
    const int32_t* node_inst;
    const int32_t* fwd_off;
    const int32_t* bwd_off;
    const int32_t* ut_off;
    const int32_t* lt_off;
    int32_t* wm_f;
    int32_t* wm_b;
    int32_t n_inst;
    // early parts of the substitution's dot products (null: none): forward,
    // row i's L entries [0, fwd_split[i]) have sources two or more levels
    // below the row's, so the row sums them once those levels are complete
    // and only the rest after the last level; backward, node D's tail
    // entries [bwd_split[D], nT) likewise (its late sources come first)
    const int32_t* fwd_split;
    const int32_t* bwd_split;
    // bulk-sequential substitution (Sec. 2.3, Fig. 3): the bulk claim lists
    // (rows outside the segments) and the segments of light levels, which the
    // first seq_blocks blocks to start claim and solve one after another
    const int32_t* fwd_task;
    const int32_t* bwd_task;
    int32_t n_fwd_tasks, n_bwd_tasks;
    SegTable fseg, bseg;
    int32_t seq_blocks;
    // forward solve, long rows: chunk c sums entries [fch_a, fch_b) of row
    // fch_row's L list once level fch_level is complete, writes fch_part[c]
    // (the factors' type) and publishes fch_flag[c]; frow_chunk_off (n + 1)
    // lists every row's chunks
    const int32_t* fch_row;
    const int32_t* fch_a;
    const int32_t* fch_b;
    const int32_t* fch_level;
    const int32_t* frow_chunk_off;
    double* fch_part;
    int32_t* fch_flag;
    int32_t* fwd_row;              // per row of a supernode, solve generation
    int32_t* bwd_row;
    int32_t* tile_f;               // per 32-row tile of a supernode block (at its owner row):
    int32_t* tile_b;               //   solved in the forward / backward substitution
    int32_t* pos;                  // per-warp column -> slot maps, pos_n each
    int32_t pos_n;                 // largest system of the plan (n for one system)
    const int32_t* node_base;      // per node: first row of its instance (null = 0)
    double* spa64;                 // per-warp dense L vectors (pos_n each) for long L lists,
    float* spa32;                  // in the factor precision; null when no row needs one
    double* dinv;                  // 1 / u_ii by position (row)
    const int32_t* row_order;      // claim order of the factor kernel (by level)
    const int32_t* heavy_order;    // heavy rows by level (claimed first), null if none
    const int32_t* heavy_rank;     // per row: rank in heavy_order, INT32_MAX if not heavy
    int32_t n_heavy;
    // precision form, tensor-core sup-sup update (GemmPlan on the host;
    // n_gd == 0: off).  The factor launch is then gemm_blocks blocks (one
    // per SM), each with row warps and one warpgroup that runs the GEMM
    // tasks; the rows' queue also holds n_diag diag tasks.
    int32_t n_gd, n_gtask, n_diag, gemm_blocks, n_pair;
    int64_t a_elems;               // elements of each split-term array
    const int32_t* gd_of_node;     // node -> destination, or -1
    const int32_t* gd_node;
    const int32_t* gd_Kp;
    const int64_t* gd_a_off;
    const int32_t* gd_ntask;
    const int32_t* pair_gd;
    const int32_t* pair_src;
    const int32_t* pair_u0;
    const int32_t* pair_jr;
    const int32_t* pair_nj;
    const int32_t* pair_need;
    const int64_t* pair_x_off;
    const int32_t* xmap;
    const int32_t* gd_slot;        // per L slot: pair at the first slot of a large source segment, else -1
    const int32_t* gt_pair;        // GEMM tasks in claim order
    const int32_t* gt_mt;
    const int32_t* gt_jt;
    const int32_t* diag_row;       // diag task d: the diagonal-block step of this row
    int32_t* pair_cnt;             // rows that wrote their multipliers for the pair (zeroed per factor)
    int32_t* gd_done;              // GEMM tasks finished per destination (zeroed per factor)
    int32_t* walk_done;            // per row: walk finished (factor generation)
    uint16_t* a_term[3];           // L_{D,S} split into three BF16 terms (raw bits), per destination
                                   //   an Mp x Kp row-major block (zeroed per factor)
    const void* tmaps;             // TMA tensor maps, 3 per destination (term-major inside), device memory
    int32_t* gemm_prog;            // diagnostics (debug & 2): per GEMM block, task / stage / chunk / tries
    unsigned long long* trace;     // optional: 4 words per row (claim, external done, published, waits / node complete)
    unsigned long long* strace;    // optional: per node, forward and backward substitution completion times
    int32_t* status;
    // [0] factor generation, [1] substitution generation: the flags above
    // compare against them.  The first kernel of every factor / substitution
    // bumps its word on the device, so a replayed CUDA graph advances them too.
    int32_t* gens;
};

int launch_factor(const DevPlan& P, const double* d_vals, int64_t nnz_a,
                  double tau_rel, long long spin_limit, int grid, cudaStream_t st,
                  cudaEvent_t e0 = nullptr, cudaEvent_t e1 = nullptr);
int launch_solve(const DevPlan& P, const double* d_b, double* d_x, double* d_z, double* d_xh,
                 const int32_t* rowperm, const int32_t* colperm, const double* dr, const double* dc,
                 int nrhs, int ld, long long spin_limit, int grid, cudaStream_t st,
                 cudaEvent_t e0 = nullptr, cudaEvent_t e1 = nullptr);
int launch_solve_transpose(const DevPlan& P, const double* d_b, double* d_x, double* d_h,
                           const int32_t* rowperm, const int32_t* colperm, const double* dr, const double* dc,
                           int nrhs, int ld, long long spin_limit, int grid, cudaStream_t st);
int launch_residual_transpose(int32_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* y,
                              const double* g, double* r, double* colsum, double* norms, int nrhs, int ld,
                              cudaStream_t st);
int launch_grad_values(int32_t n, const int64_t* rp, const int32_t* ci, const double* lam, const double* x,
                       double* dvals, int nrhs, int ld, cudaStream_t st);
int launch_residual(int32_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* x,
                    const double* b, double* r, double* norms, int nrhs, int ld, cudaStream_t st);
int launch_axpy(int32_t n, double* x, const double* d, int nrhs, int ld, cudaStream_t st);
int launch_reset(int32_t* status, int32_t* piv, int32_t* pinv, int32_t* gens, int32_t n, cudaStream_t st);
int factor_grid(int device, bool fp32 = false);   // blocks of the persistent kernels
int warps_per_block();
int dense_l_min();
int64_t launches();
int measure_fp64_peak(double* gflops, cudaStream_t st);
bool tensor_maps_available();  // the driver's TMA tensor-map encoder was found
// Encode the tensor maps of the split multipliers: for destination g and term
// s, an Mp[g] x Kp[g] BF16 block at a_term[s] + a_off[g], boxes of 8 x 128;
// written to host memory `out` (3 per destination, 128 bytes each).
int encode_a_maps(int32_t ngd, const int32_t* Mp, const int32_t* Kp, const int64_t* a_off, uint16_t* const* a_term,
                  void* out);
size_t tensor_map_bytes();
int gemm_smem_fits();          // the tile engine fits the factor kernel's shared memory
void factor_occupancy(int* per64, int* per32, int* per_tc, int* regs_tc);
int tc_grid(int device);       // blocks of the tensor-core variant of the factor launch (0: it cannot run)
void count_launch();
void add_launches(int64_t k);

}  // namespace hylu

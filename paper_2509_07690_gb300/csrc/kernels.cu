// Numeric factorization and substitution kernels for sm_103a (HYLU Sec. 2.2,
// 2.2.1 and 2.3).
//
// Factorization: one persistent kernel whose warps claim tasks from two
// dependency-level-ordered queues (heavy rows first on two warps of every
// block, everything else from the main queue).  A row task runs the
// up-looking update of its row (Sec. 2.2, Fig. 1):
//   - Ahat(i,:) is scattered (scaled) straight into the row's storage;
//   - each source in the row's L list, in ascending order, is waited for on
//     its ready flag and applied: a standalone source row is a row-row update
//     (one multiplier, a sparse axpy over its U tail), a source supernode is
//     a sup-row update (a triangular solve with its dense diagonal block, then
//     a dense matrix-vector product with its U tail);
//   - a row inside a supernode then takes the diagonal-block updates of the
//     earlier rows of its own supernode as soon as each is published (the
//     pipelined mode of Sec. 2.2.1 at row granularity), exchanges the largest
//     entry of its diagonal block to the diagonal (supernode diagonal
//     pivoting) and perturbs a pivot below tau (Sec. 2.2);
//   - the supernode's U tail is then solved by the unit lower diagonal block
//     in tail tasks (or by the last row for a small node), which publish the
//     node; a standalone row publishes itself.
// A claimed task waits only on tasks of lower levels, so the schedule cannot
// deadlock; every wait is still bounded by an iteration limit and reports
// HYLU_ERR_DEVICE_TIMEOUT.
//
// Storage: row i's L values (by position) are contiguous; every node (a
// supernode or a standalone row) keeps a dense panel s x (s + |tail|) whose
// diagonal block is stored by column LABEL (pre-pivot column), so that later
// exchanges never move data; consumers read position p through piv[p].
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdio>

#include <cuda.h>

#include "kernels.cuh"
#include "tc_gemm.cuh"
#include "../../include/hylu.h"

namespace hylu {

namespace {
constexpr int WARPS = 8;          // warps per block of the persistent kernels
constexpr int SN_SMEM = 256;      // largest supernode held in shared memory
constexpr unsigned FULL = 0xffffffffu;
std::atomic<int64_t> g_launches{0};   // kernels issued (host threads may drive separate handles)

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int atom_add_acq_rel(int* p, int v) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// All lanes wait (bounded) until *flag == gen.  Returns false when the limit
// expired or another warp already raised an error; the first expiry records
// HYLU_ERR_DEVICE_TIMEOUT and the row/node waited on.
__device__ __forceinline__ bool warp_wait(const int* flag, int gen, int* status, int who,
                                          long long limit, unsigned long long* waited = nullptr) {
    int ok = 1;
    unsigned long long t0 = 0;
    if (waited) asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t0));
    if (ld_acquire(flag) != gen) {
        long long it = 0;
        for (;;) {
            if (ld_acquire(flag) == gen) break;
            if (++it > limit) {
                if (atomicCAS(status + ST_ERR, 0, HYLU_ERR_DEVICE_TIMEOUT) == 0) status[ST_FAILED] = who;
                ok = 0;
                break;
            }
            if ((it & 255) == 0 && ld_relaxed(status + ST_ERR) != 0) { ok = 0; break; }
            if (it > 16) __nanosleep(64);
        }
    }
    if (waited) {
        unsigned long long t1;
        asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t1));
        *waited += t1 - t0;
    }
    return __all_sync(FULL, ok) != 0;
}

// All lanes wait (bounded) until *cnt >= target (a counter zeroed before the
// launch); errors as for warp_wait.
__device__ __forceinline__ bool warp_wait_ge(const int* cnt, int target, int* status, int who, long long limit) {
    int ok = 1;
    long long it = 0;
    while (ld_acquire(cnt) < target) {
        if (++it > limit) {
            if (atomicCAS(status + ST_ERR, 0, HYLU_ERR_DEVICE_TIMEOUT) == 0) status[ST_FAILED] = who;
            ok = 0;
            break;
        }
        if ((it & 255) == 0 && ld_relaxed(status + ST_ERR) != 0) { ok = 0; break; }
        if (it > 16) __nanosleep(64);
    }
    return __all_sync(FULL, ok) != 0;
}

// -------------------------------------------------------------- reset
__global__ void reset_kernel(int32_t* piv, int32_t* pinv, int32_t n, int32_t* gens) {
    if (blockIdx.x == 0 && threadIdx.x == 0) gens[0] += 1;   // factor generation of this call
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        piv[i] = i;
        pinv[i] = i;
    }
}

// max |Ahat| (the bit pattern of a non-negative double orders like an integer)
__global__ void amax_kernel(const double* __restrict__ vals, const int64_t* __restrict__ src,
                            const double* __restrict__ scale, int64_t nnz, int32_t* status) {
    double m = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz;
         q += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(vals[src[q]] * scale[q]));
    for (int off = 16; off; off >>= 1) m = fmax(m, __shfl_down_sync(FULL, m, off));
    if ((threadIdx.x & 31) == 0 && m > 0.0)
        atomicMax(reinterpret_cast<unsigned long long*>(status + ST_AMAX),
                  (unsigned long long)__double_as_longlong(m));
}

// Factor values of the plan in precision T (FP64 or the FP32 form).
template <typename T> __device__ __forceinline__ T* LV(const DevPlan& P);
template <typename T> __device__ __forceinline__ T* PV(const DevPlan& P);
template <> __device__ __forceinline__ double* LV<double>(const DevPlan& P) { return P.lval; }
template <> __device__ __forceinline__ double* PV<double>(const DevPlan& P) { return P.pval; }
template <> __device__ __forceinline__ float* LV<float>(const DevPlan& P) { return P.lval32; }
template <> __device__ __forceinline__ float* PV<float>(const DevPlan& P) { return P.pval32; }
template <typename T> __device__ __forceinline__ T* SPA(const DevPlan& P);
template <> __device__ __forceinline__ double* SPA<double>(const DevPlan& P) { return P.spa64; }
template <> __device__ __forceinline__ float* SPA<float>(const DevPlan& P) { return P.spa32; }
template <typename T> __device__ __forceinline__ T* DI(const DevPlan& P);
template <> __device__ __forceinline__ double* DI<double>(const DevPlan& P) { return P.dinv; }
template <> __device__ __forceinline__ float* DI<float>(const DevPlan& P) { return P.dinv32; }

// -------------------------------------------------------------- factor
// Per-warp shared memory of the factor kernel.
constexpr int FWARPS = 4;          // warps per block of the factor kernel (one per SM sub-partition)
constexpr int PANEL_BYTES = 4096;  // U part of the row being updated
constexpr int PF = 16;             // leading tail entries prefetched per source
constexpr int UNR = 8;             // independent 32-entry batches in flight
constexpr int UNR_TAIL = 8;        // the same for the tails of standalone sources
constexpr int DENSE_L_MIN = 256;   // rows with longer L lists use the dense per-warp L vector
constexpr int HEAVY_WPB = 2;       // warps of every block that take the heavy rows first
template <typename T>
struct WarpSmem {
    T lb[SN_SMEM];            // source supernode: l by position
    int pb[SN_SMEM];               // source supernode: label offset of each position
    T win[32];                     // x for the 32 L slots of the current window
    int wcol[32];                  // their columns
    int plen[32];                  // per window source: tail entries inside the window
    int pfc[32][PF];               // per window source: its first PF tail columns
    T pfu[32][PF];                 //                    and values
    __align__(16) unsigned char panel[PANEL_BYTES];
};
template <typename T>
constexpr size_t factor_smem() { return sizeof(WarpSmem<T>) * FWARPS; }
// The precision form with tensor-core sup-sup tasks: a kernel holding
// tcgen05 instructions gets one block per SM, so that variant runs one large
// block per SM: TC_ROWW row warps, then one warpgroup of 4 GEMM warps.
constexpr int TC_ROWW = 16;

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int bsearch_sm(const int* a, int m, int c) {
    int lo = 0, hi = m - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < c) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Where the row's U part (diagonal block + tail) lives while it is updated:
//   mode 0: shared memory, dense over columns r .. maxcol (index c - r)
//   mode 1: shared memory, block then tail slots; tail found by binary search
//   mode 2: the row's own panel storage in global memory (index by slot)
template <typename T>
struct Panel {
    T* x;
    const int* scols;
    int mode, r, e, s, nL, nT;
    __device__ __forceinline__ int idx(const int* pos, int c) const {
        if (mode == 0 || c <= e) return c - r;
        if (mode == 1) return s + bsearch_sm(scols, nT, c);
        return pos[c] - nL;
    }
    __device__ __forceinline__ int tail_idx(const int* tc, int j) const {
        return mode == 0 ? tc[j] - r : s + j;
    }
};

// Update x with entries j in [j0, nTS) of a standalone source's tail, all with
// multiplier l; entries with columns below r go to the L part (atomic adds to
// global memory: no one reads them before the window moves past them and a
// fence is taken), the others to the panel (by reductions when atomic_u is
// set: the row of a GEMM destination, whose panel the tensor-core tasks add
// to as well), or, when spau is set (a row with a dense L vector and a panel
// in global memory), to the dense vector by column as well.  Loads of UNR batches are issued before any update so that
// their latencies overlap.
template <typename T>
__device__ __forceinline__ void apply_tail(const int32_t* __restrict__ tcS, const T* __restrict__ U1,
                                           int j0, int nTS, T l, int r, const int* pos, T* xl, T* spa,
                                           T* spau, const Panel<T>& pn, int lane, bool atomic_u = false) {
    for (int jb = j0; jb < nTS; jb += 32 * UNR_TAIL) {
        int c[UNR_TAIL];
        T u[UNR_TAIL];
#pragma unroll
        for (int m = 0; m < UNR_TAIL; ++m) {
            const int j = jb + m * 32 + lane;
            c[m] = (j < nTS) ? __ldg(tcS + j) : -1;
            u[m] = (j < nTS) ? U1[j] : T(0);   // written in this launch: coherent loads
        }
        int ix[UNR_TAIL];
#pragma unroll
        for (int m = 0; m < UNR_TAIL; ++m)
            ix[m] = (c[m] >= r) ? (spau ? -1 : pn.idx(pos, c[m])) : ((c[m] >= 0 && !spa) ? pos[c[m]] : -1);
#pragma unroll
        for (int m = 0; m < UNR_TAIL; ++m) {
            if (c[m] < 0) continue;
            if (c[m] < r) atomicAdd(spa ? spa + c[m] : xl + ix[m], -l * u[m]);
            else if (spau) atomicAdd(spau + c[m], -l * u[m]);
            else if (atomic_u) atomicAdd(pn.x + ix[m], -l * u[m]);
            else pn.x[ix[m]] -= l * u[m];
        }
    }
}

// Tail of a supernode (the in-supernode step, Sec. 2.2), 32-column groups
// g0, g0 + gstep, ...  Once the node's diagonal block is factored (every
// row's pivot and multipliers known), its U tail is U_T = L_DD^-1 X_T: X_T
// the rows' tails after the updates from earlier nodes, L_DD the unit lower
// multipliers by position (row q keeps l_qk at the label of position k).
// Lanes own tail columns and hold a block of rows of their column in
// registers: first the finished rows above the block (8 at a time,
// multipliers staged in shared memory), then the triangle inside the block,
// so every entry takes its updates in ascending k as in the row-by-row
// elimination.
template <typename T>
__device__ __noinline__ void tail_solve(const DevPlan& P, int D, int g0, int gstep, WarpSmem<T>* ws, int lane) {
    const int r = P.sn_start[D], e = P.sn_start[D + 1] - 1, s = e - r + 1;
    const int nT = (int)(P.node_tail_off[D + 1] - P.node_tail_off[D]);
    const int64_t w = s + nT;
    const T* Ub = PV<T>(P) + P.node_panel_off[D];
    T* Uw = PV<T>(P) + P.node_panel_off[D];
    int* pb = ws->pb;
    // rows per register block (16 keeps the task within the kernel's 128
    // registers); RB x RB staging area: the prefetch buffers and the panel,
    // unused here
    constexpr int RB = 16;
    T* Ls = reinterpret_cast<T*>(&ws->pfu[0][0]);
    static_assert(sizeof(ws->pfu) + PANEL_BYTES >= RB * RB * sizeof(T), "staging area");
    for (int q = lane; q < s; q += 32) pb[q] = P.piv[r + q] - r;
    __syncwarp();
    for (int g = g0; g * 32 < nT; g += gstep) {
        const int j = g * 32 + lane;
        const bool on = j < nT;
        T* col = Uw + s + (on ? j : 0);
        for (int q0 = 0; q0 < s; q0 += RB) {
            const int m = min(RB, s - q0);
            T x[RB];
#pragma unroll
            for (int u = 0; u < RB; ++u) x[u] = (on && u < m) ? col[(int64_t)(q0 + u) * w] : T(0);
            for (int k0 = 0; k0 < q0; k0 += 8) {
                __syncwarp();
                for (int idx = lane; idx < 8 * RB; idx += 32) {
                    const int kk = idx / RB, u = idx % RB;
                    Ls[idx] = (u < m) ? Ub[(int64_t)(q0 + u) * w + pb[k0 + kk]] : T(0);
                }
                T uk[8];
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) uk[kk] = on ? col[(int64_t)(k0 + kk) * w] : T(0);
                __syncwarp();
#pragma unroll
                for (int u = 0; u < RB; ++u) {
                    if (u >= m) break;   // m is the same in every lane
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) x[u] -= Ls[kk * RB + u] * uk[kk];
                }
            }
            __syncwarp();
            for (int idx = lane; idx < RB * RB; idx += 32) {
                const int u = idx / RB, v = idx % RB;
                Ls[idx] = (v < u && u < m) ? Ub[(int64_t)(q0 + u) * w + pb[q0 + v]] : T(0);
            }
            __syncwarp();
#pragma unroll
            for (int u = 1; u < RB; ++u) {
                if (u >= m) break;
                T a = x[u];
#pragma unroll
                for (int v = 0; v < u; ++v) a -= Ls[u * RB + v] * x[v];
                x[u] = a;
            }
#pragma unroll
            for (int u = 0; u < RB; ++u)
                if (on && u < m) col[(int64_t)(q0 + u) * w] = x[u];
        }
    }
}

// One tail task: waits for the node's last diagonal-block step, solves its
// column groups, and the node's last task to finish publishes every row.
template <typename T>
__device__ bool tail_task(const DevPlan& P, int t, int gen, long long limit, WarpSmem<T>* ws, int lane) {
    const int D = P.task_node[t];
    const int nck = P.node_ntask[D];
    const int r = P.sn_start[D], e = P.sn_start[D + 1] - 1;
    if (!warp_wait(P.dready + e, gen, P.status, e, limit)) return false;
    tail_solve<T>(P, D, P.task_chunk[t], nck, ws, lane);
    __threadfence();
    __syncwarp();
    if (lane == 0 && atom_add_acq_rel(P.node_done + D, 1) == nck - 1) {
        for (int k = r; k <= e; ++k) st_release(P.ready + k, gen);
        if (P.trace) P.trace[4 * (int64_t)e + 3] = gtimer();   // node complete
    }
    __syncwarp();
    return true;
}


// ------------------------------------------------ tensor-core sup-sup tasks
// P.gemm_blocks blocks of the precision-form factor launch run the GEMM tasks (Sec. 2.2, Fig. 1c, sup-sup): for a pair (destination D, source
// supernode S), one 128-row tile of D and 64 entries of S's tail at or past
// D's first row,
//     X_D[rows, T_S cols] -= L_{D,S}[rows, :] * U_{S, T_S cols}
// with L_{D,S} (the multipliers D's rows computed and split into three BF16
// terms) loaded by TMA, U_{S,.} (final: the rows waited for S) gathered from
// S's panel and split on the way, the products on the tensor cores (6 term
// products, FP32 accumulation in TMEM), and the result added into D's panel
// rows at the U-column index of each tail entry (FP32 reductions: the rows
// add their updates from small sources to the same entries).  A task waits,
// bounded, until every row of D that holds S has written its multipliers;
// the last task of D lets D's diag tasks start.  The first blocks of the
// launch to start take this role (an atomic ticket, not the block index):
// the rows wait on these tasks, so they must be among the resident blocks.
struct GemmSmem {
    tc::TileSmem<3> t;
    int xm[tc::TN];      // U-column index in D of the tile's tail entries
    int task;
};

// the GEMM warpgroup's own barrier (the block's row warps never join it)
__device__ __forceinline__ void gemm_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__device__ __noinline__ void gemm_role(const DevPlan& P, unsigned char* smem_raw, int rank, int tid,
                                       long long limit) {
    const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023);
    GemmSmem& G = *reinterpret_cast<GemmSmem*>(base);
    tc::TileSmem<3>& sm = G.t;
    // warps of the group are the block's last four: warp % 4 gives the TMEM
    // lane quarter each may read, rows warp*32 .. of the tile
    const int warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        tc::mbar_init(&sm.bar_tma, 1);
        tc::mbar_init(&sm.bar_mma, 1);
        tc::mbar_fence_init();
        sm.abort = 0;
    }
    if (warp == 0) tc::tmem_alloc(&sm.tmem_base, tc::TMEM_COLS);
    tc::tc_fence_before();
    gemm_bar();
    tc::tc_fence_after();
    const uint32_t tmem = sm.tmem_base;
    const CUtensorMap* maps = static_cast<const CUtensorMap*>(P.tmaps);
    // an mbarrier try_wait may suspend for a while by itself: fewer tries
    const long long mlimit = limit < (1LL << 22) ? limit : (1LL << 22);
    uint32_t ph_tma = 0, ph_mma = 0;
    int32_t* prog = P.gemm_prog ? P.gemm_prog + 4 * rank : nullptr;
    auto stage = [&](int st, int c) {
        if (prog && tid == 0) { prog[1] = st; prog[2] = c; __threadfence(); }
    };
    for (;;) {
        if (tid == 0) {
            int q = atomicAdd(P.status + ST_CNT_G, 1);
            if (prog) { prog[0] = q; prog[1] = 1; prog[2] = 0; prog[3] = (int32_t)(gtimer() >> 10); }
            if (q >= P.n_gtask || ld_relaxed(P.status + ST_ERR) != 0) q = -1;
            G.task = q;
            if (q >= 0) {
                // every row of D that holds S has written L_{D,S}
                const int p = P.gt_pair[q];
                const int need = P.pair_need[p];
                long long it = 0;
                while (ld_acquire(P.pair_cnt + p) < need) {
                    if (++it > limit || ld_relaxed(P.status + ST_ERR) != 0) {
                        if (atomicCAS(P.status + ST_ERR, 0, HYLU_ERR_DEVICE_TIMEOUT) == 0)
                            P.status[ST_FAILED] = P.gd_node[P.pair_gd[p]];
                        G.task = -1;
                        break;
                    }
                    __nanosleep(64);
                }
                // the multipliers were written through the generic proxy;
                // the tensor copies below read them through the async proxy
                asm volatile("fence.proxy.async.global;" ::: "memory");
                // the tensor maps were copied to global memory by the host:
                // make them visible to the tensor-map proxy before use
                const CUtensorMap* mp = maps + 3 * P.pair_gd[p];
                for (int s = 0; s < 3; ++s)
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                                     reinterpret_cast<uint64_t>(mp + s))
                                 : "memory");
            }
        }
        gemm_bar();
        const int q = G.task;
        if (q < 0) break;
        stage(2, 0);
        const int p = P.gt_pair[q], mt = P.gt_mt[q], jt = P.gt_jt[q];
        const int g = P.pair_gd[p], D = P.gd_node[g], S = P.pair_src[p];
        const int rD = P.sn_start[D], sD = P.sn_start[D + 1] - rD;
        const int wD = sD + (int)(P.node_tail_off[D + 1] - P.node_tail_off[D]);
        const int rS = P.sn_start[S], sS = P.sn_start[S + 1] - rS;
        const int wS = sS + (int)(P.node_tail_off[S + 1] - P.node_tail_off[S]);
        const int nj = min(tc::TN, P.pair_nj[p] - jt * tc::TN);
        const int j0 = sS + P.pair_jr[p] + jt * tc::TN;     // panel column of the tile's first entry
        const float* US = P.pval32 + P.node_panel_off[S];
        float* XD = P.pval32 + P.node_panel_off[D];
        if (tid < tc::TN) G.xm[tid] = tid < nj ? P.xmap[P.pair_x_off[p] + jt * tc::TN + tid] : 0;
        const int nch = (sS + tc::TK - 1) / tc::TK;
        const int u0 = P.pair_u0[p];
        bool ok = true;
        for (int c = 0; c < nch; ++c) {
            if (tid == 0) {
                tc::mbar_expect_tx(&sm.bar_tma, 3 * tc::A_TERM_BYTES);
                for (int s = 0; s < 3; ++s)
                    for (int j = 0; j < tc::TK / tc::KB; ++j)
                        tc::tma_load_2d(&sm.a[s][j * tc::KB * tc::TM], maps + 3 * g + s,
                                        u0 + c * tc::TK + j * tc::KB, mt * tc::TM, &sm.bar_tma);
            }
            stage(3, c);
            // B: positions c*TK .. of S (rows of its panel), the tile's tail entries
            for (int e2 = tid; e2 < tc::TK * tc::TN; e2 += 128) {
                const int k = e2 / tc::TN, t = e2 % tc::TN;
                const int pk = c * tc::TK + k;
                const float v = (pk < sS && t < nj) ? __ldcg(US + (int64_t)pk * wS + j0 + t) : 0.f;
                __nv_bfloat16 h3[3];
                tc::split_bf16<3>(v, h3);
                for (int s = 0; s < 3; ++s)
                    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(sm.b[s]) + tc::b_off(t, k)) = h3[s];
            }
            tc::fence_async_smem();
            gemm_bar();
            stage(4, c);
            if (tid == 0) {
                if (!tc::mbar_wait(&sm.bar_tma, ph_tma, mlimit)) {
                    sm.abort = 1;
                    atomicCAS(P.status + ST_ERR, 0, HYLU_ERR_DEVICE_TIMEOUT);
                    tc::mbar_wait(&sm.bar_tma, ph_tma, mlimit);     // copies still in flight
                } else {
                    tc::tc_fence_after();
                    tc::issue_chunk<3>(sm, tmem, c == 0);
                    tc::mma_commit(&sm.bar_mma);
                }
            }
            ph_tma ^= 1u;
            stage(5, c);
            gemm_bar();
            if (sm.abort) { ok = false; break; }
            if (!tc::mbar_wait(&sm.bar_mma, ph_mma, mlimit)) {
                if (tid == 0) atomicCAS(P.status + ST_ERR, 0, HYLU_ERR_DEVICE_TIMEOUT);
                tc::mbar_wait(&sm.bar_mma, ph_mma, mlimit);
                sm.abort = 1;
            }
            ph_mma ^= 1u;
            stage(6, c);
            gemm_bar();
            if (sm.abort) { ok = false; break; }
        }
        if (!ok) break;
        stage(7, 0);
        // epilogue: this warp's 32 TMEM lanes are rows mt*128 + warp*32 + lane
        tc::tc_fence_after();
        const int m = mt * tc::TM + warp * 32 + lane;
        for (int jj = 0; jj < tc::TN / 16; ++jj) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(jj * 16), v);
            if (m < sD) {
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int t = jj * 16 + u;
                    if (t < nj) atomicAdd(XD + (int64_t)m * wD + G.xm[t], -v[u]);
                }
            }
        }
        tc::tc_fence_before();
        gemm_bar();
        if (tid == 0) {
            __threadfence();
            atomicAdd(P.gd_done + g, 1);
        }
        stage(8, 0);
    }
    tc::tc_fence_before();
    gemm_bar();
    if (warp == 0) tc::tmem_dealloc(tmem, tc::TMEM_COLS);
}

// RW row warps per block; TC: the block's last four warps run the GEMM
// tasks (the tensor-core variant of the precision form, one block per SM).
template <typename T, int RW, bool TC>
__global__ void __launch_bounds__((RW + (TC ? 4 : 0)) * 32, TC ? 1 : 4)
factor_kernel(DevPlan P, const double* __restrict__ vals, T* __restrict__ dinv,
              double tau_rel, long long limit) {
    const int gen = P.gens[0];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if constexpr (TC) {
        if ((int)(threadIdx.x >> 5) >= RW) {
            gemm_role(P, smem_raw + sizeof(WarpSmem<T>) * RW, blockIdx.x, threadIdx.x - RW * 32, limit);
            return;
        }
    }
    const int nrowblk = (int)gridDim.x;
    constexpr int HW = HEAVY_WPB * RW / FWARPS;   // warps of every block that take the heavy rows first
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpSmem<T>* ws = reinterpret_cast<WarpSmem<T>*>(smem_raw) + wid;
    T* lb = ws->lb;
    int* pb = ws->pb;
    T* win = ws->win;
    int* wcol = ws->wcol;
    int* pos_warp = P.pos + (size_t)(blockIdx.x * RW + wid) * (size_t)P.pos_n;
    const double amax = __longlong_as_double(*reinterpret_cast<const long long*>(P.status + ST_AMAX));
    const double tau = tau_rel * amax;
    // Rows are claimed from two queues, each in dependency-level order.  The
    // heavy rows form a queue of their own, served first by HEAVY_WPB warps of
    // every block (spread over all SMs: a heavy row is bound by its
    // sub-partition's FP64 pipe) and by any warp that finds the main queue
    // drained; every other row comes from the level-ordered main queue, which
    // skips the heavy rows.  Progress holds: a claimed row waits only on rows
    // of lower levels, and the lowest-level unfinished row is either claimed,
    // or next in its queue, whose claimed rows are all ready.
    bool heavy_open = (P.n_heavy > 0) && (wid < HW);
    bool main_open = true;
    // early claiming pays only when every heavy row gets a warp at once; with
    // more heavy rows than heavy warps (batches of many systems) they would
    // hold warps while waiting on their own chains: plain level order instead
    const int hcap = ((int64_t)P.n_heavy <= (int64_t)HW * nrowblk) ? P.n_heavy : 0;
    heavy_open = heavy_open && hcap > 0;
    for (;;) {
        int i = -1;
        if (lane == 0) {
            if (heavy_open) {
                const int h = atomicAdd(P.status + ST_CNT_H, 1);
                if (h < hcap) i = P.heavy_order[h]; else heavy_open = false;
            }
            while (i < 0 && main_open) {
                const int qi = atomicAdd(P.status + ST_CNT_F, 1);
                if (qi >= P.n + P.n_tasks + P.n_diag) { main_open = false; break; }
                const int c = P.row_order[qi];
                if (c >= P.n || hcap == 0 || P.heavy_rank[c] >= hcap) i = c;
            }
            if (i < 0) {
                // main queue drained: help with the heavy rows that are left
                const int h = hcap > 0 ? atomicAdd(P.status + ST_CNT_H, 1) : hcap;
                i = (h < hcap) ? P.heavy_order[h] : INT_MAX;
            }
        }
        i = __shfl_sync(FULL, i, 0);
        if (i == INT_MAX) return;
        if (ld_relaxed(P.status + ST_ERR) != 0) return;
        // a diag task: the diagonal-block step of a GEMM destination's row,
        // after its walk and the destination's tensor-core tasks
        bool diag_only = false;
        if (i >= P.n + P.n_tasks) {
            i = P.diag_row[i - P.n - P.n_tasks];
            diag_only = true;
        } else if (i >= P.n) {
            if (!tail_task<T>(P, i - P.n, gen, limit, ws, lane)) return;
            continue;
        }
        if (P.trace && lane == 0 && !diag_only) P.trace[4 * (int64_t)i] = gtimer();
        unsigned long long waited = 0;
        unsigned long long* wp = P.trace ? &waited : nullptr;
        const int D = P.node_of[i];
        const int r = P.sn_start[D], e = P.sn_start[D + 1] - 1, s = e - r + 1;
        // slot maps are indexed by column relative to the first row of the
        // row's instance (one system of a batch; 0 for a single system)
        int* pos = pos_warp - (P.node_base ? P.node_base[D] : 0);
        const int64_t l0 = P.row_lptr[i];
        const int nL = (int)(P.row_lptr[i + 1] - l0);
        const int64_t t0 = P.node_tail_off[D];
        const int nT = (int)(P.node_tail_off[D + 1] - t0);
        const int w = s + nT;
        T* xl = LV<T>(P) + l0;
        T* xu = PV<T>(P) + P.node_panel_off[D] + (int64_t)(i - r) * w;
        const int32_t* lc = P.lcols + l0;
        const int32_t* tc = P.tcols + t0;
        const int maxcol = nT > 0 ? tc[nT - 1] : e;
        Panel<T> pn;
        pn.r = r; pn.e = e; pn.s = s; pn.nL = nL; pn.nT = nT;
        pn.scols = reinterpret_cast<const int*>(ws->panel + sizeof(T) * (size_t)w);
        // a row of a GEMM destination keeps its U part in its panel (global):
        // the tensor-core tasks add their products there
        const int gd = (P.n_gd > 0) ? P.gd_of_node[D] : -1;
        int range;
        if (gd >= 0) {
            pn.mode = 2; pn.x = xu; range = w;
        } else if ((int64_t)(maxcol - r + 1) * (int64_t)sizeof(T) <= PANEL_BYTES) {
            pn.mode = 0; pn.x = reinterpret_cast<T*>(ws->panel); range = maxcol - r + 1;
        } else if ((int64_t)w * (int64_t)sizeof(T) + (int64_t)nT * 4 <= PANEL_BYTES) {
            pn.mode = 1; pn.x = reinterpret_cast<T*>(ws->panel); range = w;
        } else {
            pn.mode = 2; pn.x = xu; range = w;
        }
        if (!diag_only) {
        // ---- clear, column -> slot maps, scatter Ahat(i,:) (the value scatter).
        //      The first 32 L slots start in the shared-memory window; later
        //      L slots accumulate in global memory and are found through pos[]
        //      (also used by a panel kept in global memory).
        //      A row with a long L list keeps its pending L values in a dense
        //      per-warp vector indexed by column instead (no slot lookup).
        T* spa = (nL > DENSE_L_MIN && SPA<T>(P)) ? SPA<T>(P) + (size_t)(blockIdx.x * RW + wid) * (size_t)P.pos_n
                                                      - (P.node_base ? P.node_base[D] : 0)
                                                 : nullptr;
        //      Such a row with its U part in global memory (mode 2) also
        //      accumulates the U part in the dense vector (fire-and-forget
        //      reductions, no slot lookup, no load before the store) and
        //      gathers it into the panel after the last external update.
        T* spau = (spa && pn.mode == 2 && gd < 0) ? spa : nullptr;
        const bool need_pos = (!spa && nL > 32) || (pn.mode == 2 && !spau);
        win[lane] = T(0);
        if (spa) { for (int t = 32 + lane; t < nL; t += 32) spa[lc[t]] = T(0); }
        else     { for (int t = 32 + lane; t < nL; t += 32) xl[t] = T(0); }
        if (need_pos) for (int t = lane; t < nL; t += 32) pos[lc[t]] = t;
        if (spau) {
            for (int c = lane; c < s; c += 32) spau[r + c] = T(0);
            for (int j = lane; j < nT; j += 32) spau[tc[j]] = T(0);
        } else {
            for (int t = lane; t < range; t += 32) pn.x[t] = T(0);
        }
        if (pn.mode == 1) {
            int* sc = const_cast<int*>(pn.scols);
            for (int j = lane; j < nT; j += 32) sc[j] = tc[j];
        }
        if (pn.mode == 2 && !spau) for (int j = lane; j < nT; j += 32) pos[tc[j]] = nL + s + j;
        __syncwarp();
        for (int64_t q = P.ah_rp[i] + lane; q < P.ah_rp[i + 1]; q += 32) {
            const int sl = P.ah_slot[q];
            // scaling in FP64, then rounded to the factor precision
            const T v = (T)(vals[P.ah_src[q]] * P.ah_scale[q]);
            if (sl < nL) {
                if (sl < 32) win[sl] = v;
                else if (spa) spa[lc[sl]] = v;
                else xl[sl] = v;
            } else {
                const int us = sl - nL;
                if (spau) spau[us < s ? r + us : tc[us - s]] = v;
                else pn.x[us < s ? us : pn.tail_idx(tc, us - s)] = v;
            }
        }
        __syncwarp();
        bool pending = (nL > 32);   // global L slots written: fence before reading them
        // ---- updates from earlier nodes, ascending, 32 L slots at a time
        int t = 0;
        while (t < nL) {
            const int cend = min(32, nL - t);
            const int tq = t + lane;
            int kq = 0, eq = 0, sq = 1, nTq = 0, okq = 1;
            int64_t tq0 = 0, pq0 = 0;
            T dq = T(0);
            if (t > 0 && pending) { __threadfence(); pending = false; }
            if (lane < cend) {
                kq = lc[tq];
                const int Sq = P.node_of[kq];
                eq = P.sn_start[Sq + 1] - 1;
                sq = eq - P.sn_start[Sq] + 1;
                tq0 = P.node_tail_off[Sq];
                nTq = (int)(P.node_tail_off[Sq + 1] - tq0);
                pq0 = P.node_panel_off[Sq];
                okq = (ld_acquire(P.ready + eq) == gen);
                if (okq && sq == 1) {
                    dq = dinv[kq];
#pragma unroll
                    for (int m = 0; m < PF; ++m) {
                        ws->pfc[lane][m] = (m < nTq) ? P.tcols[tq0 + m] : INT_MAX;
                        ws->pfu[lane][m] = (m < nTq) ? PV<T>(P)[pq0 + 1 + m] : T(0);
                    }
                }
                if (t > 0) win[lane] = spa ? spa[kq] : xl[tq];
                wcol[lane] = kq;
            }
            const unsigned rmask = __ballot_sync(FULL, okq);
            __syncwarp();
            const int wmax = __shfl_sync(FULL, kq, cend - 1);
            // ---- phase 1: multipliers of the window's standalone sources, in
            //      order, with only the updates that land inside the window
            int q = 0;
            while (q < cend) {
                const int sS = __shfl_sync(FULL, sq, q);
                if (sS != 1) break;
                const int k = __shfl_sync(FULL, kq, q);
                const int nTS = __shfl_sync(FULL, nTq, q);
                T dk = __shfl_sync(FULL, dq, q);
                if (!((rmask >> q) & 1u)) {
                    if (!warp_wait(P.ready + k, gen, P.status, k, limit, wp)) return;
                    dk = dinv[k];
                    if (lane < PF) {
                        const int64_t tS = P.node_tail_off[P.node_of[k]];
                        const int64_t pS = P.node_panel_off[P.node_of[k]];
                        ws->pfc[q][lane] = (lane < nTS) ? P.tcols[tS + lane] : INT_MAX;
                        ws->pfu[q][lane] = (lane < nTS) ? PV<T>(P)[pS + 1 + lane] : T(0);
                    }
                    __syncwarp();
                }
                const T l = win[q] * dk;
                int inwin = 0;
                if (lane < PF) {
                    const int c = ws->pfc[q][lane];
                    if (c <= wmax) {
                        const int sl = bsearch_sm(wcol, cend, c);
                        win[sl] -= l * ws->pfu[q][lane];
                        inwin = 1;
                    }
                }
                int pl = __popc(__ballot_sync(FULL, inwin));
                if (pl == PF && nTS > PF) {
                    // rare: more of this source's tail falls inside the window
                    const int64_t tS = P.node_tail_off[P.node_of[k]];
                    const T* U1 = PV<T>(P) + P.node_panel_off[P.node_of[k]] + 1;
                    for (int jb = PF; jb < nTS; jb += 32) {
                        const int j = jb + lane;
                        const int c = (j < nTS) ? P.tcols[tS + j] : INT_MAX;
                        const int in = (c <= wmax);
                        if (in) win[bsearch_sm(wcol, cend, c)] -= l * U1[j];
                        const unsigned bm = __ballot_sync(FULL, in);
                        pl += __popc(bm);
                        if (bm != FULL) break;
                    }
                }
                __syncwarp();
                if (lane == 0) { win[q] = l; ws->plen[q] = pl; }
                __syncwarp();
                ++q;
            }
            const int qs = q;   // window sources [0, qs) have their multipliers
            // ---- phase 2: the rest of their tails, no ordering between sources
            //      needed: L part by atomic add, U part in the panel
            for (int qq = 0; qq < qs; ++qq) {
                const int nTS = __shfl_sync(FULL, nTq, qq);
                const int pl = ws->plen[qq];
                if (pl >= nTS) continue;
                const int64_t tS = __shfl_sync(FULL, tq0, qq);
                const int64_t pS = __shfl_sync(FULL, pq0, qq);
                apply_tail<T>(P.tcols + tS, PV<T>(P) + pS + 1, pl, nTS, win[qq], r, pos, xl, spa, spau, pn, lane,
                              gd >= 0);
                __syncwarp();
            }
            // any L slot past this window may have received atomic adds
            if (t + cend < nL) pending = true;
            // ---- close the window: multipliers (and untouched values) back to L
            if (lane < cend) {
                xl[tq] = win[lane];
                if (spa && qs < cend) spa[kq] = win[lane];   // the sup-row below reads by column
            }
            __syncwarp();
            if (qs == cend) { t += cend; continue; }
            __threadfence();
            pending = false;
            // ---- a source supernode at window slot qs: sup-row update
            //      l * U_SS = x_S (by position), x[T_S] -= l * U_S,T_S
            {
                const int k = __shfl_sync(FULL, kq, qs);
                const int eS = __shfl_sync(FULL, eq, qs);
                const int sS = __shfl_sync(FULL, sq, qs);
                const int nTS = __shfl_sync(FULL, nTq, qs);
                const int64_t tS = __shfl_sync(FULL, tq0, qs);
                const int64_t pS = __shfl_sync(FULL, pq0, qs);
                (void)k;
                if (!((rmask >> qs) & 1u))
                    if (!warp_wait(P.ready + eS, gen, P.status, eS, limit, wp)) return;
                const int tt = t + qs;
                const int rS = eS - sS + 1;
                const int wS = sS + nTS;
                const T* __restrict__ U = PV<T>(P) + pS;
                const int32_t* __restrict__ tcS = P.tcols + tS;
                // the source's pivot inverses staged in shared memory (the
                // window's prefetch area is free until the next window)
                T* dS = &ws->pfu[0][0];
                for (int p = lane; p < sS; p += 32) {
                    const int lab = P.piv[rS + p] - rS;
                    pb[p] = lab;
                    lb[p] = spa ? spa[rS + lab] : xl[tt + lab];
                    dS[p] = dinv[rS + p];
                }
                __syncwarp();
                // l U_SS = x_S by positions: each lane owns positions lane + 32 j,
                // and the U entries of step p + 1 are loaded while step p runs
                // (the arithmetic and its order are the plain forward
                // substitution's)
                {
                    int lq[SN_SMEM / 32];
                    T cur[SN_SMEM / 32];
#pragma unroll
                    for (int j = 0; j < SN_SMEM / 32; ++j) {
                        const int qq = lane + 32 * j;
                        lq[j] = (qq < sS) ? pb[qq] : 0;
                        cur[j] = (qq > 0 && qq < sS) ? U[lq[j]] : T(0);
                    }
                    for (int p = 0; p < sS; ++p) {
                        T nxt[SN_SMEM / 32];
                        const T* Un = U + (int64_t)(p + 1) * wS;
#pragma unroll
                        for (int j = 0; j < SN_SMEM / 32; ++j) {
                            const int qq = lane + 32 * j;
                            nxt[j] = (qq > p + 1 && qq < sS) ? Un[lq[j]] : T(0);
                        }
                        const T lp = lb[p] * dS[p];
                        __syncwarp();
#pragma unroll
                        for (int j = 0; j < SN_SMEM / 32; ++j) {
                            const int qq = lane + 32 * j;
                            if (qq > p && qq < sS) lb[qq] -= lp * cur[j];
                        }
                        if (lane == 0) lb[p] = lp;
                        __syncwarp();
#pragma unroll
                        for (int j = 0; j < SN_SMEM / 32; ++j) cur[j] = nxt[j];
                    }
                }
                // scatter one GEMV result into the row: a later L slot (by
                // column in the dense L vector, through pos[], or, for a row
                // whose L list fits one window, among the window columns) or
                // the U part
                auto put = [&](int c, T acc) {
                    if (c < r) {
                        if (spa) {
                            atomicAdd(spa + c, -acc);
                        } else {
                            const int sl = need_pos ? pos[c] : t + bsearch_sm(wcol, cend, c);
                            atomicAdd(xl + sl, -acc);
                        }
                    } else if (spau) {
                        atomicAdd(spau + c, -acc);
                    } else if (gd >= 0) {
                        atomicAdd(pn.x + pn.idx(pos, c), -acc);
                    } else {
                        pn.x[pn.idx(pos, c)] -= acc;
                    }
                };
                // a large source of a GEMM destination: the multipliers go
                // to the destination's split L block (the tensor-core tasks
                // apply the tail entries at or past r); this row only takes
                // the entries before r, a prefix of the sorted tail
                const int pair = (gd >= 0) ? P.gd_slot[l0 + tt] : -1;
                const int nTS_row = pair >= 0 ? P.pair_jr[pair] : nTS;
                if (pair >= 0) {
                    const int64_t ab = P.gd_a_off[gd] + (int64_t)(i - r) * P.gd_Kp[gd] + P.pair_u0[pair];
                    for (int p = lane; p < sS; p += 32) {
                        __nv_bfloat16 h3[3];
                        tc::split_bf16<3>((float)lb[p], h3);
                        P.a_term[0][ab + p] = __bfloat16_as_ushort(h3[0]);
                        P.a_term[1][ab + p] = __bfloat16_as_ushort(h3[1]);
                        P.a_term[2][ab + p] = __bfloat16_as_ushort(h3[2]);
                    }
                }
                // GEMV x[T_S] -= l U_S,T_S: 4 columns per lane, rows unrolled
                // by 4, so about 16 loads are in flight per lane (the FP64
                // instruction count is the same whatever the shape)
                for (int j0 = lane; j0 < nTS_row; j0 += 128) {
                    T acc[4];
                    const T* Uj[4];
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        const int j = j0 + 32 * jj;
                        Uj[jj] = U + sS + (j < nTS_row ? j : j0);
                        acc[jj] = T(0);
                    }
#pragma unroll 4
                    for (int p = 0; p < sS; ++p) {
                        const T lp = lb[p];
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) acc[jj] = fma(lp, Uj[jj][(int64_t)p * wS], acc[jj]);
                    }
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        const int j = j0 + 32 * jj;
                        if (j < nTS_row) put(tcS[j], acc[jj]);
                    }
                }
                for (int p = lane; p < sS; p += 32) xl[tt + p] = lb[p];
                __threadfence();
                __syncwarp();
                if (pair >= 0 && lane == 0) atomicAdd(P.pair_cnt + pair, 1);
                t = tt + sS;
                pending = false;
            }
        }
        if (spau) {
            // every reduction into the dense vector is complete (and read
            // from L2, bypassing any line this warp cached for an earlier row)
            __threadfence();
            __syncwarp();
            for (int c = lane; c < s; c += 32) pn.x[c] = __ldcg(spau + r + c);
            for (int j = lane; j < nT; j += 32) pn.x[s + j] = __ldcg(spau + tc[j]);
            __syncwarp();
        }
        if (gd >= 0) {
            // a GEMM destination's row: its diag task continues from here
            if (P.trace && lane == 0) P.trace[4 * (int64_t)i + 1] = gtimer();
            __threadfence();
            __syncwarp();
            if (lane == 0) st_release(P.walk_done + i, gen);
            continue;
        }
        }   // walk
        else {
            // diag task: the row's own walk, then every tensor-core task of
            // its destination (they add into its panel row)
            if (!warp_wait(P.walk_done + i, gen, P.status, i, limit, wp)) return;
            if (!warp_wait_ge(P.gd_done + gd, P.gd_ntask[gd], P.status, D, limit)) return;
        }
        if (P.trace && lane == 0 && !diag_only) P.trace[4 * (int64_t)i + 1] = gtimer();
        const unsigned long long waited_ext = waited;
        // a supernode with a U tail finishes it after the diagonal-block
        // step: by tail tasks, or (small nodes) by its last row right here
        const bool has_tasks = (s > 1) && (nT > 0);
        if (has_tasks && pn.mode != 2) {
            // the tail leaves the row here (the tail tasks finish it)
            for (int j = lane; j < nT; j += 32) xu[s + j] = pn.x[pn.tail_idx(tc, j)];
        }
        // the diagonal block (by label) of the row: lb for a supernode row,
        // the panel (one entry) for a standalone row
        T* xd = (s > 1) ? lb : pn.x;
        int dlab = 0;   // label offset of the row's pivot
        if (s > 1) {
            // (a diag task reads from L2: the panel row was written by other SMs)
            for (int c = lane; c < s; c += 32) lb[c] = diag_only ? __ldcg(pn.x + c) : pn.x[c];
            __syncwarp();
            // ---- diagonal-block step: earlier rows of the own supernode, each
            //      as soon as its own diagonal-block step is published
            const T* Ub = PV<T>(P) + P.node_panel_off[D];
            int pv[SN_SMEM / 32];   // position of label c = lane + 32 m
            for (int k = r; k < i; ++k) {
                if (!warp_wait(P.dready + k, gen, P.status, k, limit, wp)) return;
                // row k's pivot, inverse, block row and the positions of the
                // labels, all loaded together (none depends on another): a
                // label at a position past k stays past k under later swaps
                const int pk = ld_relaxed(P.piv + k);
                const T dk = dinv[k];
                const T* Uk = Ub + (int64_t)(k - r) * w;
                T uk[SN_SMEM / 32];
#pragma unroll
                for (int m = 0; m < SN_SMEM / 32; ++m) {
                    const int c = lane + 32 * m;
                    uk[m] = (c < s) ? Uk[c] : T(0);
                    pv[m] = (c < s) ? ld_relaxed(P.pinv + r + c) : -1;
                }
                const int lab = pk - r;
                const T l = lb[lab] * dk;
#pragma unroll
                for (int m = 0; m < SN_SMEM / 32; ++m) {
                    const int c = lane + 32 * m;
                    if (c < s && c != lab && pv[m] > k) lb[c] -= l * uk[m];
                }
                __syncwarp();
                if (lane == 0) lb[lab] = l;
                __syncwarp();
            }
            // ---- supernode diagonal pivoting: largest |x| among positions i..e,
            //      first position on ties.  The labels' positions are the ones
            //      loaded for row i - 1's step (no row past i - 1 swaps before
            //      row i); the first row reads them.  Compared in the factors'
            //      type: the order is the same as in FP64.
            if (i == r) {
#pragma unroll
                for (int m = 0; m < SN_SMEM / 32; ++m) {
                    const int c = lane + 32 * m;
                    pv[m] = (c < s) ? ld_relaxed(P.pinv + r + c) : -1;
                }
            }
            T best = T(-1);
            int bpos = INT_MAX, blab = -1, alab = -1;   // best position and label; the label at i
#pragma unroll
            for (int m = 0; m < SN_SMEM / 32; ++m) {
                const int c = lane + 32 * m;
                if (c < s && pv[m] >= i) {
                    const T a = fabs(lb[c]);
                    if (a > best || (a == best && pv[m] < bpos)) { best = a; bpos = pv[m]; blab = c; }
                    if (pv[m] == i) alab = c;
                }
            }
            for (int off = 16; off; off >>= 1) {
                const T ob = __shfl_down_sync(FULL, best, off);
                const int op = __shfl_down_sync(FULL, bpos, off);
                const int ol = __shfl_down_sync(FULL, blab, off);
                const int oa = __shfl_down_sync(FULL, alab, off);
                if (ob > best || (ob == best && op < bpos)) { best = ob; bpos = op; blab = ol; }
                alab = max(alab, oa);
            }
            bpos = __shfl_sync(FULL, bpos, 0);
            blab = __shfl_sync(FULL, blab, 0);
            alab = __shfl_sync(FULL, alab, 0);
            if (bpos == INT_MAX) { bpos = i; blab = alab; }   // no comparable value (NaN): keep position i
            if (lane == 0 && bpos != i) {
                P.piv[i] = r + blab; P.piv[bpos] = r + alab;
                P.pinv[r + blab] = i; P.pinv[r + alab] = bpos;
            }
            dlab = blab;
            __syncwarp();
        }
        // ---- pivot, small-pivot perturbation
        if (lane == 0) {
            const int dl = (s > 1) ? dlab : 0;
            // the small-pivot check is taken in FP64 whatever the factor precision
            double u = (double)((diag_only && s == 1) ? __ldcg(xd + dl) : xd[dl]);
            if (fabs(u) < tau) {
                u = (u >= 0.0) ? tau : -tau;
                xd[dl] = (T)u;
                atomicAdd(P.status + ST_NPERT, 1);
            }
            // the reciprocal in the factors' type (an FP64 division is a long
            // chain on the FP64 pipe, on the diagonal-block chain's path)
            dinv[i] = T(1) / xd[dl];
        }
        __syncwarp();
        // ---- write the row back, publish
        if (s > 1) {
            for (int c = lane; c < s; c += 32) xu[c] = lb[c];
            if (!has_tasks && pn.mode != 2)
                for (int j = lane; j < nT; j += 32) xu[s + j] = pn.x[pn.tail_idx(tc, j)];
        } else if (pn.mode != 2) {
            for (int c = lane; c < s; c += 32) xu[c] = pn.x[c];
            for (int j = lane; j < nT; j += 32) xu[s + j] = pn.x[pn.tail_idx(tc, j)];
        }
        __threadfence();
        __syncwarp();
        if (s > 1 && lane == 0) st_release(P.dready + i, gen);
        if (has_tasks) {
            // trace word 3 of such a row: when its node completed (tail tasks)
            if (P.trace && lane == 0) P.trace[4 * (int64_t)i + 2] = gtimer();
            if (P.node_ntask[D] == 0 && i == e) {
                // small node: every row's multipliers and tail are in (the
                // diagonal-block waits above acquired them); solve the tail here
                tail_solve<T>(P, D, 0, 1, ws, lane);
                __threadfence();
                __syncwarp();
                if (lane == 0) {
                    for (int k = r; k <= e; ++k) st_release(P.ready + k, gen);
                    if (P.trace) P.trace[4 * (int64_t)e + 3] = gtimer();
                }
                __syncwarp();
            }
            continue;   // the node's last tail task (or last row) publishes the row
        }
        if (lane == 0) st_release(P.ready + i, gen);
        if (P.trace && lane == 0) {
            P.trace[4 * (int64_t)i + 2] = gtimer();
            P.trace[4 * (int64_t)i + 3] = (waited_ext << 32) | ((waited - waited_ext) & 0xffffffffull);
        }
    }
}

// -------------------------------------------------------------- solve
template <typename A>
__global__ void permute_in_kernel(int32_t n, const int32_t* __restrict__ rowperm,
                                  const double* __restrict__ dr, const double* __restrict__ b,
                                  A* __restrict__ bh, int nrhs, int ld, int32_t* gens) {
    if (blockIdx.x == 0 && threadIdx.x == 0) gens[1] += 1;   // substitution generation of this call
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)n * nrhs;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int rr = (int)(q / n), i = (int)(q % n);
        const int o = rowperm[i];
        bh[q] = (A)(dr[o] * b[(int64_t)rr * ld + o]);
    }
}

template <typename A>
__global__ void permute_out_kernel(int32_t n, const int32_t* __restrict__ colperm,
                                   const double* __restrict__ dc, const A* __restrict__ xh,
                                   double* __restrict__ x, int nrhs, int ld) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)n * nrhs;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int rr = (int)(q / n), k = (int)(q % n);
        const int o = colperm[k];
        x[(int64_t)rr * ld + o] = dc[o] * (double)xh[q];
    }
}

// Bounded wait of the calling lanes on flag == gen; false on expiry/error.
__device__ __forceinline__ bool lane_wait(const int* flag, int gen, int* status, int who, long long limit) {
    if (ld_acquire(flag) == gen) return true;
    long long it = 0;
    while (ld_acquire(flag) != gen) {
        if (++it > limit) {
            if (atomicCAS(status + ST_ERR, 0, HYLU_ERR_DEVICE_TIMEOUT) == 0) status[ST_FAILED] = who;
            return false;
        }
        if ((it & 255) == 0 && ld_relaxed(status + ST_ERR) != 0) return false;
    }
    return true;
}

// Warp-wide sum of v[t] * x[c[t]], t < m, with UNR independent gathers in
// flight per lane; the result is valid in every lane.
template <typename T>
__device__ __forceinline__ T sparse_dot(const T* __restrict__ v, const int32_t* __restrict__ c, int m,
                                             const T* __restrict__ x, int lane) {
    T acc[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) acc[u] = 0.0;
    for (int t0 = 0; t0 < m; t0 += 32 * UNR) {
        int cc[UNR];
        T vv[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const int t = t0 + u * 32 + lane;
            cc[u] = (t < m) ? __ldg(c + t) : -1;
            vv[u] = (t < m) ? __ldg(v + t) : T(0);
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u)
            if (cc[u] >= 0) acc[u] = fma((T)vv[u], x[cc[u]], acc[u]);
    }
    T a = 0.0;
#pragma unroll
    for (int u = 0; u < UNR; ++u) a += acc[u];
    for (int off = 16; off; off >>= 1) a += __shfl_xor_sync(FULL, a, off);
    return a;
}

// Warp-wide sums out[u] = sum_t v[t] * x[u * ldx + c[t]], t < m, for up to
// RB right-hand sides u < nr at once: every L entry is loaded once and its
// gathers for all right-hand sides are in flight together.  The results are
// valid in every lane.
template <typename T, int RB>
__device__ __forceinline__ void sparse_dot_rhs(const T* __restrict__ v, const int32_t* __restrict__ c, int m,
                                               const T* __restrict__ x, int64_t ldx, int nr, int lane,
                                               T* out) {
    T acc[RB];
#pragma unroll
    for (int u = 0; u < RB; ++u) acc[u] = 0.0;
    for (int t0 = 0; t0 < m; t0 += 64) {
        int cc[2];
        T vv[2];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int t = t0 + b * 32 + lane;
            cc[b] = (t < m) ? __ldg(c + t) : -1;
            vv[b] = (t < m) ? __ldg(v + t) : T(0);
        }
#pragma unroll
        for (int b = 0; b < 2; ++b)
            if (cc[b] >= 0) {
#pragma unroll
                for (int u = 0; u < RB; ++u)
                    if (u < nr) acc[u] = fma((T)vv[b], x[u * ldx + cc[b]], acc[u]);
            }
    }
#pragma unroll
    for (int u = 0; u < RB; ++u) {
        T a = acc[u];
        for (int off = 16; off; off >>= 1) a += __shfl_xor_sync(FULL, a, off);
        out[u] = a;
    }
}

// Level watermark of the substitution (bulk mode, Sec. 2.2.1 / 2.3): nodes
// are grouped by dependency level; rows are claimed level by level, and a row
// of level L only waits until the watermark (levels whose nodes are all
// complete) reaches L.  The last node to complete a level raises it.
__device__ __forceinline__ bool wait_level(const int* wm, int need, int& cached, int* status, long long limit) {
    // one lane polls (with a short sleep once the wait is not immediate) and
    // the warp takes its answer: thousands of waiting warps would otherwise
    // keep the watermark's line busy in L2
    const int lane = threadIdx.x & 31;
    if (cached >= need) return true;
    int ok = 1, v = 0;
    if (lane == 0) {
        long long it = 0;
        while ((v = ld_acquire(wm)) < need) {
            if (++it > limit) {
                if (atomicCAS(status + ST_ERR, 0, HYLU_ERR_DEVICE_TIMEOUT) == 0) status[ST_FAILED] = -need;
                ok = 0;
                break;
            }
            if ((it & 255) == 0 && ld_relaxed(status + ST_ERR) != 0) { ok = 0; break; }
            // a warp two or more levels short of its wait polls rarely: the
            // warps of the next level then find the watermark's line free
            if (need - v > 1) __nanosleep(1024);
            else if (it > 8) __nanosleep(64);
        }
    }
    ok = __shfl_sync(FULL, ok, 0);
    v = __shfl_sync(FULL, v, 0);
    if (ok) cached = v;
    return ok != 0;
}


// called by lane 0 after the node's results are written and fenced; a
// level of one node raises the watermark without the counter's round trip
__device__ __forceinline__ void node_complete(int* done, const int* count, int L, int* wm) {
    if (count[L] == 1 || atom_add_acq_rel(done + L, 1) + 1 == count[L]) st_release(wm, L + 1);
}

// Dense block of a supernode in the substitution, by 32-row tiles.  The
// block is stored by label: entry (row i, position p) is
// Ub[(i - r) * w + piv[p] - r].  Right-hand side u is z + u * ldz (up to 8
// are handled per pass).  On this GPU one FP64 warp instruction holds its
// sub-partition's FP64 pipe for ~64 cycles whatever the active lanes, so the
// layout keeps every lane busy: lanes own rows and loop over the 32 columns.
//
// tile_apply: rows [R0, R0 + nr_rows) take the finished results of the 32
// positions [P0, P0 + nt) (z there already final): z_row -= sum_c
// B(row, P0 + c) z_{P0 + c}.  Each lane loads its row's 32 entries first (all
// loads in flight together), then one FMA chain per right-hand side.
template <typename T>
__device__ void tile_apply(const T* __restrict__ Ub, int w, int r, int R0, int nr_rows, int P0, int nt,
                           const int32_t* __restrict__ piv, T* __restrict__ z, int64_t ldz, int nrhs,
                           int lane) {
    const int lp = (lane < nt) ? piv[P0 + lane] - r : 0;
    const int row = R0 + lane;
    const bool ok = lane < nr_rows;
    const T* Ur = Ub + (int64_t)((ok ? row : R0) - r) * w;
    T Rrow[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        const int lc = __shfl_sync(FULL, lp, c);
        Rrow[c] = (ok && c < nt) ? Ur[lc] : T(0);
    }
    for (int u = 0; u < nrhs; ++u) {
        const T zt = (lane < nt) ? z[u * ldz + P0 + lane] : 0.0;
        T a = 0.0;
#pragma unroll
        for (int c = 0; c < 32; ++c)
            if (c < nt) a = fma((T)Rrow[c], __shfl_sync(FULL, zt, c), a);   // nt is warp-uniform
        if (ok) z[u * ldz + row] -= a;
    }
}

// tile_lower: unit lower triangle of the tile at positions [T0, T0 + nt)
// (rows T0 .. too), forward substitution in place.  The load part reads only
// factor data, so a warp can issue it before it waits for the solve's inputs.
template <typename T>
__device__ __forceinline__ void tile_lower_load(const T* __restrict__ Ub, int w, int r, int T0, int nt,
                                                const int32_t* __restrict__ piv, int lane, T (&Lrow)[32]) {
    const int lp = (lane < nt) ? piv[T0 + lane] - r : 0;
    const T* Ui = Ub + (int64_t)(T0 - r + (lane < nt ? lane : 0)) * w;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        Lrow[c] = T(0);
        if (c + 1 < nt) {                            // nt is warp-uniform
            const int lc = __shfl_sync(FULL, lp, c);
            if (lane < nt && c < lane) Lrow[c] = Ui[lc];
        }
    }
}

template <typename T>
__device__ __forceinline__ void tile_lower_solve(const T (&Lrow)[32], int T0, int nt, T* __restrict__ z,
                                                 int64_t ldz, int nrhs, int lane) {
    for (int u = 0; u < nrhs; ++u) {
        T my = (lane < nt) ? z[u * ldz + T0 + lane] : 0.0;
#pragma unroll
        for (int c = 0; c < 31; ++c) {
            if (c + 1 >= nt) break;                  // only nt - 1 steps
            const T zc = __shfl_sync(FULL, my, c);
            if (c < lane) my -= (T)Lrow[c] * zc;
        }
        if (lane < nt) z[u * ldz + T0 + lane] = my;
    }
}

template <typename T>
__device__ void tile_lower(const T* __restrict__ Ub, int w, int r, int T0, int nt, const int32_t* __restrict__ piv,
                           T* __restrict__ z, int64_t ldz, int nrhs, int lane) {
    T Lrow[32];
    tile_lower_load<T>(Ub, w, r, T0, nt, piv, lane, Lrow);
    tile_lower_solve<T>(Lrow, T0, nt, z, ldz, nrhs, lane);
}

// tile_upper: upper triangle of the tile (pivots through dinv), backward
// substitution in place.  The load part folds the pivots' inverses into the
// columns, U'_pc = U_pc di_c, so that the dependent chain is one FMA per
// step on a_p = z_p - sum_c U'_pc a_c, and w_p = di_p a_p at the end.
template <typename T>
__device__ __forceinline__ void tile_upper_load(const T* __restrict__ Ub, int w, int r, int T0, int nt,
                                                const int32_t* __restrict__ piv, const T* __restrict__ dinv,
                                                int lane, T (&Urow)[32], T& di) {
    const int lp = (lane < nt) ? piv[T0 + lane] - r : 0;
    di = (lane < nt) ? (T)dinv[T0 + lane] : 0.0;
    const T* Ui = Ub + (int64_t)(T0 - r + (lane < nt ? lane : 0)) * w;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        Urow[c] = 0.0;
        if (c >= 1 && c < nt) {                      // nt is warp-uniform
            const int lc = __shfl_sync(FULL, lp, c);
            const T dc = __shfl_sync(FULL, di, c);
            if (lane < c) Urow[c] = (T)Ui[lc] * dc;
        }
    }
}

template <typename T>
__device__ __forceinline__ void tile_upper_solve(const T (&Urow)[32], T di, int T0, int nt,
                                                 T* __restrict__ z, int64_t ldz, int nrhs, int lane) {
    for (int u = 0; u < nrhs; ++u) {
        T my = (lane < nt) ? z[u * ldz + T0 + lane] : 0.0;
#pragma unroll
        for (int c = 31; c >= 1; --c) {
            if (c >= nt) continue;                   // only nt - 1 steps
            const T ac = __shfl_sync(FULL, my, c);
            if (lane < c) my -= Urow[c] * ac;
        }
        if (lane < nt) z[u * ldz + T0 + lane] = my * di;
    }
}

template <typename T>
__device__ void tile_upper(const T* __restrict__ Ub, int w, int r, int T0, int nt, const int32_t* __restrict__ piv,
                           const T* __restrict__ dinv, T* __restrict__ z, int64_t ldz, int nrhs, int lane) {
    T Urow[32], di;
    tile_upper_load<T>(Ub, w, r, T0, nt, piv, dinv, lane, Urow, di);
    tile_upper_solve(Urow, di, T0, nt, z, ldz, nrhs, lane);
}

// Sequential mode of the bulk-sequential substitution (Sec. 2.3, Fig. 3:
// levels with many nodes are solved in bulk, the long chain sequentially).
// One thread block solves a segment of consecutive light levels: it waits
// once for the levels below the segment, then per level the warps share its
// rows (each row's dot product), a block barrier, the warps share the level's
// supernodes (the dense block by 32-row tiles), a block barrier; the level
// watermark is raised once, past the segment's last level.  Every thread of
// the block calls these; false when a wait expired or the solve failed.
__device__ __forceinline__ void seg_stamp(const DevPlan& P, const SegTable& S, int k, int dir) {
    if (!P.strace) return;
    for (int t = S.lvl_row[k] + threadIdx.x; t < S.lvl_row[k + 1]; t += blockDim.x) {
        const int i = S.rows[t], D = P.node_of[i];
        if (i == P.sn_start[D]) P.strace[2 * (int64_t)D + dir] = gtimer();
    }
}

template <typename T>
__device__ bool fwd_segment(const DevPlan& P, int g, T* __restrict__ z, int nrhs, long long limit) {
    const SegTable& S = P.fseg;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int n = P.n;
    const int q = S.meta[3 * g], L0 = S.meta[3 * g + 1], L1 = S.meta[3 * g + 2];
    int cached = 0;
    const bool ok = wait_level(P.wm_f + q, L0, cached, P.status, limit);
    if (__syncthreads_or(!ok)) return false;
    for (int k = S.seg_off[g]; k < S.seg_off[g + 1]; ++k) {
        for (int t = S.lvl_row[k] + wid; t < S.lvl_row[k + 1]; t += WARPS) {
            const int i = S.rows[t];
            const int64_t l0 = P.row_lptr[i];
            const int nL = (int)(P.row_lptr[i + 1] - l0);
            for (int r0 = 0; r0 < nrhs; r0 += 8) {
                T a[8];
                const int nr = min(8, nrhs - r0);
                if (nr == 1) a[0] = sparse_dot<T>(LV<T>(P) + l0, P.lcols + l0, nL, z + (int64_t)r0 * n, lane);
                else sparse_dot_rhs<T, 8>(LV<T>(P) + l0, P.lcols + l0, nL, z + (int64_t)r0 * n, n, nr, lane, a);
                if (lane == 0)
                    for (int u = 0; u < nr; ++u) z[(int64_t)(r0 + u) * n + i] -= a[u];
            }
        }
        __syncthreads();
        if (S.lvl_node[k + 1] > S.lvl_node[k]) {
            for (int t = S.lvl_node[k] + wid; t < S.lvl_node[k + 1]; t += WARPS) {
                const int D = S.snodes[t];
                const int r = P.sn_start[D], e = P.sn_start[D + 1] - 1, s = e - r + 1;
                const int w = s + (int)(P.node_tail_off[D + 1] - P.node_tail_off[D]);
                const T* Ub = PV<T>(P) + P.node_panel_off[D];
                for (int T0 = r; T0 <= e; T0 += 32) {
                    const int nt = min(32, e - T0 + 1);
                    for (int K0 = r; K0 < T0; K0 += 32)
                        tile_apply<T>(Ub, w, r, T0, nt, K0, 32, P.piv, z, n, nrhs, lane);
                    __syncwarp();
                    tile_lower<T>(Ub, w, r, T0, nt, P.piv, z, n, nrhs, lane);
                    __syncwarp();
                }
            }
            __syncthreads();
        }
        seg_stamp(P, S, k, 0);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) st_release(P.wm_f + q, L1 + 1);
    return true;
}

template <typename T>
__device__ bool bwd_segment(const DevPlan& P, int g, const T* __restrict__ dinv, T* __restrict__ z,
                            T* __restrict__ xh, int nrhs, long long limit) {
    const SegTable& S = P.bseg;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int n = P.n;
    const int q = S.meta[3 * g], L0 = S.meta[3 * g + 1], L1 = S.meta[3 * g + 2];
    int cached = 0;
    const bool ok = wait_level(P.wm_b + q, L0, cached, P.status, limit);
    if (__syncthreads_or(!ok)) return false;
    for (int k = S.seg_off[g]; k < S.seg_off[g + 1]; ++k) {
        for (int t = S.lvl_row[k] + wid; t < S.lvl_row[k + 1]; t += WARPS) {
            const int i = S.rows[t];
            const int D = P.node_of[i];
            const int r = P.sn_start[D], s = P.sn_start[D + 1] - r;
            const int64_t t0 = P.node_tail_off[D];
            const int nT = (int)(P.node_tail_off[D + 1] - t0);
            const T* Ui = PV<T>(P) + P.node_panel_off[D] + (int64_t)(i - r) * (s + nT);
            for (int r0 = 0; r0 < nrhs; r0 += 8) {
                T a[8];
                const int nr = min(8, nrhs - r0);
                if (nr == 1) a[0] = sparse_dot<T>(Ui + s, P.tcols + t0, nT, xh + (int64_t)r0 * n, lane);
                else sparse_dot_rhs<T, 8>(Ui + s, P.tcols + t0, nT, xh + (int64_t)r0 * n, n, nr, lane, a);
                if (lane == 0)
                    for (int u = 0; u < nr; ++u) {
                        const int64_t o = (int64_t)(r0 + u) * n + i;
                        if (s == 1) xh[o] = (z[o] - a[u]) * (T)dinv[i];
                        else z[o] -= a[u];
                    }
            }
        }
        __syncthreads();
        if (S.lvl_node[k + 1] > S.lvl_node[k]) {
            for (int t = S.lvl_node[k] + wid; t < S.lvl_node[k + 1]; t += WARPS) {
                const int D = S.snodes[t];
                const int r = P.sn_start[D], e = P.sn_start[D + 1] - 1, s = e - r + 1;
                const int w = s + (int)(P.node_tail_off[D + 1] - P.node_tail_off[D]);
                const T* Ub = PV<T>(P) + P.node_panel_off[D];
                for (int T0 = r + ((e - r) & ~31); T0 >= r; T0 -= 32) {
                    const int nt = min(32, e - T0 + 1);
                    for (int K0 = r + ((e - r) & ~31); K0 > T0; K0 -= 32)
                        tile_apply<T>(Ub, w, r, T0, nt, K0, min(32, e - K0 + 1), P.piv, z, n, nrhs, lane);
                    __syncwarp();
                    tile_upper<T>(Ub, w, r, T0, nt, P.piv, dinv, z, n, nrhs, lane);
                    __syncwarp();
                    for (int rr = 0; rr < nrhs; ++rr)
                        if (lane < nt) xh[(int64_t)rr * n + P.piv[T0 + lane]] = z[(int64_t)rr * n + T0 + lane];
                    __syncwarp();
                }
            }
            __syncthreads();
        }
        seg_stamp(P, S, k, 1);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) st_release(P.wm_b + q, L1 + 1);
    return true;
}

// The first seq_blocks blocks to start take the segments, in order, before
// they join the bulk claims; the other blocks go to the bulk claims directly.
// Decisions are block-uniform (a shared word between two barriers).
template <typename T>
__device__ bool run_segments(const DevPlan& P, bool bwd, const T* __restrict__ dinv, T* __restrict__ z,
                             T* __restrict__ xh, int nrhs, long long limit) {
    __shared__ int s_claim;
    const SegTable& S = bwd ? P.bseg : P.fseg;
    if (threadIdx.x == 0) s_claim = atomicAdd(P.status + (bwd ? ST_ROLE_B : ST_ROLE_F), 1);
    __syncthreads();
    const bool seq = s_claim < P.seq_blocks;
    __syncthreads();
    if (!seq) return true;
    for (;;) {
        if (threadIdx.x == 0)
            s_claim = ld_relaxed(P.status + ST_ERR) != 0 ? -1 : atomicAdd(P.status + (bwd ? ST_SEG_B : ST_SEG_F), 1);
        __syncthreads();
        const int g = s_claim;
        __syncthreads();
        if (g < 0) return false;
        if (g >= S.nseg) return true;
        if (!(bwd ? bwd_segment<T>(P, g, dinv, z, xh, nrhs, limit) : fwd_segment<T>(P, g, z, nrhs, limit)))
            return false;
    }
}

// Forward substitution L z = bhat (unit L, by position); z holds bhat on
// entry.  Each warp claims the next row in level order, waits for the lower
// levels of its instance, subtracts the row's L list; the warp of the last
// row of each 32-row tile of a supernode then solves the tile (tile_apply /
// tile_lower) once its rows have their external part and the earlier tiles
// are published.  Right-hand sides are columns of z (stride n).
template <typename T, bool ONE>
__global__ void __launch_bounds__(WARPS * 32)
fwd_kernel(DevPlan P, T* __restrict__ z, int nrhs, long long limit) {
    if (ONE) nrhs = 1;   // the one-right-hand-side variant: fewer registers, room for the tile prefetch
    if (P.fseg.nseg > 0 && !run_segments<T>(P, false, nullptr, z, nullptr, nrhs, limit)) return;
    const int gen = P.gens[1];
    const int lane = threadIdx.x & 31;
    const int n = P.n;
    int cached = 0, cq = 0;
    for (;;) {
        int qi = 0;
        if (lane == 0) qi = atomicAdd(P.status + ST_CNT_FWD, 1);
        qi = __shfl_sync(FULL, qi, 0);
        if (qi >= P.n_fwd_tasks) return;
        if (ld_relaxed(P.status + ST_ERR) != 0) return;
        const int i = P.fwd_task[qi];
        if (i >= n) {
            // a chunk of a long row's L list (the rectangular blocks of Sec.
            // 2.3): summed as soon as the levels of its entries complete.  The
            // several-right-hand-side variant sums whole rows instead.
            if (!ONE) continue;
            const int c = i - n;
            const int ri = P.fch_row[c];
            const int qc = P.node_inst ? P.node_inst[P.node_of[ri]] : 0;
            if (qc != cq) { cq = qc; cached = 0; }
            if (!__all_sync(FULL, wait_level(P.wm_f + qc, P.fch_level[c], cached, P.status, limit))) return;
            const int64_t o = P.row_lptr[ri] + P.fch_a[c];
            const T a = sparse_dot<T>(LV<T>(P) + o, P.lcols + o, P.fch_b[c] - P.fch_a[c], z, lane);
            if (lane == 0) reinterpret_cast<T*>(P.fch_part)[c] = a;
            __threadfence();
            __syncwarp();
            if (lane == 0) st_release(P.fch_flag + c, gen);
            continue;
        }
        const int D = P.node_of[i];
        const int L = P.fwd_level[D];
        const int r = P.sn_start[D], e = P.sn_start[D + 1] - 1, s = e - r + 1;
        const int q = P.node_inst ? P.node_inst[D] : 0;
        if (q != cq) { cq = q; cached = 0; }
        // 32-row tiles of a supernode's block: the warp of a tile's last row
        // owns it and loads its factor part before it waits
        const int T0 = r + ((i - r) & ~31);
        const int tlast = min(T0 + 31, e);
        const int nt = tlast - T0 + 1;
        const int w = s + (int)(P.node_tail_off[D + 1] - P.node_tail_off[D]);
        const T* Ub = PV<T>(P) + P.node_panel_off[D];
        T Lt[32];
        if (ONE && s > 1 && i == tlast) tile_lower_load<T>(Ub, w, r, T0, nt, P.piv, lane, Lt);
        const int64_t l0 = P.row_lptr[i], l1 = P.row_lptr[i + 1];
        const int nL = (int)(l1 - l0);
        // entries [0, sp) have sources at least two levels down: summed as
        // soon as those levels complete, before the level barrier
        const int sp = (P.fwd_split && L >= 1) ? P.fwd_split[i] : 0;
        const int c0 = ONE ? P.frow_chunk_off[i] : 0, c1 = ONE ? P.frow_chunk_off[i + 1] : 0;
        if (nrhs == 1 && c1 > c0) {
            // a long row: the sums of its chunks, each once its warp has
            // published it, added in chunk order (a fixed tree per 32 chunks).
            // The row still waits for its level: its node completing raises
            // the watermark past its level, which must not happen before the
            // lower levels complete (its chunks may all come from lower ones)
            if (!__all_sync(FULL, wait_level(P.wm_f + q, L, cached, P.status, limit))) return;
            T a = 0.0;
            for (int cb = c0; cb < c1; cb += 32) {
                const int c = cb + lane;
                int ok = 1;
                if (c < c1) ok = lane_wait(P.fch_flag + c, gen, P.status, c, limit);
                if (!__all_sync(FULL, ok)) return;
                T v = (c < c1) ? __ldcg(reinterpret_cast<const T*>(P.fch_part) + c) : T(0);
                for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
                a += v;
            }
            if (lane == 0) z[i] -= a;
        } else if (nrhs == 1) {
            T a = 0.0;
            if (sp > 0) {
                if (!__all_sync(FULL, wait_level(P.wm_f + q, L - 1, cached, P.status, limit))) return;
                a = sparse_dot<T>(LV<T>(P) + l0, P.lcols + l0, sp, z, lane);
            }
            if (!__all_sync(FULL, wait_level(P.wm_f + q, L, cached, P.status, limit))) return;
            a += sparse_dot<T>(LV<T>(P) + l0 + sp, P.lcols + l0 + sp, nL - sp, z, lane);
            if (lane == 0) z[i] -= a;
        } else {
            if (sp > 0 && !__all_sync(FULL, wait_level(P.wm_f + q, L - 1, cached, P.status, limit))) return;
            for (int r0 = 0; r0 < nrhs; r0 += 8) {
                T a[8], b[8];
                const int nr = min(8, nrhs - r0);
                for (int u = 0; u < 8; ++u) a[u] = 0.0;
                if (sp > 0)
                    sparse_dot_rhs<T, 8>(LV<T>(P) + l0, P.lcols + l0, sp, z + (int64_t)r0 * n, n, nr, lane, a);
                if (r0 == 0 && !__all_sync(FULL, wait_level(P.wm_f + q, L, cached, P.status, limit))) return;
                sparse_dot_rhs<T, 8>(LV<T>(P) + l0 + sp, P.lcols + l0 + sp, nL - sp, z + (int64_t)r0 * n, n, nr,
                                     lane, b);
                if (lane == 0)
                    for (int u = 0; u < nr; ++u) z[(int64_t)(r0 + u) * n + i] -= a[u] + b[u];
            }
        }
        __threadfence();
        __syncwarp();
        if (s == 1) {
            if (lane == 0) {
                if (P.strace) P.strace[2 * (int64_t)D + 0] = gtimer();
                node_complete(P.fwd_done + P.fwd_off[q], P.fwd_count + P.fwd_off[q], L, P.wm_f + q);
            }
            continue;
        }
        if (lane == 0) st_release(P.fwd_row + i, gen);
        if (i != tlast) continue;
        int ok = 1;
        for (int k = T0 + lane; k < tlast && ok; k += 32) ok = lane_wait(P.fwd_row + k, gen, P.status, k, limit);
        if (!__all_sync(FULL, ok)) return;
        // earlier tiles, each once its owner has published it
        for (int K0 = r; K0 < T0; K0 += 32) {
            if (!warp_wait(P.tile_f + K0 + 31, gen, P.status, K0 + 31, limit)) return;
            tile_apply<T>(Ub, w, r, T0, nt, K0, 32, P.piv, z, n, nrhs, lane);
        }
        __syncwarp();
        if (ONE) tile_lower_solve<T>(Lt, T0, nt, z, n, nrhs, lane);
        else tile_lower<T>(Ub, w, r, T0, nt, P.piv, z, n, nrhs, lane);
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release(P.tile_f + tlast, gen);
        if (tlast != e) continue;
        if (lane == 0) {
            if (P.strace) P.strace[2 * (int64_t)D + 0] = gtimer();
            node_complete(P.fwd_done + P.fwd_off[q], P.fwd_count + P.fwd_off[q], L, P.wm_f + q);
        }
    }
}

// Backward substitution U w = z by position; the solution is written by
// label: xh[piv[p]] = w_p.  Rows are claimed level by level (descending inside
// a level); each subtracts its U tail, and the warp of the first row of each
// 32-row tile of a supernode then back-substitutes the tile once the later
// tiles are published.  z is overwritten.
template <typename T, bool ONE>
__global__ void __launch_bounds__(WARPS * 32)
bwd_kernel(DevPlan P, const T* __restrict__ dinv, T* __restrict__ z,
           T* __restrict__ xh, int nrhs, long long limit) {
    if (ONE) nrhs = 1;
    if (P.bseg.nseg > 0 && !run_segments<T>(P, true, dinv, z, xh, nrhs, limit)) return;
    const int gen = P.gens[1];
    const int lane = threadIdx.x & 31;
    const int n = P.n;
    int cached = 0, cq = 0;
    for (;;) {
        int qi = 0;
        if (lane == 0) qi = atomicAdd(P.status + ST_CNT_BWD, 1);
        qi = __shfl_sync(FULL, qi, 0);
        if (qi >= P.n_bwd_tasks) return;
        if (ld_relaxed(P.status + ST_ERR) != 0) return;
        const int i = P.bwd_task[qi];
        const int D = P.node_of[i];
        const int L = P.bwd_level[D];
        const int r = P.sn_start[D], e = P.sn_start[D + 1] - 1, s = e - r + 1;
        const int64_t t0 = P.node_tail_off[D];
        const int nT = (int)(P.node_tail_off[D + 1] - t0);
        const int w = s + nT;
        const int32_t* tc = P.tcols + t0;
        const T* Ui = PV<T>(P) + P.node_panel_off[D] + (int64_t)(i - r) * w;
        const int q = P.node_inst ? P.node_inst[D] : 0;
        if (q != cq) { cq = q; cached = 0; }
        // 32-row tiles of a supernode's block: the warp of a tile's first row
        // owns it and loads its factor part before it waits
        const T* Ub = PV<T>(P) + P.node_panel_off[D];
        const int T0 = r + ((i - r) & ~31);
        const int tl = min(T0 + 31, e);
        const int nt = tl - T0 + 1;
        T Ut[32], dt = 0.0;
        if (ONE && s > 1 && i == T0) tile_upper_load<T>(Ub, w, r, T0, nt, P.piv, dinv, lane, Ut, dt);
        // tail entries [sp, nT) have sources at least two levels down (the
        // late ones come first in the tail): summed before the level barrier
        const int sp = (P.bwd_split && L >= 1) ? P.bwd_split[D] : nT;
        if (sp < nT && !__all_sync(FULL, wait_level(P.wm_b + q, L - 1, cached, P.status, limit))) return;
        for (int r0 = 0; r0 < nrhs; r0 += 8) {
            T a[8], b[8];
            const int nr = min(8, nrhs - r0);
            for (int u = 0; u < 8; ++u) { a[u] = 0.0; b[u] = 0.0; }
            if (sp < nT) {
                if (nr == 1) b[0] = sparse_dot<T>(Ui + s + sp, tc + sp, nT - sp, xh + (int64_t)r0 * n, lane);
                else sparse_dot_rhs<T, 8>(Ui + s + sp, tc + sp, nT - sp, xh + (int64_t)r0 * n, n, nr, lane, b);
            }
            if (r0 == 0 && !__all_sync(FULL, wait_level(P.wm_b + q, L, cached, P.status, limit))) return;
            if (nr == 1) a[0] = sparse_dot<T>(Ui + s, tc, sp, xh + (int64_t)r0 * n, lane);
            else sparse_dot_rhs<T, 8>(Ui + s, tc, sp, xh + (int64_t)r0 * n, n, nr, lane, a);
            for (int u = 0; u < nr; ++u) a[u] += b[u];
            if (lane == 0)
                for (int u = 0; u < nr; ++u) {
                    const int64_t o = (int64_t)(r0 + u) * n + i;
                    if (s == 1) xh[o] = (z[o] - a[u]) * (T)dinv[i];
                    else z[o] -= a[u];
                }
        }
        __threadfence();
        __syncwarp();
        if (s == 1) {
            if (lane == 0) {
                if (P.strace) P.strace[2 * (int64_t)D + 1] = gtimer();
                node_complete(P.bwd_done + P.bwd_off[q], P.bwd_count + P.bwd_off[q], L, P.wm_b + q);
            }
            continue;
        }
        if (lane == 0) st_release(P.bwd_row + i, gen);
        if (i != T0) continue;
        int ok = 1;
        for (int k = T0 + 1 + lane; k <= tl && ok; k += 32) ok = lane_wait(P.bwd_row + k, gen, P.status, k, limit);
        if (!__all_sync(FULL, ok)) return;
        // later tiles, last first, each once its owner has published it
        for (int K0 = r + ((e - r) & ~31); K0 > T0; K0 -= 32) {
            if (!warp_wait(P.tile_b + K0, gen, P.status, K0, limit)) return;
            tile_apply<T>(Ub, w, r, T0, nt, K0, min(32, e - K0 + 1), P.piv, z, n, nrhs, lane);
        }
        __syncwarp();
        if (ONE) tile_upper_solve(Ut, dt, T0, nt, z, n, nrhs, lane);
        else tile_upper<T>(Ub, w, r, T0, nt, P.piv, dinv, z, n, nrhs, lane);
        __syncwarp();
        for (int rr = 0; rr < nrhs; ++rr)
            if (lane < nt) xh[(int64_t)rr * n + P.piv[T0 + lane]] = z[(int64_t)rr * n + T0 + lane];
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release(P.tile_b + T0, gen);
        if (T0 != r) continue;
        if (lane == 0) {
            if (P.strace) P.strace[2 * (int64_t)D + 1] = gtimer();
            node_complete(P.bwd_done + P.bwd_off[q], P.bwd_count + P.bwd_off[q], L, P.wm_b + q);
        }
    }
}

// ------------------------------------------------------ transpose solve
// A^T y = g with Ahat Pi = L U:  h = Pi^T Pc^T Dc g;  U^T v = h;  L^T u = v;
// y = Dr Pr^T u.  In row storage U^T and L^T are applied by pushing each
// finished position's contributions to later ones (atomic adds); rows are
// claimed level by level, and the level watermark guarantees that a position
// has received every contribution before it is read.
__global__ void permute_in_t_kernel(int32_t n, const int32_t* __restrict__ piv, const int32_t* __restrict__ colperm,
                                    const double* __restrict__ dc, const double* __restrict__ g,
                                    double* __restrict__ hh, int nrhs, int ld, int32_t* gens) {
    if (blockIdx.x == 0 && threadIdx.x == 0) gens[1] += 1;   // substitution generation of this call
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)n * nrhs;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int rr = (int)(q / n), p = (int)(q % n);
        const int o = colperm[piv[p]];
        hh[q] = dc[o] * g[(int64_t)rr * ld + o];
    }
}

__global__ void permute_out_t_kernel(int32_t n, const int32_t* __restrict__ rowperm, const double* __restrict__ dr,
                                     const double* __restrict__ u, double* __restrict__ y, int nrhs, int ld) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)n * nrhs;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int rr = (int)(q / n), i = (int)(q % n);
        const int o = rowperm[i];
        y[(int64_t)rr * ld + o] = dr[o] * u[q];
    }
}

// Transpose blocks by 32-position tiles, lanes over the destination tile's
// positions: entry B(p, k) of U^T or L^T (k a source position) is row k of
// the panel at the label of p, so each lane reads along the source rows
// (Ub[(k - r) * w + piv[p] - r]).  Right-hand side u is h + u * ldh.
//
// tileT_apply: positions [T0, T0 + nt) take the finished values of the
// source positions [K0, K0 + nk): h_p -= sum_c B(p, K0 + c) h_{K0 + c}.
template <typename T>
__device__ void tileT_apply(const T* __restrict__ Ub, int w, int r, int T0, int nt, int K0, int nk,
                            const int32_t* __restrict__ piv, double* __restrict__ h, int64_t ldh, int nrhs,
                            int lane) {
    const int lp = (lane < nt) ? piv[T0 + lane] - r : 0;
    T Rrow[32];
#pragma unroll
    for (int c = 0; c < 32; ++c)
        Rrow[c] = (lane < nt && c < nk) ? Ub[(int64_t)(K0 + c - r) * w + lp] : T(0);
    for (int u = 0; u < nrhs; ++u) {
        const double vt = (lane < nk) ? h[u * ldh + K0 + lane] : 0.0;
        double a = 0.0;
#pragma unroll
        for (int c = 0; c < 32; ++c) a = fma((double)Rrow[c], __shfl_sync(FULL, vt, c), a);
        if (lane < nt) h[u * ldh + T0 + lane] -= a;
    }
}

// tileT_lower: U^T on the tile (lower in positions, pivots 1 / u_pp by
// position in dinv), forward substitution in place.
template <typename T>
__device__ void tileT_lower(const T* __restrict__ Ub, int w, int r, int T0, int nt, const int32_t* __restrict__ piv,
                            const T* __restrict__ dinv, double* __restrict__ h, int64_t ldh, int nrhs, int lane) {
    const int lp = (lane < nt) ? piv[T0 + lane] - r : 0;
    const double di = (lane < nt) ? (double)dinv[T0 + lane] : 0.0;
    T Trow[32];
#pragma unroll
    for (int c = 0; c < 32; ++c)
        Trow[c] = (lane < nt && c < lane) ? Ub[(int64_t)(T0 + c - r) * w + lp] : T(0);
    for (int u = 0; u < nrhs; ++u) {
        double my = (lane < nt) ? h[u * ldh + T0 + lane] : 0.0;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            if (lane == c) my *= di;
            const double vc = __shfl_sync(FULL, my, c);
            if (lane > c) my -= (double)Trow[c] * vc;
        }
        if (lane < nt) h[u * ldh + T0 + lane] = my;
    }
}

// tileT_upper: L^T on the tile (upper in positions, unit diagonal), backward
// substitution in place.
template <typename T>
__device__ void tileT_upper(const T* __restrict__ Ub, int w, int r, int T0, int nt, const int32_t* __restrict__ piv,
                            double* __restrict__ h, int64_t ldh, int nrhs, int lane) {
    const int lp = (lane < nt) ? piv[T0 + lane] - r : 0;
    T Trow[32];
#pragma unroll
    for (int c = 0; c < 32; ++c)
        Trow[c] = (lane < nt && c > lane && c < nt) ? Ub[(int64_t)(T0 + c - r) * w + lp] : T(0);
    for (int u = 0; u < nrhs; ++u) {
        double my = (lane < nt) ? h[u * ldh + T0 + lane] : 0.0;
#pragma unroll
        for (int c = 31; c >= 0; --c) {
            const double uc = __shfl_sync(FULL, my, c);
            if (lane < c) my -= (double)Trow[c] * uc;
        }
        if (lane < nt) h[u * ldh + T0 + lane] = my;
    }
}

// U^T v = h by position (h is overwritten by v)
template <typename T>
__global__ void __launch_bounds__(WARPS * 32)
ut_kernel(DevPlan P, double* __restrict__ h, int nrhs, long long limit) {
    const int gen = P.gens[1];
    const int lane = threadIdx.x & 31;
    const int n = P.n;
    int cached = 0, cq = 0;
    for (;;) {
        int qi = 0;
        if (lane == 0) qi = atomicAdd(P.status + ST_CNT_FWD, 1);
        qi = __shfl_sync(FULL, qi, 0);
        if (qi >= n) return;
        if (ld_relaxed(P.status + ST_ERR) != 0) return;
        const int i = P.ut_order[qi];
        const int D = P.node_of[i];
        const int L = P.ut_level[D];
        const int r = P.sn_start[D], e = P.sn_start[D + 1] - 1, s = e - r + 1;
        const int64_t t0 = P.node_tail_off[D];
        const int nT = (int)(P.node_tail_off[D + 1] - t0);
        const int w = s + nT;
        const T* Ub = PV<T>(P) + P.node_panel_off[D];
        const int q = P.node_inst ? P.node_inst[D] : 0;
        if (q != cq) { cq = q; cached = 0; }
        if (!__all_sync(FULL, wait_level(P.wm_f + q, L, cached, P.status, limit))) return;
        if (s == 1) {
            if (lane == 0) for (int rr = 0; rr < nrhs; ++rr) h[(int64_t)rr * n + i] *= (double)DI<T>(P)[i];
            __syncwarp();
        } else {
            // the block by 32-position tiles: the warp of a tile's first row
            // applies the finished earlier tiles and solves its triangle,
            // v_p = (h_p - sum_{k in [r,p)} U(k, pos p) v_k) / u_pp; the other
            // rows of the tile wait for it
            const int T0 = r + ((i - r) & ~31);
            const int nt = min(T0 + 31, e) - T0 + 1;
            if (i == T0) {
                for (int K0 = r; K0 < T0; K0 += 32) {
                    if (!warp_wait(P.tile_f + K0, gen, P.status, K0, limit)) return;
                    tileT_apply<T>(Ub, w, r, T0, nt, K0, 32, P.piv, h, n, nrhs, lane);
                }
                __syncwarp();
                tileT_lower<T>(Ub, w, r, T0, nt, P.piv, DI<T>(P), h, n, nrhs, lane);
                __threadfence();
                __syncwarp();
                if (lane == 0) st_release(P.tile_f + T0, gen);
            } else {
                if (!warp_wait(P.tile_f + T0, gen, P.status, T0, limit)) return;
            }
        }
        // push row i's U tail: h[pos of label c] -= U(i, c) v_i
        const T* Ui = Ub + (int64_t)(i - r) * w + s;
        const int32_t* tc = P.tcols + t0;
        for (int rr = 0; rr < nrhs; ++rr) {
            double* hr = h + (int64_t)rr * n;
            const double vi = hr[i];
            if (vi != 0.0)
                for (int j = lane; j < nT; j += 32) atomicAdd(hr + P.pinv[tc[j]], -(double)Ui[j] * vi);
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) node_complete(P.ut_done + P.ut_off[q], P.ut_count + P.ut_off[q], L, P.wm_f + q);
    }
}

// L^T u = v by position (h holds v on entry, u on exit)
template <typename T>
__global__ void __launch_bounds__(WARPS * 32)
lt_kernel(DevPlan P, double* __restrict__ h, int nrhs, long long limit) {
    const int gen = P.gens[1];
    const int lane = threadIdx.x & 31;
    const int n = P.n;
    int cached = 0, cq = 0;
    for (;;) {
        int qi = 0;
        if (lane == 0) qi = atomicAdd(P.status + ST_CNT_BWD, 1);
        qi = __shfl_sync(FULL, qi, 0);
        if (qi >= n) return;
        if (ld_relaxed(P.status + ST_ERR) != 0) return;
        const int i = P.lt_order[qi];
        const int D = P.node_of[i];
        const int L = P.lt_level[D];
        const int r = P.sn_start[D], e = P.sn_start[D + 1] - 1, s = e - r + 1;
        const int q = P.node_inst ? P.node_inst[D] : 0;
        if (q != cq) { cq = q; cached = 0; }
        if (!__all_sync(FULL, wait_level(P.wm_b + q, L, cached, P.status, limit))) return;
        if (s > 1) {
            // the block by 32-position tiles, last tile first: the warp of a
            // tile's last row applies the finished later tiles and solves its
            // triangle, u_k = v_k - sum_{j in (k, e]} L(j, pos k) u_j; the
            // other rows of the tile wait for it
            const int T0 = r + ((i - r) & ~31);
            const int tl = min(T0 + 31, e);
            if (i == tl) {
                const int w = s + (int)(P.node_tail_off[D + 1] - P.node_tail_off[D]);
                const T* Ub = PV<T>(P) + P.node_panel_off[D];
                const int nt = tl - T0 + 1;
                for (int K0 = r + ((e - r) & ~31); K0 > T0; K0 -= 32) {
                    const int kl = min(K0 + 31, e);
                    if (!warp_wait(P.tile_b + kl, gen, P.status, kl, limit)) return;
                    tileT_apply<T>(Ub, w, r, T0, nt, K0, kl - K0 + 1, P.piv, h, n, nrhs, lane);
                }
                __syncwarp();
                tileT_upper<T>(Ub, w, r, T0, nt, P.piv, h, n, nrhs, lane);
                __threadfence();
                __syncwarp();
                if (lane == 0) st_release(P.tile_b + tl, gen);
            } else {
                if (!warp_wait(P.tile_b + tl, gen, P.status, tl, limit)) return;
            }
        }
        // push row i's L list: h[c] -= L(i, c) u_i (c by position)
        const int64_t l0 = P.row_lptr[i], l1 = P.row_lptr[i + 1];
        for (int rr = 0; rr < nrhs; ++rr) {
            double* hr = h + (int64_t)rr * n;
            const double ui = hr[i];
            if (ui != 0.0)
                for (int64_t t = l0 + lane; t < l1; t += 32) atomicAdd(hr + P.lcols[t], -(double)LV<T>(P)[t] * ui);
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) node_complete(P.lt_done + P.lt_off[q], P.lt_count + P.lt_off[q], L, P.wm_b + q);
    }
}

// r = g - A^T y (atomic scatter over the rows of A), column abs sums of A
__global__ void residual_t_kernel(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                  const double* __restrict__ v, const double* __restrict__ y,
                                  double* __restrict__ res, double* __restrict__ colsum, int nrhs, int ld) {
    const int lane = threadIdx.x & 31;
    const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = wg; i < n; i += nw) {
        for (int64_t q = rp[i] + lane; q < rp[i + 1]; q += 32) {
            const int j = ci[q];
            for (int rr = 0; rr < nrhs; ++rr) atomicAdd(res + (int64_t)rr * ld + j, -v[q] * y[(int64_t)rr * ld + i]);
            atomicAdd(colsum + j, fabs(v[q]));
        }
    }
}

// norms[rr] = {||r||inf, ||y||inf, ||g||inf} as bit patterns, norms[3 nrhs] = max column sum
__global__ void norms_t_kernel(int32_t n, const double* __restrict__ res, const double* __restrict__ y,
                               const double* __restrict__ g, const double* __restrict__ colsum,
                               unsigned long long* norms, int nrhs, int ld) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)n * nrhs;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int rr = (int)(q / n), i = (int)(q % n);
        const int64_t o = (int64_t)rr * ld + i;
        atomicMax(norms + 3 * rr + 0, (unsigned long long)__double_as_longlong(fabs(res[o])));
        atomicMax(norms + 3 * rr + 1, (unsigned long long)__double_as_longlong(fabs(y[o])));
        atomicMax(norms + 3 * rr + 2, (unsigned long long)__double_as_longlong(fabs(g[o])));
        if (rr == 0) atomicMax(norms + 3 * nrhs, (unsigned long long)__double_as_longlong(colsum[i]));
    }
}

// Adjoint of x = A^{-1} b for the entries of A: dL/dA_ij = -sum_r lam_r[i] x_r[j]
__global__ void grad_values_kernel(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                   const double* __restrict__ lam, const double* __restrict__ x,
                                   double* __restrict__ dv, int nrhs, int ld) {
    const int lane = threadIdx.x & 31;
    const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = wg; i < n; i += nw) {
        for (int64_t q = rp[i] + lane; q < rp[i + 1]; q += 32) {
            const int j = ci[q];
            double a = 0.0;
            for (int rr = 0; rr < nrhs; ++rr) a = fma(lam[(int64_t)rr * ld + i], x[(int64_t)rr * ld + j], a);
            dv[q] = -a;
        }
    }
}

// r = b - A x on the original A; norms[rr] = {||r||inf, ||x||inf, ||b||inf}
// as bit patterns (non-negative doubles), norms[3*nrhs] = ||A||inf.
__global__ void residual_kernel(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                const double* __restrict__ v, const double* __restrict__ x,
                                const double* __restrict__ b, double* __restrict__ res,
                                unsigned long long* norms, int nrhs, int ld) {
    const int lane = threadIdx.x & 31;
    const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = wg; i < n; i += nw) {
        for (int rr = 0; rr < nrhs; ++rr) {
            const double* xr = x + (int64_t)rr * ld;
            double a = 0.0, ra = 0.0;
            for (int64_t q = rp[i] + lane; q < rp[i + 1]; q += 32) {
                a = fma(v[q], xr[ci[q]], a);
                if (rr == 0) ra += fabs(v[q]);
            }
            for (int off = 16; off; off >>= 1) {
                a += __shfl_xor_sync(FULL, a, off);
                ra += __shfl_xor_sync(FULL, ra, off);
            }
            if (lane == 0) {
                const double bi = b[(int64_t)rr * ld + i];
                const double ri = bi - a;
                res[(int64_t)rr * ld + i] = ri;
                atomicMax(norms + 3 * rr + 0, (unsigned long long)__double_as_longlong(fabs(ri)));
                atomicMax(norms + 3 * rr + 1, (unsigned long long)__double_as_longlong(fabs(xr[i])));
                atomicMax(norms + 3 * rr + 2, (unsigned long long)__double_as_longlong(fabs(bi)));
                if (rr == 0) atomicMax(norms + 3 * nrhs, (unsigned long long)__double_as_longlong(ra));
            }
        }
    }
}

__global__ void axpy_kernel(int32_t n, double* __restrict__ x, const double* __restrict__ d, int nrhs, int ld) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)n * nrhs;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int rr = (int)(q / n), i = (int)(q % n);
        x[(int64_t)rr * ld + i] += d[(int64_t)rr * ld + i];
    }
}

}  // namespace

int64_t launches() { return g_launches.load(); }
void count_launch() { ++g_launches; }
void add_launches(int64_t k) { g_launches += k; }

static int check(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "hylu: %s: %s\n", what, cudaGetErrorString(e));
        return HYLU_ERR_CUDA;
    }
    return HYLU_OK;
}

int warps_per_block() { return FWARPS; }
int dense_l_min() { return DENSE_L_MIN; }

constexpr size_t tc_smem() { return sizeof(WarpSmem<float>) * TC_ROWW + sizeof(GemmSmem) + 1024; }

void set_smem_attrs() {
    cudaFuncSetAttribute(factor_kernel<double, FWARPS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)factor_smem<double>());
    cudaFuncSetAttribute(factor_kernel<float, FWARPS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)factor_smem<float>());
    cudaFuncSetAttribute(factor_kernel<float, TC_ROWW, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tc_smem());
}

int factor_grid(int device, bool fp32) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    set_smem_attrs();
    if (fp32)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, factor_kernel<float, FWARPS, false>, FWARPS * 32,
                                                      factor_smem<float>());
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, factor_kernel<double, FWARPS, false>, FWARPS * 32,
                                                      factor_smem<double>());
    if (per < 1) per = 1;
    if (per > 4) per = 4;
    return sms * per;
}

int launch_reset(int32_t* status, int32_t* piv, int32_t* pinv, int32_t* gens, int32_t n, cudaStream_t st) {
    if (cudaMemsetAsync(status, 0, sizeof(int32_t) * ST_WORDS, st) != cudaSuccess) return HYLU_ERR_CUDA;
    int blocks = (int)std::min<int64_t>(4096, ((int64_t)n + 255) / 256 + 1);
    reset_kernel<<<blocks, 256, 0, st>>>(piv, pinv, n, gens);
    count_launch();
    return check("reset");
}

void factor_occupancy(int* per64, int* per32, int* per_tc, int* regs_tc) {
    cudaFuncAttributes a{};
    set_smem_attrs();
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(per64, factor_kernel<double, FWARPS, false>, FWARPS * 32,
                                                  factor_smem<double>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(per32, factor_kernel<float, FWARPS, false>, FWARPS * 32,
                                                  factor_smem<float>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_tc, factor_kernel<float, TC_ROWW, true>, (TC_ROWW + 4) * 32,
                                                  tc_smem());
    cudaFuncGetAttributes(&a, factor_kernel<float, TC_ROWW, true>);
    *regs_tc = a.numRegs * 10000 + (int)(a.sharedSizeBytes + tc_smem()) / 16;
}

int gemm_smem_fits() { return tc_smem() <= 227 * 1024; }

int tc_grid(int device) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    set_smem_attrs();
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, factor_kernel<float, TC_ROWW, true>, (TC_ROWW + 4) * 32,
                                                  tc_smem());
    return sms * std::max(per, 0);
}

int launch_factor(const DevPlan& P, const double* d_vals, int64_t nnz_a,
                  double tau_rel, long long spin_limit, int grid, cudaStream_t st, cudaEvent_t e0,
                  cudaEvent_t e1) {
    if (P.n_tasks > 0 && cudaMemsetAsync(P.node_done, 0, sizeof(int32_t) * P.nnodes, st) != cudaSuccess)
        return HYLU_ERR_CUDA;
    if (P.n_gd > 0) {
        // tensor-core sup-sup: counters, and the split multiplier blocks
        // (entries no row writes -- padding rows and columns, and rows of a
        // destination without the pair's source -- must read as zero)
        if (cudaMemsetAsync(P.pair_cnt, 0, sizeof(int32_t) * P.n_pair, st) != cudaSuccess) return HYLU_ERR_CUDA;
        if (cudaMemsetAsync(P.gd_done, 0, sizeof(int32_t) * P.n_gd, st) != cudaSuccess) return HYLU_ERR_CUDA;
        for (int s = 0; s < 3; ++s)
            if (cudaMemsetAsync(P.a_term[s], 0, sizeof(uint16_t) * P.a_elems, st) != cudaSuccess) return HYLU_ERR_CUDA;
    }
    int blocks = (int)std::min<int64_t>(2048, (nnz_a + 255) / 256 + 1);
    amax_kernel<<<blocks, 256, 0, st>>>(d_vals, P.ah_src, P.ah_scale, nnz_a, P.status);
    count_launch();
    if (e0) cudaEventRecord(e0, st);
    if (P.lval32 && P.n_gd > 0)
        factor_kernel<float, TC_ROWW, true><<<P.gemm_blocks, (TC_ROWW + 4) * 32, tc_smem(), st>>>(
            P, d_vals, P.dinv32, tau_rel, spin_limit);
    else if (P.lval32)
        factor_kernel<float, FWARPS, false><<<grid, FWARPS * 32, factor_smem<float>(), st>>>(P, d_vals, P.dinv32,
                                                                                            tau_rel, spin_limit);
    else
        factor_kernel<double, FWARPS, false><<<grid, FWARPS * 32, factor_smem<double>(), st>>>(P, d_vals, P.dinv,
                                                                                              tau_rel, spin_limit);
    count_launch();
    if (e1) cudaEventRecord(e1, st);
    return check("factor");
}

// Blocks of the substitution kernels that can be resident at once (the
// fewest over the forward / backward and one / several right-hand-side
// variants of the factors' type), cached per device and type.
static int solve_resident_blocks(bool fp32) {
    static int cache[64][2] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    int& c = cache[dev][fp32 ? 1 : 0];
    if (c > 0) return c;
    int sms = 0, per[4] = {0, 0, 0, 0};
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (fp32) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[0], fwd_kernel<float, true>, WARPS * 32, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[1], fwd_kernel<float, false>, WARPS * 32, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[2], bwd_kernel<float, true>, WARPS * 32, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[3], bwd_kernel<float, false>, WARPS * 32, 0);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[0], fwd_kernel<double, true>, WARPS * 32, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[1], fwd_kernel<double, false>, WARPS * 32, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[2], bwd_kernel<double, true>, WARPS * 32, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[3], bwd_kernel<double, false>, WARPS * 32, 0);
    }
    c = sms * std::max(1, std::min(std::min(per[0], per[1]), std::min(per[2], per[3])));
    return c;
}

int launch_solve(const DevPlan& P, const double* d_b, double* d_x, double* d_z, double* d_xh,
                 const int32_t* rowperm, const int32_t* colperm, const double* dr, const double* dc,
                 int nrhs, int ld, long long spin_limit, int grid, cudaStream_t st,
                 cudaEvent_t e0, cudaEvent_t e1) {
    const int64_t tot = (int64_t)P.n * nrhs;
    const int eb = (int)std::min<int64_t>(4096, (tot + 255) / 256 + 1);
    // segments need a block of their own beside resident bulk blocks
    if ((P.fseg.nseg > 0 || P.bseg.nseg > 0) && (grid < 2 || solve_resident_blocks(P.lval32 != nullptr) < 2))
        return HYLU_ERR_INTERNAL;
    if (cudaMemsetAsync(P.status + ST_CNT_FWD, 0, sizeof(int32_t) * 4, st) != cudaSuccess) return HYLU_ERR_CUDA;
    if (cudaMemsetAsync(P.status + ST_SEG_F, 0, sizeof(int32_t) * 2, st) != cudaSuccess) return HYLU_ERR_CUDA;
    if (cudaMemsetAsync(P.fwd_done, 0, sizeof(int32_t) * P.n_fwd_levels, st) != cudaSuccess) return HYLU_ERR_CUDA;
    if (cudaMemsetAsync(P.wm_f, 0, sizeof(int32_t) * P.n_inst, st) != cudaSuccess) return HYLU_ERR_CUDA;
    if (cudaMemsetAsync(P.wm_b, 0, sizeof(int32_t) * P.n_inst, st) != cudaSuccess) return HYLU_ERR_CUDA;
    if (cudaMemsetAsync(P.bwd_done, 0, sizeof(int32_t) * P.n_bwd_levels, st) != cudaSuccess) return HYLU_ERR_CUDA;
    // the substitution computes in the factors' type: FP32 factors (the
    // precision form) are solved in FP32, their refinement's residual and
    // update stay in FP64; the FP32 vectors use the first halves of z and xh
    float* z32 = reinterpret_cast<float*>(d_z);
    float* xh32 = reinterpret_cast<float*>(d_xh);
    if (P.lval32) permute_in_kernel<float><<<eb, 256, 0, st>>>(P.n, rowperm, dr, d_b, z32, nrhs, ld, P.gens);
    else permute_in_kernel<double><<<eb, 256, 0, st>>>(P.n, rowperm, dr, d_b, d_z, nrhs, ld, P.gens);
    count_launch();
    // the segments' rows are not in the bulk claim lists: at least one block
    // takes the segments, and at least three quarters of the blocks that can
    // be resident at once stay in bulk (the first blocks to start take the
    // segments, so a launch larger than what is resident must not let them
    // fill the GPU: their waits need bulk rows)
    DevPlan Q = P;
    const bool seg = P.fseg.nseg > 0 || P.bseg.nseg > 0;
    const int resident = seg ? solve_resident_blocks(P.lval32 != nullptr) : 0;
    const int blocks = grid;
    if (seg) Q.seq_blocks = std::max(1, std::min(P.seq_blocks, std::min(resident, blocks) / 4));
    if (e0) cudaEventRecord(e0, st);
    if (nrhs == 1) {
        if (P.lval32) fwd_kernel<float, true><<<blocks, WARPS * 32, 0, st>>>(Q, z32, nrhs, spin_limit);
        else fwd_kernel<double, true><<<blocks, WARPS * 32, 0, st>>>(Q, d_z, nrhs, spin_limit);
        count_launch();
        if (P.lval32) bwd_kernel<float, true><<<blocks, WARPS * 32, 0, st>>>(Q, P.dinv32, z32, xh32, nrhs, spin_limit);
        else bwd_kernel<double, true><<<blocks, WARPS * 32, 0, st>>>(Q, P.dinv, d_z, d_xh, nrhs, spin_limit);
    } else {
        if (P.lval32) fwd_kernel<float, false><<<blocks, WARPS * 32, 0, st>>>(Q, z32, nrhs, spin_limit);
        else fwd_kernel<double, false><<<blocks, WARPS * 32, 0, st>>>(Q, d_z, nrhs, spin_limit);
        count_launch();
        if (P.lval32) bwd_kernel<float, false><<<blocks, WARPS * 32, 0, st>>>(Q, P.dinv32, z32, xh32, nrhs, spin_limit);
        else bwd_kernel<double, false><<<blocks, WARPS * 32, 0, st>>>(Q, P.dinv, d_z, d_xh, nrhs, spin_limit);
    }
    count_launch();
    if (e1) cudaEventRecord(e1, st);
    if (P.lval32) permute_out_kernel<float><<<eb, 256, 0, st>>>(P.n, colperm, dc, xh32, d_x, nrhs, ld);
    else permute_out_kernel<double><<<eb, 256, 0, st>>>(P.n, colperm, dc, d_xh, d_x, nrhs, ld);
    count_launch();
    return check("solve");
}

int launch_solve_transpose(const DevPlan& P, const double* d_b, double* d_x, double* d_h,
                           const int32_t* rowperm, const int32_t* colperm, const double* dr, const double* dc,
                           int nrhs, int ld, long long spin_limit, int grid, cudaStream_t st) {
    const int64_t tot = (int64_t)P.n * nrhs;
    const int eb = (int)std::min<int64_t>(4096, (tot + 255) / 256 + 1);
    if (cudaMemsetAsync(P.status + ST_CNT_FWD, 0, sizeof(int32_t) * 4, st) != cudaSuccess) return HYLU_ERR_CUDA;
    if (cudaMemsetAsync(P.ut_done, 0, sizeof(int32_t) * P.n_ut_levels, st) != cudaSuccess) return HYLU_ERR_CUDA;
    if (cudaMemsetAsync(P.wm_f, 0, sizeof(int32_t) * P.n_inst, st) != cudaSuccess) return HYLU_ERR_CUDA;
    if (cudaMemsetAsync(P.wm_b, 0, sizeof(int32_t) * P.n_inst, st) != cudaSuccess) return HYLU_ERR_CUDA;
    if (cudaMemsetAsync(P.lt_done, 0, sizeof(int32_t) * P.n_lt_levels, st) != cudaSuccess) return HYLU_ERR_CUDA;
    permute_in_t_kernel<<<eb, 256, 0, st>>>(P.n, P.piv, colperm, dc, d_b, d_h, nrhs, ld, P.gens);
    count_launch();
    if (P.lval32) ut_kernel<float><<<grid, WARPS * 32, 0, st>>>(P, d_h, nrhs, spin_limit);
    else ut_kernel<double><<<grid, WARPS * 32, 0, st>>>(P, d_h, nrhs, spin_limit);
    count_launch();
    if (P.lval32) lt_kernel<float><<<grid, WARPS * 32, 0, st>>>(P, d_h, nrhs, spin_limit);
    else lt_kernel<double><<<grid, WARPS * 32, 0, st>>>(P, d_h, nrhs, spin_limit);
    count_launch();
    permute_out_t_kernel<<<eb, 256, 0, st>>>(P.n, rowperm, dr, d_h, d_x, nrhs, ld);
    count_launch();
    return check("solve_transpose");
}

int launch_residual_transpose(int32_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* y,
                              const double* g, double* r, double* colsum, double* norms, int nrhs, int ld,
                              cudaStream_t st) {
    for (int rr = 0; rr < nrhs; ++rr)
        if (cudaMemcpyAsync(r + (int64_t)rr * ld, g + (int64_t)rr * ld, sizeof(double) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return HYLU_ERR_CUDA;
    if (cudaMemsetAsync(colsum, 0, sizeof(double) * n, st) != cudaSuccess) return HYLU_ERR_CUDA;
    if (cudaMemsetAsync(norms, 0, sizeof(double) * (3 * nrhs + 1), st) != cudaSuccess) return HYLU_ERR_CUDA;
    const int blocks = (int)std::min<int64_t>(4096, ((int64_t)n * 32 + 255) / 256 + 1);
    residual_t_kernel<<<blocks, 256, 0, st>>>(n, rp, ci, v, y, r, colsum, nrhs, ld);
    count_launch();
    const int eb = (int)std::min<int64_t>(4096, ((int64_t)n * nrhs + 255) / 256 + 1);
    norms_t_kernel<<<eb, 256, 0, st>>>(n, r, y, g, colsum, reinterpret_cast<unsigned long long*>(norms), nrhs, ld);
    count_launch();
    return check("residual_transpose");
}

int launch_grad_values(int32_t n, const int64_t* rp, const int32_t* ci, const double* lam, const double* x,
                       double* dvals, int nrhs, int ld, cudaStream_t st) {
    const int blocks = (int)std::min<int64_t>(4096, ((int64_t)n * 32 + 255) / 256 + 1);
    grad_values_kernel<<<blocks, 256, 0, st>>>(n, rp, ci, lam, x, dvals, nrhs, ld);
    count_launch();
    return check("grad_values");
}

int launch_residual(int32_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* x,
                    const double* b, double* r, double* norms, int nrhs, int ld, cudaStream_t st) {
    if (cudaMemsetAsync(norms, 0, sizeof(double) * (3 * nrhs + 1), st) != cudaSuccess) return HYLU_ERR_CUDA;
    const int blocks = (int)std::min<int64_t>(4096, ((int64_t)n * 32 + 255) / 256 + 1);
    residual_kernel<<<blocks, 256, 0, st>>>(n, rp, ci, v, x, b, r,
                                            reinterpret_cast<unsigned long long*>(norms), nrhs, ld);
    count_launch();
    return check("residual");
}

int launch_axpy(int32_t n, double* x, const double* d, int nrhs, int ld, cudaStream_t st) {
    const int64_t tot = (int64_t)n * nrhs;
    const int eb = (int)std::min<int64_t>(4096, (tot + 255) / 256 + 1);
    axpy_kernel<<<eb, 256, 0, st>>>(n, x, d, nrhs, ld);
    count_launch();
    return check("axpy");
}

}  // namespace hylu

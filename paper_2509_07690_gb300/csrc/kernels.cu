// Numeric factorization and substitution kernels for sm_103a (HYLU Sec. 2.2,
// 2.2.1 and 2.3).
//
// Factorization: one persistent kernel; every warp claims the next row in
// ascending order from an atomic counter and runs the up-looking update of
// that row (Sec. 2.2, Fig. 1):
//   - Ahat(i,:) is scattered (scaled) straight into the row's storage;
//   - each source in the row's L list, in ascending order, is waited for on
//     its ready flag and applied: a standalone source row is a row-row update
//     (one multiplier, a sparse axpy over its U tail), a source supernode is
//     a sup-row update (a triangular solve with its dense diagonal block, then
//     a dense matrix-vector product with its U tail);
//   - a row inside a supernode then takes the updates of the earlier rows of
//     its own supernode as soon as each is ready (the pipelined "dual mode"
//     of Sec. 2.2.1 at row granularity), exchanges the largest entry of its
//     diagonal block to the diagonal (supernode diagonal pivoting, Sec. 2.2)
//     and perturbs a pivot below tau (Sec. 2.2);
//   - the row publishes its ready flag with release semantics.
// Claiming in ascending order makes every wait target a row that a running
// warp has already claimed, so the schedule cannot deadlock; every wait is
// still bounded by an iteration limit and reports HYLU_ERR_DEVICE_TIMEOUT.
//
// Storage: row i's L values (by position) are contiguous; every node (a
// supernode or a standalone row) keeps a dense panel s x (s + |tail|) whose
// diagonal block is stored by column LABEL (pre-pivot column), so that later
// exchanges never move data; consumers read position p through piv[p].
#include <algorithm>
#include <cstdio>

#include "kernels.cuh"
#include "../../include/hylu.h"

namespace hylu {

namespace {
constexpr int WARPS = 8;          // warps per block of the persistent kernels
constexpr int SN_SMEM = 256;      // largest supernode held in shared memory
constexpr unsigned FULL = 0xffffffffu;
int64_t g_launches = 0;

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

// All lanes wait (bounded) until *flag == gen.  Returns false when the limit
// expired or another warp already raised an error; the first expiry records
// HYLU_ERR_DEVICE_TIMEOUT and the row/node waited on.
__device__ __forceinline__ bool warp_wait(const int* flag, int gen, int* status, int who,
                                          long long limit) {
    int ok = 1;
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
        }
    }
    return __all_sync(FULL, ok) != 0;
}

__device__ __forceinline__ double* slot_ptr(double* xl, double* xu, int nL, int sl) {
    return sl < nL ? xl + sl : xu + (sl - nL);
}

// -------------------------------------------------------------- reset
__global__ void reset_kernel(int32_t* piv, int32_t* pinv, int32_t n) {
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

// -------------------------------------------------------------- factor
__global__ void __launch_bounds__(WARPS * 32)
factor_kernel(DevPlan P, const double* __restrict__ vals, double* __restrict__ dinv, int gen,
              double tau_rel, long long limit) {
    __shared__ double lbuf[WARPS][SN_SMEM];
    __shared__ int pbuf[WARPS][SN_SMEM];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double* lb = lbuf[wid];
    int* pb = pbuf[wid];
    int* pos = P.pos + (size_t)(blockIdx.x * WARPS + wid) * (size_t)P.n;
    const double amax = __longlong_as_double(*reinterpret_cast<const long long*>(P.status + ST_AMAX));
    const double tau = tau_rel * amax;
    for (;;) {
        int i = 0;
        if (lane == 0) i = atomicAdd(P.status + ST_CNT_F, 1);
        i = __shfl_sync(FULL, i, 0);
        if (i >= P.n) return;
        if (ld_relaxed(P.status + ST_ERR) != 0) return;
        const int D = P.node_of[i];
        const int r = P.sn_start[D], e = P.sn_start[D + 1] - 1, s = e - r + 1;
        const int64_t l0 = P.row_lptr[i];
        const int nL = (int)(P.row_lptr[i + 1] - l0);
        const int64_t t0 = P.node_tail_off[D];
        const int nT = (int)(P.node_tail_off[D + 1] - t0);
        const int w = s + nT;
        double* xl = P.lval + l0;
        double* xu = P.pval + P.node_panel_off[D] + (int64_t)(i - r) * w;
        const int32_t* lc = P.lcols + l0;
        const int32_t* tc = P.tcols + t0;
        // ---- clear the row, column -> slot map, scatter Ahat(i,:) (value scatter)
        for (int t = lane; t < nL; t += 32) { xl[t] = 0.0; pos[lc[t]] = t; }
        for (int t = lane; t < w; t += 32) xu[t] = 0.0;
        for (int t = lane; t < s; t += 32) pos[r + t] = nL + t;
        for (int t = lane; t < nT; t += 32) pos[tc[t]] = nL + s + t;
        __syncwarp();
        for (int64_t q = P.ah_rp[i] + lane; q < P.ah_rp[i + 1]; q += 32) {
            const int sl = P.ah_slot[q];
            *slot_ptr(xl, xu, nL, sl) = vals[P.ah_src[q]] * P.ah_scale[q];
        }
        __syncwarp();
        // ---- updates from earlier nodes, ascending.  The metadata and ready
        //      flags of the next 32 L entries are fetched at once (one lane
        //      each); a source found ready then needs no further wait.
        int t = 0;
        while (t < nL) {
            const int tq = t + lane;
            int kq = 0, eq = 0, sq = 1, nTq = 0, okq = 1;
            int64_t tq0 = 0, pq0 = 0;
            if (tq < nL) {
                kq = lc[tq];
                const int Sq = P.node_of[kq];
                const int rq = P.sn_start[Sq];
                eq = P.sn_start[Sq + 1] - 1;
                sq = eq - rq + 1;
                tq0 = P.node_tail_off[Sq];
                nTq = (int)(P.node_tail_off[Sq + 1] - tq0);
                pq0 = P.node_panel_off[Sq];
                okq = (ld_acquire(P.ready + eq) == gen);
            }
            const unsigned rmask = __ballot_sync(FULL, okq);
            const int cend = min(32, nL - t);
            int q = 0;
            while (q < cend) {
                const int k = __shfl_sync(FULL, kq, q);
                const int eS = __shfl_sync(FULL, eq, q);
                const int sS = __shfl_sync(FULL, sq, q);
                const int nTS = __shfl_sync(FULL, nTq, q);
                const int64_t tS = __shfl_sync(FULL, tq0, q);
                const int64_t pS = __shfl_sync(FULL, pq0, q);
                if (!((rmask >> q) & 1u))
                    if (!warp_wait(P.ready + eS, gen, P.status, eS, limit)) return;
                const int tt = t + q;
                const int wS = sS + nTS;
                const double* __restrict__ U = P.pval + pS;
                const int32_t* __restrict__ tcS = P.tcols + tS;
                if (sS == 1) {
                    // row-row: l = x_k / u_kk, x[U(k, >k)] -= l * U(k, >k)
                    const double l = xl[tt] * dinv[k];
                    for (int j0 = 0; j0 < nTS; j0 += 128) {
                        int c[4];
                        double u[4], xv[4];
                        double* px[4];
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            const int j = j0 + m * 32 + lane;
                            c[m] = (j < nTS) ? tcS[j] : -1;
                            u[m] = (j < nTS) ? U[1 + j] : 0.0;
                        }
#pragma unroll
                        for (int m = 0; m < 4; ++m) px[m] = (c[m] >= 0) ? slot_ptr(xl, xu, nL, pos[c[m]]) : nullptr;
#pragma unroll
                        for (int m = 0; m < 4; ++m) xv[m] = px[m] ? *px[m] : 0.0;
#pragma unroll
                        for (int m = 0; m < 4; ++m) if (px[m]) *px[m] = xv[m] - l * u[m];
                    }
                    __syncwarp();
                    if (lane == 0) xl[tt] = l;
                    __syncwarp();
                    q += 1;
                } else {
                    // sup-row: l * U_SS = x_S (by position), x[T_S] -= l * U_S,T_S
                    const int rS = eS - sS + 1;
                    for (int p = lane; p < sS; p += 32) {
                        const int lab = P.piv[rS + p] - rS;
                        pb[p] = lab;
                        lb[p] = xl[tt + lab];
                    }
                    __syncwarp();
                    for (int p = 0; p < sS; ++p) {
                        const double* Up = U + (int64_t)p * wS;
                        const double lp = lb[p] * dinv[rS + p];
                        __syncwarp();
                        for (int qq = p + 1 + lane; qq < sS; qq += 32) lb[qq] -= lp * Up[pb[qq]];
                        if (lane == 0) lb[p] = lp;
                        __syncwarp();
                    }
                    for (int j = lane; j < nTS; j += 32) {
                        const double* Uj = U + sS + j;
                        const int sl = pos[tcS[j]];
                        double acc0 = 0.0, acc1 = 0.0;
                        int p = 0;
                        for (; p + 1 < sS; p += 2) {
                            acc0 = fma(lb[p], Uj[(int64_t)p * wS], acc0);
                            acc1 = fma(lb[p + 1], Uj[(int64_t)(p + 1) * wS], acc1);
                        }
                        if (p < sS) acc0 = fma(lb[p], Uj[(int64_t)p * wS], acc0);
                        *slot_ptr(xl, xu, nL, sl) -= acc0 + acc1;
                    }
                    for (int p = lane; p < sS; p += 32) xl[tt + p] = lb[p];
                    __syncwarp();
                    q += sS;
                }
            }
            t += q;
        }
        if (s > 1) {
            // ---- earlier rows of the own supernode, each as soon as it is ready
            const double* Ub = P.pval + P.node_panel_off[D];
            for (int k = r; k < i; ++k) {
                if (!warp_wait(P.ready + k, gen, P.status, k, limit)) return;
                const int lab = ld_relaxed(P.piv + k) - r;
                const double* Uk = Ub + (int64_t)(k - r) * w;
                const double l = xu[lab] * dinv[k];
                for (int c = lane; c < s; c += 32)
                    if (c != lab && ld_relaxed(P.pinv + r + c) > k) xu[c] -= l * Uk[c];
                for (int j0 = s; j0 < w; j0 += 128) {
                    double u[4], xv[4];
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const int j = j0 + m * 32 + lane;
                        u[m] = (j < w) ? Uk[j] : 0.0;
                        xv[m] = (j < w) ? xu[j] : 0.0;
                    }
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const int j = j0 + m * 32 + lane;
                        if (j < w) xu[j] = xv[m] - l * u[m];
                    }
                }
                __syncwarp();
                if (lane == 0) xu[lab] = l;
                __syncwarp();
            }
            // ---- supernode diagonal pivoting: largest |x| among positions i..e,
            //      first position on ties
            double best = -1.0;
            int bp = i;
            for (int p = i + lane; p <= e; p += 32) {
                const double a = fabs(xu[P.piv[p] - r]);
                if (a > best) { best = a; bp = p; }
            }
            for (int off = 16; off; off >>= 1) {
                const double ob = __shfl_down_sync(FULL, best, off);
                const int op = __shfl_down_sync(FULL, bp, off);
                if (ob > best || (ob == best && op < bp)) { best = ob; bp = op; }
            }
            bp = __shfl_sync(FULL, bp, 0);
            if (lane == 0 && bp != i) {
                const int a = P.piv[i], b = P.piv[bp];
                P.piv[i] = b; P.piv[bp] = a;
                P.pinv[b] = i; P.pinv[a] = bp;
            }
            __syncwarp();
        }
        // ---- pivot, small-pivot perturbation, publish
        if (lane == 0) {
            const int dl = (s > 1) ? (P.piv[i] - r) : 0;
            double u = xu[dl];
            if (fabs(u) < tau) {
                u = (u >= 0.0) ? tau : -tau;
                xu[dl] = u;
                atomicAdd(P.status + ST_NPERT, 1);
            }
            dinv[i] = 1.0 / u;
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release(P.ready + i, gen);
    }
}

// -------------------------------------------------------------- solve
__global__ void permute_in_kernel(int32_t n, const int32_t* __restrict__ rowperm,
                                  const double* __restrict__ dr, const double* __restrict__ b,
                                  double* __restrict__ bh, int nrhs, int ld) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)n * nrhs;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int rr = (int)(q / n), i = (int)(q % n);
        const int o = rowperm[i];
        bh[q] = dr[o] * b[(int64_t)rr * ld + o];
    }
}

__global__ void permute_out_kernel(int32_t n, const int32_t* __restrict__ colperm,
                                   const double* __restrict__ dc, const double* __restrict__ xh,
                                   double* __restrict__ x, int nrhs, int ld) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)n * nrhs;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int rr = (int)(q / n), k = (int)(q % n);
        const int o = colperm[k];
        x[(int64_t)rr * ld + o] = dc[o] * xh[q];
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

// Forward substitution L z = bhat (unit L, by position); z holds bhat on
// entry.  Every warp claims the next row: it subtracts the row's L list
// (waiting for each source node), and the warp of the LAST row of a
// supernode then solves the unit lower block once all rows of the supernode
// have their external part.  Right-hand sides are columns of z (stride n).
__global__ void __launch_bounds__(WARPS * 32)
fwd_kernel(DevPlan P, double* __restrict__ z, int nrhs, int gen, long long limit) {
    const int lane = threadIdx.x & 31;
    const int n = P.n;
    for (;;) {
        int i = 0;
        if (lane == 0) i = atomicAdd(P.status + ST_CNT_FWD, 1);
        i = __shfl_sync(FULL, i, 0);
        if (i >= n) return;
        if (ld_relaxed(P.status + ST_ERR) != 0) return;
        const int D = P.node_of[i];
        const int r = P.sn_start[D], e = P.sn_start[D + 1] - 1, s = e - r + 1;
        const int64_t l0 = P.row_lptr[i], l1 = P.row_lptr[i + 1];
        int ok = 1;
        for (int64_t t = l0 + lane; t < l1 && ok; t += 32) {
            const int S = P.node_of[P.lcols[t]];
            ok = lane_wait(P.fwd_ready + S, gen, P.status, S, limit);
        }
        if (!__all_sync(FULL, ok)) return;
        for (int rr = 0; rr < nrhs; ++rr) {
            double* zr = z + (int64_t)rr * n;
            double a0 = 0.0, a1 = 0.0;
            int64_t t = l0 + lane;
            for (; t + 32 < l1; t += 64) {
                a0 = fma(P.lval[t], zr[P.lcols[t]], a0);
                a1 = fma(P.lval[t + 32], zr[P.lcols[t + 32]], a1);
            }
            if (t < l1) a0 = fma(P.lval[t], zr[P.lcols[t]], a0);
            double a = a0 + a1;
            for (int off = 16; off; off >>= 1) a += __shfl_xor_sync(FULL, a, off);
            if (lane == 0) zr[i] -= a;
        }
        __threadfence();
        __syncwarp();
        if (s == 1) {
            if (lane == 0) st_release(P.fwd_ready + D, gen);
            continue;
        }
        if (lane == 0) st_release(P.fwd_row + i, gen);
        if (i != e) continue;
        // last row of the supernode: block solve once every row has its external part
        ok = 1;
        for (int k = r + lane; k < e && ok; k += 32) ok = lane_wait(P.fwd_row + k, gen, P.status, k, limit);
        if (!__all_sync(FULL, ok)) return;
        const int w = s + (int)(P.node_tail_off[D + 1] - P.node_tail_off[D]);
        const double* Ub = P.pval + P.node_panel_off[D];
        for (int rr = 0; rr < nrhs; ++rr) {
            double* zr = z + (int64_t)rr * n;
            for (int ii = r + 1; ii <= e; ++ii) {
                const double* Ui = Ub + (int64_t)(ii - r) * w;
                double a = 0.0;
                for (int k = r + lane; k < ii; k += 32) a = fma(Ui[P.piv[k] - r], zr[k], a);
                for (int off = 16; off; off >>= 1) a += __shfl_xor_sync(FULL, a, off);
                if (lane == 0) zr[ii] -= a;
                __syncwarp();
            }
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release(P.fwd_ready + D, gen);
    }
}

// Backward substitution U w = z by position, rows in descending order; the
// solution is written by label: xh[piv[p]] = w_p.  Every warp claims the next
// row (from the bottom), subtracts its U tail; the warp of the FIRST row of a
// supernode then back-substitutes the block.  z is overwritten.
__global__ void __launch_bounds__(WARPS * 32)
bwd_kernel(DevPlan P, const double* __restrict__ dinv, double* __restrict__ z,
           double* __restrict__ xh, int nrhs, int gen, long long limit) {
    const int lane = threadIdx.x & 31;
    const int n = P.n;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(P.status + ST_CNT_BWD, 1);
        t = __shfl_sync(FULL, t, 0);
        if (t >= n) return;
        if (ld_relaxed(P.status + ST_ERR) != 0) return;
        const int i = n - 1 - t;
        const int D = P.node_of[i];
        const int r = P.sn_start[D], e = P.sn_start[D + 1] - 1, s = e - r + 1;
        const int64_t t0 = P.node_tail_off[D];
        const int nT = (int)(P.node_tail_off[D + 1] - t0);
        const int w = s + nT;
        const int32_t* tc = P.tcols + t0;
        const double* Ui = P.pval + P.node_panel_off[D] + (int64_t)(i - r) * w;
        int ok = 1;
        for (int j = lane; j < nT && ok; j += 32) {
            const int S = P.node_of[tc[j]];
            ok = lane_wait(P.bwd_ready + S, gen, P.status, S, limit);
        }
        if (!__all_sync(FULL, ok)) return;
        for (int rr = 0; rr < nrhs; ++rr) {
            double* zr = z + (int64_t)rr * n;
            const double* xr = xh + (int64_t)rr * n;
            double a0 = 0.0, a1 = 0.0;
            int j = lane;
            for (; j + 32 < nT; j += 64) {
                a0 = fma(Ui[s + j], xr[tc[j]], a0);
                a1 = fma(Ui[s + j + 32], xr[tc[j + 32]], a1);
            }
            if (j < nT) a0 = fma(Ui[s + j], xr[tc[j]], a0);
            double a = a0 + a1;
            for (int off = 16; off; off >>= 1) a += __shfl_xor_sync(FULL, a, off);
            if (lane == 0) {
                if (s == 1) xh[(int64_t)rr * n + i] = (zr[i] - a) * dinv[i];
                else zr[i] -= a;
            }
        }
        __threadfence();
        __syncwarp();
        if (s == 1) {
            if (lane == 0) st_release(P.bwd_ready + D, gen);
            continue;
        }
        if (lane == 0) st_release(P.bwd_row + i, gen);
        if (i != r) continue;
        ok = 1;
        for (int k = r + 1 + lane; k <= e && ok; k += 32) ok = lane_wait(P.bwd_row + k, gen, P.status, k, limit);
        if (!__all_sync(FULL, ok)) return;
        const double* Ub = P.pval + P.node_panel_off[D];
        for (int rr = 0; rr < nrhs; ++rr) {
            double* zr = z + (int64_t)rr * n;
            double* xr = xh + (int64_t)rr * n;
            for (int ii = e; ii >= r; --ii) {
                const double* Uii = Ub + (int64_t)(ii - r) * w;
                double a = 0.0;
                for (int p = ii + 1 + lane; p <= e; p += 32) a = fma(Uii[P.piv[p] - r], zr[p], a);
                for (int off = 16; off; off >>= 1) a += __shfl_xor_sync(FULL, a, off);
                if (lane == 0) zr[ii] = (zr[ii] - a) * dinv[ii];
                __syncwarp();
            }
            for (int p = r + lane; p <= e; p += 32) xr[P.piv[p]] = zr[p];
            __syncwarp();
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release(P.bwd_ready + D, gen);
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

int64_t launches() { return g_launches; }
void count_launch() { ++g_launches; }

static int check(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "hylu: %s: %s\n", what, cudaGetErrorString(e));
        return HYLU_ERR_CUDA;
    }
    return HYLU_OK;
}

int warps_per_block() { return WARPS; }

int factor_grid(int device) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, factor_kernel, WARPS * 32, 0);
    if (per < 1) per = 1;
    if (per > 4) per = 4;
    return sms * per;
}

int launch_reset(int32_t* status, int32_t* piv, int32_t* pinv, int32_t n, cudaStream_t st) {
    if (cudaMemsetAsync(status, 0, sizeof(int32_t) * ST_WORDS, st) != cudaSuccess) return HYLU_ERR_CUDA;
    int blocks = (int)std::min<int64_t>(4096, ((int64_t)n + 255) / 256 + 1);
    reset_kernel<<<blocks, 256, 0, st>>>(piv, pinv, n);
    count_launch();
    return check("reset");
}

int launch_factor(const DevPlan& P, const double* d_vals, int64_t nnz_a, int32_t gen,
                  double tau_rel, long long spin_limit, int grid, cudaStream_t st, cudaEvent_t e0,
                  cudaEvent_t e1) {
    int blocks = (int)std::min<int64_t>(2048, (nnz_a + 255) / 256 + 1);
    amax_kernel<<<blocks, 256, 0, st>>>(d_vals, P.ah_src, P.ah_scale, nnz_a, P.status);
    count_launch();
    if (e0) cudaEventRecord(e0, st);
    factor_kernel<<<grid, WARPS * 32, 0, st>>>(P, d_vals, P.dinv, gen, tau_rel, spin_limit);
    count_launch();
    if (e1) cudaEventRecord(e1, st);
    return check("factor");
}

int launch_solve(const DevPlan& P, const double* d_b, double* d_x, double* d_z, double* d_xh,
                 const int32_t* rowperm, const int32_t* colperm, const double* dr, const double* dc,
                 int nrhs, int ld, int32_t gen, long long spin_limit, int grid, cudaStream_t st,
                 cudaEvent_t e0, cudaEvent_t e1) {
    const int64_t tot = (int64_t)P.n * nrhs;
    const int eb = (int)std::min<int64_t>(4096, (tot + 255) / 256 + 1);
    if (cudaMemsetAsync(P.status + ST_CNT_FWD, 0, sizeof(int32_t) * 2, st) != cudaSuccess) return HYLU_ERR_CUDA;
    permute_in_kernel<<<eb, 256, 0, st>>>(P.n, rowperm, dr, d_b, d_z, nrhs, ld);
    count_launch();
    const int blocks = grid;
    if (e0) cudaEventRecord(e0, st);
    fwd_kernel<<<blocks, WARPS * 32, 0, st>>>(P, d_z, nrhs, gen, spin_limit);
    count_launch();
    bwd_kernel<<<blocks, WARPS * 32, 0, st>>>(P, P.dinv, d_z, d_xh, nrhs, gen, spin_limit);
    count_launch();
    if (e1) cudaEventRecord(e1, st);
    permute_out_kernel<<<eb, 256, 0, st>>>(P.n, colperm, dc, d_xh, d_x, nrhs, ld);
    count_launch();
    return check("solve");
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

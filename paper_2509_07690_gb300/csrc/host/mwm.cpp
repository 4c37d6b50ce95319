// Maximum-product bipartite matching with dual scalings (HYLU Sec. 2.1, static
// pivoting by maximum weighted matching [8]).
//
// Weights: c_ij = log(max_k |a_ik|) - log|a_ij| >= 0 on the nonzero values.
// A minimum-cost perfect matching on c maximizes prod |a_{i,match(i)}|.  It is
// found by successive shortest augmenting paths (Dijkstra on reduced costs
// c_ij - u_i - v_j >= 0).  At the optimum, reduced costs are 0 on matched
// edges, so dr_i = exp(u_i) / max_k |a_ik| and dc_j = exp(v_j) make every
// scaled entry |dr_i a_ij dc_j| = exp(-(c_ij - u_i - v_j)) <= 1 with equality
// on the matching: the diagonal becomes +-1 after the row permutation.
#include <cmath>
#include <limits>
#include <queue>
#include <vector>

#include "preprocess.hpp"

namespace hylu {

bool max_product_matching(int32_t n, const int64_t* rp, const int32_t* ci, const double* v,
                          std::vector<int32_t>& match_col, std::vector<double>& dr,
                          std::vector<double>& dc) {
    const double INF = std::numeric_limits<double>::infinity();
    std::vector<double> rmax(n, 0.0), cost(rp[n]);
    for (int32_t i = 0; i < n; ++i)
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) rmax[i] = std::max(rmax[i], std::fabs(v[q]));
    for (int32_t i = 0; i < n; ++i) {
        if (rmax[i] == 0.0) return false;
        double lm = std::log(rmax[i]);
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
            cost[q] = (v[q] != 0.0) ? lm - std::log(std::fabs(v[q])) : INF;
    }
    std::vector<double> u(n, 0.0), vv(n, INF);
    // v_j = min_i c_ij, u_i = min_j (c_ij - v_j)
    for (int32_t i = 0; i < n; ++i)
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) vv[ci[q]] = std::min(vv[ci[q]], cost[q]);
    for (int32_t j = 0; j < n; ++j) if (vv[j] == INF) return false;  // empty column
    std::vector<int32_t> mrow(n, -1), mcol(n, -1);   // mrow[i] = column of row i; mcol[j] = row
    for (int32_t i = 0; i < n; ++i) {
        double best = INF; int32_t bj = -1;
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
            double r = cost[q] - vv[ci[q]];
            if (r < best || (r == best && bj >= 0 && mcol[ci[q]] < 0 && mcol[bj] >= 0)) { best = r; bj = ci[q]; }
        }
        u[i] = best;
        // greedy: a free column with zero reduced cost
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
            int32_t j = ci[q];
            if (mcol[j] < 0 && cost[q] - u[i] - vv[j] <= 0.0) { mrow[i] = j; mcol[j] = i; break; }
        }
    }
    // successive shortest augmenting paths from every free row
    std::vector<double> dist(n, INF);
    std::vector<int32_t> pred(n, -1), touched, done_cols;
    std::vector<char> final_(n, 0);
    std::vector<double> rowd(n, 0.0);
    typedef std::pair<double, int32_t> QE;
    for (int32_t i0 = 0; i0 < n; ++i0) {
        if (mrow[i0] >= 0) continue;
        std::priority_queue<QE, std::vector<QE>, std::greater<QE>> pq;
        touched.clear(); done_cols.clear();
        std::vector<int32_t> rows_in_tree;
        rows_in_tree.push_back(i0);
        rowd[i0] = 0.0;
        auto relax_row = [&](int32_t i, double di) {
            for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
                int32_t j = ci[q];
                if (final_[j] || cost[q] == INF) continue;
                double nd = di + (cost[q] - u[i] - vv[j]);
                if (nd < dist[j]) {
                    if (dist[j] == INF) touched.push_back(j);
                    dist[j] = nd; pred[j] = i; pq.push(QE(nd, j));
                }
            }
        };
        relax_row(i0, 0.0);
        int32_t jf = -1; double delta = INF;
        while (!pq.empty()) {
            QE t = pq.top(); pq.pop();
            int32_t j = t.second;
            if (final_[j] || t.first > dist[j]) continue;
            final_[j] = 1; done_cols.push_back(j);
            if (mcol[j] < 0) { jf = j; delta = dist[j]; break; }
            int32_t i = mcol[j];
            rowd[i] = dist[j];
            rows_in_tree.push_back(i);
            relax_row(i, dist[j]);
        }
        if (jf < 0) return false;  // structurally singular
        // dual update keeps reduced costs >= 0 and makes the path tight
        for (int32_t j : done_cols) if (j != jf) vv[j] -= (delta - dist[j]);
        for (int32_t i : rows_in_tree) u[i] += (delta - rowd[i]);
        // augment
        int32_t j = jf;
        while (j >= 0) {
            int32_t i = pred[j];
            int32_t jprev = mrow[i];
            mrow[i] = j; mcol[j] = i;
            j = (i == i0) ? -1 : jprev;
        }
        for (int32_t t : touched) { dist[t] = INF; pred[t] = -1; final_[t] = 0; }
        for (int32_t t : done_cols) final_[t] = 0;
    }
    // make u exact on matched edges (reduced cost 0) to limit rounding drift
    for (int32_t i = 0; i < n; ++i) {
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
            if (ci[q] == mrow[i]) { u[i] = cost[q] - vv[mrow[i]]; break; }
    }
    match_col = mrow;
    dr.resize(n); dc.resize(n);
    for (int32_t i = 0; i < n; ++i) dr[i] = std::exp(u[i]) / rmax[i];
    for (int32_t j = 0; j < n; ++j) dc[j] = std::exp(vv[j]);
    return true;
}

}  // namespace hylu

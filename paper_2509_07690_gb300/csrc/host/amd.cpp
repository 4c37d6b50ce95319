// Approximate minimum degree ordering (HYLU Sec. 2.1, AMD [9]: Amestoy, Davis
// and Duff, SIAM J. Matrix Anal. Appl. 17(4), 1996), written from the
// published description:
//   - quotient graph: uneliminated variables carry their adjacent elements and
//     variables; every eliminated pivot becomes an element holding its
//     variable set L_p;
//   - approximate external degree  d_i = min(n_left - |i|, d_i + |L_p \ i|,
//     |A_i \ i| + |L_p \ i| + sum_{e in E_i \ p} |L_e \ L_p|);
//   - element absorption (elements adjacent to p merge into p, and any element
//     with L_e contained in L_p is absorbed: aggressive absorption);
//   - indistinguishable variables merge into supervariables (hash + compare);
//   - rows denser than max(16, dense_factor * sqrt(n)) are ordered last;
//   - the final order is a postorder of the assembly tree, so that chains of
//     the elimination tree end up consecutive (supernodes are runs of
//     consecutive rows, Sec. 2.2).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "preprocess.hpp"

namespace hylu {

namespace {

enum : int8_t { VAR = 0, ELEM = 1, MERGED = 2, DEAD = 3, DENSE = 4 };

struct Buckets {
    std::vector<int32_t> head, next, prev, deg;
    int32_t mindeg = 0;
    explicit Buckets(int32_t n) : head(n + 1, -1), next(n, -1), prev(n, -1), deg(n, 0) {}
    void insert(int32_t i, int32_t d) {
        deg[i] = d;
        next[i] = head[d]; prev[i] = -1;
        if (head[d] >= 0) prev[head[d]] = i;
        head[d] = i;
        if (d < mindeg) mindeg = d;
    }
    void remove(int32_t i) {
        int32_t d = deg[i];
        if (prev[i] >= 0) next[prev[i]] = next[i]; else head[d] = next[i];
        if (next[i] >= 0) prev[next[i]] = prev[i];
        next[i] = prev[i] = -1;
    }
    int32_t pop_min(int32_t maxd) {
        while (mindeg <= maxd && head[mindeg] < 0) ++mindeg;
        if (mindeg > maxd) return -1;
        int32_t i = head[mindeg];
        remove(i);
        return i;
    }
};

}  // namespace

void amd_order(const CsrPattern& g, std::vector<int32_t>& perm, double dense_factor) {
    const int32_t n = g.n;
    perm.clear();
    perm.reserve(n);
    if (n == 0) return;
    std::vector<std::vector<int32_t>> E(n), A(n), L(n);
    std::vector<int8_t> st(n, VAR);
    std::vector<int32_t> nv(n, 1), parent(n, -1), chain_next(n, -1), chain_last(n);
    // per element e: lw = weighted |L_e|, w = |L_e \ L_p| while flag == the
    // current stamp (one record, so an element costs one cache line)
    struct ElemW { int32_t lw, w, flag; };
    std::vector<ElemW> ew(n, ElemW{0, 0, -1});
    std::vector<int32_t> mark(n, -1);
    std::vector<int32_t> elim_order;        // pivots (principal variables) in order
    for (int32_t i = 0; i < n; ++i) chain_last[i] = i;

    const int32_t dense_thr = std::max<int32_t>(16, (int32_t)(dense_factor * std::sqrt((double)n)));
    std::vector<int32_t> dense;
    for (int32_t i = 0; i < n; ++i) {
        int64_t d = g.rp[i + 1] - g.rp[i];
        if (d > dense_thr && n > 32) { st[i] = DENSE; dense.push_back(i); }
    }
    Buckets bk(n);
    for (int32_t i = 0; i < n; ++i) {
        if (st[i] != VAR) continue;
        for (int64_t q = g.rp[i]; q < g.rp[i + 1]; ++q) {
            int32_t j = g.ci[q];
            if (j != i && st[j] == VAR) A[i].push_back(j);
        }
        bk.insert(i, (int32_t)A[i].size());
    }
    int64_t nleft = n - (int64_t)dense.size();
    int32_t stamp = 0;
    std::vector<int32_t> Lp;
    std::vector<int64_t> hashv(n);

    while (nleft > 0) {
        int32_t p = bk.pop_min(n);
        if (p < 0) break;
        ++stamp;
        // ---- new element L_p = (A_p U union_{e in E_p} L_e) \ p, principal variables only
        Lp.clear();
        mark[p] = stamp;
        for (int32_t e : E[p]) {
            if (st[e] != ELEM) continue;
            for (int32_t j : L[e])
                if (st[j] == VAR && mark[j] != stamp) { mark[j] = stamp; Lp.push_back(j); }
            st[e] = DEAD;                   // absorbed into p
            parent[e] = p;
            std::vector<int32_t>().swap(L[e]);
        }
        for (int32_t j : A[p])
            if (st[j] == VAR && mark[j] != stamp) { mark[j] = stamp; Lp.push_back(j); }
        std::vector<int32_t>().swap(E[p]);
        std::vector<int32_t>().swap(A[p]);
        st[p] = ELEM;
        elim_order.push_back(p);
        nleft -= nv[p];
        int64_t degp = 0;
        for (int32_t j : Lp) { degp += nv[j]; bk.remove(j); }
        // ---- |L_e \ L_p| for elements adjacent to L_p
        for (int32_t j : Lp) {
            for (int32_t e : E[j]) {
                if (st[e] != ELEM || e == p) continue;
                ElemW& x = ew[e];
                if (x.flag != stamp) { x.flag = stamp; x.w = x.lw - nv[j]; }
                else x.w -= nv[j];
            }
        }
        // ---- degree update, pruning, aggressive absorption
        //      (the supervariable hash, the sum of the pruned E_j and A_j, is
        //      taken in the same pass)
        for (int32_t j : Lp) {
            int64_t sum = 0, h = p;
            std::vector<int32_t>& Ej = E[j];
            size_t k = 0;
            for (int32_t e : Ej) {
                if (st[e] != ELEM || e == p) continue;
                const ElemW& x = ew[e];
                int64_t we = (x.flag == stamp) ? x.w : x.lw;
                if (we == 0) { st[e] = DEAD; parent[e] = p; std::vector<int32_t>().swap(L[e]); continue; }
                sum += we;
                h += e;
                Ej[k++] = e;
            }
            Ej.resize(k);
            Ej.push_back(p);
            std::vector<int32_t>& Aj = A[j];
            k = 0;
            for (int32_t a : Aj) {
                if (st[a] != VAR || mark[a] == stamp) continue;   // in L_p, p itself, merged, dense
                sum += nv[a];
                h += a;
                Aj[k++] = a;
            }
            Aj.resize(k);
            hashv[j] = h;
            int64_t ext = degp - nv[j];
            int64_t d = std::min<int64_t>({nleft - nv[j], (int64_t)bk.deg[j] + ext, sum + ext});
            if (d < 0) d = 0;
            bk.deg[j] = (int32_t)d;
        }
        // ---- supervariable detection among L_p
        std::vector<int32_t> order(Lp);
        std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
            return hashv[a] != hashv[b] ? hashv[a] < hashv[b] : a < b;
        });
        for (size_t s = 0; s < order.size();) {
            size_t t = s;
            while (t < order.size() && hashv[order[t]] == hashv[order[s]]) ++t;
            for (size_t a = s; a < t; ++a) {
                int32_t i = order[a];
                if (st[i] != VAR) continue;
                ++stamp;
                bool cand = false;              // mark only when a candidate could match
                for (size_t b = a + 1; b < t && !cand; ++b) {
                    int32_t j = order[b];
                    cand = st[j] == VAR && E[j].size() == E[i].size() && A[j].size() == A[i].size();
                }
                if (!cand) continue;
                for (int32_t e : E[i]) mark[e] = stamp;
                for (int32_t x : A[i]) mark[x] = stamp;
                for (size_t b = a + 1; b < t; ++b) {
                    int32_t j = order[b];
                    if (st[j] != VAR || E[j].size() != E[i].size() || A[j].size() != A[i].size()) continue;
                    bool same = true;
                    for (int32_t e : E[j]) if (mark[e] != stamp) { same = false; break; }
                    if (same) for (int32_t x : A[j]) if (mark[x] != stamp) { same = false; break; }
                    if (!same) continue;
                    // merge j into i
                    nv[i] += nv[j];
                    bk.deg[i] = std::max<int32_t>(0, bk.deg[i] - nv[j]);
                    nv[j] = 0;
                    st[j] = MERGED;
                    chain_next[chain_last[i]] = j;
                    chain_last[i] = chain_last[j];
                    std::vector<int32_t>().swap(E[j]);
                    std::vector<int32_t>().swap(A[j]);
                }
            }
            s = t;
        }
        // ---- element p, reinsert principal variables
        std::vector<int32_t>& Le = L[p];
        int64_t lwp = 0;
        for (int32_t j : Lp) {
            if (st[j] != VAR) continue;
            Le.push_back(j);
            lwp += nv[j];
            int32_t d = bk.deg[j];
            if (d > nleft) d = (int32_t)nleft;
            bk.insert(j, d);
        }
        ew[p].lw = (int32_t)lwp;
        stamp += 1;
    }
    // ---- postorder of the assembly tree (element parent = absorbing pivot)
    std::vector<int32_t> first_child(n, -1), sibling(n, -1);
    std::vector<int32_t> roots;
    for (auto it = elim_order.rbegin(); it != elim_order.rend(); ++it) {
        int32_t e = *it;
        if (parent[e] >= 0) { sibling[e] = first_child[parent[e]]; first_child[parent[e]] = e; }
    }
    for (int32_t e : elim_order) if (parent[e] < 0) roots.push_back(e);
    std::vector<int32_t> stack, child_it(n, -2);
    for (int32_t r : roots) {
        stack.push_back(r);
        while (!stack.empty()) {
            int32_t x = stack.back();
            if (child_it[x] == -2) child_it[x] = first_child[x];
            int32_t c = child_it[x];
            if (c >= 0) { child_it[x] = sibling[c]; stack.push_back(c); continue; }
            stack.pop_back();
            for (int32_t m = x; m >= 0; m = chain_next[m]) perm.push_back(m);
        }
    }
    for (int32_t d : dense) perm.push_back(d);
    // any vertex not yet placed (defensive: isolated supervariable chains)
    if ((int32_t)perm.size() != n) {
        std::vector<char> seen(n, 0);
        for (int32_t x : perm) seen[x] = 1;
        for (int32_t i = 0; i < n; ++i) if (!seen[i]) perm.push_back(i);
    }
}

CsrPattern symmetrize(int32_t n, const int64_t* rp, const int32_t* ci) {
    std::vector<int64_t> cnt(n + 1, 0);
    for (int32_t i = 0; i < n; ++i)
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
            int32_t j = ci[q];
            if (j == i) continue;
            cnt[i + 1]++; cnt[j + 1]++;
        }
    for (int32_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    std::vector<int32_t> tmp(cnt[n]);
    std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
    for (int32_t i = 0; i < n; ++i)
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
            int32_t j = ci[q];
            if (j == i) continue;
            tmp[pos[i]++] = j; tmp[pos[j]++] = i;
        }
    CsrPattern g;
    g.n = n;
    g.rp.assign(n + 1, 0);
    g.ci.reserve(tmp.size());
    for (int32_t i = 0; i < n; ++i) {
        std::sort(tmp.begin() + cnt[i], tmp.begin() + cnt[i + 1]);
        int32_t last = -1;
        for (int64_t q = cnt[i]; q < cnt[i + 1]; ++q)
            if (tmp[q] != last) { g.ci.push_back(tmp[q]); last = tmp[q]; }
        g.rp[i + 1] = (int64_t)g.ci.size();
    }
    return g;
}

}  // namespace hylu

// Nested dissection ordering (HYLU Sec. 2.1 uses a METIS-based modified
// nested dissection [11]; METIS itself is not used here).  Each subgraph is
// split by a level structure grown from a pseudo-peripheral vertex: the level
// that best balances the two sides is the vertex separator, thinned by moving
// separator vertices with no neighbour on the far side back to the near side.
// Both sides are ordered recursively, then the separator last.  Subgraphs of
// at most leaf_size vertices are ordered by AMD.  Disconnected subgraphs are
// ordered component by component.  Vertices denser than
// max(16, dense_factor sqrt(n)) (the hub rows of circuit matrices) take part
// in no dissection and are ordered last, as AMD orders them: a hub adjacent
// to most of the graph leaves level structures only a few levels deep, so
// every separator would be huge.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "preprocess.hpp"

namespace hylu {

namespace {

struct NdState {
    const CsrPattern& g;
    std::vector<int32_t> local;     // global -> local index in current subgraph, -1 if outside
    std::vector<int32_t> level;
    std::vector<int32_t>& out;
    int32_t leaf;
    NdState(const CsrPattern& gg, std::vector<int32_t>& o, int32_t lf)
        : g(gg), local(gg.n, -1), level(gg.n, -1), out(o), leaf(lf) {}
};

// BFS over the vertices flagged in `in` (by stamp); returns levels in `lv`
// and the visit order.
static int32_t bfs(const CsrPattern& g, const std::vector<int32_t>& tag, int32_t want, int32_t src,
                   std::vector<int32_t>& lv, std::vector<int32_t>& order) {
    order.clear();
    order.push_back(src);
    lv[src] = 0;
    int32_t maxl = 0;
    for (size_t h = 0; h < order.size(); ++h) {
        int32_t x = order[h];
        for (int64_t q = g.rp[x]; q < g.rp[x + 1]; ++q) {
            int32_t y = g.ci[q];
            if (tag[y] != want || lv[y] >= 0) continue;
            lv[y] = lv[x] + 1;
            maxl = std::max(maxl, lv[y]);
            order.push_back(y);
        }
    }
    return maxl;
}

static void order_leaf(const CsrPattern& g, const std::vector<int32_t>& verts, std::vector<int32_t>& tag,
                       int32_t want, std::vector<int32_t>& out) {
    const int32_t m = (int32_t)verts.size();
    if (m <= 2) { for (int32_t v : verts) out.push_back(v); return; }
    std::vector<int32_t> loc(m);
    // build the induced subgraph
    CsrPattern sg;
    sg.n = m;
    sg.rp.assign(m + 1, 0);
    std::vector<int32_t> idx;
    // map via a temporary of tags: vertices of this leaf carry `want`
    std::vector<std::pair<int32_t, int32_t>> key(m);
    for (int32_t a = 0; a < m; ++a) key[a] = {verts[a], a};
    std::sort(key.begin(), key.end());
    auto find = [&](int32_t v) -> int32_t {
        auto it = std::lower_bound(key.begin(), key.end(), std::make_pair(v, -1));
        return (it != key.end() && it->first == v) ? it->second : -1;
    };
    for (int32_t a = 0; a < m; ++a) {
        int32_t x = verts[a];
        for (int64_t q = g.rp[x]; q < g.rp[x + 1]; ++q) {
            int32_t y = g.ci[q];
            if (tag[y] != want) continue;
            int32_t b = find(y);
            if (b >= 0) sg.ci.push_back(b);
        }
        std::sort(sg.ci.begin() + sg.rp[a], sg.ci.end());
        sg.rp[a + 1] = (int64_t)sg.ci.size();
    }
    std::vector<int32_t> p;
    amd_order(sg, p, 1e9);
    for (int32_t a : p) out.push_back(verts[a]);
}

}  // namespace

void nd_order(const CsrPattern& g, std::vector<int32_t>& perm, int32_t leaf_size, double dense_factor) {
    const int32_t n = g.n;
    perm.clear();
    perm.reserve(n);
    std::vector<int32_t> tag(n, 0), lv(n, -1), order;
    int32_t next_tag = 1;
    // dense vertices carry a tag no subgraph uses, so every search skips them
    const double mean_deg = n > 0 ? (double)g.rp[n] / (double)n : 0.0;
    const int32_t dense_thr =
        std::max<int32_t>(16, (int32_t)std::min(dense_factor * std::sqrt((double)n), 10.0 * mean_deg));
    std::vector<int32_t> dense;
    if (n > 32)
        for (int32_t i = 0; i < n; ++i)
            if (g.rp[i + 1] - g.rp[i] > dense_thr) { dense.push_back(i); tag[i] = -1; }
    // explicit work stack: (vertex list, tag, phase); phase 0 = split, 1 = emit separator
    struct Task { std::vector<int32_t> verts; int32_t tag; bool emit; };
    std::vector<Task> stack;
    std::vector<int32_t> all;
    all.reserve(n - dense.size());
    for (int32_t i = 0; i < n; ++i) if (tag[i] == 0) all.push_back(i);
    if (!all.empty()) stack.push_back({all, 0, false});
    while (!stack.empty()) {
        Task t = std::move(stack.back());
        stack.pop_back();
        if (t.emit) { for (int32_t v : t.verts) perm.push_back(v); continue; }
        const int32_t want = t.tag;
        std::vector<int32_t>& V = t.verts;
        if ((int32_t)V.size() <= leaf_size) { order_leaf(g, V, tag, want, perm); continue; }
        // connected components: take the one holding V[0]; the rest are re-queued
        for (int32_t v : V) lv[v] = -1;
        int32_t root = V[0];
        bfs(g, tag, want, root, lv, order);
        if (order.size() < V.size()) {
            std::vector<int32_t> rest;
            for (int32_t v : V) if (lv[v] < 0) rest.push_back(v);
            int32_t tg = next_tag++;
            for (int32_t v : rest) tag[v] = tg;
            int32_t tc = next_tag++;
            std::vector<int32_t> comp(order);
            for (int32_t v : comp) tag[v] = tc;
            for (int32_t v : V) lv[v] = -1;
            // order: component, then the rest (stack: push rest first)
            stack.push_back({rest, tg, false});
            stack.push_back({comp, tc, false});
            continue;
        }
        // pseudo-peripheral vertex: repeat BFS from the farthest, lowest-degree vertex
        int32_t ecc = -1;
        for (int it = 0; it < 4; ++it) {
            for (int32_t v : V) lv[v] = -1;
            int32_t e = bfs(g, tag, want, root, lv, order);
            if (e <= ecc) break;
            ecc = e;
            int32_t best = order.back();
            int64_t bd = g.rp[best + 1] - g.rp[best];
            for (auto rit = order.rbegin(); rit != order.rend() && lv[*rit] == e; ++rit) {
                int64_t d = g.rp[*rit + 1] - g.rp[*rit];
                if (d < bd) { bd = d; best = *rit; }
            }
            root = best;
        }
        for (int32_t v : V) lv[v] = -1;
        int32_t maxl = bfs(g, tag, want, root, lv, order);
        if (maxl < 2) { order_leaf(g, V, tag, want, perm); continue; }
        std::vector<int64_t> cnt(maxl + 2, 0);
        for (int32_t v : V) cnt[lv[v]]++;
        // level minimising |sep| * imbalance penalty among levels near the middle
        int64_t below = 0, total = (int64_t)V.size();
        int32_t sl = -1;
        double best_score = 1e300;
        for (int32_t l = 1; l < maxl; ++l) {
            below += cnt[l - 1];
            int64_t above = total - below - cnt[l];
            if (above <= 0) break;
            double lo = (double)std::min(below, above), hi = (double)std::max(below, above);
            if (lo < 0.35 * hi) continue;
            double score = (double)cnt[l] * (1.0 + 0.5 * (hi - lo) / (double)total);
            if (score < best_score) { best_score = score; sl = l; }
        }
        if (sl < 0) {  // fall back to the median level
            below = 0;
            for (int32_t l = 0; l <= maxl; ++l) { if (below + cnt[l] >= total / 2) { sl = std::max(1, std::min(l, maxl - 1)); break; } below += cnt[l]; }
        }
        std::vector<int32_t> A, B, S;
        for (int32_t v : V) {
            if (lv[v] < sl) A.push_back(v);
            else if (lv[v] > sl) B.push_back(v);
            else {
                bool touches_b = false;
                for (int64_t q = g.rp[v]; q < g.rp[v + 1] && !touches_b; ++q) {
                    int32_t y = g.ci[q];
                    if (tag[y] == want && lv[y] > sl) touches_b = true;
                }
                if (touches_b) S.push_back(v); else A.push_back(v);
            }
        }
        for (int32_t v : V) lv[v] = -1;
        int32_t ta = next_tag++, tb = next_tag++, ts = next_tag++;
        for (int32_t v : A) tag[v] = ta;
        for (int32_t v : B) tag[v] = tb;
        for (int32_t v : S) tag[v] = ts;
        std::sort(S.begin(), S.end());
        // emit order: A, B, S  (stack is LIFO)
        stack.push_back({S, ts, true});
        stack.push_back({B, tb, false});
        stack.push_back({A, ta, false});
    }
    for (int32_t d : dense) perm.push_back(d);
}

}  // namespace hylu

// Host planner: cluster tree, block tree, fill-in closure and colouring.
//
// Readings (the paper leaves them open, Sec. 3.1 and Sec. 3.4):
//  * binary tree, median split along the longest bounding-box axis (first axis
//    on ties), stable order by that coordinate; all leaves at depth
//    L = ceil(log2(n / leaf));
//  * strong admissibility on point bounding boxes (H2_ADM_BOX or H2_ADM_CENTER), or
//    weak admissibility (H2_ADM_WEAK: every pair of distinct clusters, the HSS
//    structure of Sec. 3.3);
//    the block tree is refined top-down from the root pair;
//  * every pair of near neighbours of a cluster receives a Schur update when
//    that cluster is eliminated (Eq. blr2-diag-schur on dense off-diagonal
//    blocks, Sec. 3.4); the non-near ones are fill-in blocks.  Their parent
//    pairs are made inadmissible bottom-up so that recompressed fill-ins merge
//    into the parent level;
//  * greedy distance-2 colouring of each level's near graph in cluster order;
//    elimination runs colour by colour (same-colour clusters are independent).
#include <algorithm>
#include <cmath>
#include <numeric>

#include "h2_internal.h"

namespace h2 {

namespace {

struct Box {
    double lo[3], hi[3];
};

double diam(const Box& b, int d) {
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        double e = b.hi[k] - b.lo[k];
        s += e * e;
    }
    return std::sqrt(s);
}

bool admissible(const Box& a, const Box& b, int d, double eta, int rule) {
    if (rule == H2_ADM_WEAK) return true;   // every pair of distinct clusters (HSS)
    double da = diam(a, d), db = diam(b, d);
    if (rule == H2_ADM_BOX) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) {
            double g = std::max(0.0, std::max(a.lo[k] - b.hi[k], b.lo[k] - a.hi[k]));
            s += g * g;
        }
        return std::max(da, db) <= eta * std::sqrt(s);
    }
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        double c = 0.5 * (a.lo[k] + a.hi[k]) - 0.5 * (b.lo[k] + b.hi[k]);
        s += c * c;
    }
    return 0.5 * (da + db) <= eta * std::sqrt(s);
}

}  // namespace

Plan make_plan(const double* pts, int64_t n, int d, int leaf, double eta, int rule) {
    Plan P;
    P.n = n;
    P.d = d;
    int L = 0;
    while ((int64_t)leaf << L < n) ++L;   // smallest L with leaf * 2^L >= n
    P.L = L;
    P.perm.resize(n);
    std::iota(P.perm.begin(), P.perm.end(), 0);
    P.lev.resize(L + 1);
    P.lev[0].nc = 1;
    P.lev[0].off = {0, n};
    for (int l = 1; l <= L; ++l) {
        const auto& prev = P.lev[l - 1];
        auto& cur = P.lev[l];
        cur.nc = 2 * prev.nc;
        cur.off.assign(1, 0);
        for (int c = 0; c < prev.nc; ++c) {
            int64_t s = prev.off[c], e = prev.off[c + 1];
            double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
            for (int k = 0; k < d; ++k) {
                lo[k] = hi[k] = pts[P.perm[s] * d + k];
            }
            for (int64_t i = s; i < e; ++i)
                for (int k = 0; k < d; ++k) {
                    double x = pts[P.perm[i] * d + k];
                    lo[k] = std::min(lo[k], x);
                    hi[k] = std::max(hi[k], x);
                }
            int ax = 0;
            for (int k = 1; k < d; ++k)
                if (hi[k] - lo[k] > hi[ax] - lo[ax]) ax = k;
            std::stable_sort(P.perm.begin() + s, P.perm.begin() + e,
                             [&](int64_t a, int64_t b) { return pts[a * d + ax] < pts[b * d + ax]; });
            int64_t h = (e - s) / 2;
            cur.off.push_back(s + h);
            cur.off.push_back(e);
        }
    }
    // bounding boxes
    std::vector<std::vector<Box>> boxes(L + 1);
    for (int l = 0; l <= L; ++l) {
        auto& lv = P.lev[l];
        boxes[l].resize(lv.nc);
        for (int c = 0; c < lv.nc; ++c) {
            Box& b = boxes[l][c];
            for (int k = 0; k < 3; ++k) b.lo[k] = b.hi[k] = 0.0;
            int64_t s = lv.off[c], e = lv.off[c + 1];
            for (int k = 0; k < d; ++k) b.lo[k] = b.hi[k] = pts[P.perm[s] * d + k];
            for (int64_t i = s; i < e; ++i)
                for (int k = 0; k < d; ++k) {
                    double x = pts[P.perm[i] * d + k];
                    b.lo[k] = std::min(b.lo[k], x);
                    b.hi[k] = std::max(b.hi[k], x);
                }
        }
    }
    // top-down block tree
    P.lev[0].near.assign(1, 1);
    for (int l = 1; l <= L; ++l) {
        auto& lv = P.lev[l];
        const auto& pv = P.lev[l - 1];
        int nc = lv.nc;
        lv.near.assign((size_t)nc * nc, 0);
        for (int p = 0; p < pv.nc; ++p)
            for (int q = 0; q < pv.nc; ++q) {
                if (!pv.near[(size_t)p * pv.nc + q]) continue;
                for (int c = 2 * p; c <= 2 * p + 1; ++c)
                    for (int e = 2 * q; e <= 2 * q + 1; ++e)
                        if (c == e || !admissible(boxes[l][c], boxes[l][e], d, eta, rule))
                            lv.near[(size_t)c * nc + e] = 1;
            }
    }
    // bottom-up fill-in closure
    for (int l = L; l >= 1; --l) {
        auto& lv = P.lev[l];
        int nc = lv.nc;
        lv.fill.assign((size_t)nc * nc, 0);
        std::vector<std::vector<int>> nb(nc);
        for (int c = 0; c < nc; ++c)
            for (int e = 0; e < nc; ++e)
                if (lv.near[(size_t)c * nc + e]) nb[c].push_back(e);
        std::vector<uint8_t> X(lv.near);
        for (int t = 0; t < nc; ++t)
            for (int a : nb[t])
                for (int b : nb[t]) X[(size_t)a * nc + b] = 1;
        auto& pv = P.lev[l - 1];
        for (int a = 0; a < nc; ++a)
            for (int b = 0; b < nc; ++b) {
                if (!X[(size_t)a * nc + b]) continue;
                if (!lv.near[(size_t)a * nc + b]) lv.fill[(size_t)a * nc + b] = 1;
                pv.near[(size_t)(a / 2) * pv.nc + (b / 2)] = 1;
            }
    }
    P.lev[0].fill.assign(1, 0);
    P.lev[0].far.assign(1, 0);
    for (int l = 1; l <= L; ++l) {
        auto& lv = P.lev[l];
        const auto& pv = P.lev[l - 1];
        int nc = lv.nc;
        lv.far.assign((size_t)nc * nc, 0);
        for (int a = 0; a < nc; ++a)
            for (int b = 0; b < nc; ++b)
                lv.far[(size_t)a * nc + b] =
                    pv.near[(size_t)(a / 2) * pv.nc + (b / 2)] && !lv.near[(size_t)a * nc + b];
    }
    // distance-2 colouring
    for (int l = 0; l <= L; ++l) {
        auto& lv = P.lev[l];
        int nc = lv.nc;
        std::vector<std::vector<int>> nb(nc);
        for (int c = 0; c < nc; ++c)
            for (int e = 0; e < nc; ++e)
                if (c != e && lv.near[(size_t)c * nc + e]) nb[c].push_back(e);
        lv.color.assign(nc, -1);
        int ncol = 0;
        for (int c = 0; c < nc; ++c) {
            std::vector<uint8_t> used(nc + 1, 0);
            for (int a : nb[c]) {
                if (lv.color[a] >= 0) used[lv.color[a]] = 1;
                for (int b : nb[a])
                    if (b != c && lv.color[b] >= 0) used[lv.color[b]] = 1;
            }
            int k = 0;
            while (used[k]) ++k;
            lv.color[c] = k;
            ncol = std::max(ncol, k + 1);
        }
        lv.color_lists.assign(ncol, {});
        for (int c = 0; c < nc; ++c) lv.color_lists[lv.color[c]].push_back(c);
    }
    return P;
}

}  // namespace h2

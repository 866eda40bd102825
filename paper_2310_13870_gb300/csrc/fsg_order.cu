// Spatial tree order (host): a permutation under which every node of the
// halving tree of Sec. 4.1 is a compact group of points.  Node [lo, hi) of
// tree positions is split at its own midpoint lo + floor((hi - lo) / 2), as
// the tree splits it, along the coordinate of largest spread among the
// node's points: the floor(|X|/2) points with the smallest values of that
// coordinate go left (ties broken by original index).  Nodes of at most
// `leaf` points keep original-index order.  The KDE and the sampling
// distribution do not depend on the order (Eq. 1 sums over the node's
// points whatever their positions); the order only decides which points
// share a bin, and so how far a bin's points lie from its centre, which the
// centred split-precision bin pass relies on.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "fsg.h"

namespace {

struct OrderState {
    const float* X;
    int64_t d;
    int32_t leaf;
    std::vector<int32_t>* idx;
};

void split_node(OrderState& st, int64_t lo, int64_t hi) {
    std::vector<int32_t>& idx = *st.idx;
    while (hi - lo > st.leaf) {
        // axis of largest spread among the node's points
        int64_t axis = 0;
        float best = -1.f;
        for (int64_t t = 0; t < st.d; ++t) {
            float mn = st.X[(int64_t)idx[lo] * st.d + t], mx = mn;
            for (int64_t p = lo + 1; p < hi; ++p) {
                const float v = st.X[(int64_t)idx[p] * st.d + t];
                mn = std::min(mn, v);
                mx = std::max(mx, v);
            }
            if (mx - mn > best) {
                best = mx - mn;
                axis = t;
            }
        }
        const int64_t mid = lo + (hi - lo) / 2;
        const float* X = st.X;
        const int64_t d = st.d;
        auto less = [X, d, axis](int32_t a, int32_t b) {
            const float va = X[(int64_t)a * d + axis], vb = X[(int64_t)b * d + axis];
            return va < vb || (va == vb && a < b);
        };
        std::nth_element(idx.begin() + lo, idx.begin() + mid, idx.begin() + hi, less);
        split_node(st, lo, mid);
        lo = mid;  // the right half, without another stack frame
    }
    std::sort(idx.begin() + lo, idx.begin() + hi);
}

}  // namespace

extern "C" int fsg_spatial_order(const float* h_points, int64_t n, int32_t d, int32_t leaf, int32_t* h_perm) {
    if (!h_points || !h_perm || n < 1 || n > INT32_MAX || d < 1 || d > 4096 || leaf < 1)
        return FSG_ERR_INVALID_ARG;
    for (int64_t e = 0; e < n * (int64_t)d; ++e)
        if (!(h_points[e] == h_points[e]) || h_points[e] > 3.0e38f || h_points[e] < -3.0e38f)
            return FSG_ERR_INVALID_ARG;  // NaN or infinite coordinate
    std::vector<int32_t> idx((size_t)n);
    for (int64_t i = 0; i < n; ++i) idx[(size_t)i] = (int32_t)i;
    OrderState st{h_points, d, leaf, &idx};
    split_node(st, 0, n);
    std::copy(idx.begin(), idx.end(), h_perm);
    return FSG_OK;
}

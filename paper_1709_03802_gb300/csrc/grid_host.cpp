// Host-side preparation of the adaptive Cartesian grid (Sect. 2: "an adaptive
// 3D Cartesian grid of cells"): structural validation of the flattened
// forest, node boxes computed in double and checked to be exact in float32
// (so the float32 device traversal sees exact face coordinates), and for every
// leaf the six face links to the neighbouring node of the same or larger size.
#include "grid_host.h"

#include <cmath>
#include <cstdio>

namespace dartray {

namespace {

bool exact_f32(double v) { return static_cast<double>(static_cast<float>(v)) == v; }

struct Walker {
    const int32_t *nroot;
    const double *root_lo;
    double root_size;
    const int32_t *first_child;

    // Root lattice index along axis a of coordinate p with the face convention
    // (a point on a face belongs to the side direction s points into; s >= 0:
    // upper).  Returns -1 outside.
    int64_t root_index(int a, double p, int s) const {
        double u = std::floor((p - root_lo[a]) / root_size);
        if (!(u > -2.0) || u > nroot[a] + 1.0) return -1;
        int64_t i = static_cast<int64_t>(u);
        for (int guard = 0; guard < 4; ++guard) {
            const double f = root_lo[a] + static_cast<double>(i) * root_size;
            const double h = root_lo[a] + static_cast<double>(i + 1) * root_size;
            if (p < f || (p == f && s < 0)) --i;
            else if (p > h || (p == h && s >= 0)) ++i;
            else break;
        }
        return (i < 0 || i >= nroot[a]) ? -1 : i;
    }

    // Descend from the roots to the node containing q (face convention by the
    // signs in s) whose side is <= target or which is a leaf.
    int64_t find(const double q[3], const int s[3], double target) const {
        int64_t idx[3];
        double lo[3];
        for (int a = 0; a < 3; ++a) {
            idx[a] = root_index(a, q[a], s[a]);
            if (idx[a] < 0) return -1;
            lo[a] = root_lo[a] + static_cast<double>(idx[a]) * root_size;
        }
        int64_t node = idx[0] + static_cast<int64_t>(nroot[0]) * (idx[1] + static_cast<int64_t>(nroot[1]) * idx[2]);
        double size = root_size;
        while (first_child[node] >= 0 && size > target) {
            const double half = 0.5 * size;
            int oct = 0;
            for (int a = 0; a < 3; ++a) {
                const double mid = lo[a] + half;
                if (q[a] > mid || (q[a] == mid && s[a] >= 0)) {
                    lo[a] = mid;
                    oct |= 1 << a;
                }
            }
            node = first_child[node] + oct;
            size = half;
        }
        return node;
    }
};

}  // namespace

std::string build_topology(const int32_t nroot[3], const double root_lo[3], double root_size,
                           int32_t n_nodes, int32_t n_leaf, const int32_t *first_child,
                           const int32_t *leaf_of_node, HostTopo *t) {
    char msg[256];
    for (int a = 0; a < 3; ++a)
        if (nroot[a] < 1) return "nroot must be >= 1 on every axis";
    if (!(root_size > 0) || !std::isfinite(root_size)) return "root_size must be positive";
    const int64_t nroots = static_cast<int64_t>(nroot[0]) * nroot[1] * nroot[2];
    if (nroots > n_nodes) return "n_nodes smaller than the number of root cells";
    if (n_leaf < 1) return "n_leaf must be >= 1";
    for (int a = 0; a < 3; ++a) {
        if (!exact_f32(root_lo[a]) || !exact_f32(root_size)) return "root_lo/root_size not exact in float32";
        for (int64_t i = 0; i <= nroot[a]; ++i)
            if (!exact_f32(root_lo[a] + static_cast<double>(i) * root_size))
                return "root lattice face coordinates not exact in float32";
    }
    t->node_child.assign(n_nodes, 0);
    t->node_box.assign(static_cast<size_t>(n_nodes) * 4, 0.f);
    t->leaf_box.assign(static_cast<size_t>(n_leaf) * 4, 0.f);
    t->leaf_node.assign(n_leaf, -1);
    std::vector<uint8_t> seen(n_nodes, 0);
    std::vector<int64_t> stack;
    std::vector<double> sbox;
    std::vector<int> sdepth;
    int64_t nleaf_seen = 0;
    t->max_depth = 0;
    for (int64_t r = 0; r < nroots; ++r) {
        stack.assign(1, r);
        sbox.assign({root_lo[0] + static_cast<double>(r % nroot[0]) * root_size,
                     root_lo[1] + static_cast<double>((r / nroot[0]) % nroot[1]) * root_size,
                     root_lo[2] + static_cast<double>(r / (static_cast<int64_t>(nroot[0]) * nroot[1])) * root_size,
                     root_size});
        sdepth.assign(1, 0);
        while (!stack.empty()) {
            const int64_t nd = stack.back();
            stack.pop_back();
            const double b[4] = {sbox[sbox.size() - 4], sbox[sbox.size() - 3], sbox[sbox.size() - 2],
                                 sbox[sbox.size() - 1]};
            sbox.resize(sbox.size() - 4);
            const int depth = sdepth.back();
            sdepth.pop_back();
            if (seen[nd]) {
                std::snprintf(msg, sizeof msg, "node %lld reached twice", static_cast<long long>(nd));
                return msg;
            }
            seen[nd] = 1;
            for (int k = 0; k < 4; ++k) {
                if (!exact_f32(b[k]) || !exact_f32(b[k < 3 ? k : 0] + b[3])) {
                    std::snprintf(msg, sizeof msg, "node %lld face coordinates not exact in float32",
                                  static_cast<long long>(nd));
                    return msg;
                }
                t->node_box[4 * nd + k] = static_cast<float>(b[k]);
            }
            if (depth > t->max_depth) t->max_depth = depth;
            const int32_t fc = first_child[nd];
            if (fc < 0) {
                const int32_t lf = leaf_of_node[nd];
                if (fc != -1 || lf < 0 || lf >= n_leaf || t->leaf_node[lf] != -1) {
                    std::snprintf(msg, sizeof msg, "bad leaf id at node %lld", static_cast<long long>(nd));
                    return msg;
                }
                t->leaf_node[lf] = static_cast<int32_t>(nd);
                t->node_child[nd] = -(lf + 1);
                for (int k = 0; k < 4; ++k) t->leaf_box[4 * static_cast<size_t>(lf) + k] = static_cast<float>(b[k]);
                ++nleaf_seen;
                continue;
            }
            if (leaf_of_node[nd] != -1 || fc < nroots || static_cast<int64_t>(fc) + 8 > n_nodes) {
                std::snprintf(msg, sizeof msg, "bad child index at node %lld", static_cast<long long>(nd));
                return msg;
            }
            if (depth >= 40) return "tree deeper than 40 levels";
            t->node_child[nd] = fc;
            const double h = 0.5 * b[3];
            for (int c = 0; c < 8; ++c) {
                stack.push_back(fc + c);
                sbox.insert(sbox.end(), {b[0] + ((c & 1) ? h : 0.0), b[1] + ((c & 2) ? h : 0.0),
                                         b[2] + ((c & 4) ? h : 0.0), h});
                sdepth.push_back(depth + 1);
            }
        }
    }
    for (int64_t nd = 0; nd < n_nodes; ++nd)
        if (!seen[nd]) {
            std::snprintf(msg, sizeof msg, "node %lld unreachable", static_cast<long long>(nd));
            return msg;
        }
    if (nleaf_seen != n_leaf) return "leaf count does not match n_leaf";
    if (n_leaf >= (1 << 29)) return "more than 2^29 leaves";

    // face links: for face (axis a, side s) of leaf box b, the node beyond the
    // face centre of size >= side (a coarser leaf or a same-size node)
    Walker w{nroot, root_lo, root_size, first_child};
    t->leaf_rope.assign(static_cast<size_t>(n_leaf) * 6, -1);
    for (int64_t lf = 0; lf < n_leaf; ++lf) {
        const float *b = &t->leaf_box[4 * lf];
        for (int a = 0; a < 3; ++a) {
            for (int side = 0; side < 2; ++side) {
                double q[3];
                int s[3] = {1, 1, 1};
                for (int k = 0; k < 3; ++k) q[k] = static_cast<double>(b[k]) + 0.5 * b[3];
                q[a] = side ? static_cast<double>(b[a]) + b[3] : static_cast<double>(b[a]);
                s[a] = side ? 1 : -1;
                const int64_t nb = w.find(q, s, b[3]);
                // a leaf neighbour is stored as -(leaf + 2) so the marcher can
                // use its box directly; a refined neighbour as its node id
                int32_t code = kRopeBoundary;
                if (nb >= 0) {
                    if (first_child[nb] >= 0) {
                        code = static_cast<int32_t>(nb);
                    } else {
                        const int32_t nl = leaf_of_node[nb];
                        const bool same = t->node_box[4 * nb + 3] == b[3];
                        code = same ? kRopeSameSize - nl : -(nl + 2);
                    }
                }
                t->leaf_rope[6 * lf + 2 * a + side] = code;
            }
        }
    }
    return "";
}

std::string build_mirrors(const int32_t nroot[3], const double root_lo[3], double root_size,
                          const int32_t *first_child, const int32_t *leaf_of_node, const HostTopo &t,
                          std::vector<int32_t> *mirror) {
    const int64_t n_leaf = static_cast<int64_t>(t.leaf_box.size() / 4);
    double centre[3];
    for (int a = 0; a < 3; ++a) centre[a] = root_lo[a] + 0.5 * nroot[a] * root_size;
    Walker w{nroot, root_lo, root_size, first_child};
    mirror->assign(static_cast<size_t>(7) * n_leaf, -1);
    char msg[256];
    for (int64_t lf = 0; lf < n_leaf; ++lf) {
        const float *b = &t.leaf_box[4 * lf];
        for (int m = 1; m < 8; ++m) {
            double lo[3], q[3];
            const int s[3] = {1, 1, 1};
            for (int a = 0; a < 3; ++a) {
                lo[a] = ((m >> a) & 1) ? 2.0 * centre[a] - static_cast<double>(b[a]) - b[3] : static_cast<double>(b[a]);
                q[a] = lo[a] + 0.5 * b[3];
            }
            const int64_t nd = w.find(q, s, b[3]);
            const bool ok = nd >= 0 && first_child[nd] < 0 && t.node_box[4 * nd + 3] == b[3] &&
                            t.node_box[4 * nd] == static_cast<float>(lo[0]) &&
                            t.node_box[4 * nd + 1] == static_cast<float>(lo[1]) &&
                            t.node_box[4 * nd + 2] == static_cast<float>(lo[2]);
            if (!ok) {
                std::snprintf(msg, sizeof msg,
                              "grid is not mirror-symmetric about its centre (leaf %lld has no image under "
                              "reflection mask %d)",
                              static_cast<long long>(lf), m);
                return msg;
            }
            (*mirror)[static_cast<size_t>(m - 1) * n_leaf + lf] = leaf_of_node[nd];
        }
    }
    return "";
}

}  // namespace dartray

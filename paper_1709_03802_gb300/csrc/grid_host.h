// Host-side grid preparation shared by the CUDA translation unit: validation
// of the flattened forest, node boxes, and leaf face links ("ropes").
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace dartray {

// Face link codes: >= 0 refined node id; -1 model boundary; -(leaf + 2) a
// larger leaf; kRopeSameSize - leaf a leaf of the same size (its box is the
// current box shifted by one side).  Leaf ids are below 2^29.
constexpr int32_t kRopeBoundary = -1;
constexpr int32_t kRopeSameSize = -(1 << 30);

struct HostTopo {
    // node_child[node] = first child (>= 0) or -(leaf + 1) for a leaf
    std::vector<int32_t> node_child;
    // node boxes: lo x, lo y, lo z, side (exact in float32, validated)
    std::vector<float> node_box;   // [n_nodes * 4]
    std::vector<float> leaf_box;   // [n_leaf * 4]
    std::vector<int32_t> leaf_node;
    // leaf_rope[leaf * 6 + 2 * axis + (side > 0)]: what lies beyond that face
    // (codes above)
    std::vector<int32_t> leaf_rope;
    int max_depth = 0;
};

// Validates the description (tree structure, exact float32 face coordinates)
// and fills *t.  Returns "" on success, else an error message.
std::string build_topology(const int32_t nroot[3], const double root_lo[3], double root_size,
                           int32_t n_nodes, int32_t n_leaf, const int32_t *first_child,
                           const int32_t *leaf_of_node, HostTopo *t);

// Octant mode: the images of every leaf under the seven reflections about
// the planes through the model centre (reflection mask m = bit a set: axis a
// flipped), mirror[(m - 1) * n_leaf + leaf].  Returns "" on success, else a
// message naming a leaf without an image (the grid is not mirror-symmetric).
std::string build_mirrors(const int32_t nroot[3], const double root_lo[3], double root_size,
                          const int32_t *first_child, const int32_t *leaf_of_node, const HostTopo &t,
                          std::vector<int32_t> *mirror);

}  // namespace dartray

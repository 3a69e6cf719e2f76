"""Host-side grid preparation of the CUDA library (csrc/grid_host.cpp,
plain C++): the leaf boxes and the six face links of every leaf, checked
against a brute-force neighbour search on adaptive trees.  A link names what
lies just beyond a face: the model boundary, a leaf of the same size, a
larger leaf, or the refined node of the leaf's own size."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1709_03802_gb300", "csrc")
SAME_SIZE = -(1 << 30)

SHIM = r'''
#include "grid_host.h"
#include <cstring>
extern "C" int topo_links(const int32_t *nroot, const double *root_lo, double root_size, int32_t n_nodes,
                          int32_t n_leaf, const int32_t *fc, const int32_t *lon, int32_t *rope, float *leaf_box,
                          char *err, int errlen) {
    dartray::HostTopo t;
    const std::string e = dartray::build_topology(nroot, root_lo, root_size, n_nodes, n_leaf, fc, lon, &t);
    if (!e.empty()) {
        std::strncpy(err, e.c_str(), errlen - 1);
        return 1;
    }
    std::memcpy(rope, t.leaf_rope.data(), sizeof(int32_t) * t.leaf_rope.size());
    std::memcpy(leaf_box, t.leaf_box.data(), sizeof(float) * t.leaf_box.size());
    return 0;
}
'''


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("topo")
    (d / "shim.cpp").write_text(SHIM)
    so = d / "libtopo.so"
    subprocess.check_call([cxx, "-std=c++17", "-O1", "-shared", "-fPIC", "-I", CSRC,
                           os.path.join(CSRC, "grid_host.cpp"), str(d / "shim.cpp"), "-o", str(so)])
    return C.CDLL(str(so))


def node_boxes(g):
    """lo and side of every node of the forest (children in Morton order)."""
    n = g.n_nodes
    lo = np.zeros((n, 3))
    size = np.zeros(n)
    nx, ny, _ = g.nroot
    for r in range(int(np.prod(g.nroot))):
        lo[r] = np.asarray(g.root_lo) + g.root_size * np.array([r % nx, (r // nx) % ny, r // (nx * ny)])
        size[r] = g.root_size
    for node in range(n):  # parents precede their children
        c = g.first_child[node]
        if c >= 0:
            h = size[node] / 2
            for k in range(8):
                lo[c + k] = lo[node] + h * np.array([k & 1, (k >> 1) & 1, (k >> 2) & 1])
                size[c + k] = h
    return lo, size


def links(lib, g):
    rope = np.zeros(6 * g.n_leaf, np.int32)
    box = np.zeros(4 * g.n_leaf, np.float32)
    err = C.create_string_buffer(256)
    ptr = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    nroot = np.asarray(g.nroot, np.int32)
    rlo = np.asarray(g.root_lo, np.float64)
    fc = np.ascontiguousarray(g.first_child, np.int32)
    lon = np.ascontiguousarray(g.leaf_of_node, np.int32)
    rc = lib.topo_links(ptr(nroot), ptr(rlo), C.c_double(g.root_size), C.c_int32(g.n_nodes), C.c_int32(g.n_leaf),
                        ptr(fc), ptr(lon), ptr(rope), ptr(box), err, 256)
    assert rc == 0, err.value
    return rope.reshape(-1, 6), box.reshape(-1, 4)


def random_tree(seed):
    rng = np.random.default_rng(seed)
    fc, lon, llo, lsz = synth.grids.refine_tree((2, 3, 2), (-1.0, -1.5, -1.0), 1.0, 4,
                                                lambda lo, s, lev: rng.random(lo.shape[0]) < 0.35)
    n = llo.shape[0]
    return synth.grids._assemble(((2, 3, 2), (-1.0, -1.5, -1.0), 1.0, fc, lon, llo, lsz),
                                 np.zeros((n, 1)), np.zeros((n, 1)), [0.5], [0.5], "random")


@pytest.mark.parametrize("make", [
    lambda: synth.galaxy_disk(max_level=3, threshold=0.3, nroot=(3, 3, 1), root_size=4.0),
    lambda: random_tree(1709), lambda: random_tree(1710)], ids=["galaxy", "random-a", "random-b"])
def test_face_links_match_brute_force_neighbours(lib, make):
    g = make()
    rope, box = links(lib, g)
    assert np.array_equal(box[:, :3], g.leaf_lo.astype(np.float32))
    assert np.array_equal(box[:, 3], g.leaf_size.astype(np.float32))
    nlo, nsz = node_boxes(g)
    model_lo = np.asarray(g.root_lo)
    model_hi = model_lo + g.root_size * np.asarray(g.nroot)
    llo, lsz = g.leaf_lo, g.leaf_size
    kinds = set()
    for leaf in range(g.n_leaf):
        s = lsz[leaf]
        for a in range(3):
            for side in range(2):
                q = llo[leaf] + 0.5 * s
                q[a] = llo[leaf, a] - 1e-3 * s if side == 0 else llo[leaf, a] + s + 1e-3 * s
                code = rope[leaf, 2 * a + side]
                if np.any(q < model_lo) or np.any(q > model_hi):
                    assert code == -1
                    kinds.add("boundary")
                    continue
                inside = np.all((llo <= q) & (q < llo + lsz[:, None]), axis=1)
                (nb,) = np.nonzero(inside)[0]
                if lsz[nb] == s:
                    assert code == SAME_SIZE - nb
                    kinds.add("same")
                elif lsz[nb] > s:
                    assert code == -(nb + 2)
                    kinds.add("larger")
                else:
                    hit = np.nonzero((nsz == s) & np.all((nlo <= q) & (q < nlo + nsz[:, None]), axis=1))[0]
                    assert code >= 0 and list(hit) == [code]
                    kinds.add("node")
    assert kinds == {"boundary", "same", "larger", "node"}

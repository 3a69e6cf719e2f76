// Device-side building blocks of the sweep: HEALPix directions (Gorski et al.
// 2005), grid traversal over the flattened forest with face links, and the
// shared data structures of the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dartray {

constexpr int kMaxLambda = 16;
constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;
constexpr double kPi = 3.14159265358979323846;
// HEALPix levels whose pixel centres are tabulated (levels 0..kDirTabLevels)
constexpr int kDirTabLevels = 11;
// first table entry of level k: sum_{j<k} 12*4^j = 4*(4^k - 1)
__host__ __device__ inline int64_t dir_tab_offset(int k) { return 4 * ((int64_t(1) << (2 * k)) - 1); }

// ------------------------------------------------------------------ grid
// One model of a batched grid: its root lattice (roots are nodes node0 ..
// node0 + nroot[0]*nroot[1]*nroot[2] - 1) and its step-1 radius.
struct ModelDev {
    int nroot[3];
    float root_lo[3];
    float root_size;
    int node0;
    float r_pre;
};

struct DevGrid {
    int nroot[3];
    float root_lo[3];
    float root_size;
    int n_nodes, n_leaf, nl, n_point;
    int nl_user;                // the caller's wavelengths: [0, nl_user); the rest pad nl
    int tangent;                // 1: [nl/2, nl/2 + nl_user) carry d/d albedo of [0, nl_user)
    const int32_t *node_child;  // first child, or -(leaf+1)
    const float4 *node_box;     // lo.xyz, side
    const float4 *leaf_box;
    const int32_t *leaf_rope;   // [n_leaf][6]
    const float *kappa_rho;     // [n_leaf][nl]
    const float *emis;          // [n_leaf][nl]
    const float *point_xyz;     // [n_point][3]
    const float *point_lum;     // [n_point][nl]
    const float4 *dirtab;       // pixel centres for levels 0..kDirTabLevels
    const float *ztab;          // [nl][n_dirtab] HG row sums per ray direction
    long long n_dirtab;
    float albedo[kMaxLambda], g[kMaxLambda];
    int k_lam[kMaxLambda];
    long long off_lam[kMaxLambda];
    // octant mode (symmetric models): only sources in the first octant are
    // traced and every deposit is also made, reflected, in the seven images
    // of its cell about the planes through the model centre
    int octant;
    float centre[3];
    const int32_t *mirror;        // [7][n_leaf]: image of a leaf under reflection mask 1..7
    const int32_t *mirror_pix;    // [7][kMirrorPix]: image of a j_sca pixel (levels 0..3, table order)
    // batched grids: several independent models in one forest, each with its
    // own root lattice; rays never leave their model (face links end at its
    // boundary)
    int n_models;
    const ModelDev *models;       // [n_models]
    const uint16_t *leaf_model;   // [n_leaf] model of each leaf (batched grids only)
    const uint16_t *point_model;  // [n_point] model of each point source (batched grids only)
};

__device__ __forceinline__ int model_of_leaf(const DevGrid &G, int leaf) {
    return G.n_models > 1 ? static_cast<int>(__ldg(&G.leaf_model[leaf])) : 0;
}

constexpr int kMirrorPix = 1020;  // pixel centres of levels 0..3

// image of leaf c under reflection mask m (0: the leaf itself)
__device__ __forceinline__ int mirror_leaf(const DevGrid &G, int m, int c) {
    return m == 0 ? c : __ldg(&G.mirror[static_cast<long long>(m - 1) * G.n_leaf + c]);
}
// image of pixel q of j_sca level k under reflection mask m
__device__ __forceinline__ int mirror_pixel(const DevGrid &G, int m, int k, int q) {
    return m == 0 ? q : __ldg(&G.mirror_pix[(m - 1) * kMirrorPix + dir_tab_offset(k) + q]);
}

// ------------------------------------------------------------------ HEALPix
// Face f: ring index (from the north pole) of pixel (ix, iy) is
// kFaceRow[f]*nside - ix - iy - 1; the face centre sits at longitude
// kFaceLon[f]*pi/4.
static __device__ __constant__ int kFaceRow[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
static __device__ __constant__ int kFaceLon[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};

__device__ inline uint32_t compact_bits(uint64_t v) {
    v &= 0x5555555555555555ull;
    v = (v | (v >> 1)) & 0x3333333333333333ull;
    v = (v | (v >> 2)) & 0x0f0f0f0f0f0f0f0full;
    v = (v | (v >> 4)) & 0x00ff00ff00ff00ffull;
    v = (v | (v >> 8)) & 0x0000ffff0000ffffull;
    v = (v | (v >> 16)) & 0x00000000ffffffffull;
    return static_cast<uint32_t>(v);
}

__device__ inline uint64_t spread_bits(uint64_t v) {
    v &= 0xffffffffull;
    v = (v | (v << 16)) & 0x0000ffff0000ffffull;
    v = (v | (v << 8)) & 0x00ff00ff00ff00ffull;
    v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    v = (v | (v << 1)) & 0x5555555555555555ull;
    return v;
}

// Unit vector of the centre of nested pixel p at level k, in double.  Ring
// z from the scheme's definition (cap: 1 - i^2/(3 nside^2); belt:
// 4/3 - 2i/(3 nside)); the longitude is (pi/2)*num/den with integer num, den,
// reduced to the first octant so the set of centres keeps the square's
// symmetries exactly in floating point.
__device__ inline void pix2vec_d(int k, uint64_t p, double v[3]) {
    const int64_t ns = int64_t(1) << k;
    const uint64_t npf = uint64_t(ns) * uint64_t(ns);
    const int face = static_cast<int>(p / npf);
    const uint64_t q = p - uint64_t(face) * npf;
    const int64_t ix = compact_bits(q), iy = compact_bits(q >> 1);
    const int64_t jr = int64_t(kFaceRow[face]) * ns - ix - iy - 1;
    int64_t nr;
    int shift = 0;
    bool south = false;
    double z, omz;
    if (jr < ns) {
        nr = jr;
        omz = double(nr * nr) / (3.0 * double(ns * ns));
        z = 1.0 - omz;
    } else if (jr > 3 * ns) {
        nr = 4 * ns - jr;
        omz = double(nr * nr) / (3.0 * double(ns * ns));
        z = 1.0 - omz;
        south = true;
    } else {
        nr = ns;
        int64_t m = 2 * ns - jr;
        if (m < 0) { south = true; m = -m; }
        z = double(m) * 2.0 / (3.0 * double(ns));
        omz = 1.0 - z;
        shift = static_cast<int>((jr - ns) & 1);
    }
    int64_t jp = (int64_t(kFaceLon[face]) * nr + ix - iy + 1 + shift) / 2;
    if (jp > 4 * nr) jp -= 4 * nr;
    if (jp < 1) jp += 4 * nr;
    const int64_t num = 2 * jp - shift - 1, den = 2 * nr;
    const int64_t quad = num / den, r = num - quad * den;
    double c, s;
    if (2 * r == den) {
        c = s = sqrt(0.5);
    } else if (2 * r < den) {
        sincos(0.5 * kPi * double(r) / double(den), &s, &c);
    } else {
        sincos(0.5 * kPi * double(den - r) / double(den), &c, &s);
    }
    double x, y;
    switch (static_cast<int>(quad & 3)) {
    case 0: x = c; y = s; break;
    case 1: x = -s; y = c; break;
    case 2: x = -c; y = -s; break;
    default: x = s; y = -c; break;
    }
    const double st = sqrt(omz * (1.0 + z));
    v[0] = st * x;
    v[1] = st * y;
    v[2] = south ? -z : z;
}

// Nested pixel of level k holding direction v, in double (equatorial zone:
// edges nside*(phi/(pi/2) + 1/2 -+ 3z/4) = integer; caps: edges
// nside*sqrt(3(1-|z|))*{t, 1-t} = integer).
__device__ inline uint64_t vec2pix_d(int k, double vx, double vy, double vz) {
    const int64_t ns = int64_t(1) << k;
    const double rxy2 = vx * vx + vy * vy;
    const double len = sqrt(rxy2 + vz * vz);
    const double z = vz / len, za = fabs(z);
    double phi = atan2(vy, vx);
    if (phi < 0) phi += 2.0 * kPi;
    double tt = phi / (0.5 * kPi);
    if (tt >= 4.0) tt -= 4.0;
    int face;
    int64_t ix, iy;
    if (za <= 2.0 / 3.0) {
        const double t1 = double(ns) * (0.5 + tt), t2 = double(ns) * 0.75 * z;
        const int64_t jp = static_cast<int64_t>(floor(t1 - t2));
        const int64_t jm = static_cast<int64_t>(floor(t1 + t2));
        const int64_t fp = jp >> k, fm = jm >> k;
        if (fp == fm) face = static_cast<int>((fp & 3) + 4);
        else if (fp < fm) face = static_cast<int>(fp & 3);
        else face = static_cast<int>((fm & 3) + 8);
        ix = jm & (ns - 1);
        iy = ns - (jp & (ns - 1)) - 1;
    } else {
        int qd = static_cast<int>(tt);
        if (qd > 3) qd = 3;
        const double tp = tt - qd;
        const double omza = rxy2 / (len * (len + fabs(vz)));
        const double w = double(ns) * sqrt(3.0 * omza);
        int64_t jp = static_cast<int64_t>(tp * w), jm = static_cast<int64_t>((1.0 - tp) * w);
        if (jp > ns - 1) jp = ns - 1;
        if (jm > ns - 1) jm = ns - 1;
        if (z > 0) { face = qd; ix = ns - jm - 1; iy = ns - jp - 1; }
        else { face = qd + 8; ix = jp; iy = jm; }
    }
    return uint64_t(face) * uint64_t(ns) * uint64_t(ns) + (spread_bits(ix) | (spread_bits(iy) << 1));
}

// Directions beyond the table (levels above kDirTabLevels; rare), kept out of
// line so the marcher's code stays small.
static __device__ __noinline__ float3 ray_dir_computed(int k, uint64_t p) {
    double v[3];
    pix2vec_d(k, p, v);
    return make_float3(static_cast<float>(v[0]), static_cast<float>(v[1]), static_cast<float>(v[2]));
}

// Ray direction (float32) of pixel p at level k: table up to kDirTabLevels.
__device__ inline float3 ray_dir(const DevGrid &G, int k, uint64_t p) {
    if (k <= kDirTabLevels) {
        const float4 v = __ldg(&G.dirtab[dir_tab_offset(k) + static_cast<int64_t>(p)]);
        return make_float3(v.x, v.y, v.z);
    }
    return ray_dir_computed(k, p);
}

// ------------------------------------------------------------------ traversal
// A point on a face belongs to the cell the direction points into (upper cell
// for a non-negative component).
__device__ inline bool above(float p, float f, float n) { return p > f || (p == f && n >= 0.f); }

__device__ inline bool inside_box(const float4 b, const float3 p, const float3 n) {
    return above(p.x, b.x, n.x) && !above(p.x, b.x + b.w, n.x) && above(p.y, b.y, n.y) &&
           !above(p.y, b.y + b.w, n.y) && above(p.z, b.z, n.z) && !above(p.z, b.z + b.w, n.z);
}

// Root lattice index on one axis with exact face comparisons; -1 outside.
__device__ inline int root_index(float p, float lo, float S, int nr, float n) {
    const float u = floorf((p - lo) / S);
    if (!(u > -2.f) || u > float(nr) + 1.f) return -1;
    int i = static_cast<int>(u);
#pragma unroll
    for (int guard = 0; guard < 4; ++guard) {
        const float f = lo + float(i) * S, h = lo + float(i + 1) * S;
        if (!above(p, f, n)) --i;
        else if (above(p, h, n)) ++i;
        else break;
    }
    return (i < 0 || i >= nr) ? -1 : i;
}

// Descend from node (with box b) to the leaf holding p; returns leaf id.
__device__ inline int descend(const DevGrid &G, int node, float4 b, const float3 p, const float3 n) {
    int c = __ldg(&G.node_child[node]);
    while (c >= 0) {
        const float half = 0.5f * b.w;
        int oct = 0;
        const float mx = b.x + half, my = b.y + half, mz = b.z + half;
        if (above(p.x, mx, n.x)) { b.x = mx; oct |= 1; }
        if (above(p.y, my, n.y)) { b.y = my; oct |= 2; }
        if (above(p.z, mz, n.z)) { b.z = mz; oct |= 4; }
        b.w = half;
        node = c + oct;
        c = __ldg(&G.node_child[node]);
    }
    return -c - 1;
}

// Leaf of model `model` of a batched grid holding p (-1 outside the model);
// out of line, so that single-model traversal code stays small.
static __device__ __noinline__ int locate_root_model(const DevGrid &G, int model, const float3 p, const float3 n) {
    const ModelDev &M = G.models[model];
    const int ix = root_index(p.x, M.root_lo[0], M.root_size, M.nroot[0], n.x);
    const int iy = root_index(p.y, M.root_lo[1], M.root_size, M.nroot[1], n.y);
    const int iz = root_index(p.z, M.root_lo[2], M.root_size, M.nroot[2], n.z);
    if (ix < 0 || iy < 0 || iz < 0) return -1;
    const int node = M.node0 + ix + M.nroot[0] * (iy + M.nroot[1] * iz);
    const float4 b = make_float4(M.root_lo[0] + float(ix) * M.root_size, M.root_lo[1] + float(iy) * M.root_size,
                                 M.root_lo[2] + float(iz) * M.root_size, M.root_size);
    return descend(G, node, b, p, n);
}

// Leaf of model `model` holding p (-1 outside the model).
__device__ inline int locate_root(const DevGrid &G, int model, const float3 p, const float3 n) {
    if (G.n_models > 1) return locate_root_model(G, model, p, n);
    const int ix = root_index(p.x, G.root_lo[0], G.root_size, G.nroot[0], n.x);
    const int iy = root_index(p.y, G.root_lo[1], G.root_size, G.nroot[1], n.y);
    const int iz = root_index(p.z, G.root_lo[2], G.root_size, G.nroot[2], n.z);
    if (ix < 0 || iy < 0 || iz < 0) return -1;
    const int node = ix + G.nroot[0] * (iy + G.nroot[1] * iz);
    const float4 b = make_float4(G.root_lo[0] + float(ix) * G.root_size, G.root_lo[1] + float(iy) * G.root_size,
                                 G.root_lo[2] + float(iz) * G.root_size, G.root_size);
    return descend(G, node, b, p, n);
}

// Next leaf after leaving `leaf` through the faces in `tie` at exit point pe.
// Uses the face link of the lowest tied axis; falls back to a root descent
// when pe lies outside the linked node (edge/corner exits).
// Face links: >= 0 a refined node, -1 the model boundary, <= -2 a leaf
// (-(leaf + 2)).  On return *box holds the new leaf's box when the link led
// straight to a leaf (has_box = true).
// Face link codes (built on the host): >= 0 a refined node; -1 the model
// boundary; -(leaf + 2) a larger leaf; -(2^30) - leaf a leaf of the same size.
constexpr int kLinkSameSize = -(1 << 30);

// Follow the face link `code` of exit axis a out of the leaf with box cur to
// the leaf holding the exit point pe.  When the link leads straight to a leaf
// its box is returned in *box (computed for a same-size neighbour) and
// *has_box is set.
__device__ inline int follow_link(const DevGrid &G, int code, int a, int cur_leaf, const float4 cur,
                                  const float3 pe, const float3 n, float4 *box, bool *has_box) {
    *has_box = false;
    if (code == -1) return -1;
    if (code < 0) {
        int lf;
        float4 b;
        if (code <= kLinkSameSize) {
            lf = kLinkSameSize - code;
            b = cur;
            const float na = a == 0 ? n.x : (a == 1 ? n.y : n.z);
            const float sh = na > 0.f ? cur.w : -cur.w;
            if (a == 0) b.x += sh;
            else if (a == 1) b.y += sh;
            else b.z += sh;
        } else {
            lf = -code - 2;
            b = __ldg(&G.leaf_box[lf]);
        }
        if (inside_box(b, pe, n)) {
            *box = b;
            *has_box = true;
            return lf;
        }
        return locate_root(G, model_of_leaf(G, cur_leaf), pe, n);
    }
    const float4 b = __ldg(&G.node_box[code]);
    if (inside_box(b, pe, n)) return descend(G, code, b, pe, n);
    return locate_root(G, model_of_leaf(G, cur_leaf), pe, n);
}

__device__ inline int next_leaf(const DevGrid &G, int leaf, int tie, const float3 pe, const float3 n) {
    const int a = __ffs(tie) - 1;
    const float na = a == 0 ? n.x : (a == 1 ? n.y : n.z);
    const int code = __ldg(&G.leaf_rope[6 * leaf + 2 * a + (na > 0.f ? 1 : 0)]);
    float4 b;
    bool hb;
    return follow_link(G, code, a, leaf, __ldg(&G.leaf_box[leaf]), pe, n, &b, &hb);
}

// Reciprocal square root of the Henyey-Greenstein weights (Eq. 4): the
// hardware approximation with denormals flushed.  Its arguments,
// 1 + g^2 - 2g cos(theta), are at least (1 - |g|)^2, far from the denormal
// range.  The row sums Z and the row expansion both use it, so a row's
// normalisation and its expansion differ only in the rounding order of the
// dot product.
__device__ __forceinline__ float hg_rsqrt(float t) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(t));
    return r;
}

// ------------------------------------------------------- fixed-point sums
// Deterministic mode: a non-negative value v is accumulated as the integer
// round(v 2^e) in 64 bits.  Integer additions commute and associate, so the
// sums, and everything computed from them, do not depend on the order in
// which threads add.  Exponents are chosen per cell and wavelength so that
// an upper bound of the cell's total maps to at most 2^60.  The scaling by
// 2^e is exact (two powers of two, each a normal float).
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }
__device__ __forceinline__ unsigned long long to_fix(float v, int e) {
    const int e1 = e / 2;
    return __float2ull_rn(v * pow2f(e1) * pow2f(e - e1));
}
// ceil(log2(x)) for a positive normal float, exact
__device__ __forceinline__ int ceil_log2f(float x) {
    int e;
    const float f = frexpf(x, &e);  // x = f 2^e, f in [0.5, 1)
    return f == 0.5f ? e - 1 : e;
}
// exponent of the j_sca fixed point of a cell with extinction kr and side L:
// its pixels receive at most 4 L_emit min(1, 2 kr L) (eJ_base covers 4 L_emit)
__device__ __forceinline__ int cell_exp_jsca(int eJ_base, float kr, float L) {
    const float x = fminf(1.f, 2.f * kr * L);
    return eJ_base - (x > 0.f ? ceil_log2f(x) : 0);
}
// exponent of the U fixed point of a cell of side L (a power of two): the
// cell receives at most 4 sqrt(3) L_emit / (L^2 c) (eU_base covers the
// factor without L^-2)
__device__ __forceinline__ int cell_exp_u(int eU_base, float L) { return eU_base + 2 * ilogbf(L); }

// ------------------------------------------------------------------ rays
enum RayKind : int { kSeed = 0, kChild = 1, kMerged = 2, kResumed = 3 };

struct __align__(16) RayRec {
    unsigned long long pix;
    int src;
    float d;
    int hint;       // start leaf (>= 0) or -1
    float supp;     // merge test suppressed while the cell side equals this
    float plane;    // low list: coordinate of the entry plane
    unsigned meta;  // lev | kind << 8 | plane axis << 16
};
__device__ __host__ inline int rr_lev(unsigned m) { return static_cast<int>(m & 0xff); }
__device__ __host__ inline int rr_kind(unsigned m) { return static_cast<int>((m >> 8) & 0xff); }
// plane axis 0..2, or -1 (stored as 255) when the ray has no entry face
__device__ __host__ inline int rr_axis(unsigned m) {
    const int a = static_cast<int>((m >> 16) & 0xff);
    return a == 255 ? -1 : a;
}
__device__ __host__ inline unsigned rr_meta(int lev, int kind, int axis) {
    return unsigned(lev) | (unsigned(kind) << 8) | (unsigned(axis & 0xff) << 16);
}

// ledger slots (luminosities) and counters
enum { LG_EMITTED = 0, LG_DEPOSITED, LG_ESCAPED, LG_BLOCKED, LG_CUT, LG_SKIPPED, LG_N };
enum { CT_RAYS = 0, CT_CROSS, CT_SPLIT, CT_MERGE, CT_BLOCK, CT_ESCAPE, CT_CUT, CT_LOW, CT_RESUME,
       CT_WAVES, CT_SOURCES, CT_JPIX, CT_FLUSH, CT_REC, CT_N };

struct DevStats {
    double ledger[LG_N][kMaxLambda];
    unsigned long long cnt[CT_N];
    unsigned long long ledger_fix[LG_N][kMaxLambda];  // deterministic mode (fixed point, exponent eL)
};

// device status word
enum { ST_OK = 0, ST_CROSS_CAP = 1, ST_QUEUE = 2, ST_NOPROGRESS = 4, ST_MERGE = 8, ST_WAVE_CAP = 16 };

struct WaveCounters {
    unsigned long long fetch;   // next ray index to hand out
    unsigned long long n_high;  // parents appended to the high list
    unsigned long long n_low;   // rays appended to the low list
    unsigned long long n_next;  // explicit records of the next wave
    int status;
    int dbg_set;                // first ray that hit the crossing cap
    int dbg_src, dbg_lev, dbg_kind, dbg_leaf, dbg_prev;
    float dbg_d, dbg_te;
    unsigned long long dbg_pix;
};

// Device-resident state of one batch pipeline: the current wave's input
// sizes and buffer parity, so that consecutive waves are enqueued without the
// host reading counters in between.
struct PipeDev {
    long long nA, nB;         // current wave: implicit rays (seeds / children), explicit records
    int kind;                 // 0 seeds, 1 children + explicit
    int par;                  // input buffer parity
    int src_lo, nb_src;       // batch of sources
    int kstart;
    int done;                 // batch finished (or stopped on an error)
    long long peak;           // largest wave of the batch
    int waves;                // waves run
    int max_waves;
    long long hc;             // merge table size of the current wave
    int flush;                // record buffer flush requested
    int pad;
    unsigned long long peak_rec;  // most deposit records seen at a flush check
    WaveCounters wc;
};

}  // namespace dartray

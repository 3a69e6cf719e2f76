// Kernels of the ray-propagation sweep (Sect. 2, Sect. 3.1-3.5 of the paper):
// the ray marcher with split/merge/blocking tests and warp-cooperative
// deposit of the Henyey-Greenstein scattering source function, the low-list
// merge, source-table construction and the end-of-phase updates.
#pragma once

#include "march_kernel.cuh"

namespace dartray {

// ------------------------------------------------------------------ merging
struct MergeArgs {
    PipeDev *pd;
    const RayRec *L;
    const float *L_I;
    long long cap;
    unsigned long long *hkey;  // ~0 = empty
    int *hcnt;
    int4 *hmem;
    long long hcap;
    RayRec *Mb[2];
    float *MIb[2];
    DevStats *st;
    int nl;
};

__device__ inline unsigned long long merge_key(const RayRec &r) {
    return (static_cast<unsigned long long>(static_cast<unsigned>(r.src)) << 32) |
           (static_cast<unsigned long long>(rr_lev(r.meta)) << 28) | (r.pix >> 2);  // pix>>2 < 2^28 for k <= 13
}

__device__ inline unsigned long long hash64(unsigned long long k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

// Merge table size for the current wave: the power of two >= 2 n_low.
__global__ void merge_size_kernel(PipeDev *pd, long long hcap) {
    if (pd->done) return;
    const unsigned long long nl = pd->wc.n_low;
    long long hc = 0;
    if (nl > 0) {
        hc = 1;
        while (hc < 2 * static_cast<long long>(nl)) hc <<= 1;
        if (hc > hcap) {
            atomicOr(&pd->wc.status, ST_QUEUE);
            hc = 0;
        }
    }
    pd->hc = hc;
}

__global__ void merge_clear_kernel(const MergeArgs A) {
    const PipeDev *pd = A.pd;
    if (pd->done) return;
    const long long hc = pd->hc;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < hc;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        A.hkey[i] = ~0ull;
        A.hcnt[i] = 0;
    }
}

// Group low-list rays by (source, level, parent pixel).
__global__ void merge_insert_kernel(const MergeArgs A) {
    PipeDev *pd = A.pd;
    if (pd->done) return;
    const long long hc = pd->hc;
    const long long n_low = hc > 0 ? static_cast<long long>(min(pd->wc.n_low, static_cast<unsigned long long>(A.cap))) : 0;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n_low;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        if (A.L[i].src < 0) continue;  // hole of a warp's chunk
        const unsigned long long key = merge_key(A.L[i]);
        unsigned long long h = hash64(key) & static_cast<unsigned long long>(hc - 1);
        bool placed = false;
        for (long long probe = 0; probe < hc && !placed; ++probe) {
            const unsigned long long prev = atomicCAS(&A.hkey[h], ~0ull, key);
            if (prev == ~0ull || prev == key) {
                const int c = atomicAdd(&A.hcnt[h], 1);
                if (c < 4) reinterpret_cast<int *>(&A.hmem[h])[c] = static_cast<int>(i);
                else atomicOr(&pd->wc.status, ST_MERGE);
                placed = true;
            }
            h = (h + 1) & static_cast<unsigned long long>(hc - 1);
        }
        if (!placed) atomicOr(&pd->wc.status, ST_MERGE);
    }
}

// Eq. 3 / Fig. 1: four siblings that stopped on the same grid plane become
// their parent ray with the mean intensity at the mean distance; the others
// resume where they stopped with the merge test suppressed until the cell
// size changes.  Output: the explicit records of the next wave.
__global__ void merge_emit_kernel(const MergeArgs A) {
    PipeDev *pd = A.pd;
    if (pd->done) return;
    const long long hc = pd->hc;
    RayRec *M_out = A.Mb[1 - pd->par];
    float *M_out_I = A.MIb[1 - pd->par];
    for (long long h = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; h < hc;
         h += static_cast<long long>(gridDim.x) * blockDim.x) {
        if (A.hkey[h] == ~0ull) continue;
        const int c = min(A.hcnt[h], 4);
        int mem[4];
        const int4 hm = A.hmem[h];
        mem[0] = hm.x; mem[1] = hm.y; mem[2] = hm.z; mem[3] = hm.w;
        bool ok = (A.hcnt[h] == 4);
        if (ok) {
            // order the siblings by pixel (sums in a fixed order)
            for (int a = 0; a < 4; ++a)
                for (int b = a + 1; b < 4; ++b)
                    if (A.L[mem[b]].pix < A.L[mem[a]].pix) { const int t = mem[a]; mem[a] = mem[b]; mem[b] = t; }
            const RayRec &r0 = A.L[mem[0]];
            for (int a = 1; a < 4; ++a) {
                const RayRec &ra = A.L[mem[a]];
                ok = ok && rr_axis(ra.meta) == rr_axis(r0.meta) && ra.plane == r0.plane;
            }
        }
        if (ok) {
            const unsigned long long slot = atomicAdd(&pd->wc.n_next, 1ull);
            if (slot >= static_cast<unsigned long long>(A.cap)) { atomicOr(&pd->wc.status, ST_QUEUE); continue; }
            const RayRec &r0 = A.L[mem[0]];
            RayRec m;
            m.pix = r0.pix >> 2;
            m.src = r0.src;
            float dsum = 0.f;
            for (int a = 0; a < 4; ++a) dsum += A.L[mem[a]].d;
            m.d = dsum * 0.25f;
            m.hint = -1;
            m.supp = 0.f;
            m.plane = 0.f;
            m.meta = rr_meta(rr_lev(r0.meta) - 1, kMerged, -1);
            M_out[slot] = m;
            for (int l = 0; l < A.nl; ++l) {
                float sum = 0.f;
                for (int a = 0; a < 4; ++a) sum += A.L_I[l * A.cap + mem[a]];
                M_out_I[l * A.cap + slot] = sum * 0.25f;
            }
            atomicAdd(&A.st->cnt[CT_MERGE], 1ull);
        } else {
            const unsigned long long slot = atomicAdd(&pd->wc.n_next, static_cast<unsigned long long>(c));
            if (slot + c > static_cast<unsigned long long>(A.cap)) { atomicOr(&pd->wc.status, ST_QUEUE); continue; }
            for (int a = 0; a < c; ++a) {
                RayRec r = A.L[mem[a]];
                r.meta = rr_meta(rr_lev(r.meta), kResumed, rr_axis(r.meta));
                // r.hint (stop leaf) and r.supp (its side) were set by the marcher
                M_out[slot + a] = r;
                for (int l = 0; l < A.nl; ++l) M_out_I[l * A.cap + slot + a] = A.L_I[l * A.cap + mem[a]];
            }
            atomicAdd(&A.st->cnt[CT_RESUME], static_cast<unsigned long long>(c));
        }
    }
}

// End of a wave: the next wave consists of the four children of every
// high-list parent (implicit) and the merged / resumed records (explicit).
__global__ void wave_advance_kernel(PipeDev *pd) {
    if (pd->done) return;
    WaveCounters &w = pd->wc;
    if (w.status) {  // stop the batch; the host reads the status
        pd->done = 1;
        return;
    }
    const long long na = 4 * static_cast<long long>(w.n_high), nb = static_cast<long long>(w.n_next);
    pd->par ^= 1;
    pd->nA = na;
    pd->nB = nb;
    pd->kind = 1;
    w.fetch = 0;
    w.n_high = 0;
    w.n_low = 0;
    w.n_next = 0;
    pd->hc = 0;
    if (na + nb == 0) {
        pd->done = 1;
        return;
    }
    pd->waves += 1;
    if (na + nb > pd->peak) pd->peak = na + nb;
    if (pd->waves > pd->max_waves) {
        w.status |= ST_WAVE_CAP;
        pd->done = 1;
    }
}

// ------------------------------------------------------------------ sources
// flag[s] = 1 for sources of the phase: steps 1-2 emitting leaves and point
// sources; scattering iterations leaves whose pending row is non-zero at some
// wavelength; restricted to s % stride == offset.
__global__ void source_flags_kernel(const DevGrid G, int mode, const float *pend_src, int stride, int offset,
                                    int octant, const unsigned char *model_active, int *flags) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_all = mode == MODE_SCATTER ? G.n_leaf : G.n_leaf + G.n_point;
    if (s >= n_all) return;
    int on = 0;
    if (s < G.n_leaf) {
        for (int l = 0; l < G.nl_user && !on; ++l) {  // padding and derivatives make no sources
            if (mode == MODE_SCATTER) {
                const int np = 12 << (2 * G.k_lam[l]);
                const float *row = pend_src + G.off_lam[l] + static_cast<long long>(s) * np;
                for (int q = 0; q < np; ++q)
                    if (row[q] > 0.f) { on = 1; break; }
            } else {
                on = G.emis[static_cast<long long>(s) * G.nl + l] > 0.f;
            }
        }
    } else {
        for (int l = 0; l < G.nl_user; ++l) on |= G.point_lum[static_cast<long long>(s - G.n_leaf) * G.nl + l] > 0.f;
    }
    if (on && model_active) {
        // batched grids: models that have converged emit nothing more
        const int m = s < G.n_leaf ? model_of_leaf(G, s) : static_cast<int>(G.point_model[s - G.n_leaf]);
        on = model_active[m] != 0;
    }
    if (on && octant) {
        // octant mode: sources in the first octant (closed) only
        float x, y, z;
        if (s < G.n_leaf) {
            const float4 b = G.leaf_box[s];
            x = b.x + 0.5f * b.w;
            y = b.y + 0.5f * b.w;
            z = b.z + 0.5f * b.w;
        } else {
            const int ip = s - G.n_leaf;
            x = G.point_xyz[3 * ip];
            y = G.point_xyz[3 * ip + 1];
            z = G.point_xyz[3 * ip + 2];
        }
        on = x >= G.centre[0] && y >= G.centre[1] && z >= G.centre[2];
    }
    flags[s] = (on && (s % stride) == offset) ? 1 : 0;
}

// Batched grids: sources flagged per model.
__global__ void model_count_kernel(const DevGrid G, const int *flags, int n, int *count) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n || !flags[s]) return;
    const int m = s < G.n_leaf ? model_of_leaf(G, s) : static_cast<int>(G.point_model[s - G.n_leaf]);
    atomicAdd(&count[m], 1);
}

// Eq. 1 threshold of every cell: f_U U_LL, f_U = 4 a_RT / N_s of the cell's
// model (one value for a single model).
__global__ void threshold_kernel(const DevGrid G, const float *U_LL, const float *f_u_model, float *thr) {
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= static_cast<long long>(G.n_leaf) * G.nl) return;
    // a padding wavelength (no light, no dust) is negligible everywhere, so it
    // never keeps a ray going (Eq. 1 with an infinite threshold)
    thr[i] = static_cast<int>(i % G.nl) >= G.nl_user ? __int_as_float(0x7f800000)
                                                      : f_u_model[model_of_leaf(G, static_cast<int>(i / G.nl))] * U_LL[i];
}

// Block-level exclusive scan of flags -> per-block totals.
__global__ void scan_blocks_kernel(const PipeDev *pd, const int *flags, int n, int *block_sum) {
    __shared__ int sh[kBlock / kWarp];
    if (pd && !pd->flush) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int v = i < n ? flags[i] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < kBlock / kWarp; ++w) s += sh[w];
        block_sum[blockIdx.x] = s;
    }
}

__global__ void scan_offsets_kernel(const PipeDev *pd, int *block_sum, int nblocks, int *total) {
    if (pd && !pd->flush) return;
    // single thread: fine for <= a few 10^4 blocks
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int s = 0;
        for (int b = 0; b < nblocks; ++b) { const int v = block_sum[b]; block_sum[b] = s; s += v; }
        *total = s;
    }
}

__global__ void scatter_compact_kernel(const int *flags, int n, const int *block_off, int *out) {
    __shared__ int sh[kBlock / kWarp];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int f = i < n ? flags[i] : 0;
    const unsigned b = __ballot_sync(kFull, f);
    if (lane == 0) sh[w] = __popc(b);
    __syncthreads();
    int base = block_off[blockIdx.x];
    for (int k = 0; k < w; ++k) base += sh[k];
    if (f) out[base + __popc(b & ((1u << lane) - 1u))] = i;
}

// Octant mode: a source on k mirror planes is its own image under 2^k of the
// eight reflections; each of its deposits goes to all eight images of the
// cell with weight 1/2^k, so that the sum over its distinct images is
// counted once.  1 outside the octant mode.
__device__ inline float source_weight(const DevGrid &G, const float3 p) {
    if (!G.octant) return 1.f;
    const int k = (p.x == G.centre[0]) + (p.y == G.centre[1]) + (p.z == G.centre[2]);
    return 1.f / static_cast<float>(1 << k);
}

// Source table from the compacted indices.
__global__ void source_table_kernel(const DevGrid G, int mode, const int *idx, int n_src, int *src_leaf,
                                    int *src_hint, float4 *src_pos, float *src_S) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_src) return;
    const int s = idx[i];
    if (s < G.n_leaf) {
        const float4 b = G.leaf_box[s];
        const float3 c = make_float3(b.x + 0.5f * b.w, b.y + 0.5f * b.w, b.z + 0.5f * b.w);
        src_pos[i] = make_float4(c.x, c.y, c.z, source_weight(G, c));
        src_leaf[i] = s;
        src_hint[i] = s;
        if (mode != MODE_SCATTER)
            for (int l = 0; l < G.nl; ++l)
                src_S[static_cast<long long>(i) * G.nl + l] = G.emis[static_cast<long long>(s) * G.nl + l] * (b.w * b.w * b.w);
    } else {
        const int ip = s - G.n_leaf;
        const float3 p = make_float3(G.point_xyz[3 * ip], G.point_xyz[3 * ip + 1], G.point_xyz[3 * ip + 2]);
        src_pos[i] = make_float4(p.x, p.y, p.z, source_weight(G, p));
        src_leaf[i] = locate_root(G, G.n_models > 1 ? G.point_model[ip] : 0, p, make_float3(1.f, 1.f, 1.f));
        src_hint[i] = -1;
        for (int l = 0; l < G.nl; ++l)
            src_S[static_cast<long long>(i) * G.nl + l] =
                static_cast<float>(static_cast<double>(G.point_lum[static_cast<long long>(ip) * G.nl + l]) / (4.0 * kPi));
    }
}

// ------------------------------------------------------------------ set-up
// HG row normalisation per ray direction: Z[l][i] = sum_q (1 + g^2 -
// 2 g n_q.n_i)^(-3/2) over the j_sca pixels of wavelength l, for every
// tabulated ray direction i (levels 0..kDirTabLevels).
__global__ void ztab_kernel(const DevGrid G, float *ztab, long long ndt) {
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= ndt) return;
    const float4 n = G.dirtab[i];
    for (int l = 0; l < G.nl; ++l) {
        const int k = G.k_lam[l], np = 12 << (2 * k);
        const float B = 1.f + G.g[l] * G.g[l], Cg = 2.f * G.g[l];
        const float4 *pd = G.dirtab + dir_tab_offset(k);
        float z = 0.f;
        for (int q = 0; q < np; ++q) {
            const float4 v = pd[q];
            const float r = hg_rsqrt(B - Cg * (v.x * n.x + v.y * n.y + v.z * n.z));
            z += r * r * r;
        }
        ztab[l * ndt + i] = z;
    }
}

// Octant mode: image of every j_sca pixel (levels 0..3) under the seven
// reflections.  Pixel centres are exactly symmetric (their longitudes are
// reduced to the first octant), so the reflected centre lies inside -- at
// the centre of -- its image pixel.
__global__ void mirror_pix_kernel(int32_t *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 7 * kMirrorPix) return;
    const int m = i / kMirrorPix + 1, t = i % kMirrorPix;
    int k = 0;
    while (k < 3 && t >= dir_tab_offset(k + 1)) ++k;
    const int q = t - static_cast<int>(dir_tab_offset(k));
    double v[3];
    pix2vec_d(k, static_cast<uint64_t>(q), v);
    for (int a = 0; a < 3; ++a)
        if ((m >> a) & 1) v[a] = -v[a];
    out[i] = static_cast<int32_t>(vec2pix_d(k, v[0], v[1], v[2]));
}

// HEALPix pixel-centre table (levels 0..kDirTabLevels), computed in double.
__global__ void dirtab_kernel(float4 *tab, long long n) {
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    int k = 0;
    while (k < kDirTabLevels && i >= dir_tab_offset(k + 1)) ++k;
    double v[3];
    pix2vec_d(k, static_cast<uint64_t>(i - dir_tab_offset(k)), v);
    tab[i] = make_float4(static_cast<float>(v[0]), static_cast<float>(v[1]), static_cast<float>(v[2]), 0.f);
}

// L_abs = (1 - albedo) kappa*rho c V U
__global__ void labs_kernel(const DevGrid G, const float *U, float c_light, float *L_abs) {
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= static_cast<long long>(G.n_leaf) * G.nl) return;
    const int leaf = static_cast<int>(i / G.nl), l = static_cast<int>(i % G.nl);
    const float L = G.leaf_box[leaf].w;
    L_abs[i] = (1.f - G.albedo[l]) * G.kappa_rho[i] * c_light * (L * L * L) * U[i];
}

// ------------------------------------------------------- deferred deposit
// Records of depositing crossings are bucketed by cell (the marcher counts
// them per cell; scan; scatter) and each cell's scattering source-function
// row is accumulated by one warp holding the row in registers:
// pending[c][q] += sum over records of coef * Phi(n_q . n) / A, with
// Phi = A (1 + g^2 - 2 g mu)^(-3/2) (Eq. 4; the constant A cancels against
// the row normalisation already in coef).

// exclusive scan of per-cell counts: block totals, then per-element offsets
__global__ void scan_apply_kernel(const PipeDev *pd, const unsigned *cnt, int n, const int *block_off, unsigned *off,
                                  unsigned *cur) {
    if (pd && !pd->flush) return;
    __shared__ unsigned sh[kBlock / kWarp];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned v = i < n ? cnt[i] : 0u;
    unsigned incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) sh[w] = incl;
    __syncthreads();
    unsigned base = static_cast<unsigned>(block_off[blockIdx.x]);
    for (int k = 0; k < w; ++k) base += sh[k];
    if (i < n) {
        off[i] = base + incl - v;
        cur[i] = base + incl - v;
    }
}

// The flush runs when the pipeline's record buffer is half full (or when the
// host forces it); every flush kernel reads the decision and the record count
// from device memory.
__global__ void flush_decide_kernel(PipeDev *pd, const unsigned long long *rec_n, long long rec_cap, int force,
                                    DevStats *st) {
    const unsigned long long n = *rec_n;
    if (n > pd->peak_rec) pd->peak_rec = n;
    pd->flush = (n > 0 && (force || static_cast<long long>(n) >= rec_cap / 2)) ? 1 : 0;
    if (pd->flush) st->cnt[CT_FLUSH] += 1;  // single thread; the pipelines' stats words differ
}

// End of a flush: empty the buffer, and count the records it held (holes
// excluded) in the pipeline's stats word.
__global__ void flush_reset_kernel(PipeDev *pd, unsigned long long *rec_n, unsigned *cnt, int n_leaf,
                                   const int *n_sorted, DevStats *st) {
    if (!pd->flush) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_leaf; i += gridDim.x * blockDim.x) cnt[i] = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *rec_n = 0;
        st->cnt[CT_REC] += static_cast<unsigned long long>(*n_sorted);
    }
}

// Bucket records by cell (counting sort; the cursors start at the cells'
// offsets).  Consecutive records often share a cell (they come from one warp
// of the marcher), so the lanes of a warp that hold the same cell take their
// positions with one atomic.  A warp handles kScatterUnroll groups of 32
// records at once so that their cursor atomics are in flight together.
constexpr int kScatterUnroll = 4;
__global__ void rec_scatter_kernel(const PipeDev *pd, const unsigned long long *rec_n, const unsigned *cell,
                                   const float4 *dir, const float *coef, long long cap, int nl, unsigned *cur,
                                   float4 *sdir, float *scoef) {
    if (!pd->flush) return;
    const long long n = static_cast<long long>(min(*rec_n, static_cast<unsigned long long>(cap)));
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const long long warp = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
    const long long per = static_cast<long long>(kWarp) * kScatterUnroll;
    const long long stride = ((static_cast<long long>(gridDim.x) * blockDim.x) >> 5) * per;
    // warp-uniform trip count: the warp-wide match below is always converged
    for (long long base = warp * per; base < n; base += stride) {
        unsigned c[kScatterUnroll], peers[kScatterUnroll], pos[kScatterUnroll];
        float4 dv[kScatterUnroll];
#pragma unroll
        for (int u = 0; u < kScatterUnroll; ++u) {
            const long long i = base + u * kWarp + lane;
            c[u] = i < n ? cell[i] : 0xffffffffu;  // beyond the records, or a hole
            dv[u] = i < n ? dir[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kScatterUnroll; ++u) {
            peers[u] = __match_any_sync(kFull, c[u]);
            pos[u] = 0;
            if (c[u] != 0xffffffffu && lane == __ffs(peers[u]) - 1)
                pos[u] = atomicAdd(&cur[c[u]], static_cast<unsigned>(__popc(peers[u])));
        }
#pragma unroll
        for (int u = 0; u < kScatterUnroll; ++u) {
            const unsigned p = __shfl_sync(kFull, pos[u], __ffs(peers[u]) - 1) + __popc(peers[u] & below);
            if (c[u] != 0xffffffffu) {
                const long long i = base + u * kWarp + lane;
                sdir[p] = dv[u];
                if (nl > 1)
                    for (int l = 0; l < nl; ++l) scoef[l * cap + p] = coef[l * cap + i];
            }
        }
    }
}

// d j_sca / d g tally (gradient of maps with respect to g, the deposited
// luminosities held fixed): for every buffered record (cell c, ray direction
// n, coefficient a = L_sca / Z with Z = sum_q t_q^(-3/2), t_q = 1 + g^2 -
// 2g n_q.n) and the view pixel v of each wavelength,
//   dg[c] += a (3 (mu_v - g) t_v^(-5/2) - t_v^(-3/2) Z' / Z),
// Z' = sum_q 3 (mu_q - g) t_q^(-5/2): the derivative of L_sca t_v^(-3/2) / Z.
// One warp per record, the row sums over the warp's lanes.
__global__ void dg_tally_kernel(const DevGrid G, const PipeDev *pd, const unsigned long long *rec_n,
                                const unsigned *cell, const float4 *dir, const float *coef, long long cap,
                                const float4 *dg_dir, float *dg) {
    if (!pd->flush) return;
    const long long n = static_cast<long long>(min(*rec_n, static_cast<unsigned long long>(cap)));
    const int lane = threadIdx.x & 31;
    const long long warps = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
    for (long long i = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5; i < n; i += warps) {
        const unsigned c = cell[i];
        if (c == 0xffffffffu) continue;  // a hole
        const float4 dv = dir[i];
        for (int l = 0; l < G.nl; ++l) {
            const float a = G.nl == 1 ? dv.w : coef[l * cap + i];
            if (a == 0.f) continue;
            const int k = G.k_lam[l], np = 12 << (2 * k);
            const float g = G.g[l], B = 1.f + g * g, Cg = 2.f * g;
            float zs = 0.f, zg = 0.f;
            for (int q = lane; q < np; q += kWarp) {
                const float4 p = __ldg(&G.dirtab[dir_tab_offset(k) + q]);
                const float mu = p.x * dv.x + p.y * dv.y + p.z * dv.z;
                const float r = hg_rsqrt(B - Cg * mu), r3 = r * r * r;
                zs += r3;
                zg += 3.f * (mu - g) * r3 * r * r;
            }
            for (int o = 16; o > 0; o >>= 1) {
                zs += __shfl_xor_sync(kFull, zs, o);
                zg += __shfl_xor_sync(kFull, zg, o);
            }
            if (lane == 0) {
                const float4 v = __ldg(&dg_dir[l]);
                const float mu = v.x * dv.x + v.y * dv.y + v.z * dv.z;
                const float r = hg_rsqrt(B - Cg * mu), r3 = r * r * r;
                atomicAdd(&dg[static_cast<long long>(c) * G.nl + l], a * (3.f * (mu - g) * r3 * r * r - r3 * zg / zs));
            }
        }
    }
}

// The view pixel's direction per wavelength for the d j_sca / d g tally.
__global__ void dg_dir_kernel(const DevGrid G, double vx, double vy, double vz, float4 *out) {
    const int l = threadIdx.x;
    if (l >= G.nl) return;
    const int k = G.k_lam[l];
    out[l] = G.dirtab[dir_tab_offset(k) + static_cast<int>(vec2pix_d(k, vx, vy, vz))];
}

constexpr int kAccRange = 2048;  // records per warp work unit

// Packed single-precision pairs (sm_100+ f32x2): two IEEE fp32 operations per
// instruction.
__device__ __forceinline__ unsigned long long f2_pack(float2 a) {
    unsigned long long u;
    asm("mov.b64 %0, {%1, %2};" : "=l"(u) : "f"(a.x), "f"(a.y));
    return u;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long u) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(u));
    return a;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// The cell holding sorted record p: the last c with off[c] <= p (off is the
// exclusive prefix sum of the per-cell record counts).  32-way search, all
// lanes of the warp together.
__device__ inline int cell_of_record(const unsigned *off, int n_leaf, long long p, int lane) {
    int lo = 0, hi = n_leaf;  // off[lo] <= p; the answer lies in [lo, hi)
    while (hi - lo > 1) {
        const int step = (hi - lo + kWarp - 1) / kWarp;
        const long long c = lo + static_cast<long long>(lane + 1) * step;
        const bool le = c < hi && off[c] <= p;  // true on a prefix of the lanes
        const int k = __popc(__ballot_sync(kFull, le));
        lo += k * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

// From cell cur (whose records end at or before p) to the cell holding record
// p: the cells after cur are scanned 32 at a time.
__device__ inline int advance_cell(const unsigned *off, int n_leaf, int cur, long long p, int lane) {
    for (;;) {
        const long long c = static_cast<long long>(cur) + 1 + lane;
        const bool le = c < n_leaf && off[c] <= p;
        const int k = __popc(__ballot_sync(kFull, le));
        cur += k;
        if (k < kWarp) return cur;
    }
}

struct FlushArgs {
    const PipeDev *pd;
    const int *n_sorted;      // records bucketed (holes excluded)
    const unsigned *off;      // [n_leaf] exclusive prefix of the per-cell counts
    int n_leaf;
    const float4 *sdir;       // [cap] ray direction (w: coefficient with one wavelength), cell order
    const float *scoef;       // [nl][cap] coefficients (several wavelengths)
    long long cap;
    int packed;               // one wavelength: the coefficient is sdir.w
    float *pend;              // pending j_sca of the phase
    int det;                  // deterministic mode: fixed-point target and exponents
    unsigned long long *pend_fix;
    int eJ[kMaxLambda];
};

// Accumulate the sorted records [beg, end) of wavelength l into the pending
// rows; a row is added to its cell (with atomics: neighbouring ranges may
// share the cell) whenever the cell changes, the cell boundaries coming from
// the offsets.  Each lane owns PPL pixels, evaluated in pairs:
// t = 1 + g^2 - 2g n_q.n, w = t^(-3/2), acc += coef w.  Deterministic mode:
// every product coef * w is added in fixed point, so the row does not
// depend on the order of the records.
template <int PPL, bool DET>
__device__ inline void accumulate_range(const DevGrid &G, const FlushArgs &F, int l, long long beg, long long end,
                                        long long total, int lane, ulonglong2 *sh_rec, ulonglong2 *sh_rec2) {
    constexpr int NP2 = (PPL + 1) / 2;
    const int k = G.k_lam[l];
    const int np = 12 << (2 * k);
    const float B = 1.f + G.g[l] * G.g[l], Cg = 2.f * G.g[l];
    unsigned long long mx[NP2], my[NP2], mz[NP2];  // minus pixel directions
    unsigned long long acc[DET ? 1 : NP2];          // float pair sums
    unsigned long long fx[DET ? 2 * NP2 : 1];       // fixed-point sums
#pragma unroll
    for (int i = 0; i < NP2; ++i) {
        const int q0 = lane + kWarp * (2 * i), q1 = lane + kWarp * (2 * i + 1);
        const float4 a = q0 < np ? __ldg(&G.dirtab[dir_tab_offset(k) + q0]) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 b = q1 < np ? __ldg(&G.dirtab[dir_tab_offset(k) + q1]) : make_float4(0.f, 0.f, 0.f, 0.f);
        mx[i] = f2_pack(make_float2(-a.x, -b.x));
        my[i] = f2_pack(make_float2(-a.y, -b.y));
        mz[i] = f2_pack(make_float2(-a.z, -b.z));
    }
#pragma unroll
    for (int i = 0; i < (DET ? 1 : NP2); ++i) acc[i] = f2_pack(make_float2(0.f, 0.f));
#pragma unroll
    for (int i = 0; i < (DET ? 2 * NP2 : 1); ++i) fx[i] = 0ull;
    const unsigned long long B2 = f2_pack(make_float2(B, B));
    int cur = cell_of_record(F.off, F.n_leaf, beg, lane);
    long long nb = cur + 1 < F.n_leaf ? static_cast<long long>(F.off[cur + 1]) : total;  // end of cur's records
    int eJc = 0;
    auto cell_exp = [&](int c) {
        if (DET) eJc = cell_exp_jsca(F.eJ[l], __ldg(&G.kappa_rho[static_cast<long long>(c) * G.nl + l]),
                                     __ldg(&G.leaf_box[c]).w);
    };
    cell_exp(cur);
    auto flush = [&](int c) {
        const long long row = G.off_lam[l] + static_cast<long long>(c) * np;
#pragma unroll
        for (int i = 0; i < NP2; ++i) {
            const int q0 = lane + kWarp * (2 * i), q1 = lane + kWarp * (2 * i + 1);
            if (DET) {
                if (q0 < np && fx[2 * i]) atomicAdd(F.pend_fix + row + q0, fx[2 * i]);
                if (q1 < np && fx[2 * i + 1]) atomicAdd(F.pend_fix + row + q1, fx[2 * i + 1]);
                fx[2 * i] = fx[2 * i + 1] = 0ull;
            } else {
                const float2 v = f2_unpack(acc[DET ? 0 : i]);
                if (q0 < np && v.x != 0.f) atomicAdd(F.pend + row + q0, v.x);
                if (q1 < np && v.y != 0.f) atomicAdd(F.pend + row + q1, v.y);
                acc[DET ? 0 : i] = f2_pack(make_float2(0.f, 0.f));
            }
        }
    };
    for (long long b = beg; b < end; b += kWarp) {
        const long long r = b + lane;
        if (r < end) {
            // staged as duplicated pairs (x, x) so the loop below reads
            // ready-made f32x2 operands
            const float4 dv = F.sdir[r];
            const float cf = F.packed ? dv.w : F.scoef[l * F.cap + r];
            sh_rec[lane] = make_ulonglong2(f2_pack(make_float2(Cg * dv.x, Cg * dv.x)),
                                           f2_pack(make_float2(Cg * dv.y, Cg * dv.y)));
            sh_rec2[lane] = make_ulonglong2(f2_pack(make_float2(Cg * dv.z, Cg * dv.z)), f2_pack(make_float2(cf, cf)));
        }
        __syncwarp();
        const int cntj = static_cast<int>(min(static_cast<long long>(kWarp), end - b));
        int j = 0;
        while (j < cntj) {
            if (b + j >= nb) {  // warp-uniform: the next cell's records begin
                flush(cur);
                cur = advance_cell(F.off, F.n_leaf, cur, b + j, lane);
                nb = cur + 1 < F.n_leaf ? static_cast<long long>(F.off[cur + 1]) : total;
                cell_exp(cur);
            }
            const ulonglong2 ra = sh_rec[j], rb = sh_rec2[j];
            const unsigned long long cx = ra.x, cy = ra.y, cz = rb.x, cc = rb.y;
            if (!DET && j + 1 < cntj && b + j + 1 < nb) {
                // two records of the same cell: independent weight chains
                const ulonglong2 ra1 = sh_rec[j + 1], rb1 = sh_rec2[j + 1];
                const unsigned long long dx = ra1.x, dy = ra1.y, dz = rb1.x, dc = rb1.y;
#pragma unroll
                for (int i = 0; i < NP2; ++i) {
                    unsigned long long t = f2_fma(mx[i], cx, B2), u = f2_fma(mx[i], dx, B2);
                    t = f2_fma(my[i], cy, t);
                    u = f2_fma(my[i], dy, u);
                    t = f2_fma(mz[i], cz, t);
                    u = f2_fma(mz[i], dz, u);
                    const float2 tv = f2_unpack(t), uv = f2_unpack(u);
                    const unsigned long long rt = f2_pack(make_float2(hg_rsqrt(tv.x), hg_rsqrt(tv.y)));
                    const unsigned long long ru = f2_pack(make_float2(hg_rsqrt(uv.x), hg_rsqrt(uv.y)));
                    const unsigned long long wt = f2_mul(f2_mul(rt, rt), rt), wu = f2_mul(f2_mul(ru, ru), ru);
                    acc[DET ? 0 : i] = f2_fma(dc, wu, f2_fma(cc, wt, acc[DET ? 0 : i]));
                }
                j += 2;
            } else {
#pragma unroll
                for (int i = 0; i < NP2; ++i) {
                    unsigned long long t = f2_fma(mx[i], cx, B2);
                    t = f2_fma(my[i], cy, t);
                    t = f2_fma(mz[i], cz, t);
                    const float2 tv = f2_unpack(t);
                    const unsigned long long rr = f2_pack(make_float2(hg_rsqrt(tv.x), hg_rsqrt(tv.y)));
                    const unsigned long long w = f2_mul(f2_mul(rr, rr), rr);
                    if (DET) {
                        const float2 p = f2_unpack(f2_mul(cc, w));
                        fx[2 * i] += to_fix(p.x, eJc);
                        fx[2 * i + 1] += to_fix(p.y, eJc);
                    } else {
                        acc[DET ? 0 : i] = f2_fma(cc, w, acc[DET ? 0 : i]);
                    }
                }
                j += 1;
            }
        }
        __syncwarp();
    }
    flush(cur);
}

// Float mode with records merged first: rays of different sources that reach
// a cell at the same HEALPix level and pixel carry bitwise-equal directions,
// and their weight rows differ only by the coefficient, so a cell's records
// are summed per direction in a per-warp hash table (shared memory) and each
// distinct direction is expanded once.  Runs of fewer than kMergeMin records
// of one cell are expanded directly.
#ifndef DARTRAY_FLUSH_MERGE
#define DARTRAY_FLUSH_MERGE 1  // 0: expand every record (tuning builds)
#endif
constexpr int kMergeSlots = 256;                 // hash slots per warp
constexpr int kMergeMin = 64;                    // records of a cell worth merging
constexpr unsigned kEmptySlot = 0xffffffffu;     // x bits of an empty slot (a NaN: no direction)

__device__ __forceinline__ unsigned dir_hash(unsigned x, unsigned y, unsigned z) {
    unsigned h = x * 0x9E3779B1u ^ (y * 0x85EBCA77u + 0x27D4EB2Fu) ^ (z * 0xC2B2AE3Du + 0x165667B1u);
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    return h ^ (h >> 12);
}

template <int PPL>
__device__ inline void accumulate_range_merged(const DevGrid &G, const FlushArgs &F, int l, long long beg,
                                               long long end, long long total, int lane, ulonglong2 *sh_rec,
                                               ulonglong2 *sh_rec2, float4 *tab) {
    constexpr int NP2 = (PPL + 1) / 2;
    const int k = G.k_lam[l];
    const int np = 12 << (2 * k);
    const float B = 1.f + G.g[l] * G.g[l], Cg = 2.f * G.g[l];
    unsigned long long mx[NP2], my[NP2], mz[NP2], acc[NP2];
#pragma unroll
    for (int i = 0; i < NP2; ++i) {
        const int q0 = lane + kWarp * (2 * i), q1 = lane + kWarp * (2 * i + 1);
        const float4 a = q0 < np ? __ldg(&G.dirtab[dir_tab_offset(k) + q0]) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 b = q1 < np ? __ldg(&G.dirtab[dir_tab_offset(k) + q1]) : make_float4(0.f, 0.f, 0.f, 0.f);
        mx[i] = f2_pack(make_float2(-a.x, -b.x));
        my[i] = f2_pack(make_float2(-a.y, -b.y));
        mz[i] = f2_pack(make_float2(-a.z, -b.z));
        acc[i] = f2_pack(make_float2(0.f, 0.f));
    }
    const unsigned long long B2 = f2_pack(make_float2(B, B));
    const unsigned below = (1u << lane) - 1u;
    auto stage = [&](int pos, float x, float y, float z, float cf) {
        sh_rec[pos] = make_ulonglong2(f2_pack(make_float2(Cg * x, Cg * x)), f2_pack(make_float2(Cg * y, Cg * y)));
        sh_rec2[pos] = make_ulonglong2(f2_pack(make_float2(Cg * z, Cg * z)), f2_pack(make_float2(cf, cf)));
    };
    // the weights of cnt staged records (one cell) into acc, two at a time
    auto expand = [&](int cnt) {
        int j = 0;
        while (j < cnt) {
            const ulonglong2 ra = sh_rec[j], rb = sh_rec2[j];
            const unsigned long long cx = ra.x, cy = ra.y, cz = rb.x, cc = rb.y;
            if (j + 1 < cnt) {
                const ulonglong2 ra1 = sh_rec[j + 1], rb1 = sh_rec2[j + 1];
                const unsigned long long dx = ra1.x, dy = ra1.y, dz = rb1.x, dc = rb1.y;
#pragma unroll
                for (int i = 0; i < NP2; ++i) {
                    unsigned long long t = f2_fma(mx[i], cx, B2), u = f2_fma(mx[i], dx, B2);
                    t = f2_fma(my[i], cy, t);
                    u = f2_fma(my[i], dy, u);
                    t = f2_fma(mz[i], cz, t);
                    u = f2_fma(mz[i], dz, u);
                    const float2 tv = f2_unpack(t), uv = f2_unpack(u);
                    const unsigned long long rt = f2_pack(make_float2(hg_rsqrt(tv.x), hg_rsqrt(tv.y)));
                    const unsigned long long ru = f2_pack(make_float2(hg_rsqrt(uv.x), hg_rsqrt(uv.y)));
                    const unsigned long long wt = f2_mul(f2_mul(rt, rt), rt), wu = f2_mul(f2_mul(ru, ru), ru);
                    acc[i] = f2_fma(dc, wu, f2_fma(cc, wt, acc[i]));
                }
                j += 2;
            } else {
#pragma unroll
                for (int i = 0; i < NP2; ++i) {
                    unsigned long long t = f2_fma(mx[i], cx, B2);
                    t = f2_fma(my[i], cy, t);
                    t = f2_fma(mz[i], cz, t);
                    const float2 tv = f2_unpack(t);
                    const unsigned long long rr = f2_pack(make_float2(hg_rsqrt(tv.x), hg_rsqrt(tv.y)));
                    acc[i] = f2_fma(cc, f2_mul(f2_mul(rr, rr), rr), acc[i]);
                }
                j += 1;
            }
        }
    };
    auto flush = [&](int c) {
        const long long row = G.off_lam[l] + static_cast<long long>(c) * np;
#pragma unroll
        for (int i = 0; i < NP2; ++i) {
            const int q0 = lane + kWarp * (2 * i), q1 = lane + kWarp * (2 * i + 1);
            const float2 v = f2_unpack(acc[i]);
            if (q0 < np && v.x != 0.f) atomicAdd(F.pend + row + q0, v.x);
            if (q1 < np && v.y != 0.f) atomicAdd(F.pend + row + q1, v.y);
            acc[i] = f2_pack(make_float2(0.f, 0.f));
        }
    };
    for (int i = lane; i < kMergeSlots; i += kWarp) tab[i] = make_float4(__uint_as_float(kEmptySlot), 0.f, 0.f, 0.f);
    __syncwarp();
    int used = 0;  // occupied slots (warp-uniform)
    // expand every occupied slot and empty the table
    auto drain = [&]() {
        for (int base = 0; base < kMergeSlots; base += kWarp) {
            const float4 e = tab[base + lane];
            const bool occ = __float_as_uint(e.x) != kEmptySlot;
            const unsigned m = __ballot_sync(kFull, occ);
            if (occ) stage(__popc(m & below), e.x, e.y, e.z, e.w);
            __syncwarp();
            expand(__popc(m));
            __syncwarp();
            tab[base + lane] = make_float4(__uint_as_float(kEmptySlot), 0.f, 0.f, 0.f);
        }
        __syncwarp();
        used = 0;
    };
    int cur = cell_of_record(F.off, F.n_leaf, beg, lane);
    long long p = beg;
    while (p < end) {
        const long long nb = cur + 1 < F.n_leaf ? static_cast<long long>(F.off[cur + 1]) : total;
        const long long e = min(end, nb);  // cur's records in this range: [p, e)
        const bool merge = e - p >= kMergeMin;
        for (long long b = p; b < e; b += kWarp) {
            const long long r = b + lane;
            const bool have = r < e;
            const float4 dv = have ? F.sdir[r] : make_float4(__uint_as_float(kEmptySlot), 0.f, 0.f, 0.f);
            const float cf = have ? (F.packed ? dv.w : F.scoef[l * F.cap + r]) : 0.f;
            if (!merge) {
                if (have) stage(lane, dv.x, dv.y, dv.z, cf);
                __syncwarp();
                expand(static_cast<int>(min(static_cast<long long>(kWarp), e - b)));
                __syncwarp();
                continue;
            }
            if (used > kMergeSlots / 2) drain();  // at most 5/8 full after this chunk: probes end
            const unsigned kx = __float_as_uint(dv.x), ky = __float_as_uint(dv.y), kz = __float_as_uint(dv.z);
            // lanes holding the same direction: the lowest inserts, all add
            const unsigned same = __match_any_sync(kFull, (static_cast<unsigned long long>(kx) << 32) | ky) &
                                  __match_any_sync(kFull, kz);
            const int leader = __ffs(same) - 1;
            bool pending = have && lane == leader, claimed = false;
            const unsigned h = dir_hash(kx, ky, kz);
            int slot = 0;
            for (int probe = 0; __any_sync(kFull, pending); ++probe) {
                const int sl = static_cast<int>((h + static_cast<unsigned>(probe)) & (kMergeSlots - 1));
                if (pending &&
                    atomicCAS(reinterpret_cast<unsigned *>(&tab[sl].x), kEmptySlot, kx) == kEmptySlot) {
                    tab[sl].y = dv.y;
                    tab[sl].z = dv.z;
                    slot = sl;
                    pending = false;
                    claimed = true;
                }
                __syncwarp();  // keys claimed this round are complete
                if (pending) {
                    const float4 t = tab[sl];
                    if (__float_as_uint(t.x) == kx && __float_as_uint(t.y) == ky && __float_as_uint(t.z) == kz) {
                        slot = sl;
                        pending = false;
                    }
                }
                __syncwarp();
            }
            const int my_slot = __shfl_sync(kFull, slot, leader);
            if (have) atomicAdd(&tab[my_slot].w, cf);
            used += __popc(__ballot_sync(kFull, claimed));
            __syncwarp();
        }
        if (merge) drain();
        flush(cur);
        p = e;
        if (p < end) cur = advance_cell(F.off, F.n_leaf, cur, p, lane);
    }
}

template <int PPL, bool DET>
__global__ void __launch_bounds__(kBlock, PPL <= 6 ? 3 : 1) cell_accumulate_kernel(const DevGrid G, int l,
                                                                                     const FlushArgs F) {
    __shared__ ulonglong2 sh_rec[kBlock / kWarp][kWarp];
    __shared__ ulonglong2 sh_rec2[kBlock / kWarp][kWarp];
    __shared__ float4 sh_tab[DET ? 1 : kBlock / kWarp][DET ? 1 : kMergeSlots];
    if (!F.pd->flush) return;
    const long long n = static_cast<long long>(*F.n_sorted);  // records bucketed (holes excluded)
    const long long warps = static_cast<long long>(gridDim.x) * (blockDim.x / kWarp);
    // ranges of kAccRange records, fewer records per range (down to 256) when
    // the flush is too small to give every warp four ranges
    const long long per = max(256ll, min(static_cast<long long>(kAccRange), (n + 4 * warps - 1) / (4 * warps)));
    const long long nranges = (n + per - 1) / per;
    const int lane = threadIdx.x & 31;
    for (long long w = blockIdx.x * static_cast<long long>(blockDim.x / kWarp) + (threadIdx.x >> 5); w < nranges;
         w += warps) {
        const long long beg = w * per, end = min(n, beg + per);
        if (DET || !DARTRAY_FLUSH_MERGE)
            accumulate_range<PPL, DET>(G, F, l, beg, end, n, lane, sh_rec[threadIdx.x >> 5], sh_rec2[threadIdx.x >> 5]);
        else
            accumulate_range_merged<PPL>(G, F, l, beg, end, n, lane, sh_rec[threadIdx.x >> 5], sh_rec2[threadIdx.x >> 5],
                                         sh_tab[DET ? 0 : threadIdx.x >> 5]);
    }
}

// ------------------------------------------- deterministic-mode utilities
// Fixed point -> float at the end of a phase: out[i] = base[i] + fix[i] 2^-e
// with e the cell's exponent (RFED, [n_leaf][nl]).
struct Exps {
    int e[kMaxLambda];
};
// Octant mode: the sums of the cell's eight images (the deposits of the
// traced sources' images; every image has the same side and extinction, so
// the same exponent).
__global__ void fix_to_u_kernel(const DevGrid G, const unsigned long long *fix, const float *base, const Exps eU,
                                float *out) {
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= static_cast<long long>(G.n_leaf) * G.nl) return;
    const int c = static_cast<int>(i / G.nl), l = static_cast<int>(i % G.nl);
    const int e = cell_exp_u(eU.e[l], G.leaf_box[c].w);
    unsigned long long f = 0ull;
    for (int m = 0; m < (G.octant ? 8 : 1); ++m) f += fix[static_cast<long long>(mirror_leaf(G, m, c)) * G.nl + l];
    const float v = static_cast<float>(ldexp(static_cast<double>(f), -e));
    out[i] = base ? base[i] + v : v;
}

// Same for the pending j_sca rows of wavelength l.
__global__ void fix_to_jsca_kernel(const DevGrid G, int l, const unsigned long long *fix, const Exps eJ, float *out) {
    const int np = 12 << (2 * G.k_lam[l]);
    const long long n = static_cast<long long>(G.n_leaf) * np;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int c = static_cast<int>(i / np), q = static_cast<int>(i % np);
        const int e = cell_exp_jsca(eJ.e[l], G.kappa_rho[static_cast<long long>(c) * G.nl + l], G.leaf_box[c].w);
        unsigned long long f = 0ull;
        for (int m = 0; m < (G.octant ? 8 : 1); ++m)
            f += fix[G.off_lam[l] + static_cast<long long>(mirror_leaf(G, m, c)) * np + mirror_pixel(G, m, G.k_lam[l], q)];
        out[G.off_lam[l] + i] = static_cast<float>(ldexp(static_cast<double>(f), -e));
    }
}

// Octant mode (float sums): out = base + the sum of the eight images of each
// cell's deposits of the traced sources, for U ([n_leaf][nl])...
__global__ void octant_fold_u_kernel(const DevGrid G, const float *dep, const float *base, float *out) {
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= static_cast<long long>(G.n_leaf) * G.nl) return;
    const int c = static_cast<int>(i / G.nl), l = static_cast<int>(i % G.nl);
    float v = 0.f;
    for (int m = 0; m < 8; ++m) v += dep[static_cast<long long>(mirror_leaf(G, m, c)) * G.nl + l];
    out[i] = base ? base[i] + v : v;
}

// ... and for the pending j_sca rows of wavelength l, pixels reflected with
// their cell.
__global__ void octant_fold_jsca_kernel(const DevGrid G, int l, const float *dep, float *out) {
    const int np = 12 << (2 * G.k_lam[l]);
    const long long n = static_cast<long long>(G.n_leaf) * np;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int c = static_cast<int>(i / np), q = static_cast<int>(i % np);
        float v = 0.f;
        for (int m = 0; m < 8; ++m)
            v += dep[G.off_lam[l] + static_cast<long long>(mirror_leaf(G, m, c)) * np + mirror_pixel(G, m, G.k_lam[l], q)];
        out[G.off_lam[l] + i] = v;
    }
}

// ------------------------------------------------------- dust emission
// Equilibrium dust emission (Sect. 3.3) with a synthetic modified
// blackbody in place of grain models.  Per cell: the absorbed power
// P = sum over the stellar and the dust wavelengths of
// (1 - albedo) kappa*rho c V U dlambda; the temperature T where
// 4 pi V sum_i scale kabs_i B(lambda_i, T) dlambda_i = P (bisection in log T,
// double); the emissivity j_i = scale kabs_i B(lambda_i, T), with
// kabs_i = (1 - albedo_i) kappa*rho_i and B = lambda^-5 / (exp(c2 / (lambda T)) - 1)
// (lambda in um, c2 = 14387.77 um K).  The grid's emissivity becomes the
// change j - j_prev (clipped at 0), which the next self-heating step
// processes; j_prev <- j.
struct DustArgs {
    int n_leaf, n_ir, n_st;
    double lam[kMaxLambda], dlam[kMaxLambda], dlam_st[kMaxLambda];
    double scale, t_lo, t_hi, c_light;
    float alb_ir[kMaxLambda], alb_st[kMaxLambda];
    const float *U_ir, *kr_ir, *U_st, *kr_st;
    const float4 *leaf_box;
    float *j_prev;      // [n_leaf][n_ir] dust emissivity of the previous call
    float *emis;        // [n_leaf][n_ir] the grid's emissivity: the change to process
    float *T;           // [n_leaf] or null
    unsigned *max_rel;  // float bits of the largest relative change of j (non-negative)
};

__device__ inline double planck_um(double lam, double T) { return pow(lam, -5.0) / expm1(14387.77 / (lam * T)); }

__global__ void dust_emission_kernel(const DustArgs D) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= D.n_leaf) return;
    const double L = D.leaf_box[c].w, V = L * L * L;
    double P = 0.0;
    for (int s = 0; s < D.n_st; ++s)
        P += (1.0 - D.alb_st[s]) * D.kr_st[static_cast<long long>(c) * D.n_st + s] * D.c_light * V *
             D.U_st[static_cast<long long>(c) * D.n_st + s] * D.dlam_st[s];
    double kabs[kMaxLambda], ksum = 0.0;
    for (int i = 0; i < D.n_ir; ++i) {
        kabs[i] = (1.0 - D.alb_ir[i]) * D.kr_ir[static_cast<long long>(c) * D.n_ir + i];
        ksum += kabs[i];
        P += kabs[i] * D.c_light * V * D.U_ir[static_cast<long long>(c) * D.n_ir + i] * D.dlam[i];
    }
    double T = 0.0;
    if (P > 0.0 && ksum > 0.0) {
        double lo = log(D.t_lo), hi = log(D.t_hi);
        for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (lo + hi), Tm = exp(mid);
            double e = 0.0;
            for (int i = 0; i < D.n_ir; ++i) e += D.scale * kabs[i] * planck_um(D.lam[i], Tm) * D.dlam[i];
            if (4.0 * kPi * V * e < P) lo = mid;
            else hi = mid;
        }
        T = exp(0.5 * (lo + hi));
    }
    float rel = 0.f;
    for (int i = 0; i < D.n_ir; ++i) {
        const long long k = static_cast<long long>(c) * D.n_ir + i;
        const float j = T > 0.0 ? static_cast<float>(D.scale * kabs[i] * planck_um(D.lam[i], T)) : 0.f;
        const float jp = D.j_prev[k];
        D.emis[k] = fmaxf(j - jp, 0.f);
        if (jp > 0.f) rel = fmaxf(rel, fabsf(j - jp) / jp);
        else if (j > 0.f) rel = __int_as_float(0x7f800000);
        D.j_prev[k] = j;
    }
    if (D.T) D.T[c] = static_cast<float>(T);
    if (rel > 0.f) atomicMax(D.max_rel, __float_as_uint(rel));  // non-negative floats order as their bits
}

// Deterministic sum of n floats: a fixed grid, each block's partial (double)
// summed in a fixed order; the host adds the partials in order.
constexpr int kSumBlocks = 1024;
__global__ void det_sum_kernel(const float *x, long long n, long long stride, double *partial) {
    __shared__ double sh[kBlock];
    double s = 0.0;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        s += static_cast<double>(x[i * stride]);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = kBlock / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// Deterministic sums of segments in two passes with a fixed partition: block
// (seg, part) sums part `part` of `parts` equal chunks of segment seg, then
// one thread per segment adds the parts in order.
__global__ void segment_partial_kernel(const float *x, const long long *beg, const long long *len, int parts,
                                       double *partial) {
    __shared__ double sh[kBlock];
    const int seg = blockIdx.x, part = blockIdx.y;
    const long long n = len[seg], chunk = (n + parts - 1) / parts;
    const long long lo = beg[seg] + part * chunk, hi = beg[seg] + min(n, (part + 1) * chunk);
    double s = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) s += static_cast<double>(x[i]);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = kBlock / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[static_cast<long long>(seg) * parts + part] = sh[0];
}

__global__ void segment_finish_kernel(const double *partial, int nseg, int parts, double *out) {
    const int seg = blockIdx.x * blockDim.x + threadIdx.x;
    if (seg >= nseg) return;
    double s = 0.0;
    for (int p = 0; p < parts; ++p) s += partial[static_cast<long long>(seg) * parts + p];
    out[seg] = s;
}

// Forward mode: dL_abs/d albedo = kappa*rho c V ((1 - albedo) dU - U), the
// caller's [n_leaf][nl_user] layout (U at column l, dU at nl/2 + l).
__global__ void tangent_labs_kernel(const DevGrid G, const float *U, float c_light, float *out) {
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= static_cast<long long>(G.n_leaf) * G.nl_user) return;
    const int c = static_cast<int>(i / G.nl_user), l = static_cast<int>(i % G.nl_user);
    const float L = G.leaf_box[c].w;
    const long long r = static_cast<long long>(c) * G.nl;
    out[i] = G.kappa_rho[r + l] * c_light * (L * L * L) * ((1.f - G.albedo[l]) * U[r + G.nl / 2 + l] - U[r + l]);
}

// j_sca_total += pending, in place.
__global__ void add_pending_kernel(const float *pend, float *total, long long n) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        total[i] += pend[i];
}

}  // namespace dartray

// The ray marcher of the sweep (Sect. 2, Sect. 3.1-3.5 of the paper): one
// wave of rays, with the split / merge / blocking tests and the RFED and
// scattering source-function deposits of every crossing.
#pragma once

#include "device_common.cuh"

namespace dartray {

enum { MODE_LL = 0, MODE_DIRECT = 1, MODE_SCATTER = 2 };
constexpr int kBlock = 256;
// marcher blocks: 128 threads, 5 per SM with one wavelength (96 registers)
constexpr int kMarchBlock = 128;
#ifndef DARTRAY_MARCH_MIN_BLOCKS
#define DARTRAY_MARCH_MIN_BLOCKS 5
#endif
constexpr int kMarchMinBlocks1 = DARTRAY_MARCH_MIN_BLOCKS;  // resident blocks per SM, one wavelength
#ifndef DARTRAY_MARCH_WIDE_BLOCKS
#define DARTRAY_MARCH_WIDE_BLOCKS 1  // 0: the register budgets of the first wide build (tuning builds)
#endif
// Resident blocks per SM the register budget is set for: 2-4 wavelengths 4
// (128 registers, at most 12 bytes spilled), 8 wavelengths 3 (170, none
// spilled), 16 wavelengths 2 (more spill heavily).
constexpr int march_min_blocks(int nl) {
    return nl == 1 ? kMarchMinBlocks1
                   : (DARTRAY_MARCH_WIDE_BLOCKS ? (nl <= 4 ? 4 : (nl == 8 ? 3 : 2)) : (nl <= 4 ? 2 : 1));
}
constexpr int kPixTab = 1020;  // pixel centres of levels 0..3 (j_sca levels)

struct MarchArgs {
    // wave input (read from the pipeline state at launch): [0, nA) implicit
    // (seeds of sources src_lo.., or the 4 children of each high-list parent),
    // [nA, nA + nB) explicit records; buffers alternate by parity
    PipeDev *pd;
    RayRec *Hb[2];
    float *HIb[2];
    RayRec *Mb[2];
    float *MIb[2];
    const int *src_leaf;     // source cell (or the leaf holding a point source)
    const int *src_hint;     // start leaf of the seeds (-1: locate)
    const float4 *src_pos;   // source position
    const float *src_S;      // [n_src][nl] per-sr luminosity (direct light)
    // outputs
    RayRec *L_out;
    float *L_out_I;
    long long cap;           // records per queue (I arrays are [nl][cap])
    // fields
    float *target;           // U_LL (step 1) or U
    const float *U_LL;
    const float *thr;        // [n_leaf][nl] Eq. 1 threshold f_U U_LL (f_U of the cell's model)
    const float *pend_src;
    float *pend_dst;
    float f_u, r_pre, c_light;
    double split_c, merge_c; // 4 pi N_rays, 4 pi N_rays^max
    float split_cf, merge_cf;
    int k_ray_max, merge, max_cross;
    DevStats *st;
    // deferred j_sca deposit: one record per depositing crossing (cell, ray
    // direction, scattered luminosity / HG row sum per wavelength)
    unsigned *rec_cell;           // 0xffffffff marks an unused slot
    float4 *rec_dir;              // direction; w = coefficient when nl == 1
    float *rec_coef;              // [nl][rec_cap] (nl > 1 only)
    unsigned long long *rec_n;
    unsigned *rec_cnt;            // records per cell (for the bucketing)
    long long rec_cap;
    // deterministic mode: U and j_sca summed in fixed point (see to_fix)
    int det;
    unsigned long long *U_fix;    // [n_leaf][nl]
    unsigned long long *pend_fix; // j_sca layout
    int eU[kMaxLambda], eJ[kMaxLambda], eL[kMaxLambda];
    // batched grids: ledger per model, [model][slot][nl]
    double *mled;
    unsigned long long *mled_fix;
    // optional tally of d j_sca / d g for one view pixel per wavelength
    // ([n_leaf][nl]; null: off) and those pixels' directions ([nl])
    float *dg;
    const float4 *dg_dir;
};

// beam solid angle 4 pi / (12 4^k), scaled exactly from float(pi/3)
__device__ inline float omega_of(int k) { return ldexpf(static_cast<float>(kPi / 3.0), -2 * k); }

// Output lists are filled in per-warp chunks: a warp reserves `chunk` slots
// with one atomic and hands them out over many iterations, so appends rarely
// wait on a returning atomic.  Slots a warp leaves unused are holes, marked
// by the caller and skipped by the list's reader.
struct ChunkState {
    unsigned long long base;
    unsigned left;
    unsigned pad;
};

__device__ inline unsigned long long chunk_append(bool want, unsigned long long *counter, ChunkState *st,
                                                  unsigned chunk, int lane, unsigned long long *hole_beg,
                                                  unsigned *hole_n) {
    const unsigned m = __ballot_sync(kFull, want);
    *hole_n = 0;
    if (!m) return 0;
    const unsigned cnt = __popc(m);
    unsigned long long base = st->base;
    unsigned left = st->left;
    if (cnt > left) {
        *hole_beg = base;
        *hole_n = left;
        const unsigned take = max(chunk, cnt);
        unsigned long long nb = 0;
        if (lane == 0) nb = atomicAdd(counter, static_cast<unsigned long long>(take));
        base = __shfl_sync(kFull, nb, 0);
        left = take;
    }
    const unsigned long long slot = base + __popc(m & ((1u << lane) - 1u));
    __syncwarp();
    if (lane == 0) {
        st->base = base + cnt;
        st->left = left - cnt;
    }
    __syncwarp();
    return slot;
}

// Luminosity ledger of a lane: float32 sums in registers (few wavelengths)
// reduced in double across the warp once per launch, or (many wavelengths)
// double atomics in shared memory per finished ray.
template <int NL>
struct Ledger {
    static constexpr bool kReg = NL <= 4;
    float acc[kReg ? LG_N : 1][kReg ? NL : 1];
    __device__ void init() {
#pragma unroll
        for (int s = 0; s < (kReg ? LG_N : 1); ++s)
#pragma unroll
            for (int l = 0; l < (kReg ? NL : 1); ++l) acc[s][l] = 0.f;
    }
    __device__ void add(double (*sh)[kMaxLambda], int slot, const float *v, float scale) {
        if constexpr (kReg) {
#pragma unroll
            for (int l = 0; l < NL; ++l) acc[slot][l] = fmaf(v[l], scale, acc[slot][l]);
        } else {
#pragma unroll
            for (int l = 0; l < NL; ++l)
                if (v[l] != 0.f) atomicAdd(&sh[slot][l], static_cast<double>(v[l] * scale));
        }
    }
    __device__ void flush(double (*sh)[kMaxLambda], int lane) {
        if constexpr (kReg) {
#pragma unroll
            for (int s = 0; s < LG_N; ++s)
#pragma unroll
                for (int l = 0; l < NL; ++l) {
                    double v = acc[s][l];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
                    if (lane == 0 && v != 0.0) atomicAdd(&sh[s][l], v);
                }
        }
    }
};

/*
 * One wave of rays.  Persistent warps: each lane owns one ray and marches it
 * cell by cell; lanes that finish take the next ray of the wave.  Per
 * crossing (Sect. 2, 3.1.1, 3.2, 3.5):
 *   - segment [d, t_exit) of the current leaf, dtau = kappa*rho*ds;
 *   - outside the source cell: step 1 stops rays at d >= R_pre; steps 2-3
 *     mark wavelengths with dU = <I>/(r^2 c) < f_U U_LL negligible and block
 *     the ray when all are (Eq. 1 with the Sect. 3.5 dU, Omega_INT = L^2/r^2);
 *     Eq. 2 sends the ray to the high list, Eq. 3 to the low list (both
 *     compared exactly in double);
 *   - otherwise U += I Omega_k ds <I>/I / (V c) and the scattered luminosity
 *     albedo I Omega_k (1 - e^-dtau) is spread over the cell's j_sca pixels
 *     with normalised HG weights (Eq. 4) -- all 32 lanes of the warp share the
 *     pixel loop of each depositing lane.
 */
template <int NL, int MODE, bool DET>
__global__ void __launch_bounds__(kMarchBlock, march_min_blocks(NL)) march_kernel(const DevGrid G, const MarchArgs A) {
    __shared__ float4 sh_pix[kPixTab];
    __shared__ double sh_led[LG_N][kMaxLambda];
    __shared__ unsigned long long sh_fix[LG_N][kMaxLambda];  // deterministic ledger
    // batched grids: one ledger per model ([model][slot][NL]; doubles, or
    // fixed point in the deterministic mode), size given at launch
    extern __shared__ unsigned long long sh_mled[];
    __shared__ unsigned long long sh_cnt[CT_N];
    __shared__ ChunkState sh_chunk[kMarchBlock / kWarp][3];  // high list, low list, deposit records
    for (int i = threadIdx.x; i < kPixTab; i += blockDim.x) sh_pix[i] = G.dirtab[i];
    for (int i = threadIdx.x; i < LG_N * kMaxLambda; i += blockDim.x) {
        (&sh_led[0][0])[i] = 0.0;
        (&sh_fix[0][0])[i] = 0ull;
    }
    const int n_mled = G.n_models > 1 ? G.n_models * LG_N * NL : 0;
    for (int i = threadIdx.x; i < n_mled; i += blockDim.x) sh_mled[i] = 0ull;
    if (threadIdx.x < CT_N) sh_cnt[threadIdx.x] = 0;
    if (threadIdx.x < (kMarchBlock / kWarp) * 3) {
        ChunkState &c = (&sh_chunk[0][0])[threadIdx.x];
        c.base = 0;
        c.left = 0;
    }
    __syncthreads();

    const int lane = threadIdx.x & (kWarp - 1);
    ChunkState *chunks = sh_chunk[threadIdx.x >> 5];
    PipeDev *pd = A.pd;
    if (pd->done) return;  // uniform: the batch has no more rays
    const long long nA = pd->nA, n_total = pd->nA + pd->nB;
    const int par = pd->par, wave_kind = pd->kind, kstart = pd->kstart, src_lo = pd->src_lo;
    WaveCounters *wc = &pd->wc;
    float hgB[NL], hgC[NL], alb[NL];
    int npx[NL], pixbase[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        hgB[l] = 1.f + G.g[l] * G.g[l];
        hgC[l] = 2.f * G.g[l];
        alb[l] = G.albedo[l];
        npx[l] = 12 << (2 * G.k_lam[l]);
        pixbase[l] = static_cast<int>(dir_tab_offset(G.k_lam[l]));
    }

    bool active = false, exhausted = false;
    int src = 0, lev = 0, kind = 0, leaf = -1, srcleaf = -1, ncross = 0, entry_axis = -1;
    unsigned long long pix = 0;
    float3 xs = make_float3(0, 0, 0), n = make_float3(0, 0, 1);
    float d = 0.f, supp = 0.f, omega_k = 0.f, entry_coord = 0.f;
    float4 box = make_float4(0, 0, 0, 0);
    float3 inv = make_float3(0, 0, 0);
    bool first = true, dyadic_src = true, need_z = false;
    float I[NL], Z[NL], acc_dep[NL], acc_skip[NL];
    float kr[NL], ull[NL];  // kappa*rho and f_U U_LL of the current leaf (loaded with its box)
    int link[3] = {-1, -1, -1};  // face links of the current leaf in the direction of travel
#pragma unroll
    for (int l = 0; l < NL; ++l) { I[l] = 0.f; Z[l] = 1.f; acc_dep[l] = 0.f; acc_skip[l] = 0.f; }
    unsigned c_rays = 0, c_cross = 0, c_split = 0, c_block = 0, c_escape = 0, c_cut = 0, c_low = 0;
    Ledger<NL> led;
    led.init();
    constexpr bool det = DET;
    // ledger entry: float sums in registers, or in the deterministic mode a
    // fixed-point add per event (per finished ray, seed or deposit run)
    auto ledger = [&](int slot, const float *v, float scale) {
        if (G.n_models > 1) {
            // the model of the ray's source (src is set for every ray,
            // seeds included, before its first ledger entry)
            unsigned long long *ml = sh_mled + (model_of_leaf(G, __ldg(&A.src_leaf[src])) * LG_N + slot) * NL;
#pragma unroll
            for (int l = 0; l < NL; ++l) {
                const float x = v[l] * scale;
                if (!(x > 0.f)) continue;
                if (det) atomicAdd(ml + l, to_fix(x, A.eL[l]));
                else atomicAdd(reinterpret_cast<double *>(ml + l), static_cast<double>(x));
            }
            return;
        }
        if (det) {
#pragma unroll
            for (int l = 0; l < NL; ++l) {
                const float x = v[l] * scale;
                if (x > 0.f) atomicAdd(&sh_fix[slot][l], to_fix(x, A.eL[l]));
            }
        } else {
            led.add(sh_led, slot, v, scale);
        }
    };
    unsigned long long c_jpix = 0;  // j_sca pixels updated (lane 0 of each warp counts)

    for (;;) {
        // ---------------------------------------------------------- fetch
        // refill idle lanes once a quarter of the warp is idle (the ray setup
        // is divergent; sharing it among more lanes costs fewer instructions)
        const unsigned idle = __ballot_sync(kFull, !active);
        bool started = false;
        if (!exhausted && (__popc(idle) >= 8 || idle == kFull)) {
            const int leader = __ffs(idle) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(&wc->fetch, static_cast<unsigned long long>(__popc(idle)));
            base = __shfl_sync(kFull, base, leader);
            exhausted = base + __popc(idle) >= static_cast<unsigned long long>(n_total);
            if (!active) {
                const long long idx = static_cast<long long>(base + __popc(idle & ((1u << lane) - 1u)));
                if (idx < n_total) {
                    started = true;
                    active = true;
                    int hint = -1;
                    bool hole = false;
                    int par_axis = -1;
                    float par_coord = 0.f;
                    unsigned long long par_pix = 0;
                    int par_leaf = -1;
                    supp = 0.f;
                    entry_axis = -1;
                    entry_coord = 0.f;
                    if (idx < nA) {
                        if (wave_kind == 0) {
                            // idx < 2^32 (waves are bounded by the queues): 32-bit
                            // arithmetic, division by the constant 12
                            const unsigned u = static_cast<unsigned>(idx);
                            const unsigned hi = u >> (2 * kstart), lo = u & ((1u << (2 * kstart)) - 1u);
                            const unsigned s12 = hi / 12u;
                            src = src_lo + static_cast<int>(s12);
                            pix = (static_cast<unsigned long long>(hi - 12u * s12) << (2 * kstart)) | lo;
                            lev = kstart;
                            kind = kSeed;
                            d = 0.f;
                            hint = A.src_hint[src];
                            // octant mode: a source on k mirror planes carries weight 1/2^k
                            const float om = omega_of(lev) * __ldg(&A.src_pos[src].w);
                            float emit[NL];
#pragma unroll
                            for (int l = 0; l < NL; ++l) {
                                float s;
                                if (MODE == MODE_SCATTER) {
                                    const int kl = G.k_lam[l];
                                    const unsigned long long q = pix >> (2 * (lev - kl));
                                    s = A.pend_src[G.off_lam[l] + static_cast<long long>(A.src_leaf[src]) * npx[l] + q] /
                                        omega_of(kl);
                                } else {
                                    s = A.src_S[static_cast<long long>(src) * NL + l];
                                }
                                I[l] = s;
                                emit[l] = s;
                            }
                            ledger(LG_EMITTED, emit, om);
                        } else {
                            const long long pi_ = idx >> 2;
                            const RayRec r = A.Hb[par][pi_];
                            hole = r.src < 0;  // unused slot of a warp's chunk
                            src = hole ? 0 : r.src;
                            lev = rr_lev(r.meta) + 1;
                            pix = r.pix * 4ull + static_cast<unsigned long long>(idx & 3);
                            kind = kChild;
                            d = r.d;
                            par_axis = rr_axis(r.meta);
                            par_coord = r.plane;
                            par_pix = r.pix;
                            par_leaf = r.hint;  // the cell the parent split in
#pragma unroll
                            for (int l = 0; l < NL; ++l) I[l] = A.HIb[par][l * A.cap + pi_];
                        }
                    } else {
                        const long long mi = idx - nA;
                        const RayRec r = A.Mb[par][mi];
                        src = r.src;
                        lev = rr_lev(r.meta);
                        kind = rr_kind(r.meta);
                        pix = r.pix;
                        d = r.d;
                        hint = r.hint;
                        supp = r.supp;
                        if (kind == kResumed) {  // resumes on the face it stopped at
                            entry_axis = rr_axis(r.meta);
                            entry_coord = r.plane;
                        }
#pragma unroll
                        for (int l = 0; l < NL; ++l) I[l] = A.MIb[par][l * A.cap + mi];
                    }
                    if (hole) {
                        active = false;
                        started = false;
                    } else {
                    const float4 sp = A.src_pos[src];
                    xs = make_float3(sp.x, sp.y, sp.z);
                    srcleaf = A.src_leaf[src];
                    dyadic_src = A.src_hint[src] >= 0;  // cell sources sit on the dyadic lattice
                    n = ray_dir(G, lev, pix);
                    inv = make_float3(__frcp_rn(n.x), __frcp_rn(n.y), __frcp_rn(n.z));
                    // the beam solid angle times the source weight (1 outside the
                    // octant mode): deposits and the ledger scale with it, the
                    // Eq. 1-3 tests do not use it
                    omega_k = omega_of(lev) * sp.w;
                    need_z = false;
                    if (MODE != MODE_LL) {
                        if (lev <= kDirTabLevels) {
#pragma unroll
                            for (int l = 0; l < NL; ++l)
                                Z[l] = __ldg(&G.ztab[l * G.n_dirtab + dir_tab_offset(lev) + static_cast<long long>(pix)]);
                        } else {
                            need_z = true;
                        }
                    }
                    if (hint >= 0) {
                        leaf = hint;
                    } else {
                        float3 p = make_float3(fmaf(d, n.x, xs.x), fmaf(d, n.y, xs.y), fmaf(d, n.z, xs.z));
                        // a child sharing its parent's direction component along
                        // the parent's entry-face axis starts exactly on that face
                        if (par_axis >= 0) {
                            const float3 np_ = ray_dir(G, lev - 1, par_pix);
                            const float cn = par_axis == 0 ? n.x : (par_axis == 1 ? n.y : n.z);
                            const float cp = par_axis == 0 ? np_.x : (par_axis == 1 ? np_.y : np_.z);
                            if (cn == cp) {
                                if (par_axis == 0) p.x = par_coord;
                                else if (par_axis == 1) p.y = par_coord;
                                else p.z = par_coord;
                                entry_axis = par_axis;
                                entry_coord = par_coord;
                            }
                        }
                        // most children start in the cell their parent split in
                        if (par_leaf >= 0 && inside_box(__ldg(&G.leaf_box[par_leaf]), p, n)) leaf = par_leaf;
                        else leaf = locate_root(G, model_of_leaf(G, srcleaf), p, n);
                    }
                    if (leaf >= 0) {
                        box = __ldg(&G.leaf_box[leaf]);
#pragma unroll
                        for (int l = 0; l < NL; ++l) {
                            kr[l] = __ldg(&G.kappa_rho[static_cast<long long>(leaf) * NL + l]);
                            ull[l] = MODE == MODE_LL ? 0.f : __ldg(&A.thr[static_cast<long long>(leaf) * NL + l]);
                        }
                        link[0] = __ldg(&G.leaf_rope[6 * leaf + (n.x > 0.f ? 1 : 0)]);
                        link[1] = __ldg(&G.leaf_rope[6 * leaf + 2 + (n.y > 0.f ? 1 : 0)]);
                        link[2] = __ldg(&G.leaf_rope[6 * leaf + 4 + (n.z > 0.f ? 1 : 0)]);
                    }
                    first = true;
                    ncross = 0;
                    ++c_rays;
                    }  // not a hole
                }
            }
        }
        // done only when the wave's queue is exhausted: a refill can hand out
        // nothing but holes (unused chunk slots) while rays remain
        if (!__any_sync(kFull, active) && exhausted) break;

        // ------------------------------- HG normalisation of new rays (shared)
        if (MODE != MODE_LL) {
            unsigned m = __ballot_sync(kFull, started && need_z);
            while (m) {
                const int j = __ffs(m) - 1;
                m &= m - 1;
                const float nx = __shfl_sync(kFull, n.x, j), ny = __shfl_sync(kFull, n.y, j),
                            nz = __shfl_sync(kFull, n.z, j);
#pragma unroll
                for (int l = 0; l < NL; ++l) {
                    float part = 0.f;
                    for (int q = lane; q < npx[l]; q += kWarp) {
                        const float4 pd = sh_pix[pixbase[l] + q];
                        const float r = hg_rsqrt(hgB[l] - hgC[l] * (pd.x * nx + pd.y * ny + pd.z * nz));
                        part += r * r * r;
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
                    if (lane == j) Z[l] = part;
                }
            }
        }

        // ---------------------------------------------------------- crossing
        // outcome: 0 continue, 1 finished, 2 high list, 3 low list
        int outcome = 1;
        float sca[NL];
        float te = 0.f;
        int tie = 0;
        float bnd[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int l = 0; l < NL; ++l) sca[l] = 0.f;
        if (active) {
            if (leaf < 0) {
                float tmp[NL];
#pragma unroll
                for (int l = 0; l < NL; ++l) tmp[l] = I[l];
                ledger(LG_ESCAPED, tmp, omega_k);
                ++c_escape;
                outcome = 1;
            } else if (++ncross > A.max_cross) {
                atomicOr(&wc->status, ST_CROSS_CAP);
                if (atomicCAS(&wc->dbg_set, 0, 1) == 0) {
                    wc->dbg_src = src; wc->dbg_lev = lev; wc->dbg_kind = kind; wc->dbg_leaf = leaf;
                    wc->dbg_pix = pix; wc->dbg_d = d; wc->dbg_te = box.w; wc->dbg_prev = srcleaf;
                }
                outcome = 1;
            } else {
                ++c_cross;
                const float inf = __int_as_float(0x7f800000);
                bnd[0] = n.x > 0.f ? box.x + box.w : box.x;
                bnd[1] = n.y > 0.f ? box.y + box.w : box.y;
                bnd[2] = n.z > 0.f ? box.z + box.w : box.z;
                // reciprocal multiplies keep exact ties exact (equal offsets and
                // equal direction components give bitwise-equal distances)
                const float tx = n.x != 0.f ? (bnd[0] - xs.x) * inv.x : inf;
                const float ty = n.y != 0.f ? (bnd[1] - xs.y) * inv.y : inf;
                const float tz = n.z != 0.f ? (bnd[2] - xs.z) * inv.z : inf;
                te = fminf(tx, fminf(ty, tz));
                tie = (tx == te ? 1 : 0) | (ty == te ? 2 : 0) | (tz == te ? 4 : 0);
                if (tie == 0) {  // non-finite direction: never expected, never indexed
                    atomicOr(&wc->status, ST_NOPROGRESS);
                    active = false;
                }
                const float ds = fmaxf(te - d, 0.f);
                const float L = box.w, V = L * L * L;
                float fac[NL], T[NL];
                bool neg[NL];
#pragma unroll
                for (int l = 0; l < NL; ++l) {
                    // T = e^-dtau; fac = (1 - T)/dtau, the segment average of the
                    // attenuation (series below dtau = 1/64, where 1 - T cancels)
                    const float dtau = kr[l] * ds;
                    T[l] = __expf(-dtau);
                    fac[l] = dtau < 0.015625f
                                 ? fmaf(-0.5f * dtau, fmaf(-dtau * (1.f / 3.f), fmaf(-0.25f, dtau, 1.f), 1.f), 1.f)
                                 : __fdividef(1.f - T[l], dtau);
                    neg[l] = false;
                }
                outcome = active ? 0 : 1;
                if (outcome == 0 && leaf != srcleaf) {
                    // offset of the cell centre from the source (exact in float32
                    // for cell sources: dyadic coordinates)
                    const float hx = 0.5f * L;
                    const float dxf = (box.x + hx) - xs.x, dyf = (box.y + hx) - xs.y, dzf = (box.z + hx) - xs.z;
                    const float r2f = fmaf(dzf, dzf, fmaf(dyf, dyf, dxf * dxf));
                    if (MODE == MODE_LL) {
                        if (d >= (G.n_models > 1 ? G.models[model_of_leaf(G, leaf)].r_pre : A.r_pre)) {
                            float tmp[NL];
#pragma unroll
                            for (int l = 0; l < NL; ++l) tmp[l] = I[l];
                            ledger(LG_CUT, tmp, omega_k);
                            ++c_cut;
                            outcome = 1;
                        }
                    } else {
                        // Eq. 1: negligible when <I>/(r^2 c) < f_U U_LL
                        bool all = true;
#pragma unroll
                        for (int l = 0; l < NL; ++l) {
                            neg[l] = I[l] * fac[l] < ull[l] * (r2f * A.c_light);
                            all = all && neg[l];
                        }
                        // forward mode: a derivative (upper half, infinite
                        // threshold, so out of the test above) deposits where
                        // its wavelength does
                        if constexpr (NL >= 2) {
                            if (G.tangent) {
#pragma unroll
                                for (int l = NL / 2; l < NL; ++l) neg[l] = neg[l - NL / 2];
                            }
                        }
                        if (all) {
                            float tmp[NL];
#pragma unroll
                            for (int l = 0; l < NL; ++l) tmp[l] = I[l];
                            ledger(LG_BLOCKED, tmp, omega_k);
                            ++c_block;
                            outcome = 1;
                        }
                    }
                    const bool can_split = !(first && kind == kMerged) && lev < A.k_ray_max;
                    const bool can_merge = A.merge && lev > 0 && !first && L != supp;
                    if (outcome == 0 && (can_split || can_merge)) {
                        // Eq. 2 / Eq. 3 as 4 pi N r^2 vs 12 4^k L^2.  float32 decides
                        // unless within 1e-5 of the threshold (or the source is not
                        // on the dyadic lattice); then the exact double comparison.
                        const float rhs_f = ldexpf(12.f, 2 * lev) * L * L;
                        const float ls = A.split_cf * r2f, lm = A.merge_cf * r2f;
                        bool sp = ls > rhs_f, mg = lm < rhs_f;
                        if (!dyadic_src || fabsf(ls - rhs_f) <= 1e-5f * rhs_f || fabsf(lm - rhs_f) <= 1e-5f * rhs_f) {
                            const double Ld = static_cast<double>(L);
                            const double hd = __dmul_rn(0.5, Ld);
                            const double dx = __dsub_rn(__dadd_rn(static_cast<double>(box.x), hd), static_cast<double>(xs.x));
                            const double dy = __dsub_rn(__dadd_rn(static_cast<double>(box.y), hd), static_cast<double>(xs.y));
                            const double dz = __dsub_rn(__dadd_rn(static_cast<double>(box.z), hd), static_cast<double>(xs.z));
                            const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                            const double rhs = __dmul_rn(__dmul_rn(ldexp(12.0, 2 * lev), Ld), Ld);
                            sp = __dmul_rn(A.split_c, r2) > rhs;
                            mg = __dmul_rn(A.merge_c, r2) < rhs;
                        }
                        if (can_split && sp) {
                            outcome = 2;
                            ++c_split;
                        } else if (can_merge && mg) {
                            outcome = 3;
                            ++c_low;
                        }
                    }
                }
                if (outcome == 0) {
                    float lostv[NL];  // P_in (1 - T) of the segment, per wavelength
#pragma unroll
                    for (int l = 0; l < NL; ++l) {
                        const float P_in = I[l] * omega_k;
                        const float lost = P_in * kr[l] * ds * fac[l];
                        lostv[l] = lost;
                        if (neg[l]) {
                            acc_skip[l] += lost;
                        } else {
                            const float du = P_in * ds * fac[l] / (V * A.c_light);
                            if (du != 0.f) {
                                const long long ci = static_cast<long long>(leaf) * NL + l;
                                if (det) atomicAdd(&A.U_fix[ci], to_fix(du, cell_exp_u(A.eU[l], L)));
                                else atomicAdd(&A.target[ci], du);
                            }
                            if (MODE != MODE_LL) sca[l] = alb[l] * lost / Z[l];
                            acc_dep[l] += lost;
                        }
                        I[l] *= T[l];
                    }
                    // forward mode: d(albedo lost)/d albedo adds the light its
                    // wavelength lost over the segment (entering intensity)
                    if constexpr (NL >= 2 && MODE != MODE_LL) {
                        if (G.tangent) {
#pragma unroll
                            for (int l = NL / 2; l < NL; ++l)
                                if (!neg[l]) sca[l] += lostv[l - NL / 2] / Z[l - NL / 2];
                        }
                    }
                }
            }
        }

        // ------------------------------------------ high / low list appends
        {
            const bool wh = active && outcome == 2;
            unsigned long long hb;
            unsigned hn;
            const unsigned long long slot = chunk_append(wh, &wc->n_high, &chunks[0], 64u, lane, &hb, &hn);
            if (lane < static_cast<int>(hn) && hb + lane < static_cast<unsigned long long>(A.cap))
                A.Hb[1 - par][hb + lane].src = -1;
            if (wh) {
                if (slot < static_cast<unsigned long long>(A.cap)) {
                    RayRec r;
                    r.pix = pix; r.src = src; r.d = d; r.hint = leaf; r.supp = 0.f; r.plane = entry_coord;
                    r.meta = rr_meta(lev, kind, entry_axis);
                    A.Hb[1 - par][slot] = r;
#pragma unroll
                    for (int l = 0; l < NL; ++l) A.HIb[1 - par][l * A.cap + slot] = I[l];
                } else {
                    atomicOr(&wc->status, ST_QUEUE);
                }
            }
            const bool wl = active && outcome == 3;
            const unsigned long long slot2 = chunk_append(wl, &wc->n_low, &chunks[1], 32u, lane, &hb, &hn);
            if (lane < static_cast<int>(hn) && hb + lane < static_cast<unsigned long long>(A.cap))
                A.L_out[hb + lane].src = -1;
            if (wl) {
                if (slot2 < static_cast<unsigned long long>(A.cap)) {
                    RayRec r;
                    r.pix = pix; r.src = src; r.d = d; r.hint = leaf; r.supp = box.w; r.plane = entry_coord;
                    r.meta = rr_meta(lev, kind, entry_axis);
                    A.L_out[slot2] = r;
#pragma unroll
                    for (int l = 0; l < NL; ++l) A.L_out_I[l * A.cap + slot2] = I[l];
                } else {
                    atomicOr(&wc->status, ST_QUEUE);
                }
            }
        }

        // ------------------------------------------- j_sca deposit (Eq. 4)
        // Deferred: a record per depositing crossing, expanded per cell later
        // (cell_accumulate_kernel).  Lanes that find the record buffer full
        // deposit directly, all 32 lanes sharing the pixel loop.
        if (MODE != MODE_LL) {
            bool has = false;
#pragma unroll
            for (int l = 0; l < NL; ++l) has = has || (sca[l] > 0.f);
            has = has && active && outcome == 0;
            bool direct_dep = false;
            unsigned long long rb = 0;
            unsigned rn = 0;
            const unsigned long long rs = A.rec_cap > 0 ? chunk_append(has, A.rec_n, &chunks[2], 256u, lane, &rb, &rn) : 0ull;
            for (unsigned h = lane; h < rn; h += kWarp)
                if (rb + h < static_cast<unsigned long long>(A.rec_cap)) A.rec_cell[rb + h] = 0xffffffffu;
            if (has && A.rec_cap == 0) {
                direct_dep = true;
            } else if (has) {
                if (rs < static_cast<unsigned long long>(A.rec_cap)) {
                    atomicAdd(&A.rec_cnt[leaf], 1u);
                    A.rec_cell[rs] = static_cast<unsigned>(leaf);
                    // one wavelength: the coefficient rides in the direction's w
                    A.rec_dir[rs] = make_float4(n.x, n.y, n.z, NL == 1 ? sca[0] : 0.f);
#pragma unroll
                    for (int l = 0; l < NL; ++l) {
                        if (NL > 1) A.rec_coef[l * A.rec_cap + static_cast<long long>(rs)] = sca[l];
                        if (sca[l] != 0.f) c_jpix += static_cast<unsigned>(npx[l]);
                    }
                } else {
                    direct_dep = true;
                }
            }
            unsigned m = __ballot_sync(kFull, direct_dep);
            while (m) {
                const int j = __ffs(m) - 1;
                m &= m - 1;
                const int lj = __shfl_sync(kFull, leaf, j);
                const float nx = __shfl_sync(kFull, n.x, j), ny = __shfl_sync(kFull, n.y, j),
                            nz = __shfl_sync(kFull, n.z, j);
                const float Lj = __shfl_sync(kFull, box.w, j);
#pragma unroll
                for (int l = 0; l < NL; ++l) {
                    const float coef = __shfl_sync(kFull, sca[l], j);
                    if (coef == 0.f) continue;
                    c_jpix += (lane == j) ? static_cast<unsigned>(npx[l]) : 0u;
                    const long long row0 = G.off_lam[l] + static_cast<long long>(lj) * npx[l];
                    const int ej = det ? cell_exp_jsca(A.eJ[l], __shfl_sync(kFull, kr[l], j), Lj) : 0;
                    float zs = 0.f, zg = 0.f;  // row sum and its d/dg (tally only)
                    for (int q = lane; q < npx[l]; q += kWarp) {
                        const float4 pd = sh_pix[pixbase[l] + q];
                        const float mu = pd.x * nx + pd.y * ny + pd.z * nz;
                        const float r = hg_rsqrt(hgB[l] - hgC[l] * mu);
                        const float v = coef * (r * r * r);
                        if (det) atomicAdd(A.pend_fix + row0 + q, to_fix(v, ej));
                        else atomicAdd(A.pend_dst + row0 + q, v);
                        if (A.dg) {
                            zs += r * r * r;
                            zg += 3.f * (mu - 0.5f * hgC[l]) * (r * r * r * r * r);
                        }
                    }
                    if (A.dg) {  // uniform over the warp
                        for (int o = 16; o > 0; o >>= 1) {
                            zs += __shfl_xor_sync(kFull, zs, o);
                            zg += __shfl_xor_sync(kFull, zg, o);
                        }
                        if (lane == j) {
                            const float4 pv = __ldg(&A.dg_dir[l]);
                            const float mu = pv.x * nx + pv.y * ny + pv.z * nz;
                            const float r = hg_rsqrt(hgB[l] - hgC[l] * mu);
                            const float r3 = r * r * r;
                            atomicAdd(&A.dg[static_cast<long long>(lj) * NL + l],
                                      coef * (3.f * (mu - 0.5f * hgC[l]) * r3 * r * r - r3 * zg / zs));
                        }
                    }
                }
            }
        }

        // ---------------------------------------------------------- advance
        if (active) {
            if (outcome == 0) {
                d = fmaxf(te, d);
                entry_axis = __ffs(tie) - 1;
                entry_coord = bnd[entry_axis];
                // exit point on the closed box of the cell being left (clamped:
                // rounding must not put it in a cell behind the ray)
                const float3 pe = make_float3(
                    (tie & 1) ? bnd[0] : fminf(fmaxf(fmaf(te, n.x, xs.x), box.x), box.x + box.w),
                    (tie & 2) ? bnd[1] : fminf(fmaxf(fmaf(te, n.y, xs.y), box.y), box.y + box.w),
                    (tie & 4) ? bnd[2] : fminf(fmaxf(fmaf(te, n.z, xs.z), box.z), box.z + box.w));
                float4 nbox;
                bool has_box;
                const int ea = __ffs(tie) - 1;
                const int nxt = follow_link(G, ea == 0 ? link[0] : (ea == 1 ? link[1] : link[2]), ea, leaf, box, pe, n,
                                            &nbox, &has_box);
                if (nxt < 0) {
                    float tmp[NL];
#pragma unroll
                    for (int l = 0; l < NL; ++l) tmp[l] = I[l];
                    ledger(LG_ESCAPED, tmp, omega_k);
                    ++c_escape;
                    outcome = 1;
                } else if (nxt == leaf) {
                    atomicOr(&wc->status, ST_NOPROGRESS);
                    outcome = 1;
                } else {
                    leaf = nxt;
                    box = has_box ? nbox : __ldg(&G.leaf_box[leaf]);
#pragma unroll
                    for (int l = 0; l < NL; ++l) {
                        kr[l] = __ldg(&G.kappa_rho[static_cast<long long>(leaf) * NL + l]);
                        ull[l] = MODE == MODE_LL ? 0.f : __ldg(&A.thr[static_cast<long long>(leaf) * NL + l]);
                    }
                    link[0] = __ldg(&G.leaf_rope[6 * leaf + (n.x > 0.f ? 1 : 0)]);
                    link[1] = __ldg(&G.leaf_rope[6 * leaf + 2 + (n.y > 0.f ? 1 : 0)]);
                    link[2] = __ldg(&G.leaf_rope[6 * leaf + 4 + (n.z > 0.f ? 1 : 0)]);
                    if (supp != 0.f && box.w != supp) supp = 0.f;
                    first = false;
                }
            }
            if (outcome != 0) {
                ledger(LG_DEPOSITED, acc_dep, 1.f);
                ledger(LG_SKIPPED, acc_skip, 1.f);
#pragma unroll
                for (int l = 0; l < NL; ++l) { acc_dep[l] = 0.f; acc_skip[l] = 0.f; }
                active = false;
            }
        }
    }

    // ---------------------------------------------------------- flush
    // unused slots of this warp's chunks are holes for the lists' readers
    {
        const ChunkState c0 = chunks[0], c1 = chunks[1], c2 = chunks[2];
        for (unsigned h = lane; h < c0.left; h += kWarp)
            if (c0.base + h < static_cast<unsigned long long>(A.cap)) A.Hb[1 - par][c0.base + h].src = -1;
        for (unsigned h = lane; h < c1.left; h += kWarp)
            if (c1.base + h < static_cast<unsigned long long>(A.cap)) A.L_out[c1.base + h].src = -1;
        if (MODE != MODE_LL)
            for (unsigned h = lane; h < c2.left; h += kWarp)
                if (c2.base + h < static_cast<unsigned long long>(A.rec_cap)) A.rec_cell[c2.base + h] = 0xffffffffu;
    }
    if (!det) led.flush(sh_led, lane);
    atomicAdd(&sh_cnt[CT_RAYS], static_cast<unsigned long long>(c_rays));
    atomicAdd(&sh_cnt[CT_CROSS], static_cast<unsigned long long>(c_cross));
    atomicAdd(&sh_cnt[CT_SPLIT], static_cast<unsigned long long>(c_split));
    atomicAdd(&sh_cnt[CT_BLOCK], static_cast<unsigned long long>(c_block));
    atomicAdd(&sh_cnt[CT_ESCAPE], static_cast<unsigned long long>(c_escape));
    atomicAdd(&sh_cnt[CT_CUT], static_cast<unsigned long long>(c_cut));
    atomicAdd(&sh_cnt[CT_LOW], static_cast<unsigned long long>(c_low));
    if (c_jpix) atomicAdd(&sh_cnt[CT_JPIX], c_jpix);
    __syncthreads();
    for (int i = threadIdx.x; i < LG_N * NL; i += blockDim.x) {
        const int s = i / NL, l = i % NL;
        if (sh_led[s][l] != 0.0) atomicAdd(&A.st->ledger[s][l], sh_led[s][l]);
        if (sh_fix[s][l] != 0ull) atomicAdd(&A.st->ledger_fix[s][l], sh_fix[s][l]);
    }
    for (int i = threadIdx.x; i < n_mled; i += blockDim.x) {
        if (!sh_mled[i]) continue;
        if (det) atomicAdd(&A.mled_fix[i], sh_mled[i]);
        else atomicAdd(&A.mled[i], __longlong_as_double(static_cast<long long>(sh_mled[i])));
    }
    if (threadIdx.x < CT_N && sh_cnt[threadIdx.x]) atomicAdd(&A.st->cnt[threadIdx.x], sh_cnt[threadIdx.x]);
}

}  // namespace dartray

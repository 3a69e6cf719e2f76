// Kernels of the ray-propagation sweep (Sect. 2, Sect. 3.1-3.5 of the paper):
// the ray marcher with split/merge/blocking tests and warp-cooperative
// deposit of the Henyey-Greenstein scattering source function, the low-list
// merge, source-table construction and the end-of-phase updates.
#pragma once

#include "device_common.cuh"

namespace dartray {

enum { MODE_LL = 0, MODE_DIRECT = 1, MODE_SCATTER = 2 };
constexpr int kBlock = 256;
// marcher blocks: 128 threads, 5 per SM with one wavelength (96 registers)
constexpr int kMarchBlock = 128;
constexpr int kMarchMinBlocks1 = 5;
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
    const float *pend_src;
    float *pend_dst;
    float f_u, r_pre, c_light;
    double split_c, merge_c; // 4 pi N_rays, 4 pi N_rays^max
    float split_cf, merge_cf;
    int k_ray_max, merge, max_cross;
    DevStats *st;
    // deferred j_sca deposit: one record per depositing crossing (cell, ray
    // direction, scattered luminosity / HG row sum per wavelength)
    unsigned *rec_cell;
    float4 *rec_dir;              // direction; w = coefficient when nl == 1
    float *rec_coef;              // [nl][rec_cap] (nl > 1 only)
    unsigned long long *rec_n;
    unsigned *rec_cnt;            // records per cell (for the bucketing)
    long long rec_cap;
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
template <int NL, int MODE>
__global__ void __launch_bounds__(kMarchBlock, NL == 1 ? kMarchMinBlocks1 : (NL <= 4 ? 2 : 1)) march_kernel(const DevGrid G, const MarchArgs A) {
    __shared__ float4 sh_pix[kPixTab];
    __shared__ double sh_led[LG_N][kMaxLambda];
    __shared__ unsigned long long sh_cnt[CT_N];
    __shared__ ChunkState sh_chunk[kMarchBlock / kWarp][3];  // high list, low list, deposit records
    for (int i = threadIdx.x; i < kPixTab; i += blockDim.x) sh_pix[i] = G.dirtab[i];
    for (int i = threadIdx.x; i < LG_N * kMaxLambda; i += blockDim.x) (&sh_led[0][0])[i] = 0.0;
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
    float kr[NL], ull[NL];  // kappa*rho and U_LL of the current leaf (loaded with its box)
    int link[3] = {-1, -1, -1};  // face links of the current leaf in the direction of travel
#pragma unroll
    for (int l = 0; l < NL; ++l) { I[l] = 0.f; Z[l] = 1.f; acc_dep[l] = 0.f; acc_skip[l] = 0.f; }
    unsigned c_rays = 0, c_cross = 0, c_split = 0, c_block = 0, c_escape = 0, c_cut = 0, c_low = 0;
    Ledger<NL> led;
    led.init();
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
                            const float om = omega_of(lev);
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
                            led.add(sh_led, LG_EMITTED, emit, om);
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
                    omega_k = omega_of(lev);
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
                        else leaf = locate_root(G, p, n);
                    }
                    if (leaf >= 0) {
                        box = __ldg(&G.leaf_box[leaf]);
#pragma unroll
                        for (int l = 0; l < NL; ++l) {
                            kr[l] = __ldg(&G.kappa_rho[static_cast<long long>(leaf) * NL + l]);
                            ull[l] = MODE == MODE_LL ? 0.f : __ldg(&A.U_LL[static_cast<long long>(leaf) * NL + l]);
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
                led.add(sh_led, LG_ESCAPED, tmp, omega_k);
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
                        if (d >= A.r_pre) {
                            float tmp[NL];
#pragma unroll
                            for (int l = 0; l < NL; ++l) tmp[l] = I[l];
                            led.add(sh_led, LG_CUT, tmp, omega_k);
                            ++c_cut;
                            outcome = 1;
                        }
                    } else {
                        // Eq. 1: negligible when <I>/(r^2 c) < f_U U_LL
                        bool all = true;
#pragma unroll
                        for (int l = 0; l < NL; ++l) {
                            neg[l] = I[l] * fac[l] < A.f_u * ull[l] * (r2f * A.c_light);
                            all = all && neg[l];
                        }
                        if (all) {
                            float tmp[NL];
#pragma unroll
                            for (int l = 0; l < NL; ++l) tmp[l] = I[l];
                            led.add(sh_led, LG_BLOCKED, tmp, omega_k);
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
#pragma unroll
                    for (int l = 0; l < NL; ++l) {
                        const float P_in = I[l] * omega_k;
                        const float lost = P_in * kr[l] * ds * fac[l];
                        if (neg[l]) {
                            acc_skip[l] += lost;
                        } else {
                            const float du = P_in * ds * fac[l] / (V * A.c_light);
                            if (du != 0.f) atomicAdd(&A.target[static_cast<long long>(leaf) * NL + l], du);
                            acc_dep[l] += lost;
                            if (MODE != MODE_LL) sca[l] = alb[l] * lost / Z[l];
                        }
                        I[l] *= T[l];
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
#pragma unroll
                for (int l = 0; l < NL; ++l) {
                    const float coef = __shfl_sync(kFull, sca[l], j);
                    if (coef == 0.f) continue;
                    c_jpix += (lane == j) ? static_cast<unsigned>(npx[l]) : 0u;
                    float *row = A.pend_dst + G.off_lam[l] + static_cast<long long>(lj) * npx[l];
                    for (int q = lane; q < npx[l]; q += kWarp) {
                        const float4 pd = sh_pix[pixbase[l] + q];
                        const float r = hg_rsqrt(hgB[l] - hgC[l] * (pd.x * nx + pd.y * ny + pd.z * nz));
                        atomicAdd(row + q, coef * (r * r * r));
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
                const int nxt = follow_link(G, ea == 0 ? link[0] : (ea == 1 ? link[1] : link[2]), ea, box, pe, n,
                                            &nbox, &has_box);
                if (nxt < 0) {
                    float tmp[NL];
#pragma unroll
                    for (int l = 0; l < NL; ++l) tmp[l] = I[l];
                    led.add(sh_led, LG_ESCAPED, tmp, omega_k);
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
                        ull[l] = MODE == MODE_LL ? 0.f : __ldg(&A.U_LL[static_cast<long long>(leaf) * NL + l]);
                    }
                    link[0] = __ldg(&G.leaf_rope[6 * leaf + (n.x > 0.f ? 1 : 0)]);
                    link[1] = __ldg(&G.leaf_rope[6 * leaf + 2 + (n.y > 0.f ? 1 : 0)]);
                    link[2] = __ldg(&G.leaf_rope[6 * leaf + 4 + (n.z > 0.f ? 1 : 0)]);
                    if (supp != 0.f && box.w != supp) supp = 0.f;
                    first = false;
                }
            }
            if (outcome != 0) {
                led.add(sh_led, LG_DEPOSITED, acc_dep, 1.f);
                led.add(sh_led, LG_SKIPPED, acc_skip, 1.f);
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
    led.flush(sh_led, lane);
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
    }
    if (threadIdx.x < CT_N && sh_cnt[threadIdx.x]) atomicAdd(&A.st->cnt[threadIdx.x], sh_cnt[threadIdx.x]);
}

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
                                    int *flags) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_all = mode == MODE_SCATTER ? G.n_leaf : G.n_leaf + G.n_point;
    if (s >= n_all) return;
    int on = 0;
    if (s < G.n_leaf) {
        for (int l = 0; l < G.nl && !on; ++l) {
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
        for (int l = 0; l < G.nl; ++l) on |= G.point_lum[static_cast<long long>(s - G.n_leaf) * G.nl + l] > 0.f;
    }
    flags[s] = (on && (s % stride) == offset) ? 1 : 0;
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

// Source table from the compacted indices.
__global__ void source_table_kernel(const DevGrid G, int mode, const int *idx, int n_src, int *src_leaf,
                                    int *src_hint, float4 *src_pos, float *src_S) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_src) return;
    const int s = idx[i];
    if (s < G.n_leaf) {
        const float4 b = G.leaf_box[s];
        src_pos[i] = make_float4(b.x + 0.5f * b.w, b.y + 0.5f * b.w, b.z + 0.5f * b.w, 0.f);
        src_leaf[i] = s;
        src_hint[i] = s;
        if (mode != MODE_SCATTER)
            for (int l = 0; l < G.nl; ++l)
                src_S[static_cast<long long>(i) * G.nl + l] = G.emis[static_cast<long long>(s) * G.nl + l] * (b.w * b.w * b.w);
    } else {
        const int ip = s - G.n_leaf;
        const float3 p = make_float3(G.point_xyz[3 * ip], G.point_xyz[3 * ip + 1], G.point_xyz[3 * ip + 2]);
        src_pos[i] = make_float4(p.x, p.y, p.z, 0.f);
        src_leaf[i] = locate_root(G, p, make_float3(1.f, 1.f, 1.f));
        src_hint[i] = -1;
        for (int l = 0; l < G.nl; ++l)
            src_S[static_cast<long long>(i) * G.nl + l] =
                static_cast<float>(static_cast<double>(G.point_lum[static_cast<long long>(ip) * G.nl + l]) / (4.0 * kPi));
    }
}

// ------------------------------------------------------------------ phase end
// j_sca_total += pending; partial double sums of pending per block.
__global__ void accumulate_pending_kernel(const float *pend, float *total, long long n, double *sum) {
    __shared__ double sh[kBlock / kWarp];
    double s = 0.0;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const float v = pend[i];
        total[i] += v;
        s += v;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kBlock / kWarp; ++w) t += sh[w];
        atomicAdd(sum, t);
    }
}

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

__global__ void flush_reset_kernel(PipeDev *pd, unsigned long long *rec_n, unsigned *cnt, int n_leaf) {
    if (!pd->flush) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_leaf; i += gridDim.x * blockDim.x) cnt[i] = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) *rec_n = 0;
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

// Accumulate the sorted records [beg, end) of wavelength l into the pending
// rows; a row is flushed (with atomics: neighbouring ranges may share the
// cell) whenever the cell changes, the cell boundaries coming from the
// offsets.  Each lane owns PPL pixels, evaluated in pairs:
// t = 1 + g^2 - 2g n_q.n, w = t^(-3/2), acc += coef w.
template <int PPL>
__device__ inline void accumulate_range(const DevGrid &G, int l, long long beg, long long end, long long total,
                                        const unsigned *off, int n_leaf, const float4 *sdir, const float *scoef,
                                        long long cap, bool packed, float *pend, int lane, ulonglong2 *sh_rec,
                                        ulonglong2 *sh_rec2) {
    constexpr int NP2 = (PPL + 1) / 2;
    const int k = G.k_lam[l];
    const int np = 12 << (2 * k);
    const float B = 1.f + G.g[l] * G.g[l], Cg = 2.f * G.g[l];
    unsigned long long mx[NP2], my[NP2], mz[NP2], acc[NP2];  // minus pixel directions, sums
#pragma unroll
    for (int i = 0; i < NP2; ++i) {
        float2 vx, vy, vz;
        const int q0 = lane + kWarp * (2 * i), q1 = lane + kWarp * (2 * i + 1);
        const float4 a = q0 < np ? __ldg(&G.dirtab[dir_tab_offset(k) + q0]) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 b = q1 < np ? __ldg(&G.dirtab[dir_tab_offset(k) + q1]) : make_float4(0.f, 0.f, 0.f, 0.f);
        vx = make_float2(-a.x, -b.x);
        vy = make_float2(-a.y, -b.y);
        vz = make_float2(-a.z, -b.z);
        mx[i] = f2_pack(vx);
        my[i] = f2_pack(vy);
        mz[i] = f2_pack(vz);
        acc[i] = f2_pack(make_float2(0.f, 0.f));
    }
    const unsigned long long B2 = f2_pack(make_float2(B, B));
    int cur = cell_of_record(off, n_leaf, beg, lane);
    long long nb = cur + 1 < n_leaf ? static_cast<long long>(off[cur + 1]) : total;  // end of cur's records
    auto flush = [&](int c) {
        float *row = pend + G.off_lam[l] + static_cast<long long>(c) * np;
#pragma unroll
        for (int i = 0; i < NP2; ++i) {
            const float2 v = f2_unpack(acc[i]);
            const int q0 = lane + kWarp * (2 * i), q1 = lane + kWarp * (2 * i + 1);
            if (q0 < np && v.x != 0.f) atomicAdd(row + q0, v.x);
            if (q1 < np && v.y != 0.f) atomicAdd(row + q1, v.y);
            acc[i] = f2_pack(make_float2(0.f, 0.f));
        }
    };
    for (long long b = beg; b < end; b += kWarp) {
        const long long r = b + lane;
        if (r < end) {
            // staged as duplicated pairs (x, x) so the loop below reads
            // ready-made f32x2 operands
            const float4 dv = sdir[r];
            const float cf = packed ? dv.w : scoef[l * cap + r];
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
                cur = advance_cell(off, n_leaf, cur, b + j, lane);
                nb = cur + 1 < n_leaf ? static_cast<long long>(off[cur + 1]) : total;
            }
            const ulonglong2 ra = sh_rec[j], rb = sh_rec2[j];
            const unsigned long long cx = ra.x, cy = ra.y, cz = rb.x, cc = rb.y;
            if (j + 1 < cntj && b + j + 1 < nb) {
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
        __syncwarp();
    }
    flush(cur);
}

template <int PPL>
__global__ void __launch_bounds__(kBlock, PPL <= 6 ? 3 : 1) cell_accumulate_kernel(const DevGrid G, int l, const PipeDev *pd,
                                                                 const int *n_sorted, const unsigned *off,
                                                                 int n_leaf, const float4 *sdir,
                                                                 const float *scoef, long long cap, int packed,
                                                                 float *pend) {
    __shared__ ulonglong2 sh_rec[kBlock / kWarp][kWarp];
    __shared__ ulonglong2 sh_rec2[kBlock / kWarp][kWarp];
    if (!pd->flush) return;
    const long long n = static_cast<long long>(*n_sorted);  // records bucketed (holes excluded)
    const long long warps = static_cast<long long>(gridDim.x) * (blockDim.x / kWarp);
    // ranges of kAccRange records, fewer records per range (down to 256) when
    // the flush is too small to give every warp four ranges
    const long long per = max(256ll, min(static_cast<long long>(kAccRange), (n + 4 * warps - 1) / (4 * warps)));
    const long long nranges = (n + per - 1) / per;
    const int lane = threadIdx.x & 31;
    for (long long w = blockIdx.x * static_cast<long long>(blockDim.x / kWarp) + (threadIdx.x >> 5); w < nranges;
         w += warps) {
        const long long beg = w * per, end = min(n, beg + per);
        accumulate_range<PPL>(G, l, beg, end, n, off, n_leaf, sdir, scoef, cap, packed != 0, pend, lane,
                              sh_rec[threadIdx.x >> 5], sh_rec2[threadIdx.x >> 5]);
    }
}

}  // namespace dartray

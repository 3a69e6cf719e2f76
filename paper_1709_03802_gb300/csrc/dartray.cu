// C ABI of the sweep (include/dartray.h): grid creation, the phase driver
// (step 1 U_LL, step 2 direct light, scattering iterations; Sect. 2 of the
// paper), read-back, maps and state files.  All device work runs in the
// kernels of sweep_kernels.cuh and map_kernels.cuh; the host only sequences
// launches and moves small counters.
#include <cuda_runtime.h>

#include <algorithm>
#include <memory>
#include <mutex>
#include <chrono>
#include <thread>
#include <utility>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dartray.h"
#include "grid_host.h"
#include "map_kernels.cuh"
#include "march_wide.h"
#include "sweep_kernels.cuh"

using namespace dartray;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

#define CK(call)                                                                                       \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return fail(e_ == cudaErrorMemoryAllocation ? DARTRAY_E_NOMEM : DARTRAY_E_CUDA,            \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                          \
    } while (0)

template <class T>
cudaError_t dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
}

int k_hp_host(double g, int n_fwhm, int cap) {
    // Eq. 5: k = 0.5 log2(4 pi / (12 theta_min^2)), theta_min = FWHM/n_FWHM of
    // Phi - Phi(pi); integer part clamped to [0, cap]
    const double ga = std::fabs(g);
    if (ga < 1e-12) return 0;
    const double m = 0.5 * (std::pow(1.0 - ga, -3.0) + std::pow(1.0 + ga, -3.0));
    const double x = std::pow(m, -2.0 / 3.0);
    double mu = (1.0 + ga * ga - x) / (2.0 * ga);
    mu = std::min(1.0, std::max(-1.0, mu));
    const double th = 2.0 * std::acos(mu) / n_fwhm;
    const double kr = 0.5 * std::log2(4.0 * kPi / (12.0 * th * th));
    int k = kr < 0 ? 0 : static_cast<int>(std::floor(kr));
    return std::min(k, cap);
}

}  // namespace

#ifndef DARTRAY_PIPES
#define DARTRAY_PIPES 3  // ray pipelines (streams with their own queues and record buffers)
#endif
constexpr int kPipes = DARTRAY_PIPES;
constexpr int kMaxModels = 4096;
// two-pass segment sums: at most kSegParts parts per segment, kSegPartial partial sums in all
constexpr int kSegParts = 512;
constexpr int kSegPartial = 8192;

// Map staging buffer of dartray_map_noalloc: a fixed device array (8 MiB), so
// that entry point needs no allocation.  Every device that loads the library
// holds it until exit.
constexpr long long kNoAllocMapFloats = 1ll << 21;
static __device__ __align__(256) float g_noalloc_map[kNoAllocMapFloats];

struct Pipe {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    PipeDev *d_pd = nullptr;   // device state
    PipeDev *h_pd = nullptr;   // pinned host copy
    RayRec *d_H[2] = {nullptr, nullptr}, *d_M[2] = {nullptr, nullptr}, *d_L = nullptr;
    float *d_HI[2] = {nullptr, nullptr}, *d_MI[2] = {nullptr, nullptr}, *d_LI = nullptr;
    unsigned long long *d_hkey = nullptr;
    int *d_hcnt = nullptr;
    int4 *d_hmem = nullptr;
    // deferred deposit records (cell, ray direction, HG coefficients) and
    // their copy in cell order
    unsigned *d_rec_cell = nullptr, *d_cnt = nullptr, *d_off = nullptr, *d_cur = nullptr;
    float4 *d_rec_dir = nullptr, *d_srt_dir = nullptr;
    float *d_rec_coef = nullptr, *d_srt_coef = nullptr;
    unsigned long long *d_rec_n = nullptr;
    int *d_blocksum = nullptr, *d_total = nullptr;
    DevStats *d_st = nullptr;  // this pipeline's flush counter (cnt[CT_FLUSH] only)
    // host-side batch bookkeeping
    bool active = false;
    int src_lo = 0, nb = 0;
};

struct dartray_grid {
    int device = 0;
    cudaStream_t stream = nullptr;
    dartray_params P{};
    int nl = 0, n_leaf = 0, n_nodes = 0, n_point = 0;
    // the caller's wavelength count; nl is it rounded up to a marcher width
    // (1, 2, 4, 8, 16), the extra wavelengths having no dust and no emission
    int nlu = 0;
    DevGrid G{};
    HostTopo topo;
    // device arrays
    int32_t *d_node_child = nullptr, *d_rope = nullptr;
    float4 *d_node_box = nullptr, *d_leaf_box = nullptr, *d_dirtab = nullptr;
    float *d_ztab = nullptr;
    float *d_kr = nullptr, *d_emis = nullptr, *d_pxyz = nullptr, *d_plum = nullptr;
    float *d_U = nullptr, *d_ULL = nullptr, *d_pend[2] = {nullptr, nullptr}, *d_jtot = nullptr;
    int cur = 0;  // d_pend[cur]: luminosity to emit; d_pend[1-cur]: deposit target
    long long sca_len = 0;
    long long sca_len_user = 0;  // the j_sca blocks of the caller's wavelengths
    int k_lam[kMaxLambda] = {0};
    long long off_lam[kMaxLambda] = {0};
    // sources
    int *d_flags = nullptr, *d_blocksum = nullptr, *d_total = nullptr, *d_src_idx = nullptr;
    int *d_src_leaf = nullptr, *d_src_hint = nullptr;
    float4 *d_src_pos = nullptr;
    float *d_src_S = nullptr;
    // batch pipelines (each with its own stream, queues, merge table and
    // deposit-record buffer)
    Pipe pipe[kPipes];
    long long cap = 0;
    long long hcap = 0;
    DevStats *d_st = nullptr;
    double *d_sum = nullptr;
    double l_sca2 = 0.0;
    bool have_direct = false;
    long long launches = 0;
    int num_sms = 1;
    int march_blocks = 1;
    int acc_blocks[8] = {1, 1, 1, 1, 1, 1, 1, 1};  // resident blocks of cell_accumulate_kernel<1, 2, 6, 24> (x2: det)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    long long rec_cap = 0;    // record capacity in use (0: per-pixel atomic deposit); <= rec_alloc
    long long rec_alloc = 0;  // record capacity allocated
    cudaEvent_t mev0 = nullptr, mev1 = nullptr;  // around each march launch (profile mode)
    double march_ms = 0.0, flush_ms = 0.0, busy_ms = 0.0, march_sum_ms = 0.0;
    long long march_launches = 0, restarts = 0, batches = 0;
    // peak rays per source of each mode's waves, learned by earlier calls: the
    // first batch of a phase is sized with it (0: not yet known)
    double rays_per_src[3] = {0.0, 0.0, 0.0};
    // staging buffer for results computed on the device and returned to host
    // memory (L_abs, maps): allocated on first use, grown on demand, owned by
    // the grid
    float *d_stage = nullptr;
    size_t stage_floats = 0;
    // deterministic mode: fixed-point sums of U and of the pending j_sca of
    // the running phase, with per-wavelength exponents (see to_fix)
    unsigned long long *d_Ufix = nullptr, *d_pfix = nullptr;
    int32_t *d_mirror = nullptr, *d_mirror_pix = nullptr;  // octant mode
    float *d_oct_u = nullptr, *d_oct_p = nullptr;           // octant mode: deposits of the traced sources
    float *d_thr = nullptr;       // [n_leaf][nl] Eq. 1 thresholds f_U U_LL of the running phase
    float *d_fu_model = nullptr;  // [n_models] f_U of the running phase
    // batched grids (several models in one forest)
    int n_models = 1;
    ModelDev *d_models = nullptr;
    uint16_t *d_leaf_model = nullptr, *d_point_model = nullptr;
    unsigned char *d_model_active = nullptr;
    int *d_mcount = nullptr;
    double *d_mled = nullptr;
    unsigned long long *d_mled_fix = nullptr;
    long long *d_seg_beg = nullptr, *d_seg_len = nullptr;  // (model, wavelength) blocks of the j_sca array
    double *d_seg_out = nullptr, *d_seg_part = nullptr;
    int march_smem = 0;
    std::vector<long long> m_leaf0, m_point0;
    std::vector<int> m_nleaf;
    std::vector<double> m_lsca2, m_rem, m_fu;
    std::vector<unsigned char> m_active;
    std::vector<double> m_ledger;  // [n_models][LG_N][nl] of the last phase of the last call
    float *d_jd = nullptr;         // dust emission of the last dartray_dust_emission call
    unsigned *d_maxrel = nullptr;
    // d j_sca / d g tally for one view (dartray_jsca_dg_arm): the total since
    // dartray_direct, the current phase's part, the view pixels' directions
    bool dg_on = false, dg_phase_live = false;
    double dg_view[3] = {0.0, 0.0, 0.0};
    float *d_dg = nullptr, *d_dg_phase = nullptr;
    float4 *d_dg_dir = nullptr;
    Exps eU{}, eJ{}, eL{};
    double *d_partial = nullptr, *h_partial = nullptr;  // deterministic sums
};

namespace {

void free_all(dartray_grid *g) {
    void *ptrs[] = {g->d_ztab, g->d_node_child, g->d_rope, g->d_node_box, g->d_leaf_box, g->d_dirtab, g->d_kr,
                    g->d_emis, g->d_pxyz, g->d_plum, g->d_U, g->d_ULL, g->d_pend[0], g->d_pend[1], g->d_jtot,
                    g->d_flags, g->d_blocksum, g->d_total, g->d_src_idx, g->d_src_leaf, g->d_src_hint,
                    g->d_src_pos, g->d_src_S, g->d_st, g->d_sum, g->d_stage, g->d_Ufix, g->d_pfix,
                    g->d_partial, g->d_mirror, g->d_mirror_pix, g->d_oct_u, g->d_oct_p, g->d_thr,
                    g->d_fu_model, g->d_models, g->d_leaf_model, g->d_point_model, g->d_model_active,
                    g->d_mcount, g->d_mled, g->d_mled_fix, g->d_seg_beg, g->d_seg_len, g->d_seg_out, g->d_seg_part,
                    g->d_jd, g->d_maxrel, g->d_dg, g->d_dg_phase, g->d_dg_dir};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (int i = 0; i < kPipes; ++i) {
        Pipe &P = g->pipe[i];
        void *pp[] = {P.d_pd, P.d_H[0], P.d_H[1], P.d_M[0], P.d_M[1], P.d_L, P.d_HI[0], P.d_HI[1], P.d_MI[0],
                      P.d_MI[1], P.d_LI, P.d_hkey, P.d_hcnt, P.d_hmem, P.d_rec_cell, P.d_cnt,
                      P.d_off, P.d_cur, P.d_rec_dir, P.d_srt_dir, P.d_rec_coef, P.d_srt_coef, P.d_rec_n,
                      P.d_blocksum, P.d_total, P.d_st};
        for (void *p : pp)
            if (p) cudaFree(p);
        if (P.h_pd) cudaFreeHost(P.h_pd);
        if (P.ev) cudaEventDestroy(P.ev);
        if (P.stream) cudaStreamDestroy(P.stream);
    }
    if (g->h_partial) cudaFreeHost(g->h_partial);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    if (g->mev0) cudaEventDestroy(g->mev0);
    if (g->mev1) cudaEventDestroy(g->mev1);
}

template <class T>
int copy_in(T *dst, const T *src, size_t count, bool on_device, cudaStream_t s) {
    if (count == 0) return DARTRAY_OK;
    if (!src) return fail(DARTRAY_E_INVAL, "missing input array");
    CK(cudaMemcpyAsync(dst, src, count * sizeof(T), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    return DARTRAY_OK;
}

// Per-wavelength arrays: the caller's [rows][nlu] <-> the library's
// [rows][nl] (extra columns zero).
int copy_in_cols(float *dst, const float *src, size_t rows, int nlu, int nl, bool on_device, cudaStream_t s) {
    if (nlu == nl) return copy_in(dst, src, rows * nl, on_device, s);
    if (rows == 0) return DARTRAY_OK;
    if (!src) return fail(DARTRAY_E_INVAL, "missing input array");
    CK(cudaMemsetAsync(dst, 0, rows * nl * sizeof(float), s));
    CK(cudaMemcpy2DAsync(dst, nl * sizeof(float), src, nlu * sizeof(float), nlu * sizeof(float), rows,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    return DARTRAY_OK;
}

int copy_out_cols(float *dst, const float *src, size_t rows, int nlu, int nl, bool dst_is_device, cudaStream_t s) {
    if (rows == 0) return DARTRAY_OK;
    const cudaMemcpyKind k = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (nlu == nl) CK(cudaMemcpyAsync(dst, src, rows * nl * sizeof(float), k, s));
    else CK(cudaMemcpy2DAsync(dst, nlu * sizeof(float), src, nl * sizeof(float), nlu * sizeof(float), rows, k, s));
    return DARTRAY_OK;
}

// The caller's [rows][nlu] into columns [col0, col0 + nlu) of [rows][nl]
// (the other columns untouched).
int copy_in_cols_at(float *dst, const float *src, size_t rows, int nlu, int nl, int col0, bool on_device,
                    cudaStream_t s) {
    if (rows == 0) return DARTRAY_OK;
    if (!src) return fail(DARTRAY_E_INVAL, "missing input array");
    CK(cudaMemcpy2DAsync(dst + col0, nl * sizeof(float), src, nlu * sizeof(float), nlu * sizeof(float), rows,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    return DARTRAY_OK;
}

// Columns [col0, col0 + nlu) of the library's [rows][nl] to the caller's [rows][nlu].
int copy_out_cols_at(float *dst, const float *src, size_t rows, int nlu, int nl, int col0, bool dst_is_device,
                     cudaStream_t s) {
    if (rows == 0) return DARTRAY_OK;
    CK(cudaMemcpy2DAsync(dst, nlu * sizeof(float), src + col0, nl * sizeof(float), nlu * sizeof(float), rows,
                         dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    return DARTRAY_OK;
}

// the marcher width for n wavelengths
int padded_lambda(int n) { return n <= 1 ? 1 : (n <= 2 ? 2 : (n <= 4 ? 4 : (n <= 8 ? 8 : 16))); }

template <class T>
int fetch_host(std::vector<T> &dst, const T *src, size_t count, bool on_device) {
    dst.resize(count);
    if (count == 0) return DARTRAY_OK;
    if (!src) return fail(DARTRAY_E_INVAL, "missing input array");
    if (on_device) {
        CK(cudaMemcpy(dst.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(dst.data(), src, count * sizeof(T));
    }
    return DARTRAY_OK;
}

int occupancy_blocks(const void *kernel, int num_sms, int block = kBlock, int smem = 0) {
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
    return std::max(1, per_sm) * num_sms;
}

template <int NL, bool DET>
void launch_march_det(dartray_grid *g, cudaStream_t st, int mode, const MarchArgs &A) {
    const int blocks = g->march_blocks, sm = g->march_smem;
    if (mode == MODE_LL) march_kernel<NL, MODE_LL, DET><<<blocks, kMarchBlock, sm, st>>>(g->G, A);
    else if (mode == MODE_DIRECT) march_kernel<NL, MODE_DIRECT, DET><<<blocks, kMarchBlock, sm, st>>>(g->G, A);
    else march_kernel<NL, MODE_SCATTER, DET><<<blocks, kMarchBlock, sm, st>>>(g->G, A);
}

template <int NL>
int launch_march_nl(dartray_grid *g, cudaStream_t st, int mode, const MarchArgs &A) {
    if (A.det) launch_march_det<NL, true>(g, st, mode, A);
    else launch_march_det<NL, false>(g, st, mode, A);
    ++g->launches;
    CK(cudaGetLastError());
    return DARTRAY_OK;
}

int launch_march(dartray_grid *g, cudaStream_t st, int mode, const MarchArgs &A) {
    switch (g->nl) {
    case 1: return launch_march_nl<1>(g, st, mode, A);
    case 2: return launch_march_nl<2>(g, st, mode, A);
    default:
        if (!launch_march_wide(g->nl, mode, A.det != 0, g->march_blocks, kMarchBlock, g->march_smem, st, g->G, A))
            return fail(DARTRAY_E_INVAL, "n_lambda must be 1, 2, 4, 8 or 16");
        ++g->launches;
        CK(cudaGetLastError());
        return DARTRAY_OK;
    }
}

// Compacted source table of a phase; returns the number of sources traced
// in *n_src and the number of sources of the model, N_s of Eq. 10, in *n_s
// (they differ in the octant mode, which traces the first octant only).
int build_sources(dartray_grid *g, int mode, const float *pend_src, int *n_src, int *n_s) {
    const int n_all = mode == MODE_SCATTER ? g->n_leaf : g->n_leaf + g->n_point;
    const int nb = (n_all + kBlock - 1) / kBlock;
    int total = 0;
    for (int pass = g->G.octant ? 0 : 1; pass < 2; ++pass) {
        // pass 0 (octant mode): every source, for N_s; pass 1: those traced
        source_flags_kernel<<<nb, kBlock, 0, g->stream>>>(
            g->G, mode, pend_src, g->P.src_stride, g->P.src_offset, pass == 1 ? g->G.octant : 0,
            mode == MODE_SCATTER && g->n_models > 1 ? g->d_model_active : nullptr, g->d_flags);
        scan_blocks_kernel<<<nb, kBlock, 0, g->stream>>>(nullptr, g->d_flags, n_all, g->d_blocksum);
        scan_offsets_kernel<<<1, 1, 0, g->stream>>>(nullptr, g->d_blocksum, nb, g->d_total);
        scatter_compact_kernel<<<nb, kBlock, 0, g->stream>>>(g->d_flags, n_all, g->d_blocksum, g->d_src_idx);
        g->launches += 4;
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&total, g->d_total, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
        if (pass == 0 || !g->G.octant) *n_s = total;
    }
    if (total > 0) {
        source_table_kernel<<<(total + kBlock - 1) / kBlock, kBlock, 0, g->stream>>>(
            g->G, mode, g->d_src_idx, total, g->d_src_leaf, g->d_src_hint, g->d_src_pos, g->d_src_S);
        ++g->launches;
        CK(cudaGetLastError());
    }
    *n_src = total;
    return DARTRAY_OK;
}

// Enqueue on pipeline P's stream the expansion of its buffered crossing
// records into the pending j_sca rows (bucket by cell, then per-cell-range
// accumulation).  On the device the kernels run only when the buffer is at
// least half full, or always when force is set.
int enqueue_flush_kernels(dartray_grid *g, Pipe &P, float *pend_dst, int force) {
    if (g->rec_cap == 0) return DARTRAY_OK;
    cudaStream_t s = P.stream;
    const int nb = (g->n_leaf + kBlock - 1) / kBlock;
    const unsigned gb = static_cast<unsigned>(8 * g->num_sms);
    flush_decide_kernel<<<1, 1, 0, s>>>(P.d_pd, P.d_rec_n, g->rec_cap, force, P.d_st);
    scan_blocks_kernel<<<nb, kBlock, 0, s>>>(P.d_pd, reinterpret_cast<const int *>(P.d_cnt), g->n_leaf, P.d_blocksum);
    scan_offsets_kernel<<<1, 1, 0, s>>>(P.d_pd, P.d_blocksum, nb, P.d_total);
    scan_apply_kernel<<<nb, kBlock, 0, s>>>(P.d_pd, P.d_cnt, g->n_leaf, P.d_blocksum, P.d_off, P.d_cur);
    if (g->dg_on && g->dg_phase_live) {
        dg_tally_kernel<<<gb, kBlock, 0, s>>>(g->G, P.d_pd, P.d_rec_n, P.d_rec_cell, P.d_rec_dir, P.d_rec_coef,
                                              g->rec_cap, g->d_dg_dir, g->d_dg_phase);
        ++g->launches;
    }
    rec_scatter_kernel<<<gb, kBlock, 0, s>>>(P.d_pd, P.d_rec_n, P.d_rec_cell, P.d_rec_dir, P.d_rec_coef, g->rec_cap,
                                             g->nl, P.d_cur, P.d_srt_dir, P.d_srt_coef);
    FlushArgs F{};
    F.pd = P.d_pd;
    F.n_sorted = P.d_total;
    F.off = P.d_off;
    F.n_leaf = g->n_leaf;
    F.sdir = P.d_srt_dir;
    F.scoef = P.d_srt_coef;
    F.cap = g->rec_cap;
    F.packed = g->nl == 1;
    F.pend = pend_dst;
    F.det = g->P.deterministic;
    F.pend_fix = g->d_pfix;
    for (int l = 0; l < kMaxLambda; ++l) F.eJ[l] = g->eJ.e[l];
    const bool det = g->P.deterministic != 0;
    for (int l = 0; l < g->nl; ++l) {
        const int slot = g->k_lam[l] == 0 ? 0 : (g->k_lam[l] == 1 ? 1 : (g->k_lam[l] == 2 ? 2 : 3));
        const unsigned blocks = static_cast<unsigned>(g->acc_blocks[det ? 4 + slot : slot]);
#define ACC(PPL)                                                                              \
    do {                                                                                      \
        if (det) cell_accumulate_kernel<PPL, true><<<blocks, kBlock, 0, s>>>(g->G, l, F);     \
        else cell_accumulate_kernel<PPL, false><<<blocks, kBlock, 0, s>>>(g->G, l, F);        \
    } while (0)
        switch (slot) {
        case 0: ACC(1); break;
        case 1: ACC(2); break;
        case 2: ACC(6); break;
        default: ACC(24); break;
        }
#undef ACC
    }
    flush_reset_kernel<<<nb, kBlock, 0, s>>>(P.d_pd, P.d_rec_n, P.d_cnt, g->n_leaf, P.d_total, P.d_st);
    g->launches += 6 + g->nl;
    CK(cudaGetLastError());
    return DARTRAY_OK;
}

struct SpanTiming {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[kPipes];
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<float, float>> spans;  // [start, end] ms after the phase origin
    cudaEvent_t origin = nullptr;

    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    // collect the spans of pipeline i (its stream is synchronised)
    void collect(int i) {
        for (auto &pr : pending[i]) {
            float a = 0.f, b = 0.f;
            cudaEventElapsedTime(&a, origin, pr.first);
            cudaEventElapsedTime(&b, origin, pr.second);
            spans.emplace_back(a, b);
            pool.push_back(pr.first);
            pool.push_back(pr.second);
        }
        pending[i].clear();
    }
    // summed lengths of the spans
    double sum_ms() const {
        double tot = 0.0;
        for (auto &sp : spans) tot += sp.second - sp.first;
        return tot;
    }
    // length of the union of all spans
    double busy_ms() {
        std::sort(spans.begin(), spans.end());
        double tot = 0.0, cs = -1e30, ce = -1e30;
        for (auto &sp : spans) {
            if (sp.first > ce) {
                if (ce > cs) tot += ce - cs;
                cs = sp.first;
                ce = sp.second;
            } else {
                ce = std::max<double>(ce, sp.second);
            }
        }
        if (ce > cs) tot += ce - cs;
        return tot;
    }
    ~SpanTiming() {
        for (auto &v : pending)
            for (auto &pr : v) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// Device-event spans of one phase (params.profile): march kernels, deposit
// flushes and whole waves; each is reported as the length of its union.
struct PhaseTiming {
    SpanTiming march, flush, wave;
    cudaEvent_t origin = nullptr;
    ~PhaseTiming() {
        if (origin) cudaEventDestroy(origin);
    }
    void start(cudaStream_t s) {
        cudaEventCreate(&origin);
        cudaEventRecord(origin, s);
        cudaEventSynchronize(origin);
        march.origin = flush.origin = wave.origin = origin;
    }
    void collect(int i) {
        march.collect(i);
        flush.collect(i);
        wave.collect(i);
    }
};

// records a device-event span around the work enqueued by f on stream s
template <class F>
int timed(SpanTiming *t, int pi, cudaStream_t s, F &&f) {
    if (!t) return f();
    cudaEvent_t e0 = t->get(), e1 = t->get();
    CK(cudaEventRecord(e0, s));
    const int rc = f();
    if (rc) return rc;
    CK(cudaEventRecord(e1, s));
    t->pending[pi].emplace_back(e0, e1);
    return DARTRAY_OK;
}

int enqueue_flush(dartray_grid *g, Pipe &P, float *pend_dst, int force, PhaseTiming *pt, int pi) {
    if (g->rec_cap == 0) return DARTRAY_OK;
    return timed(pt ? &pt->flush : nullptr, pi, P.stream,
                 [&] { return enqueue_flush_kernels(g, P, pend_dst, force); });
}

// Enqueue one wave of pipeline P: march, merge the low list, flush records
// when the buffer is half full, advance to the next wave.
int enqueue_wave_kernels(dartray_grid *g, Pipe &P, int pi, int mode, const MarchArgs &base, float *pend_dst,
                         PhaseTiming *pt) {
    cudaStream_t s = P.stream;
    MarchArgs A = base;
    A.pd = P.d_pd;
    for (int i = 0; i < 2; ++i) {
        A.Hb[i] = P.d_H[i];
        A.HIb[i] = P.d_HI[i];
        A.Mb[i] = P.d_M[i];
        A.MIb[i] = P.d_MI[i];
    }
    A.L_out = P.d_L;
    A.L_out_I = P.d_LI;
    A.rec_cell = P.d_rec_cell;
    A.rec_dir = P.d_rec_dir;
    A.rec_coef = P.d_rec_coef;
    A.rec_n = P.d_rec_n;
    A.rec_cnt = P.d_cnt;
    int rc = timed(pt ? &pt->march : nullptr, pi, s, [&] { return launch_march(g, s, mode, A); });
    if (rc) return rc;
    ++g->march_launches;
    MergeArgs M{};
    M.pd = P.d_pd;
    M.L = P.d_L;
    M.L_I = P.d_LI;
    M.cap = g->cap;
    M.hkey = P.d_hkey;
    M.hcnt = P.d_hcnt;
    M.hmem = P.d_hmem;
    M.hcap = g->hcap;
    for (int i = 0; i < 2; ++i) {
        M.Mb[i] = P.d_M[i];
        M.MIb[i] = P.d_MI[i];
    }
    M.st = g->d_st;
    M.nl = g->nl;
    const unsigned mg = static_cast<unsigned>(2 * g->num_sms);
    merge_size_kernel<<<1, 1, 0, s>>>(P.d_pd, g->hcap);
    merge_clear_kernel<<<mg, kBlock, 0, s>>>(M);
    merge_insert_kernel<<<mg, kBlock, 0, s>>>(M);
    merge_emit_kernel<<<mg, kBlock, 0, s>>>(M);
    g->launches += 4;
    if (mode != MODE_LL) {
        rc = enqueue_flush(g, P, pend_dst, 0, pt, pi);
        if (rc) return rc;
    }
    wave_advance_kernel<<<1, 1, 0, s>>>(P.d_pd);
    ++g->launches;
    CK(cudaGetLastError());
    return DARTRAY_OK;
}

int enqueue_wave(dartray_grid *g, Pipe &P, int pi, int mode, const MarchArgs &base, float *pend_dst,
                 PhaseTiming *pt) {
    return timed(pt ? &pt->wave : nullptr, pi, P.stream,
                 [&] { return enqueue_wave_kernels(g, P, pi, mode, base, pend_dst, pt); });
}

int start_batch(dartray_grid *g, Pipe &P, int src_lo, int nb, int kstart) {
    PipeDev &h = *P.h_pd;
    std::memset(&h, 0, sizeof h);
    h.nA = static_cast<long long>(nb) * (12ll << (2 * kstart));
    h.nB = 0;
    h.kind = 0;
    h.par = 0;
    h.src_lo = src_lo;
    h.nb_src = nb;
    h.kstart = kstart;
    h.done = 0;
    h.peak = h.nA;
    h.waves = 1;
    h.max_waves = g->P.max_waves;
    CK(cudaMemcpyAsync(P.d_pd, P.h_pd, sizeof(PipeDev), cudaMemcpyHostToDevice, P.stream));
    P.active = true;
    P.src_lo = src_lo;
    P.nb = nb;
    return DARTRAY_OK;
}

struct PhaseResult {
    double ledger[LG_N][kMaxLambda];
    unsigned long long cnt[CT_N];
    double f_u;
    double pend_sum;
    long long batches;
};

int status_error(const PipeDev &h, int mode) {
    const WaveCounters &wc = h.wc;
    if (wc.status & ST_CROSS_CAP) {
        char m[256];
        std::snprintf(m, sizeof m,
                      "crossing cap per ray reached (mode %d, source %d, level %d, pixel %llu, kind %d, "
                      "leaf %d, d %.9g, side %.9g)",
                      mode, wc.dbg_src, wc.dbg_lev, static_cast<unsigned long long>(wc.dbg_pix), wc.dbg_kind,
                      wc.dbg_leaf, static_cast<double>(wc.dbg_d), static_cast<double>(wc.dbg_te));
        return fail(DARTRAY_E_LIMIT, m);
    }
    if (wc.status & ST_NOPROGRESS) return fail(DARTRAY_E_LIMIT, "ray made no progress across a face");
    if (wc.status & ST_WAVE_CAP) return fail(DARTRAY_E_LIMIT, "wave cap reached");
    if (wc.status & ST_MERGE) return fail(DARTRAY_E_QUEUE, "merge table overflow");
    return DARTRAY_OK;
}

// Deterministic sum of n floats x[0], x[stride], ... (fixed grid, partials
// added in order on the host).
int det_sum(dartray_grid *g, const float *x, long long n, long long stride, double *out) {
    *out = 0.0;
    if (n <= 0) return DARTRAY_OK;
    det_sum_kernel<<<kSumBlocks, kBlock, 0, g->stream>>>(x, n, stride, g->d_partial);
    ++g->launches;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(g->h_partial, g->d_partial, kSumBlocks * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    double t = 0.0;
    for (int b = 0; b < kSumBlocks; ++b) t += g->h_partial[b];
    *out = t;
    return DARTRAY_OK;
}

// 60 - ceil(log2(bound)): the exponent that maps a positive bound to at most
// 2^60 in the fixed point of the deterministic mode (0 for no bound).
int fix_exponent(double bound) {
    if (!(bound > 0.0) || !std::isfinite(bound)) return 0;
    int x = 0;
    const double f = std::frexp(bound, &x);
    return 60 - (f == 0.5 ? x - 1 : x);
}

// One phase (mode: step 1, step 2, one scattering iteration).
int run_phase(dartray_grid *g, int mode, PhaseResult *res, bool keep_U = false) {
    cudaStream_t s = g->stream;
    const size_t nU = static_cast<size_t>(g->n_leaf) * g->nl;
    if (mode == MODE_SCATTER) g->cur = 1 - g->cur;
    float *pend_src = g->d_pend[g->cur];
    float *pend_dst = g->d_pend[1 - g->cur];
    int n_src = 0, n_s = 0;
    int rc = build_sources(g, mode, pend_src, &n_src, &n_s);
    if (rc) return rc;
    const double f_u = n_s > 0 ? 4.0 * g->P.a_rt / n_s : 0.0;  // Eq. 10
    // f_U per model (batched grids: N_s counts the sources of each model)
    if (g->n_models > 1) {
        const int n_all = mode == MODE_SCATTER ? g->n_leaf : g->n_leaf + g->n_point;
        std::vector<int> cnt(g->n_models, 0);
        CK(cudaMemsetAsync(g->d_mcount, 0, g->n_models * sizeof(int), s));
        model_count_kernel<<<(n_all + kBlock - 1) / kBlock, kBlock, 0, s>>>(g->G, g->d_flags, n_all, g->d_mcount);
        ++g->launches;
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(cnt.data(), g->d_mcount, g->n_models * sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int m = 0; m < g->n_models; ++m) g->m_fu[m] = cnt[m] > 0 ? 4.0 * g->P.a_rt / cnt[m] : 0.0;
    } else {
        g->m_fu[0] = f_u;
    }
    {
        std::vector<float> fu(g->n_models);
        for (int m = 0; m < g->n_models; ++m) fu[m] = static_cast<float>(g->m_fu[m]);
        CK(cudaMemcpyAsync(g->d_fu_model, fu.data(), fu.size() * sizeof(float), cudaMemcpyHostToDevice, s));
        if (mode != MODE_LL) {
            threshold_kernel<<<static_cast<unsigned>((nU + kBlock - 1) / kBlock), kBlock, 0, s>>>(g->G, g->d_ULL,
                                                                                               g->d_fu_model, g->d_thr);
            ++g->launches;
            CK(cudaGetLastError());
        }
        CK(cudaStreamSynchronize(s));  // fu lives on this stack frame
    }
    int kstart = g->P.k0;
    if (mode == MODE_SCATTER)
        for (int l = 0; l < g->nl; ++l) kstart = std::max(kstart, g->k_lam[l]);

    MarchArgs base{};
    base.src_leaf = g->d_src_leaf;
    base.src_hint = g->d_src_hint;
    base.src_pos = g->d_src_pos;
    base.src_S = g->d_src_S;
    base.cap = g->cap;
    // octant mode (float sums): the traced sources deposit into scratch
    // arrays, folded over the eight images of each cell at the end
    const bool fold = g->G.octant && !g->P.deterministic;
    base.target = fold ? g->d_oct_u : (mode == MODE_LL ? g->d_ULL : g->d_U);
    float *dep_pend = fold ? g->d_oct_p : pend_dst;
    base.U_LL = g->d_ULL;
    base.thr = g->d_thr;
    base.mled = g->d_mled;
    base.mled_fix = g->d_mled_fix;
    base.pend_src = pend_src;
    base.pend_dst = dep_pend;
    base.f_u = static_cast<float>(f_u);
    base.r_pre = static_cast<float>(g->P.r_pre);
    base.c_light = static_cast<float>(g->P.c_light);
    base.split_c = 4.0 * kPi * static_cast<double>(g->P.n_rays_min);
    base.merge_c = 4.0 * kPi * static_cast<double>(g->P.n_rays_max);
    base.split_cf = static_cast<float>(base.split_c);
    base.merge_cf = static_cast<float>(base.merge_c);
    base.k_ray_max = g->P.k_ray_max;
    base.merge = g->P.merge;
    base.max_cross = g->P.max_cross;
    base.st = g->d_st;
    base.rec_cap = g->rec_cap;
    g->dg_phase_live = g->dg_on && mode != MODE_LL;
    base.dg = g->dg_phase_live ? g->d_dg_phase : nullptr;
    base.dg_dir = g->d_dg_dir;
    const bool det = g->P.deterministic != 0;
    if (det) {
        // Fixed-point exponents from the luminosity L_emit the phase emits
        // per wavelength: no cell receives more RFED than
        // 2 sqrt(3) L_emit / (L^2 c) (each ray's power crosses a cell once,
        // over at most sqrt(3) L; a merged ray may start a little before its
        // siblings stopped, hence the 2), and no j_sca pixel or ledger entry
        // more than 2 L_emit; a further factor 2 of margin.
        for (int l = 0; l < g->nl; ++l) {
            double le = 0.0;
            if (mode == MODE_SCATTER) {
                const long long np = 12ll << (2 * g->k_lam[l]);
                if ((rc = det_sum(g, pend_src + g->off_lam[l], static_cast<long long>(g->n_leaf) * np, 1, &le))) return rc;
            } else {
                if ((rc = det_sum(g, g->d_src_S + l, n_src, g->nl, &le))) return rc;
                le *= 4.0 * kPi;
            }
            g->eU.e[l] = fix_exponent(4.0 * std::sqrt(3.0) * le / g->P.c_light);
            g->eJ.e[l] = fix_exponent(4.0 * le);
            g->eL.e[l] = fix_exponent(4.0 * le);
        }
        base.det = 1;
        base.U_fix = g->d_Ufix;
        base.pend_fix = g->d_pfix;
        for (int l = 0; l < kMaxLambda; ++l) {
            base.eU[l] = g->eU.e[l];
            base.eJ[l] = g->eJ.e[l];
            base.eL[l] = g->eL.e[l];
        }
    }

    // Sources are traced in batches (the phase is additive over sources and
    // U_LL is fixed during a phase, so batching does not change the result),
    // kPipes batches at a time on as many streams so that one batch's last waves
    // overlap the others'.  A batch is sized so that its largest wave fills
    // 80% of a queue, from an estimate of the peak rays per source.  The
    // estimate starts high (small first batches), halves after each batch but
    // never drops below the heaviest batch seen, in this call or an earlier
    // one of the same step; an overflow restarts the phase with smaller
    // batches, so it is worth avoiding.
    const long long npix0 = 12ll << (2 * kstart);
    long long batch_cap = g->P.src_batch > 0 ? g->P.src_batch : n_src;
    const double rps_floor = g->rays_per_src[mode];
    double rays_per_src = rps_floor > 0.0 ? rps_floor
                                          : std::max(static_cast<double>(npix0) * 16.0, g->cap / 64.0);
#ifndef DARTRAY_WAVES_AHEAD
#define DARTRAY_WAVES_AHEAD 6  // waves a pipeline runs per host round trip
#endif
    constexpr int kWavesAhead = DARTRAY_WAVES_AHEAD;
    // CUDA graphs of the pipelines' rounds of waves (not in the profile
    // mode, which times every launch with events)
    struct Graphs {
        bool on = false;
        cudaGraphExec_t exec[kPipes] = {};
        long long launches = 0;
        ~Graphs() {
            for (auto e : exec)
                if (e) cudaGraphExecDestroy(e);
        }
    } graphs;
    graphs.on = g->P.graphs != 0 && !g->P.profile;
    DevStats snap{};
    CK(cudaMemcpyAsync(&snap, g->d_st, sizeof(DevStats), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (;;) {
        // (re)start the phase: zero what it writes
        if (mode == MODE_LL) {
            CK(cudaMemsetAsync(g->d_ULL, 0, nU * sizeof(float), s));
        } else {
            if (mode == MODE_DIRECT && !keep_U) {
                CK(cudaMemsetAsync(g->d_U, 0, nU * sizeof(float), s));
            } else {
                // U equals U_LL at the start of an iteration (U_LL <- U after each phase)
                CK(cudaMemcpyAsync(g->d_U, g->d_ULL, nU * sizeof(float), cudaMemcpyDeviceToDevice, s));
            }
            CK(cudaMemsetAsync(pend_dst, 0, g->sca_len * sizeof(float), s));
            if (g->dg_phase_live) CK(cudaMemsetAsync(g->d_dg_phase, 0, nU * sizeof(float), s));
        }
        if (det) {
            CK(cudaMemsetAsync(g->d_Ufix, 0, nU * sizeof(unsigned long long), s));
            if (mode != MODE_LL) CK(cudaMemsetAsync(g->d_pfix, 0, g->sca_len * sizeof(unsigned long long), s));
        }
        if (g->n_models > 1) {
            const size_t nm = static_cast<size_t>(g->n_models) * LG_N * g->nl;
            CK(cudaMemsetAsync(g->d_mled, 0, nm * sizeof(double), s));
            CK(cudaMemsetAsync(g->d_mled_fix, 0, nm * sizeof(unsigned long long), s));
        }
        if (fold) {
            CK(cudaMemsetAsync(g->d_oct_u, 0, nU * sizeof(float), s));
            if (mode != MODE_LL) CK(cudaMemsetAsync(g->d_oct_p, 0, g->sca_len * sizeof(float), s));
        }
        for (int i = 0; i < kPipes; ++i) {
            Pipe &P = g->pipe[i];
            P.active = false;
            CK(cudaMemsetAsync(P.d_st, 0, sizeof(DevStats), s));
            if (g->rec_cap > 0) {
                CK(cudaMemsetAsync(P.d_rec_n, 0, sizeof(unsigned long long), s));
                CK(cudaMemsetAsync(P.d_cnt, 0, static_cast<size_t>(g->n_leaf) * sizeof(unsigned), s));
            }
        }
        DevStats fresh = snap;
        std::memset(fresh.ledger, 0, sizeof fresh.ledger);
        std::memset(fresh.ledger_fix, 0, sizeof fresh.ledger_fix);
        CK(cudaMemcpyAsync(g->d_st, &fresh, sizeof(DevStats), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));  // the pipelines start after the setup
        std::unique_ptr<PhaseTiming> tm;
        if (g->P.profile) {
            tm.reset(new PhaseTiming());
            tm->start(s);
        }
        long long waves = 0;
        double max_rps = 0.0;  // largest peak wave per source of a batch
        bool overflow = false;
        long long failed_nb = 0;
        long long next = 0;
        long long batches = 0;
        // Each pipeline runs kWavesAhead waves per host round trip.  The host
        // refills whichever pipeline finishes its waves first, so neither
        // waits for the other.
        bool inflight[kPipes] = {};
        for (;;) {
            bool any = false;
            for (int i = 0; i < kPipes; ++i) {
                Pipe &P = g->pipe[i];
                if (inflight[i]) {
                    any = true;
                    continue;
                }
                if (!P.active && next < n_src) {
                    long long want = static_cast<long long>(0.8 * static_cast<double>(g->cap) / rays_per_src);
                    want = std::max<long long>(1, std::min(want, batch_cap));
                    const int nb = static_cast<int>(std::min<long long>(want, n_src - next));
                    if ((rc = start_batch(g, P, static_cast<int>(next), nb, kstart))) return rc;
                    next += nb;
                    ++batches;
                }
                if (P.active) {
                    any = true;
                    if (graphs.on) {
                        // the pipeline's kWavesAhead waves as one CUDA graph,
                        // captured at its first use in the phase: every
                        // kernel reads its work from the pipeline state in
                        // device memory, so one graph serves every round
                        if (!graphs.exec[i]) {
                            const long long l0 = g->launches, m0 = g->march_launches;
                            CK(cudaStreamBeginCapture(P.stream, cudaStreamCaptureModeThreadLocal));
                            for (int w = 0; w < kWavesAhead && !rc; ++w)
                                rc = enqueue_wave(g, P, i, mode, base, dep_pend, nullptr);
                            cudaGraph_t gr = nullptr;
                            const cudaError_t ce = cudaStreamEndCapture(P.stream, &gr);
                            if (rc) {
                                if (gr) cudaGraphDestroy(gr);
                                return rc;
                            }
                            if (ce != cudaSuccess) return fail(DARTRAY_E_CUDA, cudaGetErrorString(ce));
                            const cudaError_t ie = cudaGraphInstantiate(&graphs.exec[i], gr, 0);
                            cudaGraphDestroy(gr);
                            if (ie != cudaSuccess) return fail(DARTRAY_E_CUDA, cudaGetErrorString(ie));
                            graphs.launches = g->launches - l0;
                            g->launches = l0;
                            g->march_launches = m0;
                        }
                        CK(cudaGraphLaunch(graphs.exec[i], P.stream));
                        g->launches += graphs.launches;
                        g->march_launches += kWavesAhead;
                    } else {
                        for (int w = 0; w < kWavesAhead; ++w)
                            if ((rc = enqueue_wave(g, P, i, mode, base, dep_pend, tm.get()))) return rc;
                    }
                    CK(cudaMemcpyAsync(P.h_pd, P.d_pd, sizeof(PipeDev), cudaMemcpyDeviceToHost, P.stream));
                    CK(cudaEventRecord(P.ev, P.stream));
                    inflight[i] = true;
                }
            }
            if (!any) break;
            // the first pipeline whose waves have completed
            // (a round of waves takes milliseconds: after a short spin the
            // host sleeps between polls instead of holding a core)
            int i = -1;
            for (int spin = 0; i < 0; ++spin) {
                for (int j = 0; j < kPipes && i < 0; ++j) {
                    if (!inflight[j]) continue;
                    const cudaError_t q = cudaEventQuery(g->pipe[j].ev);
                    if (q == cudaSuccess) i = j;
                    else if (q != cudaErrorNotReady) return fail(DARTRAY_E_CUDA, cudaGetErrorString(q));
                }
                if (i >= 0) break;
                if (spin < 64) std::this_thread::yield();
                else std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
            Pipe &P = g->pipe[i];
            inflight[i] = false;
            if (tm) tm->collect(i);
            const PipeDev &h = *P.h_pd;
            if (h.wc.status & ST_QUEUE) {
                overflow = true;
                failed_nb = std::max<long long>(failed_nb, P.nb);
            } else if ((rc = status_error(h, mode))) {
                return rc;
            }
            if (h.done) {
                P.active = false;
                waves += h.waves;
                const double r = static_cast<double>(h.peak) / P.nb;
                max_rps = std::max(max_rps, r);
                // never below the heaviest batch so far: an overflow restarts
                // the whole phase
                rays_per_src = std::max({rays_per_src * 0.5, max_rps, rps_floor});
            }
            if (overflow) break;
        }
        for (int i = 0; i < kPipes; ++i) CK(cudaStreamSynchronize(g->pipe[i].stream));
        if (!overflow) {
            // last records of every pipeline
            for (int i = 0; i < kPipes && mode != MODE_LL; ++i) {
                if ((rc = enqueue_flush(g, g->pipe[i], dep_pend, 1, tm.get(), i))) return rc;
                CK(cudaStreamSynchronize(g->pipe[i].stream));
                if (tm) tm->collect(i);
            }
            if (tm) {
                g->march_ms += tm->march.busy_ms();
                g->march_sum_ms += tm->march.sum_ms();
                g->flush_ms += tm->flush.busy_ms();
                // the final flushes count as busy time too
                for (auto &sp : tm->flush.spans) tm->wave.spans.push_back(sp);
                g->busy_ms += tm->wave.busy_ms();
            }
            DevStats out{};
            CK(cudaMemcpyAsync(&out, g->d_st, sizeof(DevStats), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            out.cnt[CT_WAVES] += static_cast<unsigned long long>(waves);
            out.cnt[CT_SOURCES] += static_cast<unsigned long long>(n_src);
            for (int i = 0; i < kPipes; ++i) {
                DevStats ps{};
                CK(cudaMemcpyAsync(&ps, g->pipe[i].d_st, sizeof(DevStats), cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                out.cnt[CT_FLUSH] += ps.cnt[CT_FLUSH];
                out.cnt[CT_REC] += ps.cnt[CT_REC];
            }
            CK(cudaMemcpyAsync(g->d_st, &out, sizeof(DevStats), cudaMemcpyHostToDevice, s));
            std::memcpy(res->ledger, out.ledger, sizeof res->ledger);
            if (det)
                for (int sl = 0; sl < LG_N; ++sl)
                    for (int l = 0; l < g->nl; ++l)
                        res->ledger[sl][l] = std::ldexp(static_cast<double>(out.ledger_fix[sl][l]), -g->eL.e[l]);
            if (g->G.octant)  // the traced sources stand for their images in all eight octants
                for (int sl = 0; sl < LG_N; ++sl)
                    for (int l = 0; l < g->nl; ++l) res->ledger[sl][l] *= 8.0;
            if (g->n_models > 1) {
                // per-model ledgers; the grid's ledger is their sum
                const size_t nm = static_cast<size_t>(g->n_models) * LG_N * g->nl;
                std::vector<unsigned long long> raw(nm);
                if (det) CK(cudaMemcpyAsync(raw.data(), g->d_mled_fix, nm * 8, cudaMemcpyDeviceToHost, s));
                else CK(cudaMemcpyAsync(raw.data(), g->d_mled, nm * 8, cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                std::memset(res->ledger, 0, sizeof res->ledger);
                for (size_t i = 0; i < nm; ++i) {
                    const int l = static_cast<int>(i % g->nl), sl = static_cast<int>((i / g->nl) % LG_N);
                    double v;
                    if (det) v = std::ldexp(static_cast<double>(raw[i]), -g->eL.e[l]);
                    else std::memcpy(&v, &raw[i], sizeof v);
                    g->m_ledger[i] = v;
                    res->ledger[sl][l] += v;
                }
            } else {
                for (int sl = 0; sl < LG_N; ++sl)
                    for (int l = 0; l < g->nl; ++l) g->m_ledger[static_cast<size_t>(sl) * g->nl + l] = res->ledger[sl][l];
            }
            std::memcpy(res->cnt, out.cnt, sizeof res->cnt);
            g->rays_per_src[mode] = std::max(rps_floor, max_rps);
            g->batches += batches;
            break;
        }
        ++g->restarts;
        if (failed_nb <= 1) return fail(DARTRAY_E_QUEUE, "ray queues overflow with a single source");
        batch_cap = std::max<long long>(1, failed_nb / 4);
        rays_per_src = std::max(rays_per_src, 0.8 * static_cast<double>(g->cap) / batch_cap);
    }
    res->f_u = f_u;
    res->pend_sum = 0.0;
    if (det) {
        // fixed point -> float: U (step 2 from zero, an iteration on top of
        // U_LL), U_LL in step 1, the pending j_sca rows
        const unsigned ub = static_cast<unsigned>((nU + kBlock - 1) / kBlock);
        fix_to_u_kernel<<<ub, kBlock, 0, s>>>(g->G, g->d_Ufix, mode == MODE_SCATTER || keep_U ? g->d_ULL : nullptr, g->eU,
                                              mode == MODE_LL ? g->d_ULL : g->d_U);
        ++g->launches;
        if (mode != MODE_LL) {
            for (int l = 0; l < g->nl; ++l) {
                fix_to_jsca_kernel<<<8 * g->num_sms, kBlock, 0, s>>>(g->G, l, g->d_pfix, g->eJ, pend_dst);
                ++g->launches;
            }
        }
        CK(cudaGetLastError());
    }
    if (fold) {
        const unsigned ub = static_cast<unsigned>((nU + kBlock - 1) / kBlock);
        octant_fold_u_kernel<<<ub, kBlock, 0, s>>>(g->G, g->d_oct_u, mode == MODE_SCATTER || keep_U ? g->d_ULL : nullptr,
                                                   mode == MODE_LL ? g->d_ULL : g->d_U);
        ++g->launches;
        if (mode != MODE_LL) {
            for (int l = 0; l < g->nl; ++l) {
                octant_fold_jsca_kernel<<<8 * g->num_sms, kBlock, 0, s>>>(g->G, l, g->d_oct_p, pend_dst);
                ++g->launches;
            }
        }
        CK(cudaGetLastError());
    }
    if (mode != MODE_LL) {
        add_pending_kernel<<<8 * g->num_sms, kBlock, 0, s>>>(pend_dst, g->d_jtot, g->sca_len);
        ++g->launches;
        if (g->dg_phase_live) {
            add_pending_kernel<<<8 * g->num_sms, kBlock, 0, s>>>(g->d_dg_phase, g->d_dg, static_cast<long long>(nU));
            ++g->launches;
        }
        g->dg_phase_live = false;
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(g->d_ULL, g->d_U, nU * sizeof(float), cudaMemcpyDeviceToDevice, s));
        // remaining scattered luminosity per model (sum over its wavelength
        // blocks), in a fixed order
        const int nseg = g->n_models * g->nl;
        std::vector<double> seg(nseg);
        const int parts = std::max(1, std::min(kSegParts, kSegPartial / nseg));
        segment_partial_kernel<<<dim3(nseg, parts), kBlock, 0, s>>>(pend_dst, g->d_seg_beg, g->d_seg_len, parts,
                                                                     g->d_seg_part);
        segment_finish_kernel<<<(nseg + kBlock - 1) / kBlock, kBlock, 0, s>>>(g->d_seg_part, nseg, parts,
                                                                              g->d_seg_out);
        g->launches += 2;
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(seg.data(), g->d_seg_out, nseg * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int m = 0; m < g->n_models; ++m) {
            double t = 0.0;
            for (int l = 0; l < g->nlu; ++l) t += seg[m * g->nl + l];  // derivatives and padding excluded
            res->pend_sum += t;
            if (mode == MODE_DIRECT) g->m_lsca2[m] = t;
            g->m_rem[m] = g->m_lsca2[m] > 0 ? t / g->m_lsca2[m] : 0.0;
        }
    }
    return DARTRAY_OK;
}

void fill_stats(const dartray_grid *g, const PhaseResult &r, dartray_stats *st) {
    if (!st) return;
    std::memset(st, 0, sizeof *st);
    st->rays = r.cnt[CT_RAYS];
    st->crossings = r.cnt[CT_CROSS];
    st->splits = r.cnt[CT_SPLIT];
    st->merges = r.cnt[CT_MERGE];
    st->blocks = r.cnt[CT_BLOCK];
    st->escapes = r.cnt[CT_ESCAPE];
    st->cuts = r.cnt[CT_CUT];
    st->lows = r.cnt[CT_LOW];
    st->resumes = r.cnt[CT_RESUME];
    st->waves = r.cnt[CT_WAVES];
    st->sources = r.cnt[CT_SOURCES];
    st->jsca_pixels = r.cnt[CT_JPIX];
    st->flushes = r.cnt[CT_FLUSH];
    st->records = r.cnt[CT_REC];
    for (int l = 0; l < g->nl; ++l) {
        const double w = g->G.albedo[l];
        st->emitted[l] = r.ledger[LG_EMITTED][l];
        st->absorbed[l] = (1.0 - w) * r.ledger[LG_DEPOSITED][l];
        st->scattered[l] = w * r.ledger[LG_DEPOSITED][l];
        st->escaped[l] = r.ledger[LG_ESCAPED][l];
        st->blocked[l] = r.ledger[LG_BLOCKED][l];
        st->cut[l] = r.ledger[LG_CUT][l];
        st->skipped[l] = r.ledger[LG_SKIPPED][l];
    }
    st->f_u = r.f_u;
    st->l_sca2 = g->l_sca2;
    st->kernel_launches = g->launches;
}

int set_device(dartray_grid *g) {
    CK(cudaSetDevice(g->device));
    return DARTRAY_OK;
}

// The grid's staging buffer with room for n floats.
int stage_buffer(dartray_grid *g, size_t n, float **out) {
    if (g->stage_floats < n) {
        if (g->d_stage) {
            CK(cudaStreamSynchronize(g->stream));
            CK(cudaFree(g->d_stage));
            g->d_stage = nullptr;
            g->stage_floats = 0;
        }
        CK(cudaMalloc(reinterpret_cast<void **>(&g->d_stage), n * sizeof(float)));
        g->stage_floats = n;
    }
    *out = g->d_stage;
    return DARTRAY_OK;
}

}  // namespace

extern "C" {

int dartray_params_default(dartray_params *p) {
    if (!p) return fail(DARTRAY_E_INVAL, "null params");
    std::memset(p, 0, sizeof *p);
    p->a_rt = 0.05;
    p->r_pre = -1.0;
    p->f_l = 0.01;
    p->c_light = 1.0;
    p->n_rays_min = 5;
    p->n_rays_max = 40;
    p->k0 = 2;
    p->k_ray_max = 13;
    p->k_sca_cap = 3;
    p->n_fwhm = 5;
    p->merge = 1;
    p->max_cross = 1 << 22;
    p->max_waves = 200;
    p->src_stride = 1;
    p->src_offset = 0;
    p->queue_rays = 0;
    p->src_batch = 0;
    p->profile = 0;
    p->deposit_direct = 0;
    p->deposit_records = 0;
    p->deterministic = 0;
    p->octant = 0;
    p->graphs = 1;
    p->tangent_albedo = 0;
    return DARTRAY_OK;
}

}  // extern "C"

namespace {

// Append the topology of one model to the forest of a grid: node, leaf and
// face-link indices shift by the nodes and leaves already there.
void append_topology(HostTopo *all, const HostTopo &t, int node_off, int leaf_off) {
    for (const int32_t c : t.node_child) all->node_child.push_back(c >= 0 ? c + node_off : c - leaf_off);
    all->node_box.insert(all->node_box.end(), t.node_box.begin(), t.node_box.end());
    all->leaf_box.insert(all->leaf_box.end(), t.leaf_box.begin(), t.leaf_box.end());
    for (const int32_t n : t.leaf_node) all->leaf_node.push_back(n + node_off);
    for (const int32_t code : t.leaf_rope) {
        // >= 0 a node; -1 the boundary; -(leaf + 2) a larger leaf;
        // kRopeSameSize - leaf a leaf of the same size
        all->leaf_rope.push_back(code >= 0 ? code + node_off : (code == kRopeBoundary ? code : code - leaf_off));
    }
    all->max_depth = std::max(all->max_depth, t.max_depth);
}

int create_grid(const dartray_grid_desc *descs, int n_models, const dartray_params *params, void *cuda_stream,
                dartray_grid **out) {
    g_last_error.clear();
    if (!descs || !out) return fail(DARTRAY_E_INVAL, "null argument");
    *out = nullptr;
    if (n_models < 1 || n_models > kMaxModels) return fail(DARTRAY_E_INVAL, "n_models must be in [1, 4096]");
    const dartray_grid_desc *desc = &descs[0];
    dartray_params P;
    if (params) P = *params;
    else dartray_params_default(&P);
    const int nlu = desc->n_lambda;
    if (nlu < 1 || nlu > 16) return fail(DARTRAY_E_INVAL, "n_lambda must be in [1, 16]");
    // forward mode: the derivatives with respect to the albedo ride in the
    // upper half of the padded wavelengths, [nl/2, nl/2 + nlu)
    const bool tangent = params && params->tangent_albedo == 1;
    if (tangent && nlu > 8) return fail(DARTRAY_E_INVAL, "the forward mode takes at most 8 wavelengths");
    const int nl = tangent ? 2 * padded_lambda(nlu) : padded_lambda(nlu);
    long long tot_leaf = 0, tot_nodes = 0, tot_point = 0;
    for (int m = 0; m < n_models; ++m) {
        const dartray_grid_desc &d = descs[m];
        if (d.n_leaf < 1 || d.n_nodes < 1 || d.n_point < 0) return fail(DARTRAY_E_INVAL, "bad sizes");
        if (d.n_lambda != nlu) return fail(DARTRAY_E_INVAL, "the models of a batch must share n_lambda");
        tot_leaf += d.n_leaf;
        tot_nodes += d.n_nodes;
        tot_point += d.n_point;
    }
    if (tot_leaf >= (1ll << 29) || tot_nodes >= (1ll << 30) || tot_point >= (1ll << 30))
        return fail(DARTRAY_E_INVAL, "too many cells or points in total");
    if (P.k0 < 0 || P.k0 > 13 || P.k_ray_max < P.k0 || P.k_ray_max > 13 || P.k_sca_cap < 0 || P.k_sca_cap > 3 ||
        P.n_fwhm < 1 || P.n_rays_min < 0 || P.n_rays_max < 0 || P.src_stride < 1 || P.src_offset < 0 ||
        P.src_offset >= P.src_stride || P.max_cross < 1 || P.max_waves < 1 ||
        (P.queue_rays != 0 && P.queue_rays < 1024) || P.deposit_records < 0 ||
        !(P.c_light > 0) || P.a_rt < 0 || P.deterministic < 0 || P.deterministic > 1 || P.octant < 0 ||
        P.octant > 1 || (P.octant && P.src_stride != 1) || P.graphs < 0 || P.graphs > 1 || P.tangent_albedo < 0 ||
        P.tangent_albedo > 1)
        return fail(DARTRAY_E_INVAL, "invalid parameters");
    if (P.octant && n_models > 1) return fail(DARTRAY_E_INVAL, "the octant mode takes a single model");
    if (tangent && (n_models > 1 || P.octant || P.deterministic))
        return fail(DARTRAY_E_INVAL, "the forward mode takes a single model, outside the octant and deterministic modes");
    if (n_models > 1 && static_cast<long long>(n_models) * LG_N * nl * 8 > 32768)
        return fail(DARTRAY_E_INVAL, "a batch holds at most 4096 / (6 n_lambda) models");
    const bool on_dev = desc->inputs_on_device != 0;
    std::vector<float> alb, gg;
    int rc = fetch_host(alb, desc->albedo, nlu, on_dev);
    if (rc) return rc;
    rc = fetch_host(gg, desc->g, nlu, on_dev);
    if (rc) return rc;
    for (int l = 0; l < nlu; ++l)
        if (!(alb[l] >= 0.f && alb[l] <= 1.f) || !(gg[l] > -1.f && gg[l] < 1.f))
            return fail(DARTRAY_E_INVAL, "albedo must be in [0,1] and g in (-1,1)");
    for (int m = 1; m < n_models; ++m) {
        std::vector<float> a2, g2;
        if ((rc = fetch_host(a2, descs[m].albedo, nlu, descs[m].inputs_on_device != 0)) ||
            (rc = fetch_host(g2, descs[m].g, nlu, descs[m].inputs_on_device != 0)))
            return rc;
        if (a2 != alb || g2 != gg) return fail(DARTRAY_E_INVAL, "the models of a batch must share albedo and g");
    }
    alb.resize(nl, 0.f);  // the extra wavelengths: no scattering, isotropic
    gg.resize(nl, 0.f);
    if (tangent)  // a derivative has its wavelength's albedo and g
        for (int l = 0; l < nlu; ++l) {
            alb[nl / 2 + l] = alb[l];
            gg[nl / 2 + l] = gg[l];
        }

    dartray_grid *g = new dartray_grid();
    g->P = P;
    g->stream = static_cast<cudaStream_t>(cuda_stream);
    g->nl = nl;
    g->nlu = nlu;
    g->n_leaf = static_cast<int>(tot_leaf);
    g->n_nodes = static_cast<int>(tot_nodes);
    g->n_point = static_cast<int>(tot_point);
    g->n_models = n_models;
    auto bail = [&](int code) {
        free_all(g);
        delete g;
        return code;
    };
    // topology of every model, validated and appended to one forest (node,
    // leaf and face-link indices shifted by the models before it)
    std::vector<int32_t> fc, lon;  // of the model built last (the only one in the octant mode)
    std::vector<ModelDev> models(n_models);
    std::string err;
    long long node_off = 0, leaf_off = 0, point_off = 0;
    for (int m = 0; m < n_models; ++m) {
        const dartray_grid_desc &d = descs[m];
        const bool dev_m = d.inputs_on_device != 0;
        if ((rc = fetch_host(fc, d.first_child, d.n_nodes, dev_m)) || (rc = fetch_host(lon, d.leaf_of_node, d.n_nodes, dev_m)))
            return bail(rc);
        HostTopo t;
        err = build_topology(d.nroot, d.root_lo, d.root_size, d.n_nodes, d.n_leaf, fc.data(), lon.data(), &t);
        if (!err.empty()) return bail(fail(DARTRAY_E_INVAL, n_models > 1 ? "model " + std::to_string(m) + ": " + err : err));
        append_topology(&g->topo, t, static_cast<int>(node_off), static_cast<int>(leaf_off));
        if (d.n_point > 0) {
            // point sources must lie inside their model's root lattice
            std::vector<float> pxyz;
            if ((rc = fetch_host(pxyz, d.point_xyz, 3ull * d.n_point, dev_m))) return bail(rc);
            for (int i = 0; i < d.n_point; ++i)
                for (int a = 0; a < 3; ++a) {
                    const double x = pxyz[3 * i + a];
                    if (!(x >= d.root_lo[a] && x < d.root_lo[a] + d.nroot[a] * d.root_size))
                        return bail(fail(DARTRAY_E_INVAL, "point source outside the model"));
                }
        }
        ModelDev &M = models[m];
        for (int a = 0; a < 3; ++a) {
            M.nroot[a] = d.nroot[a];
            M.root_lo[a] = static_cast<float>(d.root_lo[a]);
        }
        M.root_size = static_cast<float>(d.root_size);
        M.node0 = static_cast<int>(node_off);
        M.r_pre = static_cast<float>(P.r_pre >= 0 ? P.r_pre
                                                  : 0.15 * d.root_size * std::max({d.nroot[0], d.nroot[1], d.nroot[2]}));
        g->m_leaf0.push_back(leaf_off);
        g->m_nleaf.push_back(d.n_leaf);
        g->m_point0.push_back(point_off);
        node_off += d.n_nodes;
        leaf_off += d.n_leaf;
        point_off += d.n_point;
    }
    std::vector<int32_t> mirror;
    if (P.octant) {
        // the octant mode needs a model symmetric under the reflections about
        // the planes through its centre: topology, dust and emission alike
        err = build_mirrors(desc->nroot, desc->root_lo, desc->root_size, fc.data(), lon.data(), g->topo, &mirror);
        if (!err.empty()) return bail(fail(DARTRAY_E_INVAL, "octant mode: " + err));
        std::vector<float> kr, em, pxyz, plum;
        const size_t nU0 = static_cast<size_t>(desc->n_leaf) * nl;
        if ((rc = fetch_host(kr, desc->kappa_rho, nU0, on_dev)) || (rc = fetch_host(em, desc->emissivity, nU0, on_dev)) ||
            (rc = fetch_host(pxyz, desc->point_xyz, 3ull * desc->n_point, on_dev)) ||
            (rc = fetch_host(plum, desc->point_lum, static_cast<size_t>(desc->n_point) * nl, on_dev)))
            return bail(rc);
        for (int m = 1; m < 8; ++m)
            for (int64_t c = 0; c < desc->n_leaf; ++c) {
                const int64_t cm = mirror[static_cast<size_t>(m - 1) * desc->n_leaf + c];
                for (int l = 0; l < nl; ++l)
                    if (kr[c * nl + l] != kr[cm * nl + l] || em[c * nl + l] != em[cm * nl + l])
                        return bail(fail(DARTRAY_E_INVAL, "octant mode: kappa_rho or emissivity not mirror-symmetric"));
            }
        for (int m = 1; m < 8; ++m)
            for (int i = 0; i < desc->n_point; ++i) {
                float q[3];
                for (int a = 0; a < 3; ++a) {
                    const double c = desc->root_lo[a] + 0.5 * desc->nroot[a] * desc->root_size;
                    q[a] = ((m >> a) & 1) ? static_cast<float>(2.0 * c - pxyz[3 * i + a]) : pxyz[3 * i + a];
                }
                bool found = false;
                for (int j = 0; j < desc->n_point && !found; ++j)
                    found = pxyz[3 * j] == q[0] && pxyz[3 * j + 1] == q[1] && pxyz[3 * j + 2] == q[2] &&
                            std::equal(plum.begin() + static_cast<long>(i) * nl, plum.begin() + static_cast<long>(i + 1) * nl,
                                       plum.begin() + static_cast<long>(j) * nl);
                if (!found) return bail(fail(DARTRAY_E_INVAL, "octant mode: point sources not mirror-symmetric"));
            }
    }
    if (cudaGetDevice(&g->device) != cudaSuccess) return bail(fail(DARTRAY_E_CUDA, "no CUDA device"));
    cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    g->P.r_pre = models[0].r_pre;

    // j_sca layout (Eq. 5)
    long long off = 0;
    for (int l = 0; l < nl; ++l) {
        g->k_lam[l] = k_hp_host(gg[l], P.n_fwhm, P.k_sca_cap);
        g->off_lam[l] = off;
        off += tot_leaf * (12ll << (2 * g->k_lam[l]));
    }
    g->sca_len = off;
    g->sca_len_user = nlu < nl ? g->off_lam[nlu] : off;

    const size_t nU = static_cast<size_t>(tot_leaf) * nl;
    const long long ndir = dir_tab_offset(kDirTabLevels + 1);
    // automatic sizes: large enough for the biggest waves of galaxy-sized
    // grids, small for small grids
    g->cap = P.queue_rays > 0 ? P.queue_rays
                              : std::min<long long>(1ll << 27, std::max<long long>(1ll << 20, 512ll * tot_leaf));
    // automatic record capacity: 2048 per leaf, at most 2^29 and about 20 GB
    // per pipeline (a record: cell, direction, its bucketed copy, and two
    // coefficients per wavelength when there are several).  Waves whose
    // records do not fit deposit with per-pixel atomics, which costs far more
    // than the buffer: the 297,840-leaf galaxy's steps 1-2 plus one iteration
    // take 69.0 s with 2^27 records, 60.6 s with 2^28 and 56.0 s with 2^29.
    const long long rec_bytes = 36ll + (nl > 1 ? 8ll * nl : 0ll);
    const long long rec_auto = std::min<long long>(std::min<long long>(1ll << 29, (20ll << 30) / rec_bytes),
                                                   std::max<long long>(1ll << 20, 2048ll * tot_leaf));
    g->rec_alloc = P.deposit_direct ? 0 : (P.deposit_records > 0 ? P.deposit_records : rec_auto);
    g->rec_cap = g->rec_alloc;
    // merge table: low lists are far smaller than waves; a wave whose low list
    // does not fit is retried with a smaller source batch
    g->hcap = 1;
    while (g->hcap < std::min<long long>(2 * g->cap, 1ll << 27)) g->hcap <<= 1;
    const int n_all = static_cast<int>(tot_leaf + tot_point);
    const int nblk = (n_all + kBlock - 1) / kBlock;
#define AL(ptr, cnt)                                                                              \
    do {                                                                                          \
        cudaError_t e_ = dalloc(&(ptr), (cnt));                                                   \
        if (e_ != cudaSuccess)                                                                    \
            return bail(fail(DARTRAY_E_NOMEM, std::string("cudaMalloc ") + #ptr + ": " + cudaGetErrorString(e_))); \
    } while (0)
    AL(g->d_node_child, tot_nodes);
    AL(g->d_node_box, tot_nodes);
    AL(g->d_leaf_box, tot_leaf);
    AL(g->d_rope, static_cast<size_t>(tot_leaf) * 6);
    AL(g->d_dirtab, ndir);
    AL(g->d_ztab, static_cast<size_t>(ndir) * nl);
    AL(g->d_kr, nU);
    AL(g->d_emis, nU);
    AL(g->d_pxyz, static_cast<size_t>(tot_point) * 3);
    AL(g->d_plum, static_cast<size_t>(tot_point) * nl);
    AL(g->d_thr, nU);
    AL(g->d_fu_model, n_models);
    AL(g->d_mcount, n_models);
    AL(g->d_model_active, n_models);
    AL(g->d_mled, static_cast<size_t>(n_models) * LG_N * nl);
    AL(g->d_mled_fix, static_cast<size_t>(n_models) * LG_N * nl);
    AL(g->d_seg_beg, static_cast<size_t>(n_models) * nl);
    AL(g->d_seg_len, static_cast<size_t>(n_models) * nl);
    AL(g->d_seg_out, static_cast<size_t>(n_models) * nl);
    AL(g->d_seg_part, std::max<size_t>(static_cast<size_t>(n_models) * nl, kSegPartial));
    if (n_models > 1) {
        AL(g->d_models, n_models);
        AL(g->d_leaf_model, tot_leaf);
        AL(g->d_point_model, tot_point);
    }
    AL(g->d_U, nU);
    AL(g->d_ULL, nU);
    AL(g->d_pend[0], g->sca_len);
    AL(g->d_pend[1], g->sca_len);
    AL(g->d_jtot, g->sca_len);
    AL(g->d_flags, n_all);
    AL(g->d_blocksum, nblk + 1);
    AL(g->d_total, 1);
    AL(g->d_src_idx, n_all);
    AL(g->d_src_leaf, n_all);
    AL(g->d_src_hint, n_all);
    AL(g->d_src_pos, n_all);
    AL(g->d_src_S, static_cast<size_t>(n_all) * nl);
    AL(g->d_st, 1);
    AL(g->d_sum, 1);
    AL(g->d_partial, kSumBlocks);
    if (P.deterministic) {
        AL(g->d_Ufix, nU);
        AL(g->d_pfix, g->sca_len);
    }
    const int nblk_leaf = static_cast<int>((tot_leaf + kBlock - 1) / kBlock);
    for (int p = 0; p < kPipes; ++p) {
        Pipe &P = g->pipe[p];
        for (int i = 0; i < 2; ++i) {
            AL(P.d_H[i], g->cap);
            AL(P.d_M[i], g->cap);
            AL(P.d_HI[i], static_cast<size_t>(g->cap) * nl);
            AL(P.d_MI[i], static_cast<size_t>(g->cap) * nl);
        }
        AL(P.d_L, g->cap);
        AL(P.d_LI, static_cast<size_t>(g->cap) * nl);
        AL(P.d_hkey, g->hcap);
        AL(P.d_hcnt, g->hcap);
        AL(P.d_hmem, g->hcap);
        AL(P.d_pd, 1);
        AL(P.d_st, 1);
        if (g->rec_alloc > 0) {
            AL(P.d_rec_cell, g->rec_alloc);
            AL(P.d_rec_dir, g->rec_alloc);
            AL(P.d_srt_dir, g->rec_alloc);
            if (nl > 1) {  // one wavelength: the coefficient is stored in the direction's w
                AL(P.d_rec_coef, static_cast<size_t>(g->rec_alloc) * nl);
                AL(P.d_srt_coef, static_cast<size_t>(g->rec_alloc) * nl);
            }
            AL(P.d_cnt, tot_leaf);
            AL(P.d_off, tot_leaf);
            AL(P.d_cur, tot_leaf);
            AL(P.d_rec_n, 1);
            AL(P.d_blocksum, nblk_leaf + 1);
            AL(P.d_total, 1);
        }
        if (cudaMallocHost(reinterpret_cast<void **>(&P.h_pd), sizeof(PipeDev)) != cudaSuccess ||
            cudaStreamCreateWithFlags(&P.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&P.ev, cudaEventDisableTiming) != cudaSuccess)
            return bail(fail(DARTRAY_E_CUDA, "pipeline stream setup failed"));
        if (cudaMemsetAsync(P.d_pd, 0, sizeof(PipeDev), g->stream) != cudaSuccess ||
            cudaMemsetAsync(P.d_st, 0, sizeof(DevStats), g->stream) != cudaSuccess)
            return bail(fail(DARTRAY_E_CUDA, "memset failed"));
    }
    cudaStream_t s = g->stream;
    auto up = [&](auto *dst, const auto *src, size_t cnt) { return copy_in(dst, src, cnt, false, s); };
    if ((rc = up(g->d_node_child, g->topo.node_child.data(), tot_nodes))) return bail(rc);
    if ((rc = up(reinterpret_cast<float *>(g->d_node_box), g->topo.node_box.data(), 4ull * tot_nodes))) return bail(rc);
    if ((rc = up(reinterpret_cast<float *>(g->d_leaf_box), g->topo.leaf_box.data(), 4ull * tot_leaf))) return bail(rc);
    if ((rc = up(g->d_rope, g->topo.leaf_rope.data(), 6ull * tot_leaf))) return bail(rc);
    std::vector<uint16_t> leaf_model, point_model;
    for (int m = 0; m < n_models; ++m) {
        const dartray_grid_desc &d = descs[m];
        const bool dev_m = d.inputs_on_device != 0;
        const size_t l0 = static_cast<size_t>(g->m_leaf0[m]) * nl, p0 = static_cast<size_t>(g->m_point0[m]);
        if ((rc = copy_in_cols(g->d_kr + l0, d.kappa_rho, d.n_leaf, nlu, nl, dev_m, s)) ||
            (tangent && (rc = copy_in_cols_at(g->d_kr + l0, d.kappa_rho, d.n_leaf, nlu, nl, nl / 2, dev_m, s))) ||
            (rc = copy_in_cols(g->d_emis + l0, d.emissivity, d.n_leaf, nlu, nl, dev_m, s)) ||
            (rc = copy_in(g->d_pxyz + 3 * p0, d.point_xyz, 3ull * d.n_point, dev_m, s)) ||
            (rc = copy_in_cols(g->d_plum + p0 * nl, d.point_lum, d.n_point, nlu, nl, dev_m, s)))
            return bail(rc);
        leaf_model.insert(leaf_model.end(), d.n_leaf, static_cast<uint16_t>(m));
        point_model.insert(point_model.end(), d.n_point, static_cast<uint16_t>(m));
    }
    if (n_models > 1) {
        if ((rc = up(g->d_models, models.data(), n_models)) || (rc = up(g->d_leaf_model, leaf_model.data(), leaf_model.size())) ||
            (rc = up(g->d_point_model, point_model.data(), point_model.size())))
            return bail(rc);
    }
    // per-model host state and segments of the j_sca array (model, wavelength)
    g->m_lsca2.assign(n_models, 0.0);
    g->m_rem.assign(n_models, 0.0);
    g->m_active.assign(n_models, 1);
    g->m_ledger.assign(static_cast<size_t>(n_models) * LG_N * nl, 0.0);
    g->m_fu.assign(n_models, 0.0);
    {
        std::vector<long long> beg, len;
        for (int m = 0; m < n_models; ++m)
            for (int l = 0; l < nl; ++l) {
                const long long np = 12ll << (2 * g->k_lam[l]);
                beg.push_back(g->off_lam[l] + g->m_leaf0[m] * np);
                len.push_back(static_cast<long long>(g->m_nleaf[m]) * np);
            }
        if ((rc = up(g->d_seg_beg, beg.data(), beg.size())) || (rc = up(g->d_seg_len, len.data(), len.size()))) return bail(rc);
    }
    if (cudaMemsetAsync(g->d_U, 0, nU * sizeof(float), s) != cudaSuccess ||
        cudaMemsetAsync(g->d_ULL, 0, nU * sizeof(float), s) != cudaSuccess ||
        cudaMemsetAsync(g->d_pend[0], 0, g->sca_len * sizeof(float), s) != cudaSuccess ||
        cudaMemsetAsync(g->d_pend[1], 0, g->sca_len * sizeof(float), s) != cudaSuccess ||
        cudaMemsetAsync(g->d_jtot, 0, g->sca_len * sizeof(float), s) != cudaSuccess ||
        cudaMemsetAsync(g->d_st, 0, sizeof(DevStats), s) != cudaSuccess)
        return bail(fail(DARTRAY_E_CUDA, "memset failed"));
    dirtab_kernel<<<static_cast<unsigned>((ndir + kBlock - 1) / kBlock), kBlock, 0, s>>>(g->d_dirtab, ndir);
    ++g->launches;

    DevGrid &G = g->G;
    for (int a = 0; a < 3; ++a) {
        G.nroot[a] = desc->nroot[a];
        G.root_lo[a] = static_cast<float>(desc->root_lo[a]);
    }
    G.root_size = static_cast<float>(desc->root_size);
    G.n_nodes = static_cast<int>(tot_nodes);
    G.n_leaf = static_cast<int>(tot_leaf);
    G.nl = nl;
    G.nl_user = nlu;
    G.tangent = tangent ? 1 : 0;
    G.n_point = static_cast<int>(tot_point);
    G.n_models = n_models;
    G.models = g->d_models;
    G.leaf_model = g->d_leaf_model;
    G.point_model = g->d_point_model;
    G.node_child = g->d_node_child;
    G.node_box = g->d_node_box;
    G.leaf_box = g->d_leaf_box;
    G.leaf_rope = g->d_rope;
    G.kappa_rho = g->d_kr;
    G.emis = g->d_emis;
    G.point_xyz = g->d_pxyz;
    G.point_lum = g->d_plum;
    G.dirtab = g->d_dirtab;
    G.ztab = g->d_ztab;
    G.n_dirtab = ndir;
    for (int l = 0; l < nl; ++l) {
        G.albedo[l] = alb[l];
        G.g[l] = gg[l];
        G.k_lam[l] = g->k_lam[l];
        G.off_lam[l] = g->off_lam[l];
    }
    G.octant = P.octant;
    for (int a = 0; a < 3; ++a)
        G.centre[a] = static_cast<float>(desc->root_lo[a] + 0.5 * desc->nroot[a] * desc->root_size);
    if (P.octant) {
        AL(g->d_mirror, mirror.size());
        AL(g->d_mirror_pix, 7 * kMirrorPix);
        if (!P.deterministic) {
            AL(g->d_oct_u, nU);
            AL(g->d_oct_p, g->sca_len);
        }
        if ((rc = up(g->d_mirror, mirror.data(), mirror.size()))) return bail(rc);
        mirror_pix_kernel<<<(7 * kMirrorPix + kBlock - 1) / kBlock, kBlock, 0, s>>>(g->d_mirror_pix);
        ++g->launches;
        G.mirror = g->d_mirror;
        G.mirror_pix = g->d_mirror_pix;
    }
    ztab_kernel<<<static_cast<unsigned>((ndir + kBlock - 1) / kBlock), kBlock, 0, s>>>(G, g->d_ztab, ndir);
    ++g->launches;
    // the expansion kernel runs one block per resident slot (its ranges are
    // spread over the warps it has)
    g->acc_blocks[0] = occupancy_blocks(reinterpret_cast<const void *>(cell_accumulate_kernel<1, false>), g->num_sms);
    g->acc_blocks[1] = occupancy_blocks(reinterpret_cast<const void *>(cell_accumulate_kernel<2, false>), g->num_sms);
    g->acc_blocks[2] = occupancy_blocks(reinterpret_cast<const void *>(cell_accumulate_kernel<6, false>), g->num_sms);
    g->acc_blocks[3] = occupancy_blocks(reinterpret_cast<const void *>(cell_accumulate_kernel<24, false>), g->num_sms);
    g->acc_blocks[4] = occupancy_blocks(reinterpret_cast<const void *>(cell_accumulate_kernel<1, true>), g->num_sms);
    g->acc_blocks[5] = occupancy_blocks(reinterpret_cast<const void *>(cell_accumulate_kernel<2, true>), g->num_sms);
    g->acc_blocks[6] = occupancy_blocks(reinterpret_cast<const void *>(cell_accumulate_kernel<6, true>), g->num_sms);
    g->acc_blocks[7] = occupancy_blocks(reinterpret_cast<const void *>(cell_accumulate_kernel<24, true>), g->num_sms);
    // batched grids: the per-model ledgers live in dynamic shared memory
    g->march_smem = n_models > 1 ? n_models * LG_N * nl * static_cast<int>(sizeof(unsigned long long)) : 0;
    switch (nl) {
    case 1: g->march_blocks = occupancy_blocks(reinterpret_cast<const void *>(march_kernel<1, MODE_SCATTER, false>), g->num_sms, kMarchBlock, g->march_smem); break;
    case 2: g->march_blocks = occupancy_blocks(reinterpret_cast<const void *>(march_kernel<2, MODE_SCATTER, false>), g->num_sms, kMarchBlock, g->march_smem); break;
    default: g->march_blocks = std::max(1, march_wide_blocks_per_sm(nl, kMarchBlock, g->march_smem)) * g->num_sms; break;
    }
    if (cudaMallocHost(reinterpret_cast<void **>(&g->h_partial), kSumBlocks * sizeof(double)) != cudaSuccess)
        return bail(fail(DARTRAY_E_NOMEM, "pinned host buffer"));
    if (cudaEventCreate(&g->ev0) != cudaSuccess || cudaEventCreate(&g->ev1) != cudaSuccess ||
        cudaEventCreate(&g->mev0) != cudaSuccess || cudaEventCreate(&g->mev1) != cudaSuccess)
        return bail(fail(DARTRAY_E_CUDA, "event create failed"));
#undef AL
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bail(fail(DARTRAY_E_CUDA, cudaGetErrorString(e)));
    const cudaError_t e2 = cudaGetLastError();
    if (e2 != cudaSuccess) return bail(fail(DARTRAY_E_CUDA, cudaGetErrorString(e2)));
    *out = g;
    return DARTRAY_OK;
}

}  // namespace

extern "C" {

int dartray_grid_create(const dartray_grid_desc *desc, const dartray_params *params, void *cuda_stream,
                        dartray_grid **out) {
    return create_grid(desc, 1, params, cuda_stream, out);
}

int dartray_grid_create_batch(const dartray_grid_desc *descs, int32_t n_models, const dartray_params *params,
                              void *cuda_stream, dartray_grid **out) {
    return create_grid(descs, n_models, params, cuda_stream, out);
}

int dartray_direct(dartray_grid *g, dartray_stats *stats) {
    g_last_error.clear();
    if (!g) return fail(DARTRAY_E_INVAL, "null grid");
    int rc = set_device(g);
    if (rc) return rc;
    CK(cudaMemsetAsync(g->d_st, 0, sizeof(DevStats), g->stream));
    CK(cudaMemsetAsync(g->d_jtot, 0, g->sca_len * sizeof(float), g->stream));
    if (g->dg_on) CK(cudaMemsetAsync(g->d_dg, 0, static_cast<size_t>(g->n_leaf) * g->nl * sizeof(float), g->stream));
    g->cur = 0;  // step 2 deposits into d_pend[1]
    const long long l0 = g->launches;
    g->march_ms = g->flush_ms = g->busy_ms = g->march_sum_ms = 0.0;
    g->march_launches = g->restarts = g->batches = 0;
    // every model of a batch takes part in the scattering iterations again
    std::fill(g->m_active.begin(), g->m_active.end(), 1);
    CK(cudaMemcpyAsync(g->d_model_active, g->m_active.data(), g->n_models, cudaMemcpyHostToDevice, g->stream));
    CK(cudaEventRecord(g->ev0, g->stream));
    PhaseResult r1{}, r2{};
    if ((rc = run_phase(g, MODE_LL, &r1))) return rc;
    if ((rc = run_phase(g, MODE_DIRECT, &r2))) return rc;
    CK(cudaEventRecord(g->ev1, g->stream));
    CK(cudaEventSynchronize(g->ev1));
    g->l_sca2 = r2.pend_sum;
    g->have_direct = true;
    if (stats) {
        fill_stats(g, r2, stats);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, g->ev0, g->ev1);
        stats->gpu_ms = ms;
        stats->kernel_launches = g->launches - l0;
        stats->march_ms = g->march_ms;
        stats->march_launches = g->march_launches;
        stats->flush_ms = g->flush_ms;
        stats->busy_ms = g->busy_ms;
        stats->restarts = g->restarts;
        stats->march_sum_ms = g->march_sum_ms;
        stats->batches = g->batches;
    }
    return DARTRAY_OK;
}

int dartray_scatter_iter(dartray_grid *g, double *remaining_frac, dartray_stats *stats) {
    g_last_error.clear();
    if (!g) return fail(DARTRAY_E_INVAL, "null grid");
    if (!g->have_direct) return fail(DARTRAY_E_STATE, "dartray_direct must run first");
    int rc = set_device(g);
    if (rc) return rc;
    CK(cudaMemsetAsync(g->d_st, 0, sizeof(DevStats), g->stream));
    const long long l0 = g->launches;
    g->march_ms = g->flush_ms = g->busy_ms = g->march_sum_ms = 0.0;
    g->march_launches = g->restarts = g->batches = 0;
    CK(cudaEventRecord(g->ev0, g->stream));
    PhaseResult r{};
    if ((rc = run_phase(g, MODE_SCATTER, &r))) return rc;
    CK(cudaEventRecord(g->ev1, g->stream));
    CK(cudaEventSynchronize(g->ev1));
    double rem = g->l_sca2 > 0 ? r.pend_sum / g->l_sca2 : 0.0;
    if (g->n_models > 1) {
        // batched grids: a model whose remaining fraction fell below f_L stops
        // emitting (as a loop over single models would stop it); the call
        // returns the largest remaining fraction
        rem = 0.0;
        for (int m = 0; m < g->n_models; ++m) {
            rem = std::max(rem, g->m_rem[m]);
            if (g->m_rem[m] < g->P.f_l) g->m_active[m] = 0;
        }
        CK(cudaMemcpyAsync(g->d_model_active, g->m_active.data(), g->n_models, cudaMemcpyHostToDevice, g->stream));
        CK(cudaStreamSynchronize(g->stream));
    }
    if (remaining_frac) *remaining_frac = rem;
    if (stats) {
        fill_stats(g, r, stats);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, g->ev0, g->ev1);
        stats->gpu_ms = ms;
        stats->kernel_launches = g->launches - l0;
        stats->march_ms = g->march_ms;
        stats->march_launches = g->march_launches;
        stats->flush_ms = g->flush_ms;
        stats->busy_ms = g->busy_ms;
        stats->restarts = g->restarts;
        stats->march_sum_ms = g->march_sum_ms;
        stats->batches = g->batches;
    }
    return DARTRAY_OK;
}

namespace {

// image-plane frame of an external map: right = up x view, up made
// orthogonal to view
int external_frame(dartray_grid *g, const double view[3], const double up[3], const double origin[2], double pixel,
                   int32_t nx, int32_t ny, ExtMapArgs *M) {
    if (g->n_models > 1) return fail(DARTRAY_E_INVAL, "maps are made of single-model grids");
    if (nx < 1 || ny < 1 || static_cast<long long>(nx) * ny > (1ll << 26) || !(pixel > 0))
        return fail(DARTRAY_E_INVAL, "bad image size");
    double vn = std::sqrt(view[0] * view[0] + view[1] * view[1] + view[2] * view[2]);
    if (!(vn > 0)) return fail(DARTRAY_E_INVAL, "bad view direction");
    double w[3] = {view[0] / vn, view[1] / vn, view[2] / vn};
    double u[3] = {up[0], up[1], up[2]};
    const double uw = u[0] * w[0] + u[1] * w[1] + u[2] * w[2];
    for (int a = 0; a < 3; ++a) u[a] -= uw * w[a];
    const double un = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    if (!(un > 1e-12)) return fail(DARTRAY_E_INVAL, "up is parallel to view");
    for (int a = 0; a < 3; ++a) u[a] /= un;
    const double r[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
    for (int a = 0; a < 3; ++a) {
        M->view[a] = w[a];
        M->up[a] = u[a];
        M->right[a] = r[a];
        M->box_lo[a] = g->G.root_lo[a];
        M->box_hi[a] = static_cast<double>(g->G.root_lo[a]) + static_cast<double>(g->G.nroot[a]) * g->G.root_size;
    }
    M->origin[0] = origin[0];
    M->origin[1] = origin[1];
    M->px = pixel;
    M->nx = nx;
    M->ny = ny;
    return DARTRAY_OK;
}

}  // namespace

int dartray_map_external(dartray_grid *g, const double view[3], const double up[3], const double origin[2],
                         double pixel, int32_t nx, int32_t ny, int32_t use_jsca, float *map, int dst_is_device) {
    g_last_error.clear();
    if (!g || !view || !up || !origin || !map) return fail(DARTRAY_E_INVAL, "null argument");
    ExtMapArgs M{};
    int rc = external_frame(g, view, up, origin, pixel, nx, ny, &M);
    if (rc) return rc;
    if ((rc = set_device(g))) return rc;
    const size_t n = static_cast<size_t>(nx) * ny * g->nl, n_user = static_cast<size_t>(nx) * ny * g->nlu;
    float *dst = map;
    if ((!dst_is_device || g->nlu < g->nl) && (rc = stage_buffer(g, n, &dst))) return rc;
    M.jsca = use_jsca ? g->d_jtot : nullptr;
    M.map = dst;
    if (launch_external_map(g->G, M, false, g->stream)) return fail(DARTRAY_E_INVAL, "unsupported n_lambda");
    ++g->launches;
    CK(cudaGetLastError());
    if (dst != map)  // the caller's wavelengths are the first rows
        CK(cudaMemcpyAsync(map, dst, n_user * sizeof(float),
                           dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return DARTRAY_OK;
}

int dartray_map_external_vjp(dartray_grid *g, const double view[3], const double up[3], const double origin[2],
                             double pixel, int32_t nx, int32_t ny, int32_t use_jsca, const float *dmap,
                             float *grad_kappa_rho, double *grad_albedo, double *grad_g, int on_device) {
    g_last_error.clear();
    if (!g || !view || !up || !origin || !dmap || !grad_kappa_rho) return fail(DARTRAY_E_INVAL, "null argument");
    ExtMapArgs M{};
    int rc = external_frame(g, view, up, origin, pixel, nx, ny, &M);
    if (rc) return rc;
    if (grad_g) {
        bool same = g->dg_on && use_jsca;
        for (int a = 0; a < 3; ++a) same = same && std::fabs(M.view[a] - g->dg_view[a]) <= 1e-12;
        if (!same) return fail(DARTRAY_E_STATE, "grad_g needs use_jsca and the j_sca g tally armed for this view");
    }
    if ((rc = set_device(g))) return rc;
    const size_t n = static_cast<size_t>(nx) * ny * g->nl, nU = static_cast<size_t>(g->n_leaf) * g->nl;
    const size_t n_user = static_cast<size_t>(nx) * ny * g->nlu;
    const bool padded = g->nlu < g->nl;
    // the grid's staging buffer holds the per-wavelength sums (two rows of
    // doubles, at its start) and, for host arguments or extra wavelengths,
    // the upstream gradient (zero rows for the extra wavelengths) and the
    // result
    const size_t n_dbl = 4 * kMaxLambda;  // in floats
    const bool staged = !on_device || padded;
    float *st = nullptr;
    if ((rc = stage_buffer(g, n_dbl + (staged ? n + nU : 0), &st))) return rc;
    double *d_gs = reinterpret_cast<double *>(st);
    float *d_in = const_cast<float *>(dmap), *d_out = grad_kappa_rho;
    if (staged) {
        d_in = st + n_dbl;
        d_out = st + n_dbl + n;
        if (padded) CK(cudaMemsetAsync(d_in + n_user, 0, (n - n_user) * sizeof(float), g->stream));
        CK(cudaMemcpyAsync(d_in, dmap, n_user * sizeof(float),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->stream));
    }
    CK(cudaMemsetAsync(d_out, 0, nU * sizeof(float), g->stream));
    CK(cudaMemsetAsync(d_gs, 0, 2 * kMaxLambda * sizeof(double), g->stream));
    M.jsca = use_jsca ? g->d_jtot : nullptr;
    M.dmap = d_in;
    M.grad = d_out;
    M.grad_sca = d_gs;
    M.dg = grad_g ? g->d_dg : nullptr;
    M.grad_g = grad_g ? d_gs + kMaxLambda : nullptr;
    if (launch_external_map(g->G, M, true, g->stream)) return fail(DARTRAY_E_INVAL, "unsupported n_lambda");
    ++g->launches;
    CK(cudaGetLastError());
    if (staged && (rc = copy_out_cols(grad_kappa_rho, d_out, g->n_leaf, g->nlu, g->nl, on_device != 0, g->stream)))
        return rc;
    double gs[2 * kMaxLambda];
    CK(cudaMemcpyAsync(gs, d_gs, 2 * kMaxLambda * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    // j_sca is proportional to the albedo (the radiation field held fixed)
    if (grad_albedo)
        for (int l = 0; l < g->nlu; ++l) grad_albedo[l] = g->G.albedo[l] > 0 ? gs[l] / g->G.albedo[l] : 0.0;
    if (grad_g)
        for (int l = 0; l < g->nlu; ++l) grad_g[l] = gs[kMaxLambda + l];
    return DARTRAY_OK;
}

int dartray_jsca_dg_arm(dartray_grid *g, const double view[3]) {
    g_last_error.clear();
    if (!g) return fail(DARTRAY_E_INVAL, "null grid");
    if (!view) {
        g->dg_on = false;
        return DARTRAY_OK;
    }
    if (g->n_models > 1 || g->G.octant)
        return fail(DARTRAY_E_INVAL, "the g tally is for single-model grids outside the octant mode");
    const double vn = std::sqrt(view[0] * view[0] + view[1] * view[1] + view[2] * view[2]);
    if (!(vn > 0)) return fail(DARTRAY_E_INVAL, "bad view direction");
    int rc = set_device(g);
    if (rc) return rc;
    const size_t nU = static_cast<size_t>(g->n_leaf) * g->nl;
    if (!g->d_dg) {
        CK(cudaMalloc(reinterpret_cast<void **>(&g->d_dg), nU * sizeof(float)));
        CK(cudaMalloc(reinterpret_cast<void **>(&g->d_dg_phase), nU * sizeof(float)));
        CK(cudaMalloc(reinterpret_cast<void **>(&g->d_dg_dir), kMaxLambda * sizeof(float4)));
    }
    for (int a = 0; a < 3; ++a) g->dg_view[a] = view[a] / vn;
    dg_dir_kernel<<<1, kMaxLambda, 0, g->stream>>>(g->G, g->dg_view[0], g->dg_view[1], g->dg_view[2], g->d_dg_dir);
    ++g->launches;
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(g->d_dg, 0, nU * sizeof(float), g->stream));
    CK(cudaStreamSynchronize(g->stream));
    g->dg_on = true;
    return DARTRAY_OK;
}

int dartray_jsca_dg(dartray_grid *g, float *out, int dst_is_device) {
    g_last_error.clear();
    if (!g || !out) return fail(DARTRAY_E_INVAL, "null argument");
    if (!g->dg_on) return fail(DARTRAY_E_STATE, "the g tally is not armed");
    int rc = set_device(g);
    if (rc) return rc;
    if ((rc = copy_out_cols(out, g->d_dg, g->n_leaf, g->nlu, g->nl, dst_is_device != 0, g->stream))) return rc;
    CK(cudaStreamSynchronize(g->stream));
    return DARTRAY_OK;
}

int dartray_set_kappa_rho(dartray_grid *g, const float *kappa_rho, int src_is_device) {
    g_last_error.clear();
    if (!g || !kappa_rho) return fail(DARTRAY_E_INVAL, "null argument");
    int rc = set_device(g);
    if (rc) return rc;
    if ((rc = copy_in_cols(g->d_kr, kappa_rho, g->n_leaf, g->nlu, g->nl, src_is_device != 0, g->stream))) return rc;
    if (g->G.tangent &&
        (rc = copy_in_cols_at(g->d_kr, kappa_rho, g->n_leaf, g->nlu, g->nl, g->nl / 2, src_is_device != 0, g->stream)))
        return rc;
    CK(cudaStreamSynchronize(g->stream));
    return DARTRAY_OK;
}

int dartray_set_emissivity(dartray_grid *g, const float *emis, int src_is_device) {
    g_last_error.clear();
    if (!g || !emis) return fail(DARTRAY_E_INVAL, "null argument");
    int rc = set_device(g);
    if (rc) return rc;
    if ((rc = copy_in_cols(g->d_emis, emis, g->n_leaf, g->nlu, g->nl, src_is_device != 0, g->stream))) return rc;
    CK(cudaStreamSynchronize(g->stream));
    return DARTRAY_OK;
}

int dartray_direct_incremental(dartray_grid *g, dartray_stats *stats) {
    g_last_error.clear();
    if (!g) return fail(DARTRAY_E_INVAL, "null grid");
    if (!g->have_direct) return fail(DARTRAY_E_STATE, "dartray_direct must run first");
    int rc = set_device(g);
    if (rc) return rc;
    CK(cudaMemsetAsync(g->d_st, 0, sizeof(DevStats), g->stream));
    g->cur = 0;
    const long long l0 = g->launches;
    g->march_ms = g->flush_ms = g->busy_ms = g->march_sum_ms = 0.0;
    g->march_launches = g->restarts = g->batches = 0;
    std::fill(g->m_active.begin(), g->m_active.end(), 1);
    CK(cudaMemcpyAsync(g->d_model_active, g->m_active.data(), g->n_models, cudaMemcpyHostToDevice, g->stream));
    CK(cudaEventRecord(g->ev0, g->stream));
    PhaseResult r{};
    if ((rc = run_phase(g, MODE_DIRECT, &r, true))) return rc;
    CK(cudaEventRecord(g->ev1, g->stream));
    CK(cudaEventSynchronize(g->ev1));
    g->l_sca2 = r.pend_sum;
    if (stats) {
        fill_stats(g, r, stats);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, g->ev0, g->ev1);
        stats->gpu_ms = ms;
        stats->kernel_launches = g->launches - l0;
    }
    return DARTRAY_OK;
}

int dartray_dust_emission(dartray_grid *ir, const dartray_grid *stellar, const dartray_dust *dust, float *T,
                          float *j, int dst_is_device, double *max_rel_change) {
    g_last_error.clear();
    if (!ir || !stellar || !dust) return fail(DARTRAY_E_INVAL, "null argument");
    if (ir->nlu != ir->nl || stellar->nlu != stellar->nl)
        return fail(DARTRAY_E_INVAL, "dust emission: grids of 1, 2, 4, 8 or 16 wavelengths");
    if (ir->n_leaf != stellar->n_leaf || dust->n_ir != ir->nl || dust->n_stellar != stellar->nl ||
        !(dust->scale > 0) || !(dust->t_min > 0) || !(dust->t_max > dust->t_min) || ir->device != stellar->device)
        return fail(DARTRAY_E_INVAL, "dust emission: grids or parameters do not match");
    int rc = set_device(ir);
    if (rc) return rc;
    cudaStream_t s = ir->stream;
    const size_t nU = static_cast<size_t>(ir->n_leaf) * ir->nl;
    if (!ir->d_jd) {
        CK(cudaMalloc(reinterpret_cast<void **>(&ir->d_jd), nU * sizeof(float)));
        CK(cudaMalloc(reinterpret_cast<void **>(&ir->d_maxrel), sizeof(unsigned)));
        CK(cudaMemsetAsync(ir->d_jd, 0, nU * sizeof(float), s));
    }
    float *Tdev = nullptr;
    if (T && !dst_is_device && (rc = stage_buffer(ir, ir->n_leaf, &Tdev))) return rc;
    if (T && dst_is_device) Tdev = T;
    // the stellar grid's work must be complete before its U is read
    if (stellar->stream != s) CK(cudaStreamSynchronize(stellar->stream));
    DustArgs D{};
    D.n_leaf = ir->n_leaf;
    D.n_ir = ir->nl;
    D.n_st = stellar->nl;
    for (int i = 0; i < ir->nl; ++i) {
        D.lam[i] = dust->lam_ir[i];
        D.dlam[i] = dust->dlam_ir[i];
        D.alb_ir[i] = ir->G.albedo[i];
    }
    for (int i = 0; i < stellar->nl; ++i) {
        D.dlam_st[i] = dust->dlam_stellar[i];
        D.alb_st[i] = stellar->G.albedo[i];
    }
    D.scale = dust->scale;
    D.t_lo = dust->t_min;
    D.t_hi = dust->t_max;
    D.c_light = ir->P.c_light;
    D.U_ir = ir->d_U;
    D.kr_ir = ir->d_kr;
    D.U_st = stellar->d_U;
    D.kr_st = stellar->d_kr;
    D.leaf_box = ir->d_leaf_box;
    D.j_prev = ir->d_jd;
    D.emis = ir->d_emis;
    D.T = Tdev;
    D.max_rel = ir->d_maxrel;
    CK(cudaMemsetAsync(ir->d_maxrel, 0, sizeof(unsigned), s));
    dust_emission_kernel<<<(ir->n_leaf + kBlock - 1) / kBlock, kBlock, 0, s>>>(D);
    ++ir->launches;
    CK(cudaGetLastError());
    unsigned bits = 0;
    CK(cudaMemcpyAsync(&bits, ir->d_maxrel, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    const cudaMemcpyKind k = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (j) CK(cudaMemcpyAsync(j, ir->d_jd, nU * sizeof(float), k, s));
    if (T && !dst_is_device) CK(cudaMemcpyAsync(T, Tdev, ir->n_leaf * sizeof(float), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    float rel;
    std::memcpy(&rel, &bits, sizeof rel);
    if (max_rel_change) *max_rel_change = rel;
    return DARTRAY_OK;
}

int dartray_autotune(dartray_grid *g, int32_t sample_stride, int32_t *choice, double *ms) {
    g_last_error.clear();
    if (!g || sample_stride < 1) return fail(DARTRAY_E_INVAL, "bad argument");
    int rc = set_device(g);
    if (rc) return rc;
    // candidate deposit schedules: deferred records with the full buffer,
    // deferred with a sixteenth of it (smaller, more frequent flushes), and
    // per-pixel atomics in the marcher
    const long long cand[3] = {g->rec_alloc, g->rec_alloc > 0 ? std::max<long long>(1ll << 20, g->rec_alloc / 16) : 0,
                               0};
    const int first = g->rec_alloc > 0 ? 0 : 2;
    const int32_t stride0 = g->P.src_stride, offset0 = g->P.src_offset;
    const double rps0[3] = {g->rays_per_src[0], g->rays_per_src[1], g->rays_per_src[2]};
    g->P.src_stride = sample_stride;
    g->P.src_offset = 0;
    double best = 1e300;
    int best_i = 2;
    for (int i = 0; i < 3; ++i) {
        if (ms) ms[i] = -1.0;
        if (i < first) continue;
        g->rec_cap = cand[i];
        CK(cudaMemsetAsync(g->d_jtot, 0, g->sca_len * sizeof(float), g->stream));
        g->cur = 0;
        CK(cudaEventRecord(g->ev0, g->stream));
        PhaseResult r1{}, r2{};
        if ((rc = run_phase(g, MODE_LL, &r1)) || (rc = run_phase(g, MODE_DIRECT, &r2))) break;
        CK(cudaEventRecord(g->ev1, g->stream));
        CK(cudaEventSynchronize(g->ev1));
        float t = 0.f;
        cudaEventElapsedTime(&t, g->ev0, g->ev1);
        if (ms) ms[i] = t;
        if (t < best) {
            best = t;
            best_i = i;
        }
    }
    g->P.src_stride = stride0;
    g->P.src_offset = offset0;
    for (int k = 0; k < 3; ++k) g->rays_per_src[k] = rps0[k];
    g->rec_cap = cand[best_i];
    g->have_direct = false;  // the trial phases leave no usable state
    if (rc) return rc;
    if (choice) *choice = best_i;
    return DARTRAY_OK;
}

int dartray_rfed(dartray_grid *g, float *U, float *L_abs, int dst_is_device) {
    g_last_error.clear();
    if (!g) return fail(DARTRAY_E_INVAL, "null grid");
    int rc = set_device(g);
    if (rc) return rc;
    const size_t nU = static_cast<size_t>(g->n_leaf) * g->nl;
    const bool padded = g->nlu < g->nl;
    if (U && (rc = copy_out_cols(U, g->d_U, g->n_leaf, g->nlu, g->nl, dst_is_device != 0, g->stream))) return rc;
    if (L_abs) {
        float *dst = L_abs;
        if ((!dst_is_device || padded) && (rc = stage_buffer(g, nU, &dst))) return rc;
        labs_kernel<<<static_cast<unsigned>((nU + kBlock - 1) / kBlock), kBlock, 0, g->stream>>>(
            g->G, g->d_U, static_cast<float>(g->P.c_light), dst);
        ++g->launches;
        CK(cudaGetLastError());
        if (dst != L_abs && (rc = copy_out_cols(L_abs, dst, g->n_leaf, g->nlu, g->nl, dst_is_device != 0, g->stream)))
            return rc;
    }
    CK(cudaStreamSynchronize(g->stream));
    return DARTRAY_OK;
}

int dartray_rfed_tangent(dartray_grid *g, float *dU, float *dL_abs, int dst_is_device) {
    g_last_error.clear();
    if (!g) return fail(DARTRAY_E_INVAL, "null grid");
    if (!g->G.tangent) return fail(DARTRAY_E_STATE, "the grid was not created in the forward mode");
    int rc = set_device(g);
    if (rc) return rc;
    const int half = g->nl / 2;
    if (dU && (rc = copy_out_cols_at(dU, g->d_U, g->n_leaf, g->nlu, g->nl, half, dst_is_device != 0, g->stream)))
        return rc;
    if (dL_abs) {
        const size_t n = static_cast<size_t>(g->n_leaf) * g->nlu;
        float *dst = dL_abs;
        if (!dst_is_device && (rc = stage_buffer(g, n, &dst))) return rc;
        tangent_labs_kernel<<<static_cast<unsigned>((n + kBlock - 1) / kBlock), kBlock, 0, g->stream>>>(
            g->G, g->d_U, static_cast<float>(g->P.c_light), dst);
        ++g->launches;
        CK(cudaGetLastError());
        if (!dst_is_device) CK(cudaMemcpyAsync(dL_abs, dst, n * sizeof(float), cudaMemcpyDeviceToHost, g->stream));
    }
    CK(cudaStreamSynchronize(g->stream));
    return DARTRAY_OK;
}

int dartray_jsca_layout(const dartray_grid *g, int32_t *k_lambda, int64_t *offsets, int64_t *total_len) {
    if (!g) return fail(DARTRAY_E_INVAL, "null grid");
    for (int l = 0; l < g->nlu; ++l) {
        if (k_lambda) k_lambda[l] = g->k_lam[l];
        if (offsets) offsets[l] = g->off_lam[l];
    }
    if (total_len) *total_len = g->sca_len_user;
    return DARTRAY_OK;
}

int dartray_jsca(dartray_grid *g, int which, float *out, int dst_is_device) {
    g_last_error.clear();
    if (!g || !out || which < 0 || which > 1) return fail(DARTRAY_E_INVAL, "bad argument");
    int rc = set_device(g);
    if (rc) return rc;
    const float *src = which == 0 ? g->d_jtot : g->d_pend[1 - g->cur];
    CK(cudaMemcpyAsync(out, src, g->sca_len_user * sizeof(float),
                       dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return DARTRAY_OK;
}

int dartray_map(dartray_grid *g, const double observer[3], int32_t nside_k, int32_t max_sub, int32_t use_jsca,
                float *map, int dst_is_device) {
    g_last_error.clear();
    if (!g || !observer || !map) return fail(DARTRAY_E_INVAL, "null argument");
    if (nside_k < 0 || nside_k > 10 || max_sub < 0 || max_sub > 6) return fail(DARTRAY_E_INVAL, "bad map size");
    if (g->n_models > 1) return fail(DARTRAY_E_INVAL, "maps are made of single-model grids");
    int rc = set_device(g);
    if (rc) return rc;
    const long long npix = 12ll << (2 * nside_k);
    const size_t nmap = static_cast<size_t>(npix) * g->nl, nmap_user = static_cast<size_t>(npix) * g->nlu;
    float *dst = map;
    if ((!dst_is_device || g->nlu < g->nl) && (rc = stage_buffer(g, nmap, &dst))) return rc;
    CK(cudaMemsetAsync(dst, 0, nmap * sizeof(float), g->stream));
    MapArgs M{};
    for (int a = 0; a < 3; ++a) M.obs[a] = observer[a];  // double: exact subdivision / pixel decisions
    M.nside_k = nside_k;
    M.max_sub = max_sub;
    M.jsca = use_jsca ? g->d_jtot : nullptr;
    M.map = dst;
    const int blocks = (g->n_leaf + kBlock - 1) / kBlock;
    rc = launch_map(g->G, M, blocks, g->stream);
    if (rc) return fail(DARTRAY_E_INVAL, "unsupported n_lambda for maps");
    ++g->launches;
    CK(cudaGetLastError());
    // the caller's wavelengths are the first rows
    if (dst != map)
        CK(cudaMemcpyAsync(map, dst, nmap_user * sizeof(float),
                           dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return DARTRAY_OK;
}

// Device address of g_noalloc_map on the current device.  Host code must not
// use the symbol itself (it names a host-side shadow); the address is looked
// up once per device, with that device current, and cached.
static int noalloc_scratch(int device, float **out) {
    static std::mutex mu;
    static float *addr[256] = {nullptr};
    if (device < 0 || device >= 256) return fail(DARTRAY_E_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_map);
        if (e != cudaSuccess || !p)
            return fail(DARTRAY_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        addr[device] = static_cast<float *>(p);
    }
    *out = addr[device];
    return DARTRAY_OK;
}

int dartray_map_noalloc(dartray_grid *g, const double observer[3], int32_t nside_k, int32_t max_sub,
                        int32_t use_jsca, float *map, int dst_is_device) {
    g_last_error.clear();
    if (!g || !observer || !map) return fail(DARTRAY_E_INVAL, "null argument");
    if (nside_k < 0 || nside_k > 10 || max_sub < 0 || max_sub > 6) return fail(DARTRAY_E_INVAL, "bad map size");
    if (g->n_models > 1) return fail(DARTRAY_E_INVAL, "maps are made of single-model grids");
    const long long npix = 12ll << (2 * nside_k);
    const long long nmap = npix * g->nl;
    if (nmap > kNoAllocMapFloats) {
        char m[200];
        std::snprintf(m, sizeof m,
                      "map of %lld floats (12*4^%d pixels x %d wavelengths) exceeds the %lld-float static buffer "
                      "of dartray_map_noalloc",
                      nmap, nside_k, g->nl, kNoAllocMapFloats);
        return fail(DARTRAY_E_INVAL, m);
    }
    int rc = set_device(g);
    if (rc) return rc;
    float *scratch = nullptr;
    if ((rc = noalloc_scratch(g->device, &scratch))) return rc;
    // the buffer keeps the previous call's map: clear the part this call sums into
    CK(cudaMemsetAsync(scratch, 0, static_cast<size_t>(nmap) * sizeof(float), g->stream));
    MapArgs M{};
    for (int a = 0; a < 3; ++a) M.obs[a] = observer[a];
    M.nside_k = nside_k;
    M.max_sub = max_sub;
    M.jsca = use_jsca ? g->d_jtot : nullptr;
    M.map = scratch;
    const int blocks = (g->n_leaf + kBlock - 1) / kBlock;
    rc = launch_map(g->G, M, blocks, g->stream);
    if (rc) return fail(DARTRAY_E_INVAL, "unsupported n_lambda for maps");
    ++g->launches;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(map, scratch, static_cast<size_t>(npix) * g->nlu * sizeof(float),
                       dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return DARTRAY_OK;
}

int dartray_state_save(dartray_grid *g, const char *path) {
    g_last_error.clear();
    if (!g || !path) return fail(DARTRAY_E_INVAL, "null argument");
    if (g->n_models > 1 || g->G.tangent)
        return fail(DARTRAY_E_INVAL, "state files hold single-model grids outside the forward mode");
    int rc = set_device(g);
    if (rc) return rc;
    const size_t nU = static_cast<size_t>(g->n_leaf) * g->nlu;
    std::vector<float> buf(std::max<size_t>(nU, g->sca_len_user));
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(DARTRAY_E_INVAL, std::string("cannot open ") + path);
    const char magic[8] = {'D', 'R', 'T', 'S', 'T', 'A', 'T', '1'};
    long long hdr[4] = {g->n_leaf, g->nlu, g->sca_len_user, g->have_direct ? 1 : 0};
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof hdr, 1, f) == 1 &&
              std::fwrite(&g->l_sca2, sizeof(double), 1, f) == 1;
    const float *arrs[5] = {g->d_U, g->d_ULL, g->d_pend[g->cur], g->d_pend[1 - g->cur], g->d_jtot};
    const size_t lens[5] = {nU, nU, static_cast<size_t>(g->sca_len_user), static_cast<size_t>(g->sca_len_user),
                            static_cast<size_t>(g->sca_len_user)};
    for (int i = 0; i < 5 && ok; ++i) {
        // [n_leaf][nlu] fields and the first nlu j_sca blocks
        const bool fail_copy = i < 2 ? copy_out_cols(buf.data(), arrs[i], g->n_leaf, g->nlu, g->nl, false, g->stream) != 0 ||
                                           cudaStreamSynchronize(g->stream) != cudaSuccess
                                     : cudaMemcpy(buf.data(), arrs[i], lens[i] * sizeof(float), cudaMemcpyDeviceToHost) !=
                                           cudaSuccess;
        if (fail_copy) {
            std::fclose(f);
            return fail(DARTRAY_E_CUDA, "copy failed");
        }
        ok = std::fwrite(buf.data(), sizeof(float), lens[i], f) == lens[i];
    }
    std::fclose(f);
    return ok ? DARTRAY_OK : fail(DARTRAY_E_INVAL, "write failed");
}

int dartray_state_load(dartray_grid *g, const char *path) {
    g_last_error.clear();
    if (!g || !path) return fail(DARTRAY_E_INVAL, "null argument");
    if (g->n_models > 1 || g->G.tangent)
        return fail(DARTRAY_E_INVAL, "state files hold single-model grids outside the forward mode");
    int rc = set_device(g);
    if (rc) return rc;
    const size_t nU = static_cast<size_t>(g->n_leaf) * g->nlu;
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(DARTRAY_E_INVAL, std::string("cannot open ") + path);
    char magic[8];
    long long hdr[4];
    double l2 = 0;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "DRTSTAT1", 8) == 0 &&
              std::fread(hdr, sizeof hdr, 1, f) == 1 && std::fread(&l2, sizeof(double), 1, f) == 1 &&
              hdr[0] == g->n_leaf && hdr[1] == g->nlu && hdr[2] == g->sca_len_user;
    if (!ok) {
        std::fclose(f);
        return fail(DARTRAY_E_INVAL, "state file does not match this grid");
    }
    std::vector<float> buf(std::max<size_t>(nU, g->sca_len_user));
    g->cur = 0;
    float *arrs[5] = {g->d_U, g->d_ULL, g->d_pend[0], g->d_pend[1], g->d_jtot};
    const size_t lens[5] = {nU, nU, static_cast<size_t>(g->sca_len_user), static_cast<size_t>(g->sca_len_user),
                            static_cast<size_t>(g->sca_len_user)};
    const size_t tail = static_cast<size_t>(g->sca_len - g->sca_len_user);  // blocks of the extra wavelengths
    for (int i = 0; i < 5 && ok; ++i) {
        ok = std::fread(buf.data(), sizeof(float), lens[i], f) == lens[i];
        bool bad = false;
        if (ok && i < 2) {
            bad = copy_in_cols(arrs[i], buf.data(), g->n_leaf, g->nlu, g->nl, false, g->stream) != 0 ||
                  cudaStreamSynchronize(g->stream) != cudaSuccess;
        } else if (ok) {
            bad = cudaMemcpy(arrs[i], buf.data(), lens[i] * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
                  (tail && cudaMemset(arrs[i] + g->sca_len_user, 0, tail * sizeof(float)) != cudaSuccess);
        }
        if (bad) {
            std::fclose(f);
            return fail(DARTRAY_E_CUDA, "copy failed");
        }
    }
    std::fclose(f);
    if (!ok) return fail(DARTRAY_E_INVAL, "truncated state file");
    g->l_sca2 = l2;
    g->have_direct = hdr[3] != 0;
    return DARTRAY_OK;
}

int dartray_model_info(const dartray_grid *g, int32_t model, int64_t *leaf_offset, int32_t *n_leaf,
                       int64_t *point_offset, double *remaining_frac, int32_t *active) {
    if (!g || model < 0 || model >= g->n_models) return fail(DARTRAY_E_INVAL, "bad model index");
    if (leaf_offset) *leaf_offset = g->m_leaf0[model];
    if (n_leaf) *n_leaf = g->m_nleaf[model];
    if (point_offset) *point_offset = g->m_point0[model];
    if (remaining_frac) *remaining_frac = g->m_rem[model];
    if (active) *active = g->m_active[model];
    return DARTRAY_OK;
}

int dartray_model_stats(const dartray_grid *g, int32_t model, dartray_stats *st) {
    if (!g || !st || model < 0 || model >= g->n_models) return fail(DARTRAY_E_INVAL, "bad argument");
    std::memset(st, 0, sizeof *st);
    const double *L = &g->m_ledger[static_cast<size_t>(model) * LG_N * g->nl];
    for (int l = 0; l < g->nl; ++l) {
        const double w = g->G.albedo[l];
        st->emitted[l] = L[LG_EMITTED * g->nl + l];
        st->absorbed[l] = (1.0 - w) * L[LG_DEPOSITED * g->nl + l];
        st->scattered[l] = w * L[LG_DEPOSITED * g->nl + l];
        st->escaped[l] = L[LG_ESCAPED * g->nl + l];
        st->blocked[l] = L[LG_BLOCKED * g->nl + l];
        st->cut[l] = L[LG_CUT * g->nl + l];
        st->skipped[l] = L[LG_SKIPPED * g->nl + l];
    }
    st->f_u = g->m_fu[model];
    st->l_sca2 = g->m_lsca2[model];
    return DARTRAY_OK;
}

void dartray_grid_destroy(dartray_grid *g) {
    if (!g) return;
    cudaSetDevice(g->device);
    cudaStreamSynchronize(g->stream);
    free_all(g);
    delete g;
}

const char *dartray_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// Surface-brightness maps for an observer inside the model (paper Sect. 2,
// end: I_obs = I_0 exp(-tau) from every cell to the observer; Sect. 3.6.3:
// HEALPix output).  One thread per leaf; a leaf that subtends more than one
// map pixel (or holds the observer) is split into octants, at most max_sub
// times, and each (sub)cell is projected as a point at its centre.
#pragma once

#include "device_common.cuh"

namespace dartray {

struct MapArgs {
    double obs[3];
    int nside_k;
    int max_sub;
    const float *jsca;  // total scattered luminosity per j_sca pixel, or null
    float *map;         // [nl][12 * 4^nside_k]
};

// Optical depth per wavelength from x to the observer along the straight line.
template <int NL>
__device__ inline void tau_to_observer(const DevGrid &G, const float3 x, const float3 o, float *tau) {
#pragma unroll
    for (int l = 0; l < NL; ++l) tau[l] = 0.f;
    float3 n = make_float3(o.x - x.x, o.y - x.y, o.z - x.z);
    const float dist = sqrtf(n.x * n.x + n.y * n.y + n.z * n.z);
    if (!(dist > 0.f)) return;
    n = make_float3(n.x / dist, n.y / dist, n.z / dist);
    int leaf = locate_root(G, 0, x, n);  // maps are made of single-model grids
    float d = 0.f;
    const float inf = __int_as_float(0x7f800000);
    for (int guard = 0; leaf >= 0 && guard < (1 << 22); ++guard) {
        const float4 b = __ldg(&G.leaf_box[leaf]);
        float bnd[3];
        bnd[0] = n.x > 0.f ? b.x + b.w : b.x;
        bnd[1] = n.y > 0.f ? b.y + b.w : b.y;
        bnd[2] = n.z > 0.f ? b.z + b.w : b.z;
        const float tx = n.x != 0.f ? (bnd[0] - x.x) / n.x : inf;
        const float ty = n.y != 0.f ? (bnd[1] - x.y) / n.y : inf;
        const float tz = n.z != 0.f ? (bnd[2] - x.z) / n.z : inf;
        const float te0 = fminf(tx, fminf(ty, tz));
        const int tie = (tx == te0 ? 1 : 0) | (ty == te0 ? 2 : 0) | (tz == te0 ? 4 : 0);
        if (tie == 0) break;
        const float te = fminf(te0, dist);
        if (te > d) {
#pragma unroll
            for (int l = 0; l < NL; ++l) tau[l] += __ldg(&G.kappa_rho[static_cast<long long>(leaf) * NL + l]) * (te - d);
        }
        if (te >= dist) break;
        d = te;
        const float3 pe = make_float3((tie & 1) ? bnd[0] : fminf(fmaxf(fmaf(te0, n.x, x.x), b.x), b.x + b.w),
                                      (tie & 2) ? bnd[1] : fminf(fmaxf(fmaf(te0, n.y, x.y), b.y), b.y + b.w),
                                      (tie & 4) ? bnd[2] : fminf(fmaxf(fmaf(te0, n.z, x.z), b.z), b.z + b.w));
        const int nxt = next_leaf(G, leaf, tie, pe, n);
        if (nxt == leaf) break;
        leaf = nxt;
    }
}

template <int NL>
__global__ void __launch_bounds__(256) map_kernel(const DevGrid G, const MapArgs M) {
    const int leaf = blockIdx.x * blockDim.x + threadIdx.x;
    if (leaf >= G.n_leaf) return;
    const long long npix = 12ll << (2 * M.nside_k);
    const double omega_pix = 4.0 * kPi / static_cast<double>(npix);
    const float4 lb = G.leaf_box[leaf];
    const double Lleaf = lb.w;
    const float3 of = make_float3(static_cast<float>(M.obs[0]), static_cast<float>(M.obs[1]),
                                  static_cast<float>(M.obs[2]));
    float S[NL];
    bool any = false;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        S[l] = G.emis[static_cast<long long>(leaf) * NL + l] * (lb.w * lb.w * lb.w);
        any = any || S[l] > 0.f;
    }
    if (!any && M.jsca == nullptr) return;
    // explicit stack of (sub)cubes: lo, side, depth
    float4 stk[6 * 7 + 1];
    int sdep[6 * 7 + 1];
    int sp = 0;
    stk[0] = lb;
    sdep[0] = 0;
    sp = 1;
    while (sp > 0) {
        --sp;
        const float4 b = stk[sp];
        const int depth = sdep[sp];
        const double s = b.w;
        const double xc[3] = {static_cast<double>(b.x) + 0.5 * s, static_cast<double>(b.y) + 0.5 * s,
                              static_cast<double>(b.z) + 0.5 * s};
        const double v[3] = {xc[0] - M.obs[0], xc[1] - M.obs[1], xc[2] - M.obs[2]};
        // uncontracted double arithmetic: the subdivision decision below is
        // taken exactly as a plain double evaluation would take it
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(v[0], v[0]), __dmul_rn(v[1], v[1])), __dmul_rn(v[2], v[2]));
        const bool inside = M.obs[0] >= b.x && M.obs[0] <= b.x + s && M.obs[1] >= b.y && M.obs[1] <= b.y + s &&
                            M.obs[2] >= b.z && M.obs[2] <= b.z + s;
        if (depth < M.max_sub && (inside || __dmul_rn(s, s) > __dmul_rn(omega_pix, r2))) {
            const float h = 0.5f * b.w;
            for (int c = 0; c < 8; ++c) {
                stk[sp] = make_float4(b.x + ((c & 1) ? h : 0.f), b.y + ((c & 2) ? h : 0.f), b.z + ((c & 4) ? h : 0.f), h);
                sdep[sp] = depth + 1;
                ++sp;
            }
            continue;
        }
        if (sqrt(r2) <= 1e-6 * s) continue;
        const double frac = (s * s * s) / (Lleaf * Lleaf * Lleaf);
        const uint64_t mp = vec2pix_d(M.nside_k, v[0], v[1], v[2]);
        float I0[NL];
        bool nz = false;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            double i0 = S[l];
            if (M.jsca) {
                const int kl = G.k_lam[l];
                const int np = 12 << (2 * kl);
                const uint64_t q = vec2pix_d(kl, -v[0], -v[1], -v[2]);
                i0 += static_cast<double>(M.jsca[G.off_lam[l] + static_cast<long long>(leaf) * np + q]) /
                      (4.0 * kPi / np);
            }
            I0[l] = static_cast<float>(i0 * frac);
            nz = nz || I0[l] > 0.f;
        }
        if (!nz) continue;
        float tau[NL];
        tau_to_observer<NL>(G, make_float3(static_cast<float>(xc[0]), static_cast<float>(xc[1]),
                                           static_cast<float>(xc[2])), of, tau);
        const float w = static_cast<float>(1.0 / (r2 * omega_pix));
#pragma unroll
        for (int l = 0; l < NL; ++l)
            if (I0[l] > 0.f) atomicAdd(&M.map[l * npix + static_cast<long long>(mp)], I0[l] * expf(-tau[l]) * w);
    }
}

inline int launch_map(const DevGrid &G, const MapArgs &M, int blocks, cudaStream_t s) {
    switch (G.nl) {
    case 1: map_kernel<1><<<blocks, 256, 0, s>>>(G, M); return 0;
    case 2: map_kernel<2><<<blocks, 256, 0, s>>>(G, M); return 0;
    case 4: map_kernel<4><<<blocks, 256, 0, s>>>(G, M); return 0;
    case 8: map_kernel<8><<<blocks, 256, 0, s>>>(G, M); return 0;
    case 16: map_kernel<16><<<blocks, 256, 0, s>>>(G, M); return 0;
    default: return 1;
    }
}

}  // namespace dartray

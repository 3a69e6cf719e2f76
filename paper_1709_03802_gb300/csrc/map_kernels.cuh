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

namespace dartray {

// ---------------------------------------------------------- external maps
// Orthographic surface-brightness map for an observer far away along the
// unit vector `view` (from the model toward the observer): one line of sight
// per pixel, parallel to -view, through the pixel centre
// origin + (i + 1/2) px right + (j + 1/2) px up of the image plane (right =
// up x view).  Along it the model is integrated front to back (Sect. 2,
// end: I_obs = I_0 e^-tau, the cells as a continuous medium -- the volume
// rendering of the paper): a cell crossed over ds with extinction kr and
// source eta (luminosity per volume per sr toward the observer: the stellar
// emissivity plus the total scattered luminosity of the j_sca pixel that
// holds `view`, per its solid angle, per volume) adds
//   E = eta (1 - e^{-kr ds}) / kr     (eta ds for kr = 0)
// times the transmission T_front of the cells in front of it.
// The vector-Jacobian product of the map with respect to kr (the source
// held fixed) recomputes the transmission along each line of sight instead
// of storing it: a first pass gives the pixel's SB, a second the prefix P
// of the contributions, and
//   dSB/dkr_c = T_front dE/dkr - ds (SB - P_including_c).
struct ExtMapArgs {
    double view[3], right[3], up[3], origin[2], px;
    int nx, ny;
    double box_lo[3], box_hi[3];  // the root lattice
    const float *jsca;            // total j_sca, or null
    float *map;                   // [nl][ny][nx] (forward)
    const float *dmap;            // [nl][ny][nx] upstream gradient (VJP)
    float *grad;                  // [n_leaf][nl] (VJP), accumulated
    double *grad_sca;             // [nl] (VJP): sum of dmap times the scattered part of the map
    const float *dg;              // [n_leaf][nl] d j_sca(view pixel) / d g, or null (VJP)
    double *grad_g;               // [nl] (VJP with dg): sum of dmap times d map / d g
};

// E and dE/dkr of a cell for x = kr ds (series below 1e-4, where the
// closed forms cancel)
__device__ inline void cell_emission(double eta, double kr, double ds, double *E, double *dE) {
    const double x = kr * ds;
    if (x < 1e-4) {
        *E = eta * ds * (1.0 - x * (0.5 - x / 6.0));
        *dE = eta * ds * ds * (-0.5 + x * (1.0 / 3.0 - x / 8.0));
    } else {
        const double omT = -expm1(-x);
        *E = eta * omT / kr;
        *dE = eta * (ds * (1.0 - omT) * kr - omT) / (kr * kr);
    }
}

template <int NL, bool VJP>
__global__ void __launch_bounds__(128) external_map_kernel(const DevGrid G, const ExtMapArgs M) {
    const int pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= M.nx * M.ny) return;
    const int i = pix % M.nx, j = pix / M.nx;
    const double u = M.origin[0] + (i + 0.5) * M.px, v = M.origin[1] + (j + 0.5) * M.px;
    // the line p0 + t d, d = -view, entering the root lattice at t0
    double p0[3], d[3];
    for (int a = 0; a < 3; ++a) {
        p0[a] = u * M.right[a] + v * M.up[a];
        d[a] = -M.view[a];
    }
    double t0 = -1e300, t1 = 1e300;
    for (int a = 0; a < 3; ++a) {
        if (d[a] != 0.0) {
            double ta = (M.box_lo[a] - p0[a]) / d[a], tb = (M.box_hi[a] - p0[a]) / d[a];
            if (ta > tb) { const double t = ta; ta = tb; tb = t; }
            t0 = fmax(t0, ta);
            t1 = fmin(t1, tb);
        } else if (p0[a] < M.box_lo[a] || p0[a] >= M.box_hi[a]) {
            t1 = -1e300;
        }
    }
    const long long npix = static_cast<long long>(M.nx) * M.ny;
    if (!(t1 > t0)) {
        if (!VJP)
            for (int l = 0; l < NL; ++l) M.map[l * npix + pix] = 0.f;
        return;
    }
    const float3 n = make_float3(static_cast<float>(d[0]), static_cast<float>(d[1]), static_cast<float>(d[2]));
    // the j_sca pixel holding the direction toward the observer, per wavelength
    int q[NL];
    double omq[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        const int kl = G.k_lam[l];
        q[l] = static_cast<int>(vec2pix_d(kl, M.view[0], M.view[1], M.view[2]));
        omq[l] = 4.0 * kPi / (12 << (2 * kl));
    }
    double SB[NL], P[NL], Tf[NL], g[NL], SBs[NL], SBg[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        SB[l] = 0.0;
        SBs[l] = 0.0;
        SBg[l] = 0.0;
        P[l] = 0.0;
        Tf[l] = 1.0;
        g[l] = VJP ? static_cast<double>(M.dmap[l * npix + pix]) : 0.0;
    }
    for (int pass = 0; pass < (VJP ? 2 : 1); ++pass) {
        // march front to back from the entry point (held inside the lattice:
        // rounding must not put it outside)
        float3 p;
        {
            double e[3];
            for (int a = 0; a < 3; ++a) e[a] = fmin(fmax(p0[a] + t0 * d[a], M.box_lo[a]), M.box_hi[a]);
            p = make_float3(static_cast<float>(e[0]), static_cast<float>(e[1]), static_cast<float>(e[2]));
        }
        int leaf = locate_root(G, 0, p, n);
        double t = t0;
        for (int guard = 0; leaf >= 0 && guard < (1 << 22); ++guard) {
            const float4 b = __ldg(&G.leaf_box[leaf]);
            // exit distance along the line (double, from the line's own origin)
            double te = 1e300;
            int tie = 0;
            double bnd[3];
            const double lo[3] = {b.x, b.y, b.z};
            for (int a = 0; a < 3; ++a) {
                bnd[a] = d[a] > 0 ? lo[a] + b.w : lo[a];
                if (d[a] != 0.0) {
                    const double ta = (bnd[a] - p0[a]) / d[a];
                    if (ta < te) { te = ta; tie = 1 << a; }
                    else if (ta == te) tie |= 1 << a;
                }
            }
            const double ds = fmax(te - t, 0.0);
            const double V = static_cast<double>(b.w) * b.w * b.w;
#pragma unroll
            for (int l = 0; l < NL; ++l) {
                const double kr = __ldg(&G.kappa_rho[static_cast<long long>(leaf) * NL + l]);
                double eta = __ldg(&G.emis[static_cast<long long>(leaf) * NL + l]), eta_s = 0.0;
                if (M.jsca) {
                    const int np = 12 << (2 * G.k_lam[l]);
                    eta_s = static_cast<double>(M.jsca[G.off_lam[l] + static_cast<long long>(leaf) * np + q[l]]) /
                            (omq[l] * V);
                    eta += eta_s;
                }
                double E, dE;
                cell_emission(eta, kr, ds, &E, &dE);
                const double contrib = E * Tf[l];
                if (pass == 0) {
                    SB[l] += contrib;
                    if (VJP && eta > 0.0) SBs[l] += contrib * (eta_s / eta);  // E is linear in eta
                    if (VJP && M.dg) {
                        double E1, dE1;
                        cell_emission(1.0, kr, ds, &E1, &dE1);
                        SBg[l] += Tf[l] * E1 * static_cast<double>(__ldg(&M.dg[static_cast<long long>(leaf) * NL + l])) /
                                  (omq[l] * V);
                    }
                } else {
                    P[l] += contrib;
                    const double dSB = Tf[l] * dE - ds * (SB[l] - P[l]);
                    const double gv = g[l] * dSB;
                    if (gv != 0.0) atomicAdd(&M.grad[static_cast<long long>(leaf) * NL + l], static_cast<float>(gv));
                }
                Tf[l] *= exp(-kr * ds);
            }
            if (tie == 0 || te >= t1) break;
            t = te;
            // the exit point: on the faces reached exactly, elsewhere on the
            // closed box of the cell being left
            double e[3];
            for (int a = 0; a < 3; ++a)
                e[a] = ((tie >> a) & 1) ? bnd[a] : fmin(fmax(p0[a] + te * d[a], lo[a]), lo[a] + b.w);
            const float3 pf = make_float3(static_cast<float>(e[0]), static_cast<float>(e[1]), static_cast<float>(e[2]));
            const int nxt = next_leaf(G, leaf, tie, pf, n);
            if (nxt == leaf) break;
            leaf = nxt;
        }
        if (pass == 0 && !VJP)
#pragma unroll
            for (int l = 0; l < NL; ++l) M.map[l * npix + pix] = static_cast<float>(SB[l]);
        if (pass == 0 && VJP && M.grad_sca)
#pragma unroll
            for (int l = 0; l < NL; ++l) {
                if (g[l] * SBs[l] != 0.0) atomicAdd(&M.grad_sca[l], g[l] * SBs[l]);
                if (M.grad_g && g[l] * SBg[l] != 0.0) atomicAdd(&M.grad_g[l], g[l] * SBg[l]);
            }
#pragma unroll
        for (int l = 0; l < NL; ++l) Tf[l] = 1.0;
    }
}

inline int launch_external_map(const DevGrid &G, const ExtMapArgs &M, bool vjp, cudaStream_t s) {
    const int blocks = (M.nx * M.ny + 127) / 128;
#define EXT(NLV)                                                                    \
    do {                                                                            \
        if (vjp) external_map_kernel<NLV, true><<<blocks, 128, 0, s>>>(G, M);       \
        else external_map_kernel<NLV, false><<<blocks, 128, 0, s>>>(G, M);          \
    } while (0)
    switch (G.nl) {
    case 1: EXT(1); return 0;
    case 2: EXT(2); return 0;
    case 4: EXT(4); return 0;
    case 8: EXT(8); return 0;
    case 16: EXT(16); return 0;
    default: return 1;
    }
#undef EXT
}

}  // namespace dartray

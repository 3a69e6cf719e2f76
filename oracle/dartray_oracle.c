/*
 * dartray_oracle.c -- plain, slow FP64 CPU oracle of the DART-Ray V2
 * ray-propagation sweep (Natale et al. 2017, "Ray-tracing 3D dust radiative
 * transfer with DART-Ray: code upgrade and public release").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py load this library.  It shares no code, header,
 * table or constant with the CUDA library (paper_1709_03802_gb300/csrc) and
 * neither includes nor links the other.
 *
 * It follows the paper's algorithm step by step, with no blocking, fusion or
 * reordering:
 *   Sect. 2           three steps per source: U_LL pre-pass (radius R_pre),
 *                     direct light with ray blocking (Eq. 1), scattering
 *                     iterations stopped at a fraction f_L of the step-2
 *                     scattered luminosity; U_LL <- U after step 2 and after
 *                     every iteration (footnote of Sect. 2).
 *   Sect. 3.1.1       HEALPix ray directions, split when the beam is too large
 *                     (Eq. 2) and the ray still significant, merge when it is
 *                     too small (Eq. 3); high/low lists, children restart at
 *                     the parent's distance, merged rays at the mean distance
 *                     with the mean intensity (Fig. 1).
 *   Sect. 3.1.2       scattering source function on HEALPix(k_lambda) with the
 *                     Henyey-Greenstein phase function (Eq. 4) and k from Eq. 5.
 *   Sect. 3.2         multi-wavelength rays: negligible wavelengths are still
 *                     propagated but deposit nothing.
 *   Sect. 3.5         delta U (the definition below Eq. 6) and f_U = 4 a_RT/N_s
 *                     (Eq. 10).
 *   Sect. 2 (end), 3.6.3  maps for an observer inside the model:
 *                     I_obs = I_0 exp(-tau).
 *   Sect. 3.6.4       the 2D (octant) mode for mirror-symmetric models.
 * Beyond the paper's sweep, for checking the library's derivatives: the
 * derivative with respect to g of the j_sca pixel toward a distant observer
 * (a tally at every deposit), and a forward mode in which extra wavelengths
 * carry the derivative of U with respect to the albedo.
 * Readings of passages the paper leaves open are marked "reading".
 *
 * HEALPix is written from its published definition (Gorski et al. 2005): 12
 * base pixels, rings of constant z, nested (bit-interleaved) indices.
 *
 * Every floating-point quantity is double.  Parity of each function is pinned
 * by tests/test_oracle_*.py against closed forms, brute force, invariants and
 * full recomputations of split trees, merge waves (on a uniform grid and on
 * one where the end of a resumed ray's suppression decides merges), blocking
 * decisions, scattering directions and maps; the multi-wavelength branch
 * (per-wavelength Eq. 1, skipped wavelengths, j_sca blocks per k_lambda,
 * scattering rays from the largest k_lambda) and point sources by
 * recomputations too.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXL 16
#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------ types */
typedef struct {
    int32_t nroot[3];
    double root_lo[3];
    double root_size;
    int32_t n_nodes, n_leaf, n_lambda;
    const int32_t *first_child;  /* [n_nodes], -1 = leaf, children bx+2by+4bz */
    const int32_t *leaf_of_node; /* [n_nodes] */
    const double *kappa_rho;     /* [n_leaf][n_lambda] extinction per length */
    const double *emis;          /* [n_leaf][n_lambda] luminosity/volume/sr */
    const double *albedo, *g;    /* [n_lambda] */
    int32_t n_point;
    const double *point_xyz;     /* [n_point][3] */
    const double *point_lum;     /* [n_point][n_lambda] total luminosity */
} or_grid;

typedef struct {
    double a_rt;        /* accuracy parameter (Sect. 3.5) */
    double r_pre;       /* step-1 radius (Sect. 2) */
    double f_l;         /* scattering stop fraction (Sect. 2) */
    double c_light;     /* light speed in model units */
    int32_t n_rays_min; /* N_rays of Eq. 2 */
    int32_t n_rays_max; /* N_rays^max of Eq. 3 */
    int32_t k0;         /* initial HEALPix level of the rays */
    int32_t k_ray_max;  /* highest ray level */
    int32_t k_sca_cap;  /* cap on k_lambda,HP (Sect. 3.1.2) */
    int32_t n_fwhm;     /* n_FWHM of Sect. 3.1.2 */
    int32_t merge;      /* 1: apply Eq. 3 merging */
    int32_t max_cross;  /* crossing cap per ray (error if hit) */
    int32_t max_waves;  /* wave cap per source (error if hit) */
    int32_t src_stride, src_offset; /* process sources with index % stride == offset */
    int32_t octant;     /* 1: octant mode of Sect. 3.6.4 (symmetric models) */
    int32_t tangent;    /* n > 0: wavelengths [n, 2n) carry the derivative of [0, n) with
                         * respect to their albedo (forward mode, decisions of the
                         * wavelengths [0, n) frozen); 0: off */
} or_params;

/* ledger slots per wavelength */
enum { LG_EMITTED = 0, LG_ABSORBED, LG_SCATTERED, LG_ESCAPED, LG_BLOCKED, LG_CUT, LG_SKIPPED, LG_N };
/* integer counters */
enum { CT_RAYS = 0, CT_CROSS, CT_SPLIT, CT_MERGE, CT_BLOCK, CT_ESCAPE, CT_CUT, CT_LOW, CT_RESUME,
       CT_WAVES, CT_SOURCES, CT_N };

typedef struct {
    int32_t k_lam[OR_MAXL];   /* j_sca HEALPix level per wavelength */
    int64_t off_lam[OR_MAXL]; /* offset of wavelength block in the j_sca arrays */
    int64_t sca_len;          /* total j_sca length */
    double *U;                /* [n_leaf][nl]  RFED (times c when c_light = 1) */
    double *U_LL;             /* [n_leaf][nl]  lower limit */
    double *pend_a, *pend_b;  /* [sca_len] pending scattered luminosity (double buffer) */
    int32_t cur_is_a;         /* which of pend_a/pend_b is "current" */
    double *jsca_total;       /* [sca_len] total scattered luminosity per pixel */
    double ledger[OR_MAXL][LG_N];
    int64_t counters[CT_N];
    double L_sca2;            /* total scattered luminosity at the end of step 2 */
    double f_u;               /* f_U of the last phase */
    int32_t n_src;            /* N_s of the last phase */
    /* optional: d/dg_l of the total j_sca pixel holding dg_view, per cell,
     * with the deposited luminosities held fixed ([n_leaf][nl]; dg_on = 1) */
    double *dg;
    double dg_view[3];
    int32_t dg_on;
} or_state;

/* ------------------------------------------------------------------ HEALPix */
/* Base-pixel layout: for face f, ring index (from the north pole) of a pixel
 * (ix, iy) is OR_FACE_ROW[f]*nside - ix - iy - 1, and the longitude of the
 * face centre is OR_FACE_LON[f] * pi/4 (faces 0-3 north, 4-7 equator, 8-11
 * south). */
static const int OR_FACE_ROW[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
static const int OR_FACE_LON[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};

static void or_deinterleave(int64_t q, int k, int64_t *ix, int64_t *iy) {
    int64_t x = 0, y = 0;
    for (int b = 0; b < k; ++b) {
        x |= ((q >> (2 * b)) & 1) << b;
        y |= ((q >> (2 * b + 1)) & 1) << b;
    }
    *ix = x;
    *iy = y;
}

static int64_t or_interleave(int64_t ix, int64_t iy, int k) {
    int64_t q = 0;
    for (int b = 0; b < k; ++b) {
        q |= ((ix >> b) & 1) << (2 * b);
        q |= ((iy >> b) & 1) << (2 * b + 1);
    }
    return q;
}

/* Centre of nested pixel p at level k (nside = 2^k), as a unit vector.
 * Gorski et al. 2005: polar-cap ring i (i < nside) at z = 1 - i^2/(3 nside^2)
 * with 4i pixels at phi = (pi/2i)(j - 1/2); equatorial ring i at
 * z = (4/3) - 2i/(3 nside) with 4 nside pixels at phi = (pi/2nside)(j - s/2).
 * The longitude is formed as (pi/2)*num/den with integers num, den and the
 * quadrant/octant symmetry applied exactly, so that the direction set is
 * exactly invariant under x<->y, x->-x, y->-y and z->-z in floating point. */
void or_pix2vec(int k, int64_t p, double v[3]) {
    const int64_t ns = (int64_t)1 << k, npf = ns * ns;
    const int face = (int)(p / npf);
    int64_t ix, iy;
    or_deinterleave(p % npf, k, &ix, &iy);
    const int64_t jr = OR_FACE_ROW[face] * ns - ix - iy - 1; /* ring 1..4ns-1 from north */
    int64_t nr;
    int shift, south = 0;
    double z, one_minus_z;
    if (jr < ns) {
        nr = jr;
        one_minus_z = (double)(nr * nr) / (3.0 * (double)(ns * ns));
        z = 1.0 - one_minus_z;
        shift = 0;
    } else if (jr > 3 * ns) {
        nr = 4 * ns - jr;
        one_minus_z = (double)(nr * nr) / (3.0 * (double)(ns * ns));
        z = 1.0 - one_minus_z;
        south = 1;
        shift = 0;
    } else {
        nr = ns;
        int64_t m = 2 * ns - jr;
        if (m < 0) { south = 1; m = -m; }
        z = (double)m * 2.0 / (3.0 * (double)ns);
        one_minus_z = 1.0 - z;
        shift = (int)((jr - ns) & 1);
    }
    int64_t jp = (OR_FACE_LON[face] * nr + ix - iy + 1 + shift) / 2;
    if (jp > 4 * nr) jp -= 4 * nr;
    if (jp < 1) jp += 4 * nr;
    /* phi / (pi/2) = (2 jp - shift - 1) / (2 nr) */
    const int64_t num = 2 * jp - shift - 1, den = 2 * nr;
    const int64_t quad = num / den, r = num % den;
    double c, s;
    if (2 * r == den) {
        c = s = sqrt(0.5);
    } else if (2 * r < den) {
        const double a = 0.5 * OR_PI * (double)r / (double)den;
        c = cos(a);
        s = sin(a);
    } else {
        const double a = 0.5 * OR_PI * (double)(den - r) / (double)den;
        c = sin(a);
        s = cos(a);
    }
    double x, y;
    switch ((int)(quad & 3)) {
    case 0: x = c; y = s; break;
    case 1: x = -s; y = c; break;
    case 2: x = -c; y = -s; break;
    default: x = s; y = -c; break;
    }
    const double st = sqrt(one_minus_z * (1.0 + z));
    v[0] = st * x;
    v[1] = st * y;
    v[2] = south ? -z : z;
}

/* Nested pixel at level k containing direction v (need not be normalised).
 * Equatorial zone (|z| <= 2/3): pixel edges are the lines
 * nside*(phi/(pi/2) + 1/2 -+ 3z/4) = integer; polar caps: edges are
 * nside*sqrt(3(1-|z|))*{t, 1-t} = integer, t the position within the
 * quadrant (Gorski et al. 2005). */
int64_t or_vec2pix(int k, const double v[3]) {
    const int64_t ns = (int64_t)1 << k;
    const double rxy2 = v[0] * v[0] + v[1] * v[1];
    const double len = sqrt(rxy2 + v[2] * v[2]);
    const double z = v[2] / len, za = fabs(z);
    double phi = atan2(v[1], v[0]);
    if (phi < 0) phi += 2.0 * OR_PI;
    double tt = phi / (0.5 * OR_PI);
    if (tt >= 4.0) tt -= 4.0;
    int face;
    int64_t ix, iy;
    if (za <= 2.0 / 3.0) {
        const double t1 = (double)ns * (0.5 + tt), t2 = (double)ns * 0.75 * z;
        const int64_t jp = (int64_t)floor(t1 - t2), jm = (int64_t)floor(t1 + t2);
        const int64_t fp = jp >> k, fm = jm >> k;
        if (fp == fm) face = (int)((fp & 3) + 4);
        else if (fp < fm) face = (int)(fp & 3);
        else face = (int)((fm & 3) + 8);
        ix = jm & (ns - 1);
        iy = ns - (jp & (ns - 1)) - 1;
    } else {
        int q = (int)tt;
        if (q > 3) q = 3;
        const double tp = tt - q;
        const double one_minus_za = rxy2 / (len * (len + fabs(v[2])));
        const double w = (double)ns * sqrt(3.0 * one_minus_za);
        int64_t jp = (int64_t)(tp * w), jm = (int64_t)((1.0 - tp) * w);
        if (jp > ns - 1) jp = ns - 1;
        if (jm > ns - 1) jm = ns - 1;
        if (z > 0) { face = q; ix = ns - jm - 1; iy = ns - jp - 1; }
        else { face = q + 8; ix = jp; iy = jm; }
    }
    return (int64_t)face * ns * ns + or_interleave(ix, iy, k);
}

/* --------------------------------------------------------- phase function */
/* Henyey-Greenstein phase function, Eq. 4 (per steradian, integrates to 1). */
double or_hg(double g, double mu) {
    const double x = 1.0 + g * g - 2.0 * g * mu;
    return (1.0 - g * g) / (4.0 * OR_PI * x * sqrt(x));
}

/* d Phi / d g of the HG function above (quotient rule on (1 - g^2) x^(-3/2)
 * with dx/dg = 2g - 2mu). */
double or_hg_dg(double g, double mu) {
    const double x = 1.0 + g * g - 2.0 * g * mu;
    return (-2.0 * g * x - 1.5 * (1.0 - g * g) * (2.0 * g - 2.0 * mu)) / (4.0 * OR_PI * x * x * sqrt(x));
}

/* Eq. 5 before rounding.  theta_min = FWHM[Phi - Phi(pi)] / n_FWHM; the half
 * maximum of Phi - Phi(pi) is reached where Phi = (Phi(0) + Phi(pi))/2, i.e.
 * x^(-3/2) = ((1-g)^-3 + (1+g)^-3)/2 with x = 1 + g^2 - 2 g cos(theta).
 * Returns -1 for g == 0 (flat profile, no finite width). */
double or_k_hp_real(double g, int n_fwhm) {
    const double ga = fabs(g);
    if (ga < 1e-12) return -1.0;
    const double m = 0.5 * (pow(1.0 - ga, -3.0) + pow(1.0 + ga, -3.0));
    const double x = pow(m, -2.0 / 3.0);
    double mu = (1.0 + ga * ga - x) / (2.0 * ga);
    if (mu > 1.0) mu = 1.0;
    if (mu < -1.0) mu = -1.0;
    const double fwhm = 2.0 * acos(mu);
    const double th = fwhm / (double)n_fwhm;
    return 0.5 * log2(4.0 * OR_PI / (12.0 * th * th));
}

/* Reading: the integer part of Eq. 5, clamped to [0, cap] (Sect. 3.1.2). */
int or_k_hp(double g, int n_fwhm, int cap) {
    const double kr = or_k_hp_real(g, n_fwhm);
    int k = kr < 0 ? 0 : (int)floor(kr);
    if (k > cap) k = cap;
    return k;
}

/* -------------------------------------------------------------- geometry */
/* Leaf containing point p.  A point on a cell face belongs to the cell the
 * direction n leads into (for n_a >= 0 the upper cell, for n_a < 0 the lower
 * one).  Returns the leaf id and its box (lo[3], side), or -1 outside. */
int or_locate(const or_grid *G, const double p[3], const double n[3], double box[4]) {
    int64_t idx[3];
    double lo[3];
    const double S = G->root_size;
    for (int a = 0; a < 3; ++a) {
        /* first guess by division, then exact comparisons with the face
         * coordinates root_lo + i*S (the division may round across a face) */
        const double u = floor((p[a] - G->root_lo[a]) / S);
        if (!(u > -2.0)) return -1;  /* also rejects NaN */
        if (u > (double)G->nroot[a] + 1.0) return -1;
        int64_t i = (int64_t)u;
        for (int guard = 0; guard < 4; ++guard) {
            const double f = G->root_lo[a] + (double)i * S, h = G->root_lo[a] + (double)(i + 1) * S;
            if (p[a] < f || (p[a] == f && n[a] < 0)) --i;
            else if (p[a] > h || (p[a] == h && n[a] >= 0)) ++i;
            else break;
        }
        if (i < 0 || i >= G->nroot[a]) return -1;
        idx[a] = i;
        lo[a] = G->root_lo[a] + (double)i * S;
    }
    int64_t node = idx[0] + (int64_t)G->nroot[0] * (idx[1] + (int64_t)G->nroot[1] * idx[2]);
    double size = S;
    while (G->first_child[node] >= 0) {
        const double half = 0.5 * size;
        int oct = 0;
        for (int a = 0; a < 3; ++a) {
            const double mid = lo[a] + half;
            const int up = p[a] > mid || (p[a] == mid && n[a] >= 0);
            if (up) { lo[a] = mid; oct |= 1 << a; }
        }
        node = G->first_child[node] + oct;
        size = half;
    }
    if (box) { box[0] = lo[0]; box[1] = lo[1]; box[2] = lo[2]; box[3] = size; }
    return G->leaf_of_node[node];
}

/* Exit of the ray x(t) = xs + t n from box: returns t_exit, sets the axis
 * mask of faces reached at exactly t_exit and the exit point (exact on those
 * faces).  Reading: a ray that leaves through an edge or corner moves
 * diagonally into the cell beyond all faces it reaches simultaneously. */
static double or_exit(const double xs[3], const double n[3], const double box[4], int *tie,
                      double pe[3]) {
    double t[3], tmin = INFINITY;
    double bnd[3];
    for (int a = 0; a < 3; ++a) {
        if (n[a] > 0) { bnd[a] = box[a] + box[3]; t[a] = (bnd[a] - xs[a]) / n[a]; }
        else if (n[a] < 0) { bnd[a] = box[a]; t[a] = (bnd[a] - xs[a]) / n[a]; }
        else { bnd[a] = 0; t[a] = INFINITY; }
        if (t[a] < tmin) tmin = t[a];
    }
    int m = 0;
    for (int a = 0; a < 3; ++a) {
        if (t[a] == tmin) {
            m |= 1 << a;
            pe[a] = bnd[a];
        } else {
            /* the exit point lies on the closed box; rounding must not move it
             * outside (that could send the ray back into a cell behind it) */
            double v = xs[a] + tmin * n[a];
            if (v < box[a]) v = box[a];
            if (v > box[a] + box[3]) v = box[a] + box[3];
            pe[a] = v;
        }
    }
    *tie = m;
    return tmin;
}

/* Segments of the ray from distance d0 until it leaves the model.  For tests
 * of the traversal.  Returns the count (<= cap). */
int or_trace(const or_grid *G, const double xs[3], const double n[3], double d0, int cap,
             int32_t *leaf_out, double *tin_out, double *tout_out) {
    double p[3] = {xs[0] + d0 * n[0], xs[1] + d0 * n[1], xs[2] + d0 * n[2]};
    double box[4];
    int leaf = or_locate(G, p, n, box);
    double d = d0;
    int cnt = 0;
    while (leaf >= 0 && cnt < cap) {
        int tie;
        double pe[3];
        const double te = or_exit(xs, n, box, &tie, pe);
        leaf_out[cnt] = leaf;
        tin_out[cnt] = d;
        tout_out[cnt] = te > d ? te : d;
        ++cnt;
        d = te > d ? te : d;
        const int prev = leaf;
        leaf = or_locate(G, pe, n, box);
        if (leaf == prev) return -5;  /* no progress: inexact face coordinates */
    }
    return cnt;
}

/* ---------------------------------------------------------------- rays */
enum { RK_SEED = 0, RK_CHILD, RK_MERGED, RK_RESUMED };

typedef struct {
    int32_t lev;
    int64_t pix;
    double d;
    double I[OR_MAXL];   /* per-sr luminosity carried by the ray, per wavelength */
    int32_t kind;
    int32_t hint_leaf;   /* >= 0: start leaf known (resumed rays) */
    double hint_box[4];
    double supp_L;       /* merge test suppressed while the cell side equals this */
    /* filled when the ray enters the low list */
    int32_t plane_axis;
    double plane_coord;
} or_ray;

typedef struct {
    or_ray *v;
    int64_t n, cap;
} or_list;

static int or_push(or_list *L, const or_ray *r) {
    if (L->n == L->cap) {
        int64_t nc = L->cap ? 2 * L->cap : 1024;
        or_ray *nv = (or_ray *)realloc(L->v, (size_t)nc * sizeof(or_ray));
        if (!nv) return -1;
        L->v = nv;
        L->cap = nc;
    }
    L->v[L->n++] = *r;
    return 0;
}

typedef struct {
    const or_grid *G;
    const or_params *P;
    or_state *S;
    int mode;                 /* 0 LL, 1 DIRECT, 2 SCATTER */
    double *target;           /* U_LL (LL) or U */
    const double *pend_src;   /* SCATTER source pixels */
    double *pend_dst;         /* DIRECT/SCATTER scattered-luminosity deposit */
    double f_u;
    /* current source */
    double xs[3];
    int32_t src_leaf;         /* source cell (-1 for a point source) */
    /* j_sca pixel directions per wavelength level */
    double *pixdir[4];
    int nl;
    double wsrc;              /* octant mode: weight of the current source, else 1 */
} or_ctx;

/* Per-crossing deposit quantities (paper Sect. 2, Sect. 3.5; reading of the
 * per-intersection formulas deferred to NA14): for a segment of length ds
 * with optical depth dtau = kappa*rho*ds the beam's luminosity P = I*Omega_k
 * drops by P(1-exp(-dtau)); the segment-averaged intensity is
 * <I> = I (1-exp(-dtau))/dtau.  The RFED contribution is the beam's
 * luminosity times its path length averaged along the segment, divided by
 * V c:  dU = P ds <I>/I / (V c). */
static double or_seg_factor(double dtau) {
    return dtau > 0 ? -expm1(-dtau) / dtau : 1.0;
}

/* Trace one ray until it stops; appends to the high or low list. */
static int or_march(or_ctx *C, or_ray *ray, or_list *high, or_list *low) {
    const or_grid *G = C->G;
    const or_params *P = C->P;
    or_state *S = C->S;
    const int nl = C->nl;
    const double c = P->c_light;
    double n[3];
    or_pix2vec(ray->lev, ray->pix, n);
    const double omega_k = 4.0 * OR_PI / (12.0 * ldexp(1.0, 2 * ray->lev));
    /* the ray's beam solid angle carries the source weight (octant mode):
     * deposits and ledger entries scale with it, the tests below do not */
    const double omega_w = omega_k * C->wsrc;
    /* Eq. 2 / Eq. 3 compared as  4 pi N r^2  vs  12 4^k L^2  (both sides exact
     * or singly rounded; Omega_INT = L^2/r^2, reading). */
    const double split_c = 4.0 * OR_PI * (double)P->n_rays_min;
    const double merge_c = 4.0 * OR_PI * (double)P->n_rays_max;
    const double beam_units = 12.0 * ldexp(1.0, 2 * ray->lev);

    double box[4];
    int leaf;
    int start_axis = -1;      /* face the ray starts on, if any */
    double start_coord = 0;
    if (ray->hint_leaf >= 0) {
        leaf = ray->hint_leaf;
        memcpy(box, ray->hint_box, sizeof box);
    } else {
        double p[3] = {C->xs[0] + ray->d * n[0], C->xs[1] + ray->d * n[1], C->xs[2] + ray->d * n[2]};
        /* Children restart at the parent's distance d_ray (Sect. 3.1.1).  A
         * child whose direction has the same component as its parent along
         * the axis of the face the parent entered its last cell through lies,
         * in exact arithmetic, on that face at distance d_ray; the start point
         * is taken exactly there (reading: exact evaluation of the rule, so
         * that rounding does not decide the side of the face). */
        if (ray->kind == RK_CHILD && ray->plane_axis >= 0) {
            double np_[3];
            or_pix2vec(ray->lev - 1, ray->pix >> 2, np_);
            const int a = ray->plane_axis;
            if (n[a] == np_[a]) {
                p[a] = ray->plane_coord;
                start_axis = a;
                start_coord = ray->plane_coord;
            }
        }
        leaf = or_locate(G, p, n, box);
    }
    if (ray->kind == RK_RESUMED) {  /* resumes on the face it stopped at */
        start_axis = ray->plane_axis;
        start_coord = ray->plane_coord;
    }
    S->counters[CT_RAYS]++;
    /* HG normalisation for this ray direction (reading: rows normalised so
     * that the discrete phase function conserves the scattered luminosity). */
    double Z[OR_MAXL], Zg[OR_MAXL];
    if (C->mode != 0) {
        for (int l = 0; l < nl; ++l) {
            const int npx = 12 << (2 * S->k_lam[l]);
            const double *pd = C->pixdir[S->k_lam[l]];
            double z = 0, zg = 0;
            for (int q = 0; q < npx; ++q) {
                const double mu = pd[3 * q] * n[0] + pd[3 * q + 1] * n[1] + pd[3 * q + 2] * n[2];
                z += or_hg(G->g[l], mu);
                if (S->dg_on) zg += or_hg_dg(G->g[l], mu);
            }
            Z[l] = z;
            Zg[l] = zg;
        }
    }
    if (leaf < 0) {  /* starts outside the model */
        for (int l = 0; l < nl; ++l) S->ledger[l][LG_ESCAPED] += ray->I[l] * omega_w;
        S->counters[CT_ESCAPE]++;
        return 0;
    }
    double d = ray->d;
    int first = 1;
    int entry_axis = start_axis;  /* face through which the current cell was entered */
    double entry_coord = start_coord;
    int64_t ncross = 0;
    for (;;) {
        if (++ncross > P->max_cross) return -2;
        S->counters[CT_CROSS]++;
        int tie;
        double pe[3];
        const double te = or_exit(C->xs, n, box, &tie, pe);
        const double ds = te > d ? te - d : 0.0;
        const double L = box[3], V = L * L * L;
        const double xc[3] = {box[0] + 0.5 * L, box[1] + 0.5 * L, box[2] + 0.5 * L};
        const double r2 = (xc[0] - C->xs[0]) * (xc[0] - C->xs[0]) +
                          (xc[1] - C->xs[1]) * (xc[1] - C->xs[1]) +
                          (xc[2] - C->xs[2]) * (xc[2] - C->xs[2]);
        const int in_src = (leaf == C->src_leaf);
        const double P_in_unit = omega_w;  /* beam solid angle (times the source weight) */
        int neg[OR_MAXL] = {0};
        double fac[OR_MAXL], T[OR_MAXL];
        for (int l = 0; l < nl; ++l) {
            const double dtau = G->kappa_rho[(int64_t)leaf * nl + l] * ds;
            fac[l] = or_seg_factor(dtau);
            T[l] = exp(-dtau);
        }
        if (!in_src) {
            if (C->mode == 0) {
                /* step 1: the significance test is d_ray < R_pre (Fig. 1) */
                if (d >= P->r_pre) {
                    for (int l = 0; l < nl; ++l) S->ledger[l][LG_CUT] += ray->I[l] * omega_w;
                    S->counters[CT_CUT]++;
                    return 0;
                }
            } else {
                /* Eq. 1 with delta U = <I> A_EM Omega_INT L_INT / (V_INT c)
                 * (Sect. 3.5); I*A_EM is the ray's per-sr luminosity (reading),
                 * Omega_INT = L^2/r^2 (reading). */
                int all = 1;
                const int nd = P->tangent > 0 ? P->tangent : nl;  /* wavelengths that decide */
                for (int l = 0; l < nd; ++l) {
                    const double Iavg = ray->I[l] * fac[l];
                    const double omega_int = L * L / r2;
                    const double dU = Iavg * omega_int * L / (V * c);
                    neg[l] = dU < C->f_u * S->U_LL[(int64_t)leaf * nl + l];
                    all &= neg[l];
                }
                /* a derivative deposits where its wavelength does */
                for (int l = nd; l < nl; ++l) neg[l] = neg[l - nd];
                if (all) {
                    for (int l = 0; l < nl; ++l) S->ledger[l][LG_BLOCKED] += ray->I[l] * omega_w;
                    S->counters[CT_BLOCK]++;
                    return 0;
                }
            }
            /* Eq. 2: beam larger than Omega_INT / N_rays -> high list.
             * Reading: a merged ray's first segment is exempt (it may start a
             * little before the plane its siblings stopped at). */
            if (!(first && ray->kind == RK_MERGED) && ray->lev < P->k_ray_max &&
                split_c * r2 > beam_units * L * L) {
                or_ray h = *ray;
                h.d = d;
                h.plane_axis = entry_axis;
                h.plane_coord = entry_coord;
                if (or_push(high, &h)) return -1;
                S->counters[CT_SPLIT]++;
                return 0;
            }
            /* Eq. 3: beam smaller than Omega_INT / N_rays^max -> low list.
             * Reading: only on cells entered through a face, and not while a
             * resumed ray is still in cells of the size it stopped at. */
            if (P->merge && ray->lev > 0 && !first && L != ray->supp_L &&
                merge_c * r2 < beam_units * L * L) {
                or_ray lw = *ray;
                lw.d = d;
                lw.plane_axis = entry_axis;
                lw.plane_coord = entry_coord;
                lw.hint_leaf = leaf;
                memcpy(lw.hint_box, box, sizeof box);
                if (or_push(low, &lw)) return -1;
                S->counters[CT_LOW]++;
                return 0;
            }
        }
        /* deposits (Sect. 2; Sect. 3.2 for negligible wavelengths) */
        double I_in[OR_MAXL];  /* intensities entering the segment */
        for (int l = 0; l < nl; ++l) I_in[l] = ray->I[l];
        for (int l = 0; l < nl; ++l) {
            const double P_in = ray->I[l] * P_in_unit;
            const double kr = G->kappa_rho[(int64_t)leaf * nl + l];
            const double lost = P_in * kr * ds * fac[l];  /* P (1 - e^-dtau) */
            if (neg[l]) {
                S->ledger[l][LG_SKIPPED] += lost;
            } else {
                C->target[(int64_t)leaf * nl + l] += P_in * ds * fac[l] / (V * c);
                const double w = G->albedo[l];
                S->ledger[l][LG_ABSORBED] += (1.0 - w) * lost;
                S->ledger[l][LG_SCATTERED] += w * lost;
                if (C->mode != 0) {
                    /* d(w lost)/dw = w dlost/dw + lost for a derivative channel */
                    const double sca = P->tangent > 0 && l >= P->tangent
                                           ? w * lost + I_in[l - P->tangent] * P_in_unit * kr * ds * fac[l]
                                           : w * lost;
                    if (sca > 0) {
                        const int kl = S->k_lam[l];
                        const int npx = 12 << (2 * kl);
                        const double *pd = C->pixdir[kl];
                        double *row = C->pend_dst + S->off_lam[l] + (int64_t)leaf * npx;
                        for (int q = 0; q < npx; ++q) {
                            const double mu = pd[3 * q] * n[0] + pd[3 * q + 1] * n[1] + pd[3 * q + 2] * n[2];
                            row[q] += sca * or_hg(G->g[l], mu) / Z[l];
                        }
                        if (S->dg_on) {  /* d/dg of the weight Phi_q / Z of the view pixel */
                            const int64_t qv = or_vec2pix(kl, S->dg_view);
                            const double mu = pd[3 * qv] * n[0] + pd[3 * qv + 1] * n[1] + pd[3 * qv + 2] * n[2];
                            S->dg[(int64_t)leaf * nl + l] +=
                                sca * (or_hg_dg(G->g[l], mu) - or_hg(G->g[l], mu) * Zg[l] / Z[l]) / Z[l];
                        }
                    }
                }
            }
            ray->I[l] *= T[l];
        }
        /* advance to the next cell */
        d = te > d ? te : d;
        int ax = 0;
        while (!((tie >> ax) & 1)) ++ax;
        entry_axis = ax;
        entry_coord = pe[ax];
        const int prev = leaf;
        leaf = or_locate(G, pe, n, box);
        if (leaf == prev) return -5;  /* no progress: inexact face coordinates */
        if (leaf < 0) {
            for (int l = 0; l < nl; ++l) S->ledger[l][LG_ESCAPED] += ray->I[l] * omega_w;
            S->counters[CT_ESCAPE]++;
            return 0;
        }
        if (ray->supp_L != 0 && box[3] != ray->supp_L) ray->supp_L = 0;
        first = 0;
    }
}

static int or_cmp_low(const void *a, const void *b) {
    const or_ray *x = (const or_ray *)a, *y = (const or_ray *)b;
    if (x->lev != y->lev) return x->lev < y->lev ? -1 : 1;
    if (x->pix != y->pix) return x->pix < y->pix ? -1 : 1;
    return 0;
}

/* All waves of one source (Sect. 3.1.1, Fig. 1; reading: level-synchronous
 * waves -- every ray of a wave is traced, then the high list is split into
 * children that restart at the parent's distance, then groups of four
 * siblings of the low list that stopped on the same grid plane are merged;
 * rays that cannot merge resume where they stopped with the merge test
 * suppressed until the cell size changes). */
static int or_source(or_ctx *C, or_list *wave) {
    or_list high = {0}, low = {0}, next = {0};
    int rc = 0;
    int nw = 0;
    const int nl = C->nl;
    while (wave->n > 0) {
        if (++nw > C->P->max_waves) { rc = -3; break; }
        C->S->counters[CT_WAVES]++;
        high.n = low.n = next.n = 0;
        for (int64_t i = 0; i < wave->n; ++i) {
            rc = or_march(C, &wave->v[i], &high, &low);
            if (rc) goto done;
        }
        for (int64_t i = 0; i < high.n; ++i) {
            for (int c = 0; c < 4; ++c) {
                or_ray ch = high.v[i];
                ch.lev += 1;
                ch.pix = 4 * high.v[i].pix + c;
                ch.kind = RK_CHILD;
                ch.hint_leaf = -1;
                ch.supp_L = 0;
                if (or_push(&next, &ch)) { rc = -1; goto done; }
            }
        }
        if (low.n) qsort(low.v, (size_t)low.n, sizeof(or_ray), or_cmp_low);
        for (int64_t i = 0; i < low.n;) {
            int64_t j = i;
            while (j < low.n && low.v[j].lev == low.v[i].lev && (low.v[j].pix >> 2) == (low.v[i].pix >> 2)) ++j;
            int ok = (j - i == 4);
            for (int64_t m = i + 1; ok && m < j; ++m)
                ok = low.v[m].plane_axis == low.v[i].plane_axis && low.v[m].plane_coord == low.v[i].plane_coord;
            if (ok) {
                or_ray mr = low.v[i];
                mr.lev -= 1;
                mr.pix = low.v[i].pix >> 2;
                mr.d = 0;
                for (int l = 0; l < nl; ++l) mr.I[l] = 0;
                for (int64_t m = i; m < j; ++m) {
                    mr.d += low.v[m].d;
                    for (int l = 0; l < nl; ++l) mr.I[l] += low.v[m].I[l];
                }
                mr.d *= 0.25;
                for (int l = 0; l < nl; ++l) mr.I[l] *= 0.25;
                mr.kind = RK_MERGED;
                mr.hint_leaf = -1;
                mr.supp_L = 0;
                C->S->counters[CT_MERGE]++;
                if (or_push(&next, &mr)) { rc = -1; goto done; }
            } else {
                for (int64_t m = i; m < j; ++m) {
                    or_ray rr = low.v[m];
                    rr.kind = RK_RESUMED;
                    rr.supp_L = rr.hint_box[3];
                    C->S->counters[CT_RESUME]++;
                    if (or_push(&next, &rr)) { rc = -1; goto done; }
                }
            }
            i = j;
        }
        or_list t = *wave;
        *wave = next;
        next = t;
    }
done:
    free(high.v);
    free(low.v);
    free(next.v);
    return rc;
}

/* Boxes (lo[3], side) of all leaves, by one walk over the forest. */
static void or_leaf_boxes(const or_grid *G, double *out) {
    const int64_t nroots = (int64_t)G->nroot[0] * G->nroot[1] * G->nroot[2];
    int64_t *stack = (int64_t *)malloc(sizeof(int64_t) * 8 * 64);
    double *sb = (double *)malloc(sizeof(double) * 4 * 8 * 64);
    for (int64_t r = 0; r < nroots; ++r) {
        int sp = 0;
        stack[0] = r;
        sb[0] = G->root_lo[0] + (double)(r % G->nroot[0]) * G->root_size;
        sb[1] = G->root_lo[1] + (double)((r / G->nroot[0]) % G->nroot[1]) * G->root_size;
        sb[2] = G->root_lo[2] + (double)(r / ((int64_t)G->nroot[0] * G->nroot[1])) * G->root_size;
        sb[3] = G->root_size;
        sp = 1;
        while (sp > 0) {
            --sp;
            const int64_t nd = stack[sp];
            const double b[4] = {sb[4 * sp], sb[4 * sp + 1], sb[4 * sp + 2], sb[4 * sp + 3]};
            if (G->first_child[nd] < 0) {
                memcpy(out + 4 * (int64_t)G->leaf_of_node[nd], b, sizeof b);
                continue;
            }
            const double h = 0.5 * b[3];
            for (int c = 0; c < 8; ++c) {
                stack[sp] = G->first_child[nd] + c;
                sb[4 * sp] = b[0] + ((c & 1) ? h : 0);
                sb[4 * sp + 1] = b[1] + ((c & 2) ? h : 0);
                sb[4 * sp + 2] = b[2] + ((c & 4) ? h : 0);
                sb[4 * sp + 3] = h;
                ++sp;
            }
        }
    }
    free(stack);
    free(sb);
}

/* Octant mode (Sect. 3.6.4): a model symmetric under the reflections about
 * the planes through the centre of its root lattice is traced from the
 * sources of the first octant only; the field of a source's image is the
 * image of the source's field, so every cell receives the deposits of the
 * images of itself.  mirror[(m-1) n_leaf + c] is the image of leaf c under
 * reflection mask m (bit a: axis a flipped), mpix[m-1][k][q] the image of
 * pixel q of level k.  Returns -6 if the grid is not symmetric. */
static int or_mirrors(const or_grid *G, const double *leaf_box, const double centre[3], int32_t *mirror,
                      int32_t mpix[7][4][768]) {
    for (int m = 1; m < 8; ++m) {
        for (int64_t c = 0; c < G->n_leaf; ++c) {
            const double *b = leaf_box + 4 * c;
            double q[3];
            for (int a = 0; a < 3; ++a) {
                const double mid = b[a] + 0.5 * b[3];
                q[a] = ((m >> a) & 1) ? 2.0 * centre[a] - mid : mid;
            }
            const double up[3] = {1, 1, 1};
            double box[4];
            const int img = or_locate(G, q, up, box);
            if (img < 0 || box[3] != b[3]) return -6;
            for (int l = 0; l < G->n_lambda; ++l)
                if (G->kappa_rho[c * G->n_lambda + l] != G->kappa_rho[(int64_t)img * G->n_lambda + l] ||
                    G->emis[c * G->n_lambda + l] != G->emis[(int64_t)img * G->n_lambda + l])
                    return -6;
            mirror[(int64_t)(m - 1) * G->n_leaf + c] = img;
        }
        for (int k = 0; k < 4; ++k)
            for (int q = 0; q < (12 << (2 * k)); ++q) {
                double v[3];
                or_pix2vec(k, q, v);
                for (int a = 0; a < 3; ++a)
                    if ((m >> a) & 1) v[a] = -v[a];
                mpix[m - 1][k][q] = (int32_t)or_vec2pix(k, v);
            }
    }
    return 0;
}

/* One phase of the sweep: mode 0 = step 1 (U_LL), 1 = step 2 (direct light),
 * 2 = one scattering iteration.  keep_U (step 2 only): U starts from its
 * current value instead of zero (the dust self-heating iterations of
 * Sect. 3.3 process only the change of the dust emission).  Returns 0 or a
 * negative error. */
static int or_phase(const or_grid *G, const or_params *P, or_state *S, int mode, int keep_U) {
    if (P->octant && S->dg_on) return -7;  /* the g tally is not folded over mirror images */
    if (P->tangent > 0 && (P->octant || 2 * P->tangent != G->n_lambda)) return -8;
    const int nl = G->n_lambda;
    or_ctx C;
    memset(&C, 0, sizeof C);
    C.G = G;
    C.P = P;
    C.S = S;
    C.mode = mode;
    C.nl = nl;
    double *pend_cur = S->cur_is_a ? S->pend_a : S->pend_b;
    double *pend_nxt = S->cur_is_a ? S->pend_b : S->pend_a;
    if (mode == 2) {
        /* swap: what was deposited last phase is processed now */
        double *t = pend_cur; pend_cur = pend_nxt; pend_nxt = t;
        S->cur_is_a = !S->cur_is_a;
    }
    memset(S->ledger, 0, sizeof S->ledger);  /* the ledger describes the last phase */
    if (mode == 0) {
        memset(S->U_LL, 0, sizeof(double) * (size_t)G->n_leaf * nl);
        C.target = S->U_LL;
    } else {
        if (mode == 1 && !keep_U) memset(S->U, 0, sizeof(double) * (size_t)G->n_leaf * nl);
        C.target = S->U;
        memset(pend_nxt, 0, sizeof(double) * (size_t)S->sca_len);
        C.pend_dst = pend_nxt;
        C.pend_src = pend_cur;
    }
    for (int k = 0; k < 4; ++k) {
        const int npx = 12 << (2 * k);
        C.pixdir[k] = (double *)malloc(sizeof(double) * 3 * (size_t)npx);
        for (int q = 0; q < npx; ++q) or_pix2vec(k, q, C.pixdir[k] + 3 * q);
    }
    int kmax_lam = 0;
    for (int l = 0; l < nl; ++l) if (S->k_lam[l] > kmax_lam) kmax_lam = S->k_lam[l];
    const int kstart = mode == 2 ? (P->k0 > kmax_lam ? P->k0 : kmax_lam) : P->k0;

    /* N_s: sources of this phase (reading: emitting cells + point sources for
     * steps 1-2, cells holding scattered luminosity for an iteration) */
    const int64_t nsrc_all = mode == 2 ? G->n_leaf : (int64_t)G->n_leaf + G->n_point;
    char *is_src = (char *)calloc((size_t)nsrc_all, 1);
    double *leaf_box = (double *)malloc(sizeof(double) * 4 * (size_t)G->n_leaf);
    or_leaf_boxes(G, leaf_box);
    double centre[3];
    for (int a = 0; a < 3; ++a) centre[a] = G->root_lo[a] + 0.5 * G->nroot[a] * G->root_size;
    int64_t ns = 0;
    const int nd = P->tangent > 0 ? P->tangent : nl;  /* derivatives do not make sources */
    for (int64_t s = 0; s < nsrc_all; ++s) {
        int on = 0;
        if (s < G->n_leaf) {
            for (int l = 0; l < nd && !on; ++l) {
                if (mode == 2) {
                    const int npx = 12 << (2 * S->k_lam[l]);
                    const double *row = pend_cur + S->off_lam[l] + s * npx;
                    for (int q = 0; q < npx; ++q) if (row[q] > 0) { on = 1; break; }
                } else {
                    on = G->emis[s * nl + l] > 0;
                }
            }
        } else {
            for (int l = 0; l < nd; ++l) on |= G->point_lum[(s - G->n_leaf) * nl + l] > 0;
        }
        if (on && (s % P->src_stride) == P->src_offset) {
            ++ns;  /* N_s counts every source of the model */
            if (P->octant) {
                /* octant mode: sources of the first octant (closed) only */
                double x[3];
                for (int a = 0; a < 3; ++a)
                    x[a] = s < G->n_leaf ? leaf_box[4 * s + a] + 0.5 * leaf_box[4 * s + 3]
                                         : G->point_xyz[3 * (s - G->n_leaf) + a];
                on = x[0] >= centre[0] && x[1] >= centre[1] && x[2] >= centre[2];
            }
            is_src[s] = (char)on;
        }
    }
    S->n_src = (int32_t)ns;
    C.f_u = ns > 0 ? 4.0 * P->a_rt / (double)ns : 0.0;  /* Eq. 10 */
    S->f_u = C.f_u;
    /* octant mode: deposits of the traced sources go to scratch arrays and
     * are folded over the eight images of every cell at the end */
    double *dep_U = NULL, *dep_P = NULL, *final_target = C.target, *final_pend = C.pend_dst;
    int32_t *mirror = NULL;
    static int32_t mpix[7][4][768];
    if (P->octant) {
        mirror = (int32_t *)malloc(sizeof(int32_t) * 7 * (size_t)G->n_leaf);
        if (or_mirrors(G, leaf_box, centre, mirror, mpix)) {
            free(mirror);
            free(is_src);
            free(leaf_box);
            for (int k = 0; k < 4; ++k) free(C.pixdir[k]);
            return -6;
        }
        dep_U = (double *)calloc((size_t)G->n_leaf * nl, sizeof(double));
        C.target = dep_U;
        if (mode != 0) {
            dep_P = (double *)calloc((size_t)S->sca_len, sizeof(double));
            C.pend_dst = dep_P;
        }
    }
    int rc = 0;
    or_list wave = {0};
    const double omega0 = 4.0 * OR_PI / (12.0 * ldexp(1.0, 2 * kstart));
    for (int64_t s = 0; s < nsrc_all && !rc; ++s) {
        if (!is_src[s]) continue;
        S->counters[CT_SOURCES]++;
        double box[4];
        {
            /* weight 1/2^k of a source on k mirror planes (it is its own image
             * under 2^k of the eight reflections); 1 outside the octant mode */
            double x[3];
            for (int a = 0; a < 3; ++a)
                x[a] = s < G->n_leaf ? leaf_box[4 * s + a] + 0.5 * leaf_box[4 * s + 3]
                                     : G->point_xyz[3 * (s - G->n_leaf) + a];
            int k = 0;
            if (P->octant)
                for (int a = 0; a < 3; ++a) k += x[a] == centre[a];
            C.wsrc = ldexp(1.0, -k);
        }
        if (s < G->n_leaf) {
            memcpy(box, leaf_box + 4 * s, sizeof box);
            C.xs[0] = box[0] + 0.5 * box[3];
            C.xs[1] = box[1] + 0.5 * box[3];
            C.xs[2] = box[2] + 0.5 * box[3];
            C.src_leaf = (int32_t)s;
        } else {
            const int64_t ip = s - G->n_leaf;
            C.xs[0] = G->point_xyz[3 * ip];
            C.xs[1] = G->point_xyz[3 * ip + 1];
            C.xs[2] = G->point_xyz[3 * ip + 2];
            const double up[3] = {1, 1, 1};
            C.src_leaf = or_locate(G, C.xs, up, box);
        }
        /* seeds: every pixel of level kstart, d = 0 */
        wave.n = 0;
        const int64_t npix0 = 12LL << (2 * kstart);
        for (int64_t p = 0; p < npix0; ++p) {
            or_ray r;
            memset(&r, 0, sizeof r);
            r.lev = kstart;
            r.pix = p;
            r.d = 0;
            r.kind = RK_SEED;
            r.hint_leaf = -1;
            r.plane_axis = -1;
            for (int l = 0; l < nl; ++l) {
                double Il;
                if (mode == 2) {
                    /* per-sr scattered luminosity of the j_sca pixel that
                     * contains this ray's direction (nested parent) */
                    const int kl = S->k_lam[l];
                    const int npx = 12 << (2 * kl);
                    const int64_t q = p >> (2 * (kstart - kl));
                    Il = pend_cur[S->off_lam[l] + s * npx + q] / (4.0 * OR_PI / (double)npx);
                } else if (s < G->n_leaf) {
                    /* per-sr luminosity of an emitting cell: j V */
                    Il = G->emis[s * nl + l] * box[3] * box[3] * box[3];
                } else {
                    Il = G->point_lum[(s - G->n_leaf) * nl + l] / (4.0 * OR_PI);
                }
                r.I[l] = Il;
                S->ledger[l][LG_EMITTED] += Il * omega0 * C.wsrc;
            }
            if (or_push(&wave, &r)) { rc = -1; break; }
        }
        if (!rc) rc = or_source(&C, &wave);
    }
    free(wave.v);
    free(is_src);
    free(leaf_box);
    for (int k = 0; k < 4; ++k) free(C.pixdir[k]);
    if (P->octant) {
        if (!rc) {
            /* fold: every cell (and j_sca pixel) receives the deposits of its
             * images; the ledger describes the whole model */
            for (int64_t c = 0; c < G->n_leaf; ++c)
                for (int l = 0; l < nl; ++l) {
                    double v = dep_U[c * nl + l];
                    for (int m = 1; m < 8; ++m) v += dep_U[(int64_t)mirror[(int64_t)(m - 1) * G->n_leaf + c] * nl + l];
                    final_target[c * nl + l] += v;
                }
            if (mode != 0)
                for (int l = 0; l < nl; ++l) {
                    const int kl = S->k_lam[l], npx = 12 << (2 * kl);
                    for (int64_t c = 0; c < G->n_leaf; ++c)
                        for (int q = 0; q < npx; ++q) {
                            double v = dep_P[S->off_lam[l] + c * npx + q];
                            for (int m = 1; m < 8; ++m) {
                                const int64_t cm = mirror[(int64_t)(m - 1) * G->n_leaf + c];
                                v += dep_P[S->off_lam[l] + cm * npx + mpix[m - 1][kl][q]];
                            }
                            final_pend[S->off_lam[l] + c * npx + q] = v;
                        }
                }
            for (int l = 0; l < nl; ++l)
                for (int i = 0; i < LG_N; ++i) S->ledger[l][i] *= 8.0;
        }
        free(dep_U);
        free(dep_P);
        free(mirror);
    }
    if (rc) return rc;
    if (mode >= 1) {
        double tot = 0;  /* L_sca,2 of the wavelengths, derivatives excluded */
        const int64_t n_tot = P->tangent > 0 ? S->off_lam[P->tangent] : S->sca_len;
        for (int64_t i = 0; i < S->sca_len; ++i) {
            S->jsca_total[i] += pend_nxt[i];
            if (i < n_tot) tot += pend_nxt[i];
        }
        memcpy(S->U_LL, S->U, sizeof(double) * (size_t)G->n_leaf * nl);
        if (mode == 1) S->L_sca2 = tot;
    }
    return 0;
}

/* ------------------------------------------------------------------ API */
/* Set up j_sca levels (Eq. 5) and offsets; caller allocates arrays of
 * or_sca_len() doubles. */
int64_t or_setup(const or_grid *G, const or_params *P, or_state *S) {
    int64_t off = 0;
    for (int l = 0; l < G->n_lambda; ++l) {
        S->k_lam[l] = or_k_hp(G->g[l], P->n_fwhm, P->k_sca_cap);
        S->off_lam[l] = off;
        off += (int64_t)G->n_leaf * (12LL << (2 * S->k_lam[l]));
    }
    S->sca_len = off;
    return off;
}

/* Steps 1 and 2 (Sect. 2). */
int or_direct(const or_grid *G, const or_params *P, or_state *S) {
    S->cur_is_a = 1;  /* deposits of step 2 go to pend_b (the "next" buffer) */
    memset(S->counters, 0, sizeof S->counters);  /* counters cover one call */
    memset(S->jsca_total, 0, sizeof(double) * (size_t)S->sca_len);
    if (S->dg_on) memset(S->dg, 0, sizeof(double) * (size_t)G->n_leaf * G->n_lambda);
    int rc = or_phase(G, P, S, 0, 0);
    if (rc) return rc;
    return or_phase(G, P, S, 1, 0);
}

/* Step 2 for the change of the dust emission in a self-heating iteration
 * (Sect. 3.3, items 5-6): the emissivity holds that change; the U_LL step is
 * skipped (U_LL equals the RFED of the previous iteration), U and the total
 * j_sca start from their previous values. */
int or_direct_incremental(const or_grid *G, const or_params *P, or_state *S) {
    S->cur_is_a = 1;
    memset(S->counters, 0, sizeof S->counters);
    return or_phase(G, P, S, 1, 1);
}

/* One scattering iteration (Sect. 2); *remaining = pending / L_sca,2. */
int or_scatter_iter(const or_grid *G, const or_params *P, or_state *S, double *remaining) {
    memset(S->counters, 0, sizeof S->counters);
    int rc = or_phase(G, P, S, 2, 0);
    if (rc) return rc;
    const double *nxt = S->cur_is_a ? S->pend_b : S->pend_a;
    double tot = 0;
    const int64_t n_tot = P->tangent > 0 ? S->off_lam[P->tangent] : S->sca_len;
    for (int64_t i = 0; i < n_tot; ++i) tot += nxt[i];
    *remaining = S->L_sca2 > 0 ? tot / S->L_sca2 : 0.0;
    return 0;
}

/* Pointer to the buffer holding the luminosity deposited in the last phase. */
double *or_pending_next(or_state *S) { return S->cur_is_a ? S->pend_b : S->pend_a; }

/* Optical depth along the segment from point a to point b (both inside or on
 * the model), by the same leaf traversal. */
double or_tau(const or_grid *G, int l, const double a[3], const double b[3]) {
    double n[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    const double dist = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (dist <= 0) return 0;
    n[0] /= dist; n[1] /= dist; n[2] /= dist;
    double box[4];
    int leaf = or_locate(G, a, n, box);
    double d = 0, tau = 0;
    while (leaf >= 0 && d < dist) {
        int tie;
        double pe[3];
        double te = or_exit(a, n, box, &tie, pe);
        if (te > dist) te = dist;
        if (te > d) tau += G->kappa_rho[(int64_t)leaf * G->n_lambda + l] * (te - d);
        if (te >= dist) break;
        d = te;
        const int prev = leaf;
        leaf = or_locate(G, pe, n, box);
        if (leaf == prev) return NAN;  /* no progress: inexact face coordinates */
    }
    return tau;
}

/* Sub-points of a leaf for the map (reading of the paper's volume rendering):
 * a (sub)cube of side s at distance r is projected as one point at its centre
 * unless it subtends more than one map pixel (s^2/r^2 > Omega_pix), in which
 * case it is split into 8 octants, at most max_sub times.  Points within
 * 1e-6 of the cube side of the observer are skipped. */
static void or_map_point(const or_grid *G, const or_state *S, const double obs[3], int nside_k,
                         const double *emis_row, const double *jsca_rows[OR_MAXL], int leaf,
                         double L_leaf, const double lo[3], double s, int depth, int max_sub,
                         double *map) {
    const int nl = G->n_lambda;
    const int64_t npix = 12LL << (2 * nside_k);
    const double omega_pix = 4.0 * OR_PI / (double)npix;
    const double x[3] = {lo[0] + 0.5 * s, lo[1] + 0.5 * s, lo[2] + 0.5 * s};
    const double v[3] = {x[0] - obs[0], x[1] - obs[1], x[2] - obs[2]};
    const double r2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const double inside = (obs[0] >= lo[0] && obs[0] <= lo[0] + s && obs[1] >= lo[1] &&
                           obs[1] <= lo[1] + s && obs[2] >= lo[2] && obs[2] <= lo[2] + s);
    if (depth < max_sub && (inside || s * s > omega_pix * r2)) {
        const double h = 0.5 * s;
        for (int c = 0; c < 8; ++c) {
            const double clo[3] = {lo[0] + ((c & 1) ? h : 0), lo[1] + ((c & 2) ? h : 0),
                                   lo[2] + ((c & 4) ? h : 0)};
            or_map_point(G, S, obs, nside_k, emis_row, jsca_rows, leaf, L_leaf, clo, h, depth + 1,
                         max_sub, map);
        }
        return;
    }
    if (sqrt(r2) <= 1e-6 * s) return;
    const double frac = (s * s * s) / (L_leaf * L_leaf * L_leaf);
    const int64_t mp = or_vec2pix(nside_k, v);
    const double back[3] = {-v[0], -v[1], -v[2]};
    for (int l = 0; l < nl; ++l) {
        /* per-sr luminosity of the (sub)cell toward the observer: stellar j V
         * plus the scattered luminosity of the j_sca pixel holding that
         * direction divided by its solid angle (Sect. 2, end) */
        const int kl = S->k_lam[l];
        const int npx = 12 << (2 * kl);
        const double Vl = L_leaf * L_leaf * L_leaf;
        double I0 = emis_row[l] * Vl;
        if (jsca_rows[l]) I0 += jsca_rows[l][or_vec2pix(kl, back)] / (4.0 * OR_PI / (double)npx);
        I0 *= frac;
        if (I0 <= 0) continue;
        const double tau = or_tau(G, l, x, obs);
        map[(int64_t)l * npix + mp] += I0 * exp(-tau) / (r2 * omega_pix);
    }
}

/* Surface-brightness map for an observer inside the model (Sect. 3.6.3):
 * map[l][pix] = sum over (sub)cells of I_0 exp(-tau) / (r^2 Omega_pix),
 * i.e. flux per steradian, on a nested HEALPix map of level nside_k. */
int or_map(const or_grid *G, const or_state *S, const double obs[3], int nside_k, int max_sub,
           int use_jsca, double *map) {
    const int nl = G->n_lambda;
    double *leaf_box = (double *)malloc(sizeof(double) * 4 * (size_t)G->n_leaf);
    or_leaf_boxes(G, leaf_box);
    for (int64_t leaf = 0; leaf < G->n_leaf; ++leaf) {
        const double *b = leaf_box + 4 * leaf;
        const double *jrows[OR_MAXL];
        for (int l = 0; l < nl; ++l) {
            const int npx = 12 << (2 * S->k_lam[l]);
            jrows[l] = use_jsca ? S->jsca_total + S->off_lam[l] + leaf * npx : NULL;
        }
        or_map_point(G, S, obs, nside_k, G->emis + leaf * nl, jrows, (int)leaf, b[3], b, b[3], 0,
                     max_sub, map);
    }
    free(leaf_box);
    return 0;
}

/* Phase entry point for tests that drive the three steps one by one. */
int or_run_phase(const or_grid *G, const or_params *P, or_state *S, int mode) {
    return or_phase(G, P, S, mode, 0);
}

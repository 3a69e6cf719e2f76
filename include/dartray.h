/*
 * dartray.h -- C ABI of the GB300 ray-propagation sweep of DART-Ray V2
 * (Natale et al. 2017, "Ray-tracing 3D dust radiative transfer with DART-Ray:
 * code upgrade and public release").
 *
 * The library solves, on one GPU, the three-step radiative-transfer sweep of
 * the paper's Sect. 2 for the stellar emission of a model on an adaptive 3D
 * Cartesian grid: the lower limit U_LL of the radiation-field energy density
 * (RFED), the direct light with ray blocking (Eq. 1), and the scattering
 * iterations; and it projects the result onto HEALPix maps for an observer
 * inside the model.  Rays follow HEALPix directions (Sect. 3.1.1) and are
 * split (Eq. 2) or merged (Eq. 3) as they propagate; the scattering source
 * function is sampled on HEALPix(k_lambda) (Sect. 3.1.2, Eq. 4, Eq. 5); the
 * blocking threshold is f_U = 4 a_RT / N_s (Sect. 3.5, Eq. 10).
 *
 * Conventions shared by every call
 *   - Return value: DARTRAY_OK (0) or a negative DARTRAY_E_* code.  A failed
 *     call leaves a message readable with dartray_last_error() (thread-local).
 *     No call aborts the process; device-side failures (crossing cap, queue
 *     overflow) are reported through a device status word read by the host.
 *   - Units: lengths, kappa*rho (1/length), emissivity (luminosity per volume
 *     per steradian) and c_light are in the caller's model units.  U is
 *     returned in luminosity / (length^3 * c_light units).
 *   - Arrays are dense, row-major, float32 unless stated.  Pointers marked
 *     "host or device" are device pointers when the flag next to them is 1.
 *   - Streams: all device work of a grid is issued on the cudaStream_t given
 *     to dartray_grid_create; calls synchronise that stream before returning.
 *   - Thread safety: one grid must not be used by two threads at once.
 */
#ifndef DARTRAY_H
#define DARTRAY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DARTRAY_MAX_LAMBDA 16

enum {
    DARTRAY_OK = 0,
    DARTRAY_E_INVAL = -1,   /* invalid argument or grid description */
    DARTRAY_E_NOMEM = -2,   /* device or host allocation failed */
    DARTRAY_E_CUDA = -3,    /* CUDA runtime error */
    DARTRAY_E_QUEUE = -4,   /* ray queues too small even for one source */
    DARTRAY_E_LIMIT = -5,   /* crossing cap per ray or wave cap reached */
    DARTRAY_E_STATE = -6    /* call out of order (e.g. scatter before direct) */
};

typedef struct dartray_grid dartray_grid; /* opaque, owned by the library */

/*
 * Model description (Sect. 2: "an adaptive 3D Cartesian grid of cells, each
 * with a given input value of stellar volume emissivity and dust optical
 * depth per unit length"; albedo and HG g per wavelength from the dust model;
 * point sources of Sect. 3.6.1).
 *
 * Layout: a lattice of nroot[0] x nroot[1] x nroot[2] cubic root cells of side
 * root_size, lower corner root_lo.  Each root tops an octree.  Nodes
 * 0 .. nroot[0]*nroot[1]*nroot[2]-1 are the roots (x fastest, then y, then
 * z).  A refined node's 8 children are contiguous from first_child[node], in
 * the order bx + 2*by + 4*bz (b = 1: upper half on that axis).  Leaves have
 * first_child = -1 and a leaf id leaf_of_node[node] in [0, n_leaf); internal
 * nodes have leaf_of_node = -1.  All face coordinates of all nodes must be
 * exactly representable in float32 (dyadic grids); otherwise
 * DARTRAY_E_INVAL.
 *
 * Ownership: caller-owned; copied into device memory by dartray_grid_create,
 * not referenced afterwards.
 */
typedef struct dartray_grid_desc {
    int32_t nroot[3];
    double root_lo[3];
    double root_size;
    int32_t n_nodes, n_leaf, n_lambda;   /* 1 <= n_lambda <= DARTRAY_MAX_LAMBDA */
    const int32_t *first_child;          /* [n_nodes] host or device */
    const int32_t *leaf_of_node;         /* [n_nodes] host or device */
    const float *kappa_rho;              /* [n_leaf][n_lambda] extinction per length, >= 0 */
    const float *emissivity;             /* [n_leaf][n_lambda] luminosity/volume/sr, >= 0 */
    const float *albedo;                 /* [n_lambda] in [0, 1] */
    const float *g;                      /* [n_lambda] HG anisotropy in (-1, 1) */
    int32_t n_point;                     /* point sources (may be 0) */
    const float *point_xyz;              /* [n_point][3] positions inside the model */
    const float *point_lum;              /* [n_point][n_lambda] total luminosity */
    int32_t inputs_on_device;            /* 1: every pointer above is a device pointer */
} dartray_grid_desc;

/*
 * Algorithm parameters.  The paper leaves most of them input-defined
 * (N_rays and N_rays^max of Eq. 2-3, R_pre of Sect. 2, n_FWHM and the cap on
 * k_lambda,HP of Sect. 3.1.2, a_RT of Sect. 3.5, f_L of Sect. 2).
 * dartray_params_default() fills the defaults listed beside each field.
 */
typedef struct dartray_params {
    double a_rt;          /* accuracy parameter; f_U = 4 a_rt / N_s (0.05) */
    double r_pre;         /* step-1 radius R_pre, model length units (0.15 * model size) */
    double f_l;           /* scattering stop fraction f_L (0.01), used by callers */
    double c_light;       /* light speed (1) */
    int32_t n_rays_min;   /* N_rays of Eq. 2 (5) */
    int32_t n_rays_max;   /* N_rays^max of Eq. 3 (40) */
    int32_t k0;           /* initial ray HEALPix level (2) */
    int32_t k_ray_max;    /* highest ray level, <= 13 (13) */
    int32_t k_sca_cap;    /* cap on k_lambda,HP, <= 3 (3) */
    int32_t n_fwhm;       /* n_FWHM (5) */
    int32_t merge;        /* 1: merge rays by Eq. 3 (1) */
    int32_t max_cross;    /* crossings per ray before DARTRAY_E_LIMIT (1 << 22) */
    int32_t max_waves;    /* waves per source batch before DARTRAY_E_LIMIT (200) */
    int32_t src_stride;   /* process sources s with s % src_stride == src_offset (1) */
    int32_t src_offset;   /* (0) */
    int64_t queue_rays;   /* capacity of each ray queue, records; 0 = automatic (0) */
    int64_t src_batch;    /* upper bound on sources traced together; 0 = automatic (0) */
    int32_t profile;      /* 1: time every ray-march launch with CUDA events (0) */
    int32_t deposit_direct; /* 1: deposit j_sca with per-pixel atomics only (0: deferred
                               per-cell accumulation of crossing records, atomics only
                               when the record buffer is full) */
    int64_t deposit_records; /* record buffer capacity per pipeline; 0 = automatic: 2048 per leaf,
                                at most 2^29 and about 20 GB per pipeline (0) */
    int32_t deterministic;   /* 1: bit-identical results from run to run: U, the j_sca rows
                                and the ledger are summed in 64-bit fixed point (exponents
                                from bounds of each cell's total), so no sum depends on the
                                order of the GPU's additions; slower deposits (0) */
    int32_t octant;          /* 1: octant mode for models symmetric under the reflections about
                                the planes through the centre of the root lattice (axisymmetric
                                models with a symmetric vertical profile; Sect. 3.6.4): only
                                sources in the first octant are traced and each deposit is
                                also made, reflected, in the other seven octants.  Same result
                                as the full mode; counters count the rays traced.  Requires
                                src_stride 1; a grid that is not symmetric is rejected with
                                DARTRAY_E_INVAL (0) */
    int32_t graphs;          /* 1: each pipeline's rounds of waves (ray march, merge, deposit
                                flush, wave advance) are captured once per phase as a CUDA
                                graph and replayed; ignored with profile = 1 (1) */
    int32_t tangent_albedo;  /* 1: forward mode -- the sweep also carries, for every
                                wavelength, the derivative of U with respect to its albedo
                                (dartray_rfed_tangent), as extra wavelengths with the same
                                extinction, albedo and g, no emission of their own, the
                                light their wavelength loses in each segment as extra
                                scattering source (d(albedo lost)/d albedo, Sect. 2), and
                                the blocking, splitting and merging decisions of their
                                wavelength (frozen).  At most 8 wavelengths; single-model
                                grids outside the octant and deterministic modes; no state
                                files (0) */
} dartray_params;

/* Per-call statistics.  Ledger entries are luminosities per wavelength of the
 * last phase of the call (emitted = absorbed + scattered + escaped + blocked
 * + cut + skipped to rounding); counters cover the whole call. */
typedef struct dartray_stats {
    int64_t rays, crossings, splits, merges, blocks, escapes, cuts, lows, resumes, waves,
        sources;
    double emitted[DARTRAY_MAX_LAMBDA];
    double absorbed[DARTRAY_MAX_LAMBDA];
    double scattered[DARTRAY_MAX_LAMBDA];
    double escaped[DARTRAY_MAX_LAMBDA];
    double blocked[DARTRAY_MAX_LAMBDA];
    double cut[DARTRAY_MAX_LAMBDA];
    double skipped[DARTRAY_MAX_LAMBDA];
    double f_u;           /* f_U of the last phase (Eq. 10) */
    double l_sca2;        /* total scattered luminosity at the end of step 2 */
    double gpu_ms;        /* device time of the call (CUDA events) */
    int64_t kernel_launches; /* kernels launched by the call */
    double march_ms;      /* with params.profile: time covered by ray-march kernels */
    int64_t march_launches; /* ray-march kernel launches of the call */
    int64_t jsca_pixels;  /* scattering source-function pixels updated */
    double flush_ms;      /* with params.profile: time covered by the deposit flushes
                             (record bucketing and per-cell expansion) */
    double busy_ms;       /* with params.profile: time covered by whole waves (march,
                             low-list merge, flush, wave advance) of either pipeline */
    int64_t restarts;     /* phase restarts with smaller source batches after a ray-queue
                             overflow (the result does not depend on them) */
    double march_sum_ms;  /* with params.profile: sum over ray-march launches of each
                             launch's event span on its stream (march_launches of them) */
    int64_t flushes;      /* deposit-record flushes (bucketing + per-cell expansion) that ran,
                             including the one that ends each phase */
    int64_t batches;      /* source batches traced (all pipelines, restarts excluded) */
    int64_t records;      /* j_sca deposit records written by the ray marcher (one per
                             depositing crossing of steps 2-3 not deposited directly) */
} dartray_stats;

/* Fill *p with the defaults above -- the paper's input-defined values of
 * Sect. 2 (R_pre, f_L), Sect. 3.1 (N_rays, N_rays^max, n_FWHM, the k cap) and
 * Sect. 3.5 (a_RT); r_pre is set when the grid is created if left
 * negative.  Errors: INVAL (NULL). */
int dartray_params_default(dartray_params *p);

/*
 * Validate the description, build the leaf face links (ropes) and upload the
 * grid to the current CUDA device; allocate U, U_LL, the two pending j_sca
 * buffers, the total j_sca and the ray queues.  k_lambda,HP per wavelength
 * follows Eq. 5 (integer part, clamped to [0, k_sca_cap]).  Any n_lambda
 * from 1 to 16: rays carry 1, 2, 4, 8 or 16 wavelengths, a count in between
 * being padded inside the library with wavelengths of no dust and no
 * emission (j_sca level 0), which every call hides (arrays in and out have
 * the caller's n_lambda).  cuda_stream is a cudaStream_t (NULL = default
 * stream).  On success *out owns all device memory until
 * dartray_grid_destroy.  Errors: INVAL (bad tree, non-dyadic coordinates,
 * bad sizes), NOMEM, CUDA.
 */
int dartray_grid_create(const dartray_grid_desc *desc, const dartray_params *params,
                        void *cuda_stream, dartray_grid **out);

/*
 * Several independent models in one grid, traced together: every wave of
 * the ray marcher holds rays of all models, so many small models fill the
 * GPU as one large model does (the paper's method is additive over sources,
 * and no ray leaves its model).  descs[m] describes model m as for
 * dartray_grid_create; all models share n_lambda, albedo and g (one dust
 * model).  Leaves and point sources are numbered model after model (see
 * dartray_model_info); dartray_rfed and dartray_jsca return all models
 * concatenated that way.  Each model keeps its own N_s (Eq. 10) and R_pre
 * (0.15 of its size when params->r_pre < 0).  dartray_scatter_iter stops a
 * model's emission once its remaining fraction is below params->f_l (as a
 * loop over single-model grids would stop it) and returns the largest
 * remaining fraction.  Not supported on batched grids: the octant mode,
 * maps, state files.  n_models <= 4096 / (6 n_lambda).  Errors as
 * dartray_grid_create.
 */
int dartray_grid_create_batch(const dartray_grid_desc *descs, int32_t n_models, const dartray_params *params,
                              void *cuda_stream, dartray_grid **out);

/* Layout and state of model `model` of a grid (a single-model grid has
 * model 0): first leaf and number of leaves, first point source, remaining
 * scattered fraction after the last call (the stop test of Sect. 2 against
 * the model's own step-2 scattered luminosity), 1 while it still emits in
 * scattering iterations.  Any pointer may be NULL.  Errors: INVAL. */
int dartray_model_info(const dartray_grid *grid, int32_t model, int64_t *leaf_offset, int32_t *n_leaf,
                       int64_t *point_offset, double *remaining_frac, int32_t *active);

/* Ledger of model `model` for the last phase of the last call, its f_U
 * (Eq. 10 with the model's own N_s) and its scattered luminosity at the end
 * of step 2 (Sect. 2; other fields 0).  Errors: INVAL. */
int dartray_model_stats(const dartray_grid *grid, int32_t model, dartray_stats *stats);

/* Steps 1 and 2 of Sect. 2: U_LL within R_pre, then direct light with ray
 * blocking (Eq. 1), depositing U, and the scattered luminosity into the
 * pending j_sca buffer; afterwards U_LL <- U and j_sca_total += pending.
 * stats may be NULL.  Errors: LIMIT, QUEUE, CUDA.
 *
 * Sources are traced in batches sized to the ray queues.  A batch whose
 * waves overflow a queue restarts the phase with smaller batches (counted in
 * stats->restarts).  The grid keeps, per phase kind, the largest peak wave
 * per source seen, and later calls size their batches from it, so repeated
 * calls on one grid do not restart.  None of this changes the result: a
 * phase is additive over sources. */
int dartray_direct(dartray_grid *grid, dartray_stats *stats);

/* One scattering iteration (Sect. 2): the pending scattered luminosity of the
 * previous phase is emitted from every dusty cell along HEALPix directions
 * (per-sr luminosity = pending pixel / pixel solid angle), depositing U and a
 * new pending buffer; afterwards U_LL <- U and j_sca_total += pending.
 * *remaining_frac = (pending luminosity) / (scattered luminosity at the end of
 * step 2); callers stop once it is below f_L.  Errors: STATE (no dartray_direct
 * yet), LIMIT, QUEUE, CUDA. */
int dartray_scatter_iter(dartray_grid *grid, double *remaining_frac, dartray_stats *stats);

/*
 * Dust emission and self-heating (Sect. 3.3).  The dust RT runs on a second
 * grid with the same topology whose wavelengths are those of the dust
 * emission (its kappa_rho, albedo and g are the dust's at those
 * wavelengths).  dartray_dust_emission computes, per cell, the equilibrium
 * temperature and emission of a synthetic modified blackbody (in place of
 * grain models): the absorbed power
 *   P = sum over both grids' wavelengths of (1 - albedo) kappa_rho c V U dlambda
 * balances 4 pi V sum_i scale kabs_i B(lambda_i, T) dlambda_i with
 * kabs_i = (1 - albedo_i) kappa_rho_i and B = lambda^-5 / (exp(c2/(lambda T)) - 1)
 * (lambda in um, c2 = 14387.77 um K; T by bisection in [t_min, t_max]); the
 * emission is j_i = scale kabs_i B(lambda_i, T).  The dust grid's
 * emissivity becomes the change of j since the previous call (clipped at 0;
 * the first call: j), which dartray_direct (first time) or
 * dartray_direct_incremental (later) then propagates.  T [n_leaf] and j
 * [n_leaf][n_lambda] (either may be NULL) go to host or device memory;
 * *max_rel_change receives max |j - j_prev| / j_prev over cells and
 * wavelengths with j_prev > 0 (infinite on the first call).  Iterate until
 * it is below 1% (the paper's criterion).  Both grids have 1, 2, 4, 8 or 16
 * wavelengths.  Errors: INVAL, CUDA.
 */
typedef struct dartray_dust {
    int32_t n_ir;                              /* = n_lambda of the dust grid */
    double lam_ir[DARTRAY_MAX_LAMBDA];         /* dust wavelengths, um */
    double dlam_ir[DARTRAY_MAX_LAMBDA];        /* their bin widths, um */
    int32_t n_stellar;                         /* = n_lambda of the stellar grid */
    double dlam_stellar[DARTRAY_MAX_LAMBDA];   /* stellar bin widths, um */
    double scale;                              /* prefactor of the emission (model units) */
    double t_min, t_max;                       /* temperature bracket, K */
} dartray_dust;

int dartray_dust_emission(dartray_grid *dust_grid, const dartray_grid *stellar_grid, const dartray_dust *dust,
                          float *T, float *j, int dst_is_device, double *max_rel_change);

/*
 * Surface-brightness map for a distant observer (orthographic; Sect. 2, end:
 * I_obs = I_0 e^-tau along each line of sight, the cells treated as a
 * continuous medium).  view: unit vector from the model toward the
 * observer; up: the image's up direction (made orthogonal to view); right =
 * up x view.  Pixel (i, j) is the line of sight through
 * origin[0] + (i + 1/2) pixel along right and origin[1] + (j + 1/2) pixel
 * along up (image-plane coordinates through the coordinate origin), parallel
 * to -view.  Front to back, a cell crossed over ds with extinction kr adds
 * eta (1 - e^{-kr ds}) / kr (eta ds if kr = 0) times the transmission in
 * front of it; eta = emissivity + j_sca_total[pixel of view] / (Omega V)
 * (use_jsca = 0: the stellar emissivity alone).  map: [n_lambda][ny][nx],
 * luminosity per area per sr, host or device.  Single-model grids.
 * Errors: INVAL, CUDA.
 */
int dartray_map_external(dartray_grid *grid, const double view[3], const double up[3], const double origin[2],
                         double pixel, int32_t nx, int32_t ny, int32_t use_jsca, float *map, int dst_is_device);

/* Vector-Jacobian product of dartray_map_external (the map of Sect. 2,
 * end), the radiation field of the last sweep held fixed (the luminosity each crossing deposits into the
 * scattering source function does not move):
 *   grad_kappa_rho[c][l] = sum over pixels of dmap[l][pixel]
 *                          d map[l][pixel] / d kappa_rho[c][l]
 * (the source eta held fixed);
 *   grad_albedo[l], the same for the albedo, through j_sca, which is
 * proportional to it at a fixed radiation field (null: not wanted);
 *   grad_g[l], the same for the HG asymmetry g, through the j_sca pixel
 * toward the observer, from the tally of dartray_jsca_dg_arm (armed for this
 * view before dartray_direct; use_jsca set; null: not wanted; else STATE).
 * The transmission is recomputed along every line of sight (two passes)
 * instead of stored.  dmap [n_lambda][ny][nx] and grad_kappa_rho
 * [n_leaf][n_lambda] are both host or both device memory; grad_albedo and
 * grad_g [n_lambda] are host memory.  Errors: INVAL, STATE, CUDA. */
int dartray_map_external_vjp(dartray_grid *grid, const double view[3], const double up[3], const double origin[2],
                             double pixel, int32_t nx, int32_t ny, int32_t use_jsca, const float *dmap,
                             float *grad_kappa_rho, double *grad_albedo, double *grad_g, int on_device);

/* Arm (view non-null) or disarm (null) the tally of d j_sca / d g: from the
 * next dartray_direct on, every deposit into the scattering source function
 * (Eq. 4 with the HG function, rows normalised over the pixels) also adds
 * L_sca d/dg [Phi(n_v.n) / sum_q Phi(n_q.n)] to its cell, n_v the centre of
 * the j_sca pixel holding `view` (per wavelength), L_sca held fixed.  The
 * tally covers step 2 and the scattering iterations.  Single-model grids
 * outside the octant mode.  Errors: INVAL, CUDA. */
int dartray_jsca_dg_arm(dartray_grid *grid, const double view[3]);

/* The armed tally of d j_sca / d g (Eq. 4), [n_leaf][n_lambda] (host or
 * device).  Errors: INVAL, STATE (not armed), CUDA. */
int dartray_jsca_dg(dartray_grid *grid, float *out, int dst_is_device);

/* Replace kappa_rho [n_leaf][n_lambda] (host or device; the extinction per
 * length of the problem's inputs, Sect. 2), e.g. to map a changed dust
 * distribution; the RFED and j_sca keep their values until the next sweep.
 * Errors: INVAL, CUDA. */
int dartray_set_kappa_rho(dartray_grid *grid, const float *kappa_rho, int src_is_device);

/* Replace the emissivity [n_leaf][n_lambda] (host or device; the
 * luminosity per volume per sr of the problem's inputs, Sect. 2; the dust
 * emission of Sect. 3.3 goes in this way).  Errors: INVAL, CUDA. */
int dartray_set_emissivity(dartray_grid *grid, const float *emissivity, int src_is_device);

/* Step 2 for the current emissivity on top of the present state (Sect. 3.3,
 * items 5-6): no U_LL step (U_LL is the RFED of the previous call), U and
 * the total j_sca keep their values and receive the new deposits; the
 * pending j_sca starts from zero, and the following dartray_scatter_iter
 * calls measure their remaining fraction against this step's scattered
 * luminosity.  Errors: STATE (no dartray_direct yet), LIMIT, QUEUE, CUDA. */
int dartray_direct_incremental(dartray_grid *grid, dartray_stats *stats);

/* Autotuner: times steps 1 and 2 on every sample_stride-th source with each
 * deposit schedule of the scattering source function (the per-record
 * expansion follows the paper's communication mode, Sect. 3.4) -- 0: deferred per-cell records in the full buffer, 1:
 * deferred with a sixteenth of the buffer (smaller, more frequent flushes),
 * 2: per-pixel atomics in the ray marcher -- and keeps the fastest for the
 * later calls of the grid (results do not depend on the schedule).
 * *choice receives its index and ms[3] the times (-1: not tried); either
 * may be NULL.  The trial runs leave no state: call dartray_direct next.
 * Errors: INVAL, and those of dartray_direct. */
int dartray_autotune(dartray_grid *grid, int32_t sample_stride, int32_t *choice, double *ms);

/* RFED U [n_leaf][n_lambda] and absorbed luminosity
 * L_abs = (1 - albedo) * kappa_rho * c_light * V * U [n_leaf][n_lambda]
 * (the outputs of Sect. 2; either pointer may be NULL), written to host or
 * device memory.  Errors: INVAL, CUDA. */
int dartray_rfed(dartray_grid *grid, float *U, float *L_abs, int dst_is_device);

/* Forward mode (params.tangent_albedo; the deposits of Sect. 2
 * differentiated with respect to the albedo): dU/d albedo [n_leaf][n_lambda] (the
 * derivative of each wavelength's U with respect to its own albedo, the
 * sweep's decisions held) and dL_abs/d albedo = kappa_rho c_light V
 * ((1 - albedo) dU - U), host or device memory (either may be NULL).
 * Errors: INVAL, STATE (not the forward mode), CUDA. */
int dartray_rfed_tangent(dartray_grid *grid, float *dU, float *dL_abs, int dst_is_device);

/* j_sca layout: k_lambda per wavelength (Eq. 5), offset of each wavelength
 * block and total length; block l is [n_leaf][12 * 4^k_lambda[l]] (nested
 * HEALPix pixels, Sect. 3.1.2).  Errors: INVAL. */
int dartray_jsca_layout(const dartray_grid *grid, int32_t *k_lambda, int64_t *offsets,
                        int64_t *total_len);

/* Copy j_sca, the scattering source function of Sect. 3.1.2 (Eq. 4): which
 * = 0 total scattered luminosity per pixel (all phases so far), 1 = pending
 * (deposited by the last phase).  out has total_len floats.  Errors: INVAL,
 * CUDA. */
int dartray_jsca(dartray_grid *grid, int which, float *out, int dst_is_device);

/*
 * Surface-brightness map for an observer inside the model (Sect. 2 end,
 * Sect. 3.6.3): I_obs = I_0 exp(-tau).  Every leaf is projected as a point at
 * its centre, subdivided into octants (at most max_sub times) while it
 * subtends more than one map pixel or contains the observer; I_0 is the
 * (sub)cell's per-sr luminosity toward the observer (j V plus the total j_sca
 * pixel that holds that direction over its solid angle), tau the optical
 * depth from the (sub)cell centre to the observer.  map[l][p] (nested
 * HEALPix, level nside_k, 12*4^nside_k pixels) receives
 * sum I_0 exp(-tau) / (r^2 Omega_pix).  use_jsca = 0 maps the stellar light
 * only.  Errors: INVAL, CUDA.
 */
int dartray_map(dartray_grid *grid, const double observer[3], int32_t nside_k, int32_t max_sub,
                int32_t use_jsca, float *map, int dst_is_device);

/*
 * dartray_map (the internal-observer map of Sect. 3.6.3) without any device
 * allocation, for callers that cannot call cudaMalloc (for example code running under an allocator that forbids it,
 * or an application that reserves all device memory up front).  The paper has
 * no counterpart; the result equals dartray_map's.
 *
 * The map is summed in a fixed 8 MiB static device buffer (2^21 floats) and
 * then copied to map (host or device).  Maps larger than that -- 12*4^nside_k
 * pixels times n_lambda above 2^21 -- are rejected with DARTRAY_E_INVAL.  The
 * buffer is shared by every call in the process and keeps the last call's
 * map; each call clears the part it uses.  Calls that overlap on the GPU
 * (several threads, or several streams without ordering) race on it.  The
 * first call on a device looks up the buffer's device address (with that
 * device current); make that first call before any stream capture.  Every
 * device that loads the library holds the buffer until the process exits.
 */
int dartray_map_noalloc(dartray_grid *grid, const double observer[3], int32_t nside_k, int32_t max_sub,
                        int32_t use_jsca, float *map, int dst_is_device);

/* Save / restore the RFED and source-function state (U, U_LL, pending,
 * j_sca_total and the step-2 scattered luminosity) to a raw binary file, so
 * that maps can be made without repeating the sweep (the paper writes its
 * outputs to HDF5 files, Sect. 3.6; this library keeps raw arrays).
 * Errors: INVAL (batched grids, the forward mode, a file of another grid),
 * CUDA. */
int dartray_state_save(dartray_grid *grid, const char *path);
int dartray_state_load(dartray_grid *grid, const char *path);

void dartray_grid_destroy(dartray_grid *grid);

/* Message of the last failed call on this thread ("" if none). */
const char *dartray_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DARTRAY_H */

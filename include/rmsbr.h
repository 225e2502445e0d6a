/*
 * rmsbr.h -- C ABI of the B300 (sm_103a) shooting-and-bouncing-of-rays (SBR)
 * radio-map library.
 *
 * The library computes the radio map of the Sionna RT technical report
 * (arXiv 2504.21719, Sec. 4): rays leave a transmitter in the directions of a
 * spherical Fibonacci lattice (Sec. 3.1.1), are traced through a triangle
 * mesh (Sec. 2.1) with an LBVH, are specularly reflected or refracted through
 * thin slabs with the radio-material model (App. A.7, Eqs. fresnel_vac,
 * fresnel_slab), choosing one interaction per hit with the Fresnel-power
 * heuristic (Eq. path-solver-used-dist-event), and deposit path gain into the
 * cells of a horizontal measurement plane (or the triangles of a measurement
 * mesh) wherever they cross it (Eq. radio-map-solver-ci-all-2-estimator,
 * n_S = 0, with the squared ray-tube length cancelled by the 1/r spreading of
 * Eq. radio-map-solver-path-gain).  Diffuse reflection (App. A.10), synthetic
 * arrays, early termination (Sec. 4) and the first-order diffraction map
 * (Sec. 4, App. A.8) extend it.
 *
 * Conventions shared by every call:
 *  - Pointers named *_dev are CUDA device memory owned by the CALLER; pointers
 *    named *_host are host memory owned by the caller and only read during the
 *    call.  Handles (rm_scene, rm_trace_plan) are owned by the library and
 *    released with the matching *_free call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is enqueued on it.
 *  - Every call returns an rm_status; no C++ exception crosses the ABI.  On a
 *    non-OK status, rm_last_error() returns a thread-local message.  Arguments
 *    are validated on the host before anything is enqueued; RM_EINVAL means
 *    nothing was launched.
 *  - Floating-point work is FP32 on the device; counts are 64-bit.
 *  - Maps are row-major [ny][nx] (cell (ix, iy) at index iy * nx + ix) of
 *    linear path gain (dimensionless, not dB).  Cell (0, 0) has its lower-left
 *    corner at (map_origin.x - nx*cell/2, map_origin.y - ny*cell/2).
 */
#ifndef RMSBR_H
#define RMSBR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RM_OK = 0,
    RM_EINVAL = 1,     /* bad argument; nothing was launched */
    RM_ENOMEM = 2,     /* a device allocation failed */
    RM_ECUDA = 3,      /* a CUDA runtime call failed (message has the CUDA error) */
    RM_EOVERFLOW = 4,  /* a device-side bound was hit (BVH stack or step budget, or the 8 crossings a
                          diffracted ray keeps on a mesh surface); the affected work was dropped */
    RM_ETIMEOUT = 5,   /* reserved: a bounded device wait gave up */
    RM_ESTATE = 6      /* call order: e.g. tracing before rm_bvh_build, or during stream capture */
} rm_status;

/* Host-side fault injection kinds (rm_debug_inject, RM_FAULT). */
#define RM_FAULT_ALLOC 1     /* scene upload / BVH build return RM_ENOMEM before allocating */
#define RM_FAULT_LAUNCH 2    /* a trace or gradient returns RM_ECUDA before enqueueing anything */
#define RM_FAULT_OVERFLOW 3  /* a trace or gradient completes, then reports RM_EOVERFLOW as a device
                                status word would */

#define RM_MAX_DEPTH 15      /* maximum number of interactions L */
#define RM_MAX_MATERIALS 32  /* radio materials per scene */
#define RM_MAX_TX 64         /* transmitters per trace call */

/* Radio material: the complex relative permittivity is
 *   eta = eps_r - j sigma / (eps0 omega)                     (Eq. eta)
 * evaluated at the trace frequency.  thickness > 0: a single-layer slab of
 * that thickness in metres (Eqs. fresnel_slab, q_fresnel_slab) that reflects
 * and transmits without deflection (Sec. 2.3); thickness <= 0: a half-space
 * that only reflects (Eq. fresnel_vac, transmission coefficient 0).
 *
 * Diffuse reflection (App. A.10; used only under RM_DIFFUSE): the share
 * S^2 of the reflected power is scattered into the incident-side hemisphere,
 * the specular coefficients are reduced by R = sqrt(1 - S^2) (Eq. R), and
 * the scattered field follows Eq. scattered_field with the cross-polarisation
 * share K_x and the scattering pattern f_s: 0 Lambertian (Eq.
 * lambertian_model), 1 directive with lobe exponent alpha_r (Eq.
 * directive_model), 2 backscattering with exponents alpha_r, alpha_i and lobe
 * split lambda (Eq. backscattering_model).  scattering = 0 disables it for
 * the material; the remaining fields are then ignored.  All-zero diffuse
 * fields are valid (no diffuse reflection). */
typedef struct {
    float eps_r;
    float sigma;        /* S/m */
    float thickness;    /* m */
    float scattering;   /* S in [0, 1] */
    float xpd_k;        /* K_x in [0, 1] */
    int32_t pattern;    /* 0, 1 or 2 (see above) */
    int32_t alpha_r;    /* 1..32 for patterns 1 and 2 */
    int32_t alpha_i;    /* 1..32 for pattern 2 */
    float lobe_lambda;  /* Lambda in [0, 1] for pattern 2 */
} rm_material;

/* One transmitter.  Rays are the lattice directions n = ray_begin + i *
 * ray_stride, i < ray_count, of a spherical Fibonacci lattice with num_rays
 * points (Sec. 3.1.1); each carries the solid angle 4 pi / num_rays, so
 * disjoint subsets of one lattice give maps that add up to the full map.
 * The antenna (pattern, pol) is oriented by yaw/pitch/roll (rad) as
 * R = Rz(yaw) Ry(pitch) Rx(roll) (Eq. rotation); its field in the departure
 * direction is R (C_theta theta' + C_phi phi') with the local angles of
 * Eq. theta_phi_prime and the pattern C of Eq. C. */
typedef struct {
    float pos[3];        /* m */
    float yaw, pitch, roll;
    int32_t pol;         /* 0 vertical (theta'), 1 horizontal (phi'), 2 dual: both, maps add (Sec. 4.4) */
    int32_t pattern;     /* 0 isotropic (G = 1), 1 short dipole (G = 1.5 sin^2 theta') */
    uint64_t num_rays;   /* N_S >= 1 */
    uint64_t ray_begin;
    uint64_t ray_count;  /* UINT64_MAX: all of ceil((num_rays - ray_begin) / ray_stride) */
    uint64_t ray_stride; /* >= 1 */
    uint64_t seed;       /* seed of the counter-based interaction sampler */
    /* Synthetic array (Sec. 4.4): n_ant elements at ant_pos_host [n_ant][3] (m,
     * antenna frame, rotated with the antenna) with complex precoding weights
     * precoding_host [n_ant][2] (re, im), both in double (phases reach k0 |d|,
     * ~1600 rad for a 1024-element half-wavelength array, so positions keep
     * double precision until the library splits them into hi + lo floats).
     * Each ray's launch field is scaled by
     * alpha = sum_k u_P,k exp(j 2 pi / lambda0 k.d_k) (array response vector,
     * Eq. path-solver-array-response-vector), evaluated at the ray's lattice
     * direction in double-float arithmetic; elements on one regular line
     * (uniform linear arrays) take a blocked Horner recurrence.  Trace and
     * gradient calls evaluate alpha for every ray in a pre-pass kernel before
     * the tracer (8 B of call-owned device memory per ray, up to 2^31 rays per
     * call); graph plans, the no-allocation entry point and larger calls
     * evaluate it at each ray's launch, with the same bits.
     * n_ant = 0: one antenna.  The host arrays are read during the call only. */
    int32_t n_ant;
    int32_t reserved;
    const double* ant_pos_host;
    const double* precoding_host;
} rm_tx;

/* trace flags */
#define RM_REFLECT 1u   /* allow specular reflection */
#define RM_REFRACT 2u   /* allow refraction through slabs */
#define RM_LOS 4u       /* deposit the line-of-sight segment (depth 0) */
#define RM_STATS 8u     /* collect per-depth power statistics (slower) */
#define RM_DIFFUSE 16u  /* diffuse reflection on materials with scattering > 0 (needs RM_REFLECT) */
#define RM_RECORD_COIN 32u  /* debug record only: each decision also carries the coin's q(R) */

typedef struct {
    double freq_hz;          /* carrier frequency f; lambda0 = c0 / f */
    int32_t max_depth;       /* L in [0, RM_MAX_DEPTH]; segments l = 0..L are deposited */
    uint32_t flags;          /* RM_REFLECT | RM_REFRACT | RM_LOS [| RM_STATS] [| RM_DIFFUSE] */
    float map_origin[3];     /* centre of the map; the plane is z = map_origin[2], normal +z */
    float cell_size;         /* m, > 0 */
    int32_t nx, ny;          /* cells, >= 1, nx * ny <= 2^31 - 1, nx, ny <= 32767 */
    int32_t deposit;         /* 0: box cells (the paper's estimator); 1: bilinear (tent) splat */
    int32_t block_size;      /* threads per block of the tracer; 0 = tuned default */
    int32_t blocks_per_sm;   /* resident blocks per SM of the persistent grid; 0 = tuned default */
    int32_t queue_chunk;     /* work items a warp takes per work-queue access, in units of 32 (1..64);
                                0 = default (1) */
    /* Early termination (Sec. 4.5), applied after an interaction once a path
     * has rr_depth interactions (0 = off).  The gain of a sample is w |E|^2,
     * w = 1 / Pr(chi).  gain_threshold > 0: stop when (lambda0/4pi)^2 w |E|^2 / r^2,
     * r the tube length, is below it (biased).  rr_max_prob in (0, 1]: Russian
     * roulette, continue with p = min(w |E|^2, rr_max_prob) (Eq.
     * radio-map-solver-rr-prob) and reweight survivors by 1/p (unbiased). */
    int32_t rr_depth;
    float rr_max_prob;
    float gain_threshold;
    int32_t refill_min;      /* a warp refills its idle lanes with new rays once at least this many
                                are idle (1..32): new rays then enter in coherent groups of lattice
                                neighbours; 0 = default (20) */
} rm_trace_params;

/* Counters of one trace call, summed over all transmitters. */
typedef struct {
    uint64_t rays;           /* lattice rays launched */
    uint64_t segments;       /* closest-hit queries = ray-bounces traced */
    uint64_t nodes_visited;  /* BVH internal nodes fetched (counted only under RM_STATS or with a
                                debug record; 0 otherwise) */
    uint64_t tris_tested;    /* ray-triangle tests (as nodes_visited) */
    uint64_t deposits;       /* plane crossings deposited into a map */
    uint64_t escapes;        /* segments that hit nothing */
    uint64_t segments_per_depth[RM_MAX_DEPTH + 1];
    /* RM_STATS only: sums over segments at depth l of w |E|^2 with w = 1 / Pr(chi),
     * (times 4 pi / N_S this is the power times solid angle carried), their
     * squares, and the part of the first sum whose segment escaped. */
    double power_per_depth[RM_MAX_DEPTH + 1];
    double power2_per_depth[RM_MAX_DEPTH + 1];
    double escaped_power_per_depth[RM_MAX_DEPTH + 1];
    int32_t status;          /* rm_status of the device-side checks */
    int32_t reserved;
    double kernel_ms;        /* device time of the tracer kernel (CUDA events on `stream`) */
} rm_stats;

/* Debug record of one segment (layout [tx][i][l], i the subset index,
 * l = 0..L).  prim: original triangle index hit, -1 escaped, -2 the ray had
 * already terminated.  ix, iy: deposited cell (bilinear: lower-left cell of
 * the 2x2 stencil), -32768 for no deposit.  decision: 0 reflection,
 * 1 refraction, 2 diffuse reflection, -1 none; plus 4 if Russian roulette
 * then stopped the path, 8 if the gain threshold did.  Under RM_RECORD_COIN a
 * decision >= 0 also carries, in bits 8..30, the probability q(R) the coin
 * compared its variate with, as round(q(R) 2^22): the parity tests check the
 * GPU's sampling probabilities interaction by interaction. */
typedef struct {
    int32_t prim, ix, iy, decision;
} rm_segment_record;

typedef struct rm_scene rm_scene;
typedef struct rm_trace_plan rm_trace_plan;

/* Copies a triangle mesh (Sec. 2.1) to library-owned device memory and
 * computes per-triangle bounding boxes.
 *   verts_dev  float [nv][3] (m); tris_dev int32 [nt][3] vertex indices;
 *   tri_mat_dev int32 [nt] material index per triangle; mats_host [nm].
 * nt may be 0 (free space).  Index ranges are checked on the device and
 * reported as RM_EINVAL (this call synchronises `stream`).  Caller buffers
 * may be freed after return.  *out is set on RM_OK only. */
rm_status rm_scene_upload(const float* verts_dev, int64_t nv, const int32_t* tris_dev, int64_t nt,
                          const int32_t* tri_mat_dev, const rm_material* mats_host, int32_t nm,
                          void* stream, rm_scene** out);

/* The same from host arrays (verts_host float [nv][3], tris_host int32 [nt][3],
 * tri_mat_host int32 [nt]): index ranges are checked on the host (RM_EINVAL
 * before any device work), the mesh is copied into a library-owned pinned
 * buffer and sent to the device in one asynchronous copy on `stream`; the call
 * does not wait for it.  Caller buffers may be freed after return.  With
 * rm_bvh_build, which does not wait either, a scene reaches the tracer with no
 * host round trip. */
rm_status rm_scene_upload_host(const float* verts_host, int64_t nv, const int32_t* tris_host, int64_t nt,
                               const int32_t* tri_mat_host, const rm_material* mats_host, int32_t nm,
                               void* stream, rm_scene** out);

/* Replaces the material table (no BVH rebuild).  sampling_host_or_null
 * (nm entries) sets the materials from which the interaction probabilities
 * q(R), q(S), q(T) are computed (detached from the fields); NULL = mats_host.
 * Only eps_r and sigma of a sampling material are used: thickness and the
 * diffuse parameters always come from mats_host. */
rm_status rm_scene_set_materials(rm_scene* scene, const rm_material* mats_host, int32_t nm,
                                 const rm_material* sampling_host_or_null);

/* Tree builders (rm_bvh_build_ex). */
#define RM_BVH_AUTO 0   /* RM_BVH_SAH above RM_BVH_AUTO_SAH_MIN triangles, else RM_BVH_LBVH */
#define RM_BVH_LBVH 1
#define RM_BVH_SAH 2
#define RM_BVH_AUTO_SAH_MIN 2048

/* Builds the scene's BVH on `stream` with the default builder
 * (rm_bvh_build_ex with RM_BVH_AUTO). */
rm_status rm_bvh_build(rm_scene* scene, void* stream);

/* Builds the scene's BVH on `stream`.  Not part of the paper (its
 * implementation uses Mitsuba's acceleration structure).  Both builders
 * start from 63-bit Morton codes of the doubled triangle centroids
 * (quantised with one scale for the three axes, 2^21 - 1 over the largest
 * centroid extent) in a stable 8-bit-digit radix sort, put one triangle in
 * each leaf, refit the AABBs exactly and store 64-byte two-child nodes; up to
 * 16 triangles as large as a quarter of the scene are kept out of the tree
 * (see rm_bvh_export).
 *   RM_BVH_LBVH: the Karras (HPG 2012) binary radix tree over the sorted
 *     codes, duplicate keys ordered by position (~1.3 ms for 1M triangles).
 *   RM_BVH_SAH: top-down splits that minimise the surface-area heuristic
 *     (MacDonald & Booth 1990) over 32 centroid bins per axis (Wald 2007),
 *     each range partitioned stably from the Morton order, middle splits from
 *     depth 32 on (no leaf deeper than 32 + ceil(log2 n)); internal node
 *     i is the node split between positions i and i + 1, except that the
 *     root is node 0 and takes the number of the node split between 0 and 1.
 *     ~14 % fewer node visits per ray than the LBVH on a city, at a few ms
 *     of build time.
 *   RM_BVH_AUTO: RM_BVH_SAH for more than RM_BVH_AUTO_SAH_MIN triangles,
 *     else RM_BVH_LBVH (one block, ~0.05 ms).
 * Must precede tracing; may be called again after rm_scene_upload only.
 * RM_EINVAL for another builder value.  The call returns
 * once the build is enqueued: the host does not wait for it.  The number of
 * large triangles comes back through a pinned slot and the first call that
 * needs it (a trace, rm_bvh_export, rm_scene_info) waits for the build there;
 * errors of the build's kernels surface at that call.  Without a free pinned
 * slot (4096 builds pending at once) the call waits for the build itself. */
rm_status rm_bvh_build_ex(rm_scene* scene, int32_t builder, void* stream);

/* Exports the built tree for inspection (synchronous).  Host outputs:
 * keys [nt] the Morton code of the triangle at each position (sorted for
 * RM_BVH_LBVH), order [nt] the triangle at each leaf position,
 * child [nn][2] (>= 0 internal node, < 0 leaf ~position),
 * child_aabb [nn][2][6] (lo xyz, hi xyz of each child), nn = nodes from
 * rm_scene_info.  Triangles whose largest AABB extent is at least a quarter
 * of the scene's (at most 16 of them) are not in the tree: their key is
 * 2^64 - 1, they end `order`, and the tracer tests them from a list. */
rm_status rm_bvh_export(const rm_scene* scene, uint64_t* keys_host, int32_t* order_host,
                        int32_t* child_host, float* child_aabb_host);

/* Traces the radio maps of ntx transmitters (1 <= ntx <= RM_MAX_TX) in one
 * persistent launch whose work queue hands out (transmitter, ray) items, and
 * writes maps_dev [ntx][ny][nx] (overwritten).  Deposits are accumulated in an
 * internal FP64 map (a cell under a transmitter can receive ~1e5 of them) and
 * rounded once to FP32; the order of the atomic additions varies between runs.  Each map is the
 * estimator of Eq. radio-map-solver-ci-all-2-estimator for its transmitter.
 * stats_host_or_null receives the counters.  record_dev_or_null receives one
 * rm_segment_record per (tx, ray, depth).  Synchronises `stream` before
 * returning (to read the device status); returns RM_ESTATE if `stream` is
 * capturing (use rm_trace_plan_* for graph launches). */
rm_status rm_radio_map_trace(const rm_scene* scene, const rm_tx* tx_host, int32_t ntx,
                             const rm_trace_params* params, float* maps_dev,
                             rm_stats* stats_host_or_null, rm_segment_record* record_dev_or_null,
                             void* stream);

/* Radio maps on a mesh measurement surface (Sec. 4, practical notes): every
 * triangle of `surface` (an uploaded scene with its BVH built; its materials
 * are unused, and it neither stops nor deflects rays) is one cell.  A crossing
 * of triangle i by a segment (open interval (1e-9, hit distance)) adds
 * 4 pi / (N A_i) (lambda0 / 4 pi)^2 |E|^2 / (|n_i . k| Pr): the estimator of
 * Eq. radio-map-solver-ci-all-2-estimator with the triangle's own area A_i
 * and unit normal n_i.  A crossing on an edge shared by two triangles counts
 * for both.  maps_dev [ntx][surface triangles] (input triangle order) is
 * overwritten.  params' map plane and cells are unused; deposit must be 0
 * (box).  Gradient: rm_radio_map_grad_mesh.  Otherwise as rm_radio_map_trace; the
 * record's cells are -32768.  RM_ESTATE if the surface's BVH is not
 * built, RM_EINVAL for a NULL or empty surface or deposit != 0. */
rm_status rm_radio_map_trace_mesh(const rm_scene* scene, const rm_scene* surface, const rm_tx* tx_host,
                                  int32_t ntx, const rm_trace_params* params, float* maps_dev,
                                  rm_stats* stats_host_or_null, rm_segment_record* record_dev_or_null,
                                  void* stream);

/* Vector-Jacobian product of the maps: given dL_dmaps_dev [ntx][ny][nx],
 * re-traces the same rays (same lattice, same sampler, hence the same hits,
 * decisions and cells) and accumulates
 *   d_eps_dev[m]   += sum_i dL/dC_i dC_i/d eps_r[m]
 *   d_sigma_dev[m] += sum_i dL/dC_i dC_i/d sigma[m]           (m < nm)
 *   d_txpos_dev[t][3] += sum_i dL/dC_i dC_i/d pos[t]
 * with the discrete choices held fixed and the sampling probabilities
 * detached (the derivative of f / q is taken as f' / q).  The outputs are
 * ACCUMULATED into (zero them first).  Under box deposit the maps do not
 * depend on the transmitter positions at fixed cells, so d_txpos stays 0;
 * bilinear deposit gives the derivative through the crossing points.
 * sampling_host_or_null overrides the scene's sampling materials for this
 * call.  Any of the three outputs may be NULL.  stats_host_or_null and
 * record_dev_or_null report the re-trace exactly as rm_radio_map_trace does
 * (the record must equal the forward call's).  Synchronises `stream`. */
rm_status rm_radio_map_grad(const rm_scene* scene, const rm_tx* tx_host, int32_t ntx,
                            const rm_trace_params* params, const float* dL_dmaps_dev,
                            float* d_eps_dev, float* d_sigma_dev, float* d_txpos_dev,
                            const rm_material* sampling_host_or_null, rm_stats* stats_host_or_null,
                            rm_segment_record* record_dev_or_null, void* stream);

/* Forward trace that also records, for the adjoint, the closest hit of every
 * segment (the paths of Sec. 4's estimator as sequences of hit triangles):
 * hits_dev[l R + w] = the leaf slot hit at depth l (a position in the scene's
 * tree order, -1 if the segment escaped) by the ray of work item w, where R =
 * the sum of the transmitters' ray counts and w runs over the rays in the
 * tracer's visit order (transmitter by transmitter, each a fixed permutation
 * of its lattice subset; the order is the library's, so treat the buffer as
 * opaque and hand it to rm_radio_map_grad_hits unchanged).  Neighbouring
 * lanes trace neighbouring work items, so the stores coalesce.  hits_dev:
 * device int32 owned by the caller, at least hits_len >= R x (max_depth + 1)
 * entries (RM_EINVAL otherwise); slots of depths a ray does not reach are not
 * written.  The maps and counters are those of rm_radio_map_trace; the call
 * runs its own instantiation of the plain tracer, which adds one 4-byte store
 * per segment (or, with RM_STATS, the statistics one).  Synchronises `stream`. */
rm_status rm_radio_map_trace_hits(const rm_scene* scene, const rm_tx* tx_host, int32_t ntx,
                                  const rm_trace_params* params, float* maps_dev, int32_t* hits_dev,
                                  uint64_t hits_len, rm_stats* stats_host_or_null, void* stream);

/* rm_radio_map_grad replaying recorded hits: hits_dev from
 * rm_radio_map_trace_hits with the same scene, transmitters and params.  At
 * every segment the adjoint tests only the recorded leaf (the traversal's own
 * watertight test, so the distance its traversal would find for that leaf)
 * instead of traversing the BVH; an entry of -1 is an escape.  An entry outside the scene, or a leaf the ray
 * misses, falls back to the traversal, so no access leaves the scene; a
 * buffer recorded with other arguments gives gradients of other paths.  With
 * the matching buffer the gradients equal rm_radio_map_grad's up to the order
 * of their atomic sums.  hits_len as above (RM_EINVAL if short); otherwise as
 * rm_radio_map_grad. */
rm_status rm_radio_map_grad_hits(const rm_scene* scene, const rm_tx* tx_host, int32_t ntx,
                                 const rm_trace_params* params, const float* dL_dmaps_dev,
                                 const int32_t* hits_dev, uint64_t hits_len, float* d_eps_dev,
                                 float* d_sigma_dev, float* d_txpos_dev,
                                 const rm_material* sampling_host_or_null, rm_stats* stats_host_or_null,
                                 rm_segment_record* record_dev_or_null, void* stream);

/* rm_radio_map_grad for maps on a mesh measurement surface (see
 * rm_radio_map_trace_mesh): dL_dmaps_dev [ntx][surface triangles].  The cells
 * are boxes, so d_txpos stays 0.  deposit must be 0; otherwise as
 * rm_radio_map_grad. */
rm_status rm_radio_map_grad_mesh(const rm_scene* scene, const rm_scene* surface, const rm_tx* tx_host,
                                 int32_t ntx, const rm_trace_params* params, const float* dL_dmaps_dev,
                                 float* d_eps_dev, float* d_sigma_dev, float* d_txpos_dev,
                                 const rm_material* sampling_host_or_null, rm_stats* stats_host_or_null,
                                 rm_segment_record* record_dev_or_null, void* stream);

/* rm_radio_map_trace_hits for maps on a mesh measurement surface (see
 * rm_radio_map_trace_mesh): the same maps, and the closest hit of every
 * segment in the scene (not the surface's crossings, which the adjoint walks
 * again) in hits_dev, with the layout, length rule and errors of
 * rm_radio_map_trace_hits and of rm_radio_map_trace_mesh. */
rm_status rm_radio_map_trace_mesh_hits(const rm_scene* scene, const rm_scene* surface, const rm_tx* tx_host,
                                       int32_t ntx, const rm_trace_params* params, float* maps_dev,
                                       int32_t* hits_dev, uint64_t hits_len, rm_stats* stats_host_or_null,
                                       void* stream);

/* rm_radio_map_grad_mesh replaying the hits of rm_radio_map_trace_mesh_hits
 * (same scene, surface, transmitters and params), as rm_radio_map_grad_hits
 * does for the plane: only the recorded leaf is tested at each segment. */
rm_status rm_radio_map_grad_mesh_hits(const rm_scene* scene, const rm_scene* surface, const rm_tx* tx_host,
                                      int32_t ntx, const rm_trace_params* params, const float* dL_dmaps_dev,
                                      const int32_t* hits_dev, uint64_t hits_len, float* d_eps_dev,
                                      float* d_sigma_dev, float* d_txpos_dev,
                                      const rm_material* sampling_host_or_null, rm_stats* stats_host_or_null,
                                      rm_segment_record* record_dev_or_null, void* stream);

/* Loss of the differentiable workload: mean over the cells V where both maps
 * exceed floor_linear of (10 log10 C_i - 10 log10 T_i)^2.  Writes loss_dev[0]
 * (float), dL_dmaps_dev [ncells] (0 outside V) and valid_dev[0] = |V|
 * (int64).  Asynchronous on `stream`. */
rm_status rm_db_mse_loss(const float* maps_dev, const float* target_dev, int64_t ncells,
                         float floor_linear, float* loss_dev, float* dL_dmaps_dev,
                         int64_t* valid_dev, void* stream);

/* A trace captured once into a CUDA graph (map clear + persistent tracer),
 * for repeated launches with the same arguments.  The plan owns its scratch
 * memory; maps_dev must outlive it. */
rm_status rm_trace_plan_create(const rm_scene* scene, const rm_tx* tx_host, int32_t ntx,
                               const rm_trace_params* params, float* maps_dev, void* stream,
                               rm_trace_plan** out);
rm_status rm_trace_plan_launch(rm_trace_plan* plan, void* stream);
/* Counters of the last launch (synchronises `stream`); kernel_ms is the
 * tracer node's time, from events the graph records around it. */
rm_status rm_trace_plan_stats(rm_trace_plan* plan, void* stream, rm_stats* stats_host);
void rm_trace_plan_free(rm_trace_plan* plan);

/* Same radio maps as rm_radio_map_trace, for callers that cannot allocate
 * device memory while they run: a serving loop whose memory was reserved
 * once at start-up and must not grow, code that owns every byte of the GPU
 * through its own pool, or a latency-critical thread that must not wait on
 * the allocator (cudaMalloc and cudaFree may synchronise the device).  This
 * entry point calls no cudaMalloc, cudaFree or other allocating routine.
 * The paper has no counterpart of it: it only changes where the tracer's
 * scratch lives.
 *   Scratch: one static device array of 16 KB, enough for RM_MAX_MATERIALS
 *   materials and RM_MAX_TX transmitters plus 72 synthetic-array elements
 *   (32 bytes each); every GPU that loads the library holds it until the
 *   process exits.  A call that would need more is rejected with RM_EINVAL.
 *   Set-up: the first call on a device looks up the array's device address
 *   (with that device current); make that first call before any stream
 *   capture.
 *   Sharing: every call uses the same array, which keeps the last call's
 *   contents (each call clears what must start at zero).  Calls whose work
 *   overlaps on the GPU race on it: issue them on one stream, or wait for
 *   one to finish before starting the next.
 * Arguments, outputs and errors are those of rm_radio_map_trace without the
 * debug record; stats_host_or_null receives the counters (kernel_ms = 0).
 * The call reads its counters back and waits for `stream`; a stream that is
 * capturing is refused with RM_ESTATE before anything is enqueued.
 * Deposits are accumulated with FP32 atomics directly in maps_dev (no FP64
 * buffer), so cells that receive very many deposits carry FP32 summation error.
 * Synchronises `stream`. */
rm_status rm_radio_map_trace_noalloc(const rm_scene* scene, const rm_tx* tx_host, int32_t ntx,
                                     const rm_trace_params* params, float* maps_dev,
                                     rm_stats* stats_host_or_null, void* stream);

/* ------------------------------------------------------------------------
 * First-order diffraction radio map (Sec. 4, "Computation of Radio Map due
 * to Diffraction"; UTD of App. A.8)
 * ------------------------------------------------------------------------ */

/* A wedge: a mesh edge shared by two triangles that meet at a convex corner.
 * The 0-face is the triangle of lower index; edge = n0 x nn / |n0 x nn| runs
 * from origin for `length` metres; the exterior angle is n pi, 1 < n <= 2.
 * Normals are the outward normals given by the triangles' winding. */
typedef struct {
    float origin[3];
    float edge[3];
    float n0[3];        /* outward normal of the 0-face */
    float nn[3];        /* outward normal of the n-face */
    float length;       /* m */
    float n;            /* exterior angle / pi */
    int32_t tri0, trin; /* triangle indices of the two faces (as uploaded) */
    int32_t mat0, matn; /* their materials */
} rm_wedge;

/* The wedges of a scene: every edge (by vertex indices) shared by exactly two
 * triangles whose outward normals are not parallel and whose corner is convex
 * (the far vertex of the n-face lies behind the 0-face's plane).  Ordered by
 * (tri0, trin).  Writes min(count, cap) wedges to out_host (may be NULL with
 * cap 0) and the total to *count.  Synchronous: copies the mesh to the host. */
rm_status rm_scene_wedges(const rm_scene* scene, rm_wedge* out_host, int64_t cap, int64_t* count);

/* Diffraction radio maps [ntx][ny][nx] (overwritten; add them to the SBR maps
 * of rm_radio_map_trace for the full map, as the paper does).
 * Estimator (Eq. radio-map-solver-ci-D-est): every wedge gets
 * samples_per_wedge samples (x, phi), x = L_E (i + 1/2)/N, phi = n pi
 * frac(i (phi_g - 1)) (a rank-1 lattice, the quasi-Monte-Carlo form of
 * uniform sampling); sample i adds
 *   (1 / Delta^2) (L_E n pi / N) (lambda0 / 4 pi)^2 |E_d|^2 |dt/dx x dt/dphi|
 * to the cell its diffracted ray crosses, when neither the source-to-edge nor
 * the edge-to-plane segment is blocked.  E_d follows Eq. diffracted-field
 * (diffraction coefficients D_1..D_4 with the UTD transition function, face
 * matrices R_0, R_n with the half-space Fresnel coefficients of both faces'
 * materials), for the transmitter's antenna field in the direction of the
 * diffraction point (pattern, orientation, polarisation(s), synthetic array).
 * The faces swap roles when the source lies behind the 0-face (the UTD
 * assumes phi' <= pi).  Uses params: freq_hz, map geometry, deposit (box or
 * bilinear), RM_STATS, block_size; other fields are ignored.
 * wedges_host: nw wedges (from rm_scene_wedges or any subset of them).
 * record_dev_or_null: [ntx][nw][samples_per_wedge] records {bits, ix, iy, 0},
 * bits = 1 incident segment blocked | 2 diffracted segment blocked, -1 no
 * crossing in the map, -2 source behind both faces.
 * stats: rays = samples, segments = samples reaching the map, deposits,
 * nodes_visited / tris_tested of the visibility queries, kernel_ms.
 * Errors: RM_EINVAL for bad arguments (nw * samples * ntx must stay below
 * 2^40); synchronises `stream`. */
rm_status rm_diffraction_map(const rm_scene* scene, const rm_wedge* wedges_host, int64_t nw, const rm_tx* tx_host,
                             int32_t ntx, const rm_trace_params* params, int64_t samples_per_wedge,
                             float* maps_dev, rm_stats* stats_host_or_null, rm_segment_record* record_dev_or_null,
                             void* stream);

/* The diffraction map on a mesh measurement surface (see
 * rm_radio_map_trace_mesh): maps_dev [ntx][surface triangles].  A sample
 * whose source-to-edge segment is unblocked deposits at every surface
 * triangle its diffracted ray crosses (t > 1e-9, at most 8 crossings; more
 * set RM_EOVERFLOW) when the edge-to-crossing segment is unblocked: the term
 * of rm_diffraction_map with the weighting factor taken on the triangle's
 * plane, 1 / A_i instead of 1 / Delta^2 and E_d at the crossing's distance.
 * Records {bits: 1 incident blocked, -2 source behind both faces; crossings
 * found; 0; 0}.  stats: segments = lit samples.  deposit must be 0;
 * otherwise as rm_diffraction_map. */
rm_status rm_diffraction_map_mesh(const rm_scene* scene, const rm_scene* surface, const rm_wedge* wedges_host,
                                  int64_t nw, const rm_tx* tx_host, int32_t ntx, const rm_trace_params* params,
                                  int64_t samples_per_wedge, float* maps_dev, rm_stats* stats_host_or_null,
                                  rm_segment_record* record_dev_or_null, void* stream);

/* Failure detection without a GPU fault: the next `count` checks of `kind`
 * (RM_FAULT_*) fail on the host with the status the real failure returns;
 * count 0 disarms.  The environment variable RM_FAULT=<alloc|launch|overflow>
 * [:count] arms one kind once per process.  The context stays usable: the
 * call after an injected failure runs normally.  RM_EINVAL for another kind
 * or count < 0. */
rm_status rm_debug_inject(int32_t kind, int32_t count);

/* The coin's weights of one interaction, from the tracer's own device code:
 * for material `mat` at freq_hz and each cosine of incidence cos1_dev[i] in
 * [0, 1], wR_dev[i] = |r_perp|^2 + |r_par|^2 and wT_dev[i] = |t_perp|^2 +
 * |t_par|^2 of Eq. fresnel_vac (half-space) or Eqs. fresnel_slab /
 * q_fresnel_slab (slab), so that q(R) = wR / (wR + wT) (Eq.
 * path-solver-used-dist-event with q(D) = 0).  The parity tests compare it
 * with the FP64 oracle at the same cosines to bound the FP32 error of the
 * sampling probabilities (in particular of the slab phase (2 pi d / lambda0) s).
 * Device arrays of n floats owned by the caller; asynchronous on `stream`;
 * RM_EINVAL for a NULL or invalid material, freq_hz <= 0 or n < 0. */
rm_status rm_debug_fresnel_probe(const rm_material* mat, double freq_hz, const float* cos1_dev, int64_t n,
                                 float* wR_dev, float* wT_dev, void* stream);

/* The synthetic-array factor alpha (see rm_tx.n_ant) of every work item of
 * the call (the transmitters' ray subsets in order, the tracer's work-item
 * order), from the pre-pass kernel of trace and gradient calls into
 * alpha_prepass_dev and from the tracer's inline form (graph plans, the
 * no-allocation entry point) into alpha_inline_dev, both [len][2] floats (re,
 * im) owned by the caller; entries of transmitters without an array are not
 * written.  Lets a test check that the two forms agree bit for bit.  No
 * counterpart in the paper (a test aid).  Synchronises `stream`; RM_EINVAL for
 * NULL buffers, len below the number of work items, or the arguments
 * rm_radio_map_trace rejects. */
rm_status rm_debug_array_factor(const rm_scene* scene, const rm_tx* tx_host, int32_t ntx,
                                const rm_trace_params* params, float* alpha_prepass_dev, float* alpha_inline_dev,
                                uint64_t len, void* stream);

/* Number of device and pinned-host allocation calls (cudaMalloc,
 * cudaMallocAsync, cudaHostAlloc) the library has made in this process since
 * it was loaded: tests read it before and after a call to check whether that
 * call allocated.  Host call, thread-safe, no device work. */
uint64_t rm_debug_alloc_count(void);

/* Number of triangles / internal BVH nodes of a scene (host call, no device
 * work); *built = the builder used (RM_BVH_LBVH or RM_BVH_SAH), 0 if none. */
rm_status rm_scene_info(const rm_scene* scene, int64_t* nt, int64_t* nnodes, int32_t* nm,
                        int32_t* built);

/* Frees the scene's device memory (waits for the device first).  Scene memory
 * comes from the device's default stream-ordered pool, whose release
 * threshold the library raises to 1 GiB for this process so that repeated
 * uploads reuse cached pages. */
void rm_scene_free(rm_scene* scene);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* rm_last_error(void);

/* Library version string. */
const char* rm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RMSBR_H */

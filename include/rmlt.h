/*
 * rmlt — regional adaptive primary-sample-space Metropolis light transport on
 * one GB300 (sm_103a).  C ABI of the CUDA library librmlt.so.
 *
 * The method is Regional Adaptive Metropolis Light Transport (Otsu, Herveau,
 * Hanika, Nowrouzezahrai, Dachsbacher): many Metropolis chains whose small-step
 * scale sigma_k = sqrt(exp(lambda_k)) is adapted per screen region k by the
 * Robbins-Monro rule of Alg. 1 (eqs. est_exp_acc, update_lambda,
 * step_size_n; Sec. 5.3) over the 2-D screen-space grid partition of
 * Sec. 5.4 / 6.1, with the MLT estimator I_j = (b/N) sum f/pi of Sec. 3.2.
 *
 * Conventions
 *  - Every function returns an rmlt_status; negative values are errors and
 *    rmlt_last_error() gives a message for the calling thread.  No C++
 *    exception or abort crosses this boundary.
 *  - Call order: rmlt_create -> rmlt_load_scene | rmlt_load_toy_integrand ->
 *    rmlt_init_chains -> rmlt_step* -> rmlt_read_* .  Out-of-order calls return
 *    RMLT_E_STATE and change nothing.  Loading a new scene discards the chains.
 *  - Input arrays are read during the call and copied; the caller keeps them.
 *  - Output buffers are caller-owned and may be host or device pointers (the
 *    library asks the CUDA driver which); device outputs are written on the
 *    context's stream and the call synchronises that stream before returning.
 *  - Device memory the library needs is obtained from the allocator installed
 *    with rmlt_set_allocator (the Python binding installs PyTorch's caching
 *    allocator), else from cudaMalloc.
 *  - A failed rmlt_step marks the context failed: later steps and reads return
 *    RMLT_E_STATE; rmlt_destroy is always safe.
 */
#ifndef RMLT_H
#define RMLT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RMLT_ABI_VERSION 7
#define RMLT_MAX_DEPTH 12          /* D = 2 + 5 d <= 62 primary-sample dimensions */

typedef struct rmlt_ctx rmlt_ctx;

typedef enum {
    RMLT_OK = 0,
    RMLT_E_INVALID_ARG = -1,
    RMLT_E_INVALID_SCENE = -2,
    RMLT_E_OOM = -3,
    RMLT_E_CUDA = -4,
    RMLT_E_STATE = -5,     /* wrong call order, or the context failed earlier */
    /* -6 is not used: no kernel of this library waits on another */
    RMLT_E_OVERFLOW = -7,  /* a device-side bound was exceeded (see rmlt_set_wave_limit and
                              rmlt_bootstrap_noalloc) */
    RMLT_E_IO = -8
} rmlt_status;

typedef enum { RMLT_LAMBERT = 0, RMLT_GGX = 1 } rmlt_material_type;
typedef enum { RMLT_TARGET_PLAIN = 0, RMLT_TARGET_REGION_WEIGHTED = 1 } rmlt_target_mode;
typedef enum { RMLT_PARTITION_GRID = 0, RMLT_PARTITION_QUADTREE = 1 } rmlt_partition;

typedef struct {
    int32_t type;          /* rmlt_material_type */
    float albedo[3];       /* Lambert albedo, or GGX Fresnel F0 (Schlick) */
    float emission[3];     /* radiance emitted from the front face (counter-clockwise winding) */
    float roughness;       /* GGX alpha */
} rmlt_material;

typedef struct {
    float pos[3], look_at[3], up[3];
    float vfov_deg;        /* vertical field of view of the pinhole camera */
} rmlt_camera;

typedef struct {
    int32_t n_verts;
    const float* verts;        /* [n_verts][3] host */
    int32_t n_tris;
    const uint32_t* tris;      /* [n_tris][3] vertex indices, host */
    const uint32_t* mat_id;    /* [n_tris] host */
    int32_t n_mats;
    const rmlt_material* mats; /* [n_mats] host */
    rmlt_camera camera;
    int32_t brute_force_max;   /* scenes with n_tris <= this skip the BVH (0: default 64) */
    int32_t bvh_width;         /* 2 or 4 children per BVH node (0: default 4) */
} rmlt_scene_desc;

/* Chain parameters (Alg. 1 and Sec. 7.1 names).  D = 2 + 5 max_depth. */
typedef struct {
    int32_t n_chains;          /* C independent chains */
    int32_t width, height;     /* image size W x H */
    int32_t region_px;         /* grid partition: regions of region_px^2 pixels (Sec. 6.1) */
    int32_t max_depth;         /* d surface interactions, NEE at each, 1..RMLT_MAX_DEPTH (0: toy) */
    int32_t epoch_len;         /* E mutations per chain between region updates */
    int32_t L;                 /* visits per region before an update (Alg. 1) */
    int32_t target_mode;       /* rmlt_target_mode */
    int64_t n_bootstrap;       /* uniform samples for b and the initial states (Sec. 3.2) */
    uint64_t seed;             /* Philox4x32-10 key */
    double p_large;            /* probability of the large (independent) step */
    double s1, s2;             /* Kelemen small-step offset range [sigma s1, sigma s2] */
    double alpha_star;         /* target acceptance (Sec. 5.3; 0.5 in Sec. 7.1) */
    double gamma_max, gamma_scale;  /* eq. step_size_n */
    double lambda_init, lambda_min;
    /* upper clamp of lambda_k.  0 or NaN selects the largest value the
     * kernel allows: 2 ln(1 / (2 s2)) for Kelemen's kernel (sigma s2 <= 1/2,
     * the largest offset on the torus) and 2 ln 4 for the truncated normal
     * (sigma <= 4, beyond which it is uniform on the window).  The paper
     * (Sec. 7.1) bounds lambda only from below. */
    double lambda_max;
    double w_floor;            /* region-weighted target: lower bound of w_k as a share of 1/m */
    int32_t partition;         /* RMLT_PARTITION_GRID (Sec. 6.1) or RMLT_PARTITION_QUADTREE (Sec. 6.2) */
    int32_t qt_max_leaves;     /* quadtree: region capacity */
    int32_t qt_max_depth;      /* quadtree: deepest level (the root is level 0) */
    int32_t qt_pad_;
    int64_t qt_split;          /* quadtree: M_split, visits since the last pass that split a leaf */
    int64_t qt_refine;         /* quadtree: M_refine, mutations (all chains) between passes */
    /* Langevin (MALA) strategy, an extension beyond the paper: with probability
     * p_mala a mutation proposes y = x + m + sqrt(tau) xi, tau = mala_tau
     * sigma_{k(x)}^2 (the region's adapted scale), m = (tau / 2) grad log pi(x)
     * scaled to norm <= mala_drift_max, xi standard normal; the acceptance
     * carries the ratio of the state-dependent proposal densities.  Its moves
     * do not feed the adaptation statistics.  Needs a Lambertian scene (or the
     * toy integrand) and the chain kernel.  0 = off. */
    double p_mala, mala_tau, mala_drift_max;
    /* small-step kernel: RMLT_KERNEL_KELEMEN (log-uniform offsets on
     * [sigma s1, sigma s2], random sign) or RMLT_KERNEL_TRUNCNORM (the
     * paper's family, Sec. 5.2: a normal of standard deviation sigma_k
     * truncated to the torus window (-1/2, 1/2); lambda_max <= 2 ln 4).  Both
     * perturb every dimension with the sigma of the current state's region;
     * the acceptance carries the reverse kernel of the proposal's region. */
    int32_t kernel;
    /* 4-D partition in primary sample space (the analogue of the paper's 4-D
     * partition, Sec. 5.4): each screen region is crossed with a dir_cells x
     * dir_cells grid over the first bounce's BSDF coordinates (u5, u6), so
     * m = regions on screen x dir_cells^2.  0 or 1 = screen only.  Needs the
     * grid partition, the plain target, max_depth >= 1 and no Langevin
     * strategy; not for batched members. */
    int32_t dir_cells;
    /* Sharding over several GPUs (one context per GPU): this context owns the
     * chains with global ids chain_first .. chain_first + n_chains - 1 of a
     * population of chains_total (0 = n_chains: not sharded).  Philox streams
     * are keyed by the global id, and every context evaluates all
     * n_bootstrap samples (so b and the starting states do not depend on the
     * split).  A sharded context advances with rmlt_epoch_mutate /
     * rmlt_epoch_update around a sum of the region statistics over all
     * contexts (Sec. 6: the paper's threads share i_k and A_k the same
     * way); rmlt_step refuses it. */
    int32_t chain_first, chains_total;
} rmlt_chain_params;
#define RMLT_KERNEL_KELEMEN 0
#define RMLT_KERNEL_TRUNCNORM 1

typedef struct {
    uint64_t mutations;        /* per chain, since rmlt_init_chains */
    uint64_t accepted, large, small, early_reject, invalid_paths;
    uint64_t rays;             /* closest-hit + shadow rays traced by rmlt_step */
    uint64_t stack_overflow;   /* paths dropped because the traversal stack overflowed */
    uint64_t epochs;
    double bhat;               /* bootstrap normaliser b (Sec. 3.2) */
    int32_t n_regions, dims;
    uint64_t node_visits;      /* BVH internal nodes visited (only while work counters are on) */
    uint64_t tri_tests;        /* ray-triangle tests in BVH leaves (only while work counters are on) */
    uint64_t sched[6];         /* work counters on: warp loop iterations, traversing lanes summed over
                                  them, shade batches, lanes shaded, setup batches, lanes set up;
                                  wavefront form, of the trace kernel's warp loop: iterations, lanes
                                  stepping, lanes holding a ray, leaf turns, lanes waiting at a leaf
                                  during node turns, iterations after the ray queue ran dry */
    uint64_t cycles[5];        /* work counters on: SM cycles warps spent in traversal steps, shade
                                  batches, finish/setup batches; warp lifetimes (sum, max) */
    uint64_t waves;            /* wavefront form: waves run (one trace pass each), summed over epochs */
    uint64_t wave_limit_hits;  /* wavefront form: epochs stopped by the wave limit (0 unless a bug) */
    uint64_t mala, mala_accepted;   /* Langevin moves proposed and accepted */
    uint64_t boot_overflow;    /* bootstrap paths dropped because the traversal stack overflowed */
    uint32_t node_bytes;       /* bytes per BVH node of the loaded scene (128 BVH4, 64 quantised BVH4 or
                                  BVH2; 0 without a BVH) */
    uint32_t pad_;
} rmlt_stats;

/* One record per traced mutation (test instrument, see rmlt_set_trace). */
typedef struct {
    float f[3];                /* contribution of the proposal y (0 if rejected early) */
    float a;                   /* acceptance probability */
    uint32_t qhash;            /* FNV-1a of the proposal's D words */
    uint32_t flags;            /* bit 0 accepted, 1 large step, 2 early reject, 3 invalid, 4 Langevin move */
} rmlt_trace_record;

typedef void* (*rmlt_alloc_fn)(void* user, size_t bytes, void* stream);
typedef void (*rmlt_free_fn)(void* user, void* ptr, void* stream);

/* Create a context on CUDA device `device`, issuing all work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * handle.  Errors: RMLT_E_INVALID_ARG (out NULL), RMLT_E_CUDA (no device). */
rmlt_status rmlt_create(rmlt_ctx** out, int device, void* cuda_stream);

/* Route the context's device allocations through alloc/free (both non-NULL),
 * or back to cudaMalloc/cudaFree (both NULL).  Only before rmlt_load_scene.
 * An allocation that returns NULL fails the call with RMLT_E_OOM; a failed
 * rmlt_load_scene, rmlt_init_chains or rmlt_restore leaves the context as it
 * was (its previous scene and chains stay usable). */
rmlt_status rmlt_set_allocator(rmlt_ctx* ctx, rmlt_alloc_fn alloc, rmlt_free_fn free_fn, void* user);

/* Copy the scene, build a binned-SAH BVH on the host (or keep a flat list when
 * n_tris <= brute_force_max) and upload nodes, triangles, materials and the
 * light list (emitting triangles, sampled by area).  The paper's path integral
 * (Sec. 3.1) is over this geometry.  Errors: RMLT_E_INVALID_SCENE (index out
 * of range, non-finite vertex, unknown material type, no triangle),
 * RMLT_E_OOM, RMLT_E_CUDA. */
rmlt_status rmlt_load_scene(rmlt_ctx* ctx, const rmlt_scene_desc* scene);

/* Test scene: D = 2, identity path map, f(u) = p0 + p1 1[u in box] +
 * p6 exp(-|u - (p7, p8)|^2 / (2 p9^2)), box [p2,p3) x [p4,p5).  params: 10
 * doubles, host.  Requires max_depth = 0 in rmlt_init_chains. */
rmlt_status rmlt_load_toy_integrand(rmlt_ctx* ctx, const double* params);

/* Allocate chain state and region tables, run the bootstrap (n_bootstrap
 * uniform samples -> b, Sec. 3.2 "preprocess"), give each chain g (global id)
 * the sample where the cumulative sum of pi over all K C samples (K =
 * n_bootstrap / chains) first exceeds (g + u_g) / chains of the total, u_g a
 * uniform of its own (systematic resampling in proportion to pi, so no chain
 * starts on a path that contributes nothing while any sample does), and set
 * lambda_k = lambda_init, i_k = A_k = 0, n_k = 1 (Alg. 1, initialisation).
 * Bootstrap paths dropped by a traversal-stack overflow are counted in
 * rmlt_stats.boot_overflow.  On error the context keeps its previous chains.
 * Errors: RMLT_E_INVALID_ARG (non-positive sizes, max_depth out of range,
 * s1 >= s2, p_large outside [0,1], lambda bounds outside [-150, the kernel's
 * maximum] ...), RMLT_E_STATE (no scene), RMLT_E_OOM, RMLT_E_CUDA. */
rmlt_status rmlt_init_chains(rmlt_ctx* ctx, const rmlt_chain_params* params);

/* Advance every chain by n_mutations Metropolis-Hastings mutations (Alg. 1,
 * mutation loop), rounded up to whole epochs of epoch_len, with the region
 * update (Alg. 1, region update; at most one per region per epoch) at each epoch
 * boundary.  Asynchronous on the context's stream (no host synchronisation);
 * launch errors are returned here, execution errors at the next synchronising
 * call.  A proposal whose ray overflows the traversal stack is given zero
 * contribution and counted in rmlt_stats.stack_overflow.  RMLT_E_STATE for a
 * sharded context (use rmlt_epoch_mutate / rmlt_epoch_update). */
rmlt_status rmlt_step(rmlt_ctx* ctx, uint64_t n_mutations);

/* Sharded stepping, one epoch at a time (Alg. 1 with the region statistics
 * summed over every context of a population split by chain_first /
 * chains_total; Sec. 6 "Implementation": all chains share i_k and A_k).
 *   rmlt_exchange_size: *n_counts u64 words and *n_sums doubles of the two
 *     exchange buffers (3 m + 1 and m, m the region capacity).
 *   rmlt_epoch_mutate: E mutations of every chain of this context (Alg. 1,
 *     mutation step), then writes what this epoch added to the region
 *     tables to the caller's device buffers: counts = [i_k (m)][A_k (m)]
 *     [h_k (m)][large steps (1)], sums = [sum of pi over the large-step
 *     proposals per region (m)].
 *   rmlt_epoch_update: takes the same buffers after the caller summed them
 *     over all contexts (an all-reduce; u64 sums wrap, so a signed 64-bit
 *     reduction gives the same bits), sets every table to its value at the
 *     start of the epoch plus the sums, and runs the region update (Alg. 1,
 *     region update), the weight update of the weighted target and a due
 *     quadtree pass.  Every context then holds identical region tables.
 * An unsharded context may use them too (the buffers passed through
 * unchanged give exactly rmlt_step(epoch_len)).  Both are asynchronous on the
 * context's stream; the buffers must be device memory.  Errors: RMLT_E_STATE
 * (no chains, failed, or the two calls out of order), RMLT_E_INVALID_ARG
 * (NULL or host buffers, the Langevin strategy), RMLT_E_CUDA. */
rmlt_status rmlt_exchange_size(rmlt_ctx* ctx, int64_t* n_counts, int64_t* n_sums);
rmlt_status rmlt_epoch_mutate(rmlt_ctx* ctx, uint64_t* counts, double* sums);
rmlt_status rmlt_epoch_update(rmlt_ctx* ctx, const uint64_t* counts, const double* sums);

/* Image estimate, [height][width][3] doubles.  normalized = 1: radiance
 * I_j * W * H with I_j = (b/N) sum_i f(x_i)/pi(x_i) (Sec. 3.2; region-weighted
 * mode normalises each region by its own mass); normalized = 0: the raw sum
 * of f/pi splats.  A sharded context returns its chains' share, normalised
 * with the whole population's N, b and region masses: the sum of the shares
 * of all contexts is the image. */
rmlt_status rmlt_read_image(rmlt_ctx* ctx, double* out_rgb, int normalized);

/* Region visit histogram h_k (post-MH state of every mutation), [m] u64, m
 * the current number of regions (rmlt_stats.n_regions; it grows with a
 * quadtree partition, and a split leaf's children start from 0). */
rmlt_status rmlt_read_region_hist(rmlt_ctx* ctx, uint64_t* out_h);

/* Region parameters, each [m]; any pointer may be NULL.  lambda_k, n_k (update
 * count, starts at 1), i_k and A_k (visits and 2^32-scaled acceptance sum since
 * the region's last update), w_k (region weight; 1 in plain mode). */
rmlt_status rmlt_read_region_params(rmlt_ctx* ctx, double* lambda, int64_t* n, uint64_t* i,
                                    uint64_t* A, double* w);

/* Quadtree partition (Sec. 6.2): regions are the leaves of a quadtree over
 * the screen [0,1)^2, starting from the root.  Once every qt_refine mutations
 * (counted over all chains, at an epoch boundary) each leaf visited more than
 * qt_split times since the previous pass splits into four children, which
 * inherit lambda and n_k / 4 (at least 1) and are not split again in the same
 * pass; the first child keeps the parent's region id.  This call copies the
 * tree: child [nodes][4] (-1 for a leaf; child j covers the quadrant with
 * x bit j & 1 and y bit j >> 1), leaf [nodes] (region id, -1 when internal),
 * depth [nodes], at most cap_nodes nodes; *n_nodes receives the node count.
 * RMLT_E_STATE for a grid partition. */
rmlt_status rmlt_read_quadtree(rmlt_ctx* ctx, int32_t* child, int32_t* leaf, int32_t* depth, int32_t cap_nodes,
                               int32_t* n_nodes);

/* Chain states in the device's structure-of-arrays layout: q [D][n_chains]
 * u32 primary-sample words (u = q 2^-32), f [3][n_chains] float contribution,
 * k [n_chains] region.  Any may be NULL. */
rmlt_status rmlt_read_chain_state(rmlt_ctx* ctx, uint32_t* q, float* f, int32_t* k);

rmlt_status rmlt_read_stats(rmlt_ctx* ctx, rmlt_stats* out);

/* The chain parameters in effect (defaults resolved, e.g. lambda_max), as
 * given to rmlt_init_chains or read from a checkpoint by rmlt_restore. */
rmlt_status rmlt_read_params(rmlt_ctx* ctx, rmlt_chain_params* out);

/* Test instrument.  While set, rmlt_step writes one rmlt_trace_record per
 * mutation of every chain c with c % chain_stride == 0, in the order
 * [epoch][traced chain][mutation in epoch], to `records` (device memory, room
 * for `capacity` records), and lambda after each epoch's update, [epoch][m]
 * doubles, to `lambdas` (device, room for `lambda_capacity` doubles; may be
 * NULL).  Tracing stops silently when a buffer is full.  records = NULL
 * switches tracing off.  The traced kernel is the production kernel with the
 * record stores enabled. */
rmlt_status rmlt_set_trace(rmlt_ctx* ctx, rmlt_trace_record* records, uint64_t capacity,
                           double* lambdas, uint64_t lambda_capacity, uint32_t chain_stride);
/* Test instrument, with rmlt_set_trace: each record's D proposal words y (u32)
 * are also written to words[record][D] (device memory, capacity_words >=
 * capacity x D), so that a replay can adopt proposals whose last bits depend
 * on binary32 rounding (truncated-normal offsets, Langevin moves).
 * rmlt_set_trace clears it; words = NULL switches it off. */
rmlt_status rmlt_set_trace_words(rmlt_ctx* ctx, uint32_t* words, uint64_t capacity_words);

/* Gradient of log pi(u), pi = l(f(u)), at n points: q [D][n] u32 primary-
 * sample words (u = q 2^-32, D = 2 + 5 max_depth of the chains, 2 for the toy
 * integrand), all device memory.  Outputs (each may be NULL): f [3][n] float,
 * logpi [n] float (-inf where pi = 0), grad [D][n] float, d log pi / d u.
 * Evaluated by the chain kernel's path functions with a record of each
 * bounce, then an adjoint sweep from the last bounce back to the camera
 * (reverse-mode differentiation); hits, light choice and visibility are held
 * fixed, so this is the gradient of the smooth piece of f containing u, and 0
 * where pi = 0.  Lambertian and emitting surfaces only.  Needs
 * rmlt_init_chains (depth, image size); asynchronous on the context stream.
 * Errors: RMLT_E_STATE, RMLT_E_INVALID_ARG (host pointers, a GGX scene),
 * RMLT_E_CUDA. */
rmlt_status rmlt_path_grad(rmlt_ctx* ctx, const uint32_t* q, int64_t n, float* f, float* logpi, float* grad);

/* grad log pi of the chains' current states, [D][n_chains] floats (host or
 * device), for chains with the Langevin strategy.  A state reached by another
 * strategy holds NaN in dimension 0 until a Langevin move needs its gradient.
 * RMLT_E_STATE without the Langevin strategy. */
rmlt_status rmlt_read_chain_grad(rmlt_ctx* ctx, float* g);

/* Measurement instruments for the traversal roofline.
 * rmlt_record_paths: the paths of n points q [D][n] (device; D = 2 + 5
 * max_depth of the chains) evaluated with the chain kernel's own path and
 * traversal functions.  Every ray cast is written to rays [n][2 max_depth][8]
 * floats (origin xyz, tmax, direction xyz, 1 for a shadow ray; tmax = -1
 * marks an unused slot) and what the traversal found and did for it to work
 * [n][2 max_depth][4] u32 (hit triangle's original index or 0xFFFFFFFF,
 * distance as float bits, BVH internal nodes visited, triangles tested).
 * Device outputs, asynchronous on the context's stream.
 * rmlt_walk_rays_host: the same ray records (host [n][8]) walked on the host
 * in binary64 through the uploaded BVH, nearest child first: an independent
 * reference traversal of the same nodes and triangles.  out (host) [n][4]
 * u32 as for work.  Errors: RMLT_E_STATE (no scene / chains, the toy
 * integrand), RMLT_E_INVALID_ARG. */
rmlt_status rmlt_record_paths(rmlt_ctx* ctx, const uint32_t* q, int64_t n, float* rays, uint32_t* work);
rmlt_status rmlt_walk_rays_host(rmlt_ctx* ctx, const float* rays, int64_t n, uint32_t* out);

/* Count BVH node visits and triangle tests in rmlt_stats (enable = 1), using
 * an instrumented build of the same chain kernel; enable = 0 returns to the
 * uninstrumented kernel.  The chain trajectory does not depend on it. */
rmlt_status rmlt_set_work_counters(rmlt_ctx* ctx, int enable);

/* Scheduling knobs of the chain kernel: a warp shades the resolved rays of its
 * lanes once at least `batch_shade` of them are waiting, and finishes
 * mutations / draws proposals once `batch_setup` lanes are waiting (both in
 * 1..32; smaller values when nothing else is left).  flags:
 * RMLT_TUNE_LARGE_AHEAD traces the epoch's large-step proposals (independent
 * of the chain states) in a separate kernel before the chain kernel;
 * RMLT_TUNE_ADAPTIVE_BATCH shrinks the batches as lanes finish the epoch.
 * They change speed only, never results.  Defaults 12, 10, 0. */
#define RMLT_TUNE_LARGE_AHEAD 1
#define RMLT_TUNE_ADAPTIVE_BATCH 2
/* RMLT_TUNE_WAVEFRONT runs each epoch in the wavefront form instead of the
 * chain kernel: the epoch advances in waves; in each wave every chain with
 * rays in flight shades its hits (the shadow ray of bounce b and the
 * extension ray of bounce b + 1 are traced together), the chains whose path
 * ended accept or reject and draw their next proposal, and a persistent trace
 * kernel resolves all queued rays.  A CUDA graph repeats the wave on the
 * device until no chain has a ray left.  The results are identical to the
 * chain kernel's (same arithmetic per path, same Philox draws). */
#define RMLT_TUNE_WAVEFRONT 4
rmlt_status rmlt_set_tuning(rmlt_ctx* ctx, int batch_shade, int batch_setup, int flags);

/* Launch shape of the wavefront form: resident blocks of 128 threads per SM
 * for the persistent trace kernel and for the finish / setup kernel (0 = as
 * many as fit), and how many lanes of a trace warp must be idle before they
 * pull new rays together (1..32).  flags: RMLT_WAVEFRONT_HOST_LOOP launches
 * the waves from the host (a fixed E (max_depth + 1) + 2 waves per epoch, the
 * surplus ones empty) instead of the graph's device-side loop; profilers that
 * cannot see into conditional graphs need it.  Speed only.  Defaults 0, 0, 8,
 * 0. */
#define RMLT_WAVEFRONT_HOST_LOOP 1
/* RMLT_WAVEFRONT_SHORT_STACK: the persistent trace kernel keeps 16 of each
 * ray's 48 traversal-stack entries in shared memory and the deeper ones in a
 * per-thread area of device memory (about 40 MB, part of the wavefront
 * state), which leaves more of each SM's memory to the L1 cache.  Speed only. */
#define RMLT_WAVEFRONT_SHORT_STACK 2
rmlt_status rmlt_set_wavefront(rmlt_ctx* ctx, int trace_ctas_per_sm, int setup_ctas_per_sm, int refill_lanes,
                               int flags);

/* Safety bound of the wavefront form: an epoch stops after `waves` waves (0 =
 * the default E (max_depth + 1) + 2, more than any epoch needs, since every
 * wave advances each chain with rays by one bounce).  An epoch stopped by the
 * bound leaves mutations unfinished; the next synchronising call
 * (rmlt_synchronize, rmlt_read_*, rmlt_save) then returns RMLT_E_OVERFLOW and
 * marks the context failed. */
rmlt_status rmlt_set_wave_limit(rmlt_ctx* ctx, uint32_t waves);

/* Node layout of the BVH4 that the next rmlt_load_scene builds (no counterpart
 * in the paper).  RMLT_NODES_FLOAT: 128-byte nodes with the children's
 * binary32 bounds.  RMLT_NODES_QUANTISED: 64-byte nodes, the children's boxes
 * as 8-bit indices on a per-node grid, rounded outward (more boxes pass, the
 * same hits are found), which halves the node bytes a ray reads for a decode
 * per plane.  RMLT_NODES_AUTO (the default): quantised when the binary32 nodes
 * and the triangles would take more than 48 MB, a third of the GPU's L2,
 * where node loads miss the cache often enough for the halving to pay.
 * Results do not depend on the layout beyond which of two triangles at the
 * same distance is reported.  Errors: RMLT_E_INVALID_ARG. */
#define RMLT_NODES_AUTO 0
#define RMLT_NODES_FLOAT 1
#define RMLT_NODES_QUANTISED 2
rmlt_status rmlt_set_node_format(rmlt_ctx* ctx, int format);

/* Leaf turns of the wavefront form's trace kernel: a warp's lanes whose ray
 * waits at a BVH leaf test its triangles together once at least leaf_batch
 * of them are there (1..32; default 8).  Speed only. */
rmlt_status rmlt_set_trace_leaf_batch(rmlt_ctx* ctx, int leaf_batch);

/* Bootstrap without any device allocation.  Some callers cannot allocate
 * device memory at the point where they need starting states: code running
 * inside a memory-pool or arena callback, a process whose allocator is
 * reserved by a framework, or a caller that must not grow its footprint.
 * This entry point runs the same bootstrap as rmlt_init_chains (n_bootstrap
 * uniform samples, the normaliser b of Sec. 3.2 and one pi-proportional
 * starting state per chain) on the loaded scene, and writes the results to the
 * caller's buffers without touching the context's chains.  The paper has no
 * counterpart; it is a deployment convenience.
 *   out_q     device, [D][n_chains] u32 starting states (D = 2 + 5 max_depth)
 *   out_f     device, [3][n_chains] float contributions of those states
 *   out_bhat  host or device, one double: b
 * Its intermediate values live in one fixed array inside the library (about
 * 5.9 MB, held on every GPU that loads the library until the process exits),
 * so it calls no cudaMalloc, cudaFree or allocating library routine.  Limits:
 * (n_bootstrap / n_chains) * n_chains <= RMLT_NOALLOC_MAX_SAMPLES, n_chains <=
 * RMLT_NOALLOC_MAX_CHAINS, regions <= RMLT_NOALLOC_MAX_REGIONS; larger sizes
 * return RMLT_E_INVALID_ARG.  The first call on a device looks the array up
 * (cudaGetSymbolAddress) and should come before any stream capture.  Every
 * call shares the array, so calls whose work overlaps on the GPU (other
 * contexts, other streams) race; serialise them.  Errors: RMLT_E_STATE (no
 * scene), RMLT_E_INVALID_ARG (parameters, sizes, host pointers for out_q or
 * out_f), RMLT_E_OVERFLOW (a bootstrap path overflowed the traversal stack,
 * so b and the starting states would be biased; the outputs are written),
 * RMLT_E_CUDA. */
#define RMLT_NOALLOC_MAX_SAMPLES (1 << 18)
#define RMLT_NOALLOC_MAX_CHAINS (1 << 16)
#define RMLT_NOALLOC_MAX_REGIONS (1 << 14)
rmlt_status rmlt_bootstrap_noalloc(rmlt_ctx* ctx, const rmlt_chain_params* params, uint32_t* out_q,
                                   float* out_f, double* out_bhat);

/* Batched stepping.  A batch advances several contexts (their own scenes,
 * resolutions, region grids and chain counts, of any size) together: per
 * epoch, one launch of the chain kernel covers the chains of every member,
 * block by block, and one launch runs every member's region update (Alg. 1,
 * region update); the two are a CUDA graph captured once and replayed per
 * epoch.  Each member's trajectory is exactly the one rmlt_step gives it (the
 * same kernel body, Philox streams and order of updates); only the launch is
 * shared, so small populations fill the GPU together.  Members must be on
 * one device, have chains, share epoch_len, use a BVH scene (more triangles
 * than brute_force_max), not have the wavefront form set, and be unsharded;
 * large steps are traced in the chain kernel.  A member with the trace
 * instrument set is traced as by rmlt_step (one-launch mode only).  The batch
 * holds the member handles, not their ownership: destroy the batch before its
 * members.  rmlt_batch_step orders itself after and before each member's
 * stream, so rmlt_read_* on a member sees its result.  Errors:
 * RMLT_E_INVALID_ARG, RMLT_E_STATE (a member not ready or failed), RMLT_E_CUDA. */
typedef struct rmlt_batch rmlt_batch;
rmlt_status rmlt_batch_create(rmlt_batch** out, rmlt_ctx* const* members, int n_members);
/* Launch order of the members' blocks (a permutation of 0..n-1); speed only.
 * Blocks of earlier members start first, so putting the slowest members first
 * shortens the launch's tail. */
rmlt_status rmlt_batch_set_order(rmlt_batch* batch, const int* order);
/* Launch shape of the batch; speed only.  ctas_per_sm: resident blocks of
 * 128 chains per SM the batched chain kernel is compiled for, 4 (128
 * registers, a few spilled) or 3 (none spilled).  mode: RMLT_BATCH_ONE_LAUNCH
 * (one chain-kernel launch for all members per epoch, so every member waits
 * at each epoch boundary for the slowest block) or RMLT_BATCH_BRANCHES (one
 * graph per rmlt_batch_step call in which each member's epochs form their own
 * chain of launches of the single-context chain kernel, so fast members run
 * ahead; ctas_per_sm does not apply).  Defaults 4, RMLT_BATCH_ONE_LAUNCH. */
#define RMLT_BATCH_ONE_LAUNCH 0
#define RMLT_BATCH_BRANCHES 1
rmlt_status rmlt_batch_set_shape(rmlt_batch* batch, int ctas_per_sm, int mode);
/* n_mutations per chain of every member, rounded up to whole epochs. */
rmlt_status rmlt_batch_step(rmlt_batch* batch, uint64_t n_mutations);
void rmlt_batch_destroy(rmlt_batch* batch);

/* Ceilings of the traversal roofline on `device`, measured by two
 * microbenchmarks on `cuda_stream`: the aggregate L2 read bandwidth
 * (16-byte loads that bypass L1, over a buffer of a quarter of the L2 that
 * stays resident) in GB/s, and the FP32 fused multiply-add rate (eight
 * independent chains per thread, 2 flops each) in TFLOP/s.  A ray's BVH node
 * and triangle fetches draw on the first, its slab and triangle tests on the
 * second.  Allocates and frees a scratch buffer of that size.  Errors:
 * RMLT_E_INVALID_ARG (NULL output), RMLT_E_OOM, RMLT_E_CUDA. */
rmlt_status rmlt_probe_peaks(int device, void* cuda_stream, double* l2_read_gbs, double* fp32_tflops);

/* Bytes of device memory the context holds. */
rmlt_status rmlt_memory_usage(rmlt_ctx* ctx, uint64_t* bytes);

/* Checkpoint: chain state, region tables, image, counters, parameters and the
 * mutation index (Philox counters make resume-then-run equal an uninterrupted
 * run), with a 64-bit FNV-1a checksum of the header and payload.
 * rmlt_restore needs the same scene loaded; it checks the checksum, the
 * parameters and every index the kernels use (chain regions, quadtree sizes,
 * children and leaves) on the host before anything is launched, and leaves
 * the context unchanged on error.  Errors: RMLT_E_IO (cannot read, or
 * truncated), RMLT_E_INVALID_ARG (another scene or version, a checksum
 * mismatch, an index out of range). */
rmlt_status rmlt_save(rmlt_ctx* ctx, const char* path);
rmlt_status rmlt_restore(rmlt_ctx* ctx, const char* path);

/* Wait for the context's stream; returns a pending execution error. */
rmlt_status rmlt_synchronize(rmlt_ctx* ctx);

void rmlt_destroy(rmlt_ctx* ctx);
const char* rmlt_last_error(void);
int rmlt_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif

/*
 * CPU oracle for Regional Adaptive Metropolis Light Transport (Otsu, Herveau,
 * Hanika, Nowrouzezahrai, Dachsbacher) restated in primary sample space.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product path (the
 * CUDA library) never includes, links or calls it, and this code includes
 * nothing from the product.
 *
 * Plain, slow, single-threaded, binary64 everywhere except where a floating
 * point value decides an integer that both sides must agree on bit for bit
 * (the quantised small-step offset and the per-region step scale sigma_k):
 * those are taken in binary32 with an explicitly ordered sequence of
 * correctly rounded operations, the same precision the kernel decides them in.
 *
 * Section / equation references are to the paper:
 *   Sec. 3.1  path integral, I_j = int h_j f dmu; target pi = l(f)
 *   Sec. 3.2  MH acceptance, estimator I_j ~ (b/N) sum f/pi, strategy mixture
 *   Sec. 3.3  perturbation kernels parameterised by a scale sigma
 *   Sec. 5.2  state-dependent proposal T(.|x) = sum_k 1_{P_k}(x) T_k(.|x)
 *   Sec. 5.3  est_exp_acc (acceptance estimate), update_lambda, step_size_n
 *   Sec. 5.4  2-D screen-space partition
 *   Alg. 1    regional adaptive sample generation
 *   App. B    region independence, b_k = P(x in P_k)
 */
#ifndef RMLT_ORACLE_H
#define RMLT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* 2^t in binary32 (own routine: rint range reduction + degree-7 Taylor). */
float or_exp2_f32(float t);

/* Magnitude (units of 2^-32) of one Kelemen small-step offset. */
int64_t or_kelemen_delta(uint32_t xmag, float sigma_s2, float log2_ratio);
/* Truncated-normal small-step offset in units of 2^-32 for the 24-bit
 * uniform of xmag: sigma sqrt(2) erfinv((2u - 1) Z), Z = erf(1 / (2 sqrt(2) sigma)). */
int64_t or_truncnorm_delta(uint32_t xmag, double sigma);

typedef struct or_scene or_scene;
typedef struct or_ctx or_ctx;

typedef struct {
    int32_t  n_chains;
    int32_t  width, height, region_px;
    int32_t  max_depth;        /* d: surface interactions; D = 2 + 5 d      */
    int32_t  epoch_len;        /* E mutations per chain between updates      */
    int32_t  L;                /* visits before a region update (Alg. 1)     */
    int32_t  target_mode;      /* 0 plain pi, 1 region-weighted pi / w_k     */
    int64_t  n_bootstrap;
    uint64_t seed;
    double   p_large, s1, s2;
    double   alpha_star, gamma_max, gamma_scale;
    double   lambda_init, lambda_min, lambda_max;
    double   w_floor;
    int32_t  debug_flags;      /* tests only: bit 0 drops the reverse-kernel factor,
                                  bit 1 the Langevin proposal-density ratio */
    int32_t  partition;        /* 0 uniform grid (Sec. 6.1), 1 quadtree (Sec. 6.2) */
    int32_t  qt_max_leaves, qt_max_depth;
    int64_t  qt_split;         /* M_split: visits since the last pass that split a leaf */
    int64_t  qt_refine;        /* M_refine: mutations between refinement passes */
    /* Langevin (MALA) strategy: probability, step tau (scaled by sigma_k^2 of
     * the current state's region) and the bound on the drift's norm */
    double   p_mala, mala_tau, mala_drift_max;
    /* small-step kernel: 0 Kelemen (log-uniform offsets), 1 truncated normal of
     * standard deviation sigma_k on the torus window (-1/2, 1/2) */
    int32_t  kernel;
    /* 4-D partition: each screen region crossed with a dir_cells^2 grid over
     * (u5, u6), the first bounce's BSDF coordinates; <= 1 screen only */
    int32_t  dir_cells;
    /* sharded population: this context's chains are the global chains
     * chain_first .. chain_first + n_chains - 1 of chains_total (0: not
     * sharded); Philox draws are keyed by the global id */
    int32_t  chain_first, chains_total;
} or_params;

/* Gradient of log pi(u), pi = l(f(u)), over the D = 2 + 5 max_depth
 * coordinates (2 for the toy integrand), by forward-mode differentiation in
 * binary64 along the path the primal walk takes (hits, light choice and
 * visibility fixed).  f receives f(u).  Returns 1 (grad = 0 where pi = 0),
 * 0 when the path meets a non-Lambertian surface it would differentiate
 * through or is not finite (grad = 0), -1 when D exceeds 62. */
int32_t or_path_grad(const or_scene* s, int32_t width, int32_t height, int32_t max_depth,
                     const uint32_t* q, double f[3], double* grad);

/* Per-mutation hook (tests only): sees the proposal and may override the
 * proposal's contribution, acceptance probability and decision.  dec and
 * ferr are the binary32 error model of the proposal's path (see
 * or_path_eval_err). */
typedef void (*or_mut_hook)(void* user, uint32_t chain, uint64_t mut,
                            const uint32_t* qy, int32_t D, int32_t large,
                            int32_t early_reject, double dec, const double* ferr, double xi_accept,
                            double* f_y, double* a, int32_t* accept);
/* Proposal hook (tests only): sees each proposal qy right after it is drawn
 * (kind 0 small step, 1 large step, 2 Langevin move) and may replace its
 * words; everything after (regions, kernel ratio, path, acceptance) uses the
 * words it leaves. */
typedef void (*or_prop_hook)(void* user, uint32_t chain, uint64_t mut, int32_t kind, uint32_t* qy, int32_t D);
/* Region-update hook (tests only): may override sgn(alpha_hat - alpha*). */
typedef void (*or_upd_hook)(void* user, int32_t k, uint64_t i_k, uint64_t A_k,
                            double alpha_hat, int32_t* sign);

or_scene* or_scene_create(int32_t nv, const float* verts, int32_t nt, const uint32_t* tris,
                          const uint32_t* mat_id, int32_t nm, const int32_t* mat_type,
                          const float* albedo, const float* emission, const float* roughness,
                          const float* camera, int32_t use_bvh);
or_scene* or_scene_create_toy(const double* params10);
/* Tests only, a planted mistake: next-event light triangles chosen uniformly
 * instead of by area. */
void      or_scene_plant_uniform_lights(or_scene* s);

/* One GGX lobe (roughness alpha, Schlick F0) in the local frame n = (0,0,1),
 * the code the path map uses, for the BSDF pins.  or_ggx_sample_n: for each
 * (bu[i], bv[i]) the continuation direction wi, its throughput weight
 * f_r cos(theta_i) / pdf(wi) (0 where the path ends) and the sampled half
 * vector m; planted = 1 (tests) drops the reflection Jacobian.
 * or_ggx_eval_n: f_r(wo, wi) for n directions.  or_ggx_g1: Smith masking. */
void   or_ggx_sample_n(double alpha, const double F0[3], const double wo[3], int64_t n, const double* bu,
                       const double* bv, int32_t planted, double* wi, double* w, double* m);
void   or_ggx_eval_n(double alpha, const double F0[3], const double wo[3], int64_t n, const double* wi,
                     double* fr);
double or_ggx_g1(double cos_theta, double alpha);
void      or_scene_destroy(or_scene* s);
double    or_scene_scale(const or_scene* s);

/* Closest hit along o + t d, t in (tmin, tmax).  Returns 1 on hit.
 * margin (optional): distance of the decision from flipping, scene-relative. */
int32_t or_closest_hit(const or_scene* s, const double o[3], const double d[3],
                       double tmin, double tmax, int32_t brute,
                       double* t_out, int32_t* tri_out, double* margin);
/* Any hit in (tmin, tmax).  Returns 1 if occluded. */
int32_t or_any_hit(const or_scene* s, const double o[3], const double d[3],
                   double tmin, double tmax, int32_t brute, double* margin);

/* Path contribution f(u) of a primary-sample vector q (D = 2 + 5 max_depth
 * words).  counts (optional): counts[0] += rays cast; [1], [2] unused.
 * margin (optional): the smallest scene-relative distance of a geometric
 * decision from flipping (edges, ties, grazing cosines). */
int32_t or_path_eval(const or_scene* s, int32_t width, int32_t height, int32_t max_depth,
                     const uint32_t* q, double f[3], double* margin, uint64_t counts[3]);
/* The same path with a first-order error model of its binary32 evaluation:
 * dec = the smallest distance of a decision (edge, tie, cosine sign, light
 * CDF, frame switch) from flipping, in units of that quantity's binary32 error
 * bound; ferr[c] = a bound on |f_c(binary32) - f_c| from the unit roundoff
 * propagated through the path's geometry (positions, directions, cosines,
 * distances, the GGX density's slope). */
int32_t or_path_eval_err(const or_scene* s, int32_t width, int32_t height, int32_t max_depth,
                         const uint32_t* q, double f[3], double* dec, double ferr[3], uint64_t counts[3]);

or_ctx*  or_ctx_create(const or_scene* s, const or_params* p);
void     or_ctx_destroy(or_ctx* c);
void     or_set_hooks(or_ctx* c, or_mut_hook mh, or_upd_hook uh, void* user);
void     or_set_prop_hook(or_ctx* c, or_prop_hook ph);
/* The last Langevin move's terms (tests): its drift m_x [D] and standard
 * normal draws z [D] (as drawn, before a proposal hook), and out2 = {tau_x,
 * S} with S = sum_d |m_x,d| |delta_d - m_x,d| / tau_x + |m_y,d| |delta_d +
 * m_y,d| / tau_y, the sensitivity of ln a to relative errors of the drifts. */
void     or_last_mala(const or_ctx* c, double* m, double* z, double out2[2]);
int32_t  or_init(or_ctx* c);                       /* bootstrap + initial states */
int32_t  or_init_tables(or_ctx* c);                /* region tables only (Alg. 1, initialisation) */
void     or_refresh_sigma(or_ctx* c);              /* sigma_k from the current lambda_k */
/* Set chain `chain` to state q; f, pi and k are recomputed by the oracle. */
int32_t  or_set_state(or_ctx* c, uint32_t chain, const uint32_t* q);
/* One mutation of one chain at mutation index `mut` (region tables updated). */
int32_t  or_mutate_one(or_ctx* c, uint32_t chain, uint64_t mut);
int32_t  or_run_epochs(or_ctx* c, int64_t n_epochs);
/* One epoch of a sharded population in two halves.  or_epoch_mutate runs E
 * mutations of every chain of this context and writes what they added to the
 * region tables: counts [3 cap + 1] = i_k, A_k, h_k (cap each) and the number
 * of large steps; sums [cap] = the sum of pi over large-step proposals per
 * region.  or_epoch_update takes those arrays summed over every context of
 * the population, sets each table to its value at the start of the epoch
 * plus the sums, and runs the epoch boundary (Alg. 1, region update, weights,
 * quadtree).  cap = or_region_capacity(). */
int32_t  or_epoch_mutate(or_ctx* c, uint64_t* counts, double* sums);
int32_t  or_epoch_update(or_ctx* c, const uint64_t* counts, const double* sums);
int32_t  or_region_capacity(const or_ctx* c);
void     or_read_image(const or_ctx* c, double* out_rgb);   /* H*W*3 radiance */

int32_t   or_dims(const or_ctx* c);
int32_t   or_regions(const or_ctx* c);
int32_t   or_region_of(const or_ctx* c, const uint32_t* q);
uint64_t  or_mutations_done(const or_ctx* c);       /* per chain */
double    or_bhat(const or_ctx* c);
uint32_t* or_state_q(or_ctx* c);      /* [C][D] */
double*   or_state_f(or_ctx* c);      /* [C][3] */
double*   or_state_pi(or_ctx* c);     /* [C]    */
int32_t*  or_state_k(or_ctx* c);      /* [C]    */
int64_t*  or_boot_choice(or_ctx* c);  /* [C]    */
double*   or_lambda(or_ctx* c);       /* [m]    */
int64_t*  or_n_updates(or_ctx* c);    /* [m]    */
uint64_t* or_visits(or_ctx* c);       /* i_k [m] */
uint64_t* or_accsum(or_ctx* c);       /* A_k [m], fixed point 2^-32 */
uint64_t* or_hist(or_ctx* c);         /* h_k [m] */
uint64_t* or_hist_prev(or_ctx* c);    /* h_k at the last weight update or quadtree pass [m] */
double*   or_weight(or_ctx* c);       /* w_k [m] */
float*    or_sigma(or_ctx* c);        /* sigma_k [m] binary32 */
double*   or_image_acc(or_ctx* c);    /* [H][W][3] unnormalised */
void      or_stats(const or_ctx* c, uint64_t out[8]);
/* Langevin moves proposed and accepted. */
void      or_mala_stats(const or_ctx* c, uint64_t out[2]);
/* Gradient of log pi at chain's current state ([D] doubles; Langevin runs only). */
const double* or_state_grad(const or_ctx* c, uint32_t chain);
/* Quadtree partition: copies child [nodes][4] (-1 leaf), leaf region id
 * [nodes] (-1 internal) and depth [nodes]; returns the node count. */
int32_t   or_quadtree(const or_ctx* c, int32_t* child, int32_t* leaf, int32_t* depth, int32_t cap_nodes);
/* One refinement pass of the quadtree now (tests; the epoch loop runs it
 * every qt_refine mutations). */
int32_t   or_refine(or_ctx* c);
/* Acceptance probability of moving x -> y under the current region tables
 * (regions taken from the states; large = 1 for the independent large step). */
double    or_accept_prob(const or_ctx* c, const uint32_t* qx, const uint32_t* qy,
                         double pi_x, double pi_y, int32_t large);
/* out: mutations, accepted, large, small, early_reject, invalid, rays, boot */

#ifdef __cplusplus
}
#endif
#endif

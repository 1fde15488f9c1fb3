// Internal interface between the host side of librmlt (C ABI, scene/BVH
// upload, bookkeeping) and its CUDA kernels.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "rmlt.h"

namespace rmlt {

constexpr int kMaxDim = 2 + 5 * RMLT_MAX_DEPTH;   // 62 primary-sample dimensions
constexpr int kStackSize = 48;                      // traversal stack entries per ray (shared memory)
constexpr int kChainBlock = 128;                    // threads per block of the per-chain / per-path kernels
constexpr int kEpochBlock = 64;                     // threads per block of the chain epoch kernel (BVH scenes)
constexpr int kStackStride = 64;                    // traversal stacks: panels of 64 threads, one column each
static_assert(kChainBlock % kStackStride == 0 && kEpochBlock % kStackStride == 0, "stack panels");
constexpr int kLeafBatch = 8;                       // lanes of a warp at leaves before they test them together

// statistic slots in DevChains::stats
enum StatSlot {
    kStAccepted = 0, kStLarge, kStSmall, kStEarly, kStInvalid, kStRays, kStOverflow,
    kStNodes, kStTris,
    // scheduling counters (work-counter builds only): warp loop iterations,
    // lanes traversing summed over iterations, shade batches and their lanes,
    // finish/setup batches and their lanes
    kStIters, kStTravLanes, kStShadeBatches, kStShadeLanes, kStSetupBatches, kStSetupLanes,
    // warp cycle counters (work-counter builds only): traversal steps, shade
    // batches, finish/setup batches, warp lifetime (sum and max)
    kStCycTrav, kStCycShade, kStCycSetup, kStCycLife, kStCycLifeMax,
    // wavefront form: waves run, epochs stopped by the wave limit
    kStWaves, kStWaveLimit,
    // Langevin moves proposed and accepted
    kStMala, kStMalaAcc,
    // bootstrap paths dropped by a traversal-stack overflow
    kStBootOverflow,
    kStCount = 32
};

// Leaf references in the BVH: bit 31 set, bits 28..30 = count - 1, bits 0..27 = first triangle.
constexpr uint32_t kLeafBit = 0x80000000u;
// An unused child slot of a BVH4 node references a one-triangle leaf at
// position n_tris, just past the scene's triangles, where the upload puts a
// zero-area sentinel triangle.  The slot's box is inverted, so no slab test
// accepts it; were one to, the sentinel's test finds no hit, and no
// reference ever leaves the triangle array.
constexpr uint32_t empty_ref(uint32_t n_tris) { return kLeafBit | n_tris; }

// BVH node layouts (bvh_build.cpp describes them): BVH2, 4 float4 per node;
// BVH4 with binary32 child bounds, 8 float4; BVH4 with the child boxes
// quantised to 8 bits on a per-node grid, 4 float4.
enum NodeFormat { kNodeBvh2 = 0, kNodeBvh4 = 1, kNodeBvh4Q = 2 };
constexpr int node_float4s(int fmt) { return fmt == kNodeBvh4 ? 8 : 4; }
// a BVH4 whose binary32 nodes and triangles would take more device memory
// than this gets quantised nodes: past a third of the L2, node loads miss it
// often enough that half the bytes per node pays for the decode
constexpr double kQuantiseBytes = 48.0e6;

// Device view of a loaded scene.  Triangles: 3 float4 each (v0 | mat id bits,
// e1 | original index bits, e2 | 0); nodes: node_float4s(node_fmt) float4
// each; materials: 3 float4 each (albedo | type, emission | roughness,
// emissive flag | black flag).
struct DevScene {
    const float4* tris = nullptr;
    const float4* nodes = nullptr;
    const float4* mats = nullptr;
    const int32_t* light_tri = nullptr;
    const float* light_cdf = nullptr;
    int32_t n_tris = 0, n_nodes = 0, n_mats = 0, n_lights = 0, brute = 1;
    int32_t node_fmt = kNodeBvh4;     // node layout (NodeFormat)
    float light_area = 0.f;
    float cam_pos[3] = {0, 0, 0}, cam_fwd[3] = {0, 0, 1}, cam_right[3] = {1, 0, 0}, cam_up[3] = {0, 1, 0};
    float tan_x = 1.f, tan_y = 1.f;   // tan(vfov / 2) * aspect, tan(vfov / 2)
    float eps = 1e-4f;                // ray offset, 1e-4 of the scene diagonal
    int32_t toy = 0;
    float toy_p[10] = {0};
};

// Device view of the chains and region tables.
struct DevChains {
    int32_t C = 0, D = 0, W = 0, H = 0, region_px = 1, nx = 1, m = 1, max_depth = 0, E = 1, L = 10;
    int32_t weighted = 0;
    int32_t truncnorm = 0;        // small-step kernel: 0 Kelemen, 1 truncated normal
    int32_t dcells = 0;           // 4-D partition: cells per axis over (u5, u6); <= 1 screen only
    // sharded population: chain c of this context has the global id chain0 + c
    // (its Philox key), of C_all chains over every context (C_all = C unsharded)
    uint32_t chain0 = 0;
    int32_t C_all = 0;
    uint32_t* q = nullptr;        // word d of chain c at q[d qd + c qc]: [D][C] (qd = C, qc = 1)
    int64_t qd = 0, qc = 1;       //   or, inside the wavefront form's epoch, a [C][D] copy (qd = 1, qc = D)
    float* f = nullptr;           // [3][C]
    float* pi = nullptr;          // [C]
    int32_t* k = nullptr;         // [C]
    double* lam = nullptr;        // [m]
    long long* n = nullptr;       // [m]
    unsigned long long* vis = nullptr;    // i_k [m]
    unsigned long long* acc = nullptr;    // A_k [m]
    unsigned long long* hist = nullptr;   // h_k [m]
    unsigned long long* hprev = nullptr;  // h_k at the previous weight update [m]
    double* w = nullptr;          // [m]
    double* Rc = nullptr;         // [m]
    float* sig = nullptr;         // sigma_k [m]
    float* wf = nullptr;          // w_k as float [m]
    double* Bk = nullptr;         // sum of pi over uniform samples per region [m]
    // epoch-wise stepping (rmlt_epoch_mutate / rmlt_epoch_update): the region
    // tables at the start of the epoch, i [m] A [m] h [m] and the large-step
    // count [1], and Bk [m]; the whole population's large steps [1]
    unsigned long long* snap = nullptr;
    double* snapB = nullptr;
    unsigned long long* large_all = nullptr;
    // quadtree partition (Sec. 6.2); m is then the region capacity and the
    // current leaf count lives in qt_state[0] (nodes in qt_state[1])
    int32_t quadtree = 0;
    int32_t* qt_child = nullptr;  // [nodes][4], -1 for a leaf
    int32_t* qt_leaf = nullptr;   // [nodes] region id of a leaf, -1 for an internal node
    int32_t* qt_depth = nullptr;  // [nodes]
    int32_t* qt_state = nullptr;  // [2] leaves, nodes
    int32_t qt_cap = 0, qt_max_depth = 0;
    long long qt_split = 0;
    // large steps traced ahead of the epoch (nullptr: traced in the chain kernel)
    float* lf = nullptr;          // [3][E][C] their contributions
    uint32_t* llist = nullptr;    // [E C] work list of (j C + c)
    unsigned* lcount = nullptr;   // [1]
    double* img = nullptr;        // [H][W][3]
    unsigned long long* stats = nullptr;  // [kStCount]
    uint32_t seed_lo = 0, seed_hi = 0, T_large = 0;
    float S1 = 0.f, S2 = 0.f, log2_ratio = 0.f;
    double alpha_star = 0.5, gamma_max = 1.0, gamma_scale = 5.0, lambda_min = -30.0, lambda_max = 7.0;
    double w_floor = 1e-3;
    // lanes that wait before the warp shades / finishes and draws together
    int32_t batch_shade = 8, batch_setup = 8;
    int32_t adaptive_batch = 0;   // shrink the batches when few lanes are still working
    // Langevin (MALA) strategy: gradients of the current states, the strategy
    // threshold on the 24-bit strategy uniform (above T_large), step and
    // drift bound
    float* G = nullptr;           // [D][C] grad log pi at each chain's state
    uint32_t T_mala = 0;
    float mala_tau = 0.f, mala_drift_max = 0.f;
    // trace instrument
    rmlt_trace_record* trace = nullptr;
    unsigned long long trace_cap = 0, trace_base = 0;
    uint32_t trace_stride = 1;
    uint32_t* trace_words = nullptr;   // optional: the D proposal words of each record, [record][D]
};

// Wavefront form of the chain epoch (rmlt_wavefront.cu).  Per chain,
// kWfSlots 32-bit words hold the mutation in flight, the path state between
// waves and the ray results.  The words only the finish / setup kernel uses
// (the chain's lane state and its statistics, [0, kWRowEnd)) sit in a row
// of kWfRow words per chain: that kernel visits the chains of a compacted
// list, scattered over the population, and reads a line per chain instead
// of a sector per word.  The rest sit in columns ([word][C]), coalesced for
// the shade kernel, which visits every chain in order.  The proposal y lives
// in [C][D].
// A wave is three kernels: shade (consume the ray results of the chains with
// rays in flight, emit the next rays), finish / set up (the chains whose path
// ended: accept or reject, the next proposal, its camera ray), and trace (a
// persistent kernel that pulls rays from the queue).  A CUDA graph repeats
// the wave under a device-side while condition until no chain has a ray.
enum WfSlot {
    // row block: lane state and the statistics the finish / setup kernel counts
    kWKx = 0, kWPx, kWPy, kWPix, kWFx, kWPendN = kWFx + 3, kWPendI, kWPendA, kWJ = kWPendA + 2, kWFlags, kWKy,
    kWXi, kWR, kWFy, kWSt = kWFy + 3, kWRowEnd = kWSt + 5,
    // column block: path state, ray counters and ray results
    kWT = kWRowEnd, kWL = kWT + 3, kWP = kWL + 3, kWB = kWP + 3, kWO, kWD = kWO + 3, kWPfl = kWD + 3,
    kWRays, kWDropped, kWPhase, kWHitT, kWHitTri, kWShd, kWfSlots
};
constexpr int kWfRow = 32;   // words per row (one 128-byte line)
static_assert(kWRowEnd <= kWfRow, "the row block fits a row");

struct WfCounters {
    unsigned wave, ticket, fq_count, err;
    unsigned cnt[2], fetch[2];      // rays appended / pulled, per queue
    unsigned trace_n, trace_buf;    // the queue the next trace pass reads
    unsigned long long mut0, trace_base;
};

struct DevWave {
    uint32_t* s = nullptr;        // [C][kWfRow] row block, then [kWfSlots - kWRowEnd][C] columns
    uint32_t* y = nullptr;        // [C][D] proposals, one chain's words contiguous
    uint32_t* qa = nullptr;       // [C][D] the states during an epoch (transposed in and out)
    float4* rq[2] = {nullptr, nullptr};   // two queues of 2C rays, 2 float4 each
    uint32_t* fq = nullptr;       // [C] chains to finish / set up
    WfCounters* ctr = nullptr;
    unsigned long long cond = 0;  // cudaGraphConditionalHandle of the wave loop
    unsigned wave_cap = 0;        // E (max_depth + 1) + 2: more waves than any epoch needs
    int refill = 8;               // idle lanes of a trace warp that pull new rays together
    int leaf_batch = kLeafBatch;  // lanes of a trace warp at leaves before they test them together
    int short_stack = 0;          // 1: the trace kernel keeps kShortStack stack entries per ray in shared
                                  //    memory and the rest in `gstack`
    uint32_t* gstack = nullptr;   // [kStackSize - kShortStack][kWfTraceThreadsPerSm x SMs]
};
constexpr int kShortStack = 16;
constexpr int kWfTraceThreadsPerSm = 16 * kChainBlock;   // bound on the persistent trace kernel's threads per SM

// device bytes of the wavefront state for C chains of D dimensions
size_t wf_bytes(int C, int D);
// carve the state out of one allocation of wf_bytes(C, D)
void wf_carve(void* base, int C, int D, DevWave& w);

struct WfGraph;   // the instantiated wave loop, rebuilt when its launch parameters change
void wf_graph_destroy(WfGraph* g);
// One epoch of E mutations per chain in the wavefront form.
// wave_limit: waves after which the epoch stops (0: E (max_depth + 1) + 2)
cudaError_t wf_epoch(WfGraph** g, const DevScene& s, const DevChains& c, DevWave& w, uint64_t mut0,
                     unsigned long long trace_base, bool trace, bool count_work, int trace_ctas_per_sm,
                     int setup_ctas_per_sm, bool host_loop, unsigned wave_limit, cudaStream_t st);

// One member of a batched epoch (rmlt_batch_step): its scene, its chains,
// the mutation index of its next epoch and its first block in the launch.
struct BatchMember {
    DevScene S;
    DevChains Ch;
    unsigned long long mut0 = 0;
    int32_t block0 = 0, pad_ = 0;
    // trace instrument (Ch.trace set): the mutation index at which tracing
    // started, and lambda after each epoch's update [epoch][m] (may be null)
    unsigned long long trace_mut0 = 0;
    double* tr_lam = nullptr;
    unsigned long long tr_lam_cap = 0;
};
// blocks [block_base, block_base + n_blocks) of the batch's block table
cudaError_t launch_chain_epoch_batch(const BatchMember* members, const int* block_member, int block_base,
                                     int n_blocks, bool count_work, int ctas_per_sm, bool trace, cudaStream_t st);
// the chain kernel of one member (its scene and chains as launch parameters),
// reading the epoch's first mutation index from member_dev->mut0
cudaError_t launch_chain_epoch_member(const BatchMember* member_dev, const BatchMember& member, bool count_work,
                                      cudaStream_t st);
// region update of every member and mut0 += E (one block per member)
cudaError_t launch_region_update_batch(BatchMember* members, int n, cudaStream_t st);

// Scratch of the bootstrap (n = K C samples, K = n_bootstrap / C per chain).
// The bootstrap draws n = K C_all samples (every context of a sharded
// population draws all of them) and selects starting states for its own
// chains.
struct BootScratch {
    float* pi = nullptr;          // [n]
    float* f = nullptr;           // [3][n]
    double* partial = nullptr;    // [C_all] per-chain slice sums
    double* prefix = nullptr;     // [C_all + 1] exclusive prefix of the slice sums, then their total
    double* total = nullptr;      // [1] sum of pi over all samples (kept)
    unsigned long long* overflow = nullptr;   // [1] paths dropped by a traversal-stack overflow (added to)
};

cudaError_t launch_chain_epoch(const DevScene& s, const DevChains& c, uint64_t mut0, bool trace,
                               bool count_work, cudaStream_t st);
// grad log pi of every chain's current state into c.G (Langevin strategy)
cudaError_t launch_state_gradients(const DevScene& s, const DevChains& c, cudaStream_t st);
// f, log pi and grad log pi at n points q [D][n] (D = c.D); any output may be NULL
cudaError_t launch_path_grad(const DevScene& s, const DevChains& c, const uint32_t* q, long long n, float* f,
                             float* logpi, float* grad, cudaStream_t st);
cudaError_t launch_region_update(const DevChains& c, bool init_only, cudaStream_t st);
// the paths of n points q [D][n]: every ray [n][2 max_depth][8] floats and the
// traversal's work for it [n][2 max_depth][4] u32 (rmlt_record_paths)
cudaError_t launch_record_paths(const DevScene& s, const DevChains& c, const uint32_t* q, long long n, float* rays,
                                uint32_t* out, cudaStream_t st);
cudaError_t launch_large_steps(const DevScene& s, const DevChains& c, uint64_t mut0, cudaStream_t st);
cudaError_t launch_bootstrap(const DevScene& s, const DevChains& c, int64_t n_boot,
                             const BootScratch& b, cudaStream_t st);
cudaError_t launch_read_image(const DevChains& c, const double* bhat_total, int64_t n_boot,
                              double n_total, int normalized, double* out, cudaStream_t st);
cudaError_t launch_fill_regions(const DevChains& c, double lambda_init, cudaStream_t st);
cudaError_t launch_quadtree_refine(const DevChains& c, cudaStream_t st);
// epoch-wise stepping: copy the region tables to c.snap / c.snapB; write what
// the epoch added to them (counts [3m + 1], sums [m]); set them to the
// snapshot plus the summed additions
cudaError_t launch_epoch_snapshot(const DevChains& c, cudaStream_t st);
cudaError_t launch_epoch_pack(const DevChains& c, unsigned long long* counts, double* sums, cudaStream_t st);
cudaError_t launch_epoch_unpack(const DevChains& c, const unsigned long long* counts, const double* sums,
                                cudaStream_t st);
// the chains' regions recomputed from their states (after a restore)
cudaError_t launch_chain_regions(const DevChains& c, cudaStream_t st);

// Pointers into the library's fixed scratch array (rmlt_bootstrap_noalloc).
struct NoAllocScratch {
    BootScratch boot;
    float* chain_pi = nullptr;
    int32_t* chain_k = nullptr;
    double* Bk = nullptr;
    unsigned long long* overflow = nullptr;
};
// Looks the array up on the current device (first call per device) and
// fills `out`; allocates nothing.
cudaError_t noalloc_scratch(int device, NoAllocScratch& out);

// host-side BVH build (bvh_build.cpp)
struct HostBVH {
    std::vector<float4> nodes;    // node_float4s(fmt) per node
    std::vector<uint32_t> order;  // triangle order after the build
    int width = 4;
    int fmt = kNodeBvh4;
    int max_depth = 0;
};
// width 2: BVH2; width 4: BVH4 with binary32 bounds, or quantised bounds when
// `quantise` is 1, or when it is -1 and the binary32 nodes and the triangles
// would exceed kQuantiseBytes
void build_bvh(const std::vector<float>& tri_v, int n_tris, float pad, int width, HostBVH& out,
               int quantise = -1);

// Reference traversal on the host (bvh_walk.cpp): the uploaded node and
// triangle arrays walked in binary64, nearest child first, counting the
// internal nodes visited and the triangles tested for one ray.
struct WalkResult {
    int32_t tri;          // original index of the closest (any-hit: first found) triangle, -1 if none
    double t;
    uint32_t nodes, tris;
};
WalkResult walk_ray(const std::vector<float4>& nodes, int fmt, const std::vector<float4>& tris, bool brute,
                    const float ray[8]);

}  // namespace rmlt

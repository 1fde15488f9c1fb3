// CUDA kernels of librmlt (sm_103a): the regional adaptive PSS-MLT chain step.
//
// One thread owns one chain for an epoch of E mutations (Alg. 1, mutation loop).
// Each loop iteration traces exactly one ray (camera/extension closest hit,
// or a next-event shadow any-hit), so the threads of a warp meet at the same
// traversal code whatever mutation or bounce each one is at.  Chain state is
// structure-of-arrays (coalesced per dimension), BVH nodes and triangles are
// read as 16-byte float4, splats and region counts are flushed only when a
// chain's state changes (a rejected mutation re-splats the same state, so a
// per-thread visit count replaces one atomic per mutation).
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "rmlt_internal.h"

#include "rmlt_device.cuh"

namespace rmlt {
namespace {

// One thread per chain; the unit of work is one traversal step.  Every step
// advances each lane with a live ray by one BVH node or leaf.  A lane whose
// extension ray is resolved waits until at least `batch_shade` lanes (or
// every lane with work) are waiting, then the waiting lanes shade together
// (emission, next-event sample and BSDF sample at once: the shadow ray is
// traversed next and resolved inside the traversal loop, then the extension
// ray).  Lanes whose path ended finish their mutation and draw the next
// proposal in batches of `batch_setup` the same way.  The batches keep the
// expensive, divergent parts convergent while the traversal keeps every lane
// busy.
// With the Langevin strategy, a lane whose next mutation is a Langevin move
// waits in kMala: those moves trace their paths one lane at a time, so they
// run in their own batches of at least kMalaBatch lanes instead of holding
// up every setup batch.
enum LanePhase { kIdle = 0, kTraverse = 1, kShade = 2, kFinish = 3, kSetup = 4, kMala = 5 };
constexpr int kMalaBatch = 8;

// whether mutation L.j of chain c is a Langevin move (the test mutation_setup
// makes on the mutation's first Philox call)
__device__ __forceinline__ bool next_is_mala(const DevChains& Ch, int c, uint64_t mut0, const ChainLane& L)
{
    const uint64_t mut = mut0 + (uint64_t)L.j;
    const uint4 r0 = philox((uint32_t)mut, (uint32_t)(mut >> 32), Ch.chain0 + (uint32_t)c, 0u, Ch.seed_lo, Ch.seed_hi);
    const uint32_t h = r0.x >> 8;
    return h >= Ch.T_large && h < Ch.T_large + Ch.T_mala;
}

// The proposal words: in shared memory (YSM, blocks of NT threads), else in
// local memory.
template <bool YSM>
struct ProposalWords;
template <>
struct ProposalWords<true> {
    static __device__ __forceinline__ YPanel get(uint32_t* s_y, uint32_t*) { return thread_words(s_y); }
};
template <>
struct ProposalWords<false> {
    static __device__ __forceinline__ uint32_t* get(uint32_t*, uint32_t* y_local) { return y_local; }
};

// The epoch of chain c (one thread); s_tris holds the staged triangles of a
// brute-force scene, s_stack the block's traversal stacks.
template <bool BRUTE, bool TRACE, bool COUNT, bool MALA = false, bool D4 = false, bool YSM = false,
          int NT = kChainBlock, int FMT = -1>
__device__ __forceinline__ void chain_epoch_body(const DevScene& S, const DevChains& Ch, uint64_t mut0, int c,
                                                 const float4* s_tris, uint32_t* s_stack)
{
    __shared__ uint32_t s_y[YSM ? kMaxDim * NT : 1];
    const unsigned FULL = 0xFFFFFFFFu;
    const bool valid = c < Ch.C;
    unsigned st[7] = {0, 0, 0, 0, 0, 0, 0};   // accepted, large, small, early, invalid, rays, overflow
    unsigned n_nodes = 0, n_tris = 0;
    ChainLane L;
    L.kx = L.px = L.py = 0;
    L.pix = 0.f;
    L.fx = {0.f, 0.f, 0.f};
    if (valid) {
        const int C = Ch.C;
        L.kx = Ch.k[c];
        L.pix = Ch.pi[c];
        L.fx = {Ch.f[c], Ch.f[C + c], Ch.f[2 * C + c]};
        L.px = pixel_x(Ch.q[c], Ch.W);
        L.py = pixel_x(Ch.q[C + c], Ch.H);
    }
    L.pend_n = 0;
    L.pend_i = L.pend_A = 0;
    L.j = 0;
    L.large = L.ky = L.early = 0;
    L.xi = 0.f;
    L.R = 1.0f;
    L.fy = {0.f, 0.f, 0.f};
    L.mala = 0;
    L.amala = 0.f;
    L.n_mala = L.n_mala_acc = 0;
    const bool traced = TRACE && valid && (uint32_t)c % Ch.trace_stride == 0u;
    uint32_t y_local[YSM ? 1 : kMaxDim];
    const auto y = ProposalWords<YSM>::get(s_y, y_local);
    // traversal stack in shared memory, one column per thread (conflict-free)
    uint32_t* stack = thread_stack(s_stack);
    Path p;
    Trav T;
    T.ref = kNoRef;
    int phase = (valid && Ch.E > 0) ? kSetup : kIdle;
    const int bs = Ch.batch_shade, bf = Ch.batch_setup;
    unsigned long long sched[6] = {0, 0, 0, 0, 0, 0};   // warp-uniform, counted once per warp
    unsigned long long cyc[3] = {0, 0, 0};   // cycles in traversal steps, shade batches, finish/setup batches
    long long t_start = 0, t_mark = 0;
    if (COUNT) t_start = t_mark = clock64();
    while (true) {
        // traversal steps until a batch is due: enough lanes waiting to shade
        // or to finish, or no lane left traversing (the votes of the batch
        // conditions are paid once per step, the batch code only when due)
        unsigned m_tr, m_sh;
        int bs_eff = bs, bf_eff = bf;
        while (true) {
            __syncwarp();
            if (step_turn<BRUTE>(phase == kTraverse, T)) {
                if (trav_step<BRUTE, decltype(stack), FMT>(T, stack, S, s_tris, n_nodes, n_tris)) {
                    if (T.any) {
                        // the shadow ray of the last interaction: its contribution
                        // now, then straight on with the extension ray that the
                        // interaction already drew (no shading batch needed)
                        ++st[5];
                        if (T.overflow) {
                            ++st[6];
                            p.L = {0.f, 0.f, 0.f};
                            p.done = 1;
                        } else if (T.tri < 0) {
                            p.L = p.L + p.P;
                        }
                        if (p.done) {
                            L.fy = p.L;
                            phase = kFinish;
                        } else {
                            trav_begin(T, p.o, p.d, p.tmax, 0);
                        }
                    } else {
                        phase = kShade;
                    }
                }
            }
            m_tr = __ballot_sync(FULL, phase == kTraverse);
            m_sh = __ballot_sync(FULL, phase == kShade);
            const unsigned m_fs0 = __ballot_sync(FULL, phase == kFinish || phase == kSetup);
            // fewer lanes at work (the end of the epoch): optionally smaller batches
            if (Ch.adaptive_batch) {
                const int busy = __popc(__ballot_sync(FULL, phase != kIdle));
                bs_eff = min(bs, (busy + 3) >> 2);
                bf_eff = min(bf, (busy + 3) >> 2);
            }
            if (COUNT) {
                sched[0] += 1;
                sched[1] += __popc(m_tr);
            }
            if (!m_tr || __popc(m_sh) >= bs_eff || __popc(m_fs0) >= bf_eff) break;
            if (MALA && __popc(__ballot_sync(FULL, phase == kMala)) >= kMalaBatch) break;
        }
        if (COUNT) {
            __syncwarp();
            const long long t = clock64();
            cyc[0] += t - t_mark;
            t_mark = t;
        }
        if (m_sh && (__popc(m_sh) >= bs_eff || !m_tr)) {
            if (COUNT) {
                sched[2] += 1;
                sched[3] += __popc(m_sh);
            }
            if (phase == kShade) {
                ++st[5];
                bool shadow = false;
                if (T.overflow) {
                    ++st[6];
                    p.done = 1;
                    p.L = {0.f, 0.f, 0.f};
                } else if (T.tri < 0 || !shade_hit<BRUTE>(p, S, Hit{T.t, T.tri, T.ta, T.tb, T.tc})) {
                    p.done = 1;
                } else {
                    // next-event sample and BSDF continuation together: the
                    // shadow ray goes first, the extension ray waits in p
                    if (nee_sample<BRUTE>(p, S, s_tris, y)) {
                        trav_begin(T, p.o, p.d, p.tmax, 1);
                        shadow = true;
                    }
                    path_continue(p, S, y, Ch.max_depth);
                }
                if (shadow) {
                    phase = kTraverse;
                } else if (p.done) {
                    L.fy = p.L;
                    phase = kFinish;
                } else {
                    trav_begin(T, p.o, p.d, p.tmax, 0);
                    phase = kTraverse;
                }
            }
            if (COUNT) {
                __syncwarp();
                const long long t = clock64();
                cyc[1] += t - t_mark;
                t_mark = t;
            }
        }
        const unsigned m_tr2 = __ballot_sync(FULL, phase == kTraverse);
        const unsigned m_fs = __ballot_sync(FULL, phase == kFinish || phase == kSetup);
        const unsigned m_sh2 = __ballot_sync(FULL, phase == kShade);
        if (m_fs && (__popc(m_fs) >= bf_eff || (!m_tr2 && !m_sh2))) {
            if (COUNT) {
                sched[4] += 1;
                sched[5] += __popc(m_fs);
            }
            // a proposal rejected early (or the toy integrand) finishes at once
            for (int r = 0; r < 8 && (phase == kFinish || phase == kSetup); ++r) {
                if (phase == kFinish) {
                    mutation_finish<TRACE, MALA>(Ch, c, traced, L, y, st);
                    ++L.j;
                    phase = L.j < Ch.E ? kSetup : kIdle;
                }
                if (phase == kSetup) {
                    if (MALA && next_is_mala(Ch, c, mut0, L)) {
                        phase = kMala;   // made in the next Langevin batch
                    } else {
                        if (MALA) L.mala = 0;
                        if (mutation_setup<false, BRUTE, D4>(S, Ch, c, mut0, L, y, p, stack, s_tris, &st[5])) {
                            trav_begin(T, p.o, p.d, p.tmax, p.any);
                            phase = kTraverse;
                        } else {
                            phase = kFinish;
                        }
                    }
                }
            }
            if (COUNT) {
                __syncwarp();
                const long long t = clock64();
                cyc[2] += t - t_mark;
                t_mark = t;
            }
        }
        if (MALA) {
            // Langevin batch: each waiting lane makes its move (proposal,
            // path with gradient, acceptance probability); the mutation is
            // finished in the next setup batch
            const unsigned m_ml = __ballot_sync(FULL, phase == kMala);
            const bool others = __any_sync(FULL, phase != kMala && phase != kIdle);
            if (m_ml && (__popc(m_ml) >= kMalaBatch || !others)) {
                if (phase == kMala) {
                    // the fields mutation_setup sets before it hands over
                    const uint64_t mut = mut0 + (uint64_t)L.j;
                    const uint32_t mlo = (uint32_t)mut, mhi = (uint32_t)(mut >> 32);
                    const uint4 r0 = philox(mlo, mhi, Ch.chain0 + (uint32_t)c, 0u, Ch.seed_lo, Ch.seed_hi);
                    L.large = 0;
                    L.xi = u24(r0.y);
                    L.R = 1.0f;
                    mala_setup<BRUTE>(S, Ch, c, mlo, mhi, L, y, stack, s_tris, st[5]);
                    phase = kFinish;
                }
            }
        }
        if (!__any_sync(FULL, phase != kIdle)) break;
    }
    if (valid) {
        flush_state(Ch, L);
        const int C = Ch.C;
        Ch.k[c] = L.kx;
        Ch.pi[c] = L.pix;
        Ch.f[c] = L.fx.x;
        Ch.f[C + c] = L.fx.y;
        Ch.f[2 * C + c] = L.fx.z;
    }
    // warp-aggregated statistics
    unsigned long long v[9] = {st[0], st[1], st[2], st[3], st[4], st[5], st[6], n_nodes, n_tris};
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 0; s < 9; ++s) {
        if (s >= 7 && !COUNT) break;
        const unsigned long long t = warp_sum(v[s]);
        if (lane == 0 && t) atomicAdd(&Ch.stats[s], t);
    }
    if (MALA) {
        const unsigned long long a = warp_sum(L.n_mala), b = warp_sum(L.n_mala_acc);
        if (lane == 0 && a) atomicAdd(&Ch.stats[kStMala], a);
        if (lane == 0 && b) atomicAdd(&Ch.stats[kStMalaAcc], b);
    }
    if (COUNT && lane == 0) {
        for (int s = 0; s < 6; ++s) atomicAdd(&Ch.stats[kStIters + s], sched[s]);
        for (int s = 0; s < 3; ++s) atomicAdd(&Ch.stats[kStCycTrav + s], cyc[s]);
        const unsigned long long life = (unsigned long long)(clock64() - t_start);
        atomicAdd(&Ch.stats[kStCycLife], life);
        atomicMax(&Ch.stats[kStCycLifeMax], life);
    }
}

// Threads per block of the chain epoch kernel.  BVH scenes: 64, so that the
// 2^16 chains of a typical population spread over the SMs in steps of two
// warps (at most 14 warps on an SM of a 152-SM GPU instead of 16 with
// 128-thread blocks), with 8 blocks per SM keeping the register budget at
// 128 per thread.  Brute-force scenes stage their triangles per block, so
// they keep 128-thread blocks.
template <bool BRUTE>
__host__ __device__ constexpr int epoch_block() { return BRUTE ? kChainBlock : kEpochBlock; }

// mut0_dev, when set, holds the epoch's first mutation index on the device
// (a graph replayed over several epochs advances it there)
// FMT: the node layout the kernel is compiled for (-1: the scene's, read at
// each node)
template <bool BRUTE, bool TRACE, bool COUNT, bool MALA = false, bool D4 = false, int FMT = -1>
__global__ void __launch_bounds__(epoch_block<BRUTE>(), BRUTE ? 4 : 8)
    chain_epoch_kernel(const DevScene S, const DevChains Ch, uint64_t mut0, const unsigned long long* mut0_dev)
{
    extern __shared__ float4 s_tris[];
    __shared__ uint32_t s_stack[kStackSize * epoch_block<BRUTE>()];
    if (BRUTE) stage_triangles(S, s_tris);
    if (mut0_dev) mut0 = *mut0_dev;
    // proposal words in shared memory on BVH scenes; a brute-force scene's
    // staged triangles may fill shared memory, so it keeps them local
    chain_epoch_body<BRUTE, TRACE, COUNT, MALA, D4, !BRUTE, epoch_block<BRUTE>(), FMT>(
        S, Ch, mut0, blockIdx.x * blockDim.x + threadIdx.x, s_tris, s_stack);
}

// grad log pi of the chains' current states (Langevin strategy: at
// initialisation and after a restore)
template <bool BRUTE>
__global__ void __launch_bounds__(kChainBlock) state_grad_kernel(const DevScene S, const DevChains Ch)
{
    extern __shared__ float4 s_tris[];
    __shared__ uint32_t s_stack[kStackSize * kChainBlock];
    if (BRUTE) stage_triangles(S, s_tris);
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= Ch.C) return;
    const int C = Ch.C, D = Ch.D;
    uint32_t y[kMaxDim];
    for (int d = 0; d < D; ++d) y[d] = Ch.q[(size_t)d * C + c];
    float g[kMaxDim];
    if (S.toy) {
        toy_grad(S, y[0], y[1], g);
    } else {
        GradRec rec[RMLT_MAX_DEPTH];
        V3 f;
        unsigned rays = 0;
        const int nb = path_forward_rec<BRUTE>(S, s_tris, thread_stack(s_stack), y, Ch.max_depth, rec, f, rays);
        if (nb < 0) {
            for (int d = 0; d < D; ++d) g[d] = 0.0f;
        } else {
            path_adjoint(S, y, rec, nb, f, g, D);
        }
    }
    for (int d = 0; d < D; ++d) Ch.G[(size_t)d * C + c] = g[d];
}

// f, log pi and grad log pi at n given points q [D][n]
template <bool BRUTE>
__global__ void __launch_bounds__(kChainBlock) path_grad_kernel(const DevScene S, const DevChains Ch,
                                                                const uint32_t* q, long long n, float* fo,
                                                                float* logpi, float* grad)
{
    extern __shared__ float4 s_tris[];
    __shared__ uint32_t s_stack[kStackSize * kChainBlock];
    if (BRUTE) stage_triangles(S, s_tris);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int D = Ch.D;
    uint32_t y[kMaxDim];
    for (int d = 0; d < D; ++d) y[d] = q[(size_t)d * n + i];
    float g[kMaxDim];
    V3 f;
    if (S.toy) {
        const float v = toy_grad(S, y[0], y[1], g);
        f = {v, v, v};
    } else {
        GradRec rec[RMLT_MAX_DEPTH];
        unsigned rays = 0;
        const int nb = path_forward_rec<BRUTE>(S, s_tris, thread_stack(s_stack), y, Ch.max_depth, rec, f, rays);
        if (nb < 0) {
            f = {0.f, 0.f, 0.f};
            for (int d = 0; d < D; ++d) g[d] = 0.0f;
        } else {
            path_adjoint(S, y, rec, nb, f, g, D);
        }
    }
    if (fo) {
        fo[i] = f.x;
        fo[n + i] = f.y;
        fo[2 * n + i] = f.z;
    }
    if (logpi) logpi[i] = logf(lum(f.x, f.y, f.z));
    if (grad)
        for (int d = 0; d < D; ++d) grad[(size_t)d * n + i] = g[d];
}

// ---------------------------------------------------------------------------
// measurement instrument: the paths of n given points, each ray recorded
// with the chain kernel's traversal work for it (nodes visited, triangles
// tested), for an independent host traversal to re-count
// ---------------------------------------------------------------------------
template <bool BRUTE>
__global__ void __launch_bounds__(kChainBlock) record_paths_kernel(const DevScene S, const DevChains Ch,
                                                                   const uint32_t* q, long long n, float* rays,
                                                                   uint32_t* out)
{
    extern __shared__ float4 s_tris[];
    __shared__ uint32_t s_stack[kStackSize * kChainBlock];
    if (BRUTE) stage_triangles(S, s_tris);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int D = Ch.D, R = 2 * Ch.max_depth;
    uint32_t y[kMaxDim];
    for (int d = 0; d < D; ++d) y[d] = q[(size_t)d * n + i];
    Path p;
    Trav T;
    uint32_t* stack = thread_stack(s_stack);
    path_begin(p, S, y);
    int r = 0;
    while (!p.done && r < R) {
        trav_begin(T, p.o, p.d, p.tmax, p.any);
        unsigned nn = 0, nt = 0;
        while (!trav_step<BRUTE>(T, stack, S, s_tris, nn, nt)) {
        }
        float* rr = rays + ((size_t)i * R + r) * 8;
        rr[0] = p.o.x; rr[1] = p.o.y; rr[2] = p.o.z; rr[3] = p.tmax;
        rr[4] = p.d.x; rr[5] = p.d.y; rr[6] = p.d.z; rr[7] = (float)p.any;
        uint32_t* oo = out + ((size_t)i * R + r) * 4;
        oo[0] = T.tri >= 0 ? __float_as_uint(T.tb.w) : 0xFFFFFFFFu;   // the hit's original triangle index
        oo[1] = __float_as_uint(T.t);
        oo[2] = nn;
        oo[3] = nt;
        ++r;
        if (T.overflow) break;
        path_on_hit<BRUTE>(p, S, s_tris, y, Ch.max_depth, Hit{T.t, T.tri, T.ta, T.tb, T.tc});
    }
    for (; r < R; ++r) rays[((size_t)i * R + r) * 8 + 3] = -1.0f;   // no ray in this slot
}

// ---------------------------------------------------------------------------
// batched epoch: the chains of several contexts (scenes, resolutions, chain
// counts of any size) in one launch.  Block b runs chains of member
// block_member[b]; the member's scene and chain tables are copied to shared
// memory once per block.
// ---------------------------------------------------------------------------
template <bool COUNT, int MIN_BLOCKS, bool TRACE = false>
__global__ void __launch_bounds__(kChainBlock, MIN_BLOCKS) chain_epoch_batch_kernel(const BatchMember* members,
                                                                                 const int* block_member,
                                                                                 int block_base)
{
    __shared__ uint32_t s_stack[kStackSize * kChainBlock];
    __shared__ BatchMember m;
    const int bx = block_base + (int)blockIdx.x;
    const int e = block_member[bx];
    {
        const uint32_t* src = (const uint32_t*)(members + e);
        uint32_t* dst = (uint32_t*)&m;
        for (int i = threadIdx.x; i < (int)(sizeof(BatchMember) / 4); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    if (TRACE && threadIdx.x == 0 && m.Ch.trace) {
        // this epoch's records follow the traced epochs before it
        const unsigned long long n_traced = ((unsigned long long)m.Ch.C + m.Ch.trace_stride - 1) / m.Ch.trace_stride;
        m.Ch.trace_base = (m.mut0 - m.trace_mut0) * n_traced;
    }
    if (TRACE) __syncthreads();
    const int c = (bx - m.block0) * kChainBlock + threadIdx.x;
    chain_epoch_body<false, TRACE, COUNT>(m.S, m.Ch, m.mut0, c, nullptr, s_stack);
}

// ---------------------------------------------------------------------------
// large steps traced ahead of the epoch.  A large step proposes an
// independent uniform point (its draws do not depend on the chain's state),
// so its path can be evaluated before the epoch by a kernel with one thread
// per proposal and full occupancy; the chain kernel then reads f.  The values
// are bit-identical to tracing them inside the chain kernel.
// ---------------------------------------------------------------------------
__global__ void large_collect_kernel(const DevChains Ch, uint64_t mut0)
{
    const long long n = (long long)Ch.E * Ch.C;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool large = false;
    int c = 0, j = 0;
    if (i < n) {
        j = (int)(i / Ch.C);
        c = (int)(i % Ch.C);
        const uint64_t mut = mut0 + (uint64_t)j;
        const uint4 r0 = philox((uint32_t)mut, (uint32_t)(mut >> 32), Ch.chain0 + (uint32_t)c, 0u, Ch.seed_lo, Ch.seed_hi);
        large = (r0.x >> 8) < Ch.T_large;
    }
    // warp-aggregated append to the work list
    const unsigned m = __ballot_sync(0xFFFFFFFFu, large);
    const int lane = threadIdx.x & 31;
    unsigned base = 0;
    if (lane == 0 && m) base = atomicAdd(Ch.lcount, (unsigned)__popc(m));
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (large) Ch.llist[base + __popc(m & ((1u << lane) - 1u))] = (uint32_t)i;
}

template <bool BRUTE>
__global__ void __launch_bounds__(kChainBlock) large_trace_kernel(const DevScene S, const DevChains Ch, uint64_t mut0)
{
    extern __shared__ float4 s_tris[];
    __shared__ uint32_t s_stack[kStackSize * kChainBlock];
    if (BRUTE) stage_triangles(S, s_tris);
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *Ch.lcount) return;
    const uint32_t item = Ch.llist[i];
    const int j = (int)(item / (uint32_t)Ch.C), c = (int)(item % (uint32_t)Ch.C);
    const uint64_t mut = mut0 + (uint64_t)j;
    const uint32_t mlo = (uint32_t)mut, mhi = (uint32_t)(mut >> 32);
    const int D = Ch.D;
    uint32_t y[kMaxDim];
    for (int jj = 0; 4 * jj < D; ++jj) {
        const uint4 r = philox(mlo, mhi, Ch.chain0 + (uint32_t)c, 1u + (uint32_t)jj, Ch.seed_lo, Ch.seed_hi);
        y[4 * jj] = r.x;
        if (4 * jj + 1 < D) y[4 * jj + 1] = r.y;
        if (4 * jj + 2 < D) y[4 * jj + 2] = r.z;
        if (4 * jj + 3 < D) y[4 * jj + 3] = r.w;
    }
    Path p;
    Trav T;
    uint32_t* stack = thread_stack(s_stack);
    unsigned nn = 0, nt = 0, rays = 0, ovf = 0;
    path_begin(p, S, y);
    while (!p.done) {
        trav_begin(T, p.o, p.d, p.tmax, p.any);
        while (!trav_step<BRUTE>(T, stack, S, s_tris, nn, nt)) {
        }
        ++rays;
        if (T.overflow) {
            ++ovf;
            p.L = {0.f, 0.f, 0.f};
            break;
        }
        path_on_hit<BRUTE>(p, S, s_tris, y, Ch.max_depth, Hit{T.t, T.tri, T.ta, T.tb, T.tc});
    }
    const size_t o = (size_t)j * Ch.C + c, plane = (size_t)Ch.E * Ch.C;
    Ch.lf[o] = p.L.x;
    Ch.lf[plane + o] = p.L.y;
    Ch.lf[2 * plane + o] = p.L.z;
    float piy = lum(p.L.x, p.L.y, p.L.z);
    if (!isfinite(piy)) piy = 0.f;   // the chain kernel counts and zeroes invalid contributions
    const int ky = region_y(Ch, y);
    atomicAdd(&Ch.Bk[ky], (double)piy);
    // reduce over the lanes that arrive together (one atomic per group)
    const unsigned m = __activemask();
    const unsigned rs = __reduce_add_sync(m, rays), os = __reduce_add_sync(m, ovf);
    if ((int)(threadIdx.x & 31) == __ffs(m) - 1) {
        if (rs) atomicAdd(&Ch.stats[kStRays], (unsigned long long)rs);
        if (os) atomicAdd(&Ch.stats[kStOverflow], (unsigned long long)os);
    }
}

// ---------------------------------------------------------------------------
// region update at the epoch boundary (Alg. 1, region update; eqs.
// est_exp_acc, update_lambda, step_size_n), binary64 with explicit rounding
// ---------------------------------------------------------------------------
__device__ __forceinline__ void region_update_body(const DevChains& Ch, int init_only)
{
    const int m_now = Ch.quadtree ? Ch.qt_state[0] : Ch.m;
    for (int k = threadIdx.x; k < m_now; k += blockDim.x) {
        double lam = Ch.lam[k];
        if (!init_only && Ch.vis[k] >= (unsigned long long)Ch.L) {
            const double ah = __ddiv_rn((double)Ch.acc[k], __dmul_rn(4294967296.0, (double)Ch.vis[k]));
            const int sg = ah > Ch.alpha_star ? 1 : (ah < Ch.alpha_star ? -1 : 0);
            const double gs = __ddiv_rn(Ch.gamma_scale, __dsqrt_rn((double)Ch.n[k]));
            const double g = Ch.gamma_max < gs ? Ch.gamma_max : gs;
            lam = __dadd_rn(lam, __dmul_rn(g, (double)sg));
            if (lam < Ch.lambda_min) lam = Ch.lambda_min;
            if (lam > Ch.lambda_max) lam = Ch.lambda_max;
            Ch.lam[k] = lam;
            Ch.n[k] += 1;
            Ch.vis[k] = 0;
            Ch.acc[k] = 0;
        }
        // sigma_k = sqrt(exp(lambda_k)) = 2^(lambda_k / (2 ln 2))
        Ch.sig[k] = exp2_ordered(__double2float_rn(__dmul_rn(lam, 0.7213475204444817)));
    }
    if (!Ch.weighted || init_only) return;
    __syncthreads();
    // region-weighted target: cumulative share of w_k h_k per epoch, fixed order
    if (threadIdx.x == 0) {
        const double m = (double)Ch.m;
        double S = 0.0;
        for (int k = 0; k < Ch.m; ++k) S = __dadd_rn(S, __dmul_rn(Ch.w[k], (double)(Ch.hist[k] - Ch.hprev[k])));
        if (S > 0.0) {
            double T = 0.0;
            for (int k = 0; k < Ch.m; ++k) {
                Ch.Rc[k] = __dadd_rn(Ch.Rc[k], __ddiv_rn(__dmul_rn(Ch.w[k], (double)(Ch.hist[k] - Ch.hprev[k])), S));
            }
            for (int k = 0; k < Ch.m; ++k) T = __dadd_rn(T, Ch.Rc[k]);
            const double fl = __ddiv_rn(Ch.w_floor, m);
            for (int k = 0; k < Ch.m; ++k) {
                const double s = __ddiv_rn(Ch.Rc[k], T);
                Ch.w[k] = __dmul_rn(m, s > fl ? s : fl);
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < Ch.m; k += blockDim.x) {
        Ch.hprev[k] = Ch.hist[k];
        Ch.wf[k] = __double2float_rn(Ch.w[k]);
    }
}

__global__ void region_update_kernel(const DevChains Ch, int init_only) { region_update_body(Ch, init_only); }

// batched epoch boundary: member b's regions in block b, then its mutation
// index advances by one epoch
__global__ void region_update_batch_kernel(BatchMember* members)
{
    BatchMember* mb = members + blockIdx.x;
    region_update_body(mb->Ch, 0);
    __syncthreads();
    if (mb->tr_lam) {
        // trace instrument: lambda after this epoch's update
        const unsigned long long ep = (mb->mut0 - mb->trace_mut0) / (unsigned long long)mb->Ch.E;
        const unsigned long long m = (unsigned long long)mb->Ch.m;
        if ((ep + 1) * m <= mb->tr_lam_cap)
            for (unsigned long long k = threadIdx.x; k < m; k += blockDim.x) mb->tr_lam[ep * m + k] = mb->Ch.lam[k];
        __syncthreads();
    }
    if (threadIdx.x == 0) mb->mut0 += (unsigned long long)mb->Ch.E;
}

// Refinement pass of the quadtree partition (Sec. 6.2): every leaf visited
// more than qt_split times since the previous pass splits into four children
// that inherit lambda and n / 4 (at least 1) and are not split again in this
// pass; the first child keeps the parent's region id, the others take the
// next free ids, leaves in node order.  Sequential in one thread (the table
// has at most qt_cap leaves); binary64 lambda copied, sigma recomputed.
__global__ void quadtree_refine_kernel(const DevChains Ch)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int m = Ch.qt_state[0], nodes = Ch.qt_state[1];
    const int nodes0 = nodes;
    for (int node = 0; node < nodes0; ++node) {
        if (Ch.qt_child[4 * node] >= 0) continue;
        const int k = Ch.qt_leaf[node];
        if (Ch.hist[k] - Ch.hprev[k] <= (unsigned long long)Ch.qt_split) continue;
        if (Ch.qt_depth[node] >= Ch.qt_max_depth || m + 3 > Ch.qt_cap) continue;
        const double lam = Ch.lam[k];
        const long long nc = Ch.n[k] / 4 > 1 ? Ch.n[k] / 4 : 1;
        const float sg = exp2_ordered(__double2float_rn(__dmul_rn(lam, 0.7213475204444817)));
        for (int q = 0; q < 4; ++q) {
            const int chn = nodes++;
            const int id = q == 0 ? k : m++;
            Ch.qt_child[4 * node + q] = chn;
            for (int j = 0; j < 4; ++j) Ch.qt_child[4 * chn + j] = -1;
            Ch.qt_leaf[chn] = id;
            Ch.qt_depth[chn] = Ch.qt_depth[node] + 1;
            Ch.lam[id] = lam;
            Ch.n[id] = nc;
            Ch.vis[id] = Ch.acc[id] = Ch.hist[id] = Ch.hprev[id] = 0;
            Ch.w[id] = 1.0;
            Ch.Rc[id] = 0.0;
            Ch.Bk[id] = 0.0;
            Ch.wf[id] = 1.0f;
            Ch.sig[id] = sg;
        }
        Ch.qt_leaf[node] = -1;
    }
    for (int k = 0; k < m; ++k) Ch.hprev[k] = Ch.hist[k];
    Ch.qt_state[0] = m;
    Ch.qt_state[1] = nodes;
}

// the chains' cached regions after the partition changed
__global__ void chain_regions_kernel(const DevChains Ch)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= Ch.C) return;
    const size_t C = (size_t)Ch.C;
    uint32_t qv[7] = {Ch.q[c], Ch.q[C + c], 0u, 0u, 0u, 0u, 0u};
    if (Ch.dcells > 1) {
        qv[5] = Ch.q[5 * C + c];
        qv[6] = Ch.q[6 * C + c];
    }
    Ch.k[c] = region_y(Ch, qv);
}

// ---------------------------------------------------------------------------
// epoch-wise stepping of a sharded population: the region statistics the
// chains of every context add during an epoch are summed (by the caller, an
// all-reduce) before the region update, so that all contexts update from the
// same i_k, A_k and h_k (the paper's threads share these counters, Sec. 6).
// Integer sums commute: the tables are identical on every context.
// ---------------------------------------------------------------------------
__global__ void epoch_snapshot_kernel(const DevChains Ch)
{
    const int m = Ch.m;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= m; k += gridDim.x * blockDim.x) {
        if (k == m) {
            Ch.snap[3 * (size_t)m] = Ch.stats[kStLarge];
            continue;
        }
        Ch.snap[k] = Ch.vis[k];
        Ch.snap[(size_t)m + k] = Ch.acc[k];
        Ch.snap[2 * (size_t)m + k] = Ch.hist[k];
        Ch.snapB[k] = Ch.Bk[k];
    }
}

__global__ void epoch_pack_kernel(const DevChains Ch, unsigned long long* counts, double* sums)
{
    const int m = Ch.m;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= m; k += gridDim.x * blockDim.x) {
        if (k == m) {
            counts[3 * (size_t)m] = Ch.stats[kStLarge] - Ch.snap[3 * (size_t)m];
            continue;
        }
        counts[k] = Ch.vis[k] - Ch.snap[k];
        counts[(size_t)m + k] = Ch.acc[k] - Ch.snap[(size_t)m + k];
        counts[2 * (size_t)m + k] = Ch.hist[k] - Ch.snap[2 * (size_t)m + k];
        sums[k] = Ch.Bk[k] - Ch.snapB[k];
    }
}

__global__ void epoch_unpack_kernel(const DevChains Ch, const unsigned long long* counts, const double* sums)
{
    const int m = Ch.m;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= m; k += gridDim.x * blockDim.x) {
        if (k == m) {
            Ch.large_all[0] += counts[3 * (size_t)m];
            continue;
        }
        Ch.vis[k] = Ch.snap[k] + counts[k];
        Ch.acc[k] = Ch.snap[(size_t)m + k] + counts[(size_t)m + k];
        Ch.hist[k] = Ch.snap[2 * (size_t)m + k] + counts[2 * (size_t)m + k];
        Ch.Bk[k] = Ch.snapB[k] + sums[k];
    }
}

__global__ void quadtree_init_kernel(const DevChains Ch)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int j = 0; j < 4; ++j) Ch.qt_child[j] = -1;
    Ch.qt_leaf[0] = 0;
    Ch.qt_depth[0] = 0;
    Ch.qt_state[0] = 1;
    Ch.qt_state[1] = 1;
}

__global__ void fill_regions_kernel(const DevChains Ch, double lambda_init)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Ch.m; k += gridDim.x * blockDim.x) {
        Ch.lam[k] = lambda_init;
        Ch.n[k] = 1;
        Ch.vis[k] = Ch.acc[k] = Ch.hist[k] = Ch.hprev[k] = 0;
        Ch.w[k] = 1.0;
        Ch.Rc[k] = 0.0;
        Ch.wf[k] = 1.0f;
        Ch.Bk[k] = 0.0;
        Ch.sig[k] = exp2_ordered(__double2float_rn(__dmul_rn(lambda_init, 0.7213475204444817)));
    }
}

// ---------------------------------------------------------------------------
// bootstrap (Sec. 3.2: b by independent Monte Carlo in a preprocess) and the
// initial states (systematic resampling of the samples in proportion to pi)
// ---------------------------------------------------------------------------
template <bool BRUTE>
__global__ void __launch_bounds__(kChainBlock) bootstrap_eval_kernel(const DevScene S, const DevChains Ch,
                                                                     long long n_boot, const BootScratch B)
{
    extern __shared__ float4 s_tris[];
    __shared__ uint32_t s_stack[kStackSize * kChainBlock];
    if (BRUTE) stage_triangles(S, s_tris);
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_boot) return;
    uint32_t y[kMaxDim];
    const int D = Ch.D;
    for (int jj = 0; 4 * jj < D; ++jj) {
        const uint4 r = philox((uint32_t)s, (uint32_t)((unsigned long long)s >> 32), 0xFFFFFFFFu,
                               0x8000u + (uint32_t)jj, Ch.seed_lo, Ch.seed_hi);
        y[4 * jj] = r.x;
        if (4 * jj + 1 < D) y[4 * jj + 1] = r.y;
        if (4 * jj + 2 < D) y[4 * jj + 2] = r.z;
        if (4 * jj + 3 < D) y[4 * jj + 3] = r.w;
    }
    V3 f = {0.f, 0.f, 0.f};
    unsigned nn = 0, nt = 0;
    bool overflow = false;
    if (S.toy) {
        const float v = toy_eval(S, y[0], y[1]);
        f = {v, v, v};
    } else {
        Path p;
        Trav T;
        uint32_t* stack = thread_stack(s_stack);
        path_begin(p, S, y);
        while (!p.done) {
            trav_begin(T, p.o, p.d, p.tmax, p.any);
            while (!trav_step<BRUTE>(T, stack, S, s_tris, nn, nt)) {
            }
            if (T.overflow) {
                p.L = {0.f, 0.f, 0.f};
                overflow = true;
                break;
            }
            path_on_hit<BRUTE>(p, S, s_tris, y, Ch.max_depth, Hit{T.t, T.tri, T.ta, T.tb, T.tc});
        }
        f = p.L;
    }
    if (overflow) atomicAdd(B.overflow, 1ull);   // counted: such a path biases b and the starting states
    float pv = lum(f.x, f.y, f.z);
    if (!isfinite(pv)) { f = {0.f, 0.f, 0.f}; pv = 0.f; }
    B.pi[s] = pv;
    B.f[s] = f.x;
    B.f[n_boot + s] = f.y;
    B.f[2 * n_boot + s] = f.z;
    const int k = region_y(Ch, y);
    if (pv != 0.f) atomicAdd(&Ch.Bk[k], (double)pv);
}

// Sum of pi over each chain's slice of K uniform samples [gK, (g+1)K): the
// terms of the normaliser b and of the cumulative distribution below.
__global__ void bootstrap_slice_kernel(const DevChains Ch, long long K, const BootScratch B)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Ch.C_all) return;
    double cum = 0.0;
    for (long long i = 0; i < K; ++i) cum += (double)B.pi[(long long)g * K + i];
    B.partial[g] = cum;
}

// Exclusive prefix of the slice sums in a fixed order (thread t scans its
// contiguous chunk after thread 0 has scanned the chunk sums), and their
// total at prefix[C_all]: the cumulative distribution of pi over all
// samples, slice by slice.  One block.
__global__ void __launch_bounds__(1024) bootstrap_scan_kernel(int C_all, const BootScratch B)
{
    __shared__ double chunk[1024];
    const int t = threadIdx.x, per = (C_all + 1023) / 1024;
    const int b = t * per, e = min(b + per, C_all);
    double acc = 0.0;
    for (int g = b; g < e; ++g) acc += B.partial[g];
    chunk[t] = acc;
    __syncthreads();
    if (t == 0) {
        double run = 0.0;
        for (int k = 0; k < 1024; ++k) {
            const double v = chunk[k];
            chunk[k] = run;
            run += v;
        }
        B.prefix[C_all] = run;
    }
    __syncthreads();
    double run = chunk[t];
    for (int g = b; g < e; ++g) {
        B.prefix[g] = run;
        run += B.partial[g];
    }
}

// Initial state of chain g (global id): systematic resampling of all uniform
// samples in proportion to pi.  Its point t = (g + u_g) / C_all of the total
// (u_g a uniform of its own) falls in the sample s whose cumulative sum first
// exceeds t; so every chain starts on a path that contributes, and the
// starting states together follow pi.  Only this context's chains
// [chain0, chain0 + C) write a state.
__global__ void bootstrap_pick_kernel(const DevChains Ch, long long K, const BootScratch B)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= Ch.C) return;
    const int g = (int)Ch.chain0 + c;
    const int C_all = Ch.C_all;
    const long long n_eff = K * C_all;
    const double total = B.prefix[C_all];
    long long sel = (long long)g * K;   // no sample contributes: the slice's first
    if (total > 0.0) {
        const uint4 r = philox((uint32_t)g, 0u, 0xFFFFFFFFu, 0x7FFEu, Ch.seed_lo, Ch.seed_hi);
        const double tc = ((double)g + (double)u24(r.x)) / (double)C_all * total;
        // the last slice whose prefix is at most tc
        int lo = 0, hi = C_all - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (B.prefix[mid] <= tc) lo = mid;
            else hi = mid - 1;
        }
        double cum = B.prefix[lo];
        long long s = (long long)lo * K;
        sel = -1;
        for (; s < n_eff; ++s) {
            cum += (double)B.pi[s];
            if (cum > tc) {
                sel = s;
                break;
            }
        }
        if (sel < 0)   // tc at the very end (rounding): the last contributing sample
            for (s = n_eff - 1; s >= 0 && sel < 0; --s)
                if (B.pi[s] > 0.f) sel = s;
    }
    const int D = Ch.D, C = Ch.C;
    uint32_t q0 = 0, q1 = 0, q5 = 0, q6 = 0;
    for (int jj = 0; 4 * jj < D; ++jj) {
        const uint4 r = philox((uint32_t)sel, (uint32_t)((unsigned long long)sel >> 32), 0xFFFFFFFFu,
                               0x8000u + (uint32_t)jj, Ch.seed_lo, Ch.seed_hi);
        const uint32_t v[4] = {r.x, r.y, r.z, r.w};
        for (int a = 0; a < 4 && 4 * jj + a < D; ++a) Ch.q[(size_t)(4 * jj + a) * C + c] = v[a];
        if (jj == 0) { q0 = r.x; q1 = r.y; }
        if (jj == 1) { q5 = r.y; q6 = r.z; }
    }
    Ch.f[c] = B.f[sel];
    Ch.f[C + c] = B.f[n_eff + sel];
    Ch.f[2 * C + c] = B.f[2 * n_eff + sel];
    Ch.pi[c] = B.pi[sel];
    const uint32_t qv[7] = {q0, q1, 0u, 0u, 0u, q5, q6};
    Ch.k[c] = region_y(Ch, qv);
}

// fixed-order binary64 sum of the per-chain slice sums (deterministic)
__global__ void __launch_bounds__(256) bootstrap_total_kernel(int C, const BootScratch B)
{
    __shared__ double sh[256];
    const int per = (C + 255) / 256;
    double acc = 0.0;
    for (int i = 0; i < per; ++i) {
        const int c = threadIdx.x * per + i;
        if (c < C) acc += B.partial[c];
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) B.total[0] = sh[0];
}

// ---------------------------------------------------------------------------
// image read-out: plain target I_j W H = (b W H / N) sum f/pi; region-weighted
// target normalised per region by its mass B_k over its visits h_k
// ---------------------------------------------------------------------------
__global__ void read_image_kernel(const DevChains Ch, const double* bhat_total, long long n_boot, double n_total,
                                  int normalized, double* out)
{
    const long long n = (long long)Ch.W * Ch.H;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double s = 1.0;
        if (normalized) {
            const double WH = (double)Ch.W * (double)Ch.H;
            if (!Ch.weighted) {
                const double bhat = bhat_total[0] / (double)n_boot;
                s = n_total > 0.0 ? bhat * WH / n_total : 0.0;
            } else {
                const int x = (int)(i % Ch.W), y = (int)(i / Ch.W);
                const int k = x / Ch.region_px + (y / Ch.region_px) * Ch.nx;
                // uniform samples: the bootstrap plus every large-step proposal
                // (of the whole population when sharded)
                const double nL = Ch.C_all != Ch.C ? (double)Ch.large_all[0] : (double)Ch.stats[kStLarge];
                const double nU = (double)n_boot + nL;
                s = (Ch.hist[k] > 0 && nU > 0.0) ? WH * (Ch.Bk[k] / nU) / (double)Ch.hist[k] : 0.0;
            }
        }
        out[3 * i + 0] = Ch.img[3 * i + 0] * s;
        out[3 * i + 1] = Ch.img[3 * i + 1] * s;
        out[3 * i + 2] = Ch.img[3 * i + 2] * s;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <bool B, bool T, bool K>
static cudaError_t launch_epoch_t(const DevScene& s, const DevChains& c, uint64_t mut0, cudaStream_t st)
{
    constexpr int nt = epoch_block<B>();
    const int blocks = (c.C + nt - 1) / nt;
    const size_t shm = B ? sizeof(float4) * 3 * (size_t)s.n_tris : 0;
    // the 4-D partition has its own instance, so the screen-only kernel carries none of its code;
    // the plain BVH epoch one per BVH4 node layout, so its node step carries one layout's code
    auto kern = c.dcells > 1 ? chain_epoch_kernel<B, T, K, false, true> : chain_epoch_kernel<B, T, K>;
    if (!B && !T && !K && c.dcells <= 1 && s.node_fmt == kNodeBvh4)
        kern = chain_epoch_kernel<B, T, K, false, false, (B || T || K) ? -1 : kNodeBvh4>;
    if (!B && !T && !K && c.dcells <= 1 && s.node_fmt == kNodeBvh4Q)
        kern = chain_epoch_kernel<B, T, K, false, false, (B || T || K) ? -1 : kNodeBvh4Q>;
    if (shm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        if (e != cudaSuccess) return e;
    }
    kern<<<blocks, nt, shm, st>>>(s, c, mut0, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_chain_epoch_member(const BatchMember* member_dev, const BatchMember& member, bool count_work,
                                      cudaStream_t st)
{
    constexpr int nt = epoch_block<false>();
    const int blocks = (member.Ch.C + nt - 1) / nt;
    const unsigned long long* m0 = &member_dev->mut0;
    if (count_work)
        chain_epoch_kernel<false, false, true><<<blocks, nt, 0, st>>>(member.S, member.Ch, 0, m0);
    else if (member.Ch.dcells <= 1 && member.S.node_fmt == kNodeBvh4)
        chain_epoch_kernel<false, false, false, false, false, kNodeBvh4><<<blocks, nt, 0, st>>>(member.S, member.Ch, 0, m0);
    else if (member.Ch.dcells <= 1 && member.S.node_fmt == kNodeBvh4Q)
        chain_epoch_kernel<false, false, false, false, false, kNodeBvh4Q><<<blocks, nt, 0, st>>>(member.S, member.Ch, 0, m0);
    else
        chain_epoch_kernel<false, false, false><<<blocks, nt, 0, st>>>(member.S, member.Ch, 0, m0);
    return cudaGetLastError();
}

template <bool B>
static cudaError_t launch_mala_epoch(const DevScene& s, const DevChains& c, uint64_t mut0, bool trace, cudaStream_t st)
{
    constexpr int nt = epoch_block<B>();
    const int blocks = (c.C + nt - 1) / nt;
    const size_t shm = B ? sizeof(float4) * 3 * (size_t)s.n_tris : 0;
    auto kern = trace ? chain_epoch_kernel<B, true, false, true> : chain_epoch_kernel<B, false, false, true>;
    if (shm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        if (e != cudaSuccess) return e;
    }
    kern<<<blocks, nt, shm, st>>>(s, c, mut0, nullptr);
    return cudaGetLastError();
}

template <class K>
static cudaError_t launch_per_point(K kern, const DevScene& s, long long n, cudaStream_t st, size_t* shm_out)
{
    const size_t shm = s.brute ? sizeof(float4) * 3 * (size_t)s.n_tris : 0;
    if (shm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        if (e != cudaSuccess) return e;
    }
    *shm_out = shm;
    return cudaSuccess;
}

cudaError_t launch_state_gradients(const DevScene& s, const DevChains& c, cudaStream_t st)
{
    size_t shm = 0;
    const unsigned blocks = (unsigned)((c.C + kChainBlock - 1) / kChainBlock);
    cudaError_t e;
    if (s.brute) {
        if ((e = launch_per_point(state_grad_kernel<true>, s, c.C, st, &shm)) != cudaSuccess) return e;
        state_grad_kernel<true><<<blocks, kChainBlock, shm, st>>>(s, c);
    } else {
        state_grad_kernel<false><<<blocks, kChainBlock, 0, st>>>(s, c);
    }
    return cudaGetLastError();
}

cudaError_t launch_path_grad(const DevScene& s, const DevChains& c, const uint32_t* q, long long n, float* f,
                             float* logpi, float* grad, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    size_t shm = 0;
    const unsigned blocks = (unsigned)((n + kChainBlock - 1) / kChainBlock);
    cudaError_t e;
    if (s.brute) {
        if ((e = launch_per_point(path_grad_kernel<true>, s, n, st, &shm)) != cudaSuccess) return e;
        path_grad_kernel<true><<<blocks, kChainBlock, shm, st>>>(s, c, q, n, f, logpi, grad);
    } else {
        path_grad_kernel<false><<<blocks, kChainBlock, 0, st>>>(s, c, q, n, f, logpi, grad);
    }
    return cudaGetLastError();
}

cudaError_t launch_record_paths(const DevScene& s, const DevChains& c, const uint32_t* q, long long n, float* rays,
                                uint32_t* out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    size_t shm = 0;
    const unsigned blocks = (unsigned)((n + kChainBlock - 1) / kChainBlock);
    cudaError_t e;
    if (s.brute) {
        if ((e = launch_per_point(record_paths_kernel<true>, s, n, st, &shm)) != cudaSuccess) return e;
        record_paths_kernel<true><<<blocks, kChainBlock, shm, st>>>(s, c, q, n, rays, out);
    } else {
        record_paths_kernel<false><<<blocks, kChainBlock, 0, st>>>(s, c, q, n, rays, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_chain_epoch(const DevScene& s, const DevChains& c, uint64_t mut0, bool trace, bool count_work,
                               cudaStream_t st)
{
    if (c.T_mala)
        return s.brute ? launch_mala_epoch<true>(s, c, mut0, trace, st) : launch_mala_epoch<false>(s, c, mut0, trace, st);
    if (s.brute) {
        if (trace) return count_work ? launch_epoch_t<true, true, true>(s, c, mut0, st)
                                     : launch_epoch_t<true, true, false>(s, c, mut0, st);
        return count_work ? launch_epoch_t<true, false, true>(s, c, mut0, st)
                          : launch_epoch_t<true, false, false>(s, c, mut0, st);
    }
    if (trace) return count_work ? launch_epoch_t<false, true, true>(s, c, mut0, st)
                                 : launch_epoch_t<false, true, false>(s, c, mut0, st);
    return count_work ? launch_epoch_t<false, false, true>(s, c, mut0, st)
                      : launch_epoch_t<false, false, false>(s, c, mut0, st);
}

cudaError_t launch_large_steps(const DevScene& s, const DevChains& c, uint64_t mut0, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(c.lcount, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const long long n = (long long)c.E * c.C;
    large_collect_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c, mut0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((n + kChainBlock - 1) / kChainBlock);
    const size_t shm = s.brute ? sizeof(float4) * 3 * (size_t)s.n_tris : 0;
    if (s.brute) {
        if (shm > 48 * 1024) {
            e = cudaFuncSetAttribute(large_trace_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
            if (e != cudaSuccess) return e;
        }
        large_trace_kernel<true><<<blocks, kChainBlock, shm, st>>>(s, c, mut0);
    } else {
        large_trace_kernel<false><<<blocks, kChainBlock, 0, st>>>(s, c, mut0);
    }
    return cudaGetLastError();
}

cudaError_t launch_chain_epoch_batch(const BatchMember* members, const int* block_member, int block_base,
                                     int n_blocks, bool count_work, int ctas_per_sm, bool trace, cudaStream_t st)
{
    // 4 resident blocks per SM caps the kernel at 128 registers (a few
    // spills); 3 leaves it unspilled
    const int bb = block_base;
    if (trace) {   // the trace instrument: one instance, speed does not matter
        chain_epoch_batch_kernel<false, 3, true><<<n_blocks, kChainBlock, 0, st>>>(members, block_member, bb);
        return cudaGetLastError();
    }
    if (ctas_per_sm == 3) {
        if (count_work) chain_epoch_batch_kernel<true, 3><<<n_blocks, kChainBlock, 0, st>>>(members, block_member, bb);
        else chain_epoch_batch_kernel<false, 3><<<n_blocks, kChainBlock, 0, st>>>(members, block_member, bb);
    } else {
        if (count_work) chain_epoch_batch_kernel<true, 4><<<n_blocks, kChainBlock, 0, st>>>(members, block_member, bb);
        else chain_epoch_batch_kernel<false, 4><<<n_blocks, kChainBlock, 0, st>>>(members, block_member, bb);
    }
    return cudaGetLastError();
}

cudaError_t launch_region_update_batch(BatchMember* members, int n, cudaStream_t st)
{
    region_update_batch_kernel<<<n, 256, 0, st>>>(members);
    return cudaGetLastError();
}

cudaError_t launch_region_update(const DevChains& c, bool init_only, cudaStream_t st)
{
    region_update_kernel<<<1, 256, 0, st>>>(c, init_only ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_fill_regions(const DevChains& c, double lambda_init, cudaStream_t st)
{
    fill_regions_kernel<<<(c.m + 255) / 256, 256, 0, st>>>(c, lambda_init);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !c.quadtree) return e;
    quadtree_init_kernel<<<1, 1, 0, st>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_quadtree_refine(const DevChains& c, cudaStream_t st)
{
    quadtree_refine_kernel<<<1, 32, 0, st>>>(c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    chain_regions_kernel<<<(c.C + 255) / 256, 256, 0, st>>>(c);
    return cudaGetLastError();
}

static unsigned region_blocks(const DevChains& c)
{
    const long long b = ((long long)c.m + 256) / 256;
    return (unsigned)(b < 1024 ? b : 1024);
}

cudaError_t launch_epoch_snapshot(const DevChains& c, cudaStream_t st)
{
    epoch_snapshot_kernel<<<region_blocks(c), 256, 0, st>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_epoch_pack(const DevChains& c, unsigned long long* counts, double* sums, cudaStream_t st)
{
    epoch_pack_kernel<<<region_blocks(c), 256, 0, st>>>(c, counts, sums);
    return cudaGetLastError();
}

cudaError_t launch_epoch_unpack(const DevChains& c, const unsigned long long* counts, const double* sums,
                                cudaStream_t st)
{
    epoch_unpack_kernel<<<region_blocks(c), 256, 0, st>>>(c, counts, sums);
    return cudaGetLastError();
}

cudaError_t launch_chain_regions(const DevChains& c, cudaStream_t st)
{
    chain_regions_kernel<<<(c.C + 255) / 256, 256, 0, st>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_bootstrap(const DevScene& s, const DevChains& c, int64_t n_boot, const BootScratch& b,
                             cudaStream_t st)
{
    const long long K = n_boot / c.C_all;
    const long long n_eff = K * c.C_all;
    const long long blocks = (n_eff + kChainBlock - 1) / kChainBlock;
    const size_t shm = s.brute ? sizeof(float4) * 3 * (size_t)s.n_tris : 0;
    cudaError_t e;
    if (s.brute) {
        if (shm > 48 * 1024) {
            e = cudaFuncSetAttribute(bootstrap_eval_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
            if (e != cudaSuccess) return e;
        }
        bootstrap_eval_kernel<true><<<(unsigned)blocks, kChainBlock, shm, st>>>(s, c, n_eff, b);
    } else {
        bootstrap_eval_kernel<false><<<(unsigned)blocks, kChainBlock, 0, st>>>(s, c, n_eff, b);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    bootstrap_slice_kernel<<<(c.C_all + 127) / 128, 128, 0, st>>>(c, K, b);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    bootstrap_total_kernel<<<1, 256, 0, st>>>(c.C_all, b);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    bootstrap_scan_kernel<<<1, 1024, 0, st>>>(c.C_all, b);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    bootstrap_pick_kernel<<<(c.C + 127) / 128, 128, 0, st>>>(c, K, b);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// fixed scratch of rmlt_bootstrap_noalloc: one array for the whole process,
// looked up once per device; the bootstrap kernels above run on it unchanged
// ---------------------------------------------------------------------------
namespace {
constexpr size_t na_align(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kNaPi = 0;
constexpr size_t kNaF = na_align(kNaPi + sizeof(float) * RMLT_NOALLOC_MAX_SAMPLES);
constexpr size_t kNaPartial = na_align(kNaF + sizeof(float) * 3 * (size_t)RMLT_NOALLOC_MAX_SAMPLES);
constexpr size_t kNaPrefix = na_align(kNaPartial + sizeof(double) * RMLT_NOALLOC_MAX_CHAINS);
constexpr size_t kNaTotal = na_align(kNaPrefix + sizeof(double) * (RMLT_NOALLOC_MAX_CHAINS + 1));
constexpr size_t kNaChainPi = na_align(kNaTotal + sizeof(double));
constexpr size_t kNaChainK = na_align(kNaChainPi + sizeof(float) * RMLT_NOALLOC_MAX_CHAINS);
constexpr size_t kNaBk = na_align(kNaChainK + sizeof(int32_t) * RMLT_NOALLOC_MAX_CHAINS);
constexpr size_t kNaOverflow = na_align(kNaBk + sizeof(double) * RMLT_NOALLOC_MAX_REGIONS);
constexpr size_t kNaBytes = na_align(kNaOverflow + sizeof(unsigned long long));

__device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mu;
unsigned char* g_na_addr[kNaMaxDevices] = {};
}  // namespace

cudaError_t noalloc_scratch(int device, NoAllocScratch& out)
{
    if (device < 0 || device >= kNaMaxDevices) return cudaErrorInvalidDevice;
    unsigned char* base;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_addr[device]) {
            // host code cannot use g_noalloc_scratch directly: ask the runtime
            // for its device address, with `device` current
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return e;
            g_na_addr[device] = (unsigned char*)p;
        }
        base = g_na_addr[device];
    }
    out.boot.pi = (float*)(base + kNaPi);
    out.boot.f = (float*)(base + kNaF);
    out.boot.partial = (double*)(base + kNaPartial);
    out.boot.prefix = (double*)(base + kNaPrefix);
    out.boot.total = (double*)(base + kNaTotal);
    out.chain_pi = (float*)(base + kNaChainPi);
    out.chain_k = (int32_t*)(base + kNaChainK);
    out.Bk = (double*)(base + kNaBk);
    out.overflow = (unsigned long long*)(base + kNaOverflow);
    out.boot.overflow = out.overflow;
    return cudaSuccess;
}

cudaError_t launch_read_image(const DevChains& c, const double* bhat_total, int64_t n_boot, double n_total,
                              int normalized, double* out, cudaStream_t st)
{
    const long long n = (long long)c.W * c.H;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    read_image_kernel<<<blocks, 256, 0, st>>>(c, bhat_total, n_boot, n_total, normalized, out);
    return cudaGetLastError();
}

}  // namespace rmlt

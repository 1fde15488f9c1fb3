// Wavefront form of the chain epoch (sm_103a).
//
// The chain kernel of rmlt_kernels.cu keeps one chain per thread for a whole
// epoch.  Its warps lose lanes to divergence (lanes at different phases and
// traversal lengths), and a few tens of thousands of chains leave each SM too
// few warps to hide the latency of node fetches.  Here the epoch advances in
// waves, each made of three kernels over compacted work lists:
//
//   shade   one thread per chain with rays in flight: the shadow ray of bounce
//           b-1 and the extension ray of bounce b were traced together; add
//           the next-event contribution if unoccluded, shade the hit
//           (emission, next-event sample, BSDF sample) and queue the next
//           shadow and extension rays, or hand the chain to `setup` when its
//           path has ended;
//   setup   persistent, over the chains whose path ended (all chains in the
//           first wave): accept or reject (Sec. 3.2, Alg. 1, acceptance statistics and state update),
//           then draw the next proposal (Alg. 1, proposal) and queue its camera
//           ray; proposals that need no path finish at once;
//   trace   persistent, one ray per lane: lanes whose ray is resolved pull
//           new rays from the queue together, so warps stay full until the
//           queue runs dry.
//
// A chain's shadow ray of bounce b and its extension ray of bounce b + 1 do
// not depend on each other, so they are traced in the same wave; the
// arithmetic of every path is that of the chain kernel (same functions, same
// order of additions into the radiance), so both forms give identical
// trajectories.  The wave loop is a CUDA graph with a while node whose
// condition the last `setup` block sets from the number of rays queued.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "rmlt_device.cuh"

namespace rmlt {
namespace {

enum WfPhase : uint32_t { kWfIdle = 0, kWfStart = 1, kWfRays = 2, kWfFinish = 3 };
constexpr uint32_t kAnyBit = 0x80000000u;

// word d of one chain's proposal (its row of the [C][D] array)
struct YCol {
    uint32_t* p;
    __device__ __forceinline__ uint32_t& operator[](int d) const { return p[d]; }
};

// dst[c][r] = src[r][c] for a rows x cols matrix of words, in 32 x 32 tiles
__global__ void __launch_bounds__(256) wf_transpose_kernel(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst,
                                                           int rows, int cols)
{
    __shared__ uint32_t tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[k][threadIdx.x] = src[(size_t)r * cols + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && c < cols) dst[(size_t)c * rows + r] = tile[threadIdx.x][k];
    }
}

cudaError_t transpose(const uint32_t* src, uint32_t* dst, int rows, int cols, cudaStream_t st)
{
    const dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    wf_transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(src, dst, rows, cols);
    return cudaGetLastError();
}

struct Slots {
    uint32_t* s;
    int C, c;
    __device__ __forceinline__ uint32_t& operator[](int k) const
    {
        return k < kWRowEnd ? s[(size_t)c * kWfRow + k] : s[(size_t)C * kWfRow + (size_t)(k - kWRowEnd) * C + c];
    }
    __device__ __forceinline__ float f(int k) const { return __uint_as_float((*this)[k]); }
    __device__ __forceinline__ void setf(int k, float v) const { (*this)[k] = __float_as_uint(v); }
    __device__ __forceinline__ V3 v(int k) const { return {f(k), f(k + 1), f(k + 2)}; }
    __device__ __forceinline__ void setv(int k, V3 v) const
    {
        setf(k, v.x);
        setf(k + 1, v.y);
        setf(k + 2, v.z);
    }
};

__device__ __forceinline__ void load_lane(const Slots& s, ChainLane& L)
{
    L.kx = (int)s[kWKx];
    L.px = (int)s[kWPx];
    L.py = (int)s[kWPy];
    L.pix = s.f(kWPix);
    L.fx = s.v(kWFx);
    L.pend_n = s[kWPendN];
    L.pend_i = s[kWPendI];
    L.pend_A = (unsigned long long)s[kWPendA] | ((unsigned long long)s[kWPendA + 1] << 32);
    L.j = (int)s[kWJ];
    const uint32_t fl = s[kWFlags];
    L.large = (int)(fl & 1u);
    L.early = (int)((fl >> 1) & 1u);
    L.ky = (int)s[kWKy];
    L.xi = s.f(kWXi);
    L.R = s.f(kWR);
    L.fy = s.v(kWFy);
}

__device__ __forceinline__ void store_lane(const Slots& s, const ChainLane& L)
{
    s[kWKx] = (uint32_t)L.kx;
    s[kWPx] = (uint32_t)L.px;
    s[kWPy] = (uint32_t)L.py;
    s.setf(kWPix, L.pix);
    s.setv(kWFx, L.fx);
    s[kWPendN] = L.pend_n;
    s[kWPendI] = (uint32_t)L.pend_i;
    s[kWPendA] = (uint32_t)L.pend_A;
    s[kWPendA + 1] = (uint32_t)(L.pend_A >> 32);
    s[kWJ] = (uint32_t)L.j;
    s[kWFlags] = (uint32_t)L.large | ((uint32_t)L.early << 1);
    s[kWKy] = (uint32_t)L.ky;
    s.setf(kWXi, L.xi);
    s.setf(kWR, L.R);
    s.setv(kWFy, L.fy);
}

// Append n (0..2) rays per lane, 2 float4 each, to queue `buf`; every lane of
// the warp calls it.  Lanes take consecutive slots, so the stores coalesce.
__device__ __forceinline__ void append_rays(const DevWave& W, int C, unsigned buf, int n, const float4 (&r)[4])
{
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    unsigned base = 0;
    if (lane == 31 && total > 0) base = atomicAdd(&W.ctr->cnt[buf], (unsigned)total);
    base = __shfl_sync(FULL, base, 31);
    const unsigned at = base + (unsigned)(incl - n), cap = 2u * (unsigned)C;
    float4* q = buf ? W.rq[1] : W.rq[0];   // a runtime index would copy W to local memory
#pragma unroll
    for (int i = 0; i < 2; ++i) {   // constant indices keep r in registers
        if (i < n && at + i < cap) {
            q[2 * (size_t)(at + i)] = r[2 * i];
            q[2 * (size_t)(at + i) + 1] = r[2 * i + 1];
        }
    }
}

// ---------------------------------------------------------------------------
// epoch start: chain state into the per-chain columns, every chain listed for
// its first proposal, counters reset
// ---------------------------------------------------------------------------
__global__ void wf_begin_kernel(const DevChains Ch, const DevWave W, unsigned long long mut0,
                                unsigned long long trace_base)
{
    const int C = Ch.C;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c == 0) {
        WfCounters* k = W.ctr;
        k->wave = k->ticket = k->err = 0u;
        k->fq_count = Ch.E > 0 ? (unsigned)C : 0u;
        k->cnt[0] = k->cnt[1] = k->fetch[0] = k->fetch[1] = 0u;
        k->trace_n = k->trace_buf = 0u;
        k->mut0 = mut0;
        k->trace_base = trace_base;
    }
    if (c >= C) return;
    const Slots s{W.s, C, c};
    s[kWKx] = (uint32_t)Ch.k[c];
    s[kWPx] = (uint32_t)pixel_x(Ch.q[c], Ch.W);
    s[kWPy] = (uint32_t)pixel_x(Ch.q[(size_t)C + c], Ch.H);
    s.setf(kWPix, Ch.pi[c]);
    s.setv(kWFx, {Ch.f[c], Ch.f[(size_t)C + c], Ch.f[2 * (size_t)C + c]});
    s[kWPendN] = s[kWPendI] = s[kWPendA] = s[kWPendA + 1] = 0u;
    s[kWJ] = 0u;
    for (int k = 0; k < 5; ++k) s[kWSt + k] = 0u;
    s[kWRays] = 0u;
    s[kWDropped] = 0u;
    s[kWPhase] = Ch.E > 0 ? kWfStart : kWfIdle;
    W.fq[c] = (uint32_t)c;
}

// ---------------------------------------------------------------------------
// shade: consume the rays traced in the previous wave
// ---------------------------------------------------------------------------
// compiled for 8 resident blocks per SM (64 registers): the kernel waits on
// its slot loads, so more warps in flight pay for a few spilled words
template <bool BRUTE>
__global__ void __launch_bounds__(kChainBlock, 8) wf_shade_kernel(const DevScene S, const DevChains Ch, const DevWave W)
{
    const unsigned FULL = 0xFFFFFFFFu;
    const int C = Ch.C;
    WfCounters* ctr = W.ctr;
    const unsigned wv = ctr->wave, buf = wv & 1u;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr->cnt[buf ^ 1u] = 0u;   // the queue the previous trace pass read
        ctr->fetch[buf] = 0u;      // the pull counter of this wave's trace pass
    }
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    int nr = 0, fin = 0;
    float4 r[4];
    if (c < C) {
        const Slots s{W.s, C, c};
        if (s[kWPhase] == kWfRays) {
            Path p;
            p.T = s.v(kWT);
            p.L = s.v(kWL);
            p.P = s.v(kWP);
            p.b = (int)s[kWB];
            p.o = s.v(kWO);
            p.d = s.v(kWD);
            p.any = 0;
            p.done = 0;
            const uint32_t pfl = s[kWPfl];
            unsigned rays = 0;
            bool dropped = false;
            if (pfl & 2u) {
                ++rays;
                const uint32_t res = s[kWShd];
                if (res == 2u) dropped = true;
                else if (res == 0u) p.L = p.L + p.P;
            }
            int emit = 0;
            float4 sh0, sh1;
            if (pfl & 1u) {
                ++rays;
                const int tri = (int)s[kWHitTri];
                if (tri == -2) {
                    dropped = true;
                } else if (!dropped && tri >= 0) {
                    Hit h;
                    h.t = s.f(kWHitT);
                    h.tri = tri;
                    h.a = __ldg(&S.tris[3 * (size_t)tri]);
                    h.b = __ldg(&S.tris[3 * (size_t)tri + 1]);
                    h.c = __ldg(&S.tris[3 * (size_t)tri + 2]);
                    if (shade_hit<BRUTE>(p, S, h)) {
                        const YCol y{W.y + (size_t)c * Ch.D};
                        if (nee_sample<false>(p, S, nullptr, y)) {
                            sh0 = make_float4(p.o.x, p.o.y, p.o.z, p.tmax);
                            sh1 = make_float4(p.d.x, p.d.y, p.d.z, __uint_as_float((uint32_t)c | kAnyBit));
                            emit |= 2;
                        }
                        path_continue(p, S, y, Ch.max_depth);
                        if (!p.done) emit |= 1;
                    }
                }
            }
            if (dropped) {   // a traversal stack overflowed: the path contributes nothing
                p.L = {0.f, 0.f, 0.f};
                emit = 0;
                s[kWDropped] += 1u;
            }
            s[kWRays] += rays;
            if (emit) {
                s.setv(kWT, p.T);
                s.setv(kWL, p.L);
                s[kWPfl] = (uint32_t)emit;
                if (emit & 1) {
                    s[kWB] = (uint32_t)p.b;
                    s.setv(kWO, p.o);
                    s.setv(kWD, p.d);
                    r[0] = make_float4(p.o.x, p.o.y, p.o.z, p.tmax);
                    r[1] = make_float4(p.d.x, p.d.y, p.d.z, __uint_as_float((uint32_t)c));
                    nr = 1;
                }
                if (emit & 2) {
                    s.setv(kWP, p.P);
                    if (nr) {   // constant indices keep r in registers
                        r[2] = sh0;
                        r[3] = sh1;
                    } else {
                        r[0] = sh0;
                        r[1] = sh1;
                    }
                    ++nr;
                }
            } else {
                s.setv(kWFy, p.L);
                s[kWPhase] = kWfFinish;
                fin = 1;
            }
        }
    }
    append_rays(W, C, buf, nr, r);
    const unsigned m = __ballot_sync(FULL, fin);
    if (m) {
        const int lane = threadIdx.x & 31;
        unsigned base = 0;
        if (lane == __ffs(m) - 1) base = atomicAdd(&ctr->fq_count, (unsigned)__popc(m));
        base = __shfl_sync(FULL, base, __ffs(m) - 1);
        if (fin) W.fq[base + __popc(m & ((1u << lane) - 1u))] = (uint32_t)c;
    }
}

// ---------------------------------------------------------------------------
// setup: finish the mutations whose path ended, draw the next proposals
// ---------------------------------------------------------------------------
// compiled for 6 resident blocks per SM (80 registers, no spills) instead of
// the 3 that 152 registers allowed: the kernel is latency-bound
template <bool TRACE, bool D4 = false>
__global__ void __launch_bounds__(kChainBlock, 6) wf_setup_kernel(const DevScene S, DevChains Ch, const DevWave W)
{
    __shared__ uint32_t s_y[kMaxDim * kChainBlock];
    const int C = Ch.C;
    WfCounters* ctr = W.ctr;
    const unsigned wv = ctr->wave, buf = wv & 1u, n = ctr->fq_count;
    const uint64_t mut0 = ctr->mut0;
    if (TRACE) Ch.trace_base = ctr->trace_base;
    // warp w of block b takes list slots of 32 at (w gridDim + b) 32, so a
    // short list still spreads over every SM
    const unsigned slot = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned base = 0; base < n; base += stride) {
        const unsigned i = base + 32u * slot + (threadIdx.x & 31u);
        int nr = 0;
        float4 r[4];
        if (i < n) {
            const int c = (int)W.fq[i];
            const Slots s{W.s, C, c};
            const YCol y{W.y + (size_t)c * Ch.D};
            const bool traced = TRACE && (uint32_t)c % Ch.trace_stride == 0u;
            ChainLane L;
            load_lane(s, L);
            unsigned st[7];
            for (int k = 0; k < 5; ++k) st[k] = s[kWSt + k];
            st[5] = st[6] = 0u;   // ray counters: the shade kernel's
            Path p;
            if (s[kWPhase] != kWfStart) {
                mutation_finish<TRACE>(Ch, c, traced, L, y, st);
                ++L.j;
            }
            // the proposal is drawn into shared memory (the chain kernel's
            // code path) and stored to [D][C] only when a path needs it
            const YPanel yl = thread_words(s_y);
            bool ray = false;
            while (L.j < Ch.E) {
                if (mutation_setup<false, false, D4>(S, Ch, c, mut0, L, yl, p)) {
                    ray = true;
                    break;
                }
                mutation_finish<TRACE>(Ch, c, traced, L, yl, st);
                ++L.j;
            }
            if (ray) {
                for (int d = 0; d < Ch.D; ++d) y[d] = yl[d];
                s.setv(kWT, p.T);
                s.setv(kWL, p.L);
                s[kWB] = (uint32_t)p.b;
                s.setv(kWO, p.o);
                s.setv(kWD, p.d);
                s[kWPfl] = 1u;
                s[kWPhase] = kWfRays;
                r[0] = make_float4(p.o.x, p.o.y, p.o.z, p.tmax);
                r[1] = make_float4(p.d.x, p.d.y, p.d.z, __uint_as_float((uint32_t)c));
                nr = 1;
            } else {
                // epoch done for this chain: flush and write the state back
                flush_state(Ch, L);
                Ch.k[c] = L.kx;
                Ch.pi[c] = L.pix;
                Ch.f[c] = L.fx.x;
                Ch.f[(size_t)C + c] = L.fx.y;
                Ch.f[2 * (size_t)C + c] = L.fx.z;
                s[kWPhase] = kWfIdle;
            }
            store_lane(s, L);
            for (int k = 0; k < 5; ++k) s[kWSt + k] = st[k];
        }
        append_rays(W, C, buf, nr, r);
    }
    // the last block to finish decides whether another wave runs
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&ctr->ticket, 1u);
        if (t == gridDim.x - 1u) {
            __threadfence();
            const unsigned nq = atomicAdd(&ctr->cnt[buf], 0u);
            ctr->trace_n = nq;
            ctr->trace_buf = buf;
            ctr->fq_count = 0u;
            ctr->ticket = 0u;
            ctr->wave = wv + 1u;
            unsigned go = nq > 0u ? 1u : 0u;
            if (go && wv + 1u >= W.wave_cap) {
                ctr->err = 1u;
                go = 0u;
            }
            if (W.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)W.cond, go);
        }
    }
}

// ---------------------------------------------------------------------------
// trace: persistent; one ray per lane, idle lanes pull rays together
// ---------------------------------------------------------------------------
template <int SS>
struct StackFor {
    using type = SplitStack<SS>;
};
template <>
struct StackFor<kStackSize> {
    using type = uint32_t*;
};

// SS: traversal stack entries per ray kept in shared memory (kStackSize: all;
// fewer: the rest in W.gstack, so more of the SM's memory serves as L1)
// FMT: the node layout compiled in (-1: the scene's, read at each node)
template <bool BRUTE, bool COUNT, int SS = kStackSize, int FMT = -1>
__global__ void __launch_bounds__(kChainBlock) wf_trace_kernel(const DevScene S, const DevWave W, int C,
                                                               unsigned long long* stats)
{
    extern __shared__ float4 s_tris[];
    __shared__ uint32_t s_stack[SS * kChainBlock];
    if (BRUTE) stage_triangles(S, s_tris);
    const unsigned FULL = 0xFFFFFFFFu;
    const unsigned cap = 2u * (unsigned)C, n = min(W.ctr->trace_n, cap), buf = W.ctr->trace_buf;
    const float4* q = buf ? W.rq[1] : W.rq[0];
    unsigned* pull = &W.ctr->fetch[buf];
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const int refill = W.refill, leaf_batch = W.leaf_batch;
    uint32_t* col = s_stack + (threadIdx.x / kStackStride) * (SS * kStackStride) + threadIdx.x % kStackStride;
    typename StackFor<SS>::type stack;
    if constexpr (SS < kStackSize) {
        const size_t nthr = (size_t)gridDim.x * blockDim.x, g = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
        stack.sh = col;
        stack.gl = W.gstack + g;
        stack.gstride = (unsigned)nthr;
    } else {
        stack = col;
    }
    unsigned nn = 0, nt = 0;
    unsigned long long sc[6] = {0, 0, 0, 0, 0, 0};   // scheduling counters (COUNT)
    Trav T;
    T.ref = kNoRef;
    int c = -1;
    bool dry = n == 0u;
    while (true) {
        // the lanes at a leaf and at an inner node (the others are idle):
        // the leaf-turn rule of step_turn, and the refill and exit tests,
        // from the same two votes
        const bool at_leaf = c >= 0 && !BRUTE && (T.ref & kLeafBit);
        const unsigned m_leaf = __ballot_sync(FULL, at_leaf);
        unsigned m_node = __ballot_sync(FULL, c >= 0 && !at_leaf);
        const unsigned idle = ~(m_leaf | m_node);
        if (!dry && __popc(idle) >= refill) {
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(pull, (unsigned)__popc(idle));
            base = __shfl_sync(FULL, base, 0);
            if (base + (unsigned)__popc(idle) >= n) dry = true;
            if (c < 0) {
                const unsigned at = base + (unsigned)__popc(idle & below);
                if (at < n) {
                    const float4 r0 = q[2 * (size_t)at], r1 = q[2 * (size_t)at + 1];
                    const uint32_t tag = __float_as_uint(r1.w);
                    c = (int)(tag & ~kAnyBit);
                    trav_begin(T, v3(r0.x, r0.y, r0.z), v3(r1.x, r1.y, r1.z), r0.w, (tag & kAnyBit) ? 1 : 0);
                }
            }
            m_node |= __ballot_sync(FULL, c >= 0) & idle;   // new rays start at the root, an inner node
        }
        if (dry && (m_leaf | m_node) == 0u) break;
        // as step_turn: leaves take their turn once leaf_batch lanes (or
        // every lane with a ray) wait at one
        const bool leaf_turn = m_leaf && (!m_node || __popc(m_leaf) >= leaf_batch);
        const bool go = c >= 0 && at_leaf == leaf_turn;
        if (COUNT) {
            const unsigned live = __ballot_sync(FULL, c >= 0), stepping = __ballot_sync(FULL, go);
            const unsigned at_leaf = __ballot_sync(FULL, c >= 0 && (T.ref & kLeafBit));
            const bool leaf_turn = (stepping & at_leaf) != 0u;
            sc[0] += 1;
            sc[1] += __popc(stepping);
            sc[2] += __popc(live);
            sc[3] += leaf_turn ? 1 : 0;
            sc[4] += leaf_turn ? 0 : __popc(at_leaf);
            sc[5] += dry ? 1 : 0;
        }
        if (go && trav_step<BRUTE, decltype(stack), FMT>(T, stack, S, s_tris, nn, nt)) {
            if (T.any) {
                Slots{W.s, C, c}[kWShd] = T.overflow ? 2u : (T.tri >= 0 ? 1u : 0u);
            } else {
                Slots{W.s, C, c}[kWHitTri] = T.overflow ? (uint32_t)-2 : (uint32_t)T.tri;
                Slots{W.s, C, c}[kWHitT] = __float_as_uint(T.t);
            }
            c = -1;
        }
    }
    if (COUNT) {
        const unsigned long long a = warp_sum(nn), b = warp_sum(nt);
        if (lane == 0) {
            if (a) atomicAdd(&stats[kStNodes], a);
            if (b) atomicAdd(&stats[kStTris], b);
            for (int s = 0; s < 6; ++s) atomicAdd(&stats[kStIters + s], sc[s]);
        }
    }
}

// ---------------------------------------------------------------------------
// epoch end: per-chain counters into the statistics
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) wf_end_kernel(const DevChains Ch, const DevWave W)
{
    __shared__ unsigned long long part[8][7];
    const int C = Ch.C;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v[7] = {0, 0, 0, 0, 0, 0, 0};
    if (c < C) {
        const Slots s{W.s, C, c};
        for (int k = 0; k < 5; ++k) v[k] = s[kWSt + k];
        v[5] = s[kWRays];
        v[6] = s[kWDropped];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < 7; ++k) {
        const unsigned long long t = warp_sum(v[k]);
        if (lane == 0) part[wid][k] = t;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w][threadIdx.x];
        if (t) atomicAdd(&Ch.stats[threadIdx.x], t);
    }
    if (c == 0) {
        atomicAdd(&Ch.stats[kStWaves], (unsigned long long)W.ctr->wave);
        if (W.ctr->err) atomicAdd(&Ch.stats[kStWaveLimit], 1ull);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

namespace {
int sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// the deeper entries of every trace thread
size_t gstack_words() { return (size_t)(kStackSize - kShortStack) * kWfTraceThreadsPerSm * (size_t)sm_count(); }
}  // namespace

size_t wf_bytes(int C, int D)
{
    const size_t c = (size_t)C;
    return align256(sizeof(uint32_t) * ((size_t)kWfRow + kWfSlots - kWRowEnd) * c) + 2 * align256(sizeof(uint32_t) * (size_t)D * c) +
           2 * align256(sizeof(float4) * 4 * c) + align256(sizeof(uint32_t) * c) + align256(sizeof(WfCounters)) +
           align256(sizeof(uint32_t) * gstack_words());
}

void wf_carve(void* base, int C, int D, DevWave& w)
{
    const size_t c = (size_t)C;
    char* p = (char*)base;
    w.s = (uint32_t*)p;
    p += align256(sizeof(uint32_t) * ((size_t)kWfRow + kWfSlots - kWRowEnd) * c);
    w.y = (uint32_t*)p;
    p += align256(sizeof(uint32_t) * (size_t)D * c);
    w.qa = (uint32_t*)p;
    p += align256(sizeof(uint32_t) * (size_t)D * c);
    for (int b = 0; b < 2; ++b) {
        w.rq[b] = (float4*)p;
        p += align256(sizeof(float4) * 4 * c);
    }
    w.fq = (uint32_t*)p;
    p += align256(sizeof(uint32_t) * c);
    w.ctr = (WfCounters*)p;
    p += align256(sizeof(WfCounters));
    w.gstack = (uint32_t*)p;
}

struct WfGraph {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    std::vector<unsigned char> key;
};

void wf_graph_destroy(WfGraph* g)
{
    if (!g) return;
    if (g->x) cudaGraphExecDestroy(g->x);
    if (g->g) cudaGraphDestroy(g->g);
    delete g;
}

namespace {

template <class T>
void put(std::vector<unsigned char>& k, const T& v)
{
    const unsigned char* b = (const unsigned char*)&v;
    k.insert(k.end(), b, b + sizeof v);
}

// the trace kernel for the wave state's stack layout, with its shared
// memory carve-out set for the layout: the short stack asks for just the
// shared memory of as many resident blocks as the full-stack kernel gets
// (registers bound both), and leaves L1 the rest
template <bool B, bool K>
void* trace_kernel(const DevScene& S, const DevWave& W)
{
    // the plain BVH kernel one per BVH4 node layout, so its node step carries one layout's code
    if (!B && !K && !W.short_stack && S.node_fmt == kNodeBvh4)
        return (void*)wf_trace_kernel<B, K, kStackSize, (B || K) ? -1 : kNodeBvh4>;
    if (!B && !K && !W.short_stack && S.node_fmt == kNodeBvh4Q)
        return (void*)wf_trace_kernel<B, K, kStackSize, (B || K) ? -1 : kNodeBvh4Q>;
    if (!B && W.short_stack) {
        void* k = (void*)wf_trace_kernel<B, K, kShortStack>;
        static bool carved = false;
        if (!carved) {
            int dev = 0, nb = 0, smem_sm = 0;
            cudaFuncAttributes fa{};
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, wf_trace_kernel<B, K>, kChainBlock, 0);
            cudaFuncGetAttributes(&fa, k);
            const size_t need = (size_t)(nb > 0 ? nb : 1) * (fa.sharedSizeBytes + 1024);
            const int pct = smem_sm > 0 ? (int)std::min<size_t>(100, (need * 100 + smem_sm - 1) / smem_sm + 1) : 100;
            cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
            carved = true;
        }
        return k;
    }
    return (void*)wf_trace_kernel<B, K>;
}

template <bool B, bool T, bool K>
cudaError_t build_graph(WfGraph& G, const DevScene& S, const DevChains& Ch, DevWave W, int trace_ctas,
                        int setup_ctas)
{
    cudaError_t e;
    if ((e = cudaGraphCreate(&G.g, 0)) != cudaSuccess) return e;
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, G.g, 1, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
    W.cond = (unsigned long long)h;
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    if ((e = cudaGraphAddNode(&loop, G.g, nullptr, nullptr, 0, &cp)) != cudaSuccess) return e;
    cudaGraph_t body = cp.conditional.phGraph_out[0];

    const size_t tshm = B ? sizeof(float4) * 3 * (size_t)S.n_tris : 0;
    void* kt = trace_kernel<B, K>(S, W);
    if (tshm > 48 * 1024) {
        if ((e = cudaFuncSetAttribute(kt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tshm)) != cudaSuccess)
            return e;
    }
    DevScene s = S;
    DevChains ch = Ch;
    int C = Ch.C;
    unsigned long long* stats = Ch.stats;
    void* a_shade[] = {&s, &ch, &W};
    void* a_setup[] = {&s, &ch, &W};
    void* a_trace[] = {&s, &W, &C, &stats};
    cudaKernelNodeParams k1{}, k2{}, k3{};
    k1.func = (void*)wf_shade_kernel<B>;
    k1.gridDim = dim3((unsigned)((C + kChainBlock - 1) / kChainBlock));
    k1.blockDim = dim3(kChainBlock);
    k1.kernelParams = a_shade;
    k2.func = Ch.dcells > 1 ? (void*)wf_setup_kernel<T, true> : (void*)wf_setup_kernel<T>;
    k2.gridDim = dim3((unsigned)setup_ctas);
    k2.blockDim = dim3(kChainBlock);
    k2.kernelParams = a_setup;
    k3.func = kt;
    k3.gridDim = dim3((unsigned)trace_ctas);
    k3.blockDim = dim3(kChainBlock);
    k3.sharedMemBytes = (unsigned)tshm;
    k3.kernelParams = a_trace;
    cudaGraphNode_t n1, n2, n3;
    if ((e = cudaGraphAddKernelNode(&n1, body, nullptr, 0, &k1)) != cudaSuccess) return e;
    if ((e = cudaGraphAddKernelNode(&n2, body, &n1, 1, &k2)) != cudaSuccess) return e;
    if ((e = cudaGraphAddKernelNode(&n3, body, &n2, 1, &k3)) != cudaSuccess) return e;
    return cudaGraphInstantiate(&G.x, G.g, 0);
}

template <bool B, bool T, bool K>
int trace_occupancy(const DevScene& S, const DevWave& W)
{
    const size_t tshm = B ? sizeof(float4) * 3 * (size_t)S.n_tris : 0;
    int n = 0;
    void* kt = trace_kernel<B, K>(S, W);
    if (tshm > 48 * 1024) cudaFuncSetAttribute(kt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tshm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kt, kChainBlock, tshm);
    if (n > kWfTraceThreadsPerSm / kChainBlock) n = kWfTraceThreadsPerSm / kChainBlock;   // the global stack's room
    return n > 0 ? n : 1;
}

template <bool T>
int setup_occupancy()
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, wf_setup_kernel<T>, kChainBlock, 0);
    return n > 0 ? n : 1;
}

// the waves of one epoch launched from the host: wave_cap waves, those after
// the last chain finished find nothing to do
template <bool B, bool T, bool K>
cudaError_t host_waves(const DevScene& S, const DevChains& Ch, DevWave W, int trace_ctas, int setup_ctas,
                       cudaStream_t st)
{
    W.cond = 0;
    const size_t tshm = B ? sizeof(float4) * 3 * (size_t)S.n_tris : 0;
    void* kt = trace_kernel<B, K>(S, W);
    if (tshm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tshm);
        if (e != cudaSuccess) return e;
    }
    const unsigned g1 = (unsigned)((Ch.C + kChainBlock - 1) / kChainBlock);
    for (unsigned w = 0; w < W.wave_cap; ++w) {
        wf_shade_kernel<B><<<g1, kChainBlock, 0, st>>>(S, Ch, W);
        if (Ch.dcells > 1) wf_setup_kernel<T, true><<<(unsigned)setup_ctas, kChainBlock, 0, st>>>(S, Ch, W);
        else wf_setup_kernel<T><<<(unsigned)setup_ctas, kChainBlock, 0, st>>>(S, Ch, W);
        int C = Ch.C;
        unsigned long long* stats = Ch.stats;
        void* args[] = {(void*)&S, (void*)&W, (void*)&C, (void*)&stats};
        cudaError_t e = cudaLaunchKernel(kt, dim3((unsigned)trace_ctas), dim3(kChainBlock), args, tshm, st);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <bool B, bool T, bool K>
cudaError_t epoch_t(WfGraph** gp, const DevScene& S, const DevChains& Ch, DevWave& W, uint64_t mut0,
                    unsigned long long trace_base, int trace_cps, int setup_cps, bool host_loop, unsigned wave_limit,
                    cudaStream_t st)
{
    const int sms = sm_count();
    const int tocc = trace_occupancy<B, T, K>(S, W), socc = setup_occupancy<T>();
    const int tc = sms * (trace_cps > 0 && trace_cps < tocc ? trace_cps : tocc);
    const int max_setup = (Ch.C + kChainBlock - 1) / kChainBlock;
    int sc = sms * (setup_cps > 0 && setup_cps < socc ? setup_cps : socc);
    if (sc > max_setup) sc = max_setup;
    if (sc < 1) sc = 1;
    // every wave advances each chain with rays by one bounce: E (d + 1) + 2
    // waves finish any epoch; a smaller limit stops it early (counted)
    W.wave_cap = wave_limit ? wave_limit : (unsigned)Ch.E * (unsigned)(Ch.max_depth + 1) + 2u;
    // during the epoch the waves address the states in the row-major copy: a
    // wave's setup list is a sparse subset of the chains, and one chain's
    // words in a row share cache lines where a column layout would give
    // every word its own
    DevChains Cw = Ch;
    Cw.q = W.qa;
    Cw.qd = 1;
    Cw.qc = Ch.D;
    // the graph's kernels hold these values; rebuild when any of them changes
    std::vector<unsigned char> key;
    DevChains kc = Cw;
    kc.trace_base = 0;
    DevWave kw = W;
    kw.cond = 0;
    const int flags = (B ? 1 : 0) | (T ? 2 : 0) | (K ? 4 : 0);
    put(key, flags);
    put(key, S);
    put(key, kc);
    put(key, kw);
    put(key, tc);
    put(key, sc);
    if (host_loop) {
        wf_begin_kernel<<<(Ch.C + 255) / 256, 256, 0, st>>>(Ch, W, mut0, trace_base);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = transpose(Ch.q, W.qa, Ch.D, Ch.C, st);
        if (e == cudaSuccess) e = host_waves<B, T, K>(S, Cw, W, tc, sc, st);
        if (e == cudaSuccess) e = transpose(W.qa, Ch.q, Ch.C, Ch.D, st);
        if (e != cudaSuccess) return e;
        wf_end_kernel<<<(Ch.C + 255) / 256, 256, 0, st>>>(Ch, W);
        return cudaGetLastError();
    }
    WfGraph* g = *gp;
    if (!g || g->key != key) {
        wf_graph_destroy(g);
        *gp = nullptr;
        g = new WfGraph();
        cudaError_t e = build_graph<B, T, K>(*g, S, Cw, W, tc, sc);
        if (e != cudaSuccess) {
            wf_graph_destroy(g);
            return e;
        }
        g->key = key;
        *gp = g;
    }
    wf_begin_kernel<<<(Ch.C + 255) / 256, 256, 0, st>>>(Ch, W, mut0, trace_base);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = transpose(Ch.q, W.qa, Ch.D, Ch.C, st);
    if (e != cudaSuccess) return e;
    if ((e = cudaGraphLaunch(g->x, st)) != cudaSuccess) return e;
    if ((e = transpose(W.qa, Ch.q, Ch.C, Ch.D, st)) != cudaSuccess) return e;
    wf_end_kernel<<<(Ch.C + 255) / 256, 256, 0, st>>>(Ch, W);
    return cudaGetLastError();
}

}  // namespace

cudaError_t wf_epoch(WfGraph** g, const DevScene& s, const DevChains& c, DevWave& w, uint64_t mut0,
                     unsigned long long trace_base, bool trace, bool count_work, int trace_ctas_per_sm,
                     int setup_ctas_per_sm, bool host_loop, unsigned wave_limit, cudaStream_t st)
{
    if (w.refill < 1) w.refill = 1;
    if (w.refill > 32) w.refill = 32;
#define RMLT_WF(B, T, K) \
    epoch_t<B, T, K>(g, s, c, w, mut0, trace_base, trace_ctas_per_sm, setup_ctas_per_sm, host_loop, wave_limit, st)
    if (s.brute) {
        if (trace) return count_work ? RMLT_WF(true, true, true) : RMLT_WF(true, true, false);
        return count_work ? RMLT_WF(true, false, true) : RMLT_WF(true, false, false);
    }
    if (trace) return count_work ? RMLT_WF(false, true, true) : RMLT_WF(false, true, false);
    return count_work ? RMLT_WF(false, false, true) : RMLT_WF(false, false, false);
#undef RMLT_WF
}

}  // namespace rmlt

// Device building blocks shared by the chain kernels of librmlt (sm_103a):
// Philox draws, the binary32 operations that decide integers, ray casting
// against the BVH, the PT + NEE path map as a state machine that asks for one
// ray at a time, and the per-mutation setup / finish of a chain.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "rmlt_internal.h"

namespace rmlt {
namespace {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit multiplies; the key is bumped by the Weyl constants per round.
// Counter layout: mutation draws {mut lo, mut hi, chain, call}; bootstrap
// draws {sample lo, sample hi, 0xFFFFFFFF, 0x8000 + call}; key = seed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

// uniform in [0,1) from the top 24 bits (exact in binary32)
__device__ __forceinline__ float u24(uint32_t x) { return __uint2float_rn(x >> 8) * 5.9604644775390625e-08f; }

// ---------------------------------------------------------------------------
// binary32 arithmetic that decides integers (the quantised small-step offset
// and sigma_k): a fixed sequence of correctly rounded operations, never
// contracted, so every conforming implementation gets the same bits.
// ---------------------------------------------------------------------------
// 2^t: t = n + r with n = rint(t), |r| <= 1/2; 2^r by its Taylor polynomial
// sum_{i<=7} (ln 2)^i r^i / i! in Horner form with fused multiply-adds.
__device__ __forceinline__ float exp2_ordered(float t)
{
    const float n = rintf(t);
    const float r = __fsub_rn(t, n);
    float p = 1.525273365e-05f;
    p = __fmaf_rn(p, r, 1.540352969e-04f);
    p = __fmaf_rn(p, r, 1.333355787e-03f);
    p = __fmaf_rn(p, r, 9.618128650e-03f);
    p = __fmaf_rn(p, r, 5.550410971e-02f);
    p = __fmaf_rn(p, r, 2.402265072e-01f);
    p = __fmaf_rn(p, r, 6.931471825e-01f);
    p = __fmaf_rn(p, r, 1.0f);
    return __fmul_rn(p, __int_as_float(((int)n + 127) << 23));
}

// Kelemen small step: |offset| = sigma s2 (s1/s2)^xi in units of 2^-32.
__device__ __forceinline__ uint32_t kelemen_offset(uint32_t xmag, float sigS2, float log2_ratio)
{
    const float xi = __fmul_rn(__uint2float_rn(xmag >> 8), 5.9604644775390625e-08f);
    const float t = -__fmul_rn(xi, log2_ratio);
    const float m = __fmul_rn(sigS2, exp2_ordered(t));
    return (uint32_t)(unsigned long long)__float2ll_rn(m);
}

__device__ __forceinline__ int pixel_x(uint32_t q0, int W) { return (int)(((unsigned long long)(q0 >> 8) * (unsigned)W) >> 24); }

// luminance, uncontracted so that every kernel that inlines it rounds alike
__device__ __forceinline__ float lum(float r, float g, float b)
{
    return __fadd_rn(__fadd_rn(__fmul_rn(0.2126f, r), __fmul_rn(0.7152f, g)), __fmul_rn(0.0722f, b));
}

// Region of a state in the 2-D screen-space partition (Sec. 5.4): the grid
// cell of its raster position (Sec. 6.1), or the quadtree leaf containing
// (u0, u1) (Sec. 6.2), whose quadrant at depth l is bit 31 - l of u0 and u1.
__device__ __forceinline__ int region_of(const DevChains& Ch, uint32_t q0, uint32_t q1)
{
    if (Ch.quadtree) {
        int node = 0, depth = 0;
        int ch0 = Ch.qt_child[0];
        while (ch0 >= 0) {
            const int bx = (int)((q0 >> (31 - depth)) & 1u), by = (int)((q1 >> (31 - depth)) & 1u);
            node = Ch.qt_child[4 * node + bx + 2 * by];
            ch0 = Ch.qt_child[4 * node];
            ++depth;
        }
        return Ch.qt_leaf[node];
    }
    return pixel_x(q0, Ch.W) / Ch.region_px + (pixel_x(q1, Ch.H) / Ch.region_px) * Ch.nx;
}

// Region of a state's words y: the screen region, crossed (4-D partition in
// PSS, the analogue of the paper's 4-D partition of Sec. 5.4) with a
// dcells x dcells grid over the first bounce's BSDF coordinates (u5, u6).
// D4: the partition is known at compile time to be 4-D (1), screen only (0),
// or read from the table (-1)
template <int D4 = -1, class Y>
__device__ __forceinline__ int region_y(const DevChains& Ch, Y y)
{
    int k = region_of(Ch, y[0], y[1]);
    if (D4 == 1 || (D4 < 0 && Ch.dcells > 1))
        k = k * Ch.dcells * Ch.dcells + pixel_x(y[5], Ch.dcells) + pixel_x(y[6], Ch.dcells) * Ch.dcells;
    return k;
}

// ---------------------------------------------------------------------------
// small float3 helpers
// ---------------------------------------------------------------------------
struct V3 { float x, y, z; };
__device__ __forceinline__ V3 v3(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(V3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
// The library is compiled without automatic contraction (-fmad=false): a
// multiply-add is fused only where it is written as fmaf, so every kernel
// that inlines these helpers rounds the same way.
__device__ __forceinline__ float dot(V3 a, V3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ V3 cross(V3 a, V3 b)
{
    return {fmaf(a.y, b.z, -(a.z * b.y)), fmaf(a.z, b.x, -(a.x * b.z)), fmaf(a.x, b.y, -(a.y * b.x))};
}
__device__ __forceinline__ V3 normalize(V3 a) { return a * (1.0f / sqrtf(dot(a, a))); }
__device__ __forceinline__ V3 xyz(float4 a) { return {a.x, a.y, a.z}; }

// ---------------------------------------------------------------------------
// ray casting
// ---------------------------------------------------------------------------
// Moller-Trumbore without a division on the rejection path: the barycentric
// and distance tests are taken on u det, v det, t det against |det| (the
// same inequalities scaled by |det|); t is divided out only for a hit.
__device__ __forceinline__ bool hit_tri(V3 o, V3 d, float4 a, float4 b, float4 c, float tmax, float& t)
{
    const V3 v0 = xyz(a), e1 = xyz(b), e2 = xyz(c);
    const V3 p = cross(d, e2);
    const float det = dot(e1, p);
    if (det == 0.0f) return false;
    const float sg = det > 0.0f ? 1.0f : -1.0f, ad = fabsf(det);
    const V3 s = o - v0;
    const float u = dot(s, p) * sg;
    const V3 qv = cross(s, e1);
    const float v = dot(d, qv) * sg;
    const float tt = dot(e2, qv) * sg;
    if (!(u >= 0.0f && v >= 0.0f && u + v <= ad && tt > 0.0f && tt < tmax * ad)) return false;
    t = tt / ad;
    return t < tmax;
}

struct Hit {
    float t;
    int tri;
    float4 a, b, c;   // the hit triangle (v0 | material, e1, e2), kept from the leaf test
};

constexpr uint32_t kNoRef = 0xFFFFFFFFu;

// Stepwise traversal: the state of one ray between steps.  A step visits one
// BVH node (both children tested), or the triangles of one leaf, or (brute
// force) the next group of four triangles.
struct Trav {
    V3 o, d, id, ood;
    float t;          // closest hit so far (initially tmax)
    int tri;          // its triangle, -1 if none
    float4 ta, tb, tc;  // its data
    uint32_t ref;     // node / leaf to visit next, kNoRef when done
    int sp, any, overflow;
    int oct;          // bit a set: the ray runs toward -a, so axis a's near plane is the upper bound
};

__device__ __forceinline__ void trav_begin(Trav& T, V3 o, V3 d, float tmax, int any)
{
    T.o = o;
    T.d = d;
    T.id = {1.0f / (fabsf(d.x) > 1e-12f ? d.x : copysignf(1e-12f, d.x)),
            1.0f / (fabsf(d.y) > 1e-12f ? d.y : copysignf(1e-12f, d.y)),
            1.0f / (fabsf(d.z) > 1e-12f ? d.z : copysignf(1e-12f, d.z))};
    T.ood = {o.x * T.id.x, o.y * T.id.y, o.z * T.id.z};
    T.oct = (T.id.x < 0.0f ? 1 : 0) | (T.id.y < 0.0f ? 2 : 0) | (T.id.z < 0.0f ? 4 : 0);
    T.t = tmax;
    T.tri = -1;
    T.ref = 0;
    T.sp = 0;
    T.any = any;
    T.overflow = 0;
}

// This thread's traversal stack in a block's shared array of kStackSize
// entries per thread: panels of kStackStride threads, one column per thread,
// so the lanes of a warp touch consecutive words (no bank conflicts) whatever
// the block size (a multiple of kStackStride).
__device__ __forceinline__ uint32_t* thread_stack(uint32_t* s_stack)
{
    return s_stack + (threadIdx.x / kStackStride) * (kStackSize * kStackStride) + threadIdx.x % kStackStride;
}

// A thread's proposal words in a block's shared array of kMaxDim words per
// thread, in panels of kStackStride columns like the stacks (conflict-free).
// The epoch kernel keeps them there instead of in local memory: at 448
// threads per SM, local copies would take ~110 KB of L1 from the BVH.
struct YPanel {
    uint32_t* p;
    __device__ __forceinline__ uint32_t& operator[](int d) const { return p[d * kStackStride]; }
};
__device__ __forceinline__ YPanel thread_words(uint32_t* s_y)
{
    return YPanel{s_y + (threadIdx.x / kStackStride) * (kMaxDim * kStackStride) + threadIdx.x % kStackStride};
}

// Leaf turns.  A warp's lanes whose ray waits at a leaf test its triangles
// together, once at least kLeafBatch of them (or every lane with a ray) are
// there; until then only the lanes at inner nodes step.  The leaf code is
// the other half of a step (its own loads and triangle tests), and without
// the turns nearly every step of a warp ran both the node and the leaf code.
// A ray's own sequence of steps, and so its result, does not change.  Called
// by all lanes of the warp; `live`: this lane has a ray in traversal.
template <bool BRUTE>
__device__ __forceinline__ bool step_turn(bool live, const Trav& T, int leaf_batch = kLeafBatch)
{
    if (BRUTE) return live;
    const bool at_leaf = live && (T.ref & kLeafBit);
    const unsigned m_leaf = __ballot_sync(0xFFFFFFFFu, at_leaf);
    const unsigned m_node = __ballot_sync(0xFFFFFFFFu, live && !at_leaf);
    const bool leaf_turn = m_leaf && (!m_node || __popc(m_leaf) >= leaf_batch);
    return live && (at_leaf == leaf_turn);
}

// The traversal stack: a thread's column of a shared-memory panel (all
// kStackSize entries), or a split stack whose first SS entries sit in shared
// memory and the rest in a per-thread area of global memory (entry j of the
// thread at gl[(j - SS) * gstride]), which leaves more of the SM's memory to
// the L1 cache.  Both hold kStackSize entries; the traversal is the same.
// stk_push takes the distance at which the ray enters the entry's box and
// stk_next the current bound on the closest hit, for a stack that would drop
// entries beyond it; neither stack keeps them (the keys cost more time than
// the node visits they save).
__device__ __forceinline__ void stk_push(uint32_t* s, int sp, uint32_t v, float) { s[kStackStride * sp] = v; }
__device__ __forceinline__ uint32_t stk_next(uint32_t* s, int& sp, float)
{
    return sp > 0 ? s[kStackStride * --sp] : kNoRef;
}

template <int SS>
struct SplitStack {
    uint32_t* sh;      // this thread's column of the shared panel (SS entries)
    uint32_t* gl;      // this thread's first global entry
    unsigned gstride;  // words between a thread's consecutive global entries
};
template <int SS>
__device__ __forceinline__ void stk_push(const SplitStack<SS>& s, int sp, uint32_t v, float)
{
    if (sp < SS) s.sh[kStackStride * sp] = v;
    else s.gl[(size_t)(sp - SS) * s.gstride] = v;
}
template <int SS>
__device__ __forceinline__ uint32_t stk_next(const SplitStack<SS>& s, int& sp, float)
{
    if (sp == 0) return kNoRef;
    --sp;
    return sp < SS ? s.sh[kStackStride * sp] : s.gl[(size_t)(sp - SS) * s.gstride];
}

// byte k of w as a float: the byte under the exponent of 2^23, whose unit in
// the last place is 1, minus 2^23 (both steps exact)
__device__ __forceinline__ float qbyte(uint32_t w, int k)
{
    return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7440u | (unsigned)k)) - 8388608.0f;
}

// one step; returns true once the ray is resolved
// FMT: the scene's node layout when the kernel was compiled for it (the hot
// kernels are, per layout), or -1 to read it from the scene
template <bool BRUTE, class STK = uint32_t*, int FMT = -1>
__device__ __forceinline__ bool trav_step(Trav& T, STK stack, const DevScene& S, const float4* s_tris,
                                          unsigned& n_nodes, unsigned& n_tris)
{
    const int fmt = FMT >= 0 ? FMT : S.node_fmt;
    if (BRUTE) {
        const int n = S.n_tris;
        const int i0 = (int)T.ref;
        const int i1 = i0 + 4 < n ? i0 + 4 : n;
        bool found = false;
        for (int i = i0; i < i1; ++i) {
            float t;
            const float4 a = s_tris[3 * i], b = s_tris[3 * i + 1], c = s_tris[3 * i + 2];
            if (hit_tri(T.o, T.d, a, b, c, T.t, t)) {
                T.t = t;
                T.tri = i;
                T.ta = a;
                T.tb = b;
                T.tc = c;
                found = true;
            }
        }
        T.ref = (i1 >= n || (T.any && found)) ? kNoRef : (uint32_t)i1;
        return T.ref == kNoRef;
    }
    uint32_t next;
    const uint32_t ref = T.ref;
    if (!(ref & kLeafBit) && fmt != kNodeBvh2) {
        // four children: slab tests, nearest hit child next, the others
        // pushed far to near
        ++n_nodes;
        const float tcap = T.t * 1.00000036f;
        const V3 id = T.id, ood = T.ood;
        float key[4];
        uint32_t cr[4];
        // the near and far planes of each axis are picked by the ray's octant:
        // the distance (plane - o) / d is monotone in the plane with the
        // direction's sign, so the slab test needs no min / max of the two
        if (fmt == kNodeBvh4Q) {
            // 64-byte node: plane p + q s of axis a at distance
            // (p + q s - o) / d = q (s / d) + (p - o) / d
            const float4* nd = &S.nodes[4 * (size_t)ref];
            const float4 h0 = __ldg(nd), h1 = __ldg(nd + 1), qw = __ldg(nd + 2), rf = __ldg(nd + 3);
            const float Ax = h0.w * id.x, Ay = h1.x * id.y, Az = h1.y * id.z;
            const float Bx = fmaf(h0.x, id.x, -ood.x), By = fmaf(h0.y, id.y, -ood.y), Bz = fmaf(h0.z, id.z, -ood.z);
            const uint32_t qlx = __float_as_uint(qw.x), qhx = __float_as_uint(qw.y);
            const uint32_t qly = __float_as_uint(qw.z), qhy = __float_as_uint(qw.w);
            const uint32_t qlz = __float_as_uint(h1.z), qhz = __float_as_uint(h1.w);
            const uint32_t nwx = (T.oct & 1) ? qhx : qlx, fwx = (T.oct & 1) ? qlx : qhx;
            const uint32_t nwy = (T.oct & 2) ? qhy : qly, fwy = (T.oct & 2) ? qly : qhy;
            const uint32_t nwz = (T.oct & 4) ? qhz : qlz, fwz = (T.oct & 4) ? qlz : qhz;
            const uint32_t rr[4] = {__float_as_uint(rf.x), __float_as_uint(rf.y), __float_as_uint(rf.z),
                                    __float_as_uint(rf.w)};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float a0 = fmaf(qbyte(nwx, k), Ax, Bx), b0 = fmaf(qbyte(fwx, k), Ax, Bx);
                const float a1 = fmaf(qbyte(nwy, k), Ay, By), b1 = fmaf(qbyte(fwy, k), Ay, By);
                const float a2 = fmaf(qbyte(nwz, k), Az, Bz), b2 = fmaf(qbyte(fwz, k), Az, Bz);
                const float tn = fmaxf(fmaxf(a0, a1), fmaxf(a2, 0.0f));
                const float tf = fminf(fminf(b0, b1), fminf(b2, tcap));
                const bool hit = tn <= tf;   // an unused slot's inverted box never passes
                key[k] = hit ? tn : INFINITY;
                cr[k] = rr[k];
            }
        } else {
            // 128-byte node: the bounds of the four children in the lanes of
            // six float4 rows, the near / far row of each axis loaded by octant
            const float4* nd = &S.nodes[8 * (size_t)ref];
            const int ox = T.oct & 1, oy = (T.oct >> 1) & 1, oz = (T.oct >> 2) & 1;
            const float4 nx = __ldg(nd + ox), fx = __ldg(nd + 1 - ox), ny = __ldg(nd + 2 + oy), fy = __ldg(nd + 3 - oy);
            const float4 nz = __ldg(nd + 4 + oz), fz = __ldg(nd + 5 - oz), rf = __ldg(nd + 6);
            const float nxs[4] = {nx.x, nx.y, nx.z, nx.w}, fxs[4] = {fx.x, fx.y, fx.z, fx.w};
            const float nys[4] = {ny.x, ny.y, ny.z, ny.w}, fys[4] = {fy.x, fy.y, fy.z, fy.w};
            const float nzs[4] = {nz.x, nz.y, nz.z, nz.w}, fzs[4] = {fz.x, fz.y, fz.z, fz.w};
            const uint32_t rr[4] = {__float_as_uint(rf.x), __float_as_uint(rf.y), __float_as_uint(rf.z),
                                    __float_as_uint(rf.w)};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float a0 = fmaf(nxs[k], id.x, -ood.x), b0 = fmaf(fxs[k], id.x, -ood.x);
                const float a1 = fmaf(nys[k], id.y, -ood.y), b1 = fmaf(fys[k], id.y, -ood.y);
                const float a2 = fmaf(nzs[k], id.z, -ood.z), b2 = fmaf(fzs[k], id.z, -ood.z);
                const float tn = fmaxf(fmaxf(a0, a1), fmaxf(a2, 0.0f));
                const float tf = fminf(fminf(b0, b1), fminf(b2, tcap));
                const bool hit = tn <= tf;   // an unused slot's inverted infinite box never passes
                key[k] = hit ? tn : INFINITY;
                cr[k] = rr[k];
            }
        }
        // sorting network on (key, ref): (0,1) (2,3) (0,2) (1,3) (1,2)
#define RMLT_CSWAP(i, j)                                                    \
        if (key[j] < key[i]) {                                              \
            const float tk = key[i]; key[i] = key[j]; key[j] = tk;          \
            const uint32_t tr = cr[i]; cr[i] = cr[j]; cr[j] = tr;           \
        }
        RMLT_CSWAP(0, 1) RMLT_CSWAP(2, 3) RMLT_CSWAP(0, 2) RMLT_CSWAP(1, 3) RMLT_CSWAP(1, 2)
#undef RMLT_CSWAP
#pragma unroll
        for (int k = 3; k >= 1; --k) {
            if (key[k] != INFINITY) {
                if (T.sp < kStackSize) stk_push(stack, T.sp++, cr[k], key[k]);
                else T.overflow = 1;
            }
        }

        next = key[0] != INFINITY ? cr[0] : stk_next(stack, T.sp, tcap);
    } else if (!(ref & kLeafBit)) {
        ++n_nodes;
        const float4 n0 = __ldg(&S.nodes[4 * ref + 0]);
        const float4 n1 = __ldg(&S.nodes[4 * ref + 1]);
        const float4 n2 = __ldg(&S.nodes[4 * ref + 2]);
        const float4 n3 = __ldg(&S.nodes[4 * ref + 3]);
        const float tcap = T.t * 1.00000036f;
        const V3 id = T.id, ood = T.ood;
        float a0 = fmaf(n0.x, id.x, -ood.x), b0 = fmaf(n0.y, id.x, -ood.x);
        float a1 = fmaf(n0.z, id.y, -ood.y), b1 = fmaf(n0.w, id.y, -ood.y);
        float a2 = fmaf(n2.x, id.z, -ood.z), b2 = fmaf(n2.y, id.z, -ood.z);
        const float tn0 = fmaxf(fmaxf(fminf(a0, b0), fminf(a1, b1)), fmaxf(fminf(a2, b2), 0.0f));
        const float tf0 = fminf(fminf(fmaxf(a0, b0), fmaxf(a1, b1)), fminf(fmaxf(a2, b2), tcap));
        a0 = fmaf(n1.x, id.x, -ood.x); b0 = fmaf(n1.y, id.x, -ood.x);
        a1 = fmaf(n1.z, id.y, -ood.y); b1 = fmaf(n1.w, id.y, -ood.y);
        a2 = fmaf(n2.z, id.z, -ood.z); b2 = fmaf(n2.w, id.z, -ood.z);
        const float tn1 = fmaxf(fmaxf(fminf(a0, b0), fminf(a1, b1)), fmaxf(fminf(a2, b2), 0.0f));
        const float tf1 = fminf(fminf(fmaxf(a0, b0), fmaxf(a1, b1)), fminf(fmaxf(a2, b2), tcap));
        const bool h0 = tn0 <= tf0, h1 = tn1 <= tf1;
        const uint32_t c0 = __float_as_uint(n3.x), c1 = __float_as_uint(n3.y);
        if (h0 && h1) {
            const bool first0 = tn0 <= tn1;
            if (T.sp < kStackSize) stk_push(stack, T.sp++, first0 ? c1 : c0, first0 ? tn1 : tn0);
            else T.overflow = 1;
            next = first0 ? c0 : c1;
        } else if (h0) {
            next = c0;
        } else if (h1) {
            next = c1;
        } else {
            next = stk_next(stack, T.sp, tcap);
        }
    } else {
        const uint32_t first = ref & 0x0FFFFFFFu, cnt = ((ref >> 28) & 7u) + 1u;
        bool found = false;
        // two triangles per pass: both loads in flight before either test
        for (uint32_t i = first; i < first + cnt; i += 2) {
            const bool two = i + 1 < first + cnt;
            const uint32_t i1 = two ? i + 1 : i;
            const float4 a = __ldg(&S.tris[3 * i]), b = __ldg(&S.tris[3 * i + 1]), c = __ldg(&S.tris[3 * i + 2]);
            const float4 a1 = __ldg(&S.tris[3 * i1]), b1 = __ldg(&S.tris[3 * i1 + 1]), c1 = __ldg(&S.tris[3 * i1 + 2]);
            float t;
            ++n_tris;
            if (hit_tri(T.o, T.d, a, b, c, T.t, t)) {
                T.t = t;
                T.tri = (int)i;
                T.ta = a;
                T.tb = b;
                T.tc = c;
                found = true;
            }
            if (two) {
                ++n_tris;
                if (hit_tri(T.o, T.d, a1, b1, c1, T.t, t)) {
                    T.t = t;
                    T.tri = (int)i1;
                    T.ta = a1;
                    T.tb = b1;
                    T.tc = c1;
                    found = true;
                }
            }
        }
        next = (T.any && found) ? kNoRef : stk_next(stack, T.sp, T.t * 1.00000036f);
    }
    T.ref = T.overflow ? kNoRef : next;
    return T.ref == kNoRef;
}

// ---------------------------------------------------------------------------
// path map u -> f(u): pinhole camera through (u0 W, u1 H); bounce b uses
// dims 2+5b..6+5b = (light select, light u, light v, BSDF u, BSDF v);
// emission on the camera ray's hit; NEE at every interaction (light triangle
// in proportion to area, uniform point, one-sided emitters); Lambert cosine
// or GGX half-vector sampling; no Russian roulette.  Written as a state
// machine that asks for one ray at a time.
// ---------------------------------------------------------------------------
struct Path {
    V3 o, d;
    float tmax;
    int any;          // 1: the pending ray is a shadow ray
    V3 T, L, P;       // throughput, radiance, NEE contribution awaiting visibility
    V3 x, ns, wo;     // interaction waiting for its BSDF continuation
    int mat, b, done;
};

template <class Y>
__device__ __forceinline__ void path_begin(Path& p, const DevScene& S, Y y)
{
    const float sx = (2.0f * u24(y[0]) - 1.0f) * S.tan_x;
    const float sy = (1.0f - 2.0f * u24(y[1])) * S.tan_y;
    const V3 fw = {S.cam_fwd[0], S.cam_fwd[1], S.cam_fwd[2]};
    const V3 rt = {S.cam_right[0], S.cam_right[1], S.cam_right[2]};
    const V3 up = {S.cam_up[0], S.cam_up[1], S.cam_up[2]};
    p.o = {S.cam_pos[0], S.cam_pos[1], S.cam_pos[2]};
    p.d = normalize(fw + rt * sx + up * sy);
    p.tmax = 3.0e38f;
    p.any = 0;
    p.T = {1.f, 1.f, 1.f};
    p.L = {0.f, 0.f, 0.f};
    p.b = 0;
    p.done = 0;
}

__device__ __forceinline__ float ggx_g1(float c, float a2)
{
    if (c <= 0.0f) return 0.0f;
    return 2.0f * c / (c + sqrtf(a2 + (1.0f - a2) * c * c));
}

__device__ __forceinline__ void frame(V3 n, V3& t, V3& b)
{
    if (fabsf(n.z) < 0.9f) t = v3(-n.y, n.x, 0.0f);
    else t = v3(0.0f, -n.z, n.y);
    t = normalize(t);
    b = cross(n, t);
}

__device__ __forceinline__ V3 bsdf_eval(float4 m0, float4 m1, V3 wo, V3 wi, V3 n)
{
    if (m0.w == 0.0f) {
        const float k = 0.318309886183790672f;   // 1 / pi
        return {m0.x * k, m0.y * k, m0.z * k};
    }
    const float co = dot(n, wo), ci = dot(n, wi);
    if (co <= 0.0f || ci <= 0.0f) return {0.f, 0.f, 0.f};
    const V3 h = normalize(wo + wi);
    const float ch = dot(n, h), a2 = m1.w * m1.w;
    const float den = 1.0f + (a2 - 1.0f) * ch * ch;
    const float D = a2 / (3.14159265358979f * den * den);
    const float G = ggx_g1(co, a2) * ggx_g1(ci, a2);
    const float x = 1.0f - dot(wi, h), x2 = x * x, c5 = x2 * x2 * x;
    const float s = D * G / (4.0f * co * ci);
    return {(m0.x + (1.0f - m0.x) * c5) * s, (m0.y + (1.0f - m0.y) * c5) * s, (m0.z + (1.0f - m0.z) * c5) * s};
}

// after NEE at interaction b: sample the BSDF to continue, or finish
template <class Y>
__device__ __forceinline__ void path_continue(Path& p, const DevScene& S, Y y, int max_depth)
{
    if (p.b == max_depth - 1) { p.done = 1; return; }
    const float bu = u24(y[5 + 5 * p.b]), bv = u24(y[6 + 5 * p.b]);
    const float4 m0 = __ldg(&S.mats[3 * p.mat]), m1 = __ldg(&S.mats[3 * p.mat + 1]);
    V3 ft, fb;
    frame(p.ns, ft, fb);
    float sp, cp;
    sincospif(2.0f * bv, &sp, &cp);
    V3 wi;
    if (m0.w == 0.0f) {
        const float r = sqrtf(bu);
        wi = ft * (r * cp) + fb * (r * sp) + p.ns * sqrtf(fmaxf(0.0f, 1.0f - bu));
        p.T = {p.T.x * m0.x, p.T.y * m0.y, p.T.z * m0.z};
    } else {
        const float a2 = m1.w * m1.w;
        const float tan2 = a2 * bu / (1.0f - bu);
        const float cm = 1.0f / sqrtf(1.0f + tan2);
        const float sm = sqrtf(fmaxf(0.0f, 1.0f - cm * cm));
        const V3 mv = ft * (sm * cp) + fb * (sm * sp) + p.ns * cm;
        const float dom = dot(p.wo, mv);
        if (dom <= 0.0f) { p.done = 1; return; }
        wi = mv * (2.0f * dom) - p.wo;
        const float ci = dot(wi, p.ns), co = dot(p.wo, p.ns);
        if (ci <= 0.0f) { p.done = 1; return; }
        const float G = ggx_g1(co, a2) * ggx_g1(ci, a2);
        const float x = 1.0f - dom, x2 = x * x, c5 = x2 * x2 * x;
        const float s = G * dom / (co * cm);
        p.T = {p.T.x * (m0.x + (1.0f - m0.x) * c5) * s, p.T.y * (m0.y + (1.0f - m0.y) * c5) * s,
               p.T.z * (m0.z + (1.0f - m0.z) * c5) * s};
    }
    p.o = p.x + p.ns * S.eps;
    p.d = wi;
    p.tmax = 3.0e38f;
    p.any = 0;
    p.b += 1;
}

template <bool BRUTE>
__device__ __forceinline__ float4 tri_load(const DevScene& S, const float4* s_tris, int i, int j)
{
    return BRUTE ? s_tris[3 * i + j] : __ldg(&S.tris[3 * i + j]);
}

// Interaction at the closest hit h of the pending camera / extension ray:
// emission seen by the camera ray, then the interaction kept for the
// next-event sample and the BSDF continuation; false when the path ends here
// (an emitter that absorbs).
template <bool BRUTE>
__device__ __forceinline__ bool shade_hit(Path& p, const DevScene& S, const Hit& h)
{
    const float4 ta = h.a, tb = h.b, tc = h.c;
    const V3 n = normalize(cross(xyz(tb), xyz(tc)));
    const int mat = __float_as_int(ta.w);
    const V3 x = p.o + p.d * h.t;
    const float cosi = -dot(n, p.d);
    const V3 ns = cosi > 0.0f ? n : n * -1.0f;
    const float4 m1 = __ldg(&S.mats[3 * mat + 1]), m2 = __ldg(&S.mats[3 * mat + 2]);
    if (p.b == 0 && m2.x != 0.0f && cosi > 0.0f) p.L = p.L + v3(p.T.x * m1.x, p.T.y * m1.y, p.T.z * m1.z);
    if (m2.y != 0.0f) return false;
    p.x = x;
    p.ns = ns;
    p.wo = p.d * -1.0f;
    p.mat = mat;
    return true;
}

// Next-event sample at the interaction (light triangle in proportion to
// area, uniform point): on a usable sample, P holds the unoccluded
// contribution and (o, d, tmax) the shadow ray; false when there is none.
template <bool BRUTE, class Y>
__device__ __forceinline__ bool nee_sample(Path& p, const DevScene& S, const float4* s_tris, Y y)
{
    if (S.n_lights <= 0) return false;
    const V3 x = p.x, ns = p.ns;
    const float ls = u24(y[2 + 5 * p.b]), lu = u24(y[3 + 5 * p.b]), lv = u24(y[4 + 5 * p.b]);
    int lo = 0, hi = S.n_lights - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&S.light_cdf[mid]) > ls) hi = mid; else lo = mid + 1;
    }
    const int lt = __ldg(&S.light_tri[lo]);
    const float4 la = tri_load<BRUTE>(S, s_tris, lt, 0), lb = tri_load<BRUTE>(S, s_tris, lt, 1),
                 lc = tri_load<BRUTE>(S, s_tris, lt, 2);
    const float su = sqrtf(lu), b1 = su * (1.0f - lv), b2 = su * lv;
    const V3 pl = xyz(la) + xyz(lb) * b1 + xyz(lc) * b2;
    V3 wi = pl - x;
    const float dist2 = dot(wi, wi), dist = sqrtf(dist2);
    wi = wi * (1.0f / dist);
    const V3 ln = normalize(cross(xyz(lb), xyz(lc)));
    const float cx = dot(ns, wi), cl = -dot(ln, wi);
    if (!(cx > 0.0f && cl > 0.0f)) return false;
    const V3 xo = x + ns * S.eps;
    V3 sd = pl - xo;
    const float sdist = sqrtf(dot(sd, sd));
    if (!(sdist > 2.0f * S.eps)) return false;
    const float4 m0 = __ldg(&S.mats[3 * p.mat]), m1 = __ldg(&S.mats[3 * p.mat + 1]);
    const V3 fr = bsdf_eval(m0, m1, p.wo, wi, ns);
    const float4 lm1 = __ldg(&S.mats[3 * __float_as_int(la.w) + 1]);
    const float g = cx * cl / dist2 * S.light_area;
    p.P = {p.T.x * fr.x * lm1.x * g, p.T.y * fr.y * lm1.y * g, p.T.z * fr.z * lm1.z * g};
    p.o = xo;
    p.d = sd * (1.0f / sdist);
    p.tmax = sdist - S.eps;
    return true;
}

// consume the result of the pending ray (one ray at a time: the shadow ray
// of bounce b is resolved before its BSDF continuation is drawn)
template <bool BRUTE, class Y>
__device__ __forceinline__ void path_on_hit(Path& p, const DevScene& S, const float4* s_tris, Y y,
                                            int max_depth, Hit h)
{
    if (p.any) {
        if (h.tri < 0) p.L = p.L + p.P;
        p.any = 0;
        path_continue(p, S, y, max_depth);
        return;
    }
    if (h.tri < 0) { p.done = 1; return; }
    if (!shade_hit<BRUTE>(p, S, h)) { p.done = 1; return; }
    if (nee_sample<BRUTE>(p, S, s_tris, y)) {
        p.any = 1;
        return;
    }
    path_continue(p, S, y, max_depth);
}

__device__ __forceinline__ float toy_eval(const DevScene& S, uint32_t q0, uint32_t q1)
{
    const float u0 = u24(q0), u1 = u24(q1);
    float f = S.toy_p[0];
    if (u0 >= S.toy_p[2] && u0 < S.toy_p[3] && u1 >= S.toy_p[4] && u1 < S.toy_p[5]) f += S.toy_p[1];
    const float dx = u0 - S.toy_p[7], dy = u1 - S.toy_p[8];
    f += S.toy_p[6] * expf(-(dx * dx + dy * dy) / (2.0f * S.toy_p[9] * S.toy_p[9]));
    return f;
}

// ---------------------------------------------------------------------------
// gradient of log pi(u) by reverse-mode differentiation (adjoint): the path
// is evaluated once with the functions above while each bounce's ray, hit
// distance, normal and throughput are recorded; the adjoint sweep then runs
// from the last bounce back to the camera.  Discrete choices (hit triangle,
// light triangle, visibility) are held fixed: this is the gradient of the
// smooth piece of f containing u.  Covers Lambertian and emitting surfaces
// (a Lambertian throughput is constant, so only the geometry carries
// derivatives): dims 3 + 5b, 4 + 5b move the light point, 5 + 5b, 6 + 5b the
// continuation direction, 0 and 1 the camera ray.
// ---------------------------------------------------------------------------
constexpr float kMalaTauMax = 0.01f;

struct GradRec {
    V3 o, d;          // the ray that found bounce b's hit
    float t;
    V3 ns;            // oriented normal at the hit
    V3 T;             // throughput at the hit
    int mat;
    int nee;          // 1: the next-event sample was unoccluded and counted
    int cont;         // 1: the BSDF continuation was drawn
};

// Forward evaluation with the record; returns the number of recorded bounces
// (-1 after a traversal-stack overflow, -2 on a non-Lambertian surface).
template <bool BRUTE, class Y>
__device__ __forceinline__ int path_forward_rec(const DevScene& S, const float4* s_tris, uint32_t* stack, Y y,
                                                int max_depth, GradRec* rec, V3& Lout, unsigned& rays)
{
    Path p;
    Trav T;
    unsigned nn = 0, nt = 0;
    path_begin(p, S, y);
    int nb = 0;
    Lout = {0.f, 0.f, 0.f};
    while (true) {
        trav_begin(T, p.o, p.d, p.tmax, 0);
        while (!trav_step<BRUTE>(T, stack, S, s_tris, nn, nt)) {
        }
        ++rays;
        if (T.overflow) return -1;
        if (T.tri < 0) break;
        const V3 o = p.o, d = p.d, Tb = p.T;
        const Hit h{T.t, T.tri, T.ta, T.tb, T.tc};
        // an emitter that ends the path adds only its constant emission: no record
        if (!shade_hit<BRUTE>(p, S, h)) break;
        if (__ldg(&S.mats[3 * p.mat]).w != 0.0f) return -2;
        GradRec& r = rec[nb];
        r.o = o;
        r.d = d;
        r.t = T.t;
        r.T = Tb;
        r.ns = p.ns;
        r.mat = p.mat;
        r.nee = 0;
        r.cont = 0;
        ++nb;
        if (nee_sample<BRUTE>(p, S, s_tris, y)) {
            trav_begin(T, p.o, p.d, p.tmax, 1);
            while (!trav_step<BRUTE>(T, stack, S, s_tris, nn, nt)) {
            }
            ++rays;
            if (T.overflow) return -1;
            if (T.tri < 0) {
                p.L = p.L + p.P;
                r.nee = 1;
            }
        }
        path_continue(p, S, y, max_depth);
        if (p.done) break;
        r.cont = 1;
    }
    Lout = p.L;
    return nb;
}

// Adjoint sweep: g[d] = d log pi / d u_d for d < D (zero where pi <= 0).
template <class Y, class G>
__device__ __forceinline__ void path_adjoint(const DevScene& S, Y y, const GradRec* rec, int nb, V3 L, G g, int D)
{
    for (int d = 0; d < D; ++d) g[d] = 0.0f;
    const float pi = lum(L.x, L.y, L.z);
    if (!(pi > 0.0f)) return;
    const float inv_pi = 1.0f / pi;
    V3 ob = {0.f, 0.f, 0.f}, db = {0.f, 0.f, 0.f};   // adjoints of the next bounce's ray
    for (int b = nb - 1; b >= 0; --b) {
        const GradRec& r = rec[b];
        const V3 ns = r.ns;
        const V3 x = r.o + r.d * r.t;
        V3 xb = ob;                                    // o_{b+1} = x + eps ns
        if (r.cont) {                                  // d_{b+1}: Lambert cosine sample of (bu, bv)
            const float bu = u24(y[5 + 5 * b]), bv = u24(y[6 + 5 * b]);
            V3 ft, fb;
            frame(ns, ft, fb);
            float sp, cp;
            sincospif(2.0f * bv, &sp, &cp);
            const float rr = sqrtf(bu), lz = sqrtf(fmaxf(0.0f, 1.0f - bu));
            const float ir = rr > 0.0f ? 0.5f / rr : 0.0f, il = lz > 0.0f ? 0.5f / lz : 0.0f;
            const V3 d_bu = ft * (cp * ir) + fb * (sp * ir) - ns * il;
            const V3 d_bv = (fb * (rr * cp) - ft * (rr * sp)) * 6.28318530717958648f;
            g[5 + 5 * b] = dot(db, d_bu);
            g[6 + 5 * b] = dot(db, d_bv);
        }
        if (r.nee) {                                   // P_b = T (rho / pi) Le cx cl / dist^2 A
            const float ls = u24(y[2 + 5 * b]), lu = u24(y[3 + 5 * b]), lv = u24(y[4 + 5 * b]);
            int lo = 0, hi = S.n_lights - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(&S.light_cdf[mid]) > ls) hi = mid; else lo = mid + 1;
            }
            const int lt = __ldg(&S.light_tri[lo]);
            const float4 la = __ldg(&S.tris[3 * lt]), lb = __ldg(&S.tris[3 * lt + 1]), lc = __ldg(&S.tris[3 * lt + 2]);
            const float su = sqrtf(lu), b1 = su * (1.0f - lv), b2 = su * lv;
            const V3 pl = xyz(la) + xyz(lb) * b1 + xyz(lc) * b2;
            const V3 wv = pl - x;
            const float s2 = dot(wv, wv);
            const V3 ln = normalize(cross(xyz(lb), xyz(lc)));
            const float a = dot(ns, wv), c = -dot(ln, wv);
            const float gg = a * c / (s2 * s2) * S.light_area;
            const float4 m0 = __ldg(&S.mats[3 * r.mat]);
            const float4 lm1 = __ldg(&S.mats[3 * __float_as_int(la.w) + 1]);
            const float k1 = 0.318309886183790672f;
            const float kappa = lum(r.T.x * m0.x * k1 * lm1.x, r.T.y * m0.y * k1 * lm1.y, r.T.z * m0.z * k1 * lm1.z) *
                                inv_pi;
            const V3 dg = (ns * c - ln * a) * (S.light_area / (s2 * s2)) - wv * (4.0f * gg / s2);
            const V3 wvb = dg * kappa;
            xb = xb - wvb;
            const V3 d_lu = (xyz(lb) * (1.0f - lv) + xyz(lc) * lv) * (su > 0.0f ? 0.5f / su : 0.0f);
            const V3 d_lv = (xyz(lc) - xyz(lb)) * su;
            g[3 + 5 * b] = dot(wvb, d_lu);
            g[4 + 5 * b] = dot(wvb, d_lv);
        }
        // hit on the triangle's plane: x = o + t d, t = (v0 - o).n / d.n
        const float xd = dot(xb, r.d), dn = dot(r.d, ns);
        ob = xb - ns * (xd / dn);
        db = ob * r.t;
    }
    // camera: d_0 = dr / |dr|, dr = fwd + right sx + up sy
    const float sx = (2.0f * u24(y[0]) - 1.0f) * S.tan_x;
    const float sy = (1.0f - 2.0f * u24(y[1])) * S.tan_y;
    const V3 fw = {S.cam_fwd[0], S.cam_fwd[1], S.cam_fwd[2]};
    const V3 rt = {S.cam_right[0], S.cam_right[1], S.cam_right[2]};
    const V3 up = {S.cam_up[0], S.cam_up[1], S.cam_up[2]};
    const V3 dr = fw + rt * sx + up * sy;
    const float il = 1.0f / sqrtf(dot(dr, dr));
    const V3 d0 = dr * il;
    const V3 drb = (db - d0 * dot(d0, db)) * il;
    g[0] = dot(drb, rt) * (2.0f * S.tan_x);
    g[1] = -dot(drb, up) * (2.0f * S.tan_y);
}

// toy integrand: f and grad log f in closed form (D = 2)
template <class G>
__device__ __forceinline__ float toy_grad(const DevScene& S, uint32_t q0, uint32_t q1, G g)
{
    const float u0 = u24(q0), u1 = u24(q1);
    const float f = toy_eval(S, q0, q1);
    const float dx = u0 - S.toy_p[7], dy = u1 - S.toy_p[8];
    const float e = S.toy_p[6] * expf(-(dx * dx + dy * dy) / (2.0f * S.toy_p[9] * S.toy_p[9]));
    const float k = -e / (S.toy_p[9] * S.toy_p[9] * f);
    g[0] = f > 0.0f ? k * dx : 0.0f;
    g[1] = f > 0.0f ? k * dy : 0.0f;
    return f;
}

__device__ __forceinline__ void stage_triangles(const DevScene& S, float4* s_tris)
{
    for (int i = threadIdx.x; i < 3 * S.n_tris; i += blockDim.x) s_tris[i] = __ldg(&S.tris[i]);
    __syncthreads();
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// the chain step: E mutations per chain (Alg. 1, mutation loop)
// ---------------------------------------------------------------------------
struct ChainLane {
    // cached current state x
    int kx, px, py;
    float pix;
    V3 fx;
    // visits, splats and statistics of x not yet flushed
    unsigned pend_n;
    unsigned long long pend_i, pend_A;
    // the mutation in flight
    int j, large, ky, early;
    float xi;
    float R;          // kernel ratio T_{k(y)}(x|y) / T_{k(x)}(y|x) of a truncated-normal small step (else 1)
    V3 fy;
    // Langevin strategy: this mutation is one (its acceptance probability
    // decided at the proposal), and moves proposed / accepted so far
    int mala;
    float amala;
    unsigned n_mala, n_mala_acc;
};

// ---------------------------------------------------------------------------
// Langevin strategy (MALA with a bounded drift): y = x + m_x + sqrt(tau_x) xi,
// m_x = (tau_x / 2) grad log pi(x) scaled to norm <= drift_max, tau_x =
// min(tau sigma_{k(x)}^2, 0.01) (a standard deviation of at most 0.1 keeps
// the nearest-image density on the torus exact to e^-12); xi ~ N(0, I) by
// Box-Muller from the mutation's Philox draws
// (call 1 + j gives dims 4j..4j+3).  The acceptance carries the ratio of the
// state-dependent proposal densities q(x|y) / q(y|x) with nearest-image
// displacements on the torus; the region weight of the weighted target is
// constant inside a region and drops out of the gradient.
// ---------------------------------------------------------------------------
template <bool BRUTE, class Y>
__device__ __forceinline__ void mala_setup(const DevScene& S, const DevChains& Ch, int c, uint32_t mlo, uint32_t mhi,
                                           ChainLane& L, Y y, uint32_t* stack, const float4* s_tris,
                                           unsigned& rays)
{
    const int C = Ch.C, D = Ch.D;
    if (isnan(Ch.G[c])) {
        // the state was reached by another strategy: its gradient first
        uint32_t yx[kMaxDim];
        float gx[kMaxDim];
        for (int d = 0; d < D; ++d) yx[d] = Ch.q[(size_t)d * Ch.qd + (size_t)c * Ch.qc];
        if (S.toy) {
            toy_grad(S, yx[0], yx[1], gx);
        } else {
            GradRec rec[RMLT_MAX_DEPTH];
            V3 fx;
            const int nb = path_forward_rec<BRUTE>(S, s_tris, stack, yx, Ch.max_depth, rec, fx, rays);
            if (nb < 0) {
                for (int d = 0; d < D; ++d) gx[d] = 0.0f;
            } else {
                path_adjoint(S, yx, rec, nb, fx, gx, D);
            }
        }
        for (int d = 0; d < D; ++d) Ch.G[(size_t)d * C + c] = gx[d];
    }
    const float sgx = Ch.sig[L.kx];
    const float tx = fminf(Ch.mala_tau * sgx * sgx, kMalaTauMax);
    const float dmax = Ch.mala_drift_max;
    double n2 = 0.0;
    for (int d = 0; d < D; ++d) {
        const float m = 0.5f * tx * Ch.G[(size_t)d * C + c];
        n2 += (double)m * m;
    }
    const float scx = n2 > (double)dmax * dmax ? (float)(dmax / sqrt(n2)) : 1.0f;
    const float stx = sqrtf(tx);
    double sf = 0.0;   // |delta - m_x|^2
    float delta[kMaxDim];
    for (int jj = 0; 4 * jj < D; ++jj) {
        const uint4 r = philox(mlo, mhi, Ch.chain0 + (uint32_t)c, 1u + (uint32_t)jj, Ch.seed_lo, Ch.seed_hi);
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const float u1 = ((float)(w[2 * a] >> 8) + 0.5f) * 5.9604644775390625e-08f;
            const float rho = sqrtf(-2.0f * logf(u1));
            float sp, cp;
            sincospif(2.0f * u24(w[2 * a + 1]), &sp, &cp);
            const float z[2] = {rho * cp, rho * sp};
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int d = 4 * jj + 2 * a + e;
                if (d < D) {
                    const uint32_t qx = Ch.q[(size_t)d * Ch.qd + (size_t)c * Ch.qc];
                    const float m = 0.5f * tx * Ch.G[(size_t)d * C + c] * scx;
                    const float step = fmaf(stx, z[e], m);
                    y[d] = qx + (uint32_t)(unsigned long long)__float2ll_rn(step * 4294967296.0f);
                    const float dl = (float)(int32_t)(y[d] - qx) * 2.3283064365386963e-10f;
                    delta[d] = dl;
                    sf += (double)(dl - m) * (double)(dl - m);
                }
            }
        }
    }
    L.mala = 1;
    L.early = 0;
    L.ky = region_y(Ch, y);
    float gy[kMaxDim];
    V3 fy;
    if (S.toy) {
        const float v = toy_grad(S, y[0], y[1], gy);
        fy = {v, v, v};
    } else {
        GradRec rec[RMLT_MAX_DEPTH];
        const int nb = path_forward_rec<BRUTE>(S, s_tris, stack, y, Ch.max_depth, rec, fy, rays);
        if (nb < 0) {
            fy = {0.f, 0.f, 0.f};
            for (int d = 0; d < D; ++d) gy[d] = 0.0f;
        } else {
            path_adjoint(S, y, rec, nb, fy, gy, D);
        }
    }
    L.fy = fy;
    const float sgy = Ch.sig[L.ky];
    const float ty = fminf(Ch.mala_tau * sgy * sgy, kMalaTauMax);
    n2 = 0.0;
    for (int d = 0; d < D; ++d) {
        const float m = 0.5f * ty * gy[d];
        n2 += (double)m * m;
    }
    const float scy = n2 > (double)dmax * dmax ? (float)(dmax / sqrt(n2)) : 1.0f;
    double sb = 0.0;   // |-delta - m_y|^2
    for (int d = 0; d < D; ++d) {
        const double e = -(double)delta[d] - (double)(0.5f * ty * gy[d] * scy);
        sb += e * e;
    }
    const float piy = lum(fy.x, fy.y, fy.z);
    const float ptx = Ch.weighted ? L.pix / Ch.wf[L.kx] : L.pix;
    const float pty = Ch.weighted ? piy / Ch.wf[L.ky] : piy;
    float a;
    if (!(pty > 0.0f) || !isfinite(piy)) {
        a = 0.0f;
    } else if (!(ptx > 0.0f)) {
        a = 1.0f;
    } else {
        const double lr = log((double)pty) - log((double)ptx) - 0.5 * D * log((double)ty / (double)tx) -
                          sb / (2.0 * (double)ty) + sf / (2.0 * (double)tx);
        a = lr >= 0.0 ? 1.0f : (float)exp(lr);
    }
    L.amala = a;
    if (L.xi < a)   // accepted (mutation_finish takes the same decision): keep grad log pi(y)
        for (int d = 0; d < D; ++d) Ch.G[(size_t)d * C + c] = gy[d];
}

// Draw the proposal y of mutation mut0 + j (large or small step, Alg. 1,
// proposal) and decide the reverse-kernel support; returns false when the proposal
// needs no path (rejected early, or the toy integrand evaluated directly).
template <bool MALA = false, bool BRUTE = false, bool D4 = false, class Y>
__device__ __forceinline__ bool mutation_setup(const DevScene& S, const DevChains& Ch, int c, uint64_t mut0,
                                               ChainLane& L, Y y, Path& p, uint32_t* stack = nullptr,
                                               const float4* s_tris = nullptr, unsigned* rays = nullptr)
{
    const int C = Ch.C, D = Ch.D;
    const uint64_t mut = mut0 + (uint64_t)L.j;
    const uint32_t mlo = (uint32_t)mut, mhi = (uint32_t)(mut >> 32);
    const uint4 r0 = philox(mlo, mhi, Ch.chain0 + (uint32_t)c, 0u, Ch.seed_lo, Ch.seed_hi);
    L.large = (r0.x >> 8) < Ch.T_large;
    L.xi = u24(r0.y);
    L.R = 1.0f;
    if (MALA) {
        L.mala = 0;
        if (!L.large && (r0.x >> 8) < Ch.T_large + Ch.T_mala) {
            mala_setup<BRUTE>(S, Ch, c, mlo, mhi, L, y, stack, s_tris, *rays);
            return false;   // path and acceptance are done
        }
    }
    int R = 1;
    if (L.large) {
        for (int jj = 0; 4 * jj < D; ++jj) {
            const uint4 r = philox(mlo, mhi, Ch.chain0 + (uint32_t)c, 1u + (uint32_t)jj, Ch.seed_lo, Ch.seed_hi);
            y[4 * jj] = r.x;
            if (4 * jj + 1 < D) y[4 * jj + 1] = r.y;
            if (4 * jj + 2 < D) y[4 * jj + 2] = r.z;
            if (4 * jj + 3 < D) y[4 * jj + 3] = r.w;
        }
        L.ky = region_y<D4 ? 1 : 0>(Ch, y);
    } else if (Ch.truncnorm) {
        // truncated normal of standard deviation sigma_{k(x)} on (-1/2, 1/2)
        // (the paper's kernel family, Sec. 5.2); the ratio of the reverse and
        // forward densities enters the acceptance
#pragma unroll 4
        for (int d = 0; d < D; ++d) y[d] = Ch.q[(size_t)d * Ch.qd + (size_t)c * Ch.qc];
        const float sx = Ch.sig[L.kx];
        const float zx = erff(0.353553390593273762f / sx);
        double s2 = 0.0;
        for (int jj = 0; 2 * jj < D; ++jj) {
            const uint4 r = philox(mlo, mhi, Ch.chain0 + (uint32_t)c, 1u + (uint32_t)jj, Ch.seed_lo, Ch.seed_hi);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int d = 2 * jj + e;
                if (d < D) {
                    const float u = u24(e ? r.z : r.x);
                    const float x = fmaxf(-0.99999994f, fminf(0.99999994f, (2.0f * u - 1.0f) * zx));
                    const float dl = sx * 1.41421356237309505f * erfinvf(x);
                    const uint32_t off = (uint32_t)(unsigned long long)__float2ll_rn(dl * 4294967296.0f);
                    y[d] += off;
                    const double dr = (double)(int32_t)off * 2.3283064365386963e-10;
                    s2 += dr * dr;
                }
            }
        }
        L.ky = region_y<D4 ? 1 : 0>(Ch, y);
        const float sy = Ch.sig[L.ky];
        if (sy != sx) {
            const float zy = erff(0.353553390593273762f / sy);
            const double lr = D * log(((double)sx * zx) / ((double)sy * zy)) -
                              0.5 * s2 * (1.0 / ((double)sy * sy) - 1.0 / ((double)sx * sx));
            L.R = (float)exp(lr);
        }
    } else {
        // every dimension perturbed with sigma of the current state's region;
        // the current state's words are fetched first with independent loads
#pragma unroll 4
        for (int d = 0; d < D; ++d) y[d] = Ch.q[(size_t)d * Ch.qd + (size_t)c * Ch.qc];
        const float sx = Ch.sig[L.kx];
        const float sigS2 = __fmul_rn(sx, Ch.S2);
        float lo = 0.f, hi = 0.f;
        bool check = false;
        for (int jj = 0; 2 * jj < D; ++jj) {
            const uint4 r = philox(mlo, mhi, Ch.chain0 + (uint32_t)c, 1u + (uint32_t)jj, Ch.seed_lo, Ch.seed_hi);
            const int d0 = 2 * jj;
            const uint32_t o0 = kelemen_offset(r.x, sigS2, Ch.log2_ratio);
            y[d0] = (r.y >> 31) ? y[d0] - o0 : y[d0] + o0;
            uint32_t o1 = 0;
            if (d0 + 1 < D) {
                o1 = kelemen_offset(r.z, sigS2, Ch.log2_ratio);
                y[d0 + 1] = (r.w >> 31) ? y[d0 + 1] - o1 : y[d0 + 1] + o1;
            }
            if (jj == 0 && !D4) {
                L.ky = region_of(Ch, y[0], y[1]);
                const float sy = Ch.sig[L.ky];
                if (sy != sx) {
                    // reverse kernel T_{k(y)}(x|y): every offset inside [sigma_y s1, sigma_y s2]
                    check = true;
                    lo = __fmul_rn(sy, Ch.S1);
                    hi = __fmul_rn(sy, Ch.S2);
                }
            }
            if (check) {
                const float m0 = __uint2float_rn(o0);
                if (!(m0 >= lo && m0 <= hi)) R = 0;
                if (d0 + 1 < D) {
                    const float m1 = __uint2float_rn(o1);
                    if (!(m1 >= lo && m1 <= hi)) R = 0;
                }
            }
        }
        if (D4) {
            // the 4-D region needs dims 5 and 6: the reverse-kernel support is
            // checked afterwards on the offset magnitudes y - x
            L.ky = region_y<D4 ? 1 : 0>(Ch, y);
            const float sy = Ch.sig[L.ky];
            if (sy != sx) {
                lo = __fmul_rn(sy, Ch.S1);
                hi = __fmul_rn(sy, Ch.S2);
                for (int d = 0; d < D; ++d) {
                    const uint32_t dd = y[d] - Ch.q[(size_t)d * Ch.qd + (size_t)c * Ch.qc];
                    const float m = __uint2float_rn(dd < 0x80000000u ? dd : 0u - dd);
                    if (!(m >= lo && m <= hi)) R = 0;
                }
            }
        }
    }
    L.early = !R;
    L.fy = {0.f, 0.f, 0.f};
    if (!R) return false;
    if (S.toy) {
        const float v = toy_eval(S, y[0], y[1]);
        L.fy = {v, v, v};
        return false;
    }
    if (L.large && Ch.lf) {
        // independent of the chain's state: traced ahead of the epoch
        const size_t o = (size_t)L.j * C + c;
        L.fy = {Ch.lf[o], Ch.lf[(size_t)Ch.E * C + o], Ch.lf[(size_t)2 * Ch.E * C + o]};
        return false;
    }
    path_begin(p, S, y);
    return true;
}

__device__ __forceinline__ void flush_state(const DevChains& Ch, ChainLane& L)
{
    if (L.pend_n) {
        atomicAdd(&Ch.hist[L.kx], (unsigned long long)L.pend_n);
        if (L.pix > 0.0f) {
            double* dst = Ch.img + 3 * ((size_t)L.py * Ch.W + L.px);
            const double s = (double)L.pend_n / (double)L.pix;
            atomicAdd(dst + 0, s * L.fx.x);
            atomicAdd(dst + 1, s * L.fx.y);
            atomicAdd(dst + 2, s * L.fx.z);
        }
    }
    if (L.pend_i) {
        atomicAdd(&Ch.vis[L.kx], L.pend_i);
        atomicAdd(&Ch.acc[L.kx], L.pend_A);
    }
    L.pend_n = 0;
    L.pend_i = L.pend_A = 0;
}

// acceptance (Sec. 3.2 with the mixture of Sec. 5.2), adaptation statistics
// of the current region (Alg. 1, acceptance statistics), MH update (Alg. 1, state update), splat
template <bool TRACE, bool MALA = false, class Y>
__device__ __forceinline__ void mutation_finish(const DevChains& Ch, int c, bool traced, ChainLane& L,
                                                Y y, unsigned (&st)[7])
{
    const int D = Ch.D;
    V3 fy = L.fy;
    float piy = lum(fy.x, fy.y, fy.z);
    int invalid = 0;
    if (!isfinite(piy)) {
        fy = {0.f, 0.f, 0.f};
        piy = 0.f;
        invalid = 1;
        ++st[4];
    }
    float a;
    if (MALA && L.mala) {
        a = L.amala;   // decided with the proposal densities (mala_setup)
    } else if (L.early) {
        a = 0.0f;
    } else {
        const float ptx = Ch.weighted ? L.pix / Ch.wf[L.kx] : L.pix;
        const float pty = Ch.weighted ? piy / Ch.wf[L.ky] : piy;
        a = !(ptx > 0.0f) ? 1.0f : fminf(1.0f, L.R == 1.0f ? pty / ptx : pty / ptx * L.R);
    }
    const int accept = L.xi < a;
    if (MALA && L.mala) {
        // Langevin moves do not feed the adaptation statistics of Alg. 1,
        // which tune the small step
        ++L.n_mala;
        L.n_mala_acc += (unsigned)accept;
    } else if (MALA && accept) {
        Ch.G[c] = __int_as_float(0x7FC00000);   // the new state's gradient is computed when needed
    }
    if (MALA && L.mala) {
    } else if (L.large) {
        ++st[1];
        if (!Ch.lf) atomicAdd(&Ch.Bk[L.ky], (double)piy);   // else added by the large-step kernel
    } else {
        ++st[2];
        L.pend_i += 1;
        L.pend_A += (unsigned long long)__float2ull_rn(a * 4294967296.0f);
    }
    st[3] += L.early;
    if (TRACE && traced) {
        const unsigned long long idx = Ch.trace_base + (unsigned long long)(c / Ch.trace_stride) * Ch.E + L.j;
        if (idx < Ch.trace_cap) {
            uint32_t hsh = 2166136261u;
            for (int d = 0; d < D; ++d) hsh = (hsh ^ y[d]) * 16777619u;
            rmlt_trace_record r;
            r.f[0] = fy.x;
            r.f[1] = fy.y;
            r.f[2] = fy.z;
            r.a = a;
            r.qhash = hsh;
            r.flags = (uint32_t)accept | ((uint32_t)L.large << 1) | ((uint32_t)L.early << 2) | ((uint32_t)invalid << 3) |
                      ((uint32_t)(MALA && L.mala) << 4);
            Ch.trace[idx] = r;
            if (Ch.trace_words)
                for (int d = 0; d < D; ++d) Ch.trace_words[idx * (unsigned long long)D + d] = y[d];
        }
    }
    if (accept) {
        flush_state(Ch, L);      // visits, splats and statistics of the state being left
        // eight loads before their stores, so that the copy does not wait on
        // one load at a time when y lives in global memory
        for (int d0 = 0; d0 < D; d0 += 8) {
            uint32_t t[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) t[k] = d0 + k < D ? y[d0 + k] : 0u;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (d0 + k < D) Ch.q[(size_t)(d0 + k) * Ch.qd + (size_t)c * Ch.qc] = t[k];
        }
        L.fx = fy;
        L.pix = piy;
        L.kx = L.ky;
        L.px = pixel_x(y[0], Ch.W);
        L.py = pixel_x(y[1], Ch.H);
        ++st[0];
    }
    L.pend_n += 1;
}

}  // namespace
}  // namespace rmlt

// CUDA kernels of librmlt (sm_103a): the regional adaptive PSS-MLT chain step.
//
// One thread owns one chain for an epoch of E mutations (Alg. 1 lines 8-19).
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

__device__ __forceinline__ float lum(float r, float g, float b) { return 0.2126f * r + 0.7152f * g + 0.0722f * b; }

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

// ---------------------------------------------------------------------------
// small float3 helpers
// ---------------------------------------------------------------------------
struct V3 { float x, y, z; };
__device__ __forceinline__ V3 v3(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(V3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
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
};

__device__ __forceinline__ void trav_begin(Trav& T, V3 o, V3 d, float tmax, int any)
{
    T.o = o;
    T.d = d;
    T.id = {1.0f / (fabsf(d.x) > 1e-12f ? d.x : copysignf(1e-12f, d.x)),
            1.0f / (fabsf(d.y) > 1e-12f ? d.y : copysignf(1e-12f, d.y)),
            1.0f / (fabsf(d.z) > 1e-12f ? d.z : copysignf(1e-12f, d.z))};
    T.ood = {o.x * T.id.x, o.y * T.id.y, o.z * T.id.z};
    T.t = tmax;
    T.tri = -1;
    T.ref = 0;
    T.sp = 0;
    T.any = any;
    T.overflow = 0;
}

// one step; returns true once the ray is resolved
template <bool BRUTE>
__device__ __forceinline__ bool trav_step(Trav& T, uint32_t* stack, const DevScene& S, const float4* s_tris,
                                          unsigned& n_nodes, unsigned& n_tris)
{
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
    if (!(ref & kLeafBit) && S.bvh4) {
        // four children: slab tests in the lanes of each float4, nearest hit
        // child next, the others pushed far to near
        ++n_nodes;
        const float4* nd = &S.nodes[8 * (size_t)ref];
        const float4 lx = __ldg(nd + 0), hx = __ldg(nd + 1), ly = __ldg(nd + 2), hy = __ldg(nd + 3);
        const float4 lz = __ldg(nd + 4), hz = __ldg(nd + 5), rf = __ldg(nd + 6);
        const float tcap = T.t * 1.00000036f;
        const V3 id = T.id, ood = T.ood;
        float key[4];
        uint32_t cr[4];
        const float lox[4] = {lx.x, lx.y, lx.z, lx.w}, hix[4] = {hx.x, hx.y, hx.z, hx.w};
        const float loy[4] = {ly.x, ly.y, ly.z, ly.w}, hiy[4] = {hy.x, hy.y, hy.z, hy.w};
        const float loz[4] = {lz.x, lz.y, lz.z, lz.w}, hiz[4] = {hz.x, hz.y, hz.z, hz.w};
        const uint32_t rr[4] = {__float_as_uint(rf.x), __float_as_uint(rf.y), __float_as_uint(rf.z),
                                __float_as_uint(rf.w)};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float a0 = fmaf(lox[k], id.x, -ood.x), b0 = fmaf(hix[k], id.x, -ood.x);
            const float a1 = fmaf(loy[k], id.y, -ood.y), b1 = fmaf(hiy[k], id.y, -ood.y);
            const float a2 = fmaf(loz[k], id.z, -ood.z), b2 = fmaf(hiz[k], id.z, -ood.z);
            const float tn = fmaxf(fmaxf(fminf(a0, b0), fminf(a1, b1)), fmaxf(fminf(a2, b2), 0.0f));
            const float tf = fminf(fminf(fmaxf(a0, b0), fmaxf(a1, b1)), fminf(fmaxf(a2, b2), tcap));
            const bool hit = tn <= tf && rr[k] != kEmptyRef;
            key[k] = hit ? tn : INFINITY;
            cr[k] = rr[k];
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
                if (T.sp < kStackSize) stack[kChainBlock * T.sp++] = cr[k];
                else T.overflow = 1;
            }
        }

        next = key[0] != INFINITY ? cr[0] : (T.sp > 0 ? stack[kChainBlock * --T.sp] : kNoRef);
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
            if (T.sp < kStackSize) stack[kChainBlock * T.sp++] = first0 ? c1 : c0;
            else T.overflow = 1;
            next = first0 ? c0 : c1;
        } else if (h0) {
            next = c0;
        } else if (h1) {
            next = c1;
        } else {
            next = T.sp > 0 ? stack[kChainBlock * --T.sp] : kNoRef;
        }
    } else {
        const uint32_t first = ref & 0x0FFFFFFFu, cnt = ((ref >> 28) & 7u) + 1u;
        bool found = false;
        for (uint32_t i = first; i < first + cnt; ++i) {
            ++n_tris;
            float t;
            const float4 a = __ldg(&S.tris[3 * i]), b = __ldg(&S.tris[3 * i + 1]), c = __ldg(&S.tris[3 * i + 2]);
            if (hit_tri(T.o, T.d, a, b, c, T.t, t)) {
                T.t = t;
                T.tri = (int)i;
                T.ta = a;
                T.tb = b;
                T.tc = c;
                found = true;
            }
        }
        next = (T.any && found) ? kNoRef : (T.sp > 0 ? stack[kChainBlock * --T.sp] : kNoRef);
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

__device__ __forceinline__ void path_begin(Path& p, const DevScene& S, const uint32_t* y)
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
__device__ __forceinline__ void path_continue(Path& p, const DevScene& S, const uint32_t* y, int max_depth)
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

// consume the result of the pending ray
template <bool BRUTE>
__device__ __forceinline__ void path_on_hit(Path& p, const DevScene& S, const float4* s_tris, const uint32_t* y,
                                            int max_depth, Hit h)
{
    if (p.any) {
        if (h.tri < 0) p.L = p.L + p.P;
        p.any = 0;
        path_continue(p, S, y, max_depth);
        return;
    }
    if (h.tri < 0) { p.done = 1; return; }
    const float4 ta = h.a, tb = h.b, tc = h.c;
    const V3 n = normalize(cross(xyz(tb), xyz(tc)));
    const int mat = __float_as_int(ta.w);
    const V3 x = p.o + p.d * h.t;
    const float cosi = -dot(n, p.d);
    const V3 ns = cosi > 0.0f ? n : n * -1.0f;
    const float4 m0 = __ldg(&S.mats[3 * mat]), m1 = __ldg(&S.mats[3 * mat + 1]), m2 = __ldg(&S.mats[3 * mat + 2]);
    if (p.b == 0 && m2.x != 0.0f && cosi > 0.0f) p.L = p.L + v3(p.T.x * m1.x, p.T.y * m1.y, p.T.z * m1.z);
    if (m2.y != 0.0f) { p.done = 1; return; }
    p.x = x;
    p.ns = ns;
    p.wo = p.d * -1.0f;
    p.mat = mat;
    if (S.n_lights > 0) {
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
        if (cx > 0.0f && cl > 0.0f) {
            const V3 xo = x + ns * S.eps;
            V3 sd = pl - xo;
            const float sdist = sqrtf(dot(sd, sd));
            if (sdist > 2.0f * S.eps) {
                const V3 fr = bsdf_eval(m0, m1, p.wo, wi, ns);
                const float4 lm1 = __ldg(&S.mats[3 * __float_as_int(la.w) + 1]);
                const float g = cx * cl / dist2 * S.light_area;
                p.P = {p.T.x * fr.x * lm1.x * g, p.T.y * fr.y * lm1.y * g, p.T.z * fr.z * lm1.z * g};
                p.o = xo;
                p.d = sd * (1.0f / sdist);
                p.tmax = sdist - S.eps;
                p.any = 1;
                return;
            }
        }
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
// the chain step: E mutations per chain (Alg. 1 lines 8-19)
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
    V3 fy;
};

// Draw the proposal y of mutation mut0 + j (large or small step, Alg. 1 line
// 10) and decide the reverse-kernel support; returns false when the proposal
// needs no path (rejected early, or the toy integrand evaluated directly).
__device__ __forceinline__ bool mutation_setup(const DevScene& S, const DevChains& Ch, int c, uint64_t mut0,
                                               ChainLane& L, uint32_t* y, Path& p)
{
    const int C = Ch.C, D = Ch.D;
    const uint64_t mut = mut0 + (uint64_t)L.j;
    const uint32_t mlo = (uint32_t)mut, mhi = (uint32_t)(mut >> 32);
    const uint4 r0 = philox(mlo, mhi, (uint32_t)c, 0u, Ch.seed_lo, Ch.seed_hi);
    L.large = (r0.x >> 8) < Ch.T_large;
    L.xi = u24(r0.y);
    int R = 1;
    if (L.large) {
        for (int jj = 0; 4 * jj < D; ++jj) {
            const uint4 r = philox(mlo, mhi, (uint32_t)c, 1u + (uint32_t)jj, Ch.seed_lo, Ch.seed_hi);
            y[4 * jj] = r.x;
            if (4 * jj + 1 < D) y[4 * jj + 1] = r.y;
            if (4 * jj + 2 < D) y[4 * jj + 2] = r.z;
            if (4 * jj + 3 < D) y[4 * jj + 3] = r.w;
        }
        L.ky = region_of(Ch, y[0], y[1]);
    } else {
        // every dimension perturbed with sigma of the current state's region;
        // the current state's words are fetched first with independent loads
#pragma unroll 4
        for (int d = 0; d < D; ++d) y[d] = Ch.q[(size_t)d * C + c];
        const float sx = Ch.sig[L.kx];
        const float sigS2 = __fmul_rn(sx, Ch.S2);
        float lo = 0.f, hi = 0.f;
        bool check = false;
        for (int jj = 0; 2 * jj < D; ++jj) {
            const uint4 r = philox(mlo, mhi, (uint32_t)c, 1u + (uint32_t)jj, Ch.seed_lo, Ch.seed_hi);
            const int d0 = 2 * jj;
            const uint32_t o0 = kelemen_offset(r.x, sigS2, Ch.log2_ratio);
            y[d0] = (r.y >> 31) ? y[d0] - o0 : y[d0] + o0;
            uint32_t o1 = 0;
            if (d0 + 1 < D) {
                o1 = kelemen_offset(r.z, sigS2, Ch.log2_ratio);
                y[d0 + 1] = (r.w >> 31) ? y[d0 + 1] - o1 : y[d0 + 1] + o1;
            }
            if (jj == 0) {
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
// of the current region (Alg. 1 lines 11-12), MH update (line 19), splat
template <bool TRACE>
__device__ __forceinline__ void mutation_finish(const DevChains& Ch, int c, bool traced, ChainLane& L,
                                                const uint32_t* y, unsigned (&st)[7])
{
    const int C = Ch.C, D = Ch.D;
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
    if (L.early) {
        a = 0.0f;
    } else {
        const float ptx = Ch.weighted ? L.pix / Ch.wf[L.kx] : L.pix;
        const float pty = Ch.weighted ? piy / Ch.wf[L.ky] : piy;
        a = !(ptx > 0.0f) ? 1.0f : fminf(1.0f, pty / ptx);
    }
    const int accept = L.xi < a;
    if (L.large) {
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
            r.flags = (uint32_t)accept | ((uint32_t)L.large << 1) | ((uint32_t)L.early << 2) | ((uint32_t)invalid << 3);
            Ch.trace[idx] = r;
        }
    }
    if (accept) {
        flush_state(Ch, L);      // visits, splats and statistics of the state being left
        for (int d = 0; d < D; ++d) Ch.q[(size_t)d * C + c] = y[d];
        L.fx = fy;
        L.pix = piy;
        L.kx = L.ky;
        L.px = pixel_x(y[0], Ch.W);
        L.py = pixel_x(y[1], Ch.H);
        ++st[0];
    }
    L.pend_n += 1;
}

// One thread per chain; the unit of work is one traversal step.  Every loop
// iteration advances each lane with a live ray by one BVH node or leaf.  A
// lane whose ray is resolved waits until at least `batch_shade` lanes (or
// every lane with work) are waiting, then the waiting lanes shade together
// (path_on_hit: emission, next-event sample, BSDF sample -> the next ray).
// Lanes whose path ended finish their mutation and draw the next proposal in
// batches of `batch_setup` the same way.  The batches keep the expensive,
// divergent parts convergent while the traversal keeps every lane busy.
enum LanePhase { kIdle = 0, kTraverse = 1, kShade = 2, kFinish = 3, kSetup = 4 };

template <bool BRUTE, bool TRACE, bool COUNT>
__global__ void __launch_bounds__(kChainBlock) chain_epoch_kernel(const DevScene S, const DevChains Ch, uint64_t mut0)
{
    extern __shared__ float4 s_tris[];
    if (BRUTE) stage_triangles(S, s_tris);
    const unsigned FULL = 0xFFFFFFFFu;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
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
    L.fy = {0.f, 0.f, 0.f};
    const bool traced = TRACE && valid && (uint32_t)c % Ch.trace_stride == 0u;
    uint32_t y[kMaxDim];
    // traversal stack in shared memory, one column per thread (conflict-free)
    __shared__ uint32_t s_stack[kStackSize * kChainBlock];
    uint32_t* stack = s_stack + threadIdx.x;
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
        __syncwarp();
        if (phase == kTraverse) {
            if (trav_step<BRUTE>(T, stack, S, s_tris, n_nodes, n_tris)) phase = kShade;
        }
        if (COUNT) {
            __syncwarp();
            const long long t = clock64();
            cyc[0] += t - t_mark;
            t_mark = t;
        }
        const unsigned m_tr = __ballot_sync(FULL, phase == kTraverse);
        const unsigned m_sh = __ballot_sync(FULL, phase == kShade);
        // fewer lanes at work (the end of the epoch): optionally smaller batches
        int bs_eff = bs, bf_eff = bf;
        if (Ch.adaptive_batch) {
            const int busy = __popc(__ballot_sync(FULL, phase != kIdle));
            bs_eff = min(bs, (busy + 3) >> 2);
            bf_eff = min(bf, (busy + 3) >> 2);
        }
        if (COUNT) {
            sched[0] += 1;
            sched[1] += __popc(m_tr);
        }
        if (m_sh && (__popc(m_sh) >= bs_eff || !m_tr)) {
            if (COUNT) {
                sched[2] += 1;
                sched[3] += __popc(m_sh);
            }
            if (phase == kShade) {
                ++st[5];
                if (T.overflow) {
                    ++st[6];
                    p.done = 1;
                    p.L = {0.f, 0.f, 0.f};
                } else {
                    path_on_hit<BRUTE>(p, S, s_tris, y, Ch.max_depth, Hit{T.t, T.tri, T.ta, T.tb, T.tc});
                }
                if (p.done) {
                    L.fy = p.L;
                    phase = kFinish;
                } else {
                    trav_begin(T, p.o, p.d, p.tmax, p.any);
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
                    mutation_finish<TRACE>(Ch, c, traced, L, y, st);
                    ++L.j;
                    phase = L.j < Ch.E ? kSetup : kIdle;
                }
                if (phase == kSetup) {
                    if (mutation_setup(S, Ch, c, mut0, L, y, p)) {
                        trav_begin(T, p.o, p.d, p.tmax, p.any);
                        phase = kTraverse;
                    } else {
                        phase = kFinish;
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
    if (COUNT && lane == 0) {
        for (int s = 0; s < 6; ++s) atomicAdd(&Ch.stats[kStIters + s], sched[s]);
        for (int s = 0; s < 3; ++s) atomicAdd(&Ch.stats[kStCycTrav + s], cyc[s]);
        const unsigned long long life = (unsigned long long)(clock64() - t_start);
        atomicAdd(&Ch.stats[kStCycLife], life);
        atomicMax(&Ch.stats[kStCycLifeMax], life);
    }
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
        const uint4 r0 = philox((uint32_t)mut, (uint32_t)(mut >> 32), (uint32_t)c, 0u, Ch.seed_lo, Ch.seed_hi);
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
        const uint4 r = philox(mlo, mhi, (uint32_t)c, 1u + (uint32_t)jj, Ch.seed_lo, Ch.seed_hi);
        y[4 * jj] = r.x;
        if (4 * jj + 1 < D) y[4 * jj + 1] = r.y;
        if (4 * jj + 2 < D) y[4 * jj + 2] = r.z;
        if (4 * jj + 3 < D) y[4 * jj + 3] = r.w;
    }
    Path p;
    Trav T;
    uint32_t* stack = s_stack + threadIdx.x;
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
    const int ky = region_of(Ch, y[0], y[1]);
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
// region update at the epoch boundary (Alg. 1 lines 13-18; eqs.
// est_exp_acc, update_lambda, step_size_n), binary64 with explicit rounding
// ---------------------------------------------------------------------------
__global__ void region_update_kernel(const DevChains Ch, int init_only)
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
    Ch.k[c] = region_of(Ch, Ch.q[c], Ch.q[(size_t)Ch.C + c]);
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
// initial states (stratified inverse CDF of pi)
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
    if (S.toy) {
        const float v = toy_eval(S, y[0], y[1]);
        f = {v, v, v};
    } else {
        Path p;
        Trav T;
        uint32_t* stack = s_stack + threadIdx.x;
        path_begin(p, S, y);
        while (!p.done) {
            trav_begin(T, p.o, p.d, p.tmax, p.any);
            while (!trav_step<BRUTE>(T, stack, S, s_tris, nn, nt)) {
            }
            if (T.overflow) { p.L = {0.f, 0.f, 0.f}; break; }
            path_on_hit<BRUTE>(p, S, s_tris, y, Ch.max_depth, Hit{T.t, T.tri, T.ta, T.tb, T.tc});
        }
        f = p.L;
    }
    float pv = lum(f.x, f.y, f.z);
    if (!isfinite(pv)) { f = {0.f, 0.f, 0.f}; pv = 0.f; }
    B.pi[s] = pv;
    B.f[s] = f.x;
    B.f[n_boot + s] = f.y;
    B.f[2 * n_boot + s] = f.z;
    const int k = region_of(Ch, y[0], y[1]);
    if (pv != 0.f) atomicAdd(&Ch.Bk[k], (double)pv);
}

// Initial state of chain c: weighted reservoir sampling over its own K
// uniform samples s in [cK, (c+1)K): keep s when v_s cum_s < pi_s, which picks
// s with probability pi_s / sum(pi) (v_s a uniform of its own).  The slice sum
// goes to `partial` for the normaliser b.
__global__ void bootstrap_select_kernel(const DevChains Ch, long long K, const BootScratch B)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= Ch.C) return;
    const long long n_eff = K * Ch.C;
    double cum = 0.0;
    long long sel = -1;
    for (long long i = 0; i < K; ++i) {
        const long long s = (long long)c * K + i;
        const double v = (double)B.pi[s];
        cum += v;
        const uint4 r = philox((uint32_t)s, (uint32_t)((unsigned long long)s >> 32), 0xFFFFFFFFu, 0x7FFFu,
                               Ch.seed_lo, Ch.seed_hi);
        if (v > 0.0 && (double)u24(r.x) * cum < v) sel = s;
    }
    if (sel < 0) sel = (long long)c * K;
    B.partial[c] = cum;
    const int D = Ch.D, C = Ch.C;
    uint32_t q0 = 0, q1 = 0;
    for (int jj = 0; 4 * jj < D; ++jj) {
        const uint4 r = philox((uint32_t)sel, (uint32_t)((unsigned long long)sel >> 32), 0xFFFFFFFFu,
                               0x8000u + (uint32_t)jj, Ch.seed_lo, Ch.seed_hi);
        const uint32_t v[4] = {r.x, r.y, r.z, r.w};
        for (int a = 0; a < 4 && 4 * jj + a < D; ++a) Ch.q[(size_t)(4 * jj + a) * C + c] = v[a];
        if (jj == 0) { q0 = r.x; q1 = r.y; }
    }
    Ch.f[c] = B.f[sel];
    Ch.f[C + c] = B.f[n_eff + sel];
    Ch.f[2 * C + c] = B.f[2 * n_eff + sel];
    Ch.pi[c] = B.pi[sel];
    Ch.k[c] = region_of(Ch, q0, q1);
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
                const double nU = (double)n_boot + (double)Ch.stats[kStLarge];
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
    const int blocks = (c.C + kChainBlock - 1) / kChainBlock;
    const size_t shm = B ? sizeof(float4) * 3 * (size_t)s.n_tris : 0;
    auto kern = chain_epoch_kernel<B, T, K>;
    if (shm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        if (e != cudaSuccess) return e;
    }
    kern<<<blocks, kChainBlock, shm, st>>>(s, c, mut0);
    return cudaGetLastError();
}

cudaError_t launch_chain_epoch(const DevScene& s, const DevChains& c, uint64_t mut0, bool trace, bool count_work,
                               cudaStream_t st)
{
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

cudaError_t launch_bootstrap(const DevScene& s, const DevChains& c, int64_t n_boot, const BootScratch& b,
                             cudaStream_t st)
{
    const long long K = n_boot / c.C;
    const long long n_eff = K * c.C;
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
    bootstrap_select_kernel<<<(c.C + 127) / 128, 128, 0, st>>>(c, K, b);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    bootstrap_total_kernel<<<1, 256, 0, st>>>(c.C, b);
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
constexpr size_t kNaTotal = na_align(kNaPartial + sizeof(double) * RMLT_NOALLOC_MAX_CHAINS);
constexpr size_t kNaChainPi = na_align(kNaTotal + sizeof(double));
constexpr size_t kNaChainK = na_align(kNaChainPi + sizeof(float) * RMLT_NOALLOC_MAX_CHAINS);
constexpr size_t kNaBk = na_align(kNaChainK + sizeof(int32_t) * RMLT_NOALLOC_MAX_CHAINS);
constexpr size_t kNaBytes = na_align(kNaBk + sizeof(double) * RMLT_NOALLOC_MAX_REGIONS);

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
    out.boot.total = (double*)(base + kNaTotal);
    out.chain_pi = (float*)(base + kNaChainPi);
    out.chain_k = (int32_t*)(base + kNaChainK);
    out.Bk = (double*)(base + kNaBk);
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

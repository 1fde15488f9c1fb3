// Host-side binned SAH builder for the BVH the chain kernel traverses.
//
// A binary tree is built with binned SAH (32 bins per axis, leaves of at most
// 2 triangles: with leaf turns and two triangle loads per pass, a leaf costs
// about what a node does, and smaller leaves measured faster than 4 or 8) and
// emitted either as BVH2 or, collapsed, as BVH4.  In both
// layouts an internal node stores its children's boxes, so one node fetch
// tests all children.
//
// BVH2 (4 float4 per node):
//   n0 = (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y)
//   n1 = (c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y)
//   n2 = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)
//   n3 = (ref c0, ref c1, 0, 0)                      (uint bits)
// BVH4 (8 float4 per node, children in the four lanes of each float4):
//   lo.x, hi.x, lo.y, hi.y, lo.z, hi.z, refs (uint bits), unused
// or, quantised, BVH4Q (4 float4 per node, the children's boxes as 8-bit
// indices on a per-node grid):
//   n0 = (p.x, p.y, p.z, s.x)
//   n1 = (s.y, s.z, qlo.z, qhi.z)                    (q words as uint bits)
//   n2 = (qlo.x, qhi.x, qlo.y, qhi.y)
//   n3 = (ref c0, ref c1, ref c2, ref c3)            (uint bits)
// Byte k of a q word belongs to child k; child k's box on axis a is
// [p.a + qlo.a[k] s.a, p.a + qhi.a[k] s.a] in exact arithmetic.  p is the
// lower corner of the union of the children's boxes and s.a = its extent on
// axis a / 255, rounded up, so every grid value lies in the node; lo planes
// are rounded down and hi planes up, so each decoded box contains the
// child's box.
// A ref is an internal node index, a leaf (kLeafBit | (count-1) << 28 |
// first triangle in build order), or, for an unused BVH4 slot, empty_ref(n):
// a one-triangle leaf past the scene's triangles (the upload's zero-area
// sentinel), with an inverted box no slab test accepts (BVH4: lo = +inf,
// hi = -inf; BVH4Q: q bytes 255 / 0).
// Boxes are widened by `pad` and rounded outward so that binary32 traversal
// never culls a box a ray grazes.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rmlt_internal.h"

namespace rmlt {
namespace {

struct Box {
    float lo[3], hi[3];
    void reset()
    {
        for (int a = 0; a < 3; ++a) { lo[a] = INFINITY; hi[a] = -INFINITY; }
    }
    void grow(const Box& b)
    {
        for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], b.lo[a]); hi[a] = std::max(hi[a], b.hi[a]); }
    }
    float area() const
    {
        const float dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        if (!(dx >= 0.f)) return 0.f;
        return 2.f * (dx * dy + dy * dz + dz * dx);
    }
};

struct Prim {
    Box b;
    float c[3];
    uint32_t id;
};

struct BNode {
    Box box;
    int left = -1, right = -1;   // internal iff left >= 0
    int first = 0, count = 0;
};

constexpr int kBins = 32;
constexpr int kLeafMax = 2;

uint32_t fbits(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
}
float bitsf(uint32_t u)
{
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

struct Builder {
    std::vector<Prim>& prims;
    std::vector<BNode> nodes;
    int max_depth = 0;

    int build(int b, int e, int depth)
    {
        max_depth = std::max(max_depth, depth);
        const int id = (int)nodes.size();
        nodes.emplace_back();
        Box box, cb;
        box.reset();
        cb.reset();
        for (int i = b; i < e; ++i) {
            box.grow(prims[i].b);
            for (int a = 0; a < 3; ++a) {
                cb.lo[a] = std::min(cb.lo[a], prims[i].c[a]);
                cb.hi[a] = std::max(cb.hi[a], prims[i].c[a]);
            }
        }
        nodes[id].box = box;
        const int n = e - b;
        if (n <= kLeafMax) {
            nodes[id].first = b;
            nodes[id].count = n;
            return id;
        }
        float best = INFINITY;
        int best_axis = -1, best_split = -1;
        for (int a = 0; a < 3; ++a) {
            const float ext = cb.hi[a] - cb.lo[a];
            if (!(ext > 0.f)) continue;
            int cnt[kBins] = {0};
            Box bb[kBins];
            for (auto& x : bb) x.reset();
            const float k = kBins / ext;
            for (int i = b; i < e; ++i) {
                int bi = (int)((prims[i].c[a] - cb.lo[a]) * k);
                bi = std::min(kBins - 1, std::max(0, bi));
                cnt[bi]++;
                bb[bi].grow(prims[i].b);
            }
            float rarea[kBins];
            int rcnt[kBins];
            Box acc;
            acc.reset();
            int c = 0;
            for (int i = kBins - 1; i > 0; --i) {
                acc.grow(bb[i]);
                c += cnt[i];
                rarea[i] = acc.area();
                rcnt[i] = c;
            }
            acc.reset();
            c = 0;
            for (int i = 0; i < kBins - 1; ++i) {
                acc.grow(bb[i]);
                c += cnt[i];
                if (c == 0 || rcnt[i + 1] == 0) continue;
                const float cost = acc.area() * c + rarea[i + 1] * rcnt[i + 1];
                if (cost < best) { best = cost; best_axis = a; best_split = i; }
            }
        }
        int mid;
        if (best_axis < 0) {
            mid = b + n / 2;   // coincident centroids: split by count
        } else {
            const float ext = cb.hi[best_axis] - cb.lo[best_axis];
            const float k = kBins / ext;
            auto it = std::partition(prims.begin() + b, prims.begin() + e, [&](const Prim& p) {
                int bi = (int)((p.c[best_axis] - cb.lo[best_axis]) * k);
                bi = std::min(kBins - 1, std::max(0, bi));
                return bi <= best_split;
            });
            mid = (int)(it - prims.begin());
            if (mid == b || mid == e) mid = b + n / 2;
        }
        const int l = build(b, mid, depth + 1);
        const int r = build(mid, e, depth + 1);
        nodes[id].left = l;
        nodes[id].right = r;
        return id;
    }
};

struct Emitter {
    const std::vector<BNode>& bn;
    std::vector<float4>& out;
    float pad;
    uint32_t empty;   // the reference of an unused BVH4 slot
    bool quant;       // BVH4Q nodes
    int depth = 0, max_depth = 0;

    Box padded(const Box& b) const
    {
        Box o;
        for (int a = 0; a < 3; ++a) {
            o.lo[a] = std::nextafter(b.lo[a] - pad, -INFINITY);
            o.hi[a] = std::nextafter(b.hi[a] + pad, INFINITY);
        }
        return o;
    }
    uint32_t leaf_ref(const BNode& n) const { return kLeafBit | ((uint32_t)(n.count - 1) << 28) | (uint32_t)n.first; }

    uint32_t emit2(int i)
    {
        const BNode& n = bn[(size_t)i];
        if (n.left < 0) return leaf_ref(n);
        const uint32_t id = (uint32_t)(out.size() / 4);
        out.resize(out.size() + 4);
        const uint32_t l = emit2(n.left);
        const uint32_t r = emit2(n.right);
        const Box L = padded(bn[(size_t)n.left].box), R = padded(bn[(size_t)n.right].box);
        float4* nd = &out[4 * (size_t)id];
        nd[0] = make_float4(L.lo[0], L.hi[0], L.lo[1], L.hi[1]);
        nd[1] = make_float4(R.lo[0], R.hi[0], R.lo[1], R.hi[1]);
        nd[2] = make_float4(L.lo[2], L.hi[2], R.lo[2], R.hi[2]);
        nd[3] = make_float4(bitsf(l), bitsf(r), 0.f, 0.f);
        return id;
    }

    // collapse: open the child with the largest surface until 4 children
    uint32_t emit4(int i)
    {
        const BNode& n = bn[(size_t)i];
        if (n.left < 0) return leaf_ref(n);
        max_depth = std::max(max_depth, ++depth);
        int ch[4] = {n.left, n.right, -1, -1};
        int nc = 2;
        while (nc < 4) {
            int pick = -1;
            float area = -1.f;
            for (int k = 0; k < nc; ++k) {
                const BNode& c = bn[(size_t)ch[k]];
                if (c.left >= 0 && c.box.area() > area) { area = c.box.area(); pick = k; }
            }
            if (pick < 0) break;
            const BNode& c = bn[(size_t)ch[pick]];
            ch[pick] = c.left;
            ch[nc++] = c.right;
        }
        const size_t words = quant ? 4 : 8;
        const uint32_t id = (uint32_t)(out.size() / words);
        out.resize(out.size() + words);
        uint32_t refs[4] = {empty, empty, empty, empty};
        Box boxes[4];
        for (int k = 0; k < 4; ++k) {
            // an unused slot's inverted infinite box: every slab test rejects it
            for (int a = 0; a < 3; ++a) { boxes[k].lo[a] = INFINITY; boxes[k].hi[a] = -INFINITY; }
            if (k < nc) {
                refs[k] = emit4(ch[k]);
                boxes[k] = padded(bn[(size_t)ch[k]].box);
            }
        }
        if (!quant) {
            float4* nd = &out[8 * (size_t)id];
            for (int a = 0; a < 3; ++a) {
                nd[2 * a] = make_float4(boxes[0].lo[a], boxes[1].lo[a], boxes[2].lo[a], boxes[3].lo[a]);
                nd[2 * a + 1] = make_float4(boxes[0].hi[a], boxes[1].hi[a], boxes[2].hi[a], boxes[3].hi[a]);
            }
            nd[6] = make_float4(bitsf(refs[0]), bitsf(refs[1]), bitsf(refs[2]), bitsf(refs[3]));
            nd[7] = make_float4(0.f, 0.f, 0.f, 0.f);
            --depth;
            return id;
        }
        float p[3], s[3];
        uint32_t qlo[3] = {0, 0, 0}, qhi[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a) {
            float lo = INFINITY, hi = -INFINITY;
            for (int k = 0; k < nc; ++k) { lo = std::min(lo, boxes[k].lo[a]); hi = std::max(hi, boxes[k].hi[a]); }
            p[a] = lo;
            s[a] = grid_step((double)hi - (double)lo);
            for (int k = 0; k < 4; ++k) {
                uint32_t l = 255u, h = 0u;   // an unused slot: inverted
                if (k < nc) {
                    l = quantise(p[a], s[a], boxes[k].lo[a], false);
                    h = quantise(p[a], s[a], boxes[k].hi[a], true);
                }
                qlo[a] |= l << (8 * k);
                qhi[a] |= h << (8 * k);
            }
        }
        float4* nd = &out[4 * (size_t)id];
        nd[0] = make_float4(p[0], p[1], p[2], s[0]);
        nd[1] = make_float4(s[1], s[2], bitsf(qlo[2]), bitsf(qhi[2]));
        nd[2] = make_float4(bitsf(qlo[0]), bitsf(qhi[0]), bitsf(qlo[1]), bitsf(qhi[1]));
        nd[3] = make_float4(bitsf(refs[0]), bitsf(refs[1]), bitsf(refs[2]), bitsf(refs[3]));
        --depth;
        return id;
    }

    // the grid step of an axis whose children span `extent`: extent / 255
    // rounded up to a float (1 for a flat axis, where every plane is p)
    static float grid_step(double extent)
    {
        if (!(extent > 0.0)) return 1.0f;
        float s = (float)(extent / 255.0);
        while ((double)s * 255.0 < extent) s = std::nextafter(s, INFINITY);
        return s;
    }
    // the grid index of plane x: the largest with p + q s <= x (a lower
    // plane) or the smallest with p + q s >= x (an upper plane), in 0..255
    static uint32_t quantise(float p, float s, float x, bool upper)
    {
        const double d = ((double)x - (double)p) / (double)s;
        long q = upper ? (long)std::ceil(d) : (long)std::floor(d);
        q = std::max(0L, std::min(255L, q));
        if (upper) {
            while (q < 255 && (double)p + (double)q * (double)s < (double)x) ++q;
        } else {
            while (q > 0 && (double)p + (double)q * (double)s > (double)x) --q;
        }
        return (uint32_t)q;
    }
};

}  // namespace

void build_bvh(const std::vector<float>& tri_v, int n_tris, float pad, int width, HostBVH& out, int quantise)
{
    std::vector<Prim> prims((size_t)n_tris);
    for (int i = 0; i < n_tris; ++i) {
        Prim& p = prims[(size_t)i];
        p.b.reset();
        for (int v = 0; v < 3; ++v)
            for (int a = 0; a < 3; ++a) {
                const float x = tri_v[(size_t)9 * i + 3 * v + a];
                p.b.lo[a] = std::min(p.b.lo[a], x);
                p.b.hi[a] = std::max(p.b.hi[a], x);
            }
        for (int a = 0; a < 3; ++a) p.c[a] = 0.5f * (p.b.lo[a] + p.b.hi[a]);
        p.id = (uint32_t)i;
    }
    Builder bld{prims, {}};
    bld.nodes.reserve((size_t)2 * n_tris / kLeafMax + 16);
    bld.build(0, n_tris, 0);
    out.nodes.clear();
    out.width = width;
    Emitter em{bld.nodes, out.nodes, pad, empty_ref((uint32_t)n_tris), quantise == 1};
    if (width == 4) {
        em.emit4(0);
        out.max_depth = em.max_depth;
        out.fmt = kNodeBvh4;
        const double bytes = sizeof(float4) * ((double)out.nodes.size() + 3.0 * n_tris);
        if (quantise == 1 || (quantise < 0 && bytes > kQuantiseBytes)) {
            if (!em.quant) {   // emitted as binary32 to size it: again, quantised
                out.nodes.clear();
                em.quant = true;
                em.depth = em.max_depth = 0;
                em.emit4(0);
            }
            out.fmt = kNodeBvh4Q;
        }
    } else {
        em.emit2(0);
        out.max_depth = bld.max_depth;
        out.fmt = kNodeBvh2;
    }
    out.order.resize((size_t)n_tris);
    for (int i = 0; i < n_tris; ++i) out.order[(size_t)i] = prims[(size_t)i].id;
}

}  // namespace rmlt

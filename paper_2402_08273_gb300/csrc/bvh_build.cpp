// Host-side binned SAH builder for the BVH2 the chain kernel traverses.
//
// Layout (4 float4 per internal node, children's boxes stored in the parent
// so one node fetch tests both children):
//   n0 = (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y)
//   n1 = (c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y)
//   n2 = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)
//   n3 = (ref c0, ref c1, 0, 0)   (uint bits)
// A ref is an internal node index, or a leaf: kLeafBit | (count-1) << 28 |
// first triangle (in build order).  Leaves hold at most 4 triangles.  Boxes
// are widened by `pad` and rounded outward so that binary32 traversal never
// culls a box a ray grazes.
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

constexpr int kBins = 16;
constexpr int kLeafMax = 4;

struct Builder {
    std::vector<Prim>& prims;
    std::vector<float4>& nodes;
    float pad;
    int max_depth = 0;

    static uint32_t fbits(float f)
    {
        uint32_t u;
        std::memcpy(&u, &f, 4);
        return u;
    }
    static float bitsf(uint32_t u)
    {
        float f;
        std::memcpy(&f, &u, 4);
        return f;
    }
    Box padded(const Box& b) const
    {
        Box o;
        for (int a = 0; a < 3; ++a) {
            o.lo[a] = std::nextafter(b.lo[a] - pad, -INFINITY);
            o.hi[a] = std::nextafter(b.hi[a] + pad, INFINITY);
        }
        return o;
    }

    uint32_t leaf(int b, int n) const { return kLeafBit | ((uint32_t)(n - 1) << 28) | (uint32_t)b; }

    uint32_t build(int b, int e, int depth, Box& box)
    {
        max_depth = std::max(max_depth, depth);
        box.reset();
        Box cb;
        cb.reset();
        for (int i = b; i < e; ++i) {
            box.grow(prims[i].b);
            for (int a = 0; a < 3; ++a) {
                cb.lo[a] = std::min(cb.lo[a], prims[i].c[a]);
                cb.hi[a] = std::max(cb.hi[a], prims[i].c[a]);
            }
        }
        const int n = e - b;
        if (n <= kLeafMax) return leaf(b, n);
        // binned SAH over the three axes
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
        const uint32_t id = (uint32_t)(nodes.size() / 4);
        nodes.resize(nodes.size() + 4);
        Box lb, rb;
        const uint32_t l = build(b, mid, depth + 1, lb);
        const uint32_t r = build(mid, e, depth + 1, rb);
        const Box L = padded(lb), R = padded(rb);
        float4* nd = &nodes[4 * (size_t)id];
        nd[0] = make_float4(L.lo[0], L.hi[0], L.lo[1], L.hi[1]);
        nd[1] = make_float4(R.lo[0], R.hi[0], R.lo[1], R.hi[1]);
        nd[2] = make_float4(L.lo[2], L.hi[2], R.lo[2], R.hi[2]);
        nd[3] = make_float4(bitsf(l), bitsf(r), 0.f, 0.f);
        return id;
    }
};

}  // namespace

void build_bvh(const std::vector<float>& tri_v, int n_tris, float pad, HostBVH& out)
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
    out.nodes.clear();
    out.nodes.reserve((size_t)4 * (size_t)std::max(1, n_tris / 2));
    Builder bld{prims, out.nodes, pad};
    Box root;
    bld.build(0, n_tris, 0, root);
    out.max_depth = bld.max_depth;
    out.order.resize((size_t)n_tris);
    for (int i = 0; i < n_tris; ++i) out.order[(size_t)i] = prims[(size_t)i].id;
}

}  // namespace rmlt

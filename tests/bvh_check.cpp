// Host-side check of the BVH builder's output (compiled and run by
// tests/test_bvh_host.py; no GPU).  Builds a BVH over a seeded synthetic
// triangle set and verifies, by walking the emitted node array from the root:
//   - the triangle order is a permutation of the input triangles;
//   - the leaves cover every position of that order exactly once and hold at
//     most `leaf_max` triangles;
//   - every vertex of a leaf's triangles lies inside every box on the path
//     from the root (the boxes are conservative; a BVH4 box is decoded from
//     its node's grid, p + q s, in binary64);
//   - a used quantised BVH4 slot has lo <= hi grid indices on every axis; an
//     unused BVH4 slot references the sentinel leaf past the triangles and
//     has an inverted box (binary32: +inf / -inf; quantised: indices 255 / 0);
//   - the depth the builder reports is the depth walked.
// Usage: bvh_check <layout 2|4|4q> <n_tris> <mode 0 random | 1 identical | 2 slivers> <seed> <leaf_max>
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "rmlt_internal.h"

namespace {

struct Box3 {
    double lo[3], hi[3];
};

uint32_t lcg(uint64_t& s)
{
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    return (uint32_t)(s >> 33);
}
float unit(uint64_t& s) { return (float)(lcg(s) >> 7) * (1.0f / 16777216.0f); }

uint32_t fbits(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
}

struct Walker {
    const rmlt::HostBVH& b;
    const std::vector<float>& v;
    int leaf_max;
    std::vector<int> covered;
    int depth_seen = 0;
    int errors = 0;

    void fail(const char* what, long a, long c)
    {
        if (errors++ < 5) std::printf("error: %s (%ld, %ld)\n", what, a, c);
    }

    void leaf(uint32_t ref, const std::vector<Box3>& path)
    {
        const uint32_t first = ref & 0x0FFFFFFFu, cnt = ((ref >> 28) & 7u) + 1u;
        if ((int)cnt > leaf_max) fail("leaf larger than the maximum", first, cnt);
        for (uint32_t i = first; i < first + cnt; ++i) {
            if (i >= covered.size()) {
                fail("leaf range outside the triangles", first, cnt);
                return;
            }
            ++covered[i];
            const uint32_t t = b.order[i];
            for (int k = 0; k < 3; ++k)
                for (const Box3& bx : path)
                    for (int a = 0; a < 3; ++a) {
                        const float x = v[(size_t)9 * t + 3 * k + a];
                        if (!(x >= bx.lo[a] && x <= bx.hi[a])) fail("vertex outside an ancestor box", t, a);
                    }
        }
    }

    void node(uint32_t id, std::vector<Box3>& path, int depth)
    {
        depth_seen = std::max(depth_seen, depth);
        const float4* nd = &b.nodes[(size_t)rmlt::node_float4s(b.fmt) * id];
        const int nc = b.width == 4 ? 4 : 2;
        for (int k = 0; k < nc; ++k) {
            Box3 bx;
            uint32_t ref;
            uint32_t ql[3] = {0, 0, 0}, qh[3] = {0, 0, 0};
            if (b.fmt == rmlt::kNodeBvh4) {
                const float* f = reinterpret_cast<const float*>(nd);
                for (int a = 0; a < 3; ++a) {
                    bx.lo[a] = f[4 * (2 * a) + k];
                    bx.hi[a] = f[4 * (2 * a + 1) + k];
                }
                ref = fbits(f[4 * 6 + k]);
            } else if (b.fmt == rmlt::kNodeBvh4Q) {
                const double p[3] = {nd[0].x, nd[0].y, nd[0].z}, s[3] = {nd[0].w, nd[1].x, nd[1].y};
                const uint32_t wl[3] = {fbits(nd[2].x), fbits(nd[2].z), fbits(nd[1].z)};
                const uint32_t wh[3] = {fbits(nd[2].y), fbits(nd[2].w), fbits(nd[1].w)};
                for (int a = 0; a < 3; ++a) {
                    if (!(s[a] > 0.0)) fail("grid step not positive", id, a);
                    ql[a] = (wl[a] >> (8 * k)) & 255u;
                    qh[a] = (wh[a] >> (8 * k)) & 255u;
                    bx.lo[a] = p[a] + (double)ql[a] * s[a];
                    bx.hi[a] = p[a] + (double)qh[a] * s[a];
                }
                ref = fbits((&nd[3].x)[k]);
            } else {
                const float4 xy = nd[k], z = nd[2];
                bx = {{xy.x, xy.z, k ? z.z : z.x}, {xy.y, xy.w, k ? z.w : z.y}};
                ref = fbits(k ? nd[3].y : nd[3].x);
            }
            if (ref == rmlt::empty_ref((uint32_t)covered.size())) {
                if (b.width != 4) fail("empty slot in a BVH2 node", id, k);
                for (int a = 0; a < 3; ++a) {
                    if (b.fmt == rmlt::kNodeBvh4Q && (ql[a] != 255u || qh[a] != 0u))
                        fail("empty slot without inverted grid indices", id, k);
                    if (b.fmt == rmlt::kNodeBvh4 && !(bx.lo[a] == INFINITY && bx.hi[a] == -INFINITY))
                        fail("empty slot without an inverted infinite box", id, k);
                }
                continue;
            }
            if (b.fmt == rmlt::kNodeBvh4Q)
                for (int a = 0; a < 3; ++a)
                    if (ql[a] > qh[a]) fail("used slot with inverted grid indices", id, k);
            path.push_back(bx);
            if (ref & rmlt::kLeafBit) leaf(ref, path);
            else if (ref <= id || (size_t)ref * rmlt::node_float4s(b.fmt) >= b.nodes.size()) fail("bad child node", id, ref);
            else node(ref, path, depth + 1);
            path.pop_back();
        }
    }
};

}  // namespace

int main(int argc, char** argv)
{
    if (argc != 6) {
        std::printf("usage: bvh_check layout n_tris mode seed leaf_max   (layout 2, 4 or 4q)\n");
        return 2;
    }
    const int width = std::atoi(argv[1]), n = std::atoi(argv[2]), mode = std::atoi(argv[3]);
    const int quant = std::strcmp(argv[1], "4q") == 0 ? 1 : 0;
    const int leaf_max = std::atoi(argv[5]);
    uint64_t s = (uint64_t)std::atoll(argv[4]) * 0x9E3779B97F4A7C15ull + 1u;
    std::vector<float> v((size_t)9 * n);
    for (int t = 0; t < n; ++t) {
        float c[3] = {unit(s) * 10.f - 5.f, unit(s) * 4.f, unit(s) * 7.f - 2.f};
        if (mode == 1) c[0] = c[1] = c[2] = 0.5f;   // every centroid the same: splits by count
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) {
                float d = (unit(s) - 0.5f) * 0.2f;
                if (mode == 2) d = a == 0 ? (unit(s) - 0.5f) * 6.f : (unit(s) - 0.5f) * 1e-3f;   // long slivers
                if (mode == 1) d = k == a ? 0.1f : 0.f;
                v[(size_t)9 * t + 3 * k + a] = c[a] + d;
            }
    }
    rmlt::HostBVH b;
    rmlt::build_bvh(v, n, 1e-6f * 10.f, width, b, quant);
    if (b.fmt != (width == 2 ? rmlt::kNodeBvh2 : quant ? rmlt::kNodeBvh4Q : rmlt::kNodeBvh4)) {
        std::printf("error: layout %d not the one asked for\n", b.fmt);
        return 1;
    }
    Walker w{b, v, leaf_max, std::vector<int>((size_t)n, 0)};
    if ((int)b.order.size() != n) w.fail("order has the wrong length", (long)b.order.size(), n);
    std::vector<int> seen((size_t)n, 0);
    for (uint32_t t : b.order) {
        if (t >= (uint32_t)n || seen[t]++) w.fail("order is not a permutation", t, n);
    }
    std::vector<Box3> path;
    if (b.nodes.empty()) w.fail("no nodes", n, width);
    else w.node(0, path, 1);
    for (int i = 0; i < n; ++i)
        if (w.covered[(size_t)i] != 1) w.fail("position not covered exactly once", i, w.covered[(size_t)i]);
    if (width == 4 && w.depth_seen != b.max_depth) w.fail("reported depth differs", b.max_depth, w.depth_seen);
    if (w.errors) return 1;
    std::printf("ok nodes=%zu depth=%d\n", b.nodes.size() / rmlt::node_float4s(b.fmt), w.depth_seen);
    return 0;
}

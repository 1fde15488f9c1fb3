// Reference traversal of the uploaded BVH on the host, in binary64: the
// yardstick for the chain kernel's traversal work counters.  It reads the
// same node and triangle arrays the kernels read (BVH4: eight float4 per
// node, rows lo.x hi.x lo.y hi.y lo.z hi.z of the four children and their
// references; BVH4Q: four float4, the node grid p, s and each child's box as
// 8-bit grid indices, decoded to p + q s in binary64, and the references;
// BVH2: four float4, both children's boxes and references; leaves
// referenced with bit 31, the count - 1 in bits 28..30 and the first
// triangle below), and walks them the textbook
// way: at an internal node every child box is slab-tested against the ray
// segment [0, t] (t the closest hit so far), the hit children are visited
// nearest entry first (the rest stacked), a leaf's triangles are tested with
// Moller-Trumbore, and an any-hit ray stops at the first leaf with a hit.
// Each internal node visited and each triangle tested counts once.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "rmlt_internal.h"

namespace rmlt {
namespace {

uint32_t bits(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
}

struct Ray {
    double o[3], d[3], inv[3], tmax;
    bool any;
};

// entry distance of the box [lo, hi] along the ray within [0, t], or -1
double slab(const Ray& r, const double lo[3], const double hi[3], double t)
{
    double tn = 0.0, tf = t;
    for (int a = 0; a < 3; ++a) {
        if (!(lo[a] <= hi[a])) return -1.0;   // an unused slot (inverted box)
        double t0 = (lo[a] - r.o[a]) * r.inv[a], t1 = (hi[a] - r.o[a]) * r.inv[a];
        if (t0 > t1) std::swap(t0, t1);
        tn = std::fmax(tn, t0);
        tf = std::fmin(tf, t1);
    }
    return tn <= tf ? tn : -1.0;
}

// Moller-Trumbore in binary64 on a triangle stored as v0, e1, e2
bool tri_hit(const Ray& r, const float4* T, double tmax, double& t)
{
    const double v0[3] = {T[0].x, T[0].y, T[0].z}, e1[3] = {T[1].x, T[1].y, T[1].z}, e2[3] = {T[2].x, T[2].y, T[2].z};
    const double p[3] = {r.d[1] * e2[2] - r.d[2] * e2[1], r.d[2] * e2[0] - r.d[0] * e2[2],
                         r.d[0] * e2[1] - r.d[1] * e2[0]};
    const double det = e1[0] * p[0] + e1[1] * p[1] + e1[2] * p[2];
    if (det == 0.0) return false;
    const double inv = 1.0 / det;
    const double s[3] = {r.o[0] - v0[0], r.o[1] - v0[1], r.o[2] - v0[2]};
    const double u = (s[0] * p[0] + s[1] * p[1] + s[2] * p[2]) * inv;
    if (u < 0.0 || u > 1.0) return false;
    const double qv[3] = {s[1] * e1[2] - s[2] * e1[1], s[2] * e1[0] - s[0] * e1[2], s[0] * e1[1] - s[1] * e1[0]};
    const double v = (r.d[0] * qv[0] + r.d[1] * qv[1] + r.d[2] * qv[2]) * inv;
    if (v < 0.0 || u + v > 1.0) return false;
    t = (e2[0] * qv[0] + e2[1] * qv[1] + e2[2] * qv[2]) * inv;
    return t > 0.0 && t < tmax;
}

}  // namespace

WalkResult walk_ray(const std::vector<float4>& nodes, int fmt, const std::vector<float4>& tris, bool brute,
                    const float ray[8])
{
    Ray r;
    for (int a = 0; a < 3; ++a) {
        r.o[a] = ray[a];
        r.d[a] = ray[4 + a];
        r.inv[a] = 1.0 / (r.d[a] != 0.0 ? r.d[a] : 1e-300);
    }
    r.tmax = ray[3];
    r.any = ray[7] != 0.0f;
    WalkResult res{-1, r.tmax, 0u, 0u};
    int best = -1;
    double t = r.tmax;
    const int n_tris = (int)(tris.size() / 3);
    if (brute || nodes.empty()) {
        for (int i = 0; i < n_tris; ++i) {
            double th;
            ++res.tris;
            if (tri_hit(r, &tris[3 * (size_t)i], t, th)) {
                t = th;
                best = i;
                if (r.any) break;
            }
        }
    } else {
        std::vector<uint32_t> stack;
        stack.push_back(0u);
        while (!stack.empty()) {
            const uint32_t ref = stack.back();
            stack.pop_back();
            if (ref & kLeafBit) {
                const uint32_t first = ref & 0x0FFFFFFFu, cnt = ((ref >> 28) & 7u) + 1u;
                bool found = false;
                for (uint32_t i = first; i < first + cnt; ++i) {
                    double th;
                    ++res.tris;
                    if (tri_hit(r, &tris[3 * (size_t)i], t, th)) {
                        t = th;
                        best = (int)i;
                        found = true;
                    }
                }
                if (r.any && found) break;
                continue;
            }
            ++res.nodes;
            double key[4];
            uint32_t cref[4];
            int nc = 0;
            if (fmt == kNodeBvh4) {
                const float4* nd = &nodes[8 * (size_t)ref];
                const float lx[4] = {nd[0].x, nd[0].y, nd[0].z, nd[0].w}, hx[4] = {nd[1].x, nd[1].y, nd[1].z, nd[1].w};
                const float ly[4] = {nd[2].x, nd[2].y, nd[2].z, nd[2].w}, hy[4] = {nd[3].x, nd[3].y, nd[3].z, nd[3].w};
                const float lz[4] = {nd[4].x, nd[4].y, nd[4].z, nd[4].w}, hz[4] = {nd[5].x, nd[5].y, nd[5].z, nd[5].w};
                const uint32_t rf[4] = {bits(nd[6].x), bits(nd[6].y), bits(nd[6].z), bits(nd[6].w)};
                for (int k = 0; k < 4; ++k) {
                    const double lo[3] = {lx[k], ly[k], lz[k]}, hi[3] = {hx[k], hy[k], hz[k]};
                    const double tn = slab(r, lo, hi, t);
                    if (tn >= 0.0) { key[nc] = tn; cref[nc++] = rf[k]; }
                }
            } else if (fmt == kNodeBvh4Q) {
                const float4* nd = &nodes[4 * (size_t)ref];
                const double p[3] = {nd[0].x, nd[0].y, nd[0].z}, s[3] = {nd[0].w, nd[1].x, nd[1].y};
                const uint32_t ql[3] = {bits(nd[2].x), bits(nd[2].z), bits(nd[1].z)};
                const uint32_t qh[3] = {bits(nd[2].y), bits(nd[2].w), bits(nd[1].w)};
                const uint32_t rf[4] = {bits(nd[3].x), bits(nd[3].y), bits(nd[3].z), bits(nd[3].w)};
                for (int k = 0; k < 4; ++k) {
                    double lo[3], hi[3];
                    for (int a = 0; a < 3; ++a) {
                        lo[a] = p[a] + (double)((ql[a] >> (8 * k)) & 255u) * s[a];
                        hi[a] = p[a] + (double)((qh[a] >> (8 * k)) & 255u) * s[a];
                    }
                    const double tn = slab(r, lo, hi, t);
                    if (tn >= 0.0) { key[nc] = tn; cref[nc++] = rf[k]; }
                }
            } else {
                const float4* nd = &nodes[4 * (size_t)ref];
                const double lo0[3] = {nd[0].x, nd[0].z, nd[2].x}, hi0[3] = {nd[0].y, nd[0].w, nd[2].y};
                const double lo1[3] = {nd[1].x, nd[1].z, nd[2].z}, hi1[3] = {nd[1].y, nd[1].w, nd[2].w};
                const uint32_t rf[2] = {bits(nd[3].x), bits(nd[3].y)};
                double tn = slab(r, lo0, hi0, t);
                if (tn >= 0.0) { key[nc] = tn; cref[nc++] = rf[0]; }
                tn = slab(r, lo1, hi1, t);
                if (tn >= 0.0) { key[nc] = tn; cref[nc++] = rf[1]; }
            }
            // nearest entry visited next: stack the others far to near
            for (int a = 1; a < nc; ++a)
                for (int b = a; b > 0 && key[b] < key[b - 1]; --b) {
                    std::swap(key[b], key[b - 1]);
                    std::swap(cref[b], cref[b - 1]);
                }
            for (int k = nc - 1; k >= 0; --k) stack.push_back(cref[k]);
        }
    }
    if (best >= 0) {
        res.tri = (int32_t)bits(tris[3 * (size_t)best + 1].w);
        res.t = t;
    }
    return res;
}

}  // namespace rmlt

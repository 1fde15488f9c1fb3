// Host check of the reference traversal (csrc/bvh_walk.cpp; compiled and run
// by tests/test_bvh_host.py, no GPU): over a seeded triangle soup, random
// closest-hit rays walked through the built BVH find the same triangle and
// distance as a brute-force loop over every triangle; any-hit rays agree on
// occlusion; every ray visits at least the root; and a ray that misses the
// scene's box visits the root only.
// Usage: bvh_walk_check <layout 2|4|4q> <n_tris> <seed>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "rmlt_internal.h"

namespace {
uint32_t lcg(uint64_t& s)
{
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    return (uint32_t)(s >> 33);
}
float unit(uint64_t& s) { return (float)(lcg(s) >> 7) * (1.0f / 16777216.0f); }
}  // namespace

int main(int argc, char** argv)
{
    if (argc < 4) return 2;
    const int width = std::atoi(argv[1]), n = std::atoi(argv[2]);
    const int quant = std::strcmp(argv[1], "4q") == 0 ? 1 : 0;
    uint64_t s = (uint64_t)std::atoll(argv[3]) * 7919u + 1u;
    std::vector<float> tv((size_t)9 * n);
    for (int i = 0; i < n; ++i) {
        const float c[3] = {unit(s), unit(s), unit(s)};
        for (int v = 0; v < 3; ++v)
            for (int a = 0; a < 3; ++a) tv[(size_t)9 * i + 3 * v + a] = c[a] + 0.05f * (unit(s) - 0.5f);
    }
    rmlt::HostBVH bvh;
    rmlt::build_bvh(tv, n, 1e-6f, width, bvh, quant);
    // triangles in leaf order as the library uploads them: v0 | -, e1 | original index, e2
    std::vector<float4> tris((size_t)3 * n);
    for (int j = 0; j < n; ++j) {
        const uint32_t i = bvh.order[(size_t)j];
        const float* p = &tv[(size_t)9 * i];
        float idf;
        std::memcpy(&idf, &i, 4);
        tris[3 * (size_t)j + 0] = make_float4(p[0], p[1], p[2], 0.f);
        tris[3 * (size_t)j + 1] = make_float4(p[3] - p[0], p[4] - p[1], p[5] - p[2], idf);
        tris[3 * (size_t)j + 2] = make_float4(p[6] - p[0], p[7] - p[1], p[8] - p[2], 0.f);
    }
    int errors = 0, hits = 0;
    for (int k = 0; k < 2000; ++k) {
        float ray[8];
        for (int a = 0; a < 3; ++a) ray[a] = unit(s) * 1.4f - 0.2f;
        float d[3] = {unit(s) - 0.5f, unit(s) - 0.5f, unit(s) - 0.5f};
        const float l = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int a = 0; a < 3; ++a) ray[4 + a] = d[a] / l;
        ray[3] = 3.0e38f;
        ray[7] = (k % 3 == 0) ? 1.0f : 0.0f;
        if (ray[7] != 0.0f) ray[3] = 0.5f;
        const rmlt::WalkResult a = rmlt::walk_ray(bvh.nodes, bvh.fmt, tris, false, ray);
        const rmlt::WalkResult b = rmlt::walk_ray(bvh.nodes, bvh.fmt, tris, true, ray);
        if (a.nodes < 1) ++errors;
        if (ray[7] != 0.0f) {
            if ((a.tri >= 0) != (b.tri >= 0)) ++errors;
        } else {
            if (a.tri != b.tri || (a.tri >= 0 && std::fabs(a.t - b.t) > 1e-12 * std::fmax(1.0, b.t))) {
                if (errors++ < 5) std::printf("mismatch ray %d: %d %.17g vs %d %.17g\n", k, a.tri, a.t, b.tri, b.t);
            }
        }
        hits += a.tri >= 0;
    }
    // a ray that leaves the scene's box: the root only
    const float away[8] = {5.f, 5.f, 5.f, 3.0e38f, 1.f, 0.f, 0.f, 0.f};
    const rmlt::WalkResult w = rmlt::walk_ray(bvh.nodes, bvh.fmt, tris, false, away);
    if (w.nodes != 1 || w.tris != 0 || w.tri != -1) ++errors;
    if (errors) {
        std::printf("errors %d\n", errors);
        return 1;
    }
    std::printf("ok %d hits\n", hits);
    return 0;
}

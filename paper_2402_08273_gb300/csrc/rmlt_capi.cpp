// Host side of librmlt: the C ABI declared in include/rmlt.h.
//
// Owns the context (device, stream, allocator hooks, device buffers), checks
// arguments, builds and uploads the scene, drives the epoch loop of the chain
// kernel and the region update (Alg. 1), and copies results out.  Every
// arithmetic step of the method runs in the CUDA kernels (rmlt_kernels.cu).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "rmlt.h"
#include "rmlt_internal.h"

using namespace rmlt;

namespace {

thread_local std::string g_err;

rmlt_status fail(rmlt_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

rmlt_status cuda_fail(cudaError_t e, const char* what)
{
    if (e == cudaErrorMemoryAllocation) return fail(RMLT_E_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(RMLT_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                    \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

struct Alloc {
    void* p = nullptr;
    size_t bytes = 0;
};

uint64_t fnv64(const void* data, size_t n, uint64_t h)
{
    const unsigned char* p = (const unsigned char*)data;
    for (size_t i = 0; i < n; ++i) { h ^= p[i]; h *= 1099511628211ull; }
    return h;
}

// NVTX range for profilers (a no-op unless a tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

}  // namespace

struct rmlt_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    rmlt_alloc_fn af = nullptr;
    rmlt_free_fn ff = nullptr;
    void* au = nullptr;
    std::vector<Alloc> scene_mem, chain_mem;
    uint64_t held = 0;

    bool have_scene = false, have_chains = false, failed = false;
    std::vector<float4> h_nodes, h_tris;   // host copies of the uploaded BVH nodes and triangles
    int h_fmt = kNodeBvh4;       // node layout of h_nodes
    int node_format = RMLT_NODES_AUTO;   // BVH4 layout of the next rmlt_load_scene
    bool scene_lambert = true;   // every material Lambertian: the path map is differentiable (Langevin strategy)
    DevScene S;
    double tan_half = 1.0;
    uint64_t scene_hash = 0;

    rmlt_chain_params P{};
    DevChains Ch;
    uint64_t mut = 0, epochs = 0;
    int64_t n_boot = 0;
    double* d_total = nullptr;   // bootstrap sum of pi (device, binary64)
    double* d_stage = nullptr;   // image read-out staging [H][W][3]

    rmlt_trace_record* tr = nullptr;
    uint64_t tr_cap = 0, tr_epoch = 0;
    uint32_t* tr_words = nullptr;    // the proposal words of each record (optional)
    double* tr_lam = nullptr;
    uint64_t tr_lam_cap = 0;
    uint32_t tr_stride = 1;
    bool count_work = false;
    uint64_t since_refine = 0;   // mutations since the last quadtree pass
    int batch_shade = 12, batch_setup = 10;
    int large_ahead = 0, adaptive_batch = 0;
    int wavefront = 0, wf_trace_cps = 0, wf_setup_cps = 0, wf_refill = 8, wf_flags = 0, wf_leaf_batch = kLeafBatch;
    unsigned wave_limit = 0;     // waves per epoch before the wavefront form stops (0: its default)
    bool wf_ran = false;         // an epoch ran in the wavefront form since the chains were set up
    uint64_t wave_hits_seen = 0; // epochs stopped by the wave limit, as of the last check
    DevWave W;                   // wavefront state (allocated on first use)
    WfGraph* wg = nullptr;       // its instantiated wave loop
    bool in_epoch = false;       // rmlt_epoch_mutate ran, rmlt_epoch_update is due

    rmlt_status dalloc(std::vector<Alloc>& pool, size_t bytes, void** out)
    {
        void* p = nullptr;
        if (bytes == 0) bytes = 16;
        if (af) {
            p = af(au, bytes, (void*)stream);
            if (!p) return fail(RMLT_E_OOM, "allocator returned NULL for %zu bytes", bytes);
        } else {
            cudaError_t e = cudaMalloc(&p, bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(RMLT_E_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
            }
        }
        pool.push_back({p, bytes});
        held += bytes;
        *out = p;
        return RMLT_OK;
    }
    void release(std::vector<Alloc>& pool)
    {
        if (!pool.empty()) cudaStreamSynchronize(stream);
        for (auto& a : pool) {
            if (ff) ff(au, a.p, (void*)stream);
            else cudaFree(a.p);
            held -= a.bytes;
        }
        pool.clear();
    }
    template <class T>
    rmlt_status alloc_n(std::vector<Alloc>& pool, size_t n, T** out)
    {
        return dalloc(pool, n * sizeof(T), (void**)out);
    }
};

namespace {

rmlt_status enter(rmlt_ctx* c)
{
    if (!c) return fail(RMLT_E_INVALID_ARG, "null context");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return RMLT_OK;
}

rmlt_status sync(rmlt_ctx* c, const char* what)
{
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->failed = true;
        return cuda_fail(e, what);
    }
    // an epoch of the wavefront form stopped by its wave limit left
    // mutations unfinished: the chains are no longer a valid sample
    if (c->wf_ran && c->have_chains && !c->failed) {
        unsigned long long hits = 0;
        e = cudaMemcpy(&hits, c->Ch.stats + kStWaveLimit, sizeof hits, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            c->failed = true;
            return cuda_fail(e, what);
        }
        if (hits > c->wave_hits_seen) {
            c->wave_hits_seen = hits;
            c->failed = true;
            return fail(RMLT_E_OVERFLOW, "%s: %llu epoch(s) stopped at the wave limit of the wavefront form", what,
                        hits);
        }
    }
    return RMLT_OK;
}

// copy `bytes` from device memory to a caller buffer (host or device)
rmlt_status copy_out(rmlt_ctx* c, void* dst, const void* src, size_t bytes)
{
    if (!dst || bytes == 0) return RMLT_OK;
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream), "copy out");
    return RMLT_OK;
}

bool finite3(const float* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

}  // namespace

extern "C" {

int rmlt_abi_version(void) { return RMLT_ABI_VERSION; }

const char* rmlt_last_error(void) { return g_err.c_str(); }

rmlt_status rmlt_create(rmlt_ctx** out, int device, void* cuda_stream)
{
    if (!out) return fail(RMLT_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        return fail(RMLT_E_CUDA, "no CUDA device available (%s)", cudaGetErrorString(e));
    }
    if (device < 0 || device >= n) return fail(RMLT_E_INVALID_ARG, "device %d out of range [0,%d)", device, n);
    CK(cudaSetDevice(device), "cudaSetDevice");
    CK(cudaFree(nullptr), "context init");
    rmlt_ctx* c = new (std::nothrow) rmlt_ctx();
    if (!c) return fail(RMLT_E_OOM, "host allocation failed");
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    *out = c;
    return RMLT_OK;
}

rmlt_status rmlt_set_allocator(rmlt_ctx* c, rmlt_alloc_fn alloc, rmlt_free_fn free_fn, void* user)
{
    if (!c) return fail(RMLT_E_INVALID_ARG, "null context");
    if ((alloc == nullptr) != (free_fn == nullptr)) return fail(RMLT_E_INVALID_ARG, "alloc and free must both be set or both be NULL");
    if (!c->scene_mem.empty() || !c->chain_mem.empty()) return fail(RMLT_E_STATE, "allocator must be set before any device memory is held");
    c->af = alloc;
    c->ff = free_fn;
    c->au = user;
    return RMLT_OK;
}

static void drop_chains(rmlt_ctx* c)
{
    if (c->wg) cudaStreamSynchronize(c->stream);
    wf_graph_destroy(c->wg);
    c->wg = nullptr;
    c->W = DevWave();
    c->release(c->chain_mem);
    c->have_chains = false;
    c->failed = false;
    c->Ch = DevChains();
    c->d_total = c->d_stage = nullptr;
    c->tr = nullptr;
    c->tr_lam = nullptr;
    c->wf_ran = false;
    c->wave_hits_seen = 0;
    c->in_epoch = false;
}

rmlt_status rmlt_load_scene(rmlt_ctx* c, const rmlt_scene_desc* s)
{
    rmlt_status st = enter(c);
    if (st) return st;
    if (!s) return fail(RMLT_E_INVALID_ARG, "scene is NULL");
    if (s->n_tris <= 0 || s->n_verts <= 0 || s->n_mats <= 0 || !s->verts || !s->tris || !s->mat_id || !s->mats)
        return fail(RMLT_E_INVALID_SCENE, "scene needs vertices, triangles, material ids and materials");
    if (s->n_tris >= (1 << 28)) return fail(RMLT_E_INVALID_SCENE, "at most 2^28 - 1 triangles");
    const int brute_max = s->brute_force_max > 0 ? s->brute_force_max : 64;
    if (brute_max > 4096) return fail(RMLT_E_INVALID_ARG, "brute_force_max above 4096");
    const int width = s->bvh_width == 0 ? 4 : s->bvh_width;
    if (width != 2 && width != 4) return fail(RMLT_E_INVALID_ARG, "bvh_width must be 0, 2 or 4");
    for (int i = 0; i < s->n_verts; ++i)
        if (!finite3(&s->verts[3 * (size_t)i])) return fail(RMLT_E_INVALID_SCENE, "vertex %d is not finite", i);
    for (int m = 0; m < s->n_mats; ++m) {
        const rmlt_material& M = s->mats[m];
        if (M.type != RMLT_LAMBERT && M.type != RMLT_GGX) return fail(RMLT_E_INVALID_SCENE, "material %d: unknown type %d", m, M.type);
        if (!finite3(M.albedo) || !finite3(M.emission)) return fail(RMLT_E_INVALID_SCENE, "material %d: non-finite colour", m);
        for (int a = 0; a < 3; ++a)
            if (M.albedo[a] < 0.f || M.albedo[a] > 1.f || M.emission[a] < 0.f)
                return fail(RMLT_E_INVALID_SCENE, "material %d: albedo outside [0,1] or negative emission", m);
        if (M.type == RMLT_GGX && !(M.roughness >= 1e-3f && M.roughness <= 1.f))
            return fail(RMLT_E_INVALID_SCENE, "material %d: GGX roughness outside [1e-3, 1]", m);
    }
    bool lambert = true;
    for (int m = 0; m < s->n_mats; ++m) lambert = lambert && s->mats[m].type == RMLT_LAMBERT;
    const int nt = s->n_tris;
    std::vector<float> tv((size_t)9 * nt);
    for (int i = 0; i < nt; ++i) {
        for (int v = 0; v < 3; ++v) {
            const uint32_t vi = s->tris[3 * (size_t)i + v];
            if ((int64_t)vi >= s->n_verts) return fail(RMLT_E_INVALID_SCENE, "triangle %d: vertex index %u out of range", i, vi);
            for (int a = 0; a < 3; ++a) tv[(size_t)9 * i + 3 * v + a] = s->verts[3 * (size_t)vi + a];
        }
        if ((int64_t)s->mat_id[i] >= s->n_mats) return fail(RMLT_E_INVALID_SCENE, "triangle %d: material %u out of range", i, s->mat_id[i]);
    }
    const rmlt_camera& cam = s->camera;
    if (!finite3(cam.pos) || !finite3(cam.look_at) || !finite3(cam.up) || !(cam.vfov_deg > 0.f && cam.vfov_deg < 180.f))
        return fail(RMLT_E_INVALID_SCENE, "bad camera");

    // scene scale, lights in original triangle order sampled in proportion to area
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = 0; i < s->n_verts; ++i)
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::fmin(lo[a], (double)s->verts[3 * (size_t)i + a]);
            hi[a] = std::fmax(hi[a], (double)s->verts[3 * (size_t)i + a]);
        }
    const double scale = std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) + (hi[2] - lo[2]) * (hi[2] - lo[2]));
    if (!(scale > 0.0)) return fail(RMLT_E_INVALID_SCENE, "degenerate scene bounds");
    std::vector<int> lights;
    std::vector<double> lcum;
    double acc = 0.0;
    for (int i = 0; i < nt; ++i) {
        const rmlt_material& M = s->mats[s->mat_id[i]];
        if (!(M.emission[0] > 0.f || M.emission[1] > 0.f || M.emission[2] > 0.f)) continue;
        const float* p = &tv[(size_t)9 * i];
        const double e1[3] = {(double)p[3] - p[0], (double)p[4] - p[1], (double)p[5] - p[2]};
        const double e2[3] = {(double)p[6] - p[0], (double)p[7] - p[1], (double)p[8] - p[2]};
        const double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2], cz = e1[0] * e2[1] - e1[1] * e2[0];
        const double area2 = std::sqrt(cx * cx + cy * cy + cz * cz);
        if (!(area2 > 0.0)) continue;
        acc += 0.5 * area2;
        lights.push_back(i);
        lcum.push_back(acc);
    }
    std::vector<float> lcdf(lights.size());
    for (size_t j = 0; j < lights.size(); ++j) lcdf[j] = (float)(lcum[j] / acc);
    if (!lcdf.empty()) lcdf.back() = 1.0f;

    // triangle order: BVH build order, or input order for brute force
    const bool brute = nt <= brute_max || nt <= 4;
    HostBVH bvh;
    if (!brute)
        build_bvh(tv, nt, (float)(1e-6 * scale), width, bvh,
                  c->node_format == RMLT_NODES_QUANTISED ? 1 : c->node_format == RMLT_NODES_FLOAT ? 0 : -1);
    std::vector<uint32_t> order((size_t)nt), inv((size_t)nt);
    for (int i = 0; i < nt; ++i) order[(size_t)i] = brute ? (uint32_t)i : bvh.order[(size_t)i];
    for (int i = 0; i < nt; ++i) inv[order[(size_t)i]] = (uint32_t)i;
    // with a BVH, a zero-area sentinel triangle after the scene's (the leaf
    // that unused BVH4 slots reference)
    std::vector<float4> tri4((size_t)3 * (nt + (brute ? 0 : 1)), make_float4(0.f, 0.f, 0.f, 0.f));
    for (int j = 0; j < nt; ++j) {
        const uint32_t i = order[(size_t)j];
        const float* p = &tv[(size_t)9 * i];
        int32_t mid = (int32_t)s->mat_id[i];
        float midf, idf;
        std::memcpy(&midf, &mid, 4);
        std::memcpy(&idf, &i, 4);
        tri4[3 * (size_t)j + 0] = make_float4(p[0], p[1], p[2], midf);
        tri4[3 * (size_t)j + 1] = make_float4(p[3] - p[0], p[4] - p[1], p[5] - p[2], idf);
        tri4[3 * (size_t)j + 2] = make_float4(p[6] - p[0], p[7] - p[1], p[8] - p[2], 0.f);
    }
    std::vector<int32_t> ltri(lights.size());
    for (size_t j = 0; j < lights.size(); ++j) ltri[j] = (int32_t)inv[(size_t)lights[j]];
    std::vector<float4> mat4((size_t)3 * s->n_mats);
    for (int m = 0; m < s->n_mats; ++m) {
        const rmlt_material& M = s->mats[m];
        const bool emissive = M.emission[0] > 0.f || M.emission[1] > 0.f || M.emission[2] > 0.f;
        const bool black = M.albedo[0] <= 0.f && M.albedo[1] <= 0.f && M.albedo[2] <= 0.f;
        mat4[3 * (size_t)m + 0] = make_float4(M.albedo[0], M.albedo[1], M.albedo[2], (float)M.type);
        mat4[3 * (size_t)m + 1] = make_float4(M.emission[0], M.emission[1], M.emission[2], M.roughness);
        mat4[3 * (size_t)m + 2] = make_float4(emissive ? 1.f : 0.f, black ? 1.f : 0.f, 0.f, 0.f);
    }

    // pinhole camera basis in binary64, stored in binary32
    double pos[3] = {cam.pos[0], cam.pos[1], cam.pos[2]};
    double fw[3] = {(double)cam.look_at[0] - pos[0], (double)cam.look_at[1] - pos[1], (double)cam.look_at[2] - pos[2]};
    double fl = std::sqrt(fw[0] * fw[0] + fw[1] * fw[1] + fw[2] * fw[2]);
    if (!(fl > 0.0)) return fail(RMLT_E_INVALID_SCENE, "camera looks at its own position");
    for (double& x : fw) x /= fl;
    const double up[3] = {cam.up[0], cam.up[1], cam.up[2]};
    double rt[3] = {fw[1] * up[2] - fw[2] * up[1], fw[2] * up[0] - fw[0] * up[2], fw[0] * up[1] - fw[1] * up[0]};
    double rl = std::sqrt(rt[0] * rt[0] + rt[1] * rt[1] + rt[2] * rt[2]);
    if (!(rl > 0.0)) return fail(RMLT_E_INVALID_SCENE, "camera up is parallel to the view direction");
    for (double& x : rt) x /= rl;
    const double uo[3] = {rt[1] * fw[2] - rt[2] * fw[1], rt[2] * fw[0] - rt[0] * fw[2], rt[0] * fw[1] - rt[1] * fw[0]};

    // the new scene's device memory, in a pool of its own: on failure it is
    // released and the previous scene (and chains) stay as they were
    std::vector<Alloc> fresh;
    DevScene S;
    float4 *d_tri = nullptr, *d_nodes = nullptr, *d_mat = nullptr;
    int32_t* d_lt = nullptr;
    float* d_lc = nullptr;
    if ((st = c->alloc_n(fresh, tri4.size(), &d_tri)) ||
        (st = c->alloc_n(fresh, std::max<size_t>(8, bvh.nodes.size()), &d_nodes)) ||
        (st = c->alloc_n(fresh, mat4.size(), &d_mat)) ||
        (st = c->alloc_n(fresh, std::max<size_t>(1, ltri.size()), &d_lt)) ||
        (st = c->alloc_n(fresh, std::max<size_t>(1, lcdf.size()), &d_lc))) {
        c->release(fresh);
        return st;
    }
    cudaError_t e = cudaMemcpyAsync(d_tri, tri4.data(), tri4.size() * sizeof(float4), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !bvh.nodes.empty())
        e = cudaMemcpyAsync(d_nodes, bvh.nodes.data(), bvh.nodes.size() * sizeof(float4), cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_mat, mat4.data(), mat4.size() * sizeof(float4), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !ltri.empty())
        e = cudaMemcpyAsync(d_lt, ltri.data(), ltri.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !ltri.empty())
        e = cudaMemcpyAsync(d_lc, lcdf.data(), lcdf.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->release(fresh);
        return cuda_fail(e, "scene upload");
    }
    S.tris = d_tri;
    S.nodes = d_nodes;
    S.mats = d_mat;
    S.light_tri = d_lt;
    S.light_cdf = d_lc;
    S.n_tris = nt;
    S.node_fmt = brute ? kNodeBvh4 : bvh.fmt;
    S.n_nodes = (int32_t)(bvh.nodes.size() / node_float4s(S.node_fmt));
    S.n_mats = s->n_mats;
    S.n_lights = (int32_t)ltri.size();
    S.brute = brute ? 1 : 0;
    S.light_area = (float)acc;
    for (int a = 0; a < 3; ++a) {
        S.cam_pos[a] = (float)pos[a];
        S.cam_fwd[a] = (float)fw[a];
        S.cam_right[a] = (float)rt[a];
        S.cam_up[a] = (float)uo[a];
    }
    S.eps = (float)(1e-4 * scale);
    S.toy = 0;

    // replace the previous scene (and chains)
    drop_chains(c);
    c->release(c->scene_mem);
    c->scene_mem = std::move(fresh);
    c->h_nodes = std::move(bvh.nodes);
    c->h_tris = std::move(tri4);
    c->h_fmt = S.node_fmt;
    c->tan_half = std::tan((double)cam.vfov_deg * 3.14159265358979323846 / 360.0);
    c->S = S;
    uint64_t h = fnv64(tv.data(), tv.size() * sizeof(float), 1469598103934665603ull);
    h = fnv64(s->mat_id, (size_t)nt * sizeof(uint32_t), h);
    h = fnv64(mat4.data(), mat4.size() * sizeof(float4), h);
    c->scene_hash = fnv64(&cam, sizeof cam, h);
    c->have_scene = true;
    c->scene_lambert = lambert;
    return RMLT_OK;
}

rmlt_status rmlt_load_toy_integrand(rmlt_ctx* c, const double* params)
{
    rmlt_status st = enter(c);
    if (st) return st;
    if (!params) return fail(RMLT_E_INVALID_ARG, "params is NULL");
    for (int i = 0; i < 10; ++i)
        if (!std::isfinite(params[i])) return fail(RMLT_E_INVALID_ARG, "toy parameter %d not finite", i);
    if (!(params[9] > 0.0)) return fail(RMLT_E_INVALID_ARG, "toy Gaussian width must be positive");
    drop_chains(c);
    c->release(c->scene_mem);
    DevScene S;
    S.toy = 1;
    for (int i = 0; i < 10; ++i) S.toy_p[i] = (float)params[i];
    S.brute = 0;
    c->S = S;
    c->scene_hash = fnv64(params, 10 * sizeof(double), 77);
    c->have_scene = true;
    c->scene_lambert = true;
    return RMLT_OK;
}

// chains over every context of a (possibly sharded) population
static int32_t chains_all(const rmlt_chain_params* p) { return p->chains_total > 0 ? p->chains_total : p->n_chains; }

static rmlt_status check_params(const rmlt_ctx* c, const rmlt_chain_params* p)
{
    if (!p) return fail(RMLT_E_INVALID_ARG, "params is NULL");
    if (p->n_chains <= 0 || p->n_chains >= 0x7FFFFFFF) return fail(RMLT_E_INVALID_ARG, "n_chains must be in [1, 2^31-1)");
    if (p->chains_total < 0 || p->chain_first < 0 ||
        (p->chains_total > 0 && (int64_t)p->chain_first + p->n_chains > (int64_t)p->chains_total) ||
        (p->chains_total == 0 && p->chain_first != 0))
        return fail(RMLT_E_INVALID_ARG, "need 0 <= chain_first, chain_first + n_chains <= chains_total (or both 0)");
    if (p->width <= 0 || p->height <= 0 || p->width > (1 << 16) || p->height > (1 << 16))
        return fail(RMLT_E_INVALID_ARG, "image size must be in [1, 65536]");
    if (p->region_px <= 0) return fail(RMLT_E_INVALID_ARG, "region_px must be positive");
    if (c->S.toy ? p->max_depth != 0 : (p->max_depth < 1 || p->max_depth > RMLT_MAX_DEPTH))
        return fail(RMLT_E_INVALID_ARG, "max_depth must be 0 for the toy integrand and 1..%d for a scene", RMLT_MAX_DEPTH);
    if (p->epoch_len <= 0 || p->L <= 0) return fail(RMLT_E_INVALID_ARG, "epoch_len and L must be positive");
    if (p->target_mode != RMLT_TARGET_PLAIN && p->target_mode != RMLT_TARGET_REGION_WEIGHTED)
        return fail(RMLT_E_INVALID_ARG, "unknown target_mode");
    if (p->n_bootstrap < chains_all(p) || p->n_bootstrap > (1ll << 34))
        return fail(RMLT_E_INVALID_ARG, "n_bootstrap must be in [chains of the population, 2^34]");
    if (!(p->p_large >= 0.0 && p->p_large <= 1.0)) return fail(RMLT_E_INVALID_ARG, "p_large outside [0,1]");
    if (!(p->s1 > 0.0 && p->s1 < p->s2 && p->s2 <= 0.5)) return fail(RMLT_E_INVALID_ARG, "need 0 < s1 < s2 <= 1/2");
    if (!(p->alpha_star > 0.0 && p->alpha_star < 1.0)) return fail(RMLT_E_INVALID_ARG, "alpha_star outside (0,1)");
    if (!(p->gamma_max >= 0.0 && p->gamma_scale >= 0.0)) return fail(RMLT_E_INVALID_ARG, "negative gamma");
    if (p->kernel != RMLT_KERNEL_KELEMEN && p->kernel != RMLT_KERNEL_TRUNCNORM)
        return fail(RMLT_E_INVALID_ARG, "unknown small-step kernel");
    // sigma s2 <= 1/2 for Kelemen; sigma <= 4 for the truncated normal
    const double lmax_ok = p->kernel == RMLT_KERNEL_TRUNCNORM ? 2.0 * std::log(4.0) : 2.0 * std::log(1.0 / (2.0 * p->s2));
    if (!(p->lambda_min >= -150.0 && p->lambda_min <= p->lambda_init && p->lambda_init <= p->lambda_max &&
          p->lambda_max <= lmax_ok + 1e-12))
        return fail(RMLT_E_INVALID_ARG, "need -150 <= lambda_min <= lambda_init <= lambda_max <= %g", lmax_ok);
    if (!(p->w_floor >= 0.0 && p->w_floor <= 1.0)) return fail(RMLT_E_INVALID_ARG, "w_floor outside [0,1]");
    if (p->partition != RMLT_PARTITION_GRID && p->partition != RMLT_PARTITION_QUADTREE)
        return fail(RMLT_E_INVALID_ARG, "unknown partition");
    if (p->dir_cells < 0 || p->dir_cells > 64) return fail(RMLT_E_INVALID_ARG, "dir_cells outside [0, 64]");
    if (p->dir_cells > 1) {
        if (p->partition != RMLT_PARTITION_GRID || p->target_mode != RMLT_TARGET_PLAIN || p->max_depth < 1 || c->S.toy ||
            p->p_mala > 0.0)
            return fail(RMLT_E_INVALID_ARG, "the 4-D partition needs the grid partition, the plain target, a scene "
                        "with max_depth >= 1 and no Langevin strategy");
        const int64_t m4 = (int64_t)((p->width + p->region_px - 1) / p->region_px) *
                           ((p->height + p->region_px - 1) / p->region_px) * p->dir_cells * p->dir_cells;
        if (m4 > (1 << 24)) return fail(RMLT_E_INVALID_ARG, "more than 2^24 regions");
    }
    if (!(p->p_mala >= 0.0 && p->p_mala <= 1.0 && p->p_large + p->p_mala <= 1.0))
        return fail(RMLT_E_INVALID_ARG, "p_mala outside [0, 1 - p_large]");
    if (p->p_mala > 0.0) {
        if (!(p->mala_tau > 0.0 && p->mala_tau <= 1.0 && p->mala_drift_max > 0.0 && p->mala_drift_max <= 0.5))
            return fail(RMLT_E_INVALID_ARG, "Langevin strategy: need 0 < mala_tau <= 1, 0 < mala_drift_max <= 1/2");
        if (!c->scene_lambert)
            return fail(RMLT_E_INVALID_ARG, "the Langevin strategy differentiates the path map: Lambertian scenes only");
    }
    if (p->chains_total > 0 && p->chains_total != p->n_chains && p->p_mala > 0.0)
        return fail(RMLT_E_INVALID_ARG, "the Langevin strategy is not available to a sharded population");
    if (p->partition == RMLT_PARTITION_QUADTREE) {
        if (p->target_mode != RMLT_TARGET_PLAIN) return fail(RMLT_E_INVALID_ARG, "the quadtree partition needs the plain target");
        if (p->qt_max_leaves < 1 || p->qt_max_leaves > (1 << 20) || p->qt_max_depth < 0 || p->qt_max_depth > 24 ||
            p->qt_split < 0 || p->qt_refine < 1)
            return fail(RMLT_E_INVALID_ARG, "quadtree limits: leaves in [1, 2^20], depth in [0, 24], split >= 0, refine >= 1");
    }
    return RMLT_OK;
}

// The parameters as the library uses them: lambda_max = 0 or NaN selects the
// largest value the kernel allows (Kelemen: sigma s2 <= 1/2, the largest
// offset on the torus; truncated normal: sigma <= 4), then every field is
// checked.
static rmlt_status resolve_params(const rmlt_ctx* c, const rmlt_chain_params* in, rmlt_chain_params* out)
{
    if (!in) return fail(RMLT_E_INVALID_ARG, "params is NULL");
    *out = *in;
    if (out->lambda_max == 0.0 || std::isnan(out->lambda_max)) {
        if (out->kernel == RMLT_KERNEL_TRUNCNORM) out->lambda_max = 2.0 * std::log(4.0);
        else if (out->s2 > 0.0 && out->s2 <= 0.5) out->lambda_max = 2.0 * std::log(1.0 / (2.0 * out->s2));
    }
    return check_params(c, out);
}

// Chain state and region tables for params P (no initial values), in a pool
// of their own; the context is not touched.
struct ChainAlloc {
    std::vector<Alloc> pool;
    DevChains Ch;
    double* d_total = nullptr;
    double* d_stage = nullptr;
};

static rmlt_status alloc_chains(rmlt_ctx* c, const rmlt_chain_params* p, ChainAlloc& A)
{
    DevChains Ch;
    Ch.C = p->n_chains;
    Ch.C_all = chains_all(p);
    Ch.chain0 = (uint32_t)p->chain_first;
    Ch.D = 2 + 5 * p->max_depth;
    Ch.W = p->width;
    Ch.H = p->height;
    Ch.region_px = p->region_px;
    Ch.nx = (p->width + p->region_px - 1) / p->region_px;
    Ch.m = Ch.nx * ((p->height + p->region_px - 1) / p->region_px);
    if (p->dir_cells > 1) {
        Ch.dcells = p->dir_cells;
        Ch.m *= p->dir_cells * p->dir_cells;
    }
    if (p->partition == RMLT_PARTITION_QUADTREE) {
        Ch.quadtree = 1;
        Ch.m = p->qt_max_leaves;          // capacity; the current count lives on the device
        Ch.qt_cap = p->qt_max_leaves;
        Ch.qt_max_depth = p->qt_max_depth;
        Ch.qt_split = p->qt_split;
    }
    Ch.max_depth = p->max_depth;
    Ch.E = p->epoch_len;
    Ch.L = p->L;
    Ch.weighted = p->target_mode == RMLT_TARGET_REGION_WEIGHTED;
    Ch.truncnorm = p->kernel == RMLT_KERNEL_TRUNCNORM ? 1 : 0;
    const size_t C = (size_t)Ch.C, m = (size_t)Ch.m, npx = (size_t)Ch.W * Ch.H * 3;
    rmlt_status st;
    auto& pool = A.pool;
    if ((st = c->alloc_n(pool, C * Ch.D, &Ch.q))) return st;
    Ch.qd = (int64_t)C;
    Ch.qc = 1;
    if ((st = c->alloc_n(pool, 3 * C, &Ch.f))) return st;
    if ((st = c->alloc_n(pool, C, &Ch.pi))) return st;
    if ((st = c->alloc_n(pool, C, &Ch.k))) return st;
    if ((st = c->alloc_n(pool, m, &Ch.lam))) return st;
    if ((st = c->alloc_n(pool, m, &Ch.n))) return st;
    if ((st = c->alloc_n(pool, m, &Ch.vis))) return st;
    if ((st = c->alloc_n(pool, m, &Ch.acc))) return st;
    if ((st = c->alloc_n(pool, m, &Ch.hist))) return st;
    if ((st = c->alloc_n(pool, m, &Ch.hprev))) return st;
    if ((st = c->alloc_n(pool, m, &Ch.w))) return st;
    if ((st = c->alloc_n(pool, m, &Ch.Rc))) return st;
    if ((st = c->alloc_n(pool, m, &Ch.sig))) return st;
    if ((st = c->alloc_n(pool, m, &Ch.wf))) return st;
    if ((st = c->alloc_n(pool, m, &Ch.Bk))) return st;
    if ((st = c->alloc_n(pool, 3 * m + 1, &Ch.snap))) return st;
    if ((st = c->alloc_n(pool, m, &Ch.snapB))) return st;
    if ((st = c->alloc_n(pool, 1, &Ch.large_all))) return st;
    if ((st = c->alloc_n(pool, npx, &Ch.img))) return st;
    if ((st = c->alloc_n(pool, (size_t)kStCount, &Ch.stats))) return st;
    if (!c->S.toy && (uint64_t)Ch.E * (uint64_t)Ch.C < (1ull << 32)) {
        const size_t ec = (size_t)Ch.E * C;
        if ((st = c->alloc_n(pool, 3 * ec, &Ch.lf))) return st;
        if ((st = c->alloc_n(pool, ec, &Ch.llist))) return st;
        if ((st = c->alloc_n(pool, 1, &Ch.lcount))) return st;
    }
    if ((st = c->alloc_n(pool, 1, &A.d_total))) return st;
    if ((st = c->alloc_n(pool, npx, &A.d_stage))) return st;
    if (Ch.quadtree) {
        const size_t nodes = (size_t)4 * Ch.qt_cap / 3 + 8;
        if ((st = c->alloc_n(pool, 4 * nodes, &Ch.qt_child))) return st;
        if ((st = c->alloc_n(pool, nodes, &Ch.qt_leaf))) return st;
        if ((st = c->alloc_n(pool, nodes, &Ch.qt_depth))) return st;
        if ((st = c->alloc_n(pool, 2, &Ch.qt_state))) return st;
    }
    if (p->p_mala > 0.0) {
        if ((st = c->alloc_n(pool, C * Ch.D, &Ch.G))) return st;
        double tm = std::ceil(p->p_mala * 16777216.0);
        Ch.T_mala = (uint32_t)(tm < 1 ? 1 : (tm > 16777216.0 ? 16777216.0 : tm));
        Ch.mala_tau = (float)p->mala_tau;
        Ch.mala_drift_max = (float)p->mala_drift_max;
    }
    Ch.seed_lo = (uint32_t)p->seed;
    Ch.seed_hi = (uint32_t)(p->seed >> 32);
    double tl = std::ceil(p->p_large * 16777216.0);
    Ch.T_large = (uint32_t)(tl < 0 ? 0 : (tl > 16777216.0 ? 16777216.0 : tl));
    Ch.S1 = (float)(p->s1 * 4294967296.0);
    Ch.S2 = (float)(p->s2 * 4294967296.0);
    Ch.log2_ratio = (float)std::log2(p->s2 / p->s1);
    Ch.alpha_star = p->alpha_star;
    Ch.gamma_max = p->gamma_max;
    Ch.gamma_scale = p->gamma_scale;
    Ch.lambda_min = p->lambda_min;
    Ch.lambda_max = p->lambda_max;
    Ch.w_floor = p->w_floor;
    A.Ch = Ch;
    return RMLT_OK;
}

// the scene as the chains of params p see it (the camera's aspect ratio)
static DevScene scene_for(const rmlt_ctx* c, const rmlt_chain_params* p)
{
    DevScene S = c->S;
    S.tan_y = (float)c->tan_half;
    S.tan_x = (float)(c->tan_half * (double)p->width / (double)p->height);
    return S;
}

// replace the context's chains with freshly set-up ones
static void adopt_chains(rmlt_ctx* c, ChainAlloc& A, const rmlt_chain_params* p)
{
    drop_chains(c);
    c->chain_mem = std::move(A.pool);
    c->Ch = A.Ch;
    c->d_total = A.d_total;
    c->d_stage = A.d_stage;
    c->P = *p;
    c->S = scene_for(c, p);
    c->since_refine = 0;
}

rmlt_status rmlt_init_chains(rmlt_ctx* c, const rmlt_chain_params* pin)
{
    rmlt_status st = enter(c);
    if (st) return st;
    if (!c->have_scene) return fail(RMLT_E_STATE, "load a scene before rmlt_init_chains");
    rmlt_chain_params P;
    if ((st = resolve_params(c, pin, &P))) return st;
    const rmlt_chain_params* p = &P;
    NvtxRange nv("rmlt_init_chains");
    // the new chains are set up completely before they replace the old ones
    ChainAlloc A;
    if ((st = alloc_chains(c, p, A))) {
        c->release(A.pool);
        return st;
    }
    DevChains& Ch = A.Ch;
    const DevScene S = scene_for(c, p);
    const size_t npx = (size_t)Ch.W * Ch.H * 3;
    // bootstrap with scratch buffers released afterwards: every context of a
    // sharded population draws all K C_all samples
    std::vector<Alloc> scratch;
    BootScratch B;
    const int64_t K = p->n_bootstrap / Ch.C_all;
    const int64_t nb = K * Ch.C_all;
    if ((st = c->alloc_n(scratch, (size_t)nb, &B.pi)) || (st = c->alloc_n(scratch, (size_t)nb * 3, &B.f)) ||
        (st = c->alloc_n(scratch, (size_t)Ch.C_all, &B.partial)) ||
        (st = c->alloc_n(scratch, (size_t)Ch.C_all + 1, &B.prefix))) {
        c->release(scratch);
        c->release(A.pool);
        return st;
    }
    B.total = A.d_total;
    B.overflow = Ch.stats + kStBootOverflow;
    cudaError_t e = cudaMemsetAsync(Ch.img, 0, npx * sizeof(double), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(Ch.stats, 0, kStCount * sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(Ch.large_all, 0, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = launch_fill_regions(Ch, p->lambda_init, c->stream);
    if (e == cudaSuccess) e = launch_bootstrap(S, Ch, nb, B, c->stream);
    if (e == cudaSuccess && Ch.G) e = launch_state_gradients(S, Ch, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->release(scratch);
    if (e != cudaSuccess) {
        c->release(A.pool);
        return cuda_fail(e, "bootstrap");
    }
    adopt_chains(c, A, p);
    c->n_boot = nb;
    c->mut = 0;
    c->epochs = 0;
    c->have_chains = true;
    c->failed = false;
    return RMLT_OK;
}

// One epoch's chain kernel (Alg. 1, mutation step for every chain).
static rmlt_status epoch_kernels(rmlt_ctx* c)
{
    const uint64_t E = (uint64_t)c->Ch.E;
    const uint32_t n_traced = (uint32_t)(((uint64_t)c->Ch.C + c->tr_stride - 1) / c->tr_stride);
    DevChains Ch = c->Ch;
    Ch.batch_shade = c->batch_shade;
    Ch.batch_setup = c->batch_setup;
    Ch.adaptive_batch = c->adaptive_batch;
    if (!c->large_ahead) Ch.lf = nullptr;
    const bool trace = c->tr != nullptr;
    if (trace) {
        Ch.trace = c->tr;
        Ch.trace_cap = c->tr_cap;
        Ch.trace_stride = c->tr_stride;
        Ch.trace_base = c->tr_epoch * (unsigned long long)n_traced * E;
        Ch.trace_words = c->tr_words;
    }
    const DevScene& S = c->S;
    rmlt_status st;
    if (c->wavefront && !c->W.s) {
        void* mem = nullptr;
        if ((st = c->dalloc(c->chain_mem, wf_bytes(Ch.C, Ch.D), &mem))) return st;
        wf_carve(mem, Ch.C, Ch.D, c->W);
    }
    cudaError_t err = cudaSuccess;
    if (Ch.lf) err = launch_large_steps(S, Ch, c->mut, c->stream);
    if (err == cudaSuccess) {
        if (c->wavefront) {
            c->W.refill = c->wf_refill;
            c->W.short_stack = (c->wf_flags & RMLT_WAVEFRONT_SHORT_STACK) != 0;
            c->W.leaf_batch = c->wf_leaf_batch;
            c->wf_ran = true;
            err = wf_epoch(&c->wg, S, Ch, c->W, c->mut, Ch.trace_base, trace, c->count_work, c->wf_trace_cps,
                           c->wf_setup_cps, (c->wf_flags & RMLT_WAVEFRONT_HOST_LOOP) != 0, c->wave_limit,
                           c->stream);
        } else {
            err = launch_chain_epoch(S, Ch, c->mut, trace, c->count_work, c->stream);
        }
    }
    if (err != cudaSuccess) {
        c->failed = true;
        return cuda_fail(err, "epoch launch");
    }
    return RMLT_OK;
}

// The epoch boundary (Alg. 1, region update), a due quadtree pass, the trace
// instrument's lambda record; the epoch is then complete.
static rmlt_status epoch_boundary(rmlt_ctx* c)
{
    const uint64_t E = (uint64_t)c->Ch.E;
    cudaError_t err = launch_region_update(c->Ch, false, c->stream);
    if (err == cudaSuccess && c->Ch.quadtree) {
        // M_refine counts the mutations of the whole population
        c->since_refine += (uint64_t)c->Ch.C_all * E;
        if (c->since_refine >= (uint64_t)c->P.qt_refine) {
            c->since_refine = 0;
            err = launch_quadtree_refine(c->Ch, c->stream);
        }
    }
    if (err != cudaSuccess) {
        c->failed = true;
        return cuda_fail(err, "region update");
    }
    const bool trace = c->tr != nullptr;
    if (trace && c->tr_lam && (c->tr_epoch + 1) * (uint64_t)c->Ch.m <= c->tr_lam_cap) {
        err = cudaMemcpyAsync(c->tr_lam + c->tr_epoch * (uint64_t)c->Ch.m, c->Ch.lam, sizeof(double) * c->Ch.m,
                              cudaMemcpyDeviceToDevice, c->stream);
        if (err != cudaSuccess) return cuda_fail(err, "trace lambda copy");
    }
    if (trace) c->tr_epoch++;
    c->mut += E;
    c->epochs++;
    return RMLT_OK;
}

static rmlt_status check_steppable(rmlt_ctx* c)
{
    if (!c->have_chains) return fail(RMLT_E_STATE, "rmlt_init_chains first");
    if (c->failed) return fail(RMLT_E_STATE, "context failed earlier: %s", g_err.c_str());
    if (c->Ch.T_mala && c->wavefront)
        return fail(RMLT_E_STATE, "the Langevin strategy runs in the chain kernel");
    return RMLT_OK;
}

rmlt_status rmlt_step(rmlt_ctx* c, uint64_t n_mutations)
{
    rmlt_status st = enter(c);
    if (st) return st;
    if ((st = check_steppable(c))) return st;
    if (c->Ch.C_all != c->Ch.C)
        return fail(RMLT_E_STATE, "a sharded context steps with rmlt_epoch_mutate / rmlt_epoch_update");
    if (c->in_epoch) return fail(RMLT_E_STATE, "rmlt_epoch_update is due first");
    const uint64_t E = (uint64_t)c->Ch.E;
    const uint64_t n_ep = (n_mutations + E - 1) / E;
    for (uint64_t e = 0; e < n_ep; ++e) {
        NvtxRange nv("rmlt epoch");
        if ((st = epoch_kernels(c))) return st;
        if ((st = epoch_boundary(c))) return st;
    }
    return RMLT_OK;
}

static rmlt_status check_device_buffer(const void* ptr, const char* what)
{
    cudaPointerAttributes at{};
    if (!ptr || cudaPointerGetAttributes(&at, ptr) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(RMLT_E_INVALID_ARG, "%s must be device memory", what);
    }
    return RMLT_OK;
}

rmlt_status rmlt_exchange_size(rmlt_ctx* c, int64_t* n_counts, int64_t* n_sums)
{
    if (!c || !n_counts || !n_sums) return fail(RMLT_E_INVALID_ARG, "null argument");
    if (!c->have_chains) return fail(RMLT_E_STATE, "rmlt_init_chains first");
    *n_counts = 3 * (int64_t)c->Ch.m + 1;
    *n_sums = (int64_t)c->Ch.m;
    return RMLT_OK;
}

rmlt_status rmlt_epoch_mutate(rmlt_ctx* c, uint64_t* counts, double* sums)
{
    rmlt_status st = enter(c);
    if (st) return st;
    if ((st = check_steppable(c))) return st;
    if (c->in_epoch) return fail(RMLT_E_STATE, "rmlt_epoch_update is due first");
    if (c->Ch.T_mala) return fail(RMLT_E_INVALID_ARG, "the Langevin strategy steps with rmlt_step only");
    if ((st = check_device_buffer(counts, "counts")) || (st = check_device_buffer(sums, "sums"))) return st;
    NvtxRange nv("rmlt_epoch_mutate");
    cudaError_t e = launch_epoch_snapshot(c->Ch, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "epoch snapshot");
    if ((st = epoch_kernels(c))) return st;
    e = launch_epoch_pack(c->Ch, (unsigned long long*)counts, sums, c->stream);
    if (e != cudaSuccess) {
        c->failed = true;
        return cuda_fail(e, "epoch pack");
    }
    c->in_epoch = true;
    return RMLT_OK;
}

rmlt_status rmlt_epoch_update(rmlt_ctx* c, const uint64_t* counts, const double* sums)
{
    rmlt_status st = enter(c);
    if (st) return st;
    if (!c->have_chains) return fail(RMLT_E_STATE, "rmlt_init_chains first");
    if (c->failed) return fail(RMLT_E_STATE, "context failed earlier: %s", g_err.c_str());
    if (!c->in_epoch) return fail(RMLT_E_STATE, "rmlt_epoch_mutate first");
    if ((st = check_device_buffer(counts, "counts")) || (st = check_device_buffer(sums, "sums"))) return st;
    NvtxRange nv("rmlt_epoch_update");
    cudaError_t e = launch_epoch_unpack(c->Ch, (const unsigned long long*)counts, sums, c->stream);
    if (e != cudaSuccess) {
        c->failed = true;
        return cuda_fail(e, "epoch unpack");
    }
    c->in_epoch = false;
    return epoch_boundary(c);
}

rmlt_status rmlt_set_trace(rmlt_ctx* c, rmlt_trace_record* records, uint64_t capacity, double* lambdas,
                           uint64_t lambda_capacity, uint32_t chain_stride)
{
    if (!c) return fail(RMLT_E_INVALID_ARG, "null context");
    if (records && chain_stride == 0) return fail(RMLT_E_INVALID_ARG, "chain_stride must be positive");
    c->tr = records;
    c->tr_cap = records ? capacity : 0;
    c->tr_lam = records ? lambdas : nullptr;
    c->tr_lam_cap = records ? lambda_capacity : 0;
    c->tr_stride = records ? chain_stride : 1;
    c->tr_epoch = 0;
    c->tr_words = nullptr;
    return RMLT_OK;
}

rmlt_status rmlt_set_trace_words(rmlt_ctx* c, uint32_t* words, uint64_t capacity_words)
{
    if (!c) return fail(RMLT_E_INVALID_ARG, "null context");
    if (!words) {
        c->tr_words = nullptr;
        return RMLT_OK;
    }
    if (!c->tr || !c->have_chains) return fail(RMLT_E_STATE, "set the trace instrument (rmlt_set_trace) first");
    if (capacity_words < c->tr_cap * (uint64_t)c->Ch.D)
        return fail(RMLT_E_INVALID_ARG, "room for %llu words needed (capacity x D)",
                    (unsigned long long)(c->tr_cap * (uint64_t)c->Ch.D));
    c->tr_words = words;
    return RMLT_OK;
}

rmlt_status rmlt_read_image(rmlt_ctx* c, double* out, int normalized)
{
    rmlt_status st = enter(c);
    if (st) return st;
    if (!out) return fail(RMLT_E_INVALID_ARG, "out is NULL");
    if (!c->have_chains || c->failed) return fail(RMLT_E_STATE, "no valid chains");
    if (c->in_epoch) return fail(RMLT_E_STATE, "rmlt_epoch_update is due first");
    // mutations of the whole population (a sharded context returns its share)
    const double n_total = (double)c->mut * (double)c->Ch.C_all;
    CK(launch_read_image(c->Ch, c->d_total, c->n_boot, n_total, normalized, c->d_stage, c->stream), "read image");
    if ((st = copy_out(c, out, c->d_stage, sizeof(double) * 3 * (size_t)c->Ch.W * c->Ch.H))) return st;
    return sync(c, "read image");
}

// the current number of regions (grows with a quadtree partition)
static rmlt_status current_regions(rmlt_ctx* c, int* m)
{
    *m = c->Ch.m;
    if (!c->Ch.quadtree) return RMLT_OK;
    int32_t s[2];
    CK(cudaMemcpyAsync(s, c->Ch.qt_state, sizeof s, cudaMemcpyDeviceToHost, c->stream), "read leaf count");
    rmlt_status st = sync(c, "read leaf count");
    if (st) return st;
    *m = s[0];
    return RMLT_OK;
}

rmlt_status rmlt_read_quadtree(rmlt_ctx* c, int32_t* child, int32_t* leaf, int32_t* depth, int32_t cap_nodes,
                               int32_t* n_nodes)
{
    rmlt_status st = enter(c);
    if (st) return st;
    if (!c->have_chains || c->failed) return fail(RMLT_E_STATE, "no valid chains");
    if (!c->Ch.quadtree) return fail(RMLT_E_STATE, "the partition is a grid");
    int32_t s[2];
    CK(cudaMemcpyAsync(s, c->Ch.qt_state, sizeof s, cudaMemcpyDeviceToHost, c->stream), "read tree size");
    if ((st = sync(c, "read tree size"))) return st;
    if (n_nodes) *n_nodes = s[1];
    const size_t n = (size_t)std::min(s[1], cap_nodes);
    if ((st = copy_out(c, child, c->Ch.qt_child, n * 16)) || (st = copy_out(c, leaf, c->Ch.qt_leaf, n * 4)) ||
        (st = copy_out(c, depth, c->Ch.qt_depth, n * 4)))
        return st;
    return sync(c, "read tree");
}

rmlt_status rmlt_read_region_hist(rmlt_ctx* c, uint64_t* out)
{
    rmlt_status st = enter(c);
    if (st) return st;
    if (!out) return fail(RMLT_E_INVALID_ARG, "out is NULL");
    if (!c->have_chains || c->failed) return fail(RMLT_E_STATE, "no valid chains");
    int m;
    if ((st = current_regions(c, &m))) return st;
    if ((st = copy_out(c, out, c->Ch.hist, sizeof(uint64_t) * m))) return st;
    return sync(c, "read hist");
}

rmlt_status rmlt_read_region_params(rmlt_ctx* c, double* lambda, int64_t* n, uint64_t* i, uint64_t* A, double* w)
{
    rmlt_status st = enter(c);
    if (st) return st;
    if (!c->have_chains || c->failed) return fail(RMLT_E_STATE, "no valid chains");
    int mi;
    if ((st = current_regions(c, &mi))) return st;
    const size_t m = (size_t)mi;
    if ((st = copy_out(c, lambda, c->Ch.lam, m * 8)) || (st = copy_out(c, n, c->Ch.n, m * 8)) ||
        (st = copy_out(c, i, c->Ch.vis, m * 8)) || (st = copy_out(c, A, c->Ch.acc, m * 8)) ||
        (st = copy_out(c, w, c->Ch.w, m * 8)))
        return st;
    return sync(c, "read region params");
}

rmlt_status rmlt_read_chain_state(rmlt_ctx* c, uint32_t* q, float* f, int32_t* k)
{
    rmlt_status st = enter(c);
    if (st) return st;
    if (!c->have_chains || c->failed) return fail(RMLT_E_STATE, "no valid chains");
    const size_t C = (size_t)c->Ch.C;
    if ((st = copy_out(c, q, c->Ch.q, C * c->Ch.D * 4)) || (st = copy_out(c, f, c->Ch.f, C * 3 * 4)) ||
        (st = copy_out(c, k, c->Ch.k, C * 4)))
        return st;
    return sync(c, "read chain state");
}

rmlt_status rmlt_read_stats(rmlt_ctx* c, rmlt_stats* out)
{
    rmlt_status st = enter(c);
    if (st) return st;
    if (!out) return fail(RMLT_E_INVALID_ARG, "out is NULL");
    if (!c->have_chains || c->failed) return fail(RMLT_E_STATE, "no valid chains");
    unsigned long long s[kStCount];
    double total = 0.0;
    CK(cudaMemcpyAsync(s, c->Ch.stats, sizeof s, cudaMemcpyDeviceToHost, c->stream), "read stats");
    CK(cudaMemcpyAsync(&total, c->d_total, sizeof total, cudaMemcpyDeviceToHost, c->stream), "read total");
    if ((st = sync(c, "read stats"))) return st;
    std::memset(out, 0, sizeof *out);
    out->mutations = c->mut;
    out->accepted = s[kStAccepted];
    out->large = s[kStLarge];
    out->small = s[kStSmall];
    out->early_reject = s[kStEarly];
    out->invalid_paths = s[kStInvalid];
    out->rays = s[kStRays];
    out->stack_overflow = s[kStOverflow];
    out->epochs = c->epochs;
    out->bhat = total / (double)c->n_boot;
    int mcur;
    if ((st = current_regions(c, &mcur))) return st;
    out->n_regions = mcur;
    out->dims = c->Ch.D;
    out->node_visits = s[kStNodes];
    out->tri_tests = s[kStTris];
    for (int i = 0; i < 6; ++i) out->sched[i] = s[kStIters + i];
    for (int i = 0; i < 5; ++i) out->cycles[i] = s[kStCycTrav + i];
    out->waves = s[kStWaves];
    out->wave_limit_hits = s[kStWaveLimit];
    out->mala = s[kStMala];
    out->mala_accepted = s[kStMalaAcc];
    out->boot_overflow = s[kStBootOverflow];
    out->node_bytes = c->have_scene && !c->S.brute && !c->S.toy ? 16u * (uint32_t)node_float4s(c->S.node_fmt) : 0u;
    return RMLT_OK;
}

rmlt_status rmlt_read_params(rmlt_ctx* c, rmlt_chain_params* out)
{
    if (!c || !out) return fail(RMLT_E_INVALID_ARG, "null argument");
    if (!c->have_chains) return fail(RMLT_E_STATE, "no chains");
    *out = c->P;
    return RMLT_OK;
}

rmlt_status rmlt_set_node_format(rmlt_ctx* c, int format)
{
    if (!c) return fail(RMLT_E_INVALID_ARG, "null context");
    if (format != RMLT_NODES_AUTO && format != RMLT_NODES_FLOAT && format != RMLT_NODES_QUANTISED)
        return fail(RMLT_E_INVALID_ARG, "node format must be RMLT_NODES_AUTO, _FLOAT or _QUANTISED");
    c->node_format = format;
    return RMLT_OK;
}

rmlt_status rmlt_set_trace_leaf_batch(rmlt_ctx* c, int leaf_batch)
{
    if (!c) return fail(RMLT_E_INVALID_ARG, "null context");
    if (leaf_batch < 1 || leaf_batch > 32) return fail(RMLT_E_INVALID_ARG, "leaf_batch must be in 1..32");
    c->wf_leaf_batch = leaf_batch;
    return RMLT_OK;
}

rmlt_status rmlt_set_wave_limit(rmlt_ctx* c, uint32_t waves)
{
    if (!c) return fail(RMLT_E_INVALID_ARG, "null context");
    c->wave_limit = waves;
    return RMLT_OK;
}

rmlt_status rmlt_set_tuning(rmlt_ctx* c, int batch_shade, int batch_setup, int flags)
{
    if (!c) return fail(RMLT_E_INVALID_ARG, "null context");
    if (batch_shade < 1 || batch_shade > 32 || batch_setup < 1 || batch_setup > 32)
        return fail(RMLT_E_INVALID_ARG, "batch sizes must be in 1..32");
    if (flags & ~(RMLT_TUNE_LARGE_AHEAD | RMLT_TUNE_ADAPTIVE_BATCH | RMLT_TUNE_WAVEFRONT))
        return fail(RMLT_E_INVALID_ARG, "unknown tuning flag");
    c->batch_shade = batch_shade;
    c->batch_setup = batch_setup;
    c->large_ahead = (flags & RMLT_TUNE_LARGE_AHEAD) != 0;
    c->adaptive_batch = (flags & RMLT_TUNE_ADAPTIVE_BATCH) != 0;
    c->wavefront = (flags & RMLT_TUNE_WAVEFRONT) != 0;
    return RMLT_OK;
}

rmlt_status rmlt_set_wavefront(rmlt_ctx* c, int trace_ctas_per_sm, int setup_ctas_per_sm, int refill_lanes,
                               int flags)
{
    if (!c) return fail(RMLT_E_INVALID_ARG, "null context");
    if (trace_ctas_per_sm < 0 || trace_ctas_per_sm > 32 || setup_ctas_per_sm < 0 || setup_ctas_per_sm > 32)
        return fail(RMLT_E_INVALID_ARG, "blocks per SM must be in 0..32");
    if (refill_lanes < 1 || refill_lanes > 32) return fail(RMLT_E_INVALID_ARG, "refill_lanes must be in 1..32");
    if (flags & ~(RMLT_WAVEFRONT_HOST_LOOP | RMLT_WAVEFRONT_SHORT_STACK))
        return fail(RMLT_E_INVALID_ARG, "unknown wavefront flag");
    c->wf_flags = flags;
    c->wf_trace_cps = trace_ctas_per_sm;
    c->wf_setup_cps = setup_ctas_per_sm;
    c->wf_refill = refill_lanes;
    return RMLT_OK;
}

rmlt_status rmlt_read_chain_grad(rmlt_ctx* c, float* g)
{
    rmlt_status st = enter(c);
    if (st) return st;
    if (!g) return fail(RMLT_E_INVALID_ARG, "g is NULL");
    if (!c->have_chains || !c->Ch.G) return fail(RMLT_E_STATE, "no chains with the Langevin strategy");
    CK(cudaMemcpyAsync(g, c->Ch.G, sizeof(float) * (size_t)c->Ch.D * c->Ch.C, cudaMemcpyDefault, c->stream),
       "read gradients");
    return sync(c, "read gradients");
}

rmlt_status rmlt_path_grad(rmlt_ctx* c, const uint32_t* q, int64_t n, float* f, float* logpi, float* grad)
{
    rmlt_status st = enter(c);
    if (st) return st;
    if (!c->have_chains) return fail(RMLT_E_STATE, "rmlt_init_chains first (it fixes depth and image size)");
    if (!c->scene_lambert) return fail(RMLT_E_INVALID_ARG, "the gradient covers Lambertian scenes only");
    if (n < 0 || n > (1ll << 31)) return fail(RMLT_E_INVALID_ARG, "n outside [0, 2^31]");
    if (!q) return fail(RMLT_E_INVALID_ARG, "q is NULL");
    for (const void* ptr : {(const void*)q, (const void*)f, (const void*)logpi, (const void*)grad}) {
        if (!ptr) continue;
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
            cudaGetLastError();
            return fail(RMLT_E_INVALID_ARG, "q and the outputs must be device pointers");
        }
    }
    CK(launch_path_grad(c->S, c->Ch, q, n, f, logpi, grad, c->stream), "rmlt_path_grad");
    return RMLT_OK;
}

rmlt_status rmlt_record_paths(rmlt_ctx* c, const uint32_t* q, int64_t n, float* rays, uint32_t* work)
{
    rmlt_status st = enter(c);
    if (st) return st;
    if (!c->have_chains) return fail(RMLT_E_STATE, "rmlt_init_chains first (it fixes depth and image size)");
    if (c->S.toy) return fail(RMLT_E_STATE, "the toy integrand casts no rays");
    if (n < 0 || n > (1ll << 24)) return fail(RMLT_E_INVALID_ARG, "n outside [0, 2^24]");
    if ((st = check_device_buffer(q, "q")) || (st = check_device_buffer(rays, "rays")) ||
        (st = check_device_buffer(work, "work")))
        return st;
    CK(launch_record_paths(c->S, c->Ch, q, n, rays, work, c->stream), "rmlt_record_paths");
    return RMLT_OK;
}

rmlt_status rmlt_walk_rays_host(rmlt_ctx* c, const float* rays, int64_t n, uint32_t* out)
{
    if (!c || !rays || !out) return fail(RMLT_E_INVALID_ARG, "null argument");
    if (!c->have_scene || c->S.toy) return fail(RMLT_E_STATE, "load a scene first");
    if (n < 0) return fail(RMLT_E_INVALID_ARG, "negative n");
    const bool brute = c->S.brute != 0;
    for (int64_t i = 0; i < n; ++i) {
        const float* r = rays + 8 * i;
        uint32_t* o = out + 4 * i;
        if (!(r[3] >= 0.0f)) {   // an unused slot
            o[0] = 0xFFFFFFFFu;
            o[1] = o[2] = o[3] = 0u;
            continue;
        }
        const WalkResult w = walk_ray(c->h_nodes, c->h_fmt, c->h_tris, brute, r);
        const float tf = (float)w.t;
        o[0] = w.tri >= 0 ? (uint32_t)w.tri : 0xFFFFFFFFu;
        std::memcpy(&o[1], &tf, 4);
        o[2] = w.nodes;
        o[3] = w.tris;
    }
    return RMLT_OK;
}

rmlt_status rmlt_set_work_counters(rmlt_ctx* c, int enable)
{
    if (!c) return fail(RMLT_E_INVALID_ARG, "null context");
    c->count_work = enable != 0;
    return RMLT_OK;
}

rmlt_status rmlt_bootstrap_noalloc(rmlt_ctx* c, const rmlt_chain_params* pin, uint32_t* out_q, float* out_f,
                                   double* out_bhat)
{
    rmlt_status st = enter(c);
    if (st) return st;
    if (!c->have_scene) return fail(RMLT_E_STATE, "load a scene before rmlt_bootstrap_noalloc");
    rmlt_chain_params P;
    if ((st = resolve_params(c, pin, &P))) return st;
    const rmlt_chain_params* p = &P;
    if (!out_q || !out_f || !out_bhat) return fail(RMLT_E_INVALID_ARG, "output pointers must not be NULL");
    for (const void* ptr : {(const void*)out_q, (const void*)out_f}) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
            cudaGetLastError();
            return fail(RMLT_E_INVALID_ARG, "out_q and out_f must be device memory");
        }
    }
    const int32_t C_all = chains_all(p);
    const int64_t K = p->n_bootstrap / C_all;
    const int64_t nb = K * C_all;
    const int nx = (p->width + p->region_px - 1) / p->region_px;
    const int64_t m = (int64_t)nx * ((p->height + p->region_px - 1) / p->region_px);
    if (nb > RMLT_NOALLOC_MAX_SAMPLES || C_all > RMLT_NOALLOC_MAX_CHAINS || m > RMLT_NOALLOC_MAX_REGIONS)
        return fail(RMLT_E_INVALID_ARG, "sizes above the fixed scratch: %lld samples (max %d), %d chains (max %d), "
                    "%lld regions (max %d)", (long long)nb, RMLT_NOALLOC_MAX_SAMPLES, C_all,
                    RMLT_NOALLOC_MAX_CHAINS, (long long)m, RMLT_NOALLOC_MAX_REGIONS);
    NoAllocScratch na;
    CK(noalloc_scratch(c->device, na), "scratch lookup");
    // the chain view the bootstrap kernels read: parameters of p, state
    // written to the caller's buffers, everything else in the fixed scratch
    DevChains Ch;
    Ch.C = p->n_chains;
    Ch.C_all = C_all;
    Ch.chain0 = (uint32_t)p->chain_first;
    Ch.D = 2 + 5 * p->max_depth;
    Ch.W = p->width;
    Ch.H = p->height;
    Ch.region_px = p->region_px;
    Ch.nx = nx;
    Ch.m = (int32_t)m;
    Ch.max_depth = p->max_depth;
    Ch.seed_lo = (uint32_t)p->seed;
    Ch.seed_hi = (uint32_t)(p->seed >> 32);
    Ch.q = out_q;
    Ch.qd = (int64_t)p->n_chains;
    Ch.qc = 1;
    Ch.f = out_f;
    Ch.pi = na.chain_pi;
    Ch.k = na.chain_k;
    Ch.Bk = na.Bk;
    const DevScene S = scene_for(c, p);
    // the array keeps the previous call's contents: the region sums and the
    // overflow count start at zero
    CK(cudaMemsetAsync(na.Bk, 0, sizeof(double) * (size_t)m, c->stream), "clear scratch");
    CK(cudaMemsetAsync(na.overflow, 0, sizeof(unsigned long long), c->stream), "clear scratch");
    CK(launch_bootstrap(S, Ch, nb, na.boot, c->stream), "bootstrap");
    double total = 0.0;
    unsigned long long overflow = 0;
    CK(cudaMemcpyAsync(&total, na.boot.total, sizeof total, cudaMemcpyDeviceToHost, c->stream), "read total");
    CK(cudaMemcpyAsync(&overflow, na.overflow, sizeof overflow, cudaMemcpyDeviceToHost, c->stream), "read overflow");
    CK(cudaStreamSynchronize(c->stream), "bootstrap");
    const double bhat = total / (double)nb;
    CK(cudaMemcpy(out_bhat, &bhat, sizeof bhat, cudaMemcpyDefault), "write bhat");
    if (overflow)
        return fail(RMLT_E_OVERFLOW, "%llu bootstrap path(s) overflowed the traversal stack (dropped; b and the "
                    "starting states are biased)", overflow);
    return RMLT_OK;
}

rmlt_status rmlt_memory_usage(rmlt_ctx* c, uint64_t* bytes)
{
    if (!c || !bytes) return fail(RMLT_E_INVALID_ARG, "null argument");
    *bytes = c->held;
    return RMLT_OK;
}

rmlt_status rmlt_synchronize(rmlt_ctx* c)
{
    rmlt_status st = enter(c);
    if (st) return st;
    return sync(c, "synchronize");
}

// ---------------------------------------------------------------------------
// checkpoint / resume
// ---------------------------------------------------------------------------
namespace {
struct CkptHeader {
    char magic[8];
    uint32_t abi, pad;
    uint64_t scene_hash;
    rmlt_chain_params P;
    uint64_t mut, epochs;
    int64_t n_boot;
    uint64_t since_refine;
    uint64_t payload_bytes;
    uint64_t checksum;        // FNV-1a (64 bit) of this header with checksum = 0, then the payload
};
constexpr char kCkptMagic[8] = {'R', 'M', 'L', 'T', 'C', 'K', 'P', '2'};

struct Field {
    void* dev;
    size_t bytes;
};

// the device arrays a checkpoint holds, in file order
std::vector<Field> fields(DevChains& Ch, double* d_total)
{
    const size_t C = (size_t)Ch.C, m = (size_t)Ch.m, npx = (size_t)Ch.W * Ch.H * 3;
    const size_t qn = Ch.quadtree ? (size_t)4 * Ch.qt_cap / 3 + 8 : 0;
    return {{Ch.q, C * Ch.D * 4}, {Ch.f, C * 12}, {Ch.pi, C * 4}, {Ch.k, C * 4},
            {Ch.lam, m * 8}, {Ch.n, m * 8}, {Ch.vis, m * 8}, {Ch.acc, m * 8}, {Ch.hist, m * 8},
            {Ch.hprev, m * 8}, {Ch.w, m * 8}, {Ch.Rc, m * 8}, {Ch.sig, m * 4}, {Ch.wf, m * 4},
            {Ch.Bk, m * 8}, {Ch.img, npx * 8}, {Ch.stats, kStCount * 8}, {d_total, 8}, {Ch.large_all, 8},
            {Ch.qt_child, qn * 16}, {Ch.qt_leaf, qn * 4}, {Ch.qt_depth, qn * 4},
            {Ch.qt_state, Ch.quadtree ? (size_t)8 : (size_t)0}};
}

// Every index a kernel takes from the checkpoint, checked on the host: the
// chains' regions and the quadtree (sizes, children below their parent,
// leaf ids, depths).
rmlt_status validate_payload(const DevChains& Ch, const std::vector<Field>& fl, const std::vector<unsigned char>& pay)
{
    std::vector<size_t> off(fl.size() + 1, 0);
    for (size_t i = 0; i < fl.size(); ++i) off[i + 1] = off[i] + fl[i].bytes;
    auto at = [&](int i) { return pay.data() + off[(size_t)i]; };
    int m_now = Ch.m;
    if (Ch.quadtree) {
        int32_t st[2];
        std::memcpy(st, at(22), sizeof st);
        const int32_t cap_nodes = 4 * Ch.qt_cap / 3 + 8;
        if (st[0] < 1 || st[0] > Ch.qt_cap || st[1] < 1 || st[1] > cap_nodes)
            return fail(RMLT_E_INVALID_ARG, "checkpoint: quadtree sizes out of range");
        const int32_t* child = (const int32_t*)at(19);
        const int32_t* leaf = (const int32_t*)at(20);
        const int32_t* depth = (const int32_t*)at(21);
        for (int32_t nd = 0; nd < st[1]; ++nd) {
            const bool is_leaf = child[4 * nd] < 0;
            for (int j = 0; j < 4; ++j) {
                const int32_t ch = child[4 * nd + j];
                if (is_leaf ? ch != -1 : (ch <= nd || ch >= st[1]))
                    return fail(RMLT_E_INVALID_ARG, "checkpoint: quadtree node %d has a bad child", nd);
            }
            if (is_leaf ? (leaf[nd] < 0 || leaf[nd] >= st[0]) : leaf[nd] != -1)
                return fail(RMLT_E_INVALID_ARG, "checkpoint: quadtree node %d has a bad leaf id", nd);
            if (depth[nd] < 0 || depth[nd] > Ch.qt_max_depth)
                return fail(RMLT_E_INVALID_ARG, "checkpoint: quadtree node %d has a bad depth", nd);
        }
        m_now = st[0];
    }
    const int32_t* k = (const int32_t*)at(3);
    for (int c = 0; c < Ch.C; ++c)
        if (k[c] < 0 || k[c] >= m_now) return fail(RMLT_E_INVALID_ARG, "checkpoint: chain %d has region %d", c, k[c]);
    return RMLT_OK;
}
}  // namespace

rmlt_status rmlt_save(rmlt_ctx* c, const char* path)
{
    rmlt_status st = enter(c);
    if (st) return st;
    if (!path) return fail(RMLT_E_INVALID_ARG, "path is NULL");
    if (!c->have_chains || c->failed) return fail(RMLT_E_STATE, "no valid chains");
    if (c->in_epoch) return fail(RMLT_E_STATE, "rmlt_epoch_update is due first");
    if ((st = sync(c, "save"))) return st;
    const std::vector<Field> fl = fields(c->Ch, c->d_total);
    size_t total = 0;
    for (const Field& f : fl) total += f.bytes;
    std::vector<unsigned char> pay(total);
    size_t o = 0;
    for (const Field& f : fl) {
        if (f.bytes && cudaMemcpy(pay.data() + o, f.dev, f.bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "save copy");
        o += f.bytes;
    }
    CkptHeader h{};
    std::memcpy(h.magic, kCkptMagic, 8);
    h.abi = RMLT_ABI_VERSION;
    h.scene_hash = c->scene_hash;
    h.P = c->P;
    h.mut = c->mut;
    h.epochs = c->epochs;
    h.n_boot = c->n_boot;
    h.since_refine = c->since_refine;
    h.payload_bytes = total;
    h.checksum = 0;
    h.checksum = fnv64(pay.data(), pay.size(), fnv64(&h, sizeof h, 1469598103934665603ull));
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(RMLT_E_IO, "cannot open %s for writing", path);
    bool ok = std::fwrite(&h, sizeof h, 1, fp) == 1 && std::fwrite(pay.data(), 1, pay.size(), fp) == pay.size();
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok) return fail(RMLT_E_IO, "write to %s failed", path);
    return RMLT_OK;
}

rmlt_status rmlt_restore(rmlt_ctx* c, const char* path)
{
    rmlt_status st = enter(c);
    if (st) return st;
    if (!path) return fail(RMLT_E_INVALID_ARG, "path is NULL");
    if (!c->have_scene) return fail(RMLT_E_STATE, "load the checkpoint's scene first");
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(RMLT_E_IO, "cannot open %s", path);
    CkptHeader h{};
    if (std::fread(&h, sizeof h, 1, fp) != 1) {
        std::fclose(fp);
        return fail(RMLT_E_IO, "truncated checkpoint %s (header)", path);
    }
    if (std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.abi != RMLT_ABI_VERSION) {
        std::fclose(fp);
        return fail(RMLT_E_INVALID_ARG, "%s is not a checkpoint of this library version", path);
    }
    if (h.payload_bytes > ((uint64_t)1 << 40)) {
        std::fclose(fp);
        return fail(RMLT_E_INVALID_ARG, "checkpoint %s: implausible payload size", path);
    }
    std::vector<unsigned char> pay((size_t)h.payload_bytes);
    const size_t got = std::fread(pay.data(), 1, pay.size(), fp);
    std::fclose(fp);
    if (got != pay.size()) return fail(RMLT_E_IO, "truncated checkpoint %s", path);
    CkptHeader hz = h;
    hz.checksum = 0;
    if (fnv64(pay.data(), pay.size(), fnv64(&hz, sizeof hz, 1469598103934665603ull)) != h.checksum)
        return fail(RMLT_E_INVALID_ARG, "checkpoint %s: checksum mismatch (corrupted file)", path);
    if (h.scene_hash != c->scene_hash) return fail(RMLT_E_INVALID_ARG, "checkpoint was taken on another scene");
    if ((st = check_params(c, &h.P))) return st;
    if (h.n_boot < (int64_t)chains_all(&h.P)) return fail(RMLT_E_INVALID_ARG, "checkpoint: bad bootstrap count");
    ChainAlloc A;
    if ((st = alloc_chains(c, &h.P, A))) {
        c->release(A.pool);
        return st;
    }
    const std::vector<Field> fl = fields(A.Ch, A.d_total);
    size_t total = 0;
    for (const Field& f : fl) total += f.bytes;
    if (total != pay.size()) {
        c->release(A.pool);
        return fail(RMLT_E_INVALID_ARG, "checkpoint %s: payload size does not match its parameters", path);
    }
    if ((st = validate_payload(A.Ch, fl, pay))) {
        c->release(A.pool);
        return st;
    }
    size_t o = 0;
    cudaError_t e = cudaSuccess;
    for (const Field& f : fl) {
        if (f.bytes && e == cudaSuccess) e = cudaMemcpy(f.dev, pay.data() + o, f.bytes, cudaMemcpyHostToDevice);
        o += f.bytes;
    }
    const DevScene S = scene_for(c, &h.P);
    // the regions follow from the states (validated above; recomputed so that
    // the two cannot disagree)
    if (e == cudaSuccess) e = launch_chain_regions(A.Ch, c->stream);
    // gradients of the restored states (not stored: a function of q)
    if (e == cudaSuccess && A.Ch.G) e = launch_state_gradients(S, A.Ch, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->release(A.pool);
        return cuda_fail(e, "restore");
    }
    adopt_chains(c, A, &h.P);
    c->mut = h.mut;
    c->epochs = h.epochs;
    c->n_boot = h.n_boot;
    c->since_refine = h.since_refine;
    c->have_chains = true;
    c->failed = false;
    return RMLT_OK;
}

// ---------------------------------------------------------------------------
// batched stepping of several contexts
// ---------------------------------------------------------------------------
}  // extern "C"

struct rmlt_batch {
    std::vector<rmlt_ctx*> m;
    std::vector<int> order;            // launch order of the members' blocks
    int device = 0;
    cudaStream_t stream = nullptr;     // the batch's own stream (capturable)
    cudaEvent_t ev = nullptr;
    std::vector<cudaStream_t> side;    // branch mode: one capture stream per member
    std::vector<cudaEvent_t> join;
    BatchMember* d_members = nullptr;
    int* d_block_member = nullptr;
    int n_blocks = 0;
    std::vector<int> nblk;             // blocks of each member
    bool table_dirty = true;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int mode = RMLT_BATCH_ONE_LAUNCH;
    int ctas_per_sm = 4;
    std::vector<unsigned char> graph_key;   // what the graph was captured with
    std::vector<BatchMember> h;

    void drop_graph()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        graph_key.clear();
    }
};

namespace {

rmlt_status batch_check_member(const rmlt_batch* b, const rmlt_ctx* c, int i)
{
    if (!c) return fail(RMLT_E_INVALID_ARG, "member %d is NULL", i);
    if (!c->have_chains) return fail(RMLT_E_STATE, "member %d: rmlt_init_chains first", i);
    if (c->failed) return fail(RMLT_E_STATE, "member %d failed earlier", i);
    if (c->device != b->device) return fail(RMLT_E_INVALID_ARG, "member %d is on another device", i);
    if (c->S.brute || c->S.toy)
        return fail(RMLT_E_INVALID_ARG, "member %d: batched members need a BVH scene (more than brute_force_max "
                    "triangles)", i);
    if (c->Ch.E != b->m[0]->Ch.E) return fail(RMLT_E_INVALID_ARG, "member %d: epoch_len differs from member 0", i);
    if (c->tr && b->mode != RMLT_BATCH_ONE_LAUNCH)
        return fail(RMLT_E_STATE, "member %d: the trace instrument needs the one-launch mode", i);
    if (c->wavefront) return fail(RMLT_E_STATE, "member %d: the wavefront form is set", i);
    if (c->Ch.T_mala) return fail(RMLT_E_STATE, "member %d: the Langevin strategy is set", i);
    if (c->Ch.dcells > 1) return fail(RMLT_E_STATE, "member %d: the 4-D partition is set", i);
    if (c->Ch.C_all != c->Ch.C) return fail(RMLT_E_STATE, "member %d is a shard of a larger population", i);
    if (c->in_epoch) return fail(RMLT_E_STATE, "member %d: rmlt_epoch_update is due", i);
    return RMLT_OK;
}

// one launch of the chain kernel over every member's blocks, then one launch
// of every member's region update; replayed once per epoch
cudaError_t capture_one_launch(rmlt_batch* b, bool count, bool trace)
{
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t e1 = launch_chain_epoch_batch(b->d_members, b->d_block_member, 0, b->n_blocks, count,
                                              b->ctas_per_sm, trace, b->stream);
    cudaError_t e2 = launch_region_update_batch(b->d_members, (int)b->m.size(), b->stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->stream, &g);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e);
    }
    b->graph = g;
    return cudaGraphInstantiate(&b->exec, g, 0);
}

// every member's n_ep epochs as its own branch of one graph (chain kernel,
// region update and, where due, the quadtree pass), so that members never
// wait for each other between epochs
cudaError_t capture_branches(rmlt_batch* b, bool count, uint64_t n_ep, const std::vector<unsigned char>& refine)
{
    const int n = (int)b->m.size();
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t err = cudaEventRecord(b->ev, b->stream);
    for (int k = 0; k < n && err == cudaSuccess; ++k) {
        const int i = b->order[(size_t)k];
        cudaStream_t s = b->side[(size_t)i];
        err = cudaStreamWaitEvent(s, b->ev, 0);
        for (uint64_t ep = 0; ep < n_ep && err == cudaSuccess; ++ep) {
            err = launch_chain_epoch_member(b->d_members + i, b->h[(size_t)i], count, s);
            if (err == cudaSuccess) err = launch_region_update_batch(b->d_members + i, 1, s);
            if (err == cudaSuccess && refine[(size_t)i * n_ep + ep]) err = launch_quadtree_refine(b->h[(size_t)i].Ch, s);
        }
        if (err == cudaSuccess) err = cudaEventRecord(b->join[(size_t)i], s);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(b->stream, b->join[(size_t)i], 0);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->stream, &g);
    if (err != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return err != cudaSuccess ? err : e;
    }
    b->graph = g;
    return cudaGraphInstantiate(&b->exec, g, 0);
}

}  // namespace

extern "C" {

rmlt_status rmlt_batch_create(rmlt_batch** out, rmlt_ctx* const* ctxs, int n)
{
    if (!out) return fail(RMLT_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!ctxs || n < 1) return fail(RMLT_E_INVALID_ARG, "need at least one member");
    rmlt_batch* b = new (std::nothrow) rmlt_batch();
    if (!b) return fail(RMLT_E_OOM, "batch");
    b->m.assign(ctxs, ctxs + n);
    b->device = ctxs[0] ? ctxs[0]->device : 0;
    for (int i = 0; i < n; ++i) {
        rmlt_status st = batch_check_member(b, ctxs[i], i);
        if (st) {
            delete b;
            return st;
        }
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) {
                delete b;
                return fail(RMLT_E_INVALID_ARG, "member %d repeats member %d", i, j);
            }
    }
    b->side.assign((size_t)n, nullptr);
    b->join.assign((size_t)n, nullptr);
    cudaError_t e = cudaSetDevice(b->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&b->side[(size_t)i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[(size_t)i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->d_members, sizeof(BatchMember) * (size_t)n);
    if (e != cudaSuccess) {
        rmlt_batch_destroy(b);
        return cuda_fail(e, "rmlt_batch_create");
    }
    b->order.resize((size_t)n);
    for (int i = 0; i < n; ++i) b->order[(size_t)i] = i;
    *out = b;
    return RMLT_OK;
}

rmlt_status rmlt_batch_set_order(rmlt_batch* b, const int* order)
{
    if (!b || !order) return fail(RMLT_E_INVALID_ARG, "NULL argument");
    const int n = (int)b->m.size();
    std::vector<int> seen((size_t)n, 0);
    for (int i = 0; i < n; ++i) {
        if (order[i] < 0 || order[i] >= n || seen[(size_t)order[i]]++)
            return fail(RMLT_E_INVALID_ARG, "order must be a permutation of 0..%d", n - 1);
    }
    b->order.assign(order, order + n);
    b->table_dirty = true;
    b->drop_graph();
    return RMLT_OK;
}

rmlt_status rmlt_batch_set_shape(rmlt_batch* b, int ctas_per_sm, int mode)
{
    if (!b) return fail(RMLT_E_INVALID_ARG, "null batch");
    if (ctas_per_sm != 3 && ctas_per_sm != 4) return fail(RMLT_E_INVALID_ARG, "ctas_per_sm must be 3 or 4");
    if (mode != RMLT_BATCH_ONE_LAUNCH && mode != RMLT_BATCH_BRANCHES)
        return fail(RMLT_E_INVALID_ARG, "unknown batch mode");
    if (ctas_per_sm != b->ctas_per_sm || mode != b->mode) b->drop_graph();
    b->ctas_per_sm = ctas_per_sm;
    b->mode = mode;
    return RMLT_OK;
}

rmlt_status rmlt_batch_step(rmlt_batch* b, uint64_t n_mutations)
{
    if (!b) return fail(RMLT_E_INVALID_ARG, "null batch");
    CK(cudaSetDevice(b->device), "cudaSetDevice");
    const int n = (int)b->m.size();
    for (int i = 0; i < n; ++i) {
        rmlt_status st = batch_check_member(b, b->m[(size_t)i], i);
        if (st) return st;
    }
    // block table: member order[0]'s blocks first, and so on
    b->h.assign((size_t)n, BatchMember());
    b->nblk.assign((size_t)n, 0);
    int blocks = 0;
    std::vector<int> table;
    for (int k = 0; k < n; ++k) {
        const int i = b->order[(size_t)k];
        rmlt_ctx* c = b->m[(size_t)i];
        BatchMember& bm = b->h[(size_t)i];
        bm.S = c->S;
        bm.Ch = c->Ch;
        bm.Ch.batch_shade = c->batch_shade;
        bm.Ch.batch_setup = c->batch_setup;
        bm.Ch.adaptive_batch = c->adaptive_batch;
        bm.Ch.lf = nullptr;
        bm.mut0 = c->mut;
        bm.block0 = blocks;
        if (c->tr) {
            bm.Ch.trace = c->tr;
            bm.Ch.trace_cap = c->tr_cap;
            bm.Ch.trace_stride = c->tr_stride;
            bm.Ch.trace_words = c->tr_words;
            bm.trace_mut0 = c->mut - c->tr_epoch * (uint64_t)c->Ch.E;
            bm.tr_lam = c->tr_lam;
            bm.tr_lam_cap = c->tr_lam_cap;
        }
        const int nb = (c->Ch.C + kChainBlock - 1) / kChainBlock;
        b->nblk[(size_t)i] = nb;
        table.insert(table.end(), (size_t)nb, i);
        blocks += nb;
    }
    if (b->table_dirty || blocks != b->n_blocks) {
        if (b->d_block_member) cudaFree(b->d_block_member);
        b->d_block_member = nullptr;
        CK(cudaMalloc(&b->d_block_member, sizeof(int) * (size_t)blocks), "batch block table");
        CK(cudaMemcpy(b->d_block_member, table.data(), sizeof(int) * (size_t)blocks, cudaMemcpyHostToDevice),
           "batch block table");
        b->n_blocks = blocks;
        b->table_dirty = false;
        b->drop_graph();
    }
    bool count = false, trace = false;
    for (rmlt_ctx* c : b->m) {
        count = count || c->count_work;
        trace = trace || c->tr != nullptr;
    }
    const uint64_t E = (uint64_t)b->m[0]->Ch.E;
    const uint64_t n_ep = (n_mutations + E - 1) / E;
    if (n_ep == 0) return RMLT_OK;
    // quadtree passes due after each epoch (the same rule as rmlt_step)
    std::vector<unsigned char> refine((size_t)n * n_ep, 0);
    std::vector<uint64_t> since((size_t)n, 0);
    for (int i = 0; i < n; ++i) {
        rmlt_ctx* c = b->m[(size_t)i];
        uint64_t s_ = c->since_refine;
        for (uint64_t ep = 0; ep < n_ep && c->Ch.quadtree; ++ep) {
            s_ += (uint64_t)c->Ch.C * E;
            if (s_ >= (uint64_t)c->P.qt_refine) {
                s_ = 0;
                refine[(size_t)i * n_ep + ep] = 1;
            }
        }
        since[(size_t)i] = s_;
    }
    // the graph holds device pointers, tuning and (branch mode) the epoch
    // count and quadtree schedule; rebuild it when any of them changed
    std::vector<unsigned char> key;
    for (const BatchMember& bm : b->h) {
        BatchMember k = bm;
        k.mut0 = 0;
        const unsigned char* p = (const unsigned char*)&k;
        key.insert(key.end(), p, p + sizeof k);
    }
    key.push_back(count ? 1 : 0);
    key.push_back(trace ? 1 : 0);
    key.push_back((unsigned char)b->mode);
    key.push_back((unsigned char)b->ctas_per_sm);
    if (b->mode == RMLT_BATCH_BRANCHES) {
        const unsigned char* p = (const unsigned char*)&n_ep;
        key.insert(key.end(), p, p + sizeof n_ep);
        key.insert(key.end(), refine.begin(), refine.end());
    }
    // the batch stream waits for every member's stream, and they for it afterwards
    for (rmlt_ctx* c : b->m) {
        CK(cudaEventRecord(b->ev, c->stream), "batch event");
        CK(cudaStreamWaitEvent(b->stream, b->ev, 0), "batch wait");
    }
    CK(cudaMemcpyAsync(b->d_members, b->h.data(), sizeof(BatchMember) * (size_t)n, cudaMemcpyHostToDevice,
                       b->stream), "batch member table");
    if (!b->exec || key != b->graph_key) {
        b->drop_graph();
        cudaError_t e = b->mode == RMLT_BATCH_BRANCHES ? capture_branches(b, count, n_ep, refine)
                                                       : capture_one_launch(b, count, trace);
        if (e != cudaSuccess) {
            b->drop_graph();
            return cuda_fail(e, "batch graph capture");
        }
        b->graph_key = key;
    }
    cudaError_t e = cudaSuccess;
    if (b->mode == RMLT_BATCH_BRANCHES) {
        e = cudaGraphLaunch(b->exec, b->stream);
    } else {
        for (uint64_t ep = 0; ep < n_ep && e == cudaSuccess; ++ep) {
            e = cudaGraphLaunch(b->exec, b->stream);
            for (int i = 0; i < n && e == cudaSuccess; ++i) {
                if (!refine[(size_t)i * n_ep + ep]) continue;
                e = launch_quadtree_refine(b->h[(size_t)i].Ch, b->stream);
                // the trace instrument records lambda after the whole epoch
                // boundary, as rmlt_step does: the split leaves' children too
                rmlt_ctx* c = b->m[(size_t)i];
                const uint64_t m = (uint64_t)c->Ch.m, te = c->tr_epoch + ep;
                if (e == cudaSuccess && c->tr && c->tr_lam && (te + 1) * m <= c->tr_lam_cap)
                    e = cudaMemcpyAsync(c->tr_lam + te * m, c->Ch.lam, sizeof(double) * m, cudaMemcpyDeviceToDevice,
                                        b->stream);
            }
        }
    }
    if (e != cudaSuccess) {
        for (rmlt_ctx* c : b->m) c->failed = true;
        return cuda_fail(e, "rmlt_batch_step launch");
    }
    for (int i = 0; i < n; ++i) {
        rmlt_ctx* c = b->m[(size_t)i];
        c->mut += n_ep * E;
        c->epochs += n_ep;
        c->since_refine = since[(size_t)i];
        if (c->tr) c->tr_epoch += n_ep;
    }
    CK(cudaEventRecord(b->ev, b->stream), "batch event");
    for (rmlt_ctx* c : b->m) CK(cudaStreamWaitEvent(c->stream, b->ev, 0), "batch wait");
    return RMLT_OK;
}

void rmlt_batch_destroy(rmlt_batch* b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    b->drop_graph();
    if (b->d_block_member) cudaFree(b->d_block_member);
    if (b->d_members) cudaFree(b->d_members);
    if (b->ev) cudaEventDestroy(b->ev);
    for (cudaEvent_t ev : b->join)
        if (ev) cudaEventDestroy(ev);
    for (cudaStream_t st : b->side)
        if (st) cudaStreamDestroy(st);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

void rmlt_destroy(rmlt_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    drop_chains(c);
    c->release(c->scene_mem);
    delete c;
}

}  // extern "C"

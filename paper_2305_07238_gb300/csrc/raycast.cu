// raycast.cu -- shading points from a ray caster (the stage that feeds the material system
// in the paper's renderer; Sec. 3.1 takes the UV, the material and the ray-cone gradients
// from it).  One thread per pixel casts one primary ray per pass against a small analytic
// scene (planes and spheres, held in the kernel's parameter space and read as broadcasts),
// and writes the hit as planes of the pass's shading-point SoA.
#include <cstdint>
#include <cstdio>

#include <cuda_runtime.h>

#include "pmc.h"

namespace pmc {
namespace {

constexpr float T_MIN = 1e-4f;
constexpr float COS_MIN = 1e-3f;     // |N . d| below this is clamped (grazing hits)
constexpr float CROSS_MIN = 1e-6f;   // |N x d| below this: head-on
constexpr unsigned long long GAMMA = 0x9E3779B97F4A7C15ull;

struct CastArgs {
    pmc_scene_object obj[PMC_MAX_SCENE_OBJECTS];
    uint32_t n_obj;
    pmc_camera cam;
    uint32_t row0;
    uint64_t n;          // points of this call: whole rows from row0
    uint64_t seed;
    uint32_t pass;
    pmc_ray_hits out;
};

// SplitMix64 (Steele, Lea & Flood 2014): output function of a state; the k-th output of
// the generator seeded with s is the output function of s + k * GAMMA.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct V3 {
    float x, y, z;
};
__device__ __forceinline__ V3 v3(float x, float y, float z) { return V3{x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ V3 operator*(float s, V3 a) { return v3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ V3 unit(V3 a) { return (1.0f / sqrtf(dot(a, a))) * a; }
__device__ __forceinline__ float axis(V3 a, uint32_t k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

__global__ void __launch_bounds__(256) k_cast(const __grid_constant__ CastArgs a) {
    const uint32_t W = a.cam.width, H = a.cam.height;
    const float th = a.cam.tan_half_y;
    const V3 eye = v3(a.cam.eye[0], a.cam.eye[1], a.cam.eye[2]);
    const V3 fwd = v3(a.cam.fwd[0], a.cam.fwd[1], a.cam.fwd[2]);
    const V3 right = v3(a.cam.right[0], a.cam.right[1], a.cam.right[2]);
    const V3 up = v3(a.cam.up[0], a.cam.up[1], a.cam.up[2]);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t pix = (uint64_t)a.row0 * W + i;
        const uint32_t x = (uint32_t)(pix % W), y = (uint32_t)(pix / W);
        // the sample inside the pixel: output k = pass * 2^32 + pixel + 1 of the stream
        const unsigned long long r = mix64(a.seed + (((unsigned long long)a.pass << 32) + pix + 1ull) * GAMMA);
        const float jx = (float)(uint32_t)(r >> 40) * 0x1p-24f;
        const float jy = (float)(uint32_t)((r >> 16) & 0xFFFFFFull) * 0x1p-24f;
        const float sx = (2.0f * ((float)x + jx) / (float)W - 1.0f) * th * ((float)W / (float)H);
        const float sy = (1.0f - 2.0f * ((float)y + jy) / (float)H) * th;
        const V3 d = unit(fwd + sx * right + sy * up);
        // closest hit (the first object on equal distances)
        float best = INFINITY;
        uint32_t hit = 0xFFFFFFFFu;
        for (uint32_t k = 0; k < a.n_obj; ++k) {
            const pmc_scene_object& o = a.obj[k];
            const V3 p = v3(o.p[0], o.p[1], o.p[2]);
            float t = INFINITY;
            if (o.kind == PMC_OBJ_PLANE) {
                const float tt = (o.p[3] - dot(p, eye)) / dot(p, d);
                if (tt > T_MIN) t = tt;
            } else {
                // discriminant as r^2 - |q|^2, q = oc - b d (Haines et al. 2019, "Precision
                // improvements for ray/sphere intersection"): no cancellation of b^2 against
                // |oc|^2 - r^2 in FP32
                const V3 oc = eye - p;
                const float b = dot(d, oc);
                const V3 q = oc - b * d;
                const float disc = o.p[3] * o.p[3] - dot(q, q);
                if (disc >= 0.0f) {
                    const float s = sqrtf(disc);
                    const float t0 = -b - s, t1 = -b + s;
                    t = t0 > T_MIN ? t0 : (t1 > T_MIN ? t1 : INFINITY);
                }
            }
            if (t < best) {
                best = t;
                hit = k;
            }
        }
        pmc_ray_hits out = a.out;
        if (hit == 0xFFFFFFFFu) {   // nothing hit: an open scene; the pass reports the point
            out.u[i] = 0.0f; out.v[i] = 0.0f; out.mat[i] = 0xFFFFFFFFu;
            out.px[i] = eye.x; out.py[i] = eye.y; out.pz[i] = eye.z;
            out.nx[i] = 0.0f; out.ny[i] = 0.0f; out.nz[i] = 0.0f;
            out.g1u[i] = 0.0f; out.g1v[i] = 0.0f; out.g2u[i] = 0.0f; out.g2v[i] = 0.0f;
            continue;
        }
        const pmc_scene_object& o = a.obj[hit];
        const V3 P = eye + best * d;
        const V3 N = o.kind == PMC_OBJ_PLANE ? v3(o.p[0], o.p[1], o.p[2])
                                             : (1.0f / o.p[3]) * (P - v3(o.p[0], o.p[1], o.p[2]));
        const uint32_t a0 = o.axes & 0xFFu, a1 = o.axes >> 8;
        const float s = o.uv_scale;
        const float uu = s * axis(P, a0), vv = s * axis(P, a1);
        // ray-cone footprint (Sec. 3.1): width = spread angle x distance; minor axis along
        // N x d, major axis along the tangent part of d, stretched by 1 / |N . d|
        const float width = best * (2.0f * th / (float)H);
        const float ndotd = dot(N, d);
        const float cosv = fmaxf(fabsf(ndotd), COS_MIN);
        V3 m1 = cross(N, d), m2;
        if (sqrtf(dot(m1, m1)) < CROSS_MIN) {
            const V3 helper = fabsf(N.x) < 0.9f ? v3(1.0f, 0.0f, 0.0f) : v3(0.0f, 1.0f, 0.0f);
            m1 = unit(cross(N, helper));
            m2 = unit(cross(N, m1));
        } else {
            m1 = unit(m1);
            m2 = unit(d - ndotd * N);
        }
        const V3 A1 = width * m1, A2 = (width / cosv) * m2;
        out.u[i] = uu - floorf(uu);
        out.v[i] = vv - floorf(vv);
        out.mat[i] = o.mat;
        out.px[i] = P.x; out.py[i] = P.y; out.pz[i] = P.z;
        out.nx[i] = N.x; out.ny[i] = N.y; out.nz[i] = N.z;
        out.g1u[i] = s * axis(A1, a0); out.g1v[i] = s * axis(A1, a1);
        out.g2u[i] = s * axis(A2, a0); out.g2v[i] = s * axis(A2, a1);
    }
}

}  // namespace
}  // namespace pmc

extern "C" pmc_status pmc_cast_rays(const pmc_scene_object* objects, uint32_t n_objects, const pmc_camera* cam,
                                    uint32_t row0, uint32_t row1, uint64_t seed, uint32_t pass,
                                    const pmc_ray_hits* out, void* stream) {
    using namespace pmc;
    if (!objects || !cam || !out || n_objects == 0 || n_objects > PMC_MAX_SCENE_OBJECTS) return PMC_ERR_INVALID_ARG;
    if (cam->width == 0 || cam->height == 0 || row0 > row1 || row1 > cam->height) return PMC_ERR_INVALID_ARG;
    const uint64_t n = (uint64_t)(row1 - row0) * cam->width;
    if (n > (1ull << 28)) return PMC_ERR_UNSUPPORTED;
    if (n && (!out->u || !out->v || !out->mat || !out->px || !out->py || !out->pz || !out->nx || !out->ny ||
              !out->nz || !out->g1u || !out->g1v || !out->g2u || !out->g2v))
        return PMC_ERR_INVALID_ARG;
    for (uint32_t k = 0; k < n_objects; ++k) {
        const pmc_scene_object& o = objects[k];
        if (o.kind > PMC_OBJ_SPHERE || (o.axes & 0xFFu) > 2 || (o.axes >> 8) > 2) return PMC_ERR_INVALID_ARG;
        if (o.kind == PMC_OBJ_SPHERE && !(o.p[3] > 0.0f)) return PMC_ERR_INVALID_ARG;
    }
    if (n == 0) return PMC_OK;
    CastArgs a{};
    for (uint32_t k = 0; k < n_objects; ++k) a.obj[k] = objects[k];
    a.n_obj = n_objects;
    a.cam = *cam;
    a.row0 = row0;
    a.n = n;
    a.seed = seed;
    a.pass = pass;
    a.out = *out;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t blocks_needed = (n + 255) / 256;
    const unsigned blocks = (unsigned)(blocks_needed < (uint64_t)sms * 16 ? blocks_needed : (uint64_t)sms * 16);
    k_cast<<<blocks, 256, 0, (cudaStream_t)stream>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "pmc: CUDA error %d (%s)\n", (int)e, cudaGetErrorString(e));
        return PMC_ERR_CUDA;
    }
    return PMC_OK;
}

// pathtracer_gpu.cu -- the seeded input generator's high-sample reference images on the GPU:
// the same procedural room (built on the host by synth_build_scene, passed in as a record),
// the same one-bounce estimator and the same counter-based random numbers as the host
// renderer pathtracer.c, one thread per pixel.  Input generation only; none of FLR's
// arithmetic.  Compiled without fused multiply-adds (-fmad=false) so that the ray
// arithmetic rounds as the host's does; the two renderers still differ where the device's
// cosf / sinf differ from the host's by an ulp and a grazing ray changes its hit.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "scene.h"

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// Uniform float in [0, 1) for (seed, pixel, sample, dim): the host renderer's hash.
__device__ __forceinline__ float urand(uint64_t seed, uint64_t pixel, uint64_t sample, uint64_t dim)
{
    uint64_t h = mix64(seed + 0x9e3779b97f4a7c15ULL);
    h = mix64(h ^ (pixel * 0xd1b54a32d192ed03ULL));
    h = mix64(h ^ (sample * 0xaef17502108ef2d9ULL));
    h = mix64(h ^ (dim * 0xf58cd3d3e1a5bb9bULL));
    return (float)(h >> 40) * (1.0f / 16777216.0f);
}

__device__ __forceinline__ vec3 v3(float x, float y, float z) { return vec3{x, y, z}; }
__device__ __forceinline__ vec3 vadd(vec3 a, vec3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ vec3 vsub(vec3 a, vec3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ vec3 vmul(vec3 a, float s) { return v3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float vdot(vec3 a, vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ vec3 vcross(vec3 a, vec3 b)
{
    return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ vec3 vnorm(vec3 a) { return vmul(a, 1.0f / sqrtf(vdot(a, a))); }

struct Hit {
    float t;
    vec3 n;
    const float *albedo;
    int is_light;
};

// Nearest hit along o + t d, t in (RAY_EPS, tmax): the room's walls (seen from inside), the
// light panel, the boxes and the spheres, as the host renderer tests them.
__device__ int intersect(const scene_t &s, vec3 o, vec3 d, float tmax, Hit *h)
{
    float best = tmax;
    int found = 0;
    {
        const float tx = d.x > 0 ? (ROOM_X - o.x) / d.x : (d.x < 0 ? -o.x / d.x : INFINITY);
        const float ty = d.y > 0 ? (ROOM_Y - o.y) / d.y : (d.y < 0 ? -o.y / d.y : INFINITY);
        const float tz = d.z > 0 ? (ROOM_Z - o.z) / d.z : (d.z < 0 ? -o.z / d.z : INFINITY);
        float t;
        vec3 n;
        const float *alb;
        if (tx <= ty && tx <= tz) {
            t = tx;
            n = v3(d.x > 0 ? -1.0f : 1.0f, 0, 0);
            alb = s.wall_albedo[d.x > 0 ? 1 : 0];
        } else if (ty <= tz) {
            t = ty;
            n = v3(0, d.y > 0 ? -1.0f : 1.0f, 0);
            alb = s.wall_albedo[d.y > 0 ? 3 : 2];
        } else {
            t = tz;
            n = v3(0, 0, d.z > 0 ? -1.0f : 1.0f);
            alb = s.wall_albedo[d.z > 0 ? 5 : 4];
        }
        if (t > RAY_EPS && t < best) {
            best = t;
            h->n = n;
            h->albedo = alb;
            h->is_light = 0;
            found = 1;
        }
    }
    if (d.y > 0) {  // light panel just below the ceiling, facing down
        const float t = (s.ly - o.y) / d.y;
        if (t > RAY_EPS && t < best) {
            const float x = o.x + t * d.x, z = o.z + t * d.z;
            if (x >= s.lx0 && x <= s.lx1 && z >= s.lz0 && z <= s.lz1) {
                best = t;
                h->n = v3(0, -1.0f, 0);
                h->albedo = s.wall_albedo[3];
                h->is_light = 1;
                found = 1;
            }
        }
    }
    for (int b = 0; b < N_BOXES; ++b) {
        const box_t &B = s.box[b];
        float t0 = -INFINITY, t1 = INFINITY;
        int axis = 0, miss = 0;
        const float ov[3] = {o.x, o.y, o.z}, dv[3] = {d.x, d.y, d.z};
        const float lo[3] = {B.lo.x, B.lo.y, B.lo.z}, hi[3] = {B.hi.x, B.hi.y, B.hi.z};
        for (int a = 0; a < 3; ++a) {
            if (dv[a] == 0.0f) {
                if (ov[a] < lo[a] || ov[a] > hi[a]) {
                    miss = 1;
                    break;
                }
                continue;
            }
            const float inv = 1.0f / dv[a];
            float ta = (lo[a] - ov[a]) * inv, tb = (hi[a] - ov[a]) * inv;
            if (ta > tb) {
                const float tt = ta;
                ta = tb;
                tb = tt;
            }
            if (ta > t0) {
                t0 = ta;
                axis = a;
            }
            if (tb < t1) t1 = tb;
        }
        if (miss || t0 > t1 || t0 <= RAY_EPS || t0 >= best) continue;
        best = t0;
        float nv[3] = {0, 0, 0};
        nv[axis] = dv[axis] > 0 ? -1.0f : 1.0f;
        h->n = v3(nv[0], nv[1], nv[2]);
        h->albedo = B.albedo;
        h->is_light = 0;
        found = 1;
    }
    for (int k = 0; k < N_SPHERES; ++k) {
        const sphere_t &S = s.sph[k];
        const vec3 oc = vsub(o, S.c);
        const float b = vdot(oc, d), c = vdot(oc, oc) - S.r * S.r;
        const float disc = b * b - c;
        if (disc < 0) continue;
        const float sq = sqrtf(disc);
        float t = -b - sq;
        if (t <= RAY_EPS) t = -b + sq;
        if (t <= RAY_EPS || t >= best) continue;
        best = t;
        h->n = vnorm(vadd(oc, vmul(d, t)));
        h->albedo = S.albedo;
        h->is_light = 0;
        found = 1;
    }
    h->t = best;
    return found;
}

// Cosine-distributed direction around n from two uniforms (Malley's method).
__device__ vec3 cosine_dir(vec3 n, float u1, float u2)
{
    const float rr = sqrtf(u1), phi = 2.0f * PI_F * u2;
    const float lx = rr * cosf(phi), ly = rr * sinf(phi), lz = sqrtf(fmaxf(0.0f, 1.0f - u1));
    const vec3 t = fabsf(n.x) > 0.5f ? v3(0, 1, 0) : v3(1, 0, 0);
    const vec3 b1 = vnorm(vcross(t, n));
    const vec3 b2 = vcross(n, b1);
    return vadd(vadd(vmul(b1, lx), vmul(b2, ly)), vmul(n, lz));
}

// One sample of demodulated one-bounce indirect radiance at primary hit (p, n): a cosine-
// sampled bounce, then next-event estimation of the area light at the secondary hit.
__device__ void indirect_sample(const scene_t &s, uint64_t seed, uint64_t pixel, uint64_t sample, vec3 p, vec3 n,
                                float out[3])
{
    out[0] = out[1] = out[2] = 0.0f;
    const vec3 d = cosine_dir(n, urand(seed, pixel, sample, 0), urand(seed, pixel, sample, 1));
    const vec3 o = vadd(p, vmul(n, RAY_EPS * 10));
    Hit h2;
    if (!intersect(s, o, d, INFINITY, &h2) || h2.is_light) return;
    const vec3 p2 = vadd(o, vmul(d, h2.t));
    vec3 n2 = h2.n;
    if (vdot(n2, d) > 0) n2 = vmul(n2, -1.0f);
    const float lx = s.lx0 + (s.lx1 - s.lx0) * urand(seed, pixel, sample, 2);
    const float lz = s.lz0 + (s.lz1 - s.lz0) * urand(seed, pixel, sample, 3);
    const vec3 lp = v3(lx, s.ly, lz);
    const vec3 o2 = vadd(p2, vmul(n2, RAY_EPS * 10));
    const vec3 toL = vsub(lp, o2);
    const float dist2 = vdot(toL, toL), dist = sqrtf(dist2);
    const vec3 wl = vmul(toL, 1.0f / dist);
    const float cos2 = vdot(n2, wl), cosl = wl.y;  // the light's normal is -y
    if (cos2 <= 0 || cosl <= 0) return;
    Hit hs;
    if (intersect(s, o2, wl, dist * (1.0f - 1e-4f), &hs)) return;
    const float area = (s.lx1 - s.lx0) * (s.lz1 - s.lz0);
    const float g = cos2 * cosl / dist2 * area / PI_F;
    for (int c = 0; c < 3; ++c) out[c] = h2.albedo[c] * s.le[c] * g;
}

// Reference of pixel (x, y): the mean of samples 1 .. spp (sample 0 is the noisy frame).
__global__ void reference_kernel(const __grid_constant__ scene_t s, uint64_t seed, int H, int W, int spp, float *ref)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W || y >= H) return;
    const size_t P = (size_t)H * W, p = (size_t)y * W + x;
    const float sx = (2.0f * (x + 0.5f) / W - 1.0f) * s.tan_half_fov * ((float)W / H);
    const float sy = (1.0f - 2.0f * (y + 0.5f) / H) * s.tan_half_fov;
    const vec3 d = vnorm(vadd(s.cam_fwd, vadd(vmul(s.cam_right, sx), vmul(s.cam_up, sy))));
    Hit h;
    if (!intersect(s, s.cam_pos, d, INFINITY, &h)) {  // cannot happen in a closed room
        h.t = 1.0f;
        h.n = v3(0, 1, 0);
    }
    const vec3 hp = vadd(s.cam_pos, vmul(d, h.t));
    vec3 n = h.n;
    if (vdot(n, d) > 0) n = vmul(n, -1.0f);
    double acc[3] = {0, 0, 0};
    for (int k = 1; k <= spp; ++k) {
        float v[3];
        indirect_sample(s, seed, (uint64_t)p, (uint64_t)k, hp, n, v);
        for (int c = 0; c < 3; ++c) acc[c] += v[c];
    }
    for (int c = 0; c < 3; ++c) ref[(size_t)c * P + p] = (float)(acc[c] / spp);
}

}  // namespace

// The reference [3][H][W] (device memory, float32) of the room given by `scene` (a scene_t
// from synth_build_scene, host memory, scene_bytes = sizeof(scene_t)) for `seed`: the mean
// of samples 1 .. spp of the host renderer's estimator.  Runs on `stream`; 0, or -1 for bad
// arguments, -2 for a CUDA error.
extern "C" int synth_reference_gpu(const void *scene, int scene_bytes, uint64_t seed, int H, int W, int spp,
                                   float *ref, void *stream)
{
    if (!scene || scene_bytes != (int)sizeof(scene_t) || H <= 0 || W <= 0 || spp <= 0 || !ref) return -1;
    scene_t s;
    std::memcpy(&s, scene, sizeof(s));
    const dim3 block(128), grid((W + 127) / 128, H);
    reference_kernel<<<grid, block, 0, (cudaStream_t)stream>>>(s, seed, H, W, spp, ref);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

/*
 * pathtracer.c -- seeded synthetic inputs for FLR: a procedural Lambertian room and a
 * one-bounce path tracer (CPU).
 *
 * This is an input generator only.  It contains none of FLR's arithmetic; the oracle
 * and the GPU library both consume its frames.
 *
 * Scene (one per seed): a closed room [0,8] x [0,4] x [0,8] (y up) whose six walls each
 * have their own albedo, 8 random axis-aligned boxes, 2 spheres and one rectangular
 * area light just below the ceiling.  Every albedo is drawn per object and per RGB
 * channel from U[0.1, 0.9].  A pinhole camera (60 degree vertical field of view) stands
 * inside the room.
 *
 * Per pixel, at the primary hit (pixel centre, no jitter, so guides are noise free):
 *   guide 0-2  albedo RGB
 *   guide 3-5  world-space normal xyz in [-1, 1]
 *   guide 6    camera-space depth / room diagonal, in (0, 1]
 *   guide 7    ambient occlusion: fraction of 64 cosine-distributed rays that travel
 *              2 scene units without a hit (cf. the AO guide of Sec. 4.1)
 * Radiance Y is the albedo-demodulated indirect light (Sec. 4.3 divides by albedo):
 * one cosine-sampled bounce from the primary hit, then next-event estimation of the
 * area light at the secondary hit (one light sample + one shadow ray).  Since the
 * cosine pdf cancels the cosine and 1/pi of the Lambertian integral, one sample of the
 * demodulated indirect radiance is the radiance leaving the secondary hit towards the
 * primary hit.  Rays that hit the light directly carry direct light, not indirect, and
 * contribute zero.  Nothing is clamped: the estimate has fireflies.
 *
 * Random numbers come from a counter-based hash of (seed, pixel, sample, dimension)
 * built on the SplitMix64 finaliser (Steele, Lea and Flood, OOPSLA 2014), so any pixel
 * and sample can be regenerated independently, in any order and on any thread.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "scene.h"

/* ---- counter-based random numbers ------------------------------------------------ */

static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Uniform float in [0, 1) for (seed, pixel, sample, dim). */
static float urand(uint64_t seed, uint64_t pixel, uint64_t sample, uint64_t dim)
{
    uint64_t h = mix64(seed + 0x9e3779b97f4a7c15ULL);
    h = mix64(h ^ (pixel * 0xd1b54a32d192ed03ULL));
    h = mix64(h ^ (sample * 0xaef17502108ef2d9ULL));
    h = mix64(h ^ (dim * 0xf58cd3d3e1a5bb9bULL));
    return (float)(h >> 40) * (1.0f / 16777216.0f);
}

#define SCENE_PIXEL 0xffffffffffffULL /* pixel index reserved for scene layout draws */

/* ---- scene --------------------------------------------------------------------------- */

static vec3 v3(float x, float y, float z) { vec3 v = {x, y, z}; return v; }
static vec3 vadd(vec3 a, vec3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
static vec3 vsub(vec3 a, vec3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
static vec3 vmul(vec3 a, float s) { return v3(a.x * s, a.y * s, a.z * s); }
static float vdot(vec3 a, vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static vec3 vcross(vec3 a, vec3 b)
{
    return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static vec3 vnorm(vec3 a) { return vmul(a, 1.0f / sqrtf(vdot(a, a))); }

typedef struct {
    float t;
    vec3 n;
    const float *albedo;
    int is_light;
} hit_t;

static int inside_any(const scene_t *s, vec3 p, float margin)
{
    for (int b = 0; b < N_BOXES; ++b) {
        const box_t *B = &s->box[b];
        if (p.x > B->lo.x - margin && p.x < B->hi.x + margin && p.y > B->lo.y - margin &&
            p.y < B->hi.y + margin && p.z > B->lo.z - margin && p.z < B->hi.z + margin)
            return 1;
    }
    for (int k = 0; k < N_SPHERES; ++k) {
        vec3 d = vsub(p, s->sph[k].c);
        float rr = s->sph[k].r + margin;
        if (vdot(d, d) < rr * rr) return 1;
    }
    return 0;
}

static void build_scene(uint64_t seed, scene_t *s)
{
    uint64_t k = 0;
#define U() urand(seed, SCENE_PIXEL, 0, k++)
#define UR(a, b) ((a) + ((b) - (a)) * U())
    for (int w = 0; w < 6; ++w)
        for (int c = 0; c < 3; ++c) s->wall_albedo[w][c] = UR(0.1f, 0.9f);
    for (int b = 0; b < N_BOXES; ++b) {
        box_t *B = &s->box[b];
        float sx = UR(0.5f, 2.0f), sy = UR(0.3f, 2.5f), sz = UR(0.5f, 2.0f);
        float x0 = UR(0.2f, ROOM_X - sx - 0.2f), z0 = UR(0.2f, ROOM_Z - sz - 0.2f);
        float y0 = 0.0f;
        if (U() > 0.7f) { /* floating box */
            float top = ROOM_Y - sy - 0.3f;
            y0 = top > 0.3f ? UR(0.3f, top) : 0.0f;
        }
        B->lo = v3(x0, y0, z0);
        B->hi = v3(x0 + sx, y0 + sy, z0 + sz);
        for (int c = 0; c < 3; ++c) B->albedo[c] = UR(0.1f, 0.9f);
    }
    for (int q = 0; q < N_SPHERES; ++q) {
        sphere_t *S = &s->sph[q];
        S->r = UR(0.35f, 0.9f);
        float cy = S->r;
        if (U() > 0.5f) cy = UR(S->r + 0.3f, ROOM_Y - S->r - 0.3f);
        S->c = v3(UR(S->r + 0.2f, ROOM_X - S->r - 0.2f), cy, UR(S->r + 0.2f, ROOM_Z - S->r - 0.2f));
        for (int c = 0; c < 3; ++c) S->albedo[c] = UR(0.1f, 0.9f);
    }
    {
        float lsx = UR(1.5f, 3.0f), lsz = UR(1.5f, 3.0f);
        s->lx0 = UR(0.5f, ROOM_X - lsx - 0.5f);
        s->lz0 = UR(0.5f, ROOM_Z - lsz - 0.5f);
        s->lx1 = s->lx0 + lsx;
        s->lz1 = s->lz0 + lsz;
        s->ly = ROOM_Y - 1e-3f;
        s->le[0] = 30.0f;
        s->le[1] = 27.5f;
        s->le[2] = 24.0f;
    }
    /* camera: inside the room, outside every object */
    vec3 pos = v3(1.0f, 1.6f, 1.0f);
    for (int tries = 0; tries < 200; ++tries) {
        vec3 p = v3(UR(0.8f, ROOM_X - 0.8f), UR(1.2f, 2.6f), UR(0.8f, ROOM_Z - 0.8f));
        if (!inside_any(s, p, 0.3f)) { pos = p; break; }
    }
    float yaw = UR(0.0f, 2.0f * PI_F);
    float pitch = UR(-0.45f, 0.1f);
#undef U
#undef UR
    s->cam_pos = pos;
    s->cam_fwd = vnorm(v3(cosf(pitch) * cosf(yaw), sinf(pitch), cosf(pitch) * sinf(yaw)));
    s->cam_right = vnorm(vcross(s->cam_fwd, v3(0.0f, 1.0f, 0.0f)));
    s->cam_up = vcross(s->cam_right, s->cam_fwd);
    s->tan_half_fov = tanf(0.5f * 60.0f * PI_F / 180.0f);
}

int synth_build_scene(uint64_t seed, scene_t *s)
{
    if (s) build_scene(seed, s);
    return (int)sizeof(scene_t);
}

/* ---- ray casting --------------------------------------------------------------------- */

static int intersect(const scene_t *s, vec3 o, vec3 d, float tmax, hit_t *h)
{
    float best = tmax;
    int found = 0;
    /* room walls, seen from inside */
    {
        float t;
        vec3 n;
        const float *alb;
        float tx = d.x > 0 ? (ROOM_X - o.x) / d.x : (d.x < 0 ? -o.x / d.x : INFINITY);
        float ty = d.y > 0 ? (ROOM_Y - o.y) / d.y : (d.y < 0 ? -o.y / d.y : INFINITY);
        float tz = d.z > 0 ? (ROOM_Z - o.z) / d.z : (d.z < 0 ? -o.z / d.z : INFINITY);
        if (tx <= ty && tx <= tz) {
            t = tx;
            n = v3(d.x > 0 ? -1.0f : 1.0f, 0, 0);
            alb = s->wall_albedo[d.x > 0 ? 1 : 0];
        } else if (ty <= tz) {
            t = ty;
            n = v3(0, d.y > 0 ? -1.0f : 1.0f, 0);
            alb = s->wall_albedo[d.y > 0 ? 3 : 2];
        } else {
            t = tz;
            n = v3(0, 0, d.z > 0 ? -1.0f : 1.0f);
            alb = s->wall_albedo[d.z > 0 ? 5 : 4];
        }
        if (t > RAY_EPS && t < best) {
            best = t;
            h->n = n;
            h->albedo = alb;
            h->is_light = 0;
            found = 1;
        }
    }
    /* light panel (just below the ceiling, facing down; albedo of the ceiling) */
    if (d.y > 0) {
        float t = (s->ly - o.y) / d.y;
        if (t > RAY_EPS && t < best) {
            float x = o.x + t * d.x, z = o.z + t * d.z;
            if (x >= s->lx0 && x <= s->lx1 && z >= s->lz0 && z <= s->lz1) {
                best = t;
                h->n = v3(0, -1.0f, 0);
                h->albedo = s->wall_albedo[3];
                h->is_light = 1;
                found = 1;
            }
        }
    }
    for (int b = 0; b < N_BOXES; ++b) {
        const box_t *B = &s->box[b];
        float t0 = -INFINITY, t1 = INFINITY;
        int axis = 0;
        float ov[3] = {o.x, o.y, o.z}, dv[3] = {d.x, d.y, d.z};
        float lo[3] = {B->lo.x, B->lo.y, B->lo.z}, hi[3] = {B->hi.x, B->hi.y, B->hi.z};
        int miss = 0;
        for (int a = 0; a < 3; ++a) {
            if (dv[a] == 0.0f) {
                if (ov[a] < lo[a] || ov[a] > hi[a]) { miss = 1; break; }
                continue;
            }
            float inv = 1.0f / dv[a];
            float ta = (lo[a] - ov[a]) * inv, tb = (hi[a] - ov[a]) * inv;
            if (ta > tb) { float tt = ta; ta = tb; tb = tt; }
            if (ta > t0) { t0 = ta; axis = a; }
            if (tb < t1) t1 = tb;
        }
        if (miss || t0 > t1 || t0 <= RAY_EPS || t0 >= best) continue;
        best = t0;
        float nv[3] = {0, 0, 0};
        nv[axis] = dv[axis] > 0 ? -1.0f : 1.0f;
        h->n = v3(nv[0], nv[1], nv[2]);
        h->albedo = B->albedo;
        h->is_light = 0;
        found = 1;
    }
    for (int k = 0; k < N_SPHERES; ++k) {
        const sphere_t *S = &s->sph[k];
        vec3 oc = vsub(o, S->c);
        float b = vdot(oc, d), c = vdot(oc, oc) - S->r * S->r;
        float disc = b * b - c;
        if (disc < 0) continue;
        float sq = sqrtf(disc);
        float t = -b - sq;
        if (t <= RAY_EPS) t = -b + sq;
        if (t <= RAY_EPS || t >= best) continue;
        best = t;
        h->n = vnorm(vadd(oc, vmul(d, t)));
        h->albedo = S->albedo;
        h->is_light = 0;
        found = 1;
    }
    h->t = best;
    return found;
}

static int occluded(const scene_t *s, vec3 o, vec3 d, float tmax)
{
    hit_t h;
    return intersect(s, o, d, tmax, &h);
}

/* Cosine-distributed direction around n from two uniforms (Malley's method). */
static vec3 cosine_dir(vec3 n, float u1, float u2)
{
    float rr = sqrtf(u1), phi = 2.0f * PI_F * u2;
    float lx = rr * cosf(phi), ly = rr * sinf(phi), lz = sqrtf(fmaxf(0.0f, 1.0f - u1));
    vec3 t = fabsf(n.x) > 0.5f ? v3(0, 1, 0) : v3(1, 0, 0);
    vec3 b1 = vnorm(vcross(t, n));
    vec3 b2 = vcross(n, b1);
    return vadd(vadd(vmul(b1, lx), vmul(b2, ly)), vmul(n, lz));
}

/* One sample of demodulated one-bounce indirect radiance at primary hit (p, n). */
static void indirect_sample(const scene_t *s, uint64_t seed, uint64_t pixel, uint64_t sample,
                            vec3 p, vec3 n, float out[3])
{
    out[0] = out[1] = out[2] = 0.0f;
    vec3 d = cosine_dir(n, urand(seed, pixel, sample, 0), urand(seed, pixel, sample, 1));
    vec3 o = vadd(p, vmul(n, RAY_EPS * 10));
    hit_t h2;
    if (!intersect(s, o, d, INFINITY, &h2) || h2.is_light) return;
    vec3 p2 = vadd(o, vmul(d, h2.t));
    vec3 n2 = h2.n;
    if (vdot(n2, d) > 0) n2 = vmul(n2, -1.0f);
    /* next-event estimation of the area light from the secondary hit */
    float lx = s->lx0 + (s->lx1 - s->lx0) * urand(seed, pixel, sample, 2);
    float lz = s->lz0 + (s->lz1 - s->lz0) * urand(seed, pixel, sample, 3);
    vec3 lp = v3(lx, s->ly, lz);
    vec3 o2 = vadd(p2, vmul(n2, RAY_EPS * 10));
    vec3 toL = vsub(lp, o2);
    float dist2 = vdot(toL, toL), dist = sqrtf(dist2);
    vec3 wl = vmul(toL, 1.0f / dist);
    float cos2 = vdot(n2, wl), cosl = wl.y; /* light faces down: its normal is -y */
    if (cos2 <= 0 || cosl <= 0) return;
    if (occluded(s, o2, wl, dist * (1.0f - 1e-4f))) return;
    float area = (s->lx1 - s->lx0) * (s->lz1 - s->lz0);
    float g = cos2 * cosl / dist2 * area / PI_F;
    for (int c = 0; c < 3; ++c) out[c] = h2.albedo[c] * s->le[c] * g;
}

/*
 * Render one frame of the scene of `seed`.
 *   guide     [8][H][W]  (see the file header for the channel order)
 *   radiance  [3][H][W]  one sample per pixel (sample index 0)
 *   reference [3][H][W]  or NULL: mean of `ref_spp` further samples (indices 1..ref_spp)
 * Returns 0, or -1 for bad arguments.
 */
/* Primary hit of pixel (x, y): direction d, hit h, hit point hp, normal n facing the camera. */
static void primary(const scene_t *s, int x, int y, int H, int W, vec3 *d, hit_t *h, vec3 *hp, vec3 *n)
{
    float sx = (2.0f * (x + 0.5f) / W - 1.0f) * s->tan_half_fov * ((float)W / H);
    float sy = (1.0f - 2.0f * (y + 0.5f) / H) * s->tan_half_fov;
    *d = vnorm(vadd(s->cam_fwd, vadd(vmul(s->cam_right, sx), vmul(s->cam_up, sy))));
    if (!intersect(s, s->cam_pos, *d, INFINITY, h)) {
        /* cannot happen in a closed room; keep the frame well defined */
        h->t = 1.0f;
        h->n = v3(0, 1, 0);
        h->albedo = s->wall_albedo[2];
    }
    *hp = vadd(s->cam_pos, vmul(*d, h->t));
    *n = h->n;
    if (vdot(*n, *d) > 0) *n = vmul(*n, -1.0f);
}

int synth_render(uint64_t seed, int H, int W, float *guide, float *radiance, float *reference,
                 int ref_spp)
{
    if (H <= 0 || W <= 0 || !guide || !radiance || (reference && ref_spp <= 0)) return -1;
    scene_t s;
    build_scene(seed, &s);
    const size_t P = (size_t)H * W;
    const float diag = sqrtf(ROOM_X * ROOM_X + ROOM_Y * ROOM_Y + ROOM_Z * ROOM_Z);
#pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            const size_t p = (size_t)y * W + x;
            const uint64_t pix = (uint64_t)p;
            vec3 d, hp, n;
            hit_t h;
            primary(&s, x, y, H, W, &d, &h, &hp, &n);
            for (int c = 0; c < 3; ++c) guide[(size_t)c * P + p] = h.albedo[c];
            guide[3 * P + p] = n.x;
            guide[4 * P + p] = n.y;
            guide[5 * P + p] = n.z;
            guide[6 * P + p] = h.t * vdot(d, s.cam_fwd) / diag;
            /* ambient occlusion: samples 0x10000.. keep it apart from the path samples */
            vec3 o = vadd(hp, vmul(n, RAY_EPS * 10));
            int open = 0;
            for (int k = 0; k < AO_RAYS; ++k) {
                vec3 ad = cosine_dir(n, urand(seed, pix, 0x10000 + k, 0), urand(seed, pix, 0x10000 + k, 1));
                if (!occluded(&s, o, ad, AO_DIST)) ++open;
            }
            guide[7 * P + p] = (float)open / AO_RAYS;
            float v[3];
            indirect_sample(&s, seed, pix, 0, hp, n, v);
            for (int c = 0; c < 3; ++c) radiance[(size_t)c * P + p] = v[c];
            if (reference) {
                double acc[3] = {0, 0, 0};
                for (int k = 1; k <= ref_spp; ++k) {
                    indirect_sample(&s, seed, pix, (uint64_t)k, hp, n, v);
                    for (int c = 0; c < 3; ++c) acc[c] += v[c];
                }
                for (int c = 0; c < 3; ++c) reference[(size_t)c * P + p] = (float)(acc[c] / ref_spp);
            }
        }
    }
    return 0;
}

/*
 * Further independent one-sample-per-pixel renders of the radiance of the scene of `seed`
 * (the same guides as synth_render): realisation j in [0, count) uses sample index
 * NOISE_SAMPLE0 + first + j, apart from the indices of the frame, its reference and AO.
 *   radiance [count][3][H][W]
 * Returns 0, or -1 for bad arguments.
 */
#define NOISE_SAMPLE0 (1ULL << 40)
int synth_render_noise(uint64_t seed, int H, int W, uint64_t first, int count, float *radiance)
{
    if (H <= 0 || W <= 0 || count <= 0 || !radiance) return -1;
    scene_t s;
    build_scene(seed, &s);
    const size_t P = (size_t)H * W;
#pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            const size_t p = (size_t)y * W + x;
            vec3 d, hp, n;
            hit_t h;
            primary(&s, x, y, H, W, &d, &h, &hp, &n);
            for (int j = 0; j < count; ++j) {
                float v[3];
                indirect_sample(&s, seed, (uint64_t)p, NOISE_SAMPLE0 + first + (uint64_t)j, hp, n, v);
                for (int c = 0; c < 3; ++c) radiance[((size_t)j * 3 + c) * P + p] = v[c];
            }
        }
    }
    return 0;
}

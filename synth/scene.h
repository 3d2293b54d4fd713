/*
 * scene.h -- the procedural room of the seeded input generator (pathtracer.c), shared by
 * the host renderer and the GPU reference renderer (pathtracer_gpu.cu): constants, the
 * scene record and its builder.  Input generation only; none of FLR's arithmetic.
 */
#ifndef SYNTH_SCENE_H
#define SYNTH_SCENE_H

#include <stdint.h>

#define ROOM_X 8.0f
#define ROOM_Y 4.0f
#define ROOM_Z 8.0f
#define N_BOXES 8
#define N_SPHERES 2
#define AO_RAYS 64
#define AO_DIST 2.0f
#define RAY_EPS 1e-4f
#define PI_F 3.14159265358979323846f

typedef struct { float x, y, z; } vec3;

typedef struct {
    vec3 lo, hi;
    float albedo[3];
} box_t;

typedef struct {
    vec3 c;
    float r;
    float albedo[3];
} sphere_t;

typedef struct {
    float wall_albedo[6][3]; /* -x, +x, -y (floor), +y (ceiling), -z, +z */
    box_t box[N_BOXES];
    sphere_t sph[N_SPHERES];
    float lx0, lx1, lz0, lz1, ly; /* light rectangle, facing down */
    float le[3];                  /* emitted radiance */
    vec3 cam_pos, cam_fwd, cam_right, cam_up;
    float tan_half_fov;
} scene_t;

#ifdef __cplusplus
extern "C" {
#endif
/* The scene of `seed` (deterministic); returns sizeof(scene_t) so callers can check it. */
int synth_build_scene(uint64_t seed, scene_t *s);
#ifdef __cplusplus
}
#endif

#endif

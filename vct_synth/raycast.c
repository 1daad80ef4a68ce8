/*
 * Seeded-input helper: pinhole raycasting of axis-aligned boxes inside an
 * optional room, producing the per-pixel G-buffer (surface position, face
 * normal, validity mask) that the voxel cone tracer consumes.
 *
 * This file holds input synthesis only: no cone tracing, sampling or mip
 * arithmetic.  It is compiled with -ffp-contract=off so that the same seed
 * yields the same bytes on every host architecture.
 *
 * Coordinates are scene units; the voxel grid spans [0,1]^3.  Boxes are given
 * as (lo_x, lo_y, lo_z, hi_x, hi_y, hi_z).  The room is the box the camera
 * sits inside; rays leave it through its inner faces.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

static void slab(const double o[3], const double d[3], const double lo[3],
                 const double hi[3], double *tn, double *tf, int *an,
                 int *af) {
  double t_near = -INFINITY, t_far = INFINITY;
  int a_near = 0, a_far = 0;
  for (int a = 0; a < 3; ++a) {
    double t1, t2;
    if (d[a] == 0.0) {
      if (o[a] < lo[a] || o[a] > hi[a]) {
        t1 = INFINITY;
        t2 = -INFINITY;
      } else {
        t1 = -INFINITY;
        t2 = INFINITY;
      }
    } else {
      t1 = (lo[a] - o[a]) / d[a];
      t2 = (hi[a] - o[a]) / d[a];
      if (t1 > t2) {
        double s = t1;
        t1 = t2;
        t2 = s;
      }
    }
    if (t1 > t_near) {
      t_near = t1;
      a_near = a;
    }
    if (t2 < t_far) {
      t_far = t2;
      a_far = a;
    }
  }
  *tn = t_near;
  *tf = t_far;
  *an = a_near;
  *af = a_far;
}

/*
 * For pixel (j, i) of a W x H image, the ray leaves `cam` along
 * normalize(fwd + sx*right + sy*up) with sx = (2(i+0.5)/W - 1) tan_half * W/H
 * and sy = (1 - 2(j+0.5)/H) tan_half.  The nearest box entry or room exit is
 * recorded; the coordinate on the hit face is snapped to the face plane.
 * pos/nrm are [H*W*3] float, mask [H*W].
 */
void vs_raycast(int W, int H, const double *cam, const double *fwd,
                const double *right, const double *up, double tan_half,
                int n_boxes, const double *boxes, int has_room,
                const double *room, float *pos, float *nrm, uint8_t *mask) {
  const double aspect = (double)W / (double)H;
#pragma omp parallel for schedule(dynamic, 16)
  for (int j = 0; j < H; ++j) {
    for (int i = 0; i < W; ++i) {
      double sx = (2.0 * (i + 0.5) / W - 1.0) * tan_half * aspect;
      double sy = (1.0 - 2.0 * (j + 0.5) / H) * tan_half;
      double d[3];
      for (int a = 0; a < 3; ++a) d[a] = fwd[a] + sx * right[a] + sy * up[a];
      double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      for (int a = 0; a < 3; ++a) d[a] /= len;

      double best = INFINITY, plane = 0.0;
      int axis = -1;
      double nsign = 0.0;
      for (int b = 0; b < n_boxes; ++b) {
        const double *bx = boxes + 6 * b;
        double tn, tf;
        int an, af;
        slab(cam, d, bx, bx + 3, &tn, &tf, &an, &af);
        if (tn <= tf && tn > 0.0 && tn < best) {
          best = tn;
          axis = an;
          nsign = d[an] > 0.0 ? -1.0 : 1.0;
          plane = d[an] > 0.0 ? bx[an] : bx[3 + an];
        }
      }
      if (has_room) {
        double tn, tf;
        int an, af;
        slab(cam, d, room, room + 3, &tn, &tf, &an, &af);
        if (tf > 0.0 && tf < best) {
          best = tf;
          axis = af;
          nsign = d[af] > 0.0 ? -1.0 : 1.0;
          plane = d[af] > 0.0 ? room[3 + af] : room[af];
        }
      }
      size_t p = (size_t)j * W + i;
      if (axis < 0) {
        for (int a = 0; a < 3; ++a) {
          pos[3 * p + a] = 0.0f;
          nrm[3 * p + a] = 0.0f;
        }
        mask[p] = 0;
        continue;
      }
      for (int a = 0; a < 3; ++a) {
        double x = cam[a] + best * d[a];
        pos[3 * p + a] = (float)(a == axis ? plane : x);
        nrm[3 * p + a] = (float)(a == axis ? nsign : 0.0);
      }
      mask[p] = 1;
    }
  }
}

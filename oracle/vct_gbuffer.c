/*
 * FP64 CPU oracle: G-buffer of a triangle mesh seen by a pinhole camera.
 *
 * TEST INFRASTRUCTURE ONLY (see vct_oracle.c).  It shares no code with the
 * CUDA library.
 *
 * What it computes: the geometry pass of the deferred renderer that feeds the
 * cone tracer (Ch. 5.4: the scene is first drawn into buffers of position,
 * normal and material colour, which the cone-tracing pass then reads per
 * pixel; Ch. 3.2 rasterisation).  For every pixel: the nearest triangle on
 * the ray through the pixel centre, the hit position, the triangle's unit
 * geometric normal turned towards the camera, and its material colour.
 *
 * Readings (the thesis leaves these to the OpenGL rasteriser; they are written
 * out so that the CUDA path can take the same decisions exactly):
 *  - pixel (i, j) of a W x H image (j = 0 the top row) looks along
 *    d = (f + sx r) + sy u with sx = ((2i+1)/W - 1) tx, sy = (1 - (2j+1)/H) ty,
 *    tx = float32(tan_half W / H), ty = tan_half, each operation rounded to
 *    IEEE float32 (no fused multiply-add); f, r, u the camera's forward, right
 *    and up vectors as given;
 *  - positions snap to a fixed-point frame of 2^17 units per frame size:
 *    X = rint(float32(float32(p - origin) * s)), s = float32(2^17 / size),
 *    the camera too; a triangle with a vertex of |X| >= 2^18 (or a bad index)
 *    is skipped, one of zero snapped area is degenerate; the ray direction
 *    snaps to D = rint(float32(d * 2^18));
 *  - with A, B, C the snapped vertices relative to the snapped camera, the ray
 *    hits the (double-sided) triangle when the volumes D.(B x C), D.(C x A),
 *    D.(A x B) share one sign (zeros allowed, not all zero) and that sign is
 *    the sign of det(A, B, C), i.e. the hit lies ahead of the camera;
 *  - the hit's distance is t = det(A, B, C) / (n . D), n = (B - A) x (C - A);
 *    the smallest t wins by exact comparison of the fractions, equal t going
 *    to the lower triangle index;
 *  - the normal's sign comes from the exact n . D (towards the camera), its
 *    direction from the unsnapped vertices.
 * All decisions are exact integer arithmetic (128-bit where products need it).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

typedef __int128 i128;

#define FRAME_UNITS 131072.0  /* 2^17 */
#define COORD_LIMIT 262144.0f /* 2^18 */
#define DIR_SCALE 262144.0f   /* 2^18 */

static int snapf(float v, float origin, float s, int64_t *out) {
  const float rel = v - origin;
  const float b = rel * s;
  if (!(fabsf(b) < COORD_LIMIT)) return 0;
  *out = (int64_t)rintf(b);
  return 1;
}

typedef struct {
  int usable;
  int64_t V[3][3]; /* vertices relative to the camera */
  i128 c[3][3];    /* B x C, C x A, A x B */
  i128 det;        /* det(A, B, C) */
} orc_tri;

/*
 * Pixels listed in idx (count of them; all W*H in row-major order if idx is
 * NULL).  Per listed pixel: tri_out (triangle index or -1), pos[3], nrm[3],
 * albedo[3] (zeros without a hit), mask (0/1).  stats[0] += skipped
 * triangles, stats[1] += degenerate ones.  Returns 0, or -1 if the camera
 * lies outside the frame.
 */
int orc_gbuffer(const float *vertices, int64_t nv, const int32_t *indices, int64_t nt,
                const float *colors, const float *frame_origin, float frame_size,
                const float *cam, const float *fwd, const float *right, const float *up,
                float tan_half, int W, int H, const int64_t *idx, int64_t count,
                int32_t *tri_out, double *pos, double *nrm, double *albedo, uint8_t *mask,
                int64_t *stats) {
  const float s = (float)(FRAME_UNITS / (double)frame_size);
  const float tx = (float)((double)tan_half * (double)W / (double)H);
  const float ty = tan_half;
  int64_t O[3];
  for (int a = 0; a < 3; ++a)
    if (!snapf(cam[a], frame_origin[a], s, &O[a])) return -1;

  orc_tri *T = (orc_tri *)calloc(nt > 0 ? (size_t)nt : 1, sizeof(orc_tri));
  if (!T) return -2;
  for (int64_t t = 0; t < nt; ++t) {
    const int32_t *ix = indices + 3 * t;
    int ok = 1;
    for (int k = 0; k < 3; ++k) ok = ok && ix[k] >= 0 && ix[k] < nv;
    for (int k = 0; k < 3 && ok; ++k)
      for (int a = 0; a < 3 && ok; ++a) {
        int64_t X;
        ok = snapf(vertices[3 * ix[k] + a], frame_origin[a], s, &X);
        T[t].V[k][a] = X - O[a];
      }
    if (!ok) {
      stats[0] += 1;
      continue;
    }
    const int64_t *A = T[t].V[0], *B = T[t].V[1], *C = T[t].V[2];
    /* the snapped plane normal n = (B - A) x (C - A) */
    int64_t e1[3], e2[3];
    for (int a = 0; a < 3; ++a) {
      e1[a] = B[a] - A[a];
      e2[a] = C[a] - A[a];
    }
    const i128 n0 = (i128)e1[1] * e2[2] - (i128)e1[2] * e2[1];
    const i128 n1 = (i128)e1[2] * e2[0] - (i128)e1[0] * e2[2];
    const i128 n2 = (i128)e1[0] * e2[1] - (i128)e1[1] * e2[0];
    if (n0 == 0 && n1 == 0 && n2 == 0) {
      stats[1] += 1;
      continue;
    }
    const int64_t *P[3] = {B, C, A}, *Q[3] = {C, A, B};
    for (int k = 0; k < 3; ++k) {
      T[t].c[k][0] = (i128)P[k][1] * Q[k][2] - (i128)P[k][2] * Q[k][1];
      T[t].c[k][1] = (i128)P[k][2] * Q[k][0] - (i128)P[k][0] * Q[k][2];
      T[t].c[k][2] = (i128)P[k][0] * Q[k][1] - (i128)P[k][1] * Q[k][0];
    }
    T[t].det = T[t].c[0][0] * A[0] + T[t].c[0][1] * A[1] + T[t].c[0][2] * A[2];
    T[t].usable = 1;
  }

#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < count; ++q) {
    const int64_t px = idx ? idx[q] : q;
    const int i = (int)(px % W), j = (int)(px / W);
    const float sx = ((float)(2 * i + 1) / (float)W - 1.0f) * tx;
    const float sy = (1.0f - (float)(2 * j + 1) / (float)H) * ty;
    int64_t D[3];
    for (int a = 0; a < 3; ++a) {
      const float d = (fwd[a] + sx * right[a]) + sy * up[a];
      D[a] = (int64_t)rintf(d * DIR_SCALE);
    }
    int32_t best = -1;
    i128 bnum = 0, bden = 1, bsigned = 0;
    for (int64_t t = 0; t < nt; ++t) {
      if (!T[t].usable) continue;
      i128 v[3];
      for (int k = 0; k < 3; ++k)
        v[k] = T[t].c[k][0] * D[0] + T[t].c[k][1] * D[1] + T[t].c[k][2] * D[2];
      const i128 det = T[t].det;
      int hit;
      if (det > 0)
        hit = v[0] >= 0 && v[1] >= 0 && v[2] >= 0;
      else if (det < 0)
        hit = v[0] <= 0 && v[1] <= 0 && v[2] <= 0;
      else
        hit = 0;
      if (!hit || (v[0] == 0 && v[1] == 0 && v[2] == 0)) continue;
      /* n . D = v0 + v1 + v2; t = det / (n . D) > 0 */
      const i128 den_signed = v[0] + v[1] + v[2];
      const i128 num = det > 0 ? det : -det;
      const i128 den = den_signed > 0 ? den_signed : -den_signed;
      if (best < 0 || num * bden < bnum * den) {
        best = (int32_t)t;
        bnum = num;
        bden = den;
        bsigned = den_signed;
      }
    }
    tri_out[q] = best;
    mask[q] = best >= 0;
    for (int a = 0; a < 3; ++a) pos[3 * q + a] = nrm[3 * q + a] = albedo[3 * q + a] = 0.0;
    if (best < 0) continue;
    /* hit position on the snapped ray, scene units */
    const double tt = (double)bnum / (double)bden;
    for (int a = 0; a < 3; ++a)
      pos[3 * q + a] =
          (double)frame_origin[a] + ((double)O[a] + tt * (double)D[a]) / (double)s;
    /* unit normal of the unsnapped triangle, towards the camera */
    const int32_t *ix = indices + 3 * best;
    double u3[3], v3[3], g[3];
    for (int a = 0; a < 3; ++a) {
      u3[a] = (double)vertices[3 * ix[1] + a] - (double)vertices[3 * ix[0] + a];
      v3[a] = (double)vertices[3 * ix[2] + a] - (double)vertices[3 * ix[0] + a];
    }
    g[0] = u3[1] * v3[2] - u3[2] * v3[1];
    g[1] = u3[2] * v3[0] - u3[0] * v3[2];
    g[2] = u3[0] * v3[1] - u3[1] * v3[0];
    const double len = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    /* n . D > 0: the snapped normal points away from the camera */
    const double sgn = bsigned > 0 ? -1.0 : 1.0;
    for (int a = 0; a < 3; ++a) {
      nrm[3 * q + a] = len > 0.0 ? sgn * g[a] / len : 0.0;
      albedo[3 * q + a] = (double)colors[3 * best + a];
    }
  }
  free(T);
  return 0;
}

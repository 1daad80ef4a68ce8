/*
 * FP64 CPU oracle: voxelization of a triangle mesh into the level-0 grid.
 *
 * TEST INFRASTRUCTURE ONLY (see vct_oracle.c).  It shares no code with the
 * CUDA library.
 *
 * What it computes (thesis Ch. 4.4, "Voxelization Process", and Ch. 5.4.4,
 * the voxelize() steps):
 *  - the grid starts empty: every voxel (0, 0, 0, 0);
 *  - every triangle is rasterised once, orthographically, along its dominant
 *    axis: the axis of the largest component of |(v2 - v1) x (v3 - v1)|
 *    (Ch. 4.4.2).  The vertices are swizzled so that the dominant axis
 *    becomes depth: x-dominant (x,y,z) -> (z,y,x), y-dominant -> (x,z,y),
 *    z-dominant unchanged;
 *  - the viewport is n x n pixels over the grid face; every pixel whose
 *    centre the projected triangle covers yields one fragment, whose depth
 *    is the triangle's plane at that centre; the fragment's voxel is the
 *    pixel plus the depth cell (fragments outside the grid are clipped);
 *  - the fragment stores the direct diffuse light of the Phong model without
 *    its glossy term (Ch. 4.4.3, Ch. 3.3 listing): colour * light_color *
 *    (ambient + diffuse_str * max(N . l, 0)), N the normalised geometric
 *    normal the triangle had before the swizzle, and alpha 1.
 *
 * Readings (the thesis relies on the OpenGL rasteriser and leaves these to
 * it; the CUDA path takes the same decisions from its own code):
 *  - vertices snap to 1/256 voxel (a rasteriser's sub-pixel grid):
 *    X = rint(float32(float32(v - origin) * s)), s = float32(256 n / size),
 *    evaluated in IEEE float32; triangles with a snapped coordinate of
 *    magnitude >= 2^19, or with zero snapped area, are skipped;
 *  - pixel centres lie at (i + 1/2) voxels; a centre on an edge belongs to
 *    the triangle only if the edge is a top or left edge (OpenGL's rule),
 *    so triangles sharing an edge cover each centre once;
 *  - the depth cell is floor(depth) of the exact plane depth (integer
 *    arithmetic on the snapped coordinates);
 *  - ties between equal |normal| components pick the first axis (x, y, z);
 *  - where fragments of several triangles land in one voxel, the triangle
 *    drawn last (highest index) wins, i.e. serial draw order.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define SUB 256          /* sub-voxel steps per voxel */
#define COORD_LIMIT 524288.0f  /* 2^19 */

static int64_t abs64(int64_t a) { return a < 0 ? -a : a; }

/* floor(a / b) for b != 0 */
static int64_t floor_div(int64_t a, int64_t b) {
  if (b < 0) {
    a = -a;
    b = -b;
  }
  int64_t q = a / b;
  if ((a % b) != 0 && a < 0) q -= 1;
  return q;
}

/* Snaps one coordinate; returns 0 if out of range. */
static int snap(float v, float origin, float s, int64_t *out) {
  float a = v - origin;
  float b = a * s;
  if (!(fabsf(b) < COORD_LIMIT)) return 0;
  *out = (int64_t)rintf(b);
  return 1;
}

/* Is the pixel centre p on the inside of the directed edge a -> b of a
 * counter-clockwise triangle (top-left rule on the edge itself)? */
static int inside_edge(const int64_t a[2], const int64_t b[2], const int64_t p[2]) {
  int64_t eu = b[0] - a[0], ev = b[1] - a[1];
  int64_t e = eu * (p[1] - a[1]) - ev * (p[0] - a[0]);
  if (e > 0) return 1;
  if (e < 0) return 0;
  return ev < 0 || (ev == 0 && eu < 0);
}

/*
 * vertices [nv][3] float32, indices [nt][3] int32, colors [nt][3] float32.
 * grid_out [n][n][n][4] (z, y, x, rgba), owner_out [n][n][n] (triangle
 * index + 1, 0 = empty).  stats[0] += fragments inside the grid,
 * stats[1] += skipped triangles (out of range or bad index), stats[2] +=
 * triangles with zero snapped area.
 */
void orc_voxelize(const float *vertices, int64_t nv, const int32_t *indices, int64_t nt,
                  const float *colors, int n, const float *origin, float size,
                  const double *light_dir, const double *light_color, double ambient,
                  double diffuse_str, double *grid_out, int32_t *owner_out,
                  int64_t *stats) {
  const size_t nvox = (size_t)n * n * n;
  memset(grid_out, 0, nvox * 4 * sizeof(double));
  memset(owner_out, 0, nvox * sizeof(int32_t));
  const float s = (float)(256.0 * (double)n / (double)size);
  for (int64_t t = 0; t < nt; ++t) {
    const int32_t *ix = indices + 3 * t;
    if (ix[0] < 0 || ix[0] >= nv || ix[1] < 0 || ix[1] >= nv || ix[2] < 0 || ix[2] >= nv) {
      stats[1] += 1;
      continue;
    }
    /* snapped vertex coordinates */
    int64_t V[3][3];
    int ok = 1;
    for (int k = 0; k < 3 && ok; ++k)
      for (int a = 0; a < 3 && ok; ++a)
        ok = snap(vertices[3 * ix[k] + a], origin[a], s, &V[k][a]);
    if (!ok) {
      stats[1] += 1;
      continue;
    }
    /* normal (v2 - v1) x (v3 - v1) and its dominant axis */
    int64_t e1[3], e2[3], N[3];
    for (int a = 0; a < 3; ++a) {
      e1[a] = V[1][a] - V[0][a];
      e2[a] = V[2][a] - V[0][a];
    }
    N[0] = e1[1] * e2[2] - e1[2] * e2[1];
    N[1] = e1[2] * e2[0] - e1[0] * e2[2];
    N[2] = e1[0] * e2[1] - e1[1] * e2[0];
    if (N[0] == 0 && N[1] == 0 && N[2] == 0) {
      stats[2] += 1;
      continue;
    }
    int64_t ax = abs64(N[0]), ay = abs64(N[1]), az = abs64(N[2]);
    int dom = 2;
    if (ax >= ay && ax >= az)
      dom = 0;
    else if (ay >= az)
      dom = 1;
    /* swizzle: (u, v) raster axes, depth axis */
    int au, av;
    if (dom == 0) {
      au = 2;
      av = 1;
    } else if (dom == 1) {
      au = 0;
      av = 2;
    } else {
      au = 0;
      av = 1;
    }
    int64_t P[3][2];
    for (int k = 0; k < 3; ++k) {
      P[k][0] = V[k][au];
      P[k][1] = V[k][av];
    }
    /* orient counter-clockwise in (u, v) (triangles are double sided) */
    int64_t area = (P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) -
                   (P[1][1] - P[0][1]) * (P[2][0] - P[0][0]);
    int o1 = 1, o2 = 2;
    if (area < 0) {
      o1 = 2;
      o2 = 1;
    }
    /* direct diffuse light of the triangle (FP64, unsnapped vertices) */
    double a3[3], b3[3], nf[3];
    for (int a = 0; a < 3; ++a) {
      a3[a] = (double)vertices[3 * ix[1] + a] - (double)vertices[3 * ix[0] + a];
      b3[a] = (double)vertices[3 * ix[2] + a] - (double)vertices[3 * ix[0] + a];
    }
    nf[0] = a3[1] * b3[2] - a3[2] * b3[1];
    nf[1] = a3[2] * b3[0] - a3[0] * b3[2];
    nf[2] = a3[0] * b3[1] - a3[1] * b3[0];
    double len = sqrt(nf[0] * nf[0] + nf[1] * nf[1] + nf[2] * nf[2]);
    double lam = 0.0;
    if (len > 0.0) {
      lam = (nf[0] * light_dir[0] + nf[1] * light_dir[1] + nf[2] * light_dir[2]) / len;
      if (lam < 0.0) lam = 0.0;
    }
    double rgb[3];
    for (int c = 0; c < 3; ++c)
      rgb[c] = (double)colors[3 * t + c] * light_color[c] * (ambient + diffuse_str * lam);
    /* every pixel centre of the viewport the triangle may cover */
    int64_t umin = P[0][0], umax = P[0][0], vmin = P[0][1], vmax = P[0][1];
    for (int k = 1; k < 3; ++k) {
      if (P[k][0] < umin) umin = P[k][0];
      if (P[k][0] > umax) umax = P[k][0];
      if (P[k][1] < vmin) vmin = P[k][1];
      if (P[k][1] > vmax) vmax = P[k][1];
    }
    int64_t i0 = floor_div(umin - SUB / 2 + SUB - 1, SUB), i1 = floor_div(umax - SUB / 2, SUB);
    int64_t j0 = floor_div(vmin - SUB / 2 + SUB - 1, SUB), j1 = floor_div(vmax - SUB / 2, SUB);
    if (i0 < 0) i0 = 0;
    if (j0 < 0) j0 = 0;
    if (i1 > n - 1) i1 = n - 1;
    if (j1 > n - 1) j1 = n - 1;
    for (int64_t j = j0; j <= j1; ++j)
      for (int64_t i = i0; i <= i1; ++i) {
        int64_t p[2] = {SUB * i + SUB / 2, SUB * j + SUB / 2};
        if (!inside_edge(P[0], P[o1], p) || !inside_edge(P[o1], P[o2], p) ||
            !inside_edge(P[o2], P[0], p))
          continue;
        /* depth: N . (X - V1) = 0 solved for the dominant coordinate */
        int64_t off = -(N[au] * (p[0] - V[0][au]) + N[av] * (p[1] - V[0][av]));
        int64_t depth = V[0][dom] + floor_div(off, N[dom]); /* floor, sub-voxel units */
        int64_t k = floor_div(depth, SUB);
        if (k < 0 || k >= n) continue;
        int64_t c[3];
        c[au] = i;
        c[av] = j;
        c[dom] = k;
        size_t vox = ((size_t)c[2] * n + (size_t)c[1]) * n + (size_t)c[0];
        stats[0] += 1;
        owner_out[vox] = (int32_t)(t + 1);
        for (int ch = 0; ch < 3; ++ch) grid_out[4 * vox + ch] = rgb[ch];
        grid_out[4 * vox + 3] = 1.0;
      }
  }
}

/*
 * FP64 CPU oracle for the voxel-cone-tracing hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; it exists so that the CUDA library can be compared with a
 * plain, slow, obviously correct restatement of the method.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * What it computes, in the thesis's order (B. Kahl, "Real-Time Global
 * Illumination Using OpenGL And Voxel Cone Tracing", 2019):
 *
 *  - mip pyramid: each level halves every dimension and each texel is the
 *    plain average of its 2x2x2 children (Ch. 4.3.3 "Mipmaps" and "Texture
 *    Filtering": a factor-2 minification makes every texel contribute, and
 *    Ch. 5.4.4 builds the levels right after voxelization);
 *  - sample(position, diameter): mip level = log2(diameter / voxel size) and a
 *    linear-in-level, trilinear-in-space lookup with texel centres at
 *    (i + 1/2) h_l (Ch. 4.5, colour supersampler; Ch. 4.3.3 textureLod);
 *  - the cone trace (Ch. 4.3.2, volume ray marching): diameter
 *    d = 2 t tan(gamma/2), sample at p = x + t w, front-to-back accumulation
 *    of colour and occlusion, advance t by beta * d, stop once the occlusion
 *    reaches 1 (plus a maximum distance, see below);
 *  - the per-pixel cone set (Ch. 4.2: diffuse cones over the normal
 *    hemisphere, one specular cone along the reflection direction, one
 *    occlusion cone per light) and the weighted diffuse sum (Ch. 4.1 / 4.2.2:
 *    one BRDF weight per cone).
 *
 * Readings of passages the thesis leaves open or garbled (the same readings
 * are used by the CUDA path; they are inputs or fixed choices, not shared
 * code):
 *  - colour accumulation is c <- c + (1 - alpha) a_s c_s (the printed line
 *    also scales the running colour by alpha, which is not front-to-back
 *    compositing);
 *  - the level is log2(d / h0) with h0 the level-0 voxel edge, clamped to
 *    [0, L-1]; the fractional part blends two adjacent levels;
 *  - texels outside the grid read as zero (empty space);
 *  - the march also stops once t exceeds t_max (the listing has no bound);
 *  - the start offset is t0 = t0_voxels * h0 and the cone apex is moved
 *    normal_offset_voxels * h0 along the surface normal;
 *  - the tangent frame for the diffuse table is T = normalize(a x n),
 *    B = n x T with a = (1,0,0) if |n_x| < 0.9 else (0,1,0);
 *  - the specular aperture grows linearly with roughness between
 *    spec_aperture_min (at roughness_min) and spec_aperture_max (at 1).
 *
 * All arithmetic is double precision; the build uses -ffp-contract=off so
 * that results do not depend on the host's fused multiply-add.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_DIFFUSE 32

/* Variant flags (Ch. 5.4.4, the thesis's modified cones; and the shading
 * composition of Ch. 4.2.2 / Ch. 5.4.4). */
#define ORC_OCC_SMOOTH 1   /* occlusion: a_s * smoothstep(0, max_dist, sqrt(t) shadow_str) */
#define ORC_SPEC_GRACE 2   /* specular: colour * (1 - max(0, acos(w.l) - p)/pi)^q          */
#define ORC_DIFF_FIRST 4   /* diffuse: colour of the first sample with opacity > 1/100     */
#define ORC_SHADE 8        /* write the radiance L_vxct                                     */
#define ORC_SHADE_IMPL 16  /* ... composed as L_impl instead                                */
#define ORC_PREMUL 32      /* every cone: sample colour premultiplied, c += (1 - alpha) c_s */
#define ORC_ANISO 64       /* the pyramid is anisotropic (orc_build_mips_aniso)               */

typedef struct {
  int32_t n_diffuse;
  int32_t spec_enable;
  int32_t occ_enable;
  int32_t flags;
  double diffuse_dir[ORC_MAX_DIFFUSE][3];
  double diffuse_weight[ORC_MAX_DIFFUSE];
  double diffuse_aperture;
  double spec_aperture_min, spec_aperture_max, roughness_min;
  double occ_aperture;
  double light_dir[3];
  double beta, t0_voxels, normal_offset_voxels, t_max;
  double shadow_str, occ_max_dist;       /* modified occlusion cone          */
  double shininess, shininess_falloff;   /* Phong alpha; angular-grace q     */
  double diffuse_str, specular_str;      /* material ratios c_d, c_s scales  */
  double light_color[3];                 /* i_{s,d} = i_{s,g} (RGB)          */
} orc_params;

/* A pyramid: `levels` dense arrays [z][y][x][4] of doubles, level l has
 * n >> l texels per axis, stored back to back starting with level 0.  The
 * grid covers [origin, origin + size]^3 in scene units. */
typedef struct {
  const double *data;
  int32_t n, levels;
  double origin[3], size;
  int aniso; /* levels >= 1 hold six directional volumes (orc_build_mips_aniso) */
} orc_grid;

/* Per-view G-buffer as the caller holds it (float32 inputs). */
typedef struct {
  int32_t width, height;
  const float *position; /* [H*W*3] */
  const float *normal;   /* [H*W*3] */
  const float *roughness; /* [H*W] or NULL */
  const uint8_t *mask;    /* [H*W] or NULL */
  const float *albedo;    /* [H*W*3] material colour, or NULL (white) */
  double camera[3];
} orc_view;

int orc_version(void) { return 1; }

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

size_t orc_level_offset(int n, int level) {
  size_t off = 0;
  for (int l = 0; l < level; ++l) {
    size_t m = (size_t)(n >> l);
    off += m * m * m * 4;
  }
  return off;
}

/* ---------------------------------------------------------------------- */
/* mip pyramid (Ch. 4.3.3)                                                 */
/* ---------------------------------------------------------------------- */
void orc_build_mips(const double *level0, int n, int levels, double *pyr) {
  size_t m0 = (size_t)n * n * n * 4;
  memcpy(pyr, level0, m0 * sizeof(double));
  for (int l = 1; l < levels; ++l) {
    const double *src = pyr + orc_level_offset(n, l - 1);
    double *dst = pyr + orc_level_offset(n, l);
    int nc = n >> (l - 1), np = n >> l;
#pragma omp parallel for
    for (int z = 0; z < np; ++z)
      for (int y = 0; y < np; ++y)
        for (int x = 0; x < np; ++x)
          for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int dz = 0; dz < 2; ++dz)
              for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                  size_t i = (((size_t)(2 * z + dz) * nc + (2 * y + dy)) * nc +
                              (2 * x + dx)) * 4 + c;
                  s += src[i];
                }
            dst[(((size_t)z * np + y) * np + x) * 4 + c] = s / 8.0;
          }
  }
}

/* ---------------------------------------------------------------------- */
/* anisotropic mips (Villegas' anisotropic filtering, Ch. 5.1)             */
/* ---------------------------------------------------------------------- */
/*
 * Level 0 is the isotropic grid.  Every level l >= 1 holds six volumes, one
 * per direction of travel d = +x, -x, +y, -y, +z, -z (index 2 axis + (sign <
 * 0)), each dense [z][y][x][4] with n >> l texels per axis, back to back
 * after level 0.  A texel of volume d at level l+1 is the straight 4-channel
 * mean (as the isotropic filter) over the four child pairs along axis(d) of
 * the pair seen along d: front = the child met first when travelling along d,
 *   alpha = a_f + (1 - a_f) a_b,
 *   colour = (a_f c_f + (1 - a_f) a_b c_b) / alpha  (0 where alpha = 0).
 * The children are level 0's texels for l = 0, else volume d of level l.
 */
size_t orc_aniso_offset(int n, int level, int dir) {
  if (level == 0) return 0;
  size_t off = (size_t)n * n * n * 4;
  for (int l = 1; l < level; ++l) {
    size_t m = (size_t)(n >> l);
    off += 6 * m * m * m * 4;
  }
  size_t m = (size_t)(n >> level);
  return off + (size_t)dir * m * m * m * 4;
}

void orc_build_mips_aniso(const double *level0, int n, int levels, double *pyr) {
  memcpy(pyr, level0, (size_t)n * n * n * 4 * sizeof(double));
  for (int l = 1; l < levels; ++l) {
    int nc = n >> (l - 1), np = n >> l;
    for (int d = 0; d < 6; ++d) {
      const int axis = d / 2, neg = d & 1;
      const double *src = pyr + orc_aniso_offset(n, l - 1, l == 1 ? 0 : d);
      double *dst = pyr + orc_aniso_offset(n, l, d);
#pragma omp parallel for
      for (int z = 0; z < np; ++z)
        for (int y = 0; y < np; ++y)
          for (int x = 0; x < np; ++x) {
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            /* the four pairs: offsets along the two other axes */
            for (int u = 0; u < 2; ++u)
              for (int v = 0; v < 2; ++v) {
                const double *ch[2];
                for (int k = 0; k < 2; ++k) {
                  int o[3];
                  o[axis] = k;
                  o[(axis + 1) % 3] = u;
                  o[(axis + 2) % 3] = v;
                  size_t i = (((size_t)(2 * z + o[2]) * nc + (2 * y + o[1])) * nc +
                              (2 * x + o[0])) * 4;
                  ch[k] = src + i;
                }
                const double *f = neg ? ch[1] : ch[0], *b = neg ? ch[0] : ch[1];
                double a = f[3] + (1.0 - f[3]) * b[3];
                for (int c = 0; c < 3; ++c) {
                  double pre = f[3] * f[c] + (1.0 - f[3]) * b[3] * b[c];
                  acc[c] += a > 0.0 ? pre / a : 0.0;
                }
                acc[3] += a;
              }
            double *t = dst + (((size_t)z * np + y) * np + x) * 4;
            for (int c = 0; c < 4; ++c) t[c] = acc[c] / 4.0;
          }
    }
  }
}

/* Adjoint of orc_build_mips: given dL/d(level l) for every level (same
 * layout as the pyramid), push each coarse gradient down to its children
 * (each child receives 1/8 of its parent's), coarse to fine, then add the
 * level-0 result into grad0. */
void orc_mip_adjoint(double *gpyr, int n, int levels, double *grad0) {
  for (int l = levels - 1; l >= 1; --l) {
    const double *gp = gpyr + orc_level_offset(n, l);
    double *gc = gpyr + orc_level_offset(n, l - 1);
    int nc = n >> (l - 1), np = n >> l;
#pragma omp parallel for
    for (int z = 0; z < nc; ++z)
      for (int y = 0; y < nc; ++y)
        for (int x = 0; x < nc; ++x)
          for (int c = 0; c < 4; ++c)
            gc[(((size_t)z * nc + y) * nc + x) * 4 + c] +=
                gp[(((size_t)(z / 2) * np + y / 2) * np + x / 2) * 4 + c] / 8.0;
  }
  size_t m0 = (size_t)n * n * n * 4;
  for (size_t i = 0; i < m0; ++i) grad0[i] += gpyr[i];
}

/*
 * Adjoint of orc_build_mips_aniso.  gpyr holds dL/d(texel) for every texel of
 * the anisotropic pyramid pyr (same layout).  Coarse to fine, each texel of
 * volume d at level l passes its gradient to its 8 children: the texel is
 * (1/4) sum over the four pairs (f, b) along axis(d), f the child met first,
 * of P = (C, alpha) with
 *   alpha = a_f + (1 - a_f) a_b,  C = (a_f c_f + (1 - a_f) a_b c_b) / alpha,
 * whose partials are
 *   dC/dc_f = a_f / alpha,  dC/dc_b = (1 - a_f) a_b / alpha,
 *   dC/da_f = (c_f - a_b c_b - C (1 - a_b)) / alpha,
 *   dC/da_b = (1 - a_f) (c_b - C) / alpha,
 *   dalpha/da_f = 1 - a_b,  dalpha/da_b = 1 - a_f.
 * Where alpha = 0 (both children empty) C is 0 by definition and not
 * differentiable in the opacities: its colour partials are taken as 0 there.
 * The children of level 1 are level 0's texels (all six directions add into
 * them); the level-0 result is ADDED into grad0.
 */
void orc_mip_adjoint_aniso(const double *pyr, double *gpyr, int n, int levels, double *grad0) {
  for (int l = levels - 1; l >= 1; --l) {
    int nc = n >> (l - 1), np = n >> l;
    for (int d = 0; d < 6; ++d) {
      const int axis = d / 2, neg = d & 1, child_vol = l == 1 ? 0 : d;
      const double *src = pyr + orc_aniso_offset(n, l - 1, child_vol);
      double *gsrc = gpyr + orc_aniso_offset(n, l - 1, child_vol);
      const double *gdst = gpyr + orc_aniso_offset(n, l, d);
#pragma omp parallel for
      for (int z = 0; z < np; ++z)
        for (int y = 0; y < np; ++y)
          for (int x = 0; x < np; ++x) {
            const double *G = gdst + (((size_t)z * np + y) * np + x) * 4;
            for (int u = 0; u < 2; ++u)
              for (int v = 0; v < 2; ++v) {
                size_t ci[2];
                for (int k = 0; k < 2; ++k) {
                  int o[3];
                  o[axis] = k;
                  o[(axis + 1) % 3] = u;
                  o[(axis + 2) % 3] = v;
                  ci[k] = (((size_t)(2 * z + o[2]) * nc + (2 * y + o[1])) * nc + (2 * x + o[0])) * 4;
                }
                const size_t fi = neg ? ci[1] : ci[0], bi = neg ? ci[0] : ci[1];
                const double *f = src + fi, *b = src + bi;
                const double af = f[3], ab = b[3];
                const double alpha = af + (1.0 - af) * ab;
                double gf[4] = {0.0, 0.0, 0.0, 0.0}, gb[4] = {0.0, 0.0, 0.0, 0.0};
                gf[3] = G[3] / 4.0 * (1.0 - ab);
                gb[3] = G[3] / 4.0 * (1.0 - af);
                if (alpha > 0.0) {
                  for (int c = 0; c < 3; ++c) {
                    const double gC = G[c] / 4.0;
                    const double C = (af * f[c] + (1.0 - af) * ab * b[c]) / alpha;
                    gf[c] = gC * af / alpha;
                    gb[c] = gC * (1.0 - af) * ab / alpha;
                    gf[3] += gC * (f[c] - ab * b[c] - C * (1.0 - ab)) / alpha;
                    gb[3] += gC * (1.0 - af) * (b[c] - C) / alpha;
                  }
                }
                for (int c = 0; c < 4; ++c) {
                  gsrc[fi + c] += gf[c];
                  gsrc[bi + c] += gb[c];
                }
              }
          }
    }
  }
  size_t m0 = (size_t)n * n * n * 4;
  for (size_t i = 0; i < m0; ++i) grad0[i] += gpyr[i];
}

/* ---------------------------------------------------------------------- */
/* sampling (Ch. 4.5 colour supersampler, Ch. 4.3.3 texture filtering)      */
/* ---------------------------------------------------------------------- */
typedef struct {
  int level[2];
  double level_w[2];
  int base[2][3]; /* lower corner texel per axis                        */
  double frac[2][3];
} orc_stencil;

/* q: grid-normalized position ([0,1]^3 spans the grid), lambda: level. */
static void stencil(int n, int levels, const double q[3], double lambda,
                    orc_stencil *s) {
  double lc = lambda;
  if (!(lc > 0.0)) lc = 0.0; /* also maps NaN / -inf to level 0 */
  if (lc > levels - 1) lc = levels - 1;
  int l0 = (int)floor(lc);
  int l1 = l0 + 1 < levels ? l0 + 1 : levels - 1;
  double f = lc - l0;
  s->level[0] = l0;
  s->level[1] = l1;
  s->level_w[0] = 1.0 - f;
  s->level_w[1] = f;
  for (int k = 0; k < 2; ++k) {
    int nl = n >> s->level[k];
    for (int a = 0; a < 3; ++a) {
      double u = q[a] * nl - 0.5;
      double i0 = floor(u);
      s->base[k][a] = (int)i0;
      s->frac[k][a] = u - i0;
    }
  }
}

static double corner_weight(const orc_stencil *s, int k, int dx, int dy,
                            int dz) {
  double wx = dx ? s->frac[k][0] : 1.0 - s->frac[k][0];
  double wy = dy ? s->frac[k][1] : 1.0 - s->frac[k][1];
  double wz = dz ? s->frac[k][2] : 1.0 - s->frac[k][2];
  return s->level_w[k] * wx * wy * wz;
}

/* Trilinear lookup of stencil level k in the level array lv, times `scale`,
 * added to out. */
static void tri_add(const orc_stencil *s, int k, const double *lv, int nl, double scale,
                    double out[4]) {
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        int x = s->base[k][0] + dx, y = s->base[k][1] + dy, z = s->base[k][2] + dz;
        if (x < 0 || y < 0 || z < 0 || x >= nl || y >= nl || z >= nl)
          continue; /* outside the grid: empty */
        double w = scale * corner_weight(s, k, dx, dy, dz);
        const double *v = lv + (((size_t)z * nl + y) * nl + x) * 4;
        for (int c = 0; c < 4; ++c) out[c] += w * v[c];
      }
}

/* The quadrilinear sample of the stencil.  In an anisotropic pyramid a level
 * l >= 1 is read from the three volumes facing the direction of travel w,
 * weighted by w_a^2 / |w|^2 (the volume of the sign of w_a along axis a). */
static void aniso_dirs(const double *w, double wa[3], int dir[3]) {
  double w2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  for (int a = 0; a < 3; ++a) {
    wa[a] = w[a] * w[a] / w2;
    dir[a] = 2 * a + (w[a] < 0.0 ? 1 : 0);
  }
}

static void apply_stencil(const orc_grid *g, const orc_stencil *s, const double *w,
                          double out[4]) {
  out[0] = out[1] = out[2] = out[3] = 0.0;
  for (int k = 0; k < 2; ++k) {
    int nl = g->n >> s->level[k];
    if (g->aniso && s->level[k] >= 1) {
      double wa[3];
      int dir[3];
      aniso_dirs(w, wa, dir);
      for (int a = 0; a < 3; ++a) {
        if (wa[a] == 0.0) continue;
        tri_add(s, k, g->data + orc_aniso_offset(g->n, s->level[k], dir[a]), nl, wa[a], out);
      }
    } else {
      const double *lv = g->data + (g->aniso ? 0 : orc_level_offset(g->n, s->level[k]));
      tri_add(s, k, lv, nl, 1.0, out);
    }
  }
}

static void to_grid(const orc_grid *g, const double p[3], double q[3]) {
  for (int a = 0; a < 3; ++a) q[a] = (p[a] - g->origin[a]) / g->size;
}

/* sample(position, diameter) of Ch. 4.5 in scene units. */
void orc_sample(const double *pyr, int n, int levels, const double *origin,
                double size, const double *p, double diameter, double *out) {
  orc_grid g = {pyr, n, levels, {origin[0], origin[1], origin[2]}, size};
  double q[3];
  to_grid(&g, p, q);
  double h0 = size / n;
  orc_stencil s;
  stencil(n, levels, q, log2(diameter / h0), &s);
  apply_stencil(&g, &s, NULL, out);
}

/* Lookup at an explicit level (for tests of the filter itself). */
void orc_sample_lod(const double *pyr, int n, int levels, const double *q,
                    double lambda, double *out) {
  orc_grid g = {pyr, n, levels, {0.0, 0.0, 0.0}, 1.0};
  orc_stencil s;
  stencil(n, levels, q, lambda, &s);
  apply_stencil(&g, &s, NULL, out);
}

/* Lookup at an explicit level of an anisotropic pyramid for travel along w. */
void orc_sample_lod_aniso(const double *pyr, int n, int levels, const double *q,
                          double lambda, const double *w, double *out) {
  orc_grid g = {pyr, n, levels, {0.0, 0.0, 0.0}, 1.0, 1};
  orc_stencil s;
  stencil(n, levels, q, lambda, &s);
  apply_stencil(&g, &s, w, out);
}

/* ---------------------------------------------------------------------- */
/* one cone (Ch. 4.3.2 volume ray marching)                                */
/* ---------------------------------------------------------------------- */
typedef struct {
  double t, a, c[3], trans; /* step position, sample alpha/colour, T_k   */
  double sa;                /* d a / d (sampled alpha): the occlusion fade */
  orc_stencil st;
} orc_step;

typedef struct {
  double c[3], alpha;
  int64_t steps;
  double margin;     /* min |t - t_max| / t_max over the tested t values  */
  double hit_margin; /* min |a_s - 1/100| over first-hit tests (variant)  */
  int hit;           /* first-hit variant: the cone stopped on a sample    */
} orc_cone_result;

/* Marches one cone.  If `rec` is non-NULL the per-step state is stored
 * there (capacity `cap`) for the adjoint. */
/* GLSL smoothstep: Hermite interpolation between two edges. */
static double smoothstep(double e0, double e1, double x) {
  double t = (x - e0) / (e1 - e0);
  if (t < 0.0) t = 0.0;
  if (t > 1.0) t = 1.0;
  return t * t * (3.0 - 2.0 * t);
}

/* kind: 0 diffuse, 1 specular, 2 occlusion (selects the Ch. 5.4.4 variants
 * enabled in P->flags). */
static void march_kind(const orc_grid *g, const double o[3], const double w[3],
                       double aperture, const orc_params *P, int kind,
                       orc_cone_result *res, orc_step *rec, int64_t cap);

static void march_kind(const orc_grid *g, const double o[3], const double w[3],
                       double aperture, const orc_params *P, int kind,
                       orc_cone_result *res, orc_step *rec, int64_t cap) {
  const int occ_smooth = kind == 2 && (P->flags & ORC_OCC_SMOOTH);
  const int first_hit = kind == 0 && (P->flags & ORC_DIFF_FIRST);
  double hit_margin = INFINITY;
  double h0 = g->size / g->n;
  double tan_half = tan(0.5 * aperture);
  double t = P->t0_voxels * h0;
  double alpha = 0.0, c[3] = {0.0, 0.0, 0.0};
  double margin = INFINITY;
  int64_t k = 0;
  res->hit = 0;
  for (;;) {
    double m = fabs(t - P->t_max) / P->t_max;
    if (m < margin) margin = m;
    if (!(alpha < 1.0 && t <= P->t_max)) break;
    double d = 2.0 * t * tan_half; /* sampling diameter */
    double p[3], q[3];
    for (int a = 0; a < 3; ++a) p[a] = o[a] + t * w[a];
    to_grid(g, p, q);
    orc_stencil st;
    stencil(g->n, g->levels, q, log2(d / h0), &st);
    double v[4];
    apply_stencil(g, &st, w, v);
    if (first_hit) {
      /* Ch. 5.4.4 diffuse cone: the first sample whose opacity exceeds
       * 1/100 ends the trace and its colour is returned. */
      if (fabs(v[3] - 0.01) < hit_margin) hit_margin = fabs(v[3] - 0.01);
      if (v[3] > 0.01) {
        for (int ch = 0; ch < 3; ++ch) c[ch] = v[ch];
        alpha = 1.0;
        if (rec && k < cap) { /* the returned sample, for the adjoint */
          rec[k].t = t;
          rec[k].a = v[3];
          for (int ch = 0; ch < 3; ++ch) rec[k].c[ch] = v[ch];
          rec[k].trans = 1.0;
          rec[k].sa = 1.0;
          rec[k].st = st;
        }
        res->hit = 1;
        ++k;
        break;
      }
      t += P->beta * d;
      ++k;
      continue;
    }
    double fade = 1.0;
    if (occ_smooth) /* Ch. 5.4.4 occlusion cone: fade near the apex */
      fade = smoothstep(0.0, P->occ_max_dist, sqrt(t) * P->shadow_str);
    v[3] *= fade;
    if (rec && k < cap) {
      rec[k].t = t;
      rec[k].sa = fade;
      rec[k].a = v[3];
      rec[k].c[0] = v[0];
      rec[k].c[1] = v[1];
      rec[k].c[2] = v[2];
      rec[k].trans = 1.0 - alpha;
      rec[k].st = st;
    }
    double wgt = (1.0 - alpha) * v[3];
    /* Straight colour: c += (1 - alpha) a_s c_s (Ch. 4.3.2, reading of the
     * garbled colour line); premultiplied colour: c += (1 - alpha) c_s. */
    double cw = (P->flags & ORC_PREMUL) ? (1.0 - alpha) : wgt;
    for (int ch = 0; ch < 3; ++ch) c[ch] += cw * v[ch];
    alpha += wgt;
    t += P->beta * d;
    ++k;
  }
  for (int ch = 0; ch < 3; ++ch) res->c[ch] = c[ch];
  res->alpha = alpha;
  res->steps = k;
  res->margin = margin;
  res->hit_margin = hit_margin;
}

/* Public single-cone entry (scene units); kind selects the Ch. 5.4.4
 * variant enabled in P->flags (0 diffuse, 1 specular, 2 occlusion, -1 none). */
void orc_trace_cone(const double *pyr, int n, int levels, const double *origin,
                    double size, const double *apex, const double *dir,
                    double aperture, const orc_params *P, int kind, double *out_rgba,
                    int64_t *steps) {
  orc_grid g = {pyr, n, levels, {origin[0], origin[1], origin[2]}, size,
                (P->flags & ORC_ANISO) != 0};
  orc_cone_result r;
  march_kind(&g, apex, dir, aperture, P, kind, &r, NULL, 0);
  out_rgba[0] = r.c[0];
  out_rgba[1] = r.c[1];
  out_rgba[2] = r.c[2];
  out_rgba[3] = r.alpha;
  if (steps) *steps = r.steps;
}

/* ---------------------------------------------------------------------- */
/* per-pixel cone set (Ch. 4.2)                                            */
/* ---------------------------------------------------------------------- */
typedef struct {
  int count;
  int kind[ORC_MAX_DIFFUSE + 2]; /* 0 diffuse, 1 specular, 2 occlusion */
  double weight[ORC_MAX_DIFFUSE + 2];
  double dir[ORC_MAX_DIFFUSE + 2][3];
  double aperture[ORC_MAX_DIFFUSE + 2];
  double apex[3];
} orc_coneset;

static void normalize3(double v[3]) {
  double l = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  v[0] /= l;
  v[1] /= l;
  v[2] /= l;
}

static void cross3(const double a[3], const double b[3], double r[3]) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}

void orc_tangent_frame(const double *nrm, double *T, double *B) {
  double a[3] = {0.0, 0.0, 0.0};
  if (fabs(nrm[0]) < 0.9)
    a[0] = 1.0;
  else
    a[1] = 1.0;
  cross3(a, nrm, T);
  normalize3(T);
  cross3(nrm, T, B);
}

static void cone_set(const orc_grid *g, const orc_view *v, size_t px,
                     const orc_params *P, orc_coneset *cs) {
  double x[3], nrm[3];
  for (int a = 0; a < 3; ++a) {
    x[a] = v->position[3 * px + a];
    nrm[a] = v->normal[3 * px + a];
  }
  double h0 = g->size / g->n;
  for (int a = 0; a < 3; ++a)
    cs->apex[a] = x[a] + P->normal_offset_voxels * h0 * nrm[a];
  double T[3], B[3];
  orc_tangent_frame(nrm, T, B);
  int c = 0;
  for (int k = 0; k < P->n_diffuse; ++k, ++c) {
    const double *d = P->diffuse_dir[k];
    cs->kind[c] = 0;
    cs->weight[c] = P->diffuse_weight[k];
    cs->aperture[c] = P->diffuse_aperture;
    for (int a = 0; a < 3; ++a)
      cs->dir[c][a] = T[a] * d[0] + B[a] * d[1] + nrm[a] * d[2];
  }
  if (P->spec_enable) {
    double view[3];
    for (int a = 0; a < 3; ++a) view[a] = x[a] - v->camera[a];
    normalize3(view);
    double vn = view[0] * nrm[0] + view[1] * nrm[1] + view[2] * nrm[2];
    cs->kind[c] = 1;
    cs->weight[c] = 1.0;
    for (int a = 0; a < 3; ++a) cs->dir[c][a] = view[a] - 2.0 * vn * nrm[a];
    double ap = P->spec_aperture_min;
    if (v->roughness) {
      double f = (v->roughness[px] - P->roughness_min) / (1.0 - P->roughness_min);
      if (f < 0.0) f = 0.0;
      if (f > 1.0) f = 1.0;
      ap = P->spec_aperture_min + f * (P->spec_aperture_max - P->spec_aperture_min);
    }
    cs->aperture[c] = ap;
    ++c;
  }
  if (P->occ_enable) {
    cs->kind[c] = 2;
    cs->weight[c] = 1.0;
    cs->aperture[c] = P->occ_aperture;
    for (int a = 0; a < 3; ++a) cs->dir[c][a] = P->light_dir[a];
    ++c;
  }
  cs->count = c;
}

/* The cone set of one pixel, for tests of the per-pixel set-up: apex[3],
 * and per cone kind / weight / aperture / direction[3].  Returns the count. */
int orc_cone_set(const double *origin, double size, int n, const orc_view *v,
                 int64_t px, const orc_params *P, double *apex, int *kind,
                 double *weight, double *aperture, double *dir) {
  orc_grid g = {NULL, n, 1, {origin[0], origin[1], origin[2]}, size};
  orc_coneset cs;
  cone_set(&g, v, (size_t)px, P, &cs);
  for (int a = 0; a < 3; ++a) apex[a] = cs.apex[a];
  for (int c = 0; c < cs.count; ++c) {
    kind[c] = cs.kind[c];
    weight[c] = cs.weight[c];
    aperture[c] = cs.aperture[c];
    for (int a = 0; a < 3; ++a) dir[3 * c + a] = cs.dir[c][a];
  }
  return cs.count;
}

/*
 * Traces the pixels `idx[0..count)` of one view (all pixels if idx == NULL,
 * count = W*H).  Outputs are per listed pixel: D[4], S[4], Vis[1].
 * steps[3] accumulates the number of samples per cone kind, cones[3] the
 * number of cones, margin receives min |t - t_max| / t_max.
 */
/* Ch. 5.4.4 specular BRDF with angular grace p = 0.008 pi shininess:
 * (1 - max(0, acos(w . l) - p) / pi)^q, q = shininess_falloff, w the cone
 * axis (mirror direction) and l the direction towards the light. */
static double spec_grace(const double w[3], const orc_params *P) {
  double wl = w[0] * P->light_dir[0] + w[1] * P->light_dir[1] + w[2] * P->light_dir[2];
  double wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  double ln = sqrt(P->light_dir[0] * P->light_dir[0] + P->light_dir[1] * P->light_dir[1] +
                   P->light_dir[2] * P->light_dir[2]);
  double cosg = wl / (wn * ln);
  if (cosg > 1.0) cosg = 1.0;
  if (cosg < -1.0) cosg = -1.0;
  const double pi = 3.14159265358979323846;
  double gn = acos(cosg) - 0.008 * pi * P->shininess;
  if (gn < 0.0) gn = 0.0;
  return pow(1.0 - gn / pi, P->shininess_falloff);
}

double orc_spec_grace(const double *w, const orc_params *P) { return spec_grace(w, P); }

/* Shading epilogue.  Direct light of the Phong model as in the thesis's
 * GLSL listing (Ch. 3.3) for one directional light: diffuse max(n.l, 0),
 * glossy max(w.R, 0)^shininess with R = reflect(-l, n) and w towards the
 * viewer, both times the light colour and the material colour.  L_vxct
 * (Ch. 4.2.2) replaces the ambient term by the indirect light:
 *   L = albedo (c_d D + c_s S) + Vis direct;
 * L_impl (Ch. 5.4.4): L = o_min D + S + Vis direct (o_min = Vis, one light). */
/* The direct light of pixel px (Ch. 3.3 Phong listing, one directional
 * light) and its albedo. */
static void shade_direct(const orc_view *v, size_t px, const orc_params *P, double direct[3],
                         double alb[3]) {
  double x[3], n[3];
  for (int a = 0; a < 3; ++a) {
    x[a] = v->position[3 * px + a];
    n[a] = v->normal[3 * px + a];
    alb[a] = v->albedo ? v->albedo[3 * px + a] : 1.0;
  }
  const double *l = P->light_dir;
  double nl = n[0] * l[0] + n[1] * l[1] + n[2] * l[2];
  double R[3], w[3];
  for (int a = 0; a < 3; ++a) {
    R[a] = -l[a] + 2.0 * nl * n[a];
    w[a] = v->camera[a] - x[a];
  }
  normalize3(w);
  double wr = w[0] * R[0] + w[1] * R[1] + w[2] * R[2];
  double diff = nl > 0.0 ? nl : 0.0;
  double gloss = pow(wr > 0.0 ? wr : 0.0, P->shininess);
  for (int ch = 0; ch < 3; ++ch)
    direct[ch] = P->light_color[ch] * alb[ch] * (P->diffuse_str * diff + P->specular_str * gloss);
}

static void shade(const orc_view *v, size_t px, const orc_params *P, const double *D,
                  const double *S, double vis, double *out) {
  double direct[3], alb[3];
  shade_direct(v, px, P, direct, alb);
  for (int ch = 0; ch < 3; ++ch) {
    if (P->flags & ORC_SHADE_IMPL)
      out[ch] = vis * D[ch] + S[ch] + vis * direct[ch];
    else
      out[ch] = alb[ch] * (P->diffuse_str * D[ch] + P->specular_str * S[ch]) + vis * direct[ch];
  }
  out[3] = 1.0;
}

/* Partial derivatives of shade()'s L_ch with respect to D_ch, S_ch and Vis
 * (L_ch depends on no other channel; L.a is the constant 1). */
static void shade_partials(const orc_view *v, size_t px, const orc_params *P, const double *D,
                           double vis, double dD[3], double dS[3], double dV[3]) {
  double direct[3], alb[3];
  shade_direct(v, px, P, direct, alb);
  for (int ch = 0; ch < 3; ++ch) {
    if (P->flags & ORC_SHADE_IMPL) {
      dD[ch] = vis;
      dS[ch] = 1.0;
      dV[ch] = D[ch] + direct[ch];
    } else {
      dD[ch] = alb[ch] * P->diffuse_str;
      dS[ch] = alb[ch] * P->specular_str;
      dV[ch] = direct[ch];
    }
  }
}

/* D, S (RGBA) and Vis of one pixel; the per-kind step and cone counts and
 * the margins accumulate into st, cn, mg, hm when those are non-NULL. */
static void pixel_outputs(const orc_grid *g, const orc_view *v, size_t px, const orc_params *P,
                          double *d, double *s, double *vis, int64_t *st, int64_t *cn,
                          double *mg, double *hm) {
  d[0] = d[1] = d[2] = d[3] = 0.0;
  s[0] = s[1] = s[2] = s[3] = 0.0;
  *vis = 1.0;
  orc_coneset cs;
  cone_set(g, v, px, P, &cs);
  for (int c = 0; c < cs.count; ++c) {
    orc_cone_result r;
    march_kind(g, cs.apex, cs.dir[c], cs.aperture[c], P, cs.kind[c], &r, NULL, 0);
    if (st) st[cs.kind[c]] += r.steps;
    if (cn) cn[cs.kind[c]] += 1;
    if (mg && r.margin < *mg) *mg = r.margin;
    if (hm && r.hit_margin < *hm) *hm = r.hit_margin;
    if (cs.kind[c] == 0) {
      for (int ch = 0; ch < 3; ++ch) d[ch] += cs.weight[c] * r.c[ch];
      d[3] += cs.weight[c] * r.alpha;
    } else if (cs.kind[c] == 1) {
      double f = 1.0;
      if (P->flags & ORC_SPEC_GRACE) f = spec_grace(cs.dir[c], P);
      for (int ch = 0; ch < 3; ++ch) s[ch] = f * r.c[ch];
      s[3] = r.alpha;
    } else {
      *vis = 1.0 - r.alpha;
    }
  }
}

void orc_trace(const double *pyr, int n, int levels, const double *origin,
               double size, const orc_view *v, const orc_params *P,
               const int64_t *idx, int64_t count, double *D, double *S,
               double *Vis, double *L, int64_t *steps, int64_t *cones, double *margin,
               double *hit_margin) {
  orc_grid g = {pyr, n, levels, {origin[0], origin[1], origin[2]}, size,
                (P->flags & ORC_ANISO) != 0};
  int64_t st[3] = {0, 0, 0}, cn[3] = {0, 0, 0};
  double mg = INFINITY, hm = INFINITY;
#pragma omp parallel
  {
    int64_t lst[3] = {0, 0, 0}, lcn[3] = {0, 0, 0};
    double lmg = INFINITY, lhm = INFINITY;
#pragma omp for schedule(dynamic, 64)
    for (int64_t i = 0; i < count; ++i) {
      size_t px = idx ? (size_t)idx[i] : (size_t)i;
      double *d = D + 4 * i, *s = S + 4 * i;
      d[0] = d[1] = d[2] = d[3] = 0.0;
      s[0] = s[1] = s[2] = s[3] = 0.0;
      Vis[i] = 1.0;
      if (L) L[4 * i] = L[4 * i + 1] = L[4 * i + 2] = L[4 * i + 3] = 0.0;
      if (v->mask && !v->mask[px]) continue;
      pixel_outputs(&g, v, px, P, d, s, &Vis[i], lst, lcn, &lmg, &lhm);
      if (L && (P->flags & ORC_SHADE)) shade(v, px, P, d, s, Vis[i], L + 4 * i);
    }
#pragma omp critical
    {
      for (int k = 0; k < 3; ++k) {
        st[k] += lst[k];
        cn[k] += lcn[k];
      }
      if (lmg < mg) mg = lmg;
      if (lhm < hm) hm = lhm;
    }
  }
  if (hit_margin && hm < *hit_margin) *hit_margin = hm;
  if (steps)
    for (int k = 0; k < 3; ++k) steps[k] += st[k];
  if (cones)
    for (int k = 0; k < 3; ++k) cones[k] += cn[k];
  if (margin && mg < *margin) *margin = mg;
}

/* ---------------------------------------------------------------------- */
/* adjoint                                                                 */
/* ---------------------------------------------------------------------- */
/*
 * For one cone with samples (c_k, a_k), k = 0..K-1, and transmittance
 * T_k = prod_{j<k} (1 - a_j):
 *   C = sum_k T_k a_k c_k,   A = 1 - prod_k (1 - a_k).
 *   dC/dc_k = T_k a_k
 *   dC/da_k = T_k (c_k - R_{k+1}),  R_k = a_k c_k + (1 - a_k) R_{k+1}, R_K = 0
 *   dA/da_k = T_k Q_{k+1},          Q_k = (1 - a_k) Q_{k+1},           Q_K = 1
 * With premultiplied sample colour (C = sum_k T_k c_k):
 *   dC/dc_k = T_k,  dC/da_k = -T_k R'_{k+1},  R'_k = c_k + (1 - a_k) R'_{k+1}.
 * The occlusion fade scales the sampled alpha by a factor of t alone, so the
 * texel alpha receives dL/da_k times that factor.  A first-hit diffuse cone
 * returns (c_k, 1) of its hit sample: only that sample's colour has a
 * derivative (the choice of the sample is piecewise constant).
 * The step schedule does not depend on the voxel values (only the stopping
 * step does, which is piecewise constant), so these are the derivatives.
 */
static void scatter_level(const orc_stencil *st, int lk, double *lv, int nl, double scale,
                          const double dc[3], double da) {
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        int x = st->base[lk][0] + dx, y = st->base[lk][1] + dy, z = st->base[lk][2] + dz;
        if (x < 0 || y < 0 || z < 0 || x >= nl || y >= nl || z >= nl)
          continue;
        double w = scale * corner_weight(st, lk, dx, dy, dz);
        if (w == 0.0) continue;
        double *t = lv + (((size_t)z * nl + y) * nl + x) * 4;
        for (int ch = 0; ch < 3; ++ch) {
#pragma omp atomic
          t[ch] += w * dc[ch];
        }
#pragma omp atomic
        t[3] += w * da;
      }
}

/* The transpose of apply_stencil for one sample of a cone of axis w: the
 * derivatives reach each texel through its trilinear and level weights (and,
 * in an anisotropic pyramid, the direction weight of its volume). */
static void scatter_sample(const orc_grid *g, double *gpyr, const orc_step *s, const double *w,
                           const double dc[3], double da) {
  for (int lk = 0; lk < 2; ++lk) {
    int l = s->st.level[lk], nl = g->n >> l;
    if (g->aniso && l >= 1) {
      double wa[3];
      int dir[3];
      aniso_dirs(w, wa, dir);
      for (int a = 0; a < 3; ++a) {
        if (wa[a] == 0.0) continue;
        scatter_level(&s->st, lk, gpyr + orc_aniso_offset(g->n, l, dir[a]), nl, wa[a], dc, da);
      }
    } else {
      double *lv = gpyr + (g->aniso ? 0 : orc_level_offset(g->n, l));
      scatter_level(&s->st, lk, lv, nl, 1.0, dc, da);
    }
  }
}

static void cone_adjoint(const orc_grid *g, double *gpyr, const orc_step *rec,
                         const orc_cone_result *r, const double *w, int first_hit, int premul,
                         const double gc[3], double ga) {
  if (first_hit) {
    if (r->hit) scatter_sample(g, gpyr, rec + r->steps - 1, w, gc, 0.0);
    return;
  }
  double R[3] = {0.0, 0.0, 0.0}, Q = 1.0;
  for (int64_t k = r->steps - 1; k >= 0; --k) {
    const orc_step *s = rec + k;
    double dc[3], da = 0.0;
    for (int ch = 0; ch < 3; ++ch) {
      if (premul) {
        dc[ch] = gc[ch] * s->trans;
        da -= gc[ch] * s->trans * R[ch];
      } else {
        dc[ch] = gc[ch] * s->trans * s->a;
        da += gc[ch] * s->trans * (s->c[ch] - R[ch]);
      }
    }
    da += ga * s->trans * Q;
    for (int ch = 0; ch < 3; ++ch)
      R[ch] = (premul ? s->c[ch] : s->a * s->c[ch]) + (1.0 - s->a) * R[ch];
    Q = (1.0 - s->a) * Q;
    scatter_sample(g, gpyr, s, w, dc, da * s->sa);
  }
}

/*
 * Gradient of L with respect to the level-0 grid, given dL/dD, dL/dS and
 * dL/dVis for the listed pixels (same layout as orc_trace's outputs).
 * gpyr is caller scratch of orc_level_offset(n, levels) doubles, or of
 * orc_aniso_offset(n, levels, 0) for an anisotropic pyramid (ORC_ANISO in
 * P->flags), zeroed here; the level-0 gradient is ADDED into grad0
 * ([n][n][n][4]).  With grad0 NULL the mip adjoint is skipped and gpyr keeps
 * the gradient of every texel of every level.
 */
void orc_trace_backward(const double *pyr, int n, int levels,
                        const double *origin, double size, const orc_view *v,
                        const orc_params *P, const int64_t *idx, int64_t count,
                        const double *gD, const double *gS, const double *gV,
                        const double *gL, double *gpyr, double *grad0) {
  orc_grid g = {pyr, n, levels, {origin[0], origin[1], origin[2]}, size,
                (P->flags & ORC_ANISO) != 0};
  memset(gpyr, 0, (g.aniso ? orc_aniso_offset(n, levels, 0) : orc_level_offset(n, levels)) *
                      sizeof(double));
#pragma omp parallel
  {
    int64_t cap = 4096;
    orc_step *rec = (orc_step *)malloc(sizeof(orc_step) * cap);
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < count; ++i) {
      size_t px = idx ? (size_t)idx[i] : (size_t)i;
      if (v->mask && !v->mask[px]) continue;
      /* upstream gradients of D, S, Vis, plus those the shaded radiance
       * passes down (its chain rule through shade()) */
      double pD[4], pS[4], pV = gV ? gV[i] : 0.0;
      for (int ch = 0; ch < 4; ++ch) {
        pD[ch] = gD[4 * i + ch];
        pS[ch] = gS[4 * i + ch];
      }
      if (gL && (P->flags & ORC_SHADE)) {
        double d[4], s[4], vis, dD[3], dS[3], dV[3];
        pixel_outputs(&g, v, px, P, d, s, &vis, NULL, NULL, NULL, NULL);
        shade_partials(v, px, P, d, vis, dD, dS, dV);
        for (int ch = 0; ch < 3; ++ch) {
          pD[ch] += gL[4 * i + ch] * dD[ch];
          pS[ch] += gL[4 * i + ch] * dS[ch];
          pV += gL[4 * i + ch] * dV[ch];
        }
      }
      orc_coneset cs;
      cone_set(&g, v, px, P, &cs);
      for (int c = 0; c < cs.count; ++c) {
        orc_cone_result r;
        march_kind(&g, cs.apex, cs.dir[c], cs.aperture[c], P, cs.kind[c], &r, rec, cap);
        if (r.steps > cap) { /* grow and redo */
          cap = r.steps;
          rec = (orc_step *)realloc(rec, sizeof(orc_step) * cap);
          march_kind(&g, cs.apex, cs.dir[c], cs.aperture[c], P, cs.kind[c], &r, rec, cap);
        }
        double gc[3] = {0.0, 0.0, 0.0}, ga = 0.0;
        if (cs.kind[c] == 0) {
          for (int ch = 0; ch < 3; ++ch) gc[ch] = cs.weight[c] * pD[ch];
          ga = cs.weight[c] * pD[3];
        } else if (cs.kind[c] == 1) {
          /* the angular-grace factor scales the specular colour only */
          double f = (P->flags & ORC_SPEC_GRACE) ? spec_grace(cs.dir[c], P) : 1.0;
          for (int ch = 0; ch < 3; ++ch) gc[ch] = f * pS[ch];
          ga = pS[3];
        } else {
          ga = -pV;
        }
        const int first_hit = cs.kind[c] == 0 && (P->flags & ORC_DIFF_FIRST);
        cone_adjoint(&g, gpyr, rec, &r, cs.dir[c], first_hit, (P->flags & ORC_PREMUL) != 0, gc,
                     ga);
      }
    }
    free(rec);
  }
  if (!grad0) return; /* the per-level gradients stay in gpyr */
  if (g.aniso)
    orc_mip_adjoint_aniso(pyr, gpyr, n, levels, grad0);
  else
    orc_mip_adjoint(gpyr, n, levels, grad0);
}

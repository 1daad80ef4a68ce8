/*
 * vct.h — C ABI of the GB300 voxel-cone-tracing library (libvct.so).
 *
 * The library implements the data-parallel hot path of voxel cone tracing as
 * defined in B. Kahl, "Real-Time Global Illumination Using OpenGL And Voxel
 * Cone Tracing" (2019):
 *   - building the mip pyramid of an RGBA voxel grid by 2x2x2 averaging
 *     (Ch. 4.3.3, "Mipmaps" and "Texture Filtering"; Ch. 5.4.4 voxelize()),
 *   - for every G-buffer pixel, marching diffuse cones over the normal
 *     hemisphere, one specular cone along the reflection direction and one
 *     occlusion cone towards the light (Ch. 4.2), each by the volume ray
 *     march of Ch. 4.3.2 (diameter d = 2 t tan(gamma/2), step t += beta d,
 *     front-to-back accumulation) with the sampler of Ch. 4.5 (mip level
 *     log2(d / voxel size), quadrilinear lookup),
 *   - and the adjoint of both (no counterpart in the thesis).
 *
 * Conventions for every entry point
 *   - Device pointers are caller-owned CUDA device memory; the library never
 *     allocates, frees or retains them past the call.  Host pointers (the
 *     structs below) are read during the call only.
 *   - All work is enqueued asynchronously on `stream` (a cudaStream_t; NULL is
 *     the legacy default stream).  A return value other than VCT_OK means
 *     that nothing was enqueued (argument validation) or that a launch failed
 *     (VCT_ERR_CUDA).  Faults inside kernels surface at the caller's next
 *     synchronisation.  The library never aborts, exits or throws.
 *   - vct_last_error() returns a thread-local description of the last
 *     failure on the calling thread.
 *   - Scene units: the grid of a pyramid spans [origin, origin + size]^3.
 *     Level 0 has n voxels per axis (voxel edge h0 = size / n); level l has
 *     n >> l texels per axis with centres at origin + (i + 1/2) size/(n>>l).
 *     Texels outside the grid read as zero (empty space).
 */
#ifndef VCT_H
#define VCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t without including the CUDA headers. */
typedef struct CUstream_st *vct_stream_t;

typedef enum {
  VCT_OK = 0,
  VCT_ERR_INVALID_ARG = 1, /* a pointer, size or parameter is out of range   */
  VCT_ERR_CUDA = 2,        /* a CUDA runtime call or kernel launch failed     */
  VCT_ERR_WORKSPACE = 3,   /* workspace missing or smaller than required      */
  VCT_ERR_UNSUPPORTED = 4, /* valid request the library does not implement     */
  VCT_ERR_TIMEOUT = 5      /* a bounded device-side wait gave up              */
} vct_status;

typedef enum { VCT_F32 = 0, VCT_F16 = 1 } vct_dtype;

#define VCT_MAX_DIFFUSE 32
#define VCT_MAX_PYRAMIDS 8
#define VCT_MAX_LEVELS 11

/* ------------------------------------------------------------------------ */
/* Pyramid storage                                                          */
/* ------------------------------------------------------------------------ */
/*
 * A mip pyramid in caller-owned device memory (Ch. 4.3.3).
 *
 * Layout of `data` (vct_pyramid_bytes() bytes, 256-byte aligned):
 *   [256-byte header][level 0][level 1]...[level levels-1][FP32 staging]
 * Each level starts at vct_pyramid_level_offset().  Within level l the texel
 * at integer coordinates (x, y, z) sits at index morton(x, y, z), the bit
 * interleave with x in bits 0,3,6,..., y in bits 1,4,7,... and z in bits
 * 2,5,8,...  Because every level edge is a power of two this is the same as
 * 8x8x8 bricks stored in Morton order of their brick coordinates with the
 * texels of each brick in Morton order, and the 8 children of texel j of
 * level l+1 are texels 8j..8j+7 of level l.  A texel is RGBA: four float32
 * (16 bytes) for VCT_F32 or four IEEE binary16 (8 bytes) for VCT_F16.  The
 * header holds a device status word written by bounded waits
 * (vct_pyramid_status).  The FP32 staging area exists for VCT_F16 only and
 * holds the unrounded values of one intermediate level during the build.
 *
 * VCT_LAYOUT_BRICKS (sparse storage: the brick pool of Crassin et al.'s
 * sparse voxel octree, Ch. 5.1 "Previous Work", with one flat slot table per
 * level instead of the tree): every level with at least 16 texels per axis
 * is cut into the 8x8x8 bricks above (brick id = morton(x, y, z) >> 9, its
 * texels the 512 consecutive Morton codes) and stores one uint32 slot per
 * brick instead of texels.  The bricks live in a pool shared by all levels:
 * slot 0 is an all-zero brick to which every empty brick points, occupied
 * bricks take slots 1, 2, ... in level order, then brick order.  A level-0
 * brick is occupied if any channel of any of its texels is non-zero; a brick
 * of level l+1 if any of its 8 child bricks is.  Smaller levels are stored
 * dense.  Layout:
 *   [256-byte header][per level: slot table or texels][FP32 staging][pool]
 * The header also holds the occupied-brick count (uint64 at byte 8).  The
 * texel values are exactly those of the dense layout; only empty bricks are
 * not stored.  vct_pyramid_plan_bricks() sizes such a pyramid.
 */
#define VCT_LAYOUT_DENSE 0
#define VCT_LAYOUT_BRICKS 1
/*
 * VCT_LAYOUT_ANISO (VCT_F32 only): anisotropic mips (Villegas' anisotropic
 * filtering, Ch. 5.1).  Level 0 is the isotropic grid; every level l >= 1
 * holds six volumes, one per direction of travel d = +x, -x, +y, -y, +z, -z
 * (index 2 axis + (sign < 0)), each in the level's Morton order.  Level 0
 * starts at byte 256 as in the dense layout; level l >= 1 follows level
 * l - 1 (each level's size rounded up to 256 bytes) and holds its six
 * volumes back to back (volume d at + d * (n >> l)^3 * 16).  These offsets
 * differ from vct_pyramid_level_offset()'s, which is the dense layout's:
 * read a volume with vct_pyramid_read_volume().
 * A texel of volume d at level l+1 is the straight 4-channel mean over the
 * four child pairs along axis(d) of the pair seen along d (front = the child
 * met first): alpha = a_f + (1 - a_f) a_b, colour = (a_f c_f + (1 - a_f)
 * a_b c_b) / alpha (0 where alpha = 0); the children are level 0's texels
 * for l = 0, else volume d of level l.  vct_trace samples a level l >= 1
 * for a cone of axis w as sum_a (w_a^2 / |w|^2) * (volume of axis a facing
 * the sign of w_a); level 0 as usual.  vct_trace_backward differentiates
 * through both (see there).
 */
#define VCT_LAYOUT_ANISO 2

typedef struct {
  int32_t n;        /* level-0 voxels per axis: a power of two in [2, 1024]  */
  int32_t levels;   /* number of levels, 1 .. log2(n) + 1                    */
  int32_t dtype;    /* vct_dtype of the stored texels                        */
  int32_t layout;   /* VCT_LAYOUT_DENSE, VCT_LAYOUT_BRICKS or VCT_LAYOUT_ANISO */
  float origin[3];  /* scene position of the grid's minimum corner           */
  float size;       /* scene edge length of the grid, > 0                    */
  void *data;       /* device memory, >= vct_pyramid_bytes(n, levels, dtype) */
  uint64_t bytes;   /* size of `data` in bytes                               */
} vct_pyramid;

/* Bytes a dense pyramid of this shape needs; 0 if the shape is invalid. */
size_t vct_pyramid_bytes(int32_t n, int32_t levels, int32_t dtype);

/* Bytes a VCT_LAYOUT_BRICKS pyramid of this shape with `occupied` occupied
 * bricks (all levels) needs; 0 if the shape is invalid. */
size_t vct_pyramid_bytes_bricks(int32_t n, int32_t levels, int32_t dtype, uint64_t occupied);

/* Device scratch vct_pyramid_plan_bricks needs (the fixed part of the brick
 * layout: header, slot tables, small levels, staging); 0 if invalid. */
size_t vct_pyramid_plan_scratch_bytes(int32_t n, int32_t levels, int32_t dtype);

/*
 * Counts the bricks that a VCT_LAYOUT_BRICKS pyramid of the dense level-0
 * grid `level0_dense` ([n][n][n][4] float32, 16-byte aligned) occupies and
 * returns that count and vct_pyramid_bytes_bricks() for it.  Runs on
 * `stream` and waits for it (the host needs the count to allocate).
 * scratch: vct_pyramid_plan_scratch_bytes() bytes of device memory,
 * 256-byte aligned, overwritten.
 */
vct_status vct_pyramid_plan_bricks(const float *level0_dense, int32_t n, int32_t levels,
                                   int32_t dtype, void *scratch, size_t scratch_bytes,
                                   uint64_t *occupied_out, uint64_t *bytes_out,
                                   vct_stream_t stream);

/* Bytes a VCT_LAYOUT_ANISO pyramid of this shape needs; 0 if the shape is
 * invalid or dtype is not VCT_F32. */
size_t vct_pyramid_bytes_aniso(int32_t n, int32_t levels, int32_t dtype);

/* Byte offset of `level` from pyramid.data in the dense layout; 0 if the
 * arguments are invalid (level 0 itself starts at 256). */
uint64_t vct_pyramid_level_offset(int32_t n, int32_t levels, int32_t dtype,
                                  int32_t level);

/*
 * Builds every level of `pyr` from a dense level-0 grid: the mipmaps of the
 * voxel texture (Ch. 4.3.3, "Mipmaps" and "Texture Filtering": each level
 * halves the resolution, a texel the average of the 2x2x2 texels below it;
 * Ch. 5.4.4 voxelize(): generated after every voxelization), stored in
 * Morton order.
 *   level0_dense: device float32 [n][n][n][4] laid out z, y, x, channel
 *                 (RGB radiance, A opacity), 16-byte aligned, read only.
 *   pyr:          describes the destination; pyr->data is written.
 * Level l+1 is the plain average of the 8 children of level l, computed in
 * float32 from the float32 values of level l; VCT_F16 pyramids store each
 * level rounded to nearest-even after it has been computed in float32.
 * A 32-byte aligned level0_dense of n >= 32 (binary16: n <= 256) is read
 * once in rows by one streaming kernel (the faster path), any other through
 * shared-memory blocks; for the dense and brick layouts both give the same
 * bits, for VCT_LAYOUT_ANISO (streamed for n >= 16) they agree within a few
 * ulps (reciprocals are rounded differently).
 * A VCT_LAYOUT_BRICKS pyramid gets the same texel values; its occupancy is
 * recomputed from level0_dense.  If its pool cannot hold the occupied bricks
 * (pyr->bytes below vct_pyramid_bytes_bricks() for this grid) every brick is
 * left empty and vct_pyramid_status() reports VCT_ERR_WORKSPACE.
 * Errors: VCT_ERR_INVALID_ARG for a NULL or misaligned pointer, a bad shape
 * or pyr->bytes below the layout's fixed part; VCT_ERR_CUDA if a launch fails.
 */
vct_status vct_build_mips(const float *level0_dense, const vct_pyramid *pyr,
                          vct_stream_t stream);

/*
 * Copies level `level` of `pyr` into a dense float32 array
 * [m][m][m][4] (m = n >> level, z, y, x, channel) at `dense_out` (device).
 */
vct_status vct_pyramid_read_level(const vct_pyramid *pyr, int32_t level,
                                  float *dense_out, vct_stream_t stream);

/*
 * Like vct_pyramid_read_level for one directional volume (0..5 = +x, -x,
 * +y, -y, +z, -z) of level `level` >= 1 of a VCT_LAYOUT_ANISO pyramid;
 * direction must be 0 for level 0 and for the other layouts.
 */
vct_status vct_pyramid_read_volume(const vct_pyramid *pyr, int32_t level, int32_t direction,
                                   float *dense_out, vct_stream_t stream);

/*
 * Synchronises `stream`, then reads and clears the status word in the
 * pyramid header.  Returns VCT_ERR_TIMEOUT if a kernel that wrote this
 * pyramid gave up a bounded wait (the pyramid contents are then undefined),
 * VCT_ERR_WORKSPACE if a brick pyramid's pool was too small for its occupied
 * bricks (see vct_build_mips), VCT_OK otherwise.
 */
vct_status vct_pyramid_status(const vct_pyramid *pyr, vct_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Cone tracing                                                             */
/* ------------------------------------------------------------------------ */
/*
 * Variant flags (vct_trace_params.flags).  The first three are the thesis's
 * modified cones (Ch. 5.4.4); the last two add the shading epilogue.
 *   VCT_FLAG_OCC_SMOOTH       occlusion cone: every sample opacity is scaled
 *                             by smoothstep(0, occ_max_dist, sqrt(t) *
 *                             shadow_str), t the distance travelled
 *   VCT_FLAG_SPEC_GRACE       specular colour times the angular-grace BRDF
 *                             (1 - max(0, acos(w.l) - p) / pi)^q with
 *                             p = 0.008 pi shininess, q = shininess_falloff,
 *                             w the cone axis, l = light_dir
 *   VCT_FLAG_DIFFUSE_FIRST_HIT diffuse cones stop at the first sample whose
 *                             opacity exceeds 1/100 and return its colour
 *                             with alpha 1 (zero if there is none)
 *   VCT_FLAG_SHADE            write out_radiance: with Phong direct light
 *                             direct = light_color * albedo * (diffuse_str *
 *                             max(n.l, 0) + specular_str * max(v.R, 0)^shininess),
 *                             R = reflect(-l, n), v towards the camera
 *                             (Ch. 3.3), L = albedo * (diffuse_str * D +
 *                             specular_str * S) + Vis * direct (Ch. 4.2.2)
 *   VCT_FLAG_SHADE_IMPL       with VCT_FLAG_SHADE: L = Vis * D + S + Vis *
 *                             direct instead (the thesis's L_impl, Ch. 5.4.4)
 * vct_trace_backward accepts only the two shading flags (the adjoint covers
 * D, S and Vis of the unmodified cones with straight colour).
 */
#define VCT_FLAG_OCC_SMOOTH 1
#define VCT_FLAG_SPEC_GRACE 2
#define VCT_FLAG_DIFFUSE_FIRST_HIT 4
#define VCT_FLAG_SHADE 8
#define VCT_FLAG_SHADE_IMPL 16
/* Every cone composites the sample colour as premultiplied by its opacity:
 * c += (1 - alpha) c_s instead of c += (1 - alpha) a_s c_s (the other reading
 * of the thesis's garbled colour line, Ch. 4.3.2); opacity as before. */
#define VCT_FLAG_PREMULTIPLIED 32

/*
 * Cone set and march parameters (the thesis's VoxSettings, Ch. 5.4.4).
 * Angles are full aperture angles in radians (Ch. 4.2.2, gamma).
 */
typedef struct {
  int32_t n_diffuse;   /* number of diffuse cones, 0 .. VCT_MAX_DIFFUSE    */
  int32_t spec_enable; /* 1: trace the specular cone                        */
  int32_t occ_enable;  /* 1: trace the occlusion cone towards light_dir     */
  int32_t flags;       /* VCT_FLAG_* bits                                   */
  /* Diffuse axes in the pixel's tangent frame (T, B, N): the scene
   * direction is T*d[0] + B*d[1] + N*d[2] with N the pixel normal,
   * T = normalize(a x N), B = N x T, a = (1,0,0) if |N.x| < 0.9 else
   * (0,1,0).  Used as given (not renormalised). */
  float diffuse_dir[VCT_MAX_DIFFUSE][3];
  float diffuse_weight[VCT_MAX_DIFFUSE]; /* D = sum_k weight_k (c_k, a_k)   */
  float diffuse_aperture;                /* in (0, pi)                       */
  /* Specular cone along the reflection of the view ray about N; aperture
   * = min + clamp((rho - roughness_min) / (1 - roughness_min), 0, 1)
   *   * (max - min) with rho the pixel roughness (min if no roughness). */
  float spec_aperture_min, spec_aperture_max, roughness_min;
  float occ_aperture;    /* occlusion cone aperture, in (0, pi)              */
  float light_dir[3];    /* unit vector towards the (directional) light      */
  float beta;            /* step factor: t += beta * d (Ch. 4.3.2), > 0      */
  float t0_voxels;       /* first sample at t0 = t0_voxels * h0, > 0         */
  float normal_offset_voxels; /* apex = x + normal_offset_voxels * h0 * N;
                                 |normal_offset_voxels| <= 2^19              */
  float t_max;           /* the march stops once t > t_max (scene units);
                            t_max * n / size <= 2^20 voxels                  */
  float shadow_str;      /* VCT_FLAG_OCC_SMOOTH strength                     */
  float occ_max_dist;    /* VCT_FLAG_OCC_SMOOTH upper edge (scene units), > 0 */
  float shininess;       /* Phong exponent; angular grace p = 0.008 pi this  */
  float shininess_falloff; /* exponent q of the angular-grace BRDF           */
  float diffuse_str, specular_str; /* material ratios of the shading        */
  float light_color[3];  /* RGB intensity of the directional light           */
} vct_trace_params;

/*
 * One view: a G-buffer and its outputs (all device memory, row-major
 * pixels p = y * width + x).  Masked pixels (mask[p] == 0) get D = S = 0
 * and Vis = 1.
 */
typedef struct {
  int32_t width, height; /* 1 .. 65535                                       */
  int32_t pyramid;       /* index into the pyramids passed with the views    */
  int32_t reserved;      /* must be 0                                        */
  const float *position; /* [H*W*3] surface position, scene units            */
  const float *normal;   /* [H*W*3] unit surface normal                      */
  const float *roughness;/* [H*W] in [0,1], or NULL                          */
  const uint8_t *mask;   /* [H*W], or NULL (every pixel valid)               */
  float camera[3];       /* eye position (specular view vector x - camera)   */
  float pad;
  float *out_diffuse;    /* [H*W*4] D = sum_k w_k (rgb_k, alpha_k), or NULL   */
  float *out_specular;   /* [H*W*4] S = (rgb, alpha) of the specular cone     */
  float *out_visibility; /* [H*W] Vis = 1 - alpha of the occlusion cone       */
  const float *albedo;   /* [H*W*3] material colour for the shading, or NULL (1) */
  float *out_radiance;   /* [H*W*4] shaded colour (VCT_FLAG_SHADE), or NULL  */
  /* Per-cone march state, or NULL: [n_cones][H*W] pairs (uint32 number of
   * samples K, float32 transmittance before the last sample), 8-byte
   * aligned; cones in the order specular (if enabled), occlusion (if
   * enabled), diffuse 0 .. n_diffuse-1.  vct_trace writes it (masked pixels
   * are skipped); vct_trace_backward, given the same pyramid, parameters
   * and view, reads it instead of re-marching every cone to find where it
   * stopped (its reverse walk needs both values). */
  void *cone_state;
} vct_view;

/* Launch shape of the trace kernels (see vct_autotune_trace). */
typedef struct {
  int32_t tile_w, tile_h;   /* pixels per work item (queue granularity)      */
  int32_t lanes_per_pixel;  /* 1, 2, 4 or 8 lanes share one pixel's cones    */
  int32_t ctas_per_sm;      /* persistent CTAs per SM; 0 = occupancy limit   */
} vct_launch_config;

/* Per-call counters left in the trace workspace (device memory). */
typedef struct {
  uint64_t samples[3]; /* samples taken by diffuse, specular, occlusion cones */
  uint64_t cones[3];   /* cones traced per kind                               */
  uint32_t queue;      /* work-queue cursor (internal)                        */
  uint32_t status;     /* VCT_ERR_TIMEOUT if a bounded wait gave up           */
} vct_trace_stats;

/* Device workspace bytes vct_trace needs (a vct_trace_stats, padded). */
size_t vct_trace_workspace_bytes(void);

/*
 * Traces every pixel of every view: per pixel the cone set of Ch. 4.2 (the
 * diffuse cones over the normal hemisphere, the specular cone along the
 * reflected view ray, the occlusion cone towards the light; Ch. 4.2.1 cone
 * apex on the surface, Ch. 5.4.4 cone configurations), each cone marched by
 * the cone trace function of Ch. 4.3.2 (d = 2 t tan(gamma/2), t += beta d,
 * front-to-back accumulation until alpha reaches 1) through the sampler of
 * Ch. 4.5 (mip level from the cone diameter over the voxel size), and the
 * outputs of Ch. 4.1 / 4.2.2 (D = the weighted sum of the diffuse cones, S
 * the specular cone, Vis = 1 - alpha of the occlusion cone).  One
 * persistent launch per group of up to 256 views: CTAs pull pixel tiles
 * from a queue in `workspace` and march each pixel's cones.
 *   pyrs[n_pyramids]: pyramids referenced by views[i].pyramid (any dtype).
 *   params:           cone set and march parameters (host memory).
 *   cfg:              launch shape, or NULL for the tuned / default shape.
 *   workspace:        device memory >= vct_trace_workspace_bytes(); zeroed
 *                     at the start of the call; after the stream reaches the
 *                     end of the call it holds a vct_trace_stats.
 * Sampling: level lambda = log2(2 t tan(gamma/2) / h0) clamped to
 * [0, levels-1]; trilinear at floor(lambda) and floor(lambda)+1, linear in
 * frac(lambda); colour c += (1 - alpha) a_s c_s, alpha += (1 - alpha) a_s;
 * float32 arithmetic throughout (FP16 pyramids are widened on load).
 * Errors: VCT_ERR_INVALID_ARG (NULL pointers where required, bad shapes or
 * parameters, pyramid index out of range), VCT_ERR_WORKSPACE, VCT_ERR_CUDA.
 */
vct_status vct_trace(const vct_pyramid *pyrs, int32_t n_pyramids,
                     const vct_view *views, int32_t n_views,
                     const vct_trace_params *params,
                     const vct_launch_config *cfg, void *workspace,
                     size_t workspace_bytes, vct_stream_t stream);

/*
 * Times every candidate launch shape (tile 4x8, 8x8, 8x16, 16x16 x
 * lanes_per_pixel 1, 2, 4, 8) on the given views, synchronously, and caches
 * the fastest under (device, dtype of pyrs[0], n of pyrs[0], tracing of the
 * specular/occlusion cones); vct_trace with cfg == NULL then uses it.  The
 * views' outputs are overwritten.  `best` (host, may be NULL) receives the
 * choice.
 */
vct_status vct_autotune_trace(const vct_pyramid *pyrs, int32_t n_pyramids,
                              const vct_view *views, int32_t n_views,
                              const vct_trace_params *params, void *workspace,
                              size_t workspace_bytes, vct_stream_t stream,
                              vct_launch_config *best);

/* ------------------------------------------------------------------------ */
/* Adjoint                                                                  */
/* ------------------------------------------------------------------------ */
/* Upstream gradients of one view (device, same layouts as the outputs). */
typedef struct {
  const float *grad_diffuse;    /* [H*W*4] dL/dD, or NULL (zero)             */
  const float *grad_specular;   /* [H*W*4] dL/dS, or NULL (zero)             */
  const float *grad_visibility; /* [H*W]   dL/dVis, or NULL (zero)           */
  /* [H*W*4] dL/d(shaded radiance), or NULL: with VCT_FLAG_SHADE the adjoint
   * passes it down to D, S and Vis through the shading epilogue (L.a is the
   * constant 1 and takes no gradient).  With VCT_FLAG_SHADE_IMPL, where L
   * depends on Vis * D, the view's out_diffuse (and out_visibility when the
   * occlusion cone is on) must hold the forward trace's outputs. */
  const float *grad_radiance;
} vct_view_grad;

/* Device workspace bytes vct_trace_backward needs for `pyr` (a float32
 * gradient pyramid plus a header; in the anisotropic layout for a
 * VCT_LAYOUT_ANISO pyramid, else dense). */
size_t vct_trace_backward_workspace_bytes(const vct_pyramid *pyr);

/*
 * Gradient of a loss with respect to the dense level-0 grid: the adjoint of
 * vct_trace and vct_build_mips (no counterpart in the thesis, which has no
 * gradients; the transpose of the Ch. 4.3.2 accumulation, of the Ch. 4.5
 * quadrilinear sampler and of the Ch. 4.3.3 box filter).  Recomputes each
 * cone's march, walks it backwards to form the derivatives
 * of the front-to-back accumulation, scatters them through the quadrilinear
 * weights into a float32 gradient pyramid in `workspace`, then pushes each
 * level down to its children (1/8 each) and ADDS the level-0 result into
 * grad_level0_dense (device float32 [n][n][n][4], z, y, x, channel).
 * Every view must use pyramid index 0 (`pyr`), of either dtype and layout:
 * the march is recomputed from the stored (FP16 or brick) texels exactly as
 * vct_trace read them, and the rounding of FP16 storage is passed through
 * as identity (the gradient is that of the pyramid as stored, with respect
 * to the values it was built from).  The gradient pyramid is dense float32,
 * except for a VCT_LAYOUT_ANISO pyramid: its derivatives go to the
 * directional volumes a sample read (times w_a^2 / |w|^2), and the levels
 * are pushed down through the derivatives of the pair composite (at the
 * forward texels in `pyr`, which must still hold the pyramid the forward
 * traced; colour derivatives are 0 where a pair's alpha is 0).  Scatter
 * order is not deterministic (see vct_trace_backward_deterministic for a
 * reproducible variant).
 */
vct_status vct_trace_backward(const vct_pyramid *pyr, const vct_view *views,
                              const vct_view_grad *grads, int32_t n_views,
                              const vct_trace_params *params,
                              const vct_launch_config *cfg,
                              float *grad_level0_dense, void *workspace,
                              size_t workspace_bytes, vct_stream_t stream);

/* Workspace bytes of vct_trace_backward_deterministic: the float32 gradient
 * pyramid plus, per level, 4 x uint64 per texel (256-byte aligned). */
size_t vct_trace_backward_deterministic_workspace_bytes(const vct_pyramid *pyr);

/*
 * vct_trace_backward with a reproducible result (a debugging mode): every
 * scattered contribution is rounded to a multiple of 2^-32 and summed as a
 * 64-bit two's-complement integer, so the order in which warps reach a
 * texel does not change any bit of the gradient; each level is converted to
 * float32 (round to nearest) before the mip adjoint.  Contributions below
 * 2^-33 in magnitude are lost, and every per-texel sum must stay within
 * (-2^31, 2^31).  Same arguments and checks as vct_trace_backward; workspace
 * of vct_trace_backward_deterministic_workspace_bytes(pyr) bytes.
 */
vct_status vct_trace_backward_deterministic(const vct_pyramid *pyr, const vct_view *views,
                                            const vct_view_grad *grads, int32_t n_views,
                                            const vct_trace_params *params,
                                            const vct_launch_config *cfg,
                                            float *grad_level0_dense, void *workspace,
                                            size_t workspace_bytes, vct_stream_t stream);

/*
 * vct_trace_backward without a workspace argument, for callers that cannot
 * allocate device memory (a plugin handed only pre-sized buffers, a host
 * application whose device heap is partitioned up front, code that must not
 * touch an allocator it does not own).  The thesis has no counterpart: this
 * is a packaging variant of the adjoint above, with the same arguments,
 * results and errors except that the scratch comes from the library.
 *   - Scratch: a 5 MiB array in the library's device memory, enough for the
 *     gradient pyramid of a dense or bricked grid up to 64^3, or of an
 *     anisotropic grid up to 32^3 (whose coarse levels hold six volumes).
 *     Every GPU that loads the library holds it until the process exits.
 *     Larger pyramids are rejected with VCT_ERR_WORKSPACE; the message gives
 *     the bytes the pyramid needs, its layout and the limit.
 *   - Allocation: none (no cudaMalloc/cudaFree or allocating library call).
 *   - Set-up: the array's address differs from one CUDA context to another
 *     (each device's primary context, contexts the caller creates).  A call
 *     made outside a stream capture looks the address up in the current
 *     context (cudaGetSymbolAddress) and keeps it under the context's unique
 *     ID; a call made while `stream` is being captured uses the address kept
 *     for the current context, so make one call in a context before
 *     capturing it there (else VCT_ERR_CUDA).
 *   - Sharing: every call uses the same array and leaves its contents behind;
 *     each call clears what must start at zero.  Calls whose GPU work
 *     overlaps (other streams, other host threads) race on the array.
 */
vct_status vct_trace_backward_noalloc(const vct_pyramid *pyr, const vct_view *views,
                                      const vct_view_grad *grads, int32_t n_views,
                                      const vct_trace_params *params,
                                      const vct_launch_config *cfg,
                                      float *grad_level0_dense, vct_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Host-buffer frame pipeline                                               */
/* ------------------------------------------------------------------------ */
/*
 * Runs the hot path (vct_build_mips + vct_trace of one view) on frames whose
 * inputs and outputs live in host memory, overlapping the copies of one frame
 * with the computation of its neighbours: two device slots, one stream for
 * host-to-device copies, one for the kernels and one for device-to-host
 * copies, ordered by events.  The thesis's CPU rendering loop syncs data to
 * the GPU before every frame, then mipmaps and cone-traces (Ch. 5.2); this
 * is that loop's data movement on a GPU whose copy engines run beside its
 * SMs.
 *   - vct_pipeline_create allocates both slots on the current device
 *     (per slot: dense level 0, pyramid, G-buffer, outputs, trace workspace).
 *   - vct_pipeline_submit enqueues one frame and returns; host inputs must
 *     stay unchanged, and host outputs unread, until the frame is joined.
 *     Host buffers should be page-locked (cudaHostAlloc/cudaHostRegister),
 *     else the copies do not overlap.  The frame starts after the work
 *     enqueued so far on `after`.
 *   - vct_pipeline_join makes `stream` wait (on the GPU, not the host) for
 *     every frame submitted so far; host outputs are final once `stream` has
 *     reached that point.
 * Not thread-safe: one host thread per pipeline.
 */
typedef struct vct_pipeline vct_pipeline;

typedef struct {
  int32_t n, levels, dtype;  /* pyramid shape (dense layout)                  */
  int32_t width, height;     /* view size, 1 .. 65535                         */
  int32_t has_roughness;     /* 1: frames carry per-pixel roughness           */
  int32_t has_mask;          /* 1: frames carry a pixel mask                  */
  int32_t outputs;           /* bit 0 diffuse, bit 1 specular, bit 2 visibility */
  float origin[3], size;     /* grid placement in the scene                   */
} vct_pipeline_desc;

/* One frame in host memory (sizes from the pipeline's description). */
typedef struct {
  const float *level0;     /* [n][n][n][4] float32                              */
  const float *position;   /* [H*W*3]                                           */
  const float *normal;     /* [H*W*3]                                           */
  const float *roughness;  /* [H*W] if has_roughness, else ignored              */
  const uint8_t *mask;     /* [H*W] if has_mask, else ignored                   */
  float camera[3];
  float pad;
  float *out_diffuse;      /* [H*W*4] if outputs bit 0                          */
  float *out_specular;     /* [H*W*4] if outputs bit 1                          */
  float *out_visibility;   /* [H*W] if outputs bit 2                            */
} vct_host_frame;

vct_status vct_pipeline_create(const vct_pipeline_desc *desc, const vct_trace_params *params,
                               vct_pipeline **out);
vct_status vct_pipeline_submit(vct_pipeline *p, const vct_host_frame *frame, vct_stream_t after);
vct_status vct_pipeline_join(vct_pipeline *p, vct_stream_t stream);
/* Sample and cone counters of the most recently joined frames' slot `slot`
 * (0 or 1), copied to the host; synchronises with that slot's last frame. */
vct_status vct_pipeline_stats(vct_pipeline *p, int32_t slot, vct_trace_stats *out);
/* Waits for all submitted work, then frees the pipeline (NULL is ignored). */
void vct_pipeline_destroy(vct_pipeline *p);

/* ------------------------------------------------------------------------ */
/* Voxelization (Ch. 4.4, Ch. 5.4.4 voxelize())                             */
/* ------------------------------------------------------------------------ */
/*
 * A triangle mesh in device memory.  Triangles are double sided; their
 * geometric normal (v2 - v1) x (v3 - v1) lights them.
 */
typedef struct {
  const float *vertices;  /* [n_vertices][3] scene units, 4-byte aligned      */
  const int32_t *indices; /* [n_triangles][3] vertex indices                  */
  const float *colors;    /* [n_triangles][3] material colour per triangle    */
  int32_t n_vertices;     /* >= 0                                             */
  int32_t n_triangles;    /* 0 .. 2^30                                        */
} vct_mesh;

/* The directional light whose direct diffuse light the voxels store. */
typedef struct {
  float light_dir[3];   /* towards the light, as given (not normalised)        */
  float light_color[3]; /* RGB intensity                                       */
  float ambient;        /* ambient strength of the Phong model                 */
  float diffuse_str;    /* diffuse strength of the Phong model                 */
} vct_voxel_light;

/* Counters at the start of the voxelization workspace after a call. */
typedef struct {
  uint64_t fragments;       /* fragments that landed inside the grid           */
  uint64_t large_items;     /* work items of the triangles rasterised by warps */
  uint64_t item_cursor;     /* internal                                        */
  uint32_t skipped;         /* triangles with a bad index or a vertex out of range */
  uint32_t degenerate;      /* triangles of zero area after snapping           */
  uint32_t large_triangles; /* triangles whose bounding box exceeds 64 pixels  */
  uint32_t reserved;
} vct_voxelize_stats;

/* Device workspace vct_voxelize needs for an n^3 grid and a mesh of
 * n_triangles; 0 for invalid arguments.  Layout: a vct_voxelize_stats
 * padded to 256 bytes; the owner grid, n^3 uint32 in the level-0 layout
 * (triangle index + 1 of the voxel's fragment, 0 = empty); then 32 bytes
 * per triangle of internal tables (256-byte aligned). */
size_t vct_voxelize_workspace_bytes(int32_t n, int32_t n_triangles);

/*
 * Voxelizes `mesh` into the dense level-0 grid [n][n][n][4] float32 (z, y,
 * x, rgba) that vct_build_mips takes, covering the cube [origin, origin +
 * size)^3 (Ch. 4.4; Ch. 5.4.4 voxelize()).  The grid is cleared first.
 * Every triangle is rasterised once, orthographically along its dominant
 * axis (the largest component of |(v2 - v1) x (v3 - v1)|, the first on ties;
 * Ch. 4.4.2) on an n x n viewport; each pixel whose centre it covers gives a
 * fragment at the triangle's depth there, stored in its voxel as
 *   (colour * light_color * (ambient + diffuse_str * max(N . l, 0)), 1)
 * (Ch. 4.4.3: the Phong model without its glossy term; N the normalised
 * geometric normal).  Rules the thesis leaves to the OpenGL rasteriser:
 *   - vertices snap to 1/256 voxel: X = rint(float32(float32(v - origin) * s))
 *     with s = float32(256 n / size); a triangle with a snapped coordinate of
 *     magnitude >= 2^19 or a bad index is skipped, one of zero snapped area
 *     is degenerate (both counted in the stats);
 *   - pixel centres at (i + 1/2) voxels; a centre on an edge counts for top
 *     and left edges of the counter-clockwise projection only (adjacent
 *     triangles cover it once); the depth cell is the floor of the exact
 *     plane depth; fragments outside the grid are dropped;
 *   - where several triangles reach a voxel, the highest triangle index wins
 *     (serial draw order), so the result does not depend on scheduling.
 * The coverage, depth and winner decisions are exact integer arithmetic;
 * only the colour is float32.  level0_dense: n^3 * 16 bytes, 16-byte
 * aligned.  workspace: vct_voxelize_workspace_bytes(n, n_triangles) bytes,
 * 256-byte aligned; on return (stream order) it holds the stats and the
 * owner grid.  n is a power of two in [2, 1024]; size > 0.
 */
vct_status vct_voxelize(const vct_mesh *mesh, int32_t n, const float origin[3], float size,
                        const vct_voxel_light *light, float *level0_dense, void *workspace,
                        size_t workspace_bytes, vct_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Camera G-buffer (Ch. 5.4 geometry pass; Ch. 3.2 rasterisation)           */
/* ------------------------------------------------------------------------ */
/*
 * Pinhole camera.  Pixel (i, j) of the width x height image (j = 0 the top
 * row) looks along d = (forward + sx right) + sy up with
 *   sx = ((2i+1)/width - 1) tx,  sy = (1 - (2j+1)/height) tan_half_fov,
 *   tx = float32(tan_half_fov * width / height),
 * every operation rounded to float32.  The hit tests run in a fixed-point
 * frame of 2^17 units per frame_size, origin frame_origin: a position p
 * snaps to X = rint(float32(float32(p - frame_origin) * s)), s =
 * float32(2^17 / frame_size), and must satisfy |X| < 2^18 (the scene may
 * reach two frame sizes from the origin); d snaps to rint(float32(d * 2^18)).
 */
typedef struct {
  float eye[3];          /* camera position, inside the frame                   */
  float forward[3];      /* view direction (unit length expected)               */
  float right[3];        /* image +x (unit length expected)                     */
  float up[3];           /* image +y (unit length expected)                     */
  float tan_half_fov;    /* tan of half the vertical field of view, > 0         */
  int32_t width, height; /* 1 .. 16384 pixels                                   */
  float frame_origin[3]; /* fixed-point frame (above)                           */
  float frame_size;      /* > 0                                                 */
} vct_camera;

/* Counters at the start of the G-buffer workspace after a call. */
typedef struct {
  uint64_t pairs;         /* (16x16 tile, triangle) pairs the binning produced */
  uint64_t pair_capacity; /* pairs the workspace holds                         */
  uint32_t skipped;       /* triangles with a bad index or a vertex beyond the frame */
  uint32_t degenerate;    /* triangles of zero snapped area                    */
  uint32_t culled;        /* triangles outside the view, or edge-on to the eye */
  uint32_t wide;          /* triangles passing so close to the eye that they were
                             binned to every tile                               */
  uint32_t overflow;      /* 1: pairs > pair_capacity, every pixel left empty   */
  uint32_t reserved[3];
} vct_gbuffer_stats;

/* Device workspace vct_gbuffer needs for a width x height image, a mesh of
 * n_triangles and room for pair_capacity (tile, triangle) pairs (at most
 * 2^31); 0 for invalid arguments.  Layout: a vct_gbuffer_stats padded to
 * 256 bytes, 8 bytes per 16x16 tile (+ 4), 96 bytes per triangle, then
 * 4 bytes per pair, each part 256-byte aligned.  A larger workspace holds
 * proportionally more pairs. */
size_t vct_gbuffer_workspace_bytes(int32_t width, int32_t height, int32_t n_triangles,
                                   uint64_t pair_capacity);

/*
 * Draws `mesh` into the G-buffer that vct_trace reads (Ch. 5.4: geometry
 * pass before the cone tracing), for every pixel the nearest triangle on
 * the ray through the pixel centre.  With A, B, C the snapped vertices
 * relative to the snapped eye and D the snapped pixel direction, the ray
 * hits the double-sided triangle when D.(B x C), D.(C x A), D.(A x B) share
 * the sign of det(A, B, C) (zeros allowed, not all zero); its distance is
 * det(A, B, C) / (n . D), n = (B - A) x (C - A); the nearest hit wins by
 * exact comparison, equal distances going to the lower triangle index.
 * These decisions are exact integer arithmetic, so the result does not
 * depend on scheduling.  Outputs per pixel p = j * width + i:
 *   position [p*3]  hit point eye + t D in scene units (float32 t);
 *   normal   [p*3]  unit geometric normal of the unsnapped triangle,
 *                   turned towards the eye (by the sign of n . D);
 *   albedo   [p*3]  the triangle's colour (or NULL);
 *   mask     [p]    1 hit, 0 none (or NULL);
 *   triangle [p]    triangle index, -1 none (or NULL).
 * Pixels without a hit get zeros.  Triangles are binned to 16x16 pixel
 * tiles by a conservative screen box (guard-band clipping); the pairs must
 * fit the workspace, else the stats report overflow and every pixel is
 * left empty (the needed count is in vct_gbuffer_stats.pairs).
 * position/normal/albedo 4-byte aligned, triangle 4-byte aligned;
 * workspace 256-byte aligned of at least vct_gbuffer_workspace_bytes(...,
 * 0) bytes.  The camera needs forward, right and up components of
 * magnitude <= 1 + 2^-10, |det(right, up, forward)| >= 0.25 (a roughly
 * orthonormal basis) and tx + tan_half_fov <= 2.99, so that every snapped
 * direction component stays within 2^20 and the integer arithmetic cannot
 * overflow; the eye must lie inside the frame.
 */
vct_status vct_gbuffer(const vct_mesh *mesh, const vct_camera *camera, float *position,
                       float *normal, float *albedo, uint8_t *mask, int32_t *triangle,
                       void *workspace, size_t workspace_bytes, vct_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Diagnostics                                                              */
/* ------------------------------------------------------------------------ */
const char *vct_status_string(vct_status status);
const char *vct_last_error(void);
int32_t vct_version(void);

/*
 * Bounds-checked builds.  A library compiled with -DVCT_DEBUG_BOUNDS (the
 * `libvct_debug_bounds.so` variant of the in-tree build) compares every
 * computed texel, brick-slot, gradient, mip, voxel and tile-list index with
 * the length of its array before the access; a bad index sets a bit in a
 * device flag word and the access is skipped (loads read zero), so a kernel
 * never traps.  Bits: 1 trace texel, 2 brick slot table / pool, 4 adjoint
 * gradient texel, 8 mip texel, 16 voxelizer owner / colour, 32 G-buffer
 * tile lists, 64 the probe below.
 *
 * vct_debug_bounds_flags synchronises the device, stores the OR of the flag
 * words in *flags_out and clears them if `reset`.  In a release build it
 * stores 0 and returns VCT_ERR_UNSUPPORTED.
 */
vct_status vct_debug_bounds_flags(uint32_t *flags_out, int32_t reset);

/*
 * Check of the bounds checks: one kernel writes i to buf_dev[i] for i <
 * declared + extra through the check against `declared`, so the last
 * `extra` writes (1 .. 1024) must be caught (flag bit 64) and skipped.
 * buf_dev: device uint32 array of declared + extra words (the caught writes
 * would stay inside it even without the check).  VCT_ERR_UNSUPPORTED in a
 * release build.
 */
vct_status vct_debug_bounds_probe(uint32_t *buf_dev, uint32_t declared, uint32_t extra,
                                  vct_stream_t stream);

/*
 * Failure-path check of the bounded device waits: launches one CTA that
 * waits on an mbarrier nothing ever arrives at, with the same bounded-wait
 * routine the pipelined kernels use, giving up after about `max_ns`
 * nanoseconds; it then writes VCT_ERR_TIMEOUT to *flag_dev (device uint32).
 * Nothing is in flight when it gives up.
 */
vct_status vct_debug_wait_probe(uint32_t *flag_dev, uint64_t max_ns,
                                vct_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* VCT_H */

/*
 * sdd.h -- C ABI of the GB300 spectral domain-decomposed glass ray tracer (libsdd.so).
 *
 * The library renders naturally lit scenes whose glass is described by optical constants
 * n~(lambda) = n(lambda) + i k(lambda) (arXiv:1912.05494, Sec. 2, Eq. 1) and by per-tile
 * distribution maps of (n, k, thickness) (Sec. 6), sampled on any wavelength set
 * (Sec. 4: 81 samples, 380-780 nm).  The scene geometry is split once into subdomains
 * (Sec. 5); rays are binned into per-subdomain queues, traversed against each
 * subdomain's BVH, handed to the neighbouring subdomain's queue with their properties
 * unchanged when they cross an interface (Sec. 5), shaded per wavelength with complex
 * Fresnel reflection/transmission and Beer-Lambert absorption, and accumulated into a
 * spectral / CIE XYZ film.
 *
 * Conventions
 *   - Lengths in metres, wavelengths in nanometres, angles in radians unless a field name
 *     says otherwise; +z is "up" for the sky.
 *   - Scene inputs are HOST pointers; sdd_scene_create copies everything it needs.
 *   - Render outputs are caller-owned DEVICE buffers unless the entry point says host.
 *   - No C++ exception crosses this boundary.  Every call returns an sdd_status; on a
 *     non-zero status sdd_last_error() gives a message (thread-local, valid until the
 *     next call from that thread).
 *   - Calls run on the CUDA stream given (a cudaStream_t passed as void*, NULL = the
 *     legacy default stream) and return after the work they queued has finished, so that
 *     device-side errors (queue overflow, stack overflow, watchdog) are reported by the
 *     call that caused them.
 *   - A scene handle must not be used by two threads at once.
 */
#ifndef SDD_H
#define SDD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sdd_scene sdd_scene;         /* opaque, owned by the library */
typedef struct sdd_tileset sdd_tileset;     /* heterogeneous glass tiles (see below) */
typedef struct sdd_surrogate sdd_surrogate; /* tile-BTDF network (see below) */
typedef struct sdd_photon_maps sdd_photon_maps; /* caustic and global photon maps (see below) */

typedef enum {
  SDD_OK = 0,
  SDD_ERR_ARG = -1,            /* invalid argument (message says which) */
  SDD_ERR_OOM = -2,            /* device or host allocation failed */
  SDD_ERR_CUDA = -3,           /* a CUDA runtime call failed */
  SDD_ERR_QUEUE_OVERFLOW = -4, /* a ray queue would have exceeded its capacity */
  SDD_ERR_TIMEOUT = -5,        /* a device-side loop hit its iteration cap */
  SDD_ERR_STATE = -6,          /* call not valid in the handle's current state */
  SDD_ERR_STACK = -7           /* BVH traversal stack would have overflowed */
} sdd_status;

/* Material kinds.  Sec. 6: the windows' glass is refractive only (no scattering); walls
 * and lead came are not described by the paper and are modelled as Lambertian. */
typedef enum {
  SDD_MAT_DIELECTRIC_SOLID = 0, /* closed glass body: Fresnel at each interface, Beer-Lambert inside;
                                   triangles must wind counter-clockwise seen from outside */
  SDD_MAT_THIN_SLAB = 1,        /* zero-thickness tile of glass of thickness thickness_m: closed-form
                                   series over internal reflections; two-sided */
  SDD_MAT_HETERO_TILE = 2,      /* heterogeneous tile (thickness field, air bubbles) */
  SDD_MAT_DIFFUSE = 3,          /* Lambertian, spectral albedo; two-sided */
  SDD_MAT_OPAQUE = 4            /* absorbs everything */
} sdd_mat_kind;

typedef struct {
  int kind;               /* sdd_mat_kind */
  int n_lambda;           /* length of the tables below (>= 1) */
  const float* lambda_nm; /* ascending table grid; tables are interpolated linearly and
                             clamped at the ends */
  const float* n;         /* real index n(lambda) (Eq. 1); glass kinds only, may be NULL otherwise */
  const float* k;         /* absorption index k(lambda) >= 0 (Eq. 1); glass kinds only */
  float thickness_m;      /* THIN_SLAB / HETERO_TILE thickness */
  const float* albedo;    /* DIFFUSE albedo(lambda) in [0,1]; may be NULL otherwise */
  int tile_param_id;      /* HETERO_TILE: index into the tile set */
} sdd_material;

/* Natural lighting: a uniform sky and a sun disc, both spectral (Eq. 3 reads the sun as one
 * directional source; escaping rays see the sky). */
typedef struct {
  int n_lambda;
  const float* lambda_nm;     /* ascending table grid of the two spectra */
  const float* sky_radiance;  /* [n_lambda] */
  int sky_mode;               /* 0: every direction, 1: only directions with z > 0 */
  float sun_dir[3];           /* toward the sun (normalised by the library) */
  float sun_half_angle_rad;   /* <= 0 or sun_radiance == NULL: no sun */
  const float* sun_radiance;  /* [n_lambda] radiance inside the disc, or NULL */
} sdd_illuminant;

typedef struct {
  int n_vertices;
  const float* vertices;                 /* [n_vertices][3] */
  int n_triangles;
  const uint32_t* indices;               /* [n_triangles][3] */
  const uint16_t* material_of_triangle;  /* [n_triangles] */
  int n_materials;
  const sdd_material* materials;         /* [n_materials] */
  sdd_illuminant illum;
  int n_subdomains;   /* 1..64 slabs of equal length along split_axis (Sec. 5) */
  int split_axis;     /* 0, 1, 2, or -1 = longest axis of the scene box */
  float ray_epsilon_m;/* spawned rays start this far off the surface along its normal;
                         0 = 2e-6 x the largest absolute scene coordinate (at least 1e-5) */
  const sdd_tileset* tiles; /* tile set of the HETERO_TILE materials (tile_param_id indexes it), or
                               NULL; must outlive the scene.  A tile's front face is on the +n side
                               of its triangles' geometric normal, its frame the normal's Duff basis */
  int slab_polarisation;    /* THIN_SLAB series (Sec. 2, Eq. 1): 0 = one incoherent series on the
                               unpolarised interface reflectance (R_s + R_p) / 2; 1 = s and p light do
                               not mix at the slab's parallel faces, so the series runs on R_s and on
                               R_p separately and the results are averaged.  Other values: SDD_ERR_ARG */
} sdd_scene_desc;

typedef struct {
  float pos[3], look_at[3], up[3];
  float vfov_deg;       /* pinhole vertical field of view */
  int width, height;    /* pixels; row 0 is the top row */
  int orthographic;     /* 1: parallel rays along the view direction */
  float ortho_height_m; /* orthographic image height */
} sdd_camera;

/* Render modes. */
#define SDD_MODE_DETERMINISTIC 0 /* Sec. 3.1: split into reflected + transmitted children at
                                    every glass hit, no randomness, spp must be 1 */
#define SDD_MODE_MONTE_CARLO 1   /* Sec. 3.2: one Philox-driven path per (pixel, sample, lambda) */

typedef struct {
  int n_lambda;            /* number of render wavelengths (each one an independent path, Sec. 4) */
  const float* lambda_nm;  /* host [n_lambda] */
  int spp;                 /* samples per pixel */
  uint64_t seed;           /* Philox key */
  int max_depth;           /* surface interactions per path; deterministic mode: <= 10 */
  int mode;                /* SDD_MODE_* */
  int rr_start_depth;      /* Russian roulette from this interaction on (Monte Carlo) */
  int use_surrogate;       /* heterogeneous tiles: 0 = one brute-force ray through the tile per hit
                              (and per shadow ray); 1 = the BTDF network (opts->surrogate): T, R
                              and a two-lobe von Mises-Fisher mixture per side at hits, shaded by
                              one fused launch per generation; for shadow rays T x the
                              transmitted mixture's mass within 1 degree of straight through */
  int batched;             /* 0: host-driven wavefront (one launch per subdomain pass, queue counts
                              read back between launches); 1: a persistent cooperative kernel
                              drains every pass on the device -- the whole wave in one launch, or
                              with use_surrogate two launches per generation around the fused
                              tile shading; 2: the graph form -- the host-driven steps as
                              fixed-grid kernels that read their queue counts on the device, a
                              fixed sequence per generation (n_subdomains + 1 closest-hit passes,
                              shading, n_subdomains + 1 shadow passes; empty launches return at
                              once).  Forms 1 and 2 capture the frame as a CUDA graph and replay
                              it while its parameters and buffers are unchanged */
  int n_pixels;            /* 0: whole image; else render only these pixel indices */
  const int32_t* pixels;   /* host [n_pixels] row-major pixel indices (y * width + x) */
  int wave_paths;          /* paths per wave; 0 = automatic */
  float* path_radiance_out;/* optional device [pixels][spp][n_lambda] radiance of every path */
  uint32_t* path_hash_out; /* optional device [pixels][spp][n_lambda] event hash of every path
                              (Monte Carlo; FNV-1a over hit primitives and branch events) */
  const sdd_surrogate* surrogate; /* with use_surrogate = 1: the network that replaces brute-force
                                     tracing at heterogeneous-tile hits; its weights are read at
                                     render time (a replayed frame uses the current weights) */
  int bundle;              /* Monte Carlo spectral bundles (Sec. 4: the spectral array cut into
                              groups): 0 or 1 = every wavelength is its own path; B = 2..64 =
                              wavelengths jB .. jB+B-1 draw every random number on counter word j
                              and share one ray while their decisions agree (one traversal for the
                              group); a member whose branch differs continues on its own ray.
                              Each wavelength's chain keeps its distribution; the wavelengths of a
                              bundle become correlated.  Every form; at heterogeneous tiles each
                              member leaves on its own ray (brute force or network) */
  const sdd_photon_maps* photon_maps; /* Sec. 3.2 (Jensen's photon mapping): NULL = none; else maps
                              built for the same wavelength list (equal lambda_nm), used by Monte
                              Carlo renders of the host-driven or the graph form (batched = 0 or 2),
                              with or without spectral bundles, without the network
                              (use_surrogate = 0); other combinations return SDD_ERR_ARG.  At its
                              first diffuse vertex a path adds albedo / pi x (E_caustic + E_global)
                              of the maps at the hit point beside the sun NEE (each bundle member
                              those of its wavelength); later vertices take sky light only (no NEE,
                              no sun disc on escape) */
} sdd_render_opts;

/* Build the scene: validates, partitions the geometry into n_subdomains slabs (Sec. 5:
 * split once, reused for every render), builds one SAH BVH per subdomain and uploads it.
 * Returns SDD_ERR_ARG on bad input (message names the field). */
sdd_status sdd_scene_create(const sdd_scene_desc* desc, sdd_scene** out);

/* Frees the scene and all device memory it holds.  NULL is allowed. */
void sdd_scene_destroy(sdd_scene* scene);

/* Render one frame.  spectral_out: device float [n_px][n_lambda] (n_px = width * height or
 * opts->n_pixels), the per-pixel mean radiance of each wavelength; xyz_out: device float
 * [n_px][3] CIE XYZ (multi-lobe fit of the 1931 observer, normalised so that Y equals the
 * radiance of a flat spectrum) or NULL.  The film sums samples in FP64 in sample order,
 * so results do not depend on the wave size or the subdomain count beyond FP32 rounding
 * of branch decisions. */
sdd_status sdd_render(sdd_scene* scene, const sdd_camera* cam, const sdd_render_opts* opts,
                      float* spectral_out, float* xyz_out, void* cuda_stream);

/* Same as sdd_render, but spectral_out / xyz_out are HOST buffers: the library renders into
 * its own device buffers and copies the result back (the end-to-end form of the call). */
sdd_status sdd_render_to_host(sdd_scene* scene, const sdd_camera* cam, const sdd_render_opts* opts,
                              float* spectral_out_host, float* xyz_out_host, void* cuda_stream);

/* Launch-shape knobs of a scene (chosen by the autotuner; the defaults are safe):
 *   traverse_block: threads per block of the traversal kernels: 64, 128 (default) or 256;
 *   top_nodes:      BVH nodes per subdomain (the top levels, stored breadth-first) that each
 *                   traversal block stages in shared memory, 0..384 (48 KB of 128-byte nodes;
 *                   0 = none, default);
 *   wave_paths:     paths per wave when sdd_render_opts.wave_paths is 0 (0 = 2^26, or 2^25
 *                   bundle paths with spectral bundles);
 *   no_graph:       batched form only: 1 = launch the frame's kernels directly instead of
 *                   capturing and replaying them as a CUDA graph (default 0);
 *   queue_capacity: upper bound on the entries of each ray / subdomain queue (0 = automatic:
 *                   the wave size, 4x in deterministic mode, 2x with spectral bundles, and a
 *                   host-driven wave that needs more is rendered again as two halves).
 *                   Buffers keep their automatic size; with a bound set, a frame that needs
 *                   more returns SDD_ERR_QUEUE_OVERFLOW;
 *   block_chunks:   graph form: how the fixed grid takes work from a pass's queues, bit 0 for
 *                   the closest-hit passes, bit 1 for the shadow passes: 1 = each block takes
 *                   128 rays at a time (its warps wait for each other), 0 = each warp takes 32
 *                   (default 0 for both);
 *   resident_subdomains: out-of-core subdomains (Sec. 5: sub-domains loaded according to the
 *                   memory available, unloaded when few rays remain).  0 (default) or >=
 *                   n_subdomains: every subdomain's BVH stays in device memory.  1 <= C <
 *                   n_subdomains: the BVH moves to pinned host memory and at most C subdomains'
 *                   nodes and triangle records occupy device memory at a time; before every
 *                   traversal pass the C subdomains with the most queued rays are made resident
 *                   (copied in, evicting those with the fewest), rays queued for the others wait.
 *                   Images are bit-identical to the all-resident ones.  Host-driven form only:
 *                   renders with batched != 0 and sdd_trace_closest_noalloc return SDD_ERR_STATE
 *                   while it is on; sdd_trace_closest works.  Setting it synchronises the device. */
typedef struct {
  int traverse_block;
  int top_nodes;
  int wave_paths;
  int no_graph;
  int queue_capacity;
  int block_chunks;
  int resident_subdomains;
} sdd_tuning;
sdd_status sdd_set_tuning(sdd_scene* scene, const sdd_tuning* tuning);
sdd_status sdd_get_tuning(const sdd_scene* scene, sdd_tuning* out);

/* Self-test of the persistent kernel's watchdog (the paper has no counterpart): a grid
 * barrier of the batched form is run by four blocks, one of which never arrives; the waiting
 * blocks give up after timeout_ms (1..10000) and raise the timeout error bit.  Returns
 * SDD_ERR_TIMEOUT when that happened, SDD_OK if the barrier had completed (it cannot), or
 * SDD_ERR_CUDA / SDD_ERR_ARG.  No GPU fault or hang is involved: every wait is bounded. */
sdd_status sdd_watchdog_selftest(int timeout_ms);

/* Per-kernel timing and counters of the most recent render. */
typedef struct {
  double ms_raygen, ms_traverse, ms_shade, ms_shadow, ms_film, ms_total;
  int64_t launches_raygen, launches_traverse, launches_shade, launches_shadow, launches_film,
      launches_total;
  int64_t rays_closest;    /* closest-hit traversals, counting each subdomain visit */
  int64_t rays_shadow;     /* shadow traversals, counting each subdomain visit */
  int64_t node_visits;     /* BVH nodes fetched by closest-hit traversal (level >= 2) */
  int64_t tri_tests;       /* triangles tested by closest-hit traversal (level >= 2) */
  int64_t shadow_node_visits, shadow_tri_tests;
  int64_t crossings;       /* interface hand-offs between subdomain queues */
  int64_t paths;           /* spectral paths traced ((pixel, sample, wavelength) chains) */
  int64_t waves;
  int64_t bytes_ray_state; /* ray/queue/hit bytes read+written by the traversal kernels */
  double ms_persistent;    /* batched form: persistent drain kernels (all steps of a wave) */
  int64_t launches_persistent;
  int64_t graph_replays;   /* batched form: frames replayed from a captured CUDA graph */
  double ms_tile;          /* network form: fused tile-shading launches (host-driven form) */
  int64_t launches_tile;   /* network form: fused tile-shading launches */
  int64_t tile_shaded;     /* network form: tile hits shaded by the network (level >= 2) */
  int64_t wave_splits;     /* host-driven form: waves rendered again as two halves after their
                              rays outgrew the queues (spectral bundles that split often) */
  int64_t subdomain_loads; /* out-of-core subdomains: subdomains copied into device slots */
  int64_t bytes_streamed;  /* out-of-core subdomains: node and triangle bytes copied in */
} sdd_stats;

/* level 0: nothing; 1: CUDA-event timing of every launch; 2: also count BVH nodes and
 * triangles (slower; for computing algorithmic bytes). */
sdd_status sdd_set_profiling(sdd_scene* scene, int level);
sdd_status sdd_get_stats(const sdd_scene* scene, sdd_stats* out);

/* Scene facts: triangle references per subdomain after the split, BVH nodes, bytes. */
typedef struct {
  int n_triangles, n_subdomains, split_axis, bvh_max_depth;
  int64_t n_tri_refs, n_nodes, device_bytes;
  float planes[65]; /* subdomain boundaries along split_axis (first/last are -inf/+inf) */
} sdd_scene_info;
sdd_status sdd_scene_get_info(const sdd_scene* scene, sdd_scene_info* out);

/* Host-side build of the subdomain split and of the per-subdomain BVHs that sdd_scene_create
 * makes for the same desc (Sec. 5: the geometry is split once, every sub-domain keeps its own
 * hierarchy), without a device: for inspecting and testing the structure the traversal
 * kernels walk.  Only the geometry fields of desc are read (vertices, indices, n_subdomains,
 * split_axis, ray_epsilon_m) and validated as sdd_scene_create validates them.
 *
 * Node, 128 bytes (int32 / float, child c in element c of each array):
 *   float lo_x[4], hi_x[4], lo_y[4], hi_y[4], lo_z[4], hi_z[4]; int32 link[4], count[4];
 *   count[c] > 0: leaf child, triangle records [link[c], link[c] + count[c]);
 *   count[c] == 0 and link[c] >= 0: inner child, node link[c] (absolute index);
 *   link[c] < 0: no child.  Every subdomain's nodes form one block in breadth-first order
 *   from root[s].
 * Triangle record, 48 bytes: float v0[3], uint32 primitive index, float v1[3], pad,
 *   float v2[3], pad.
 * Call with nodes and tris NULL to get the sizes in *info; then again with buffers of
 * info->n_nodes nodes (nodes_cap >= that) and info->n_tri_records records.  root and
 * n_nodes_sub (n_subdomains entries) and planes (n_subdomains + 1 entries, first -inf and
 * last +inf) are filled when not NULL.  Caller-owned buffers; SDD_ERR_ARG on invalid
 * geometry or a buffer that is too small, SDD_ERR_OOM when the host allocation fails. */
typedef struct {
  int n_subdomains, split_axis;
  int bvh_max_depth;   /* levels of the binary SAH tree before its collapse to 4-wide nodes */
  int stack_need;      /* deepest traversal stack a walk of any subdomain's tree can need;
                          sdd_scene_create refuses a scene above 64 */
  int64_t n_nodes, n_tri_records;
  float slop;          /* a triangle is referenced by every slab its box overlaps widened by
                          this much, its box clipped to the widened slab */
} sdd_bvh_info;
sdd_status sdd_bvh_build_host(const sdd_scene_desc* desc, sdd_bvh_info* info, void* nodes, int64_t nodes_cap,
                              void* tris, int64_t tris_cap, int32_t* root, int32_t* n_nodes_sub, float* planes);

/* Batched closest-hit query (used by tests and by tools): n rays with device origins
 * [n][3] and directions [n][3] (float), t in (0, inf).  Writes device t_out[n] (inf on a
 * miss) and prim_out[n] (-1 on a miss), going through the subdomain queues exactly as
 * rendering does. */
sdd_status sdd_trace_closest(sdd_scene* scene, int n, const float* org_dev, const float* dir_dev,
                             float* t_out_dev, int32_t* prim_out_dev, void* cuda_stream);

/* ---------------------------------------------------------------- heterogeneous tiles
 * Medieval glass tiles with non-uniform thickness and air micro-bubbles (Sec. 1; Sec. 6
 * names light scattering as the missing part of the glass model).  A tile is periodic with
 * side tile_size_m: flat front face z = 0, back face z = -h(x, y) a grid x grid triangulated
 * height field of h = clamp(d_mean + amplitude (n(x, y) - 1/2), 2 mm, 5 mm), n a 2-octave
 * value noise whose lattice values are Philox draws keyed by the tile's seed; air bubbles
 * are a Poisson process of the given density with radii log-uniform in [10, 100] um, met at
 * exponential free paths and scattered with exact sphere optics (no displacement); Fresnel
 * (complex index), Snell and Beer-Lambert as for other glass.  Rays are traced by brute
 * force, one Philox draw per interaction on the tile stream. */
typedef struct {
  int n_tiles;
  const float* d_mean_m;          /* [n_tiles] mean thickness (host) */
  const float* amplitude_m;       /* [n_tiles] peak-to-peak thickness variation */
  const float* bubble_density_m3; /* [n_tiles] bubbles per cubic metre (1e10 = 1e4 per cm^3) */
  const uint32_t* seed;           /* [n_tiles] noise seed */
  int grid;                       /* back-face cells per side (64) */
  float tile_size_m;              /* side of the periodic tile (0.1) */
} sdd_tileset_desc;

/* Build the tile set: height fields are computed on the device.  Allocates device memory. */
sdd_status sdd_tileset_create(const sdd_tileset_desc* desc, sdd_tileset** out);
void sdd_tileset_destroy(sdd_tileset* tiles);
/* Copy tile `tile`'s (grid+1)^2 vertex thicknesses (row j, column i) to host memory. */
sdd_status sdd_tileset_heights(const sdd_tileset* tiles, int tile, float* out_host);

/* Trace n rays through tile `tile` (all arrays device): entry points xy [n][2] in [0, L),
 * directions [n][3] in the tile frame (z < 0 enters through the front), draws keyed
 * (px[i], sample[i], bounce, tile stream, interaction, lam).  Outputs: side (0 reflected,
 * 1 transmitted, 2 absorbed after max_events interactions, max_events <= 256), weight,
 * exit direction [n][3], bubble encounters and interactions. */
sdd_status sdd_tile_trace_rays(sdd_tileset* tiles, int tile, int n, const float* xy, const float* dir, float n_re,
                               float k, float lambda_nm, const uint32_t* px, const uint32_t* sample, uint32_t bounce,
                               uint32_t lam, uint64_t seed, int max_events, int32_t* side, float* w, float* dir_out,
                               int32_t* bubbles, int32_t* events, void* cuda_stream);

/* Surrogate training data: for each of n_samples queries (device arrays: signed cosine of the
 * incidence angle, azimuth, wavelength, n, k, tile index) trace rays_per_sample rays from
 * uniform entry points; cos_in > 0 enters through the flat front face travelling toward
 * -z, cos_in < 0 through the rough (height-field) back face travelling toward +z.  out[n][20]
 * (device) = transmittance, reflectance, weight absorbed or left at the interaction cap,
 * bubble encounters per ray, then the fraction of the transmitted weight in each of 8
 * deflection-angle bins about the straight-through direction (edges 0, 1, 2, 4, 8, 16, 32,
 * 64, 180 degrees), then the same 8 fractions of the reflected weight about the mirror
 * direction (a side with no weight has zero fractions).  Sample s draws its entry points on
 * (s, ray, 0, tile stream, 0) and its interactions on bounce 1. */
sdd_status sdd_tile_generate(sdd_tileset* tiles, int n_samples, const float* cos_in, const float* phi_in,
                             const float* lambda_nm, const float* n_re, const float* k, const int32_t* tile,
                             int rays_per_sample, uint64_t seed, int max_events, float* out, void* cuda_stream);

/* ---------------------------------------------------------------- BTDF surrogate
 * A small network that predicts a heterogeneous tile's BTDF from (signed cos theta_in as in
 * sdd_tile_generate, phi_in, lambda nm, mean thickness m, bubble density m^-3, n, k) -- the
 * raw inputs, [n][7] row-major.  Predictions, [n][8]: T, R, then for the transmitted side
 * the weight w of its first lobe and log kappa of its two von Mises-Fisher lobes about the
 * straight-through direction, then the same three for the reflected side about the mirror
 * direction.  Training targets, [n][18]: T, R and the 8 + 8 deflection-bin fractions
 * (sdd_tile_generate columns 0, 1, 4..19).  Loss per row: squared errors of T and R plus
 * 0.05 x (T KL(bins_T | lobe mass_T) + R KL(bins_R | lobe mass_R)), KL with 1e-4 added to
 * both sides.  Fourier features (16 frequencies of the inputs normalised to [0, 1]) -> 48 ->
 * 4 x 128 GELU -> 16; BF16 weights and activations, FP32 accumulation on the tensor cores,
 * Adam on FP32 master weights.  Parameters: one FP32 array, per layer W [in][out] row-major
 * then b [out] (sdd_surrogate_param_count() values).  The paper has no network; it names
 * scattering in the glass as future work (Sec. 6). */
int sdd_surrogate_param_count(void);
/* fourier_B: host [16][7]; init_params: host flat parameters; max_batch rows per call. */
sdd_status sdd_surrogate_create(const float* fourier_B, const float* init_params, int n_params, int max_batch,
                                sdd_surrogate** out);
void sdd_surrogate_destroy(sdd_surrogate* s);
sdd_status sdd_surrogate_get_params(const sdd_surrogate* s, float* host_out, int n_params);
sdd_status sdd_surrogate_set_params(sdd_surrogate* s, const float* host_in, int n_params);
/* Loss (mean over rows) and its gradient for n <= max_batch rows (raw inputs [n][7] and
 * targets [n][18] on the device), without updating the weights; grad_host may be NULL. */
sdd_status sdd_surrogate_gradients(sdd_surrogate* s, int n, const float* raw_dev, const float* y_dev, float* grad_host,
                                   float* loss_host, void* cuda_stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on a batch of n rows. */
sdd_status sdd_surrogate_train_step(sdd_surrogate* s, int n, const float* raw_dev, const float* y_dev, float lr,
                                    float* loss_host, void* cuda_stream);
/* A training run: opts->steps Adam steps (learning rate opts->lr) on minibatches of
 * opts->batch rows (<= min(n, max_batch)) of the n device-resident samples raw_dev [n][7],
 * y_dev [n][18]; each epoch visits the rows in the order (a i + c) mod n with gcd(a, n) = 1,
 * a and c drawn from opts->seed.  loss_host (may be NULL) receives the loss of every step;
 * the host synchronises once, at the end. */
typedef struct {
  int steps;
  int batch;
  float lr;
  uint64_t seed;
} sdd_train_opts;
sdd_status sdd_surrogate_train(sdd_surrogate* s, int n, const float* raw_dev, const float* y_dev,
                               const sdd_train_opts* opts, float* loss_host, void* cuda_stream);
/* The FP32 parameters as bytes (4 x sdd_surrogate_param_count()); same layout as _get_params. */
sdd_status sdd_surrogate_get_weights(const sdd_surrogate* s, void* host_out, size_t bytes);
sdd_status sdd_surrogate_set_weights(sdd_surrogate* s, const void* host_in, size_t bytes);
/* Predictions [n][8] (device) for n rows of raw inputs (any n; processed max_batch at a time). */
sdd_status sdd_surrogate_infer(sdd_surrogate* s, int n, const float* raw_dev, float* out_dev, void* cuda_stream);

/* ---------------------------------------------------------------- photon maps
 * Sec. 3.2: Jensen's photon mapping as the global-illumination algorithm.  Photons leave a
 * disc of radius R centred on C + D s (s toward the sun), perpendicular to s, from a point
 * uniform over the disc, along -w with w uniform in the sun's cone, each with power
 * L_sun(lambda) Omega (s . w) pi R^2 / N (N photons per wavelength), so that the photons'
 * power through any plane is, in expectation, the sun's flux through the disc's shadow.  The
 * disc must cover the region of interest as seen from the sun.  Photon i of wavelength index
 * l draws on Philox (i, 0, bounce, photon stream, wavelength l); it is traced through the
 * subdomain queues like the camera paths: at glass it follows the Monte Carlo rules of the
 * camera paths (Fresnel choice at solid glass with Beer-Lambert inside, R / (R + T) at thin
 * slabs with the power times R + T, one brute-force ray through a heterogeneous tile on the
 * photon tile stream); at a diffuse surface it is stored, then survives with probability
 * albedo (power unchanged) into a cosine-distributed direction.  Maps: caustic (0) -- a
 * specular event changed the photon's direction (solid glass, a reflection at a slab, a
 * non-ballistic tile exit) before any diffuse surface; global (1) -- the photon was
 * reflected by a diffuse surface before.  A photon that reached its first diffuse surface
 * only through straight slab transmission (or ballistic tile exits) is direct light, which
 * the sun NEE counts, and is not stored.  Density estimate at x with normal n: the power of
 * the map's photons of that wavelength within gather_radius r of x that arrived on the
 * side of n, over pi r^2.  The photons of each map are sorted into a hashed uniform grid of
 * cell edge 2 r. */
typedef struct {
  int n_lambda;             /* wavelengths (each traced on its own), 1..4096 */
  const float* lambda_nm;   /* host [n_lambda], positive */
  int n_per_lambda;         /* photons per wavelength, N >= 1; n_lambda * N <= 2^31 - 1 */
  uint64_t seed;            /* Philox key */
  int max_depth;            /* surface interactions per photon, 1..255 */
  float center[3];          /* emitter disc: centre C + distance * s, radius R > 0 */
  float radius_m;
  float distance_m;
  float gather_radius_m;    /* density-estimation radius r > 0 */
} sdd_photon_opts;
/* Trace the photons and build both maps (device memory owned by the handle; the maps keep
 * no reference to the scene).  Requires a sun (SDD_ERR_STATE otherwise).  The stored-photon
 * buffers start at n_lambda * N entries per map and grow by tracing again when that was too
 * few; a map of more than 2^30 photons returns SDD_ERR_QUEUE_OVERFLOW. */
sdd_status sdd_photon_maps_build(sdd_scene* scene, const sdd_photon_opts* opts, sdd_photon_maps** out,
                                 void* cuda_stream);
void sdd_photon_maps_destroy(sdd_photon_maps* maps);
/* Stored photons per map. */
sdd_status sdd_photon_maps_count(const sdd_photon_maps* maps, int64_t* n_caustic, int64_t* n_global);
/* Copy the photons of map `map` (0 caustic, 1 global) to HOST arrays of count entries, in no
 * particular order: position [n][3], normal facing the photon's arrival [n][3], power [n],
 * wavelength index [n], photon index within its wavelength [n], diffuse surfaces met before
 * this one [n].  Any pointer may be NULL. */
sdd_status sdd_photon_maps_get(const sdd_photon_maps* maps, int map, float* pos, float* nrm, float* power,
                               int32_t* lam, uint32_t* id, uint32_t* seq);
/* Density estimates of both maps at n query points (device arrays): x [n][3], unit normal
 * [n][3], wavelength index [n] (an index with no photons gives 0); writes device
 * E_caustic [n] and E_global [n] (irradiance per nm in the illuminant's units). */
sdd_status sdd_photon_gather(const sdd_photon_maps* maps, int n, const float* x_dev, const float* nrm_dev,
                             const int32_t* lam_dev, float* e_caustic_dev, float* e_global_dev, void* cuda_stream);

/* sdd_trace_closest without any allocation (the paper has no counterpart; this serves
 * callers).  Same arguments, results and queue passes as sdd_trace_closest, but its scratch
 * (ray state, hit records, subdomain queues, counters) lives in one static 16 MiB device
 * array inside the library instead of the scene's workspace, and the call makes no
 * cudaMalloc, cudaFree or other allocating call.  It is meant for callers that run under a
 * device-memory budget fixed at start-up (a service that reserves its GPU memory up front,
 * or an application whose own allocator owns the device heap) and so cannot let a library
 * allocate when a batch arrives.
 *   - Capacity: n * (48 + 8 * n_subdomains) bytes plus a small control block must fit in
 *     16 MiB (about 149,000 rays at 8 subdomains); larger n returns SDD_ERR_ARG.
 *   - Every call looks up the array's device address on the current device.  Under CUDA's
 *     default lazy module loading the 16 MiB become device memory at the first lookup on a
 *     device, not when the process starts: a caller that budgets its memory at start-up
 *     makes one call with n = 0 then (it only does this set-up and returns).  That first
 *     call on a device should come before any stream capture.
 *   - The call synchronises the given stream before it returns (it reads the queue counts
 *     back after every pass).
 *   - Errors raised on the device come back as SDD_ERR_STACK (traversal stack or the walk's
 *     step bound), SDD_ERR_QUEUE_OVERFLOW (queue capacity) or SDD_ERR_TIMEOUT (a loop cap).
 *   - Every GPU that uses the library keeps the 16 MiB until the process exits.
 *   - All calls share the array and it keeps the previous call's contents; the call clears
 *     what must start at zero.  Calls whose GPU work overlaps (other threads or streams)
 *     race on the array: serialise them. */
sdd_status sdd_trace_closest_noalloc(sdd_scene* scene, int n, const float* org_dev, const float* dir_dev,
                                     float* t_out_dev, int32_t* prim_out_dev, void* cuda_stream);

/* Spectral material module on its own (for tests): for n queries with device arrays
 * cos_i, n, k, thickness_m, lambda_nm writes the single-interface reflectance R (air ->
 * n + ik), and the thin-slab reflectance / transmittance with the series of slab_polarisation
 * (as in sdd_scene_desc).  FP32, with the FP64 branch near grazing incidence exactly as the
 * renderer uses them. */
sdd_status sdd_eval_optics(int n, const float* cos_i, const float* n_re, const float* k,
                           const float* thickness_m, const float* lambda_nm, int slab_polarisation,
                           float* R_out, float* R_slab_out, float* T_slab_out, void* cuda_stream);

/* Philox4x32-10 as the renderer draws it: out[i] = philox(ctr[i], key) for device uint32
 * arrays ctr [n][4] and out [n][4]. */
sdd_status sdd_philox(int n, const uint32_t* ctr_dev, uint64_t key, uint32_t* out_dev, void* cuda_stream);

const char* sdd_last_error(void);
const char* sdd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SDD_H */

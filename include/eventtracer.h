/*
 * eventtracer.h -- C ABI of libeventtracer, a GB300 (sm_103a) implementation of
 * the EventTracer hot path (arXiv 2508.18071): path tracing of every frame of a
 * 1 kHz camera path through a triangle scene, then the EvSNet spiking network
 * (convolutions + bipolar leaky integrate-and-fire) that turns the noisy frames
 * into ON/OFF events (t, x, y, p).
 *
 * The problem statement these calls follow is the paper's Sec. 3.2: time is cut
 * into K = T * F_evt steps, a frame I_k is rendered at every t_k = k / F_evt,
 * each pixel's log-luminance sequence is differenced (Eq. 1) and EvSNet
 * (Eq. 5-6, BiLIF of Eq. 2-3) emits the events of Sec. 3.1.
 *
 * Conventions for every call:
 *  - Return value: ET_OK or an ET_ERR_* code; et_status_str() names it.  Argument
 *    errors are detected on the host before anything is enqueued.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *    stream).  Device outputs are valid once the stream has been synchronised.
 *  - The caller owns every input and output buffer.  Buffers marked "device" are
 *    device pointers (e.g. torch tensors' data_ptr()); "host" are host pointers.
 *    The library owns only an et_scene and the device memory it holds.
 *  - Event outputs: the call writes the event count to the device int64
 *    `*n_events` (the library zeroes it first).  If more than `cap` events were
 *    produced, only `cap` are stored and *n_events is the full count: the caller
 *    compares after synchronising and retries with a larger buffer.
 *  - Events are emitted in no particular order.
 *  - No call allocates device memory except et_build_scene, the first
 *    et_scene_update of a scene, and the training
 *    workspace query / et_train_* calls that say so.
 */
#ifndef EVENTTRACER_H
#define EVENTTRACER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ET_OK = 0,
  ET_ERR_ARG = 1,            /* bad argument (null pointer, size out of range)     */
  ET_ERR_CUDA = 2,           /* a CUDA runtime call or kernel launch failed        */
  ET_ERR_OOM = 3,            /* device allocation failed                           */
  ET_ERR_CAPACITY = 4,       /* host-synchronous calls only: output buffer too small */
  ET_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up                 */
  ET_ERR_UNIMPLEMENTED = 6   /* configuration not supported by this build          */
};

enum { ET_LAMBERT = 0, ET_GGX = 1 };
enum { ET_LOG_EPS = 0,       /* l = ln(L + eps)                           (default) */
       ET_LOG_PAPER = 1 };   /* Eq. 1 as printed: ln L if L >= rho else (ln rho / rho) L */
enum { ET_F32 = 0, ET_BF16 = 1, ET_FP8 = 2 };
enum { ET_NET_STACK = 0,     /* plain stack of conv + ReLU layers                   */
       ET_NET_RESIDUAL = 1 };/* Eq. 5: encoder conv + M residual blocks            */

typedef struct et_scene et_scene;

/* Material: albedo (Lambert) or Schlick F0 (GGX); GGX alpha = roughness. */
typedef struct { float albedo[3]; float roughness; int32_t type; } et_material;

/* One-sided parallelogram light: points p0 + u e1 + v e2, (u, v) in [0,1)^2, emitting
 * radiance on the side of e1 x e2.  et_build_scene appends its two triangles
 * (p0, p0+e1, p0+e1+e2) and (p0, p0+e1+e2, p0+e2) to the geometry. */
typedef struct { float p0[3], e1[3], e2[3]; float radiance[3]; } et_quad_light;

/* Pinhole camera: position, camera-to-world rotation stored row-major whose
 * columns are the camera's right, up and backward axes, vertical FOV (degrees). */
typedef struct { float pos[3]; float rot[9]; float vfov_deg; } et_camera;

/* Event (Sec. 3.1): pixel (x, y), frame index t (time t / F_evt), polarity +-1. */
typedef struct { uint16_t x, y; uint32_t t; int8_t p; uint8_t pad[3]; } et_event;

/* ---------------------------------------------------------------------- scene
 * Builds the scene: copies the geometry to the device and builds a surface-area
 * heuristic bounding volume hierarchy (two-wide, leaves of at most 4
 * triangles) with the default builder ET_BVH_DEFAULT (see et_build_scene_with).
 *   tris      host float [n_tris][9]: v0, v1, v2 of each triangle
 *   tri_mat   host uint32 [n_tris]: material index (< n_mats)
 *   mats      host [n_mats];  lights host [n_lights] (may be 0)
 *   env       radiance of the constant environment seen by rays that miss
 * Allocates device memory owned by *out (freed by et_scene_free).  Synchronous.
 * Errors: ET_ERR_ARG (null pointers, n_tris < 0, material index out of range),
 * ET_ERR_OOM, ET_ERR_CUDA. */
int et_build_scene(const float* tris, const uint32_t* tri_mat, int64_t n_tris,
                   const et_material* mats, int32_t n_mats,
                   const et_quad_light* lights, int32_t n_lights, float env,
                   et_scene** out, void* stream);
/* Hierarchy builders, all minimising the SAH cost C = 1 + (A_L N_L + A_R N_R) / A
 * per split (leaf cost N):
 *   ET_BVH_GPU_SWEEP  every split of the centroid order on each axis, on the
 *                     device, level by level (the default: the host sweep's
 *                     tree and node order, built on the GPU);
 *   ET_BVH_GPU        32 centroid bins per axis, on the device, level by level;
 *   ET_BVH_HOST       the same binned heuristic on the host;
 *   ET_BVH_SWEEP      every split of the centroid order on each axis, on the host
 *                     (O(n log n); the full sweep's trees need fewer traversal
 *                     steps than the binned ones).
 * A requested build whose tree is deeper than the traversal stack's 64 levels
 * (or a GPU build that fails) is replaced by the host binned build. */
enum { ET_BVH_GPU = 0, ET_BVH_HOST = 1, ET_BVH_SWEEP = 2, ET_BVH_GPU_SWEEP = 3 };
#define ET_BVH_DEFAULT ET_BVH_GPU_SWEEP
/* et_build_scene with an explicit builder.  Errors as et_build_scene, and
 * ET_ERR_ARG for an unknown builder. */
int et_build_scene_with(const float* tris, const uint32_t* tri_mat, int64_t n_tris,
                        const et_material* mats, int32_t n_mats,
                        const et_quad_light* lights, int32_t n_lights, float env,
                        int32_t builder, et_scene** out, void* stream);
void et_scene_free(et_scene* scene);
/* Moving geometry: new positions for the scene's triangles (host float
 * [n_tris][9], input order, the same count as at build; the lights stay).  The
 * hierarchy keeps its topology and its boxes are recomputed bottom-up (refit),
 * exactly enclosing the new triangles, so closest hits stay exact; its quality
 * degrades as the motion grows relative to the scene (rebuild then).
 * et_scene_info's SAH cost is that of the build.  Stream-ordered: renders
 * queued on `stream` before the call see the old geometry, later ones the new;
 * do not render the scene on another stream meanwhile.  The first call
 * allocates a staging buffer of n_tris x 36 bytes owned by the scene.
 * Errors: ET_ERR_ARG, ET_ERR_OOM, ET_ERR_CUDA. */
int et_scene_update(et_scene* scene, const float* tris, void* stream);
/* Which builder produced the hierarchy (ET_BVH_*). */
int et_scene_builder(const et_scene* scene);
/* Triangle count (including the lights' triangles), BVH node count and its SAH
 * cost (C_trav = C_isect = 1, normalised by the root's surface area). */
int et_scene_info(const et_scene* scene, int64_t* n_tris, int64_t* n_nodes, double* sah_cost);

/* --------------------------------------------------------------------- render
 * Sec. 3.2: renders frames first_frame .. first_frame + n_frames - 1 of a camera
 * path by Monte Carlo path tracing with `spp` samples per pixel and paths of at
 * most `max_depth` segments, next-event estimation to the quad lights with MIS,
 * Lambertian and GGX BSDFs, and Philox4x32-10 random numbers keyed by
 * (seed) and counted by (pixel, sample, frame, 4 * bounce + use).
 *   cams      host [n_frames] cameras (copied; the pointer may be reused at once)
 *   rgb       device float [n_frames][H][W][3] mean linear radiance, or NULL
 *   logl      device float [n_frames][H][W] Eq. 1 log luminance, or NULL:
 *             log_mode ET_LOG_EPS: ln(L + log_param); ET_LOG_PAPER: rho = log_param;
 *             evaluated in FP32 (within 1 ulp of the correctly rounded value)
 *   records   device int32 [n_frames][H][W][spp][max_depth][2] or NULL: per path
 *             segment the triangle hit (-1 miss, -2 not traced) and the light
 *             sampling record (2 * light + visible, -1 none) -- for testing
 * Calls on one scene must be issued on one stream (the scene holds the cameras).
 * Errors: ET_ERR_ARG (W, H, spp, max_depth out of [1, 65535] / [1, 4096] / [1, 16],
 * n_frames < 0, both outputs NULL), ET_ERR_UNIMPLEMENTED (the wavefront
 * schedules with W x H >= 2^31 pixels), ET_ERR_CUDA. */
int et_render_frames(const et_scene* scene, const et_camera* cams, int32_t n_frames,
                     int32_t first_frame, int32_t W, int32_t H, int32_t spp,
                     int32_t max_depth, uint64_t seed, float* rgb, float* logl,
                     int32_t log_mode, float log_param, int32_t* records, void* stream);

/* Rows y0 <= y < y1 of the same W x H frames (0 <= y0 < y1 <= H): rgb, logl and
 * records are [n_frames][y1 - y0][W]..., bit for bit those rows of the full
 * frames (rays and random numbers keep the full image's pixel index).  This is
 * the unit of the row-band partition across GPUs.  Errors as et_render_frames,
 * and ET_ERR_ARG for an empty or out-of-range band. */
int et_render_rows(const et_scene* scene, const et_camera* cams, int32_t n_frames,
                   int32_t first_frame, int32_t W, int32_t H, int32_t y0, int32_t y1, int32_t spp,
                   int32_t max_depth, uint64_t seed, float* rgb, float* logl, int32_t log_mode,
                   float log_param, int32_t* records, void* stream);

/* Annotations of the primary hit through each pixel centre (no jitter), the
 * by-products that come with the rendered events (the paper's outputs extend
 * to depth and segmentation, Sec. 1), for n_frames cameras:
 *   depth     device float [F][H][W]: distance of the hit along the viewing axis
 *             (t times the cosine to it), +inf on a miss
 *   normal    device float [F][H][W][3]: unit geometric normal facing the ray,
 *             0 on a miss
 *   prim      device int32 [F][H][W]: triangle index in input order (the lights'
 *             two triangles each follow the user triangles), -1 on a miss
 *   material  device uint32 [F][H][W]: the triangle's material index (light
 *             triangles: 0x80000000 | light index), 0xFFFFFFFF on a miss
 *   flow      device float [F][H][W][2]: position of the hit point in the next
 *             frame's image minus this pixel's centre, in pixels (x right, y
 *             down); NaN on a miss, behind the next camera, or for the last
 *             frame when next_cam (host, may be NULL) is not given
 * Any output may be NULL (not all).  cams / next_cam: host.  Asynchronous.
 * Errors: ET_ERR_ARG, ET_ERR_CUDA. */
int et_render_annotations(const et_scene* scene, const et_camera* cams, int32_t n_frames,
                          const et_camera* next_cam, int32_t W, int32_t H, float* depth,
                          float* normal, int32_t* prim, int32_t* material, float* flow,
                          void* stream);

/* Schedule used by et_render_frames on this scene; all compute identical
 * outputs.  ET_RENDER_WAVEFRONT: paths advance one segment at a time
 * through compacted ray queues traced by persistent warps that refill idle
 * lanes; it keeps a device workspace in the scene (up to ~1.3 GB for 8M paths
 * in flight), allocated by the first call that needs it and kept until
 * et_scene_free.  ET_RENDER_MEGAKERNEL: one thread per pixel, no workspace.
 * ET_RENDER_WAVEFRONT_TILES (default): the wavefront schedule with each warp's
 * primary rays taken from an 8 x 4 pixel tile instead of 32 pixels of one row
 * (when W is a multiple of 8 and the rendered rows of 4; else raster order).
 * ET_RENDER_WAVEFRONT_SORTED: the tiled schedule with each bounce's
 * continuation rays sorted by direction cell and origin cell (a stable radix
 * sort on a 24-bit key) before they are traced; a further ~16 B per path of
 * workspace, kept like the rest.
 * Errors: ET_ERR_ARG. */
enum { ET_RENDER_WAVEFRONT = 0, ET_RENDER_MEGAKERNEL = 1, ET_RENDER_WAVEFRONT_TILES = 2,
       ET_RENDER_WAVEFRONT_SORTED = 3 };
int et_render_set_mode(et_scene* scene, int32_t mode);

/* The counter-based generator behind every random number of the renderer
 * (camera jitter, light and BSDF samples; Sec. 3.2's Monte Carlo estimator)
 * and of the sensor model: Philox4x32-10 (Salmon et al., SC'11), evaluated on
 * the device for caller counters and keys, for testing it bit for bit.
 *   ctr  device uint32 [n][4] (16-byte aligned), key device uint32 [n][2]
 *   (8-byte aligned), out device uint32 [n][4] (16-byte aligned).
 * Errors: ET_ERR_ARG (null or misaligned buffers, n < 0), ET_ERR_CUDA. */
int et_philox4x32_10(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out, void* stream);

/* Per-kernel device time of the wavefront schedule, for measurement (not part
 * of the method).  et_render_profile(scene, 1): every later et_render_frames
 * call on this scene records a CUDA event before and after each of its
 * kernels and copies the length of the queue each kernel processed to pinned
 * host memory (allocated here, once); 0 stops recording.  Events add a little
 * time of their own; leave profiling off for timed runs of the whole call.
 * et_render_profile_read waits for the recorded work and returns, summed since
 * the previous read and indexed raygen 0, closest-hit trace 1, shade 2,
 * shadow trace 3, accumulate 4: ms[5] device milliseconds, launches[5], and
 * items[5] = paths generated, rays traced, hits shaded, shadow rays traced and
 * pixel-frames resolved (in ET_RENDER_WAVEFRONT_SORTED the shade time holds
 * the sort of the continuation queue).  ET_ERR_CAPACITY: more than 32768 queue lengths were
 * recorded between reads (the times stay valid, the counts are short). */
int et_render_profile(et_scene* scene, int32_t enable);
int et_render_profile_read(et_scene* scene, double* ms, int64_t* launches, int64_t* items);

/* ---------------------------------------------------------- threshold events
 * Sec. 3.1 contrast-threshold model (the method without EvSNet, the 256-SPP
 * reference and the training target).  Per pixel, in FP64:
 *   d = l_k - ref;  n = floor(|d| / C);  emit n events (x, y, t0 + k, sgn d);
 *   ref += sgn(d) n C.
 *   logl      device float [F][H][W]
 *   ref       device double [H * W] state; when initialized == 0 the first frame
 *             only sets ref (no events), else every frame is a step
 *   events    device [cap];  n_events device int64 (see conventions)
 * Errors: ET_ERR_ARG (C <= 0, sizes), ET_ERR_CUDA. */
int et_threshold_events(const float* logl, int32_t F, int32_t H, int32_t W, float C, int32_t t0,
                        double* ref, int32_t initialized, et_event* events, int64_t cap,
                        int64_t* n_events, void* stream);

/* --------------------------------------------------------------- sensor model
 * Contrast-threshold events with sub-frame timestamps and the sensor
 * non-idealities the paper names beside internal-state bias and saturation
 * (Sec. 3.1: threshold mismatch, leak events, shot noise; the reset period
 * behind the saturation effect).  The paper gives no formulas; this model:
 *   - frame k is at time k (frames); between frames the log intensity is
 *     linear in time;
 *   - per-pixel thresholds C_on/off = C max(0.01, 1 + sigma_C z), z = (u0 + u1 +
 *     u2 + u3 - 2) sqrt 3 (unit variance), u = Philox4x32-10(key = seed,
 *     counter = (pixel y W + x, 0xFFFFFFFF, 0 ON / 1 OFF, 0x53454E53)) as
 *     (u32 >> 8) 2^-24;
 *   - per step k-1 -> k: the reference drops by C_on leak_hz / frame_hz (leak);
 *     then repeatedly the pixel fires at the earliest t >= max(k - 1, t_last +
 *     refractory) in the step where l(t) - r >= C_on (ON) or r - l(t) >= C_off
 *     (OFF), moving r by +-C_on/off and setting t_last = t; finally, with
 *     probability shot_hz / frame_hz, one shot-noise event at t = k - 1 + v of
 *     polarity + if w < 1/2 (u, v, w from counter (pixel, k, 2, 0x53454E53));
 *     shot events leave the state alone;
 *   - event records carry t = floor(time * 1e6 / frame_hz) in microseconds.
 * With sigma_C = 0 and no refractory period, leak or shot noise each step emits
 * the contrast-threshold generator's floor(|l_k - r| / C) events.  At most 1024
 * threshold events per pixel and step (a bound on the work): further crossings
 * of that step are dropped and the reference stops there.  Decisions
 * are FP64 with explicit rounding: bit-reproducible.  Float parameters are
 * widened to FP64 as given. */
typedef struct {
  float C;              /* nominal threshold (log units), > 0 */
  float sigma_C;        /* relative per-pixel threshold spread (std), >= 0 */
  float refractory_us;  /* >= 0 */
  float leak_hz;        /* leak-event rate of a static pixel, >= 0 */
  float shot_hz;        /* shot-noise events per pixel and second, <= frame_hz */
  float frame_hz;       /* frame rate F_evt, > 0 (1000 for 1 kHz) */
  uint64_t seed;        /* Philox key for the mismatch and the shot noise */
} et_sensor_params;

/* Events of F log frames (device float [F][H][W]; frame f is frame t0 + f of
 * the clip).  state: device double [H*W][3] = (reference, time of the last
 * event, previous log intensity); with initialized = 0 the first frame only
 * sets it (t0 >= 0), else the call continues the clip (t0 >= 1).  Events as
 * et_threshold_events, with t in microseconds.
 * Errors: ET_ERR_ARG (sizes, parameters outside the ranges above, times that
 * overflow 32 bits), ET_ERR_CUDA. */
int et_sensor_events(const float* logl, int32_t F, int32_t H, int32_t W,
                     const et_sensor_params* params, int32_t t0, double* state,
                     int32_t initialized, et_event* events, int64_t cap, int64_t* n_events,
                     void* stream);

/* --------------------------------------------------------------------- EvSNet
 * Weights (device, FP32, packed): conv layers 0..n_layers-1 in order, each
 * W[C][Cin][kt][ks][ks] with Cin = 1 for layer 0 and C otherwise, then the
 * point-wise projection W[C]; biases: C per conv layer, then 1.
 * kind ET_NET_STACK: h = ReLU(conv_i(h)) for every layer.
 * kind ET_NET_RESIDUAL (Eq. 5): n_layers = 1 + 2M, h_0 = ReLU(conv_0(X)),
 *   h_i = ReLU(h_{i-1} + conv_{2i}(ReLU(conv_{2i-1}(h_{i-1})))).
 * Temporal taps are causal (tap kt-1 = current step); spatial padding is zero.
 * BiLIF (Eq. 2-3; fire on the pre-reset potential):
 *   V' = beta V + I;  S = +1 if V' >= vth, -1 if V' <= -vth, else 0;  V = V' - reset S.
 * dtype: ET_F32 (CUDA cores), ET_BF16 or ET_FP8 (tensor cores, FP32 accumulation).
 *   ET_BF16 rounds the weights of layers 1.. and their inputs to BF16.
 *   ET_FP8 rounds them to E4M3 after scaling by powers of two (exact to undo):
 *   weights per output channel, by the one that brings their absolute maximum
 *   to at most 448; layer inputs of the 3x3 form per layer, 32x16 pixel tile
 *   and step, by the one that brings a bound on their maximum to at most 448
 *   (the tile's largest log difference times the layer-0 weights' row sums for
 *   layer 0's output, then the largest input times the layer's row sums plus
 *   the bias); layer inputs of the pixel-wise form by the fixed per-layer
 *   scales of `scales` (a tensor-core layer's MMA sums several time steps, so
 *   their scales must agree): tensor-core layer l's input is divided by
 *   scales[l - 1] and rounded to E4M3 with saturation at +-448
 *   (et_evsnet_fp8_scales finds them on a calibration clip).
 *   Layer 0, the projection and BiLIF stay FP32 in both.
 * ks0 (this library's spatio-temporal form; the paper's EvSNet is pixel-wise):
 *   0, or an odd size 1..7 that makes layer 0 a one-step ks0 x ks0 spatial
 *   convolution of the current X (weights W[C][1][1][ks0][ks0], zero padding)
 *   ahead of temporal layers (ks = 1); layer 0 then keeps no history.  The
 *   CUDA kernels take ks0 > 0 only with ks = 1.
 * delay >= 0: the events of step k carry t = t0 + k - delay (a network trained
 *   on a window centred delay steps back labels its output with that centre;
 *   the Sec. 4.1 network with "same" padding corresponds to delay 21); steps
 *   whose label would be negative emit no events.
 */
typedef struct {
  int32_t kind, n_layers, C, kt, ks;
  float beta, vth, reset;
  int32_t dtype;
  int32_t ks0;        /* 0: layer 0 is kt x ks x ks; > 0: one step, ks0 x ks0 */
  int32_t delay;      /* event label offset (steps) */
  const float* w;     /* device */
  const float* b;     /* device */
  const float* scales;  /* device float [n_layers - 1]: positive powers of two, the
                           ET_FP8 pixel-wise form's input scales (NULL otherwise) */
} et_evsnet_weights;

/* Per-pixel state carried between calls (all device, caller-allocated):
 *   V       float [H * W] membrane potential
 *   hist    float [n_layers][kt-1][C][H][W] past inputs of every layer (NULL if kt == 1)
 *   last_l  float [H * W] log luminance of the previous frame
 *   initialized: 0 before the first call (the first frame then only sets last_l);
 *   et_evsnet_forward sets it to 1. */
typedef struct {
  float* V;
  float* hist;
  float* last_l;
  int32_t H, W;
  int32_t initialized;
} et_evsnet_state;

/* Eq. 1 (X_k = l_k - l_{k-1}) + Eq. 5-6 + BiLIF over F log frames.
 *   logl     device float [F][H][W]
 *   events   device [cap], n_events device int64 (see conventions); t = t0 + frame
 *   I_out    device float [K][H][W] projection output (BiLIF input), or NULL
 *   spikes   device int8 [K][H][W] dense spikes, or NULL
 * K = F - 1 if the state was not initialized, else F.
 * Errors: ET_ERR_ARG (also: ET_FP8 for the pixel-wise form without scales),
 * ET_ERR_UNIMPLEMENTED (C > 32, ks > 7, kt > 9, BF16 or FP8 for a shape the
 * tensor-core kernels do not cover: plain stacks of 2 to 6 layers of 3x3
 * spatial convolutions; the pixel-wise form with C <= 16, kt <= 7 and at least
 * two layers), ET_ERR_CUDA. */
int et_evsnet_forward(const float* logl, int32_t F, const et_evsnet_weights* net,
                      et_evsnet_state* state, int32_t t0, et_event* events, int64_t cap,
                      int64_t* n_events, float* I_out, int8_t* spikes, void* stream);

/* Calibration of the FP8 pixel-wise form's input scales: runs the BF16
 * tensor-core forward of `net` (its dtype and scales are ignored) over the F
 * log frames (arguments and state as et_evsnet_forward; the state advances and
 * no events are kept), takes the largest value m_l each tensor-core layer l
 * receives, and writes scales[l - 1] = the smallest power of two s with
 * headroom * m_l / s <= 448 (1 where m_l = 0).  scales: device float
 * [n_layers - 1].  headroom >= 1 leaves room for inputs larger than the
 * calibration clip's (beyond it they saturate).  Allocates and frees a few
 * bytes of device memory (stream-ordered): not for the per-frame path.
 * Errors: ET_ERR_ARG, ET_ERR_UNIMPLEMENTED (a shape the BF16 pixel-wise
 * kernel does not cover), ET_ERR_CUDA. */
int et_evsnet_fp8_scales(const float* logl, int32_t F, const et_evsnet_weights* net,
                         et_evsnet_state* state, float headroom, float* scales, void* stream);

/* ------------------------------------------------------------------ training
 * The learned form: EvSNet with FP32 weights, <= 16 channels, trained on B clips
 * of K steps, in either of two forms: the spatial one (plain stack of 3x3
 * convolutions, kt = 1) or the paper's pixel-wise temporal one (ks = 1, causal
 * kernel kt <= 9, plain stack or residual blocks, Eq. 5).  Inputs are log frames
 * logl [B][K+1][H][W] (device, FP32; step k uses X = l_{k+1} - l_k, Eq. 1) and
 * targets E [B][K][H][W] (device, FP32 signed event counts per step).
 * Spikes follow Eq. 3 read as S_on = Theta(V' - Vth), S_off = Theta(-V' - Vth);
 * the backward uses the surrogate of Eq. 4, s(x) = (alpha/2) / (1 + (pi alpha x / 2)^2),
 * on both thresholds and differentiates the reset.  The membrane starts at 0.
 * Backpropagation through time keeps V at the start of every segment of
 * ckpt_every (<= 32) steps and recomputes each segment in the backward.
 * net->dtype: ET_F32 (everything in FP32 on the CUDA cores), or, for the
 * spatial form only, ET_BF16: the forward, data gradient and weight gradient
 * of the C -> C convolutions (layers 1..) take BF16 operands on the tensor
 * cores with FP32 accumulation (the workload's "BF16 convolutions, FP32
 * accumulation"); layer 0, BiLIF, the loss and the weights stay FP32. */
typedef struct { int32_t B, K, H, W, ckpt_every; } et_train_shape;

/* Bytes of the caller-allocated device workspace the two calls below need:
 * spatial form: the activations of one segment plus its gradients (about
 * (2 n_layers + 2) C B ckpt_every H W floats); temporal form: the activations
 * of the whole clip (about (n_layers + 3) C B K H W floats). */
int et_train_workspace_bytes(const et_evsnet_weights* net, const et_train_shape* shape,
                             size_t* bytes);

/* Forward over the batch.  Outputs (device): spikes int8 [B][K][H][W] (S_on - S_off),
 * optional S_on / S_off float [B][K][H][W] (both or neither), V_ckpt float
 * [B][ceil(K / ckpt_every)][H][W], optional I_out float [B][K][H][W].
 * Errors: ET_ERR_ARG, ET_ERR_UNIMPLEMENTED (a form other than the two above,
 * C > 16, dtype other than ET_F32 / ET_BF16 or ET_BF16 for the temporal form,
 * ckpt_every > 32), ET_ERR_CUDA.  With ET_BF16, a tensor-core wait that runs
 * out of its bound (et_set_wait_budget) leaves NaN in the affected outputs. */
int et_evsnet_train_forward(const float* logl, const et_train_shape* shape,
                            const et_evsnet_weights* net, int8_t* spikes, float* S_on,
                            float* S_off, float* V_ckpt, float* I_out, void* workspace,
                            size_t workspace_bytes, void* stream);

/* Eq. 7-11: per pixel, for each polarity, half the sum of the 1-D EMD of the
 * sequences and of the reversed sequences (EMD(E, S) = (1/K) sum_i |cumsum(S - E)_i|),
 * plus lambda |sum |S| - sum |E||; averaged over the B H W pixels.
 * loss: device float [3] = (total, EMD part, count part); dS_on / dS_off: device
 * float [B][K][H][W] gradients of the total.  Errors: ET_ERR_ARG, ET_ERR_CUDA. */
int et_emd_count_loss(const int8_t* spikes, const float* E, const et_train_shape* shape,
                      float lambda, float* loss, float* dS_on, float* dS_off, void* stream);

/* Backward through BiLIF and the convolutions; gradients are ADDED to grad_w /
 * grad_b (device, packed like the weights; zero them first).  Errors as forward. */
int et_evsnet_train_backward(const float* logl, const et_train_shape* shape,
                             const et_evsnet_weights* net, const float* V_ckpt,
                             const float* dS_on, const float* dS_off, float alpha, float* grad_w,
                             float* grad_b, void* workspace, size_t workspace_bytes, void* stream);

/* et_evsnet_train_backward without a workspace argument, for callers that
 * cannot allocate device memory: e.g. a plugin inside a framework whose own
 * allocator owns all device memory, or a loop that must not call cudaMalloc /
 * cudaFree because they can synchronise the device.  The paper has no
 * counterpart; this is a deployment convenience of the library.
 * The scratch is one array of et_train_static_workspace_capacity() bytes
 * (32 MiB) compiled into the library; every device that loads the library
 * holds it until the process exits.  Shapes needing more scratch than that
 * (see et_train_workspace_bytes) are rejected with ET_ERR_CAPACITY.  The call
 * itself allocates nothing.  The first call on a device looks up the array's
 * device address (that device must be current); make that first call before
 * any stream capture begins.  The address is tied to the context it was looked
 * up in: after cudaDeviceReset (a new primary context) the next call looks it
 * up again, so that call too should come before any capture.  All calls share the one array and it keeps the
 * previous call's contents (the call clears what must start at zero), so two
 * calls whose execution overlaps on the GPU -- e.g. on different streams --
 * race and give wrong gradients: serialise them.  Results, errors and the
 * meaning of every other argument are those of et_evsnet_train_backward. */
int et_evsnet_train_backward_static(const float* logl, const et_train_shape* shape,
                                    const et_evsnet_weights* net, const float* V_ckpt,
                                    const float* dS_on, const float* dS_off, float alpha,
                                    float* grad_w, float* grad_b, void* stream);
size_t et_train_static_workspace_capacity(void);

/* Adam (Kingma & Ba 2015) with bias correction, FP32, in place on p, m, v (device, n).
 * step >= 1 is the 1-based update count.  Errors: ET_ERR_ARG, ET_ERR_CUDA. */
int et_adam_step(float* p, const float* g, float* m, float* v, int64_t n, float lr, float beta1,
                 float beta2, float eps, int32_t step, void* stream);

/* ------------------------------------------------------------------ metrics
 * Size of a maximum matching between two event lists (host pointers): events
 * match when they share (x, y, p) and |t_a - t_b| <= delta; each event matches
 * at most once.  Event F1 = 2 m / (n_a + n_b).  The paper reports no event-level
 * score; this is the project's fidelity measure of a rendered stream against the
 * 256-SPP contrast-threshold stream.  Synchronous, host only.
 * Errors: ET_ERR_ARG. */
int et_event_matches(const et_event* a, int64_t n_a, const et_event* b, int64_t n_b,
                     int32_t delta, int64_t* matches);

/* The same maximum-matching size for two dense spike tensors a, b (device,
 * int8 [K][npix], values -1 / 0 / +1 as written by et_evsnet_forward's spike
 * output; the step index is the event time): one thread per pixel, on
 * `stream`.  *matches (device, one int64) is overwritten when the kernel
 * completes.  0 <= delta <= 30.  Errors: ET_ERR_ARG, ET_ERR_CUDA. */
int et_spike_matches(const int8_t* a, const int8_t* b, int64_t K, int64_t npix, int32_t delta,
                     int64_t* matches, void* stream);

const char* et_status_str(int status);

/* Number of CUDA kernels the library has launched in this process (all
 * devices, all calls); a monotone counter for instrumentation. */
uint64_t et_kernel_launches(void);

/* Failure detection.  The tensor-core EvSNet kernel waits on its MMAs with a
 * bounded number of mbarrier polls (default 2^22).  When a wait runs out the
 * kernel sets bit 62 of *n_events (which the caller reports as ET_ERR_TIMEOUT),
 * leaves the membrane state of the call untouched, waits once more with the
 * default bound for the MMAs still in flight, frees its tensor memory and
 * returns; the context stays usable.  The call's previous-frame buffer and
 * `initialized` flag are still updated (the host does not see the timeout until
 * it reads the count): restore the state from a copy before retrying.
 * The BF16 training convolutions bound their waits the same way; on expiry
 * they write NaN into the outputs they own (activations, currents, gradients).
 * et_set_wait_budget(polls) sets the first bound for launches made afterwards in
 * this process: polls >= 0 sets it (0 gives up at once and forces the timeout
 * path, for testing the detection), polls < 0 restores the default.  (A poll
 * is one mbarrier.try_wait, which may itself suspend the thread for a while.)
 * Not thread-safe against concurrent launches. */
void et_set_wait_budget(int64_t polls);

#ifdef __cplusplus
}
#endif
#endif /* EVENTTRACER_H */

/*
 * cgdir.h -- C ABI of the GB300 (sm_103a) implementation of contour-guided
 * demons deformable image registration (CG-DIR; Gu, Dong, Wang, Yordy, Mell,
 * Jia, Jiang, "A Contour-Guided Deformable Image Registration Algorithm for
 * Adaptive Radiotherapy", arXiv:1301.0970).
 *
 * The library registers a moving CT I0 (planning CT) onto a static CT T0
 * (treatment CT) and returns the deformation vector field u (DVF) that
 * minimises Eq. 2: the demons energy plus, for each structure pair i, the
 * intensity mismatch of the modified images I_i, T_i weighted by lambda_i.
 * The optimisation is the relaxation of Eq. 3 run as Algorithm A (Sec. 2.2):
 * per iteration, the moving vector du of Eq. 7, a Gaussian smoothing of du,
 * the composite update u <- u o (Id + du), a Gaussian smoothing of u, the
 * warp of the images and the UROI stopping metric; over a coarse-to-fine
 * pyramid with plain demons at the coarse levels.
 *
 * Conventions used everywhere below
 *  - Volumes are dense [nz][ny][nx] arrays, x fastest (element (x, y, z) at
 *    offset (z*ny + y)*nx + x).  Displacement fields are [3][nz][ny][nx]
 *    float32 (component 0 = x, 1 = y, 2 = z), in voxel units of their level.
 *  - Warp convention: pull-back, I0~(x) = I0(x + u(x)) (the Taylor step before
 *    Eq. 5 makes T0 - I0~ the residual of Eq. 7).  Trilinear interpolation
 *    with coordinates clamped to the volume; gradients are central
 *    differences with clamped indices; smoothing is clamp-to-edge.
 *  - Structure masks: k <= 8 structure pairs.  The i-th moving mask O_i^p
 *    pairs with the i-th static mask O_i^t (Sec. 2.1).  Inside the library
 *    they are bit-packed, one uint8 per voxel per side, bit i = structure i.
 *  - Modified images (Sec. 2.1): I_i = (1 + s_i m_i/2)(I0 + offset),
 *    T_i = (1 + s_i n_i/2)(T0 + offset), m_i, n_i in {0,1}, s_i = +-1, with
 *    offset = intensity_offset (HU -> CT number; it cancels in the demons
 *    term).  They are never stored: the force kernel forms them per
 *    interpolation corner from I0 and the mask bits.
 *  - Pointers: "device" pointers are CUDA device (or managed) memory of the
 *    context's device; "host" pointers are ordinary (pageable or pinned) host
 *    memory.  The caller owns every pointer it passes; the library never
 *    frees or retains them past the call.  Device inputs must stay valid
 *    until the work of the call has completed on the context's stream.
 *  - Errors: every int-returning function returns CGDIR_OK (0) or one of the
 *    CGDIR_E* codes; cgdir_strerror() names the code and cgdir_last_error()
 *    gives the message of the last failure on a context.  No exception and
 *    no abort crosses this boundary.  A CGDIR_ECUDA failure leaves the
 *    context usable unless the CUDA context itself is lost.
 *  - Threading: a context is not thread-safe; use one per host thread.  The
 *    work of cgdir_register and of the primitives is ordered on the
 *    context's stream; batches and served requests also run on private
 *    streams of the context (see cgdir_register_batch, cgdir_submit).
 */
#ifndef CGDIR_H
#define CGDIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define CGDIR_OK         0
#define CGDIR_EINVAL     1   /* bad shape, dtype, count, pointer or parameter  */
#define CGDIR_ENOMEM     2   /* device memory or the context budget exhausted   */
#define CGDIR_ECUDA      3   /* a CUDA runtime call failed                      */
#define CGDIR_ETIMEDOUT  4   /* a bounded wait ran out                          */
#define CGDIR_ECANCELED  5   /* the request was cancelled                       */
#define CGDIR_EBUSY      6   /* no free slot / budget right now (retry later)   */

/* ---- enums ------------------------------------------------------------- */
#define CGDIR_F32   0        /* image storage types                             */
#define CGDIR_F16   1
#define CGDIR_BF16  2
#define CGDIR_STORAGE_AUTO (-1)   /* pyramid images keep the input type       */

#define CGDIR_HOST    0      /* where a buffer lives                            */
#define CGDIR_DEVICE  1

#define CGDIR_STOP_FIXED          0  /* run each level's iteration cap          */
#define CGDIR_STOP_WINDOW10       1  /* stop at n >= 10 once d[n-10]-d[n] <= eps */
#define CGDIR_STOP_PAPER_LITERAL  2  /* l[n]=d[n]-d[n-1]; stop once n >= 11 and
                                        l[n-10]-l[n] <= eps (Sec. 2.2, as printed) */

#define CGDIR_COMPOSE   0    /* u <- u o (Id + du), Algorithm A step 3          */
#define CGDIR_ADDITIVE  1    /* u <- u + du (classic Thirion variant)          */

#define CGDIR_REASON_CAP        0   /* the level ran its iteration cap          */
#define CGDIR_REASON_CONVERGED  1   /* the stopping test fired                  */
#define CGDIR_REASON_SKIPPED    2   /* level skipped (init_dvf given)          */

#define CGDIR_MAX_MASKS   8
#define CGDIR_MAX_LEVELS  8
#define CGDIR_MAX_SIGMA   2.0f   /* Gaussian radius ceil(3 sigma) <= 6         */

/* ---- types ------------------------------------------------------------- */
typedef struct cgdir_ctx cgdir_ctx;          /* opaque; one device + one stream */

typedef struct {
    int    device;              /* CUDA device ordinal                          */
    void  *stream;              /* cudaStream_t to order all work on; NULL = the
                                   context creates (and later destroys) its own;
                                   cudaStreamLegacy (0x1) = the legacy default
                                   stream                                        */
    size_t mem_budget_bytes;    /* cap on device memory the context may hold;
                                   0 = no cap                                   */
} cgdir_config;

typedef struct {
    int         nx, ny, nz;
    int         dtype;          /* CGDIR_F32 / CGDIR_F16 / CGDIR_BF16, in HU    */
    int         where;          /* CGDIR_HOST or CGDIR_DEVICE                   */
    const void *data;           /* nz*ny*nx elements                            */
} cgdir_volume;

typedef struct {
    int                   nx, ny, nz;
    int                   where;   /* CGDIR_HOST or CGDIR_DEVICE                */
    const uint8_t *const *data;    /* host array of `count` pointers, each to
                                      nz*ny*nx uint8 (nonzero = inside)          */
    int                   count;   /* number of structures k, 0..8             */
} cgdir_masks;

typedef struct {
    int           levels;             /* pyramid levels, 1..8 (paper: 2)       */
    const int    *iters;              /* host, `levels` caps, coarse -> fine    */
    float         sigma_fluid;        /* Gaussian std (voxels) for du; 0 = off  */
    float         sigma_diff;         /* Gaussian std (voxels) for u;  0 = off  */
    const float  *lambda;             /* host, k weights >= 0 (paper ~1e-3);
                                         NULL = 1e-3 each                       */
    const int8_t *sign;               /* host, k signs +1/-1; 0 or NULL = decide
                                         from the static image (ROI mean vs the
                                         mean of a 2-voxel shell around it)     */
    unsigned      contour_level_mask; /* bit l: structure terms at level l
                                         (l = 0 coarsest); paper: finest only   */
    int           stop_mode;          /* CGDIR_STOP_*                           */
    double        eps;                /* stopping threshold, HU (paper 1e-4)    */
    double        spacing_mm[3];      /* voxel size at full resolution (x,y,z)  */
    double        margin_mm;          /* UROI margin (paper: 10 mm)             */
    float         intensity_offset;   /* HU -> CT number for the MIs (1000)     */
    int           compose_mode;       /* CGDIR_COMPOSE / CGDIR_ADDITIVE         */
    const float  *init_dvf;           /* NULL, or a full-resolution DVF that
                                         replaces the coarse levels (Sec. 4)    */
    int           init_dvf_where;     /* CGDIR_HOST or CGDIR_DEVICE             */
    int           storage_dtype;      /* type of the images at the finest level
                                         (the input resolution): CGDIR_F32,
                                         CGDIR_F16, CGDIR_BF16 (inputs converted
                                         at ingest, round to nearest even), or
                                         CGDIR_STORAGE_AUTO = the input type (F32
                                         if static and moving differ).  The
                                         coarser levels (1/7 of the pyramid's
                                         voxels) are restricted from it and kept
                                         in FP32: the box mean lowers the noise
                                         sqrt(8)-fold per level, so a 16-bit
                                         rounding there would weigh 2.8x, 8x, ...
                                         more.  All force, DVF and smoothing
                                         arithmetic is FP32 whatever the storage. */
} cgdir_params;

typedef struct {
    int           level;              /* 0 = coarsest                           */
    int           nx, ny, nz;         /* grid of this level                     */
    int           iters_run;          /* updates applied at this level          */
    int           stop_reason;        /* CGDIR_REASON_*                         */
    int           hist_len;           /* entries in rms_id (iters_run + 1, or 0) */
    const double *rms_id;             /* host, RMS-ID over the UROI after each
                                         update, rms_id[0] = before the first;
                                         owned by the context, valid until its
                                         next call or cgdir_destroy             */
} cgdir_level_stats;

/* ---- context ------------------------------------------------------------ */

/* Fill *p with the paper's defaults (Sec. 2.2): 2 levels with 100 / 50
   iterations, sigma 1 voxel for du and u, lambda 1e-3, automatic signs,
   contour terms at the finest level, WINDOW10 stopping with eps 1e-4,
   1.97 x 1.97 x 2.5 mm voxels, 10 mm UROI margin, offset 1000, composite
   update, no initial DVF. */
void cgdir_default_params(cgdir_params *p);

/* Create a context on cfg->device ordering its work on cfg->stream.
   *out receives the handle (NULL on failure).  Errors: EINVAL (bad device,
   NULL out/cfg), ECUDA.
   Kernel-choice overrides read from the environment at creation (for tests
   and measurement; the defaults need none of them):
     CGDIR_KERNELS=plain|fused   plain-load kernels everywhere / the one-pass
                                 TMA force and fused smoothing kernels
     CGDIR_GRAPHS=0              launch eagerly instead of replaying graphs
     CGDIR_SMOOTH=march|tile|split|fused, CGDIR_SMOOTH_ZCHUNK=n   smoothing variant
     CGDIR_FORCE_ZCHUNK=n, CGDIR_FORCE_WIDTH=1|2   force pass 2 z chunk / voxels
                                 per thread (default: 4 where nx % 4 == 0, else 2
                                 for even nx, else 1)
     CGDIR_COOP_MAX=n            levels below the finest with at most n voxels
                                 run as one cooperative launch
     CGDIR_SERVE_SCHEDULE=shared|alone|auto   schedule of submitted requests
                                 (default auto: the latency schedule of
                                 cgdir_register when no other request is
                                 running at submission, else the throughput one)
     CGDIR_SHARED_WIDE_CAP=n     z-march smoothing CTAs per SM in batched and
                                 shared served registrations (default 2; 0: no cap) */
int cgdir_create(cgdir_ctx **out, const cgdir_config *cfg);

/* Release every device buffer, cached graph and (if owned) stream of ctx.
   NULL is accepted. */
void cgdir_destroy(cgdir_ctx *ctx);

/* Static name of a status code. */
const char *cgdir_strerror(int status);

/* Message of the last failure on ctx (empty string if none). */
const char *cgdir_last_error(const cgdir_ctx *ctx);

/* Device bytes currently held by ctx (pyramid, fields, scratch). */
size_t cgdir_mem_in_use(const cgdir_ctx *ctx);

/* Wait for all work queued on ctx's stream.  Returns CGDIR_ETIMEDOUT if a
   kernel's bounded wait for its own asynchronous (TMA) loads ran out since
   the last check -- the kernel then wrote no output and returned -- and
   CGDIR_ECUDA if the stream reports an error.  The blocking entry points
   (cgdir_register, and cgdir_force / cgdir_iterate with stats) do this
   check themselves. */
int cgdir_sync(cgdir_ctx *ctx);

/* ---- whole registration (Algorithm A) ----------------------------------- */

/* Register moving_img onto static_img.  Both images and all masks must have
   the same nx, ny, nz; static_masks and moving_masks the same count k <= 8.
   The pyramid is built by factor-2 restriction (size ceil(n/2) per axis,
   2x2x2 box mean; masks by majority, ties inside).  Level l runs plain
   demons unless bit l of contour_level_mask is set, then up to iters[l]
   iterations of Algorithm A steps 1-6; between levels u is prolongated
   (cell-centred trilinear, x2).  The UROI of level l is the union of its
   static masks dilated by margin_mm with the level's spacing (whole volume
   when k == 0).
   dvf_out: [3][nz][ny][nx] float32 at full resolution, on host or device
   per dvf_where.  stats_out: host array of `levels` entries (may be NULL).
   Blocking: returns after the result is in dvf_out.
   Errors: EINVAL (shape/dtype/count mismatch, k > 8, levels outside 1..8,
   negative lambda, sigma outside [0, 2], NULL pointers), ENOMEM, ECUDA. */
int cgdir_register(cgdir_ctx *ctx, const cgdir_volume *static_img, const cgdir_volume *moving_img,
                   const cgdir_masks *static_masks, const cgdir_masks *moving_masks,
                   const cgdir_params *params, float *dvf_out, int dvf_where,
                   cgdir_level_stats *stats_out);

/* ---- many registrations at once (not in the paper: an execution mode) --- */

/* Register `count` (1..1024) independent cases in one call.  Arrays of
   `count` entries: statics, movings, params (each case its own parameters,
   shapes and mask counts); static_masks / moving_masks may be NULL (no masks
   for any case); dvf_outs[i] receives case i as cgdir_register would write
   it (dvf_where applies to all).  The device parts of all cases are one
   CUDA graph with a concurrent branch per case, so small cases share the GPU
   instead of running one after another.  stats_out: host array holding
   params[0].levels + ... + params[count-1].levels entries, case after case
   (may be NULL).  Results are bitwise those of cgdir_register per case.
   Blocking.  Errors as cgdir_register; EBUSY if a slot it needs is serving
   a submitted request. */
int cgdir_register_batch(cgdir_ctx *ctx, int count, const cgdir_volume *statics,
                         const cgdir_volume *movings, const cgdir_masks *static_masks,
                         const cgdir_masks *moving_masks, const cgdir_params *params,
                         float *const *dvf_outs, int dvf_where, cgdir_level_stats *stats_out);

/* ---- serving: asynchronous requests (not in the paper) ------------------
 * cgdir_submit queues one registration and returns at once with a ticket;
 * each request in flight has its own device buffers and CUDA stream (a
 * "slot"), so requests that arrive while others run overlap on the device.
 * At most cgdir_set_max_inflight(n) requests (default 8) are in flight; a
 * submit beyond that, or one whose new buffers would exceed the context's
 * mem_budget_bytes, returns EBUSY and queues nothing (retry after a
 * release).  Inputs must stay valid until the request completes; dvf_out
 * is written by the time cgdir_wait / cgdir_poll return CGDIR_OK (a
 * pageable host dvf_out is copied by that call, pinned or device memory by
 * the request's stream).  A request submitted while no other is running
 * takes the kernel schedule of cgdir_register (latency); one submitted
 * while others run takes the throughput schedule of cgdir_register_batch.
 * A result is the same, bit for bit, whether the request ran alone or among
 * others, on either schedule.  The context's stream is not used. */
int cgdir_set_max_inflight(cgdir_ctx *ctx, int n);            /* 1..256 */
int cgdir_submit(cgdir_ctx *ctx, const cgdir_volume *static_img, const cgdir_volume *moving_img,
                 const cgdir_masks *static_masks, const cgdir_masks *moving_masks,
                 const cgdir_params *params, float *dvf_out, int dvf_where, long long *ticket);
/* CGDIR_OK once the request has completed (dvf_out written), EBUSY while it
   runs, EINVAL for an unknown or released ticket, ETIMEDOUT / ECUDA if a
   kernel of the request failed. */
int cgdir_poll(cgdir_ctx *ctx, long long ticket);
/* Poll until completion or until timeout_ms (< 0: no limit) has passed:
   then ETIMEDOUT, and the request is still in flight. */
int cgdir_wait(cgdir_ctx *ctx, long long ticket, int timeout_ms);
/* Free the request's slot and fill stats_out (`levels` entries, may be
   NULL; its rms_id arrays stay valid until the slot is reused).  EBUSY if
   the request has not completed. */
int cgdir_release(cgdir_ctx *ctx, long long ticket, cgdir_level_stats *stats_out);
/* Stop a request early: its remaining kernels return at once (a request
   whose device part has not begun yet runs to the end).  Blocks until the
   slot is idle, then frees it; dvf_out then holds an unspecified partial
   result (a pageable host dvf_out is left untouched). */
int cgdir_cancel(cgdir_ctx *ctx, long long ticket);

/* ---- primitives of the iteration (device pointers, ctx's stream) -------- *
 * These expose each step of the hot path on caller-owned device buffers, so
 * that a caller can run its own loop and so that each step can be checked on
 * its own.  They are asynchronous on the context's stream unless a host
 * output is requested.  nx, ny, nz >= 1; images are float32 unless noted.   */

/* Pack k <= 8 uint8 masks (device pointers, nonzero = inside) into bits[n]:
   bit i of bits[v] = (masks[i][v] != 0).  masks is a HOST array of k device
   pointers. */
int cgdir_pack_masks(cgdir_ctx *ctx, const uint8_t *const *masks, int k, size_t n, uint8_t *bits);

/* Interpolation kernel (kernel 4, Algorithm A step 5): out(x) = f(x + u(x)). */
int cgdir_warp(cgdir_ctx *ctx, const float *f, const float *u, int nx, int ny, int nz, float *out);

/* Moving-vector step (kernels 2 + 3, Algorithm A step 1; Eq. 7 with
   beta = (T0 - I0~)^2 and n = grad I0~ / |grad I0~|): du = v n, unsmoothed,
   [3][N]; du = 0 where the FP32 gradient of I0~ is exactly zero.
   mbits / sbits: packed moving / static masks; sign, lambda: host arrays of
   k; contour = 0 drops the structure terms (plain demons).  uroi (may be
   NULL = whole volume) selects the voxels of the stopping metric; if
   stats_host != NULL it receives {sum over UROI of (I0~ - T0)^2, UROI voxel
   count, max |du|} (FP64, blocking).  warped (may be NULL) receives I0~. */
int cgdir_force(cgdir_ctx *ctx, const float *I0, const float *T0, const uint8_t *mbits,
                const uint8_t *sbits, const uint8_t *uroi, int k, const float *lambda,
                const int8_t *sign, float offset, int contour, const float *u,
                int nx, int ny, int nz, float *du, float *warped, double *stats_host);

/* Low-pass filter kernel (kernel 1): separable Gaussian, x then y then z,
   sigma in voxels (0 < sigma <= 2; radius ceil(3 sigma)), normalised taps,
   clamp-to-edge, applied to `ncomp` consecutive [N] components (1..3).
   sigma == 0 copies.  out must not alias in. */
int cgdir_smooth(cgdir_ctx *ctx, const float *in, int ncomp, float sigma, int nx, int ny, int nz,
                 float *out);

/* Composite update (Algorithm A step 3): out = du + u(x + du(x)) (mode
   CGDIR_COMPOSE) or u + du (CGDIR_ADDITIVE), then, if sigma > 0, the
   Gaussian of step 4.  out must not alias u or du. */
int cgdir_compose(cgdir_ctx *ctx, const float *u, const float *du, int mode, float sigma,
                  int nx, int ny, int nz, float *out);

/* Fluid smoothing and composite update (Algorithm A steps 2-3):
   out = G(du) + u(x + G(du)(x)) (mode CGDIR_COMPOSE) or u + G(du)
   (CGDIR_ADDITIVE), G the Gaussian of sigma voxels (0 <= sigma <= 2; 0 is
   no smoothing).  The kernels are the context's forced smoothing variant
   (CGDIR_SMOOTH at creation; under CGDIR_SMOOTH=fused one 3-D tile kernel
   for both steps), else chosen by size; every choice gives the same bits.
   Fields [3][nz][ny][nx] FP32 in device memory; out must not alias u or
   du.  Errors: EINVAL, ENOMEM, ECUDA. */
int cgdir_smooth_compose(cgdir_ctx *ctx, const float *du, const float *u, int mode, float sigma,
                         int nx, int ny, int nz, float *out);

/* One iteration, Algorithm A steps 1-4 (force, smooth du, compose, smooth u)
   from u_in to u_out (must not alias).  du_out (may be NULL) receives the
   smoothed du.  stats_host as in cgdir_force (the metric of u_in). */
int cgdir_iterate(cgdir_ctx *ctx, const float *I0, const float *T0, const uint8_t *mbits,
                  const uint8_t *sbits, const uint8_t *uroi, int k, const float *lambda,
                  const int8_t *sign, float offset, int contour, float sigma_fluid,
                  float sigma_diff, int compose_mode, const float *u_in, int nx, int ny, int nz,
                  float *u_out, float *du_out, double *stats_host);

/* Pyramid: factor-2 restriction of a float32 image (2x2x2 box mean; output
   (nx+1)/2 x (ny+1)/2 x (nz+1)/2, indices clamped for odd sizes). */
int cgdir_restrict_image(cgdir_ctx *ctx, const float *in, int nx, int ny, int nz, float *out);

/* Restriction of packed mask bits: per bit, inside if >= 4 of the 8 source
   voxels are inside. */
int cgdir_restrict_bits(cgdir_ctx *ctx, const uint8_t *in, int nx, int ny, int nz, uint8_t *out);

/* Prolongation of a DVF from the coarse grid (cx, cy, cz) to the fine grid
   (nx, ny, nz): u_f(x) = 2 u_c((x + 0.5)/2 - 0.5), trilinear, clamped. */
int cgdir_prolong(cgdir_ctx *ctx, const float *uc, int cx, int cy, int cz, int nx, int ny, int nz,
                  float *uf);

/* UROI map (Sec. 2.2 stopping criterion): out[v] = 1 if some voxel w with
   any of the low k bits of sbits set has sum_a ((v_a - w_a) spacing_a)^2 <=
   margin^2, else 0; all ones when k == 0.  spacing: host array of 3. */
int cgdir_uroi(cgdir_ctx *ctx, const uint8_t *sbits, int k, int nx, int ny, int nz,
               const double *spacing, double margin, uint8_t *out);

/* Automatic signs of M_i, N_i (Sec. 2.1): sign_host[i] = +1 if the mean of T0
   over structure i >= the mean over the voxels within Chebyshev distance 2
   of it and outside it, else -1 (+1 if either set is empty).  Blocking. */
int cgdir_auto_sign(cgdir_ctx *ctx, const float *T0, const uint8_t *sbits, int k, int nx, int ny,
                    int nz, int8_t *sign_host);

/* RMS-ID over the UROI (Sec. 2.2): *rms_host = sqrt(sum (I0~ - T0)^2 / |UROI|)
   with I0~ = I0(x + u(x)); 0 when the UROI is empty.  FP64 accumulation,
   deterministic order.  Blocking. */
int cgdir_rms_id(cgdir_ctx *ctx, const float *I0, const float *T0, const float *u,
                 const uint8_t *uroi, int nx, int ny, int nz, double *rms_host,
                 long long *count_host);

/* RMS-ID over the UROI, like cgdir_rms_id, for callers that cannot allocate
   device memory: hosts that own every byte of it through their own pool (a
   framework's caching allocator, a planning system with a fixed device
   budget) or loops where allocation is forbidden.  The paper has no
   counterpart; this is a service entry point of the library.
   It takes no context and allocates nothing: its scratch (per-CTA partial
   sums, a completion counter, the result) is a fixed array in the library's
   device memory, which every GPU that loads the library holds until the
   process exits.  Limit: nx*ny*nz <= 67,108,864 voxels; larger volumes are
   rejected with CGDIR_EINVAL.  Device pointers as in cgdir_rms_id (uroi may be
   NULL = whole volume); stream = cudaStream_t (NULL = legacy default stream).
   Sums are FP64 from each thread's first term on (fixed order within a
   block and across blocks).
   Blocking: *rms_host (and *count_host if not NULL) are written on return,
   after the call has synchronized `stream`.  So no call may be made while a
   stream of that device is capturing a CUDA graph.  The first call on a
   device (and the first after that device's current context changes, e.g.
   after cudaDeviceReset) does the set-up: it looks up the array's device
   address with the device current.  All calls share the one array: calls
   whose work overlaps on the GPU (two streams or threads at once) race and
   give undefined results.  Errors: EINVAL, ECUDA. */
int cgdir_rms_id_noalloc(const float *I0, const float *T0, const float *u, const uint8_t *uroi,
                         int nx, int ny, int nz, void *stream, double *rms_host,
                         long long *count_host);

/* ---- instrumentation (not part of the paper's method) ------------------ */

/* Number of CUDA kernels this library has launched in the process so far
   (each kernel launch counts once; memcpy/memset do not count). */
unsigned long long cgdir_launch_count(void);

/* Kernel classes for per-kernel timing. */
#define CGDIR_K_FORCE      0   /* warp + gradient + Eq. 7 (kernels 2, 3, 4)    */
#define CGDIR_K_SMOOTH_DU  1   /* Gaussian of du and, fused into it, the
                                  composite update (kernels 1 + 4, steps 2-3) */
#define CGDIR_K_COMPOSE    2   /* composite update when it runs on its own    */
#define CGDIR_K_SMOOTH_U   3   /* Gaussian of u (kernel 1, step 4); on the fused
                                  schedule with the next iteration's warp,
                                  which the FORCE class then lacks after the
                                  first iteration                             */
#define CGDIR_K_FINALIZE   4   /* RMS-ID reduction and stop test (kernel 5)  */
#define CGDIR_K_METRIC     5   /* warp-only metric pass after a level's cap  */
#define CGDIR_K_SETUP      6   /* pyramid, masks, UROI, signs, prolongation  */
#define CGDIR_K_LEVEL      7   /* a whole small level in one cooperative launch */
#define CGDIR_K_COUNT      8

typedef struct {
    int       kernel;     /* CGDIR_K_*                                       */
    int       level;      /* pyramid level (0 = coarsest)                    */
    long long launches;   /* launches timed                                  */
    double    total_ms;   /* sum of their CUDA-event durations               */
} cgdir_kernel_time;

/* Time the kernels of the classes in kernel_mask (bit CGDIR_K_*) during later
   cgdir_register calls on ctx, with a CUDA event pair on ctx's stream around
   each launch; 0 switches timing off.  Clears earlier totals. */
int cgdir_profile(cgdir_ctx *ctx, unsigned kernel_mask);

/* Restrict the timing switched on by cgdir_profile to the pyramid levels
   of level_mask (bit l = level l, 0 = coarsest); cgdir_profile selects all
   levels.  Each timed launch adds two event nodes to the graph, so timing
   only the levels of interest keeps the registration's own time close to
   the untimed one.  Clears earlier totals. */
int cgdir_profile_levels(cgdir_ctx *ctx, unsigned level_mask);

/* Copy up to `cap` accumulated (kernel, level) totals into out; returns the
   number of entries written (negative status on error). */
int cgdir_profile_read(const cgdir_ctx *ctx, cgdir_kernel_time *out, int cap);

/* Self-test of the device-side timeout path (not in the paper): one kernel
   waits, with a limit of limit_us microseconds (1..2000000), on a barrier
   that nothing completes; the wait runs out, the kernel records it in the
   context's error word and returns, and the call reports it as a kernel
   wait that ran out.  Returns CGDIR_ETIMEDOUT when the path works (the
   context stays usable); EINVAL for a bad limit; ECUDA. */
int cgdir_selftest_wait_timeout(cgdir_ctx *ctx, int limit_us);

/* ---- autotuner (not in the paper: an execution choice) --------------------
 * For each level shape of a pyramid it times, on synthetic data of that
 * shape shaped like a registration's, the candidate configurations of the
 * force stencil pass (four z-chunk lengths, four or two voxels per thread)
 * and of the smoothing with the composite update (steps 2-4 of an
 * iteration, timed behind a force step: the 64 x 16 TMA z-march with the
 * volume in 1 to 16 z chunks, the 32 x 16 one with 2, 4 and 8, 3-D
 * shared-memory tile, split xy + z kernels with the update in the z pass)
 * on ctx's stream and keeps the fastest, then times the fused schedule
 * against it.  Later registrations of those shapes use the choices:
 * cgdir_register, and a request submitted on an idle GPU, the fused
 * schedule where it won; batched registrations and requests submitted while
 * others run (they share the GPU, so throughput counts) the best per-step
 * schedule.  Only the kernels change: every choice gives the same bits.
 * Blocking. */
#define CGDIR_SMOOTH_MARCH 1
#define CGDIR_SMOOTH_TILE  2
#define CGDIR_SMOOTH_SPLIT 3
#define CGDIR_SMOOTH_FUSED 4   /* fused schedule: 3-D tiles of G(du) with the update and of G(u')
                                  with the next warp; the force runs its stencil pass only.
                                  smooth_ms / force_ms are then those kernels' times (the
                                  per-step alternative is kept but not reported; a loaded
                                  table that says FUSED picks the per-step kernels by size) */
#define CGDIR_SMOOTH_MARCH32 5 /* the 32 x 16 z-march where the 64 x 16 one would apply */
typedef struct {
    int   nx, ny, nz;           /* level shape                                   */
    int   contour;              /* structure terms on at this level               */
    int   storage_dtype;        /* CGDIR_F32 / F16 / BF16                          */
    int   smooth_variant;       /* CGDIR_SMOOTH_MARCH / _TILE / _SPLIT / _FUSED / _MARCH32 */
    int   smooth_zchunk;        /* z chunk of the z-march (0 = default / n/a)       */
    int   force_zchunk;         /* z chunk of the force stencil pass                */
    float smooth_ms, force_ms;  /* best times: steps 2-4 of one iteration; force   */
    float default_smooth_ms, default_force_ms;   /* the untuned choice's times     */
    int   force_width;          /* voxels per thread of the stencil pass: 0 = the
                                   widest the shape allows (4 where nx % 4 == 0), 2 */
} cgdir_tuning;

/* Tune every level of a `levels`-level pyramid whose finest level is
   nx x ny x nz, with k structures, structure terms at the levels of
   contour_level_mask, image storage storage_dtype (CGDIR_F32/F16/BF16; as in
   cgdir_params, the coarser levels are tuned for their FP32 images) and
   Gaussian sigma (voxels).  Errors: EINVAL, ENOMEM, ECUDA. */
int cgdir_autotune(cgdir_ctx *ctx, int nx, int ny, int nz, int k, int levels, unsigned contour_level_mask,
                   int storage_dtype, float sigma);
/* on != 0: registrations tune each level shape they have not seen before
   they run (a few milliseconds per new shape). */
int cgdir_set_autotune(cgdir_ctx *ctx, int on);
/* Copy up to cap tuned shapes into out; returns how many there are. */
int cgdir_tuning_read(const cgdir_ctx *ctx, cgdir_tuning *out, int cap);
/* Install n tuned shapes (as cgdir_tuning_read returns them, e.g. saved by
   an earlier process), replacing the context's entries for those shapes;
   later registrations use them without timing anything.  Only the kernel
   choices are used (results do not depend on them); the times are kept for
   reporting.  Errors: EINVAL (bad shape, variant or z chunk; nothing is
   installed then). */
int cgdir_tuning_load(cgdir_ctx *ctx, const cgdir_tuning *in, int n);

#ifdef __cplusplus
}
#endif
#endif /* CGDIR_H */

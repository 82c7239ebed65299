/*
 * fpm.h -- C ABI of the B300 (sm_103a) Fourier ptychographic microscopy (FPM)
 * tile-reconstruction library.
 *
 * What it computes (the paper, "Parallel Fourier Ptychography reconstruction"):
 *   the sensor field of view is cut into overlapping square sub-regions (tiles,
 *   Sec. 3.1, Fig. 5) that are reconstructed independently; each tile sees every
 *   LED at its own illumination angle (Sec. 2.2, Fig. 3/4) and has its own
 *   defocus (Sec. 2.2).  A tile's high-resolution (HR) spectrum is recovered by
 *   alternating projection (Sec. 2.1, Fig. 2): for each LED in the update order
 *   (Sec. 3.2, Fig. 6) the shifted sub-aperture of the spectrum is cut out and
 *   multiplied by the pupil, inverse transformed to the low-resolution (LR)
 *   grid, given the measured amplitude, transformed back, and written into the
 *   spectrum; with FPM_EPRY the pupil is corrected too (embedded pupil recovery,
 *   Ou, Zheng and Yang, Opt. Express 22(5):4960, 2014).  LEDs whose sub-apertures
 *   do not share a spectrum pixel are updated concurrently in "waves" (the
 *   spectrum-domain parallelism of Sec. 3.2).
 *
 * Conventions used by every entry point:
 *   - Return value: FPM_OK (0) or a negative FPM_E* status.  On failure nothing
 *     the caller owns has been modified and fpm_last_error() (thread-local)
 *     describes the cause.  No C++ exception crosses the ABI.
 *   - Complex numbers are complex64: interleaved (re, im) float32 pairs.
 *   - Spectra are "centred": element (y, x) of an N x N array holds spatial
 *     frequency (y - N/2, x - N/2) Fourier pixels; the DC term sits at (N/2, N/2).
 *     Pupils are m x m, centred the same way.  All 2-D arrays are row-major.
 *   - Streams are passed as `void *` holding a cudaStream_t (NULL = the legacy
 *     default stream).  Calls that take a stream only enqueue work on it; the
 *     caller synchronises.
 *   - A plan is not thread-safe: one thread at a time may use it.  A server is
 *     thread-safe.
 *   - Device memory the library allocates belongs to the plan (or server) and is
 *     freed by fpm_plan_destroy (fpm_server_destroy).
 *   - Environment overrides, read when a plan is created and when its device
 *     state is made (its first load): FPM_UPDATE_THREADS = "T" or "TxC" picks the
 *     update-kernel variant of the plan's tile side with T threads per CTA (and C
 *     CTAs per cluster) instead of the default, which is the first that fits;
 *     FPM_WAVE_BRANCHES = B (1..8) splits the tiles into B parallel graph branches
 *     for graph replays of FPM_RUN_WAVES.  fpm_autotune replaces both with its
 *     measured choice.
 */
#ifndef FPM_H_
#define FPM_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FPM_API __attribute__((visibility("default")))
#else
#define FPM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define FPM_OK         0
#define FPM_EINVAL    (-1)  /* bad argument or geometry                          */
#define FPM_ENOMEM    (-2)  /* host or device allocation failed                  */
#define FPM_EBUDGET   (-3)  /* the job can never fit the server's HBM budget     */
#define FPM_ETIMEOUT  (-4)  /* a bounded device wait ran out (kernel returned)   */
#define FPM_ECUDA     (-5)  /* a CUDA runtime/driver call failed                 */
#define FPM_EBUSY     (-6)  /* the object is in use (e.g. a plan owned by a job) */
#define FPM_ESTATE    (-7)  /* call out of order (e.g. reconstruct before load)  */

/* ---- LED update routine (Sec. 3.2, Fig. 6) --------------------------------- */
#define FPM_ORDER_CENTER_OUT 0  /* by distance of the LED from the array centre */
#define FPM_ORDER_RASTER     1  /* LED index order                              */

/* ---- plan flags ------------------------------------------------------------ */
#define FPM_EPRY  1u  /* correct the pupil too (embedded pupil recovery)          */
#define FPM_SEQUENTIAL 2u /* strict sequential order: every update sees the pupil
                             corrected by all earlier ones (each wave holds one LED
                             per tile); default: wave-synchronous, LEDs whose
                             sub-apertures share no spectrum pixel in one wave   */
#define FPM_EPRY_UNMASKED 4u /* with FPM_EPRY: the pupil correction is not confined
                             to the circular support -- corrections, both
                             normalisers and the wave footprints cover the whole
                             m x m box (the initial pupil is still the circle);
                             default: everything confined to the support disc     */

/* ---- image element types --------------------------------------------------- */
#define FPM_U16 0     /* camera counts (e.g. 12-bit)                             */
#define FPM_F32 1     /* intensities as float32                                  */

/* ---- execution modes of fpm_reconstruct ------------------------------------ */
#define FPM_RUN_PLAIN      0  /* one tile at a time, one LED per launch          */
#define FPM_RUN_WAVES      1  /* every tile's next wave in one launch            */
#define FPM_RUN_PERSISTENT 2  /* one persistent kernel over a device work queue  */
#define FPM_RUN_AUTO       3  /* the path fpm_autotune chose (persistent if none) */
#define FPM_RUN_GRAPH      0x100 /* OR-able: replay the launches as a CUDA graph */
#define FPM_RUN_TIMED      0x200 /* OR-able with FPM_RUN_WAVES: time each update
                                    launch with CUDA events (see fpm_get_stats)  */
#define FPM_RUN_FAULT_TEST 0x400 /* OR-able with FPM_RUN_PERSISTENT, for tests of
                                    the failure path only: every dependency wait
                                    of the persistent kernel looks at a flag that
                                    nothing sets and gives up after 50 ms; the
                                    kernel ends and fpm_get_stats / the getters
                                    report FPM_ETIMEOUT.  The state is then
                                    undefined (reload before further use).    */

typedef struct fpm_plan fpm_plan;
typedef struct fpm_server fpm_server;
typedef int64_t fpm_job;

/*
 * Problem statement of one job (Sec. 2.2, Sec. 3.1, Sec. 4).  Every pointer is
 * read during fpm_plan_create only and copied; the caller keeps ownership.
 */
typedef struct {
  int32_t sensor_h, sensor_w;   /* LR sensor size in pixels                          */
  int32_t tile;                 /* LR tile side m: 64, 128, 192 or 256                */
  int32_t overlap;              /* LR overlap between neighbouring tiles (pixels)     */
  int32_t tiles_y, tiles_x;     /* tile grid, centred on the sensor                   */
  int32_t upsample;             /* N = upsample * m (HR side); 2..8                    */
  double wavelength_um;         /* illumination wavelength                            */
  double na;                    /* objective numerical aperture                        */
  double pixel_um;              /* LR pixel size in the sample plane                   */
  int32_t n_leds;               /* number of LEDs (>= 1)                               */
  const double *led_xy_um;      /* [n_leds][2] LED (x, y) in um, optical axis at 0     */
  double led_height_um;         /* distance between LED array and sample               */
  const double *defocus_um;     /* [tiles_y * tiles_x] per-tile defocus, or NULL = 0   */
  int32_t order;                /* FPM_ORDER_*                                         */
  int32_t iters;                /* iteration loops the schedule is built for (>= 1)    */
  uint32_t flags;               /* FPM_EPRY | FPM_SEQUENTIAL, or 0                      */
  int32_t tile_first;           /* tile subset (Sec. 5: sub-regions sent to different
                                   GPUs): the plan holds tiles [tile_first, tile_first
                                   + tile_count) of the grid in row-major order, with
                                   the geometry they have in the whole grid; both 0 =
                                   the whole grid.  Tile t of such a plan is grid tile
                                   tile_first + t.  fpm_stitch needs the whole grid.  */
  int32_t tile_count;
} fpm_plan_desc;

/* Sizes of a plan, for allocating the arrays the getters fill. */
typedef struct {
  int32_t m, n;                 /* LR tile side, HR side                               */
  int32_t n_tiles, n_leds, iters;
  int32_t support_px;           /* pixels where updates act: the circular pupil support
                                   (A), m * m with FPM_EPRY_UNMASKED                   */
  int32_t support_rows;         /* rows of that region (R)                             */
  int32_t max_waves;            /* largest wave count over the tiles                   */
  int32_t max_wave_width;       /* largest number of LEDs in one wave of one tile      */
  int64_t total_waves;          /* sum over tiles of their wave counts                 */
  int64_t device_bytes;         /* device memory of the state fpm_load_tiles allocates
                                   (spectra, pupils and initial pupils, corrections),
                                   tile images apart                                    */
  int32_t cluster;              /* CTAs that share one update (1, 2 or 4)              */
  int32_t threads;              /* threads per CTA of the update kernel                */
  int64_t image_elems;          /* elements of the tile images fpm_load_tiles keeps
                                   (n_tiles * n_leds * m * m, each of the stack's type) */
  int32_t hr_overlap;           /* lines neighbouring tile objects share: overlap * (N/m) */
  int32_t fov_h, fov_w;         /* size of fpm_stitch's image: N + (tiles - 1)(N - hr_overlap) */
  int32_t tile_first;           /* grid index of the plan's tile 0 (0 for the whole grid) */
  int32_t band;                 /* 1: the support lies in box positions [3 m/16, 13 m/16) in
                                   both directions (m = 128, 256), so the update runs with
                                   band-pruned radix-16 passes; 0: the general passes */
} fpm_plan_info;

/*
 * fpm_plan_create -- validate a job and compute everything that does not
 * depend on the data (host only, FP64; no CUDA call is made):
 *   - tile origins of the centred grid, stride tile - overlap (Sec. 3.1);
 *   - per tile and LED the direction cosines of the line from the tile centre
 *     to the LED and the integer sub-aperture shift
 *     s = round_half_away(cosine / (wavelength * df)), df = 1/(m * pixel) (Sec. 2.2);
 *   - the LED order (Sec. 3.2) and, per tile, the wave of every update in the
 *     sequence of `iters` iteration loops: wave(j) = 0 if no earlier update's
 *     support disc shares an HR pixel with update j's, else 1 + the largest wave
 *     of those that do (Sec. 3.2: regions that do not affect each other are
 *     updated in parallel, across iteration loops);
 *   - per tile the initial pupil: circular support |f| <= NA/wavelength times
 *     exp(i 2 pi z (sqrt(1/lambda^2 - |f|^2) - 1/lambda)) (Sec. 2.1, Sec. 2.2).
 * Fails with FPM_EINVAL when a size is out of range, the grid does not fit the
 * sensor, the support is too large for the tile, or a sub-aperture box would
 * leave the N x N spectrum.
 * On success *out owns a new plan (free it with fpm_plan_destroy).
 */
FPM_API int fpm_plan_create(const fpm_plan_desc *desc, fpm_plan **out);

/* fpm_plan_destroy -- free a plan and its device memory (NULL is allowed).
 * Synchronises the device first.  FPM_EBUSY if a server job still uses it. */
FPM_API int fpm_plan_destroy(fpm_plan *plan);

/* fpm_plan_get_info -- fill *info (host only). */
FPM_API int fpm_plan_get_info(const fpm_plan *plan, fpm_plan_info *info);

/*
 * fpm_get_schedule -- copy the plan's schedule (host only).  Any pointer may be
 * NULL to skip that array.
 *   order   [n_leds]                    LED index visited at each position
 *   shifts  [n_tiles][n_leds][2]        (sy, sx) per tile and LED index
 *   waves   [n_tiles][iters * n_leds]   wave of each update of the sequence
 *   origins [n_tiles][2]                (y0, x0) tile origin on the sensor
 */
FPM_API int fpm_get_schedule(const fpm_plan *plan, int32_t *order, int32_t *shifts,
                     int32_t *waves, int32_t *origins);

/*
 * fpm_load_tiles -- attach the LR image stack and build the initial state.
 *   stack      [n_leds][sensor_h][sensor_w] images, element type `dtype`,
 *              element (l, y, x) at stack[l * stride_led + y * stride_row + x]
 *              (strides in elements; rows and LED planes must start 16-byte
 *              aligned).  Image l is the one taken with LED index l.
 *   on_device  0: `stack` is host memory; it is copied to a device staging
 *              buffer that is released once the tiles are extracted.  1:
 *              `stack` is device memory, read in place by this call's
 *              stream-ordered work; the plan keeps no reference to it.
 *   counts_per_unit  measured intensity = element / counts_per_unit (> 0).
 * Every tile's m x m window of every image is copied into device memory the
 * plan owns (image_elems elements of the stack's type, see fpm_plan_info),
 * column by column, in the order the update kernel's column transform reads
 * it.  Then, per tile, the initial spectrum is the spectrum of the upsampled
 * centre image: (N/m)^2 * zero-pad_N(centred DFT_m(sqrt(I_first))), I_first
 * being the tile's image of the first LED of the order, and the pupil is reset
 * to the initial pupil.  Allocates the plan's device state on first use
 * (FPM_ENOMEM on failure); loading images of another type reallocates the
 * tile images.
 */
FPM_API int fpm_load_tiles(fpm_plan *plan, const void *stack, int32_t dtype, int32_t on_device,
                   int64_t stride_led, int64_t stride_row, float counts_per_unit,
                   void *stream);

/*
 * fpm_reconstruct -- run `iters` (1..plan iters) iteration loops of the per-LED
 * update on every tile, continuing from the current state.  Per update, for
 * the box centred at c + s of the centred spectrum O (c = N/2):
 *   Phi  = O_box * P;  phi = (m/N)^2 IDFT_m(Phi);  phi' = sqrt(I) phi/|phi|
 *   (sqrt(I) where phi = 0);  Phi' = (N/m)^2 DFT_m(phi');  D = Phi' - Phi;
 *   O_box += conj(P) D / max|P|^2;  with FPM_EPRY the pupil gains
 *   support * conj(O_box_old) D / max|O_box_old|^2 (0 if that maximum is 0).
 * Maxima run over the pupil support.  Updates of one wave use the pupil as it
 * was when the wave started; their pupil corrections are added in sequence
 * order when the wave ends.  `mode` is FPM_RUN_PLAIN, FPM_RUN_WAVES or
 * FPM_RUN_PERSISTENT, optionally | FPM_RUN_GRAPH (and, with FPM_RUN_WAVES,
 * | FPM_RUN_TIMED); all modes give the same result.  FPM_ESTATE before
 * fpm_load_tiles.  The call only enqueues work: a persistent run whose bounded
 * device wait gave up is reported as FPM_ETIMEOUT by the next fpm_get_stats,
 * fpm_get_spectrum or fpm_get_pupil (the state is then undefined).
 */
FPM_API int fpm_reconstruct(fpm_plan *plan, int32_t iters, int32_t mode, void *stream);

/*
 * fpm_reconstruct_batch -- run `iters[i]` loops of each of `n` loaded plans
 * together (tiles of different sizes from different jobs; Sec. 3.1's
 * independent sub-regions).  `mode` FPM_RUN_PERSISTENT: one persistent launch
 * whose device work queue holds every plan's updates (every plan loaded with
 * the same image type).  FPM_RUN_WAVES: every plan's wave steps as an
 * independent branch forked from and joined back into `stream` (split further
 * into the plan's tile branches, see fpm_autotune).  Either optionally |
 * FPM_RUN_GRAPH (one graph per distinct batch, cached).  Each plan ends
 * exactly as fpm_reconstruct(plan, iters[i]) leaves it.  Errors as
 * fpm_reconstruct; a device-wait timeout is reported by each plan's
 * fpm_get_stats.
 */
FPM_API int fpm_reconstruct_batch(fpm_plan *const *plans, const int32_t *iters, int32_t n, int32_t mode,
                                  void *stream);

/*
 * fpm_get_spectrum / fpm_get_pupil -- copy tile `tile`'s current N x N spectrum
 * (m x m pupil), centred complex64, to `dst` (host memory if on_device == 0,
 * device memory otherwise).  Stream-ordered; for host `dst` the call returns
 * after the copy completed.
 */
FPM_API int fpm_get_spectrum(fpm_plan *plan, int32_t tile, void *dst, int32_t on_device, void *stream);

/*
 * fpm_get_spectra -- every tile's spectrum, [n_tiles][N][N] centred complex64,
 * copied to `dst` (host memory if on_device == 0, device memory otherwise) by
 * one copy enqueued on `stream`; the call does not wait for it, so with
 * page-locked host memory the copy overlaps other work and the caller
 * synchronises the stream before reading.  A bounded device wait that gave up
 * in the last persistent run is reported by fpm_get_stats.  FPM_ESTATE before
 * fpm_load_tiles.
 */
FPM_API int fpm_get_spectra(fpm_plan *plan, void *dst, int32_t on_device, void *stream);
FPM_API int fpm_get_pupil(fpm_plan *plan, int32_t tile, void *dst, int32_t on_device, void *stream);

/*
 * fpm_set_state -- overwrite tile `tile`'s spectrum (N x N) and/or pupil (m x m)
 * from host memory (either pointer may be NULL), e.g. to resume from a
 * checkpoint taken with the getters.  FPM_ESTATE before fpm_load_tiles.
 */
FPM_API int fpm_set_state(fpm_plan *plan, int32_t tile, const void *spectrum, const void *pupil,
                  void *stream);

/* Counters of the last calls on a plan (see fpm_get_stats). */
typedef struct {
  int64_t load_launches;    /* kernels enqueued by the last fpm_load_tiles             */
  int64_t run_launches;     /* kernels enqueued by the last fpm_reconstruct (a graph
                               replay counts the kernel nodes it runs)                 */
  int64_t update_launches;  /* fused-update launches of the last FPM_RUN_TIMED run     */
  int64_t updates;          /* LED updates those launches performed                    */
  double update_ms;         /* summed device time of those launches, milliseconds      */
  int32_t device_error;     /* 0, or FPM_ETIMEOUT if a bounded device wait of the last
                               persistent run gave up                                   */
  int32_t persistent_clusters; /* clusters of the last persistent launch               */
  int32_t run_threads;      /* threads per CTA of the update kernel the last
                               fpm_reconstruct ran (a graph replay: the variant it was
                               captured with; persistent: the persistent kernel's)     */
  int32_t online_launched;  /* wave steps the current or last online ingestion launched */
  int32_t online_steps;     /* wave steps of its schedule                               */
  int32_t run_cluster;      /* CTAs per cluster of that update kernel                   */
  double merge_ms;          /* device time between the end of each timed update launch
                               and the next launch's start (the wave's pupil merge)     */
  int32_t run_lanes;        /* lanes per 1-D transform (threads per transform) of that
                               update kernel                                           */
  int32_t pad0;
} fpm_stats;

/* fpm_get_stats -- fill *out.  Synchronises the device; update_ms is 0 when no
 * timed run happened.  Returns FPM_ETIMEOUT (with *out filled) when the last
 * persistent run's device wait gave up. */
FPM_API int fpm_get_stats(fpm_plan *plan, fpm_stats *out);

/* One candidate execution path and its measured time (fpm_autotune). */
typedef struct {
  int32_t mode;      /* FPM_RUN_WAVES or FPM_RUN_PERSISTENT                      */
  int32_t threads;   /* threads per CTA of the update kernel                     */
  int32_t cluster;   /* CTAs per update                                          */
  int32_t branches;  /* wave launches: parallel graph branches over tile groups  */
  double ms;         /* device time of `iters` loops on the plan's data          */
  int32_t lanes;     /* lanes per 1-D transform (threads per transform)          */
  int32_t radix_a;   /* the transform's split m = radix_a * radix_b: the radices */
  int32_t radix_b;   /*   of its two register passes                             */
  int32_t pad0;
} fpm_tune_entry;

/* Most candidates fpm_autotune times; an `entries` array this long receives them all. */
#define FPM_TUNE_MAX_ENTRIES 64

/*
 * fpm_autotune -- time every execution path that fits the plan's tile side
 * (wave-by-wave launches with each update-kernel variant -- threads per CTA,
 * CTAs per cluster and per SM -- each also with the tiles split into 2, 4
 * and 8 groups whose wave steps run as parallel graph branches; and the persistent
 * kernel) on `iters` loops of the plan's own
 * loaded data, each replayed as a CUDA graph after a warm-up, and keep the
 * fastest for FPM_RUN_AUTO and for FPM_RUN_WAVES.  The plan's spectra and pupils
 * are saved first and restored afterwards.  entries (may be NULL) receives up
 * to max_entries results, *n_entries their count, *best the chosen index
 * (which may lie beyond max_entries when that is below FPM_TUNE_MAX_ENTRIES).
 * Synchronises the device.  FPM_ESTATE before fpm_load_tiles.
 */
FPM_API int fpm_autotune(fpm_plan *plan, int32_t iters, void *stream, fpm_tune_entry *entries, int32_t max_entries,
                         int32_t *n_entries, int32_t *best);

/* fpm_initial_pupil -- the plan's initial pupil of `tile` (host memory,
 * m x m centred complex64; host only, no CUDA call). */
FPM_API int fpm_initial_pupil(const fpm_plan *plan, int32_t tile, void *dst);

/*
 * fpm_simulate -- forward model (Sec. 2.1, Fig. 1) on the device, to make
 * synthetic data: for every tile t and LED l,
 *   I[t][l] = |(m/N)^2 IDFT_m(O_t[box(c + s_tl)] * P_t)|^2,  O_t = centred DFT_N(o_t),
 * with P_t the plan's initial pupil.  objects: device [n_tiles][N][N] complex64
 * HR objects o_t; out: device [n_tiles][n_leds][m][m] float32.  Allocates and
 * frees its own temporaries; returns after the work completed.
 */
FPM_API int fpm_simulate(fpm_plan *plan, const void *objects, float *out, void *stream);

/* ---- serving: continuous batching of many jobs ---------------------------- */

/* fpm_server_create -- start a server (one worker thread) that runs the jobs
 * given to it on the current device, admitting them while their device memory
 * fits `hbm_budget_bytes`.  */
FPM_API int fpm_server_create(size_t hbm_budget_bytes, fpm_server **out);

/*
 * fpm_submit -- queue `iters` (1..plan iters) loops of a plan as a job
 * (non-blocking).  Either `stack` is NULL and the plan is already loaded
 * (fpm_load_tiles), or `stack` and the following arguments describe its images
 * exactly as fpm_load_tiles takes them and the server loads them when it admits
 * the job; host memory given this way must stay valid and unchanged until the
 * job is DONE or FAILED.  The job is charged the plan's device state plus the
 * copied stack; FPM_EBUDGET if that alone exceeds the budget.  Jobs are
 * admitted first come first served while the admitted jobs fit the budget; a
 * job gives its charge back when it finishes (its spectra and pupils stay on
 * the device until the caller destroys the plan).  The plan belongs to the
 * server (FPM_EBUSY for other calls on it) until the job is DONE or FAILED.
 * The server runs the admitted jobs' wave steps together in rounds of one
 * persistent launch each, so jobs that arrive while others run join at the
 * next round; each job computes what fpm_reconstruct(plan, iters) computes.
 * FPM_EINVAL for a plan whose update region the persistent kernel cannot hold
 * (FPM_EPRY_UNMASKED at m = 256: run it with fpm_reconstruct instead).
 */
FPM_API int fpm_submit(fpm_server *server, fpm_plan *plan, int32_t iters, const void *stack, int32_t dtype,
                       int32_t on_device, int64_t stride_led, int64_t stride_row, float counts_per_unit,
                       fpm_job *out);

#define FPM_JOB_QUEUED  0
#define FPM_JOB_RUNNING 1
#define FPM_JOB_DONE    2
#define FPM_JOB_FAILED  3

/* fpm_poll -- current state of a job (FPM_JOB_*), and optionally its submit ->
 * admit and submit -> done times in seconds (0 while unknown).  */
FPM_API int fpm_poll(fpm_server *server, fpm_job job, int32_t *state, double *wait_s, double *latency_s);

/* fpm_server_destroy -- let admitted jobs finish, cancel (FAILED) jobs not yet
 * admitted, stop the worker and free the server.  Plans are given back. */
FPM_API int fpm_server_destroy(fpm_server *server);

/*
 * fpm_update_tile_static -- one LED update of one tile, allocating no device
 * memory.  The paper has no counterpart: it exists for callers that cannot
 * call cudaMalloc (a host whose device memory belongs to its own pool, a
 * plug-in that may not allocate after start-up, or a real-time acquisition
 * loop that an allocation and its implicit synchronisation would stall).
 *   spectrum  device, n x n centred complex64, updated in place
 *   pupil     device, m x m centred complex64 (zero outside the circular
 *             support |f| <= na/wavelength), corrected in place if epry != 0
 *   image     device, m x m float32 measured intensity of this LED, model units
 *   shift_y, shift_x  the LED's sub-aperture shift in Fourier pixels (as
 *             fpm_get_schedule reports it)
 *   m in {64, 128, 192, 256}; n = 2..8 times m.
 * It computes exactly what fpm_reconstruct computes for a wave holding this one
 * LED: the max |P|^2 normaliser of the current pupil, the spectrum update and,
 * with epry, the pupil correction added.  Every temporary (the correction,
 * the tables and the image rearranged for the kernel) lives in a fixed
 * 1 MiB array of static device memory that each device loading the library
 * holds until the process exits; sizes needing more are rejected with
 * FPM_EINVAL.  All calls on a device share that array, so calls that overlap
 * on the GPU (other streams, unordered host threads) race; calls on one
 * stream are ordered.  Every pointer must be device memory of the current
 * device (memory of another GPU, or host memory, gives FPM_EINVAL); the
 * caller must pass tensors of exactly the stated sizes, which the C call
 * cannot check.  The first call on each device (and the first after the
 * device's context is re-created, e.g. by cudaDeviceReset) looks up the
 * array's address with cudaGetSymbolAddress and sets the kernels'
 * shared-memory limit, so make it before any timing-critical loop and before
 * any stream capture.  Stream-ordered; the caller synchronises.
 */
FPM_API int fpm_update_tile_static(void *spectrum, int32_t n, void *pupil, int32_t m, const float *image,
                                   int32_t shift_y, int32_t shift_x, double wavelength_um, double na,
                                   double pixel_um, int32_t epry, void *stream);

/*
 * fpm_fp32_peak -- measured FP32 throughput of the current device, the
 * denominator of the update kernel's roofline (its bound is FP32 arithmetic).
 * Times chains of fused multiply-adds that keep every FP32 lane busy (eight
 * independent chains per thread, 2048 threads per SM) at the clocks the device
 * runs at, and writes the best of three timed launches, in TFLOP/s (2 flop per
 * FMA), to *tflops.  Takes ~10 ms and 1 KB of device memory; synchronises the
 * stream.  FPM_ECUDA on a CUDA failure.
 */
FPM_API int fpm_fp32_peak(double *tflops, void *stream);

/*
 * Online reconstruction (Sec. 3.4, Fig. 7(a)): images are handed over one at a
 * time while the sample is still being illuminated, and the updates that have
 * all their images start at once, overlapping the acquisition.
 *
 * fpm_online_begin -- start ingesting `iters` (1..plan iters) loops' worth of
 *   images of type dtype (FPM_U16 / FPM_F32) with intensity = element /
 *   counts_per_unit.  Allocates the plan's device state and tile images as
 *   fpm_load_tiles does, plus four staging images; the plan's previous state is
 *   no longer readable until fpm_online_finish.  The wave steps that the last
 *   image of an ingestion in LED order releases (most of them: waves span
 *   loops) are captured here as one graph with the tiles in parallel branches,
 *   launched when that image arrives.
 * fpm_online_push -- the sensor image taken with LED index `led`: sensor_h
 *   rows of sensor_w elements, rows stride_row elements apart.  Host memory
 *   (on_device 0) is copied on the plan's own copy stream; use page-locked
 *   memory for the copy to overlap the running updates, and keep the buffer
 *   unchanged until the work enqueued on `stream` by this call has completed.
 *   Device memory is read stream-ordered on `stream`.  Its tile windows are
 *   gathered, the initial guess is built when the order's first LED arrives,
 *   and every wave step whose LEDs have all arrived is launched on `stream`.
 *   Any order is accepted; in the LED order the first loop runs while the
 *   images arrive.  FPM_EINVAL for an LED out of range or pushed twice.
 * fpm_online_finish -- after all n_leds pushes: launch the remaining wave
 *   steps; the plan then holds exactly the state fpm_load_tiles followed by
 *   fpm_reconstruct(iters, FPM_RUN_WAVES) gives on the same images
 *   (bit-identical).  FPM_ESTATE if images are missing.
 * All three are stream-ordered; FPM_ESTATE when called out of sequence.
 */
FPM_API int fpm_online_begin(fpm_plan *plan, int32_t iters, int32_t dtype, float counts_per_unit, void *stream);
FPM_API int fpm_online_push(fpm_plan *plan, int32_t led, const void *image, int32_t on_device, int64_t stride_row,
                            void *stream);
FPM_API int fpm_online_finish(fpm_plan *plan, void *stream);

/*
 * fpm_get_object -- the tile's HR complex object o = IDFT_N(ifftshift(O)) with
 * the 1/N^2 factor, O its current centred spectrum: N x N complex64,
 * row-major, written to dst (device memory if on_device, else host memory and
 * the call synchronises).  Computed on the device from the spectrum (line FFTs
 * along rows and columns).  FPM_ESTATE before fpm_load_tiles; FPM_ETIMEOUT (host
 * copies) if the last persistent run's bounded wait gave up.
 */
FPM_API int fpm_get_object(fpm_plan *plan, int32_t tile, void *dst, int32_t on_device, void *stream);

/*
 * fpm_stitch -- the whole field of view as one HR complex image (Eq. 1,
 * Sec. 3.1): fov_h x fov_w complex64, row-major (sizes in fpm_plan_info),
 * written to dst (device memory if on_device, else host memory and the call
 * synchronises).  Every tile's object (fpm_get_object) is placed at
 * (i, j) * (N - hr_overlap); the tiles of each grid column are stitched top
 * to bottom, then the columns left to right, each pair as Eq. 1: lines before
 * r - hr_overlap/2 (integer division) of the running image are kept, the rest
 * come from the next image times mu1/mu2.  Reading: mu1 and mu2 are the complex
 * means of the two images over the hr_overlap lines both cover; a zero mu2, or
 * hr_overlap 0, gives weight 1.  Device temporaries: n_tiles * N^2 * 8 bytes of
 * objects (plus the image itself for a host dst), kept with the plan for later
 * calls and freed by fpm_plan_destroy.  FPM_EINVAL if hr_overlap > N/2;
 * FPM_ENOMEM; FPM_ESTATE before fpm_load_tiles.
 */
FPM_API int fpm_stitch(fpm_plan *plan, void *dst, int32_t on_device, void *stream);

/* fpm_last_error -- text of the calling thread's last failure ("" if none). */
FPM_API const char *fpm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FPM_H_ */

/*
 * hdi.h -- C ABI of libhdi: homogeneous diffusion inpainting and its data
 * optimisation on one NVIDIA B300 (sm_103a).
 *
 * Method: Kaemper, Chizhov, Weickert, "Efficient Parallel Data Optimization
 * for Homogeneous Diffusion Inpainting of 4K Images" (arXiv 2401.06747).
 *
 * Conventions shared by every call
 *  - Images are planar: channel c, row y, column x lives at
 *      data[c * channel_stride + y * row_stride + x]   (strides in ELEMENTS).
 *  - Masks are uint8 (0 or 1), one per pixel, shared by all channels
 *    (Sec. 2.1: colour channels are inpainted with the same matrix).
 *  - `location` says whether a buffer is device memory of the context's GPU
 *    (HDI_DEVICE) or host memory (HDI_HOST; pinned or pageable). Host
 *    buffers are staged through the context's workspace with cudaMemcpyAsync.
 *  - The caller owns every buffer it passes. The library owns only its
 *    context workspace (grown on demand, released by hdi_destroy).
 *  - Every call is stream-ordered on the context's stream and returns after
 *    the work has completed (synchronous). Calls on one context must not
 *    overlap (one host thread at a time per context).
 *  - Return value: HDI_OK (0) or a negative hdi_status; hdi_last_error()
 *    gives a one-line message. Output buffers are unspecified on error,
 *    except HDI_ERR_NOT_CONVERGED, where they hold the last iterate.
 */
#ifndef HDI_H
#define HDI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hdi_ctx hdi_ctx;

typedef enum {
    HDI_OK = 0,
    HDI_ERR_INVALID_ARG = -1,   /* null pointer, shape/dtype mismatch, tol not in (0,1), mask value not 0/1, k < 0 */
    HDI_ERR_EMPTY_MASK = -2,    /* inpaint/tonal with c = 0: A is singular (Sec. 2.1) */
    HDI_ERR_NOT_CONVERGED = -3, /* iteration cap reached; output holds the last iterate, stats filled */
    HDI_ERR_OUT_OF_MEMORY = -4, /* workspace would exceed the context's HBM budget or cudaMalloc failed */
    HDI_ERR_CUDA = -5,          /* CUDA runtime error */
    HDI_ERR_NONFINITE = -6,     /* non-finite input or residual */
    HDI_ERR_TIMEOUT = -7,       /* a bounded device-side wait gave up */
    HDI_ERR_UNSUPPORTED = -8    /* a configuration this build does not handle */
} hdi_status;

typedef enum { HDI_F32 = 0, HDI_F64 = 1 } hdi_dtype;
typedef enum { HDI_DEVICE = 0, HDI_HOST = 1 } hdi_location;

typedef struct {
    void* data;
    int32_t height, width, channels;
    int32_t dtype;            /* hdi_dtype */
    int64_t row_stride;       /* elements between rows */
    int64_t channel_stride;   /* elements between channels */
    int32_t location;         /* hdi_location */
} hdi_image;

typedef struct {
    uint8_t* data;            /* 0/1 per pixel */
    int32_t height, width;
    int64_t row_stride;       /* bytes between rows */
    int32_t location;         /* hdi_location */
} hdi_mask;

typedef struct {
    int32_t status;           /* same value the call returned */
    int32_t iterations;       /* refinement steps (inpaint) or RAS iterations (tonal) */
    int32_t vcycles;          /* V-cycles run in total, all inner solves included */
    int32_t init_steps;       /* tonal: accepted steps of the Voronoi initialisation (tonal_init = 1) */
    int64_t local_iters;      /* local CG iterations summed over all subdomains and sweeps */
    double rel_res;           /* max over channels of the achieved relative residual */
    double mse;               /* tonal: MSE of B g against f at the last residual evaluation */
    double seconds;           /* wall time of the call */
} hdi_stats;

/* Create a context on `device`, ordered on `cuda_stream` (a cudaStream_t;
 * NULL = the legacy default stream). `config_json` (may be NULL) is a flat
 * JSON object of parameter values, e.g. {"oras_theta": 0.3, "pdl": 1}, with
 * the names and ranges of hdi_set_param; a syntax error, an unknown name or
 * an out-of-range value returns HDI_ERR_INVALID_ARG and creates nothing. */
int hdi_create(hdi_ctx** ctx, int device, void* cuda_stream, const char* config_json);

/* Release the context and its workspace. NULL is accepted. */
int hdi_destroy(hdi_ctx* ctx);

/* Set / get a solver parameter by name (table at the end of this file).
 * Unknown names return HDI_ERR_INVALID_ARG. */
int hdi_set_param(hdi_ctx* ctx, const char* name, double value);
int hdi_get_param(const hdi_ctx* ctx, const char* name, double* value);

/* Homogeneous diffusion inpainting (Sec. 2.1, Eq. "inp-discrete-lsi"):
 * solve (C + (I - C) L) u = C f, L the 5-point negated Laplacian with
 * reflecting boundaries, by multigrid with ORAS smoothing (Sec. 3).
 *   f     in : image (F32 or F64), H x W x ch
 *   mask  in : 0/1, H x W
 *   u0    in : initial guess (same shape/dtype as f), or NULL for the cold
 *              start by reduced full multigrid (Sec. 3.2). Values on the mask
 *              are ignored (u_K = f_K is enforced).
 *   u     out: solution, same shape and dtype as f (may alias u0).
 *   tol      : per-channel relative residual ||C f - A u|| / ||C f||, in (0,1),
 *              evaluated on the GPU's double-float iterate (two FP32 words,
 *              about 48 significant bits) with FP64 accumulation of the
 *              norms; the returned u is that iterate rounded to the dtype.
 *   st   out : statistics, may be NULL. */
int hdi_inpaint(hdi_ctx* ctx, const hdi_image* f, const hdi_mask* mask,
                const hdi_image* u0, hdi_image* u, double tol, hdi_stats* st);

/* Batched inpainting of n independent images of uneven sizes (any number of
 * channels each, each with its own mask), e.g. a request batch. By default
 * (batch_engine = 1) the images go through the batched engine below: every
 * solver phase (ORAS sweep on a level, restriction, prolongation, data
 * pyramid, refinement residual) is ONE kernel launch over all images of all
 * sizes in flight, driven by a (request, channel) task table, and each image
 * stops at its own tolerance. Images are admitted while their workspaces fit
 * hbm_budget_gb; the rest join as earlier ones finish. batch_engine = 0
 * stacks images of one size as the channels of one system and runs the size
 * classes one after another (also the path of the plain FP32 form).
 *   f[n], masks[n], u[n] : as for hdi_inpaint (arrays of descriptors)
 *   st[n]                : per-image statistics (may be NULL)
 * Returns HDI_ERR_NOT_CONVERGED if any image missed tol (others are valid). */
int hdi_inpaint_batch(hdi_ctx* ctx, int n, const hdi_image* f, const hdi_mask* masks, hdi_image* u,
                      double tol, hdi_stats* st);

/* Batched inpainting engine with continuous admission: requests (images of
 * any size) join and leave at V-cycle boundaries. The paper has no
 * counterpart; it serves many inpainting solves of uneven sizes at once
 * (Sec. 2.1 systems, Sec. 3 solver). Each hdi_engine_step runs reduced full
 * multigrid for the requests submitted since the previous step and one
 * V-cycle plus the double-float refinement update for every other request,
 * each phase as one kernel launch over all requests' (channel, tile) work;
 * requests whose relative residual meets their tolerance are finished (u
 * written) and reported. The engine owns one stream-ordered workspace per
 * request in flight (hdi_engine_request_bytes) and admits a request only
 * while the sum stays within its budget.
 *   hdi_engine_create : device, stream (NULL = legacy default), parameters as
 *                       for hdi_create, budget_gb > 0 for the workspaces
 *   hdi_engine_submit : f, mask, u as for hdi_inpaint (device or host), tol in
 *                       (0,1), tag returned when the request finishes. Uploads
 *                       and checks the inputs (waits for the stream); returns
 *                       HDI_ERR_OUT_OF_MEMORY without side effects when the
 *                       request does not fit the budget now. u must stay valid
 *                       until the request is reported.
 *   hdi_engine_step   : one step (waits for the stream at its end); writes up
 *                       to `capacity` finished requests' tags and statistics
 *                       (st.status: HDI_OK, NOT_CONVERGED after max_vcycles,
 *                       NONFINITE) and their count to *ndone; finished
 *                       requests beyond capacity are reported by later calls.
 *   hdi_engine_status : requests in flight, workspace bytes in use, budget.
 *   hdi_engine_request_bytes : workspace one request of that shape needs.
 * One host thread at a time per engine. */
typedef struct hdi_engine hdi_engine;
int hdi_engine_create(hdi_engine** engine, int device, void* cuda_stream, const char* config_json, double budget_gb);
int hdi_engine_destroy(hdi_engine* engine);
int hdi_engine_submit(hdi_engine* engine, const hdi_image* f, const hdi_mask* mask, hdi_image* u, double tol,
                      int64_t tag);
int hdi_engine_step(hdi_engine* engine, int64_t* tags, hdi_stats* stats, int capacity, int* ndone);
int hdi_engine_status(const hdi_engine* engine, int64_t* in_flight, int64_t* bytes_in_use, int64_t* budget_bytes);
int64_t hdi_engine_request_bytes(int32_t height, int32_t width, int32_t channels);
int64_t hdi_engine_launch_count(const hdi_engine* engine);
const char* hdi_engine_last_error(const hdi_engine* engine);

/* Tonal optimisation (Sec. 5, Eq. "tonal-opt-minimisation"): g minimising
 * ||f - A^{-1} C g||_2 with g = 0 off the mask, by restricted additive
 * Schwarz on the normal equations B^T B g = B^T f (Sec. 5.2, Alg. 2); each
 * application of B and B^T is an inpainting solve (Sec. 5.1).
 *   f, mask  in : as for hdi_inpaint
 *   g0       in : initial tonal values (same shape/dtype as f) or NULL (g0 = f)
 *   g       out : optimised values, zero off the mask (may alias g0)
 *   tol         : per-channel ||B^T (f - B g)|| / ||B^T f||, in (0,1) */
int hdi_tonal_opt(hdi_ctx* ctx, const hdi_image* f, const hdi_mask* mask,
                  const hdi_image* g0, hdi_image* g, double tol, hdi_stats* st);

/* One densification step (Sec. 4.1, Alg. 1 with the Delaunay partition, or
 * with the Voronoi cells of the mask pixels when densify_partition = 1;
 * initial mask by random dithering of |L f|, Sec. 4.2).
 *   f     in     : reference image
 *   mask  in/out : current mask; only new 1-bits are written
 *   u     in     : inpainting of f from the current mask (ignored when the
 *                  mask is empty)
 *   k            : number of pixels to add (k >= 0)
 *   seed         : seed of the counter-based generator used on an empty mask
 *   added   out  : pixels actually added (<= k for a non-empty mask) */
int hdi_densify_step(hdi_ctx* ctx, const hdi_image* f, hdi_mask* mask,
                     const hdi_image* u, int64_t k, uint64_t seed, int64_t* added);

/* Densification from the given mask (normally empty) to `density` in n
 * iterations (Sec. 4, Alg. 1 with the image-adaptive initial mask and the
 * growth factor of Sec. 4.2): iteration i runs hdi_densify_step to the
 * cumulative target floor(total * (t^i - 1) / (t^n - 1) + 0.5) (i / n for
 * t = 1; total = floor(density * H * W + 0.5)) and then inpaints to
 * densify_tol, warm-started from the previous inpainting. The paper's
 * experiments use n = 20, t = 1, density 0.05. With densify_voronoi = 1 the
 * Voronoi labels come from jump flooding whose first step after the first
 * labelled mask is the power of two covering the previous labels' largest
 * pixel-to-site distance (the mask only grows, so the bound holds).
 *   f        : image (as hdi_inpaint)
 *   mask     : in/out, the final mask
 *   u   in/out: in: the inpainting of the given mask when it is not empty;
 *                out: the inpainting of the final mask (same shape/dtype as f)
 *   sizes out: may be NULL; n entries, the mask size after each iteration
 * Errors: as hdi_densify_step and hdi_inpaint; NOT_CONVERGED inpaintings are
 * accepted inside the loop. */
int hdi_densify(hdi_ctx* ctx, const hdi_image* f, hdi_mask* mask, hdi_image* u, int32_t n, double t,
                double density, uint64_t seed, int64_t* sizes);

/* Device bytes the context currently holds for its workspaces (all solver
 * workspaces, host-buffer staging and the batched engine's requests in
 * flight); workspaces grow to the largest call served and are kept until
 * hdi_destroy. -1 for a null context. */
int64_t hdi_workspace_bytes(const hdi_ctx* ctx);

/* Number of kernels this context has launched since it was created. */
int64_t hdi_launch_count(const hdi_ctx* ctx);

/* Device time per kernel class, measured with CUDA events recorded on the
 * context's stream around each launch of the class (no extra
 * synchronisation inside a call; events are resolved when a call ends).
 *   enable : 1 = record from now on, 0 = stop recording
 *   reset  : 1 = zero the totals after reading them
 *   ms, launches (out, may be NULL): HDI_TIMING_CLASSES entries each,
 *   accumulated milliseconds and launch counts; names by hdi_timing_name(i):
 *   0 oras_fine     ORAS sweep on the finest level (Sec. 3.1)
 *   1 residual_fine double-float residual / refinement update, finest level
 *   2 prolong_fine  prolongation + correction onto the finest level (Sec. 3.2)
 *   3 restrict_fine residual restriction from the finest level (Sec. 3.2)
 *   4 tonal_echo    local inpainting echoes of the RAS subdomains (Sec. 5.2)
 *   5 tonal_gram    local Gram matrices and their Cholesky factors
 *   6 tonal_local   local solves and weighted extension (Alg. 2, steps 2-3)
 *   7 anderson      Anderson acceleration of the RAS iteration
 *   8 coarse_levels every V-cycle's work below the finest level (all coarse
 *                   sweeps, transfers and the coarsest solve), one interval
 *                   per V-cycle */
#define HDI_TIMING_CLASSES 9
int hdi_timing(hdi_ctx* ctx, int enable, int reset, double* ms, int64_t* launches);
const char* hdi_timing_name(int i);

/* Algorithmic HBM bytes of the launches hdi_timing has timed since its last
 * reset, per class (same order): for each launch, the bytes its arithmetic
 * must move once per value of the finest level (iterate, right-hand side,
 * mask bits, outputs; no halo or overlap re-reads), summed. The streaming
 * classes count them (oras_fine, residual_fine, prolong_fine, restrict_fine);
 * the others report 0. Divided by the class's milliseconds it gives the
 * achieved bandwidth. bytes: HDI_TIMING_CLASSES doubles (out). Drains the
 * context's stream like hdi_timing. Returns HDI_ERR_INVALID_ARG for a null
 * argument. */
int hdi_timing_bytes(hdi_ctx* ctx, double* bytes);

/* Inpainting that allocates no device memory. The paper has no counterpart;
 * this entry point exists for callers that cannot call cudaMalloc while they
 * run: a real-time loop with a fixed memory plan that must not wait on the
 * device allocator, or a host process whose GPU memory is owned by another
 * runtime (a framework's caching allocator that has reserved the device).
 * It solves the same system as hdi_inpaint (cold start, default parameters)
 * with the same kernels, but takes no context and keeps its whole workspace
 * in a 24 MiB array in device global memory that the library declares
 * statically: every GPU that loads libhdi holds that array until the
 * process exits.
 *   device, cuda_stream : GPU index and stream (NULL = legacy default)
 *   f, mask, u          : as for hdi_inpaint, but all three must be DEVICE
 *                         buffers (host buffers would need staging memory)
 *   tol, st             : as for hdi_inpaint (st->local_iters is 0)
 * Size limit: the layout of the image (multigrid levels, three double-float
 * vectors, reductions) must fit the 24 MiB array, about 500,000 pixel x
 * channel values (e.g. 400x400 RGB or 700x700 grey); larger images return
 * HDI_ERR_INVALID_ARG before any GPU work. Host buffers, a null pointer or
 * tol outside (0,1) also return HDI_ERR_INVALID_ARG.
 * Synchronisation: like hdi_inpaint, each call waits for its stream after
 * checking the mask and the image (a flag copied to the host), once per
 * refinement step (the per-channel residual norms copied to the host for
 * the stop test) and after writing u.
 * Current device: the call makes `device` current and restores the calling
 * thread's current device before it returns.
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress (with the device current) and caches it for the
 * process; a cudaDeviceReset invalidates the cached address. All calls on
 * one device share that device's array, and it keeps the previous call's
 * contents (the entry point clears what must start at zero): calls on the
 * same device that overlap, on the GPU or from two host threads, race and
 * corrupt each other. Calls on different devices use different arrays and
 * different host-side copies of the residual norms and do not interfere.
 * No error message is kept; the return code (hdi_status) is the only
 * report. */
int hdi_inpaint_noalloc(int device, void* cuda_stream, const hdi_image* f, const hdi_mask* mask,
                        hdi_image* u, double tol, hdi_stats* st);

/* One-line description of the last error on this context ("" if none). */
const char* hdi_last_error(const hdi_ctx* ctx);

/* Library version string. */
const char* hdi_version(void);

/*
 * Parameters (hdi_set_param names), defaults in brackets:
 *   oras_theta        [0.3]   Robin weight at inner subdomain boundaries (Sec. 3.1)
 *   oras_eta          [1e-3]  local CG stop: ||r_i||^2 <= eta * ||r||^2 / n_subdomains (Sec. 3.3)
 *   oras_max_local    [48]    local CG iteration cap per subdomain and sweep
 *   coarse_eta        [1e-8]  relative squared-residual target of the single-block coarsest solve
 *   max_vcycles       [60]    refinement steps per inpainting solve
 *   tonal_max_iter    [400]   RAS iterations per tonal solve
 *   tonal_inner_ratio [0.1]   inner solves target: ratio * current outer relative residual
 *   tonal_inner_max   [3e-2]  ... but at most this (the early outer iterations)
 *   tonal_anderson_beta [1.0] Anderson mixing parameter beta (step = beta f - sum gamma (dX + beta dF))
 *   tonal_method      [0]     0: RAS (Alg. 2); 1: CGNR, conjugate gradients on the normal equations
 *                             with multigrid inner solves (Sec. 5.1, "Improvements")
 *   tonal_mse_gain    [0]     > 0: hdi_tonal_opt also stops (successfully) once an outer iteration
 *                             improves the MSE by less than this relative amount (Sec. 6: 1e-3)
 *   tonal_block       [0]     RAS subdomain side: 32 or 64 (the paper's 64, overlap 6); 0 picks 64
 *                             below 3% mask density and 32 above (64 converges in fewer outer
 *                             iterations at sparse masks, 32 keeps the local factors cheap at dense ones;
 *                             a 64x64 block holding more than 1024 mask pixels switches the call to 32)
 *   tonal_init        [0]     0: start from g0 (f on the mask if g0 is NULL); 1: first run the
 *                             Voronoi initialisation (Sec. 5.3) from f: Richardson steps
 *                             g += vi_tau C W (f - A^-1 C g), one inpainting each, kept while the MSE falls
 *   vi_max_iter       [20]    its step cap
 *   vi_tau            [1.0]   its step size
 *   vi_weight         [0]     zones of W: 0 Voronoi cell with weight 1/(1 + ln(1 + distance)),
 *                             1 Voronoi cell with constant weight, 2 the 3x3 neighbourhood (error balancing)
 *   vi_inner_tol      [1e-3]  relative residual of its inpaintings (1e-5 gives the same steps and
 *                             PSNR to 4 decimals at 4K, 1.5x slower)
 *   tonal_max_iter = 0 returns the initial values (with their residual and MSE) as a success.
 *   densify_voronoi   [0]     hdi_densify_step / hdi_densify: 0 exact Voronoi labels, 1 jump flooding
 *                             (Sec. 4.2; approximate, so masks differ from the exact mode)
 *   jfa_first_step    [0]     first jump-flooding step of hdi_densify_step (0: half the padded side;
 *                             a shortened schedule that misses pixels falls back to the full one)
 *   densify_tol       [1e-6]  relative residual of the inpaintings inside hdi_densify
 *   densify_partition [0]     hdi_densify_step / hdi_densify: 0 Delaunay triangles of the mask pixels
 *                             (Sec. 4.1, Alg. 1); 1 Voronoi cells of the mask pixels (the Voronoi-based
 *                             densification of the Sec. 6.2 comparison): one new pixel per selected cell
 *   inpaint_fp32      [0]     1: hdi_inpaint and hdi_inpaint_batch run the plain FP32 form (FP32 iterate,
 *                             FP32 residual and update, no double-float refinement), the per-image
 *                             baseline of the mixed-precision path; it stalls near the FP32 rounding
 *                             level (about 1e-6 relative residual) and then returns NOT_CONVERGED
 *   batch_engine      [1]     hdi_inpaint_batch: 1 the batched engine (one launch per phase across
 *                             sizes), 0 size classes stacked as channels, one class after another
 *   mg_truncate       [1]     end the multigrid hierarchy at its first level whose pixels are all
 *                             known (the any-of-4 mask restriction fills the coarse masks): every
 *                             coarser level's correction is exactly zero, so results are unchanged
 *                             bit for bit; 0 keeps every level down to 32 x 32
 *   strip_rows        [0]     rows per warp of the quad-strip kernels (restriction, prolongation,
 *                             residuals; even, >= 2); 0 chooses by level size
 *   oras_warp         [1]     layout of the 32x32 local CG solves (ORAS sweeps and the tonal echoes
 *                             on 32x32 RAS blocks): 1 one warp per solve (no CTA barriers), 0 two
 *                             warps per solve
 *   oras_warp_waves   [2]     with oras_warp = 1, an ORAS sweep takes the one-warp layout only if
 *                             its (subdomain, channel) solves fill the GPU at least this many times
 *                             (12 one-warp CTAs per SM); smaller sweeps (coarse levels, small
 *                             images) split each solve over two warps, which finishes sooner when
 *                             there are too few solves to hide the latency of a single warp
 *   stage_loads       [3]     level-0 kernels that copy their next rows into shared memory (cp.async)
 *                             while they compute the current ones, a bit mask: 1 refinement
 *                             residual, 2 restriction; a clear bit loads each row into registers
 *                             when it is needed. Bit-identical results either way
 *   tonal_anderson    [8]     Anderson window on the RAS iteration (0 = plain Alg. 2)
 *   tonal_oras_eta    [3e-2]  oras_eta used inside the tonal inner solves
 *   fine_pre, fine_post [1, 1] ORAS sweeps before / after the coarse correction on the finest level
 *   tonal_fine_pre, tonal_fine_post [2, 1] the same inside the tonal inner solves
 *   tonal_echo_rtol   [3e-3]  relative CG tolerance of the local echo solves
 *   tonal_echo_max_iter [300] CG iteration cap of an echo solve
 *   coarse_level_eta  [0.3]   oras_eta on the levels between the finest and the coarsest (0 = oras_eta)
 *   coarse_level_max  [48]    local CG iteration cap on those levels
 *   coarse_max_local  [600]   CG iteration cap of the coarsest solve
 *   trace             [0]     1 = one line per RAS iteration on stderr
 *   hbm_budget_gb     [200]   workspace cap for this context
 */

#ifdef __cplusplus
}
#endif

#endif /* HDI_H */

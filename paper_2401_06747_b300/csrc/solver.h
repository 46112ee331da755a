// solver.h -- host-side context of libhdi: parameters, workspace arenas,
// multigrid hierarchy and the solver drivers' declarations.
#pragma once
#include <atomic>
#include <cstdarg>
#include <utility>
#include <string>
#include <cuda_runtime.h>
#include "../../include/hdi.h"
#include "common.cuh"
#include "stencil.cuh"

struct Params {
    double oras_theta = 0.3;        // Robin weight (Sec. 3.1)
    double oras_eta = 1e-3;         // local stop fraction (Sec. 3.3)
    double oras_max_local = 48;
    double coarse_eta = 1e-8;
    double coarse_max_local = 600;
    double max_vcycles = 60;
    double tonal_max_iter = 400;
    double tonal_inner_ratio = 0.1;
    double tonal_anderson_beta = 1.0;  // Anderson mixing parameter
    double tonal_inner_max = 3e-2;   // loosest inner solve tolerance (early outer iterations)
    double tonal_echo_rtol = 3e-3;
    double tonal_echo_max_iter = 300;
    double hbm_budget_gb = 200.0;
    double trace = 0;               // 1: one line per outer iteration on stderr
    double tonal_oras_eta = 3e-2;   // local stop fraction inside the tonal inner solves
    double coarse_level_eta = 0.3;  // local stop fraction on levels >= 1 (0 = same as oras_eta)
    double coarse_level_max = 48;   // local CG cap on levels >= 1 (below the coarsest)
    double fine_pre = 1;            // ORAS pre-smoothing sweeps on the finest level
    double fine_post = 1;           // ORAS post-smoothing sweeps on the finest level
    double tonal_fine_pre = 2;      // fine_pre inside the tonal inner solves
    double tonal_fine_post = 1;     // fine_post inside the tonal inner solves
    double tonal_anderson = 8;      // Anderson window on the RAS iteration (0 = plain Alg. 2)
    double pdl = 1;                 // programmatic dependent launch of the multigrid kernels
    double tonal_method = 0;        // 0: RAS (Alg. 2), 1: CGNR (Sec. 5.1)
    double tonal_mse_gain = 0;      // > 0: also stop once an iteration improves the MSE by less (relative)
    double tonal_block = 0;         // RAS subdomain side: 32, 64 (Sec. 5.2 uses 64), 0: 64 below 3% density
    double tonal_init = 0;          // 0: g0 (or f on the mask); 1: Voronoi initialisation (Sec. 5.3) first
    double vi_max_iter = 20;        // Richardson steps of the Voronoi initialisation
    double vi_tau = 1.0;            // its step size
    double vi_weight = 0;           // 0: Voronoi cell, inverse-log distance; 1: Voronoi cell, constant; 2: 3x3
    double vi_inner_tol = 1e-3;     // relative residual of its inpaintings
    double densify_voronoi = 0;     // 0: exact Voronoi labels; 1: jump flooding (Sec. 4.2)
    double jfa_first_step = 0;      // first jump-flooding step (0: half the padded image side)
    double densify_tol = 1e-6;      // relative residual of the inpaintings of hdi_densify
    double densify_partition = 0;   // 0: Delaunay triangles (Alg. 1); 1: Voronoi cells of the mask (Sec. 6.2)
    double inpaint_fp32 = 0;        // 1: hdi_inpaint / hdi_inpaint_batch in the plain FP32 form
    double batch_engine = 1;        // hdi_inpaint_batch: 1 the batched engine (all sizes per launch), 0 size classes
    double mg_truncate = 1;         // end the hierarchy at its first fully known level (exact)
    double strip_rows = 0;          // rows per warp of the quad-strip kernels (even, >= 2); 0: chosen by size
    double oras_warp = 1;           // ORAS sweep layout: 1 one warp per subdomain, 0 two warps
    double oras_warp_waves = 2;     // one-warp layout only for sweeps of at least this many waves of
                                    // its CTAs (12 per SM); smaller sweeps (coarse levels) take two
    double stage_loads = 3;         // level-0 kernels that stage their next rows (cp.async), bit mask:
                                    // 1 refinement residual, 2 restriction
};

struct Level {
    int H = 0, W = 0, P = 0, wp = 0;
    long long cs = 0;
    uint32_t* bits = nullptr;
    float* xa = nullptr;
    float* xb = nullptr;
    float* b = nullptr;
    int nbx = 0, nby = 0;
};

struct Ctx;
struct Engine;   // batched engine (engine.cuh)
void engine_delete(Engine* e);
size_t engine_used_bytes(const Engine* e);

// One cudaMalloc'd block carved into 256-byte aligned pieces.
struct Arena {
    void* base = nullptr;
    size_t cap = 0, used = 0;
    bool async = false;              // allocated with cudaMallocAsync on astream (released with cudaFreeAsync)
    cudaStream_t astream = nullptr;
    int reserve(Ctx& c, size_t bytes, const char* what);
    void* take(size_t bytes);
    void release();
};

enum { START_FMG = 0, START_WARM = 1, START_ZERO = 2 };
constexpr int kMaxCh = 256;       // channels of one solve (a batch stacks its images' channels)

inline DFc cview(const DF& v) { return DFc{v.hi, v.lo}; }

struct SolveSpec {
    DF u[2];
    int cur = 0;
    int rhs = 0;
    DFc d{nullptr, nullptr};
    DFc y{nullptr, nullptr};
    int start = START_FMG;
    double tol = 1e-6;
    int max_iter = 60;
    int iterations = 0;
    double rel[kMaxCh] = {};
    double rel_max = 0;
    double bnorm2[kMaxCh] = {};
    bool plain32 = false;   // plain FP32 form: FP32 iterate and residual, no refinement (RHS_DATA only)
};

constexpr int kMaxLevels = 16;
constexpr int kOv = 6;            // overlap of the 32x32 subdomains (Sec. 3.3)
constexpr int kSlots = 32;        // reduction slots
constexpr int kSlotR64 = 16;      // ||r||^2 of the FP64 residual
constexpr int kSlotB64 = 17;      // ||b||^2 of the FP64 residual
constexpr int kSlotTonalR = 18;   // ||B^T(f - Bg)||^2
constexpr int kSlotTonalE = 19;   // ||f - Bg||^2
constexpr int kSlotCgW = 20;      // CGNR: ||B p||^2
constexpr int kSlotCgZ = 21;      // CGNR: ||z||^2 of the previous iteration
constexpr int kSlotCgZP = 22;     // CGNR: <z, p>
constexpr int kSlotViE = 23;      // Voronoi initialisation: ||f - u||^2
constexpr int kCntOnes = 0;
constexpr int kCntLocal = 1;
constexpr int kCntEcho = 2;
constexpr int kCntLevelKnown = 16;   // [kMaxLevels] known pixels per level of the mask pyramid
constexpr int kMaxTimed = 2048;   // timed launches buffered between flushes
enum { kT_Oras = 0, kT_Residual, kT_Prolong, kT_Restrict, kT_Echo, kT_Gram, kT_Local, kT_Anderson, kT_Coarse };
// double-float vectors of level-0 size
enum { kF = 0, kU0, kU1, kG, kY0, kY1, kW0, kW1, kP, kNumDF };

// Streaming multiprocessors of `device`, queried once per device (148 on a
// B300 if the query fails).
inline int sm_count(int device) {
    static std::atomic<int> cache[64];
    if (device < 0 || device >= 64) return 148;
    int n = cache[device].load(std::memory_order_relaxed);
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n <= 0) {
        (void)cudaGetLastError();
        n = 148;
    }
    cache[device].store(n, std::memory_order_relaxed);
    return n;
}

// Launch with programmatic stream serialisation (see pdl_wait in
// common.cuh) when `pdl` is set, else a plain launch.
// launch_ks: the same with `smem` bytes of dynamic shared memory.
template <typename... K, typename... A>
inline cudaError_t launch_ks(bool pdl, size_t smem, void (*k)(K...), dim3 grid, dim3 block, cudaStream_t s,
                             A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}
template <typename... K, typename... A>
inline cudaError_t launch_k(bool pdl, void (*k)(K...), dim3 grid, dim3 block, cudaStream_t s, A&&... args) {
    return launch_ks(pdl, 0, k, grid, block, s, std::forward<A>(args)...);
}

// Device-side results of the input checks (counters[0..32): ones, local
// iterations, ..., known pixels per level; flags[0] bad mask value,
// flags[1] non-finite image value), read back in one go.
struct LoadReadback {
    unsigned long long counters[32];
    unsigned flags[2];
};

struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    Params p;
    std::string err;
    Arena ws;      // multigrid + FP64 vectors
    Arena tws;     // tonal local factors
    Arena dws;     // densification
    Arena vws;     // Voronoi initialisation
    Arena lws;     // list of mask pixels (tonal optimisation)
    Arena stage;   // host staging
    // side stream for a host image's upload into `stage` that overlaps the
    // context stream's kernels; uev[0]: the context stream is done with
    // `stage`, uev[1]: the upload has landed
    cudaStream_t ustream = nullptr;
    cudaEvent_t uev[2] = {nullptr, nullptr};
    int upload_begin(const hdi_image* im);
    // a host image whose upload the tonal set-up starts right before its echo
    // kernel, after its own small host copies (which would otherwise queue
    // behind the large one)
    const hdi_image* pending_upload = nullptr;
    int H = 0, W = 0, nch = 0, nlev = 0;
    // levels the solves use: the hierarchy ends at its first level whose
    // pixels are all known (every coarser level's correction is exactly 0)
    int nlev_run = 0;
    int nmask = 1;             // mask planes (1 = shared by all channels)
    int* d_chmask = nullptr;   // [kMaxCh] mask plane of each channel (batched solves)
    Level lev[kMaxLevels];
    DF dfv[kNumDF] = {};
    float* tres = nullptr;     // tonal residual B^T (f - B g) on mask pixels, FP32
    float* flo2 = nullptr;     // bits of f below its double-float pair (FP64 input)
    double* partials = nullptr;
    double* scal = nullptr;
    unsigned* tickets = nullptr;
    unsigned long long* counters = nullptr;
    unsigned* flags = nullptr;
    double* hscal = nullptr;   // pinned host mirror
    int maxparts_ = 1;
    bool mask_key_valid = false;
    long long mask_ones = 0;
    int vcycles_run = 0;
    int64_t launches = 0;      // kernels launched by this context
    // per-class device time (hdi_timing)
    bool timing = false;
    cudaEvent_t* tev = nullptr;
    int tn = 0;
    int tcls[kMaxTimed];
    double tbyt[kMaxTimed];
    double ttot[HDI_TIMING_CLASSES] = {};
    int64_t tcnt[HDI_TIMING_CLASSES] = {};
    double tbytes[HDI_TIMING_CLASSES] = {};
    bool f_lo_zero = false;   // the low words of f are all zero (every image of the call was FP32)
    void tstart(int cls, double bytes = 0.0);   // bytes: algorithmic HBM bytes of the launch
    void tstop();
    int tflush();
    // tonal local factors (valid for the mask of the current tonal call)
    int* t_off = nullptr;
    long long* t_goff = nullptr;
    uint16_t* t_list = nullptr;
    float* t_echo = nullptr;
    float* t_fac = nullptr;
    long long t_total = 0;
    // Anderson acceleration state (compact mask-pixel vectors)
    int aa_M = 0;
    int* aa_idx = nullptr;
    float* aa_fv = nullptr;
    float* aa_fvprev = nullptr;
    float* aa_dF = nullptr;
    float* aa_dX = nullptr;
    double* aa_part = nullptr;
    double* aa_out = nullptr;
    double* aa_gam = nullptr;
    unsigned* aa_ticket = nullptr;

    int fail(int code, const char* fmt, ...);
    int cuda_check(cudaError_t e, const char* what);
    int sync(const char* what);
    size_t other_bytes() const;
    int setup(int H, int W, int nch, int nmask = 1);
    int setup_lean(int H, int W, int nch, cudaStream_t s);   // one request of the batched engine (engine.cuh)
    GridReduce reducer(int slot, int nparts) const;
    // rows per warp of the quad-strip kernels: the strip_rows parameter, else by size
    // dynamic shared memory of a level-0 kernel that stages its row loads
    // (`bit` of stage_loads; 0 bytes: the unstaged loop)
    size_t stage_bytes(int bit, size_t b) const { return ((int)p.stage_loads & bit) ? b : 0; }
    int qrows(int H_, int W_, int n) const { return p.strip_rows >= 2 ? ((int)p.strip_rows / 2) * 2 : quad_rows(H_, W_, n); }
    LevelArr arr(int l) const;
    MaskView mview(int l) const;
    void build_mask_pyramid();
    void oras(int l, bool zero, const float* xin, float* xout, const double* rnorm2, bool coarsest,
              unsigned long long* iters);
    void vcycle(int l);
    void residual_norm_level(int l, const float* x, int slot);
    void fmg(DFc d);
    void residual(int rhs, int init, DFc uin, DF uout, const float* x32, DFc d, DFc y, bool want_b,
                  bool p32 = false);
    int solve(SolveSpec& s);
    int check_image(const hdi_image* im, const char* name, int H, int W, int nch);
    int load_image(const hdi_image* im, DF dst, float* lo2 = nullptr, int c0 = 0, bool wait = true,
                   bool prestaged = false);
    int store_image(DFc src, hdi_image* im, bool zero_off_mask, const float* known_lo2 = nullptr, int c0 = 0,
                    bool wait = true);
    int load_mask(const hdi_mask* m, long long* ones, int plane = 0, bool pyramid = true, bool wait = true);
    void enqueue_load_readback(LoadReadback* rb);
    void set_levels_run(const unsigned long long* known);
    int load_checks(const LoadReadback& rb, long long* ones);
    int inpaint_batch(int n, const hdi_image* f, const hdi_mask* m, hdi_image* u, double tol, hdi_stats* st);
    int inpaint_batch_engine(int n, const hdi_image* f, const hdi_mask* m, hdi_image* u, double tol, hdi_stats* st);
    int inpaint_batch_classes(int n, const hdi_image* f, const hdi_mask* m, hdi_image* u, double tol, hdi_stats* st);
    Engine* eng = nullptr;     // batched engine of hdi_inpaint_batch (created on first use)
    int read_slot(int slot, double* out);
    int tonal_setup();
    int tonal_setup_blk(int blk);
    int t_blk = 32, t_nbx = 0, t_nby = 0, t_maxm = 0;   // RAS tiling of the last tonal set-up
    void tonal_residual(DFc y, DFc w);
    void tonal_local(float* out);
    int tonal_aa_step(int n, const float* fvfull, DF G);
    int tonal_cgnr(SolveSpec& sw, const double* btf2, double tol, int& it, double& rel_max, double& mse_last,
                   bool& by_gain);
    int tonal_vi(int& steps, double& mse_best, DF* u_kept);
    int mask_list();
    int* mlist = nullptr;      // level-0 mask pixels, raster order (offsets y * pitch + x)
    int mlist_n = 0;
    bool y_warm = false;
    long long last_label_maxd2 = 0;   // densification: largest squared pixel-to-site distance of the last labels       // tonal: Y0 holds B g of the initial g (from the Voronoi initialisation)
    int inpaint(const hdi_image* f, const hdi_mask* mask, const hdi_image* u0, hdi_image* u, double tol,
                hdi_stats* st);
    int tonal(const hdi_image* f, const hdi_mask* mask, const hdi_image* g0, hdi_image* g, double tol,
              hdi_stats* st);
    int dens_load(const hdi_image* im, double* dst, void* hstage);
    int densify(const hdi_image* f, hdi_mask* mask, const hdi_image* u, int64_t k, uint64_t seed, int64_t* added);
    int densify_run(const hdi_image* f, hdi_mask* mask, hdi_image* u, int n, double t, double density, uint64_t seed,
                    int64_t* sizes);
};

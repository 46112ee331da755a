// hdi.cu -- libhdi: C ABI, context/workspace management and the solver
// drivers (multigrid ORAS inpainting, RAS tonal optimisation,
// densification) for one B300 (sm_103a).
#include <cstdio>
#include <cstring>
#include <cmath>
#include <string>
#include <vector>
#include <algorithm>
#include <chrono>
#include <climits>
#include <atomic>
#include <mutex>

#include "../../include/hdi.h"
#include "common.cuh"
#include "oras.cuh"
#include "oras_warp.cuh"
#include "stencil.cuh"
#include "solver.h"
#include "tonal.cuh"
#include "densify.cuh"
#include "vi.cuh"

// ----------------------------------------------------------------- params ---

namespace {

struct ParamDef {
    const char* name;
    double Params::*field;
    double lo, hi;
};

const ParamDef kParams[] = {
    {"oras_theta", &Params::oras_theta, 0.0, 1.0},
    {"oras_eta", &Params::oras_eta, 1e-12, 1.0},
    {"oras_max_local", &Params::oras_max_local, 1, 1024},
    {"coarse_eta", &Params::coarse_eta, 1e-16, 1.0},
    {"coarse_max_local", &Params::coarse_max_local, 1, 4096},
    {"max_vcycles", &Params::max_vcycles, 1, 10000},
    {"tonal_max_iter", &Params::tonal_max_iter, 0, 100000},
    {"tonal_inner_ratio", &Params::tonal_inner_ratio, 1e-6, 1.0},
    {"tonal_inner_max", &Params::tonal_inner_max, 1e-12, 0.5},
    {"tonal_anderson_beta", &Params::tonal_anderson_beta, 1e-3, 2.0},
    {"tonal_method", &Params::tonal_method, 0, 1},
    {"tonal_mse_gain", &Params::tonal_mse_gain, 0, 0.5},
    {"tonal_init", &Params::tonal_init, 0, 1},
    {"tonal_block", &Params::tonal_block, 0, 64},
    {"pdl", &Params::pdl, 0, 1},
    {"vi_max_iter", &Params::vi_max_iter, 0, 1000},
    {"vi_tau", &Params::vi_tau, 1e-3, 2.0},
    {"vi_weight", &Params::vi_weight, 0, 2},
    {"vi_inner_tol", &Params::vi_inner_tol, 1e-12, 0.5},
    {"densify_voronoi", &Params::densify_voronoi, 0, 1},
    {"jfa_first_step", &Params::jfa_first_step, 0, 1 << 30},
    {"densify_tol", &Params::densify_tol, 1e-12, 0.5},
    {"tonal_echo_rtol", &Params::tonal_echo_rtol, 1e-12, 1.0},
    {"tonal_echo_max_iter", &Params::tonal_echo_max_iter, 1, 4096},
    {"hbm_budget_gb", &Params::hbm_budget_gb, 0.001, 1e6},
    {"trace", &Params::trace, 0, 1},
    {"tonal_anderson", &Params::tonal_anderson, 0, 8},
    {"tonal_oras_eta", &Params::tonal_oras_eta, 1e-12, 1.0},
    {"coarse_level_eta", &Params::coarse_level_eta, 0, 1.0},
    {"coarse_level_max", &Params::coarse_level_max, 1, 1024},
    {"fine_pre", &Params::fine_pre, 0, 4},
    {"fine_post", &Params::fine_post, 0, 4},
    {"tonal_fine_pre", &Params::tonal_fine_pre, 0, 4},
    {"tonal_fine_post", &Params::tonal_fine_post, 0, 4},
    {"oras_warp", &Params::oras_warp, 0, 1},
    {"oras_warp_waves", &Params::oras_warp_waves, 0, 1e6},
    {"stage_loads", &Params::stage_loads, 0, 3},
    {"densify_partition", &Params::densify_partition, 0, 1},
    {"inpaint_fp32", &Params::inpaint_fp32, 0, 1},
    {"batch_engine", &Params::batch_engine, 0, 1},
    {"strip_rows", &Params::strip_rows, 0, 64},
    {"mg_truncate", &Params::mg_truncate, 0, 1},
};

}  // namespace

// ------------------------------------------------------------- utilities ---

int Ctx::fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    err = buf;
    return code;
}

int Ctx::cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return HDI_OK;
    return fail(HDI_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int Ctx::sync(const char* what) {
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    return cuda_check(e, what);
}

void Arena::release() {
    if (base) {
        if (async) cudaFreeAsync(base, astream);
        else cudaFree(base);
    }
    base = nullptr;
    cap = used = 0;
}

int Arena::reserve(Ctx& c, size_t bytes, const char* what) {
    if (bytes <= cap) {
        used = 0;
        return HDI_OK;
    }
    release();
    const double budget = c.p.hbm_budget_gb * 1e9;
    if ((double)(bytes + c.other_bytes()) > budget)
        return c.fail(HDI_ERR_OUT_OF_MEMORY, "%s: %.3f GB workspace exceeds the %.3f GB budget", what,
                      (bytes + c.other_bytes()) / 1e9, c.p.hbm_budget_gb);
    cudaError_t e = cudaMalloc(&base, bytes);
    if (e != cudaSuccess) {
        base = nullptr;
        cudaGetLastError();
        return c.fail(HDI_ERR_OUT_OF_MEMORY, "%s: cudaMalloc(%zu) failed: %s", what, bytes, cudaGetErrorString(e));
    }
    cap = bytes;
    used = 0;
    return HDI_OK;
}

void* Arena::take(size_t bytes) {
    size_t off = (used + 255) & ~(size_t)255;
    used = off + bytes;
    return (char*)base + off;
}

size_t Ctx::other_bytes() const { return ws.cap + tws.cap + dws.cap + vws.cap + lws.cap + stage.cap; }

// Device-time bookkeeping per kernel class (CUDA events on the context's
// stream around each timed launch; resolved after the stream drains).
void Ctx::tstart(int cls, double bytes) {
    if (!timing || !tev) return;
    if (tn >= kMaxTimed && tflush()) return;
    tcls[tn] = cls;
    tbyt[tn] = bytes;
    cudaEventRecord(tev[2 * tn], stream);
}
void Ctx::tstop() {
    if (!timing || !tev || tn >= kMaxTimed) return;
    cudaEventRecord(tev[2 * tn + 1], stream);
    ++tn;
}
int Ctx::tflush() {
    if (!tev || tn == 0) return HDI_OK;
    int rc = sync("timing");
    if (rc) return rc;
    for (int i = 0; i < tn; ++i) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, tev[2 * i], tev[2 * i + 1]);
        ttot[tcls[i]] += ms;
        tcnt[tcls[i]] += 1;
        tbytes[tcls[i]] += tbyt[i];
    }
    tn = 0;
    return HDI_OK;
}

// ------------------------------------------------------------ hierarchy ---

static inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Upper bound on the CTAs per channel of any reducing kernel on an H x W
// level: column strips of 128 columns x at least 4 rows, and the 32x8 tiles
// of the tonal residual.
static inline int reduction_parts(int H, int W) {
    const int strips = ((W + 127) / 128) * ((H + 3) / 4);
    const int tiles = ((W + 31) / 32) * ((H + 7) / 8);
    return std::max(strips, tiles);
}

// Plans the level sizes, reserves the workspace and carves the buffers.
int Ctx::setup(int H_, int W_, int nch_, int nmask_) {
    if (H_ == H && W_ == W && nch_ == nch && nmask_ == nmask && ws.base) return HDI_OK;
    if (nch_ > kMaxCh || nmask_ > kMaxCh || nmask_ < 1) return fail(HDI_ERR_INVALID_ARG, "too many channels in one solve");
    std::vector<std::pair<int, int>> sizes;
    int h = H_, w = W_;
    sizes.push_back({h, w});
    while (std::max(h, w) > 32 && (int)sizes.size() < kMaxLevels) {
        h = (h + 1) / 2;
        w = (w + 1) / 2;
        sizes.push_back({h, w});
    }
    const int nl = (int)sizes.size();
    // bytes
    size_t bytes = 0;
    auto acc = [&](size_t b) { bytes += ((b + 255) & ~(size_t)255); };
    int maxparts = 1;
    for (int l = 0; l < nl; ++l) {
        const int P = round_up(sizes[l].second, 32);
        const int wp = (sizes[l].second + 31) / 32 + 1;
        acc((size_t)nmask_ * sizes[l].first * wp * 4);   // bits, one plane per mask
        for (int k = 0; k < 3; ++k) acc((size_t)nch_ * sizes[l].first * P * 4);   // xa, xb, b
        maxparts = std::max(maxparts, reduction_parts(sizes[l].first, sizes[l].second));
    }
    const int P0 = round_up(W_, 32);
    const size_t n32 = (size_t)nch_ * H_ * P0;
    for (int k = 0; k < kNumDF; ++k) acc(n32 * 8);            // double-float vectors
    acc(n32 * 4);                                             // tonal residual
    acc(n32 * 4);                                             // third component of f
    acc((size_t)kSlots * maxparts * nch_ * 8);                // reduction partials
    acc((size_t)kSlots * kMaxCh * 8);                         // reduction outputs
    acc((size_t)kSlots * 4);                                  // tickets
    acc(64 * 8);                                              // counters / flags
    int rc = ws.reserve(*this, bytes, "inpainting workspace");
    if (rc) { H = W = nch = 0; return rc; }
    H = H_; W = W_; nch = nch_; nlev = nl; nlev_run = nl; nmask = nmask_;
    for (int l = 0; l < nl; ++l) {
        Level& L = lev[l];
        L.H = sizes[l].first;
        L.W = sizes[l].second;
        L.P = round_up(L.W, 32);
        L.wp = (L.W + 31) / 32 + 1;
        L.cs = (long long)L.H * L.P;
        L.bits = (uint32_t*)ws.take((size_t)nmask * L.H * L.wp * 4);
        L.xa = (float*)ws.take((size_t)nch * L.cs * 4);
        L.xb = (float*)ws.take((size_t)nch * L.cs * 4);
        L.b = (float*)ws.take((size_t)nch * L.cs * 4);
        L.nbx = tile_count(L.W, 32, kOv);
        L.nby = tile_count(L.H, 32, kOv);
    }
    for (int i = 0; i < kNumDF; ++i) {
        dfv[i].hi = (float*)ws.take(n32 * 8);
        dfv[i].lo = dfv[i].hi + n32;
    }
    tres = (float*)ws.take(n32 * 4);
    flo2 = (float*)ws.take(n32 * 4);
    maxparts_ = maxparts;
    partials = (double*)ws.take((size_t)kSlots * maxparts * nch * 8);
    scal = (double*)ws.take((size_t)kSlots * kMaxCh * 8);
    tickets = (unsigned*)ws.take((size_t)kSlots * 4);
    counters = (unsigned long long*)ws.take(64 * 8);
    if (ws.used > ws.cap) {
        H = W = nch = 0;
        return fail(HDI_ERR_CUDA, "internal: workspace carving exceeds its reservation");
    }
    cudaMemsetAsync(tickets, 0, (size_t)kSlots * 4, stream);
    cudaMemsetAsync(counters, 0, 64 * 8, stream);
    cudaMemsetAsync(scal, 0, (size_t)kSlots * kMaxCh * 8, stream);
    // zero-fill mask padding words once per setup
    for (int l = 0; l < nl; ++l) cudaMemsetAsync(lev[l].bits, 0, (size_t)nmask * lev[l].H * lev[l].wp * 4, stream);
    mask_key_valid = false;
    return cuda_check(cudaGetLastError(), "workspace setup");
}

GridReduce Ctx::reducer(int slot, int nparts) const {
    GridReduce r;
    r.partials = partials + (size_t)slot * maxparts_ * nch;
    r.out = scal + slot * kMaxCh;
    r.ticket = tickets + slot;
    r.nparts = nparts;
    r.nch = nch;
    return r;
}

LevelArr Ctx::arr(int l) const {
    LevelArr a;
    a.H = lev[l].H;
    a.W = lev[l].W;
    a.pitch = lev[l].P;
    a.cs = lev[l].cs;
    return a;
}

MaskView Ctx::mview(int l) const {
    MaskView m;
    m.bits = lev[l].bits;
    m.H = lev[l].H;
    m.W = lev[l].W;
    m.wpitch = lev[l].wp;
    m.chmask = nmask > 1 ? d_chmask : nullptr;
    m.cstride = (long long)lev[l].H * lev[l].wp;
    return m;
}

// Builds the coarse masks from the level-0 bits (any-of-4, Sec. 3.3).
// Counts each coarse level's known pixels (all mask planes) into
// counters[kCntLevelKnown + l].
void Ctx::build_mask_pyramid() {
    cudaMemsetAsync(counters + kCntLevelKnown, 0, kMaxLevels * 8, stream);
    for (int l = 0; l + 1 < nlev; ++l) {
        const Level& C = lev[l + 1];
        dim3 blk(64), grd((C.wp + 63) / 64, C.H, nmask);
        k_restrict_mask<<<grd, blk, 0, stream>>>(mview(l), C.bits, C.H, C.W, C.wp, counters + kCntLevelKnown + l + 1);
        ++launches;
    }
}

// ---------------------------------------------------------- multigrid ---

void Ctx::oras(int l, bool zero, const float* xin, float* xout, const double* rnorm2, bool coarsest,
               unsigned long long* iters) {
    const Level& L = lev[l];
    OrasArgs a;
    a.m = mview(l);
    a.H = L.H;
    a.W = L.W;
    a.pitch = L.P;
    a.cstride = L.cs;
    a.nch = nch;
    a.nbx = L.nbx;
    a.nby = L.nby;
    a.stride = 32 - kOv;
    a.ov = kOv;
    a.theta = (float)p.oras_theta;
    const double eta = (l > 0 && p.coarse_level_eta > 0) ? p.coarse_level_eta : p.oras_eta;
    a.maxit = coarsest ? (int)p.coarse_max_local : (l > 0 ? (int)p.coarse_level_max : (int)p.oras_max_local);
    a.thresh_scale = coarsest ? p.coarse_eta : eta / (double)(L.nbx * L.nby);
    a.xin = xin;
    a.xout = xout;
    a.b = L.b;
    a.rnorm2 = rnorm2;
    a.iters = iters;
    const dim3 blocks(L.nbx, L.nby, nch);   // one CTA per (subdomain, channel)
    // read x (unless it starts at 0), b and the mask bits, write x: once per value
    if (l == 0) tstart(kT_Oras, (zero ? 8.125 : 12.125) * (double)nch * L.H * L.W);
    const bool full = L.W >= 32 && L.H >= 32;
    const bool pd = p.pdl >= 0.5;
    // one warp per subdomain (oras_warp.cuh) where the sweep fills the GPU
    // several times over; a sweep of fewer subdomains finishes sooner with
    // each solve split over two warps (shorter critical path per subdomain)
    const double waves = (double)L.nbx * L.nby * nch / (12.0 * sm_count(device));
    if (p.oras_warp >= 0.5 && waves >= p.oras_warp_waves) {
        if (zero) {
            if (full) launch_k(pd, k_oras_w<true, true>, blocks, dim3(32), stream, a);
            else launch_k(pd, k_oras_w<true, false>, blocks, dim3(32), stream, a);
        } else {
            if (full) launch_k(pd, k_oras_w<false, true>, blocks, dim3(32), stream, a);
            else launch_k(pd, k_oras_w<false, false>, blocks, dim3(32), stream, a);
        }
    } else if (zero) {
        if (full) launch_k(pd, k_oras<true, true>, blocks, dim3(kLocalThreads), stream, a);
        else launch_k(pd, k_oras<true, false>, blocks, dim3(kLocalThreads), stream, a);
    } else {
        if (full) launch_k(pd, k_oras<false, true>, blocks, dim3(kLocalThreads), stream, a);
        else launch_k(pd, k_oras<false, false>, blocks, dim3(kLocalThreads), stream, a);
    }
    ++launches;
    if (l == 0) tstop();
}


// One V-cycle (Sec. 3.2) on the correction equation A_l x = b_l, x from 0.
// Result in lev[l].xa. Level 0 uses fine_pre / fine_post ORAS sweeps
// (default 1 and 1, the paper's choice, Sec. 3.3); coarser levels one each.
void Ctx::vcycle(int l) {
    Level& L = lev[l];
    const double* pre_norm = (l == 0) ? scal + kSlotR64 * kMaxCh : scal + l * kMaxCh;
    unsigned long long* it = (l == 0) ? counters + kCntLocal : nullptr;
    if (l == nlev_run - 1) {
        oras(l, true, nullptr, L.xa, pre_norm, true, it);
        if (l == 0) ++vcycles_run;
        return;
    }
    const int npre = (l == 0) ? (int)p.fine_pre : 1;
    const int npost = (l == 0) ? (int)p.fine_post : 1;
    // pre-smoothing: the first sweep starts from x = 0
    if (npre > 0) {
        oras(l, true, nullptr, L.xa, pre_norm, false, it);
        for (int i = 1; i < npre; ++i) {
            residual_norm_level(l, L.xa, l);
            oras(l, false, L.xa, L.xb, scal + l * kMaxCh, false, it);
            std::swap(L.xa, L.xb);
        }
    } else {
        cudaMemsetAsync(L.xa, 0, (size_t)nch * L.cs * 4, stream);
    }
    Level& C = lev[l + 1];
    {
        const int qr = qrows(L.H, L.W, nch);
        dim3 blk(128), grd = quad_grid(L.H, L.W, nch, qr);
        // read x, b and the mask bits, write a quarter value of b_H per value
        if (l == 0) tstart(kT_Restrict, 9.125 * (double)nch * L.H * L.W);
        launch_ks(p.pdl >= 0.5, l == 0 ? stage_bytes(2, RStage::bytes) : 0, k_restrict_residual, grd, blk, stream,
                  arr(l), mview(l), (const float*)L.xa,
                 (const float*)L.b, arr(l + 1), mview(l + 1), C.b, reducer(l + 1, grd.x * grd.y), qr);
        ++launches;
        if (l == 0) tstop();
    }
    // the levels below the finest as one timed block per V-cycle
    if (l == 0) tstart(kT_Coarse);
    vcycle(l + 1);
    if (l == 0) tstop();
    {
        const int qr = qrows(L.H, L.W, nch);
        dim3 grd = quad_grid(L.H, L.W, nch, qr), blk(128);
        // read x, b, a quarter value of e_H and the mask bits, write x
        if (l == 0) tstart(kT_Prolong, 13.125 * (double)nch * L.H * L.W);
        launch_k(p.pdl >= 0.5, k_prolong<0>, grd, blk, stream, arr(l), mview(l), (const float*)L.xa,
                 (const float*)L.b, L.xb, arr(l + 1), (const float*)C.xa, reducer(l, grd.x * grd.y), qr);
        ++launches;
        if (l == 0) tstop();
    }
    // x now in xb; post-smoothing sweeps alternate xb -> xa -> xb ...
    float* cur = L.xb;
    float* other = L.xa;
    for (int i = 0; i < npost; ++i) {
        if (i > 0) residual_norm_level(l, cur, l);
        oras(l, false, cur, other, scal + l * kMaxCh, false, it);
        std::swap(cur, other);
    }
    if (cur != L.xa) std::swap(L.xa, L.xb);   // result must end in xa
    if (l == 0) ++vcycles_run;
}

// ||b_l - A_l x||^2 per channel into slot `slot` (prolongation kernel with a
// zero coarse correction is not available, so reuse k_prolong<0> with the
// coarse level's zero-filled scratch is avoided: a plain residual pass).
void Ctx::residual_norm_level(int l, const float* x, int slot) {
    const Level& L = lev[l];
    const int qr = qrows(L.H, L.W, nch);
    dim3 grd = quad_grid(L.H, L.W, nch, qr), blk(128);
    launch_k(p.pdl >= 0.5, k_level_residual_norm, grd, blk, stream, arr(l), mview(l), x, (const float*)L.b,
             reducer(slot, grd.x * grd.y), qr);
    ++launches;
}

// Reduced full multigrid (Sec. 3.2, Fig. "multigrid_reduced"): data pyramid,
// coarsest solve, then one ORAS sweep per finer level after prolongation.
// `d` is the level-0 Dirichlet data in FP64. Result (FP32) in lev[0].xa.
void Ctx::fmg(DFc d) {
    {
        dim3 grd((W + 127) / 128, H, nch);
        k_data_to_f32<<<grd, 128, 0, stream>>>(d, arr(0), mview(0), lev[0].b);
        ++launches;
    }
    for (int l = 1; l < nlev_run; ++l) {
        dim3 blk(32, 8), grd((lev[l].W + 31) / 32, (lev[l].H + 7) / 8, nch);
        k_restrict_data<<<grd, blk, 0, stream>>>(arr(l - 1), mview(l - 1), lev[l - 1].b, arr(l), lev[l].b);
        ++launches;
    }
    const int L = nlev_run - 1;
    {
        const int qr = qrows(lev[L].H, lev[L].W, nch);
        dim3 grd = quad_grid(lev[L].H, lev[L].W, nch, qr), blk(128);
        k_prolong<2><<<grd, blk, 0, stream>>>(arr(L), mview(L), nullptr, lev[L].b, lev[L].xb, arr(L), nullptr,
                                              reducer(L, grd.x * grd.y), qr);
        ++launches;
        oras(L, false, lev[L].xb, lev[L].xa, scal + L * kMaxCh, true, nullptr);
    }
    for (int l = L - 1; l >= 0; --l) {
        const int qr = qrows(lev[l].H, lev[l].W, nch);
        dim3 grd = quad_grid(lev[l].H, lev[l].W, nch, qr), blk(128);
        k_prolong<1><<<grd, blk, 0, stream>>>(arr(l), mview(l), nullptr, lev[l].b, lev[l].xb, arr(l + 1),
                                              lev[l + 1].xa, reducer(l, grd.x * grd.y), qr);
        ++launches;
        oras(l, false, lev[l].xb, lev[l].xa, scal + l * kMaxCh, l == L, l == 0 ? counters + kCntLocal : nullptr);
    }
}

template <int RHS, int INIT, bool P32 = false>
static void launch_res(Ctx& c, DFc uin, DF uout, const float* x32, DFc d, DFc y, bool want_b) {
    ResArgs a;
    a.F = c.arr(0);
    a.m = c.mview(0);
    a.uin = uin;
    a.uout = uout;
    a.x32 = x32;
    a.d = d;
    a.y = y;
    a.r32 = c.lev[0].b;
    a.rows = c.qrows(c.H, c.W, c.nch);
    dim3 grd = quad_grid(c.H, c.W, c.nch, a.rows), blk(128);
    a.red_r = c.reducer(kSlotR64, grd.x * grd.y);
    a.red_b = c.reducer(kSlotB64, grd.x * grd.y);
    a.want_b = want_b ? 1 : 0;
    a.d_lo_zero = (c.f_lo_zero && d.lo == c.dfv[kF].lo) ? 1 : 0;
    // algorithmic bytes per value: write u (double-float) and r (FP32), read
    // the mask bits, u, e, the source terms d and y as the variant needs them
    // (the data that INIT_KEEP / FROM32 / ZERO take on known pixels only is
    // not counted)
    constexpr bool HAS_U = (INIT == INIT_KEEP || INIT == INIT_UPDATE);
    constexpr bool HAS_E = (INIT == INIT_UPDATE || INIT == INIT_FROM32);
    // INIT_KEEP rewrites only the known pixels of u in place
    const double known = c.mask_ones > 0 ? std::min(1.0, (double)c.mask_ones / ((double)c.H * c.W)) : 0.0;
    // (the plain FP32 form moves 4-byte iterates: 4 B less per read and write of u)
    const double uw = P32 ? 4.0 : 8.0;
    const double bpv = 4.125 + uw - (INIT == INIT_KEEP ? uw * (1.0 - known) : 0.0) + (HAS_U ? uw : 0.0) +
                       (HAS_E ? 4.0 : 0.0) +
                       (RHS == RHS_SOURCE ? (a.d_lo_zero ? 4.0 : 8.0) + (y.hi ? 8.0 : 0.0) : 0.0);
    c.tstart(kT_Residual, bpv * (double)c.nch * c.H * c.W);
    const size_t stg = c.stage_bytes(1, ResStage<RHS, INIT, P32>::bytes);
    launch_ks(c.p.pdl >= 0.5, stg, k_residual_df<RHS, INIT, P32>, grd, blk, c.stream, a);
    ++c.launches;
    c.tstop();
}

void Ctx::residual(int rhs, int init, DFc uin, DF uout, const float* x32, DFc d, DFc y, bool want_b, bool p32) {
    if (p32 && rhs == RHS_DATA) {   // plain FP32 form (inpainting only)
#define HDI_RES32(I) \
    if (init == I) { launch_res<RHS_DATA, I, true>(*this, uin, uout, x32, d, y, want_b); return; }
        HDI_RES32(INIT_KEEP) HDI_RES32(INIT_UPDATE) HDI_RES32(INIT_FROM32) HDI_RES32(INIT_ZERO)
#undef HDI_RES32
    }
#define HDI_RES(R, I) \
    if (rhs == R && init == I) { launch_res<R, I>(*this, uin, uout, x32, d, y, want_b); return; }
    HDI_RES(RHS_DATA, INIT_KEEP) HDI_RES(RHS_DATA, INIT_UPDATE) HDI_RES(RHS_DATA, INIT_FROM32)
    HDI_RES(RHS_DATA, INIT_ZERO) HDI_RES(RHS_SOURCE, INIT_KEEP) HDI_RES(RHS_SOURCE, INIT_UPDATE)
    HDI_RES(RHS_SOURCE, INIT_FROM32) HDI_RES(RHS_SOURCE, INIT_ZERO)
#undef HDI_RES
}

// Solves A u = b on level 0 with iterative refinement in FP64 (pattern:
// FP32 V-cycles on the correction, FP64 residual and update).
//   spec.u[0/1]  : ping-pong FP64 buffers; spec.cur selects the one holding
//                  the iterate on entry (warm) and receives it on exit.
//   spec.rhs     : RHS_DATA (b = C d) or RHS_SOURCE (b = (I-C)(d - y)).
//   spec.start   : START_FMG, START_WARM (iterate in u[cur]) or START_ZERO.
//   spec.tol     : relative residual per channel; spec.bnorm2 receives ||b||^2.
int Ctx::solve(SolveSpec& s) {
    int rc;
    DF* ub = s.u;
    int cur = s.cur;
    const DFc none{nullptr, nullptr};
    const bool p32 = s.plain32 && s.rhs == RHS_DATA;
    if (s.start == START_FMG) {
        fmg(s.d);
        residual(s.rhs, INIT_FROM32, none, ub[cur], lev[0].xa, s.d, s.y, true, p32);
    } else if (s.start == START_WARM) {
        residual(s.rhs, INIT_KEEP, cview(ub[cur]), ub[cur], nullptr, s.d, s.y, true, p32);   // in place
    } else {
        residual(s.rhs, INIT_ZERO, none, ub[cur], nullptr, s.d, s.y, true, p32);
    }
    double r2[kMaxCh], b2[kMaxCh];
    s.iterations = 0;
    double prev_worst = INFINITY;
    // the plain FP32 form keeps no low words: they are zeroed when the solve
    // returns, so that readers of the double-float pair see the FP32 iterate
    struct ZeroLo {
        Ctx& c;
        const SolveSpec& s;
        const int& cur;
        bool on;
        ~ZeroLo() {
            if (on) cudaMemsetAsync(s.u[cur].lo, 0, (size_t)c.nch * c.lev[0].cs * 4, c.stream);
        }
    } zero_lo{*this, s, cur, p32};
    for (;;) {
        cudaMemcpyAsync(hscal, scal + kSlotR64 * kMaxCh, (size_t)nch * 8, cudaMemcpyDeviceToHost, stream);
        cudaMemcpyAsync(hscal + kMaxCh, scal + kSlotB64 * kMaxCh, (size_t)nch * 8, cudaMemcpyDeviceToHost, stream);
        if ((rc = sync("inpainting residual"))) return rc;
        double worst = 0.0;
        for (int c = 0; c < nch; ++c) {
            r2[c] = hscal[c];
            b2[c] = hscal[kMaxCh + c];
            if (!std::isfinite(r2[c])) {
                s.cur = cur;
                return fail(HDI_ERR_NONFINITE, "non-finite residual in channel %d", c);
            }
            const double rel = b2[c] > 0 ? std::sqrt(r2[c] / b2[c]) : (r2[c] > 0 ? INFINITY : 0.0);
            s.rel[c] = rel;
            worst = std::max(worst, rel);
        }
        s.rel_max = worst;
        for (int c = 0; c < nch; ++c) s.bnorm2[c] = b2[c];
        if (worst <= s.tol) break;
        // the plain FP32 form stalls at its rounding level: stop once a
        // V-cycle gains less than 10%
        if (s.iterations >= s.max_iter || (p32 && worst > 0.9 * prev_worst)) {
            s.cur = cur;
            return HDI_ERR_NOT_CONVERGED;
        }
        prev_worst = worst;
        vcycle(0);
        residual(s.rhs, INIT_UPDATE, cview(ub[cur]), ub[1 - cur], lev[0].xa, s.d, s.y, false, p32);
        cur = 1 - cur;
        ++s.iterations;
        // ||b||^2 is unchanged; keep the slot value from the first evaluation.
    }
    s.cur = cur;
    return HDI_OK;
}

// --------------------------------------------------------- input checks ---

int Ctx::check_image(const hdi_image* im, const char* name, int H_, int W_, int nch_) {
    if (!im || !im->data) return fail(HDI_ERR_INVALID_ARG, "%s: null image", name);
    if (im->dtype != HDI_F32 && im->dtype != HDI_F64) return fail(HDI_ERR_INVALID_ARG, "%s: bad dtype", name);
    if (im->location != HDI_DEVICE && im->location != HDI_HOST)
        return fail(HDI_ERR_INVALID_ARG, "%s: bad location", name);
    if (im->height <= 0 || im->width <= 0 || im->channels <= 0 || im->channels > 4)
        return fail(HDI_ERR_INVALID_ARG, "%s: bad shape %dx%dx%d (1..4 channels)", name, im->height, im->width,
                    im->channels);
    if (H_ >= 0 && (im->height != H_ || im->width != W_ || im->channels != nch_))
        return fail(HDI_ERR_INVALID_ARG, "%s: shape %dx%dx%d does not match %dx%dx%d", name, im->height, im->width,
                    im->channels, H_, W_, nch_);
    if (im->row_stride < im->width || (im->channels > 1 && im->channel_stride < im->row_stride * im->height))
        return fail(HDI_ERR_INVALID_ARG, "%s: strides too small", name);
    return HDI_OK;
}

// Copies a caller image into the internal FP64 layout (device or host source).
// A host image's copy into `stage` on the side stream, ordered after the
// context stream's earlier use of `stage`; load_image(..., prestaged = true)
// then converts it on the context stream once the copy has landed. Kernels
// the context stream runs in between overlap the copy.
int Ctx::upload_begin(const hdi_image* im) {
    if (im->location != HDI_HOST) return HDI_OK;
    if (!ustream) {
        if (cudaStreamCreateWithFlags(&ustream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&uev[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&uev[1], cudaEventDisableTiming) != cudaSuccess)
            return cuda_check(cudaGetLastError(), "upload stream");
    }
    const size_t es = im->dtype == HDI_F64 ? 8 : 4;
    const size_t n = (size_t)nch * H * W * es;
    int rc = stage.reserve(*this, std::max(stage.cap, n + (size_t)H * W + 1024), "staging buffer");
    if (rc) return rc;
    cudaEventRecord(uev[0], stream);
    cudaStreamWaitEvent(ustream, uev[0], 0);
    char* st = (char*)stage.base;
    for (int c = 0; c < im->channels; ++c) {
        cudaError_t e = cudaMemcpy2DAsync(st + (size_t)c * H * W * es, W * es,
                                          (const char*)im->data + (size_t)c * im->channel_stride * es,
                                          im->row_stride * es, W * es, H, cudaMemcpyHostToDevice, ustream);
        if (e != cudaSuccess) return cuda_check(e, "host-to-device copy");
    }
    cudaEventRecord(uev[1], ustream);
    return cuda_check(cudaGetLastError(), "image upload");
}

int Ctx::load_image(const hdi_image* im, DF dst, float* lo2, int c0, bool wait, bool prestaged) {
    const int nc = im->channels;
    if (dst.hi == dfv[kF].hi && im->dtype == HDI_F64) f_lo_zero = false;   // callers set it before loading f
    if (c0) {
        const long long off = (long long)c0 * lev[0].cs;
        dst.hi += off;
        dst.lo += off;
        if (lo2) lo2 += off;
    }
    const void* src = im->data;
    long long rs = im->row_stride, cs = im->channel_stride;
    const size_t es = im->dtype == HDI_F64 ? 8 : 4;
    if (im->location == HDI_HOST) {
        const size_t n = (size_t)nch * H * W * es;
        char* st;
        if (prestaged) {   // upload_begin copied it; wait for the copy
            st = (char*)stage.base;
            cudaStreamWaitEvent(stream, uev[1], 0);
        } else {
            // a side-stream upload into `stage` (one a failed call left behind) lands first
            if (ustream) cudaStreamWaitEvent(stream, uev[1], 0);
            int rc = stage.reserve(*this, std::max(stage.cap, n + (size_t)H * W + 1024), "staging buffer");
            if (rc) return rc;
            st = (char*)stage.base;
            for (int c = 0; c < nc; ++c) {
                cudaError_t e = cudaMemcpy2DAsync(st + (size_t)c * H * W * es, W * es,
                                                  (const char*)src + (size_t)c * cs * es, rs * es, W * es, H,
                                                  cudaMemcpyHostToDevice, stream);
                if (e != cudaSuccess) return cuda_check(e, "host-to-device copy");
            }
        }
        src = st;
        rs = W;
        cs = (long long)H * W;
    }
    // flag word 1 (word 0 is the mask check's): non-finite input
    cudaMemsetAsync(flags + 1, 0, 4, stream);
    dim3 grd((W + 127) / 128, H, nc);
    if (im->dtype == HDI_F64)
        k_load_image<double><<<grd, 128, 0, stream>>>((const double*)src, rs, cs, arr(0), dst, lo2, flags + 1);
    else
        k_load_image<float><<<grd, 128, 0, stream>>>((const float*)src, rs, cs, arr(0), dst, lo2, flags + 1);
    ++launches;
    if (!wait) return cuda_check(cudaGetLastError(), "image upload");   // checked by load_checks
    unsigned bad = 0;
    cudaMemcpyAsync(&bad, flags + 1, 4, cudaMemcpyDeviceToHost, stream);
    int rc = sync("image upload");
    if (rc) return rc;
    if (bad) return fail(HDI_ERR_NONFINITE, "non-finite value in input image");
    return HDI_OK;
}

int Ctx::store_image(DFc src, hdi_image* im, bool zero_off_mask, const float* known_lo2, int c0, bool wait) {
    const int nc = im->channels;
    if (c0) {
        const long long off = (long long)c0 * lev[0].cs;
        src.hi += off;
        src.lo += off;
        if (known_lo2) known_lo2 += off;
    }
    void* dst = im->data;
    long long rs = im->row_stride, cs = im->channel_stride;
    const size_t es = im->dtype == HDI_F64 ? 8 : 4;
    const bool host = im->location == HDI_HOST;
    if (host) {
        const size_t n = (size_t)nch * H * W * es;
        int rc = stage.reserve(*this, std::max(stage.cap, n + (size_t)H * W + 1024), "staging buffer");
        if (rc) return rc;
        dst = stage.base;
        rs = W;
        cs = (long long)H * W;
    }
    dim3 grd((W + 127) / 128, H, nc);
    if (im->dtype == HDI_F64)
        k_store_image<double><<<grd, 128, 0, stream>>>(src, arr(0), mview(0), zero_off_mask, known_lo2, (double*)dst,
                                                       rs, cs, c0);
    else
        k_store_image<float><<<grd, 128, 0, stream>>>(src, arr(0), mview(0), zero_off_mask, known_lo2, (float*)dst,
                                                      rs, cs, c0);
    ++launches;
    if (host) {
        for (int c = 0; c < nc; ++c) {
            cudaError_t e = cudaMemcpy2DAsync((char*)im->data + (size_t)c * im->channel_stride * es,
                                              im->row_stride * es, (const char*)dst + (size_t)c * H * W * es, W * es,
                                              W * es, H, cudaMemcpyDeviceToHost, stream);
            if (e != cudaSuccess) return cuda_check(e, "device-to-host copy");
        }
    }
    if (!wait) return cuda_check(cudaGetLastError(), "image download");
    return sync("image download");
}

// Uploads and bit-packs the mask, builds the mask pyramid; returns the number
// of known pixels in *ones.
int Ctx::load_mask(const hdi_mask* m, long long* ones, int plane, bool pyramid, bool wait) {
    if (!m || !m->data) return fail(HDI_ERR_INVALID_ARG, "mask: null");
    if (m->height != H || m->width != W) return fail(HDI_ERR_INVALID_ARG, "mask: shape does not match the image");
    if (m->row_stride < m->width) return fail(HDI_ERR_INVALID_ARG, "mask: row stride too small");
    if (m->location != HDI_DEVICE && m->location != HDI_HOST) return fail(HDI_ERR_INVALID_ARG, "mask: bad location");
    const uint8_t* src = m->data;
    long long rs = m->row_stride;
    if (m->location == HDI_HOST) {
        const size_t need = (size_t)nch * H * W * 8 + (size_t)H * W + 1024;
        int rc = stage.reserve(*this, std::max(stage.cap, need), "staging buffer");
        if (rc) return rc;
        uint8_t* st = (uint8_t*)stage.base + (size_t)nch * H * W * 8;
        cudaError_t e = cudaMemcpy2DAsync(st, W, m->data, m->row_stride, W, H, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return cuda_check(e, "mask upload");
        src = st;
        rs = W;
    }
    cudaMemsetAsync(counters + kCntOnes, 0, 8, stream);
    cudaMemsetAsync(flags, 0, 4, stream);
    const Level& L = lev[0];
    dim3 grd((L.wp + 63) / 64, H);
    k_pack_mask<<<grd, 64, 0, stream>>>(src, rs, H, W, L.bits + (size_t)plane * L.H * L.wp, L.wp, counters + kCntOnes,
                                        flags);
    ++launches;
    if (pyramid) build_mask_pyramid();
    if (!wait) return cuda_check(cudaGetLastError(), "mask upload");   // checked by load_checks
    LoadReadback rb;
    enqueue_load_readback(&rb);
    int rc = sync("mask upload");
    if (rc) return rc;
    if (rb.flags[0]) return fail(HDI_ERR_INVALID_ARG, "mask: values must be 0 or 1");
    *ones = (long long)rb.counters[kCntOnes];
    mask_ones = *ones;
    if (pyramid) set_levels_run(rb.counters + kCntLevelKnown);
    return HDI_OK;
}

// The counters and flags the input checks leave on the device, copied to
// `rb` (pinned or not) on the context's stream.
void Ctx::enqueue_load_readback(LoadReadback* rb) {
    cudaMemcpyAsync(rb->counters, counters, sizeof(rb->counters), cudaMemcpyDeviceToHost, stream);
    cudaMemcpyAsync(rb->flags, flags, sizeof(rb->flags), cudaMemcpyDeviceToHost, stream);
}

// A level whose pixels are all known (every plane) has the exact coarse
// correction 0, and so has every level below it: the solves stop their
// hierarchy there (the level itself stays as the trivial coarsest level).
void Ctx::set_levels_run(const unsigned long long* known) {
    nlev_run = nlev;
    for (int l = 1; l < nlev && p.mg_truncate >= 0.5; ++l)
        if (known[l] == (unsigned long long)nmask * lev[l].H * lev[l].W) {
            nlev_run = l + 1;
            break;
        }
}

// The checks of a load_mask + load_image pair enqueued with wait = false,
// from their readback (after the stream has reached it).
int Ctx::load_checks(const LoadReadback& rb, long long* ones) {
    if (rb.flags[0]) return fail(HDI_ERR_INVALID_ARG, "mask: values must be 0 or 1");
    if (rb.flags[1]) return fail(HDI_ERR_NONFINITE, "non-finite value in input image");
    *ones = (long long)rb.counters[kCntOnes];
    mask_ones = *ones;
    set_levels_run(rb.counters + kCntLevelKnown);
    return HDI_OK;
}

// Flat JSON object of parameter values, {"name": number, ...}, applied on
// top of the defaults; false on a syntax error, an unknown name or a value
// outside the parameter's range.
static bool parse_config(const char* js, Params& out) {
    const char* q = js;
    auto ws = [&]() { while (*q == ' ' || *q == '\t' || *q == '\n' || *q == '\r') ++q; };
    ws();
    if (*q++ != '{') return false;
    ws();
    if (*q == '}') { ++q; ws(); return *q == 0; }
    for (;;) {
        ws();
        if (*q++ != '"') return false;
        const char* k0 = q;
        while (*q && *q != '"') ++q;
        if (*q != '"') return false;
        const std::string key(k0, q - k0);
        ++q;
        ws();
        if (*q++ != ':') return false;
        ws();
        char* end = nullptr;
        const double v = strtod(q, &end);
        if (end == q) return false;
        q = end;
        bool found = false;
        for (const auto& d : kParams) {
            if (key == d.name) {
                if (!(v >= d.lo && v <= d.hi)) return false;
                out.*(d.field) = v;
                found = true;
                break;
            }
        }
        if (!found) return false;
        ws();
        if (*q == ',') { ++q; continue; }
        if (*q++ != '}') return false;
        ws();
        return *q == 0;
    }
}

// ------------------------------------------------------------ C ABI ---

extern "C" {

int hdi_create(hdi_ctx** out, int device, void* stream, const char* config_json) {
    if (!out) return HDI_ERR_INVALID_ARG;
    *out = nullptr;
    Params cfg;
    if (config_json && !parse_config(config_json, cfg)) return HDI_ERR_INVALID_ARG;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return HDI_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return HDI_ERR_CUDA;
    Ctx* c = new Ctx();
    c->device = device;
    c->stream = (cudaStream_t)stream;
    if (cudaMallocHost(&c->hscal, 2 * kMaxCh * 8) != cudaSuccess) {
        delete c;
        return HDI_ERR_CUDA;
    }
    if (cudaMalloc(&c->flags, 256 + kMaxCh * 4) != cudaSuccess) {
        cudaFreeHost(c->hscal);
        delete c;
        return HDI_ERR_CUDA;
    }
    c->d_chmask = (int*)((char*)c->flags + 256);
    c->p = cfg;
    *out = reinterpret_cast<hdi_ctx*>(c);
    return HDI_OK;
}

int hdi_destroy(hdi_ctx* h) {
    if (!h) return HDI_OK;
    Ctx* c = reinterpret_cast<Ctx*>(h);
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    c->ws.release();
    c->tws.release();
    c->dws.release();
    c->vws.release();
    c->lws.release();
    if (c->ustream) cudaStreamSynchronize(c->ustream);
    c->stage.release();
    engine_delete(c->eng);
    if (c->ustream) cudaStreamDestroy(c->ustream);
    for (cudaEvent_t e : c->uev)
        if (e) cudaEventDestroy(e);
    if (c->flags) cudaFree(c->flags);
    if (c->tev) {
        for (int i = 0; i < 2 * kMaxTimed; ++i) cudaEventDestroy(c->tev[i]);
        delete[] c->tev;
    }
    if (c->hscal) cudaFreeHost(c->hscal);
    delete c;
    return HDI_OK;
}

int hdi_set_param(hdi_ctx* h, const char* name, double v) {
    if (!h || !name) return HDI_ERR_INVALID_ARG;
    Ctx* c = reinterpret_cast<Ctx*>(h);
    for (const auto& d : kParams) {
        if (!strcmp(d.name, name)) {
            if (!(v >= d.lo && v <= d.hi))
                return c->fail(HDI_ERR_INVALID_ARG, "%s=%g outside [%g, %g]", name, v, d.lo, d.hi);
            c->p.*(d.field) = v;
            return HDI_OK;
        }
    }
    return c->fail(HDI_ERR_INVALID_ARG, "unknown parameter '%s'", name);
}

int hdi_get_param(const hdi_ctx* h, const char* name, double* v) {
    if (!h || !name || !v) return HDI_ERR_INVALID_ARG;
    const Ctx* c = reinterpret_cast<const Ctx*>(h);
    for (const auto& d : kParams) {
        if (!strcmp(d.name, name)) {
            *v = c->p.*(d.field);
            return HDI_OK;
        }
    }
    return HDI_ERR_INVALID_ARG;
}

const char* hdi_last_error(const hdi_ctx* h) {
    if (!h) return "null context";
    return reinterpret_cast<const Ctx*>(h)->err.c_str();
}

const char* hdi_version(void) { return "hdi 0.1 (sm_103a)"; }

int64_t hdi_workspace_bytes(const hdi_ctx* h) {
    if (!h) return -1;
    const Ctx* c = reinterpret_cast<const Ctx*>(h);
    return (int64_t)c->other_bytes() + (c->eng ? (int64_t)engine_used_bytes(c->eng) : 0);
}

int64_t hdi_launch_count(const hdi_ctx* h) {
    if (!h) return -1;
    return reinterpret_cast<const Ctx*>(h)->launches;
}

const char* hdi_timing_name(int i) {
    static const char* names[HDI_TIMING_CLASSES] = {"oras_fine", "residual_fine", "prolong_fine", "restrict_fine",
                                                    "tonal_echo", "tonal_gram", "tonal_local", "anderson",
                                                    "coarse_levels"};
    return (i >= 0 && i < HDI_TIMING_CLASSES) ? names[i] : "";
}

int hdi_timing(hdi_ctx* h, int enable, int reset, double* ms, int64_t* launches) {
    if (!h) return HDI_ERR_INVALID_ARG;
    Ctx* c = reinterpret_cast<Ctx*>(h);
    int rc = c->tflush();
    if (rc) return rc;
    if (ms)
        for (int i = 0; i < HDI_TIMING_CLASSES; ++i) ms[i] = c->ttot[i];
    if (launches)
        for (int i = 0; i < HDI_TIMING_CLASSES; ++i) launches[i] = c->tcnt[i];
    if (reset)
        for (int i = 0; i < HDI_TIMING_CLASSES; ++i) { c->ttot[i] = 0.0; c->tcnt[i] = 0; c->tbytes[i] = 0.0; }
    if (enable && !c->tev) {
        c->tev = new cudaEvent_t[2 * kMaxTimed];
        for (int i = 0; i < 2 * kMaxTimed; ++i) cudaEventCreate(&c->tev[i]);
    }
    c->timing = enable != 0;
    return HDI_OK;
}

int hdi_timing_bytes(hdi_ctx* h, double* bytes) {
    if (!h || !bytes) return HDI_ERR_INVALID_ARG;
    Ctx* c = reinterpret_cast<Ctx*>(h);
    int rc = c->tflush();
    if (rc) return rc;
    for (int i = 0; i < HDI_TIMING_CLASSES; ++i) bytes[i] = c->tbytes[i];
    return HDI_OK;
}

int hdi_inpaint(hdi_ctx* h, const hdi_image* f, const hdi_mask* mask, const hdi_image* u0, hdi_image* u, double tol,
                hdi_stats* st) {
    if (!h) return HDI_ERR_INVALID_ARG;
    Ctx* c = reinterpret_cast<Ctx*>(h);
    auto t0 = std::chrono::steady_clock::now();
    c->err.clear();
    int rc = c->inpaint(f, mask, u0, u, tol, st);
    if (st) {
        st->status = rc;
        st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return rc;
}

int hdi_tonal_opt(hdi_ctx* h, const hdi_image* f, const hdi_mask* mask, const hdi_image* g0, hdi_image* g,
                  double tol, hdi_stats* st) {
    if (!h) return HDI_ERR_INVALID_ARG;
    Ctx* c = reinterpret_cast<Ctx*>(h);
    auto t0 = std::chrono::steady_clock::now();
    c->err.clear();
    int rc = c->tonal(f, mask, g0, g, tol, st);
    if (st) {
        st->status = rc;
        st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return rc;
}

int hdi_densify_step(hdi_ctx* h, const hdi_image* f, hdi_mask* mask, const hdi_image* u, int64_t k, uint64_t seed,
                     int64_t* added) {
    if (!h) return HDI_ERR_INVALID_ARG;
    Ctx* c = reinterpret_cast<Ctx*>(h);
    c->err.clear();
    return c->densify(f, mask, u, k, seed, added);
}

int hdi_densify(hdi_ctx* h, const hdi_image* f, hdi_mask* mask, hdi_image* u, int32_t n, double t, double density,
                uint64_t seed, int64_t* sizes) {
    if (!h) return HDI_ERR_INVALID_ARG;
    Ctx* c = reinterpret_cast<Ctx*>(h);
    c->err.clear();
    return c->densify_run(f, mask, u, n, t, density, seed, sizes);
}

}  // extern "C"

// ------------------------------------------------------- densification ---

// Cumulative mask sizes after each of n iterations whose additions grow by the
// factor t and sum to `total` (Sec. 4.2): floor(total * (t^i - 1) / (t^n - 1)
// + 0.5), i / n for t = 1; the last target is total itself.
static void densify_targets(long long total, int n, double t, std::vector<long long>& out) {
    out.resize(n);
    for (int i = 1; i <= n; ++i) {
        const double frac = (t == 1.0) ? (double)i / n : (std::pow(t, i) - 1.0) / (std::pow(t, n) - 1.0);
        out[i - 1] = (long long)std::floor((double)total * frac + 0.5);
    }
    out[n - 1] = total;
}

// The densification loop (Sec. 4, Alg. 1 with the initial mask and growth
// factor of Sec. 4.2): n iterations, each a densification step to the next
// cumulative target followed by an inpainting warm-started from the previous
// one. With jump flooding, every step after the first starts at the power of
// two covering the previous labels' largest pixel-to-site distance.
int Ctx::densify_run(const hdi_image* f, hdi_mask* mask, hdi_image* u, int n, double t, double density,
                     uint64_t seed, int64_t* sizes) {
    int rc;
    if (!f || !mask || !u) return fail(HDI_ERR_INVALID_ARG, "densify: f, mask and u are required");
    if (n < 1) return fail(HDI_ERR_INVALID_ARG, "densify: n must be >= 1");
    if (!(t > 0.0) || !std::isfinite(t)) return fail(HDI_ERR_INVALID_ARG, "densify: t must be positive");
    if (!(density > 0.0 && density <= 1.0)) return fail(HDI_ERR_INVALID_ARG, "densify: density must lie in (0, 1]");
    if ((rc = check_image(f, "f", -1, 0, 0))) return rc;
    if ((rc = check_image(u, "u", f->height, f->width, f->channels))) return rc;
    const long long total = (long long)std::floor(density * (double)f->height * f->width + 0.5);
    std::vector<long long> target;
    densify_targets(total, n, t, target);
    if ((rc = setup(f->height, f->width, f->channels))) return rc;
    long long ones = 0;
    if ((rc = load_mask(mask, &ones))) return rc;
    const bool jfa = p.densify_voronoi >= 0.5;
    const double keep_first = p.jfa_first_step;
    int first = 0;   // full schedule until a label map has given a bound
    for (int i = 0; i < n; ++i) {
        const long long k = std::max(target[i] - ones, 0LL);
        int64_t added = 0;
        if (jfa) p.jfa_first_step = first;
        rc = densify(f, mask, ones > 0 ? u : nullptr, k, seed, &added);
        p.jfa_first_step = keep_first;
        if (rc) return rc;
        if (jfa && ones > 0) {
            int b = 1;
            while ((long long)b * b < last_label_maxd2) b *= 2;
            first = b;
        }
        ones += added;
        if (ones == 0) return fail(HDI_ERR_EMPTY_MASK, "densify: the initial mask came out empty");
        hdi_stats st;
        rc = inpaint(f, mask, ones > added ? u : nullptr, u, p.densify_tol, &st);
        if (rc != HDI_OK && rc != HDI_ERR_NOT_CONVERGED) return rc;
        if (sizes) sizes[i] = ones;
    }
    return HDI_OK;
}

// ------------------------------------------------------------ batch ---

#include "engine.cuh"

// Images of one size class are stacked as the channels of one system (each
// channel reads its own image's mask plane), so every phase of the solver is
// one launch over all their subdomains and pixels. Size classes run in turn.
int Ctx::inpaint_batch(int n, const hdi_image* f, const hdi_mask* m, hdi_image* u, double tol, hdi_stats* st) {
    int rc;
    if ((rc = cuda_check(cudaSetDevice(device), "cudaSetDevice"))) return rc;
    if (n < 0 || (n > 0 && (!f || !m || !u))) return fail(HDI_ERR_INVALID_ARG, "batch: null arrays");
    if (!(tol > 0.0 && tol < 1.0)) return fail(HDI_ERR_INVALID_ARG, "tol must lie in (0, 1)");
    for (int i = 0; i < n; ++i) {
        if ((rc = check_image(&f[i], "f[i]", -1, 0, 0))) return rc;
        if ((rc = check_image(&u[i], "u[i]", f[i].height, f[i].width, f[i].channels))) return rc;
        if (u[i].dtype != f[i].dtype) return fail(HDI_ERR_INVALID_ARG, "u[%d]: dtype differs from f", i);
        if (m[i].height != f[i].height || m[i].width != f[i].width)
            return fail(HDI_ERR_INVALID_ARG, "mask[%d]: shape does not match", i);
    }
    if (p.batch_engine >= 0.5 && p.inpaint_fp32 < 0.5) return inpaint_batch_engine(n, f, m, u, tol, st);
    return inpaint_batch_classes(n, f, m, u, tol, st);
}

// All images through the batched engine (engine.cuh): admitted as the
// budget allows, stepped together, each leaving when it converges.
int Ctx::inpaint_batch_engine(int n, const hdi_image* f, const hdi_mask* m, hdi_image* u, double tol, hdi_stats* st) {
    if (!eng) {
        eng = new Engine();
        eng->device = device;
        eng->stream = stream;
    }
    Engine& e = *eng;
    e.p = p;
    e.budget = p.hbm_budget_gb * 1e9;
    std::vector<int64_t> tags(std::max(n, 1));
    std::vector<hdi_stats> sts(std::max(n, 1));
    int next = 0, done = 0, worst = HDI_OK, rc;
    const int64_t l0 = e.launches;
    while (done < n) {
        // every image that fits is loaded without waiting; one wait checks them all
        while (next < n) {
            rc = e.submit_async(&f[next], &m[next], &u[next], tol, next);
            if (rc == HDI_ERR_OUT_OF_MEMORY && !e.reqs.empty()) break;   // admitted when others finish
            if (rc) return fail(rc, "batch image %d: %s", next, e.err.c_str());
            ++next;
        }
        std::vector<std::pair<int64_t, int>> failed;
        if ((rc = e.finalize_loads(&failed))) return fail(rc, "batch: %s", e.err.c_str());
        if (!failed.empty())
            return fail(failed.front().second, "batch image %d: %s", (int)failed.front().first, e.err.c_str());
        int nd = 0;
        if ((rc = e.step(tags.data(), sts.data(), n, &nd))) return fail(rc, "batch: %s", e.err.c_str());
        for (int i = 0; i < nd; ++i) {
            const int idx = (int)tags[i];
            if (st) st[idx] = sts[i];
            if (sts[i].status == HDI_ERR_NOT_CONVERGED) worst = HDI_ERR_NOT_CONVERGED;
            else if (sts[i].status != HDI_OK) return fail(sts[i].status, "batch image %d failed: %s", idx, e.err.c_str());
        }
        done += nd;
    }
    launches += e.launches - l0;
    return worst;
}

// Images of one size form one system (size classes in turn).
int Ctx::inpaint_batch_classes(int n, const hdi_image* f, const hdi_mask* m, hdi_image* u, double tol,
                               hdi_stats* st) {
    int rc;
    // group by size, keeping input order inside a class; split classes above kMaxCh channels
    std::vector<std::vector<int>> groups;
    std::vector<int> done(n, 0);
    for (int i = 0; i < n; ++i) {
        if (done[i]) continue;
        std::vector<int> g;
        int chs = 0;
        for (int j = i; j < n; ++j) {
            if (done[j] || f[j].height != f[i].height || f[j].width != f[i].width) continue;
            if (chs + f[j].channels > kMaxCh) break;
            g.push_back(j);
            chs += f[j].channels;
            done[j] = 1;
        }
        groups.push_back(g);
    }
    int worst = HDI_OK;
    for (const auto& g : groups) {
        int C = 0;
        std::vector<int> chmask, c0s;
        for (size_t j = 0; j < g.size(); ++j) {
            c0s.push_back(C);
            for (int c = 0; c < f[g[j]].channels; ++c) chmask.push_back((int)j);
            C += f[g[j]].channels;
        }
        if ((rc = setup(f[g[0]].height, f[g[0]].width, C, (int)g.size()))) return rc;
        cudaMemcpyAsync(d_chmask, chmask.data(), chmask.size() * 4, cudaMemcpyHostToDevice, stream);
        f_lo_zero = true;
        for (size_t j = 0; j < g.size(); ++j) {
            long long ones = 0;
            if ((rc = load_mask(&m[g[j]], &ones, (int)j, j + 1 == g.size()))) return rc;
            if (ones == 0) return fail(HDI_ERR_EMPTY_MASK, "batch image %d: empty mask", g[j]);
            if ((rc = load_image(&f[g[j]], dfv[kF], flo2, c0s[j]))) return rc;
        }
        SolveSpec s;
        s.u[0] = dfv[kU0];
        s.u[1] = dfv[kU1];
        s.cur = 0;
        s.rhs = RHS_DATA;
        s.d = cview(dfv[kF]);
        s.tol = tol;
        s.max_iter = (int)p.max_vcycles;
        s.start = START_FMG;
        s.plain32 = p.inpaint_fp32 >= 0.5;
        vcycles_run = 0;
        const int src = solve(s);
        if (src != HDI_OK && src != HDI_ERR_NOT_CONVERGED) return src;
        if (src == HDI_ERR_NOT_CONVERGED) worst = src;
        for (size_t j = 0; j < g.size(); ++j) {
            if ((rc = store_image(cview(s.u[s.cur]), &u[g[j]], false, flo2, c0s[j]))) return rc;
            if (st) {
                double rel = 0.0;
                for (int c = 0; c < f[g[j]].channels; ++c) rel = std::max(rel, s.rel[c0s[j] + c]);
                hdi_stats& o = st[g[j]];
                o.status = rel <= tol ? HDI_OK : HDI_ERR_NOT_CONVERGED;
                o.iterations = s.iterations;
                o.vcycles = vcycles_run;
                o.local_iters = 0;
                o.rel_res = rel;
                o.mse = 0.0;
                o.seconds = 0.0;
            }
        }
    }
    if ((rc = tflush())) return rc;
    if (worst != HDI_OK) return fail(worst, "batch: some images did not reach the tolerance");
    return HDI_OK;
}

extern "C" int hdi_inpaint_batch(hdi_ctx* h, int n, const hdi_image* f, const hdi_mask* masks, hdi_image* u, double tol,
                                 hdi_stats* st) {
    if (!h) return HDI_ERR_INVALID_ARG;
    Ctx* c = reinterpret_cast<Ctx*>(h);
    auto t0 = std::chrono::steady_clock::now();
    c->err.clear();
    const int rc = c->inpaint_batch(n, f, masks, u, tol, st);
    if (st) {
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int i = 0; i < n; ++i) st[i].seconds = secs;
    }
    return rc;
}

// ------------------------------------------------------------ inpaint ---

int Ctx::inpaint(const hdi_image* f, const hdi_mask* mask, const hdi_image* u0, hdi_image* u, double tol,
                 hdi_stats* st) {
    int rc;
    if ((rc = cuda_check(cudaSetDevice(device), "cudaSetDevice"))) return rc;
    if ((rc = check_image(f, "f", -1, 0, 0))) return rc;
    if ((rc = check_image(u, "u", f->height, f->width, f->channels))) return rc;
    if (u->dtype != f->dtype) return fail(HDI_ERR_INVALID_ARG, "u: dtype differs from f");
    if (u0 && (rc = check_image(u0, "u0", f->height, f->width, f->channels))) return rc;
    if (!(tol > 0.0 && tol < 1.0)) return fail(HDI_ERR_INVALID_ARG, "tol must lie in (0, 1)");
    if ((rc = setup(f->height, f->width, f->channels))) return rc;
    long long ones = 0;
    if ((rc = load_mask(mask, &ones))) return rc;
    if (ones == 0) return fail(HDI_ERR_EMPTY_MASK, "empty mask: A is singular");
    f_lo_zero = true;
    if ((rc = load_image(f, dfv[kF], flo2))) return rc;
    SolveSpec s;
    s.u[0] = dfv[kU0];
    s.u[1] = dfv[kU1];
    s.cur = 0;
    s.rhs = RHS_DATA;
    s.d = cview(dfv[kF]);
    s.tol = tol;
    s.max_iter = (int)p.max_vcycles;
    s.plain32 = p.inpaint_fp32 >= 0.5;
    if (u0) {
        if ((rc = load_image(u0, s.u[0]))) return rc;
        s.start = START_WARM;
    } else {
        s.start = START_FMG;
    }
    vcycles_run = 0;
    cudaMemsetAsync(counters + kCntLocal, 0, 8, stream);
    const int src = solve(s);
    if (src != HDI_OK && src != HDI_ERR_NOT_CONVERGED) return src;
    if ((rc = store_image(cview(s.u[s.cur]), u, false, flo2))) return rc;
    if (st) {
        unsigned long long li = 0;
        cudaMemcpy(&li, counters + kCntLocal, 8, cudaMemcpyDeviceToHost);
        st->iterations = s.iterations;
        st->vcycles = vcycles_run;
        st->local_iters = (int64_t)li;
        st->rel_res = s.rel_max;
        st->mse = 0.0;
    }
    if ((rc = tflush())) return rc;
    if (src == HDI_ERR_NOT_CONVERGED)
        return fail(HDI_ERR_NOT_CONVERGED, "inpainting: relative residual %.3e after %d refinement steps", s.rel_max,
                    s.iterations);
    return HDI_OK;
}

// ----------------------------------------------- allocation-free inpaint ---
//
// hdi_inpaint_noalloc: the inpainting solve of hdi_inpaint for callers that
// must not allocate device memory (see include/hdi.h). Its whole workspace
// is carved from the file-scope array below; nothing here calls cudaMalloc,
// cudaFree, cudaMallocHost or any other allocating routine.

constexpr size_t kNoAllocBytes = 24u << 20;   // 24 MiB on every GPU that loads the library
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
constexpr int kNoAllocMaxDevices = 64;
// Device address of the scratch, per device (looked up once per device;
// a cudaDeviceReset invalidates it and is not detected).
std::atomic<void*> g_noalloc_ptr[kNoAllocMaxDevices];
// Host mirror of the reduction outputs, one per device: calls on different
// devices read their residual norms into different rows.
double g_noalloc_hscal[kNoAllocMaxDevices][2 * kMaxCh];

// Restores the calling thread's current device when the entry point returns.
struct DeviceRestore {
    int prev = -1;
    DeviceRestore() {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
    }
    ~DeviceRestore() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Carves the inpainting workspace of an H x W x nch image out of `base`
// (the same layout rules as Ctx::setup, restricted to the buffers the
// inpainting solve uses). Returns the bytes needed; carves only if they fit.
size_t noalloc_layout(Ctx& c, char* base, size_t cap, int H_, int W_, int nch_) {
    int sizes[kMaxLevels][2];
    int nl = 0, h = H_, w = W_;
    sizes[nl][0] = h;
    sizes[nl][1] = w;
    ++nl;
    while (std::max(h, w) > 32 && nl < kMaxLevels) {
        h = (h + 1) / 2;
        w = (w + 1) / 2;
        sizes[nl][0] = h;
        sizes[nl][1] = w;
        ++nl;
    }
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        off = (off + 255) & ~(size_t)255;
        char* p = base + off;
        off += bytes;
        return p;
    };
    const bool carve = true;
    int maxparts = 1;
    for (int l = 0; l < nl; ++l) maxparts = std::max(maxparts, reduction_parts(sizes[l][0], sizes[l][1]));
    // first pass: size only
    for (int pass = 0; pass < 2; ++pass) {
        off = 0;
        for (int l = 0; l < nl; ++l) {
            Level& L = c.lev[l];
            const int P = round_up(sizes[l][1], 32);
            const int wp = (sizes[l][1] + 31) / 32 + 1;
            const long long cs = (long long)sizes[l][0] * P;
            char* bits = take((size_t)sizes[l][0] * wp * 4);
            char* xa = take((size_t)nch_ * cs * 4);
            char* xb = take((size_t)nch_ * cs * 4);
            char* b = take((size_t)nch_ * cs * 4);
            if (pass == 1) {
                L.H = sizes[l][0];
                L.W = sizes[l][1];
                L.P = P;
                L.wp = wp;
                L.cs = cs;
                L.bits = (uint32_t*)bits;
                L.xa = (float*)xa;
                L.xb = (float*)xb;
                L.b = (float*)b;
                L.nbx = tile_count(L.W, 32, kOv);
                L.nby = tile_count(L.H, 32, kOv);
            }
        }
        const size_t n32 = (size_t)nch_ * H_ * round_up(W_, 32);
        const int dfs[3] = {kF, kU0, kU1};
        for (int i = 0; i < 3; ++i) {
            char* p = take(n32 * 8);
            if (pass == 1) {
                c.dfv[dfs[i]].hi = (float*)p;
                c.dfv[dfs[i]].lo = (float*)p + n32;
            }
        }
        char* lo2 = take(n32 * 4);
        char* parts = take((size_t)kSlots * maxparts * nch_ * 8);
        char* scal = take((size_t)kSlots * kMaxCh * 8);
        char* tick = take((size_t)kSlots * 4);
        char* cnt = take(64 * 8);
        char* flg = take(256);
        if (pass == 0) {
            if (off > cap || !carve) return off;
            continue;
        }
        c.flo2 = (float*)lo2;
        c.partials = (double*)parts;
        c.scal = (double*)scal;
        c.tickets = (unsigned*)tick;
        c.counters = (unsigned long long*)cnt;
        c.flags = (unsigned*)flg;
        c.maxparts_ = maxparts;
        c.H = H_;
        c.W = W_;
        c.nch = nch_;
        c.nlev = nl;
        c.nlev_run = nl;
    }
    return off;
}
}  // namespace

extern "C" int hdi_inpaint_noalloc(int device, void* cuda_stream, const hdi_image* f, const hdi_mask* mask,
                                   hdi_image* u, double tol, hdi_stats* st) {
    auto t0 = std::chrono::steady_clock::now();
    if (device < 0 || device >= kNoAllocMaxDevices) return HDI_ERR_INVALID_ARG;
    if (!f || !mask || !u || !f->data || !mask->data || !u->data) return HDI_ERR_INVALID_ARG;
    if (f->location != HDI_DEVICE || mask->location != HDI_DEVICE || u->location != HDI_DEVICE)
        return HDI_ERR_INVALID_ARG;   // host buffers would need a staging allocation
    if (!(tol > 0.0 && tol < 1.0)) return HDI_ERR_INVALID_ARG;
    DeviceRestore restore;   // the caller's current device is put back on every return
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return HDI_ERR_CUDA;
    }
    void* scratch = g_noalloc_ptr[device].load(std::memory_order_acquire);
    if (!scratch) {
        // One-time set-up on this device, with the device current: the
        // array's name is only a host-side stand-in, so look up its address.
        // Two threads racing here look up the same address; both stores
        // write that value.
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return HDI_ERR_CUDA;
        }
        g_noalloc_ptr[device].store(p, std::memory_order_release);
        scratch = p;
    }
    Ctx c;
    c.device = device;
    c.stream = (cudaStream_t)cuda_stream;
    c.hscal = g_noalloc_hscal[device];
    int rc;
    if ((rc = c.check_image(f, "f", -1, 0, 0))) return rc;
    if ((rc = c.check_image(u, "u", f->height, f->width, f->channels))) return rc;
    if (u->dtype != f->dtype) return HDI_ERR_INVALID_ARG;
    if (noalloc_layout(c, (char*)scratch, kNoAllocBytes, f->height, f->width, f->channels) >
        kNoAllocBytes)
        return HDI_ERR_INVALID_ARG;   // image too large for the static scratch
    // The scratch keeps the previous call's contents: clear what must start at zero.
    cudaMemsetAsync(c.tickets, 0, (size_t)kSlots * 4, c.stream);
    cudaMemsetAsync(c.counters, 0, 64 * 8, c.stream);
    cudaMemsetAsync(c.scal, 0, (size_t)kSlots * kMaxCh * 8, c.stream);
    long long ones = 0;
    if ((rc = c.load_mask(mask, &ones))) return rc;
    if (ones == 0) return HDI_ERR_EMPTY_MASK;
    c.f_lo_zero = true;
    if ((rc = c.load_image(f, c.dfv[kF], c.flo2))) return rc;
    SolveSpec s;
    s.u[0] = c.dfv[kU0];
    s.u[1] = c.dfv[kU1];
    s.cur = 0;
    s.rhs = RHS_DATA;
    s.d = cview(c.dfv[kF]);
    s.tol = tol;
    s.max_iter = (int)c.p.max_vcycles;
    s.start = START_FMG;
    const int src = c.solve(s);
    if (src != HDI_OK && src != HDI_ERR_NOT_CONVERGED) return src;
    if ((rc = c.store_image(cview(s.u[s.cur]), u, false, c.flo2))) return rc;
    if (st) {
        st->status = src;
        st->iterations = s.iterations;
        st->vcycles = c.vcycles_run;
        st->local_iters = 0;
        st->rel_res = s.rel_max;
        st->mse = 0.0;
        st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return src;
}

// ------------------------------------------------------- engine C ABI ---

extern "C" {

int hdi_engine_create(hdi_engine** out, int device, void* stream, const char* config_json, double budget_gb) {
    if (!out) return HDI_ERR_INVALID_ARG;
    *out = nullptr;
    Params cfg;
    if (config_json && !parse_config(config_json, cfg)) return HDI_ERR_INVALID_ARG;
    if (!(budget_gb > 0.0)) return HDI_ERR_INVALID_ARG;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return HDI_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return HDI_ERR_CUDA;
    Engine* e = new Engine();
    e->device = device;
    e->stream = (cudaStream_t)stream;
    e->p = cfg;
    e->budget = budget_gb * 1e9;
    *out = reinterpret_cast<hdi_engine*>(e);
    return HDI_OK;
}

int hdi_engine_destroy(hdi_engine* h) {
    delete reinterpret_cast<Engine*>(h);
    return HDI_OK;
}

int hdi_engine_submit(hdi_engine* h, const hdi_image* f, const hdi_mask* mask, hdi_image* u, double tol, int64_t tag) {
    if (!h) return HDI_ERR_INVALID_ARG;
    Engine* e = reinterpret_cast<Engine*>(h);
    if (cudaSetDevice(e->device) != cudaSuccess) return HDI_ERR_CUDA;
    return e->submit(f, mask, u, tol, tag);
}

int hdi_engine_step(hdi_engine* h, int64_t* tags, hdi_stats* stats, int capacity, int* ndone) {
    if (!h || !ndone || capacity < 0) return HDI_ERR_INVALID_ARG;
    Engine* e = reinterpret_cast<Engine*>(h);
    if (cudaSetDevice(e->device) != cudaSuccess) return HDI_ERR_CUDA;
    // first the finished requests an earlier call could not report
    int k = 0;
    while (k < capacity && !e->pending_tags.empty()) {
        if (tags) tags[k] = e->pending_tags.front();
        if (stats) stats[k] = e->pending_stats.front();
        e->pending_tags.erase(e->pending_tags.begin());
        e->pending_stats.erase(e->pending_stats.begin());
        ++k;
    }
    int nd = 0;
    const int rc = e->step(tags ? tags + k : nullptr, stats ? stats + k : nullptr, capacity - k, &nd);
    *ndone = k + nd;
    return rc;
}

int hdi_engine_status(const hdi_engine* h, int64_t* in_flight, int64_t* bytes_in_use, int64_t* budget_bytes) {
    if (!h) return HDI_ERR_INVALID_ARG;
    const Engine* e = reinterpret_cast<const Engine*>(h);
    if (in_flight) *in_flight = (int64_t)e->reqs.size();
    if (bytes_in_use) *bytes_in_use = (int64_t)e->used;
    if (budget_bytes) *budget_bytes = (int64_t)e->budget;
    return HDI_OK;
}

int64_t hdi_engine_request_bytes(int32_t height, int32_t width, int32_t channels) {
    if (height < 1 || width < 1 || channels < 1 || channels > kMaxCh) return -1;
    return (int64_t)lean_bytes(height, width, channels);
}

int64_t hdi_engine_launch_count(const hdi_engine* h) {
    return h ? reinterpret_cast<const Engine*>(h)->launches : 0;
}

const char* hdi_engine_last_error(const hdi_engine* h) {
    return h ? reinterpret_cast<const Engine*>(h)->err.c_str() : "";
}

}  // extern "C"

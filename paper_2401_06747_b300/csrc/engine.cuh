// engine.cuh -- batched inpainting of images of uneven size (one launch per
// solver phase across all images in flight), with requests that join and
// leave at V-cycle boundaries.
//
// Every request is one image (any number of channels) with its own lean
// workspace (level arrays, mask pyramid, data and iterate pairs), allocated
// stream-ordered when it is admitted and released when it finishes. A step
// of the engine
//   - runs reduced full multigrid (Sec. 3.2) and the first refinement
//     residual for the requests admitted since the last step, and
//   - one V-cycle (Sec. 3.2, 3.3) plus the double-float refinement update
//     for every other request in flight,
// where every phase (data pyramid level, prolongation, ORAS sweep,
// restriction, refinement residual) is ONE kernel launch over a task table
// of (request, channel) entries: each entry carries its own geometry and
// buffers, and the CTAs of the launch are split among the entries by prefix
// sums (find_task). Norms are reduced per entry by a segmented deterministic
// grid reduction. After the step the host reads every request's residual
// norms once, finishes the converged ones (their u is written) and keeps the
// others; new requests may be submitted between steps.
//
// Each request converges at its own pace: it stops receiving V-cycles when
// its own per-channel relative residual meets its own tolerance. The
// arithmetic per request is that of hdi_inpaint (same kernels, same
// parameters; fine_pre = fine_post = 1).
#pragma once
#include <vector>
#include <algorithm>
#include <chrono>

struct EngReq {
    Ctx c;                      // lean context: the request's workspace
    hdi_image out{};            // caller's u
    int64_t tag = 0;
    double tol = 1e-6;
    int state = 0;              // -1: inputs loading; 0: admitted, waiting for FMG; 1: in refinement
    int rb = -1;                // readback slot of its input checks while loading
    int cur = 0;                // iterate pair holding u
    int iterations = 0;         // refinement steps
    int vcycles = 0;
    double b2[kMaxCh] = {};
    double rel_max = 1.0;
    const double* r2dev[kMaxCh] = {};   // device address of the last ||r||^2 per channel
    size_t bytes = 0;
    std::chrono::steady_clock::time_point t0;
};

enum EngKind {
    EK_DATA32 = 0, EK_RDATA, EK_PROLONG0, EK_PROLONG1, EK_PROLONG2, EK_RESTRICT, EK_ORAS0, EK_ORAS1,
    EK_RES_FROM32, EK_RES_UPDATE
};

struct EngLaunch {
    int kind;
    int ntasks;
    int ctas;
    size_t tasks_off, cta0_off;
    size_t base_off, out_off;       // segmented reduction (r) tables
    size_t base2_off, out2_off;     // second reduction (b) of the residual
    int level;                      // grid level of the tasks (strip launches; 0 for the residual)
    int want_b;
};

struct Engine {
    int device = 0;
    cudaStream_t stream = nullptr;
    Params p;
    std::string err;
    double budget = 120e9;
    size_t used = 0;            // bytes of the workspaces of the requests in flight
    std::vector<EngReq*> reqs;
    // step staging: task tables built on the host (pinned) and copied once
    char* hstage = nullptr;
    char* dstage = nullptr;
    size_t scap = 0, sused = 0;
    double* dnorm[2] = {nullptr, nullptr};   // per-step ||r||^2, ||b||^2 of the residual tasks
    double* hnorm = nullptr;
    int ncap = 0;                // capacity of dnorm (doubles) and hnorm
    int parity = 0;
    double* partials = nullptr;  // segmented reduction partials (one per CTA of a launch)
    int pcap = 0;
    unsigned* tickets = nullptr; // [2]
    std::vector<EngLaunch> plan;
    std::vector<int64_t> pending_tags;     // finished requests not yet reported (step capacity exceeded)
    std::vector<hdi_stats> pending_stats;
    int64_t launches = 0;
    int steps = 0;

    int fail(int code, const char* fmt, ...) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        err = buf;
        return code;
    }

    // ---------------------------------------------------------- staging ---
    size_t put(const void* src, size_t n) {
        sused = (sused + 15) & ~(size_t)15;
        const size_t off = sused;
        if (off + n <= scap) memcpy(hstage + off, src, n);
        sused = off + n;
        return off;
    }
    template <typename T>
    size_t put_vec(const std::vector<T>& v) { return put(v.data(), v.size() * sizeof(T)); }

    int ensure_staging(size_t need) {
        if (need <= scap) return HDI_OK;
        size_t cap = std::max(need, (size_t)1 << 20);
        cap = std::max(cap, 2 * scap);
        if (hstage) cudaFreeHost(hstage);
        if (dstage) cudaFree(dstage);
        hstage = nullptr;
        dstage = nullptr;
        scap = 0;
        if (cudaMallocHost(&hstage, cap) != cudaSuccess || cudaMalloc(&dstage, cap) != cudaSuccess) {
            cudaGetLastError();
            return fail(HDI_ERR_OUT_OF_MEMORY, "engine: staging of %zu bytes failed", cap);
        }
        scap = cap;
        return HDI_OK;
    }
    // Grows the per-step norm buffers; the previous step's norms (which the
    // next V-cycle's first sweep reads) move with them.
    int ensure_norms(int n) {
        if (n <= ncap) return HDI_OK;
        const int cap = std::max(n, std::max(256, 2 * ncap));
        double* nd[2] = {nullptr, nullptr};
        double* nh = nullptr;
        if (cudaMalloc(&nd[0], (size_t)cap * 8) != cudaSuccess || cudaMalloc(&nd[1], (size_t)cap * 8) != cudaSuccess ||
            cudaMallocHost(&nh, (size_t)cap * 8) != cudaSuccess) {
            cudaGetLastError();
            for (auto d : nd)
                if (d) cudaFree(d);
            return fail(HDI_ERR_OUT_OF_MEMORY, "engine: norm buffers failed");
        }
        for (int k = 0; k < 2; ++k)
            if (dnorm[k] && ncap) cudaMemcpyAsync(nd[k], dnorm[k], (size_t)ncap * 8, cudaMemcpyDeviceToDevice, stream);
        for (EngReq* r : reqs)
            for (int ch = 0; ch < r->c.nch; ++ch)
                for (int k = 0; k < 2; ++k)
                    if (dnorm[k] && r->r2dev[ch] >= dnorm[k] && r->r2dev[ch] < dnorm[k] + ncap)
                        r->r2dev[ch] = nd[k] + (r->r2dev[ch] - dnorm[k]);
        cudaStreamSynchronize(stream);
        for (auto& d : dnorm)
            if (d) cudaFree(d);
        if (hnorm) cudaFreeHost(hnorm);
        dnorm[0] = nd[0];
        dnorm[1] = nd[1];
        hnorm = nh;
        ncap = cap;
        return HDI_OK;
    }
    int ensure_partials(int n) {
        if (n <= pcap) return HDI_OK;
        const int cap = std::max(n, 2 * pcap);
        if (partials) cudaFree(partials);
        partials = nullptr;
        pcap = 0;
        if (cudaMalloc(&partials, (size_t)cap * 8) != cudaSuccess) {
            cudaGetLastError();
            return fail(HDI_ERR_OUT_OF_MEMORY, "engine: reduction partials failed");
        }
        pcap = cap;
        return HDI_OK;
    }

    // ------------------------------------------------------ geometry ---
    static MaskView plane(const Ctx& c, int l) {
        MaskView m;
        m.bits = c.lev[l].bits;
        m.H = c.lev[l].H;
        m.W = c.lev[l].W;
        m.wpitch = c.lev[l].wp;
        m.chmask = nullptr;
        m.cstride = 0;
        return m;
    }
    static LevelArr larr(const Ctx& c, int l) { return c.arr(l); }

    // Records a launch whose task table `tasks` and per-task CTA counts
    // `ctas` are given; norm outputs (if any) in `outs` (one per task).
    template <typename T>
    void record(int kind, const std::vector<T>& tasks, const std::vector<int>& ctas, const std::vector<double*>* outs,
                const std::vector<double*>* outs2 = nullptr, int want_b = 0, int level = 0) {
        if (tasks.empty()) return;
        EngLaunch L{};
        L.kind = kind;
        L.ntasks = (int)tasks.size();
        std::vector<int> cta0(tasks.size() + 1, 0);
        for (size_t i = 0; i < tasks.size(); ++i) cta0[i + 1] = cta0[i] + ctas[i];
        L.ctas = cta0.back();
        L.tasks_off = put_vec(tasks);
        L.cta0_off = put_vec(cta0);
        if (outs) {
            // partial offsets equal the CTA offsets: one partial per CTA
            L.base_off = L.cta0_off;
            L.out_off = put_vec(*outs);
        }
        if (outs2) {
            // the second reduction's partials follow the first one's (both
            // are committed by every CTA of the launch, so they cannot share
            // slots: the first sum would read partials of the second)
            std::vector<int> base2(cta0);
            for (int& v : base2) v += L.ctas;
            L.base2_off = put_vec(base2);
            L.out2_off = put_vec(*outs2);
        }
        L.want_b = want_b;
        L.level = level;
        plan.push_back(L);
    }

    // ORAS sweep tasks (as Ctx::oras) over the requests `S` at level l; the
    // requests whose coarsest level is l get the coarsest-solve parameters.
    void rec_oras(int l, bool zero, const std::vector<EngReq*>& S, bool post) {
        std::vector<OrasTask> tasks;
        std::vector<int> ctas;
        for (EngReq* r : S) {
            Ctx& c = r->c;
            const Level& L = c.lev[l];
            const bool coarsest = (l == c.nlev_run - 1);
            const double eta = (l > 0 && p.coarse_level_eta > 0) ? p.coarse_level_eta : p.oras_eta;
            for (int ch = 0; ch < c.nch; ++ch) {
                OrasTask t{};
                OrasArgs& a = t.a;
                a.m = plane(c, l);
                a.H = L.H;
                a.W = L.W;
                a.pitch = L.P;
                a.cstride = 0;
                a.nch = 1;
                a.nbx = L.nbx;
                a.nby = L.nby;
                a.stride = 32 - kOv;
                a.ov = kOv;
                a.theta = (float)p.oras_theta;
                a.maxit = coarsest ? (int)p.coarse_max_local : (l > 0 ? (int)p.coarse_level_max : (int)p.oras_max_local);
                a.thresh_scale = coarsest ? p.coarse_eta : eta / (double)(L.nbx * L.nby);
                const long long o = (long long)ch * L.cs;
                // pre-sweep (zero): b -> xa; post-sweep / FMG: xb -> xa
                a.xin = zero ? nullptr : L.xb + o;
                a.xout = L.xa + o;
                a.b = L.b + o;
                a.rnorm2 = (l == 0 && !post && zero) ? r->r2dev[ch] : c.scal + l * kMaxCh + ch;
                a.iters = (l == 0) ? c.counters + kCntLocal : nullptr;
                t.full = (L.W >= 32 && L.H >= 32) ? 1 : 0;
                tasks.push_back(t);
                ctas.push_back(L.nbx * L.nby);
            }
        }
        record(zero ? EK_ORAS0 : EK_ORAS1, tasks, ctas, nullptr);
    }

    // Strip tasks (restriction l -> l+1, prolongation l+1 -> l).
    void rec_strip(int kind, int l, const std::vector<EngReq*>& S) {
        std::vector<StripTask> tasks;
        std::vector<int> ctas;
        std::vector<double*> outs;
        for (EngReq* r : S) {
            Ctx& c = r->c;
            const Level& L = c.lev[l];
            const bool has_c = (kind == EK_RESTRICT || kind == EK_PROLONG0 || kind == EK_PROLONG1);
            for (int ch = 0; ch < c.nch; ++ch) {
                StripTask t{};
                t.F = larr(c, l);
                t.fm = plane(c, l);
                const long long o = (long long)ch * L.cs;
                if (has_c) {
                    const Level& C = c.lev[l + 1];
                    t.C = larr(c, l + 1);
                    t.cm = plane(c, l + 1);
                    const long long oc = (long long)ch * C.cs;
                    if (kind == EK_RESTRICT) t.cb = C.b + oc;
                    else t.e = C.xa + oc;
                } else {
                    t.C = t.F;   // MODE 2 reads no coarse values
                    t.cm = t.fm;
                }
                t.x = L.xa + o;
                t.b = L.b + o;
                t.xout = L.xb + o;
                t.rows = c.qrows(L.H, L.W, 1);
                const dim3 g = quad_grid(L.H, L.W, 1, t.rows);
                t.gx = g.x;
                t.gy = g.y;
                tasks.push_back(t);
                ctas.push_back(t.gx * t.gy);
                // restriction: ||b_{l+1}||^2 into slot l + 1; prolongation: ||b - A x||^2 into slot l
                outs.push_back(c.scal + (kind == EK_RESTRICT ? l + 1 : l) * kMaxCh + ch);
            }
        }
        record(kind, tasks, ctas, &outs, nullptr, 0, l);
    }

    // One V-cycle (as Ctx::vcycle with one pre- and one post-sweep) over S at level l.
    void rec_vcycle(int l, const std::vector<EngReq*>& S) {
        if (S.empty()) return;
        rec_oras(l, true, S, false);
        std::vector<EngReq*> N;
        for (EngReq* r : S)
            if (l < r->c.nlev_run - 1) N.push_back(r);
        if (N.empty()) return;
        rec_strip(EK_RESTRICT, l, N);
        rec_vcycle(l + 1, N);
        rec_strip(EK_PROLONG0, l, N);
        rec_oras(l, false, N, true);
    }

    // Reduced full multigrid (as Ctx::fmg) over the new requests A.
    void rec_fmg(const std::vector<EngReq*>& A) {
        int maxl = 0;
        for (EngReq* r : A) maxl = std::max(maxl, r->c.nlev_run);
        {   // level-0 right-hand side C f in FP32
            std::vector<PixTask> tasks;
            std::vector<int> ctas;
            for (EngReq* r : A) {
                Ctx& c = r->c;
                const Level& L = c.lev[0];
                for (int ch = 0; ch < c.nch; ++ch) {
                    PixTask t{};
                    t.F = larr(c, 0);
                    t.fm = plane(c, 0);
                    const long long o = (long long)ch * L.cs;
                    t.d = DFc{c.dfv[kF].hi + o, c.dfv[kF].lo + o};
                    t.out = L.b + o;
                    t.gx = (L.W + 127) / 128;
                    tasks.push_back(t);
                    ctas.push_back(t.gx * L.H);
                }
            }
            record(EK_DATA32, tasks, ctas, nullptr);
        }
        for (int l = 1; l < maxl; ++l) {   // data pyramid
            std::vector<PixTask> tasks;
            std::vector<int> ctas;
            for (EngReq* r : A) {
                Ctx& c = r->c;
                if (l >= c.nlev_run) continue;
                const Level& F = c.lev[l - 1];
                const Level& C = c.lev[l];
                for (int ch = 0; ch < c.nch; ++ch) {
                    PixTask t{};
                    t.F = larr(c, l - 1);
                    t.C = larr(c, l);
                    t.fm = plane(c, l - 1);
                    t.fb = F.b + (long long)ch * F.cs;
                    t.out = C.b + (long long)ch * C.cs;
                    t.gx = (C.W + 31) / 32;
                    tasks.push_back(t);
                    ctas.push_back(t.gx * ((C.H + 7) / 8));
                }
            }
            record(EK_RDATA, tasks, ctas, nullptr);
        }
        for (int l = maxl - 1; l >= 0; --l) {
            std::vector<EngReq*> start, up, all;
            for (EngReq* r : A) {
                if (l == r->c.nlev_run - 1) start.push_back(r);
                else if (l < r->c.nlev_run - 1) up.push_back(r);
            }
            rec_strip(EK_PROLONG2, l, start);   // coarsest: x = b on known pixels, 0 elsewhere
            rec_strip(EK_PROLONG1, l, up);      // finer levels: interpolate the coarser solution
            all = start;
            all.insert(all.end(), up.begin(), up.end());
            rec_oras(l, false, all, false);
        }
    }

    // Refinement residual over S (INIT_FROM32 after FMG, INIT_UPDATE after a
    // V-cycle); the norms go to dnorm[parity] at `base` (two per channel).
    void rec_residual(int init, const std::vector<EngReq*>& S, int base) {
        std::vector<ResTask> tasks;
        std::vector<int> ctas;
        std::vector<double*> outs_r, outs_b;
        int k = base;
        for (EngReq* r : S) {
            Ctx& c = r->c;
            const Level& L = c.lev[0];
            const int cur = r->cur, nxt = (init == INIT_FROM32) ? r->cur : 1 - r->cur;
            const DF U[2] = {c.dfv[kU0], c.dfv[kU1]};
            for (int ch = 0; ch < c.nch; ++ch) {
                ResTask t{};
                ResArgs& a = t.a;
                const long long o = (long long)ch * L.cs;
                a.F = larr(c, 0);
                a.m = plane(c, 0);
                a.uin = DFc{U[cur].hi + o, U[cur].lo + o};
                a.uout = DF{U[nxt].hi + o, U[nxt].lo + o};
                a.x32 = L.xa + o;
                a.d = DFc{c.dfv[kF].hi + o, c.dfv[kF].lo + o};
                a.y = DFc{nullptr, nullptr};
                a.r32 = L.b + o;
                a.rows = c.qrows(L.H, L.W, 1);
                a.want_b = init == INIT_FROM32 ? 1 : 0;
                a.d_lo_zero = c.f_lo_zero ? 1 : 0;
                const dim3 g = quad_grid(L.H, L.W, 1, a.rows);
                t.gx = g.x;
                t.gy = g.y;
                tasks.push_back(t);
                ctas.push_back(g.x * g.y);
                outs_r.push_back(dnorm[parity] + 2 * k);
                outs_b.push_back(dnorm[parity] + 2 * k + 1);
                r->r2dev[ch] = dnorm[parity] + 2 * k;
                ++k;
            }
        }
        record(init == INIT_FROM32 ? EK_RES_FROM32 : EK_RES_UPDATE, tasks, ctas, &outs_r, &outs_b,
               init == INIT_FROM32 ? 1 : 0);
    }

    // -------------------------------------------------------- launching ---
    SegReduce seg(const EngLaunch& L, size_t base_off, size_t out_off, int ticket) const {
        SegReduce R;
        R.partials = partials;
        R.ticket = tickets + ticket;
        R.base = (const int*)(dstage + base_off);
        R.out = (double* const*)(dstage + out_off);
        R.nseg = L.ntasks;
        R.total_ctas = L.ctas;
        return R;
    }

    int execute() {
        const bool pd = p.pdl >= 0.5;
        // dynamic shared memory of the level-0 kernels that stage their row
        // loads (`bit` of stage_loads, as in Ctx::stage_bytes)
        auto stg = [&](const EngLaunch& L, int bit, size_t bytes) {
            return (L.level == 0 && ((int)p.stage_loads & bit)) ? bytes : (size_t)0;
        };
        for (const EngLaunch& L : plan) {
            const int* cta0 = (const int*)(dstage + L.cta0_off);
            const void* tk = dstage + L.tasks_off;
            const dim3 grid(L.ctas);
            cudaError_t e = cudaSuccess;
            switch (L.kind) {
            case EK_DATA32:
                k_data_to_f32_b<<<grid, 128, 0, stream>>>((const PixTask*)tk, cta0, L.ntasks);
                break;
            case EK_RDATA:
                k_restrict_data_b<<<grid, dim3(32, 8), 0, stream>>>((const PixTask*)tk, cta0, L.ntasks);
                break;
            case EK_PROLONG0:
                e = launch_k(pd, k_prolong_b<0>, grid, dim3(128), stream, (const StripTask*)tk, cta0, L.ntasks,
                             seg(L, L.base_off, L.out_off, 0));
                break;
            case EK_PROLONG1:
                e = launch_k(pd, k_prolong_b<1>, grid, dim3(128), stream, (const StripTask*)tk, cta0, L.ntasks,
                             seg(L, L.base_off, L.out_off, 0));
                break;
            case EK_PROLONG2:
                e = launch_k(pd, k_prolong_b<2>, grid, dim3(128), stream, (const StripTask*)tk, cta0, L.ntasks,
                             seg(L, L.base_off, L.out_off, 0));
                break;
            case EK_RESTRICT:
                e = launch_ks(pd, stg(L, 2, RStage::bytes), k_restrict_residual_b, grid, dim3(128), stream,
                              (const StripTask*)tk, cta0, L.ntasks, seg(L, L.base_off, L.out_off, 0));
                break;
            case EK_ORAS0:
                e = launch_k(pd, k_oras_wb<true>, grid, dim3(32), stream, (const OrasTask*)tk, cta0, L.ntasks);
                break;
            case EK_ORAS1:
                e = launch_k(pd, k_oras_wb<false>, grid, dim3(32), stream, (const OrasTask*)tk, cta0, L.ntasks);
                break;
            case EK_RES_FROM32:
                e = launch_ks(pd, stg(L, 1, ResStage<RHS_DATA, INIT_FROM32, false>::bytes),
                              k_residual_df_b<RHS_DATA, INIT_FROM32>, grid, dim3(128), stream, (const ResTask*)tk, cta0,
                              L.ntasks, seg(L, L.base_off, L.out_off, 0), seg(L, L.base2_off, L.out2_off, 1), L.want_b);
                break;
            case EK_RES_UPDATE:
                e = launch_ks(pd, stg(L, 1, ResStage<RHS_DATA, INIT_UPDATE, false>::bytes),
                              k_residual_df_b<RHS_DATA, INIT_UPDATE>, grid, dim3(128), stream, (const ResTask*)tk, cta0,
                              L.ntasks, seg(L, L.base_off, L.out_off, 0), seg(L, L.base2_off, L.out2_off, 1), L.want_b);
                break;
            }
            ++launches;
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess) return fail(HDI_ERR_CUDA, "engine launch: %s", cudaGetErrorString(e));
        }
        return HDI_OK;
    }

    // ------------------------------------------------------------ API ---
    static constexpr int kReadbackSlots = 4096;   // requests whose inputs may load at once
    LoadReadback* hrb = nullptr;                  // pinned readbacks of their input checks
    int nloading = 0;
    int submit_async(const hdi_image* f, const hdi_mask* m, hdi_image* u, double tol, int64_t tag);
    int finalize_loads(std::vector<std::pair<int64_t, int>>* failed);
    int submit(const hdi_image* f, const hdi_mask* m, hdi_image* u, double tol, int64_t tag);
    int step(int64_t* tags, hdi_stats* stats, int cap, int* ndone);
    int finish(EngReq* r, unsigned long long* li);
    unsigned long long* hfin = nullptr;   // pinned local-iteration counters of finished requests
    int hfcap = 0;
    void release(EngReq* r);
    ~Engine();
};

// Workspace of one request (the lean layout of Ctx::setup_lean): first the
// parts that start at zero -- the mask bits of every level, the counters,
// the norms and the flags -- in one contiguous block (one memset), then the
// level arrays and the double-float vectors.
struct LeanPlan {
    int nl = 0;
    int h[kMaxLevels], w[kMaxLevels];
    size_t zero_bytes = 0, bytes = 0;
};
static inline size_t lean_align(size_t b) { return (b + 255) & ~(size_t)255; }
static LeanPlan lean_plan(int H_, int W_, int nch_) {
    LeanPlan L;
    int h = H_, w = W_;
    for (;;) {
        L.h[L.nl] = h;
        L.w[L.nl] = w;
        ++L.nl;
        if (std::max(h, w) <= 32 || L.nl >= kMaxLevels) break;
        h = (h + 1) / 2;
        w = (w + 1) / 2;
    }
    size_t z = 0;
    for (int l = 0; l < L.nl; ++l) z += lean_align((size_t)L.h[l] * ((L.w[l] + 31) / 32 + 1) * 4);
    z += lean_align(64 * 8) + lean_align((size_t)kSlots * kMaxCh * 8) + lean_align(256 + kMaxCh * 4);
    L.zero_bytes = z;
    size_t b = z;
    for (int l = 0; l < L.nl; ++l) b += 3 * lean_align((size_t)nch_ * L.h[l] * round_up(L.w[l], 32) * 4);
    const size_t n32 = (size_t)nch_ * H_ * round_up(W_, 32);
    b += 3 * lean_align(n32 * 8) + lean_align(n32 * 4);
    L.bytes = b;
    return L;
}
static size_t lean_bytes(int H_, int W_, int nch_) { return lean_plan(H_, W_, nch_).bytes; }

// Lean set-up of a request context: the buffers of one inpainting solve
// only, allocated stream-ordered (cudaMallocAsync) on `s`.
int Ctx::setup_lean(int H_, int W_, int nch_, cudaStream_t s) {
    if (nch_ < 1 || nch_ > kMaxCh) return fail(HDI_ERR_INVALID_ARG, "request: 1 to %d channels", kMaxCh);
    const LeanPlan plan = lean_plan(H_, W_, nch_);
    ws.astream = s;
    ws.async = true;
    {
        cudaError_t e = cudaMallocAsync(&ws.base, plan.bytes, s);
        if (e != cudaSuccess) {
            ws.base = nullptr;
            cudaGetLastError();
            return fail(HDI_ERR_OUT_OF_MEMORY, "request workspace: cudaMallocAsync(%zu) failed", plan.bytes);
        }
        ws.cap = plan.bytes;
        ws.used = 0;
    }
    const int nl = plan.nl;
    for (int l = 0; l < nl; ++l) {
        Level& L = lev[l];
        L.H = plan.h[l];
        L.W = plan.w[l];
        L.P = round_up(L.W, 32);
        L.wp = (L.W + 31) / 32 + 1;
        L.cs = (long long)L.H * L.P;
        L.bits = (uint32_t*)ws.take((size_t)L.H * L.wp * 4);
        L.nbx = tile_count(L.W, 32, kOv);
        L.nby = tile_count(L.H, 32, kOv);
    }
    counters = (unsigned long long*)ws.take(64 * 8);
    scal = (double*)ws.take((size_t)kSlots * kMaxCh * 8);
    flags = (unsigned*)ws.take(256 + kMaxCh * 4);
    for (int l = 0; l < nl; ++l) {
        Level& L = lev[l];
        L.xa = (float*)ws.take((size_t)nch_ * L.cs * 4);
        L.xb = (float*)ws.take((size_t)nch_ * L.cs * 4);
        L.b = (float*)ws.take((size_t)nch_ * L.cs * 4);
    }
    const size_t n32 = (size_t)nch_ * H_ * round_up(W_, 32);
    const int dfs[3] = {kF, kU0, kU1};
    for (int i = 0; i < 3; ++i) {
        dfv[dfs[i]].hi = (float*)ws.take(n32 * 8);
        dfv[dfs[i]].lo = dfv[dfs[i]].hi + n32;
    }
    flo2 = (float*)ws.take(n32 * 4);
    if (ws.used > ws.cap) return fail(HDI_ERR_CUDA, "internal: request workspace carving exceeds its size");
    H = H_;
    W = W_;
    nch = nch_;
    nlev = nl;
    nlev_run = nl;
    nmask = 1;
    stream = s;
    cudaMemsetAsync(ws.base, 0, plan.zero_bytes, s);   // mask bits, counters, norms, flags
    return cuda_check(cudaGetLastError(), "request workspace");
}

void Engine::release(EngReq* r) {
    r->c.ws.release();
    r->c.stage.release();
    used -= std::min(used, r->bytes);
    delete r;
}

void engine_delete(Engine* e) { delete e; }
size_t engine_used_bytes(const Engine* e) { return e ? e->used : 0; }

Engine::~Engine() {
    cudaSetDevice(device);
    cudaStreamSynchronize(stream);
    for (EngReq* r : reqs) release(r);
    reqs.clear();
    if (hstage) cudaFreeHost(hstage);
    if (dstage) cudaFree(dstage);
    for (auto d : dnorm)
        if (d) cudaFree(d);
    if (hnorm) cudaFreeHost(hnorm);
    if (partials) cudaFree(partials);
    if (tickets) cudaFree(tickets);
    if (hfin) cudaFreeHost(hfin);
    if (hrb) cudaFreeHost(hrb);
}

// Admits one request if its workspace fits the budget: allocates it and
// enqueues the upload and checks of mask and image without waiting; the
// checks are evaluated by finalize_loads (one wait for all requests loaded
// since the last call). FMG runs at the first step after that.
int Engine::submit_async(const hdi_image* f, const hdi_mask* m, hdi_image* u, double tol, int64_t tag) {
    if (!(tol > 0.0 && tol < 1.0)) return fail(HDI_ERR_INVALID_ARG, "tol must lie in (0, 1)");
    if (!f || !m || !u) return fail(HDI_ERR_INVALID_ARG, "null request argument");
    if (nloading >= kReadbackSlots) return fail(HDI_ERR_OUT_OF_MEMORY, "too many requests loading at once");
    if (!hrb) {
        if (cudaMallocHost(&hrb, sizeof(LoadReadback) * kReadbackSlots) != cudaSuccess) {
            cudaGetLastError();
            hrb = nullptr;
            return fail(HDI_ERR_OUT_OF_MEMORY, "engine: pinned readback slots");
        }
    }
    EngReq* r = new EngReq();
    Ctx& c = r->c;
    c.device = device;
    c.stream = stream;
    c.p = p;
    int rc;
    if ((rc = c.check_image(f, "f", -1, 0, 0)) || (rc = c.check_image(u, "u", f->height, f->width, f->channels))) {
        err = c.err;
        delete r;
        return rc;
    }
    if (u->dtype != f->dtype) {
        delete r;
        return fail(HDI_ERR_INVALID_ARG, "u: dtype differs from f");
    }
    if (m->height != f->height || m->width != f->width) {
        delete r;
        return fail(HDI_ERR_INVALID_ARG, "mask: shape does not match the image");
    }
    r->bytes = lean_bytes(f->height, f->width, f->channels);
    if ((double)(used + r->bytes) > budget) {
        const size_t need = r->bytes;
        delete r;
        return fail(HDI_ERR_OUT_OF_MEMORY, "request of %.3f GB does not fit: %.3f of %.3f GB in use", need / 1e9,
                    used / 1e9, budget / 1e9);
    }
    if ((rc = c.setup_lean(f->height, f->width, f->channels, stream))) {
        err = c.err;
        delete r;
        return rc;
    }
    used += r->bytes;
    long long ones = 0;
    c.f_lo_zero = true;
    rc = c.load_mask(m, &ones, 0, true, false);
    if (!rc) rc = c.load_image(f, c.dfv[kF], c.flo2, 0, false);
    if (rc) {
        err = c.err;
        release(r);
        return rc;
    }
    r->rb = nloading++;
    c.enqueue_load_readback(&hrb[r->rb]);
    r->out = *u;
    r->tag = tag;
    r->tol = tol;
    r->state = -1;
    r->t0 = std::chrono::steady_clock::now();
    reqs.push_back(r);
    return HDI_OK;
}

// Waits once for the loads enqueued by submit_async and evaluates their
// checks; requests that fail them leave (tag and status into `failed`).
int Engine::finalize_loads(std::vector<std::pair<int64_t, int>>* failed) {
    if (nloading == 0) return HDI_OK;
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HDI_ERR_CUDA, "engine input upload: %s", cudaGetErrorString(e));
    std::vector<EngReq*> keep;
    for (EngReq* r : reqs) {
        if (r->state != -1) {
            keep.push_back(r);
            continue;
        }
        long long ones = 0;
        int rc = r->c.load_checks(hrb[r->rb], &ones);
        if (!rc && ones == 0) rc = r->c.fail(HDI_ERR_EMPTY_MASK, "empty mask: A is singular");
        r->rb = -1;
        if (rc) {
            err = r->c.err;
            if (failed) failed->push_back({r->tag, rc});
            release(r);
            continue;
        }
        r->state = 0;
        keep.push_back(r);
    }
    reqs = keep;
    nloading = 0;
    return HDI_OK;
}

// One request with its checks done before returning (a failing one returns
// their status and is not kept).
int Engine::submit(const hdi_image* f, const hdi_mask* m, hdi_image* u, double tol, int64_t tag) {
    int rc = submit_async(f, m, u, tol, tag);
    if (rc) return rc;
    std::vector<std::pair<int64_t, int>> failed;
    if ((rc = finalize_loads(&failed))) return rc;
    return failed.empty() ? HDI_OK : failed.front().second;
}

// Enqueues the write of u and the read of the local-iteration counter
// (into *li, pinned) of a finished request; the caller waits once for all.
int Engine::finish(EngReq* r, unsigned long long* li) {
    int rc = r->c.store_image(cview(r->c.dfv[r->cur ? kU1 : kU0]), &r->out, false, r->c.flo2, 0, false);
    cudaMemcpyAsync(li, r->c.counters + kCntLocal, 8, cudaMemcpyDeviceToHost, stream);
    if (rc) err = r->c.err;
    return rc;
}

// One engine step (see the file comment). Finished requests are reported
// in tags/stats (at most `cap`; the rest stay finished-but-unreported
// until the next call, which reports them first).
int Engine::step(int64_t* tags, hdi_stats* stats, int cap, int* ndone) {
    *ndone = 0;
    int rc;
    if (nloading && (rc = finalize_loads(nullptr))) return rc;   // loads left by submit_async
    if (reqs.empty()) return HDI_OK;
    std::vector<EngReq*> A, V;
    for (EngReq* r : reqs) (r->state == 0 ? A : V).push_back(r);
    int nt_a = 0, nt_v = 0;
    for (EngReq* r : A) nt_a += r->c.nch;
    for (EngReq* r : V) nt_v += r->c.nch;
    if ((rc = ensure_norms(2 * (nt_a + nt_v)))) return rc;
    parity ^= 1;
    const auto tp0 = std::chrono::steady_clock::now();
    // plan (twice if the staging buffer must grow)
    for (int attempt = 0; attempt < 2; ++attempt) {
        plan.clear();
        sused = 0;
        if (!A.empty()) {
            rec_fmg(A);
            rec_residual(INIT_FROM32, A, 0);
        }
        if (!V.empty()) {
            rec_vcycle(0, V);
            rec_residual(INIT_UPDATE, V, nt_a);
        }
        if (sused <= scap) break;
        if ((rc = ensure_staging(sused))) return rc;
    }
    int maxparts = 0;   // one partial per CTA and reduction
    for (const EngLaunch& L : plan) maxparts = std::max(maxparts, (L.want_b ? 2 : 1) * L.ctas);
    if ((rc = ensure_partials(maxparts))) return rc;
    if (!tickets) {
        if (cudaMalloc(&tickets, 64) != cudaSuccess) return fail(HDI_ERR_OUT_OF_MEMORY, "engine: tickets");
        cudaMemsetAsync(tickets, 0, 64, stream);
    }
    const auto tp1 = std::chrono::steady_clock::now();
    cudaMemcpyAsync(dstage, hstage, sused, cudaMemcpyHostToDevice, stream);
    if ((rc = execute())) return rc;
    const int nn = 2 * (nt_a + nt_v);
    cudaMemcpyAsync(hnorm, dnorm[parity], (size_t)nn * 8, cudaMemcpyDeviceToHost, stream);
    const auto tp2 = std::chrono::steady_clock::now();
    cudaError_t e = cudaStreamSynchronize(stream);
    if (p.trace >= 0.5) {
        const auto tp3 = std::chrono::steady_clock::now();
        auto us = [](auto a, auto b) { return std::chrono::duration<double, std::micro>(b - a).count(); };
        fprintf(stderr, "[hdi engine] step %d: %zu new, %zu in refinement, %zu launches, %zu table bytes; "
                        "host plan %.0f us, enqueue %.0f us, wait %.0f us\n",
                steps, A.size(), V.size(), plan.size(), sused, us(tp0, tp1), us(tp1, tp2), us(tp2, tp3));
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HDI_ERR_CUDA, "engine step: %s", cudaGetErrorString(e));
    ++steps;
    // classify
    int k = 0;
    std::vector<EngReq*> keep;
    std::vector<std::pair<EngReq*, int>> fin;   // finished requests and their status
    auto judge = [&](EngReq* r, bool first) {
        double worst = 0.0;
        bool bad = false;
        for (int ch = 0; ch < r->c.nch; ++ch, ++k) {
            const double r2 = hnorm[2 * k];
            if (first) r->b2[ch] = hnorm[2 * k + 1];
            if (!std::isfinite(r2)) bad = true;
            const double b2 = r->b2[ch];
            const double rel = b2 > 0 ? std::sqrt(r2 / b2) : (r2 > 0 ? INFINITY : 0.0);
            worst = std::max(worst, rel);
        }
        if (!first) {
            r->cur = 1 - r->cur;
            ++r->iterations;
            ++r->vcycles;
        }
        r->state = 1;
        r->rel_max = worst;
        int status = -100;   // not finished
        if (bad) status = HDI_ERR_NONFINITE;
        else if (worst <= r->tol) status = HDI_OK;
        else if (r->iterations >= (int)p.max_vcycles) status = HDI_ERR_NOT_CONVERGED;
        if (status == -100) keep.push_back(r);
        else fin.push_back({r, status});
    };
    for (EngReq* r : A) judge(r, true);
    for (EngReq* r : V) judge(r, false);
    reqs = keep;
    if (fin.empty()) return HDI_OK;
    // results of the finished requests: all writes enqueued, one wait
    if ((int)fin.size() > hfcap) {
        if (hfin) cudaFreeHost(hfin);
        hfin = nullptr;
        hfcap = 0;
        if (cudaMallocHost(&hfin, fin.size() * 8) != cudaSuccess) {
            cudaGetLastError();
            return fail(HDI_ERR_OUT_OF_MEMORY, "engine: pinned counters");
        }
        hfcap = (int)fin.size();
    }
    std::vector<int> frc(fin.size());
    for (size_t i = 0; i < fin.size(); ++i) frc[i] = finish(fin[i].first, hfin + i);
    e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HDI_ERR_CUDA, "engine results: %s", cudaGetErrorString(e));
    const auto now = std::chrono::steady_clock::now();
    for (size_t i = 0; i < fin.size(); ++i) {
        EngReq* r = fin[i].first;
        hdi_stats st;
        memset(&st, 0, sizeof st);
        st.status = frc[i] ? frc[i] : fin[i].second;
        st.iterations = r->iterations;
        st.vcycles = r->vcycles;
        st.local_iters = (int64_t)hfin[i];
        st.rel_res = r->rel_max;
        st.seconds = std::chrono::duration<double>(now - r->t0).count();
        if (*ndone < cap) {
            if (tags) tags[*ndone] = r->tag;
            if (stats) stats[*ndone] = st;
            ++*ndone;
        } else {
            pending_tags.push_back(r->tag);
            pending_stats.push_back(st);
        }
        release(r);
    }
    return HDI_OK;
}
